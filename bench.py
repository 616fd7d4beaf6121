"""Benchmark: wdot + analytic Jacobian throughput of the QSS hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload hydrocarbon|tiny|large] [--ncells C]

One step = one pass of the hot path (state unpack, thermo, rates, falloff,
QSS solve, production rates, temperature equation, analytic Jacobian through
the QSS chain rule) over one batch of cells of the workload, launched through
the C ABI (qss_jacobian).  The default workload is the hydrocarbon-scale
synthetic mechanism (35 transported + 18 QSS species, 268 reactions) at 2^20
cells.  Inputs and outputs exceed the 126 MB L2 (310 MB in, 11 GB out), so no
L2 flush is needed between steps.

Prints one JSON line (rank 0).  Under torchrun every rank processes its own
batch (weak scaling, no collective on the data path); the time is the max over
ranks.  ``--impl reference`` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "wdot+Jacobian cells/s"
UNIT = "cells/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="hydrocarbon", choices=["tiny", "hydrocarbon", "large"])
    p.add_argument("--ncells", type=int, default=0)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-implicit", action="store_true")
    p.add_argument("--integrate", action="store_true",
                   help="also time qss_integrate (backward Euler vs BDF2 substeps; about 30 s)")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--implicit-ncells", type=int, default=0)
    p.add_argument("--jac-parts", type=int, default=-1,
                   help="Jacobian as a prefix + this many column-group kernels (default: per workload)")
    p.add_argument("--jac-format", default="dense", choices=["dense", "csr"],
                   help="store every Jacobian entry or only the structural nonzeros")
    p.add_argument("--serve-seconds", type=float, default=8.0)
    return p.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                f = [x.strip() for x in out.split(",")]
                if len(f) >= 7:
                    self.samples.append(f)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(s[0]) for s in self.samples) if v is not None]
        mx = [v for v in (num(s[1]) for s in self.samples) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# distributed helpers (torchrun)
# ---------------------------------------------------------------------------
def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------
def cubin_digest(path):
    import hashlib
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def _profile_lines(kernel, workload):
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    vals = {}
    if os.path.exists(path):
        for line in open(path):
            if line.startswith("@") and ":" in line:
                k, v = line[1:].split(":", 1)
                vals[k.strip()] = v.strip()
    return vals


def profile_value(kernel, workload, cubin_key, name):
    """A figure of the committed ncu summary of this kernel ('@name: value'),
    if it was taken on the same compiled kernel; e.g. hw_fp64_frac, the
    hardware FP64 flops ((2 dfma + dadd + dmul) per cycle, ncu) over twice
    the DFMA peak rate."""
    vals = _profile_lines(kernel, workload)
    try:
        return float(vals[name]) if vals.get("cubin_sha256") == cubin_key else None
    except (KeyError, ValueError):
        return None


def traffic_from_profile(kernel, workload, cubin_key, ncells):
    """DRAM bytes per launch from the committed ncu summary of this kernel
    (lines starting with '@'), if it was taken on the same compiled kernel
    (digest of its cubin); the capture's bytes per cell are scaled to the
    launch's cells (the traffic is per cell: inputs, outputs and the
    per-thread spill stack)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if line.startswith("@") and ":" in line:
            k, v = line[1:].split(":", 1)
            vals[k.strip()] = v.strip()
    try:
        if vals.get("cubin_sha256") != cubin_key:
            return None
        return float(vals["dram_bytes_per_cell"]) * ncells
    except (KeyError, ValueError):
        return None


def cpu_baseline(mech, states_cfg, seconds, ncells_cap=1 << 20):
    """The oracle (C++ with OpenMP over cells, as it stands) on a bounded
    sample of the workload's cells, on all host cores."""
    import oracle
    from paper_2405_05974_b300 import mechgen
    om = oracle.OracleMech(mech)
    cores = os.cpu_count() or 1
    chunk = 512
    done = 0
    gen_s = 0.0
    t0 = time.perf_counter()
    while done < ncells_cap:
        cfg = type(states_cfg)(**{**states_cfg.__dict__, "seed": states_cfg.seed + 7 + done})
        g0 = time.perf_counter()
        rho, T, Y = mechgen.generate_states(mech, cfg, chunk)
        gen_s += time.perf_counter() - g0
        om.eval(rho, T, Y, jac=True, nthreads=cores)
        done += chunk
        if time.perf_counter() - t0 - gen_s >= seconds:
            break
        chunk = min(chunk * 2, 8192)
    el = time.perf_counter() - t0 - gen_s
    # one host thread on a short sample, for the per-core rate
    cfg = type(states_cfg)(**{**states_cfg.__dict__, "seed": states_cfg.seed + 99})
    rho, T, Y = mechgen.generate_states(mech, cfg, 256)
    n1, t1 = 0, time.perf_counter()
    while time.perf_counter() - t1 < min(2.0, seconds / 4):
        om.eval(rho, T, Y, jac=True, nthreads=1)
        n1 += 256
    single = n1 / (time.perf_counter() - t1)
    return {"value": done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": single,
            "sample": f"{done} seeded cells of the workload, wdot+Tdot+Jacobian, "
                      f"{el:.1f} s on {cores} host threads (input generation excluded); "
                      f"single_core_value: {n1} cells on one thread"}


# ---------------------------------------------------------------------------
# implicit step (backward Euler, FP64 LU vs FP32 LU + FP64 refinement)
# ---------------------------------------------------------------------------
def implicit_bench(gm, mech, ncells, dt, oracle_sample=0):
    """One timed step per precision on the implicit workload (2^20 hydrocarbon
    cells, dt = 1e-6 s) after one warm-up step."""
    import torch
    from paper_2405_05974_b300 import binding, mechgen, workloads
    rho, T, Y = mechgen.generate_states(mech, workloads.STATES["implicit"], ncells)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    r = d(rho)
    dtt = torch.full((1,), dt, dtype=torch.float64, device="cuda")
    res = {}
    out = {}
    for prec, name in ((binding.QSS_LU_FP64, "fp64"), (binding.QSS_LU_FP32_IR, "fp32ir")):
        times = []
        for rep in range(2):
            t, y = d(T), d(Y)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            it, st = gm.implicit_step(r, t, y, dtt, precision=prec)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = times[-1]
        stn, itn = st.cpu().numpy(), it.cpu().numpy()
        out[name] = (t.cpu().numpy(), y.cpu().numpy(), stn)
        conv = stn == 0
        res[name] = {"cells_per_s": ncells / (ms * 1e-3), "ms": ms,
                     "status_counts": {"converged": int(conv.sum()), "maxiter": int((stn == 1).sum()),
                                       "nonfinite": int((stn == 2).sum()), "singular": int((stn == 3).sum())},
                     "newton_iters_mean": float(itn[conv].mean()) if conv.any() else None,
                     "newton_iters_max": int(itn[conv].max()) if conv.any() else None}
    a, b = out["fp64"], out["fp32ir"]
    both = (a[2] == 0) & (b[2] == 0)
    W = np.array(gm.W)[:, None]
    ca, cb = rho[None, :] * a[1] / W, rho[None, :] * b[1] / W
    pa, pb = np.vstack([ca, a[0][None]]), np.vstack([cb, b[0][None]])
    atol = np.r_[np.full(gm.N, 1e-20), 1e-10][:, None]
    rel = np.max(np.abs(pa - pb) / (np.abs(pa) + 10 * atol), axis=0)[both]
    res["fp32ir_vs_fp64"] = {"cells_converged_both": int(both.sum()),
                             "frac_within_1e-8": float(np.mean(rel <= 1e-8)) if both.any() else None,
                             "median_rel": float(np.median(rel)) if both.any() else None,
                             "max_rel": float(rel.max()) if both.any() else None,
                             "metric": "max_k |dphi_k| / (|phi_k| + 10 atol_k) per cell"}
    res["speedup_fp32ir_over_fp64"] = res["fp32ir"]["cells_per_s"] / res["fp64"]["cells_per_s"]
    res["workload"] = f"{mech['name']} backward Euler, dt = {dt:g} s, {ncells} cells"
    return res


def integrate_bench(gm, mech, ncells=16384, D=1e-9, rtol=1e-3, max_rounds=400):
    """Integration of the implicit workload's first cells over an interval D
    (qss_integrate, FP32 LU + FP64 refinement), backward-Euler and BDF2
    substeps at the same tolerance: cells/s over the interval, substeps per
    cell, outcome counts.  One untimed run on a small batch first.  The wall
    time is set by the slowest cells: every round is a sequence of Newton
    launches, and one cell's Jacobian evaluation alone takes about a
    millisecond (one thread computes it), so max_rounds bounds the run."""
    import torch
    from paper_2405_05974_b300 import binding, mechgen, workloads
    rho, T, Y = mechgen.generate_states(mech, workloads.STATES["implicit"], ncells)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    r = d(rho)
    res = {"workload": f"{mech['name']}: {ncells} cells over {D:g} s, rtol {rtol:g}, atol_C 1e-6, "
                       f"atol_T 1e-3, at most {max_rounds} substep attempts, FP32 LU + FP64 refinement"}
    for order in (1, 2):
        opts = binding.integrate_opts(rtol=rtol, atol_C=1e-6, atol_T=1e-3, order=order, max_rounds=max_rounds)
        gm.integrate(d(rho[:256]), d(T[:256]), d(Y[:, :256]), D, precision=binding.QSS_LU_FP32_IR, opts=opts)
        t, y = d(T), d(Y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        ns, st = gm.integrate(r, t, y, D, precision=binding.QSS_LU_FP32_IR, opts=opts)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ns, st = ns.cpu().numpy(), st.cpu().numpy()
        done = st == 0
        res[f"order{order}"] = {
            "cells_per_s": ncells / (ms * 1e-3), "ms": ms,
            "status_counts": {"done": int(done.sum()), "rounds_exhausted": int((st == 1).sum()),
                              "below_h_min": int((st == 2).sum())},
            "substeps_median": float(np.median(ns[done])) if done.any() else None,
            "substeps_mean": float(ns[done].mean()) if done.any() else None}
    return res


# ---------------------------------------------------------------------------
# Section 3.2 figures: simplified Jacobians, FD Jacobian
# ---------------------------------------------------------------------------
def variants_bench(key, gm, r, t, y, ncells_fd=1 << 18):
    """The relative Frobenius error (Eq. frobErr) of the exact, constant-QSS
    and zero-QSS Jacobians against the central FD Jacobian (step 1e-4) over
    100 states of the Section 3.2.1 protocol, the nonzero fraction of their
    species blocks (Table memQSS), and the throughput of the FD Jacobian
    kernel against the analytic one on the bench workload's first cells."""
    import torch
    from paper_2405_05974_b300 import analysis, binding, mechgen, workloads
    from paper_2405_05974_b300.qssc.build import build_mechanism
    mech = workloads.mechanism(key)
    rng = np.random.default_rng(11)
    C = rng.uniform(1e-4, 1.0, size=(gm.N, 100))
    Tp = rng.uniform(300.0, 1300.0, size=100)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    pr, pt, py = (d(x) for x in mechgen.concentrations_to_state(mech, C, Tp))
    Jfd = gm.jacobian_fd(pr, pt, py, 1e-4, 1e-4)
    out = {"protocol": "100 states, C ~ U[1e-4, 1] mol/m^3, T ~ U[300, 1300] K, central FD step 1e-4",
           "eps_J": {}, "nonzero_fraction": {}}
    for v in ("exact", "const_qss", "zero_qss"):
        vm = gm if v == "exact" else binding.Mechanism(build_mechanism(mech, jac_variant=v), gm.device)
        J, _, _ = vm.jacobian(pr, pt, py)
        out["eps_J"][v] = analysis.frobenius_error(J, Jfd)
        out["nonzero_fraction"][v] = analysis.nonzero_fraction(J, gm.N)
    nc = min(ncells_fd, t.shape[0])
    n = gm.n
    J = torch.empty((n * n, t.shape[0]), dtype=torch.float64, device="cuda")
    ms = {}
    for name, fn in (("analytic", lambda: gm.jacobian(r, t, y, jac=J, ncells=nc, want_rates=False)),
                     ("fd", lambda: gm.jacobian_fd(r, t, y, 1e-4, 1e-4, jac=J, ncells=nc))):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms[name] = e0.elapsed_time(e1)
    out["fd_jacobian_cells_per_s"] = nc / (ms["fd"] * 1e-3)
    out["analytic_jacobian_cells_per_s"] = nc / (ms["analytic"] * 1e-3)
    out["analytic_over_fd_speedup"] = ms["fd"] / ms["analytic"]
    out["timing_cells"] = nc
    del J
    return out


def implicit_capacity(gm, key, prec, ncells=65536):
    """Cells/s of one implicit step of `ncells` cells of workload `key` (after
    one warm-up step), the serving bench's capacity estimate."""
    import torch
    from paper_2405_05974_b300 import mechgen, workloads
    m = workloads.mechanism(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    r = d(rho)
    ms = 0.0
    for rep in range(2):
        t, y = d(T), d(Y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        gm.implicit_step(r, t, y, 1e-6, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    return ncells / (ms * 1e-3)


# ---------------------------------------------------------------------------
# serving: Poisson request stream over the continuous-batching server
# ---------------------------------------------------------------------------
def serve_bench(mechs, weights, precision, seconds, capacity_cells_s, seed=104, load=0.7):
    import torch
    from paper_2405_05974_b300 import binding, mechgen, workloads
    rng = np.random.default_rng(seed)
    lo, hi = 256, 65536
    mean_cells = (hi - lo) / np.log(hi / lo)
    rate = load * capacity_cells_s / mean_cells
    pools = {}
    for key, gm in mechs.items():
        m = workloads.mechanism(key)
        rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], hi)
        pools[key] = (gm, rho, T, np.ascontiguousarray(Y))
    keys = list(mechs)
    srv = binding.Server(0, budget_bytes=60 << 30, n_streams=4, max_batch_cells=1 << 18)
    reqs = []
    t0 = time.perf_counter()
    t_next = t0
    while True:
        now = time.perf_counter()
        if now - t0 >= seconds:
            break
        if now < t_next:
            time.sleep(min(t_next - now, 0.005))
            continue
        key = keys[rng.choice(len(keys), p=weights)]
        gm, rho, T, Y = pools[key]
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        dt = float(np.exp(rng.uniform(np.log(1e-7), np.log(1e-5))))
        off = int(rng.integers(0, hi - n + 1))
        rh = torch.from_numpy(rho[off:off + n].copy()).pin_memory()
        th = torch.from_numpy(T[off:off + n].copy()).pin_memory()
        yh = torch.from_numpy(np.ascontiguousarray(Y[:, off:off + n])).pin_memory()
        reqs.append((srv.submit(gm, rh, th, yh, dt, precision), n))
        t_next += rng.exponential(1.0 / rate)
    for rid, _ in reqs:
        srv.wait(rid)
    el = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    return {"requests": len(reqs), "offered_rate_per_s": rate, "cells": int(sum(n for _, n in reqs)),
            "p50_latency_ms": st["p50_latency_us"] / 1e3, "p99_latency_ms": st["p99_latency_us"] / 1e3,
            "cells_per_s": st["cells_per_s"], "batches": st["batches"],
            "graph_batches": st["graph_batches"], "graphs_captured": st["graphs_captured"],
            "bytes_peak": st["bytes_peak"], "wall_s": el}


# ---------------------------------------------------------------------------
def main():
    a = parse()
    rank, world, local, pg = dist_setup()
    from paper_2405_05974_b300 import workloads
    key = a.workload
    mech = workloads.mechanism(key)
    ncells = a.ncells or workloads.NCELLS[key]
    cfg = {"workload": f"{mech['name']} wdot+Jacobian", "ncells_per_gpu": ncells,
           "mechanism": {"transported": sum(1 for s in mech["species"] if not s["qss"]),
                         "qss": sum(1 for s in mech["species"] if s["qss"]),
                         "reactions": len(mech["reactions"])},
           "layout": "SoA fp64, ld = ncells" + ("" if a.jac_format == "dense" else
                                                    ", Jacobian as its structural nonzeros (CSR order)"), "l2": "inputs and outputs larger than L2 (no flush)",
           "parallelism": f"independent batches x{world}"}

    if a.impl == "reference":
        if rank != 0:
            return
        vals = []
        base = None
        per = max(2.0, a.cpu_seconds / max(a.steps + a.warmup, 1))
        for s in range(a.warmup + a.steps):
            b = cpu_baseline(mech, workloads.STATES[key], seconds=per, ncells_cap=1 << 16)
            if s >= a.warmup:
                vals.append(b["value"])
                base = b
        v = float(np.median(vals))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ncells / v * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded)", "config": cfg,
                "cpu_baseline": {**base, "value": v},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_2405_05974_b300 import autotune, binding, mechgen
    from paper_2405_05974_b300.qssc.build import build_mechanism, load_meta
    torch.cuda.set_device(local)
    opts = workloads.build_options(key)
    if a.jac_parts >= 0:
        opts["jac_parts"] = a.jac_parts
    if a.jac_format != "dense":
        opts["jac_format"] = a.jac_format
    art = autotune.artefact(mech, torch.cuda.get_device_name(local), **opts)
    meta = load_meta(art)
    gm = binding.Mechanism(art, local)
    st_cfg = workloads.STATES[key]
    st_cfg = type(st_cfg)(**{**st_cfg.__dict__, "seed": st_cfg.seed + 1000 * rank})
    rho, T, Y = mechgen.generate_states(mech, st_cfg, ncells)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    r, t, y = d(rho), d(T), d(Y)
    n = gm.n
    J = torch.empty((gm.jac_nnz, ncells), dtype=torch.float64, device="cuda")
    w = torch.empty((gm.N, ncells), dtype=torch.float64, device="cuda")
    td = torch.empty(ncells, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        gm.jacobian(r, t, y, jac=J, wdot=w, Tdot=td, stream=stream)

    for _ in range(max(a.warmup, 3)):
        step()
    torch.cuda.synchronize()
    peak = binding.measure_fp64_peak(local, 200)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    barrier(pg)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        g0.record(stream)
        for i in range(a.steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        g1.record(stream)
        torch.cuda.synchronize()
    barrier(pg)
    total_ms = max_over_ranks(pg, g0.elapsed_time(g1))
    per = [e0.elapsed_time(e1) for e0, e1 in ev]
    ms_step = total_ms / a.steps
    value = ncells * world * a.steps / (total_ms * 1e-3)
    kernel_ms = float(np.mean(per))
    flops_cell = meta["flops_jac"]
    achieved = flops_cell * ncells / (kernel_ms * 1e-3) / 1e12
    parts = int(meta.get("jac_parts", 0) or 0)
    # a partitioned Jacobian runs in chunks that fit the handle's frontier
    # buffer: one prefix and `parts` group launches each
    launches_per_step = gm.jacobian_launches(ncells)
    jac_kernel = "qss_jac_kernel" if parts < 2 else f"qss_jac_prefix_kernel + {parts} x qss_jac_group_kernel"
    cubin_key = cubin_digest(os.path.join(art, "jac.cubin")) if parts < 2 else None
    traffic = traffic_from_profile("qss_jac_kernel", key, cubin_key, ncells) if parts < 2 else None
    hw_frac = profile_value("qss_jac_kernel", key, cubin_key, "hw_fp64_frac") if parts < 2 else None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": "measured live on this GPU: FP64 DFMA microbenchmark "
                           "(qss_measure_fp64_peak); MEASURED_PEAKS.json has no FP64 entry",
            "flops_per_cell": flops_cell, "fp64_instr_per_cell_est": meta.get("fp64_instr_jac"),
            "hw_fp64_frac_ncu": hw_frac,
            "kernel": jac_kernel, "kernel_ms": kernel_ms,
            "hbm_algorithmic_gbs": (8.0 * (2 + gm.N + gm.N + 1 + gm.jac_nnz) * ncells) / (kernel_ms * 1e-3) / 1e9}

    e2e = None
    if not a.no_e2e:
        rh = torch.from_numpy(rho).pin_memory()
        th = torch.from_numpy(T).pin_memory()
        yh = torch.from_numpy(np.ascontiguousarray(Y)).pin_memory()
        Jh = torch.empty((gm.jac_nnz, ncells), dtype=torch.float64).pin_memory()
        wh = torch.empty((gm.N, ncells), dtype=torch.float64).pin_memory()
        tdh = torch.empty(ncells, dtype=torch.float64).pin_memory()
        gm.jacobian_host(rh, th, yh, jac=Jh, wdot=wh, Tdot=tdh)     # warm-up (staging alloc)
        e_steps = max(1, min(a.steps, 3))
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(e_steps):
            gm.jacobian_host(rh, th, yh, jac=Jh, wdot=wh, Tdot=tdh)
        el = max_over_ranks(pg, time.perf_counter() - t0)
        nchunks = -(-ncells // 65536)
        # the host link on its own: one 2 GiB device -> pinned host copy
        hb = torch.empty(1 << 28, dtype=torch.float64).pin_memory()
        db = torch.empty(1 << 28, dtype=torch.float64, device="cuda")
        hb.copy_(db)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        hb.copy_(db)
        torch.cuda.synchronize()
        link = hb.numel() * 8 / (time.perf_counter() - t1) / 1e9
        del hb, db
        d2h = 8 * (gm.jac_nnz + gm.N + 1) * ncells
        e2e = {"value": ncells * world * e_steps / el, "unit": UNIT,
               "h2d_bytes_per_step": 8 * (2 + gm.N) * ncells,
               "d2h_bytes_per_step": d2h,
               "api": "qss_jacobian_host (pinned host arrays, chunked copy/compute overlap)",
               "gpu_launches_per_step": nchunks,
               "d2h_gbs_achieved": d2h * e_steps / el / 1e9,
               "host_link_d2h_gbs": link}
        del Jh
    variants = None
    if not a.no_variants and rank == 0 and key in ("tiny", "hydrocarbon"):
        variants = variants_bench(key, gm, r, t, y)
    implicit = None
    if not a.no_implicit and key == "hydrocarbon":
        implicit = implicit_bench(gm, mech, a.implicit_ncells or workloads.NCELLS["implicit"],
                                  workloads.IMPLICIT_DT)
    integration = None
    if a.integrate and key == "hydrocarbon" and rank == 0:
        integration = integrate_bench(gm, mech)
    serving = None
    if not a.no_serve and key == "hydrocarbon" and rank == 0:
        from paper_2405_05974_b300 import binding as _b
        mechs = {k: (gm if k == "hydrocarbon" else
                     _b.Mechanism(build_mechanism(workloads.mechanism(k), **workloads.build_options(k)), local))
                 for k in ("tiny", "hydrocarbon", "large")}
        weights = [0.2, 0.6, 0.2]
        serving = {"mix": "tiny 0.2 / hydrocarbon 0.6 / large 0.2 (by request)",
                   "sizes": "log-uniform 256..65536 cells", "dt": "log-uniform 1e-7..1e-5 s",
                   "budget_bytes": 60 << 30, "load": 0.7, "graphs": True,
                   "capacity": "cells/s of one implicit step of 65536 cells per mechanism, "
                               "combined by the mix's cell-weighted harmonic mean"}
        for prec, name in ((_b.QSS_LU_FP32_IR, "fp32ir"), (_b.QSS_LU_FP64, "fp64")):
            caps = {k: implicit_capacity(mechs[k], k, prec) for k in mechs}
            cap = 1.0 / sum(w / caps[k] for w, k in zip(weights, mechs))
            serving[name] = serve_bench(mechs, weights, prec, a.serve_seconds, cap)
            serving[name]["capacity_cells_per_s"] = {**caps, "mix": cap}
    cpu = None
    if rank == 0 and not a.no_cpu:
        cpu = cpu_baseline(mech, workloads.STATES[key], a.cpu_seconds)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded mechanism and states)",
            "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": a.steps * launches_per_step, "clocks": clk.summary(),
            "implicit": implicit, "integration": integration, "serving": serving,
            "jacobian_variants": variants,
            "kernel": {"ptxas": {k: v for k, v in meta["kernels"].items() if k.startswith("qss_jac")},
                       "defines": meta.get("defines", []),
                       "ops_per_cell": meta["ops_jac"], "artefact": os.path.basename(art)}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
