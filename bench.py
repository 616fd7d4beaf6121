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
    p.add_argument("--serve-seconds", type=float, default=16.0)
    p.add_argument("--fp64-probe", action="store_true",
                   help="print the FP64 pipe probe grid (latency, warps per SM, active lanes) and exit")
    p.add_argument("--memory-study", action="store_true",
                   help="time the Section 4.1 memory-footprint variants that are built (Alg. 2 n_op, "
                        "Alg. 3 on/off) and exit")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the tiny and large workloads' entries (by_config)")
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
def _phi(gm, rho, T, Y):
    W = np.array(gm.W)[:, None]
    return np.vstack([rho[None, :] * Y / W, T[None, :]])


def _rel_err(gm, pa, pb):
    """max_k |pa_k - pb_k| / (|pb_k| + 10 atol_k) per cell (atol_C 1e-20, atol_T 1e-10)."""
    atol = np.r_[np.full(gm.N, 1e-20), 1e-10][:, None]
    with np.errstate(invalid="ignore"):
        return np.max(np.abs(pa - pb) / (np.abs(pb) + 10 * atol), axis=0)


STATUS = ("converged", "maxiter", "nonfinite", "singular")


def implicit_bench(gm, mech, ncells, dt):
    """One timed step per precision (after one warm-up step) of the implicit
    workload: hydrocarbon mechanism and states, `ncells` cells, step dt.
    Reports the throughput over all cells and over the cells that converged,
    the status counts, Newton iterations, the FP32-IR/FP64 difference on the
    cells both converge on and the cells whose status differs.  Returns the
    line and the host copies of the results (for the oracle comparison of the
    CPU-baseline leg)."""
    import torch
    from paper_2405_05974_b300 import binding, mechgen, workloads
    rho, T, Y = mechgen.generate_states(mech, workloads.STATES["implicit"], ncells)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    r = d(rho)
    dtt = torch.full((1,), dt, dtype=torch.float64, device="cuda")
    res = {}
    out = {}
    reuse = binding.newton_opts(jac_reuse=1)
    forms = [(binding.QSS_LU_FP64, "fp64", None), (binding.QSS_LU_FP32_IR, "fp32ir", None),
             (binding.QSS_LU_FP64, "fp64_reuse", reuse), (binding.QSS_LU_FP32_IR, "fp32ir_reuse", reuse)]
    if gm.has_jac32:
        forms += [(binding.QSS_LU_MIXED, "mixed", None), (binding.QSS_LU_MIXED, "mixed_reuse", reuse)]
    for prec, name, opts in forms:
        times = []
        for rep in range(2):
            t, y = d(T), d(Y)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            it, st = gm.implicit_step(r, t, y, dtt, precision=prec, opts=opts)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = times[-1]
        stn, itn = st.cpu().numpy(), it.cpu().numpy()
        out[name] = (t.cpu().numpy(), y.cpu().numpy(), stn)
        conv = stn == 0
        res[name] = {"cells_per_s": ncells / (ms * 1e-3),
                     "converged_cells_per_s": int(conv.sum()) / (ms * 1e-3),
                     "converged_fraction": float(conv.mean()), "ms": ms,
                     "status_counts": {nm: int((stn == i).sum()) for i, nm in enumerate(STATUS)},
                     "newton_iters_mean": float(itn[conv].mean()) if conv.any() else None,
                     "newton_iters_max": int(itn[conv].max()) if conv.any() else None}
    for other in [x for x in ("fp32ir", "mixed") if x in out]:
        res[other + "_vs_fp64"] = _vs_fp64(gm, rho, out["fp64"], out[other])
    res["speedup_fp32ir_over_fp64"] = res["fp32ir"]["cells_per_s"] / res["fp64"]["cells_per_s"]
    if "mixed" in out:
        res["speedup_mixed_over_fp64"] = res["mixed"]["cells_per_s"] / res["fp64"]["cells_per_s"]
        res["speedup_mixed_reuse_over_fp64"] = res["mixed_reuse"]["cells_per_s"] / res["fp64"]["cells_per_s"]
        res["converged_speedup_mixed_over_fp64"] = (res["mixed"]["converged_cells_per_s"] /
                                                    max(res["fp64"]["converged_cells_per_s"], 1e-30))
    # Jacobian reuse (opt-in) against full Newton of the same precision
    for name, gate in (("fp64", 1e-10), ("fp32ir", 1e-8), ("mixed", 1e-8)):
        if name not in out:
            continue
        f, rr = out[name], out[name + "_reuse"]
        both = (f[2] == 0) & (rr[2] == 0)
        rel = _rel_err(gm, _phi(gm, rho, rr[0], rr[1]), _phi(gm, rho, f[0], f[1]))[both]
        res[name + "_reuse_vs_full"] = {
            "cells_converged_both": int(both.sum()),
            "frac_within_gate": float(np.mean(rel <= gate)) if both.any() else None,
            "gate": f"{gate:g} relative + 10 atol", "max_rel": float(rel.max()) if both.any() else None,
            "speedup": res[name + "_reuse"]["cells_per_s"] / res[name]["cells_per_s"]}
    res["speedup_fp32ir_reuse_over_fp64"] = res["fp32ir_reuse"]["cells_per_s"] / res["fp64"]["cells_per_s"]
    res["workload"] = f"{mech['name']} backward Euler, dt = {dt:g} s, {ncells} cells"
    res["forms"] = ("fp64 / fp32ir: full Newton (the analytic Jacobian every iteration, the oracle's "
                    "definition); mixed: fp32ir with the Jacobian's derivative terms assembled in FP32 "
                    "(qss_jacobian_mixed; rates, K_c, the QSS solve and the residual in FP64); *_reuse: a cell "
                    "keeps its Jacobian while its update norm contracts by 0.3x per iteration (jac_reuse = 1)")
    return res, (rho, T, Y, out)


def _vs_fp64(gm, rho, a, b):
    """Form b's implicit-step results against the FP64 form's (a)."""
    both = (a[2] == 0) & (b[2] == 0)
    rel = _rel_err(gm, _phi(gm, rho, b[0], b[1]), _phi(gm, rho, a[0], a[1]))[both]
    differ = a[2] != b[2]
    # cells both forms converged on but to different states: the backward-
    # Euler system can have more than one root, and the Newton path (which the
    # precision of the solve perturbs) decides which one is found; count how
    # many of those states hold a negative concentration (a non-physical root)
    pa_, pb_ = _phi(gm, rho, a[0], a[1]), _phi(gm, rho, b[0], b[1])
    far = np.zeros(both.shape, bool)
    far[both] = rel > 1e-8
    neg = (pa_[:gm.N] < 0).any(0) | (pb_[:gm.N] < 0).any(0)
    return {"cells_converged_both": int(both.sum()), "cells_beyond_1e-8": int(far.sum()),
            "of_those_with_a_negative_concentration": int((far & neg).sum()),
            "example_cells_beyond_1e-8": np.nonzero(far)[0][:8].tolist(),
            "frac_within_1e-8": float(np.mean(rel <= 1e-8)) if both.any() else None,
            "median_rel": float(np.median(rel)) if both.any() else None,
            "max_rel": float(rel.max()) if both.any() else None,
            "metric": "max_k |dphi_k| / (|phi_k| + 10 atol_k) per cell",
            "status_differs": int(differ.sum()),
            "status_pairs_from_fp64": {
                f"{STATUS[i]}->{STATUS[j]}": int(((a[2] == i) & (b[2] == j)).sum())
                for i in range(4) for j in range(4) if i != j and ((a[2] == i) & (b[2] == j)).any()}}


def implicit_cpu_baseline(gm, mech, dt, data, seconds):
    """The oracle's backward-Euler step (as it stands, OpenMP on all host
    threads) on a bounded sample of the same cells: its cells/s, and the GPU
    results of the same sampled cells compared with it, for both forms."""
    import oracle
    rho, T, Y, out = data
    n = rho.shape[0]
    om = oracle.OracleMech(mech)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(7)
    order = rng.permutation(n)
    done, chunk, el = 0, 256, 0.0
    idx_all, res = [], []
    while done < n and el < seconds:
        idx = np.sort(order[done:done + chunk])
        t0 = time.perf_counter()
        To, Yo, ito, sto = om.be_step(rho[idx], T[idx], np.ascontiguousarray(Y[:, idx]), dt, max_iter=20,
                                      nthreads=cores)
        el += time.perf_counter() - t0
        idx_all.append(idx)
        res.append((To, Yo, sto))
        done += idx.size
        chunk = min(chunk * 2, 4096)
    idx = np.concatenate(idx_all)
    To = np.concatenate([r[0] for r in res])
    Yo = np.concatenate([r[1] for r in res], axis=1)
    sto = np.concatenate([r[2] for r in res])
    po = _phi(gm, rho[idx], To, Yo)
    cmp = {}
    for name, gate in (("fp64", 1e-10), ("fp32ir", 1e-8), ("fp64_reuse", 1e-10), ("fp32ir_reuse", 1e-8),
                       ("mixed", 1e-8), ("mixed_reuse", 1e-8)):
        if name not in out:
            continue
        Tg, Yg, stg = out[name]
        pg = _phi(gm, rho[idx], Tg[idx], Yg[:, idx])
        both = (sto == 0) & (stg[idx] == 0)
        rel = _rel_err(gm, pg, po)[both]
        cmp[name] = {"cells_compared": int(both.sum()),
                     "status_agrees_with_oracle": float(np.mean(sto == stg[idx])),
                     "frac_within_gate": float(np.mean(rel <= gate)) if both.any() else None,
                     "gate": f"{gate:g} relative + 10 atol", "median_rel": float(np.median(rel)) if both.any() else None,
                     "max_rel": float(rel.max()) if both.any() else None}
    return {"value": done / el, "unit": "cells/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} randomly sampled cells of the step's {n}, {el:.1f} s on {cores} host threads",
            "oracle_converged_fraction": float(np.mean(sto == 0)),
            "gpu_vs_oracle_on_sample": cmp}


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
    """precision: one for every mechanism, or a dict by workload key."""
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
        prec = precision[key] if isinstance(precision, dict) else precision
        reqs.append((srv.submit(gm, rh, th, yh, dt, prec), n))
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
def _config(mech, key, ncells, world, jac_format="dense", l2="inputs and outputs larger than L2 (no flush)"):
    return {"workload": f"{mech['name']} wdot+Jacobian", "ncells_per_gpu": ncells,
            "mechanism": {"transported": sum(1 for s in mech["species"] if not s["qss"]),
                          "qss": sum(1 for s in mech["species"] if s["qss"]),
                          "reactions": len(mech["reactions"])},
            "layout": "SoA fp64, ld = ncells" + ("" if jac_format == "dense" else
                                                   ", Jacobian as its structural nonzeros (CSR order)"),
            "l2": l2, "parallelism": f"independent batches x{world}"}


def _jac_cubin_digest(art, parts):
    """Digest of the Jacobian's cubins (the single kernel, or the prefix and
    group kernels in order), matched against the committed ncu summary."""
    import hashlib
    from paper_2405_05974_b300.qssc.build import cubin_file
    names = ["jac.cubin"] if parts < 2 else ["jac_prefix.cubin"] + [f"jac_g{i}.cubin" for i in range(parts)]
    h = hashlib.sha256()
    for nm in names:
        h.update(open(cubin_file(art, nm), "rb").read())
    return h.hexdigest()[:16] if parts >= 2 else cubin_digest(cubin_file(art, "jac.cubin"))


def jacobian_bench(key, ncells, steps, warmup, local, rank, world, pg, do_e2e=True, cpu_seconds=0.0,
                   jac_parts=-1, jac_format="dense", flush_l2=False, keep_sample=0):
    """Timed qss_jacobian steps (wdot + Tdot + J of `ncells` cells of workload
    `key`) through the C ABI, CUDA events on the launching stream, max over
    ranks; the roofline of the Jacobian kernel(s) against the FP64 peak
    measured live; optionally the end-to-end rate from pinned host arrays and
    the oracle's CPU baseline.  With flush_l2 a 256 MB buffer is written
    between timed steps (for workloads whose arrays fit in L2) and only the
    steps themselves are timed."""
    import torch
    from paper_2405_05974_b300 import autotune, binding, mechgen, workloads
    from paper_2405_05974_b300.qssc.build import load_meta
    mech = workloads.mechanism(key)
    opts = {}
    if jac_parts >= 0:
        opts["jac_parts"] = jac_parts
    if jac_format != "dense":
        opts["jac_format"] = jac_format
    if key in workloads.MIXED_JACOBIAN:
        opts["jac32"] = True     # the mixed-precision kernels beside the FP64 ones (same FP64 cubins)
    art = autotune.artefact(mech, torch.cuda.get_device_name(local), defaults=workloads.build_options(key),
                            ncells=ncells, **opts)
    meta = load_meta(art)
    gm = binding.Mechanism(art, local)
    st_cfg = workloads.STATES[key]
    st_cfg = type(st_cfg)(**{**st_cfg.__dict__, "seed": st_cfg.seed + 1000 * rank})
    rho, T, Y = mechgen.generate_states(mech, st_cfg, ncells)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    r, t, y = d(rho), d(T), d(Y)
    J = torch.empty((gm.jac_nnz, ncells), dtype=torch.float64, device="cuda")
    w = torch.empty((gm.N, ncells), dtype=torch.float64, device="cuda")
    td = torch.empty(ncells, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(32 << 20, dtype=torch.float64, device="cuda") if flush_l2 else None

    def step():
        gm.jacobian(r, t, y, jac=J, wdot=w, Tdot=td, stream=stream)

    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    peak = binding.measure_fp64_peak(local, 200)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier(pg)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        g0.record(stream)
        for i in range(steps):
            if flush is not None:
                flush.fill_(float(i))
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        g1.record(stream)
        torch.cuda.synchronize()
    barrier(pg)
    # the mixed-precision Jacobian (derivative terms in FP32) on the same
    # cells, timed the same way after the FP64 steps (it overwrites J)
    mixed = None
    if gm.has_jac32:
        J32 = torch.empty_like(J)
        for _ in range(3):
            gm.jacobian(r, t, y, jac=J32, wdot=w, Tdot=td, stream=stream, mixed=True)
        m_ms = []
        for i in range(steps):
            if flush is not None:
                flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gm.jacobian(r, t, y, jac=J32, wdot=w, Tdot=td, stream=stream, mixed=True)
            e1.record(stream)
            e1.synchronize()
            m_ms.append(e0.elapsed_time(e1))
        mixed = {"kernel": "qss_jac32_kernel", "ms": float(np.mean(m_ms)),
                 "cells_per_s": ncells / (float(np.mean(m_ms)) * 1e-3),
                 "fp64_instr_per_cell_est": meta.get("fp64_instr_jac32"),
                 "form": "qss_jacobian_mixed: wdot, Tdot and everything they need in FP64, the Jacobian's "
                         "derivative terms in FP32 (stored as FP64); the Newton matrix of the mixed implicit step"}
    sample = None
    if keep_sample:
        # a seeded sample of the timed step's cells, with their outputs, for
        # the oracle comparison of the CPU-baseline leg
        idx = np.sort(np.random.default_rng(17).choice(ncells, size=min(keep_sample, ncells), replace=False))
        ii = torch.from_numpy(idx).cuda()
        sample = {"idx": idx, "rho": rho[idx], "T": T[idx], "Y": np.ascontiguousarray(Y[:, idx]),
                  "jac": J.index_select(1, ii).cpu().numpy(), "wdot": w.index_select(1, ii).cpu().numpy(),
                  "Tdot": td.index_select(0, ii).cpu().numpy(), "jac_format": jac_format}
        if mixed is not None:
            sample["jac32"] = J32.index_select(1, ii).cpu().numpy()
    if mixed is not None:
        del J32
    per = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms = max_over_ranks(pg, float(np.sum(per)) if flush is not None else g0.elapsed_time(g1))
    ms_step = total_ms / steps
    value = ncells * world * steps / (total_ms * 1e-3)
    kernel_ms = float(np.mean(per))
    if mixed is not None:
        mixed["speedup_over_fp64_kernel"] = kernel_ms / mixed["ms"]
    parts = int(meta.get("jac_parts", 0) or 0)
    flops_cell = meta["flops_jac_parts"] if parts >= 2 else meta["flops_jac"]
    achieved = flops_cell * ncells / (kernel_ms * 1e-3) / 1e12
    launches_per_step = gm.jacobian_launches(ncells)
    if parts < 2:
        jac_kernel, prof = "qss_jac_kernel", "qss_jac_kernel"
    else:
        jac_kernel, prof = f"qss_jac_prefix_kernel + {parts} x qss_jac_group_kernel", "qss_jac_parts"
    cubin_key = _jac_cubin_digest(art, parts)
    traffic = traffic_from_profile(prof, key, cubin_key, ncells)
    hw_frac = profile_value(prof, key, cubin_key, "hw_fp64_frac")
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": "measured live on this GPU: FP64 DFMA microbenchmark "
                           "(qss_measure_fp64_peak); MEASURED_PEAKS.json has no FP64 entry",
            "flops_per_cell": flops_cell, "fp64_instr_per_cell_est": meta.get("fp64_instr_jac"),
            "hw_fp64_frac_ncu": hw_frac, "kernel": jac_kernel, "kernel_ms": kernel_ms,
            "cubin_digest": cubin_key,
            "algorithmic_bytes_per_cell": 8 * (2 + gm.N + gm.N + 1 + gm.jac_nnz),
            "hbm_algorithmic_gbs": (8.0 * (2 + gm.N + gm.N + 1 + gm.jac_nnz) * ncells) / (kernel_ms * 1e-3) / 1e9}
    e2e = None
    if do_e2e:
        rh = torch.from_numpy(rho).pin_memory()
        th = torch.from_numpy(T).pin_memory()
        yh = torch.from_numpy(np.ascontiguousarray(Y)).pin_memory()
        Jh = torch.empty((gm.jac_nnz, ncells), dtype=torch.float64).pin_memory()
        wh = torch.empty((gm.N, ncells), dtype=torch.float64).pin_memory()
        tdh = torch.empty(ncells, dtype=torch.float64).pin_memory()
        gm.jacobian_host(rh, th, yh, jac=Jh, wdot=wh, Tdot=tdh)     # warm-up (staging alloc)
        # small batches take a fraction of a millisecond end to end: repeat
        # them enough for the host clock (the same count on every rank)
        e_steps = max(1, min(steps, 3)) if ncells >= (1 << 18) else 50
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(e_steps):
            gm.jacobian_host(rh, th, yh, jac=Jh, wdot=wh, Tdot=tdh)
        el = max_over_ranks(pg, time.perf_counter() - t0)
        nchunks = -(-ncells // 65536)
        d2h = 8 * (gm.jac_nnz + gm.N + 1) * ncells
        e2e = {"value": ncells * world * e_steps / el, "unit": UNIT,
               "h2d_bytes_per_step": 8 * (2 + gm.N) * ncells, "d2h_bytes_per_step": d2h,
               "api": "qss_jacobian_host (pinned host arrays, chunked copy/compute overlap)",
               "gpu_launches_per_step": nchunks * (1 if parts < 2 else parts + 1),
               "d2h_gbs_achieved": d2h * e_steps / el / 1e9}
        del Jh
    cpu = None
    if rank == 0 and cpu_seconds > 0:
        cpu = cpu_baseline(mech, workloads.STATES[key], cpu_seconds)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms_step, "steps": steps,
           "warmup": max(warmup, 3), "config": _config(mech, key, ncells, world, jac_format,
                                                         "arrays fit in L2: a 256 MB buffer is written between "
                                                         "timed steps" if flush_l2 else
                                                         "inputs and outputs larger than L2 (no flush)"),
           "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": steps * launches_per_step,
           "mixed_jacobian": mixed,
           "clocks": clk.summary(),
           "kernel": {"ptxas": {k: v for k, v in meta["kernels"].items() if k.startswith("qss_jac")},
                      "defines": meta.get("defines", []),
                      "ops_per_cell": meta["ops_jac"] if parts < 2 else
                      {"prefix": meta["ops_prefix"], "groups": meta["ops_groups"]},
                      "artefact": os.path.basename(art)}}
    return out, (gm, r, t, y, mech, sample)


def memory_study(local):
    """Section 4.1 on this GPU: the Jacobian kernel built with Alg. 2's
    replacement thresholds n_op = 0, 10, 20 and with Alg. 3's recycling off
    (every value computed before any output is stored), for the tiny (2^20
    cells) and hydrocarbon (2^19 cells) workloads.  Per variant: the kernel
    time (median of 5 CUDA-event timings), the stored values of the emitted
    code, its FP64 instructions per cell, registers and spills.  Variants
    that are not built are listed as such (they are not compiled here)."""
    from paper_2405_05974_b300 import autotune, workloads
    from paper_2405_05974_b300.qssc.build import find_artefact, load_meta
    out = []
    for key, nc in (("tiny", 1 << 20), ("hydrocarbon", 1 << 19)):
        mech = workloads.mechanism(key)
        for opts in ({}, {"replace_nop": 10}, {"replace_nop": 20}, {"emit_order": "all_first"}):
            # n_op = 0: the workload's own build (its FP64 Jacobian kernel is
            # the plain one; the mixed kernel beside it is not timed here)
            art = find_artefact(mech, **(opts or workloads.build_options(key)))
            rec = {"workload": key, "ncells": nc, "options": opts}
            if art is None:
                rec["status"] = "not built"
                out.append(rec)
                continue
            meta = load_meta(art)
            rec.update({"ms": autotune.time_jacobian(art, key, nc, device=local),
                        "stored_values": meta.get("stored_values_jac"),
                        "fp64_instr_per_cell": meta.get("fp64_instr_jac"), "dag_flops": meta.get("flops_jac"),
                        "ptxas": meta["kernels"].get("qss_jac_kernel")})
            out.append(rec)
    return out


def parity_on_sample(mech, sample, seconds=20.0):
    """The timed step's sampled cells against the oracle (CPU-baseline leg):
    the per-entry gate |x - x_ref| <= 1e-10 |x_ref| + 1e-20 + 16 e_ref (e_ref
    the oracle's running-error bound), how many entries needed the rounding
    allowance, and for those the distance to the oracle's binary128 rerun."""
    import oracle
    om = oracle.OracleMech(mech)
    t0 = time.perf_counter()
    ref = om.eval(sample["rho"], sample["T"], sample["Y"])
    eb = om.errbound(sample["rho"], sample["T"], sample["Y"])
    out = {"cells": int(sample["idx"].size)}
    for name in ("wdot", "Tdot", "jac"):
        if name == "jac" and sample["jac_format"] != "dense":
            continue
        x, rf, b = sample[name], ref[name], eb[name]
        err = np.abs(x - rf)
        tol = 1e-10 * np.abs(rf) + 1e-20
        ok = (err <= tol + 16 * b) & np.isfinite(x)
        needed = ok & (err > tol)
        big = np.abs(rf) > 1e-20     # relative errors of entries above the absolute floor
        d = {"entries": int(x.size), "fail": int((~ok).sum()), "needed_bound": int(needed.sum()),
             "max_rel": float(np.max(err[big] / np.abs(rf[big]))) if big.any() else 0.0}
        if needed.any() and time.perf_counter() - t0 < seconds:
            cells = np.unique(np.nonzero(needed)[-1])
            q = om.eval_q128(sample["rho"][cells], sample["T"][cells],
                             np.ascontiguousarray(sample["Y"][:, cells]))[name]
            sub = needed[..., cells]
            xv, qv, bv = x[..., cells][sub], q[sub], b[..., cells][sub]
            eq = np.abs(xv - qv)
            d["needed_within_target_of_binary128"] = int((eq <= 1e-10 * np.abs(qv) + 1e-20).sum())
            d["needed_within_gate_of_binary128"] = int((eq <= 1e-10 * np.abs(qv) + 1e-20 + 16 * bv).sum())
            qb = np.abs(qv) > 1e-20
            d["needed_max_rel_to_binary128"] = float(np.max(eq[qb] / np.abs(qv[qb]))) if qb.any() else 0.0
        out[name] = d
    out["gate"] = "|x - x_ref| <= 1e-10 |x_ref| + 1e-20 + 16 e_ref (e_ref: the oracle's running-error bound)"
    if "jac32" in sample and sample["jac_format"] == "dense":
        # the mixed-precision Jacobian against the FP32 form of the same bound
        x, rf = sample["jac32"], ref["jac"]
        err = np.abs(x - rf)
        bound = 2.0 ** 29 * eb["jac"] + 1e-20
        big = np.abs(rf) > 1e-20
        out["jac32"] = {"entries": int(x.size), "fail": int((~(err <= bound)).sum()),
                        "max_err_over_bound": float(np.max(err / bound)),
                        "median_rel": float(np.median(err[big] / np.abs(rf[big]))) if big.any() else 0.0,
                        "gate": "|J - J_ref| <= 2^29 e_ref + 1e-20 (the FP32 form of the FP64 rounding bound)"}
    return out


def main():
    a = parse()
    rank, world, local, pg = dist_setup()
    from paper_2405_05974_b300 import workloads
    key = a.workload
    mech = workloads.mechanism(key)
    ncells = a.ncells or workloads.NCELLS[key]
    cfg = _config(mech, key, ncells, world, a.jac_format)

    if a.impl == "reference":
        if rank != 0:
            return
        vals, walls, cells = [], [], []
        base = None
        per = max(2.0, a.cpu_seconds / max(a.steps + a.warmup, 1))
        for s in range(a.warmup + a.steps):
            t0 = time.perf_counter()
            b = cpu_baseline(mech, workloads.STATES[key], seconds=per, ncells_cap=1 << 16)
            wall = time.perf_counter() - t0
            if s >= a.warmup:
                vals.append(b["value"])
                walls.append(wall)
                base = b
        v = float(np.median(vals))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": float(np.median(walls)) * 1e3,
                "ms_per_step_note": "wall time of one step = one bounded sample of the workload (see "
                                    "cpu_baseline.sample); the full workload at this rate would take "
                                    f"{ncells / v * 1e3:.0f} ms (extrapolated, cells are independent)",
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded)", "config": cfg,
                "cpu_baseline": {**base, "value": v},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_2405_05974_b300 import binding
    from paper_2405_05974_b300.qssc.build import build_mechanism
    torch.cuda.set_device(local)
    if a.memory_study:
        print(json.dumps({"memory_study": memory_study(local)}))
        return
    if a.fp64_probe:
        grid = []
        for wps, lanes, dep in [(4, 32, True), (8, 32, True), (4, 32, False), (8, 32, False), (16, 32, False),
                                (32, 32, False), (16, 16, False), (16, 8, False), (16, 4, False), (16, 1, False)]:
            tf, cyc = binding.measure_fp64_pipe(wps, lanes, dep, local)
            grid.append({"warps_per_sm": wps, "active_lanes": lanes, "dependent_chain": dep,
                         "lane_tflops": tf, "cycles_per_warp_fma": cyc})
        print(json.dumps({"fp64_pipe_probe": grid, "peak_tflops": binding.measure_fp64_peak(local, 200)}))
        return
    head, (gm, r, t, y, _, sample) = jacobian_bench(key, ncells, a.steps, a.warmup, local, rank, world, pg,
                                                   do_e2e=not a.no_e2e, jac_parts=a.jac_parts,
                                                   jac_format=a.jac_format,
                                                   keep_sample=0 if (a.no_cpu or rank) else 512)
    if head["e2e"] is not None:
        # the host link on its own: one 2 GiB device -> pinned host copy
        hb = torch.empty(1 << 28, dtype=torch.float64).pin_memory()
        db = torch.empty(1 << 28, dtype=torch.float64, device="cuda")
        hb.copy_(db)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        hb.copy_(db)
        torch.cuda.synchronize()
        head["e2e"]["host_link_d2h_gbs"] = hb.numel() * 8 / (time.perf_counter() - t1) / 1e9
        del hb, db
    # the other workloads of the wdot+Jacobian metric (tiny: 4096 cells,
    # L2-resident; large: 2^20 cells, partitioned Jacobian), each with its own
    # roofline, end-to-end rate and CPU baseline
    by_config = None
    if not a.no_configs and key == "hydrocarbon" and ncells == workloads.NCELLS["hydrocarbon"]:
        by_config = {}
        for k2 in ("tiny", "large"):
            c2, (g2, *_rest) = jacobian_bench(k2, workloads.NCELLS[k2], min(a.steps, 10), 3, local, rank, world,
                                              pg, do_e2e=not a.no_e2e,
                                              cpu_seconds=0.0 if a.no_cpu else 4.0, flush_l2=(k2 == "tiny"),
                                              keep_sample=0 if (a.no_cpu or rank) else 128)
            if c2["cpu_baseline"] is not None and _rest[-1] is not None:
                c2["cpu_baseline"]["gpu_vs_oracle_on_sample"] = parity_on_sample(workloads.mechanism(k2), _rest[-1])
            by_config[k2] = c2
            del g2, _rest
            torch.cuda.empty_cache()
    variants = None
    if not a.no_variants and rank == 0 and key in ("tiny", "hydrocarbon"):
        variants = variants_bench(key, gm, r, t, y)
    implicit = None
    if not a.no_implicit and key == "hydrocarbon":
        implicit = {}
        for tag, dt in (("dt_1e-6", workloads.IMPLICIT_DT), ("dt_1e-11", workloads.IMPLICIT_DT_CONVERGING)):
            res, data = implicit_bench(gm, mech, a.implicit_ncells or workloads.NCELLS["implicit"], dt)
            if rank == 0 and not a.no_cpu:
                res["cpu_baseline"] = implicit_cpu_baseline(gm, mech, dt, data, 4.0)
            implicit[tag] = res
            del data
        implicit["note"] = ("dt_1e-6 is the configured step; at dt_1e-11 plain Newton from the initial "
                            "state converges in >= 95 % of the cells (the synthetic states' fastest "
                            "time scales are ~1e-11 s), so both forms are compared on nearly every cell")
    integration = None
    if a.integrate and key == "hydrocarbon" and rank == 0:
        integration = integrate_bench(gm, mech)
    serving = None
    if not a.no_serve and key == "hydrocarbon" and rank == 0:
        from paper_2405_05974_b300 import autotune
        gpu_name = torch.cuda.get_device_name(local)
        # the tuned variant of each mechanism for the serving size class
        # (batches of up to 65536 cells)
        arts = {k: autotune.artefact(workloads.mechanism(k), gpu_name, defaults=workloads.build_options(k),
                                     ncells=65536, **({"jac32": True} if k in workloads.MIXED_JACOBIAN else {}))
                for k in ("tiny", "hydrocarbon", "large")}
        mechs = {k: (gm if os.path.samefile(arts[k], gm.dir) else binding.Mechanism(arts[k], local))
                 for k in arts}
        weights = [0.2, 0.6, 0.2]
        serving = {"mix": "tiny 0.2 / hydrocarbon 0.6 / large 0.2 (by request)",
                   "artefacts": "the autotuned Jacobian variant of each mechanism for batches of up to 65536 "
                                "cells (tuning.json)",
                   "sizes": "log-uniform 256..65536 cells", "dt": "log-uniform 1e-7..1e-5 s",
                   "budget_bytes": 60 << 30, "load": 0.7, "graphs": True,
                   "capacity": "cells/s of one implicit step of 65536 cells per mechanism, "
                               "combined by the mix's cell-weighted harmonic mean"}
        # mixed: the mixed-precision Jacobian where the artefact has it (single
        # kernel or partitioned), else FP32-IR
        mixed = {k: (binding.QSS_LU_MIXED if mechs[k].has_jac32 else binding.QSS_LU_FP32_IR) for k in mechs}
        serving["mixed_precision_by_mechanism"] = {k: ("mixed" if v == binding.QSS_LU_MIXED else "fp32ir")
                                                   for k, v in mixed.items()}
        for prec, name in ((mixed, "mixed"), (binding.QSS_LU_FP32_IR, "fp32ir"), (binding.QSS_LU_FP64, "fp64")):
            caps = {k: implicit_capacity(mechs[k], k, prec[k] if isinstance(prec, dict) else prec) for k in mechs}
            cap = 1.0 / sum(w / caps[k] for w, k in zip(weights, mechs))
            serving[name] = serve_bench(mechs, weights, prec, a.serve_seconds, cap)
            serving[name]["capacity_cells_per_s"] = {**caps, "mix": cap}
    cpu = None
    if rank == 0 and not a.no_cpu:
        cpu = cpu_baseline(mech, workloads.STATES[key], a.cpu_seconds)
        if sample is not None:
            cpu["gpu_vs_oracle_on_sample"] = parity_on_sample(mech, sample)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded mechanism and states)", "config": cfg, "roofline": head["roofline"],
            "cpu_baseline": cpu, "e2e": head["e2e"], "gpu_launches": head["gpu_launches"],
            "clocks": head["clocks"], "mixed_jacobian": head["mixed_jacobian"], "by_config": by_config,
            "implicit": implicit,
            "integration": integration, "serving": serving, "jacobian_variants": variants,
            "kernel": head["kernel"]}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
