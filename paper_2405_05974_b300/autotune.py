"""Per-GPU tuning of the analytic Jacobian kernel's build variant.

The generated Jacobian of a mechanism holds far more live values than a
thread has registers, so every variant spills; what the build options change
is how the spill traffic, the resident warps that hide its latency and the
launch granularity trade against each other.  Which side wins depends on the
mechanism and the GPU, so it is measured.  The searched grid, per mechanism:

  block        threads per block: 64, 128, 256 (one cell per thread)
  minblocks    register budget through __launch_bounds__(block, minblocks):
               1 (up to 255 registers), 3 (168), 4 (128) at 128 threads;
               also 3 and 4 combined with 64 and 48 shared-memory slots
               (what three or four blocks per SM leave room for)
  smem_spill   part of the spills placed in shared memory by ptxas
               (QSS_SMEM_SPILL; about 100 bytes per thread)
  smem_slots   60, 80 or 100 of the values a register file would reload
               most often (a Belady simulation of the emitted body) kept in
               shared memory by the generated code (dynamic shared memory,
               100 slots = 100 KB a 128-thread block)
  jac_parts    the register-pressure split: one kernel per cell (0), or a
               prefix kernel plus K column-group kernels (2, 4, 8) exchanging
               per-cell values through a frontier buffer (with 60 or 100
               shared-memory slots in each of its kernels as well)
  cells per thread  1 or 2 (cells_per_thread; 2 at 128 threads): each
               thread evaluates two cells, the generated body and its copy
               interleaved line by line (twice the independent work per
               warp, twice the live values)

(A warp-slice per cell, K lanes of a warp cooperating on one cell's DAG, is
not in the grid: on this part an FP64 instruction occupies the FP64 pipe for
the whole warp whatever its active lanes (measured), so lanes that compute
different DAG nodes multiply the FP64 time by K; the column split across
kernels is the register-pressure split that keeps every lane busy.)

Each candidate artefact is built ahead of time (``--build-only``, CPU), then
timed with CUDA events on two batch sizes of the workload's states (65536
cells, the serving size class, and 2^20 cells, the benchmark's batch); per
size bucket the fastest is recorded for (GPU name, mechanism digest) in the
JSON table together with the whole grid's times (a batch takes the choice of
the smallest timed size at or above its cells, else the largest size's).  A
non-default variant must be at least 2 % faster than the default to be
chosen.

    python -m paper_2405_05974_b300.autotune --mech hydrocarbon --build-only
    python -m paper_2405_05974_b300.autotune --mech hydrocarbon --write

``artefact(mech, ncells=...)`` returns the artefact built with the recorded
choice for the current GPU and that batch size (the default build when the
table has no entry); the benchmark and the serving loop load mechanisms
through it.
"""
from __future__ import annotations

import argparse
import json
import os
from typing import Dict, List, Optional

from .qssc.build import build_mechanism, load_meta

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
MIN_GAIN = 0.02      # relative speed-up a non-default variant must show
UNTUNED = ("jac32", "jac32_slots", "jac32_minblocks")   # options outside the searched grid (the mixed kernel)
SIZES = (1 << 16, 1 << 20)


def _digest(mech: dict) -> str:
    from .qssc import mech as qmech
    return qmech.parse(mech).digest


def candidates(key: str) -> List[dict]:
    """The searched build variants of workload `key` (the first is the
    default).  The large mechanism's single-kernel form does not compile in
    reasonable time, so only its partitioned forms are searched."""
    from . import workloads
    base = workloads.build_options(key)
    if base.get("jac_parts", 0) >= 2:
        return [dict(base)] + [{**base, "jac_parts": k} for k in (2, 8) if k != base["jac_parts"]] + \
            [{**base, "block": 64}, {**base, "smem_slots": 60}, {**base, "smem_slots": 100}]
    return [dict(base), {**base, "block": 64}, {**base, "block": 256},
            {**base, "defines": ("QSS_MINBLOCKS=3",)}, {**base, "defines": ("QSS_MINBLOCKS=4",)},
            {**base, "defines": ("QSS_SMEM_SPILL=1",)}, {**base, "smem_slots": 60},
            {**base, "smem_slots": 80}, {**base, "smem_slots": 100},
            # a smaller register budget (more resident warps) with as many
            # shared-memory slots as that many blocks per SM leave room for
            {**base, "defines": ("QSS_MINBLOCKS=3",), "smem_slots": 64},
            {**base, "defines": ("QSS_MINBLOCKS=4",), "smem_slots": 48},
            {**base, "cells_per_thread": 2},
            {**base, "jac_parts": 4}]


def _norm(opts: dict) -> dict:
    o = dict(opts)
    for k in ("defines", "ptxas"):
        if k in o:
            o[k] = list(o[k])
    return o


def load_table(path: str = TABLE) -> Dict[str, dict]:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def _opts(c: dict) -> dict:
    c = dict(c)
    for k in ("defines", "ptxas"):
        if k in c:
            c[k] = tuple(c[k])
    return c


def choice_for(mech: dict, gpu_name: str, table: Optional[dict] = None, ncells: Optional[int] = None) -> dict:
    """Build options recorded for (GPU, mechanism); {} if none.  With
    `ncells`, the choice of the size bucket that batch falls in (the
    smallest timed size >= ncells, else the largest), where the record has
    per-size choices."""
    table = load_table() if table is None else table
    rec = table.get(gpu_name, {}).get(_digest(mech))
    if not rec or "choice" not in rec:
        return {}
    by_size = rec.get("choice_by_size")
    if ncells is not None and by_size:
        sizes = sorted(int(n) for n in by_size)
        n = next((x for x in sizes if x >= ncells), sizes[-1])
        return _opts(by_size[str(n)])
    return _opts(rec["choice"])


def all_choices(mech: dict, gpu_name: str, table: Optional[dict] = None) -> List[dict]:
    """Every distinct choice recorded for (GPU, mechanism), all size buckets."""
    table = load_table() if table is None else table
    rec = table.get(gpu_name, {}).get(_digest(mech)) or {}
    out = []
    for c in [rec.get("choice")] + list((rec.get("choice_by_size") or {}).values()):
        if c is not None and _opts(c) not in out:
            out.append(_opts(c))
    return out


def artefact(mech: dict, gpu_name: Optional[str] = None, defaults: Optional[dict] = None,
             ncells: Optional[int] = None, **build_kw) -> str:
    """The mechanism's artefact with the tuned Jacobian kernel for this GPU:
    the recorded choice (for batches of `ncells` cells, when given), else
    `defaults` (the workload's build options); explicit keyword build
    options override either."""
    if gpu_name is None:
        import torch
        gpu_name = torch.cuda.get_device_name() if torch.cuda.is_available() else ""
    return build_mechanism(mech, **{**tuned_options(mech, gpu_name, defaults, ncells), **build_kw})


def tuned_options(mech: dict, gpu_name: str, defaults: Optional[dict] = None, ncells: Optional[int] = None,
                  table: Optional[dict] = None) -> dict:
    """The recorded choice, else `defaults`; options the tuning does not
    decide (the mixed-precision kernels, jac32) come from `defaults` either
    way."""
    base = dict(defaults or {})
    opts = dict(choice_for(mech, gpu_name, table, ncells=ncells) or base)
    for k in UNTUNED:
        if k in base and k not in opts:
            opts[k] = base[k]
    return opts


def all_tuned_artefacts(mechs: Dict[str, dict], table: Optional[dict] = None):
    """Build every artefact the table selects for any GPU and size bucket
    (ahead of time)."""
    table = load_table() if table is None else table
    return [build_mechanism(m, **c) for gpu in table for m in mechs.values() for c in all_choices(m, gpu, table)]


def time_jacobian(art: str, key: str, ncells: int, reps: int = 5, device: int = 0) -> float:
    """Median milliseconds of one qss_jacobian call over ``ncells`` cells of
    the workload ``key``'s state distribution."""
    import numpy as np
    import torch

    from . import binding, mechgen, workloads
    mech = workloads.mechanism(key)
    gm = binding.Mechanism(art, device)
    rho, T, Y = mechgen.generate_states(mech, workloads.STATES[key], ncells)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    r, t, y = d(rho), d(T), d(Y)
    J = torch.empty((gm.jac_nnz, ncells), dtype=torch.float64, device="cuda")
    w = torch.empty((gm.N, ncells), dtype=torch.float64, device="cuda")
    td = torch.empty(ncells, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    for _ in range(2):
        gm.jacobian(r, t, y, jac=J, wdot=w, Tdot=td, stream=s)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        gm.jacobian(r, t, y, jac=J, wdot=w, Tdot=td, stream=s)
        e1.record(s)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    gm.close()
    del J, w, td, r, t, y
    torch.cuda.empty_cache()
    return float(np.median(ms))


def tune(key: str, sizes=SIZES, device: int = 0) -> dict:
    import torch

    from . import workloads
    mech = workloads.mechanism(key)
    res = []
    for opts in candidates(key):
        art = build_mechanism(mech, **opts)
        meta = load_meta(art)
        k = meta["kernels"]
        jk = "qss_jac_kernel" if "qss_jac_kernel" in k else "qss_jac_prefix_kernel"
        res.append({"opts": _norm(opts), "ms": {str(n): time_jacobian(art, key, n, device=device) for n in sizes},
                    "regs": k[jk].get("regs"), "stack": k[jk].get("stack"), "spill_st": k[jk].get("spill_st")})
    def pick(n):
        best = min(range(len(res)), key=lambda i: res[i]["ms"][n])
        if best != 0 and res[best]["ms"][n] > (1.0 - MIN_GAIN) * res[0]["ms"][n]:
            best = 0
        return res[best]["opts"]

    big = str(max(sizes))
    return {"gpu": torch.cuda.get_device_name(device), "digest": _digest(mech), "name": mech.get("name"),
            "sizes": list(sizes), "choice": pick(big), "choice_by_size": {str(n): pick(str(n)) for n in sizes},
            "candidates": res,
            "rule": f"per size bucket, the fastest at that size (a batch takes the smallest timed size >= its "
                    f"cells, else the largest; 'choice' is the largest size's); a non-default variant must "
                    f"win by {MIN_GAIN:.0%}"}


def build_candidates(keys) -> List[str]:
    """Compile every candidate artefact of the given workloads (CPU)."""
    from concurrent.futures import ThreadPoolExecutor

    from . import workloads
    jobs = [(workloads.mechanism(k), o) for k in keys for o in candidates(k)]
    with ThreadPoolExecutor(4) as ex:
        return [f.result() for f in [ex.submit(build_mechanism, m, **o) for m, o in jobs]]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--mech", action="append", default=None, help="workload key (repeatable)")
    ap.add_argument("--build-only", action="store_true", help="compile the candidates and exit (no GPU)")
    ap.add_argument("--write", action="store_true", help="record the choice in the table")
    ap.add_argument("--table", default=TABLE)
    ap.add_argument("--out", default=None, help="also write the records to this JSON file")
    a = ap.parse_args(argv)
    keys = a.mech or ["hydrocarbon"]
    if a.build_only:
        for p in build_candidates(keys):
            print(p)
        return
    recs = []
    for key in keys:
        rec = tune(key)
        print(json.dumps(rec), flush=True)
        recs.append(rec)
    if a.write:
        table = load_table(a.table)
        for rec in recs:
            table.setdefault(rec["gpu"], {})[rec["digest"]] = {
                k: rec[k] for k in ("name", "choice", "choice_by_size", "sizes", "candidates", "rule")}
        with open(a.table, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(recs, f, indent=1)


if __name__ == "__main__":
    main()
