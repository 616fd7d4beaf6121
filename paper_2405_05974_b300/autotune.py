"""Per-GPU tuning of the analytic Jacobian kernel's register budget.

The generated Jacobian of a mechanism holds far more live values than a
thread has registers, so the kernel spills whatever register budget it gets;
the budget only trades spill traffic (local memory, L1/L2) against the number
of resident warps that hide its latency.  Which side wins depends on the
mechanism and the GPU, so it is measured: each candidate blocks-per-SM bound
(``__launch_bounds__(QSS_BLOCK, QSS_MINBLOCKS)``: 1 -> up to 255 registers,
3 -> 168, 4 -> 128 at 128 threads a block) is compiled, timed with CUDA
events on a batch larger than L2, and the fastest is recorded in a JSON table
keyed by GPU name and mechanism digest (a non-default budget must be at least
2% faster than the default to be chosen).

    python -m paper_2405_05974_b300.autotune --mech hydrocarbon --write

``artefact(mech)`` returns the artefact built with the recorded choice for
the current GPU (the default build when the table has no entry).
"""
from __future__ import annotations

import argparse
import json
import os
from typing import Dict, Optional

from .qssc.build import build_mechanism, load_meta

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
CANDIDATES = (1, 3, 4)
MIN_GAIN = 0.02      # relative speed-up a non-default register budget must show


def _digest(mech: dict) -> str:
    from .qssc import mech as qmech
    return qmech.parse(mech).digest


def load_table(path: str = TABLE) -> Dict[str, dict]:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def defines_for(mech: dict, gpu_name: str, table: Optional[dict] = None) -> tuple:
    """Preprocessor definitions recorded for (GPU, mechanism); () if none."""
    table = load_table() if table is None else table
    rec = table.get(gpu_name, {}).get(_digest(mech))
    if not rec or rec.get("minblocks", 1) == 1:
        return ()
    return (f"QSS_MINBLOCKS={int(rec['minblocks'])}",)


def artefact(mech: dict, gpu_name: Optional[str] = None, **build_kw) -> str:
    """The mechanism's artefact with the tuned Jacobian kernel for this GPU."""
    if gpu_name is None:
        import torch
        gpu_name = torch.cuda.get_device_name() if torch.cuda.is_available() else ""
    return build_mechanism(mech, defines=defines_for(mech, gpu_name), **build_kw)


def all_tuned_artefacts(mechs: Dict[str, dict], table: Optional[dict] = None):
    """Build every artefact the table selects for any GPU (ahead of time)."""
    table = load_table() if table is None else table
    out = []
    for gpu in table:
        for m in mechs.values():
            d = defines_for(m, gpu, table)
            if d:
                out.append(build_mechanism(m, defines=d))
    return out


def time_jacobian(art: str, key: str, ncells: int, reps: int = 5, device: int = 0) -> float:
    """Median milliseconds of one qss_jacobian launch over ``ncells`` cells
    of the workload ``key``'s state distribution."""
    import numpy as np
    import torch

    from . import binding, mechgen, workloads
    mech = workloads.mechanism(key)
    scfg = workloads.STATES[key]
    gm = binding.Mechanism(art, device)
    rho, T, Y = mechgen.generate_states(mech, scfg, ncells)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    r, t, y = d(rho), d(T), d(Y)
    n = gm.n
    J = torch.empty((n * n, ncells), dtype=torch.float64, device="cuda")
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


def tune_jacobian(key: str, ncells: int = 1 << 19, candidates=CANDIDATES, device: int = 0) -> dict:
    import torch

    from . import workloads
    mech = workloads.mechanism(key)
    res = {}
    for mb in candidates:
        d = () if mb == 1 else (f"QSS_MINBLOCKS={mb}",)
        art = build_mechanism(mech, defines=d)
        meta = load_meta(art)
        res[mb] = {"ms": time_jacobian(art, key, ncells, device=device),
                   "regs": meta["kernels"]["qss_jac_kernel"].get("regs"),
                   "spill_st": meta["kernels"]["qss_jac_kernel"].get("spill_st")}
    # a non-default budget must win by more than the run-to-run spread
    best = min(res, key=lambda k: res[k]["ms"])
    if best != 1 and res[best]["ms"] > (1.0 - MIN_GAIN) * res[1]["ms"]:
        best = 1
    return {"gpu": torch.cuda.get_device_name(device), "digest": _digest(mech), "name": mech.get("name"),
            "ncells": ncells, "minblocks": best, "candidates": {str(k): v for k, v in res.items()}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--mech", action="append", default=None, help="workload key (repeatable)")
    ap.add_argument("--ncells", type=int, default=1 << 19)
    ap.add_argument("--write", action="store_true", help="record the choice in the table")
    ap.add_argument("--table", default=TABLE)
    ap.add_argument("--out", default=None, help="also write the records to this JSON file")
    a = ap.parse_args(argv)
    recs = []
    for key in a.mech or ["hydrocarbon"]:
        rec = tune_jacobian(key, a.ncells)
        print(json.dumps(rec), flush=True)
        recs.append(rec)
    if a.write:
        table = load_table(a.table)
        for rec in recs:
            table.setdefault(rec["gpu"], {})[rec["digest"]] = {
                k: rec[k] for k in ("name", "minblocks", "ncells", "candidates")}
        with open(a.table, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(recs, f, indent=1)


if __name__ == "__main__":
    main()
