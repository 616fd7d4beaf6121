"""Parity gate between the CUDA path and the CPU oracle.

An output x_gpu passes against the oracle's x_ref when

    |x_gpu - x_ref| <= 1e-10 |x_ref| + 1e-20 + K * e_ref

where e_ref is the oracle's first-order rounding-error bound for that output
(running error analysis in the oracle; pinned against binary128 by
tests/test_oracle_pins.py) and K = 16.  The first two terms are the stated
per-entry target (relative 1e-10, absolute floor 1e-20).  The third term
covers entries whose terms cancel: two correct FP64 evaluations of such an
entry differ by up to the sum of their rounding errors, and the CUDA path
evaluates the same expressions in a different order (and with its own
exp/log implementations), so its error is bounded by a small multiple of the
oracle's bound.  Every report states how many entries needed the third term.
"""
from __future__ import annotations

import numpy as np

REL = 1e-10
ABS = 1e-20
K_BOUND = 16.0


def gate(x, ref, bound, rel=REL, abs_floor=ABS, k=K_BOUND):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    bound = np.asarray(bound, dtype=np.float64)
    err = np.abs(x - ref)
    tol_rel = rel * np.abs(ref) + abs_floor
    ok = err <= tol_rel + k * bound
    ok &= np.isfinite(x)
    ok_rel = err <= tol_rel
    n = ok.size
    worst = float(np.max(err / (tol_rel + k * bound))) if n else 0.0
    return {"ok": bool(ok.all()), "n": int(n), "n_fail": int((~ok).sum()),
            "n_needed_bound": int((ok & ~ok_rel).sum()), "worst_ratio": worst,
            "max_rel_err": float(np.max(err / np.maximum(np.abs(ref), 1e-300))) if n else 0.0,
            "fail_idx": np.argwhere(~ok)[:5].tolist()}


def assert_gate(name, x, ref, bound, **kw):
    r = gate(x, ref, bound, **kw)
    assert r["ok"], f"{name}: {r}"
    return r


def assert_gate_exact(name, x, ref, bound, q128_of_cells, rel=REL, abs_floor=ABS, k=K_BOUND):
    """The gate, and for every entry that passes only through the rounding
    allowance K e_ref (its terms cancel) a second judgement against the
    oracle's binary128 rerun of the same cell: the GPU value must lie within
    rel |x_q| + abs_floor + K e_ref of the exact value x_q as well, i.e. it is
    close to the exact result and not only to the FP64 oracle's.  Reports
    how many entries needed the allowance, how many of them are within the
    plain target of the binary128 value, and the largest relative distance.
    q128_of_cells(cells) returns the binary128 result of those cells (cells
    on the last axis, as in x)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    bound = np.asarray(bound, dtype=np.float64)
    r = gate(x, ref, bound, rel=rel, abs_floor=abs_floor, k=k)
    assert r["ok"], f"{name}: {r}"
    err = np.abs(x - ref)
    needed = err > rel * np.abs(ref) + abs_floor
    r["q128_checked"] = int(needed.sum())
    if needed.any():
        cells = np.unique(np.nonzero(needed)[-1])
        q = np.asarray(q128_of_cells(cells), dtype=np.float64)
        sub = needed[..., cells]
        xv, qv, bv = x[..., cells][sub], q[sub], bound[..., cells][sub]
        eq = np.abs(xv - qv)
        ok_q = eq <= rel * np.abs(qv) + abs_floor + k * bv
        r["q128_within_target"] = int((eq <= rel * np.abs(qv) + abs_floor).sum())
        r["q128_max_rel"] = float(np.max(eq / np.maximum(np.abs(qv), 1e-300)))
        r["q128_fail"] = int((~ok_q).sum())
        assert ok_q.all(), f"{name}: entries that needed the rounding allowance are not close to the binary128 value: {r}"
    return r
