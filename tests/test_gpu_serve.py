"""Serving loop: continuous batching of implicit-step requests.

Each request's result must not depend on what it was batched with: cells are
independent, so a request served alone, served merged with others, and run
through qss_implicit_step directly must agree bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2405_05974_b300 import binding, mechgen, workloads
from paper_2405_05974_b300.qssc.build import build_mechanism

pytestmark = pytest.mark.gpu

_m = {}


def mech(key):
    if key not in _m:
        m = workloads.mechanism(key)
        # the workload's artefact: the mixed-precision Jacobian beside the FP64 one
        _m[key] = (m, binding.Mechanism(build_mechanism(m, **workloads.build_options(key)), 0))
    return _m[key]


def host_state(key, n, seed):
    m, _ = mech(key)
    cfg = workloads.STATES[key]
    cfg = type(cfg)(**{**cfg.__dict__, "seed": seed})
    rho, T, Y = mechgen.generate_states(m, cfg, n)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    return pin(rho), pin(T), pin(Y)


def clone(state):
    return tuple(x.clone().pin_memory() for x in state)


def direct(key, state, dt, prec):
    _, gm = mech(key)
    r, t, y = (x.cuda() for x in state)
    it, st = gm.implicit_step(r, t, y, dt, precision=prec)
    torch.cuda.synchronize()
    return t.cpu(), y.cpu(), st.cpu()


@pytest.mark.parametrize("prec", [binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR])
def test_same_result_alone_and_in_the_mix(prec):
    _, tiny = mech("tiny")
    _, hc = mech("hydrocarbon")
    probe = host_state("tiny", 777, 11)
    dt = 2e-6
    ref_T, ref_Y, ref_st = direct("tiny", clone(probe), dt, prec)
    srv = binding.Server(0, budget_bytes=2 << 30, n_streams=1, max_batch_cells=1 << 15)
    try:
        alone = clone(probe)
        st_alone = torch.empty(777, dtype=torch.int32).pin_memory()
        rid = srv.submit(tiny, *alone, dt, prec, status=st_alone)
        assert srv.wait(rid) == 0
        # a mix queued behind a long request (one stream): other tiny requests
        # are merged with the probe, hydrocarbon ones form their own batches
        head = host_state("hydrocarbon", 30000, 77)
        ids, keep = [srv.submit(hc, *head, 1e-6, prec)], [head]
        for i in range(6):
            s = host_state("tiny", 300 + 97 * i, 100 + i)
            keep.append(s)
            ids.append(srv.submit(tiny, *s, dt * (1 + i), prec))
            h = host_state("hydrocarbon", 256 + 50 * i, 200 + i)
            keep.append(h)
            ids.append(srv.submit(hc, *h, 1e-6, prec))
            if i == 3:
                mixed = clone(probe)
                st_mixed = torch.empty(777, dtype=torch.int32).pin_memory()
                mid = srv.submit(tiny, *mixed, dt, prec, status=st_mixed)
        for r in ids + [mid]:
            assert srv.wait(r) == 0
        st = srv.stats()
        assert st["completed"] == 15 and st["queued"] == 0
        assert st["batches"] < 10          # queued requests were merged
        assert st["p50_latency_us"] <= st["p99_latency_us"]
    finally:
        srv.close()
    for got_T, got_Y, got_st in ((alone[1], alone[2], st_alone), (mixed[1], mixed[2], st_mixed)):
        # bit for bit (cells that ended non-finite are NaN/inf in both)
        assert np.array_equal(got_T.numpy(), ref_T.numpy(), equal_nan=True)
        assert np.array_equal(got_Y.numpy(), ref_Y.numpy(), equal_nan=True)
        assert torch.equal(got_st, ref_st)


@pytest.mark.parametrize("prec", [binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR, binding.QSS_LU_MIXED])
def test_same_result_with_overlapping_batches(prec):
    """Four streams: batches of three mechanisms run side by side on the
    device (the server reports several in flight at once) while the probe is
    served once early and once in the middle of the burst; both copies equal
    the direct call bit for bit."""
    _, tiny = mech("tiny")
    _, hc = mech("hydrocarbon")
    _, lg = mech("large")
    probe = host_state("hydrocarbon", 1500, 31)
    dt = 1e-8
    ref_T, ref_Y, ref_st = direct("hydrocarbon", clone(probe), dt, prec)
    srv = binding.Server(0, budget_bytes=8 << 30, n_streams=4, max_batch_cells=1 << 14)
    try:
        keep, ids = [], []
        first = clone(probe)
        st_first = torch.empty(1500, dtype=torch.int32).pin_memory()
        ids.append(srv.submit(hc, *first, dt, prec, status=st_first))
        for i in range(12):
            for key, gm, n, dti in (("large", lg, 700 + 31 * i, 1e-9), ("tiny", tiny, 4000 + 97 * i, 1e-6),
                                    ("hydrocarbon", hc, 3000 + 53 * i, 1e-7)):
                s = host_state(key, n, 300 + 10 * i + len(keep))
                keep.append(s)
                ids.append(srv.submit(gm, *s, dti, prec))
            if i == 6:
                mid = clone(probe)
                st_mid = torch.empty(1500, dtype=torch.int32).pin_memory()
                ids.append(srv.submit(hc, *mid, dt, prec, status=st_mid))
        for r in ids:
            assert srv.wait(r) == 0
        st = srv.stats()
        assert st["completed"] == len(ids) and st["queued"] == 0
        assert st["in_flight_peak"] >= 2, st
    finally:
        srv.close()
    for got_T, got_Y, got_st in ((first[1], first[2], st_first), (mid[1], mid[2], st_mid)):
        assert np.array_equal(got_T.numpy(), ref_T.numpy(), equal_nan=True)
        assert np.array_equal(got_Y.numpy(), ref_Y.numpy(), equal_nan=True)
        assert torch.equal(got_st, ref_st)


def test_budget_admission_and_rejection():
    _, hc = mech("hydrocarbon")
    per_cell = 37 * 8 * 4 + 36 * 36 * 8 + 3 * 36 * 8   # io + FP64 scratch, approx
    budget = 64 << 20
    srv = binding.Server(0, budget_bytes=budget, n_streams=4, max_batch_cells=1 << 20)
    try:
        big = host_state("hydrocarbon", (budget // per_cell) * 2, 5)
        with pytest.raises(binding.QSSError) as e:
            srv.submit(hc, *big, 1e-6)
        assert e.value.code == -7
        # many requests that fit only a few at a time: all complete
        reqs = [host_state("hydrocarbon", 2000, 300 + i) for i in range(8)]
        refs = [direct("hydrocarbon", clone(s), 1e-6, binding.QSS_LU_FP64) for s in reqs]
        ids = [srv.submit(hc, *s, 1e-6) for s in reqs]
        for rid in ids:
            assert srv.wait(rid) == 0
        st = srv.stats()
        assert st["bytes_peak"] <= budget and st["rejected"] == 1
        for s, (rT, rY, _) in zip(reqs, refs):
            assert np.array_equal(s[1].numpy(), rT.numpy(), equal_nan=True)
            assert np.array_equal(s[2].numpy(), rY.numpy(), equal_nan=True)
    finally:
        srv.close()


def test_wait_timeout_then_completion():
    _, hc = mech("hydrocarbon")
    srv = binding.Server(0, budget_bytes=4 << 30)
    try:
        s = host_state("hydrocarbon", 60000, 9)
        rid = srv.submit(hc, *s, 1e-6)
        try:
            srv.wait(rid, timeout_us=0)
        except binding.QSSError as e:
            assert e.code == -6
        assert srv.wait(rid) == 0
        with pytest.raises(binding.QSSError):
            srv.wait(rid)            # id released
    finally:
        srv.close()


@pytest.mark.parametrize("prec", [binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR])
def test_graph_replay_matches_direct_launches(prec):
    """The same requests served with graph replay and with direct launches
    give identical results; repeated sizes reuse their bucket's graph, and a
    bucket's graph serves any batch up to its size (the real count is read on
    the device)."""
    sizes = [300, 300, 5000, 257, 511, 1500, 300, 4096]
    results = {}
    for graphs in (True, False):
        srv = binding.Server(0, budget_bytes=2 << 30, n_streams=2, max_batch_cells=1 << 14, graphs=graphs)
        try:
            keep, ids = [], []
            for i, n in enumerate(sizes):
                key = "tiny" if i % 2 == 0 else "hydrocarbon"
                _, gm = mech(key)
                s = host_state(key, n, 500 + i)
                keep.append(s)
                ids.append(srv.submit(gm, *s, 1e-6 * (1 + i % 3), prec))
                assert srv.wait(ids[-1]) == 0      # one at a time: no merging
            st = srv.stats()
        finally:
            srv.close()
        results[graphs] = (keep, st)
    (kg, sg), (kd, sd) = results[True], results[False]
    for a, b in zip(kg, kd):
        assert np.array_equal(a[1].numpy(), b[1].numpy(), equal_nan=True)
        assert np.array_equal(a[2].numpy(), b[2].numpy(), equal_nan=True)
    assert sd["graph_batches"] == 0 and sd["graphs_captured"] == 0
    assert sg["graph_batches"] == len(sizes)
    # buckets used: tiny 512, 8192, 512, 512 and hydrocarbon 512, 2048, 4096 -> 5 graphs
    assert sg["graphs_captured"] == 5, sg


@pytest.mark.parametrize("prec", [binding.QSS_LU_FP64, binding.QSS_LU_MIXED])
def test_graph_replay_partitioned_mechanism(prec):
    """The large mechanism's partitioned Jacobian runs its column groups side
    by side on the handle's streams (forked after the prefix, joined back),
    and a captured graph records them as parallel branches: requests served
    with graph replay, with direct launches and by the direct call give
    identical results."""
    sizes = [300, 700, 300]
    results = {}
    for graphs in (True, False):
        srv = binding.Server(0, budget_bytes=4 << 30, n_streams=2, max_batch_cells=1 << 12, graphs=graphs)
        try:
            keep = []
            for i, n in enumerate(sizes):
                _, gm = mech("large")
                s = host_state("large", n, 900 + i)
                keep.append(s)
                rid = srv.submit(gm, *s, 1e-9, prec)
                assert srv.wait(rid) == 0      # one at a time: no merging
            st = srv.stats()
        finally:
            srv.close()
        results[graphs] = (keep, st)
    (kg, sg), (kd, sd) = results[True], results[False]
    for a, b in zip(kg, kd):
        assert np.array_equal(a[1].numpy(), b[1].numpy(), equal_nan=True)
        assert np.array_equal(a[2].numpy(), b[2].numpy(), equal_nan=True)
    assert sg["graph_batches"] == len(sizes) and sg["graphs_captured"] == 2, sg
    assert sd["graph_batches"] == 0
    # the direct call (the implicit step on the caller's stream) agrees too
    ref_T, ref_Y, _ = direct("large", clone(host_state("large", 300, 900)), 1e-9, prec)
    assert np.array_equal(kg[0][1].numpy(), ref_T.numpy(), equal_nan=True)
    assert np.array_equal(kg[0][2].numpy(), ref_Y.numpy(), equal_nan=True)
