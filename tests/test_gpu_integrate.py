"""qss_integrate (backward-Euler or variable-step BDF2 substeps with local
error control) on the GPU against the oracle's integrator.

Both run the same controller; a substep decision (accept/reject, err <= 1)
can flip where err is within rounding of 1, after which the two substep
sequences differ (both valid).  So: most cells take the same number of
substeps with the same outcome, and on those the final states agree within
the accumulated Newton tolerance (each substep's solution is pinned to the
oracle's within 1e-10 relative for FP64 LU, 1e-8 for FP32 LU + refinement).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_05974_b300 import binding, mechgen, workloads
from paper_2405_05974_b300.qssc.build import build_mechanism

pytestmark = pytest.mark.gpu
OPTS = dict(rtol=1e-3, atol_C=1e-6, atol_T=1e-3)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("key,ncells,D", [("tiny", 512, 1e-7), ("hydrocarbon", 64, 1e-8), ("large", 32, 1e-10)])
@pytest.mark.parametrize("prec", [binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR])
def test_integrate_matches_oracle(key, ncells, D, prec, order):
    m = workloads.mechanism(key)
    om = oracle.OracleMech(m)
    gm = binding.Mechanism(build_mechanism(m, **workloads.build_options(key)), 0)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    t, y = dev(T), dev(Y)
    ns, st = gm.integrate(dev(rho), t, y, D, precision=prec, opts=binding.integrate_opts(**OPTS, order=order))
    ns, st = ns.cpu().numpy(), st.cpu().numpy()
    To, Yo, nso, sto = om.integrate(rho, T, Y, D, order=order, **OPTS)
    same = (st == sto) & (ns == nso)
    assert same.mean() >= 0.9, (np.bincount(st, minlength=3), np.bincount(sto, minlength=3))
    done = same & (st == 0)
    assert done.mean() >= 0.7
    W = om.W[:, None]
    pg = np.vstack([rho[None] * y.cpu().numpy() / W, t.cpu().numpy()[None]])[:, done]
    po = np.vstack([rho[None] * Yo / W, To[None]])[:, done]
    rel = 1e-8 if prec == binding.QSS_LU_FP64 else 1e-6
    atol = np.r_[np.full(om.N, 1e-12), 1e-8][:, None]
    ok = np.abs(pg - po) <= rel * np.abs(po) + atol
    assert ok.all(axis=0).mean() >= 0.99, np.argwhere(~ok)[:5]


def test_integrate_rejects_bad_options():
    m = workloads.mechanism("tiny")
    gm = binding.Mechanism(build_mechanism(m), 0)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["tiny"], 64)
    for bad in (dict(atol_C=0.0), dict(h_min=0.0), dict(max_rounds=0), dict(rtol=-1.0), dict(order=3),
                dict(order=0)):
        with pytest.raises(binding.QSSError):
            gm.integrate(dev(rho), dev(T), dev(Y), 1e-7, opts=binding.integrate_opts(**bad))


def test_integrate_reaches_where_one_step_fails():
    """Cells whose single backward-Euler step over the interval does not
    converge reach the end of it by substeps."""
    key, ncells, D = "tiny", 512, 1e-7
    m = workloads.mechanism(key)
    gm = binding.Mechanism(build_mechanism(m), 0)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    t1, y1 = dev(T), dev(Y)
    _, st1 = gm.implicit_step(dev(rho), t1, y1, D * 10)
    t2, y2 = dev(T), dev(Y)
    _, st2 = gm.integrate(dev(rho), t2, y2, D * 10, opts=binding.integrate_opts(**OPTS))
    st1, st2 = st1.cpu().numpy(), st2.cpu().numpy()
    rescued = (st1 != 0) & (st2 == 0)
    assert rescued.sum() > 0, (np.bincount(st1), np.bincount(st2, minlength=3))


def test_bdf2_needs_fewer_substeps():
    """At the same tolerance the second-order substeps cover the interval in
    far fewer substeps (the oracle's pins fix the order of accuracy)."""
    key, ncells, D = "tiny", 512, 1e-7
    m = workloads.mechanism(key)
    gm = binding.Mechanism(build_mechanism(m), 0)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    res = {}
    for order in (1, 2):
        ns, st = gm.integrate(dev(rho), dev(T), dev(Y), D, opts=binding.integrate_opts(
            rtol=1e-5, atol_C=1e-8, atol_T=1e-5, order=order, max_rounds=4000))
        res[order] = (ns.cpu().numpy(), st.cpu().numpy())
    both = (res[1][1] == 0) & (res[2][1] == 0)
    assert both.mean() > 0.5
    assert np.median(res[2][0][both]) * 2 < np.median(res[1][0][both]), (
        np.median(res[1][0][both]), np.median(res[2][0][both]))


@pytest.mark.parametrize("order", [1, 2])
def test_integrate_per_cell_intervals_and_ragged_tail(order):
    """Per-cell intervals (dt_stride 1), ncells < ld: the tail columns are
    untouched, and the integrated cells follow the oracle's integrator."""
    key = "tiny"
    m = workloads.mechanism(key)
    om = oracle.OracleMech(m)
    gm = binding.Mechanism(build_mechanism(m), 0)
    ld, ncells = 600, 600 - 17
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells, ld=ld)
    D = np.exp(np.random.default_rng(9).uniform(np.log(1e-9), np.log(1e-7), ld))
    t, y = dev(T), dev(Y)
    ns = torch.full((ld,), -5, dtype=torch.int32, device="cuda")
    st = torch.full((ld,), -5, dtype=torch.int32, device="cuda")
    gm.integrate(dev(rho), t, y, dev(D), precision=binding.QSS_LU_FP64, ncells=ncells, nsteps=ns, status=st,
                 opts=binding.integrate_opts(**OPTS, order=order))
    t, y, ns, st = t.cpu().numpy(), y.cpu().numpy(), ns.cpu().numpy(), st.cpu().numpy()
    assert (ns[ncells:] == -5).all() and (st[ncells:] == -5).all()
    assert np.array_equal(t[ncells:], T[ncells:]) and np.array_equal(y[:, ncells:], Y[:, ncells:])
    To, Yo, nso, sto = om.integrate(rho[:ncells], T[:ncells], Y[:, :ncells], D[:ncells], order=order, **OPTS)
    same = (st[:ncells] == sto) & (ns[:ncells] == nso)
    assert same.mean() >= 0.9
    done = same & (sto == 0)
    assert done.mean() >= 0.7
    W = om.W[:, None]
    pg = np.vstack([rho[None, :ncells] * y[:, :ncells] / W, t[None, :ncells]])[:, done]
    po = np.vstack([rho[None, :ncells] * Yo / W, To[None]])[:, done]
    atol = np.r_[np.full(om.N, 1e-12), 1e-8][:, None]
    ok = np.abs(pg - po) <= 1e-8 * np.abs(po) + atol
    assert ok.all(axis=0).mean() >= 0.99
