"""GPU implicit (backward-Euler) step against the CPU oracle's step.

The oracle and both GPU forms run the same algorithm (Newton on
G = phi - phi0 - dt f with I - dt J, the analytic J re-evaluated every
iteration, the weighted-RMS stopping rule).  Two converged Newton iterates
differ by at most the sum of their last updates, which the stopping rule
bounds by rtol |phi_i| + atol_i each, plus rounding noise; the gates below
are that bound with margin:
  FP64 LU     vs oracle:   |d phi_i| <= 1e-10 |phi_i| + 10 atol_i
  FP32 LU+IR  vs FP64 LU:  |d phi_i| <= 1e-8  |phi_i| + 10 atol_i
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2405_05974_b300 import binding, mechgen, workloads
from paper_2405_05974_b300.qssc.build import build_mechanism
from tests import mechs as hm

pytestmark = pytest.mark.gpu

ATOL_C, ATOL_T, RTOL = 1e-20, 1e-10, 1e-12
_cache = {}


def mech(key):
    if key not in _cache:
        m = workloads.mechanism(key)
        _cache[key] = (m, binding.Mechanism(build_mechanism(m, **workloads.build_options(key)), 0), oracle.OracleMech(m))
    return _cache[key]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_step(gm, rho, T, Y, dt, precision, ncells=None, opts=None):
    r, t, y = dev(rho), dev(T), dev(Y)
    dtt = dev(np.atleast_1d(np.asarray(dt, dtype=np.float64)))
    it, st = gm.implicit_step(r, t, y, dtt, precision=precision, ncells=ncells, opts=opts)
    torch.cuda.synchronize()
    return t.cpu().numpy(), y.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()


def phi_of(om, rho, T, Y):
    return np.vstack([om.conc(rho, Y), T[None, :]])


def close(pa, pb, rel, N):
    atol = np.r_[np.full(N, ATOL_C), ATOL_T][:, None]
    return np.abs(pa - pb) <= rel * np.abs(pb) + 10 * atol


@pytest.mark.parametrize("key,ncells,dt,min_conv", [("tiny", 4096, workloads.IMPLICIT_DT, 0.25),
                                                    ("hydrocarbon", 1024, workloads.IMPLICIT_DT, 0.25),
                                                    ("hydrocarbon", 2048, workloads.IMPLICIT_DT_CONVERGING, 0.95),
                                                    ("large", 512, 1e-9, 0.25),
                                                    ("large", 1024, 1e-12, 0.95)])
def test_implicit_step_parity(key, ncells, dt, min_conv):
    """Converged cells against the oracle's step.  At the configured step
    (1e-6 s; the large mechanism at 1e-9 s) plain Newton from phi0 converges
    in only part of the synthetic cells; at 1e-11 s (hydrocarbon) and 1e-12 s
    (large) it converges in >= 95 % of them, so the comparison covers nearly
    every cell."""
    m, gm, om = mech(key)
    st_cfg = workloads.STATES["implicit"] if key == "hydrocarbon" else workloads.STATES[key]
    rho, T, Y = mechgen.generate_states(m, st_cfg, ncells)
    To, Yo, ito, sto = om.be_step(rho, T, Y, dt, max_iter=20)
    T64, Y64, it64, st64 = gpu_step(gm, rho, T, Y, dt, binding.QSS_LU_FP64)
    T32, Y32, it32, st32 = gpu_step(gm, rho, T, Y, dt, binding.QSS_LU_FP32_IR)
    N = gm.N
    both = (sto == 0) & (st64 == 0)
    assert both.sum() >= min_conv * ncells, (np.bincount(sto), np.bincount(st64))
    # the same cells converge (Newton paths only differ by rounding)
    agree = np.mean((sto == 0) == (st64 == 0))
    assert agree >= 0.97, agree
    po, p64, p32 = phi_of(om, rho, To, Yo), phi_of(om, rho, T64, Y64), phi_of(om, rho, T32, Y32)
    ok = close(p64[:, both], po[:, both], 1e-10, N)
    assert ok.all(), np.argwhere(~ok)[:5]
    both32 = (st32 == 0) & (st64 == 0)
    assert np.mean((st32 == 0) == (st64 == 0)) >= 0.97
    ok = close(p32[:, both32], p64[:, both32], 1e-8, N)
    assert ok.all(), np.argwhere(~ok)[:5]
    # iteration counts follow the oracle's
    assert np.mean(np.abs(it64[both].astype(int) - ito[both]) <= 1) >= 0.95
    # mass: sum_k Y_k is unchanged by a converged step (rho fixed)
    assert np.allclose(Y64[:, both].sum(0), Y[:, both].sum(0), rtol=1e-11, atol=0)
    print(key, "oracle", np.bincount(sto, minlength=4), "fp64", np.bincount(st64, minlength=4),
          "fp32ir", np.bincount(st32, minlength=4), "iters fp64 mean %.2f fp32ir %.2f" %
          (it64[st64 == 0].mean(), it32[st32 == 0].mean()))


@pytest.mark.parametrize("key,ncells,dt_lo,dt_hi", [("tiny", 2048, 1e-5, 1e-2),
                                                    ("hydrocarbon", 1024, 1e-7, 1e-4)])
def test_implicit_step_large_dt(key, ncells, dt_lo, dt_hi):
    """Steps up to 1e-2 s (tiny) and 1e-4 s (hydrocarbon; at larger steps few of
    its cells converge) make M = I - dt J far from diagonally dominant, so the
    eliminations exchange rows; converged cells still match the oracle's step
    (its own partial-pivoting LU) within the same gates."""
    m, gm, om = mech(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    dts = np.exp(np.random.default_rng(11).uniform(np.log(dt_lo), np.log(dt_hi), ncells))
    To, Yo, ito, sto = om.be_step(rho, T, Y, dts, max_iter=20)
    N = gm.N
    po = phi_of(om, rho, To, Yo)
    res = {}
    for prec in (binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR):
        T1, Y1, it, st = gpu_step(gm, rho, T, Y, dts, prec)
        both = (sto == 0) & (st == 0)
        assert both.sum() >= 0.1 * ncells, (np.bincount(sto, minlength=4), np.bincount(st, minlength=4))
        fp64 = prec == binding.QSS_LU_FP64
        # the FP32 factors may stop refining on the worst-conditioned matrices,
        # so the converged sets may differ a little more there
        assert np.mean((sto == 0) == (st == 0)) >= (0.9 if fp64 else 0.8)
        rel = 1e-10 if fp64 else 1e-8
        p1 = phi_of(om, rho, T1, Y1)
        ok = close(p1[:, both], po[:, both], rel, N)
        assert ok.all(), np.argwhere(~ok)[:5]
        res[prec] = np.bincount(st, minlength=4)
    print(key, "oracle", np.bincount(sto, minlength=4), res)


def test_linear_closed_form():
    """A <=> B with Tdot = 0: the step is the 2x2 linear solve (Newton reaches it
    in one update, the second confirms)."""
    T0 = 1300.0
    sp = [hm.species("A", {"C": 1, "H": 2, "O": 1}, nasa=[1.0, 0, 0, 0, 0, 0, 0.0]),
          hm.species("B", {"C": 1, "H": 2, "O": 1}, nasa=[1.0, 0, 0, 0, 0, 0, -0.4]),
          hm.species("N2", {"N": 2})]
    mm = hm.mech("ab_lin", sp, [hm.reaction({"A": 1}, {"B": 1}, 2.0e6)])
    gm = binding.Mechanism(build_mechanism(mm), 0)
    CA0, CB0 = 1.5, 0.25
    rho, T, Y = mechgen.concentrations_to_state(mm, np.array([[CA0], [CB0], [1.0]]), np.array([T0]))
    dt = 3e-7
    kf, kb = 2.0e6, 2.0e6 / math.exp(-0.4)
    CA = ((1 + dt * kb) * CA0 + dt * kb * CB0) / (1 + dt * kf + dt * kb)
    W = np.array([s["W"] for s in mm["species"]])
    for prec in (binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR):
        T1, Y1, it, st = gpu_step(gm, rho, T, Y, dt, prec)
        C1 = rho * Y1[:, 0] / W
        assert st[0] == 0 and it[0] <= 2
        assert C1[0] == pytest.approx(CA, rel=1e-13)
        assert C1[1] == pytest.approx(CA0 + CB0 - CA, rel=1e-13)
        assert T1[0] == pytest.approx(T0, rel=1e-15)


def test_per_cell_dt_and_ragged_tail():
    key = "tiny"
    m, gm, om = mech(key)
    ncells, ld = 1000 - 13, 1000
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells, ld=ld)
    dts = np.exp(np.random.default_rng(2).uniform(np.log(1e-7), np.log(1e-5), ld))
    r, t, y = dev(rho), dev(T), dev(Y)
    it = torch.full((ld,), -7, dtype=torch.int32, device="cuda")
    st = torch.full((ld,), -7, dtype=torch.int32, device="cuda")
    gm.implicit_step(r, t, y, dev(dts), precision=binding.QSS_LU_FP64, ncells=ncells, iters=it, status=st)
    torch.cuda.synchronize()
    t, y, it, st = t.cpu().numpy(), y.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    assert (it[ncells:] == -7).all() and (st[ncells:] == -7).all()
    assert np.array_equal(t[ncells:], T[ncells:]) and np.array_equal(y[:, ncells:], Y[:, ncells:])
    To, Yo, ito, sto = om.be_step(rho, T, Y, dts, ncells=ncells, max_iter=20)
    both = (sto[:ncells] == 0) & (st[:ncells] == 0)
    assert both.mean() > 0.5
    p, po = phi_of(om, rho, t, y)[:, :ncells], phi_of(om, rho, To, Yo)[:, :ncells]
    assert close(p[:, both], po[:, both], 1e-10, gm.N).all()


def test_empty_and_bad_arguments():
    _, gm, _ = mech("tiny")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    Y = torch.zeros((gm.N, 8), dtype=torch.float64, device="cuda")
    L = binding.lib()
    assert L.qss_implicit_step(gm.h, 0, 8, x.data_ptr(), 0, x.data_ptr(), x.data_ptr(), Y.data_ptr(),
                               0, None, None, None, None) == 0
    assert L.qss_implicit_step(gm.h, 9, 8, x.data_ptr(), 0, x.data_ptr(), x.data_ptr(), Y.data_ptr(),
                               0, None, None, None, None) == -1
    assert L.qss_implicit_step(gm.h, 8, 8, x.data_ptr(), 0, x.data_ptr(), x.data_ptr(), Y.data_ptr(),
                               7, None, None, None, None) == -1


def test_fp32ir_reports_no_status_fp64_does_not():
    """The mixed form falls back to the FP64 solve for a cell whose FP32
    factorisation fails, so it never ends a cell SINGULAR where the FP64 form
    does not, and its statuses follow the FP64 form's."""
    m, gm, om = mech("hydrocarbon")
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["implicit"], 8192)
    _, _, _, st64 = gpu_step(gm, rho, T, Y, workloads.IMPLICIT_DT, binding.QSS_LU_FP64)
    _, _, _, st32 = gpu_step(gm, rho, T, Y, workloads.IMPLICIT_DT, binding.QSS_LU_FP32_IR)
    assert not np.any((st32 == 3) & (st64 != 3)), np.bincount(st32, minlength=4)
    assert np.mean(st32 == st64) >= 0.97, (np.bincount(st64, minlength=4), np.bincount(st32, minlength=4))


def test_small_newton_scratch_limit_same_results():
    """A Newton scratch limit of 2 MB (the 3000-cell batch then runs in chunks
    of 160 cells instead of one) changes nothing in the results."""
    m, gm, om = mech("hydrocarbon")
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["implicit"], 3000)
    ref = gpu_step(gm, rho, T, Y, 1e-8, binding.QSS_LU_FP64)
    try:
        gm.set_newton_bytes(2 << 20)
        got = gpu_step(gm, rho, T, Y, 1e-8, binding.QSS_LU_FP64)
    finally:
        gm.set_newton_bytes(4 << 30)
    assert np.array_equal(got[3], ref[3]) and np.array_equal(got[2], ref[2])
    fin = ref[3] != 2
    assert np.array_equal(got[0][fin], ref[0][fin]) and np.array_equal(got[1][:, fin], ref[1][:, fin])


@pytest.mark.parametrize("key,ncells,dt,min_ratio", [("tiny", 4096, workloads.IMPLICIT_DT, 0.9),
                                                     ("hydrocarbon", 2048, workloads.IMPLICIT_DT_CONVERGING, 0.95),
                                                     ("hydrocarbon", 2048, 1e-8, 0.9),
                                                     ("large", 512, 1e-12, 0.95)])
def test_jacobian_reuse_reaches_the_same_state(key, ncells, dt, min_ratio):
    """Keeping a cell's Jacobian while its Newton update contracts
    (jac_reuse = 1, at most 40 iterations; only f is evaluated in those
    iterations) changes the iteration, not the solution: the cells that
    converge with full Newton and with reuse agree within 1e-8 relative + 10
    atol (all but a few per cent, which must be roots of the backward-Euler
    system by the oracle's f: the system can have several)
    (the iterations that keep J take f from the source-term kernel, whose
    emitted arithmetic rounds differently from the Jacobian kernel's f, so the
    roots differ by rounding, as between the FP32-IR and FP64 forms), for
    both precisions; reuse converges nearly as many cells (95 % of full
    Newton's count at the step sizes where plain Newton converges almost
    everywhere, 90 % at the larger ones, where frozen Jacobians need more
    iterations).  The large mechanism exercises the partitioned Jacobian and
    its frontier next to the kept Jacobians."""
    m, gm, om = mech(key)
    st_cfg = workloads.STATES["implicit"] if key == "hydrocarbon" else workloads.STATES[key]
    rho, T, Y = mechgen.generate_states(m, st_cfg, ncells)
    reuse = binding.newton_opts(jac_reuse=1)
    for prec in (binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR):
        Tf, Yf, itf, stf = gpu_step(gm, rho, T, Y, dt, prec)
        Tr, Yr, itr, str_ = gpu_step(gm, rho, T, Y, dt, prec, opts=reuse)
        both = (stf == 0) & (str_ == 0)
        assert (str_ == 0).sum() >= min_ratio * (stf == 0).sum(), (np.bincount(stf, minlength=4),
                                                                  np.bincount(str_, minlength=4))
        pf, pr = phi_of(om, rho, Tf, Yf), phi_of(om, rho, Tr, Yr)
        ok = close(pr[:, both], pf[:, both], 1e-8, gm.N).all(axis=0)
        # the backward-Euler system of these stiff states can have more than
        # one root, and iterations whose paths differ can end on different
        # ones: at most 5 % of the cells (1.7 % at 1e-8 s, 0.1 % at 1e-11 s
        # measured), and each such state must be a root of
        # G(phi) = phi - phi0 - dt f(phi) by the oracle's f
        assert ok.mean() >= 0.95, (ok.mean(), np.nonzero(~ok)[0][:8])
        cells = np.nonzero(both)[0][~ok]
        if cells.size:
            phi0 = phi_of(om, rho, T, Y)[:, cells]
            for p_ in (pf[:, cells], pr[:, cells]):
                f, _ = om.eval_phi(np.ascontiguousarray(p_), jac=False, strict=False)
                G = p_ - phi0 - dt * f
                scale = np.abs(p_) + np.abs(phi0) + dt * np.abs(f)
                assert np.all(np.abs(G) <= 1e-8 * scale.max(axis=0)), cells
        print(key, dt, prec, "converged full %d reuse %d" % ((stf == 0).sum(), (str_ == 0).sum()),
              "different roots %d" % cells.size,
              "full iters %.2f" % itf[stf == 0].mean(), "reuse iters %.2f" % itr[str_ == 0].mean())
