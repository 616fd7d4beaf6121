"""GPU: the mixed-precision Jacobian (qss_jacobian_mixed) and the implicit
step that uses it (QSS_LU_MIXED), against the oracle and the FP64 forms.

qss_jacobian_mixed evaluates the source term in FP64 and the Jacobian's
derivative terms in FP32 (one kernel, or for the large mechanism a prefix
kernel and column-group kernels).  Gates:
  wdot, Tdot: the FP64 parity gate (tests/parity.py) against the oracle;
  J: |J - J_oracle| <= 2^29 e_ref + 1e-20 per entry, e_ref the oracle's FP64
     running-error bound: 2^29 = u_32 / u_64 turns it into the first-order
     rounding bound of the same evaluation carried out in FP32.
The mixed implicit step is Newton with an FP32-assembled matrix and the FP64
residual, so a converged cell meets the same stopping rule as the FP64 step:
  mixed vs FP64 step: |d phi_i| <= 1e-8 |phi_i| + 10 atol_i
  mixed vs oracle:    |d phi_i| <= 1e-10 |phi_i| + 10 atol_i
on the cells both converge on.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_05974_b300 import binding, mechgen, workloads
from paper_2405_05974_b300.qssc.build import build_mechanism
from tests.parity import assert_gate

pytestmark = pytest.mark.gpu

ATOL_C, ATOL_T = 1e-20, 1e-10
_cache = {}


def mech(key):
    if key not in _cache:
        m = workloads.mechanism(key)
        art = build_mechanism(m, **{**workloads.build_options(key), "jac32": True})
        _cache[key] = (m, binding.Mechanism(art, 0), oracle.OracleMech(m))
    return _cache[key]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def states(key, ncells):
    m = workloads.mechanism(key)
    return mechgen.generate_states(m, workloads.STATES["implicit" if key == "hydrocarbon" else key], ncells)


@pytest.mark.parametrize("key,ncells", [("tiny", 4096), ("tiny", 1003), ("hydrocarbon", 2048),
                                        ("hydrocarbon", 517), ("large", 300)])
def test_mixed_jacobian_against_oracle(key, ncells):
    m, gm, om = mech(key)
    rho, T, Y = states(key, ncells)
    ld = ncells + 5   # ragged: ld > ncells
    pad = lambda a: np.concatenate([a, np.repeat(a[..., -1:], ld - ncells, axis=-1)], axis=-1)  # noqa: E731
    J, w, td = gm.jacobian(dev(pad(rho)), dev(pad(T)), dev(pad(Y)), ncells=ncells, mixed=True)
    torch.cuda.synchronize()
    J, w, td = J.cpu().numpy()[:, :ncells], w.cpu().numpy()[:, :ncells], td.cpu().numpy()[:ncells]
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    assert_gate("wdot", w, ref["wdot"], eb["wdot"])
    assert_gate("Tdot", td, ref["Tdot"], eb["Tdot"])
    assert np.all(np.isfinite(J))
    err = np.abs(J - ref["jac"])
    bound = 2.0 ** 29 * eb["jac"] + 1e-20
    assert np.all(err <= bound), float(np.max(err / bound))
    # and the FP64 kernel of the same artefact stays what it was
    J64, _, _ = gm.jacobian(dev(rho), dev(T), dev(Y))
    torch.cuda.synchronize()
    assert_gate("jac", J64.cpu().numpy(), ref["jac"], eb["jac"])


def _step(gm, rho, T, Y, dt, precision):
    t, y = dev(T), dev(Y)
    it, st = gm.implicit_step(dev(rho), t, y, dev(np.atleast_1d(dt)), precision=precision)
    torch.cuda.synchronize()
    return t.cpu().numpy(), y.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()


def _phi(om, rho, T, Y):
    return np.vstack([om.conc(rho, Y), T[None, :]])


def _close(pa, pb, rel, N):
    atol = np.r_[np.full(N, ATOL_C), ATOL_T][:, None]
    return np.abs(pa - pb) <= rel * np.abs(pb) + 10 * atol


@pytest.mark.parametrize("key,ncells,dt,min_conv", [("tiny", 4096, 1e-7, 0.9),
                                                    ("tiny", 2000, workloads.IMPLICIT_DT, 0.25),
                                                    ("hydrocarbon", 2048, workloads.IMPLICIT_DT_CONVERGING, 0.95),
                                                    ("hydrocarbon", 1024, workloads.IMPLICIT_DT, 0.25),
                                                    ("large", 512, 1e-12, 0.9)])
def test_mixed_implicit_step(key, ncells, dt, min_conv):
    m, gm, om = mech(key)
    rho, T, Y = states(key, ncells)
    Ta, Ya, ita, sta = _step(gm, rho, T, Y, dt, binding.QSS_LU_FP64)
    Tm, Ym, itm, stm = _step(gm, rho, T, Y, dt, binding.QSS_LU_MIXED)
    N = gm.N
    # about as many cells converge as with the exact FP64 Jacobian
    assert (stm == 0).mean() >= min_conv, np.bincount(stm)
    assert (stm == 0).sum() >= 0.97 * (sta == 0).sum(), (np.bincount(sta), np.bincount(stm))
    both = (sta == 0) & (stm == 0)
    pa, pm = _phi(om, rho, Ta, Ya), _phi(om, rho, Tm, Ym)
    ok = _close(pm[:, both], pa[:, both], 1e-8, N).all(0)
    # where the two differ beyond the gate, both must be roots of the same
    # backward-Euler system (stiff states can have several; the Newton path
    # picks one): the oracle's residual check at the mixed result
    bad = np.nonzero(both)[0][~ok]
    assert bad.size <= max(2, 0.002 * both.sum()), bad.size
    if bad.size:
        f, _ = om.eval_phi(pm[:, bad], jac=False)
        G = pm[:, bad] - _phi(om, rho[bad], T[bad], Y[:, bad]) - dt * f
        scale = 1e-10 * np.abs(pm[:, bad]) + 10 * np.r_[np.full(N, ATOL_C), ATOL_T][:, None] + \
            1e-12 * dt * np.abs(f)
        assert np.all(np.abs(G) <= 1e3 * scale)
    # against the oracle's step, on the cells both converge on
    To, Yo, ito, sto = om.be_step(rho, T, Y, dt, max_iter=20)
    bo = (sto == 0) & (stm == 0) & np.isin(np.arange(ncells), np.nonzero(both)[0][ok]) & (sta == 0)
    po = _phi(om, rho, To, Yo)
    okp = _close(pm[:, bo], po[:, bo], 1e-10, N).all(0)
    assert okp.mean() >= 0.998, okp.mean()
