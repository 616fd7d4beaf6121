"""Jacobian variants and the finite-difference Jacobian on the GPU.

* The simplified Jacobians of Section 3.2.1 (constant-QSS, zero-QSS) and the
  finite-difference temperature column of Section 3.2.2, each a build option
  of the mechanism compiler, against the oracle's own implementation of the
  same variant (same gate as the exact Jacobian).
* qss_jacobian_fd (central differences of the source term) against the
  oracle's FD Jacobian, with the running-error bound of the differences.
* The Section 3.2 figures: the relative Frobenius error, Eq. (frobErr), of
  each construction against the FD Jacobian on the paper's sampling protocol,
  and the nonzero fraction of the species block (Table memQSS).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_05974_b300 import analysis, binding, mechgen, workloads
from paper_2405_05974_b300.qssc.build import build_mechanism
from tests.parity import assert_gate

pytestmark = pytest.mark.gpu

VARIANTS = [("const_qss", "analytic"), ("zero_qss", "analytic"), ("exact", "fd")]
_cache = {}


def gpu_mech(key, jac_variant="exact", t_column="analytic"):
    k = (key, jac_variant, t_column)
    if k not in _cache:
        m = workloads.mechanism(key)
        # the exact Jacobian: the workload's own artefact
        kw = workloads.build_options(key) if (jac_variant, t_column) == ("exact", "analytic") else \
            {"jac_variant": jac_variant, "t_column": t_column}
        _cache[k] = binding.Mechanism(build_mechanism(m, **kw), 0)
    return _cache[k]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def paper_states(m, n, seed):
    """Section 3.2.1 protocol: C ~ U[1e-4, 1] mol/m^3, T ~ U[300, 1300] K."""
    rng = np.random.default_rng(seed)
    N = sum(1 for s in m["species"] if not s["qss"])
    C = rng.uniform(1e-4, 1.0, size=(N, n))
    T = rng.uniform(300.0, 1300.0, size=n)
    return mechgen.concentrations_to_state(m, C, T)


@pytest.mark.parametrize("key,ncells", [("tiny", 2048), ("hydrocarbon", 1024)])
@pytest.mark.parametrize("jac_variant,t_column", VARIANTS)
def test_variant_parity(key, ncells, jac_variant, t_column):
    m = workloads.mechanism(key)
    om = oracle.OracleMech(m)
    gm = gpu_mech(key, jac_variant, t_column)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    J, w, td = gm.jacobian(dev(rho), dev(T), dev(Y))
    ref = om.eval_variant(rho, T, Y, jac_variant, t_column)
    eb = om.errbound(rho, T, Y, jac=False)
    assert_gate("wdot", w.cpu().numpy(), ref["wdot"], eb["wdot"])
    assert_gate("Tdot", td.cpu().numpy(), ref["Tdot"], eb["Tdot"])
    r = assert_gate("jac", J.cpu().numpy(), ref["jac"], ref["jac_err"])
    print(key, jac_variant, t_column, r)


@pytest.mark.parametrize("key,ncells", [("tiny", 1000), ("hydrocarbon", 300)])
def test_fd_jacobian_kernel_parity(key, ncells):
    m = workloads.mechanism(key)
    om = oracle.OracleMech(m)
    gm = gpu_mech(key)
    for rho, T, Y in (mechgen.generate_states(m, workloads.STATES[key], ncells),
                      paper_states(m, ncells, 5)):
        for dC, dT in ((1e-4, 1e-4), (1e-6, 1e-2)):
            J = gm.jacobian_fd(dev(rho), dev(T), dev(Y), dC, dT).cpu().numpy()
            ref, err = om.jac_fd_errbound(rho, T, Y, dC, dT)
            assert_gate(f"jac_fd {dC} {dT}", J, ref, err)


def test_fd_jacobian_rejects_bad_steps():
    gm = gpu_mech("tiny")
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    Y = torch.ones((gm.N, 4), dtype=torch.float64, device="cuda")
    for dC, dT in ((0.0, 1.0), (1e-4, -1.0), (float("nan"), 1.0), (1e-4, float("inf"))):
        with pytest.raises(binding.QSSError):
            gm.jacobian_fd(x, x, Y, dC, dT)


@pytest.mark.parametrize("key", ["tiny", "hydrocarbon"])
def test_section3_frobenius_error_and_sparsity(key):
    """Eq. (frobErr) over 100 states of the Section 3.2.1 protocol, FD step
    1e-4: the exact construction is close to the FD Jacobian (the paper's
    Fig. symb_stats: below 1e-5 relative), the simplified ones are not (Tab.
    nosymb_stab_stats: 8-72 %); zero-QSS removes nonzeros of the species block
    relative to constant-QSS, which removes some relative to the exact one
    (Table memQSS)."""
    m = workloads.mechanism(key)
    rho, T, Y = (dev(a) for a in paper_states(m, 100, 11))
    Jfd = gpu_mech(key).jacobian_fd(rho, T, Y, 1e-4, 1e-4)
    eps, nnz = {}, {}
    for v in ("exact", "const_qss", "zero_qss"):
        gm = gpu_mech(key, v)
        J, _, _ = gm.jacobian(rho, T, Y)
        eps[v] = analysis.frobenius_error(J, Jfd)
        nnz[v] = analysis.nonzero_fraction(J, gm.N)
    print(key, "eps_J", eps, "nonzero fraction", nnz)
    assert eps["exact"] < 1e-5
    assert eps["const_qss"] > 1e3 * eps["exact"] and eps["zero_qss"] > 1e3 * eps["exact"]
    assert nnz["exact"] >= nnz["const_qss"] >= nnz["zero_qss"] > 0
