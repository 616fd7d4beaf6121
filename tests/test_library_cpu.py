"""CPU-side checks of the boundary and the mechanism compiler (no GPU)."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import oracle
from paper_2405_05974_b300 import binding, build_ext, mechgen, workloads
from paper_2405_05974_b300.qssc import build as qbuild
from paper_2405_05974_b300.qssc import graph as qgraph
from paper_2405_05974_b300.qssc import mech as qmech
from paper_2405_05974_b300.qssc import model as qmodel
from tests import mechs as hm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(qss_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    build_ext.build()
    L = ctypes.CDLL(binding.LIB_PATH)
    names = _declared_functions()
    assert len(names) >= 9
    for nm in names:
        assert hasattr(L, nm), nm


def test_calls_without_driver_report_errors():
    L = binding.lib()
    h = ctypes.c_void_p()
    rc = L.qss_mech_load(b"/nonexistent", 0, ctypes.byref(h))
    assert rc == -2
    art = qbuild.build_mechanism(workloads.mechanism("tiny"))
    rc = L.qss_mech_load(art.encode(), 0, ctypes.byref(h))
    assert rc in (-3, 0)   # no driver on a CPU-only machine
    if rc:
        assert L.qss_last_error()
    assert L.qss_wdot(None, 1, 1, None, None, None, None, None, None) == -1


def test_compiler_tarjan_fig2():
    g = json.load(open(os.path.join(GOLDEN, "tarjan_fig2.json")))
    names = sorted({v for e in g["edges_as_drawn"] for v in e})
    ix = {nm: i for i, nm in enumerate(names)}
    adj = [[] for _ in names]
    for a, b in g["edges_as_drawn"]:
        adj[ix[a]].append(ix[b])
    comps = qgraph.tarjan_scc(adj)
    assert sorted(sorted(names[v] for v in c) for c in comps) == sorted(sorted(c) for c in g["expected_sccs"])
    pos = {v: ci for ci, c in enumerate(comps) for v in c}
    for u, nb in enumerate(adj):
        for v in nb:
            assert pos[v] <= pos[u]
    ce = qgraph.condensed_edges(adj, comps)
    assert len(ce) == 1
    # agrees with the oracle's independent implementation
    oc = oracle.tarjan(len(names), [(ix[a], ix[b]) for a, b in g["edges_as_drawn"]])
    assert sorted(map(sorted, oc)) == sorted(map(sorted, comps))


@pytest.mark.parametrize("key", ["tiny", "hydrocarbon"])
def test_symbolic_model_matches_oracle(key):
    """The compiler's symbolic model, evaluated in Python, against the oracle."""
    m = workloads.mechanism(key)
    ir = qmech.parse(m)
    mod = qmodel.build_model(ir)
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], 4)
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    C = om.conc(rho, Y)
    N = ir.N
    n = N + 1
    outs = list(mod.wdot) + [mod.Tdot] + [mod.jac[i][j] for i in range(n) for j in range(n)]
    for c in range(4):
        env = {mod.C[k]: C[k, c] for k in range(N)}
        env[mod.T] = T[c]
        v = np.array(mod.g.evaluate(outs, env, fns=mod.bind))
        assert np.all(np.abs(v[:N] - ref["wdot"][:, c]) <= 2 * eb["wdot"][:, c] + 1e-300)
        assert abs(v[N] - ref["Tdot"][c]) <= 2 * eb["Tdot"][c]
        assert np.all(np.abs(v[N + 1:] - ref["jac"][:, c]) <= 2 * eb["jac"][:, c] + 1e-300)
    assert sorted(map(len, mod.groups)) == sorted(map(len, m["planned_qss_groups"]))


def test_compiler_rejects_quadratic_qss_coupling():
    sp = [hm.species("A", {"H": 2}), hm.species("N2", {"N": 2}),
          hm.species("q1", {"H": 1}, qss=True), hm.species("q2", {"H": 1}, qss=True)]
    m = hm.mech("quad", sp, [hm.reaction({"q1": 1, "q2": 1}, {"A": 1}, 1e12)])
    with pytest.raises(qmech.MechanismError):
        qmech.parse(m)


def test_artefact_build_tiny():
    art = qbuild.build_mechanism(workloads.mechanism("tiny"))
    for f in ("meta.txt", "meta.json"):
        assert os.path.exists(os.path.join(art, f)), f
    for f in ("jac.cubin", "wdot.cubin", "newton.cubin"):   # shared copies named in meta.txt
        assert os.path.exists(qbuild.cubin_file(art, f)), f
    meta = qbuild.load_meta(art)
    assert meta["N"] == 9 and meta["Q"] == 3 and meta["M"] == 30
    assert meta["flops_jac"] > meta["flops_wdot"] > 0
    assert "qss_jac_kernel" in meta["kernels"]


@pytest.mark.parametrize("variant,tcol", [("const_qss", "analytic"), ("zero_qss", "analytic"), ("exact", "fd")])
def test_jacobian_variant_models_match_oracle_on_cpu(variant, tcol):
    """The compiler's symbolic variant models, evaluated on the CPU by the DAG
    interpreter, agree with the oracle's implementation of the same variant
    (the FD temperature column uses the compiler's exact power-of-two step)."""
    import math
    import numpy as np
    import oracle
    from paper_2405_05974_b300 import mechgen
    from paper_2405_05974_b300.qssc import model as qmodel

    m = workloads.mechanism("tiny")
    ir = qmech.parse(m)
    mod = qmodel.build_model(ir, jac_variant=variant, t_column=tcol)
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["tiny"], 3)
    ref = om.eval_variant(rho, T, Y, variant, tcol)
    C = om.conc(rho, Y)
    n = ir.N + 1
    for c in range(3):
        env = {mod.C[k]: float(C[k, c]) for k in range(ir.N)}
        env[mod.T] = float(T[c])
        if mod.fd_vars is not None:
            _, e = math.frexp(T[c])
            h = math.ldexp(1.0, e - 21)
            env[mod.fd_vars[0]] = T[c] + h
            env[mod.fd_vars[1]] = T[c] - h
            env[mod.fd_vars[2]] = 0.5 / h
        outs = [mod.jac[i][j] for i in range(n) for j in range(n)]
        got = np.array(mod.g.evaluate(outs, env, fns=mod.bind))
        want = ref["jac"][:, c]
        tol = 1e-9 * np.abs(want) + 1e-20 + 64 * ref["jac_err"][:, c]
        assert np.all(np.abs(got - want) <= tol), np.argwhere(np.abs(got - want) > tol)[:5]


@pytest.mark.parametrize("key", ["tiny", "hydrocarbon"])
def test_csr_layout_is_the_structural_pattern(key):
    """The CSR storage order lists exactly the entries whose expression is not
    identically zero, row by row with increasing columns; every such entry is
    nonzero at some sampled state (the oracle's dense Jacobian), so the pattern
    is not padded with entries that are always zero."""
    from paper_2405_05974_b300.qssc import emit as qemit
    m = workloads.mechanism(key)
    ir = qmech.parse(m)
    mod = qmodel.build_model(ir)
    n = ir.N + 1
    pos, row_ptr, col = qemit.jac_layout(mod, "csr")
    assert row_ptr[0] == 0 and row_ptr[-1] == len(col) == len(pos) and len(row_ptr) == n + 1
    for i in range(n):
        cols = col[row_ptr[i]:row_ptr[i + 1]]
        assert cols == sorted(set(cols))
        for p, c in zip(range(row_ptr[i], row_ptr[i + 1]), cols):
            assert pos[(i, c)] == p
    nz = {(i, c) for i in range(n) for c in range(n) if mod.jac[i][c] != mod.g.ZERO}
    assert set(pos) == nz
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], 64)
    J = om.eval(rho, T, Y)["jac"]
    seen = np.any(J != 0.0, axis=1).reshape(n, n)
    assert all(seen[i, c] for i, c in nz)
    assert not any(seen[i, c] for i in range(n) for c in range(n) if (i, c) not in nz)
    dpos, drp, dcol = qemit.jac_layout(mod, "dense")
    assert len(dpos) == n * n and dpos[(2, 3)] == 2 * n + 3 and drp == [i * n for i in range(n + 1)]


def test_csr_artefact_source_and_meta():
    """A CSR artefact stores each pattern position exactly once in the
    generated Jacobian (and in the partitioned groups), and its meta.txt
    carries the pattern the runtime validates."""
    m = workloads.mechanism("tiny")
    for parts in (0, 2):
        art = qbuild.build_mechanism(m, jac_format="csr", jac_parts=parts)
        meta = qbuild.load_meta(art)
        nnz = meta["jac_stored"]
        assert meta["jac_format"] == "csr" and nnz == meta["jac_nnz"] < (meta["N"] + 1) ** 2
        srcd = qbuild.source_dir(art)   # the generated sources are kept beside the artefact
        srcs = [f for f in os.listdir(srcd) if f.startswith("mech_jac")]
        stored = []
        for f in srcs:
            stored += [int(x) for x in re.findall(r"jac\[(\d+) \* jstride\]", open(os.path.join(srcd, f)).read())]
        assert sorted(stored) == list(range(nnz))
        sizes = open(os.path.join(qbuild.source_dir(art), "mech_sizes.inc")).read()
        assert f"#define QSS_JAC_NNZ {nnz}" in sizes and "#define QSS_JAC_CSR 1" in sizes
        n = meta["N"] + 1
        rc = [int(x) for x in re.search(r"qss_jac_rc\[QSS_JAC_NNZ\] = \{([^}]*)\}", sizes).group(1).split(",")]
        assert rc == [i * n + c for i in range(n) for c in meta["jac_col"][meta["jac_row_ptr"][i]:meta["jac_row_ptr"][i + 1]]]
        txt = dict(line.split(" ", 1) for line in open(os.path.join(art, "meta.txt")).read().splitlines())
        assert int(txt["jac_nnz"]) == nnz
        assert [int(x) for x in txt["jac_row_ptr"].split()] == meta["jac_row_ptr"]
        assert [int(x) for x in txt["jac_col"].split()] == meta["jac_col"]
    dense = qbuild.load_meta(qbuild.build_mechanism(m))
    assert dense["jac_format"] == "dense" and dense["jac_stored"] == (dense["N"] + 1) ** 2


def test_mixed_jacobian_build_option_checks():
    """jac32 (the mixed-precision Jacobian) is built for the exact Jacobian
    with the analytic temperature column only; the artefact's meta.txt then
    announces it to the runtime."""
    m = workloads.mechanism("tiny")
    for bad in ({"jac_variant": "const_qss"}, {"t_column": "fd"}, {"replace_nop": 10}):
        with pytest.raises(ValueError):
            qbuild.build_mechanism(m, jac32=True, **bad)
    art = qbuild.build_mechanism(m, jac32=True)
    assert "jac32 1" in open(os.path.join(art, "meta.txt")).read().splitlines()
    assert os.path.exists(qbuild.cubin_file(art, "jac32.cubin"))
    assert "qss_jac32_kernel" in qbuild.load_meta(art)["kernels"]
    assert "jac32 1" not in open(os.path.join(qbuild.build_mechanism(m), "meta.txt")).read().splitlines()
