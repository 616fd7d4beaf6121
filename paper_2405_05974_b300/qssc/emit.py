"""CUDA emission of the symbolic model.

The model's outputs are emitted as straight-line FP64 code: one SSA
``const double`` per DAG node, in a depth-first post-order from the outputs,
so that every value is produced shortly before its first use and every output
is stored as soon as it is final (the emission order plays the role of the
paper's subexpression recycling, Alg. 3: a value's register is free after its
last use, which the register allocator sees directly).  A product used once
by a sum is emitted as ``fma`` (also when the product is shared).  Constants are literals (nvcc places FP64
literals in the constant bank, the "constant global arrays" of Appendix A).

Two device functions are produced per mechanism:
  qss_eval_wdot(C, T, wdot, Tdot, wstride)
  qss_eval_jac (C, T, wdot, Tdot, jac, wstride, jstride)
with outputs written at ``wdot[i * wstride]`` and ``jac[e * jstride]``.
"""
from __future__ import annotations

from collections import Counter
from typing import Dict, List, Tuple

from .expr import ADD, CONST, EXP, FACT, LOG, LT, MUL, NEG, RECIP, SELECT, SUB, VAR


def _lit(v: float) -> str:
    r = repr(float(v))
    if "inf" in r or "nan" in r:
        raise ValueError(f"non-finite constant {v}")
    if "e" not in r and "." not in r:
        r += ".0"
    return r


class Emitter:
    def __init__(self, model, input_names: Dict[int, str]):
        self.m = model
        self.g = model.g
        self.inputs = input_names     # VAR node -> C identifier

    def _resolve(self, i):
        g = self.g
        while g.op[i] == VAR and i in self.m.bind:
            i = self.m.bind[i]
        return i

    def _children(self, i):
        g = self.g
        op = g.op[i]
        a = g.args[i]
        if op in (CONST, VAR):
            return []
        if op == FACT:
            return [self._resolve(a[0])]
        if op == LT:
            return [self._resolve(a[0])]
        return [self._resolve(x) for x in a]

    def emit(self, outputs: List[Tuple[str, int]], indent="  "):
        """outputs: list of (store-statement format with {v}, node).  Returns
        (code lines, op counts)."""
        g = self.g
        roots = [self._resolve(n) for _, n in outputs]
        # needed set and reference counts
        refc = Counter()
        seen = set()
        stack = list(roots)
        while stack:
            n = stack.pop()
            if n in seen:
                continue
            seen.add(n)
            for c in self._children(n):
                refc[c] += 1
                stack.append(c)
        for r in roots:
            refc[r] += 1
        # which nodes are folded into their user (fma, negation, constants)
        inline = set()
        for n in seen:
            op = g.op[n]
            if op in (CONST, NEG, LT):
                inline.add(n)
            elif op == VAR:
                inline.add(n)
            elif op == FACT:
                inline.add(n)
        # Fused multiply-add: a sum node absorbs one product operand as fma.
        # A product whose every user absorbs it is never materialised (the
        # multiply is repeated inside each fma at no cost: an fma is one
        # instruction, the same as the add it replaces).  Materialising a
        # product shared by k sums costs 1 + k instructions, absorbing it k.
        fma_of = {}
        for n in seen:
            if g.op[n] in (ADD, SUB):
                a, b = [self._resolve(x) for x in g.args[n]]
                cands = [(w, x) for w, x in ((0, a), (1, b)) if g.op[x] == MUL and x not in inline]
                if not cands:
                    continue
                if len(cands) == 2:
                    cands.sort(key=lambda wx: refc[wx[1]])
                fma_of[n] = cands[0]
        absorbed = Counter()
        for n, (_, x) in fma_of.items():
            absorbed[x] += 1
        root_set = set(roots)
        for x, k in absorbed.items():
            if k == refc[x] and x not in root_set:
                inline.add(x)
        names: Dict[int, str] = {}
        lines: List[str] = []
        counts = Counter()

        def ref(n):
            n = self._resolve(n)
            op = g.op[n]
            if op == CONST:
                v = g.val[n]
                return _lit(v) if v >= 0 else f"({_lit(v)})"
            if op == VAR:
                if n not in self.inputs:
                    raise KeyError(f"unbound variable {g.name[n]}")
                return self.inputs[n]
            if op == NEG:
                return f"(-{ref(g.args[n][0])})"
            if op == FACT:
                return ref(g.args[n][0])
            if op == LT:
                return f"({ref(g.args[n][0])} < {_lit(g.args[n][1])})"
            return names[n]

        def expr_of(n):
            op = g.op[n]
            a = [self._resolve(x) for x in g.args[n]]
            if n in fma_of:
                which, mnode = fma_of[n]
                other = a[1 - which]
                ma, mb = [self._resolve(x) for x in g.args[mnode]]
                counts["fma"] += 1
                if op == ADD:
                    return f"fma({ref(ma)}, {ref(mb)}, {ref(other)})"
                if which == 1:   # other - ma*mb
                    return f"fma(-{ref(ma)}, {ref(mb)}, {ref(other)})"
                return f"fma({ref(ma)}, {ref(mb)}, -{ref(other)})"
            if op == ADD:
                counts["add"] += 1
                return f"{ref(a[0])} + {ref(a[1])}"
            if op == SUB:
                counts["add"] += 1
                return f"{ref(a[0])} - {ref(a[1])}"
            if op == MUL:
                counts["mul"] += 1
                return f"{ref(a[0])} * {ref(a[1])}"
            if op == RECIP:
                counts["rcp"] += 1
                return f"qss_rcp({ref(a[0])})"
            if op == EXP:
                counts["exp"] += 1
                return f"qss_exp({ref(a[0])})"
            if op == LOG:
                counts["log"] += 1
                return f"qss_log({ref(a[0])})"
            if op == SELECT:
                counts["select"] += 1
                return f"({ref(g.args[n][0])} ? {ref(a[1])} : {ref(a[2])})"
            raise ValueError(op)

        done = set()

        def visit(root):
            st = [(root, False)]
            while st:
                n, ready = st.pop()
                if n in done:
                    continue
                if not ready:
                    st.append((n, True))
                    for c in reversed(self._children(n)):
                        if c not in done:
                            st.append((c, False))
                    continue
                done.add(n)
                if n in inline:
                    continue
                names[n] = f"t{n}"
                lines.append(f"{indent}const double t{n} = {expr_of(n)};")

        for (fmt, node), root in zip(outputs, roots):
            visit(root)
            lines.append(indent + fmt.format(v=ref(root)))
        # algorithmic count: each DAG operation once, independent of fusion
        dag = Counter()
        for n in seen:
            op = g.op[n]
            if op in (ADD, SUB):
                dag["add"] += 1
            elif op == MUL:
                dag["mul"] += 1
            elif op == RECIP:
                dag["rcp"] += 1
            elif op == EXP:
                dag["exp"] += 1
            elif op == LOG:
                dag["log"] += 1
        counts["dag_flops"] = sum(dag.values())
        return lines, counts


def algorithmic_flops(counts) -> int:
    """FP64 operations of the CSE'd DAG: each add/sub/mul/reciprocal/exp/log node
    counts once (an fma in the emitted code is the add plus the multiply it
    absorbed, so the count does not depend on how products were fused)."""
    return counts["dag_flops"]


def fp64_instructions(counts, exp_cost=10, log_cost=36, rcp_cost=10) -> int:
    """Estimated FP64-pipe instructions per cell of the emitted code."""
    return (counts["add"] + counts["mul"] + counts["fma"] + exp_cost * counts["exp"]
            + log_cost * counts["log"] + rcp_cost * counts["rcp"])


def emit_mechanism_source(model, block_hint=128) -> Tuple[str, dict]:
    ir = model.ir
    N, Q = ir.N, ir.Q
    n = N + 1
    g = model.g
    inputs = {model.C[k]: f"C{k}" for k in range(N)}
    inputs[model.T] = "T"
    fd_prologue = []
    if model.fd_vars is not None:
        for v, name in zip(model.fd_vars, ("Tp", "Tm", "inv2h")):
            inputs[v] = name
        # h = 2^(e - 20) for T in [2^e, 2^(e+1)): T +- h and 1/(2h) are exact
        fd_prologue = [
            "  const double qss_p2 = __longlong_as_double(__double_as_longlong(T) & 0x7ff0000000000000LL);",
            "  const double qss_h = qss_p2 * 0x1p-20;",
            "  const double Tp = T + qss_h, Tm = T - qss_h, inv2h = 0x1p19 / qss_p2;"]
    em = Emitter(model, inputs)
    out_w = [(f"if (wdot) wdot[{i} * wstride] = {{v}};", model.wdot[i]) for i in range(N)]
    out_t = [("if (Tdot) Tdot[0] = {v};", model.Tdot)]
    body_w, cnt_w = em.emit(out_w + out_t, indent="  ")
    # Jacobian: column by column, so that dC_Q/dphi for one column is live at a time
    out_j = []
    for c in range(n):
        for i in range(n):
            out_j.append((f"jac[{i * n + c} * jstride] = {{v}};", model.jac[i][c]))
    em2 = Emitter(model, inputs)
    body_j, cnt_j = em2.emit(out_w + out_t + out_j, indent="  ")
    hdr = [
        f"// Generated by qssc for mechanism '{ir.name}' (digest {ir.digest}).",
        f"// N = {N} transported species, Q = {Q} QSS species, M = {len(ir.rxns)} reactions.",
        f"// QSS solve order (SCC groups): {model.groups}",
        "#pragma once",
        f"#define QSS_N {N}",
        f"#define QSS_Q {Q}",
        f"#define QSS_NN {n}",
        "",
    ]
    unpack = [f"  const double C{k} = C[{k}];" for k in range(N)]
    hdr.append("__constant__ double qss_inv_W[QSS_N] = {" + ", ".join(_lit(1.0 / w) for w in ir.W) + "};")
    hdr.append("")
    src = "\n".join(hdr)
    src += "\n".join([
        "__device__ __forceinline__ void qss_eval_wdot(const double* __restrict__ C, const double T,",
        "    double* __restrict__ wdot, double* __restrict__ Tdot, const long long wstride) {",
        *unpack, *body_w, "}", "",
        "__device__ __forceinline__ void qss_eval_jac(const double* __restrict__ C, const double T,",
        "    double* __restrict__ wdot, double* __restrict__ Tdot, double* __restrict__ jac,",
        "    const long long wstride, const long long jstride) {",
        *unpack, *fd_prologue, *body_j, "}", ""])
    meta = {
        "N": N, "Q": Q, "M": len(ir.rxns), "n": n, "digest": ir.digest, "name": ir.name,
        "W": ir.W, "species": ir.names, "groups": model.groups,
        "jac_variant": model.jac_variant, "t_column": model.t_column,
        "ops_wdot": dict(cnt_w), "ops_jac": dict(cnt_j),
        "flops_wdot": algorithmic_flops(cnt_w), "flops_jac": algorithmic_flops(cnt_j),
        "fp64_instr_wdot": fp64_instructions(cnt_w), "fp64_instr_jac": fp64_instructions(cnt_j),
        "dag_nodes": len(g.op), "jac_nnz": sum(1 for i in range(n) for c in range(n)
                                               if model.jac[i][c] != g.ZERO),
    }
    return src, meta
