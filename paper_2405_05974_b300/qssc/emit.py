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

import re
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


def _lit32(v: float) -> str:
    """A single-precision literal of v (rounded to the nearest float)."""
    import numpy as np
    with np.errstate(over="ignore"):
        f = float(np.float32(v))
    if f != f or f in (float("inf"), float("-inf")):
        raise ValueError(f"constant {v} has no single-precision value")
    return _lit(f) + "f"


class Emitter:
    def __init__(self, model, input_names: Dict[int, str], leaves: Dict[int, str] = None,
                 replace_nop: int = 0, emit_order: str = "first_use"):
        self.m = model
        self.g = model.g
        self.inputs = input_names     # VAR node -> C identifier
        self.leaves = leaves or {}    # any node -> C identifier of an already computed value
        self.replace_nop = replace_nop   # Alg. 2 threshold n_op (0: no replacement)
        if emit_order not in EMIT_ORDERS:
            raise ValueError(f"unknown emission order {emit_order!r}")
        # Alg. 3 on ("first_use": every output stored as soon as it is final,
        # each value computed just before its first use) or off ("all_first":
        # every value computed before any output is stored, so no value dies
        # before the stores begin)
        self.emit_order = emit_order
        self.smem_slot = {}   # node -> shared-memory slot (values kept there, not in registers)
        # mixed precision: FP32 values kept in shared memory, by key ("n", node)
        # for an FP32 node, ("c", key) for the FP32 copy of an FP64 value
        self.smem32 = {}
        self.conv_names = {}  # after emit(): FP32-copy name (s<i>) -> its key

    def _resolve(self, i):
        g = self.g
        while g.op[i] == VAR and i in self.m.bind:
            i = self.m.bind[i]
        return i

    def _children(self, i):
        g = self.g
        op = g.op[i]
        a = g.args[i]
        if op in (CONST, VAR) or i in self.leaves:
            return []
        if op == FACT:
            return [self._resolve(a[0])]
        if op == LT:
            return [self._resolve(a[0])]
        return [self._resolve(x) for x in a]

    def emit(self, outputs: List[Tuple[str, int]], indent="  ", fp64_outputs: int = None):
        """outputs: list of (store-statement format with {v}, node).  Returns
        (code lines, op counts).

        fp64_outputs = k (mixed precision): the nodes the first k outputs
        need are computed in FP64 as usual; every other node (the part only
        the later outputs need: the Jacobian's derivative terms) is computed
        in FP32 (`const float`, fmaf), its FP64 operands converted once each
        (qss_f32, at their first FP32 use) and its stored results widened
        back (qss_f64)."""
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
        # mixed precision: FP32 for the nodes that the FP64 outputs do not need
        f32 = set()
        if fp64_outputs is not None:
            if self.replace_nop or self.smem_slot:
                raise ValueError("mixed precision is emitted without replacement or FP64 shared-memory slots")
            val = set()
            stack = list(roots[:fp64_outputs])
            while stack:
                n = stack.pop()
                if n in val:
                    continue
                val.add(n)
                stack.extend(self._children(n))
            f32 = seen - val
        # which nodes are folded into their user (fma, negation, constants)
        inline = set()
        for n in seen:
            op = g.op[n]
            if n in self.leaves:
                inline.add(n)
            elif op in (CONST, NEG, LT):
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
        # Alg. 2 (common-subexpression replacement by operation count): for
        # thresholds 1..n_op, a stored subexpression whose replacement adds
        # (uses - 1) x (operations in its line) < threshold operations is
        # written out inside each of its users instead of being stored.
        replaced = set()
        if self.replace_nop > 0:
            order = sorted(seen)     # node ids are topological (children first)
            nop = {}

            def line_ops(n):
                if g.op[n] in (CONST, VAR, LT, FACT) or n in self.leaves:
                    return 0
                own = 1 if g.op[n] != NEG else 0
                return own + sum(nop.get(c, 0) for c in self._children(n) if c in replaced or
                                 (c in inline and g.op[c] not in (CONST, VAR)))
            for thr in range(1, self.replace_nop + 1):
                for n in order:
                    nop[n] = line_ops(n)
                    if n in inline or n in replaced or n in root_set or n in self.leaves:
                        continue
                    if g.op[n] in (CONST, VAR, LT, FACT):
                        continue
                    if (refc[n] - 1) * nop[n] < thr:
                        replaced.add(n)

        names: Dict[int, str] = {}
        lines: List[str] = []
        counts = Counter()
        conv = {}      # FP64 value -> the name of its FP32 copy (mixed precision)
        pending = []   # conversions to emit before the next line

        def as32(x, key):
            if key not in conv:
                nm = f"s{len(conv)}"
                self.conv_names[nm] = key
                if ("c", key) in self.smem32:
                    conv[key] = f"qss_sm32[{self.smem32[('c', key)]} * QSS_BLOCK]"
                    pending.append(f"{indent}{conv[key]} = qss_f32({x});")
                else:
                    conv[key] = nm
                    pending.append(f"{indent}const float {nm} = qss_f32({x});")
                counts["cvt_f32"] += 1
            return conv[key]

        def is32(n):
            n = self._resolve(n)
            op = g.op[n]
            if n in self.leaves or op in (CONST, VAR, LT):
                return False
            if op in (NEG, FACT):
                return is32(g.args[n][0])
            return n in f32

        def ref(n, f=False):
            """C expression of node n's value; f: in an FP32 expression."""
            n = self._resolve(n)
            op = g.op[n]
            if n in self.leaves:
                return as32(self.leaves[n], ("leaf", n)) if f else self.leaves[n]
            if op == CONST:
                v = g.val[n]
                lit = _lit32(v) if f else _lit(v)
                return lit if v >= 0 else f"({lit})"
            if op == VAR:
                if n not in self.inputs:
                    raise KeyError(f"unbound variable {g.name[n]}")
                return as32(self.inputs[n], n) if f else self.inputs[n]
            if op == NEG:
                return f"(-{ref(g.args[n][0], f)})"
            if op == FACT:
                return ref(g.args[n][0], f)
            if op == LT:
                c = self._resolve(g.args[n][0])
                if is32(c):
                    return f"({ref(c, True)} < {_lit32(g.args[n][1])})"
                return f"({ref(c)} < {_lit(g.args[n][1])})"
            if n in replaced:
                return f"({expr_of(n)})"
            if n in self.smem_slot:
                return f"qss_sm[{self.smem_slot[n]} * QSS_BLOCK]"
            if n in f32:
                if not f:
                    raise AssertionError("an FP32 value used by an FP64 expression")
                return names[n]
            return as32(names[n], n) if f else names[n]

        def out_ref(n):
            return f"qss_f64({ref(n, True)})" if is32(n) else ref(n)

        def expr_of(n):
            op = g.op[n]
            f = n in f32
            k = "f32_" if f else ""
            a = [self._resolve(x) for x in g.args[n]]
            if n in fma_of:
                which, mnode = fma_of[n]
                other = a[1 - which]
                ma, mb = [self._resolve(x) for x in g.args[mnode]]
                counts[k + "fma"] += 1
                fn = "fmaf" if f else "fma"
                if op == ADD:
                    return f"{fn}({ref(ma, f)}, {ref(mb, f)}, {ref(other, f)})"
                if which == 1:   # other - ma*mb
                    return f"{fn}(-{ref(ma, f)}, {ref(mb, f)}, {ref(other, f)})"
                return f"{fn}({ref(ma, f)}, {ref(mb, f)}, -{ref(other, f)})"
            if op == ADD:
                counts[k + "add"] += 1
                return f"{ref(a[0], f)} + {ref(a[1], f)}"
            if op == SUB:
                counts[k + "add"] += 1
                return f"{ref(a[0], f)} - {ref(a[1], f)}"
            if op == MUL:
                counts[k + "mul"] += 1
                return f"{ref(a[0], f)} * {ref(a[1], f)}"
            if op == RECIP:
                counts[k + "rcp"] += 1
                return f"__frcp_rn({ref(a[0], True)})" if f else f"qss_rcp({ref(a[0])})"
            if op == EXP:
                counts[k + "exp"] += 1
                return f"expf({ref(a[0], True)})" if f else f"qss_exp({ref(a[0])})"
            if op == LOG:
                counts[k + "log"] += 1
                return f"logf({ref(a[0], True)})" if f else f"qss_log({ref(a[0])})"
            if op == SELECT:
                counts[k + "select"] += 1
                return f"({ref(g.args[n][0])} ? {ref(a[1], f)} : {ref(a[2], f)})"
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
                if n in inline or n in replaced:
                    continue
                names[n] = f"t{n}"
                e = expr_of(n)
                lines.extend(pending)
                pending.clear()
                if ("n", n) in self.smem32:
                    names[n] = f"qss_sm32[{self.smem32[('n', n)]} * QSS_BLOCK]"
                    lines.append(f"{indent}{names[n]} = {e};")
                elif n in self.smem_slot:
                    lines.append(f"{indent}qss_sm[{self.smem_slot[n]} * QSS_BLOCK] = {e};")
                else:
                    lines.append(f"{indent}const {'float' if n in f32 else 'double'} t{n} = {e};")

        def store(fmt, root):
            v = out_ref(root)
            lines.extend(pending)
            pending.clear()
            lines.append(indent + fmt.format(v=v))

        if self.emit_order == "first_use":
            for (fmt, node), root in zip(outputs, roots):
                visit(root)
                store(fmt, root)
        else:
            for root in roots:
                visit(root)
            for (fmt, node), root in zip(outputs, roots):
                store(fmt, root)
        # algorithmic count: each DAG operation once, independent of fusion
        dag = Counter()
        for n in seen:
            if n in self.leaves:
                continue
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


def fp64_instructions(counts, exp_cost=7, log_cost=12, rcp_cost=3) -> int:
    """Estimated FP64-pipe instructions per cell of the emitted code."""
    return (counts["add"] + counts["mul"] + counts["fma"] + exp_cost * counts["exp"]
            + log_cost * counts["log"] + rcp_cost * counts["rcp"])


def choose_smem_values32(lines, slots: int, registers: int = 340):
    """choose_smem_values for a mixed-precision body: the `slots` FP32
    values (t<id> float nodes and s<i> FP32 copies) that a register file of
    `registers` 32-bit registers would reload most often (a double takes two
    of them; furthest-next-use eviction).  Returns their names, most
    reloaded first."""
    tok = re.compile(r"\b([ts]\d+)\b")
    defn = re.compile(r"\s*const (float|double) ([ts]\d+) = (.*);")
    seq, width = [], {}
    for ln in lines:
        m = defn.match(ln)
        if m:
            width[m.group(2)] = 1 if m.group(1) == "float" else 2
            seq.append((m.group(2), tok.findall(m.group(3))))
        else:
            seq.append((None, tok.findall(ln)))
    uses = {}
    for i, (d, u) in enumerate(seq):
        for x in u:
            uses.setdefault(x, []).append(i)
    pos = {x: 0 for x in uses}
    resident, reloads = set(), Counter()

    def next_use(x, i):
        v = uses[x]
        while pos[x] < len(v) and v[pos[x]] <= i:
            pos[x] += 1
        return v[pos[x]] if pos[x] < len(v) else None
    for i, (d, u) in enumerate(seq):
        for x in u:
            if x not in resident:
                reloads[x] += 1
                resident.add(x)
        if d is not None and d in uses:
            resident.add(d)
        nu = {x: next_use(x, i) for x in resident}
        resident = {x for x in resident if nu[x] is not None}
        used = sum(width.get(x, 2) for x in resident)
        if used > registers:
            for x in sorted(resident, key=lambda y: (-nu[y], y)):
                if used <= registers:
                    break
                resident.discard(x)
                used -= width.get(x, 2)
    return [x for x, _ in reloads.most_common() if width.get(x) == 1][:slots]


def choose_smem_names(lines, slots: int, registers: int = 170):
    """choose_smem_values over every named double of a column-group body:
    computed values (t<id>) and the frontier values it loads (F<slot>,
    defined by their load).  Returns the names, most reloaded first."""
    tok = re.compile(r"\b([tF]\d+)\b")
    defn = re.compile(r"\s*const double ([tF]\d+) = (.*);")
    seq = []
    for ln in lines:
        m = defn.match(ln)
        if m:
            seq.append((m.group(1), tok.findall(m.group(2))))
        else:
            seq.append((None, tok.findall(ln)))
    uses = {}
    for i, (d, u) in enumerate(seq):
        for x in u:
            uses.setdefault(x, []).append(i)
    pos = {x: 0 for x in uses}
    resident, reloads = set(), Counter()

    def next_use(x, i):
        v = uses[x]
        while pos[x] < len(v) and v[pos[x]] <= i:
            pos[x] += 1
        return v[pos[x]] if pos[x] < len(v) else None
    for i, (d, u) in enumerate(seq):
        for x in u:
            if x not in resident:
                reloads[x] += 1
                resident.add(x)
        if d is not None and d in uses:
            resident.add(d)
        nu = {x: next_use(x, i) for x in resident}
        resident = {x for x in resident if nu[x] is not None}
        if len(resident) > registers:
            for x in sorted(resident, key=lambda y: (-nu[y], y))[:len(resident) - registers]:
                resident.discard(x)
    return [x for x, _ in reloads.most_common(slots)]


def choose_smem_values(lines, slots: int, registers: int = 170):
    """The `slots` values of an emitted straight-line body that a register
    file of `registers` doubles would reload most often: a Belady (furthest
    next use) eviction simulation over the SSA sequence counts, per value,
    the uses that find it evicted.  Returns the node ids (from the t<id>
    names), most reloaded first.  (255 registers hold about 120 doubles; a
    simulated file of 170 picks values whose reuse distances are longer,
    and measured slightly faster on B300: 77.7-78.0 vs 78.3 ms per 2^20
    hydrocarbon cells with 100 slots; 70: 78.0, 250: 78.1.)"""
    tok = re.compile(r"\bt(\d+)\b")
    seq = []
    for ln in lines:
        m = re.match(r"\s*const double t(\d+) = (.*);", ln)
        if m:
            seq.append((int(m.group(1)), [int(x) for x in tok.findall(m.group(2))]))
        else:
            seq.append((None, [int(x) for x in tok.findall(ln)]))
    uses = {}
    for i, (d, u) in enumerate(seq):
        for x in u:
            uses.setdefault(x, []).append(i)
    pos = {x: 0 for x in uses}
    resident, reloads = set(), Counter()

    def next_use(x, i):
        v = uses[x]
        while pos[x] < len(v) and v[pos[x]] <= i:
            pos[x] += 1
        return v[pos[x]] if pos[x] < len(v) else None
    for i, (d, u) in enumerate(seq):
        for x in u:
            if x not in resident:
                reloads[x] += 1
                resident.add(x)
        if d is not None and d in uses:
            resident.add(d)
        nu = {x: next_use(x, i) for x in resident}
        resident = {x for x in resident if nu[x] is not None}
        if len(resident) > registers:
            for x in sorted(resident, key=lambda y: -nu[y])[:len(resident) - registers]:
                resident.discard(x)
    return [x for x, _ in reloads.most_common(slots)]


JAC_FORMATS = ("dense", "csr")
EMIT_ORDERS = ("first_use", "all_first")


def jac_layout(model, jac_format: str = "dense"):
    """Storage position of each Jacobian entry (i, c) that the kernels write.
    "dense": every entry, position i (N+1) + c.  "csr": only the structural
    nonzeros (entries whose expression is not identically zero), in row-major
    order, position = index in the CSR value array.  Returns (pos, row_ptr,
    col_idx); row_ptr / col_idx describe the stored pattern in both formats."""
    if jac_format not in JAC_FORMATS:
        raise ValueError(f"unknown Jacobian format {jac_format!r}")
    g = model.g
    n = model.ir.N + 1
    pos, row_ptr, col = {}, [0], []
    for i in range(n):
        for c in range(n):
            if jac_format == "dense" or model.jac[i][c] != g.ZERO:
                pos[(i, c)] = len(col)
                col.append(c)
        row_ptr.append(len(col))
    return pos, row_ptr, col


_RENAME_B = [(re.compile(r"\bt(\d+)\b"), r"tb\1"), (re.compile(r"\bC(\d+)\b"), r"Cb\1"),
             (re.compile(r"\bT\b"), "Tb"), (re.compile(r"^(\s*)jac\["), r"\1if (jac_b) jac_b["),
             (re.compile(r"\bwdot\b"), "wdot_b"), (re.compile(r"\bTdot\b"), "Tdot_b")]


def two_cell_body(lines):
    """The Jacobian body for two cells per thread: every line of the one-cell
    body (cell a) followed by its copy for cell b (values t<id> -> tb<id>,
    inputs C<k>, T -> Cb<k>, Tb, outputs through jac_b / wdot_b / Tdot_b,
    a null jac_b skipping cell b's stores), so that the two cells'
    independent chains interleave."""
    out = []
    for ln in lines:
        b = ln
        for rx, rep in _RENAME_B:
            b = rx.sub(rep, b)
        out += [ln, b]
    return out


def emit_mechanism_source(model, block_hint=128, replace_nop: int = 0,
                          jac_format: str = "dense", emit_order: str = "first_use",
                          col_order=None, smem_slots: int = 0, cells_per_thread: int = 1) -> Tuple[str, dict]:
    ir = model.ir
    N, Q = ir.N, ir.Q
    n = N + 1
    g = model.g
    pos, row_ptr, col = jac_layout(model, jac_format)
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
    em = Emitter(model, inputs, replace_nop=replace_nop, emit_order=emit_order)
    out_w = [(f"if (wdot) wdot[{i} * wstride] = {{v}};", model.wdot[i]) for i in range(N)]
    out_t = [("if (Tdot) Tdot[0] = {v};", model.Tdot)]
    body_w, cnt_w = em.emit(out_w + out_t, indent="  ")
    # Jacobian: column by column, so that dC_Q/dphi for one column is live at a time
    out_j = []
    for c in (range(n) if col_order is None else col_order):
        for i in range(n):
            if (i, c) in pos:
                out_j.append((f"jac[{pos[(i, c)]} * jstride] = {{v}};", model.jac[i][c]))
    em2 = Emitter(model, inputs, replace_nop=replace_nop, emit_order=emit_order)
    body_j, cnt_j = em2.emit(out_w + out_t + out_j, indent="  ")
    smem_prologue = []
    if smem_slots > 0:
        # the values a register file would reload most often (simulated) live
        # in shared memory (slot k of this thread at qss_sm[k * QSS_BLOCK];
        # the kernel is launched with smem_slots * QSS_BLOCK doubles of
        # dynamic shared memory); volatile, so that every use is a shared
        # load and no register copy is kept
        chosen = choose_smem_values(body_j, smem_slots)
        em2 = Emitter(model, inputs, replace_nop=replace_nop, emit_order=emit_order)
        em2.smem_slot = {x: k for k, x in enumerate(chosen)}
        body_j, cnt_j = em2.emit(out_w + out_t + out_j, indent="  ")
        smem_prologue = ["  extern __shared__ double qss_smem_dyn[];",
                         "  volatile double* const qss_sm = qss_smem_dyn + threadIdx.x;"]
    hdr = [
        f"// Generated by qssc for mechanism '{ir.name}' (digest {ir.digest}).",
        f"// N = {N} transported species, Q = {Q} QSS species, M = {len(ir.rxns)} reactions.",
        f"// QSS solve order (SCC groups): {model.groups}",
        "#pragma once",
        f"#define QSS_N {N}",
        f"#define QSS_Q {Q}",
        f"#define QSS_NN {n}",
        f"#define QSS_JAC_NNZ {len(col)}   // stored Jacobian entries per cell ({jac_format})",
        "",
    ]
    if jac_format == "csr":
        # position p of the CSR value array -> i * (N+1) + c, for kernels that
        # need the dense matrix (the Newton update)
        rc = [i * n + c for i in range(n) for c in col[row_ptr[i]:row_ptr[i + 1]]]
        hdr.append("#define QSS_JAC_CSR 1")
        hdr.append("__constant__ unsigned short qss_jac_rc[QSS_JAC_NNZ] = {" + ", ".join(map(str, rc)) + "};")
        hdr.append("")
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
        *unpack, *fd_prologue, *smem_prologue, *body_j, "}", ""])
    if cells_per_thread == 2:
        # two cells per thread (qss_jac2_kernel.cuh): the one-cell
        # body and its copy for the second cell, interleaved line by line
        if smem_slots > 0 or model.fd_vars is not None:
            raise ValueError("two cells per thread are emitted without shared-memory values and with "
                             "the analytic temperature column")
        unpack_b = [f"  const double Cb{k} = Cb_in[{k}];" for k in range(N)]
        src += "\n".join([
            "__device__ __forceinline__ void qss_eval_jac2(const double* __restrict__ C, const double T,",
            "    double* __restrict__ wdot, double* __restrict__ Tdot, double* __restrict__ jac,",
            "    const double* __restrict__ Cb_in, const double Tb, double* __restrict__ wdot_b,",
            "    double* __restrict__ Tdot_b, double* __restrict__ jac_b,",
            "    const long long wstride, const long long jstride) {",
            *unpack, *unpack_b, *two_cell_body(body_j), "}", ""])
    elif cells_per_thread != 1:
        raise ValueError("cells_per_thread is 1 or 2")
    meta = {
        "N": N, "Q": Q, "M": len(ir.rxns), "n": n, "digest": ir.digest, "name": ir.name,
        "W": ir.W, "species": ir.names, "groups": model.groups,
        "jac_variant": model.jac_variant, "t_column": model.t_column, "replace_nop": replace_nop,
        "emit_order": emit_order, "smem_slots": len(em2.smem_slot), "cells_per_thread": cells_per_thread,
        "jac_format": jac_format, "jac_stored": len(col), "jac_row_ptr": row_ptr, "jac_col": col,
        "ops_wdot": dict(cnt_w), "ops_jac": dict(cnt_j),
        "flops_wdot": algorithmic_flops(cnt_w), "flops_jac": algorithmic_flops(cnt_j),
        "fp64_instr_wdot": fp64_instructions(cnt_w), "fp64_instr_jac": fp64_instructions(cnt_j),
        "stored_values_jac": sum(1 for ln in body_j if ln.lstrip().startswith("const double t")),
        "dag_nodes": len(g.op), "jac_nnz": sum(1 for i in range(n) for c in range(n)
                                               if model.jac[i][c] != g.ZERO),
    }
    return src, meta


def emit_jac32_source(model, jac_format: str = "dense", smem_slots: int = 0) -> Tuple[str, dict]:
    """The mixed-precision Jacobian device function

        qss_eval_jac32(C, T, wdot, Tdot, jac, wstride, jstride)

    with qss_eval_jac's interface.  Everything wdot and Tdot need -- state,
    thermo, Arrhenius exponentials, equilibrium constants, third bodies and
    falloff, the QSS solve, the rates of progress -- is computed in FP64 by
    the operations qss_eval_jac uses, so wdot and Tdot are its values; the
    nodes only the Jacobian needs (the derivatives of the rates, dC_Q/dphi,
    the chain-rule products G + P X) are computed in FP32 and stored widened
    to FP64.  For the Newton iteration matrix of the mixed-precision implicit
    step, whose residual stays FP64.  smem_slots > 0: that many of the FP32
    values a register file would reload most often (choose_smem_values32)
    live in dynamic shared memory (slot k of this thread at
    qss_sm32[k * QSS_BLOCK]; smem_slots * QSS_BLOCK floats per block)."""
    ir = model.ir
    N = ir.N
    n = N + 1
    pos, _, _ = jac_layout(model, jac_format)
    if model.fd_vars is not None:
        raise ValueError("the mixed-precision Jacobian needs the analytic temperature column")
    inputs = {model.C[k]: f"C{k}" for k in range(N)}
    inputs[model.T] = "T"
    out_w = [(f"if (wdot) wdot[{i} * wstride] = {{v}};", model.wdot[i]) for i in range(N)]
    out_t = [("if (Tdot) Tdot[0] = {v};", model.Tdot)]
    out_j = []
    for c in range(n):
        for i in range(n):
            if (i, c) in pos:
                out_j.append((f"jac[{pos[(i, c)]} * jstride] = {{v}};", model.jac[i][c]))
    nval = len(out_w) + len(out_t)
    em = Emitter(model, inputs)
    body, cnt = em.emit(out_w + out_t + out_j, indent="  ", fp64_outputs=nval)
    prologue = []
    if smem_slots > 0:
        chosen = choose_smem_values32(body, smem_slots)
        keys = {nm: (("n", int(nm[1:])) if nm[0] == "t" else ("c", em.conv_names[nm])) for nm in chosen}
        em = Emitter(model, inputs)
        em.smem32 = {keys[nm]: k for k, nm in enumerate(chosen)}
        body, cnt = em.emit(out_w + out_t + out_j, indent="  ", fp64_outputs=nval)
        prologue = ["  extern __shared__ float qss_smem32_dyn[];",
                    "  volatile float* const qss_sm32 = qss_smem32_dyn + threadIdx.x;"]
    unpack = [f"  const double C{k} = C[{k}];" for k in range(N)]
    src = "\n".join([
        "__device__ __forceinline__ void qss_eval_jac32(const double* __restrict__ C, const double T,",
        "    double* __restrict__ wdot, double* __restrict__ Tdot, double* __restrict__ jac,",
        "    const long long wstride, const long long jstride) {",
        *unpack, *prologue, *body, "}", ""])
    meta = {"ops_jac32": dict(cnt), "flops_jac32": algorithmic_flops(cnt),
            "fp64_instr_jac32": fp64_instructions(cnt), "jac32_slots": len(em.smem32)}
    return src, meta


# ---------------------------------------------------------------------------
# Partitioned Jacobian: a shared prefix kernel and K column-group kernels
# ---------------------------------------------------------------------------
_MATERIAL = (ADD, SUB, MUL, RECIP, EXP, LOG, SELECT)
_FRONTIER_NAME = re.compile(r"\bF\d+\b")


def _op_cost(g, x):
    op = g.op[x]
    if op == EXP:
        return 8
    if op == LOG:
        return 13
    if op == RECIP:
        return 3
    return 1 if op in _MATERIAL else 0


def partition_jacobian(model, K: int, split_t: bool = True):
    """Split the Jacobian's entries into K groups (whole concentration
    columns, balanced by cost; the temperature column by rows when split_t)
    and its DAG into the part needed by two or more groups (the prefix,
    which also yields wdot and Tdot) and the parts needed by one group only.
    Returns (groups, frontier, needs): the (row, column) entries of each
    group, the prefix values a group kernel reads (node ids, in topological
    order), and for each group the frontier nodes it reads.  Every operation
    of the DAG is computed exactly once."""
    g = model.g
    N = model.ir.N
    n = N + 1
    em = Emitter(model, {})
    res, kids = em._resolve, em._children
    roots_w = [res(x) for x in model.wdot] + [res(model.Tdot)]
    roots_c = [[res(model.jac[i][c]) for i in range(n)] for c in range(n)]
    # the temperature column's entries are spread over the groups by row
    # (its shared derivative terms then belong to the prefix); its
    # single-group form is by far the slowest unit to compile
    tcol = N if (split_t and K > 1) else None
    # topological order of everything needed (children before users)
    order, seen = [], set()
    for r0 in roots_w + [r for col in roots_c for r in col]:
        if r0 in seen:
            continue
        st = [(r0, False)]
        while st:
            x, done = st.pop()
            if done:
                order.append(x)
                continue
            if x in seen:
                continue
            seen.add(x)
            st.append((x, True))
            st.extend((k, False) for k in kids(x) if k not in seen)

    def entry_group(i, c, col_group, ngroups):
        return (i % ngroups) if c == tcol else col_group[c]

    def masks(col_group, ngroups):
        m = {}
        for c in range(n):
            for i, r in enumerate(roots_c[c]):
                m[r] = m.get(r, 0) | (1 << entry_group(i, c, col_group, ngroups))
        full = (1 << ngroups) - 1
        for r in roots_w:
            m[r] = full
        for x in reversed(order):
            mx = m.get(x, 0)
            for k in kids(x):
                m[k] = m.get(k, 0) | mx
        return m

    # balance: each column's cost when every column is its own group, then
    # longest-first assignment to the least loaded group
    saved = tcol
    tcol = None
    m1 = masks(list(range(n)), n)
    tcol = saved
    col_cost = [0] * n
    for x in order:
        mx = m1[x]
        if mx and mx & (mx - 1) == 0:
            col_cost[mx.bit_length() - 1] += _op_cost(g, x)
    load = [0] * K
    col_group = [0] * n
    for c in sorted((c for c in range(n) if c != tcol), key=lambda c: -col_cost[c]):
        gi = min(range(K), key=lambda i: load[i])
        col_group[c] = gi
        load[gi] += col_cost[c]
    m = masks(col_group, K)
    shared = {x for x in order if m[x] & (m[x] - 1)}
    # frontier: shared computed values reached from a group's own nodes
    # (through inline operations such as negation)
    needs = []
    frontier = set()
    for gi in range(K):
        need = set()
        st = [r for c in range(n) for i, r in enumerate(roots_c[c])
              if entry_group(i, c, col_group, K) == gi]
        vis = set()
        while st:
            x = st.pop()
            if x in vis:
                continue
            vis.add(x)
            if x in shared and g.op[x] in _MATERIAL:
                need.add(x)
                continue
            st.extend(kids(x))
        needs.append(sorted(need))
        frontier |= need
    groups = [[(i, c) for c in range(n) for i in range(n) if entry_group(i, c, col_group, K) == gi]
              for gi in range(K)]
    return groups, sorted(frontier), needs


def emit_partitioned_source(model, K: int, jac_format: str = "dense", mixed: bool = False,
                            smem_slots: int = 0):
    """Sources of the partitioned Jacobian: the prefix device function
    qss_jac_prefix(C, T, wdot, Tdot, wstride, fr, fstride) and, per group,
    qss_jac_group(fr, fstride, jac, jstride).  The frontier array fr holds,
    per cell, C_1..C_N and T in slots 0..N, then the prefix values the groups
    read (slot N + 1 + i for the i-th frontier node).  mixed: the
    mixed-precision form (emit_jac32_source's split): the prefix computes
    what wdot and Tdot need in FP64 and its other values in FP32 (stored to
    the FP64 frontier widened); the group kernels, whose nodes wdot and Tdot
    never need, compute in FP32 from the frontier values narrowed.
    smem_slots > 0 (FP64 form): in the prefix and in every group, the
    values a 170-double register file would reload most often are kept in
    dynamic shared memory as in the single kernel (choose_smem_values; in
    the groups the frontier values are candidates too, choose_smem_names;
    each kernel is launched with smem_slots * QSS_BLOCK doubles)."""
    ir = model.ir
    N = ir.N
    n = N + 1
    groups, frontier, needs = partition_jacobian(model, K)
    pos, _, _ = jac_layout(model, jac_format)
    slot = {x: n + i for i, x in enumerate(frontier)}
    inputs = {model.C[k]: f"C{k}" for k in range(N)}
    inputs[model.T] = "T"
    fd_prologue = []
    if model.fd_vars is not None:
        for v, name in zip(model.fd_vars, ("Tp", "Tm", "inv2h")):
            inputs[v] = name
        fd_prologue = [
            "  const double qss_p2 = __longlong_as_double(__double_as_longlong(T) & 0x7ff0000000000000LL);",
            "  const double qss_h = qss_p2 * 0x1p-20;",
            "  const double Tp = T + qss_h, Tm = T - qss_h, inv2h = 0x1p19 / qss_p2;"]
    out_w = [(f"if (wdot) wdot[{i} * wstride] = {{v}};", model.wdot[i]) for i in range(N)]
    out_t = [("if (Tdot) Tdot[0] = {v};", model.Tdot)]
    out_f = [(f"fr[{slot[x]} * fstride] = {{v}};", x) for x in frontier]
    if mixed and model.fd_vars is not None:
        raise ValueError("the mixed-precision Jacobian needs the analytic temperature column")
    if mixed and smem_slots > 0:
        raise ValueError("shared-memory values apply to the FP64 partitioned Jacobian")
    smem_prologue = ["  extern __shared__ double qss_smem_dyn[];",
                     "  volatile double* const qss_sm = qss_smem_dyn + threadIdx.x;"]

    def emit_body(outs, leaves=None, fp64_outputs=None):
        body, cnt = Emitter(model, inputs, leaves).emit(outs, indent="  ", fp64_outputs=fp64_outputs)
        if smem_slots <= 0:
            return body, cnt, [], 0
        chosen = choose_smem_values(body, smem_slots)
        em = Emitter(model, inputs, leaves)
        em.smem_slot = {x: k for k, x in enumerate(chosen)}
        body, cnt = em.emit(outs, indent="  ", fp64_outputs=fp64_outputs)
        return body, cnt, (smem_prologue if chosen else []), len(chosen)

    body_p, cnt_p, sm_p, used_p = emit_body(out_w + out_t + out_f,
                                            fp64_outputs=(len(out_w) + len(out_t)) if mixed else None)
    slots_used = [used_p]
    unpack = [f"  const double C{k} = C[{k}];" for k in range(N)]
    store_state = [f"  fr[{k} * fstride] = C{k};" for k in range(N)] + [f"  fr[{N} * fstride] = T;"]
    prefix = "\n".join([
        "__device__ __forceinline__ void qss_jac_prefix(const double* __restrict__ C, const double T,",
        "    double* __restrict__ wdot, double* __restrict__ Tdot, const long long wstride,",
        "    double* __restrict__ fr, const long long fstride) {",
        *unpack, *store_state, *fd_prologue, *sm_p, *body_p, "}", ""])
    group_src, group_cnt = [], []
    def lazy_loads(body, pending):
        # each frontier value is loaded just before its first use: loaded all
        # at the top, a group's hundreds of values go straight from the load
        # to the spill stack
        pending = dict(pending)
        lazy = []
        for line in body:
            for nm in _FRONTIER_NAME.findall(line):
                if nm in pending:
                    lazy.append(pending.pop(nm))
            lazy.append(line)
        return lazy + list(pending.values())

    for gi, entries in enumerate(groups):
        leaves = {x: f"F{slot[x]}" for x in needs[gi]}
        out_j = [(f"jac[{pos[(i, c)]} * jstride] = {{v}};", model.jac[i][c]) for i, c in entries
                 if (i, c) in pos]
        fp = 0 if mixed else None
        body_g, cnt_g = Emitter(model, inputs, leaves).emit(out_j, indent="  ", fp64_outputs=fp)
        pending = {f"F{slot[x]}": f"  const double F{slot[x]} = fr[{slot[x]} * fstride];" for x in needs[gi]}
        body_g = lazy_loads(body_g, pending)
        sm_g, used_g = [], 0
        if smem_slots > 0:
            # a group's most-reloaded values are mostly frontier values: those
            # chosen are loaded into their shared-memory slot (the slot's
            # expression keeps the F name in a comment, so that the load is
            # still placed before the first use)
            chosen = choose_smem_names(body_g, smem_slots)
            if chosen:
                node_of = {f"F{slot[x]}": x for x in needs[gi]}
                leaves2 = dict(leaves)
                for k, nm in enumerate(chosen):
                    if nm[0] == "F":
                        leaves2[node_of[nm]] = f"qss_sm[{k} * QSS_BLOCK /*{nm}*/]"
                        pending[nm] = f"  qss_sm[{k} * QSS_BLOCK] = fr[{nm[1:]} * fstride];"
                em = Emitter(model, inputs, leaves2)
                em.smem_slot = {int(nm[1:]): k for k, nm in enumerate(chosen) if nm[0] == "t"}
                body_g, cnt_g = em.emit(out_j, indent="  ", fp64_outputs=fp)
                body_g = lazy_loads(body_g, pending)
                sm_g, used_g = smem_prologue, len(chosen)
        slots_used.append(used_g)
        loads = [f"  const double C{k} = fr[{k} * fstride];" for k in range(N)]
        loads += [f"  const double T = fr[{N} * fstride];"]
        group_src.append("\n".join([
            f"// entry group {gi} of {K}: columns {sorted({c for _, c in entries if c != N})}"
            + (f" and rows {sorted(i for i, c in entries if c == N)} of the T column" if any(c == N for _, c in entries) else ""),
            "__device__ __forceinline__ void qss_jac_group(const double* __restrict__ fr,",
            "    const long long fstride, double* __restrict__ jac, const long long jstride) {",
            *loads, *fd_prologue, *sm_g, *body_g, "}", ""]))
        group_cnt.append(cnt_g)
    meta = {"jac_parts": K, "frontier": n + len(frontier), "groups": groups, "smem_slots_parts": slots_used,
            "ops_prefix": dict(cnt_p), "ops_groups": [dict(c) for c in group_cnt],
            "flops_jac_parts": algorithmic_flops(cnt_p) + sum(algorithmic_flops(c) for c in group_cnt)}
    return prefix, group_src, meta
