"""Hash-consed expression DAG with symbolic differentiation.

Every node is created through ``Graph``; structurally equal nodes are the same
node, so common subexpressions are eliminated as the expressions are built
(the role the paper gives to CSE, Section 3.2.2 and Appendix D).  Algebraic
simplification is limited to what cannot change rounding in a way that
matters: folding of constants, identities with 0 and 1, and merging of like
terms ``c1*x + c2*x``.

Node kinds
  CONST value          VAR name (an input or a placeholder bound later)
  ADD a b   SUB a b    MUL a b    NEG a    RECIP a   (1/a)
  EXP a     LOG a      SELECT cond a b (cond = LT x const)
  FACT v l  -- evaluates as v; its derivative is FACT * dl.  Used for
               quantities known to equal exp(l) but computed more cheaply as
               a product of shared factors (equilibrium-constant ratios).
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional

CONST, VAR, ADD, SUB, MUL, NEG, RECIP, EXP, LOG, SELECT, LT, FACT = range(12)
OPNAMES = ["const", "var", "add", "sub", "mul", "neg", "recip", "exp", "log", "select", "lt", "fact"]


class Graph:
    def __init__(self):
        self.op: List[int] = []
        self.args: List[tuple] = []
        self.val: List[float] = []       # constants
        self.name: List[Optional[str]] = []
        self.deps: List[int] = []        # bitset of VAR indices the node depends on
        self._key: Dict[tuple, int] = {}
        self.var_bit: Dict[int, int] = {}  # node id -> bit index
        self.var_nodes: List[int] = []
        self._dcache: Dict[tuple, int] = {}
        self._scache: Dict[tuple, int] = {}
        self.ZERO = self.const(0.0)
        self.ONE = self.const(1.0)

    # ------------------------------------------------------------------ nodes
    def _new(self, op, args, val=0.0, name=None, deps=0):
        key = (op, args, val if op == CONST else None, name if op == VAR else None)
        hit = self._key.get(key)
        if hit is not None:
            return hit
        i = len(self.op)
        self.op.append(op)
        self.args.append(args)
        self.val.append(val)
        self.name.append(name)
        self.deps.append(deps)
        self._key[key] = i
        return i

    def const(self, v: float) -> int:
        v = float(v)
        if v == 0.0:
            v = 0.0  # fold -0.0
        return self._new(CONST, (), v)

    def var(self, name: str) -> int:
        key = (VAR, (), None, name)
        if key in self._key:
            return self._key[key]
        bit = len(self.var_nodes)
        i = self._new(VAR, (), 0.0, name, 1 << bit)
        self.var_bit[i] = bit
        self.var_nodes.append(i)
        return i

    def is_const(self, a, v=None):
        return self.op[a] == CONST and (v is None or self.val[a] == v)

    def _coef(self, a):
        """Split a into (c, x) with a = c*x, c a constant."""
        if self.op[a] == MUL and self.op[self.args[a][0]] == CONST:
            return self.val[self.args[a][0]], self.args[a][1]
        if self.op[a] == NEG:
            return -1.0, self.args[a][0]
        return 1.0, a

    def add(self, a, b):
        if self.is_const(a) and self.is_const(b):
            return self.const(self.val[a] + self.val[b])
        if self.is_const(a, 0.0):
            return b
        if self.is_const(b, 0.0):
            return a
        if self.op[b] == NEG:
            return self.sub(a, self.args[b][0])
        if self.op[a] == NEG:
            return self.sub(b, self.args[a][0])
        ca, xa = self._coef(a)
        cb, xb = self._coef(b)
        if xa == xb and not self.is_const(xa):
            return self.mul(self.const(ca + cb), xa)
        if a > b:
            a, b = b, a
        return self._new(ADD, (a, b), deps=self.deps[a] | self.deps[b])

    def sub(self, a, b):
        if self.is_const(a) and self.is_const(b):
            return self.const(self.val[a] - self.val[b])
        if self.is_const(b, 0.0):
            return a
        if self.is_const(a, 0.0):
            return self.neg(b)
        if a == b:
            return self.ZERO
        if self.op[b] == NEG:
            return self.add(a, self.args[b][0])
        ca, xa = self._coef(a)
        cb, xb = self._coef(b)
        if xa == xb and not self.is_const(xa):
            return self.mul(self.const(ca - cb), xa)
        return self._new(SUB, (a, b), deps=self.deps[a] | self.deps[b])

    def neg(self, a):
        if self.is_const(a):
            return self.const(-self.val[a])
        if self.op[a] == NEG:
            return self.args[a][0]
        if self.op[a] == SUB:
            x, y = self.args[a]
            return self.sub(y, x)
        if self.op[a] == MUL and self.op[self.args[a][0]] == CONST:
            return self.mul(self.const(-self.val[self.args[a][0]]), self.args[a][1])
        return self._new(NEG, (a,), deps=self.deps[a])

    def mul(self, a, b):
        if self.is_const(a) and self.is_const(b):
            return self.const(self.val[a] * self.val[b])
        if self.is_const(b):
            a, b = b, a
        if self.is_const(a):
            c = self.val[a]
            if c == 0.0:
                return self.ZERO
            if c == 1.0:
                return b
            if c == -1.0:
                return self.neg(b)
            if self.op[b] == MUL and self.op[self.args[b][0]] == CONST:
                return self.mul(self.const(c * self.val[self.args[b][0]]), self.args[b][1])
            if self.op[b] == NEG:
                return self.mul(self.const(-c), self.args[b][0])
            return self._new(MUL, (a, b), deps=self.deps[b])
        if self.op[a] == NEG and self.op[b] == NEG:
            a, b = self.args[a][0], self.args[b][0]
        elif self.op[a] == NEG:
            return self.neg(self.mul(self.args[a][0], b))
        elif self.op[b] == NEG:
            return self.neg(self.mul(a, self.args[b][0]))
        if a > b:
            a, b = b, a
        return self._new(MUL, (a, b), deps=self.deps[a] | self.deps[b])

    def recip(self, a):
        if self.is_const(a):
            return self.const(1.0 / self.val[a])
        if self.op[a] == RECIP:
            return self.args[a][0]
        return self._new(RECIP, (a,), deps=self.deps[a])

    def div(self, a, b):
        if self.is_const(b):
            return self.mul(self.const(1.0 / self.val[b]), a)
        return self.mul(a, self.recip(b))

    def exp(self, a):
        if self.is_const(a):
            return self.const(math.exp(self.val[a]))
        return self._new(EXP, (a,), deps=self.deps[a])

    def log(self, a):
        if self.is_const(a):
            return self.const(math.log(self.val[a]))
        return self._new(LOG, (a,), deps=self.deps[a])

    def lt(self, x, c):
        return self._new(LT, (x, c), deps=0)

    def select(self, cond, a, b):
        if a == b:
            return a
        return self._new(SELECT, (cond, a, b), deps=self.deps[a] | self.deps[b])

    def fact(self, v, l):
        """A node equal to v, whose derivative is (this node) * dl."""
        return self._new(FACT, (v, l), deps=self.deps[v] | self.deps[l])

    def sum(self, terms):
        acc = self.ZERO
        for t in terms:
            acc = self.add(acc, t)
        return acc

    def prod(self, factors):
        acc = self.ONE
        for f in factors:
            acc = self.mul(acc, f)
        return acc

    def powi(self, x, n):
        assert n >= 0
        r = self.ONE
        for _ in range(n):
            r = self.mul(r, x)
        return r

    # ------------------------------------------------------- differentiation
    def d(self, node: int, v: int) -> int:
        """Symbolic derivative of ``node`` with respect to VAR node ``v``."""
        bit = 1 << self.var_bit[v]
        return self._d(node, v, bit)

    def _d(self, node, v, bit):
        if not (self.deps[node] & bit):
            return self.ZERO
        key = (node, v)
        hit = self._dcache.get(key)
        if hit is not None:
            return hit
        op = self.op[node]
        a = self.args[node]
        if op == VAR:
            r = self.ONE if node == v else self.ZERO
        elif op == ADD:
            r = self.add(self._d(a[0], v, bit), self._d(a[1], v, bit))
        elif op == SUB:
            r = self.sub(self._d(a[0], v, bit), self._d(a[1], v, bit))
        elif op == NEG:
            r = self.neg(self._d(a[0], v, bit))
        elif op == MUL:
            r = self.add(self.mul(self._d(a[0], v, bit), a[1]), self.mul(a[0], self._d(a[1], v, bit)))
        elif op == RECIP:
            r = self.neg(self.mul(self.mul(node, node), self._d(a[0], v, bit)))
        elif op == EXP:
            r = self.mul(node, self._d(a[0], v, bit))
        elif op == LOG:
            r = self.mul(self._d(a[0], v, bit), self.recip(a[0]))
        elif op == SELECT:
            r = self.select(a[0], self._d(a[1], v, bit), self._d(a[2], v, bit))
        elif op == FACT:
            r = self.mul(node, self._d(a[1], v, bit))
        else:
            raise ValueError(f"cannot differentiate {OPNAMES[op]}")
        self._dcache[key] = r
        return r

    def subs(self, node: int, mapping: Dict[int, int]) -> int:
        """Replace VAR nodes by other nodes (memoised per mapping)."""
        mkey = tuple(sorted(mapping.items()))
        mask = 0
        for k in mapping:
            mask |= 1 << self.var_bit[k]
        return self._subs(node, mapping, mkey, mask)

    def _subs(self, node, mapping, mkey, mask):
        if not (self.deps[node] & mask):
            return node
        key = (node, mkey)
        hit = self._scache.get(key)
        if hit is not None:
            return hit
        op = self.op[node]
        a = self.args[node]
        s = lambda x: self._subs(x, mapping, mkey, mask)  # noqa: E731
        if op == VAR:
            r = mapping.get(node, node)
        elif op == ADD:
            r = self.add(s(a[0]), s(a[1]))
        elif op == SUB:
            r = self.sub(s(a[0]), s(a[1]))
        elif op == NEG:
            r = self.neg(s(a[0]))
        elif op == MUL:
            r = self.mul(s(a[0]), s(a[1]))
        elif op == RECIP:
            r = self.recip(s(a[0]))
        elif op == EXP:
            r = self.exp(s(a[0]))
        elif op == LOG:
            r = self.log(s(a[0]))
        elif op == SELECT:
            cx, cc = self.args[a[0]]
            cond = self.lt(s(cx), cc) if self.deps[cx] & mask else a[0]
            r = self.select(cond, s(a[1]), s(a[2]))
        elif op == FACT:
            r = self.fact(s(a[0]), s(a[1]))
        else:
            raise ValueError(OPNAMES[op])
        self._scache[key] = r
        return r

    def depends_on(self, node, v):
        return bool(self.deps[node] & (1 << self.var_bit[v]))

    # ------------------------------------------------------------ evaluation
    def evaluate(self, outputs, env: Dict[int, float], fns=None):
        """Evaluate nodes in Python (float or complex), for compiler tests.
        ``env`` maps VAR node ids to values; placeholders may map to nodes via
        ``fns`` = {var: node} and are evaluated recursively."""
        import cmath
        fns = fns or {}
        memo: Dict[int, object] = {}

        def ev(i):
            if i in memo:
                return memo[i]
            stack = [(i, False)]
            while stack:
                n, ready = stack.pop()
                if n in memo:
                    continue
                op = self.op[n]
                a = self.args[n]
                if op == VAR and n in fns:
                    kids = [fns[n]]
                elif op == FACT:
                    kids = [a[0]]
                elif op == LT:
                    kids = [a[0]]
                elif op in (CONST, VAR):
                    kids = []
                else:
                    kids = list(a)
                if not ready:
                    stack.append((n, True))
                    for k in kids:
                        if k not in memo:
                            stack.append((k, False))
                    continue
                if op == CONST:
                    r = self.val[n]
                elif op == VAR:
                    r = memo[fns[n]] if n in fns else env[n]
                elif op == ADD:
                    r = memo[a[0]] + memo[a[1]]
                elif op == SUB:
                    r = memo[a[0]] - memo[a[1]]
                elif op == MUL:
                    r = memo[a[0]] * memo[a[1]]
                elif op == NEG:
                    r = -memo[a[0]]
                elif op == RECIP:
                    r = 1.0 / memo[a[0]]
                elif op == EXP:
                    x = memo[a[0]]
                    r = cmath.exp(x) if isinstance(x, complex) else math.exp(x)
                elif op == LOG:
                    x = memo[a[0]]
                    r = cmath.log(x) if isinstance(x, complex) else math.log(x)
                elif op == LT:
                    x = memo[a[0]]
                    r = (x.real if isinstance(x, complex) else x) < a[1]
                elif op == SELECT:
                    r = memo[a[1]] if memo[a[0]] else memo[a[2]]
                elif op == FACT:
                    r = memo[a[0]]
                memo[n] = r
            return memo[i]

        return [ev(o) for o in outputs]
