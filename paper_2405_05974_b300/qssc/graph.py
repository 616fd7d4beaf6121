"""QSS dependency digraph and its strongly connected components.

Section 2.3 and Appendix B: QSS species m *needs* QSS species n when the
production rate of m contains a term proportional to C_n (structurally, a
nonzero A_mn).  Strongly connected components (SCCs) are found with Tarjan's
algorithm in one depth-first traversal over an adjacency list, O(V + E); the
components come out in an order where each appears after the components it
needs, which is the order of algebraic resolution (back substitution between
components, elimination inside each).  The traversal here is iterative (an
explicit stack of (vertex, next-child) frames) so that it needs no recursion.
"""
from __future__ import annotations

from typing import List, Sequence


def tarjan_scc(adj: Sequence[Sequence[int]]) -> List[List[int]]:
    """SCCs of the digraph ``adj`` (adj[v] = vertices that v needs), in an
    order in which every component follows all components it needs."""
    n = len(adj)
    index = [-1] * n
    low = [0] * n
    on_stack = [False] * n
    stack: List[int] = []
    comps: List[List[int]] = []
    counter = 0
    for root in range(n):
        if index[root] >= 0:
            continue
        frames = [(root, 0)]
        index[root] = low[root] = counter
        counter += 1
        stack.append(root)
        on_stack[root] = True
        while frames:
            v, i = frames[-1]
            if i < len(adj[v]):
                frames[-1] = (v, i + 1)
                w = adj[v][i]
                if index[w] < 0:
                    index[w] = low[w] = counter
                    counter += 1
                    stack.append(w)
                    on_stack[w] = True
                    frames.append((w, 0))
                elif on_stack[w]:
                    low[v] = min(low[v], index[w])
                continue
            frames.pop()
            if frames:
                parent = frames[-1][0]
                low[parent] = min(low[parent], low[v])
            if low[v] == index[v]:
                comp = []
                while True:
                    w = stack.pop()
                    on_stack[w] = False
                    comp.append(w)
                    if w == v:
                        break
                comps.append(sorted(comp))
    return comps


def condensed_edges(adj, comps):
    """Edges between components (component index pairs, u needs v)."""
    where = {}
    for ci, c in enumerate(comps):
        for v in c:
            where[v] = ci
    out = set()
    for u, nbrs in enumerate(adj):
        for w in nbrs:
            if where[u] != where[w]:
                out.add((where[u], where[w]))
    return sorted(out)
