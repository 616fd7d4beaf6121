"""Jacobian quality and structure figures of Section 3.2, on device tensors.

These are reporting helpers (reductions over cells of Jacobians produced by
the kernels), not part of the evaluation path.  Jacobians use the library's
layout: jac[(i * n + j), c] for cell c, n = N + 1.
"""
from __future__ import annotations

import torch


def frobenius_error(JA: torch.Tensor, JFD: torch.Tensor, ncells: int = None) -> float:
    """Eq. (frobErr): the mean over cells of ||J_A - J_FD||_F / ||J_FD||_F,
    the norm taken over all rows and columns."""
    nc = JA.shape[1] if ncells is None else ncells
    a, b = JA[:, :nc], JFD[:, :nc]
    num = torch.linalg.vector_norm(a - b, dim=0)
    den = torch.linalg.vector_norm(b, dim=0)
    return float((num / den).mean())


def nonzero_fraction(J: torch.Tensor, N: int, ncells: int = None) -> float:
    """Fraction of nonzero entries in the first N rows and N columns (the
    species block), averaged over cells (the statistic of Table memQSS)."""
    nc = J.shape[1] if ncells is None else ncells
    n = N + 1
    blk = J[:, :nc].reshape(n, n, nc)[:N, :N]
    return float((blk != 0).to(torch.float64).mean())
