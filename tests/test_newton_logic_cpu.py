"""CPU emulation of the index logic of the FP32 factorisation in the
mixed-precision Newton update (qss_solve_fp32ir / qss_lu32_step in
csrc/qss_newton.cuh), against numpy's dense solve.

The device code keeps row r = lane + 32 slot of the scaled matrix in
registers, shifted left one column per pivot step (the pivot column is always
entry 0), and runs the pivot steps in four phases of decreasing static width
W = n - k0 (k0 = ceil(n ph / 4)): every entry at or beyond the phase's width
must already be zero when the phase starts.  This emulation follows the same
steps with the same widths (argmax on the magnitude bits, lowest row on ties;
multipliers and U rows in LU[r][k]; forward substitution over the pivot
order, column-oriented back substitution), asserts that invariant, and
solves random and stiff systems for n = 1..63 to FP32 rounding.
"""
import numpy as np
import pytest


def phases(n):
    k1, k2, k3 = (n + 3) // 4, (2 * n + 3) // 4, (3 * n + 3) // 4
    return [(0, k1, n), (k1, k2, n - k1), (k2, k3, n - k2), (k3, n, n - k3)]


def factor_and_solve(M, b):
    n = M.shape[0]
    f = np.float32
    A = M.astype(f).copy()
    ordk = np.full(n, -1)
    LU = np.zeros((n, n + 1), dtype=f)
    piv, pinv = np.zeros(n, int), np.zeros(n, f)
    for k0, k1, W in phases(n):
        if k0 < k1:
            assert not A[:, W:].any(), "entries beyond the phase's width are not zero"
        for k in range(k0, k1):
            keys = np.where(ordk < 0, np.abs(A[:, 0]).view(np.int32), -1)
            brow = int(np.argmax(keys))               # first (lowest) row of the largest key
            assert keys[brow] > 0
            p = A[brow, :W].copy()
            inv = f(1) / p[0]
            piv[k], pinv[k] = brow, inv
            m = min(W, n - k)
            LU[brow, k:k + m] = p[:m]
            ordk[brow] = k
            for r in range(n):
                el = ordk[r] < 0
                lr = A[r, 0] * inv if el else f(0)
                if el:
                    LU[r, k] = lr
                A[r, :W - 1] = (-lr * p[1:W] + A[r, 1:W]).astype(f)
                A[r, W - 1] = 0
    # forward substitution over the pivot order
    z = b.astype(f).copy()
    for k in range(n):
        zp = z[piv[k]]
        for r in range(n):
            if ordk[r] > k:
                z[r] = f(z[r] - LU[r, k] * zp)
    # back substitution: x_k from the pivot row of step k, column oriented
    x = np.zeros(n, f)
    for k in range(n - 1, -1, -1):
        xk = f(z[piv[k]] * pinv[k])
        x[k] = xk
        for r in range(n):
            if ordk[r] < k:
                z[r] = f(z[r] - LU[r, k] * xk)
    return x


@pytest.mark.parametrize("n", list(range(1, 64)))
def test_phased_fp32_factorisation_solves(n):
    rng = np.random.default_rng(n)
    for kind in ("random", "stiff"):
        if kind == "random":
            M = rng.standard_normal((n, n))
        else:   # I - h J with a wide spread of scales (as the Newton matrix)
            J = rng.standard_normal((n, n)) * 10.0 ** rng.uniform(-3, 3, (n, 1))
            M = np.eye(n) - 1e-2 * J
        b = rng.standard_normal(n)
        x = factor_and_solve(M, b)
        ref = np.linalg.solve(M, b)
        cond = np.linalg.cond(M)
        assert np.max(np.abs(x - ref)) <= 1e-4 * cond * np.max(np.abs(ref)), (kind, n, cond)
