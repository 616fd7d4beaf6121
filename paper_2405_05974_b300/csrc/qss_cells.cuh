// Cell layout shared by the per-cell kernels (one thread per cell).
//
// Layout (all FP64, structure of arrays with leading dimension ld >= ncells):
//   rho[ld], T[ld], Y[k * ld + c] (k < N), wdot[k * ld + c], Tdot[ld],
//   jac[(i * (N + 1) + j) * ld + c]  (row i = d f_i, column j = d/d phi_j,
//   phi = (C_1..C_N, T)).
// Consecutive threads take consecutive cells, so every load and store of a
// warp is one contiguous 256-byte segment.
#pragma once

#ifndef QSS_BLOCK
#define QSS_BLOCK 128
#endif

// QSS_SMEM_SPILL=1 lets ptxas place part of a kernel's register spills in
// shared memory before local memory (the enable_smem_spilling PTX pragma of
// CUDA 13); the Jacobian kernels use no shared memory otherwise.  A tuning
// option: ptxas moves about 100 bytes per thread there.
#if defined(QSS_SMEM_SPILL) && QSS_SMEM_SPILL
#define QSS_SPILL_TO_SMEM() asm volatile(".pragma \"enable_smem_spilling\";")
#else
#define QSS_SPILL_TO_SMEM() do { } while (0)
#endif

// C_k = rho Y_k / W_k for the transported species.
__device__ __forceinline__ void qss_unpack(long long c, long long ld, const double* __restrict__ rho,
                                           const double* __restrict__ Y, double* C) {
  const double r = __ldg(rho + c);
#pragma unroll
  for (int k = 0; k < QSS_N; ++k) C[k] = r * __ldg(Y + k * ld + c) * qss_inv_W[k];
}
