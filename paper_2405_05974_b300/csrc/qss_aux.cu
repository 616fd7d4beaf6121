#include "qss_device.cuh"

// Auxiliary kernels of libqss (compiled to qss_aux.cubin for sm_103a).
//
// qss_fp64_fma_probe: dependent FMA chains, 8 independent chains per thread,
// for the FP64 roofline denominator.  Each thread performs iters * 8 FMAs and
// writes one value so that nothing is eliminated.
extern "C" __global__ void qss_fp64_fma_probe(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
  double x4 = x0 + 4.0, x5 = x0 + 5.0, x6 = x0 + 6.0, x7 = x0 + 7.0;
  for (int it = 0; it < iters; ++it) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// qss_fp64_pipe_probe: the FP64 pipe's behaviour for kernel design.  Lanes
// with lane % stride == 0 run 8 FMAs per iteration, as 8 independent chains
// (dep = 0) or as one dependent chain (dep = 1); the other lanes skip them,
// so a stride of 2, 4, 8 runs warps with 16, 8, 4 active lanes.  Each thread
// writes one value so that nothing is eliminated.
extern "C" __global__ void qss_fp64_pipe_probe(double* out, int iters, double a, double b, int stride,
                                               int dep) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
  double x4 = x0 + 4.0, x5 = x0 + 5.0, x6 = x0 + 6.0, x7 = x0 + 7.0;
  if ((threadIdx.x & 31) % stride == 0) {
    if (dep) {
      for (int it = 0; it < iters; ++it) {
        x0 = fma(x0, a, b); x0 = fma(x0, a, b); x0 = fma(x0, a, b); x0 = fma(x0, a, b);
        x0 = fma(x0, a, b); x0 = fma(x0, a, b); x0 = fma(x0, a, b); x0 = fma(x0, a, b);
      }
    } else {
      for (int it = 0; it < iters; ++it) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
      }
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// Writes `n` doubles (used to evict the L2 between timed iterations).
extern "C" __global__ void qss_l2_flush(double* buf, long long n, double v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    buf[i] = v + (double)i;
}

// Elementwise evaluation of the device math used by generated code, for tests:
// fn 0 = qss_exp_table, 1 = library exp, 2 = qss_log_table, 3 = qss_rcp,
// 4 = library log, 5 = library reciprocal (correctly rounded).
extern "C" __global__ void qss_math_probe(int fn, long long n, const double* __restrict__ x,
                                          double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  double r;
  switch (fn) {
    case 0: r = qss_exp_table(v); break;
    case 1: r = exp(v); break;
    case 2: r = qss_log_table(v); break;
    case 4: r = log(v); break;
    case 5: r = __drcp_rn(v); break;
    default: r = qss_rcp(v); break;
  }
  y[i] = r;
}
