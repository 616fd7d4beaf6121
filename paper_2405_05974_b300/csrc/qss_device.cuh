// Device math used by the generated mechanism code (sm_103a, FP64).
//
// The generated straight-line code calls only qss_exp, qss_log and qss_rcp for
// its non-elementary operations; everything else is add/mul/fma.
#pragma once
#include <cuda_runtime.h>

__device__ __forceinline__ double qss_rcp(double x) { return __drcp_rn(x); }

#ifndef QSS_TABLE_EXP
__device__ __forceinline__ double qss_exp(double x) { return exp(x); }
#endif
__device__ __forceinline__ double qss_log(double x) { return log(x); }
