// CUDA driver API resolved at run time (dlopen of libcuda.so.1), so that
// libqss.so loads on machines without a GPU driver and reports QSS_ERR_CUDA
// from its calls instead of failing to load.
#pragma once
#include <cuda.h>

#define QSS_DRV_FUNCS(X)                                                                 \
  X(cuInit) X(cuDeviceGetCount) X(cuDeviceGet) X(cuDevicePrimaryCtxRetain)               \
  X(cuDevicePrimaryCtxRelease) X(cuCtxSetCurrent) X(cuCtxGetCurrent) X(cuCtxSynchronize) \
  X(cuModuleLoad) X(cuModuleUnload) X(cuModuleGetFunction) X(cuModuleGetGlobal)          \
  X(cuLaunchKernel) X(cuMemAlloc) X(cuMemFree) X(cuMemcpy2DAsync) X(cuMemcpyHtoDAsync)   \
  X(cuMemcpyDtoHAsync) X(cuMemcpyDtoDAsync) X(cuMemsetD8Async) X(cuMemsetD32Async)       \
  X(cuStreamCreate) X(cuStreamDestroy) X(cuStreamSynchronize) X(cuStreamWaitEvent)       \
  X(cuStreamQuery) X(cuEventCreate) X(cuEventDestroy) X(cuEventRecord)                   \
  X(cuEventSynchronize) X(cuEventElapsedTime) X(cuEventQuery) X(cuGetErrorString)        \
  X(cuDeviceGetAttribute) X(cuFuncGetAttribute) X(cuFuncSetAttribute) X(cuMemGetInfo)    \
  X(cuOccupancyMaxActiveBlocksPerMultiprocessor) X(cuMemHostAlloc) X(cuMemFreeHost)      \
  X(cuStreamBeginCapture) X(cuStreamEndCapture) X(cuGraphInstantiate) X(cuGraphLaunch)   \
  X(cuGraphDestroy) X(cuGraphExecDestroy)

namespace qss {
struct Driver {
#define QSS_DRV_MEMBER(f) decltype(&::f) f = nullptr;
  QSS_DRV_FUNCS(QSS_DRV_MEMBER)
#undef QSS_DRV_MEMBER
  bool ok = false;
};
// The driver table (loaded on first use; `ok` false when libcuda is absent).
Driver& drv();
}  // namespace qss
