// FP64 throughput measurement (roofline denominator) on the auxiliary cubin.
#include <cuda.h>

#include <string>

#include "qss_internal.h"
#include "qss_driver.h"

using namespace qss;

extern "C" int qss_measure_fp64_peak(int device, int millis, double* tflops) {
  if (!tflops || millis <= 0) return fail(QSS_ERR_INVALID_ARG, "bad argument");
  CUdevice dev;
  CUcontext ctx;
  int rc = ctx_for_device(device, &dev, &ctx);
  if (rc) return rc;
  CUmodule mod;
  std::string path = lib_dir() + "/qss_aux.cubin";
  CUresult r = drv().cuModuleLoad(&mod, path.c_str());
  if (r != CUDA_SUCCESS) {
    drv().cuDevicePrimaryCtxRelease(dev);
    return cu_fail(r, "drv().cuModuleLoad(qss_aux.cubin)");
  }
  CUfunction f;
  int sms = 0;
  CUdeviceptr out = 0;
  CUevent e0 = nullptr, e1 = nullptr;
  int status = QSS_OK;
  do {
    if ((r = drv().cuModuleGetFunction(&f, mod, "qss_fp64_fma_probe")) != CUDA_SUCCESS) break;
    if ((r = drv().cuDeviceGetAttribute(&sms, CU_DEVICE_ATTRIBUTE_MULTIPROCESSOR_COUNT, dev))) break;
    const int block = 256, grid = sms * 4;
    if ((r = drv().cuMemAlloc(&out, (size_t)grid * block * sizeof(double)))) break;
    if ((r = drv().cuEventCreate(&e0, CU_EVENT_DEFAULT)) || (r = drv().cuEventCreate(&e1, CU_EVENT_DEFAULT))) break;
    double a = 1.0000001, b = 1e-7;
    int iters = 256;
    float ms = 0.f;
    // grow the iteration count until one launch takes ~millis
    for (int attempt = 0; attempt < 16; ++attempt) {
      void* args[] = {&out, &iters, &a, &b};
      if ((r = drv().cuEventRecord(e0, 0))) break;
      if ((r = drv().cuLaunchKernel(f, grid, 1, 1, block, 1, 1, 0, 0, args, nullptr))) break;
      if ((r = drv().cuEventRecord(e1, 0))) break;
      if ((r = drv().cuEventSynchronize(e1))) break;
      if ((r = drv().cuEventElapsedTime(&ms, e0, e1))) break;
      if (ms >= 0.5f * millis || iters > (1 << 26)) break;
      iters *= 2;
    }
    if (r) break;
    double flops = 2.0 * 8.0 * (double)iters * grid * block;
    *tflops = flops / (ms * 1e-3) / 1e12;
  } while (0);
  if (r != CUDA_SUCCESS) status = cu_fail(r, "fp64 probe");
  if (e0) drv().cuEventDestroy(e0);
  if (e1) drv().cuEventDestroy(e1);
  if (out) drv().cuMemFree(out);
  drv().cuModuleUnload(mod);
  drv().cuDevicePrimaryCtxRelease(dev);
  return status;
}

extern "C" int qss_selftest_math(int device, int fn, int64_t n, const double* x, double* y,
                                 void* stream) {
  if (n < 0 || (n > 0 && (!x || !y)) || fn < 0 || fn > 5) return fail(QSS_ERR_INVALID_ARG, "bad argument");
  if (n == 0) return QSS_OK;
  CUdevice dev;
  CUcontext ctx;
  int rc = ctx_for_device(device, &dev, &ctx);
  if (rc) return rc;
  static CUmodule mod = nullptr;
  static CUfunction f = nullptr;
  if (!mod) {
    std::string path = lib_dir() + "/qss_aux.cubin";
    CU_TRY(drv().cuModuleLoad(&mod, path.c_str()));
    CU_TRY(drv().cuModuleGetFunction(&f, mod, "qss_math_probe"));
  }
  long long nn = n;
  void* args[] = {&fn, &nn, &x, &y};
  const int block = 256;
  long long grid = (n + block - 1) / block;
  CU_TRY(drv().cuLaunchKernel(f, (unsigned)grid, 1, 1, block, 1, 1, 0, (CUstream)stream, args, nullptr));
  drv().cuDevicePrimaryCtxRelease(dev);
  return QSS_OK;
}
