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

extern "C" int qss_measure_fp64_pipe(int device, int warps_per_sm, int active_lanes, int dependent,
                                     double* lane_tflops, double* cycles_per_warp_fma) {
  if (!lane_tflops || warps_per_sm < 1 || warps_per_sm > 32 ||
      (active_lanes != 32 && active_lanes != 16 && active_lanes != 8 && active_lanes != 4 && active_lanes != 1))
    return fail(QSS_ERR_INVALID_ARG, "bad argument");
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
  int sms = 0, clk_khz = 0;
  CUdeviceptr out = 0;
  CUevent e0 = nullptr, e1 = nullptr;
  int status = QSS_OK;
  do {
    if ((r = drv().cuModuleGetFunction(&f, mod, "qss_fp64_pipe_probe")) != CUDA_SUCCESS) break;
    if ((r = drv().cuDeviceGetAttribute(&sms, CU_DEVICE_ATTRIBUTE_MULTIPROCESSOR_COUNT, dev))) break;
    if ((r = drv().cuDeviceGetAttribute(&clk_khz, CU_DEVICE_ATTRIBUTE_CLOCK_RATE, dev))) break;
    const int block = 32 * warps_per_sm, grid = sms;
    if ((r = drv().cuMemAlloc(&out, (size_t)grid * block * sizeof(double)))) break;
    if ((r = drv().cuEventCreate(&e0, CU_EVENT_DEFAULT)) || (r = drv().cuEventCreate(&e1, CU_EVENT_DEFAULT))) break;
    double a = 1.0000001, b = 1e-7;
    int iters = 64, stride = 32 / active_lanes, dep = dependent ? 1 : 0;
    float ms = 0.f;
    for (int attempt = 0; attempt < 20; ++attempt) {   // one launch of >= ~20 ms
      void* args[] = {&out, &iters, &a, &b, &stride, &dep};
      if ((r = drv().cuEventRecord(e0, 0))) break;
      if ((r = drv().cuLaunchKernel(f, grid, 1, 1, block, 1, 1, 0, 0, args, nullptr))) break;
      if ((r = drv().cuEventRecord(e1, 0))) break;
      if ((r = drv().cuEventSynchronize(e1))) break;
      if ((r = drv().cuEventElapsedTime(&ms, e0, e1))) break;
      if (ms >= 20.f || iters > (1 << 24)) break;
      iters *= 2;
    }
    if (r) break;
    const double fmas = 8.0 * (double)iters;   // per active lane
    *lane_tflops = 2.0 * fmas * active_lanes * warps_per_sm * grid / (ms * 1e-3) / 1e12;
    // SM cycles per warp-wide FMA instruction on one SM sub-partition (4 per
    // SM), at the device's nominal clock
    if (cycles_per_warp_fma)
      *cycles_per_warp_fma = (ms * 1e-3) * (clk_khz * 1e3) * 4.0 / (fmas * warps_per_sm);
  } while (0);
  if (r != CUDA_SUCCESS) status = cu_fail(r, "fp64 pipe probe");
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
