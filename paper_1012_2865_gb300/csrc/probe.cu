// probe.cu -- measurement aid, not part of the method: the rate at which
// the GPU completes atomic reductions (RED) into one array, which is the
// roof of the trace's k_ph / Gamma deposits (Eqs. "kph", "gamma") when the
// rate arrays stay resident in L2.
//
// Every thread of a full-occupancy grid issues `per_thread` reductions of
// 1 into elements of a power-of-two array chosen by a counter-based hash of
// (thread, iteration), so consecutive reductions of a warp land on
// unrelated cache lines -- the access pattern of lanes following diverging
// rays.  The result is not read, so the compiler emits RED (no return
// value).  The rate is the best of several event-timed launches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "rt.h"

namespace {

thread_local std::string g_probe_error;

int probe_fail(int code, const char* what, cudaError_t e = cudaSuccess) {
  char buf[256];
  snprintf(buf, sizeof buf, "rt_probe_red: %s%s%s", what, e != cudaSuccess ? ": " : "",
           e != cudaSuccess ? cudaGetErrorString(e) : "");
  g_probe_error = buf;
  return code;
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

template <class T>
__global__ void red_kernel(T* a, uint32_t mask, int per_thread) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t h = mix32(tid * 0x9e3779b9U + 0x632be5abU);
  for (int i = 0; i < per_thread; ++i) {
    h = mix32(h + (uint32_t)i);
    atomicAdd(&a[h & mask], (T)1);
  }
}

}  // namespace

extern "C" {

const char* rt_probe_last_error(void) { return g_probe_error.c_str(); }

int rt_probe_red(int device, int dtype, uint64_t words, double* reds_per_s) {
  if (!reds_per_s) return probe_fail(RT_ERR_INVALID_ARG, "reds_per_s is NULL");
  if (dtype != RT_DTYPE_F32 && dtype != RT_DTYPE_F64) return probe_fail(RT_ERR_INVALID_ARG, "dtype");
  if (words < 1024 || words > (1ULL << 30) || (words & (words - 1)) != 0)
    return probe_fail(RT_ERR_INVALID_ARG, "words must be a power of two in [2^10, 2^30]");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return probe_fail(RT_ERR_INVALID_ARG, "cudaSetDevice", e);
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
    return probe_fail(RT_ERR_CUDA, "device attribute", e);
  const int block = 256;
  int per_sm = 0;
  e = dtype == RT_DTYPE_F32
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, red_kernel<float>, block, 0)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, red_kernel<double>, block, 0);
  if (e != cudaSuccess) return probe_fail(RT_ERR_CUDA, "occupancy", e);
  if (per_sm < 1) per_sm = 1;
  const int grid = per_sm * sms;
  const int per_thread = 256;
  const size_t bytes = (size_t)words * (dtype == RT_DTYPE_F32 ? 4 : 8);
  void* a = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best = 0.0;
  int rc = RT_OK;
  if ((e = cudaMalloc(&a, bytes)) != cudaSuccess) return probe_fail(RT_ERR_OOM, "cudaMalloc", e);
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
      (e = cudaMemsetAsync(a, 0, bytes, st)) != cudaSuccess) {
    rc = probe_fail(RT_ERR_CUDA, "set-up", e);
  }
  // one untimed launch brings the array into L2, then the best of five
  for (int rep = 0; rep < 6 && rc == RT_OK; ++rep) {
    cudaEventRecord(e0, st);
    if (dtype == RT_DTYPE_F32)
      red_kernel<float><<<grid, block, 0, st>>>((float*)a, (uint32_t)(words - 1), per_thread);
    else
      red_kernel<double><<<grid, block, 0, st>>>((double*)a, (uint32_t)(words - 1), per_thread);
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
      rc = probe_fail(RT_ERR_CUDA, "probe launch", e);
      break;
    }
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
      rc = probe_fail(RT_ERR_CUDA, "event timing", e);
      break;
    }
    const double rate = (double)grid * block * per_thread / (ms * 1e-3);
    if (rep > 0 && rate > best) best = rate;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(a);
  if (rc == RT_OK) {
    *reds_per_s = best;
    g_probe_error.clear();
  }
  return rc;
}

}  // extern "C"
