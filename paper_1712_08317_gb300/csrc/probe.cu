// Throughput probes of the SM pipes the reconstruction runs on (measurement aid
// for the roofline of the FP32 / FP64 kernels; no counterpart in the method).
//
// Every thread runs kChains independent dependency chains of one instruction
// for `iters` iterations, so the pipe, not the latency, sets the rate:
//   kind 0  FP32 fused multiply-add, scalar   (fma.rn.f32)
//   kind 1  FP32 fused multiply-add, paired   (__ffma2_rn: two FMAs per instruction)
//   kind 2  FP64 fused multiply-add           (fma.rn.f64)
//   kind 3  FP32 approximate reciprocal        (rcp.approx.ftz.f32, the MUFU pipe; each also
//           takes one FP32 add on the FMA pipe, whose rate is far higher)
// An FMA counts as one operation.  The chains' results are stored, so nothing
// is dead code.
#include <cuda_runtime.h>

#include <string>

#include "weno3.h"

namespace weno {
int set_error(int code, const std::string& msg);  // solver.cu: the message weno_last_error returns
}

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__global__ void __launch_bounds__(kThreads) k_probe_ffma(float b, float c, int iters, float* out) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_ffma2(float b, float c, int iters, float* out) {
  float2 a[kChains];
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_dfma(double b, double c, int iters, float* out) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

__device__ __forceinline__ float probe_rcp(float x) {
  float r;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__global__ void __launch_bounds__(kThreads) k_probe_rcp(float b, float c, int iters, float* out) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = b + c * (float)(threadIdx.x + k + 1);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = probe_rcp(a[k] + c);  // not an involution: nothing folds
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int probe_fail(int code, const std::string& msg) { return weno::set_error(code, msg); }

}  // namespace

extern "C" {

int weno_probe_peak(int32_t kind, int32_t iters, void* cuda_stream, double* ops, float* ms) {
  if (kind < 0 || kind > 3 || iters <= 0 || !ops || !ms) return probe_fail(WENO_EINVAL, "weno_probe_peak: bad argument");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return probe_fail(WENO_ECUDA, "weno_probe_peak: no device");
  const int blocks = nsm * kBlocksPerSm;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = WENO_OK;
  auto launch = [&]() {
    switch (kind) {
      case 0: k_probe_ffma<<<blocks, kThreads, 0, st>>>(1.0000001f, 1e-7f, iters, out); break;
      case 1: k_probe_ffma2<<<blocks, kThreads, 0, st>>>(1.0000001f, 1e-7f, iters, out); break;
      case 2: k_probe_dfma<<<blocks, kThreads, 0, st>>>(1.0000000001, 1e-10, iters, out); break;
      default: k_probe_rcp<<<blocks, kThreads, 0, st>>>(0.5f, 0.25f, iters, out); break;
    }
  };
  float best = 1e30f;
  if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(float)) != cudaSuccess) {
    return probe_fail(WENO_ENOMEM, "weno_probe_peak: cudaMalloc failed");
  }
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = probe_fail(WENO_ECUDA, "weno_probe_peak: cudaEventCreate failed");
  } else {
    launch();  // warm-up
    for (int r = 0; r < 3 && rc == WENO_OK; ++r) {
      cudaEventRecord(e0, st);
      launch();
      cudaEventRecord(e1, st);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) {
        rc = probe_fail(WENO_ECUDA, std::string("weno_probe_peak: ") + cudaGetErrorString(e));
        break;
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      best = t < best ? t : best;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != WENO_OK) return rc;
  *ms = best;
  *ops = (double)blocks * kThreads * (double)iters * kChains * (kind == 1 ? 2.0 : 1.0);
  return WENO_OK;
}

}  // extern "C"
