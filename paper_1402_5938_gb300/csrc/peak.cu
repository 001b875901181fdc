// Measured arithmetic peaks of the current device, the denominators of the operator's
// rooflines: FP64 and FP32 fused multiply-add loops on the CUDA cores, and the FP64
// tensor-core MMA (m8n8k4) for comparison with the FP64 FMA rate. Each kernel runs
// independent dependency chains in every thread of a grid that fills every SM several
// times over, long enough (tens of milliseconds) that launch overhead does not matter;
// the rate is the best of three timed launches with CUDA events after a warm-up launch.
#include <math.h>

#include <string>

#include "common.cuh"

namespace hmg {

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == (T)-12345.0) out[blockIdx.x] = s;  // never true for these inputs; keeps the loop live
}

// FP64 tensor-core MMA: D = A B + C with 8x8x4 FP64 tiles per warp, 4 independent accumulators.
__global__ void __launch_bounds__(256) k_dmma_peak(double* out, int iters) {
  double a = 1e-3 * (threadIdx.x & 7), b = 1.0 - 1e-9 * (threadIdx.x & 3);
  double d[4][2];
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k][0] = d[k][1] = 0.0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(d[k][0]), "+d"(d[k][1])
                     : "d"(a), "d"(b));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += d[k][0] + d[k][1];
  if (s == -12345.0) out[blockIdx.x] = s;
}

// Both at once: warps 0-3 of each block run the FP64 FMA chains, warps 4-7 the FP64 MMAs; if the
// two used separate units the combined rate would exceed either alone.
__global__ void __launch_bounds__(256) k_fp64_mixed_peak(double* out, int iters_f, int iters_m) {
  const int w = threadIdx.x >> 5;
  double s = 0.0;
  if (w < 4) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters_f; ++i) {
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], 1.0 - 1e-12, 1e-9);
    }
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
  } else {
    double a = 1e-3 * (threadIdx.x & 7), b = 1.0 - 1e-9 * (threadIdx.x & 3);
    double d[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k][0] = d[k][1] = 0.0;
    for (int i = 0; i < iters_m; ++i) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                       : "+d"(d[k][0]), "+d"(d[k][1])
                       : "d"(a), "d"(b));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) s += d[k][0] + d[k][1];
  }
  if (s == -12345.0) out[blockIdx.x] = s;
}

template <typename K>
cudaError_t best_of(K launch, double work, double* rate) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  double best = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    if ((e = cudaEventRecord(e0, 0)) != cudaSuccess) break;
    launch();
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaEventRecord(e1, 0)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
    if (rep > 0 && ms > 0.f) best = fmax(best, work / (ms * 1e-3));   // rep 0 is the warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *rate = best;
  return e;
}

}  // namespace

}  // namespace hmg

using namespace hmg;

extern "C" hmg_status hmg_measure_peak(int what, double* tflops) {
  if (!tflops || what < 0 || what > 3) {
    set_error("hmg_measure_peak: what must be 0 (FP64 FMA), 1 (FP32 FMA), 2 (FP64 MMA) or 3 (both FP64 at once)");
    return HMG_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || sms <= 0) {
    set_error(std::string("hmg_measure_peak: ") + cudaGetErrorString(e));
    return HMG_EDEVICE;
  }
  double* out = nullptr;
  if ((e = dev_alloc((void**)&out, 8 * 4096 * sizeof(double), 0)) != cudaSuccess) {
    set_error("hmg_measure_peak: device allocation failed");
    return HMG_ENOMEM;
  }
  const int threads = 256, blocks = sms * 8;
  double rate = 0.0;
  if (what == 0) {
    const int iters = 2000;  // ~8 GFLOP: tens of ms at the FP64 rate
    const double work = 2.0 * kChains * 8 * (double)iters * threads * blocks;
    e = best_of([&] { k_fma_peak<double><<<blocks, threads>>>(out, iters, 1.0 - 1e-12, 1e-9); }, work, &rate);
  } else if (what == 1) {
    const int iters = 60000;
    const double work = 2.0 * kChains * 8 * (double)iters * threads * blocks;
    e = best_of([&] { k_fma_peak<float><<<blocks, threads>>>((float*)out, iters, 1.0f - 1e-6f, 1e-7f); }, work,
                &rate);
  } else if (what == 2) {
    const int iters = 1000;
    const double work = 2.0 * 8 * 8 * 4 * 16.0 * iters * (threads / 32) * blocks;
    e = best_of([&] { k_dmma_peak<<<blocks, threads>>>(out, iters); }, work, &rate);
  } else {
    const int itf = 2000, itm = 1000;  // about equal time for each half alone
    const double work = (2.0 * kChains * 8 * (double)itf * 32 * 4 + 2.0 * 8 * 8 * 4 * 16.0 * itm * 4) * blocks;
    e = best_of([&] { k_fp64_mixed_peak<<<blocks, threads>>>(out, itf, itm); }, work, &rate);
  }
  add_launches(4);
  dev_free(out, 0);
  cudaError_t e2 = cudaStreamSynchronize(0);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    set_error(std::string("hmg_measure_peak: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    return HMG_EDEVICE;
  }
  *tflops = rate / 1e12;
  return HMG_OK;
}
