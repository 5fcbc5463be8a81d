// FMA throughput of the device in FP64 and FP32, and its FP64 tensor-core
// (MMA) rate (instrumentation: the denominators of the FP64 KKT matvec's pipe
// fraction, and the check of whether FP64 MMA could serve the dense panels;
// the paper has no counterpart).  Every thread runs 8 independent multiply-add chains
// x <- x a + b for `iters` rounds, all in registers, so the count of
// multiply-adds is exact and nothing else limits the rate; the time is
// taken with CUDA events on the given stream.

#include "internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_chains(T* __restrict__ out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1) out[blockIdx.x] = s;   // never true: keeps the chains live
}

template <typename T>
kkt_status run(int iters, int blocks, T* out, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  KKT_TRY_CUDA(cudaEventCreate(&e0));
  KKT_TRY_CUDA(cudaEventCreate(&e1));
  fma_chains<T><<<blocks, kPeakThreads, 0, s>>>(out, iters, (T)0.999999, (T)1e-3);   // warm-up
  KKT_TRY_CUDA(cudaEventRecord(e0, s));
  fma_chains<T><<<blocks, kPeakThreads, 0, s>>>(out, iters, (T)0.999999, (T)1e-3);
  KKT_TRY_CUDA(cudaEventRecord(e1, s));
  KKT_COUNT(2);
  KKT_TRY_CUDA(cudaGetLastError());
  KKT_TRY_CUDA(cudaEventSynchronize(e1));
  KKT_TRY_CUDA(cudaEventElapsedTime(ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return KKT_OK;
}

// FP64 matrix multiply-accumulate: every warp runs kChains independent chains
// D <- A B + D of the m8n8k4 FP64 warp-level MMA (512 flops per instruction
// and warp), operands in registers.
__global__ void __launch_bounds__(kPeakThreads) dmma_chains(double* __restrict__ out, int iters) {
  const double a = 1.0 + 1e-6 * threadIdx.x, b = 1e-3;
  double d0[kChains], d1[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) d0[c] = d1[c] = (double)c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d0[c]), "+d"(d1[c])
                   : "d"(a), "d"(b));
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += d0[c] + d1[c];
  if (s == -1.0) out[blockIdx.x] = s;   // never true: keeps the chains live
}

}  // namespace

// FP64 tensor-core (MMA) rate of the current device; see stkkt.h.
extern "C" kkt_status kkt_mma_peak(double* tflops, double* ms, void* stream) {
  if (!tflops) {
    set_error("kkt_mma_peak: a tflops output is required");
    return KKT_ERR_ARG;
  }
  int dev = 0, nsm = 0;
  KKT_TRY_CUDA(cudaGetDevice(&dev));
  KKT_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 8, iters = 1024;
  double* out = nullptr;
  KKT_TRY_CUDA(cudaMalloc(&out, blocks * sizeof(double)));
  const cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  float t = 0.f;
  kkt_status st = KKT_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = KKT_ERR_CUDA;
  if (st == KKT_OK) {
    dmma_chains<<<blocks, kPeakThreads, 0, s>>>(out, iters);   // warm-up
    cudaEventRecord(e0, s);
    dmma_chains<<<blocks, kPeakThreads, 0, s>>>(out, iters);
    cudaEventRecord(e1, s);
    KKT_COUNT(2);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
      st = KKT_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaFree(out);
  if (st != KKT_OK) {
    set_error("kkt_mma_peak: CUDA error");
    return st;
  }
  const double flops = 512.0 * kChains * (double)iters * (kPeakThreads / 32) * blocks;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return KKT_OK;
}

extern "C" kkt_status kkt_fma_peak(int precision, double* tflops, double* ms, void* stream) {
  if ((precision != 64 && precision != 32) || !tflops) {
    set_error("kkt_fma_peak: precision 64 or 32 and a tflops output");
    return KKT_ERR_ARG;
  }
  int dev = 0, nsm = 0;
  KKT_TRY_CUDA(cudaGetDevice(&dev));
  KKT_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 8;                       // 2048 threads per SM
  const int iters = precision == 64 ? 4096 : 65536; // ~10-20 ms either way
  void* out = nullptr;
  KKT_TRY_CUDA(cudaMalloc(&out, blocks * sizeof(double)));
  float t = 0.f;
  const cudaStream_t s = (cudaStream_t)stream;
  const kkt_status st = precision == 64 ? run<double>(iters, blocks, (double*)out, s, &t)
                                        : run<float>(iters, blocks, (float*)out, s, &t);
  cudaFree(out);
  if (st != KKT_OK) return st;
  const double flops = 2.0 * kChains * (double)iters * kPeakThreads * blocks;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return KKT_OK;
}
