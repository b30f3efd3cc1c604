// Throughput probes for the roofline denominators of this GPU: FP32 FMA on the CUDA cores
// and tcgen05 MMA of kind tf32 on the tensor cores (the two arithmetic engines the update
// kernels use). Each is timed with CUDA events on the caller's stream after one warm-up
// launch; the numbers are what the hardware sustains for a pure instruction stream, with no
// memory traffic.
#include <cuda_runtime.h>

#include <cmath>

#include "tc.cuh"

namespace ltsdev {

constexpr int PEAK_FMA_THREADS = 256;
constexpr int PEAK_FMA_CHAINS = 8;    // independent dependency chains per thread
constexpr int PEAK_FMA_UNROLL = 32;   // FMAs per chain per loop iteration

// FP32: every thread runs PEAK_FMA_CHAINS independent chains a <- a m + c.
__global__ void __launch_bounds__(PEAK_FMA_THREADS) k_peak_fma(float* out, int iters, float seed) {
  float a[PEAK_FMA_CHAINS];
#pragma unroll
  for (int j = 0; j < PEAK_FMA_CHAINS; ++j) a[j] = seed + 1e-3f * (float)(threadIdx.x + j);
  const float m = 0.9999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PEAK_FMA_UNROLL; ++u)
#pragma unroll
      for (int j = 0; j < PEAK_FMA_CHAINS; ++j) a[j] = fmaf(a[j], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < PEAK_FMA_CHAINS; ++j) s += a[j];
  if (s == 1234.5f) out[blockIdx.x * PEAK_FMA_THREADS + threadIdx.x] = s;   // keeps the chains live
}

// TF32: one CTA per SM (the dynamic shared memory leaves room for one). D (128 lanes x 256
// columns) accumulates nmma products A (128 x 8, tensor memory columns 256..263) times B
// (256 x 8, shared memory, K-major core matrices: LBO 128, SBO 256 bytes), all issued by one
// thread and committed to an mbarrier; the wait is bounded by wait_cycles, after which the
// CTA records the timeout in *err, releases its tensor memory and returns.
constexpr int PEAK_TC_N = 256, PEAK_TC_COLS = 512, PEAK_TC_SMEM = 120 * 1024;
__global__ void __launch_bounds__(128, 1) k_peak_tf32(int nmma, long long wait_cycles, int* err) {
  extern __shared__ __align__(128) float psm[];
  float* sB = psm;                                                  // 256 x 8 tf32 = 8 KB
  uint64_t* bar = reinterpret_cast<uint64_t*>(psm + PEAK_TC_N * 8);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(psm + PEAK_TC_N * 8 + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < PEAK_TC_N * 8; i += 128) sB[i] = tc::tf32_round(0.5f + 1e-3f * (float)(i % 7));
  if (warp == 0) {
    tc::tmem_alloc(taddr_s, PEAK_TC_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *taddr_s;
  {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = tc::tf32_round(0.25f + 1e-2f * (float)j);
    tc::tmem_st8(tmem + ((uint32_t)(warp * 32) << 16) + PEAK_TC_N, a);
  }
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    tc::fence_after_sync();
    constexpr uint32_t idesc = tc::idesc_tf32(128, PEAK_TC_N);
    const uint64_t bd = tc::smem_desc(tc::smem_u32(sB), 128, 256);
    for (int i = 0; i < nmma; ++i) tc::mma_tf32_ts(tmem, tmem + PEAK_TC_N, bd, idesc, i > 0 ? 1u : 0u);
    tc::commit(bar);
  }
  bool ok = tc::mbar_wait(bar, 0, wait_cycles);
  ok = __syncthreads_and(ok) != 0;
  tc::fence_after_sync();
  if (!ok && tid == 0) atomicOr(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, PEAK_TC_COLS);
}

// Runs both probes on `stream`; out[0] FP32 TFLOP/s, out[1] tf32 TFLOP/s, out[2], out[3]
// the timed durations (ms). Returns a CUDA error, or cudaErrorTimeout if a tensor-core wait
// ran out (the probe's TMEM is released either way).
cudaError_t measure_peaks(cudaStream_t stream, double* out) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_peak_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, PEAK_TC_SMEM)) !=
      cudaSuccess)
    return e;
  float* dout = nullptr;
  int* derr = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  const int fma_blocks = nsm * 8, fma_iters = 4096;
  const int nmma = 8192;
  float ms_fma = 0.f, ms_tc = 0.f;
  int herr = 0;
  auto done = [&](cudaError_t r) {
    if (dout) cudaFree(dout);
    if (derr) cudaFree(derr);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    return r;
  };
  if ((e = cudaMalloc(&dout, sizeof(float) * fma_blocks * PEAK_FMA_THREADS)) != cudaSuccess) return done(e);
  if ((e = cudaMalloc(&derr, sizeof(int))) != cudaSuccess) return done(e);
  if ((e = cudaMemsetAsync(derr, 0, sizeof(int), stream)) != cudaSuccess) return done(e);
  if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) return done(e);
  const long long wait_cycles = 4000000000LL;
  for (int rep = 0; rep < 2; ++rep) {   // rep 0 warms up
    cudaEventRecord(t0, stream);
    k_peak_fma<<<fma_blocks, PEAK_FMA_THREADS, 0, stream>>>(dout, fma_iters, 1.0f);
    cudaEventRecord(t1, stream);
    if ((e = cudaEventSynchronize(t1)) != cudaSuccess) return done(e);
    cudaEventElapsedTime(&ms_fma, t0, t1);
    cudaEventRecord(t0, stream);
    k_peak_tf32<<<nsm, 128, PEAK_TC_SMEM, stream>>>(nmma, wait_cycles, derr);
    cudaEventRecord(t1, stream);
    if ((e = cudaEventSynchronize(t1)) != cudaSuccess) return done(e);
    cudaEventElapsedTime(&ms_tc, t0, t1);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
  if ((e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return done(e);
  if (herr) return done(cudaErrorTimeout);
  const double fma_flops = 2.0 * PEAK_FMA_UNROLL * PEAK_FMA_CHAINS * (double)fma_iters * fma_blocks * PEAK_FMA_THREADS;
  const double tc_flops = 2.0 * 128 * PEAK_TC_N * 8 * (double)nmma * nsm;
  out[0] = fma_flops / (ms_fma * 1e-3) / 1e12;
  out[1] = tc_flops / (ms_tc * 1e-3) / 1e12;
  out[2] = ms_fma;
  out[3] = ms_tc;
  return done(cudaSuccess);
}

}  // namespace ltsdev
