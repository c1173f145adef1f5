// Microbenchmarks of the on-chip roofs that bound the operator kernels: the
// FP32 FMA rate, the shared-memory load bandwidth, and the L2 and DRAM read
// bandwidths.  The projectors (Sec. 4.1.1 discrete Radon transform and its
// transposes) are neither HBM- nor tensor-bound: every interpolation sample
// costs a few FP32 operations and two shared-memory taps, so their roofline
// is the larger of (FP32 work / FMA rate) and (tap bytes / shared-memory
// bandwidth); the DRAM and L2 figures bound the elementwise kernels and the
// band-sum workspace.
#include "common.cuh"

namespace skei {
namespace {

constexpr int kRoofThreads = 256;

// Eight independent FMA chains per thread, 16 x 8 FMAs per iteration.
__global__ void __launch_bounds__(kRoofThreads) roof_fma_kernel(float *sink, int iters, float a,
                                                                float b) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 1234.5f) sink[blockIdx.x] = s;   // never true; keeps the chains alive
}

// 16-byte shared-memory loads, 8 per iteration, consecutive lanes on
// consecutive 16-byte words (no bank conflicts); XOR-folded so that the
// arithmetic stays far below the load rate.
__global__ void __launch_bounds__(kRoofThreads) roof_smem_kernel(unsigned *sink, int iters) {
  __shared__ uint4 buf[2048];   // 32 KB
  for (int i = threadIdx.x; i < 2048; i += kRoofThreads)
    buf[i] = make_uint4(i, 3u * i + 1u, 5u * i + 2u, 7u * i + 3u);
  __syncthreads();
  uint4 acc = make_uint4(0u, 0u, 0u, 0u);
  int idx = threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      const uint4 v = buf[(idx + u * kRoofThreads) & 2047];
      const uint4 w = buf[(idx + (u + 1) * kRoofThreads) & 2047];
      acc.x ^= v.x ^ w.x;
      acc.y ^= v.y ^ w.y;
      acc.z ^= v.z ^ w.z;
      acc.w ^= v.w ^ w.w;
    }
    idx = (idx + 32) & 2047;
  }
  if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x9e3779b9u) sink[blockIdx.x] = 1u;
}

// Streaming 16-byte reads cached in L2 only (ld.global.cg), four in flight
// per thread; `passes` sweeps over n4 words.
__global__ void __launch_bounds__(kRoofThreads) roof_read_kernel(const uint4 *buf, size_t n4,
                                                                 int passes, unsigned *sink) {
  uint4 acc = make_uint4(0u, 0u, 0u, 0u);
  const size_t stride = (size_t)gridDim.x * kRoofThreads;
  for (int p = 0; p < passes; ++p) {
    size_t i = (size_t)blockIdx.x * kRoofThreads + threadIdx.x;
    for (; i + 3 * stride < n4; i += 4 * stride) {
      const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
      const uint4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
      acc.x ^= a.x ^ b.x ^ c.x ^ d.x;
      acc.y ^= a.y ^ b.y ^ c.y ^ d.y;
      acc.z ^= a.z ^ b.z ^ c.z ^ d.z;
      acc.w ^= a.w ^ b.w ^ c.w ^ d.w;
    }
    for (; i < n4; i += stride) {
      const uint4 a = __ldcg(buf + i);
      acc.x ^= a.x;
      acc.y ^= a.y;
      acc.z ^= a.z;
      acc.w ^= a.w;
    }
  }
  if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x9e3779b9u) sink[blockIdx.x] = 1u;
}

// Milliseconds of `launch()` on st, after one untimed run.
template <typename F>
int time_ms(cudaStream_t st, F launch, float *ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e == cudaSuccess ? SKEI_OK : cuda_error(e, "roof microbenchmark");
}

}  // namespace
}  // namespace skei

using namespace skei;

extern "C" int skei_measure_roofs(void *work, size_t work_bytes, skei_roofs *out, void *stream) {
  SKEI_RANGE("skei_measure_roofs");
  if (!out) return set_error(SKEI_EINVAL, "skei_measure_roofs: out is NULL");
  SKEI_TRY(check_dev_ptr(work, "work"));
  if (work_bytes < SKEI_ROOFS_WORK_BYTES)
    return set_error(SKEI_EINVAL, "skei_measure_roofs: work of %zu bytes, %zu needed", work_bytes,
                     (size_t)SKEI_ROOFS_WORK_BYTES);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int sms = sm_count();
  const int blocks = sms * 8;   // 2048 threads per SM
  unsigned *sink = static_cast<unsigned *>(work);
  const uint4 *buf = reinterpret_cast<const uint4 *>(static_cast<char *>(work) + 65536);
  *out = skei_roofs{};
  out->sms = sms;
  float ms = 0.0f;

  const int fma_iters = 4096;
  SKEI_TRY(time_ms(st, [&] {
    roof_fma_kernel<<<blocks, kRoofThreads, 0, st>>>(reinterpret_cast<float *>(sink), fma_iters,
                                                      0.9999999f, 1e-7f);
  }, &ms));
  out->fp32_flops = 2.0 * 16 * 8 * (double)fma_iters * blocks * kRoofThreads / (ms * 1e-3);

  const int smem_iters = 8192;
  SKEI_TRY(time_ms(st, [&] {
    roof_smem_kernel<<<blocks, kRoofThreads, 0, st>>>(sink, smem_iters);
  }, &ms));
  out->smem_bytes = 16.0 * 8 * (double)smem_iters * blocks * kRoofThreads / (ms * 1e-3);

  // L2: a buffer well inside the 129 MB L2, swept 16 times per launch
  const size_t l2_n4 = (size_t)SKEI_ROOFS_L2_BYTES / 16;
  const int l2_passes = 16;
  SKEI_TRY(time_ms(st, [&] {
    roof_read_kernel<<<blocks, kRoofThreads, 0, st>>>(buf, l2_n4, l2_passes, sink);
  }, &ms));
  out->l2_bytes = 16.0 * (double)l2_n4 * l2_passes / (ms * 1e-3);

  // DRAM: the rest of the work buffer (several times the L2), swept once
  const size_t dram_n4 = (work_bytes - 65536) / 16;
  SKEI_TRY(time_ms(st, [&] {
    roof_read_kernel<<<blocks, kRoofThreads, 0, st>>>(buf, dram_n4, 1, sink);
  }, &ms));
  out->dram_read_bytes = 16.0 * (double)dram_n4 / (ms * 1e-3);
  return SKEI_OK;
}
