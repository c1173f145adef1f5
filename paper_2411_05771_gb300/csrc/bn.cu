// Batch normalisation with batch statistics and a fused activation: the BN
// layers that BN-only test-time training adapts (Sec. 3.3).  For channel c
// of v [B][C][HW], over its M = B HW values,
//   mean_c = (1/M) sum v,  var_c = (1/M) sum (v - mean_c)^2,
//   out = act(scale_c (v - mean_c) / sqrt(var_c + eps) + shift_c),
// act = ReLU or the identity; the backward returns dL/dv, dL/dscale and
// dL/dshift.  Two launches each way: per-chunk partial sums (FP32 within a
// thread and warp, FP64 across warps and chunks, fixed order), then the
// elementwise pass, whose CTAs each finish their channel's sums.
#include <type_traits>

#include "common.cuh"

using bf16 = __nv_bfloat16;

namespace skei {
namespace {

constexpr int kBnThreads = 256;
constexpr int kBnChunk = 16384;  // values of one (b, c) plane per CTA
constexpr int kBnPer = kBnChunk / kBnThreads;

// Values e0 + 4 t + 4 kBnThreads j (j < kBnPer / 4) of a plane, or the
// scalar equivalent; f(value index, value) for each one inside [e0, e1).
template <typename T, typename Fn>
__device__ __forceinline__ void chunk_each(const T *pl, long long e0, long long e1, bool vec,
                                           Fn f) {
  const int t = threadIdx.x;
  if (vec) {
#pragma unroll 4
    for (int j = 0; j < kBnPer / 4; ++j) {
      const long long e = e0 + 4LL * (t + j * kBnThreads);
      if (e < e1) {
        const float4 x = __ldg(reinterpret_cast<const float4 *>(pl + e));
        f(e, x.x);
        f(e + 1, x.y);
        f(e + 2, x.z);
        f(e + 3, x.w);
      }
    }
  } else {
#pragma unroll 4
    for (int j = 0; j < kBnPer; ++j) {
      const long long e = e0 + t + (long long)j * kBnThreads;
      if (e < e1) f(e, ldg_f(pl + e));
    }
  }
}

// The FP32 fast path (HW % 4 == 0, 16-byte aligned planes): thread t takes
// the float4 groups e0 + 4 t + 4 kBnThreads j of the chunk;
// f(e, v4, g4) for each, with g4 the same group of a second plane (or 0).
template <typename Fn>
__device__ __forceinline__ void chunk_each4(const float *pv, const float *pg, long long e0,
                                            long long e1, Fn f) {
  const int t = threadIdx.x;
#pragma unroll 4
  for (int j = 0; j < kBnPer / 4; ++j) {
    const long long e = e0 + 4LL * (t + j * kBnThreads);
    if (e < e1) {
      const float4 x = __ldg(reinterpret_cast<const float4 *>(pv + e));
      const float4 g = pg ? __ldg(reinterpret_cast<const float4 *>(pg + e))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
      f(e, x, g);
    }
  }
}

// Sum over the CTA of two FP32 per-thread values in a fixed order: FP32
// within a warp (FP64 arithmetic is scarce on this GPU), FP64 across the
// warps; the result is valid in thread 0.
__device__ __forceinline__ double2 cta_sum2(float a, float b) {
  __shared__ double2 red[kBnThreads / 32];
  float x = a, y = b;
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = make_double2(x, y);
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int i = 0; i < kBnThreads / 32; ++i) {
      s.x += red[i].x;
      s.y += red[i].y;
    }
  return s;
}

// Sum of a channel's np partial pairs, in a fixed order (warp 0; lane-strided
// sums, then a shuffle tree); the result is valid in every lane of warp 0.
__device__ __forceinline__ double2 channel_sum2(const double2 *part, int np) {
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) {
    x += part[i].x;
    y += part[i].y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  return make_double2(x, y);
}

// grid (B * nch, C): CTA (b, q) of channel c sums chunk q of plane (b, c).
// Partials of d = v - K_c, K_c = v[0][c][0] (a shift against cancellation
// in the variance): (sum d, sum d^2).
template <typename T>
__global__ void __launch_bounds__(kBnThreads)
    bn_stats_kernel(const T *v, int C, long long HW, int nch, bool vec, double2 *part) {
  pdl_enter();
  const int c = blockIdx.y, b = blockIdx.x / nch, q = blockIdx.x - b * nch;
  const T *pl = v + ((size_t)b * C + c) * HW;
  const float K = ldg_f(v + (size_t)c * HW);
  const long long e0 = (long long)q * kBnChunk, e1 = min(HW, e0 + kBnChunk);
  float s = 0.0f, s2 = 0.0f;
  chunk_each(pl, e0, e1, vec, [&](long long, float x) {
    const float d = x - K;
    s += d;
    s2 = fmaf(d, d, s2);
  });
  const double2 r = cta_sum2(s, s2);
  if (threadIdx.x == 0) part[(size_t)c * gridDim.x + blockIdx.x] = r;
}

// Scale a = scale rstd and offset bb = shift - mean a of the affine map
// out = act(v a + bb), from the FP32 statistics (the backward recomputes them
// from the same values, so it sees the same activation mask).
__device__ __forceinline__ void affine_of(float scale, float shift, float mean, float rstd,
                                          float *a, float *bb) {
  *a = scale * rstd;
  *bb = fmaf(-mean, *a, shift);
}

template <typename T>
__global__ void __launch_bounds__(kBnThreads)
    bn_apply_kernel(const T *v, int C, long long HW, int nch, bool vec, const double2 *part,
                    const float *scale, const float *shift, int relu, double eps, T *out,
                    float *mean_out, float *rstd_out) {
  pdl_enter();
  __shared__ float s_mean, s_rstd;
  const int c = blockIdx.y, b = blockIdx.x / nch, q = blockIdx.x - b * nch;
  if (threadIdx.x < 32) {
    const double2 S = channel_sum2(part + (size_t)c * gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      const double M = (double)gridDim.x / nch * (double)HW;
      const double md = S.x / M;
      const double var = fmax(S.y / M - md * md, 0.0);
      const float mean = (float)((double)ldg_f(v + (size_t)c * HW) + md);
      const float rstd = (float)(1.0 / sqrt(var + eps));
      s_mean = mean;
      s_rstd = rstd;
      if (blockIdx.x == 0) {
        mean_out[c] = mean;
        rstd_out[c] = rstd;
      }
    }
  }
  __syncthreads();
  float a, bb;
  affine_of(__ldg(scale + c), __ldg(shift + c), s_mean, s_rstd, &a, &bb);
  const size_t o = ((size_t)b * C + c) * HW;
  const long long e0 = (long long)q * kBnChunk, e1 = min(HW, e0 + kBnChunk);
  T *po = out + o;
  auto act = [&](float x) {
    const float y = fmaf(x, a, bb);
    return relu ? fmaxf(y, 0.0f) : y;
  };
  if constexpr (std::is_same<T, float>::value) {
    if (vec) {
      chunk_each4(v + o, nullptr, e0, e1, [&](long long e, float4 x, float4) {
        *reinterpret_cast<float4 *>(po + e) = make_float4(act(x.x), act(x.y), act(x.z), act(x.w));
      });
      return;
    }
  }
  chunk_each(v + o, e0, e1, false, [&](long long e, float x) { st_f(po + e, act(x)); });
}

// Backward partials: gy = g where the activation passes (y > 0 for ReLU),
// x^ = (v - mean) rstd; (sum gy, sum gy x^) per chunk.
template <typename T>
__global__ void __launch_bounds__(kBnThreads)
    bn_bwd_stats_kernel(const T *v, const T *g, int C, long long HW, int nch, bool vec,
                        const float *scale, const float *shift, const float *mean,
                        const float *rstd, int relu, double2 *part) {
  pdl_enter();
  const int c = blockIdx.y, b = blockIdx.x / nch, q = blockIdx.x - b * nch;
  const size_t o = ((size_t)b * C + c) * HW;
  const long long e0 = (long long)q * kBnChunk, e1 = min(HW, e0 + kBnChunk);
  const float mu = __ldg(mean + c), rs = __ldg(rstd + c);
  float a, bb;
  affine_of(__ldg(scale + c), __ldg(shift + c), mu, rs, &a, &bb);
  const T *pg = g + o;
  float s = 0.0f, sx = 0.0f;
  auto acc = [&](float x, float gy) {
    if (relu && !(fmaf(x, a, bb) > 0.0f)) gy = 0.0f;
    s += gy;
    sx = fmaf(gy, (x - mu) * rs, sx);
  };
  bool done = false;
  if constexpr (std::is_same<T, float>::value) {
    if (vec) {
      chunk_each4(v + o, pg, e0, e1, [&](long long, float4 x, float4 gg) {
        acc(x.x, gg.x);
        acc(x.y, gg.y);
        acc(x.z, gg.z);
        acc(x.w, gg.w);
      });
      done = true;
    }
  }
  if (!done) chunk_each(v + o, e0, e1, false, [&](long long e, float x) { acc(x, ldg_f(pg + e)); });
  const double2 r = cta_sum2(s, sx);
  if (threadIdx.x == 0) part[(size_t)c * gridDim.x + blockIdx.x] = r;
}

// dL/dv = a (gy - dshift / M - x^ dscale / M), a = scale rstd;
// dscale = sum gy x^, dshift = sum gy over the channel.
template <typename T>
__global__ void __launch_bounds__(kBnThreads)
    bn_bwd_apply_kernel(const T *v, const T *g, int C, long long HW, int nch, bool vec,
                        const double2 *part, const float *scale, const float *shift,
                        const float *mean, const float *rstd, int relu, T *gv, float *g_scale,
                        float *g_shift) {
  pdl_enter();
  __shared__ float s_k1, s_k2;
  const int c = blockIdx.y, b = blockIdx.x / nch, q = blockIdx.x - b * nch;
  if (threadIdx.x < 32) {
    const double2 S = channel_sum2(part + (size_t)c * gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      const double M = (double)gridDim.x / nch * (double)HW;
      s_k1 = (float)(S.x / M);
      s_k2 = (float)(S.y / M);
      if (blockIdx.x == 0) {
        g_shift[c] = (float)S.x;
        g_scale[c] = (float)S.y;
      }
    }
  }
  __syncthreads();
  const float mu = __ldg(mean + c), rs = __ldg(rstd + c);
  float a, bb;
  affine_of(__ldg(scale + c), __ldg(shift + c), mu, rs, &a, &bb);
  const float k1 = s_k1, k2 = s_k2;
  const size_t o = ((size_t)b * C + c) * HW;
  const long long e0 = (long long)q * kBnChunk, e1 = min(HW, e0 + kBnChunk);
  const T *pg = g + o;
  T *pv = gv + o;
  auto grad = [&](float x, float gy) {
    if (relu && !(fmaf(x, a, bb) > 0.0f)) gy = 0.0f;
    return a * (gy - k1 - (x - mu) * rs * k2);
  };
  if constexpr (std::is_same<T, float>::value) {
    if (vec) {
      chunk_each4(v + o, pg, e0, e1, [&](long long e, float4 x, float4 gg) {
        *reinterpret_cast<float4 *>(pv + e) =
            make_float4(grad(x.x, gg.x), grad(x.y, gg.y), grad(x.z, gg.z), grad(x.w, gg.w));
      });
      return;
    }
  }
  chunk_each(v + o, e0, e1, false, [&](long long e, float x) { st_f(pv + e, grad(x, ldg_f(pg + e))); });
}

struct BnGrid {
  int nch;
  dim3 grid;
};

int bn_grid(int B, int C, int64_t HW, BnGrid *g) {
  if (B < 1 || C < 1 || HW < 1)
    return set_error(SKEI_EINVAL, "batch norm: B=%d, C=%d, HW=%lld must be >= 1", B, C,
                     (long long)HW);
  if (C > 65535) return set_error(SKEI_EINVAL, "batch norm: C=%d > 65535 channels", C);
  const int64_t nch = (HW + kBnChunk - 1) / kBnChunk;
  if ((int64_t)B * nch > ((int64_t)1 << 30))
    return set_error(SKEI_EINVAL, "batch norm: B * HW too large");
  g->nch = (int)nch;
  g->grid = dim3((unsigned)(B * nch), (unsigned)C);
  return SKEI_OK;
}

}  // namespace
}  // namespace skei

using namespace skei;

extern "C" {

size_t skei_bn_workspace_size(int B, int C, int64_t HW) {
  BnGrid g;
  if (bn_grid(B, C, HW, &g) != SKEI_OK) return 0;
  return (size_t)g.grid.x * g.grid.y * sizeof(double2);
}

int skei_bn_act_fwd(int dtype, const void *v, int B, int C, int64_t HW, const float *scale,
                    const float *shift, int relu, double eps, void *out, float *mean,
                    float *rstd, void *work, size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_bn_act_fwd");
  SKEI_TRY(check_dtype(dtype));
  BnGrid g;
  SKEI_TRY(bn_grid(B, C, HW, &g));
  if (!(eps > 0.0)) return set_error(SKEI_EINVAL, "batch norm: eps must be > 0");
  SKEI_TRY(check_dev_ptr(v, "v"));
  SKEI_TRY(check_dev_ptr(scale, "scale"));
  SKEI_TRY(check_dev_ptr(shift, "shift"));
  SKEI_TRY(check_dev_ptr(out, "out"));
  SKEI_TRY(check_dev_ptr(mean, "mean"));
  SKEI_TRY(check_dev_ptr(rstd, "rstd"));
  SKEI_TRY(check_dev_ptr(work, "work"));
  if (reinterpret_cast<uintptr_t>(work) % 16)
    return set_error(SKEI_EINVAL, "batch norm: work must be 16-byte aligned");
  const size_t need = (size_t)g.grid.x * g.grid.y * sizeof(double2);
  if (work_bytes < need)
    return set_error(SKEI_EINVAL, "batch norm: work has %zu bytes, %zu needed", work_bytes, need);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double2 *part = static_cast<double2 *>(work);
  const bool vec = dtype == SKEI_F32 && HW % 4 == 0 &&
                   ((reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  if (dtype == SKEI_F32) {
    launch_k(bn_stats_kernel<float>, g.grid, dim3(kBnThreads), 0, st, (const float *)v, C,
             (long long)HW, g.nch, vec, part);
    SKEI_TRY(check_launch("batch norm statistics launch"));
    launch_k(bn_apply_kernel<float>, g.grid, dim3(kBnThreads), 0, st, (const float *)v, C,
             (long long)HW, g.nch, vec, (const double2 *)part, scale, shift, relu, eps,
             (float *)out, mean, rstd);
  } else {
    launch_k(bn_stats_kernel<bf16>, g.grid, dim3(kBnThreads), 0, st, (const bf16 *)v, C,
             (long long)HW, g.nch, false, part);
    SKEI_TRY(check_launch("batch norm statistics launch"));
    launch_k(bn_apply_kernel<bf16>, g.grid, dim3(kBnThreads), 0, st, (const bf16 *)v, C,
             (long long)HW, g.nch, false, (const double2 *)part, scale, shift, relu, eps,
             (bf16 *)out, mean, rstd);
  }
  return check_launch("batch norm apply launch");
}

int skei_bn_act_bwd(int dtype, const void *v, const void *g_out, int B, int C, int64_t HW,
                    const float *scale, const float *shift, const float *mean,
                    const float *rstd, int relu, void *g_v, float *g_scale, float *g_shift,
                    void *work, size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_bn_act_bwd");
  SKEI_TRY(check_dtype(dtype));
  BnGrid g;
  SKEI_TRY(bn_grid(B, C, HW, &g));
  SKEI_TRY(check_dev_ptr(v, "v"));
  SKEI_TRY(check_dev_ptr(g_out, "g_out"));
  SKEI_TRY(check_dev_ptr(scale, "scale"));
  SKEI_TRY(check_dev_ptr(shift, "shift"));
  SKEI_TRY(check_dev_ptr(mean, "mean"));
  SKEI_TRY(check_dev_ptr(rstd, "rstd"));
  SKEI_TRY(check_dev_ptr(g_v, "g_v"));
  SKEI_TRY(check_dev_ptr(g_scale, "g_scale"));
  SKEI_TRY(check_dev_ptr(g_shift, "g_shift"));
  SKEI_TRY(check_dev_ptr(work, "work"));
  if (reinterpret_cast<uintptr_t>(work) % 16)
    return set_error(SKEI_EINVAL, "batch norm: work must be 16-byte aligned");
  const size_t need = (size_t)g.grid.x * g.grid.y * sizeof(double2);
  if (work_bytes < need)
    return set_error(SKEI_EINVAL, "batch norm: work has %zu bytes, %zu needed", work_bytes, need);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double2 *part = static_cast<double2 *>(work);
  const bool vec = dtype == SKEI_F32 && HW % 4 == 0 &&
                   ((reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(g_out) |
                     reinterpret_cast<uintptr_t>(g_v)) & 15) == 0;
  if (dtype == SKEI_F32) {
    launch_k(bn_bwd_stats_kernel<float>, g.grid, dim3(kBnThreads), 0, st, (const float *)v,
             (const float *)g_out, C, (long long)HW, g.nch, vec, scale, shift, mean, rstd, relu,
             part);
    SKEI_TRY(check_launch("batch norm backward partials launch"));
    launch_k(bn_bwd_apply_kernel<float>, g.grid, dim3(kBnThreads), 0, st, (const float *)v,
             (const float *)g_out, C, (long long)HW, g.nch, vec, (const double2 *)part, scale,
             shift, mean, rstd, relu, (float *)g_v, g_scale, g_shift);
  } else {
    launch_k(bn_bwd_stats_kernel<bf16>, g.grid, dim3(kBnThreads), 0, st, (const bf16 *)v,
             (const bf16 *)g_out, C, (long long)HW, g.nch, false, scale, shift, mean, rstd,
             relu, part);
    SKEI_TRY(check_launch("batch norm backward partials launch"));
    launch_k(bn_bwd_apply_kernel<bf16>, g.grid, dim3(kBnThreads), 0, st, (const bf16 *)v,
             (const bf16 *)g_out, C, (long long)HW, g.nch, false, (const double2 *)part, scale,
             shift, mean, rstd, relu, (bf16 *)g_v, g_scale, g_shift);
  }
  return check_launch("batch norm backward launch");
}

}  // extern "C"
