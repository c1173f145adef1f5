// Operators that sum over image "lines" (rows when |cos| >= |sin|, columns
// otherwise) for every detector bin: Joseph's forward projector A
// (Sec. 4.1.1, the discrete Radon transform; Eq. (e:skeiloss): A_S = S A)
// and the transpose B_S^T of pixel-driven back-projection (needed to
// differentiate through A_S^dagger = (pi/m) B_S H, Algorithm 2's update).
//
// A cluster of 8 CTAs covers a group of images and a block of AB angles;
// CTA r stages lines [r R, (r+1) R) (R = ceil(N/8)) in shared memory - rows
// as they are, columns transposed - sub-band by sub-band, and accumulates
// per-bin sums in its own shared memory.  After a cluster barrier each CTA
// reduces 1/8 of the bins over the 8 CTAs' sums through distributed shared
// memory, in a fixed order: deterministic, no atomics, no global scratch.
// (Measured on GB300: double-buffered cp.async staging and cutting the bins
// into chunks per cluster were both slower at 512^2.)
//
//   A:    one thread per ray gathers the linear interpolation on each line.
//   B^T:  one thread per bin gathers, on each line, the (at most 3) pixels
//         whose bin coordinate lies within one bin of it, with exactly the
//         back-projector's weights.
//
// Image groups.  All images of a job share the angle list, so positions,
// weights and candidate pixels are the same for every image of a group of
// NI = 4: they can be computed once and applied to the 4 images, staged
// interleaved ([line][position][image], one 16-byte load per tap for the
// whole group).  Jobs whose image count is not a multiple of 4 finish with
// single-image groups.  Every image sees the same sequence of operations in
// either form, and the per-bin sums run over the lines of the band in order
// whatever the staging sub-band, so results do not depend on the grouping.
//
// Up to two jobs share a launch (grid.z spans the groups of both), e.g. the
// MC projection of x1 and the EI projection of x2 of one SkEI step.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <queue>
#include <vector>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace skei {
namespace {

// Build-time tuning knobs (defaults are the measured best on GB300 for the
// 512^2 steps): largest image group of A and of B^T (1 or 4; B^T's 3
// candidate weights per line gain from sharing when the launch has clusters
// to spare, A's 2 taps do not), staged lines per
// sub-band for groups of 4, a fixed number of angles per cluster (0:
// chosen per launch), and threads per CTA.
#ifndef SKEI_BAND_GROUP_FWD
#define SKEI_BAND_GROUP_FWD 1
#endif
#ifndef SKEI_BAND_GROUP_BPADJ
#define SKEI_BAND_GROUP_BPADJ 4
#endif
#ifndef SKEI_BAND_SB1_FWD
#define SKEI_BAND_SB1_FWD 32   // staged lines per sub-band of the single-image forward (16 or 32)
#endif
#ifndef SKEI_BAND_SB4
#define SKEI_BAND_SB4 8
#endif
#ifndef SKEI_BAND_AB
#define SKEI_BAND_AB 0
#endif
#ifndef SKEI_BAND_THREADS
#define SKEI_BAND_THREADS 256
#endif

constexpr int kBands = 8;    // cluster size = number of line bands
constexpr int kPad = 4;      // zero positions on each side of a staged line
constexpr int kMaxAB = 8;    // angles per cluster
constexpr int kThreads = SKEI_BAND_THREADS;
constexpr int kWarps = kThreads / 32;

__host__ __device__ constexpr int group_max(int op) {
  return op == OP_JOSEPH ? SKEI_BAND_GROUP_FWD : SKEI_BAND_GROUP_BPADJ;
}

struct BandGeom {
  int N, n_det, n_angles;
  int NI;      // images per group (1 or 4), interleaved in shared memory
  int R;       // lines per band
  int SB;      // lines per staged sub-band
  int Prow;    // pitch (positions) of staged rows
  int Pcol;    // pitch (positions) of staged columns (conflict-free transposed writes)
  int AB;      // angles per cluster
  int fast;    // N % 8 == 0: 16-byte staging of single-image rows
};

struct BandArgs {
  Jobs jobs;
  const AngleConst *ang;
  int *status;
  BandGeom g1, g4;   // geometry of single-image and 4-image groups
  int gmax;          // group size of this launch (1 or 4)
};

// Staging geometry of one image size, operator and group size with AB
// angles per task.
__host__ __device__ __forceinline__ BandGeom band_geom(int N, int n_det, int n_angles, int op,
                                                       int AB, int NI) {
  BandGeom g;
  g.N = N;
  g.n_det = n_det;
  g.n_angles = n_angles;
  g.NI = NI;
  g.R = (N + kBands - 1) / kBands;
  g.Prow = (N + 2 * kPad + 3) & ~3;
  if (NI == 1) {
    // A: 32 staged lines (fewer per-ray range setups); B^T: 16 (its per-bin
    // work per line is larger, and the smaller band leaves room for more CTAs)
    const int sb = op == OP_JOSEPH ? SKEI_BAND_SB1_FWD : 16;
    g.SB = g.R < sb ? g.R : sb;
    // transposed staging writes lines 4q..4q+3 of (32 / (SB/4)) positions
    // per warp: a pitch = 2 mod 8 (16 lines) or odd (32 lines) keeps them in
    // distinct banks
    g.Pcol = g.SB == 32 ? ((N + 2 * kPad) | 1) : ((N + 2 * kPad - 2 + 7) & ~7) + 2;
  } else {
    // 16 bytes per position: an odd pitch puts the 8 lines of one position
    // that 8 consecutive threads write in distinct bank quads (both modes)
    g.SB = g.R < SKEI_BAND_SB4 ? g.R : SKEI_BAND_SB4;
    g.Pcol = (N + 2 * kPad) | 1;
    g.Prow = g.Pcol;
  }
  g.fast = (N % 8 == 0) ? 1 : 0;
  const int Pmax = g.Prow > g.Pcol ? g.Prow : g.Pcol;
  while (g.SB > 1 && g.SB * Pmax * 4 * NI > 96 * 1024) --g.SB;  // large N: slow staging
  g.AB = AB;
  return g;
}

// Dynamic shared memory of a band task: the per-bin sums of AB angles, then
// the staged sub-band.
__host__ __device__ __forceinline__ size_t band_part_floats(const BandGeom &g) {
  return (size_t)((g.AB * g.n_det * g.NI + 3) & ~3);
}
__host__ __device__ __forceinline__ size_t band_smem(const BandGeom &g) {
  const int Pmax = g.Prow > g.Pcol ? g.Prow : g.Pcol;
  return (band_part_floats(g) + (size_t)g.SB * Pmax * g.NI) * 4;
}

// 4 consecutive image values at element offset i as floats (16-byte aligned
// for float, 8-byte for bfloat16).
__device__ __forceinline__ float4 load4(const void *x, size_t i, int bf16) {
  if (bf16) {
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(static_cast<const __nv_bfloat16 *>(x) + i));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
  }
  return __ldg(reinterpret_cast<const float4 *>(static_cast<const float *>(x) + i));
}

// A shared-memory store of the band staging, range-checked in the check
// build.
template <typename V>
__device__ __forceinline__ void sts(V *p, const V &v) {
  if (SKEI_CHECK && !ck_smem(p, sizeof(V), CK_BAND_STAGE)) return;
  *p = v;
}

// Stages lines [s0, s0 + nl) of one image (element offset xo in x) into buf
// (pitch P positions): mode 1 copies rows, mode 0 copies columns
// transposed.  PAD zero positions on each side.
template <int PAD = kPad>
__device__ __forceinline__ void stage1(const void *x, size_t xo, int bf16, int N, int mode,
                                       int s0, int nl, float *buf, int P, bool fast) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (mode == 1) {
    if (fast) {
      // 4 loads in flight per thread before their stores
      for (int r = warp; r < nl; r += kWarps) {
        const size_t src = xo + (size_t)(s0 + r) * N;
        float *dst = buf + r * P + PAD;
        int c = 4 * lane;
        for (; c + 384 < N; c += 512) {
          const float4 a = load4(x, src + c, bf16), b = load4(x, src + c + 128, bf16);
          const float4 d = load4(x, src + c + 256, bf16), e = load4(x, src + c + 384, bf16);
          sts(reinterpret_cast<float4 *>(dst + c), a);
          sts(reinterpret_cast<float4 *>(dst + c + 128), b);
          sts(reinterpret_cast<float4 *>(dst + c + 256), d);
          sts(reinterpret_cast<float4 *>(dst + c + 384), e);
        }
        for (; c < N; c += 128)
          sts(reinterpret_cast<float4 *>(dst + c), load4(x, src + c, bf16));
      }
    } else {
      for (int r = warp; r < nl; r += kWarps) {
        const size_t src = xo + (size_t)(s0 + r) * N;
        float *dst = buf + r * P + PAD;
        for (int c = lane; c < N; c += 32) sts(dst + c, ld_any(x, src + c, bf16));
      }
    }
  } else {
    if (fast && (nl == 8 || nl == 16 || nl == 32) && (s0 & 3) == 0) {
      // lane = (nl/4) * (position within a group) + quarter of the lines; 4
      // consecutive lines of a column start 16-byte aligned (N % 8 == 0)
      const int qn = nl >> 2, qs = nl == 8 ? 1 : (nl == 16 ? 2 : 3);
      const int q = lane & (qn - 1);
      const int per_warp = 32 / qn;
      const int step = kWarps * per_warp;
      auto put = [&](int p, const float4 &v) {
        float *dst = buf + (4 * q) * P + PAD + p;
        sts(dst, v.x);
        sts(dst + P, v.y);
        sts(dst + 2 * P, v.z);
        sts(dst + 3 * P, v.w);
      };
      int p = warp * per_warp + (lane >> qs);
      // 4 loads in flight per thread before their stores
      for (; p + 3 * step < N; p += 4 * step) {
        const float4 a = load4(x, xo + (size_t)p * N + s0 + 4 * q, bf16);
        const float4 b = load4(x, xo + (size_t)(p + step) * N + s0 + 4 * q, bf16);
        const float4 d = load4(x, xo + (size_t)(p + 2 * step) * N + s0 + 4 * q, bf16);
        const float4 e = load4(x, xo + (size_t)(p + 3 * step) * N + s0 + 4 * q, bf16);
        put(p, a);
        put(p + step, b);
        put(p + 2 * step, d);
        put(p + 3 * step, e);
      }
      for (; p < N; p += step) put(p, load4(x, xo + (size_t)p * N + s0 + 4 * q, bf16));
    } else {
      for (int p = warp; p < N; p += kWarps)
        for (int l = lane; l < nl; l += 32)
          sts(buf + l * P + PAD + p, ld_any(x, xo + (size_t)p * N + s0 + l, bf16));
    }
  }
  const int npad = P - N;
  for (int r = warp; r < nl; r += kWarps)
    for (int c = lane; c < npad; c += 32) sts(buf + r * P + (c < PAD ? c : N + c), 0.0f);
}

// The same for 4 images (element offset xo + i N^2), interleaved: position
// p of line l holds the 4 images' values at buf[4 (l P + PAD + p) + i].
// Needs nl <= 8 and an odd pitch P.
//
// Fast path (N, s0, nl multiples of 4): every thread loads 4 consecutive
// values of each image with one 16-byte load (8 bytes for BF16), transposes the
// 4 x 4 block in registers and stores 4 positions of 16 bytes; loads are
// issued in batches of NB blocks before the stores.  The thread mapping
// keeps the stores of each quarter warp in distinct bank quads: rows (mode
// 1): 8 lines x 4 position groups per warp; columns (mode 0): pairs of
// 4-line groups x consecutive positions.
#ifndef SKEI_STAGE_BATCH
#define SKEI_STAGE_BATCH 4
#endif
// 4 x 4 blocks in flight per thread before their stores: the band-sums form
// (whose kernels hold 128 registers) takes kStageBatch, the cluster form 2
// (more would raise its register count and spill)
constexpr int kStageBatch = SKEI_STAGE_BATCH;
__device__ __forceinline__ void store_block(float4 *dst, int step, const float4 (&v)[4]) {
  sts(dst, make_float4(v[0].x, v[1].x, v[2].x, v[3].x));
  sts(dst + step, make_float4(v[0].y, v[1].y, v[2].y, v[3].y));
  sts(dst + 2 * step, make_float4(v[0].z, v[1].z, v[2].z, v[3].z));
  sts(dst + 3 * step, make_float4(v[0].w, v[1].w, v[2].w, v[3].w));
}

template <int PAD = kPad, bool BF = false, int NB = 2>
__device__ __forceinline__ void stage4_t(const void *x, size_t xo, int N, int mode,
                                       int s0, int nl, float *buf, int P) {
  const size_t plane = (size_t)N * N;
  float4 *b4 = reinterpret_cast<float4 *>(buf);
  const int tid = threadIdx.x;
  const bool fast = (N & 3) == 0 && (s0 & 3) == 0 && (nl & 3) == 0;
  // 4 consecutive values of image i at element offset 4 q of the job's
  // group (16 bytes of FP32, 8 of BF16)
  constexpr int bf16 = BF ? 1 : 0;
  const size_t plane4 = plane >> 2;
  const float4 *x4 = reinterpret_cast<const float4 *>(static_cast<const float *>(x) + xo);
  const uint2 *h4 = reinterpret_cast<const uint2 *>(static_cast<const __nv_bfloat16 *>(x) + xo);
  auto ld4 = [&](int i, size_t q4) {
    if constexpr (BF) {
      const uint2 u = __ldg(h4 + i * plane4 + q4);
      return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                         __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
    } else {
      return __ldg(x4 + i * plane4 + q4);
    }
  };
  if (fast && mode == 1) {
    const int pg = tid >> 3;                          // position group
    const int ngroups = N >> 2, step_g = kThreads >> 3;
    const int r = tid & 7;                            // line
    if (r < nl) {
      const size_t row4 = ((size_t)(s0 + r) * N) >> 2;
      float4 *dst = b4 + r * P + PAD;
      int g = pg;
      for (; g + (NB - 1) * step_g < ngroups; g += NB * step_g) {
        float4 v[NB][4];
#pragma unroll
        for (int u = 0; u < NB; ++u)
#pragma unroll
          for (int i = 0; i < 4; ++i) v[u][i] = ld4(i, row4 + g + u * step_g);
#pragma unroll
        for (int u = 0; u < NB; ++u) store_block(dst + 4 * (g + u * step_g), 1, v[u]);
      }
      for (; g < ngroups; g += (NB == 2 ? ngroups : step_g)) {   // NB - 1 blocks at most
        float4 va[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) va[i] = ld4(i, row4 + g);
        store_block(dst + 4 * g, 1, va);
      }
    }
  } else if (fast) {
    const int lgs = nl >> 2;                          // 4-line groups (1 or 2)
    const int lg = tid % lgs, p0 = tid / lgs, step_p = kThreads / lgs;
    float4 *dst = b4 + (4 * lg) * P + PAD;
    int p = p0;
    for (; p + (NB - 1) * step_p < N; p += NB * step_p) {
      float4 v[NB][4];
#pragma unroll
      for (int u = 0; u < NB; ++u)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          v[u][i] = ld4(i, (((size_t)(p + u * step_p) * N + s0) >> 2) + lg);
#pragma unroll
      for (int u = 0; u < NB; ++u) store_block(dst + p + u * step_p, P, v[u]);
    }
    for (; p < N; p += (NB == 2 ? N : step_p)) {   // NB - 1 blocks at most
      float4 va[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) va[i] = ld4(i, (((size_t)p * N + s0) >> 2) + lg);
      store_block(dst + p, P, va);
    }
  } else if (mode == 1) {
    // one position per thread: 4 coalesced loads, one 16-byte store
    for (int r = 0; r < nl; ++r) {
      const size_t src = xo + (size_t)(s0 + r) * N;
      float4 *dst = b4 + r * P + PAD;
      for (int c = tid; c < N; c += kThreads)
        sts(dst + c, make_float4(ld_any(x, src + c, bf16), ld_any(x, src + plane + c, bf16),
                                 ld_any(x, src + 2 * plane + c, bf16),
                                 ld_any(x, src + 3 * plane + c, bf16)));
    }
  } else {
    // 8 consecutive threads take the 8 lines of one position: with an odd
    // pitch their 16-byte stores fall in distinct bank quads
    const int l = tid & 7;
    if (l < nl) {
      for (int p = tid >> 3; p < N; p += kThreads / 8) {
        const size_t src = xo + (size_t)p * N + s0 + l;
        sts(b4 + l * P + PAD + p,
            make_float4(ld_any(x, src, bf16), ld_any(x, src + plane, bf16),
                        ld_any(x, src + 2 * plane, bf16), ld_any(x, src + 3 * plane, bf16)));
      }
    }
  }
  const int npad = P - N;
  for (int e = tid; e < nl * npad; e += kThreads) {
    const int r = e / npad, c = e - r * npad;
    sts(b4 + r * P + (c < PAD ? c : N + c), make_float4(0.0f, 0.0f, 0.0f, 0.0f));
  }
}

// stage4 with the storage type a template argument (no per-load test) and
// NB blocks in flight per thread.
template <int PAD = kPad, int NB = 2>
__device__ __forceinline__ void stage4(const void *x, size_t xo, int bf16, int N, int mode,
                                       int s0, int nl, float *buf, int P) {
  if (bf16) stage4_t<PAD, true, NB>(x, xo, N, mode, s0, nl, buf, P);
  else stage4_t<PAD, false, NB>(x, xo, N, mode, s0, nl, buf, P);
}

// A riding single image's band of 8 lines (FP32, N <= 512, s0 % 4 == 0)
// in two halves, so that its loads fly while the group's band is staged:
// ride_load issues the thread's (at most 4) 16-byte loads in stage1's
// thread mapping, ride_store stores them and zeroes the padding; together
// they write what stage1 writes.
__device__ __forceinline__ bool ride_split(int bf16, int N, int s0, int nl, bool fast) {
  return fast && !bf16 && N <= 512 && nl == 8 && kWarps == 8 && (s0 & 3) == 0;
}
__device__ __forceinline__ void ride_load(const void *x, size_t xo, int N, int mode, int s0,
                                          float4 (&v)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    v[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (mode == 1) {
      const int c = 4 * lane + 128 * u;   // line s0 + warp, positions c .. c+3
      if (c < N) v[u] = load4(x, xo + (size_t)(s0 + warp) * N + c, 0);
    } else {
      const int p = warp * 16 + (lane >> 1) + 128 * u;   // column p, lines s0 + 4 (lane & 1) ..
      if (p < N) v[u] = load4(x, xo + (size_t)p * N + s0 + 4 * (lane & 1), 0);
    }
  }
}
template <int PAD>
__device__ __forceinline__ void ride_store(int N, int mode, float *buf, int P,
                                           const float4 (&v)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (mode == 1) {
      const int c = 4 * lane + 128 * u;
      if (c < N) sts(reinterpret_cast<float4 *>(buf + warp * P + PAD + c), v[u]);
    } else {
      const int p = warp * 16 + (lane >> 1) + 128 * u;
      if (p < N) {
        float *dst = buf + (4 * (lane & 1)) * P + PAD + p;
        sts(dst, v[u].x);
        sts(dst + P, v[u].y);
        sts(dst + 2 * P, v[u].z);
        sts(dst + 3 * P, v[u].w);
      }
    }
  }
  const int npad = P - N;
  for (int r = warp; r < 8; r += kWarps)
    for (int c = lane; c < npad; c += 32) sts(buf + r * P + (c < PAD ? c : N + c), 0.0f);
}

// Line range [lo, hi) within [s0, s1) on which lam0 + L * lam1 lies in
// (lo_bound, hi_bound); inv1 = 1 / lam1.
__device__ __forceinline__ void line_range(float lam0, float lam1, float inv1, float lo_bound,
                                           float hi_bound, int s0, int s1, int *lo, int *hi) {
  if (fabsf(lam1) < 1e-20f) {
    const bool in = lam0 > lo_bound && lam0 < hi_bound;
    *lo = s0;
    *hi = in ? s1 : s0;
    return;
  }
  const float la = (lo_bound - lam0) * inv1, lb = (hi_bound - lam0) * inv1;
  const float lmin = fmaxf(fminf(la, lb), (float)s0);
  const float lmax = fminf(fmaxf(la, lb), (float)(s1 - 1));
  *lo = (int)ceilf(lmin);
  *hi = (int)floorf(lmax) + 1;
}

// Joseph: adds to acc[i] the linear interpolations of image i of the group
// at the fixed-point crossings pos(L, k) = G + k A + L T of lines [s0, s1)
// of the staged band, line by line in order; with XTRA also those of a
// riding single image staged at bufx (pitch Px) into *accx, from the same
// positions and weights.
template <int NI, bool XTRA = false>
__device__ __forceinline__ void joseph_lines(const AngleConst &C, int k, int s0, int s1, int N,
                                             const float *buf, int P, float (&acc)[NI],
                                             const float *bufx = nullptr, int Px = 0,
                                             float *accx = nullptr) {
  int lo, hi;
  // taps are nonzero only for pos in (-1, N); the relaxed window keeps every
  // such line and never reads beyond the kPad zero positions
  line_range(fmaf((float)k, C.Af, C.Gf), C.Tf, C.invT, -1.5f, (float)N + 0.5f, s0, s1, &lo, &hi);
  if (lo >= hi) return;
  const long long T = C.T;
  long long pos = C.G + (long long)k * C.A + (long long)lo * T;
  const float *row = buf + ((lo - s0) * P + kPad) * NI;
  const float *rowx = XTRA ? bufx + (lo - s0) * Px + kPad : nullptr;
  float ax = XTRA ? *accx : 0.0f;
#pragma unroll 4
  for (int l = lo; l < hi; ++l) {
    const int j0 = ipart(pos);
    const float f = frac23(pos);
    const float g = 1.0f - f;
    if (NI == 4) {
      const float4 v0 = *reinterpret_cast<const float4 *>(row + 4 * j0);
      const float4 v1 = *reinterpret_cast<const float4 *>(row + 4 * j0 + 4);
      acc[0] = fmaf(g, v0.x, fmaf(f, v1.x, acc[0]));
      acc[1] = fmaf(g, v0.y, fmaf(f, v1.y, acc[1]));
      acc[2] = fmaf(g, v0.z, fmaf(f, v1.z, acc[2]));
      acc[3] = fmaf(g, v0.w, fmaf(f, v1.w, acc[3]));
    } else {
      acc[0] = fmaf(g, row[j0], fmaf(f, row[j0 + 1], acc[0]));
    }
    if (XTRA) {
      ax = fmaf(g, rowx[j0], fmaf(f, rowx[j0 + 1], ax));
      rowx += Px;
    }
    row += P * NI;
    pos += T;
  }
  if (XTRA) *accx = ax;
}

// A tap weight max(1 - |e|, 0) of an offset e = E 2^-28 whose sign is known
// (NEG: E < 0; else E >= 0), exactly as the back-projector weights it
// (fraction truncated to 2^-23), clamped in FP32.
template <bool NEG>
__device__ __forceinline__ float side_weight(int E) {
  const int a = E >> (kFxBits - 23);
  const float w = __int_as_float(NEG ? 0x40000000 + a : 0x40000000 - a) - 1.0f;
  return fmaxf(w, 0.0f);
}

// B^T for bin k: adds to acc[i] the pixels of lines [s0, s1) of image i
// whose bin coordinate t(L, P) = t00 + L bline + P bstep lies in (k-1, k+1),
// weighted exactly as the back-projector weights them.  At most 3 pixels per
// line (|bstep| >= 1/sqrt 2): the nearest one, r, at the exact offset
// D = t(L, r) - k (|D| <= |bstep|/2, 32-bit fixed point), and its two
// neighbours at D -+ |bstep|.  r and D are carried from line to line: D
// grows by bline (|bline| <= |bstep|), and one step of r re-centres it.
template <int NI>
__device__ __forceinline__ void bpadj_lines(const AngleConst &C, int k, int s0, int s1, int N,
                                            const float *buf, int P, float (&acc)[NI]) {
  const float kf = (float)k;
  const float inv = C.inv_bstep;
  int lo, hi;
  // the nearest pixel must come within sqrt(2) of [0, N-1]; relaxed window,
  // so that r stays in [-3, N+2] and its neighbours in the kPad zero positions
  line_range((kf - C.t00f) * inv, -C.blinef * inv, -C.bstepf * C.inv_bline, -2.5f,
             (float)N + 1.5f, s0, s1, &lo, &hi);
  if (lo >= hi) return;
  const int bs = (int)(unsigned)C.bstep, bl = (int)(unsigned)C.bline;
  const int abs_bs = abs(bs), half = abs_bs >> 1, sgn = bs < 0 ? -1 : 1;
  int r = round_int((kf - fmaf((float)lo, C.blinef, C.t00f)) * inv);
  // D = t(lo, r) - k on the low words (exact: |D| < 2^31)
  int D = (int)((unsigned)(C.t00 + (long long)lo * C.bline) + (unsigned)r * (unsigned)bs -
                ((unsigned)k << kFxBits));
  // the neighbour at offset D - |bs| sits at r - sgn, the one at D + |bs| at
  // r + sgn
  const int step = sgn * NI;
  const float *row = buf + ((lo - s0) * P + kPad) * NI;
  for (int l = lo; l < hi; ++l) {
    if (D > half) { r -= sgn; D -= abs_bs; }
    else if (D < -half) { r += sgn; D += abs_bs; }
    const float w_lo = side_weight<true>(D - abs_bs);
    const float w_mid = __int_as_float(0x40000000 - abs(D >> (kFxBits - 23))) - 1.0f;
    const float w_hi = side_weight<false>(D + abs_bs);
    const float *q = row + r * NI;
    if (NI == 4) {
      const float4 a = *reinterpret_cast<const float4 *>(q - step);
      const float4 b = *reinterpret_cast<const float4 *>(q);
      const float4 c = *reinterpret_cast<const float4 *>(q + step);
      acc[0] = fmaf(w_hi, c.x, fmaf(w_mid, b.x, fmaf(w_lo, a.x, acc[0])));
      acc[1] = fmaf(w_hi, c.y, fmaf(w_mid, b.y, fmaf(w_lo, a.y, acc[1])));
      acc[2] = fmaf(w_hi, c.z, fmaf(w_mid, b.z, fmaf(w_lo, a.z, acc[2])));
      acc[3] = fmaf(w_hi, c.w, fmaf(w_mid, b.w, fmaf(w_lo, a.w, acc[3])));
    } else {
      acc[0] = fmaf(w_hi, q[step], fmaf(w_mid, q[0], fmaf(w_lo, q[-step], acc[0])));
    }
    D += bl;
    row += P * NI;
  }
}

// The list positions spos[0 .. na) of slots a_begin .. a_begin + na - 1 of
// the mode-partitioned order of an angle list (the row-mode angles in list
// order, then the others: column mode and bad indices), so that a block of
// consecutive slots stages its band in one layout; at most one block of a
// launch holds both.  The list lives on the device (a sketch drawn per
// step), so every CTA ranks it: a count, then a ballot scan per chunk.
__device__ __forceinline__ bool row_mode_at(const int *idx, int i, int n_angles,
                                            const AngleConst *ang) {
  const int ai = idx ? idx[i] : i;
  return ai >= 0 && ai < n_angles && ang[ai].mode == 1;
}

__device__ void partition_block(const int *idx, int m, int n_angles, const AngleConst *ang,
                                int a_begin, int na, int *spos, int *wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int rows_total = 0;
  for (int c0 = 0; c0 < m; c0 += kThreads) {
    const int i = c0 + tid;
    const unsigned bal = __ballot_sync(0xffffffffu, i < m && row_mode_at(idx, i, n_angles, ang));
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    for (int w = 0; w < kWarps; ++w) rows_total += wsum[w];
    __syncthreads();
  }
  int base = 0;
  for (int c0 = 0; c0 < m; c0 += kThreads) {
    const int i = c0 + tid;
    const bool f = i < m && row_mode_at(idx, i, n_angles, ang);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = base;   // row-mode angles before position i
    for (int w = 0; w < warp; ++w) before += wsum[w];
    before += __popc(bal & ((1u << lane) - 1u));
    const int slot = f ? before : rows_total + (i - before);
    if (i < m && slot >= a_begin && slot < a_begin + na) spos[slot - a_begin] = i;
    for (int w = 0; w < kWarps; ++w) base += wsum[w];
    __syncthreads();
  }
}

// One task: the NI images b0.. of job J, slots [a_begin, a_begin + g.AB)
// of the mode-partitioned order of its angle list, computed by the 8 CTAs of
// this cluster.  Ends with a cluster barrier, after which the CTA's shared
// memory may be reused.
template <int OP, int NI>
__device__ __forceinline__ void band_task(const Job &J, int b0, int a_begin, const BandGeom &g,
                                          const AngleConst *ang, int *status, float *smem,
                                          AngleConst *sc, int *sai, int *spos, int *wsum,
                                          cg::cluster_group &cluster) {
  const int tid = threadIdx.x;
  const int band = (int)cluster.block_rank();
  if (a_begin >= J.m) return;  // uniform over the cluster: no peer waits for it
  const int na = min(g.AB, J.m - a_begin);
  const int nd = g.n_det, N = g.N;
  float *part = smem;                                       // [AB][n_det][NI]
  float *buf = smem + band_part_floats(g);                  // [SB][P][NI], 16-byte aligned

  const int *idx = job_idx(J, b0);
  partition_block(idx, J.m, g.n_angles, ang, a_begin, na, spos, wsum);
  if (tid < kMaxAB) {
    int ai = -1;
    if (tid < na) {
      ai = idx ? idx[spos[tid]] : spos[tid];
      if (ai < 0 || ai >= g.n_angles) {
        if (band == 0) atomicOr(status, 1);
        ai = -1;
      }
    }
    sai[tid] = ai;
    if (ai >= 0) sc[tid] = ang[ai];
  }
  for (int e = tid; e < na * nd * NI; e += kThreads) part[e] = 0.0f;
  __syncthreads();

  const size_t xo = (size_t)b0 * N * N;
  const int L0 = band * g.R, L1 = min(N, L0 + g.R);
  for (int mode = 1; mode >= 0; --mode) {
    bool any = false;
    for (int a = 0; a < na; ++a) any |= (sai[a] >= 0 && sc[a].mode == mode);
    if (!any) continue;
    const int P = mode ? g.Prow : g.Pcol;
    for (int s0 = L0; s0 < L1; s0 += g.SB) {
      const int s1 = min(L1, s0 + g.SB), nl = s1 - s0;
      __syncthreads();  // the previous sub-band is no longer read
      if (NI == 4) stage4(J.in, xo, J.in_bf16, N, mode, s0, nl, buf, P);
      else stage1(J.in, xo, J.in_bf16, N, mode, s0, nl, buf, P, g.fast != 0);
      __syncthreads();
      for (int a = 0; a < na; ++a) {
        if (sai[a] < 0 || sc[a].mode != mode) continue;
        for (int k = tid; k < nd; k += kThreads) {
          float *pp = part + (a * nd + k) * NI;
          float acc[NI];
          if (NI == 4) {
            const float4 t = *reinterpret_cast<const float4 *>(pp);
            acc[0] = t.x;
            acc[1] = t.y;
            acc[2] = t.z;
            acc[3] = t.w;
          } else {
            acc[0] = pp[0];
          }
          if (OP == OP_JOSEPH) joseph_lines<NI>(sc[a], k, s0, s1, N, buf, P, acc);
          else bpadj_lines<NI>(sc[a], k, s0, s1, N, buf, P, acc);
          if (NI == 4)
            *reinterpret_cast<float4 *>(pp) = make_float4(acc[0], acc[1], acc[2], acc[3]);
          else
            pp[0] = acc[0];
        }
      }
    }
  }

  cluster.sync();
  const int n_items = na * nd;
  for (int it = band * kThreads + tid; it < n_items; it += kBands * kThreads) {
    const int a = it / nd, k = it - a * nd;
    float s[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) s[i] = 0.0f;
#pragma unroll
    for (int q = 0; q < kBands; ++q) {
      const float *pq = cluster.map_shared_rank(part, q) + it * NI;
      if (NI == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(pq);
        s[0] += t.x;
        s[1] += t.y;
        s[2] += t.z;
        s[3] += t.w;
      } else {
        s[0] += pq[0];
      }
    }
    const int ai = sai[a];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int b = b0 + i;
      const size_t o = ((size_t)b * J.m + spos[a]) * nd + k;
      float v;
      if (ai < 0) {
        v = 0.0f;
      } else if (OP == OP_JOSEPH) {
        v = s[i] * sc[a].W;
        if (J.aux) v = ld_any(J.aux, ((size_t)b * g.n_angles + ai) * nd + k, J.aux_bf16) - v;
        v *= J.alpha;
      } else {
        v = s[i] * J.alpha;
      }
      st_any(J.out, o, v, J.out_bf16);
    }
  }
  cluster.sync();  // keep this CTA's sums alive until every peer has read them
}

template <int OP>
__global__ void __cluster_dims__(kBands, 1, 1) __launch_bounds__(kThreads)
    band_kernel(const BandArgs args) {
  pdl_enter();
  extern __shared__ float4 smem4[];
  __shared__ AngleConst sc[kMaxAB];
  __shared__ int sai[kMaxAB], spos[kMaxAB], wsum[kWarps];
  cg::cluster_group cluster = cg::this_cluster();
  // the job and image group of this cluster
  const int z = blockIdx.z;
  const int g0 = n_groups(args.jobs.j[0].nimg, args.gmax);
  const int jn = (args.jobs.njobs > 1 && z >= g0) ? 1 : 0;
  const Job &J = args.jobs.j[jn];
  int b0, ni;
  group_at(J.nimg, z - (jn ? g0 : 0), &b0, &ni, args.gmax);
  float *smem = reinterpret_cast<float *>(smem4);
  if (ni == 4)
    band_task<OP, 4>(J, b0, blockIdx.y * args.g4.AB, args.g4, args.ang, args.status, smem, sc,
                     sai, spos, wsum, cluster);
  else
    band_task<OP, 1>(J, b0, blockIdx.y * args.g1.AB, args.g1, args.ang, args.status, smem, sc,
                     sai, spos, wsum, cluster);
}

// Persistent form over the tasks of a batch of instances (plans of their
// own): each cluster takes the next task from a global counter (tasks come
// in decreasing cost order) until none is left; the last cluster to finish
// resets the counter for the next launch.  Task = (item, b0 << 3 | group
// size, first angle, 0).
template <int OP>
__global__ void __cluster_dims__(kBands, 1, 1) __launch_bounds__(kThreads)
    band_batch_kernel(const BatchItem *items, const int4 *tasks, int n_tasks, int AB,
                      int *queue) {
  extern __shared__ float4 smem4[];
  __shared__ AngleConst sc[kMaxAB];
  __shared__ int sai[kMaxAB], spos[kMaxAB], wsum[kWarps];
  __shared__ int s_task;
  cg::cluster_group cluster = cg::this_cluster();
  const bool leader = cluster.block_rank() == 0 && threadIdx.x == 0;
  float *smem = reinterpret_cast<float *>(smem4);
  for (;;) {
    if (leader) s_task = atomicAdd(queue, 1);
    cluster.sync();
    const int t = *cluster.map_shared_rank(&s_task, 0);
    cluster.sync();  // every CTA has read it: the leader may overwrite it, or exit
    if (t >= n_tasks) break;
    const int4 tk = tasks[t];
    const BatchItem &it = items[tk.x];
    const Job J{it.in, nullptr, it.out, it.idx, it.m, it.B, it.alpha, 0.0f,
                it.in_bf16, 0, it.out_bf16};
    const int b0 = tk.y >> 3, ni = tk.y & 7;
    if (ni == 4) {
      const BandGeom g = band_geom(it.N, it.n_det, it.n_angles, OP, AB, 4);
      band_task<OP, 4>(J, b0, tk.z, g, it.ang, it.status, smem, sc, sai, spos, wsum, cluster);
    } else {
      const BandGeom g = band_geom(it.N, it.n_det, it.n_angles, OP, AB, 1);
      band_task<OP, 1>(J, b0, tk.z, g, it.ang, it.status, smem, sc, sai, spos, wsum, cluster);
    }
  }
  if (leader) queue_retire(queue, gridDim.x / kBands);
}

template <int OP>
int set_band_smem(size_t smem) {
  static size_t configured[64] = {0}, configured_batch[64] = {0};
  SKEI_TRY(opt_in_smem(band_kernel<OP>, smem, configured, "band kernel: shared memory attribute"));
  SKEI_TRY(opt_in_smem(band_batch_kernel<OP>, smem, configured_batch,
                       "band kernel: shared memory attribute"));
  return SKEI_OK;
}

// Estimated time of a launch with `ab` angles per cluster: greedy list
// scheduling of its cluster tasks (decreasing cost, each to the slot that
// frees first) on `slots` concurrent clusters.  A task of a group of ni
// images costs ni (angles x bin passes + staging), the staging of the band
// counting as `stage4` angles for groups of 4 and `stage1` for single images.
double band_estimate(const Jobs &jobs, int nd, int ab, int slots, int gm, double stage4,
                     double stage1) {
  std::vector<double> cost;
  const double cw = (double)nd / kThreads;   // bin passes per thread
  for (int q = 0; q < jobs.njobs; ++q) {
    const Job &J = jobs.j[q];
    const int g4 = gm == 4 ? J.nimg >> 2 : 0, g1 = J.nimg - 4 * g4;
    for (int a0 = 0; a0 < J.m; a0 += ab) {
      const int na = std::min(ab, J.m - a0);
      for (int i = 0; i < g4; ++i) cost.push_back(4.0 * (na * cw + stage4));
      for (int i = 0; i < g1; ++i) cost.push_back(na * cw + stage1);
    }
  }
  std::sort(cost.begin(), cost.end(), [](double x, double y) { return x > y; });
  std::priority_queue<double, std::vector<double>, std::greater<double>> load;
  for (int i = 0; i < std::max(slots, 1); ++i) load.push(0.0);
  double span = 0.0;
  for (double c : cost) {
    const double t = load.top() + c;
    load.pop();
    load.push(t);
    span = std::max(span, t);
  }
  return span;
}

// Angles per cluster for group size gm: the smallest estimated time, ties
// to the larger block (less staging).  Also returns the number of cluster
// tasks and concurrent cluster slots of that choice.
template <int OP>
int choose_ab(skei_plan p, const Jobs &jobs, int gm, int *tasks, int *slots_out) {
  int m_max = 0;
  bool any4 = false, any1 = false;
  for (int q = 0; q < jobs.njobs; ++q) {
    m_max = max(m_max, jobs.j[q].m);
    any4 |= gm == 4 && jobs.j[q].nimg >= 4;
    any1 |= gm != 4 || (jobs.j[q].nimg & 3) != 0;
  }
  const int ab_max = min(kMaxAB, m_max);
  int best_ab = 1, best_slots = 1;
  double best_cost = 1e300;
  for (int ab = 1; ab <= ab_max; ++ab) {
    size_t bytes = 0;
    if (any4)
      bytes = std::max(bytes, band_smem(band_geom(p->N, p->n_det, p->n_angles, OP, ab, 4)));
    if (any1)
      bytes = std::max(bytes, band_smem(band_geom(p->N, p->n_det, p->n_angles, OP, ab, 1)));
    if (bytes > 200 * 1024) continue;
    int per_sm = (int)((228 * 1024) / (bytes + 2304));
    per_sm = max(1, min(per_sm, 8));
    const int slots = max(1, sm_count() * per_sm / kBands);
    // a single image's staging costs about 0.4 angles per 16 staged lines
    const int sb1 = band_geom(p->N, p->n_det, p->n_angles, OP, ab, 1).SB;
    const double cost = band_estimate(jobs, p->n_det, ab, slots, gm, 1.0, 0.4 * sb1 / 16.0);
    if (cost <= best_cost) { best_cost = cost; best_ab = ab; best_slots = slots; }
  }
  if (SKEI_BAND_AB > 0) best_ab = min(SKEI_BAND_AB, ab_max);
  int n = 0;
  for (int q = 0; q < jobs.njobs; ++q)
    n += n_groups(jobs.j[q].nimg, gm) * ((jobs.j[q].m + best_ab - 1) / best_ab);
  *tasks = n;
  *slots_out = best_slots;
  return best_ab;
}

template <int OP>
int launch_band(skei_plan p, const Jobs &jobs, cudaStream_t st) {
  // groups of 4 pay only when, with one angle per cluster, they still leave
  // a cluster task for every concurrent cluster slot: otherwise the launch
  // runs single images
  int gm = jobs_groupable(jobs) ? group_max(OP) : 1, tasks = 0, slots = 1;
  if (gm == 4) {
    int t1 = 0;
    for (int q = 0; q < jobs.njobs; ++q) t1 += n_groups(jobs.j[q].nimg, 4) * jobs.j[q].m;
    const size_t bytes = band_smem(band_geom(p->N, p->n_det, p->n_angles, OP, 1, 4));
    const int per_sm = max(1, min((int)((228 * 1024) / (bytes + 2304)), 8));
    if (t1 < max(1, sm_count() * per_sm / kBands)) gm = 1;
  }
  const int ab = choose_ab<OP>(p, jobs, gm, &tasks, &slots);
  int m_max = 0, ngroups = 0;
  bool any4 = false, any1 = false;
  for (int q = 0; q < jobs.njobs; ++q) {
    m_max = max(m_max, jobs.j[q].m);
    ngroups += n_groups(jobs.j[q].nimg, gm);
    any4 |= gm == 4 && jobs.j[q].nimg >= 4;
    any1 |= gm != 4 || (jobs.j[q].nimg & 3) != 0;
  }
  if (ngroups > 65535) return set_error(SKEI_EINVAL, "too many images in one launch");
  BandArgs a{jobs, p->d_ang, p->d_status,
             band_geom(p->N, p->n_det, p->n_angles, OP, ab, 1),
             band_geom(p->N, p->n_det, p->n_angles, OP, ab, 4), gm};
  size_t smem = 0;
  if (any4) smem = std::max(smem, band_smem(a.g4));
  if (any1) smem = std::max(smem, band_smem(a.g1));
  if (smem > 227 * 1024)
    return set_error(SKEI_EINVAL, "detector of %d bins needs too much shared memory", p->n_det);
  SKEI_TRY(set_band_smem<OP>(smem));
  const int blocks = (m_max + ab - 1) / ab;
  dim3 grid(kBands, blocks, ngroups);
  launch_k(band_kernel<OP>, grid, dim3(kThreads), smem, st, a);
  return check_launch(OP == OP_JOSEPH ? "joseph forward launch" : "back-projection transpose launch");
}

// The persistent launch of a batch: `clusters` clusters of kBands CTAs over
// `n_tasks` tasks; smem is the largest task's dynamic shared memory.
template <int OP>
int launch_band_batch(const BatchItem *items, const int4 *tasks, int n_tasks, int AB,
                      size_t smem, int clusters, int *queue, cudaStream_t st) {
  SKEI_TRY(set_band_smem<OP>(smem));
  band_batch_kernel<OP><<<clusters * kBands, kThreads, smem, st>>>(items, tasks, n_tasks, AB,
                                                                 queue);
  return check_launch(OP == OP_JOSEPH ? "batched joseph forward launch"
                                      : "batched back-projection transpose launch");
}

template <int OP>
int band_batch_clusters(size_t smem, int *clusters) {
  SKEI_TRY(set_band_smem<OP>(smem));
  // the kernel's cluster shape is compiled in (__cluster_dims__)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kBands * 64, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&n, band_batch_kernel<OP>, &cfg);
  if (e != cudaSuccess) return cuda_error(e, "band kernel: cluster occupancy");
  *clusters = n > 0 ? n : 1;
  return SKEI_OK;
}

// ------------------------------------------------ band-partial form --
// For callers that pass a workspace (the fused SkEI step): a CTA stages a
// thin band of SBL lines of an image group ONCE and computes every angle of
// its angle block over it, writing the per-band sums to the workspace,
// [image][band][angle][bin]; a second kernel adds the bands in order and
// applies the epilogue.  Each image band is read from L2 once per angle
// block instead of once per angle, and the CTAs are many and short.
#ifndef SKEI_PART_SBL1
#define SKEI_PART_SBL1 16
#endif
#ifndef SKEI_PART_AB
#define SKEI_PART_AB 0        // angles per partial CTA (0: from SKEI_PART_CTAS)
#endif
// The 4-image partial kernel comes in two register budgets: 128 registers
// (2 CTAs per SM) for launches that fit one wave at 2 per SM, 80 (3 per SM)
// for larger ones.
#ifndef SKEI_PART_MERGE
#define SKEI_PART_MERGE 1
#endif
#ifndef SKEI_PART_MINB1
#define SKEI_PART_MINB1 1     // CTAs per SM the single-image kernel's registers must allow
#endif
#ifndef SKEI_PART_SBL4
#define SKEI_PART_SBL4 8
#endif
static_assert(SKEI_PART_SBL4 == 8, "4-image bands are staged 8 lines at a time");
#ifndef SKEI_PART_GROUP
#define SKEI_PART_GROUP 4
#endif
#ifndef SKEI_PART_CTAS
#define SKEI_PART_CTAS 2      // CTAs per SM of the one wave the angle block aims at
#endif
#ifndef SKEI_PART_MINB4
#define SKEI_PART_MINB4 2     // CTAs per SM the one-wave 4-image kernel's registers must allow
#endif
constexpr int kMaxABP = 32;      // angles per partial CTA

// Staging geometry of one band of SB lines (0: the group size's default).
// A staged line carries kPartPad(SB) zero positions on each side: wide
// enough that every tap of a ray (A) or bin (B^T) that meets the band at all
// falls inside the padded line, so the band's lines are summed without
// per-line range tests.  Transposed single-image staging writes 4-line
// groups of (32 / (SB/4)) positions per warp: a column pitch = 4 mod 8
// (8 lines), 2 mod 8 (16) or odd (32) keeps them in distinct banks.
__host__ __device__ constexpr int kPartPad(int SB) { return SB + 8; }
__host__ __device__ __forceinline__ BandGeom part_geom(int N, int n_det, int n_angles, int NI,
                                                       int SB = 0) {
  BandGeom g;
  g.N = N;
  g.n_det = n_det;
  g.n_angles = n_angles;
  g.NI = NI;
  g.R = 0;
  g.SB = SB > 0 ? SB : (NI == 1 ? SKEI_PART_SBL1 : SKEI_PART_SBL4);
  const int pad = kPartPad(g.SB);
  if (NI == 1) {
    g.Prow = (N + 2 * pad + 3) & ~3;
    g.Pcol = g.SB == 32   ? ((N + 2 * pad) | 1)
             : g.SB == 16 ? ((N + 2 * pad - 2 + 7) & ~7) + 2
                          : ((N + 2 * pad - 4 + 7) & ~7) + 4;
  } else {
    g.Pcol = (N + 2 * pad) | 1;
    g.Prow = g.Pcol;
  }
  g.AB = 0;
  g.fast = (N % 8 == 0) ? 1 : 0;
  return g;
}
__host__ __device__ __forceinline__ size_t part_smem(const BandGeom &g) {
  const int Pmax = g.Prow > g.Pcol ? g.Prow : g.Pcol;
  return (size_t)g.SB * Pmax * g.NI * 4;
}

struct PartArgs {
  Jobs jobs;
  const AngleConst *ang;
  int *status;
  BandGeom g1, g4;
  int gmax[kMaxJobs];   // image group size of each job (1 or 4)
  int AB;            // angles per CTA
  int nbands;        // ceil(N / SBL); both group sizes use SBL of their own
  float *part;       // workspace
  size_t off[kMaxJobs];   // float offset of each job's sums
  int merge;         // A: job 0's image z rides with job 1's group 4z .. 4z+3 (same angles)
  size_t work_floats;   // workspace extent (range checks of the check build)
};

// Joseph over the SB staged lines of a band for ray k: adds to acc[i] the
// linear interpolations of image i of the group at the crossings
// pos(s0 + l, k) = G0 + k A + l T, l = 0 .. SB-1 (G0 = G + s0 T), line by
// line in order; with XTRA also those of a riding single image staged at
// bufx (pitch Px) into ax, from the same positions and weights.
//
// The positions are exact: every 8 lines the 64-bit crossing is split into
// its nearest integer J0 and a 32-bit offset r (|r| <= 1/2 px), and r + l T
// (|T| <= 1 px, l < 8, so |r| < 8 px: no overflow of the 28 fractional
// bits) gives each line's integer part J0 + (r >> 28) and the 23-bit
// fraction of its low bits, bitwise those of the 64-bit position.  A ray
// with no crossing inside (-1, N) on any line of the band adds nothing and
// is skipped; for the others every tap lies within SB + 1 positions of the
// image, inside the kPartPad(SB) zero positions of each staged line, so
// crossings outside the image read zeros and add exact zeros: no per-line
// range test.
template <int SB, int NI, bool XTRA>
__device__ __forceinline__ void joseph_band(const AngleConst &C, long long G0, int k, int N,
                                            const float *buf, int P, float (&acc)[NI],
                                            const float *bufx, int Px, float &ax) {
  static_assert(SB % 8 == 0, "bands of whole 8-line blocks");
  constexpr int PAD = kPartPad(SB);
  const long long T = C.T;
  const long long p0 = G0 + (long long)k * C.A;
  const long long pl = p0 + (long long)(SB - 1) * T;
  const long long lo = p0 < pl ? p0 : pl, hi = p0 < pl ? pl : p0;
  if (hi <= -kFxOne || lo >= ((long long)N << kFxBits)) return;
  const int T32 = (int)T;
  // the 4 images' sums as two FP32 pairs (f32x2 FMAs)
  f2x a01 = 0ull, a23 = 0ull;
  if constexpr (NI == 4) {
    a01 = f2_pack(acc[0], acc[1]);
    a23 = f2_pack(acc[2], acc[3]);
  }
#pragma unroll
  for (int h = 0; h < SB; h += 8) {
    const long long ph = p0 + (long long)h * T;
    const int J0 = (int)((ph + (kFxOne >> 1)) >> kFxBits);
    int r = (int)(ph - ((long long)J0 << kFxBits));
    const float *row = buf + (h * P + J0 + PAD) * NI;
    const float *rowx = XTRA ? bufx + h * Px + J0 + PAD : nullptr;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int j = r >> kFxBits;
      const float f =
          __uint_as_float(0x3F800000u | (((unsigned)r >> (kFxBits - 23)) & 0x7FFFFFu)) - 1.0f;
      const float g = 1.0f - f;
      const float *q = row + (l * P + j) * NI;
      if (NI == 4) {
        const ulonglong2 v0 = lds_ck(reinterpret_cast<const ulonglong2 *>(q), CK_BAND_TAP);
        const ulonglong2 v1 = lds_ck(reinterpret_cast<const ulonglong2 *>(q + 4), CK_BAND_TAP);
        const f2x ff = f2_pack(f, f), gg = f2_pack(g, g);
        a01 = f2_fma(gg, v0.x, f2_fma(ff, v1.x, a01));
        a23 = f2_fma(gg, v0.y, f2_fma(ff, v1.y, a23));
      } else {
        acc[0] = fmaf(g, lds_ck(q, CK_BAND_TAP), fmaf(f, lds_ck(q + 1, CK_BAND_TAP), acc[0]));
      }
      if (XTRA) {
        const float *qx = rowx + l * Px + j;
        ax = fmaf(g, lds_ck(qx, CK_BAND_TAP), fmaf(f, lds_ck(qx + 1, CK_BAND_TAP), ax));
      }
      r += T32;
    }
  }
  if constexpr (NI == 4) {
    acc[0] = f2_lo(a01);
    acc[1] = f2_hi(a01);
    acc[2] = f2_lo(a23);
    acc[3] = f2_hi(a23);
  }
}

// The weight max(1 - |E|, 0) of an exact offset E = e 2^-28 of known sign
// (NEG: E < 0), as the back-projector weights it: the fraction truncated to
// 23 bits, clamped by a saturating add.
template <bool NEG>
__device__ __forceinline__ float side_weight_sat(int E) {
  const int a = E >> (kFxBits - 23);
  return __saturatef(__int_as_float(NEG ? 0x40000000 + a : 0x40000000 - a) - 1.0f);
}

// One line of B^T for bin k: the nearest pixel r (exact offset D = t(L, r)
// - k, |D| <= |bstep|/2 after one re-centring step) and its neighbours r-1,
// r+1, weighted as the back-projector weights them, added in the order
// r-1, r, r+1.  UP: D can only leave [-half, half] upwards (bline >= 0) or,
// with !UP, downwards; FIRST checks both sides (the first line's r comes
// from an FP32 estimate).
template <int NI, bool FIRST, bool UP>
__device__ __forceinline__ void bpadj_line(int &r, int &D, int half, int abs_bs, int sgn,
                                           const float *row, float (&acc)[NI], f2x &a01,
                                           f2x &a23) {
  if (FIRST ? D > half : (UP && D > half)) { r -= sgn; D -= abs_bs; }
  else if (FIRST ? D < -half : (!UP && D < -half)) { r += sgn; D += abs_bs; }
  const float w_m = side_weight_sat<true>(D - abs_bs);     // pixel r - sgn
  const float w_mid = __int_as_float(0x40000000 - abs(D >> (kFxBits - 23))) - 1.0f;
  const float w_p = side_weight_sat<false>(D + abs_bs);    // pixel r + sgn
  const float wl = sgn > 0 ? w_m : w_p, wr = sgn > 0 ? w_p : w_m;
  const float *q = row + r * NI;
  if (NI == 4) {
    // the 4 images' sums as two FP32 pairs (f32x2 FMAs)
    const ulonglong2 a = lds_ck(reinterpret_cast<const ulonglong2 *>(q - 4), CK_BAND_TAP);
    const ulonglong2 b = lds_ck(reinterpret_cast<const ulonglong2 *>(q), CK_BAND_TAP);
    const ulonglong2 c = lds_ck(reinterpret_cast<const ulonglong2 *>(q + 4), CK_BAND_TAP);
    const f2x wl2 = f2_pack(wl, wl), wm2 = f2_pack(w_mid, w_mid), wr2 = f2_pack(wr, wr);
    a01 = f2_fma(wr2, c.x, f2_fma(wm2, b.x, f2_fma(wl2, a.x, a01)));
    a23 = f2_fma(wr2, c.y, f2_fma(wm2, b.y, f2_fma(wl2, a.y, a23)));
  } else {
    acc[0] = fmaf(wr, lds_ck(q + 1, CK_BAND_TAP),
                  fmaf(w_mid, lds_ck(q, CK_BAND_TAP), fmaf(wl, lds_ck(q - 1, CK_BAND_TAP), acc[0])));
  }
}

// B^T over the SB staged lines of a band for bin k: on each line
// L = s0 + l the pixels whose bin coordinate t(L, P) = T0 + l bline +
// P bstep (T0 = t00 + s0 bline) lies within one bin of k.  r and D are
// carried from line to line (D grows by bline, |bline| <= |bstep|, so one
// re-centring step per line keeps |D| <= |bstep|/2).  A bin whose nearest
// pixels stay more than 2 positions outside the image on every line of the
// band adds nothing and is skipped; for the others every tap lies within
// SB + 4 positions of the image, inside the zero padding.
template <int SB, int NI>
__device__ __forceinline__ void bpadj_band(const AngleConst &C, long long T0, float T0f, int k,
                                           int N, const float *buf, int P, float (&acc)[NI]) {
  constexpr int PAD = kPartPad(SB);
  const float inv = C.inv_bstep;
  const float c0 = ((float)k - T0f) * inv;                       // nearest pixel, first line
  const float cl = fmaf(-(float)(SB - 1) * C.blinef, inv, c0);   // and last line
  if (fmaxf(c0, cl) < -3.0f || fminf(c0, cl) > (float)N + 2.0f) return;
  int r = round_int(c0);
  const int bs = (int)(unsigned)C.bstep, bl = (int)(unsigned)C.bline;
  const int abs_bs = abs(bs), half = abs_bs >> 1, sgn = bs < 0 ? -1 : 1;
  // D = t(s0, r) - k on the low words (exact: |D| < 2^31)
  int D = (int)((unsigned)T0 + (unsigned)r * (unsigned)bs - ((unsigned)k << kFxBits));
  const float *row = buf + PAD * NI;
  f2x a01 = 0ull, a23 = 0ull;
  if constexpr (NI == 4) {
    a01 = f2_pack(acc[0], acc[1]);
    a23 = f2_pack(acc[2], acc[3]);
  }
  bpadj_line<NI, true, true>(r, D, half, abs_bs, sgn, row, acc, a01, a23);
  if (bl >= 0) {
#pragma unroll
    for (int l = 1; l < SB; ++l) {
      D += bl;
      bpadj_line<NI, false, true>(r, D, half, abs_bs, sgn, row + l * P * NI, acc, a01, a23);
    }
  } else {
#pragma unroll
    for (int l = 1; l < SB; ++l) {
      D += bl;
      bpadj_line<NI, false, false>(r, D, half, abs_bs, sgn, row + l * P * NI, acc, a01, a23);
    }
  }
  if constexpr (NI == 4) {
    acc[0] = f2_lo(a01);
    acc[1] = f2_hi(a01);
    acc[2] = f2_lo(a23);
    acc[3] = f2_hi(a23);
  }
}

// With XTRA (Joseph only), image bx of job JX, whose angle list is J's,
// rides along: staged after the group's band (geometry gx, same lines), it
// shares every crossing's position and weights and costs only its taps;
// its sums go to partx.  Bands are SB lines; a band past the last image
// line stages zero lines.
template <int OP, int NI, int SB, bool XTRA = false, int NB = kStageBatch>
__device__ __forceinline__ void partial_task(const Job &J, float *part, int b0, int band,
                                             int a_begin, int AB, int nbands, const BandGeom &g,
                                             const AngleConst *ang, int *status, float *buf,
                                             AngleConst *sc, int *sai, int *spos, int *wsum,
                                             long long *s0c, float *s0f, const float *wlo,
                                             const float *whi, const Job *JX = nullptr,
                                             float *partx = nullptr, int bx = 0,
                                             const BandGeom *gx = nullptr) {
  constexpr int PAD = kPartPad(SB);
  const int tid = threadIdx.x;
  const int na = min(AB, J.m - a_begin);
  const int nd = g.n_det, N = g.N;
  const int s0 = band * SB, s1 = min(N, s0 + SB), nl = s1 - s0;
  if (na <= 0 || s0 >= N) return;  // uniform over the CTA
  const int *idx = job_idx(J, b0);
  partition_block(idx, J.m, g.n_angles, ang, a_begin, na, spos, wsum);
  if (tid < kMaxABP) {
    int ai = -1;
    if (tid < na) {
      ai = idx ? idx[spos[tid]] : spos[tid];
      if (ai < 0 || ai >= g.n_angles) {
        if (band == 0) atomicOr(status, 1);
        ai = -1;
      }
    }
    sai[tid] = ai;
    if (ai >= 0) {
      const AngleConst C = ang[ai];
      sc[tid] = C;
      // the band's first line: A's crossing constant G + s0 T, B^T's bin
      // coordinate t00 + s0 bline (exact) and its FP32 estimate
      s0c[tid] = OP == OP_JOSEPH ? C.G + (long long)s0 * C.T : C.t00 + (long long)s0 * C.bline;
      s0f[tid] = fmaf((float)s0, C.blinef, C.t00f);
    }
  }
  __syncthreads();
  const size_t xo = (size_t)b0 * N * N;
  const size_t plane = (size_t)nbands * J.m * nd;   // floats per image of sums
  const int Pm = g.Prow > g.Pcol ? g.Prow : g.Pcol;
  float *bufx = nullptr;
  if (XTRA) bufx = buf + (size_t)SB * Pm * NI;
  for (int mode = 1; mode >= 0; --mode) {
    bool any = false;
    for (int a = 0; a < na; ++a) any |= (sai[a] >= 0 && sc[a].mode == mode);
    // angles of the other mode still write their (zero) sums below
    const int P = mode ? g.Prow : g.Pcol;
    const int Px = XTRA ? (mode ? gx->Prow : gx->Pcol) : 0;
    if (any) {
      __syncthreads();  // the previous mode's band is no longer read
      const bool split = XTRA && ride_split(JX->in_bf16, N, s0, nl, gx->fast != 0);
      float4 rv[4];
      if (split) ride_load(JX->in, (size_t)bx * N * N, N, mode, s0, rv);
      if (NI == 4) stage4<PAD, NB>(J.in, xo, J.in_bf16, N, mode, s0, nl, buf, P);
      else stage1<PAD>(J.in, xo, J.in_bf16, N, mode, s0, nl, buf, P, g.fast != 0);
      if (split) ride_store<PAD>(N, mode, bufx, Px, rv);
      else if (XTRA)
        stage1<PAD>(JX->in, (size_t)bx * N * N, JX->in_bf16, N, mode, s0, nl, bufx, Px,
                    gx->fast != 0);
      // lines past the image (last band) read as zeros
      for (int e = tid; e < (SB - nl) * P * NI; e += kThreads) sts(buf + nl * P * NI + e, 0.0f);
      if (XTRA)
        for (int e = tid; e < (SB - nl) * Px; e += kThreads) sts(bufx + nl * Px + e, 0.0f);
      __syncthreads();
    }
    for (int a = 0; a < na; ++a) {
      const bool live = sai[a] >= 0;
      if (live ? sc[a].mode != mode : mode != 0) continue;   // dead angles: written once
      float *pa = part + ((size_t)b0 * nbands + band) * J.m * nd + (size_t)spos[a] * nd;
      float *pax = XTRA ? partx + ((size_t)bx * nbands + band) * JX->m * nd + (size_t)spos[a] * nd
                        : nullptr;
      for (int k = tid; k < nd; k += kThreads) {
        float acc[NI], ax = 0.0f;
#pragma unroll
        for (int i = 0; i < NI; ++i) acc[i] = 0.0f;
        if (live) {
          if (OP == OP_JOSEPH)
            joseph_band<SB, NI, XTRA>(sc[a], s0c[a], k, N, buf, P, acc, bufx, Px, ax);
          else
            bpadj_band<SB, NI>(sc[a], s0c[a], s0f[a], k, N, buf, P, acc);
        }
#pragma unroll
        for (int i = 0; i < NI; ++i)
          if (!SKEI_CHECK || ck_range(pa + i * plane + k, 4, wlo, whi, CK_BAND_SUMS))
            pa[i * plane + k] = acc[i];
        if (XTRA && (!SKEI_CHECK || ck_range(pax + k, 4, wlo, whi, CK_BAND_SUMS))) pax[k] = ax;
      }
    }
  }
}

// Image groups of size 4 per job (none when the launch works on single
// images); the job's remaining images form single-image groups.
__device__ __forceinline__ int quads(int nimg, int gmax) { return gmax == 4 ? nimg >> 2 : 0; }

// One CTA: band blockIdx.x (SB lines), angle block blockIdx.y, image group
// blockIdx.z among the launch's groups of NI images (job 0's, then job 1's).
template <int OP, int NI, int MINB, int SB>
__global__ void __launch_bounds__(kThreads, MINB) band_partial_kernel(const PartArgs args) {
  constexpr int kNB = kStageBatch;   // staging blocks in flight per thread
  pdl_enter();
  extern __shared__ float4 smem4[];
  __shared__ AngleConst sc[kMaxABP];
  __shared__ long long s0c[kMaxABP];
  __shared__ float s0f[kMaxABP];
  __shared__ int sai[kMaxABP], spos[kMaxABP], wsum[kWarps];
  const int z = blockIdx.z;
  const Job &J0 = args.jobs.j[0];
  if constexpr (OP == OP_JOSEPH && NI == 4) {
    if (args.merge) {
      // group z of job 1 (images 4z .. 4z+3) with image z of job 0
      partial_task<OP, 4, SB, true, kNB>(args.jobs.j[1], args.part + args.off[1], 4 * z, blockIdx.x,
                                    blockIdx.y * args.AB, args.AB, args.nbands, args.g4,
                                    args.ang, args.status, reinterpret_cast<float *>(smem4), sc,
                                    sai, spos, wsum, s0c, s0f, args.part,
                                    args.part + args.work_floats, &J0, args.part + args.off[0], z,
                                    &args.g1);
      return;
    }
  }
  const int q0 = quads(J0.nimg, args.gmax[0]);
  const int c0 = NI == 4 ? q0 : J0.nimg - 4 * q0;
  const int jn = (args.jobs.njobs > 1 && z >= c0) ? 1 : 0;
  const Job &J = args.jobs.j[jn];
  const int zz = z - (jn ? c0 : 0);
  const int b0 = NI == 4 ? 4 * zz : 4 * quads(J.nimg, args.gmax[jn]) + zz;
  partial_task<OP, NI, SB, false, kNB>(J, args.part + args.off[jn], b0, blockIdx.x, blockIdx.y * args.AB,
                           args.AB, args.nbands, NI == 4 ? args.g4 : args.g1, args.ang,
                           args.status, reinterpret_cast<float *>(smem4), sc, sai, spos, wsum,
                           s0c, s0f, args.part, args.part + args.work_floats);
}

// out[b][a][k] = epilogue(sum over bands, in order, of the band sums).
template <int OP>
__global__ void __launch_bounds__(256)
    band_reduce_kernel(const Jobs jobs, const AngleConst *ang, int n_angles, int nd, int nbands,
                       const float *part, size_t off0, size_t off1, size_t work_floats) {
  pdl_enter();
  const int y = blockIdx.y;
  const int jn = (jobs.njobs > 1 && y >= jobs.j[0].nimg) ? 1 : 0;
  const Job &J = jobs.j[jn];
  const int b = y - (jn ? jobs.j[0].nimg : 0);
  const int n = J.m * nd;
  const float *pb = part + (jn ? off1 : off0) + (size_t)b * nbands * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    // the bands in order, 16 loads in flight at a time
    float s = 0.0f;
    int q = 0;
    for (; q + 16 <= nbands; q += 16) {
      float v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = __ldg(pb + (size_t)(q + u) * n + e);
#pragma unroll
      for (int u = 0; u < 16; ++u) s += v[u];
    }
    for (; q < nbands; ++q) s += __ldg(pb + (size_t)q * n + e);
    if (SKEI_CHECK) {
      // the first and last band this output read, and the output
      ck_range(pb + e, 4, part, part + work_floats, CK_BAND_SUMS);
      ck_range(pb + (size_t)(nbands - 1) * n + e, 4, part, part + work_floats, CK_BAND_SUMS);
      if (!ck((long long)b * n + e, (long long)J.nimg * n, CK_BAND_OUT)) continue;
    }
    const int a = e / nd, k = e - a * nd;
    const int *idx = job_idx(J, b);
    int ai = idx ? idx[a] : a;
    float v;
    if (ai < 0 || ai >= n_angles) {
      v = 0.0f;
    } else if (OP == OP_JOSEPH) {
      v = s * ang[ai].W;
      if (J.aux) v = ld_any(J.aux, ((size_t)b * n_angles + ai) * nd + k, J.aux_bf16) - v;
      v *= J.alpha;
    } else {
      v = s * J.alpha;
    }
    st_any(J.out, (size_t)b * n + e, v, J.out_bf16);
  }
}

int part_layout(skei_plan p, const Jobs &jobs, int *nbands1, int *nbands4, size_t off[kMaxJobs],
                size_t *floats, int gm) {
  const int sb1 = part_geom(p->N, p->n_det, p->n_angles, 1).SB;
  const int sb4 = part_geom(p->N, p->n_det, p->n_angles, 4).SB;
  *nbands1 = (p->N + sb1 - 1) / sb1;
  *nbands4 = (p->N + sb4 - 1) / sb4;
  // one band count per launch: the finer of the two if both group sizes occur
  size_t total = 0;
  for (int q = 0; q < jobs.njobs; ++q) {
    off[q] = total;
    total += (size_t)jobs.j[q].nimg * std::max(*nbands1, gm == 4 ? *nbands4 : *nbands1) *
             jobs.j[q].m * p->n_det;
  }
  *floats = total;
  return SKEI_OK;
}

template <int OP, int NI, int MINB, int SB>
int set_partial_smem(size_t smem) {
  if (smem > 227 * 1024)
    return set_error(SKEI_EINVAL, "band of %zu bytes needs too much shared memory", smem);
  static size_t configured[64] = {0};
  return opt_in_smem(band_partial_kernel<OP, NI, MINB, SB>, smem, configured,
                     "band partial kernel: shared memory attribute");
}

}  // namespace

// Joseph over two jobs on the same angle lists, 4 images of job 1 per image
// of job 0 (the MC and EI terms of a step, G = 4): job 0's image z rides
// with job 1's group z; with a list per sample, image z and images
// 4z .. 4z+3 must read the same row.
bool band_sums_merge(const Jobs &jobs) {
  const Job &j0 = jobs.j[0], &j1 = jobs.j[1];
  return SKEI_PART_MERGE && SKEI_PART_GROUP == 4 && jobs.njobs == 2 && job_groupable(j1) &&
         j0.idx == j1.idx && j0.m == j1.m && j1.nimg == 4 * j0.nimg &&
         ((j0.idx_per <= 0 && j1.idx_per <= 0) ||
          (j0.idx_per > 0 && j1.idx_per == 4 * j0.idx_per));
}

namespace {

template <int OP>
int launch_band_partial(skei_plan p, const Jobs &jobs, float *work, size_t work_floats,
                        cudaStream_t st, const FilterReq *fr) {
  // groups of 4 per job, where its images' angle lists allow them; the
  // workspace layout is the one band_partial_floats sizes
  int gmj[kMaxJobs] = {1, 1};
  for (int q = 0; q < jobs.njobs; ++q)
    gmj[q] = SKEI_PART_GROUP == 4 && job_groupable(jobs.j[q]) ? 4 : 1;
  int nb1 = 0, nb4 = 0;
  size_t off[kMaxJobs] = {0, 0}, need = 0;
  part_layout(p, jobs, &nb1, &nb4, off, &need, SKEI_PART_GROUP);
  if (need > work_floats)
    return set_error(SKEI_EINVAL, "band sums need %zu floats of workspace, %zu given", need,
                     work_floats);
  // both group sizes stage bands of their own height; a launch uses one
  // band count, so single images follow the 4-image band height when both
  // occur
  BandGeom g1 = part_geom(p->N, p->n_det, p->n_angles, 1);
  const BandGeom g4 = part_geom(p->N, p->n_det, p->n_angles, 4);
  int nbands = nb1;
  bool any4 = false;
  for (int q = 0; q < jobs.njobs; ++q) any4 |= gmj[q] == 4 && jobs.j[q].nimg >= 4;
  if (any4) {
    g1 = part_geom(p->N, p->n_det, p->n_angles, 1, g4.SB);
    nbands = nb4;
  }
  int m_max = 0, ngroups = 0, n4 = 0, n1 = 0;
  for (int q = 0; q < jobs.njobs; ++q) {
    m_max = max(m_max, jobs.j[q].m);
    ngroups += n_groups(jobs.j[q].nimg, gmj[q]);
    const int q4 = gmj[q] == 4 ? jobs.j[q].nimg >> 2 : 0;
    n4 += q4;
    n1 += jobs.j[q].nimg - 4 * q4;
  }
  const int merge = OP == OP_JOSEPH && band_sums_merge(jobs);
  if (merge) {
    ngroups = n4 = jobs.j[0].nimg;
    n1 = 0;
  }
  if (ngroups > 65535) return set_error(SKEI_EINVAL, "too many images in one launch");
  // angles per CTA (measured on GB300: a CTA costs about one angle of
  // staging plus its angles; a short second wave or a lone CTA per SM costs
  // more than larger blocks): the smallest block whose CTAs fit one wave of
  // SKEI_PART_CTAS (2) per SM with the 128-register kernel; where none does
  // (many bands or images), about 3 CTAs per SM with the 80-register one
  const long long units = (long long)nbands * ngroups;
  const int ab_cap = std::min(m_max, kMaxABP);
  const long long slots = (long long)sm_count() * SKEI_PART_CTAS;
  int AB = 0;
  for (int ab = 1; ab <= ab_cap && !AB; ++ab)
    if (units * ((m_max + ab - 1) / ab) <= slots) AB = ab;
  const bool one_wave = AB > 0;
  if (!one_wave) {
    long long blocks = (3LL * sm_count() + units - 1) / units;
    blocks = std::max(1LL, std::min(blocks, (long long)m_max));
    AB = (int)((m_max + blocks - 1) / blocks);
  }
  if (SKEI_PART_AB > 0) AB = SKEI_PART_AB;
  AB = std::max(1, std::min(AB, kMaxABP));
  const int nblk = (m_max + AB - 1) / AB;
  AB = (m_max + nblk - 1) / nblk;   // balanced blocks
  PartArgs a{jobs, p->d_ang, p->d_status, g1, g4, {gmj[0], gmj[1]}, AB, nbands, work,
             {off[0], off[1]}, merge, work_floats};
  const size_t smem4 = part_smem(g4) + (merge ? part_smem(g1) : 0);
  constexpr int sb4 = SKEI_PART_SBL4, sb1 = SKEI_PART_SBL1;
  if (n4 > 0 && one_wave) {
    constexpr int m4 = SKEI_PART_MINB4;
    SKEI_TRY((set_partial_smem<OP, 4, m4, sb4>(smem4)));
    launch_k(band_partial_kernel<OP, 4, m4, sb4>, dim3(nbands, nblk, n4), dim3(kThreads), smem4,
             st, a);
  } else if (n4 > 0) {
    SKEI_TRY((set_partial_smem<OP, 4, 3, sb4>(smem4)));
    launch_k(band_partial_kernel<OP, 4, 3, sb4>, dim3(nbands, nblk, n4), dim3(kThreads), smem4,
             st, a);
  }
  if (n1 > 0) {
    // single images take the 4-image band height when both occur
    constexpr int m1 = SKEI_PART_MINB1;
    if (g1.SB == sb4) {
      SKEI_TRY((set_partial_smem<OP, 1, m1, sb4>(part_smem(g1))));
      launch_k(band_partial_kernel<OP, 1, m1, sb4>, dim3(nbands, nblk, n1), dim3(kThreads),
               part_smem(g1), st, a);
    } else {
      SKEI_TRY((set_partial_smem<OP, 1, m1, sb1>(part_smem(g1))));
      launch_k(band_partial_kernel<OP, 1, m1, sb1>, dim3(nbands, nblk, n1), dim3(kThreads),
               part_smem(g1), st, a);
    }
  }
  SKEI_TRY(check_launch("band partial sums launch"));
  if (fr)
    return launch_band_sum_filter(p, OP, jobs, nbands, nbands, work, off[0], off[1], work_floats,
                                  *fr, st);
  int nimg = 0;
  for (int q = 0; q < jobs.njobs; ++q) nimg += jobs.j[q].nimg;
  const int n_max = m_max * p->n_det;
  const int gx = std::max(1, std::min((n_max + 255) / 256, 4 * sm_count() / std::max(nimg, 1) + 1));
  launch_k(band_reduce_kernel<OP>, dim3(gx, nimg), dim3(256), 0, st, jobs,
           (const AngleConst *)p->d_ang, p->n_angles, p->n_det, nbands, (const float *)work,
           off[0], off[1], work_floats);
  return check_launch("band sums reduction launch");
}

}  // namespace

SKEI_CHECK_READER(check_read_band)

int launch_band_jobs(skei_plan p, int op, const Jobs &jobs, cudaStream_t st) {
  if (op == OP_JOSEPH) return launch_band<OP_JOSEPH>(p, jobs, st);
  if (op == OP_BP_ADJ) return launch_band<OP_BP_ADJ>(p, jobs, st);
  return set_error(SKEI_EINVAL, "band launch: unknown operator %d", op);
}

size_t band_partial_floats(skei_plan p, const Jobs &jobs) {
  int nb1 = 0, nb4 = 0;
  size_t off[kMaxJobs] = {0, 0}, need = 0;
  part_layout(p, jobs, &nb1, &nb4, off, &need, SKEI_PART_GROUP);
  return need;
}

int launch_band_partial_jobs(skei_plan p, int op, const Jobs &jobs, float *work,
                             size_t work_floats, cudaStream_t st, const FilterReq *fr) {
  if (op == OP_JOSEPH) return launch_band_partial<OP_JOSEPH>(p, jobs, work, work_floats, st, fr);
  if (op == OP_BP_ADJ) return launch_band_partial<OP_BP_ADJ>(p, jobs, work, work_floats, st, fr);
  return set_error(SKEI_EINVAL, "band partial launch: unknown operator %d", op);
}

size_t band_batch_smem(int op, int N, int n_det, int n_angles, int AB, int NI) {
  return band_smem(band_geom(N, n_det, n_angles, op, AB, NI));
}

int band_batch_occupancy(int op, size_t smem, int *clusters) {
  if (op == OP_JOSEPH) return band_batch_clusters<OP_JOSEPH>(smem, clusters);
  if (op == OP_BP_ADJ) return band_batch_clusters<OP_BP_ADJ>(smem, clusters);
  return set_error(SKEI_EINVAL, "band batch: unknown operator %d", op);
}

int launch_band_batch_op(int op, const BatchItem *items, const int4 *tasks, int n_tasks, int AB,
                         size_t smem, int clusters, int *queue, cudaStream_t st) {
  if (op == OP_JOSEPH)
    return launch_band_batch<OP_JOSEPH>(items, tasks, n_tasks, AB, smem, clusters, queue, st);
  if (op == OP_BP_ADJ)
    return launch_band_batch<OP_BP_ADJ>(items, tasks, n_tasks, AB, smem, clusters, queue, st);
  return set_error(SKEI_EINVAL, "band batch: unknown operator %d", op);
}

}  // namespace skei
