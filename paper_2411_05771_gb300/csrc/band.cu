// Ray-driven operators over image bands: Joseph's forward projector A
// (Sec. 4.1.1: the discrete Radon transform; Eq. (e:skeiloss): A_S = S A)
// and the transpose B_S^T of pixel-driven back-projection (needed to
// differentiate through A_S^dagger = (pi/m) B_S H, Algorithm 2's update).
//
// Both sum, for every detector bin (a, k), contributions from every image
// "line" (a row when |cos| >= |sin|, a column otherwise).  A cluster of 8
// CTAs covers one image and a block of AB angles; CTA r stages lines
// [r R, (r+1) R) (R = ceil(N/8)) in shared memory - rows as they are,
// columns transposed - sub-band by sub-band, accumulates per-bin partial
// sums in its own shared memory, and after a cluster barrier reduces 1/8 of
// the bins over the 8 CTAs' partials through distributed shared memory.  The
// reduction order is fixed, so results are deterministic; there are no
// atomics and no global scratch.
#include <cooperative_groups.h>

#include <cmath>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace skei {
namespace {

constexpr int kBands = 8;    // cluster size = number of line bands
constexpr int kPad = 2;      // zero columns on each side of a staged line
constexpr int kMaxAB = 8;    // angles per cluster
constexpr int kThreads = 256;

enum { OP_JOSEPH = 0, OP_BP_ADJ = 1 };

struct BandGeom {
  int N, n_det, n_angles;
  int R;   // lines per band
  int SB;  // lines per staged sub-band
  int P;   // pitch of a staged line (odd, >= N + 2 kPad)
  int AB;  // angles per cluster
};

template <typename Tin, typename Tout>
struct BandArgs {
  const Tin *x;        // [B][N][N]
  const Tout *y;       // OP_JOSEPH residual source [B][n_angles][n_det] or null
  Tout *out;           // [B][m][n_det]
  const int *idx;      // [m] or null
  int m;
  const AngleConst *ang;
  int *status;
  float alpha;         // OP_BP_ADJ output scale
  BandGeom g;
};

// Line range [lo, hi) within [s0, s1) on which lam0 + L * lam1 lies in
// (lo_bound, hi_bound).
__device__ __forceinline__ void line_range(float lam0, float lam1, float lo_bound,
                                           float hi_bound, int s0, int s1, int *lo,
                                           int *hi) {
  if (fabsf(lam1) < 1e-20f) {
    bool in = lam0 > lo_bound && lam0 < hi_bound;
    *lo = s0;
    *hi = in ? s1 : s0;
    return;
  }
  float inv = 1.0f / lam1;
  float la = (lo_bound - lam0) * inv, lb = (hi_bound - lam0) * inv;
  float lmin = fmaxf(fminf(la, lb), (float)s0);
  float lmax = fminf(fmaxf(la, lb), (float)(s1 - 1));
  *lo = (int)ceilf(lmin);
  *hi = (int)floorf(lmax) + 1;
}

// Joseph: sum over lines [s0,s1) of the linear interpolation at the
// fixed-point crossing pos(L, k) = G + k A + L T on the staged band.
__device__ __forceinline__ float joseph_partial(const AngleConst &C, int k, int s0,
                                                int s1, int N, const float *buf,
                                                int P) {
  int lo, hi;
  // taps are nonzero only for pos in (-1, N); the relaxed window keeps every
  // such line and never reads beyond the kPad zero columns
  line_range(fmaf((float)k, C.Af, C.Gf), C.Tf, -1.5f, (float)N + 0.5f, s0, s1, &lo, &hi);
  float acc = 0.0f;
  if (lo < hi) {
    const long long T = C.T;
    long long pos = C.G + (long long)k * C.A + (long long)lo * T;
    const float *row = buf + (lo - s0) * P + kPad;
#pragma unroll 4
    for (int l = lo; l < hi; ++l) {
      const int j0 = ipart(pos);
      const float f = frac23(pos);
      const float v0 = row[j0], v1 = row[j0 + 1];
      acc += fmaf(f, v1 - v0, v0);
      row += P;
      pos += T;
    }
  }
  return acc;
}

// B^T: for bin k, sum over lines of the pixels whose bin coordinate
// t(L, P) = t00 + L bline + P bstep lies in (k-1, k+1), weighted exactly as
// the back-projector weights them.  At most 3 pixels per line
// (|bstep| >= 1/sqrt 2), found around P = (k - t(L, 0)) / bstep.
__device__ __forceinline__ float bpadj_partial(const AngleConst &C, int k, int s0,
                                               int s1, int N, const float *buf,
                                               int P) {
  const float kf = (float)k;
  const float inv = C.inv_bstep;
  int lo, hi;
  // the candidate centre must come within sqrt(2) of [0, N-1]; relaxed window
  line_range((kf - C.t00f) * inv, -C.blinef * inv, -2.5f, (float)N + 1.5f, s0, s1, &lo, &hi);
  float acc = 0.0f;
  if (lo < hi) {
    const long long bstep = C.bstep, bline = C.bline;
    long long tl = C.t00 + (long long)lo * bline;
    float tlf = fmaf((float)lo, C.blinef, C.t00f);
    const float *row = buf + (lo - s0) * P + kPad;
    for (int l = lo; l < hi; ++l) {
      int r = round_int((kf - tlf) * inv);
      r = min(max(r, -1), N);
      long long t = tl + (long long)(r - 1) * bstep;
      const float *q = row + r;
      acc = fmaf(tap_weight(t, k), q[-1], acc);
      t += bstep;
      acc = fmaf(tap_weight(t, k), q[0], acc);
      t += bstep;
      acc = fmaf(tap_weight(t, k), q[1], acc);
      row += P;
      tl += bline;
      tlf += C.blinef;
    }
  }
  return acc;
}

template <int OP, typename Tin, typename Tout>
__global__ void __cluster_dims__(kBands, 1, 1) __launch_bounds__(kThreads)
    band_kernel(const BandArgs<Tin, Tout> args) {
  extern __shared__ float4 smem4[];
  float *smem = reinterpret_cast<float *>(smem4);
  __shared__ AngleConst sc[kMaxAB];
  __shared__ int sai[kMaxAB];

  cg::cluster_group cluster = cg::this_cluster();
  const BandGeom g = args.g;
  const int tid = threadIdx.x;
  const int band = (int)cluster.block_rank();
  const int b = blockIdx.z;
  const int a_begin = blockIdx.y * g.AB;
  const int na = min(g.AB, args.m - a_begin);
  const int nd = g.n_det, N = g.N, P = g.P;
  float *part = smem;                 // [AB][n_det]
  float *buf = smem + g.AB * nd;      // [SB][P]

  if (tid < kMaxAB) {
    int ai = -1;
    if (tid < na) {
      ai = args.idx ? args.idx[a_begin + tid] : a_begin + tid;
      if (ai < 0 || ai >= g.n_angles) {
        if (band == 0) atomicOr(args.status, 1);
        ai = -1;
      }
    }
    sai[tid] = ai;
    if (ai >= 0) sc[tid] = args.ang[ai];
  }
  for (int e = tid; e < na * nd; e += kThreads) part[e] = 0.0f;
  __syncthreads();

  const Tin *xb = args.x + (size_t)b * N * N;
  const int L0 = band * g.R, L1 = min(N, L0 + g.R);
  for (int mode = 1; mode >= 0; --mode) {
    bool any = false;
    for (int a = 0; a < na; ++a) any |= (sai[a] >= 0 && sc[a].mode == mode);
    if (!any) continue;
    for (int s0 = L0; s0 < L1; s0 += g.SB) {
      const int s1 = min(L1, s0 + g.SB), nl = s1 - s0;
      __syncthreads();  // the previous sub-band is no longer read
      if (mode == 1) {
        for (int e = tid; e < nl * N; e += kThreads) {
          const int l = e / N, p = e - l * N;
          buf[l * P + kPad + p] = ldg_f(xb + (size_t)(s0 + l) * N + p);
        }
      } else {
        for (int e = tid; e < nl * N; e += kThreads) {
          const int p = e / nl, l = e - p * nl;
          buf[l * P + kPad + p] = ldg_f(xb + (size_t)p * N + s0 + l);
        }
      }
      const int npad = P - N;
      for (int e = tid; e < nl * npad; e += kThreads) {
        const int l = e / npad, q = e - l * npad;
        buf[l * P + (q < kPad ? q : N + q)] = 0.0f;
      }
      __syncthreads();
      for (int it = tid; it < na * nd; it += kThreads) {
        const int a = it / nd, k = it - a * nd;
        if (sai[a] < 0 || sc[a].mode != mode) continue;
        const float v = OP == OP_JOSEPH ? joseph_partial(sc[a], k, s0, s1, N, buf, P)
                                        : bpadj_partial(sc[a], k, s0, s1, N, buf, P);
        part[it] += v;
      }
    }
  }

  cluster.sync();
  const int n_items = na * nd;
  for (int it = band * kThreads + tid; it < n_items; it += kBands * kThreads) {
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < kBands; ++q) s += cluster.map_shared_rank(part, q)[it];
    const int a = it / nd, k = it - a * nd;
    const int ai = sai[a];
    Tout *o = args.out + ((size_t)b * args.m + a_begin + a) * nd + k;
    float v;
    if (ai < 0) {
      v = 0.0f;
    } else if (OP == OP_JOSEPH) {
      v = s * sc[a].W;
      if (args.y) v = ldg_f(args.y + ((size_t)b * g.n_angles + ai) * nd + k) - v;
    } else {
      v = s * args.alpha;
    }
    st_f(o, v);
  }
  cluster.sync();  // keep this CTA's partials alive until every peer has read them
}

int sm_count() {
  static int count[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!count[dev]) {
    int c = 0;
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    count[dev] = c > 0 ? c : 1;
  }
  return count[dev];
}

template <int OP, typename Tin, typename Tout>
int launch_band(skei_plan p, const Tin *x, int B, const int *idx, int m,
                const Tout *y, float alpha, Tout *out, cudaStream_t st) {
  BandGeom g;
  g.N = p->N;
  g.n_det = p->n_det;
  g.n_angles = p->n_angles;
  g.R = (g.N + kBands - 1) / kBands;
  g.P = g.N + 2 * kPad;
  if (g.P % 2 == 0) g.P += 1;  // odd pitch: transposed staging writes hit distinct banks
  g.SB = min(g.R, 32);
  while (g.SB > 1 && (size_t)g.SB * g.P * 4 > 96 * 1024) --g.SB;

  // angles per cluster: fewest waves x angles per CTA (the per-CTA time),
  // ties to the larger block (less staging)
  int ab_max = min(kMaxAB, m);
  while (ab_max > 1 && (size_t)ab_max * g.n_det * 4 > 48 * 1024) --ab_max;
  const size_t band_bytes = (size_t)g.SB * g.P * 4;
  int best_ab = 1;
  double best_cost = 1e300;
  for (int ab = 1; ab <= ab_max; ++ab) {
    const size_t bytes = band_bytes + (size_t)ab * g.n_det * 4;
    int per_sm = (int)((227 * 1024) / (bytes + 1024));
    per_sm = max(1, min(per_sm, 8));
    const double slots = (double)sm_count() * per_sm;
    const double ctas = (double)kBands * ((m + ab - 1) / ab) * B;
    const double cost = std::ceil(ctas / slots) * ab;
    if (cost <= best_cost) { best_cost = cost; best_ab = ab; }
  }
  g.AB = best_ab;
  const size_t smem = band_bytes + (size_t)g.AB * g.n_det * 4;

  auto kern = band_kernel<OP, Tin, Tout>;
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "band kernel: shared memory attribute");
    configured = smem;
  }
  BandArgs<Tin, Tout> a{x, y, out, idx, m, p->d_ang, p->d_status, alpha, g};
  dim3 grid(kBands, (m + g.AB - 1) / g.AB, B);
  kern<<<grid, kThreads, smem, st>>>(a);
  return check_launch(OP == OP_JOSEPH ? "joseph forward launch" : "back-projection transpose launch");
}

}  // namespace

template <typename Tin, typename Tout>
int launch_proj_fwd(skei_plan p, const Tin *x, int B, const int *idx, int m,
                    const Tout *y, Tout *out, cudaStream_t st) {
  return launch_band<OP_JOSEPH, Tin, Tout>(p, x, B, idx, m, y, 1.0f, out, st);
}

template <typename Tin, typename Tout>
int launch_backproject_adj(skei_plan p, const Tin *x, int B, const int *idx, int m,
                           float alpha, Tout *q, cudaStream_t st) {
  return launch_band<OP_BP_ADJ, Tin, Tout>(p, x, B, idx, m, nullptr, alpha, q, st);
}

#define SKEI_BAND_INST(TI, TO)                                                              \
  template int launch_proj_fwd<TI, TO>(skei_plan, const TI *, int, const int *, int,        \
                                       const TO *, TO *, cudaStream_t);                     \
  template int launch_backproject_adj<TI, TO>(skei_plan, const TI *, int, const int *, int, \
                                              float, TO *, cudaStream_t);
SKEI_BAND_INST(float, float)
SKEI_BAND_INST(__nv_bfloat16, __nv_bfloat16)
SKEI_BAND_INST(__nv_bfloat16, float)
#undef SKEI_BAND_INST

}  // namespace skei
