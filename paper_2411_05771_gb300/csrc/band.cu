// Operators that sum over image "lines" (rows when |cos| >= |sin|, columns
// otherwise) for every detector bin: Joseph's forward projector A
// (Sec. 4.1.1, the discrete Radon transform; Eq. (e:skeiloss): A_S = S A)
// and the transpose B_S^T of pixel-driven back-projection (needed to
// differentiate through A_S^dagger = (pi/m) B_S H, Algorithm 2's update).
//
// A cluster of 8 CTAs covers one image and a block of AB angles; CTA r
// stages lines [r R, (r+1) R) (R = ceil(N/8)) in shared memory - rows as
// they are, columns transposed - sub-band by sub-band, and accumulates
// per-bin partial sums in its own shared memory.  After a cluster barrier
// each CTA reduces 1/8 of the bins over the 8 CTAs' partials through
// distributed shared memory, in a fixed order: deterministic, no atomics, no
// global scratch.
//
//   A:    one thread per ray gathers the linear interpolation on each line.
//   B^T:  one thread per bin gathers, on each line, the (at most 3) pixels
//         whose bin coordinate lies within one bin of it, with exactly the
//         back-projector's weights.
//
// Up to two jobs share a launch (grid.z spans the images of both), e.g. the
// MC projection of x1 and the EI projection of x2 of one SkEI step.
#include <cooperative_groups.h>

#include <cmath>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace skei {
namespace {

constexpr int kBands = 8;    // cluster size = number of line bands
constexpr int kPad = 4;      // zero columns on each side of a staged line
constexpr int kMaxAB = 8;    // angles per cluster
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct BandGeom {
  int N, n_det, n_angles;
  int R;       // lines per band
  int SB;      // lines per staged sub-band
  int Prow;    // pitch of staged rows (multiple of 4: 16-byte aligned rows)
  int Pcol;    // pitch of staged columns (conflict-free transposed writes)
  int AB;      // angles per cluster
  int C;       // OP_BP_ADJ: warps (partial rows) per angle = kWarps / AB
  int fast;    // N % 8 == 0: vectorised staging
};

struct BandArgs {
  Jobs jobs;
  const AngleConst *ang;
  int *status;
  BandGeom g;
};

// Staging geometry of one image size and operator with AB angles per task.
__host__ __device__ __forceinline__ BandGeom band_geom(int N, int n_det, int n_angles, int op,
                                                       int AB) {
  BandGeom g;
  g.N = N;
  g.n_det = n_det;
  g.n_angles = n_angles;
  g.R = (N + kBands - 1) / kBands;
  g.Prow = (N + 2 * kPad + 3) & ~3;
  // A: 32 staged lines (fewer per-ray range setups); B^T: 16 (its per-bin
  // work per line is larger, and the smaller band leaves room for more CTAs)
  const int sb = op == OP_JOSEPH ? 32 : 16;
  g.SB = g.R < sb ? g.R : sb;
  // transposed staging writes lines 4q..4q+3 of (32 / (SB/4)) positions per
  // warp: a pitch = 2 mod 8 (16 lines) or odd (32 lines) keeps them in
  // distinct banks
  g.Pcol = g.SB == 32 ? ((N + 2 * kPad) | 1) : ((N + 2 * kPad - 2 + 7) & ~7) + 2;
  g.fast = (N % 8 == 0) ? 1 : 0;
  const int Pmax = g.Prow > g.Pcol ? g.Prow : g.Pcol;
  while (g.SB > 1 && g.SB * Pmax * 4 > 96 * 1024) --g.SB;  // large N: slow staging
  g.AB = AB;
  g.C = 1;
  return g;
}

// Dynamic shared memory of a band task: AB rows of partial bins, then the
// staged sub-band.
inline size_t band_smem(const BandGeom &g) {
  const int Pmax = g.Prow > g.Pcol ? g.Prow : g.Pcol;
  return (size_t)g.SB * Pmax * 4 + (size_t)((g.AB * g.n_det + 3) & ~3) * 4;
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

// Stages lines [s0, s0 + nl) of image xb (element offset xo in x) into buf
// (pitch P): mode 1 copies rows, mode 0 copies columns transposed.  kPad
// zero columns on each side.
__device__ __forceinline__ void stage(const void *x, size_t xo, int bf16, int N, int mode,
                                      int s0, int nl, float *buf, int P, bool fast) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (mode == 1) {
    if (fast) {
      for (int r = warp; r < nl; r += kWarps) {
        const size_t src = xo + (size_t)(s0 + r) * N;
        float *dst = buf + r * P + kPad;
        for (int c = 4 * lane; c < N; c += 128)
          *reinterpret_cast<float4 *>(dst + c) = load4(x, src + c, bf16);
      }
    } else {
      for (int r = warp; r < nl; r += kWarps) {
        const size_t src = xo + (size_t)(s0 + r) * N;
        float *dst = buf + r * P + kPad;
        for (int c = lane; c < N; c += 32) dst[c] = ld_any(x, src + c, bf16);
      }
    }
  } else {
    if (fast && (nl == 16 || nl == 32) && (s0 & 3) == 0) {
      // lane = (nl/4) * (position within a group) + quarter of the lines; 4
      // consecutive lines of a column start 16-byte aligned (N % 8 == 0)
      const int qn = nl >> 2, qs = nl == 16 ? 2 : 3;
      const int q = lane & (qn - 1);
      const int per_warp = 32 / qn;
      for (int p = warp * per_warp + (lane >> qs); p < N; p += kWarps * per_warp) {
        const float4 v = load4(x, xo + (size_t)p * N + s0 + 4 * q, bf16);
        float *dst = buf + (4 * q) * P + kPad + p;
        dst[0] = v.x;
        dst[P] = v.y;
        dst[2 * P] = v.z;
        dst[3 * P] = v.w;
      }
    } else {
      for (int p = warp; p < N; p += kWarps)
        for (int l = lane; l < nl; l += 32)
          buf[l * P + kPad + p] = ld_any(x, xo + (size_t)p * N + s0 + l, bf16);
    }
  }
  const int npad = P - N;
  for (int r = warp; r < nl; r += kWarps)
    for (int c = lane; c < npad; c += 32) buf[r * P + (c < kPad ? c : N + c)] = 0.0f;
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

// Joseph: sum over lines [s0,s1) of the linear interpolation at the
// fixed-point crossing pos(L, k) = G + k A + L T on the staged band.
__device__ __forceinline__ float joseph_partial(const AngleConst &C, int k, int s0, int s1,
                                                int N, const float *buf, int P) {
  int lo, hi;
  // taps are nonzero only for pos in (-1, N); the relaxed window keeps every
  // such line and never reads beyond the kPad zero columns
  line_range(fmaf((float)k, C.Af, C.Gf), C.Tf, C.invT, -1.5f, (float)N + 0.5f, s0, s1, &lo, &hi);
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

// B^T for bin k: the pixels of lines [s0, s1) whose bin coordinate
// t(L, P) = t00 + L bline + P bstep lies in (k-1, k+1), weighted exactly as
// the back-projector weights them.  At most 3 pixels per line
// (|bstep| >= 1/sqrt 2): the nearest one, r, and its two neighbours.  r and
// its exact offset D = t(L, r) - k (32-bit fixed point, |D| <= |bstep|/2)
// are carried from line to line: D grows by bline (|bline| <= |bstep|), and
// one step of r re-centres it.
__device__ __forceinline__ float bpadj_partial(const AngleConst &C, int k, int s0, int s1,
                                               int N, const float *buf, int P) {
  const float kf = (float)k;
  const float inv = C.inv_bstep;
  int lo, hi;
  // the nearest pixel must come within sqrt(2) of [0, N-1]; relaxed window,
  // so that r stays in [-3, N+2] and its neighbours in the kPad zero columns
  line_range((kf - C.t00f) * inv, -C.blinef * inv, -C.bstepf * C.inv_bline, -2.5f,
             (float)N + 1.5f, s0, s1, &lo, &hi);
  float acc = 0.0f;
  if (lo < hi) {
    const int bs = (int)(unsigned)C.bstep, bl = (int)(unsigned)C.bline;
    const int abs_bs = abs(bs), half = abs_bs >> 1, sgn = bs < 0 ? -1 : 1;
    int r = round_int((kf - fmaf((float)lo, C.blinef, C.t00f)) * inv);
    // D = t(lo, r) - k on the low words (exact: |D| < 2^31)
    int D = (int)((unsigned)(C.t00 + (long long)lo * C.bline) + (unsigned)r * (unsigned)bs -
                  ((unsigned)k << kFxBits));
    const float *row = buf + (lo - s0) * P + kPad;
    for (int l = lo; l < hi; ++l) {
      if (D > half) { r -= sgn; D -= abs_bs; }
      else if (D < -half) { r += sgn; D += abs_bs; }
      const float *q = row + r;
      acc = fmaf(w23_to_float(tap_w23(D - bs)), q[-1], acc);
      acc = fmaf(w23_to_float(tap_w23(D)), q[0], acc);
      acc = fmaf(w23_to_float(tap_w23(D + bs)), q[1], acc);
      D += bl;
      row += P;
    }
  }
  return acc;
}

// One task: image b of job J, angles [a_begin, a_begin + g.AB) of its list,
// computed by the 8 CTAs of this cluster.  Ends with a cluster barrier, after
// which the CTA's shared memory may be reused.
template <int OP>
__device__ __forceinline__ void band_task(const Job &J, int b, int a_begin, const BandGeom &g,
                                          const AngleConst *ang, int *status, float *smem,
                                          AngleConst *sc, int *sai, cg::cluster_group &cluster) {
  const int tid = threadIdx.x;
  const int band = (int)cluster.block_rank();
  if (a_begin >= J.m) return;  // uniform over the cluster: no peer waits for it
  const int na = min(g.AB, J.m - a_begin);
  const int nd = g.n_det, N = g.N;
  const int nrows = g.AB;                              // rows of partial bins
  float *part = smem;                                  // [nrows][n_det]
  float *buf = smem + ((nrows * nd + 3) & ~3);         // [SB][P], 16-byte aligned

  if (tid < kMaxAB) {
    int ai = -1;
    if (tid < na) {
      ai = J.idx ? J.idx[a_begin + tid] : a_begin + tid;
      if (ai < 0 || ai >= g.n_angles) {
        if (band == 0) atomicOr(status, 1);
        ai = -1;
      }
    }
    sai[tid] = ai;
    if (ai >= 0) sc[tid] = ang[ai];
  }
  for (int e = tid; e < nrows * nd; e += kThreads) part[e] = 0.0f;
  __syncthreads();

  const size_t xo = (size_t)b * N * N;
  const int L0 = band * g.R, L1 = min(N, L0 + g.R);
  for (int mode = 1; mode >= 0; --mode) {
    bool any = false;
    for (int a = 0; a < na; ++a) any |= (sai[a] >= 0 && sc[a].mode == mode);
    if (!any) continue;
    const int P = mode ? g.Prow : g.Pcol;
    for (int s0 = L0; s0 < L1; s0 += g.SB) {
      const int s1 = min(L1, s0 + g.SB), nl = s1 - s0;
      __syncthreads();  // the previous sub-band is no longer read
      stage(J.in, xo, J.in_bf16, N, mode, s0, nl, buf, P, g.fast != 0);
      __syncthreads();
      for (int a = 0; a < na; ++a) {
        if (sai[a] < 0 || sc[a].mode != mode) continue;
        for (int k = tid; k < nd; k += kThreads)
          part[a * nd + k] += OP == OP_JOSEPH ? joseph_partial(sc[a], k, s0, s1, N, buf, P)
                                              : bpadj_partial(sc[a], k, s0, s1, N, buf, P);
      }
    }
  }

  cluster.sync();
  const int n_items = na * nd;
  for (int it = band * kThreads + tid; it < n_items; it += kBands * kThreads) {
    const int a = it / nd, k = it - a * nd;
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < kBands; ++q) s += cluster.map_shared_rank(part, q)[it];
    const int ai = sai[a];
    const size_t o = ((size_t)b * J.m + a_begin + a) * nd + k;
    float v;
    if (ai < 0) {
      v = 0.0f;
    } else if (OP == OP_JOSEPH) {
      v = s * sc[a].W;
      if (J.aux) v = ld_any(J.aux, ((size_t)b * g.n_angles + ai) * nd + k, J.aux_bf16) - v;
      v *= J.alpha;
    } else {
      v = s * J.alpha;
    }
    st_any(J.out, o, v, J.out_bf16);
  }
  cluster.sync();  // keep this CTA's partials alive until every peer has read them
}

template <int OP>
__global__ void __cluster_dims__(kBands, 1, 1) __launch_bounds__(kThreads)
    band_kernel(const BandArgs args) {
  extern __shared__ float4 smem4[];
  __shared__ AngleConst sc[kMaxAB];
  __shared__ int sai[kMaxAB];
  cg::cluster_group cluster = cg::this_cluster();
  // the job and image of this cluster
  const int z = blockIdx.z;
  const int jn = (args.jobs.njobs > 1 && z >= args.jobs.j[0].nimg) ? 1 : 0;
  const Job &J = args.jobs.j[jn];
  const int b = z - (jn ? args.jobs.j[0].nimg : 0);
  band_task<OP>(J, b, blockIdx.y * args.g.AB, args.g, args.ang, args.status,
                reinterpret_cast<float *>(smem4), sc, sai, cluster);
}

// Persistent form over the tasks of a batch of instances (plans of their
// own): each cluster takes the next task from a global counter (tasks come
// in decreasing cost order) until none is left; the last cluster to finish
// resets the counter for the next launch.
template <int OP>
__global__ void __cluster_dims__(kBands, 1, 1) __launch_bounds__(kThreads)
    band_batch_kernel(const BatchItem *items, const int4 *tasks, int n_tasks, int AB,
                      int *queue) {
  extern __shared__ float4 smem4[];
  __shared__ AngleConst sc[kMaxAB];
  __shared__ int sai[kMaxAB];
  __shared__ int s_task;
  cg::cluster_group cluster = cg::this_cluster();
  const bool leader = cluster.block_rank() == 0 && threadIdx.x == 0;
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
    const BandGeom g = band_geom(it.N, it.n_det, it.n_angles, OP, AB);
    band_task<OP>(J, tk.y, tk.z, g, it.ang, it.status, reinterpret_cast<float *>(smem4), sc,
                  sai, cluster);
  }
  if (leader) queue_retire(queue, gridDim.x / kBands);
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

template <int OP>
int set_band_smem(size_t smem) {
  static size_t configured[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (smem > 48 * 1024 && smem > configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(band_kernel<OP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(band_batch_kernel<OP>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "band kernel: shared memory attribute");
    configured[dev] = smem;
  }
  return SKEI_OK;
}

template <int OP>
int launch_band(skei_plan p, const Jobs &jobs, cudaStream_t st) {
  int m_max = 0, nimg = 0;
  for (int q = 0; q < jobs.njobs; ++q) {
    m_max = max(m_max, jobs.j[q].m);
    nimg += jobs.j[q].nimg;
  }
  if (nimg > 65535) return set_error(SKEI_EINVAL, "too many images (%d) in one launch", nimg);

  // angles per cluster: fewest waves x angles per CTA (the per-CTA time),
  // ties to the larger block (less staging)
  const int ab_max = min(kMaxAB, m_max);
  int best_ab = 1;
  double best_cost = 1e300;
  for (int ab = 1; ab <= ab_max; ++ab) {
    const size_t bytes = band_smem(band_geom(p->N, p->n_det, p->n_angles, OP, ab));
    if (bytes > 200 * 1024) continue;
    int per_sm = (int)((227 * 1024) / (bytes + 1024));
    per_sm = max(1, min(per_sm, 8));
    const double slots = (double)sm_count() * per_sm;
    double ctas = 0.0;
    for (int q = 0; q < jobs.njobs; ++q)
      ctas += (double)kBands * ((jobs.j[q].m + ab - 1) / ab) * jobs.j[q].nimg;
    const double cost = std::ceil(ctas / slots) * ab;
    if (cost <= best_cost) { best_cost = cost; best_ab = ab; }
  }
  const BandGeom g = band_geom(p->N, p->n_det, p->n_angles, OP, best_ab);
  const size_t smem = band_smem(g);
  if (smem > 227 * 1024)
    return set_error(SKEI_EINVAL, "detector of %d bins needs too much shared memory", g.n_det);
  SKEI_TRY(set_band_smem<OP>(smem));
  BandArgs a{jobs, p->d_ang, p->d_status, g};
  dim3 grid(kBands, (m_max + g.AB - 1) / g.AB, nimg);
  band_kernel<OP><<<grid, kThreads, smem, st>>>(a);
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

}  // namespace

int launch_band_jobs(skei_plan p, int op, const Jobs &jobs, cudaStream_t st) {
  if (op == OP_JOSEPH) return launch_band<OP_JOSEPH>(p, jobs, st);
  if (op == OP_BP_ADJ) return launch_band<OP_BP_ADJ>(p, jobs, st);
  return set_error(SKEI_EINVAL, "band launch: unknown operator %d", op);
}

size_t band_batch_smem(int op, int N, int n_det, int n_angles, int AB) {
  return band_smem(band_geom(N, n_det, n_angles, op, AB));
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
