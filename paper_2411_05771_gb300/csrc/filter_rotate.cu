// Ram-Lak filtering H of FBP (Sec. 2.1 / 4.1.1: FBP as the stable
// approximation of A^dagger) and the bilinear rotations T_g of the CT
// transform group (Sec. 4.1.3) with their exact gathered transposes.
#include <cmath>
#include <mutex>
#include <type_traits>

#include "fft.cuh"

namespace skei {

// Ram-Lak taps h(n) for n = 0..SKEI_MAX_NDET-1 (unit bins): h(0) = 1/4,
// h(odd n) = -1/(pi^2 n^2), h(even n) = 0.  They do not depend on the plan,
// so one copy lives in constant memory, where a warp-uniform read is a
// broadcast that costs no shared-memory bandwidth.
__constant__ float c_ramlak[SKEI_MAX_NDET];
// The odd taps as pairs (h(n), h(n)), n = 2i + 1 (the even taps beyond h(0)
// are zero): one 8-byte constant load feeds a packed FP32 pair.
__constant__ float2 c_ramlak_odd[SKEI_MAX_NDET / 2 + 4];
__constant__ float2 c_ramlak_pair0[1];   // (h(0), h(0))

// Uploads the taps once per device (called by skei_plan_create, so never
// inside a stream capture).
int ensure_ramlak_taps() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return set_error(SKEI_ECUDA, "ramlak taps: no current device");
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return SKEI_OK;
  std::vector<float> taps(SKEI_MAX_NDET);
  for (int n = 0; n < SKEI_MAX_NDET; ++n)
    taps[n] = n == 0 ? 0.25f
                     : (n % 2 == 0 ? 0.0f : (float)(-1.0 / (M_PI * M_PI * (double)n * (double)n)));
  cudaError_t e = cudaMemcpyToSymbol(c_ramlak, taps.data(), sizeof(float) * SKEI_MAX_NDET);
  if (e != cudaSuccess) return cuda_error(e, "ramlak taps upload");
  std::vector<float2> odd(SKEI_MAX_NDET / 2 + 4, make_float2(0.0f, 0.0f));
  for (int i = 0; 2 * i + 1 < SKEI_MAX_NDET; ++i) odd[i] = make_float2(taps[2 * i + 1], taps[2 * i + 1]);
  e = cudaMemcpyToSymbol(c_ramlak_odd, odd.data(), sizeof(float2) * odd.size());
  if (e != cudaSuccess) return cuda_error(e, "ramlak odd taps upload");
  const float2 h0 = make_float2(taps[0], taps[0]);
  e = cudaMemcpyToSymbol(c_ramlak_pair0, &h0, sizeof(float2));
  if (e != cudaSuccess) return cuda_error(e, "ramlak taps upload");
  done[dev] = true;
  return SKEI_OK;
}

// The Ram-Lak taps' spectrum on L points, L the smallest power of two
// >= 2 n_det - 1 (so that the circular convolution of a zero-padded row is
// the linear one): H[f] = h(0) + 2 sum_{n odd < n_det} h(n) cos(2 pi f n / L)
// (h is real and even, so H is real), in FP64.  Rows of up to 2048 bins.
int make_filter_spectrum(skei_plan p) {
  const int nd = p->n_det;
  int L = 1;
  while (L < 2 * nd - 1) L *= 2;
  if (nd < 64 || L > 4096) return SKEI_OK;   // direct form only
  std::vector<float> H(L);
  for (int f = 0; f < L; ++f) {
    double s = 0.25;
    for (int n = 1; n < nd; n += 2)
      s += 2.0 * (-1.0 / (M_PI * M_PI * (double)n * (double)n)) *
           std::cos(2.0 * M_PI * (double)(((long long)f * n) % L) / (double)L);
    H[f] = (float)s;
  }
  cudaError_t e = dev_malloc(reinterpret_cast<void **>(&p->d_hspec), sizeof(float) * L);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_hspec, H.data(), sizeof(float) * L, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p->d_hspec);
    p->d_hspec = nullptr;
    return e == cudaErrorMemoryAllocation ? set_error(SKEI_ENOMEM, "filter spectrum allocation")
                                          : cuda_error(e, "filter spectrum upload");
  }
  p->fft_len = L;
  return SKEI_OK;
}

namespace {

// ---------------------------------------------------- Ram-Lak, FFT form --
// One CTA per pair of rows r, r+1, packed as z = p_r + i p_{r+1} and zero
// padded to L: FFT, times scale H / L, inverse FFT.  With h real and even,
// H is real and the result is q_r + i q_{r+1}.  The same linear
// convolution as the direct form, in O(L log L) per pair of rows.
constexpr int kFftThreads = 512;

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kFftThreads)
    ramlak_fft_kernel(const Tin *in, Tout *out, int rows, int nd, int L, const float *hspec,
                      float scale) {
  pdl_enter();
  extern __shared__ float2 fsm[];
  float2 *tw = fsm, *A = fsm + L / 2, *Bf = A + L;
  twiddles(tw, L);
  const int r0 = 2 * blockIdx.x;
  const bool two = r0 + 1 < rows;
  const Tin *p0 = in + (size_t)r0 * nd, *p1 = p0 + nd;
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    float x = 0.0f, y = 0.0f;
    if (t < nd) {
      x = ldg_f(p0 + t);
      if (two) y = ldg_f(p1 + t);
    }
    A[t] = make_float2(x, y);
  }
  __syncthreads();
  float2 *R = fft_smem(A, Bf, L, 1, 0, 1, tw, false, false);
  const float s = scale / (float)L;
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    const float h = __ldg(hspec + t) * s;
    R[t] = make_float2(R[t].x * h, R[t].y * h);
  }
  __syncthreads();
  const float2 *Q = fft_smem(R, R == A ? Bf : A, L, 1, 0, 1, tw, true, false);
  Tout *q0 = out + (size_t)r0 * nd, *q1 = q0 + nd;
  for (int t = threadIdx.x; t < nd; t += blockDim.x) {
    st_f(q0 + t, Q[t].x);
    if (two) st_f(q1 + t, Q[t].y);
  }
}

// ------------------------------------------------------------- Ram-Lak --
//   q[k] = scale (h0 p[k] + sum_{n odd} h(n) (p[k-n] + p[k+n]))
// (the even taps beyond h(0) are zero).  A thread owns 8 consecutive
// outputs as 4 pairs; for an odd tap n it needs the pairs
// (p[k-n], p[k-n+1]) and (p[k+n], p[k+n+1]) of each output pair, which
// start at odd offsets from the even outputs, so the row is staged a second
// time shifted by one element (`po`), where they are 8-byte aligned.  From
// tap n to n+2 the left window slides by one pair and the right one the
// other way: two 8-byte loads per tap serve 8 output-taps, and the packed
// FP32 pair instructions (add.f32x2, fma.rn.f32x2) do two IEEE operations
// each.  The odd taps are split into kFSeg segments handled by different
// warps (short dependency chains, more warps), whose partial sums are added
// in a fixed order.  Lanes are 8 outputs (32 bytes) apart, so the staged
// rows are skewed by two words per 32 to keep their 8-byte loads free of
// bank conflicts.  Build-time knob: kFSeg.
#ifndef SKEI_FILTER_SEGMENTS
#define SKEI_FILTER_SEGMENTS 8
#endif
constexpr int kFSeg = SKEI_FILTER_SEGMENTS;
// Skewed shared-memory index of row element e: two pad words per 32, the
// boundaries placed so that the 4 pairs that one tap group loads from a
// window never straddle one (left window: boundary after e = 5 mod 32;
// right window: after 7 mod 32), so a group needs one address computation.
__host__ __device__ constexpr int skewL(int e) { return e + 2 * ((e + 26) >> 5); }
__host__ __device__ constexpr int skewR(int e) { return e + 2 * ((e + 24) >> 5); }
__host__ __device__ constexpr int f_outs(int GW) { return 256 * GW; }   // outputs per pass
__host__ __device__ inline int f_lp(int nd) { return (nd + 10 + 7) & ~7; }  // left margin
__host__ __device__ inline int f_len(int nd, int outs) {
  const int passes = (nd + outs - 1) / outs;
  return (f_lp(nd) + passes * outs + nd + 24 + 31) & ~31;
}
__host__ __device__ inline int f_words(int len) { return len + 2 * (len / 32 + 2); }
// Group warps (each 256 outputs of a pass) of the launch for rows of nd bins.
inline int f_group_warps(int nd) { return nd > 512 ? 3 : (nd > 256 ? 2 : 1); }
// Shared memory: the segments' partial sums, then three skewed copies of the
// row (even-aligned; shifted by one for each window).
inline size_t f_smem(int nd, int GW) {
  const int outs = f_outs(GW);
  return sizeof(float) * ((size_t)kFSeg * outs + 3 * (size_t)f_words(f_len(nd, outs)));
}

// Stages one row, p[k] = load(k) for k < nd, into pe (pe[e] = p[e - lp],
// skewL) and the shifted copies pl, pr (p[e + 1 - lp], skewL and skewR),
// zero outside the row; all threads, then a barrier.
template <typename F>
__device__ __forceinline__ void f_stage(F load, int nd, int len, float *pe, float *pl, float *pr) {
  const int lp = f_lp(nd);
  for (int e = threadIdx.x; e < len; e += blockDim.x) {
    const int k = e - lp;
    const float v = (k >= 0 && k < nd) ? load(k) : 0.0f;
    if (!SKEI_CHECK || ck_smem(pe + skewL(e), 4, CK_FILT_STAGE)) pe[skewL(e)] = v;
    if (e > 0) {
      if (!SKEI_CHECK || ck_smem(pl + skewL(e - 1), 4, CK_FILT_STAGE)) pl[skewL(e - 1)] = v;
      if (!SKEI_CHECK || ck_smem(pr + skewR(e - 1), 4, CK_FILT_STAGE)) pr[skewR(e - 1)] = v;
    }
  }
  if (threadIdx.x == 0) {
    if (!SKEI_CHECK || ck_smem(pl + skewL(len - 1), 4, CK_FILT_STAGE)) pl[skewL(len - 1)] = 0.0f;
    if (!SKEI_CHECK || ck_smem(pr + skewR(len - 1), 4, CK_FILT_STAGE)) pr[skewR(len - 1)] = 0.0f;
  }
  __syncthreads();
}

// Filters the staged row: out[k] = scale (H p)[k], k < nd, for the passes
// pass0, pass0 + pstep, ... of f_outs(GW) outputs.  32 GW kFSeg threads.
template <int GW, typename Tout>
__device__ __forceinline__ void f_compute(int nd, float scale, float *red, const float *pe,
                                          const float *pl, const float *pr, Tout *out, int pass0,
                                          int pstep, int ostride = 1) {
  constexpr int outs = f_outs(GW);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = warp % GW, seg = warp / GW;
  const int lp = f_lp(nd);
  // odd taps 1, 3, ..., split into kFSeg runs of whole 4-tap groups
  const int groups = (nd / 2 + 3) / 4;
  const int g0 = (groups * seg) / kFSeg, g1 = (groups * (seg + 1)) / kFSeg;
  const f2x h0 = reinterpret_cast<const f2x *>(c_ramlak_pair0)[0];
  const f2x *hodd = reinterpret_cast<const f2x *>(c_ramlak_odd);
  // the pair (p[k], p[k+1]) for k + lp odd (shifted copies) and even (pe)
  auto ldl = [&](int k) {
    return lds_ck(reinterpret_cast<const f2x *>(pl + skewL(k + lp - 1)), CK_FILT_TAP);
  };
  auto ldr = [&](int k) {
    return lds_ck(reinterpret_cast<const f2x *>(pr + skewR(k + lp - 1)), CK_FILT_TAP);
  };
  auto lde = [&](int k) {
    return lds_ck(reinterpret_cast<const f2x *>(pe + skewL(k + lp)), CK_FILT_TAP);
  };
  for (int kb = pass0 * outs; kb < nd; kb += pstep * outs) {
    const int ko = 8 * (lane + 32 * gw);
    const int k0 = kb + ko;
    f2x acc[4], L[4], R[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = seg == 0 ? f2_mul(h0, lde(k0 + 2 * j)) : 0ull;
    const int n1 = 1 + 8 * g0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      L[j] = ldl(k0 + 2 * j - n1);
      R[j] = ldr(k0 + 2 * j + n1);
    }
    for (int gi = g0; gi < g1; ++gi) {
      // the group's new left pairs start at element index bL - 2t (bL = 4
      // mod 8), the right ones at bR + 2t (bR = 0 mod 8): one skewed base
      // each, no boundary inside
      const f2x *ql = reinterpret_cast<const f2x *>(pl + skewL(k0 + lp - 4 - 8 * gi));
      const f2x *qr = reinterpret_cast<const f2x *>(pr + skewR(k0 + lp + 8 + 8 * gi));
      const f2x *hg = hodd + 4 * gi;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const f2x hh = hg[t];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] = f2_fma(hh, f2_add(L[j], R[j]), acc[j]);
        L[3] = L[2]; L[2] = L[1]; L[1] = L[0]; L[0] = lds_ck(ql - t, CK_FILT_TAP);
        R[0] = R[1]; R[1] = R[2]; R[2] = R[3]; R[3] = lds_ck(qr + t, CK_FILT_TAP);
      }
    }
    __syncthreads();   // red of the previous pass is no longer read
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (!SKEI_CHECK || ck_smem(red + seg * outs + ko + 2 * j, 8, CK_FILT_STAGE))
        *reinterpret_cast<f2x *>(red + seg * outs + ko + 2 * j) = acc[j];
    __syncthreads();
    for (int o = threadIdx.x; o < outs; o += blockDim.x) {
      const int k = kb + o;
      if (k >= nd) continue;
      float v = red[o];
#pragma unroll
      for (int sg = 1; sg < kFSeg; ++sg) v += red[sg * outs + o];
      st_f(out + (size_t)k * ostride, scale * v);
    }
  }
}

// Filters one row from global memory (a CTA of 32 GW kFSeg threads).
template <int GW, typename Tin, typename Tout>
__device__ __forceinline__ void ramlak_row(const Tin *pr, Tout *po_out, int nd, float scale,
                                           float *smem, int pass0, int pstep) {
  constexpr int outs = f_outs(GW);
  const int len = f_len(nd, outs), words = f_words(len);
  float *red = smem, *pe = red + kFSeg * outs, *pl = pe + words, *prr = pl + words;
  f_stage([&](int k) { return ldg_f(pr + k); }, nd, len, pe, pl, prr);
  f_compute<GW>(nd, scale, red, pe, pl, prr, po_out, pass0, pstep);
}

template <int GW, typename Tin, typename Tout>
__global__ void __launch_bounds__(32 * GW * kFSeg)
    ramlak_kernel(const Tin *in, Tout *out, int nd, float scale) {
  pdl_enter();
  extern __shared__ float4 smem4[];
  const size_t row = blockIdx.x;
  ramlak_row<GW, Tin, Tout>(in + row * nd, out + row * nd, nd, scale,
                            reinterpret_cast<float *>(smem4), blockIdx.y, gridDim.y);
}

// Persistent form over the rows of a batch of instances (task = item, row;
// rows come in decreasing n_det order); every row in passes of 768 outputs.
constexpr int kFBatchGW = 3;
constexpr int kFilterThreads = 32 * kFBatchGW * kFSeg;
__global__ void __launch_bounds__(kFilterThreads)
    ramlak_batch_kernel(const BatchItem *items, const int4 *tasks, int n_tasks, int *queue) {
  extern __shared__ float4 smem4[];
  float *smem = reinterpret_cast<float *>(smem4);
  __shared__ int s_task;
  for (;;) {
    __syncthreads();  // the previous row's shared memory and s_task are no longer read
    if (threadIdx.x == 0) s_task = atomicAdd(queue, 1);
    __syncthreads();
    const int t = s_task;
    if (t >= n_tasks) break;
    const int4 tk = tasks[t];
    const BatchItem &it = items[tk.x];
    const int nd = it.n_det;
    const size_t o = (size_t)tk.y * nd;
    constexpr int G = kFBatchGW;
    if (it.in_bf16) {
      const __nv_bfloat16 *pi = static_cast<const __nv_bfloat16 *>(it.in) + o;
      if (it.out_bf16)
        ramlak_row<G>(pi, static_cast<__nv_bfloat16 *>(it.out) + o, nd, it.alpha, smem, 0, 1);
      else ramlak_row<G>(pi, static_cast<float *>(it.out) + o, nd, it.alpha, smem, 0, 1);
    } else {
      const float *pi = static_cast<const float *>(it.in) + o;
      if (it.out_bf16)
        ramlak_row<G>(pi, static_cast<__nv_bfloat16 *>(it.out) + o, nd, it.alpha, smem, 0, 1);
      else ramlak_row<G>(pi, static_cast<float *>(it.out) + o, nd, it.alpha, smem, 0, 1);
    }
  }
  if (threadIdx.x == 0) queue_retire(queue, gridDim.x);
}

// ------------------------------------------ band sums, then the filter --
// The second pass of the workspace form of A or B^T (the per-band sums of
// the band kernels, [image][band][angle][bin]) fused with the Ram-Lak
// filter of the step: one CTA per sinogram row adds the row's bands in
// order (as the separate reduction does) and applies the operator's
// epilogue; rows of job `fjob` are then filtered in the same CTA and only
// their filtered values are written (to fout, FP32, fscale H), the other
// job's rows are written as they are (A's MC residual y - A x).
template <int OP, int GW>
__global__ void __launch_bounds__(32 * GW * kFSeg)
    band_sum_filter_kernel(const Jobs jobs, const AngleConst *ang, int n_angles, int nd, int nb0,
                           int nb1, const float *part, size_t off0, size_t off1,
                           size_t part_floats, int fjob, float fscale, float *fout,
                           int fil4) {
  pdl_enter();
  extern __shared__ float4 smem4[];
  constexpr int outs = f_outs(GW);
  const int row = blockIdx.x;
  const int rows0 = jobs.j[0].nimg * jobs.j[0].m;
  const int jn = row >= rows0 ? 1 : 0;
  const Job &J = jobs.j[jn];
  const int r = row - (jn ? rows0 : 0);
  const int b = r / J.m, a = r - b * J.m;
  const int nb = jn ? nb1 : nb0;
  const size_t n = (size_t)J.m * nd;
  const float *pb = part + (jn ? off1 : off0) + (size_t)b * nb * n + (size_t)a * nd;
  const int *idx = job_idx(J, b);
  const int ai = idx ? idx[a] : a;
  const bool dead = ai < 0 || ai >= n_angles;
  const float W = (OP == 0 && !dead) ? ang[ai].W : 1.0f;
  // the row's value at bin k: its bands in order, 32 loads in flight
  auto value = [&](int k) {
    float s = 0.0f;
    int q = 0;
    for (; q + 32 <= nb; q += 32) {
      float v[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) v[u] = __ldg(pb + (size_t)(q + u) * n + k);
#pragma unroll
      for (int u = 0; u < 32; ++u) s += v[u];
    }
    for (; q < nb; ++q) s += __ldg(pb + (size_t)q * n + k);
    if (SKEI_CHECK) {
      // the first and last band this value read
      ck_range(pb + k, 4, part, part + part_floats, CK_FILT_SUMS);
      ck_range(pb + (size_t)(nb - 1) * n + k, 4, part, part + part_floats, CK_FILT_SUMS);
    }
    float v;
    if (dead) {
      v = 0.0f;
    } else if (OP == 0) {
      v = s * W;
      if (J.aux) v = ld_any(J.aux, ((size_t)b * n_angles + ai) * nd + k, J.aux_bf16) - v;
      v *= J.alpha;
    } else {
      v = s * J.alpha;
    }
    return v;
  };
  if (jn != fjob) {
    for (int k = threadIdx.x; k < nd; k += blockDim.x)
      st_any(J.out, (size_t)b * n + (size_t)a * nd + k, value(k), J.out_bf16);
    return;
  }
  const int len = f_len(nd, outs), words = f_words(len);
  float *red = reinterpret_cast<float *>(smem4), *pe = red + kFSeg * outs, *pl = pe + words,
        *prr = pl + words;
  f_stage(value, nd, len, pe, pl, prr);
  if (fil4)   // interleaved by groups of 4 images (Job::in_il4)
    f_compute<GW>(nd, fscale, red, pe, pl, prr,
                  fout + ((size_t)(b >> 2) * J.m + a) * nd * 4 + (b & 3), 0, 1, 4);
  else
    f_compute<GW>(nd, fscale, red, pe, pl, prr, fout + (size_t)r * nd, 0, 1);
}

// ----------------------------------------- Ram-Lak, tensor-core form --
// The filter of a tile of 16 rows and 32 outputs as the matrix product
// Q = P H^T with H[k][j] = h(|k - j|) (Toeplitz in the taps): warp-level TF32
// tensor-core MMAs (m16n8k8).  Each FP32 operand is split into a TF32 head
// and a TF32 tail, x = hi + lo, and the three products hi.hi + hi.lo + lo.hi
// (the lo.lo term is below FP32 rounding) of each step of 8 bins go to a
// fresh accumulator that one IEEE addition adds to the running sum: with
// the tensor cores' own accumulation over the whole row, smooth sinograms
// (whose filtered rows are 160-310 times smaller than the rows) lost 4x the
// direct form's accuracy; with fresh steps, 2x.  The 8 warps of a CTA split the row length
// and add their partial tiles in a fixed order.  Rows of up to kTcMaxNd
// bins (the staged tile must fit shared memory); longer rows take the
// direct form.
// (Measured on GB300 at 120 rows of 725 bins: 9.4 us against the direct
// form's 7.9; 16, 64 and 128 outputs per CTA or 4 warps were slower still.)
constexpr int kTcRows = 16, kTcOuts = 32, kTcWarps = 8, kTcThreads = 32 * kTcWarps;
constexpr int kTcMaxNd = 2048;
constexpr int kTcTapPad = kTcOuts + 16;   // zero taps beyond n_det that an index may reach

__host__ __device__ __forceinline__ int tc_pitch(int nd) {
  // a multiple of 32 plus 4 words: the A-fragment loads (rows g, columns t)
  // of a warp hit 32 distinct banks
  return ((((nd + 7) & ~7) + 31) & ~31) + 4;
}
static size_t tc_smem(int nd) {
  return sizeof(float) * ((size_t)kTcRows * tc_pitch(nd) + 2 * (size_t)(nd + kTcTapPad) +
                          (size_t)kTcWarps * kTcRows * kTcOuts);
}

__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// c += a b for one 16 x 8 x 8 TF32 product: a row-major 16 x 8 (lane
// g = lane / 4, t = lane % 4 holds (g, t), (g+8, t), (g, t+4), (g+8, t+4)),
// b 8 x 8 by columns ((t, g), (t+4, g)), c 16 x 8 ((g, 2t), (g, 2t+1),
// (g+8, 2t), (g+8, 2t+1)).
__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kTcThreads)
    ramlak_tc_kernel(const Tin *in, Tout *out, int rows, int nd, float scale,
                     const float *taps) {
  extern __shared__ float4 smem4[];
  const int pitch = tc_pitch(nd), Kp = (nd + 7) & ~7, ntap = nd + kTcTapPad;
  float *Ps = reinterpret_cast<float *>(smem4);          // [16][pitch] rows of P
  float *th = Ps + kTcRows * pitch, *tl = th + ntap;     // tap heads and tails
  float *red = tl + ntap;                                // [warps][16][32]
  const int r0 = blockIdx.y * kTcRows, k0 = blockIdx.x * kTcOuts;
  // the taps do not depend on the preceding kernel: split them first (read
  // through a global pointer: the lanes' distinct addresses would serialise
  // in the constant cache)
  for (int d = threadIdx.x; d < ntap; d += kTcThreads) {
    const float h = d < nd ? __ldg(taps + d) : 0.0f;
    const float hi = __uint_as_float(to_tf32(h));
    th[d] = hi;
    tl[d] = __uint_as_float(to_tf32(h - hi));
  }
  pdl_enter();
  // the 16 rows, zero beyond the rows and bins: every load in flight at once
  // (FP32: asynchronous copies, zero-filled where out of range)
  for (int r = 0; r < kTcRows; ++r) {
    const bool live = r0 + r < rows;
    const Tin *pr = in + (size_t)(live ? r0 + r : 0) * nd;
    for (int j = threadIdx.x; j < Kp; j += kTcThreads) {
      const bool ok = live && j < nd;
      if constexpr (std::is_same<Tin, float>::value)
        cp_async4(&Ps[r * pitch + j], ok ? pr + j : in, ok);
      else
        Ps[r * pitch + j] = ok ? ldg_f(pr + j) : 0.0f;
    }
  }
  if constexpr (std::is_same<Tin, float>::value) {
    cp_async_commit();
    cp_async_wait_all();
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int steps = Kp / 8;
  const int s0 = warp * steps / kTcWarps, s1 = (warp + 1) * steps / kTcWarps;
  float acc[kTcOuts / 8][4];
#pragma unroll
  for (int nb = 0; nb < kTcOuts / 8; ++nb)
    acc[nb][0] = acc[nb][1] = acc[nb][2] = acc[nb][3] = 0.0f;
  for (int s = s0; s < s1; ++s) {
    const int j = 8 * s + t;
    const float x[4] = {Ps[g * pitch + j], Ps[(g + 8) * pitch + j], Ps[g * pitch + j + 4],
                        Ps[(g + 8) * pitch + j + 4]};
    unsigned ah[4], al[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ah[i] = to_tf32(x[i]);
      al[i] = to_tf32(x[i] - __uint_as_float(ah[i]));
    }
#pragma unroll
    for (int nb = 0; nb < kTcOuts / 8; ++nb) {
      // B[j][k] = h(|k - j|) at (j, k0 + 8 nb + g) and (j + 4, ...)
      const int d = k0 + 8 * nb + g - j;
      const int i0 = abs(d), i1 = abs(d - 4);
      const unsigned bh0 = __float_as_uint(th[i0]), bh1 = __float_as_uint(th[i1]);
      const unsigned bl0 = __float_as_uint(tl[i0]), bl1 = __float_as_uint(tl[i1]);
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      mma_tf32(c, al, bh0, bh1);
      mma_tf32(c, ah, bl0, bl1);
      mma_tf32(c, ah, bh0, bh1);
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[nb][i] += c[i];
    }
  }
  float *rw = red + warp * (kTcRows * kTcOuts);
#pragma unroll
  for (int nb = 0; nb < kTcOuts / 8; ++nb) {
    const int c = 8 * nb + 2 * t;
    rw[g * kTcOuts + c] = acc[nb][0];
    rw[g * kTcOuts + c + 1] = acc[nb][1];
    rw[(g + 8) * kTcOuts + c] = acc[nb][2];
    rw[(g + 8) * kTcOuts + c + 1] = acc[nb][3];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < kTcRows * kTcOuts; o += kTcThreads) {
    float v = red[o];
#pragma unroll
    for (int w = 1; w < kTcWarps; ++w) v += red[w * (kTcRows * kTcOuts) + o];
    const int row = r0 + o / kTcOuts, k = k0 + o % kTcOuts;
    if (row < rows && k < nd) st_f(out + (size_t)row * nd + k, scale * v);
  }
}

// ------------------------------------------------------------ rotation --
// Output pixel (i, j) samples the input at R(-g)(x_j, y_i), in fixed point
//   row = R0 + j s + i c,   col = C0 + j c - i s,
// R0 = h(1 - s - c), C0 = h(1 + s - c), h = (N-1)/2; bilinear weights
// (1-fr)(1-fc), (1-fr)fc, fr(1-fc), fr fc; taps outside the image are 0.
// Pixels per thread (knobs; measured on GB300 at 4 x 512^2: 8 for the
// rotation, 2 for its transpose; 4 / 2 and 1 / 4 were slower).
#ifndef SKEI_ROT_Q
#define SKEI_ROT_Q 8
#endif
#ifndef SKEI_ROTADJ_Q
#define SKEI_ROTADJ_Q 2
#endif
constexpr int kRotX = 32, kRotY = 8, kRotQ = SKEI_ROT_Q;  // CTA tile 32 x 8 kRotQ
constexpr int kRotThreads = kRotX * kRotY;

struct RotConst {
  long long c, s, C0, R0;  // 32.32
  float cf, sf, C0f, R0f;  // FP32 copies to choose candidates
};

__device__ __forceinline__ RotConst rot_const(double deg, int N) {
  double c, s;
  trig_deg(deg, &c, &s);
  const double h = 0.5 * (N - 1);
  const double C0 = h * (1.0 + s - c), R0 = h * (1.0 - s - c);
  return RotConst{to_fx(c), to_fx(s), to_fx(C0), to_fx(R0),
                  (float)c, (float)s, (float)C0, (float)R0};
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kRotThreads)
    rotate_kernel(const Tin *x, int N, int G, int Ch, const double *g_deg, Tout *out) {
  pdl_enter();
  __shared__ RotConst rc;
  // blockIdx.z = (b G + g) Ch + ch: output image; its angle is g_deg[b G + g]
  const int bgc = blockIdx.z, bg = bgc / Ch, b = bg / G, ch = bgc - bg * Ch;
  if (threadIdx.x == 0) rc = rot_const(g_deg[bg], N);
  __syncthreads();
  const int tx = threadIdx.x % kRotX, ty = threadIdx.x / kRotX;
  const int j = blockIdx.x * kRotX + tx;
  const int i_first = blockIdx.y * kRotY * kRotQ + ty;
  if (j >= N) return;
  const Tin *xb = x + ((size_t)b * Ch + ch) * N * N;
  Tout *ob = out + (size_t)bgc * N * N + j;
  long long row = rc.R0 + (long long)j * rc.s + (long long)i_first * rc.c;
  long long col = rc.C0 + (long long)j * rc.c - (long long)i_first * rc.s;
  const long long drow = rc.c * kRotY, dcol = -rc.s * kRotY;
  // Taps outside the image read as 0 through predicated loads, with no
  // branch: fma(w, 0, v) = v, so the FMA chain gives what skipping them
  // would.
#pragma unroll 2
  for (int q = 0; q < kRotQ; ++q, row += drow, col += dcol) {
    const int i = i_first + kRotY * q;
    const int i0 = ipart(row), j0 = ipart(col);
    const float fr = frac23(row), fc = frac23(col);
    const float gr = 1.0f - fr, gc = 1.0f - fc;
    const bool r0 = (unsigned)i0 < (unsigned)N, r1 = (unsigned)(i0 + 1) < (unsigned)N;
    const bool c0 = (unsigned)j0 < (unsigned)N, c1 = (unsigned)(j0 + 1) < (unsigned)N;
    const Tin *pa = xb + (ptrdiff_t)i0 * N + j0;
    const float x00 = (r0 & c0) ? ldg_f(pa) : 0.0f, x01 = (r0 & c1) ? ldg_f(pa + 1) : 0.0f;
    const float x10 = (r1 & c0) ? ldg_f(pa + N) : 0.0f;
    const float x11 = (r1 & c1) ? ldg_f(pa + N + 1) : 0.0f;
    float v = fmaf(gr * gc, x00, 0.0f);
    v = fmaf(gr * fc, x01, v);
    v = fmaf(fr * gc, x10, v);
    v = fmaf(fr * fc, x11, v);
    if (i < N) st_f(ob + (size_t)i * N, v);
  }
}

// Transpose, gathered per input pixel (a, bb): the output pixels whose
// sample lands in (a-1, a+1) x (bb-1, bb+1) lie within sqrt 2 of the
// rotated position of (a, bb), i.e. among 3x3 candidates; each candidate's
// sample is recomputed exactly in the forward's fixed-point form and
// weighted by its exact tap weights, reproducing the forward's bitwise.
constexpr int kAdjT = 16, kAdjQ = SKEI_ROTADJ_Q;  // CTA tile 16 x 16 kAdjQ
constexpr int kMaxG = 64;

// Linear-interpolation weight of a sample at fixed-point offset D (|D| < 8,
// 32-bit) from an integer position q, D = pos - q: 1-f if floor(pos) == q,
// f if floor(pos) == q-1, with f the 23-bit fraction of pos.  With
// a = D >> 5 (floor division) both are 1 - |a| 2^-23: for D >= 0, a is f's
// 23 bits; for D < 0, f's bits are a + 2^23.  Evaluated as the float with
// bits 0x40000000 - |a| (= 2 - |a| 2^-23, exact) minus 1; the result is
// <= 0 exactly when the tap gets no weight.
__device__ __forceinline__ float tap_wf(unsigned D) {
  return __int_as_float(0x40000000 - abs((int)D >> (kFxBits - 23))) - 1.0f;
}

template <typename Tin>
__device__ __forceinline__ float rot_adj_one(const RotConst &r, const Tin *gb, int N, int a,
                                             int bb, float s) {
  const float dc = (float)bb - r.C0f, dr = (float)a - r.R0f;
  const int ri = round_int(fmaf(-r.sf, dc, r.cf * dr));
  const int rj = round_int(fmaf(r.cf, dc, r.sf * dr));
  // exact offsets of candidate (ri-1, rj-1)'s sample from (a, bb); an
  // i step adds (c, -s), a j step (s, c); all within a few pixels, so
  // exact in 32-bit wrapping arithmetic on the low words
  const unsigned c32 = (unsigned)r.c, s32 = (unsigned)r.s;
  const unsigned dr0 = (unsigned)(r.R0 + (long long)(rj - 1) * r.s +
                                  (long long)(ri - 1) * r.c) - ((unsigned)a << kFxBits);
  const unsigned dc0 = (unsigned)(r.C0 + (long long)(rj - 1) * r.c -
                                  (long long)(ri - 1) * r.s) - ((unsigned)bb << kFxBits);
  bool jv[3];
#pragma unroll
  for (int dj = 0; dj < 3; ++dj) jv[dj] = (unsigned)(rj - 1 + dj) < (unsigned)N;
#pragma unroll
  for (int di = 0; di < 3; ++di) {
    const int i = ri - 1 + di;
    const bool iv = (unsigned)i < (unsigned)N;
    const Tin *row = gb + (ptrdiff_t)i * N + (rj - 1);
    const unsigned Dr1 = dr0 + di * c32, Dc1 = dc0 - di * s32;
#pragma unroll
    for (int dj = 0; dj < 3; ++dj) {
      const float wr = tap_wf(Dr1 + dj * s32), wc = tap_wf(Dc1 + dj * c32);
      if (iv & jv[dj] & (wr > 0.0f) & (wc > 0.0f)) s = fmaf(wr * wc, ldg_f(row + dj), s);
    }
  }
  return s;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kAdjT *kAdjT)
    rotate_adj_kernel(const Tin *gout, int N, int G, int Ch, const double *g_deg, float alpha,
                      float beta, Tout *gx) {
  pdl_enter();
  __shared__ RotConst rc[kMaxG];
  // blockIdx.z = b Ch + ch: output image
  const int bc = blockIdx.z, b = bc / Ch, ch = bc - b * Ch;
  const int t = threadIdx.y * kAdjT + threadIdx.x;
  const int bb = blockIdx.x * kAdjT + threadIdx.x;
  float acc[kAdjQ];
#pragma unroll
  for (int q = 0; q < kAdjQ; ++q) acc[q] = 0.0f;
  for (int g0 = 0; g0 < G; g0 += kMaxG) {
    const int ng = min(kMaxG, G - g0);
    __syncthreads();
    if (t < ng) rc[t] = rot_const(g_deg[(size_t)b * G + g0 + t], N);
    __syncthreads();
    if (bb >= N) continue;
    const size_t plane = (size_t)N * N * Ch;   // one rotation's images
    const Tin *gb = gout + ((size_t)b * G + g0) * plane + (size_t)ch * N * N;
    int g = 0;
    // two rotations at a time: twice the loads in flight; the sum over g
    // keeps its order
    for (; g + 2 <= ng; g += 2) {
      const RotConst r0 = rc[g], r1 = rc[g + 1];
#pragma unroll
      for (int q = 0; q < kAdjQ; ++q) {
        const int a = min((blockIdx.y * kAdjQ + q) * kAdjT + threadIdx.y, N - 1);
        acc[q] = rot_adj_one(r1, gb + (g + 1) * plane, N, a, bb,
                             rot_adj_one(r0, gb + g * plane, N, a, bb, acc[q]));
      }
    }
    for (; g < ng; ++g) {
      const RotConst r0 = rc[g];
#pragma unroll
      for (int q = 0; q < kAdjQ; ++q) {
        const int a = min((blockIdx.y * kAdjQ + q) * kAdjT + threadIdx.y, N - 1);
        acc[q] = rot_adj_one(r0, gb + g * plane, N, a, bb, acc[q]);
      }
    }
  }
  if (bb >= N) return;
#pragma unroll
  for (int q = 0; q < kAdjQ; ++q) {
    const int a = (blockIdx.y * kAdjQ + q) * kAdjT + threadIdx.y;
    if (a >= N) continue;
    const size_t o = ((size_t)bc * N + a) * N + bb;
    float v = alpha * acc[q];
    if (beta != 0.0f) v = fmaf(beta, ldg_f(gx + o), v);
    st_f(gx + o, v);
  }
}

// The rotation of x1 = x0 + theta (the residual network's output): every
// tap is x1 as stored (the FP32 sum rounded to T), so the result is bitwise
// the rotation of a stored x1; the CTAs of rotation g = 0 also store x1 at
// their own pixels.
template <typename T>
__global__ void __launch_bounds__(kRotThreads)
    rotate_residual_kernel(const T *x0, const float *theta, int N, int G, const double *g_deg,
                           T *x1, T *out) {
  pdl_enter();
  __shared__ RotConst rc;
  const int bg = blockIdx.z, b = bg / G, g = bg - b * G;
  if (threadIdx.x == 0) rc = rot_const(g_deg[bg], N);
  __syncthreads();
  const int tx = threadIdx.x % kRotX, ty = threadIdx.x / kRotX;
  const int j = blockIdx.x * kRotX + tx;
  const int i_first = blockIdx.y * kRotY * kRotQ + ty;
  if (j >= N) return;
  const T *xb = x0 + (size_t)b * N * N;
  T *ob = out + (size_t)bg * N * N + j;
  long long row = rc.R0 + (long long)j * rc.s + (long long)i_first * rc.c;
  long long col = rc.C0 + (long long)j * rc.c - (long long)i_first * rc.s;
  const long long drow = rc.c * kRotY, dcol = -rc.s * kRotY;
  auto x1v = [&](ptrdiff_t e) { return rnd_store<T>(ldg_f(xb + e) + __ldg(theta + e)); };
#pragma unroll 2
  for (int q = 0; q < kRotQ; ++q, row += drow, col += dcol) {
    const int i = i_first + kRotY * q;
    const int i0 = ipart(row), j0 = ipart(col);
    const float fr = frac23(row), fc = frac23(col);
    const float gr = 1.0f - fr, gc = 1.0f - fc;
    const bool r0 = (unsigned)i0 < (unsigned)N, r1 = (unsigned)(i0 + 1) < (unsigned)N;
    const bool c0 = (unsigned)j0 < (unsigned)N, c1 = (unsigned)(j0 + 1) < (unsigned)N;
    const ptrdiff_t e = (ptrdiff_t)i0 * N + j0;
    const float x00 = (r0 & c0) ? x1v(e) : 0.0f, x01 = (r0 & c1) ? x1v(e + 1) : 0.0f;
    const float x10 = (r1 & c0) ? x1v(e + N) : 0.0f;
    const float x11 = (r1 & c1) ? x1v(e + N + 1) : 0.0f;
    float v = fmaf(gr * gc, x00, 0.0f);
    v = fmaf(gr * fc, x01, v);
    v = fmaf(fr * gc, x10, v);
    v = fmaf(fr * fc, x11, v);
    if (i < N) {
      st_f(ob + (size_t)i * N, v);
      if (g == 0) {
        const size_t o = (size_t)i * N + j;
        st_f(x1 + (size_t)b * N * N + o, ldg_f(xb + o) + __ldg(theta + o));
      }
    }
  }
}

// The last launch of the residual network's step, one measurement: the
// rotation transpose gx = sum_g T_g^T gout[g] + gx (gx holds the MC term's
// A^T part; stored as T), then, per pixel, Adam on theta with the gradient
// d loss / d theta = gx + sum_g g_x3[g] (as stored), summed in that order;
// CTA 0 also does the loss's final pass (its partials are complete: the
// launches in between did not touch them).
template <typename T>
__global__ void __launch_bounds__(kAdjT *kAdjT)
    rotate_adj_adam_kernel(const float *gout, int N, int G, const double *g_deg, T *gx,
                           const T *g_x3, const AdamArgs adam, const LossFinal lf) {
  pdl_enter();
  __shared__ RotConst rc[kMaxG];
  extern __shared__ double seg_sum[];
  const int t = threadIdx.y * kAdjT + threadIdx.x;
  const int bb = blockIdx.x * kAdjT + threadIdx.x;
  float acc[kAdjQ];
#pragma unroll
  for (int q = 0; q < kAdjQ; ++q) acc[q] = 0.0f;
  const size_t plane = (size_t)N * N;
  for (int g0 = 0; g0 < G; g0 += kMaxG) {
    const int ng = min(kMaxG, G - g0);
    __syncthreads();
    if (t < ng) rc[t] = rot_const(g_deg[g0 + t], N);
    __syncthreads();
    if (bb >= N) continue;
    const float *gb = gout + (size_t)g0 * plane;
    int g = 0;
    for (; g + 2 <= ng; g += 2) {
      const RotConst r0 = rc[g], r1 = rc[g + 1];
#pragma unroll
      for (int q = 0; q < kAdjQ; ++q) {
        const int a = min((blockIdx.y * kAdjQ + q) * kAdjT + threadIdx.y, N - 1);
        acc[q] = rot_adj_one(r1, gb + (g + 1) * plane, N, a, bb,
                             rot_adj_one(r0, gb + g * plane, N, a, bb, acc[q]));
      }
    }
    for (; g < ng; ++g) {
      const RotConst r0 = rc[g];
#pragma unroll
      for (int q = 0; q < kAdjQ; ++q) {
        const int a = min((blockIdx.y * kAdjQ + q) * kAdjT + threadIdx.y, N - 1);
        acc[q] = rot_adj_one(r0, gb + g * plane, N, a, bb, acc[q]);
      }
    }
  }
  if (bb < N) {
    const float tstep = (float)max(__ldg(adam.step), 1);
    const float bc1 = -expm1f(tstep * adam.lnb1), bc2 = -expm1f(tstep * adam.lnb2);
#pragma unroll
    for (int q = 0; q < kAdjQ; ++q) {
      const int a = (blockIdx.y * kAdjQ + q) * kAdjT + threadIdx.y;
      if (a >= N) continue;
      const size_t o = (size_t)a * N + bb;
      const float v = fmaf(1.0f, ldg_f(gx + o), acc[q]);
      st_f(gx + o, v);
      float gr = 0.0f;
      gr += rnd_store<T>(v);
      for (int c = 0; c < G; ++c) gr += ldg_f(g_x3 + (size_t)c * plane + o);
      const float mi = fmaf(adam.b1, adam.m[o], adam.omb1 * gr);
      const float vi = fmaf(adam.b2, adam.v[o], adam.omb2 * gr * gr);
      adam.m[o] = mi;
      adam.v[o] = vi;
      adam.theta[o] -= adam.lr * (mi / bc1) / (sqrtf(vi / bc2) + adam.eps);
    }
  }
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    __syncthreads();
    ei_final_block(lf.partial, lf.B, lf.G, lf.cpi, lf.cpr, lf.lambda, lf.mc_scale, lf.mc_out,
                   lf.ei_out, lf.loss_out, seg_sum);
  }
}

}  // namespace

SKEI_CHECK_READER(check_read_filter)

// Dynamic shared memory of a batched filter CTA for rows of nd bins.
static size_t filter_smem(int nd) { return f_smem(nd, kFBatchGW); }

static int set_filter_batch_smem(size_t smem) {
  static size_t configured[64] = {0};
  return opt_in_smem(ramlak_batch_kernel, smem, configured,
                     "batched ramlak: shared memory attribute");
}

size_t filter_batch_smem(int n_det_max) { return filter_smem(n_det_max); }

int filter_batch_occupancy(size_t smem, int *ctas_per_sm) {
  SKEI_TRY(set_filter_batch_smem(smem));
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ramlak_batch_kernel,
                                                                kFilterThreads, smem);
  if (e != cudaSuccess) return cuda_error(e, "batched ramlak: occupancy");
  *ctas_per_sm = n > 0 ? n : 1;
  return SKEI_OK;
}

int launch_filter_batch(const BatchItem *items, const int4 *tasks, int n_tasks, size_t smem,
                        int ctas, int *queue, cudaStream_t st) {
  SKEI_TRY(set_filter_batch_smem(smem));
  ramlak_batch_kernel<<<ctas, kFilterThreads, smem, st>>>(items, tasks, n_tasks, queue);
  return check_launch("batched ramlak filter launch");
}

template <int GW, typename Tin, typename Tout>
int launch_filter_gw(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                     cudaStream_t st) {
  const int nd = p->n_det;
  const size_t smem = f_smem(nd, GW);
  auto kern = ramlak_kernel<GW, Tin, Tout>;
  static size_t configured[64] = {0};
  SKEI_TRY(opt_in_smem(kern, smem, configured, "ramlak: shared memory attribute"));
  const int passes = (nd + f_outs(GW) - 1) / f_outs(GW);
  launch_k(kern, dim3(rows, passes), dim3(32 * GW * kFSeg), smem, st, in, out, nd, scale);
  return check_launch("ramlak filter launch");
}

template <typename Tin, typename Tout>
int launch_filter(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                  cudaStream_t st) {
  switch (f_group_warps(p->n_det)) {
    case 1: return launch_filter_gw<1>(p, in, rows, scale, out, st);
    case 2: return launch_filter_gw<2>(p, in, rows, scale, out, st);
    default: return launch_filter_gw<3>(p, in, rows, scale, out, st);
  }
}

template <int OP, int GW>
int launch_band_sum_filter_gw(skei_plan p, const Jobs &jobs, int nb0, int nb1, const float *part,
                              size_t off0, size_t off1, size_t part_floats, const FilterReq &fr,
                              cudaStream_t st) {
  const int nd = p->n_det;
  const size_t smem = f_smem(nd, GW);
  auto kern = band_sum_filter_kernel<OP, GW>;
  static size_t configured[64] = {0};
  SKEI_TRY(opt_in_smem(kern, smem, configured, "band sums + filter: shared memory attribute"));
  long long rows = 0;
  for (int q = 0; q < jobs.njobs; ++q) rows += (long long)jobs.j[q].nimg * jobs.j[q].m;
  if (rows > 0x7fffffff) return set_error(SKEI_EINVAL, "band sums + filter: too many rows");
  launch_k(kern, dim3((unsigned)rows), dim3(32 * GW * kFSeg), smem, st, jobs,
           (const AngleConst *)p->d_ang, p->n_angles, nd, nb0, nb1, part, off0, off1,
           part_floats, fr.job, fr.scale, fr.out, fr.il4);
  return check_launch("band sums + filter launch");
}

int launch_band_sum_filter(skei_plan p, int op, const Jobs &jobs, int nb0, int nb1,
                           const float *part, size_t off0, size_t off1, size_t part_floats,
                           const FilterReq &fr, cudaStream_t st) {
  const int gw = f_group_warps(p->n_det);
  if (op == OP_JOSEPH) {
    if (gw == 1)
      return launch_band_sum_filter_gw<OP_JOSEPH, 1>(p, jobs, nb0, nb1, part, off0, off1,
                                                      part_floats, fr, st);
    if (gw == 2)
      return launch_band_sum_filter_gw<OP_JOSEPH, 2>(p, jobs, nb0, nb1, part, off0, off1,
                                                      part_floats, fr, st);
    return launch_band_sum_filter_gw<OP_JOSEPH, 3>(p, jobs, nb0, nb1, part, off0, off1,
                                                    part_floats, fr, st);
  }
  if (gw == 1)
    return launch_band_sum_filter_gw<OP_BP_ADJ, 1>(p, jobs, nb0, nb1, part, off0, off1,
                                                    part_floats, fr, st);
  if (gw == 2)
    return launch_band_sum_filter_gw<OP_BP_ADJ, 2>(p, jobs, nb0, nb1, part, off0, off1,
                                                    part_floats, fr, st);
  return launch_band_sum_filter_gw<OP_BP_ADJ, 3>(p, jobs, nb0, nb1, part, off0, off1,
                                                  part_floats, fr, st);
}

template <typename Tin, typename Tout>
int launch_filter_tc(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                     cudaStream_t st) {
  const int nd = p->n_det;
  if (nd > kTcMaxNd || rows > 65535 * kTcRows) return launch_filter(p, in, rows, scale, out, st);
  const size_t smem = tc_smem(nd);
  auto kern = ramlak_tc_kernel<Tin, Tout>;
  static size_t configured[64] = {0};
  static const float *taps[64] = {nullptr};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!taps[dev]) {
    void *a = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, c_ramlak);
    if (e != cudaSuccess) return cuda_error(e, "ramlak taps: symbol address");
    taps[dev] = static_cast<const float *>(a);
  }
  SKEI_TRY(opt_in_smem(kern, smem, configured, "ramlak tensor-core form: shared memory attribute"));
  launch_k(kern, dim3((nd + kTcOuts - 1) / kTcOuts, (rows + kTcRows - 1) / kTcRows),
           dim3(kTcThreads), smem, st, in, out, rows, nd, scale, taps[dev]);
  return check_launch("ramlak tensor-core launch");
}

// The EI step's filter form (knob: 0 direct, 1 FFT, 2 tensor-core).  At 120
// rows of 725 bins on GB300: direct 7.9 us, tensor-core 9.4 us, FFT 14.7 us
// (60 CTAs of 22 barrier-separated radix-2 stages are latency-bound), so the
// step keeps the direct form.
#ifndef SKEI_STEP_FILTER
#define SKEI_STEP_FILTER 0
#endif
template <typename Tin, typename Tout>
int launch_filter_fft(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                      cudaStream_t st);

template <typename Tin, typename Tout>
int launch_filter_step(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                       cudaStream_t st) {
  if (SKEI_STEP_FILTER == 1) return launch_filter_fft(p, in, rows, scale, out, st);
  if (SKEI_STEP_FILTER == 2) return launch_filter_tc(p, in, rows, scale, out, st);
  return launch_filter(p, in, rows, scale, out, st);
}

template <typename Tin, typename Tout>
int launch_filter_fft(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                      cudaStream_t st) {
  if (p->fft_len == 0) return launch_filter(p, in, rows, scale, out, st);
  const int L = p->fft_len;
  const size_t smem = (size_t)(L / 2 + 2 * L) * sizeof(float2);
  auto kern = ramlak_fft_kernel<Tin, Tout>;
  static size_t configured[64] = {0};
  SKEI_TRY(opt_in_smem(kern, smem, configured, "ramlak FFT: shared memory attribute"));
  launch_k(kern, dim3((rows + 1) / 2), dim3(kFftThreads), smem, st, in, out, rows, p->n_det, L,
           (const float *)p->d_hspec, scale);
  return check_launch("ramlak FFT filter launch");
}

template <typename Tin, typename Tout>
int launch_rotate(const Tin *x, int B, int N, const double *g_deg, int G, Tout *out,
                  cudaStream_t st, int Ch) {
  dim3 grid((N + kRotX - 1) / kRotX, (N + kRotY * kRotQ - 1) / (kRotY * kRotQ), B * G * Ch);
  launch_k(rotate_kernel<Tin, Tout>, grid, dim3(kRotThreads), 0, st, x, N, G, Ch, g_deg, out);
  return check_launch("rotation launch");
}

template <typename Tin, typename Tout>
int launch_rotate_adj(const Tin *gout, int B, int N, const double *g_deg, int G,
                      float alpha, float beta, Tout *gx, cudaStream_t st, int Ch) {
  dim3 grid((N + kAdjT - 1) / kAdjT, (N + kAdjT * kAdjQ - 1) / (kAdjT * kAdjQ), B * Ch);
  launch_k(rotate_adj_kernel<Tin, Tout>, grid, dim3(kAdjT, kAdjT), 0, st, gout, N, G, Ch,
           g_deg, alpha, beta, gx);
  return check_launch("rotation transpose launch");
}

template <typename T>
int launch_rotate_residual(const T *x0, const float *theta, int B, int N, const double *g_deg,
                           int G, T *x1, T *out, cudaStream_t st) {
  dim3 grid((N + kRotX - 1) / kRotX, (N + kRotY * kRotQ - 1) / (kRotY * kRotQ), B * G);
  launch_k(rotate_residual_kernel<T>, grid, dim3(kRotThreads), 0, st, x0, theta, N, G, g_deg, x1,
           out);
  return check_launch("residual rotation launch");
}

template <typename T>
int launch_rotate_adj_adam(const float *gout, int N, const double *g_deg, int G, T *gx,
                           const T *g_x3, const AdamArgs &adam, const LossFinal &lf,
                           cudaStream_t st) {
  dim3 grid((N + kAdjT - 1) / kAdjT, (N + kAdjT * kAdjQ - 1) / (kAdjT * kAdjQ), 1);
  const size_t smem = sizeof(double) * (size_t)(lf.B * lf.G + lf.B);
  // dynamic shared memory below 40 KB: with the kernel's static part, under the 48 KB default
  if (smem > 40 * 1024)
    return set_error(SKEI_EINVAL, "B*G + B = %d segments is too many", lf.B * lf.G + lf.B);
  launch_k(rotate_adj_adam_kernel<T>, grid, dim3(kAdjT, kAdjT), smem, st, gout, N, G, g_deg, gx,
           g_x3, adam, lf);
  return check_launch("rotation transpose + Adam launch");
}
template int launch_rotate_residual<float>(const float *, const float *, int, int,
                                           const double *, int, float *, float *, cudaStream_t);
template int launch_rotate_residual<__nv_bfloat16>(const __nv_bfloat16 *, const float *, int,
                                                   int, const double *, int, __nv_bfloat16 *,
                                                   __nv_bfloat16 *, cudaStream_t);
template int launch_rotate_adj_adam<float>(const float *, int, const double *, int, float *,
                                           const float *, const AdamArgs &, const LossFinal &,
                                           cudaStream_t);
template int launch_rotate_adj_adam<__nv_bfloat16>(const float *, int, const double *, int,
                                                   __nv_bfloat16 *, const __nv_bfloat16 *,
                                                   const AdamArgs &, const LossFinal &,
                                                   cudaStream_t);

#define SKEI_FR_INST(TI, TO)                                                                  \
  template int launch_filter<TI, TO>(skei_plan, const TI *, int, float, TO *, cudaStream_t);  \
  template int launch_filter_fft<TI, TO>(skei_plan, const TI *, int, float, TO *,             \
                                         cudaStream_t);                                      \
  template int launch_filter_step<TI, TO>(skei_plan, const TI *, int, float, TO *,            \
                                          cudaStream_t);                                     \
  template int launch_filter_tc<TI, TO>(skei_plan, const TI *, int, float, TO *,              \
                                        cudaStream_t);                                       \
  template int launch_rotate<TI, TO>(const TI *, int, int, const double *, int, TO *,         \
                                     cudaStream_t, int);                                     \
  template int launch_rotate_adj<TI, TO>(const TI *, int, int, const double *, int, float,    \
                                         float, TO *, cudaStream_t, int);
SKEI_FR_INST(float, float)
SKEI_FR_INST(__nv_bfloat16, __nv_bfloat16)
SKEI_FR_INST(float, __nv_bfloat16)
SKEI_FR_INST(__nv_bfloat16, float)
#undef SKEI_FR_INST

}  // namespace skei
