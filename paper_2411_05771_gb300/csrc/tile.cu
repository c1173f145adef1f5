// Pixel-driven gathers over 8 x 128 image tiles: the exact transpose A_S^T
// of Joseph's projector (the gradient of the MC and EI terms, Algorithm 2)
// and the back-projection B_S of FBP (A_S^dagger = (pi/m) B_S H, Sec. 2.1
// and 3.1).
//
// A CTA owns one tile of a group of images (one warp per tile row; a thread
// holds 4 pixels 32 columns apart, so that neighbouring lanes read
// neighbouring bins, free of shared-memory bank conflicts, and the warp
// stores 32 consecutive pixels at a time) and walks the angle list in chunks; for
// each angle it stages in shared memory only the window of detector bins
// the tile projects onto.  Every thread accumulates its pixels in registers
// and writes each once: no atomics.  Up to two jobs share a launch (grid.z
// spans the image groups of both), e.g. the MC-term and EI-term adjoints of
// one SkEI step.
//
// Image groups: the images of a job share its angle list, so a pixel's
// rays, bins and weights are the same for all of them.  A group of 4 images
// computes them once and reads the 4 images' bins with one 16-byte load
// (the window holds [bin][image]); jobs whose image count is not a multiple
// of 4 finish with single-image groups.  When both jobs of a launch use the
// same angle list and the second has 4 images per image of the first (the
// MC and EI terms of a step with G = 4), each CTA carries one image of the
// first job along with a group of the second.  Each image sees the same
// sequence of operations in every form.
//
// A^T: pixel (L, P) (line, position) receives, for each angle, from the two
// rays whose crossing with line L has integer part P (weight 1-f) and P-1
// (weight f).  With u = P - G - L T and r the ray nearest to P
// (r = round(u / A)), the exact fixed-point offset D = pos(L, r) - P =
// r A - u lies in (-1, 1); its sign says whether r is the "1-f" or the "f"
// ray, and the other one is r's neighbour on the opposite side, at
// D -+ |A|.  Both offsets are small, so they are exact in 32-bit wrapping
// arithmetic on the low words of the fixed-point values, and their 23-bit
// fractions are bitwise the forward's interpolation weights.
#include "common.cuh"

namespace skei {
namespace {

// Build-time tuning knobs: the largest tile height (rows, <= 8; a launch
// picks between 4 and this to balance its CTAs over the SMs, the batch
// kernel uses it as is); angle split (1 or 2): with 2 (measured faster for
// B on GB300), two warps share each tile row, taking alternate angles of
// every chunk, and their sums are added in a fixed order at the end;
// pixels per thread (4: 8 measured slower at 96 registers, one CTA per SM);
// angles per chunk (16: half the chunk barriers of 8, measured faster at
// 512^2 with 30 angles; 4 slower).
#ifndef SKEI_TILE_ROWS
#define SKEI_TILE_ROWS 8
#endif
#ifndef SKEI_TILE_SPLIT
#define SKEI_TILE_SPLIT 2
#endif
#ifndef SKEI_TILE_PPT
#define SKEI_TILE_PPT 4
#endif
#ifndef SKEI_TILE_AC
#define SKEI_TILE_AC 16
#endif

constexpr int kPPT = SKEI_TILE_PPT;      // pixels per thread, 32 columns apart
constexpr int kTW = 32 * kPPT;           // tile width (columns)
constexpr int kTH = SKEI_TILE_ROWS;      // tile height (rows)
constexpr int kSplit = SKEI_TILE_SPLIT;  // warps per tile row
constexpr int kThreads = 32 * kTH * kSplit;
constexpr int kWin = kTW + 32;           // staged bins per angle (>= kTW + kTH + 6)
constexpr int kAC = SKEI_TILE_AC;        // angles per chunk

struct TileArgs {
  Jobs jobs;
  int N, n_det, n_angles;
  const AngleConst *ang;
  int *status;
  int merge;   // job 0's image b rides with job 1's group 4b .. 4b+3 (same angles)
  int gmax[kMaxJobs];   // image group size per job (4, or 1 where groups would
                        // straddle the per-sample angle lists)
};

// Shared memory of a tile task (dynamic: above the 48 KB of static shared
// memory): two windows, each the bins of kAC angles for up to 4 images,
// [angle][bin][image], and three slots of chunk constants.  Chunk c is
// computed from window c % 2 while window c+1 fills by cp.async and the
// constants of chunk c+2 are set up.
struct TileSmem {
  alignas(16) float win[2][kAC * kWin * 4];
  float winx[2][kAC * kWin];   // the bins of a riding image of another job
  AngleConst sc[3][kAC];
  int sai[3][kAC];
  int kw0[3][kAC];
};
constexpr size_t kTileSmem = sizeof(TileSmem);

// Constants of chunk c (angles c0 .. c0 + nac - 1 of J's list) into slot
// `slot`: angle index (or -1 if out of range, reported), its AngleConst and
// the first bin of the window the tile projects onto.  Threads 0 .. nac-1.
template <int OP>
__device__ __forceinline__ void tile_setup(const Job &J, int b0, int c0, int nac, int i0, int j0,
                                           int i_last, int j_last, int n_angles,
                                           const AngleConst *ang, int *status, bool report,
                                           TileSmem &sm, int slot) {
  const int tid = threadIdx.x;
  if (tid >= nac) return;
  const int *idx = job_idx(J, b0);
  int ai = idx ? idx[c0 + tid] : c0 + tid;
  if (ai < 0 || ai >= n_angles) {
    if (report) atomicOr(status, 1);
    ai = -1;
  }
  sm.sai[slot][tid] = ai;
  if (ai < 0) return;
  const AngleConst C = ang[ai];
  sm.sc[slot][tid] = C;
  // bin range of the tile: extremes of an affine function at corners
  float lo = 3.0e38f;
  for (int ci = 0; ci < 2; ++ci)
    for (int cj = 0; cj < 2; ++cj) {
      const float fi_ = (float)(ci ? i_last : i0), fj_ = (float)(cj ? j_last : j0);
      const float L = C.mode ? fi_ : fj_, Pp = C.mode ? fj_ : fi_;
      float v;
      if (OP == OP_JOSEPH_ADJ) v = (Pp - fmaf(L, C.Tf, C.Gf)) * C.invA;
      else v = fmaf(fj_, C.tjf, fmaf(fi_, C.tif, C.t00f));
      lo = fminf(lo, v);
    }
  sm.kw0[slot][tid] = (int)floorf(lo) - 3;
}

// Window of chunk c (constants in `slot`) into window buffer `wb`, the
// group's images side by side; bins outside the sinogram and dead angles
// read as 0.  A warp fills runs of 32 bins of one angle at a time, so that
// the angle's row addresses are computed once per run.  FP32 inputs are
// copied by cp.async (the caller waits, then synchronises the CTA); BF16
// inputs are converted and stored.
template <int NI, bool XTRA>
__device__ __forceinline__ void tile_window(const Job &J, int b0, int c0, int nac, int nd,
                                            TileSmem &sm, int slot, int wb, const Job *JX,
                                            int bx) {
  constexpr int kRuns = (kWin + 31) / 32;   // runs of 32 bins per angle
  // FP32 inputs by cp.async, BF16 ones through registers (a riding BF16
  // image does not hold back the group's copies)
  const bool async = !J.in_bf16, asyncx = XTRA && !JX->in_bf16;
  float *win = sm.win[wb], *winx = sm.winx[wb];
  const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int u = threadIdx.x >> 5; u < nac * kRuns; u += nwarps) {
    const int a = u / kRuns, w = (u - a * kRuns) * 32 + lane;   // a is warp-uniform
    if (w >= kWin) continue;
    const int k = sm.kw0[slot][a] + w;
    const bool ok = sm.sai[slot][a] >= 0 && k >= 0 && k < nd;
    const int kk = ok ? k : 0;
    const size_t row = ((size_t)b0 * J.m + c0 + a) * nd;     // image b0's row of angle a
    const size_t img = (size_t)J.m * nd;                      // one image's rows
    // interleaved input: the group's 4 values of bin k at il(k)
    auto il = [&](int k) {
      return ((((size_t)(b0 >> 2) * J.m + c0 + a) * nd + k) << 2) + (b0 & 3);
    };
    const size_t rowx = XTRA ? ((size_t)bx * JX->m + c0 + a) * nd : 0;
    const int e = a * kWin + w;
    if (SKEI_CHECK) {
      // every window slot this thread fills lies in shared memory, and every
      // bin it reads in the job's input
      bool in = ck_smem(win + e * NI, 4 * NI, CK_TILE_WIN) &&
                (!XTRA || ck_smem(winx + e, 4, CK_TILE_WIN));
      if (ok) {
        in = in && ck(J.in_il4 ? (long long)(il(kk) + NI - 1)
                               : (long long)(row + (NI - 1) * img + kk),
                      (long long)J.nimg * img, CK_TILE_IN);
        if (XTRA)
          in = in && ck((long long)(rowx + kk), (long long)JX->nimg * JX->m * nd, CK_TILE_IN);
      }
      if (!in) continue;
    }
    if (async && J.in_il4) {
      const float *src = static_cast<const float *>(J.in) + il(kk);
      if (NI == 4) cp_async16(win + e * 4, src, ok);
      else cp_async4(win + e * NI, src, ok);
    } else if (async) {
      const float *src = static_cast<const float *>(J.in) + row + kk;
#pragma unroll
      for (int n = 0; n < NI; ++n) cp_async4(win + e * NI + n, src + n * img, ok);
    } else {
#pragma unroll
      for (int n = 0; n < NI; ++n)
        win[e * NI + n] = ok ? ld_any(J.in, row + n * img + k, J.in_bf16) : 0.0f;
    }
    if (asyncx) cp_async4(winx + e, static_cast<const float *>(JX->in) + rowx + kk, ok);
    else if (XTRA) winx[e] = ok ? ld_any(JX->in, rowx + k, JX->in_bf16) : 0.0f;
  }
  cp_async_commit();
}

// One task: the tile at (i0, j0) of images b0 .. b0 + NI - 1 of job J;
// with XTRA, also image bx of job JX, whose angle list is J's: it shares
// the pixels' rays and weights and costs only its own taps.
template <int OP, int NI, bool XTRA = false>
__device__ __forceinline__ void tile_task(const Job &J, int b0, int i0, int j0, int N, int nd,
                                          int n_angles, const AngleConst *ang, int *status,
                                          bool report, TileSmem &sm, const Job *JX = nullptr,
                                          int bx = 0) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int th = blockDim.x / (32 * kSplit);  // tile rows of this launch (<= kTH)
  const int half = warp / th;              // which angles of each chunk
  const int i_last = min(i0 + th, N) - 1, j_last = min(j0 + kTW, N) - 1;
  const int i = i0 + warp % th;            // this thread's row
  const int jb = j0 + lane;                // its first column; then every 32nd

  float acc[NI][kPPT], accx[kPPT];
#pragma unroll
  for (int n = 0; n < NI; ++n)
#pragma unroll
    for (int q = 0; q < kPPT; ++q) acc[n][q] = 0.0f;
#pragma unroll
  for (int q = 0; q < kPPT; ++q) accx[q] = 0.0f;

  const int nch = (J.m + kAC - 1) / kAC;
  tile_setup<OP>(J, b0, 0, min(kAC, J.m), i0, j0, i_last, j_last, n_angles, ang, status, report,
                 sm, 0);
  if (nch > 1)
    tile_setup<OP>(J, b0, kAC, min(kAC, J.m - kAC), i0, j0, i_last, j_last, n_angles, ang,
                   status, report, sm, 1);
  __syncthreads();
  tile_window<NI, XTRA>(J, b0, 0, min(kAC, J.m), nd, sm, 0, 0, JX, bx);

  for (int c = 0; c < nch; ++c) {
    const int c0 = c * kAC, nac = min(kAC, J.m - c0), slot = c % 3;
    cp_async_wait_all();
    __syncthreads();  // window c and the constants of chunk c+1 are in place
    if (c + 1 < nch)
      tile_window<NI, XTRA>(J, b0, c0 + kAC, min(kAC, J.m - c0 - kAC), nd, sm, (c + 1) % 3,
                            (c + 1) & 1, JX, bx);
    if (c + 2 < nch)
      tile_setup<OP>(J, b0, c0 + 2 * kAC, min(kAC, J.m - c0 - 2 * kAC), i0, j0, i_last, j_last,
                     n_angles, ang, status, report, sm, (c + 2) % 3);

    for (int a = half; a < nac; a += kSplit) {
      if (sm.sai[slot][a] < 0) continue;
      const AngleConst &C = sm.sc[slot][a];
      const float *wa = sm.win[c & 1] + a * kWin * NI;
      const float *wx = sm.winx[c & 1] + a * kWin;
      const int base = sm.kw0[slot][a];
      if (OP == OP_JOSEPH_ADJ) {
        const bool row = C.mode != 0;
        const long long A = C.A, T = C.T, G = C.G;
        const unsigned A32 = (unsigned)A;
        const int absA32 = (int)(unsigned)(A < 0 ? -A : A);
        const int sA = A < 0 ? -1 : 1;
        const float Tf = C.Tf, Gf = C.Gf, invA = C.invA, W = C.W;
        // u = P - G - L T for the first pixel (low word; exact modulo 2^32);
        // per column along the row, row mode (P = j) adds 1, column mode
        // (L = j) subtracts T; the thread's pixels are 32 columns apart
        const int L0 = row ? i : jb, P0 = row ? jb : i;
        unsigned u = (unsigned)(((long long)P0 << kFxBits) - G - (long long)L0 * T);
        const unsigned du = 32u * (row ? (unsigned)kFxOne : (unsigned)(-T));
        const float kc0 = ((float)P0 - fmaf((float)L0, Tf, Gf)) * invA;
        const float dkc = 32.0f * (row ? invA : -Tf * invA);
#pragma unroll
        for (int q = 0; q < kPPT; ++q) {
          const int r = round_int(fmaf((float)q, dkc, kc0));
          const int D = (int)((unsigned)r * A32 - u);   // pos(L, r) - P, in (-1, 1)
          const bool right = D >= 0;                     // r is the "1-f" ray
          const int D2 = right ? D - absA32 : D + absA32;
          // window slots; the tile's bins lie inside the window by
          // construction, the clamp only bounds the read
          const int s1 = min(max(r - base, 1), kWin - 2);
          const int s2 = s1 + (right ? -sA : sA);
          // tap weights times the angle's W (the bins are staged unscaled):
          // with x = 2 - |a| 2^-23, the weight x - 1 is exact, so one FMA
          // W x - W rounds W (x - 1) once, as the product would (W > 0)
          const float w1 = fmaf(W, __int_as_float(0x40000000 - abs(D >> (kFxBits - 23))), -W);
          const float w2 =
              fmaxf(fmaf(W, __int_as_float(0x40000000 - abs(D2 >> (kFxBits - 23))), -W), 0.0f);
          if (NI == 4) {
            const float4 v1 = lds_ck(reinterpret_cast<const float4 *>(wa) + s1, CK_TILE_TAP);
            const float4 v2 = lds_ck(reinterpret_cast<const float4 *>(wa) + s2, CK_TILE_TAP);
            acc[0][q] = fmaf(w1, v1.x, fmaf(w2, v2.x, acc[0][q]));
            acc[1][q] = fmaf(w1, v1.y, fmaf(w2, v2.y, acc[1][q]));
            acc[2][q] = fmaf(w1, v1.z, fmaf(w2, v2.z, acc[2][q]));
            acc[3][q] = fmaf(w1, v1.w, fmaf(w2, v2.w, acc[3][q]));
          } else {
            acc[0][q] = fmaf(w1, lds_ck(wa + s1, CK_TILE_TAP),
                             fmaf(w2, lds_ck(wa + s2, CK_TILE_TAP), acc[0][q]));
          }
          if (XTRA)
            accx[q] = fmaf(w1, lds_ck(wx + s1, CK_TILE_TAP),
                           fmaf(w2, lds_ck(wx + s2, CK_TILE_TAP), accx[q]));
          u += du;
        }
      } else {
        // t(i, j) = t00 + j tj + i ti, stepping along the row by 32 tj
        long long t = C.t00 + (long long)jb * C.tj + (long long)i * C.ti;
        const long long tj = 32 * C.tj;
#pragma unroll
        for (int q = 0; q < kPPT; ++q) {
          int k0 = ipart(t) - base;
          k0 = min(max(k0, 0), kWin - 2);
          const float w = frac23(t);
          const float g = 1.0f - w;
          if (NI == 4) {
            const float4 v0 = lds_ck(reinterpret_cast<const float4 *>(wa) + k0, CK_TILE_TAP);
            const float4 v1 = lds_ck(reinterpret_cast<const float4 *>(wa) + k0 + 1, CK_TILE_TAP);
            acc[0][q] = fmaf(w, v1.x, fmaf(g, v0.x, acc[0][q]));
            acc[1][q] = fmaf(w, v1.y, fmaf(g, v0.y, acc[1][q]));
            acc[2][q] = fmaf(w, v1.z, fmaf(g, v0.z, acc[2][q]));
            acc[3][q] = fmaf(w, v1.w, fmaf(g, v0.w, acc[3][q]));
          } else {
            acc[0][q] = fmaf(w, lds_ck(wa + k0 + 1, CK_TILE_TAP),
                             fmaf(g, lds_ck(wa + k0, CK_TILE_TAP), acc[0][q]));
          }
          if (XTRA)
            accx[q] = fmaf(w, lds_ck(wx + k0 + 1, CK_TILE_TAP),
                           fmaf(g, lds_ck(wx + k0, CK_TILE_TAP), accx[q]));
          t += tj;
        }
      }
    }
  }

  if (kSplit > 1) {
    // the second half's sums through shared memory (the window is free)
    __syncthreads();
    float *red = sm.win[0];
    const int t0 = tid % (32 * th);
    if (half == 1) {
#pragma unroll
      for (int n = 0; n < NI; ++n)
#pragma unroll
        for (int q = 0; q < kPPT; ++q) red[(n * kPPT + q) * 32 * th + t0] = acc[n][q];
      if (XTRA)
#pragma unroll
        for (int q = 0; q < kPPT; ++q) sm.winx[0][q * 32 * th + t0] = accx[q];
    }
    __syncthreads();
    if (half != 0) return;
#pragma unroll
    for (int n = 0; n < NI; ++n)
#pragma unroll
      for (int q = 0; q < kPPT; ++q) acc[n][q] += red[(n * kPPT + q) * 32 * th + t0];
    if (XTRA)
#pragma unroll
      for (int q = 0; q < kPPT; ++q) accx[q] += sm.winx[0][q * 32 * th + t0];
  }
  if (i >= N) return;
  // pixel q of the thread is column jb + 32 q: a warp stores 32 consecutive
  // pixels per q
#pragma unroll
  for (int n = 0; n < NI; ++n) {
    const size_t o = ((size_t)(b0 + n) * N + i) * N + jb;
#pragma unroll
    for (int q = 0; q < kPPT; ++q) {
      if (jb + 32 * q >= N) break;
      if (SKEI_CHECK && !ck((long long)(o + 32 * q), (long long)J.nimg * N * N, CK_TILE_OUT))
        continue;
      float v = J.alpha * acc[n][q];
      if (J.beta != 0.0f && J.aux) v = fmaf(J.beta, ld_any(J.aux, o + 32 * q, J.aux_bf16), v);
      st_any(J.out, o + 32 * q, v, J.out_bf16);
      if (J.out2) {
        // the value as stored, then the residual: what a separate
        // out + add2 pass would read and write
        const float vs = J.out_bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
        st_any(J.out2, o + 32 * q, vs + __ldg(J.add2 + (size_t)i * N + jb + 32 * q),
               J.out2_bf16);
      }
    }
  }
  if (XTRA) {
    const size_t o = ((size_t)bx * N + i) * N + jb;
#pragma unroll
    for (int q = 0; q < kPPT; ++q) {
      if (jb + 32 * q >= N) break;
      if (SKEI_CHECK && !ck((long long)(o + 32 * q), (long long)JX->nimg * N * N, CK_TILE_OUT))
        continue;
      float v = JX->alpha * accx[q];
      if (JX->beta != 0.0f && JX->aux) v = fmaf(JX->beta, ld_any(JX->aux, o + 32 * q, JX->aux_bf16), v);
      st_any(JX->out, o + 32 * q, v, JX->out_bf16);
    }
  }
}

template <int OP>
// two CTAs per SM: at most 64 registers
__global__ void __launch_bounds__(kThreads, 2) tile_kernel(const TileArgs args) {
  pdl_enter();
  extern __shared__ float4 tile_smem4[];
  TileSmem &sm = *reinterpret_cast<TileSmem *>(tile_smem4);
  const int z = blockIdx.z;
  const int th = blockDim.x / (32 * kSplit);   // tile rows chosen by the launch
  const bool report = blockIdx.x == 0 && blockIdx.y == 0;
  if (args.merge) {
    // group z of job 1 (images 4z .. 4z+3) with image z of job 0
    tile_task<OP, 4, true>(args.jobs.j[1], 4 * z, blockIdx.y * th, blockIdx.x * kTW, args.N,
                           args.n_det, args.n_angles, args.ang, args.status, report, sm,
                           &args.jobs.j[0], z);
    return;
  }
  const int g0 = n_groups(args.jobs.j[0].nimg, args.gmax[0]);
  const int jn = (args.jobs.njobs > 1 && z >= g0) ? 1 : 0;
  const Job &J = args.jobs.j[jn];
  int b0, ni;
  group_at(J.nimg, z - (jn ? g0 : 0), &b0, &ni, args.gmax[jn]);
  if (ni == 4)
    tile_task<OP, 4>(J, b0, blockIdx.y * th, blockIdx.x * kTW, args.N, args.n_det,
                     args.n_angles, args.ang, args.status, report, sm);
  else
    tile_task<OP, 1>(J, b0, blockIdx.y * th, blockIdx.x * kTW, args.N, args.n_det,
                     args.n_angles, args.ang, args.status, report, sm);
}

// Persistent form over the tile tasks of a batch of instances: each CTA takes
// the next task from a global counter (tasks come in decreasing cost order)
// until none is left.  Task = (item, b0 << 3 | group size, tile row, tile
// column).
// CTAs per SM the registers of the persistent tile kernel allow (2: a few
// bytes of spills, measured faster than 1 CTA of 96 registers)
#ifndef SKEI_TILE_BATCH_MINB
#define SKEI_TILE_BATCH_MINB 2
#endif
template <int OP>
__global__ void __launch_bounds__(kThreads, SKEI_TILE_BATCH_MINB)
    tile_batch_kernel(const BatchItem *items, const int4 *tasks, int n_tasks, int *queue) {
  extern __shared__ float4 tile_smem4[];
  TileSmem &sm = *reinterpret_cast<TileSmem *>(tile_smem4);
  __shared__ int s_task;
  for (;;) {
    __syncthreads();  // the previous task's reads of s_task and shared memory are done
    if (threadIdx.x == 0) s_task = atomicAdd(queue, 1);
    __syncthreads();
    const int t = s_task;
    if (t >= n_tasks) break;
    const int4 tk = tasks[t];
    const BatchItem &it = items[tk.x];
    const Job J{it.in, nullptr, it.out, it.idx, it.m, it.B, it.alpha, 0.0f,
                it.in_bf16, 0, it.out_bf16};
    const int b0 = tk.y >> 3, ni = tk.y & 7;
    const bool report = tk.z == 0 && tk.w == 0;
    if (ni == 4)
      tile_task<OP, 4>(J, b0, tk.z * kTH, tk.w * kTW, it.N, it.n_det, it.n_angles, it.ang,
                       it.status, report, sm);
    else
      tile_task<OP, 1>(J, b0, tk.z * kTH, tk.w * kTW, it.N, it.n_det, it.n_angles, it.ang,
                       it.status, report, sm);
  }
  if (threadIdx.x == 0) queue_retire(queue, gridDim.x);
}

// Opts a tile kernel in to its dynamic shared memory, once per device.
template <typename K>
int set_tile_smem(K kern, size_t *configured) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (configured[dev] < kTileSmem) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    if (e != cudaSuccess) return cuda_error(e, "tile kernel: shared memory attribute");
    configured[dev] = kTileSmem;
  }
  return SKEI_OK;
}
template <int OP>
int set_tile_kernel_smem() {
  static size_t configured[64] = {0};
  return set_tile_smem(tile_kernel<OP>, configured);
}
template <int OP>
int set_tile_batch_smem() {
  static size_t configured[64] = {0};
  return set_tile_smem(tile_batch_kernel<OP>, configured);
}

template <int OP>
int launch_tile(skei_plan p, const Jobs &jobs, cudaStream_t st) {
  int gmax[kMaxJobs] = {4, 4};
  int ngroups = 0;
  for (int q = 0; q < jobs.njobs; ++q) {
    gmax[q] = job_groupable(jobs.j[q]) ? 4 : 1;
    ngroups += n_groups(jobs.j[q].nimg, gmax[q]);
  }
  // two jobs over the same angle lists with 4 images of job 1 per image of
  // job 0 (the MC and EI terms of a step, G = 4): one CTA carries both;
  // with a list per sample, image b of job 0 and images 4b .. 4b+3 of job 1
  // must read the same row
  const Job &j0 = jobs.j[0], &j1 = jobs.j[1];
  const int merge = jobs.njobs == 2 && gmax[1] == 4 && j0.idx == j1.idx && j0.m == j1.m &&
                    j1.nimg == 4 * j0.nimg &&
                    ((j0.idx_per <= 0 && j1.idx_per <= 0) ||
                     (j0.idx_per > 0 && j1.idx_per == 4 * j0.idx_per));
  if (merge) ngroups = jobs.j[0].nimg;
  if (ngroups > 65535) return set_error(SKEI_EINVAL, "too many images in one launch");
  TileArgs a{jobs, p->N, p->n_det, p->n_angles, p->d_ang, p->d_status, merge,
             {gmax[0], gmax[1]}};
  // tile rows th <= kTH: the fewest CTA rounds per SM times the rows each
  // CTA covers (measured on GB300: 7 rows at 512^2, i.e. 296 CTAs for 304
  // slots, beat 8 rows' 256 CTAs by 8 %)
  const int cols = (p->N + kTW - 1) / kTW;
  int th = kTH;
  long long best = -1;
  for (int t = kTH; t >= 4; --t) {
    const long long ctas = (long long)cols * ((p->N + t - 1) / t) * ngroups;
    const long long cost = (ctas + sm_count() - 1) / sm_count() * t;
    if (best < 0 || cost < best) {
      best = cost;
      th = t;
    }
  }
  dim3 grid(cols, (p->N + th - 1) / th, ngroups);
  SKEI_TRY(set_tile_kernel_smem<OP>());
  launch_k(tile_kernel<OP>, grid, dim3(32 * th * kSplit), kTileSmem, st, a);
  return check_launch(OP == OP_JOSEPH_ADJ ? "joseph adjoint launch" : "back-projection launch");
}

}  // namespace

SKEI_CHECK_READER(check_read_tile)

int launch_tile_jobs(skei_plan p, int op, const Jobs &jobs, cudaStream_t st) {
  if (op == OP_JOSEPH_ADJ) return launch_tile<OP_JOSEPH_ADJ>(p, jobs, st);
  if (op == OP_BACKPROJECT) return launch_tile<OP_BACKPROJECT>(p, jobs, st);
  return set_error(SKEI_EINVAL, "tile launch: unknown operator %d", op);
}

void tile_batch_shape(int *rows, int *cols) {
  *rows = kTH;
  *cols = kTW;
}

int tile_batch_occupancy(int op, int *ctas_per_sm) {
  if (op == OP_JOSEPH_ADJ) SKEI_TRY(set_tile_batch_smem<OP_JOSEPH_ADJ>());
  else SKEI_TRY(set_tile_batch_smem<OP_BACKPROJECT>());
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &n, op == OP_JOSEPH_ADJ ? tile_batch_kernel<OP_JOSEPH_ADJ> : tile_batch_kernel<OP_BACKPROJECT>,
      kThreads, kTileSmem);
  if (e != cudaSuccess) return cuda_error(e, "tile kernel: occupancy");
  *ctas_per_sm = n > 0 ? n : 1;
  return SKEI_OK;
}

int launch_tile_batch_op(int op, const BatchItem *items, const int4 *tasks, int n_tasks,
                         int ctas, int *queue, cudaStream_t st) {
  if (op == OP_JOSEPH_ADJ) {
    SKEI_TRY(set_tile_batch_smem<OP_JOSEPH_ADJ>());
    tile_batch_kernel<OP_JOSEPH_ADJ><<<ctas, kThreads, kTileSmem, st>>>(items, tasks, n_tasks,
                                                                          queue);
  } else if (op == OP_BACKPROJECT) {
    SKEI_TRY(set_tile_batch_smem<OP_BACKPROJECT>());
    tile_batch_kernel<OP_BACKPROJECT><<<ctas, kThreads, kTileSmem, st>>>(items, tasks, n_tasks,
                                                                           queue);
  } else
    return set_error(SKEI_EINVAL, "tile batch: unknown operator %d", op);
  return check_launch(op == OP_JOSEPH_ADJ ? "batched joseph adjoint launch"
                                          : "batched back-projection launch");
}

}  // namespace skei
