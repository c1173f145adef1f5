// Pixel-driven gathers over 32x32 image tiles: the exact transpose A_S^T of
// Joseph's projector (the gradient of the MC and EI terms, Algorithm 2) and
// the back-projection B_S of FBP (A_S^dagger = (pi/m) B_S H, Sec. 2.1 and
// 3.1).
//
// A CTA owns one tile of one image and walks the angle list in chunks; for
// each angle it stages in shared memory only the window of detector bins
// that the tile projects onto (at most ~50 bins).  Every thread accumulates
// 4 pixels in registers and writes each once, so no atomics are needed.
//
// A^T: pixel (L, P) (line, position) receives, for each angle, from the rays
// whose crossing with line L lies in (P-1, P+1) - at most 3 candidates
// around k = (P - G - L T) / A.  The crossing is recomputed exactly in the
// forward's fixed-point form and weighted with tap_weight(), so the gathered
// weights equal bitwise the forward's interpolation weights.
#include "common.cuh"

namespace skei {
namespace {

constexpr int kTile = 32;
constexpr int kRows = 8;   // thread rows; each thread owns kTile/kRows pixels
constexpr int kWin = 64;   // staged bins per angle
constexpr int kAC = 16;    // angles per chunk
constexpr int kThreads = kTile * kRows;

enum { OP_JOSEPH_ADJ = 0, OP_BACKPROJECT = 1 };

template <typename Tin, typename Tadd, typename Tout>
struct TileArgs {
  const Tin *sino;    // [B][m][n_det]
  const Tadd *add;    // [B][N][N] or null
  Tout *out;          // [B][N][N]
  const int *idx;
  int m, N, n_det, n_angles;
  float alpha, beta;
  const AngleConst *ang;
  int *status;
};

template <int OP, typename Tin, typename Tadd, typename Tout>
__global__ void __launch_bounds__(kThreads)
    tile_kernel(const TileArgs<Tin, Tadd, Tout> args) {
  __shared__ float win[kAC][kWin];
  __shared__ AngleConst sc[kAC];
  __shared__ long long c0w[kAC];   // Joseph: G + kw0 A, the window's first ray at line 0
  __shared__ int sai[kAC];
  __shared__ int kw0[kAC];

  const int tid = threadIdx.x;
  const int tx = tid % kTile, ty = tid / kTile;
  const int N = args.N, nd = args.n_det;
  const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
  const int b = blockIdx.z;
  const int i_last = min(i0 + kTile, N) - 1, j_last = min(j0 + kTile, N) - 1;

  float acc[kTile / kRows];
#pragma unroll
  for (int q = 0; q < kTile / kRows; ++q) acc[q] = 0.0f;
  const int j = j0 + tx;
  const float fj = (float)j;

  for (int c0 = 0; c0 < args.m; c0 += kAC) {
    const int nac = min(kAC, args.m - c0);
    __syncthreads();  // previous chunk no longer read
    if (tid < nac) {
      int ai = args.idx ? args.idx[c0 + tid] : c0 + tid;
      if (ai < 0 || ai >= args.n_angles) {
        if (blockIdx.x == 0 && blockIdx.y == 0) atomicOr(args.status, 1);
        ai = -1;
      }
      sai[tid] = ai;
      if (ai >= 0) {
        const AngleConst C = args.ang[ai];
        sc[tid] = C;
        // bin range of the tile: extremes of an affine function at corners
        float lo = 3.0e38f;
        for (int ci = 0; ci < 2; ++ci)
          for (int cj = 0; cj < 2; ++cj) {
            const float fi_ = (float)(ci ? i_last : i0), fj_ = (float)(cj ? j_last : j0);
            const float L = C.mode ? fi_ : fj_, Pp = C.mode ? fj_ : fi_;
            float v;
            if (OP == OP_JOSEPH_ADJ) v = (Pp - fmaf(L, C.Tf, C.Gf)) * C.invA;
            else v = fmaf(Pp, C.bstepf, fmaf(L, C.blinef, C.t00f));
            lo = fminf(lo, v);
          }
        const int k0 = (int)floorf(lo) - (OP == OP_JOSEPH_ADJ ? 2 : 1);
        kw0[tid] = k0;
        c0w[tid] = C.G + (long long)k0 * C.A;
      }
    }
    __syncthreads();
    for (int e = tid; e < nac * kWin; e += kThreads) {
      const int a = e / kWin, w = e - a * kWin;
      const int ai = sai[a];
      float v = 0.0f;
      if (ai >= 0) {
        const int k = kw0[a] + w;
        if (k >= 0 && k < nd) {
          v = ldg_f(args.sino + ((size_t)b * args.m + c0 + a) * nd + k);
          if (OP == OP_JOSEPH_ADJ) v *= sc[a].W;
        }
      }
      win[a][w] = v;
    }
    __syncthreads();

    for (int a = 0; a < nac; ++a) {
      if (sai[a] < 0) continue;
      const AngleConst &C = sc[a];
      const int base = kw0[a];
      const float *wa = win[a];
      if (OP == OP_JOSEPH_ADJ) {
        const long long A = C.A, T = C.T;
        const long long c0 = c0w[a];
#pragma unroll
        for (int q = 0; q < kTile / kRows; ++q) {
          const int i = i0 + ty + kRows * q;
          const int L = C.mode ? i : j, Pp = C.mode ? j : i;
          const float kc = ((float)Pp - fmaf((float)L, C.Tf, C.Gf)) * C.invA;
          int r = round_int(kc) - 1 - base;       // window slot of the first candidate
          r = min(max(r, 0), kWin - 3);
          long long pos = c0 + (long long)r * A + (long long)L * T;
          float s = acc[q];
          s = fmaf(tap_weight(pos, Pp), wa[r], s);
          pos += A;
          s = fmaf(tap_weight(pos, Pp), wa[r + 1], s);
          pos += A;
          s = fmaf(tap_weight(pos, Pp), wa[r + 2], s);
          acc[q] = s;
        }
      } else {
        const long long step = C.ti * kRows;
        long long t = C.t00 + (long long)j * C.tj + (long long)(i0 + ty) * C.ti;
#pragma unroll
        for (int q = 0; q < kTile / kRows; ++q) {
          int k0 = ipart(t) - base;
          k0 = min(max(k0, 0), kWin - 2);
          const float w = frac23(t);
          const float v0 = wa[k0], v1 = wa[k0 + 1];
          acc[q] += fmaf(w, v1 - v0, v0);
          t += step;
        }
      }
    }
  }

  if (j >= N) return;
#pragma unroll
  for (int q = 0; q < kTile / kRows; ++q) {
    const int i = i0 + ty + kRows * q;
    if (i >= N) continue;
    const size_t o = ((size_t)b * N + i) * N + j;
    float v = args.alpha * acc[q];
    if (args.beta != 0.0f && args.add) v = fmaf(args.beta, ldg_f(args.add + o), v);
    st_f(args.out + o, v);
  }
}

template <int OP, typename Tin, typename Tadd, typename Tout>
int launch_tile(skei_plan p, const Tin *sino, int B, const int *idx, int m, float alpha,
                float beta, const Tadd *add, Tout *out, cudaStream_t st) {
  TileArgs<Tin, Tadd, Tout> a{sino, add, out, idx, m, p->N, p->n_det, p->n_angles,
                              alpha, beta, p->d_ang, p->d_status};
  dim3 grid((p->N + kTile - 1) / kTile, (p->N + kTile - 1) / kTile, B);
  tile_kernel<OP, Tin, Tadd, Tout><<<grid, kThreads, 0, st>>>(a);
  return check_launch(OP == OP_JOSEPH_ADJ ? "joseph adjoint launch" : "back-projection launch");
}

}  // namespace

template <typename Tin, typename Tadd, typename Tout>
int launch_proj_adj(skei_plan p, const Tin *sino, int B, const int *idx, int m,
                    float alpha, float beta, const Tadd *add, Tout *out, cudaStream_t st) {
  return launch_tile<OP_JOSEPH_ADJ>(p, sino, B, idx, m, alpha, beta, add, out, st);
}

template <typename Tin, typename Tadd, typename Tout>
int launch_backproject(skei_plan p, const Tin *q, int B, const int *idx, int m,
                       float alpha, float beta, const Tadd *add, Tout *out, cudaStream_t st) {
  return launch_tile<OP_BACKPROJECT>(p, q, B, idx, m, alpha, beta, add, out, st);
}

#define SKEI_TILE_INST(TI, TA, TO)                                                           \
  template int launch_proj_adj<TI, TA, TO>(skei_plan, const TI *, int, const int *, int,     \
                                           float, float, const TA *, TO *, cudaStream_t);    \
  template int launch_backproject<TI, TA, TO>(skei_plan, const TI *, int, const int *, int,  \
                                              float, float, const TA *, TO *, cudaStream_t);
SKEI_TILE_INST(float, float, float)
SKEI_TILE_INST(__nv_bfloat16, __nv_bfloat16, __nv_bfloat16)
SKEI_TILE_INST(float, __nv_bfloat16, float)
SKEI_TILE_INST(float, __nv_bfloat16, __nv_bfloat16)
#undef SKEI_TILE_INST

}  // namespace skei
