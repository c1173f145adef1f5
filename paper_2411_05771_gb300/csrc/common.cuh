// Internal definitions shared by the kernels of libskei (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "skei.h"

namespace skei {

// Per-angle constants, derived in FP64 on the host.  Positions are kept in
// 32.32 fixed point (int64: integer part in the high word, fraction in the
// low word), so that every kernel evaluates them EXACTLY, in any order:
// forward operators and their gathered transposes then see bitwise the same
// positions and interpolation weights, and the weights are accurate to
// ~1e-7 (FP32 positions near 512 would only be good to ~3e-5).
//
// Joseph's projector (Sec. 4.1.1, discrete Radon transform): ray k crosses
// "line" L (an image row in row mode, a column in column mode) at
//     pos(L, k) = G + k A + L T                      (fixed point)
// and the sample is the linear interpolation between positions floor(pos)
// and floor(pos)+1 of that line; the ray sum is multiplied by
// W = 1/|cos| (1/|sin|).
//
// Pixel-driven back-projection (the B of FBP): pixel (i, j) lands on bin
//     t(i, j) = t00 + j tj + i ti                    (fixed point)
// and B_S^T walks lines L with position P: (L, P) = (i, j) in row mode,
// (j, i) in column mode, i.e. t = t00 + L bline + P bstep.
struct AngleConst {
  long long T, A, G;             // Joseph, 32.32
  long long t00, bline, bstep;   // back-projection, 32.32
  long long tj, ti;              // back-projection per column / per row, 32.32
  float Tf, Af, Gf;              // FP32 copies, only to choose candidates
  float W;                       // 1/|cos| (row mode) or 1/|sin| (column mode)
  float invA;                    // 1/A
  float t00f, blinef, bstepf, inv_bstep;
  float tjf, tif;
  int mode;                      // 1: lines are rows (position = column j)
};
static_assert(sizeof(AngleConst) == 112, "AngleConst layout");

// The fraction of a 32.32 position, truncated to 23 bits: an exact multiple
// of 2^-23 in [0, 1), so that 1 - f is exact too.
__device__ __forceinline__ float frac23(long long pos) {
  const unsigned lo = (unsigned)pos;
  return __uint_as_float(0x3F800000u | (lo >> 9)) - 1.0f;
}
__device__ __forceinline__ int ipart(long long pos) { return (int)(pos >> 32); }

// Weight with which a sample at fixed-point position `pos` reaches integer
// position q under linear interpolation between floor(pos) and
// floor(pos)+1: 1-f if floor(pos) == q, f if floor(pos) == q-1, else 0.
__device__ __forceinline__ float tap_weight(long long pos, int q) {
  const int h = ipart(pos);
  const float f = frac23(pos);
  return h == q ? 1.0f - f : (h == q - 1 ? f : 0.0f);
}

}  // namespace skei

struct skei_plan_s {
  int N = 0, n_det = 0, n_angles = 0, device = -1;
  std::vector<double> angles_deg;
  skei::AngleConst *d_ang = nullptr;  // [n_angles]
  int *d_status = nullptr;            // bit 0: bad angle index seen
};

namespace skei {

// ---------------------------------------------------------------- errors --
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *where);
inline int check_launch(const char *where) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SKEI_OK : cuda_error(e, where);
}

int check_plan(skei_plan p);
int check_dtype(int dtype);
int check_dev_ptr(const void *p, const char *name);
int check_idx(skei_plan p, const int *idx, int m);
int check_batch(int B);
int ensure_ramlak_taps();

// ------------------------------------------------------- storage types --
template <typename T>
__device__ __forceinline__ float ldg_f(const T *p);
template <>
__device__ __forceinline__ float ldg_f<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldg_f<__nv_bfloat16>(const __nv_bfloat16 *p) {
  return __bfloat162float(__ldg(p));
}

template <typename T>
__device__ __forceinline__ void st_f(T *p, float v);
template <>
__device__ __forceinline__ void st_f<float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void st_f<__nv_bfloat16>(__nv_bfloat16 *p, float v) {
  *p = __float2bfloat16_rn(v);
}

// round-to-nearest(x) as an integer, |x| < 2^22.
__device__ __forceinline__ int round_int(float x) {
  const float M = 12582912.0f;
  return __float_as_int(__fadd_rn(x, M)) - 0x4B400000;
}

// 32.32 fixed point of a double (|v| < 2^30).
__device__ __forceinline__ long long to_fx(double v) { return __double2ll_rn(v * 4294967296.0); }

// cos and sin in FP64 of an angle in degrees, reduced exactly to
// [-45, 45] first (exact 0/+-1 at multiples of 90 degrees).
__device__ __forceinline__ void trig_deg(double deg, double *c, double *s) {
  double q = floor(deg / 90.0 + 0.5);
  double r = deg - 90.0 * q;
  double sr, cr;
  sincospi(r / 180.0, &sr, &cr);
  long long qi = ((long long)q % 4 + 4) % 4;
  if (qi == 0) { *c = cr;  *s = sr; }
  else if (qi == 1) { *c = -sr; *s = cr; }
  else if (qi == 2) { *c = -cr; *s = -sr; }
  else { *c = sr; *s = -cr; }
}

inline size_t ceil_div(size_t a, size_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------ internal launches --
// Joseph forward on a batch: out[b][a][k] = (A_S x_b) (or y_S - A_S x_b).
template <typename Tin, typename Tout>
int launch_proj_fwd(skei_plan p, const Tin *x, int B, const int *idx, int m,
                    const Tout *y, Tout *out, cudaStream_t st);
// Joseph adjoint: out = alpha A_S^T sino + beta add (add may alias out).
template <typename Tin, typename Tadd, typename Tout>
int launch_proj_adj(skei_plan p, const Tin *sino, int B, const int *idx, int m,
                    float alpha, float beta, const Tadd *add, Tout *out,
                    cudaStream_t st);
// Back-projection: out = alpha B_S q + beta add.
template <typename Tin, typename Tadd, typename Tout>
int launch_backproject(skei_plan p, const Tin *q, int B, const int *idx, int m,
                       float alpha, float beta, const Tadd *add, Tout *out,
                       cudaStream_t st);
// Back-projection transpose: q = alpha B_S^T x.
template <typename Tin, typename Tout>
int launch_backproject_adj(skei_plan p, const Tin *x, int B, const int *idx,
                           int m, float alpha, Tout *q, cudaStream_t st);
// Ram-Lak: q = scale H p, `rows` rows.
template <typename Tin, typename Tout>
int launch_filter(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                  cudaStream_t st);
// Rotation: out[b][g] = T_g x[b].
template <typename Tin, typename Tout>
int launch_rotate(const Tin *x, int B, int N, const double *g_deg, int G,
                  Tout *out, cudaStream_t st);
// Rotation transpose: gx[b] = alpha sum_g T_g^T gout[b][g] + beta gx[b].
template <typename Tin, typename Tout>
int launch_rotate_adj(const Tin *gout, int B, int N, const double *g_deg, int G,
                      float alpha, float beta, Tout *gx, cudaStream_t st);

}  // namespace skei
