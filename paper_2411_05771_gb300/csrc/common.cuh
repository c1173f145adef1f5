// Internal definitions shared by the kernels of libskei (sm_103a).
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>

#include "skei.h"

namespace skei {

// Per-angle constants, derived in FP64 on the host.  Positions are kept in
// 36.28 fixed point (int64: value * 2^28), so that every kernel evaluates
// them EXACTLY, in any order: forward operators and their gathered
// transposes then see bitwise the same positions and interpolation weights.
// Constants are rounded to 2^-29, so a position is within (k + L + 1) 2^-29
// (~2e-6 px at 512^2) of its FP64 value; FP32 positions near 512 would only
// be good to ~3e-5.  Differences of positions that are known to be small
// (|D| < 8) are exact in 32-bit wrapping arithmetic on the low words.
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
constexpr int kFxBits = 28;
constexpr long long kFxOne = 1LL << kFxBits;
struct AngleConst {
  long long T, A, G;             // Joseph, fixed point
  long long t00, bline, bstep;   // back-projection, fixed point
  long long tj, ti;              // back-projection per column / per row, fixed point
  float Tf, Af, Gf;              // FP32 copies, only to choose candidates
  float W;                       // 1/|cos| (row mode) or 1/|sin| (column mode)
  float invA;                    // 1/A
  float t00f, blinef, bstepf, inv_bstep;
  float tjf, tif;
  float invT;                    // 1/T (0 when T == 0)
  float inv_bline;               // 1/bline (0 when bline == 0)
  int mode;                      // 1: lines are rows (position = column j)
  int pad0;
};
static_assert(sizeof(AngleConst) == 128, "AngleConst layout");

// The fraction of a fixed-point position, truncated to 23 bits: an exact
// multiple of 2^-23 in [0, 1), so that 1 - f is exact too.
__device__ __forceinline__ float frac23(long long pos) {
  const unsigned lo = (unsigned)pos;
  return __uint_as_float(0x3F800000u | ((lo >> (kFxBits - 23)) & 0x7FFFFFu)) - 1.0f;
}
__device__ __forceinline__ float frac23(int d) { return frac23((long long)d); }
__device__ __forceinline__ int ipart(long long pos) { return (int)(pos >> kFxBits); }
__device__ __forceinline__ int ipart(int d) { return d >> kFxBits; }

}  // namespace skei

struct skei_plan_s {
  int N = 0, n_det = 0, n_angles = 0, device = -1;
  std::vector<double> angles_deg;
  skei::AngleConst *d_ang = nullptr;  // [n_angles]
  int *d_status = nullptr;            // bit 0: bad angle index seen
  // FFT form of the Ram-Lak filter: length fft_len (a power of two
  // >= 2 n_det - 1; 0 = not available) and the real spectrum of the taps
  // h(n), |n| < n_det, sampled on it
  int fft_len = 0;
  float *d_hspec = nullptr;
};

namespace skei {

// ------------------------------------------------------------ cp.async --
// 4-byte asynchronous copy global -> shared; with ok false nothing is read
// and the shared word is zeroed.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, bool ok) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem),
               "r"(ok ? 4 : 0)
               : "memory");
}
// 16 bytes, zero-filled when !ok (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool ok) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(ok ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ------------------------------------------------- dependent launches --
// Build-time knob: SKEI_PDL 1 or 2 launches the operator kernels with
// programmatic stream serialisation.  Each kernel waits (griddepcontrol.wait)
// for its predecessor's memory before it touches any; with 1 it also lets
// its successor be scheduled as soon as all its own CTAs run, with 2 only
// once they exit, which hides the successor's launch behind the grid's
// completion.  1 measured slower on the 512^2 step (a successor's CTAs
// pack onto the first SMs to free up), 2 about 1 % faster than 0.
#ifndef SKEI_PDL
#define SKEI_PDL 2
#endif
__device__ __forceinline__ void pdl_enter() {
#if SKEI_PDL
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
#endif
#if SKEI_PDL == 1
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
#endif
}
template <typename... ExpTypes, typename... ActTypes>
inline void launch_k(void (*kern)(ExpTypes...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t st, ActTypes &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = SKEI_PDL ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, std::forward<ActTypes>(args)...);
}

// ---------------------------------------------------- bounds-check build --
// SKEI_CHECK = 1 (a separate build, libskei_check.so) range-checks the shared
// and global indices of the operator kernels.  An index outside its buffer
// (shared: outside the CTA's shared allocation; global: outside the
// buffer's extent) sets the site's bit in its translation unit's check
// word, and the access is skipped (a load reads 0).  No assert, no trap:
// the kernel finishes and the host reads the bits (skei_check_status).
// With SKEI_CHECK = 0 the checks compile to nothing.
#ifndef SKEI_CHECK
#define SKEI_CHECK 0
#endif
#if SKEI_CHECK
static __device__ unsigned g_skei_check;   // one word per translation unit
#endif
// Bits: band kernels 0-7, tile kernels 8-15, filter and rotations 16-23.
enum : unsigned {
  CK_BAND_STAGE = 1u << 0, CK_BAND_TAP = 1u << 1, CK_BAND_SUMS = 1u << 2,
  CK_BAND_OUT = 1u << 3,
  CK_TILE_WIN = 1u << 8, CK_TILE_TAP = 1u << 9, CK_TILE_IN = 1u << 10, CK_TILE_OUT = 1u << 11,
  CK_FILT_STAGE = 1u << 16, CK_FILT_TAP = 1u << 17, CK_FILT_SUMS = 1u << 18,
  CK_FILT_OUT = 1u << 19,
};
// Whether index i lies in [0, n); records `bit` if not.
__device__ __forceinline__ bool ck(long long i, long long n, unsigned bit) {
#if SKEI_CHECK
  if ((unsigned long long)i < (unsigned long long)n) return true;
  atomicOr(&g_skei_check, bit);
  return false;
#else
  (void)i; (void)n; (void)bit;
  return true;
#endif
}
// Whether the `bytes` at pointer p lie inside the CTA's dynamic shared
// memory (where every checked shared buffer lives: all extern __shared__
// arrays start at its base); records `bit` if not.
extern __shared__ float4 skei_dyn_smem[];
__device__ __forceinline__ bool ck_smem(const void *p, int bytes, unsigned bit) {
#if SKEI_CHECK
  unsigned dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  const unsigned base = (unsigned)__cvta_generic_to_shared(skei_dyn_smem);
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  if (__isShared(p) && a >= base && a + (unsigned)bytes <= base + dyn) return true;
  atomicOr(&g_skei_check, bit);
  return false;
#else
  (void)p; (void)bytes; (void)bit;
  return true;
#endif
}
// Whether [p, p + bytes) lies inside [lo, hi); records `bit` if not.
__device__ __forceinline__ bool ck_range(const void *p, int bytes, const void *lo, const void *hi,
                                         unsigned bit) {
#if SKEI_CHECK
  const char *c = static_cast<const char *>(p);
  if (c >= static_cast<const char *>(lo) && c + bytes <= static_cast<const char *>(hi))
    return true;
  atomicOr(&g_skei_check, bit);
  return false;
#else
  (void)p; (void)bytes; (void)lo; (void)hi; (void)bit;
  return true;
#endif
}
// Checked shared-memory loads (0 where out of range).
template <typename V>
__device__ __forceinline__ V lds_ck(const V *p, unsigned bit) {
  if (SKEI_CHECK && !ck_smem(p, sizeof(V), bit)) return V{};
  return *p;
}
// Host side: ORs this translation unit's check word into *bits (reset: then
// clears it).  One per .cu file (SKEI_CHECK_READER).
#if SKEI_CHECK
#define SKEI_CHECK_READER(name)                                                         \
  int name(unsigned *bits, int reset) {                                                 \
    unsigned v = 0;                                                                     \
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_skei_check, sizeof v);                   \
    if (e == cudaSuccess && reset) {                                                    \
      const unsigned z = 0;                                                             \
      e = cudaMemcpyToSymbol(g_skei_check, &z, sizeof z);                               \
    }                                                                                   \
    if (e != cudaSuccess) return cuda_error(e, "check word");                           \
    *bits |= v;                                                                         \
    return SKEI_OK;                                                                     \
  }
#else
#define SKEI_CHECK_READER(name) \
  int name(unsigned *bits, int) { (void)bits; return SKEI_OK; }
#endif
int check_read_band(unsigned *bits, int reset);
int check_read_tile(unsigned *bits, int reset);
int check_read_filter(unsigned *bits, int reset);

// ---------------------------------------------------------------- errors --
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *where);
#define SKEI_TRY(expr)                     \
  do {                                     \
    if (int rc_ = (expr)) return rc_;      \
  } while (0)
inline int check_launch(const char *where) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SKEI_OK : cuda_error(e, where);
}

int check_plan(skei_plan p);
int check_dtype(int dtype);
// A pair of FP32 values held in one 64-bit register pair (low word first),
// the operand of the packed instructions (add.rn.f32x2, mul.rn.f32x2,
// fma.rn.f32x2: two IEEE operations each, the same results as two scalar
// ones); loads, stores and arithmetic move it whole.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2_add(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2x f2_pack(float lo, float hi) {
  f2x d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ float f2_lo(f2x a) { return __uint_as_float((unsigned)a); }
__device__ __forceinline__ float f2_hi(f2x a) { return __uint_as_float((unsigned)(a >> 32)); }

// An NVTX range over one C-ABI call, named after it (the calls show up on
// Nsight timelines and can be selected with ncu --nvtx); a few nanoseconds
// when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
#define SKEI_RANGE(name) ::skei::NvtxRange skei_nvtx_range_(name)

// Device allocations of the library go through dev_malloc, which fails
// the n-th of them in the process (cudaErrorMemoryAllocation, nothing
// allocated) when the environment variable SKEI_FAULT_ALLOC is n >= 1: a
// host-side fault injection for the failure paths' tests.
cudaError_t dev_malloc(void **ptr, size_t bytes);

int sm_count();   // SMs of the current device

// Opts kernel `kern` in to `smem` bytes of dynamic shared memory where they
// and its static shared memory together pass the 48 KB default; once per
// device and size increase (`configured`: the caller's record, 64 devices).
template <typename K>
int opt_in_smem(K kern, size_t smem, size_t *configured, const char *what) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (smem <= configured[dev]) return SKEI_OK;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e == cudaSuccess && smem + fa.sharedSizeBytes > 48 * 1024)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_error(e, what);
  configured[dev] = smem;
  return SKEI_OK;
}
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

// Fixed point of a double (|v| < 2^34).
__device__ __forceinline__ long long to_fx(double v) { return __double2ll_rn(v * (double)kFxOne); }

// cos and sin in FP64 of an angle in degrees, reduced exactly to
// [-45, 45] first (exact 0/+-1 at multiples of 90 degrees).  On the reduced
// angle x (|x| <= pi/4) the Taylor series of sin (through x^15) and cos
// (through x^16), evaluated in x^2 by Horner's rule, are within 1e-16: a
// short dependent chain of FP64 FMAs, which matters because a rotation CTA
// waits for it.
__device__ __forceinline__ void sincos_taylor(double x, double *s, double *c) {
  const double x2 = x * x;
  // sin x = x (1 - x^2/3! + x^4/5! - ... - x^14/15!)
  double ps = -1.0 / 1307674368000.0;                 // -1/15!
  ps = fma(ps, x2, 1.0 / 6227020800.0);               //  1/13!
  ps = fma(ps, x2, -1.0 / 39916800.0);                // -1/11!
  ps = fma(ps, x2, 1.0 / 362880.0);                   //  1/9!
  ps = fma(ps, x2, -1.0 / 5040.0);                    // -1/7!
  ps = fma(ps, x2, 1.0 / 120.0);                      //  1/5!
  ps = fma(ps, x2, -1.0 / 6.0);                       // -1/3!
  *s = fma(ps * x2, x, x);
  // cos x = 1 - x^2/2! + x^4/4! - ... + x^16/16!
  double pc = 1.0 / 20922789888000.0;                 //  1/16!
  pc = fma(pc, x2, -1.0 / 87178291200.0);             // -1/14!
  pc = fma(pc, x2, 1.0 / 479001600.0);                //  1/12!
  pc = fma(pc, x2, -1.0 / 3628800.0);                 // -1/10!
  pc = fma(pc, x2, 1.0 / 40320.0);                    //  1/8!
  pc = fma(pc, x2, -1.0 / 720.0);                     // -1/6!
  pc = fma(pc, x2, 1.0 / 24.0);                       //  1/4!
  pc = fma(pc, x2, -0.5);                             // -1/2!
  *c = fma(pc, x2, 1.0);
}

__device__ __forceinline__ void trig_deg(double deg, double *c, double *s) {
  // quadrant by a multiply, not a division (a shorter dependent chain; at a
  // tie, deg = 45 + 90 k, either neighbour gives a valid reduced angle)
  double q = floor(fma(deg, 1.0 / 90.0, 0.5));
  double r = fma(-90.0, q, deg);
  double sr, cr;
  sincos_taylor(r * (3.14159265358979323846 / 180.0), &sr, &cr);
  long long qi = ((long long)q % 4 + 4) % 4;
  if (qi == 0) { *c = cr;  *s = sr; }
  else if (qi == 1) { *c = -sr; *s = cr; }
  else if (qi == 2) { *c = -cr; *s = -sr; }
  else { *c = sr; *s = -cr; }
}

inline size_t ceil_div(size_t a, size_t b) { return (a + b - 1) / b; }

// --------------------------------------------- dtype-erased device data --
// Loads/stores of image and sinogram buffers whose storage type (float or
// bfloat16) is a runtime flag; kernels branch on it only where the branch is
// uniform across a CTA (staging, window fills, final stores).
__device__ __forceinline__ float ld_any(const void *p, size_t i, int bf16) {
  return bf16 ? __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(p) + i))
              : __ldg(static_cast<const float *>(p) + i);
}
__device__ __forceinline__ void st_any(void *p, size_t i, float v, int bf16) {
  if (bf16) static_cast<__nv_bfloat16 *>(p)[i] = __float2bfloat16_rn(v);
  else static_cast<float *>(p)[i] = v;
}
template <typename T> __host__ __device__ constexpr int is_bf16() { return 0; }
template <> __host__ __device__ constexpr int is_bf16<__nv_bfloat16>() { return 1; }

// Rounds an FP32 value to storage type T and back (what storing then
// loading it gives).
template <typename T>
__device__ __forceinline__ float rnd_store(float v) {
  if constexpr (is_bf16<T>()) return __bfloat162float(__float2bfloat16_rn(v));
  else return v;
}

// The final pass of the loss reductions, by one CTA of any shape whose
// thread count is a whole number (>= 1) of warps (seg_sum: B G + B doubles
// of shared memory): the segment sums of the per-chunk partials in a fixed
// order, then
// loss = (1/B) sum_b [mc_scale ||r_b||^2 + (lambda/G) sum_g ||x2 - x3||^2].
__device__ __forceinline__ void ei_final_block(const double *partial, int B, int G, int cpi,
                                               int cpr, double lambda, double mc_scale,
                                               double *mc_out, double *ei_out, double *loss_out,
                                               double *seg_sum) {
  const int nseg = B * G + B;
  // linear thread index: the CTA may be 2D or 3D
  const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthreads >> 5;
  for (int sgi = warp; sgi < nseg; sgi += nwarps) {
    const bool img = sgi < B * G;
    const int nch = img ? cpi : cpr;
    const double *src = img ? partial + (size_t)sgi * cpi
                            : partial + (size_t)B * G * cpi + (size_t)(sgi - B * G) * cpr;
    double s = 0.0;
    for (int c = lane; c < nch; c += 32) s += src[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) seg_sum[sgi] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double loss = 0.0;
    for (int b = 0; b < B; ++b) {
      const double mc = mc_scale * seg_sum[B * G + b];
      double ei = 0.0;
      for (int g = 0; g < G; ++g) {
        const double e = seg_sum[b * G + g];
        if (ei_out) ei_out[b * G + g] = e;
        ei += e;
      }
      if (mc_out) mc_out[b] = mc;
      loss += mc + lambda / G * ei;
    }
    if (loss_out) *loss_out = loss / B;
  }
}

// Adam's constants (Kingma and Ba 2015) as the kernels take them.
struct AdamArgs {
  float *theta, *m, *v;
  const int *step;
  float lr, b1, b2, omb1, omb2, eps, lnb1, lnb2;
};
// The loss's final pass, done by one CTA of a later launch.
struct LossFinal {
  const double *partial;
  int B, G, cpi, cpr;
  double lambda, mc_scale;
  double *mc_out, *ei_out, *loss_out;
};

// One operator application over a batch of images, as the band and tile
// kernels see it.  Up to kMaxJobs jobs share a launch (grid.z spans the
// images of all of them): the fused EI step projects x1 (MC term) and x2
// (EI term) in one launch, and back-projects r and the EI gradient in one.
//   band (A, B^T):   in = images [nimg][N][N]; out = [nimg][m][n_det];
//                    aux = NULL or full measurement y [nimg][n_angles][n_det]
//                    (A only: out = S y - A_S x)
//   tile (A^T, B):   in = sinograms [nimg][m][n_det]; out = [nimg][N][N];
//                    out = alpha * op(in) + beta * aux (aux may alias out)
struct Job {
  const void *in;
  const void *aux;
  void *out;
  const int *idx;     // device angle list [m] or NULL (all angles)
  int m, nimg;
  float alpha, beta;
  int in_bf16, aux_bf16, out_bf16;
  // > 0: idx holds one list per sample, [rows][m], and images
  // r idx_per .. (r+1) idx_per - 1 use row r (a sketch per sample, Algorithm 1)
  int idx_per = 0;
  // tile operators only: a second output out2 = (out as stored) + add2, add2
  // one FP32 image [N][N] for every image of the job (the residual network
  // F(u) = u + theta applied to the output)
  void *out2 = nullptr;
  const float *add2 = nullptr;
  int out2_bf16 = 0;
  // tile operators only: the FP32 input holds the images interleaved by
  // groups of 4, value (b, row, k) at ((b / 4 * m + row) n_det + k) 4 + b % 4,
  // so a group's 4 bins are one 16-byte load (written so by the fused band
  // sums + filter of the SkEI step)
  int in_il4 = 0;
};
constexpr int kMaxJobs = 2;
struct Jobs {
  Job j[kMaxJobs];
  int njobs;
};

enum { OP_JOSEPH = 0, OP_BP_ADJ = 1, OP_JOSEPH_ADJ = 2, OP_BACKPROJECT = 3 };

// The angle list of image b of job J (NULL: all angles).
__host__ __device__ __forceinline__ const int *job_idx(const Job &J, int b) {
  return (J.idx && J.idx_per > 0) ? J.idx + (size_t)(b / J.idx_per) * J.m : J.idx;
}
// Whether groups of 4 consecutive images of J share one angle list.
__host__ __device__ __forceinline__ bool job_groupable(const Job &J) {
  return !J.idx || J.idx_per <= 0 || J.idx_per % 4 == 0;
}
inline bool jobs_groupable(const Jobs &J) {
  for (int q = 0; q < J.njobs; ++q)
    if (!job_groupable(J.j[q])) return false;
  return true;
}

// Image groups.  The images of one job share its angle list, so the
// operator kernels compute positions and weights once per group of 4 images
// and apply them to all 4; a job of n images is cut into n / 4 groups of 4,
// then single images.
// gmax = 1 turns grouping off.
__host__ __device__ __forceinline__ int n_groups(int n, int gmax = 4) {
  return gmax == 4 ? (n >> 2) + (n & 3) : n;
}
__host__ __device__ __forceinline__ void group_at(int n, int g, int *b0, int *ni, int gmax = 4) {
  const int q = gmax == 4 ? n >> 2 : 0;
  if (g < q) {
    *b0 = 4 * g;
    *ni = 4;
  } else {
    *b0 = 4 * q + (g - q);
    *ni = 1;
  }
}

int launch_band_jobs(skei_plan p, int op, const Jobs &jobs, cudaStream_t st);
int launch_tile_jobs(skei_plan p, int op, const Jobs &jobs, cudaStream_t st);
// The band operators with a workspace of band sums (two launches: sums per
// thin band, then their ordered reduction): faster when the caller can give
// band_partial_floats(p, jobs) floats.
size_t band_partial_floats(skei_plan p, const Jobs &jobs);
// With a filter request, the second launch also filters the rows of one
// job: fout = scale H (the job's rows), FP32, written instead of the job's
// own output (the step's filtered sinograms); the other job's rows are
// written as usual.
struct FilterReq {
  int job;        // 0 or 1
  float scale;
  float *out;     // [rows of the job][n_det], or interleaved by 4 images (il4)
  int il4 = 0;    // out in the layout of Job::in_il4
};
int launch_band_partial_jobs(skei_plan p, int op, const Jobs &jobs, float *work,
                             size_t work_floats, cudaStream_t st,
                             const FilterReq *fr = nullptr);
// The second pass of the band sums fused with the filter (in the filter's
// translation unit, next to its taps).
int launch_band_sum_filter(skei_plan p, int op, const Jobs &jobs, int nb0, int nb1,
                           const float *part, size_t off0, size_t off1, size_t part_floats,
                           const FilterReq &fr, cudaStream_t st);
// Whether Joseph's band sums over these two jobs carry job 0's images in the
// CTAs of job 1's groups of 4 (same angle lists, 4 images of job 1 per image
// of job 0).
bool band_sums_merge(const Jobs &jobs);

// ------------------------------------------------- batched (persistent) --
// One instance of a batch - images of one size and angle list, with its own
// sketch - as the persistent kernels see it: out = alpha op_S(in).
struct BatchItem {
  const AngleConst *ang;   // the instance's plan
  int *status;
  const void *in;
  void *out;
  const int *idx;          // sketch rows [m] or NULL
  int N, n_det, n_angles, m, B;
  float alpha;
  int in_bf16, out_bf16;
};

// A persistent launch hands out tasks through queue[0] and counts finished
// workers in queue[1]; the last worker to finish resets both, so the next
// launch (stream-ordered after this one) starts from zero.  Called by one
// thread per worker after its last atomicAdd on queue[0].
__device__ __forceinline__ void queue_retire(int *queue, int workers) {
  __threadfence();
  if (atomicAdd(queue + 1, 1) == workers - 1) {
    atomicExch(queue, 0);
    atomicExch(queue + 1, 0);
  }
}

// Band operators (A: OP_JOSEPH, B^T: OP_BP_ADJ): AB angles and an image
// group of NI (1 or 4) per task.  Tasks: int4 (item, b0 << 3 | NI, first
// angle or tile row, tile column).
size_t band_batch_smem(int op, int N, int n_det, int n_angles, int AB, int NI);
int band_batch_occupancy(int op, size_t smem, int *clusters);
int launch_band_batch_op(int op, const BatchItem *items, const int4 *tasks, int n_tasks, int AB,
                         size_t smem, int clusters, int *queue, cudaStream_t st);
// Tile operators (A^T: OP_JOSEPH_ADJ, B: OP_BACKPROJECT): one tile of an
// image group per task; tile_batch_shape gives the tile size.
void tile_batch_shape(int *rows, int *cols);
int tile_batch_occupancy(int op, int *ctas_per_sm);
int launch_tile_batch_op(int op, const BatchItem *items, const int4 *tasks, int n_tasks,
                         int ctas, int *queue, cudaStream_t st);
// Ram-Lak rows: one row per task (items' in/out are sinograms, alpha the
// filter's scale).
size_t filter_batch_smem(int n_det_max);
int filter_batch_occupancy(size_t smem, int *ctas_per_sm);
int launch_filter_batch(const BatchItem *items, const int4 *tasks, int n_tasks, size_t smem,
                        int ctas, int *queue, cudaStream_t st);

// ------------------------------------------------------ internal launches --
// Single-job conveniences over the two above.
template <typename Tin, typename Tout>
int launch_proj_fwd(skei_plan p, const Tin *x, int B, const int *idx, int m,
                    const Tout *y, Tout *out, cudaStream_t st) {
  Jobs J{};
  J.njobs = 1;
  J.j[0] = Job{x, y, out, idx, m, B, 1.0f, 0.0f, is_bf16<Tin>(), is_bf16<Tout>(), is_bf16<Tout>()};
  return launch_band_jobs(p, OP_JOSEPH, J, st);
}
// Joseph adjoint: out = alpha A_S^T sino + beta add (add may alias out).
template <typename Tin, typename Tadd, typename Tout>
int launch_proj_adj(skei_plan p, const Tin *sino, int B, const int *idx, int m,
                    float alpha, float beta, const Tadd *add, Tout *out,
                    cudaStream_t st) {
  Jobs J{};
  J.njobs = 1;
  J.j[0] = Job{sino, add, out, idx, m, B, alpha, beta, is_bf16<Tin>(), is_bf16<Tadd>(),
               is_bf16<Tout>()};
  return launch_tile_jobs(p, OP_JOSEPH_ADJ, J, st);
}
// Back-projection: out = alpha B_S q + beta add.
template <typename Tin, typename Tadd, typename Tout>
int launch_backproject(skei_plan p, const Tin *q, int B, const int *idx, int m,
                       float alpha, float beta, const Tadd *add, Tout *out,
                       cudaStream_t st) {
  Jobs J{};
  J.njobs = 1;
  J.j[0] = Job{q, add, out, idx, m, B, alpha, beta, is_bf16<Tin>(), is_bf16<Tadd>(),
               is_bf16<Tout>()};
  return launch_tile_jobs(p, OP_BACKPROJECT, J, st);
}
// Back-projection transpose: q = alpha B_S^T x.
template <typename Tin, typename Tout>
int launch_backproject_adj(skei_plan p, const Tin *x, int B, const int *idx,
                           int m, float alpha, Tout *q, cudaStream_t st) {
  Jobs J{};
  J.njobs = 1;
  J.j[0] = Job{x, nullptr, q, idx, m, B, alpha, 0.0f, is_bf16<Tin>(), 0, is_bf16<Tout>()};
  return launch_band_jobs(p, OP_BP_ADJ, J, st);
}
// Ram-Lak: q = scale H p, `rows` rows.
template <typename Tin, typename Tout>
int launch_filter(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                  cudaStream_t st);
// The same through the plan's FFT form (falls back to the direct form when
// the plan has none).
template <typename Tin, typename Tout>
int launch_filter_fft(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                      cudaStream_t st);
// The same as tensor-core matrix products (3 TF32 products per FP32 product;
// the direct form beyond 2048 bins).
template <typename Tin, typename Tout>
int launch_filter_tc(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                     cudaStream_t st);
// The form the EI step uses (build-time choice).
template <typename Tin, typename Tout>
int launch_filter_step(skei_plan p, const Tin *in, int rows, float scale, Tout *out,
                       cudaStream_t st);
// Plan set-up of the FFT form (host: the spectrum in FP64, then upload).
int make_filter_spectrum(skei_plan p);
// Rotation: out[b][g][ch] = T_g x[b][ch] (Ch channels share each angle).
template <typename Tin, typename Tout>
int launch_rotate(const Tin *x, int B, int N, const double *g_deg, int G,
                  Tout *out, cudaStream_t st, int Ch = 1);
// Rotation transpose: gx[b][ch] = alpha sum_g T_g^T gout[b][g][ch] + beta gx[b][ch].
template <typename Tin, typename Tout>
int launch_rotate_adj(const Tin *gout, int B, int N, const double *g_deg, int G,
                      float alpha, float beta, Tout *gx, cudaStream_t st, int Ch = 1);
// The rotation of the residual network's output: x1 = x0 + theta (stored as
// T) and out[b][g] = T_g x1[b], in one launch.
template <typename T>
int launch_rotate_residual(const T *x0, const float *theta, int B, int N, const double *g_deg,
                           int G, T *x1, T *out, cudaStream_t st);
// The last launch of the residual network's step (one measurement):
// gx = sum_g T_g^T gout[g] + gx (stored as T), then Adam on theta with the
// gradient gx + sum_g g_x3[g] (F(u) = u + theta is applied to x1 and to the
// G reconstructions); the loss's final pass rides in the first CTA.
template <typename T>
int launch_rotate_adj_adam(const float *gout, int N, const double *g_deg, int G, T *gx,
                           const T *g_x3, const AdamArgs &adam, const LossFinal &lf,
                           cudaStream_t st);

}  // namespace skei
