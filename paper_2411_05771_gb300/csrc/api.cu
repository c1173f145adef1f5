// C-ABI entry points of libskei: argument validation, dtype dispatch and the
// composition of the EI / SkEI loss (Eq. (e:skeiloss), Algorithm 2) from the
// operator kernels, plus the FP64 loss reductions and the stand-in network's
// helpers (residual add, Adam).
#include <cmath>
#include <type_traits>

#include "common.cuh"

using bf16 = __nv_bfloat16;

namespace skei {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kChunk = 2048;     // elements per partial sum of the loss
constexpr int kRedThreads = 256;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// ------------------------------------------------------ loss reductions --
// Pass 1: one CTA per chunk of one segment.  Image segments (b, g) hold
// d = x2 - x3 and also emit g_x2 = kappa d, g_x3 = -kappa d; residual
// segments b hold r.  Each CTA writes sum d^2 (FP64) of its chunk.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    ei_partials_kernel(const T *x2, const T *x3, const T *r, int64_t n_img, int n_imgseg,
                       int cpi, int64_t r_len, int cpr, float kappa, T *g_x2, T *g_x3,
                       double *partial) {
  pdl_enter();
  __shared__ double red[kRedThreads / 32];
  const int blk = blockIdx.x;
  // each thread sums its few elements in FP32, the block adds the threads'
  // sums in FP64 in a fixed order
  float s = 0.0f;
  if (blk < n_imgseg * cpi) {
    const int seg = blk / cpi, ch = blk - seg * cpi;
    const int64_t base = (int64_t)seg * n_img;
    const int64_t e0 = (int64_t)ch * kChunk, e1 = min(e0 + kChunk, n_img);
    int64_t e = e0 + threadIdx.x;
    if (!is_bf16<T>() && n_img % 4 == 0) {
      // four elements per access; chunks start on multiples of kChunk
      const float4 *a4 = reinterpret_cast<const float4 *>(x2 + base);
      const float4 *b4 = reinterpret_cast<const float4 *>(x3 + base);
      float4 *g2 = reinterpret_cast<float4 *>(g_x2 + base);
      float4 *g3 = reinterpret_cast<float4 *>(g_x3 + base);
      for (int64_t e4 = e0 / 4 + threadIdx.x; e4 < e1 / 4; e4 += kRedThreads) {
        const float4 a = __ldg(a4 + e4), c = __ldg(b4 + e4);
        const float4 d = make_float4(a.x - c.x, a.y - c.y, a.z - c.z, a.w - c.w);
        s = fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, fmaf(d.w, d.w, s))));
        if (g_x2) g2[e4] = make_float4(kappa * d.x, kappa * d.y, kappa * d.z, kappa * d.w);
        if (g_x3) g3[e4] = make_float4(-kappa * d.x, -kappa * d.y, -kappa * d.z, -kappa * d.w);
      }
      e = e1;
    }
    for (; e < e1; e += kRedThreads) {
      const float d = ldg_f(x2 + base + e) - ldg_f(x3 + base + e);
      s = fmaf(d, d, s);
      if (g_x2) st_f(g_x2 + base + e, kappa * d);
      if (g_x3) st_f(g_x3 + base + e, -kappa * d);
    }
  } else {
    const int rb = blk - n_imgseg * cpi;
    const int seg = rb / cpr, ch = rb - seg * cpr;
    const int64_t base = (int64_t)seg * r_len;
    const int64_t e0 = (int64_t)ch * kChunk, e1 = min(e0 + kChunk, r_len);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kRedThreads) {
      const float v = ldg_f(r + base + e);
      s = fmaf(v, v, s);
    }
  }
  double sd = (double)s;
  for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) t += red[w];
    partial[blk] = t;
  }
}

// Pass 2 (one CTA): segment sums in a fixed order, then
// loss = (1/B) sum_b [mc_scale ||r_b||^2 + (lambda/G) sum_g ||x2 - x3||^2].
__global__ void __launch_bounds__(kRedThreads)
    ei_final_kernel(const double *partial, int B, int G, int cpi, int cpr, double lambda,
                    double mc_scale, double *mc_out, double *ei_out, double *loss_out) {
  pdl_enter();
  extern __shared__ double seg_sum[];  // [B*G + B]
  ei_final_block(partial, B, G, cpi, cpr, lambda, mc_scale, mc_out, ei_out, loss_out, seg_sum);
}

// --------------------------------------------------- stand-in network --
template <typename T>
__global__ void residual_add_kernel(const T *u, const float *theta, int n, T *out) {
  pdl_enter();
  // blockIdx.y selects the image, so no division or modulo per element
  const size_t base = (size_t)blockIdx.y * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    st_f(out + base + e, ldg_f(u + base + e) + __ldg(theta + e));
}

// FP32, n % 4 == 0: four elements per thread and access.
__global__ void residual_add4_kernel(const float4 *u, const float4 *theta, int n4, float4 *out) {
  pdl_enter();
  const size_t base = (size_t)blockIdx.y * n4;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += gridDim.x * blockDim.x) {
    const float4 a = __ldg(u + base + e), t = __ldg(theta + e);
    out[base + e] = make_float4(a.x + t.x, a.y + t.y, a.z + t.z, a.w + t.w);
  }
}

// Bias corrections 1 - beta^t evaluated as -expm1(t ln beta) with ln beta
// from FP64 on the host: no cancellation, so FP32 keeps them to ~1e-7.
template <typename T>
__global__ void adam_kernel(float *theta, int64_t n, const T *g1, int c1, const T *g2, int c2,
                            float *m, float *v, const int *step, float lr, float b1, float b2,
                            float omb1, float omb2, float eps, float lnb1, float lnb2) {
  pdl_enter();
  const float t = (float)max(__ldg(step), 1);
  const float bc1 = -expm1f(t * lnb1), bc2 = -expm1f(t * lnb2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float g = 0.0f;
    for (int c = 0; c < c1; ++c) g += ldg_f(g1 + (int64_t)c * n + i);
    for (int c = 0; c < c2; ++c) g += ldg_f(g2 + (int64_t)c * n + i);
    const float mi = fmaf(b1, m[i], omb1 * g);
    const float vi = fmaf(b2, v[i], omb2 * g * g);
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// FP32 gradients, n % 4 == 0: four elements per thread and access.
__global__ void adam4_kernel(float4 *theta, int n4, const float4 *g1, int c1, const float4 *g2,
                             int c2, float4 *m, float4 *v, const int *step, float lr, float b1,
                             float b2, float omb1, float omb2, float eps, float lnb1,
                             float lnb2) {
  pdl_enter();
  const float t = (float)max(__ldg(step), 1);
  const float bc1 = -expm1f(t * lnb1), bc2 = -expm1f(t * lnb2);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int c = 0; c < c1; ++c) {
      const float4 a = __ldg(g1 + (size_t)c * n4 + i);
      g.x += a.x; g.y += a.y; g.z += a.z; g.w += a.w;
    }
    for (int c = 0; c < c2; ++c) {
      const float4 a = __ldg(g2 + (size_t)c * n4 + i);
      g.x += a.x; g.y += a.y; g.z += a.z; g.w += a.w;
    }
    float4 mi = m[i], vi = v[i], th = theta[i];
    float *pm = &mi.x, *pv = &vi.x, *pt = &th.x;
    const float *pg = &g.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      pm[q] = fmaf(b1, pm[q], omb1 * pg[q]);
      pv[q] = fmaf(b2, pv[q], omb2 * pg[q] * pg[q]);
      pt[q] -= lr * (pm[q] / bc1) / (sqrtf(pv[q] / bc2) + eps);
    }
    m[i] = mi;
    v[i] = vi;
    theta[i] = th;
  }
}

// Row *counter of a resident table of per-iteration draws into dst, then
// *counter + 1 (Algorithm 2 draws a sketch and G rotations every
// iteration); a counter outside [0, n_rows) copies nothing and becomes -1.
// V: uint4 where the row is a whole number of aligned 16-byte words, else
// unsigned char.
template <typename V>
__global__ void step_draws_kernel(const V *table, int n_rows, int64_t row_words, int *counter,
                                  V *dst) {
  pdl_enter();
  __shared__ int s_row;
  if (threadIdx.x == 0) s_row = *counter;
  __syncthreads();
  const int r = s_row;
  if (r < 0 || r >= n_rows) {
    if (threadIdx.x == 0) *counter = -1;
    return;
  }
  const V *src = table + (size_t)r * row_words;
  for (int64_t i = threadIdx.x; i < row_words; i += blockDim.x) dst[i] = src[i];
  if (threadIdx.x == 0) *counter = r + 1;
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 32);
}

// ------------------------------------------------------------ FBP helpers --
template <typename T>
int fbp_impl(skei_plan p, const T *sino, int B, const int *idx, int m, T *x, float *work,
             cudaStream_t st) {
  if (int rc = launch_filter<T, float>(p, sino, B * m, (float)(kPi / m), work, st)) return rc;
  return launch_backproject<float, T, T>(p, work, B, idx, m, 1.0f, 0.0f, nullptr, x, st);
}

template <typename T>
int fbp_adj_impl(skei_plan p, const T *x, int B, const int *idx, int m, T *sino, float *work,
                 cudaStream_t st) {
  if (int rc = launch_backproject_adj<T, float>(p, x, B, idx, m, 1.0f, work, st)) return rc;
  return launch_filter<float, T>(p, work, B * m, (float)(kPi / m), sino, st);
}

// -------------------------------------------------------------- EI loss --
// Image-angle-lines from which the SkEI step's forward projection uses the
// band-sums form (build-time knob).
#ifndef SKEI_STEP_FWD_SUMS_MIN
#define SKEI_STEP_FWD_SUMS_MIN 200000
#endif
constexpr double kStepFwdSumsMin = SKEI_STEP_FWD_SUMS_MIN;

struct EiWork {
  size_t p_bytes, img_bytes, part_bytes, band_off, band_floats, fwd_band_floats, total;
  int cpi, cpr;
};

EiWork ei_work(skei_plan p, int B, int G, int mc_m, int sk_m) {
  EiWork w;
  const size_t bg = (size_t)B * G;
  w.p_bytes = align256(bg * sk_m * p->n_det * sizeof(float));
  w.img_bytes = align256(bg * p->N * p->N * sizeof(float));
  w.cpi = (int)ceil_div((size_t)p->N * p->N, kChunk);
  w.cpr = (int)ceil_div((size_t)mc_m * p->n_det, kChunk);
  w.part_bytes = align256((bg * w.cpi + (size_t)B * w.cpr) * sizeof(double));
  const size_t fwd = 2 * w.p_bytes;
  const size_t bwd = 2 * w.p_bytes + w.img_bytes;
  w.band_off = std::max(std::max(fwd, bwd), w.part_bytes);
  // band sums of B^T (EI job) and of the fused A launch (MC + EI jobs),
  // the latter only where the step uses them
  Jobs jb{}, jf{};
  jb.njobs = 1;
  jb.j[0].nimg = (int)bg;
  jb.j[0].m = sk_m;
  jf.njobs = 2;
  jf.j[0].nimg = B;
  jf.j[0].m = mc_m;
  jf.j[1].nimg = (int)bg;
  jf.j[1].m = sk_m;
  w.fwd_band_floats = band_partial_floats(p, jf);
  w.band_floats = band_partial_floats(p, jb);
  // (G = 4 with equal list lengths: the MC image may ride, if the lists
  // are one)
  if (((double)B * mc_m + (double)bg * sk_m) * p->N >= kStepFwdSumsMin ||
      (G == 4 && mc_m == sk_m))
    w.band_floats = std::max(w.band_floats, w.fwd_band_floats);
  w.total = w.band_off + align256(w.band_floats * sizeof(float));
  return w;
}

// The two jobs of the step's fused A launch (MC term, EI term).
Jobs ei_fwd_jobs(const void *x1, const void *y, void *r, int B, const int *mc_idx, int mc_m,
                 const void *x2, void *pbuf, const int *sk_idx, int sk_m, int G, int tb,
                 bool per_sample) {
  Jobs J{};
  J.njobs = 2;
  const int mc_per = per_sample && mc_idx ? 1 : 0, sk_per = per_sample && sk_idx ? G : 0;
  J.j[0] = Job{x1, y, r, mc_idx, mc_m, B, 1.0f, 0.0f, tb, tb, tb, mc_per};
  J.j[1] = Job{x2, nullptr, pbuf, sk_idx, sk_m, B * G, 1.0f, 0.0f, tb, 0, 0, sk_per};
  return J;
}

// Whether the fused A launch takes the band-sums form: it pays on large
// launches (many image-angles) and where the MC image rides in the EI
// group's CTAs; the cluster form on small launches otherwise (measured on
// GB300: 8 x 256^2 x 180 angles 79 vs 147 us; 5 x 512^2 x 30 angles 44 vs
// 37 us apart, 32 vs 36 us riding).
bool ei_fwd_sums(skei_plan p, const EiWork &w, const Jobs &J) {
  const double work_units = ((double)J.j[0].nimg * J.j[0].m + (double)J.j[1].nimg * J.j[1].m) *
                            p->N;
  return (work_units >= kStepFwdSumsMin || band_sums_merge(J)) &&
         w.band_floats >= w.fwd_band_floats;
}

// per_sample: mc_idx and sk_idx hold one angle list per measurement,
// [B][m] (Algorithm 1 draws a sketch per sample); the G transformed images
// of measurement b use row b.
// The residual network F(u) = u + theta folded into the step (all NULL
// otherwise): x1 = x0 + theta is computed by the rotation launch (x1 is
// then an output), and x3 = z + theta by the back-projection's epilogue.
template <typename T>
struct Residual {
  const T *x0 = nullptr;
  const float *theta = nullptr;
  T *x3 = nullptr;
};

template <typename T>
int ei_fwd_impl(skei_plan p, const T *x1, const T *y, int B, const int *mc_idx, int mc_m,
                const int *sk_idx, int sk_m, const double *g_deg, int G, T *r, T *x2, T *z,
                char *work, cudaStream_t st, bool per_sample = false,
                const Residual<T> &res = Residual<T>()) {
  const EiWork w = ei_work(p, B, G, mc_m, sk_m);
  float *pbuf = reinterpret_cast<float *>(work);
  float *qbuf = reinterpret_cast<float *>(work + w.p_bytes);
  const int BG = B * G;
  const int tb = is_bf16<T>();
  int rc;
  if (res.x0) {
    if ((rc = launch_rotate_residual<T>(res.x0, res.theta, B, p->N, g_deg, G,
                                        const_cast<T *>(x1), x2, st)))
      return rc;
  } else if ((rc = launch_rotate<T, T>(x1, B, p->N, g_deg, G, x2, st))) {
    return rc;
  }
  // one launch: r = S_mc y - A_mc x1 (MC term) and p = A_S x2 (EI term)
  const Jobs J = ei_fwd_jobs(x1, y, r, B, mc_idx, mc_m, x2, pbuf, sk_idx, sk_m, G, tb, per_sample);
  const int sk_per = per_sample && sk_idx ? G : 0;
  // q passes from the filter to B interleaved by groups of 4 images (one
  // 16-byte copy per bin of a group in B's windows) where all groups are 4
  Job jq{};
  jq.idx = sk_idx;
  jq.idx_per = sk_per;
  const int il4 = (BG % 4 == 0 && job_groupable(jq)) ? 1 : 0;
  bool q_il4 = false;
  if (ei_fwd_sums(p, w, J)) {
    // band sums; their reduction also filters the EI rows: q = (pi/m) H A_S x2
    const FilterReq fr{1, (float)(kPi / sk_m), qbuf, il4};
    q_il4 = il4 != 0;
    if ((rc = launch_band_partial_jobs(p, OP_JOSEPH, J,
                                      reinterpret_cast<float *>(work + w.band_off),
                                      w.band_floats, st, &fr)))
      return rc;
  } else {
    if ((rc = launch_band_jobs(p, OP_JOSEPH, J, st))) return rc;
    if ((rc = launch_filter_step<float, float>(p, pbuf, BG * sk_m, (float)(kPi / sk_m), qbuf,
                                               st)))
      return rc;
  }
  Jobs Jz{};
  Jz.njobs = 1;
  Jz.j[0] = Job{qbuf, nullptr, z, sk_idx, sk_m, BG, 1.0f, 0.0f, 0, tb, tb, sk_per};
  Jz.j[0].in_il4 = q_il4 ? 1 : 0;
  if (res.x3) {
    Jz.j[0].out2 = res.x3;
    Jz.j[0].add2 = res.theta;
    Jz.j[0].out2_bf16 = tb;
  }
  return launch_tile_jobs(p, OP_BACKPROJECT, Jz, st);
}

// With last_rotation false (and g_z given) the final rotation transpose is
// left to the caller: g_x1 then holds the MC term only, and the EI term's
// unrotated gradients g_x2 + A_S^T v are in the workspace (FP32,
// [B][G][N][N] at 2 p_bytes).
template <typename T>
int ei_bwd_impl(skei_plan p, const T *r, const T *g_x2, const T *g_z, int B, const int *mc_idx,
                int mc_m, const int *sk_idx, int sk_m, const double *g_deg, int G,
                double mc_coef, T *g_x1, char *work, cudaStream_t st, bool per_sample = false,
                bool last_rotation = true) {
  const EiWork w = ei_work(p, B, G, mc_m, sk_m);
  const int mc_per = per_sample && mc_idx ? 1 : 0, sk_per = per_sample && sk_idx ? G : 0;
  float *ubuf = reinterpret_cast<float *>(work);
  float *vbuf = reinterpret_cast<float *>(work + w.p_bytes);
  float *gtot = reinterpret_cast<float *>(work + 2 * w.p_bytes);
  const int BG = B * G;
  const int tb = is_bf16<T>();
  const float amc = (float)(-2.0 * mc_coef);
  int rc;
  if (g_z) {
    // through z = (pi/m) B_S H A_S x2:  g_x2 + (pi/m) A_S^T H B_S^T g_z
    Jobs Jb{};
    Jb.njobs = 1;
    Jb.j[0] = Job{g_z, nullptr, ubuf, sk_idx, sk_m, BG, 1.0f, 0.0f, tb, 0, 0, sk_per};
    // band sums of B_S^T g_z; their reduction also filters: v = (pi/m) H B_S^T g_z
    // (interleaved by groups of 4 images for A^T's windows where all groups are 4)
    const int il4 = (BG % 4 == 0 && job_groupable(Jb.j[0])) ? 1 : 0;
    const FilterReq fr{0, (float)(kPi / sk_m), vbuf, il4};
    if ((rc = launch_band_partial_jobs(p, OP_BP_ADJ, Jb,
                                      reinterpret_cast<float *>(work + w.band_off),
                                      w.band_floats, st, &fr)))
      return rc;
    // one launch: g_x1 = -2 mc_coef A_mc^T r (MC term) and
    // gtot = g_x2 + A_S^T v (EI term)
    Jobs J{};
    J.njobs = 2;
    J.j[0] = Job{r, nullptr, g_x1, mc_idx, mc_m, B, amc, 0.0f, tb, tb, tb, mc_per};
    J.j[1] = Job{vbuf, g_x2, gtot, sk_idx, sk_m, BG, 1.0f, g_x2 ? 1.0f : 0.0f, 0, tb, 0, sk_per};
    J.j[1].in_il4 = il4;
    if ((rc = launch_tile_jobs(p, OP_JOSEPH_ADJ, J, st))) return rc;
    if (!last_rotation) return SKEI_OK;
    return launch_rotate_adj<float, T>(gtot, B, p->N, g_deg, G, 1.0f, 1.0f, g_x1, st);
  }
  // MC term: g_x1 = -2 mc_coef A_mc^T r
  Jobs Jm{};
  Jm.njobs = 1;
  Jm.j[0] = Job{r, nullptr, g_x1, mc_idx, mc_m, B, amc, 0.0f, tb, tb, tb, mc_per};
  if ((rc = launch_tile_jobs(p, OP_JOSEPH_ADJ, Jm, st))) return rc;
  if (g_x2) return launch_rotate_adj<T, T>(g_x2, B, p->N, g_deg, G, 1.0f, 1.0f, g_x1, st);
  return SKEI_OK;
}

template <typename T>
int ei_finish_impl(const T *x2, const T *x3, const T *r, int B, int G, int64_t n_img, int r_len,
                   double lambda, double mc_scale, double *mc_out, double *ei_out,
                   double *loss_out, T *g_x2, T *g_x3, char *work, cudaStream_t st) {
  const int cpi = (int)ceil_div((size_t)n_img, kChunk);
  const int cpr = (int)ceil_div((size_t)r_len, kChunk);
  double *partial = reinterpret_cast<double *>(work);
  const int nblk = B * G * cpi + B * cpr;
  const float kappa = (float)(2.0 * lambda / ((double)B * G));
  launch_k(ei_partials_kernel<T>, dim3(nblk), dim3(kRedThreads), 0, st, x2, x3, r, n_img, B * G,
           cpi, r_len, cpr, kappa, g_x2, g_x3, partial);
  if (int rc = check_launch("loss partial sums launch")) return rc;
  const size_t smem = sizeof(double) * (size_t)(B * G + B);
  // dynamic shared memory below 40 KB: with the kernel's static part, under the 48 KB default
  if (smem > 40 * 1024) return set_error(SKEI_EINVAL, "B*G + B = %d segments is too many", B * G + B);
  launch_k(ei_final_kernel, dim3(1), dim3(kRedThreads), smem, st, (const double *)partial, B, G,
           cpi, cpr, lambda, mc_scale, mc_out, ei_out, loss_out);
  return check_launch("loss final reduction launch");
}

// ------------------------------------------------ residual-network step --
// Algorithm 2's iteration for the network F_theta(u) = u + theta, the
// operator launches of skei_ei_loss_fwd / finish / bwd and Adam with the
// network folded in (see skei_ttt_residual_step).
size_t ttt_loss_off(skei_plan p, int B, int G, int mc_m, int sk_m) {
  return align256(ei_work(p, B, G, mc_m, sk_m).total);
}

void adam_consts(double lr, double beta1, double beta2, double eps, AdamArgs *a) {
  a->lr = (float)lr;
  a->b1 = (float)beta1;
  a->b2 = (float)beta2;
  // 1 - beta from FP64: 1 - (float)0.999 would be 1.3e-5 off 0.001
  a->omb1 = (float)(1.0 - beta1);
  a->omb2 = (float)(1.0 - beta2);
  a->eps = (float)eps;
  a->lnb1 = (float)std::log(beta1);
  a->lnb2 = (float)std::log(beta2);
}

template <typename T>
int ttt_step_impl(skei_plan p, const T *x0, float *theta, float *m, float *v, const int *step,
                  const T *y, int B, const int *mc_idx, int mc_m, const int *sk_idx, int sk_m,
                  const double *g_deg, int G, double lambda, double mc_scale, const AdamArgs &ad,
                  T *x1, T *r, T *x2, T *z, T *x3, T *g_x2, T *g_x3, T *g_x1, double *mc_out,
                  double *ei_out, double *loss_out, char *work, cudaStream_t st) {
  const int N = p->N;
  Residual<T> res;
  res.x0 = x0;
  res.theta = theta;
  res.x3 = x3;
  SKEI_TRY(ei_fwd_impl<T>(p, x1, y, B, mc_idx, mc_m, sk_idx, sk_m, g_deg, G, r, x2, z, work, st,
                          false, res));
  // loss partials (and the backward seeds g_x2, g_x3) into their own
  // workspace region: the final pass runs in the last launch
  const int64_t n_img = (int64_t)N * N;
  const int r_len = mc_m * p->n_det;
  const int cpi = (int)ceil_div((size_t)n_img, kChunk), cpr = (int)ceil_div((size_t)r_len, kChunk);
  double *partial = reinterpret_cast<double *>(work + ttt_loss_off(p, B, G, mc_m, sk_m));
  const float kappa = (float)(2.0 * lambda / ((double)B * G));
  launch_k(ei_partials_kernel<T>, dim3(B * G * cpi + B * cpr), dim3(kRedThreads), 0, st,
           (const T *)x2, (const T *)x3, (const T *)r, n_img, B * G, cpi, (int64_t)r_len, cpr,
           kappa, g_x2, g_x3, partial);
  SKEI_TRY(check_launch("loss partial sums launch"));
  const LossFinal lf{partial, B, G, cpi, cpr, lambda, mc_scale, mc_out, ei_out, loss_out};
  // F's Jacobian is the identity: dL/dz = dL/dx3
  const double mc_coef = mc_scale / B;
  if (B == 1) {
    SKEI_TRY(ei_bwd_impl<T>(p, r, g_x2, g_x3, B, mc_idx, mc_m, sk_idx, sk_m, g_deg, G, mc_coef,
                            g_x1, work, st, false, false));
    const EiWork w = ei_work(p, B, G, mc_m, sk_m);
    const float *gtot = reinterpret_cast<const float *>(work + 2 * w.p_bytes);
    return launch_rotate_adj_adam<T>(gtot, N, g_deg, G, g_x1, g_x3, ad, lf, st);
  }
  // several measurements share theta: the gradient sums over them, so the
  // update is a launch of its own
  SKEI_TRY(ei_bwd_impl<T>(p, r, g_x2, g_x3, B, mc_idx, mc_m, sk_idx, sk_m, g_deg, G, mc_coef,
                          g_x1, work, st));
  const size_t smem = sizeof(double) * (size_t)(B * G + B);
  launch_k(ei_final_kernel, dim3(1), dim3(kRedThreads), smem, st, (const double *)partial, B, G,
           cpi, cpr, lambda, mc_scale, mc_out, ei_out, loss_out);
  SKEI_TRY(check_launch("loss final reduction launch"));
  const int n = N * N;
  if (std::is_same<T, float>::value && n % 4 == 0) {
    launch_k(adam4_kernel, dim3(grid_for(n / 4, 256)), dim3(256), 0, st,
             reinterpret_cast<float4 *>(theta), n / 4, reinterpret_cast<const float4 *>(g_x1), B,
             reinterpret_cast<const float4 *>(g_x3), B * G, reinterpret_cast<float4 *>(m),
             reinterpret_cast<float4 *>(v), step, ad.lr, ad.b1, ad.b2, ad.omb1, ad.omb2, ad.eps,
             ad.lnb1, ad.lnb2);
  } else {
    launch_k(adam_kernel<T>, dim3(grid_for(n, 256)), dim3(256), 0, st, theta, (int64_t)n,
             (const T *)g_x1, B, (const T *)g_x3, B * G, m, v, step, ad.lr, ad.b1, ad.b2,
             ad.omb1, ad.omb2, ad.eps, ad.lnb1, ad.lnb2);
  }
  return check_launch("adam launch");
}

// --------------------------------------------------------- validation --

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

int check_common(skei_plan p, int dtype, int B) {
  SKEI_TRY(check_plan(p));
  SKEI_TRY(check_dtype(dtype));
  return check_batch(B);
}

int check_work(void *work, size_t have, size_t need) {
  if (need == 0) return SKEI_OK;
  SKEI_TRY(check_dev_ptr(work, "work"));
  if (have < need)
    return set_error(SKEI_EINVAL, "workspace of %zu bytes is smaller than the %zu needed", have,
                     need);
  return SKEI_OK;
}

int to_jobs(skei_plan plan, const skei_job *jobs, int njobs, bool fwd, Jobs *J) {
  if (!jobs || njobs < 1 || njobs > SKEI_MAX_JOBS)
    return set_error(SKEI_EINVAL, "njobs=%d outside [1, %d]", njobs, SKEI_MAX_JOBS);
  int total = 0;
  J->njobs = njobs;
  for (int q = 0; q < njobs; ++q) {
    const skei_job &s = jobs[q];
    SKEI_TRY(check_dtype(s.dtype_in));
    SKEI_TRY(check_dtype(s.dtype_out));
    SKEI_TRY(check_batch(s.B));
    SKEI_TRY(check_dev_ptr(s.in, "job.in"));
    SKEI_TRY(check_dev_ptr(s.out, "job.out"));
    SKEI_TRY(check_idx(plan, s.idx, s.m));
    const bool use_aux = fwd ? s.aux != nullptr : (s.aux != nullptr && s.beta != 0.0f);
    if (use_aux) {
      SKEI_TRY(check_dtype(s.dtype_aux));
      SKEI_TRY(check_dev_ptr(s.aux, "job.aux"));
    }
    total += s.B;
    J->j[q] = Job{s.in, use_aux ? s.aux : nullptr, s.out, s.idx, s.m, s.B,
                  fwd ? 1.0f : s.alpha, fwd ? 0.0f : (use_aux ? s.beta : 0.0f),
                  s.dtype_in == SKEI_BF16, s.dtype_aux == SKEI_BF16, s.dtype_out == SKEI_BF16};
  }
  if (total > 65535) return set_error(SKEI_EINVAL, "jobs hold %d images (max 65535)", total);
  return SKEI_OK;
}

int check_rot(int dtype, int B, int N, const double *g_deg, int G) {
  SKEI_TRY(check_dtype(dtype));
  SKEI_TRY(check_batch(B));
  if (N < 1 || N > SKEI_MAX_N) return set_error(SKEI_EINVAL, "N=%d outside [1, %d]", N, SKEI_MAX_N);
  if (G < 1 || (int64_t)B * G > 65535)
    return set_error(SKEI_EINVAL, "G=%d with B=%d: need G >= 1 and B*G <= 65535", G, B);
  return check_dev_ptr(g_deg, "g_deg");
}

}  // namespace
}  // namespace skei

using namespace skei;

extern "C" {

int skei_proj_fwd(skei_plan plan, int dtype, const void *x, int B, const int *idx, int m,
                  const void *y, void *out, void *stream) {
  SKEI_RANGE("skei_proj_fwd");
  SKEI_TRY(check_common(plan, dtype, B));
  SKEI_TRY(check_dev_ptr(x, "x"));
  SKEI_TRY(check_dev_ptr(out, "out"));
  if (y) SKEI_TRY(check_dev_ptr(y, "y"));
  SKEI_TRY(check_idx(plan, idx, m));
  if (dtype == SKEI_F32)
    return launch_proj_fwd<float, float>(plan, (const float *)x, B, idx, m, (const float *)y,
                                         (float *)out, as_stream(stream));
  return launch_proj_fwd<bf16, bf16>(plan, (const bf16 *)x, B, idx, m, (const bf16 *)y,
                                     (bf16 *)out, as_stream(stream));
}

int skei_proj_fwd_multi(skei_plan plan, const skei_job *jobs, int njobs, void *stream) {
  SKEI_RANGE("skei_proj_fwd_multi");
  SKEI_TRY(check_plan(plan));
  Jobs J{};
  SKEI_TRY(to_jobs(plan, jobs, njobs, true, &J));
  return launch_band_jobs(plan, OP_JOSEPH, J, as_stream(stream));
}

size_t skei_band_sums_workspace_size(skei_plan plan, const skei_job *jobs, int njobs) {
  if (check_plan(plan) || !jobs || njobs < 1 || njobs > SKEI_MAX_JOBS) return 0;
  Jobs J{};
  J.njobs = njobs;
  for (int q = 0; q < njobs; ++q) {
    if (jobs[q].B < 1 || jobs[q].m < 1) return 0;
    J.j[q].nimg = jobs[q].B;
    J.j[q].m = jobs[q].m;
  }
  return band_partial_floats(plan, J) * sizeof(float);
}

int skei_proj_fwd_multi_ws(skei_plan plan, const skei_job *jobs, int njobs, void *work,
                           size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_proj_fwd_multi_ws");
  SKEI_TRY(check_plan(plan));
  Jobs J{};
  SKEI_TRY(to_jobs(plan, jobs, njobs, true, &J));
  const size_t need = band_partial_floats(plan, J) * sizeof(float);
  SKEI_TRY(check_work(work, work_bytes, need));
  return launch_band_partial_jobs(plan, OP_JOSEPH, J, static_cast<float *>(work),
                                  work_bytes / sizeof(float), as_stream(stream));
}

int skei_backproject_adj_multi_ws(skei_plan plan, const skei_job *jobs, int njobs, void *work,
                                  size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_backproject_adj_multi_ws");
  SKEI_TRY(check_plan(plan));
  Jobs J{};
  SKEI_TRY(to_jobs(plan, jobs, njobs, false, &J));
  for (int q = 0; q < J.njobs; ++q) {
    J.j[q].aux = nullptr;
    J.j[q].beta = 0.0f;
  }
  const size_t need = band_partial_floats(plan, J) * sizeof(float);
  SKEI_TRY(check_work(work, work_bytes, need));
  return launch_band_partial_jobs(plan, OP_BP_ADJ, J, static_cast<float *>(work),
                                  work_bytes / sizeof(float), as_stream(stream));
}

int skei_proj_adj_multi(skei_plan plan, const skei_job *jobs, int njobs, void *stream) {
  SKEI_RANGE("skei_proj_adj_multi");
  SKEI_TRY(check_plan(plan));
  Jobs J{};
  SKEI_TRY(to_jobs(plan, jobs, njobs, false, &J));
  return launch_tile_jobs(plan, OP_JOSEPH_ADJ, J, as_stream(stream));
}

int skei_proj_adj(skei_plan plan, int dtype, const void *sino, int B, const int *idx, int m,
                  float alpha, float beta, void *x, void *stream) {
  SKEI_RANGE("skei_proj_adj");
  SKEI_TRY(check_common(plan, dtype, B));
  SKEI_TRY(check_dev_ptr(sino, "sino"));
  SKEI_TRY(check_dev_ptr(x, "x"));
  SKEI_TRY(check_idx(plan, idx, m));
  if (dtype == SKEI_F32)
    return launch_proj_adj<float, float, float>(plan, (const float *)sino, B, idx, m, alpha, beta,
                                                (const float *)x, (float *)x, as_stream(stream));
  return launch_proj_adj<bf16, bf16, bf16>(plan, (const bf16 *)sino, B, idx, m, alpha, beta,
                                           (const bf16 *)x, (bf16 *)x, as_stream(stream));
}

int skei_filter(skei_plan plan, int dtype, const void *p, int rows, float scale, void *q,
                void *stream) {
  SKEI_RANGE("skei_filter");
  SKEI_TRY(check_plan(plan));
  SKEI_TRY(check_dtype(dtype));
  if (rows < 1) return set_error(SKEI_EINVAL, "rows=%d must be >= 1", rows);
  SKEI_TRY(check_dev_ptr(p, "p"));
  SKEI_TRY(check_dev_ptr(q, "q"));
  if (dtype == SKEI_F32)
    return launch_filter<float, float>(plan, (const float *)p, rows, scale, (float *)q,
                                       as_stream(stream));
  return launch_filter<bf16, bf16>(plan, (const bf16 *)p, rows, scale, (bf16 *)q,
                                   as_stream(stream));
}

int skei_filter_fft(skei_plan plan, int dtype, const void *p, int rows, float scale, void *q,
                    void *stream) {
  SKEI_RANGE("skei_filter_fft");
  SKEI_TRY(check_plan(plan));
  SKEI_TRY(check_dtype(dtype));
  if (rows < 1) return set_error(SKEI_EINVAL, "rows=%d must be >= 1", rows);
  SKEI_TRY(check_dev_ptr(p, "p"));
  SKEI_TRY(check_dev_ptr(q, "q"));
  if (p == q) return set_error(SKEI_EINVAL, "filter: p and q must not alias");
  if (dtype == SKEI_F32)
    return launch_filter_fft<float, float>(plan, (const float *)p, rows, scale, (float *)q,
                                           as_stream(stream));
  return launch_filter_fft<bf16, bf16>(plan, (const bf16 *)p, rows, scale, (bf16 *)q,
                                       as_stream(stream));
}

int skei_filter_tc(skei_plan plan, int dtype, const void *p, int rows, float scale, void *q,
                   void *stream) {
  SKEI_RANGE("skei_filter_tc");
  SKEI_TRY(check_plan(plan));
  SKEI_TRY(check_dtype(dtype));
  if (rows < 1) return set_error(SKEI_EINVAL, "rows=%d must be >= 1", rows);
  SKEI_TRY(check_dev_ptr(p, "p"));
  SKEI_TRY(check_dev_ptr(q, "q"));
  if (p == q) return set_error(SKEI_EINVAL, "filter: p and q must not alias");
  if (dtype == SKEI_F32)
    return launch_filter_tc<float, float>(plan, (const float *)p, rows, scale, (float *)q,
                                          as_stream(stream));
  return launch_filter_tc<bf16, bf16>(plan, (const bf16 *)p, rows, scale, (bf16 *)q,
                                      as_stream(stream));
}

int skei_backproject(skei_plan plan, int dtype, const void *q, int B, const int *idx, int m,
                     float alpha, float beta, void *x, void *stream) {
  SKEI_RANGE("skei_backproject");
  SKEI_TRY(check_common(plan, dtype, B));
  SKEI_TRY(check_dev_ptr(q, "q"));
  SKEI_TRY(check_dev_ptr(x, "x"));
  SKEI_TRY(check_idx(plan, idx, m));
  if (dtype == SKEI_F32)
    return launch_backproject<float, float, float>(plan, (const float *)q, B, idx, m, alpha, beta,
                                                   (const float *)x, (float *)x,
                                                   as_stream(stream));
  return launch_backproject<bf16, bf16, bf16>(plan, (const bf16 *)q, B, idx, m, alpha, beta,
                                              (const bf16 *)x, (bf16 *)x, as_stream(stream));
}

int skei_backproject_adj(skei_plan plan, int dtype, const void *x, int B, const int *idx, int m,
                         float alpha, void *q, void *stream) {
  SKEI_RANGE("skei_backproject_adj");
  SKEI_TRY(check_common(plan, dtype, B));
  SKEI_TRY(check_dev_ptr(x, "x"));
  SKEI_TRY(check_dev_ptr(q, "q"));
  SKEI_TRY(check_idx(plan, idx, m));
  if (dtype == SKEI_F32)
    return launch_backproject_adj<float, float>(plan, (const float *)x, B, idx, m, alpha,
                                                (float *)q, as_stream(stream));
  return launch_backproject_adj<bf16, bf16>(plan, (const bf16 *)x, B, idx, m, alpha, (bf16 *)q,
                                            as_stream(stream));
}

size_t skei_fbp_workspace_size(skei_plan plan, int dtype, int B, int m) {
  if (check_plan(plan) || check_dtype(dtype) || B < 1 || m < 1) return 0;
  return align256((size_t)B * m * plan->n_det * sizeof(float));
}

int skei_fbp(skei_plan plan, int dtype, const void *sino, int B, const int *idx, int m, void *x,
             void *work, size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_fbp");
  SKEI_TRY(check_common(plan, dtype, B));
  SKEI_TRY(check_dev_ptr(sino, "sino"));
  SKEI_TRY(check_dev_ptr(x, "x"));
  SKEI_TRY(check_idx(plan, idx, m));
  SKEI_TRY(check_work(work, work_bytes, skei_fbp_workspace_size(plan, dtype, B, m)));
  if (dtype == SKEI_F32)
    return fbp_impl<float>(plan, (const float *)sino, B, idx, m, (float *)x, (float *)work,
                           as_stream(stream));
  return fbp_impl<bf16>(plan, (const bf16 *)sino, B, idx, m, (bf16 *)x, (float *)work,
                        as_stream(stream));
}

int skei_fbp_adj(skei_plan plan, int dtype, const void *x, int B, const int *idx, int m,
                 void *sino, void *work, size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_fbp_adj");
  SKEI_TRY(check_common(plan, dtype, B));
  SKEI_TRY(check_dev_ptr(x, "x"));
  SKEI_TRY(check_dev_ptr(sino, "sino"));
  SKEI_TRY(check_idx(plan, idx, m));
  SKEI_TRY(check_work(work, work_bytes, skei_fbp_workspace_size(plan, dtype, B, m)));
  if (dtype == SKEI_F32)
    return fbp_adj_impl<float>(plan, (const float *)x, B, idx, m, (float *)sino, (float *)work,
                               as_stream(stream));
  return fbp_adj_impl<bf16>(plan, (const bf16 *)x, B, idx, m, (bf16 *)sino, (float *)work,
                            as_stream(stream));
}

int skei_rotate_channels(int dtype, const void *x, int B, int Ch, int N, const double *g_deg,
                         int G, void *out, void *stream) {
  SKEI_RANGE("skei_rotate_channels");
  SKEI_TRY(check_rot(dtype, B, N, g_deg, G));
  if (Ch < 1 || (int64_t)B * G * Ch > 65535)
    return set_error(SKEI_EINVAL, "rotation: Ch=%d outside [1, 65535 / (B G)]", Ch);
  SKEI_TRY(check_dev_ptr(x, "x"));
  SKEI_TRY(check_dev_ptr(out, "out"));
  if (dtype == SKEI_F32)
    return launch_rotate<float, float>((const float *)x, B, N, g_deg, G, (float *)out,
                                       as_stream(stream), Ch);
  return launch_rotate<bf16, bf16>((const bf16 *)x, B, N, g_deg, G, (bf16 *)out,
                                   as_stream(stream), Ch);
}

int skei_rotate(int dtype, const void *x, int B, int N, const double *g_deg, int G, void *out,
                void *stream) {
  SKEI_RANGE("skei_rotate");
  return skei_rotate_channels(dtype, x, B, 1, N, g_deg, G, out, stream);
}

int skei_rotate_adj_channels(int dtype, const void *gout, int B, int Ch, int N,
                             const double *g_deg, int G, float alpha, float beta, void *gx,
                             void *stream) {
  SKEI_RANGE("skei_rotate_adj_channels");
  SKEI_TRY(check_rot(dtype, B, N, g_deg, G));
  if (Ch < 1 || (int64_t)B * Ch > 65535)
    return set_error(SKEI_EINVAL, "rotation transpose: Ch=%d outside [1, 65535 / B]", Ch);
  SKEI_TRY(check_dev_ptr(gout, "gout"));
  SKEI_TRY(check_dev_ptr(gx, "gx"));
  if (dtype == SKEI_F32)
    return launch_rotate_adj<float, float>((const float *)gout, B, N, g_deg, G, alpha, beta,
                                           (float *)gx, as_stream(stream), Ch);
  return launch_rotate_adj<bf16, bf16>((const bf16 *)gout, B, N, g_deg, G, alpha, beta,
                                       (bf16 *)gx, as_stream(stream), Ch);
}

int skei_rotate_adj(int dtype, const void *gout, int B, int N, const double *g_deg, int G,
                    float alpha, float beta, void *gx, void *stream) {
  SKEI_RANGE("skei_rotate_adj");
  return skei_rotate_adj_channels(dtype, gout, B, 1, N, g_deg, G, alpha, beta, gx, stream);
}

size_t skei_ei_workspace_size(skei_plan plan, int dtype, int B, int G, int mc_m, int sk_m) {
  if (check_plan(plan) || check_dtype(dtype) || B < 1 || G < 1 || mc_m < 1 || sk_m < 1) return 0;
  return ei_work(plan, B, G, mc_m, sk_m).total;
}

int skei_ei_fwd_form(skei_plan plan, int B, int G, const int *mc_idx, int mc_m,
                     const int *sk_idx, int sk_m, int per_sample) {
  if (check_plan(plan) || B < 1 || G < 1 || mc_m < 1 || sk_m < 1 || mc_m > plan->n_angles ||
      sk_m > plan->n_angles)
    return set_error(SKEI_EINVAL, "skei_ei_fwd_form: bad arguments");
  const Jobs J = ei_fwd_jobs(nullptr, nullptr, nullptr, B, mc_idx, mc_m, nullptr, nullptr, sk_idx,
                             sk_m, G, 0, per_sample != 0);
  return ei_fwd_sums(plan, ei_work(plan, B, G, mc_m, sk_m), J) ? 1 : 0;
}

static int ei_fwd_entry(skei_plan plan, int dtype, const void *x1, const void *y, int B,
                        const int *mc_idx, int mc_m, const int *sk_idx, int sk_m,
                        const double *g_deg, int G, void *r, void *x2, void *z, void *work,
                        size_t work_bytes, void *stream, bool per_sample) {
  SKEI_TRY(check_common(plan, dtype, B));
  SKEI_TRY(check_rot(dtype, B, plan->N, g_deg, G));
  SKEI_TRY(check_dev_ptr(x1, "x1"));
  SKEI_TRY(check_dev_ptr(y, "y"));
  SKEI_TRY(check_dev_ptr(r, "r"));
  SKEI_TRY(check_dev_ptr(x2, "x2"));
  SKEI_TRY(check_dev_ptr(z, "z"));
  SKEI_TRY(check_idx(plan, mc_idx, mc_m));
  SKEI_TRY(check_idx(plan, sk_idx, sk_m));
  SKEI_TRY(check_work(work, work_bytes, skei_ei_workspace_size(plan, dtype, B, G, mc_m, sk_m)));
  if (dtype == SKEI_F32)
    return ei_fwd_impl<float>(plan, (const float *)x1, (const float *)y, B, mc_idx, mc_m, sk_idx,
                              sk_m, g_deg, G, (float *)r, (float *)x2, (float *)z, (char *)work,
                              as_stream(stream), per_sample);
  return ei_fwd_impl<bf16>(plan, (const bf16 *)x1, (const bf16 *)y, B, mc_idx, mc_m, sk_idx, sk_m,
                           g_deg, G, (bf16 *)r, (bf16 *)x2, (bf16 *)z, (char *)work,
                           as_stream(stream), per_sample);
}

int skei_ei_loss_fwd(skei_plan plan, int dtype, const void *x1, const void *y, int B,
                     const int *mc_idx, int mc_m, const int *sk_idx, int sk_m,
                     const double *g_deg, int G, void *r, void *x2, void *z, void *work,
                     size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_ei_loss_fwd");
  return ei_fwd_entry(plan, dtype, x1, y, B, mc_idx, mc_m, sk_idx, sk_m, g_deg, G, r, x2, z,
                      work, work_bytes, stream, false);
}

int skei_ei_loss_fwd_per_sample(skei_plan plan, int dtype, const void *x1, const void *y, int B,
                                const int *mc_idx, int mc_m, const int *sk_idx, int sk_m,
                                const double *g_deg, int G, void *r, void *x2, void *z,
                                void *work, size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_ei_loss_fwd_per_sample");
  return ei_fwd_entry(plan, dtype, x1, y, B, mc_idx, mc_m, sk_idx, sk_m, g_deg, G, r, x2, z,
                      work, work_bytes, stream, true);
}

size_t skei_ei_finish_len_workspace_size(int B, int G, int64_t img_len, int r_len) {
  if (B < 1 || G < 1 || img_len < 1 || r_len < 1) return 0;
  return align256(((size_t)B * G * ceil_div((size_t)img_len, kChunk) +
                   (size_t)B * ceil_div((size_t)r_len, kChunk)) * sizeof(double));
}

size_t skei_ei_finish_workspace_size(int B, int G, int N, int r_len) {
  if (N < 1) return 0;
  return skei_ei_finish_len_workspace_size(B, G, (int64_t)N * N, r_len);
}

int skei_ei_loss_finish_len(int dtype, const void *x2, const void *x3, const void *r, int B,
                            int G, int64_t img_len, int r_len, double lambda, double mc_scale,
                            double *mc_out, double *ei_out, double *loss_out, void *g_x2,
                            void *g_x3, void *work, size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_ei_loss_finish_len");
  SKEI_TRY(check_dtype(dtype));
  SKEI_TRY(check_batch(B));
  if (G < 1 || (int64_t)B * G > 65535) return set_error(SKEI_EINVAL, "bad G=%d", G);
  if (img_len < 1 || img_len > ((int64_t)1 << 31))
    return set_error(SKEI_EINVAL, "img_len=%lld outside [1, 2^31]", (long long)img_len);
  if (r_len < 1) return set_error(SKEI_EINVAL, "r_len=%d must be >= 1", r_len);
  SKEI_TRY(check_dev_ptr(x2, "x2"));
  SKEI_TRY(check_dev_ptr(x3, "x3"));
  SKEI_TRY(check_dev_ptr(r, "r"));
  if (g_x2) SKEI_TRY(check_dev_ptr(g_x2, "g_x2"));
  if (g_x3) SKEI_TRY(check_dev_ptr(g_x3, "g_x3"));
  if (mc_out && (reinterpret_cast<uintptr_t>(mc_out) % 8)) return set_error(SKEI_EINVAL, "mc_out misaligned");
  if (ei_out && (reinterpret_cast<uintptr_t>(ei_out) % 8)) return set_error(SKEI_EINVAL, "ei_out misaligned");
  if (loss_out && (reinterpret_cast<uintptr_t>(loss_out) % 8)) return set_error(SKEI_EINVAL, "loss_out misaligned");
  SKEI_TRY(check_work(work, work_bytes,
                      skei_ei_finish_len_workspace_size(B, G, img_len, r_len)));
  if (dtype == SKEI_F32)
    return ei_finish_impl<float>((const float *)x2, (const float *)x3, (const float *)r, B, G,
                                 img_len, r_len, lambda, mc_scale, mc_out, ei_out, loss_out,
                                 (float *)g_x2, (float *)g_x3, (char *)work, as_stream(stream));
  return ei_finish_impl<bf16>((const bf16 *)x2, (const bf16 *)x3, (const bf16 *)r, B, G,
                              img_len, r_len, lambda, mc_scale, mc_out, ei_out, loss_out,
                              (bf16 *)g_x2, (bf16 *)g_x3, (char *)work, as_stream(stream));
}

int skei_ei_loss_finish(int dtype, const void *x2, const void *x3, const void *r, int B, int G,
                        int N, int r_len, double lambda, double mc_scale, double *mc_out,
                        double *ei_out, double *loss_out, void *g_x2, void *g_x3, void *work,
                        size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_ei_loss_finish");
  if (N < 1 || N > SKEI_MAX_N) return set_error(SKEI_EINVAL, "N=%d outside [1, %d]", N, SKEI_MAX_N);
  return skei_ei_loss_finish_len(dtype, x2, x3, r, B, G, (int64_t)N * N, r_len, lambda, mc_scale,
                                 mc_out, ei_out, loss_out, g_x2, g_x3, work, work_bytes, stream);
}

static int ei_bwd_entry(skei_plan plan, int dtype, const void *r, const void *g_x2,
                        const void *g_z, int B, const int *mc_idx, int mc_m, const int *sk_idx,
                        int sk_m, const double *g_deg, int G, double mc_coef, void *g_x1,
                        void *work, size_t work_bytes, void *stream, bool per_sample) {
  SKEI_TRY(check_common(plan, dtype, B));
  SKEI_TRY(check_rot(dtype, B, plan->N, g_deg, G));
  SKEI_TRY(check_dev_ptr(r, "r"));
  SKEI_TRY(check_dev_ptr(g_x1, "g_x1"));
  if (g_x2) SKEI_TRY(check_dev_ptr(g_x2, "g_x2"));
  if (g_z) SKEI_TRY(check_dev_ptr(g_z, "g_z"));
  SKEI_TRY(check_idx(plan, mc_idx, mc_m));
  SKEI_TRY(check_idx(plan, sk_idx, sk_m));
  SKEI_TRY(check_work(work, work_bytes, skei_ei_workspace_size(plan, dtype, B, G, mc_m, sk_m)));
  if (dtype == SKEI_F32)
    return ei_bwd_impl<float>(plan, (const float *)r, (const float *)g_x2, (const float *)g_z, B,
                              mc_idx, mc_m, sk_idx, sk_m, g_deg, G, mc_coef, (float *)g_x1,
                              (char *)work, as_stream(stream), per_sample);
  return ei_bwd_impl<bf16>(plan, (const bf16 *)r, (const bf16 *)g_x2, (const bf16 *)g_z, B, mc_idx,
                           mc_m, sk_idx, sk_m, g_deg, G, mc_coef, (bf16 *)g_x1, (char *)work,
                           as_stream(stream), per_sample);
}

int skei_ei_loss_bwd(skei_plan plan, int dtype, const void *r, const void *g_x2, const void *g_z,
                     int B, const int *mc_idx, int mc_m, const int *sk_idx, int sk_m,
                     const double *g_deg, int G, double mc_coef, void *g_x1, void *work,
                     size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_ei_loss_bwd");
  return ei_bwd_entry(plan, dtype, r, g_x2, g_z, B, mc_idx, mc_m, sk_idx, sk_m, g_deg, G,
                      mc_coef, g_x1, work, work_bytes, stream, false);
}

int skei_ei_loss_bwd_per_sample(skei_plan plan, int dtype, const void *r, const void *g_x2,
                                const void *g_z, int B, const int *mc_idx, int mc_m,
                                const int *sk_idx, int sk_m, const double *g_deg, int G,
                                double mc_coef, void *g_x1, void *work, size_t work_bytes,
                                void *stream) {
  SKEI_RANGE("skei_ei_loss_bwd_per_sample");
  return ei_bwd_entry(plan, dtype, r, g_x2, g_z, B, mc_idx, mc_m, sk_idx, sk_m, g_deg, G,
                      mc_coef, g_x1, work, work_bytes, stream, true);
}

size_t skei_ttt_residual_workspace_size(skei_plan plan, int dtype, int B, int G, int mc_m,
                                        int sk_m) {
  if (check_plan(plan) || check_dtype(dtype) || B < 1 || G < 1 || mc_m < 1 || sk_m < 1) return 0;
  return ttt_loss_off(plan, B, G, mc_m, sk_m) +
         skei_ei_finish_len_workspace_size(B, G, (int64_t)plan->N * plan->N, mc_m * plan->n_det);
}

int skei_ttt_residual_step(skei_plan plan, int dtype, const void *x0, float *theta, float *m,
                           float *v, const int *step, const void *y, int B, const int *mc_idx,
                           int mc_m, const int *sk_idx, int sk_m, const double *g_deg, int G,
                           double lambda, double mc_scale, double lr, double beta1, double beta2,
                           double eps, void *x1, void *r, void *x2, void *z, void *x3, void *g_x2,
                           void *g_x3, void *g_x1, double *mc_out, double *ei_out,
                           double *loss_out, void *work, size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_ttt_residual_step");
  SKEI_TRY(check_common(plan, dtype, B));
  SKEI_TRY(check_rot(dtype, B, plan->N, g_deg, G));
  const void *ptrs[] = {x0, theta, m, v, y, x1, r, x2, z, x3, g_x2, g_x3, g_x1};
  const char *names[] = {"x0", "theta", "m", "v", "y", "x1", "r", "x2", "z", "x3", "g_x2",
                         "g_x3", "g_x1"};
  for (int i = 0; i < 13; ++i) SKEI_TRY(check_dev_ptr(ptrs[i], names[i]));
  if (!step || reinterpret_cast<uintptr_t>(step) % 4)
    return set_error(SKEI_EINVAL, "step is NULL or misaligned");
  for (const double *q : {mc_out, ei_out, loss_out})
    if (q && reinterpret_cast<uintptr_t>(q) % 8) return set_error(SKEI_EINVAL, "a loss output is misaligned");
  if (!(beta1 > 0.0 && beta1 < 1.0 && beta2 > 0.0 && beta2 < 1.0))
    return set_error(SKEI_EINVAL, "Adam betas must lie in (0, 1)");
  if (!mc_idx) mc_m = plan->n_angles;
  if (!sk_idx) sk_m = plan->n_angles;
  SKEI_TRY(check_idx(plan, mc_idx, mc_m));
  SKEI_TRY(check_idx(plan, sk_idx, sk_m));
  SKEI_TRY(check_work(work, work_bytes,
                      skei_ttt_residual_workspace_size(plan, dtype, B, G, mc_m, sk_m)));
  AdamArgs ad{theta, m, v, step};
  adam_consts(lr, beta1, beta2, eps, &ad);
  cudaStream_t st = as_stream(stream);
  if (dtype == SKEI_F32)
    return ttt_step_impl<float>(plan, (const float *)x0, theta, m, v, step, (const float *)y, B,
                                mc_idx, mc_m, sk_idx, sk_m, g_deg, G, lambda, mc_scale, ad,
                                (float *)x1, (float *)r, (float *)x2, (float *)z, (float *)x3,
                                (float *)g_x2, (float *)g_x3, (float *)g_x1, mc_out, ei_out,
                                loss_out, (char *)work, st);
  return ttt_step_impl<bf16>(plan, (const bf16 *)x0, theta, m, v, step, (const bf16 *)y, B, mc_idx,
                             mc_m, sk_idx, sk_m, g_deg, G, lambda, mc_scale, ad, (bf16 *)x1,
                             (bf16 *)r, (bf16 *)x2, (bf16 *)z, (bf16 *)x3, (bf16 *)g_x2,
                             (bf16 *)g_x3, (bf16 *)g_x1, mc_out, ei_out, loss_out, (char *)work,
                             st);
}

int skei_residual_add(int dtype, const void *u, const float *theta, int count, int64_t n,
                      void *out, void *stream) {
  SKEI_RANGE("skei_residual_add");
  SKEI_TRY(check_dtype(dtype));
  if (count < 1 || n < 1) return set_error(SKEI_EINVAL, "count=%d, n=%lld must be >= 1", count, (long long)n);
  SKEI_TRY(check_dev_ptr(u, "u"));
  SKEI_TRY(check_dev_ptr(theta, "theta"));
  SKEI_TRY(check_dev_ptr(out, "out"));
  if (n > (int64_t)1 << 30 || count > 65535)
    return set_error(SKEI_EINVAL, "residual add: n=%lld or count=%d too large", (long long)n, count);
  const dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 1024), (unsigned)count);
  if (dtype == SKEI_F32 && n % 4 == 0) {
    const dim3 grid4((unsigned)std::min<int64_t>((n / 4 + 255) / 256, 1024), (unsigned)count);
    launch_k(residual_add4_kernel, grid4, dim3(256), 0, as_stream(stream), (const float4 *)u,
             (const float4 *)theta, (int)(n / 4), (float4 *)out);
  } else if (dtype == SKEI_F32)
    launch_k(residual_add_kernel<float>, grid, dim3(256), 0, as_stream(stream), (const float *)u,
             theta, (int)n, (float *)out);
  else
    launch_k(residual_add_kernel<bf16>, grid, dim3(256), 0, as_stream(stream), (const bf16 *)u,
             theta, (int)n, (bf16 *)out);
  return check_launch("residual add launch");
}

int skei_step_draws(const void *table, int n_rows, int64_t row_bytes, int *counter, void *dst,
                    void *stream) {
  SKEI_RANGE("skei_step_draws");
  if (n_rows < 1 || row_bytes < 1)
    return set_error(SKEI_EINVAL, "step draws: n_rows=%d, row_bytes=%lld must be >= 1", n_rows,
                     (long long)row_bytes);
  SKEI_TRY(check_dev_ptr(table, "table"));
  SKEI_TRY(check_dev_ptr(dst, "dst"));
  if (!counter || reinterpret_cast<uintptr_t>(counter) % 4)
    return set_error(SKEI_EINVAL, "counter is NULL or misaligned");
  const bool vec = row_bytes % 16 == 0 && reinterpret_cast<uintptr_t>(table) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(dst) % 16 == 0;
  if (vec)
    launch_k(step_draws_kernel<uint4>, dim3(1), dim3(256), 0, as_stream(stream),
             (const uint4 *)table, n_rows, row_bytes / 16, counter, (uint4 *)dst);
  else
    launch_k(step_draws_kernel<unsigned char>, dim3(1), dim3(256), 0, as_stream(stream),
             (const unsigned char *)table, n_rows, row_bytes, counter, (unsigned char *)dst);
  return check_launch("step draws launch");
}

int skei_adam_step(float *theta, int64_t n, int dtype, const void *g1, int c1, const void *g2,
                   int c2, float *m, float *v, const int *step, double lr, double beta1,
                   double beta2, double eps, void *stream) {
  SKEI_RANGE("skei_adam_step");
  SKEI_TRY(check_dtype(dtype));
  if (n < 1 || c1 < 1 || c2 < 0) return set_error(SKEI_EINVAL, "bad sizes n=%lld c1=%d c2=%d", (long long)n, c1, c2);
  SKEI_TRY(check_dev_ptr(theta, "theta"));
  SKEI_TRY(check_dev_ptr(g1, "g1"));
  if (c2 > 0) SKEI_TRY(check_dev_ptr(g2, "g2"));
  SKEI_TRY(check_dev_ptr(m, "m"));
  SKEI_TRY(check_dev_ptr(v, "v"));
  if (!step || reinterpret_cast<uintptr_t>(step) % 4) return set_error(SKEI_EINVAL, "step is NULL or misaligned");
  if (!(beta1 > 0.0 && beta1 < 1.0 && beta2 > 0.0 && beta2 < 1.0))
    return set_error(SKEI_EINVAL, "Adam betas must lie in (0, 1)");
  const int grid = grid_for(n, 256);
  const float lnb1 = (float)std::log(beta1), lnb2 = (float)std::log(beta2);
  // 1 - beta from FP64: 1 - (float)0.999 would be 1.3e-5 off 0.001
  const float omb1 = (float)(1.0 - beta1), omb2 = (float)(1.0 - beta2);
  const bool vec = dtype == SKEI_F32 && n % 4 == 0 && n / 4 < (int64_t)1 << 30 &&
                   ((reinterpret_cast<uintptr_t>(g2) & 15) == 0);
  if (vec)
    launch_k(adam4_kernel, dim3(grid_for(n / 4, 256)), dim3(256), 0, as_stream(stream),
             (float4 *)theta, (int)(n / 4), (const float4 *)g1, c1, (const float4 *)g2, c2,
             (float4 *)m, (float4 *)v, step, (float)lr, (float)beta1, (float)beta2, omb1, omb2,
             (float)eps, lnb1, lnb2);
  else if (dtype == SKEI_F32)
    launch_k(adam_kernel<float>, dim3(grid), dim3(256), 0, as_stream(stream), theta, n,
             (const float *)g1, c1, (const float *)g2, c2, m, v, step, (float)lr, (float)beta1,
             (float)beta2, omb1, omb2, (float)eps, lnb1, lnb2);
  else
    launch_k(adam_kernel<bf16>, dim3(grid), dim3(256), 0, as_stream(stream), theta, n,
             (const bf16 *)g1, c1, (const bf16 *)g2, c2, m, v, step, (float)lr, (float)beta1,
             (float)beta2, omb1, omb2, (float)eps, lnb1, lnb2);
  return check_launch("adam launch");
}

}  // extern "C"
