// Multi-coil MRI operators of the coil-sketched EI (Sec. 3.4, Eq. (e:mri)):
//   A x = M F (C x):  k_c = M (F (C_c x)),  c = 1 .. N_c,
// with C_c the coil sensitivity maps, F the unitary 2D DFT of an N x N image
// (sum_{p,q} s[p][q] e^{-2 pi i (u p + v q) / N} / N) and M a 0/1 sampling
// mask shared by the coils; the adjoint
//   A^H k = sum_c conj(C_c) F^H (M k_c),
// its coil-combined inverse A^dagger k = D^-1 A^H k (D = sum_c |C_c|^2, 0
// where D = 0), and the coil mixing out_j = sum_i W_ji in_i that forms the
// PCA virtual coils and the coil sketch S_c.
//
// Complex data are planar: an image is [2][N][N] (real plane, imaginary
// plane), k-space [N_c][2][N][N], maps [N_c][2][N][N].  A 2D DFT is two
// passes through an L2-resident interleaved workspace: one CTA per group of
// rows (then of columns) of one (image, coil) plane, each running a
// radix-2 Stockham FFT in shared memory, so that one image already spreads
// over N / 8 x N_c CTAs.  N is a power of two in [8, 256].
#include "fft.cuh"

namespace skei {
namespace {

constexpr int kMriThreads = 256;
constexpr int kCpc = 16;   // columns per CTA in the column pass (128-byte rows of float2;
                           // N when N < 16)

struct MriArgs {
  int N, Nc, rpc, cpc;     // rows per CTA in the row pass, columns in the column pass
  const float *x;          // image [B][2][N][N] (forward input / adjoint output)
  const float *maps;       // [Nc][2][N][N]
  const float *mask;       // [N][N] or NULL (all sampled)
  const float *xw;         // forward: real weight [N][N] on x, or NULL
  const float *aux;        // forward: k - A x residual base [B][Nc][2][N][N], or NULL
  float *k;                // k-space [B][Nc][2][N][N]
  float2 *T;               // workspace [B][Nc][N][N] interleaved
  float *W;                // adjoint per-coil images [B][Nc][2][N][N]
  float alpha;
};

// Forward row pass: s = C_c x_b, FFT along each row -> T.
__global__ void __launch_bounds__(kMriThreads) mri_fwd_rows_kernel(const MriArgs a) {
  pdl_enter();
  extern __shared__ float2 sm[];
  const int N = a.N, rpc = a.rpc, r0 = blockIdx.x * rpc, c = blockIdx.y, b = blockIdx.z;
  const int ld = N + 1;
  float2 *tw = sm, *A = sm + N / 2, *Bf = A + rpc * ld;
  twiddles(tw, N);
  const size_t plane = (size_t)N * N;
  const float *xr = a.x + (size_t)b * 2 * plane, *xi = xr + plane;
  const float *cr = a.maps + (size_t)c * 2 * plane, *ci = cr + plane;
  for (int e = threadIdx.x; e < rpc * N; e += blockDim.x) {
    const int r = e / N, q = e - r * N;
    const size_t o = (size_t)(r0 + r) * N + q;
    const float w = a.xw ? __ldg(a.xw + o) : 1.0f;
    A[r * ld + q] = cmul(make_float2(__ldg(cr + o), __ldg(ci + o)),
                         make_float2(w * __ldg(xr + o), w * __ldg(xi + o)));
  }
  __syncthreads();
  const float2 *R = fft_smem(A, Bf, N, rpc, ld, 1, tw, false, false);
  float2 *T = a.T + ((size_t)b * a.Nc + c) * plane;
  for (int e = threadIdx.x; e < rpc * N; e += blockDim.x) {
    const int r = e / N, q = e - r * N;
    T[(size_t)(r0 + r) * N + q] = R[r * ld + q];
  }
}

// Forward column pass: FFT along each column of T, times 1/N (unitary),
// mask, residual and scale -> k (planar).
__global__ void __launch_bounds__(kMriThreads) mri_fwd_cols_kernel(const MriArgs a) {
  pdl_enter();
  extern __shared__ float2 sm[];
  const int N = a.N, cpc = a.cpc, q0 = blockIdx.x * cpc, c = blockIdx.y, b = blockIdx.z;
  float2 *tw = sm, *A = sm + N / 2, *Bf = A + N * cpc;
  twiddles(tw, N);
  const size_t plane = (size_t)N * N;
  const float2 *T = a.T + ((size_t)b * a.Nc + c) * plane;
  for (int e = threadIdx.x; e < N * cpc; e += blockDim.x) {
    const int p = e / cpc, s = e - p * cpc;
    A[p * cpc + s] = T[(size_t)p * N + q0 + s];
  }
  __syncthreads();
  const float2 *R = fft_smem(A, Bf, N, cpc, 1, cpc, tw, false, true);
  const float sc = 1.0f / (float)N;
  const size_t ko = ((size_t)b * a.Nc + c) * 2 * plane;
  float *kr = a.k + ko, *ki = kr + plane;
  for (int e = threadIdx.x; e < N * cpc; e += blockDim.x) {
    const int p = e / cpc, s = e - p * cpc;
    const size_t o = (size_t)p * N + q0 + s;
    const float m = a.mask ? __ldg(a.mask + o) : 1.0f;
    float re = R[p * cpc + s].x * sc * m, im = R[p * cpc + s].y * sc * m;
    if (a.aux) {
      re = __ldg(a.aux + ko + o) - re;
      im = __ldg(a.aux + ko + plane + o) - im;
    }
    kr[o] = a.alpha * re;
    ki[o] = a.alpha * im;
  }
}

// Adjoint column pass: M k_c, inverse FFT along each column -> T.
__global__ void __launch_bounds__(kMriThreads) mri_adj_cols_kernel(const MriArgs a) {
  pdl_enter();
  extern __shared__ float2 sm[];
  const int N = a.N, cpc = a.cpc, q0 = blockIdx.x * cpc, c = blockIdx.y, b = blockIdx.z;
  float2 *tw = sm, *A = sm + N / 2, *Bf = A + N * cpc;
  twiddles(tw, N);
  const size_t plane = (size_t)N * N;
  const float *kr = a.k + ((size_t)b * a.Nc + c) * 2 * plane, *ki = kr + plane;
  for (int e = threadIdx.x; e < N * cpc; e += blockDim.x) {
    const int p = e / cpc, s = e - p * cpc;
    const size_t o = (size_t)p * N + q0 + s;
    const float m = a.mask ? __ldg(a.mask + o) : 1.0f;
    A[p * cpc + s] = make_float2(__ldg(kr + o) * m, __ldg(ki + o) * m);
  }
  __syncthreads();
  const float2 *R = fft_smem(A, Bf, N, cpc, 1, cpc, tw, true, true);
  float2 *T = a.T + ((size_t)b * a.Nc + c) * plane;
  for (int e = threadIdx.x; e < N * cpc; e += blockDim.x) {
    const int p = e / cpc, s = e - p * cpc;
    T[(size_t)p * N + q0 + s] = R[p * cpc + s];
  }
}

// Adjoint row pass: inverse FFT along each row of T, times 1/N, times
// conj(C_c) -> the coil's image W[b][c] (planar).
__global__ void __launch_bounds__(kMriThreads) mri_adj_rows_kernel(const MriArgs a) {
  pdl_enter();
  extern __shared__ float2 sm[];
  const int N = a.N, rpc = a.rpc, r0 = blockIdx.x * rpc, c = blockIdx.y, b = blockIdx.z;
  const int ld = N + 1;
  float2 *tw = sm, *A = sm + N / 2, *Bf = A + rpc * ld;
  twiddles(tw, N);
  const size_t plane = (size_t)N * N;
  const float2 *T = a.T + ((size_t)b * a.Nc + c) * plane;
  for (int e = threadIdx.x; e < rpc * N; e += blockDim.x) {
    const int r = e / N, q = e - r * N;
    A[r * ld + q] = T[(size_t)(r0 + r) * N + q];
  }
  __syncthreads();
  const float2 *R = fft_smem(A, Bf, N, rpc, ld, 1, tw, true, false);
  const float sc = 1.0f / (float)N;
  const float *cr = a.maps + (size_t)c * 2 * plane, *ci = cr + plane;
  float *wr = a.W + ((size_t)b * a.Nc + c) * 2 * plane, *wi = wr + plane;
  for (int e = threadIdx.x; e < rpc * N; e += blockDim.x) {
    const int r = e / N, q = e - r * N;
    const size_t o = (size_t)(r0 + r) * N + q;
    const float2 v = cmulc(R[r * ld + q], make_float2(__ldg(cr + o), __ldg(ci + o)));
    wr[o] = v.x * sc;
    wi[o] = v.y * sc;
  }
}

// x[b] = alpha dinv sum_c W[b][c] + beta x[b], coils in order; planar.
__global__ void mri_coil_sum_kernel(const float *W, int Nc, int plane, const float *dinv,
                                    float alpha, float beta, float *x) {
  pdl_enter();
  const int b = blockIdx.y;
  const size_t n2 = 2 * (size_t)plane;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * plane;
       e += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < Nc; ++c) s += __ldg(W + ((size_t)b * Nc + c) * n2 + e);
    if (dinv) s *= __ldg(dinv + (e < plane ? e : e - plane));
    float v = alpha * s;
    const size_t o = (size_t)b * n2 + e;
    if (beta != 0.0f) v = fmaf(beta, x[o], v);
    x[o] = v;
  }
}

// out[b][j] = sum_i Wm[j][i] in[b][i], complex weights Wm [n_out][n_in][2].
__global__ void coil_mix_kernel(const float *in, int n_in, int n_out, int plane,
                                const float *Wm, float *out) {
  pdl_enter();
  extern __shared__ float2 wsm[];
  for (int t = threadIdx.x; t < n_in * n_out; t += blockDim.x)
    wsm[t] = make_float2(Wm[2 * t], Wm[2 * t + 1]);
  __syncthreads();
  const int b = blockIdx.y;
  const float *ib = in + (size_t)b * n_in * 2 * plane;
  float *ob = out + (size_t)b * n_out * 2 * plane;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < plane; p += gridDim.x * blockDim.x) {
    for (int j = 0; j < n_out; ++j) {
      float2 s = make_float2(0.0f, 0.0f);
      for (int i = 0; i < n_in; ++i) {
        const float2 v = make_float2(__ldg(ib + (size_t)i * 2 * plane + p),
                                     __ldg(ib + (size_t)i * 2 * plane + plane + p));
        const float2 w = wsm[j * n_in + i];
        s.x = fmaf(w.x, v.x, fmaf(-w.y, v.y, s.x));
        s.y = fmaf(w.x, v.y, fmaf(w.y, v.x, s.y));
      }
      ob[(size_t)j * 2 * plane + p] = s.x;
      ob[(size_t)j * 2 * plane + plane + p] = s.y;
    }
  }
}

// dinv[p] = 1 / sum_c |C_c[p]|^2, or 0 where the sum is 0.
__global__ void mri_dinv_kernel(const float *maps, int Nc, int plane, float *dinv) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < plane; p += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < Nc; ++c) {
      const float re = __ldg(maps + (size_t)c * 2 * plane + p);
      const float im = __ldg(maps + (size_t)c * 2 * plane + plane + p);
      s = fmaf(re, re, fmaf(im, im, s));
    }
    dinv[p] = s > 0.0f ? 1.0f / s : 0.0f;
  }
}

int mri_check(int N, int Nc, int B) {
  if (N < 8 || N > 256 || (N & (N - 1)))
    return set_error(SKEI_EINVAL, "MRI: N=%d must be a power of two in [8, 256]", N);
  if (Nc < 1 || Nc > 64) return set_error(SKEI_EINVAL, "MRI: Nc=%d outside [1, 64]", Nc);
  if (B < 1 || B > 65535) return set_error(SKEI_EINVAL, "MRI: B=%d outside [1, 65535]", B);
  return SKEI_OK;
}

size_t mri_ws_bytes(int N, int Nc, int B) {
  // T (interleaved) then W (planar per-coil images)
  return 2 * (size_t)B * Nc * N * N * sizeof(float2);
}

size_t rows_smem(int N, int rpc) { return (size_t)(N / 2 + 2 * rpc * (N + 1)) * sizeof(float2); }
size_t cols_smem(int N, int cpc) { return (size_t)(N / 2 + 2 * N * cpc) * sizeof(float2); }

template <typename K>
int mri_set_smem(K kern, size_t smem, size_t *configured) {
  return opt_in_smem(kern, smem, configured, "MRI kernel: shared memory attribute");
}

int mri_launch_pair(bool fwd, MriArgs &a, int B, cudaStream_t st) {
  static size_t cfg[4][64] = {};
  const int N = a.N;
  a.rpc = std::min(N, 1024 / N);
  a.cpc = std::min(N, kCpc);
  const dim3 grow(N / a.rpc, a.Nc, B), gcol(N / a.cpc, a.Nc, B);
  const size_t sr = rows_smem(N, a.rpc), sc = cols_smem(N, a.cpc);
  if (fwd) {
    SKEI_TRY(mri_set_smem(mri_fwd_rows_kernel, sr, cfg[0]));
    SKEI_TRY(mri_set_smem(mri_fwd_cols_kernel, sc, cfg[1]));
    launch_k(mri_fwd_rows_kernel, grow, dim3(kMriThreads), sr, st, a);
    SKEI_TRY(check_launch("MRI forward row pass"));
    launch_k(mri_fwd_cols_kernel, gcol, dim3(kMriThreads), sc, st, a);
    return check_launch("MRI forward column pass");
  }
  SKEI_TRY(mri_set_smem(mri_adj_cols_kernel, sc, cfg[2]));
  SKEI_TRY(mri_set_smem(mri_adj_rows_kernel, sr, cfg[3]));
  launch_k(mri_adj_cols_kernel, gcol, dim3(kMriThreads), sc, st, a);
  SKEI_TRY(check_launch("MRI adjoint column pass"));
  launch_k(mri_adj_rows_kernel, grow, dim3(kMriThreads), sr, st, a);
  return check_launch("MRI adjoint row pass");
}

}  // namespace
}  // namespace skei

using namespace skei;

extern "C" {

size_t skei_mri_workspace_size(int N, int Nc, int B) {
  if (mri_check(N, Nc, B) != SKEI_OK) return 0;
  return mri_ws_bytes(N, Nc, B);
}

int skei_mri_fwd(int N, int Nc, int B, const float *x, const float *maps, const float *mask,
                 const float *xw, const float *aux, float alpha, float *k, void *work,
                 size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_mri_fwd");
  SKEI_TRY(mri_check(N, Nc, B));
  SKEI_TRY(check_dev_ptr(x, "x"));
  SKEI_TRY(check_dev_ptr(maps, "maps"));
  if (mask) SKEI_TRY(check_dev_ptr(mask, "mask"));
  if (xw) SKEI_TRY(check_dev_ptr(xw, "xw"));
  if (aux) SKEI_TRY(check_dev_ptr(aux, "aux"));
  SKEI_TRY(check_dev_ptr(k, "k"));
  SKEI_TRY(check_dev_ptr(work, "work"));
  if (reinterpret_cast<uintptr_t>(work) % 16)
    return set_error(SKEI_EINVAL, "MRI: work must be 16-byte aligned");
  if (work_bytes < mri_ws_bytes(N, Nc, B))
    return set_error(SKEI_EINVAL, "MRI: work has %zu bytes, %zu needed", work_bytes,
                     mri_ws_bytes(N, Nc, B));
  MriArgs a{N, Nc, 0, 0, x, maps, mask, xw, aux, k, static_cast<float2 *>(work), nullptr,
            alpha};
  return mri_launch_pair(true, a, B, reinterpret_cast<cudaStream_t>(stream));
}

int skei_mri_adj(int N, int Nc, int B, const float *k, const float *maps, const float *mask,
                 const float *dinv, float alpha, float beta, float *x, void *work,
                 size_t work_bytes, void *stream) {
  SKEI_RANGE("skei_mri_adj");
  SKEI_TRY(mri_check(N, Nc, B));
  SKEI_TRY(check_dev_ptr(k, "k"));
  SKEI_TRY(check_dev_ptr(maps, "maps"));
  if (mask) SKEI_TRY(check_dev_ptr(mask, "mask"));
  if (dinv) SKEI_TRY(check_dev_ptr(dinv, "dinv"));
  SKEI_TRY(check_dev_ptr(x, "x"));
  SKEI_TRY(check_dev_ptr(work, "work"));
  if (reinterpret_cast<uintptr_t>(work) % 16)
    return set_error(SKEI_EINVAL, "MRI: work must be 16-byte aligned");
  if (work_bytes < mri_ws_bytes(N, Nc, B))
    return set_error(SKEI_EINVAL, "MRI: work has %zu bytes, %zu needed", work_bytes,
                     mri_ws_bytes(N, Nc, B));
  float2 *T = static_cast<float2 *>(work);
  float *W = reinterpret_cast<float *>(T + (size_t)B * Nc * N * N);
  MriArgs a{N, Nc, 0, 0, x, maps, mask, nullptr, nullptr, const_cast<float *>(k), T, W, 1.0f};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SKEI_TRY(mri_launch_pair(false, a, B, st));
  const int plane = N * N;
  const dim3 g((unsigned)std::min(ceil_div((size_t)2 * plane, (size_t)256), (size_t)1024),
               (unsigned)B);
  launch_k(mri_coil_sum_kernel, g, dim3(256), 0, st, (const float *)W, Nc, plane, dinv, alpha,
           beta, x);
  return check_launch("MRI coil sum");
}

int skei_mri_dinv(int N, int Nc, const float *maps, float *dinv, void *stream) {
  SKEI_RANGE("skei_mri_dinv");
  SKEI_TRY(mri_check(N, Nc, 1));
  SKEI_TRY(check_dev_ptr(maps, "maps"));
  SKEI_TRY(check_dev_ptr(dinv, "dinv"));
  const int plane = N * N;
  mri_dinv_kernel<<<(plane + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      maps, Nc, plane, dinv);
  return check_launch("MRI sensitivity normalisation");
}

int skei_coil_mix(int plane, int B, int n_in, int n_out, const float *Wm, const float *in,
                  float *out, void *stream) {
  SKEI_RANGE("skei_coil_mix");
  if (plane < 1 || B < 1 || B > 65535 || n_in < 1 || n_out < 1 || n_in > 64 || n_out > 64)
    return set_error(SKEI_EINVAL, "coil mix: bad sizes plane=%d B=%d n_in=%d n_out=%d", plane,
                     B, n_in, n_out);
  SKEI_TRY(check_dev_ptr(Wm, "W"));
  SKEI_TRY(check_dev_ptr(in, "in"));
  SKEI_TRY(check_dev_ptr(out, "out"));
  if (in == out) return set_error(SKEI_EINVAL, "coil mix: in and out must not alias");
  const dim3 g((unsigned)std::min((plane + 255) / 256, 1024), (unsigned)B);
  launch_k(coil_mix_kernel, g, dim3(256), (size_t)n_in * n_out * sizeof(float2),
           reinterpret_cast<cudaStream_t>(stream), in, n_in, n_out, plane, Wm, out);
  return check_launch("coil mix");
}

}  // extern "C"
