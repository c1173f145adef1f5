// Plans, status codes and argument validation of libskei.
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "common.cuh"

namespace skei {

cudaError_t dev_malloc(void **ptr, size_t bytes) {
  static std::atomic<long long> count{0};
  static const long long fail_at = [] {
    const char *v = std::getenv("SKEI_FAULT_ALLOC");
    return v ? std::atoll(v) : 0LL;
  }();
  if (fail_at > 0 && ++count == fail_at) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}

static thread_local std::string g_last_error;

int set_error(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_error(cudaError_t e, const char *where) {
  return set_error(SKEI_ECUDA, "%s: %s (%s)", where, cudaGetErrorString(e),
                   cudaGetErrorName(e));
}

int check_plan(skei_plan p) {
  if (!p || !p->d_ang) return set_error(SKEI_EINVAL, "plan is NULL or destroyed");
  return SKEI_OK;
}

int check_dtype(int dtype) {
  if (dtype != SKEI_F32 && dtype != SKEI_BF16)
    return set_error(SKEI_EINVAL, "dtype %d is neither SKEI_F32 nor SKEI_BF16", dtype);
  return SKEI_OK;
}

int check_dev_ptr(const void *p, const char *name) {
  if (!p) return set_error(SKEI_EINVAL, "%s is NULL", name);
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0)
    return set_error(SKEI_EINVAL, "%s is not 16-byte aligned", name);
  return SKEI_OK;
}

int check_idx(skei_plan p, const int *idx, int m) {
  if (m < 1 || m > p->n_angles)
    return set_error(SKEI_EINVAL, "angle count m=%d outside [1, %d]", m, p->n_angles);
  if (!idx && m != p->n_angles)
    return set_error(SKEI_EINVAL, "idx is NULL but m=%d != n_angles=%d", m, p->n_angles);
  if (idx && (reinterpret_cast<uintptr_t>(idx) % 4 != 0))
    return set_error(SKEI_EINVAL, "idx is not 4-byte aligned");
  return SKEI_OK;
}

// SM count of the current device (cached per device).
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

int check_batch(int B) {
  if (B < 1 || B > 65535) return set_error(SKEI_EINVAL, "batch B=%d outside [1, 65535]", B);
  return SKEI_OK;
}

// cos/sin of an angle in degrees with exact reduction to [-45, 45].
static void host_trig(double deg, double *c, double *s) {
  double q = std::floor(deg / 90.0 + 0.5);
  double r = deg - 90.0 * q;
  double rad = r * (M_PI / 180.0);
  double cr = std::cos(rad), sr = std::sin(rad);
  long long qi = ((long long)q % 4 + 4) % 4;
  if (qi == 0) { *c = cr;  *s = sr; }
  else if (qi == 1) { *c = -sr; *s = cr; }
  else if (qi == 2) { *c = -cr; *s = -sr; }
  else { *c = sr; *s = -cr; }
}

static long long fx(double v) { return std::llround(std::ldexp(v, kFxBits)); }

// Derives the constants documented on AngleConst for one angle.
static AngleConst make_angle(double deg, int N, int n_det) {
  double c, s;
  host_trig(deg, &c, &s);
  double phi = std::fmod(deg, 180.0);
  if (phi < 0) phi += 180.0;
  const bool row = (phi <= 45.0) || (phi > 135.0);
  const double h = 0.5 * (N - 1), D = 0.5 * (n_det - 1);
  double T, A, G, W;
  if (row) {
    // ray {x c + y s = u_k} meets row i (y = h - i) at column
    // (u_k - y s)/c + h = i (s/c) + k (1/c) + (h - D/c - h s/c)
    T = s / c;
    A = 1.0 / c;
    G = h - D / c - h * s / c;
    W = 1.0 / std::fabs(c);
  } else {
    // ... meets column j (x = j - h) at row coordinate
    // h - (u_k - x c)/s = j (c/s) + k (-1/s) + (h + D/s - h c/s)
    T = c / s;
    A = -1.0 / s;
    G = h + D / s - h * c / s;
    W = 1.0 / std::fabs(s);
  }
  // t(i, j) = x_j c + y_i s + D = j c - i s + (D - h c + h s)
  const double t00 = D - h * c + h * s, tj = c, ti = -s;
  AngleConst a{};
  a.T = fx(T);
  a.A = fx(A);
  a.G = fx(G);
  a.t00 = fx(t00);
  a.tj = fx(tj);
  a.ti = fx(ti);
  a.bline = row ? a.ti : a.tj;   // lines are rows (i) or columns (j)
  a.bstep = row ? a.tj : a.ti;
  a.Tf = (float)T;
  a.Af = (float)A;
  a.Gf = (float)G;
  a.W = (float)W;
  a.invA = (float)(1.0 / A);
  a.t00f = (float)t00;
  a.tjf = (float)tj;
  a.tif = (float)ti;
  a.blinef = (float)(row ? ti : tj);
  a.bstepf = (float)(row ? tj : ti);
  a.inv_bstep = (float)(1.0 / (row ? tj : ti));
  a.invT = T != 0.0 ? (float)(1.0 / T) : 0.0f;
  const double bl = row ? ti : tj;
  a.inv_bline = bl != 0.0 ? (float)(1.0 / bl) : 0.0f;
  a.mode = row ? 1 : 0;
  return a;
}

}  // namespace skei

using namespace skei;

extern "C" {

int skei_version(void) { return 10000; }

int skei_check_build(void) { return SKEI_CHECK; }

int skei_check_status(unsigned *bits, int reset) {
  if (!bits) return set_error(SKEI_EINVAL, "skei_check_status: bits is NULL");
  *bits = 0;
  if (!SKEI_CHECK) return SKEI_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "skei_check_status: synchronize");
  SKEI_TRY(check_read_band(bits, reset));
  SKEI_TRY(check_read_tile(bits, reset));
  return check_read_filter(bits, reset);
}

const char *skei_last_error(void) { return g_last_error.c_str(); }

int skei_plan_create(int N, int n_det, int n_angles, const double *angles_deg,
                     skei_plan *out) {
  SKEI_RANGE("skei_plan_create");
  if (!out) return set_error(SKEI_EINVAL, "out is NULL");
  *out = nullptr;
  if (N < 1 || N > SKEI_MAX_N) return set_error(SKEI_EINVAL, "N=%d outside [1, %d]", N, SKEI_MAX_N);
  if (n_det == 0) {
    n_det = (int)std::ceil(N * std::sqrt(2.0));
    if (n_det % 2 == 0) ++n_det;
  }
  if (n_det < 1 || n_det > SKEI_MAX_NDET)
    return set_error(SKEI_EINVAL, "n_det=%d outside [1, %d]", n_det, SKEI_MAX_NDET);
  if (n_angles < 1 || n_angles > SKEI_MAX_ANGLES)
    return set_error(SKEI_EINVAL, "n_angles=%d outside [1, %d]", n_angles, SKEI_MAX_ANGLES);
  if (angles_deg)
    for (int a = 0; a < n_angles; ++a)
      if (!std::isfinite(angles_deg[a]) || std::fabs(angles_deg[a]) > 1e6)
        return set_error(SKEI_EINVAL, "angle %d is not a finite value below 1e6 degrees", a);

  skei_plan p = new (std::nothrow) skei_plan_s;
  if (!p) return set_error(SKEI_ENOMEM, "host allocation of the plan failed");
  p->N = N;
  p->n_det = n_det;
  p->n_angles = n_angles;
  cudaGetDevice(&p->device);
  p->angles_deg.resize(n_angles);
  std::vector<AngleConst> host(n_angles);
  for (int a = 0; a < n_angles; ++a) {
    p->angles_deg[a] = angles_deg ? angles_deg[a] : 180.0 * a / n_angles;
    host[a] = make_angle(p->angles_deg[a], N, n_det);
  }
  int rc = ensure_ramlak_taps();
  cudaError_t e = cudaSuccess;
  if (rc != SKEI_OK) {
    // message already set
  } else if ((e = dev_malloc(reinterpret_cast<void **>(&p->d_ang),
                             sizeof(AngleConst) * n_angles)) != cudaSuccess ||
             (e = dev_malloc(reinterpret_cast<void **>(&p->d_status), sizeof(int))) !=
                 cudaSuccess) {
    rc = e == cudaErrorMemoryAllocation ? set_error(SKEI_ENOMEM, "plan device allocation failed")
                                        : cuda_error(e, "skei_plan_create: cudaMalloc");
  } else if ((e = cudaMemcpy(p->d_ang, host.data(), sizeof(AngleConst) * n_angles,
                             cudaMemcpyHostToDevice)) != cudaSuccess ||
             (e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess) {
    rc = cuda_error(e, "skei_plan_create: upload");
  }
  if (rc == SKEI_OK) rc = make_filter_spectrum(p);
  if (rc != SKEI_OK) {
    cudaFree(p->d_ang);
    cudaFree(p->d_status);
    cudaFree(p->d_hspec);
    delete p;
    return rc;
  }
  *out = p;
  return SKEI_OK;
}

int skei_plan_destroy(skei_plan p) {
  SKEI_RANGE("skei_plan_destroy");
  if (!p) return SKEI_OK;
  cudaFree(p->d_ang);
  cudaFree(p->d_status);
  cudaFree(p->d_hspec);
  p->d_ang = nullptr;
  delete p;
  return SKEI_OK;
}

int skei_plan_geometry(skei_plan p, int *N, int *n_det, int *n_angles) {
  if (int rc = check_plan(p)) return rc;
  if (N) *N = p->N;
  if (n_det) *n_det = p->n_det;
  if (n_angles) *n_angles = p->n_angles;
  return SKEI_OK;
}

int skei_plan_status(skei_plan p, int reset, int *word) {
  if (int rc = check_plan(p)) return rc;
  if (!word) return set_error(SKEI_EINVAL, "word is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "skei_plan_status: synchronize");
  if ((e = cudaMemcpy(word, p->d_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_error(e, "skei_plan_status: read");
  if (reset && (e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess)
    return cuda_error(e, "skei_plan_status: reset");
  return SKEI_OK;
}

}  // extern "C"
