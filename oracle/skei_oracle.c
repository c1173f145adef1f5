/*
 * Plain, slow FP64 CPU oracle for the operators inside one sketched
 * Equivariant Imaging (SkEI) step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes (paper Sec. 2.1: y ~ A x with A the discrete Radon
 * transform of parallel-beam CT, Sec. 4.1.1; A^dagger approximated by
 * filtered back-projection, Sec. 2.1; T_g rotations, Sec. 4.1.3):
 *
 *   oracle_joseph_fwd      A   : Joseph's linear-interpolation line integrals
 *   oracle_joseph_adj      A^T : the same weights, scattered (a different loop)
 *   oracle_ramlak          H   : discrete Ram-Lak filter, full linear convolution
 *   oracle_backproject     B   : pixel-driven linear-interpolation back-projection
 *   oracle_backproject_adj B^T : the same weights, scattered
 *   oracle_rotate          T_g : bilinear, zero padded, counter-clockwise
 *   oracle_rotate_adj      T_g^T : scattered
 *
 * The paper does not fix the discretisation; the readings used here are:
 *   pixel (i,j), row i from the top, centre x_j = j-(N-1)/2, y_i = (N-1)/2-i;
 *   bin k at u_k = k-(n_det-1)/2; ray = {x cos t + y sin t = u};
 *   Joseph row mode iff (t mod 180) in [0,45] or (135,180), else column mode;
 *   interpolation taps outside the image are zero;
 *   Ram-Lak h(0)=1/4, h(odd n)=-1/(pi^2 n^2), h(even n != 0)=0 (unit bins);
 *   FBP = (pi/m') B H where m' is the number of angles used.
 * Every function is FP64 and single threaded.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

/* Smallest odd integer >= N*sqrt(2): a detector that covers the image
 * diagonal with unit bins centred on the rotation axis. */
int oracle_ndet(int N)
{
    int k = (int)ceil((double)N * sqrt(2.0));
    if (k % 2 == 0) k += 1;
    return k;
}

/* cos and sin of an angle in degrees, reduced exactly to [-45,45] first so
 * that multiples of 90 degrees give exact 0 and +-1. */
void oracle_trig(double deg, double *c, double *s)
{
    double q = floor(deg / 90.0 + 0.5);
    double r = deg - 90.0 * q;
    double rad = r * (ORACLE_PI / 180.0);
    double cr = cos(rad), sr = sin(rad);
    long qi = ((long)q % 4 + 4) % 4;
    switch (qi) {
    case 0: *c = cr;  *s = sr;  break;
    case 1: *c = -sr; *s = cr;  break;
    case 2: *c = -cr; *s = -sr; break;
    default: *c = sr; *s = -cr; break;
    }
}

/* 1 when Joseph's method walks the rows (the ray is closer to vertical). */
int oracle_row_mode(double deg)
{
    double phi = fmod(deg, 180.0);
    if (phi < 0.0) phi += 180.0;
    return (phi <= 45.0) || (phi > 135.0);
}

static double pix(const double *x, int N, int i, int j)
{
    if (i < 0 || i >= N || j < 0 || j >= N) return 0.0;
    return x[(size_t)i * N + j];
}

static void add_pix(double *x, int N, int i, int j, double v)
{
    if (i < 0 || i >= N || j < 0 || j >= N) return;
    x[(size_t)i * N + j] += v;
}

/* A: p[a][k] = sum over rows (or columns) of the linear interpolation of x
 * where ray (a,k) crosses that row (column), times 1/|cos| (1/|sin|). */
void oracle_joseph_fwd(int N, int n_det, int n_ang, const double *ang_deg,
                       const double *x, double *p)
{
    double h = 0.5 * (N - 1);
    for (int a = 0; a < n_ang; ++a) {
        double c, s;
        oracle_trig(ang_deg[a], &c, &s);
        int row = oracle_row_mode(ang_deg[a]);
        for (int k = 0; k < n_det; ++k) {
            double u = k - 0.5 * (n_det - 1);
            double acc = 0.0;
            if (row) {
                for (int i = 0; i < N; ++i) {
                    double y = h - i;
                    double col = (u - y * s) / c + h;
                    double j0 = floor(col);
                    double f = col - j0;
                    acc += (1.0 - f) * pix(x, N, i, (int)j0) + f * pix(x, N, i, (int)j0 + 1);
                }
                p[(size_t)a * n_det + k] = acc / fabs(c);
            } else {
                for (int j = 0; j < N; ++j) {
                    double xx = j - h;
                    double r = h - (u - xx * c) / s;
                    double i0 = floor(r);
                    double f = r - i0;
                    acc += (1.0 - f) * pix(x, N, (int)i0, j) + f * pix(x, N, (int)i0 + 1, j);
                }
                p[(size_t)a * n_det + k] = acc / fabs(s);
            }
        }
    }
}

/* A^T p, written as a scatter over rays and samples: x = A^T p (overwritten). */
void oracle_joseph_adj(int N, int n_det, int n_ang, const double *ang_deg,
                       const double *p, double *x)
{
    double h = 0.5 * (N - 1);
    memset(x, 0, sizeof(double) * (size_t)N * N);
    for (int a = 0; a < n_ang; ++a) {
        double c, s;
        oracle_trig(ang_deg[a], &c, &s);
        int row = oracle_row_mode(ang_deg[a]);
        for (int k = 0; k < n_det; ++k) {
            double u = k - 0.5 * (n_det - 1);
            double v = p[(size_t)a * n_det + k];
            if (row) {
                double w = v / fabs(c);
                for (int i = 0; i < N; ++i) {
                    double y = h - i;
                    double col = (u - y * s) / c + h;
                    double j0 = floor(col);
                    double f = col - j0;
                    add_pix(x, N, i, (int)j0, (1.0 - f) * w);
                    add_pix(x, N, i, (int)j0 + 1, f * w);
                }
            } else {
                double w = v / fabs(s);
                for (int j = 0; j < N; ++j) {
                    double xx = j - h;
                    double r = h - (u - xx * c) / s;
                    double i0 = floor(r);
                    double f = r - i0;
                    add_pix(x, N, (int)i0, j, (1.0 - f) * w);
                    add_pix(x, N, (int)i0 + 1, j, f * w);
                }
            }
        }
    }
}

/* The discrete Ram-Lak kernel for unit detector spacing. */
double oracle_ramlak_tap(int n)
{
    if (n == 0) return 0.25;
    if (n % 2 == 0) return 0.0;
    return -1.0 / (ORACLE_PI * ORACLE_PI * (double)n * (double)n);
}

/* H: q[r][k] = sum_{k'} h(k-k') p[r][k'], linear convolution, zero outside
 * the detector, for each of `rows` sinogram rows. */
void oracle_ramlak(int n_det, int rows, const double *p, double *q)
{
    for (int r = 0; r < rows; ++r) {
        const double *pr = p + (size_t)r * n_det;
        double *qr = q + (size_t)r * n_det;
        for (int k = 0; k < n_det; ++k) {
            double acc = 0.0;
            for (int kk = 0; kk < n_det; ++kk)
                acc += oracle_ramlak_tap(k - kk) * pr[kk];
            qr[k] = acc;
        }
    }
}

static double bin(const double *qa, int n_det, int k)
{
    if (k < 0 || k >= n_det) return 0.0;
    return qa[k];
}

/* B (unscaled): x[i][j] = sum_a of the linear interpolation of q[a] at
 * t = x_j cos + y_i sin + (n_det-1)/2.  x is overwritten. */
void oracle_backproject(int N, int n_det, int n_ang, const double *ang_deg,
                        const double *q, double *x)
{
    double h = 0.5 * (N - 1);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double xx = j - h, y = h - i, acc = 0.0;
            for (int a = 0; a < n_ang; ++a) {
                double c, s;
                oracle_trig(ang_deg[a], &c, &s);
                double t = xx * c + y * s + 0.5 * (n_det - 1);
                double k0 = floor(t);
                double w = t - k0;
                const double *qa = q + (size_t)a * n_det;
                acc += (1.0 - w) * bin(qa, n_det, (int)k0) + w * bin(qa, n_det, (int)k0 + 1);
            }
            x[(size_t)i * N + j] = acc;
        }
}

/* B^T, a scatter of each pixel into its two bins: q = B^T x (overwritten). */
void oracle_backproject_adj(int N, int n_det, int n_ang, const double *ang_deg,
                            const double *x, double *q)
{
    double h = 0.5 * (N - 1);
    memset(q, 0, sizeof(double) * (size_t)n_ang * n_det);
    for (int a = 0; a < n_ang; ++a) {
        double c, s;
        oracle_trig(ang_deg[a], &c, &s);
        double *qa = q + (size_t)a * n_det;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                double xx = j - h, y = h - i;
                double t = xx * c + y * s + 0.5 * (n_det - 1);
                double k0 = floor(t);
                double w = t - k0;
                double v = x[(size_t)i * N + j];
                int kk = (int)k0;
                if (kk >= 0 && kk < n_det) qa[kk] += (1.0 - w) * v;
                if (kk + 1 >= 0 && kk + 1 < n_det) qa[kk + 1] += w * v;
            }
    }
}

/* T_g: counter-clockwise rotation by g degrees about the image centre.
 * Output pixel (x_j, y_i) samples the input at R(-g)(x_j, y_i), bilinear,
 * zero outside. */
void oracle_rotate(int N, double g_deg, const double *x, double *out)
{
    double h = 0.5 * (N - 1), c, s;
    oracle_trig(g_deg, &c, &s);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double xx = j - h, y = h - i;
            double xs = c * xx + s * y;
            double ys = -s * xx + c * y;
            double col = xs + h, row = h - ys;
            double i0 = floor(row), j0 = floor(col);
            double fr = row - i0, fc = col - j0;
            int ii = (int)i0, jj = (int)j0;
            out[(size_t)i * N + j] =
                (1.0 - fr) * (1.0 - fc) * pix(x, N, ii, jj) +
                (1.0 - fr) * fc * pix(x, N, ii, jj + 1) +
                fr * (1.0 - fc) * pix(x, N, ii + 1, jj) +
                fr * fc * pix(x, N, ii + 1, jj + 1);
        }
}

/* T_g^T as a scatter: gx = T_g^T gout (overwritten). */
void oracle_rotate_adj(int N, double g_deg, const double *gout, double *gx)
{
    double h = 0.5 * (N - 1), c, s;
    oracle_trig(g_deg, &c, &s);
    memset(gx, 0, sizeof(double) * (size_t)N * N);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double xx = j - h, y = h - i;
            double xs = c * xx + s * y;
            double ys = -s * xx + c * y;
            double col = xs + h, row = h - ys;
            double i0 = floor(row), j0 = floor(col);
            double fr = row - i0, fc = col - j0;
            int ii = (int)i0, jj = (int)j0;
            double v = gout[(size_t)i * N + j];
            add_pix(gx, N, ii, jj, (1.0 - fr) * (1.0 - fc) * v);
            add_pix(gx, N, ii, jj + 1, (1.0 - fr) * fc * v);
            add_pix(gx, N, ii + 1, jj, fr * (1.0 - fc) * v);
            add_pix(gx, N, ii + 1, jj + 1, fr * fc * v);
        }
}
