/*
 * FP64 CPU oracle for the discretised 2D parallel-beam operators.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header, table or
 * helper with the CUDA path; it is plain, slow and written to be checked by eye
 * against the paper:
 *
 *   Koshev, Helou, Miqueles, "Fast Backprojection Techniques for High Resolution
 *   Tomography" (arXiv:1608.03589).
 *
 * Geometry (Table "tab:symbols", Section 5):
 *   pixel centres   x_i = -1 + (i + 1/2) dx,  dx = 2/N,  image b[iy*N + ix], y = row
 *   detector centres t_j = (j - (n_det-1)/2) dt,  sinogram g[k*n_det + j]
 *   u(x, k) = (x . xi_k)/dt + (n_det-1)/2  = detector coordinate in bins,
 *   xi_k = (cos theta_k, sin theta_k)           (Section 1, eq "L")
 *
 * Quadrature: b(x) ~ dtheta * sum_k g(x . xi_k, theta_k) (Section 2, eq "bp_app").  For
 * arbitrary angle sets the constant dtheta generalises to w_k = half the sum of the two
 * angular gaps around theta_k (angles taken mod pi, wrapped with period pi); for
 * theta_k = k pi / N_theta this is exactly pi / N_theta.
 *
 * Every function is single-precision free: all arithmetic is double.  Loops over
 * output pixels / angles are parallelised with OpenMP; each output value is computed
 * by one thread in the textbook summation order, so results do not depend on the
 * thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------------
 * Quadrature weights w_k for the angle sum of eq "bp_app" (Section 2).
 * Sort the angles mod pi; w = (next - prev)/2 with wrap-around of period pi.
 * ------------------------------------------------------------------------------- */
typedef struct { double a; int k; } or_ang;

static int or_cmp(const void *p, const void *q)
{
    double a = ((const or_ang *)p)->a, b = ((const or_ang *)q)->a;
    return (a < b) ? -1 : (a > b) ? 1 : 0;
}

int oracle_weights(int n_theta, const double *theta, double *w)
{
    if (n_theta <= 0) return -1;
    if (n_theta == 1) { w[0] = OR_PI; return 0; }
    or_ang *s = (or_ang *)malloc(sizeof(or_ang) * (size_t)n_theta);
    if (!s) return -2;
    for (int k = 0; k < n_theta; ++k) {
        double a = fmod(theta[k], OR_PI);
        if (a < 0) a += OR_PI;
        s[k].a = a;
        s[k].k = k;
    }
    qsort(s, (size_t)n_theta, sizeof(or_ang), or_cmp);
    for (int i = 0; i < n_theta; ++i) {
        double prev = (i == 0) ? s[n_theta - 1].a - OR_PI : s[i - 1].a;
        double next = (i == n_theta - 1) ? s[0].a + OR_PI : s[i + 1].a;
        w[s[i].k] = 0.5 * (next - prev);
    }
    free(s);
    return 0;
}

/* Detector coordinate (in bins) of the point (x, y) for angle theta (eq "L"). */
static double or_u(double x, double y, double ct, double st, double dt, int n_det)
{
    return (x * ct + y * st) / dt + 0.5 * (double)(n_det - 1);
}

/* Linear interpolation of one projection row at bin coordinate u, zero outside the
 * detector (Section 2: "a linear interpolation for x . xi on the grid of -1 <= t <= 1").
 * j = floor(u), f = u - j, value = (1-f) g_j + f g_{j+1}. */
static double or_lerp(const double *row, int n_det, double u)
{
    double jf = floor(u);
    double f = u - jf;
    long j = (long)jf;
    double g0 = (j >= 0 && j < n_det) ? row[j] : 0.0;
    double g1 = (j + 1 >= 0 && j + 1 < n_det) ? row[j + 1] : 0.0;
    return (1.0 - f) * g0 + f * g1;
}

/* ---------------------------------------------------------------------------------
 * R*: direct (pixel-driven) backprojection, Section 2 eq "bp_app" with linear
 * interpolation:  b(x_p) = sum_k w_k * lerp(g_k, u(x_p, k)).
 * ------------------------------------------------------------------------------- */
static double or_bp_pixel(int N, int n_det, int n_theta, const double *ct, const double *st,
                          const double *w, double dt, const double *g, int ix, int iy)
{
    double dx = 2.0 / N;
    double x = -1.0 + (ix + 0.5) * dx;
    double y = -1.0 + (iy + 0.5) * dx;
    double acc = 0.0;
    for (int k = 0; k < n_theta; ++k)
        acc += w[k] * or_lerp(g + (size_t)k * n_det, n_det, or_u(x, y, ct[k], st[k], dt, n_det));
    return acc;
}

static int or_trig_tables(int n_theta, const double *theta, double **ct, double **st, double **w)
{
    *ct = (double *)malloc(sizeof(double) * (size_t)n_theta);
    *st = (double *)malloc(sizeof(double) * (size_t)n_theta);
    *w = (double *)malloc(sizeof(double) * (size_t)n_theta);
    if (!*ct || !*st || !*w) return -2;
    for (int k = 0; k < n_theta; ++k) { (*ct)[k] = cos(theta[k]); (*st)[k] = sin(theta[k]); }
    return oracle_weights(n_theta, theta, *w);
}

static void or_free3(double *a, double *b, double *c) { free(a); free(b); free(c); }

int oracle_bp_linear(int N, int n_det, int n_theta, const double *theta, double dt,
                     const double *g, double *b)
{
    double *ct, *st, *w;
    int rc = or_trig_tables(n_theta, theta, &ct, &st, &w);
    if (rc) { or_free3(ct, st, w); return rc; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int iy = 0; iy < N; ++iy)
        for (int ix = 0; ix < N; ++ix)
            b[(size_t)iy * N + ix] = or_bp_pixel(N, n_det, n_theta, ct, st, w, dt, g, ix, iy);
    or_free3(ct, st, w);
    return 0;
}

/* Same operator, evaluated only at the listed pixels (flat index iy*N + ix). */
int oracle_bp_linear_points(int N, int n_det, int n_theta, const double *theta, double dt,
                            const double *g, int npts, const long *pix, double *out)
{
    double *ct, *st, *w;
    int rc = or_trig_tables(n_theta, theta, &ct, &st, &w);
    if (rc) { or_free3(ct, st, w); return rc; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < npts; ++i) {
        int iy = (int)(pix[i] / N), ix = (int)(pix[i] % N);
        out[i] = or_bp_pixel(N, n_det, n_theta, ct, st, w, dt, g, ix, iy);
    }
    or_free3(ct, st, w);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * R: the transpose of the discrete R*, scaled to approximate the line integral of
 * eq "P_theta" (Section 1).  With A the matrix of R* (A[p,(k,j)] = w_k hat(u_pk - j)),
 *   R = (dx^2/dt) diag(1/w_k) A^T,   i.e.  (R f)_{kj} = (dx^2/dt) sum_p hat(u_pk - j) f_p,
 * so that the weighted discrete adjoint identity (eq "adjoint")
 *   sum_k w_k dt sum_j (R f)_{kj} g_{kj} = dx^2 sum_p f_p (R* g)_p
 * holds exactly.  Each pixel scatters (1-f) f_p to bin j and f f_p to bin j+1.
 * ------------------------------------------------------------------------------- */
int oracle_radon(int N, int n_det, int n_theta, const double *theta, double dt,
                 const double *f, double *g)
{
    double dx = 2.0 / N;
    double scale = dx * dx / dt;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < n_theta; ++k) {
        double ct = cos(theta[k]), st = sin(theta[k]);
        double *row = g + (size_t)k * n_det;
        for (int j = 0; j < n_det; ++j) row[j] = 0.0;
        for (int iy = 0; iy < N; ++iy) {
            double y = -1.0 + (iy + 0.5) * dx;
            for (int ix = 0; ix < N; ++ix) {
                double x = -1.0 + (ix + 0.5) * dx;
                double u = or_u(x, y, ct, st, dt, n_det);
                double jf = floor(u);
                double fr = u - jf;
                long j = (long)jf;
                double v = f[(size_t)iy * N + ix];
                if (j >= 0 && j < n_det) row[j] += (1.0 - fr) * v;
                if (j + 1 >= 0 && j + 1 < n_det) row[j + 1] += fr * v;
            }
        }
        for (int j = 0; j < n_det; ++j) row[j] *= scale;
    }
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Filter F of FBP (Section 3, Remark 1 (ii), eq "fbp": widehat{Fg} = |nu| g^), and the
 * Tikhonov-regularised filter |nu| / (1 + lambda |nu|) of Section 6.  Discretised as a
 * linear (non-circular) convolution along each projection row,
 *   q_j = dt * sum_{i=0}^{n_det-1} h(j - i) g_i,
 * with h the band-limited spatial kernel of the filter's frequency response on
 * |nu| <= 1/(2 dt):
 *   kind 0 Ram-Lak:     h(0) = 1/(4 dt^2); h(n odd) = -1/(pi^2 n^2 dt^2); h(n even) = 0
 *   kind 1 Shepp-Logan: h(n) = -2 / (pi^2 dt^2 (4 n^2 - 1))   (|nu| sinc(nu dt))
 *   kind 2 Tikhonov:    h(n) = 2 int_0^{1/(2dt)} nu/(1 + lambda nu) cos(2 pi nu n dt) dnu,
 *                       by composite Simpson quadrature with 2^16 panels.
 * ------------------------------------------------------------------------------- */
static double or_tikhonov_h(long n, double dt, double lam)
{
    const int M = 1 << 16;
    double W = 0.5 / dt, hstep = W / M, s = 0.0;
    for (int i = 0; i <= M; ++i) {
        double nu = i * hstep;
        double v = nu / (1.0 + lam * nu) * cos(2.0 * OR_PI * nu * (double)n * dt);
        double c = (i == 0 || i == M) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        s += c * v;
    }
    return 2.0 * s * hstep / 3.0;
}

int oracle_filter_kernel(int n_det, double dt, int kind, double param, double *h /* 2n_det-1, h[n + n_det-1] */)
{
    for (long n = -(long)(n_det - 1); n <= (long)(n_det - 1); ++n) {
        double v;
        if (kind == 0) {
            if (n == 0) v = 1.0 / (4.0 * dt * dt);
            else if (n & 1) v = -1.0 / (OR_PI * OR_PI * (double)n * (double)n * dt * dt);
            else v = 0.0;
        } else if (kind == 1) {
            v = -2.0 / (OR_PI * OR_PI * dt * dt * (4.0 * (double)n * (double)n - 1.0));
        } else if (kind == 2) {
            v = or_tikhonov_h(n, dt, param);
        } else {
            return -1;
        }
        h[n + n_det - 1] = v;
    }
    return 0;
}

int oracle_filter(int rows, int n_det, double dt, int kind, double param,
                  const double *g, double *q)
{
    double *h = (double *)malloc(sizeof(double) * (size_t)(2 * n_det - 1));
    if (!h) return -2;
    int rc = oracle_filter_kernel(n_det, dt, kind, param, h);
    if (rc) { free(h); return rc; }
#pragma omp parallel for schedule(static)
    for (int r = 0; r < rows; ++r) {
        const double *gr = g + (size_t)r * n_det;
        double *qr = q + (size_t)r * n_det;
        for (int j = 0; j < n_det; ++j) {
            double acc = 0.0;
            for (int i = 0; i < n_det; ++i) acc += h[j - i + n_det - 1] * gr[i];
            qr[j] = dt * acc;
        }
    }
    free(h);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Fourier-path operator (Section 3, eq "bst"; Section 5.3 Steps 1-4).  The BST form
 * backprojects the band-limited (trigonometric) interpolant of each zero-padded
 * projection: with G_k[m] = sum_j g_kj e^{-2 pi i m j / P} (P-point DFT, Step 2.2) and
 * the Nyquist bin dropped,
 *   T_k(u) = (1/P) sum_{|m| < P/2} G_k[m] e^{2 pi i m u / P} = sum_j g_kj D_P(u - j),
 *   D_P(v) = sin(pi v (P-1)/P) / (P sin(pi v / P)),   D_P(0) = (P-1)/P,
 * and b_F(x_p) = sum_k w_k T_k(u(x_p, k)).
 * Two independent evaluations are provided: the spatial Dirichlet sum (small sizes)
 * and the spectral sum from given half-spectra G_k[0..P/2-1] (sampled pixels).
 * ------------------------------------------------------------------------------- */
static double or_dirichlet(double v, int P)
{
    double s = sin(OR_PI * v / P);
    if (fabs(s) < 1e-300 || fabs(v) < 1e-12) return (double)(P - 1) / P;
    return sin(OR_PI * v * (double)(P - 1) / P) / ((double)P * s);
}

int oracle_bp_trig_dirichlet(int N, int n_det, int n_theta, const double *theta, double dt, int P,
                             const double *g, double *b)
{
    double *ct, *st, *w;
    int rc = or_trig_tables(n_theta, theta, &ct, &st, &w);
    if (rc) { or_free3(ct, st, w); return rc; }
    double dx = 2.0 / N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int iy = 0; iy < N; ++iy) {
        double y = -1.0 + (iy + 0.5) * dx;
        for (int ix = 0; ix < N; ++ix) {
            double x = -1.0 + (ix + 0.5) * dx;
            double acc = 0.0;
            for (int k = 0; k < n_theta; ++k) {
                double u = or_u(x, y, ct[k], st[k], dt, n_det);
                const double *row = g + (size_t)k * n_det;
                double t = 0.0;
                for (int j = 0; j < n_det; ++j) t += row[j] * or_dirichlet(u - j, P);
                acc += w[k] * t;
            }
            b[(size_t)iy * N + ix] = acc;
        }
    }
    or_free3(ct, st, w);
    return 0;
}

/* Spectral evaluation at listed pixels.  Gre/Gim: [n_theta][P/2], m = 0..P/2-1.
 * Real g gives G[-m] = conj G[m], so T(u) = (1/P)(G[0] + 2 sum_{m=1}^{P/2-1} Re(G[m] e^{2 pi i m u/P})). */
int oracle_bp_trig_points(int N, int n_det, int n_theta, const double *theta, double dt, int P,
                          const double *Gre, const double *Gim, int npts, const long *pix, double *out)
{
    double *ct, *st, *w;
    int rc = or_trig_tables(n_theta, theta, &ct, &st, &w);
    if (rc) { or_free3(ct, st, w); return rc; }
    double dx = 2.0 / N;
    int H = P / 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < npts; ++i) {
        int iy = (int)(pix[i] / N), ix = (int)(pix[i] % N);
        double x = -1.0 + (ix + 0.5) * dx, y = -1.0 + (iy + 0.5) * dx;
        double acc = 0.0;
        for (int k = 0; k < n_theta; ++k) {
            double u = or_u(x, y, ct[k], st[k], dt, n_det);
            const double *re = Gre + (size_t)k * H, *im = Gim + (size_t)k * H;
            double t = re[0];
            for (int m = 1; m < H; ++m) {
                double ph = 2.0 * OR_PI * (double)m * u / P;
                t += 2.0 * (re[m] * cos(ph) - im[m] * sin(ph));
            }
            acc += w[k] * t / P;
        }
        out[i] = acc;
    }
    or_free3(ct, st, w);
    return 0;
}

/* Transpose of the Fourier-path operator, scaled like oracle_radon:
 *   (R_F f)_{kj} = (dx^2/dt) sum_p D_P(u_pk - j) f_p, evaluated for listed (k, j) pairs. */
int oracle_radon_trig_points(int N, int n_det, int n_theta, const double *theta, double dt, int P,
                             const double *f, int npts, const long *kj, double *out)
{
    double dx = 2.0 / N;
    double scale = dx * dx / dt;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < npts; ++i) {
        int k = (int)(kj[i] / n_det), j = (int)(kj[i] % n_det);
        double ct = cos(theta[k]), st = sin(theta[k]);
        double acc = 0.0;
        for (int iy = 0; iy < N; ++iy) {
            double y = -1.0 + (iy + 0.5) * dx;
            for (int ix = 0; ix < N; ++ix) {
                double x = -1.0 + (ix + 0.5) * dx;
                acc += f[(size_t)iy * N + ix] * or_dirichlet(or_u(x, y, ct, st, dt, n_det) - j, P);
            }
        }
        out[i] = scale * acc;
    }
    return 0;
}
