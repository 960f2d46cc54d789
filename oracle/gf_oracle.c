/*
 * gf_oracle.c -- plain, slow, FP64 CPU oracle for the FFT-based algorithm of
 * B. Zhang & R. Zhang, "An FFT-based algorithm for efficient computation of
 * Green's functions for the Helmholtz and Maxwell's equations in periodic
 * domains" (arXiv:1801.05977).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so, which is
 * loaded by the tests, by __graft_entry__.smoke() and by the CPU-baseline leg
 * of bench.py -- never by the library.  It shares no code, header, table or
 * helper with the CUDA library; the two meet only in the seeded input
 * generators, which hold none of the method's arithmetic.
 *
 * Everything is double precision (std C99 `double complex`), written in the
 * order and notation of the paper, with no blocking, fusion or reordering:
 *   - cutoffs X (chi) and Y_eps: C^8 (Sec. 5 states "C^8"); we use the order-8
 *     generalized smoothstep S8 (reading of a silent point);
 *   - beta branch: Sec. 1, definitions under Eqs. (ei) and (he);
 *   - 2D coefficients: Eq. (fck-coef), Eqs. (fcl-coef), (fcf1-coef), (fcf2-coef);
 *   - 3D coefficients: Eq. (kdj1) and Eq. (fj); Maxwell: Sec. 4 (-c^p c^q factor);
 *   - grid synthesis: truncated series (fcln)/(ln), by a NAIVE row-column
 *     inverse DFT (O(M^2) per line), not an FFT;
 *   - point evaluation: Algorithms 1, 2 and 3 (branch, reduction, cubic
 *     interpolation on the 4^d nearest nodes, singular add-back, phase);
 *   - far branch / exact reference: eigenfunction expansions (ei), (he) and
 *     their second derivatives;
 *   - 2D derivatives (Sec. 2.4): the gradient fields K_1 - h_1, K_2 - h_2 and
 *     the second-derivative differences T_pq - h_pq for two wave numbers, their
 *     singular parts' coefficients by the plane Fourier transform reduced to
 *     Hankel transforms, and the term-by-term derivatives of (ei).
 * The integrals that the paper evaluates "by FFT" (the X' integrals in
 * (fck-coef)/(kdj1), the singular-part transform in (fj) and Phi_1-hat,
 * Phi_2-hat in (fcf1-coef)/(fcf2-coef)) are evaluated by Gauss-Legendre
 * quadrature on the (compact) support of the integrand after the exact radial
 * reduction; see the per-function comments.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Parameters of one problem; mirrored field by field in oracle/oracle.py. */
typedef struct {
    int dim;        /* 2: G of Sec. 2;  3: G_d of Sec. 3 (or the tensor of Sec. 4) */
    int M[3];       /* grid points per axis (x1, x2[, x3]); paper's 2N per axis */
    int Q;          /* Gauss-Legendre nodes for every 1D integral */
    int maxwell;    /* 3D only: 1 = Algorithm 3 (seven grids) */
    double k;       /* wave number */
    double alpha[2];/* quasi-periodicity alpha (2D: alpha[0]) */
    double c;       /* |x_last| <= c uses the grid, > c the eigen-series */
    double ct;      /* c~: half period of the artificial periodisation */
    double eps;     /* singular cutoff radius: Y_eps = 1 on [0,eps], 0 beyond 2 eps */
    double tau;     /* relative truncation tolerance of the eigen-series */
} or_params;

/* Threads of the OpenMP loops below (n > 0 sets them); returns the count in
 * effect.  Only the timing of the CPU baseline uses it (1 thread and all). */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Cutoff functions.                                                          */
/* ------------------------------------------------------------------------ */

static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

/* Order-8 generalized smoothstep on [0,1] (0 below, 1 above) and its first two
 * derivatives (d = 0, 1, 2).  S8 is the regularized incomplete beta function
 * I_s(9,9): S8' = 17!/(8! 8!) s^8 (1-s)^8, which vanishes to 8th order at both
 * ends, giving the C^8 cutoffs of Sec. 5.  The value is summed in Bernstein
 * form, S8(s) = sum_{m=9}^{17} C(17,m) s^m (1-s)^{17-m}, whose terms are all
 * positive (no cancellation anywhere on [0,1]). */
double or_smooth8(double s, int d)
{
    if (s <= 0.0) return 0.0;
    if (s >= 1.0) return d == 0 ? 1.0 : 0.0;
    double u = 1.0 - s;
    if (d == 0) {
        double acc = 0.0;
        for (int m = 9; m <= 17; ++m) acc += binom(17, m) * pow(s, m) * pow(u, 17 - m);
        return acc;
    }
    double C = binom(17, 8) * 9.0; /* 17!/(8! 8!) */
    if (d == 1) return C * pow(s * u, 8);
    return C * 8.0 * pow(s * u, 7) * (1.0 - 2.0 * s);
}

/* X(t) for t >= 0: 1 on [0,c], 0 on [(c+c~)/2, inf), smooth in between
 * (Sec. 2.1).  d-th derivative in t, d = 0, 1, 2. */
double or_chi(double t, double c, double ct, int d)
{
    double w = 0.5 * (ct - c);
    double s = (t - c) / w;
    double v = or_smooth8(s, d);
    if (d == 0) return 1.0 - v;
    if (d == 1) return -v / w;
    return -v / (w * w);
}

/* Y_eps(r): 1 on [0,eps], 0 on [2 eps, inf), smooth in between (Sec. 2.2). */
double or_yps(double r, double eps, int d)
{
    double s = (r - eps) / eps;
    double v = or_smooth8(s, d);
    if (d == 0) return 1.0 - v;
    if (d == 1) return -v / eps;
    return -v / (eps * eps);
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes/weights on [-1,1] by Newton's method on P_Q, with P_Q */
/* and P_Q' from the three-term recurrence.                                   */
/* ------------------------------------------------------------------------ */
void or_gauss_legendre(int Q, double *x, double *w)
{
    for (int i = 0; i < Q; ++i) {
        double z = cos(M_PI * (i + 0.75) / (Q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int n = 2; n <= Q; ++n) {
                double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            if (Q == 1) { p1 = z; p0 = 1.0; }
            dp = Q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged node */
        double p0 = 1.0, p1 = z;
        for (int n = 2; n <= Q; ++n) {
            double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
            p0 = p1;
            p1 = p2;
        }
        dp = Q * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;   /* ascending order */
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* ------------------------------------------------------------------------ */
/* beta branch (Sec. 1): a2 = |alpha_n|^2.                                   */
/*   beta = sqrt(k^2 - a2)       if a2 <= k^2                                */
/*   beta = i sqrt(a2 - k^2)     otherwise                                    */
/* k^2 - a2 is formed as (k - a)(k + a) with a = sqrt(a2).                    */
/* ------------------------------------------------------------------------ */
static cplx beta_of(double k, double a2)
{
    double a = sqrt(a2);
    if (a <= k) return sqrt((k - a) * (k + a));
    return I * sqrt((a - k) * (a + k));
}

void or_beta(double k, double a2, double *re, double *im)
{
    cplx b = beta_of(k, a2);
    *re = creal(b);
    *im = cimag(b);
}

/* ------------------------------------------------------------------------ */
/* Bessel J0, J1 (2D only): trapezoidal rule on Bessel's integral            */
/*   J_n(z) = (1/2pi) int_0^{2pi} cos(n th - z sin th) d th,                  */
/* exponentially convergent for this periodic integrand once the number of    */
/* points exceeds |z| + n by a margin.                                        */
/* ------------------------------------------------------------------------ */
void or_bessel_j01(double z, double *j0, double *j1)
{
    int P = 2 * (int)ceil(fabs(z)) + 64;
    double s0 = 0.0, s1 = 0.0;
    for (int m = 0; m < P; ++m) {
        double th = 2.0 * M_PI * m / P;
        double sn = sin(th);
        s0 += cos(-z * sn);
        s1 += cos(th - z * sn);
    }
    *j0 = s0 / P;
    *j1 = s1 / P;
}

/* ------------------------------------------------------------------------ */
/* Integrals of the cutoff derivative X' appearing in (fck-coef) / (kdj1):    */
/*   I(gamma) = int_0^{c~} e^{i gamma t} X'(t) dt                             */
/* X' vanishes outside [c, (c+c~)/2], so Gauss-Legendre on that interval.     */
/* ------------------------------------------------------------------------ */
static cplx chi_prime_integral(const or_params *p, const double *gx, const double *gw, cplx gamma)
{
    double a = p->c, b = 0.5 * (p->c + p->ct);
    double hw = 0.5 * (b - a), mid = 0.5 * (a + b);
    cplx s = 0.0;
    for (int m = 0; m < p->Q; ++m) {
        double t = mid + hw * gx[m];
        s += gw[m] * hw * cexp(I * gamma * t) * or_chi(t, p->c, p->ct, 1);
    }
    return s;
}

/* sqrt(V) * K-hat_j for the periodised, cut-off K (Eq. (fck-coef), 2D; Eq.
 * (kdj1), 3D).  a2 = |alpha_j|^2 of the in-plane wave vector, q = j_last pi/c~.
 *   sqrt(V) K-hat = 1/(a2 + q^2 - k^2)
 *                 + I(beta - q) / (2 beta (q - beta))
 *                 - I(beta + q) / (2 beta (q + beta))                        */
static cplx sqrtV_Khat(const or_params *p, const double *gx, const double *gw, double a2, double q)
{
    cplx beta = beta_of(p->k, a2);
    cplx I1 = chi_prime_integral(p, gx, gw, beta - q);
    cplx I2 = chi_prime_integral(p, gx, gw, beta + q);
    return 1.0 / (a2 + q * q - p->k * p->k)
         + I1 / (2.0 * beta * (q - beta))
         - I2 / (2.0 * beta * (q + beta));
}

/* 3D singular part, Eq. (fj):  sqrt(V) F-hat_j = (1 - h(s)) / (s^2 - k^2),
 * s = |xi_j|, where the 3D integral of
 *     e^{ik|x|}/(4 pi |x|) (2 i k Y' + Y'') e^{-i xi.x}
 * is reduced to the radial form (the integrand is radial):
 *     h(s) = int_eps^{2eps} e^{ikr} (2ik Y'(r) + Y''(r)) sin(s r)/s dr,
 * with sin(sr)/s -> r at s = 0.  Gauss-Legendre on [eps, 2 eps]. */
static cplx singular_h3(const or_params *p, const double *gx, const double *gw, double s)
{
    double a = p->eps, b = 2.0 * p->eps;
    double hw = 0.5 * (b - a), mid = 0.5 * (a + b);
    cplx acc = 0.0;
    for (int m = 0; m < p->Q; ++m) {
        double r = mid + hw * gx[m];
        double ker = (s == 0.0) ? r : sin(s * r) / s;
        cplx f = cexp(I * p->k * r) * (2.0 * I * p->k * or_yps(r, p->eps, 1) + or_yps(r, p->eps, 2));
        acc += gw[m] * hw * f * ker;
    }
    return acc;
}

/* Phi_1(r) = (2 + ln r) Y'(r)/r + Y''(r) ln r  (Sec. 2.2). */
static double Phi1(double r, double eps)
{
    return (2.0 + log(r)) * or_yps(r, eps, 1) / r + or_yps(r, eps, 2) * log(r);
}

/* 2D singular parts, Eqs. (fcf1-coef) and (fcf2-coef), scaled by sqrt(V):
 *   eta = (j1, j2 pi/c~),
 *   sqrt(V) Phi1-hat = 2 pi int Phi_1(r) J0(|eta| r) r dr
 *   sqrt(V) Phi2-hat = -2 pi i (j1/|eta|) int Phi_1(r) J1(|eta| r) r^2 dr
 *   sqrt(V) F1-hat   = (1 + sqrt(V) Phi1-hat/(2 pi)) / |eta|^2
 *   sqrt(V) F2-hat   = (-2 i j1 sqrt(V) F1-hat + sqrt(V) Phi2-hat/(2 pi)) / |eta|^2
 * and at j = 0:  sqrt(V) F1-hat_0 = -int_0^{2eps} t ln t Y(t) dt, F2-hat_0 = 0,
 * the [0, eps] part in closed form eps^2/2 ln eps - eps^2/4.
 * (The radial forms follow from the Fourier transform of radial functions in
 * the plane; Phi_1 and Y', Y'' vanish outside [eps, 2 eps].) */
static void sqrtV_F12hat(const or_params *p, const double *gx, const double *gw,
                         int j1, double q, cplx *F1, cplx *F2)
{
    double a = p->eps, b = 2.0 * p->eps;
    double hw = 0.5 * (b - a), mid = 0.5 * (a + b);
    double eta2 = (double)j1 * j1 + q * q;
    if (eta2 == 0.0) {
        double e = p->eps;
        double acc = 0.5 * e * e * log(e) - 0.25 * e * e;
        for (int m = 0; m < p->Q; ++m) {
            double t = mid + hw * gx[m];
            acc += gw[m] * hw * t * log(t) * or_yps(t, e, 0);
        }
        *F1 = -acc;
        *F2 = 0.0;
        return;
    }
    double eta = sqrt(eta2);
    double s0 = 0.0, s1 = 0.0;
    for (int m = 0; m < p->Q; ++m) {
        double r = mid + hw * gx[m];
        double J0, J1;
        or_bessel_j01(eta * r, &J0, &J1);
        double ph = Phi1(r, p->eps);
        s0 += gw[m] * hw * ph * J0 * r;
        s1 += gw[m] * hw * ph * J1 * r * r;
    }
    cplx Phi1hat = 2.0 * M_PI * s0;
    cplx Phi2hat = -2.0 * M_PI * I * ((double)j1 / eta) * s1;
    *F1 = (1.0 + Phi1hat / (2.0 * M_PI)) / eta2;
    *F2 = (-2.0 * I * (double)j1 * (*F1) + Phi2hat / (2.0 * M_PI)) / eta2;
}

/* signed frequency of FFT-order index b on an axis of M points */
static int freq_of(int b, int M) { return b < M / 2 ? b : b - M; }

static int nfields(const or_params *p) { return (p->dim == 3 && p->maxwell) ? 7 : 1; }

/* Number of Maxwell fields stored by or_coef / or_grid: L_d followed by the six
 * L^{pq} in the order xx, yy, zz, xy, xz, yz. */
static const int PQ[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};

/* Remainder coefficients sqrt(V) L-hat_j for every j in S_N, stored in FFT
 * order (index b_i = j_i mod M_i), layout [field][b3][b2][b1] (3D) or
 * [b2][b1] (2D), complex interleaved.
 *   2D (Eq. (fcl-coef)):  L-hat = K-hat - F1-hat + i alpha F2-hat.
 *   3D (Algorithm 2, step 1b):  L-hat_d = K-hat_d - F-hat.
 *   Maxwell (Algorithm 3, step 1c): L-hat^{pq} = -c^p c^q L-hat_d with
 *   c = (alpha1 + j1, alpha2 + j2, j3 pi/c~).
 * Returns 0, or -1 on a Wood anomaly (beta = 0) or resonance (beta = +-q). */
int or_coef(const or_params *p, double *out)
{
    double *gx = malloc(sizeof(double) * p->Q), *gw = malloc(sizeof(double) * p->Q);
    or_gauss_legendre(p->Q, gx, gw);
    int bad = 0;
    cplx *C = (cplx *)out;
    if (p->dim == 2) {
        int M1 = p->M[0], M2 = p->M[1];
#pragma omp parallel for collapse(2) schedule(dynamic, 16) reduction(| : bad)
        for (int b2 = 0; b2 < M2; ++b2)
            for (int b1 = 0; b1 < M1; ++b1) {
                int j1 = freq_of(b1, M1), j2 = freq_of(b2, M2);
                double a = p->alpha[0] + j1, q = j2 * M_PI / p->ct;
                cplx beta = beta_of(p->k, a * a);
                if (cabs(beta) == 0.0 || cabs(beta - q) == 0.0 || cabs(beta + q) == 0.0) bad = 1;
                cplx K = sqrtV_Khat(p, gx, gw, a * a, q);
                cplx F1, F2;
                sqrtV_F12hat(p, gx, gw, j1, q, &F1, &F2);
                C[(size_t)b2 * M1 + b1] = K - F1 + I * p->alpha[0] * F2;
            }
    } else {
        int M1 = p->M[0], M2 = p->M[1], M3 = p->M[2];
        size_t NN = (size_t)M1 * M2 * M3;
        int nf = nfields(p);
#pragma omp parallel for collapse(3) schedule(dynamic, 16) reduction(| : bad)
        for (int b3 = 0; b3 < M3; ++b3)
            for (int b2 = 0; b2 < M2; ++b2)
                for (int b1 = 0; b1 < M1; ++b1) {
                    int j1 = freq_of(b1, M1), j2 = freq_of(b2, M2), j3 = freq_of(b3, M3);
                    double a1 = p->alpha[0] + j1, a2 = p->alpha[1] + j2;
                    double q = j3 * M_PI / p->ct;
                    double A2 = a1 * a1 + a2 * a2;
                    cplx beta = beta_of(p->k, A2);
                    if (cabs(beta) == 0.0 || cabs(beta - q) == 0.0 || cabs(beta + q) == 0.0) bad = 1;
                    cplx K = sqrtV_Khat(p, gx, gw, A2, q);
                    double s = sqrt(A2 + q * q);
                    cplx F = (1.0 - singular_h3(p, gx, gw, s)) / (A2 + q * q - p->k * p->k);
                    cplx L = K - F;
                    size_t idx = ((size_t)b3 * M2 + b2) * M1 + b1;
                    C[idx] = L;
                    if (nf == 7) {
                        double cv[3] = {a1, a2, q};
                        for (int e = 0; e < 6; ++e)
                            C[(size_t)(1 + e) * NN + idx] = -cv[PQ[e][0]] * cv[PQ[e][1]] * L;
                    }
                }
    }
    free(gx);
    free(gw);
    return bad ? -1 : 0;
}

/* Diagnostic parts of one coefficient (for the coefficient pins):
 * 3D: out = {sqrt(V) K-hat_d, sqrt(V) F-hat};  2D: {sqrt(V) K-hat, sqrt(V) F1-hat, sqrt(V) F2-hat}. */
void or_coef_parts(const or_params *p, int j1, int j2, int j3, double *out)
{
    double *gx = malloc(sizeof(double) * p->Q), *gw = malloc(sizeof(double) * p->Q);
    or_gauss_legendre(p->Q, gx, gw);
    cplx *o = (cplx *)out;
    if (p->dim == 2) {
        double a = p->alpha[0] + j1, q = j2 * M_PI / p->ct;
        o[0] = sqrtV_Khat(p, gx, gw, a * a, q);
        sqrtV_F12hat(p, gx, gw, j1, q, &o[1], &o[2]);
    } else {
        double a1 = p->alpha[0] + j1, a2 = p->alpha[1] + j2, q = j3 * M_PI / p->ct;
        double A2 = a1 * a1 + a2 * a2;
        o[0] = sqrtV_Khat(p, gx, gw, A2, q);
        double s = sqrt(A2 + q * q);
        o[1] = (1.0 - singular_h3(p, gx, gw, s)) / (A2 + q * q - p->k * p->k);
    }
    free(gx);
    free(gw);
}

/* ------------------------------------------------------------------------ */
/* Grid synthesis: L_N(x_l) = V^{-1} sum_{j in S_N} C_j exp(i pi sum j_i l_i/N_i) */
/* (Eqs. (fcln), (ln); C_j = sqrt(V) L-hat_j).  Naive O(M^2) inverse DFT,     */
/* one axis after the other (row-column).  Node index l_i in [0, M_i) stands  */
/* for the node x_i = l_i h_i, taken modulo the period.                       */
/* ------------------------------------------------------------------------ */
static void idft_axis(cplx *a, const int *dims, int ndim, int axis)
{
    /* dims[0] is the fastest axis.  A line along `axis` has stride s_axis. */
    size_t stride = 1;
    for (int d = 0; d < axis; ++d) stride *= dims[d];
    int M = dims[axis];
    size_t total = 1;
    for (int d = 0; d < ndim; ++d) total *= dims[d];
    size_t nlines = total / M;
    cplx *tw = malloc(sizeof(cplx) * M);
    for (int m = 0; m < M; ++m) tw[m] = cos(2.0 * M_PI * m / M) + I * sin(2.0 * M_PI * m / M);
#pragma omp parallel for schedule(static)
    for (size_t L = 0; L < nlines; ++L) {
        size_t lo = L % stride, hi = L / stride;
        size_t base = hi * stride * M + lo;
        cplx *in = malloc(sizeof(cplx) * M);
        for (int j = 0; j < M; ++j) in[j] = a[base + (size_t)j * stride];
        for (int l = 0; l < M; ++l) {
            cplx s = 0.0;
            for (int j = 0; j < M; ++j) s += in[j] * tw[((size_t)j * l) % M];
            a[base + (size_t)l * stride] = s;
        }
        free(in);
    }
    free(tw);
}

/* grid = V^{-1} * IDFT(C) for every field; C and grid may alias. */
void or_grid(const or_params *p, const double *C, double *grid)
{
    int ndim = p->dim;
    int dims[3] = {p->M[0], p->M[1], ndim == 3 ? p->M[2] : 1};
    size_t NN = (size_t)dims[0] * dims[1] * dims[2];
    int nf = nfields(p);
    double V = (ndim == 3) ? 8.0 * M_PI * M_PI * p->ct : 4.0 * M_PI * p->ct;
    cplx *g = (cplx *)grid;
    if (grid != C) memcpy(grid, C, sizeof(cplx) * NN * nf);
    for (int f = 0; f < nf; ++f) {
        cplx *a = g + (size_t)f * NN;
        for (int ax = 0; ax < ndim; ++ax) idft_axis(a, dims, ndim, ax);
        for (size_t i = 0; i < NN; ++i) a[i] /= V;
    }
}

/* ------------------------------------------------------------------------ */
/* Point evaluation helpers.                                                  */
/* ------------------------------------------------------------------------ */

/* x = 2 pi n + t with t in [-pi, pi)  (Algorithm 1 step 2c, Algorithm 2 step 2c). */
static void reduce_period(double x, double *t, double *n)
{
    double nn = floor((x + M_PI) / (2.0 * M_PI));
    double tt = x - 2.0 * M_PI * nn;
    if (tt >= M_PI) { tt -= 2.0 * M_PI; nn += 1.0; }
    if (tt < -M_PI) { tt += 2.0 * M_PI; nn -= 1.0; }
    *t = tt;
    *n = nn;
}

/* cubic Lagrange weights on the nodes -1, 0, 1, 2 at offset f in [0,1) */
static void lagrange4(double f, double w[4])
{
    w[0] = -f * (f - 1.0) * (f - 2.0) / 6.0;
    w[1] = (f + 1.0) * (f - 1.0) * (f - 2.0) / 2.0;
    w[2] = -(f + 1.0) * f * (f - 2.0) / 2.0;
    w[3] = (f + 1.0) * f * (f - 1.0) / 6.0;
}

/* Stencil of the coordinate y on an axis whose node a (a = 0..M-1) sits at
 * y0 + a h modulo the period: u = (y - y0)/h, i0 = floor(u), f = u - i0,
 * stencil nodes (i0 - 1 .. i0 + 2) mod M.  With node index l standing for
 * l h (mod period) and y0 = -M h / 2, node a is index (a + M/2) mod M. */
static void stencil(double y, double y0, double h, int M, int idx[4], double w[4])
{
    double u = (y - y0) / h;
    double i0 = floor(u);
    double f = u - i0;
    lagrange4(f, w);
    long base = (long)i0;
    for (int d = 0; d < 4; ++d) {
        long a = base - 1 + d + M / 2;
        a %= M;
        if (a < 0) a += M;
        idx[d] = (int)a;
    }
}

/* Tensor cubic interpolation (Sec. 2.3 "bicubic ... nearest 16 points";
 * Sec. 3.3 tricubic, 64 points).  Returns the interpolant of one field. */
static cplx interp3(const cplx *g, const int *M, const double u[3], const double y0[3], const double h[3])
{
    int i1[4], i2[4], i3[4];
    double w1[4], w2[4], w3[4];
    stencil(u[0], y0[0], h[0], M[0], i1, w1);
    stencil(u[1], y0[1], h[1], M[1], i2, w2);
    stencil(u[2], y0[2], h[2], M[2], i3, w3);
    cplx s = 0.0;
    for (int c = 0; c < 4; ++c)
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a)
                s += w3[c] * w2[b] * w1[a] * g[((size_t)i3[c] * M[1] + i2[b]) * M[0] + i1[a]];
    return s;
}

static cplx interp2(const cplx *g, const int *M, const double u[2], const double y0[2], const double h[2])
{
    int i1[4], i2[4];
    double w1[4], w2[4];
    stencil(u[0], y0[0], h[0], M[0], i1, w1);
    stencil(u[1], y0[1], h[1], M[1], i2, w2);
    cplx s = 0.0;
    for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) s += w2[b] * w1[a] * g[(size_t)i2[b] * M[0] + i1[a]];
    return s;
}

/* Interpolate field values at fractional grid coordinates (test hook for the
 * interpolation pins): y[i] in the same units as the axis coordinates. */
void or_interp(const or_params *p, const double *grid, const double *y, long n, double *out)
{
    const cplx *g = (const cplx *)grid;
    cplx *o = (cplx *)out;
    if (p->dim == 3) {
        double h[3] = {2.0 * M_PI / p->M[0], 2.0 * M_PI / p->M[1], 2.0 * p->ct / p->M[2]};
        double y0[3] = {-M_PI, -M_PI, -p->ct};
        for (long i = 0; i < n; ++i) o[i] = interp3(g, p->M, y + 3 * i, y0, h);
    } else {
        double h[2] = {2.0 * M_PI / p->M[0], 2.0 * p->ct / p->M[1]};
        double y0[2] = {-M_PI, -p->ct};
        for (long i = 0; i < n; ++i) o[i] = interp2(g, p->M, y + 2 * i, y0, h);
    }
}

/* number of series terms kept: |alpha_n|^2 <= k^2 + (T/|z|)^2, T = ln(1/tau) + 3 */
static double series_radius2(const or_params *p, double z)
{
    double T = log(1.0 / p->tau) + 3.0;
    double r = T / fabs(z);
    return p->k * p->k + r * r;
}

/* ------------------------------------------------------------------------ */
/* Eigenfunction expansions (exact reference and far branch).                 */
/*   2D (ei): G   = (i/4pi)    sum_n beta_n^{-1} e^{i alpha_n x1 + i beta_n |x2|}   */
/*   3D (he): G_d = (i/8pi^2)  sum_n beta_n^{-1} e^{i alpha_n.x' + i beta_n |x3|}  */
/*   Maxwell (me)/(mg): G_pq = delta_pq G_d + k^{-2} d_p d_q G_d, where d_p d_q  */
/*   multiplies each term by -c^p c^q, c = (alpha1+n1, alpha2+n2, beta sgn x3).   */
/* The in-plane coordinate is reduced first (x = 2 pi m + t) and the phase     */
/* e^{i 2 pi alpha.m} applied at the end, which is the same sum.              */
/* which: 1 = G_d, 2 = six tensor entries, 3 = six entries + G_d.             */
/* ------------------------------------------------------------------------ */
static void series_point(const or_params *p, const double *x, int which, cplx *out)
{
    double k = p->k;
    if (p->dim == 2) {
        double t, m;
        reduce_period(x[0], &t, &m);
        double z = fabs(x[1]);
        double R2 = series_radius2(p, x[1]);
        double R = sqrt(R2);
        long nlo = (long)floor(-p->alpha[0] - R) - 1, nhi = (long)ceil(-p->alpha[0] + R) + 1;
        cplx s = 0.0;
        for (long n = nlo; n <= nhi; ++n) {
            double a = p->alpha[0] + n;
            if (a * a > R2) continue;
            cplx beta = beta_of(k, a * a);
            s += cexp(I * a * t + I * beta * z) / beta;
        }
        double ph = p->alpha[0] * m;
        ph -= round(ph);
        out[0] = cexp(2.0 * M_PI * I * ph) * (I / (4.0 * M_PI)) * s;
        return;
    }
    double t1, m1, t2, m2;
    reduce_period(x[0], &t1, &m1);
    reduce_period(x[1], &t2, &m2);
    double z = fabs(x[2]);
    double sg = x[2] >= 0.0 ? 1.0 : -1.0;
    double R2 = series_radius2(p, x[2]);
    double R = sqrt(R2);
    long n1lo = (long)floor(-p->alpha[0] - R) - 1, n1hi = (long)ceil(-p->alpha[0] + R) + 1;
    long n2lo = (long)floor(-p->alpha[1] - R) - 1, n2hi = (long)ceil(-p->alpha[1] + R) + 1;
    cplx sG = 0.0, sT[6] = {0, 0, 0, 0, 0, 0};
    for (long n1 = n1lo; n1 <= n1hi; ++n1)
        for (long n2 = n2lo; n2 <= n2hi; ++n2) {
            double a1 = p->alpha[0] + n1, a2 = p->alpha[1] + n2;
            double A2 = a1 * a1 + a2 * a2;
            if (A2 > R2) continue;
            cplx beta = beta_of(k, A2);
            cplx term = cexp(I * (a1 * t1 + a2 * t2) + I * beta * z) / beta;
            sG += term;
            if (which >= 2) {
                cplx cv[3] = {a1, a2, beta * sg};
                for (int e = 0; e < 6; ++e) sT[e] += -cv[PQ[e][0]] * cv[PQ[e][1]] * term;
            }
        }
    double ph = p->alpha[0] * m1 + p->alpha[1] * m2;
    ph -= round(ph);
    cplx pre = cexp(2.0 * M_PI * I * ph) * (I / (8.0 * M_PI * M_PI));
    if (which == 1) {
        out[0] = pre * sG;
        return;
    }
    for (int e = 0; e < 6; ++e) {
        cplx d = (PQ[e][0] == PQ[e][1]) ? sG : 0.0;
        out[e] = pre * (d + sT[e] / (k * k));
    }
    if (which == 3) out[6] = pre * sG;
}

static int n_entries(int which) { return which == 2 ? 6 : which == 3 ? 7 : 1; }

/* Direct eigen-series at arbitrary points (exact reference; far branch). */
void or_series(const or_params *p, const double *x, long n, int which, double *out)
{
    int ne = n_entries(which);
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(dynamic, 4)
    for (long i = 0; i < n; ++i) series_point(p, x + (size_t)p->dim * i, which, o + (size_t)ne * i);
}

/* ------------------------------------------------------------------------ */
/* Algorithms 1-3, calculation step, at n points.                             */
/* grid: output of or_grid (one field, or seven for Maxwell).                 */
/* which: 0 = G (2D), 1 = G_d, 2 = six tensor entries, 3 = six + G_d.         */
/* ------------------------------------------------------------------------ */
static void eval_point(const or_params *p, const cplx *g, const double *x, int which, cplx *out)
{
    double k = p->k;
    if (p->dim == 2) {
        /* Algorithm 1 step 2b: branch on |x2| */
        if (fabs(x[1]) > p->c) { series_point(p, x, 0, out); return; }
        double t, m;
        reduce_period(x[0], &t, &m);                          /* step 2c */
        double h[2] = {2.0 * M_PI / p->M[0], 2.0 * p->ct / p->M[1]};
        double y0[2] = {-M_PI, -p->ct};
        double u[2] = {t, x[1]};
        cplx L = interp2(g, p->M, u, y0, h);                  /* step 2d */
        double r = sqrt(t * t + x[1] * x[1]);
        cplx Kv = L;
        if (r < 2.0 * p->eps) {
            double f1 = -log(r) * or_yps(r, p->eps, 0) / (2.0 * M_PI);
            double f2 = t * f1;                               /* f2 = x1 f1 at (t, x2) */
            Kv += f1 - I * p->alpha[0] * f2;                  /* K_N = L_N + f1 - i alpha f2 */
        }
        double ph = p->alpha[0] * m;
        ph -= round(ph);
        /* step 2e: G = e^{i alpha x1} K = e^{i alpha t} e^{i 2 pi alpha m} K */
        out[0] = cexp(I * p->alpha[0] * t) * cexp(2.0 * M_PI * I * ph) * Kv;
        return;
    }
    /* Algorithms 2 / 3, step 2b: branch on |x3| */
    if (which == 4 && fabs(x[2]) > p->c) { out[0] = NAN; return; }
    if (fabs(x[2]) > p->c) { series_point(p, x, which, out); return; }
    double t1, m1, t2, m2;
    reduce_period(x[0], &t1, &m1);                            /* step 2c */
    reduce_period(x[1], &t2, &m2);
    double h[3] = {2.0 * M_PI / p->M[0], 2.0 * M_PI / p->M[1], 2.0 * p->ct / p->M[2]};
    double y0[3] = {-M_PI, -M_PI, -p->ct};
    double u[3] = {t1, t2, x[2]};
    size_t NN = (size_t)p->M[0] * p->M[1] * p->M[2];
    cplx back = cexp(-I * (p->alpha[0] * t1 + p->alpha[1] * t2));
    double r = sqrt(t1 * t1 + t2 * t2 + x[2] * x[2]);
    double ph = p->alpha[0] * m1 + p->alpha[1] * m2;
    ph -= round(ph);
    cplx lift = cexp(I * (p->alpha[0] * t1 + p->alpha[1] * t2)) * cexp(2.0 * M_PI * I * ph);

    cplx Ld = interp3(g, p->M, u, y0, h);                     /* step 2d */
    /* F = e^{-i alpha.t} e^{ikr}/(4 pi r) Y_eps(r)  (Sec. 3.2), zero for r >= 2 eps */
    cplx F = 0.0, Phi = 0.0, dPhi = 0.0, d2Phi = 0.0;
    if (r < 2.0 * p->eps) {
        cplx gr = cexp(I * k * r) / (4.0 * M_PI * r);
        cplx g1 = gr * (I * k - 1.0 / r);
        cplx g2 = gr * ((I * k - 1.0 / r) * (I * k - 1.0 / r) + 1.0 / (r * r));
        double Y0 = or_yps(r, p->eps, 0), Y1 = or_yps(r, p->eps, 1), Y2 = or_yps(r, p->eps, 2);
        Phi = gr * Y0;
        dPhi = g1 * Y0 + gr * Y1;
        d2Phi = g2 * Y0 + 2.0 * g1 * Y1 + gr * Y2;
        F = back * Phi;
    }
    if (which == 4) { out[0] = Ld; return; }                  /* the remainder alone (step 2d) */
    cplx Kd = Ld + F;                                         /* step 2e */
    if (which <= 1) { out[0] = lift * Kd; return; }           /* step 2f + lift */

    /* Algorithm 3: seven interpolations, K^{pq} = L^{pq} + F^{pq}, with
     * F^{pq} = e^{-i alpha.x'} d_p d_q [Phi(r)] and
     * d_p d_q Phi = Phi'' xh_p xh_q + (Phi'/r)(delta_pq - xh_p xh_q). */
    double xv[3] = {t1, t2, x[2]};
    for (int e = 0; e < 6; ++e) {
        int P = PQ[e][0], Qq = PQ[e][1];
        cplx Lpq = interp3(g + (size_t)(1 + e) * NN, p->M, u, y0, h);
        cplx Fpq = 0.0;
        if (r < 2.0 * p->eps) {
            double xp = xv[P] / r, xq = xv[Qq] / r;
            double dl = (P == Qq) ? 1.0 : 0.0;
            Fpq = back * (d2Phi * xp * xq + (dPhi / r) * (dl - xp * xq));
        }
        cplx Kpq = Lpq + Fpq;
        cplx Gd = lift * Kd, D2 = lift * Kpq;                 /* steps 2g, 2h */
        out[e] = ((P == Qq) ? Gd : 0.0) + D2 / (k * k);       /* step 2i, Eq. (mg) */
    }
    if (which == 3) out[6] = lift * Kd;
}

void or_eval(const or_params *p, const double *grid, const double *x, long n, int which, double *out)
{
    int ne = n_entries(which);
    const cplx *g = (const cplx *)grid;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < n; ++i) eval_point(p, g, x + (size_t)p->dim * i, which, o + (size_t)ne * i);
}

/* ------------------------------------------------------------------------ */
/* Far-region grid.  The paper sums the eigen-series (he) for |x3| > c         */
/* (Algorithm 2 step 2b); the far-region grid replaces it on a slab           */
/* c < |x3| <= zmax by the same device as the near branch: for z = |x3| > 0   */
/*   F(t, z) = e^{-i alpha.t} G_d(t, z)                                       */
/*           = (i/8pi^2) sum_n beta_n^{-1} e^{i beta_n z} e^{i n.t}           */
/* is smooth and 2pi-periodic in t, its coefficients decaying like            */
/* e^{-|n| z}.  Planes m = 0 .. Nz + 2 sit at z_m = c + (m - 1) hz,           */
/* hz = (zmax - c)/Nz; on each, F at the Mf1 x Mf2 in-plane nodes (node l at  */
/* x = l h, h = 2 pi/Mf, as for the near grid) is the inverse DFT of           */
/* a_n(z_m) = (i/8pi^2) e^{i beta_n z_m}/beta_n over -Mf/2 <= n_i < Mf/2.      */
/* Maxwell (Sec. 4): seven fields, the six combined                           */
/* (delta_pq - c^p c^q/k^2) a_n with c = (alpha_n, beta_n) (z > 0), then a_n. */
/* Layout [field][m][l2][l1].                                                 */
/* ------------------------------------------------------------------------ */
void or_far_grid(const or_params *p, int Mf1, int Mf2, int Nz, double zmax, double *out)
{
    const int nz = Nz + 3, nf = nfields(p);
    const double hz = (zmax - p->c) / Nz;
    const size_t per = (size_t)Mf1 * Mf2 * nz;
    cplx *g = (cplx *)out;
    for (int m = 0; m < nz; ++m) {
        const double z = p->c + (m - 1) * hz;
        for (int b2 = 0; b2 < Mf2; ++b2)
            for (int b1 = 0; b1 < Mf1; ++b1) {
                const int n1 = freq_of(b1, Mf1), n2 = freq_of(b2, Mf2);
                const double a1 = p->alpha[0] + n1, a2 = p->alpha[1] + n2;
                const cplx beta = beta_of(p->k, a1 * a1 + a2 * a2);
                const cplx an = (I / (8.0 * M_PI * M_PI)) * cexp(I * beta * z) / beta;
                const size_t idx = ((size_t)m * Mf2 + b2) * Mf1 + b1;
                if (nf == 1) {
                    g[idx] = an;
                } else {
                    const cplx cv[3] = {a1, a2, beta};
                    for (int e = 0; e < 6; ++e) {
                        const cplx d = (PQ[e][0] == PQ[e][1]) ? 1.0 : 0.0;
                        g[(size_t)e * per + idx] = (d - cv[PQ[e][0]] * cv[PQ[e][1]] / (p->k * p->k)) * an;
                    }
                    g[(size_t)6 * per + idx] = an;
                }
            }
    }
    /* naive inverse DFT along x1, then x2, of every plane of every field */
    int dims[3] = {Mf1, Mf2, nz};
    for (int f = 0; f < nf; ++f) {
        idft_axis(g + (size_t)f * per, dims, 3, 0);
        idft_axis(g + (size_t)f * per, dims, 3, 1);
    }
}

/* Far-grid evaluation of targets with c < |x3| <= zmax (the caller sends only
 * those): reduce t, interpolate the far grid by tensor cubics (in-plane as the
 * near grid, periodic; in z from the plane origin c - hz with the stencil
 * origin clamped to Nz, the last full interval), lift by e^{i alpha.t}
 * e^{i 2 pi alpha.m}.  which: 1 = G_d, 2 / 3 = six tensor entries (/ + G_d);
 * the xz and yz entries change sign with x3. */
void or_eval_far_grid(const or_params *p, int Mf1, int Mf2, int Nz, double zmax, const double *fgrid,
                      const double *x, long n, int which, double *out)
{
    const int nz = Nz + 3, ne = n_entries(which);
    const double hz = (zmax - p->c) / Nz;
    const size_t per = (size_t)Mf1 * Mf2 * nz;
    const cplx *g = (const cplx *)fgrid;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < n; ++i) {
        const double *xi = x + 3 * i;
        double t1, m1, t2, m2;
        reduce_period(xi[0], &t1, &m1);
        reduce_period(xi[1], &t2, &m2);
        const double z = fabs(xi[2]);
        int i1[4], i2[4];
        double w1[4], w2[4], w3[4];
        stencil(t1, -M_PI, 2.0 * M_PI / Mf1, Mf1, i1, w1);
        stencil(t2, -M_PI, 2.0 * M_PI / Mf2, Mf2, i2, w2);
        double u3 = (z - (p->c - hz)) / hz;
        double i03 = floor(u3);
        if (i03 > (double)Nz) i03 = (double)Nz;
        lagrange4(u3 - i03, w3);
        const int m0 = (int)i03 - 1;
        double ph = p->alpha[0] * m1 + p->alpha[1] * m2;
        ph -= round(ph);
        const cplx lift = cexp(I * (p->alpha[0] * t1 + p->alpha[1] * t2)) * cexp(2.0 * M_PI * I * ph);
        for (int e = 0; e < ne; ++e) {
            const int f = (which <= 1) ? 0 : (e < 6 ? e : 6);
            cplx s = 0.0;
            for (int c3 = 0; c3 < 4; ++c3)
                for (int b = 0; b < 4; ++b)
                    for (int a = 0; a < 4; ++a)
                        s += w3[c3] * w2[b] * w1[a] *
                             g[(size_t)f * per + ((size_t)(m0 + c3) * Mf2 + i2[b]) * Mf1 + i1[a]];
            if (which >= 2 && (e == 4 || e == 5) && xi[2] < 0.0) s = -s;
            o[(size_t)ne * i + e] = lift * s;
        }
    }
}

/* Grid values at selected nodes only, straight from the truncated series
 * (no FFT, no row-column split): L_N(x_l) = V^{-1} sum_j C_j e^{2 pi i sum j_i l_i / M_i}.
 * Used to check single grid values of very large grids. nodes: [n][dim] ints. */
void or_grid_nodes(const or_params *p, const double *C, int field, const int *nodes, long n, double *out)
{
    int ndim = p->dim;
    int M1 = p->M[0], M2 = p->M[1], M3 = ndim == 3 ? p->M[2] : 1;
    size_t NN = (size_t)M1 * M2 * M3;
    const cplx *c = (const cplx *)C + (size_t)field * NN;
    double V = (ndim == 3) ? 8.0 * M_PI * M_PI * p->ct : 4.0 * M_PI * p->ct;
    cplx *o = (cplx *)out;
    for (long i = 0; i < n; ++i) {
        int l1 = nodes[ndim * i], l2 = nodes[ndim * i + 1], l3 = ndim == 3 ? nodes[ndim * i + 2] : 0;
        cplx s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
        for (int b3 = 0; b3 < M3; ++b3) {
            cplx s3 = 0.0;
            for (int b2 = 0; b2 < M2; ++b2)
                for (int b1 = 0; b1 < M1; ++b1) {
                    long ph = ((long)b1 * l1) % M1 * (long)(M2 * M3) + ((long)b2 * l2) % M2 * (long)(M1 * M3) +
                              ((long)b3 * l3) % M3 * (long)(M1 * M2);
                    double arg = 2.0 * M_PI * (double)(ph % (long)NN) / (double)NN;
                    s3 += c[((size_t)b3 * M2 + b2) * M1 + b1] * (cos(arg) + I * sin(arg));
                }
            s += s3;
        }
        o[i] = s / V;
    }
}

/* ======================================================================== */
/* 2D derivatives (Sec. 2.4).                                                 */
/*   Sec. 2.4.1: K_1 = e^{-i alpha x1} dG/dx1, K_2 = e^{-i alpha x1} dG/dx2,     */
/*     with Fourier coefficients i(alpha + j1) K-hat_j and i (j2 pi/c~) K-hat_j; */
/*     singular parts h_1, h_2 removed, K_i - h_i synthesised by inverse DFT,   */
/*     interpolated, h_i added back.                                          */
/*   Sec. 2.4.2: T_pq = K^{(k)}_pq - K^{(k2)}_pq, the differences of            */
/*     e^{-i alpha x1} d_p d_q G for two wave numbers, coefficients            */
/*     -(alpha+j1)^2 dK-hat, -(alpha+j1)(j2 pi/c~) dK-hat, -(j2 pi/c~)^2 dK-hat  */
/*     (dK-hat = K-hat^{(k)} - K-hat^{(k2)}), singular parts h_11, h_12, h_22.  */
/* The singular parts, with two readings of the printed text (derived from  */
/* (i/4) H_0(kr) = -(1/2pi) ln r + (k^2/8pi) r^2 ln r + smooth, times         */
/* e^{-i alpha x1} = 1 - i alpha x1 - alpha^2 x1^2/2 + ...):                   */
/*   h_1  = -(1/2pi) [ -(k^2/2) x1 ln r + x1/r^2 - i alpha x1^2/r^2             */
/*                     - (alpha^2/2) x1^3/r^2 ] Y                               */
/*   h_2  = -(1/2pi) [ -(k^2/2) x2 ln r + x2/r^2 - i alpha x1 x2/r^2            */
/*                     - (alpha^2/2) x1^2 x2/r^2 ] Y      (x2 ln r, not x1 ln r) */
/*   h_11 = +(dk2/2pi) [ ln r/2 - (i alpha/2) x1 ln r + x1^2/(2 r^2)           */
/*                       - i alpha x1^3/(2 r^2) ] Y                             */
/*   h_12 = +(dk2/2pi) [ x1 x2/(2 r^2) - (i alpha/2) x1^2 x2/r^2 ] Y            */
/*   h_22 = +(dk2/2pi) [ ln r/2 - (i alpha/2) x1 ln r + x2^2/(2 r^2)           */
/*                       - (i alpha/2) x1 x2^2/r^2 ] Y                          */
/* with dk2 = k^2 - k2^2 (the + sign: d_11 of (k^2/8pi) r^2 ln r is            */
/* (k^2/2pi)(ln r/2 + x1^2/(2r^2)) + const), Y = Y_eps(r).                     */
/* ======================================================================== */

/* J_0 .. J_3 at z together, by the trapezoidal rule on Bessel's integral with
 * P >= |z| + 16 (|z|/2 + 1)^{1/3} + 40 points: the rule's error is made of the
 * aliases J_{P -+ n}(z), which decay faster than e^{-30} once the order
 * passes |z| by that margin (Airy-type decay beyond the turning point). */
static void bessel_j0123(double z, double J[4])
{
    int P = (int)(fabs(z) + 16.0 * cbrt(0.5 * fabs(z) + 1.0)) + 40;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int m = 0; m < P; ++m) {
        double th = 2.0 * M_PI * m / P, zs = z * sin(th);
        for (int n = 0; n < 4; ++n) s[n] += cos(n * th - zs);
    }
    for (int n = 0; n < 4; ++n) J[n] = s[n] / P;
}

void or_bessel_j0123(double z, double *J) { bessel_j0123(z, J); }

/* The five Hankel integrals of the cutoff int_0^{2 eps} Y(r) J_n(rho r) r^pw dr
 * used below, (n, pw) = (1,0), (0,1), (2,1), (1,2), (3,2), into out[0..4].
 * The integrand is analytic on [0, eps] (Y = 1) and on [eps, 2 eps] (Y a
 * polynomial); each piece is cut into 1 + rho eps / 16 panels (at most about
 * three oscillations of J_n(rho r) per panel) of Gauss-Legendre with the
 * plan's Q nodes. */
static void hankel_Y5(const or_params *p, const double *gx, const double *gw, double rho, double out[5])
{
    double e = p->eps;
    int np = 1 + (int)(rho * e / 16.0);
    for (int i = 0; i < 5; ++i) out[i] = 0.0;
    for (int piece = 0; piece < 2; ++piece) {
        double a0 = piece * e, w = e / np;
        for (int s = 0; s < np; ++s) {
            double a = a0 + s * w, hw = 0.5 * w, mid = a + hw;
            for (int m = 0; m < p->Q; ++m) {
                double r = mid + hw * gx[m], J[4];
                bessel_j0123(rho * r, J);
                double y = (piece == 0 ? 1.0 : or_yps(r, e, 0)) * gw[m] * hw;
                out[0] += y * J[1];
                out[1] += y * J[0] * r;
                out[2] += y * J[2] * r;
                out[3] += y * J[1] * r * r;
                out[4] += y * J[3] * r * r;
            }
        }
    }
}

/* sqrt(V) times the coefficients of x2 ln r Y scaled like f_2: the x2 analogue
 * of (fcf2-coef), F2'-hat = (-2 i eta2 F1-hat + Phi2'-hat/(2 pi))/|eta|^2 with
 * Phi2' = x2 Phi_1 (the same derivation: Delta(x2 g) = x2 Delta g + 2 d2 g). */
static cplx sqrtV_F2y(const or_params *p, const double *gx, const double *gw, int j1, double q, cplx F1)
{
    double eta2 = (double)j1 * j1 + q * q;
    if (eta2 == 0.0) return 0.0;
    double eta = sqrt(eta2), a = p->eps, b = 2.0 * p->eps;
    double hw = 0.5 * (b - a), mid = 0.5 * (a + b), s1 = 0.0;
    for (int m = 0; m < p->Q; ++m) {
        double r = mid + hw * gx[m];
        double J0, J1;
        or_bessel_j01(eta * r, &J0, &J1);
        s1 += gw[m] * hw * Phi1(r, p->eps) * J1 * r * r;
    }
    cplx Phi2y = -2.0 * M_PI * I * (q / eta) * s1;
    return (-2.0 * I * q * F1 + Phi2y / (2.0 * M_PI)) / eta2;
}

/* The plane Fourier transforms int int g(x) e^{-i eta.x} dx (= sqrt(V) times
 * the coefficient) of the singular functions g, eta = (j1, q), by the
 * angular reduction  FT[g(r) cos(m th)] = 2 pi (-i)^m cos(m phi) int g J_m(rho r) r dr
 * (and sin for sin), rho = |eta|, eta = rho (cos phi, sin phi):
 *   out[0] P0  = FT[ln r Y]        = -2 pi sqrt(V) F1-hat
 *   out[1] P1c = FT[x1 ln r Y]     = -2 pi sqrt(V) F2-hat
 *   out[2] P1s = FT[x2 ln r Y]     = -2 pi sqrt(V) F2'-hat
 *   out[3] Q1c = FT[x1/r^2 Y],  out[4] Q1s = FT[x2/r^2 Y]       (m = 1 of Y/r)
 *   out[5] R0  = FT[Y]                                           (m = 0)
 *   out[6] R2c = FT[cos 2th Y], out[7] R2s = FT[sin 2th Y]       (m = 2)
 *   out[8] S1c = FT[x1 Y],      out[9] S1s = FT[x2 Y]             (m = 1 of r Y)
 *   out[10] S3c = FT[r cos 3th Y], out[11] S3s = FT[r sin 3th Y]  (m = 3 of r Y) */
static void singular_transforms(const or_params *p, const double *gx, const double *gw, int j1, double q, cplx *out)
{
    cplx F1, F2;
    sqrtV_F12hat(p, gx, gw, j1, q, &F1, &F2);
    out[0] = -2.0 * M_PI * F1;
    out[1] = -2.0 * M_PI * F2;
    out[2] = -2.0 * M_PI * sqrtV_F2y(p, gx, gw, j1, q, F1);
    double rho = sqrt((double)j1 * j1 + q * q), hk[5];
    hankel_Y5(p, gx, gw, rho, hk);
    out[5] = 2.0 * M_PI * hk[1];
    if (rho == 0.0) {
        for (int i = 3; i < 12; ++i)
            if (i != 5) out[i] = 0.0;
        return;
    }
    double cp = j1 / rho, sp = q / rho;
    double c2 = cp * cp - sp * sp, s2 = 2.0 * cp * sp;
    double c3 = cp * (4.0 * cp * cp - 3.0), s3 = sp * (3.0 - 4.0 * sp * sp);
    double q1 = hk[0], r2 = hk[2], s1 = hk[3], s3v = hk[4];
    out[3] = -2.0 * M_PI * I * cp * q1;
    out[4] = -2.0 * M_PI * I * sp * q1;
    out[6] = -2.0 * M_PI * c2 * r2;
    out[7] = -2.0 * M_PI * s2 * r2;
    out[8] = -2.0 * M_PI * I * cp * s1;
    out[9] = -2.0 * M_PI * I * sp * s1;
    out[10] = 2.0 * M_PI * I * c3 * s3v;
    out[11] = 2.0 * M_PI * I * s3 * s3v;
}

/* sqrt(V) times the coefficients of h_1, h_2, h_11, h_12, h_22 (in that order)
 * from the transforms above (x1^2/r^2 = (1 + cos 2th)/2, x2^2/r^2 = (1 - cos 2th)/2,
 * x1 x2/r^2 = sin 2th/2, x1^3/r^2 = r (3 cos th + cos 3th)/4,
 * x1^2 x2/r^2 = r (sin th + sin 3th)/4, x1 x2^2/r^2 = r (cos th - cos 3th)/4). */
static void sqrtV_Hhat(const or_params *p, const double *gx, const double *gw, double k2, int j1, double q,
                       cplx *H)
{
    cplx T[12];
    singular_transforms(p, gx, gw, j1, q, T);
    double al = p->alpha[0], kk = p->k * p->k, dk2 = p->k * p->k - k2 * k2;
    cplx x1sq = 0.5 * (T[5] + T[6]), x2sq = 0.5 * (T[5] - T[6]), x1x2 = 0.5 * T[7];
    cplx x1cub = 0.25 * (3.0 * T[8] + T[10]), x1sqx2 = 0.25 * (T[9] + T[11]), x1x2sq = 0.25 * (T[8] - T[10]);
    H[0] = -(1.0 / (2.0 * M_PI)) * (-0.5 * kk * T[1] + T[3] - I * al * x1sq - 0.5 * al * al * x1cub);
    H[1] = -(1.0 / (2.0 * M_PI)) * (-0.5 * kk * T[2] + T[4] - I * al * x1x2 - 0.5 * al * al * x1sqx2);
    H[2] = (dk2 / (2.0 * M_PI)) * (0.5 * T[0] - 0.5 * I * al * T[1] + 0.5 * x1sq - I * al * 0.5 * x1cub);
    H[3] = (dk2 / (2.0 * M_PI)) * (0.5 * x1x2 - 0.5 * I * al * x1sqx2);
    H[4] = (dk2 / (2.0 * M_PI)) * (0.5 * T[0] - 0.5 * I * al * T[1] + 0.5 * x2sq - 0.5 * I * al * x1x2sq);
}

/* Diagnostic: the twelve transforms and the five sqrt(V) H-hat of one index. */
void or_deriv2_parts(const or_params *p, double k2, int j1, int j2, double *out)
{
    double *gx = malloc(sizeof(double) * p->Q), *gw = malloc(sizeof(double) * p->Q);
    or_gauss_legendre(p->Q, gx, gw);
    double q = j2 * M_PI / p->ct;
    singular_transforms(p, gx, gw, j1, q, (cplx *)out);
    sqrtV_Hhat(p, gx, gw, k2, j1, q, (cplx *)out + 12);
    free(gx);
    free(gw);
}

/* Remainder coefficients of the five derivative fields, sqrt(V)-scaled, FFT
 * order, layout [field][b2][b1], fields K_1 - h_1, K_2 - h_2, T_11 - h_11,
 * T_12 - h_12, T_22 - h_22 (the last three only when k2 > 0).  Returns 0, or
 * -1 on a Wood anomaly or resonance for k or k2. */
int or_coef_deriv2(const or_params *p, double k2, double *out)
{
    double *gx = malloc(sizeof(double) * p->Q), *gw = malloc(sizeof(double) * p->Q);
    or_gauss_legendre(p->Q, gx, gw);
    or_params p2 = *p;
    p2.k = k2;
    int M1 = p->M[0], M2 = p->M[1], nf = k2 > 0.0 ? 5 : 2, bad = 0;
    size_t NN = (size_t)M1 * M2;
    cplx *C = (cplx *)out;
#pragma omp parallel for collapse(2) schedule(dynamic, 16) reduction(| : bad)
    for (int b2 = 0; b2 < M2; ++b2)
        for (int b1 = 0; b1 < M1; ++b1) {
            int j1 = freq_of(b1, M1), j2 = freq_of(b2, M2);
            double a = p->alpha[0] + j1, q = j2 * M_PI / p->ct;
            cplx beta = beta_of(p->k, a * a);
            if (cabs(beta) == 0.0 || cabs(beta - q) == 0.0 || cabs(beta + q) == 0.0) bad = 1;
            cplx K = sqrtV_Khat(p, gx, gw, a * a, q), H[5];
            sqrtV_Hhat(p, gx, gw, k2 > 0.0 ? k2 : p->k, j1, q, H);
            size_t i = (size_t)b2 * M1 + b1;
            C[i] = I * a * K - H[0];
            C[NN + i] = I * q * K - H[1];
            if (nf == 5) {
                cplx beta2 = beta_of(k2, a * a);
                if (cabs(beta2) == 0.0 || cabs(beta2 - q) == 0.0 || cabs(beta2 + q) == 0.0) bad = 1;
                cplx dK = K - sqrtV_Khat(&p2, gx, gw, a * a, q);
                C[2 * NN + i] = -a * a * dK - H[2];
                C[3 * NN + i] = -a * q * dK - H[3];
                C[4 * NN + i] = -q * q * dK - H[4];
            }
        }
    free(gx);
    free(gw);
    return bad ? -1 : 0;
}

/* The singular parts at (x1, x2) = (t, x2) in the cell, r < 2 eps (zero beyond):
 * out = {h_1, h_2, h_11, h_12, h_22}. */
static void deriv2_singular(const or_params *p, double k2, double x1, double x2, cplx *h)
{
    double r2 = x1 * x1 + x2 * x2, r = sqrt(r2);
    for (int e = 0; e < 5; ++e) h[e] = 0.0;
    if (r >= 2.0 * p->eps) return;
    double Y = or_yps(r, p->eps, 0), lr = log(r), al = p->alpha[0];
    double kk = p->k * p->k, dk2 = kk - k2 * k2;
    h[0] = -(1.0 / (2.0 * M_PI)) * (-0.5 * kk * x1 * lr + x1 / r2 - I * al * x1 * x1 / r2 - 0.5 * al * al * x1 * x1 * x1 / r2) * Y;
    h[1] = -(1.0 / (2.0 * M_PI)) * (-0.5 * kk * x2 * lr + x2 / r2 - I * al * x1 * x2 / r2 - 0.5 * al * al * x1 * x1 * x2 / r2) * Y;
    h[2] = (dk2 / (2.0 * M_PI)) * (0.5 * lr - 0.5 * I * al * x1 * lr + x1 * x1 / (2.0 * r2) - I * al * x1 * x1 * x1 / (2.0 * r2)) * Y;
    h[3] = (dk2 / (2.0 * M_PI)) * (x1 * x2 / (2.0 * r2) - 0.5 * I * al * x1 * x1 * x2 / r2) * Y;
    h[4] = (dk2 / (2.0 * M_PI)) * (0.5 * lr - 0.5 * I * al * x1 * lr + x2 * x2 / (2.0 * r2) - 0.5 * I * al * x1 * x2 * x2 / r2) * Y;
}

/* The singular parts at n points (x1, x2) of the cell, out = n x {h_1, h_2,
 * h_11, h_12, h_22} (test hook). */
void or_deriv2_singular_at(const or_params *p, double k2, const double *x, long n, double *out)
{
    cplx *o = (cplx *)out;
    for (long i = 0; i < n; ++i) deriv2_singular(p, k2, x[2 * i], x[2 * i + 1], o + 5 * i);
}

/* Term-by-term derivatives of (ei) (exact reference and far branch):
 *   dG/dx1 = (i/4pi) sum (i alpha_n/beta_n) E_n,  dG/dx2 = (i/4pi) sum i sgn(x2) E_n,
 *   d11 G = (i/4pi) sum (-alpha_n^2/beta_n) E_n, d12 G = (i/4pi) sum (-alpha_n sgn) E_n,
 *   d22 G = (i/4pi) sum (-beta_n) E_n,   E_n = e^{i alpha_n x1 + i beta_n |x2|};
 * which 0: {dG/dx1, dG/dx2};  which 1: {T_11, T_12, T_22} (k minus k2).
 * Truncated at |alpha_n|^2 <= max(k, k2)^2 + (T/|x2|)^2. */
static void series_deriv2_point(const or_params *p, double k2, const double *x, int which, cplx *out)
{
    double t, m;
    reduce_period(x[0], &t, &m);
    double z = fabs(x[1]), sg = x[1] >= 0.0 ? 1.0 : -1.0;
    double kmax = (which == 1 && k2 > p->k) ? k2 : p->k;
    double T = log(1.0 / p->tau) + 3.0, R2 = kmax * kmax + (T / z) * (T / z), R = sqrt(R2);
    long nlo = (long)floor(-p->alpha[0] - R) - 1, nhi = (long)ceil(-p->alpha[0] + R) + 1;
    cplx s[3] = {0.0, 0.0, 0.0};
    for (long n = nlo; n <= nhi; ++n) {
        double a = p->alpha[0] + n;
        if (a * a > R2) continue;
        cplx b1 = beta_of(p->k, a * a), E1 = cexp(I * a * t + I * b1 * z);
        if (which == 0) {
            s[0] += I * a / b1 * E1;
            s[1] += I * sg * E1;
        } else {
            cplx b2 = beta_of(k2, a * a), E2 = cexp(I * a * t + I * b2 * z);
            s[0] += -a * a * (E1 / b1 - E2 / b2);
            s[1] += -a * sg * (E1 - E2);
            s[2] += -(b1 * E1 - b2 * E2);
        }
    }
    double ph = p->alpha[0] * m;
    ph -= round(ph);
    cplx pre = cexp(2.0 * M_PI * I * ph) * (I / (4.0 * M_PI));
    for (int e = 0; e < (which == 0 ? 2 : 3); ++e) out[e] = pre * s[e];
}

void or_series_deriv2(const or_params *p, double k2, const double *x, long n, int which, double *out)
{
    int ne = which == 0 ? 2 : 3;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(dynamic, 4)
    for (long i = 0; i < n; ++i) series_deriv2_point(p, k2, x + 2 * i, which, o + (size_t)ne * i);
}

/* Algorithm 1's calculation step for the derivative fields: |x2| > c by the
 * differentiated series; otherwise x1 = 2 pi m + t, the remainder grids
 * (grid: the five (or two) fields of or_coef_deriv2 after or_grid, layout
 * [field][l2][l1]) interpolated at (t, x2), the singular parts added back and
 * the result lifted by e^{i alpha t} e^{i 2 pi alpha m}.
 * which 0: {dG/dx1, dG/dx2};  which 1: {T_11, T_12, T_22}. */
void or_eval_deriv2(const or_params *p, double k2, const double *grid, const double *x, long n, int which,
                    double *out)
{
    int ne = which == 0 ? 2 : 3, f0 = which == 0 ? 0 : 2;
    size_t NN = (size_t)p->M[0] * p->M[1];
    const cplx *g = (const cplx *)grid;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < n; ++i) {
        const double *xi = x + 2 * i;
        cplx *oi = o + (size_t)ne * i;
        if (fabs(xi[1]) > p->c) {
            series_deriv2_point(p, k2, xi, which, oi);
            continue;
        }
        double t, m;
        reduce_period(xi[0], &t, &m);
        double h[2] = {2.0 * M_PI / p->M[0], 2.0 * p->ct / p->M[1]};
        double y0[2] = {-M_PI, -p->ct};
        double u[2] = {t, xi[1]};
        cplx hs[5];
        deriv2_singular(p, k2, t, xi[1], hs);
        double ph = p->alpha[0] * m;
        ph -= round(ph);
        cplx lift = cexp(I * p->alpha[0] * t) * cexp(2.0 * M_PI * I * ph);
        for (int e = 0; e < ne; ++e) oi[e] = lift * (interp2(g + (size_t)(f0 + e) * NN, p->M, u, y0, h) + hs[f0 + e]);
    }
}
