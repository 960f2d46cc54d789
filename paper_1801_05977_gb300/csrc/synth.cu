// Plan-time device work (Algorithms 1-3, step 1): remainder Fourier
// coefficients (Eqs. (fck-coef), (fcl-coef)-(fcf2-coef), (kdj1), (fj), and the
// Maxwell multipliers of Sec. 4) generated in double precision and fused into
// the first inverse-FFT pass, then the remaining inverse-FFT passes, the last
// of which scatters the grid into the padded gather layout used at evaluation.
//
// Inverse DFT convention (Eqs. (fcln), (ln)): with C_j = sqrt(V) L-hat_j,
//   L_N(x_l) = V^{-1} sum_{j in S_N} C_j exp(2 pi i sum_i j_i l_i / M_i),
// node index l standing for x = l h (mod period).  Each pass is a radix-2
// Stockham autosort transform held in shared memory (one CTA owns a batch of
// whole lines, so every pass reads and writes global memory exactly once).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "gf_internal.cuh"
#include "umma_gemm.cuh"

namespace {

__device__ __forceinline__ int freq_of(int b, int M) { return b < (M >> 1) ? b : b - M; }

// beta branch of Sec. 1: sqrt(k^2 - a2) if a2 <= k^2, else i sqrt(a2 - k^2),
// with k^2 - a2 formed as (k - a)(k + a).
__device__ __forceinline__ double2 beta_of(double k, double a2)
{
    double a = sqrt(a2);
    if (a <= k) return make_double2(sqrt((k - a) * (k + a)), 0.0);
    return make_double2(0.0, sqrt((a - k) * (a + k)));
}

// The X'-integral terms of Eq. (fck-coef)/(kdj1) for one coefficient:
//   T1 - T2 = I1/(2 beta (q - beta)) - I2/(2 beta (q + beta)),
// I1 = sum A conj(E), I2 = sum A E over the Gauss nodes (A_m = w_m X'(t_m)
// e^{i beta t_m}, E_m = e^{i q t_m}).  Evanescent beta = i g: A_m is real, I1 =
// s1 - i s3, I2 = s1 + i s3 and T1 - T2 = (g s1 - q s3)/(g (g^2 + q^2)); for g >
// gskip both terms are below double rounding of the coefficient (|I| <= e^{-g c},
// |2 beta (q -+ beta)| >= 2 g^2) and are not formed.
__device__ __forceinline__ double2 xprime_terms(double2 beta, double q, const double2 *Am, const double2 *Em, int Q,
                                                double gskip)
{
    double2 T12 = make_double2(0.0, 0.0);
    if (beta.y > 0.0 && beta.y <= gskip) {
        double s1 = 0.0, s3 = 0.0;
        for (int m = 0; m < Q; ++m) {
            const double A = Am[m].x;
            const double2 E = Em[m];
            s1 = fma(A, E.x, s1);
            s3 = fma(A, E.y, s3);
        }
        const double g = beta.y;
        T12.x = (g * s1 - q * s3) / (g * (g * g + q * q));
    } else if (beta.y <= gskip) {
        double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
        for (int m = 0; m < Q; ++m) {
            const double2 A = Am[m], E = Em[m];
            s1 = fma(A.x, E.x, s1);
            s2 = fma(A.y, E.y, s2);
            s3 = fma(A.x, E.y, s3);
            s4 = fma(A.y, E.x, s4);
        }
        // propagating beta (real)
        const double2 I1 = make_double2(s1 + s2, s4 - s3);
        const double2 I2 = make_double2(s1 - s2, s3 + s4);
        const double2 tb = cscale(beta, 2.0);
        const double2 T1 = cdiv(I1, cmul(tb, make_double2(q - beta.x, -beta.y)));
        const double2 T2 = cdiv(I2, cmul(tb, make_double2(q + beta.x, beta.y)));
        T12 = csub(T1, T2);
    }
    return T12;
}

// Clenshaw sum of one panel's Chebyshev coefficients (two real functions packed
// in a double2) at x in [-1, 1].
__device__ __forceinline__ double2 cheb_eval(const double2 *cc, int deg, double x)
{
    double b1r = 0.0, b1i = 0.0, b2r = 0.0, b2i = 0.0;
    for (int kk = deg; kk >= 1; --kk) {
        const double2 ck = cc[kk];
        const double tr = fma(2.0 * x, b1r, ck.x - b2r);
        const double ti = fma(2.0 * x, b1i, ck.y - b2i);
        b2r = b1r;
        b2i = b1i;
        b1r = tr;
        b1i = ti;
    }
    return make_double2(fma(x, b1r, cc[0].x - b2r), fma(x, b1i, cc[0].y - b2i));
}

// e^{2 pi i m/n} for 0 <= m < n from the table of the first half (tw[m] =
// e^{2 pi i m/n}, m < n/2): the second half is its negative.
template <typename C>
__device__ __forceinline__ C twiddle(const C *tw, int m, int half)
{
    if (m < half) return tw[m];
    const C v = tw[m - half];
    return cmk(-v.x, -v.y);
}

// Stockham autosort inverse transform (+ sign, unnormalised) of `nlines`
// contiguous lines of length n = 2^lg held in shared memory x; y is scratch of
// the same size.  Radix-4 stages, preceded by one radix-2 stage when lg is odd:
// a stage that combines sub-transforms of length Ns takes, for j < n/4 and
// k = j mod Ns, v_r = x[j + r n/4] e^{2 pi i r k/(4 Ns)} and writes the 4-point
// inverse DFT of (v_0..v_3) to y[4(j - k) + k + m Ns], m = 0..3.  Returns the
// buffer holding the result.  All threads of the CTA must call it.
template <typename C>
__device__ C *stockham_inverse(C *x, C *y, int n, int lg, int nlines, const C *tw)
{
    const int half = n >> 1;
    int Ns = 1, lns = 0;
    if (lg & 1) {
        // radix 2, Ns = 1: no twiddles
        const int total = nlines * half;
        for (int it = threadIdx.x; it < total; it += blockDim.x) {
            const int L = it >> (lg - 1), j = it & (half - 1);
            const C *xl = x + L * n;
            C *yl = y + L * n;
            const C v0 = xl[j], v1 = xl[j + half];
            yl[2 * j] = cadd(v0, v1);
            yl[2 * j + 1] = csub(v0, v1);
        }
        __syncthreads();
        C *t = x;
        x = y;
        y = t;
        Ns = 2;
        lns = 1;
    }
    const int q = n >> 2;
    for (; Ns < n; Ns <<= 2, lns += 2) {
        const int total = nlines * q, sh = lg - 2 - lns;  // e^{2 pi i r k/(4 Ns)} = tw[(r k) << sh]
        for (int it = threadIdx.x; it < total; it += blockDim.x) {
            const int L = it >> (lg - 2), j = it & (q - 1), k = j & (Ns - 1);
            const C *xl = x + L * n;
            C *yl = y + L * n;
            const C a = xl[j];
            const C b = cmul(xl[j + q], twiddle(tw, k << sh, half));
            const C c = cmul(xl[j + 2 * q], twiddle(tw, (2 * k) << sh, half));
            const C d = cmul(xl[j + 3 * q], twiddle(tw, (3 * k) << sh, half));
            const C apc = cadd(a, c), amc = csub(a, c), bpd = cadd(b, d), bmd = csub(b, d);
            const int o = ((j - k) << 2) + k;
            yl[o] = cadd(apc, bpd);
            yl[o + Ns] = cmk(amc.x - bmd.y, amc.y + bmd.x);       // amc + i bmd
            yl[o + 2 * Ns] = csub(apc, bpd);
            yl[o + 3 * Ns] = cmk(amc.x + bmd.y, amc.y - bmd.x);   // amc - i bmd
        }
        __syncthreads();
        C *t = x;
        x = y;
        y = t;
    }
    return x;
}

// The same transform of nlines lines held in x, `group` lines at a time, with a
// scratch y of only `group` lines; the result is left in x.  Lets a pass hold
// every field of its lines plus one field's worth of scratch instead of two full
// copies.  All threads of the CTA must call it.
template <typename C>
__device__ void stockham_inverse_grouped(C *x, C *y, int n, int lg, int nlines, int group, const C *tw)
{
    for (int g0 = 0; g0 < nlines; g0 += group) {
        C *xg = x + (size_t)g0 * n;
        const C *res = stockham_inverse(xg, y, n, lg, group, tw);
        if (res != xg) {
            for (int i = threadIdx.x; i < group * n; i += blockDim.x) xg[i] = res[i];
            __syncthreads();
        }
    }
}

// tw[i] = e^{2 pi i i/n}, i < n/2, in the pass's precision (float passes take
// the float sincospi: within an ulp, and no double arithmetic in a float pass)
// The same transform on an interleaved tile: element j of line L at x[j NL + L]
// (NL = 2^lgNL lines), the layout a 2D tensor copy of NL adjacent columns gives.
// Consecutive threads take consecutive lines, so shared-memory accesses stay
// contiguous.  Returns the buffer holding the result.
template <typename C>
__device__ C *stockham_inverse_il(C *x, C *y, int n, int lg, int lgNL, const C *tw)
{
    const int half = n >> 1, NL = 1 << lgNL;
    int Ns = 1, lns = 0;
    if (lg & 1) {
        const int total = NL * half;
        for (int it = threadIdx.x; it < total; it += blockDim.x) {
            const int L = it & (NL - 1), j = it >> lgNL;
            const C v0 = x[j * NL + L], v1 = x[(j + half) * NL + L];
            y[(2 * j) * NL + L] = cadd(v0, v1);
            y[(2 * j + 1) * NL + L] = csub(v0, v1);
        }
        __syncthreads();
        C *t = x;
        x = y;
        y = t;
        Ns = 2;
        lns = 1;
    }
    const int q = n >> 2;
    for (; Ns < n; Ns <<= 2, lns += 2) {
        const int total = NL * q, sh = lg - 2 - lns;
        for (int it = threadIdx.x; it < total; it += blockDim.x) {
            const int L = it & (NL - 1), j = it >> lgNL, k = j & (Ns - 1);
            const C a = x[j * NL + L];
            const C b = cmul(x[(j + q) * NL + L], twiddle(tw, k << sh, half));
            const C c = cmul(x[(j + 2 * q) * NL + L], twiddle(tw, (2 * k) << sh, half));
            const C d = cmul(x[(j + 3 * q) * NL + L], twiddle(tw, (3 * k) << sh, half));
            const C apc = cadd(a, c), amc = csub(a, c), bpd = cadd(b, d), bmd = csub(b, d);
            const int o = ((j - k) << 2) + k;
            y[o * NL + L] = cadd(apc, bpd);
            y[(o + Ns) * NL + L] = cmk(amc.x - bmd.y, amc.y + bmd.x);
            y[(o + 2 * Ns) * NL + L] = csub(apc, bpd);
            y[(o + 3 * Ns) * NL + L] = cmk(amc.x + bmd.y, amc.y - bmd.x);
        }
        __syncthreads();
        C *t = x;
        x = y;
        y = t;
    }
    return x;
}

template <typename R>
__device__ void load_twiddles(typename cplx_t<R>::T *tw, int n)
{
    for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
        if (sizeof(R) == 4) {
            float s, c;
            sincospif(2.0f * (float)i / (float)n, &s, &c);
            tw[i] = cmk((R)c, (R)s);
        } else {
            double s, c;
            sincospi(2.0 * (double)i / (double)n, &s, &c);
            tw[i] = cmk((R)c, (R)s);
        }
    }
}

// The derivative fields of one 2D coefficient (Sec. 2.4), sqrt(V)-scaled before
// the 1/V of the synthesis: fields 1 .. nf-1 of buf0 (field 0, L, is the
// caller's).  K = sqrt(V) K-hat(k); eta = |(j1, q)| (0 at j = 0); F1 = sqrt(V)
// F1-hat; S1 = int Phi_1 J1(eta r) r^2 dr; (pnl, x) the Chebyshev panel and
// position of eta; Am2, beta2: the second wave number's X' weights and beta.
// The singular parts' coefficients come from plane transforms reduced by the
// angle, FT[g(r) cos(m th)] = 2 pi (-i)^m cos(m phi) int g J_m(eta r) r dr:
//   ln r Y -> -2 pi F1, x1 ln r Y -> -2 pi F2, x2 ln r Y -> -2 pi F2' (F2 with q
//   for j1), x_i/r^2 Y (m = 1 of Y/r: Q1), Y (R0), cos 2th Y, sin 2th Y (R2),
//   x_i Y (m = 1 of r Y: S1), r cos 3th Y, r sin 3th Y (S3),
// read from the dcheb tables (Q1, R0), (R2, S1), (S3, -); the even-angle
// transforms are real, the odd-angle ones imaginary, so H_1, H_2 are imaginary
// and H_11, H_12, H_22 real:
//   h_1  = -(1/2pi)[-(k^2/2) x1 ln r + x1/r^2 - i alpha x1^2/r^2 - (alpha^2/2) x1^3/r^2] Y
//   h_2  = -(1/2pi)[-(k^2/2) x2 ln r + x2/r^2 - i alpha x1 x2/r^2 - (alpha^2/2) x1^2 x2/r^2] Y
//   h_11 = (dk2/2pi)[ln r/2 - (i alpha/2) x1 ln r + x1^2/(2r^2) - i alpha x1^3/(2r^2)] Y
//   h_12 = (dk2/2pi)[x1 x2/(2r^2) - (i alpha/2) x1^2 x2/r^2] Y
//   h_22 = (dk2/2pi)[ln r/2 - (i alpha/2) x1 ln r + x2^2/(2r^2) - (i alpha/2) x1 x2^2/r^2] Y
// (dk2 = k^2 - k2^2), with x1^2/r^2 = (1 + cos 2th)/2, x2^2/r^2 = (1 - cos 2th)/2,
// x1 x2/r^2 = sin 2th/2, x1^3/r^2 = r (3 cos th + cos 3th)/4, x1^2 x2/r^2 =
// r (sin th + sin 3th)/4, x1 x2^2/r^2 = r (cos th - cos 3th)/4.  Then
//   K_1 - h_1: i (alpha + j1) K - H_1,   K_2 - h_2: i q K - H_2,
//   T_pq - h_pq: -c_p c_q (K - K(k2)) - H_pq,  c = (alpha + j1, q).
template <typename C>
__device__ void deriv_fields_2d(const SynthArgs &a, C *buf0, int TJ, int t, int n, int b, int jx, double q,
                                double eta, double F1, double S1, double2 K, double A2, const double2 *Am2,
                                const double2 *Em, double2 beta2, int pnl, double x)
{
    typedef decltype(C().x) R;
    const double ip = 2.0 * GF_PI, al = a.a1, kk = a.k * a.k, c1 = al + jx;
    const int nd = a.hdeg + 1;
    const size_t tab = (size_t)a.hnpan * nd;
    const double2 d0 = cheb_eval(a.dcheb + (size_t)pnl * nd, a.hdeg, x);            // (Q1, R0)
    const double2 d1 = cheb_eval(a.dcheb + tab + (size_t)pnl * nd, a.hdeg, x);      // (R2, S1)
    const double S3 = cheb_eval(a.dcheb + 2 * tab + (size_t)pnl * nd, a.hdeg, x).x;  // S3
    double cp = 0.0, sp = 0.0, f2i = 0.0, f2yi = 0.0;
    if (eta > 0.0) {
        cp = jx / eta;
        sp = q / eta;
        const double ie2 = 1.0 / (eta * eta);
        f2i = (-2.0 * jx * F1 - cp * S1) * ie2;   // sqrt(V) F2-hat = i f2i
        f2yi = (-2.0 * q * F1 - sp * S1) * ie2;   // its x2 analogue
    }
    const double c2 = cp * cp - sp * sp, s2 = 2.0 * cp * sp;
    const double c3 = cp * (4.0 * cp * cp - 3.0), s3 = sp * (3.0 - 4.0 * sp * sp);
    const double Q1 = d0.x, R0 = d0.y, R2 = d1.x, S1Y = d1.y;
    // real parts of the even-angle transforms, imaginary parts of the odd-angle ones
    const double x1sq = 0.5 * ip * (R0 - c2 * R2), x2sq = 0.5 * ip * (R0 + c2 * R2), x1x2 = -0.5 * ip * s2 * R2;
    const double x1cub = 0.25 * ip * (-3.0 * cp * S1Y + c3 * S3);
    const double x1sqx2 = 0.25 * ip * (-sp * S1Y + s3 * S3);
    const double x1x2sq = 0.25 * ip * (-cp * S1Y - c3 * S3);
    const double H1i = -((0.5 * kk) * ip * f2i - ip * cp * Q1 - al * x1sq - 0.5 * al * al * x1cub) / ip;
    const double H2i = -((0.5 * kk) * ip * f2yi - ip * sp * Q1 - al * x1x2 - 0.5 * al * al * x1sqx2) / ip;
    const double sc = a.invV;
    buf0[(1 * TJ + t) * n + b] = cmk((R)(-c1 * K.y * sc), (R)((c1 * K.x - H1i) * sc));
    buf0[(2 * TJ + t) * n + b] = cmk((R)(-q * K.y * sc), (R)((q * K.x - H2i) * sc));
    if (a.nf < 6) return;
    const double dk2 = kk - a.k2 * a.k2;
    const double2 T12 = xprime_terms(beta2, q, Am2, Em, a.Q, a.gskip);
    const double iD2 = 1.0 / (A2 + q * q - a.k2 * a.k2);
    const double2 dK = make_double2(K.x - (iD2 + T12.x), K.y - T12.y);
    const double base = -0.5 * ip * F1 - 0.5 * al * ip * f2i;  // P0/2 - (i alpha/2) P1c
    const double H11 = dk2 / ip * (base + 0.5 * x1sq + 0.5 * al * x1cub);
    const double H12 = dk2 / ip * (0.5 * x1x2 + 0.5 * al * x1sqx2);
    const double H22 = dk2 / ip * (base + 0.5 * x2sq + 0.5 * al * x1x2sq);
    const double f[3] = {-c1 * c1, -c1 * q, -q * q}, H[3] = {H11, H12, H22};
#pragma unroll
    for (int e = 0; e < 3; ++e)
        buf0[((3 + e) * TJ + t) * n + b] = cmk((R)((f[e] * dK.x - H[e]) * sc), (R)(f[e] * dK.y * sc));
}

// DERIV: the 2D derivative plans' instance (their extra fields, a second X'
// table); a separate instance so that the other plans' kernel keeps its registers.
template <typename R, bool DERIV>
__device__ void synth_first_pass_body(const SynthArgs &a, int blk, unsigned char *smem)
{
    typedef typename cplx_t<R>::T C;
    const int n = a.Mlast, lg = a.lgMlast, TJ = a.TJ, Q = a.Q, nf = a.nf;
    double2 *Av = reinterpret_cast<double2 *>(smem);   // [TJ][Q]
    double2 *betas = Av + TJ * Q;                        // [TJ]
    C *tw = reinterpret_cast<C *>(betas + TJ);           // [n/2]
    C *buf0 = tw + (n >> 1);                             // [nf][TJ][n]
    C *buf1 = buf0 + nf * TJ * n;                      // [TJ][n] scratch of the transforms
    double *A2s = reinterpret_cast<double *>(buf1 + TJ * n); // [TJ]
    // split plans, float coefficients: A_m [TJ][Q] (16-byte aligned so that the X'-integral
    // loop reads it four nodes at a time), |alpha_j|^2 in float [TJ]
    float *Avf = reinterpret_cast<float *>(reinterpret_cast<uintptr_t>(A2s + TJ + 1) & ~(uintptr_t)15);
    float *A2f = Avf + ((TJ * Q + 3) & ~3);
    // float-column data: |alpha_j|^2 - k^2 and q_b^2 as float pairs (hi, lo), g in
    // float, and per column bit 0 = X'-integrals skipped, bit 1 = float coefficient
    float2 *A2mkf = reinterpret_cast<float2 *>((reinterpret_cast<uintptr_t>(A2f + TJ) + 15) & ~(uintptr_t)15);
    float2 *qqf = A2mkf + TJ;
    float *gcol = reinterpret_cast<float *>(qqf + n);
    int *cflag = reinterpret_cast<int *>(gcol + TJ);
    // float copies of the quadrature weights and nodes [Q] each, q_b in float [n]
    float *tWs = reinterpret_cast<float *>(cflag + TJ);
    float *tts = tWs + Q;
    float *qfs = tts + Q;
    // 2D derivative plans with a second wave number: its A_m [TJ][Q] and beta [TJ]
    const bool need_k2 = DERIV && a.k2 > 0.0;
    double2 *Av2 = reinterpret_cast<double2 *>((reinterpret_cast<uintptr_t>(qfs + n) + 15) & ~(uintptr_t)15);
    double2 *betas2 = Av2 + TJ * Q;
    const int ncols = (a.dim == 3) ? a.M1 * a.M2 : a.M1;
    // tiles alternately from both ends of the column range: the low frequencies
    // (whose X'-integrals are formed, the expensive tiles) sit at both ends, so
    // they are scheduled first and the last wave holds the cheap middle
    const int ntiles = ncols / TJ;
    const int col0 = ((blk & 1) ? ntiles - 1 - (blk >> 1) : (blk >> 1)) * TJ;
    const bool fcoef = sizeof(R) == 4 && a.dim == 3;

    load_twiddles<R>(tw, n);
    for (int t = threadIdx.x; t < TJ; t += blockDim.x) {
        int col = col0 + t;
        double A2;
        if (a.dim == 3) {
            int jx = freq_of(col % a.M1, a.M1), jy = freq_of(col / a.M1, a.M2);
            double x1 = a.a1 + jx, x2 = a.a2 + jy;
            A2 = x1 * x1 + x2 * x2;
        } else {
            int jx = freq_of(col, a.M1);
            double x1 = a.a1 + jx;
            A2 = x1 * x1;
        }
        A2s[t] = A2;
        const double2 bt = beta_of(a.k, A2);
        betas[t] = bt;
        if (need_k2) betas2[t] = beta_of(a.k2, A2);
        if (fcoef) {
            const double d = A2 - a.k * a.k;
            A2f[t] = (float)A2;
            const float h = (float)d;
            A2mkf[t] = make_float2(h, (float)(d - (double)h));
            gcol[t] = (float)bt.y;
            cflag[t] = (bt.y > a.gskip ? 1 : 0) | (bt.y >= a.gfloat ? 2 : 0);
        }
    }
    if (fcoef) {
        // q_b = j q_s and q_b^2 as float pairs from q_s's pair (qsh, qsl), with no
        // double operation: j q_sh by TwoProd (j is an integer below 2^12), then the
        // square of the pair (its l^2 term dropped), about 2^-46 relative
        for (int b = threadIdx.x; b < n; b += blockDim.x) {
            const float jf = (float)freq_of(b, n);
            const float ph = jf * a.qsh;
            const float pl = __fmaf_rn(jf, a.qsh, -ph) + jf * a.qsl;
            const float h = ph * ph;
            const float l = __fmaf_rn(ph, ph, -h) + 2.0f * ph * pl;
            const float s = h + l;
            qqf[b] = make_float2(s, l - (s - h));
            qfs[b] = ph + pl;
        }
        for (int m = threadIdx.x; m < Q; m += blockDim.x) {
            tWs[m] = (float)a.tW[m];
            tts[m] = (float)a.tt[m];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TJ * Q; i += blockDim.x) {
        int t = i / Q, m = i - t * Q;
        if (fcoef) {
            // the column's flags: bit 0 skipped X'-integrals, bit 1 float coefficient
            const int f = cflag[t];
            if (f & 1) continue;
            if (f & 2) {
                Avf[i] = tWs[m] * expf(-gcol[t] * tts[m]);
                continue;
            }
        }
        double2 b = betas[t];
        if (b.y > a.gskip) continue;  // this column's X'-integrals are not used
        double tm = a.tt[m];
        double2 e;
        if (b.y == 0.0) {
            double s, c;
            sincos(b.x * tm, &s, &c);
            e = make_double2(c, s);
        } else {
            e = make_double2(exp(-b.y * tm), 0.0);
        }
        Av[i] = cscale(e, a.tW[m]);
    }
    if (need_k2)
        for (int i = threadIdx.x; i < TJ * Q; i += blockDim.x) {
            const int t = i / Q, m = i - t * Q;
            const double2 b = betas2[t];
            if (b.y > a.gskip) continue;
            const double tm = a.tt[m];
            double2 e;
            if (b.y == 0.0) {
                double sn, cs;
                sincos(b.x * tm, &sn, &cs);
                e = make_double2(cs, sn);
            } else {
                e = make_double2(exp(-b.y * tm), 0.0);
            }
            Av2[i] = cscale(e, a.tW[m]);
        }
    __syncthreads();

    const double k2 = a.k * a.k, ik2 = 1.0 / k2;
    // the float branch's constants, converted once
    const float ihpanf = (float)a.ihpan, hpanf = (float)a.hpan, invVf = (float)a.invV;
    // The coefficients are even in the last-axis index j (they depend on q_j
    // through q_j^2, and the two X' terms of Eqs. (fck-coef)/(kdj1) trade places
    // under q -> -q), except the Maxwell xz and yz fields, whose factor c^3 = q_j
    // makes them odd (Sec. 4).  Only b = 0 .. n/2 (j = 0 .. n/2 - 1 and the
    // Nyquist index j = -n/2) are formed here; b > n/2 (j = b - n) is filled
    // below from b' = n - b (j' = -j).
    // items: (t, b) for b < n/2 by shift and mask, then the Nyquist b = n/2 of each column
    const int nh = (n >> 1) + 1, lgh = lg - 1, nlow = TJ << lgh;
    const float hmaxf = (float)(a.hnpan - 1);
    for (int i = threadIdx.x; i < TJ * nh; i += blockDim.x) {
        const bool low = i < nlow;
        const int t = low ? (i >> lgh) : i - nlow, b = low ? (i & ((n >> 1) - 1)) : (n >> 1);
        int col = col0 + t;
        int jl = freq_of(b, n);
        if (fcoef && (cflag[t] & 2)) {
            // Split plans, evanescent column clear of Wood anomalies (g >= gfloat):
            // the coefficient in float, with no double operation.  D = |xi|^2 - k^2
            // (small near the resonance sphere) is the sum of two float pairs, exact
            // to ~2^-46 relative to its terms (Knuth's TwoSum), then rounded: since
            // |D| >= 1e-6 k^2 (the resonance rule), this is below float rounding of D.
            // Every other factor is O(1) in relative terms.
            const float qf = qfs[b];
            const float g = gcol[t];
            float T12f = 0.f;
            if (!(cflag[t] & 1)) {
                const float *Am = Avf + t * Q;
                const float2 *Em = a.Ef + (size_t)b * Q;
                float s1 = 0.f, s3 = 0.f;
                int m = 0;
                if ((Q & 3) == 0) {
                    // four nodes per step: one 16-byte shared load of A, two of E
                    const float4 *A4 = reinterpret_cast<const float4 *>(Am);
                    const float4 *E4 = reinterpret_cast<const float4 *>(Em);
                    for (int m4 = 0; m4 < (Q >> 2); ++m4) {
                        const float4 A = A4[m4], E01 = __ldg(E4 + 2 * m4), E23 = __ldg(E4 + 2 * m4 + 1);
                        s1 = fmaf(A.x, E01.x, s1);
                        s3 = fmaf(A.x, E01.y, s3);
                        s1 = fmaf(A.y, E01.z, s1);
                        s3 = fmaf(A.y, E01.w, s3);
                        s1 = fmaf(A.z, E23.x, s1);
                        s3 = fmaf(A.z, E23.y, s3);
                        s1 = fmaf(A.w, E23.z, s1);
                        s3 = fmaf(A.w, E23.w, s3);
                    }
                    m = Q;
                }
                for (; m < Q; ++m) {
                    const float A = Am[m];
                    const float2 E = Em[m];
                    s1 = fmaf(A, E.x, s1);
                    s3 = fmaf(A, E.y, s3);
                }
                T12f = (g * s1 - qf * s3) * __frcp_rn(g * (g * g + qf * qf));
            }
            const float2 Ad = A2mkf[t], Qd = qqf[b];
            const float dh = __fadd_rn(Ad.x, Qd.x), dv = __fsub_rn(dh, Ad.x);
            const float de = __fadd_rn(__fsub_rn(Ad.x, __fsub_rn(dh, dv)), __fsub_rn(Qd.x, dv));
            const float iD = __frcp_rn(__fadd_rn(dh, __fadd_rn(de, __fadd_rn(Ad.y, Qd.y))));
            // |xi| by the hardware reciprocal square root (its ~2^-23 relative error moves
            // the Chebyshev point by less than the float rounding of h)
            const float s2 = fmaf(qf, qf, A2f[t]);
            const float sf = s2 > 0.f ? s2 * rsqrtf(s2) : 0.f;
            const float pf = fminf(floorf(sf * ihpanf), hmaxf);
            const int pnl = (int)pf;
            const float x = (sf - (pf + 0.5f) * hpanf) * (2.0f / hpanf);
            const float2 *cc = a.hchebf + (size_t)pnl * (a.hdeg + 1);
            float b1r = 0.f, b1i = 0.f, b2r = 0.f, b2i = 0.f;
            for (int kk = a.hdeg; kk >= 1; --kk) {
                const float2 ck = cc[kk];
                const float tr = fmaf(2.0f * x, b1r, ck.x - b2r);
                const float ti = fmaf(2.0f * x, b1i, ck.y - b2i);
                b2r = b1r;
                b2i = b1i;
                b1r = tr;
                b1i = ti;
            }
            const float hr = fmaf(x, b1r, cc[0].x - b2r), hi = fmaf(x, b1i, cc[0].y - b2i);
            const float cr = fmaf(hr, iD, T12f) * invVf, ci = hi * iD * invVf;
            if (nf == 1) {
                buf0[t * n + b] = cmk((R)cr, (R)ci);
            } else {
                const int jx = freq_of(col % a.M1, a.M1), jy = freq_of(col / a.M1, a.M2);
                const float ik2f = (float)ik2;
                const float cv0 = (float)(a.a1 + jx), cv1 = (float)(a.a2 + jy), cv2 = qf;
                const float f[7] = {1.f - cv0 * cv0 * ik2f, 1.f - cv1 * cv1 * ik2f, 1.f - cv2 * cv2 * ik2f,
                                    -cv0 * cv1 * ik2f,      -cv0 * cv2 * ik2f,      -cv1 * cv2 * ik2f, 1.f};
#pragma unroll
                for (int e = 0; e < 7; ++e) buf0[(e * TJ + t) * n + b] = cmk((R)(f[e] * cr), (R)(f[e] * ci));
            }
            continue;
        }
        const double2 beta = betas[t];
        double q = (double)jl * a.qs;
        double A2 = A2s[t];
        const double2 *Am = Av + t * Q;
        const double2 *Em = a.E + (size_t)b * Q;
        const double2 T12 = xprime_terms(beta, q, Am, Em, Q, a.gskip);
        double D = A2 + q * q - k2;
        double2 Cj;
        if (a.dim == 3) {
            // h(s) = sum_m B_m sin(s r_m)/s, read from its piecewise Chebyshev
            // interpolant (Clenshaw); h has bandwidth 2 eps in s, so degree 14 on
            // panels of width 2 reproduces the quadrature to rounding.
            double s = sqrt(A2 + q * q);
            int pnl = min((int)(s * a.ihpan), a.hnpan - 1);
            double x = (s - (pnl + 0.5) * a.hpan) * (2.0 / a.hpan);
            const double2 *cc = a.hcheb + (size_t)pnl * (a.hdeg + 1);
            double b1r = 0.0, b1i = 0.0, b2r = 0.0, b2i = 0.0;
            for (int kk = a.hdeg; kk >= 1; --kk) {
                double2 ck = cc[kk];
                double tr = fma(2.0 * x, b1r, ck.x - b2r);
                double ti = fma(2.0 * x, b1i, ck.y - b2i);
                b2r = b1r;
                b2i = b1i;
                b1r = tr;
                b1i = ti;
            }
            double hr = fma(x, b1r, cc[0].x - b2r);
            double hi = fma(x, b1i, cc[0].y - b2i);
            const double iD = 1.0 / D;
            Cj = make_double2(fma(hr, iD, T12.x), fma(hi, iD, T12.y));
        } else {
            int jx = freq_of(col, a.M1);
            double2 K = make_double2(1.0 / D + T12.x, T12.y);
            double eta2 = (double)jx * jx + q * q;
            double2 F1, F2;
            if (eta2 == 0.0) {
                F1 = make_double2(a.F10, 0.0);
                F2 = make_double2(0.0, 0.0);
            } else {
                // S0 = sum_m P0_m J0(eta r_m), S1 = sum_m P1_m J1(eta r_m) from their
                // piecewise Chebyshev interpolants (band-limited in eta: r_m <= 2 eps)
                double eta = sqrt(eta2);
                int pnl = min((int)(eta * a.ihpan), a.hnpan - 1);
                double x = (eta - (pnl + 0.5) * a.hpan) * (2.0 / a.hpan);
                const double2 *cc = a.hcheb + (size_t)pnl * (a.hdeg + 1);
                double b1r = 0.0, b1i = 0.0, b2r = 0.0, b2i = 0.0;
                for (int kk = a.hdeg; kk >= 1; --kk) {
                    double2 ck = cc[kk];
                    double tr = fma(2.0 * x, b1r, ck.x - b2r);
                    double ti = fma(2.0 * x, b1i, ck.y - b2i);
                    b2r = b1r;
                    b2i = b1i;
                    b1r = tr;
                    b1i = ti;
                }
                const double S0 = fma(x, b1r, cc[0].x - b2r);
                const double S1 = fma(x, b1i, cc[0].y - b2i);
                // F1 = (1 + Phi1-hat/(2 pi))/eta^2,  Phi1-hat/(2 pi) = S0
                F1 = make_double2((1.0 + S0) / eta2, 0.0);
                // F2 = (-2 i j1 F1 + Phi2-hat/(2 pi))/eta^2,  Phi2-hat/(2 pi) = -i (j1/eta) S1
                F2 = make_double2(0.0, (-2.0 * jx * F1.x - ((double)jx / eta) * S1) / eta2);
                if (DERIV) deriv_fields_2d(a, buf0, TJ, t, n, b, jx, q, eta, F1.x, S1, K, A2, Av2 + t * Q, Em,
                                             need_k2 ? betas2[t] : make_double2(0.0, 0.0), pnl, x);
            }
            if (DERIV && eta2 == 0.0) deriv_fields_2d(a, buf0, TJ, t, n, b, jx, q, 0.0, F1.x, 0.0, K, A2, Av2 + t * Q,
                                                        Em, need_k2 ? betas2[t] : make_double2(0.0, 0.0), 0, -1.0);
            // C = K - F1 + i alpha F2
            Cj = make_double2(K.x - F1.x - a.a1 * F2.y, K.y - F1.y + a.a1 * F2.x);
            if (DERIV) {
                Cj = cscale(Cj, a.invV);
                buf0[t * n + b] = cmk((R)Cj.x, (R)Cj.y);
                continue;
            }
        }
        Cj = cscale(Cj, a.invV);
        if (nf == 1) {
            buf0[t * n + b] = cmk((R)Cj.x, (R)Cj.y);
        } else {
            // Maxwell (Sec. 4): combined fields (delta_pq - c^p c^q / k^2) C, c = (alpha1+j1, alpha2+j2, q),
            // order xx, yy, zz, xy, xz, yz, then the plain field C (for G_d).
            int jx = freq_of(col % a.M1, a.M1), jy = freq_of(col / a.M1, a.M2);
            double cv0 = a.a1 + jx, cv1 = a.a2 + jy, cv2 = q;
            double f[7] = {1.0 - cv0 * cv0 * ik2, 1.0 - cv1 * cv1 * ik2, 1.0 - cv2 * cv2 * ik2,
                           -cv0 * cv1 * ik2,      -cv0 * cv2 * ik2,      -cv1 * cv2 * ik2, 1.0};
#pragma unroll
            for (int e = 0; e < 7; ++e) buf0[(e * TJ + t) * n + b] = cmk((R)(f[e] * Cj.x), (R)(f[e] * Cj.y));
        }
    }
    __syncthreads();
    C *W = reinterpret_cast<C *>(a.work);
    const int planes = a.L3count + a.nyq;  // 3D work planes per field
    if (a.nyq) {
        // the odd fields' Nyquist coefficients (b = n/2, j3 = -n/2), before the x3 transform
        for (int i = threadIdx.x; i < 2 * TJ; i += blockDim.x) {
            const int f = 4 + i / TJ, t = i % TJ;
            W[((size_t)f * planes + a.L3count) * ncols + col0 + t] = buf0[(f * TJ + t) * n + (n >> 1)];
        }
    }
    {
        const int nm = (n >> 1) - 1;  // b = n/2 + 1 .. n - 1
        for (int i = threadIdx.x; i < nf * TJ * nm; i += blockDim.x) {
            const int line = i / nm, b = (n >> 1) + 1 + (i - line * nm);
            const int e = line / TJ;
            const C v = buf0[line * n + (n - b)];
            // the odd fields (Maxwell xz, yz; 2D K_2, T_12) change sign with j
            buf0[line * n + b] = ((a.oddmask >> e) & 1) ? cmk(-v.x, -v.y) : v;
        }
    }
    __syncthreads();
    stockham_inverse_grouped(buf0, buf1, n, lg, nf * TJ, TJ, tw);
    const C *res = buf0;
    if (a.dim == 3) {
        // only the x3 nodes the last two passes transform (a3first .. a3first +
        // L3count - 1), compact: work plane y holds node a3first + y, whose output
        // index is l = (a + n/2) mod n
        const int tot = nf * a.L3count * TJ;
        for (int i = threadIdx.x; i < tot; i += blockDim.x) {
            const int t = i % TJ, rest = i / TJ;
            const int y = rest % a.L3count, f = rest / a.L3count;
            const int l = (a.a3first + y + (n >> 1)) & (n - 1);
            W[((size_t)f * planes + y) * ncols + col0 + t] = res[(f * TJ + t) * n + l];
        }
    } else {
        const int tot = nf * n * TJ;
        for (int i = threadIdx.x; i < tot; i += blockDim.x) {
            int t = i % TJ;
            int rest = i / TJ;
            int l = rest & (n - 1);
            int f = rest >> lg;
            W[((size_t)f * n + l) * ncols + col0 + t] = res[(f * TJ + t) * n + l];
        }
    }
}

// Middle pass (3D only): inverse transform along x2 for fixed (field, x3 node, b1-tile);
// only the x3 nodes of the stored planes are transformed.
template <typename R>
__device__ void synth_x2_body(const SynthArgs &a, int bx, int y, int f, unsigned char *smem)
{
    typedef typename cplx_t<R>::T C;
    const int n = a.M2, TJ = a.TJ2, lg2 = a.lg2;
    // x3 node a3first + y, stored at plane y of the (compact) work buffer
    C *tw = reinterpret_cast<C *>(smem);
    C *buf0 = tw + (n >> 1);
    C *buf1 = buf0 + TJ * n;
    const int b10 = bx * TJ;
    // work plane L3count (half-grid Maxwell plans) holds the Nyquist row of the odd fields only
    if (y == a.L3count && f != 4 && f != 5) return;
    C *W = reinterpret_cast<C *>(a.work) + ((size_t)f * (a.L3count + a.nyq) + y) * (size_t)a.M2 * a.M1;
    load_twiddles<R>(tw, n);
    for (int i = threadIdx.x; i < TJ * n; i += blockDim.x) {
        int t = i % TJ, b2 = i / TJ;
        buf0[t * n + b2] = W[(size_t)b2 * a.M1 + b10 + t];
    }
    __syncthreads();
    C *res = stockham_inverse(buf0, buf1, n, lg2, TJ, tw);
    for (int i = threadIdx.x; i < TJ * n; i += blockDim.x) {
        int t = i % TJ, l2 = i / TJ;
        W[(size_t)l2 * a.M1 + b10 + t] = res[t * n + l2];
    }
}

__device__ __forceinline__ int pad_dests(int a_node, int M, int *p)
{
    // padded index p = a + 1 for a in [-1, M+1]; node a is periodic mod M
    int nd = 0;
    p[nd++] = a_node + 1;
    if (a_node <= 1) p[nd++] = a_node + 1 + M;
    if (a_node == M - 1) p[nd++] = 0;
    return nd;
}

// Last pass: inverse transform along x1 of RB1 consecutive rows (all fields),
// then scatter into the padded, field-interleaved gather grid G[p3][p2][p1][f],
// where padded index p = a + 1 holds node a = (l + M/2) mod M, i.e. x = -pi + a h
// (x3: -c~ + a h3), with one halo node before and two after on every periodic
// axis so that a cubic stencil never wraps.
template <typename R>
__device__ void synth_x1_body(const SynthArgs &a, int blk, unsigned char *smem, uint64_t *bar, uint32_t parity)
{
    typedef typename cplx_t<R>::T C;
    const int n = a.M1, nf = a.nf, lg1 = a.lg1, RB = a.RB1;
    C *tw = reinterpret_cast<C *>(smem);
    C *buf0 = tw + (n >> 1);       // [nf][RB][n]: each field's RB rows, as stored in the work buffer
    C *buf1 = buf0 + RB * nf * n;  // [RB][n] scratch of the transforms
    // row = y * M2 + l2 (3D: x3 node a3first + y at compact work plane y); 2D: l2
    const size_t fstride = (size_t)(a.dim == 3 ? (a.L3count + a.nyq) * a.M2 : a.Mlast) * a.M1;
    const C *W = reinterpret_cast<const C *>(a.work);
    const int row0 = blk * RB;
    // Each field's RB rows are one contiguous run of the work buffer: one bulk
    // copy per field (TMA; 16-byte aligned, a multiple of 16 bytes) into shared
    // memory, completed on the mbarrier by transaction count.
    if (threadIdx.x == 0) {
        const uint32_t row_bytes = (uint32_t)(RB * n * sizeof(C));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(umma::smem_u32(bar)),
                     "r"(row_bytes * (uint32_t)nf)
                     : "memory");
        for (int f = 0; f < nf; ++f)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             umma::smem_u32(buf0 + (size_t)f * RB * n)),
                         "l"(W + f * fstride + (size_t)row0 * n), "r"(row_bytes), "r"(umma::smem_u32(bar))
                         : "memory");
    }
    load_twiddles<R>(tw, n);
    if (!umma::mbar_wait_n(umma::smem_u32(bar), parity, umma::WAIT_LIMIT)) {
        // the copies did not land: record it, give them a second bounded wait, go on
        if (a.err) atomicExch(a.err, 1);
        umma::mbar_wait_n(umma::smem_u32(bar), parity, umma::WAIT_LIMIT);
    }
    __syncthreads();
    stockham_inverse_grouped(buf0, buf1, n, lg1, RB * nf, RB, tw);
    const C *res = buf0;
    C *G = reinterpret_cast<C *>(a.grid);
    const int rowlen = a.P1 * nf;
    for (int r = 0; r < RB; ++r) {
        const int row = row0 + r;
        int l2, a3 = 0;
        if (a.dim == 3) {
            const int y = row / a.M2;
            l2 = row - y * a.M2;
            a3 = a.a3first + y;
        } else {
            l2 = row;
        }
        int p2[3], p3[3];
        int n2 = pad_dests((l2 + (a.M2 >> 1)) % a.M2, a.M2, p2);
        // field f of this row: res[(f RB + r) n + l1]
        const C *rr = res + (size_t)r * n;
        const size_t fs = (size_t)RB * n;
        if (a.dim == 3 && a.nyq && row / a.M2 == a.L3count) {
            // Nyquist row of the odd fields -> nyqgrid [p2][p1][2]
            C *NG = reinterpret_cast<C *>(a.nyqgrid);
            for (int d2 = 0; d2 < n2; ++d2) {
                C *dst = NG + (size_t)p2[d2] * a.P1 * 2;
                for (int i = threadIdx.x; i < 2 * a.P1; i += blockDim.x) {
                    const int p1 = i >> 1, f = 4 + (i & 1);
                    const int a1 = (p1 - 1 + n) % n;
                    dst[i] = rr[f * fs + (a1 + (n >> 1)) % n];
                }
            }
            continue;
        }
        int n3 = 1;
        p3[0] = 0;
        if (a.dim == 3) {
            if (a.zlinear)
                p3[0] = a3;  // far-region planes: node = plane, no halo
            else
                n3 = pad_dests(a3, a.M3, p3);
        }
        for (int d3 = 0; d3 < n3; ++d3) {
            // only the stored planes Q3lo .. Q3lo + P3 - 1
            const int q3 = p3[d3] - a.Q3lo;
            if (q3 < 0 || q3 >= a.P3) continue;
            for (int d2 = 0; d2 < n2; ++d2) {
                C *dst = G + ((size_t)q3 * a.P2 + p2[d2]) * rowlen;
                for (int i = threadIdx.x; i < rowlen; i += blockDim.x) {
                    int p1 = i / nf, f = i - p1 * nf;
                    int a1 = (p1 - 1 + n) % n;
                    int l1 = (a1 + (n >> 1)) % n;
                    dst[i] = rr[f * fs + l1];
                }
            }
        }
    }
}

template <typename R, bool DERIV>
__global__ void __launch_bounds__(256) synth_first_pass(SynthArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    synth_first_pass_body<R, DERIV>(a, blockIdx.x, smem);
}

template <typename R>
__global__ void __launch_bounds__(256) synth_x2_pass(SynthArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    synth_x2_body<R>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

// mbarrier of the last pass's bulk copies: one arrival (the issuing thread's
// expect_tx) per phase
__device__ __forceinline__ void init_copy_barrier(uint64_t *bar)
{
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
}

// Middle pass with tensor-map copies (single plans): the TJ columns b10 .. b10+TJ-1
// of the M2 rows of plane (f, y) are one 2D box of the work buffer seen as a
// [rows][M1] matrix of 8-byte units (a complex is U = sizeof(C)/8 units), loaded
// by cp.async.bulk.tensor in boxes of at most 256 rows into an interleaved tile
// [b2][t], transformed there, and written back the same way by a TMA store.
// The box's first unit x = b10 U is even (TJ >= 2), so x * 8 bytes is a multiple
// of 16 as the tensor copy requires.
constexpr int X2_BOX_ROWS = 256;

template <typename R>
__global__ void __launch_bounds__(256) synth_x2_pass_tma(SynthArgs a, const __grid_constant__ CUtensorMap tm)
{
    typedef typename cplx_t<R>::T C;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    const int n = a.M2, TJ = a.TJ2, lg2 = a.lg2;
    const int bx = blockIdx.x, y = blockIdx.y, f = blockIdx.z;
    if (y == a.L3count && f != 4 && f != 5) return;  // the Nyquist plane is only for xz, yz
    int lgTJ = 0;
    while ((1 << lgTJ) < TJ) ++lgTJ;
    C *tw = reinterpret_cast<C *>(smem);
    C *buf0 = reinterpret_cast<C *>(smem + ((sizeof(C) * (n >> 1) + 127) & ~(size_t)127));
    C *buf1 = buf0 + TJ * n;
    const int U = (int)(sizeof(C) / 8);
    const int x0 = bx * TJ * U, row0 = (f * (a.L3count + a.nyq) + y) * n;
    const int boxr = n < X2_BOX_ROWS ? n : X2_BOX_ROWS;
    const uint64_t tmap = reinterpret_cast<uint64_t>(&tm);
    init_copy_barrier(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(umma::smem_u32(&bar)),
                     "r"((uint32_t)(n * TJ * sizeof(C)))
                     : "memory");
        for (int r = 0; r < n; r += boxr)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                    umma::smem_u32(buf0 + (size_t)r * TJ)),
                "l"(tmap), "r"(x0), "r"(row0 + r), "r"(umma::smem_u32(&bar))
                : "memory");
    }
    load_twiddles<R>(tw, n);
    if (!umma::mbar_wait_n(umma::smem_u32(&bar), 0u, umma::WAIT_LIMIT)) {
        if (a.err) atomicExch(a.err, 1);
        umma::mbar_wait_n(umma::smem_u32(&bar), 0u, umma::WAIT_LIMIT);
    }
    __syncthreads();
    C *res = stockham_inverse_il(buf0, buf1, n, lg2, lgTJ, tw);
    // the transformed tile is read by the async proxy: order the generic writes first
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int r = 0; r < n; r += boxr)
            asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(tmap),
                         "r"(x0), "r"(row0 + r), "r"(umma::smem_u32(res + (size_t)r * TJ))
                         : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

template <typename R>
__global__ void __launch_bounds__(256) synth_x1_pass(SynthArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    init_copy_barrier(&bar);
    synth_x1_body<R>(a, blockIdx.x, smem, &bar, 0u);
}

// pair of virtual block vb: largest p with prefix[p] <= vb
__device__ __forceinline__ int batch_pair(const int *prefix, int np, int vb)
{
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= vb)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Batched synthesis passes: one persistent launch per pass walks the
// (pair, block) work list of all plans of a sweep; prefix[p] is the first
// virtual block of pair p (prefix[np] = total).
template <typename R>
__global__ void __launch_bounds__(256) synth_first_pass_batch(const SynthArgs *args, const int *prefix, int np)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ SynthArgs sa;
    const int total = prefix[np];
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const int p = batch_pair(prefix, np, vb);
        if (threadIdx.x == 0) sa = args[p];
        __syncthreads();
        synth_first_pass_body<R, false>(sa, vb - prefix[p], smem);
        __syncthreads();
    }
}

template <typename R>
__global__ void __launch_bounds__(256) synth_x2_pass_batch(const SynthArgs *args, const int *prefix, int np)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ SynthArgs sa;
    const int total = prefix[np];
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const int p = batch_pair(prefix, np, vb);
        if (threadIdx.x == 0) sa = args[p];
        __syncthreads();
        int loc = vb - prefix[p];
        const int nbx = sa.M1 / sa.TJ2;
        const int bx = loc % nbx;
        loc /= nbx;
        const int pl = sa.L3count + sa.nyq;
        const int y = loc % pl, f = loc / pl;
        synth_x2_body<R>(sa, bx, y, f, smem);
        __syncthreads();
    }
}

template <typename R>
__global__ void __launch_bounds__(256) synth_x1_pass_batch(const SynthArgs *args, const int *prefix, int np)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ SynthArgs sa;
    __shared__ __align__(8) uint64_t bar;
    init_copy_barrier(&bar);
    const int total = prefix[np];
    uint32_t phase = 0;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x, phase ^= 1u) {
        const int p = batch_pair(prefix, np, vb);
        if (threadIdx.x == 0) sa = args[p];
        __syncthreads();
        synth_x1_body<R>(sa, vb - prefix[p], smem, &bar, phase);
        __syncthreads();
    }
}

// gf_eval_grid: padded gather grid -> node order [f][l3][l2][l1]
template <typename R>
__global__ void extract_grid(SynthArgs a, void *out)
{
    typedef typename cplx_t<R>::T C;
    const C *G = reinterpret_cast<const C *>(a.grid);
    C *o = reinterpret_cast<C *>(out);
    const size_t per = (size_t)a.M1 * a.M2 * (a.dim == 3 ? a.M3 : 1);
    const size_t total = per * a.nf;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int f = (int)(i / per);
        size_t r = i - (size_t)f * per;
        int l1 = (int)(r % a.M1);
        size_t r2 = r / a.M1;
        int l2 = (int)(r2 % a.M2);
        int l3 = (int)(r2 / a.M2);
        int p1 = (l1 + (a.M1 >> 1)) % a.M1 + 1;
        int p2 = (l2 + (a.M2 >> 1)) % a.M2 + 1;
        int p3 = a.dim == 3 ? (l3 + (a.M3 >> 1)) % a.M3 + 1 - a.Q3lo : 0;
        o[i] = G[(((size_t)p3 * a.P2 + p2) * a.P1 + p1) * a.nf + f];
    }
}

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// Tile choices and shared-memory sizes of the three passes for one plan
// (tj_max caps the first pass's columns per CTA; the batch autotuner varies it).
template <typename R>
void synth_config_t(SynthArgs &a, int tj_max, size_t sm[3])
{
    typedef typename cplx_t<R>::T C;
    const int ncols = (a.dim == 3) ? a.M1 * a.M2 : a.M1;
    // per column: A_m (double2 and float), beta, |alpha|^2 (double), |alpha|^2 - k^2, its float;
    // float-column data (|alpha|^2 - k^2 as a float pair, g, flags); per b: twiddles, q_b^2
    // and its float pair, q_b in float; the quadrature weights and nodes in float; plus the
    // two line buffers
    auto bytes = [&](int TJ) {
        return sizeof(C) * (a.Mlast / 2) + sizeof(double) * a.Mlast + sizeof(float2) * a.Mlast +
               TJ * (sizeof(double2) * a.Q + sizeof(double2) + 2 * sizeof(double) + sizeof(float)) +
               TJ * (sizeof(float2) + sizeof(float) + sizeof(int)) +
               sizeof(float) * ((TJ * a.Q + 3) & ~3) + sizeof(C) * (a.nf + 1) * TJ * a.Mlast + 64 +
               sizeof(float) * (2 * a.Q + a.Mlast) + 16 +
               (a.deriv && a.k2 > 0.0 ? TJ * sizeof(double2) * (a.Q + 1) + 16 : 0);
    };
    int TJ = tj_max;
    while (TJ > 1 && (TJ > ncols || bytes(TJ) > 160 * 1024)) TJ >>= 1;
    a.TJ = TJ;
    sm[0] = bytes(TJ);
    int TJ2 = 8;
    while (TJ2 > 1 && (TJ2 > a.M1 || sizeof(C) * (a.M2 / 2 + 2 * TJ2 * a.M2) > 160 * 1024)) TJ2 >>= 1;
    a.TJ2 = TJ2;
    a.lg2 = ilog2(a.M2);
    a.lg1 = ilog2(a.M1);
    sm[1] = a.dim == 3 ? sizeof(C) * (a.M2 / 2 + 2 * TJ2 * a.M2) : 0;
    // last pass: RB1 rows per CTA (up to 2048 values, a power of two dividing the rows)
    const int nrows = a.dim == 3 ? (a.L3count + a.nyq) * a.M2 : a.M2;
    int RB1 = 8;
    while (RB1 > 1 && (RB1 > nrows || RB1 * a.nf * a.M1 > 2048 ||
                       sizeof(C) * (a.M1 / 2 + (a.nf + 1) * RB1 * a.M1) > 160 * 1024))
        RB1 >>= 1;
    a.RB1 = RB1;
    sm[2] = sizeof(C) * (a.M1 / 2 + (a.nf + 1) * RB1 * a.M1);
}

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point
// query, so the library needs no link to libcuda); null when unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Middle pass of a single plan: tensor-map copies when the tile allows them
// (TJ >= 2 columns, a map the driver accepts), the plain staged loop otherwise.
template <typename R>
cudaError_t launch_x2(const SynthArgs &a, size_t smem_plain, cudaStream_t s)
{
    typedef typename cplx_t<R>::T C;
    const dim3 grid(a.M1 / a.TJ2, a.L3count + a.nyq, a.nf);
    PFN_cuTensorMapEncodeTiled_v12000 enc = a.TJ2 >= 2 ? tensor_map_encoder() : nullptr;
    if (enc) {
        const int U = (int)(sizeof(C) / 8);
        const cuuint64_t dims[2] = {(cuuint64_t)a.M1 * U, (cuuint64_t)a.M2 * (a.L3count + a.nyq) * a.nf};
        const cuuint64_t strides[1] = {(cuuint64_t)a.M1 * sizeof(C)};
        const cuuint32_t box[2] = {(cuuint32_t)(a.TJ2 * U), (cuuint32_t)(a.M2 < X2_BOX_ROWS ? a.M2 : X2_BOX_ROWS)};
        const cuuint32_t estr[2] = {1, 1};
        CUtensorMap tm;
        if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, a.work, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
            const size_t sm = ((sizeof(C) * (a.M2 >> 1) + 127) & ~(size_t)127) + 2 * sizeof(C) * a.TJ2 * a.M2;
            cudaError_t e = cudaFuncSetAttribute(synth_x2_pass_tma<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            synth_x2_pass_tma<R><<<grid, 256, sm, s>>>(a, tm);
            gf_count_launch(1);
            return cudaGetLastError();
        }
    }
    cudaError_t e = cudaFuncSetAttribute(synth_x2_pass<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_plain);
    if (e != cudaSuccess) return e;
    synth_x2_pass<R><<<grid, 256, smem_plain, s>>>(a);
    gf_count_launch(1);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_synth_t(const SynthArgs &a0, cudaStream_t s)
{
    SynthArgs a = a0;
    size_t sm[3];
    synth_config_t<R>(a, sizeof(R) == 4 ? 16 : 8, sm);
    const int ncols = (a.dim == 3) ? a.M1 * a.M2 : a.M1;
    cudaError_t e;
    if (a.deriv) {
        e = cudaFuncSetAttribute(synth_first_pass<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[0]);
        if (e != cudaSuccess) return e;
        synth_first_pass<R, true><<<ncols / a.TJ, 256, sm[0], s>>>(a);
    } else {
        e = cudaFuncSetAttribute(synth_first_pass<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[0]);
        if (e != cudaSuccess) return e;
        synth_first_pass<R, false><<<ncols / a.TJ, 256, sm[0], s>>>(a);
    }
    gf_count_launch(1);
    if (a.dim == 3) {
        e = launch_x2<R>(a, sm[1], s);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(synth_x1_pass<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[2]);
    if (e != cudaSuccess) return e;
    int rows = (a.dim == 3) ? (a.L3count + a.nyq) * a.M2 : a.M2;
    synth_x1_pass<R><<<rows / a.RB1, 256, sm[2], s>>>(a);
    gf_count_launch(1);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_synth_batch_t(const SynthBatch &b, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(synth_first_pass_batch<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)b.smem[0])) != cudaSuccess ||
        (e = cudaFuncSetAttribute(synth_x2_pass_batch<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)b.smem[1])) != cudaSuccess ||
        (e = cudaFuncSetAttribute(synth_x1_pass_batch<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)b.smem[2])) != cudaSuccess)
        return e;
    // persistent grids of resident CTAs only: a CTA beyond the resident count
    // would start its share of the work list only after another CTA had finished
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    auto resident = [&](int per, int want) {
        if (per < 1) {
            cudaGetLastError();
            per = 1;
        }
        return want < per * nsm ? want : per * nsm;
    };
    int per[3] = {0, 0, 0};
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[0], synth_first_pass_batch<R>, 256, b.smem[0]);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[1], synth_x2_pass_batch<R>, 256, b.smem[1]);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[2], synth_x1_pass_batch<R>, 256, b.smem[2]);
    synth_first_pass_batch<R><<<resident(per[0], b.grid[0]), 256, b.smem[0], s>>>(b.args, b.prefix[0], b.np);
    synth_x2_pass_batch<R><<<resident(per[1], b.grid[1]), 256, b.smem[1], s>>>(b.args, b.prefix[1], b.np);
    synth_x1_pass_batch<R><<<resident(per[2], b.grid[2]), 256, b.smem[2], s>>>(b.args, b.prefix[2], b.np);
    gf_count_launch(3);
    return cudaGetLastError();
}

}  // namespace

cudaError_t gf_launch_synth(const SynthArgs &a, int precision, cudaStream_t s)
{
    return precision == GF_FP64 ? launch_synth_t<double>(a, s) : launch_synth_t<float>(a, s);
}

namespace {
// Piecewise Chebyshev interpolants of the radial transforms, one CTA per panel
// [p w, (p+1) w]: values at the nn <= 16 Chebyshev points (sixteen threads per
// point share the quadrature sum, reduced by shuffles), then the discrete
// cosine transform to coefficients.
//   3D: h(s) = sum_m B_m sin(s r_m)/s (complex).
//   2D: (S0, S1)(s) = (sum_m P0_m J0(s r_m), sum_m P1_m J1(s r_m)) (two real functions).
template <int DIM>
__global__ void __launch_bounds__(256) cheb_table_kernel(const double *rr, const double2 *B, const double *P0,
                                                         const double *P1, int Q, int nn, double w, double2 *out,
                                                         float2 *outf)
{
    __shared__ double2 fv[16];
    const int p = blockIdx.x, t = threadIdx.x, k = t >> 4, g = t & 15;
    const double cen = (p + 0.5) * w, hh = 0.5 * w;
    double ar = 0.0, ai = 0.0, s = 0.0;
    if (k < nn) {
        s = cen + hh * cospi((k + 0.5) / nn);
        for (int m = g; m < Q; m += 16) {
            const double z = s * rr[m];
            if (DIM == 3) {
                const double ker = (s == 0.0) ? rr[m] : sin(z);
                ar = fma(B[m].x, ker, ar);
                ai = fma(B[m].y, ker, ai);
            } else {
                ar = fma(P0[m], j0(z), ar);
                ai = fma(P1[m], j1(z), ai);
            }
        }
    }
    for (int o = 8; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (k < nn && g == 0) {
        if (DIM == 3 && s != 0.0) {
            ar /= s;
            ai /= s;
        }
        fv[k] = make_double2(ar, ai);
    }
    __syncthreads();
    if (t < nn) {
        double cr = 0.0, ci = 0.0;
        for (int q = 0; q < nn; ++q) {
            const double c = cospi((double)t * (q + 0.5) / nn);
            cr = fma(fv[q].x, c, cr);
            ci = fma(fv[q].y, c, ci);
        }
        const double sc = (t == 0 ? 1.0 : 2.0) / nn;
        out[(size_t)p * nn + t] = make_double2(cr * sc, ci * sc);
        if (outf) outf[(size_t)p * nn + t] = make_float2((float)(cr * sc), (float)(ci * sc));
    }
}
// The 2D derivative plans' Hankel transforms of the cutoff Y on the same panels:
// at each Chebyshev point s, sums over the nodes r_m of [0, eps] and [eps, 2 eps]
// with weights wy_m = w_m Y(r_m):
//   table 0: (Q1, R0) = (sum wy J1(s r), sum wy J0(s r) r)
//   table 1: (R2, S1) = (sum wy J2(s r) r, sum wy J1(s r) r^2)
//   table 2: (S3, 0)  = (sum wy J3(s r) r^2, 0)
// out: [3][npan][nn].
__global__ void __launch_bounds__(256) cheb_deriv_kernel(const double *rr, const double *wy, int Q2, int nn, double w,
                                                         int npan, double2 *out)
{
    __shared__ double fv[16][5];
    const int p = blockIdx.x, t = threadIdx.x, k = t >> 4, g = t & 15;
    const double cen = (p + 0.5) * w, hh = 0.5 * w;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (k < nn) {
        const double s = cen + hh * cospi((k + 0.5) / nn);
        for (int m = g; m < Q2; m += 16) {
            const double r = rr[m], z = s * r, wm = wy[m];
            const double J0 = j0(z), J1 = j1(z), J2 = jn(2, z), J3 = jn(3, z);
            acc[0] = fma(wm, J1, acc[0]);
            acc[1] = fma(wm * r, J0, acc[1]);
            acc[2] = fma(wm * r, J2, acc[2]);
            acc[3] = fma(wm * r * r, J1, acc[3]);
            acc[4] = fma(wm * r * r, J3, acc[4]);
        }
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
        for (int o = 8; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    if (k < nn && g == 0)
#pragma unroll
        for (int i = 0; i < 5; ++i) fv[k][i] = acc[i];
    __syncthreads();
    if (t < nn) {
        double c[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int q = 0; q < nn; ++q) {
            const double cq = cospi((double)t * (q + 0.5) / nn);
#pragma unroll
            for (int i = 0; i < 5; ++i) c[i] = fma(fv[q][i], cq, c[i]);
        }
        const double sc = (t == 0 ? 1.0 : 2.0) / nn;
        const size_t tab = (size_t)npan * nn, o = (size_t)p * nn + t;
        out[o] = make_double2(c[0] * sc, c[1] * sc);
        out[tab + o] = make_double2(c[2] * sc, c[3] * sc);
        out[2 * tab + o] = make_double2(c[4] * sc, 0.0);
    }
}
}  // namespace

cudaError_t gf_launch_cheb_deriv(const double *rr, const double *wy, int Q2, int npan, int deg, double w, double2 *out,
                                 cudaStream_t s)
{
    cheb_deriv_kernel<<<npan, 256, 0, s>>>(rr, wy, Q2, deg + 1, w, npan, out);
    gf_count_launch(1);
    return cudaGetLastError();
}

// E[b][m] = e^{i q_b t_m}, q_b = j qs (qs = pi / c~) with j = b for b < Mlast/2, else
// b - Mlast (the last-axis frequencies of Eq. (fck-coef)), t_m the Gauss nodes
// of the X' integrals.
__global__ void e_table_kernel(const double *tt, int Q, int Mlast, double qs, double2 *E, float2 *Ef)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Mlast * Q; i += gridDim.x * blockDim.x) {
        const int b = i / Q, m = i - b * Q;
        const int jl = b < Mlast / 2 ? b : b - Mlast;
        const double q = (double)jl * qs;
        double sv, cv;
        sincos(q * tt[m], &sv, &cv);
        E[i] = make_double2(cv, sv);
        if (Ef) Ef[i] = make_float2((float)cv, (float)sv);
    }
}

namespace {
// Far-region grid coefficients (the far branch's series (he) on planes): for
// in-plane index n (FFT order b) and plane m at z = z0 + m hz,
//   a_n(z) = (i/8pi^2) e^{i beta_n z}/beta_n
// = e^{-b z}/(8pi^2 b) for evanescent beta_n = i b, and (-sin + i cos)(beta z)/(8pi^2 beta)
// for propagating ones; Maxwell fields (delta_pq - c^p c^q/k^2) a_n with
// c = (alpha_n, beta_n), then a_n.  Work layout [f][m][b2][b1], working precision.
// One thread per in-plane index walks the planes: |alpha_n|^2 - k^2 is formed once
// in double; split plans take b and the exponentials in float (a relative error
// of about 1e-7 per coefficient) except within 0.05 k of a Wood anomaly, where b
// comes from the double difference as in the near grid's coefficients.
template <typename R>
__global__ void __launch_bounds__(256) fargrid_coef(SynthArgs a, double k, double a1, double a2, double z0, double hz)
{
    typedef typename cplx_t<R>::T C;
    C *W = reinterpret_cast<C *>(a.work);
    const int plane = a.M1 * a.M2;
    const size_t per = (size_t)plane * a.L3count;
    const double k2 = k * k, ik2 = 1.0 / k2, s8 = 1.0 / (8.0 * GF_PI * GF_PI);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += gridDim.x * blockDim.x) {
        const int b1 = i % a.M1, b2 = i / a.M1;
        const double c1 = a1 + freq_of(b1, a.M1), c2 = a2 + freq_of(b2, a.M2);
        const double d = fma(c1, c1, fma(c2, c2, -k2));  // |alpha_n|^2 - k^2
        const bool ev = d > 0.0;
        // b = |beta_n|: float where it is not small against k (split plans)
        const bool fast = sizeof(R) == 4 && d > 0.0025 * k2;
        double bd = 0.0;
        float bf = 0.f;
        if (fast)
            bf = sqrtf((float)d);
        else
            bd = sqrt(fabs(d));
        const double bb = fast ? (double)bf : bd;
        if (fast && a.nf == 1) {
            // split plans, evanescent and clear of Wood anomalies: all in float (z to
            // an ulp, e^{-b z} to a few ulps where it is not negligible)
            const float zf0 = (float)z0, hzf = (float)hz, blog = -bf * 1.44269504f, w = (float)s8 / bf;
            C *Wc = W + i;
            for (int m = 0; m < a.L3count; ++m) Wc[(size_t)m * plane] = cmk((R)(exp2f(blog * fmaf((float)m, hzf, zf0)) * w), (R)0);
            continue;
        }
        for (int m = 0; m < a.L3count; ++m) {
            const double z = z0 + m * hz;
            double2 an;
            if (ev) {
                if (fast)
                    an = make_double2((double)(exp2f(-bf * (float)z * 1.44269504f) * ((float)s8 / bf)), 0.0);
                else
                    an = make_double2(exp(-bd * z) * s8 / bd, 0.0);
            } else {
                double sz, cz;
                sincos(bd * z, &sz, &cz);
                an = make_double2(-sz * s8 / bd, cz * s8 / bd);
            }
            const size_t o = (size_t)m * plane + i;
            if (a.nf == 1) {
                W[o] = cmk((R)an.x, (R)an.y);
            } else {
                // c = (c1, c2, beta): beta = i b (evanescent) or b (propagating)
                const double2 beta = ev ? make_double2(0.0, bb) : make_double2(bb, 0.0);
                const double2 cv[3] = {make_double2(c1, 0.0), make_double2(c2, 0.0), beta};
                const int P[6] = {0, 1, 2, 0, 0, 1}, Q[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
                for (int e = 0; e < 6; ++e) {
                    const double2 cc = cmul(cv[P[e]], cv[Q[e]]);
                    const double2 f = make_double2((P[e] == Q[e] ? 1.0 : 0.0) - cc.x * ik2, -cc.y * ik2);
                    const double2 v = cmul(f, an);
                    W[(size_t)e * per + o] = cmk((R)v.x, (R)v.y);
                }
                W[(size_t)6 * per + o] = cmk((R)an.x, (R)an.y);
            }
        }
    }
}

template <typename R>
cudaError_t launch_far_grid_t(const SynthArgs &a0, double k, double a1, double a2, double z0, double hz, cudaStream_t s)
{
    SynthArgs a = a0;
    size_t sm[3];
    synth_config_t<R>(a, 8, sm);
    const int plane = a.M1 * a.M2;
    int blocks = (plane + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    fargrid_coef<R><<<blocks, 256, 0, s>>>(a, k, a1, a2, z0, hz);
    cudaError_t e = launch_x2<R>(a, sm[1], s);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(synth_x1_pass<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[2]);
    if (e != cudaSuccess) return e;
    synth_x1_pass<R><<<a.L3count * a.M2 / a.RB1, 256, sm[2], s>>>(a);
    gf_count_launch(2);
    return cudaGetLastError();
}
}  // namespace

cudaError_t gf_launch_far_grid(const SynthArgs &a, int precision, double k, double a1, double a2, double z0,
                               double hz, cudaStream_t s)
{
    return precision == GF_FP64 ? launch_far_grid_t<double>(a, k, a1, a2, z0, hz, s)
                                : launch_far_grid_t<float>(a, k, a1, a2, z0, hz, s);
}

cudaError_t gf_launch_e_table(const double *tt, int Q, int Mlast, double qs, double2 *E, float2 *Ef, cudaStream_t s)
{
    int blocks = (Mlast * Q + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    e_table_kernel<<<blocks, 256, 0, s>>>(tt, Q, Mlast, qs, E, Ef);
    gf_count_launch(1);
    return cudaGetLastError();
}

cudaError_t gf_launch_cheb_table(int dim, const double *rr, const double2 *B, const double *P0, const double *P1, int Q,
                                 int npan, int deg, double w, double2 *out, float2 *outf, cudaStream_t s)
{
    if (deg + 1 > 16 || npan < 1) return cudaErrorInvalidValue;
    if (dim == 3)
        cheb_table_kernel<3><<<npan, 256, 0, s>>>(rr, B, P0, P1, Q, deg + 1, w, out, outf);
    else
        cheb_table_kernel<2><<<npan, 256, 0, s>>>(rr, B, P0, P1, Q, deg + 1, w, out, outf);
    gf_count_launch(1);
    return cudaGetLastError();
}

// Largest dynamic shared memory the plan's own synthesis launches ask for.
size_t gf_synth_smem_need(const SynthArgs &a0, int precision)
{
    SynthArgs a = a0;
    size_t sm[3];
    if (precision == GF_FP64)
        synth_config_t<double>(a, 8, sm);
    else
        synth_config_t<float>(a, 16, sm);
    size_t m = sm[0];
    if (a.dim == 3 && sm[1] > m) m = sm[1];
    return sm[2] > m ? sm[2] : m;
}

void gf_synth_config(SynthArgs &a, int precision, int tj_max, size_t smem[3])
{
    if (precision == GF_FP64)
        synth_config_t<double>(a, tj_max, smem);
    else
        synth_config_t<float>(a, tj_max, smem);
}

cudaError_t gf_launch_synth_batch(const SynthBatch &b, int precision, cudaStream_t s)
{
    return precision == GF_FP64 ? launch_synth_batch_t<double>(b, s) : launch_synth_batch_t<float>(b, s);
}

cudaError_t gf_launch_extract(const SynthArgs &a, int precision, void *dev_out, cudaStream_t s)
{
    if (precision == GF_FP64)
        extract_grid<double><<<1024, 256, 0, s>>>(a, dev_out);
    else
        extract_grid<float><<<1024, 256, 0, s>>>(a, dev_out);
    gf_count_launch(1);
    return cudaGetLastError();
}
