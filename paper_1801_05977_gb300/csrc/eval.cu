// Evaluation at targets (Algorithms 1-3, step 2 "Calculation").
//
//  near kernel  (|x_last| <= c): reduce to the unit cell (step 2c), gather the
//               4^d stencil of the padded grid with separable cubic Lagrange
//               weights (step 2d), add the singular part back in double
//               precision (step 2e), apply the quasi-periodic phase (step 2f);
//               far targets are appended to a scratch list instead.
//  far kernel   (|x_last| > c, step 2b): the eigen-series (ei)/(he) (and its
//               second derivatives for the Maxwell tensor), truncated to
//               |alpha_n|^2 <= k^2 + (T/|x_last|)^2, one thread per target,
//               the 32 lanes of a warp walking the same index set so that the
//               per-index table of beta_n is read by broadcast.
#include <math_constants.h>

#include "gf_internal.cuh"

namespace {

constexpr double TWO_PI = 2.0 * GF_PI;

// x = 2 pi m + t, t in [-pi, pi), with explicit round-to-nearest operations
// (no contraction) so that the cell decision is reproducible.
__device__ __forceinline__ void reduce_period(double x, double &t, double &m)
{
    double mm = floor(__ddiv_rn(__dadd_rn(x, GF_PI), TWO_PI));
    double tt = __dsub_rn(x, __dmul_rn(TWO_PI, mm));
    if (tt >= GF_PI) {
        tt = __dsub_rn(tt, TWO_PI);
        mm += 1.0;
    }
    if (tt < -GF_PI) {
        tt = __dadd_rn(tt, TWO_PI);
        mm -= 1.0;
    }
    t = tt;
    m = mm;
}

// stencil origin on an axis: u = (y - y0)/h, i0 = floor(u) clamped to [0, M-1],
// f = u - i0; the padded nodes i0 .. i0+3 hold the stencil nodes i0-1 .. i0+2.
__device__ __forceinline__ int stencil_origin(double y, double y0, double h, int M, double &f)
{
    double u = __ddiv_rn(__dsub_rn(y, y0), h);
    double i0 = floor(u);
    if (i0 > (double)(M - 1)) i0 = (double)(M - 1);
    if (i0 < 0.0) i0 = 0.0;
    f = u - i0;
    return (int)i0;
}

__device__ __forceinline__ void lagrange4(double f, double w[4])
{
    double fm1 = f - 1.0, fm2 = f - 2.0, fp1 = f + 1.0;
    w[0] = -f * fm1 * fm2 * (1.0 / 6.0);
    w[1] = fp1 * fm1 * fm2 * 0.5;
    w[2] = -fp1 * f * fm2 * 0.5;
    w[3] = fp1 * f * fm1 * (1.0 / 6.0);
}

// quasi-periodic lift e^{i 2 pi <alpha . m>} (fractional part taken first)
__device__ __forceinline__ double2 lattice_phase(double a1, double m1, double a2, double m2)
{
    double ph = a1 * m1 + a2 * m2;
    ph -= rint(ph);
    double s, c;
    sincospi(2.0 * ph, &s, &c);
    return make_double2(c, s);
}

__device__ __forceinline__ void store_out(double2 *o, double2 v) { *o = v; }
__device__ __forceinline__ void store_out(float2 *o, double2 v) { *o = make_float2((float)v.x, (float)v.y); }

template <typename R> __device__ __forceinline__ typename cplx_t<R>::T nan_c();
template <> __device__ __forceinline__ double2 nan_c<double>() { return make_double2(CUDART_NAN, CUDART_NAN); }
template <> __device__ __forceinline__ float2 nan_c<float>() { return make_float2(CUDART_NAN_F, CUDART_NAN_F); }

__device__ __forceinline__ double2 ld_grid(const double2 *p) { return __ldg(p); }
__device__ __forceinline__ double2 ld_grid(const float2 *p)
{
    float2 v = __ldg(p);
    return make_double2(v.x, v.y);
}

// entries written per target
__host__ __device__ __forceinline__ int n_entries(int which) { return which == GF_OUT_MAXWELL6 ? 6 : which == GF_OUT_MAXWELL7 ? 7 : 1; }

// Warp-aggregated append of far targets to the scratch list.
__device__ __forceinline__ void push_far(bool isfar, int i, int *list, int *count)
{
    unsigned mask = __ballot_sync(0xffffffffu, isfar);
    if (mask == 0u) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (isfar) list[base + __popc(mask & ((1u << lane) - 1u))] = i;
}

// ---------------------------------------------------------------------------
// 3D near kernel.  NF = 1: Helmholtz (field L_d).  NF = 7: Maxwell
// (fields 0..5 = (delta_pq - c^p c^q/k^2) L_d, field 6 = L_d).
// R = storage/accumulation type of the grid (double: GF_FP64, float: split).
// ---------------------------------------------------------------------------
template <typename R, int NF>
__global__ void __launch_bounds__(256) near3d(EvalArgs a)
{
    typedef typename cplx_t<R>::T C;
    const C *G = reinterpret_cast<const C *>(a.grid);
    C *out = reinterpret_cast<C *>(a.out);
    const int ne = n_entries(a.which);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool valid = i < a.n;
        double x1 = 0, x2 = 0, x3 = 0;
        if (valid) {
            x1 = a.x[3 * i];
            x2 = a.x[3 * i + 1];
            x3 = a.x[3 * i + 2];
        }
        bool finite = isfinite(x1) && isfinite(x2) && isfinite(x3);
        bool isfar = valid && finite && fabs(x3) > a.c;
        push_far(isfar, (int)i, a.far_idx, a.far_count);
        if (!valid || isfar) continue;
        C *o = out + i * ne;
        if (!finite) {
            for (int e = 0; e < ne; ++e) o[e] = nan_c<R>();
            continue;
        }
        double t1, m1, t2, m2;
        reduce_period(x1, t1, m1);
        reduce_period(x2, t2, m2);
        double f1, f2, f3;
        int i1 = stencil_origin(t1, -GF_PI, a.h1, a.M1, f1);
        int i2 = stencil_origin(t2, -GF_PI, a.h2, a.M2, f2);
        int i3 = stencil_origin(x3, -a.ct, a.h3, a.M3, f3);
        double w1d[4], w2d[4], w3d[4];
        lagrange4(f1, w1d);
        lagrange4(f2, w2d);
        lagrange4(f3, w3d);
        R w1[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) w1[d] = (R)w1d[d];
        R acc[NF][2];
#pragma unroll
        for (int e = 0; e < NF; ++e) acc[e][0] = acc[e][1] = (R)0;
#pragma unroll
        for (int d3 = 0; d3 < 4; ++d3) {
#pragma unroll
            for (int d2 = 0; d2 < 4; ++d2) {
                const C *row = G + (((size_t)(i3 + d3) * a.P2 + (i2 + d2)) * a.P1 + i1) * NF;
                R w23 = (R)(w3d[d3] * w2d[d2]);
#pragma unroll
                for (int e = 0; e < NF; ++e) {
                    R sr = 0, si = 0;
#pragma unroll
                    for (int d1 = 0; d1 < 4; ++d1) {
                        C g = __ldg(row + d1 * NF + e);
                        sr = fma(w1[d1], g.x, sr);
                        si = fma(w1[d1], g.y, si);
                    }
                    acc[e][0] = fma(w23, sr, acc[e][0]);
                    acc[e][1] = fma(w23, si, acc[e][1]);
                }
            }
        }
        // lift = e^{i alpha.t} e^{i 2 pi <alpha.m>}; G = lift L + e^{i 2pi<alpha.m>} Phi Y (K = L + F, F = e^{-i alpha.t} Phi Y)
        double2 lat = lattice_phase(a.a1, m1, a.a2, m2);
        double sa, ca;
        sincos(a.a1 * t1 + a.a2 * t2, &sa, &ca);
        double2 lift = cmul(make_double2(ca, sa), lat);
        double r = sqrt(t1 * t1 + t2 * t2 + x3 * x3);
        bool sing = r < 2.0 * a.eps;
        double2 PhiY = make_double2(0, 0), dPhi = make_double2(0, 0), d2Phi = make_double2(0, 0);
        if (sing) {
            // Phi(r) = e^{ikr}/(4 pi r) Y_eps(r) and its r-derivatives (Sec. 3.2, Sec. 4)
            double sk, ck;
            sincos(a.k * r, &sk, &ck);
            double ir = 1.0 / r;
            double2 g0 = make_double2(ck * ir * (0.25 / GF_PI), sk * ir * (0.25 / GF_PI));
            double s = (r - a.eps) / a.eps;
            double Y0 = 1.0 - smooth8(s);
            PhiY = cscale(g0, Y0);
            if (NF > 1) {
                double Y1 = -smooth8_d1(s) / a.eps;
                double Y2 = -smooth8_d2(s) / (a.eps * a.eps);
                double2 L1 = make_double2(-ir, a.k);                  // ik - 1/r
                double2 g1 = cmul(g0, L1);
                double2 L2 = cmul(L1, L1);
                L2.x += ir * ir;
                double2 g2 = cmul(g0, L2);
                dPhi = cadd(cscale(g1, Y0), cscale(g0, Y1));
                d2Phi = cadd(cadd(cscale(g2, Y0), cscale(g1, 2.0 * Y1)), cscale(g0, Y2));
            }
        }
        if (NF == 1) {
            double2 L = make_double2((double)acc[0][0], (double)acc[0][1]);
            double2 v = cadd(cmul(lift, L), cmul(lat, PhiY));
            store_out(o, v);
        } else {
            const double ik2 = 1.0 / (a.k * a.k);
            const double xv[3] = {t1, t2, x3};
            const int PP[6] = {0, 1, 2, 0, 0, 1}, QQ[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                double2 L = make_double2((double)acc[e][0], (double)acc[e][1]);
                double2 v = cmul(lift, L);
                if (sing) {
                    double ir = 1.0 / r;
                    double xp = xv[PP[e]] * ir, xq = xv[QQ[e]] * ir;
                    double dl = PP[e] == QQ[e] ? 1.0 : 0.0;
                    // delta_pq Phi + k^-2 [Phi'' xp xq + (Phi'/r)(delta_pq - xp xq)]
                    double2 s = cadd(cscale(d2Phi, xp * xq), cscale(dPhi, ir * (dl - xp * xq)));
                    s = cscale(s, ik2);
                    if (dl != 0.0) s = cadd(s, PhiY);
                    v = cadd(v, cmul(lat, s));
                }
                store_out(o + e, v);
            }
            if (a.which == GF_OUT_MAXWELL7) {
                double2 L = make_double2((double)acc[6][0], (double)acc[6][1]);
                store_out(o + 6, cadd(cmul(lift, L), cmul(lat, PhiY)));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 2D near kernel (Algorithm 1): K = L + f1 - i alpha f2, G = e^{i alpha x1} K,
// f1 = -(1/2pi) ln r Y_eps(r), f2 = t f1 at the reduced point (t, x2).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) near2d(EvalArgs a)
{
    typedef typename cplx_t<R>::T C;
    const C *G = reinterpret_cast<const C *>(a.grid);
    C *out = reinterpret_cast<C *>(a.out);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool valid = i < a.n;
        double x1 = 0, x2 = 0;
        if (valid) {
            x1 = a.x[2 * i];
            x2 = a.x[2 * i + 1];
        }
        bool finite = isfinite(x1) && isfinite(x2);
        bool isfar = valid && finite && fabs(x2) > a.c;
        push_far(isfar, (int)i, a.far_idx, a.far_count);
        if (!valid || isfar) continue;
        if (!finite) {
            out[i] = nan_c<R>();
            continue;
        }
        double t, m;
        reduce_period(x1, t, m);
        double f1, f2;
        int i1 = stencil_origin(t, -GF_PI, a.h1, a.M1, f1);
        int i2 = stencil_origin(x2, -a.ct, a.h2, a.M2, f2);
        double w1[4], w2[4];
        lagrange4(f1, w1);
        lagrange4(f2, w2);
        double Lr = 0, Li = 0;
#pragma unroll
        for (int d2 = 0; d2 < 4; ++d2) {
            const C *row = G + (size_t)(i2 + d2) * a.P1 + i1;
            double sr = 0, si = 0;
#pragma unroll
            for (int d1 = 0; d1 < 4; ++d1) {
                double2 g = ld_grid(row + d1);
                sr = fma(w1[d1], g.x, sr);
                si = fma(w1[d1], g.y, si);
            }
            Lr = fma(w2[d2], sr, Lr);
            Li = fma(w2[d2], si, Li);
        }
        double2 K = make_double2(Lr, Li);
        double r = sqrt(t * t + x2 * x2);
        if (r < 2.0 * a.eps) {
            double Y = 1.0 - smooth8((r - a.eps) / a.eps);
            double fa = -log(r) * Y * (0.5 / GF_PI);
            double fb = t * fa;
            K.x += fa;                 // + f1
            K.y -= a.a1 * fb;          // - i alpha f2
        }
        double2 lat = lattice_phase(a.a1, m, 0.0, 0.0);
        double sa, ca;
        sincos(a.a1 * t, &sa, &ca);
        store_out(out + i, cmul(cmul(make_double2(ca, sa), lat), K));
    }
}

// ---------------------------------------------------------------------------
// Far-series table: beta_n and 1/beta_n on the index box (plan time, double).
// ---------------------------------------------------------------------------
template <typename E>
__global__ void beta_table(EvalArgs a, E *tab)
{
    const int W2 = a.n2hi - a.n2lo + 1;
    const int tot = (a.n1hi - a.n1lo + 1) * W2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
        int n1 = a.n1lo + i / W2, n2 = a.n2lo + i % W2;
        double c1 = a.a1 + n1, c2 = a.a2 + n2;
        double A2 = c1 * c1 + c2 * c2;
        double aa = sqrt(A2);
        double br = 0, bi = 0;
        if (aa <= a.k)
            br = sqrt((a.k - aa) * (a.k + aa));
        else
            bi = sqrt((aa - a.k) * (aa + a.k));
        // 1/beta: real beta -> 1/br; imaginary beta = i bi -> -i/bi
        double ibr = br != 0.0 ? 1.0 / br : 0.0;
        double ibi = bi != 0.0 ? -1.0 / bi : 0.0;
        E e;
        e.br = br;
        e.bi = bi;
        e.ibr = ibr;
        e.ibi = ibi;
        tab[i] = e;
    }
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// 3D far kernel, double precision (GF_FP64 plans).
// G_d = e^{i2pi<alpha.m>} (i/8pi^2) sum_n beta_n^{-1} e^{i alpha_n.t + i beta_n |x3|};
// Maxwell entries multiply each term by (delta_pq - c^p c^q / k^2),
// c = (alpha1+n1, alpha2+n2, beta_n sgn x3).
// ---------------------------------------------------------------------------
template <int NF>
__global__ void __launch_bounds__(128) far3d_f64(EvalArgs a)
{
    const BetaEntry *tab = reinterpret_cast<const BetaEntry *>(a.btab);
    double2 *out = reinterpret_cast<double2 *>(a.out);
    const int ne = n_entries(a.which);
    const int W2 = a.n2hi - a.n2lo + 1;
    const int count = *a.far_count;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const double k2 = a.k * a.k, ik2 = 1.0 / k2;
    for (int w = gw; w * 32 < count; w += nw) {
        int slot = w * 32 + lane;
        bool valid = slot < count;
        int idx = valid ? a.far_idx[slot] : 0;
        double x1 = 0, x2 = 0, x3 = 1;
        if (valid) {
            x1 = a.x[3 * (size_t)idx];
            x2 = a.x[3 * (size_t)idx + 1];
            x3 = a.x[3 * (size_t)idx + 2];
        }
        double t1, m1, t2, m2;
        reduce_period(x1, t1, m1);
        reduce_period(x2, t2, m2);
        double z = fabs(x3), sg = x3 >= 0.0 ? 1.0 : -1.0;
        double Tz = a.T / z;
        double R2 = valid ? k2 + Tz * Tz : 0.0;
        double R2m = warp_max(R2);
        double Rm = sqrt(R2m);
        int n1a = max(a.n1lo, (int)floor(-a.a1 - Rm) - 1), n1b = min(a.n1hi, (int)ceil(-a.a1 + Rm) + 1);
        double s2, c2;
        sincos(t2, &s2, &c2);
        const double2 step = make_double2(c2, s2);
        double acc[NF][2];
#pragma unroll
        for (int e = 0; e < NF; ++e) acc[e][0] = acc[e][1] = 0.0;
        for (int n1 = n1a; n1 <= n1b; ++n1) {
            double c1 = a.a1 + n1;
            double rem = R2m - c1 * c1;
            if (rem < 0.0) continue;
            double sr = sqrt(rem);
            int n2a = max(a.n2lo, (int)floor(-a.a2 - sr)), n2b = min(a.n2hi, (int)ceil(-a.a2 + sr));
            double sp, cp;
            sincos(c1 * t1 + (a.a2 + n2a) * t2, &sp, &cp);
            double2 p = make_double2(cp, sp);
            const BetaEntry *row = tab + (size_t)(n1 - a.n1lo) * W2 - a.n2lo;
            for (int n2 = n2a; n2 <= n2b; ++n2) {
                double c2v = a.a2 + n2;
                double A2 = c1 * c1 + c2v * c2v;
                BetaEntry be = row[n2];
                if (valid && A2 <= R2) {
                    double2 ez;
                    if (be.bi == 0.0) {
                        double sz, cz;
                        sincos(be.br * z, &sz, &cz);
                        ez = make_double2(cz, sz);
                    } else {
                        ez = make_double2(exp(-be.bi * z), 0.0);
                    }
                    double2 term = cmul(cmul(make_double2(be.ibr, be.ibi), ez), p);
                    if (NF == 1) {
                        acc[0][0] += term.x;
                        acc[0][1] += term.y;
                    } else {
                        // c3 = beta sgn: c3^2 = beta^2, c1 c3 = c1 beta sgn, ...
                        double2 b = make_double2(be.br * sg, be.bi * sg);
                        double2 b2 = make_double2(be.br * be.br - be.bi * be.bi, 2.0 * be.br * be.bi);
                        double2 f[6] = {make_double2(1.0 - c1 * c1 * ik2, 0.0), make_double2(1.0 - c2v * c2v * ik2, 0.0),
                                        make_double2(1.0 - b2.x * ik2, -b2.y * ik2), make_double2(-c1 * c2v * ik2, 0.0),
                                        make_double2(-c1 * b.x * ik2, -c1 * b.y * ik2),
                                        make_double2(-c2v * b.x * ik2, -c2v * b.y * ik2)};
#pragma unroll
                        for (int e = 0; e < 6; ++e) {
                            double2 tf = cmul(f[e], term);
                            acc[e][0] += tf.x;
                            acc[e][1] += tf.y;
                        }
                        acc[6][0] += term.x;
                        acc[6][1] += term.y;
                    }
                }
                p = cmul(p, step);
            }
        }
        if (!valid) continue;
        double2 lat = lattice_phase(a.a1, m1, a.a2, m2);
        double2 pre = cmul(lat, make_double2(0.0, 1.0 / (8.0 * GF_PI * GF_PI)));
        double2 *o = out + (size_t)idx * ne;
        if (NF == 1) {
            o[0] = cmul(pre, make_double2(acc[0][0], acc[0][1]));
        } else {
            for (int e = 0; e < 6; ++e) o[e] = cmul(pre, make_double2(acc[e][0], acc[e][1]));
            if (a.which == GF_OUT_MAXWELL7) o[6] = cmul(pre, make_double2(acc[6][0], acc[6][1]));
        }
    }
}

// ---------------------------------------------------------------------------
// 3D far kernel, split precision: per-target quantities (reduction, lattice
// phase, row phases) in double, the series terms and sums in float.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 row_phase_f32(double arg)
{
    // reduce in double, evaluate in float
    double r = arg - TWO_PI * rint(arg * (1.0 / TWO_PI));
    float s, c;
    __sincosf((float)r, &s, &c);
    return make_float2(c, s);
}

template <int NF>
__global__ void __launch_bounds__(128) far3d_f32(EvalArgs a)
{
    const BetaEntryF *tab = reinterpret_cast<const BetaEntryF *>(a.btab);
    float2 *out = reinterpret_cast<float2 *>(a.out);
    const int ne = n_entries(a.which);
    const int W2 = a.n2hi - a.n2lo + 1;
    const int count = *a.far_count;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const double k2 = a.k * a.k;
    const float ik2 = (float)(1.0 / k2);
    for (int w = gw; w * 32 < count; w += nw) {
        int slot = w * 32 + lane;
        bool valid = slot < count;
        int idx = valid ? a.far_idx[slot] : 0;
        double x1 = 0, x2 = 0, x3 = 1;
        if (valid) {
            x1 = a.x[3 * (size_t)idx];
            x2 = a.x[3 * (size_t)idx + 1];
            x3 = a.x[3 * (size_t)idx + 2];
        }
        double t1, m1, t2, m2;
        reduce_period(x1, t1, m1);
        reduce_period(x2, t2, m2);
        double zd = fabs(x3);
        float z = (float)zd, sg = x3 >= 0.0 ? 1.f : -1.f;
        double Tz = a.T / zd;
        double R2 = valid ? k2 + Tz * Tz : 0.0;
        double R2m = warp_max(R2);
        double Rm = sqrt(R2m);
        float R2f = (float)R2;
        int n1a = max(a.n1lo, (int)floor(-a.a1 - Rm) - 1), n1b = min(a.n1hi, (int)ceil(-a.a1 + Rm) + 1);
        float s2, c2;
        __sincosf((float)t2, &s2, &c2);
        const float2 step = make_float2(c2, s2);
        float acc[NF][2];
#pragma unroll
        for (int e = 0; e < NF; ++e) acc[e][0] = acc[e][1] = 0.f;
        for (int n1 = n1a; n1 <= n1b; ++n1) {
            double c1d = a.a1 + n1;
            double rem = R2m - c1d * c1d;
            if (rem < 0.0) continue;
            double sr = sqrt(rem);
            int n2a = max(a.n2lo, (int)floor(-a.a2 - sr)), n2b = min(a.n2hi, (int)ceil(-a.a2 + sr));
            float2 p = row_phase_f32(c1d * t1 + (a.a2 + n2a) * t2);
            float c1 = (float)c1d;
            const BetaEntryF *row = tab + (size_t)(n1 - a.n1lo) * W2 - a.n2lo;
            for (int n2 = n2a; n2 <= n2b; ++n2) {
                float c2v = (float)(a.a2 + n2);
                float A2 = c1 * c1 + c2v * c2v;
                BetaEntryF be = row[n2];
                if (valid && A2 <= R2f) {
                    float2 ez;
                    if (be.bi == 0.f) {
                        float sz, cz;
                        sincosf(be.br * z, &sz, &cz);
                        ez = make_float2(cz, sz);
                    } else {
                        ez = make_float2(__expf(-be.bi * z), 0.f);
                    }
                    float2 term = cmul(cmul(make_float2(be.ibr, be.ibi), ez), p);
                    if (NF == 1) {
                        acc[0][0] += term.x;
                        acc[0][1] += term.y;
                    } else {
                        float2 b = make_float2(be.br * sg, be.bi * sg);
                        float2 b2 = make_float2(be.br * be.br - be.bi * be.bi, 2.f * be.br * be.bi);
                        float2 f[6] = {make_float2(1.f - c1 * c1 * ik2, 0.f), make_float2(1.f - c2v * c2v * ik2, 0.f),
                                       make_float2(1.f - b2.x * ik2, -b2.y * ik2), make_float2(-c1 * c2v * ik2, 0.f),
                                       make_float2(-c1 * b.x * ik2, -c1 * b.y * ik2),
                                       make_float2(-c2v * b.x * ik2, -c2v * b.y * ik2)};
#pragma unroll
                        for (int e = 0; e < 6; ++e) {
                            float2 tf = cmul(f[e], term);
                            acc[e][0] += tf.x;
                            acc[e][1] += tf.y;
                        }
                        acc[6][0] += term.x;
                        acc[6][1] += term.y;
                    }
                }
                p = cmul(p, step);
            }
        }
        if (!valid) continue;
        double2 lat = lattice_phase(a.a1, m1, a.a2, m2);
        double2 pre = cmul(lat, make_double2(0.0, 1.0 / (8.0 * GF_PI * GF_PI)));
        float2 *o = out + (size_t)idx * ne;
        if (NF == 1) {
            store_out(o, cmul(pre, make_double2(acc[0][0], acc[0][1])));
        } else {
            for (int e = 0; e < 6; ++e) store_out(o + e, cmul(pre, make_double2(acc[e][0], acc[e][1])));
            if (a.which == GF_OUT_MAXWELL7) store_out(o + 6, cmul(pre, make_double2(acc[6][0], acc[6][1])));
        }
    }
}

// ---------------------------------------------------------------------------
// 2D far kernel: G = e^{i2pi alpha m} (i/4pi) sum_n beta_n^{-1} e^{i alpha_n t + i beta_n |x2|}
// (terms and sums in double for both precisions; the 1D series is short).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128) far2d(EvalArgs a)
{
    typedef typename cplx_t<R>::T C;
    C *out = reinterpret_cast<C *>(a.out);
    const int count = *a.far_count;
    const double k2 = a.k * a.k;
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < count; slot += gridDim.x * blockDim.x) {
        int idx = a.far_idx[slot];
        double x1 = a.x[2 * (size_t)idx], x2 = a.x[2 * (size_t)idx + 1];
        double t, m;
        reduce_period(x1, t, m);
        double z = fabs(x2);
        double Tz = a.T / z;
        double R2 = k2 + Tz * Tz, Rr = sqrt(R2);
        int na = (int)floor(-a.a1 - Rr) - 1, nb = (int)ceil(-a.a1 + Rr) + 1;
        double st, ct;
        sincos(t, &st, &ct);
        const double2 step = make_double2(ct, st);
        double sp, cp;
        sincos((a.a1 + na) * t, &sp, &cp);
        double2 p = make_double2(cp, sp);
        double sr = 0, si = 0;
        for (int n = na; n <= nb; ++n) {
            double c1 = a.a1 + n;
            double A2 = c1 * c1;
            if (A2 <= R2) {
                double aa = fabs(c1);
                double2 term;
                if (aa <= a.k) {
                    double b = sqrt((a.k - aa) * (a.k + aa));
                    double sz, cz;
                    sincos(b * z, &sz, &cz);
                    term = cscale(cmul(make_double2(cz, sz), p), 1.0 / b);
                } else {
                    double b = sqrt((aa - a.k) * (aa + a.k));
                    double e = exp(-b * z) / b;
                    term = cmul(make_double2(0.0, -e), p);  // (1/(i b)) e^{-b z} p
                }
                sr += term.x;
                si += term.y;
            }
            p = cmul(p, step);
        }
        double2 lat = lattice_phase(a.a1, m, 0.0, 0.0);
        double2 pre = cmul(lat, make_double2(0.0, 0.25 / GF_PI));
        store_out(out + idx, cmul(pre, make_double2(sr, si)));
    }
}

template <typename R>
cudaError_t launch_eval_t(const EvalArgs &a, cudaStream_t s, cudaEvent_t ev_mid)
{
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (a.n + 255) / 256;
    if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
    if (blocks < 1) blocks = 1;
    const int farblocks = nsm * 8;
    if (a.dim == 2) {
        near2d<R><<<(int)blocks, 256, 0, s>>>(a);
        if (ev_mid) cudaEventRecord(ev_mid, s);
        far2d<R><<<farblocks, 128, 0, s>>>(a);
    } else if (a.nf == 1) {
        near3d<R, 1><<<(int)blocks, 256, 0, s>>>(a);
        if (ev_mid) cudaEventRecord(ev_mid, s);
        if (sizeof(R) == 8)
            far3d_f64<1><<<farblocks, 128, 0, s>>>(a);
        else
            far3d_f32<1><<<farblocks, 128, 0, s>>>(a);
    } else {
        near3d<R, 7><<<(int)blocks, 256, 0, s>>>(a);
        if (ev_mid) cudaEventRecord(ev_mid, s);
        if (sizeof(R) == 8)
            far3d_f64<7><<<farblocks, 128, 0, s>>>(a);
        else
            far3d_f32<7><<<farblocks, 128, 0, s>>>(a);
    }
    gf_count_launch(2);
    return cudaGetLastError();
}

}  // namespace

cudaError_t gf_launch_beta_table(const EvalArgs &a, int precision, cudaStream_t s)
{
    if (precision == GF_FP64)
        beta_table<BetaEntry><<<256, 256, 0, s>>>(a, (BetaEntry *)a.btab);
    else
        beta_table<BetaEntryF><<<256, 256, 0, s>>>(a, (BetaEntryF *)a.btab);
    gf_count_launch(1);
    return cudaGetLastError();
}

cudaError_t gf_launch_eval(const EvalArgs &a, int precision, cudaStream_t s, cudaEvent_t ev_mid)
{
    return precision == GF_FP64 ? launch_eval_t<double>(a, s, ev_mid) : launch_eval_t<float>(a, s, ev_mid);
}
