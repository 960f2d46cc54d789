// Evaluation at targets (Algorithms 1-3, step 2 "Calculation").
//
//  near branch  (|x_last| <= c): reduce to the unit cell (step 2c), gather the
//               4^d stencil of the padded grid with separable cubic Lagrange
//               weights (step 2d), add the singular part back in double
//               precision (step 2e), apply the quasi-periodic phase (step 2f).
//               3D evaluations first classify the targets (a far list sorted
//               by |x3| bucket, a near list), then run the near targets from
//               their list in full warps.
//  far branch   (|x_last| > c, step 2b): the eigen-series (ei)/(he) (and its
//               second derivatives for the Maxwell tensor), truncated to
//               |alpha_n|^2 <= k^2 + (T/|x_last|)^2, one thread per target,
//               the 32 lanes of a warp walking the same index set so that the
//               per-index table of beta_n is read by broadcast; for
//               double-precision plans two kernels, the double and float-float
//               core sums and the float tails, run side by side.
#include <math_constants.h>

#include "gf_internal.cuh"

namespace {

constexpr double TWO_PI = 2.0 * GF_PI;
constexpr double INV_TWO_PI = 1.0 / (2.0 * GF_PI);

// floor of the correctly rounded quotient a/b.  The product a * ib (ib = fl(1/b))
// differs from that quotient by a few ulps, so it decides the floor unless it
// lies within 1e-14 max(1, |a/b|) of an integer, where the quotient is formed.
// q receives the value the floor was taken of.
__device__ __forceinline__ double floor_quot(double a, double b, double ib, double &q)
{
    q = __dmul_rn(a, ib);
    const double fq = floor(q), fr = q - fq;
    const double g = 1e-14 * fmax(1.0, fabs(q));
    if (fr < g || fr > 1.0 - g) {
        q = __ddiv_rn(a, b);
        return floor(q);
    }
    return fq;
}

// x = 2 pi m + t, t in [-pi, pi), with explicit round-to-nearest operations
// (no contraction) so that the cell decision is reproducible: m is the floor of
// the correctly rounded (x + pi)/(2 pi).
__device__ __forceinline__ void reduce_period(double x, double &t, double &m)
{
    double q;
    double mm = floor_quot(__dadd_rn(x, GF_PI), TWO_PI, INV_TWO_PI, q);
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
// i0 is the floor of the correctly rounded quotient (ih = fl(1/h)).
__device__ __forceinline__ int stencil_origin(double y, double y0, double h, double ih, int M, double &f)
{
    double u;
    double i0 = floor_quot(__dsub_rn(y, y0), h, ih, u);
    if (i0 > (double)(M - 1)) i0 = (double)(M - 1);
    if (i0 < 0.0) i0 = 0.0;
    f = u - i0;
    return (int)i0;
}

template <typename T>
__device__ __forceinline__ void lagrange4(T f, T w[4])
{
    const T fm1 = f - (T)1, fm2 = f - (T)2, fp1 = f + (T)1;
    w[0] = -f * fm1 * fm2 * (T)(1.0 / 6.0);
    w[1] = fp1 * fm1 * fm2 * (T)0.5;
    w[2] = -fp1 * f * fm2 * (T)0.5;
    w[3] = fp1 * f * fm1 * (T)(1.0 / 6.0);
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
__device__ __forceinline__ void add_out(double2 *o, double2 v)
{
    atomicAdd(&o->x, v.x);
    atomicAdd(&o->y, v.y);
}
__device__ __forceinline__ void add_out_f(float2 *o, float2 v)
{
    atomicAdd(&o->x, v.x);
    atomicAdd(&o->y, v.y);
}
__device__ __forceinline__ void add_c(double2 *o, double2 v) { add_out(o, v); }
__device__ __forceinline__ void add_c(float2 *o, float2 v) { add_out_f(o, v); }

// A far kernel's share (entries v[0 .. ne-1]) of target idx, from row slab `slab`
// of `nslab` of chunk w.  With one slab per chunk, or no slab scratch, it is
// added into the output at once.  Otherwise each slab stores its partials; the
// chunk's last slab to finish (the one that draws the last ticket; nobody waits)
// adds them up in slab order and deposits the total.  The output, zeroed by the
// near pass, then receives one addend per far kernel (two at most), and a sum of
// two terms onto zero is the same in either order: the result does not depend on
// which slab or kernel finishes first.
template <typename C, int NE>
__device__ __forceinline__ void far_deposit(const EvalArgs &a, int kind, int w, int slab, int nslab, int nslot,
                                            bool valid, int idx, int ne, const C (&v)[NE])
{
    C *o = reinterpret_cast<C *>(a.out) + (size_t)idx * ne;
    C *buf = reinterpret_cast<C *>(a.slabbuf[kind]);
    if (nslab <= 1 || buf == nullptr) {
        if (valid)
#pragma unroll
            for (int e = 0; e < NE; ++e)
                if (e < ne) add_c(o + e, v[e]);
        return;
    }
    const int lane = threadIdx.x & 31;
    const size_t slot = (size_t)w * 32 + lane;
    if (valid)
#pragma unroll
        for (int e = 0; e < NE; ++e)
            if (e < ne) buf[((size_t)slab * nslot + slot) * ne + e] = v[e];
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) last = atomicAdd(a.slabtick[kind] + w, 1) == nslab - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last || !valid) return;
    __threadfence();
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        if (e >= ne) break;
        C sum = __ldcg(buf + slot * ne + e);
        for (int s = 1; s < nslab; ++s) sum = cadd(sum, __ldcg(buf + ((size_t)s * nslot + slot) * ne + e));
        add_c(o + e, sum);
    }
}

// Row slabs per chunk of a far launch, capped by the slab scratch (kind 0: the
// main far kernel, 1: the float tails).
__device__ __forceinline__ int far_slabs_capped(const EvalArgs &a, int kind, int nch, int S)
{
    if (a.slabbuf[kind] == nullptr || nch <= 0) return S;
    const int64_t fit = a.slabcap / ((int64_t)nch * 32);
    return (int)(fit < 1 ? 1 : (fit < S ? fit : S));
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R> __device__ __forceinline__ typename cplx_t<R>::T zero_c();
template <> __device__ __forceinline__ double2 zero_c<double>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 zero_c<float>() { return make_float2(0.f, 0.f); }

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
__host__ __device__ __forceinline__ int n_entries(int which) { return gf_out_entries(which); }

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

// Adds the number of lanes that vote `take` to *count (one atomic per warp).
__device__ __forceinline__ void count_votes(bool take, int *count)
{
    unsigned mask = __ballot_sync(0xffffffffu, take);
    if (mask != 0u && (threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(count, __popc(mask));
}
__device__ __forceinline__ int far_bucket(double z, double c)
{
    double r = (double)GF_FAR_BUCKETS * c / z;
    int b = (int)r;
    return b < GF_FAR_BUCKETS - 1 ? b : GF_FAR_BUCKETS - 1;
}

// ---------------------------------------------------------------------------
// 3D near kernel.  NF = 1: Helmholtz (field L_d).  NF = 7: Maxwell
// (fields 0..5 = (delta_pq - c^p c^q/k^2) L_d, field 6 = L_d).
// R = storage/accumulation type of the grid (double: GF_FP64, float: split).
// ---------------------------------------------------------------------------
// The near branch at one target i (valid, finite, |x_last| <= c): cell
// reduction, tensor cubic interpolation of the stored grid, phases and the
// singular part (Algorithm 2, calculation step).
template <typename R, int NF>
__device__ __forceinline__ void near_point(const EvalArgs &a, int64_t i, double x1, double x2, double x3, double ih1,
                                           double ih2, double ih3)
{
    typedef typename cplx_t<R>::T C;
    const C *G = reinterpret_cast<const C *>(a.grid);
    const int ne = n_entries(a.which);
    C *o = reinterpret_cast<C *>(a.out) + i * ne;
    const bool only_L = NF == 1 && a.which == GF_OUT_LD;
    double t1, m1, t2, m2;
    reduce_period(x1, t1, m1);
    reduce_period(x2, t2, m2);
    double f1, f2, f3;
    int i1 = stencil_origin(t1, -GF_PI, a.h1, ih1, a.M1, f1);
    int i2 = stencil_origin(t2, -GF_PI, a.h2, ih2, a.M2, f2);
    // stored planes from Q3lo: a Helmholtz grid (even in x3) holds x3 >= -h3 only
    // and is read at |x3|; so is a Maxwell grid that keeps the odd fields' Nyquist
    // planes (nyqgrid), otherwise it holds the slab |x3| <= c
    const bool mirror = NF == 1 || a.nyqgrid != nullptr;
    const int i3n = stencil_origin(mirror ? fabs(x3) : x3, -a.ct, a.h3, ih3, a.M3, f3);
    const int i3 = i3n - a.Q3lo;
    // weights in the grid's precision (f itself is formed in double)
    R w1[4], w2[4], w3[4];
    lagrange4<R>((R)f1, w1);
    lagrange4<R>((R)f2, w2);
    lagrange4<R>((R)f3, w3);
    R acc[NF][2];
#pragma unroll
    for (int e = 0; e < NF; ++e) acc[e][0] = acc[e][1] = (R)0;
#pragma unroll
    for (int d3 = 0; d3 < 4; ++d3) {
#pragma unroll
        for (int d2 = 0; d2 < 4; ++d2) {
            const C *row = G + (((size_t)(i3 + d3) * a.P2 + (i2 + d2)) * a.P1 + i1) * NF;
            const R w23 = w3[d3] * w2[d2];
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
    if (NF > 1 && a.nyqgrid != nullptr && x3 < 0.0) {
        // The stencil of x3 < 0 is the mirror of the one read at |x3| (nodes
        // a' = i3n - 1 .. i3n + 2 <-> M3 - a').  Even fields: the same values.  Odd
        // fields (4: xz, 5: yz): L(M3 - a') = -L(a') + 2 (-1)^(M3/2 + a') P(t), so
        // the interpolant is -acc + 2 (-1)^(M3/2) (sum_d w3_d (-1)^(a'_d)) P(t),
        // P interpolated bicubically from the Nyquist planes.
        R sgn = w3[0] - w3[1] + w3[2] - w3[3];
        if (((i3n - 1) ^ (a.M3 >> 1)) & 1) sgn = -sgn;
        const C *NG = reinterpret_cast<const C *>(a.nyqgrid);
        R pr[2] = {0, 0}, pi[2] = {0, 0};
#pragma unroll
        for (int d2 = 0; d2 < 4; ++d2) {
            const C *row = NG + ((size_t)(i2 + d2) * a.P1 + i1) * 2;
            R s4r = 0, s4i = 0, s5r = 0, s5i = 0;
#pragma unroll
            for (int d1 = 0; d1 < 4; ++d1) {
                const C g4 = __ldg(row + 2 * d1), g5 = __ldg(row + 2 * d1 + 1);
                s4r = fma(w1[d1], g4.x, s4r);
                s4i = fma(w1[d1], g4.y, s4i);
                s5r = fma(w1[d1], g5.x, s5r);
                s5i = fma(w1[d1], g5.y, s5i);
            }
            pr[0] = fma(w2[d2], s4r, pr[0]);
            pi[0] = fma(w2[d2], s4i, pi[0]);
            pr[1] = fma(w2[d2], s5r, pr[1]);
            pi[1] = fma(w2[d2], s5i, pi[1]);
        }
        const R two_s = (R)2 * sgn;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            acc[4 + q][0] = fma(two_s, pr[q], -acc[4 + q][0]);
            acc[4 + q][1] = fma(two_s, pi[q], -acc[4 + q][1]);
        }
    }

    // lift = e^{i alpha.t} e^{i 2 pi <alpha.m>}; G = lift L + e^{i 2pi<alpha.m>} Phi Y (K = L + F, F = e^{-i alpha.t} Phi Y).
    // Split plans: the fractional part in double, the two phases in float.
    double2 lat, lift;
    float2 latf = make_float2(0.f, 0.f), liftf = make_float2(0.f, 0.f);
    if (sizeof(R) == 4) {
        double ph = a.a1 * m1 + a.a2 * m2;
        ph -= rint(ph);
        float sl, cl, sa, ca;
        sincospif(2.0f * (float)ph, &sl, &cl);
        sincosf((float)a.a1 * (float)t1 + (float)a.a2 * (float)t2, &sa, &ca);
        latf = make_float2(cl, sl);
        liftf = cmulf(make_float2(ca, sa), latf);
        lat = make_double2(cl, sl);
        lift = make_double2(liftf.x, liftf.y);
    } else {
        lat = lattice_phase(a.a1, m1, a.a2, m2);
        double sa, ca;
        sincos(a.a1 * t1 + a.a2 * t2, &sa, &ca);
        lift = cmul(make_double2(ca, sa), lat);
    }
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
        if (only_L) {
            store_out(o, L);
            return;
        }
        if (sizeof(R) == 4) {
            // split: the combination in float (the singular part was formed in double)
            const float2 v = cmulf(liftf, make_float2((float)acc[0][0], (float)acc[0][1]));
            const float2 u = sing ? cmulf(latf, make_float2((float)PhiY.x, (float)PhiY.y)) : make_float2(0.f, 0.f);
            reinterpret_cast<float2 *>(o)[0] = make_float2(v.x + u.x, v.y + u.y);
            return;
        }
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

// Far-region grid at one target i (valid, finite, c < |x3| <= fzmax): the same
// cell reduction as the near branch, tensor cubic interpolation of the far
// planes (in z from fz0 with the stencil origin clamped to the last full
// interval), and the lift e^{i alpha.t} e^{i 2 pi <alpha.m>}; the Maxwell xz and
// yz entries change sign with x3.  No singular part: |x3| > c >= 2 eps.
template <typename R, int NF>
__device__ __forceinline__ void far_grid_point(const EvalArgs &a, int64_t i, double x1, double x2, double x3)
{
    typedef typename cplx_t<R>::T C;
    const C *G = reinterpret_cast<const C *>(a.fargrid);
    const int ne = n_entries(a.which);
    C *o = reinterpret_cast<C *>(a.out) + i * ne;
    double t1, m1, t2, m2;
    reduce_period(x1, t1, m1);
    reduce_period(x2, t2, m2);
    double f1, f2, f3;
    const int i1 = stencil_origin(t1, -GF_PI, a.fh1, 1.0 / a.fh1, a.fM1, f1);
    const int i2 = stencil_origin(t2, -GF_PI, a.fh2, 1.0 / a.fh2, a.fM2, f2);
    // planes are not padded: the stencil planes are i0 - 1 .. i0 + 2, i0 <= fNZ - 3
    const int i3 = stencil_origin(fabs(x3), a.fz0, a.fhz, 1.0 / a.fhz, a.fNZ - 2, f3) - 1;
    R w1[4], w2[4], w3[4];
    lagrange4<R>((R)f1, w1);
    lagrange4<R>((R)f2, w2);
    lagrange4<R>((R)f3, w3);
    R acc[NF][2];
#pragma unroll
    for (int e = 0; e < NF; ++e) acc[e][0] = acc[e][1] = (R)0;
#pragma unroll
    for (int d3 = 0; d3 < 4; ++d3) {
#pragma unroll
        for (int d2 = 0; d2 < 4; ++d2) {
            const C *row = G + (((size_t)(i3 + d3) * a.fP2 + (i2 + d2)) * a.fP1 + i1) * NF;
            const R w23 = w3[d3] * w2[d2];
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
    if (sizeof(R) == 4) {
        double ph = a.a1 * m1 + a.a2 * m2;
        ph -= rint(ph);
        float sl, cl, sa, ca;
        sincospif(2.0f * (float)ph, &sl, &cl);
        sincosf((float)a.a1 * (float)t1 + (float)a.a2 * (float)t2, &sa, &ca);
        const float2 lift = cmulf(make_float2(ca, sa), make_float2(cl, sl));
        float2 *of = reinterpret_cast<float2 *>(o);
        for (int e = 0; e < ne; ++e) {
            const int f = NF == 1 ? 0 : (e < 6 ? e : 6);
            float2 v = cmulf(lift, make_float2((float)acc[f][0], (float)acc[f][1]));
            if (NF > 1 && (e == 4 || e == 5) && x3 < 0.0) v = make_float2(-v.x, -v.y);
            of[e] = v;
        }
    } else {
        const double2 lat = lattice_phase(a.a1, m1, a.a2, m2);
        double sa, ca;
        sincos(a.a1 * t1 + a.a2 * t2, &sa, &ca);
        const double2 lift = cmul(make_double2(ca, sa), lat);
        for (int e = 0; e < ne; ++e) {
            const int f = NF == 1 ? 0 : (e < 6 ? e : 6);
            double2 v = cmul(lift, make_double2((double)acc[f][0], (double)acc[f][1]));
            if (NF > 1 && (e == 4 || e == 5) && x3 < 0.0) v = make_double2(-v.x, -v.y);
            store_out(o + e, v);
        }
    }
}

// Append to the end of the near list, backwards (far-grid targets): the list
// holds the near targets from its start and these from its end, so that the
// warps of the list kernel see one kind or the other.
__device__ __forceinline__ void push_back_end(bool take, int i, int *list, int64_t cap, int *count)
{
    unsigned mask = __ballot_sync(0xffffffffu, take);
    if (mask == 0u) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (take) list[cap - 1 - (base + __popc(mask & ((1u << lane) - 1u)))] = i;
}

// MODE 0: classify every target (far list, bucket histogram, zeroed far
// outputs, NaN for non-finite ones) and evaluate the near ones (and those of
// the far-region grid) here; MODE 1: classify only, appending the near targets
// to the start of a.near_idx and the far-grid targets to its end, so that
// near3d_list evaluates them in full warps.
template <typename R, int NF, int MODE>
__device__ void near3d_tiles(const EvalArgs &a, int64_t base0, int64_t stride, int *hist)
{
    typedef typename cplx_t<R>::T C;
    C *out = reinterpret_cast<C *>(a.out);
    const int ne = n_entries(a.which);
    const double ih1 = 1.0 / a.h1, ih2 = 1.0 / a.h2, ih3 = 1.0 / a.h3;
    for (int64_t base = base0; base < a.n; base += stride) {
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
        const bool only_L = NF == 1 && a.which == GF_OUT_LD;
        if (only_L && isfar) {
            out[i] = nan_c<R>();  // the remainder alone is served on the near region only
            isfar = false;
            valid = false;
        }
        // far targets inside the far-region grid's slab are gathered, not summed
        const bool fgrid = isfar && a.fargrid != nullptr && fabs(x3) <= a.fzmax;
        if (fgrid) isfar = false;
        if (a.seghist) {
            // stable far list: the bucket code here, the list laid out afterwards
            count_votes(isfar, a.far_count);
            if (i < a.n) a.far_idx[i] = isfar ? far_bucket(fabs(x3), a.c) : -1;
        } else {
            push_far(isfar, (int)i, a.far_idx, a.far_count);
        }
        // (every lane of the warp reaches the appends: they vote by ballot)
        if (MODE == 1) {
            push_far(valid && finite && !isfar && !fgrid, (int)i, a.near_idx, a.far_count + GF_NEAR_SLOT);
            push_back_end(fgrid, (int)i, a.near_idx, a.n, a.far_count + GF_FGRID_SLOT);
        }
        C *o = out + i * ne;
        if (fgrid) {
            if (MODE == 0) far_grid_point<R, NF>(a, i, x1, x2, x3);
            continue;
        }
        if (isfar) {
            // the far kernels add their row slabs into these entries
            atomicAdd(&hist[far_bucket(fabs(x3), a.c)], 1);
            for (int e = 0; e < ne; ++e) o[e] = zero_c<R>();
            continue;
        }
        if (!valid) continue;
        if (!finite) {
            for (int e = 0; e < ne; ++e) o[e] = nan_c<R>();
            continue;
        }
        if (MODE == 0) near_point<R, NF>(a, i, x1, x2, x3, ih1, ih2, ih3);
    }
}

// Entry j of the targets listed by a MODE-1 classification pass: the near
// targets (j < nnear) from the start of the list, then the far-grid ones from
// its end.
template <typename R, int NF>
__device__ __forceinline__ void list_point(const EvalArgs &a, int j, int nnear, double ih1, double ih2, double ih3)
{
    if (j < nnear) {
        const int64_t i = a.near_idx[j];
        near_point<R, NF>(a, i, a.x[3 * i], a.x[3 * i + 1], a.x[3 * i + 2], ih1, ih2, ih3);
    } else {
        const int64_t i = a.near_idx[a.n - 1 - (j - nnear)];
        far_grid_point<R, NF>(a, i, a.x[3 * i], a.x[3 * i + 1], a.x[3 * i + 2]);
    }
}

// The targets listed by a MODE-1 classification pass, one per thread.
template <typename R, int NF>
__global__ void __launch_bounds__(256) near3d_list(EvalArgs a)
{
    const int nnear = a.far_count[GF_NEAR_SLOT];
    const int count = nnear + a.far_count[GF_FGRID_SLOT];
    const double ih1 = 1.0 / a.h1, ih2 = 1.0 / a.h2, ih3 = 1.0 / a.h3;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x)
        list_point<R, NF>(a, j, nnear, ih1, ih2, ih3);
}

template <typename R, int NF, int MODE = 0>
__global__ void __launch_bounds__(256) near3d(EvalArgs a)
{
    __shared__ int hist[GF_FAR_BUCKETS];
    for (int b = threadIdx.x; b < GF_FAR_BUCKETS; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    near3d_tiles<R, NF, MODE>(a, (int64_t)blockIdx.x * blockDim.x, (int64_t)gridDim.x * blockDim.x, hist);
    __syncthreads();
    for (int b = threadIdx.x; b < GF_FAR_BUCKETS; b += blockDim.x)
        if (hist[b]) atomicAdd(&a.far_count[1 + b], hist[b]);
}

// Batched near kernel: persistent CTAs walk the (pair, 256-target tile) list.
__device__ __forceinline__ int batch_pair_e(const int *prefix, int np, int vb)
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

template <typename R, int NF, int MODE = 0>
__global__ void __launch_bounds__(256) near3d_batch(const EvalArgs *args, const int *prefix, int np)
{
    __shared__ int hist[GF_FAR_BUCKETS];
    __shared__ EvalArgs sa;
    const int total = prefix[np];
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const int p = batch_pair_e(prefix, np, vb);
        if (threadIdx.x == 0) sa = args[p];
        for (int b = threadIdx.x; b < GF_FAR_BUCKETS; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const int64_t base = (int64_t)(vb - prefix[p]) * blockDim.x;
        near3d_tiles<R, NF, MODE>(sa, base, sa.n + blockDim.x, hist);
        __syncthreads();
        for (int b = threadIdx.x; b < GF_FAR_BUCKETS; b += blockDim.x)
            if (hist[b]) atomicAdd(&sa.far_count[1 + b], hist[b]);
        __syncthreads();
    }
}

// Batched near targets from the pairs' near lists (filled by a MODE-1
// near3d_batch pass): every CTA walks the pairs in order, and within a pair the
// list is spread over the grid starting at a CTA that rotates by the previous
// pairs' block counts, so that small lists land on different CTAs.
template <typename R, int NF>
__global__ void __launch_bounds__(256) near3d_list_batch(const EvalArgs *args, int np)
{
    __shared__ EvalArgs sa;
    int rot = 0;
    for (int p = 0; p < np; ++p) {
        __syncthreads();
        if (threadIdx.x == 0) sa = args[p];
        __syncthreads();
        const int nnear = sa.far_count[GF_NEAR_SLOT];
        const int count = nnear + sa.far_count[GF_FGRID_SLOT];
        const double ih1 = 1.0 / sa.h1, ih2 = 1.0 / sa.h2, ih3 = 1.0 / sa.h3;
        const int cta = (int)((blockIdx.x + (unsigned)rot) % gridDim.x);
        for (int j = cta * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x)
            list_point<R, NF>(sa, j, nnear, ih1, ih2, ih3);
        rot = (int)((rot + (count + blockDim.x - 1) / blockDim.x) % gridDim.x);
    }
}

// ---------------------------------------------------------------------------
// 2D near kernel (Algorithm 1): K = L + f1 - i alpha f2, G = e^{i alpha x1} K,
// f1 = -(1/2pi) ln r Y_eps(r), f2 = t f1 at the reduced point (t, x2).
// NF fields per node: 1 (L), 3 (derivative plans: L, K_1 - h_1, K_2 - h_2) or
// 6 (and T_11 - h_11, T_12 - h_12, T_22 - h_22).  Outputs: G; GF_OUT_GRAD = G,
// dG/dx1, dG/dx2 (Sec. 2.4.1: K_i = (K_i - h_i)_N + h_i, dG/dx_i = e^{i alpha x1}
// K_i); GF_OUT_HESSDIFF = T_11, T_12, T_22 (Sec. 2.4.2, the same with h_pq), the
// singular parts
//   h_1  = -(1/2pi)[-(k^2/2) x1 ln r + x1/r^2 - i alpha x1^2/r^2 - (alpha^2/2) x1^3/r^2] Y
//   h_2  = -(1/2pi)[-(k^2/2) x2 ln r + x2/r^2 - i alpha x1 x2/r^2 - (alpha^2/2) x1^2 x2/r^2] Y
//   h_11 = (dk2/2pi)[ln r/2 - (i alpha/2) x1 ln r + x1^2/(2r^2) - i alpha x1^3/(2r^2)] Y
//   h_12 = (dk2/2pi)[x1 x2/(2r^2) - (i alpha/2) x1^2 x2/r^2] Y
//   h_22 = (dk2/2pi)[ln r/2 - (i alpha/2) x1 ln r + x2^2/(2r^2) - (i alpha/2) x1 x2^2/r^2] Y
// (dk2 = k^2 - k2^2) at (x1, x2) = (t, x2), in double.
// ---------------------------------------------------------------------------
template <typename R, int NF>
__global__ void __launch_bounds__(256) near2d(EvalArgs a)
{
    typedef typename cplx_t<R>::T C;
    const C *G = reinterpret_cast<const C *>(a.grid);
    C *out = reinterpret_cast<C *>(a.out);
    const double ih1 = 1.0 / a.h1, ih2 = 1.0 / a.h2;
    const int ne = n_entries(a.which);
    const int f0 = a.which == GF_OUT_HESSDIFF ? 3 : 0;
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
            for (int e = 0; e < ne; ++e) out[i * ne + e] = nan_c<R>();
            continue;
        }
        double t, m;
        reduce_period(x1, t, m);
        double f1, f2;
        int i1 = stencil_origin(t, -GF_PI, a.h1, ih1, a.M1, f1);
        int i2 = stencil_origin(x2, -a.ct, a.h2, ih2, a.M2, f2);
        double w1[4], w2[4];
        lagrange4(f1, w1);
        lagrange4(f2, w2);
        double acc[3][2] = {{0, 0}, {0, 0}, {0, 0}};
#pragma unroll
        for (int d2 = 0; d2 < 4; ++d2) {
            const C *row = G + ((size_t)(i2 + d2) * a.P1 + i1) * NF + f0;
#pragma unroll
            for (int e = 0; e < (NF == 1 ? 1 : 3); ++e) {
                if (e >= ne) break;
                double sr = 0, si = 0;
#pragma unroll
                for (int d1 = 0; d1 < 4; ++d1) {
                    double2 g = ld_grid(row + d1 * NF + e);
                    sr = fma(w1[d1], g.x, sr);
                    si = fma(w1[d1], g.y, si);
                }
                acc[e][0] = fma(w2[d2], sr, acc[e][0]);
                acc[e][1] = fma(w2[d2], si, acc[e][1]);
            }
        }
        double r = sqrt(t * t + x2 * x2);
        if (r < 2.0 * a.eps) {
            const double Y = 1.0 - smooth8((r - a.eps) / a.eps), lr = log(r), ir2 = 1.0 / (r * r);
            const double al = a.a1, kk = a.k * a.k, i2p = 0.5 / GF_PI;
            if (a.which != GF_OUT_HESSDIFF) {
                // K = L + f1 - i alpha f2
                const double fa = -lr * Y * i2p;
                acc[0][0] += fa;
                acc[0][1] -= al * t * fa;
            }
            if (a.which == GF_OUT_GRAD) {
                acc[1][0] += -i2p * (-0.5 * kk * t * lr + t * ir2 - 0.5 * al * al * t * t * t * ir2) * Y;
                acc[1][1] += i2p * al * t * t * ir2 * Y;
                acc[2][0] += -i2p * (-0.5 * kk * x2 * lr + x2 * ir2 - 0.5 * al * al * t * t * x2 * ir2) * Y;
                acc[2][1] += i2p * al * t * x2 * ir2 * Y;
            } else if (a.which == GF_OUT_HESSDIFF) {
                const double s = (kk - a.k2 * a.k2) * i2p * Y;
                acc[0][0] += s * (0.5 * lr + 0.5 * t * t * ir2);
                acc[0][1] += s * (-0.5 * al * t * lr - 0.5 * al * t * t * t * ir2);
                acc[1][0] += s * (0.5 * t * x2 * ir2);
                acc[1][1] += s * (-0.5 * al * t * t * x2 * ir2);
                acc[2][0] += s * (0.5 * lr + 0.5 * x2 * x2 * ir2);
                acc[2][1] += s * (-0.5 * al * t * lr - 0.5 * al * t * x2 * x2 * ir2);
            }
        }
        double sa, ca;
        sincos(a.a1 * t, &sa, &ca);
        const double2 lift = cmul(make_double2(ca, sa), lattice_phase(a.a1, m, 0.0, 0.0));
#pragma unroll
        for (int e = 0; e < 3; ++e)
            if (e < ne) store_out(out + i * ne + e, cmul(lift, make_double2(acc[e][0], acc[e][1])));
    }
}

// ---------------------------------------------------------------------------
// Counting-sort scatter of the far list by |x3| bucket, largest truncation
// radius first (bucket NB-1 first), so that warps see homogeneous lanes and
// the heaviest targets are scheduled first.
// ---------------------------------------------------------------------------
// Start of each bucket's run in the far list, the buckets in descending order
// (nearest the slab first), from the counts a.far_count[1 + b]; called by all
// threads of the block, by one warp: lane l takes the descending positions
// l PER .. l PER + PER - 1.
__device__ void far_bucket_starts(const EvalArgs &a, int *off)
{
    static_assert(GF_FAR_BUCKETS % 32 == 0, "bucket count: a multiple of 32");
    if (threadIdx.x < 32) {
        constexpr int PER = GF_FAR_BUCKETS / 32;
        const int lane = threadIdx.x;
        int c[PER], tot = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            c[i] = a.far_count[1 + (GF_FAR_BUCKETS - 1 - (lane * PER + i))];
            tot += c[i];
        }
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int s = incl - tot;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            off[GF_FAR_BUCKETS - 1 - (lane * PER + i)] = s;
            s += c[i];
        }
    }
    __syncthreads();
}

// Bucket sort of the appended far list (the batched sweeps): positions within a
// bucket in the order of the cursor atomics.
__device__ void far_scatter_body(const EvalArgs &a, int blk, int nblk, int *off)
{
    far_bucket_starts(a, off);
    const int count = a.far_count[0];
    int *cursor = a.far_count + 1 + GF_FAR_BUCKETS;
    for (int i = blk * blockDim.x + threadIdx.x; i < count; i += nblk * blockDim.x) {
        int idx = a.far_idx[i];
        double z = fabs(a.x[3 * (size_t)idx + 2]);
        int b = far_bucket(z, a.c);
        int pos = off[b] + atomicAdd(&cursor[b], 1);
        a.far_sorted[pos] = idx;
    }
}

// Stable counting sort of the far targets (single-plan evaluations), from the
// bucket codes the classification pass left in a.far_idx: the far kernels' warps
// take 32 consecutive list entries and set their truncation and precision bands
// from them, so a list that is the same from call to call makes the sums the same
// bit for bit.  Three passes over segments of a.segsize targets, one warp each:
// counts per segment and bucket, their exclusive scan over the segments (per
// bucket, from the bucket's start), and the scatter in index order.
__global__ void __launch_bounds__(256) far_seg_count(EvalArgs a)
{
    __shared__ int h[8][GF_FAR_BUCKETS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = blockIdx.x * 8 + w;
    if (seg >= a.nseg) return;
    for (int b = lane; b < GF_FAR_BUCKETS; b += 32) h[w][b] = 0;
    __syncwarp();
    const int64_t i0 = (int64_t)seg * a.segsize, i1 = min(i0 + (int64_t)a.segsize, a.n);
    for (int64_t i = i0 + lane; i < i1; i += 32) {
        const int c = a.far_idx[i];
        if (c >= 0) atomicAdd(&h[w][c], 1);
    }
    __syncwarp();
    int *dst = a.seghist + (size_t)seg * GF_FAR_BUCKETS;
    for (int b = lane; b < GF_FAR_BUCKETS; b += 32) dst[b] = h[w][b];
}

// One block per 32 buckets (a lane each), 32 warps over contiguous ranges of
// segments: each warp's sum, the warps' exclusive prefix, then the running
// position written back over the counts.
__global__ void __launch_bounds__(1024) far_seg_scan(EvalArgs a)
{
    __shared__ int start[GF_FAR_BUCKETS];
    __shared__ int part[32][32];
    far_bucket_starts(a, start);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * 32 + lane;
    const int per = (a.nseg + 31) / 32;
    const int s0 = min(w * per, a.nseg), s1 = min(s0 + per, a.nseg);
    int *col = a.seghist + b;
    int sum = 0;
#pragma unroll 8
    for (int sg = s0; sg < s1; ++sg) sum += col[(size_t)sg * GF_FAR_BUCKETS];
    part[w][lane] = sum;
    __syncthreads();
    int run = start[b];
    for (int v = 0; v < w; ++v) run += part[v][lane];
#pragma unroll 8
    for (int sg = s0; sg < s1; ++sg) {
        const int c = col[(size_t)sg * GF_FAR_BUCKETS];
        col[(size_t)sg * GF_FAR_BUCKETS] = run;
        run += c;
    }
}

// Each warp walks its segment in index order, 32 targets a step: the lanes with
// the same bucket take consecutive positions from the segment's running start.
__global__ void __launch_bounds__(256) far_seg_scatter(EvalArgs a)
{
    __shared__ int pos0[8][GF_FAR_BUCKETS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = blockIdx.x * 8 + w;
    if (seg >= a.nseg) return;
    const int *src = a.seghist + (size_t)seg * GF_FAR_BUCKETS;
    for (int b = lane; b < GF_FAR_BUCKETS; b += 32) pos0[w][b] = src[b];
    __syncwarp();
    const unsigned below = (1u << lane) - 1u;
    const int64_t i0 = (int64_t)seg * a.segsize, i1 = min(i0 + (int64_t)a.segsize, a.n);
    for (int64_t j = i0; j < i1; j += 32) {
        const int64_t i = j + lane;
        const int c = i < i1 ? a.far_idx[i] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const int before = __popc(peers & below);
        const int pos = c >= 0 ? pos0[w][c] + before : 0;
        __syncwarp();
        if (c >= 0) {
            a.far_sorted[pos] = (int)i;
            if (before == 0) pos0[w][c] += __popc(peers);
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) far_scatter(EvalArgs a)
{
    __shared__ int off[GF_FAR_BUCKETS];
    far_scatter_body(a, blockIdx.x, gridDim.x, off);
}

// batched: `per` CTAs per pair, persistent over the np * per work list
__global__ void __launch_bounds__(256) far_scatter_batch(const EvalArgs *args, int np, int per)
{
    __shared__ int off[GF_FAR_BUCKETS];
    __shared__ EvalArgs sa;
    for (int vb = blockIdx.x; vb < np * per; vb += gridDim.x) {
        if (threadIdx.x == 0) sa = args[vb / per];
        __syncthreads();
        far_scatter_body(sa, vb % per, per, off);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Far-series tables: |beta_n|, ln|beta_n| and 1/|beta_n| for evanescent n
// (beta_n = i |beta_n|); zeros for propagating n, whose terms are summed from
// the short list PropEntry instead.
// ---------------------------------------------------------------------------
// Propagating n (b = 0) get bl2 = +inf, so that the float sums' ex2(-bl2 z) is 0
// for them without a test.
__device__ __forceinline__ void set_entry(BetaEntry &e, double b, double ib)
{
    e.b = b;
    e.lnb = b > 0.0 ? log(b) : 0.0;
    e.bf = (float)b;
    e.blo = (float)(b - (double)e.bf);
    e.lnbf = (float)e.lnb;
    e.lnblo = (float)(e.lnb - (double)e.lnbf);
}
__device__ __forceinline__ void set_entry(BetaEntryF &e, double b, double ib)
{
    e.bl2 = b > 0.0 ? (float)(b * 1.4426950408889634) : CUDART_INF_F;  // b log2(e)
    e.ib = (float)ib;
    e.b = (float)b;
    e.pad = 0.f;
}

// Series tables of a 3D plan, built on the device: the b table over the index
// box, the exponential table e^{-(j - j0)/128}, and (block 0, warp 0) the list
// of propagating indices in row-major order of the sub-box pbox = [n1lo, n1hi,
// n2lo, n2hi] (ballot compaction keeps the order fixed).
template <typename E>
__global__ void series_tables(EvalArgs a, E *tab, double2 *exptab, PropEntry *prop, int *nprop, int4 pbox)
{
    const int W2 = a.n2hi - a.n2lo + 1;
    const int tot = (a.n1hi - a.n1lo + 1) * W2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
        int n1 = a.n1lo + i / W2, n2 = a.n2lo + i % W2;
        double c1 = a.a1 + n1, c2 = a.a2 + n2;
        double aa = sqrt(c1 * c1 + c2 * c2);
        E e;
        if (aa <= a.k) {
            set_entry(e, 0.0, 0.0);
        } else {
            double b = sqrt((aa - a.k) * (aa + a.k));
            set_entry(e, b, 1.0 / b);
        }
        tab[i] = e;
    }
    if (exptab)
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.exptab_n; j += gridDim.x * blockDim.x)
        {
            const double off = (double)(j - a.exptab_j0) * (1.0 / GF_EXPTAB_STEPS);
            const double ev = exp(-off);
            exptab[j] = make_double2(ev, off);
            // the float-float copy after it: (hi, lo) of e^{-y_j} and y_j (exact in float)
            const float hi = (float)ev;
            reinterpret_cast<float4 *>(exptab + a.exptab_n)[j] = make_float4(hi, (float)(ev - (double)hi), (float)off, 0.f);
        }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const int pw = pbox.w - pbox.z + 1, ptot = (pbox.y - pbox.x + 1) * pw;
        const int N0 = (int)rint(-a.a2);
        int cnt = 0;
        for (int base = 0; base < ptot; base += 32) {
            const int i = base + (int)threadIdx.x;
            bool in = false;
            double c1 = 0, c2 = 0, aa = 0;
            if (i < ptot) {
                c1 = a.a1 + (pbox.x + i / pw);
                c2 = a.a2 + (pbox.z + i % pw);
                aa = sqrt(c1 * c1 + c2 * c2);
                in = aa <= a.k;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, in);
            if (in) {
                const double br = sqrt((a.k - aa) * (a.k + aa));
                prop[cnt + __popc(bal & ((1u << threadIdx.x) - 1u))] =
                    PropEntry{c1, c2, br, 1.0 / br, (double)(pbox.z + i % pw - N0), 1, pbox.x + i / pw,
                              (float)c1, (float)c2, (float)br, (float)(1.0 / br)};
            }
            cnt += __popc(bal);
        }
        __syncwarp();
        // row starts: first = 0 where the previous entry is (n1, n2 - 1) (reads n1
        // and m2, writes only first)
        for (int q = (int)threadIdx.x; q < cnt; q += 32)
            prop[q].first = (q > 0 && prop[q - 1].n1 == prop[q].n1 && prop[q - 1].m2 + 1.0 == prop[q].m2) ? 0 : 1;
        if (threadIdx.x == 0) *nprop = cnt;
    }
}

// Warp maximum / minimum of non-negative doubles, compared as 64-bit integers
// (for x >= 0 the IEEE bit pattern orders like the value), which keeps the
// comparisons off the FP64 pipe; the result is one of the lanes' values.
__device__ __forceinline__ double warp_max(double v)
{
    long long b = __double_as_longlong(v);
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    return __longlong_as_double(b);
}

__device__ __forceinline__ double warp_min(double v)
{
    long long b = __double_as_longlong(v);
    for (int o = 16; o > 0; o >>= 1) b = min(b, __shfl_xor_sync(0xffffffffu, b, o));
    return __longlong_as_double(b);
}

// A float as a double by integer operations (no conversion instruction, which
// would occupy the FP64 pipe): exact for zero and normal floats; denormal floats
// (below 1.2e-38) read as zero.  Not for infinities or NaN.
__device__ __forceinline__ double f2d_exact(float f)
{
    const unsigned u = __float_as_uint(f);
    const bool nz = (u & 0x7F800000u) != 0u;
    const unsigned hi = (u & 0x80000000u) | (nz ? ((u & 0x7FFFFFFFu) >> 3) + 0x38000000u : 0u);
    return __hiloint2double((int)hi, nz ? (int)(u << 29) : 0);
}

// e^{-y} by Tang's table-driven method (ACM TOMS 15, 1989): y = y_j + r with
// y_j = (j - j0)/S, S = GF_EXPTAB_STEPS, |r| <= (1/2 + 4e-2)/S; e^{-y} = T[j] e^{-r},
// the plan table holding (e^{-y_j}, y_j).  The index is rint(S yf) + j0 for a
// float evaluation yf of y (|yf - y| < 6e-8 (2 b|x3| + 2 |ln b| + |y|), so that
// |S (yf - y)| < 4e-2 for the core terms, b|x3| < 20, and S <= 4096; rounding
// by the 1.5 * 2^23 shift), clamped to the table (callers discard the
// terms whose y lies beyond it).  Returns e^{-r} by its Taylor polynomial of
// degree DEG and T[j].x.  The truncation relative to e^{-y} is at most
// |r|^{DEG+1}/(DEG+1)! e^{|r|}; the far kernel takes three degrees (EXP_DEG_A >
// B > C), switching where a term lies e^{EXP_GAP_B} and e^{EXP_GAP_C} below the
// largest term of its series, so that every term's truncation stays below
// about 1e-17 of that largest term (bounds at |r| = 0.51/S, 0.52/S for S = 2048,
// 0.54/S for S = 4096):
//   S = 128: degrees 5/4/3 (5.6e-18, 8.4e-15, 1.1e-11), gaps 7 and 14;
//   S = 256: degrees 5/4/3 (8.7e-20, 2.6e-16, 6.6e-13), gaps 4 and 12;
//   S = 512: degrees 4/3/2 (8.2e-18, 4.1e-14, 1.7e-10), gaps 9 and 17.5;
//   S = 1024: degrees 4/3/2 (2.6e-19, 2.6e-15, 2.1e-11), gaps 6.25 and 15.25;
//   S = 2048: degrees 4/3/2 (8.8e-21, 1.7e-16, 2.7e-12), gaps 3.5 and 13.25;
//   S = 4096: degrees 3/2/1 (1.3e-17, 3.8e-13, 8.7e-9), gaps 10.75 and 20.75.
constexpr int EXP_DEG_A = GF_EXPTAB_STEPS >= 4096 ? 3 : GF_EXPTAB_STEPS >= 512 ? 4 : 5;
constexpr int EXP_DEG_B = EXP_DEG_A - 1, EXP_DEG_C = EXP_DEG_A - 2;
constexpr double EXP_GAP_B = GF_EXPTAB_STEPS >= 4096 ? 10.75 : GF_EXPTAB_STEPS >= 2048 ? 3.5
                           : GF_EXPTAB_STEPS >= 1024 ? 6.25 : GF_EXPTAB_STEPS >= 512 ? 9.0
                           : GF_EXPTAB_STEPS >= 256  ? 4.0 : 7.0;
constexpr double EXP_GAP_C = GF_EXPTAB_STEPS >= 4096 ? 20.75 : GF_EXPTAB_STEPS >= 2048 ? 13.25
                           : GF_EXPTAB_STEPS >= 1024 ? 15.25 : GF_EXPTAB_STEPS >= 512 ? 17.5
                           : GF_EXPTAB_STEPS >= 256  ? 12.0 : 14.0;

// (-1)^i / i!
__host__ __device__ constexpr double exp_taylor_coef(int i) { return i == 0 ? 1.0 : -exp_taylor_coef(i - 1) / i; }

template <int DEG>
__device__ __forceinline__ double exp_neg_split(double y, float yf, const double2 *__restrict__ T, int j0, int jmax,
                                                double &Tj)
{
    const float jm = fmaf((float)GF_EXPTAB_STEPS, yf, 12582912.0f);
    const int idx = min(max(__float_as_int(jm) - 0x4B400000 + j0, 0), jmax);
    const double2 t = __ldg(T + idx);
    const double r = y - t.y;
    Tj = t.x;
    if (DEG <= 1) return 1.0 - r;
    constexpr double c5 = exp_taylor_coef(5), c4 = exp_taylor_coef(4), c3 = exp_taylor_coef(3),
                     c2 = exp_taylor_coef(2);
    double p;
    if (DEG >= 5) {
        p = fma(r, c5, c4);
        p = fma(p, r, c3);
    } else if (DEG == 4) {
        p = fma(r, c4, c3);
    } else {
        p = c3;
    }
    if (DEG >= 3)
        p = fma(p, r, c2);
    else
        p = c2;
    p = fma(p, r, -1.0);
    return fma(p, r, 1.0);
}

// x with its sign bit flipped where m = 0x80000000 (an integer operation).
__device__ __forceinline__ double flip_sign(double x, int m)
{
    return __hiloint2double(__double2hiint(x) ^ m, __double2loint(x));
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Per-lane set-up of a far target (double): reduced t, lattice index m, z, sign.
struct FarLane {
    double t1, m1, t2, m2, z, iz, sg, R2;
    int idx;
    bool valid;
};

__device__ __forceinline__ FarLane far_lane(const EvalArgs &a, int slot, int count)
{
    FarLane L;
    L.valid = slot < count;
    L.idx = L.valid ? a.far_sorted[slot] : 0;
    double x1 = 0, x2 = 0, x3 = 1;
    if (L.valid) {
        x1 = a.x[3 * (size_t)L.idx];
        x2 = a.x[3 * (size_t)L.idx + 1];
        x3 = a.x[3 * (size_t)L.idx + 2];
    }
    // cell reduction by a multiply and a floor: the series does not depend on
    // the decomposition x = 2 pi m + t, so the near branch's exact cell decision
    // is not needed here
    L.m1 = floor(fma(x1, INV_TWO_PI, 0.5));
    L.m2 = floor(fma(x2, INV_TWO_PI, 0.5));
    L.t1 = fma(-TWO_PI, L.m1, x1);
    L.t2 = fma(-TWO_PI, L.m2, x2);
    L.z = fabs(x3);
    L.sg = x3 >= 0.0 ? 1.0 : -1.0;
    // explicitly rounded (no contraction): R2 decides the row split, which the
    // double-precision and float-tail kernels must reproduce exactly
    L.iz = __ddiv_rn(1.0, L.z);
    const double Tz = __dmul_rn(a.T, L.iz);
    L.R2 = L.valid ? __dadd_rn(__dmul_rn(a.k, a.k), __dmul_rn(Tz, Tz)) : 0.0;
    return L;
}

// Per-lane constants of Reinsch's form of the Clenshaw recurrence for the row
// sums sum_{k>=0} w_k e^{ik theta}, theta = t2, real weights w_k:
//   s = sign(cos theta), lambda = 2 cos theta - 2 s (-4 sin^2(theta/2) or 4 cos^2(theta/2)),
//   d_k = w_k + lambda b_{k+1} + s d_{k+1},  b_k = d_k + s b_{k+1},
//   sum = d_0 - (lambda/2) b_1 + i b_1 sin theta,  b_1 = s (b_0 - d_0).
// Unlike the plain three-term recurrence it keeps its accuracy for theta near
// 0 and pi (C. Reinsch, 1967; error analysis by Gentleman, Comput. J. 12, 1969).
struct Reinsch {
    double lam, hlam, sv;
    int m;  // sign bit of s
};

__device__ __forceinline__ Reinsch reinsch_lane(double sv, double cv)
{
    // 2 - 2 cos = 2 sin^2/(1 + cos) and 2 + 2 cos = 2 sin^2/(1 - cos), free of
    // cancellation on the side where each is used
    Reinsch R;
    const double s2 = 2.0 * sv * sv;
    R.m = cv >= 0.0 ? 0 : (int)0x80000000;
    R.lam = cv >= 0.0 ? -s2 / (1.0 + cv) : s2 / (1.0 - cv);
    R.hlam = 0.5 * R.lam;
    R.sv = sv;
    return R;
}

// Double-precision Reinsch state of NH row sums.  NH = 1 (G_d): w = e^{-bz}/b.
// NH = 6 (Maxwell partial sums): A = sum w, B = sum c2 w, C = sum c2^2 w,
// D = sum b^2 w, E = sum b w, F = sum c2 b w.
template <int NH>
struct RState {
    double d[NH], b[NH];
};

// ---------------------------------------------------------------------------
// Float-float arithmetic: a value is an unevaluated sum h + l of two floats
// (about 48 significant bits).  Error-free sum by Knuth's TwoSum, product by
// an fma (Dekker, Numer. Math. 18, 1971).  Every operation is explicitly
// rounded, so no contraction can break the error-free steps.
// ---------------------------------------------------------------------------
struct FF {
    float h, l;
};

__device__ __forceinline__ FF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    return FF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v))};
}

// a double as a float pair
__device__ __forceinline__ FF ff_split(double x)
{
    const float h = (float)x;
    return FF{h, (float)(x - (double)h)};
}

// Float-float Reinsch state of one sum (Helmholtz far series).
struct RStateFF {
    float dh, dl, bh, bl;
};

// The terms of the float-float band: n2, n2 + dir, ... (count of them), each
// at least e^{-FF_GAP} below the largest term of the series.  Float-float
// rounding perturbs y by about 1.3e-14 max(|y|, 1) (emulated over random b,
// |x3|), so a term at y = y_max + 8 is off by about 1.4e-13 e^{-8} < 5e-17 of
// the largest term: below half a double rounding of that term.  Per term: y = b z + ln b and e^{-y} =
// T[j] e^{-r} (the float-float table of the same step, r = y - y_j, |r| <=
// 0.54/S, e^{-r} to r^3 with r^2/2 - r^3/6 in float), then one Reinsch step:
// d' = w + lambda b + s d, b' = d' + s b.
constexpr float FF_GAP = 8.0f;

// One float-float Reinsch step with the term n2 (weight 0 outside the lane's
// truncation set).  Lazy form: the high words follow the recurrence in plain
// float, d' = (lambda b + w) + s d, b' = d' + s b; their rounding errors, exact
// by TwoProd and TwoSum, go into the low words, which follow the same
// recurrence.  The caller renormalizes the pairs every second step, so a low
// word stays within a few units of the high word's last place, while the high
// words' dependency chain is four float operations per term (a normalized
// float-float step chains about a dozen).
__device__ __forceinline__ void ff_step(RStateFF &st, const BetaEntry *__restrict__ row, int n2, float c2f,
                                        float c1sq, float R2f, FF z, FF lam, float sf, const float4 *__restrict__ T,
                                        int j0, int jmax)
{
    const float4 q = *reinterpret_cast<const float4 *>(&row[n2].bf);  // b hi, lo; ln b hi, lo
    const bool ok = fmaf(c2f, c2f, c1sq) <= R2f && q.x != 0.f;
    const float p = __fmul_rn(q.x, z.h);
    float pe = __fmaf_rn(q.x, z.h, -p);
    pe = __fmaf_rn(q.x, z.l, __fmaf_rn(q.y, z.h, pe));
    const FF y0 = two_sum(p, q.z);
    const FF y = two_sum(y0.h, __fadd_rn(__fadd_rn(y0.l, pe), q.w));
    const float jm = __fmaf_rn((float)GF_EXPTAB_STEPS, y.h, 12582912.0f);
    const int idx = min(max(__float_as_int(jm) - 0x4B400000 + j0, 0), jmax);
    const float4 t = __ldg(T + idx);
    const float rh = __fsub_rn(y.h, t.z);
    const float rs = __fadd_rn(rh, y.l);
    const float qq = __fmul_rn(__fmul_rn(rs, rs), __fmaf_rn(rs, -1.0f / 6.0f, 0.5f));
    const FF a = two_sum(1.0f, -rh);
    const float al = __fadd_rn(__fsub_rn(a.l, y.l), qq);
    float wh = __fmul_rn(t.x, a.h);
    float wl = __fmaf_rn(t.x, a.h, -wh);
    wl = __fmaf_rn(t.x, al, __fmaf_rn(t.y, a.h, wl));
    wh = ok ? wh : 0.f;
    wl = ok ? wl : 0.f;
    // high words
    const float m = __fmul_rn(lam.h, st.bh);
    const float me = __fmaf_rn(lam.h, st.bh, -m);
    const FF u = two_sum(m, wh);
    const FF dn = two_sum(u.h, __fmul_rn(sf, st.dh));
    // low words: the errors, then lambda b and s d on the low parts
    const float dl = __fadd_rn(__fadd_rn(__fadd_rn(me, u.l), __fadd_rn(dn.l, wl)),
                               __fmaf_rn(lam.h, st.bl, __fmaf_rn(lam.l, st.bh, __fmul_rn(sf, st.dl))));
    const FF bn = two_sum(dn.h, __fmul_rn(sf, st.bh));
    st.bl = __fadd_rn(__fadd_rn(bn.l, dl), __fmul_rn(sf, st.bl));
    st.dh = dn.h;
    st.dl = dl;
    st.bh = bn.h;
}

// Renormalized pair (Fast2Sum of the high and the low word).
__device__ __forceinline__ void ff_renorm(float &h, float &l)
{
    const float s = __fadd_rn(h, l);
    l = __fsub_rn(l, __fsub_rn(s, h));
    h = s;
}

__device__ __forceinline__ void reinsch_seg_ff(RStateFF &st, const BetaEntry *__restrict__ row, int &n2, int count,
                                               int dir, float &c2f, float c1sq, float R2f, FF z, FF lam, float sf,
                                               const float4 *__restrict__ T, int j0, int jmax)
{
    const float df = (float)dir;
    int i = 0;
    for (; i + 1 < count; i += 2, n2 += 2 * dir, c2f += 2.0f * df) {
        ff_step(st, row, n2, c2f, c1sq, R2f, z, lam, sf, T, j0, jmax);
        ff_step(st, row, n2 + dir, c2f + df, c1sq, R2f, z, lam, sf, T, j0, jmax);
        ff_renorm(st.dh, st.dl);
        ff_renorm(st.bh, st.bl);
    }
    if (i < count) {
        ff_step(st, row, n2, c2f, c1sq, R2f, z, lam, sf, T, j0, jmax);
        ff_renorm(st.dh, st.dl);
        ff_renorm(st.bh, st.bl);
        n2 += dir;
        c2f += df;
    }
}

// Feed `count` terms n2, n2 + dir, ... into the state (the first has the
// highest recurrence index), advancing n2 and c2; weights on the lane's own
// truncation set, exponential of degree DEG.  Per term and sum the recurrence
// costs three FP64 operations; for NH = 1 the product T[j] e^{-r} is folded
// into the first.
template <int NH, int DEG>
__device__ __forceinline__ void reinsch_seg(RState<NH> &st, const BetaEntry *__restrict__ row, int &n2, int count,
                                            int dir, float &c2f, double &c2, float c1sq, float R2f, double z,
                                            const Reinsch &RS, const double2 *__restrict__ T, int j0, int jmax)
{
    const float zf = (float)z;
    const float df = (float)dir;
    const double dd = (double)dir;
#pragma unroll 2
    for (int i = 0; i < count; ++i, n2 += dir, c2f += df) {
        const BetaEntry be = row[n2];
        const bool ok = fmaf(c2f, c2f, c1sq) <= R2f && be.bf != 0.f;
        double Tj;
        double p = exp_neg_split<DEG>(fma(be.b, z, be.lnb), fmaf(be.bf, zf, be.lnbf), T, j0, jmax, Tj);
        p = ok ? p : 0.0;
        if (NH == 1) {
            const double dn = fma(RS.lam, st.b[0], fma(Tj, p, flip_sign(st.d[0], RS.m)));
            st.b[0] = dn + flip_sign(st.b[0], RS.m);
            st.d[0] = dn;
        } else {
            double wv[NH];
            wv[0] = Tj * p;
            wv[1] = c2 * wv[0];
            wv[2] = c2 * wv[1];
            wv[4] = be.b * wv[0];
            wv[3] = be.b * wv[4];
            wv[5] = c2 * wv[4];
            c2 += dd;
#pragma unroll
            for (int e = 0; e < NH; ++e) {
                const double dn = fma(RS.lam, st.b[e], wv[e] + flip_sign(st.d[e], RS.m));
                st.b[e] = dn + flip_sign(st.b[e], RS.m);
                st.d[e] = dn;
            }
        }
    }
}

// The terms n2 = start, start + dir, ... (nc + nb + na of them, from the outer
// end of the row towards the anchor): the first nc with the degree-EXP_DEG_C
// exponential, the next nb with degree EXP_DEG_B, the rest with EXP_DEG_A.
template <int NH>
__device__ __forceinline__ void reinsch_run(RState<NH> &st, const BetaEntry *__restrict__ row, int start, int dir,
                                            int nc, int nb, int na, double a2, float c1sq, float a2f, float R2f,
                                            double z, const Reinsch &RS, const double2 *__restrict__ T, int j0, int jmax)
{
    int n2 = start;
    float c2f = a2f + (float)start;
    double c2 = a2 + start;
    reinsch_seg<NH, EXP_DEG_C>(st, row, n2, nc, dir, c2f, c2, c1sq, R2f, z, RS, T, j0, jmax);
    reinsch_seg<NH, EXP_DEG_B>(st, row, n2, nb, dir, c2f, c2, c1sq, R2f, z, RS, T, j0, jmax);
    reinsch_seg<NH, EXP_DEG_A>(st, row, n2, na, dir, c2f, c2, c1sq, R2f, z, RS, T, j0, jmax);
}

// Helmholtz rows: the first nff terms (the outer ones, all in the float-float
// band) in float-float, the state then carried over to double for the
// remaining nd terms (all within e^{-FF_GAP} of the largest term, where the
// degree-EXP_DEG_A exponential is exact to double precision).
__device__ __forceinline__ void reinsch_run_ff(RState<1> &st, const BetaEntry *__restrict__ row, int start, int dir,
                                               int nff, int nd, float c1sq, float a2f, float R2f, double z, FF zff,
                                               const Reinsch &RS, FF lamff, float sf, const double2 *__restrict__ T,
                                               int j0, int jmax)
{
    int n2 = start;
    float c2f = a2f + (float)start;
    double c2 = 0.0;  // not used by single sums
    if (nff > 0) {
        RStateFF f{0.f, 0.f, 0.f, 0.f};
        reinsch_seg_ff(f, row, n2, nff, dir, c2f, c1sq, R2f, zff, lamff, sf,
                       reinterpret_cast<const float4 *>(T + (jmax + 1)), j0, jmax);
        st.d[0] = f2d_exact(f.dh) + f2d_exact(f.dl);
        st.b[0] = f2d_exact(f.bh) + f2d_exact(f.bl);
    }
    reinsch_seg<1, EXP_DEG_A>(st, row, n2, nd, dir, c2f, c2, c1sq, R2f, z, RS, T, j0, jmax);
}

// One recurrence step with zero weight (recurrence index 0 of a sum whose
// index-0 term belongs to another sum).
template <int NH>
__device__ __forceinline__ void reinsch_zero(RState<NH> &st, const Reinsch &RS)
{
#pragma unroll
    for (int e = 0; e < NH; ++e) {
        const double dn = fma(RS.lam, st.b[e], flip_sign(st.d[e], RS.m));
        st.b[e] = dn + flip_sign(st.b[e], RS.m);
        st.d[e] = dn;
    }
}

// sin x and cos x in float for |x| < 6000, by Cody and Waite's reduction
// (Software Manual for the Elementary Functions, 1980): r = x - q pi/2 with
// pi/2 in three parts (the first two of 12 significant bits, so q times each
// is exact for |q| <= 4096), |r| <= pi/4, then the Taylor polynomials of sin
// (to r^9, truncation < 2e-9) and cos (to r^10, < 2e-10) at 0 and the quadrant
// q mod 4.  Error about 1.5 ulp; float arithmetic only (no FP64-pipe
// conversion, no MUFU).
__device__ __forceinline__ void sincos_cw(float x, float &s, float &c)
{
    const float qm = fmaf(x, 0.636619772f, 12582912.0f);  // rint(2x/pi) + 1.5 * 2^23
    const int q = __float_as_int(qm) - 0x4B400000;
    const float qf = qm - 12582912.0f;
    float r = fmaf(-qf, 1.5703125f, x);
    r = fmaf(-qf, 4.837512969970703e-4f, r);
    r = fmaf(-qf, 7.549790126404332e-8f, r);
    const float r2 = r * r;
    float ps = fmaf(r2, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = fmaf(ps, r2, 1.0f / 120.0f);
    ps = fmaf(ps, r2, -1.0f / 6.0f);
    const float sr = fmaf(ps * r2, r, r);
    float pc = fmaf(r2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = fmaf(pc, r2, -1.0f / 720.0f);
    pc = fmaf(pc, r2, 1.0f / 24.0f);
    pc = fmaf(pc, r2, -0.5f);
    const float cr = fmaf(pc, r2, 1.0f);
    const bool odd = (q & 1) != 0;
    const float ss = odd ? cr : sr, cc = odd ? sr : cr;
    s = (q & 2) ? -ss : ss;
    c = ((q + 1) & 2) ? -cc : cc;
}

// e^{i m t2} in float for an integer |m| < 2^11, with no double arithmetic:
// t2 = th + tl with th of 12 significant bits (m th exact in float), the
// product reduced by 2 pi = C1 + C2 + C3 (C1 of 8 bits, so k C1 is exact).
struct PhaseF {
    float th, tl;
};

__device__ __forceinline__ PhaseF phase_split(double t2)
{
    PhaseF P;
    P.th = __int_as_float(__float_as_int((float)t2) & (int)0xFFFFF800);
    P.tl = (float)(t2 - (double)P.th);
    return P;
}

__device__ __forceinline__ void phase_m(const PhaseF &P, int m, float &s, float &c)
{
    const float mf = (float)m;
    const float x = mf * P.th;
    const float kq = rintf(x * 0.15915494f);
    float r = fmaf(-kq, 6.28125f, x);
    r = fmaf(-kq, 1.9353071693331003e-3f, r);
    r = fmaf(-kq, 1.0253131677018246e-11f, r);
    r = fmaf(mf, P.tl, r);
    sincos_cw(r, s, c);
}

// Row sums combined into the outputs with the row's real factors (c1 fixed):
// G: A; xx: (1 - c1^2/k^2) A; yy: A - C/k^2; zz: A + D/k^2; xy: -(c1/k^2) B;
// xz: -(c1/k^2) E (real factor); yz: -(1/k^2) F (real factor).
template <int NH, typename F>
__device__ __forceinline__ void add_row(F S[][2], const F rr[][2], F c1, F ik2)
{
    if (NH == 1) {
        S[0][0] += rr[0][0];
        S[0][1] += rr[0][1];
    } else {
        const F fxx = (F)1 - c1 * c1 * ik2;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            S[0][q] += rr[0][q];
            S[1][q] += fxx * rr[0][q];
            S[2][q] += rr[0][q] - ik2 * rr[2][q];
            S[3][q] += rr[0][q] + ik2 * rr[3][q];
            S[4][q] += -c1 * ik2 * rr[1][q];
            S[5][q] += -c1 * ik2 * rr[4][q];
            S[6][q] += -ik2 * rr[5][q];
        }
    }
}

// The same segment sums in float (hardware ex2 and rsqrt), for the
// exponentially small tail of a double-precision plan:
// sum_{n2=lo}^{hi} w(n2) v^{n2-lo}, v = e^{i t2}.  b and 1/b come from the
// lattice index itself (b^2 = c1^2 + c2^2 - k^2, one rsqrt), so the loop loads
// nothing; in float b is good to ~1e-7 relative, e^{-b|x3|} to ~4e-6 for
// b|x3| <= 40, well inside the tail's error budget.  The terms go in groups of
// four aligned at lo, by Horner's rule in v^4 from the top group down: each
// group adds w0 + w1 v + w2 v^2 + w3 v^3 (powers formed once per target), so
// the dependent chain is one complex multiply-add per four terms and the four
// weights are independent work.
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// weights of one index: q0 = c1^2 - k^2, zl2 = |x3| log2(e); propagating n
// (b^2 <= 0) get weight 0.  No per-lane truncation test: the terms of the
// warp's disk beyond the lane's own set are below e^{-T} of its largest term
// (they add accuracy).
template <int NH>
__device__ __forceinline__ void tail_weights(float c2, float q0, float zl2, float wv[NH])
{
    const float x = fmaf(c2, c2, q0);
    const bool ev = x > 0.f;
    const float ib = rsqrt_approx(ev ? x : 1.f);
    const float b = x * ib;
    const float e = ev ? ex2_approx(-b * zl2) : 0.f;
    wv[0] = e * ib;
    if (NH > 1) {
        wv[1] = c2 * wv[0];
        wv[2] = c2 * wv[1];
        wv[3] = b * e;
        wv[4] = e;
        wv[5] = c2 * e;
    }
}

// Powers v, v^2, v^3, v^4 of v = (cv, sv).
struct VPow {
    float x[4], y[4];
};

__device__ __forceinline__ VPow vpowers(float cv, float sv)
{
    VPow P;
    P.x[0] = cv;
    P.y[0] = sv;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        P.x[k] = P.x[k - 1] * cv - P.y[k - 1] * sv;
        P.y[k] = P.x[k - 1] * sv + P.y[k - 1] * cv;
    }
    return P;
}

// One group n0 .. n0+3 (GUARD: indices above hi weigh zero): acc = acc v^4 +
// sum_t w(n0 + t) v^t.
template <int NH, bool GUARD>
__device__ __forceinline__ void horner_group_f32(int n0, int hi, float a2f, float q0, float zl2, const VPow &V,
                                                 float acc[NH][2])
{
    float w[4][NH];
    const float cb = a2f + (float)n0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        tail_weights<NH>(cb + (float)t, q0, zl2, w[t]);
        if (GUARD && n0 + t > hi) {
#pragma unroll
            for (int e = 0; e < NH; ++e) w[t][e] = 0.f;
        }
    }
#pragma unroll
    for (int e = 0; e < NH; ++e) {
        const float cx = fmaf(w[3][e], V.x[2], fmaf(w[2][e], V.x[1], fmaf(w[1][e], V.x[0], w[0][e])));
        const float cy = fmaf(w[3][e], V.y[2], fmaf(w[2][e], V.y[1], w[1][e] * V.y[0]));
        const float nx = fmaf(acc[e][0], V.x[3], fmaf(-acc[e][1], V.y[3], cx));
        const float ny = fmaf(acc[e][0], V.y[3], fmaf(acc[e][1], V.x[3], cy));
        acc[e][0] = nx;
        acc[e][1] = ny;
    }
}

template <int NH>
__device__ __forceinline__ void seg_horner_f32(int lo, int hi, float a2f, float q0, float zl2, const VPow &V,
                                               float acc[NH][2])
{
#pragma unroll
    for (int e = 0; e < NH; ++e) acc[e][0] = acc[e][1] = 0.f;
    const int g = (hi - lo + 4) >> 2;  // groups; the top one may pass hi
    if (g <= 0) return;
    horner_group_f32<NH, true>(lo + 4 * (g - 1), hi, a2f, q0, zl2, V, acc);
    for (int j = g - 2; j >= 0; --j) horner_group_f32<NH, false>(lo + 4 * j, hi, a2f, q0, zl2, V, acc);
}

// ---------------------------------------------------------------------------
// 3D far kernel for double-precision plans.  Series (he), and for Maxwell the
// second derivatives (each term times delta_pq - c^p c^q/k^2, c = (alpha_n,
// beta sgn x3)):
//   S = sum_n beta_n^{-1} e^{i beta_n |x3|} e^{i alpha_n . t},  G_d = e^{i2pi<alpha.m>} (i/8pi^2) S.
// Propagating n (|alpha_n| < k, a handful) are summed from a list.  For the
// evanescent n, beta = i b and 1/beta = -i/b; with w = e^{-bz}/b (real) the row
// n1 contributes -i sum_{n2} w e^{i(c1 t1 + c2 t2)}.  Every row is summed
// relative to the fixed anchor n2 = N0: the core outwards from N0 by two
// Reinsch recurrences, the float tails by Horner's rule in v = e^{i t2} from
// their first index, moved to N0 by a float phase.  The row phase e^{i c1 t1}
// follows a recurrence over the rows and e^{i(alpha_2 + N0) t2} is applied once
// per target.  Each lane keeps only its own truncation set
// |alpha_n|^2 <= k^2 + (T/z)^2.
//
// Precision, by term size (every term is at most e^{-(b - bmin) z} of the
// largest): the warp's core disk |alpha_n|^2 <= k^2 + (Y0/z_min)^2 (b z_min <=
// Y0 = 18, z_min the warp's smallest |x3|) is summed by the recurrences, its
// outer band (b >= bmin + FF_GAP/z_min, Helmholtz) in float-float and its inner
// terms in double with the table-driven exponential; the remaining terms, each
// below e^{-18} = 1.5e-8 of the leading ones and all together below
// 2 pi e^{-18}/z of the series scale, are summed in float (by far3d_tail, or
// here when TAILS): their float rounding (< 1e-5 relative) contributes < 2e-12
// of the series scale.
// ---------------------------------------------------------------------------
constexpr double FAR_CORE_Y0 = 18.0;

// Row slab `slab` of `nslab` of the rows of a chunk: the warp's core rows
// (|c1| <= sqrt(Rc2)) split evenly, the tail-only rows below and above the core
// joined to the first and the last slab.  Every row falls in exactly one slab.
__device__ __forceinline__ void slab_rows(int n1a, int n1b, float Rc2f, float a1f, int slab, int nslab, int &lo, int &hi)
{
    lo = n1a;
    hi = n1b;
    if (nslab <= 1) return;
    const float rcf = sqrtf(fmaxf(Rc2f, 0.f));
    const int k0 = max(n1a, (int)ceilf(-a1f - rcf)), k1 = min(n1b, (int)floorf(-a1f + rcf));
    const int Lc = max(k1 - k0 + 1, 0);
    if (slab > 0) lo = k0 + (slab * Lc) / nslab;
    if (slab < nslab - 1) hi = k0 + ((slab + 1) * Lc) / nslab - 1;
}

// The rows of a warp's far sums and their core segments.  The double-precision
// kernel and the float-tail kernel must split every row identically, so every
// operation here (and in far_lane) is explicitly rounded: no contraction can
// make the two kernels disagree on a term.
struct FarWarp {
    double izmax;      // 1/z_min over the warp's lanes
    float R2mf, Rc2f;  // truncation disk |alpha_n|^2 <= R2m (warp maximum) and core disk Rc2
    float a1f, a2f;
    float k2f, bff;    // k^2; the float-float band edge b >= bff = bmin + FF_GAP/z_min (Helmholtz)
    int n1a, n1b;      // rows of the truncation disk (one index of margin)
    int N0;            // anchor n2 = rint(-alpha_2)
};

__device__ __forceinline__ FarWarp far_warp(const EvalArgs &a, const FarLane &L)
{
    FarWarp W;
    const double R2m = warp_max(L.R2);
    W.izmax = warp_max(L.valid ? L.iz : 0.0);
    // core disk of the warp: b z_min <= Y0
    const double Rc2 = fmin(__dadd_rn(__dmul_rn(a.k, a.k), __dmul_rn(__dmul_rn(FAR_CORE_Y0 * FAR_CORE_Y0, W.izmax), W.izmax)), R2m);
    W.R2mf = __double2float_rn(R2m);
    W.Rc2f = __double2float_rn(Rc2);
    W.a1f = __double2float_rn(a.a1);
    W.a2f = __double2float_rn(a.a2);
    const float Rmf = __fsqrt_rn(W.R2mf);
    W.n1a = max(a.n1lo, (int)floorf(__fsub_rn(-W.a1f, Rmf)) - 1);
    W.n1b = min(a.n1hi, (int)ceilf(__fadd_rn(-W.a1f, Rmf)) + 1);
    W.N0 = (int)rint(-a.a2);
    W.k2f = __double2float_rn(__dmul_rn(a.k, a.k));
    W.bff = __double2float_rn(__fma_rn((double)FF_GAP, W.izmax, a.bmin));
    return W;
}

// Row n1 of the float-float band edge (Helmholtz): q^2 = bff^2 + k^2 - c1^2 raised
// by more than the float roundings of its parts (1e-5 of their sizes, and 1e-3),
// so that every term with |c2| >= sqrt(q^2) has b >= bff (below zero: the whole
// row lies in the band).
__device__ __forceinline__ float far_ff_q2(const FarWarp &W, float c1sq)
{
    const float qq = __fmaf_rn(W.bff, W.bff, W.k2f);
    return __fadd_rn(__fmaf_rn(1e-5f, __fadd_rn(qq, c1sq), 1e-3f), __fsub_rn(qq, c1sq));
}

// Row n1 of the warp's truncation disk: its index range [n2a, n2b] (false when
// the row is empty) and core segment [ca, cb] (ca > cb: no core), the core
// widened to contain N0.  Bounds are formed in float with a one-index margin:
// every lane still keeps exactly its own truncation set in the double sums, and
// the core/tail split only moves terms of size ~e^-18 between double and float.
__device__ __forceinline__ bool far_row(const FarWarp &W, const EvalArgs &a, int n1, float &c1f, float &c1sq, int &n2a,
                                        int &n2b, int &ca, int &cb)
{
    c1f = __fadd_rn(W.a1f, (float)n1);
    c1sq = __fmul_rn(c1f, c1f);
    const float remf = __fsub_rn(W.R2mf, c1sq);
    if (remf < -1.0f) return false;
    const float srf = __fsqrt_rn(fmaxf(remf, 0.f));
    n2a = max(a.n2lo, (int)floorf(__fsub_rn(-W.a2f, srf)) - 1);
    n2b = min(a.n2hi, (int)ceilf(__fadd_rn(-W.a2f, srf)) + 1);
    if (n2a > n2b) return false;
    ca = n2b + 1;
    cb = n2b;
    const float remc = __fsub_rn(W.Rc2f, c1sq);
    if (remc >= 0.f) {
        const float src = __fsqrt_rn(remc);
        ca = max(n2a, (int)ceilf(__fsub_rn(-W.a2f, src)));
        cb = min(n2b, (int)floorf(__fadd_rn(-W.a2f, src)));
        if (ca > cb) {
            ca = n2b + 1;
            cb = n2b;
        } else {
            ca = min(ca, W.N0);
            cb = max(cb, W.N0);
        }
    }
    return true;
}

// The float tails of row n1 (the segments outside its core, or the whole row
// when it has none), each by Horner's rule from its first index and moved to the
// anchor N0, rotated by the row phase A = e^{i c1 t1} and added into Sf.
template <int NH, int NS>
__device__ __forceinline__ void far_row_tails(int n2a, int n2b, int ca, int cb, int N0, float a2f, float c1f,
                                              float c1sq, float k2f, float zf, const VPow &V, const PhaseF &PF,
                                              float Ax, float Ay, float ik2f, float Sf[NS][2])
{
    const float q0 = c1sq - k2f, zl2 = zf * 1.44269504f;
    const int tl_hi = (ca <= cb) ? ca - 1 : n2b;
    const int th_lo = (ca <= cb) ? cb + 1 : n2b + 1;
    if (n2a > tl_hi && th_lo > n2b) return;
    float tf[NH][2];
#pragma unroll
    for (int e = 0; e < NH; ++e) tf[e][0] = tf[e][1] = 0.f;
    if (n2a <= tl_hi) {
        float acc[NH][2], ps, pc;
        seg_horner_f32<NH>(n2a, tl_hi, a2f, q0, zl2, V, acc);
        phase_m(PF, n2a - N0, ps, pc);
#pragma unroll
        for (int e = 0; e < NH; ++e) {
            tf[e][0] += pc * acc[e][0] - ps * acc[e][1];
            tf[e][1] += pc * acc[e][1] + ps * acc[e][0];
        }
    }
    if (th_lo <= n2b) {
        float acc[NH][2], ps, pc;
        seg_horner_f32<NH>(th_lo, n2b, a2f, q0, zl2, V, acc);
        phase_m(PF, th_lo - N0, ps, pc);
#pragma unroll
        for (int e = 0; e < NH; ++e) {
            tf[e][0] += pc * acc[e][0] - ps * acc[e][1];
            tf[e][1] += pc * acc[e][1] + ps * acc[e][0];
        }
    }
#pragma unroll
    for (int e = 0; e < NH; ++e) {
        const float x = tf[e][0], y = tf[e][1];
        tf[e][0] = Ax * x - Ay * y;
        tf[e][1] = Ax * y + Ay * x;
    }
    add_row<NH, float>(Sf, tf, c1f, ik2f);
}

// One warp, row slab `slab` of `nslab` of chunk w (32 consecutive entries of
// the sorted far list).  The slab's share of the series is added into the
// output entries, which the near pass set to zero; the propagating terms go
// with slab 0.  TAILS: the float tails are summed here too; otherwise the
// float-tail kernel (far3d_tail) adds them.
template <int NF, bool TAILS>
__device__ void far3d_f64_chunk(const EvalArgs &a, int w, int count, int slab, int nslab)
{
    constexpr int NH = NF == 1 ? 1 : 6;
    constexpr int NS = NF == 1 ? 1 : 7;
    const BetaEntry *tab = reinterpret_cast<const BetaEntry *>(a.btab);
    double2 *out = reinterpret_cast<double2 *>(a.out);
    const int ne = n_entries(a.which);
    const int W2 = a.n2hi - a.n2lo + 1;
    const int lane = threadIdx.x & 31;
    const double k2 = a.k * a.k, ik2 = 1.0 / k2;
    const float ik2f = (float)ik2;
    const double2 *T = a.exptab;
    const int jmax = a.exptab_n - 1, j0 = a.exptab_j0;
    const float a2f = (float)a.a2;
    {
        FarLane L = far_lane(a, w * 32 + lane, count);
        const FarWarp W = far_warp(a, L);
        const float R2f = (float)L.R2;
        const double izmax = W.izmax;
        // every row is summed from the anchor n2 = N0 outwards (the centre of all
        // rows' truncation intervals); e^{i(alpha_2 + N0) t2} multiplies the total
        const int N0 = W.N0;
        double sv, cv, s1, c1v;
        sincos(L.t2, &sv, &cv);
        sincos(L.t1, &s1, &c1v);
        const double2 E1 = make_double2(c1v, s1);
        const Reinsch RS = reinsch_lane(sv, cv);
        const PhaseF PF = phase_split(L.t2);
        // every term is at most e^{-(b - bmin) z_min} of the largest one (e^{-bz}/b
        // decreases in b): degree B from b >= bmin + EXP_GAP_B/z_min, C from
        // bmin + EXP_GAP_C/z_min
        const float b4 = (float)(a.bmin + EXP_GAP_B * izmax), b3 = (float)(a.bmin + EXP_GAP_C * izmax);
        // Helmholtz: the float-float band from b >= W.bff = bmin + FF_GAP/z_min
        const FF zff = ff_split(L.z), lamff = ff_split(RS.lam);
        const float sgn = RS.m ? -1.0f : 1.0f;
        const float k2f = (float)k2;
        const float svf = (float)sv, cvf = (float)cv, zf = (float)L.z;
        const VPow VP = vpowers(cvf, svf);
        double P[NF][2];
        double S[NS][2];
        float Sf[NS][2];
#pragma unroll
        for (int e = 0; e < NF; ++e) P[e][0] = P[e][1] = 0.0;
#pragma unroll
        for (int e = 0; e < NS; ++e) S[e][0] = S[e][1] = 0.0, Sf[e][0] = Sf[e][1] = 0.f;
        // propagating terms, in the anchor frame: e^{i(c1 t1 + (c2 - alpha_2 - N0) t2)};
        // the list is in row-major order, so within a row the phase steps by e^{i t2}.
        // e^{i beta z} = e^{i beta z_w} e^{i beta (z - z_w)}, z_w the warp's smallest
        // |x3|: the lanes share a narrow |x3| bucket, so the first factor is one sincos
        // per entry per warp (lane q mod 32 forms it, shuffles hand it out) and the
        // second a Taylor polynomial while |beta (z - z_w)| <= 0.02 (cos to theta^6,
        // sin to theta^7: truncation below 1e-17); a warp whose spread is wider takes
        // a sincos per lane.
        double2 ph = make_double2(1.0, 0.0);
        const int nq = slab == 0 ? *a.nprop : 0;
        const double zw = warp_min(L.valid ? L.z : 1e300);
        const double dz = L.z - zw;
        const bool taylor = nq > 0 && warp_max(L.valid ? dz : 0.0) * a.k <= 0.02;
        double ewx = 1.0, ewy = 0.0;  // e^{i beta_{q0 + lane} z_w} / beta_{q0 + lane}
        for (int q = 0; q < nq; ++q) {
            if (taylor && (q & 31) == 0) {
                if (q + lane < nq) {
                    const PropEntry &pl = a.prop[q + lane];
                    sincos(pl.br * zw, &ewy, &ewx);
                    ewx *= pl.ibr;
                    ewy *= pl.ibr;
                }
            }
            const PropEntry &pe = a.prop[q];
            if (pe.first) {
                double sp, cp;
                sincos(fma(pe.c1, L.t1, pe.m2 * L.t2), &sp, &cp);
                ph = make_double2(cp, sp);
            } else {
                ph = cmul(ph, make_double2(cv, sv));
            }
            // u = e^{i beta z} / beta
            double ux, uy;
            if (taylor) {
                const double Ex = __shfl_sync(0xffffffffu, ewx, q & 31), Ey = __shfl_sync(0xffffffffu, ewy, q & 31);
                const double th = pe.br * dz, th2 = th * th;
                const double ct = fma(fma(fma(th2, -1.0 / 720.0, 1.0 / 24.0), th2, -0.5), th2, 1.0);
                const double st = th * fma(fma(fma(th2, -1.0 / 5040.0, 1.0 / 120.0), th2, -1.0 / 6.0), th2, 1.0);
                ux = Ex * ct - Ey * st;
                uy = Ex * st + Ey * ct;
            } else {
                double sz, cz;
                sincos(pe.br * L.z, &sz, &cz);
                ux = pe.ibr * cz;
                uy = pe.ibr * sz;
            }
            const double cp = ph.x, sp = ph.y;
            if (NF == 1) {
                P[0][0] = fma(ux, cp, fma(-uy, sp, P[0][0]));
                P[0][1] = fma(ux, sp, fma(uy, cp, P[0][1]));
            }
            if (NF > 1) {
                const double tx = ux * cp - uy * sp, ty = ux * sp + uy * cp;
                P[0][0] += tx;
                P[0][1] += ty;
                double b3 = pe.br * L.sg;
                double f[6] = {1.0 - pe.c1 * pe.c1 * ik2, 1.0 - pe.c2 * pe.c2 * ik2, 1.0 - b3 * b3 * ik2,
                               -pe.c1 * pe.c2 * ik2, -pe.c1 * b3 * ik2, -pe.c2 * b3 * ik2};
#pragma unroll
                for (int e = 0; e < 6; ++e) {
                    P[1 + e][0] += f[e] * tx;
                    P[1 + e][1] += f[e] * ty;
                }
            }
        }
        int r_lo, r_hi;
        slab_rows(W.n1a, W.n1b, W.Rc2f, W.a1f, slab, nslab, r_lo, r_hi);
        if (!TAILS) {
            // only rows with a core segment: |c1| <= sqrt(Rc2), one row of margin
            const float rcf = sqrtf(fmaxf(W.Rc2f, 0.f));
            r_lo = max(r_lo, (int)ceilf(-W.a1f - rcf) - 1);
            r_hi = min(r_hi, (int)floorf(-W.a1f + rcf) + 1);
        }
        double2 A = make_double2(1.0, 0.0);  // e^{i c1 t1}
        // Helmholtz: Reinsch's closing step is linear in the state (d, b), so the
        // rows' final states, times the row phase A, are summed first and closed
        // once: DR, BR from the right sums (index n2 - N0 >= 0), DL, BL from the
        // left ones (index N0 - n2 >= 1, before their zero step)
        double2 DR = make_double2(0.0, 0.0), BR = DR, DL = DR, BL = DR;
        for (int n1 = r_lo; n1 <= r_hi; ++n1) {
            // row phase by recurrence, re-anchored every 16 rows
            if (((n1 - r_lo) & 15) == 0) {
                double sa, ca_;
                sincos((a.a1 + n1) * L.t1, &sa, &ca_);
                A = make_double2(ca_, sa);
            } else {
                A = cmul(A, E1);
            }
            // float tails fold into the double sums every 8 rows
            if (TAILS && ((n1 - r_lo) & 7) == 7) {
#pragma unroll
                for (int e = 0; e < NS; ++e) {
                    S[e][0] += f2d_exact(Sf[e][0]);
                    S[e][1] += f2d_exact(Sf[e][1]);
                    Sf[e][0] = Sf[e][1] = 0.f;
                }
            }
            float c1f, c1sq;
            int n2a, n2b, ca, cb;
            if (!far_row(W, a, n1, c1f, c1sq, n2a, n2b, ca, cb)) continue;
            const BetaEntry *row = tab + (size_t)(n1 - a.n1lo) * W2 - a.n2lo;
            if (ca <= cb) {
                // right: n2 = cb .. N0 (index n2 - N0); left: n2 = ca .. N0-1 (index
                // N0 - n2, e^{-i theta}) and a zero step for index 0
                RState<NH> R, Lt;
#pragma unroll
                for (int e = 0; e < NH; ++e) R.d[e] = R.b[e] = Lt.d[e] = Lt.b[e] = 0.0;
                // degree bands (Maxwell): |c2| >= q3 (degree C), >= q4 (degree B),
                // one index of margin; Helmholtz: |c2| >= qff (float-float, from
                // far_ff_q2: no term with b < bff leaves the double band, no margin)
                const float q3 = sqrtf(fmaxf(b3 * b3 + k2f - c1sq, 0.f)), q4 = sqrtf(fmaxf(b4 * b4 + k2f - c1sq, 0.f));
                const float qff = sqrtf(fmaxf(far_ff_q2(W, c1sq), 0.f));
                if (NH == 1) {
                    const int tot = cb - N0 + 1;
                    const int mff = max(0, cb - max((int)ceilf(qff - a2f), N0) + 1);
                    reinsch_run_ff(*reinterpret_cast<RState<1> *>(&R), row, cb, -1, mff, tot - mff, c1sq, a2f, R2f, L.z,
                                   zff, RS, lamff, sgn, T, j0, jmax);
                    DR.x = fma(A.x, R.d[0], DR.x);
                    DR.y = fma(A.y, R.d[0], DR.y);
                    BR.x = fma(A.x, R.b[0], BR.x);
                    BR.y = fma(A.y, R.b[0], BR.y);
                    if (ca < N0) {
                        const int mffl = max(0, min((int)floorf(-qff - a2f), N0 - 1) - ca + 1);
                        reinsch_run_ff(*reinterpret_cast<RState<1> *>(&Lt), row, ca, 1, mffl, N0 - ca - mffl, c1sq, a2f,
                                       R2f, L.z, zff, RS, lamff, sgn, T, j0, jmax);
                        DL.x = fma(A.x, Lt.d[0], DL.x);
                        DL.y = fma(A.y, Lt.d[0], DL.y);
                        BL.x = fma(A.x, Lt.b[0], BL.x);
                        BL.y = fma(A.y, Lt.b[0], BL.y);
                    }
                } else {
                    const int tot = cb - N0 + 1;
                    const int r3 = (int)ceilf(q3 - a2f) + 1, r4 = (int)ceilf(q4 - a2f) + 1;
                    const int m3 = max(0, cb - max(r3, N0) + 1);
                    const int m4 = max(0, min(cb - m3, cb) - max(r4, N0) + 1);
                    reinsch_run<NH>(R, row, cb, -1, m3, m4, tot - m3 - m4, a.a2, c1sq, a2f, R2f, L.z, RS, T, j0, jmax);
                    // Maxwell: each row closed and combined with its own factors in c1
                    double rr[NH][2];
#pragma unroll
                    for (int e = 0; e < NH; ++e) {
                        const double b1 = flip_sign(R.b[e] - R.d[e], RS.m);
                        rr[e][0] = fma(-RS.hlam, b1, R.d[e]);
                        rr[e][1] = b1 * RS.sv;
                    }
                    if (ca < N0) {
                        const int totl = N0 - ca;
                        const int l3 = (int)floorf(-q3 - a2f) - 1, l4 = (int)floorf(-q4 - a2f) - 1;
                        const int m3l = max(0, min(l3, N0 - 1) - ca + 1);
                        const int m4l = max(0, min(l4, N0 - 1) - (ca + m3l) + 1);
                        reinsch_run<NH>(Lt, row, ca, 1, m3l, m4l, totl - m3l - m4l, a.a2, c1sq, a2f, R2f, L.z, RS, T, j0,
                                        jmax);
                        reinsch_zero<NH>(Lt, RS);
#pragma unroll
                        for (int e = 0; e < NH; ++e) {
                            const double b1 = flip_sign(Lt.b[e] - Lt.d[e], RS.m);
                            rr[e][0] += fma(-RS.hlam, b1, Lt.d[e]);
                            rr[e][1] -= b1 * RS.sv;
                        }
                    }
#pragma unroll
                    for (int e = 0; e < NH; ++e) {
                        const double x = rr[e][0], y = rr[e][1];
                        rr[e][0] = A.x * x - A.y * y;
                        rr[e][1] = A.x * y + A.y * x;
                    }
                    add_row<NH, double>(S, rr, a.a1 + n1, ik2);
                }
            }
            // float tails [n2a, ca-1] and [cb+1, n2b] (the whole row when there is
            // no core)
            if (TAILS)
                far_row_tails<NH, NS>(n2a, n2b, ca, cb, N0, a2f, c1f, c1sq, k2f, zf, VP, PF, (float)A.x, (float)A.y,
                                      ik2f, Sf);
        }
        if (NH == 1) {
            // right: sum = D + U (-lambda/2 + i sin theta), U = s (B - D);
            // left, after the zero step: sum = s D + B (lambda/2 - i sin theta)
            const double ux = flip_sign(BR.x - DR.x, RS.m), uy = flip_sign(BR.y - DR.y, RS.m);
            S[0][0] += fma(-RS.hlam, ux, fma(-RS.sv, uy, DR.x));
            S[0][1] += fma(-RS.hlam, uy, fma(RS.sv, ux, DR.y));
            S[0][0] += fma(RS.hlam, BL.x, fma(RS.sv, BL.y, flip_sign(DL.x, RS.m)));
            S[0][1] += fma(RS.hlam, BL.y, fma(-RS.sv, BL.x, flip_sign(DL.y, RS.m)));
        }
        if (TAILS) {
#pragma unroll
            for (int e = 0; e < NS; ++e) {
                S[e][0] += f2d_exact(Sf[e][0]);
                S[e][1] += f2d_exact(Sf[e][1]);
            }
        }
        // back from the anchor frame with the lattice phase: one factor
        // e^{i(2 pi <alpha.m> + (alpha_2 + N0) t2)} (i/8pi^2)
        double ph2 = a.a1 * L.m1 + a.a2 * L.m2;
        ph2 -= rint(ph2);
        double sN, cN;
        sincos(fma(2.0 * GF_PI, ph2, (a.a2 + N0) * L.t2), &sN, &cN);
        const double2 pre = make_double2(-sN / (8.0 * GF_PI * GF_PI), cN / (8.0 * GF_PI * GF_PI));
        // evanescent sums carry the factor -i (from 1/beta = -i/b), except the
        // xz, yz entries whose factor (-i)(-i sgn) = -sgn is real
        constexpr int NE = NF == 1 ? 1 : 7;
        double2 vals[NE];
        if (NF == 1) {
            vals[0] = cmul(pre, make_double2(P[0][0] + S[0][1], P[0][1] - S[0][0]));
        } else {
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                const double *s = S[1 + e];
                double2 v;
                if (e < 4)
                    v = make_double2(P[1 + e][0] + s[1], P[1 + e][1] - s[0]);
                else
                    v = make_double2(P[1 + e][0] + L.sg * s[0], P[1 + e][1] + L.sg * s[1]);
                vals[e] = cmul(pre, v);
            }
            vals[NE - 1] = cmul(pre, make_double2(P[0][0] + S[0][1], P[0][1] - S[0][0]));
        }
        far_deposit(a, 0, w, slab, nslab, ((count + 31) >> 5) * 32, L.valid, L.idx, ne, vals);
        (void)out;
    }
}

// Far work items (a row slab of a chunk of 32 consecutive entries of the
// sorted list) are handed out one at a time from a counter, the most expensive
// chunks first: the list is in ascending bucket order and the bucket
// GF_FAR_BUCKETS c/|x3| grows as the target nears the slab, where the truncation
// disk (radius ~ T/|x3|) is largest, so the t-th item taken is slab t % S of
// chunk nch-1-t/S.  S (row slabs per chunk) is chosen so that there are about
// per_warp items per resident warp, which keeps the end of the launch short; the
// double-precision kernel asks for four, so that long lists keep one slab per
// chunk and its per-target set-up (double sines, divisions) is not repeated.
__device__ __forceinline__ int far_slabs(int nch, int smax, int per_warp = 8)
{
    const int nwarps = (int)(gridDim.x * blockDim.x) >> 5;
    if (nch <= 0) return 1;
    const int s = (per_warp * nwarps + nch - 1) / nch;
    return s < 1 ? 1 : s > smax ? smax : s;
}

__device__ __forceinline__ int far_take(int *counter, int nitems)
{
    int t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    return t < nitems ? t : -1;
}

template <int NF, bool TAILS>
__global__ void __launch_bounds__(128, NF == 1 ? 5 : 1) far3d_f64(EvalArgs a)
{
    const int count = a.far_count[0];
    const int nch = (count + 31) >> 5, S = far_slabs_capped(a, 0, nch, far_slabs(nch, 8));
    int *ctr = a.far_count + GF_WORK_SLOT;
    for (int t = far_take(ctr, nch * S); t >= 0; t = far_take(ctr, nch * S))
        far3d_f64_chunk<NF, TAILS>(a, nch - 1 - t / S, count, t % S, S);
}

// ---------------------------------------------------------------------------
// Float tails of a double-precision plan's far series, as a kernel of their
// own: the terms of each warp's truncation disk outside its core disk (the
// same chunks of the sorted far list and the same row split as far3d_f64, from
// far_warp and far_row), summed in float with the hardware ex2 and added into
// the double outputs.  Kept apart from the double sums so that the FP64 pipe is
// fed only by warps with double work, while these warps run on the FP32 and
// transcendental pipes.  The per-target set-up and the lattice phase are in
// double; the row phase e^{i c1 t1} = e^{i alpha_1 t1} e^{i n1 t1} in float.
// ---------------------------------------------------------------------------

template <int NF>
__device__ void far3d_tail_chunk(const EvalArgs &a, int w, int count, int slab, int nslab)
{
    constexpr int NH = NF == 1 ? 1 : 6;
    constexpr int NS = NF == 1 ? 1 : 7;
    double2 *out = reinterpret_cast<double2 *>(a.out);
    const int ne = n_entries(a.which);
    const int lane = threadIdx.x & 31;
    const float ik2f = (float)(1.0 / (a.k * a.k)), k2f = (float)(a.k * a.k);
    const FarLane L = far_lane(a, w * 32 + lane, count);
    const FarWarp W = far_warp(a, L);
    const int N0 = W.N0;
    const float zf = (float)L.z;
    float svf, cvf;
    sincos_cw((float)L.t2, svf, cvf);
    const VPow VP = vpowers(cvf, svf);
    const PhaseF P1 = phase_split(L.t1), P2 = phase_split(L.t2);
    // e^{i alpha_1 t1} in float (the tails are summed in float; this kernel
    // leaves the FP64 pipe to the double sums running beside it)
    float A0x, A0y;
    sincos_cw(W.a1f * (float)L.t1, A0y, A0x);
    double S[NS][2];
    float Sf[NS][2];
#pragma unroll
    for (int e = 0; e < NS; ++e) S[e][0] = S[e][1] = 0.0, Sf[e][0] = Sf[e][1] = 0.f;
    // the rows split evenly over the slabs
    const int nr = W.n1b - W.n1a + 1;
    const int r_lo = W.n1a + (slab * nr) / nslab, r_hi = W.n1a + ((slab + 1) * nr) / nslab - 1;
    for (int n1 = r_lo; n1 <= r_hi; ++n1) {
        if (((n1 - r_lo) & 7) == 7) {
#pragma unroll
            for (int e = 0; e < NS; ++e) {
                S[e][0] += f2d_exact(Sf[e][0]);
                S[e][1] += f2d_exact(Sf[e][1]);
                Sf[e][0] = Sf[e][1] = 0.f;
            }
        }
        float c1f, c1sq;
        int n2a, n2b, ca, cb;
        if (!far_row(W, a, n1, c1f, c1sq, n2a, n2b, ca, cb)) continue;
        float sn, cn;
        phase_m(P1, n1, sn, cn);
        far_row_tails<NH, NS>(n2a, n2b, ca, cb, N0, W.a2f, c1f, c1sq, k2f, zf, VP, P2, A0x * cn - A0y * sn,
                              A0x * sn + A0y * cn, ik2f, Sf);
    }
#pragma unroll
    for (int e = 0; e < NS; ++e) {
        S[e][0] += f2d_exact(Sf[e][0]);
        S[e][1] += f2d_exact(Sf[e][1]);
    }
    // the same lattice phase and factors as far3d_f64_chunk (no propagating
    // terms); the fractional part of <alpha.m> in double, its sine and cosine in
    // float
    double ph2 = a.a1 * L.m1 + a.a2 * L.m2;
    ph2 -= rint(ph2);
    float sNf, cNf;
    sincos_cw((float)fma(2.0 * GF_PI, ph2, (a.a2 + N0) * L.t2), sNf, cNf);
    constexpr double i8pi2 = 1.0 / (8.0 * GF_PI * GF_PI);
    const double2 pre = make_double2(-f2d_exact(sNf) * i8pi2, f2d_exact(cNf) * i8pi2);
    constexpr int NE = NF == 1 ? 1 : 7;
    double2 vals[NE];
    if (NF == 1) {
        vals[0] = cmul(pre, make_double2(S[0][1], -S[0][0]));
    } else {
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            const double *s = S[1 + e];
            const double2 v = e < 4 ? make_double2(s[1], -s[0]) : make_double2(L.sg * s[0], L.sg * s[1]);
            vals[e] = cmul(pre, v);
        }
        vals[NE - 1] = cmul(pre, make_double2(S[0][1], -S[0][0]));
    }
    far_deposit(a, 1, w, slab, nslab, ((count + 31) >> 5) * 32, L.valid, L.idx, ne, vals);
    (void)out;
}

template <int NF>
__global__ void __launch_bounds__(128) far3d_tail(EvalArgs a)
{
    const int count = a.far_count[0];
    const int nch = (count + 31) >> 5, S = far_slabs_capped(a, 1, nch, far_slabs(nch, 8));
    int *ctr = a.far_count + GF_TAIL_SLOT;
    for (int t = far_take(ctr, nch * S); t >= 0; t = far_take(ctr, nch * S))
        far3d_tail_chunk<NF>(a, nch - 1 - t / S, count, t % S, S);
}

// ---------------------------------------------------------------------------
// 3D far kernel, split precision: the same sums in float with the hardware
// ex2; the per-target cell reduction and the lattice phase's fractional part in
// double, everything else in float.
// ---------------------------------------------------------------------------
template <int NF>
__device__ void far3d_f32_chunk(const EvalArgs &a, int w, int count, int slab, int nslab)
{
    const BetaEntryF *tab = reinterpret_cast<const BetaEntryF *>(a.btab);
    float2 *out = reinterpret_cast<float2 *>(a.out);
    const int ne = n_entries(a.which);
    const int W2 = a.n2hi - a.n2lo + 1;
    const int lane = threadIdx.x & 31;
    const float ik2 = (float)(1.0 / (a.k * a.k));
    const float a2f = (float)a.a2;
    {
        // per-target set-up: the cell reduction in double, the rest in float
        const int slot = w * 32 + lane;
        const bool valid = slot < count;
        const int idx = valid ? a.far_sorted[slot] : 0;
        double x1 = 0, x2 = 0, x3 = 1;
        if (valid) {
            x1 = a.x[3 * (size_t)idx];
            x2 = a.x[3 * (size_t)idx + 1];
            x3 = a.x[3 * (size_t)idx + 2];
        }
        // cell reduction by a multiply and a floor: the series is the same for any
        // decomposition x = 2 pi m + t (e^{i alpha_n . x} = e^{i alpha_n . t}
        // e^{i 2 pi alpha . m}), so the exact cell decision of the near branch
        // is not needed here
        const double m1 = floor(fma(x1, INV_TWO_PI, 0.5)), m2 = floor(fma(x2, INV_TWO_PI, 0.5));
        const double t1d = fma(-TWO_PI, m1, x1), t2d = fma(-TWO_PI, m2, x2);
        const float z = fabsf((float)x3), t1 = (float)t1d, t2 = (float)t2d, sg = x3 >= 0.0 ? 1.f : -1.f;
        const float Tz = (float)a.T / z;
        const float R2f = valid ? (float)(a.k * a.k) + Tz * Tz : 0.f;
        float R2mf = R2f;
        for (int o = 16; o > 0; o >>= 1) R2mf = fmaxf(R2mf, __shfl_xor_sync(0xffffffffu, R2mf, o));
        float sv, cv;
        sincos_cw(t2, sv, cv);
        float P[NF][2];
        float S[NF == 1 ? 1 : 7][2];
#pragma unroll
        for (int e = 0; e < NF; ++e) P[e][0] = P[e][1] = 0.f;
#pragma unroll
        for (int e = 0; e < (NF == 1 ? 1 : 7); ++e) S[e][0] = S[e][1] = 0.f;
        for (int q = 0, nq = slab == 0 ? *a.nprop : 0; q < nq; ++q) {
            const PropEntry &pe = a.prop[q];
            const float br = pe.brf, ibr = pe.ibrf, c1 = pe.c1f, c2 = pe.c2f;
            float sz, cz, sp, cp;
            sincos_cw(br * z, sz, cz);
            sincos_cw(c1 * t1 + c2 * t2, sp, cp);
            float tx = ibr * (cz * cp - sz * sp), ty = ibr * (cz * sp + sz * cp);
            P[0][0] += tx;
            P[0][1] += ty;
            if (NF > 1) {
                float b3 = br * sg;
                float f[6] = {1.f - c1 * c1 * ik2, 1.f - c2 * c2 * ik2, 1.f - b3 * b3 * ik2,
                              -c1 * c2 * ik2, -c1 * b3 * ik2, -c2 * b3 * ik2};
#pragma unroll
                for (int e = 0; e < 6; ++e) {
                    P[1 + e][0] += f[e] * tx;
                    P[1 + e][1] += f[e] * ty;
                }
            }
        }
        // row bounds in float with a one-index margin
        const float a1f = (float)a.a1;
        const float Rmf = sqrtf(R2mf);
        const int n1a = max(a.n1lo, (int)floorf(-a1f - Rmf) - 1), n1b = min(a.n1hi, (int)ceilf(-a1f + Rmf) + 1);
        // row slab: the rows split evenly
        const int nr = n1b - n1a + 1;
        const int r_lo = n1a + (slab * nr) / nslab, r_hi = n1a + ((slab + 1) * nr) / nslab - 1;
        for (int n1 = r_lo; n1 <= r_hi; ++n1) {
            const float c1 = a1f + (float)n1;
            const float c1sq = c1 * c1;
            const float remf = R2mf - c1sq;
            if (remf < -1.0f) continue;
            const float srf = sqrtf(fmaxf(remf, 0.f));
            const int n2a = max(a.n2lo, (int)floorf(-a2f - srf) - 1), n2b = min(a.n2hi, (int)ceilf(-a2f + srf) + 1);
            if (n2a > n2b) continue;
            const BetaEntryF *row = tab + (size_t)(n1 - a.n1lo) * W2 - a.n2lo;
            float c2 = a2f + (float)n2b;
            float h[NF == 1 ? 1 : 6][2];
#pragma unroll
            for (int e = 0; e < (NF == 1 ? 1 : 6); ++e) h[e][0] = h[e][1] = 0.f;
            for (int n2 = n2b; n2 >= n2a; --n2, c2 -= 1.0f) {
                const BetaEntryF be = row[n2];
                // propagating n (summed separately) have bl2 = +inf, so e = 0; no
                // per-lane truncation test (terms beyond the lane's set are below e^{-T})
                const float e = ex2_approx(-be.bl2 * z);
                float wv[NF == 1 ? 1 : 6];
                if (NF == 1) {
                    wv[0] = e * be.ib;
                } else {
                    wv[0] = e * be.ib;
                    wv[1] = c2 * wv[0];
                    wv[2] = c2 * wv[1];
                    wv[3] = be.b * e;
                    wv[4] = e;
                    wv[5] = c2 * e;
                }
#pragma unroll
                for (int e2 = 0; e2 < (NF == 1 ? 1 : 6); ++e2) {
                    const float nx = fmaf(h[e2][0], cv, fmaf(-h[e2][1], sv, wv[e2]));
                    const float ny = fmaf(h[e2][0], sv, h[e2][1] * cv);
                    h[e2][0] = nx;
                    h[e2][1] = ny;
                }
            }
            float sp, cp;
            sincos_cw(c1 * t1 + (a2f + (float)n2a) * t2, sp, cp);
            float r[NF == 1 ? 1 : 6][2];
#pragma unroll
            for (int e2 = 0; e2 < (NF == 1 ? 1 : 6); ++e2) {
                r[e2][0] = cp * h[e2][0] - sp * h[e2][1];
                r[e2][1] = cp * h[e2][1] + sp * h[e2][0];
            }
            if (NF == 1) {
                S[0][0] += r[0][0];
                S[0][1] += r[0][1];
            } else {
                const float fxx = 1.f - c1 * c1 * ik2;
                S[0][0] += r[0][0];
                S[0][1] += r[0][1];
                S[1][0] += fxx * r[0][0];
                S[1][1] += fxx * r[0][1];
                S[2][0] += r[0][0] - ik2 * r[2][0];
                S[2][1] += r[0][1] - ik2 * r[2][1];
                S[3][0] += r[0][0] + ik2 * r[3][0];
                S[3][1] += r[0][1] + ik2 * r[3][1];
                S[4][0] += -c1 * ik2 * r[1][0];
                S[4][1] += -c1 * ik2 * r[1][1];
                S[5][0] += -c1 * ik2 * r[4][0];
                S[5][1] += -c1 * ik2 * r[4][1];
                S[6][0] += -ik2 * r[5][0];
                S[6][1] += -ik2 * r[5][1];
            }
        }
        // e^{i 2pi <alpha.m>} (i/8pi^2): the fractional part in double, the phase in float
        double ph = a.a1 * m1 + a.a2 * m2;
        ph -= rint(ph);
        float sl, cl;
        sincospif(2.0f * (float)ph, &sl, &cl);
        const float sc = (float)(1.0 / (8.0 * GF_PI * GF_PI));
        const float2 pre = make_float2(-sl * sc, cl * sc);
        constexpr int NE = NF == 1 ? 1 : 7;
        float2 vals[NE];
        if (NF == 1) {
            vals[0] = cmulf(pre, make_float2(P[0][0] + S[0][1], P[0][1] - S[0][0]));
        } else {
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                const float *s = S[1 + e];
                float2 v;
                if (e < 4)
                    v = make_float2(P[1 + e][0] + s[1], P[1 + e][1] - s[0]);
                else
                    v = make_float2(P[1 + e][0] + sg * s[0], P[1 + e][1] + sg * s[1]);
                vals[e] = cmulf(pre, v);
            }
            vals[NE - 1] = cmulf(pre, make_float2(P[0][0] + S[0][1], P[0][1] - S[0][0]));
        }
        far_deposit(a, 0, w, slab, nslab, ((count + 31) >> 5) * 32, valid, idx, ne, vals);
        (void)out;
    }
}

template <int NF>
__global__ void __launch_bounds__(128) far3d_f32(EvalArgs a)
{
    const int count = a.far_count[0];
    const int nch = (count + 31) >> 5, S = far_slabs_capped(a, 0, nch, far_slabs(nch, 4));
    int *ctr = a.far_count + GF_WORK_SLOT;
    for (int t = far_take(ctr, nch * S); t >= 0; t = far_take(ctr, nch * S))
        far3d_f32_chunk<NF>(a, nch - 1 - t / S, count, t % S, S);
}

// Batched far kernel: one persistent launch for all pairs.  The work items of
// all pairs form one global list (pair after pair, each pair's chunks most
// expensive first, S row slabs per chunk with S from the total chunk count)
// handed out from pair 0's work counter, so no pair waits for another and the
// load stays balanced across pair boundaries.  The taken index only grows, so
// each warp walks the pair list forward.
template <typename R, int NF>
__global__ void far3d_batch(const EvalArgs *args, int np)
{
    if (np <= 0) return;
    int tot = 0;
    for (int q = 0; q < np; ++q) tot += (args[q].far_count[0] + 31) >> 5;
    const int S = far_slabs(tot, sizeof(R) == 8 ? 8 : 4);
    int *ctr = args[0].far_count + GF_WORK_SLOT;
    int p = 0, base = 0;
    int count = args[0].far_count[0];
    int nit = ((count + 31) >> 5) * S;
    for (;;) {
        int t = 0;
        if ((threadIdx.x & 31) == 0) t = atomicAdd(ctr, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        while (p < np && t >= base + nit) {
            base += nit;
            if (++p < np) {
                count = args[p].far_count[0];
                nit = ((count + 31) >> 5) * S;
            }
        }
        if (p >= np) return;
        const int u = t - base, nch = nit / S;
        if (sizeof(R) == 8)
            far3d_f64_chunk<NF, true>(args[p], nch - 1 - u / S, count, u % S, S);
        else
            far3d_f32_chunk<NF>(args[p], nch - 1 - u / S, count, u % S, S);
    }
}

// ---------------------------------------------------------------------------
// 2D far kernel: G = e^{i2pi alpha m} (i/4pi) sum_n beta_n^{-1} e^{i alpha_n t + i beta_n |x2|}
// (terms and sums in double for both precisions).  One warp per target: lane l
// takes n = na + l, na + l + 32, ... (phase e^{i alpha_n t} from a sincos and the
// step e^{i 32 t}), and the lanes' sums are added by shuffles.
// ---------------------------------------------------------------------------
// Term n of (ei) without its factor i/(4pi): beta_n, E_n = e^{i alpha_n t + i beta_n
// |x2|} (p = e^{i alpha_n t} given) and E_n / beta_n (beta_n = b or i b, so the
// quotient is E/b or -i E/b).
__device__ __forceinline__ void ei_term(double kk, double aa, double z, double2 p, double2 &beta, double2 &E,
                                        double2 &term)
{
    if (aa <= kk) {
        const double b = sqrt((kk - aa) * (kk + aa)), ib = 1.0 / b;
        double sz, cz;
        sincos(b * z, &sz, &cz);
        beta = make_double2(b, 0.0);
        E = cmul(make_double2(cz, sz), p);
        term = make_double2(E.x * ib, E.y * ib);
    } else {
        const double b = sqrt((aa - kk) * (aa + kk)), ib = 1.0 / b;
        beta = make_double2(0.0, b);
        E = cscale(p, exp(-b * z));
        term = make_double2(E.y * ib, -E.x * ib);
    }
}

// 2D far branch (|x2| > c): (ei) summed by one warp per target, lanes over n.
// GF_OUT_GRAD adds the term-by-term derivatives (i alpha_n/beta_n) E_n and
// i sgn(x2) E_n; GF_OUT_HESSDIFF sums, over the indices of both wave numbers'
// truncation sets, -alpha_n^2 (E_n/beta_n - E'_n/beta'_n), -alpha_n sgn (E_n - E'_n)
// and -(beta_n E_n - beta'_n E'_n) (primes: k2).
// OUT: the output kind (GF_OUT_G, GF_OUT_GRAD or GF_OUT_HESSDIFF), one kernel
// instance each so that the plain G sum carries none of the others' registers.
template <typename R, int OUT>
__global__ void __launch_bounds__(128) far2d(EvalArgs a)
{
    typedef typename cplx_t<R>::T C;
    C *out = reinterpret_cast<C *>(a.out);
    const int count = *a.far_count;
    constexpr int ne = OUT == GF_OUT_G ? 1 : 3;
    constexpr bool hess = OUT == GF_OUT_HESSDIFF, grad = OUT == GF_OUT_GRAD;
    const double kmax = (hess && a.k2 > a.k) ? a.k2 : a.k;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int slot = gw; slot < count; slot += nw) {
        const int idx = a.far_idx[slot];
        const double x1 = a.x[2 * (size_t)idx], x2 = a.x[2 * (size_t)idx + 1];
        double t, m;
        reduce_period(x1, t, m);
        const double z = fabs(x2), sg = x2 >= 0.0 ? 1.0 : -1.0;
        const double Tz = a.T * (1.0 / z);
        const double R2 = kmax * kmax + Tz * Tz, Rr = sqrt(R2);
        const int na = (int)floor(-a.a1 - Rr) - 1, nb = (int)ceil(-a.a1 + Rr) + 1;
        double sp, cp, s32, c32;
        sincos((a.a1 + (na + lane)) * t, &sp, &cp);
        sincos(32.0 * t, &s32, &c32);
        double2 p = make_double2(cp, sp);
        const double2 step = make_double2(c32, s32);
        double acc[ne][2];
#pragma unroll
        for (int e = 0; e < ne; ++e) acc[e][0] = acc[e][1] = 0.0;
        for (int n = na + lane; n <= nb; n += 32, p = cmul(p, step)) {
            const double c1 = a.a1 + n;
            if (c1 * c1 > R2) continue;
            const double aa = fabs(c1);
            double2 beta, E, term;
            ei_term(a.k, aa, z, p, beta, E, term);
            if constexpr (!hess) {
                acc[0][0] += term.x;
                acc[0][1] += term.y;
                if constexpr (grad) {
                    acc[1][0] -= c1 * term.y;  // i c1 term
                    acc[1][1] += c1 * term.x;
                    acc[2][0] -= sg * E.y;     // i sgn E
                    acc[2][1] += sg * E.x;
                }
            } else {
                double2 beta2, E2, term2;
                ei_term(a.k2, aa, z, p, beta2, E2, term2);
                const double2 d0 = csub(term, term2), d1 = csub(E, E2);
                const double2 d2 = csub(cmul(beta, E), cmul(beta2, E2));
                acc[0][0] -= c1 * c1 * d0.x;
                acc[0][1] -= c1 * c1 * d0.y;
                acc[1][0] -= c1 * sg * d1.x;
                acc[1][1] -= c1 * sg * d1.y;
                acc[2][0] -= d2.x;
                acc[2][1] -= d2.y;
            }
        }
#pragma unroll
        for (int e = 0; e < ne; ++e)
            for (int o = 16; o > 0; o >>= 1) {
                acc[e][0] += __shfl_xor_sync(0xffffffffu, acc[e][0], o);
                acc[e][1] += __shfl_xor_sync(0xffffffffu, acc[e][1], o);
            }
        if (lane == 0) {
            const double2 lat = lattice_phase(a.a1, m, 0.0, 0.0);
            const double2 pre = cmul(lat, make_double2(0.0, 0.25 / GF_PI));
            for (int e = 0; e < ne; ++e)
                store_out(out + (size_t)idx * ne + e, cmul(pre, make_double2(acc[e][0], acc[e][1])));
        }
    }
}

// Persistent far grid: as many 128-thread CTAs as are resident at once (a
// grid beyond that would leave the extra CTAs waiting for a second wave).
template <void (*K)(EvalArgs)>
int resident_grid(int nsm)
{
    static const int per = [] {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, K, 128, 0) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        return v;
    }();
    return per * nsm;
}

// Concurrent far kernels of a Helmholtz double-precision plan: the double
// kernel gives up FAR_F64_DROP of its resident CTAs per SM, and the float-tail
// kernel (64-thread CTAs) fills the registers left free, so that both run at
// once on every SM.
constexpr int FAR_F64_DROP = 1;

struct FarShare {
    int f64, tail;  // resident CTAs per SM of each kernel
};

FarShare far_share()
{
    FarShare sh{1, 1};
    int dev = 0, regs_sm = 65536, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes fa, ta;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, far3d_f64<1, false>, 128, 0) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, far3d_f64<1, false>) != cudaSuccess ||
        cudaFuncGetAttributes(&ta, far3d_tail<1>) != cudaSuccess) {
        cudaGetLastError();
        return sh;
    }
    // registers are allocated per warp in units of 8 per thread
    auto cta_regs = [](int regs, int threads) { return (regs + 7) / 8 * 8 * 32 * ((threads + 31) / 32); };
    sh.f64 = per > FAR_F64_DROP ? per - FAR_F64_DROP : 1;
    sh.tail = (regs_sm - sh.f64 * cta_regs(fa.numRegs, 128)) / cta_regs(ta.numRegs, 64);
    if (sh.tail < 1) sh.tail = 1;
    return sh;
}

// The double sums and float tails of a double-precision plan's far series.
// With a fork (Helmholtz only), the tails run on the side stream alongside the
// double kernel, with the resident CTAs split by far_share; otherwise (and for
// Maxwell plans, whose double kernel leaves too few registers) after it, at full
// occupancy.
template <int NF>
cudaError_t launch_far_f64(const EvalArgs &a, int nsm, cudaStream_t s, const EvalFork *fork)
{
    if (NF != 1) fork = nullptr;
    if (!fork) {
        far3d_f64<NF, false><<<resident_grid<far3d_f64<NF, false>>(nsm), 128, 0, s>>>(a);
        far3d_tail<NF><<<resident_grid<far3d_tail<NF>>(nsm), 128, 0, s>>>(a);
        return cudaSuccess;
    }
    static const FarShare sh = far_share();
    cudaError_t e;
    if ((e = cudaEventRecord(fork->fork, s)) != cudaSuccess || (e = cudaStreamWaitEvent(fork->aux, fork->fork, 0)) != cudaSuccess)
        return e;
    far3d_f64<NF, false><<<sh.f64 * nsm, 128, 0, s>>>(a);
    far3d_tail<NF><<<sh.tail * nsm, 64, 0, fork->aux>>>(a);
    if ((e = cudaEventRecord(fork->join, fork->aux)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(s, fork->join, 0);
}

// The far list, bucket-sorted: stable when the evaluation brought segment
// scratch, else from the appended list.
void launch_far_list(const EvalArgs &a, int nsm, cudaStream_t s)
{
    if (a.seghist) {
        const int blocks = (a.nseg + 7) / 8;
        far_seg_count<<<blocks, 256, 0, s>>>(a);
        far_seg_scan<<<GF_FAR_BUCKETS / 32, 1024, 0, s>>>(a);
        far_seg_scatter<<<blocks, 256, 0, s>>>(a);
    } else {
        far_scatter<<<nsm * 2, 256, 0, s>>>(a);
    }
}

template <typename R>
cudaError_t launch_eval_t(const EvalArgs &a, cudaStream_t s, cudaEvent_t ev_mid, const EvalFork *fork)
{
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (a.n + 255) / 256;
    if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
    if (blocks < 1) blocks = 1;
    if (a.dim == 2) {
        if (a.nf == 1)
            near2d<R, 1><<<(int)blocks, 256, 0, s>>>(a);
        else if (a.nf == 3)
            near2d<R, 3><<<(int)blocks, 256, 0, s>>>(a);
        else
            near2d<R, 6><<<(int)blocks, 256, 0, s>>>(a);
        if (ev_mid) cudaEventRecord(ev_mid, s);
        if (a.which == GF_OUT_GRAD)
            far2d<R, GF_OUT_GRAD><<<resident_grid<far2d<R, GF_OUT_GRAD>>(nsm), 128, 0, s>>>(a);
        else if (a.which == GF_OUT_HESSDIFF)
            far2d<R, GF_OUT_HESSDIFF><<<resident_grid<far2d<R, GF_OUT_HESSDIFF>>(nsm), 128, 0, s>>>(a);
        else
            far2d<R, GF_OUT_G><<<resident_grid<far2d<R, GF_OUT_G>>(nsm), 128, 0, s>>>(a);
    } else if (a.nf == 1) {
        // with a near list: classify, then the near targets in full warps
        if (a.near_idx) {
            near3d<R, 1, 1><<<(int)blocks, 256, 0, s>>>(a);
            near3d_list<R, 1><<<(int)blocks, 256, 0, s>>>(a);
        } else {
            near3d<R, 1><<<(int)blocks, 256, 0, s>>>(a);
        }
        if (ev_mid) cudaEventRecord(ev_mid, s);
        launch_far_list(a, nsm, s);
        if (sizeof(R) == 8) {
            cudaError_t e = launch_far_f64<1>(a, nsm, s, fork);
            if (e != cudaSuccess) return e;
        } else
            far3d_f32<1><<<resident_grid<far3d_f32<1>>(nsm), 128, 0, s>>>(a);
    } else {
        if (a.near_idx) {
            near3d<R, 7, 1><<<(int)blocks, 256, 0, s>>>(a);
            near3d_list<R, 7><<<(int)blocks, 256, 0, s>>>(a);
        } else {
            near3d<R, 7><<<(int)blocks, 256, 0, s>>>(a);
        }
        if (ev_mid) cudaEventRecord(ev_mid, s);
        launch_far_list(a, nsm, s);
        if (sizeof(R) == 8) {
            cudaError_t e = launch_far_f64<7>(a, nsm, s, fork);
            if (e != cudaSuccess) return e;
        } else
            far3d_f32<7><<<resident_grid<far3d_f32<7>>(nsm), 128, 0, s>>>(a);
    }
    gf_count_launch(a.dim == 2 ? 2 : (sizeof(R) == 8 ? 4 : 3) + (a.near_idx ? 1 : 0) + (a.seghist ? 2 : 0));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_eval_batch_t(const EvalBatch &b, cudaStream_t s)
{
    if (b.nf == 1) {
        if (b.near_lists) {
            // classification, then the near targets in full warps
            int per = 0, dev = 0, nsm = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, near3d_list_batch<R, 1>, 256, 0) != cudaSuccess ||
                per < 1) {
                cudaGetLastError();
                per = 1;
            }
            near3d_batch<R, 1, 1><<<b.grid_near, 256, 0, s>>>(b.args, b.prefix, b.np);
            near3d_list_batch<R, 1><<<per * nsm, 256, 0, s>>>(b.args, b.np);
            gf_count_launch(1);
        } else {
            near3d_batch<R, 1><<<b.grid_near, 256, 0, s>>>(b.args, b.prefix, b.np);
        }
        far_scatter_batch<<<b.grid_scatter, 256, 0, s>>>(b.args, b.np, b.scatter_per_pair);
        far3d_batch<R, 1><<<b.grid_far, b.block_far, 0, s>>>(b.args, b.np);
    } else {
        near3d_batch<R, 7><<<b.grid_near, 256, 0, s>>>(b.args, b.prefix, b.np);
        far_scatter_batch<<<b.grid_scatter, 256, 0, s>>>(b.args, b.np, b.scatter_per_pair);
        far3d_batch<R, 7><<<b.grid_far, b.block_far, 0, s>>>(b.args, b.np);
    }
    gf_count_launch(3);
    return cudaGetLastError();
}

}  // namespace

cudaError_t gf_launch_eval_batch(const EvalBatch &b, int precision, cudaStream_t s)
{
    return precision == GF_FP64 ? launch_eval_batch_t<double>(b, s) : launch_eval_batch_t<float>(b, s);
}

cudaError_t gf_launch_series_tables(const EvalArgs &a, int precision, double2 *exptab, PropEntry *prop, int *nprop,
                                    const int pbox[4], cudaStream_t s)
{
    const int4 pb = make_int4(pbox[0], pbox[1], pbox[2], pbox[3]);
    if (precision == GF_FP64)
        series_tables<BetaEntry><<<256, 256, 0, s>>>(a, (BetaEntry *)const_cast<void *>(a.btab), exptab, prop, nprop, pb);
    else
        series_tables<BetaEntryF><<<256, 256, 0, s>>>(a, (BetaEntryF *)const_cast<void *>(a.btab), exptab, prop, nprop, pb);
    gf_count_launch(1);
    return cudaGetLastError();
}

cudaError_t gf_launch_eval(const EvalArgs &a, int precision, cudaStream_t s, cudaEvent_t ev_mid, const EvalFork *fork)
{
    return precision == GF_FP64 ? launch_eval_t<double>(a, s, ev_mid, fork) : launch_eval_t<float>(a, s, ev_mid, fork);
}
