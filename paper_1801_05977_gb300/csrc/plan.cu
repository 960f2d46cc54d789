// Host side of the C ABI (include/gf.h): argument checks, the Wood and
// resonance checks of Secs. 1, 2.1 and 3.1, the small host tables (Gauss
// nodes and cutoff weights), device memory, and the launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "gf_internal.cuh"

namespace {

thread_local char g_err[512] = "";
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_timing{0};

gf_status fail(gf_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? GF_ERR_NOMEM : GF_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
    } while (0)

bool pow2_in(int m, int lo, int hi) { return m >= lo && m <= hi && (m & (m - 1)) == 0; }

// Gauss-Legendre nodes/weights on [-1, 1]: Newton iteration on P_Q from the
// Chebyshev-like first guess, P_Q and P_Q' by the Bonnet recurrence (two more
// steps once the update is at rounding level).  Computed once per Q.
void gauss_legendre_compute(int Q, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(Q, 0.0);
    w.assign(Q, 0.0);
    for (int i = 0; i < (Q + 1) / 2; ++i) {
        double z = cos(GF_PI * (4.0 * i + 3.0) / (4.0 * Q + 2.0));
        double pd = 1.0;
        for (int it = 0, extra = 0; it < 100 && extra < 2; ++it) {
            double pm = 1.0, pc = z;
            for (int n = 1; n < Q; ++n) {
                double pn = ((2 * n + 1) * z * pc - n * pm) / (n + 1);
                pm = pc;
                pc = pn;
            }
            pd = Q * (pm - z * pc) / (1.0 - z * z);
            double dz = pc / pd;
            z -= dz;
            if (fabs(dz) <= 1e-15) ++extra;
        }
        double pm = 1.0, pc = z;
        for (int n = 1; n < Q; ++n) {
            double pn = ((2 * n + 1) * z * pc - n * pm) / (n + 1);
            pm = pc;
            pc = pn;
        }
        pd = Q * (pm - z * pc) / (1.0 - z * z);
        double wt = 2.0 / ((1.0 - z * z) * pd * pd);
        x[i] = -z;
        x[Q - 1 - i] = z;
        w[i] = wt;
        w[Q - 1 - i] = wt;
    }
}

std::mutex g_gl_mu;
std::map<int, std::pair<std::vector<double>, std::vector<double>>> g_gl;

void gauss_legendre(int Q, std::vector<double> &x, std::vector<double> &w)
{
    std::lock_guard<std::mutex> lk(g_gl_mu);
    auto it = g_gl.find(Q);
    if (it == g_gl.end()) {
        std::vector<double> xx, ww;
        gauss_legendre_compute(Q, xx, ww);
        it = g_gl.emplace(Q, std::make_pair(std::move(xx), std::move(ww))).first;
    }
    x = it->second.first;
    w = it->second.second;
}

double chi_d1(double t, double c, double ct)
{
    double w = 0.5 * (ct - c);
    return -smooth8_d1((t - c) / w) / w;
}
double yps0(double r, double eps) { return 1.0 - smooth8((r - eps) / eps); }
double yps1(double r, double eps) { return -smooth8_d1((r - eps) / eps) / eps; }
double yps2(double r, double eps) { return -smooth8_d2((r - eps) / eps) / (eps * eps); }

}  // namespace

struct gf_plan_s {
    int dim = 3, M[3] = {1, 1, 1}, nf = 1, precision = GF_FP64, kind = GF_HELMHOLTZ;
    double k = 1, alpha[2] = {0, 0};
    gf_trunc_t tr{};
    double T = 0;
    int P1 = 1, P2 = 1, P3 = 1;
    int Q3lo = 0, a3first = 0, L3count = 1;  // stored x3 planes of the gather grid (3D)
    int nyq = 0;                      // Maxwell half grid: odd fields' Nyquist planes in nyqgrid
    void *nyqgrid = nullptr;          // [P2][P1][2] complex
    // far-region grid (far_grid_M > 0): [fNZ][fM + 3][fM + 3][nf], plane m at z = fz0 + m fhz
    void *fargrid = nullptr;
    size_t far_bytes = 0;
    int *errw = nullptr;              // device error word of the synthesis (bounded waits)
    int fM = 0, fNZ = 0;
    double fz0 = 0, fhz = 0, fzmax = 0;
    size_t elem = 16;                 // bytes per complex value
    void *grid = nullptr;             // padded gather grid
    size_t grid_bytes = 0;
    void *tables = nullptr;           // synthesis tables
    void *btab = nullptr;             // far-series beta table
    PropEntry *prop = nullptr;        // propagating indices, then their count
    int *nprop_dev = nullptr;
    cudaStream_t stream = nullptr;    // stream of the plan's creation
    double2 *exptab = nullptr;        // (e^{-y_j}, y_j), y_j = (j - exptab_j0)/GF_EXPTAB_STEPS, then a float4 copy
    int exptab_n = 0, exptab_j0 = 0;
    double bmin_ev = 1e300;           // smallest evanescent |beta_n|
    int n1lo = 0, n1hi = -1, n2lo = 0, n2hi = -1;
    SynthArgs sa{};
    // Launch lock: serialises the host-side enqueue of concurrent calls on this
    // plan (the fork/join event pair and the phase-timing events are recorded
    // under it).  Device memory of an evaluation is per call, so the plan itself
    // is never modified after gf_plan.
    std::mutex mu;
    // phase timing: [0] synth start, [1] synth end, [2] table end, [3] near start, [4] near end, [5] far end
    bool timing = false;
    cudaEvent_t ev[6] = {};
    bool ev_plan = false, ev_eval = false;
    // fork/join events of the concurrent far kernels (3D double-precision plans)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

void gf_count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" {

int64_t gf_launch_count(void) { return g_launches.load(); }

const char *gf_last_error(void) { return g_err; }

const char *gf_status_string(gf_status s)
{
    switch (s) {
    case GF_OK: return "ok";
    case GF_ERR_ARG: return "invalid argument";
    case GF_ERR_WOOD: return "Wood anomaly: some beta_n vanishes";
    case GF_ERR_RESONANCE: return "resonance: beta = +-j pi / c~ for some j";
    case GF_ERR_NOMEM: return "out of device memory";
    case GF_ERR_CUDA: return "CUDA error";
    case GF_ERR_TIMEOUT: return "device wait timed out";
    case GF_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

gf_status gf_trunc_default(gf_trunc_t *t)
{
    if (!t) return fail(GF_ERR_ARG, "gf_trunc_default: NULL");
    t->c = 0.6;
    t->c_tilde = 1.0;
    t->eps = 0.45;
    t->series_tol = 0.0;
    t->quad_nodes = 0;
    t->precision = GF_FP64;
    t->kind = GF_HELMHOLTZ;
    t->resonance_policy = GF_PERTURB_CTILDE;
    t->far_grid_M = 0;
    t->far_grid_nz = 0;
    t->far_grid_zmax = 0.0;
    t->k2 = 0.0;
    return GF_OK;
}

gf_status gf_plan(int dim, double k, const double *alpha, const int *M, const gf_trunc_t *trunc,
                  void *cuda_stream, gf_plan_t *out)
{
    if (!out) return fail(GF_ERR_ARG, "gf_plan: out is NULL");
    *out = nullptr;
    g_err[0] = 0;
    if (dim != 2 && dim != 3) return fail(GF_ERR_ARG, "gf_plan: dim must be 2 or 3 (got %d)", dim);
    if (!alpha || !M) return fail(GF_ERR_ARG, "gf_plan: alpha and M must not be NULL");
    if (!(k > 0.0) || !isfinite(k)) return fail(GF_ERR_ARG, "gf_plan: k must be finite and > 0");
    for (int i = 0; i < dim - 1; ++i)
        if (!isfinite(alpha[i])) return fail(GF_ERR_ARG, "gf_plan: alpha must be finite");
    // 3D grids up to 1024 points per axis, 2D up to 2048 (the paper's 2D examples
    // reach N = 1024, i.e. 2048 points per axis, Sec. 5.1)
    const int Mmax = dim == 2 ? 2048 : 1024;
    for (int i = 0; i < dim; ++i)
        if (!pow2_in(M[i], 8, Mmax))
            return fail(GF_ERR_ARG, "gf_plan: M[%d] = %d is not a power of two in [8, %d]", i, M[i], Mmax);
    gf_trunc_t tr;
    gf_trunc_default(&tr);
    if (trunc) tr = *trunc;
    if (!(tr.c > 0.0) || !(tr.c_tilde > tr.c) || !isfinite(tr.c_tilde))
        return fail(GF_ERR_ARG, "gf_plan: need 0 < c < c_tilde");
    if (!(tr.eps > 0.0) || !(2.0 * tr.eps < tr.c_tilde) || !(2.0 * tr.eps < GF_PI))
        return fail(GF_ERR_ARG, "gf_plan: need 0 < 2 eps < min(c_tilde, pi)");
    if (tr.kind != GF_HELMHOLTZ && tr.kind != GF_MAXWELL && tr.kind != GF_DERIV2D) return fail(GF_ERR_ARG, "gf_plan: bad kind");
    if (tr.kind == GF_MAXWELL && dim != 3) return fail(GF_ERR_ARG, "gf_plan: the Maxwell tensor needs dim = 3");
    if (tr.kind == GF_DERIV2D && dim != 2)
        return fail(GF_ERR_ARG, "gf_plan: the derivative fields (GF_DERIV2D) are for 2D plans");
    if (tr.kind == GF_DERIV2D) {
        if (!(tr.k2 >= 0.0) || !isfinite(tr.k2) || tr.k2 == k)
            return fail(GF_ERR_ARG, "gf_plan: k2 must be 0 (gradient only) or finite, > 0 and different from k");
    } else if (tr.k2 != 0.0) {
        return fail(GF_ERR_ARG, "gf_plan: k2 is for GF_DERIV2D plans");
    }
    // the wave numbers whose coefficients the plan forms
    const double kmax = tr.k2 > k ? tr.k2 : k;
    if (tr.quad_nodes <= 0) {
        // Automatic: the 1D integrals of the coefficients oscillate at the grid's
        // frequencies -- h(s) over [eps, 2 eps] at s up to |xi|_max, the X' integrals
        // over [c, (c + c~)/2] at up to q_max + k -- and Gauss-Legendre resolves
        // e^{i w t} on a half-width a once Q exceeds w a by a margin (24 nodes more
        // reach rounding level).  64 nodes at least, a multiple of 8, at most 1024.
        const double qmax = (M[dim - 1] / 2 + 1) * GF_PI / tr.c_tilde;
        double smax;
        if (dim == 3) {
            const double m1 = fabs(alpha[0]) + M[0] / 2 + 1, m2 = fabs(alpha[1]) + M[1] / 2 + 1;
            smax = sqrt(m1 * m1 + m2 * m2 + qmax * qmax);
        } else {
            const double m1 = M[0] / 2 + 1;
            smax = sqrt(m1 * m1 + qmax * qmax);
        }
        const double need = fmax(smax * 0.5 * tr.eps, (qmax + kmax) * 0.25 * (tr.c_tilde - tr.c)) + 24.0;
        int Qa = (int)ceil(need);
        Qa = (Qa + 7) / 8 * 8;
        tr.quad_nodes = Qa < 64 ? 64 : Qa > 1024 ? 1024 : Qa;
    }
    if (tr.quad_nodes < 8 || tr.quad_nodes > 1024) return fail(GF_ERR_ARG, "gf_plan: quad_nodes must be in [8, 1024]");
    if (tr.precision != GF_FP64 && tr.precision != GF_FP32_SPLIT) return fail(GF_ERR_ARG, "gf_plan: bad precision");
    if (tr.far_grid_M != 0) {
        if (dim != 3) return fail(GF_ERR_ARG, "gf_plan: the far-region grid is for 3D plans");
        if (!pow2_in(tr.far_grid_M, 16, 2048))
            return fail(GF_ERR_ARG, "gf_plan: far_grid_M = %d is not a power of two in [16, 2048]", tr.far_grid_M);
        if (tr.far_grid_nz == 0) tr.far_grid_nz = 16;
        if (tr.far_grid_nz < 1 || tr.far_grid_nz > 4096) return fail(GF_ERR_ARG, "gf_plan: far_grid_nz out of [1, 4096]");
        if (!(tr.far_grid_zmax > 0.0)) tr.far_grid_zmax = tr.c_tilde;
        if (!(tr.far_grid_zmax > tr.c) || !isfinite(tr.far_grid_zmax))
            return fail(GF_ERR_ARG, "gf_plan: need far_grid_zmax > c");
    }
    if (!(tr.series_tol > 0.0)) tr.series_tol = tr.precision == GF_FP64 ? 1e-16 : 1e-8;
    if (!(tr.series_tol < 1.0)) return fail(GF_ERR_ARG, "gf_plan: series_tol must be < 1");
    const double a1 = alpha[0], a2 = dim == 3 ? alpha[1] : 0.0;

    // Wood anomaly (Sec. 1): beta_n = 0 for some n.  Only |alpha_n| ~ k matters.
    double bmin_ev = 1e300;
    for (int kw = 0; kw < (tr.k2 > 0.0 ? 2 : 1); ++kw) {
        // the second pass (derivative plans with k2) checks only for a Wood anomaly
        const double kc = kw == 0 ? k : tr.k2;
        int R = (int)ceil(kc) + 2;
        int r2 = dim == 3 ? R : 0;
        double bmin = 1e300;
        for (int n1 = -R - (int)fabs(a1); n1 <= R + (int)fabs(a1); ++n1)
            for (int n2 = -r2 - (int)fabs(a2); n2 <= r2 + (int)fabs(a2); ++n2) {
                double c1 = a1 + n1, c2 = a2 + n2;
                double aa = sqrt(c1 * c1 + c2 * c2);
                double b = sqrt(fabs((kc - aa) * (kc + aa)));
                if (b < bmin) bmin = b;
                // the smallest evanescent b (attained at the smallest |alpha_n| > k, inside this box)
                if (kw == 0 && aa > k && b < bmin_ev) bmin_ev = b;
            }
        if (bmin < 1e-8 * kc) return fail(GF_ERR_WOOD, "gf_plan: |beta_n| = %.3g < 1e-8 k (Wood anomaly)", bmin);
    }
    // Resonance beta_{j'} = +-q_{j_last} (Secs. 2.1, 3.1): perturb c~ or fail.
    const int Mlast = M[dim - 1];
    const double ct0 = tr.c_tilde;
    for (int attempt = 0;; ++attempt) {
        double worst = 1e300;
        int N1 = M[0] / 2, N2 = dim == 3 ? M[1] / 2 : 1;
        for (int kw = 0; kw < (tr.k2 > 0.0 ? 2 : 1); ++kw)
        for (int j1 = -N1; j1 < N1; ++j1)
            for (int j2 = (dim == 3 ? -N2 : 0); j2 < (dim == 3 ? N2 : 1); ++j2) {
                double c1 = a1 + j1, c2 = a2 + j2;
                double A2 = c1 * c1 + c2 * c2;
                const double kc = kw == 0 ? k : tr.k2;
                if (A2 >= kc * kc) continue;  // evanescent beta cannot equal a real q
                for (int j3 = 0; j3 <= Mlast / 2; ++j3) {
                    double q = j3 * GF_PI / tr.c_tilde;
                    double d = fabs(kc * kc - A2 - q * q) / (kc * kc) * (k * k);
                    if (d < worst) worst = d;
                }
            }
        if (worst >= 1e-6 * k * k) break;
        if (tr.resonance_policy == GF_FAIL)
            return fail(GF_ERR_RESONANCE, "gf_plan: |beta^2 - q^2| = %.3g < 1e-6 k^2", worst);
        if (attempt >= 100) return fail(GF_ERR_RESONANCE, "gf_plan: could not perturb c_tilde away from resonance");
        // c~ -> c~0 (1 + 1e-3 m), m = 1, 2, ... (the paper: "avoided by a perturbation of c~")
        tr.c_tilde = ct0 * (1.0 + 1e-3 * (attempt + 1));
    }

    gf_plan_s *p = new gf_plan_s();
    p->dim = dim;
    p->k = k;
    p->alpha[0] = a1;
    p->alpha[1] = a2;
    for (int i = 0; i < 3; ++i) p->M[i] = i < dim ? M[i] : 1;
    p->tr = tr;
    p->bmin_ev = bmin_ev;
    p->precision = tr.precision;
    p->kind = tr.kind;
    p->nf = tr.kind == GF_MAXWELL ? 7 : tr.kind == GF_DERIV2D ? (tr.k2 > 0.0 ? 6 : 3) : 1;
    p->elem = tr.precision == GF_FP64 ? 16 : 8;
    p->T = log(1.0 / tr.series_tol) + 3.0;
    p->P1 = p->M[0] + 3;
    p->P2 = dim == 3 ? p->M[1] + 3 : p->M[1] + 3;
    p->P3 = dim == 3 ? p->M[2] + 3 : 1;
    p->L3count = dim == 3 ? p->M[2] : 1;
    if (dim == 3) {
        // The gather grid keeps only the x3 planes the near branch reads at |x3|:
        // stencil origins i0 from M3/2 - 1 (x3 >= -h3) to floor((c + c~)/h3) + 1 (one
        // index of margin each way), padded planes i0 .. i0 + 3.  The grid of L_d and
        // the even Maxwell fields (xx, yy, zz, xy) are even in x3: node a mirrors node
        // M3 - a, the Nyquist row included.  The odd fields xz, yz (factor c^3 = q_j)
        // are odd except for their Nyquist row j3 = -M3/2, which has no mirror
        // partner and is even at the nodes: L(M3 - a) = -L(a) + 2 (-1)^(M3/2 + a) P(t)
        // with P the in-plane transform of that row, which a Maxwell plan keeps
        // beside the grid (nyqgrid) for the targets with x3 < 0.
        const int M3 = p->M[2];
        const double h3 = 2.0 * tr.c_tilde / M3;
        const int i0min = M3 / 2 - 1;
        const int i0max = std::min(M3 - 1, (int)floor((tr.c + tr.c_tilde) / h3) + 1);
        if (i0max + 3 <= M3 && i0min >= 1) {
            p->Q3lo = i0min;
            p->P3 = i0max + 3 - i0min + 1;
            p->a3first = p->Q3lo - 1;
            p->L3count = p->P3;
            p->nyq = p->nf == 7 ? 1 : 0;
        }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (dim == 3 && tr.precision == GF_FP64 && tr.kind == GF_HELMHOLTZ &&
        (cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
        gf_destroy(p);
        return fail(GF_ERR_CUDA, "gf_plan: event creation failed");
    }
    if (g_timing.load()) {
        p->timing = true;
        for (int i = 0; i < 6; ++i)
            if (cudaEventCreate(&p->ev[i]) != cudaSuccess) p->timing = false;
    }

    // ---- host tables
    const int Q = tr.quad_nodes;
    std::vector<double> gx, gw;
    gauss_legendre(Q, gx, gw);
    const double c = tr.c, ct = tr.c_tilde, eps = tr.eps, cm = 0.5 * (c + ct);
    std::vector<double> tt(Q), tW(Q), rr(Q), P0(Q, 0.0), P1(Q, 0.0);
    std::vector<double2> B(Q);
    {
        double hw = 0.5 * (cm - c), mid = 0.5 * (cm + c);
        for (int m = 0; m < Q; ++m) {
            tt[m] = mid + hw * gx[m];
            tW[m] = gw[m] * hw * chi_d1(tt[m], c, ct);
        }
        double hr = 0.5 * eps, midr = 1.5 * eps;
        for (int m = 0; m < Q; ++m) {
            double r = midr + hr * gx[m];
            rr[m] = r;
            double wr = gw[m] * hr;
            // w e^{ikr}(2ik Y' + Y'')
            double y1 = yps1(r, eps), y2 = yps2(r, eps);
            double cr = cos(k * r), sr = sin(k * r);
            double2 f = make_double2(y2, 2.0 * k * y1);
            B[m] = make_double2(wr * (cr * f.x - sr * f.y), wr * (cr * f.y + sr * f.x));
            // Phi_1(r) = (2 + ln r) Y'/r + Y'' ln r
            double ph1 = (2.0 + log(r)) * y1 / r + y2 * log(r);
            P0[m] = wr * ph1 * r;
            P1[m] = wr * ph1 * r * r;
        }
    }
    // derivative plans: Gauss-Legendre nodes on [0, eps] and [eps, 2 eps] with
    // weights w Y(r) for the Hankel transforms of the cutoff
    const bool deriv = tr.kind == GF_DERIV2D;
    std::vector<double> rrd(deriv ? 2 * Q : 0), wyd(deriv ? 2 * Q : 0);
    if (deriv) {
        const double hr = 0.5 * eps;
        for (int piece = 0; piece < 2; ++piece)
            for (int m = 0; m < Q; ++m) {
                const double r = (piece + 0.5) * eps + hr * gx[m];
                rrd[piece * Q + m] = r;
                wyd[piece * Q + m] = gw[m] * hr * (piece == 0 ? 1.0 : yps0(r, eps));
            }
    }
    // Piecewise Chebyshev interpolants (degree 14, panels of width 2) of the
    // radial transforms on [0, s_max], s_max >= the largest frequency norm:
    // 3D h(s) = sum_m B_m sin(s r_m)/s, 2D the Bessel sums of F1-hat, F2-hat.
    // (computed on the device from the quadrature tables, see gf_launch_cheb_table)
    const int hdeg = 14;
    const double hpan = 2.0;
    int hnpan = 1;
    size_t hcheb_n = 0;
    {
        double smax;
        if (dim == 3) {
            double m1 = fabs(a1) + M[0] / 2 + 1, m2 = fabs(a2) + M[1] / 2 + 1, m3 = (M[2] / 2 + 1) * GF_PI / ct;
            smax = sqrt(m1 * m1 + m2 * m2 + m3 * m3) + hpan;
        } else {
            double m1 = M[0] / 2 + 1, m2 = (M[1] / 2 + 1) * GF_PI / ct;
            smax = sqrt(m1 * m1 + m2 * m2) + hpan;
        }
        hnpan = (int)ceil(smax / hpan) + 1;
        hcheb_n = (size_t)hnpan * (hdeg + 1);
    }
    double F10 = 0.0;
    if (dim == 2) {
        // sqrt(V) F1-hat_0 = -int_0^{2eps} t ln t Y dt; [0, eps] in closed form
        double s = 0.5 * eps * eps * log(eps) - 0.25 * eps * eps;
        double hr = 0.5 * eps, midr = 1.5 * eps;
        for (int m = 0; m < Q; ++m) {
            double t = midr + hr * gx[m];
            s += gw[m] * hr * t * log(t) * yps0(t, eps);
        }
        F10 = -s;
    }

    // ---- device memory (stream-ordered, from the library pool) and the tables:
    // the small host tables go up through pinned staging; the last-axis phase
    // table, the Chebyshev table of h(s) and the series tables are built on
    // the device.  Nothing here waits for the stream.
    const size_t nodes_padded = (size_t)p->P1 * p->P2 * p->P3;
    p->grid_bytes = nodes_padded * p->nf * p->elem;
    const size_t E_n = (size_t)Mlast * Q;
    const size_t host_tab_bytes = sizeof(double) * 5 * Q + sizeof(double2) * Q + (deriv ? sizeof(double) * 4 * Q : 0);
    const bool ftabs = tr.precision == GF_FP32_SPLIT;  // float copies for the split plans' coefficients
    const size_t dcheb_n = deriv ? 3 * hcheb_n : 0;
    const size_t tab_bytes = host_tab_bytes + sizeof(double2) * (E_n + hcheb_n + dcheb_n) +
                             (ftabs ? sizeof(float2) * (E_n + hcheb_n) : 0);
    const size_t work_bytes = gf_plan_work_bytes(p);
    void *work = nullptr;
    gf_status st_err = GF_OK;
    p->stream = st;
    do {
        cudaError_t e;
        if ((e = gf_dev_alloc((void **)&p->errw, sizeof(int), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(p->errw, 0, sizeof(int), st)) != cudaSuccess ||
            (p->nyq && (e = gf_dev_alloc(&p->nyqgrid, (size_t)p->P1 * p->P2 * 2 * p->elem, st)) != cudaSuccess) ||
            (e = gf_dev_alloc(&p->grid, p->grid_bytes, st)) != cudaSuccess ||
            (e = gf_dev_alloc(&p->tables, tab_bytes, st)) != cudaSuccess ||
            (e = gf_dev_alloc(&work, work_bytes, st)) != cudaSuccess) {
            st_err = fail(e == cudaErrorMemoryAllocation ? GF_ERR_NOMEM : GF_ERR_CUDA, "gf_plan: device allocation: %s",
                          cudaGetErrorString(e));
            break;
        }
        char *tb = (char *)p->tables;
        double *d_tt = (double *)tb, *d_tW = d_tt + Q, *d_rr = d_tW + Q, *d_P0 = d_rr + Q, *d_P1 = d_P0 + Q;
        double2 *d_B = (double2 *)(d_P1 + Q);
        double *d_rrd = (double *)(d_B + Q), *d_wyd = d_rrd + (deriv ? 2 * Q : 0);
        double2 *d_E = (double2 *)(d_wyd + (deriv ? 2 * Q : 0)), *d_H = d_E + E_n, *d_D = d_H + hcheb_n;
        float2 *d_Ef = ftabs ? (float2 *)(d_D + dcheb_n) : nullptr, *d_Hf = ftabs ? d_Ef + E_n : nullptr;
        {
            std::vector<char> pack(host_tab_bytes);
            char *hb = pack.data();
            memcpy(hb + ((char *)d_tt - tb), tt.data(), sizeof(double) * Q);
            memcpy(hb + ((char *)d_tW - tb), tW.data(), sizeof(double) * Q);
            memcpy(hb + ((char *)d_rr - tb), rr.data(), sizeof(double) * Q);
            memcpy(hb + ((char *)d_P0 - tb), P0.data(), sizeof(double) * Q);
            memcpy(hb + ((char *)d_P1 - tb), P1.data(), sizeof(double) * Q);
            memcpy(hb + ((char *)d_B - tb), B.data(), sizeof(double2) * Q);
            if (deriv) {
                memcpy(hb + ((char *)d_rrd - tb), rrd.data(), sizeof(double) * 2 * Q);
                memcpy(hb + ((char *)d_wyd - tb), wyd.data(), sizeof(double) * 2 * Q);
            }
            if ((e = gf_stage_upload(tb, hb, host_tab_bytes, st)) != cudaSuccess ||
                (e = gf_launch_e_table(d_tt, Q, Mlast, GF_PI / ct, d_E, d_Ef, st)) != cudaSuccess ||
                (e = gf_launch_cheb_table(dim, d_rr, d_B, d_P0, d_P1, Q, hnpan, hdeg, hpan, d_H, d_Hf, st)) != cudaSuccess ||
                (deriv && (e = gf_launch_cheb_deriv(d_rrd, d_wyd, 2 * Q, hnpan, hdeg, hpan, d_D, st)) != cudaSuccess)) {
                st_err = fail(GF_ERR_CUDA, "gf_plan: tables: %s", cudaGetErrorString(e));
                break;
            }
        }
        SynthArgs &sa = p->sa;
        sa.dim = dim;
        sa.M1 = p->M[0];
        sa.M2 = p->M[1];
        sa.M3 = dim == 3 ? p->M[2] : 1;
        sa.Mlast = Mlast;
        sa.lgMlast = 0;
        while ((1 << sa.lgMlast) < Mlast) ++sa.lgMlast;
        sa.Q = Q;
        sa.nf = p->nf;
        sa.k = k;
        sa.a1 = a1;
        sa.a2 = a2;
        sa.ct = ct;
        sa.qs = GF_PI / ct;
        sa.qsh = (float)sa.qs;
        sa.qsl = (float)(sa.qs - (double)sa.qsh);
        // smallest g with e^{-g c}/(2 g^2) < 1e-20 (the function decreases in g)
        {
            double g = 1.0;
            while (exp(-g * c) / (2.0 * g * g) >= 1e-20) g += 0.25;
            sa.gskip = g;
        }
        sa.invV = dim == 3 ? 1.0 / (8.0 * GF_PI * GF_PI * ct) : 1.0 / (4.0 * GF_PI * ct);
        sa.tW = d_tW;
        sa.tt = d_tt;
        sa.E = d_E;
        sa.Ef = d_Ef;
        sa.hchebf = d_Hf;
        // split plans form a column's coefficients in float when its beta is evanescent
        // and at least 0.05 k (clear of Wood anomalies; propagating columns stay double)
        sa.gfloat = ftabs ? 0.05 * k : 1e300;
        sa.rr = d_rr;
        sa.B = d_B;
        sa.hcheb = d_H;
        sa.hdeg = hdeg;
        sa.hnpan = hnpan;
        sa.hpan = hpan;
        sa.ihpan = 1.0 / hpan;
        sa.Pw0 = d_P0;
        sa.Pw1 = d_P1;
        sa.F10 = F10;
        sa.work = work;
        sa.grid = p->grid;
        sa.P1 = p->P1;
        sa.P2 = p->P2;
        sa.P3 = p->P3;
        sa.Q3lo = p->Q3lo;
        sa.a3first = p->a3first;
        sa.L3count = p->L3count;
        sa.nyq = p->nyq;
        sa.nyqgrid = p->nyqgrid;
        sa.err = p->errw;
        sa.oddmask = tr.kind == GF_MAXWELL ? (1 << 4) | (1 << 5) : deriv ? (1 << 2) | (1 << 4) : 0;
        sa.deriv = deriv ? 1 : 0;
        sa.k2 = tr.k2;
        sa.dcheb = deriv ? d_D : nullptr;
        {
            // one CTA holds whole lines of every stored field in shared memory
            int dev = 0, optin = 232448;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
                cudaGetLastError();
                optin = 232448;
            }
            const size_t need = gf_synth_smem_need(sa, p->precision);
            if (need > (size_t)optin) {
                st_err = fail(GF_ERR_UNSUPPORTED,
                              "gf_plan: the synthesis of this grid needs %zu bytes of shared memory per CTA (limit %d): "
                              "fewer points per axis, fewer fields or the split precision",
                              need, optin);
                break;
            }
        }
        if (p->timing) cudaEventRecord(p->ev[0], st);
        if ((e = gf_launch_synth(sa, p->precision, st)) != cudaSuccess) {
            st_err = fail(GF_ERR_CUDA, "gf_plan: synthesis launch: %s", cudaGetErrorString(e));
            break;
        }
        if (tr.far_grid_M > 0) {
            // far-region grid: planes z_m = c + (m - 1) hz, m = 0 .. nz + 2
            p->fM = tr.far_grid_M;
            p->fNZ = tr.far_grid_nz + 3;
            p->fhz = (tr.far_grid_zmax - c) / tr.far_grid_nz;
            p->fz0 = c - p->fhz;
            p->fzmax = tr.far_grid_zmax;
            const int fP = p->fM + 3;
            p->far_bytes = (size_t)fP * fP * p->fNZ * p->nf * p->elem;
            void *fwork = nullptr;
            if ((e = gf_dev_alloc(&p->fargrid, p->far_bytes, st)) != cudaSuccess ||
                (e = gf_dev_alloc(&fwork, (size_t)p->fM * p->fM * p->fNZ * p->nf * p->elem, st)) != cudaSuccess) {
                st_err = fail(e == cudaErrorMemoryAllocation ? GF_ERR_NOMEM : GF_ERR_CUDA,
                              "gf_plan: device allocation (far-region grid): %s", cudaGetErrorString(e));
                if (fwork) gf_dev_free(fwork, st);
                break;
            }
            SynthArgs fa = sa;
            fa.M1 = fa.M2 = p->fM;
            fa.M3 = p->fNZ;
            fa.P1 = fa.P2 = fP;
            fa.P3 = p->fNZ;
            fa.Q3lo = 0;
            fa.a3first = 0;
            fa.L3count = p->fNZ;
            fa.nyq = 0;
            fa.nyqgrid = nullptr;
            fa.zlinear = 1;
            fa.work = fwork;
            fa.grid = p->fargrid;
            e = gf_launch_far_grid(fa, p->precision, k, a1, a2, p->fz0, p->fhz, st);
            gf_dev_free(fwork, st);
            if (e != cudaSuccess) {
                st_err = fail(GF_ERR_CUDA, "gf_plan: far-region grid launch: %s", cudaGetErrorString(e));
                break;
            }
        }
        if (p->timing) cudaEventRecord(p->ev[1], st);
        // far-series tables: index box covering |alpha_n|^2 <= k^2 + (T/c)^2
        if (dim == 3) {
            double Rc = sqrt(k * k + (p->T / c) * (p->T / c));
            p->n1lo = (int)floor(-a1 - Rc) - 1;
            p->n1hi = (int)ceil(-a1 + Rc) + 1;
            p->n2lo = (int)floor(-a2 - Rc) - 1;
            p->n2hi = (int)ceil(-a2 + Rc) + 1;
            size_t ne = (size_t)(p->n1hi - p->n1lo + 1) * (p->n2hi - p->n2lo + 1);
            size_t eb = p->precision == GF_FP64 ? sizeof(BetaEntry) : sizeof(BetaEntryF);
            // propagating indices lie in the sub-box |c1|, |c2| <= k
            const int pbox[4] = {(int)floor(-a1 - k) - 1, (int)ceil(-a1 + k) + 1, (int)floor(-a2 - k) - 1,
                                 (int)ceil(-a2 + k) + 1};
            const size_t nprop_max = (size_t)(pbox[1] - pbox[0] + 1) * (pbox[3] - pbox[2] + 1);
            // T[j] = e^{-(j - j0)/S}, S = GF_EXPTAB_STEPS: the core weights e^{-y},
            // y = b|x3| + ln b, of a lane's truncation set (b|x3| <= T) have
            // ln(bmin) <= y <= T + ln(bmax), bmax <= sqrt(2) (Rc + 2) over the index box
            constexpr int S = GF_EXPTAB_STEPS;
            p->exptab_j0 = S * ((int)ceil(-log(fmin(bmin_ev, 1.0))) + 1);
            if (p->exptab_j0 < S) p->exptab_j0 = S;
            p->exptab_n = p->exptab_j0 + S * ((int)ceil(p->T + log(1.4143 * (Rc + 2.0))) + 2) + 1;
            const bool want_exp = p->precision == GF_FP64;
            if ((e = gf_dev_alloc(&p->btab, ne * eb, st)) != cudaSuccess ||
                (e = gf_dev_alloc((void **)&p->prop, sizeof(PropEntry) * nprop_max + 16, st)) != cudaSuccess ||
                (want_exp && (e = gf_dev_alloc((void **)&p->exptab, 2 * sizeof(double2) * p->exptab_n, st)) != cudaSuccess)) {
                st_err = fail(GF_ERR_NOMEM, "gf_plan: device allocation (series tables): %s", cudaGetErrorString(e));
                break;
            }
            p->nprop_dev = (int *)(p->prop + nprop_max);
            EvalArgs ea{};
            ea.k = k;
            ea.a1 = a1;
            ea.a2 = a2;
            ea.n1lo = p->n1lo;
            ea.n1hi = p->n1hi;
            ea.n2lo = p->n2lo;
            ea.n2hi = p->n2hi;
            ea.btab = p->btab;
            ea.exptab_n = want_exp ? p->exptab_n : 0;
            ea.exptab_j0 = p->exptab_j0;
            if ((e = gf_launch_series_tables(ea, p->precision, want_exp ? p->exptab : nullptr, p->prop, p->nprop_dev,
                                             pbox, st)) != cudaSuccess) {
                st_err = fail(GF_ERR_CUDA, "gf_plan: series table launch: %s", cudaGetErrorString(e));
                break;
            }
        }
        if (p->timing) cudaEventRecord(p->ev[2], st);
        p->ev_plan = p->timing;
        // the work buffer goes back to the pool in stream order once the synthesis is done
        gf_dev_free(work, st);
        work = nullptr;
        p->sa.work = nullptr;
    } while (0);
    if (st_err != GF_OK) {
        if (work) gf_dev_free(work, st);
        gf_destroy(p);
        return st_err;
    }
    *out = p;
    return GF_OK;
}

size_t gf_grid_bytes(gf_plan_t p)
{
    if (!p) return 0;
    return (size_t)p->M[0] * p->M[1] * p->M[2] * p->nf * p->elem;
}

gf_status gf_eval_grid(gf_plan_t p, void *dev_out, size_t out_bytes, void *cuda_stream)
{
    if (!p || !dev_out) return fail(GF_ERR_ARG, "gf_eval_grid: NULL argument");
    if (out_bytes < gf_grid_bytes(p)) return fail(GF_ERR_ARG, "gf_eval_grid: out_bytes %zu < %zu", out_bytes, gf_grid_bytes(p));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (p->dim == 3 && (p->Q3lo != 0 || p->L3count != p->M[2])) {
        // the plan keeps only the near planes: synthesise the whole grid once more
        // into pool buffers returned in stream order
        SynthArgs fs = p->sa;
        fs.Q3lo = 0;
        fs.P3 = p->M[2] + 3;
        fs.a3first = 0;
        fs.L3count = p->M[2];
        fs.nyq = 0;
        fs.nyqgrid = nullptr;
        void *work = nullptr, *grid = nullptr;
        CU(gf_dev_alloc(&work, (size_t)p->M[0] * p->M[1] * p->M[2] * p->nf * p->elem, st));
        cudaError_t e = gf_dev_alloc(&grid, (size_t)fs.P1 * fs.P2 * fs.P3 * p->nf * p->elem, st);
        if (e == cudaSuccess) {
            fs.work = work;
            fs.grid = grid;
            e = gf_launch_synth(fs, p->precision, st);
            if (e == cudaSuccess) e = gf_launch_extract(fs, p->precision, dev_out, st);
        }
        gf_dev_free(work, st);
        gf_dev_free(grid, st);
        CU(e);
        return GF_OK;
    }
    CU(gf_launch_extract(p->sa, p->precision, dev_out, st));
    return GF_OK;
}

// Scratch of one evaluation (ints): the counters, padded to GF_COUNTER_PAD, then
// the far list in append order (3D: the targets' bucket codes), the bucket-sorted
// far list and the near list, n entries each; for 3D plans then one ticket per
// 32-target chunk for each of the two far kernels, the segment counts of the
// stable far list and, 256-byte aligned, the far kernels' slab partials (2 n_pad
// target slots of the output's entries each).  With these the far sums are the
// same bit for bit from call to call: the same list, and slab partials added in
// slab order.
constexpr int64_t GF_COUNTER_PAD = 1024;
static_assert(GF_SCRATCH_COUNTERS <= GF_COUNTER_PAD, "counter block too small");

// Segments of the stable far list: 512 targets, more when that would make over
// 8192 segments (the scan's work per bucket stays bounded).
static int64_t far_segment_size(int64_t n)
{
    const int64_t segs = (n + 511) / 512;
    return segs <= 8192 ? 512 : ((n + 8191) / 8192 + 31) / 32 * 32;
}

gf_status gf_eval_points(gf_plan_t p, const double *dev_xyz, int64_t n, int which, void *dev_out,
                         void *cuda_stream)
{
    EvalArgs a;
    gf_status s = gf_plan_eval_args(p, dev_xyz, n, which, dev_out, &a, "gf_eval_points");
    if (s != GF_OK || n == 0) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // per-call scratch from the stream-ordered pool on the caller's stream, returned
    // to the pool in stream order after the kernels: concurrent calls on other
    // streams each have their own, and the plan stays unchanged
    const bool slabs = p->dim == 3;
    const int64_t npad = (n + 31) / 32 * 32, nchmax = npad / 32, slabcap = 2 * npad;
    const int64_t segsize = far_segment_size(n), nseg = (n + segsize - 1) / segsize;
    const size_t ints = (size_t)(GF_COUNTER_PAD + 3 * n + (slabs ? 2 * nchmax + nseg * GF_FAR_BUCKETS : 0));
    const size_t off_buf = (sizeof(int) * ints + 255) / 256 * 256;
    const size_t buf_bytes = slabs ? (size_t)slabcap * gf_out_entries(which) * p->elem : 0;
    int *scratch = nullptr;
    CU(gf_dev_alloc((void **)&scratch, off_buf + 2 * buf_bytes, st));
    a.far_count = scratch;
    a.far_idx = scratch + GF_COUNTER_PAD;
    a.far_sorted = a.far_idx + n;
    a.near_idx = p->dim == 3 ? a.far_idx + 2 * n : nullptr;
    cudaError_t e = cudaMemsetAsync(a.far_count, 0, sizeof(int) * GF_SCRATCH_COUNTERS, st);
    if (slabs && e == cudaSuccess) {
        a.slabtick[0] = a.far_idx + 3 * n;
        a.slabtick[1] = a.slabtick[0] + nchmax;
        a.slabbuf[0] = (char *)scratch + off_buf;
        a.slabbuf[1] = (char *)scratch + off_buf + buf_bytes;
        a.slabcap = slabcap;
        a.seghist = a.slabtick[1] + nchmax;
        a.segsize = (int)segsize;
        a.nseg = (int)nseg;
        e = cudaMemsetAsync(a.slabtick[0], 0, sizeof(int) * 2 * nchmax, st);
    }
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(p->mu);
        // 3D double-precision Helmholtz plans run the far series' double sums and
        // float tails as two concurrent kernels (the tails on the library's side stream)
        EvalFork fk{};
        const EvalFork *fork = nullptr;
        if (p->ev_fork) {
            fk.aux = gf_aux_stream();
            fk.fork = p->ev_fork;
            fk.join = p->ev_join;
            if (fk.aux) fork = &fk;
        }
        if (p->timing) cudaEventRecord(p->ev[3], st);
        e = gf_launch_eval(a, p->precision, st, p->timing ? p->ev[4] : nullptr, fork);
        if (p->timing && e == cudaSuccess) {
            cudaEventRecord(p->ev[5], st);
            p->ev_eval = true;
        }
    }
    gf_dev_free(scratch, st);
    CU(e);
    return GF_OK;
}

}  // extern "C"

// Validation and argument set-up of one evaluation (everything but the
// scratch pointers), shared by gf_eval_points, the allocation-free entry
// point (noalloc.cu) and the batched sweeps; `who` names the caller in errors.
gf_status gf_plan_eval_args(gf_plan_t p, const double *dev_xyz, int64_t n, int which, void *dev_out,
                            EvalArgs *a_out, const char *who)
{
    if (!p || !a_out) return fail(GF_ERR_ARG, "%s: NULL plan", who);
    if (n < 0 || n > (int64_t)0x7fffffff) return fail(GF_ERR_ARG, "%s: n = %lld out of range", who, (long long)n);
    if (n > 0 && (!dev_xyz || !dev_out)) return fail(GF_ERR_ARG, "%s: NULL buffer", who);
    bool ok = (p->dim == 2 && which == GF_OUT_G) || (p->dim == 3 && p->kind == GF_HELMHOLTZ && (which == GF_OUT_GD || which == GF_OUT_LD)) ||
              (p->kind == GF_MAXWELL && (which == GF_OUT_MAXWELL6 || which == GF_OUT_MAXWELL7)) ||
              (p->kind == GF_DERIV2D && (which == GF_OUT_GRAD || (which == GF_OUT_HESSDIFF && p->nf == 6)));
    if (!ok) return fail(GF_ERR_ARG, "%s: output kind %d does not match the plan", who, which);
    EvalArgs a{};
    a.dim = p->dim;
    a.M1 = p->M[0];
    a.M2 = p->M[1];
    a.M3 = p->M[2];
    a.P1 = p->P1;
    a.P2 = p->P2;
    a.P3 = p->P3;
    a.Q3lo = p->Q3lo;
    a.nf = p->nf;
    a.which = which;
    a.k = p->k;
    a.k2 = p->tr.k2;
    a.a1 = p->alpha[0];
    a.a2 = p->alpha[1];
    a.c = p->tr.c;
    a.ct = p->tr.c_tilde;
    a.eps = p->tr.eps;
    a.h1 = 2.0 * GF_PI / p->M[0];
    a.h2 = p->dim == 3 ? 2.0 * GF_PI / p->M[1] : 2.0 * p->tr.c_tilde / p->M[1];
    a.h3 = p->dim == 3 ? 2.0 * p->tr.c_tilde / p->M[2] : 1.0;
    a.T = p->T;
    a.grid = p->grid;
    a.x = dev_xyz;
    a.out = dev_out;
    a.n = n;
    a.btab = p->btab;
    a.n1lo = p->n1lo;
    a.n1hi = p->n1hi;
    a.n2lo = p->n2lo;
    a.n2hi = p->n2hi;
    a.prop = p->prop;
    a.nprop = p->nprop_dev;
    a.exptab = p->exptab;
    a.exptab_n = p->exptab_n;
    a.exptab_j0 = p->exptab_j0;
    a.bmin = p->bmin_ev;
    a.nyqgrid = p->nyqgrid;
    a.fargrid = p->fargrid;
    if (p->fargrid) {
        a.fM1 = a.fM2 = p->fM;
        a.fP1 = a.fP2 = p->fM + 3;
        a.fNZ = p->fNZ;
        a.fz0 = p->fz0;
        a.fhz = p->fhz;
        a.fzmax = p->fzmax;
        a.fh1 = a.fh2 = 2.0 * GF_PI / p->fM;
    }
    *a_out = a;
    return GF_OK;
}

gf_status gf_set_error(gf_status s, const char *msg) { return fail(s, "%s", msg); }

// Synthesis arguments of a plan (batched sweeps re-run the synthesis of many
// plans with their own work buffers) and the bytes of its work buffer.
SynthArgs gf_plan_synth_args(gf_plan_t p) { return p->sa; }
// (3D: only the stored x3 planes, compact; 2D: the whole grid)
size_t gf_plan_work_bytes(gf_plan_t p)
{
    return (size_t)p->M[0] * p->M[1] * (p->dim == 3 ? p->L3count + p->nyq : 1) * p->nf * p->elem;
}
int gf_plan_precision(gf_plan_t p) { return p->precision; }

extern "C" {

gf_status gf_set_phase_timing(int on)
{
    g_timing.store(on ? 1 : 0);
    return GF_OK;
}

gf_status gf_plan_phase_ms(gf_plan_t p, float ms[4])
{
    if (!p || !ms) return fail(GF_ERR_ARG, "gf_plan_phase_ms: NULL argument");
    for (int i = 0; i < 4; ++i) ms[i] = -1.0f;
    if (p->ev_plan) {
        CU(cudaEventSynchronize(p->ev[2]));
        CU(cudaEventElapsedTime(&ms[0], p->ev[0], p->ev[1]));
        CU(cudaEventElapsedTime(&ms[1], p->ev[1], p->ev[2]));
    }
    if (p->ev_eval) {
        CU(cudaEventSynchronize(p->ev[5]));
        CU(cudaEventElapsedTime(&ms[2], p->ev[3], p->ev[4]));
        CU(cudaEventElapsedTime(&ms[3], p->ev[4], p->ev[5]));
    }
    return GF_OK;
}

gf_status gf_eval_points_host(gf_plan_t p, const double *host_xyz, int64_t n, int which, void *host_out,
                              void *cuda_stream)
{
    if (!p) return fail(GF_ERR_ARG, "gf_eval_points_host: NULL plan");
    if (n < 0) return fail(GF_ERR_ARG, "gf_eval_points_host: n < 0");
    if (n == 0) return GF_OK;
    if (!host_xyz || !host_out) return fail(GF_ERR_ARG, "gf_eval_points_host: NULL buffer");
    int ne = gf_out_entries(which);
    size_t xb = sizeof(double) * p->dim * (size_t)n, ob = p->elem * ne * (size_t)n;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // device staging per call from the stream-ordered pool (pool hits after the first call).
    // The targets go up on the library's copy stream, allocated there and joined to
    // cuda_stream by an event, so the upload overlaps work already queued on cuda_stream
    // (a plan's synthesis); without that stream, on cuda_stream itself.
    cudaStream_t cs = gf_copy_stream();
    cudaEvent_t up = nullptr;
    if (cs && cudaEventCreateWithFlags(&up, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        up = nullptr;
    }
    if (!up) cs = st;
    void *dx = nullptr, *dout = nullptr;
    cudaError_t e = gf_dev_alloc(&dx, xb, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx, host_xyz, xb, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && up) {
        e = cudaEventRecord(up, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, up, 0);
    }
    if (up) cudaEventDestroy(up);  // released once its work completes
    if (e != cudaSuccess) {
        if (dx) gf_dev_free(dx, cs);
        CU(e);
    }
    e = gf_dev_alloc(&dout, ob, st);
    gf_status s = GF_OK;
    if (e == cudaSuccess) {
        s = gf_eval_points(p, (const double *)dx, n, which, dout, cuda_stream);
        if (s == GF_OK) e = cudaMemcpyAsync(host_out, dout, ob, cudaMemcpyDeviceToHost, st);
    }
    gf_dev_free(dout, st);
    gf_dev_free(dx, st);
    if (s != GF_OK) return s;
    CU(e);
    CU(cudaStreamSynchronize(st));
    return GF_OK;
}

gf_status gf_plan_get_info(gf_plan_t p, gf_plan_info_t *info)
{
    if (!p || !info) return fail(GF_ERR_ARG, "gf_plan_get_info: NULL argument");
    memset(info, 0, sizeof(*info));
    info->dim = p->dim;
    for (int i = 0; i < 3; ++i) info->M[i] = p->M[i];
    info->nfields = p->nf;
    info->precision = p->precision;
    info->kind = p->kind;
    info->k = p->k;
    info->alpha[0] = p->alpha[0];
    info->alpha[1] = p->alpha[1];
    info->c = p->tr.c;
    info->c_tilde = p->tr.c_tilde;
    info->eps = p->tr.eps;
    info->series_tol = p->tr.series_tol;
    info->quad_nodes = p->tr.quad_nodes;
    info->series_n1_lo = p->n1lo;
    info->series_n1_hi = p->n1hi;
    info->series_n2_lo = p->n2lo;
    info->series_n2_hi = p->n2hi;
    info->grid_device_bytes = p->grid_bytes;
    info->far_grid_M = p->fM;
    info->far_grid_nz = p->fNZ ? p->fNZ - 3 : 0;
    info->far_grid_zmax = p->fzmax;
    info->far_grid_device_bytes = p->far_bytes;
    info->k2 = p->tr.k2;
    return GF_OK;
}

gf_status gf_plan_status(gf_plan_t p, void *cuda_stream)
{
    if (!p) return fail(GF_ERR_ARG, "gf_plan_status: NULL plan");
    if (!p->errw) return GF_OK;
    int host = 0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    CU(cudaMemcpyAsync(&host, p->errw, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (host) return fail(GF_ERR_TIMEOUT, "gf_plan_status: a bounded wait for staged copies ran out in the synthesis");
    return GF_OK;
}

gf_status gf_release_memory(void)
{
    CU(gf_trim_pool());
    return GF_OK;
}

gf_status gf_destroy(gf_plan_t p)
{
    if (!p) return GF_OK;
    // the plan may have been used on any stream: wait for the device, then hand
    // the buffers back to the pool
    cudaDeviceSynchronize();
    void *bufs[] = {p->grid, p->nyqgrid, p->fargrid, p->tables, p->btab, p->prop, p->exptab, p->errw};
    for (void *b : bufs) gf_dev_free(b, 0);
    for (int i = 0; i < 6; ++i)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    delete p;
    return GF_OK;
}

}  // extern "C"
