// Internal declarations of the GB300 library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gf.h"

#define GF_PI 3.14159265358979323846

// ---------------------------------------------------------------------------
// complex helpers (double2 / float2)
// ---------------------------------------------------------------------------
template <typename R> struct cplx_t;
template <> struct cplx_t<double> { typedef double2 T; };
template <> struct cplx_t<float> { typedef float2 T; };

__host__ __device__ inline double2 cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ inline float2 cmk(float r, float i) { return make_float2(r, i); }
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ inline double2 cdiv(double2 a, double2 b)
{
    // a / b with Smith's scaling
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    }
    double r = b.x / b.y, d = b.y + b.x * r;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}

// ---------------------------------------------------------------------------
// Order-8 smoothstep (C^8 at both ends), the profile of both cutoffs X and
// Y_eps: S(s) = s^9 P(-s) on [0, 1/2] with P(y) = sum_n a_n y^n,
// a_n = C(8+n, n) C(17, 8-n); S(s) = 1 - S(1-s) on the other half.
// S'(s) = 218790 (s(1-s))^8, S''(s) = 8 * 218790 (s(1-s))^7 (1-2s).
// ---------------------------------------------------------------------------
__host__ __device__ inline double smooth8_lo(double s)
{
    const double y = -s;
    double p = 12870.0;
    p = fma(p, y, 109395.0);
    p = fma(p, y, 408408.0);
    p = fma(p, y, 875160.0);
    p = fma(p, y, 1178100.0);
    p = fma(p, y, 1021020.0);
    p = fma(p, y, 556920.0);
    p = fma(p, y, 175032.0);
    p = fma(p, y, 24310.0);
    double s3 = s * s * s;
    return s3 * s3 * s3 * p;
}
__host__ __device__ inline double smooth8(double s)
{
    if (s <= 0.0) return 0.0;
    if (s >= 1.0) return 1.0;
    return s <= 0.5 ? smooth8_lo(s) : 1.0 - smooth8_lo(1.0 - s);
}
__host__ __device__ inline double smooth8_d1(double s)
{
    if (s <= 0.0 || s >= 1.0) return 0.0;
    double u = s * (1.0 - s), u2 = u * u, u4 = u2 * u2;
    return 218790.0 * u4 * u4;
}
__host__ __device__ inline double smooth8_d2(double s)
{
    if (s <= 0.0 || s >= 1.0) return 0.0;
    double u = s * (1.0 - s), u2 = u * u, u4 = u2 * u2;
    return 8.0 * 218790.0 * u4 * u2 * u * (1.0 - 2.0 * s);
}

// ---------------------------------------------------------------------------
// Parameters of the synthesis kernels (coefficients + inverse FFT), by value.
// ---------------------------------------------------------------------------
struct SynthArgs {
    int dim;            // 2 or 3
    int M1, M2, M3;     // grid points per axis (2D: M3 = 1)
    int Mlast;          // points on the last axis (x2 in 2D, x3 in 3D)
    int lgMlast;
    int Q;              // Gauss nodes
    int nf;             // stored fields: 1 (Helmholtz) or 7 (Maxwell: 6 combined + L_d)
    int TJ;             // columns per CTA in the first pass (power of two)
    double k, a1, a2;   // wave number, alpha
    double ct;          // c~ (possibly perturbed)
    double qs;          // pi / c~: last-axis frequency q_b = freq(b) qs
    float qsh, qsl;     // qs as a float pair (split plans' float coefficients)
    double gskip;       // evanescent |beta| above which e^{-|beta| c}/(2 |beta|^2) < 1e-20
    double gfloat;      // split plans (3D): evanescent |beta| from which a column's coefficients are formed in float
    double invV;        // 1 / |D|: 1/(8 pi^2 c~) in 3D, 1/(4 pi c~) in 2D
    const double *tW;   // [Q] w_m hw X'(t_m) on [c, (c+c~)/2]
    const double *tt;   // [Q] t_m
    const double2 *E;   // [Mlast][Q] e^{i q_b t_m}, q_b = freq(b) pi / c~
    const float2 *Ef;   // the same in float (split plans)
    const double *rr;   // [Q] r_m on [eps, 2 eps]
    const double2 *B;   // [Q] 3D: w_m hw e^{i k r_m}(2 i k Y'(r_m) + Y''(r_m))
    const double2 *hcheb; // Chebyshev coefficients per panel [hnpan][hdeg + 1]: 3D h(s); 2D (S0, S1)(eta)
    const float2 *hchebf; // the same in float (split plans)
    int hdeg, hnpan;
    double hpan, ihpan; // panel width in s and its inverse
    const double *Pw0;  // [Q] 2D: w_m hw Phi_1(r_m) r_m      (J0 weights)
    const double *Pw1;  // [Q] 2D: w_m hw Phi_1(r_m) r_m^2    (J1 weights)
    double F10;         // 2D: sqrt(V) F1-hat_0
    int TJ2, lg1, lg2;  // x2-pass columns per CTA; log2 M1, log2 M2
    int RB1;            // last-pass rows per CTA
    void *work;         // 3D: [nf][L3count][M2][M1] complex (the transformed x3 planes, compact); 2D: [M2][M1]
    void *grid;         // padded gather grid
    int P1, P2, P3;     // padded extents (M + 3 per periodic axis); P3 = stored x3 planes (1 in 2D)
    int Q3lo;           // padded x3 index of the first stored plane
    int a3first, L3count; // x3 nodes the last two passes transform: a3first .. a3first + L3count - 1
    // Maxwell plans keeping only the x3 >= -h3 planes: 1, and the in-plane
    // transforms P_e of the odd fields' (e = 4, 5: xz, yz) Nyquist row j3 = -M3/2
    // go through the last two passes as work plane L3count of those fields into
    // nyqgrid [P2][P1][2] (padded like the grid)
    int nyq;
    void *nyqgrid;
    // far-region grid: the x3 axis is a run of L3count planes, not periodic; the
    // last pass writes work plane y to grid plane y (no halo, no wrap)
    int zlinear;
    // device error word of the plan: set to 1 when a bounded wait for staged
    // copies ran out (gf_plan_status reports it)
    int *err;
    // fields odd in the last-axis index (bit e: field e; their coefficients are
    // mirrored with a sign): the Maxwell xz, yz fields, the 2D K_2 and T_12 fields
    int oddmask;
    // 2D derivative plans (Sec. 2.4): deriv = 1; fields L, K_1 - h_1, K_2 - h_2,
    // and with k2 > 0 T_11 - h_11, T_12 - h_12, T_22 - h_22.  dcheb: three more
    // Chebyshev tables [3][hnpan][hdeg + 1] on the panels of hcheb, of the Hankel
    // transforms of the cutoff (Q1, R0), (R2, S1), (S3, 0) (see synth.cu)
    int deriv;
    double k2;
    const double2 *dcheb;
};

// Complex entries per target of an output selection (gf_eval_points `which`).
__host__ __device__ inline int gf_out_entries(int which)
{
    return which == GF_OUT_MAXWELL6 ? 6 : which == GF_OUT_MAXWELL7 ? 7 : (which == GF_OUT_GRAD || which == GF_OUT_HESSDIFF) ? 3 : 1;
}

// Far-series table entry for one in-plane index n: b = |beta_n|, ln b and 1/b
// for evanescent n (beta_n = i b); zeros for propagating n (|alpha_n| <= k).
// The double-precision core sums the weights e^{-b|x3|}/b = e^{-(b|x3| + ln b)}.
struct __align__(16) BetaEntry {
    double b, lnb;                // double-precision core terms
    float bf, blo, lnbf, lnblo;   // b and ln b as float pairs (hi + lo): the float-float band; hi parts index the table
};

struct BetaEntryF {
    float bl2, ib, b, pad;  // b log2(e), 1/b, b
};
// Propagating index n: in-plane wave vector alpha_n, real beta_n and 1/beta_n;
// m2 = n2 - N0 (N0 = rint(-alpha_2), exact), first = 0 when the entry before
// it in the list is (n1, n2 - 1), 1 otherwise, the row index n1, and float
// copies of c1, c2, beta_n, 1/beta_n for the float kernels.
struct PropEntry {
    double c1, c2, br, ibr, m2;
    int first, n1;
    float c1f, c2f, brf, ibrf;
};

struct EvalArgs {
    int dim;
    int M1, M2, M3;
    int P1, P2, P3;
    int Q3lo;           // padded x3 index of the grid's first stored plane
    int nf;             // stored fields per node
    int which;
    double k, a1, a2;
    double k2;          // 2D derivative plans: the second wave number of the T fields (0: none)
    double c, ct, eps;
    double h1, h2, h3;  // node spacings
    double T;           // ln(1/series_tol) + 3
    const void *grid;
    const double *x;    // [n][dim]
    void *out;          // [n][entries]
    int64_t n;
    int *far_idx;       // scratch: far-branch target indices, in append order; with
                        // seghist, each target's far bucket instead (-1: not summed)
    int *far_sorted;    // scratch: the same indices ordered by |x_last| bucket (3D)
    int *far_count;     // scratch counters (GF_SCRATCH_COUNTERS ints, zero before each evaluation)
    int *near_idx;      // scratch (3D, may be null): near-branch target indices, in append order
    // far-series slab partials (3D, may be null): [0] for the main far kernel, [1] for
    // the float-tail kernel, each [slab][slot][entries] with slabcap slots per slab set
    // in all (a launch uses at most slabcap / slots-per-slab slabs), and one ticket
    // per 32-target chunk, zero before the evaluation.  Null: slab results are added
    // into the output atomically (in a run-dependent order)
    void *slabbuf[2];
    int *slabtick[2];
    int64_t slabcap;
    // stable far list (3D, may be null): per segment of segsize consecutive targets
    // its far-bucket counts, then the segment's first position in far_sorted for each
    // bucket ([nseg][GF_FAR_BUCKETS]); far_sorted then lists the far targets by
    // descending bucket and ascending index.  Null: the list comes out in the order
    // of the appends (run-dependent)
    int *seghist;
    int segsize, nseg;
    const void *btab;   // far-series table [n1][n2] (BetaEntry or BetaEntryF)
    int n1lo, n1hi, n2lo, n2hi;
    const PropEntry *prop;  // propagating indices (|alpha_n| <= k)
    const int *nprop;       // their number (device)
    const void *nyqgrid;    // Maxwell half grids: in-plane Nyquist transforms of the odd fields ([P2][P1][2]), else null
    // far-region grid (null: far targets by the series): planes [fNZ][fP2][fP1][nf],
    // plane m at z = fz0 + m fhz, in-plane node spacing fh1, fh2 (padded like the
    // near grid); targets with c < |x3| <= fzmax read it
    const void *fargrid;
    int fM1, fM2, fNZ, fP1, fP2;
    double fz0, fhz, fzmax, fh1, fh2;
    const double2 *exptab;  // (e^{-y_j}, y_j), y_j = (j - exptab_j0)/GF_EXPTAB_STEPS, j = 0 .. exptab_n - 1,
                            // followed by exptab_n float4 (hi, lo of e^{-y_j}, y_j, 0)
    int exptab_n, exptab_j0;
    double bmin;            // smallest |beta_n| over the evanescent n (this value or a larger one, never smaller)
};

// Entries per unit of y of the far kernel's exponential table e^{-y_j}
// (a power of two from 128 to 4096).
#ifndef GF_EXPTAB_STEPS
#define GF_EXPTAB_STEPS 4096
#endif

// Far targets are bucketed by b = floor(NB c / |x_last|) (clamped to NB-1) so
// that the lanes of a warp share nearly the same series truncation radius.
#define GF_FAR_BUCKETS 256
// scratch counters: [0] far count, [1..NB] bucket sizes, [NB+1..2NB] cursors,
// [GF_WORK_SLOT] far work items handed out so far, [GF_TAIL_SLOT] the same for
// the float-tail kernel of double-precision plans, [GF_NEAR_SLOT] length of the
// near list
#define GF_WORK_SLOT (1 + 2 * GF_FAR_BUCKETS)
#define GF_TAIL_SLOT (2 + 2 * GF_FAR_BUCKETS)
#define GF_NEAR_SLOT (3 + 2 * GF_FAR_BUCKETS)
// [GF_FGRID_SLOT] far-grid targets, listed from the end of the near list backwards
#define GF_FGRID_SLOT (4 + 2 * GF_FAR_BUCKETS)
#define GF_SCRATCH_COUNTERS (5 + 2 * GF_FAR_BUCKETS)

// A sweep of plans run as batched persistent launches: per-pass virtual-block
// prefix sums over the pairs (device arrays of np + 1 ints), the per-pair
// arguments (device array), persistent grid sizes and shared-memory sizes.
struct SynthBatch {
    const SynthArgs *args;
    const int *prefix[3];
    int np;
    int grid[3];
    size_t smem[3];
};
struct EvalBatch {
    const EvalArgs *args;   // per pair: x, out, n and scratch pointers filled in
    const int *prefix;      // near-kernel tiles (256 targets) per pair, prefix sums (np + 1)
    int np;
    int nf;
    int grid_near, grid_scatter, grid_far, block_far;
    int scatter_per_pair;
    bool near_lists;        // per-pair near lists present (EvalArgs::near_idx): classify, then near3d_list_batch
};

// launch helpers implemented in synth.cu / eval.cu
cudaError_t gf_launch_synth(const SynthArgs &a, int precision, cudaStream_t s);
cudaError_t gf_launch_extract(const SynthArgs &a, int precision, void *dev_out, cudaStream_t s);
void gf_synth_config(SynthArgs &a, int precision, int tj_max, size_t smem[3]);
size_t gf_synth_smem_need(const SynthArgs &a, int precision);
cudaError_t gf_launch_cheb_table(int dim, const double *rr, const double2 *B, const double *P0, const double *P1, int Q,
                                 int npan, int deg, double w, double2 *out, float2 *outf, cudaStream_t s);
// 2D derivative plans: the cutoff's Hankel transform tables (see SynthArgs::dcheb)
cudaError_t gf_launch_cheb_deriv(const double *rr, const double *wy, int Q2, int npan, int deg, double w, double2 *out,
                                 cudaStream_t s);
cudaError_t gf_launch_synth_batch(const SynthBatch &b, int precision, cudaStream_t s);
cudaError_t gf_launch_eval_batch(const EvalBatch &b, int precision, cudaStream_t s);
cudaError_t gf_launch_series_tables(const EvalArgs &a, int precision, double2 *exptab, PropEntry *prop, int *nprop,
                                    const int pbox[4], cudaStream_t s);
cudaError_t gf_launch_e_table(const double *tt, int Q, int Mlast, double qs, double2 *E, float2 *Ef, cudaStream_t s);
// far-region grid: the planes' coefficients into a.work ([nf][L3count][M2][M1], FFT
// order), then the x2 and x1 passes into a.grid (a.zlinear set)
cudaError_t gf_launch_far_grid(const SynthArgs &a, int precision, double k, double a1, double a2, double z0,
                               double hz, cudaStream_t s);

// runtime.cu: stream-ordered pool allocations, pinned upload staging
cudaError_t gf_dev_alloc(void **ptr, size_t bytes, cudaStream_t s);
void gf_dev_free(void *ptr, cudaStream_t s);
cudaError_t gf_stage_upload(void *dev_dst, const void *src, size_t bytes, cudaStream_t s);
cudaError_t gf_trim_pool();
// A side stream and two events: the double-precision far kernel and the
// float-tail kernel run concurrently, the tails on `aux` between `fork` (recorded
// on the caller's stream) and `join` (waited for by the caller's stream).
struct EvalFork {
    cudaStream_t aux;
    cudaEvent_t fork, join;
};
// fork == nullptr: every kernel on stream s, in order
cudaError_t gf_launch_eval(const EvalArgs &a, int precision, cudaStream_t s, cudaEvent_t ev_mid,
                           const EvalFork *fork = nullptr);
// per-device side stream of the library (non-blocking, lives until the process exits)
cudaStream_t gf_aux_stream();
cudaStream_t gf_copy_stream();

void gf_count_launch(int n);
gf_status gf_plan_eval_args(gf_plan_t p, const double *dev_xyz, int64_t n, int which, void *dev_out, EvalArgs *a,
                            const char *who);
gf_status gf_set_error(gf_status s, const char *msg);
SynthArgs gf_plan_synth_args(gf_plan_t p);
size_t gf_plan_work_bytes(gf_plan_t p);
int gf_plan_precision(gf_plan_t p);
