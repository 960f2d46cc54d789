/*
 * gf.h -- C ABI of the GB300 library for quasi-periodic Green's functions by
 * the FFT-based method of B. Zhang & R. Zhang (arXiv:1801.05977).
 *
 * The problem (Sec. 1): for a wave number k > 0 and quasi-periodicity alpha,
 *   2D  G(x)    = (i/4 pi)   sum_n   beta_n^{-1}  exp(i alpha_n x1 + i beta_n |x2|)          Eq. (ei)
 *   3D  G_d(x)  = (i/8 pi^2) sum_n1,n2 beta_n^{-1} exp(i alpha_n . x' + i beta_n |x3|)      Eq. (he)
 *   Maxwell     GG(x) = G_d(x) I + k^{-2} grad grad (G_d(x) I)                             Eq. (me)
 * with alpha_n = alpha + n, beta_n = sqrt(k^2 - |alpha_n|^2) (Im beta >= 0),
 * period 2 pi in x1 (and x2), and no Wood anomaly (beta_n != 0).
 *
 * The method (Algorithms 1, 2, 3): split G into a closed-form singular part
 * near the lattice point and a smooth periodic remainder L; generate L's
 * Fourier coefficients (Eqs. (fck-coef), (fcl-coef)-(fcf2-coef) in 2D,
 * (kdj1) and (fj) in 3D, -c^p c^q multipliers for Maxwell, Sec. 4), synthesise
 * L on a uniform grid by inverse FFT, and at each target reduce to the unit
 * cell, interpolate L by tensor cubics, add the singular part back and apply
 * the quasi-periodic phase; targets with |x_last| > c use the eigen-series.
 *
 * Conventions shared by every entry point:
 *   - All device pointers are plain CUDA device addresses (for example from
 *     torch tensors); host pointers are ordinary host memory (pinned memory
 *     makes the host variants faster).  No entry point takes ownership of a
 *     caller buffer.
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it and the call returns without
 *     synchronising, except where a function says otherwise.
 *   - Every function returns a gf_status; nothing throws across the ABI.  On
 *     failure gf_last_error() returns a thread-local description.
 *   - Complex outputs are interleaved (re, im): complex128 for GF_FP64 plans,
 *     complex64 for GF_FP32_SPLIT plans.
 */
#ifndef GF_H_
#define GF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gf_plan_s *gf_plan_t;

typedef enum {
    GF_OK = 0,
    GF_ERR_ARG = 1,          /* invalid argument (size, pointer, parameter range) */
    GF_ERR_WOOD = 2,         /* some beta_n vanishes (Sec. 1: "away from Wood anomalies") */
    GF_ERR_RESONANCE = 3,    /* beta = +-j_last pi / c~ for some j, policy GF_FAIL (Sec. 2.1, 3.1) */
    GF_ERR_NOMEM = 4,        /* device allocation failed */
    GF_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    GF_ERR_TIMEOUT = 6,      /* a bounded device wait ran out */
    GF_ERR_UNSUPPORTED = 7   /* valid request the library does not implement */
} gf_status;

enum { GF_FP64 = 0, GF_FP32_SPLIT = 1 };          /* gf_trunc_t.precision */
enum { GF_HELMHOLTZ = 0, GF_MAXWELL = 1, GF_DERIV2D = 2 };  /* gf_trunc_t.kind */
enum { GF_PERTURB_CTILDE = 0, GF_FAIL = 1 };      /* gf_trunc_t.resonance_policy */
enum {                                            /* gf_eval_points `which` */
    GF_OUT_G = 0,         /* 2D plans: G, 1 entry */
    GF_OUT_GD = 1,        /* 3D plans: G_d, 1 entry */
    GF_OUT_MAXWELL6 = 2,  /* Maxwell plans: GG_xx, GG_yy, GG_zz, GG_xy, GG_xz, GG_yz */
    GF_OUT_MAXWELL7 = 3,  /* Maxwell plans: the six entries above, then G_d */
    GF_OUT_LD = 4,        /* 3D Helmholtz plans: the interpolated remainder L_dN at the in-cell
                             point (t1, t2, x3), no singular part, no phase (Alg. 2 step 2d);
                             targets with |x3| > c give NaN */
    GF_OUT_GRAD = 5,      /* GF_DERIV2D plans: G, dG/dx1, dG/dx2 (Sec. 2.4.1), 3 entries */
    GF_OUT_HESSDIFF = 6   /* GF_DERIV2D plans with k2 > 0: T_11, T_12, T_22, the differences
                             d_p d_q G_k - d_p d_q G_k2 (Sec. 2.4.2), 3 entries */
};

/* Method parameters.  Defaults (gf_trunc_default): c = 0.6, c~ = 1 (Sec. 5),
 * eps = 0.45, series_tol = 0 (automatic), quad_nodes = 0 (automatic), GF_FP64,
 * GF_HELMHOLTZ, GF_PERTURB_CTILDE, far_grid_M = 0 (far branch by the series).
 *   c          |x_last| <= c: grid + interpolation; > c: eigen-series (Alg. 1-3, step 2b)
 *   c_tilde    half period of the artificial periodisation in x_last (c < c~); the cutoff
 *              X(t) falls from 1 at t = c to 0 at t = (c + c~)/2 (Sec. 2.1)
 *   eps        singular cutoff Y_eps: 1 on [0, eps], 0 beyond 2 eps (Sec. 2.2, 3.2);
 *              requires 2 eps < min(c~, pi)
 *   series_tol far-series truncation: terms with |alpha_n|^2 <= k^2 + (T/|x_last|)^2,
 *              T = ln(1/series_tol) + 3, are summed; <= 0 selects 1e-16 for GF_FP64
 *              and 1e-8 for GF_FP32_SPLIT
 *   quad_nodes Gauss-Legendre nodes Q for the 1D integrals in the coefficients, in
 *              [8, 1024]; <= 0 picks Q from the grid's highest frequencies (the
 *              integrands oscillate like sin(s r) on [eps, 2 eps] with s up to
 *              |xi|_max, and like e^{i(beta -+ q)t} on [c, (c + c~)/2]): Q = max(64,
 *              max(s_max eps/2, (q_max + k)(c~ - c)/4) + 24), rounded up to a
 *              multiple of 8 (64 for the grids of up to about 128 points per axis)
 *   precision  GF_FP64: everything in double.  GF_FP32_SPLIT: grid synthesis,
 *              interpolation and series in float; coefficients, singular part,
 *              reduction and phase in double.
 *   kind       GF_MAXWELL (3D only) stores seven fields per node: the six combined
 *              fields (delta_pq - c^p c^q / k^2) L_d (Sec. 4; one interpolation per
 *              tensor entry) and L_d itself (for G_d)
 *   far_grid_M (3D) 0: far targets (|x3| > c) by the eigen-series (he), as in
 *              Algorithm 2 step 2b.  > 0: the far-region grid, which the paper does
 *              not have: F = e^{-i alpha.t} G_d (and its Maxwell fields) synthesised
 *              on planes z_m = c + (m - 1) hz, m = 0 .. far_grid_nz + 2, hz =
 *              (far_grid_zmax - c)/far_grid_nz, each by an inverse FFT of the series
 *              terms (i/8pi^2) e^{i beta_n z_m}/beta_n over far_grid_M x far_grid_M
 *              in-plane indices (a power of two in [16, 2048]), then far targets with
 *              |x3| <= far_grid_zmax interpolated by tensor cubics like the near
 *              branch (the others keep the series).  Interpolation caps its accuracy
 *              at O(h^4): about 1.4e-5 (M = 128), 7e-7 (256), 5e-8 (512) relative
 *              to max|G| at c = 0.6; meant for GF_FP32_SPLIT plans.
 *   far_grid_nz  intervals in z (0: 16); far_grid_zmax  end of the slab (<= 0: c~)
 *   kind = GF_DERIV2D (2D only): the plan also serves the derivatives of Sec. 2.4.
 *              It stores, beside L of Eq. (fcl-coef), the remainder fields K_1 - h_1
 *              and K_2 - h_2 (Sec. 2.4.1: K_1 = e^{-i alpha x1} dG/dx1, K_2 =
 *              e^{-i alpha x1} dG/dx2, coefficients i (alpha + j1) K-hat and
 *              i (j2 pi/c~) K-hat less those of the singular parts h_1, h_2), and
 *              with k2 > 0 the fields T_pq - h_pq of the differences of second
 *              derivatives for wave numbers k and k2 (Sec. 2.4.2, coefficients
 *              -(alpha+j1)^2, -(alpha+j1)(j2 pi/c~), -(j2 pi/c~)^2 times K-hat(k) -
 *              K-hat(k2), less h_11, h_12, h_22's).  The singular parts are the
 *              paper's with two readings: x2 ln|x| (not x1 ln|x|) in h_2, and the sign
 *              +(k^2 - k2^2)/2pi of h_11, h_12, h_22.  The x2-derivative fields carry
 *              the cutoff X's transition multiplied by j2 or j2^2 and converge once
 *              the grid resolves it: a wider window c~ - c (c~ = 1.4 at c = 0.6, say)
 *              or more points along x2 (errors against the exact series, c~ = 1.4,
 *              M = 128^2: dG/dx1 2.7e-4, dG/dx2 6.4e-5, T 3.5e-4 .. 4.3e-3 of max)
 *   k2         second wave number of GF_DERIV2D plans (0: the gradient only); must
 *              be 0 for the other kinds
 */
typedef struct {
    double c, c_tilde, eps;
    double series_tol;
    int quad_nodes;
    int precision;
    int kind;
    int resonance_policy;
    int far_grid_M, far_grid_nz;
    double far_grid_zmax;
    double k2;
} gf_trunc_t;

/* Fill *t with the defaults listed above.  Returns GF_ERR_ARG if t is NULL. */
gf_status gf_trunc_default(gf_trunc_t *t);

/* Build a plan (Algorithms 1-3, step 1 "Preparation"): check the parameters,
 * generate the remainder's Fourier coefficients on S_N in double precision and
 * synthesise the grid by inverse FFT on the device.
 *   dim        2 (G, Sec. 2) or 3 (G_d / GG, Secs. 3-4)
 *   k          wave number, > 0
 *   alpha      dim-1 doubles (host memory)
 *   M          dim ints (host memory): grid points per axis (x1, x2[, x3]) = the
 *              paper's 2N; each a power of two in [8, 1024] (3D) or [8, 2048] (2D)
 *   trunc      parameters, NULL for the defaults
 *   cuda_stream  stream on which the synthesis kernels run
 *   out        receives the plan handle; the plan owns its device memory
 * Device memory comes from the library's stream-ordered memory pool on
 * cuda_stream; the coefficient and FFT kernels are enqueued on cuda_stream (the
 * plan is usable by later work on that stream, and by work on other streams
 * once they are ordered after it).  The plan is immutable afterwards.
 * Errors: GF_ERR_ARG (bad sizes/parameters), GF_ERR_WOOD, GF_ERR_RESONANCE,
 * GF_ERR_NOMEM, GF_ERR_CUDA, GF_ERR_UNSUPPORTED (a synthesis pass would need
 * more shared memory than one CTA has: double-precision Maxwell plans with
 * 1024 points on an axis).  On error *out is set to NULL. */
gf_status gf_plan(int dim, double k, const double *alpha, const int *M,
                  const gf_trunc_t *trunc, void *cuda_stream, gf_plan_t *out);

/* Copy the synthesised remainder grid L_N (Eqs. (fcln), (ln)) to dev_out in
 * node order [field][l3][l2][l1] (l_i = 0..M_i-1 is the node x_i = l_i h_i
 * modulo the period, h = 2 pi / M in-plane and 2 c~ / M_last in x_last).  One
 * field for Helmholtz plans; for Maxwell plans seven: the six combined fields
 * (delta_pq - c^p c^q / k^2) L_d in the order xx, yy, zz, xy, xz, yz, then L_d;
 * for GF_DERIV2D plans three (L, K_1 - h_1, K_2 - h_2) or, with k2 > 0, six
 * (then T_11 - h_11, T_12 - h_12, T_22 - h_22).
 * out_bytes must be >= gf_grid_bytes(plan).  Errors: GF_ERR_ARG, GF_ERR_CUDA. */
gf_status gf_eval_grid(gf_plan_t plan, void *dev_out, size_t out_bytes, void *cuda_stream);

/* Bytes gf_eval_grid writes (0 for a NULL plan). */
size_t gf_grid_bytes(gf_plan_t plan);

/* Evaluate at n targets (Algorithms 1-3, step 2 "Calculation").
 *   dev_xyz   n * dim doubles, row-major [n][dim], device memory
 *   which     GF_OUT_G (2D), GF_OUT_GD (3D Helmholtz), GF_OUT_MAXWELL6/7 (Maxwell),
 *             GF_OUT_GRAD and GF_OUT_HESSDIFF (GF_DERIV2D plans; the latter with k2 > 0)
 *   dev_out   n * entries complex values, [n][entries], device memory
 * The plan is not modified by an evaluation: each call takes its scratch (the
 * far- and near-branch target lists, 12 bytes per target plus 4 KiB; for 3D
 * plans also about 2.3 bytes per target of far-list counts and tickets and the
 * far sums' slab partials, 4 * entries * (8 or 16) bytes per target for float or
 * double plans) from the library's stream-ordered memory pool on cuda_stream
 * and returns it in stream order, so calls on one plan may run concurrently on
 * different streams and threads.  Results are reproducible: the same plan and
 * targets give the same bits at every call (the far targets are grouped by a
 * stable sort, and each far sum adds its row-slab partials in slab order).
 * For 3D double-precision Helmholtz plans
 * part of the far series runs on a side stream that the library owns (one per
 * device): it waits for an event recorded on cuda_stream and cuda_stream waits
 * for its completion, so the call keeps the ordinary stream semantics.
 * Non-finite targets give NaN
 * outputs; targets on a lattice point give non-finite outputs.
 * Errors: GF_ERR_ARG (n < 0, NULL pointers with n > 0, `which` not valid for the
 * plan), GF_ERR_NOMEM, GF_ERR_CUDA. */
gf_status gf_eval_points(gf_plan_t plan, const double *dev_xyz, int64_t n, int which,
                         void *dev_out, void *cuda_stream);

/* As gf_eval_points, with HOST input and output buffers: copies the targets to
 * the device, evaluates and copies the results back, then synchronises
 * cuda_stream.  The upload runs on a copy stream the library owns (one per
 * device) and the evaluation on cuda_stream waits for it, so the upload overlaps
 * work already queued on cuda_stream (for example the synthesis of a plan just
 * created); host_xyz is therefore read as soon as the call is made, not in
 * cuda_stream's order.  The device staging buffers are taken from the library's
 * memory pool per call. */
gf_status gf_eval_points_host(gf_plan_t plan, const double *host_xyz, int64_t n, int which,
                              void *host_out, void *cuda_stream);

/* Allocation-free variant of gf_eval_points.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * while they evaluate, for example a solver that reserved all free device
 * memory for its own pool at start-up, or a latency-critical loop in which a
 * cudaMalloc/cudaFree (which can synchronise the whole device) is not
 * acceptable.  gf_eval_points takes its scratch lists from the library's
 * memory pool at every call, which reaches the driver whenever the pool has to
 * grow; this function instead uses one
 * fixed scratch array compiled into the library (about 2 MiB: room for
 * GF_NOALLOC_MAX_TARGETS targets), which every GPU that loads the library
 * holds until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   Arguments, layout and results are those of gf_eval_points; n must be
 *   <= GF_NOALLOC_MAX_TARGETS, otherwise GF_ERR_ARG is returned and nothing is
 *   launched.  The plan itself must already exist (gf_plan allocates).
 *   The first call on each device looks up the device address of the scratch
 *   array (cudaGetSymbolAddress) with that device current; make that first
 *   call before any stream capture.
 *   All calls share the one scratch array: each call resets its counters on
 *   cuda_stream before use, and calls of this function whose work overlaps on
 *   the GPU (other streams, other threads) race on it and give wrong results;
 *   serialise them.  Calls of gf_eval_points on the same plan do not touch the
 *   array and may overlap with it.  The plan is only read (no per-plan state,
 *   no fork/join events, so no lock is taken): calls of gf_eval_points and
 *   gf_eval_grid on the same plan may run alongside; gf_destroy may not, as for
 *   every other call on the plan.
 *   The far sums' row slabs are added into the outputs atomically here (there
 *   is no room for their partials), so results agree with gf_eval_points' to
 *   rounding (about 1e-16 of max|G| for double plans), not bit for bit.
 *   The device address found at the first call is kept for the life of the
 *   process: the library (this array, its memory pool and its side streams) is
 *   not usable across a cudaDeviceReset.
 * Errors: GF_ERR_ARG, GF_ERR_CUDA, GF_ERR_UNSUPPORTED (device ordinal >= 64). */
#define GF_NOALLOC_MAX_TARGETS (1 << 18)
gf_status gf_eval_points_noalloc(gf_plan_t plan, const double *dev_xyz, int64_t n, int which,
                                 void *dev_out, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Batched (alpha, k) sweeps.  Many plans with their own k, alpha and grid
 * (Algorithms 1-3 applied pair by pair, as in a Bloch or frequency sweep) run
 * as batched persistent launches over a (pair, block) work list: three
 * launches re-synthesise every pair's grid, a counter reset and three
 * launches evaluate every pair's targets.  3D plans only (Secs. 3-4).
 * ------------------------------------------------------------------------- */
typedef struct gf_batch_s *gf_batch_t;

/* Build one plan per pair (as gf_plan; grids are synthesised once on
 * cuda_stream) plus the batch's work arena and launch tables.
 *   npairs  number of pairs, >= 1
 *   k       [npairs] wave numbers;  alpha [npairs][2];  M [npairs][3]  (host memory)
 *   trunc   shared parameters (precision, kind, ...), NULL for the defaults
 * Errors: as gf_plan for any pair (the message names the pair), GF_ERR_NOMEM,
 * GF_ERR_UNSUPPORTED for kind GF_DERIV2D (derivative plans are single plans). */
gf_status gf_plan_batch(int npairs, const double *k, const double *alpha, const int *M,
                        const gf_trunc_t *trunc, void *cuda_stream, gf_batch_t *out);

/* Re-run the synthesis (coefficients + inverse FFTs) of every pair: three
 * batched persistent launches on cuda_stream. */
gf_status gf_batch_synthesize(gf_batch_t batch, void *cuda_stream);

/* Evaluate every pair at its own targets.  dev_xyz holds all targets,
 * [offsets[npairs]][3] doubles, pair p owning rows offsets[p] .. offsets[p+1]-1;
 * dev_out receives [offsets[npairs]][entries] complex values in the same rows.
 * offsets is host memory (npairs + 1 entries, offsets[0] = 0, non-decreasing).
 * The batch owns the scratch (grown synchronously when a call brings more
 * targets than before); calls on one batch must not overlap in time. */
gf_status gf_batch_eval_points(gf_batch_t batch, const double *dev_xyz, const int64_t *offsets, int which,
                               void *dev_out, void *cuda_stream);

/* Choose the launch shapes (first-pass columns per CTA; far-kernel block size
 * and CTAs per SM) by timing candidates on this batch and these targets, then
 * keep them for this batch and for later batches of the same shape in this
 * process.  Synchronises the stream; overwrites dev_out. */
gf_status gf_batch_autotune(gf_batch_t batch, const double *dev_xyz, const int64_t *offsets, int which,
                            void *dev_out, void *cuda_stream);

/* The chosen shapes: out[0] first-pass columns per CTA (cap), out[1] far-kernel
 * block size, out[2] far-kernel 128-thread CTAs per SM. */
gf_status gf_batch_get_tuning(gf_batch_t batch, int out[3]);

/* Synthesis + evaluation of the whole sweep as one CUDA graph: captured on
 * cuda_stream (which must not be the legacy default stream) at the first call
 * for given (dev_xyz, offsets, which, dev_out), then replayed. */
gf_status gf_batch_run_graph(gf_batch_t batch, const double *dev_xyz, const int64_t *offsets, int which,
                             void *dev_out, void *cuda_stream);

/* Borrow the plan of pair i (owned by the batch; do not destroy it). */
gf_status gf_batch_get_plan(gf_batch_t batch, int i, gf_plan_t *out);

/* Release the batch, its plans and graphs (synchronises the device).  NULL is accepted. */
gf_status gf_batch_destroy(gf_batch_t batch);

/* ---------------------------------------------------------------------------
 * Tensor-core BF16 GEMM (the building block of the surrogate below):
 *   C[M x N] (fp32, row stride ldc) = A . B^T with A(m,k) = A[m*lda + k]
 *   (a_trans: A[k*lda + m]) and B(n,k) = B[n*ldb + k] (b_trans: B[k*ldb + n]),
 *   bf16 operands, fp32 accumulation in tensor memory (tcgen05).  M, N, K
 *   positive multiples of 16; leading dimensions multiples of 8 elements and
 *   pointers 16-byte aligned.  ksplit > 1 splits K over CTAs (C is zeroed and
 *   accumulated atomically).  All pointers are device memory. */
gf_status gf_gemm_bf16(const void *A, int64_t lda, int a_trans, const void *B, int64_t ldb, int b_trans,
                       int M, int N, int K, float *C, int64_t ldc, int ksplit, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Learned surrogate of the smooth remainder L_d (spec extension; the
 * paper has no learned part).  A 5-layer MLP 80 -> 256 -> 256 -> 256 -> 256 -> 2
 * with SiLU activations: bf16 weights and activations, fp32 accumulation on the
 * tensor cores, fp32 master weights with Adam.  Inputs per sample, float
 * [n][6]: (t1, t2, x3, alpha1, alpha2, k) with t the in-cell coordinates; the
 * 80 features are cos/sin of n1 t1 + n2 t2 + m3 pi x3 / c~ for 32 fixed integer
 * vectors, then 2 alpha1, 2 alpha2, (k - 2.5)/1.5, the in-cell radius r and 12
 * Gaussian radial bumps exp(-((r - 0.15 j)/0.15)^2 / 2), j = 0..11.  Output
 * float [n][2]: the real and imaginary parts of L_d / scale.
 * ------------------------------------------------------------------------- */
typedef struct gf_mlp_s *gf_mlp_t;

/* Create a network with uniform(+-1/sqrt(fan_in)) weights drawn from `seed`
 * (counter-based, reproducible) and zero biases; c_tilde sets the x3 period. */
gf_status gf_mlp_create(uint64_t seed, double c_tilde, gf_mlp_t *out);
/* Number of floats of gf_mlp_params: per layer W [out][in] then b [out]. */
int64_t gf_mlp_param_count(void);
/* Copy the fp32 parameters to (to_device = 0) or from (to_device = 1) host
 * memory (checkpointing; gradient checks).  Synchronises the device. */
gf_status gf_mlp_params(gf_mlp_t mlp, float *host, int64_t count, int to_device);
/* Scale of the targets: the network learns L_d / scale. */
gf_status gf_mlp_set_scale(gf_mlp_t mlp, double scale);
/* Forward pass of n samples (device pointers), output float [n][2]: one fused
 * persistent tensor-core kernel (activations stay on chip). */
gf_status gf_mlp_forward(gf_mlp_t mlp, const float *dev_in, int n, float *dev_out, void *cuda_stream);
/* One Adam step (lr; beta 0.9/0.999) on the mean-squared loss
 * sum (Y - T)^2 / (2n) of one batch (targets float [n][2]); the batch loss is
 * written to dev_loss (device float) when not NULL. */
gf_status gf_mlp_train_step(gf_mlp_t mlp, const float *dev_in, const float *dev_target, int n, float lr,
                            float *dev_loss, void *cuda_stream);
/* Gradients of that loss (no update), copied to host in the layout of
 * gf_mlp_params; the loss to *host_loss when not NULL.  Synchronises. */
gf_status gf_mlp_gradients(gf_mlp_t mlp, const float *dev_in, const float *dev_target, int n, float *host_grads,
                           float *host_loss, void *cuda_stream);
/* Tensor-core error word (1 after a bounded wait ran out): GF_ERR_TIMEOUT if set. */
gf_status gf_mlp_error_word(gf_mlp_t mlp, int *out);
/* G_d at near targets (|x3| <= c) of many (alpha, k) pairs, with the network
 * standing in for the interpolated remainder: G = e^{i2pi<alpha.m>}(e^{i alpha.t}
 * scale*MLP + e^{ikr} Y_eps/(4 pi r)).  Pairs whose Wood distance
 * min_n | |alpha_n| - k | is below wood_delta are evaluated by the FFT path
 * instead (a 128 x 128 x 64 double-precision plan); their count is written to
 * *n_fallback_pairs.  k [npairs], alpha [npairs][2], offsets [npairs + 1] are host
 * memory; dev_xyz [offsets[npairs]][3] doubles and dev_out complex128 are device
 * memory.  Targets with |x3| > c get NaN (outside the surrogate's domain).
 * Stream-ordered on cuda_stream: without fallback pairs the call returns once the
 * work is queued (the host arrays may be reused at once); fallback pairs are
 * evaluated before it returns. */
gf_status gf_surrogate_eval(gf_mlp_t mlp, int npairs, const double *k, const double *alpha, const int64_t *offsets,
                            const double *dev_xyz, void *dev_out, double wood_delta, const gf_trunc_t *trunc,
                            int *n_fallback_pairs, void *cuda_stream);
/* Residual form of gf_surrogate_eval (the surrogate's fallback design when the
 * network alone cannot reach the FFT path's accuracy; the paper has no learned
 * part): the network was trained on L_d minus a coarse FFT-path value of it, and
 * the caller passes that coarse value at every target,
 *   dev_base  complex128 [offsets[npairs]] device memory: the remainder L_d of a
 *             coarse plan per pair at the same targets (for example gf_plan_batch
 *             with 32^3 points and gf_batch_eval_points(..., GF_OUT_LD, ...)),
 * so that G = e^{i2pi<alpha.m>}(e^{i alpha.t}(L_base + scale*MLP) + e^{ikr} Y_eps/(4 pi r)).
 * Everything else as gf_surrogate_eval.  Errors: as gf_surrogate_eval;
 * GF_ERR_ARG for a NULL dev_base with targets. */
gf_status gf_surrogate_eval_residual(gf_mlp_t mlp, int npairs, const double *k, const double *alpha,
                                     const int64_t *offsets, const double *dev_xyz, const void *dev_base,
                                     void *dev_out, double wood_delta, const gf_trunc_t *trunc,
                                     int *n_fallback_pairs, void *cuda_stream);
gf_status gf_mlp_destroy(gf_mlp_t mlp);

/* Device status of a plan's synthesis: the inverse-FFT passes stage their tiles
 * with TMA copies completed on mbarriers, and every such wait has a poll limit;
 * a wait that ran out sets the plan's device error word instead of hanging.
 * Synchronises cuda_stream, then returns GF_ERR_TIMEOUT if the word is set,
 * GF_OK otherwise.  Errors: GF_ERR_ARG, GF_ERR_CUDA. */
gf_status gf_plan_status(gf_plan_t plan, void *cuda_stream);

/* Plan facts (host memory).  Returns GF_ERR_ARG on NULL arguments. */
typedef struct {
    int dim, M[3], nfields, precision, kind;
    double k, alpha[2];
    double c, c_tilde, eps, series_tol;  /* c_tilde after any resonance perturbation */
    int quad_nodes;
    int series_n1_lo, series_n1_hi, series_n2_lo, series_n2_hi; /* far-series index box */
    size_t grid_device_bytes;            /* padded gather grid held by the plan */
    int far_grid_M, far_grid_nz;         /* far-region grid (0: none) */
    double far_grid_zmax;
    size_t far_grid_device_bytes;
    double k2;                           /* second wave number of GF_DERIV2D plans (0: none) */
} gf_plan_info_t;
gf_status gf_plan_get_info(gf_plan_t plan, gf_plan_info_t *info);

/* Release the plan (synchronises the device first).  NULL is accepted.  Its
 * device buffers go back to the library's memory pool, which keeps freed
 * memory reserved so that the next plan's allocations do not reach the driver
 * (plans and their evaluation scratch are allocated stream-ordered from this
 * pool on the stream passed to gf_plan / gf_eval_points). */
gf_status gf_destroy(gf_plan_t plan);

/* Return the memory the library's pool holds for the current device and no
 * live plan uses to the driver (synchronises the device).  GF_ERR_CUDA on a
 * driver error. */
gf_status gf_release_memory(void);

/* Arithmetic peak probe (diagnostic; the paper has no counterpart): one launch
 * of independent fused multiply-add chains filling every SM, for measuring the
 * FP64 (pipe = GF_PROBE_FP64) or FP32 (GF_PROBE_FP32) pipe's rate, which the
 * far-series roofline divides by.  The caller times the launch on cuda_stream
 * (CUDA events) and divides *flops (host; an FMA counts 2) by the time.
 * The overlap modes run FP64 chains on the even warps and FP32 chains
 * (GF_PROBE_FP32_PER_FP64 times as many trips) on the odd ones: only the FP64
 * half (GF_PROBE_FP64_HALF), only the FP32 half (GF_PROBE_FP32_HALF) or both
 * (GF_PROBE_BOTH_HALVES); both taking the longer of the halves' times means
 * the two pipes overlap, their sum that they do not.
 *   iters     loop trips per thread (each trip is 64 FMAs per thread),
 *             1 <= iters <= 2^20
 *   dev_sink  device buffer of at least 8 bytes (written only to keep the
 *             chains alive; its content is meaningless)
 * Errors: GF_ERR_ARG, GF_ERR_CUDA. */
enum { GF_PROBE_FP64 = 0, GF_PROBE_FP32 = 1, GF_PROBE_FP64_HALF = 2, GF_PROBE_FP32_HALF = 3, GF_PROBE_BOTH_HALVES = 4 };
#define GF_PROBE_FP32_PER_FP64 64
gf_status gf_peak_probe(int pipe, int64_t iters, void *dev_sink, int64_t *flops, void *cuda_stream);

/* Self-test of the bounded device waits (diagnostic; the paper has no
 * counterpart).  The tensor-core kernels wait on mbarriers with a poll limit and
 * report GF_ERR_TIMEOUT instead of hanging; this launches one warp that waits
 * the same way on a barrier that only it could arrive on, with `polls` polls,
 * arriving first when `arrive` is non-zero.  Synchronises cuda_stream.
 * Returns GF_ERR_TIMEOUT when the wait ran out (arrive = 0), GF_OK when it
 * completed (arrive != 0); the context stays usable either way.
 * Errors: GF_ERR_ARG (polls outside [1, 2^40]), GF_ERR_NOMEM, GF_ERR_CUDA. */
gf_status gf_wait_selftest(int64_t polls, int arrive, void *cuda_stream);

/* Static description of a status code. */
const char *gf_status_string(gf_status s);

/* Thread-local description of the last failure in this thread ("" if none). */
const char *gf_last_error(void);

/* Number of kernels the library enqueued from this process so far (all
 * threads); used to report launch counts. */
int64_t gf_launch_count(void);

/* Per-phase device timing (tracing).  With gf_set_phase_timing(1), plans
 * created afterwards record CUDA events around their phases on the stream they
 * run on: synthesis (coefficients + all inverse-FFT passes), the far-series
 * table, and, for each gf_eval_points call, the near kernel and the far
 * kernel.  gf_plan_phase_ms synchronises on those events and writes
 * ms[0] synthesis, ms[1] far-series table, ms[2] near kernel, ms[3] far
 * kernel of the latest plan build / evaluation (-1 where nothing was
 * recorded).  Timing is off by default; turning it off affects later plans. */
gf_status gf_set_phase_timing(int on);
gf_status gf_plan_phase_ms(gf_plan_t plan, float ms[4]);

#ifdef __cplusplus
}
#endif
#endif /* GF_H_ */
