// Learned surrogate of the smooth remainder L_d (not in the paper): a 5-layer
// BF16 MLP with FP32 accumulation on the tensor cores (tcgen05 GEMMs of
// umma_gemm.cuh), Fourier-feature inputs of (t1, t2, x3) plus (alpha1, alpha2, k),
// trained by the library's own forward, backward and Adam kernels on samples of
// the FFT path, and evaluated with the FFT path as fallback near Wood anomalies.
//
// Network: 80 -> 256 -> 256 -> 256 -> 256 -> 2 (Re, Im of L_d / scale), SiLU
// between layers.  Input features: cos and sin of n1 t1 + n2 t2 + m3 pi x3 / c~
// for 32 fixed integer vectors (n1, n2, m3) (|n_i| <= 3, m3 <= 3), then
// 2 alpha1, 2 alpha2, (k - 2.5)/1.5, then the in-cell distance r = |(t, x3)| and
// 12 Gaussian shells of r (the remainder's main structure is radial: the
// transition of the singular cutoff around the lattice point).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "gf_internal.cuh"
#include "umma_gemm.cuh"

typedef __nv_bfloat16 bf16;

namespace {

constexpr int K0 = 80, HID = 256, NL = 5;
const int IN_DIM[NL] = {K0, HID, HID, HID, HID};
const int OUT_DIM[NL] = {HID, HID, HID, HID, 2};

// the 32 frequency vectors (n1, n2, m3) of the Fourier features
__constant__ int c_freq[32][3];

gf_status err(gf_status s, const char *fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    return gf_set_error(s, msg);
}

#define CUM(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return err(e_ == cudaErrorMemoryAllocation ? GF_ERR_NOMEM : GF_ERR_CUDA, "%s: %s", #call, \
                       cudaGetErrorString(e_));                                                    \
    } while (0)

// counter-based uniform in [0, 1) (splitmix64 finaliser)
__host__ __device__ inline double u01(unsigned long long seed, unsigned long long i)
{
    unsigned long long z = seed * 0x9E3779B97F4A7C15ull + i * 0xBF58476D1CE4E5B9ull + 0x94D049BB133111EBull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void features_kernel(const float *in, int n, bf16 *X0, float pi_ct)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float *p = in + 6 * (size_t)i;
        const float t1 = p[0], t2 = p[1], x3 = p[2];
        bf16 *o = X0 + (size_t)i * K0;
#pragma unroll 4
        for (int f = 0; f < 32; ++f) {
            float ph = c_freq[f][0] * t1 + c_freq[f][1] * t2 + c_freq[f][2] * pi_ct * x3;
            float s, c;
            sincosf(ph, &s, &c);
            o[2 * f] = __float2bfloat16(c);
            o[2 * f + 1] = __float2bfloat16(s);
        }
        o[64] = __float2bfloat16(2.f * p[3]);
        o[65] = __float2bfloat16(2.f * p[4]);
        o[66] = __float2bfloat16((p[5] - 2.5f) / 1.5f);
        // radial features of the in-cell distance to the lattice point: r and
        // Gaussian shells exp(-((r - 0.15 j)/0.15)^2 / 2), j = 0..11
        const float r = sqrtf(t1 * t1 + t2 * t2 + x3 * x3);
        o[67] = __float2bfloat16(r);
        for (int j = 0; j < 12; ++j) {
            const float d = (r - 0.15f * j) * (1.f / 0.15f);
            o[68 + j] = __float2bfloat16(__expf(-0.5f * d * d));
        }
    }
}

// Y = H4 W5^T + b5 (one warp per sample); with targets: loss += sum (Y - T)^2 / (2n), dY = (Y - T)/n
__global__ void head_fwd_kernel(const bf16 *H4, const float *W5, const float *b5, float *Y, int n, const float *T,
                                float *dY, float *loss, float invn)
{
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    float lsum = 0.f;
    for (int i = w; i < n; i += nw) {
        float a0 = 0.f, a1 = 0.f;
        for (int j = lane; j < HID; j += 32) {
            float h = __bfloat162float(H4[(size_t)i * HID + j]);
            a0 = fmaf(h, W5[j], a0);
            a1 = fmaf(h, W5[HID + j], a1);
        }
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        }
        if (lane == 0) {
            float y0 = a0 + b5[0], y1 = a1 + b5[1];
            Y[2 * (size_t)i] = y0;
            Y[2 * (size_t)i + 1] = y1;
            if (T) {
                float d0 = y0 - T[2 * (size_t)i], d1 = y1 - T[2 * (size_t)i + 1];
                dY[2 * (size_t)i] = d0 * invn;
                dY[2 * (size_t)i + 1] = d1 * invn;
                lsum += 0.5f * (d0 * d0 + d1 * d1) * invn;
            }
        }
    }
    if (T && lane == 0 && lsum != 0.f) atomicAdd(loss, lsum);
}

// dZ4 = (dY W5) * silu'(Z4)
__global__ void head_bwd_kernel(const float *dY, const float *W5, const bf16 *Z4, bf16 *dZ4, int n)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * HID;
         e += (size_t)gridDim.x * blockDim.x) {
        size_t i = e / HID;
        int j = (int)(e % HID);
        float d = dY[2 * i] * W5[j] + dY[2 * i + 1] * W5[HID + j];
        dZ4[e] = __float2bfloat16(d * umma::dsilu(__bfloat162float(Z4[e])));
    }
}

// gW5[o][j] += sum_i dY[i][o] H4[i][j]; gb5[o] += sum_i dY[i][o]   (block: 256 threads = columns j)
__global__ void head_wgrad_kernel(const float *dY, const bf16 *H4, float *gW5, float *gb5, int n, int rows_per_block)
{
    const int j = threadIdx.x;
    const int i0 = blockIdx.x * rows_per_block, i1 = min(n, i0 + rows_per_block);
    float s0 = 0.f, s1 = 0.f, t0 = 0.f, t1 = 0.f;
    for (int i = i0; i < i1; ++i) {
        float h = __bfloat162float(H4[(size_t)i * HID + j]);
        float d0 = dY[2 * (size_t)i], d1 = dY[2 * (size_t)i + 1];
        s0 = fmaf(d0, h, s0);
        s1 = fmaf(d1, h, s1);
        if (j == 0) {
            t0 += d0;
            t1 += d1;
        }
    }
    atomicAdd(&gW5[j], s0);
    atomicAdd(&gW5[HID + j], s1);
    if (j == 0) {
        atomicAdd(&gb5[0], t0);
        atomicAdd(&gb5[1], t1);
    }
}

// gb[j] += sum_i dZ[i][j]
__global__ void bias_grad_kernel(const bf16 *dZ, float *gb, int n, int rows_per_block)
{
    const int j = threadIdx.x;
    const int i0 = blockIdx.x * rows_per_block, i1 = min(n, i0 + rows_per_block);
    float s = 0.f;
    for (int i = i0; i < i1; ++i) s += __bfloat162float(dZ[(size_t)i * HID + j]);
    atomicAdd(&gb[j], s);
}

// Adam (Kingma & Ba) on one flat parameter array
__global__ void adam_kernel(float *w, const float *g, float *m, float *v, int count, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// bf16 copies W [out][in] and W^T [in][out]
__global__ void convert_kernel(const float *W, bf16 *Wb, bf16 *WTb, int out, int in)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < out * in; e += gridDim.x * blockDim.x) {
        int o = e / in, i = e % in;
        bf16 b = __float2bfloat16(W[e]);
        Wb[e] = b;
        WTb[(size_t)i * out + o] = b;
    }
}

// Shared-memory images of a layer's weight stages for the fused inference kernel:
// chunk c (32 KiB) holds rows 0..HID-1, K range [c KC, (c + 1) KC) of the bf16
// weights W [HID][K] in the core-matrix layout of the B operand (zero beyond K), so
// that one bulk copy puts a stage in place.
__global__ void stage_images_kernel(const bf16 *W, int K, int nch, bf16 *img)
{
    constexpr int CH = HID * (umma::KC / 8);  // 16-byte pieces per stage
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nch * CH; i += gridDim.x * blockDim.x) {
        const int c = i / CH, rem = i - c * CH;
        const int r = rem / (umma::KC / 8), kb = rem - r * (umma::KC / 8);
        const int gk = c * umma::KC + kb * 8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gk < K) v = *reinterpret_cast<const uint4 *>(W + (size_t)r * K + gk);
        *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(img) + (size_t)c * (HID * umma::KC * 2) +
                                   umma::core_off(r, kb * 8)) = v;
    }
}

__global__ void init_kernel(float *W, int count, float bound, unsigned long long seed)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        W[i] = (float)((2.0 * u01(seed, i) - 1.0) * bound);
}

// pair of target i from the offsets (largest p with off[p] <= i)
__device__ __forceinline__ int pair_of_target(const int64_t *off, int np, int64_t i)
{
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Surrogate inputs of near targets: (t1, t2, x3, alpha1, alpha2, k) in float,
// with the pair of each target from the offsets.
__global__ void surrogate_inputs_kernel(const double *x, int n, int64_t base, const int64_t *off, int np,
                                        const double *pk, float *in)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = pair_of_target(off, np, base + i);
        // cell reduction by a multiply (the network's features are periodic in t,
        // so a cell choice off by one at a boundary changes nothing)
        const double x1 = x[3 * (size_t)i], x2 = x[3 * (size_t)i + 1];
        const double t1 = fma(-2.0 * GF_PI, floor(fma(x1, 0.5 / GF_PI, 0.5)), x1);
        const double t2 = fma(-2.0 * GF_PI, floor(fma(x2, 0.5 / GF_PI, 0.5)), x2);
        float *o = in + 6 * (size_t)i;
        o[0] = (float)t1;
        o[1] = (float)t2;
        o[2] = (float)x[3 * (size_t)i + 2];
        o[3] = (float)pk[3 * p];
        o[4] = (float)pk[3 * p + 1];
        o[5] = (float)pk[3 * p + 2];
    }
}

// G = e^{i2pi<alpha.m>} (e^{i alpha.t} L + e^{ikr} Y_eps(r)/(4 pi r)) for near targets
// (L = scale * network output, plus the caller's base value of the remainder
// when Lb is not null: the residual form); far targets (|x3| > c) are outside
// the surrogate's domain and get NaN.
__global__ void surrogate_assemble_kernel(const double *x, int n, int64_t base, const int64_t *off, int np,
                                          const double *pk, const float *Y, double scale, double c, double eps,
                                          const double2 *Lb, double2 *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = pair_of_target(off, np, base + i);
        const double a1 = pk[3 * p], a2 = pk[3 * p + 1], k = pk[3 * p + 2];
        const double x1 = x[3 * (size_t)i], x2 = x[3 * (size_t)i + 1], x3 = x[3 * (size_t)i + 2];
        if (!(fabs(x3) <= c)) {
            out[i] = make_double2(nan(""), nan(""));
            continue;
        }
        // the reduction and the lattice phase's fractional part in double (a few
        // operations), the rest in float: the network's error (~1e-1) is far
        // above float rounding; the singular part (targets within 2 eps of a
        // lattice point, ~1%) stays in double
        const double m1 = floor(fma(x1, 0.5 / GF_PI, 0.5)), m2 = floor(fma(x2, 0.5 / GF_PI, 0.5));
        const double t1 = fma(-2.0 * GF_PI, m1, x1), t2 = fma(-2.0 * GF_PI, m2, x2);
        double ph = a1 * m1 + a2 * m2;
        ph -= rint(ph);
        float sl, cl, sa, ca;
        sincospif(2.0f * (float)ph, &sl, &cl);
        const float t1f = (float)t1, t2f = (float)t2, x3f = (float)x3;
        sincosf((float)a1 * t1f + (float)a2 * t2f, &sa, &ca);
        const float lx = ca * cl - sa * sl, ly = ca * sl + sa * cl;  // lift
        const float sc = (float)scale;
        float Lx = sc * Y[2 * (size_t)i], Ly = sc * Y[2 * (size_t)i + 1];
        if (Lb) {
            const double2 b = Lb[i];
            Lx += (float)b.x;
            Ly += (float)b.y;
        }
        double2 v = make_double2((double)(lx * Lx - ly * Ly), (double)(lx * Ly + ly * Lx));
        const float rf = sqrtf(t1f * t1f + t2f * t2f + x3f * x3f);
        if (rf < (float)(2.0 * eps)) {
            const double r = sqrt(t1 * t1 + t2 * t2 + x3 * x3);
            if (r < 2.0 * eps) {
                double sk, ck;
                sincos(k * r, &sk, &ck);
                const double Yc = 1.0 - smooth8((r - eps) / eps);
                const double f = Yc * 0.25 / (GF_PI * r);
                v = cadd(v, cmul(make_double2(cl, sl), make_double2(ck * f, sk * f)));
            }
        }
        out[i] = v;
    }
}

// ---------------------------------------------------------------------------
// Fused inference: all five layers of the network for 2 x 128 rows per
// iteration of a persistent CTA (one per SM).  The two 128 x 256 bf16
// activation tiles stay in shared memory (canonical K-major layout), the two
// 128 x 256 fp32 accumulators in tensor memory (all 512 columns); each
// layer's weights stream through three 256 x 64 stages, their copies issued up
// to three chunks ahead of the MMAs (the biases and head weights are read
// through L1 to leave the shared memory to them); the epilogue applies
// bias + SiLU and writes the next layer's input back into shared memory; the
// 256 -> 2 head is folded into the last epilogue.  HBM traffic per sample:
// 6 input floats and 2 output floats.
// ---------------------------------------------------------------------------
namespace fused {
// SiLU of two pre-activations on bf16 pairs: z rounded to bf16, halved
// (exact), one hardware tanh for both (tanh.approx.bf16x2) and one packed
// fma, z/2 + (z/2) tanh(z/2) = z sigmoid(z).  Returns the bf16 pair (z0 in the
// low half), the layout of the next layer's activations; the extra rounding of
// z to bf16 is of the size of the activation's own bf16 rounding.
__device__ __forceinline__ uint32_t silu2_bf16(float z0, float z1)
{
    uint32_t zb, hz, th, r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(zb) : "f"(z1), "f"(z0));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(hz) : "r"(zb), "r"(0x3F003F00u));
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(th) : "r"(hz));
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(hz), "r"(th), "r"(hz));
    return r;
}

constexpr int ROWS = 128, NT = 2;
constexpr int ACT_BYTES = ROWS * HID * 2;                // 64 KiB per tile
constexpr int WST_BYTES = HID * umma::KC * 2;           // 32 KiB per weight stage
constexpr int NS = 3;                           // weight stages in flight
constexpr int NCW = 8 * NT;                     // consumer warps (8 per tile: 4 row quarters x 2 column halves)
constexpr int THREADS = (NCW + 1) * 32;         // plus one producer warp
constexpr int SMEM = NT * ACT_BYTES + NS * WST_BYTES + 128;
static_assert(SMEM <= 232448, "shared memory of one CTA");
constexpr int TMEM_COLS = 512;

// act tile: [k/8][r/8] core matrices, the 16 row groups of a K block adjacent
// (LBO 2048 B along K, SBO 128 B along M), so that the 32 rows a warp writes for one
// K block are 512 contiguous bytes (no shared-memory bank conflicts)
constexpr uint32_t ACT_LBO = (ROWS / 8) * 128, ACT_SBO = 128;
__device__ __forceinline__ uint32_t act_off(int r, int k)
{
    return (k >> 3) * ACT_LBO + (r >> 3) * ACT_SBO + (r & 7) * 16 + (k & 7) * 2;
}

struct Args {
    const float *in;
    int n;
    float pi_ct;
    const bf16 *W[4];
    const bf16 *Wimg[4];  // per layer: its K chunks as ready 32 KiB shared-memory images
    const float *b[4];
    const float *W5, *b5;
    float *Y;
    int *err;
};
}  // namespace fused

// Producer warp (warp 16, one lane): weight-stage bulk copies and MMA issue,
// layer by layer, tile 0 then tile 1.  The sixteen consumer warps take every
// tile's epilogue in turn: warp w reads TMEM lanes 32 (w % 4) .. +31, i.e. its 32
// rows, and the column quarter w / 4 of the 256 columns, so four warps share each
// row's epilogue (and features).  While the consumers run one tile's epilogue
// (bias, SiLU, bf16 activations back into shared memory) the tensor cores work
// on the other tile.  The 256 -> 2 head's four column quarters meet in shared
// memory and are added in quarter order by the row quarter's first warp, which
// writes the output (the same result at every call).
//   lbar[b]  stage copy landed in buffer b    mbar[b]  MMAs of that stage done
//   accf[t]  tile t's layer MMAs done         actr[t]  tile t's activations written
//                                                      and its accumulator read (one arrival
//                                                      per consumer warp, after __syncwarp)
//   hbar[q]  the head partial sums of row quarter q written (one arrival per warp)
// Every wait is bounded; a timeout sets *err and makes every warp leave.
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(fused::THREADS, 1) mlp_infer_fused(fused::Args A)
{
    using namespace fused;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *act[NT] = {smem, smem + ACT_BYTES};
    uint8_t *wst0 = smem + NT * ACT_BYTES;  // NS weight stages of WST_BYTES
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NT * ACT_BYTES + NS * WST_BYTES);
    uint64_t *mbar = bars, *lbar = bars + NS, *accf = bars + 2 * NS, *actr = bars + 2 * NS + 2, *hbar = bars + 2 * NS + 4;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * NS + 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(umma::smem_u32(tslot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 2 * NS + 2; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_u32(&bars[q])));
        for (int q = 2 * NS + 2; q < 2 * NS + 4; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(umma::smem_u32(&bars[q])), "r"(NCW));
        for (int q = 2 * NS + 4; q < 2 * NS + 8; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(umma::smem_u32(&bars[q])), "r"(NCW / 4));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = umma::make_idesc(ROWS, HID);

    if (warp == NCW) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            // The weight chunks follow one fixed order per tile pair (layer, tile,
            // K chunk), so their copies run up to NS chunks ahead of the MMAs:
            // chunks 0 .. NS-1 at the start, chunk g - 1 + NS into the buffer of
            // chunk g - 1 once the MMAs of chunk g are issued and those of chunk
            // g - 1 are done.  Chunk g uses buffer g % NS, whose k-th use is phase k & 1.
            constexpr int NCH0 = (K0 + umma::KC - 1) / umma::KC, NCHH = HID / umma::KC;
            constexpr int PER_PAIR = NT * (NCH0 + 3 * NCHH);
            int npairs = 0;
            for (int tp = blockIdx.x; tp * (NT * ROWS) < A.n; tp += gridDim.x) ++npairs;
            const int total = npairs * PER_PAIR;
            auto issue = [&](int gg) {
                int q = gg % PER_PAIR, l = 0;
                if (q < NT * NCH0) {
                    q %= NCH0;
                } else {
                    q -= NT * NCH0;
                    l = 1 + q / (NT * NCHH);
                    q %= NCHH;
                }
                const int buf = gg % NS;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(umma::smem_u32(&lbar[buf])),
                             "r"(WST_BYTES)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        umma::smem_u32(wst0 + buf * WST_BYTES)),
                    "l"(A.Wimg[l] + (size_t)q * (WST_BYTES / 2)), "r"(WST_BYTES), "r"(umma::smem_u32(&lbar[buf]))
                    : "memory");
            };
            int g = 0, issued = min(NS, total) - 1, landed = -1, committed = -1, ua[NT] = {0, 0};
            for (int gg = 0; gg <= issued; ++gg) issue(gg);
            bool ok = true;
            for (int tp = blockIdx.x; ok && tp * (NT * ROWS) < A.n; tp += gridDim.x)
                for (int l = 0; ok && l < 4; ++l) {
                    const int K = l == 0 ? K0 : HID;
                    const int nch = (K + umma::KC - 1) / umma::KC;
                    for (int t = 0; ok && t < NT; ++t) {
                        // tile t's activations for layer l are written and its accumulator is free
                        ok = umma::mbar_wait_sleep(umma::smem_u32(&actr[t]), ua[t] & 1) && !*abort_flag;
                        ++ua[t];
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        for (int c = 0; ok && c < nch; ++c, ++g) {
                            const int buf = g % NS;
                            ok = umma::mbar_wait_sleep(umma::smem_u32(&lbar[buf]), (g / NS) & 1);
                            if (!ok) break;
                            landed = g;
                            asm volatile("tcgen05.fence::after_thread_sync;");
                            const int ksteps = (min(umma::KC, K - c * umma::KC) + 15) / 16;
                            const uint32_t b0 = umma::smem_u32(wst0 + buf * WST_BYTES), a0 = umma::smem_u32(act[t]);
                            for (int kk = 0; kk < ksteps; ++kk) {
                                const uint64_t ad = umma::make_desc(a0 + (c * 8 + kk * 2) * ACT_LBO, ACT_LBO, ACT_SBO);
                                const uint64_t bd = umma::make_desc(b0 + kk * 256, 128, (umma::KC / 8) * 128);
                                const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
                                asm volatile(
                                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + t * HID),
                                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                            }
                            asm volatile(
                                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                    umma::smem_u32(&mbar[buf])));
                            committed = g;
                            // refill the buffer of chunk g - 1 with chunk g - 1 + NS
                            if (g >= 1 && g - 1 + NS < total) {
                                ok = umma::mbar_wait_sleep(umma::smem_u32(&mbar[(g - 1) % NS]), ((g - 1) / NS) & 1);
                                if (!ok) break;
                                issue(g - 1 + NS);
                                issued = g - 1 + NS;
                            }
                        }
                        if (!ok) break;
                        // tile t's accumulator is complete once its MMAs are
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            umma::smem_u32(&accf[t])));
                    }
                }
            if (!ok) {
                *abort_flag = 1;
                if (A.err) atomicExch(A.err, 1);
            }
            // before the CTA exits: every issued copy has landed and every MMA has completed
            for (int gg = landed + 1; gg <= issued; ++gg) umma::mbar_wait_sleep(umma::smem_u32(&lbar[gg % NS]), (gg / NS) & 1);
            if (committed >= 0) umma::mbar_wait_sleep(umma::smem_u32(&mbar[committed % NS]), (committed / NS) & 1);
        }
    } else {
        // ---------------------------------------------------------------- consumers
        const int quarter = warp & 3, cq = warp >> 2, r = quarter * 32 + lane;
        const float b50 = A.b5[0], b51 = A.b5[1];
        int fa[NT] = {0, 0}, hp = 0;
        bool ok = true;
        for (int tp = blockIdx.x; ok && tp * (NT * ROWS) < A.n; tp += gridDim.x) {
          for (int t = 0; t < NT; ++t) {
            uint8_t *at = act[t];
            const int i = tp * NT * ROWS + t * ROWS + r;
            const bool live = i < A.n;
            // features of this row into the first 80 columns of the tile
            {
                float t1 = 0.f, t2 = 0.f, x3 = 0.f, p3 = 0.f, p4 = 0.f, p5 = 2.5f;
                if (live) {
                    const float *p = A.in + 6 * (size_t)i;
                    t1 = p[0];
                    t2 = p[1];
                    x3 = p[2];
                    p3 = p[3];
                    p4 = p[4];
                    p5 = p[5];
                }
                const float rr = sqrtf(t1 * t1 + t2 * t2 + x3 * x3);
                // ten blocks of 8 features: blocks 0..7 hold cos/sin of 4 frequencies each;
                // the four column quarters of a row write blocks 0..1, 2..4, 5..6 and 7..9
                for (int kb = (cq * (K0 / 8)) / 4; kb < ((cq + 1) * (K0 / 8)) / 4; ++kb) {
                    float v[8];
                    if (kb < 8) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int j = kb * 4 + u;
                            // |phase| < 30: the fast sine/cosine error (~1e-5 there) is far below bf16 rounding
                            const float ph = c_freq[j][0] * t1 + c_freq[j][1] * t2 + c_freq[j][2] * A.pi_ct * x3;
                            __sincosf(ph, &v[2 * u + 1], &v[2 * u]);
                        }
                    } else if (kb == 8) {
                        v[0] = 2.f * p3;
                        v[1] = 2.f * p4;
                        v[2] = (p5 - 2.5f) / 1.5f;
                        v[3] = rr;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float d = (rr - 0.15f * u) * (1.f / 0.15f);
                            v[4 + u] = __expf(-0.5f * d * d);
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float d = (rr - 0.15f * (4 + u)) * (1.f / 0.15f);
                            v[u] = __expf(-0.5f * d * d);
                        }
                    }
                    uint32_t pk[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const __nv_bfloat162 hb = __floats2bfloat162_rn(live ? v[2 * e] : 0.f, live ? v[2 * e + 1] : 0.f);
                        pk[e] = (uint32_t)__bfloat16_as_ushort(hb.x) | ((uint32_t)__bfloat16_as_ushort(hb.y) << 16);
                    }
                    *reinterpret_cast<uint4 *>(at + act_off(r, kb * 8)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(umma::smem_u32(&actr[t]));
          }
            for (int l = 0; ok && l < 4; ++l)
              for (int t = 0; ok && t < NT; ++t) {
                uint8_t *at = act[t];
                const int i = tp * NT * ROWS + t * ROWS + r;
                const bool live = i < A.n;
                ok = __all_sync(0xffffffffu, umma::mbar_wait_sleep(umma::smem_u32(&accf[t]), fa[t] & 1) && !*abort_flag);
                ++fa[t];
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const float *bias = A.b[l];
                float y0 = 0.f, y1 = 0.f;
                for (int j = cq * (HID / 4); j < (cq + 1) * (HID / 4); j += 32) {
                    uint32_t v[32];
                    const uint32_t taddr = tmem + t * HID + ((uint32_t)(quarter * 32) << 16) + (uint32_t)j;
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    uint32_t pk[16];  // bf16 pairs, kept in registers
#pragma unroll
                    for (int e = 0; e < 32; e += 4) {
                        const float4 bb = __ldg(reinterpret_cast<const float4 *>(bias + j + e));  // broadcast, L1
                        const float z[4] = {__uint_as_float(v[e]) + bb.x, __uint_as_float(v[e + 1]) + bb.y,
                                            __uint_as_float(v[e + 2]) + bb.z, __uint_as_float(v[e + 3]) + bb.w};
                        const uint32_t h01 = silu2_bf16(z[0], z[1]), h23 = silu2_bf16(z[2], z[3]);
                        pk[e >> 1] = h01;
                        pk[(e >> 1) + 1] = h23;
                        if (l == 3) {
                            const float4 w0 = __ldg(reinterpret_cast<const float4 *>(A.W5 + j + e));
                            const float4 w1 = __ldg(reinterpret_cast<const float4 *>(A.W5 + HID + j + e));
                            const float h[4] = {__uint_as_float(h01 << 16), __uint_as_float(h01 & 0xFFFF0000u),
                                                __uint_as_float(h23 << 16), __uint_as_float(h23 & 0xFFFF0000u)};
                            y0 = fmaf(h[0], w0.x, fmaf(h[1], w0.y, fmaf(h[2], w0.z, fmaf(h[3], w0.w, y0))));
                            y1 = fmaf(h[0], w1.x, fmaf(h[1], w1.y, fmaf(h[2], w1.z, fmaf(h[3], w1.w, y1))));
                        }
                    }
                    if (l < 3) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            *reinterpret_cast<uint4 *>(at + act_off(r, j + 8 * q)) =
                                make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                    }
                }
                if (l < 3) {
                    // next layer's input written, accumulator read: hand the tile back
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(umma::smem_u32(&actr[t]));
                } else {
                    // the head: the four column quarters' partial sums of row r meet in
                    // the last 4 KiB of the tile's activations (K columns 240..255, not
                    // written again before this tile's next layer-0 epilogue, which
                    // follows every warp's next features) and are added in quarter order
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    float *part = reinterpret_cast<float *>(at + ACT_BYTES - 4096);  // [quarter][row][2]
                    part[(cq * ROWS + r) * 2] = y0;
                    part[(cq * ROWS + r) * 2 + 1] = y1;
                    __syncwarp();
                    if (lane == 0) mbar_arrive(umma::smem_u32(&hbar[quarter]));
                    if (cq == 0) {
                        ok = __all_sync(0xffffffffu, umma::mbar_wait_sleep(umma::smem_u32(&hbar[quarter]), hp & 1));
                        ++hp;
                        if (!ok) break;
                        if (live) {
                            float s0 = b50, s1 = b51;
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                s0 += part[(q * ROWS + r) * 2];
                                s1 += part[(q * ROWS + r) * 2 + 1];
                            }
                            A.Y[2 * (size_t)i] = s0;
                            A.Y[2 * (size_t)i + 1] = s1;
                        }
                    }
                }
            }
        }
        if (!ok) {
            *abort_flag = 1;
            if (A.err) atomicExch(A.err, 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace

struct gf_mlp_s {
    float *W[NL] = {}, *b[NL] = {}, *mW[NL] = {}, *vW[NL] = {}, *mb[NL] = {}, *vb[NL] = {}, *gW[NL] = {}, *gb[NL] = {};
    bf16 *Wb[NL] = {}, *WTb[NL] = {};
    bf16 *Wimg = nullptr;   // weight-stage images of layers 1-4 (fused inference)
    int wver = 1, imgver = 0;  // bf16 weights version / version the images were built from
    int cap = 0;
    bf16 *X0 = nullptr, *Z[4] = {}, *H[4] = {}, *dZ[4] = {};
    float *Y = nullptr, *dY = nullptr, *in = nullptr, *loss = nullptr;
    int *errw = nullptr;
    int adam_t = 0;
    double scale = 1.0;
    double ct = 1.0;
    int nsm = 152;
};

namespace {

gf_status ensure_cap(gf_mlp_t m, int n)
{
    if (n <= m->cap) return GF_OK;
    CUM(cudaDeviceSynchronize());
    auto fr = [](void *p) {
        if (p) cudaFree(p);
    };
    fr(m->X0);
    fr(m->Y);
    fr(m->dY);
    fr(m->in);
    for (int l = 0; l < 4; ++l) {
        fr(m->Z[l]);
        fr(m->H[l]);
        fr(m->dZ[l]);
    }
    int cap = (n + 127) / 128 * 128;
    CUM(cudaMalloc(&m->X0, sizeof(bf16) * (size_t)cap * K0));
    CUM(cudaMalloc(&m->Y, sizeof(float) * 2 * (size_t)cap));
    CUM(cudaMalloc(&m->dY, sizeof(float) * 2 * (size_t)cap));
    CUM(cudaMalloc(&m->in, sizeof(float) * 6 * (size_t)cap));
    for (int l = 0; l < 4; ++l) {
        CUM(cudaMalloc(&m->Z[l], sizeof(bf16) * (size_t)cap * HID));
        CUM(cudaMalloc(&m->H[l], sizeof(bf16) * (size_t)cap * HID));
        CUM(cudaMalloc(&m->dZ[l], sizeof(bf16) * (size_t)cap * HID));
    }
    m->cap = cap;
    return GF_OK;
}

cudaError_t launch_gemm(const umma::GemmArgs &g0, bool at, bool bt, int ksplit, cudaStream_t s)
{
    umma::GemmArgs g = g0;
    g.kper = ksplit > 1 ? ((g.K + ksplit - 1) / ksplit + umma::KC - 1) / umma::KC * umma::KC : g.K;
    int zs = (g.K + g.kper - 1) / g.kper;
    dim3 grid((g.M + umma::BM - 1) / umma::BM, (g.N + g.BN - 1) / g.BN, zs);
    cudaError_t e;
    if (!at && !bt) {
        e = cudaFuncSetAttribute(umma::gemm_bf16<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, umma::SMEM);
        if (e != cudaSuccess) return e;
        umma::gemm_bf16<false, false><<<grid, 128, umma::SMEM, s>>>(g);
    } else if (at && bt) {
        e = cudaFuncSetAttribute(umma::gemm_bf16<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, umma::SMEM);
        if (e != cudaSuccess) return e;
        umma::gemm_bf16<true, true><<<grid, 128, umma::SMEM, s>>>(g);
    } else if (at) {
        e = cudaFuncSetAttribute(umma::gemm_bf16<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, umma::SMEM);
        if (e != cudaSuccess) return e;
        umma::gemm_bf16<true, false><<<grid, 128, umma::SMEM, s>>>(g);
    } else {
        e = cudaFuncSetAttribute(umma::gemm_bf16<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, umma::SMEM);
        if (e != cudaSuccess) return e;
        umma::gemm_bf16<false, true><<<grid, 128, umma::SMEM, s>>>(g);
    }
    gf_count_launch(1);
    return cudaGetLastError();
}

// forward of n samples whose float inputs are in m->in; output m->Y
gf_status forward(gf_mlp_t m, int n, cudaStream_t s)
{
    const int blocks = m->nsm * 8;
    features_kernel<<<blocks, 256, 0, s>>>(m->in, n, m->X0, (float)(GF_PI / m->ct));
    gf_count_launch(1);
    const bf16 *A = m->X0;
    for (int l = 0; l < 4; ++l) {
        umma::GemmArgs g{};
        g.A = A;
        g.lda = IN_DIM[l];
        g.B = m->Wb[l];
        g.ldb = IN_DIM[l];
        g.M = n;
        g.N = HID;
        g.K = IN_DIM[l];
        g.BN = HID;
        g.epi = umma::EPI_BIAS_SILU;
        g.bias = m->b[l];
        g.Z = m->Z[l];
        g.H = m->H[l];
        g.ldz = HID;
        g.err = m->errw;
        CUM(launch_gemm(g, false, false, 1, s));
        A = m->H[l];
    }
    return GF_OK;
}

int64_t nparams(int l) { return (int64_t)OUT_DIM[l] * IN_DIM[l]; }

// inference of n samples whose float inputs are in m->in, output float [n][2]
constexpr int IMG_CHUNKS[4] = {(K0 + umma::KC - 1) / umma::KC, HID / umma::KC, HID / umma::KC, HID / umma::KC};

gf_status infer(gf_mlp_t m, int n, float *Y, cudaStream_t s)
{
    fused::Args A{};
    const size_t stage = (size_t)HID * umma::KC;  // bf16 elements per image
    if (!m->Wimg) {
        int tot = 0;
        for (int l = 0; l < 4; ++l) tot += IMG_CHUNKS[l];
        CUM(cudaMalloc(&m->Wimg, sizeof(bf16) * stage * tot));
    }
    {
        size_t off = 0;
        for (int l = 0; l < 4; ++l) {
            if (m->imgver != m->wver) {
                stage_images_kernel<<<64, 256, 0, s>>>(m->Wb[l], IN_DIM[l], IMG_CHUNKS[l], m->Wimg + off);
                gf_count_launch(1);
            }
            A.Wimg[l] = m->Wimg + off;
            off += stage * IMG_CHUNKS[l];
        }
        CUM(cudaGetLastError());
        m->imgver = m->wver;
    }
    A.in = m->in;
    A.n = n;
    A.pi_ct = (float)(GF_PI / m->ct);
    for (int l = 0; l < 4; ++l) {
        A.W[l] = m->Wb[l];
        A.b[l] = m->b[l];
    }
    A.W5 = m->W[4];
    A.b5 = m->b[4];
    A.Y = Y;
    A.err = m->errw;
    CUM(cudaFuncSetAttribute(mlp_infer_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, fused::SMEM));
    int tiles = (n + fused::NT * fused::ROWS - 1) / (fused::NT * fused::ROWS);
    int grid = tiles < m->nsm ? tiles : m->nsm;
    mlp_infer_fused<<<grid, fused::THREADS, fused::SMEM, s>>>(A);
    gf_count_launch(1);
    CUM(cudaGetLastError());
    return GF_OK;
}

}  // namespace

extern "C" {

gf_status gf_gemm_bf16(const void *A, int64_t lda, int a_trans, const void *B, int64_t ldb, int b_trans, int M, int N,
                       int K, float *C, int64_t ldc, int ksplit, void *cuda_stream)
{
    if (!A || !B || !C) return err(GF_ERR_ARG, "gf_gemm_bf16: NULL buffer");
    if (M <= 0 || N <= 0 || K <= 0 || M % 16 || N % 16 || K % 16)
        return err(GF_ERR_ARG, "gf_gemm_bf16: M, N, K must be positive multiples of 16");
    if (ksplit < 1) ksplit = 1;
    umma::GemmArgs g{};
    g.A = (const bf16 *)A;
    g.lda = lda;
    g.B = (const bf16 *)B;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.BN = N < umma::BN_MAX ? N : umma::BN_MAX;
    if (N > umma::BN_MAX && N % umma::BN_MAX) g.BN = 128;
    g.epi = umma::EPI_F32;
    g.C = C;
    g.ldc = ldc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (ksplit > 1) CUM(cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * ldc, s));
    CUM(launch_gemm(g, a_trans != 0, b_trans != 0, ksplit, s));
    return GF_OK;
}

gf_status gf_mlp_create(uint64_t seed, double c_tilde, gf_mlp_t *out)
{
    if (!out) return err(GF_ERR_ARG, "gf_mlp_create: out is NULL");
    *out = nullptr;
    gf_mlp_s *m = new gf_mlp_s();
    m->ct = c_tilde > 0 ? c_tilde : 1.0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, dev);
    // frequency vectors: (n1, n2) in {-1,0,1}^2, m3 in {0,1} without (0,0,0) (17 vectors), then 15 higher ones
    int fr[32][3], nf = 0;
    for (int m3 = 0; m3 <= 1; ++m3)
        for (int n1 = -1; n1 <= 1; ++n1)
            for (int n2 = -1; n2 <= 1; ++n2)
                if (n1 || n2 || m3) {
                    fr[nf][0] = n1;
                    fr[nf][1] = n2;
                    fr[nf][2] = m3;
                    ++nf;
                }
    const int extra[15][3] = {{0, 0, 2}, {0, 0, 3}, {2, 0, 0}, {-2, 0, 0}, {0, 2, 0}, {0, -2, 0}, {2, 0, 1}, {0, 2, 1},
                              {3, 0, 0}, {0, 3, 0}, {-3, 0, 0}, {0, -3, 0}, {1, 1, 2}, {-1, 1, 2}, {2, 2, 0}};
    for (int e = 0; e < 15; ++e, ++nf) memcpy(fr[nf], extra[e], sizeof(int) * 3);
    gf_status s = GF_OK;
    do {
        cudaError_t e;
        if ((e = cudaMemcpyToSymbol(c_freq, fr, sizeof(fr))) != cudaSuccess) {
            s = err(GF_ERR_CUDA, "gf_mlp_create: %s", cudaGetErrorString(e));
            break;
        }
        if ((e = cudaMalloc(&m->errw, sizeof(int))) != cudaSuccess || (e = cudaMalloc(&m->loss, sizeof(float))) != cudaSuccess) {
            s = err(GF_ERR_NOMEM, "gf_mlp_create: cudaMalloc");
            break;
        }
        cudaMemset(m->errw, 0, sizeof(int));
        for (int l = 0; l < NL && s == GF_OK; ++l) {
            size_t nw = nparams(l), nb = OUT_DIM[l];
            float **f[8] = {&m->W[l], &m->mW[l], &m->vW[l], &m->gW[l], &m->b[l], &m->mb[l], &m->vb[l], &m->gb[l]};
            size_t sz[8] = {nw, nw, nw, nw, nb, nb, nb, nb};
            for (int q = 0; q < 8; ++q)
                if (cudaMalloc(f[q], sizeof(float) * sz[q]) != cudaSuccess) s = err(GF_ERR_NOMEM, "gf_mlp_create: cudaMalloc");
            if (s != GF_OK) break;
            if (cudaMalloc(&m->Wb[l], sizeof(bf16) * nw) != cudaSuccess ||
                cudaMalloc(&m->WTb[l], sizeof(bf16) * nw) != cudaSuccess) {
                s = err(GF_ERR_NOMEM, "gf_mlp_create: cudaMalloc");
                break;
            }
            for (int q = 1; q < 8; ++q)
                if (q != 4) cudaMemset(*f[q], 0, sizeof(float) * sz[q]);
            cudaMemset(m->b[l], 0, sizeof(float) * nb);
            // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
            init_kernel<<<64, 256>>>(m->W[l], (int)nw, (float)(1.0 / sqrt((double)IN_DIM[l])), seed * 16 + l);
            convert_kernel<<<64, 256>>>(m->W[l], m->Wb[l], m->WTb[l], OUT_DIM[l], IN_DIM[l]);
            ++m->wver;
            gf_count_launch(2);
        }
    } while (0);
    if (s == GF_OK && cudaDeviceSynchronize() != cudaSuccess) s = err(GF_ERR_CUDA, "gf_mlp_create: init failed");
    if (s != GF_OK) {
        gf_mlp_destroy(m);
        return s;
    }
    *out = m;
    return GF_OK;
}

gf_status gf_mlp_set_scale(gf_mlp_t m, double scale)
{
    if (!m || !(scale > 0)) return err(GF_ERR_ARG, "gf_mlp_set_scale: bad argument");
    m->scale = scale;
    return GF_OK;
}

gf_status gf_mlp_params(gf_mlp_t m, float *host, int64_t count, int to_device)
{
    if (!m || !host) return err(GF_ERR_ARG, "gf_mlp_params: NULL argument");
    int64_t need = 0;
    for (int l = 0; l < NL; ++l) need += nparams(l) + OUT_DIM[l];
    if (count < need) return err(GF_ERR_ARG, "gf_mlp_params: need %lld floats", (long long)need);
    CUM(cudaDeviceSynchronize());
    int64_t off = 0;
    for (int l = 0; l < NL; ++l) {
        size_t nw = nparams(l), nb = OUT_DIM[l];
        if (to_device) {
            CUM(cudaMemcpy(m->W[l], host + off, sizeof(float) * nw, cudaMemcpyHostToDevice));
            CUM(cudaMemcpy(m->b[l], host + off + nw, sizeof(float) * nb, cudaMemcpyHostToDevice));
            convert_kernel<<<64, 256>>>(m->W[l], m->Wb[l], m->WTb[l], OUT_DIM[l], IN_DIM[l]);
            ++m->wver;
            gf_count_launch(1);
        } else {
            CUM(cudaMemcpy(host + off, m->W[l], sizeof(float) * nw, cudaMemcpyDeviceToHost));
            CUM(cudaMemcpy(host + off + nw, m->b[l], sizeof(float) * nb, cudaMemcpyDeviceToHost));
        }
        off += nw + nb;
    }
    CUM(cudaDeviceSynchronize());
    return GF_OK;
}

int64_t gf_mlp_param_count(void)
{
    int64_t need = 0;
    for (int l = 0; l < NL; ++l) need += nparams(l) + OUT_DIM[l];
    return need;
}

gf_status gf_mlp_forward(gf_mlp_t m, const float *dev_in, int n, float *dev_out, void *cuda_stream)
{
    if (!m || n < 0 || (n > 0 && (!dev_in || !dev_out))) return err(GF_ERR_ARG, "gf_mlp_forward: bad argument");
    if (n == 0) return GF_OK;
    gf_status s = ensure_cap(m, n);
    if (s != GF_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    CUM(cudaMemcpyAsync(m->in, dev_in, sizeof(float) * 6 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    return infer(m, n, dev_out, st);
}

// Gradients of the mean-squared loss over one batch (into the grad buffers);
// optionally followed by one Adam step.
static gf_status train_or_grad(gf_mlp_t m, const float *dev_in, const float *dev_target, int n, float lr, int do_step,
                               float *dev_loss, cudaStream_t st)
{
    gf_status s = ensure_cap(m, n);
    if (s != GF_OK) return s;
    CUM(cudaMemcpyAsync(m->in, dev_in, sizeof(float) * 6 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    for (int l = 0; l < NL; ++l) {
        CUM(cudaMemsetAsync(m->gW[l], 0, sizeof(float) * nparams(l), st));
        CUM(cudaMemsetAsync(m->gb[l], 0, sizeof(float) * OUT_DIM[l], st));
    }
    CUM(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
    if ((s = forward(m, n, st)) != GF_OK) return s;
    const int blocks = m->nsm * 8;
    head_fwd_kernel<<<blocks, 256, 0, st>>>(m->H[3], m->W[4], m->b[4], m->Y, n, dev_target, m->dY, m->loss, 1.f / n);
    head_bwd_kernel<<<blocks, 256, 0, st>>>(m->dY, m->W[4], m->Z[3], m->dZ[3], n);
    const int rpb = 64;
    head_wgrad_kernel<<<(n + rpb - 1) / rpb, HID, 0, st>>>(m->dY, m->H[3], m->gW[4], m->gb[4], n, rpb);
    gf_count_launch(3);
    for (int l = 3; l >= 0; --l) {
        // weight gradient gW_l = dZ_l^T . A_l  (A_0 = X0, A_l = H_{l-1}); reduction over the batch, split-K
        umma::GemmArgs g{};
        g.A = m->dZ[l];
        g.lda = HID;
        g.B = l == 0 ? m->X0 : m->H[l - 1];
        g.ldb = IN_DIM[l];
        g.M = HID;
        g.N = IN_DIM[l];
        g.K = n;
        g.BN = IN_DIM[l];
        g.epi = umma::EPI_F32;
        g.C = m->gW[l];
        g.ldc = IN_DIM[l];
        g.err = m->errw;
        int ks = n / 512 > 1 ? n / 512 : 1;
        if (ks > 64) ks = 64;
        CUM(launch_gemm(g, true, true, ks, st));
        bias_grad_kernel<<<(n + rpb - 1) / rpb, HID, 0, st>>>(m->dZ[l], m->gb[l], n, rpb);
        gf_count_launch(1);
        if (l > 0) {
            // dZ_{l-1} = (dZ_l . W_l) * silu'(Z_{l-1})
            umma::GemmArgs h{};
            h.A = m->dZ[l];
            h.lda = HID;
            h.B = m->WTb[l];
            h.ldb = HID;
            h.M = n;
            h.N = IN_DIM[l];
            h.K = HID;
            h.BN = IN_DIM[l];
            h.epi = umma::EPI_DSILU;
            h.Zin = m->Z[l - 1];
            h.dZ = m->dZ[l - 1];
            h.ldz = HID;
            h.err = m->errw;
            CUM(launch_gemm(h, false, false, 1, st));
        }
    }
    if (do_step) {
        m->adam_t += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
        for (int l = 0; l < NL; ++l) {
            adam_kernel<<<256, 256, 0, st>>>(m->W[l], m->gW[l], m->mW[l], m->vW[l], (int)nparams(l), lr, b1, b2, 1e-8f, c1, c2);
            adam_kernel<<<4, 256, 0, st>>>(m->b[l], m->gb[l], m->mb[l], m->vb[l], OUT_DIM[l], lr, b1, b2, 1e-8f, c1, c2);
            convert_kernel<<<128, 256, 0, st>>>(m->W[l], m->Wb[l], m->WTb[l], OUT_DIM[l], IN_DIM[l]);
            ++m->wver;
            gf_count_launch(3);
        }
    }
    if (dev_loss) CUM(cudaMemcpyAsync(dev_loss, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
    CUM(cudaGetLastError());
    return GF_OK;
}

gf_status gf_mlp_train_step(gf_mlp_t m, const float *dev_in, const float *dev_target, int n, float lr, float *dev_loss,
                            void *cuda_stream)
{
    if (!m || n <= 0 || !dev_in || !dev_target) return err(GF_ERR_ARG, "gf_mlp_train_step: bad argument");
    return train_or_grad(m, dev_in, dev_target, n, lr, 1, dev_loss, (cudaStream_t)cuda_stream);
}

gf_status gf_mlp_gradients(gf_mlp_t m, const float *dev_in, const float *dev_target, int n, float *host_grads,
                           float *host_loss, void *cuda_stream)
{
    if (!m || n <= 0 || !dev_in || !dev_target || !host_grads) return err(GF_ERR_ARG, "gf_mlp_gradients: bad argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    gf_status s = train_or_grad(m, dev_in, dev_target, n, 0.f, 0, nullptr, st);
    if (s != GF_OK) return s;
    CUM(cudaStreamSynchronize(st));
    int64_t off = 0;
    for (int l = 0; l < NL; ++l) {
        size_t nw = nparams(l), nb = OUT_DIM[l];
        CUM(cudaMemcpy(host_grads + off, m->gW[l], sizeof(float) * nw, cudaMemcpyDeviceToHost));
        CUM(cudaMemcpy(host_grads + off + nw, m->gb[l], sizeof(float) * nb, cudaMemcpyDeviceToHost));
        off += nw + nb;
    }
    if (host_loss) CUM(cudaMemcpy(host_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return GF_OK;
}

gf_status gf_mlp_error_word(gf_mlp_t m, int *out)
{
    if (!m || !out) return err(GF_ERR_ARG, "gf_mlp_error_word: NULL argument");
    CUM(cudaMemcpy(out, m->errw, sizeof(int), cudaMemcpyDeviceToHost));
    return *out ? GF_ERR_TIMEOUT : GF_OK;
}

}  // extern "C"

// Shared body of gf_surrogate_eval (dev_base null) and gf_surrogate_eval_residual.
static gf_status surrogate_eval_impl(gf_mlp_t m, int npairs, const double *k, const double *alpha,
                                     const int64_t *offsets, const double *dev_xyz, const double2 *dev_base,
                                     void *dev_out, double wood_delta, const gf_trunc_t *trunc, int *n_fallback_pairs,
                                     void *cuda_stream)
{
    if (!m || npairs <= 0 || !k || !alpha || !offsets || (offsets[npairs] > 0 && (!dev_xyz || !dev_out)))
        return err(GF_ERR_ARG, "gf_surrogate_eval: bad argument");
    if (offsets[0] != 0) return err(GF_ERR_ARG, "gf_surrogate_eval: offsets[0] must be 0");
    for (int p = 0; p < npairs; ++p)
        if (offsets[p + 1] < offsets[p]) return err(GF_ERR_ARG, "gf_surrogate_eval: offsets must be non-decreasing");
    gf_trunc_t tr;
    gf_trunc_default(&tr);
    if (trunc) tr = *trunc;
    tr.precision = GF_FP64;
    tr.kind = GF_HELMHOLTZ;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t total = offsets[npairs];
    if (total > 0x7fffffff) return err(GF_ERR_ARG, "gf_surrogate_eval: too many targets");
    // Wood distance per pair: min_n | |alpha_n| - k |
    std::vector<int> fallback(npairs, 0);
    int nfb = 0;
    for (int p = 0; p < npairs; ++p) {
        const double a1 = alpha[2 * p], a2 = alpha[2 * p + 1], kk = k[p];
        const int R = (int)ceil(kk) + 2;
        double dmin = 1e300;
        for (int n1 = -R - (int)fabs(a1); n1 <= R + (int)fabs(a1); ++n1)
            for (int n2 = -R - (int)fabs(a2); n2 <= R + (int)fabs(a2); ++n2) {
                double d = fabs(sqrt((a1 + n1) * (a1 + n1) + (a2 + n2) * (a2 + n2)) - kk);
                dmin = d < dmin ? d : dmin;
            }
        if (dmin < wood_delta) {
            fallback[p] = 1;
            ++nfb;
        }
    }
    if (n_fallback_pairs) *n_fallback_pairs = nfb;
    // network pairs: pair parameters and offsets on the device
    std::vector<double> pk(3 * (size_t)npairs);
    for (int p = 0; p < npairs; ++p) {
        pk[3 * p] = alpha[2 * p];
        pk[3 * p + 1] = alpha[2 * p + 1];
        pk[3 * p + 2] = k[p];
    }
    if (total > 0) {
        // network activations are held for at most kChunk targets at a time
        const int64_t kChunk = 1 << 20;
        gf_status s = ensure_cap(m, (int)(total < kChunk ? total : kChunk));
        if (s != GF_OK) return s;
        // pair offsets and parameters: stream-ordered pool memory, uploaded through
        // the pinned staging ring (nothing here waits for the device)
        int64_t *d_off = nullptr;
        double *d_pk = nullptr;
        CUM(gf_dev_alloc((void **)&d_off, sizeof(int64_t) * (npairs + 1), st));
        CUM(gf_dev_alloc((void **)&d_pk, sizeof(double) * pk.size(), st));
        CUM(gf_stage_upload(d_off, offsets, sizeof(int64_t) * (npairs + 1), st));
        CUM(gf_stage_upload(d_pk, pk.data(), sizeof(double) * pk.size(), st));
        const int blocks = m->nsm * 8;
        for (int64_t base = 0; base < total; base += kChunk) {
            const int n = (int)(total - base < kChunk ? total - base : kChunk);
            surrogate_inputs_kernel<<<blocks, 256, 0, st>>>(dev_xyz + 3 * base, n, base, d_off, npairs, d_pk, m->in);
            gf_count_launch(1);
            if ((s = infer(m, n, m->Y, st)) != GF_OK) return s;
            surrogate_assemble_kernel<<<blocks, 256, 0, st>>>(dev_xyz + 3 * base, n, base, d_off, npairs, d_pk, m->Y,
                                                              m->scale, tr.c, tr.eps, dev_base ? dev_base + base : nullptr,
                                                              (double2 *)dev_out + base);
            gf_count_launch(1);
        }
        gf_dev_free(d_off, st);
        gf_dev_free(d_pk, st);
    }
    // FFT-path fallback near Wood anomalies: overwrite those pairs' rows
    for (int p = 0; p < npairs; ++p) {
        if (!fallback[p] || offsets[p + 1] == offsets[p]) continue;
        const int M[3] = {128, 128, 64};
        gf_plan_t pl = nullptr;
        gf_status s = gf_plan(3, k[p], alpha + 2 * p, M, &tr, cuda_stream, &pl);
        if (s != GF_OK) return s;
        s = gf_eval_points(pl, dev_xyz + 3 * offsets[p], offsets[p + 1] - offsets[p], GF_OUT_GD,
                           (double2 *)dev_out + offsets[p], cuda_stream);
        CUM(cudaStreamSynchronize(st));
        gf_destroy(pl);
        if (s != GF_OK) return s;
    }
    return GF_OK;
}

extern "C" {

gf_status gf_surrogate_eval(gf_mlp_t m, int npairs, const double *k, const double *alpha, const int64_t *offsets,
                            const double *dev_xyz, void *dev_out, double wood_delta, const gf_trunc_t *trunc,
                            int *n_fallback_pairs, void *cuda_stream)
{
    return surrogate_eval_impl(m, npairs, k, alpha, offsets, dev_xyz, nullptr, dev_out, wood_delta, trunc,
                               n_fallback_pairs, cuda_stream);
}

gf_status gf_surrogate_eval_residual(gf_mlp_t m, int npairs, const double *k, const double *alpha,
                                     const int64_t *offsets, const double *dev_xyz, const void *dev_base,
                                     void *dev_out, double wood_delta, const gf_trunc_t *trunc,
                                     int *n_fallback_pairs, void *cuda_stream)
{
    if (!dev_base && offsets && npairs > 0 && offsets[npairs] > 0)
        return err(GF_ERR_ARG, "gf_surrogate_eval_residual: dev_base is NULL");
    return surrogate_eval_impl(m, npairs, k, alpha, offsets, dev_xyz, (const double2 *)dev_base, dev_out, wood_delta,
                               trunc, n_fallback_pairs, cuda_stream);
}

gf_status gf_mlp_destroy(gf_mlp_t m)
{
    if (!m) return GF_OK;
    cudaDeviceSynchronize();
    auto fr = [](void *p) {
        if (p) cudaFree(p);
    };
    for (int l = 0; l < NL; ++l) {
        fr(m->W[l]);
        fr(m->b[l]);
        fr(m->mW[l]);
        fr(m->vW[l]);
        fr(m->mb[l]);
        fr(m->vb[l]);
        fr(m->gW[l]);
        fr(m->gb[l]);
        fr(m->Wb[l]);
        fr(m->WTb[l]);
    }
    fr(m->Wimg);
    fr(m->X0);
    fr(m->Y);
    fr(m->dY);
    fr(m->in);
    fr(m->loss);
    fr(m->errw);
    for (int l = 0; l < 4; ++l) {
        fr(m->Z[l]);
        fr(m->H[l]);
        fr(m->dZ[l]);
    }
    delete m;
    return GF_OK;
}

}  // extern "C"
