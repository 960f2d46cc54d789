// Hand-written BF16 GEMM on the 5th-generation tensor cores (tcgen05):
//   C[M x N] = A[M x K] . B[N x K]^T   (both operands K-major in shared memory),
// FP32 accumulation in tensor memory (TMEM), fused epilogues.  One CTA of 128
// threads owns a 128 x BN tile (BN <= 256, multiple of 16); operands are staged
// by all threads into the canonical no-swizzle K-major layout (8-row x 16-byte
// core matrices) in two shared-memory stages, one elected thread issues
// tcgen05.mma for a stage while the others load the next, and completion is
// tracked with tcgen05.commit on an mbarrier.  Every mbarrier wait is bounded:
// on timeout the kernel records an error word, stops issuing work, waits
// (bounded) for what it already issued, frees its TMEM and returns.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace umma {

constexpr int BM = 128;
constexpr int KC = 64;                 // K elements per stage (4 MMAs of K = 16)
constexpr int BN_MAX = 256;
constexpr int A_STAGE = BM * KC * 2;   // 16 KiB
constexpr int B_STAGE = BN_MAX * KC * 2;  // 32 KiB
constexpr int SMEM = 2 * (A_STAGE + B_STAGE) + 64;
constexpr int TMEM_COLS = 256;
constexpr long long WAIT_LIMIT = 1ll << 24;  // try_wait polls before declaring a timeout

enum Epi {
    EPI_F32 = 0,        // C (fp32) = acc             (atomicAdd when split over K)
    EPI_BIAS_SILU = 1,  // Z = acc + bias (bf16), H = silu(Z) (bf16)
    EPI_BIAS = 2,       // C (fp32) = acc + bias
    EPI_DSILU = 3       // dZ = acc * silu'(Zin) (bf16)
};

struct GemmArgs {
    const __nv_bfloat16 *A;
    long long lda;      // A(m,k) = A[m*lda + k], or A[k*lda + m] when transposed
    const __nv_bfloat16 *B;
    long long ldb;      // B(n,k) = B[n*ldb + k], or B[k*ldb + n] when transposed
    int M, N, K;        // K multiple of 16
    int BN;             // N-tile (multiple of 16, <= 256)
    int kper;           // K range per blockIdx.z (multiple of 64), split-K
    int epi;
    float *C;
    long long ldc;
    const float *bias;
    __nv_bfloat16 *Z, *H;
    const __nv_bfloat16 *Zin;
    __nv_bfloat16 *dZ;
    long long ldz;
    int *err;           // set to 1 on a bounded-wait timeout
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// SM100 shared-memory matrix descriptor, no swizzle: start address, leading
// (K-direction) and stride (M/N-direction) byte offsets between core matrices.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for sm_100 family
    return d;                // base offset 0, layout SWIZZLE_NONE (0)
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major.
__host__ __device__ __forceinline__ uint32_t make_idesc(int M, int N)
{
    return (1u << 4)                       // D format F32
           | (1u << 7)                     // A format BF16
           | (1u << 10)                    // B format BF16
           | ((uint32_t)(N >> 3) << 17)    // N / 8
           | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z)
{
    float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// Wait for the phase of `parity` of the mbarrier to complete, polling at most
// `limit` times; false when the limit ran out (the caller records an error and
// unwinds instead of hanging).
__device__ __forceinline__ bool mbar_wait_n(uint32_t mbar, uint32_t parity, long long limit)
{
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// The same wait with a suspend-time hint: a thread whose phase is not complete
// is suspended (it issues nothing) until the phase completes or the hint runs
// out, so that waiting warps leave the issue slots to the working ones.  Bounded
// in time by the global timer (2 s), not by a poll count, as a try may return
// early or late.
constexpr unsigned SUSPEND_NS = 20000;
constexpr unsigned long long WAIT_NS = 2000000000ull;
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_wait_sleep(uint32_t mbar, uint32_t parity)
{
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "r"(SUSPEND_NS)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > WAIT_NS) return false;
    }
}

// byte offset of element (r, k) of a stage (rows x KC) in the core-matrix layout
// [r/8][k/8] of 128-byte core matrices: LBO (K direction) = 128, SBO (row groups) = KC/8 * 128
__device__ __forceinline__ uint32_t core_off(int r, int k) { return ((r >> 3) * (KC / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// Stage rows [r0, r0 + rows) x K range [k0, k0 + KC) of a bf16 operand into smem.
template <bool TRANS>
__device__ __forceinline__ void load_stage(uint8_t *dst, const __nv_bfloat16 *src, long long ld, int r0, int rows,
                                           int rmax, int k0, int kmax)
{
    if (!TRANS) {
        // 16-byte chunks: (row, 8 consecutive k)
        for (int i = threadIdx.x; i < rows * (KC / 8); i += blockDim.x) {
            int r = i / (KC / 8), kb = i % (KC / 8);
            int gr = r0 + r, gk = k0 + kb * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (gr < rmax && gk < kmax) v = *reinterpret_cast<const uint4 *>(src + (long long)gr * ld + gk);
            *reinterpret_cast<uint4 *>(dst + core_off(r, kb * 8)) = v;
        }
    } else {
        // element (r, k) at src[k*ld + r]: read 8 consecutive r at fixed k
        for (int i = threadIdx.x; i < (rows / 8) * KC; i += blockDim.x) {
            int k = i / (rows / 8), rb = i % (rows / 8);
            int gr = r0 + rb * 8, gk = k0 + k;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (gr < rmax && gk < kmax) v = *reinterpret_cast<const uint4 *>(src + (long long)gk * ld + gr);
            const uint16_t *e = reinterpret_cast<const uint16_t *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<uint16_t *>(dst + core_off(rb * 8 + j, k)) = e[j];
        }
    }
}

template <bool AT, bool BT>
__global__ void __launch_bounds__(128, 1) gemm_bf16(GemmArgs g)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA[2] = {smem, smem + A_STAGE};
    uint8_t *sB[2] = {smem + 2 * A_STAGE, smem + 2 * A_STAGE + B_STAGE};
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 2 * (A_STAGE + B_STAGE));
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * g.BN;
    const int kz0 = blockIdx.z * g.kper;
    const int kz1 = min(g.K, kz0 + g.kper);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = make_idesc(BM, g.BN);
    const int nchunks = (kz1 - kz0 + KC - 1) / KC;
    bool ok = true;
    int issued = 0;  // chunks whose MMAs were issued
    for (int c = 0; c < nchunks && ok; ++c) {
        const int buf = c & 1;
        // the decision to go on is taken by the whole CTA (barrier + vote)
        if (c >= 2) ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[buf]), ((c - 2) >> 1) & 1)) != 0;
        if (!ok) break;
        const int k0 = kz0 + c * KC;
        load_stage<AT>(sA[buf], g.A, g.lda, m0, BM, g.M, k0, kz1);
        load_stage<BT>(sB[buf], g.B, g.ldb, n0, g.BN, g.N, k0, kz1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int ksteps = (min(KC, kz1 - k0) + 15) / 16;  // a zero-filled tail adds nothing
            const uint32_t a0 = smem_u32(sA[buf]), b0 = smem_u32(sB[buf]);
            for (int kk = 0; kk < ksteps; ++kk) {
                const uint64_t ad = make_desc(a0 + kk * 256, 128, (KC / 8) * 128);
                const uint64_t bd = make_desc(b0 + kk * 256, 128, (KC / 8) * 128);
                const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[buf])));
        }
        issued = c + 1;
    }
    // wait for the last issued chunk (its commit covers all earlier MMAs)
    if (issued > 0) {
        const int c = issued - 1;
        ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[c & 1]), (c >> 1) & 1) && ok) != 0;
    }
    if (!ok && threadIdx.x == 0 && g.err) atomicExch(g.err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (ok && nchunks > 0) {
        const int row = m0 + warp * 32 + lane;
        for (int j = 0; j < g.BN; j += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row >= g.M) continue;
            const int nb = n0 + j;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = nb + i;
                if (n >= g.N) break;
                float a = __uint_as_float(v[i]);
                const long long off = (long long)row * g.ldz + n;
                switch (g.epi) {
                case EPI_F32:
                    if (gridDim.z > 1)
                        atomicAdd(g.C + (long long)row * g.ldc + n, a);
                    else
                        g.C[(long long)row * g.ldc + n] = a;
                    break;
                case EPI_BIAS:
                    g.C[(long long)row * g.ldc + n] = a + g.bias[n];
                    break;
                case EPI_BIAS_SILU: {
                    float z = a + g.bias[n];
                    __nv_bfloat16 zb = __float2bfloat16(z);
                    g.Z[off] = zb;
                    g.H[off] = __float2bfloat16(silu(__bfloat162float(zb)));
                    break;
                }
                case EPI_DSILU:
                    g.dZ[off] = __float2bfloat16(a * dsilu(__bfloat162float(g.Zin[off])));
                    break;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace umma
