// Arithmetic peak probes (diagnostics; the paper has no counterpart).
//
// The far-series kernels are bound by the FP64 and FP32 pipes, whose rates are
// not in the measured-peak record of the machine (it holds the HBM copy rate
// and the BF16 tensor rate).  These kernels measure them the plain way: every
// thread runs ILP independent chains of fused multiply-adds, so the pipe never
// waits on a result, and the grid fills every SM at full occupancy.
#include "gf_internal.cuh"
#include "umma_gemm.cuh"

namespace {

constexpr int PROBE_ILP = 8;
constexpr int PROBE_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) fma_chains(int64_t iters, T never, T *sink)
{
    T a[PROBE_ILP];
#pragma unroll
    for (int j = 0; j < PROBE_ILP; ++j) a[j] = (T)(threadIdx.x + 1 + j) * (T)1e-3;
    const T m = (T)0.9999999, c = (T)1e-7;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int j = 0; j < PROBE_ILP; ++j) a[j] = fma(a[j], m, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < PROBE_ILP; ++j) s += a[j];
    // never true (the chains stay positive); keeps the chains from being removed
    if (s == never) sink[0] = s;
}

// The overlap probe: even warps run FP64 chains (iters trips), odd warps FP32
// chains (GF_PROBE_FP32_PER_FP64 * iters trips, about as long at the two pipes'
// rates); `halves` selects which of them run (bit 0: FP64, bit 1: FP32).
template <typename T>
__device__ __forceinline__ T chains(int64_t iters, T never)
{
    T a[PROBE_ILP];
#pragma unroll
    for (int j = 0; j < PROBE_ILP; ++j) a[j] = (T)(threadIdx.x + 1 + j) * (T)1e-3;
    const T m = (T)0.9999999, c = (T)1e-7;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int j = 0; j < PROBE_ILP; ++j) a[j] = fma(a[j], m, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < PROBE_ILP; ++j) s += a[j];
    return s == never ? s : (T)0;
}

__global__ void __launch_bounds__(PROBE_THREADS) split_chains(int halves, int64_t iters, double *sink)
{
    const bool odd = ((threadIdx.x >> 5) & 1) != 0;
    double s = 0;
    if (!odd && (halves & 1)) s = chains<double>(iters, -1.0);
    if (odd && (halves & 2)) s = (double)chains<float>(iters * GF_PROBE_FP32_PER_FP64, -1.0f);
    if (s != 0) sink[0] = s;  // never (the chains stay positive)
}

}  // namespace

extern "C" gf_status gf_peak_probe(int pipe, int64_t iters, void *dev_sink, int64_t *flops, void *cuda_stream)
{
    if (pipe < GF_PROBE_FP64 || pipe > GF_PROBE_BOTH_HALVES || iters < 1 || iters > ((int64_t)1 << 20) ||
        !dev_sink || !flops)
        return gf_set_error(GF_ERR_ARG, "gf_peak_probe: bad argument");
    int dev = 0, nsm = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if (pipe >= GF_PROBE_FP64_HALF) {
        const int halves = pipe == GF_PROBE_FP64_HALF ? 1 : pipe == GF_PROBE_FP32_HALF ? 2 : 3;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, split_chains, PROBE_THREADS, 0);
        if (e == cudaSuccess) split_chains<<<per * nsm, PROBE_THREADS, 0, st>>>(halves, iters, (double *)dev_sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return gf_set_error(GF_ERR_CUDA, "gf_peak_probe: launch failed");
        gf_count_launch(1);
        const int64_t per_half = (int64_t)2 * PROBE_ILP * 8 * iters * (int64_t)per * nsm * (PROBE_THREADS / 2);
        *flops = ((halves & 1) ? per_half : 0) + ((halves & 2) ? per_half * GF_PROBE_FP32_PER_FP64 : 0);
        return GF_OK;
    }
    if (pipe == GF_PROBE_FP64) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fma_chains<double>, PROBE_THREADS, 0);
        if (e == cudaSuccess) fma_chains<double><<<per * nsm, PROBE_THREADS, 0, st>>>(iters, -1.0, (double *)dev_sink);
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fma_chains<float>, PROBE_THREADS, 0);
        if (e == cudaSuccess) fma_chains<float><<<per * nsm, PROBE_THREADS, 0, st>>>(iters, -1.0f, (float *)dev_sink);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return gf_set_error(GF_ERR_CUDA, "gf_peak_probe: launch failed");
    gf_count_launch(1);
    *flops = (int64_t)2 * PROBE_ILP * 8 * iters * (int64_t)per * nsm * PROBE_THREADS;
    return GF_OK;
}

namespace {

// One warp: lane 0 initialises an mbarrier expecting one arrival, arrives on it
// only when `arrive` is set, then waits for its phase 0 with the same bounded
// wait the tensor-core kernels use; the outcome goes to *flag (1: the wait ran
// out).  Nothing else touches the barrier, so without the arrival the wait can
// only end by its limit.
__global__ void wait_selftest_kernel(long long polls, int arrive, int *flag)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_u32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        if (arrive) {
            uint64_t state;
            asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(umma::smem_u32(&bar)) : "memory");
            (void)state;
        }
        *flag = umma::mbar_wait_n(umma::smem_u32(&bar), 0u, polls) ? 0 : 1;
    }
}

}  // namespace

extern "C" gf_status gf_wait_selftest(int64_t polls, int arrive, void *cuda_stream)
{
    if (polls < 1 || polls > ((int64_t)1 << 40)) return gf_set_error(GF_ERR_ARG, "gf_wait_selftest: polls out of range");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int *flag = nullptr;
    cudaError_t e = gf_dev_alloc((void **)&flag, sizeof(int), st);
    if (e != cudaSuccess) return gf_set_error(GF_ERR_NOMEM, "gf_wait_selftest: allocation failed");
    int host = -1;
    e = cudaMemsetAsync(flag, 0xff, sizeof(int), st);
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32, 0, st>>>((long long)polls, arrive ? 1 : 0, flag);
        gf_count_launch(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    gf_dev_free(flag, st);
    if (e != cudaSuccess) return gf_set_error(GF_ERR_CUDA, "gf_wait_selftest: CUDA error");
    if (host == 1) return gf_set_error(GF_ERR_TIMEOUT, "gf_wait_selftest: the bounded wait ran out");
    if (host != 0) return gf_set_error(GF_ERR_CUDA, "gf_wait_selftest: no result");
    return GF_OK;
}
