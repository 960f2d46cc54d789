// Device-memory pool and pinned upload staging shared by all plans.
//
// Plans are often built and dropped at a high rate (one per (alpha, k) pair of
// a sweep, one per step of a benchmark).  Their buffers come from a per-device
// stream-ordered memory pool that keeps freed memory reserved (release
// threshold: unlimited), so a new plan's allocations are pool hits, not driver
// calls; gf_release_memory() trims the pool.  Small host tables go up through
// a ring of pinned staging slots, so the upload is asynchronous and the host
// never waits for the stream except to recycle a slot still in flight.
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>

#include "gf_internal.cuh"

namespace {

std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t pool_for_current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps pr;
    memset(&pr, 0, sizeof(pr));
    pr.allocType = cudaMemAllocationTypePinned;
    pr.handleTypes = cudaMemHandleTypeNone;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &pr) != cudaSuccess) return nullptr;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pools[dev] = pool;
    return pool;
}

constexpr int kSlots = 8;
constexpr size_t kSlotBytes = 64 << 10;

struct Staging {
    char *base = nullptr;
    cudaEvent_t ev[kSlots] = {};
    bool pending[kSlots] = {};
    int next = 0;
};
std::mutex g_stage_mu;
std::map<int, Staging> g_stage;

}  // namespace

cudaError_t gf_dev_alloc(void **ptr, size_t bytes, cudaStream_t s)
{
    *ptr = nullptr;
    cudaMemPool_t pool = pool_for_current_device();
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(ptr, bytes ? bytes : 16, pool, s);
}

void gf_dev_free(void *ptr, cudaStream_t s)
{
    if (ptr) cudaFreeAsync(ptr, s);
}

cudaError_t gf_stage_upload(void *dev_dst, const void *src, size_t bytes, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_stage_mu);
    Staging &S = g_stage[dev];
    if (!S.base) {
        if ((e = cudaMallocHost((void **)&S.base, kSlots * kSlotBytes)) != cudaSuccess) {
            S.base = nullptr;
            return e;
        }
        for (int i = 0; i < kSlots; ++i)
            if ((e = cudaEventCreateWithFlags(&S.ev[i], cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    for (size_t off = 0; off < bytes; off += kSlotBytes) {
        const size_t m = bytes - off < kSlotBytes ? bytes - off : kSlotBytes;
        const int i = S.next;
        S.next = (S.next + 1) % kSlots;
        if (S.pending[i] && (e = cudaEventSynchronize(S.ev[i])) != cudaSuccess) return e;
        char *slot = S.base + (size_t)i * kSlotBytes;
        memcpy(slot, (const char *)src + off, m);
        if ((e = cudaMemcpyAsync((char *)dev_dst + off, slot, m, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(S.ev[i], s)) != cudaSuccess) return e;
        S.pending[i] = true;
    }
    return cudaSuccess;
}

cudaStream_t gf_aux_stream()
{
    static std::mutex mu;
    static std::map<int, cudaStream_t> streams;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    auto it = streams.find(dev);
    if (it != streams.end()) return it->second;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    streams[dev] = s;
    return s;
}

// One non-blocking stream per device for the host-buffer entry point's uploads,
// which then overlap work already queued on the caller's stream (null on failure).
cudaStream_t gf_copy_stream()
{
    static std::mutex mu;
    static std::map<int, cudaStream_t> streams;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    auto it = streams.find(dev);
    if (it != streams.end()) return it->second;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    streams[dev] = s;
    return s;
}

cudaError_t gf_trim_pool()
{
    cudaMemPool_t pool = pool_for_current_device();
    if (!pool) return cudaSuccess;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    return cudaMemPoolTrimTo(pool, 0);
}
