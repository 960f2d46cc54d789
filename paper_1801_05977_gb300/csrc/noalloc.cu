// Allocation-free evaluation entry point (gf_eval_points_noalloc).
//
// gf_eval_points keeps its far-target scratch list in the plan and grows it
// with cudaMalloc when a call brings more targets than before.  This variant
// instead uses one fixed scratch array declared below at file scope, so it
// never allocates or frees device memory.  The array is sized for
// GF_NOALLOC_MAX_TARGETS targets; it stays resident on every GPU that loads
// the library until the process exits, and all calls share it.
#include <mutex>
#include <stdio.h>

#include "gf_internal.cuh"

namespace {

// counters first (padded to 1024 ints), then the far list in append order and
// the bucket-sorted far list, each GF_NOALLOC_MAX_TARGETS long
constexpr int kCounterSlots = 1024;
static_assert(GF_SCRATCH_COUNTERS <= kCounterSlots, "counter block too small");
constexpr size_t kScratchInts = kCounterSlots + 2 * (size_t)GF_NOALLOC_MAX_TARGETS;

static __device__ __align__(256) int g_noalloc_scratch[kScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
int *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the symbol is only a host-side stand-in, so the address is obtained once
// per device with cudaGetSymbolAddress while that device is current.
gf_status scratch_for_current_device(int **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gf_set_error(GF_ERR_CUDA, "gf_eval_points_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return gf_set_error(GF_ERR_UNSUPPORTED, "gf_eval_points_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        int *ptr = nullptr;
        e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            char msg[256];
            snprintf(msg, sizeof(msg), "gf_eval_points_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return gf_set_error(GF_ERR_CUDA, msg);
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return GF_OK;
}

}  // namespace

extern "C" gf_status gf_eval_points_noalloc(gf_plan_t plan, const double *dev_xyz, int64_t n, int which,
                                            void *dev_out, void *cuda_stream)
{
    if (n > GF_NOALLOC_MAX_TARGETS) {
        char msg[160];
        snprintf(msg, sizeof(msg), "gf_eval_points_noalloc: n = %lld exceeds the fixed scratch limit of %d targets",
                 (long long)n, GF_NOALLOC_MAX_TARGETS);
        return gf_set_error(GF_ERR_ARG, msg);
    }
    EvalArgs a;
    gf_status s = gf_plan_eval_args(plan, dev_xyz, n, which, dev_out, &a, "gf_eval_points_noalloc");
    if (s != GF_OK) return s;
    if (n == 0) return GF_OK;
    int *scratch = nullptr;
    s = scratch_for_current_device(&scratch);
    if (s != GF_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the counters must start at zero; the lists are fully rewritten before they are read
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * kCounterSlots, st);
    if (e != cudaSuccess) return gf_set_error(GF_ERR_CUDA, "gf_eval_points_noalloc: counter reset failed");
    a.far_count = scratch;
    a.far_idx = scratch + kCounterSlots;
    a.far_sorted = scratch + kCounterSlots + GF_NOALLOC_MAX_TARGETS;
    gf_plan_info_t info;
    s = gf_plan_get_info(plan, &info);
    if (s != GF_OK) return s;
    e = gf_launch_eval(a, info.precision, st, nullptr);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "gf_eval_points_noalloc: launch failed: %s", cudaGetErrorString(e));
        return gf_set_error(GF_ERR_CUDA, msg);
    }
    return GF_OK;
}
