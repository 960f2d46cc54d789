// Batched (alpha, k) sweeps: many plans with uneven grids run as batched
// persistent launches (3 for the synthesis, a counter reset and 3 for the
// evaluation), captured once into a CUDA graph and replayed.  The launch
// shapes are chosen by a small autotuner that times candidates on the batch
// itself.  Each pair keeps its own plan (tables, grid); the kernels are the
// bodies of the single-plan kernels, so a pair's results equal those of its
// plan evaluated alone (up to the grouping of far targets into warps).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <tuple>
#include <vector>

#include "gf_internal.cuh"

namespace {

struct GraphKey {
    const void *x;
    const void *out;
    int which;
    std::vector<int64_t> off;
    bool operator<(const GraphKey &o) const
    {
        return std::tie(x, out, which, off) < std::tie(o.x, o.out, o.which, o.off);
    }
};

// process-wide tuning cache: (pairs, total grid cells, precision, fields) -> choice
struct TuneChoice {
    int tj_max, far_block, far_per_sm;
};
std::map<std::tuple<int, long long, int, int>, TuneChoice> g_tune_cache;

gf_status err(gf_status s, const char *fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    return gf_set_error(s, msg);
}

#define CUB(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return err(e_ == cudaErrorMemoryAllocation ? GF_ERR_NOMEM : GF_ERR_CUDA, "%s: %s", #call, \
                       cudaGetErrorString(e_));                                                    \
    } while (0)

}  // namespace

struct gf_batch_s {
    int np = 0, precision = GF_FP64, nf = 1, nsm = 152;
    std::vector<gf_plan_t> plans;
    std::vector<SynthArgs> sargs;
    void *work = nullptr;             // synthesis work arena (all pairs)
    SynthArgs *d_sargs = nullptr;
    int *d_prefix = nullptr;          // 3 synthesis prefixes + near prefix, each np + 1
    std::vector<int> h_prefix[3];
    SynthBatch sb{};
    // evaluation
    EvalArgs *d_eargs = nullptr;
    int *scratch = nullptr;           // far lists: 2 * cap ints
    int64_t cap = 0;
    int *counters = nullptr;          // GF_SCRATCH_COUNTERS per pair
    EvalBatch eb{};
    GraphKey cur{};
    bool have_cur = false;
    TuneChoice tune{8, 128, 8};
    bool tuned = false;
    std::map<GraphKey, cudaGraphExec_t> graphs;
};

static gf_status batch_synth_setup(gf_batch_t b)
{
    // per-pass virtual-block prefix sums and the largest shared-memory need
    size_t smax[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) b->h_prefix[i].assign(b->np + 1, 0);
    for (int p = 0; p < b->np; ++p) {
        SynthArgs &a = b->sargs[p];
        size_t sm[3];
        gf_synth_config(a, b->precision, b->tune.tj_max, sm);
        for (int i = 0; i < 3; ++i) smax[i] = sm[i] > smax[i] ? sm[i] : smax[i];
        const int ncols = a.M1 * a.M2;
        b->h_prefix[0][p + 1] = b->h_prefix[0][p] + ncols / a.TJ;
        b->h_prefix[1][p + 1] = b->h_prefix[1][p] + (a.M1 / a.TJ2) * (a.L3count + a.nyq) * a.nf;
        b->h_prefix[2][p + 1] = b->h_prefix[2][p] + (a.L3count + a.nyq) * a.M2 / a.RB1;
    }
    for (int i = 0; i < 3; ++i)
        CUB(cudaMemcpy(b->d_prefix + i * (b->np + 1), b->h_prefix[i].data(), sizeof(int) * (b->np + 1),
                       cudaMemcpyHostToDevice));
    CUB(cudaMemcpy(b->d_sargs, b->sargs.data(), sizeof(SynthArgs) * b->np, cudaMemcpyHostToDevice));
    b->sb.args = b->d_sargs;
    b->sb.np = b->np;
    for (int i = 0; i < 3; ++i) {
        b->sb.prefix[i] = b->d_prefix + i * (b->np + 1);
        b->sb.smem[i] = smax[i];
        int tot = b->h_prefix[i][b->np];
        int g = b->nsm * 4;
        b->sb.grid[i] = tot < g ? tot : g;
    }
    return GF_OK;
}

static gf_status batch_eval_setup(gf_batch_t b, const double *x, const int64_t *off, int which, void *out)
{
    const int64_t total = off[b->np];
    if (total > b->cap) {
        CUB(cudaDeviceSynchronize());
        if (b->scratch) cudaFree(b->scratch);
        b->scratch = nullptr;
        b->cap = 0;
        CUB(cudaMalloc(&b->scratch, sizeof(int) * 3 * (size_t)(total > 0 ? total : 1)));
        b->cap = total;
    }
    const size_t elem = b->precision == GF_FP64 ? 16 : 8;
    const int ne = gf_out_entries(which);
    std::vector<EvalArgs> ea(b->np);
    std::vector<int> pre(b->np + 1, 0);
    for (int p = 0; p < b->np; ++p) {
        const int64_t n = off[p + 1] - off[p];
        gf_status s = gf_plan_eval_args(b->plans[p], x + 3 * off[p], n, which, (char *)out + elem * ne * off[p], &ea[p],
                                        "gf_batch_eval_points");
        if (s != GF_OK) return s;
        ea[p].far_idx = b->scratch + off[p];
        ea[p].far_sorted = b->scratch + b->cap + off[p];
        ea[p].near_idx = b->scratch + 2 * b->cap + off[p];
        ea[p].far_count = b->counters + (size_t)GF_SCRATCH_COUNTERS * p;
        pre[p + 1] = pre[p] + (int)((n + 255) / 256);
    }
    CUB(cudaMemcpy(b->d_eargs, ea.data(), sizeof(EvalArgs) * b->np, cudaMemcpyHostToDevice));
    CUB(cudaMemcpy(b->d_prefix + 3 * (b->np + 1), pre.data(), sizeof(int) * (b->np + 1), cudaMemcpyHostToDevice));
    b->eb.args = b->d_eargs;
    b->eb.prefix = b->d_prefix + 3 * (b->np + 1);
    b->eb.np = b->np;
    b->eb.nf = b->nf;
    b->eb.grid_near = pre[b->np] < b->nsm * 16 ? (pre[b->np] > 0 ? pre[b->np] : 1) : b->nsm * 16;
    b->eb.scatter_per_pair = 2;
    b->eb.near_lists = b->nf == 1;
    b->eb.grid_scatter = b->np * 2 < b->nsm * 4 ? b->np * 2 : b->nsm * 4;
    b->eb.block_far = b->tune.far_block;
    b->eb.grid_far = b->nsm * b->tune.far_per_sm * 128 / b->tune.far_block;
    b->cur = GraphKey{x, out, which, std::vector<int64_t>(off, off + b->np + 1)};
    b->have_cur = true;
    return GF_OK;
}

static gf_status batch_enqueue_eval(gf_batch_t b, cudaStream_t st)
{
    CUB(cudaMemsetAsync(b->counters, 0, sizeof(int) * GF_SCRATCH_COUNTERS * (size_t)b->np, st));
    CUB(gf_launch_eval_batch(b->eb, b->precision, st));
    return GF_OK;
}

static gf_status prepare_eval(gf_batch_t b, const double *x, const int64_t *off, int which, void *out)
{
    if (!off) return err(GF_ERR_ARG, "gf_batch: offsets is NULL");
    if (off[0] != 0) return err(GF_ERR_ARG, "gf_batch: offsets[0] must be 0");
    for (int p = 0; p < b->np; ++p)
        if (off[p + 1] < off[p]) return err(GF_ERR_ARG, "gf_batch: offsets must be non-decreasing");
    if (off[b->np] > 0x7fffffff) return err(GF_ERR_ARG, "gf_batch: too many targets");
    if (off[b->np] > 0 && (!x || !out)) return err(GF_ERR_ARG, "gf_batch: NULL buffer");
    GraphKey k{x, out, which, std::vector<int64_t>(off, off + b->np + 1)};
    if (b->have_cur && !(k < b->cur) && !(b->cur < k)) return GF_OK;
    return batch_eval_setup(b, x, off, which, out);
}

extern "C" {

gf_status gf_plan_batch(int npairs, const double *k, const double *alpha, const int *M, const gf_trunc_t *trunc,
                        void *cuda_stream, gf_batch_t *out)
{
    if (!out) return err(GF_ERR_ARG, "gf_plan_batch: out is NULL");
    *out = nullptr;
    if (npairs <= 0 || npairs > (1 << 20)) return err(GF_ERR_ARG, "gf_plan_batch: npairs = %d out of range", npairs);
    if (!k || !alpha || !M) return err(GF_ERR_ARG, "gf_plan_batch: NULL parameter array");
    gf_trunc_t tr;
    gf_trunc_default(&tr);
    if (trunc) tr = *trunc;
    if (tr.kind == GF_DERIV2D)
        return err(GF_ERR_UNSUPPORTED, "gf_plan_batch: derivative plans (GF_DERIV2D) are not batched; use gf_plan");
    gf_batch_s *b = new gf_batch_s();
    b->np = npairs;
    b->precision = tr.precision;
    b->nf = tr.kind == GF_MAXWELL ? 7 : 1;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    gf_status s = GF_OK;
    size_t wtot = 0;
    std::vector<size_t> woff(npairs);
    for (int p = 0; p < npairs && s == GF_OK; ++p) {
        gf_plan_t pl = nullptr;
        s = gf_plan(3, k[p], alpha + 2 * p, M + 3 * p, &tr, cuda_stream, &pl);
        if (s != GF_OK) {
            char msg[320];
            snprintf(msg, sizeof(msg), "gf_plan_batch: pair %d: %s", p, gf_last_error());
            gf_set_error(s, msg);
            break;
        }
        b->plans.push_back(pl);
        b->sargs.push_back(gf_plan_synth_args(pl));
        woff[p] = wtot;
        wtot += (gf_plan_work_bytes(pl) + 255) / 256 * 256;
    }
    if (s == GF_OK) {
        cudaError_t e;
        if ((e = cudaMalloc(&b->work, wtot)) != cudaSuccess ||
            (e = cudaMalloc(&b->d_sargs, sizeof(SynthArgs) * npairs)) != cudaSuccess ||
            (e = cudaMalloc(&b->d_prefix, sizeof(int) * 4 * (npairs + 1))) != cudaSuccess ||
            (e = cudaMalloc(&b->d_eargs, sizeof(EvalArgs) * npairs)) != cudaSuccess ||
            (e = cudaMalloc(&b->counters, sizeof(int) * GF_SCRATCH_COUNTERS * (size_t)npairs)) != cudaSuccess) {
            s = err(GF_ERR_NOMEM, "gf_plan_batch: cudaMalloc: %s", cudaGetErrorString(e));
        } else {
            for (int p = 0; p < npairs; ++p) b->sargs[p].work = (char *)b->work + woff[p];
            auto key = std::make_tuple(npairs, (long long)(wtot >> 10), b->precision, b->nf);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                b->tune = it->second;
                b->tuned = true;
            }
            s = batch_synth_setup(b);
        }
    }
    if (s != GF_OK) {
        gf_batch_destroy(b);
        return s;
    }
    *out = b;
    return GF_OK;
}

gf_status gf_batch_synthesize(gf_batch_t b, void *cuda_stream)
{
    if (!b) return err(GF_ERR_ARG, "gf_batch_synthesize: NULL batch");
    CUB(gf_launch_synth_batch(b->sb, b->precision, (cudaStream_t)cuda_stream));
    return GF_OK;
}

gf_status gf_batch_eval_points(gf_batch_t b, const double *dev_xyz, const int64_t *offsets, int which, void *dev_out,
                               void *cuda_stream)
{
    if (!b) return err(GF_ERR_ARG, "gf_batch_eval_points: NULL batch");
    gf_status s = prepare_eval(b, dev_xyz, offsets, which, dev_out);
    if (s != GF_OK) return s;
    return batch_enqueue_eval(b, (cudaStream_t)cuda_stream);
}

gf_status gf_batch_autotune(gf_batch_t b, const double *dev_xyz, const int64_t *offsets, int which, void *dev_out,
                            void *cuda_stream)
{
    if (!b) return err(GF_ERR_ARG, "gf_batch_autotune: NULL batch");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    gf_status s = prepare_eval(b, dev_xyz, offsets, which, dev_out);
    if (s != GF_OK) return s;
    cudaEvent_t e0, e1;
    CUB(cudaEventCreate(&e0));
    CUB(cudaEventCreate(&e1));
    // synthesis: columns per CTA of the first pass
    float best = 1e30f;
    int best_tj = b->tune.tj_max;
    const int tjs[4] = {2, 4, 8, 16};
    for (int i = 0; i < 4; ++i) {
        b->tune.tj_max = tjs[i];
        if ((s = batch_synth_setup(b)) != GF_OK) return s;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            CUB(cudaEventRecord(e0, st));
            CUB(gf_launch_synth_batch(b->sb, b->precision, st));
            CUB(cudaEventRecord(e1, st));
            CUB(cudaEventSynchronize(e1));
            CUB(cudaEventElapsedTime(&ms, e0, e1));
        }
        if (ms < best) {
            best = ms;
            best_tj = tjs[i];
        }
    }
    b->tune.tj_max = best_tj;
    if ((s = batch_synth_setup(b)) != GF_OK) return s;
    // far kernel: block size and CTAs per SM (in units of 128-thread blocks)
    best = 1e30f;
    TuneChoice bc = b->tune;
    const int blocks[3] = {64, 128, 256};
    const int per[3] = {4, 8, 16};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            b->tune.far_block = blocks[i];
            b->tune.far_per_sm = per[j];
            b->eb.block_far = blocks[i];
            b->eb.grid_far = b->nsm * per[j] * 128 / blocks[i];
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                CUB(cudaEventRecord(e0, st));
                if ((s = batch_enqueue_eval(b, st)) != GF_OK) return s;
                CUB(cudaEventRecord(e1, st));
                CUB(cudaEventSynchronize(e1));
                CUB(cudaEventElapsedTime(&ms, e0, e1));
            }
            if (ms < best) {
                best = ms;
                bc = b->tune;
            }
        }
    b->tune = bc;
    b->eb.block_far = bc.far_block;
    b->eb.grid_far = b->nsm * bc.far_per_sm * 128 / bc.far_block;
    b->tuned = true;
    size_t wtot = 0;
    for (int p = 0; p < b->np; ++p) wtot += (gf_plan_work_bytes(b->plans[p]) + 255) / 256 * 256;
    g_tune_cache[std::make_tuple(b->np, (long long)(wtot >> 10), b->precision, b->nf)] = bc;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // graphs captured with the old shapes are stale
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    return GF_OK;
}

gf_status gf_batch_get_tuning(gf_batch_t b, int out[3])
{
    if (!b || !out) return err(GF_ERR_ARG, "gf_batch_get_tuning: NULL argument");
    out[0] = b->tune.tj_max;
    out[1] = b->tune.far_block;
    out[2] = b->tune.far_per_sm;
    return GF_OK;
}

gf_status gf_batch_run_graph(gf_batch_t b, const double *dev_xyz, const int64_t *offsets, int which, void *dev_out,
                             void *cuda_stream)
{
    if (!b) return err(GF_ERR_ARG, "gf_batch_run_graph: NULL batch");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!st) return err(GF_ERR_ARG, "gf_batch_run_graph: needs a non-default stream");
    gf_status s = prepare_eval(b, dev_xyz, offsets, which, dev_out);
    if (s != GF_OK) return s;
    auto it = b->graphs.find(b->cur);
    if (it == b->graphs.end()) {
        cudaGraph_t g = nullptr;
        CUB(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = gf_launch_synth_batch(b->sb, b->precision, st);
        gf_status s2 = e1 == cudaSuccess ? batch_enqueue_eval(b, st) : GF_ERR_CUDA;
        cudaError_t e2 = cudaStreamEndCapture(st, &g);
        if (e1 != cudaSuccess || s2 != GF_OK || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return err(GF_ERR_CUDA, "gf_batch_run_graph: capture failed (%s / %s)", cudaGetErrorString(e1),
                       cudaGetErrorString(e2));
        }
        cudaGraphExec_t ex = nullptr;
        cudaError_t e3 = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) return err(GF_ERR_CUDA, "gf_batch_run_graph: instantiate: %s", cudaGetErrorString(e3));
        it = b->graphs.emplace(b->cur, ex).first;
    }
    CUB(cudaGraphLaunch(it->second, st));
    gf_count_launch(7);
    return GF_OK;
}

gf_status gf_batch_get_plan(gf_batch_t b, int i, gf_plan_t *out)
{
    if (!b || !out || i < 0 || i >= b->np) return err(GF_ERR_ARG, "gf_batch_get_plan: bad argument");
    *out = b->plans[i];
    return GF_OK;
}

gf_status gf_batch_destroy(gf_batch_t b)
{
    if (!b) return GF_OK;
    cudaDeviceSynchronize();
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (gf_plan_t p : b->plans) gf_destroy(p);
    if (b->work) cudaFree(b->work);
    if (b->d_sargs) cudaFree(b->d_sargs);
    if (b->d_prefix) cudaFree(b->d_prefix);
    if (b->d_eargs) cudaFree(b->d_eargs);
    if (b->scratch) cudaFree(b->scratch);
    if (b->counters) cudaFree(b->counters);
    delete b;
    return GF_OK;
}

}  // extern "C"
