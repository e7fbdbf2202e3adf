// C ABI of the library (declared in include/mcpd.h): contexts, plans, runs, result transfer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define MCPD_NVTX 1
#endif

#include "mcpd_internal.h"

namespace {
// A named NVTX range over one library call (host side; a no-op unless a profiler is attached, and
// compiled out where the toolkit has no NVTX headers).
struct NvtxRange {
#ifdef MCPD_NVTX
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
#else
    explicit NvtxRange(const char *) {}
#endif
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

struct mcpd_plan {
    int device = -1;                 // the creating context's device (the context may go first)
    mcpd::Tables t;
    mcpd::KParams kp{};
    int grid = 0, block = 0;
    size_t smem = 0;
    long long pairs = 0;
    bool dirty = true;
    bool ran = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void *> allocs;
    double *est_dev = nullptr, *se_dev = nullptr;    // used by mcpd_decode
    int64_t n_trace = 0;
    int64_t slots_run = 0;           // slots in the buckets since the last run that cleared them
    long long last_pairs = 0;        // pairs the last launch held (its grid x block)
    mutable int64_t h2d_bytes = 0, d2h_bytes = 0;   // bytes copied between host and device (fetches too)
};

namespace {

int set_err(mcpd_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cu_status(mcpd_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return MCPD_OK;
    return set_err(ctx, e == cudaErrorMemoryAllocation ? MCPD_ENOMEM : MCPD_ECUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

// CU returns the library's status on a failed CUDA call; CU_OR runs `cleanup` first (used where
// the call fails after the object under construction holds device memory).
#define CU(call)                                                                              \
    do {                                                                                      \
        const int r_ = cu_status(ctx, (call), #call);                                         \
        if (r_ != MCPD_OK) return r_;                                                         \
    } while (0)
#define CU_OR(call, cleanup)                                                                  \
    do {                                                                                      \
        const int r_ = cu_status(ctx, (call), #call);                                         \
        if (r_ != MCPD_OK) { cleanup; return r_; }                                            \
    } while (0)

template <typename T>
int dev_alloc(mcpd_ctx *ctx, mcpd_plan *pl, T **ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) return MCPD_OK;
    void *p = nullptr;
    CU(cudaMalloc(&p, count * sizeof(T)));
    pl->allocs.push_back(p);
    *ptr = static_cast<T *>(p);
    return MCPD_OK;
}

}  // namespace

// The classes of a batch (mcpd_batch_create, mcpd_batch_classes): each instance's class in
// cls_of, classes numbered 0, 1, ... in launch order; returns their number.
static int assign_classes(const std::vector<mcpd::Tables> &t, int want_classes, int sm_count,
                          std::vector<int32_t> *cls_out) {
    const int32_t n_inst = static_cast<int32_t>(t.size());
    // Size classes: instances by pair state (words per column), largest first, cut into classes
    // of about equal work (slots x slot length), as many as whole rounds of a full launch allow
    // (at most four) unless the caller fixed the number.  With the number left to the library,
    // coupled instances of one uniform degree (3 to 8) are grouped by that degree first, so that
    // each class launches the build compiled for its degree, and every group is cut by size into
    // that many classes (at most one per instance).  Measured on 512 uneven instances with
    // degrees 4 to 8: four size classes per degree group beat one and two.
    auto work_of = [&](int32_t i) { return static_cast<double>(t[i].P) * static_cast<double>(std::max(t[i].B, t[i].unit)); };
    int64_t total_slots = 0;
    double total_work = 0.0;
    for (int32_t i = 0; i < n_inst; ++i) { total_slots += t[i].P; total_work += work_of(i); }
    int n_cls = want_classes;
    if (n_cls == 0) {
        const int64_t round = static_cast<int64_t>(sm_count) * 32 * 20;
        n_cls = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(4, total_slots / std::max<int64_t>(1, round))));
    }
    n_cls = std::min(n_cls, n_inst);
    std::vector<int32_t> key(n_inst, 0);       // degree group (0: any degree, the generic build)
    if (want_classes == 0)
        for (int32_t i = 0; i < n_inst; ++i) key[i] = mcpd::batch_kernel_degree(t[0].coupled ? 1 : 0, 0, t[i].udeg);
    // instances by group, then largest pair state first
    std::vector<int32_t> by_size(n_inst);
    for (int32_t i = 0; i < n_inst; ++i) by_size[i] = i;
    std::stable_sort(by_size.begin(), by_size.end(), [&](int32_t a, int32_t c) {
        if (key[a] != key[c]) return key[a] < key[c];
        return t[a].wpp > t[c].wpp;
    });
    std::vector<int32_t> cls_of(n_inst, 0);
    {
        int base = 0;
        for (int32_t g0 = 0; g0 < n_inst;) {
            int32_t g1 = g0;
            double gwork = 0.0;
            while (g1 < n_inst && key[by_size[g1]] == key[by_size[g0]]) gwork += work_of(by_size[g1++]);
            const int32_t gn = g1 - g0;
            const int ng = std::max(1, std::min(n_cls, gn));
            double acc = 0.0;
            for (int32_t pos = g0; pos < g1; ++pos) {
                const int32_t i = by_size[pos];
                const int32_t k = pos - g0;
                int c = static_cast<int>(gwork > 0 ? acc / gwork * ng : 0.0);
                c = std::min(c, ng - 1);
                // every class keeps at least one instance
                c = std::max(c, ng - (gn - k));
                c = std::min(c, k);
                cls_of[i] = base + c;
                acc += work_of(i);
            }
            base += ng;
            g0 = g1;
        }
        // number the classes that received instances 0, 1, ... (a heavy instance may skip one)
        int next = 0, last = -1;
        for (int32_t pos = 0; pos < n_inst; ++pos) {
            const int32_t i = by_size[pos];
            if (cls_of[i] != last) { last = cls_of[i]; ++next; }
            cls_of[i] = next - 1;
        }
    }
    *cls_out = cls_of;
    int n_cls_out = 0;
    for (int32_t i = 0; i < n_inst; ++i) n_cls_out = std::max(n_cls_out, cls_of[i] + 1);
    return n_cls_out;
}

extern "C" {

int mcpd_ctx_create(int device, void *cuda_stream, mcpd_ctx **out) {
    if (!out) return MCPD_EINVAL;
    *out = nullptr;
    mcpd_ctx *ctx = new (std::nothrow) mcpd_ctx();
    if (!ctx) return MCPD_ENOMEM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        mcpd::pairs_max_smem(device, &ctx->smem_optin) != MCPD_OK) {
        delete ctx;
        return MCPD_ECUDA;
    }
    *out = ctx;
    return MCPD_OK;
}

void mcpd_ctx_destroy(mcpd_ctx *ctx) { delete ctx; }

const char *mcpd_last_error(const mcpd_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void mcpd_plan_destroy(mcpd_plan *pl) {
    if (!pl) return;
    if (pl->device >= 0) cudaSetDevice(pl->device);
    for (void *p : pl->allocs) cudaFree(p);
    if (pl->ev0) cudaEventDestroy(pl->ev0);
    if (pl->ev1) cudaEventDestroy(pl->ev1);
    delete pl;
}

int mcpd_plan_create(mcpd_ctx *ctx, const mcpd_design *design, const uint8_t *y,
                     const mcpd_params *params, mcpd_plan **out) {
    NvtxRange nvtx_range("mcpd.plan_create");
    if (!ctx || !out) return MCPD_EINVAL;
    *out = nullptr;
    mcpd_plan *pl = new (std::nothrow) mcpd_plan();
    if (!pl) return set_err(ctx, MCPD_ENOMEM, "host allocation");
    pl->device = ctx->device;
    std::string err;
    int rc = mcpd::build_tables(design, y, params, &pl->t, &err);
    if (rc != MCPD_OK) { delete pl; return set_err(ctx, rc, err); }
    const mcpd::Tables &t = pl->t;
    if (cudaSetDevice(ctx->device) != cudaSuccess) { delete pl; return set_err(ctx, MCPD_ECUDA, "cudaSetDevice"); }

    // Launch shape: tables first in shared memory, then one 32-column region per warp and the
    // Y regions.
    const size_t tables = mcpd::kernel_table_bytes(t);
    mcpd::PairsShape shape;
    rc = mcpd::pairs_shape(t.coupled, t.scan, t.udeg, false, tables, t.wpp, ctx->smem_optin, t.P,
                           ctx->sm_count, 0, t.capped || t.lag > 1, !t.Tnu.empty(), &shape);
    if (rc != MCPD_OK) {
        delete pl;
        return set_err(ctx, rc, rc == MCPD_ETOO_LARGE ? "instance too large for the one-thread-per-pair layout"
                                                      : "launch shape (cudaFuncSetAttribute / occupancy)");
    }
    const int warps = shape.warps;
    pl->block = warps * 32;
    pl->smem = shape.smem;
    pl->grid = ctx->sm_count * shape.per_sm;
    pl->pairs = static_cast<long long>(pl->grid) * pl->block;

    mcpd::KParams &kp = pl->kp;
    uint64_t *d_alias = nullptr, *d_T = nullptr, *d_Tnu = nullptr;
    uint16_t *d_rows = nullptr;
    uint32_t *d_init = nullptr;
#define ALLOC(ptr, n)                                                        \
    do {                                                                     \
        int r_ = dev_alloc(ctx, pl, &(ptr), (n));                            \
        if (r_ != MCPD_OK) { mcpd_plan_destroy(pl); return r_; }             \
    } while (0)
    ALLOC(d_alias, t.alias.size());
    ALLOC(d_rows, mcpd::kernel_rows(t).size());
    ALLOC(d_T, mcpd::kernel_T(t).size());
    ALLOC(d_Tnu, t.Tnu.size());
    ALLOC(d_init, t.init_pairs.size());
    ALLOC(kp.pair_scratch, static_cast<size_t>(pl->pairs) * mcpd::pair_words(t.na, t.W));
    ALLOC(kp.y_state, static_cast<size_t>(pl->pairs) * t.wpp);
    ALLOC(kp.S1, static_cast<size_t>(t.nb) * t.na);
    ALLOC(kp.S2lo, static_cast<size_t>(t.nb) * t.na);
    ALLOC(kp.S2hi, static_cast<size_t>(t.nb) * t.na);
    ALLOC(kp.bcount, static_cast<size_t>(t.nb));
    ALLOC(kp.counters, static_cast<size_t>(mcpd::kNumCounters));
    ALLOC(kp.error, 1);
    ALLOC(pl->est_dev, static_cast<size_t>(t.na));
    ALLOC(pl->se_dev, static_cast<size_t>(t.na));
    if (t.record_slots) {
        ALLOC(kp.slot_nstar, static_cast<size_t>(t.P));
        ALLOC(kp.slot_S, static_cast<size_t>(t.P));
        ALLOC(kp.slot_reps, static_cast<size_t>(t.P));
    }
    if (t.trace_stride > 0) {
        pl->n_trace = (t.P + t.trace_stride - 1) / t.trace_stride;
        ALLOC(kp.trace_G, static_cast<size_t>(pl->n_trace) * t.na);
        if (t.trace_steps > 0)
            ALLOC(kp.trace_rec, static_cast<size_t>(pl->n_trace) * t.trace_reps * (4 + t.trace_steps));
    }
#undef ALLOC
    CU_OR(cudaMemcpyAsync(d_alias, t.alias.data(), t.alias.size() * 8, cudaMemcpyHostToDevice, ctx->stream), mcpd_plan_destroy(pl));
    CU_OR(cudaMemcpyAsync(d_rows, mcpd::kernel_rows(t).data(), mcpd::kernel_rows(t).size() * 2, cudaMemcpyHostToDevice, ctx->stream), mcpd_plan_destroy(pl));
    CU_OR(cudaMemcpyAsync(d_T, mcpd::kernel_T(t).data(), mcpd::kernel_T(t).size() * 8, cudaMemcpyHostToDevice, ctx->stream), mcpd_plan_destroy(pl));
    if (!t.Tnu.empty())
        CU_OR(cudaMemcpyAsync(d_Tnu, t.Tnu.data(), t.Tnu.size() * 8, cudaMemcpyHostToDevice, ctx->stream), mcpd_plan_destroy(pl));
    if (!t.init_pairs.empty())
        CU_OR(cudaMemcpyAsync(d_init, t.init_pairs.data(), t.init_pairs.size() * 4, cudaMemcpyHostToDevice, ctx->stream), mcpd_plan_destroy(pl));
    pl->h2d_bytes += static_cast<int64_t>(t.alias.size() * 8 + mcpd::kernel_rows(t).size() * 2 +
                                          mcpd::kernel_T(t).size() * 8 + t.Tnu.size() * 8 + t.init_pairs.size() * 4);
    kp.alias = d_alias; kp.rows = d_rows; kp.T = d_T; kp.Tnu = t.Tnu.empty() ? nullptr : d_Tnu;
    kp.init_pairs = d_init; kp.n_init_pairs = static_cast<int32_t>(t.init_pairs.size());
    kp.na = t.na; kp.m = t.m; kp.W = t.W; kp.Mp = t.Mp; kp.wpp = t.wpp; kp.deg = t.deg_max; kp.udeg = t.udeg;
    kp.nb = static_cast<int32_t>(t.nb); kp.scan = t.scan;
    kp.dummy_entry = t.dummy_entry; kp.dummy_word = t.dummy_word;
    kp.dummy_word_index = t.dummy_word_index; kp.coupled = t.coupled ? 1 : 0;
    kp.P = t.P; kp.B = t.B; kp.k = t.k; kp.ell = t.ell; kp.L = t.L; kp.burn = t.burn;
    kp.length = t.length; kp.unit = t.unit; kp.step_limit = t.step_limit; kp.tau_audit = t.tau_audit;
    kp.capped = t.capped ? 1 : 0;
    kp.lag = static_cast<int32_t>(t.lag);
    kp.slot_offset = t.slot_offset; kp.trace_stride = t.trace_stride;
    kp.trace_reps = static_cast<int32_t>(t.trace_reps); kp.trace_steps = static_cast<int32_t>(t.trace_steps);
    kp.seed = t.seed; mcpd::philox_round_keys(t.seed, kp.rk); kp.instance = t.instance; kp.warps = warps;
    kp.smem_tables = static_cast<uint32_t>(tables);
    kp.nT = static_cast<int32_t>(mcpd::kernel_T(t).size());
    kp.y_regions = shape.y_regions;
    CU_OR(cudaEventCreate(&pl->ev0), mcpd_plan_destroy(pl));
    CU_OR(cudaEventCreate(&pl->ev1), mcpd_plan_destroy(pl));
    CU_OR(cudaStreamSynchronize(ctx->stream), mcpd_plan_destroy(pl));
    *out = pl;
    return MCPD_OK;
}

int mcpd_plan_info(const mcpd_plan *pl, int64_t info[16]) {
    if (!pl || !info) return MCPD_EINVAL;
    const mcpd::Tables &t = pl->t;
    std::memset(info, 0, 16 * sizeof(int64_t));
    info[0] = t.na; info[1] = t.nb; info[2] = t.B;
    info[3] = t.k; info[4] = t.ell; info[5] = t.L; info[6] = t.P;
    info[7] = pl->block / 32; info[8] = pl->pairs; info[9] = static_cast<int64_t>(pl->smem);
    info[10] = 1; info[11] = pl->grid; info[12] = t.step_limit; info[13] = t.deg_max;
    return MCPD_OK;
}

int mcpd_plan_active(const mcpd_plan *pl, int32_t *active) {
    if (!pl || !active) return MCPD_EINVAL;
    std::memcpy(active, pl->t.active.data(), pl->t.active.size() * sizeof(int32_t));
    return MCPD_OK;
}

namespace {

// Enqueue the sampler over `slots` slots and the finalize.  accumulate = 0: the buckets are cleared
// and the slots are the plan's first (global ids slot_offset + 0 ..); accumulate = 1: the slots
// continue the ones already in the buckets (global ids slot_offset + slots_run ..) and their sums
// are added.  Either way est/se are finalized over every slot in the buckets.
int run_range(mcpd_ctx *ctx, mcpd_plan *pl, int64_t slots, bool accumulate, double *est_dev, double *se_dev) {
    if (!ctx || !pl || !est_dev || !se_dev) return MCPD_EINVAL;
    const mcpd::Tables &t = pl->t;
    if (slots < 1) return set_err(ctx, MCPD_EINVAL, "slots must be >= 1");
    if (accumulate && !pl->ran) return set_err(ctx, MCPD_EINVAL, "nothing to accumulate onto: run the plan first");
    const int64_t first = accumulate ? pl->slots_run : 0;
    if (first + slots > (int64_t(1) << 31) || t.slot_offset + first + slots > (int64_t(1) << 32))
        return set_err(ctx, MCPD_EINVAL, "accumulated slots beyond 2^31, or global slot ids beyond 32 bits");
    if ((t.record_slots || t.trace_stride > 0) && (accumulate || slots > t.P))
        return set_err(ctx, MCPD_EINVAL, "per-slot records and traces cover one run of at most the plan's slots");
    CU(cudaSetDevice(ctx->device));
    mcpd::KParams kp = pl->kp;
    kp.P = slots;
    kp.slot_offset = t.slot_offset + first;
    // Launch shape: the plan's, with its warps per block trimmed to the fewest that need no more
    // rounds of slots for this run (the plan's own slot count gives the plan's shape).
    int warps = pl->block / 32;
    {
        const long long per_round = static_cast<long long>(pl->grid) * 32;
        const long long rounds = (slots + per_round * warps - 1) / (per_round * warps);
        const long long w = (slots + rounds * per_round - 1) / (rounds * per_round);
        if (w >= 1 && w < warps) warps = static_cast<int>(w);
    }
    kp.warps = warps;
    kp.y_regions = mcpd::pairs_y_regions(t.coupled, warps);
    const size_t smem = mcpd::pairs_smem_bytes(kp.smem_tables, t.wpp, warps, kp.y_regions);
    const size_t nbna = static_cast<size_t>(t.nb) * t.na;
    if (!accumulate) {
        CU(cudaMemsetAsync(kp.S1, 0, nbna * 8, ctx->stream));
        CU(cudaMemsetAsync(kp.S2lo, 0, nbna * 8, ctx->stream));
        CU(cudaMemsetAsync(kp.S2hi, 0, nbna * 8, ctx->stream));
        CU(cudaMemsetAsync(kp.bcount, 0, static_cast<size_t>(t.nb) * 8, ctx->stream));
    }
    CU(cudaMemsetAsync(kp.counters, 0, mcpd::kNumCounters * 8, ctx->stream));
    CU(cudaMemsetAsync(kp.error, 0, sizeof(int), ctx->stream));
    if (pl->dirty) {   // the kernel leaves these zeroed when it completes normally
        CU(cudaMemsetAsync(kp.pair_scratch, 0, static_cast<size_t>(pl->pairs) * mcpd::pair_words(t.na, t.W) * 8, ctx->stream));
        CU(cudaMemsetAsync(kp.y_state, 0, static_cast<size_t>(pl->pairs) * t.wpp * 4, ctx->stream));
    }
    if (kp.trace_G) CU(cudaMemsetAsync(kp.trace_G, 0, static_cast<size_t>(pl->n_trace) * t.na * 8, ctx->stream));
    if (kp.trace_rec)
        CU(cudaMemsetAsync(kp.trace_rec, 0, static_cast<size_t>(pl->n_trace) * t.trace_reps * (4 + t.trace_steps) * 4,
                           ctx->stream));
    if (kp.slot_nstar) {
        CU(cudaMemsetAsync(kp.slot_nstar, 0, static_cast<size_t>(t.P) * 4, ctx->stream));
        CU(cudaMemsetAsync(kp.slot_S, 0, static_cast<size_t>(t.P) * 8, ctx->stream));
        CU(cudaMemsetAsync(kp.slot_reps, 0, static_cast<size_t>(t.P) * 4, ctx->stream));
    }
    pl->dirty = true;
    pl->ran = false;                 // until the launches are enqueued
    CU(cudaEventRecord(pl->ev0, ctx->stream));
    if (mcpd::launch_pairs(kp, pl->grid, warps * 32, smem, ctx->stream) != MCPD_OK)
        return set_err(ctx, MCPD_ECUDA, std::string("pairs kernel launch: ") + cudaGetErrorString(cudaGetLastError()));
    CU(cudaEventRecord(pl->ev1, ctx->stream));
    if (mcpd::launch_finalize(kp.S1, kp.S2lo, kp.S2hi, t.na, static_cast<int>(t.nb), first + slots, t.L, est_dev,
                              se_dev, ctx->stream) != MCPD_OK)
        return set_err(ctx, MCPD_ECUDA, "finalize kernel launch");
    pl->ran = true;
    pl->slots_run = first + slots;
    pl->last_pairs = static_cast<long long>(pl->grid) * warps * 32;
    return MCPD_OK;
}

}  // namespace

int mcpd_run_async(mcpd_ctx *ctx, mcpd_plan *pl, double *est_dev, double *se_dev) {
    NvtxRange nvtx_range("mcpd.run");
    if (!pl) return MCPD_EINVAL;
    return run_range(ctx, pl, pl->t.P, false, est_dev, se_dev);
}

int mcpd_run_slots_async(mcpd_ctx *ctx, mcpd_plan *pl, int64_t slots, int32_t accumulate, double *est_dev,
                         double *se_dev) {
    NvtxRange nvtx_range("mcpd.run_slots");
    if (accumulate != 0 && accumulate != 1) return set_err(ctx, MCPD_EINVAL, "accumulate must be 0 or 1");
    return run_range(ctx, pl, slots, accumulate != 0, est_dev, se_dev);
}

int mcpd_collect(mcpd_ctx *ctx, mcpd_plan *pl, mcpd_stats *stats) {
    NvtxRange nvtx_range("mcpd.collect");
    if (!ctx || !pl) return MCPD_EINVAL;
    if (!pl->ran) return set_err(ctx, MCPD_EINVAL, "no run to collect");
    CU(cudaSetDevice(ctx->device));
    unsigned long long c[mcpd::kNumCounters];
    int error = 0;
    CU(cudaMemcpyAsync(c, pl->kp.counters, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(&error, pl->kp.error, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    pl->d2h_bytes += static_cast<int64_t>(sizeof(c) + sizeof(int));
    CU(cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, pl->ev0, pl->ev1));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        mcpd::counters_to_stats(c, stats);
        stats->n_buckets = pl->t.nb;
        stats->n_active = pl->t.na;
        stats->kernel_ms = ms;
        stats->resident_pairs = pl->last_pairs;
        stats->h2d_bytes = pl->h2d_bytes;
        stats->d2h_bytes = pl->d2h_bytes;
    }
    if (error) return set_err(ctx, MCPD_ESTEP_LIMIT, "a pair reached the step limit without meeting");
    pl->dirty = false;
    return MCPD_OK;
}

size_t mcpd_fetch_bytes(const mcpd_plan *pl, int what) {
    if (!pl) return 0;
    const size_t nbna = static_cast<size_t>(pl->t.nb) * pl->t.na;
    switch (what) {
        case MCPD_FETCH_S1: case MCPD_FETCH_S2_LO: case MCPD_FETCH_S2_HI: return nbna * 8;
        case MCPD_FETCH_COUNT: return static_cast<size_t>(pl->t.nb) * 8;
        case MCPD_FETCH_SLOT_NSTAR: return pl->kp.slot_nstar ? static_cast<size_t>(pl->t.P) * 4 : 0;
        case MCPD_FETCH_SLOT_S: return pl->kp.slot_S ? static_cast<size_t>(pl->t.P) * 8 : 0;
        case MCPD_FETCH_SLOT_REPS: return pl->kp.slot_reps ? static_cast<size_t>(pl->t.P) * 4 : 0;
        case MCPD_FETCH_TRACE_G: return pl->kp.trace_G ? static_cast<size_t>(pl->n_trace) * pl->t.na * 8 : 0;
        case MCPD_FETCH_TRACE_REC:
            return pl->kp.trace_rec ? static_cast<size_t>(pl->n_trace) * pl->t.trace_reps * (4 + pl->t.trace_steps) * 4 : 0;
        default: return 0;
    }
}

int mcpd_fetch(mcpd_ctx *ctx, const mcpd_plan *pl, int what, void *host_dst, size_t bytes) {
    if (!ctx || !pl || !host_dst) return MCPD_EINVAL;
    const size_t need = mcpd_fetch_bytes(pl, what);
    if (need == 0 || bytes != need) return set_err(ctx, MCPD_EINVAL, "fetch: wrong kind or size");
    const void *src = nullptr;
    switch (what) {
        case MCPD_FETCH_S1: src = pl->kp.S1; break;
        case MCPD_FETCH_S2_LO: src = pl->kp.S2lo; break;
        case MCPD_FETCH_S2_HI: src = pl->kp.S2hi; break;
        case MCPD_FETCH_COUNT: src = pl->kp.bcount; break;
        case MCPD_FETCH_SLOT_NSTAR: src = pl->kp.slot_nstar; break;
        case MCPD_FETCH_SLOT_S: src = pl->kp.slot_S; break;
        case MCPD_FETCH_SLOT_REPS: src = pl->kp.slot_reps; break;
        case MCPD_FETCH_TRACE_G: src = pl->kp.trace_G; break;
        case MCPD_FETCH_TRACE_REC: src = pl->kp.trace_rec; break;
    }
    CU(cudaSetDevice(ctx->device));
    CU(cudaMemcpyAsync(host_dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    pl->d2h_bytes += static_cast<int64_t>(bytes);
    return MCPD_OK;
}

int mcpd_decode(mcpd_ctx *ctx, const mcpd_design *design, const uint8_t *y,
                const mcpd_params *params, double *est, double *se, int32_t *active,
                mcpd_stats *stats) {
    NvtxRange nvtx_range("mcpd.decode");
    if (!ctx || !design || !est || !se) return MCPD_EINVAL;
    mcpd_plan *pl = nullptr;
    int rc = mcpd_plan_create(ctx, design, y, params, &pl);
    if (rc != MCPD_OK) return rc;
    rc = mcpd_run_async(ctx, pl, pl->est_dev, pl->se_dev);
    if (rc == MCPD_OK) rc = mcpd_collect(ctx, pl, stats);
    if (rc == MCPD_OK || rc == MCPD_ESTEP_LIMIT) {
        const int32_t na = pl->t.na;
        std::vector<double> e(na), s(na);
        cudaError_t c1 = cudaMemcpyAsync(e.data(), pl->est_dev, na * 8, cudaMemcpyDeviceToHost, ctx->stream);
        cudaError_t c2 = cudaMemcpyAsync(s.data(), pl->se_dev, na * 8, cudaMemcpyDeviceToHost, ctx->stream);
        cudaError_t c3 = cudaStreamSynchronize(ctx->stream);
        if (c1 != cudaSuccess || c2 != cudaSuccess || c3 != cudaSuccess) {
            rc = set_err(ctx, MCPD_ECUDA, "copying results to the host");
        } else {
            if (stats) stats->d2h_bytes += static_cast<int64_t>(2 * na * 8);
            for (int32_t i = 0; i < design->n_clones; ++i) { est[i] = 0.0; se[i] = 0.0; if (active) active[i] = 0; }
            for (int32_t a = 0; a < na; ++a) {
                const int32_t i = pl->t.active[a];
                est[i] = e[a]; se[i] = s[a];
                if (active) active[i] = 1;
            }
        }
    }
    mcpd_plan_destroy(pl);
    return rc;
}

int mcpd_inspect(const mcpd_design *design, const uint8_t *y, const mcpd_params *params,
                 int64_t info[16], int32_t *active, double *w, uint64_t *alias, uint64_t *T) {
    NvtxRange nvtx_range("mcpd.inspect");
    if (!info) return MCPD_EINVAL;
    mcpd::Tables t;
    std::string err;
    const int rc = mcpd::build_tables(design, y, params, &t, &err);
    if (rc != MCPD_OK) return rc;
    std::memset(info, 0, 16 * sizeof(int64_t));
    info[0] = t.na; info[1] = t.nb; info[2] = t.B; info[3] = t.k; info[4] = t.ell; info[5] = t.L;
    info[6] = t.P; info[12] = t.step_limit; info[13] = t.deg_max;
    if (active) std::memcpy(active, t.active.data(), t.active.size() * sizeof(int32_t));
    if (w) std::memcpy(w, t.w.data(), t.w.size() * sizeof(double));
    if (alias) std::memcpy(alias, t.alias.data(), t.alias.size() * sizeof(uint64_t));
    if (T) std::memcpy(T, t.T.data(), t.T.size() * sizeof(uint64_t));
    return MCPD_OK;
}

int mcpd_batch_classes(int32_t n_inst, const mcpd_design *designs, const uint8_t *const *ys,
                       const mcpd_params *params, int32_t order_mode, int32_t sm_count,
                       int32_t *class_of, int32_t *n_classes) {
    if (n_inst < 1 || !designs || !ys || !params || !class_of || !n_classes || sm_count < 1) return MCPD_EINVAL;
    const int32_t want_classes = (order_mode >> 8) & 0xFF;
    if ((order_mode & 0xFF) > 1 || want_classes > 8 || (order_mode >> 16) != 0) return MCPD_EINVAL;
    std::vector<mcpd::Tables> t(n_inst);
    for (int32_t i = 0; i < n_inst; ++i) {
        std::string err;
        const int rc = mcpd::build_tables(&designs[i], ys[i], &params[i], &t[i], &err);
        if (rc != MCPD_OK) return rc;
        if (t[i].coupled != t[0].coupled || (t[i].scan == MCPD_SCAN_SYSTEMATIC) != (t[0].scan == MCPD_SCAN_SYSTEMATIC))
            return MCPD_EINVAL;
    }
    std::vector<int32_t> cls;
    *n_classes = assign_classes(t, want_classes, sm_count, &cls);
    std::memcpy(class_of, cls.data(), static_cast<size_t>(n_inst) * sizeof(int32_t));
    return MCPD_OK;
}

int mcpd_philox_device(mcpd_ctx *ctx, const uint32_t *ctr_dev, uint32_t key0, uint32_t key1,
                       uint32_t *out_dev, int64_t n) {
    if (!ctx || (n > 0 && (!ctr_dev || !out_dev)) || n < 0) return MCPD_EINVAL;
    CU(cudaSetDevice(ctx->device));
    if (mcpd::launch_philox(ctr_dev, key0, key1, out_dev, n, ctx->stream) != MCPD_OK)
        return set_err(ctx, MCPD_ECUDA, "philox kernel launch");
    CU(cudaStreamSynchronize(ctx->stream));
    return MCPD_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Batched decoding: many instances of uneven size in one persistent launch.

// One size class of a batch: instances with similar pair state, launched together so that the
// launch shape (warps per block) fits their columns rather than the largest instance's.
struct BatchClass {
    int32_t first = 0, count = 0;      // positions [first, first + count) of the launch order
    mcpd::BParams bp{};                // this class's launch arguments (insts = d_insts + first)
    int grid = 0, block = 0, warps = 0;
    size_t smem = 0;
    long long pairs = 0, scratch_pairs = 0;
    std::vector<void *> scratch;       // per-pair scratch (resized by the tuner)
};

struct mcpd_batch {
    int device = -1;                       // the creating context's device (the context may go first)
    std::vector<mcpd::Tables> t;
    std::vector<int32_t> order;            // launch order of instances (class-major, then instance-major)
    std::vector<int64_t> out_offset;       // [n + 1] offsets of each instance's clones in est/se
    std::vector<int64_t> bucket_offset;    // [n] offsets of each instance's buckets (in nb*na units)
    std::vector<int64_t> count_offset;     // [n]
    std::vector<BatchClass> cls;
    int32_t n_inst = 0, lanes = 1;
    bool coupled = true;
    mcpd::InstDesc *d_insts = nullptr;
    std::vector<mcpd::InstDesc> insts;     // in launch order, as the device holds them
    std::vector<mcpd::InstDesc> insts0;    // the descriptors of a decode from the first slot
    std::vector<long long> total_work0;    // per class, for those
    bool extended = false;                 // the device descriptors describe an extension
    // The size classes launch concurrently, each on its own stream forked from the context's
    // stream and joined back before the finalize: a class's last, partly filled round of pairs
    // overlaps the next class's launch instead of leaving SMs idle.
    std::vector<cudaStream_t> cls_streams;
    std::vector<cudaEvent_t> cls_done;
    cudaEvent_t fork = nullptr;
    int32_t *d_clone_inst = nullptr, *d_clone_local = nullptr;
    unsigned long long *d_buckets = nullptr;   // S1 | S2lo | S2hi, each total_bucket_words
    unsigned long long *d_bcount = nullptr;
    unsigned long long *d_counters = nullptr;  // [classes][kNumCounters]
    int *d_error = nullptr;
    size_t total_bucket_words = 0, total_counts = 0;
    int64_t total_active = 0, total_slots = 0;
    bool dirty = true, ran = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<void *> allocs;            // tables, descriptors, buckets (fixed)
};

namespace {

template <typename T>
int balloc(mcpd_ctx *ctx, std::vector<void *> &list, T **ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) return MCPD_OK;
    void *p = nullptr;
    CU(cudaMalloc(&p, count * sizeof(T)));
    list.push_back(p);
    *ptr = static_cast<T *>(p);
    return MCPD_OK;
}

void free_list(std::vector<void *> &list) {
    for (void *p : list) cudaFree(p);
    list.clear();
}

// Launch shape of every class: `lanes` per pair (1: one thread per pair; 8, 16, 32: a lane group
// per pair) and at most `warps` per block (0: as many as fit the class's largest pair state),
// and the per-pair scratch it needs.
int batch_shape(mcpd_ctx *ctx, mcpd_batch *b, int warps, int lanes = 1) {
    if (lanes != 1 && lanes != 8 && lanes != 16 && lanes != 32)
        return set_err(ctx, MCPD_EINVAL, "lanes per pair must be 1, 8, 16 or 32");
    if (lanes > 1 && !b->coupled) return set_err(ctx, MCPD_EINVAL, "lane groups run coupled batches only");
    for (size_t ci = 0; ci < b->cls.size(); ++ci) {
        BatchClass &c = b->cls[ci];
        int per_sm = 1, w = 0;
        if (lanes == 1) {
            mcpd::PairsShape shape;
            int rc = mcpd::pairs_shape(c.bp.coupled, c.bp.scan, c.bp.udeg, true, 0, c.bp.max_wpp, ctx->smem_optin, 0,
                                       ctx->sm_count, 0, c.bp.ext != 0, true, &shape);
            if (rc == MCPD_ETOO_LARGE) return set_err(ctx, rc, "largest instance does not fit one warp of pair state");
            if (rc != MCPD_OK) return set_err(ctx, rc, "cudaFuncSetAttribute / occupancy");
            if (warps > 0 && warps < shape.warps) {
                rc = mcpd::pairs_shape(c.bp.coupled, c.bp.scan, c.bp.udeg, true, 0, c.bp.max_wpp, ctx->smem_optin, 0,
                                       ctx->sm_count, warps, c.bp.ext != 0, true, &shape);
                if (rc != MCPD_OK) return set_err(ctx, rc, "launch shape");
            }
            w = shape.warps;
            c.smem = shape.smem;
            c.bp.y_regions = shape.y_regions;
            c.bp.wide = shape.wide ? 1 : 0;
            per_sm = shape.per_sm;
        } else {
            const size_t per_warp = static_cast<size_t>(32 / lanes) * 2 * c.bp.max_wpp * 4;
            const int cap = mcpd::group_max_threads(lanes) / 32;
            const int fit = static_cast<int>(std::min<size_t>(cap, ctx->smem_optin / per_warp));
            if (fit < 1) return set_err(ctx, MCPD_ETOO_LARGE, "largest instance does not fit one warp of pair state");
            w = warps > 0 ? std::min(warps, fit) : fit;
            c.smem = per_warp * w;
            c.bp.y_regions = 0;
            // a permission shared by the launches of all classes: the device's opt-in maximum
            if (mcpd::set_group_smem(lanes, ctx->smem_optin) != MCPD_OK) return set_err(ctx, MCPD_ECUDA, "cudaFuncSetAttribute");
            if (mcpd::group_occupancy(lanes, w * 32, c.smem, &per_sm) != MCPD_OK || per_sm < 1) per_sm = 1;
        }
        c.warps = w;
        c.block = w * 32;
        c.bp.lanes = lanes;
        // A class with fewer slots than one full launch holds pairs for launches only the blocks
        // its slots fill: a block keeps its shared memory until its last warp ends, so blocks
        // whose warps find no slot would hold SMs that the concurrently running classes need.
        const long long class_slots = ci < b->total_work0.size() ? b->total_work0[ci] : c.bp.total_work;
        const long long pairs_per_block = std::max(1, c.block / lanes);
        c.grid = static_cast<int>(std::max<long long>(
            1, std::min<long long>(static_cast<long long>(ctx->sm_count) * per_sm,
                                   (class_slots + pairs_per_block - 1) / pairs_per_block)));
        c.pairs = static_cast<long long>(c.grid) * c.block / lanes;
        if (c.pairs > c.scratch_pairs) {
            free_list(c.scratch);
            int rc;
            if ((rc = balloc(ctx, c.scratch, &c.bp.pair_scratch,
                             static_cast<size_t>(c.pairs) * mcpd::pair_words(c.bp.max_na, c.bp.max_W))) != MCPD_OK)
                return rc;
            if ((rc = balloc(ctx, c.scratch, &c.bp.y_state, static_cast<size_t>(c.pairs) * c.bp.max_wpp)) != MCPD_OK) return rc;
            c.scratch_pairs = c.pairs;
            b->dirty = true;
        }
    }
    b->lanes = lanes;
    if (b->graph_exec) { cudaGraphExecDestroy(b->graph_exec); b->graph_exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    return MCPD_OK;
}

// Put back the descriptors of a decode from each instance's first slot after an extension.
int restore_descriptors(mcpd_ctx *ctx, mcpd_batch *b) {
    if (!b->extended) return MCPD_OK;
    b->insts = b->insts0;
    for (size_t c = 0; c < b->cls.size(); ++c) b->cls[c].bp.total_work = b->total_work0[c];
    CU(cudaMemcpyAsync(b->d_insts, b->insts.data(), sizeof(mcpd::InstDesc) * b->insts.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    b->extended = false;
    return MCPD_OK;
}

int batch_enqueue(mcpd_ctx *ctx, mcpd_batch *b, double *est_dev, double *se_dev, bool always_clear,
                  bool accumulate = false) {
    const cudaStream_t s = ctx->stream;
    if (!accumulate) {
        CU(cudaMemsetAsync(b->d_buckets, 0, b->total_bucket_words * 3 * 8, s));
        CU(cudaMemsetAsync(b->d_bcount, 0, b->total_counts * 8, s));
    }
    CU(cudaMemsetAsync(b->d_counters, 0, b->cls.size() * mcpd::kNumCounters * 8, s));
    CU(cudaMemsetAsync(b->d_error, 0, sizeof(int), s));
    for (BatchClass &c : b->cls) {
        if (b->dirty || always_clear) {
            CU(cudaMemsetAsync(c.bp.pair_scratch, 0,
                               static_cast<size_t>(c.pairs) * mcpd::pair_words(c.bp.max_na, c.bp.max_W) * 8, s));
            CU(cudaMemsetAsync(c.bp.y_state, 0, static_cast<size_t>(c.pairs) * c.bp.max_wpp * 4, s));
        }
    }
    CU(cudaEventRecord(b->fork, s));
    for (size_t k = 0; k < b->cls.size(); ++k) {
        const BatchClass &c = b->cls[k];
        const cudaStream_t cs = b->cls_streams[k];
        CU(cudaStreamWaitEvent(cs, b->fork, 0));
        if (c.bp.total_work != 0) {                      // an extension may leave a class without work
            if ((c.bp.lanes == 1 ? mcpd::launch_batch(c.bp, c.grid, c.block, c.smem, cs)
                                 : mcpd::launch_group(c.bp, c.grid, c.block, c.smem, cs)) != MCPD_OK)
                return set_err(ctx, MCPD_ECUDA, std::string("batch kernel launch: ") + cudaGetErrorString(cudaGetLastError()));
        }
        CU(cudaEventRecord(b->cls_done[k], cs));
        CU(cudaStreamWaitEvent(s, b->cls_done[k], 0));
    }
    if (mcpd::launch_finalize_batch(b->d_insts, b->n_inst, b->d_clone_inst, b->d_clone_local,
                                    b->total_active, est_dev, se_dev, s) != MCPD_OK)
        return set_err(ctx, MCPD_ECUDA, "batch finalize launch");
    return MCPD_OK;
}

}  // namespace

extern "C" {

void mcpd_batch_destroy(mcpd_batch *b) {
    if (!b) return;
    if (b->device >= 0) cudaSetDevice(b->device);
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    free_list(b->allocs);
    for (BatchClass &c : b->cls) free_list(c.scratch);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    for (cudaStream_t cs : b->cls_streams) if (cs) cudaStreamDestroy(cs);
    for (cudaEvent_t e : b->cls_done) if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

int mcpd_batch_create(mcpd_ctx *ctx, int32_t n_inst, const mcpd_design *designs,
                      const uint8_t *const *ys, const mcpd_params *params, int32_t order_mode,
                      mcpd_batch **out) {
    NvtxRange nvtx_range("mcpd.batch_create");
    if (!ctx || !out || n_inst < 1 || !designs || !ys || !params) return MCPD_EINVAL;
    const int32_t mode = order_mode & 0xFF, want_classes = (order_mode >> 8) & 0xFF;
    if (mode > 1 || want_classes > 8 || (order_mode >> 16) != 0) return set_err(ctx, MCPD_EINVAL, "order_mode: order 0 or 1, classes 0..8");
    *out = nullptr;
    mcpd_batch *b = new (std::nothrow) mcpd_batch();
    if (!b) return set_err(ctx, MCPD_ENOMEM, "host allocation");
    b->device = ctx->device;
    b->n_inst = n_inst;
    b->t.resize(n_inst);
    for (int32_t i = 0; i < n_inst; ++i) {
        std::string err;
        const int rc = mcpd::build_tables(&designs[i], ys[i], &params[i], &b->t[i], &err);
        if (rc != MCPD_OK) { mcpd_batch_destroy(b); return set_err(ctx, rc, "instance " + std::to_string(i) + ": " + err); }
        if (b->t[i].coupled != b->t[0].coupled || (b->t[i].scan == MCPD_SCAN_SYSTEMATIC) != (b->t[0].scan == MCPD_SCAN_SYSTEMATIC)) {
            mcpd_batch_destroy(b);
            return set_err(ctx, MCPD_EINVAL, "all instances of a batch must share coupled and systematic settings");
        }
        if (b->t[i].record_slots || b->t[i].trace_stride) {
            mcpd_batch_destroy(b);
            return set_err(ctx, MCPD_EINVAL, "batches keep no per-slot records or traces");
        }
    }
    b->coupled = b->t[0].coupled;
    if (cudaSetDevice(ctx->device) != cudaSuccess) { mcpd_batch_destroy(b); return set_err(ctx, MCPD_ECUDA, "cudaSetDevice"); }

    std::vector<int32_t> cls_of;
    int n_cls = assign_classes(b->t, want_classes, ctx->sm_count, &cls_of);
    int64_t total_slots = 0;
    for (int32_t i = 0; i < n_inst; ++i) total_slots += b->t[i].P;
    // Launch order: class by class; within a class, 0 = input order, 1 = longest slots first.
    b->order.resize(n_inst);
    for (int32_t i = 0; i < n_inst; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int32_t a, int32_t c) {
        if (cls_of[a] != cls_of[c]) return cls_of[a] < cls_of[c];
        if (mode == 1) return std::max(b->t[a].B, b->t[a].unit) > std::max(b->t[c].B, b->t[c].unit);
        return false;
    });

    // Sizes.
    size_t table_bytes = 0;
    b->out_offset.assign(n_inst + 1, 0);
    b->bucket_offset.assign(n_inst, 0);
    b->count_offset.assign(n_inst, 0);
    auto up16 = [](size_t x) { return (x + 15) / 16 * 16; };
    for (int32_t i = 0; i < n_inst; ++i) {
        const mcpd::Tables &t = b->t[i];
        table_bytes += up16(t.alias.size() * 8) + up16(t.rows.size() * 2) + up16(t.T.size() * 8) + up16(t.Tnu.size() * 8) +
                       up16(t.init_pairs.size() * 4) + up16(t.rows_pool.size() * 2) + up16(t.rows_mask.size() * 2) +
                       up16(t.T_mask.size() * 8);
        b->out_offset[i + 1] = b->out_offset[i] + t.na;
        b->bucket_offset[i] = static_cast<int64_t>(b->total_bucket_words);
        b->total_bucket_words += static_cast<size_t>(t.nb) * t.na;
        b->count_offset[i] = static_cast<int64_t>(b->total_counts);
        b->total_counts += static_cast<size_t>(t.nb);
    }
    b->total_active = b->out_offset[n_inst];
    unsigned char *d_tables = nullptr;
    int rc;
#define BALLOC(ptr, n) do { if ((rc = balloc(ctx, b->allocs, &(ptr), (n))) != MCPD_OK) { mcpd_batch_destroy(b); return rc; } } while (0)
    BALLOC(d_tables, table_bytes);
    BALLOC(b->d_buckets, b->total_bucket_words * 3);
    BALLOC(b->d_bcount, b->total_counts);
    BALLOC(b->d_insts, static_cast<size_t>(n_inst));
    BALLOC(b->d_clone_inst, static_cast<size_t>(b->total_active));
    BALLOC(b->d_clone_local, static_cast<size_t>(b->total_active));
    BALLOC(b->d_counters, static_cast<size_t>(n_cls) * mcpd::kNumCounters);
    BALLOC(b->d_error, 1);
#undef BALLOC
    // Tables (host staging buffer, one copy) and descriptors in launch order; each class's work
    // items are numbered from 0.
    std::vector<unsigned char> host(table_bytes, 0);
    size_t off = 0;
    b->insts.resize(n_inst);
    b->cls.assign(n_cls, BatchClass());
    long long work = 0;
    for (int32_t pos = 0; pos < n_inst; ++pos) {
        const int32_t i = b->order[pos];
        const mcpd::Tables &t = b->t[i];
        BatchClass &c = b->cls[cls_of[i]];
        if (c.count == 0) { c.first = pos; work = 0; }
        ++c.count;
        mcpd::InstDesc &d = b->insts[pos];
        std::memset(&d, 0, sizeof(d));
        auto put = [&](const void *src, size_t bytes) -> const void * {
            if (bytes == 0) return nullptr;
            std::memcpy(host.data() + off, src, bytes);
            const void *dev = d_tables + off;
            off += up16(bytes);
            return dev;
        };
        d.alias = static_cast<const uint64_t *>(put(t.alias.data(), t.alias.size() * 8));
        d.rows = static_cast<const uint16_t *>(put(t.rows.data(), t.rows.size() * 2));
        d.T = static_cast<const uint64_t *>(put(t.T.data(), t.T.size() * 8));
        d.Tnu = static_cast<const uint64_t *>(put(t.Tnu.data(), t.Tnu.size() * 8));
        d.init_pairs = static_cast<const uint32_t *>(put(t.init_pairs.data(), t.init_pairs.size() * 4));
        d.n_init_pairs = static_cast<int32_t>(t.init_pairs.size());
        d.rows_pool = static_cast<const uint16_t *>(put(t.rows_pool.data(), t.rows_pool.size() * 2));
        d.rows_mask = static_cast<const uint16_t *>(put(t.rows_mask.data(), t.rows_mask.size() * 2));
        d.T_mask = static_cast<const uint64_t *>(put(t.T_mask.data(), t.T_mask.size() * 8));
        d.S1 = b->d_buckets + b->bucket_offset[i];
        d.S2lo = b->d_buckets + b->total_bucket_words + b->bucket_offset[i];
        d.S2hi = b->d_buckets + 2 * b->total_bucket_words + b->bucket_offset[i];
        d.bcount = b->d_bcount + b->count_offset[i];
        d.na = t.na; d.W = t.W; d.wpp = t.wpp; d.deg = t.deg_max; d.nb = static_cast<int32_t>(t.nb);
        d.dummy_word_index = t.dummy_word_index; d.dummy_entry = t.dummy_entry; d.dummy_word = t.dummy_word;
        d.P = t.P; d.B = t.B; d.k = t.k; d.ell = t.ell; d.L = t.L; d.burn = t.burn; d.length = t.length;
        d.unit = t.unit; d.step_limit = t.step_limit; d.slot_offset = t.slot_offset; d.tau_audit = t.tau_audit;
        d.capped = t.capped ? 1 : 0;
        d.lag = static_cast<int32_t>(t.lag);
        d.work_begin = work; work += t.P;
        d.P_total = t.P;
        d.seed = t.seed; d.instance = t.instance;
        mcpd::BParams &bp = c.bp;
        bp.total_work = work;
        if (t.capped || t.lag > 1) bp.ext = 1;
        if (!t.Tnu.empty()) bp.any_init = 1;
        // the class's uniform degree: the first instance's, kept while every instance shares it
        if (d.work_begin == 0) bp.udeg = t.udeg;
        else if (bp.udeg != t.udeg) bp.udeg = 0;
        bp.max_na = std::max(bp.max_na, t.na); bp.max_W = std::max(bp.max_W, t.W);
        bp.max_wpp = std::max(bp.max_wpp, t.wpp); bp.max_m = std::max(bp.max_m, t.m);
    }
    b->total_slots = total_slots;
    for (int c = 0; c < n_cls; ++c) {
        mcpd::BParams &bp = b->cls[c].bp;
        bp.insts = b->d_insts + b->cls[c].first;
        bp.n_inst = b->cls[c].count;
        bp.coupled = b->coupled ? 1 : 0;
        bp.scan = b->t[0].scan;
        bp.lanes = 1;
        bp.counters = b->d_counters + static_cast<size_t>(c) * mcpd::kNumCounters;
        bp.error = b->d_error;
    }
    std::vector<int32_t> ci(b->total_active), cl(b->total_active);
    for (int32_t pos = 0; pos < n_inst; ++pos) {
        const int32_t i = b->order[pos];
        for (int32_t a = 0; a < b->t[i].na; ++a) { ci[b->out_offset[i] + a] = pos; cl[b->out_offset[i] + a] = a; }
    }
    CU_OR(cudaMemcpyAsync(d_tables, host.data(), table_bytes, cudaMemcpyHostToDevice, ctx->stream), mcpd_batch_destroy(b));
    CU_OR(cudaMemcpyAsync(b->d_insts, b->insts.data(), sizeof(mcpd::InstDesc) * n_inst, cudaMemcpyHostToDevice, ctx->stream), mcpd_batch_destroy(b));
    b->insts0 = b->insts;
    for (const BatchClass &c : b->cls) b->total_work0.push_back(c.bp.total_work);
    CU_OR(cudaMemcpyAsync(b->d_clone_inst, ci.data(), ci.size() * 4, cudaMemcpyHostToDevice, ctx->stream), mcpd_batch_destroy(b));
    CU_OR(cudaMemcpyAsync(b->d_clone_local, cl.data(), cl.size() * 4, cudaMemcpyHostToDevice, ctx->stream), mcpd_batch_destroy(b));
    if ((rc = batch_shape(ctx, b, 0)) != MCPD_OK) { mcpd_batch_destroy(b); return rc; }
    b->cls_streams.assign(b->cls.size(), nullptr);
    b->cls_done.assign(b->cls.size(), nullptr);
    for (size_t k = 0; k < b->cls.size(); ++k) {
        CU_OR(cudaStreamCreateWithFlags(&b->cls_streams[k], cudaStreamNonBlocking), mcpd_batch_destroy(b));
        CU_OR(cudaEventCreateWithFlags(&b->cls_done[k], cudaEventDisableTiming), mcpd_batch_destroy(b));
    }
    CU_OR(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), mcpd_batch_destroy(b));
    CU_OR(cudaEventCreate(&b->ev0), mcpd_batch_destroy(b));
    CU_OR(cudaEventCreate(&b->ev1), mcpd_batch_destroy(b));
    CU_OR(cudaStreamSynchronize(ctx->stream), mcpd_batch_destroy(b));
    *out = b;
    return MCPD_OK;
}

int mcpd_batch_info(const mcpd_batch *b, int64_t info[16]) {
    if (!b || !info) return MCPD_EINVAL;
    std::memset(info, 0, 16 * sizeof(int64_t));
    int32_t max_na = 0;
    int64_t pairs = 0, wmax = 0, ext = 0, degree_builds = 0;
    for (const BatchClass &c : b->cls) {
        max_na = std::max(max_na, c.bp.max_na);
        pairs = std::max<int64_t>(pairs, c.pairs);
        wmax = std::max<int64_t>(wmax, c.warps);
        ext += c.bp.ext;
        if (b->lanes == 1 && mcpd::batch_kernel_degree(c.bp.coupled, c.bp.ext, c.bp.udeg) > 0) ++degree_builds;
    }
    const BatchClass &c0 = b->cls[0];
    info[0] = b->total_active; info[1] = b->n_inst; info[2] = b->total_slots; info[3] = max_na;
    info[4] = c0.warps; info[5] = c0.grid; info[6] = pairs; info[7] = static_cast<int64_t>(c0.smem);
    info[8] = b->lanes; info[9] = static_cast<int64_t>(b->cls.size()); info[10] = wmax; info[11] = ext;
    info[12] = degree_builds;
    return MCPD_OK;
}

int mcpd_batch_offsets(const mcpd_batch *b, int64_t *offsets) {
    if (!b || !offsets) return MCPD_EINVAL;
    std::memcpy(offsets, b->out_offset.data(), b->out_offset.size() * sizeof(int64_t));
    return MCPD_OK;
}

int mcpd_batch_set_shape(mcpd_ctx *ctx, mcpd_batch *b, int32_t lanes_per_pair, int32_t warps_per_block) {
    if (!ctx || !b) return MCPD_EINVAL;
    CU(cudaSetDevice(ctx->device));
    return batch_shape(ctx, b, warps_per_block, lanes_per_pair);
}

int mcpd_batch_run_async(mcpd_ctx *ctx, mcpd_batch *b, double *est_dev, double *se_dev) {
    NvtxRange nvtx_range("mcpd.batch_run");
    if (!ctx || !b || !est_dev || !se_dev) return MCPD_EINVAL;
    CU(cudaSetDevice(ctx->device));
    int rc = restore_descriptors(ctx, b);
    if (rc != MCPD_OK) return rc;
    CU(cudaEventRecord(b->ev0, ctx->stream));
    rc = batch_enqueue(ctx, b, est_dev, se_dev, false);
    if (rc != MCPD_OK) return rc;
    CU(cudaEventRecord(b->ev1, ctx->stream));
    b->dirty = true;
    b->ran = true;
    return MCPD_OK;
}

int mcpd_batch_extend_async(mcpd_ctx *ctx, mcpd_batch *b, const int32_t *mask, double *est_dev, double *se_dev) {
    NvtxRange nvtx_range("mcpd.batch_extend");
    if (!ctx || !b || !est_dev || !se_dev) return MCPD_EINVAL;
    if (!b->ran) return set_err(ctx, MCPD_EINVAL, "nothing to extend: run the batch first");
    CU(cudaSetDevice(ctx->device));
    // Each chosen instance runs its next P_i slots (the next global ids after those in its
    // buckets); the others run none.  Work items are renumbered per class.
    size_t pos = 0;
    for (BatchClass &c : b->cls) {
        long long work = 0;
        for (int32_t k = 0; k < c.count; ++k, ++pos) {
            mcpd::InstDesc &d = b->insts[pos];
            const mcpd::Tables &t = b->t[b->order[pos]];
            const bool go = !mask || mask[b->order[pos]] != 0;
            if (go && (d.P_total + t.P > (int64_t(1) << 31) || t.slot_offset + d.P_total + t.P > (int64_t(1) << 32)))
                return set_err(ctx, MCPD_EINVAL, "extension beyond 2^31 slots or 32-bit global slot ids");
            d.work_begin = work;
            d.P = go ? t.P : 0;
            if (go) {
                d.slot_offset = t.slot_offset + d.P_total;
                d.P_total += t.P;
                work += t.P;
            }
        }
        c.bp.total_work = work;
    }
    b->extended = true;
    CU(cudaMemcpyAsync(b->d_insts, b->insts.data(), sizeof(mcpd::InstDesc) * b->insts.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaEventRecord(b->ev0, ctx->stream));
    const int rc = batch_enqueue(ctx, b, est_dev, se_dev, false, true);
    if (rc != MCPD_OK) return rc;
    CU(cudaEventRecord(b->ev1, ctx->stream));
    b->dirty = true;
    return MCPD_OK;
}

int mcpd_batch_capture_graph(mcpd_ctx *ctx, mcpd_batch *b, double *est_dev, double *se_dev) {
    NvtxRange nvtx_range("mcpd.batch_capture_graph");
    if (!ctx || !b || !est_dev || !se_dev) return MCPD_EINVAL;
    CU(cudaSetDevice(ctx->device));
    if (!ctx->stream) return set_err(ctx, MCPD_EINVAL, "graph capture needs a non-default stream");
    {
        const int r = restore_descriptors(ctx, b);
        if (r != MCPD_OK) return r;
    }
    if (b->graph_exec) { cudaGraphExecDestroy(b->graph_exec); b->graph_exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = batch_enqueue(ctx, b, est_dev, se_dev, true);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (rc != MCPD_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return set_err(ctx, MCPD_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    b->graph = g;
    CU(cudaGraphInstantiate(&b->graph_exec, g, 0));
    return MCPD_OK;
}

int mcpd_batch_launch_graph(mcpd_ctx *ctx, mcpd_batch *b) {
    NvtxRange nvtx_range("mcpd.batch_launch_graph");
    if (!ctx || !b || !b->graph_exec) return MCPD_EINVAL;
    CU(cudaSetDevice(ctx->device));
    {
        const int r = restore_descriptors(ctx, b);
        if (r != MCPD_OK) return r;
    }
    CU(cudaEventRecord(b->ev0, ctx->stream));
    CU(cudaGraphLaunch(b->graph_exec, ctx->stream));
    CU(cudaEventRecord(b->ev1, ctx->stream));
    b->dirty = true;
    b->ran = true;
    return MCPD_OK;
}

int mcpd_batch_collect(mcpd_ctx *ctx, mcpd_batch *b, mcpd_stats *stats) {
    NvtxRange nvtx_range("mcpd.batch_collect");
    if (!ctx || !b) return MCPD_EINVAL;
    if (!b->ran) return set_err(ctx, MCPD_EINVAL, "no run to collect");
    CU(cudaSetDevice(ctx->device));
    std::vector<unsigned long long> cc(b->cls.size() * mcpd::kNumCounters);
    int error = 0;
    CU(cudaMemcpyAsync(cc.data(), b->d_counters, cc.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(&error, b->d_error, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    unsigned long long c[mcpd::kNumCounters] = {};
    for (size_t k = 0; k < b->cls.size(); ++k)
        for (int i = 0; i < mcpd::kNumCounters; ++i) {
            const unsigned long long v = cc[k * mcpd::kNumCounters + i];
            c[i] = i == mcpd::kMaxTau ? std::max(c[i], v) : c[i] + v;
        }
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        mcpd::counters_to_stats(c, stats);
        stats->n_buckets = static_cast<int64_t>(b->total_counts);
        stats->n_active = b->total_active;
        stats->kernel_ms = ms;
        for (const BatchClass &cl : b->cls) stats->resident_pairs = std::max<int64_t>(stats->resident_pairs, cl.pairs);
    }
    if (error) return set_err(ctx, MCPD_ESTEP_LIMIT, "a pair reached the step limit without meeting");
    b->dirty = false;
    return MCPD_OK;
}

int mcpd_batch_fetch(mcpd_ctx *ctx, const mcpd_batch *b, int32_t inst, int what, void *host_dst,
                     size_t bytes) {
    if (!ctx || !b || !host_dst || inst < 0 || inst >= b->n_inst) return MCPD_EINVAL;
    const mcpd::Tables &t = b->t[inst];
    const size_t words = static_cast<size_t>(t.nb) * t.na;
    const unsigned long long *src = nullptr;
    size_t need = words * 8;
    switch (what) {
        case MCPD_FETCH_S1: src = b->d_buckets + b->bucket_offset[inst]; break;
        case MCPD_FETCH_S2_LO: src = b->d_buckets + b->total_bucket_words + b->bucket_offset[inst]; break;
        case MCPD_FETCH_S2_HI: src = b->d_buckets + 2 * b->total_bucket_words + b->bucket_offset[inst]; break;
        case MCPD_FETCH_COUNT: src = b->d_bcount + b->count_offset[inst]; need = static_cast<size_t>(t.nb) * 8; break;
        default: return set_err(ctx, MCPD_EINVAL, "batch fetch: buckets and counts only");
    }
    if (bytes != need) return set_err(ctx, MCPD_EINVAL, "batch fetch: wrong size");
    CU(cudaSetDevice(ctx->device));
    CU(cudaMemcpyAsync(host_dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return MCPD_OK;
}

// Time each candidate launch shape (lanes per pair, warps per block) on the batch itself (reps
// timed decodes after one warm-up each) and keep the fastest; times[c] receives the mean
// milliseconds of candidate c (-1 if it does not fit).
int mcpd_batch_autotune(mcpd_ctx *ctx, mcpd_batch *b, const int32_t *cand_lanes,
                        const int32_t *cand_warps, int32_t n_cand, int32_t reps, double *est_dev,
                        double *se_dev, int32_t *best_index, double *times) {
    NvtxRange nvtx_range("mcpd.batch_autotune");
    if (!ctx || !b || !cand_lanes || !cand_warps || n_cand < 1 || reps < 1 || !est_dev || !se_dev) return MCPD_EINVAL;
    CU(cudaSetDevice(ctx->device));
    double best = 1e300;
    int32_t best_c = -1;
    for (int32_t c = 0; c < n_cand; ++c) {
        int rc = batch_shape(ctx, b, cand_warps[c], cand_lanes[c]);
        if (rc != MCPD_OK) { if (times) times[c] = -1.0; ctx->err.clear(); continue; }
        double total = 0.0;
        for (int32_t r = 0; r <= reps; ++r) {
            if ((rc = mcpd_batch_run_async(ctx, b, est_dev, se_dev)) != MCPD_OK) return rc;
            mcpd_stats st;
            rc = mcpd_batch_collect(ctx, b, &st);         // a step-limit stop still times the shape
            if (rc != MCPD_OK && rc != MCPD_ESTEP_LIMIT) return rc;
            if (r > 0) total += st.kernel_ms;
        }
        const double mean = total / reps;
        if (times) times[c] = mean;
        if (mean < best) { best = mean; best_c = c; }
    }
    if (best_c < 0) return set_err(ctx, MCPD_EINVAL, "no candidate shape fits");
    if (best_index) *best_index = best_c;
    return batch_shape(ctx, b, cand_warps[best_c], cand_lanes[best_c]);
}

}  // extern "C"
