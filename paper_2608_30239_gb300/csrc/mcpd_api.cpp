// C ABI of the library (declared in include/mcpd.h): contexts, plans, runs, result transfer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mcpd_internal.h"

namespace mcpd {
int pairs_occupancy(int coupled, int scan, int block, size_t smem, int *blocks_per_sm);
}

struct mcpd_plan {
    mcpd_ctx *ctx = nullptr;
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
};

namespace {

int set_err(mcpd_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return set_err(ctx, e_ == cudaErrorMemoryAllocation ? MCPD_ENOMEM : MCPD_ECUDA,   \
                           std::string(#call) + ": " + cudaGetErrorString(e_));               \
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
    if (pl->ctx) cudaSetDevice(pl->ctx->device);
    for (void *p : pl->allocs) cudaFree(p);
    if (pl->ev0) cudaEventDestroy(pl->ev0);
    if (pl->ev1) cudaEventDestroy(pl->ev1);
    delete pl;
}

int mcpd_plan_create(mcpd_ctx *ctx, const mcpd_design *design, const uint8_t *y,
                     const mcpd_params *params, mcpd_plan **out) {
    if (!ctx || !out) return MCPD_EINVAL;
    *out = nullptr;
    mcpd_plan *pl = new (std::nothrow) mcpd_plan();
    if (!pl) return set_err(ctx, MCPD_ENOMEM, "host allocation");
    pl->ctx = ctx;
    std::string err;
    int rc = mcpd::build_tables(design, y, params, &pl->t, &err);
    if (rc != MCPD_OK) { delete pl; return set_err(ctx, rc, err); }
    const mcpd::Tables &t = pl->t;
    if (cudaSetDevice(ctx->device) != cudaSuccess) { delete pl; return set_err(ctx, MCPD_ECUDA, "cudaSetDevice"); }

    // Launch shape: tables first in shared memory, then one 32-lane region per warp.
    const size_t tables = ((static_cast<size_t>(t.na) * 24 + mcpd::kTSide * mcpd::kTSide * 8) + 15) / 16 * 16;
    const size_t per_warp = static_cast<size_t>(t.wpp) * 128;
    if (tables + per_warp > ctx->smem_optin) {
        delete pl;
        return set_err(ctx, MCPD_ETOO_LARGE, "instance too large for the one-thread-per-pair layout");
    }
    int warps = static_cast<int>(std::min<size_t>(16, (ctx->smem_optin - tables) / per_warp));
    // Prefer several blocks per SM when the pair state is small: cap a block at what half of the
    // shared memory holds, so two blocks fit, when that still leaves 8 warps per block.
    const size_t half = ctx->smem_optin / 2;
    if (half > tables && (half - tables) / per_warp >= 8)
        warps = static_cast<int>(std::min<size_t>(warps, (half - tables) / per_warp));
    pl->block = warps * 32;
    pl->smem = tables + per_warp * warps;
    if (mcpd::set_pairs_smem(pl->smem, t.coupled) != MCPD_OK) {
        delete pl;
        return set_err(ctx, MCPD_ECUDA, "cudaFuncSetAttribute(max dynamic shared memory)");
    }
    int per_sm = 1;
    if (mcpd::pairs_occupancy(t.coupled, t.scan, pl->block, pl->smem, &per_sm) != MCPD_OK || per_sm < 1) per_sm = 1;
    pl->grid = ctx->sm_count * per_sm;
    pl->pairs = static_cast<long long>(pl->grid) * pl->block;

    mcpd::KParams &kp = pl->kp;
    uint64_t *d_alias = nullptr, *d_T = nullptr, *d_Tnu = nullptr;
    uint16_t *d_rows = nullptr;
#define ALLOC(ptr, n)                                                        \
    do {                                                                     \
        int r_ = dev_alloc(ctx, pl, &(ptr), (n));                            \
        if (r_ != MCPD_OK) { mcpd_plan_destroy(pl); return r_; }             \
    } while (0)
    ALLOC(d_alias, t.alias.size());
    ALLOC(d_rows, t.rows.size());
    ALLOC(d_T, t.T.size());
    ALLOC(d_Tnu, t.Tnu.size());
    ALLOC(kp.rep_acc, static_cast<size_t>(pl->pairs) * t.na);
    ALLOC(kp.slot_acc, static_cast<size_t>(pl->pairs) * t.na);
    ALLOC(kp.touched_rep, static_cast<size_t>(pl->pairs) * t.W);
    ALLOC(kp.touched_slot, static_cast<size_t>(pl->pairs) * t.W);
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
    }
#undef ALLOC
    CU(cudaMemcpyAsync(d_alias, t.alias.data(), t.alias.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(d_rows, t.rows.data(), t.rows.size() * 2, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(d_T, t.T.data(), t.T.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    if (!t.Tnu.empty())
        CU(cudaMemcpyAsync(d_Tnu, t.Tnu.data(), t.Tnu.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    kp.alias = d_alias; kp.rows = d_rows; kp.T = d_T; kp.Tnu = t.Tnu.empty() ? nullptr : d_Tnu;
    kp.na = t.na; kp.m = t.m; kp.W = t.W; kp.Mp = t.Mp; kp.wpp = t.wpp; kp.deg = t.deg_max;
    kp.nb = static_cast<int32_t>(t.nb); kp.scan = t.scan;
    kp.dummy_entry = t.dummy_entry; kp.dummy_word = t.dummy_word;
    kp.dummy_word_index = t.dummy_word_index; kp.coupled = t.coupled ? 1 : 0;
    kp.P = t.P; kp.B = t.B; kp.k = t.k; kp.ell = t.ell; kp.L = t.L; kp.burn = t.burn;
    kp.length = t.length; kp.unit = t.unit; kp.step_limit = t.step_limit;
    kp.slot_offset = t.slot_offset; kp.trace_stride = t.trace_stride;
    kp.seed = t.seed; kp.instance = t.instance; kp.warps = warps;
    kp.smem_tables = static_cast<uint32_t>(tables);
    CU(cudaEventCreate(&pl->ev0));
    CU(cudaEventCreate(&pl->ev1));
    CU(cudaStreamSynchronize(ctx->stream));
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

int mcpd_run_async(mcpd_ctx *ctx, mcpd_plan *pl, double *est_dev, double *se_dev) {
    if (!ctx || !pl || !est_dev || !se_dev) return MCPD_EINVAL;
    CU(cudaSetDevice(ctx->device));
    const mcpd::Tables &t = pl->t;
    mcpd::KParams &kp = pl->kp;
    const size_t nbna = static_cast<size_t>(t.nb) * t.na;
    CU(cudaMemsetAsync(kp.S1, 0, nbna * 8, ctx->stream));
    CU(cudaMemsetAsync(kp.S2lo, 0, nbna * 8, ctx->stream));
    CU(cudaMemsetAsync(kp.S2hi, 0, nbna * 8, ctx->stream));
    CU(cudaMemsetAsync(kp.bcount, 0, static_cast<size_t>(t.nb) * 8, ctx->stream));
    CU(cudaMemsetAsync(kp.counters, 0, mcpd::kNumCounters * 8, ctx->stream));
    CU(cudaMemsetAsync(kp.error, 0, sizeof(int), ctx->stream));
    if (pl->dirty) {   // the kernel leaves these zeroed when it completes normally
        const size_t pn = static_cast<size_t>(pl->pairs) * t.na;
        CU(cudaMemsetAsync(kp.rep_acc, 0, pn * 8, ctx->stream));
        CU(cudaMemsetAsync(kp.slot_acc, 0, pn * 8, ctx->stream));
        CU(cudaMemsetAsync(kp.touched_rep, 0, static_cast<size_t>(pl->pairs) * t.W * 4, ctx->stream));
        CU(cudaMemsetAsync(kp.touched_slot, 0, static_cast<size_t>(pl->pairs) * t.W * 4, ctx->stream));
    }
    if (kp.trace_G) CU(cudaMemsetAsync(kp.trace_G, 0, static_cast<size_t>(pl->n_trace) * t.na * 8, ctx->stream));
    if (kp.slot_nstar) {
        CU(cudaMemsetAsync(kp.slot_nstar, 0, static_cast<size_t>(t.P) * 4, ctx->stream));
        CU(cudaMemsetAsync(kp.slot_S, 0, static_cast<size_t>(t.P) * 8, ctx->stream));
        CU(cudaMemsetAsync(kp.slot_reps, 0, static_cast<size_t>(t.P) * 4, ctx->stream));
    }
    pl->dirty = true;
    CU(cudaEventRecord(pl->ev0, ctx->stream));
    if (mcpd::launch_pairs(kp, pl->grid, pl->block, pl->smem, ctx->stream) != MCPD_OK)
        return set_err(ctx, MCPD_ECUDA, std::string("pairs kernel launch: ") + cudaGetErrorString(cudaGetLastError()));
    CU(cudaEventRecord(pl->ev1, ctx->stream));
    if (mcpd::launch_finalize(kp.S1, kp.S2lo, kp.S2hi, t.na, static_cast<int>(t.nb), t.P, t.L, est_dev,
                              se_dev, ctx->stream) != MCPD_OK)
        return set_err(ctx, MCPD_ECUDA, "finalize kernel launch");
    pl->ran = true;
    return MCPD_OK;
}

int mcpd_collect(mcpd_ctx *ctx, mcpd_plan *pl, mcpd_stats *stats) {
    if (!ctx || !pl) return MCPD_EINVAL;
    if (!pl->ran) return set_err(ctx, MCPD_EINVAL, "no run to collect");
    CU(cudaSetDevice(ctx->device));
    unsigned long long c[mcpd::kNumCounters];
    int error = 0;
    CU(cudaMemcpyAsync(c, pl->kp.counters, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(&error, pl->kp.error, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, pl->ev0, pl->ev1));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->progress_units = static_cast<int64_t>(c[mcpd::kProgress]);
        stats->reps_started = static_cast<int64_t>(c[mcpd::kRepsStarted]);
        stats->reps_retained = static_cast<int64_t>(c[mcpd::kRepsRetained]);
        stats->reps_aborted = static_cast<int64_t>(c[mcpd::kRepsAborted]);
        stats->zero_completion_slots = static_cast<int64_t>(c[mcpd::kZeroCompletion]);
        stats->step_limit_hits = static_cast<int64_t>(c[mcpd::kStepLimitHits]);
        stats->max_tau = static_cast<int64_t>(c[mcpd::kMaxTau]);
        stats->sum_tau = static_cast<int64_t>(c[mcpd::kSumTau]);
        stats->site_updates = pl->t.coupled ? 2 * stats->progress_units - stats->reps_started
                                            : stats->progress_units;
        stats->n_buckets = pl->t.nb;
        stats->n_active = pl->t.na;
        stats->kernel_ms = ms;
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
    }
    CU(cudaSetDevice(ctx->device));
    CU(cudaMemcpyAsync(host_dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return MCPD_OK;
}

int mcpd_decode(mcpd_ctx *ctx, const mcpd_design *design, const uint8_t *y,
                const mcpd_params *params, double *est, double *se, int32_t *active,
                mcpd_stats *stats) {
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
