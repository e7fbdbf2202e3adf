// mcpd_decode_noalloc: the coupled decode without any device allocation.
//
// Who needs this: a caller whose device memory is owned by someone else and who therefore may not
// call cudaMalloc / cudaFree itself, for example a plug-in inside an application or server that
// gives every component a fixed memory budget up front through its own pool allocator, or a
// latency-sensitive host loop that cannot afford the device-wide synchronisation cudaMalloc and
// cudaFree can imply.  Such a caller passes the host inputs and two device output arrays it
// already owns; everything else the sampling kernel needs (the staged tables, the per-pair
// accumulators, the N*_p buckets and the counters) lives in one file-scope device array that is
// part of the library image.
//
// Limits and sharing:
//   - The array holds kNoAllocScratchBytes (64 MiB) on every GPU that loads this library, until
//     the process exits.  A problem whose tables plus buckets plus one warp of pair accumulators do
//     not fit is rejected with MCPD_ETOO_LARGE; a problem that fits runs with as many resident
//     pairs as fit (fewer than the allocating path may use, same results).
//   - Every call uses the same array and leaves its contents behind; each call clears what must
//     start at zero.  Two calls whose work overlaps on the GPU (other streams, other host threads,
//     on the same device) race on the array: serialise them.
//   - Every call looks the array's device address up with cudaGetSymbolAddress, with the context's
//     device current, so the address is never stale (a primary-context reset gives the array a new
//     one).  The first lookup on a device may load the library's device code: make the first call
//     before any stream capture.
//   - The output arrays must be device (or managed) memory of the context's device, in the CUDA
//     primary context the runtime uses; the call checks their device before any launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "mcpd_internal.h"

namespace mcpd {

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array on `device`, which the caller has made current.  Looked up on every
// call (it costs a table lookup in the runtime): a cached address would outlive a reset of the
// primary context.
int scratch_address(int device, void **out, std::string *err) {
    if (device < 0 || device >= kMaxDevices) { *err = "device index out of range"; return MCPD_EINVAL; }
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
        *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return MCPD_ECUDA;
    }
    *out = ptr;
    return MCPD_OK;
}

// The caller's output array lives on `device` (device or managed memory).
bool on_device(const void *ptr, int device) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return false;
    return a.device == device;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace mcpd

namespace {
int fail(mcpd_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}
}  // namespace

#define CUN(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return fail(ctx, MCPD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" int mcpd_decode_noalloc(mcpd_ctx *ctx, const mcpd_design *design, const uint8_t *y,
                                   const mcpd_params *params, double *est_dev, double *se_dev,
                                   mcpd_stats *stats) {
    using namespace mcpd;
    if (!ctx || !est_dev || !se_dev) return MCPD_EINVAL;
    Tables t;
    std::string err;
    int rc = build_tables(design, y, params, &t, &err);
    if (rc != MCPD_OK) return fail(ctx, rc, err);
    if (t.record_slots || t.trace_stride > 0)
        return fail(ctx, MCPD_EINVAL, "no-alloc decode keeps no per-slot records or traces");
    CUN(cudaSetDevice(ctx->device));
    if (!on_device(est_dev, ctx->device) || !on_device(se_dev, ctx->device))
        return fail(ctx, MCPD_EINVAL, "est_dev and se_dev must be device memory of the context's device");
    void *base = nullptr;
    rc = scratch_address(ctx->device, &base, &err);
    if (rc != MCPD_OK) return fail(ctx, rc, err);

    // Fixed part of the layout: tables, buckets, counters.
    const size_t na = static_cast<size_t>(t.na), nb = static_cast<size_t>(t.nb);
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off += up256(bytes); return at; };
    const size_t o_alias = take(na * 8), o_rows = take(na * 16), o_T = take(kernel_T(t).size() * 8);
    const size_t o_Tnu = take(t.Tnu.size() * 8), o_init = take(t.init_pairs.size() * 4);
    const size_t o_S1 = take(nb * na * 8), o_S2lo = take(nb * na * 8), o_S2hi = take(nb * na * 8);
    const size_t o_bc = take(nb * 8), o_cnt = take(kNumCounters * 8), o_err = take(sizeof(int));
    const size_t fixed = off;

    // Launch shape as the allocating path would choose it, then as many whole warps as fit.
    const size_t tables = kernel_table_bytes(t);
    PairsShape shape;
    const int src = pairs_shape(t.coupled, t.scan, t.udeg, false, tables, t.wpp, ctx->smem_optin, t.P,
                                ctx->sm_count, 0, t.capped || t.lag > 1, !t.Tnu.empty(), &shape);
    if (src == MCPD_ETOO_LARGE) return fail(ctx, src, "instance too large for the one-thread-per-pair layout");
    if (src != MCPD_OK) return fail(ctx, MCPD_ECUDA, "launch shape (cudaFuncSetAttribute / occupancy)");
    // scratch block (sums, statistics, touched sets) and Y column
    const size_t per_pair = static_cast<size_t>(pair_words(t.na, t.W)) * 8 + static_cast<size_t>(t.wpp) * 4;
    // room for the pair scratch and the Y columns, each rounded up to 256 bytes
    if (fixed + 2 * 256 > kNoAllocScratchBytes)
        return fail(ctx, MCPD_ETOO_LARGE, "tables and N*_p buckets exceed the 64 MiB no-alloc scratch");
    const size_t fit_warps = (kNoAllocScratchBytes - fixed - 2 * 256) / (32 * per_pair);
    if (fit_warps < 1)
        return fail(ctx, MCPD_ETOO_LARGE, "not even one warp of pair accumulators fits the 64 MiB no-alloc scratch");
    const int warps = static_cast<int>(std::min<size_t>(shape.warps, fit_warps));
    const int y_regions = pairs_y_regions(t.coupled, warps);
    const size_t smem = pairs_smem_bytes(tables, t.wpp, warps, y_regions);
    const int grid = static_cast<int>(std::min<size_t>(static_cast<size_t>(ctx->sm_count) * shape.per_sm, fit_warps / warps));
    const size_t pairs = static_cast<size_t>(grid) * warps * 32;
    const size_t o_pair = take(pairs * static_cast<size_t>(pair_words(t.na, t.W)) * 8);
    const size_t o_y = take(pairs * t.wpp * 4);
    if (off > kNoAllocScratchBytes) return fail(ctx, MCPD_ETOO_LARGE, "no-alloc scratch layout overflow");

    unsigned char *b = static_cast<unsigned char *>(base);
    cudaStream_t s = ctx->stream;
    CUN(cudaMemsetAsync(b, 0, off, s));     // the array keeps the previous call's contents
    CUN(cudaMemcpyAsync(b + o_alias, t.alias.data(), na * 8, cudaMemcpyHostToDevice, s));
    CUN(cudaMemcpyAsync(b + o_rows, kernel_rows(t).data(), kernel_rows(t).size() * 2, cudaMemcpyHostToDevice, s));
    CUN(cudaMemcpyAsync(b + o_T, kernel_T(t).data(), kernel_T(t).size() * 8, cudaMemcpyHostToDevice, s));
    if (!t.Tnu.empty()) CUN(cudaMemcpyAsync(b + o_Tnu, t.Tnu.data(), t.Tnu.size() * 8, cudaMemcpyHostToDevice, s));
    if (!t.init_pairs.empty())
        CUN(cudaMemcpyAsync(b + o_init, t.init_pairs.data(), t.init_pairs.size() * 4, cudaMemcpyHostToDevice, s));

    KParams kp{};
    kp.alias = reinterpret_cast<const uint64_t *>(b + o_alias);
    kp.rows = reinterpret_cast<const uint16_t *>(b + o_rows);
    kp.T = reinterpret_cast<const uint64_t *>(b + o_T);
    kp.Tnu = t.Tnu.empty() ? nullptr : reinterpret_cast<const uint64_t *>(b + o_Tnu);
    kp.init_pairs = reinterpret_cast<const uint32_t *>(b + o_init);
    kp.n_init_pairs = static_cast<int32_t>(t.init_pairs.size());
    kp.pair_scratch = reinterpret_cast<long long *>(b + o_pair);
    kp.y_state = reinterpret_cast<uint32_t *>(b + o_y);
    kp.S1 = reinterpret_cast<unsigned long long *>(b + o_S1);
    kp.S2lo = reinterpret_cast<unsigned long long *>(b + o_S2lo);
    kp.S2hi = reinterpret_cast<unsigned long long *>(b + o_S2hi);
    kp.bcount = reinterpret_cast<unsigned long long *>(b + o_bc);
    kp.counters = reinterpret_cast<unsigned long long *>(b + o_cnt);
    kp.error = reinterpret_cast<int *>(b + o_err);
    kp.na = t.na; kp.m = t.m; kp.W = t.W; kp.Mp = t.Mp; kp.wpp = t.wpp; kp.deg = t.deg_max; kp.udeg = t.udeg;
    kp.nb = static_cast<int32_t>(t.nb); kp.scan = t.scan;
    kp.dummy_entry = t.dummy_entry; kp.dummy_word = t.dummy_word;
    kp.dummy_word_index = t.dummy_word_index; kp.coupled = t.coupled ? 1 : 0;
    kp.P = t.P; kp.B = t.B; kp.k = t.k; kp.ell = t.ell; kp.L = t.L; kp.burn = t.burn;
    kp.length = t.length; kp.unit = t.unit; kp.step_limit = t.step_limit; kp.tau_audit = t.tau_audit;
    kp.capped = t.capped ? 1 : 0;
    kp.lag = static_cast<int32_t>(t.lag);
    kp.slot_offset = t.slot_offset; kp.trace_stride = 0;
    kp.seed = t.seed; philox_round_keys(t.seed, kp.rk); kp.instance = t.instance; kp.warps = warps;
    kp.smem_tables = static_cast<uint32_t>(tables);
    kp.nT = static_cast<int32_t>(kernel_T(t).size());
    kp.y_regions = y_regions;
    if (launch_pairs(kp, grid, warps * 32, smem, s) != MCPD_OK)
        return fail(ctx, MCPD_ECUDA, std::string("pairs kernel launch: ") + cudaGetErrorString(cudaGetLastError()));
    if (launch_finalize(kp.S1, kp.S2lo, kp.S2hi, t.na, static_cast<int>(t.nb), t.P, t.L, est_dev, se_dev, s) != MCPD_OK)
        return fail(ctx, MCPD_ECUDA, "finalize kernel launch");
    unsigned long long c[kNumCounters];
    int error = 0;
    CUN(cudaMemcpyAsync(c, kp.counters, sizeof(c), cudaMemcpyDeviceToHost, s));
    CUN(cudaMemcpyAsync(&error, kp.error, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUN(cudaStreamSynchronize(s));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        counters_to_stats(c, stats);
        stats->n_buckets = t.nb;
        stats->n_active = t.na;
        stats->resident_pairs = static_cast<int64_t>(pairs);
    }
    if (error) return fail(ctx, MCPD_ESTEP_LIMIT, "a pair reached the step limit without meeting");
    return MCPD_OK;
}
