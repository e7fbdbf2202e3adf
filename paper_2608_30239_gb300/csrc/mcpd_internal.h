// Private declarations shared by the host table builder, the C ABI and the CUDA kernels.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include <cuda_runtime_api.h>

#include "../../include/mcpd.h"

// A context: one device, one stream.  Defined here so every translation unit of the library
// sees the same definition.
struct mcpd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    size_t smem_optin = 0;
    std::string err;
};

namespace mcpd {

constexpr int kRow = 8;              // pool entries per clone row (one 16-byte shared load)
constexpr int kTSide = kRow + 1;     // acceptance table is kTSide x kTSide, indexed 9 n+ + n-
constexpr int kMaskDeg = 6;          // uniform degrees up to this use mask-indexed thresholds
constexpr int kWarpsPerYRegion = 8; // one 32-column Y region per 8 warps (pairs not yet met)
constexpr int kMaxClones = 65535;
constexpr int kMaxPools = 1022;      // pool byte offsets must fit 16 bits
constexpr int kMaxPoolSize = 255;    // per-pool counts are bytes
constexpr int64_t kMaxBuckets = 1 << 16;

// Counter slots of the device statistics block.
enum Counter {
    kWork = 0, kProgress, kSiteUpdates, kRepsStarted, kRepsRetained, kRepsAborted,
    kZeroCompletion, kStepLimitHits, kMaxTau, kSumTau, kTauOverAudit, kPackLost, kNumCounters = 16
};

// Per-pair statistics record of the one-thread-per-pair kernel, summed into the counters at exit.
enum PairStat {
    kPsProgress = 0, kPsStarted, kPsRetained, kPsAborted, kPsZero, kPsLimit, kPsSumTau, kPsMaxTau,
    kPsTauAudit, kPsSiteUpdates, kPairStats = 10
};

// Per-pair scratch, one contiguous block of 8-byte words per pair: the replication's and the
// slot's sums G in [0, 2 na) (interleaved per clone in the one-thread-per-pair kernel, in two
// halves in the lane-group kernel), the statistics record [2 na, 2 na + kPairStats), then the
// touched-clone bit sets of the replication and of the slot (W 32-bit words each).
#ifdef __CUDACC__
__host__ __device__
#endif
inline long long pair_words(long long na, long long W) { return 2 * na + kPairStats + W; }

// Everything the sampler needs, built on the host from (design, y, params).
struct Tables {
    int32_t n = 0, m = 0, na = 0, deg_max = 0;
    int32_t scan = MCPD_SCAN_SCORE;
    bool coupled = true;
    std::vector<int32_t> active;      // [na] original index of active clone a, ascending
    std::vector<uint64_t> alias;      // [na] prob (low 32) | alias index (high 32)
    std::vector<uint16_t> rows;       // [na * kRow] byte offset of the pool's count | y << 15
    std::vector<uint16_t> rows_pool;  // [na * kRow] pool id | y << 15, 0xFFFF past the clone's pools
    std::vector<uint64_t> T;          // [kTSide * kTSide]
    std::vector<uint64_t> Tnu;        // [na] or empty
    std::vector<uint32_t> init_pairs; // even clone ids a with Tnu[a] or Tnu[a+1] nonzero
    std::vector<double> w;            // [na] scan weights
    std::vector<uint16_t> rows_mask;  // [na * kRow] uniform degree <= kMaskDeg: see build_tables
    std::vector<uint64_t> T_mask;     // [(kMaskDeg + 1) * 64] or empty
    // shared-memory layout of one pair (32-bit words, interleaved over the 32 lanes of a warp)
    int32_t udeg = 0;                 // d if every active clone sits in exactly d pools, else 0
    int32_t W = 0;                    // bit-set words per chain
    int32_t Mp = 0;                   // count words (four pools per word, the padding pool included)
    int32_t wpp = 0;                  // words per column = W + Mp (one chain)
    uint16_t dummy_entry = 0;         // row entry of the padding pool
    uint32_t dummy_word = 0;          // initial value of the word holding the padding pool
    int32_t dummy_word_index = 0;
    // run shape
    int64_t k = 0, ell = 0, L = 0, burn = 0, length = 0, unit = 1;
    int64_t P = 0, B = 0, nb = 1, step_limit = 0, slot_offset = 0, trace_stride = 0, tau_audit = 0;
    bool capped = false;              // meeting cap: step_limit is the cap, a capped pair is kept
    int64_t lag = 1;                  // coupled lag L
    int64_t trace_steps = 0, trace_reps = 0;   // per-replication trajectory records (tests)
    uint64_t seed = 0;
    uint32_t instance = 0;
    bool record_slots = false;
};

int build_tables(const mcpd_design *design, const uint8_t *y, const mcpd_params *params,
                 Tables *out, std::string *err);

// The run's counters (summed over launches) as mcpd_stats; n_buckets, n_active and kernel_ms are
// the caller's.
inline void counters_to_stats(const unsigned long long *c, mcpd_stats *s) {
    const bool lost = c[kPackLost] != 0;
    s->progress_units = static_cast<int64_t>(c[kProgress]);
    s->site_updates = lost ? -1 : static_cast<int64_t>(c[kSiteUpdates]);
    s->reps_started = lost ? -1 : static_cast<int64_t>(c[kRepsStarted]);
    s->reps_retained = lost ? -1 : static_cast<int64_t>(c[kRepsRetained]);
    s->reps_aborted = static_cast<int64_t>(c[kRepsAborted]);
    s->zero_completion_slots = static_cast<int64_t>(c[kZeroCompletion]);
    s->step_limit_hits = static_cast<int64_t>(c[kStepLimitHits]);
    s->max_tau = static_cast<int64_t>(c[kMaxTau]);
    s->sum_tau = static_cast<int64_t>(c[kSumTau]);
    s->tau_over_audit = lost ? -1 : static_cast<int64_t>(c[kTauOverAudit]);
}

// The rows and thresholds the single-instance kernel stages (mask-indexed when available).
inline const std::vector<uint16_t> &kernel_rows(const Tables &t) { return t.rows_mask.empty() ? t.rows : t.rows_mask; }
inline const std::vector<uint64_t> &kernel_T(const Tables &t) { return t.T_mask.empty() ? t.T : t.T_mask; }
inline size_t kernel_table_bytes(const Tables &t) {
    return (static_cast<size_t>(t.na) * 24 + kernel_T(t).size() * 8 + 15) / 16 * 16;
}

// Kernel arguments (plain types only: shared by host and device compilation units).
struct KParams {
    const uint64_t *alias;
    const uint16_t *rows;
    const uint64_t *T;
    const uint64_t *Tnu;
    const uint32_t *init_pairs;       // [n_init_pairs]
    int32_t n_init_pairs;
    long long *pair_scratch;          // [pairs][pair_words(na, W)]
    uint32_t *y_state;                // [pairs / 32][wpp][32] fallback Y columns (pairs not yet met)
    unsigned long long *S1;           // [nb][na]
    unsigned long long *S2lo;         // [nb][na]
    unsigned long long *S2hi;         // [nb][na]
    unsigned long long *bcount;       // [nb]
    unsigned long long *counters;     // [kNumCounters]
    int *error;
    int32_t *slot_nstar;
    long long *slot_S;
    int32_t *slot_reps;
    long long *trace_G;
    int32_t na, m, W, Mp, wpp, deg, nb, scan;
    int32_t udeg, capped;             // uniform degree (0: mixed); 1: the step limit is a meeting cap
    uint32_t dummy_entry, dummy_word;
    int32_t dummy_word_index, coupled;
    long long P, B, k, ell, L, burn, length, unit, step_limit, slot_offset, trace_stride, tau_audit;
    unsigned long long seed;
    uint32_t instance;
    int32_t warps;
    uint32_t smem_tables;             // bytes of staged tables at the start of shared memory
    int32_t y_regions;                // 32-column Y regions in shared memory
    uint32_t rk[20];                  // Philox round keys of the seed
    int32_t nT;                       // threshold entries staged (kTSide^2, or mask-indexed)
    int32_t lag;                      // coupled lag L >= 1
    int32_t *trace_rec;               // [n_trace][trace_reps][4 + trace_steps] or null
    int32_t trace_reps, trace_steps;
};

// Philox4x32-10 round keys of a 64-bit seed: (lo + i 0x9E3779B9, hi + i 0xBB67AE85), i = 0..9.
inline void philox_round_keys(uint64_t seed, uint32_t rk[20]) {
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        rk[2 * i] = k0;
        rk[2 * i + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// One instance of a batched launch (plain types; read by the kernels from global memory).
struct InstDesc {
    const uint64_t *alias;            // [na]
    const uint16_t *rows;             // [na * kRow] count offsets for the interleaved pair layout
    const uint64_t *T;                // [kTSide * kTSide]
    const uint64_t *Tnu;              // [na] or null
    const uint32_t *init_pairs;       // [n_init_pairs] even clone ids with a nonzero threshold
    const uint16_t *rows_pool;        // [na * kRow] pool id | y << 15 (lane-group kernels)
    const uint16_t *rows_mask;        // [na * kRow] mask-indexed rows (uniform degree 3..kMaskDeg) or null
    const uint64_t *T_mask;           // [(kMaskDeg + 1) * 64] or null
    unsigned long long *S1, *S2lo, *S2hi, *bcount;   // this instance's N*_p buckets
    int32_t n_init_pairs, capped;     // capped: the step limit is a meeting cap
    int32_t na, W, wpp, deg, nb, dummy_word_index;
    uint32_t dummy_entry, dummy_word;
    long long P, B, k, ell, L, burn, length, unit, step_limit, slot_offset, tau_audit;
    long long work_begin;             // global index of this instance's first slot in the launch
    long long P_total;                // slots in this instance's buckets (the finalize's P)
    unsigned long long seed;
    uint32_t instance;
    int32_t lag;                      // coupled lag L >= 1
};

// Arguments of a batched launch.
struct BParams {
    const InstDesc *insts;
    int32_t n_inst, coupled, scan, max_wpp;
    int32_t lanes, max_m;             // lanes per pair (1, 8, 16, 32); largest pool count
    long long total_work;
    long long *pair_scratch;          // [pairs][pair_words(max_na, max_W)]
    uint32_t *y_state;                // [pairs / 32][max_wpp][32] fallback Y columns
    unsigned long long *counters;
    int *error;
    int32_t max_na, max_W;
    int32_t y_regions;                // 32-column Y regions in shared memory
    int32_t wide;                     // launch the 20-warp variant of the batch kernel
    int32_t ext;                      // some instance has a meeting cap or a lag > 1
    int32_t udeg;                     // every instance of the class has this uniform degree (0: mixed)
    int32_t any_init;                 // some instance of the class has a random start
};

// Launch shape of the one-thread-per-pair kernel (mcpd_kernels.cu).
struct PairsShape {
    int warps = 0;                    // warps per block
    int y_regions = 0;                // 32-column Y regions per block
    bool wide = false;                // (batches) the 20-warp variant of the kernel
    int per_sm = 1;                   // resident blocks per SM
    size_t smem = 0;                  // dynamic shared memory per block
};
int pairs_y_regions(int coupled, int warps);
size_t pairs_smem_bytes(size_t tables, int wpp, int warps, int y_regions);
// tables: bytes staged at the start of shared memory (0 for batches); wpp: words per column;
// P: slots of a single instance (0 = do not shape by rounds); warps: requested warps (0 = auto);
// ext: the run launches the kernel variant with meeting caps and lags > 1; rnd: a single
// instance with random starts (batches ignore it).
int pairs_shape(int coupled, int scan, int udeg, bool batch, size_t tables, int wpp, size_t smem_optin,
                long long P, int sm_count, int warps, bool ext, bool rnd, PairsShape *out);

// The batched sampling-kernel variants (mcpd_batch.cu): the kernel for a class, and the
// compile-time degree a class of uniform degree udeg runs with (0: the generic build).
using PairsKernelFn = void (*)(const KParams, const BParams);
PairsKernelFn pick_batch(int coupled, int scan, int udeg, bool wide, bool ext);
PairsKernelFn pick_batch_degree(int udeg, bool wide);       // coupled, degrees 4, 5, 7, 8 (mcpd_batch_deg.cu)
PairsKernelFn pick_batch_ext_degree(int udeg, bool wide);   // coupled, cap / lag, degrees 3..8 (mcpd_batch_ext.cu)
int batch_kernel_degree(int coupled, int ext, int udeg);

// Launchers (mcpd_kernels.cu).
int launch_batch(const BParams &bp, int grid, int block, size_t smem, void *stream);
int launch_group(const BParams &bp, int grid, int block, size_t smem, void *stream);
int set_group_smem(int lanes, size_t bytes);
int group_max_threads(int lanes);
int group_occupancy(int lanes, int block, size_t smem, int *blocks_per_sm);
int pairs_max_threads(int coupled, int scan, int udeg, bool batch, bool wide = false, bool ext = false,
                      bool rnd = true);
int launch_finalize_batch(const InstDesc *insts, int n_inst, const int32_t *clone_inst,
                          const int32_t *clone_local, long long total_clones, double *est,
                          double *se, void *stream);
int launch_pairs(const KParams &kp, int grid, int block, size_t smem, void *stream);
// The recording variants (mcpd_trace.cu): launched by launch_pairs when kp.trace_rec is set.
int launch_pairs_trace(const KParams &kp, int grid, int block, size_t smem, void *stream);
int set_trace_smem(size_t bytes);
int launch_finalize(const unsigned long long *S1, const unsigned long long *S2lo,
                    const unsigned long long *S2hi, int na, int nb, long long P, long long L,
                    double *est, double *se, void *stream);
int launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, long long n,
                  void *stream);
int pairs_max_smem(int device, size_t *bytes);

}  // namespace mcpd
