// Internal declarations shared by the CUDA translation units of the aligner.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/aim.h"

namespace aim {

constexpr int kWarp = 32;
constexpr int16_t kNeg16 = -16384;           // invalid wavefront offset (any value < 0 is invalid)
constexpr int32_t kInf = 1 << 28;            // DP infinity
constexpr uint32_t kMaxWfaLength16 = 32000;  // the 8-byte wavefront entries store offsets as int16
constexpr uint32_t kMaxWfaLength16c = 16382; // the 16-bit compact history stores h + 1 in 14 bits
constexpr uint32_t kCompactMinLength = 2048; // reads longer than this use a compact history (exact, >= 32 lanes)
constexpr uint32_t kMaxWfaLength = 1u << 20; // the wavefront algorithms' length limit (32-bit compact history)
constexpr int kMaxDpBand = 127;              // DP kernels: 2*band+1 diagonals over R <= 4 lane blocks

// BAM CIGAR op codes
constexpr uint32_t kOpMatch = 7, kOpMismatch = 8, kOpIns = 1, kOpDel = 2;

// ---- packed sequence access (2 bits per base, first base in the top bits) ----

__device__ __forceinline__ uint32_t base_at(const uint64_t* __restrict__ w, uint32_t i) {
    return (uint32_t)(__ldg(w + (i >> 5)) >> (62 - 2 * (i & 31))) & 3u;
}

// The 64 bits that start sh bits (0..63) into the 128-bit value hi:lo, built from 32-bit halves with two
// funnel shifts: for sh < 32 the halves (hi.1, hi.0, lo.1) shift by sh, else (hi.0, lo.1, lo.0) by sh - 32.
// This is (hi << sh) | (lo >> (64 - sh)) (just hi for sh == 0) without 64-bit variable shifts.
__device__ __forceinline__ uint64_t join_window(uint64_t hi, uint64_t lo, uint32_t sh) {
    const uint32_t h1 = (uint32_t)(hi >> 32), h0 = (uint32_t)hi, l1 = (uint32_t)(lo >> 32), l0 = (uint32_t)lo;
    const bool up = (sh & 32u) != 0;
    const uint32_t a = up ? h0 : h1, b = up ? l1 : h0, c = up ? l0 : l1;
    return ((uint64_t)__funnelshift_l(b, a, sh) << 32) | __funnelshift_l(c, b, sh);
}

// 32 bases starting at base `pos` of a sequence of `nwords` words, first base in the top bits.
// Bases past the last word read as 0; callers cap comparisons by the remaining length.
__device__ __forceinline__ uint64_t window32(const uint64_t* __restrict__ w, uint32_t nwords, uint32_t pos) {
    const uint32_t wi = pos >> 5, sh = 2 * (pos & 31);
    const uint64_t hi = wi < nwords ? __ldg(w + wi) : 0ull;
    const uint64_t lo = (wi + 1 < nwords) ? __ldg(w + wi + 1) : 0ull;
    return join_window(hi, lo, sh);
}

// ---- per-call description handed to the kernels ----

struct Costs {
    int32_t x, o, e;   // mismatch, gap open, gap extend (match is 0)
};

struct PairsView {
    const uint64_t* reads;
    const uint64_t* targets;
    const uint64_t* read_off;
    const uint64_t* target_off;
    const uint32_t* read_len;
    const uint32_t* target_len;
    const uint8_t* bad_r;        // optional per-read input-error flags (ASCII path), may be null
    const uint8_t* bad_t;        // optional per-target input-error flags, may be null
    uint32_t num_pairs;
    uint32_t max_length;
    uint64_t stride;             // words per sequence when the offset arrays are null
};

__device__ __forceinline__ const uint64_t* read_words(const PairsView& P, uint32_t i) {
    return P.reads + (P.read_off ? __ldg(P.read_off + i) : (uint64_t)i * P.stride);
}
__device__ __forceinline__ const uint64_t* target_words(const PairsView& P, uint32_t i) {
    return P.targets + (P.target_off ? __ldg(P.target_off + i) : (uint64_t)i * P.stride);
}

struct OutView {
    int32_t* scores;
    uint32_t* cigars;            // may be null
    const uint64_t* cigar_off;   // may be null
    uint32_t* cigar_lens;        // may be null
    uint8_t* flags;
    unsigned long long* stats;   // work counters (see aim_stats_read), may be null
};

struct LimitView {
    int64_t limit;               // limit for every pair when per_pair is null (kUnbounded: none)
    const int32_t* per_pair;     // per-pair max_edits, or null
    int32_t max_edits_bound;     // upper bound for per_pair entries
    int32_t edit_cost;           // limit = per_pair * edit_cost (unit: 1, affine: max(x, o+e))
};

constexpr int64_t kUnbounded = (int64_t)1 << 40;

// limit of pair i; -2 if its per-pair threshold exceeds the stated bound
__device__ __forceinline__ bool pair_bad(const PairsView& P, uint32_t i) {
    return (P.bad_r && P.bad_r[i]) || (P.bad_t && P.bad_t[i]);
}

__device__ __forceinline__ int64_t pair_limit(const LimitView& L, uint32_t i) {
    if (L.per_pair == nullptr) return L.limit;
    int32_t me = __ldg(L.per_pair + i);
    if (me > L.max_edits_bound) return -2;
    if (me < 0) return kUnbounded;
    return (int64_t)me * L.edit_cost;
}

// ---- launchers (each returns a cudaError_t) ----

cudaError_t launch_pack(const uint8_t* ascii, const uint64_t* char_off, const uint32_t* len, uint32_t count,
                        uint64_t* packed, const uint64_t* word_off, uint64_t word_stride, uint8_t* bad,
                        cudaStream_t st);

struct DpPlan {
    int band;            // effective band b (2b+1 diagonals)
    int blocks;          // lane blocks R (1, 2 or 4)
    int pairs_per_warp;  // 1, or 2 / 4 for bands up to 15 / 7 (one pair per segment of 16 / 8 lanes)
    bool unit;
    size_t slot_bytes;   // per-warp scratch
};
DpPlan plan_dp(bool unit, int band, uint32_t max_length, int64_t max_limit_hint);
cudaError_t launch_dp(const DpPlan& plan, const Costs& c, const PairsView& P, const LimitView& L, const OutView& O,
                      int64_t max_limit, uint8_t* scratch, size_t scratch_bytes, uint32_t* counter,
                      int num_sms, cudaStream_t st, int* warps_used);

constexpr int kMaxBuckets = 32;
// wavefront history: one entry per (score, diagonal) holds M~, I~, D~ and a spare slot as four int16, so an entry
// is written with one 8-byte store
constexpr int kEntryElems = 4;

struct WfaPlan {
    int g;               // gcd of the costs; scores run in units of g
    int x, oe, e;        // scaled mismatch, open+extend, extend
    int64_t smax;        // largest scaled score any pair may reach
    int band;            // < 0: none
    uint32_t max_length; // longest read or target of the call
    size_t hist_entries; // wavefront history entries (score, diagonal) per pair, worst case
    uint32_t live_w;     // compact forms: entries per live-ring slot (a power of 2 above the widest wavefront)
    uint32_t live_slots; // compact forms: live-ring slots (a power of 2 above the farthest source score)
    int runs_cap;        // CIGAR runs staged per pair
    int rec_pad;         // empty records before record 0 (max(x, oe, e)): every source record s - x, s - oe,
                         // s - e of a score s >= 0 can be read without a check
    size_t meta_bytes;   // those and the per-score (lo, count, base, width) records, int4 each
    size_t runs_bytes;   // run staging
    int adapt_min_len;   // WFA-adaptive: prune wavefronts spanning >= this many diagonals (< 0: exact WFA)
    int adapt_max_dist;  // WFA-adaptive: drop outer diagonals more than this behind the closest to the end
    int retry_only;      // launch aligns only the pairs a previous pass flagged AIM_F_STEP_CAP
    int32_t* bound;      // per pair: a scaled score some alignment reaches (written by a bound pass, -1: none);
                         // exact launches take min(limit, bound) as the pair's limit when set (null: none)
    int bound_pass;      // the launch is a bound pass: pruned, no history, no traceback; writes bound
    int bound_min_len, bound_max_dist;   // the bound pass's pruning (as adapt_min_len, adapt_max_dist)
};
// the bound pass's pruning: wavefronts of at least kBoundMinLen diagonals keep those within kBoundMaxDist of the
// diagonal closest to the end
constexpr int kBoundMinLen = 4;
constexpr int kBoundMaxDist = 3;
// scratch one pair of a bound pass needs (meta records and the live ring)
size_t wfa_bound_pair_bytes(const WfaPlan& p);
// the plan with its history sized for wavefronts at most `width` diagonals wide (a compact first pass)
WfaPlan wfa_plan_compact(const WfaPlan& full, int64_t width);
WfaPlan plan_wfa(const Costs& c, int band, uint32_t max_length, int64_t max_limit);
// worst-case history entries of one pair: every wavefront as wide as its sources allow and, when clamp (the exact
// kernels), no wider than the diagonals that can still end within the limit
size_t wfa_hist_entries(const WfaPlan& p, int64_t max_len, int64_t smax, bool clamp);
// lanes per pair suited to the widest wavefront the plan allows (4, 8, 16, 32 or 256; 1 and 2 are valid too;
// at least 32 beyond kMaxWfaLength16)
int wfa_default_group(const WfaPlan& p, uint32_t max_length);
// storage form of a launch with `group` lanes per pair: 0 8-byte entries, 1 16-bit compact, 2 32-bit compact
int wfa_format(const WfaPlan& p, int group);
size_t wfa_live_bytes(const WfaPlan& p, int fmt);
// scratch one pair may need with `group` lanes per pair (its history sized for p.hist_entries, or `entries`)
size_t wfa_pair_bytes(const WfaPlan& p, int group);
size_t wfa_pair_bytes_capped(const WfaPlan& p, int group, size_t entries);
// scratch per warp for `group` lanes per pair (256: the block's 8 warps share one pair's scratch)
size_t wfa_warp_bytes(int group, size_t pair_bytes);

struct WfaArgs {
    int X, OE, E, g;
    int64_t smax;
    int band;
    PairsView P;
    LimitView L;
    OutView O;
    uint8_t* scratch;
    size_t warp_bytes;         // scratch per warp; a warp of G-lane groups gives each group warp_bytes / (32/G)
    size_t pair_bytes;         // scratch one pair of a G-lane group may need (G <= 32; the rest of the group's
                               // share holds finished pairs awaiting their traceback)
    size_t meta_bytes, runs_bytes;
    uint32_t rec_pad;          // empty records before record 0 in each pair's region
    uint32_t runs_cap;
    uint32_t nwarps;
    uint32_t seq_slot_words;   // words per sequence copy in shared memory (0: the extend reads global memory)
    uint32_t meta_ring;        // records per group in a shared-memory ring of recent scores (power of 2; 0: none)
    uint32_t ring_off;         // byte offset of the rings in dynamic shared memory (after the sequence copies)
    uint32_t live_w, live_slots;   // compact histories: live-ring slot width and slot count (powers of 2)
    size_t live_bytes;             // compact histories: bytes of a pair's live ring (at the end of its region)
    const uint32_t* order;     // pair index at each queue position, or null (identity)
    const uint32_t* bounds;    // bucket b covers queue positions [bounds[b], bounds[b+1]); null: one bucket of all
    uint32_t* counters;        // one claim counter per bucket, zero at launch
    int nbuckets;
    int adapt_min_len, adapt_max_dist;   // WFA-adaptive pruning and source-following traceback (min_len < 0: off)
    int retry_only;            // align only pairs whose flag is AIM_F_STEP_CAP (a second pass with larger scratch)
    int32_t* bound;            // per-pair scaled score bounds: the bound pass writes them, exact passes read them
    int16_t group[kMaxBuckets]; // lanes per pair of each bucket (1..32, or 256: a whole block)
};

// bucketed queues (longest-first order given by the caller): one launch per distinct group size among the
// buckets, each draining the buckets of its size; warps_used: the largest grid (0: nothing fitted)
cudaError_t launch_wfa_buckets(const WfaPlan& plan, const PairsView& P, const LimitView& L, const OutView& O,
                               const uint32_t* order, const uint32_t* bounds, const int* groups, int nbuckets,
                               size_t warp_bytes, uint8_t* scratch, size_t scratch_bytes, uint32_t* counters,
                               int num_sms, cudaStream_t st, int* warps_used);
// one launch over all pairs in index order with `group` lanes per pair
cudaError_t launch_wfa(const WfaPlan& plan, int group, const PairsView& P, const LimitView& L, const OutView& O,
                       uint8_t* scratch, size_t scratch_bytes, uint32_t* counter, int num_sms, cudaStream_t st,
                       int* warps_used);

// GenASM (windowed bitap): scratch per warp for windows of W bases under the largest threshold max_limit
size_t genasm_warp_bytes(int W, int64_t max_limit, uint32_t max_length);
cudaError_t launch_genasm(int W, int O, const PairsView& P, const LimitView& L, const OutView& Ov, int64_t max_limit,
                          uint8_t* scratch, size_t scratch_bytes, uint32_t* counter, int num_sms, cudaStream_t st,
                          int* warps_used);

}  // namespace aim

namespace aim {

constexpr uint32_t kFull = 0xffffffffu;

__host__ __device__ __forceinline__ size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Run-length encoder for ops produced end-first (one thread).  Runs land in
// `runs` in end-first order; `n` counts every run, even past `cap`.
struct RunWriter {
    uint32_t* runs;
    uint32_t cap;
    uint32_t n;
    uint32_t op;
    uint32_t len;
    __device__ __forceinline__ void init(uint32_t* r, uint32_t c) { runs = r; cap = c; n = 0; op = 0; len = 0; }
    __device__ __forceinline__ void flush() {
        if (len) {
            if (n < cap) runs[n] = (len << 4) | op;
            ++n;
        }
    }
    __device__ __forceinline__ void put(uint32_t o, uint32_t l) {
        if (o == op) { len += l; return; }
        flush();
        op = o; len = l;
    }
    __device__ __forceinline__ void finish() { flush(); len = 0; }
};

// Lane 0 only: score/flags/run count of pair i.
__device__ __forceinline__ void write_header(const OutView& O, uint32_t i, int32_t score, uint8_t flags,
                                             uint32_t nruns) {
    O.scores[i] = score;
    O.flags[i] = flags;
    if (O.cigar_lens) O.cigar_lens[i] = nruns;
}

// Whole warp: copy end-first staged runs into pair i's CIGAR in start-first
// order, or flag an overflow.  `nruns` and `staged_ok` must be warp-uniform.
__device__ __forceinline__ void write_cigar(const OutView& O, uint32_t i, int32_t score, const uint32_t* staged,
                                            uint32_t nruns, bool staged_ok, uint32_t lane) {
    uint8_t flags = staged_ok ? 0 : AIM_F_STEP_CAP;
    if (O.cigars && O.cigar_off && staged_ok) {
        const uint64_t off = O.cigar_off[i];
        const uint64_t cap = O.cigar_off[i + 1] - off;
        if (nruns <= cap) {
            for (uint32_t j = lane; j < nruns; j += 32) O.cigars[off + j] = staged[nruns - 1 - j];
        } else {
            flags |= AIM_F_CIGAR_OVERFLOW;
        }
    }
    if (lane == 0) write_header(O, i, staged_ok ? score : -1, flags, nruns);
}

}  // namespace aim

namespace aim {

// Whole warp: add each lane's counter into stats[slot] with one atomic per warp.
__device__ __forceinline__ void warp_stat_add(unsigned long long* stats, int slot, unsigned long long v,
                                              uint32_t lane) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (stats && lane == 0 && v) atomicAdd(stats + slot, v);
}

}  // namespace aim

// ---- context (shared by the C ABI translation units) ----

namespace aim {
constexpr int kTimedLaunches = 4096;
constexpr size_t kHeaderBytes = 256;   // launch counter and work counters at the start of the workspace
constexpr size_t kStatsOffset = 64;    // five uint64 work counters
constexpr int kStats = 5;
struct KernelTimes;
}  // namespace aim

struct aim_ctx {
    int device;
    int num_sms;
    uint8_t* ws;                  // workspace (device): [launch counter | stats | ...][scratch]
    size_t ws_bytes;
    bool timing;
    aim::KernelTimes* times[2];   // 0: packer, 1: alignment kernels; created on first enable
    int wfa_group;                // lanes per pair for the WFA; 0: chosen from the plan
    int adapt_min_len, adapt_max_dist;   // WFA-adaptive parameters
    int genasm_w, genasm_o;       // GenASM window and overlap
    int batch_compact;            // batch plans: 0 tuner decides on compact first passes, 1 always, 2 never
    int batch_bound;              // batch plans: 0 tuner decides on bound passes, 1 always, 2 never
    void* tune_cache;             // autotuner choices (owned; see batch.cu)
    void* host_pipe;              // buffers, streams and plans of aim_align_batch_host (owned; see host.cu)
};

namespace aim {

struct Resolved {
    Costs costs;
    LimitView lim;
    int64_t max_limit;   // largest limit of any pair (kUnbounded: none)
};

int cuda_status(cudaError_t e);
unsigned long long* stats_of(aim_ctx* ctx);
int time_begin(aim_ctx* ctx, int kind, cudaStream_t st);
void time_end(aim_ctx* ctx, int kind, int slot, cudaStream_t st);
int resolve(int algo, const aim_penalties_t* pen, int32_t max_edits, const int32_t* per_pair, Resolved* r);
// timing ring access for launches recorded inside a graph: claim a slot (-1: timing off or ring full)
int time_slot(aim_ctx* ctx, int kind);
cudaEvent_t timing_start_event(aim_ctx* ctx, int kind, int slot);
cudaEvent_t timing_stop_event(aim_ctx* ctx, int kind, int slot);
void free_tune_cache(void* cache);
void free_host_pipe(void* pipe);
int batch_plan_impl(aim_ctx* ctx, const uint8_t* reads, const uint8_t* targets, const uint64_t* read_char_offsets,
                    const uint64_t* target_char_offsets, const uint32_t* read_lengths, const uint32_t* target_lengths,
                    uint32_t num_pairs, uint32_t max_length, const aim_penalties_t* pen, int32_t max_edits,
                    const int32_t* max_edits_per_pair, int32_t* out_scores, uint32_t* out_cigars,
                    const uint64_t* cigar_offsets, uint32_t* out_cigar_lens, uint8_t* out_flags, size_t scratch_bytes,
                    int autotune, uint8_t* ext_scratch, size_t ext_scratch_bytes, aim_batch** out);

struct DeviceGuardImpl {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuardImpl(int dev);
    ~DeviceGuardImpl();
};

}  // namespace aim
