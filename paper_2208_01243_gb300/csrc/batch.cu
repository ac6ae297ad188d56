// Batched form of the wavefront aligner: pairs of uneven length and error
// rate go through length-bucketed work queues into persistent launches (one
// per lanes-per-pair value), with the lanes per pair of every bucket chosen by
// an autotuner and the whole run (packing, bucketing, alignment) replayed as a
// CUDA graph.
//
// Buckets.  Each pair's work is bounded by its threshold: with S = limit/g
// scaled score steps, no wavefront is wider than W = min(2 S/E + 3, n+m+1,
// 2 band + 1) diagonals, and the whole pair computes at most C = (S+1) W
// wavefront entries.  A pair's bucket combines a work class (floor(log2(C+1))/3,
// 8 classes) with a width class (W <= 64, 128, 256, more); buckets are
// numbered heaviest work class first, so warps drain the longest pairs first
// and the tail of the launch holds the shortest ones.  Bucketing runs on the
// device (a block-aggregated histogram, a one-warp scan, a block-aggregated
// scatter into an order array), so a replay needs no host round trip.
//
// Launches.  Once the lanes per pair of every bucket are known, the queue
// order groups the buckets that share a group size (heaviest first inside and
// between groups), and each group is one persistent launch over one queue
// range, of the kernel compiled for that group size alone (one kernel holding
// every group size spilled registers and ran 14 % slower).
//
// Autotuner.  For every non-empty bucket, timed trial launches on a sample of
// its pairs large enough to fill the device several times try the group sizes that suit its width class (so
// that no lane walks more than about 64 diagonals per score step; the widest
// class may also use a whole block per pair) and keep the fastest; choices are cached in the context per (costs, band, bucket).
//
// Two passes.  A bucket's scratch is sized for its worst case, which for long
// pairs under a loose threshold only fits one pair per warp.  Most pairs end
// far below their threshold and need a fraction of that history, so the tuner
// also times a compact first pass: fewer lanes per pair and a history capped
// at 16 diagonals per lane on average, followed by a second pass, with the
// bucket's full scratch, over the pairs that outgrew the cap (the first pass
// flags them AIM_F_STEP_CAP; a count/scan/scatter over those flags builds the
// second pass's queues on the device).  Both passes run the exact algorithm,
// so results do not depend on which pairs were retried.
//
// Bound pass.  An exact pass clamps every wavefront to the diagonals that can
// still end within the pair's limit S; a pair whose optimum lies far below S
// computes wavefronts that the clamp barely touches.  A bound pass first runs
// a pruned forward pass (no history, no traceback, wavefronts of a few
// diagonals) whose end score U is the cost of a real alignment, so the
// optimum is at most U; the exact pass then takes min(S, U) as the pair's
// limit and clamps its wavefronts to a diamond around the optimal path.  The
// scores and CIGARs are those of the exact pass alone (the optimum and every
// entry on an optimal path survive the clamp), so the tuner may add a bound
// pass to any bucket it makes faster.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <new>
#include <tuple>
#include <vector>

#include "aim_internal.cuh"
#include "ranges.h"

namespace aim {
namespace {

constexpr int kBuckets = 32;
constexpr int kWidthClasses = 4;
constexpr int kWorkClasses = 8;
constexpr int kCandidates[7] = {1, 2, 4, 8, 16, 32, 256};

struct BucketParams {
    int g, E, band;
    int64_t smax;
    int8_t perm[kBuckets];          // queue order of the buckets (identity, or grouped by lanes per pair)
    int8_t gstart[kBuckets + 1];    // groups of consecutive permuted buckets sharing one lanes-per-pair value
    int ngroups;                    // 0: no groups
};

__device__ __forceinline__ int bucket_of(const PairsView& P, const LimitView& L, const BucketParams& bp, uint32_t i) {
    const int64_t n = P.read_len[i], m = P.target_len[i];
    const int64_t lim = pair_limit(L, i);
    int64_t S = lim < 0 ? 0 : lim / bp.g;
    if (S > bp.smax) S = bp.smax;
    int64_t W = 2 * (S / bp.E) + 3;
    W = min(W, n + m + 1);
    if (bp.band >= 0) W = min(W, 2 * (int64_t)bp.band + 1);
    const int64_t C = (S + 1) * W;
    const int wc = W <= 64 ? 0 : W <= 128 ? 1 : W <= 256 ? 2 : 3;
    int kc = (63 - __clzll((long long)(C + 1))) / 3;
    if (kc > kWorkClasses - 1) kc = kWorkClasses - 1;
    return bp.perm[(kWorkClasses - 1 - kc) * kWidthClasses + (kWidthClasses - 1 - wc)];
}

// `capped` (optional): count and scatter only the pairs whose flag is AIM_F_STEP_CAP (the second pass's queues)
__device__ __forceinline__ bool queued(const uint8_t* capped, uint32_t i) {
    return capped == nullptr || capped[i] == AIM_F_STEP_CAP;
}

__global__ void __launch_bounds__(256) bucket_count_kernel(PairsView P, LimitView L, BucketParams bp,
                                                           uint32_t* counts, const uint8_t* capped) {
    __shared__ uint32_t h[kBuckets];
    if (threadIdx.x < kBuckets) h[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P.num_pairs; i += gridDim.x * blockDim.x)
        if (queued(capped, i)) atomicAdd(&h[bucket_of(P, L, bp, i)], 1u);
    __syncthreads();
    if (threadIdx.x < kBuckets && h[threadIdx.x]) atomicAdd(&counts[threadIdx.x], h[threadIdx.x]);
}

// one warp: bounds[b] = first queue position of bucket b, bounds[32] = total; clears the fill and claim counters.
// With groups, gbounds[j] = first queue position of group j (gbounds[ngroups] = total).
__global__ void bucket_scan_kernel(const uint32_t* counts, uint32_t* bounds, uint32_t* fill, uint32_t* claims,
                                   BucketParams bp, uint32_t* gbounds) {
    const uint32_t lane = threadIdx.x;
    const uint32_t c = counts[lane];
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if ((int)lane >= o) incl += t;
    }
    bounds[lane] = incl - c;
    if (lane == 31) bounds[32] = incl;
    fill[lane] = 0;
    claims[lane] = 0;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const int x = (int)lane <= bp.ngroups ? bp.gstart[lane] : 0;
    const uint32_t at = __shfl_sync(kFull, incl - c, x < 32 ? x : 0);   // every lane takes part
    if (gbounds && (int)lane <= bp.ngroups) gbounds[lane] = x < 32 ? at : total;
}

__global__ void __launch_bounds__(256) bucket_scatter_kernel(PairsView P, LimitView L, BucketParams bp,
                                                             const uint32_t* bounds, uint32_t* fill,
                                                             uint32_t* order, const uint8_t* capped) {
    __shared__ uint32_t h[kBuckets], base[kBuckets];
    for (uint32_t chunk = blockIdx.x * blockDim.x; chunk < P.num_pairs; chunk += gridDim.x * blockDim.x) {
        if (threadIdx.x < kBuckets) h[threadIdx.x] = 0;
        __syncthreads();
        const uint32_t i = chunk + threadIdx.x;
        int b = -1;
        uint32_t r = 0;
        if (i < P.num_pairs && queued(capped, i)) {
            b = bucket_of(P, L, bp, i);
            r = atomicAdd(&h[b], 1u);
        }
        __syncthreads();
        if (threadIdx.x < kBuckets && h[threadIdx.x])
            base[threadIdx.x] = bounds[threadIdx.x] + atomicAdd(&fill[threadIdx.x], h[threadIdx.x]);
        __syncthreads();
        if (b >= 0) order[base[b] + r] = i;
        __syncthreads();
    }
}

// scratch one pair of bucket b can need (bounds of its classes, capped by the plan's worst case)
// (every wavefront of a pair in width class wc is at most 64/128/256 diagonals wide, and a
// pair in work class kc computes fewer than 2^(3(kc+1)) entries per component)
size_t bucket_pair_bytes(const WfaPlan& plan, int b, int G) {
    const int kc = kWorkClasses - 1 - b / kWidthClasses;
    const int wc = kWidthClasses - 1 - b % kWidthClasses;
    size_t hist = plan.hist_entries;
    if (kc < kWorkClasses - 1) {
        const size_t cmax = ((size_t)1 << (3 * (kc + 1))) - 1;
        hist = std::min(hist, cmax + 1);
    }
    if (wc < kWidthClasses - 1) {
        const size_t wmax = (size_t)64 << wc;
        hist = std::min(hist, ((size_t)plan.smax + 1) * wmax + 1);
    }
    return wfa_pair_bytes_capped(plan, G, hist);
}

constexpr int kCompactDiagonalsPerLane = 16;   // first-pass history: wavefronts of about 16 diagonals per lane
constexpr int kBoundDefaultGroup = 4;          // lanes per pair of a forced bound pass
constexpr float kBoundGain = 0.97f;            // a bound pass must save at least 3 % of the bucket's trial time

// scratch one pair of bucket b gets in a compact first pass with G lanes per pair
size_t bucket_compact_bytes(const WfaPlan& plan, int b, int G) {
    const size_t full = bucket_pair_bytes(plan, b, G);
    const size_t compact = wfa_pair_bytes(wfa_plan_compact(plan, (int64_t)kCompactDiagonalsPerLane * G), G);
    return std::min(full, compact);
}

// reads beyond the 8-byte entries' int16 offsets need at least 32 lanes per pair (a compact history)
int default_group_for_bucket(int b, uint32_t max_length) {
    const int wc = kWidthClasses - 1 - b % kWidthClasses;
    const int g = wc == 0 ? 4 : wc == 1 ? 8 : wc == 2 ? 16 : 32;
    return max_length > kMaxWfaLength16 ? std::max(g, 32) : g;
}

}  // namespace
}  // namespace aim

struct aim_batch {
    aim_ctx* ctx;
    uint32_t num_pairs, max_length;
    aim_penalties_t pen;
    int32_t max_edits;
    aim::Resolved r;
    aim::WfaPlan plan;
    aim::PairsView P;
    aim::OutView O;
    const uint8_t *reads, *targets;
    const uint64_t *read_coff, *target_coff;
    uint64_t stride;
    // owned device memory
    uint8_t* mem;
    size_t mem_bytes;
    uint64_t *pr, *pt;
    uint8_t *br, *bt;
    uint32_t *counts, *bounds, *fill, *claims, *trial_bounds, *order;
    uint8_t* scratch;
    size_t scratch_bytes, warp_bytes;   // warp_bytes: the full-scratch pass
    int groups[aim::kBuckets];          // lanes per pair with the bucket's full scratch
    int groups1[aim::kBuckets];         // lanes per pair of a compact first pass (0: the bucket runs in one pass)
    int bound1[aim::kBuckets];          // lanes per pair of a bound pass before the exact one (0: none)
    int32_t* bound;                     // per pair: the bound pass's score (scaled), -1: none
    bool two_pass;
    size_t warp_bytes1;                 // the first pass's scratch per warp when two_pass
    uint32_t *rcounts, *rbounds, *rfill, *rclaims, *rorder;   // second-pass queues
    uint32_t* gbounds;                  // queue range of each group of buckets sharing lanes per pair
    int ggroup[aim::kBuckets];          // lanes per pair of each group
    int gbound[aim::kBuckets];          // lanes per pair of each group's bound pass (0: none)
    size_t gwarp_bytes[aim::kBuckets];  // scratch per warp of each group
    uint32_t host_counts[aim::kBuckets];
    aim::BucketParams bp;
    cudaStream_t stream;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaGraphNode_t ev_start_node, ev_stop_node;
    cudaEvent_t ev_start, ev_stop;   // captured placeholders
    int warps;
};

namespace aim {
namespace {

using TuneKey = std::tuple<int, int, int, int, int, int64_t>;   // x, o, e, band, bucket, smax
using TuneChoice = std::tuple<int, int, int>;   // full-scratch lanes, compact first-pass lanes, bound-pass lanes
std::map<TuneKey, TuneChoice>& tune_cache(aim_ctx* ctx) {
    if (!ctx->tune_cache) ctx->tune_cache = new std::map<TuneKey, TuneChoice>();
    return *static_cast<std::map<TuneKey, TuneChoice>*>(ctx->tune_cache);
}

// packing and bucketing on `st`
cudaError_t enqueue_prepare(aim_batch* b, cudaStream_t st) {
    cudaError_t e = launch_pack(b->reads, b->read_coff, b->P.read_len, b->num_pairs, b->pr, nullptr, b->stride, b->br,
                                st);
    if (e != cudaSuccess) return e;
    e = launch_pack(b->targets, b->target_coff, b->P.target_len, b->num_pairs, b->pt, nullptr, b->stride, b->bt, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->counts, 0, kBuckets * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)std::min<uint64_t>((b->num_pairs + 255) / 256, (uint64_t)b->ctx->num_sms * 8);
    bucket_count_kernel<<<blocks, 256, 0, st>>>(b->P, b->r.lim, b->bp, b->counts, nullptr);
    bucket_scan_kernel<<<1, 32, 0, st>>>(b->counts, b->bounds, b->fill, b->claims, b->bp,
                                         b->bp.ngroups ? b->gbounds : nullptr);
    bucket_scatter_kernel<<<blocks, 256, 0, st>>>(b->P, b->r.lim, b->bp, b->bounds, b->fill, b->order, nullptr);
    return cudaGetLastError();
}

cudaError_t enqueue_align(aim_batch* b, cudaStream_t st, int* warps) {
    if (!b->two_pass) {
        // one launch per group of buckets sharing lanes per pair (and bound-pass lanes), each over one contiguous
        // queue range; a group with a bound pass first runs it over the same range (claim counters of their own)
        *warps = 0;
        bool any_bound = false;
        for (int j = 0; j < b->bp.ngroups; ++j) any_bound |= b->gbound[j] != 0;
        if (any_bound) {
            const cudaError_t e = cudaMemsetAsync(b->rclaims, 0, kBuckets * sizeof(uint32_t), st);
            if (e != cudaSuccess) return e;
        }
        for (int j = 0; j < b->bp.ngroups; ++j) {
            int w = 0;
            WfaPlan exact = b->plan;
            if (b->gbound[j]) {
                WfaPlan bp = b->plan;
                bp.bound = b->bound;
                bp.bound_pass = 1;
                const size_t wb = wfa_warp_bytes(b->gbound[j], wfa_bound_pair_bytes(b->plan));
                const cudaError_t e = launch_wfa_buckets(bp, b->P, b->r.lim, b->O, b->order, b->gbounds + j,
                                                         &b->gbound[j], 1, wb, b->scratch, b->scratch_bytes,
                                                         b->rclaims + j, b->ctx->num_sms, st, &w);
                if (e != cudaSuccess) return e;
                if (w == 0) { *warps = 0; return cudaSuccess; }
                exact.bound = b->bound;
            }
            const cudaError_t e = launch_wfa_buckets(exact, b->P, b->r.lim, b->O, b->order, b->gbounds + j,
                                                     &b->ggroup[j], 1, b->gwarp_bytes[j], b->scratch,
                                                     b->scratch_bytes, b->claims + j, b->ctx->num_sms, st, &w);
            if (e != cudaSuccess) return e;
            if (w == 0) { *warps = 0; return cudaSuccess; }
            *warps = std::max(*warps, w);
        }
        return cudaSuccess;
    }
    int g1[kBuckets];
    for (int k = 0; k < kBuckets; ++k) g1[k] = b->groups1[k] ? b->groups1[k] : b->groups[k];
    cudaError_t e = launch_wfa_buckets(b->plan, b->P, b->r.lim, b->O, b->order, b->bounds, g1, kBuckets,
                                       b->warp_bytes1, b->scratch, b->scratch_bytes, b->claims, b->ctx->num_sms, st,
                                       warps);
    if (e != cudaSuccess || *warps == 0) return e;
    // second pass: queues of the pairs the first pass flagged, then the full scratch
    e = cudaMemsetAsync(b->rcounts, 0, kBuckets * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)std::min<uint64_t>((b->num_pairs + 255) / 256, (uint64_t)b->ctx->num_sms * 8);
    bucket_count_kernel<<<blocks, 256, 0, st>>>(b->P, b->r.lim, b->bp, b->rcounts, b->O.flags);
    bucket_scan_kernel<<<1, 32, 0, st>>>(b->rcounts, b->rbounds, b->rfill, b->rclaims, b->bp, nullptr);
    bucket_scatter_kernel<<<blocks, 256, 0, st>>>(b->P, b->r.lim, b->bp, b->rbounds, b->rfill, b->rorder, b->O.flags);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    WfaPlan retry = b->plan;
    retry.retry_only = 1;
    int w2 = 0;
    e = launch_wfa_buckets(retry, b->P, b->r.lim, b->O, b->rorder, b->rbounds, b->groups, kBuckets, b->warp_bytes,
                           b->scratch, b->scratch_bytes, b->rclaims, b->ctx->num_sms, st, &w2);
    if (e == cudaSuccess && w2 == 0) *warps = 0;
    return e;
}

// one timed trial launch over order positions tb[0]..tb[1] with G lanes per pair and warp_bytes of scratch
cudaError_t trial(aim_batch* b, const WfaPlan& plan, const uint32_t tb[2], int G, size_t wb, cudaEvent_t t0,
                  cudaEvent_t t1, float* ms) {
    cudaStream_t st = b->stream;
    cudaError_t e = cudaMemcpyAsync(b->trial_bounds, tb, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->claims, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaEventRecord(t0, st);
    int w = 0;
    if (e == cudaSuccess)
        e = launch_wfa_buckets(plan, b->P, b->r.lim, b->O, b->order, b->trial_bounds, &G, 1, wb, b->scratch,
                               b->scratch_bytes, b->claims, b->ctx->num_sms, st, &w);
    if (e == cudaSuccess) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, t0, t1);
    return e;
}

// a compact first pass with G1 lanes for bucket k: it must save scratch, use no more lanes than the full pass,
// and fit the device several times over
bool compact_allowed(const aim_batch* b, int k, int G1, int g_full) {
    if (b->max_length > kMaxWfaLength16 && G1 < 32) return false;
    const size_t full = bucket_pair_bytes(b->plan, k, g_full);
    const size_t need = bucket_compact_bytes(b->plan, k, G1);
    if (need >= full || G1 > g_full) return false;
    const size_t min_warps = (size_t)b->ctx->num_sms * 8;
    return wfa_warp_bytes(G1, need) * min_warps <= b->scratch_bytes &&
           wfa_warp_bytes(g_full, full) <= b->scratch_bytes;
}

int autotune(aim_batch* b) {
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) return AIM_ERR_CUDA;
    uint32_t bounds[kBuckets + 1];
    cudaError_t e = cudaMemcpy(bounds, b->bounds, sizeof(bounds), cudaMemcpyDeviceToHost);
    const size_t min_warps = (size_t)b->ctx->num_sms * 8;
    WfaPlan retry = b->plan;
    retry.retry_only = 1;
    for (int k = 0; k < kBuckets && e == cudaSuccess; ++k) {
        const uint32_t count = b->host_counts[k];
        if (!count) continue;
        // a sample that fills the device several times over, so the trial measures throughput, not the
        // latency of a handful of pairs
        const uint32_t sample = std::min<uint32_t>(count, (uint32_t)std::max<size_t>(4096, 16 * min_warps * 4));
        const uint32_t tb[2] = {bounds[k], bounds[k] + sample};
        float best = 1e30f;
        int best_g = b->groups[k];
        // lanes per pair worth trying for this width class: at most ~64 diagonals per lane and score step
        const int wc = kWidthClasses - 1 - k % kWidthClasses;
        const int gmin = wc == 0 ? 1 : wc == 1 ? 2 : wc == 2 ? 4 : 8;
        const int gmax = wc == 0 ? 8 : wc == 1 ? 16 : wc == 2 ? 32 : 256;
        for (int G : kCandidates) {
            if (G < gmin || G > gmax || (b->max_length > kMaxWfaLength16 && G < 32)) continue;
            const size_t wb = wfa_warp_bytes(G, bucket_pair_bytes(b->plan, k, G));
            if (wb * min_warps > b->scratch_bytes) continue;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = trial(b, b->plan, tb, G, wb, t0, t1, &ms);
            if (e == cudaSuccess && ms < best) { best = ms; best_g = G; }
        }
        // compact first pass with fewer lanes, then the full-scratch pass over the pairs that outgrew it
        int best_g1 = 0;
        if (b->ctx->batch_compact != 2) {
            const size_t wb_full = wfa_warp_bytes(best_g, bucket_pair_bytes(b->plan, k, best_g));
            for (int G1 : {4, 8, 16, 32}) {
                if (!compact_allowed(b, k, G1, best_g)) continue;
                const size_t wb = wfa_warp_bytes(G1, bucket_compact_bytes(b->plan, k, G1));
                if (b->ctx->batch_compact == 1) { best_g1 = G1; break; }   // forced: the fewest lanes that fit
                float ms1 = 0.f, ms2 = 0.f;
                for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                    e = trial(b, b->plan, tb, G1, wb, t0, t1, &ms1);
                    if (e == cudaSuccess) e = trial(b, retry, tb, best_g, wb_full, t0, t1, &ms2);
                }
                if (e == cudaSuccess && ms1 + ms2 < best) { best = ms1 + ms2; best_g1 = G1; }
            }
        }
        // a bound pass, then the exact pass clamped at each pair's bound (only where no compact pass was chosen)
        int best_gb = 0;
        if (best_g1 == 0 && b->ctx->batch_bound != 2 && b->max_length <= kMaxWfaLength16) {
            WfaPlan bp = b->plan, ep = b->plan;
            bp.bound = ep.bound = b->bound;
            bp.bound_pass = 1;
            const size_t wb_full = wfa_warp_bytes(best_g, bucket_pair_bytes(b->plan, k, best_g));
            const size_t bpb = wfa_bound_pair_bytes(b->plan);
            if (b->ctx->batch_bound == 1) {
                best_gb = kBoundDefaultGroup;   // forced: the default lanes, no trials
            } else {
                for (int Gb : {4, 8, 16, 32}) {
                    if (wfa_warp_bytes(Gb, bpb) * min_warps > b->scratch_bytes) continue;
                    float ms1 = 0.f, ms2 = 0.f;
                    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                        e = trial(b, bp, tb, Gb, wfa_warp_bytes(Gb, bpb), t0, t1, &ms1);
                        if (e == cudaSuccess) e = trial(b, ep, tb, best_g, wb_full, t0, t1, &ms2);
                    }
                    if (e == cudaSuccess && ms1 + ms2 < kBoundGain * best) { best = ms1 + ms2; best_gb = Gb; }
                }
            }
        }
        b->groups[k] = best_g;
        b->groups1[k] = best_g1;
        b->bound1[k] = best_gb;
        tune_cache(b->ctx)[TuneKey(b->r.costs.x, b->r.costs.o, b->r.costs.e, b->pen.band, k, b->plan.smax)] =
            TuneChoice(best_g, best_g1, best_gb);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return cuda_status(e);
}

void free_batch(aim_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->ev_stop) cudaEventDestroy(b->ev_stop);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->mem) cudaFree(b->mem);
    delete b;
}

}  // namespace

void free_tune_cache(void* cache) { delete static_cast<std::map<TuneKey, TuneChoice>*>(cache); }

}  // namespace aim

namespace aim {

// aim_batch_plan, with the scratch optionally supplied by the caller (ext_scratch, ext_scratch_bytes) instead of
// allocated with the plan: plans whose runs never overlap (the host-buffer pipeline's slots, which share one
// compute stream) can then share one region.
int batch_plan_impl(aim_ctx* ctx, const uint8_t* reads, const uint8_t* targets, const uint64_t* read_char_offsets,
                    const uint64_t* target_char_offsets, const uint32_t* read_lengths, const uint32_t* target_lengths,
                    uint32_t num_pairs, uint32_t max_length, const aim_penalties_t* pen, int32_t max_edits,
                    const int32_t* max_edits_per_pair, int32_t* out_scores, uint32_t* out_cigars,
                    const uint64_t* cigar_offsets, uint32_t* out_cigar_lens, uint8_t* out_flags, size_t scratch_bytes,
                    int autotune, uint8_t* ext_scratch, size_t ext_scratch_bytes, aim_batch** out) {
    if (!out) return AIM_ERR_ARG;
    *out = nullptr;
    if (!ctx || !pen || pen->match != 0 || pen->mismatch < 1 || pen->gap_open < 0 || pen->gap_extend < 1)
        return AIM_ERR_ARG;
    if (num_pairs == 0 || !reads || !targets || !read_char_offsets || !target_char_offsets || !read_lengths ||
        !target_lengths || !out_scores || !out_flags || ((out_cigars == nullptr) != (cigar_offsets == nullptr)))
        return AIM_ERR_ARG;
    if (max_length > kMaxWfaLength) return AIM_ERR_UNSUPPORTED;
    DeviceGuardImpl guard(ctx->device);
    aim_batch* b = new (std::nothrow) aim_batch();
    if (!b) return AIM_ERR_NOMEM;
    std::memset(b, 0, sizeof(*b));
    b->ctx = ctx;
    b->num_pairs = num_pairs;
    b->max_length = max_length;
    b->pen = *pen;
    b->max_edits = max_edits;
    int rc = resolve(AIM_ALGO_WFA_AFFINE, pen, max_edits, max_edits_per_pair, &b->r);
    if (rc) { free_batch(b); return rc; }
    b->plan = plan_wfa(b->r.costs, pen->band, max_length, b->r.max_limit);
    b->bp = BucketParams{};
    b->bp.g = b->plan.g; b->bp.E = b->plan.e; b->bp.band = pen->band; b->bp.smax = b->plan.smax;
    for (int k = 0; k < kBuckets; ++k) b->bp.perm[k] = (int8_t)k;
    b->bp.ngroups = 0;
    b->reads = reads; b->targets = targets; b->read_coff = read_char_offsets; b->target_coff = target_char_offsets;
    b->stride = ((uint64_t)max_length + 31) / 32;

    // groups: cached choice, else the width-class default in one pass
    for (int k = 0; k < kBuckets; ++k) {
        b->groups[k] = default_group_for_bucket(k, max_length);
        b->groups1[k] = 0;
        b->bound1[k] = 0;
        if (ctx->tune_cache) {
            auto& c = tune_cache(ctx);
            auto it = c.find(TuneKey(b->r.costs.x, b->r.costs.o, b->r.costs.e, pen->band, k, b->plan.smax));
            if (it != c.end()) std::tie(b->groups[k], b->groups1[k], b->bound1[k]) = it->second;
        }
    }
    // owned memory: packed sequences, flags, bucket arrays, order, scratch
    const size_t seq_bytes = align_up((size_t)num_pairs * b->stride * 8, 256);
    const size_t flag_bytes = align_up(num_pairs, 256);
    const size_t small_bytes = align_up(10 * (kBuckets + 1) * sizeof(uint32_t), 256);
    const size_t order_bytes = align_up((size_t)num_pairs * sizeof(uint32_t), 256);
    b->scratch_bytes = ext_scratch ? ext_scratch_bytes : scratch_bytes ? scratch_bytes : ctx->ws_bytes;
    b->mem_bytes = 2 * seq_bytes + 2 * flag_bytes + small_bytes + 3 * order_bytes + (ext_scratch ? 0 : b->scratch_bytes);
    cudaError_t e = cudaMalloc(&b->mem, b->mem_bytes);
    if (e != cudaSuccess) { cudaGetLastError(); free_batch(b); return AIM_ERR_NOMEM; }
    uint8_t* p = b->mem;
    b->pr = reinterpret_cast<uint64_t*>(p); p += seq_bytes;
    b->pt = reinterpret_cast<uint64_t*>(p); p += seq_bytes;
    b->br = p; p += flag_bytes;
    b->bt = p; p += flag_bytes;
    uint32_t* sm = reinterpret_cast<uint32_t*>(p); p += small_bytes;
    b->counts = sm; b->bounds = sm + (kBuckets + 1); b->fill = sm + 2 * (kBuckets + 1);
    b->claims = sm + 3 * (kBuckets + 1); b->trial_bounds = sm + 4 * (kBuckets + 1);
    b->rcounts = sm + 5 * (kBuckets + 1); b->rbounds = sm + 6 * (kBuckets + 1);
    b->rfill = sm + 7 * (kBuckets + 1); b->rclaims = sm + 8 * (kBuckets + 1);
    b->gbounds = sm + 9 * (kBuckets + 1);
    b->order = reinterpret_cast<uint32_t*>(p); p += order_bytes;
    b->rorder = reinterpret_cast<uint32_t*>(p); p += order_bytes;
    b->bound = reinterpret_cast<int32_t*>(p); p += order_bytes;
    b->scratch = ext_scratch ? ext_scratch : p;
    b->P = PairsView{b->pr, b->pt, nullptr, nullptr, read_lengths, target_lengths, b->br, b->bt, num_pairs, max_length};
    b->P.stride = b->stride;
    b->O = OutView{out_scores, out_cigars, cigar_offsets, out_cigar_lens, out_flags, stats_of(ctx)};
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { free_batch(b); return cuda_status(e); }

    // prepare once (synchronously) to see the bucket sizes, then tune
    e = enqueue_prepare(b, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaMemcpy(b->host_counts, b->counts, sizeof(b->host_counts), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { free_batch(b); return cuda_status(e); }
    if (autotune) {
        rc = aim::autotune(b);
        if (rc) { free_batch(b); return rc; }
    } else {
        // without trials: forced compact first passes where they fit, or none; forced bound passes, or none
        for (int k = 0; k < kBuckets; ++k) {
            if (ctx->batch_compact != 0) {
                b->groups1[k] = 0;
                if (ctx->batch_compact == 1 && b->host_counts[k])
                    for (int G1 : {4, 8, 16, 32})
                        if (compact_allowed(b, k, G1, b->groups[k])) { b->groups1[k] = G1; break; }
            }
            if (ctx->batch_bound == 2) b->bound1[k] = 0;
            if (ctx->batch_bound == 1)   // bound passes run 4 to 32 lanes per pair, whatever the exact pass uses
                b->bound1[k] = b->max_length <= kMaxWfaLength16 && !b->groups1[k] ? kBoundDefaultGroup : 0;
        }
    }
    // buckets empty at planning keep one pair per warp, so their worst case does not shrink the grid
    for (int k = 0; k < kBuckets; ++k)
        if (!b->host_counts[k]) { b->groups[k] = 32; b->groups1[k] = 0; b->bound1[k] = 0; }
    // scratch per warp of the full pass: the largest need over all buckets (a replay may see a different mix)
    size_t wb = 0;
    for (int k = 0; k < kBuckets; ++k)
        wb = std::max(wb, wfa_warp_bytes(b->groups[k], bucket_pair_bytes(b->plan, k, b->groups[k])));
    b->warp_bytes = wb;
    if (wb > b->scratch_bytes) { free_batch(b); return AIM_ERR_NOMEM; }
    // with a compact first pass, its scratch per warp covers the buckets seen at planning; a pair of another
    // bucket that does not fit is flagged and aligned again by the full pass like any other
    b->two_pass = false;
    for (int k = 0; k < kBuckets; ++k) b->two_pass |= b->groups1[k] != 0;
    b->warp_bytes1 = wb;
    if (b->two_pass) {
        size_t wb1 = 0;
        for (int k = 0; k < kBuckets; ++k) {
            if (!b->host_counts[k]) continue;
            wb1 = std::max(wb1, b->groups1[k] ? wfa_warp_bytes(b->groups1[k], bucket_compact_bytes(b->plan, k,
                                                                                               b->groups1[k]))
                                              : wfa_warp_bytes(b->groups[k], bucket_pair_bytes(b->plan, k,
                                                                                               b->groups[k])));
        }
        b->warp_bytes1 = std::max<size_t>(wb1, 16);
    } else {
        // one pass: the buckets sharing lanes per pair (and bound-pass lanes) become one contiguous queue range
        // (groups in the order of their heaviest bucket, buckets heaviest first inside), and each group is one
        // launch of the kernel compiled for its group size, with scratch per warp sized for that group alone
        int ng = 0;
        for (int k = 0; k < kBuckets; ++k) {
            bool seen = false;
            for (int j = 0; j < ng; ++j) seen |= b->ggroup[j] == b->groups[k] && b->gbound[j] == b->bound1[k];
            if (!seen) { b->ggroup[ng] = b->groups[k]; b->gbound[ng] = b->bound1[k]; ++ng; }
        }
        int next = 0;
        for (int j = 0; j < ng; ++j) {
            b->bp.gstart[j] = (int8_t)next;
            size_t wbj = 16;
            for (int k = 0; k < kBuckets; ++k) {
                if (b->groups[k] != b->ggroup[j] || b->bound1[k] != b->gbound[j]) continue;
                b->bp.perm[k] = (int8_t)next++;
                wbj = std::max(wbj, wfa_warp_bytes(b->groups[k], bucket_pair_bytes(b->plan, k, b->groups[k])));
            }
            b->gwarp_bytes[j] = wbj;
        }
        b->bp.gstart[ng] = (int8_t)kBuckets;
        b->bp.ngroups = ng;
    }

    // record prepare + align as a graph; the two event records bracket the alignment kernel
    if (cudaEventCreate(&b->ev_start) != cudaSuccess || cudaEventCreate(&b->ev_stop) != cudaSuccess) {
        free_batch(b);
        return AIM_ERR_CUDA;
    }
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t ce = enqueue_prepare(b, b->stream);
        if (ce == cudaSuccess) ce = cudaEventRecordWithFlags(b->ev_start, b->stream, cudaEventRecordExternal);
        if (ce == cudaSuccess) ce = enqueue_align(b, b->stream, &b->warps);
        if (ce == cudaSuccess) ce = cudaEventRecordWithFlags(b->ev_stop, b->stream, cudaEventRecordExternal);
        e = cudaStreamEndCapture(b->stream, &b->graph);
        if (ce != cudaSuccess) e = ce;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e == cudaSuccess) {
        size_t nn = 0;
        e = cudaGraphGetNodes(b->graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess) e = cudaGraphGetNodes(b->graph, nodes.data(), &nn);
        for (size_t i = 0; i < nn && e == cudaSuccess; ++i) {
            cudaGraphNodeType t;
            e = cudaGraphNodeGetType(nodes[i], &t);
            if (e != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            e = cudaGraphEventRecordNodeGetEvent(nodes[i], &ev);
            if (ev == b->ev_start) b->ev_start_node = nodes[i];
            if (ev == b->ev_stop) b->ev_stop_node = nodes[i];
        }
    }
    if (e != cudaSuccess || b->warps == 0) {
        free_batch(b);
        return e != cudaSuccess ? cuda_status(e) : AIM_ERR_NOMEM;
    }
    *out = b;
    return AIM_OK;
}

}  // namespace aim

extern "C" {

int aim_batch_plan(aim_ctx* ctx, const uint8_t* reads, const uint8_t* targets, const uint64_t* read_char_offsets,
                   const uint64_t* target_char_offsets, const uint32_t* read_lengths, const uint32_t* target_lengths,
                   uint32_t num_pairs, uint32_t max_length, const aim_penalties_t* pen, int32_t max_edits,
                   const int32_t* max_edits_per_pair, int32_t* out_scores, uint32_t* out_cigars,
                   const uint64_t* cigar_offsets, uint32_t* out_cigar_lens, uint8_t* out_flags, size_t scratch_bytes,
                   int autotune, aim_batch** out) {
    aim::Range range("aim_batch_plan");
    return aim::batch_plan_impl(ctx, reads, targets, read_char_offsets, target_char_offsets, read_lengths,
                                target_lengths, num_pairs, max_length, pen, max_edits, max_edits_per_pair, out_scores,
                                out_cigars, cigar_offsets, out_cigar_lens, out_flags, scratch_bytes, autotune, nullptr,
                                0, out);
}

int aim_batch_run(aim_batch* b, aim_stream_t stream) {
    aim::Range range("aim_batch_run");
    using namespace aim;
    if (!b) return AIM_ERR_ARG;
    DeviceGuardImpl guard(b->ctx->device);
    cudaError_t e = cudaSuccess;
    aim_ctx* ctx = b->ctx;
    if (b->ev_start_node && b->ev_stop_node) {
        const int slot = ctx->timing ? time_slot(ctx, 1) : -1;
        cudaEvent_t s0 = slot >= 0 ? timing_start_event(ctx, 1, slot) : b->ev_start;
        cudaEvent_t s1 = slot >= 0 ? timing_stop_event(ctx, 1, slot) : b->ev_stop;
        e = cudaGraphExecEventRecordNodeSetEvent(b->exec, b->ev_start_node, s0);
        if (e == cudaSuccess) e = cudaGraphExecEventRecordNodeSetEvent(b->exec, b->ev_stop_node, s1);
        if (e != cudaSuccess) return cuda_status(e);
    }
    e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    return cuda_status(e);
}

int aim_batch_info(aim_batch* b, int* groups, uint32_t* counts) {
    if (!b || !groups || !counts) return AIM_ERR_ARG;
    for (int k = 0; k < aim::kBuckets; ++k) {
        groups[k] = b->groups1[k] ? b->groups1[k] : b->groups[k];
        counts[k] = b->host_counts[k];
    }
    return aim::kBuckets;
}

int aim_batch_passes(aim_batch* b, int* first_pass, int* full_pass) {
    if (!b || !first_pass || !full_pass) return AIM_ERR_ARG;
    int compact = 0;
    for (int k = 0; k < aim::kBuckets; ++k) {
        first_pass[k] = b->groups1[k];
        full_pass[k] = b->groups[k];
        compact += b->groups1[k] != 0;
    }
    return compact;
}

int64_t aim_tune_export(aim_ctx* ctx, char* buf, size_t cap) {
    if (!ctx || (cap && !buf)) return AIM_ERR_ARG;
    std::string text;
    if (ctx->tune_cache) {
        char line[160];
        for (const auto& kv : aim::tune_cache(ctx)) {
            const auto& k = kv.first;
            const auto& c = kv.second;
            std::snprintf(line, sizeof(line), "%d %d %d %d %d %lld %d %d %d\n", std::get<0>(k), std::get<1>(k),
                          std::get<2>(k), std::get<3>(k), std::get<4>(k), (long long)std::get<5>(k), std::get<0>(c),
                          std::get<1>(c), std::get<2>(c));
            text += line;
        }
    }
    if (cap) {
        const size_t n = std::min(text.size(), cap - 1);
        std::memcpy(buf, text.data(), n);
        buf[n] = 0;
    }
    return (int64_t)text.size();
}

int aim_tune_import(aim_ctx* ctx, const char* text) {
    if (!ctx || !text) return AIM_ERR_ARG;
    std::vector<std::pair<aim::TuneKey, aim::TuneChoice>> parsed;
    const char* p = text;
    while (*p) {
        int x, o, e, band, bucket, g, g1, gb, used = 0;
        long long smax;
        if (std::sscanf(p, "%d %d %d %d %d %lld %d %d %d%n", &x, &o, &e, &band, &bucket, &smax, &g, &g1, &gb,
                        &used) != 9)
            return AIM_ERR_ARG;
        const auto lanes_ok = [](int v, bool zero) { return (zero && v == 0) || v == 1 || v == 2 || v == 4 ||
                                                            v == 8 || v == 16 || v == 32 || v == 256; };
        if (bucket < 0 || bucket >= aim::kBuckets || !lanes_ok(g, false) || !lanes_ok(g1, true) ||
            !(gb == 0 || gb == 4 || gb == 8 || gb == 16 || gb == 32))
            return AIM_ERR_ARG;
        parsed.emplace_back(aim::TuneKey(x, o, e, band, bucket, (int64_t)smax), aim::TuneChoice(g, g1, gb));
        p += used;
        while (*p == '\n' || *p == ' ' || *p == '\r' || *p == '\t') ++p;
    }
    for (const auto& kv : parsed) aim::tune_cache(ctx)[kv.first] = kv.second;
    return AIM_OK;
}

int aim_batch_bound_passes(aim_batch* b, int* bound_pass) {
    if (!b || !bound_pass) return AIM_ERR_ARG;
    int n = 0;
    for (int k = 0; k < aim::kBuckets; ++k) {
        bound_pass[k] = b->two_pass ? 0 : b->bound1[k];
        n += bound_pass[k] != 0;
    }
    return n;
}

int aim_batch_destroy(aim_batch* b) {
    if (!b) return AIM_OK;
    aim::DeviceGuardImpl guard(b->ctx->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    aim::free_batch(b);
    return aim::cuda_status(e);
}

}  // extern "C"
