// C ABI of the aligner: context, argument checks, threshold rule, dispatch.
// Declarations and contracts are in include/aim.h.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>

#include "aim_internal.cuh"
#include "ranges.h"

namespace aim {
struct KernelTimes {
    cudaEvent_t start[kTimedLaunches];
    cudaEvent_t stop[kTimedLaunches];
    int recorded;     // launches with events
    int launches;     // all launches since the last read
};
}  // namespace aim

namespace {
thread_local int g_last_cuda_error = 0;
}  // namespace

namespace aim {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return AIM_OK;
    g_last_cuda_error = (int)e;
    return AIM_ERR_CUDA;
}

unsigned long long* stats_of(aim_ctx* ctx) { return reinterpret_cast<unsigned long long*>(ctx->ws + kStatsOffset); }

// Record the start event of one launch of `kind` (when timing is on); returns its slot or -1.
int time_begin(aim_ctx* ctx, int kind, cudaStream_t st) {
    if (!ctx->timing) return -1;
    KernelTimes* t = ctx->times[kind];
    const int i = t->recorded;
    ++t->launches;
    if (i >= kTimedLaunches) return -1;
    cudaEventRecord(t->start[i], st);
    return i;
}

void time_end(aim_ctx* ctx, int kind, int slot, cudaStream_t st) {
    if (slot < 0) return;
    KernelTimes* t = ctx->times[kind];
    cudaEventRecord(t->stop[slot], st);
    t->recorded = slot + 1;
}

int time_slot(aim_ctx* ctx, int kind) {
    if (!ctx->timing) return -1;
    KernelTimes* t = ctx->times[kind];
    const int i = t->recorded;
    ++t->launches;
    if (i >= kTimedLaunches) return -1;
    t->recorded = i + 1;
    return i;
}

cudaEvent_t timing_start_event(aim_ctx* ctx, int kind, int slot) { return ctx->times[kind]->start[slot]; }
cudaEvent_t timing_stop_event(aim_ctx* ctx, int kind, int slot) { return ctx->times[kind]->stop[slot]; }

}  // namespace aim

using aim::cuda_status;
using aim::kHeaderBytes;
using aim::KernelTimes;
using aim::kTimedLaunches;
using aim::stats_of;
using aim::time_begin;
using aim::time_end;

namespace aim {
DeviceGuardImpl::DeviceGuardImpl(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
}
DeviceGuardImpl::~DeviceGuardImpl() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}
}  // namespace aim

namespace {
using DeviceGuard = aim::DeviceGuardImpl;

bool penalties_ok(const aim_penalties_t* p) {
    return p && p->match == 0 && p->mismatch >= 1 && p->gap_open >= 0 && p->gap_extend >= 1 &&
           p->mismatch <= (1 << 20) && p->gap_open <= (1 << 20) && p->gap_extend <= (1 << 20);
}

}  // namespace

namespace aim {
// The threshold rule of aim.h: max_score overrides; else max_edits (x unit cost, or x max(x, o+e)).
int resolve(int algo, const aim_penalties_t* pen, int32_t max_edits, const int32_t* per_pair, Resolved* r) {
    const bool unit = algo == AIM_ALGO_EDIT_NW || algo == AIM_ALGO_GENASM;
    r->costs = unit ? aim::Costs{1, 0, 1} : aim::Costs{pen->mismatch, pen->gap_open, pen->gap_extend};
    const int32_t edit_cost = unit ? 1 : std::max(r->costs.x, r->costs.o + r->costs.e);
    r->lim.per_pair = nullptr;
    r->lim.max_edits_bound = max_edits;
    r->lim.edit_cost = edit_cost;
    if (pen->max_score >= 0) {
        r->lim.limit = pen->max_score;
        r->max_limit = pen->max_score;
        return AIM_OK;
    }
    if (per_pair) {
        if (max_edits < 0) return AIM_ERR_ARG;   // the bound sizes the scratch
        r->lim.per_pair = per_pair;
        r->lim.limit = (int64_t)max_edits * edit_cost;
        r->max_limit = r->lim.limit;
        return AIM_OK;
    }
    r->lim.limit = max_edits < 0 ? aim::kUnbounded : (int64_t)max_edits * edit_cost;
    r->max_limit = r->lim.limit;
    return AIM_OK;
}
}  // namespace aim

using aim::Resolved;
using aim::resolve;

namespace {

int align_packed(aim_ctx* ctx, const aim::PairsView& P, int algo, const aim_penalties_t* pen, int32_t max_edits,
                 const int32_t* per_pair, const aim::OutView& O, cudaStream_t st, uint8_t* scratch,
                 size_t scratch_bytes) {
    Resolved r;
    int rc = resolve(algo, pen, max_edits, per_pair, &r);
    if (rc) return rc;
    uint32_t* counter = reinterpret_cast<uint32_t*>(ctx->ws);
    int warps = 0;
    cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(uint32_t), st);
    if (err != cudaSuccess) return cuda_status(err);
    int slot = -1;
    if (algo == AIM_ALGO_GENASM) {
        if (pen->band >= 0) return AIM_ERR_UNSUPPORTED;
        if (aim::genasm_warp_bytes(ctx->genasm_w, r.max_limit, P.max_length) + 256 > scratch_bytes)
            return AIM_ERR_NOMEM;
        slot = time_begin(ctx, 1, st);
        err = aim::launch_genasm(ctx->genasm_w, ctx->genasm_o, P, r.lim, O, r.max_limit, scratch, scratch_bytes,
                                 counter, ctx->num_sms, st, &warps);
    } else if (algo == AIM_ALGO_WFA_AFFINE || algo == AIM_ALGO_WFA_ADAPTIVE) {
        if (P.max_length > aim::kMaxWfaLength) return AIM_ERR_UNSUPPORTED;
        // WFA-adaptive keeps 8-byte wavefront entries (int16 offsets)
        if (algo == AIM_ALGO_WFA_ADAPTIVE && P.max_length > aim::kMaxWfaLength16) return AIM_ERR_UNSUPPORTED;
        aim::WfaPlan plan = aim::plan_wfa(r.costs, pen->band, P.max_length, r.max_limit);
        // launches use whole blocks of 8 warps: widen the groups until 8 warps' scratch fits (and to 32 lanes
        // for reads beyond the 8-byte entries' int16 offsets)
        auto fit_group = [&](const aim::WfaPlan& pl, int g0) {
            int g = P.max_length > aim::kMaxWfaLength16 ? std::max(g0, 32) : g0;
            while (g <= 32 && 8 * aim::wfa_warp_bytes(g, aim::wfa_pair_bytes(pl, g)) > scratch_bytes)
                g = g == 32 ? 256 : g * 2;
            return 8 * aim::wfa_warp_bytes(g, aim::wfa_pair_bytes(pl, g)) > scratch_bytes ? 0 : g;
        };
        if (algo == AIM_ALGO_WFA_ADAPTIVE) {
            plan.adapt_min_len = ctx->adapt_min_len;
            plan.adapt_max_dist = ctx->adapt_max_dist;
            // the adaptive kernels keep the unclamped wavefronts their pruning rule reads
            plan.hist_entries = aim::wfa_hist_entries(plan, P.max_length, plan.smax, false);
            // pruning keeps wavefronts narrow: a first pass sized and grouped for a typical pruned width, then
            // a second pass with the full worst-case scratch for any pair that outgrew it
            int64_t width = 4 * ((int64_t)plan.adapt_max_dist + plan.adapt_min_len) + 64;
            width = std::min<int64_t>(width, 2 * (plan.smax / std::max(plan.e, 1)) + 3);   // never wider than exact
            width = std::min<int64_t>(width, 2 * (int64_t)P.max_length + 1);
            const aim::WfaPlan compact = aim::wfa_plan_compact(plan, width);
            int g1 = ctx->wfa_group ? ctx->wfa_group : (width <= 64 ? 4 : width <= 128 ? 8 : width <= 256 ? 16 : 32);
            g1 = fit_group(compact, g1);
            int group = fit_group(plan, ctx->wfa_group ? ctx->wfa_group : aim::wfa_default_group(plan, P.max_length));
            if (!g1 || !group) return AIM_ERR_NOMEM;
            slot = time_begin(ctx, 1, st);
            err = aim::launch_wfa(compact, g1, P, r.lim, O, scratch, scratch_bytes, counter, ctx->num_sms, st, &warps);
            if (err == cudaSuccess && warps > 0) {
                aim::WfaPlan retry = plan;
                retry.retry_only = 1;
                err = cudaMemsetAsync(counter, 0, sizeof(uint32_t), st);
                int w2 = 0;
                if (err == cudaSuccess)
                    err = aim::launch_wfa(retry, group, P, r.lim, O, scratch, scratch_bytes, counter, ctx->num_sms, st,
                                          &w2);
                if (err == cudaSuccess && w2 == 0) warps = 0;
            }
        } else {
            const int group = fit_group(plan, ctx->wfa_group ? ctx->wfa_group
                                                             : aim::wfa_default_group(plan, P.max_length));
            if (!group) return AIM_ERR_NOMEM;
            slot = time_begin(ctx, 1, st);
            err = aim::launch_wfa(plan, group, P, r.lim, O, scratch, scratch_bytes, counter, ctx->num_sms, st, &warps);
        }
    } else {
        const bool unit = algo == AIM_ALGO_EDIT_NW;
        int64_t b = P.max_length;
        if (pen->band >= 0) b = std::min<int64_t>(b, pen->band);
        if (r.max_limit < aim::kUnbounded) {
            int64_t derived;
            if (unit) derived = r.max_limit;   // a path of cost <= limit never leaves |h - v| <= limit
            else derived = r.max_limit >= r.costs.o ? (r.max_limit - r.costs.o) / r.costs.e : 0;
            b = std::min(b, derived);
        }
        if (b > aim::kMaxDpBand) return AIM_ERR_UNSUPPORTED;
        const aim::DpPlan plan = aim::plan_dp(unit, (int)b, P.max_length, r.max_limit);
        if (plan.slot_bytes > scratch_bytes) return AIM_ERR_NOMEM;
        slot = time_begin(ctx, 1, st);
        err = aim::launch_dp(plan, r.costs, P, r.lim, O, r.max_limit, scratch, scratch_bytes, counter, ctx->num_sms,
                             st, &warps);
    }
    time_end(ctx, 1, slot, st);
    if (err != cudaSuccess) return cuda_status(err);
    if (warps == 0 && P.num_pairs > 0) return AIM_ERR_NOMEM;
    return AIM_OK;
}

bool common_args_ok(aim_ctx* ctx, const void* rl, const void* tl, uint32_t num_pairs, int algo,
                    const aim_penalties_t* pen, int32_t* out_scores, uint32_t* out_cigars,
                    const uint64_t* cigar_offsets, uint8_t* out_flags) {
    if (!ctx || !pen) return false;
    if (algo < AIM_ALGO_EDIT_NW || algo > AIM_ALGO_GENASM) return false;
    const bool unit = algo == AIM_ALGO_EDIT_NW || algo == AIM_ALGO_GENASM;
    if (!unit && !penalties_ok(pen)) return false;
    if (unit && pen->match != 0) return false;
    if (num_pairs == 0) return true;
    if (!rl || !tl || !out_scores || !out_flags) return false;
    if ((out_cigars == nullptr) != (cigar_offsets == nullptr)) return false;
    return true;
}

}  // namespace

extern "C" {

int aim_version(void) { return 100; }

const char* aim_status_string(int status) {
    switch (status) {
        case AIM_OK: return "ok";
        case AIM_ERR_ARG: return "bad argument";
        case AIM_ERR_INPUT: return "bad input";
        case AIM_ERR_NOMEM: return "workspace too small";
        case AIM_ERR_CUDA: return "CUDA error";
        case AIM_ERR_UNSUPPORTED: return "unsupported";
        case AIM_ERR_CANCELLED: return "cancelled";
        case AIM_ERR_BUSY: return "already admitted";
        default: return "unknown status";
    }
}

int aim_last_cuda_error(void) { return g_last_cuda_error; }

int aim_create(aim_ctx** out, int device, size_t workspace_bytes) {
    if (!out) return AIM_ERR_ARG;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_status(e);
    if (device < 0 || device >= count) return AIM_ERR_ARG;
    DeviceGuard g(device);
    if (!g.ok) return cuda_status(cudaGetLastError());
    aim_ctx* c = new (std::nothrow) aim_ctx();
    if (!c) return AIM_ERR_NOMEM;
    c->device = device;
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) { delete c; return cuda_status(e); }
    c->ws_bytes = workspace_bytes ? workspace_bytes : ((size_t)1 << 30);
    if (c->ws_bytes < kHeaderBytes + 4096) c->ws_bytes = kHeaderBytes + 4096;
    e = cudaMalloc(&c->ws, c->ws_bytes);
    if (e != cudaSuccess) { delete c; cudaGetLastError(); return AIM_ERR_NOMEM; }
    e = cudaMemset(c->ws, 0, kHeaderBytes);
    if (e != cudaSuccess) { cudaFree(c->ws); delete c; return cuda_status(e); }
    c->timing = false;
    c->times[0] = c->times[1] = nullptr;
    c->wfa_group = 0;
    c->tune_cache = nullptr;
    c->adapt_min_len = 10;
    c->adapt_max_dist = 50;
    c->genasm_w = 64;
    c->genasm_o = 24;
    c->batch_compact = 0;
    c->batch_bound = 0;
    c->host_pipe = nullptr;
    *out = c;
    return AIM_OK;
}

int aim_destroy(aim_ctx* ctx) {
    if (!ctx) return AIM_OK;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    aim::free_host_pipe(ctx->host_pipe);
    cudaFree(ctx->ws);
    for (KernelTimes* t : ctx->times) {
        if (!t) continue;
        for (int i = 0; i < kTimedLaunches; ++i) { cudaEventDestroy(t->start[i]); cudaEventDestroy(t->stop[i]); }
        delete t;
    }
    aim::free_tune_cache(ctx->tune_cache);
    delete ctx;
    return cuda_status(e);
}

int aim_wfa_scratch_per_pair(uint32_t max_length, const aim_penalties_t* pen, int32_t max_edits, int lanes,
                             size_t* bytes) {
    if (!bytes || !penalties_ok(pen) || max_length > aim::kMaxWfaLength) return AIM_ERR_ARG;
    if (!(lanes == 0 || lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32 ||
          lanes == 256))
        return AIM_ERR_ARG;
    Resolved r;
    const int rc = resolve(AIM_ALGO_WFA_AFFINE, pen, max_edits, nullptr, &r);
    if (rc) return rc;
    const aim::WfaPlan plan = aim::plan_wfa(r.costs, pen->band, max_length, r.max_limit);
    int g = lanes ? lanes : aim::wfa_default_group(plan, max_length);
    if (max_length > aim::kMaxWfaLength16) g = std::max(g, 32);
    *bytes = aim::wfa_pair_bytes(plan, g);
    return AIM_OK;
}

int aim_set_wfa_group(aim_ctx* ctx, int lanes) {
    if (!ctx || !(lanes == 0 || lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32 ||
                  lanes == 256))
        return AIM_ERR_ARG;
    ctx->wfa_group = lanes;
    return AIM_OK;
}

int aim_set_wfa_adaptive(aim_ctx* ctx, int min_length, int max_distance) {
    if (!ctx || min_length < 0 || max_distance < 0) return AIM_ERR_ARG;
    ctx->adapt_min_len = min_length;
    ctx->adapt_max_dist = max_distance;
    return AIM_OK;
}

int aim_set_batch_compact(aim_ctx* ctx, int mode) {
    if (!ctx || mode < 0 || mode > 2) return AIM_ERR_ARG;
    ctx->batch_compact = mode;
    return AIM_OK;
}

int aim_set_batch_bound(aim_ctx* ctx, int mode) {
    if (!ctx || mode < 0 || mode > 2) return AIM_ERR_ARG;
    ctx->batch_bound = mode;
    return AIM_OK;
}

int aim_set_genasm_window(aim_ctx* ctx, int window, int overlap) {
    if (!ctx || window < 1 || window > 64 || overlap < 0 || overlap >= window) return AIM_ERR_ARG;
    ctx->genasm_w = window;
    ctx->genasm_o = overlap;
    return AIM_OK;
}

int aim_stats_reset(aim_ctx* ctx, aim_stream_t stream) {
    if (!ctx) return AIM_ERR_ARG;
    DeviceGuard g(ctx->device);
    return cuda_status(cudaMemsetAsync(stats_of(ctx), 0, aim::kStats * sizeof(uint64_t), (cudaStream_t)stream));
}

int aim_stats_read(aim_ctx* ctx, uint64_t* out) {
    if (!ctx || !out) return AIM_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(cudaMemcpy(out, stats_of(ctx), aim::kStats * sizeof(uint64_t), cudaMemcpyDeviceToHost));
}

int aim_timing_enable(aim_ctx* ctx, int on) {
    if (!ctx) return AIM_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (on) {
        for (KernelTimes*& t : ctx->times) {
            if (t) continue;
            t = new (std::nothrow) KernelTimes();
            if (!t) return AIM_ERR_NOMEM;
            for (int i = 0; i < kTimedLaunches; ++i) {
                cudaError_t e1 = cudaEventCreate(&t->start[i]);
                cudaError_t e2 = cudaEventCreate(&t->stop[i]);
                if (e1 != cudaSuccess || e2 != cudaSuccess) return cuda_status(e1 != cudaSuccess ? e1 : e2);
            }
            t->recorded = t->launches = 0;
        }
    }
    ctx->timing = on != 0;
    return AIM_OK;
}

int aim_timing_read(aim_ctx* ctx, int kind, double* total_ms, int* launches) {
    if (!ctx || kind < 0 || kind > 1 || !total_ms || !launches) return AIM_ERR_ARG;
    *total_ms = 0.0; *launches = 0;
    KernelTimes* t = ctx->times[kind];
    if (!t) return AIM_OK;
    DeviceGuard g(ctx->device);
    double sum = 0.0;
    for (int i = 0; i < t->recorded; ++i) {
        cudaError_t e = cudaEventSynchronize(t->stop[i]);
        if (e != cudaSuccess) return cuda_status(e);
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, t->start[i], t->stop[i]);
        if (e != cudaSuccess) return cuda_status(e);
        sum += ms;
    }
    *total_ms = sum;
    *launches = t->launches;
    t->recorded = t->launches = 0;
    return AIM_OK;
}

int aim_pack_2bit(aim_ctx* ctx, const uint8_t* ascii, const uint64_t* char_offsets, const uint32_t* lengths,
                  uint32_t count, uint64_t* packed, const uint64_t* word_offsets, uint8_t* bad,
                  aim_stream_t stream) {
    aim::Range range("aim_pack_2bit");
    if (!ctx) return AIM_ERR_ARG;
    if (count == 0) return AIM_OK;
    if (!ascii || !char_offsets || !lengths || !packed || !word_offsets) return AIM_ERR_ARG;
    DeviceGuard g(ctx->device);
    const int slot = time_begin(ctx, 0, (cudaStream_t)stream);
    const cudaError_t e = aim::launch_pack(ascii, char_offsets, lengths, count, packed, word_offsets, 0, bad,
                                           (cudaStream_t)stream);
    time_end(ctx, 0, slot, (cudaStream_t)stream);
    return cuda_status(e);
}

int aim_align_batch(aim_ctx* ctx, const uint64_t* packed_reads, const uint64_t* packed_targets,
                    const uint64_t* read_offsets, const uint64_t* target_offsets, const uint32_t* read_lengths,
                    const uint32_t* target_lengths, uint32_t num_pairs, uint32_t max_length, int algo,
                    const aim_penalties_t* pen, int32_t max_edits, const int32_t* max_edits_per_pair,
                    int32_t* out_scores, uint32_t* out_cigars, const uint64_t* cigar_offsets,
                    uint32_t* out_cigar_lens, uint8_t* out_flags, aim_stream_t stream) {
    aim::Range range("aim_align_batch");
    if (!common_args_ok(ctx, read_lengths, target_lengths, num_pairs, algo, pen, out_scores, out_cigars,
                        cigar_offsets, out_flags))
        return AIM_ERR_ARG;
    if (num_pairs == 0) return AIM_OK;
    if (!packed_reads || !packed_targets || !read_offsets || !target_offsets) return AIM_ERR_ARG;
    DeviceGuard g(ctx->device);
    aim::PairsView P{packed_reads, packed_targets, read_offsets, target_offsets, read_lengths, target_lengths,
                     nullptr, nullptr, num_pairs, max_length};
    aim::OutView O{out_scores, out_cigars, cigar_offsets, out_cigar_lens, out_flags, stats_of(ctx)};
    return align_packed(ctx, P, algo, pen, max_edits, max_edits_per_pair, O, (cudaStream_t)stream,
                        ctx->ws + kHeaderBytes, ctx->ws_bytes - kHeaderBytes);
}

int aim_align_batch_ascii(aim_ctx* ctx, const uint8_t* reads, const uint8_t* targets,
                          const uint64_t* read_char_offsets, const uint64_t* target_char_offsets,
                          const uint32_t* read_lengths, const uint32_t* target_lengths, uint32_t num_pairs,
                          uint32_t max_length, int algo, const aim_penalties_t* pen, int32_t max_edits,
                          const int32_t* max_edits_per_pair, int32_t* out_scores, uint32_t* out_cigars,
                          const uint64_t* cigar_offsets, uint32_t* out_cigar_lens, uint8_t* out_flags,
                          aim_stream_t stream) {
    aim::Range range("aim_align_batch_ascii");
    if (!common_args_ok(ctx, read_lengths, target_lengths, num_pairs, algo, pen, out_scores, out_cigars,
                        cigar_offsets, out_flags))
        return AIM_ERR_ARG;
    if (num_pairs == 0) return AIM_OK;
    if (!reads || !targets || !read_char_offsets || !target_char_offsets) return AIM_ERR_ARG;
    DeviceGuard g(ctx->device);
    // workspace: [header][packed reads][packed targets][bad reads][bad targets][scratch]
    const uint64_t stride = ((uint64_t)max_length + 31) / 32;
    const size_t seq_bytes = aim::align_up((size_t)num_pairs * stride * 8, 256);
    const size_t bad_bytes = aim::align_up(num_pairs, 256);
    const size_t used = kHeaderBytes + 2 * seq_bytes + 2 * bad_bytes;
    if (used >= ctx->ws_bytes) return AIM_ERR_NOMEM;
    uint8_t* base = ctx->ws + kHeaderBytes;
    uint64_t* pr = reinterpret_cast<uint64_t*>(base);
    uint64_t* pt = reinterpret_cast<uint64_t*>(base + seq_bytes);
    uint8_t* br = base + 2 * seq_bytes;
    uint8_t* bt = br + bad_bytes;
    cudaStream_t st = (cudaStream_t)stream;
    int slot = time_begin(ctx, 0, st);
    cudaError_t e = aim::launch_pack(reads, read_char_offsets, read_lengths, num_pairs, pr, nullptr, stride, br, st);
    time_end(ctx, 0, slot, st);
    if (e != cudaSuccess) return cuda_status(e);
    slot = time_begin(ctx, 0, st);
    e = aim::launch_pack(targets, target_char_offsets, target_lengths, num_pairs, pt, nullptr, stride, bt, st);
    time_end(ctx, 0, slot, st);
    if (e != cudaSuccess) return cuda_status(e);
    // word offsets i * stride are implied: pass a null offset array through a small view
    aim::PairsView P{pr, pt, nullptr, nullptr, read_lengths, target_lengths, br, bt, num_pairs, max_length};
    P.stride = stride;
    aim::OutView O{out_scores, out_cigars, cigar_offsets, out_cigar_lens, out_flags, stats_of(ctx)};
    return align_packed(ctx, P, algo, pen, max_edits, max_edits_per_pair, O, st, ctx->ws + used,
                        ctx->ws_bytes - used);
}

}  // extern "C"
