// Serving loop: requests of different sizes arrive over time and are aligned
// with continuous batching on one GPU.
//
// A request (host buffers: ASCII pairs, per-pair thresholds, outputs) is
// copied at submission and queued.  A worker thread admits queued requests in
// arrival order as soon as three fixed arenas have room for them:
//   - pinned host staging (inputs out, results back),
//   - device I/O (sequences, packed words, lengths, thresholds, results),
//   - device wavefront scratch: the memory budget for wavefront state,
// and enough streams are free for it.  At submission a request's pairs are
// grouped into jobs by the bound on their wavefront work (the bucket rule of
// the batched form), heaviest first; each job gets its own plan, lanes per
// pair and scratch per warp, so short pairs do not pay for the scratch of the
// longest one.  An admitted request receives one scratch grant (what its jobs
// want, capped at 1/16 of the budget so that many requests share the device
// at once, never less than one block of scratch for each of its jobs), split
// between its jobs; a request whose heaviest pair would not fit even an empty
// budget is refused at submission.  An admitted request holds its own streams:
// one for the H2D copy and the 2-bit packing, then one per job (one WFA launch
// each, on its slice of the grant), joined again for the copy back, so the
// jobs of one request and the work of requests that arrive while others run
// overlap on the device without waiting behind each other; wavefront state
// never leaves the device.  A host function enqueued behind the request's work
// stamps its completion time and wakes the worker, which copies results to
// the caller's buffers, releases the arenas and streams (admitting waiting
// requests) and marks the ticket done.  Each pair is aligned independently
// and deterministically, so a request's results are the same alone and in any
// mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "aim_internal.cuh"
#include "ranges.h"

namespace aim {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit sub-allocator over [0, size) with coalescing; offsets are 256-byte aligned.
class Arena {
public:
    explicit Arena(size_t size = 0) { reset(size); }
    void reset(size_t size) {
        free_.clear();
        size_ = size;
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align_up(std::max<size_t>(bytes, 1), 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(std::max<size_t>(bytes, 1), 256);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }
    size_t largest() const {
        size_t m = 0;
        for (auto& kv : free_) m = std::max(m, kv.second);
        return m;
    }
    size_t size() const { return size_; }

private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0;
};

struct Request {
    uint64_t ticket;
    uint32_t n;
    uint32_t max_len;
    int32_t max_edits_bound;
    // host copies of the inputs (byte layout of the device I/O region)
    std::vector<uint8_t> reads, targets;
    std::vector<uint64_t> roff, toff, coff;
    std::vector<uint32_t> rl, tl;
    std::vector<int32_t> me;
    std::vector<uint32_t> order;     // pair indices grouped into jobs (heaviest job first)
    struct Job {
        uint32_t begin, count;
        WfaPlan plan;
        int group;
        int bound_group;     // lanes per pair of a bound pass before the exact one (0: none)
        size_t warp_bytes;
        size_t warps;        // wanted
        size_t slice_off, slice_bytes;   // its part of the request's scratch grant
    };
    std::vector<Job> jobs;
    // caller's output buffers
    int32_t* out_scores;
    uint8_t* out_flags;
    uint32_t* out_lens;
    uint32_t* out_cigars;
    uint64_t cigar_total;
    // planning
    size_t io_bytes, scratch_bytes, scratch_min, scratch_want;
    // resources while admitted
    size_t io_off, host_off, scratch_off;
    cudaStream_t stream;
    std::vector<cudaStream_t> job_streams;
    std::vector<cudaEvent_t> events;    // [0]: inputs ready; [1 + j]: job j done
    Clock::time_point t_submit, t_done;
    bool done;
    int status;
};

// Byte layout of one request inside the device I/O region (and its pinned staging twin).
struct IoLayout {
    size_t reads, targets, roff, toff, rl, tl, me, coff, order, packed_r, packed_t, bad_r, bad_t, counter, bound, scores,
        flags, lens, cigars, total, in_bytes;
    uint64_t stride;
};

IoLayout layout_of(const Request& r) {
    IoLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + std::max<size_t>(bytes, 1), 256); return at; };
    L.stride = ((uint64_t)r.max_len + 31) / 32;
    // inputs first, contiguous, so one H2D copy moves them
    L.reads = take(r.reads.size());
    L.targets = take(r.targets.size());
    L.roff = take(r.n * 8);
    L.toff = take(r.n * 8);
    L.rl = take(r.n * 4);
    L.tl = take(r.n * 4);
    L.me = take(r.n * 4);
    L.coff = take((r.n + 1) * 8);
    L.order = take(r.n * 4);
    L.in_bytes = o;
    // results next, contiguous, so one D2H copy moves them
    L.scores = take(r.n * 4);
    L.flags = take(r.n);
    L.lens = take(r.n * 4);
    L.cigars = take(r.cigar_total * 4);
    const size_t out_end = o;
    L.packed_r = take((size_t)r.n * L.stride * 8);
    L.packed_t = take((size_t)r.n * L.stride * 8);
    L.bad_r = take(r.n);
    L.bad_t = take(r.n);
    L.counter = take(64 * sizeof(uint32_t));   // per job: the exact pass's claim counter, then the bound pass's
    L.bound = take(r.n * 4);                    // per pair: the bound pass's score bound
    L.total = o;
    (void)out_end;
    return L;
}

}  // namespace
}  // namespace aim

struct aim_server {
    aim_ctx* ctx;
    aim::Costs costs;
    aim_penalties_t pen;
    int num_sms;
    int warps_cap;
    uint8_t* dev_io;
    uint8_t* dev_scratch;
    uint8_t* host_stage;
    aim::Arena io, scratch, stage;
    std::vector<cudaStream_t> streams;
    std::vector<cudaStream_t> free_streams;
    size_t next_stream;
    std::vector<cudaEvent_t> event_pool;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<aim::Request*> queue;
    std::vector<aim::Request*> running;
    std::deque<aim::Request*> completed;   // filled by stream callbacks
    std::unordered_map<uint64_t, std::unique_ptr<aim::Request>> tickets;
    uint64_t next_ticket;
    bool stop;
    bool paused;                // admit nothing while set
    uint32_t inject_countdown;  // > 0: the request admitted when it reaches 0 fails at launch (tests)
    std::thread worker;
    uint64_t n_submitted, n_completed, pairs_completed, n_failed;
};

namespace aim {
namespace {

void CUDART_CB on_request_done(void* arg) {
    auto* pair = static_cast<std::pair<aim_server*, Request*>*>(arg);
    aim_server* s = pair->first;
    Request* r = pair->second;
    delete pair;
    r->t_done = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->completed.push_back(r);
    }
    s->cv_work.notify_one();
}

// Try to place the request in the three arenas; called with the lock held.
bool try_admit(aim_server* s, Request* r) {
    size_t io_off, host_off, scr_off;
    if (!s->io.alloc(r->io_bytes, &io_off)) return false;
    const IoLayout L = layout_of(*r);
    if (!s->stage.alloc(L.total, &host_off)) { s->io.release(io_off, r->io_bytes); return false; }
    // one scratch grant per request, split between its jobs (which run side by side on their own streams):
    // what they want up to 1/16 of the budget (so that many requests share the device at once), never less
    // than one block of scratch for each job
    const size_t cap = std::max(r->scratch_min, s->scratch.size() / 16);
    const size_t grant = std::min(std::min(r->scratch_want, cap), s->scratch.largest());
    if (grant < r->scratch_min || !s->scratch.alloc(grant, &scr_off)) {
        s->io.release(io_off, r->io_bytes);
        s->stage.release(host_off, L.total);
        return false;
    }
    size_t extra_want = 0;
    for (auto& j : r->jobs) extra_want += align_up(j.warps * j.warp_bytes, 256) - align_up(8 * j.warp_bytes, 256);
    const size_t extra = grant - r->scratch_min;
    size_t at = 0;
    for (auto& j : r->jobs) {
        const size_t lo = align_up(8 * j.warp_bytes, 256);
        const size_t more = align_up(j.warps * j.warp_bytes, 256) - lo;
        size_t give = extra_want ? (size_t)((double)extra * ((double)more / (double)extra_want)) : 0;
        give = give / 256 * 256;
        j.slice_off = at;
        j.slice_bytes = lo + give;
        at += j.slice_bytes;
    }
    r->io_off = io_off; r->host_off = host_off; r->scratch_off = scr_off;
    r->scratch_bytes = grant;
    return true;
}

void release(aim_server* s, Request* r) {
    for (cudaEvent_t ev : r->events) if (ev) s->event_pool.push_back(ev);
    r->events.clear();
    if (r->stream) s->free_streams.push_back(r->stream);
    for (cudaStream_t js : r->job_streams) s->free_streams.push_back(js);
    r->stream = nullptr;
    r->job_streams.clear();
    const IoLayout L = layout_of(*r);
    s->io.release(r->io_off, r->io_bytes);
    s->stage.release(r->host_off, L.total);
    s->scratch.release(r->scratch_off, r->scratch_bytes);
}

// Enqueue the request's work on its stream (no lock needed: its arena ranges are its own).
int launch_request(aim_server* s, Request* r) {
    aim::Range range("aim_server_launch");
    const IoLayout L = layout_of(*r);
    uint8_t* h = s->host_stage + r->host_off;
    uint8_t* d = s->dev_io + r->io_off;
    std::memcpy(h + L.reads, r->reads.data(), r->reads.size());
    std::memcpy(h + L.targets, r->targets.data(), r->targets.size());
    std::memcpy(h + L.roff, r->roff.data(), r->n * 8);
    std::memcpy(h + L.toff, r->toff.data(), r->n * 8);
    std::memcpy(h + L.rl, r->rl.data(), r->n * 4);
    std::memcpy(h + L.tl, r->tl.data(), r->n * 4);
    std::memcpy(h + L.me, r->me.data(), r->n * 4);
    std::memcpy(h + L.coff, r->coff.data(), (r->n + 1) * 8);
    std::memcpy(h + L.order, r->order.data(), r->n * 4);
    cudaStream_t st = r->stream;
    cudaError_t e = cudaMemcpyAsync(d, h, L.in_bytes, cudaMemcpyHostToDevice, st);
    // the whole CIGAR region is copied back: runs past each pair's count read as zero, not as an earlier request's
    if (e == cudaSuccess)
        e = launch_pack(d + L.reads, reinterpret_cast<const uint64_t*>(d + L.roff),
                        reinterpret_cast<const uint32_t*>(d + L.rl), r->n, reinterpret_cast<uint64_t*>(d + L.packed_r),
                        nullptr, L.stride, d + L.bad_r, st);
    if (e == cudaSuccess)
        e = launch_pack(d + L.targets, reinterpret_cast<const uint64_t*>(d + L.toff),
                        reinterpret_cast<const uint32_t*>(d + L.tl), r->n, reinterpret_cast<uint64_t*>(d + L.packed_t),
                        nullptr, L.stride, d + L.bad_t, st);
    LimitView lim;
    lim.per_pair = reinterpret_cast<const int32_t*>(d + L.me);
    lim.max_edits_bound = r->max_edits_bound;
    lim.edit_cost = std::max(s->costs.x, s->costs.o + s->costs.e);
    lim.limit = (int64_t)r->max_edits_bound * lim.edit_cost;
    OutView O{reinterpret_cast<int32_t*>(d + L.scores),
              r->out_cigars ? reinterpret_cast<uint32_t*>(d + L.cigars) : nullptr,
              r->out_cigars ? reinterpret_cast<const uint64_t*>(d + L.coff) : nullptr,
              reinterpret_cast<uint32_t*>(d + L.lens), d + L.flags, stats_of(s->ctx)};
    const uint32_t* order = reinterpret_cast<const uint32_t*>(d + L.order);
    if (e == cudaSuccess) e = cudaEventRecord(r->events[0], st);
    for (size_t j = 0; j < r->jobs.size() && e == cudaSuccess; ++j) {
        const Request::Job& job = r->jobs[j];
        cudaStream_t js = r->job_streams[j];
        uint32_t* counter = reinterpret_cast<uint32_t*>(d + L.counter) + j % 32;
        e = cudaStreamWaitEvent(js, r->events[0], 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), js);
        if (e == cudaSuccess && job.bound_group) e = cudaMemsetAsync(counter + 32, 0, sizeof(uint32_t), js);
        if (e != cudaSuccess) break;
        PairsView P{reinterpret_cast<const uint64_t*>(d + L.packed_r), reinterpret_cast<const uint64_t*>(d + L.packed_t),
                    nullptr, nullptr, reinterpret_cast<const uint32_t*>(d + L.rl),
                    reinterpret_cast<const uint32_t*>(d + L.tl), d + L.bad_r, d + L.bad_t, job.count, r->max_len};
        P.stride = L.stride;
        uint8_t* slice = s->dev_scratch + r->scratch_off + job.slice_off;
        WfaPlan exact = job.plan;
        int warps = 0;
        if (job.bound_group) {
            // a bound pass in the job's scratch slice first (the exact pass then reuses the slice); if not one
            // block of it fits, the exact pass runs alone
            WfaPlan bp = job.plan;
            bp.bound = reinterpret_cast<int32_t*>(d + L.bound);
            bp.bound_pass = 1;
            int bg = job.bound_group;
            const size_t bwb = wfa_warp_bytes(bg, wfa_bound_pair_bytes(job.plan));
            if (8 * bwb <= job.slice_bytes) {
                e = launch_wfa_buckets(bp, P, lim, O, order + job.begin, nullptr, &bg, 1, bwb, slice, job.slice_bytes,
                                       counter + 32, s->num_sms, js, &warps);
                if (e == cudaSuccess && warps > 0) exact.bound = bp.bound;
            }
            if (e != cudaSuccess) break;
        }
        e = launch_wfa_buckets(exact, P, lim, O, order + job.begin, nullptr, &job.group, 1, job.warp_bytes, slice,
                               job.slice_bytes, counter, s->num_sms, js, &warps);
        if (e == cudaSuccess && warps == 0) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaEventRecord(r->events[1 + j], js);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, r->events[1 + j], 0);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h + L.scores, d + L.scores, L.cigars + r->cigar_total * 4 - L.scores,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) {
        auto* arg = new (std::nothrow) std::pair<aim_server*, Request*>(s, r);
        e = arg ? cudaLaunchHostFunc(st, on_request_done, arg) : cudaErrorMemoryAllocation;
    }
    return e == cudaSuccess ? AIM_OK : cuda_status(e);
}

void finish(aim_server* s, Request* r) {
    aim::Range range("aim_server_finish");
    const IoLayout L = layout_of(*r);
    const uint8_t* h = s->host_stage + r->host_off;
    std::memcpy(r->out_scores, h + L.scores, r->n * 4);
    std::memcpy(r->out_flags, h + L.flags, r->n);
    if (r->out_lens) std::memcpy(r->out_lens, h + L.lens, r->n * 4);
    if (r->out_cigars) {
        // each pair's runs only (a few hundred bytes), not the request's whole run capacity: the worker thread that
        // does this also admits and completes the other requests
        const uint32_t* lens = reinterpret_cast<const uint32_t*>(h + L.lens);
        const uint32_t* runs = reinterpret_cast<const uint32_t*>(h + L.cigars);
        for (uint32_t i = 0; i < r->n; ++i) {
            const uint64_t at = r->coff[i], cap = r->coff[i + 1] - at;
            const uint64_t cnt = std::min<uint64_t>(lens[i], cap);
            if (cnt) std::memcpy(r->out_cigars + at, runs + at, cnt * 4);
        }
    }
}

void worker_loop(aim_server* s) {
    DeviceGuardImpl guard(s->ctx->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        // completions: results out, arenas back
        while (!s->completed.empty()) {
            Request* r = s->completed.front();
            s->completed.pop_front();
            lock.unlock();
            finish(s, r);
            lock.lock();
            release(s, r);
            s->running.erase(std::find(s->running.begin(), s->running.end(), r));
            r->done = true;
            ++s->n_completed;
            s->pairs_completed += r->n;
            s->cv_done.notify_all();
        }
        // admissions, in arrival order
        while (!s->paused && !s->queue.empty()) {
            Request* r = s->queue.front();
            if (s->free_streams.size() < r->jobs.size() + 1) break;   // a request holds its own streams
            if (!try_admit(s, r)) break;
            s->queue.pop_front();
            r->stream = s->free_streams.back();
            s->free_streams.pop_back();
            r->job_streams.clear();
            for (size_t j = 0; j < r->jobs.size(); ++j) {
                r->job_streams.push_back(s->free_streams.back());
                s->free_streams.pop_back();
            }
            r->events.clear();
            for (size_t j = 0; j <= r->jobs.size(); ++j) {
                cudaEvent_t ev = nullptr;
                if (!s->event_pool.empty()) { ev = s->event_pool.back(); s->event_pool.pop_back(); }
                else cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
                r->events.push_back(ev);
            }
            s->running.push_back(r);
            const bool injected = s->inject_countdown > 0 && --s->inject_countdown == 0;
            lock.unlock();
            const int rc = injected ? AIM_ERR_CUDA : launch_request(s, r);
            lock.lock();
            if (rc != AIM_OK) {   // the request fails as a whole; its ticket completes with an error status
                lock.unlock();
                cudaStreamSynchronize(r->stream);   // work enqueued before the failure drains first
                lock.lock();
                r->status = rc;
                r->t_done = Clock::now();
                ++s->n_failed;
                release(s, r);
                s->running.erase(std::find(s->running.begin(), s->running.end(), r));
                r->done = true;
                ++s->n_completed;
                s->cv_done.notify_all();
            }
        }
        if (s->stop && s->queue.empty() && s->running.empty()) break;
        s->cv_work.wait_for(lock, std::chrono::milliseconds(5));
    }
}

}  // namespace
}  // namespace aim

extern "C" {

int aim_server_create(aim_ctx* ctx, const aim_penalties_t* pen, size_t wavefront_budget_bytes, size_t io_budget_bytes,
                      aim_server** out) {
    using namespace aim;
    if (!out) return AIM_ERR_ARG;
    *out = nullptr;
    if (!ctx || !pen || pen->match != 0 || pen->mismatch < 1 || pen->gap_open < 0 || pen->gap_extend < 1 ||
        pen->max_score >= 0)
        return AIM_ERR_ARG;
    DeviceGuardImpl guard(ctx->device);
    aim_server* s = new (std::nothrow) aim_server();
    if (!s) return AIM_ERR_NOMEM;
    s->ctx = ctx;
    s->pen = *pen;
    s->costs = Costs{pen->mismatch, pen->gap_open, pen->gap_extend};
    s->num_sms = ctx->num_sms;
    s->warps_cap = ctx->num_sms * 32;
    s->next_stream = 0; s->next_ticket = 1; s->stop = false; s->paused = false; s->inject_countdown = 0;
    s->n_submitted = s->n_completed = s->pairs_completed = s->n_failed = 0;
    if (!wavefront_budget_bytes) wavefront_budget_bytes = (size_t)4 << 30;
    if (!io_budget_bytes) io_budget_bytes = (size_t)1 << 30;
    cudaError_t e = cudaMalloc(&s->dev_scratch, wavefront_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->dev_io, io_budget_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&s->host_stage, io_budget_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (s->dev_scratch) cudaFree(s->dev_scratch);
        if (s->dev_io) cudaFree(s->dev_io);
        delete s;
        return AIM_ERR_NOMEM;
    }
    s->scratch.reset(wavefront_budget_bytes);
    s->io.reset(io_budget_bytes);
    s->stage.reset(io_budget_bytes);
    for (int i = 0; i < 128; ++i) {   // requests and their jobs spread over 128 streams
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) s->streams.push_back(st);
    }
    s->free_streams = s->streams;
    if (s->streams.empty()) { cudaFree(s->dev_scratch); cudaFree(s->dev_io); cudaFreeHost(s->host_stage); delete s;
                              return AIM_ERR_CUDA; }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return AIM_OK;
}

int aim_server_submit(aim_server* s, const aim_request* q, uint64_t* ticket) {
    aim::Range range("aim_server_submit");
    using namespace aim;
    if (!s || !q || !ticket) return AIM_ERR_ARG;
    *ticket = 0;
    if (q->num_pairs == 0 || !q->reads || !q->targets || !q->read_offsets || !q->target_offsets ||
        !q->read_lengths || !q->target_lengths || !q->out_scores || !q->out_flags ||
        ((q->out_cigars == nullptr) != (q->cigar_offsets == nullptr)))
        return AIM_ERR_ARG;
    auto r = std::make_unique<Request>();
    const uint32_t n = q->num_pairs;
    r->n = n;
    r->max_len = 1;
    uint64_t rb = 0, tb = 0;
    for (uint32_t i = 0; i < n; ++i) {
        r->max_len = std::max(r->max_len, std::max(q->read_lengths[i], q->target_lengths[i]));
        rb += q->read_lengths[i];
        tb += q->target_lengths[i];
    }
    if (r->max_len > kMaxWfaLength) return AIM_ERR_UNSUPPORTED;
    // sequences repacked back to back
    r->reads.resize(rb); r->targets.resize(tb);
    r->roff.resize(n); r->toff.resize(n); r->rl.assign(q->read_lengths, q->read_lengths + n);
    r->tl.assign(q->target_lengths, q->target_lengths + n);
    r->me.resize(n);
    uint64_t a = 0, b = 0;
    int32_t bound = 0;
    for (uint32_t i = 0; i < n; ++i) {
        std::memcpy(r->reads.data() + a, q->reads + q->read_offsets[i], q->read_lengths[i]);
        std::memcpy(r->targets.data() + b, q->targets + q->target_offsets[i], q->target_lengths[i]);
        r->roff[i] = a; r->toff[i] = b;
        a += q->read_lengths[i]; b += q->target_lengths[i];
        r->me[i] = q->max_edits ? q->max_edits[i] : q->max_edits_all;
        if (r->me[i] < 0) return AIM_ERR_ARG;   // the server needs a threshold to bound wavefront state
        bound = std::max(bound, r->me[i]);
    }
    r->max_edits_bound = bound;
    r->coff.resize(n + 1);
    r->coff[0] = 0;
    for (uint32_t i = 0; i < n; ++i)
        r->coff[i + 1] = r->coff[i] + (q->cigar_offsets ? q->cigar_offsets[i + 1] - q->cigar_offsets[i] : 0);
    r->cigar_total = r->coff[n];
    r->out_scores = q->out_scores; r->out_flags = q->out_flags; r->out_lens = q->out_cigar_lens;
    r->out_cigars = q->out_cigars;
    // jobs: pairs grouped by the bound on their wavefront work (the rule of the batched form), heaviest first;
    // each job has its own plan, lanes per pair and scratch per warp
    const int32_t ecost = std::max(s->costs.x, s->costs.o + s->costs.e);
    WfaPlan probe = plan_wfa(s->costs, s->pen.band, 1, 0);
    std::vector<std::pair<int, uint32_t>> keyed(n);
    for (uint32_t i = 0; i < n; ++i) {
        const int64_t nn = r->rl[i], mm = r->tl[i];
        int64_t S = (int64_t)r->me[i] * ecost / probe.g;
        int64_t W = 2 * (S / std::max(probe.e, 1)) + 3;
        W = std::min(W, nn + mm + 1);
        if (s->pen.band >= 0) W = std::min<int64_t>(W, 2 * (int64_t)s->pen.band + 1);
        const uint64_t C = (uint64_t)(S + 1) * (uint64_t)W;
        int lg = 63;
        while (lg > 0 && !((C + 1) >> lg)) --lg;
        const int kc = std::min(7, lg / 3);
        const int wc = W <= 64 ? 0 : W <= 128 ? 1 : W <= 256 ? 2 : 3;
        keyed[i] = {(7 - kc) * 4 + (3 - wc), i};
    }
    std::stable_sort(keyed.begin(), keyed.end());
    r->order.resize(n);
    for (uint32_t i = 0; i < n; ++i) r->order[i] = keyed[i].second;
    r->scratch_min = 0;
    r->scratch_want = 0;
    for (uint32_t i = 0; i < n;) {
        uint32_t j = i;
        uint32_t jl = 1;
        int32_t jme = 0;
        while (j < n && keyed[j].first == keyed[i].first) {
            const uint32_t p = keyed[j].second;
            jl = std::max(jl, std::max(r->rl[p], r->tl[p]));
            jme = std::max(jme, r->me[p]);
            ++j;
        }
        Request::Job job;
        job.begin = i; job.count = j - i;
        job.plan = plan_wfa(s->costs, s->pen.band, jl, (int64_t)jme * ecost);
        job.group = wfa_default_group(job.plan, jl);
        job.warp_bytes = wfa_warp_bytes(job.group, wfa_pair_bytes(job.plan, job.group));
        if (job.warp_bytes > s->scratch.size() / 64 && job.group < 32) {   // one pair per warp when scratch is scarce
            job.group = 32;
            job.warp_bytes = wfa_pair_bytes(job.plan, 32);
        }
        // a bound pass before the exact one for the heaviest classes (work class >= 5, wavefronts over 256
        // diagonals), where the batched form's tuner keeps one: 4 lanes per pair before groups of up to 32 lanes,
        // 16 before whole blocks.  Results are the exact pass's either way.
        const int key = keyed[i].first, kc = 7 - key / 4, wc = 3 - key % 4;
        job.bound_group = kc >= 5 && wc == 3 && r->max_len <= kMaxWfaLength16 ? (job.group > 32 ? 16 : 4) : 0;
        // warps wanted: every pair in flight at once (a 256-lane group uses 8 warps), within the device's capacity
        const size_t want = job.group > 32 ? (size_t)job.count * (job.group / 32)
                                           : (job.count + (32 / job.group) - 1) / (size_t)(32 / job.group);
        job.warps = std::min<size_t>((want + 7) / 8 * 8, (size_t)s->warps_cap);
        r->scratch_min += align_up(8 * job.warp_bytes, 256);   // launches use whole blocks
        r->scratch_want += align_up(job.warps * job.warp_bytes, 256);
        r->jobs.push_back(job);
        i = j;
    }
    if (r->jobs.size() > 32 || r->jobs.size() + 1 > s->streams.size()) return AIM_ERR_UNSUPPORTED;
    r->io_bytes = layout_of(*r).total;
    if (r->scratch_min > s->scratch.size() || r->io_bytes > s->io.size()) return AIM_ERR_NOMEM;
    r->done = false;
    r->status = AIM_OK;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return AIM_ERR_ARG;
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->tickets[r->ticket] = std::move(r);
    ++s->n_submitted;
    s->cv_work.notify_one();
    return AIM_OK;
}

int aim_server_poll(aim_server* s, uint64_t ticket, int* done, uint64_t* latency_ns) {
    if (!s || !done) return AIM_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return AIM_ERR_ARG;
    aim::Request* r = it->second.get();
    *done = r->done ? 1 : 0;
    if (r->done) {
        if (latency_ns)
            *latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(r->t_done - r->t_submit).count();
        const int st = r->status;
        s->tickets.erase(it);
        return st;
    }
    return AIM_OK;
}

int aim_server_wait(aim_server* s, uint64_t ticket, uint64_t* latency_ns) {
    if (!s) return AIM_ERR_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return AIM_ERR_ARG;
    aim::Request* r = it->second.get();
    s->cv_done.wait(lock, [&] { return r->done; });
    if (latency_ns)
        *latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(r->t_done - r->t_submit).count();
    const int st = r->status;
    s->tickets.erase(it);
    return st;
}

int aim_server_stats(aim_server* s, uint64_t* out) {
    if (!s || !out) return AIM_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    out[0] = s->n_submitted; out[1] = s->n_completed; out[2] = s->pairs_completed; out[3] = s->n_failed;
    out[4] = s->queue.size(); out[5] = s->running.size();
    return AIM_OK;
}

int aim_server_pause(aim_server* s, int paused) {
    if (!s || (paused != 0 && paused != 1)) return AIM_ERR_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->paused = paused != 0;
    }
    s->cv_work.notify_one();
    return AIM_OK;
}

int aim_server_cancel(aim_server* s, uint64_t ticket) {
    if (!s) return AIM_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return AIM_ERR_ARG;
    aim::Request* r = it->second.get();
    auto q = std::find(s->queue.begin(), s->queue.end(), r);
    if (q == s->queue.end()) return AIM_ERR_BUSY;   // admitted (running or done): it completes as usual
    s->queue.erase(q);
    r->status = AIM_ERR_CANCELLED;
    r->t_done = aim::Clock::now();
    r->done = true;
    ++s->n_completed;
    ++s->n_failed;
    s->cv_done.notify_all();
    s->cv_work.notify_one();   // the requests behind it may fit now
    return AIM_OK;
}

int aim_server_inject_failure(aim_server* s, uint32_t countdown) {
    if (!s) return AIM_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    s->inject_countdown = countdown;
    return AIM_OK;
}

int aim_server_destroy(aim_server* s) {
    if (!s) return AIM_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->paused = false;   // everything queued is finished
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    aim::DeviceGuardImpl guard(s->ctx->device);
    for (cudaStream_t st : s->streams) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    for (cudaEvent_t ev : s->event_pool) cudaEventDestroy(ev);
    cudaFree(s->dev_scratch);
    cudaFree(s->dev_io);
    cudaFreeHost(s->host_stage);
    delete s;
    return AIM_OK;
}

}  // extern "C"
