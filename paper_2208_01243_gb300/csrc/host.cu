// aim_align_batch_host: the whole batch from host memory to host memory in
// one call, with the transfers inside it (the paper's timed region runs from
// the parallel transfer of the pairs to the memory banks, through alignment
// and traceback, to the transfer of scores and operations back: Section 2.2,
// Steps 2-6, and Section 3.1).
//
// The batch is cut into chunks of C pairs, aligned through two device slots
// in turn.  Each slot holds device copies of one chunk's inputs (ASCII bytes,
// offsets rebased to the chunk, lengths, thresholds, CIGAR offsets) and
// outputs.  A copy-in stream, a copy-out stream and one compute stream per
// slot form the pipeline: while chunk j aligns in one slot, the copy-in
// stream fills the other slot with chunk j + 1 and the copy-out stream
// returns chunk j - 1's results, so the copy engines work beside the SMs, and
// chunk j + 1's launches start while the last long pairs of chunk j finish.
// Events order each slot's reuse: new inputs only once the slot's previous
// alignment has read its inputs, and a new alignment only once the slot's
// previous results have left.
//
// The wavefront algorithm runs in the batched form: each slot owns a batch
// plan (bucketed queues, lanes per pair from the context's autotuner, CUDA
// graph) bound to its buffers, planned on the first chunk it holds and then
// replayed with each new chunk's contents; a short last chunk is padded with
// empty pairs.  Each plan draws its scratch from its own half of the context
// workspace, so the two slots' launches may overlap.  The other algorithms run
// the plain ASCII form on each chunk; those share the workspace, so both slots
// then use one compute stream.  Slots, streams and plans stay in the context
// for later calls of the same shape.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "aim_internal.cuh"
#include "ranges.h"

namespace aim {
namespace {

struct Slot {
    // device copies of one chunk
    uint8_t *reads, *targets;
    uint64_t *roff, *toff, *coff;
    uint32_t *rlen, *tlen, *lens, *cigars;
    int32_t *me, *scores;
    uint8_t* flags;
    aim_batch* plan;
    cudaEvent_t in_done, comp_done, out_done;
    bool used;
};

struct HostPipe {
    // shape the slots were built for
    int algo;
    aim_penalties_t pen;
    int32_t max_edits;
    bool per_pair, cigars;
    uint32_t max_length, chunk;
    uint64_t read_cap, target_cap, cigar_cap;   // bytes, bytes, runs per slot
    uint8_t* mem;
    cudaStream_t h2d, d2h, comp[2];   // comp[1] == comp[0] when the slots share the workspace
    Slot slot[2];
};

// A chunk's offsets arrive as the caller wrote them; this rebases them to the chunk's own byte and run ranges and
// fills the padding of a short last chunk (batched form) with empty pairs whose runs start at the chunk's end.
__global__ void __launch_bounds__(256) rebase_kernel(uint64_t* roff, uint64_t* toff, uint64_t* coff, uint32_t* rlen,
                                                     uint32_t* tlen, int32_t* me, uint32_t k, uint32_t padded,
                                                     uint64_t rlo, uint64_t tlo, uint64_t cbase, uint64_t cend,
                                                     int per_pair, int cigars) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= padded; i += gridDim.x * blockDim.x) {
        if (i < k) {
            roff[i] -= rlo;
            toff[i] -= tlo;
            if (cigars) coff[i] -= cbase;
        } else if (i < padded) {
            roff[i] = toff[i] = 0;
            rlen[i] = tlen[i] = 0;
            if (per_pair) me[i] = 0;
            if (cigars) coff[i] = cend;
        } else if (cigars) {
            coff[i] = cend;   // entry `padded`: the end of the last pair's runs
        }
    }
}

void destroy_pipe(HostPipe* hp) {
    if (!hp) return;
    for (cudaStream_t c : hp->comp)
        if (c) cudaStreamSynchronize(c);
    if (hp->h2d) cudaStreamSynchronize(hp->h2d);
    if (hp->d2h) cudaStreamSynchronize(hp->d2h);
    for (Slot& s : hp->slot) {
        if (s.plan) aim_batch_destroy(s.plan);
        if (s.in_done) cudaEventDestroy(s.in_done);
        if (s.comp_done) cudaEventDestroy(s.comp_done);
        if (s.out_done) cudaEventDestroy(s.out_done);
    }
    if (hp->h2d) cudaStreamDestroy(hp->h2d);
    if (hp->comp[0]) cudaStreamDestroy(hp->comp[0]);
    if (hp->comp[1] && hp->comp[1] != hp->comp[0]) cudaStreamDestroy(hp->comp[1]);
    if (hp->d2h) cudaStreamDestroy(hp->d2h);
    if (hp->mem) cudaFree(hp->mem);
    delete hp;
}

bool same_shape(const HostPipe* hp, int algo, const aim_penalties_t* pen, int32_t max_edits, bool per_pair,
                bool cigars, uint32_t max_length, uint32_t chunk, uint64_t rc, uint64_t tc, uint64_t cc) {
    return hp && hp->algo == algo && std::memcmp(&hp->pen, pen, sizeof(*pen)) == 0 && hp->max_edits == max_edits &&
           hp->per_pair == per_pair && hp->cigars == cigars && hp->max_length == max_length && hp->chunk == chunk &&
           hp->read_cap >= rc && hp->target_cap >= tc && hp->cigar_cap >= cc;
}

HostPipe* make_pipe(int algo, const aim_penalties_t* pen, int32_t max_edits, bool per_pair, bool cigars,
                    uint32_t max_length, uint32_t C, uint64_t rc, uint64_t tc, uint64_t cc, cudaError_t* err) {
    HostPipe* hp = new (std::nothrow) HostPipe();
    if (!hp) { *err = cudaErrorMemoryAllocation; return nullptr; }
    std::memset(hp, 0, sizeof(*hp));
    hp->algo = algo; hp->pen = *pen; hp->max_edits = max_edits; hp->per_pair = per_pair; hp->cigars = cigars;
    hp->max_length = max_length; hp->chunk = C;
    hp->read_cap = std::max<uint64_t>(rc, 1); hp->target_cap = std::max<uint64_t>(tc, 1);
    hp->cigar_cap = std::max<uint64_t>(cc, 1);
    const size_t a = 256;
    const size_t per_slot = align_up(hp->read_cap, a) + align_up(hp->target_cap, a) +
                            3 * align_up((size_t)C * 8 + 8, a) + 4 * align_up((size_t)C * 4, a) +
                            align_up((size_t)C * 4, a) + align_up(C, a) + align_up(hp->cigar_cap * 4, a);
    cudaError_t e = cudaMalloc(&hp->mem, 2 * per_slot);
    uint8_t* p = hp->mem;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        Slot& s = hp->slot[k];
        s.reads = p; p += align_up(hp->read_cap, a);
        s.targets = p; p += align_up(hp->target_cap, a);
        s.roff = reinterpret_cast<uint64_t*>(p); p += align_up((size_t)C * 8 + 8, a);
        s.toff = reinterpret_cast<uint64_t*>(p); p += align_up((size_t)C * 8 + 8, a);
        s.coff = reinterpret_cast<uint64_t*>(p); p += align_up((size_t)C * 8 + 8, a);
        s.rlen = reinterpret_cast<uint32_t*>(p); p += align_up((size_t)C * 4, a);
        s.tlen = reinterpret_cast<uint32_t*>(p); p += align_up((size_t)C * 4, a);
        s.me = reinterpret_cast<int32_t*>(p); p += align_up((size_t)C * 4, a);
        s.lens = reinterpret_cast<uint32_t*>(p); p += align_up((size_t)C * 4, a);
        s.scores = reinterpret_cast<int32_t*>(p); p += align_up((size_t)C * 4, a);
        s.flags = p; p += align_up(C, a);
        s.cigars = reinterpret_cast<uint32_t*>(p); p += align_up(hp->cigar_cap * 4, a);
        e = cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.comp_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->comp[0], cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        if (algo == AIM_ALGO_WFA_AFFINE) e = cudaStreamCreateWithFlags(&hp->comp[1], cudaStreamNonBlocking);
        else hp->comp[1] = hp->comp[0];
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->d2h, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cudaGetLastError(); destroy_pipe(hp); *err = e; return nullptr; }
    *err = cudaSuccess;
    return hp;
}

// byte range [lo, hi) holding sequences [c0, c1) of a host layout
void byte_range(const uint64_t* off, const uint32_t* len, uint32_t c0, uint32_t c1, uint64_t* lo, uint64_t* hi) {
    uint64_t l = UINT64_MAX, h = 0;
    for (uint32_t i = c0; i < c1; ++i) {
        l = std::min<uint64_t>(l, off[i]);
        h = std::max<uint64_t>(h, off[i] + len[i]);
    }
    if (l > h) l = h = 0;
    *lo = l; *hi = h;
}

}  // namespace

void free_host_pipe(void* pipe) { destroy_pipe(static_cast<HostPipe*>(pipe)); }

}  // namespace aim

extern "C" int aim_align_batch_host(aim_ctx* ctx, const uint8_t* reads, const uint8_t* targets,
                                    const uint64_t* read_char_offsets, const uint64_t* target_char_offsets,
                                    const uint32_t* read_lengths, const uint32_t* target_lengths, uint32_t num_pairs,
                                    uint32_t max_length, int algo, const aim_penalties_t* pen, int32_t max_edits,
                                    const int32_t* max_edits_per_pair, int32_t* out_scores, uint32_t* out_cigars,
                                    const uint64_t* cigar_offsets, uint32_t* out_cigar_lens, uint8_t* out_flags,
                                    uint32_t chunk_pairs, uint64_t* bytes_moved) {
    aim::Range range("aim_align_batch_host");
    using namespace aim;
    if (bytes_moved) bytes_moved[0] = bytes_moved[1] = 0;
    if (!ctx || !pen || algo < AIM_ALGO_EDIT_NW || algo > AIM_ALGO_GENASM) return AIM_ERR_ARG;
    if (num_pairs == 0) return AIM_OK;
    if (!reads || !targets || !read_char_offsets || !target_char_offsets || !read_lengths || !target_lengths ||
        !out_scores || !out_flags || ((out_cigars == nullptr) != (cigar_offsets == nullptr)))
        return AIM_ERR_ARG;
    if (max_edits_per_pair && max_edits < 0) return AIM_ERR_ARG;
    DeviceGuardImpl guard(ctx->device);
    if (!guard.ok) return AIM_ERR_CUDA;

    // chunks: C pairs (default: a quarter of the batch, at least 65,536 pairs; on 4M uneven pairs an eighth,
    // a half and the whole batch measured 3-15 % slower end to end).  Each chunk's byte ranges are
    // found (and its CIGAR offsets checked) when its turn comes, so that host work overlaps the device work of
    // the chunks before it; the slots are sized from the first chunk with a quarter of headroom and grow (after
    // the device has finished with them) if a later chunk needs more.
    uint32_t C = chunk_pairs ? chunk_pairs : std::max<uint32_t>((num_pairs + 3) / 4, 65536u);
    C = std::min(C, num_pairs);
    const uint32_t nchunks = (num_pairs + C - 1) / C;
    const bool wfa_batched = algo == AIM_ALGO_WFA_AFFINE;
    auto chunk_ranges = [&](uint32_t j, uint64_t r[4]) -> bool {
        const uint32_t c0 = j * C, c1 = std::min(num_pairs, c0 + C);
        for (uint32_t i = c0; cigar_offsets && i < c1; ++i)
            if (cigar_offsets[i + 1] < cigar_offsets[i]) return false;   // capacities are differences
        byte_range(read_char_offsets, read_lengths, c0, c1, &r[0], &r[1]);
        byte_range(target_char_offsets, target_lengths, c0, c1, &r[2], &r[3]);
        return true;
    };
    auto headroom = [](uint64_t x) { return x + x / 4; };
    uint64_t r0[4];
    if (!chunk_ranges(0, r0)) return AIM_ERR_ARG;
    HostPipe* hp = static_cast<HostPipe*>(ctx->host_pipe);
    auto rebuild = [&](uint64_t rc, uint64_t tc, uint64_t cc) -> int {
        destroy_pipe(hp);   // waits for the device to finish with the old slots
        ctx->host_pipe = nullptr;
        cudaError_t err;
        hp = make_pipe(algo, pen, max_edits, max_edits_per_pair != nullptr, out_cigars != nullptr, max_length, C,
                       headroom(rc), headroom(tc), headroom(cc), &err);
        if (!hp) return err == cudaErrorMemoryAllocation ? AIM_ERR_NOMEM : cuda_status(err);
        ctx->host_pipe = hp;
        return AIM_OK;
    };
    {
        const uint64_t cc0 = cigar_offsets ? cigar_offsets[std::min(num_pairs, C)] - cigar_offsets[0] : 0;
        if (!same_shape(hp, algo, pen, max_edits, max_edits_per_pair != nullptr, out_cigars != nullptr, max_length, C,
                        r0[1] - r0[0], r0[3] - r0[2], cc0)) {
            const int st = rebuild(r0[1] - r0[0], r0[3] - r0[2], cc0);
            if (st != AIM_OK) return st;
        }
    }

    uint64_t h2d = 0, d2h = 0;
    cudaError_t e = cudaSuccess;
    int rc_status = AIM_OK;
    for (uint32_t j = 0; j < nchunks && e == cudaSuccess && rc_status == AIM_OK; ++j) {
        const uint32_t c0 = j * C, c1 = std::min(num_pairs, c0 + C), k = c1 - c0;
        uint64_t r[4];
        if (j == 0) {
            std::memcpy(r, r0, sizeof(r));
        } else if (!chunk_ranges(j, r)) {
            rc_status = AIM_ERR_ARG;
            break;
        }
        const uint64_t rlo = r[0], rhi = r[1], tlo = r[2], thi = r[3];
        const uint64_t cbase = cigar_offsets ? cigar_offsets[c0] : 0;
        const uint64_t cend = cigar_offsets ? cigar_offsets[c1] - cbase : 0;
        if (rhi - rlo > hp->read_cap || thi - tlo > hp->target_cap || cend > hp->cigar_cap) {
            // a chunk that needs larger slots: the earlier chunks' results are finished first (their copies out
            // complete), then the slots are rebuilt (and replanned) with room for this one
            rc_status = rebuild(std::max(rhi - rlo, hp->read_cap), std::max(thi - tlo, hp->target_cap),
                                std::max(cend, hp->cigar_cap));
            if (rc_status != AIM_OK) break;
        }
        Slot& s = hp->slot[j & 1];
        cudaStream_t comp = hp->comp[j & 1];
        const uint32_t padded = wfa_batched ? C : k;
        // copy in straight from the caller's arrays, once the slot's previous alignment has read its inputs
        if (s.used) e = cudaStreamWaitEvent(hp->h2d, s.comp_done, 0);
        auto in = [&](void* dst, const void* src, size_t bytes) {
            if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, hp->h2d);
            h2d += bytes;
        };
        in(s.reads, reads + rlo, rhi - rlo);
        in(s.targets, targets + tlo, thi - tlo);
        in(s.roff, read_char_offsets + c0, (size_t)k * 8);
        in(s.toff, target_char_offsets + c0, (size_t)k * 8);
        if (cigar_offsets) in(s.coff, cigar_offsets + c0, ((size_t)k + 1) * 8);
        in(s.rlen, read_lengths + c0, (size_t)k * 4);
        in(s.tlen, target_lengths + c0, (size_t)k * 4);
        if (max_edits_per_pair) in(s.me, max_edits_per_pair + c0, (size_t)k * 4);
        if (e == cudaSuccess) e = cudaEventRecord(s.in_done, hp->h2d);
        if (e != cudaSuccess) break;
        // align, once the inputs are in and the slot's previous results have left
        e = cudaStreamWaitEvent(comp, s.in_done, 0);
        if (e == cudaSuccess && s.used) e = cudaStreamWaitEvent(comp, s.out_done, 0);
        if (e != cudaSuccess) break;
        {
            const unsigned blocks = (unsigned)std::min<uint64_t>(((uint64_t)padded + 256) / 256, 1024);
            rebase_kernel<<<blocks, 256, 0, comp>>>(s.roff, s.toff, s.coff, s.rlen, s.tlen, s.me, k, padded, rlo, tlo,
                                                    cbase, cend, max_edits_per_pair != nullptr,
                                                    cigar_offsets != nullptr);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
        }
        // runs past each pair's count read as zero in the host buffer, as with the device entry points
        if (cigar_offsets && cend) e = cudaMemsetAsync(s.cigars, 0, cend * 4, comp);
        if (e != cudaSuccess) break;
        if (wfa_batched) {
            if (!s.plan) {
                // planned on the chunk it first holds (planning packs and buckets the bound inputs, so they are
                // rebased first); the second slot's plan takes the lanes the first one tuned from the context's
                // cache.  Each slot's plan has its own half of the workspace as scratch.
                e = cudaStreamSynchronize(comp);
                if (e != cudaSuccess) break;
                const size_t half = ((ctx->ws_bytes - kHeaderBytes) / 2) & ~(size_t)255;
                rc_status = batch_plan_impl(ctx, s.reads, s.targets, s.roff, s.toff, s.rlen, s.tlen, C, max_length,
                                            pen, max_edits, max_edits_per_pair ? s.me : nullptr, s.scores,
                                            cigar_offsets ? s.cigars : nullptr, cigar_offsets ? s.coff : nullptr,
                                            s.lens, s.flags, 0, (j & 1) == 0 ? 1 : 0,
                                            ctx->ws + kHeaderBytes + (j & 1) * half, half, &s.plan);
                if (rc_status != AIM_OK) break;
            }
            rc_status = aim_batch_run(s.plan, comp);
        } else {
            rc_status = aim_align_batch_ascii(ctx, s.reads, s.targets, s.roff, s.toff, s.rlen, s.tlen, k, max_length,
                                              algo, pen, max_edits, max_edits_per_pair ? s.me : nullptr, s.scores,
                                              cigar_offsets ? s.cigars : nullptr, cigar_offsets ? s.coff : nullptr,
                                              s.lens, s.flags, comp);
        }
        if (rc_status != AIM_OK) break;
        e = cudaEventRecord(s.comp_done, comp);
        // copy out, once aligned
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->d2h, s.comp_done, 0);
        auto out = [&](void* dst, const void* src, size_t bytes) {
            if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, hp->d2h);
            d2h += bytes;
        };
        out(out_scores + c0, s.scores, (size_t)k * 4);
        out(out_flags + c0, s.flags, k);
        if (out_cigar_lens) out(out_cigar_lens + c0, s.lens, (size_t)k * 4);
        if (cigar_offsets) out(out_cigars + cbase, s.cigars, cend * 4);
        if (e == cudaSuccess) e = cudaEventRecord(s.out_done, hp->d2h);
        s.used = true;
    }
    // every result in host memory before returning (also after an error, so no copy outlives the call; a failed
    // rebuild has already waited for the old slots and left no pipe)
    if (!hp) return rc_status != AIM_OK ? rc_status : AIM_ERR_CUDA;
    const cudaError_t e1 = cudaStreamSynchronize(hp->h2d);
    cudaError_t e2 = cudaStreamSynchronize(hp->comp[0]);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(hp->comp[1]);
    const cudaError_t e3 = cudaStreamSynchronize(hp->d2h);
    if (bytes_moved) { bytes_moved[0] = h2d; bytes_moved[1] = d2h; }
    if (rc_status != AIM_OK) return rc_status;
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
    return cuda_status(e);
}
