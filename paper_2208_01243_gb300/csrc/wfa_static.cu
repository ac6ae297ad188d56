// aim_wfa_align_static: the wavefront aligner for callers that cannot allocate
// device memory.
//
// Some callers of this library are not free to call cudaMalloc.  A plugin
// inside a host application may be handed a fixed device-memory budget by
// that application and forbidden to allocate on its own.  A latency-critical
// loop may not tolerate an allocation call, which can block on the device.
// A deployment may need its device footprint fixed when the process starts.
// Such callers cannot create a context either, because aim_create allocates
// the context workspace.  This entry point therefore takes no context: the
// WFA kernel's per-warp scratch (wavefront history, CIGAR run staging) and
// its launch counter live in one file-scope device array of fixed size,
// reserved on every GPU where the library's device code is loaded and held
// until the process exits.
//
// Host code cannot use the array's name as a device address, so on the first
// call on each device (that device current) the array's address is looked up
// with cudaGetSymbolAddress and cached.  A context reset (cudaDeviceReset) or
// another context on the device loads the module again, possibly at another
// address, so every later call that is not being captured into a graph looks
// the address up again (a cheap host-side lookup once the module is loaded);
// a call made during stream capture uses the address of the last call made
// outside capture.
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "aim_internal.cuh"
#include "ranges.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB per device
constexpr size_t kStaticHeaderBytes = 256;                  // launch counter at the start

static __device__ __align__(256) uint8_t g_wfa_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_lookup_mu;
uint8_t* g_scratch_addr[kMaxDevices];   // device address of g_wfa_static_scratch per device, null until looked up
int g_num_sms[kMaxDevices];

int static_status(cudaError_t e) { return e == cudaSuccess ? AIM_OK : AIM_ERR_CUDA; }

// Device address of the static scratch on the current device: looked up on the first call on the device and
// again on every call whose stream is not capturing (so a reset context is never addressed through a stale
// pointer); during capture, the address of the last lookup.
int scratch_for_current_device(cudaStream_t st, uint8_t** addr, int* sms) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_status(e);
    if (dev < 0 || dev >= kMaxDevices) return AIM_ERR_UNSUPPORTED;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) {          // e.g. the legacy stream queried while another stream captures
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;
    }
    std::lock_guard<std::mutex> lock(g_lookup_mu);
    if (!g_scratch_addr[dev] || cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_wfa_static_scratch);
        if (e != cudaSuccess || p == nullptr) return AIM_ERR_CUDA;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return static_status(e);
        g_num_sms[dev] = n;
        g_scratch_addr[dev] = static_cast<uint8_t*>(p);
    }
    *addr = g_scratch_addr[dev];
    *sms = g_num_sms[dev];
    return AIM_OK;
}

}  // namespace

extern "C" int aim_wfa_align_static(const uint64_t* packed_reads, const uint64_t* packed_targets,
                                    const uint64_t* read_offsets, const uint64_t* target_offsets,
                                    const uint32_t* read_lengths, const uint32_t* target_lengths,
                                    uint32_t num_pairs, uint32_t max_length, const aim_penalties_t* pen,
                                    int32_t max_edits, const int32_t* max_edits_per_pair, int32_t* out_scores,
                                    uint32_t* out_cigars, const uint64_t* cigar_offsets, uint32_t* out_cigar_lens,
                                    uint8_t* out_flags, aim_stream_t stream) {
    aim::Range range("aim_wfa_align_static");
    if (!pen || pen->match != 0 || pen->mismatch < 1 || pen->gap_open < 0 || pen->gap_extend < 1 ||
        pen->mismatch > (1 << 20) || pen->gap_open > (1 << 20) || pen->gap_extend > (1 << 20))
        return AIM_ERR_ARG;
    if (num_pairs == 0) return AIM_OK;
    if (!packed_reads || !packed_targets || !read_offsets || !target_offsets || !read_lengths ||
        !target_lengths || !out_scores || !out_flags)
        return AIM_ERR_ARG;
    if ((out_cigars == nullptr) != (cigar_offsets == nullptr)) return AIM_ERR_ARG;
    if (max_length > aim::kMaxWfaLength) return AIM_ERR_UNSUPPORTED;

    // the threshold rule of aim.h
    const aim::Costs costs{pen->mismatch, pen->gap_open, pen->gap_extend};
    aim::LimitView lim;
    lim.per_pair = nullptr;
    lim.max_edits_bound = max_edits;
    lim.edit_cost = std::max(costs.x, costs.o + costs.e);
    int64_t max_limit;
    if (pen->max_score >= 0) {
        lim.limit = max_limit = pen->max_score;
    } else if (max_edits_per_pair) {
        if (max_edits < 0) return AIM_ERR_ARG;
        lim.per_pair = max_edits_per_pair;
        lim.limit = max_limit = (int64_t)max_edits * lim.edit_cost;
    } else {
        lim.limit = max_limit = max_edits < 0 ? aim::kUnbounded : (int64_t)max_edits * lim.edit_cost;
    }

    const aim::WfaPlan plan = aim::plan_wfa(costs, pen->band, max_length, max_limit);
    const size_t capacity = kStaticScratchBytes - kStaticHeaderBytes;
    int group = aim::wfa_default_group(plan, max_length);
    while (group <= 32 && 8 * aim::wfa_warp_bytes(group, aim::wfa_pair_bytes(plan, group)) > capacity)
        group = group == 32 ? 256 : group * 2;
    if (8 * aim::wfa_warp_bytes(group, aim::wfa_pair_bytes(plan, group)) > capacity)
        return AIM_ERR_NOMEM;   // one pair is too big

    uint8_t* base = nullptr;
    int sms = 0;
    int rc = scratch_for_current_device((cudaStream_t)stream, &base, &sms);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* counter = reinterpret_cast<uint32_t*>(base);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), st);   // the launch counter starts at zero
    if (e != cudaSuccess) return AIM_ERR_CUDA;
    aim::PairsView P{packed_reads, packed_targets, read_offsets, target_offsets, read_lengths, target_lengths,
                     nullptr, nullptr, num_pairs, max_length};
    aim::OutView O{out_scores, out_cigars, cigar_offsets, out_cigar_lens, out_flags, nullptr};
    int warps = 0;
    e = aim::launch_wfa(plan, group, P, lim, O, base + kStaticHeaderBytes, capacity, counter, sms, st, &warps);
    if (e != cudaSuccess) return AIM_ERR_CUDA;
    return warps > 0 ? AIM_OK : AIM_ERR_NOMEM;
}
