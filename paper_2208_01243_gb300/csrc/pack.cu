// 2-bit packer: ASCII A/C/G/T -> 0/1/2/3, first base in the top two bits of each 64-bit word.
//
// One warp per sequence; each lane converts one byte per 32-base word and the
// warp ORs the lanes' 2-bit codes together (two 32-bit halves).  Lane w%32
// keeps word w and the warp stores 32 words at a time with one coalesced store.
#include "aim_internal.cuh"

namespace aim {
namespace {

__device__ __forceinline__ uint32_t ascii_code(uint32_t c, bool& ok) {
    // A 0x41, C 0x43, G 0x47, T 0x54
    uint32_t code = (c == 'C') ? 1u : (c == 'G') ? 2u : (c == 'T') ? 3u : 0u;
    ok = (c == 'A') | (c == 'C') | (c == 'G') | (c == 'T');
    return code;
}

__global__ void __launch_bounds__(256) pack_kernel(const uint8_t* __restrict__ ascii,
                                                   const uint64_t* __restrict__ char_off,
                                                   const uint32_t* __restrict__ len, uint32_t count,
                                                   uint64_t* __restrict__ packed,
                                                   const uint64_t* __restrict__ word_off, uint64_t word_stride,
                                                   uint8_t* __restrict__ bad) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = warp; i < count; i += nwarps) {
        const uint8_t* s = ascii + __ldg(char_off + i);
        const uint32_t L = __ldg(len + i);
        uint64_t* out = packed + (word_off ? __ldg(word_off + i) : (uint64_t)i * word_stride);
        const uint32_t nw = (L + 31) >> 5;
        if (!word_off && nw > word_stride) {   // longer than the fixed per-sequence slot: flag, write nothing
            if (bad && lane == 0) bad[i] = 1;
            continue;
        }
        bool any_bad = false;
        uint64_t mine = 0;
        for (uint32_t w = 0; w < nw; ++w) {
            const uint32_t pos = (w << 5) + lane;
            uint32_t code = 0;
            if (pos < L) {
                bool ok;
                code = ascii_code(__ldg(s + pos), ok);
                any_bad |= !ok;
            }
            const uint32_t hi = __reduce_or_sync(0xffffffffu, lane < 16 ? code << (30 - 2 * lane) : 0u);
            const uint32_t lo = __reduce_or_sync(0xffffffffu, lane >= 16 ? code << (30 - 2 * (lane - 16)) : 0u);
            if (lane == (w & 31)) mine = ((uint64_t)hi << 32) | lo;
            if ((w & 31) == 31 || w + 1 == nw) {
                const uint32_t first = w & ~31u;
                if (first + lane <= w) out[first + lane] = mine;
            }
        }
        const bool b = __any_sync(0xffffffffu, any_bad);
        if (bad && lane == 0) bad[i] = b ? 1 : 0;
    }
}

}  // namespace

cudaError_t launch_pack(const uint8_t* ascii, const uint64_t* char_off, const uint32_t* len, uint32_t count,
                        uint64_t* packed, const uint64_t* word_off, uint64_t word_stride, uint8_t* bad,
                        cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t warps_needed = count;
    uint32_t blocks = (warps_needed + 7) / 8;
    const uint32_t cap = (uint32_t)sms * 8;   // 8 blocks of 8 warps per SM, grid-stride beyond that
    if (blocks > cap) blocks = cap;
    pack_kernel<<<blocks, 256, 0, st>>>(ascii, char_off, len, count, packed, word_off, word_stride, bad);
    return cudaGetLastError();
}

}  // namespace aim
