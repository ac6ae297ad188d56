// 2-bit packer: ASCII A/C/G/T -> 0/1/2/3, first base in the top two bits of each 64-bit word.
//
// Fixed slots (every sequence at word i * stride, the form the ASCII entry points use): one thread per output
// word.  It reads the word's 32 bytes as aligned 4-byte loads (each load holds at least one byte of the word, so
// none crosses into another page), lines them up with funnel shifts, and converts four bytes at a time:
// ((c >> 1) ^ (c >> 2)) & 3 maps A, C, G, T (0x41, 0x43, 0x47, 0x54) to 0, 1, 2, 3; a byte whose code's letter
// (looked up for four bytes by one byte permute) is not the byte itself flags the pair; one multiply gathers the
// four 2-bit codes into a byte, first base on top.  The slot of a thread comes from a multiply, not a division.
//
// Explicit word offsets (aim_pack_2bit): one warp per sequence; each lane converts one byte per 32-base word
// and the warp ORs the lanes' 2-bit codes together (two 32-bit halves).  Lane w%32 keeps word w and the warp
// stores 32 words at a time with one coalesced store.
#include <type_traits>

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

// four ASCII bytes (first in the low byte) -> their 2-bit codes, first base in bits 7..6; *bad: a byte in `keep`
// (0xff per byte to look at) that is not A, C, G or T.  Every byte c gets the code ((c >> 1) ^ (c >> 2)) & 3,
// and c is one of the four letters exactly when it equals the letter of its code, "ACGT"[code]: one byte
// permute looks the four letters up, with the codes as its selector nibbles.
__device__ __forceinline__ uint32_t pack4(uint32_t x, uint32_t keep, bool& bad) {
    const uint32_t codes = ((x >> 1) ^ (x >> 2)) & 0x03030303u;   // byte k: code of byte k
    const uint32_t pairs = codes | (codes >> 4);                   // byte 0: c0 | c1 << 4; byte 2: c2 | c3 << 4
    const uint32_t sel = __byte_perm(pairs, 0u, 0x4420u);          // nibble k: c_k
    const uint32_t letters = __byte_perm(0x54474341u, 0u, sel);    // byte k: "ACGT"[c_k]
    bad |= ((letters ^ x) & keep) != 0;
    // byte k holds code k; times 2^30 + 2^20 + 2^10 + 1 puts code k at bits 30-2k..31-2k with no carries
    return ((codes & keep) * 0x40100401u) >> 24;
}

// g / d for any 32-bit g, by a multiply: with s = ceil(log2 d) and M = ceil(2^(32+s) / d) = 2^32 + m (d <= 2^s
// puts M in [2^32, 2^33)), g * M / 2^(32+s) = g / d + g (M d - 2^(32+s)) / (d 2^(32+s)), and the second term
// is below 1 / d since M d - 2^(32+s) < d <= 2^s and g < 2^32: its floor is g / d rounded down.
struct Divider {
    uint32_t m, s;
    __device__ uint32_t div(uint32_t g) const { return (uint32_t)(((uint64_t)__umulhi(g, m) + g) >> s); }
};

Divider make_divider(uint32_t d) {   // 1 <= d <= 2^31
    uint32_t s = 0;
    while (((uint64_t)1 << s) < d) ++s;
    const uint64_t M = (((uint64_t)1 << (32 + s)) + d - 1) / d;
    return Divider{(uint32_t)(M - ((uint64_t)1 << 32)), s};
}

template <bool WIDE>
__global__ void __launch_bounds__(256) pack_words_kernel(const uint8_t* __restrict__ ascii,
                                                         const uint64_t* __restrict__ char_off,
                                                         const uint32_t* __restrict__ len, uint32_t count,
                                                         uint64_t* __restrict__ packed, uint32_t stride,
                                                         Divider by_stride, uint8_t* __restrict__ bad) {
    using Index = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
    const Index total = (Index)count * stride;
    for (Index g = (Index)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (Index)gridDim.x * blockDim.x) {
        const uint32_t i = WIDE ? (uint32_t)(g / stride) : by_stride.div((uint32_t)g);
        const uint32_t w = (uint32_t)(g - (Index)i * stride);
        const uint32_t L = __ldg(len + i);
        const uint32_t nw = (L + 31) >> 5;
        if (nw > stride) {   // longer than the fixed per-sequence slot: flag, write nothing
            if (bad && w == 0) bad[i] = 1;
            continue;
        }
        if (w >= nw) continue;
        // first byte of this word; alignment is taken from the address itself (the buffer may start anywhere)
        const uintptr_t at = reinterpret_cast<uintptr_t>(ascii) + __ldg(char_off + i) + 32ull * w;
        const uint32_t nb = min(32u, L - 32u * w);              // bytes of this word
        const uint32_t* base = reinterpret_cast<const uint32_t*>(at & ~(uintptr_t)3);
        const uint32_t sh = 8u * (uint32_t)(at & 3);
        const uint32_t last = (uint32_t)(((at & 3) + nb - 1) >> 2);     // last aligned word holding a byte
        uint32_t u[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) u[q] = (uint32_t)q <= last ? __ldg(base + q) : 0u;
        bool b = false;
        uint32_t hi = 0, lo = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint32_t x = __funnelshift_r(u[q], u[q + 1], sh);
            const int have = (int)nb - 4 * q;                       // bytes of this group inside the word
            const uint32_t keep = have >= 4 ? 0xffffffffu : have <= 0 ? 0u : ((1u << (8 * have)) - 1u);
            const uint32_t byte = pack4(x, keep, b);
            if (q < 4) hi |= byte << (24 - 8 * q);
            else lo |= byte << (24 - 8 * (q - 4));
        }
        packed[g] = ((uint64_t)hi << 32) | lo;
        if (bad && b) bad[i] = 1;
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
    if (!word_off && word_stride > 0 && word_stride <= 0xffffffffull) {
        // fixed slots: one thread per word; bad flags start at 0 and threads that see a bad byte set them
        if (bad) {
            const cudaError_t e = cudaMemsetAsync(bad, 0, count, st);
            if (e != cudaSuccess) return e;
        }
        const uint64_t total = (uint64_t)count * word_stride;
        uint64_t blocks = (total + 255) / 256;
        const uint64_t cap = (uint64_t)sms * 32;   // grid-stride beyond 32 blocks of 256 per SM
        if (blocks > cap) blocks = cap;
        // the reciprocal needs 2^(32+s) in 64 bits (a stride up to 2^31); anything wider divides
        const bool narrow = total <= 0xffffffffull && word_stride <= ((uint64_t)1 << 31);
        const Divider by_stride = narrow ? make_divider((uint32_t)word_stride) : Divider{0u, 0u};
        if (narrow)
            pack_words_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(ascii, char_off, len, count, packed,
                                                                        (uint32_t)word_stride, by_stride, bad);
        else
            pack_words_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(ascii, char_off, len, count, packed,
                                                                       (uint32_t)word_stride, by_stride, bad);
        return cudaGetLastError();
    }
    const uint32_t warps_needed = count;
    uint32_t blocks = (warps_needed + 7) / 8;
    const uint32_t cap = (uint32_t)sms * 8;   // 8 blocks of 8 warps per SM, grid-stride beyond that
    if (blocks > cap) blocks = cap;
    pack_kernel<<<blocks, 256, 0, st>>>(ascii, char_off, len, count, packed, word_off, word_stride, bad);
    return cudaGetLastError();
}

}  // namespace aim
