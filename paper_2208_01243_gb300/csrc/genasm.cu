// GenASM (Section 2.4.3): windowed bit-parallel edit distance (bitap) with a
// forward traceback, under a threshold of k edits.  One thread aligns one pair.
//
// Window.  At read position i and target position j a window holds
// wp = min(W, n-i) read bases and wt = min(W, m-j) target bases (W <= 64).  The
// read ends inside it when n-i <= W, the target when m-j <= W.  f(a, c) is the
// least number of edits of a path from (a, c) to the window's far edge; an edge
// whose sequence goes on past the window is free (cost 0 there), an edge whose
// sequence ends inside it charges one edit per base left on the other side.
//
// Status vectors.  Bit b of A_d(t) (one 64-bit word) is [f(wp-1-b, t) <= d]:
// bit 0 is the last read base of the window, bit wp-1 the first.  With
// EQ[c] = the bits whose read base equals c, and e(t, d) = [f(wp, t) <= d] the
// empty read suffix, the recurrence over the target position t (from wt down) is
//   A_d(wt) = target ends ? low d bits : all bits
//   A_d(t)  = ((A_d(t+1) << 1 | e(t+1, d)) & EQ[T[t]])       match
//           | (A_{d-1}(t+1) << 1 | e(t+1, d-1))              mismatch
//           | (A_{d-1}(t) << 1 | e(t, d-1))                  I (read base)
//           | A_{d-1}(t+1)                                   D (target base)
// which is the suffix edit-distance recurrence one distance level at a time.
// Bits above wp-1 carry no meaning; shifts only move them further up.  The
// window distance is the first d with bit wp-1 of A_d(0) set.  A window whose
// distance exceeds the edits left ends the pair: any way the alignment goes on
// crosses the window's far edge, so the count only grows.
//
// Sweeps.  Levels are computed in blocks of four or eight, target position by
// target position (t descending): a block keeps its vectors in registers and
// reads only the top level of the block below, A_{L0-1}(t), from a per-lane
// carry row that it overwrites in place with its own top level (written only
// when another block may follow).
//
// Traceback, forward from (0, 0) with budget d (the window distance): after an
// I, I first; after a D, D first; then M, X, I, D, each only when the rest still
// fits (a match always does: on equal bases f(a, c) = f(a+1, c+1), since the
// values of neighbouring cells differ by at most one).  Match runs are taken
// with 32-base XOR compares.  A non-final window stops once W-O read or W-O
// target bases have been consumed in it; the final window runs to its corner.
// The traceback reads level d-1 at target positions c and c+1 only, for c up
// to W-O in a non-final window, and only near the diagonal: a path with d
// edits never strays more than d diagonals.  So the stored copy of A_d(t) is
// kept for t up to the last position the traceback can read, and, when no
// window can need more than 14 levels, only as the 32 bits from 16 below the
// diagonal position wp-1-t (or from bit 0).
//
// Scratch per warp, lane-interleaved (32 lanes of a step store one contiguous
// row): the carry row, (W+1) x 32 words, then levels x (W+1) x 32 stored
// vectors (32 or 64 bits each).
#include <type_traits>

#include "aim_internal.cuh"

namespace aim {
namespace {

// distance levels per register block, one size per call: blocks of 8 when the threshold allows about two or
// more edits per window (then most windows would need a second block of 4, and a whole warp waits for the
// sweeps any one of its lanes needs), blocks of 4 otherwise
constexpr int kSmallBlock = 4, kBigBlock = 8;
constexpr int kBandLevels = 14;         // widest window distance a 32-bit band serves

struct GenasmArgs {
    PairsView P;
    LimitView L;
    OutView O;
    uint8_t* scratch;
    size_t warp_bytes;              // carry row + stored levels of one warp
    size_t carry_bytes;             // offset of the stored levels inside a warp's scratch
    int W, overlap;
    bool big_blocks;                // blocks of kBigBlock levels (else kSmallBlock): picks the kernel instance
    uint32_t nwarps;
    uint32_t* counter;
};

constexpr uint32_t kNoOp = 0;

__device__ __forceinline__ uint64_t low_bits(int d) { return d >= 64 ? ~0ull : ((1ull << d) - 1ull); }

// The stored copy of A_d(t): the whole word, or the 32 bits from band_start(wp, t) up, which hold every bit
// the traceback can ask for (within 16 of the diagonal position wp-1-t, never below bit 0).
__device__ __forceinline__ int band_start(int wp, int t) { return max(wp - 17 - t, 0); }
template <typename Band>
__device__ __forceinline__ Band band_of(uint64_t v, int s);
template <>
__device__ __forceinline__ uint64_t band_of<uint64_t>(uint64_t v, int) { return v; }
template <>
__device__ __forceinline__ uint32_t band_of<uint32_t>(uint64_t v, int s) {   // bits s..s+31, s in [0, 47]
    const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    return s < 32 ? __funnelshift_r(lo, hi, (uint32_t)s) : (hi >> (s - 32));
}
// bit b of a stored copy whose band starts at bit s
__device__ __forceinline__ bool band_bit(uint64_t x, int b, int) { return (x >> b) & 1ull; }
__device__ __forceinline__ bool band_bit(uint32_t x, int b, int s) { return (x >> (b - s)) & 1u; }

// 32 even bits (bit 2s) of x -> bits s of the result
__device__ __forceinline__ uint32_t even_bits(uint64_t x) {
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
    x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
    x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
    return (uint32_t)x;
}

// one bit per base of a 32-base window word (first base in the top bits): 1 where the base is `code`
__device__ __forceinline__ uint32_t match_bits(uint64_t w, uint32_t code) {
    const uint64_t x = w ^ (0x5555555555555555ull * code);
    return even_bits(~(x | (x >> 1)));
}

// matching bases of read[p..] and target[q..], at most `cap`
__device__ __forceinline__ int match_run(const uint64_t* rw, uint32_t nrw, uint32_t p, const uint64_t* tw,
                                         uint32_t ntw, uint32_t q, int cap) {
    int run = 0;
    while (run < cap) {
        const uint64_t x = window32(rw, nrw, p + run) ^ window32(tw, ntw, q + run);
        const int same = __clzll((long long)x) >> 1;   // __clzll(0) = 64: the whole window matches
        run += same;
        if (same < 32) break;
    }
    return run < cap ? run : cap;
}

struct Window {
    uint64_t eq[4];     // read bases of the window, one mask per base code
    uint64_t t0, t1;    // target bases 0..31 and 32..63 of the window
    int wp, wt;
    int tmax;           // last target position the traceback can read
    bool end_r, end_t;
};

// One sweep of the B levels L0..L0+B-1 over t = wt..0.  FREE_R: the read goes on past the window (the
// empty read suffix costs nothing); BANDS: store the levels for the traceback (positions up to w.tmax);
// CARRY_OUT: overwrite the carry row with level L0+B-1; CARRY_IN: read level L0-1 from the carry row.
template <int B, typename Band, bool FREE_R, bool BANDS, bool CARRY_OUT, bool CARRY_IN>
__device__ __forceinline__ void sweep(const Window& w, int L0, Band* lv, size_t lstride, uint64_t* carry,
                                      uint64_t (&cur)[B]) {
    const int wp = w.wp, wt = w.wt;
    const uint64_t edge = w.end_t ? 0ull : ~0ull;   // A_d(wt) = edge | low d bits
#pragma unroll
    for (int q = 0; q < B; ++q) {
        cur[q] = edge | low_bits(L0 + q);
        if (BANDS && wt <= w.tmax)
            lv[(size_t)(L0 + q) * lstride + (size_t)wt * 32] = band_of<Band>(cur[q], band_start(wp, wt));
    }
    if (CARRY_OUT) carry[(size_t)wt * 32] = cur[B - 1];
    uint64_t lo_old = CARRY_IN ? (edge | low_bits(L0 - 1)) : 0ull;   // A_{L0-1}(t+1)
    auto step = [&](const int t, auto keep_tag) {
        constexpr bool KEEP = decltype(keep_tag)::value;
        const uint64_t tword = t < 32 ? w.t0 : w.t1;
        const uint32_t code = (uint32_t)(tword >> (62 - 2 * (t & 31))) & 3u;
        const uint64_t e01 = (code & 1) ? w.eq[1] : w.eq[0], e23 = (code & 1) ? w.eq[3] : w.eq[2];
        const uint64_t eqc = (code & 2) ? e23 : e01;
        const uint64_t lo_new = CARRY_IN ? carry[(size_t)t * 32] : 0ull;   // A_{L0-1}(t)
        // the empty read suffix at t+1 fits level d iff the wt-t-1 target bases left fit: e(t+1, d) = [x <= q],
        // e(t+1, d-1) = [x + 1 <= q] (which covers e(t, d-1) too); on a free read edge both are 1
        const int x = wt - t - 1 - L0;
        const int s = KEEP ? band_start(wp, t) : 0;
        uint64_t b_old = lo_old, b_new = lo_new;
#pragma unroll
        for (int q = 0; q < B; ++q) {
            const uint64_t old = cur[q];
            const uint64_t e1 = (FREE_R || x <= q) ? 1ull : 0ull;
            uint64_t v = ((old << 1) | e1) & eqc;
            if (CARRY_IN || q > 0) {
                const uint64_t e2 = (FREE_R || x + 1 <= q) ? 1ull : 0ull;
                v |= ((b_old | b_new) << 1) | e2 | b_old;
            }
            cur[q] = v;
            if (KEEP) lv[(size_t)(L0 + q) * lstride + (size_t)t * 32] = band_of<Band>(v, s);
            b_old = old;
            b_new = v;
        }
        if (CARRY_OUT) carry[(size_t)t * 32] = cur[B - 1];
        lo_old = lo_new;
    };
    // positions past the last one the traceback can read are computed but not stored
    const int split = BANDS ? min(w.tmax, wt - 1) : -1;
    for (int t = wt - 1; t > split; --t) step(t, std::false_type{});
    if (BANDS)
        for (int t = split; t >= 0; --t) step(t, std::true_type{});
}

// Levels from L0 on in blocks of B until one reaches the window's start (or lmax is passed); the first
// block (L0 = 0) reads no carry.  Returns the window's distance or -1.
template <int B, typename Band, bool FREE_R>
__device__ __forceinline__ int blocks_from(const Window& w, int lmax, Band* lv, size_t lstride, uint64_t* carry) {
    uint64_t cur[B];
    int found = -1;
    for (int L0 = 0; found < 0 && L0 <= lmax; L0 += B) {
        // a block fills the carry row whenever another may follow: lanes of a warp move together, so one lane
        // that needs the next block makes the whole warp wait for it
        const bool more = L0 + B <= lmax;
        if (L0 == 0) {
            if (more) sweep<B, Band, FREE_R, true, true, false>(w, 0, lv, lstride, carry, cur);
            else sweep<B, Band, FREE_R, true, false, false>(w, 0, lv, lstride, carry, cur);
        } else {
            if (more) sweep<B, Band, FREE_R, true, true, true>(w, L0, lv, lstride, carry, cur);
            else sweep<B, Band, FREE_R, true, false, true>(w, L0, lv, lstride, carry, cur);
        }
#pragma unroll
        for (int q = 0; q < B; ++q)
            if (found < 0 && L0 + q <= lmax && ((cur[q] >> (w.wp - 1)) & 1ull)) found = L0 + q;
    }
    return found;
}

// The window's distance (the first level whose bit wp-1 is set at t = 0), or -1 if it exceeds lmax.
template <int B, typename Band, bool FREE_R>
__device__ __forceinline__ int window_distance(const Window& w, int lmax, Band* lv, size_t lstride, uint64_t* carry) {
    return blocks_from<B, Band, FREE_R>(w, lmax, lv, lstride, carry);
}

// 5 blocks of 128 threads per SM (96 registers) measured faster than 6 (80) or 8 (64, with spills)
#ifndef AIM_GENASM_MIN_BLOCKS
#define AIM_GENASM_MIN_BLOCKS 5
#endif

// B: distance levels per register block, a kernel instance per block size (one call uses one)
template <typename Band, int B>
__global__ void __launch_bounds__(128, AIM_GENASM_MIN_BLOCKS) genasm_kernel(GenasmArgs a) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gwarp >= a.nwarps) return;
    const int W = a.W, stop = a.W - a.overlap;
    const size_t lstride = (size_t)(W + 1) * 32;                  // stored entries per level
    uint8_t* slot = a.scratch + (size_t)gwarp * a.warp_bytes;
    uint64_t* carry = reinterpret_cast<uint64_t*>(slot) + lane;
    Band* lv = reinterpret_cast<Band*>(slot + a.carry_bytes) + lane;
    unsigned long long st_cells = 0, st_pairs = 0;

    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(a.counter, 32u);
        base = __shfl_sync(kFull, base, 0);
        if (base >= a.P.num_pairs) break;
        const uint32_t pi = base + lane;
        if (pi >= a.P.num_pairs) continue;
        ++st_pairs;

        const uint32_t n = a.P.read_len[pi], m = a.P.target_len[pi];
        const int64_t k = pair_limit(a.L, pi);
        if (pair_bad(a.P, pi) || n > a.P.max_length || m > a.P.max_length || k == -2) {
            write_header(a.O, pi, -1, AIM_F_BAD_PAIR, 0);
            continue;
        }
        const uint64_t* rw = read_words(a.P, pi);
        const uint64_t* tw = target_words(a.P, pi);
        const uint32_t nrw = (n + 31) >> 5, ntw = (m + 31) >> 5;
        RunWriter out;
        uint32_t cap = 0;
        uint32_t* runs = nullptr;
        if (a.O.cigars && a.O.cigar_off) {
            const uint64_t off = a.O.cigar_off[pi];
            runs = a.O.cigars + off;
            cap = (uint32_t)(a.O.cigar_off[pi + 1] - off);
        }
        out.init(runs, cap);

        uint32_t i = 0, j = 0, prev = kNoOp;
        int64_t used = 0;
        bool rejected = false;
        while (i < n && j < m) {
            Window w;
            w.wp = (int)min(n - i, (uint32_t)W);
            w.wt = (int)min(m - j, (uint32_t)W);
            w.end_r = n - i <= (uint32_t)W;
            w.end_t = m - j <= (uint32_t)W;
            const bool fin = w.end_r && w.end_t;
            const int wp = w.wp, wt = w.wt;
            w.tmax = fin ? wt : min(stop, wt);
            // read window masks: bit wp-1-a is read base i+a
            const uint64_t r0 = window32(rw, nrw, i), r1 = window32(rw, nrw, i + 32);
#pragma unroll
            for (uint32_t c = 0; c < 4; ++c)
                w.eq[c] = (((uint64_t)match_bits(r0, c) << 32) | match_bits(r1, c)) >> (64 - wp);
            w.t0 = window32(tw, ntw, j);
            w.t1 = window32(tw, ntw, j + 32);

            // distance levels, in blocks, until the window's start is reached
            const int64_t left = k - used;
            const int lmax = (int)(left < (int64_t)max(wp, wt) ? left : (int64_t)max(wp, wt));
            const int found = w.end_r ? window_distance<B, Band, false>(w, lmax, lv, lstride, carry)
                                      : window_distance<B, Band, true>(w, lmax, lv, lstride, carry);
            // work of a plain bitap: levels 0..d (0..lmax when the window is over the budget) at every position
            st_cells += (unsigned long long)((found < 0 ? lmax : found) + 1) * wt;
            if (found < 0) { rejected = true; break; }

            // traceback
            int ta = 0, tc = 0, d = found;
            for (;;) {
                if (!fin && (ta >= stop || tc >= stop)) break;
                if (ta == wp && tc == wt) break;
                uint32_t op;
                int len = 1;
                if (ta == wp) {
                    op = kOpDel;
                } else if (tc == wt) {
                    op = kOpIns;
                } else {
                    const uint32_t pa = (uint32_t)(__ldg(rw + ((i + ta) >> 5)) >> (62 - 2 * ((i + ta) & 31))) & 3u;
                    const uint32_t pb = (uint32_t)(__ldg(tw + ((j + tc) >> 5)) >> (62 - 2 * ((j + tc) & 31))) & 3u;
                    const bool same = pa == pb;
                    const int b = wp - 1 - ta;
                    bool fI = false, fD = false, fX = false;
                    if (d > 0) {
                        const Band* ld = lv + (size_t)(d - 1) * lstride;
                        const Band at_c = ld[(size_t)tc * 32], at_c1 = ld[(size_t)(tc + 1) * 32];
                        const int p_c = band_start(wp, tc), p_c1 = band_start(wp, tc + 1);
                        const bool e_c = !w.end_r || wt - tc <= d - 1, e_c1 = !w.end_r || wt - tc - 1 <= d - 1;
                        fI = b >= 1 ? band_bit(at_c, b - 1, p_c) : e_c;
                        fD = band_bit(at_c1, b, p_c1);
                        fX = b >= 1 ? band_bit(at_c1, b - 1, p_c1) : e_c1;
                    }
                    if (prev == kOpIns && fI) op = kOpIns;
                    else if (prev == kOpDel && fD) op = kOpDel;
                    else if (same) {
                        op = kOpMatch;
                        int lim = min(wp - ta, wt - tc);
                        if (!fin) lim = min(lim, min(stop - ta, stop - tc));
                        len = match_run(rw, nrw, i + ta, tw, ntw, j + tc, lim);
                    } else if (fX) op = kOpMismatch;
                    else if (fI) op = kOpIns;
                    else op = kOpDel;
                }
                out.put(op, (uint32_t)len);
                prev = op;
                if (op != kOpMatch) { --d; ++used; }
                if (op == kOpMatch || op == kOpMismatch) { ta += len; tc += len; }
                else if (op == kOpIns) ++ta;
                else ++tc;
            }
            i += (uint32_t)ta;
            j += (uint32_t)tc;
            if (used > k) { rejected = true; break; }
        }
        if (!rejected) {
            // one sequence is used up: the rest of the other is one gap
            if (i < n) { out.put(kOpIns, n - i); used += n - i; }
            if (j < m) { out.put(kOpDel, m - j); used += m - j; }
            if (used > k) rejected = true;
        }
        if (rejected) {
            write_header(a.O, pi, -1, AIM_F_REJECTED, 0);
            continue;
        }
        out.finish();
        const uint8_t flags = (runs && out.n > cap) ? AIM_F_CIGAR_OVERFLOW : 0;
        write_header(a.O, pi, (int32_t)used, flags, out.n);
    }
    warp_stat_add(a.O.stats, 4, st_cells, lane);
    warp_stat_add(a.O.stats, 3, st_pairs, lane);
}

// blocks of kBigBlock levels when the threshold allows about two or more edits per window of W bases
bool big_blocks_for(int W, int64_t max_limit, uint32_t max_length) {
    const int64_t len = max_length > (uint32_t)W ? (int64_t)max_length : (int64_t)W;
    return max_limit >= kSmallBlock && max_limit * W >= 2 * len;
}

// distance levels a window can need under the largest threshold, in whole register blocks
int levels_for(int W, int64_t max_limit, bool big) {
    const int64_t top = max_limit < W ? max_limit : W;   // a window's distance never exceeds W
    const int B = big ? kBigBlock : kSmallBlock;
    return (int)((top + 1 + B - 1) / B * B);
}

bool banded(int W, int64_t max_limit) { return (max_limit < W ? max_limit : W) <= kBandLevels; }

size_t carry_bytes_for(int W) { return align_up((size_t)(W + 1) * 32 * sizeof(uint64_t), 256); }

}  // namespace

size_t genasm_warp_bytes(int W, int64_t max_limit, uint32_t max_length) {
    const size_t band = banded(W, max_limit) ? sizeof(uint32_t) : sizeof(uint64_t);
    const int levels = levels_for(W, max_limit, big_blocks_for(W, max_limit, max_length));
    return carry_bytes_for(W) + align_up((size_t)levels * (W + 1) * 32 * band, 256);
}

cudaError_t launch_genasm(int W, int O, const PairsView& P, const LimitView& L, const OutView& Ov, int64_t max_limit,
                          uint8_t* scratch, size_t scratch_bytes, uint32_t* counter, int num_sms, cudaStream_t st,
                          int* warps_used) {
    *warps_used = 0;
    if (P.num_pairs == 0) return cudaSuccess;
    GenasmArgs a;
    a.P = P; a.L = L; a.O = Ov;
    a.W = W; a.overlap = O;
    a.counter = counter;
    a.carry_bytes = carry_bytes_for(W);
    a.big_blocks = big_blocks_for(W, max_limit, P.max_length);
    a.warp_bytes = genasm_warp_bytes(W, max_limit, P.max_length);
    // warp slots start on 256-byte boundaries so that every stored row is one aligned segment
    uint8_t* base = reinterpret_cast<uint8_t*>(align_up(reinterpret_cast<size_t>(scratch), 256));
    const size_t skip = (size_t)(base - scratch);
    if (skip >= scratch_bytes) return cudaSuccess;
    a.scratch = base;
    const bool band = banded(W, max_limit);
    // the four kernel instances: stored copies as 32-bit bands or whole words, blocks of 4 or 8 levels
    void (*kernel)(GenasmArgs) = band ? (a.big_blocks ? genasm_kernel<uint32_t, kBigBlock>
                                                      : genasm_kernel<uint32_t, kSmallBlock>)
                                      : (a.big_blocks ? genasm_kernel<uint64_t, kBigBlock>
                                                      : genasm_kernel<uint64_t, kSmallBlock>);
    int bps = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, 128, 0);
    if (err != cudaSuccess) return err;
    if (bps < 1) bps = 1;
    size_t warps = (size_t)num_sms * bps * 4;
    const size_t fit = (scratch_bytes - skip) / a.warp_bytes;
    if (warps > fit) warps = fit;
    const size_t need = ((size_t)P.num_pairs + 31) / 32;
    if (warps > need) warps = need;
    if (warps == 0) return cudaSuccess;
    a.nwarps = (uint32_t)warps;
    const unsigned blocks = (unsigned)((warps + 3) / 4);
    kernel<<<blocks, 128, 0, st>>>(a);
    *warps_used = (int)warps;
    return cudaGetLastError();
}

}  // namespace aim
