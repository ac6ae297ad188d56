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
// window distance is the first d with bit wp-1 of A_d(0) set.
//
// Levels are computed in blocks of four, target position by target position
// (t descending), so that a block keeps its four current vectors in registers
// and reads only the top level of the block below from memory.  Every vector
// is stored: the traceback needs level d-1 at two target positions per edit.
// A window whose distance exceeds the edits left ends the pair: any way the
// alignment goes on crosses the window's far edge, so the count only grows.
//
// Traceback, forward from (0, 0) with budget d (the window distance): after an
// I, I first; after a D, D first; then M, X, I, D, each only when the rest still
// fits (a match always does: on equal bases f(a, c) = f(a+1, c+1), since the
// values of neighbouring cells differ by at most one).  Match runs are taken
// with 32-base XOR compares.  A non-final window stops once W-O read or W-O
// target bases have been consumed in it; the final window runs to its corner.
//
// Scratch: per warp, levels x (W+1) x 32 words, lane-interleaved so that the
// 32 lanes of a step store one contiguous 256-byte row.
#include "aim_internal.cuh"

namespace aim {
namespace {

constexpr int kGenasmBlock = 4;     // distance levels per register block

struct GenasmArgs {
    PairsView P;
    LimitView L;
    OutView O;
    uint64_t* scratch;
    int W, overlap;
    int levels;                     // level slots per lane (a multiple of kGenasmBlock)
    uint32_t nwarps;
    uint32_t* counter;
};

constexpr uint32_t kNoOp = 0;

__device__ __forceinline__ uint64_t low_bits(int d) { return d >= 64 ? ~0ull : ((1ull << d) - 1ull); }

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
        const int same = x ? (__clzll(x) >> 1) : 32;
        run += same;
        if (same < 32) break;
    }
    return run < cap ? run : cap;
}

__global__ void __launch_bounds__(128, 8) genasm_kernel(GenasmArgs a) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gwarp >= a.nwarps) return;
    const int W = a.W, stop = a.W - a.overlap;
    const size_t row = (size_t)(W + 1) * 32;                     // words per level
    uint64_t* S = a.scratch + (size_t)gwarp * a.levels * row + lane;
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
            const int wp = (int)min(n - i, (uint32_t)W), wt = (int)min(m - j, (uint32_t)W);
            const bool end_r = n - i <= (uint32_t)W, end_t = m - j <= (uint32_t)W, fin = end_r && end_t;
            // read window masks: bit wp-1-a is read base i+a
            const uint64_t r0 = window32(rw, nrw, i), r1 = window32(rw, nrw, i + 32);
            uint64_t eq[4];
#pragma unroll
            for (uint32_t c = 0; c < 4; ++c)
                eq[c] = (((uint64_t)match_bits(r0, c) << 32) | match_bits(r1, c)) >> (64 - wp);
            const uint64_t t0 = window32(tw, ntw, j), t1 = window32(tw, ntw, j + 32);

            // distance levels, blocks of four, until the window's start is reached
            const int64_t left = k - used;
            const int lmax = (int)(left < (int64_t)max(wp, wt) ? left : (int64_t)max(wp, wt));
            const uint64_t edge = end_t ? 0ull : ~0ull;       // A_d(wt) = edge | low d bits
            int found = -1;
            for (int L0 = 0; found < 0 && L0 <= lmax; L0 += kGenasmBlock) {
                uint64_t cur[kGenasmBlock];
#pragma unroll
                for (int q = 0; q < kGenasmBlock; ++q) {
                    cur[q] = edge | low_bits(L0 + q);
                    S[((size_t)(L0 + q) * (W + 1) + wt) * 32] = cur[q];
                }
                uint64_t lo_old = L0 ? (edge | low_bits(L0 - 1)) : 0ull;   // A_{L0-1}(t+1)
                const uint64_t* below = L0 ? S + (size_t)(L0 - 1) * row : S;   // level L0-1 (read only when L0 > 0)
                for (int t = wt - 1; t >= 0; --t) {
                    const uint64_t tword = t < 32 ? t0 : t1;
                    const uint32_t code = (uint32_t)(tword >> (62 - 2 * (t & 31))) & 3u;
                    const uint64_t e01 = (code & 1) ? eq[1] : eq[0], e23 = (code & 1) ? eq[3] : eq[2];
                    const uint64_t eqc = (code & 2) ? e23 : e01;
                    const uint64_t lo_new = L0 ? below[(size_t)t * 32] : 0ull;   // A_{L0-1}(t)
                    const int r = wt - t;                                         // target bases t..wt-1
                    uint64_t b_old = lo_old, b_new = lo_new;
#pragma unroll
                    for (int q = 0; q < kGenasmBlock; ++q) {
                        const int d = L0 + q;
                        const uint64_t old = cur[q];
                        // e(t+1, d) = [f(wp, t+1) <= d]: free edge, or the r-1 target bases left fit in d
                        const uint64_t e1 = (!end_r || r - 1 <= d) ? 1ull : 0ull;
                        uint64_t v = ((old << 1) | e1) & eqc;
                        if (d > 0) {
                            // e(t+1, d-1) covers e(t, d-1) too (fewer bases left at t+1)
                            const uint64_t e2 = (!end_r || r <= d) ? 1ull : 0ull;
                            v |= ((b_old | b_new) << 1) | e2 | b_old;
                        }
                        cur[q] = v;
                        S[((size_t)d * (W + 1) + t) * 32] = v;
                        b_old = old;
                        b_new = v;
                    }
                    lo_old = lo_new;
                }
                st_cells += (unsigned long long)kGenasmBlock * wt;
#pragma unroll
                for (int q = 0; q < kGenasmBlock; ++q)
                    if (found < 0 && L0 + q <= lmax && ((cur[q] >> (wp - 1)) & 1ull)) found = L0 + q;
            }
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
                        const uint64_t* lv = S + (size_t)(d - 1) * row;
                        const uint64_t at_c = lv[(size_t)tc * 32], at_c1 = lv[(size_t)(tc + 1) * 32];
                        const bool e_c = !end_r || wt - tc <= d - 1, e_c1 = !end_r || wt - tc - 1 <= d - 1;
                        fI = b >= 1 ? ((at_c >> (b - 1)) & 1ull) : e_c;
                        fD = (at_c1 >> b) & 1ull;
                        fX = b >= 1 ? ((at_c1 >> (b - 1)) & 1ull) : e_c1;
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

}  // namespace

size_t genasm_warp_bytes(int W, int levels) { return (size_t)levels * (W + 1) * 32 * sizeof(uint64_t); }

int genasm_levels(int W, int64_t max_limit) {
    const int64_t top = max_limit < W ? max_limit : W;   // a window's distance never exceeds W
    return (int)((top + 1 + kGenasmBlock - 1) / kGenasmBlock * kGenasmBlock);
}

cudaError_t launch_genasm(int W, int O, const PairsView& P, const LimitView& L, const OutView& Ov, int64_t max_limit,
                          uint8_t* scratch, size_t scratch_bytes, uint32_t* counter, int num_sms, cudaStream_t st,
                          int* warps_used) {
    *warps_used = 0;
    if (P.num_pairs == 0) return cudaSuccess;
    GenasmArgs a;
    a.P = P; a.L = L; a.O = Ov;
    a.W = W; a.overlap = O;
    a.levels = genasm_levels(W, max_limit);
    a.counter = counter;
    // scratch rows must start on 256-byte boundaries for whole-row stores
    uint8_t* base = reinterpret_cast<uint8_t*>(align_up(reinterpret_cast<size_t>(scratch), 256));
    const size_t skip = (size_t)(base - scratch);
    if (skip >= scratch_bytes) return cudaSuccess;
    a.scratch = reinterpret_cast<uint64_t*>(base);
    int bps = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, genasm_kernel, 128, 0);
    if (err != cudaSuccess) return err;
    if (bps < 1) bps = 1;
    size_t warps = (size_t)num_sms * bps * 4;
    const size_t fit = (scratch_bytes - skip) / genasm_warp_bytes(W, a.levels);
    if (warps > fit) warps = fit;
    const size_t need = ((size_t)P.num_pairs + 31) / 32;
    if (warps > need) warps = need;
    if (warps == 0) return cudaSuccess;
    a.nwarps = (uint32_t)warps;
    genasm_kernel<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(a);
    *warps_used = (int)warps;
    return cudaGetLastError();
}

}  // namespace aim
