// Banded global DP with traceback: NW edit distance (Section 2.4.1, unit
// costs) and gap-affine Gotoh with three states M, I, D (Section 2.4.2).
//
// One warp aligns one pair, or, for narrow bands, 32/GS pairs side by side
// in segments of GS = 16 or 8 lanes (a band of b <= GS - 1 fits one segment:
// with band 10, 21 diagonals would otherwise leave two thirds of a warp's
// lanes idle).  The band |h - v| <= b holds 2b+1 diagonals; lane j of lane
// block r (of a segment) owns the two diagonals q = 2(GS r + j) and q + 1
// (q = k + b).  The sweep runs over anti-diagonals d = v + h: cell (v, h)
// of diagonal k sits on anti-diagonal d with v = (d - k) / 2, so at step d
// exactly the diagonals with k = d (mod 2) hold a cell, i.e. one of each
// lane's two diagonals: every lane computes one cell per block per step.
//   M(v,h) needs (v-1,h-1): same diagonal, two steps ago  -> own register
//   I(v,h) needs (v-1,h):   diagonal k+1, previous step   -> own register or lane+1
//   D(v,h) needs (v,h-1):   diagonal k-1, previous step   -> own register or lane-1
// Cells outside the matrix or the band are infinite; M(0,0) = 0 seeds the
// sweep and the recurrences then give the borders I(v,0) = o+e*v and
// D(0,h) = o+e*h by themselves.
//
// Trace bits: for each state S of a cell, which predecessor states P reach
// S's value exactly (P(pred) + cost(P->S) == S).  The canonical traceback
// (among optimal alignments the one whose ops read backward are smallest
// under X < I < D < M) follows the set of "tight" states: the chosen state's
// tight predecessors are exactly the states whose values meet the cost the
// remaining prefix must have.  Unit cost has one state, so three bits
// (diagonal, up, left) say which neighbours reach H(v,h).
//
// Base comparisons: a lane's cells on one diagonal read consecutive bases of
// both sequences, so every 64 anti-diagonals the warp builds, per diagonal, a
// 32-bit mask of the next 32 cells' mismatches from two 32-base windows
// (XOR, fold each 2-bit field, gather the bits); a cell then tests one bit.
//
// Early exit (threshold): costs never decrease along a path and every path
// touches one of any two consecutive anti-diagonals, so once every cell of
// two consecutive anti-diagonals exceeds the limit the pair is rejected.
//
// Trace bits are stored per pair as rows of anti-diagonals, entry (d, q/2),
// so the 32 lanes of a step write one contiguous row.  A warp keeps up to 32
// pair slots: finished pairs wait in them, and once they are all taken (or
// the queue is drained) lane j traces back slot j, so the serial tracebacks
// run side by side.
#include <type_traits>
#include <utility>

#include "aim_internal.cuh"

namespace aim {
namespace {

struct DpArgs {
    Costs c;
    PairsView P;
    LimitView L;
    OutView O;
    int band;
    uint8_t* scratch;
    size_t slot_bytes;       // one pair's trace rows and run staging
    size_t trace_bytes;      // offset of the run staging area inside a slot
    uint32_t defer;          // slots per warp: finished pairs wait in them and are traced back side by side
    uint32_t runs_cap;
    uint32_t nwarps;
    uint32_t* counter;
};

__device__ __forceinline__ int32_t cap_inf(int32_t v) { return v > kInf ? kInf : v; }

// A new value is at most its predecessor's plus the largest cost, so after d anti-diagonals every value is at
// most kInf + d * (largest cost).  When that stays within int32 for the whole sweep (the host checks), values
// need no cap: an unreachable cell then holds some value above kInf instead of kInf itself, which every test
// reads the same way (above any limit; its trace bits are never read).
template <bool CAP>
__device__ __forceinline__ int32_t capped(int32_t v) { return CAP ? cap_inf(v) : v; }
__device__ __forceinline__ int32_t min3(int32_t a, int32_t b, int32_t c) { return min(min(a, b), c); }

// 32 bases from base `pos` of a sequence, first base in the top bits; positions before 0 or past the end read 0
__device__ __forceinline__ uint64_t window_from(const uint64_t* w, uint32_t nwords, int pos) {
    if (pos >= 0) return window32(w, nwords, (uint32_t)pos);
    if (pos <= -32) return 0ull;
    return window32(w, nwords, 0u) >> (2 * -pos);
}

// Mismatch bits of 32 consecutive cells of one diagonal: bit j is set when read base iv + j differs from target
// base ih + j.  The XOR of the two 32-base windows has a nonzero 2-bit field where the bases differ; those fields
// fold onto their low bits, the even bits are gathered into 32 (bit 31 - j for base j) and reversed.  Bases past
// a sequence's end read as 0; the sweep never asks for them.
__device__ __forceinline__ uint32_t mismatch_mask(const uint64_t* Pw, uint32_t nwP, int iv, const uint64_t* Tw,
                                                  uint32_t nwT, int ih) {
    const uint64_t x = window_from(Pw, nwP, iv) ^ window_from(Tw, nwT, ih);
    uint64_t f = (x | (x >> 1)) & 0x5555555555555555ull;
    f = (f | (f >> 1)) & 0x3333333333333333ull;
    f = (f | (f >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    f = (f | (f >> 4)) & 0x00FF00FF00FF00FFull;
    f = (f | (f >> 8)) & 0x0000FFFF0000FFFFull;
    f = (f | (f >> 16)) & 0x00000000FFFFFFFFull;
    return __brev((uint32_t)f);
}

// finished pairs awaiting their traceback, one record per slot of a warp: pair, score, tight end states
__shared__ int4 s_dp_pend[256];

// Canonical traceback of one finished pair by one lane, from its trace rows; returns the number of runs,
// staged end-first.  ok turns false if a step finds no tight state (not expected) or the runs overflow.
template <bool UNIT, int RW>
__device__ uint32_t dp_traceback(const DpArgs& a, const uint8_t* slot, uint32_t* staged, uint32_t pi, uint32_t ends,
                                 bool& ok) {
    using TB = typename std::conditional<UNIT, uint8_t, uint16_t>::type;
    const TB* trace = reinterpret_cast<const TB*>(slot);
    const int b = a.band;
    const uint64_t* Pw = read_words(a.P, pi);
    const uint64_t* Tw = target_words(a.P, pi);
    RunWriter w;
    w.init(staged, a.runs_cap);
    bool tM = ends & 1u, tI = (ends >> 1) & 1u, tD = (ends >> 2) & 1u;
    int v = (int)a.P.read_len[pi], h = (int)a.P.target_len[pi];
    while (v > 0 || h > 0) {
        const int k = h - v;
        if (k < -b || k > b) { ok = false; break; }
        const uint32_t bits = trace[(size_t)(v + h) * RW + ((k + b) >> 1)];
        if (UNIT) { tM = bits & 1u; tI = (bits >> 1) & 1u; tD = (bits >> 2) & 1u; }
        const bool match = v > 0 && h > 0 && base_at(Pw, v - 1) == base_at(Tw, h - 1);
        uint32_t op;
        if (tM && v > 0 && h > 0 && !match) op = kOpMismatch;
        else if (tI) op = kOpIns;
        else if (tD) op = kOpDel;
        else if (tM && match) op = kOpMatch;
        else { ok = false; break; }
        if (!UNIT) {
            const uint32_t sh = (op == kOpIns) ? 3 : (op == kOpDel) ? 6 : 0;
            const uint32_t t = bits >> sh;
            if (op == kOpIns) { tM = t & 1u; tD = (t >> 1) & 1u; tI = (t >> 2) & 1u; }
            else { tM = t & 1u; tI = (t >> 1) & 1u; tD = (t >> 2) & 1u; }
        }
        if (op == kOpMismatch || op == kOpMatch) { --v; --h; }
        else if (op == kOpIns) { --v; }
        else { --h; }
        w.put(op, 1);
    }
    w.finish();
    ok = ok && w.n <= w.cap;
    return w.n;
}

// Whole warp: lane j traces back the pair waiting in slot j (so up to 32 tracebacks run side by side), then
// the warp writes each pair's result.  A slot whose record holds pair -1 is empty (its segment's pair was
// rejected or flagged).
template <bool UNIT, int RW>
__device__ __forceinline__ void dp_finish(const DpArgs& a, uint8_t* warp_slots, const int4* pend, uint32_t npend,
                                          uint32_t lane) {
    __syncwarp();   // trace rows and records written by every lane are visible
    uint32_t nruns = 0;
    bool ok = true;
    if (lane < npend && pend[lane].x >= 0) {
        const int4 r = pend[lane];
        uint8_t* slot = warp_slots + (size_t)lane * a.slot_bytes;
        nruns = dp_traceback<UNIT, RW>(a, slot, reinterpret_cast<uint32_t*>(slot + a.trace_bytes), (uint32_t)r.x,
                                       (uint32_t)r.z, ok);
    }
    __syncwarp();
    for (uint32_t j = 0; j < npend; ++j) {
        const int4 r = pend[j];
        const uint32_t nj = __shfl_sync(kFull, nruns, j);
        const bool okj = __shfl_sync(kFull, ok ? 1 : 0, j) != 0;
        if (r.x < 0) continue;
        const uint32_t* staged = reinterpret_cast<const uint32_t*>(warp_slots + (size_t)j * a.slot_bytes + a.trace_bytes);
        write_cigar(a.O, (uint32_t)r.x, r.y, staged, nj, okj, lane);
    }
    __syncwarp();
}

// 4 blocks of 256 per SM (64 registers) with one lane block, 2 with two
template <bool UNIT, int R, int SUB, bool CAP>
__global__ void __launch_bounds__(256, R == 1 ? 4 : R == 2 ? 2 : 1) dp_kernel(DpArgs a) {
    static_assert(SUB == 1 || R == 1, "several pairs per warp only for one lane block");
    using TB = typename std::conditional<UNIT, uint8_t, uint16_t>::type;
    constexpr int GS = 32 / SUB;    // lanes per pair (a segment of the warp)
    constexpr int RW = GS * R;      // trace entries per anti-diagonal row
    const uint32_t lane = threadIdx.x & 31;
    const int sl = (int)lane % GS, sg = (int)lane / GS;   // lane within the segment, segment
    const uint32_t seg = GS == 32 ? kFull : (((1u << GS) - 1u) << (sg * GS));
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gwarp >= a.nwarps) return;
    uint8_t* warp_slots = a.scratch + (size_t)gwarp * a.defer * a.slot_bytes;
    int4* pend = s_dp_pend + (threadIdx.x & ~31u);
    uint32_t npend = 0;   // slots taken: 0 .. npend-1 (warp-uniform; SUB per round, some possibly empty)
    const int b = a.band;
    const int32_t x = UNIT ? 1 : a.c.x;
    const int32_t oe = UNIT ? 1 : a.c.o + a.c.e;
    const int32_t e = UNIT ? 1 : a.c.e;
    // this lane's cells and pairs over the launch, in 32 bits (a lane sweeps one cell per block and step: 2^32
    // of them would take minutes)
    uint32_t st_cells = 0, st_pairs = 0;

    for (;;) {
        uint32_t p0 = 0;
        if (lane == 0) p0 = atomicAdd(a.counter, (uint32_t)SUB);
        p0 = __shfl_sync(kFull, p0, 0);
        if (p0 >= a.P.num_pairs) break;
        const uint32_t pi = p0 + (uint32_t)sg;
        // this segment's pair: live until it is aligned, rejected or flagged
        bool live = pi < a.P.num_pairs;
        uint32_t n = 0, m = 0;
        int64_t lim = 0;
        int kend = 0;
        if (live) {
            st_pairs += sl == 0;
            n = a.P.read_len[pi]; m = a.P.target_len[pi];
            lim = pair_limit(a.L, pi);
            if (pair_bad(a.P, pi) || n > a.P.max_length || m > a.P.max_length || lim == -2) {
                if (sl == 0) write_header(a.O, pi, -1, AIM_F_BAD_PAIR, 0);
                live = false;
            } else {
                kend = (int)m - (int)n;
                if (kend > b || -kend > b) {
                    if (sl == 0) write_header(a.O, pi, -1, AIM_F_REJECTED, 0);
                    live = false;
                }
            }
        }
        const uint32_t slot_i = npend + (uint32_t)sg;
        if (!__any_sync(kFull, live)) {
            if constexpr (SUB > 1) {   // the round's slots stay empty
                if (sl == 0) pend[slot_i] = make_int4(-1, 0, 0, 0);
                npend += SUB;
                if (npend + SUB > a.defer) { dp_finish<UNIT, RW>(a, warp_slots, pend, npend, lane); npend = 0; }
            }
            continue;
        }
        const int32_t limc = lim >= (int64_t)kInf ? kInf - 1 : (int32_t)lim;
        TB* trace = reinterpret_cast<TB*>(warp_slots + (size_t)slot_i * a.slot_bytes);
        const uint64_t* Pw = live ? read_words(a.P, pi) : nullptr;
        const uint64_t* Tw = live ? target_words(a.P, pi) : nullptr;

        // per slot (parity p, block r): the latest cell of that diagonal, the anti-diagonal range where the
        // diagonal holds cells of this pair, and the mismatch bits of the diagonal's next cells (mm: up to 32
        // cells from read base mi0, refreshed for the whole warp every 64 anti-diagonals)
        int32_t Ms[2][R], Is[2][R], Ds[2][R];
        int dlo[2][R], dhi[2][R];
        uint32_t mm[2][R];
        int mi0[2][R];
        const uint32_t nwP = (n + 31) >> 5, nwT = (m + 31) >> 5;
#pragma unroll
        for (int pp = 0; pp < 2; ++pp)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                Ms[pp][r] = Is[pp][r] = Ds[pp][r] = kInf;
                const int q = 2 * (GS * r + sl) + pp, k = q - b;
                // cell (v,h) of diagonal k lies on anti-diagonal d = 2v + k: v >= 0, h >= 0, v <= n, h <= m
                dlo[pp][r] = live && q <= 2 * b ? (k < 0 ? -k : k) : (1 << 30);
                dhi[pp][r] = min(2 * (int)n + k, 2 * (int)m - k);
                mi0[pp][r] = -(1 << 30);
                mm[pp][r] = 0;
            }
        {   // seed: cell (0,0) on diagonal k = 0, q = b
            const int i0 = b >> 1, p0s = b & 1;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (live && r == (i0 / GS) && sl == (i0 % GS)) Ms[p0s][r] = 0;
        }
        bool prev_over = false;
        const int dend = live ? (int)(n + m) : 0;
        // several pairs per warp: the sweep runs on past a pair's last anti-diagonal (for the other segments), so the
        // lane that computes the end cell (n, m) keeps its values here
        int32_t xM = kInf, xI = kInf, xD = kInf;
        if (SUB > 1 && live && dend == 0 && sl == (b >> 1) % GS) xM = 0;   // both sequences empty: the seed cell
        const int dmax = SUB == 1 ? dend : (int)__reduce_max_sync(kFull, (unsigned)dend);

        // one anti-diagonal step on the slots of parity P (P == (d + b) & 1); returns whether every cell of this
        // segment's pair on it exceeds the limit (true for a segment with no live pair)
        auto step = [&](const int d, auto parity) -> bool {
            constexpr int P = decltype(parity)::value;
            bool over = true;
            TB* trow = trace + (size_t)d * RW;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                // neighbour slot on the other parity: P == 0 needs q-1 (lane-1, wrapping to block r-1),
                // P == 1 needs q+1 (lane+1, wrapping to block r+1); shuffles stay inside the segment
                int32_t nM, nI = kInf, nD = kInf;
                if (P == 0) {
                    nM = __shfl_up_sync(kFull, Ms[1][r], 1, GS);
                    if (!UNIT) { nI = __shfl_up_sync(kFull, Is[1][r], 1, GS); nD = __shfl_up_sync(kFull, Ds[1][r], 1, GS); }
                    if constexpr (R > 1) {
                        const int rr = r > 0 ? r - 1 : 0;
                        const int32_t wM = __shfl_sync(kFull, r > 0 ? Ms[1][rr] : kInf, 31);
                        int32_t wI = kInf, wD = kInf;
                        if (!UNIT) {
                            wI = __shfl_sync(kFull, r > 0 ? Is[1][rr] : kInf, 31);
                            wD = __shfl_sync(kFull, r > 0 ? Ds[1][rr] : kInf, 31);
                        }
                        if (lane == 0) { nM = wM; nI = wI; nD = wD; }
                    } else if (sl == 0) {
                        nM = kInf; nI = kInf; nD = kInf;
                    }
                } else {
                    nM = __shfl_down_sync(kFull, Ms[0][r], 1, GS);
                    if (!UNIT) { nI = __shfl_down_sync(kFull, Is[0][r], 1, GS); nD = __shfl_down_sync(kFull, Ds[0][r], 1, GS); }
                    if constexpr (R > 1) {
                        const int rr = r + 1 < R ? r + 1 : r;
                        const int32_t wM = __shfl_sync(kFull, r + 1 < R ? Ms[0][rr] : kInf, 0);
                        int32_t wI = kInf, wD = kInf;
                        if (!UNIT) {
                            wI = __shfl_sync(kFull, r + 1 < R ? Is[0][rr] : kInf, 0);
                            wD = __shfl_sync(kFull, r + 1 < R ? Ds[0][rr] : kInf, 0);
                        }
                        if (lane == 31) { nM = wM; nI = wI; nD = wD; }
                    } else if (sl == GS - 1) {
                        nM = kInf; nI = kInf; nD = kInf;
                    }
                }
                // diagonal predecessor = own slot of parity P; up = q+1, left = q-1
                const int32_t dM = Ms[P][r], dI = Is[P][r], dD = Ds[P][r];
                const int32_t uM = P ? nM : Ms[1][r], uI = P ? nI : Is[1][r], uD = P ? nD : Ds[1][r];
                const int32_t lM = P ? Ms[0][r] : nM, lI = P ? Is[0][r] : nI, lD = P ? Ds[0][r] : nD;
                int32_t Mv = kInf, Iv = kInf, Dv = kInf;
                if (d >= dlo[P][r] && d <= dhi[P][r]) {
                    const int k = 2 * (GS * r + sl) + P - b;
                    const int v = (d - k) >> 1, h = (d + k) >> 1;
                    uint32_t bits = 0;
                    if (v >= 1 && h >= 1) {
                        // this cell's bit of the diagonal's mask (refreshed for the whole warp every 64 steps)
                        const int32_t delta = (mm[P][r] >> (v - 1 - mi0[P][r])) & 1u ? x : 0;
                        if (UNIT) {
                            Mv = capped<CAP>(dM + delta);
                        } else {
                            // the mismatch cost is common to the three predecessors: compare them with their
                            // minimum.  (Bits of an unreachable cell are never read: the traceback walks reachable
                            // cells only, so no test of the value against infinity is needed.)
                            const int32_t mn = min3(dM, dI, dD);
                            Mv = capped<CAP>(mn + delta);
                            bits |= (dM == mn ? 1u : 0u) | (dI == mn ? 2u : 0u) | (dD == mn ? 4u : 0u);
                        }
                    }
                    if (v >= 1) {
                        if (UNIT) {
                            Iv = capped<CAP>(uM + 1);
                        } else {
                            const int32_t a0 = uM + oe, a1 = uD + oe, a2 = uI + e, mn = min3(a0, a1, a2);
                            Iv = capped<CAP>(mn);
                            bits |= (a0 == mn ? 8u : 0u) | (a1 == mn ? 16u : 0u) | (a2 == mn ? 32u : 0u);
                        }
                    }
                    if (h >= 1) {
                        if (UNIT) {
                            Dv = capped<CAP>(lM + 1);
                        } else {
                            const int32_t a0 = lM + oe, a1 = lI + oe, a2 = lD + e, mn = min3(a0, a1, a2);
                            Dv = capped<CAP>(mn);
                            bits |= (a0 == mn ? 64u : 0u) | (a1 == mn ? 128u : 0u) | (a2 == mn ? 256u : 0u);
                        }
                    }
                    if (UNIT) {
                        // one state: H is the min; keep it in the M slot and mark which neighbours reach it
                        const int32_t H = min3(Mv, Iv, Dv);
                        bits = (Mv == H && H < kInf ? 1u : 0u) | (Iv == H && H < kInf ? 2u : 0u) |
                               (Dv == H && H < kInf ? 4u : 0u);
                        Mv = H; Iv = kInf; Dv = kInf;
                    }
                    trow[GS * r + sl] = (TB)bits;
                    if constexpr (SUB > 1) {
                        if (d == dend && k == kend) { xM = Mv; xI = Iv; xD = Dv; }
                    }
                    ++st_cells;
                    over = over && min3(Mv, Iv, Dv) > limc;
                }
                Ms[P][r] = Mv; Is[P][r] = Iv; Ds[P][r] = Dv;
            }
            if constexpr (SUB == 1) return __all_sync(kFull, over);
            else return (__ballot_sync(kFull, over) & seg) == seg;
        };
        // the mismatch masks of every slot for the anti-diagonals dr .. dr + 63: slot (p, r) holds the cells on
        // anti-diagonals of its diagonal's parity, at most 32 of them in 64 steps, from read base mi0 on.  The
        // whole warp refreshes at the same steps, so no lane waits on another's loads.
        int covered = 0;   // last anti-diagonal the masks cover
        auto refresh = [&](const int dr) {
#pragma unroll
            for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int k = 2 * (GS * r + sl) + pp - b;
                    const int d1 = dr + ((dr - k) & 1);   // first anti-diagonal >= dr holding a cell of k
                    mi0[pp][r] = ((d1 - k) >> 1) - 1;
                    mm[pp][r] = live ? mismatch_mask(Pw, nwP, mi0[pp][r], Tw, nwT, mi0[pp][r] + k) : 0u;
                }
            covered = dr + 63;
        };
        using P0 = std::integral_constant<int, 0>;
        using P1 = std::integral_constant<int, 1>;
        if constexpr (SUB == 1) {
            bool rejected = false;
            int d = 1;
            if (d <= dend) refresh(d);
            if (d <= dend && ((d + b) & 1)) {   // start on parity 1 so the loop below alternates 0, 1
                prev_over = step(d, P1{});
                ++d;
            }
            for (; d <= dend; d += 2) {
                if (d + 1 > covered) refresh(d);
                bool o = step(d, P0{});
                if (o && prev_over) { rejected = true; break; }
                prev_over = o;
                if (d + 1 > dend) break;
                o = step(d + 1, P1{});
                if (o && prev_over) { rejected = true; break; }
                prev_over = o;
            }
            if (rejected) {
                if (lane == 0) write_header(a.O, pi, -1, AIM_F_REJECTED, 0);
                continue;
            }
        } else {
            // a segment whose pair is rejected (two consecutive anti-diagonals over the limit, inside its own
            // range) stops computing: its ranges are emptied.  The warp runs while any segment's pair is live; a
            // segment past its own last anti-diagonal has finished and takes no further decision.
            auto rejects = [&](bool o, int dd) {
                if (!live || dd > dend) return;
                if (o && prev_over) {
                    live = false;
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                        for (int r = 0; r < R; ++r) dlo[pp][r] = 1 << 30;
                    if (sl == 0) write_header(a.O, pi, -1, AIM_F_REJECTED, 0);
                }
                prev_over = o;
            };
            int d = 1;
            if (d <= dmax) refresh(d);
            if (d <= dmax && ((d + b) & 1)) {
                rejects(step(d, P1{}), d);
                ++d;
            }
            for (; d <= dmax; d += 2) {
                if (d + 1 > covered) refresh(d);
                rejects(step(d, P0{}), d);
                if (!__any_sync(kFull, live)) break;
                if (d + 1 > dmax) break;
                rejects(step(d + 1, P1{}), d + 1);
                if (!__any_sync(kFull, live)) break;
            }
        }
        // values at (n, m)
        const int qe = kend + b, ie = qe >> 1, pe = qe & 1, re = ie / GS, je = ie % GS;
        int32_t eM = kInf, eI = kInf, eD = kInf;
        if constexpr (SUB == 1) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r == re) {
                    eM = pe ? Ms[1][r] : Ms[0][r]; eI = pe ? Is[1][r] : Is[0][r]; eD = pe ? Ds[1][r] : Ds[0][r];
                }
        } else {
            (void)re; (void)pe;
            eM = xM; eI = xI; eD = xD;
        }
        const int src = sg * GS + (live ? je : 0);
        eM = __shfl_sync(kFull, eM, src); eI = __shfl_sync(kFull, eI, src); eD = __shfl_sync(kFull, eD, src);
        const int32_t sc = min3(eM, eI, eD);
        if (live && sc > limc) {
            if (sl == 0) write_header(a.O, pi, -1, AIM_F_REJECTED, 0);
            live = false;
        }
        if constexpr (SUB == 1) {   // a slot only for an aligned pair
            if (!live) continue;
            if (lane == 0) pend[npend] = make_int4((int)pi, sc, (int)((eM == sc) | (eI == sc) << 1 | (eD == sc) << 2), 0);
            if (++npend == a.defer) {
                dp_finish<UNIT, RW>(a, warp_slots, pend, npend, lane);
                npend = 0;
            }
        } else {   // a round of SUB slots, empty for a segment whose pair was rejected or flagged
            if (sl == 0)
                pend[slot_i] = live ? make_int4((int)pi, sc, (int)((eM == sc) | (eI == sc) << 1 | (eD == sc) << 2), 0)
                                    : make_int4(-1, 0, 0, 0);
            npend += SUB;
            if (npend + SUB > a.defer) {
                dp_finish<UNIT, RW>(a, warp_slots, pend, npend, lane);
                npend = 0;
            }
        }
    }
    dp_finish<UNIT, RW>(a, warp_slots, pend, npend, lane);
    warp_stat_add(a.O.stats, 2, (unsigned long long)st_cells, lane);
    warp_stat_add(a.O.stats, 3, (unsigned long long)st_pairs, lane);
}

template <bool UNIT, int R, int SUB, bool CAP>
cudaError_t launch_t(const DpArgs& args0, int num_sms, cudaStream_t st, int* warps_used, size_t scratch_bytes) {
    int bps = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, dp_kernel<UNIT, R, SUB, CAP>, 256, 0);
    if (err != cudaSuccess) return err;
    if (bps < 1) bps = 1;
    size_t warps = (size_t)num_sms * bps * 8;
    const size_t fit = scratch_bytes / (args0.slot_bytes * SUB);   // a warp needs a slot per segment at least
    if (warps > fit) warps = fit;
    const size_t need = (args0.P.num_pairs + SUB - 1) / SUB;
    if (warps > need) warps = need;
    if (warps == 0) { *warps_used = 0; return cudaSuccess; }
    DpArgs a = args0;
    a.nwarps = (uint32_t)warps;
    // slots per warp: the scratch spread over the launch's warps, up to one per lane, a whole number of rounds
    const size_t per_warp = scratch_bytes / warps / args0.slot_bytes;
    a.defer = (uint32_t)((per_warp > 32 ? 32 : per_warp) / SUB * SUB);
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    dp_kernel<UNIT, R, SUB, CAP><<<blocks, 256, 0, st>>>(a);
    *warps_used = (int)warps;
    return cudaGetLastError();
}

template <bool CAP>
cudaError_t launch_dp_t(const DpPlan& plan, const DpArgs& a, int num_sms, cudaStream_t st, int* warps_used,
                        size_t scratch_bytes) {
    if (plan.unit) {
        if (plan.pairs_per_warp == 4) return launch_t<true, 1, 4, CAP>(a, num_sms, st, warps_used, scratch_bytes);
        if (plan.pairs_per_warp == 2) return launch_t<true, 1, 2, CAP>(a, num_sms, st, warps_used, scratch_bytes);
        if (plan.blocks == 1) return launch_t<true, 1, 1, CAP>(a, num_sms, st, warps_used, scratch_bytes);
        if (plan.blocks == 2) return launch_t<true, 2, 1, CAP>(a, num_sms, st, warps_used, scratch_bytes);
        return launch_t<true, 4, 1, CAP>(a, num_sms, st, warps_used, scratch_bytes);
    }
    if (plan.pairs_per_warp == 4) return launch_t<false, 1, 4, CAP>(a, num_sms, st, warps_used, scratch_bytes);
    if (plan.pairs_per_warp == 2) return launch_t<false, 1, 2, CAP>(a, num_sms, st, warps_used, scratch_bytes);
    if (plan.blocks == 1) return launch_t<false, 1, 1, CAP>(a, num_sms, st, warps_used, scratch_bytes);
    if (plan.blocks == 2) return launch_t<false, 2, 1, CAP>(a, num_sms, st, warps_used, scratch_bytes);
    return launch_t<false, 4, 1, CAP>(a, num_sms, st, warps_used, scratch_bytes);
}

}  // namespace

DpPlan plan_dp(bool unit, int band, uint32_t max_length, int64_t max_limit) {
    DpPlan p;
    p.unit = unit;
    p.band = band;
    p.blocks = band <= 31 ? 1 : band <= 63 ? 2 : 4;
    // narrow bands: several pairs per warp, one per segment of 32 / pairs lanes (2b + 1 diagonals on 2 per lane)
    p.pairs_per_warp = band <= 7 ? 4 : band <= 15 ? 2 : 1;
    const size_t te = unit ? 1 : 2;
    const size_t rows = 2 * (size_t)max_length + 1;
    const size_t trace = align_up(rows * (32 / p.pairs_per_warp) * p.blocks * te, 16);
    p.slot_bytes = trace;   // run staging appended by launch_dp
    (void)max_limit;
    return p;
}

cudaError_t launch_dp(const DpPlan& plan, const Costs& c, const PairsView& P, const LimitView& L, const OutView& O,
                      int64_t max_limit, uint8_t* scratch, size_t scratch_bytes, uint32_t* counter, int num_sms,
                      cudaStream_t st, int* warps_used) {
    *warps_used = 0;
    if (P.num_pairs == 0) return cudaSuccess;
    DpArgs a;
    a.c = c; a.P = P; a.L = L; a.O = O; a.band = plan.band;
    a.scratch = scratch; a.counter = counter; a.nwarps = 0;
    // staged runs: every edit run costs at least min(x, o+e), and runs alternate with match runs
    const int64_t minc = plan.unit ? 1 : (c.x < c.o + c.e ? c.x : c.o + c.e);
    int64_t cap = 2 * (int64_t)P.max_length + 1;
    if (max_limit < kUnbounded && minc > 0) {
        const int64_t by_cost = 2 * (max_limit / minc) + 1;
        if (by_cost < cap) cap = by_cost;
    }
    a.runs_cap = (uint32_t)cap;
    a.trace_bytes = plan.slot_bytes;
    a.slot_bytes = align_up(plan.slot_bytes + (size_t)cap * 4, 128);
    // values need no cap when kInf + (anti-diagonals + 1) * (largest cost) fits int32
    const int64_t maxc = plan.unit ? 1 : std::max<int64_t>(std::max<int64_t>(c.x, (int64_t)c.o + c.e), c.e);
    const bool need_cap = (2 * (int64_t)P.max_length + 2) * maxc >= (int64_t)INT32_MAX - kInf - maxc;
    return need_cap ? launch_dp_t<true>(plan, a, num_sms, st, warps_used, scratch_bytes)
                    : launch_dp_t<false>(plan, a, num_sms, st, warps_used, scratch_bytes);
}

}  // namespace aim
