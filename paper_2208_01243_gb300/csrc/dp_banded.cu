// Banded global DP with traceback: NW edit distance (Section 2.4.1, unit
// costs) and gap-affine Gotoh with three states M, I, D (Section 2.4.2).
//
// One warp aligns one pair.  The band |h - v| <= b holds 2b+1 diagonals;
// lane j of lane block r owns the two diagonals q = 2(32r + j) and q + 1
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
// Early exit (threshold): costs never decrease along a path and every path
// touches one of any two consecutive anti-diagonals, so once every cell of
// two consecutive anti-diagonals exceeds the limit the pair is rejected.
//
// Trace bits are stored per warp as rows of anti-diagonals, entry (d, q/2),
// so the 32 lanes of a step write one contiguous row.
#include <type_traits>

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
    size_t slot_bytes;
    size_t trace_bytes;      // offset of the run staging area inside a slot
    uint32_t runs_cap;
    uint32_t nwarps;
    uint32_t* counter;
};

__device__ __forceinline__ int32_t cap_inf(int32_t v) { return v > kInf ? kInf : v; }
__device__ __forceinline__ int32_t min3(int32_t a, int32_t b, int32_t c) { return min(min(a, b), c); }

template <bool UNIT, int R>
__global__ void __launch_bounds__(256) dp_kernel(DpArgs a) {
    using TB = typename std::conditional<UNIT, uint8_t, uint16_t>::type;
    constexpr int RW = 32 * R;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gwarp >= a.nwarps) return;
    uint8_t* slot = a.scratch + (size_t)gwarp * a.slot_bytes;
    TB* trace = reinterpret_cast<TB*>(slot);
    uint32_t* staged = reinterpret_cast<uint32_t*>(slot + a.trace_bytes);
    const int b = a.band;
    const int32_t x = UNIT ? 1 : a.c.x;
    const int32_t oe = UNIT ? 1 : a.c.o + a.c.e;
    const int32_t e = UNIT ? 1 : a.c.e;
    unsigned long long st_cells = 0, st_pairs = 0;

    for (;;) {
        uint32_t pi = 0;
        if (lane == 0) pi = atomicAdd(a.counter, 1u);
        pi = __shfl_sync(kFull, pi, 0);
        if (pi >= a.P.num_pairs) break;
        st_pairs += lane == 0;

        const uint32_t n = a.P.read_len[pi], m = a.P.target_len[pi];
        const int64_t lim = pair_limit(a.L, pi);
        const bool bad = pair_bad(a.P, pi) || n > a.P.max_length || m > a.P.max_length || lim == -2;
        if (bad) {
            if (lane == 0) write_header(a.O, pi, -1, AIM_F_BAD_PAIR, 0);
            continue;
        }
        const int kend = (int)m - (int)n;
        if (kend > b || -kend > b) {
            if (lane == 0) write_header(a.O, pi, -1, AIM_F_REJECTED, 0);
            continue;
        }
        const int32_t limc = lim >= (int64_t)kInf ? kInf - 1 : (int32_t)lim;
        const uint64_t* Pw = read_words(a.P, pi);
        const uint64_t* Tw = target_words(a.P, pi);

        // per slot (block r, parity p): the latest cell of that diagonal
        int32_t M0[R], I0[R], D0[R], M1[R], I1[R], D1[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { M0[r] = I0[r] = D0[r] = M1[r] = I1[r] = D1[r] = kInf; }
        {   // seed: cell (0,0) on diagonal k = 0, q = b
            const int i0 = b >> 1, p0 = b & 1;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r == (i0 >> 5) && (int)lane == (i0 & 31)) { if (p0) M1[r] = 0; else M0[r] = 0; }
        }
        bool prev_over = false, rejected = false;
        const int dend = (int)(n + m);
        for (int d = 1; d <= dend; ++d) {
            const int p = (d + b) & 1;
            bool over = true;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = 32 * r + (int)lane;
                const int q = 2 * i + p;
                const int k = q - b;
                const int v = (d - k) >> 1, h = (d + k) >> 1;
                const bool valid = q <= 2 * b && v >= 0 && h >= 0 && v <= (int)n && h <= (int)m;
                // neighbour on the other parity: p == 0 needs q-1 (lane-1, wraps to block r-1),
                // p == 1 needs q+1 (lane+1, wraps to block r+1)
                int32_t nM, nI, nD;
                if (p == 0) {
                    nM = __shfl_up_sync(kFull, M1[r], 1);
                    nI = __shfl_up_sync(kFull, I1[r], 1);
                    nD = __shfl_up_sync(kFull, D1[r], 1);
                    const int32_t wM = __shfl_sync(kFull, r > 0 ? M1[r > 0 ? r - 1 : 0] : kInf, 31);
                    const int32_t wI = __shfl_sync(kFull, r > 0 ? I1[r > 0 ? r - 1 : 0] : kInf, 31);
                    const int32_t wD = __shfl_sync(kFull, r > 0 ? D1[r > 0 ? r - 1 : 0] : kInf, 31);
                    if (lane == 0) { nM = wM; nI = wI; nD = wD; }
                } else {
                    nM = __shfl_down_sync(kFull, M0[r], 1);
                    nI = __shfl_down_sync(kFull, I0[r], 1);
                    nD = __shfl_down_sync(kFull, D0[r], 1);
                    const int32_t wM = __shfl_sync(kFull, r + 1 < R ? M0[r + 1 < R ? r + 1 : r] : kInf, 0);
                    const int32_t wI = __shfl_sync(kFull, r + 1 < R ? I0[r + 1 < R ? r + 1 : r] : kInf, 0);
                    const int32_t wD = __shfl_sync(kFull, r + 1 < R ? D0[r + 1 < R ? r + 1 : r] : kInf, 0);
                    if (lane == 31) { nM = wM; nI = wI; nD = wD; }
                }
                // diagonal predecessor = own slot of parity p; up = q+1, left = q-1
                const int32_t dM = p ? M1[r] : M0[r], dI = p ? I1[r] : I0[r], dD = p ? D1[r] : D0[r];
                const int32_t uM = p ? nM : M1[r], uI = p ? nI : I1[r], uD = p ? nD : D1[r];
                const int32_t lM = p ? M0[r] : nM, lI = p ? I0[r] : nI, lD = p ? D0[r] : nD;

                int32_t Mv = kInf, Iv = kInf, Dv = kInf;
                uint32_t bits = 0;
                if (valid) {
                    if (v >= 1 && h >= 1) {
                        const int32_t delta = base_at(Pw, v - 1) == base_at(Tw, h - 1) ? 0 : x;
                        const int32_t Hd = min3(dM, dI, dD);
                        Mv = cap_inf(Hd + delta);
                        if (Mv < kInf) {
                            if (UNIT) bits |= 1u;
                            else bits |= (dM + delta == Mv ? 1u : 0u) | (dI + delta == Mv ? 2u : 0u) |
                                         (dD + delta == Mv ? 4u : 0u);
                        }
                    }
                    if (v >= 1) {
                        if (UNIT) {
                            Iv = cap_inf(min3(uM, uI, uD) + 1);
                        } else {
                            Iv = cap_inf(min3(uM + oe, uD + oe, uI + e));
                            if (Iv < kInf)
                                bits |= (uM + oe == Iv ? 8u : 0u) | (uD + oe == Iv ? 16u : 0u) |
                                        (uI + e == Iv ? 32u : 0u);
                        }
                    }
                    if (h >= 1) {
                        if (UNIT) {
                            Dv = cap_inf(min3(lM, lI, lD) + 1);
                        } else {
                            Dv = cap_inf(min3(lM + oe, lI + oe, lD + e));
                            if (Dv < kInf)
                                bits |= (lM + oe == Dv ? 64u : 0u) | (lI + oe == Dv ? 128u : 0u) |
                                        (lD + e == Dv ? 256u : 0u);
                        }
                    }
                    if (UNIT) {
                        // one state: H is the min; keep it in the M slot and mark which neighbours reach it
                        const int32_t H = min3(Mv, Iv, Dv);
                        bits = (Mv == H && H < kInf ? 1u : 0u) | (Iv == H && H < kInf ? 2u : 0u) |
                               (Dv == H && H < kInf ? 4u : 0u);
                        Mv = H; Iv = kInf; Dv = kInf;
                    }
                    trace[(size_t)d * RW + i] = (TB)bits;
                    ++st_cells;
                    over = over && min3(Mv, Iv, Dv) > limc;
                }
                if (p) { M1[r] = Mv; I1[r] = Iv; D1[r] = Dv; } else { M0[r] = Mv; I0[r] = Iv; D0[r] = Dv; }
            }
            const bool all_over = __all_sync(kFull, over);
            if (all_over && prev_over) { rejected = true; break; }
            prev_over = all_over;
        }
        if (rejected) {
            if (lane == 0) write_header(a.O, pi, -1, AIM_F_REJECTED, 0);
            continue;
        }
        // values at (n, m)
        const int qe = kend + b, ie = qe >> 1, pe = qe & 1, re = ie >> 5, je = ie & 31;
        int32_t eM = kInf, eI = kInf, eD = kInf;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (r == re) { eM = pe ? M1[r] : M0[r]; eI = pe ? I1[r] : I0[r]; eD = pe ? D1[r] : D0[r]; }
        eM = __shfl_sync(kFull, eM, je); eI = __shfl_sync(kFull, eI, je); eD = __shfl_sync(kFull, eD, je);
        const int32_t s = min3(eM, eI, eD);
        if (s > limc) {
            if (lane == 0) write_header(a.O, pi, -1, AIM_F_REJECTED, 0);
            continue;
        }
        __syncwarp();   // trace rows written by every lane are visible to lane 0
        uint32_t nruns = 0;
        bool ok = true;
        if (lane == 0) {
            RunWriter w;
            w.init(staged, a.runs_cap);
            bool tM = eM == s, tI = eI == s, tD = eD == s;
            int v = (int)n, h = (int)m;
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
            nruns = w.n;
            ok = ok && w.n <= w.cap;
        }
        __syncwarp();
        nruns = __shfl_sync(kFull, nruns, 0);
        ok = __shfl_sync(kFull, ok, 0);
        write_cigar(a.O, pi, s, staged, nruns, ok, lane);
        __syncwarp();
    }
    warp_stat_add(a.O.stats, 2, st_cells, lane);
    warp_stat_add(a.O.stats, 3, st_pairs, lane);
}

template <bool UNIT, int R>
cudaError_t launch_t(const DpArgs& args0, int num_sms, cudaStream_t st, int* warps_used, size_t scratch_bytes) {
    int bps = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, dp_kernel<UNIT, R>, 256, 0);
    if (err != cudaSuccess) return err;
    if (bps < 1) bps = 1;
    size_t warps = (size_t)num_sms * bps * 8;
    const size_t fit = scratch_bytes / args0.slot_bytes;
    if (warps > fit) warps = fit;
    if (warps > args0.P.num_pairs) warps = args0.P.num_pairs;
    if (warps == 0) { *warps_used = 0; return cudaSuccess; }
    DpArgs a = args0;
    a.nwarps = (uint32_t)warps;
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    dp_kernel<UNIT, R><<<blocks, 256, 0, st>>>(a);
    *warps_used = (int)warps;
    return cudaGetLastError();
}

}  // namespace

DpPlan plan_dp(bool unit, int band, uint32_t max_length, int64_t max_limit) {
    DpPlan p;
    p.unit = unit;
    p.band = band;
    p.blocks = band <= 31 ? 1 : band <= 63 ? 2 : 4;
    const size_t te = unit ? 1 : 2;
    const size_t rows = 2 * (size_t)max_length + 1;
    const size_t trace = align_up(rows * 32 * p.blocks * te, 16);
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
    if (plan.unit) {
        if (plan.blocks == 1) return launch_t<true, 1>(a, num_sms, st, warps_used, scratch_bytes);
        if (plan.blocks == 2) return launch_t<true, 2>(a, num_sms, st, warps_used, scratch_bytes);
        return launch_t<true, 4>(a, num_sms, st, warps_used, scratch_bytes);
    }
    if (plan.blocks == 1) return launch_t<false, 1>(a, num_sms, st, warps_used, scratch_bytes);
    if (plan.blocks == 2) return launch_t<false, 2>(a, num_sms, st, warps_used, scratch_bytes);
    return launch_t<false, 4>(a, num_sms, st, warps_used, scratch_bytes);
}

}  // namespace aim
