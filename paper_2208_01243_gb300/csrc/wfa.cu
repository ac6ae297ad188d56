// Gap-affine wavefront alignment (WFA, Section 2.4.4) with the canonical
// traceback, one warp per pair.
//
// Scores run in units of g = gcd(x, o, e) (every path cost is a sum of x,
// o+e and e, so every reachable score is a multiple of g): X = x/g,
// OE = (o+e)/g, E = e/g.  For score s and diagonal k = h - v the wavefront
// holds furthest-reaching offsets h (read position v = h - k):
//   I~[s,k] = max(M~[s-OE, k+1], I~[s-E, k+1])          (consumes a read base)
//   D~[s,k] = max(M~[s-OE, k-1], D~[s-E, k-1]) + 1      (consumes a target base)
//   f0      = max(M~[s-X, k] + 1, I~[s,k], D~[s,k])     (each candidate dropped if
//                                                        it leaves the matrix)
//   M~[s,k] = f0 + LCP(P[f0-k..], T[f0..])              (extend along matches)
// ("compute_next" then "extend"); the pair is done at the first s with
// M~[s, m-n] == m, and rejected once s passes the threshold (early exit).
// Lane j handles diagonals lo+j, lo+j+32, ...  The extend compares 32 bases
// at a time: a two-word funnel shift aligns each sequence to the current
// base, XOR marks mismatching bases, and clz/2 counts the leading matches.
//
// Every wavefront (M~, I~, D~ as int16 offsets) is kept in the warp's
// scratch for the traceback (the paper's WRAM+MRAM variant keeps all
// wavefront components in the larger memory and fetches what the next
// wavefront needs, Section 2.4.4).
//
// Traceback.  Along a diagonal with match cost 0, the optimal cost of each
// state is non-decreasing, so "state S of cell (v,h) is reachable with cost
// <= t" is exactly "h <= the furthest-reaching offset of S at some score
// <= t".  The backward greedy keeps, per state, the cost the remaining prefix
// must have; optimality of the whole alignment already rules out anything
// cheaper, so each "tight" test reduces to one furthest-reaching comparison:
//   X tight  iff mismatch and M~[cM - X, k] >= h - 1
//   I tight  iff I~[cI, k] >= h
//   D tight  iff D~[cD, k] >= h
//   M tight  iff match    and M~[cM, k] >= h - 1
// taken in the order X, I, D, M -- the same canonical alignment as the DP
// (among optimal alignments, ops read backward smallest under X < I < D < M).
// A run of M's continues while the bases match and neither I~[c,k] nor
// D~[c,k] reaches the current offset.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "aim_internal.cuh"

namespace aim {
namespace {

struct WfaArgs {
    int X, OE, E, g;
    int64_t smax;
    int band;
    PairsView P;
    LimitView L;
    OutView O;
    uint8_t* scratch;
    size_t slot_bytes;
    size_t hist_elems;
    size_t meta_off;     // byte offset of the per-score (lo, hi, base) table in a slot
    size_t runs_off;     // byte offset of the run staging area
    uint32_t runs_cap;
    uint32_t nwarps;
    uint32_t* counter;
};

struct Wf {
    int lo, hi, base, w;   // w == 0: empty
};

__device__ __forceinline__ Wf load_wf(const int* meta, int s) {
    Wf f;
    if (s < 0) { f.lo = 1; f.hi = 0; f.base = 0; f.w = 0; return f; }
    f.lo = meta[3 * s]; f.hi = meta[3 * s + 1]; f.base = meta[3 * s + 2];
    f.w = f.hi >= f.lo ? f.hi - f.lo + 1 : 0;
    return f;
}

// component c (0 M, 1 I, 2 D) of wavefront f at diagonal k, or a negative value
__device__ __forceinline__ int wf_get(const int16_t* hist, const Wf& f, int c, int k) {
    if (k < f.lo || k > f.hi) return kNeg16;
    return hist[f.base + c * f.w + (k - f.lo)];
}

// furthest offset reached from (h - k, h) along matches on diagonal k
__device__ __forceinline__ int extend(const uint64_t* Pw, uint32_t nwP, int n, const uint64_t* Tw, uint32_t nwT,
                                      int m, int k, int h, unsigned long long& words) {
    int v = h - k;
    while (v < n && h < m) {
        ++words;
        const uint64_t d = window32(Pw, nwP, (uint32_t)v) ^ window32(Tw, nwT, (uint32_t)h);
        const int rem = min(n - v, m - h);
        int adv = d ? (__clzll((long long)d) >> 1) : 32;
        if (adv > rem) adv = rem;
        v += adv; h += adv;
        if (adv < 32) break;
    }
    return h;
}

__global__ void __launch_bounds__(256) wfa_kernel(WfaArgs a) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gwarp >= a.nwarps) return;
    uint8_t* slot = a.scratch + (size_t)gwarp * a.slot_bytes;
    int16_t* hist = reinterpret_cast<int16_t*>(slot);
    int* meta = reinterpret_cast<int*>(slot + a.meta_off);
    uint32_t* staged = reinterpret_cast<uint32_t*>(slot + a.runs_off);
    const int X = a.X, OE = a.OE, E = a.E;
    unsigned long long st_cells = 0, st_words = 0, st_pairs = 0;

    for (;;) {
        uint32_t pi = 0;
        if (lane == 0) pi = atomicAdd(a.counter, 1u);
        pi = __shfl_sync(kFull, pi, 0);
        if (pi >= a.P.num_pairs) break;
        st_pairs += lane == 0;

        const int n = (int)a.P.read_len[pi], m = (int)a.P.target_len[pi];
        const int64_t lim = pair_limit(a.L, pi);
        const bool bad = pair_bad(a.P, pi) || (uint32_t)n > a.P.max_length ||
                         (uint32_t)m > a.P.max_length || lim == -2;
        if (bad) {
            if (lane == 0) write_header(a.O, pi, -1, AIM_F_BAD_PAIR, 0);
            continue;
        }
        const int kend = m - n;
        if (a.band >= 0 && (kend > a.band || -kend > a.band)) {
            if (lane == 0) write_header(a.O, pi, -1, AIM_F_REJECTED, 0);
            continue;
        }
        int64_t S64 = lim / a.g;
        if (S64 > a.smax) S64 = a.smax;
        const int S = (int)S64;
        const uint64_t* Pw = read_words(a.P, pi);
        const uint64_t* Tw = target_words(a.P, pi);
        const uint32_t nwP = (uint32_t)(n + 31) >> 5, nwT = (uint32_t)(m + 31) >> 5;
        const int klo = a.band >= 0 ? max(-n, -a.band) : -n;
        const int khi = a.band >= 0 ? min(m, a.band) : m;

        // score 0: diagonal 0 only
        int top = 3;
        int found = 0;
        if (lane == 0) {
            const int m0 = extend(Pw, nwP, n, Tw, nwT, m, 0, 0, st_words);
            ++st_cells;
            hist[0] = (int16_t)m0; hist[1] = kNeg16; hist[2] = kNeg16;
            meta[0] = 0; meta[1] = 0; meta[2] = 0;
            found = (kend == 0 && m0 >= m);
        }
        found = __shfl_sync(kFull, found, 0);
        __syncwarp();
        int s = 0;
        uint8_t status = 0;   // 0 running/found, AIM_F_REJECTED, AIM_F_STEP_CAP
        while (!found) {
            ++s;
            if (s > S) { status = AIM_F_REJECTED; break; }
            const Wf fx = load_wf(meta, s - X), fo = load_wf(meta, s - OE), fe = load_wf(meta, s - E);
            int lo = 1 << 30, hi = -(1 << 30);
            if (fx.w) { lo = min(lo, fx.lo); hi = max(hi, fx.hi); }
            if (fo.w) { lo = min(lo, fo.lo - 1); hi = max(hi, fo.hi + 1); }
            if (fe.w) { lo = min(lo, fe.lo - 1); hi = max(hi, fe.hi + 1); }
            lo = max(lo, klo); hi = min(hi, khi);
            if (lo > hi) {
                if (lane == 0) { meta[3 * s] = 1; meta[3 * s + 1] = 0; meta[3 * s + 2] = top; }
                __syncwarp();
                continue;
            }
            const int w = hi - lo + 1;
            if ((size_t)top + 3 * (size_t)w > a.hist_elems) { status = AIM_F_STEP_CAP; break; }
            bool hit = false;
            for (int k = lo + (int)lane; k <= hi; k += 32) {
                int ins = max(wf_get(hist, fo, 0, k + 1), wf_get(hist, fe, 1, k + 1));
                if (ins >= 0 && ins - k > n) ins = kNeg16;
                int del = max(wf_get(hist, fo, 0, k - 1), wf_get(hist, fe, 2, k - 1));
                del = del >= 0 ? del + 1 : kNeg16;
                if (del > m) del = kNeg16;
                int mis = wf_get(hist, fx, 0, k);
                mis = mis >= 0 ? mis + 1 : kNeg16;
                if (mis > m || mis - k > n) mis = kNeg16;
                const int f0 = max(mis, max(ins, del));
                const int mv = f0 >= 0 ? extend(Pw, nwP, n, Tw, nwT, m, k, f0, st_words) : kNeg16;
                ++st_cells;
                const int j = k - lo;
                hist[top + j] = (int16_t)mv;
                hist[top + w + j] = (int16_t)ins;
                hist[top + 2 * w + j] = (int16_t)del;
                hit |= (k == kend && mv >= m);
            }
            found = __any_sync(kFull, hit);
            if (lane == 0) { meta[3 * s] = lo; meta[3 * s + 1] = hi; meta[3 * s + 2] = top; }
            top += 3 * w;
            __syncwarp();
        }
        if (!found) {
            if (lane == 0) write_header(a.O, pi, -1, status, 0);
            continue;
        }
        const int32_t score = s * a.g;

        // canonical traceback on lane 0
        uint32_t nruns = 0;
        bool ok = true;
        if (lane == 0) {
            RunWriter wr;
            wr.init(staged, a.runs_cap);
            int v = n, h = m, cM = s, cI = s, cD = s;
            while (v > 0 || h > 0) {
                const int k = h - v;
                const bool diag = v > 0 && h > 0;
                const bool match = diag && base_at(Pw, v - 1) == base_at(Tw, h - 1);
                if (diag && !match && wf_get(hist, load_wf(meta, cM - X), 0, k) >= h - 1) {
                    const int c = cM - X;
                    cM = cI = cD = c; --v; --h;
                    wr.put(kOpMismatch, 1);
                } else if (v > 0 && wf_get(hist, load_wf(meta, cI), 1, k) >= h) {
                    const int c = cI;
                    cM = c - OE; cD = c - OE; cI = c - E; --v;
                    wr.put(kOpIns, 1);
                } else if (h > 0 && wf_get(hist, load_wf(meta, cD), 2, k) >= h) {
                    const int c = cD;
                    cM = c - OE; cI = c - OE; cD = c - E; --h;
                    wr.put(kOpDel, 1);
                } else if (match && wf_get(hist, load_wf(meta, cM), 0, k) >= h - 1) {
                    const int c = cM;
                    const Wf f = load_wf(meta, c);
                    const int stop = max(wf_get(hist, f, 1, k), wf_get(hist, f, 2, k));
                    int run = 0;
                    do {
                        --v; --h; ++run;
                    } while (v > 0 && h > 0 && h > stop && base_at(Pw, v - 1) == base_at(Tw, h - 1));
                    cM = cI = cD = c;
                    wr.put(kOpMatch, (uint32_t)run);
                } else {
                    ok = false;
                    break;
                }
            }
            wr.finish();
            nruns = wr.n;
            ok = ok && wr.n <= wr.cap;
        }
        __syncwarp();
        nruns = __shfl_sync(kFull, nruns, 0);
        ok = __shfl_sync(kFull, ok, 0);
        write_cigar(a.O, pi, score, staged, nruns, ok, lane);
        __syncwarp();
    }
    warp_stat_add(a.O.stats, 0, st_cells, lane);
    warp_stat_add(a.O.stats, 1, st_words, lane);
    warp_stat_add(a.O.stats, 3, st_pairs, lane);
}

int gcd_i(int a, int b) {
    while (b) { const int t = a % b; a = b; b = t; }
    return a < 0 ? -a : a;
}

}  // namespace

WfaPlan plan_wfa(const Costs& c, int band, uint32_t max_length, int64_t max_limit) {
    WfaPlan p;
    p.g = gcd_i(gcd_i(c.x, c.o), c.e);
    if (p.g <= 0) p.g = 1;
    p.x = c.x / p.g; p.oe = (c.o + c.e) / p.g; p.e = c.e / p.g;
    p.band = band;
    const int64_t L = max_length;
    const int64_t trivial = ((int64_t)c.x * L + c.o + (int64_t)c.e * L) / p.g;   // an alignment that always exists
    int64_t smax = max_limit >= kUnbounded ? trivial : max_limit / p.g;
    if (smax > trivial) smax = trivial;
    p.smax = smax;
    // worst-case wavefront ranges: every source wavefront non-empty
    const int64_t klo = band >= 0 ? -std::min<int64_t>(L, band) : -L;
    const int64_t khi = band >= 0 ? std::min<int64_t>(L, band) : L;
    std::vector<int64_t> lo(smax + 1), hi(smax + 1);
    lo[0] = 0; hi[0] = 0;
    size_t elems = 3;
    for (int64_t s = 1; s <= smax; ++s) {
        int64_t l = INT64_MAX, h = INT64_MIN;
        auto take = [&](int64_t src, int64_t grow) {
            if (src < 0 || lo[src] > hi[src]) return;
            l = std::min(l, lo[src] - grow); h = std::max(h, hi[src] + grow);
        };
        take(s - p.x, 0); take(s - p.oe, 1); take(s - p.e, 1);
        l = std::max(l, klo); h = std::min(h, khi);
        lo[s] = l; hi[s] = h;
        if (l <= h) elems += 3 * (size_t)(h - l + 1);
    }
    p.hist_elems = elems;
    const int64_t minc = std::min<int64_t>(p.x, p.oe);
    int64_t runs = 2 * L + 1;
    if (minc > 0) runs = std::min<int64_t>(runs, 2 * (smax / minc) + 1);
    p.runs_cap = (int)runs;
    const size_t meta_off = align_up(elems * sizeof(int16_t), 16);
    const size_t runs_off = align_up(meta_off + (size_t)(smax + 1) * 3 * sizeof(int), 16);
    p.slot_bytes = align_up(runs_off + (size_t)p.runs_cap * sizeof(uint32_t), 128);
    return p;
}

cudaError_t launch_wfa(const WfaPlan& plan, const Costs& c, const PairsView& P, const LimitView& L,
                       const OutView& O, uint8_t* scratch, size_t scratch_bytes, uint32_t* counter, int num_sms,
                       cudaStream_t st, int* warps_used) {
    (void)c;
    *warps_used = 0;
    if (P.num_pairs == 0) return cudaSuccess;
    WfaArgs a;
    a.X = plan.x; a.OE = plan.oe; a.E = plan.e; a.g = plan.g; a.smax = plan.smax; a.band = plan.band;
    a.P = P; a.L = L; a.O = O; a.scratch = scratch; a.slot_bytes = plan.slot_bytes;
    a.hist_elems = plan.hist_elems;
    a.meta_off = align_up(plan.hist_elems * sizeof(int16_t), 16);
    a.runs_off = align_up(a.meta_off + (size_t)(plan.smax + 1) * 3 * sizeof(int), 16);
    a.runs_cap = (uint32_t)plan.runs_cap;
    a.counter = counter;
    int bps = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, wfa_kernel, 256, 0);
    if (err != cudaSuccess) return err;
    if (bps < 1) bps = 1;
    size_t warps = (size_t)num_sms * bps * 8;
    const size_t fit = scratch_bytes / plan.slot_bytes;
    if (warps > fit) warps = fit;
    if (warps > P.num_pairs) warps = P.num_pairs;
    if (warps == 0) return cudaSuccess;
    a.nwarps = (uint32_t)warps;
    wfa_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(a);
    *warps_used = (int)warps;
    return cudaGetLastError();
}

}  // namespace aim
