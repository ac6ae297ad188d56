// Gap-affine wavefront alignment (WFA, Section 2.4.4) with the canonical
// traceback.  A group of G lanes (G = 1, 2, 4, 8, 16 or 32) aligns one pair; a warp
// runs 32/G pairs in lockstep over the score loop, so the per-score work of
// one pair is shared by G lanes and the warp-uniform bookkeeping by 32/G pairs.
// For very wide wavefronts (long, noisy pairs) a whole block of 256 threads
// aligns one pair (G = 256), with block barriers in place of warp votes.
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
// ("compute_next" then "extend").  A pair is done at the first s with
// M~[s, m-n] == m and rejected once s passes its threshold (early exit).
// Lane j of a group handles diagonals lo+j, lo+j+G, ...  The extend compares
// 32 bases at a time: a two-word funnel shift aligns each sequence to the
// current base, XOR marks mismatching bases, and clz/2 counts leading matches.
// Launches of groups up to 16 lanes first copy each pair's packed read and
// target into shared memory (when a block's copies fit in 24 KB), so their
// extends read at shared-memory latency.
// Each wavefront is trimmed to the diagonals that hold a valid entry, so the
// next range grows only from reachable diagonals.
//
// Every wavefront (M~, I~, D~ as int16 offsets) stays in the group's scratch
// for the traceback (the paper's WRAM+MRAM variant keeps all wavefront
// components in the larger memory and fetches what the next wavefront needs,
// Section 2.4.4).
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
// D~[c,k] reaches the current offset; its length comes from a backward
// comparison of 32-base windows (XOR, count trailing zero base pairs).
// A traceback is one lane's serial walk, so groups defer it: a group of up
// to 32 lanes finishes up to G pairs in fresh parts of its scratch arena and
// then traces them back side by side, lane j taking the j-th; a whole block
// keeps up to one pair per warp, traced back by the warp's first lane.
//
// Work distribution: a launch is compiled for one group size G and walks the
// buckets of that size (each a range of a pair order array); warps take 32/G
// consecutive positions of a bucket from its device counter and move to the
// next bucket when it is exhausted, so a longest-first bucket order leaves
// short pairs for the tail.  Callers with buckets of several sizes get one
// launch per size.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "aim_internal.cuh"

namespace aim {
namespace {

struct Wf {
    int lo, cnt, base, w;   // diagonals lo .. lo+cnt-1 (cnt == 0: empty); component c of diagonal k at element
                            // (base + k) * kEntryElems + c (base: first entry, already offset by -lo); w: set by
                            // the compact forms to the live-slot entry of diagonal 0
    int hi;                 // lo + cnt - 1, stored in the record (an empty record has lo > hi, far apart, so a
                            // union of source ranges needs no test for empty ones)
};
// a score record (lo, count, base, hi) and the empty one
constexpr int kEmptyLo = 1 << 29, kEmptyHi = -(1 << 29);
__device__ __forceinline__ int4 empty_rec() { return make_int4(kEmptyLo, 0, 0, kEmptyHi); }

// record of score s: element s & mask of rec (mask -1: the group's records in scratch; R-1: its ring of the
// last R scores in shared memory)
__device__ __forceinline__ Wf load_wf(const int4* rec, int s, int mask) {
    Wf f;
    if (s < 0) { f.lo = kEmptyLo; f.cnt = 0; f.base = 0; f.w = 0; f.hi = kEmptyHi; return f; }
    const int4 q = rec[s & mask];
    f.lo = q.x; f.cnt = q.y; f.base = q.z; f.w = 0; f.hi = q.w;
    return f;
}

__device__ __forceinline__ Wf load_wf(const int* meta, int s) {
    Wf f;
    if (s < 0) { f.lo = kEmptyLo; f.cnt = 0; f.base = 0; f.w = 0; f.hi = kEmptyHi; return f; }
    const int4 q = reinterpret_cast<const int4*>(meta)[s];
    f.lo = q.x; f.cnt = q.y; f.base = q.z; f.w = 0; f.hi = q.w;
    return f;
}

// the same for a score s >= -rec_pad of a pair region whose padding records are written (no check)
__device__ __forceinline__ Wf load_rec(const int* meta, int s) {
    const int4 q = reinterpret_cast<const int4*>(meta)[s];
    Wf f;
    f.lo = q.x; f.cnt = q.y; f.base = q.z; f.w = 0; f.hi = q.w;
    return f;
}

// component c (0 M, 1 I, 2 D) of wavefront f at diagonal k, or a negative value
__device__ __forceinline__ int wf_get(const int16_t* hist, const Wf& f, int c, int k) {
    if ((unsigned)(k - f.lo) >= (unsigned)f.cnt) return kNeg16;   // one compare covers both ends and empty
    return hist[(f.base + k) * kEntryElems + c];
}

// Storage forms of the wavefronts (one kernel instance each):
//   kFmt8   every wavefront kept whole: one 8-byte entry (M~, I~, D~ as int16 and a spare slot) per (score,
//           diagonal), which the forward pass reads back and the traceback reads (short reads: offsets < 32,768).
//   kFmt16  long reads: the forward pass reads and writes the last few wavefronts whole in a small "live" ring of
//           slots (entries as in kFmt8), and the history keeps one 16-bit word per (score, diagonal): h + 1 of M~
//           in bits 0-13 (0: invalid; reads up to 16,382 bp) and two source bits, set when I~ (bit 14) or D~
//           (bit 15) came from the gap extension rather than the opening.  The traceback rebuilds I~ and D~ by
//           following those bits back to the gap's opening.  A quarter of kFmt8's history bytes.
//   kFmt32  the same with 32-bit words (h + 1 in bits 0-29, source bits 30 and 31) and int32 live entries, for
//           reads beyond 16,382 bp: half of kFmt8's bytes, and no 32,000 bp limit.
//   kFmtBound  no history at all, only the live ring (int16 entries): the bound pass, a pruned forward pass whose
//           only result is the score at which it reached the end (an upper bound on the pair's optimum, since
//           every entry it computes is an offset some path of that score reaches), for a following exact pass to
//           clamp its wavefronts with.
enum : int { kFmt8 = 0, kFmt16 = 1, kFmt32 = 2, kFmtBound = 3 };
template <int FMT>
struct FmtT {                       // kFmt8, kFmt16, kFmtBound
    using V = int16_t;              // live value type
    using H = uint16_t;             // history word (compact forms)
    static constexpr int kNeg = kNeg16;
    static constexpr int kBits = 14;
};
template <>
struct FmtT<kFmt32> {
    using V = int32_t;
    using H = uint32_t;
    static constexpr int kNeg = -(1 << 30);
    static constexpr int kBits = 30;
};

// component c of wavefront f at diagonal k in a live ring slot, or a negative value.  A slot holds diagonal k at
// entry f.w + k (f.w: the slot's first entry plus its centre; every diagonal a pair reaches by score smax lies
// within smax / E + 1 of 0, and a slot is wider than twice that).
template <int FMT>
__device__ __forceinline__ int live_get(const typename FmtT<FMT>::V* live, const Wf& f, int c, int k) {
    if ((unsigned)(k - f.lo) >= (unsigned)f.cnt) return FmtT<FMT>::kNeg;
    return live[(size_t)(f.w + k) * kEntryElems + c];
}

// a compact history word for offset mv (negative: invalid) and the two source bits
template <int FMT>
__device__ __forceinline__ typename FmtT<FMT>::H hist_word(int mv, bool ins_ext, bool del_ext) {
    using H = typename FmtT<FMT>::H;
    constexpr int B = FmtT<FMT>::kBits;
    return (H)((uint32_t)(mv >= 0 ? mv + 1 : 0) | ((uint32_t)ins_ext << B) | ((uint32_t)del_ext << (B + 1)));
}

// 32 bases starting at base pos of a sequence of nwords words in global memory, for pos inside the sequence
// (so word pos / 32 exists); the word after it reads as 0 past the end.
__device__ __forceinline__ uint64_t window_in(const uint64_t* __restrict__ w, uint32_t nwords, uint32_t pos) {
    const uint32_t wi = pos >> 5, sh = 2 * (pos & 31);
    const uint64_t hi = __ldg(w + wi);
    const uint64_t lo = wi + 1 < nwords ? __ldg(w + wi + 1) : 0ull;
    return join_window(hi, lo, sh);
}

// dynamic shared memory of staged launches: copies of the pairs' packed sequences, one slot per group, then
// each group's ring of recent score records (at byte offset ring_off)
extern __shared__ uint64_t s_seq[];

// the same window from a copy at word offset `off` of s_seq, which holds a spare word after the sequence, so
// both loads stay inside it without a check
__device__ __forceinline__ uint64_t window_shared(uint32_t off, uint32_t pos) {
    const uint32_t wi = off + (pos >> 5), sh = 2 * (pos & 31);
    return join_window(s_seq[wi], s_seq[wi + 1], sh);
}

// the extend's view of one pair: global memory, or the group's copies in shared memory
template <bool STAGE>
struct PairSeqs;
template <>
struct PairSeqs<false> {
    const uint64_t *P, *T;
    uint32_t nwP, nwT;
    __device__ uint64_t read_window(uint32_t pos) const { return window_in(P, nwP, pos); }
    __device__ uint64_t target_window(uint32_t pos) const { return window_in(T, nwT, pos); }
};
template <>
struct PairSeqs<true> {
    uint32_t offP, offT;
    __device__ uint64_t read_window(uint32_t pos) const { return window_shared(offP, pos); }
    __device__ uint64_t target_window(uint32_t pos) const { return window_shared(offT, pos); }
};

// furthest offset reached from (h - k, h) along matches on diagonal k; a negative h (no valid start) comes back
// unchanged without reading the sequences
template <bool STAGE>
__device__ __forceinline__ int extend(const PairSeqs<STAGE>& q, int n, int m, int k, int h, uint32_t& windows) {
    int v = h - k;
    int rem = h >= 0 ? min(n - v, m - h) : 0;   // bases left on both sequences (none for an invalid start)
    while (rem > 0) {
        ++windows;
        const uint64_t d = q.read_window((uint32_t)v) ^ q.target_window((uint32_t)h);
        const int adv = min(__clzll((long long)d) >> 1, rem);   // __clzll(0) = 64: the whole window matches
        v += adv; h += adv; rem -= adv;
        if (adv < 32) break;
    }
    return h;
}

// 32 bases ending at base p (inclusive) with base p in the low two bits; for
// p < 31 only bases 0..p are present (in the low bits).
__device__ __forceinline__ uint64_t window_ending(const uint64_t* w, uint32_t nwords, int p) {
    if (p >= 31) return window32(w, nwords, (uint32_t)(p - 31));
    return window32(w, nwords, 0) >> (2 * (31 - p));
}

// number of consecutive matches P[v-1-i] == T[h-1-i], i = 0, 1, ... (at most min(v, h))
__device__ __forceinline__ int match_run_back(const uint64_t* Pw, uint32_t nwP, int v, const uint64_t* Tw,
                                              uint32_t nwT, int h) {
    int run = 0;
    for (;;) {
        const int pv = v - 1 - run, ph = h - 1 - run;
        if (pv < 0 || ph < 0) break;
        const uint64_t d = window_ending(Pw, nwP, pv) ^ window_ending(Tw, nwT, ph);
        const int avail = min(min(pv, ph) + 1, 32);
        int z = d ? ((__ffsll((long long)d) - 1) >> 1) : 32;
        if (z > avail) z = avail;
        run += z;
        if (z < 32) break;
    }
    return run;
}

enum : int { kRun = 0, kDone = 1, kRejected = 2, kCap = 3, kBad = 4, kIdle = 5 };

// Collectives of one group.  G <= 32: a warp holds 32/G groups that run in lockstep, so loop
// conditions are warp-wide and group results come from masked ballots and butterflies.  G == 256:
// the whole block is one group and block barriers carry the same results.
template <int G, bool BLOCK = (G > 32)>
struct Group;

template <int G>
struct Group<G, false> {
    int gl, leader;
    uint32_t gmask;
    __device__ explicit Group(uint32_t lane) {
        gl = (int)lane % G;
        leader = (int)lane - gl;
        gmask = G == 32 ? kFull : (((1u << G) - 1u) << leader);
    }
    __device__ int index(uint32_t lane) const { return (int)lane / G; }
    // with G == 32 the warp is one group, whose status and width every lane computes alike: no vote needed
    __device__ bool any_running(bool x) const {
        if constexpr (G == 32) return x;
        else return __any_sync(kFull, x);
    }
    __device__ int iterations(int w) const {
        if constexpr (G == 32) return (w + 31) / 32;
        else return (int)__reduce_max_sync(kFull, (unsigned)((w + G - 1) / G));
    }
    __device__ void min_max(int& lo, int& hi) const {
        if constexpr (G == 32) {   // the whole warp is one group: one warp-wide reduction each
            lo = __reduce_min_sync(kFull, lo);
            hi = __reduce_max_sync(kFull, hi);
        } else {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                lo = min(lo, __shfl_xor_sync(kFull, lo, o));
                hi = max(hi, __shfl_xor_sync(kFull, hi, o));
            }
        }
    }
    __device__ bool group_any(bool x) const {
        if constexpr (G == 32) return __any_sync(kFull, x);
        else return (__ballot_sync(kFull, x) & gmask) != 0;
    }
    __device__ int bcast(int x) const { return __shfl_sync(kFull, x, leader); }
    __device__ void sync() const { __syncwarp(); }
};

template <int G>
struct Group<G, true> {
    int gl, leader;
    __device__ explicit Group(uint32_t) { gl = (int)threadIdx.x; leader = 0; }
    __device__ int index(uint32_t) const { return 0; }
    __device__ bool any_running(bool x) const { return __syncthreads_or(x) != 0; }
    __device__ int iterations(int w) const { return (w + G - 1) / G; }   // w is block-uniform
    __device__ void min_max(int& lo, int& hi) const {
        __shared__ int s_lo, s_hi;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(kFull, lo, o));
            hi = max(hi, __shfl_xor_sync(kFull, hi, o));
        }
        if (threadIdx.x == 0) { s_lo = 1 << 30; s_hi = -(1 << 30); }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) { atomicMin(&s_lo, lo); atomicMax(&s_hi, hi); }
        __syncthreads();
        lo = s_lo; hi = s_hi;
        __syncthreads();
    }
    __device__ bool group_any(bool x) const { return __syncthreads_or(x) != 0; }
    __device__ int bcast(int x) const {
        __shared__ int s_v;
        if (threadIdx.x == 0) s_v = x;
        __syncthreads();
        const int r = s_v;
        __syncthreads();
        return r;
    }
    __device__ void sync() const { __syncthreads(); }
};

struct Counters {
    unsigned long long cells, windows, pairs;
};

// Result of a pair's forward pass: its status, the score it ended at, the history entries it used.
struct Forward {
    int status, final_s, top;
    uint32_t pi;
};

// Forward pass of one step of the warp's work: groups g = 0 .. 32/G - 1 take the pairs at order positions
// q0 + g (those < qend), each in its own region of region_bytes (meta records, run staging, history).  All
// lanes must call this together.  The traceback runs later, from the region as this leaves it.
// ADAPT: WFA-adaptive pruning (a kernel of its own, so the exact algorithm carries none of its registers).
// STAGE: each group first copies its pair's packed read and target into its slot of s_seq (the launch gives
// every group a slot of 2 * seq_slot_words words) and the extend reads the copies.
template <int G, bool ADAPT, bool STAGE, int FMT>
__device__ __forceinline__ Forward forward_pair(const WfaArgs& a, uint8_t* region, size_t region_bytes, uint32_t q0,
                                                uint32_t qend, uint32_t lane, Counters& st) {
    static_assert(!STAGE || G <= 32, "sequence staging is per group of a warp");
    static_assert(FMT == kFmt8 || (!ADAPT && !STAGE), "compact histories are for the exact, unstaged kernels");
    static_assert(FMT != kFmtBound, "bound passes run bound_pass_run");
    using V = typename FmtT<FMT>::V;
    using H = typename FmtT<FMT>::H;
    constexpr int kNeg = FmtT<FMT>::kNeg;
    const Group<G> grp(lane);
    const int g = grp.index(lane), gl = grp.gl;
    int* meta = reinterpret_cast<int*>(region + (size_t)a.rec_pad * sizeof(int4));   // record 0
    // kFmt8: the history holds every wavefront whole and the forward pass reads it back.  Compact forms: the live
    // ring sits at the end of the region (each forward pass of the group uses the same place), the history of
    // compact words after the run staging.
    int16_t* hist = reinterpret_cast<int16_t*>(region + a.meta_bytes + a.runs_bytes);
    H* hc = reinterpret_cast<H*>(region + a.meta_bytes + a.runs_bytes);
    V* live = reinterpret_cast<V*>(region + region_bytes - (FMT == kFmt8 ? 0 : a.live_bytes));
    const size_t hist_cap = FMT == kFmt8
        ? (region_bytes - a.meta_bytes - a.runs_bytes) / (kEntryElems * sizeof(int16_t))
        : (region_bytes - a.meta_bytes - a.runs_bytes - a.live_bytes) / sizeof(H);
    const int hist_cap32 = (int)(hist_cap < (size_t)INT32_MAX ? hist_cap : (size_t)INT32_MAX);
    const int center = (int)(a.live_w / 2);
    const int X = a.X, OE = a.OE, E = a.E;

    const uint32_t q = q0 + (uint32_t)g;
    int status = kIdle;
    uint32_t pi = 0;
    int n = 0, m = 0, S = 0, kend = 0, klo = 0, khi = 0;
    const uint64_t *Pw = nullptr, *Tw = nullptr;
    uint32_t nwP = 0, nwT = 0;
    if (q < qend && a.retry_only && a.O.flags[a.order ? a.order[q] : q] != AIM_F_STEP_CAP) {
        // second pass: this pair already has its result
    } else if (q < qend) {
        pi = a.order ? a.order[q] : q;
        n = (int)a.P.read_len[pi];
        m = (int)a.P.target_len[pi];
        const int64_t lim = pair_limit(a.L, pi);
        kend = m - n;
        if (pair_bad(a.P, pi) || (uint32_t)n > a.P.max_length || (uint32_t)m > a.P.max_length || lim == -2) {
            status = kBad;
        } else if (a.band >= 0 && (kend > a.band || -kend > a.band)) {
            status = kRejected;
        } else {
            status = kRun;
            int64_t S64 = lim / a.g;
            S = (int)(S64 > a.smax ? a.smax : S64);
            // a bound pass found an alignment of score ub (scaled): the optimum is at most ub, so a limit of ub
            // rejects nothing the limit S would accept, and the reach clamp below keeps fewer diagonals
            if (a.bound) {
                const int ub = a.bound[pi];
                if (ub >= 0 && ub < S) S = ub;
            }
            Pw = read_words(a.P, pi);
            Tw = target_words(a.P, pi);
            nwP = (uint32_t)(n + 31) >> 5;
            nwT = (uint32_t)(m + 31) >> 5;
            klo = a.band >= 0 ? max(-n, -a.band) : -n;
            khi = a.band >= 0 ? min(m, a.band) : m;
        }
        if (gl == 0) st.pairs += 1;
    }

    // reach = (S - s) / E for the current score s, kept by a remainder instead of a division per score
    int reach = 0, rrem = 0;
    if (status == kRun) { reach = S / E; rrem = S - reach * E; }

    // the extend's view of the pair: with STAGE, the group's copy in shared memory (a spare zero word after
    // each sequence), read at shared-memory latency
    PairSeqs<STAGE> seqs;
    if constexpr (STAGE) {
        const uint32_t slot = (threadIdx.x >> 5) * (uint32_t)(32 / G) + (uint32_t)g;
        seqs.offP = slot * 2 * a.seq_slot_words;
        seqs.offT = seqs.offP + a.seq_slot_words;
        if (status == kRun) {
            for (uint32_t j = (uint32_t)gl; j < nwP; j += (uint32_t)G) s_seq[seqs.offP + j] = __ldg(Pw + j);
            for (uint32_t j = (uint32_t)gl; j < nwT; j += (uint32_t)G) s_seq[seqs.offT + j] = __ldg(Tw + j);
            if (gl == 0) { s_seq[seqs.offP + nwP] = 0; s_seq[seqs.offT + nwT] = 0; }
        }
        grp.sync();
    } else {
        seqs.P = Pw; seqs.T = Tw; seqs.nwP = nwP; seqs.nwT = nwT;
    }

    // exact staged launches: the records the next scores read come from a ring of the last meta_ring scores in
    // shared memory, when the launch gives one (the records in scratch stay for the traceback).  Groups of 32
    // lanes, whole blocks and the adaptive kernels read their records from scratch: a ring measured slower there.
    constexpr bool kRing = STAGE && !ADAPT;
    const int4* src = reinterpret_cast<const int4*>(meta);
    int4* ring = nullptr;
    int mask = -1;
    if constexpr (kRing) {
        if (a.meta_ring) {
            const uint32_t gib = (threadIdx.x >> 5) * (uint32_t)(32 / G) + (uint32_t)g;
            ring = reinterpret_cast<int4*>(reinterpret_cast<char*>(s_seq) + a.ring_off) + (size_t)gib * a.meta_ring;
            src = ring;
            mask = (int)a.meta_ring - 1;
        }
    }

    // the empty records before record 0 (the sources of the first scores), written by the group's lanes
    if (status == kRun)
        for (int j = gl; j < (int)a.rec_pad; j += G) reinterpret_cast<int4*>(meta)[-1 - j] = empty_rec();

    // score 0: diagonal 0 only.  The pair's entries (top) and extend windows are added to the launch's counters
    // once, at its end.
    uint32_t pair_windows = 0;
    int top = 0, final_s = 0;
    int found0 = 0;
    if (status == kRun && gl == 0) {
        const int m0 = extend<STAGE>(seqs, n, m, 0, 0, pair_windows);
        if constexpr (FMT == kFmt8) {
            hist[0] = (int16_t)m0; hist[1] = kNeg16; hist[2] = kNeg16; hist[3] = 0;
        } else {   // live slot 0 at diagonal 0; history word 0
            V* e0 = live + (size_t)center * kEntryElems;
            e0[0] = (V)m0; e0[1] = (V)kNeg; e0[2] = (V)kNeg; e0[3] = 0;
            hc[0] = hist_word<FMT>(m0, false, false);
        }
        reinterpret_cast<int4*>(meta)[0] = make_int4(0, 1, 0, 0);
        if (kRing && ring) ring[0] = make_int4(0, 1, 0, 0);
        found0 = (kend == 0 && m0 >= m);
    }
    found0 = grp.bcast(found0);
    if (status == kRun) {
        top = 1;   // entries used
        if (found0) status = kDone;
    }
    grp.sync();

    int s = 0;
    while (grp.any_running(status == kRun)) {
        ++s;
        if (--rrem < 0) { rrem += E; --reach; }
        bool run = status == kRun;
        if (run && s > S) { status = kRejected; run = false; }
        int lo = 0, hi = -1, w = 0;
        Wf fx, fo, fe;
        if (run) {
            if constexpr (kRing) {
                fx = load_wf(src, s - X, mask); fo = load_wf(src, s - OE, mask); fe = load_wf(src, s - E, mask);
            } else {
                fx = load_rec(meta, s - X); fo = load_rec(meta, s - OE); fe = load_rec(meta, s - E);
            }
            if constexpr (FMT != kFmt8) {   // Wf.w becomes the entry of diagonal 0 in the source's live slot
                const uint32_t sm = a.live_slots - 1;
                fx.w = (int)(((uint32_t)(s - X) & sm) * a.live_w) + center;
                fo.w = (int)(((uint32_t)(s - OE) & sm) * a.live_w) + center;
                fe.w = (int)(((uint32_t)(s - E) & sm) * a.live_w) + center;
            }
            // the union of the sources' ranges, the gap sources one diagonal wider (an empty one is neutral)
            lo = min(fx.lo, min(fo.lo, fe.lo) - 1);
            hi = max(fx.hi, max(fo.hi, fe.hi) + 1);
            lo = max(lo, klo); hi = min(hi, khi);
            if constexpr (!ADAPT) {
                // threshold: a path through diagonal k at score s still has to reach the end diagonal, a gap of
                // |k - kend| bases costing at least E each, so only diagonals within (S - s) / E of kend can lie on
                // an alignment of score <= S.  The sources of every entry kept lie within the same bound, so each
                // kept entry has its exact value, and the traceback only reads entries on optimal paths (a prefix
                // of cost c at diagonal k has c + E |k - kend| <= optimum <= S).
                lo = max(lo, kend - reach); hi = min(hi, kend + reach);
            }
            w = lo <= hi ? hi - lo + 1 : 0;
            if (w && (top + w > hist_cap32 ||
                      (FMT != kFmt8 && (lo + center < 0 || hi + center >= (int)a.live_w)))) {
                status = kCap; run = false; w = 0; hi = lo - 1;
            }
        }
        const int iters = grp.iterations(w);
        int mv_end = kNeg16;   // M~ on the end diagonal kend, in the lane that computes it
        int vlo = 1 << 30, vhi = -(1 << 30);   // trimmed range: diagonals holding a valid entry
        const int base = top - lo;
        const int live_slot = FMT == kFmt8 ? 0 : (int)(((uint32_t)s & (a.live_slots - 1)) * a.live_w) + center;
        int dmin = 1 << 30, dmax = -(1 << 30);   // WFA-adaptive: distances of the new entries to the end cell
        for (int it = 0; it < iters; ++it) {
            const int k = lo + gl + it * G;
            if (k <= hi) {   // a group that does not run this score has an empty range (hi < lo)
                // a candidate offset h is valid iff 0 <= h <= min(m, n + k) (h <= m and v = h - k <= n): one
                // unsigned comparison, since an invalid source entry is kNeg16 and stays negative after + 1
                const unsigned hmax = (unsigned)min(m, n + k);
                int ins, del, mis;
                bool ins_ext = false, del_ext = false;
                if constexpr (FMT == kFmt8) {
                    ins = max(wf_get(hist, fo, 0, k + 1), wf_get(hist, fe, 1, k + 1));
                    del = max(wf_get(hist, fo, 0, k - 1), wf_get(hist, fe, 2, k - 1)) + 1;
                    mis = wf_get(hist, fx, 0, k) + 1;
                } else {   // sources from the live ring; the source bits record which term won (ties: the opening)
                    const int oi = live_get<FMT>(live, fo, 0, k + 1), ei = live_get<FMT>(live, fe, 1, k + 1);
                    const int od = live_get<FMT>(live, fo, 0, k - 1), ed = live_get<FMT>(live, fe, 2, k - 1);
                    ins_ext = ei > oi; del_ext = ed > od;
                    ins = max(oi, ei);
                    del = max(od, ed) + 1;
                    mis = live_get<FMT>(live, fx, 0, k) + 1;
                }
                if ((unsigned)ins > hmax) ins = kNeg;
                if ((unsigned)del > hmax) del = kNeg;
                if ((unsigned)mis > hmax) mis = kNeg;
                const int f0 = max(mis, max(ins, del));   // >= 0 iff any candidate is valid
                const int mv = extend<STAGE>(seqs, n, m, k, f0, pair_windows);   // f0 stays negative if invalid
                if constexpr (FMT == kFmt8) {
                    *reinterpret_cast<uint64_t*>(hist + (size_t)(base + k) * kEntryElems) =
                        (uint64_t)(uint16_t)mv | ((uint64_t)(uint16_t)ins << 16) | ((uint64_t)(uint32_t)del << 32);
                    // (the spare slot, bits 48-63, takes del's sign bits: nothing reads it)
                } else {
                    V* e = live + (size_t)(live_slot + k) * kEntryElems;
                    if constexpr (FMT != kFmt32)
                        *reinterpret_cast<uint64_t*>(e) = (uint64_t)(uint16_t)mv | ((uint64_t)(uint16_t)ins << 16) |
                                                          ((uint64_t)(uint32_t)del << 32);
                    else
                        *reinterpret_cast<int4*>(e) = make_int4(mv, ins, del, 0);
                    hc[base + k] = hist_word<FMT>(mv, ins_ext, del_ext);
                }
                if (k == kend) mv_end = mv;
                if (f0 >= 0) { vlo = min(vlo, k); vhi = max(vhi, k); }
                if (ADAPT && mv >= 0) {
                    const int dist = max(n - (mv - k), m - mv);
                    dmin = min(dmin, dist);
                    dmax = max(dmax, dist);
                }
            }
        }
        grp.min_max(vlo, vhi);   // group-wide trimmed range
        const bool group_hit = grp.group_any(mv_end >= m);
        if constexpr (ADAPT) {
            // WFA-adaptive: once the wavefront spans at least adapt_min_len diagonals, drop outer diagonals
            // whose distance to the end cell, max(n - v, m - h), exceeds the smallest by more than
            // adapt_max_dist.  The loop above gave each lane the smallest and largest distance of its
            // entries; the pass over the wavefront runs only where some entry is that far out.
            grp.min_max(dmin, dmax);
            const bool prune = run && !group_hit && vlo <= vhi && vhi - vlo + 1 >= a.adapt_min_len &&
                               dmax - dmin > a.adapt_max_dist;
            if (grp.any_running(prune)) {
                int klo = 1 << 30, khi = -(1 << 30);
                for (int it = 0; it < iters; ++it) {
                    const int k = lo + gl + it * G;
                    if (prune && k >= vlo && k <= vhi) {
                        const int h = hist[(size_t)(base + k) * kEntryElems];
                        if (h >= 0 && max(n - (h - k), m - h) - dmin <= a.adapt_max_dist) {
                            klo = min(klo, k);
                            khi = max(khi, k);
                        }
                    }
                }
                grp.min_max(klo, khi);
                if (prune) { vlo = klo; vhi = khi; }
            }
        }
        if (run) {
            if (gl == 0) {
                const int4 rec = vlo <= vhi ? make_int4(vlo, vhi - vlo + 1, base, vhi) : empty_rec();
                reinterpret_cast<int4*>(meta)[s] = rec;
                if (kRing && ring) ring[s & mask] = rec;
            }
            top += w;
            if (group_hit) { status = kDone; final_s = s; }
        }
        grp.sync();
    }

    if (gl == 0) st.cells += (unsigned)top;   // the pair's entries, computed by the group's lanes
    st.windows += pair_windows;
    return Forward{status, final_s, top, pi};
}

// Bound pass with asynchronous groups: each group of G lanes runs its own pair and, the moment that pair ends,
// records its bound and claims the next pair, which starts at score 0 while the warp's other groups carry on; a
// warp never waits for its slowest pair (error rates vary tenfold within a bucket).  Every lane of the warp runs
// each score step, each group on its own pair and score; the collectives are group-local and only the count of
// diagonal iterations is warp-wide.  The step is the forward recurrence of the live-ring form with the pruning of
// WFA-adaptive and the threshold clamp; nothing is kept for a traceback.
template <int G, bool STAGE>
__device__ __forceinline__ void bound_pass_run(const WfaArgs& a, int b, uint8_t* warp_slot, uint32_t lane,
                                               Counters& st) {
    static_assert(G <= 32, "bound passes use groups of a warp");
    using V = int16_t;
    constexpr int kNeg = kNeg16;
    constexpr int P = 32 / G;
    const Group<G> grp(lane);
    const int g = grp.index(lane), gl = grp.gl;
    const uint32_t begin = a.bounds ? a.bounds[b] : 0;
    const uint32_t end = a.bounds ? a.bounds[b + 1] : a.P.num_pairs;
    const uint32_t arena16 = (uint32_t)((a.warp_bytes / P) >> 4);
    uint8_t* region = warp_slot + ((size_t)g * arena16 << 4);
    const int* meta = reinterpret_cast<const int*>(region + (size_t)a.rec_pad * sizeof(int4));   // record 0
    int4* rec = reinterpret_cast<int4*>(region + (size_t)a.rec_pad * sizeof(int4));
    V* live = reinterpret_cast<V*>(region + ((size_t)arena16 << 4) - a.live_bytes);
    const int center = (int)(a.live_w / 2);
    const uint32_t smask = a.live_slots - 1;
    const int X = a.X, OE = a.OE, E = a.E;
    PairSeqs<STAGE> seqs;
    if constexpr (STAGE) {
        const uint32_t slot = (threadIdx.x >> 5) * (uint32_t)P + (uint32_t)g;
        seqs.offP = slot * 2 * a.seq_slot_words;
        seqs.offT = seqs.offP + a.seq_slot_words;
    }
    int status = kIdle;   // kRun: the group's pair is running; otherwise it takes the next one
    uint32_t p_cells = 0, p_windows = 0;   // the running pair's entries and windows, added to st when it ends
    bool more = true;     // the queue may still hold pairs
    uint32_t pi = 0;
    int n = 0, m = 0, S = 0, kend = 0, klo = 0, khi = 0, s = 0, reach = 0, rrem = 0;
    for (;;) {
        const bool need = status != kRun && more;
        if (__any_sync(kFull, need)) {
            uint32_t pos = 0;
            if (need && gl == 0) pos = atomicAdd(a.counters + b, 1u);
            pos = (uint32_t)grp.bcast((int)pos);
            bool fresh = false;   // the group starts a pair now
            if (need) {
                if (pos >= end - begin || end <= begin) {
                    more = false;
                } else {
                    pi = a.order ? a.order[begin + pos] : begin + pos;
                    n = (int)a.P.read_len[pi];
                    m = (int)a.P.target_len[pi];
                    const int64_t lim = pair_limit(a.L, pi);
                    kend = m - n;
                    const bool usable = !pair_bad(a.P, pi) && (uint32_t)n <= a.P.max_length &&
                                        (uint32_t)m <= a.P.max_length && lim != -2 &&
                                        (a.band < 0 || (kend <= a.band && -kend <= a.band));
                    if (!usable) {
                        if (gl == 0) a.bound[pi] = -1;   // the exact pass reports the pair
                    } else {
                        const int64_t S64 = lim / a.g;
                        S = (int)(S64 > a.smax ? a.smax : S64);
                        klo = a.band >= 0 ? max(-n, -a.band) : -n;
                        khi = a.band >= 0 ? min(m, a.band) : m;
                        reach = S / E; rrem = S - reach * E;
                        s = 0;
                        fresh = true;
                    }
                }
            }
            const uint64_t* Pw = fresh ? read_words(a.P, pi) : nullptr;
            const uint64_t* Tw = fresh ? target_words(a.P, pi) : nullptr;
            const uint32_t nwP = (uint32_t)(n + 31) >> 5, nwT = (uint32_t)(m + 31) >> 5;
            if constexpr (STAGE) {
                if (fresh) {
                    for (uint32_t j = (uint32_t)gl; j < nwP; j += (uint32_t)G) s_seq[seqs.offP + j] = __ldg(Pw + j);
                    for (uint32_t j = (uint32_t)gl; j < nwT; j += (uint32_t)G) s_seq[seqs.offT + j] = __ldg(Tw + j);
                    if (gl == 0) { s_seq[seqs.offP + nwP] = 0; s_seq[seqs.offT + nwT] = 0; }
                }
                __syncwarp();
            } else if (fresh) {
                seqs.P = Pw; seqs.T = Tw; seqs.nwP = nwP; seqs.nwT = nwT;
            }
            if (fresh)   // the empty records before record 0
                for (int j = gl; j < (int)a.rec_pad; j += G) rec[-1 - j] = empty_rec();
            // score 0: diagonal 0 only (live slot 0)
            int found0 = 0;
            if (fresh && gl == 0) {
                const int m0 = extend<STAGE>(seqs, n, m, 0, 0, p_windows);
                ++p_cells;
                *reinterpret_cast<uint64_t*>(live + (size_t)center * kEntryElems) =
                    (uint64_t)(uint16_t)m0 | ((uint64_t)(uint16_t)kNeg << 16) | ((uint64_t)(uint16_t)kNeg << 32);
                rec[0] = make_int4(0, 1, 0, 0);
                found0 = kend == 0 && m0 >= m;
            }
            found0 = grp.bcast(found0);
            if (fresh) {
                if (found0) {
                    if (gl == 0) a.bound[pi] = 0;
                    st.cells += p_cells; st.windows += p_windows; p_cells = p_windows = 0;
                } else {
                    status = kRun;
                }
            }
            __syncwarp();
        }
        if (!__any_sync(kFull, status == kRun)) {
            if (__any_sync(kFull, more)) continue;   // groups whose pair could not run claim again
            break;
        }
        // one score step of every running group
        bool run = status == kRun;
        if (run) {
            ++s;
            if (--rrem < 0) { rrem += E; --reach; }
            if (s > S) { status = kRejected; run = false; }
        }
        int lo = 0, hi = -1, w = 0;
        Wf fx{0, 0, 0, 0}, fo{0, 0, 0, 0}, fe{0, 0, 0, 0};
        if (run) {
            fx = load_rec(meta, s - X); fo = load_rec(meta, s - OE); fe = load_rec(meta, s - E);
            fx.w = (int)(((uint32_t)(s - X) & smask) * a.live_w) + center;
            fo.w = (int)(((uint32_t)(s - OE) & smask) * a.live_w) + center;
            fe.w = (int)(((uint32_t)(s - E) & smask) * a.live_w) + center;
            // the union of the sources' ranges, the gap sources one diagonal wider (an empty one is neutral)
            lo = min(fx.lo, min(fo.lo, fe.lo) - 1);
            hi = max(fx.hi, max(fo.hi, fe.hi) + 1);
            lo = max(lo, klo); hi = min(hi, khi);
            lo = max(lo, kend - reach); hi = min(hi, kend + reach);   // the threshold clamp
            w = lo <= hi ? hi - lo + 1 : 0;
            if (w && (lo + center < 0 || hi + center >= (int)a.live_w)) { status = kCap; run = false; w = 0; hi = lo - 1; }
        }
        const int iters = grp.iterations(w);
        int mv_end = kNeg;
        int vlo = 1 << 30, vhi = -(1 << 30);
        const int live_slot = (int)(((uint32_t)s & smask) * a.live_w) + center;
        int dmin = 1 << 30, dmax = -(1 << 30);
        for (int it = 0; it < iters; ++it) {
            const int k = lo + gl + it * G;
            if (k <= hi) {
                const unsigned hmax = (unsigned)min(m, n + k);
                int ins = max(live_get<kFmtBound>(live, fo, 0, k + 1), live_get<kFmtBound>(live, fe, 1, k + 1));
                int del = max(live_get<kFmtBound>(live, fo, 0, k - 1), live_get<kFmtBound>(live, fe, 2, k - 1)) + 1;
                int mis = live_get<kFmtBound>(live, fx, 0, k) + 1;
                if ((unsigned)ins > hmax) ins = kNeg;
                if ((unsigned)del > hmax) del = kNeg;
                if ((unsigned)mis > hmax) mis = kNeg;
                const int f0 = max(mis, max(ins, del));
                const int mv = extend<STAGE>(seqs, n, m, k, f0, p_windows);
                *reinterpret_cast<uint64_t*>(live + (size_t)(live_slot + k) * kEntryElems) =
                    (uint64_t)(uint16_t)mv | ((uint64_t)(uint16_t)ins << 16) | ((uint64_t)(uint32_t)del << 32);
                if (k == kend) mv_end = mv;
                if (f0 >= 0) { vlo = min(vlo, k); vhi = max(vhi, k); }
                if (mv >= 0) {
                    const int dist = max(n - (mv - k), m - mv);
                    dmin = min(dmin, dist);
                    dmax = max(dmax, dist);
                }
            }
        }
        if (gl == 0) p_cells += (unsigned)w;
        grp.min_max(vlo, vhi);
        const bool group_hit = grp.group_any(mv_end >= m);
        // pruning as in WFA-adaptive: a wavefront of at least adapt_min_len diagonals keeps those within
        // adapt_max_dist of the closest distance to the end
        grp.min_max(dmin, dmax);
        const bool prune = run && !group_hit && vlo <= vhi && vhi - vlo + 1 >= a.adapt_min_len &&
                           dmax - dmin > a.adapt_max_dist;
        if (__any_sync(kFull, prune)) {
            int plo = 1 << 30, phi = -(1 << 30);
            for (int it = 0; it < iters; ++it) {
                const int k = lo + gl + it * G;
                if (prune && k >= vlo && k <= vhi) {
                    const int h = live[(size_t)(live_slot + k) * kEntryElems];
                    if (h >= 0 && max(n - (h - k), m - h) - dmin <= a.adapt_max_dist) {
                        plo = min(plo, k);
                        phi = max(phi, k);
                    }
                }
            }
            grp.min_max(plo, phi);
            if (prune) { vlo = plo; vhi = phi; }
        }
        if (run) {
            if (gl == 0) rec[s] = vlo <= vhi ? make_int4(vlo, vhi - vlo + 1, 0, vhi) : empty_rec();
            if (group_hit) status = kDone;
        }
        // a pair that ended in this step: its bound (the score at which it reached the end), or none
        if (status == kDone || status == kRejected || status == kCap) {
            if (gl == 0) a.bound[pi] = status == kDone ? s : -1;
            st.cells += p_cells; st.windows += p_windows; p_cells = p_windows = 0;
            status = kIdle;
        }
        __syncwarp();
    }
}

// Traceback of one finished pair by one lane, from its region as the forward pass left it.  Returns the
// number of runs, staged end-first after the meta records; ok turns false if a step finds no source (not
// expected) or the runs overflow the staging area.
template <bool ADAPT>
__device__ uint32_t traceback(const WfaArgs& a, uint8_t* region, uint32_t pi, int final_s, bool& ok) {
    const int* meta = reinterpret_cast<const int*>(region + (size_t)a.rec_pad * sizeof(int4));
    uint32_t* staged = reinterpret_cast<uint32_t*>(region + a.meta_bytes);
    const int16_t* hist = reinterpret_cast<const int16_t*>(region + a.meta_bytes + a.runs_bytes);
    const int n = (int)a.P.read_len[pi], m = (int)a.P.target_len[pi];
    const int X = a.X, OE = a.OE, E = a.E;
    uint32_t nruns = 0;
    if constexpr (ADAPT) {
        const int kend = m - n;
        // WFA-adaptive: follow the sources.  State M at offset h of (c, k): the matches run back to f0, whose
        // source is the mismatch candidate, then I, then D; state I (value h): an extension I[c-E, k+1] == h
        // before an opening M[c-OE, k+1] == h; state D likewise with D[c-E, k-1] + 1 and M[c-OE, k-1] + 1.
        RunWriter wr;
        wr.init(staged, a.runs_cap);
        int state = 0, c = final_s, k = kend, h = m;
        for (int guard = 0; ok; ++guard) {
            if (guard > n + m + 1) { ok = false; break; }
            if (state == 0) {
                if (c == 0 && k == 0) { if (h > 0) wr.put(kOpMatch, (uint32_t)h); break; }
                int mis = wf_get(hist, load_wf(meta, c - X), 0, k);
                mis = mis >= 0 ? mis + 1 : kNeg16;
                if (mis > m || mis - k > n) mis = kNeg16;
                const Wf fc = load_wf(meta, c);
                const int ins = wf_get(hist, fc, 1, k), del = wf_get(hist, fc, 2, k);
                const int f0 = max(mis, max(ins, del));
                if (f0 < 0 || f0 > h) { ok = false; break; }
                if (h > f0) wr.put(kOpMatch, (uint32_t)(h - f0));
                h = f0;
                if (f0 == mis) { wr.put(kOpMismatch, 1); --h; c -= X; }
                else if (f0 == ins) state = 1;
                else state = 2;
            } else if (state == 1) {
                wr.put(kOpIns, 1);
                if (wf_get(hist, load_wf(meta, c - E), 1, k + 1) == h) { c -= E; }
                else if (wf_get(hist, load_wf(meta, c - OE), 0, k + 1) == h) { c -= OE; state = 0; }
                else { ok = false; break; }
                k += 1;
            } else {
                wr.put(kOpDel, 1);
                const int ext = wf_get(hist, load_wf(meta, c - E), 2, k - 1);
                const int opn = wf_get(hist, load_wf(meta, c - OE), 0, k - 1);
                if (ext >= 0 && ext + 1 == h) { c -= E; }
                else if (opn >= 0 && opn + 1 == h) { c -= OE; state = 0; }
                else { ok = false; break; }
                k -= 1; h -= 1;
            }
        }
        wr.finish();
        nruns = wr.n;
        ok = ok && wr.n <= wr.cap;
    } else {
        // canonical traceback; every step issues the loads of all four tight tests at once (two memory round
        // trips per step instead of a chain of dependent ones)
        const int* __restrict__ cmeta = meta;
        const int16_t* __restrict__ chist = hist;
        const uint64_t* Pg = read_words(a.P, pi);     // the pair in global memory
        const uint64_t* Tg = target_words(a.P, pi);
        const uint32_t gwP = (uint32_t)(n + 31) >> 5, gwT = (uint32_t)(m + 31) >> 5;
        RunWriter wr;
        wr.init(staged, a.runs_cap);
        int v = n, h = m, cM = final_s, cI = final_s, cD = final_s;
        while (v > 0 || h > 0) {
            const int k = h - v;
            const bool diag = v > 0 && h > 0;
            const Wf fX = load_wf(cmeta, cM - X), fI = load_wf(cmeta, cI), fD = load_wf(cmeta, cD);
            const Wf fM = load_wf(cmeta, cM);
            const uint32_t pb = diag ? base_at(Pg, v - 1) : 0u, tb = diag ? base_at(Tg, h - 1) : 1u;
            const int vX = wf_get(chist, fX, 0, k), vI = wf_get(chist, fI, 1, k), vD = wf_get(chist, fD, 2, k);
            const int vM = wf_get(chist, fM, 0, k);
            const int stop = max(wf_get(chist, fM, 1, k), wf_get(chist, fM, 2, k));
            const bool match = diag && pb == tb;
            if (diag && !match && vX >= h - 1) {
                const int c = cM - X;
                cM = cI = cD = c; --v; --h;
                wr.put(kOpMismatch, 1);
            } else if (v > 0 && vI >= h) {
                const int c = cI;
                cM = c - OE; cD = c - OE; cI = c - E; --v;
                wr.put(kOpIns, 1);
            } else if (h > 0 && vD >= h) {
                const int c = cD;
                cM = c - OE; cI = c - OE; cD = c - E; --h;
                wr.put(kOpDel, 1);
            } else if (match && vM >= h - 1) {
                const int c = cM;
                int run = match_run_back(Pg, gwP, v, Tg, gwT, h);
                if (run > h - stop) run = h - stop;
                if (run < 1) { ok = false; break; }
                v -= run; h -= run;
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
    return nruns;
}

// Canonical traceback of a pair aligned with a compact history (kFmt16, kFmt32): the same tight tests as the
// kFmt8 traceback, taken in the order X, I, D, M and evaluated one after another.  M~ comes from the history word;
// I~[c, k] follows the I source bits back along the gap, (c, k) -> (c - E, k + 1), to the score where the gap
// opened, and is M~[c' - OE, k' + 1] there, dropped if it leaves the matrix at k; D~[c, k] likewise along
// (c - E, k - 1), adding one target base per step back.  (A source bit is set only when the extension's value
// was valid and larger, so every step back stays inside the stored wavefronts.)
template <int FMT>
__device__ __noinline__ uint32_t traceback_compact(const WfaArgs& a, uint8_t* region, uint32_t pi, int final_s, bool& ok) {
    using H = typename FmtT<FMT>::H;
    constexpr int B = FmtT<FMT>::kBits;
    constexpr uint32_t kField = (1u << B) - 1;
    constexpr int kNeg = FmtT<FMT>::kNeg;
    const int* meta = reinterpret_cast<const int*>(region + (size_t)a.rec_pad * sizeof(int4));
    uint32_t* staged = reinterpret_cast<uint32_t*>(region + a.meta_bytes);
    const H* hc = reinterpret_cast<const H*>(region + a.meta_bytes + a.runs_bytes);
    const int n = (int)a.P.read_len[pi], m = (int)a.P.target_len[pi];
    const int X = a.X, OE = a.OE, E = a.E;
    // history word of (c, k), or false outside the stored wavefront
    auto word = [&](int c, int k, uint32_t& e) -> bool {
        if (c < 0) return false;
        const Wf f = load_wf(meta, c);
        if ((unsigned)(k - f.lo) >= (unsigned)f.cnt) return false;
        e = hc[f.base + k];
        return true;
    };
    auto mval = [&](int c, int k) -> int {
        uint32_t e;
        if (!word(c, k, e)) return kNeg;
        const uint32_t v = e & kField;
        return v ? (int)v - 1 : kNeg;
    };
    auto ival = [&](int c, int k) -> int {
        int cc = c, kk = k;
        uint32_t e;
        for (int guard = 0;; ++guard) {
            if (guard > n + m + 1 || !word(cc, kk, e)) return kNeg;
            if (!((e >> B) & 1u)) break;
            cc -= E; kk += 1;
        }
        const int v = mval(cc - OE, kk + 1);
        return (unsigned)v > (unsigned)min(m, n + k) ? kNeg : v;
    };
    auto dval = [&](int c, int k) -> int {
        int cc = c, kk = k, j = 0;
        uint32_t e;
        for (;; ++j) {
            if (j > n + m + 1 || !word(cc, kk, e)) return kNeg;
            if (!((e >> (B + 1)) & 1u)) break;
            cc -= E; kk -= 1;
        }
        const int v = mval(cc - OE, kk - 1);
        if (v < 0) return kNeg;
        const int d = v + 1 + j;
        return (unsigned)d > (unsigned)min(m, n + k) ? kNeg : d;
    };
    const uint64_t* Pg = read_words(a.P, pi);
    const uint64_t* Tg = target_words(a.P, pi);
    const uint32_t gwP = (uint32_t)(n + 31) >> 5, gwT = (uint32_t)(m + 31) >> 5;
    RunWriter wr;
    wr.init(staged, a.runs_cap);
    int v = n, h = m, cM = final_s, cI = final_s, cD = final_s;
    while (v > 0 || h > 0) {
        const int k = h - v;
        const bool diag = v > 0 && h > 0;
        const bool match = diag && base_at(Pg, v - 1) == base_at(Tg, h - 1);
        if (diag && !match && mval(cM - X, k) >= h - 1) {
            const int c = cM - X;
            cM = cI = cD = c; --v; --h;
            wr.put(kOpMismatch, 1);
        } else if (v > 0 && ival(cI, k) >= h) {
            const int c = cI;
            cM = c - OE; cD = c - OE; cI = c - E; --v;
            wr.put(kOpIns, 1);
        } else if (h > 0 && dval(cD, k) >= h) {
            const int c = cD;
            cM = c - OE; cI = c - OE; cD = c - E; --h;
            wr.put(kOpDel, 1);
        } else if (match && mval(cM, k) >= h - 1) {
            const int c = cM;
            const int stop = max(ival(cM, k), dval(cM, k));
            int run = match_run_back(Pg, gwP, v, Tg, gwT, h);
            if (run > h - stop) run = h - stop;
            if (run < 1) { ok = false; break; }
            v -= run; h -= run;
            cM = cI = cD = c;
            wr.put(kOpMatch, (uint32_t)run);
        } else {
            ok = false;
            break;
        }
    }
    wr.finish();
    ok = ok && wr.n <= wr.cap;
    return wr.n;
}

// Result of a finished pair: score, flags, run count, and its runs (staged end-first) copied start-first by
// lanes gl, gl + G, ... of its group; every lane of the group calls this with the same values.
__device__ __forceinline__ void emit_done(const WfaArgs& a, uint32_t pi, int final_s, uint32_t nruns, bool ok,
                                          const uint32_t* staged, int gl, int G) {
    const int32_t score = final_s * a.g;
    uint8_t flags = ok ? 0 : AIM_F_STEP_CAP;
    if (ok && a.O.cigars && a.O.cigar_off) {
        const uint64_t off = a.O.cigar_off[pi];
        const uint64_t cap = a.O.cigar_off[pi + 1] - off;
        if (nruns <= cap) {
            for (uint32_t j = (uint32_t)gl; j < nruns; j += (uint32_t)G) a.O.cigars[off + j] = staged[nruns - 1 - j];
        } else {
            flags |= AIM_F_CIGAR_OVERFLOW;
        }
    }
    if (gl == 0) write_header(a.O, pi, ok ? score : -1, flags, nruns);
}

// One lane: result of a pair that ended without an alignment.
__device__ __forceinline__ void emit_failed(const WfaArgs& a, uint32_t pi, int status) {
    const uint8_t f = status == kBad ? AIM_F_BAD_PAIR : status == kRejected ? AIM_F_REJECTED : AIM_F_STEP_CAP;
    write_header(a.O, pi, -1, f, 0);
}

// finished pairs awaiting their traceback: G records per group, 32 per warp (pair, final score, region
// offset in 16-byte units)
__shared__ int4 s_pend[256];

// Whole warp: lane gl of each group traces back the group's pending pair gl (so up to 32 tracebacks run side
// by side instead of one per group), then the group writes each pair's result.
template <int G, bool ADAPT, int FMT>
__device__ __forceinline__ void finish_pending(const WfaArgs& a, const Group<G>& grp, uint8_t* arena,
                                               const int4* pend, int npend) {
    __syncwarp();
    const int gl = grp.gl;
    uint32_t pi = 0, nruns = 0, off = 0;
    int final_s = 0;
    bool ok = true;
    if (gl < npend) {
        const int4 r = pend[gl];
        pi = (uint32_t)r.x; final_s = r.y; off = (uint32_t)r.z;
        if constexpr (FMT == kFmt8) nruns = traceback<ADAPT>(a, arena + ((size_t)off << 4), pi, final_s, ok);
        else nruns = traceback_compact<FMT>(a, arena + ((size_t)off << 4), pi, final_s, ok);
    }
    __syncwarp();
    for (int j = 0; j < G; ++j) {
        const int src = grp.leader + j;
        const uint32_t pj = __shfl_sync(kFull, pi, src), nj = __shfl_sync(kFull, nruns, src);
        const uint32_t oj = __shfl_sync(kFull, off, src);
        const int fj = __shfl_sync(kFull, final_s, src);
        const bool okj = __shfl_sync(kFull, ok ? 1 : 0, src) != 0;
        if (j < npend)
            emit_done(a, pj, fj, nj, okj, reinterpret_cast<const uint32_t*>(arena + ((size_t)oj << 4) + a.meta_bytes),
                      gl, G);
    }
    __syncwarp();
}

// Drains bucket b.  Groups defer tracebacks: a group keeps finishing pairs in fresh parts of its arena (its
// share of the scratch) and traces them back side by side once it holds as many as it has tracing lanes (G
// for a group of up to 32 lanes, one per warp for a whole block), once its arena has less room left than
// one pair may need (pair_bytes), or when the bucket is drained.  A pair's forward pass therefore always has
// at least pair_bytes, as without deferral.
template <int G, bool ADAPT, bool STAGE, int FMT>
__device__ __forceinline__ void run_bucket(const WfaArgs& a, int b, uint8_t* warp_slot, uint32_t lane, Counters& st) {
    // bytes of history per entry of a finished pair (a compact form's live ring is not kept)
    constexpr size_t kEntryBytes = FMT == kFmt8 ? kEntryElems * sizeof(int16_t) : sizeof(typename FmtT<FMT>::H);
    const uint32_t begin = a.bounds ? a.bounds[b] : 0;
    const uint32_t end = a.bounds ? a.bounds[b + 1] : a.P.num_pairs;
    if constexpr (FMT == kFmtBound) {
        // bound pass: asynchronous groups, each in its own region (meta records, then the live ring at its end)
        (void)begin; (void)end;
        bound_pass_run<G, STAGE>(a, b, warp_slot, lane, st);
    } else if constexpr (G > 32) {
        // the whole block takes one pair at a time in its arena (its warps' scratch regions); finished pairs
        // wait there, up to one per warp, and the first lane of warp w traces back the w-th
        constexpr int kWarps = G / 32;
        __shared__ uint32_t s_pos;
        __shared__ int4 s_bpend[kWarps];   // pair, final score, region offset in 16-byte units
        __shared__ uint2 s_bres[kWarps];   // run count, traceback ok
        const size_t block_bytes = (size_t)kWarps * a.warp_bytes;
        uint8_t* block_slot = a.scratch + (size_t)blockIdx.x * block_bytes;
        const uint32_t arena16 = (uint32_t)(block_bytes >> 4);
        const uint32_t pair16 = (uint32_t)((a.pair_bytes + 15) >> 4);
        uint32_t used16 = 0;
        int npend = 0;
        auto finish = [&]() {
            __syncthreads();
            const int w = (int)(threadIdx.x >> 5);
            if ((threadIdx.x & 31) == 0 && w < npend) {
                const int4 r = s_bpend[w];
                bool ok = true;
                uint32_t nr;
                if constexpr (FMT == kFmt8) nr = traceback<ADAPT>(a, block_slot + ((size_t)r.z << 4), (uint32_t)r.x, r.y, ok);
                else nr = traceback_compact<FMT>(a, block_slot + ((size_t)r.z << 4), (uint32_t)r.x, r.y, ok);
                s_bres[w] = make_uint2(nr, ok ? 1u : 0u);
            }
            __syncthreads();
            for (int j = 0; j < npend; ++j) {
                const int4 r = s_bpend[j];
                const uint2 q = s_bres[j];
                emit_done(a, (uint32_t)r.x, r.y, q.x, q.y != 0,
                          reinterpret_cast<const uint32_t*>(block_slot + ((size_t)r.z << 4) + a.meta_bytes),
                          (int)threadIdx.x, G);
            }
            __syncthreads();
        };
        for (;;) {
            if (threadIdx.x == 0) s_pos = atomicAdd(a.counters + b, 1u);
            __syncthreads();
            const uint32_t pos = s_pos;
            __syncthreads();
            if (pos >= end - begin || end <= begin) break;
            if (npend == kWarps || arena16 - used16 < pair16) {
                finish();
                used16 = 0;
                npend = 0;
            }
            const Forward f = forward_pair<G, ADAPT, false, FMT>(a, block_slot + ((size_t)used16 << 4),
                                                            (size_t)(arena16 - used16) << 4, begin + pos, end, lane, st);
            if (f.status == kDone) {
                if (threadIdx.x == 0) s_bpend[npend] = make_int4((int)f.pi, f.final_s, (int)used16, 0);
                ++npend;
                used16 += (uint32_t)((a.meta_bytes + a.runs_bytes + (size_t)f.top * kEntryBytes + 15) >> 4);
            } else if (f.status != kIdle && threadIdx.x == 0) {
                emit_failed(a, f.pi, f.status);
            }
        }
        finish();
    } else {
        constexpr int P = 32 / G;
        const Group<G> grp(lane);
        const int gl = grp.gl;
        // the group's arena and its pending records (recomputed where needed, to keep registers for the
        // forward pass); used16: bytes of the arena taken by pending pairs, in 16-byte units
        const uint32_t arena16 = (uint32_t)((a.warp_bytes / P) >> 4);
        const uint32_t pair16 = (uint32_t)((a.pair_bytes + 15) >> 4);
        uint32_t used16 = 0;
        int npend = 0;
        for (;;) {
            uint32_t pos = 0;
            if (lane == 0) pos = atomicAdd(a.counters + b, (uint32_t)P);
            pos = __shfl_sync(kFull, pos, 0);
            if (pos >= end - begin || end <= begin) break;
            if (__any_sync(kFull, npend == G || arena16 - used16 < pair16)) {
                finish_pending<G, ADAPT, FMT>(a, grp, warp_slot + ((size_t)grp.index(lane) * arena16 << 4),
                                              s_pend + (threadIdx.x & ~31u) + grp.index(lane) * G, npend);
                used16 = 0;
                npend = 0;
            }
            uint8_t* region = warp_slot + (((size_t)grp.index(lane) * arena16 + used16) << 4);
            const Forward f =
                forward_pair<G, ADAPT, STAGE, FMT>(a, region, (size_t)(arena16 - used16) << 4, begin + pos, end, lane, st);
            if (f.status == kDone) {
                if (gl == 0)
                    s_pend[(threadIdx.x & ~31u) + grp.index(lane) * G + npend] = make_int4((int)f.pi, f.final_s, (int)used16, 0);
                ++npend;
                used16 += (uint32_t)((a.meta_bytes + a.runs_bytes + (size_t)f.top * kEntryBytes + 15) >> 4);
            } else if (f.status != kIdle && gl == 0) {
                emit_failed(a, f.pi, f.status);
            }
        }
        finish_pending<G, ADAPT, FMT>(a, grp, warp_slot + ((size_t)grp.index(lane) * arena16 << 4),
                                      s_pend + (threadIdx.x & ~31u) + grp.index(lane) * G, npend);
    }
}

// blocks of 256 per SM the register budget must allow: 3 (80 registers).  At 4 (64 registers) the deferred
// tracebacks made every instance but the plain 32-lane one spill; the exact 32-lane kernel also measured 2.5 %
// faster at 3 on long pairs, and whole-block groups 4 % faster.
// The compact-history instances (long reads) carry the live ring's addressing as well: whole-block groups fit
// 80 registers with the traceback as a separate call; the 32-lane one spills there and is built for 2 blocks per SM.
template <int G, bool ADAPT, bool STAGE, int FMT>
constexpr int wfa_min_blocks() { return FMT == kFmt8 || FMT == kFmtBound || G > 32 ? 3 : 2; }

// One persistent launch per group size G: it drains, in order, the buckets whose group size is G.  Only
// that G is compiled into the kernel, so it carries the registers of one variant instead of all seven (a
// kernel with every variant spilled about 1 KB per thread and ran 14 % slower).
// STAGE (groups up to 16 lanes): the launch gives each group a shared-memory slot for its pair's sequences.
template <int G, bool ADAPT, bool STAGE, int FMT>
__global__ void __launch_bounds__(256, (wfa_min_blocks<G, ADAPT, STAGE, FMT>())) wfa_kernel(WfaArgs a) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gwarp >= a.nwarps) return;
    uint8_t* warp_slot = a.scratch + (size_t)gwarp * a.warp_bytes;
    Counters st{0, 0, 0};
    if (a.nbuckets == 1) {
        // one queue range (plain calls, and the batched form's groups): measured 7 % faster than the loop below
        run_bucket<G, ADAPT, STAGE, FMT>(a, 0, warp_slot, lane, st);
    } else {
        for (int b = 0; b < a.nbuckets; ++b)
            if ((a.group[b] > 32 ? 256 : a.group[b]) == G) run_bucket<G, ADAPT, STAGE, FMT>(a, b, warp_slot, lane, st);
    }
    warp_stat_add(a.O.stats, 0, st.cells, lane);
    warp_stat_add(a.O.stats, 1, st.windows, lane);
    warp_stat_add(a.O.stats, 3, st.pairs, lane);
}

template <bool ADAPT, bool STAGE>
void (*kernel_for(int G))(WfaArgs) {
    switch (G) {
        case 1: return wfa_kernel<1, ADAPT, STAGE, kFmt8>;
        case 2: return wfa_kernel<2, ADAPT, STAGE, kFmt8>;
        case 4: return wfa_kernel<4, ADAPT, STAGE, kFmt8>;
        case 8: return wfa_kernel<8, ADAPT, STAGE, kFmt8>;
        case 16: return wfa_kernel<16, ADAPT, STAGE, kFmt8>;
        case 32: return wfa_kernel<32, ADAPT, false, kFmt8>;
        default: return wfa_kernel<256, ADAPT, false, kFmt8>;
    }
}

// the bound pass (pruned, no history): groups of 4 to 32 lanes, staged up to 16
void (*bound_kernel_for(int G, bool stage))(WfaArgs) {
    switch (G) {
        case 4: return stage ? wfa_kernel<4, true, true, kFmtBound> : wfa_kernel<4, true, false, kFmtBound>;
        case 8: return stage ? wfa_kernel<8, true, true, kFmtBound> : wfa_kernel<8, true, false, kFmtBound>;
        case 16: return stage ? wfa_kernel<16, true, true, kFmtBound> : wfa_kernel<16, true, false, kFmtBound>;
        default: return wfa_kernel<32, true, false, kFmtBound>;
    }
}

// the exact kernels of 32-lane and whole-block groups with a compact history
void (*compact_kernel_for(int G, int fmt))(WfaArgs) {
    if (G == 32) return fmt == kFmt16 ? wfa_kernel<32, false, false, kFmt16> : wfa_kernel<32, false, false, kFmt32>;
    return fmt == kFmt16 ? wfa_kernel<256, false, false, kFmt16> : wfa_kernel<256, false, false, kFmt32>;
}

// Groups of up to 16 lanes (many pairs per SM) stage their pairs' sequences in shared memory when a block's
// copies fit in kStageBytes (kBoundStageBytes for bound passes, which keep no history: 4-lane bound passes over
// reads of up to 1,000 bp then stage their 34 KB, 139.0 -> 138.4 ms on the default step); groups of 32 lanes
// and whole blocks (one long pair per warp or block) gained nothing from it and read global memory.
constexpr int kStageMaxGroup = 16;
constexpr size_t kStageBytes = 24 << 10;
constexpr size_t kBoundStageBytes = 48 << 10;

int gcd_i(int a, int b) {
    while (b) { const int t = a % b; a = b; b = t; }
    return a < 0 ? -a : a;
}

}  // namespace

// Worst-case entries of the wavefront history of one pair: every wavefront as wide as its sources allow.
size_t wfa_hist_entries(const WfaPlan& p, int64_t max_len, int64_t smax, bool clamp) {
    const int64_t klo = p.band >= 0 ? -std::min<int64_t>(max_len, p.band) : -max_len;
    const int64_t khi = p.band >= 0 ? std::min<int64_t>(max_len, p.band) : max_len;
    std::vector<int64_t> lo(smax + 1), hi(smax + 1);
    lo[0] = 0; hi[0] = 0;
    size_t entries = 1;
    for (int64_t s = 1; s <= smax; ++s) {
        int64_t l = INT64_MAX, h = INT64_MIN;
        auto take = [&](int64_t src, int64_t grow) {
            if (src < 0 || lo[src] > hi[src]) return;
            l = std::min(l, lo[src] - grow); h = std::max(h, hi[src] + grow);
        };
        take(s - p.x, 0); take(s - p.oe, 1); take(s - p.e, 1);
        l = std::max(l, klo); h = std::min(h, khi);
        lo[s] = l; hi[s] = h;
        if (l <= h) {
            // exact kernels also clamp each wavefront to the 2 (S - s) / E + 1 diagonals around the end diagonal
            // that can still end within the limit S <= smax (where they lie depends on the pair; how many does not)
            int64_t w = h - l + 1;
            if (clamp) w = std::min<int64_t>(w, 2 * ((smax - s) / std::max(p.e, 1)) + 1);
            entries += (size_t)w;
        }
    }
    return entries;
}

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
    p.max_length = max_length;
    p.hist_entries = wfa_hist_entries(p, L, smax, true);   // exact kernels (adaptive plans recompute it)
    // the live ring of the compact forms: a power-of-2 slot count above the farthest source (max(X, OE, E)
    // scores back) and a power-of-2 slot width above the widest wavefront (it grows by at most one diagonal on
    // each side per E score units: 2 smax / E + 3, within the matrix and the band)
    int64_t wmax = 2 * (smax / std::max(p.e, 1)) + 3;
    wmax = std::min<int64_t>(wmax, 2 * L + 1);
    if (band >= 0) wmax = std::min<int64_t>(wmax, 2 * (int64_t)band + 1);
    p.live_w = 1;
    while ((int64_t)p.live_w < wmax) p.live_w <<= 1;
    p.live_slots = 1;
    while ((int)p.live_slots < std::max(std::max(p.x, p.oe), p.e) + 1) p.live_slots <<= 1;
    const int64_t minc = std::min<int64_t>(p.x, p.oe);
    int64_t runs = 2 * L + 1;
    if (minc > 0) runs = std::min<int64_t>(runs, 2 * (smax / minc) + 1);
    p.runs_cap = (int)runs;
    p.rec_pad = std::max(std::max(p.x, p.oe), p.e);
    p.meta_bytes = align_up((size_t)(smax + 1 + p.rec_pad) * 4 * sizeof(int), 16);
    p.runs_bytes = align_up((size_t)p.runs_cap * sizeof(uint32_t), 16);
    p.adapt_min_len = -1;
    p.adapt_max_dist = 0;
    p.retry_only = 0;
    p.bound = nullptr;
    p.bound_pass = 0;
    p.bound_min_len = kBoundMinLen;
    p.bound_max_dist = kBoundMaxDist;
    return p;
}

WfaPlan wfa_plan_compact(const WfaPlan& full, int64_t width) {
    WfaPlan p = full;
    const size_t compact = (size_t)(full.smax + 1) * (size_t)std::max<int64_t>(width, 1) + 1;
    if (compact < p.hist_entries) p.hist_entries = compact;
    return p;
}

// Storage form for a launch: the exact kernels of 32-lane and whole-block groups keep a compact history for
// reads longer than kCompactMinLength (the live ring costs more than it saves on short ones); everything else,
// and the adaptive algorithm, keeps 8-byte entries.
int wfa_format(const WfaPlan& p, int group) {
    if (p.adapt_min_len >= 0 || group < 32 || p.max_length <= kCompactMinLength) return kFmt8;
    return p.max_length <= kMaxWfaLength16c ? kFmt16 : kFmt32;
}

size_t wfa_live_bytes(const WfaPlan& p, int fmt) {
    if (fmt == kFmt8) return 0;
    return align_up((size_t)p.live_slots * p.live_w * kEntryElems * (fmt == kFmt32 ? 4 : 2), 16);
}

size_t wfa_bound_pair_bytes(const WfaPlan& p) { return align_up(p.meta_bytes + wfa_live_bytes(p, kFmtBound), 16); }

size_t wfa_pair_bytes_capped(const WfaPlan& p, int group, size_t entries) {
    const int fmt = wfa_format(p, group);
    const size_t per_entry = fmt == kFmt8 ? kEntryElems * sizeof(int16_t) : fmt == kFmt16 ? 2 : 4;
    return align_up(p.meta_bytes + p.runs_bytes + wfa_live_bytes(p, fmt) + entries * per_entry, 16);
}

size_t wfa_pair_bytes(const WfaPlan& p, int group) { return wfa_pair_bytes_capped(p, group, p.hist_entries); }

int wfa_default_group(const WfaPlan& p, uint32_t max_length) {
    // widest wavefront a pair can reach: 2 * smax / E + 1 diagonals, clamped by the matrix and the band
    int64_t w = 2 * (p.smax / std::max(p.e, 1)) + 1;
    w = std::min<int64_t>(w, 2 * (int64_t)max_length + 1);
    if (p.band >= 0) w = std::min<int64_t>(w, 2 * (int64_t)p.band + 1);
    const int g = w <= 64 ? 4 : w <= 128 ? 8 : w <= 256 ? 16 : w <= 1024 ? 32 : 256;
    return max_length > kMaxWfaLength16 ? std::max(g, 32) : g;   // int16 offsets: reads up to 32,000 bp
}

cudaError_t launch_wfa_buckets(const WfaPlan& plan, const PairsView& P, const LimitView& L, const OutView& O,
                               const uint32_t* order, const uint32_t* bounds, const int* groups, int nbuckets,
                               size_t warp_bytes, uint8_t* scratch, size_t scratch_bytes, uint32_t* counters,
                               int num_sms, cudaStream_t st, int* warps_used) {
    *warps_used = 0;
    if (P.num_pairs == 0) return cudaSuccess;
    if (nbuckets < 1 || nbuckets > kMaxBuckets) return cudaErrorInvalidValue;
    WfaArgs a;
    a.X = plan.x; a.OE = plan.oe; a.E = plan.e; a.g = plan.g; a.smax = plan.smax; a.band = plan.band;
    a.P = P; a.L = L; a.O = O;
    a.scratch = scratch; a.warp_bytes = warp_bytes;
    a.meta_bytes = plan.meta_bytes; a.runs_bytes = plan.runs_bytes; a.runs_cap = (uint32_t)plan.runs_cap;
    a.rec_pad = (uint32_t)plan.rec_pad;
    a.order = order; a.bounds = bounds; a.counters = counters; a.nbuckets = nbuckets;
    // a bound pass prunes with its own parameters and writes plan.bound; exact passes read it when it is set
    const bool bound_pass = plan.bound_pass != 0;
    if (bound_pass && (!plan.bound || plan.adapt_min_len >= 0 || P.max_length > kMaxWfaLength16))
        return cudaErrorInvalidValue;
    a.adapt_min_len = bound_pass ? plan.bound_min_len : plan.adapt_min_len;
    a.adapt_max_dist = bound_pass ? plan.bound_max_dist : plan.adapt_max_dist;
    a.bound = plan.bound;
    a.retry_only = plan.retry_only;
    a.live_w = plan.live_w; a.live_slots = plan.live_slots;
    for (int b = 0; b < kMaxBuckets; ++b) a.group[b] = (int16_t)(b < nbuckets ? groups[b] : 32);
    const bool adapt = plan.adapt_min_len >= 0;
    int launched = 0;
    // one launch per distinct group size, in the order the buckets (heaviest first) first use it; each sized
    // by its own instance's occupancy (whole blocks of 8 warps: a 256-lane group uses all of them)
    int seen[kMaxBuckets];
    int nseen = 0;
    for (int b = 0; b < nbuckets; ++b) {
        const int G = a.group[b] > 32 ? 256 : a.group[b];
        bool dup = false;
        for (int i = 0; i < nseen; ++i) dup |= seen[i] == G;
        if (dup) continue;
        seen[nseen++] = G;
        // sequence copies in shared memory when the group size takes them and a block's fit in kStageBytes
        const size_t slot_words = ((size_t)P.max_length + 31) / 32 + 1;
        size_t smem = (size_t)8 * (32 / std::min(G, 32)) * 2 * slot_words * sizeof(uint64_t);
        if (G > kStageMaxGroup || smem > (bound_pass ? kBoundStageBytes : kStageBytes)) smem = 0;
        a.seq_slot_words = smem ? (uint32_t)slot_words : 0u;
        if (bound_pass && (G < 4 || G > 32)) return cudaErrorInvalidValue;
        const int fmt = bound_pass ? kFmtBound : wfa_format(plan, G);
        a.live_bytes = wfa_live_bytes(plan, fmt);
        if (fmt != kFmt8 && fmt != kFmtBound) smem = 0;
        void (*kernel)(WfaArgs) = bound_pass ? bound_kernel_for(G, smem != 0)
                                : fmt != kFmt8 ? compact_kernel_for(G, fmt)
                                : adapt ? (smem ? kernel_for<true, true>(G) : kernel_for<true, false>(G))
                                        : (smem ? kernel_for<false, true>(G) : kernel_for<false, false>(G));
        // exact staged launches: a ring of the last R score records per group, R a power of 2 above the
        // farthest source (max(X, OE)), after the sequence copies, when a block's rings fit beside them in 48 KB
        uint32_t R = 1;
        while (R < (uint32_t)std::max(plan.x, plan.oe) + 1) R <<= 1;
        const size_t ring_bytes = (G > 32 ? 1 : (size_t)8 * (32 / G)) * R * sizeof(int4);
        a.meta_ring = 0; a.ring_off = (uint32_t)smem;
        if (smem && !adapt && !bound_pass && R <= 64 && smem + ring_bytes <= (48u << 10)) {
            a.meta_ring = R;
            smem += ring_bytes;
        }
        int bps = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, 256, smem);
        if (err != cudaSuccess) return err;
        if (bps < 1) bps = 1;
        size_t warps = (size_t)num_sms * bps * 8;
        const size_t fit = scratch_bytes / warp_bytes;
        if (warps > fit) warps = fit;
        if (!bounds) {
            const size_t need = G > 32 ? (size_t)P.num_pairs * (G / 32) : (P.num_pairs + (32 / G) - 1) / (32 / G);
            if (warps > need) warps = (need + 7) / 8 * 8 <= fit ? (need + 7) / 8 * 8 : need;
        }
        warps = warps / 8 * 8;
        if (warps == 0) { *warps_used = 0; return cudaSuccess; }   // not one block's scratch fits: caller reports it
        a.nwarps = (uint32_t)warps;
        // the launch spreads the scratch over its warps: what a pair may need stays pair_bytes, and the rest
        // holds finished pairs until their tracebacks run side by side.  A group's arena stops at one worst-case
        // pair plus as many finished pairs as the group defers (G, or a block's 8), each at most a worst-case
        // pair: deferral then runs exactly as with the whole scratch, on a compact footprint (250 bp with band
        // 25 on 32 GiB: 23.1 -> 21.4 ms, from arenas 9 MB apart to a few hundred KB).  The kernel counts an
        // arena in 16-byte units in 32 bits, so it also stops at 32 GiB per group; a plan that needs more for
        // one pair keeps its size.
        a.pair_bytes = G > 32 ? warp_bytes * (size_t)(G / 32) : (warp_bytes / (size_t)(32 / G)) & ~(size_t)15;
        const size_t max_group = ((size_t)32 << 30) - 16;
        const size_t max_warp = G > 32 ? max_group / (size_t)(G / 32) : max_group * (size_t)(32 / G);
        const size_t full_defer = G > 32 ? (a.pair_bytes * (size_t)(G / 32 + 1) + (size_t)(G / 32) - 1) / (size_t)(G / 32)
                                          : (size_t)(32 / G) * a.pair_bytes * (size_t)(G + 1);
        a.warp_bytes = std::min(std::min(std::max(warp_bytes, (scratch_bytes / warps) & ~(size_t)15),
                                         std::max(warp_bytes, max_warp & ~(size_t)15)),
                                std::max(warp_bytes, align_up(full_defer, 16)));
        kernel<<<(unsigned)(warps / 8), 256, smem, st>>>(a);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        launched = std::max(launched, (int)warps);
    }
    *warps_used = launched;
    return cudaSuccess;
}

size_t wfa_warp_bytes(int group, size_t pair_bytes) {
    if (group > 32) return align_up((pair_bytes + (size_t)(group / 32) - 1) / (size_t)(group / 32), 16);
    return (size_t)(32 / group) * pair_bytes;
}

cudaError_t launch_wfa(const WfaPlan& plan, int group, const PairsView& P, const LimitView& L, const OutView& O,
                       uint8_t* scratch, size_t scratch_bytes, uint32_t* counter, int num_sms, cudaStream_t st,
                       int* warps_used) {
    const size_t warp_bytes = wfa_warp_bytes(group, wfa_pair_bytes(plan, group));
    return launch_wfa_buckets(plan, P, L, O, nullptr, nullptr, &group, 1, warp_bytes, scratch, scratch_bytes,
                              counter, num_sms, st, warps_used);
}

}  // namespace aim
