/*
 * ORACLE -- test infrastructure only.  Plain, slow, obviously correct CPU
 * implementation of what the alignment hot path computes.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may call it; the CUDA
 * product path never does.  It shares no code with the CUDA library.
 *
 * What it computes (per pair of read P[0..n) and target T[0..m)):
 *
 *   Exact global alignment under gap-affine costs (Section 2.4.2: SWG, three
 *   tables M, I, D; NW's scheme with separate costs for opening and for
 *   extending a gap); NW edit distance (Section 2.4.1) is the same DP with
 *   mismatch 1, open 0, extend 1.  The recurrences are the textbook Gotoh ones (the paper names
 *   the method but does not print them), written out over the full matrix:
 *
 *     M(v,h) = min(M,I,D)(v-1,h-1) + (P[v-1]==T[h-1] ? 0 : x)
 *     I(v,h) = min(M(v-1,h)+o+e, D(v-1,h)+o+e, I(v-1,h)+e)      (consumes a read base)
 *     D(v,h) = min(M(v,h-1)+o+e, I(v,h-1)+o+e, D(v,h-1)+e)      (consumes a target base)
 *     M(0,0) = 0, I(v,0) = o+e*v, D(0,h) = o+e*h, every other border entry infinite.
 *     Cells with |h-v| > band are infinite when a band is given.
 *     score = min(M,I,D)(n,m)
 *
 *   Threshold (Section 1: every pair is aligned under an edit limit): the pair is rejected
 *   iff score > limit (or |n-m| > band); a rejected pair reports score -1,
 *   flag 1 and no CIGAR.
 *
 *   Canonical CIGAR (the paper fixes no tie-break): among all optimal
 *   alignments, the one whose op string read backward from the end is
 *   lexicographically smallest under X < I < D < M.  Computed by a backward
 *   greedy over the set of states whose DP value equals the cost the suffix
 *   requires of them ("tight" states), taking at each cell the op of the
 *   highest-priority tight state.
 *
 * Pinned by: brute-force enumeration of every op string on tiny pairs,
 * closed forms, hand-worked examples and invariants (tests/test_oracle_*.py).
 *
 * Build: gcc -O2 -fPIC -shared aim_oracle.c -o liboracle.so -lpthread
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define INF ((int32_t)1 << 29)

static int32_t min2(int32_t a, int32_t b) { return a < b ? a : b; }
static int32_t min3(int32_t a, int32_t b, int32_t c) { return min2(min2(a, b), c); }
static int32_t cap_inf(int32_t a) { return a >= INF ? INF : a; }

/* BAM op codes used in the CIGAR runs: '=' 7, 'X' 8, 'I' 1, 'D' 2; a run is len << 4 | code. */
static uint32_t bam_code(char op) {
    switch (op) { case 'M': return 7; case 'X': return 8; case 'I': return 1; default: return 2; }
}

/*
 * Align one pair.  Returns 0 on success, -3 if memory could not be allocated.
 * cigar may be NULL (score only).  *ncig receives the number of runs even when
 * it exceeds cap; runs beyond cap are not written and flag 2 is set.
 */
int oracle_align(const char *P, uint32_t n, const char *T, uint32_t m, int32_t x, int32_t o, int32_t e,
                 int32_t band, int64_t limit, int32_t *score, uint8_t *flags, uint32_t *cigar, uint32_t cap,
                 uint32_t *ncig) {
    *score = -1; *flags = 0; *ncig = 0;
    int64_t dnm = (int64_t)m - (int64_t)n;
    if (band >= 0 && (dnm > band || -dnm > band)) { *flags = 1; return 0; }
    size_t W = (size_t)m + 1, cells = ((size_t)n + 1) * W;
    int32_t *Mt = (int32_t *)malloc(cells * sizeof(int32_t));
    int32_t *It = (int32_t *)malloc(cells * sizeof(int32_t));
    int32_t *Dt = (int32_t *)malloc(cells * sizeof(int32_t));
    char *ops = (char *)malloc((size_t)n + m + 1);
    if (!Mt || !It || !Dt || !ops) { free(Mt); free(It); free(Dt); free(ops); return -3; }
#define AT(t, v, h) (t)[(size_t)(v) * W + (size_t)(h)]
    for (uint32_t v = 0; v <= n; ++v) {
        for (uint32_t h = 0; h <= m; ++h) {
            int32_t Mv = INF, Iv = INF, Dv = INF;
            int64_t k = (int64_t)h - (int64_t)v;
            int inband = band < 0 || (k <= band && -k <= band);
            if (inband) {
                if (v == 0 && h == 0) {
                    Mv = 0;
                } else {
                    if (v >= 1 && h >= 1) {
                        int32_t d = (P[v - 1] == T[h - 1]) ? 0 : x;
                        Mv = cap_inf(min3(AT(Mt, v - 1, h - 1), AT(It, v - 1, h - 1), AT(Dt, v - 1, h - 1)) + d);
                    }
                    if (v >= 1)
                        Iv = cap_inf(min3(AT(Mt, v - 1, h) + o + e, AT(Dt, v - 1, h) + o + e, AT(It, v - 1, h) + e));
                    if (h >= 1)
                        Dv = cap_inf(min3(AT(Mt, v, h - 1) + o + e, AT(It, v, h - 1) + o + e, AT(Dt, v, h - 1) + e));
                }
            }
            AT(Mt, v, h) = Mv; AT(It, v, h) = Iv; AT(Dt, v, h) = Dv;
        }
    }
    int32_t s = min3(AT(Mt, n, m), AT(It, n, m), AT(Dt, n, m));
    if (s >= INF || (int64_t)s > limit) {
        *flags = 1;
        free(Mt); free(It); free(Dt); free(ops);
        return 0;
    }
    *score = s;
    /* state-set backward greedy; req* < 0 means the state is not required */
    int64_t reqM = s, reqI = s, reqD = s;
    uint32_t v = n, h = m, nops = 0;
    while (v > 0 || h > 0) {
        int tM = reqM >= 0 && AT(Mt, v, h) == reqM;
        int tI = reqI >= 0 && AT(It, v, h) == reqI;
        int tD = reqD >= 0 && AT(Dt, v, h) == reqD;
        int match = (v > 0 && h > 0) && P[v - 1] == T[h - 1];
        char op;
        if (tM && v > 0 && h > 0 && !match) op = 'X';
        else if (tI) op = 'I';
        else if (tD) op = 'D';
        else if (tM && match) op = 'M';
        else { free(Mt); free(It); free(Dt); free(ops); return -5; /* cannot happen: no tight state */ }
        ops[nops++] = op;
        if (op == 'X' || op == 'M') {
            int64_t c = reqM - (op == 'X' ? x : 0);
            reqM = reqI = reqD = c; --v; --h;
        } else if (op == 'I') {
            int64_t c = reqI;
            reqM = c - o - e; reqD = c - o - e; reqI = c - e; --v;
        } else {
            int64_t c = reqD;
            reqM = c - o - e; reqI = c - o - e; reqD = c - e; --h;
        }
    }
    /* ops were produced end-first; run-length encode them start-first */
    uint32_t runs = 0;
    for (int64_t i = (int64_t)nops - 1; i >= 0;) {
        char op = ops[i]; uint32_t len = 0;
        while (i >= 0 && ops[i] == op) { ++len; --i; }
        if (cigar && runs < cap) cigar[runs] = (len << 4) | bam_code(op);
        ++runs;
    }
    *ncig = runs;
    if (cigar && runs > cap) *flags |= 2;
#undef AT
    free(Mt); free(It); free(Dt); free(ops);
    return 0;
}

/*
 * The same alignment (same recurrences, same border, same band, same canonical
 * backward greedy) for long pairs, with memory linear in m per block of rows
 * instead of the whole (n+1) x (m+1) matrix: a 10 kbp pair needs 1.2 GB as a
 * full matrix of three int32 tables, and about 30 MB here.
 *
 *   Forward: rows v = 0 .. n in order, each from the row above it exactly as
 *   in oracle_align (two rows live); every row v with v % K == 0 is saved.
 *   Traceback: the greedy reads the DP values of the cell it stands on, and its
 *   rows only decrease.  The rows of the block [bK, bK + K - 1] holding the
 *   current row are recomputed from the saved row bK by the same row step, so
 *   each value read equals the full matrix's value.
 *
 * K = ceil(sqrt(n + 1)) when rows_per_block <= 0.  Pinned against oracle_align
 * (scores, flags and CIGARs) on pairs up to 1 kbp, with several K.
 */

/* Row v of the three tables from row v-1 (ignored for v = 0), as in oracle_align. */
static void row_step(const char *P, const char *T, uint32_t m, int32_t x, int32_t o, int32_t e, int32_t band,
                     uint32_t v, const int32_t *pM, const int32_t *pI, const int32_t *pD, int32_t *cM, int32_t *cI,
                     int32_t *cD) {
    for (uint32_t h = 0; h <= m; ++h) {
        int32_t Mv = INF, Iv = INF, Dv = INF;
        int64_t k = (int64_t)h - (int64_t)v;
        int inband = band < 0 || (k <= band && -k <= band);
        if (inband) {
            if (v == 0 && h == 0) {
                Mv = 0;
            } else {
                if (v >= 1 && h >= 1) {
                    int32_t d = (P[v - 1] == T[h - 1]) ? 0 : x;
                    Mv = cap_inf(min3(pM[h - 1], pI[h - 1], pD[h - 1]) + d);
                }
                if (v >= 1) Iv = cap_inf(min3(pM[h] + o + e, pD[h] + o + e, pI[h] + e));
                if (h >= 1) Dv = cap_inf(min3(cM[h - 1] + o + e, cI[h - 1] + o + e, cD[h - 1] + e));
            }
        }
        cM[h] = Mv; cI[h] = Iv; cD[h] = Dv;
    }
}

int oracle_align_rows(const char *P, uint32_t n, const char *T, uint32_t m, int32_t x, int32_t o, int32_t e,
                      int32_t band, int64_t limit, int32_t rows_per_block, int32_t *score, uint8_t *flags,
                      uint32_t *cigar, uint32_t cap, uint32_t *ncig) {
    *score = -1; *flags = 0; *ncig = 0;
    int64_t dnm = (int64_t)m - (int64_t)n;
    if (band >= 0 && (dnm > band || -dnm > band)) { *flags = 1; return 0; }
    uint32_t K = (uint32_t)(rows_per_block > 0 ? rows_per_block : 1);
    if (rows_per_block <= 0) while ((uint64_t)K * K < (uint64_t)n + 1) ++K;
    const size_t W = (size_t)m + 1, nck = (size_t)n / K + 1;
    /* saved rows: ck[c] holds row c*K, tables M, I, D one after another */
    int32_t *ck = (int32_t *)malloc(nck * 3 * W * sizeof(int32_t));
    /* block rows: blk[r] holds row b*K + r */
    int32_t *blk = (int32_t *)malloc((size_t)K * 3 * W * sizeof(int32_t));
    int32_t *two = (int32_t *)malloc(2 * 3 * W * sizeof(int32_t));
    char *ops = (char *)malloc((size_t)n + m + 1);
    if (!ck || !blk || !two || !ops) { free(ck); free(blk); free(two); free(ops); return -3; }
#define TAB(base, t) ((base) + (size_t)(t) * W)
    int32_t *prev = two, *cur = two + 3 * W;
    for (uint32_t v = 0; v <= n; ++v) {
        row_step(P, T, m, x, o, e, band, v, TAB(prev, 0), TAB(prev, 1), TAB(prev, 2), TAB(cur, 0), TAB(cur, 1),
                 TAB(cur, 2));
        if (v % K == 0) memcpy(ck + (size_t)(v / K) * 3 * W, cur, 3 * W * sizeof(int32_t));
        int32_t *t = prev; prev = cur; cur = t;
    }
    /* prev holds row n */
    int32_t s = min3(TAB(prev, 0)[m], TAB(prev, 1)[m], TAB(prev, 2)[m]);
    if (s >= INF || (int64_t)s > limit) {
        *flags = 1;
        free(ck); free(blk); free(two); free(ops);
        return 0;
    }
    *score = s;
    int64_t reqM = s, reqI = s, reqD = s;
    uint32_t v = n, h = m, nops = 0;
    int64_t have = -1;   /* block whose rows blk holds */
    while (v > 0 || h > 0) {
        const uint32_t b = v / K;
        if ((int64_t)b != have) {
            memcpy(blk, ck + (size_t)b * 3 * W, 3 * W * sizeof(int32_t));
            for (uint32_t r = 1; r < K && b * K + r <= n; ++r) {
                int32_t *pr = blk + (size_t)(r - 1) * 3 * W, *cr = blk + (size_t)r * 3 * W;
                row_step(P, T, m, x, o, e, band, b * K + r, TAB(pr, 0), TAB(pr, 1), TAB(pr, 2), TAB(cr, 0),
                         TAB(cr, 1), TAB(cr, 2));
            }
            have = b;
        }
        const int32_t *row = blk + (size_t)(v - b * K) * 3 * W;
        int tM = reqM >= 0 && TAB(row, 0)[h] == reqM;
        int tI = reqI >= 0 && TAB(row, 1)[h] == reqI;
        int tD = reqD >= 0 && TAB(row, 2)[h] == reqD;
        int match = (v > 0 && h > 0) && P[v - 1] == T[h - 1];
        char op;
        if (tM && v > 0 && h > 0 && !match) op = 'X';
        else if (tI) op = 'I';
        else if (tD) op = 'D';
        else if (tM && match) op = 'M';
        else { free(ck); free(blk); free(two); free(ops); return -5; /* cannot happen: no tight state */ }
        ops[nops++] = op;
        if (op == 'X' || op == 'M') {
            int64_t c = reqM - (op == 'X' ? x : 0);
            reqM = reqI = reqD = c; --v; --h;
        } else if (op == 'I') {
            int64_t c = reqI;
            reqM = c - o - e; reqD = c - o - e; reqI = c - e; --v;
        } else {
            int64_t c = reqD;
            reqM = c - o - e; reqI = c - o - e; reqD = c - e; --h;
        }
    }
#undef TAB
    uint32_t runs = 0;
    for (int64_t i = (int64_t)nops - 1; i >= 0;) {
        char op = ops[i]; uint32_t len = 0;
        while (i >= 0 && ops[i] == op) { ++len; --i; }
        if (cigar && runs < cap) cigar[runs] = (len << 4) | bam_code(op);
        ++runs;
    }
    *ncig = runs;
    if (cigar && runs > cap) *flags |= 2;
    free(ck); free(blk); free(two); free(ops);
    return 0;
}

/* Textbook one-state Levenshtein distance (two rows), an independent cross-check for the unit-cost case. */
int32_t oracle_levenshtein(const char *P, uint32_t n, const char *T, uint32_t m) {
    int32_t *prev = (int32_t *)malloc(((size_t)m + 1) * sizeof(int32_t));
    int32_t *cur = (int32_t *)malloc(((size_t)m + 1) * sizeof(int32_t));
    if (!prev || !cur) { free(prev); free(cur); return -3; }
    for (uint32_t h = 0; h <= m; ++h) prev[h] = (int32_t)h;
    for (uint32_t v = 1; v <= n; ++v) {
        cur[0] = (int32_t)v;
        for (uint32_t h = 1; h <= m; ++h) {
            int32_t sub = prev[h - 1] + (P[v - 1] != T[h - 1]);
            int32_t del = prev[h] + 1, ins = cur[h - 1] + 1;
            cur[h] = sub < del ? (sub < ins ? sub : ins) : (del < ins ? del : ins);
        }
        int32_t *t = prev; prev = cur; cur = t;
    }
    int32_t r = prev[m];
    free(prev); free(cur);
    return r;
}

/* ---- batch driver: one pair per task over plain pthreads ---- */

typedef struct {
    const char *reads, *targets;
    const uint64_t *read_off, *target_off;
    const uint32_t *read_len, *target_len;
    uint64_t num_pairs;
    int32_t x, o, e, band;
    const int64_t *limit;          /* per pair */
    int32_t *scores; uint8_t *flags;
    uint32_t *cigars; const uint64_t *cigar_off; uint32_t *cigar_lens;
    volatile int64_t next;
    volatile int err;
    int32_t rows;                  /* 0: full matrix (oracle_align); else oracle_align_rows with this K (< 0: auto) */
} batch_job;

static void *batch_worker(void *arg) {
    batch_job *j = (batch_job *)arg;
    for (;;) {
        int64_t i = __atomic_fetch_add(&j->next, 1, __ATOMIC_RELAXED);
        if (i >= (int64_t)j->num_pairs) break;
        uint32_t *cig = NULL, cap = 0;
        if (j->cigars) { cig = j->cigars + j->cigar_off[i]; cap = (uint32_t)(j->cigar_off[i + 1] - j->cigar_off[i]); }
        int r = j->rows == 0
                    ? oracle_align(j->reads + j->read_off[i], j->read_len[i], j->targets + j->target_off[i],
                                   j->target_len[i], j->x, j->o, j->e, j->band, j->limit[i], &j->scores[i],
                                   &j->flags[i], cig, cap, &j->cigar_lens[i])
                    : oracle_align_rows(j->reads + j->read_off[i], j->read_len[i], j->targets + j->target_off[i],
                                        j->target_len[i], j->x, j->o, j->e, j->band, j->limit[i], j->rows,
                                        &j->scores[i], &j->flags[i], cig, cap, &j->cigar_lens[i]);
        if (r) j->err = r;
    }
    return NULL;
}

/*
 * Align num_pairs pairs on `threads` host threads.  cigars/cigar_off may be
 * NULL (scores only); cigar_off has num_pairs + 1 entries when given.
 */
static int align_batch_mode(const char *reads, const uint64_t *read_off, const uint32_t *read_len,
                            const char *targets, const uint64_t *target_off, const uint32_t *target_len,
                            uint64_t num_pairs, int32_t x, int32_t o, int32_t e, int32_t band, const int64_t *limit,
                            int32_t *scores, uint8_t *flags, uint32_t *cigars, const uint64_t *cigar_off,
                            uint32_t *cigar_lens, int threads, int32_t rows) {
    batch_job j = {reads, targets, read_off, target_off, read_len, target_len, num_pairs, x, o, e, band, limit,
                   scores, flags, cigars, cigar_off, cigar_lens, 0, 0, rows};
    if (threads < 1) threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    if (!th) return -3;
    int started = 0;
    for (int t = 0; t < threads; ++t)
        if (pthread_create(&th[t], NULL, batch_worker, &j) == 0) ++started;
    if (started == 0) batch_worker(&j);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    return j.err;
}

int oracle_align_batch(const char *reads, const uint64_t *read_off, const uint32_t *read_len, const char *targets,
                       const uint64_t *target_off, const uint32_t *target_len, uint64_t num_pairs, int32_t x,
                       int32_t o, int32_t e, int32_t band, const int64_t *limit, int32_t *scores, uint8_t *flags,
                       uint32_t *cigars, const uint64_t *cigar_off, uint32_t *cigar_lens, int threads) {
    return align_batch_mode(reads, read_off, read_len, targets, target_off, target_len, num_pairs, x, o, e, band,
                            limit, scores, flags, cigars, cigar_off, cigar_lens, threads, 0);
}

/* As oracle_align_batch with oracle_align_rows (rows_per_block <= 0: K = ceil(sqrt(n + 1))). */
int oracle_align_rows_batch(const char *reads, const uint64_t *read_off, const uint32_t *read_len,
                            const char *targets, const uint64_t *target_off, const uint32_t *target_len,
                            uint64_t num_pairs, int32_t x, int32_t o, int32_t e, int32_t band, const int64_t *limit,
                            int32_t *scores, uint8_t *flags, uint32_t *cigars, const uint64_t *cigar_off,
                            uint32_t *cigar_lens, int threads, int32_t rows_per_block) {
    return align_batch_mode(reads, read_off, read_len, targets, target_off, target_len, num_pairs, x, o, e, band,
                            limit, scores, flags, cigars, cigar_off, cigar_lens, threads,
                            rows_per_block > 0 ? rows_per_block : -1);
}

/* ---------------------------------------------------------------------------
 * WFA-adaptive (Section 2.4.4: a heuristic form of the WFA that keeps its
 * wavefronts narrow by dropping the outer diagonals least likely to lie on an
 * optimal path).  The paper gives no parameters; this is our reading, written
 * out step by step:
 *
 *   Scores run in units of g = gcd(x, o, e) (X = x/g, OE = (o+e)/g, E = e/g).
 *   Wavefront s spans diagonals [lo_s, hi_s]; for each k in the candidate
 *   range (one beyond the source ranges, clamped to [-n, m] and the band):
 *     I[s,k] = max(M[s-OE,k+1], I[s-E,k+1])      dropped if it leaves the matrix
 *     D[s,k] = max(M[s-OE,k-1], D[s-E,k-1]) + 1  dropped if it leaves the matrix
 *     f0     = max(M[s-X,k] + 1, I[s,k], D[s,k]) (the mismatch candidate dropped likewise)
 *     M[s,k] = f0 extended along matches
 *   The wavefront's range becomes the diagonals holding a valid entry.  Done
 *   when M[s, m-n] == m (before any pruning of that wavefront).  Otherwise,
 *   if the range spans at least L_min diagonals, every diagonal's distance to
 *   the end cell is max(n - v, m - h) at its M offset h (v = h - k); outer
 *   diagonals (from both ends inward, up to the first one kept) whose distance
 *   exceeds the smallest by more than D_max are removed.  L_min < 0: no
 *   pruning (exact WFA).
 *
 *   Traceback follows the sources: in state M at offset h of (s, k) the
 *   matches run back to f0; f0's source is taken in the order mismatch
 *   candidate, I, D.  In state I (value h at (s, k)) an extension I[s-E,k+1]
 *   == h is taken before an opening M[s-OE,k+1] == h; in state D likewise
 *   with D[s-E,k-1] + 1 and M[s-OE,k-1] + 1.
 *
 * Pinned by: with pruning off the score equals the full-matrix DP optimum
 * and the CIGAR re-costs to it (brute force and DP tests); with pruning the
 * CIGAR is a valid alignment that re-costs to the reported score, and
 * hand-worked cases (tests/golden/adaptive_prune.txt) fix the pruning step
 * itself: the kept range at every score, the score and the ops, including a
 * tie exactly max_distance behind, a width exactly min_length, distances at the
 * extended offset, both ends trimmed, far interior diagonals kept, a pair
 * rejected because its end diagonal was pruned and one pruned above its optimum.
 * --------------------------------------------------------------------------- */

static int32_t gcd32(int32_t a, int32_t b) { while (b) { int32_t t = a % b; a = b; b = t; } return a < 0 ? -a : a; }

typedef struct {
    int32_t lo, hi;          /* lo > hi: empty */
    int32_t *M, *I, *D;      /* indexed by k - lo */
} wfa_front;

#define WNEG (-(1 << 30))

static int32_t wf_val(const wfa_front *F, int64_t s, int which, int32_t k) {
    if (s < 0) return WNEG;
    const wfa_front *f = &F[s];
    if (f->lo > f->hi || k < f->lo || k > f->hi) return WNEG;
    const int32_t *a = which == 0 ? f->M : which == 1 ? f->I : f->D;
    return a[k - f->lo];
}

static int32_t wfa_extend_plain(const char *P, int32_t n, const char *T, int32_t m, int32_t k, int32_t h) {
    int32_t v = h - k;
    while (v < n && h < m && P[v] == T[h]) { ++v; ++h; }
    return h;
}

/* kept (may be NULL): for s = 0, 1, ... the diagonal range [lo, hi] kept at score s (lo > hi: empty), two
 * entries per score, up to the score the pair finished at (or the last score tried); *nkept: scores written. */
static int wfa_adaptive_run(const char *P, uint32_t un, const char *T, uint32_t um, int32_t x, int32_t o, int32_t e,
                            int32_t band, int64_t limit, int32_t lmin, int32_t dmax, int32_t *score, uint8_t *flags,
                            uint32_t *cigar, uint32_t cap, uint32_t *ncig, int32_t *kept, int64_t kept_cap,
                            int64_t *nkept) {
    const int32_t n = (int32_t)un, m = (int32_t)um;
    *score = -1; *flags = 0; *ncig = 0;
    if (nkept) *nkept = 0;
    const int32_t kend = m - n;
    if (band >= 0 && (kend > band || -kend > band)) { *flags = 1; return 0; }
    int32_t g = gcd32(gcd32(x, o), e);
    if (g <= 0) g = 1;
    const int32_t X = x / g, OE = (o + e) / g, E = e / g;
    int64_t trivial = ((int64_t)x * (n > m ? n : m) + o + (int64_t)e * (n > m ? n : m)) / g;
    int64_t S = limit / g;
    if (S > trivial) S = trivial;
    const int32_t klo = band >= 0 ? (-n > -band ? -n : -band) : -n;
    const int32_t khi = band >= 0 ? (m < band ? m : band) : m;
    wfa_front *F = (wfa_front *)calloc((size_t)S + 1, sizeof(wfa_front));
    if (!F) return -3;
    int64_t s = 0, found = -1;
    F[0].lo = F[0].hi = 0;
    F[0].M = (int32_t *)malloc(sizeof(int32_t)); F[0].I = (int32_t *)malloc(sizeof(int32_t));
    F[0].D = (int32_t *)malloc(sizeof(int32_t));
    int rc = 0;
    if (!F[0].M || !F[0].I || !F[0].D) { rc = -3; goto done; }
    F[0].M[0] = wfa_extend_plain(P, n, T, m, 0, 0); F[0].I[0] = WNEG; F[0].D[0] = WNEG;
    if (kend == 0 && F[0].M[0] >= m) found = 0;
    for (s = 1; found < 0 && s <= S; ++s) {
        int32_t lo = 1 << 30, hi = -(1 << 30);
        const int64_t src[3] = {s - X, s - OE, s - E};
        for (int j = 0; j < 3; ++j) {
            if (src[j] < 0 || F[src[j]].lo > F[src[j]].hi) continue;
            const int32_t grow = j == 0 ? 0 : 1;
            if (F[src[j]].lo - grow < lo) lo = F[src[j]].lo - grow;
            if (F[src[j]].hi + grow > hi) hi = F[src[j]].hi + grow;
        }
        if (lo < klo) lo = klo;
        if (hi > khi) hi = khi;
        F[s].lo = 1; F[s].hi = 0;
        if (lo > hi) continue;
        const int32_t w = hi - lo + 1;
        int32_t *Mv = (int32_t *)malloc(sizeof(int32_t) * w), *Iv = (int32_t *)malloc(sizeof(int32_t) * w);
        int32_t *Dv = (int32_t *)malloc(sizeof(int32_t) * w);
        if (!Mv || !Iv || !Dv) { free(Mv); free(Iv); free(Dv); rc = -3; goto done; }
        int32_t vlo = 1 << 30, vhi = -(1 << 30);
        for (int32_t k = lo; k <= hi; ++k) {
            int32_t ins = wf_val(F, s - OE, 0, k + 1), t = wf_val(F, s - E, 1, k + 1);
            if (t > ins) ins = t;
            if (ins >= 0 && ins - k > n) ins = WNEG;
            int32_t del = wf_val(F, s - OE, 0, k - 1);
            t = wf_val(F, s - E, 2, k - 1);
            if (t > del) del = t;
            del = del >= 0 ? del + 1 : WNEG;
            if (del > m) del = WNEG;
            int32_t mis = wf_val(F, s - X, 0, k);
            mis = mis >= 0 ? mis + 1 : WNEG;
            if (mis > m || mis - k > n) mis = WNEG;
            int32_t f0 = mis;
            if (ins > f0) f0 = ins;
            if (del > f0) f0 = del;
            Mv[k - lo] = f0 >= 0 ? wfa_extend_plain(P, n, T, m, k, f0) : WNEG;
            Iv[k - lo] = ins; Dv[k - lo] = del;
            if (f0 >= 0) { if (k < vlo) vlo = k; if (k > vhi) vhi = k; }
            if (k == kend && Mv[k - lo] >= m) found = s;
        }
        if (vlo > vhi) { free(Mv); free(Iv); free(Dv); continue; }
        if (found < 0 && lmin >= 0 && vhi - vlo + 1 >= lmin) {
            /* distance of every valid diagonal to the end cell; drop outer ones too far behind the closest */
            int64_t dmin = INT64_MAX;
            for (int32_t k = vlo; k <= vhi; ++k) {
                const int32_t h = Mv[k - lo];
                if (h < 0) continue;
                const int64_t dv = (int64_t)n - (h - k), dh = (int64_t)m - h;
                const int64_t d = dv > dh ? dv : dh;
                if (d < dmin) dmin = d;
            }
            int32_t a = vlo, b = vhi;
            while (a <= b) {
                const int32_t h = Mv[a - lo];
                const int64_t dv = (int64_t)n - (h - a), dh = (int64_t)m - h, d = dv > dh ? dv : dh;
                if (h >= 0 && d - dmin <= dmax) break;
                ++a;
            }
            while (b >= a) {
                const int32_t h = Mv[b - lo];
                const int64_t dv = (int64_t)n - (h - b), dh = (int64_t)m - h, d = dv > dh ? dv : dh;
                if (h >= 0 && d - dmin <= dmax) break;
                --b;
            }
            vlo = a; vhi = b;
        }
        /* keep [vlo, vhi] */
        const int32_t nw = vhi - vlo + 1;
        F[s].lo = vlo; F[s].hi = vhi;
        F[s].M = (int32_t *)malloc(sizeof(int32_t) * nw); F[s].I = (int32_t *)malloc(sizeof(int32_t) * nw);
        F[s].D = (int32_t *)malloc(sizeof(int32_t) * nw);
        if (!F[s].M || !F[s].I || !F[s].D) { free(Mv); free(Iv); free(Dv); rc = -3; goto done; }
        memcpy(F[s].M, Mv + (vlo - lo), sizeof(int32_t) * nw);
        memcpy(F[s].I, Iv + (vlo - lo), sizeof(int32_t) * nw);
        memcpy(F[s].D, Dv + (vlo - lo), sizeof(int32_t) * nw);
        free(Mv); free(Iv); free(Dv);
        if (found >= 0) break;
    }
    if (found < 0) { *flags = 1; goto done; }
    {
        /* source-following traceback, ops collected end-first */
        char *ops = (char *)malloc((size_t)n + m + 1);
        if (!ops) { rc = -3; goto done; }
        uint32_t nops = 0;
        int state = 0; /* 0 M, 1 I, 2 D */
        int64_t c = found;
        int32_t k = kend, h = m;
        for (;;) {
            if (state == 0) {
                if (c == 0 && k == 0) { while (h > 0) { ops[nops++] = 'M'; --h; } break; }
                int32_t mis = wf_val(F, c - X, 0, k);
                mis = mis >= 0 ? mis + 1 : WNEG;
                if (mis > m || mis - k > n) mis = WNEG;
                const int32_t ins = wf_val(F, c, 1, k), del = wf_val(F, c, 2, k);
                int32_t f0 = mis;
                if (ins > f0) f0 = ins;
                if (del > f0) f0 = del;
                if (f0 < 0 || f0 > h) { free(ops); rc = -5; goto done; }
                while (h > f0) { ops[nops++] = 'M'; --h; }
                if (f0 == mis) { ops[nops++] = 'X'; --h; c -= X; }
                else if (f0 == ins) state = 1;
                else state = 2;
            } else if (state == 1) {
                ops[nops++] = 'I';
                if (wf_val(F, c - E, 1, k + 1) == h) { c -= E; }
                else if (wf_val(F, c - OE, 0, k + 1) == h) { c -= OE; state = 0; }
                else { free(ops); rc = -5; goto done; }
                k += 1;
            } else {
                ops[nops++] = 'D';
                if (wf_val(F, c - E, 2, k - 1) + 1 == h) { c -= E; }
                else if (wf_val(F, c - OE, 0, k - 1) + 1 == h) { c -= OE; state = 0; }
                else { free(ops); rc = -5; goto done; }
                k -= 1; h -= 1;
            }
            if (nops > (uint32_t)(n + m)) { free(ops); rc = -5; goto done; }
        }
        *score = (int32_t)(found * g);
        uint32_t runs = 0;
        for (int64_t i = (int64_t)nops - 1; i >= 0;) {
            char op = ops[i]; uint32_t len = 0;
            while (i >= 0 && ops[i] == op) { ++len; --i; }
            if (cigar && runs < cap) cigar[runs] = (len << 4) | bam_code(op);
            ++runs;
        }
        *ncig = runs;
        if (cigar && runs > cap) *flags |= 2;
        free(ops);
    }
done:
    if (kept && rc == 0) {
        /* scores computed: up to the finishing one, else every score up to S */
        const int64_t last = found >= 0 ? found : S;
        int64_t t = 0;
        for (; t <= last && t < kept_cap; ++t) { kept[2 * t] = F[t].lo; kept[2 * t + 1] = F[t].hi; }
        if (nkept) *nkept = t;
    }
    for (int64_t t = 0; t <= S; ++t) { free(F[t].M); free(F[t].I); free(F[t].D); }
    free(F);
    return rc;
}

int oracle_wfa_adaptive(const char *P, uint32_t un, const char *T, uint32_t um, int32_t x, int32_t o, int32_t e,
                        int32_t band, int64_t limit, int32_t lmin, int32_t dmax, int32_t *score, uint8_t *flags,
                        uint32_t *cigar, uint32_t cap, uint32_t *ncig) {
    return wfa_adaptive_run(P, un, T, um, x, o, e, band, limit, lmin, dmax, score, flags, cigar, cap, ncig, NULL, 0,
                            NULL);
}

/* The same, also reporting the diagonal range kept at every score (see wfa_adaptive_run). */
int oracle_wfa_adaptive_kept(const char *P, uint32_t un, const char *T, uint32_t um, int32_t x, int32_t o, int32_t e,
                             int32_t band, int64_t limit, int32_t lmin, int32_t dmax, int32_t *score, uint8_t *flags,
                             int32_t *kept, int64_t kept_cap, int64_t *nkept) {
    uint32_t ncig = 0;
    return wfa_adaptive_run(P, un, T, um, x, o, e, band, limit, lmin, dmax, score, flags, NULL, 0, &ncig, kept,
                            kept_cap, nkept);
}

/* ---- batch driver for the adaptive WFA (same layout as oracle_align_batch) ---- */

typedef struct {
    batch_job base;
    int32_t lmin, dmax;
} adaptive_job;

static void *adaptive_worker(void *arg) {
    adaptive_job *aj = (adaptive_job *)arg;
    batch_job *j = &aj->base;
    for (;;) {
        int64_t i = __atomic_fetch_add(&j->next, 1, __ATOMIC_RELAXED);
        if (i >= (int64_t)j->num_pairs) break;
        uint32_t *cig = NULL, cap = 0;
        if (j->cigars) { cig = j->cigars + j->cigar_off[i]; cap = (uint32_t)(j->cigar_off[i + 1] - j->cigar_off[i]); }
        int r = oracle_wfa_adaptive(j->reads + j->read_off[i], j->read_len[i], j->targets + j->target_off[i],
                                    j->target_len[i], j->x, j->o, j->e, j->band, j->limit[i], aj->lmin, aj->dmax,
                                    &j->scores[i], &j->flags[i], cig, cap, &j->cigar_lens[i]);
        if (r) j->err = r;
    }
    return NULL;
}

int oracle_wfa_adaptive_batch(const char *reads, const uint64_t *read_off, const uint32_t *read_len,
                              const char *targets, const uint64_t *target_off, const uint32_t *target_len,
                              uint64_t num_pairs, int32_t x, int32_t o, int32_t e, int32_t band, const int64_t *limit,
                              int32_t lmin, int32_t dmax, int32_t *scores, uint8_t *flags, uint32_t *cigars,
                              const uint64_t *cigar_off, uint32_t *cigar_lens, int threads) {
    adaptive_job aj = {{reads, targets, read_off, target_off, read_len, target_len, num_pairs, x, o, e, band, limit,
                        scores, flags, cigars, cigar_off, cigar_lens, 0, 0}, lmin, dmax};
    if (threads < 1) threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    if (!th) return -3;
    int started = 0;
    for (int t = 0; t < threads; ++t)
        if (pthread_create(&th[t], NULL, adaptive_worker, &aj) == 0) ++started;
    if (started == 0) adaptive_worker(&aj);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    return aj.base.err;
}

/* ---------------------------------------------------------------------------
 * GenASM (Section 2.4.3): an edit-distance aligner built on the bitap
 * algorithm, with a traceback added, under a threshold of k edits.  The paper
 * names the method and its working data (a bit mask per pattern character,
 * status bit-vectors, one intermediate vector per kind of edit) but prints
 * neither the algorithm nor its parameters.  Our reading, step by step:
 *
 *   The pair is aligned window by window from its start.  At read position i
 *   and target position j a window holds wp = min(W, n-i) read bases and
 *   wt = min(W, m-j) target bases.  The read ends inside it when n-i <= W,
 *   the target when m-j <= W; the window is final when both do.
 *
 *   Window distance.  For a in [0, wp] and c in [0, wt], f(a, c) is the least
 *   number of edits of a path from (a, c) to the window's far edge.  A side
 *   whose sequence goes on past the window is a free end: the path may stop
 *   as soon as that window is used up, leaving the rest to the next window.
 *   A side whose sequence ends inside the window is not: bases left on the
 *   other side then cost one gap edit each.  (In the final window this is the
 *   global alignment of the two rests.)  Written out as the suffix
 *   edit-distance recurrence:
 *     f(wp, c) = read ends ? wt - c : 0      f(a, wt) = target ends ? wp - a : 0
 *     f(a, c)  = min(f(a+1, c+1) + [read base != target base], f(a+1, c) + 1, f(a, c+1) + 1)
 *   A bitap status vector of distance level d holds, for every read suffix,
 *   the bit [f(a, c) <= d]; the window distance is d = f(0, 0).  Any way the
 *   alignment goes on from (i, j) crosses the window's far edge, so it makes
 *   at least d more edits: a window whose distance exceeds the edits left
 *   (k minus the edits so far) rejects the pair at once, which is the same
 *   outcome as finishing it (an early exit; the distance levels of a window
 *   never need to go past the edits left).
 *
 *   Traceback, forward from (0, 0) with budget d: take the first op of this
 *   list whose successor still fits the budget (an edit spends one):
 *     after an I, I first; after a D, D first (gap extension before anything
 *     else: the affine-gap preference); then M (bases equal, f(a+1, c+1) <= d),
 *     X (bases differ, f(a+1, c+1) <= d-1), I (f(a+1, c) <= d-1),
 *     D (f(a, c+1) <= d-1).
 *   With the read window used up only D remains, with the target window used
 *   up only I.  A non-final window stops once W-O read bases or W-O target
 *   bases have been consumed in it (or at its corner); the final window runs
 *   to its corner.  Then i += a, j += c and the next window starts; the last
 *   op so far counts as the previous op.
 *
 *   When one sequence is used up, the rest of the other is one gap.  The
 *   score is the number of edits of the alignment; as soon as the edits so
 *   far exceed k the pair is rejected (score -1, flag 1, no CIGAR).
 *
 * W = 64 (one machine word per status vector) and O = 24 are our defaults.
 * Pinned by: with both sequences inside one window the score is the edit
 * distance (against the separate Levenshtein routine and brute force) and the
 * CIGAR the first optimal op string in the order above (brute force over all
 * op strings); hand-worked multi-window examples; closed forms; and validity
 * invariants at any size (tests/test_oracle_genasm.py).
 * --------------------------------------------------------------------------- */

/* one window: fill f ((wp+1) x (wt+1), row a, column c) */
static void genasm_window_table(const char *R, int wp, const char *Tt, int wt, int end_r, int end_t, int32_t *f) {
#define F(a, c) f[(size_t)(a) * (size_t)(wt + 1) + (size_t)(c)]
    for (int c = 0; c <= wt; ++c) F(wp, c) = end_r ? wt - c : 0;
    for (int a = 0; a <= wp; ++a) F(a, wt) = end_t ? wp - a : 0;
    for (int a = wp - 1; a >= 0; --a)
        for (int c = wt - 1; c >= 0; --c)
            F(a, c) = min3(F(a + 1, c + 1) + (R[a] != Tt[c]), F(a + 1, c) + 1, F(a, c + 1) + 1);
#undef F
}

int oracle_genasm(const char *P, uint32_t n, const char *T, uint32_t m, int64_t k, int32_t W, int32_t O,
                  int32_t *score, uint8_t *flags, uint32_t *cigar, uint32_t cap, uint32_t *ncig) {
    *score = -1; *flags = 0; *ncig = 0;
    if (W < 1 || W > 64 || O < 0 || O >= W) return -1;
    int32_t *f = (int32_t *)malloc((size_t)(W + 1) * (size_t)(W + 1) * sizeof(int32_t));
    char *ops = (char *)malloc((size_t)n + m + 1);
    if (!f || !ops) { free(f); free(ops); return -3; }
    uint32_t i = 0, j = 0, nops = 0;
    int64_t used = 0;
    char prev = 0;
    int rejected = 0;
    while (i < n && j < m) {
        int wp = (int)((n - i) < (uint32_t)W ? (n - i) : (uint32_t)W);
        int wt = (int)((m - j) < (uint32_t)W ? (m - j) : (uint32_t)W);
        int end_r = (n - i) <= (uint32_t)W, end_t = (m - j) <= (uint32_t)W, final = end_r && end_t;
        genasm_window_table(P + i, wp, T + j, wt, end_r, end_t, f);
#define F(a, c) f[(size_t)(a) * (size_t)(wt + 1) + (size_t)(c)]
        int32_t d = F(0, 0);
        if (d > k - used) { rejected = 1; break; }
        int a = 0, c = 0;
        for (;;) {
            if (!final && (a >= W - O || c >= W - O)) break;
            if (a == wp && c == wt) break;
            char op;
            if (a == wp) op = 'D';
            else if (c == wt) op = 'I';
            else if (prev == 'I' && d >= 1 && F(a + 1, c) <= d - 1) op = 'I';
            else if (prev == 'D' && d >= 1 && F(a, c + 1) <= d - 1) op = 'D';
            else if (P[i + a] == T[j + c] && F(a + 1, c + 1) <= d) op = 'M';
            else if (P[i + a] != T[j + c] && d >= 1 && F(a + 1, c + 1) <= d - 1) op = 'X';
            else if (d >= 1 && F(a + 1, c) <= d - 1) op = 'I';
            else if (d >= 1 && F(a, c + 1) <= d - 1) op = 'D';
            else { free(f); free(ops); return -5; /* cannot happen: f(a, c) <= d */ }
            ops[nops++] = op;
            prev = op;
            if (op != 'M') { --d; ++used; }
            if (op == 'M' || op == 'X') { ++a; ++c; }
            else if (op == 'I') ++a;
            else ++c;
        }
#undef F
        i += (uint32_t)a; j += (uint32_t)c;
        if (used > k) { rejected = 1; break; }
    }
    if (!rejected) {
        /* one sequence is used up: the rest of the other is one gap */
        for (; i < n; ++i) { ops[nops++] = 'I'; ++used; }
        for (; j < m; ++j) { ops[nops++] = 'D'; ++used; }
        if (used > k) rejected = 1;
    }
    if (rejected) { *flags = 1; free(f); free(ops); return 0; }
    *score = (int32_t)used;
    uint32_t runs = 0;
    for (uint32_t q = 0; q < nops;) {
        char op = ops[q]; uint32_t len = 0;
        while (q < nops && ops[q] == op) { ++len; ++q; }
        if (cigar && runs < cap) cigar[runs] = (len << 4) | bam_code(op);
        ++runs;
    }
    *ncig = runs;
    if (cigar && runs > cap) *flags |= 2;
    free(f); free(ops);
    return 0;
}

/* ---- batch driver for GenASM (same layout as oracle_align_batch; x, o, e unused) ---- */

typedef struct {
    batch_job base;
    int32_t W, O;
} genasm_job;

static void *genasm_worker(void *arg) {
    genasm_job *gj = (genasm_job *)arg;
    batch_job *j = &gj->base;
    for (;;) {
        int64_t i = __atomic_fetch_add(&j->next, 1, __ATOMIC_RELAXED);
        if (i >= (int64_t)j->num_pairs) break;
        uint32_t *cig = NULL, cap = 0;
        if (j->cigars) { cig = j->cigars + j->cigar_off[i]; cap = (uint32_t)(j->cigar_off[i + 1] - j->cigar_off[i]); }
        int r = oracle_genasm(j->reads + j->read_off[i], j->read_len[i], j->targets + j->target_off[i],
                              j->target_len[i], j->limit[i], gj->W, gj->O, &j->scores[i], &j->flags[i], cig, cap,
                              &j->cigar_lens[i]);
        if (r) j->err = r;
    }
    return NULL;
}

int oracle_genasm_batch(const char *reads, const uint64_t *read_off, const uint32_t *read_len, const char *targets,
                        const uint64_t *target_off, const uint32_t *target_len, uint64_t num_pairs,
                        const int64_t *limit, int32_t W, int32_t O, int32_t *scores, uint8_t *flags,
                        uint32_t *cigars, const uint64_t *cigar_off, uint32_t *cigar_lens, int threads) {
    genasm_job gj = {{reads, targets, read_off, target_off, read_len, target_len, num_pairs, 0, 0, 0, -1, limit,
                      scores, flags, cigars, cigar_off, cigar_lens, 0, 0}, W, O};
    if (threads < 1) threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    if (!th) return -3;
    int started = 0;
    for (int t = 0; t < threads; ++t)
        if (pthread_create(&th[t], NULL, genasm_worker, &gj) == 0) ++started;
    if (started == 0) genasm_worker(&gj);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    return gj.base.err;
}
