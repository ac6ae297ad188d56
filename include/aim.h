/*
 * aim.h -- C ABI of the GB300 batched pairwise aligner.
 *
 * The library aligns very many independent read/target pairs, each under an
 * edit threshold, and returns for every pair a score and a CIGAR or a reject
 * flag.  This is the data-parallel core of the Alignment-in-Memory framework
 * (Section 2.2, Fig. 2, Steps 3-5: fetch a pair, align it and trace back the
 * alignment operations, write the score and operations back), with the
 * dispatch over DPUs replaced by one GPU.
 *
 * Algorithms (Section 2.4):
 *   AIM_ALGO_EDIT_NW       Needleman-Wunsch edit distance (Section 2.4.1), unit costs
 *                          (mismatch 1, gap open 0, gap extend 1); a banded DP.
 *   AIM_ALGO_GOTOH_BANDED  gap-affine global DP with three tables M, I, D
 *                          (Section 2.4.2, "SWG"; read as global alignment), banded.
 *   AIM_ALGO_WFA_AFFINE    gap-affine wavefront algorithm (Section 2.4.4), exact.
 *   AIM_ALGO_WFA_ADAPTIVE  WFA-adaptive (Section 2.4.4: keeps wavefronts narrow by
 *                          dropping outer diagonals), a heuristic; see
 *                          aim_set_wfa_adaptive for the rule and its CIGAR.
 *   AIM_ALGO_GENASM        GenASM (Section 2.4.3): bit-parallel (bitap) edit distance
 *                          with a traceback, in windows; see aim_set_genasm_window.
 * The three exact algorithms compute the same optimum for the same costs; the
 * CIGAR is the canonical one (below), so they agree bit for bit.
 *
 * Conventions (the paper fixes none of these; they are this library's):
 *   - Read P[0..n) is the query, target T[0..m) the reference.  Op M/'='
 *     is a match (cost 0), X a mismatch (cost x), I consumes a read base, D a
 *     target base.  A maximal run of L I's (or D's) costs o + L*e.
 *   - CIGAR runs are uint32 len << 4 | BAM code: '=' 7, X 8, I 1, D 2.
 *   - Canonical CIGAR: among all optimal alignments, the one whose op
 *     string read backward from the end is lexicographically smallest under
 *     X < I < D < M (gaps and mismatches as late as possible).
 *   - Threshold: limit = pen->max_score if >= 0; else max_edits for
 *     EDIT_NW; else max_edits * max(x, o + e).  A pair whose optimum
 *     (inside the band, if one is given) exceeds limit, or whose |n - m|
 *     exceeds the band, is rejected: score -1, flag AIM_F_REJECTED, 0 runs.
 *     max_edits < 0 and max_score < 0 means no threshold.
 *   - Sequences are 2-bit packed (aim_pack_2bit): A,C,G,T = 0,1,2,3, base j
 *     in word j/32 at bits [63-2(j%32)-1, 63-2(j%32)], every sequence starting
 *     on a word boundary, unused bits zero.
 *
 * Memory and streams: every data pointer is device memory owned by the
 * caller, unless a comment says "host".  The library owns only its context
 * workspace.  Calls are asynchronous on `stream` (a cudaStream_t, NULL = the
 * legacy default stream); argument errors are returned synchronously and
 * per-pair problems come back as flags, never as faults.  Calls that share
 * one context must not run concurrently (they share its workspace).
 * Outputs do not depend on batch composition, order or launch form.
 */
#ifndef AIM_H
#define AIM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AIM_API __attribute__((visibility("default")))
#else
#define AIM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aim_ctx aim_ctx;
typedef void *aim_stream_t; /* cudaStream_t */

/* call status */
enum {
    AIM_OK = 0,
    AIM_ERR_ARG = -1,         /* bad argument (null pointer, bad penalties, size out of range) */
    AIM_ERR_INPUT = -2,       /* bad input data detected synchronously */
    AIM_ERR_NOMEM = -3,       /* workspace too small even for one pair in flight */
    AIM_ERR_CUDA = -4,        /* a CUDA call failed; aim_last_cuda_error() has the code */
    AIM_ERR_UNSUPPORTED = -5, /* valid but not supported (e.g. a band wider than 127 for the DP) */
    AIM_ERR_CANCELLED = -6,   /* serving: the request was cancelled before it was admitted */
    AIM_ERR_BUSY = -7         /* serving: the request is already admitted (it completes as usual) */
};

/* per-pair flags (out_flags) */
enum {
    AIM_F_REJECTED = 1,        /* optimum above the limit, or |n - m| above the band */
    AIM_F_CIGAR_OVERFLOW = 2,  /* score valid; CIGAR needed more runs than its capacity (length still reported) */
    AIM_F_BAD_PAIR = 4,        /* non-ACGT byte, length above max_length, or per-pair max_edits above max_edits */
    AIM_F_STEP_CAP = 8         /* internal bound hit (scratch exhausted); no result */
};

typedef enum {
    AIM_ALGO_EDIT_NW = 0,
    AIM_ALGO_GOTOH_BANDED = 1,
    AIM_ALGO_WFA_AFFINE = 2,
    AIM_ALGO_WFA_ADAPTIVE = 3,  /* heuristic: see aim_set_wfa_adaptive */
    AIM_ALGO_GENASM = 4         /* windowed bitap edit distance: see aim_set_genasm_window */
} aim_algo_t;

typedef struct {
    int32_t match;      /* must be 0 (the wavefront algorithm needs it; Section 2.4.4 uses a=0) */
    int32_t mismatch;   /* x >= 1 */
    int32_t gap_open;   /* o >= 0 */
    int32_t gap_extend; /* e >= 1 */
    int32_t max_score;  /* >= 0: score limit; < 0: derive it from max_edits */
    int32_t band;       /* >= 0: only alignments with |h - v| <= band; < 0: none */
} aim_penalties_t;

/* Library version (major * 10000 + minor * 100 + patch). */
AIM_API int aim_version(void);

/* Static text for a status code. */
AIM_API const char *aim_status_string(int status);

/* cudaError_t of the last failing CUDA call in this thread (0 if none). */
AIM_API int aim_last_cuda_error(void);

/*
 * Create a context on CUDA device `device` with a device workspace of
 * workspace_bytes (0: 1 GiB).  The workspace holds per-warp scratch
 * (wavefront history, DP trace bits, CIGAR staging) and, for the ASCII entry
 * point, the packed copies of the sequences.  A call that needs more scratch
 * than fits runs fewer pairs at once; it fails with AIM_ERR_NOMEM only when
 * not even one pair's scratch fits.  Scratch beyond what the resident warps
 * need holds finished pairs whose tracebacks then run side by side (one lane
 * each), so a larger workspace can be faster; results never depend on it.
 * *out is NULL on failure.
 */
AIM_API int aim_create(aim_ctx **out, int device, size_t workspace_bytes);

/* Destroy a context (synchronises the device first).  NULL is accepted. */
AIM_API int aim_destroy(aim_ctx *ctx);

/*
 * 2-bit packer (one of the hot-path steps: sequences are moved to device
 * memory compactly before alignment; the paper transfers pairs to the memory
 * banks first, Section 2.2 Step 2).
 *   ascii        count sequences, sequence i at byte ascii + char_offsets[i], lengths[i] bytes
 *   packed       output words; sequence i written at packed + word_offsets[i], ceil(lengths[i]/32) words
 *   bad          optional (NULL): bad[i] = 1 if sequence i holds a byte other than A/C/G/T, else 0;
 *                such a sequence's words are written with the offending bases as 0
 * Returns AIM_ERR_ARG for null required pointers.
 */
AIM_API int aim_pack_2bit(aim_ctx *ctx, const uint8_t *ascii, const uint64_t *char_offsets, const uint32_t *lengths,
                  uint32_t count, uint64_t *packed, const uint64_t *word_offsets, uint8_t *bad,
                  aim_stream_t stream);

/*
 * Align num_pairs packed pairs (Section 2.2 Steps 3-5 for every pair at once).
 *   packed_reads/_targets      2-bit words (see aim_pack_2bit)
 *   read_offsets/target_offsets  word offset of each sequence (uint64, num_pairs entries)
 *   read_lengths/target_lengths  bases (uint32, num_pairs entries)
 *   max_length                 host value: upper bound on every read and target length in the call;
 *                              longer pairs are flagged AIM_F_BAD_PAIR.  Sizes the scratch.
 *   algo, pen                  algorithm and costs (pen is a host pointer)
 *   max_edits                  edit threshold (see the threshold rule above); when max_edits_per_pair
 *                              is given it must bound every entry, and pairs above it are flagged BAD_PAIR
 *   max_edits_per_pair         optional (NULL): per-pair thresholds (int32, device)
 *   out_scores                 int32 per pair: optimum, or -1 if rejected / bad
 *   out_cigars, cigar_offsets  optional (both NULL: scores only).  Pair i's runs go to
 *                              out_cigars + cigar_offsets[i], capacity cigar_offsets[i+1] - cigar_offsets[i]
 *                              (cigar_offsets has num_pairs + 1 entries)
 *   out_cigar_lens             optional: runs per pair (the full count even on overflow)
 *   out_flags                  uint8 per pair (AIM_F_*)
 * Limits: the wavefront algorithms need max_length <= 32000; the DP algorithms
 * need an effective band <= 127 (edit distance: min(band, limit); Gotoh:
 * min(band, (limit - o) / e)), else AIM_ERR_UNSUPPORTED.
 */
AIM_API int aim_align_batch(aim_ctx *ctx, const uint64_t *packed_reads, const uint64_t *packed_targets,
                    const uint64_t *read_offsets, const uint64_t *target_offsets, const uint32_t *read_lengths,
                    const uint32_t *target_lengths, uint32_t num_pairs, uint32_t max_length, int algo,
                    const aim_penalties_t *pen, int32_t max_edits, const int32_t *max_edits_per_pair,
                    int32_t *out_scores, uint32_t *out_cigars, const uint64_t *cigar_offsets,
                    uint32_t *out_cigar_lens, uint8_t *out_flags, aim_stream_t stream);

/*
 * Same as aim_align_batch on ASCII input: packs reads and targets into the
 * context workspace (ceil(max_length/32) words per sequence), then aligns.
 * Pairs with a non-ACGT byte get AIM_F_BAD_PAIR and score -1.
 *   reads/targets          bytes (device); sequence i at reads + read_char_offsets[i]
 */
AIM_API int aim_align_batch_ascii(aim_ctx *ctx, const uint8_t *reads, const uint8_t *targets,
                          const uint64_t *read_char_offsets, const uint64_t *target_char_offsets,
                          const uint32_t *read_lengths, const uint32_t *target_lengths, uint32_t num_pairs,
                          uint32_t max_length, int algo, const aim_penalties_t *pen, int32_t max_edits,
                          const int32_t *max_edits_per_pair, int32_t *out_scores, uint32_t *out_cigars,
                          const uint64_t *cigar_offsets, uint32_t *out_cigar_lens, uint8_t *out_flags,
                          aim_stream_t stream);

/*
 * Host-buffer form: aim_align_batch_ascii from HOST memory to HOST memory in
 * one blocking call, the transfers inside it (the paper's timed region covers
 * the transfer of the pairs in, alignment, traceback and the transfer of the
 * scores and operations back: Section 2.2, Steps 2-6; Section 3.1).
 *   Every pointer except ctx and pen is host memory.  Inputs as for
 *   aim_align_batch_ascii (byte offsets into reads/targets, any layout);
 *   cigar_offsets has num_pairs + 1 non-decreasing entries and pair i's runs go
 *   to out_cigars + cigar_offsets[i] (entries past its run count are written as
 *   zero).  Pinned (page-locked) host buffers let the copies overlap the
 *   kernels; pageable ones work but copy synchronously.
 *   chunk_pairs   pairs per chunk (0: a quarter of the batch, at least 65,536)
 *   bytes_moved   optional host[2]: bytes copied host-to-device and device-to-host
 * The batch goes through the device in chunks, two device slots in turn: while
 * one chunk aligns, the next one's inputs copy in and the previous one's
 * results copy out.  AIM_ALGO_WFA_AFFINE runs the batched form (each slot holds
 * a batch plan, autotuned on the first chunk; a short last chunk is padded with
 * empty pairs; each slot's plan takes half of the context workspace as its
 * scratch, so one chunk's launches overlap the next one's); the other
 * algorithms run the plain form per chunk.  The slots, streams and plans stay
 * in the context for later calls of the same shape (algorithm, costs,
 * thresholds, max_length, chunk size), whose first call pays for planning;
 * they are freed by aim_destroy or replaced by a call of another shape.
 * Each chunk's byte ranges are found, and its cigar_offsets checked, when its
 * turn comes, overlapping the device work of the chunks before it; the slots
 * are sized from the first chunk (with a quarter of headroom) and grow when a
 * later chunk needs more, once the earlier chunks' results are in host memory.
 * A decreasing cigar_offsets entry returns AIM_ERR_ARG; the chunks before the
 * one holding it have then been aligned and their results written.
 * Nothing else may use the context during the call.  Returns once every
 * result is in host memory; results equal aim_align_batch_ascii's bit for bit.
 */
AIM_API int aim_align_batch_host(aim_ctx *ctx, const uint8_t *reads, const uint8_t *targets,
                                 const uint64_t *read_char_offsets, const uint64_t *target_char_offsets,
                                 const uint32_t *read_lengths, const uint32_t *target_lengths, uint32_t num_pairs,
                                 uint32_t max_length, int algo, const aim_penalties_t *pen, int32_t max_edits,
                                 const int32_t *max_edits_per_pair, int32_t *out_scores, uint32_t *out_cigars,
                                 const uint64_t *cigar_offsets, uint32_t *out_cigar_lens, uint8_t *out_flags,
                                 uint32_t chunk_pairs, uint64_t *bytes_moved);

/*
 * Worst-case device scratch of one pair in flight for the gap-affine WFA
 * (AIM_ALGO_WFA_AFFINE) with `lanes` lanes per pair (as for aim_set_wfa_group;
 * 0: the library's choice), for pairs no longer than max_length under the
 * threshold rule above (pen, max_edits; host values): per-score records, CIGAR
 * run staging and the wavefront history, every wavefront as wide as its
 * sources allow and no wider than the 2 (S - s) / e + 1 diagonals (scaled
 * units) that can still end within the limit S, as the exact kernels clamp
 * it.  Groups of 32 lanes or whole blocks on reads longer than
 * 2,048 bp keep a compact history (2 bytes per wavefront entry up to 16,382
 * bp, 4 beyond, plus a small ring of the last few wavefronts) instead of 8
 * bytes per entry (Section 3.3: the long-read limit comes from memory).  The
 * workspace must hold at least 8 warps' worth of it (a whole-block group's
 * warps share one pair's).  Host-only; no device needed.
 */
AIM_API int aim_wfa_scratch_per_pair(uint32_t max_length, const aim_penalties_t *pen, int32_t max_edits, int lanes,
                                     size_t *bytes);

/*
 * WFA-adaptive parameters of a context (defaults 10 and 50; the paper gives
 * none).  After wavefront s (unless the pair finished at s), if it spans at
 * least min_length diagonals, each diagonal's distance to the end cell,
 * max(n - v, m - h) at its furthest offset, is compared with the smallest,
 * and outer diagonals (from both ends inward, up to the first one kept) more
 * than max_distance behind are dropped.  The CIGAR of AIM_ALGO_WFA_ADAPTIVE
 * follows the wavefront sources (mismatch, then I, then D for a match run's
 * start; gap extension before gap opening), so it is a valid alignment of the
 * reported score but not necessarily the canonical one; the score can exceed
 * the optimum and a pair can be rejected when pruning loses the end cell.
 * Scratch: a first pass sizes each pair's wavefront history (and its lanes per
 * pair) for pruned wavefronts of about 4 (max_distance + min_length) + 64
 * diagonals; pairs that outgrow it are aligned again in a second pass with
 * the exact algorithm's worst-case scratch, so results never depend on it.
 */
AIM_API int aim_set_wfa_adaptive(aim_ctx *ctx, int min_length, int max_distance);

/*
 * GenASM (AIM_ALGO_GENASM; Section 2.4.3: the bitap algorithm with a traceback
 * added, under a limit of k edits).  The paper prints no algorithm; this is
 * the library's reading.  Unit edit costs: the penalties are ignored (match
 * must be 0), k is the threshold of the threshold rule above (max_score if
 * >= 0, else max_edits or the per-pair array), and a band is not supported
 * (pen->band >= 0 gives AIM_ERR_UNSUPPORTED).  Any max_length is accepted.
 *
 * The pair is aligned in windows of `window` bases (1..64: one 64-bit word per
 * bitap status vector; default 64) that overlap by `overlap` bases (0..window-1,
 * default 24).  A window's distance is its edit distance to the window's far
 * edge, where an edge is free if its sequence goes on past the window (the
 * last window, holding both ends, is a global alignment).  A forward traceback
 * then takes, at each step, the first op that still fits the window's
 * distance: after an I, I first; after a D, D first (gap extension before
 * anything else, the affine-gap preference); then M, X, I, D.  A window that is
 * not the last stops once window - overlap read or target bases have been
 * consumed.  When one sequence is used up, the rest of the other is one gap.
 * The score is the number of edits of the whole alignment; a pair is rejected
 * iff it exceeds k.  Inside one window this is the exact edit distance; across
 * windows the score can exceed it.
 *
 * Work counter [4] (aim_stats_read) counts the 64-bit status vectors computed
 * (one distance level at one target position of one window).
 */
AIM_API int aim_set_genasm_window(aim_ctx *ctx, int window, int overlap);

/*
 * Batched form (wavefront algorithm): pairs of uneven length and error rate
 * in persistent launches over length-bucketed queues.  The batch is planned
 * once and then replayed:
 *   - packing, length/threshold bucketing of the pairs (on the device: a
 *     histogram, a scan and a scatter into an order array, heaviest work class
 *     first, buckets sharing a lanes-per-pair value kept contiguous) and one
 *     persistent alignment launch per lanes-per-pair value, each draining its
 *     queue range in that order, are recorded as one CUDA graph;
 *   - with `autotune`, the lanes per pair of every non-empty bucket are chosen by
 *     timed trial launches on a device-filling sample of its pairs (each choice cached in
 *     the context per costs, band and bucket); otherwise from the bucket's
 *     width class or an earlier cached choice.
 * Arguments are those of aim_align_batch_ascii (the same buffers are bound to
 * the plan: every aim_batch_run aligns their current contents, which may
 * change between runs as long as the shapes and bounds still hold).
 *   scratch_bytes  device scratch the plan may allocate for wavefronts (0: the
 *                  context's workspace size)
 * aim_batch_plan synchronises the device, allocates the plan's own device
 * memory (packed copies, bucket arrays, order, scratch) and launches trial
 * runs; aim_batch_run is asynchronous on `stream` (one graph launch).
 * Planning packs and buckets the bound inputs, so they must already hold
 * valid pairs (offsets and lengths inside their arrays) when it is called.
 * Results are bit-identical to aim_align_batch_ascii with AIM_ALGO_WFA_AFFINE.
 * One plan must not run concurrently with itself.
 */
typedef struct aim_batch aim_batch;
AIM_API int aim_batch_plan(aim_ctx *ctx, const uint8_t *reads, const uint8_t *targets,
                           const uint64_t *read_char_offsets, const uint64_t *target_char_offsets,
                           const uint32_t *read_lengths, const uint32_t *target_lengths, uint32_t num_pairs,
                           uint32_t max_length, const aim_penalties_t *pen, int32_t max_edits,
                           const int32_t *max_edits_per_pair, int32_t *out_scores, uint32_t *out_cigars,
                           const uint64_t *cigar_offsets, uint32_t *out_cigar_lens, uint8_t *out_flags,
                           size_t scratch_bytes, int autotune, aim_batch **out);
AIM_API int aim_batch_run(aim_batch *batch, aim_stream_t stream);
/* Per bucket (32): lanes per pair of its first pass and pairs seen at planning; returns the bucket count. */
AIM_API int aim_batch_info(aim_batch *batch, int *groups /* host[32] */, uint32_t *counts /* host[32] */);
/*
 * Two passes.  A bucket's full scratch is its worst case, which for long pairs
 * under a loose threshold leaves room for one pair per warp, while most pairs
 * end far below their threshold.  A bucket can therefore run a compact first
 * pass (fewer lanes per pair, a history of about 16 diagonals per lane) and
 * leave the pairs that outgrow it to a second pass with the full scratch; the
 * plan then builds the second pass's queues on the device from the first
 * pass's flags.  Results are the same either way (both passes are the exact
 * algorithm).  aim_batch_passes reports, per bucket, the first-pass lanes (0:
 * one pass only) and the full-pass lanes; it returns the number of buckets with
 * a compact first pass.  aim_set_batch_compact sets how later plans of the
 * context choose: 0 (default) by timed trials when autotuning, 1 always where
 * the scratch allows, 2 never.
 */
AIM_API int aim_batch_passes(aim_batch *batch, int *first_pass /* host[32] */, int *full_pass /* host[32] */);
AIM_API int aim_set_batch_compact(aim_ctx *ctx, int mode);
/*
 * Bound pass.  The exact algorithm clamps each wavefront to the diagonals
 * that can still end within the pair's limit (every gap base costs at least
 * the gap-extension cost), so a pair whose optimum lies far below its limit
 * gains little from the clamp.  A bucket can therefore first run a bound
 * pass: a forward pass of the same recurrences that keeps only the diagonals
 * within a few bases of the one closest to the end, stores no history and
 * traces nothing back.  The score at which it reaches the end is that of a
 * real alignment, so it bounds the optimum from above; the exact pass then
 * runs with min(limit, bound) as the pair's limit, and its clamp keeps only
 * a diamond around the optimal paths.  Scores, flags and CIGARs are those of
 * the exact pass alone.  aim_batch_bound_passes reports, per bucket, the
 * bound pass's lanes per pair (0: none) and returns the number of buckets
 * with one.  aim_set_batch_bound sets how later plans of the context choose:
 * 0 (default) by timed trials when autotuning, 1 always (reads up to 32,000
 * bp), 2 never.  Plans with a compact first pass run no bound pass.  Work
 * counters [0] and [1] include the bound pass's entries and windows.
 */
AIM_API int aim_batch_bound_passes(aim_batch *batch, int *bound_pass /* host[32] */);
AIM_API int aim_set_batch_bound(aim_ctx *ctx, int mode);
/*
 * Autotuner choices, so that a later process can plan exactly as a tuned one
 * did.  The context caches, per (costs, band, bucket, largest scaled score),
 * the lanes per pair, the compact first-pass lanes (0: none) and the
 * bound-pass lanes (0: none) its plans chose; plans made with autotune 0 take
 * cached choices where present.  aim_tune_export writes the cache as text,
 * one line "x o e band bucket smax lanes compact bound" per entry, into buf
 * (host, cap bytes, always NUL-terminated when cap > 0) and returns the
 * text's length without the NUL (a larger value than cap - 1 means buf was
 * too small; cap 0 only asks the length), or a negative status.
 * aim_tune_import adds the entries of such a text (host, NUL-terminated) to
 * the cache; a malformed line returns AIM_ERR_ARG and imports nothing.
 */
AIM_API int64_t aim_tune_export(aim_ctx *ctx, char *buf, size_t cap);
AIM_API int aim_tune_import(aim_ctx *ctx, const char *text);
AIM_API int aim_batch_destroy(aim_batch *batch);

/*
 * Serving loop (wavefront algorithm, continuous batching).  Requests of 1 to
 * many pairs arrive over time from host memory; a worker thread admits them
 * in arrival order whenever the server's fixed arenas have room: pinned
 * staging and device I/O (io_budget_bytes each, 0: 1 GiB) and device
 * wavefront scratch (wavefront_budget_bytes, 0: 4 GiB; the memory budget for
 * wavefront state, which never leaves the device).  A request's pairs are
 * grouped into jobs by their work bound (each job with its own scratch per
 * warp); an admitted request gets one scratch grant of up to 1/16 of the
 * budget, split between its jobs, and runs on its own streams (copy in, pack,
 * one launch per job side by side, copy out), so its jobs and the requests
 * that arrive while others run overlap on the device.  Jobs of the heaviest
 * work classes (work class >= 5, wavefronts over 256 diagonals; reads up to
 * 32,000 bp) run a bound pass first, as the batched form's tuner chooses for
 * such buckets.  Results are those of
 * aim_align_batch_ascii for the same pairs, independent of what else runs.
 * aim_server_create allocates the arenas and starts the worker thread.
 */
typedef struct aim_server aim_server;
typedef struct {
    const uint8_t *reads, *targets;                 /* host: ASCII */
    const uint64_t *read_offsets, *target_offsets;  /* host: byte offsets */
    const uint32_t *read_lengths, *target_lengths;  /* host */
    const int32_t *max_edits;                       /* host: per pair, or NULL to use max_edits_all */
    int32_t max_edits_all;                          /* >= 0 (the server needs a threshold) */
    uint32_t num_pairs;
    int32_t *out_scores;                            /* host, written when the request completes */
    uint8_t *out_flags;                             /* host */
    uint32_t *out_cigar_lens;                       /* host, optional */
    uint32_t *out_cigars;                           /* host, optional (with cigar_offsets) */
    const uint64_t *cigar_offsets;                  /* host, num_pairs + 1 entries, optional */
} aim_request;
/* pen: costs and band for every request (max_score must be < 0: thresholds are per pair). */
AIM_API int aim_server_create(aim_ctx *ctx, const aim_penalties_t *pen, size_t wavefront_budget_bytes,
                              size_t io_budget_bytes, aim_server **out);
/* Copies the request's inputs and queues it; the output buffers must stay valid until it completes (only each
 * pair's first cigar_lens[i] CIGAR entries are written; entries past them keep what the caller left there).
 * AIM_ERR_NOMEM: one pair's wavefront scratch or the request's I/O exceeds the server's budgets. */
AIM_API int aim_server_submit(aim_server *server, const aim_request *request, uint64_t *ticket);
/* *done = 1 once the request's results are in its output buffers; then the ticket is released and
 * *latency_ns (optional) holds submission-to-completion time.  Returns the request's status when done. */
AIM_API int aim_server_poll(aim_server *server, uint64_t ticket, int *done, uint64_t *latency_ns);
/* Blocks until the request completes (then as aim_server_poll with done = 1). */
AIM_API int aim_server_wait(aim_server *server, uint64_t ticket, uint64_t *latency_ns);
/* out[6]: submitted, completed, pairs completed, failed (cancelled ones included), queued now, running now. */
AIM_API int aim_server_stats(aim_server *server, uint64_t *out);
/* paused = 1: admit no further request (queued ones wait; running ones complete); 0: admit again. */
AIM_API int aim_server_pause(aim_server *server, int paused);
/* Cancels a request that is still queued: it leaves the queue at once and its ticket completes with
 * AIM_ERR_CANCELLED (poll/wait return that status; its output buffers are not touched).  AIM_ERR_BUSY: it was
 * already admitted and completes as usual.  AIM_ERR_ARG: unknown or already released ticket. */
AIM_API int aim_server_cancel(aim_server *server, uint64_t ticket);
/* Host-side fault injection, for tests of the failure path: the countdown-th request admitted from now on
 * (1: the next one) fails at launch as if a CUDA call had failed.  None of its work is enqueued, its arenas are
 * released, its ticket completes with AIM_ERR_CUDA, and the server carries on with the others.  0 disarms. */
AIM_API int aim_server_inject_failure(aim_server *server, uint32_t countdown);
/* Finishes every queued and running request (resuming a paused server), then frees the server. */
AIM_API int aim_server_destroy(aim_server *server);

/*
 * Lanes that cooperate on one pair in the wavefront kernel: 1, 2, 4, 8, 16 or 32
 * (a warp then aligns 32/lanes pairs in lockstep), 256 (a whole block of 8
 * warps aligns one pair: for long, noisy pairs), or 0 to let the library
 * choose from the widest wavefront the call's lengths and threshold allow.
 * Results do not depend on it; throughput does.  A choice whose scratch does
 * not fit the workspace is widened until it fits.
 */
AIM_API int aim_set_wfa_group(aim_ctx *ctx, int lanes);

/*
 * Work counters, accumulated by the kernels of every call since the last
 * reset (the figures behind cells/s and the roofline report):
 *   [0] wavefront entries computed by the WFA (each holds M~, I~, D~)
 *   [1] 32-base windows compared by the WFA extend
 *   [2] DP cells computed (in-band cells actually swept, up to early exit)
 *   [3] pairs aligned (every pair a kernel finished, any flag)
 *   [4] GenASM status vectors computed (one distance level at one target position of one window)
 * aim_stats_reset is asynchronous on `stream`; aim_stats_read synchronises
 * the device and copies the five counters to host memory `out`.
 */
AIM_API int aim_stats_reset(aim_ctx *ctx, aim_stream_t stream);
AIM_API int aim_stats_read(aim_ctx *ctx, uint64_t *out /* host, 5 entries */);

/*
 * Kernel timing.  While enabled, every call records a CUDA event pair on its
 * stream around each kernel it launches.  aim_timing_read synchronises on the
 * recorded events, returns the summed device time (ms) and the number of
 * launches of one kernel kind (0: 2-bit packer, 1: alignment kernels) since
 * the last read, then clears them.  Up to 4096 launches are kept per kind;
 * later ones are counted but not timed (*launches still counts them).
 */
AIM_API int aim_timing_enable(aim_ctx *ctx, int on);
AIM_API int aim_timing_read(aim_ctx *ctx, int kind, double *total_ms /* host */, int *launches /* host */);

/*
 * Measured int32 ALU throughput of `device` (a measurement helper: the
 * denominator of the roofline fraction reported for the alignment kernels,
 * whose work is integer add/max/compare/logic, not a dense contraction).
 * A kernel fills every SM with independent dependency chains of int32
 * operations, in two mixes: add/max/xor (the cell updates) and add/xor/shift/add
 * (the extend's window arithmetic).  *ops_per_s is the higher rate, in
 * source-level int32 operations per second (the unit of the work counters
 * above), each mix's rate the best of five timed launches; *kernel_ms
 * (optional) is that launch's duration and per_mix (optional, host[2]) each
 * mix's rate.  Synchronous; it allocates and frees a few KB of device memory.
 */
AIM_API int aim_measure_int_peak(int device, double *ops_per_s, double *kernel_ms, double *per_mix);

/*
 * aim_wfa_align_static -- the gap-affine wavefront aligner (as aim_align_batch
 * with AIM_ALGO_WFA_AFFINE) for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a deployment convenience.
 *
 * Who needs it: code that is not free to call cudaMalloc -- a plugin inside a
 * host application that owns a fixed device-memory budget, a latency-critical
 * loop that must not make a call that can block on the device, or a process
 * whose device footprint must be fixed at start-up.  Such callers cannot create
 * a context (aim_create allocates its workspace), so this call takes none.
 *
 * Memory: the call allocates nothing.  The caller passes inputs and outputs
 * exactly as for aim_align_batch.  Scratch comes from one 32 MiB device array
 * inside the library, which every GPU that loads the library's device code
 * holds until the process exits.  Every call on a device shares that array:
 * calls that overlap on the GPU (two streams, two threads) race and give wrong
 * results, so serialise them.  Each call clears what must start at zero.
 *
 * Set-up: the first call on each device (run it with that device current)
 * looks up the array's device address and caches it; make that first call
 * before any stream capture.  A reset context (cudaDeviceReset) or another
 * context on the device holds the array at another address: every call made
 * outside stream capture looks the address up again, so after a reset make one
 * call outside capture before capturing any.
 *
 * Limits: if one pair's scratch (from max_length, the threshold and the band;
 * about 5.5 KB for 150 bp reads at 6 edits, about 1.3 MB for 1 kbp at 100 edits)
 * exceeds the 32 MiB array, the call returns AIM_ERR_NOMEM and launches
 * nothing.  Smaller scratch needs let more warps run at once.  Otherwise
 * arguments, flags and results are those of aim_align_batch, bit for bit.
 */
AIM_API int aim_wfa_align_static(const uint64_t *packed_reads, const uint64_t *packed_targets,
                                 const uint64_t *read_offsets, const uint64_t *target_offsets,
                                 const uint32_t *read_lengths, const uint32_t *target_lengths, uint32_t num_pairs,
                                 uint32_t max_length, const aim_penalties_t *pen, int32_t max_edits,
                                 const int32_t *max_edits_per_pair, int32_t *out_scores, uint32_t *out_cigars,
                                 const uint64_t *cigar_offsets, uint32_t *out_cigar_lens, uint8_t *out_flags,
                                 aim_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* AIM_H */
