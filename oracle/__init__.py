"""ORACLE -- test infrastructure only.

A plain, slow, obviously correct CPU implementation of what the alignment hot
path computes, used by the tests, the smoke check and the benchmark's CPU
baseline leg, and by nothing else.  It shares no code with the CUDA library
and never imports it.

Contents:
  aim_oracle.c  full-matrix 3-state DP (Gotoh; NW edit distance as the unit-cost
                special case) with the canonical backward state-set traceback,
                the same DP with rows recomputed block by block for long pairs,
                plus a textbook one-state Levenshtein (Sections 2.4.1, 2.4.2),
                the WFA-adaptive heuristic written out step by step
                (Section 2.4.4; exact WFA when pruning is off), and GenASM's
                windowed bit-vector distance with its forward traceback
                (Section 2.4.3), from the suffix edit-distance table
  brute.py      brute-force enumeration of every op string on tiny pairs
  cigar.py      decode / re-cost / reconstruct helpers for CIGAR runs
  pack.py       the 2-bit layout written out per base (pins the device packer)

Every function is pinned in tests/test_oracle_*.py against brute force,
closed forms, hand-worked examples and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aim_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

# BAM op codes of a CIGAR run (len << 4 | code)
OP_CODE = {"M": 7, "X": 8, "I": 1, "D": 2}
CODE_OP = {v: k for k, v in OP_CODE.items()}
F_REJECTED = 1
F_CIGAR_OVERFLOW = 2
F_BAD_PAIR = 4

UNIT = (0, 1, 0, 1)   # (match, mismatch, gap_open, gap_extend) of NW edit distance


def build(force: bool = False) -> str:
    """Compile aim_oracle.c with gcc into oracle/_build/liboracle.so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", _SRC, "-o", tmp, "-lpthread"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        i32, u32, u64, i64 = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
        lib.oracle_align.argtypes = [ctypes.c_char_p, u32, ctypes.c_char_p, u32, i32, i32, i32, i32, i64,
                                     ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint8), p, u32,
                                     ctypes.POINTER(u32)]
        lib.oracle_levenshtein.argtypes = [ctypes.c_char_p, u32, ctypes.c_char_p, u32]
        lib.oracle_levenshtein.restype = i32
        lib.oracle_align_batch.argtypes = [p, p, p, p, p, p, u64, i32, i32, i32, i32, p, p, p, p, p, p,
                                           ctypes.c_int]
        lib.oracle_align_rows.argtypes = [ctypes.c_char_p, u32, ctypes.c_char_p, u32, i32, i32, i32, i32, i64, i32,
                                          ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint8), p, u32,
                                          ctypes.POINTER(u32)]
        lib.oracle_align_rows_batch.argtypes = [p, p, p, p, p, p, u64, i32, i32, i32, i32, p, p, p, p, p, p,
                                                ctypes.c_int, i32]
        lib.oracle_wfa_adaptive.argtypes = [ctypes.c_char_p, u32, ctypes.c_char_p, u32, i32, i32, i32, i32, i64,
                                            i32, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint8), p, u32,
                                            ctypes.POINTER(u32)]
        lib.oracle_wfa_adaptive_kept.argtypes = [ctypes.c_char_p, u32, ctypes.c_char_p, u32, i32, i32, i32, i32,
                                                 i64, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint8),
                                                 p, i64, ctypes.POINTER(i64)]
        lib.oracle_wfa_adaptive_batch.argtypes = [p, p, p, p, p, p, u64, i32, i32, i32, i32, p, i32, i32, p, p, p, p,
                                                  p, ctypes.c_int]
        lib.oracle_genasm.argtypes = [ctypes.c_char_p, u32, ctypes.c_char_p, u32, i64, i32, i32, ctypes.POINTER(i32),
                                      ctypes.POINTER(ctypes.c_uint8), p, u32, ctypes.POINTER(u32)]
        lib.oracle_genasm_batch.argtypes = [p, p, p, p, p, p, u64, p, i32, i32, p, p, p, p, p, ctypes.c_int]
        _lib = lib
    return _lib


def limit_for(penalties, max_edits: int, max_score: int = -1, unit: bool = False) -> int:
    """Score limit of the threshold reading: max_score if given, else max_edits
    for edit distance, else max_edits * max(mismatch, gap_open + gap_extend)
    (every edit costs at most that much).  No threshold: effectively infinite."""
    if max_score >= 0:
        return int(max_score)
    if max_edits < 0:
        return 1 << 62
    if unit:
        return int(max_edits)
    _, x, o, e = penalties
    return int(max_edits) * max(x, o + e)


def align(read: bytes, target: bytes, penalties=(0, 4, 6, 2), band: int = -1, limit: int = 1 << 62,
          cigar: bool = True):
    """One pair -> (score, flags, [runs]).  Score -1 and flag 1 when rejected."""
    lib = _load()
    _, x, o, e = penalties
    sc = ctypes.c_int32(); fl = ctypes.c_uint8(); nc = ctypes.c_uint32()
    cap = len(read) + len(target) + 1
    buf = np.zeros(cap, np.uint32)
    r = lib.oracle_align(bytes(read), len(read), bytes(target), len(target), x, o, e, band, limit,
                         ctypes.byref(sc), ctypes.byref(fl), ctypes.c_void_p(buf.ctypes.data) if cigar else None,
                         cap, ctypes.byref(nc))
    if r:
        raise RuntimeError(f"oracle_align failed: {r}")
    return sc.value, fl.value, [int(v) for v in buf[:nc.value]]


# WFA-adaptive parameters (our reading; the paper gives none): prune when a wavefront spans at
# least ADAPT_MIN_LEN diagonals, dropping outer diagonals more than ADAPT_MAX_DIST behind the closest to the end.
ADAPT_MIN_LEN = 10
ADAPT_MAX_DIST = 50


def wfa_adaptive(read: bytes, target: bytes, penalties=(0, 4, 6, 2), band: int = -1, limit: int = 1 << 62,
                 min_len: int = ADAPT_MIN_LEN, max_dist: int = ADAPT_MAX_DIST):
    """One pair through the step-by-step WFA-adaptive (min_len < 0: no pruning) -> (score, flags, [runs])."""
    lib = _load()
    _, x, o, e = penalties
    sc = ctypes.c_int32(); fl = ctypes.c_uint8(); nc = ctypes.c_uint32()
    cap = len(read) + len(target) + 1
    buf = np.zeros(cap, np.uint32)
    r = lib.oracle_wfa_adaptive(bytes(read), len(read), bytes(target), len(target), x, o, e, band, limit, min_len,
                                max_dist, ctypes.byref(sc), ctypes.byref(fl), ctypes.c_void_p(buf.ctypes.data), cap,
                                ctypes.byref(nc))
    if r:
        raise RuntimeError(f"oracle_wfa_adaptive failed: {r}")
    return sc.value, fl.value, [int(v) for v in buf[:nc.value]]


def wfa_adaptive_kept(read: bytes, target: bytes, penalties=(0, 4, 6, 2), band: int = -1, limit: int = 1 << 62,
                      min_len: int = ADAPT_MIN_LEN, max_dist: int = ADAPT_MAX_DIST):
    """One pair through the WFA-adaptive -> (score, flags, {s: (lo, hi)}): the diagonal range kept at every score
    (scaled by gcd(x, o, e)) whose wavefront is not empty, up to the score the pair finished at."""
    lib = _load()
    _, x, o, e = penalties
    sc = ctypes.c_int32(); fl = ctypes.c_uint8(); nk = ctypes.c_int64()
    cap = 4 * (len(read) + len(target)) * max(x, o + e, 1) + 8
    buf = np.zeros(2 * cap, np.int32)
    r = lib.oracle_wfa_adaptive_kept(bytes(read), len(read), bytes(target), len(target), x, o, e, band, limit,
                                     min_len, max_dist, ctypes.byref(sc), ctypes.byref(fl),
                                     ctypes.c_void_p(buf.ctypes.data), cap, ctypes.byref(nk))
    if r:
        raise RuntimeError(f"oracle_wfa_adaptive_kept failed: {r}")
    kept = {s: (int(buf[2 * s]), int(buf[2 * s + 1])) for s in range(nk.value) if buf[2 * s] <= buf[2 * s + 1]}
    return sc.value, fl.value, kept


def wfa_adaptive_batch(pairs, penalties, limits: np.ndarray, band: int = -1, min_len: int = ADAPT_MIN_LEN,
                       max_dist: int = ADAPT_MAX_DIST, threads: int | None = None):
    """gen.Pairs through the WFA-adaptive -> (scores, flags, cigar_off, cigars, cigar_lens)."""
    lib = _load()
    n = len(pairs)
    _, x, o, e = penalties
    threads = threads or os.cpu_count() or 1
    lim = np.ascontiguousarray(limits, dtype=np.int64)
    scores = np.empty(n, np.int32); flags = np.empty(n, np.uint8); lens = np.zeros(n, np.uint32)
    cap = pairs.read_len.astype(np.uint64) + pairs.target_len.astype(np.uint64) + 1
    off = np.zeros(n + 1, np.uint64); off[1:] = np.cumsum(cap, dtype=np.uint64)
    cig = np.zeros(int(off[-1]), np.uint32)
    P = lambda a: ctypes.c_void_p(a.ctypes.data)
    r = lib.oracle_wfa_adaptive_batch(P(pairs.reads), P(pairs.read_off), P(pairs.read_len), P(pairs.targets),
                                      P(pairs.target_off), P(pairs.target_len), n, x, o, e, band, P(lim), min_len,
                                      max_dist, P(scores), P(flags), P(cig), P(off), P(lens), threads)
    if r:
        raise RuntimeError(f"oracle_wfa_adaptive_batch failed: {r}")
    return scores, flags, off, cig, lens


# GenASM window and overlap (our reading; the paper gives none): one 64-bit word per status vector.
GENASM_W = 64
GENASM_O = 24


def genasm(read: bytes, target: bytes, k: int = 1 << 62, W: int = GENASM_W, O: int = GENASM_O):
    """One pair through the windowed GenASM -> (score, flags, [runs]); k < 0 or huge: no threshold."""
    lib = _load()
    sc = ctypes.c_int32(); fl = ctypes.c_uint8(); nc = ctypes.c_uint32()
    cap = len(read) + len(target) + 1
    buf = np.zeros(cap, np.uint32)
    k = (1 << 62) if k < 0 else int(k)
    r = lib.oracle_genasm(bytes(read), len(read), bytes(target), len(target), k, W, O, ctypes.byref(sc),
                          ctypes.byref(fl), ctypes.c_void_p(buf.ctypes.data), cap, ctypes.byref(nc))
    if r:
        raise RuntimeError(f"oracle_genasm failed: {r}")
    return sc.value, fl.value, [int(v) for v in buf[:nc.value]]


def genasm_batch(pairs, limits: np.ndarray, W: int = GENASM_W, O: int = GENASM_O, threads: int | None = None):
    """gen.Pairs through the windowed GenASM -> (scores, flags, cigar_off, cigars, cigar_lens)."""
    lib = _load()
    n = len(pairs)
    threads = threads or os.cpu_count() or 1
    lim = np.ascontiguousarray(limits, dtype=np.int64)
    scores = np.empty(n, np.int32); flags = np.empty(n, np.uint8); lens = np.zeros(n, np.uint32)
    cap = pairs.read_len.astype(np.uint64) + pairs.target_len.astype(np.uint64) + 1
    off = np.zeros(n + 1, np.uint64); off[1:] = np.cumsum(cap, dtype=np.uint64)
    cig = np.zeros(int(off[-1]), np.uint32)
    P = lambda a: ctypes.c_void_p(a.ctypes.data)
    r = lib.oracle_genasm_batch(P(pairs.reads), P(pairs.read_off), P(pairs.read_len), P(pairs.targets),
                                P(pairs.target_off), P(pairs.target_len), n, P(lim), W, O, P(scores), P(flags),
                                P(cig), P(off), P(lens), threads)
    if r:
        raise RuntimeError(f"oracle_genasm_batch failed: {r}")
    return scores, flags, off, cig, lens


def align_rows(read: bytes, target: bytes, penalties=(0, 4, 6, 2), band: int = -1, limit: int = 1 << 62,
               rows_per_block: int = 0):
    """align() for long pairs: the same DP and traceback with rows recomputed block by block from saved rows
    (memory linear in the target length per block; rows_per_block <= 0: ceil(sqrt(n + 1)))."""
    lib = _load()
    _, x, o, e = penalties
    sc = ctypes.c_int32(); fl = ctypes.c_uint8(); nc = ctypes.c_uint32()
    cap = len(read) + len(target) + 1
    buf = np.zeros(cap, np.uint32)
    r = lib.oracle_align_rows(bytes(read), len(read), bytes(target), len(target), x, o, e, band, limit,
                              rows_per_block, ctypes.byref(sc), ctypes.byref(fl), ctypes.c_void_p(buf.ctypes.data),
                              cap, ctypes.byref(nc))
    if r:
        raise RuntimeError(f"oracle_align_rows failed: {r}")
    return sc.value, fl.value, [int(v) for v in buf[:nc.value]]


def levenshtein(read: bytes, target: bytes) -> int:
    return int(_load().oracle_levenshtein(bytes(read), len(read), bytes(target), len(target)))


def align_batch(pairs, penalties, limits: np.ndarray, band: int = -1, cigar: bool = True, threads: int | None = None,
                cigar_cap: np.ndarray | None = None, rows_per_block: int | None = None):
    """Align gen.Pairs on host threads (rows_per_block not None: the row-block form of align_rows, for long pairs).

    Returns (scores int32, flags uint8, cigar_off uint64[n+1], cigars uint32, cigar_lens uint32).
    """
    lib = _load()
    n = len(pairs)
    _, x, o, e = penalties
    threads = threads or os.cpu_count() or 1
    lim = np.ascontiguousarray(limits, dtype=np.int64)
    scores = np.empty(n, np.int32); flags = np.empty(n, np.uint8); lens = np.zeros(n, np.uint32)
    if cigar:
        cap = (cigar_cap if cigar_cap is not None
               else (pairs.read_len.astype(np.uint64) + pairs.target_len.astype(np.uint64) + 1))
        off = np.zeros(n + 1, np.uint64); off[1:] = np.cumsum(cap, dtype=np.uint64)
        cig = np.zeros(int(off[-1]), np.uint32)
        cp, op = ctypes.c_void_p(cig.ctypes.data), ctypes.c_void_p(off.ctypes.data)
    else:
        off = np.zeros(n + 1, np.uint64); cig = np.zeros(0, np.uint32); cp = op = None
    P = lambda a: ctypes.c_void_p(a.ctypes.data)
    if rows_per_block is None:
        r = lib.oracle_align_batch(P(pairs.reads), P(pairs.read_off), P(pairs.read_len), P(pairs.targets),
                                   P(pairs.target_off), P(pairs.target_len), n, x, o, e, band, P(lim), P(scores),
                                   P(flags), cp, op, P(lens), threads)
    else:
        r = lib.oracle_align_rows_batch(P(pairs.reads), P(pairs.read_off), P(pairs.read_len), P(pairs.targets),
                                        P(pairs.target_off), P(pairs.target_len), n, x, o, e, band, P(lim),
                                        P(scores), P(flags), cp, op, P(lens), threads, int(rows_per_block))
    if r:
        raise RuntimeError(f"oracle_align_batch failed: {r}")
    return scores, flags, off, cig, lens
