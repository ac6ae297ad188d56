"""Seeded synthetic read/target pairs (no alignment arithmetic lives here).

The workload shapes stand in for the paper's datasets (Section 3.1, Table 2):
short reads of 100/150/250 bp and long reads up to 10 kbp, with a given
fraction of random edits.  The real read sets and the WFA repository's
generator are not available, so uniform random DNA with seeded edits is used.

Every pair is reproducible from (seed, index) alone: pair i draws from its own
xoshiro256** stream, so a sample of a large workload can be regenerated
without generating the rest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aimgen.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libaimgen.so")


def build(force: bool = False) -> str:
    """Compile the generator with gcc into gen/_build/libaimgen.so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Spec(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("len_min", ctypes.c_uint32), ("len_max", ctypes.c_uint32),
                ("rate_min", ctypes.c_double), ("rate_max", ctypes.c_double),
                ("unrelated_frac", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        lib.aimgen_sizes.argtypes = [ctypes.POINTER(_Spec), ctypes.c_uint64, ctypes.c_uint64, p, p, p, p, p, p]
        lib.aimgen_fill.argtypes = [ctypes.POINTER(_Spec), ctypes.c_uint64, ctypes.c_uint64, p, p, p, p]
        lib.aimgen_arrivals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint32,
                                        ctypes.c_uint32, p, p]
        _lib = lib
    return _lib


@dataclass(frozen=True)
class Workload:
    """A synthetic workload and the alignment settings it is run with."""
    name: str
    seed: int
    pairs: int
    len_min: int
    len_max: int
    rate_min: float
    rate_max: float
    unrelated_frac: float
    algo: str                      # "edit" | "gotoh" | "wfa" | "gotoh+wfa" | "wfa_adaptive" | "genasm"
    penalties: tuple               # (match, mismatch, gap_open, gap_extend)
    max_edits: int | None          # scalar threshold, or None when it is per pair
    max_edits_frac: float | None = None   # per-pair threshold ceil(frac * read length)
    band: int = -1

    def spec(self) -> _Spec:
        return _Spec(self.seed, self.len_min, self.len_max, self.rate_min, self.rate_max, self.unrelated_frac)


# The five workloads.  Names state what each one is.
EDIT_NW_100BP = Workload("edit_nw_100bp_2pct_10k", 1, 10_000, 100, 100, 0.02, 0.02, 0.0,
                         "edit", (0, 1, 0, 1), 10)
WFA_150BP = Workload("wfa_150bp_4pct_1M_unrel10", 2, 1_000_000, 150, 150, 0.04, 0.04, 0.10,
                     "wfa", (0, 4, 6, 2), 6)
GOTOH_WFA_250BP = Workload("gotoh_wfa_250bp_10pct_band25_1M", 3, 1_000_000, 250, 250, 0.10, 0.10, 0.0,
                           "gotoh+wfa", (0, 4, 6, 2), 25, band=25)
WFA_UNEVEN = Workload("wfa_uneven_100_1000bp_1_10pct_4M", 4, 4_000_000, 100, 1000, 0.01, 0.10, 0.0,
                      "wfa", (0, 4, 6, 2), None, max_edits_frac=0.10)
SERVE_LONG = Workload("serve_100_10000bp_1_10pct", 5, 0, 100, 10_000, 0.01, 0.10, 0.0,
                      "wfa", (0, 4, 6, 2), None, max_edits_frac=0.10)
ALL = [EDIT_NW_100BP, WFA_150BP, GOTOH_WFA_250BP, WFA_UNEVEN, SERVE_LONG]

# Long reads on their own (the serving workload's long end): 2-10 kbp, 1-10 % edits, thresholds at 10 % of length.
WFA_LONG = Workload("wfa_long_2000_10000bp_1_10pct_20k", 63, 20_000, 2000, 10_000, 0.01, 0.10, 0.0, "wfa",
                    (0, 4, 6, 2), None, max_edits_frac=0.10)

# WFA-adaptive in the shapes of the paper's Table 3 (read length x edit rate), with the paper's costs
# (x=3, o=4, e=1, Section 2.4.4) and thresholds at the edit rate: ceil(rate * length) edits.
TABLE3 = {
    (150, 2): Workload("wfa_adaptive_150bp_2pct_1M", 31, 1_000_000, 150, 150, 0.02, 0.02, 0.0, "wfa_adaptive",
                       (0, 3, 4, 1), 3),
    (150, 5): Workload("wfa_adaptive_150bp_5pct_1M", 32, 1_000_000, 150, 150, 0.05, 0.05, 0.0, "wfa_adaptive",
                       (0, 3, 4, 1), 8),
    (1000, 2): Workload("wfa_adaptive_1000bp_2pct_200k", 33, 200_000, 1000, 1000, 0.02, 0.02, 0.0, "wfa_adaptive",
                        (0, 3, 4, 1), 20),
    (1000, 5): Workload("wfa_adaptive_1000bp_5pct_200k", 34, 200_000, 1000, 1000, 0.05, 0.05, 0.0, "wfa_adaptive",
                        (0, 3, 4, 1), 50),
    (10000, 2): Workload("wfa_adaptive_10000bp_2pct_10k", 35, 10_000, 10_000, 10_000, 0.02, 0.02, 0.0,
                         "wfa_adaptive", (0, 3, 4, 1), 200),
    (10000, 5): Workload("wfa_adaptive_10000bp_5pct_4k", 36, 4_000, 10_000, 10_000, 0.05, 0.05, 0.0,
                         "wfa_adaptive", (0, 3, 4, 1), 500),
}


# GenASM (Section 2.4.3) at the paper's read lengths and edit levels (1 % and 5 %), unit costs, threshold
# k = ceil(rate * length) edits.
GENASM = {
    (100, 1): Workload("genasm_100bp_1pct_1M", 41, 1_000_000, 100, 100, 0.01, 0.01, 0.0, "genasm", (0, 1, 0, 1), 1),
    (100, 5): Workload("genasm_100bp_5pct_1M", 42, 1_000_000, 100, 100, 0.05, 0.05, 0.0, "genasm", (0, 1, 0, 1), 5),
    (150, 1): Workload("genasm_150bp_1pct_1M", 43, 1_000_000, 150, 150, 0.01, 0.01, 0.0, "genasm", (0, 1, 0, 1), 2),
    (150, 5): Workload("genasm_150bp_5pct_1M", 44, 1_000_000, 150, 150, 0.05, 0.05, 0.0, "genasm", (0, 1, 0, 1), 8),
    (250, 1): Workload("genasm_250bp_1pct_1M", 45, 1_000_000, 250, 250, 0.01, 0.01, 0.0, "genasm", (0, 1, 0, 1), 3),
    (250, 5): Workload("genasm_250bp_5pct_1M", 46, 1_000_000, 250, 250, 0.05, 0.05, 0.0, "genasm", (0, 1, 0, 1), 13),
    (1000, 1): Workload("genasm_1000bp_1pct_200k", 47, 200_000, 1000, 1000, 0.01, 0.01, 0.0, "genasm",
                        (0, 1, 0, 1), 10),
    (1000, 5): Workload("genasm_1000bp_5pct_200k", 48, 200_000, 1000, 1000, 0.05, 0.05, 0.0, "genasm",
                        (0, 1, 0, 1), 50),
}

@dataclass
class Pairs:
    """ASCII pairs laid out back to back; offsets are byte offsets into reads/targets."""
    reads: np.ndarray          # uint8
    read_off: np.ndarray       # uint64, one per pair
    read_len: np.ndarray       # uint32
    targets: np.ndarray        # uint8
    target_off: np.ndarray     # uint64
    target_len: np.ndarray     # uint32
    n_sub: np.ndarray          # uint32 edits applied, per kind
    n_ins: np.ndarray
    n_del: np.ndarray
    unrelated: np.ndarray      # uint8
    first: int = 0
    extra: dict = field(default_factory=dict)

    def __len__(self) -> int:
        return int(self.read_len.shape[0])

    def read(self, i: int) -> bytes:
        o = int(self.read_off[i]); return self.reads[o:o + int(self.read_len[i])].tobytes()

    def target(self, i: int) -> bytes:
        o = int(self.target_off[i]); return self.targets[o:o + int(self.target_len[i])].tobytes()


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def generate(w: Workload, count: int | None = None, first: int = 0, index: np.ndarray | None = None) -> Pairs:
    """Pairs [first, first+count) of workload w (or the listed pair indices)."""
    lib = _load()
    sp = w.spec()
    if index is not None:
        parts = [generate(w, 1, int(i)) for i in np.asarray(index)]
        return concat(parts)
    count = w.pairs if count is None else count
    rl = np.empty(count, np.uint32); tl = np.empty(count, np.uint32)
    ns = np.empty(count, np.uint32); ni = np.empty(count, np.uint32); nd = np.empty(count, np.uint32)
    un = np.empty(count, np.uint8)
    if lib.aimgen_sizes(ctypes.byref(sp), first, count, _ptr(rl), _ptr(tl), _ptr(ns), _ptr(ni), _ptr(nd), _ptr(un)):
        raise MemoryError("aimgen_sizes failed")
    ro = np.zeros(count, np.uint64); to = np.zeros(count, np.uint64)
    if count:
        ro[1:] = np.cumsum(rl[:-1], dtype=np.uint64); to[1:] = np.cumsum(tl[:-1], dtype=np.uint64)
    reads = np.empty(int(rl.sum(dtype=np.uint64)), np.uint8)
    targets = np.empty(int(tl.sum(dtype=np.uint64)), np.uint8)
    if lib.aimgen_fill(ctypes.byref(sp), first, count, _ptr(reads), _ptr(ro), _ptr(targets), _ptr(to)):
        raise MemoryError("aimgen_fill failed")
    return Pairs(reads, ro, rl, targets, to, tl, ns, ni, nd, un, first)


def concat(parts: list[Pairs]) -> Pairs:
    rl = np.concatenate([p.read_len for p in parts]); tl = np.concatenate([p.target_len for p in parts])
    reads = np.concatenate([p.reads for p in parts]) if parts else np.empty(0, np.uint8)
    targets = np.concatenate([p.targets for p in parts]) if parts else np.empty(0, np.uint8)
    ro = np.zeros(len(rl), np.uint64); to = np.zeros(len(tl), np.uint64)
    if len(rl):
        ro[1:] = np.cumsum(rl[:-1], dtype=np.uint64); to[1:] = np.cumsum(tl[:-1], dtype=np.uint64)
    cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
    return Pairs(reads, ro, rl, targets, to, tl, cat("n_sub"), cat("n_ins"), cat("n_del"), cat("unrelated"))


def from_strings(reads: list[bytes | str], targets: list[bytes | str]) -> Pairs:
    """Hand-written pairs in the same layout (for fixtures and edge cases)."""
    enc = lambda s: s.encode() if isinstance(s, str) else bytes(s)
    rb = [enc(s) for s in reads]; tb = [enc(s) for s in targets]
    rl = np.array([len(s) for s in rb], np.uint32); tl = np.array([len(s) for s in tb], np.uint32)
    ro = np.zeros(len(rb), np.uint64); to = np.zeros(len(tb), np.uint64)
    if len(rb):
        ro[1:] = np.cumsum(rl[:-1], dtype=np.uint64); to[1:] = np.cumsum(tl[:-1], dtype=np.uint64)
    z = np.zeros(len(rb), np.uint32)
    return Pairs(np.frombuffer(b"".join(rb), np.uint8).copy(), ro, rl,
                 np.frombuffer(b"".join(tb), np.uint8).copy(), to, tl, z, z.copy(), z.copy(),
                 np.zeros(len(rb), np.uint8))


def per_pair_max_edits(w: Workload, p: Pairs) -> np.ndarray:
    """Threshold per pair: the workload's scalar, or ceil(frac * read length)."""
    if w.max_edits is not None:
        return np.full(len(p), w.max_edits, np.int32)
    return np.ceil(w.max_edits_frac * p.read_len.astype(np.float64) - 1e-9).astype(np.int32)


def arrivals(seed: int, count: int, rate_per_s: float, size_min: int = 1, size_max: int = 4096):
    """Poisson arrival times (s) and log-uniform request sizes (pairs)."""
    lib = _load()
    t = np.empty(count, np.float64); s = np.empty(count, np.uint32)
    lib.aimgen_arrivals(seed, count, rate_per_s, size_min, size_max, _ptr(t), _ptr(s))
    return t, s


def script_cost_bound(p: Pairs, mismatch: int, gap_open: int, gap_extend: int) -> np.ndarray:
    """Cost of the generator's own edit script with every edit priced alone.

    Each substitution is one mismatch, each inserted or deleted base a
    one-base gap.  That script is one valid alignment, so the optimum can only
    be lower or equal (unrelated pairs get no bound: -1).
    """
    c = (p.n_sub.astype(np.int64) * mismatch
         + (p.n_ins.astype(np.int64) + p.n_del.astype(np.int64)) * (gap_open + gap_extend))
    return np.where(p.unrelated.astype(bool), -1, c)

