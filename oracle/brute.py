"""ORACLE -- test infrastructure only.  Brute-force optimum and canonical CIGAR.

Enumerates EVERY op string over {M, X, I, D} that aligns a tiny read to a tiny
target, prices each with the closed-form gap-affine cost (a maximal run of L
gap ops costs o + L*e; a mismatch costs x; a match 0), and returns the minimum
cost and, among the minimum-cost strings, the one that is lexicographically
smallest when read backward from the end under X < I < D < M.

This is the definition of the result, with no dynamic programming in it; it
pins the full-matrix DP oracle (score, tie-break and CIGAR) on small inputs.
Exponential: only for pairs with n + m <= ~9.
"""
from __future__ import annotations

from .cigar import cost

RANK = {"X": 0, "I": 1, "D": 2, "M": 3}


def _strings(n: int, m: int):
    """Every op sequence consuming exactly n read and m target bases."""
    def rec(v, h, acc):
        if v == n and h == m:
            yield "".join(acc); return
        if v < n and h < m:
            for op in "MX":
                acc.append(op); yield from rec(v + 1, h + 1, acc); acc.pop()
        if v < n:
            acc.append("I"); yield from rec(v + 1, h, acc); acc.pop()
        if h < m:
            acc.append("D"); yield from rec(v, h + 1, acc); acc.pop()
    yield from rec(0, 0, [])


def best(read: bytes, target: bytes, penalties, band: int = -1):
    """(score, ops) of the canonical optimum; (None, None) when no path fits the band."""
    found = None
    for ops in _strings(len(read), len(target)):
        c = cost(ops, read, target, penalties)
        if c is None:
            continue
        if band >= 0:
            v = h = 0; ok = True
            for op in ops:
                v += op in "MXI"; h += op in "MXD"
                if abs(h - v) > band:
                    ok = False; break
            if not ok:
                continue
        key = (c, [RANK[q] for q in reversed(ops)])
        if found is None or key < found[0]:
            found = (key, ops)
    if found is None:
        return None, None
    return found[0][0], found[1]


# GenASM traceback order (Section 2.4.3, our reading): after an I the I comes first, after a D the D; then M, X, I, D.
_GENASM_ORDER = {"I": "IMXD", "D": "DMXI"}


def _genasm_before(a: str, b: str) -> bool:
    """a precedes b: at their first difference, a's op comes earlier in the order that the op before it sets."""
    p = next(q for q in range(min(len(a), len(b))) if a[q] != b[q])
    order = _GENASM_ORDER.get(a[p - 1] if p else "", "MXID")
    return order.index(a[p]) < order.index(b[p])


def genasm_first(read: bytes, target: bytes):
    """(edit distance, the first optimal op string in the GenASM traceback order), by enumeration."""
    found = None
    for ops in _strings(len(read), len(target)):
        c = cost(ops, read, target, (0, 1, 0, 1))
        if c is None:
            continue
        if found is None or c < found[0] or (c == found[0] and _genasm_before(ops, found[1])):
            found = (c, ops)
    return found
