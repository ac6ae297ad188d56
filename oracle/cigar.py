"""ORACLE -- test infrastructure only.  CIGAR helpers used to check invariants.

A CIGAR is a list of uint32 runs, len << 4 | BAM code ('=' 7, 'X' 8, 'I' 1,
'D' 2).  I consumes a read base, D a target base (read as query, target as
reference).  The paper asks for the score and the alignment operations of
every pair (Section 2.2, Steps 4 and 5); this encoding is our reading.
"""
from __future__ import annotations

from . import CODE_OP, OP_CODE


def decode(runs) -> str:
    """Runs -> op string over M, X, I, D."""
    out = []
    for r in runs:
        r = int(r)
        out.append(CODE_OP[r & 15] * (r >> 4))
    return "".join(out)


def encode(ops: str) -> list[int]:
    """Op string -> runs (maximal runs of one op)."""
    runs, i = [], 0
    while i < len(ops):
        j = i
        while j < len(ops) and ops[j] == ops[i]:
            j += 1
        runs.append(((j - i) << 4) | OP_CODE[ops[i]])
        i = j
    return runs


def cost(ops: str, read: bytes, target: bytes, penalties) -> int | None:
    """Cost of an op string under gap-affine costs, or None if it is not a
    valid alignment of read to target (M on a mismatch, X on a match, or the
    wrong number of bases consumed).  A maximal run of L gap ops of one kind
    costs o + L*e; M costs 0 and X costs x."""
    _, x, o, e = penalties
    v = h = 0
    c = 0
    prev = None
    for op in ops:
        if op in "MX":
            if v >= len(read) or h >= len(target):
                return None
            if (read[v] == target[h]) != (op == "M"):
                return None
            c += 0 if op == "M" else x
            v += 1; h += 1
        elif op == "I":
            if v >= len(read):
                return None
            c += e + (o if prev != "I" else 0)
            v += 1
        elif op == "D":
            if h >= len(target):
                return None
            c += e + (o if prev != "D" else 0)
            h += 1
        else:
            return None
        prev = op
    if v != len(read) or h != len(target):
        return None
    return c


def reconstruct_target(ops: str, read: bytes) -> bytes | None:
    """Rebuild the target from the read and the ops; X positions are unknown
    and come back as b'?'.  None if the ops consume the wrong read length."""
    out = bytearray()
    v = 0
    for op in ops:
        if op == "M":
            if v >= len(read):
                return None
            out.append(read[v]); v += 1
        elif op == "X":
            if v >= len(read):
                return None
            out.append(ord("?")); v += 1
        elif op == "I":
            v += 1
        else:
            out.append(ord("?"))
    return bytes(out) if v == len(read) else None


def max_deviation(ops: str) -> int:
    """Largest |h - v| visited by the path."""
    v = h = best = 0
    for op in ops:
        if op in "MX":
            v += 1; h += 1
        elif op == "I":
            v += 1
        else:
            h += 1
        best = max(best, abs(h - v))
    return best
