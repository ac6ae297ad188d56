"""ORACLE -- test infrastructure only.  The 2-bit sequence layout, base by base.

Layout (our reading of the packed 2-bit storage):
A, C, G, T -> 0, 1, 2, 3; base j of a sequence sits in word j // 32 at bits
[63 - 2*(j % 32) - 1, 63 - 2*(j % 32)], so the first base is in the top two
bits; every sequence starts on a word boundary; unused low bits are zero.
Any other byte is an input error.

Written one base at a time with Python integers so a reader can check it
against the statement above.  Used only to pin the device packer.
"""
from __future__ import annotations

import numpy as np

CODE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}


def words_for(length: int) -> int:
    return (length + 31) // 32


def pack_one(seq: bytes) -> list[int]:
    """One sequence -> its words (Python ints, 64-bit).  Raises on a non-ACGT byte."""
    words = [0] * words_for(len(seq))
    for j, b in enumerate(seq):
        if b not in CODE:
            raise ValueError(f"byte {b!r} at {j} is not A/C/G/T")
        shift = 62 - 2 * (j % 32)
        words[j // 32] |= CODE[b] << shift
    return words


def pack_all(seqs: list[bytes]) -> tuple[np.ndarray, np.ndarray]:
    """Sequences -> (words uint64, word offsets uint64[count + 1])."""
    offs = [0]
    out: list[int] = []
    for s in seqs:
        out.extend(pack_one(s))
        offs.append(len(out))
    return np.array(out, dtype=np.uint64), np.array(offs, dtype=np.uint64)
