"""GB300 batched pairwise aligner: a thin Python binding over libaim.so.

The functions below carry the C names of include/aim.h and only marshal
arguments (torch CUDA tensors -> device pointers, the current torch stream
-> cudaStream_t).  Every step of the alignment runs in the library's CUDA
kernels; there is no CPU path, and importing a function whose library is not
built raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import torch

from .build import LIB

AIM_OK, AIM_ERR_ARG, AIM_ERR_INPUT, AIM_ERR_NOMEM, AIM_ERR_CUDA, AIM_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
AIM_ERR_CANCELLED, AIM_ERR_BUSY = -6, -7
AIM_F_REJECTED, AIM_F_CIGAR_OVERFLOW, AIM_F_BAD_PAIR, AIM_F_STEP_CAP = 1, 2, 4, 8
AIM_ALGO_EDIT_NW, AIM_ALGO_GOTOH_BANDED, AIM_ALGO_WFA_AFFINE, AIM_ALGO_WFA_ADAPTIVE, AIM_ALGO_GENASM = 0, 1, 2, 3, 4
ALGO = {"edit": AIM_ALGO_EDIT_NW, "gotoh": AIM_ALGO_GOTOH_BANDED, "wfa": AIM_ALGO_WFA_AFFINE,
        "wfa_adaptive": AIM_ALGO_WFA_ADAPTIVE, "genasm": AIM_ALGO_GENASM}


class aim_penalties_t(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32), ("max_score", ctypes.c_int32), ("band", ctypes.c_int32)]


class aim_request(ctypes.Structure):
    _fields_ = [("reads", ctypes.c_void_p), ("targets", ctypes.c_void_p), ("read_offsets", ctypes.c_void_p),
                ("target_offsets", ctypes.c_void_p), ("read_lengths", ctypes.c_void_p),
                ("target_lengths", ctypes.c_void_p), ("max_edits", ctypes.c_void_p), ("max_edits_all", ctypes.c_int32),
                ("num_pairs", ctypes.c_uint32), ("out_scores", ctypes.c_void_p), ("out_flags", ctypes.c_void_p),
                ("out_cigar_lens", ctypes.c_void_p), ("out_cigars", ctypes.c_void_p),
                ("cigar_offsets", ctypes.c_void_p)]


class AimError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_lib().aim_status_string(status).decode()} ({status})"
                         + (f", cudaError {_lib().aim_last_cuda_error()}" if status == AIM_ERR_CUDA else ""))


_LIB = None
EXPORTS = ["aim_version", "aim_status_string", "aim_last_cuda_error", "aim_create", "aim_destroy",
           "aim_pack_2bit", "aim_align_batch", "aim_align_batch_ascii", "aim_stats_reset", "aim_stats_read",
           "aim_timing_enable", "aim_timing_read"]


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is not built (run __graft_entry__.build()); the aligner has no CPU path")
        lib = ctypes.CDLL(LIB)
        p, u32, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32
        lib.aim_version.restype = ctypes.c_int
        lib.aim_status_string.restype = ctypes.c_char_p
        lib.aim_status_string.argtypes = [ctypes.c_int]
        lib.aim_create.argtypes = [ctypes.POINTER(p), ctypes.c_int, ctypes.c_size_t]
        lib.aim_destroy.argtypes = [p]
        lib.aim_pack_2bit.argtypes = [p, p, p, p, u32, p, p, p, p]
        lib.aim_align_batch.argtypes = [p, p, p, p, p, p, p, u32, u32, ctypes.c_int, ctypes.POINTER(aim_penalties_t),
                                        i32, p, p, p, p, p, p, p]
        lib.aim_align_batch_ascii.argtypes = lib.aim_align_batch.argtypes
        lib.aim_wfa_align_static.argtypes = [p, p, p, p, p, p, u32, u32, ctypes.POINTER(aim_penalties_t), i32, p, p,
                                             p, p, p, p, p]
        lib.aim_set_wfa_group.argtypes = [p, ctypes.c_int]
        lib.aim_set_wfa_adaptive.argtypes = [p, ctypes.c_int, ctypes.c_int]
        lib.aim_set_genasm_window.argtypes = [p, ctypes.c_int, ctypes.c_int]
        lib.aim_set_batch_compact.argtypes = [p, ctypes.c_int]
        lib.aim_batch_passes.argtypes = [p, p, p]
        lib.aim_set_batch_bound.argtypes = [p, ctypes.c_int]
        lib.aim_batch_bound_passes.argtypes = [p, p]
        lib.aim_tune_export.argtypes = [p, ctypes.c_char_p, ctypes.c_size_t]
        lib.aim_tune_export.restype = ctypes.c_int64
        lib.aim_tune_import.argtypes = [p, ctypes.c_char_p]
        lib.aim_batch_plan.argtypes = [p, p, p, p, p, p, p, u32, u32, ctypes.POINTER(aim_penalties_t), i32, p, p, p,
                                       p, p, p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(p)]
        lib.aim_batch_run.argtypes = [p, p]
        lib.aim_server_create.argtypes = [p, ctypes.POINTER(aim_penalties_t), ctypes.c_size_t, ctypes.c_size_t,
                                          ctypes.POINTER(p)]
        lib.aim_server_submit.argtypes = [p, ctypes.POINTER(aim_request), ctypes.POINTER(ctypes.c_uint64)]
        lib.aim_server_poll.argtypes = [p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_uint64)]
        lib.aim_server_wait.argtypes = [p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
        lib.aim_server_stats.argtypes = [p, p]
        lib.aim_server_destroy.argtypes = [p]
        lib.aim_server_pause.argtypes = [p, ctypes.c_int]
        lib.aim_server_cancel.argtypes = [p, ctypes.c_uint64]
        lib.aim_server_inject_failure.argtypes = [p, u32]
        lib.aim_batch_info.argtypes = [p, p, p]
        lib.aim_batch_destroy.argtypes = [p]
        lib.aim_stats_reset.argtypes = [p, p]
        lib.aim_stats_read.argtypes = [p, p]
        lib.aim_timing_enable.argtypes = [p, ctypes.c_int]
        lib.aim_timing_read.argtypes = [p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        lib.aim_align_batch_host.argtypes = [p, p, p, p, p, p, p, u32, u32, ctypes.c_int,
                                             ctypes.POINTER(aim_penalties_t), i32, p, p, p, p, p, p, u32, p]
        lib.aim_wfa_scratch_per_pair.argtypes = [u32, ctypes.POINTER(aim_penalties_t), i32, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_size_t)]
        lib.aim_measure_int_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), p]
        _LIB = lib
    return _LIB


def _check(rc: int, what: str):
    if rc != AIM_OK:
        raise AimError(rc, what)


# a C uint64/uint32 array may be passed as the signed torch type of the same width
_SAME_WIDTH = {torch.uint64: (torch.uint64, torch.int64), torch.uint32: (torch.uint32, torch.int32),
               torch.int32: (torch.int32, torch.uint32), torch.uint8: (torch.uint8, torch.int8)}


def _ptr(t, dtype=None, name="tensor", optional=False):
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype not in _SAME_WIDTH.get(dtype, (dtype,)):
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def penalties(mismatch=4, gap_open=6, gap_extend=2, max_score=-1, band=-1, match=0) -> aim_penalties_t:
    return aim_penalties_t(match, mismatch, gap_open, gap_extend, max_score, band)


def aim_version() -> int:
    return int(_lib().aim_version())


def aim_create(device: int = 0, workspace_bytes: int = 0) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(_lib().aim_create(ctypes.byref(ctx), device, workspace_bytes), "aim_create")
    return ctx


def aim_destroy(ctx) -> None:
    _check(_lib().aim_destroy(ctx), "aim_destroy")


def aim_pack_2bit(ctx, ascii, char_offsets, lengths, packed, word_offsets, bad=None, stream=None) -> None:
    u8, u64, u32 = torch.uint8, torch.uint64, torch.uint32
    _check(_lib().aim_pack_2bit(ctx, _ptr(ascii, u8, "ascii"), _ptr(char_offsets, u64, "char_offsets"),
                                _ptr(lengths, u32, "lengths"), int(lengths.numel()), _ptr(packed, u64, "packed"),
                                _ptr(word_offsets, u64, "word_offsets"), _ptr(bad, u8, "bad", True),
                                _stream(stream)), "aim_pack_2bit")


def aim_wfa_align_static(packed_reads, packed_targets, read_offsets, target_offsets, read_lengths, target_lengths,
                         max_length, pen, max_edits, max_edits_per_pair, out_scores, out_cigars, cigar_offsets,
                         out_cigar_lens, out_flags, stream=None) -> None:
    """The WFA with the library's fixed 32 MiB scratch: no context, nothing allocated (see aim.h)."""
    u64, u32 = torch.uint64, torch.uint32
    n = int(read_lengths.numel())
    args = _align_args(n, max_length, AIM_ALGO_WFA_AFFINE, pen, max_edits, max_edits_per_pair, out_scores,
                       out_cigars, cigar_offsets, out_cigar_lens, out_flags, stream)
    del args[2]   # no algorithm argument
    _check(_lib().aim_wfa_align_static(_ptr(packed_reads, u64, "packed_reads"),
                                       _ptr(packed_targets, u64, "packed_targets"),
                                       _ptr(read_offsets, u64, "read_offsets"),
                                       _ptr(target_offsets, u64, "target_offsets"),
                                       _ptr(read_lengths, u32, "read_lengths"),
                                       _ptr(target_lengths, u32, "target_lengths"), *args),
           "aim_wfa_align_static")


def aim_batch_plan(ctx, reads, targets, read_char_offsets, target_char_offsets, read_lengths, target_lengths,
                   max_length, pen, max_edits, max_edits_per_pair, out_scores, out_cigars, cigar_offsets,
                   out_cigar_lens, out_flags, scratch_bytes: int = 0, autotune: bool = True):
    """Plan a batched WFA run over the bound buffers (see aim.h); returns the plan handle."""
    u8, u64, u32 = torch.uint8, torch.uint64, torch.uint32
    n = int(read_lengths.numel())
    args = _align_args(n, max_length, AIM_ALGO_WFA_AFFINE, pen, max_edits, max_edits_per_pair, out_scores,
                       out_cigars, cigar_offsets, out_cigar_lens, out_flags, None)
    del args[2]          # no algorithm argument
    del args[-1]         # no stream
    plan = ctypes.c_void_p()
    _check(_lib().aim_batch_plan(ctx, _ptr(reads, u8, "reads"), _ptr(targets, u8, "targets"),
                                 _ptr(read_char_offsets, u64, "read_char_offsets"),
                                 _ptr(target_char_offsets, u64, "target_char_offsets"),
                                 _ptr(read_lengths, u32, "read_lengths"), _ptr(target_lengths, u32, "target_lengths"),
                                 *args, ctypes.c_size_t(scratch_bytes), int(bool(autotune)), ctypes.byref(plan)),
           "aim_batch_plan")
    return plan


def aim_batch_run(batch, stream=None) -> None:
    _check(_lib().aim_batch_run(batch, _stream(stream)), "aim_batch_run")


def aim_batch_info(batch):
    """(lanes per pair, pairs at planning) for each of the 32 buckets."""
    g = (ctypes.c_int * 32)(); c = (ctypes.c_uint32 * 32)()
    nb = _lib().aim_batch_info(batch, g, c)
    if nb < 0:
        raise AimError(nb, "aim_batch_info")
    return list(g)[:nb], list(c)[:nb]


def aim_batch_destroy(batch) -> None:
    _check(_lib().aim_batch_destroy(batch), "aim_batch_destroy")


def _host(a, dtype, name, optional=False):
    import numpy as np
    if a is None:
        if optional:
            return None, None
        raise ValueError(f"{name} is required")
    a = np.ascontiguousarray(a)
    if a.dtype.itemsize != np.dtype(dtype).itemsize:
        raise TypeError(f"{name} must be {np.dtype(dtype)}")
    return a, ctypes.c_void_p(a.ctypes.data)


def aim_server_create(ctx, pen, wavefront_budget_bytes: int = 0, io_budget_bytes: int = 0):
    s = ctypes.c_void_p()
    _check(_lib().aim_server_create(ctx, ctypes.byref(pen), wavefront_budget_bytes, io_budget_bytes, ctypes.byref(s)),
           "aim_server_create")
    return s


def aim_server_submit(server, reads, targets, read_offsets, target_offsets, read_lengths, target_lengths,
                      max_edits, out_scores, out_flags, out_cigar_lens=None, out_cigars=None, cigar_offsets=None,
                      max_edits_all: int = 0):
    """Queue one request (numpy host arrays; outputs are filled when it completes).  Returns (ticket, keep):
    `keep` holds the arrays the server reads or writes and must live until the request completes."""
    import numpy as np
    keep = []
    def h(a, dt, name, optional=False):
        arr, ptr = _host(a, dt, name, optional)
        keep.append(arr)
        return ptr
    q = aim_request(h(reads, np.uint8, "reads"), h(targets, np.uint8, "targets"),
                    h(read_offsets, np.uint64, "read_offsets"), h(target_offsets, np.uint64, "target_offsets"),
                    h(read_lengths, np.uint32, "read_lengths"), h(target_lengths, np.uint32, "target_lengths"),
                    h(max_edits, np.int32, "max_edits", True), int(max_edits_all), int(len(read_lengths)),
                    h(out_scores, np.int32, "out_scores"), h(out_flags, np.uint8, "out_flags"),
                    h(out_cigar_lens, np.uint32, "out_cigar_lens", True), h(out_cigars, np.uint32, "out_cigars", True),
                    h(cigar_offsets, np.uint64, "cigar_offsets", True))
    for name, a in (("out_scores", out_scores), ("out_flags", out_flags), ("out_cigar_lens", out_cigar_lens),
                    ("out_cigars", out_cigars)):
        if a is not None and not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
            raise TypeError(f"{name} must be a C-contiguous numpy array (the server writes into it)")
    t = ctypes.c_uint64()
    _check(_lib().aim_server_submit(server, ctypes.byref(q), ctypes.byref(t)), "aim_server_submit")
    return t.value, keep


def aim_server_poll(server, ticket: int):
    """(done, latency_s or None)."""
    d = ctypes.c_int(); lat = ctypes.c_uint64()
    rc = _lib().aim_server_poll(server, ticket, ctypes.byref(d), ctypes.byref(lat))
    _check(rc, "aim_server_poll")
    return bool(d.value), (lat.value * 1e-9 if d.value else None)


def aim_server_wait(server, ticket: int) -> float:
    """Block until the request completes; returns its latency in seconds."""
    lat = ctypes.c_uint64()
    _check(_lib().aim_server_wait(server, ticket, ctypes.byref(lat)), "aim_server_wait")
    return lat.value * 1e-9


def aim_server_stats(server) -> dict:
    import numpy as np
    o = np.zeros(6, np.uint64)
    _check(_lib().aim_server_stats(server, ctypes.c_void_p(o.ctypes.data)), "aim_server_stats")
    return dict(zip(["submitted", "completed", "pairs_completed", "failed", "queued", "running"], map(int, o)))


def aim_server_pause(server, paused: bool = True) -> None:
    _check(_lib().aim_server_pause(server, 1 if paused else 0), "aim_server_pause")


def aim_server_cancel(server, ticket: int) -> bool:
    """True: the queued request was cancelled (its ticket completes with AIM_ERR_CANCELLED); False: it was already
    admitted and completes as usual."""
    rc = _lib().aim_server_cancel(server, ticket)
    if rc == AIM_ERR_BUSY:
        return False
    _check(rc, "aim_server_cancel")
    return True


def aim_server_inject_failure(server, countdown: int = 1) -> None:
    """Host-side fault injection: the countdown-th request admitted from now fails at launch (0 disarms)."""
    _check(_lib().aim_server_inject_failure(server, int(countdown)), "aim_server_inject_failure")


def aim_server_destroy(server) -> None:
    _check(_lib().aim_server_destroy(server), "aim_server_destroy")


def aim_set_batch_compact(ctx, mode: int = 0) -> None:
    """Batch plans of this context: 0 tuner decides on compact first passes, 1 always, 2 never."""
    _check(_lib().aim_set_batch_compact(ctx, int(mode)), "aim_set_batch_compact")


def aim_batch_passes(plan) -> tuple[list[int], list[int], int]:
    """(first-pass lanes per bucket (0: one pass), full-pass lanes per bucket, buckets with a compact pass)."""
    import numpy as np
    first = np.zeros(32, np.int32); full = np.zeros(32, np.int32)
    n = _lib().aim_batch_passes(plan, ctypes.c_void_p(first.ctypes.data), ctypes.c_void_p(full.ctypes.data))
    if n < 0:
        _check(n, "aim_batch_passes")
    return first.tolist(), full.tolist(), int(n)


def aim_set_batch_bound(ctx, mode: int = 0) -> None:
    """Batch plans of this context: 0 tuner decides on bound passes, 1 always, 2 never."""
    _check(_lib().aim_set_batch_bound(ctx, int(mode)), "aim_set_batch_bound")


def aim_batch_bound_passes(plan) -> tuple[list[int], int]:
    """(bound-pass lanes per bucket (0: none), buckets with a bound pass)."""
    import numpy as np
    lanes = np.zeros(32, np.int32)
    n = _lib().aim_batch_bound_passes(plan, ctypes.c_void_p(lanes.ctypes.data))
    if n < 0:
        _check(n, "aim_batch_bound_passes")
    return lanes.tolist(), int(n)


def aim_tune_export(ctx) -> str:
    """The context's autotuner choices as text (one line per cached bucket choice)."""
    n = _lib().aim_tune_export(ctx, None, 0)
    if n < 0:
        _check(int(n), "aim_tune_export")
    buf = ctypes.create_string_buffer(int(n) + 1)
    _lib().aim_tune_export(ctx, buf, int(n) + 1)
    return buf.value.decode()


def aim_tune_import(ctx, text: str) -> None:
    """Add choices exported by aim_tune_export to the context's cache (plans with autotune off use them)."""
    _check(_lib().aim_tune_import(ctx, text.encode()), "aim_tune_import")


def aim_set_genasm_window(ctx, window: int = 64, overlap: int = 24) -> None:
    _check(_lib().aim_set_genasm_window(ctx, int(window), int(overlap)), "aim_set_genasm_window")


def aim_set_wfa_adaptive(ctx, min_length: int = 10, max_distance: int = 50) -> None:
    _check(_lib().aim_set_wfa_adaptive(ctx, int(min_length), int(max_distance)), "aim_set_wfa_adaptive")


def aim_set_wfa_group(ctx, lanes: int) -> None:
    _check(_lib().aim_set_wfa_group(ctx, int(lanes)), "aim_set_wfa_group")


def aim_stats_reset(ctx, stream=None) -> None:
    _check(_lib().aim_stats_reset(ctx, _stream(stream)), "aim_stats_reset")


def aim_stats_read(ctx) -> dict:
    import numpy as np
    out = np.zeros(5, np.uint64)
    _check(_lib().aim_stats_read(ctx, ctypes.c_void_p(out.ctypes.data)), "aim_stats_read")
    return {"wf_entries": int(out[0]), "extend_windows": int(out[1]), "dp_cells": int(out[2]), "pairs": int(out[3]),
            "bitap_words": int(out[4])}


def aim_timing_enable(ctx, on: bool = True) -> None:
    _check(_lib().aim_timing_enable(ctx, int(bool(on))), "aim_timing_enable")


def aim_timing_read(ctx, kind: int) -> tuple[float, int]:
    """(total device ms, launches) of kernel kind 0 (packer) or 1 (alignment) since the last read."""
    ms = ctypes.c_double(); n = ctypes.c_int()
    _check(_lib().aim_timing_read(ctx, kind, ctypes.byref(ms), ctypes.byref(n)), "aim_timing_read")
    return ms.value, n.value


def aim_align_batch_host(ctx, reads, targets, read_char_offsets, target_char_offsets, read_lengths, target_lengths,
                         max_length, algo, pen, max_edits, max_edits_per_pair, out_scores, out_cigars, cigar_offsets,
                         out_cigar_lens, out_flags, chunk_pairs: int = 0) -> tuple[int, int]:
    """Host numpy arrays in, host numpy arrays out, transfers inside the call (see aim.h; pinned arrays, e.g.
    torch.empty(..., pin_memory=True).numpy(), let the copies overlap the kernels).  Returns the bytes copied
    (host-to-device, device-to-host)."""
    import numpy as np
    n = len(read_lengths)

    def h(a, dt, name, optional=False, writable=False):
        if a is None:
            if optional:
                return None
            raise ValueError(f"{name} is required")
        if not isinstance(a, np.ndarray) or not a.flags.c_contiguous or a.dtype.itemsize != np.dtype(dt).itemsize:
            raise TypeError(f"{name} must be a C-contiguous numpy array of {np.dtype(dt)}")
        if writable and not a.flags.writeable:
            raise TypeError(f"{name} must be writable")
        return ctypes.c_void_p(a.ctypes.data)
    moved = np.zeros(2, np.uint64)
    a = ALGO[algo] if isinstance(algo, str) else int(algo)
    _check(_lib().aim_align_batch_host(
        ctx, h(reads, np.uint8, "reads"), h(targets, np.uint8, "targets"),
        h(read_char_offsets, np.uint64, "read_char_offsets"), h(target_char_offsets, np.uint64, "target_char_offsets"),
        h(read_lengths, np.uint32, "read_lengths"), h(target_lengths, np.uint32, "target_lengths"),
        ctypes.c_uint32(n), ctypes.c_uint32(max_length), ctypes.c_int(a), ctypes.byref(pen),
        ctypes.c_int32(max_edits), h(max_edits_per_pair, np.int32, "max_edits_per_pair", True),
        h(out_scores, np.int32, "out_scores", writable=True), h(out_cigars, np.uint32, "out_cigars", True, True),
        h(cigar_offsets, np.uint64, "cigar_offsets", True), h(out_cigar_lens, np.uint32, "out_cigar_lens", True, True),
        h(out_flags, np.uint8, "out_flags", writable=True), ctypes.c_uint32(chunk_pairs),
        ctypes.c_void_p(moved.ctypes.data)), "aim_align_batch_host")
    return int(moved[0]), int(moved[1])


def aim_wfa_scratch_per_pair(max_length: int, pen, max_edits: int, lanes: int = 0) -> int:
    """Worst-case device scratch (bytes) of one WFA pair in flight with `lanes` lanes per pair (see aim.h)."""
    b = ctypes.c_size_t()
    _check(_lib().aim_wfa_scratch_per_pair(ctypes.c_uint32(max_length), ctypes.byref(pen), ctypes.c_int32(max_edits),
                                           int(lanes), ctypes.byref(b)), "aim_wfa_scratch_per_pair")
    return b.value


def aim_measure_int_peak(device: int = 0) -> tuple[float, float, list[float]]:
    """(int32 operations per second, kernel ms, [add/max/xor rate, add/xor/shift rate]) of the library's ALU
    microbenchmark on `device`."""
    import numpy as np
    ops = ctypes.c_double(); ms = ctypes.c_double(); mix = np.zeros(2, np.float64)
    _check(_lib().aim_measure_int_peak(int(device), ctypes.byref(ops), ctypes.byref(ms),
                                       ctypes.c_void_p(mix.ctypes.data)), "aim_measure_int_peak")
    return ops.value, ms.value, mix.tolist()


def _align_args(num_pairs, max_length, algo, pen, max_edits, max_edits_per_pair, out_scores, out_cigars,
                cigar_offsets, out_cigar_lens, out_flags, stream):
    a = ALGO[algo] if isinstance(algo, str) else int(algo)
    return [ctypes.c_uint32(num_pairs), ctypes.c_uint32(max_length), ctypes.c_int(a), ctypes.byref(pen),
            ctypes.c_int32(max_edits), _ptr(max_edits_per_pair, torch.int32, "max_edits_per_pair", True),
            _ptr(out_scores, torch.int32, "out_scores"), _ptr(out_cigars, torch.uint32, "out_cigars", True),
            _ptr(cigar_offsets, torch.uint64, "cigar_offsets", True),
            _ptr(out_cigar_lens, torch.uint32, "out_cigar_lens", True), _ptr(out_flags, torch.uint8, "out_flags"),
            _stream(stream)]


def aim_align_batch(ctx, packed_reads, packed_targets, read_offsets, target_offsets, read_lengths, target_lengths,
                    max_length, algo, pen, max_edits, max_edits_per_pair, out_scores, out_cigars, cigar_offsets,
                    out_cigar_lens, out_flags, stream=None) -> None:
    u64, u32 = torch.uint64, torch.uint32
    n = int(read_lengths.numel())
    _check(_lib().aim_align_batch(ctx, _ptr(packed_reads, u64, "packed_reads"),
                                  _ptr(packed_targets, u64, "packed_targets"), _ptr(read_offsets, u64, "read_offsets"),
                                  _ptr(target_offsets, u64, "target_offsets"), _ptr(read_lengths, u32, "read_lengths"),
                                  _ptr(target_lengths, u32, "target_lengths"),
                                  *_align_args(n, max_length, algo, pen, max_edits, max_edits_per_pair, out_scores,
                                               out_cigars, cigar_offsets, out_cigar_lens, out_flags, stream)),
           "aim_align_batch")


def aim_align_batch_ascii(ctx, reads, targets, read_char_offsets, target_char_offsets, read_lengths,
                          target_lengths, max_length, algo, pen, max_edits, max_edits_per_pair, out_scores,
                          out_cigars, cigar_offsets, out_cigar_lens, out_flags, stream=None) -> None:
    u8, u64, u32 = torch.uint8, torch.uint64, torch.uint32
    n = int(read_lengths.numel())
    _check(_lib().aim_align_batch_ascii(ctx, _ptr(reads, u8, "reads"), _ptr(targets, u8, "targets"),
                                        _ptr(read_char_offsets, u64, "read_char_offsets"),
                                        _ptr(target_char_offsets, u64, "target_char_offsets"),
                                        _ptr(read_lengths, u32, "read_lengths"),
                                        _ptr(target_lengths, u32, "target_lengths"),
                                        *_align_args(n, max_length, algo, pen, max_edits, max_edits_per_pair,
                                                     out_scores, out_cigars, cigar_offsets, out_cigar_lens, out_flags,
                                                     stream)),
           "aim_align_batch_ascii")


class Aligner:
    """Owns a context; allocates outputs as torch tensors on its device."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0):
        self.device = device
        self.ctx = aim_create(device, workspace_bytes)

    def close(self):
        if self.ctx is not None:
            aim_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self, num_pairs: int, cigar_capacity=None):
        """Output tensors; cigar_capacity: per-pair run capacity (tensor/int) or None for scores only."""
        dev = torch.device("cuda", self.device)
        out = {"scores": torch.empty(num_pairs, dtype=torch.int32, device=dev),
               "flags": torch.empty(num_pairs, dtype=torch.uint8, device=dev),
               "cigar_lens": torch.empty(num_pairs, dtype=torch.int32, device=dev),
               "cigars": None, "cigar_offsets": None}
        if cigar_capacity is not None:
            cap = (torch.full((num_pairs,), int(cigar_capacity), dtype=torch.int64, device=dev)
                   if isinstance(cigar_capacity, int) else cigar_capacity.to(dev, torch.int64))
            off = torch.zeros(num_pairs + 1, dtype=torch.int64, device=dev)
            off[1:] = torch.cumsum(cap, 0)
            out["cigar_offsets"] = off
            out["cigars"] = torch.empty(int(off[-1].item()), dtype=torch.int32, device=dev)
        return out

    def align_ascii(self, reads, targets, read_char_offsets, target_char_offsets, read_lengths, target_lengths,
                    max_length, algo, pen, max_edits, max_edits_per_pair=None, out=None, stream=None):
        n = int(read_lengths.numel())
        out = out or self.outputs(n, None)
        return self._run_ascii(out, reads, targets, read_char_offsets, target_char_offsets, read_lengths,
                               target_lengths, max_length, algo, pen, max_edits, max_edits_per_pair, stream)

    def _run_ascii(self, out, reads, targets, read_char_offsets, target_char_offsets, read_lengths, target_lengths,
                   max_length, algo, pen, max_edits, max_edits_per_pair, stream):
        aim_align_batch_ascii(self.ctx, reads, targets, read_char_offsets, target_char_offsets, read_lengths,
                              target_lengths, max_length, algo, pen, max_edits, max_edits_per_pair, out["scores"],
                              out["cigars"], out["cigar_offsets"], out["cigar_lens"], out["flags"], stream)
        return out


def upload(*arrays, device: int = 0):
    """numpy arrays -> CUDA tensors (uint64 as int64, uint32 as int32: same bits)."""
    import numpy as np
    out = []
    for a in arrays:
        a = np.ascontiguousarray(a)
        if not a.flags.writeable:    # torch wraps only writable arrays; the copy to the device reads it once
            a = a.copy()
        if a.dtype == np.uint64:
            a = a.view(np.int64)
        elif a.dtype == np.uint32:
            a = a.view(np.int32)
        out.append(torch.from_numpy(a).to(torch.device("cuda", device)))
    return out
