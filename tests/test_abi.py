"""The C ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"AIM_API\s+[\w\s\*]+?\b(aim_\w+)\s*\(", src)
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2208_01243_gb300 import build
    lib_path = build.build()
    declared = _declared()
    assert {"aim_create", "aim_destroy", "aim_pack_2bit", "aim_align_batch", "aim_align_batch_ascii"} <= set(declared)
    lib = ctypes.CDLL(lib_path)
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(aim_\w+)", out))
    assert set(declared) <= exported
    assert all(n.startswith("aim_") for n in exported)


def test_host_only_calls_without_gpu():
    import paper_2208_01243_gb300 as aim
    lib = aim._lib()
    assert aim.aim_version() >= 100
    assert lib.aim_status_string(aim.AIM_ERR_NOMEM) == b"workspace too small"
    # argument errors come back synchronously, before any device work
    assert lib.aim_align_batch(None, None, None, None, None, None, None, 0, 0, 0, None, 0, None, None, None, None,
                               None, None, None) == aim.AIM_ERR_ARG
    assert lib.aim_create(None, 0, 0) == aim.AIM_ERR_ARG



def test_wfa_scratch_per_pair_compact_history():
    """Host-only sizing query: on long reads, 32-lane and whole-block groups keep a compact history (2 bytes per
    wavefront entry up to 16,382 bp, 4 beyond) instead of the 8-byte entries of narrower groups."""
    import paper_2208_01243_gb300 as aim
    pen = aim.penalties(4, 6, 2)
    f8 = aim.aim_wfa_scratch_per_pair(10_000, pen, 1000, lanes=16)
    c16 = aim.aim_wfa_scratch_per_pair(10_000, pen, 1000, lanes=32)
    assert c16 == aim.aim_wfa_scratch_per_pair(10_000, pen, 1000, lanes=256)
    assert f8 / c16 > 3.8                       # 8 -> 2 bytes per entry, plus the records and the live ring
    c32 = aim.aim_wfa_scratch_per_pair(20_000, pen, 200, lanes=32)
    f8b = aim.aim_wfa_scratch_per_pair(20_000, pen, 200, lanes=16)
    assert 1.5 < f8b / c32 < 2.1                # 4-byte words against 8-byte entries, plus a 32-bit live ring
    # short reads keep the 8-byte entries whatever the group
    assert aim.aim_wfa_scratch_per_pair(150, pen, 6, lanes=32) == aim.aim_wfa_scratch_per_pair(150, pen, 6, lanes=4)
    # past 32,000 bp only the compact history can hold the offsets: 32 lanes at least, whatever is asked
    assert aim.aim_wfa_scratch_per_pair(40_000, pen, 100, lanes=4) == aim.aim_wfa_scratch_per_pair(40_000, pen, 100,
                                                                                                   lanes=32)
