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

