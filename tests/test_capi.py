"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point include/psdproj.h declares; host-side behaviour that needs
no GPU (defaults, status strings, argument rejection before any launch)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2410_19208_gb300 import build as b
    b.build()
    import paper_2410_19208_gb300 as ps
    return ps.lib()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(psdproj_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 19
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_status_strings(lib):
    import paper_2410_19208_gb300 as ps
    o = ps.Opts()
    lib.psdproj_default_opts(ctypes.byref(o))
    assert (o.prec, o.syrk_prec, o.N, o.out_mode) == (0, 0, 10, 0)
    assert (o.deterministic, o.spin_limit, list(o.reserved)) == (0, 0, [0, 0])
    for code in range(8):
        s = lib.psdproj_status_string(code)
        assert s.startswith(b"PSDPROJ")
    assert b"unknown" in lib.psdproj_status_string(99)


def test_rejects_bad_arguments_without_a_gpu(lib):
    # NULL contexts and out-of-range sizes fail in the argument checks,
    # before any CUDA call
    assert lib.psdproj_alg1(None, None, 10, 10, 2, 2, 0, 1, None, 10, None, 10, None, None) == 1
    assert lib.psdproj_destroy(None) == 0
    assert lib.psdproj_sync_status(None) == 1
    assert lib.psdproj_create(None, 0, None, 0) == 1
    assert lib.psdproj_set_reserved_sms(None, 1) == 1
    assert lib.psdproj_set_batch_streams(None, 4) == 1
    h = ctypes.c_void_p()
    # device index out of range (no device here, or index too large)
    assert lib.psdproj_create(ctypes.byref(h), 1 << 20, None, 0) != 0


def test_built_for_sm_103a_only():
    src = open(os.path.join(ROOT, "paper_2410_19208_gb300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src


def test_batched_descriptor_layout_and_rejection(lib):
    import ctypes
    import paper_2410_19208_gb300 as ps
    # the ctypes mirror of psdproj_problem has the C layout (8-byte members first)
    assert ctypes.sizeof(ps.Problem) == 112
    assert ps.Problem.seed.offset == 40 and ps.Problem.d_rank.offset == 104
    # no context: argument error before any device work
    assert lib.psdproj_batched(None, 1, None, None) == 1
    assert lib.psdproj_batched_grouped(None, 1, None, None) == 1
    assert lib.psdproj_batched_grouped(None, -1, None, None) == 1


def test_struct_layouts_match_the_c_header(tmp_path):
    # the ctypes mirrors against offsetof / sizeof from the header itself
    import subprocess
    import paper_2410_19208_gb300 as ps
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "psdproj.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu\\n", sizeof(psdproj_problem), sizeof(psdproj_request),\n'
        "         offsetof(psdproj_request, footprint_bytes), sizeof(psdproj_server_stats));\n"
        '  printf("%zu %zu %zu\\n", offsetof(psdproj_server_stats, inflight_peak_bytes), sizeof(psdproj_opts),\n'
        "         offsetof(psdproj_opts, spin_limit));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    got = [int(x) for x in out]
    want = [ctypes.sizeof(ps.Problem), ctypes.sizeof(ps.Request), ps.Request.footprint_bytes.offset,
            ctypes.sizeof(ps.ServerStats), ps.ServerStats.inflight_peak_bytes.offset, ctypes.sizeof(ps.Opts),
            ps.Opts.spin_limit.offset]
    assert got == want


def test_server_rejects_bad_arguments_without_a_gpu(lib):
    import paper_2410_19208_gb300 as ps
    h = ctypes.c_void_p()
    assert lib.psdproj_server_create(None, 0, 4, 1 << 30, None) == 1
    assert lib.psdproj_server_create(ctypes.byref(h), 0, 0, 1 << 30, None) == 1      # no workers
    assert lib.psdproj_server_create(ctypes.byref(h), 0, 4, 0, None) == 1            # no budget
    t = ctypes.c_uint64()
    assert lib.psdproj_server_submit(None, None, ctypes.byref(t)) == 1
    assert lib.psdproj_server_wait(None, 1, 0.0, None, None) == 1
    assert lib.psdproj_server_drain(None, 0.0) == 1
    st = ps.ServerStats()
    assert lib.psdproj_server_get_stats(None, ctypes.byref(st)) == 1
    assert lib.psdproj_server_destroy(None) == 0


def test_tuning_table_and_its_cache_file(lib, tmp_path, monkeypatch):
    # the batch tuning table needs no GPU: entries by bucket (log2 of the
    # median side and of the count), kept in the file PSDPROJ_TUNE_CACHE names
    import paper_2410_19208_gb300 as ps
    f1 = tmp_path / "tune1.txt"
    monkeypatch.setenv("PSDPROJ_TUNE_CACHE", str(f1))
    assert ps.tune_lookup("Test GPU", 7, 1000, 40) is None
    ps.tune_store("Test GPU", 7, 1000, 40, 4)
    assert ps.tune_lookup("Test GPU", 7, 1000, 40) == 4
    assert ps.tune_lookup("Test GPU", 7, 600, 33) == 4      # same bucket: 2^9 <= 600 < 2^10, 2^5 <= 33
    assert ps.tune_lookup("Test GPU", 7, 2048, 40) is None   # another side bucket
    assert ps.tune_lookup("Test GPU", 8, 1000, 40) is None   # another SM count
    assert ps.tune_lookup("Other", 7, 1000, 40) is None
    text = f1.read_text()
    assert "Test_GPU:7:9:5\t4" in text
    # a second file starts from its own contents
    f2 = tmp_path / "tune2.txt"
    f2.write_text("Test_GPU:7:9:5\t16\nbad line\nTest_GPU:7:3:1\t99\n")
    monkeypatch.setenv("PSDPROJ_TUNE_CACHE", str(f2))
    assert ps.tune_lookup("Test GPU", 7, 1000, 40) == 16
    assert ps.tune_lookup("Test GPU", 7, 8, 2) is None       # 99 is out of range (1..64): dropped
    with pytest.raises(RuntimeError):
        ps.tune_store("Test GPU", 7, 1000, 40, 65)
