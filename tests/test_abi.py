"""CPU checks of the C-ABI library: it builds, loads, and exports exactly the
entry points include/sev.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "sev.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sev_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1604_03703_gb300 import build as B

    B.build()
    from paper_1604_03703_gb300 import _lib

    return _lib.load()


def test_header_declares_the_path():
    names = declared_functions()
    for required in ("sev_eigvalsh", "sev_full_to_band", "sev_band_to_band", "sev_tridiag_bisect"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(lib):
    from paper_1604_03703_gb300 import _lib

    assert set(_lib.SIGNATURES) == set(declared_functions())


def test_status_strings_and_kernel_names(lib):
    assert lib.sev_status_string(0) == b"ok"
    assert lib.sev_status_string(-3) == b"invalid argument"
    assert b"wait" in lib.sev_status_string(3)
    k = lib.sev_kernel_count()
    names = [lib.sev_kernel_name(i).decode() for i in range(k)]
    assert len(set(names)) == k and "syr2k" in names and "band_chase" in names


def test_null_handle_is_rejected(lib):
    assert lib.sev_eigvalsh(None, 4, None, 4, 2, 0, None) == -1
    assert lib.sev_tridiag_bisect(None, 4, None, None, 1e-14, None) == -1


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_1604_03703_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f


def test_band_schedule_host_query(lib):
    """The host-only schedule query: stage widths of the library (and the
    mirror the benchmark uses to name its workload agree with it)."""
    import bench
    from paper_1604_03703_gb300 import api, _lib as L

    assert api.band_schedule(16384, 128, L.SEV_MIXED) == [128, 32, 16, 1]
    assert api.band_schedule(16384, 64, L.SEV_MIXED) == [64, 16, 1]
    assert api.band_schedule(16384, 0, L.SEV_MIXED) == [64, 16, 1]  # default b0
    assert api.band_schedule(512, 32, L.SEV_FP64) == [32, 16, 1]
    assert api.band_schedule(10, 64, L.SEV_FP64) == [9, 1]  # b0 clamped to n - 1
    assert api.band_schedule(1, 8, L.SEV_FP64) == []
    for b0 in (2, 4, 8, 16, 24, 32, 48, 64, 96, 128, 256):
        for prec, elem in ((L.SEV_MIXED, 4), (L.SEV_FP64, 8)):
            assert api.band_schedule(100000, b0, prec) == bench.schedule(b0, elem), (b0, prec)
    buf = (__import__("ctypes").c_int * 2)()
    assert lib.sev_band_schedule(16384, 128, L.SEV_MIXED, buf, 2) == -5
    assert lib.sev_band_schedule(-1, 8, L.SEV_MIXED, buf, 2) == -1


def test_missing_library_fails_loudly():
    """Without the built library the binding raises; nothing falls back to
    the CPU (fresh interpreter, since a loaded library is cached)."""
    import subprocess
    import sys

    code = (
        "from paper_1604_03703_gb300 import _lib\n"
        "try:\n"
        "    _lib.load('/nonexistent/libsev.so')\n"
        "except RuntimeError as e:\n"
        "    assert 'no CPU fallback' in str(e), e\n"
        "    print('raised')\n"
    )
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "raised", out.stderr


def test_status_errors_are_raised(lib):
    from paper_1604_03703_gb300 import _lib as L

    with pytest.raises(L.SevError) as ei:
        L.check(3, "probe")  # SEV_ERR_TIMEOUT
    assert ei.value.code == 3 and "probe" in str(ei.value)
    with pytest.raises(L.SevError) as ei:
        L.check(-4, "probe")
    assert "argument 4" in str(ei.value)
    L.check(0, "probe")
