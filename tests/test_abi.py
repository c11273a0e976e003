"""The C ABI library: it builds for sm_103a, loads, and exports every entry
point include/ad.h declares.  Host-only entry points are exercised; nothing
here launches device work (no GPU needed)."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ad.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ad_[a-z0-9_]+)\s*\(", text)) - {"ad_alloc_fn", "ad_free_fn"})


@pytest.fixture(scope="module")
def lib():
    from paper_1601_05527_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 25
    raw = ctypes.CDLL(os.path.join(ROOT, "paper_1601_05527_gb300", "libad.so"))
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    from paper_1601_05527_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.exported_symbols())


def test_version_and_status_strings(lib):
    from paper_1601_05527_gb300 import _lib
    assert re.match(r"^\d+\.\d+\.\d+$", _lib.ad_version())
    for code, name in _lib.STATUS.items():
        assert _lib.ad_status_string(code) == name


def test_segment_ratios_match_paper_example(lib):
    from paper_1601_05527_gb300 import _lib
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "level_span_segments.json")))
    for seg in ("coarse", "middle", "fine"):
        r = _lib.ad_ml_segment_ratios(gold["levels"], seg, gold["level_span"], gold["value"])
        np.testing.assert_array_equal(r, gold[seg])


def test_argument_errors_without_device_work(lib):
    from paper_1601_05527_gb300 import _lib
    with pytest.raises(_lib.ADError) as ei:
        _lib.ad_ml_segment_ratios(0, "coarse", 1, 0.5)
    assert ei.value.status == 1
    assert "segment" in _lib.ad_last_error()
    with pytest.raises(_lib.ADError):
        _lib.ad_graph_create(-1, np.zeros(1, np.int64), np.zeros(0, np.int32))


def test_entry_points_fail_loudly_without_the_library():
    """No CPU fallback: with libad.so absent every entry point raises instead of
    computing anything (run in a fresh process, where nothing is loaded yet)."""
    import subprocess
    import sys
    code = (
        "import os, numpy as np\n"
        "real = os.path.exists\n"
        "os.path.exists = lambda p: False if str(p).endswith('libad.so') else real(p)\n"
        "from paper_1601_05527_gb300 import _lib as L\n"
        "for call in (lambda: L.ad_graph_create(2, np.array([0, 1, 2]), np.array([1, 0], np.int32), None),\n"
        "             lambda: L.ad_version(), lambda: L.load()):\n"
        "    try:\n"
        "        call()\n"
        "        print('computed')\n"
        "    except ImportError as e:\n"
        "        print('raised:', e)\n"
    )
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    lines = r.stdout.strip().splitlines()
    assert len(lines) == 3 and all(l.startswith("raised:") and "missing" in l for l in lines), r.stdout + r.stderr


def test_noalloc_entry_point_names_no_allocation():
    """ad_select_whole_graph_noalloc (for callers that cannot let a library
    allocate device memory) calls no allocating routine: its body and the
    helpers it calls in select.cu name no malloc/free or the library's own
    allocation helpers."""
    src = open(os.path.join(ROOT, "paper_1601_05527_gb300", "csrc", "select.cu")).read()
    start = src.index("// Whole-graph selection that allocates nothing")
    body = re.sub(r"//[^\n]*", "", src[start:])
    for word in ("cudaMalloc", "cudaFree", "malloc(", "free(", "dalloc", "dfree", "ensure(", "DevBuf",
                 "stage_in", "copy_in", "copy_out", "new ", "cudaMemPool"):
        assert word not in body, word
