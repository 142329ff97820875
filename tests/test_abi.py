"""The C-ABI library builds, loads and exports every entry point its headers
declare; host-side validation rejects bad arguments before touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(qpadl_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2510_03631_gb300 import pir
    return pir.load(build_if_missing=True)


def test_headers_declare_the_documented_calls():
    names = _declared_symbols()
    for required in ("qpadl_pir_setup", "qpadl_pir_hint", "qpadl_pir_answer", "qpadl_pir_answer_batch",
                     "qpadl_pir_recover", "qpadl_pir_query", "qpadl_pir_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_version(lib):
    from paper_2510_03631_gb300 import pir
    assert lib.qpadl_version() >= 10000
    assert pir.strerror(pir.QPADL_EINVAL) == "invalid argument"
    assert pir.strerror(pir.QPADL_EBUSY).startswith("busy")


@pytest.mark.parametrize("field,value", [("rows", 0), ("cols", 0), ("n", 0), ("n", 16385), ("log_q", 31),
                                         ("p", 3), ("p", 512), ("p", 1), ("rows", 1 << 31)])
def test_invalid_params_rejected_before_any_launch(lib, field, value):
    from paper_2510_03631_gb300 import pir
    prm = pir.params(64, 64, 8)
    setattr(prm, field, value)
    # gen_a validates the parameters before it looks at the device
    rc = lib.qpadl_pir_gen_a(ctypes.byref(prm), ctypes.c_void_p(16), None)
    assert rc == pir.QPADL_EINVAL
    rc = lib.qpadl_pir_query(ctypes.byref(prm), ctypes.c_void_p(16), ctypes.c_void_p(16),
                             ctypes.c_void_p(16), 0, ctypes.c_void_p(16), None)
    assert rc == pir.QPADL_EINVAL


def test_null_pointers_rejected(lib):
    from paper_2510_03631_gb300 import pir
    prm = pir.params(64, 64, 8)
    out = ctypes.c_void_p()
    assert lib.qpadl_pir_setup(ctypes.byref(prm), None, None, ctypes.byref(out)) == pir.QPADL_EINVAL
    assert lib.qpadl_pir_answer(None, None, None, None) == pir.QPADL_EINVAL
    assert lib.qpadl_pir_answer_batch(None, None, 0, None, None) == pir.QPADL_EINVAL
    assert lib.qpadl_pir_hint(None, None, None, None) == pir.QPADL_EINVAL
    assert lib.qpadl_pir_destroy(None) == pir.QPADL_OK
    # target column out of range
    assert lib.qpadl_pir_query(ctypes.byref(prm), ctypes.c_void_p(16), ctypes.c_void_p(16),
                               ctypes.c_void_p(16), 64, ctypes.c_void_p(16), None) == pir.QPADL_EINVAL


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2510_03631_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "qpadl_oracle" not in text, path


@pytest.mark.parametrize("field,value", [("max_batch", 0), ("max_batch", 65536), ("num_streams", 0),
                                         ("num_streams", 9), ("max_inflight", 0), ("host_budget_bytes", 100),
                                         ("group_size_ratio", -1.0), ("group_size_ratio", float("nan"))])
def test_invalid_server_config_rejected_before_any_allocation(lib, field, value):
    from paper_2510_03631_gb300 import pir
    cfg = pir.server_config()
    setattr(cfg, field, value)
    out = ctypes.c_void_p()
    assert lib.qpadl_server_create(ctypes.byref(cfg), ctypes.byref(out)) == pir.QPADL_EINVAL
    assert out.value is None


def test_replay_rejects_a_null_server(lib):
    from paper_2510_03631_gb300 import pir
    assert lib.qpadl_server_replay(None, 0, None, None, None, None, None, None, None) == pir.QPADL_EINVAL


def test_delta_compression_calls_reject_bad_arguments(lib):
    # NULL pointers, an empty entry list, empty blocks and byte widths outside 1..4 fail before any
    # device work
    from paper_2510_03631_gb300 import pir
    w = ctypes.c_uint32(0)
    buf = ctypes.c_void_p(16)   # never dereferenced: every call below fails validation first
    assert lib.qpadl_pir_delta_width(None, 10, 4, ctypes.byref(w), None) == pir.QPADL_EINVAL
    assert lib.qpadl_pir_delta_width(buf, 0, 4, ctypes.byref(w), None) == pir.QPADL_EINVAL
    assert lib.qpadl_pir_delta_width(buf, 10, 0, ctypes.byref(w), None) == pir.QPADL_EINVAL
    for E, wd in ((0, 1), (4, 0), (4, 5)):
        assert lib.qpadl_pir_delta_encode(buf, 10, E, wd, buf, None) == pir.QPADL_EINVAL
        assert lib.qpadl_pir_delta_decode(buf, 1, E, wd, buf, None) == pir.QPADL_EINVAL
    assert lib.qpadl_pir_delta_encode(None, 10, 4, 1, buf, None) == pir.QPADL_EINVAL
    assert lib.qpadl_pir_delta_decode(buf, 0, 4, 1, buf, None) == pir.QPADL_EINVAL
    assert lib.qpadl_pir_delta_decode(buf, 1, 1 << 30, 4, buf, None) == pir.QPADL_EINVAL   # R' >= 2^31
