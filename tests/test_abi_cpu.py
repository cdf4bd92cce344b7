"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every function that include/*.h declares.  No compute call is made
(there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in ("hsk.h", "hsk_stages.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s*]+(hsk_[a-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2407_07718_gb300 import _build
    return _build.build()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ["hsk_create", "hsk_count", "hsk_count_device", "hsk_destroy", "hsk_count_batch",
                     "hsk_submit", "hsk_poll", "hsk_wait", "hsk_release", "hsk_last_error",
                     "hsk_stage_encode", "hsk_stage_windows", "hsk_stage_supermers", "hsk_stage_sort",
                     "hsk_stage_rle", "hsk_stage_order"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_config_default_without_gpu(libpath):
    import paper_2407_07718_gb300 as hsk
    lib = hsk.load()
    cfg = hsk._Config()
    assert lib.hsk_config_default(ctypes.byref(cfg)) == 0
    assert cfg.hist_len == 65536 and cfg.radix_bits == 8 and cfg.seed == hsk.DEFAULT_SEED
    assert lib.hsk_config_default(None) == hsk.HSK_EINVAL
    # NULL-safe destroy, NULL context errors
    lib.hsk_destroy(None)
    assert lib.hsk_count(None, None, None, 0, 31, 17, 2, 8, None) == hsk.HSK_EINVAL


def test_host_pool_self_check(libpath):
    """The host block pool behind the batched and served results (size
    classes, best-fit reuse, the cap on kept blocks, arrays giving their
    blocks back); host memory only, no device call."""
    import paper_2407_07718_gb300 as hsk
    assert hsk.load().hsk_debug_host_pool_check() == 0


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA path include nothing from each other."""
    ora = open(os.path.join(ROOT, "oracle", "hsk_oracle.cpp")).read()
    assert "paper_2407_07718_gb300" not in ora and "#include \"" not in ora
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2407_07718_gb300")):
        for f in files:
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|include)\s+\S*", src).__str__(), f
