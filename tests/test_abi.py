"""The C-ABI library builds, loads without a GPU and exports every function
that include/sptt.h declares (no compute calls: this runs on CPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sptt.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(sptt_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libsptt():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_1812_05961_gb300 as sptt
    path = sptt.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("sptt_csf_build", "sptt_mttkrp", "sptt_cpd_als", "sptt_csf_free",
                     "sptt_cpd_create", "sptt_cpd_iterate", "sptt_status_str", "sptt_gram"):
        assert required in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(libsptt):
    missing = [n for n in _declared_functions() if not hasattr(libsptt, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libsptt):
    libsptt.sptt_status_str.restype = ctypes.c_char_p
    assert libsptt.sptt_status_str(0) == b"SPTT_OK"
    assert libsptt.sptt_status_str(-1) == b"SPTT_ERR_BAD_ARG"
    assert libsptt.sptt_status_str(-6) == b"SPTT_ERR_UNSUPPORTED"


def test_python_binding_names_match_abi(libsptt):
    import paper_1812_05961_gb300 as sptt
    for n in _declared_functions():
        assert hasattr(sptt, n), "binding lacks %s" % n


def test_oracle_is_not_imported_by_the_package():
    import paper_1812_05961_gb300
    pkg = os.path.dirname(paper_1812_05961_gb300.__file__)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "oracle.c" not in text, f
