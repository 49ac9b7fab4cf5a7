"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (CPU only: no compute call needs a GPU here)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2509_21963_gb300 as cur
from paper_2509_21963_gb300 import build as curbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cur_[A-Za-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libcur():
    curbuild.build()
    return ctypes.CDLL(curbuild.LIB)


def test_every_declared_symbol_is_exported(libcur):
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in sorted(declared) if not hasattr(libcur, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    assert set(cur.EXPORTED) == _declared()


def test_argument_errors_without_a_gpu(libcur):
    # cur_create must fail cleanly (no abort) for a device that does not exist
    ptr = ctypes.c_void_p()
    libcur.cur_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_size_t]
    st = libcur.cur_create(ctypes.byref(ptr), 4096, None, 0)
    assert st == cur.CUR_EINVAL and not ptr.value
    libcur.cur_result_rank.argtypes = [ctypes.c_void_p]
    libcur.cur_result_rank.restype = ctypes.c_int64
    assert libcur.cur_result_rank(None) == 0
    libcur.cur_free.argtypes = [ctypes.c_void_p]
    libcur.cur_free(None)  # no-op


def test_header_comments_cite_the_paper():
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        assert "2509.21963" in text and "Algorithm 1" in text
