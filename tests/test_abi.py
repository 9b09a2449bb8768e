"""The C-ABI library loads on a machine without a GPU and exports every
function include/fbpt.h declares; the binding's struct layouts match the
library's.  No compute call is made here."""
import ctypes
import os
import re

import pytest

import paper_2311_10201_gb300 as fbpt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fbpt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(fbpt_[a-z_0-9]+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    fbpt.build()
    return fbpt.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fbpt_graph_create", "fbpt_sample", "fbpt_select_seeds", "fbpt_sample_batched"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert name in fbpt._SIGS, f"binding lacks {name}"


def test_struct_layouts_match(lib):
    sizes = (ctypes.c_uint64 * 3)()
    assert lib.fbpt_abi_sizes(sizes, 3) == 0
    assert list(sizes) == [ctypes.sizeof(fbpt.Opts), ctypes.sizeof(fbpt.RRSetsC), ctypes.sizeof(fbpt.Stats)]
    all6 = (ctypes.c_uint64 * 6)()
    assert lib.fbpt_abi_sizes(all6, 6) == 0
    assert list(all6) == [ctypes.sizeof(fbpt.Opts), ctypes.sizeof(fbpt.RRSetsC), ctypes.sizeof(fbpt.Stats),
                          ctypes.sizeof(fbpt.Tuning), ctypes.sizeof(fbpt.ImmResult), fbpt.TRACE_DTYPE.itemsize]
    assert lib.fbpt_version() == 1


def test_argument_errors_need_no_gpu(lib):
    h = ctypes.c_void_p()
    rc = lib.fbpt_graph_create(0, 0, None, None, None, 0, None, ctypes.byref(h))
    assert rc == fbpt.EINVAL
    assert b"n must be" in lib.fbpt_last_error()
    rc = lib.fbpt_sample(None, 0, 0, 10, None, None, None)
    assert rc == fbpt.EINVAL
