"""The C-ABI library builds, loads and exports every function include/*.h declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import glob
import os
import re

from paper_2508_05990_b300 import bayer_me, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(bayer_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_binding_exports():
    assert declared_functions() == set(bayer_me.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu():
    build.build()
    assert bayer_me.status_string(0) == "ok"
    assert bayer_me.status_string(1) == "invalid argument"
    assert bayer_me.status_string(99) == "unknown status"


def test_params_struct_layout():
    # int x5, int[4], int, int[4], int[4], float, int, (pad) long long x2
    assert ctypes.sizeof(bayer_me.Params) == 96
    assert bayer_me.Params.ref_batch_stride.offset == 80
