"""CPU checks of the C interface: the library builds for sm_103a, loads, and
exports every function that include/chargax_b300.h declares.  No GPU call."""
import ctypes
import os
import re

import pytest

from paper_2507_01522_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "chargax_b300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\*?\s+\*?(chx_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_expected_entry_points():
    from paper_2507_01522_b300.chargax import EXPORTS
    assert declared_functions() == sorted(EXPORTS)


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_loads_library(lib_path):
    from paper_2507_01522_b300 import chargax
    L = chargax.load_library()
    assert L.chx_last_error() is not None


def test_build_targets_sm103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "--use_fast_math" not in B.FLAGS
