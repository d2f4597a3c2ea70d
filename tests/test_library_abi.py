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


def test_pack_levels4_layout():
    """Two levels per byte, the even slot in the low nibble, each step's row
    padded to whole bytes (the layout chx_rollout_host_levels4 reads)."""
    import numpy as np
    from paper_2507_01522_b300.chargax import pack_levels4
    lv = np.array([[1, 2, 3, 4, 5], [10, 0, 15, 7, 9]], dtype=np.int8)
    p = pack_levels4(lv)
    assert p.dtype == np.uint8 and p.shape == (2, 3)
    np.testing.assert_array_equal(p, [[0x21, 0x43, 0x05], [0x0A, 0x7F, 0x09]])
    rng = np.random.default_rng(3)
    lv = rng.integers(0, 16, size=(7, 12), dtype=np.int8)
    p = pack_levels4(lv)
    np.testing.assert_array_equal(p & 15, lv[:, 0::2])
    np.testing.assert_array_equal(p >> 4, lv[:, 1::2])
