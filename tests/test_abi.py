"""The C-ABI library builds, loads and exports every symbol include/bs.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bs.h")


@pytest.fixture(scope="module")
def lib():
    from paper_0712_1695_gb300 import build, load

    build()
    return load()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^BS_API\s+[\w\s\*]+?\b(bs_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("bs_create", "bs_velocity", "bs_destroy", "bs_update", "bs_last_error", "bs_batch_create",
                     "bs_batch_velocity", "bs_autotune"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_0712_1695_gb300.binding import EXPORTED

    names = declared_symbols()
    assert sorted(EXPORTED) == names
    for n in names:
        assert hasattr(lib, n), n


def test_params_struct_layout():
    from paper_0712_1695_gb300.binding import bs_params

    # double far_ratio; int order, n_theta, n_phi, precision; int32_t *counts; int near_rule
    assert ctypes.sizeof(bs_params) == 40
    assert bs_params.counts.offset == 24
    assert bs_params.near_rule.offset == 32


def test_argument_errors_without_gpu(lib):
    """Calls rejected by argument checks touch no device and report an error."""
    from paper_0712_1695_gb300 import binding

    h = ctypes.c_void_p()
    rc = lib.bs_create(None, 0, None, 0, None, ctypes.byref(h))
    assert rc == binding.BS_ERR_ARG and b"NULL" in lib.bs_last_error()
    assert lib.bs_destroy(None) == binding.BS_ERR_ARG
    assert lib.bs_tet_rule(5, None, None) == binding.BS_ERR_ORDER
    assert lib.bs_direction_table(0, 4, None, None) == binding.BS_ERR_ARG
    assert lib.bs_set_wait_limits(None, 0, 0, 0) == binding.BS_ERR_ARG
