"""Host-only checks of the C ABI: the library builds, loads without a GPU,
exports every symbol the header declares, and its pure-host helpers agree
with the oracle.  No kernel is launched here."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbf():
    from paper_0812_1282_gb300 import _build

    _build.build()
    import paper_0812_1282_gb300 as m

    return m


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "lbfe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_header_and_binding_agree(lbf):
    assert sorted(lbf.EXPORTS) == _declared_functions()


def test_library_exports_every_declared_symbol(lbf):
    L = ctypes.CDLL(lbf.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(L, name), name


def test_error_strings(lbf):
    L = lbf.lib()
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert L.lb_error_string(code).decode()
    assert L.lb_error_string(-99).decode() == "unknown error"


def test_device_bytes_layout(lbf):
    b32 = lbf.lb_device_bytes(lbf.LB_FP32, [100], [50])
    b64 = lbf.lb_device_bytes(lbf.LB_FP64, [100], [50])
    # two ping-pong buffers of 18 planes, pitch rounded to 128 bytes
    assert b32 >= 2 * 18 * 128 * 50 * 4
    assert b64 >= 2 * 18 * 112 * 50 * 8
    assert lbf.lb_device_bytes(lbf.LB_FP32, [2], [50]) == 0       # below 3x3
    assert lbf.lb_device_bytes(lbf.LB_FP32, [20000], [20000]) == 0  # over 2^31 elements
    assert lbf.lb_device_bytes(7, [100], [50]) == 0


@pytest.mark.parametrize("theta", [0.0, 15.0, 30.0, 60.0, 89.0, 90.0, 91.0, 120.0, 150.0, 180.0])
def test_wetting_h_matches_oracle(lbf, theta):
    import oracle

    for a, kappa in ((0.04, 0.04), (0.02, 0.03)):
        assert lbf.lb_wetting_h(theta, a, kappa) == pytest.approx(
            oracle.wetting_h(theta, a, kappa), abs=1e-14)


def test_wetting_h_rejects_out_of_range(lbf):
    assert math.isnan(lbf.lb_wetting_h(-1.0, 0.04, 0.04))
    assert math.isnan(lbf.lb_wetting_h(181.0, 0.04, 0.04))
    assert math.isnan(lbf.lb_wetting_h(60.0, 0.0, 0.04))


def test_no_cpu_fallback_without_device(lbf):
    """On a machine without a CUDA device creating a lattice fails loudly."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(lbf.LBError):
        lbf.Lattice(lbf.params(), 16, 16)
