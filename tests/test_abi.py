"""The C-ABI library loads without a GPU, exports every entry point that
include/qds.h declares, and validates the statement of a solve (host-side
checks only; no compute call)."""
import ctypes
import os
import re

import pytest

from paper_2609_03550_b300 import build as B
from paper_2609_03550_b300 import qds as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(qds_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build_cuda()
    return ctypes.CDLL(B.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def _bytes(**kw):
    base = dict(nx=64, nr=16, n_modes=2, dr=2.0)
    base.update(kw)
    return Q.state_bytes(Q.Params(**base))


def test_state_bytes_of_valid_statements():
    up = lambda x: (x + 255) // 256 * 256
    for nr in (16, 17):
        for flags, eb in ((0, 16), (Q.FP32, 8)):
            # two ping-pong state copies (15 planes + phi_prev) and four scratch
            # planes; in FP32 the row stride is nr rounded up to even
            ld = nr + (nr & 1) if flags & Q.FP32 else nr
            plane = 2 * 64 * ld
            assert _bytes(nr=nr, flags=flags) == 2 * up((15 * plane + 2 * 64) * eb) + up(4 * plane * eb)


@pytest.mark.parametrize("bad", [
    dict(dx=1.0, dr=1.2),                 # below the m <= 1 bound
    dict(n_modes=3, dr=2.0),              # m = 2 needs dr >= 2.25
    dict(n_modes=4, dr=3.0),              # m = 3 needs dr >= 3.25
    dict(n_modes=2, dr=2.0, m_a=0.5),     # mass widens the bound
    dict(n_modes=5, dr=9.0),              # at most 4 modes
    dict(nr=3),
    dict(flags=Q.MOVING_WINDOW | Q.X_PERIODIC),
    dict(flags=Q.AREM),                   # needs the axion
    dict(flags=1 << 12),
    dict(nx=7),                           # below the smallest window
    dict(nx=65536, nr=1024, n_modes=4, dr=3.25),  # 2^31 state elements or more per instance
    dict(dx=1.0, dr=2.0, m_a=1.5),        # dx m_a > 1
])
def test_invalid_or_unstable_statements_are_rejected(bad):
    assert _bytes(**bad) == 0


def test_largest_instance_below_the_element_limit_is_accepted():
    """15 M nx ld + M nx < 2^31 (ld = nr, rounded up to even in FP32): with 4
    modes and nx = 4096, nr = 8738 is the largest grid that fits and 8739
    the smallest that does not (in FP32 too, whose stride of 8739 is 8740)."""
    assert _bytes(nx=4096, nr=8738, n_modes=4, dr=3.25) > 0
    assert _bytes(nx=4096, nr=8739, n_modes=4, dr=3.25) == 0
    assert _bytes(nx=4096, nr=8738, n_modes=4, dr=3.25, flags=Q.FP32) > 0
    assert _bytes(nx=4096, nr=8737, n_modes=4, dr=3.25, flags=Q.FP32) > 0
    assert _bytes(nx=4096, nr=8739, n_modes=4, dr=3.25, flags=Q.FP32) == 0


def test_stability_rule_matches_limits():
    assert _bytes(n_modes=3, dr=2.25) > 0
    assert _bytes(n_modes=4, dr=3.25) > 0
    assert _bytes(n_modes=2, dr=3.0, m_a=0.5) > 0
