"""The CUDA kernel's tile stages, compiled for the host with bounds checks on
every global and shared-memory access (libqds_emu.so), against the FP64
oracle: same arithmetic to rounding for every boundary mode, mode count and
tile shape (including ragged tiles).  Runs without a GPU."""
import ctypes

import numpy as np
import pytest

from paper_2609_03550_b300 import build as B
from tests._helpers import group_errors, oracle_run, parity_cases, random_case, stable_dr

_emu = None


def emu():
    global _emu
    if _emu is None:
        L = ctypes.CDLL(B.build_emu())
        dp = ctypes.POINTER(ctypes.c_double)
        L.qds_emu_steps.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint32,
                                    dp, dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int]
        _emu = L
    return _emu


def run_emu(M, buf, nx, nr, dr, m_a, g, flags, src, nsteps, TX, TR, nth=64, fused=True):
    dp = ctypes.POINTER(ctypes.c_double)
    out = np.zeros_like(buf)
    s = [None if a is None else np.ascontiguousarray(a, np.complex128) for a in src]
    P = lambda a: None if a is None else a.ctypes.data_as(dp)
    rc = emu().qds_emu_steps(M, P(buf), P(out), nx, nr, 1.0, dr, m_a, g, flags, *[P(a) for a in s],
                             nsteps, TX, TR, nth, int(fused))
    assert rc == 0
    return out


# fused: 1 = fused tile kernel, 0 = warp-column passes, 2 = one pass per
# stage over 8 x 32 tiles, 3 = the stage passes over flat point ranges,
# 4 = as 3 with one (point, mode) per thread in the mode-independent passes
@pytest.mark.parametrize("M,flags", parity_cases())
@pytest.mark.parametrize("tile,fused", [((8, 32), 1), ((5, 3), 1), ((8, 32), 0), ((3, 4), 0), ((8, 32), 2),
                                        ((3, 4), 2), ((8, 32), 3), ((8, 32), 4)])
def test_emulated_kernel_matches_oracle_fp64(M, flags, tile, fused):
    nx, nr = 21, 11
    dr, m_a, g = stable_dr(M, 0.1), 0.1, 0.3
    buf, src = random_case(M * 100 + flags, M, nx, nr)
    ref = oracle_run(buf, M, nx, nr, dr, flags, 3, g=g, m_a=m_a, src=src)
    got = run_emu(M, buf, nx, nr, dr, m_a, g, flags, src, 3, *tile, nth=tile[0] * tile[1] if fused != 1 else 64,
                  fused=fused)
    for name, e in group_errors(got, ref, M, nx, nr).items():
        assert e < 1e-13, (name, e)


@pytest.mark.parametrize("fused", [0, 3, 4])
@pytest.mark.parametrize("M,flags", [c for c in parity_cases() if c[1] & 2])
def test_warp_passes_span_several_row_tiles(M, flags, fused):
    """nr = 70: P1 warps at rows 0, 31, 62 and P2 warps based at 0, 29, 59
    (outputs from 0, 30, 60), so every seam between warps is crossed; nx = 30
    gives interior (unchecked) and edge tiles; the flat passes (fused = 3)
    cover 256 points per block across column boundaries."""
    nx, nr = 30, 70
    dr, m_a, g = stable_dr(M, 0.1), 0.1, 0.3
    buf, src = random_case(M * 17 + flags, M, nx, nr)
    ref = oracle_run(buf, M, nx, nr, dr, flags, 2, g=g, m_a=m_a, src=src)
    got = run_emu(M, buf, nx, nr, dr, m_a, g, flags, src, 2, 8, 32, nth=256, fused=fused)
    for name, e in group_errors(got, ref, M, nx, nr).items():
        assert e < 1e-13, (name, e)


@pytest.mark.parametrize("fused", [1, 0, 2, 3, 4])
@pytest.mark.parametrize("M", [2, 3])
def test_emulated_kernel_fp32_scaled(M, fused):
    nx, nr = 24, 12
    dr, g = stable_dr(M), 1e-6
    flags = 1 | 2 | 4  # axion, regenerated fields, moving window
    buf, src = random_case(7 + M, M, nx, nr)
    n = M * nx * nr
    buf[6 * n:9 * n] *= g          # physical phi ~ g
    buf[15 * n:] *= g
    buf[9 * n:15 * n] *= g * g     # regenerated fields ~ g^2
    src[3] = None
    ref = oracle_run(buf, M, nx, nr, dr, flags, 4, g=g, src=src)
    got = run_emu(M, buf, nx, nr, dr, 0.0, g, flags | 32, src, 4, 8, 16, nth=128 if fused != 1 else 64, fused=fused)
    for name, e in group_errors(got, ref, M, nx, nr).items():
        assert e < 2e-6, (name, e)
