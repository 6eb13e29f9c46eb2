"""The CUDA step kernels' code, compiled for the host with bounds checks on
the shared-memory and global accesses (libqds_emu.so), against the oracle:
same arithmetic to rounding for every boundary mode and mode count, for the
flat stage passes and for the x-marching kernels (bands of rows with radial
halos, ragged segments of columns, the bulk copies' zero fill emulated).
Runs without a GPU."""
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


FLAT, MARCH = 0, 1


def run_emu(M, buf, nx, nr, dr, m_a, g, flags, src, nsteps, mode=MARCH, rows=(24, 16), seg=7):
    dp = ctypes.POINTER(ctypes.c_double)
    out = np.zeros_like(buf)
    s = [None if a is None else np.ascontiguousarray(a, np.complex128) for a in src]
    P = lambda a: None if a is None else a.ctypes.data_as(dp)
    rc = emu().qds_emu_steps(M, P(buf), P(out), nx, nr, 1.0, dr, m_a, g, flags, *[P(a) for a in s],
                             nsteps, rows[0], rows[1], seg, mode)
    assert rc == 0
    return out


@pytest.mark.parametrize("M,flags", parity_cases())
@pytest.mark.parametrize("mode,rows,seg", [(FLAT, (24, 16), 7), (MARCH, (24, 16), 7),
                                           (MARCH, (64, 64), 128)])
def test_emulated_kernels_match_oracle_fp64(M, flags, mode, rows, seg):
    """nr = 11: one band per kernel; nx = 21 with 7-column segments gives
    three CTAs along x, the first and last at the open (or periodic) ends."""
    nx, nr = 21, 11
    dr, m_a, g = stable_dr(M, 0.1), 0.1, 0.3
    buf, src = random_case(M * 100 + flags, M, nx, nr)
    ref = oracle_run(buf, M, nx, nr, dr, flags, 3, g=g, m_a=m_a, src=src)
    got = run_emu(M, buf, nx, nr, dr, m_a, g, flags, src, 3, mode=mode, rows=rows, seg=seg)
    for name, e in group_errors(got, ref, M, nx, nr).items():
        assert e < 1e-13, (name, e)


@pytest.mark.parametrize("M,flags", [c for c in parity_cases() if c[1] & 2])
@pytest.mark.parametrize("rows,seg", [((24, 16), 5), ((32, 24), 9), ((24, 24), 30), ((8, 8), 4), ((16, 8), 1)])
def test_march_bands_and_segments(M, flags, rows, seg):
    """nr = 45 odd (padded row stride in FP32), several bands per kernel
    (first kernel with 24 ring rows: owned rows [0, 21), [21, 39), [39, 45),
    each later band's ring starting 3-4 rows below it at an even row; the
    smallest rings, 8 rows, give bands of one or two rows), segments of
    1, 4, 5, 9 and 30 columns over nx = 30 (a ragged last segment, one CTA
    for the whole x)."""
    nx, nr = 30, 45
    dr, m_a, g = stable_dr(M, 0.1), 0.1, 0.3
    buf, src = random_case(M * 17 + flags, M, nx, nr)
    ref = oracle_run(buf, M, nx, nr, dr, flags, 2, g=g, m_a=m_a, src=src)
    got = run_emu(M, buf, nx, nr, dr, m_a, g, flags, src, 2, rows=rows, seg=seg)
    for name, e in group_errors(got, ref, M, nx, nr).items():
        assert e < 1e-13, (name, e)


@pytest.mark.parametrize("mode", [FLAT, MARCH])
@pytest.mark.parametrize("M", [2, 3])
@pytest.mark.parametrize("nr", [12, 13])
def test_emulated_kernels_fp32_scaled(M, mode, nr):
    nx = 24
    dr, g = stable_dr(M), 1e-6
    flags = 1 | 2 | 4  # axion, regenerated fields, moving window
    buf, src = random_case(7 + M, M, nx, nr)
    n = M * nx * nr
    buf[6 * n:9 * n] *= g          # physical phi ~ g
    buf[15 * n:] *= g
    buf[9 * n:15 * n] *= g * g     # regenerated fields ~ g^2
    src[3] = None
    ref = oracle_run(buf, M, nx, nr, dr, flags, 4, g=g, src=src)
    got = run_emu(M, buf, nx, nr, dr, 0.0, g, flags | 32, src, 4, mode=mode, rows=(24, 16), seg=6)
    for name, e in group_errors(got, ref, M, nx, nr).items():
        assert e < 2e-6, (name, e)


def run_emu_inflow(M, buf, nx, nr, dr, m_a, g, flags, src, inflow, nsteps, mode=MARCH, rows=(24, 16), seg=7):
    L = emu()
    dp = ctypes.POINTER(ctypes.c_double)
    if not hasattr(L, "_inflow_set"):
        L.qds_emu_steps_inflow.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint32,
                                           dp, dp, dp, dp, dp, dp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L._inflow_set = True
    out = np.zeros_like(buf)
    s = [None if a is None else np.ascontiguousarray(a, np.complex128) for a in src]
    ins = [np.ascontiguousarray(a, np.complex128) for a in inflow]
    P = lambda a: None if a is None else a.ctypes.data_as(dp)
    rc = L.qds_emu_steps_inflow(M, P(buf), P(out), nx, nr, 1.0, dr, m_a, g, flags, *[P(a) for a in s],
                                P(ins[0]), P(ins[1]), M * nr, nsteps, rows[0], rows[1], seg, mode)
    assert rc == 0
    return out


@pytest.mark.parametrize("M", [1, 2, 3, 4])
@pytest.mark.parametrize("flags", [0, 1 | 2, 1 | 2 | 4, 1 | 2 | 16])
@pytest.mark.parametrize("mode,rows,seg", [(FLAT, (24, 16), 7), (MARCH, (16, 8), 5), (MARCH, (64, 64), 64)])
def test_injection_at_xmin_matches_oracle(M, flags, mode, rows, seg):
    """Laser injection at x_min (a different inflow T_r^+, T_th^- every step)
    on random states with sources: the flat passes and the x-marching
    kernels (several bands, ragged segments) against the oracle."""
    nx, nr, N = 23, 19, 4
    dr, m_a, g = stable_dr(M, 0.1), 0.1, 0.3
    buf, src = random_case(M * 7 + flags + 3, M, nx, nr)
    rng = np.random.default_rng(M + 100 * flags)
    inflow = [rng.standard_normal((N, M, nr)) + 1j * rng.standard_normal((N, M, nr)) for _ in range(2)]
    ref = oracle_run_inflow(buf, M, nx, nr, dr, flags, N, g, m_a, src, inflow)
    got = run_emu_inflow(M, buf, nx, nr, dr, m_a, g, flags, src, inflow, N, mode=mode, rows=rows, seg=seg)
    for name, e in group_errors(got, ref, M, nx, nr).items():
        assert e < 1e-13, (name, e)


def oracle_run_inflow(buf, M, nx, nr, dr, flags, nsteps, g, m_a, src, inflow):
    import oracle
    st = oracle.State(M, nx, nr, buf)
    oracle.step(dict(nx=nx, nr=nr, M=M, h=1.0, dr=dr, g=g, m_a=m_a, flags=flags & 31), st, *src,
                nsteps=nsteps, extended=True, inflow=inflow)
    return st.buf
