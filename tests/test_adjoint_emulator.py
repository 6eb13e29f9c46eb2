"""The transposed step (qds_adjoint.cuh), run by the host emulator, against
the FP64 oracle's linearisation.  The step is at most quadratic in the state
(the axion source is bilinear in the EM fields), so the oracle's central
difference [F(s + d) - F(s - d)] / 2 is exactly the Jacobian action J d, and
the adjoint must satisfy <lambda, J d> = <J^T lambda, d> to rounding.
d L / d g of L = <lambda, F(s)> is checked the same way (the step is linear
in g).  Runs without a GPU."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2609_03550_b300 import build as B
from paper_2609_03550_b300 import inputs as I
from tests._helpers import stable_dr

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(B.build_emu())
        dp = ctypes.POINTER(ctypes.c_double)
        L.qds_emu_adjoint.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint32,
                                      dp, dp, dp]
        _lib = L
    return _lib


def P(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def emu_adjoint(M, fwd, lam_new, nx, nr, dr, m_a, g, flags, jx=None, jt=None):
    out = np.zeros_like(fwd)
    dg = np.zeros(1)
    rc = lib().qds_emu_adjoint(M, P(fwd), P(lam_new), P(out), nx, nr, 1.0, dr, m_a, g, flags, P(jx), P(jt), P(dg))
    assert rc == 0
    return out, dg[0]


def em_axion_mask(M, nx, nr):
    """True on the EM and axion components (and phi_prev), False on the
    regenerated group, whose adjoint is zero for these functionals."""
    n = M * nx * nr
    m = np.zeros(15 * n + M * nx, bool)
    m[:9 * n] = True
    m[15 * n:] = True
    return m


def rdot(a, b):
    return float(np.sum(a.real * b.real + a.imag * b.imag))


def oracle_step(buf, M, nx, nr, dr, m_a, g, flags, jx=None, jr=None, jt=None):
    st = oracle.State(M, nx, nr, buf)
    oracle.step(dict(nx=nx, nr=nr, M=M, h=1.0, dr=dr, m_a=m_a, g=g, flags=flags), st, jx, jr, jt)
    return st.buf


@pytest.mark.parametrize("M", [1, 2, 3, 4])
@pytest.mark.parametrize("mw", [False, True])
def test_adjoint_step_dot_product(M, mw):
    nx, nr = 23, 9
    m_a, g = 0.15, 0.7
    dr = stable_dr(M, m_a)
    flags = oracle.AXION | (oracle.MOVING_WINDOW if mw else 0)
    rng = np.random.default_rng(100 + M + 10 * mw)
    mask = em_axion_mask(M, nx, nr)
    s = I.random_state(rng, M, nx, nr)
    jx, jr, jt = I.random_sources(rng, M, nx, nr, 0.3)
    for trial in range(3):
        d = I.random_state(rng, M, nx, nr) * mask
        lam = I.random_state(rng, M, nx, nr, axis_consistent=False) * mask
        Jd = 0.5 * (oracle_step(s + d, M, nx, nr, dr, m_a, g, flags, jx, jr, jt) -
                    oracle_step(s - d, M, nx, nr, dr, m_a, g, flags, jx, jr, jt))
        lt, _ = emu_adjoint(M, s, lam, nx, nr, dr, m_a, g, flags, jx, jt)
        lhs, rhs = rdot(lam * mask, Jd * mask), rdot(lt, d)
        scale = np.linalg.norm(lam) * np.linalg.norm(Jd)
        assert abs(lhs - rhs) < 1e-12 * scale, (trial, lhs, rhs)
        assert np.all(lt[~mask] == 0)


@pytest.mark.parametrize("M", [2, 3])
def test_adjoint_coupling_derivative(M):
    nx, nr = 21, 8
    dr = stable_dr(M)
    flags = oracle.AXION | oracle.MOVING_WINDOW
    rng = np.random.default_rng(7 + M)
    mask = em_axion_mask(M, nx, nr)
    s = I.random_state(rng, M, nx, nr)
    lam = I.random_state(rng, M, nx, nr, axis_consistent=False) * mask
    g, dgs = 0.4, 0.1
    Fp = oracle_step(s, M, nx, nr, dr, 0.0, g + dgs, flags)
    Fm = oracle_step(s, M, nx, nr, dr, 0.0, g - dgs, flags)
    fd = rdot(lam * mask, (Fp - Fm) * mask) / (2 * dgs)
    _, dg = emu_adjoint(M, s, lam, nx, nr, dr, 0.0, g, flags)
    assert abs(dg - fd) < 1e-10 * (abs(fd) + 1e-300) + 1e-12, (dg, fd)


@pytest.mark.parametrize("M,mw", [(1, False), (2, True), (3, False)])
def test_adjoint_step_elementwise_vs_oracle_columns(M, mw):
    """Every entry of J^T lambda against the oracle's Jacobian columns
    (tiny grid; includes the on-axis entries the regularity rules fix)."""
    from tests._helpers import oracle_vjp
    nx, nr = 9, 5
    m_a, g = 0.1, 0.8
    dr = stable_dr(M, m_a)
    flags = oracle.AXION | (oracle.MOVING_WINDOW if mw else 0)
    rng = np.random.default_rng(40 + M)
    s = I.random_state(rng, M, nx, nr)
    jx, jr, jt = I.random_sources(rng, M, nx, nr, 0.3)
    lam = I.random_state(rng, M, nx, nr, axis_consistent=False) * em_axion_mask(M, nx, nr)
    ref = oracle_vjp(s, lam, M, nx, nr, dr, flags, g=g, m_a=m_a, src=(jx, jr, jt, None))
    got, _ = emu_adjoint(M, s, lam, nx, nr, dr, m_a, g, flags, jx, jt)
    err = np.abs(got - ref)
    tol = 1e-12 * np.abs(ref).max()
    bad = np.argwhere(err > tol)
    assert bad.size == 0, (bad[:10].ravel(), got[bad[:5].ravel()], ref[bad[:5].ravel()])
