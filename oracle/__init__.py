"""FP64 CPU oracle of the QDS Maxwell + axion field step.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg are the only callers.  The product path never imports this
package.  The arithmetic lives in ``qds_oracle.c`` (plain C loops written from
the paper's equations); this module only marshals numpy arrays.

State layout (complex128): ``fields[15, M, nx, nr]`` in the order
``Trp Trm Ttp Ttm Ex Bx phi Tap Tam Trp1 Trm1 Ttp1 Ttm1 Ex1 Bx1`` and
``phi_prev[M, nx]`` (phi on the outermost half row at time n-1).
"""
import ctypes
import os

import numpy as np

from . import build as _build

AXION, AREM, MOVING_WINDOW, X_PERIODIC, R_CLOSED = 1, 2, 4, 8, 16
# test reading only: the outer phi row by the paper's printed three-level update
AXION_R_PRINTED = 1024
FIELDS = ("Trp", "Trm", "Ttp", "Ttm", "Ex", "Bx", "phi", "Tap", "Tam",
          "Trp1", "Trm1", "Ttp1", "Ttm1", "Ex1", "Bx1")
N_FIELDS = len(FIELDS)

_libs = {}


def lib(extended=False):
    """The FP64 build, or the long double build (``extended``) that serves
    as the parity reference where the paper's E.B form cancels."""
    if extended not in _libs:
        path = _build.build(extended=extended)
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.ora_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               dp, dp, dp, dp, dp]
        L.ora_step.restype = ctypes.c_int
        L.ora_step_n.argtypes = L.ora_step.argtypes + [ctypes.c_int]
        L.ora_step_n.restype = ctypes.c_int
        L.ora_step_inflow.argtypes = L.ora_step.argtypes + [dp, dp, ctypes.c_longlong, ctypes.c_int]
        L.ora_step_inflow.restype = ctypes.c_int
        L.ora_diagnostics.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, dp, dp, dp]
        L.ora_diagnostics.restype = ctypes.c_int
        L.ora_mode_conv.argtypes = [ctypes.c_int, dp, dp, dp]
        L.ora_mode_conv.restype = None
        L.ora_mode_products.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        L.ora_mode_products.restype = ctypes.c_int
        L.ora_mode_products_theta.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                              dp, dp]
        L.ora_mode_products_theta.restype = ctypes.c_int
        L.ora_set_threads.argtypes = [ctypes.c_int]
        L.ora_set_threads.restype = ctypes.c_int
        _libs[extended] = L
    return _libs[extended]


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.complex128 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class State:
    """Oracle state: contiguous complex128 buffer viewed as fields + phi_prev."""

    def __init__(self, M, nx, nr, buf=None):
        self.M, self.nx, self.nr = M, nx, nr
        n = N_FIELDS * M * nx * nr + M * nx
        self.buf = np.zeros(n, np.complex128) if buf is None else np.ascontiguousarray(buf, np.complex128).copy()
        assert self.buf.size == n

    @property
    def fields(self):
        return self.buf[: N_FIELDS * self.M * self.nx * self.nr].reshape(N_FIELDS, self.M, self.nx, self.nr)

    @property
    def phi_prev(self):
        return self.buf[N_FIELDS * self.M * self.nx * self.nr:].reshape(self.M, self.nx)

    def __getitem__(self, name):
        return self.fields[FIELDS.index(name)]

    def copy(self):
        return State(self.M, self.nx, self.nr, self.buf)


def step(p, st, jx=None, jr=None, jt=None, s_ext=None, nsteps=1, extended=False, inflow=None):
    """Advance ``st`` in place by ``nsteps`` steps with constant sources.

    ``p``: dict with nx, nr, M, h, dr, m_a, g, flags.  Sources are complex128
    arrays [M, nx, nr] at the native staggered positions (or None).
    ``inflow``: laser injection at x_min, a pair (T_r^+, T_th^-) of the
    exterior cell behind x_min, each [M, nr] (the same every step) or
    [nsteps, M, nr] (step by step); None keeps the open boundary.  With
    ``extended`` the steps run in long double (state rounded to complex128
    only on return)."""
    L = lib(extended)
    srcs = [None if a is None else np.ascontiguousarray(a, np.complex128) for a in (jx, jr, jt, s_ext)]
    ins, istride = [None, None], 0
    if inflow is not None:
        ins = [np.ascontiguousarray(a, np.complex128) for a in inflow]
        shape = (p["M"], p["nr"])
        assert ins[0].shape == ins[1].shape and ins[0].shape in (shape, (nsteps,) + shape)
        istride = 0 if ins[0].ndim == 2 else p["M"] * p["nr"]
    rc = L.ora_step_inflow(p["nx"], p["nr"], p["M"], p["h"], p["dr"], p.get("m_a", 0.0), p.get("g", 0.0),
                           p.get("flags", 0), _ptr(st.buf), *[_ptr(a) for a in srcs], _ptr(ins[0]),
                           _ptr(ins[1]), istride, int(nsteps))
    if rc != 0:
        raise RuntimeError(f"ora_step failed: {rc}")
    return st


def diagnostics(p, st, profile=False):
    """Energies: dict(em0, axion, em1, cross[, profile])."""
    L = lib()
    out = np.zeros(4)
    prof = np.zeros(p["nx"]) if profile else None
    L.ora_diagnostics(p["nx"], p["nr"], p["M"], p["h"], p["dr"], p.get("m_a", 0.0), p.get("g", 0.0),
                      p.get("flags", 0), _ptr(st.buf),
                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      None if prof is None else prof.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    d = dict(em0=out[0], axion=out[1], em1=out[2], cross=out[3])
    if profile:
        d["profile"] = prof
    return d


def mode_conv(A, B):
    """C_m{A, B} for m = 0..M-1 (Eq. mode_convolution); A, B complex [M]."""
    A = np.ascontiguousarray(A, np.complex128)
    B = np.ascontiguousarray(B, np.complex128)
    out = np.zeros(A.size, np.complex128)
    lib().ora_mode_conv(A.size, _ptr(A), _ptr(B), _ptr(out))
    return out


def mode_products(A, B, w, ntheta=None):
    """sum_p w[p] C_m{A[p], B[p]} at every point (Sec. 3.3): A, B complex
    [npairs, M, npts], w [npairs]; returns [M, npts].  ntheta None: the
    convolution sums (Eq. mode_convolution); else the theta-grid procedure
    with ntheta angles (plain DFT sums)."""
    A = np.ascontiguousarray(A, np.complex128)
    B = np.ascontiguousarray(B, np.complex128)
    w = np.ascontiguousarray(w, np.float64)
    npairs, M, npts = A.shape
    out = np.zeros((M, npts), np.complex128)
    wp = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if ntheta is None:
        rc = lib().ora_mode_products(M, npairs, npts, _ptr(A), _ptr(B), wp, _ptr(out))
    else:
        rc = lib().ora_mode_products_theta(M, npairs, npts, int(ntheta), _ptr(A), _ptr(B), wp, _ptr(out))
    if rc != 0:
        raise RuntimeError(f"mode products failed: {rc}")
    return out


def set_threads(n):
    """Threads of the oracle's OpenMP loops (n <= 0: the default); returns
    the count in force."""
    return int(lib().ora_set_threads(int(n)))
