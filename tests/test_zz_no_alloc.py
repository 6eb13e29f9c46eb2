"""qds_advance_noalloc: the field step for callers that cannot allocate device
memory (runtimes or memory pools that forbid allocation after start-up,
plug-ins that must not grow a host application's device footprint,
real-time loops where an allocation may stall or fail).

The entry point keeps its descriptor, counters and scratch planes in a static
device array; the test allocates the caller-side buffers (input, output,
working state) with torch, as such a caller would have them already.  Its
result after each of two calls in a row must equal the regular path's
(qds_create / qds_set_state / qds_step / qds_get_state).
"""
import ctypes

import numpy as np
import pytest

from paper_2609_03550_b300 import build as B
from paper_2609_03550_b300 import inputs as I
from paper_2609_03550_b300 import qds as Q
from tests._helpers import group_errors

STEPS = 12


@pytest.fixture(scope="module")
def lib():
    B.build_cuda()
    return Q.lib()


def _workload():
    wl = I.two_colour(nx=200, nr=40)
    wl.M = 3
    for L in wl.lasers:
        L.w0, L.x0, L.fwhm = 60.0, 140.0, 30.0
    return wl


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, Q.FP32])
def test_noalloc_matches_regular_path_on_two_calls(lib, prec):
    torch = pytest.importorskip("torch")
    dev = "cuda:0"
    wl = _workload()
    g = 1e-3
    p = Q.Params(wl.nx, wl.nr, wl.M, wl.dr, g=g, flags=Q.AXION | Q.AREM | Q.MOVING_WINDOW | prec)
    buf = wl.initial_state()

    s = Q.QDSSolver(p, device=dev)
    s.set_state(torch.from_numpy(buf).to(dev))
    s.step(STEPS)
    ref1 = s.get_state().cpu().numpy()
    s.step(STEPS)
    ref2 = s.get_state().cpu().numpy()

    nbytes = Q.state_bytes(p)
    work = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    wptr = work.data_ptr() + (-work.data_ptr()) % 256
    x_in = torch.from_numpy(buf).to(dev)
    out1 = torch.empty_like(x_in)
    out2 = torch.empty_like(x_in)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    pc = p.c()
    rc = lib.qds_advance_noalloc(ctypes.byref(pc), ctypes.c_void_p(x_in.data_ptr()), ctypes.c_void_p(out1.data_ptr()),
                                 ctypes.c_void_p(wptr), nbytes, STEPS, stream)
    assert rc == 0, lib.qds_last_error().decode()
    rc = lib.qds_advance_noalloc(ctypes.byref(pc), ctypes.c_void_p(out1.data_ptr()), ctypes.c_void_p(out2.data_ptr()),
                                 ctypes.c_void_p(wptr), nbytes, STEPS, stream)
    assert rc == 0, lib.qds_last_error().decode()
    torch.cuda.synchronize()
    got1, got2 = out1.cpu().numpy(), out2.cpu().numpy()
    if prec == 0:
        tol = {"em": 1e-12, "axion": 1e-12, "arem": 1e-12}
    else:
        tol = {"em": 1e-5, "axion": 1e-4, "arem": 1e-4}
    for got, ref in ((got1, ref1), (got2, ref2)):
        e = group_errors(got, ref, wl.M, wl.nx, wl.nr)
        assert all(e[k] <= tol[k] for k in e), e
    assert np.abs(got2 - got1).max() > 0  # the second call advanced the state


def test_noalloc_rejects_grids_beyond_its_scratch(lib):
    """4 scratch planes of 4 x 8192 x 256 complex128 exceed the static array;
    the size check runs before any device call."""
    p = Q.Params(8192, 256, 4, 5.0, g=1e-3, flags=Q.AXION | Q.AREM)
    pc = p.c()
    big = 1 << 40
    rc = lib.qds_advance_noalloc(ctypes.byref(pc), ctypes.c_void_p(256), ctypes.c_void_p(256),
                                 ctypes.c_void_p(256), big, 1, None)
    assert rc == 1  # QDS_ERR_INVALID_ARG
    assert "too large" in lib.qds_last_error().decode()
