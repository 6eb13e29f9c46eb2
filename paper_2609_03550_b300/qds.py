"""Python binding of the QDS field-step library (include/qds.h).

Argument marshalling only: every step of the solve runs in the CUDA kernels
of libqds.so.  PyTorch provides the device memory (state, sources, outputs)
and the stream.  There is no CPU path: without the built library or a CUDA
device every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqds.so")

AXION, AREM, MOVING_WINDOW, X_PERIODIC, R_CLOSED, FP32, SCALE_G = 1, 2, 4, 8, 16, 32, 64
STEP_DEFAULT, STEP_FLAT, STEP_MARCH = range(3)
FIELDS = ("Trp", "Trm", "Ttp", "Ttm", "Ex", "Bx", "phi", "Tap", "Tam",
          "Trp1", "Trm1", "Ttp1", "Ttm1", "Ex1", "Bx1")
N_FIELDS = 15


class QDSError(RuntimeError):
    pass


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nr", ctypes.c_int32), ("n_modes", ctypes.c_int32),
                ("modes", ctypes.POINTER(ctypes.c_int32)), ("dx", ctypes.c_double),
                ("dr", ctypes.c_double), ("dt", ctypes.c_double), ("omega0", ctypes.c_double),
                ("m_a", ctypes.c_double), ("g", ctypes.c_double), ("flags", ctypes.c_uint32)]


class _Sources(ctypes.Structure):
    _fields_ = [("jx", ctypes.c_void_p), ("jr", ctypes.c_void_p), ("jth", ctypes.c_void_p),
                ("s_ext", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libqds.so; raises if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise QDSError(f"{LIB_PATH} is not built; run paper_2609_03550_b300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(_Params)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        H = ctypes.c_void_p
        sig = {
            "qds_state_bytes": (sz, [P]),
            "qds_batch_state_bytes": (sz, [i, P]),
            "qds_create": (i, [P, vp, sz, ctypes.POINTER(H)]),
            "qds_batch_create": (i, [i, P, vp, sz, ctypes.POINTER(H)]),
            "qds_set_state": (i, [H, vp, vp]),
            "qds_get_state": (i, [H, vp, vp]),
            "qds_set_state_i": (i, [H, i, vp, vp]),
            "qds_get_state_i": (i, [H, i, vp, vp]),
            "qds_step": (i, [H, ctypes.POINTER(_Sources), i, vp]),
            "qds_set_sources_i": (i, [H, i, ctypes.POINTER(_Sources), ctypes.c_longlong, vp]),
            "qds_set_inflow_i": (i, [H, i, vp, vp, ctypes.c_longlong, vp]),
            "qds_mode_products": (i, [i, i, i, vp, vp, ctypes.POINTER(ctypes.c_double), vp, i, i, vp]),
            "qds_mode_products_theta_points": (i, [i]),
            "qds_bunch_currents": (i, [i, i, i, ctypes.c_ulonglong, ctypes.c_ulonglong, i, ctypes.c_double, vp, vp,
                                       vp, vp, i, vp]),
            "qds_diagnostics": (i, [H, ctypes.POINTER(ctypes.c_double), vp, vp]),
            "qds_diagnostics_i": (i, [H, i, ctypes.POINTER(ctypes.c_double), vp, vp]),
            "qds_num_instances": (i, [H]),
            "qds_diagnostics_all": (i, [H, vp, vp]),
            "qds_set_tile": (i, [H, i, i]),
            "qds_set_step_mode": (i, [H, i]),
            "qds_status": (i, [H, vp]),
            "qds_test_withhold_copy": (i, [H, i, vp]),
            "qds_step_launches": (i, [H]),
            "qds_get_tile": (i, [H, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
            "qds_free": (None, [H]),
            "qds_last_error": (ctypes.c_char_p, []),
            "qds_advance_noalloc": (i, [P, vp, vp, vp, sz, i, vp]),
            "qds_adjoint_work_bytes": (sz, [H, i]),
            "qds_adjoint_work_bytes_w": (sz, [H, i]),
            "qds_adjoint_step_w": (i, [H, i, ctypes.POINTER(_Sources), vp, vp, ctypes.c_ulonglong, vp, vp, vp, sz, vp,
                                       vp]),
            "qds_working_bytes": (sz, [H, i]),
            "qds_steps_taken": (ctypes.c_ulonglong, [H]),
            "qds_save_working": (i, [H, i, vp, sz, vp]),
            "qds_restore_working": (i, [H, vp, sz, ctypes.c_ulonglong, vp]),
            "qds_adjoint_step": (i, [H, i, ctypes.POINTER(_Sources), vp, vp, vp, sz, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise QDSError(f"qds error {rc}: {lib().qds_last_error().decode()}")


@dataclass
class Params:
    """Statement of one solve (Sec. 2): grid, retained modes, axion."""
    nx: int
    nr: int
    n_modes: int
    dr: float
    dx: float = 1.0
    m_a: float = 0.0
    g: float = 0.0
    flags: int = 0
    omega0: float = 1.0

    def c(self) -> _Params:
        return _Params(self.nx, self.nr, self.n_modes, None, self.dx, self.dr, self.dx, self.omega0,
                       self.m_a, self.g, self.flags)

    @property
    def fp32(self):
        return bool(self.flags & FP32)

    def state_elems(self):
        return N_FIELDS * self.n_modes * self.nx * self.nr + self.n_modes * self.nx


def state_bytes(p: Params) -> int:
    return lib().qds_state_bytes(ctypes.byref(p.c()))


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class QDSSolver:
    """One or several independent QDS solves on the current CUDA device."""

    def __init__(self, params, device="cuda"):
        if not torch.cuda.is_available():
            raise QDSError("QDSSolver needs a CUDA device")
        plist = params if isinstance(params, (list, tuple)) else [params]
        self.params = list(plist)
        L = lib()
        arr = (_Params * len(plist))(*[p.c() for p in plist])
        nbytes = L.qds_batch_state_bytes(len(plist), arr)
        if nbytes == 0:
            _check(L.qds_create(ctypes.byref(arr[0]), None, 0, ctypes.byref(ctypes.c_void_p())))
            raise QDSError("invalid parameters")
        self.device = torch.device(device)
        self.state = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.state.data_ptr()
        off = (-base) % 256
        self._state_ptr = base + off
        self._nbytes = nbytes
        self.h = ctypes.c_void_p()
        _check(L.qds_batch_create(len(plist), arr, ctypes.c_void_p(self._state_ptr), nbytes, ctypes.byref(self.h)))
        self._keep = []

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.qds_free(self.h)
            self.h = None

    @property
    def rdtype(self):
        return torch.complex64 if self.params[0].fp32 else torch.complex128

    def set_state(self, canon: torch.Tensor, i: int = 0, stream=None):
        """canon: complex128 device tensor in the canonical layout (physical units)."""
        p = self.params[i]
        assert canon.dtype == torch.complex128 and canon.is_cuda and canon.numel() == p.state_elems()
        canon = canon.contiguous()
        _check(lib().qds_set_state_i(self.h, i, ctypes.c_void_p(canon.data_ptr()), _stream_ptr(stream)))
        self._keep = [canon]

    def get_state(self, i: int = 0, stream=None) -> torch.Tensor:
        p = self.params[i]
        out = torch.empty(p.state_elems(), dtype=torch.complex128, device=self.device)
        _check(lib().qds_get_state_i(self.h, i, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def _src_ptr(self, t):
        if t is None:
            return None
        assert t.is_cuda and t.dtype == self.rdtype and t.is_contiguous()
        return t.data_ptr()

    def step(self, nsteps=1, jx=None, jr=None, jth=None, s_ext=None, stream=None):
        """Advance ``nsteps`` steps.  Sources given here (device tensors
        [M, nx, nr] in the working precision) are used for every step of the
        call; with none given, the sources set by ``set_sources`` stay in
        effect if there are any, else the step runs without sources."""
        given = any(t is not None for t in (jx, jr, jth, s_ext))
        if not given and getattr(self, "_per_instance", False):
            _check(lib().qds_step(self.h, None, int(nsteps), _stream_ptr(stream)))
            return
        self._per_instance = False
        src = _Sources(self._src_ptr(jx), self._src_ptr(jr), self._src_ptr(jth), self._src_ptr(s_ext))
        self._src_keep = (jx, jr, jth, s_ext)
        _check(lib().qds_step(self.h, ctypes.byref(src), int(nsteps), _stream_ptr(stream)))

    def set_sources(self, i=0, jx=None, jr=None, jth=None, s_ext=None, per_step=False, stream=None):
        """Sources of instance ``i`` for the following ``step`` calls made
        without sources.  ``per_step=False``: tensors [M, nx, nr], the same
        every step; ``per_step=True``: tensors [n, M, nx, nr] whose slice k
        drives step k of each later call (calls of at most n steps)."""
        p = self.params[i]
        plane = p.n_modes * p.nx * p.nr
        for t in (jx, jr, jth, s_ext):
            if t is not None:
                assert t.numel() % plane == 0 and (per_step or t.numel() == plane)
        src = _Sources(self._src_ptr(jx), self._src_ptr(jr), self._src_ptr(jth), self._src_ptr(s_ext))
        keep = getattr(self, "_inst_src_keep", {})
        keep[i] = (jx, jr, jth, s_ext)
        self._inst_src_keep = keep
        self._per_instance = True
        _check(lib().qds_set_sources_i(self.h, int(i), ctypes.byref(src), plane if per_step else 0,
                                       _stream_ptr(stream)))

    def set_inflow(self, i=0, tr_plus=None, tth_minus=None, per_step=False, stream=None):
        """Laser injection at x_min of instance ``i`` for the following
        ``step`` calls (qds_set_inflow_i): the inflow T_r^+ and T_theta^- of
        the exterior cell behind x_min, tensors [M, nr] (the same every step)
        or [n, M, nr] (slice k drives step k of each later call, per_step);
        None gives zero inflow (both None: the open boundary)."""
        p = self.params[i]
        plane = p.n_modes * p.nr
        for t in (tr_plus, tth_minus):
            if t is not None:
                assert t.numel() % plane == 0 and (per_step or t.numel() == plane)
        keep = getattr(self, "_inflow_keep", {})
        keep[i] = (tr_plus, tth_minus)
        self._inflow_keep = keep
        _check(lib().qds_set_inflow_i(self.h, int(i), self._src_ptr(tr_plus), self._src_ptr(tth_minus),
                                      plane if per_step else 0, _stream_ptr(stream)))

    def adjoint_step(self, fwd, lam, i: int = 0, jx=None, jth=None, s_ext=None, dLdg=None, stream=None):
        """One transposed step (qds_adjoint_step): ``fwd`` is the canonical
        complex128 state at the start of the step, ``lam`` (complex128, same
        layout) holds the adjoint of the state after the step and is
        overwritten with the adjoint of the state before it; dL/dg of the
        step is added to ``dLdg`` (a float64 device tensor of one element)."""
        p = self.params[i]
        for t in (fwd, lam):
            assert t.dtype == torch.complex128 and t.is_cuda and t.is_contiguous() and t.numel() == p.state_elems()

        def ptr(t):
            if t is None:
                return None
            assert t.is_cuda and t.dtype == self.rdtype and t.is_contiguous()
            return t.data_ptr()
        if dLdg is not None:
            assert dLdg.dtype == torch.float64 and dLdg.is_cuda
        nbytes = lib().qds_adjoint_work_bytes(self.h, i)
        if nbytes == 0:
            _check(1)
        work = getattr(self, "_adj_work", None)
        if work is None or work.numel() < nbytes + 256:
            work = self._adj_work = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        wptr = work.data_ptr() + (-work.data_ptr()) % 256
        src = _Sources(ptr(jx), None, ptr(jth), ptr(s_ext))
        self._adj_keep = (fwd, lam, jx, jth, s_ext, dLdg)
        _check(lib().qds_adjoint_step(self.h, i, ctypes.byref(src), ctypes.c_void_p(fwd.data_ptr()),
                                      ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(wptr), nbytes,
                                      None if dLdg is None else ctypes.c_void_p(dLdg.data_ptr()),
                                      _stream_ptr(stream)))

    # -- working snapshots and the conversion-free transposed step --------
    def steps_taken(self) -> int:
        return int(lib().qds_steps_taken(self.h))

    def working_bytes(self, i: int = 0, em_only=False) -> int:
        nbytes = int(lib().qds_working_bytes(self.h, i))
        if em_only:  # the EM group's six plane sets lead the working state
            p = self.params[i]
            ld = p.nr + (p.nr & 1) if p.fp32 else p.nr
            nbytes = 6 * p.n_modes * p.nx * ld * (8 if p.fp32 else 16)
        return nbytes

    def save_working(self, i: int = 0, out=None, em_only=False, stream=None):
        """Copy of the current state as the kernels hold it (a uint8 device
        tensor of qds_working_bytes; ``em_only``: only the EM group's planes,
        all the transposed step reads), and the step count it belongs to."""
        nbytes = self.working_bytes(i, em_only)
        if out is None:
            out = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        _check(lib().qds_save_working(self.h, i, ctypes.c_void_p(out.data_ptr()), out.numel(), _stream_ptr(stream)))
        return out, self.steps_taken()

    def restore_working(self, snap, step: int, stream=None):
        _check(lib().qds_restore_working(self.h, ctypes.c_void_p(snap.data_ptr()), snap.numel(), int(step),
                                         _stream_ptr(stream)))

    def adjoint_step_w(self, fwd_snap, fwd_step: int, lam_in, lam_out, i: int = 0, jx=None, jth=None, s_ext=None,
                       dLdg=None, fwd_next=None, stream=None):
        """One transposed step without conversions (qds_adjoint_step_w):
        ``fwd_snap`` a working snapshot at the start of the step taken
        ``fwd_step`` steps after the import (``fwd_next``, optional: the one
        at its end, whose E_x, B_x spare their recomputation); ``lam_in`` / ``lam_out`` the
        adjoint after / before the step, canonical layout in the working
        precision (complex64 in FP32), distinct tensors; the regenerated
        planes of ``lam_out`` are left as they are."""
        p = self.params[i]
        for t in (lam_in, lam_out):
            assert t.is_cuda and t.is_contiguous() and t.numel() == p.state_elems()
            assert t.dtype == (torch.complex64 if p.fp32 else torch.complex128)

        def ptr(t):
            if t is None:
                return None
            assert t.is_cuda and t.dtype == self.rdtype and t.is_contiguous()
            return t.data_ptr()
        if dLdg is not None:
            assert dLdg.dtype == torch.float64 and dLdg.is_cuda
        nbytes = lib().qds_adjoint_work_bytes_w(self.h, i)
        if nbytes == 0:
            _check(1)
        work = getattr(self, "_adj_work_w", None)
        if work is None or work.numel() < nbytes + 256:
            work = self._adj_work_w = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        wptr = work.data_ptr() + (-work.data_ptr()) % 256
        src = _Sources(ptr(jx), None, ptr(jth), ptr(s_ext))
        self._adj_keep_w = (fwd_snap, fwd_next, lam_in, lam_out, jx, jth, s_ext, dLdg)
        nxt = None if fwd_next is None else ctypes.c_void_p(fwd_next.data_ptr())
        _check(lib().qds_adjoint_step_w(self.h, i, ctypes.byref(src), ctypes.c_void_p(fwd_snap.data_ptr()), nxt,
                                        int(fwd_step), ctypes.c_void_p(lam_in.data_ptr()),
                                        ctypes.c_void_p(lam_out.data_ptr()), ctypes.c_void_p(wptr), nbytes,
                                        None if dLdg is None else ctypes.c_void_p(dLdg.data_ptr()),
                                        _stream_ptr(stream)))

    def diagnostics(self, i: int = 0, profile=False, stream=None):
        out = (ctypes.c_double * 4)()
        prof = torch.zeros(self.params[i].nx, dtype=torch.float64, device=self.device) if profile else None
        _check(lib().qds_diagnostics_i(self.h, i, out, None if prof is None else ctypes.c_void_p(prof.data_ptr()),
                                       _stream_ptr(stream)))
        d = dict(em0=out[0], axion=out[1], em1=out[2], cross=out[3])
        if profile:
            d["profile"] = prof
        return d

    def diagnostics_all(self, out=None, stream=None):
        """Energies of every instance, [n, 4] float64 device tensor (async)."""
        if out is None:
            out = torch.empty((len(self.params), 4), dtype=torch.float64, device=self.device)
        _check(lib().qds_diagnostics_all(self.h, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def status(self, stream=None) -> int:
        """Device error state (synchronises): 0, or the QDS_ERR_* code of a
        timed-out bulk copy (4) or a non-finite value in the state (3)."""
        return int(lib().qds_status(self.h, _stream_ptr(stream)))

    def test_withhold_copy(self, on: bool, stream=None):
        """Test hook: the x-marching CTAs withhold their first bulk copy, so
        that the bounded wait runs out and qds_status reports a timeout."""
        _check(lib().qds_test_withhold_copy(self.h, int(bool(on)), _stream_ptr(stream)))

    def check(self, stream=None):
        """Raise QDSError if the device error state is set."""
        _check(self.status(stream))

    def autotune(self, steps: int = 4, candidates=None, stream=None):
        """Time the step on this batch for the flat passes and for the
        x-marching kernels over a set of work splits (rows per CTA, columns
        per CTA) and keep the fastest.  The trial steps advance the state:
        call before set_state.  Returns (mode, rows, cols)."""
        if candidates is None:
            candidates = [(STEP_MARCH, 0, c) for c in (64, 128, 256)]
            candidates += [(STEP_MARCH, r, 128) for r in (32, 48)]
            candidates += [(STEP_FLAT, 0, 0)]
        s = stream if stream is not None else torch.cuda.current_stream()
        best, best_t = None, None
        self.timings = {}
        for cand in candidates:
            mode, rows, cols = cand
            try:
                self.set_tile(rows, cols)
            except QDSError:
                continue
            self.set_step_mode(mode)
            self.step(2, stream=s)  # first launches of this configuration
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            self.step(steps, stream=s)
            e1.record(s)
            e1.synchronize()
            t = e0.elapsed_time(e1) / steps
            self.timings[cand] = t
            if best_t is None or t < best_t:
                best, best_t = cand, t
        mode, rows, cols = best
        self.set_tile(rows, cols)
        self.set_step_mode(mode)
        return best

    def step_mode_name(self) -> str:
        names = {STEP_DEFAULT: "stage passes over flat point ranges (default)", STEP_FLAT: "stage passes over flat point ranges",
                 STEP_MARCH: "x-marching kernels"}
        return names[getattr(self, "_mode", STEP_DEFAULT)]

    def step_launches(self) -> int:
        """Kernel launches of one step in the current step mode."""
        return int(lib().qds_step_launches(self.h))

    def set_step_mode(self, mode: int):
        """STEP_DEFAULT, STEP_FLAT or STEP_MARCH."""
        _check(lib().qds_set_step_mode(self.h, int(mode)))
        self._mode = int(mode)

    def set_tile(self, rows, cols):
        """Work split of the x-marching kernels: radial rows per CTA (with the
        halo; 0 = default) and window columns per CTA (0 = default)."""
        _check(lib().qds_set_tile(self.h, int(rows), int(cols)))

    def tile(self):
        a, b, c, d = (ctypes.c_int() for _ in range(4))
        _check(lib().qds_get_tile(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
        return dict(rows=a.value, cols=b.value, ctas=c.value, smem=d.value)


MODES_DIRECT, MODES_THETA = 0, 1


def bunch_currents(seed: int, step: int, amp: float, bunch, jx, jr, jth, stream=None):
    """Synthetic currents (qds_bunch_currents) written into the device
    tensors jx, jr, jth: [M, nx, nr] for step ``step``, or [count, M, nx, nr]
    for the steps step .. step + count - 1 (complex64 or complex128): uniform
    noise of amplitude amp, m = 0 real, plus the float64 bunch [nx, nr] (or
    None) on j_x of m = 0."""
    M, nx, nr = jx.shape[-3:]
    count = jx.shape[0] if jx.dim() == 4 else 1
    fp32 = jx.dtype == torch.complex64
    for t in (jx, jr, jth):
        assert t.is_cuda and t.is_contiguous() and t.dtype == jx.dtype and t.shape == jx.shape
    if bunch is not None:
        assert bunch.is_cuda and bunch.dtype == torch.float64 and bunch.is_contiguous() and bunch.numel() == nx * nr
    _check(lib().qds_bunch_currents(int(M), int(nx), int(nr), int(seed), int(step), int(count), float(amp),
                                    None if bunch is None else ctypes.c_void_p(bunch.data_ptr()),
                                    ctypes.c_void_p(jx.data_ptr()), ctypes.c_void_p(jr.data_ptr()),
                                    ctypes.c_void_p(jth.data_ptr()), int(fp32), _stream_ptr(stream)))


def mode_products(A, B, w, method=MODES_DIRECT, out=None, stream=None):
    """sum_p w[p] C_m{A[p], B[p]} at every point (qds_mode_products): A, B
    complex64 or complex128 CUDA tensors [npairs, M, npts], w a sequence of
    npairs floats; returns [M, npts] (or fills ``out``).  method
    MODES_DIRECT: the convolution sums; MODES_THETA: the theta-grid
    procedure with FFTs (Sec. 3.3)."""
    assert A.shape == B.shape and A.dim() == 3 and A.dtype == B.dtype and A.is_cuda
    assert A.dtype in (torch.complex64, torch.complex128) and A.is_contiguous() and B.is_contiguous()
    npairs, M, npts = A.shape
    if out is None:
        out = torch.empty((M, npts), dtype=A.dtype, device=A.device)
    wa = (ctypes.c_double * npairs)(*[float(x) for x in w])
    _check(lib().qds_mode_products(M, npts, npairs, A.data_ptr(), B.data_ptr(), wa, out.data_ptr(), int(method),
                                   1 if A.dtype == torch.complex64 else 0, _stream_ptr(stream)))
    return out
