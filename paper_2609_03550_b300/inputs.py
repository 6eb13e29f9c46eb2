"""Seeded synthetic inputs for the QDS field step.

This module holds workload recipes only: initial laser fields, prescribed
currents and the parameter draws of the batched scan.  It contains none of the
step arithmetic and imports neither the CUDA binding nor the oracle, so both
may consume what it produces.

Units are normalised (c = eps0 = mu0 = hbar = 1, h = dx = c dt = 1).  Field
amplitudes follow a0 = E_peak / omega (so E_peak = a0 * omega), Sec. 4.1.

State layout (canonical, shared by every consumer): complex planes
``fields[15, M, nx, nr]`` in the order
``Trp Trm Ttp Ttm Ex Bx phi Tap Tam Trp1 Trm1 Ttp1 Ttm1 Ex1 Bx1`` followed by
``phi_prev[M, nx]``.  Positions: T_r at (i, (j+1/2) dr), T_theta at (i, j dr).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FIELDS = ("Trp", "Trm", "Ttp", "Ttm", "Ex", "Bx", "phi", "Tap", "Tam",
          "Trp1", "Trm1", "Ttp1", "Ttm1", "Ex1", "Bx1")
N_FIELDS = len(FIELDS)


def state_size(M: int, nx: int, nr: int) -> int:
    return N_FIELDS * M * nx * nr + M * nx


def empty_state(M: int, nx: int, nr: int) -> np.ndarray:
    return np.zeros(state_size(M, nx, nr), np.complex128)


def view_fields(buf: np.ndarray, M: int, nx: int, nr: int) -> np.ndarray:
    return buf[: N_FIELDS * M * nx * nr].reshape(N_FIELDS, M, nx, nr)


@dataclass
class Laser:
    """An m = 1 linearly polarised Gaussian pulse travelling towards +x.

    A(x, r) = a0 omega exp(-r^2/w0^2) exp(-2 ln2 (x-x0)^2 / fwhm^2) cos(k (x-x0))
    with fwhm the intensity FWHM and w0 the 1/e field radius.  For y
    polarisation E_r^(1) = A, E_theta^(1) = -iA, B_theta^(1) = A, B_r^(1) = iA
    (so E_r = i E_theta on the axis, Sec. 2.3); z polarisation multiplies
    all four by i."""
    a0: float
    lam: float
    w0: float
    fwhm: float
    x0: float
    pol: str = "y"

    def amplitude(self, x, r, xp=np):
        k = 2.0 * math.pi / self.lam
        return (self.a0 * k * xp.exp(-(r ** 2) / self.w0 ** 2)
                * xp.exp(-2.0 * math.log(2.0) * (x - self.x0) ** 2 / self.fwhm ** 2)
                * xp.cos(k * (x - self.x0)))


def add_lasers(buf, M, nx, nr, dr, lasers, x_offset=0.0):
    """Add forward m = 1 pulses: T_r^+ = E_r + B_theta = 2 A p, T_theta^- =
    E_theta - B_r = -2i A p with p = 1 (y) or i (z); T_r^- = T_theta^+ = 0."""
    if M < 2:
        return buf
    xp = np
    if not isinstance(buf, np.ndarray):  # a torch tensor: build on its device
        import torch as xp
    F = buf[: N_FIELDS * M * nx * nr].reshape(N_FIELDS, M, nx, nr)
    if xp is np:
        x = (np.arange(nx) + x_offset)[:, None]
        r_half = ((np.arange(nr) + 0.5) * dr)[None, :]
        r_int = (np.arange(nr) * dr)[None, :]
    else:
        kw = dict(dtype=xp.float64, device=buf.device)
        x = (xp.arange(nx, **kw) + x_offset)[:, None]
        r_half = ((xp.arange(nr, **kw) + 0.5) * dr)[None, :]
        r_int = (xp.arange(nr, **kw) * dr)[None, :]
    for L in lasers:
        p = 1.0 if L.pol == "y" else 1j
        F[FIELDS.index("Trp"), 1] += 2.0 * p * L.amplitude(x, r_half, xp)
        F[FIELDS.index("Ttm"), 1] += -2j * p * L.amplitude(x, r_int, xp)
    return buf


def laser_inflow(lasers, M, nr, dr, nsteps, h=1.0):
    """Inflow arrays for injecting forward m = 1 pulses at x_min
    (qds_set_inflow_i): T_r^+ and T_theta^- of the exterior cell behind x_min
    at steps 0..nsteps-1, each [nsteps, M, nr] complex128.  A pulse given
    with its centre x0 < 0 (window coordinates, behind the box) enters as a
    forward wave would: the value at step n is its initial profile at
    x = -1 - n h (the c dt = dx shift), i.e. the field on the plane x_min
    without the diffraction it would undergo before reaching it."""
    in_rp = np.zeros((nsteps, M, nr), np.complex128)
    in_tm = np.zeros((nsteps, M, nr), np.complex128)
    if M < 2:
        return in_rp, in_tm
    x = (-1.0 - h * np.arange(nsteps))[:, None]
    r_half = ((np.arange(nr) + 0.5) * dr)[None, :]
    r_int = (np.arange(nr) * dr)[None, :]
    for L in lasers:
        p = 1.0 if L.pol == "y" else 1j
        in_rp[:, 1] += 2.0 * p * L.amplitude(x, r_half)
        in_tm[:, 1] += -2j * p * L.amplitude(x, r_int)
    return in_rp, in_tm


def random_state(rng, M, nx, nr, scale=1.0, axis_consistent=True):
    """Random complex state for tiny-grid parity checks.  Mode 0 is kept real
    (the m = 0 fields of a real field are real).  With ``axis_consistent`` the
    on-axis values obey the regularity rules of Sec. 2.3 (E_x^(m!=0) = 0,
    T_theta^(m!=1) = 0 on the axis)."""
    buf = empty_state(M, nx, nr)
    buf[:] = scale * (rng.standard_normal(buf.size) + 1j * rng.standard_normal(buf.size))
    F = view_fields(buf, M, nx, nr)
    F[:, 0] = F[:, 0].real
    pp = buf[N_FIELDS * M * nx * nr:].reshape(M, nx)
    pp[0] = pp[0].real
    if axis_consistent:
        for m in range(M):
            if m != 0:
                F[FIELDS.index("Ex"), m, :, 0] = 0
                F[FIELDS.index("Ex1"), m, :, 0] = 0
            if m != 1:
                for n in ("Ttp", "Ttm", "Ttp1", "Ttm1"):
                    F[FIELDS.index(n), m, :, 0] = 0
    return buf


def random_sources(rng, M, nx, nr, scale=1.0):
    out = []
    for _ in range(3):
        a = scale * (rng.standard_normal((M, nx, nr)) + 1j * rng.standard_normal((M, nx, nr)))
        a[0] = a[0].real
        out.append(np.ascontiguousarray(a))
    return out


# ---------------------------------------------------------------------------
# Workloads shaped like the paper's tests (Sec. 4).
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    nx: int
    nr: int
    M: int
    dr: float
    steps: int
    lasers: list
    axion: bool = False
    arem: bool = False
    moving_window: bool = False
    g: float = 0.0
    m_a: float = 0.0
    bunch: dict | None = None
    h: float = 1.0
    extra: dict = field(default_factory=dict)

    def initial_state(self, device=None):
        """Canonical complex128 initial state: numpy on the host, or a torch
        tensor built on ``device``."""
        if device is None:
            buf = empty_state(self.M, self.nx, self.nr)
        else:
            import torch
            buf = torch.zeros(state_size(self.M, self.nx, self.nr), dtype=torch.complex128, device=device)
        return add_lasers(buf, self.M, self.nx, self.nr, self.dr, self.lasers)

    def cell_modes(self):
        return self.nx * self.nr * self.M


def vacuum_pulse():
    """Plain vacuum EM step: nx=256, nr=32, modes {0,1}, dx=1, dr=2, 200
    steps, moving window; m=1 y-polarised pulse, lambda 16, intensity FWHM
    4 wavelengths, waist 8 dr, a0 = 1, centred at x = 64."""
    return Workload("vacuum_pulse_256x32_m2", 256, 32, 2, 2.0, 200,
                    [Laser(1.0, 16.0, 16.0, 64.0, 64.0, "y")], moving_window=True)


def driven_wake():
    """Wakefield-shaped driven run: nx=2048, nr=256, modes {0,1,2}, 2000 steps,
    dr = 5 dx (mode 2 needs dr >= 2.25 dx);
    m=1 pulse a0=2, lambda 32, waist 40 dr, FWHM 128, x0 = 1536; m=0 current
    of a Gaussian electron bunch (sigma_x 8, sigma_r 6 dr, density peak 0.05)
    256 cells behind the pulse moving at c, plus 1% uniform noise on j_x, j_r,
    j_theta redrawn every step (seed 1)."""
    dr = 5.0
    return Workload("driven_wake_2048x256_m3", 2048, 256, 3, dr, 2000,
                    [Laser(2.0, 32.0, 40 * dr, 128.0, 1536.0, "y")],
                    bunch=dict(rho=-0.05, sx=8.0, sr=6 * dr, x0=1280.0, noise=0.01, seed=1))


def two_colour(nx=8192, nr=256, steps=20000):
    """Two-colour axion generation: EM modes {0,1} + axion + regenerated
    fields, moving window, dr = 5 dx; pulse 1 lambda 16 a0 0.5 (y), pulse 2 omega2 =
    0.8 omega1 (lambda 20) a0 0.5 (z), waist 32 dr, FWHM 4 lambda1, both at
    x0 = 0.75 nx; vacuum phase matching of omega1 - omega2 gives m_a = 0;
    g = 1e-6."""
    x0 = 0.75 * nx
    dr = 5.0
    return Workload(f"two_colour_{nx}x{nr}_m2", nx, nr, 2, dr, steps,
                    [Laser(0.5, 16.0, 32 * dr, 64.0, x0, "y"), Laser(0.5, 20.0, 32 * dr, 64.0, x0, "z")],
                    axion=True, arem=True, moving_window=True, g=1e-6, m_a=0.0)


def batched_scan(n=512, seed=2, steps=1000, dr=5.0):
    """Batched vacuum two-colour scan: per instance (draw order nx, nr, m_max,
    omega2/omega1, g from numpy PCG64(seed)): nx log-uniform [512, 4096], nr
    log-uniform [32, 256], m_max uniform {1,2,3} (modes 0..m_max, so the m=1
    pulses are always represented), omega2/omega1 uniform [0.5, 0.9], g
    log-uniform [1e-8, 1e-4]; m_a = 0; pulse 1 lambda 16 a0 0.5 (y), pulse 2
    (z) a0 0.5, waist min(32 dr, R/4), FWHM 64, x0 = 0.75 nx; moving window;
    dr = 5 dx (the paper's mesh ratio dx = lambda/10, dr = lambda/2; m_max = 3
    needs dr >= 3.25 dx for stability)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(n):
        nx = int(round(math.exp(rng.uniform(math.log(512), math.log(4096)))))
        nr = int(round(math.exp(rng.uniform(math.log(32), math.log(256)))))
        mmax = int(rng.integers(1, 4))
        ratio = float(rng.uniform(0.5, 0.9))
        g = float(math.exp(rng.uniform(math.log(1e-8), math.log(1e-4))))
        w0 = min(32 * dr, 0.25 * nr * dr)
        x0 = 0.75 * nx
        lam1 = 16.0
        out.append(Workload(f"scan_{b}", nx, nr, mmax + 1, dr, steps,
                            [Laser(0.5, lam1, w0, 64.0, x0, "y"),
                             Laser(0.5, lam1 / ratio, w0, 64.0, x0, "z")],
                            axion=True, arem=True, moving_window=True, g=g, m_a=0.0,
                            extra=dict(ratio=ratio)))
    return out


def bunch_currents(wl: Workload, step: int):
    """Currents of the driven wake run at step ``step``: j_x at (i+1/2, j, n),
    j_r at (i, j+1/2, n+1/2), j_theta at (i, j, n+1/2); the bunch (m=0)
    carries j_x = rho c, moving at c; every component, mode, real/imaginary
    part (imaginary part zero for m=0) and cell gets an independent uniform
    noise of amplitude noise * max|rho|, drawn from PCG64 seeded by
    (seed, step)."""
    b = wl.bunch
    M, nx, nr, dr, h = wl.M, wl.nx, wl.nr, wl.dr, wl.h
    xb = b["x0"] + step * h
    x_face = (np.arange(nx) + 0.5)[:, None]
    r_int = (np.arange(nr) * dr)[None, :]
    jx = np.zeros((M, nx, nr), np.complex128)
    jx[0] = b["rho"] * np.exp(-((x_face - xb) ** 2) / (2 * b["sx"] ** 2)) * np.exp(-(r_int ** 2) / (2 * b["sr"] ** 2))
    jr = np.zeros((M, nx, nr), np.complex128)
    jt = np.zeros((M, nx, nr), np.complex128)
    amp = b["noise"] * abs(b["rho"])
    rng = np.random.Generator(np.random.PCG64([b["seed"], step]))
    for a in (jx, jr, jt):
        re = rng.uniform(-1.0, 1.0, (M, nx, nr))
        im = rng.uniform(-1.0, 1.0, (M, nx, nr))
        im[0] = 0.0
        a += amp * (re + 1j * im)
    return jx, jr, jt


def adjoint_run(nx=4096, nr=128, steps=8000):
    """Gradient workload: the two-colour pair of the two-colour run (pulse 1
    lambda 16, a0 0.5, y; pulse 2 omega2 = 0.8 omega1, a0 0.5, z; waist
    32 dr, FWHM 64, x0 = 0.75 nx) with modes {0, 1, 2}, plus the driven-wake
    electron bunch (rho -0.05, sigma_x 8, sigma_r 6 dr) 256 cells behind the
    pulses and 1% uniform noise on every current, redrawn each step (seed 1);
    moving window, dr = 5, g = 1e-6, m_a = 0.  ``lasers`` holds pulse 1
    only: pulse 2 is the differentiated input (its radial profile and
    omega2), with its default values in ``extra``."""
    dr = 5.0
    x0 = 0.75 * nx
    lam1, a0, w0, fwhm = 16.0, 0.5, 32 * dr, 64.0
    omega2 = 0.8 * 2 * math.pi / lam1
    r_half = (np.arange(nr) + 0.5) * dr
    profile2 = (a0 * omega2 * np.exp(-(r_half ** 2) / w0 ** 2)).astype(np.complex128)
    return Workload(f"adjoint_two_colour_bunch_{nx}x{nr}_m3", nx, nr, 3, dr, steps,
                    [Laser(a0, lam1, w0, fwhm, x0, "y")], axion=True, arem=True, moving_window=True,
                    g=1e-6, m_a=0.0,
                    bunch=dict(rho=-0.05, sx=8.0, sr=6 * dr, x0=x0 - 256.0, noise=0.01, seed=1),
                    extra=dict(x0=x0, fwhm=fwhm, omega2=omega2, profile2=profile2, window=(int(x0) - 256, int(x0) + 256)))


class DeviceBunchSources:
    """Per-step currents of a bunch workload on a CUDA device, written into
    three fixed buffers (so a solver sees the same source pointers every
    step): the m = 0 bunch j_x, stationary in a window that moves at c, plus
    uniform noise of amplitude noise * |rho| on every component, mode and
    cell (imaginary part zero for m = 0).  The noise is counter-based
    (qds_bunch_currents: SplitMix64 keyed by (seed, step)) and FP32-exact, the
    bunch added in FP64 and rounded once, so an FP32 run sees the FP64 run's
    values rounded, and calling it with the same step reproduces the same
    values."""

    def __init__(self, wl, device, dtype):
        import torch
        b = wl.bunch
        self.torch = torch
        self.M, self.nx, self.nr = wl.M, wl.nx, wl.nr
        self.seed, self.amp = int(b["seed"]), float(b["noise"] * abs(b["rho"]))
        self.dtype, self.device = dtype, device
        x = (torch.arange(wl.nx, dtype=torch.float64, device=device) + 0.5)[:, None]
        r = (torch.arange(wl.nr, dtype=torch.float64, device=device) * wl.dr)[None, :]
        self.bunch_re = (b["rho"] * torch.exp(-((x - b["x0"]) ** 2) / (2 * b["sx"] ** 2))
                         * torch.exp(-(r ** 2) / (2 * b["sr"] ** 2))).contiguous()
        self.buf = [torch.zeros((wl.M, wl.nx, wl.nr), dtype=dtype, device=device) for _ in range(3)]

    def _draw(self, step, out):
        """The currents of step ``step`` into ``out`` ([M, nx, nr] each), or
        of the steps step .. step + count - 1 ([count, M, nx, nr] each), in
        one launch."""
        from . import qds as Q
        Q.bunch_currents(self.seed, int(step), self.amp, self.bunch_re, *out,
                         stream=self.torch.cuda.current_stream(self.device))

    def __call__(self, step):
        self._draw(step, self.buf)
        return tuple(self.buf)

    def fill(self, n0, count, out=None):
        """The currents of steps n0 .. n0+count-1 (the values __call__ gives)
        as three tensors [count, M, nx, nr], in buffers kept for reuse (or in
        ``out``, three such tensors of at least ``count`` steps)."""
        torch = self.torch
        blk = out if out is not None else getattr(self, "_blk", None)
        if blk is None or blk[0].shape[0] < count:
            assert out is None
            blk = self._blk = [torch.empty((count, self.M, self.nx, self.nr), dtype=self.dtype, device=self.device)
                               for _ in range(3)]
        views = [b[:count] for b in blk]
        self._draw(n0, views)
        return tuple(views)
