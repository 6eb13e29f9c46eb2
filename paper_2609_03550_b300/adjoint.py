"""Gradients of an axion-signal functional through N QDS steps.

``run_qds(state0, g, spec)`` maps an initial canonical state (complex128,
physical variables) and the coupling g to the state after ``spec.nsteps``
steps, as a ``torch.autograd.Function``.  Its backward pass is the
hand-written transpose of the step (``qds_adjoint_step``) with
checkpoint-and-recompute: the forward keeps the state every ``spec.every``
steps (about sqrt(N) of them) as working snapshots, and the backward re-runs
each segment from its checkpoint, keeping the EM planes of that segment's
states, and then applies the transposed steps to it in reverse order in the
working precision.  Memory: N / every working states and ``every`` EM-plane
copies.

The adjoint covers the EM group and the axion: the regenerated fields never
feed back into them, so the gradient is exact for functionals of the EM
fields and the axion; a cotangent with a nonzero regenerated part is
rejected.  The adjoint of a complex value z is dL/dRe z + i dL/dIm z, which
is the gradient PyTorch gives for a real loss of a complex tensor, so the
function composes with torch code before (an initial state built from laser
parameters) and after it (a loss on the final state).

The loss and the initial-state builders below are ordinary torch
expressions on the caller's side of the boundary; every field step and
every transposed step runs in libqds.so.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Optional

import torch

from . import qds as Q

N_FIELDS = 15
F_PHI, F_TAP, F_TAM = 6, 7, 8
F_TRP, F_TTM = 0, 3


@dataclass
class RunSpec:
    """A run of ``nsteps`` steps of one solve.

    params: the statement (its ``g`` is replaced by the value passed to
        ``run_qds``).
    every: checkpoint interval (``None``: round(sqrt(nsteps))).
    sources: ``sources(n)`` -> (jx, jr, jth) device tensors in the working
        precision for step n (window order), or ``None`` for no drive.  It
        is called again for every step during the backward pass and must
        return the same values.
    """
    params: Q.Params
    nsteps: int
    every: Optional[int] = None
    sources: Optional[Callable[[int], tuple]] = None
    device: str = "cuda"

    def interval(self):
        if self.every:
            return int(self.every)
        return max(1, int(round(math.sqrt(self.nsteps))))


def _params_with_g(p: Q.Params, g: float) -> Q.Params:
    return Q.Params(p.nx, p.nr, p.n_modes, p.dr, dx=p.dx, m_a=p.m_a, g=float(g), flags=p.flags, omega0=p.omega0)


def _advance(solver, spec, n0, count):
    """Advance the solver ``count`` steps from step index n0.  With a source
    object that can fill a block of steps (``fill``), the block runs as one
    call with per-step sources (graph replays)."""
    if spec.sources is None:
        solver.step(count)
        return
    if hasattr(spec.sources, "fill"):
        bufs = spec.sources.fill(n0, count)
        solver.set_sources(0, *bufs, per_step=True)
        solver.step(count)
        return
    for n in range(n0, n0 + count):
        jx, jr, jt = spec.sources(n)
        solver.step(1, jx=jx, jr=jr, jth=jt)


class _Run(torch.autograd.Function):
    """Forward: checkpoints are working snapshots (the state as the kernels
    hold it, qds_save_working).  Backward: per segment, the checkpoint is
    restored into a handle that advances the EM group alone, the segment
    re-run keeping the EM planes of the state before every step (all the
    transposed step reads), and the transposed steps
    (qds_adjoint_step_w) run in reverse on the adjoint held in the working
    precision, two buffers in turn: no conversion to complex128 between
    steps."""

    @staticmethod
    def forward(ctx, state0, g, spec: RunSpec):
        p = _params_with_g(spec.params, float(g.detach().cpu()))
        solver = Q.QDSSolver(p, device=spec.device)
        K = spec.interval()
        ckpts = []
        solver.set_state(state0.detach().contiguous())
        n = 0
        while n < spec.nsteps:
            snap, taken = solver.save_working()
            assert taken == n
            ckpts.append((n, snap))
            cnt = min(K, spec.nsteps - n)
            _advance(solver, spec, n, cnt)
            n += cnt
        out = solver.get_state()
        ctx.spec, ctx.solver, ctx.ckpts = spec, solver, ckpts
        return out

    @staticmethod
    def backward(ctx, lam_out):
        spec, solver, ckpts = ctx.spec, ctx.solver, ctx.ckpts
        p = spec.params
        plane = p.n_modes * p.nx * p.nr
        lam128 = lam_out.detach().to(torch.complex128).contiguous()
        if bool((lam128[9 * plane:N_FIELDS * plane] != 0).any()):
            raise Q.QDSError("the adjoint covers the EM fields and the axion; "
                             "the loss must not depend on the regenerated fields")
        lam = lam128.to(solver.rdtype).contiguous()
        lam_b = torch.zeros_like(lam)  # the transposed step leaves the regenerated planes as they are
        dg = torch.zeros(1, dtype=torch.float64, device=lam.device)
        K = spec.interval()
        em_bytes = solver.working_bytes(0, em_only=True)
        pool = [torch.empty(em_bytes, dtype=torch.uint8, device=lam.device) for _ in range(K + 1)]
        fill = spec.sources is not None and hasattr(spec.sources, "fill")
        # The re-runs advance the EM group alone: it is driven by the currents
        # only (S_a and j_a never feed back into it, Sec. 2.2), and the
        # transposed step reads no other forward field.  A handle without the
        # axion and the regenerated group has the same working layout.
        rp = _params_with_g(p, p.g)
        rp.flags = p.flags & ~(Q.AXION | Q.AREM)
        em = Q.QDSSolver(rp, device=spec.device)
        for n0, ck in reversed(ckpts):
            cnt = min(K, spec.nsteps - n0)
            em.restore_working(ck, n0)
            # the segment's currents, drawn once for the re-run and the transpose
            if spec.sources is None:
                blk = [(None, None, None)] * cnt
            elif fill:
                jx, jr, jt = spec.sources.fill(n0, cnt)
                blk = [(jx[k], jr[k], jt[k]) for k in range(cnt)]
            else:
                blk = None
            for k in range(cnt):
                em.save_working(out=pool[k], em_only=True)
                jx, jr, jt = blk[k] if blk is not None else spec.sources(n0 + k)
                em.step(1, jx=jx, jr=jr, jth=jt)
            em.save_working(out=pool[cnt], em_only=True)  # the segment's end: E_x, B_x of its last step
            for k in range(cnt - 1, -1, -1):
                jx, _, jt = blk[k] if blk is not None else spec.sources(n0 + k)
                solver.adjoint_step_w(pool[k], n0 + k, lam, lam_b, jx=jx, jth=jt, dLdg=dg, fwd_next=pool[k + 1])
                lam, lam_b = lam_b, lam
        ctx.ckpts = None
        return lam.to(torch.complex128), dg.reshape(()).to(torch.float64), None


def run_qds(state0: torch.Tensor, g: torch.Tensor, spec: RunSpec) -> torch.Tensor:
    """State after ``spec.nsteps`` steps from ``state0`` with coupling ``g``
    (a 0-d float64 tensor), differentiable in both."""
    return _Run.apply(state0, g, spec)


# ---------------------------------------------------------------------------
# caller-side helpers: a loss on the final state and a differentiable
# initial state


def axion_energy(state: torch.Tensor, p: Q.Params, x_lo: int = 0, x_hi: Optional[int] = None) -> torch.Tensor:
    """Axion energy in the cells [x_lo, x_hi) of the window: the mode-weighted
    volume integral of (1/2)(|d_t phi|^2 + |d_x phi|^2 + |d_r phi|^2 +
    (m^2/r^2 + m_a^2)|phi|^2), with (1/2)(|T_a^+|^2 + |T_a^-|^2) for the
    first two terms (the axion term of the energy diagnostic)."""
    M, nx, nr, dr, h = p.n_modes, p.nx, p.nr, p.dr, p.dx
    F = state[: N_FIELDS * M * nx * nr].reshape(N_FIELDS, M, nx, nr)[:, :, x_lo:x_hi]
    phi, tap, tam = F[F_PHI], F[F_TAP], F[F_TAM]
    kw = dict(dtype=torch.float64, device=state.device)
    m = torch.arange(M, **kw)
    w = torch.where(m == 0, torch.ones_like(m), 0.5 * torch.ones_like(m))[:, None, None]
    rh = ((torch.arange(nr, **kw) + 0.5) * dr)[None, None, :]
    ri = (torch.arange(nr, **kw) * dr)[None, None, 1:]
    u = w * rh * 0.5 * (tap.abs() ** 2 + tam.abs() ** 2)
    u = u + w * rh * ((m[:, None, None] ** 2) / rh ** 2 + p.m_a ** 2) * phi.abs() ** 2
    d = (phi[:, :, 1:] - phi[:, :, :-1]) / dr
    ur = w * ri * d.abs() ** 2
    return 0.5 * 2.0 * math.pi * dr * h * (u.sum() + ur.sum())


def laser2_state(base: torch.Tensor, p: Q.Params, profile: torch.Tensor, omega2: torch.Tensor, x0: float,
                 fwhm: float) -> torch.Tensor:
    """``base`` plus a z-polarised m = 1 pulse with a complex radial profile:
    A(x, r_j) = profile[j] exp(-2 ln2 (x - x0)^2 / fwhm^2) cos(omega2 (x - x0))
    (c = 1), entering T_r^+ = E_r + B_theta = 2 i A at the half rows and
    T_theta^- = E_theta - B_r = 2 A at the integer rows (Sec. 2.3, forward
    m = 1 wave).  Differentiable in ``profile`` ([nr] complex128) and
    ``omega2`` (0-d float64)."""
    M, nx, nr = p.n_modes, p.nx, p.nr
    kw = dict(dtype=torch.float64, device=base.device)
    x = torch.arange(nx, **kw)[:, None]
    env = torch.exp(-2.0 * math.log(2.0) * (x - x0) ** 2 / fwhm ** 2) * torch.cos(omega2 * (x - x0))
    A = env.to(torch.complex128) * profile[None, :]
    plane = M * nx * nr
    add = torch.zeros_like(base)
    add_f = add[: N_FIELDS * plane].reshape(N_FIELDS, M, nx, nr)
    add_f[F_TRP, 1] = 2j * A
    add_f[F_TTM, 1] = 2.0 * A
    return base + add
