"""GPU transpose of the step (qds_adjoint_step) and the checkpointed gradient
(run_qds) against the oracle.

Per step: every entry of J^T lambda against the oracle's Jacobian columns on
a tiny grid, and <lambda, J d> = <J^T lambda, d> with J d from the oracle on
grids that span several thread blocks with a ragged tail.  Through N steps:
the gradient of an axion-energy loss with respect to a laser-2 radial
profile, omega2 and g against central differences of the same loss
evaluated by the oracle, and dL/dg = 2 L / g for an axion grown from zero.
"""
import numpy as np
import pytest

import oracle
from paper_2609_03550_b300 import inputs as I
from tests._helpers import oracle_run, oracle_vjp, stable_dr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _Q():
    from paper_2609_03550_b300 import build as B
    B.build_cuda()
    from paper_2609_03550_b300 import qds as Q
    return Q


def em_axion_mask(M, nx, nr):
    n = M * nx * nr
    m = np.zeros(15 * n + M * nx, bool)
    m[:9 * n] = True
    m[15 * n:] = True
    return m


def rdot(a, b):
    return float(np.sum(a.real * b.real + a.imag * b.imag))


def gpu_vjp(Q, p, s, lam, src=(None, None, None), dg=False):
    solver = Q.QDSSolver(p, device=DEV)
    rd = solver.rdtype
    jx, jr, jt = (None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(rd) for a in src)
    fwd = torch.from_numpy(s).to(DEV)
    lt = torch.from_numpy(lam.copy()).to(DEV)
    acc = torch.zeros(1, dtype=torch.float64, device=DEV) if dg else None
    solver.adjoint_step(fwd, lt, jx=jx, jth=jt, dLdg=acc)
    torch.cuda.synchronize()
    out = lt.cpu().numpy()
    return (out, float(acc.item())) if dg else out


@pytest.mark.parametrize("M,mw,prec", [(1, False, 0), (2, True, 0), (3, False, 0), (4, True, 0), (2, True, 32)])
def test_adjoint_step_elementwise_vs_oracle_columns(M, mw, prec):
    Q = _Q()
    nx, nr = 9, 5
    m_a, g = 0.1, 0.8
    dr = stable_dr(M, m_a)
    flags = oracle.AXION | (oracle.MOVING_WINDOW if mw else 0)
    rng = np.random.default_rng(60 + M)
    s = I.random_state(rng, M, nx, nr)
    jx, jr, jt = I.random_sources(rng, M, nx, nr, 0.3)
    if prec:  # the sources in the working precision, identical on both sides
        jx, jt = (a.astype(np.complex64).astype(np.complex128) for a in (jx, jt))
    lam = I.random_state(rng, M, nx, nr, axis_consistent=False) * em_axion_mask(M, nx, nr)
    ref = oracle_vjp(s, lam, M, nx, nr, dr, flags, g=g, m_a=m_a, src=(jx, jr, jt, None))
    p = Q.Params(nx, nr, M, dr, m_a=m_a, g=g, flags=flags | prec)
    got = gpu_vjp(Q, p, s, lam, (jx, jr, jt))
    tol = (1e-12 if prec == 0 else 2e-6) * np.abs(ref).max()
    bad = np.argwhere(np.abs(got - ref) > tol).ravel()
    assert bad.size == 0, (bad[:10], got[bad[:5]], ref[bad[:5]])


@pytest.mark.parametrize("M", [1, 2, 3, 4])
@pytest.mark.parametrize("mw", [False, True])
@pytest.mark.parametrize("prec", [0, 32])
def test_adjoint_step_dot_product(M, mw, prec):
    """nx * nr = 4960 points: 19 full blocks of 256 threads and a ragged one."""
    Q = _Q()
    nx, nr = 124, 40
    m_a, g = 0.05, 0.6
    dr = stable_dr(M, m_a)
    flags = oracle.AXION | oracle.AREM | (oracle.MOVING_WINDOW if mw else 0)
    rng = np.random.default_rng(200 + 10 * M + mw)
    s = I.random_state(rng, M, nx, nr)
    jx, jr, jt = I.random_sources(rng, M, nx, nr, 0.3)
    if prec:
        jx, jt = (a.astype(np.complex64).astype(np.complex128) for a in (jx, jt))
    mask = em_axion_mask(M, nx, nr)
    p = Q.Params(nx, nr, M, dr, m_a=m_a, g=g, flags=flags | prec)
    for trial in range(2):
        d = I.random_state(rng, M, nx, nr) * mask
        lam = I.random_state(rng, M, nx, nr, axis_consistent=False) * mask
        F = lambda b: oracle_run(b, M, nx, nr, dr, flags, 1, g=g, m_a=m_a, src=(jx, jr, jt, None), extended=False)
        Jd = 0.5 * (F(s + d) - F(s - d))
        lt = gpu_vjp(Q, p, s, lam, (jx, jr, jt))
        lhs, rhs = rdot(lam, Jd * mask), rdot(lt, d)
        scale = np.linalg.norm(lam) * np.linalg.norm(Jd)
        tol = 1e-12 if prec == 0 else 1e-6
        assert abs(lhs - rhs) < tol * scale, (trial, lhs, rhs)
        assert np.all(lt[~mask] == 0)


@pytest.mark.parametrize("prec", [0, 32])
def test_adjoint_step_coupling_derivative(prec):
    Q = _Q()
    M, nx, nr = 3, 70, 24
    dr = stable_dr(M)
    flags = oracle.AXION | oracle.MOVING_WINDOW
    rng = np.random.default_rng(31)
    s = I.random_state(rng, M, nx, nr)
    lam = I.random_state(rng, M, nx, nr, axis_consistent=False) * em_axion_mask(M, nx, nr)
    g, dgs = 0.4, 0.1
    Fp = oracle_run(s, M, nx, nr, dr, flags, 1, g=g + dgs, extended=False)
    Fm = oracle_run(s, M, nx, nr, dr, flags, 1, g=g - dgs, extended=False)
    fd = rdot(lam * em_axion_mask(M, nx, nr), Fp - Fm) / (2 * dgs)
    p = Q.Params(nx, nr, M, dr, g=g, flags=flags | prec)
    _, dg = gpu_vjp(Q, p, s, lam, dg=True)
    tol = 1e-11 if prec == 0 else 1e-5
    assert abs(dg - fd) < tol * abs(fd), (dg, fd)


@pytest.mark.parametrize("M,mw", [(1, False), (3, True), (4, True), (2, False)])
@pytest.mark.parametrize("prec", [0, 32])
def test_working_transpose_matches_canonical_transpose(M, mw, prec):
    """qds_adjoint_step_w on an EM-only working snapshot taken after a few
    steps (ring offset 5 in the moving window) gives what qds_adjoint_step
    gives on the canonical state of the same moment, entry for entry (the
    canonical path only converts), with and without the snapshot at the end
    of the step (E_x, B_x^(n+1/2) read instead of recomputed)."""
    Q = _Q()
    nx, nr = 124, 41
    m_a, g = 0.05, 0.6
    dr = stable_dr(M, m_a)
    flags = oracle.AXION | oracle.AREM | (oracle.MOVING_WINDOW if mw else 0)
    rng = np.random.default_rng(700 + 10 * M + mw)
    p = Q.Params(nx, nr, M, dr, m_a=m_a, g=g, flags=flags | prec)
    solver = Q.QDSSolver(p, device=DEV)
    rd = solver.rdtype
    solver.set_state(torch.from_numpy(I.random_state(rng, M, nx, nr)).to(DEV))
    jx, jr, jt = (torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(rd) for a in I.random_sources(rng, M, nx, nr, 0.3))
    solver.step(5, jx=jx, jr=jr, jth=jt)
    snap, k = solver.save_working(em_only=True)
    assert k == 5 and snap.numel() == solver.working_bytes(0, em_only=True)
    fwd = solver.get_state()
    lam = I.random_state(rng, M, nx, nr, axis_consistent=False) * em_axion_mask(M, nx, nr)
    lam_w = torch.from_numpy(lam).to(DEV).to(rd).contiguous()
    lam_c = lam_w.to(torch.complex128, copy=True)  # a copy also in FP64: adjoint_step works in place
    out_w = torch.zeros_like(lam_w)  # the regenerated planes are not written
    dg_c = torch.zeros(1, dtype=torch.float64, device=DEV)
    dg_w = torch.zeros(1, dtype=torch.float64, device=DEV)
    solver.adjoint_step(fwd, lam_c, jx=jx, jth=jt, dLdg=dg_c)
    solver.adjoint_step_w(snap, k, lam_w, out_w, jx=jx, jth=jt, dLdg=dg_w)
    # the same with the snapshot at the end of the step, whose E_x, B_x^(n+1/2)
    # replace their recomputation (the step's own rounding)
    solver.step(1, jx=jx, jr=jr, jth=jt)
    nxt, _ = solver.save_working(em_only=True)
    out_n = torch.zeros_like(lam_w)
    dg_n = torch.zeros(1, dtype=torch.float64, device=DEV)
    solver.adjoint_step_w(snap, k, lam_w, out_n, jx=jx, jth=jt, dLdg=dg_n, fwd_next=nxt)
    torch.cuda.synchronize()
    b = lam_c.cpu().numpy()
    for out, dg, eps in ((out_w, dg_w, 1e-14 if prec == 0 else 1e-6), (out_n, dg_n, 1e-12 if prec == 0 else 1e-5)):
        a = out.to(torch.complex128).cpu().numpy()
        bad = np.argwhere(np.abs(a - b) > eps * np.abs(b).max()).ravel()
        assert bad.size == 0, (eps, bad[:10], a[bad[:5]], b[bad[:5]])
        assert abs(float(dg.item()) - float(dg_c.item())) <= eps * abs(float(dg_c.item()))


@pytest.mark.parametrize("prec", [0, 32])
def test_em_only_handle_reproduces_the_em_planes(prec):
    """The backward re-runs segments on a handle without the axion and the
    regenerated group: after driven steps from a restored working snapshot,
    its EM fields equal the full step's bit for bit (the EM group does not
    depend on the other groups)."""
    import copy
    Q = _Q()
    M, nx, nr = 3, 150, 37
    dr = stable_dr(M, 0.05)
    rng = np.random.default_rng(900 + prec)
    p = Q.Params(nx, nr, M, dr, m_a=0.05, g=0.7, flags=oracle.AXION | oracle.AREM | oracle.MOVING_WINDOW | prec)
    pe = copy.copy(p)
    pe.flags = p.flags & ~(oracle.AXION | oracle.AREM)
    full, em = Q.QDSSolver(p, device=DEV), Q.QDSSolver(pe, device=DEV)
    full.set_state(torch.from_numpy(I.random_state(rng, M, nx, nr)).to(DEV))
    srcs = [tuple(torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(full.rdtype)
                  for a in I.random_sources(rng, M, nx, nr, 0.3)) for _ in range(4)]
    full.step(2, jx=srcs[0][0], jr=srcs[0][1], jth=srcs[0][2])
    ck, n0 = full.save_working()
    em.restore_working(ck, n0)
    for jx, jr, jt in srcs[1:]:
        full.step(1, jx=jx, jr=jr, jth=jt)
        em.step(1, jx=jx, jr=jr, jth=jt)
    assert full.steps_taken() == em.steps_taken() == 5
    # the EM planes of the canonical state (the working layout pads FP32 rows)
    n6 = 6 * M * nx * nr
    a, b = full.get_state()[:n6], em.get_state()[:n6]
    assert torch.equal(a, b)


def test_adjoint_rejects_unsupported_boundaries():
    Q = _Q()
    p = Q.Params(16, 8, 2, 2.0, g=0.5, flags=oracle.AXION | oracle.X_PERIODIC)
    s = np.zeros(p.state_elems(), np.complex128)
    with pytest.raises(Q.QDSError, match="open boundaries"):
        gpu_vjp(Q, p, s, s.copy())


# ---------------------------------------------------------------------------
# gradients through N steps


class Case:
    """A small two-colour run with a drive: laser 1 fixed, laser 2 given by
    a complex radial profile and omega2; an m = 0 bunch current and uniform
    noise on every current redrawn each step; loss = axion energy in the
    front window cells."""

    def __init__(self, prec, nx=96, nr=16, M=3, nsteps=30, every=7, seed=5):
        self.M, self.nx, self.nr, self.nsteps, self.every = M, nx, nr, nsteps, every
        self.dr = stable_dr(M) * 1.6
        self.flags = oracle.AXION | oracle.AREM | oracle.MOVING_WINDOW
        self.prec = prec
        self.g = 0.3
        self.x0, self.fwhm = 0.6 * nx, 24.0
        wl = I.Workload("adjoint_case", nx, nr, M, self.dr, nsteps,
                        [I.Laser(0.5, 16.0, 4 * self.dr, 24.0, self.x0, "y")])
        self.base = wl.initial_state()
        rng = np.random.default_rng(seed)
        r = (np.arange(nr) + 0.5) * self.dr
        self.profile0 = 0.5 * (2 * np.pi / 20.0) * np.exp(-(r / (4 * self.dr)) ** 2) * (1 + 0.2j * rng.standard_normal(nr))
        self.omega2 = 2 * np.pi / 20.0
        self.src = []
        xf = (np.arange(nx) + 0.5)[:, None]
        ri = (np.arange(nr) * self.dr)[None, :]
        for n in range(nsteps):
            jx = np.zeros((M, nx, nr), np.complex128)
            jx[0] = -0.05 * np.exp(-((xf - 0.3 * nx) ** 2) / (2 * 8.0 ** 2)) * np.exp(-(ri ** 2) / (2 * (2 * self.dr) ** 2))
            parts = []
            for a in (jx, np.zeros_like(jx), np.zeros_like(jx)):
                noise = 5e-4 * (rng.uniform(-1, 1, a.shape) + 1j * rng.uniform(-1, 1, a.shape))
                noise[0] = noise[0].real
                b = a + noise
                if prec:
                    b = b.astype(np.complex64).astype(np.complex128)
                parts.append(np.ascontiguousarray(b))
            self.src.append(tuple(parts))
        self.Q = _Q()
        self.p = self.Q.Params(nx, nr, M, self.dr, g=self.g, flags=self.flags | prec)
        self._dev_src = None

    def sources(self, n):
        if self._dev_src is None:
            rd = torch.complex64 if self.prec else torch.complex128
            self._dev_src = [tuple(torch.from_numpy(a).to(DEV).to(rd) for a in t) for t in self.src]
        return self._dev_src[n]

    def state0(self, profile, omega2, device):
        from paper_2609_03550_b300.adjoint import laser2_state
        base = torch.from_numpy(self.base).to(device)
        return laser2_state(base, self.p, profile, omega2, self.x0, self.fwhm)

    def loss(self, state):
        from paper_2609_03550_b300.adjoint import axion_energy
        return axion_energy(state, self.p, self.nx - 32, self.nx)

    def oracle_loss(self, profile, omega2, g):
        s0 = self.state0(torch.as_tensor(profile, dtype=torch.complex128), torch.tensor(float(omega2), dtype=torch.float64),
                         "cpu").numpy().copy()
        st = oracle.State(self.M, self.nx, self.nr, s0)
        pd = dict(nx=self.nx, nr=self.nr, M=self.M, h=1.0, dr=self.dr, g=g, m_a=0.0, flags=self.flags)
        for n in range(self.nsteps):
            jx, jr, jt = self.src[n]
            oracle.step(pd, st, jx, jr, jt)
        return float(self.loss(torch.from_numpy(st.buf)))

    def gpu_grad(self):
        from paper_2609_03550_b300.adjoint import RunSpec, run_qds
        prof = torch.tensor(self.profile0, dtype=torch.complex128, device=DEV, requires_grad=True)
        om = torch.tensor(self.omega2, dtype=torch.float64, device=DEV, requires_grad=True)
        g = torch.tensor(self.g, dtype=torch.float64, device=DEV, requires_grad=True)
        spec = RunSpec(self.p, self.nsteps, every=self.every, sources=self.sources, device=DEV)
        L = self.loss(run_qds(self.state0(prof, om, DEV), g, spec))
        L.backward()
        return float(L), prof.grad.cpu().numpy(), float(om.grad), float(g.grad)


def _richardson(f, x0, h):
    """Central difference with one Richardson step (error O(h^4))."""
    d1 = (f(x0 + h) - f(x0 - h)) / (2 * h)
    d2 = (f(x0 + h / 2) - f(x0 - h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("prec", [0, 32])
def test_run_gradient_vs_oracle_central_differences(prec):
    c = Case(prec)
    L, gprof, gom, gg = c.gpu_grad()
    L0 = c.oracle_loss(c.profile0, c.omega2, c.g)
    print(f"loss gpu {L!r} oracle {L0!r}")
    assert abs(L - L0) < (1e-12 if prec == 0 else 1e-4) * abs(L0), (L, L0)
    tol = 1e-8 if prec == 0 else 1e-4
    rng = np.random.default_rng(9)
    # profile: along a random complex direction, step 1e-4 of the profile
    dirn = rng.standard_normal(c.nr) + 1j * rng.standard_normal(c.nr)
    dirn *= np.linalg.norm(c.profile0) / np.linalg.norm(dirn)
    fd = _richardson(lambda t: c.oracle_loss(c.profile0 + t * dirn, c.omega2, c.g), 0.0, 1e-4)
    ad = rdot(gprof, dirn)
    print(f"profile adjoint {ad!r} fd {fd!r}")
    assert abs(ad - fd) < tol * abs(fd), ("profile", ad, fd)
    fd = _richardson(lambda w: c.oracle_loss(c.profile0, w, c.g), c.omega2, 1e-4 * c.omega2)
    print(f"omega2 adjoint {gom!r} fd {fd!r}")
    assert abs(gom - fd) < tol * abs(fd), ("omega2", gom, fd)
    fd = _richardson(lambda gg_: c.oracle_loss(c.profile0, c.omega2, gg_), c.g, 1e-4 * c.g)
    print(f"g adjoint {gg!r} fd {fd!r} 2L/g {2 * L / c.g!r}")
    assert abs(gg - fd) < tol * abs(fd), ("g", gg, fd)
    # the axion grows from zero and is linear in g, so L is quadratic in g
    assert abs(gg - 2 * L / c.g) < (1e-10 if prec == 0 else 1e-5) * abs(gg), (gg, 2 * L / c.g)


def test_run_rejects_regenerated_cotangent():
    from paper_2609_03550_b300.adjoint import RunSpec, run_qds
    Q = _Q()
    p = Q.Params(32, 8, 2, 2.0, g=0.5, flags=oracle.AXION | oracle.AREM)
    s0 = torch.zeros(p.state_elems(), dtype=torch.complex128, device=DEV, requires_grad=True)
    g = torch.tensor(0.5, dtype=torch.float64, device=DEV)
    out = run_qds(s0, g, RunSpec(p, 3, device=DEV))
    n = 2 * 32 * 8
    with pytest.raises(Q.QDSError, match="regenerated"):
        out[9 * n:10 * n].real.sum().backward()


# ---------------------------------------------------------------------------
# the gradient workload itself (4096 x 128, modes 0..2, bunch + noise)


def _gradient_case(steps):
    import math
    from paper_2609_03550_b300 import adjoint as A
    Q = _Q()
    wl = I.adjoint_run(steps=steps)
    ex = wl.extra
    base = wl.initial_state(device=DEV)

    def params(prec):
        return Q.Params(wl.nx, wl.nr, wl.M, wl.dr, g=wl.g, m_a=wl.m_a, flags=Q.AXION | Q.AREM | Q.MOVING_WINDOW | prec)

    def state0(p, prof, om):
        return A.laser2_state(base, p, prof, om, ex["x0"], ex["fwhm"])

    def gradient(prec):
        p = params(prec)
        src = I.DeviceBunchSources(wl, DEV, torch.complex64 if prec else torch.complex128)
        spec = A.RunSpec(p, steps, every=max(1, int(round(math.sqrt(steps)))), sources=src, device=DEV)
        prof = torch.tensor(ex["profile2"], dtype=torch.complex128, device=DEV, requires_grad=True)
        om = torch.tensor(ex["omega2"], dtype=torch.float64, device=DEV, requires_grad=True)
        g = torch.tensor(wl.g, dtype=torch.float64, device=DEV, requires_grad=True)
        L = A.axion_energy(A.run_qds(state0(p, prof, om), g, spec), p, *ex["window"])
        L.backward()
        return float(L.detach()), prof.grad.cpu().numpy(), float(om.grad), float(g.grad)

    def loss64(prof, om, g):
        """Forward only, FP64."""
        p = params(0)
        p.g = g
        src = I.DeviceBunchSources(wl, DEV, torch.complex128)
        s = Q.QDSSolver(p, device=DEV)
        with torch.no_grad():
            s.set_state(state0(p, torch.as_tensor(prof, device=DEV), torch.tensor(om, dtype=torch.float64, device=DEV)))
        for n in range(steps):
            jx, jr, jt = src(n)
            s.step(1, jx=jx, jr=jr, jth=jt)
        return float(A.axion_energy(s.get_state(), p, *ex["window"]))

    return wl, gradient, loss64


def test_gradient_workload_fp64_and_fp32_against_fp64_central_differences():
    """The gradient workload at full grid size (steps from QDS_FD_STEPS,
    default 1000; 8000 is the benchmark's length): the FP64 and FP32
    gradients with respect to the laser-2 profile (a random complex
    direction), omega2 and g against FP64 central differences (step 1e-4
    relative) of the same loss on the GPU's FP64 path, itself pinned to the
    oracle at 1e-12 on reduced sizes."""
    import os
    steps = int(os.environ.get("QDS_FD_STEPS", "1000"))
    wl, gradient, loss64 = _gradient_case(steps)
    ex = wl.extra
    L64, gp64, go64, gg64 = gradient(0)
    L32, gp32, go32, gg32 = gradient(32)
    rng = np.random.default_rng(3)
    d = rng.standard_normal(wl.nr) + 1j * rng.standard_normal(wl.nr)
    d *= np.linalg.norm(ex["profile2"]) / np.linalg.norm(d)
    h = 1e-4
    fd_p = (loss64(ex["profile2"] + h * d, ex["omega2"], wl.g) - loss64(ex["profile2"] - h * d, ex["omega2"], wl.g)) / (2 * h)
    ho = h * ex["omega2"]
    fd_o = (loss64(ex["profile2"], ex["omega2"] + ho, wl.g) - loss64(ex["profile2"], ex["omega2"] - ho, wl.g)) / (2 * ho)
    hg = h * wl.g
    fd_g = (loss64(ex["profile2"], ex["omega2"], wl.g + hg) - loss64(ex["profile2"], ex["omega2"], wl.g - hg)) / (2 * hg)
    rows = [("profile", rdot(gp64, d), rdot(gp32, d), fd_p), ("omega2", go64, go32, fd_o), ("g", gg64, gg32, fd_g)]
    for name, a64, a32, fd in rows:
        print(f"steps {steps} {name}: fd {fd!r} adjoint fp64 {a64!r} ({abs(a64 - fd) / abs(fd):.2e}) "
              f"fp32 {a32!r} ({abs(a32 - fd) / abs(fd):.2e})")
    print(f"L fp64 {L64!r} fp32 {L32!r} ({abs(L32 - L64) / L64:.2e})")
    for name, a64, a32, fd in rows:
        assert abs(a64 - fd) < 1e-5 * abs(fd), (name, a64, fd)
        assert abs(a32 - fd) < 1e-4 * abs(fd), (name, a32, fd)
