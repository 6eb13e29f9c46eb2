"""Shared test helpers (no method arithmetic)."""
import math

import numpy as np

import oracle
from paper_2609_03550_b300 import inputs as I

GROUPS = (("em", 0, 6), ("axion", 6, 9), ("arem", 9, 15))


def group_errors(got, ref, M, nx, nr):
    """Relative L2 error per field group; phi_prev counts with the axion."""
    n = M * nx * nr
    out = {}
    for name, a, b in GROUPS:
        sg = got[a * n:b * n]
        sr = ref[a * n:b * n]
        if name == "axion":
            sg = np.concatenate([sg, got[15 * n:]])
            sr = np.concatenate([sr, ref[15 * n:]])
        den = np.linalg.norm(sr)
        out[name] = (np.linalg.norm(sg - sr) / den) if den > 0 else np.linalg.norm(sg)
    return out


def oracle_run(buf, M, nx, nr, dr, flags, nsteps, g=0.0, m_a=0.0, src=(None, None, None, None), extended=True):
    """The oracle as the parity reference: long double by default, so that the
    paper's E.B form (a difference of nearly equal products between
    co-propagating waves) does not leave FP64 rounding in the reference."""
    st = oracle.State(M, nx, nr, buf)
    oracle.step(dict(nx=nx, nr=nr, M=M, h=1.0, dr=dr, g=g, m_a=m_a, flags=flags & 31), st, *src,
                nsteps=nsteps, extended=extended)
    return st.buf


def parity_cases():
    """(M, flags) combinations covering every boundary mode."""
    out = []
    for M in (1, 2, 3, 4):
        for flags in (0, oracle.AXION, oracle.AXION | oracle.AREM,
                      oracle.AXION | oracle.AREM | oracle.MOVING_WINDOW,
                      oracle.AXION | oracle.AREM | oracle.X_PERIODIC,
                      oracle.AXION | oracle.AREM | oracle.R_CLOSED):
            out.append((M, flags))
    return out


def random_case(seed, M, nx, nr):
    rng = np.random.default_rng(seed)
    buf = I.random_state(rng, M, nx, nr)
    src = I.random_sources(rng, M, nx, nr, 0.3)
    sext = 0.2 * (rng.standard_normal((M, nx, nr)) + 1j * rng.standard_normal((M, nx, nr)))
    sext[0] = sext[0].real
    return buf, src + [np.ascontiguousarray(sext)]


def stable_dr(M, m_a=0.0):
    return max(1.5, (M - 1) + 0.25) * (1 + m_a)


def reference_and_tolerance(buf, M, nx, nr, dr, flags, nsteps, g=0.0, m_a=0.0, src=(None, None, None, None),
                            base=1e-12):
    """Long double reference and per-group FP64 tolerance: ``base``, raised to
    ten times the distance between the FP64 and long double evaluations of
    the same run where the problem itself is worse conditioned (the axion
    of co-propagating vacuum waves is a small residue of O(1) products)."""
    ref = oracle_run(buf, M, nx, nr, dr, flags, nsteps, g=g, m_a=m_a, src=src, extended=True)
    r64 = oracle_run(buf, M, nx, nr, dr, flags, nsteps, g=g, m_a=m_a, src=src, extended=False)
    floor = group_errors(r64, ref, M, nx, nr)
    return ref, {k: max(base, 10.0 * v) for k, v in floor.items()}


def phase_matched_scales(wl, T):
    """Amplitudes the two-colour pair of workload wl would drive in T time
    units if phase matched (manufactured resonance of Sec. 2.2: a source
    S0 cos(kx - wt) grows phi as g S0 t / (2 w)): phi ~ g A1 A2 T / (2 dw)
    with A1, A2 the peak pulse fields and dw = w1 - w2, and the regenerated
    fields, driven by j_a ~ g A1 dw phi, ~ g A1 dw phi T / 2."""
    l1, l2 = wl.lasers[0], wl.lasers[1]
    w1, w2 = 2 * math.pi / l1.lam, 2 * math.pi / l2.lam
    A1, A2 = l1.a0 * w1, l2.a0 * w2
    phi = wl.g * A1 * A2 * T / (2 * (w1 - w2))
    return phi, wl.g * A1 * (w1 - w2) * phi * T / 2


def scaled_errors(got, ref, wl, T):
    """Max |got - ref| of phi and of the regenerated fields over their
    phase-matched scales (phase_matched_scales)."""
    n = wl.M * wl.nx * wl.nr
    s_phi, s_e1 = phase_matched_scales(wl, T)
    return (float(np.abs(got[6 * n:7 * n] - ref[6 * n:7 * n]).max() / s_phi),
            float(np.abs(got[9 * n:15 * n] - ref[9 * n:15 * n]).max() / s_e1))


def amplitude_error(got, ref, M, nx, nr):
    """Per group: max |got - ref| / max |ref| (the error of the field's
    amplitude, for groups whose relative L2 is ill-conditioned)."""
    n = M * nx * nr
    out = {}
    for name, a, b in GROUPS:
        sg = got[a * n:b * n]
        sr = ref[a * n:b * n]
        den = np.max(np.abs(sr))
        out[name] = float(np.max(np.abs(sg - sr)) / den) if den > 0 else float(np.max(np.abs(sg)))
    return out


def oracle_vjp(s, lam, M, nx, nr, dr, flags, g=0.0, m_a=0.0, src=(None, None, None, None), extended=False):
    """J^T lam of one oracle step at state s, column by column: the step is at
    most quadratic in the state, so (F(s + e) - F(s - e)) / 2 is exactly the
    Jacobian column for a basis direction e.  Adjoint convention: the entry
    for a complex value z is dL/dRe z + i dL/dIm z with L = <lam, F> (real
    inner product).  Only the EM and axion components (and phi_prev) are
    probed; the regenerated components of the result are left at zero."""
    n = M * nx * nr
    idx = list(range(9 * n)) + list(range(15 * n, 15 * n + M * nx))
    out = np.zeros_like(s)
    lr, li = lam.real, lam.imag

    def F(buf):
        return oracle_run(buf, M, nx, nr, dr, flags, 1, g=g, m_a=m_a, src=src, extended=extended)

    for q in idx:
        for unit in (1.0, 1j):
            e = np.zeros_like(s)
            e[q] = unit
            col = 0.5 * (F(s + e) - F(s - e))
            v = float(np.sum(lr * col.real + li * col.imag))
            if unit == 1.0:
                out[q] += v
            else:
                out[q] += 1j * v
    return out
