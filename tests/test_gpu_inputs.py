"""qds_bunch_currents, the synthetic per-step currents of the driven
workloads: sampled elements against SplitMix64 written out here from its
published definition (Steele, Lea and Flood, OOPSLA 2014), the m = 0 modes
real, the bunch on j_x of m = 0, the FP32 draw equal to the FP64 draw
rounded, reproducible per step (alone or in a block of steps), and the
noise's first two moments."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
MASK = (1 << 64) - 1


def splitmix64(z):
    z = (z + 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def sym_noise(z, amp):
    """(float)amp * (u 2^-23 - 1) in FP32 arithmetic, u the top 24 bits of z."""
    u = np.float32(z >> 40) * np.float32(2.0 ** -23) - np.float32(1.0)
    return float(np.float32(amp) * u)


def draw(M, nx, nr, seed, step, amp, bunch, dtype, count=None):
    from paper_2609_03550_b300 import qds as Q
    shape = (M, nx, nr) if count is None else (count, M, nx, nr)
    out = [torch.full(shape, float("nan"), dtype=dtype, device=DEV) for _ in range(3)]
    Q.bunch_currents(seed, step, amp, bunch, *out)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def test_bunch_currents_against_splitmix64_and_their_structure():
    from paper_2609_03550_b300 import build as B
    B.build_cuda()
    M, nx, nr, seed, step, amp = 3, 37, 29, 12345, 77, 0.25
    rng = np.random.default_rng(1)
    bunch_np = rng.standard_normal((nx, nr))
    bunch = torch.from_numpy(bunch_np).to(DEV)
    j64 = draw(M, nx, nr, seed, step, amp, bunch, torch.complex128)
    j32 = draw(M, nx, nr, seed, step, amp, bunch, torch.complex64)
    again = draw(M, nx, nr, seed, step, amp, bunch, torch.complex128)
    other = draw(M, nx, nr, seed, step + 1, amp, bunch, torch.complex128)
    key = splitmix64(splitmix64(seed) ^ step)
    plane = M * nx * nr
    for e in list(range(0, 3 * plane, 97)) + [3 * plane - 1]:
        c, q = divmod(e, plane)
        m, rem = divmod(q, nx * nr)
        w, j = divmod(rem, nr)
        re = sym_noise(splitmix64((key + 2 * e) & MASK), amp)
        im = 0.0 if m == 0 else sym_noise(splitmix64((key + 2 * e + 1) & MASK), amp)
        if c == 0 and m == 0:
            re += bunch_np[w, j]
        assert j64[c][m, w, j] == complex(re, im), (e, j64[c][m, w, j], re, im)
    for c in range(3):
        assert np.all(j64[c] == again[c])
        assert np.all(j64[c][0].imag == 0)
        assert np.all(j32[c] == j64[c].astype(np.complex64))  # the FP64 values rounded once
        assert np.mean(j64[c] != other[c]) > 0.99
        noise = j64[c] - (np.pad(bunch_np[None], ((0, M - 1), (0, 0), (0, 0))) if c == 0 else 0)
        tol = amp + 1e-12  # the bunch is added with one rounding
        assert np.abs(noise.real).max() <= tol and np.abs(noise.imag).max() <= tol
        # uniform on [-amp, amp): mean 0, variance amp^2 / 3 (n ~ 3e3 values)
        v = np.concatenate([noise.real.ravel(), noise[1:].imag.ravel()])
        assert abs(v.mean()) < 5 * amp / np.sqrt(3 * v.size)
        assert abs(v.var() / (amp ** 2 / 3) - 1) < 0.1


def test_bunch_currents_block_of_steps_equals_single_steps():
    M, nx, nr, seed, amp = 2, 19, 11, 7, 0.5
    bunch = torch.linspace(-1, 1, nx * nr, dtype=torch.float64, device=DEV).reshape(nx, nr).contiguous()
    blk = draw(M, nx, nr, seed, 40, amp, bunch, torch.complex64, count=5)
    for k in range(5):
        one = draw(M, nx, nr, seed, 40 + k, amp, bunch, torch.complex64)
        assert all(np.all(blk[c][k] == one[c]) for c in range(3)), k


def test_bunch_currents_without_bunch_and_zero_amplitude():
    M, nx, nr = 2, 8, 5
    z = draw(M, nx, nr, 1, 0, 0.0, None, torch.complex128)
    assert all(np.all(t == 0) for t in z)
    y = draw(M, nx, nr, 1, 0, 1.0, None, torch.complex64)
    assert all(np.all(np.isfinite(t)) for t in y) and np.all(y[0][0].imag == 0)
