"""NEXT-3: the mode products of many retained modes (Sec. 3.3) on the GPU,
by the convolution sums and by the theta-grid procedure with FFTs, against
the oracle's convolution sums (Eq. mode_convolution): relative error
<= 1e-12 in FP64 and <= 1e-5 in FP32 (max over the output, scaled by its
largest entry), at mode counts up to 64 and ragged point counts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2609_03550_b300 import qds as Q  # noqa: E402

DEV = "cuda:0"


def _case(M, npairs, npts, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((npairs, M, npts)) + 1j * rng.standard_normal((npairs, M, npts))
    B = rng.standard_normal((npairs, M, npts)) + 1j * rng.standard_normal((npairs, M, npts))
    A[:, 0] = A[:, 0].real  # real fields: real m = 0 components
    B[:, 0] = B[:, 0].real
    w = [1.0, 0.5, -0.5, 0.25][:npairs]
    return A, B, w


@pytest.mark.parametrize("method", [Q.MODES_DIRECT, Q.MODES_THETA])
@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 11, 16, 33, 64])
@pytest.mark.parametrize("fp32", [False, True])
def test_mode_products_match_oracle(method, M, fp32):
    npairs, npts = 3, 203
    A, B, w = _case(M, npairs, npts, 17 * M + method)
    ref = oracle.mode_products(A, B, w)
    dt = torch.complex64 if fp32 else torch.complex128
    got = Q.mode_products(torch.from_numpy(A).to(DEV).to(dt), torch.from_numpy(B).to(DEV).to(dt), w, method=method)
    torch.cuda.synchronize()
    err = np.abs(got.cpu().numpy().astype(np.complex128) - ref).max() / np.abs(ref).max()
    assert err < (1e-5 if fp32 else 1e-12), err


def test_theta_points_rule():
    for M, N in [(1, 2), (2, 4), (4, 16), (11, 32), (22, 64), (23, 128), (64, 256)]:
        assert Q.lib().qds_mode_products_theta_points(M) == N
        assert N >= 3 * M - 2 and (N // 2 < 3 * M - 2 or N == 2)
