"""Edge cases of the GPU step against the oracle: the smallest grids the
library accepts (nx = 8, nr = 4), both step implementations on them, zero
steps, an all-zero state (stays zero), and a batch mixing the smallest grid
with large ragged ones."""
import numpy as np
import pytest

import oracle
from paper_2609_03550_b300 import inputs as I
from tests._helpers import group_errors, oracle_run, random_case, stable_dr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _Q():
    from paper_2609_03550_b300 import build as B
    B.build_cuda()
    from paper_2609_03550_b300 import qds as Q
    return Q


ALL = 1 | 2 | 4


@pytest.mark.parametrize("M", [1, 2])
@pytest.mark.parametrize("flags", [ALL, 1 | 2 | 8, 1 | 2 | 16])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_smallest_grid_every_step_mode(M, flags, mode):
    Q = _Q()
    nx, nr = 8, 4
    dr, g = stable_dr(M), 0.3
    buf, src = random_case(11 * M + flags, M, nx, nr)
    ref = oracle_run(buf, M, nx, nr, dr, flags, 5, g=g, src=src)
    s = Q.QDSSolver(Q.Params(nx, nr, M, dr, g=g, flags=flags), device=DEV)
    s.set_step_mode(mode)
    s.set_state(torch.from_numpy(buf).to(DEV))
    kw = {n: torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for n, a in zip(("jx", "jr", "jth", "s_ext"), src)}
    s.step(5, **kw)
    got = s.get_state().cpu().numpy()
    for name, e in group_errors(got, ref, M, nx, nr).items():
        assert e < 1e-12, (name, e)


def test_zero_steps_and_zero_state():
    Q = _Q()
    M, nx, nr = 3, 40, 12
    p = Q.Params(nx, nr, M, stable_dr(M), g=0.5, flags=ALL)
    s = Q.QDSSolver(p, device=DEV)
    buf, _ = random_case(3, M, nx, nr)
    s.set_state(torch.from_numpy(buf).to(DEV))
    s.step(0)
    assert np.array_equal(s.get_state().cpu().numpy(), buf)
    s.set_state(torch.zeros(p.state_elems(), dtype=torch.complex128, device=DEV))
    s.step(20)
    assert not bool(s.get_state().abs().max() > 0)


def test_batch_with_smallest_and_ragged_grids():
    Q = _Q()
    shapes = [(8, 4, 1), (200, 37, 3), (8, 4, 2), (333, 61, 2), (97, 250, 4)]
    flags, g = ALL, 0.2
    params, bufs = [], []
    for i, (nx, nr, M) in enumerate(shapes):
        params.append(Q.Params(nx, nr, M, stable_dr(M), g=g, flags=flags))
        bufs.append(random_case(50 + i, M, nx, nr)[0])
    s = Q.QDSSolver(params, device=DEV)
    for i, b in enumerate(bufs):
        s.set_state(torch.from_numpy(b).to(DEV), i)
    s.step(17)  # one captured graph of 16 steps and one single step
    for i, ((nx, nr, M), b) in enumerate(zip(shapes, bufs)):
        ref = oracle_run(b, M, nx, nr, stable_dr(M), flags, 17, g=g)
        got = s.get_state(i).cpu().numpy()
        for name, e in group_errors(got, ref, M, nx, nr).items():
            assert e < 1e-12, (i, name, e)


def test_nonfinite_state_is_reported():
    """A NaN current makes the state non-finite: the x-marching kernels flag
    it at once (qds_status), the flat passes through the energy reduction
    (qds_diagnostics); a new state clears the flag."""
    Q = _Q()
    M, nx, nr = 2, 40, 12
    for mode in (Q.STEP_MARCH, Q.STEP_FLAT):
        p = Q.Params(nx, nr, M, stable_dr(M), g=0.5, flags=ALL)
        s = Q.QDSSolver(p, device=DEV)
        s.set_step_mode(mode)
        buf, _ = random_case(4, M, nx, nr)
        s.set_state(torch.from_numpy(buf).to(DEV))
        s.step(2)
        assert s.status() == 0
        jx = torch.zeros((M, nx, nr), dtype=torch.complex128, device=DEV)
        jx[0, 20, 3] = float("nan")
        s.step(1, jx=jx)
        if mode == Q.STEP_MARCH:
            assert s.status() == 3  # QDS_ERR_NONFINITE
        with pytest.raises(Q.QDSError, match="non-finite"):
            s.diagnostics()
        assert s.status() == 3
        s.set_state(torch.from_numpy(buf).to(DEV))
        s.step(2)
        assert s.status() == 0
        assert np.isfinite(s.diagnostics()["em0"])


def test_bulk_copy_wait_runs_out_and_reports_a_timeout():
    """The bounded wait of the x-marching kernels: with the test hook the
    first column of every CTA is never fetched; the wait runs out, the CTA
    sets the timeout bit and exits, qds_status reports QDS_ERR_TIMEOUT, and
    the context stays usable (the next solve matches the oracle)."""
    Q = _Q()
    M, nx, nr, flags = 2, 24, 10, ALL
    p = Q.Params(nx, nr, M, stable_dr(M), g=0.3, flags=flags)
    s = Q.QDSSolver(p, device=DEV)
    s.set_step_mode(Q.STEP_MARCH)
    buf, _ = random_case(6, M, nx, nr)
    s.set_state(torch.from_numpy(buf).to(DEV))
    s.test_withhold_copy(True)
    s.step(1)
    assert s.status() == 4  # QDS_ERR_TIMEOUT
    s.test_withhold_copy(False)
    s.set_state(torch.from_numpy(buf).to(DEV))
    s.step(3)
    assert s.status() == 0
    ref = oracle_run(buf, M, nx, nr, stable_dr(M), flags, 3, g=0.3)
    for name, e in group_errors(s.get_state().cpu().numpy(), ref, M, nx, nr).items():
        assert e < 1e-12, (name, e)
