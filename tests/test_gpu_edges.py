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
