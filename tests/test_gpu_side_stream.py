"""The starts of the large levels on a second stream of the solve graph, through the C ABI.

After a full set-up the start of every level of at least 2^22 nodes (its state, the Dirichlet
shell and ||f_h|| with b / c) is issued before level 2 on a side stream of the CUDA graph and
joined before that level's EXP_finite; the host-driven loop issues the same starts in the same
place on its one stream. The kernels and their inputs are the same, so the two solves agree bit
for bit: iterates of every level, EXP_true, iteration and replacement counts and ||f_h||. A
solve from a finer level (no set-up, so no side stream) agrees with them too. The 256^3 level
of these problems (257^3 nodes) is the smallest that takes the side stream."""
import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_02983_gb300 import build
    build.build()
    from paper_1506_02983_gb300 import ecmg
    return ecmg


def _np(t):
    return t.detach().cpu().numpy()


def _run(E, p, first=0, **kw):
    s = E.solver_from_problem(p, **kw)
    st, status = s.solve()
    assert status == 0, st
    if first:
        st = s.solve_from(first)  # raises on a failed solve
    L = p["levels"]
    out = (st, [_np(s.get(E.ECMG_VEC_U, l)) for l in range(L)], _np(s.get(E.ECMG_VEC_UTILDE)))
    s.close()
    return out


@pytest.mark.parametrize("precision", [1, 0])
def test_side_stream_starts_are_bitwise_the_one_stream_solve(E, precision):
    p = inputs.cos_cube(levels=6, n0=(8, 8, 8), rtol=1e-10)
    g = _run(E, p, precision=precision, use_graph=1)
    h = _run(E, p, precision=precision, use_graph=0)
    for key in ("iters", "updates", "rhs_norm"):
        assert g[0][key] == h[0][key], (key, g[0][key], h[0][key])
    for l in range(p["levels"]):
        assert np.array_equal(g[1][l], h[1][l]), l
    assert np.array_equal(g[2], h[2])


def test_solve_from_a_fine_level_after_side_stream_starts(E):
    """solve_from(4) records a graph without the set-up and without the side stream; it re-solves
    levels 4 and 5 from the kept coarser solutions and lands on the same iterates."""
    p = inputs.cos_cube(levels=6, n0=(8, 8, 8), rtol=1e-10)
    full = _run(E, p, precision=1, use_graph=1)
    again = _run(E, p, first=4, precision=1, use_graph=1)
    assert again[0]["iters"][4:] == full[0]["iters"][4:]
    for l in range(p["levels"]):
        assert np.array_equal(again[1][l], full[1][l]), l
