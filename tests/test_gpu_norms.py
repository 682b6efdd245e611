"""GPU parity of the error norms of Sec. 5 (max |a - b| and the root mean square over all nodes)
computed by ecmg_error_norms, against the oracle's or_norms and numpy on the same vectors.

The vectors are real level vectors of a ragged hierarchy (node rows that do not fill the padded
pitch of the device layout), with b given and b = NULL; the max must agree exactly (a max does
not depend on the order of the reduction) and the RMS to 1e-12 relative. A NaN anywhere in
a - b must make both norms NaN."""
import math

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
    return t.detach().cpu().numpy().ravel()


@pytest.mark.parametrize("precision", [0, 1])
def test_error_norms_match_oracle_on_every_level_of_a_ragged_hierarchy(E, oracle_mod, precision):
    p = inputs.random_problem(7, n0=(3, 5, 2), levels=4)
    s = E.solver_from_problem(p, precision=precision)
    s.solve()
    for l in range(p["levels"]):
        U, B = s.get(E.ECMG_VEC_U, l), s.get(E.ECMG_VEC_B, l)
        pairs = [(U, None), (U, B), (B, U)]
        if l >= 2:
            pairs.append((s.get(E.ECMG_VEC_W, l), U))
            pairs.append((s.get(E.ECMG_VEC_UTILDE, l), U))
        for a, b in pairs:
            want = oracle_mod.norms(_np(a), None if b is None else _np(b))
            got = s.norms(a, b, level=l)
            assert got[0] == want[0], (l, got, want)
            assert got[1] == pytest.approx(want[1], rel=1e-12, abs=0.0), (l, got, want)
            d = _np(a) - (0.0 if b is None else _np(b))
            assert got[0] == np.abs(d).max()
            assert got[1] == pytest.approx(math.sqrt(np.mean(d * d)), rel=1e-12)
    s.close()


def test_error_norms_of_the_exact_solution_error(E, oracle_mod):
    """||U - u||: the quantity the tables of Sec. 5 print, on config 1's problem."""
    import torch
    p = inputs.exp_cube(levels=4, rtol=1e-10)
    s = E.solver_from_problem(p)
    s.solve()
    U = s.get(E.ECMG_VEC_U)
    ue = torch.tensor(np.asarray(p["u_exact"]), device="cuda")
    want = oracle_mod.norms(_np(U), np.asarray(p["u_exact"]).ravel())
    got = s.norms(U, ue)
    assert got[0] == want[0]
    assert got[1] == pytest.approx(want[1], rel=1e-12)
    s.close()


@pytest.mark.parametrize("where", ["first", "middle", "last"])
def test_a_nan_in_the_difference_makes_both_norms_nan(E, where):
    p = inputs.exp_cube(levels=3, rtol=1e-10)
    s = E.solver_from_problem(p)
    s.solve()
    U = s.get(E.ECMG_VEC_U)
    a = U.clone().view(-1)
    k = {"first": 0, "middle": a.numel() // 2, "last": a.numel() - 1}[where]
    a[k] = float("nan")
    a = a.view(U.shape)
    for args in ((a, None), (a, U), (U, a)):
        mx, rms = s.norms(*args)
        assert math.isnan(mx) and math.isnan(rms), (where, mx, rms)
    # a large finite difference elsewhere does not hide the NaN
    b = U.clone().view(-1)
    b[(k + 1) % b.numel()] += 1e300
    mx, _ = s.norms(a, b.view(U.shape))
    assert math.isnan(mx)
    # and the same vectors without the NaN give finite norms again
    mx, rms = s.norms(U, U)
    assert mx == 0.0 and rms == 0.0
    s.close()
