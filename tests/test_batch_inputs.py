"""The batched workload generator: 64 all-Dirichlet problems with per-axis sizes drawn from
{32, 48, 64, 96, 128} cubic elements of side 1/128, lognormal beta clipped to a contrast of
1e2, f ~ U[-1, 1] per node, and the coarsest-grid rule (halve while all axes are even and stay
>= 4). Host-side checks only."""
import numpy as np

from paper_1506_02983_gb300 import inputs


def test_coarsest_split_rule():
    assert inputs.coarsest_split((32, 48, 128)) == ([4, 6, 16], 4)
    assert inputs.coarsest_split((48, 48, 48)) == ([6, 6, 6], 4)
    assert inputs.coarsest_split((96, 32, 64)) == ([12, 4, 8], 4)
    assert inputs.coarsest_split((128, 128, 128)) == ([4, 4, 4], 6)
    assert inputs.coarsest_split((64, 64, 32)) == ([8, 8, 4], 4)


def test_batch_problems_shape_and_statistics():
    ps = inputs.batch_problems()
    assert len(ps) == 64
    sizes = {32, 48, 64, 96, 128}
    seen = set()
    for p in ps:
        N = inputs.finest(p["n0"], p["levels"])
        assert all(v in sizes for v in N)
        seen.update(N)
        assert p["levels"] >= 3
        assert all(v >= 4 for v in p["n0"])
        assert np.allclose(p["hi"], [v / 128.0 for v in N])
        assert p["beta"].shape == (N[2], N[1], N[0])
        assert p["f"].shape == (N[2] + 1, N[1] + 1, N[0] + 1)
        assert p["beta"].min() >= 0.1 - 1e-15 and p["beta"].max() <= 10.0 + 1e-12
        assert np.abs(p["f"]).max() <= 1.0
        assert p["face_bc"] == [0] * 6 and p["gD"] is None
    assert seen == sizes
    allb = np.log(np.concatenate([p["beta"].ravel() for p in ps]))
    # lognormal with sigma 1 clipped at +-ln 10: mean ~0, std a little below 1, both clips hit
    assert abs(allb.mean()) < 0.01 and 0.9 < allb.std() < 1.0
    assert np.isclose(allb.max(), np.log(10.0)) and np.isclose(allb.min(), -np.log(10.0))


def test_batch_problems_are_seeded():
    a = inputs.batch_problems(count=3)
    b = inputs.batch_problems(count=3)
    c = inputs.batch_problems(count=3, seed=7)
    assert all(np.array_equal(x["beta"], y["beta"]) and np.array_equal(x["f"], y["f"]) for x, y in zip(a, b))
    assert not np.array_equal(a[0]["f"].ravel()[:10], c[0]["f"].ravel()[:10]) or a[0]["n0"] != c[0]["n0"]
