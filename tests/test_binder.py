"""Binder ratio: the estimator on series with closed-form answers (CPU), and
the batched temperature sweep against exact enumeration (GPU)."""
import math

import numpy as np
import pytest

from paper_1110_0899_gb300.binder import binder_from_series, crossing


def test_binder_closed_forms():
    rng = np.random.default_rng(3)
    # Gaussian magnetisation (high T): <M^4> = 3 <M^2>^2, U -> 0
    U, err = binder_from_series(rng.normal(size=400_000) * 37.0)
    assert abs(U) < 4 * err + 1e-3 and err < 0.01
    # two-valued +-M (ordered): <M^4> = <M^2>^2, U = 2/3 exactly
    U, err = binder_from_series(np.where(rng.uniform(size=10_000) < 0.5, -9.0, 9.0))
    assert abs(U - 2.0 / 3.0) < 1e-12 and err < 1e-12
    # uniform on [-1, 1]: <M^2> = 1/3, <M^4> = 1/5, U = 1 - (1/5)/(3/9) = 2/5
    U, err = binder_from_series(rng.uniform(-1, 1, size=400_000))
    assert abs(U - 0.4) < 4 * err + 1e-3


def test_crossing_interpolates():
    # U(8) - U(16) = -0.15 + 0.1 T: zero at T = 1.5
    pts = [{"L": 8, "T": t, "U": 0.6 - 0.1 * t} for t in (1.0, 2.0, 3.0)]
    pts += [{"L": 16, "T": t, "U": 0.75 - 0.2 * t} for t in (1.0, 2.0, 3.0)]
    assert abs(crossing(pts, 8, 16) - 1.5) < 1e-12
    # U(8) - U(16) = -0.25 + 0.1 T after a shift: zero at T = 2.5
    pts2 = [dict(p, U=p["U"] - (0.1 if p["L"] == 8 else 0.0)) for p in pts]
    assert abs(crossing(pts2, 8, 16) - 2.5) < 1e-12
    assert crossing([dict(p, U=p["U"] + (1.0 if p["L"] == 8 else 0.0)) for p in pts], 8, 16) is None


@pytest.mark.gpu
def test_sweep_matches_exact_enumeration():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1110_0899_gb300 import binder
    tc = 2.0 / math.log(1.0 + math.sqrt(2.0))
    Ts = [1.5, tc, 3.5]
    pts = binder.sweep(2, [4], Ts, discard=500, measure=200_000, chunk=50_000)
    g = oracle.density_of_states(2, 4)[0]
    for p in pts:
        ex = oracle.exact_moments(2, 4, 1.0, p["T"], g)
        U_exact = 1.0 - ex["M4"] / (3.0 * ex["M2"] ** 2)
        assert abs(p["U"] - U_exact) < 3.0 * p["U_err"] + 1e-9, (p, U_exact)
    pts3 = binder.sweep(3, [2], [4.5115], discard=500, measure=200_000, chunk=50_000)
    ex = oracle.exact_moments(3, 2, 1.0, 4.5115)
    U_exact = 1.0 - ex["M4"] / (3.0 * ex["M2"] ** 2)
    assert abs(pts3[0]["U"] - U_exact) < 3.0 * pts3[0]["U_err"] + 1e-9
