"""The FP64 elementary functions of the near-field sums (one- and two-step
Newton reciprocal square root on the SFU estimate, Taylor 2^x) against their
error bounds, with NumPy's FP64 functions and CUDA's library forms as
references."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1506_03745_gb300 as pgb  # noqa: E402


def test_newton_rsqrt_error_bounds():
    rng = np.random.default_rng(11)
    x = np.concatenate([10.0 ** rng.uniform(-12, 12, 200000), [1.0, 2.0, 4.0, 0.25, 3.0, 1e-12, 1e12]])
    out = pgb.pgb_math_check(x)
    ref = 1.0 / np.sqrt(x)
    e1 = np.abs(out[:, 0] / ref - 1).max()
    e2 = np.abs(out[:, 1] / ref - 1).max()
    elib = np.abs(out[:, 3] / ref - 1).max()
    # one step: 1.5 d^2 with d < 2^-22 of the SFU estimate
    assert e1 < 2e-13
    assert e2 < 4e-16
    assert elib < 4e-16


def test_taylor_exp2_error_bounds():
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.uniform(-60, 0, 200000), rng.uniform(-1020, 1000, 50000),
                        np.arange(-40, 41) * 0.5, [0.0, -0.0, 1e-300, -1e-300, -1020.0]])
    out = pgb.pgb_math_check(x)
    ref = np.exp2(x)
    err = np.abs(out[:, 2] / ref - 1).max()
    elib = np.abs(out[:, 4] / ref - 1).max()
    assert err < 2e-14
    assert elib < 4e-16
    # integers are exact
    k = np.arange(-1020, 1001).astype(np.float64)
    assert np.array_equal(pgb.pgb_math_check(k)[:, 2], np.exp2(k))
    # below 2^-1020 the result is 0
    tiny = np.array([-1021.0, -1100.0, -5000.0, -1e6])
    assert np.all(pgb.pgb_math_check(tiny)[:, 2] == 0.0)
