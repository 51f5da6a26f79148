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


def test_double_single_rsqrt_and_exp2():
    """The double-single forms of the PGB_FP64_DS product: rsqrt by one Newton
    step on the SFU estimate (about 1.5 d^2 with d < 2^-22.9, plus the ~2^-47
    rounding of the pair), 2^x by the split Taylor series (truncation below
    2e-16, FP32 tail below 1e-14, rounding of seven double-single steps)."""
    rng = np.random.default_rng(13)
    x = np.concatenate([10.0 ** rng.uniform(-20, 20, 200000), [1.0, 2.0, 4.0, 0.25, 3.0]])
    out = pgb.pgb_math_check(x)
    assert np.abs(out[:, 5] * np.sqrt(x) - 1).max() < 1e-13
    t = np.concatenate([rng.uniform(-60, 0, 200000), rng.uniform(-100, 126, 50000), np.arange(-40, 41) * 0.5,
                        [0.0, 1e-30, -1e-30]])
    out = pgb.pgb_math_check(t)
    # beyond the method's own error, the argument held to 48 bits moves 2^t
    # by up to |t| ln 2 2^-48 (relative)
    err = np.abs(out[:, 6] / np.exp2(t) - 1)
    assert np.all(err < 3e-14 + 5e-15 * np.abs(t)), err.max()
    assert err[np.abs(t) <= 4].max() < 3e-14
    # integers are exact
    k = np.arange(-100, 127).astype(np.float64)
    assert np.array_equal(pgb.pgb_math_check(k)[:, 6], np.exp2(k))
