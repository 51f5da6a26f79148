"""The library's far-field tables (pgb_far_table, host code, no GPU): the
far field they give, sum_p D^p G(r) E_p(R) with E = table . moments, equals
the oracle's truncated Taylor expansion of order P (Section 3.2) summed over
point sources with single- and double-layer strengths, for Laplace and
Yukawa kernels and P = 0..8, 10, 12 and 15 (the paper's Tables 1 and 2)."""
import math

import numpy as np
import pytest

from oracle.treecode import truncated_kernel


def _graded(P):
    return [(x, y, n - x - y) for n in range(P + 1) for x in range(n, -1, -1) for y in range(n - x, -1, -1)]


def _evaluation_order(P):
    return [(a, b, c) for a in range(P + 1) for b in range(P + 1 - a) for c in range(P + 1 - a - b)]


def _moments(P, u, q, p):
    """M_k = sum_s (q_s + p_s . grad_u) u_s^k, u = node centre - source."""
    M = []
    for (a, b, c) in _graded(P):
        mono = u[:, 0] ** a * u[:, 1] ** b * u[:, 2] ** c
        g = np.zeros_like(u)
        if a:
            g[:, 0] = a * u[:, 0] ** (a - 1) * u[:, 1] ** b * u[:, 2] ** c
        if b:
            g[:, 1] = b * u[:, 0] ** a * u[:, 1] ** (b - 1) * u[:, 2] ** c
        if c:
            g[:, 2] = c * u[:, 0] ** a * u[:, 1] ** b * u[:, 2] ** (c - 1)
        M.append(float((q * mono + (p * g).sum(1)).sum()))
    return np.array(M)


def _far(P, kappa, tab, M, R, laplace):
    r2 = float(R @ R)
    r = math.sqrt(r2)
    S = R / r2
    x = kappa * r
    E = tab @ M
    mono = np.array([S[0] ** a * S[1] ** b * S[2] ** c for (a, b, c) in _evaluation_order(P)])
    if laplace:
        return float(E @ mono) / r
    deg = np.array([a + b + c for (a, b, c) in _evaluation_order(P)])
    g = [1.0, -(1.0 + x)]
    for n in range(2, P + 1):
        g.append(x * x * g[n - 2] - (2 * n - 1) * g[n - 1])
    return math.exp(-x) / r * float((E * mono * np.array(g)[deg]).sum())


@pytest.mark.parametrize("P", [0, 1, 2, 4, 6, 8, 10, 12, 15])
@pytest.mark.parametrize("kappa", [0.0, 0.125, 0.9])
def test_far_table_reproduces_truncated_expansion(P, kappa):
    import paper_1506_03745_gb300._lib as L
    Y, Lt = L.pgb_far_table(P, kappa)
    rng = np.random.default_rng(100 * P + int(10 * kappa))
    for trial in range(3):
        ns = 9
        d = rng.normal(size=(ns, 3)) * 0.5          # source - centre
        q = rng.normal(size=ns)
        p = rng.normal(size=(ns, 3))
        R = rng.normal(size=3)
        R *= (2.5 + trial) / np.linalg.norm(R)       # target - centre
        M = _moments(P, -d, q, p)
        for laplace in ((True, False) if kappa == 0 else (False,)):
            F, dF = truncated_kernel(np.tile(R, (ns, 1)), d, p, kappa, P, laplace)
            # the oracle's sum over sources of q F - p . grad_y F, times 4 pi
            ref = 4 * math.pi * (float(q @ F) - float(dF.sum()))
            got = _far(P, kappa, Lt if laplace else Y, M, R, laplace)
            assert got == pytest.approx(ref, rel=1e-12, abs=1e-14)


def test_far_table_argument_errors():
    import ctypes
    import paper_1506_03745_gb300._lib as L
    lib = L.lib()
    buf = (ctypes.c_double * 8)()
    assert lib.pgb_far_table(16, 0.1, buf, 8) == L.PGB_EINVAL
    assert lib.pgb_far_table(9, 0.1, buf, 8) == L.PGB_EINVAL
    assert lib.pgb_far_table(0, -1.0, buf, 2) == L.PGB_EINVAL
    assert lib.pgb_far_table(0, 0.1, buf, 3) == L.PGB_EINVAL
    assert lib.pgb_far_table(0, 0.1, None, 2) == L.PGB_EINVAL
