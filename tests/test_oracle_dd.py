"""Pins for the oracle's domain-decomposition coupling (Sections 3.3-3.5) against the exact
transmission solution of a plane wave normally incident on layers (Appendix A): fourth-order
convergence of the DD solution at receivers inside every layer."""
import numpy as np
import pytest

import workloads as W
from oracle.dd import Strip


def layered_exact(ks, x_if):
    """u_j(x) = A_j e^{i k_j x} + B_j e^{-i k_j x} with A_0 = 1 (incident), B_last = 0 (outgoing),
    continuity of u and du/dx at the interfaces x_if (Appendix A, N-layer system)."""
    n = len(ks)
    # unknowns: B_0, (A_j, B_j) for j = 1..n-2, A_{n-1}
    nu = 2 * n - 2
    M = np.zeros((nu, nu), complex)
    rhs = np.zeros(nu, complex)

    def col(j, which):  # which 0: A, 1: B
        if j == 0:
            return None if which == 0 else 0
        if j == n - 1:
            return None if which == 1 else nu - 1
        return 1 + 2 * (j - 1) + which

    for i, x in enumerate(x_if):  # interface between layer i and i+1
        for eq, der in ((2 * i, 0), (2 * i + 1, 1)):
            for j, sgn in ((i, 1.0), (i + 1, -1.0)):
                for which, e in ((0, 1.0), (1, -1.0)):
                    f = np.exp(1j * e * ks[j] * x) * ((1j * e * ks[j]) if der else 1.0)
                    c = col(j, which)
                    if c is None:
                        if j == 0 and which == 0:      # A_0 = 1 known
                            rhs[eq] -= sgn * f
                    else:
                        M[eq, c] += sgn * f
    sol = np.linalg.solve(M, rhs)
    A = [1.0 + 0j] + [sol[col(j, 0)] for j in range(1, n)]
    B = [sol[col(j, 1)] for j in range(n - 1)] + [0.0 + 0j]

    def u(j, x):
        return A[j] * np.exp(1j * ks[j] * x) + B[j] * np.exp(-1j * ks[j] * x)

    def du(j, x):
        return 1j * ks[j] * (A[j] * np.exp(1j * ks[j] * x) - B[j] * np.exp(-1j * ks[j] * x))

    return u, du


def run(n, ks, M):
    subs = [W.unit_subdomain(j, 0, n, k, W.AP_DIRX_SOMMY, M) for j, k in enumerate(ks)]
    u, du = layered_exact(ks, [float(j) for j in range(1, len(ks))])

    def bc(j, side):
        s_ = subs[j]
        if side in (1, 2):          # du/dn = 0 on the horizontal sides (u independent of y)
            return 0.0, 1.0, lambda s: np.zeros_like(s, dtype=complex)
        x = s_.x0 if side == 3 else s_.x1
        sign = -1.0 if side == 3 else 1.0   # outward normal -x on the left, +x on the right
        ik = 1j * ks[j]
        return ik, 1.0, lambda s: np.full(s.shape, sign * du(j, x) + ik * u(j, x))

    strip = Strip(subs, bc)
    rows = []
    for s_ in subs:
        y = s_.ay0 + np.arange(s_.ny) * s_.h
        rows.append(int(np.argmin(np.abs(y - 0.5))))
    _, urec, _ = strip.solve(rows)
    err = 0.0
    for j, (s_, r) in enumerate(zip(subs, rows)):
        x = s_.ax0 + np.arange(s_.nx) * s_.h
        from oracle.projection import APSystem
        mlo, mhi, _, _ = APSystem(s_).mplus_range()
        ex = u(j, x[mlo + 1:mhi])
        err = max(err, np.abs(urec[j] - ex).max() / np.abs(ex).max())
    return err


@pytest.mark.slow
def test_two_layer_transmission_converges_fourth_order():
    errs = [run(n, [5.0, 9.0], 16) for n in (33, 65, 129)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-4 and np.all(rates > 3.4), (errs, rates)


def test_four_layer_transmission_is_accurate():
    err = run(65, [3.0, 5.0, 8.0, 6.0], 12)
    assert err < 2e-3, err
