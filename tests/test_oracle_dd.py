"""Pins for the oracle's domain-decomposition coupling (Sections 3.3-3.5) against the exact
transmission solution of a plane wave normally incident on layers (Appendix A): fourth-order
convergence of the DD solution at receivers inside every layer."""
import numpy as np
import pytest

import workloads as W
from oracle.dd import Strip
from exact_solutions import layered_exact


def run(n, ks, M, ap=W.AP_DIRX_SOMMY, values=False):
    subs = [W.unit_subdomain(j, 0, n, k, ap, M) for j, k in enumerate(ks)]
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
    if values:
        return urec
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


def test_coupled_solution_does_not_depend_on_the_ap_rows():
    """Each subdomain enters the coupled solve through P_gamma, whose range does not depend
    on the AP (P5); only the least-squares residual of a truncated Chebyshev basis still
    weights by P_gamma itself. So with the Sommerfeld rows as printed (second-order) or the
    all-Dirichlet AP instead of the default rows, the receivers differ by an amount that
    vanishes as M* grows (measured: 2e-3 at M* = 8, 6e-10 at M* = 16), down to rounding."""
    ks = [3.0, 5.0, 8.0, 6.0]

    def diff(ap, M):
        ref = run(33, ks, M, values=True)
        other = run(33, ks, M, ap=ap, values=True)
        return max(float(np.abs(a - b).max() / np.abs(a).max()) for a, b in zip(ref, other))

    for ap in (W.AP_DIRX_SOMMY_PAPER, W.AP_DIRICHLET4):
        d8, d16 = diff(ap, 8), diff(ap, 16)
        assert d16 < 1e-8 and d16 < 1e-4 * d8, (ap, d8, d16)
