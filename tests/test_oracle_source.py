"""Pins for the oracle's inhomogeneous terms (oracle/source.py): B^(h) on a plane wave in closed
form; the full extension Ex^(H) + Ex^(I) of a manufactured solution reproduces it at gamma to
fifth order; the inhomogeneous BEP residual of exact data vanishes at fourth order; the strip
DD with a source converges at fourth order to the manufactured solution."""
import numpy as np
import pytest

import workloads as W
from oracle.dd import Strip, side_points
from oracle.extension import extend_data
from oracle.projection import APSystem
from oracle.source import apply_B, source_foot_data, source_on_grid, source_terms

AL, BE = 3.0, 2.0   # manufactured solution u = exp(i (AL x + BE y)), f = (k^2 - AL^2 - BE^2) u


def plane(k):
    def fun(x, y):
        u = np.exp(1j * (AL * x + BE * y))
        f = (k**2 - AL**2 - BE**2) * u
        return f, 1j * AL * f, 1j * BE * f, -AL**2 * f, -BE**2 * f
    return fun


def u_exact(x, y):
    return np.exp(1j * (AL * x + BE * y))


def test_B_of_a_plane_wave_is_the_closed_form():
    sub = W.small_subdomain(33, 7.0, W.AP_DIRX_SOMMY, 2)
    f = source_on_grid(sub, plane(7.0))
    g = apply_B(f)
    h = sub.h
    factor = 1.0 + (2 * np.cos(AL * h) + 2 * np.cos(BE * h) - 4.0) / 12.0
    assert np.abs(g[1:-1, 1:-1] - factor * f[1:-1, 1:-1]).max() < 1e-14 * np.abs(f).max()
    assert np.all(g[0] == 0) and np.all(g[-1] == 0) and np.all(g[:, 0] == 0) and np.all(g[:, -1] == 0)


def exact_density(S, sub, k):
    """Ex^(H)(u, d_n u) + Ex^(I) f for the manufactured solution."""
    def data(side, s, L):
        x, y = side_points(sub, side, s)
        u = u_exact(x, y)
        if side in (1, 2):
            t2, nrm = -AL**2, (-1.0 if side == 1 else 1.0) * 1j * BE
        else:
            t2, nrm = -BE**2, (-1.0 if side == 3 else 1.0) * 1j * AL
        return u, t2 * u, t2 * t2 * u, nrm * u, t2 * nrm * u
    from oracle.source import extend_source
    return extend_data(S.gs, k, data) + extend_source(S.gs, k, source_foot_data(S.gs, sub, plane(k)))


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
def test_full_extension_is_fifth_order_and_the_bep_residual_fourth(ap):
    errs, res = [], []
    k = 7.0
    for n in (33, 65):
        sub = W.small_subdomain(n, k, ap, 2)
        S = APSystem(sub)
        xi = exact_density(S, sub, k)
        x = sub.ax0 + S.gs.gamma_m * sub.h
        y = sub.ay0 + S.gs.gamma_n * sub.h
        errs.append(np.abs(xi - u_exact(x, y)).max())
        F, _ = source_terms(S, source_on_grid(sub, plane(k)), source_foot_data(S.gs, sub, plane(k)))
        # Q xi_H = F for the homogeneous part xi_H = xi - Ex^(I) f: (P - I) xi + Tr G B f = 0
        ub = S.solve(np.where(S.gs.Mp, apply_B(source_on_grid(sub, plane(k))), 0.0))
        res.append(np.abs(S.apply(xi, kind="Q") + S.trace(ub)).max())
        assert np.isfinite(F).all()
    assert np.log2(errs[0] / errs[1]) > 4.5, errs
    assert np.log2(res[0] / res[1]) > 3.5, res


def run_strip(n, ks, M):
    subs = [W.unit_subdomain(j, 0, n, k, W.AP_DIRX_SOMMY, M) for j, k in enumerate(ks)]

    def bc(j, side):
        ik = 1j * ks[j]

        def phi(s, side=side, j=j):
            x, y = side_points(subs[j], side, s)
            u = u_exact(x, y)
            dn = {1: -1j * BE, 2: 1j * BE, 3: -1j * AL, 4: 1j * AL}[side] * u
            return dn + ik * u
        return ik, 1.0, phi

    strip = Strip(subs, bc, source=lambda j: plane(ks[j]))
    rows = [n // 2] * len(subs)
    _, urec, _ = strip.solve(rows)
    err = 0.0
    for s_, r, ur in zip(subs, rows, urec):
        S = APSystem(s_)
        mlo, mhi, _, _ = S.mplus_range()
        x = s_.ax0 + np.arange(mlo + 1, mhi) * s_.h
        y = s_.ay0 + r * s_.h
        ex = u_exact(x, y)
        err = max(err, np.abs(ur - ex).max() / np.abs(ex).max())
    return err


def test_strip_with_a_source_converges_fourth_order():
    errs = [run_strip(n, [5.0, 8.0], 12) for n in (33, 65)]
    rate = np.log2(errs[0] / errs[1])
    assert errs[1] < 2e-4 and rate > 3.4, (errs, rate)


def run_layout(n_of, ks, M):
    """2 x 2 layout (subdomain (i, j) -> index 2 j + i) with per-subdomain k and grid size."""
    pos = [(i, j) for j in range(2) for i in range(2)]
    subs = [W.unit_subdomain(i, j, n_of[2 * j + i], ks[2 * j + i], W.AP_DIRX_SOMMY, M) for (i, j) in pos]

    def bc(j, side):
        ik = 1j * ks[j]

        def phi(s, side=side, j=j):
            x, y = side_points(subs[j], side, s)
            u = u_exact(x, y)
            dn = {1: -1j * BE, 2: 1j * BE, 3: -1j * AL, 4: 1j * AL}[side] * u
            return dn + ik * u
        return ik, 1.0, phi

    strip = Strip(subs, bc, source=lambda j: plane(ks[j]), positions=pos)
    rows = [s_.ny // 2 for s_ in subs]
    _, urec, _ = strip.solve(rows)
    err = 0.0
    for s_, r, ur in zip(subs, rows, urec):
        mlo, mhi, _, _ = APSystem(s_).mplus_range()
        ex = u_exact(s_.ax0 + np.arange(mlo + 1, mhi) * s_.h, s_.ay0 + r * s_.h)
        err = max(err, np.abs(ur - ex).max() / np.abs(ex).max())
    return err


def test_two_by_two_checkerboard_with_mixed_grids_converges_fourth_order():
    """A 2 x 2 layout (interfaces along x and y, a corner shared by four subdomains) with a
    checkerboard wavenumber and a finer grid on the high-k subdomains (Section 4's checkerboard
    setting, scaled down), sources making u = exp(i (3x + 2y)) exact: fourth order."""
    ks = [4.0, 7.0, 7.0, 4.0]
    errs = [run_layout([n, 2 * n - 1, 2 * n - 1, n], ks, 12) for n in (17, 33)]
    rate = np.log2(errs[0] / errs[1])
    assert rate > 3.4 and errs[1] < 1e-4, (errs, rate)
