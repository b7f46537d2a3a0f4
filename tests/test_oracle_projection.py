"""Pins for the oracle's extension, basis, P_gamma, Q columns and adjoint
(Sections 3.2.2-3.2.5) against closed forms, invariants and convergence orders."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as C

import workloads as W
from oracle.extension import basis_column, extend_data, chebyshev_derivs
from oracle.grid import grid_sets, node_coordinates
from oracle.projection import APSystem
from test_oracle_scheme import discrete_plane_wave


def plane_wave_data(k, t, sub):
    """Cauchy data of u = exp(i k (x cos t + y sin t)) on the four sides of the unit
    square, as (xi0, xi0'', xi0'''', xi1, xi1'') in arc length (outward normals)."""
    kx, ky = k * np.cos(t), k * np.sin(t)

    def data(side, s, L):
        if side in (1, 2):
            x = sub.x0 + (s + 1) / 2 * L
            y = np.full_like(s, sub.y0 if side == 1 else sub.y1)
            kt = kx
            dn = -1j * ky if side == 1 else 1j * ky
        else:
            y = sub.y0 + (s + 1) / 2 * L
            x = np.full_like(s, sub.x0 if side == 3 else sub.x1)
            kt = ky
            dn = -1j * kx if side == 3 else 1j * kx
        u = np.exp(1j * (kx * x + ky * y))
        return u, -kt**2 * u, kt**4 * u, dn * u, -kt**2 * dn * u

    def exact(x, y):
        return np.exp(1j * (kx * x + ky * y))

    return data, exact


def test_chebyshev_basis_closed_forms():
    """T_n(cos th) = cos(n th); T_n''(1) = n^2(n^2-1)/3; T_n''''(1) = n^2(n^2-1)(n^2-4)(n^2-9)/105;
    T_n(+-1) parity; extrapolation T_n(cosh a) = cosh(n a)."""
    th = np.linspace(0, np.pi, 7)
    for n in (0, 1, 2, 5, 15, 63):
        t0, t2, t4 = chebyshev_derivs(n + 1, np.cos(th), 2.0)   # L = 2: no scaling
        np.testing.assert_allclose(t0, np.cos(n * th), atol=1e-13)
        t0, t2, t4 = chebyshev_derivs(n + 1, np.array([1.0, -1.0]), 2.0)
        n2 = n * n
        np.testing.assert_allclose(t2, [n2 * (n2 - 1) / 3, (-1) ** n * n2 * (n2 - 1) / 3], rtol=1e-12)
        d4 = n2 * (n2 - 1) * (n2 - 4) * (n2 - 9) / 105
        np.testing.assert_allclose(t4, [d4, (-1) ** n * d4], rtol=1e-11, atol=1e-9)
        a = 0.01
        t0, _, _ = chebyshev_derivs(n + 1, np.array([np.cosh(a)]), 2.0)
        np.testing.assert_allclose(t0, np.cosh(n * a), rtol=1e-12)
    # arc-length scaling: L = 1 multiplies the p-th derivative by 2^p
    _, t2a, t4a = chebyshev_derivs(8, np.array([0.3]), 2.0)
    _, t2b, t4b = chebyshev_derivs(8, np.array([0.3]), 1.0)
    np.testing.assert_allclose([t2b[0], t4b[0]], [4 * t2a[0], 16 * t4a[0]], rtol=1e-14)


def test_extension_of_normal_wave_is_taylor_polynomial():
    """P7 closed form: for u = exp(i k x) the right side carries xi0 = e^{ik}, xi1 = ik e^{ik}
    and no tangential variation, so Ex gives e^{ik} sum_{p<=4} (i k rho)^p / p! exactly."""
    sub = W.small_subdomain(65, 7.0, W.AP_DIRX_SOMMY, 4)
    gs = grid_sets(sub)
    k = sub.k

    def data(side, s, L):
        z = np.zeros_like(s, dtype=complex)
        if side != 4:
            return z, z, z, z, z
        e = np.exp(1j * k) + z
        return e, z, z, 1j * k * e, z

    v = extend_data(gs, k, data)
    sel = gs.owner == 4
    ikr = 1j * k * gs.rho[sel]
    taylor = np.exp(1j * k) * (1 + ikr + ikr**2 / 2 + ikr**3 / 6 + ikr**4 / 24)
    np.testing.assert_allclose(v[sel], taylor, atol=1e-15, rtol=1e-14)
    assert np.all(v[~sel] == 0)


def test_extension_is_fifth_order_at_gamma():
    """P7: for a plane wave the extension error at gamma is O(h^5) (Section 3.2.3)."""
    errs = []
    for n in (65, 129, 257, 513):
        sub = W.small_subdomain(n, 10.0, W.AP_DIRX_SOMMY, 4)
        gs = grid_sets(sub)
        data, exact = plane_wave_data(10.0, 0.3, sub)
        x, y = node_coordinates(sub)
        v = extend_data(gs, 10.0, data)
        errs.append(np.abs(v - exact(x[gs.gamma_m], y[gs.gamma_n])).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 4.6), rates


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
@pytest.mark.parametrize("n,k", [(33, 3.0), (129, 10.0), (257, 30.0)])
def test_homogeneous_bep_for_discrete_plane_wave(ap, n, k):
    """P3: the trace of an exact discrete solution satisfies P_gamma xi = xi (Eq.
    discrete_BEP_homo), so its Q-type residual is round-off."""
    sub = W.small_subdomain(n, k, ap, 4)
    S = APSystem(sub)
    v = discrete_plane_wave(sub, 0.3)
    xi = S.trace(v)
    assert np.abs(S.apply(xi, "Q")).max() < 1e-11 * np.abs(xi).max()
    # and the difference potential reproduces the wave on N+ (Eq. potential_solution_homo)
    pot = S.potential(xi)
    Np = S.gs.Np
    assert np.abs(pot[Np] - v[Np]).max() < 1e-11


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY, W.AP_DIRX_SOMMY_PAPER])
@pytest.mark.parametrize("n", [17, 33])
def test_pgamma_is_a_projection(ap, n):
    """P4: P_gamma^2 = P_gamma (Section 3.2.2)."""
    S = APSystem(W.small_subdomain(n, 4.0, ap, 4))
    P = S.pgamma_matrix()
    assert np.abs(P @ P - P).max() < 1e-10 * np.abs(P).max()
    assert np.abs(P - np.eye(P.shape[0])).max() > 0.1  # not the identity


@pytest.mark.parametrize("aps", [(W.AP_DIRICHLET4, W.AP_DIRX_SOMMY), (W.AP_DIRICHLET4, W.AP_DIRX_SOMMY_PAPER),
                                 (W.AP_DIRX_SOMMY, W.AP_DIRX_SOMMY_PAPER)])
@pytest.mark.parametrize("n", [17, 33])
def test_range_is_independent_of_the_auxiliary_problem(n, aps):
    """P5: only the range of P_gamma (traces of discrete solutions) is AP-independent,
    so P_a P_b = P_b and P_b P_a = P_a for any two APs -- including the Sommerfeld rows as
    printed in the paper, which are only second-order accurate."""
    Pd = APSystem(W.small_subdomain(n, 4.0, aps[0], 4)).pgamma_matrix()
    Ps = APSystem(W.small_subdomain(n, 4.0, aps[1], 4)).pgamma_matrix()
    scale = max(np.abs(Pd).max(), np.abs(Ps).max())
    assert np.abs(Pd @ Ps - Ps).max() < 1e-9 * scale
    assert np.abs(Ps @ Pd - Pd).max() < 1e-9 * scale
    assert np.abs(Pd - Ps).max() > 1e-3 * scale  # the projections themselves differ


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY, W.AP_DIRX_SOMMY_PAPER])
def test_continuous_bep_residual_is_fourth_order(ap):
    """P6: for the Cauchy data of a plane wave, (P_gamma - I) Ex(u, du/dn) = O(h^4), whatever
    the AP's boundary rows (the residual depends on the range of P_gamma only)."""
    errs = []
    for n in (65, 129, 257):
        sub = W.small_subdomain(n, 10.0, ap, 4)
        S = APSystem(sub)
        data, _ = plane_wave_data(10.0, 0.3, sub)
        errs.append(np.abs(S.apply(extend_data(S.gs, 10.0, data), "Q")).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.5), (errs, rates)


def test_basis_columns_expand_the_boundary_data():
    """Column order, side order, s orientation and (2/L)^p scaling: the Chebyshev
    interpolants of the plane-wave data on each side, expanded in the basis columns
    (Eqs. boundary_finite_gamma, extension_xiG), reproduce Ex of the exact data."""
    M = 24
    sub = W.small_subdomain(129, 10.0, W.AP_DIRX_SOMMY, M)
    gs = grid_sets(sub)
    data, _ = plane_wave_data(10.0, 0.3, sub)
    xi = np.zeros(gs.owner.size, dtype=complex)
    for kind in (0, 1):
        for side in (1, 2, 3, 4):
            f = lambda s: data(side, s, 1.0)[0 if kind == 0 else 3]
            c = C.chebinterpolate(lambda s: f(s).real, M - 1) + 1j * C.chebinterpolate(lambda s: f(s).imag, M - 1)
            for j in range(M):
                xi += c[j] * basis_column(gs, 10.0, M, kind * 4 * M + (side - 1) * M + j)
    ref = extend_data(gs, 10.0, data)
    assert np.abs(xi - ref).max() < 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
def test_adjoint_dot_product(ap):
    """P9: <c, Q xi> = <Q^H c, xi> for random complex densities and cotangents."""
    S = APSystem(W.small_subdomain(33, 6.0, ap, 4))
    ng = S.n_gamma
    xi = W.random_complex((3, ng), seed=2)
    c = W.random_complex((3, ng), seed=3)
    for kind in ("Q", "P"):
        out = S.columns(xi=xi, kind=kind)
        gx, _ = S.adjoint(c, kind=kind, xi=xi)
        lhs = np.vdot(c, out)
        rhs = np.vdot(gx, xi)
        assert abs(lhs - rhs) < 1e-10 * abs(lhs)


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
@pytest.mark.parametrize("kind", ["Q", "P"])
@pytest.mark.parametrize("basis", [True, False])
def test_wavenumber_gradient_matches_central_differences(ap, kind, basis):
    """P9: dLoss/dk from the adjoint equals central finite differences of the forward
    map for Loss = Re sum_b <c_b, out_b(k)> (basis columns carry Ex's own k-dependence)."""
    sub = W.small_subdomain(33, 6.0, ap, 3)
    cols = [0, 4, 13, 22]
    ng = APSystem(sub).n_gamma
    c = W.random_complex((len(cols), ng), seed=4)
    xi = None if basis else W.random_complex((len(cols), ng), seed=5)

    def loss(k):
        S = APSystem(sub.with_k(k))
        out = S.columns(cols=cols, kind=kind) if basis else S.columns(xi=xi, kind=kind)
        return np.real(np.vdot(c, out))

    _, gk = APSystem(sub).adjoint(c, kind=kind, xi=xi, cols=cols)
    d = 1e-4 * sub.k   # fourth-order central difference (the loss is curved near resonances)
    fd = (8 * (loss(sub.k + d) - loss(sub.k - d)) - (loss(sub.k + 2 * d) - loss(sub.k - 2 * d))) / (12 * d)
    assert abs(gk - fd) < 1e-6 * max(abs(fd), 1e-30), (gk, fd)


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
def test_receivers_reproduce_a_discrete_plane_wave(ap):
    """Receiver rows (Eq. potential_solution_homo at interior nodes): for the trace of an exact
    discrete solution v, the difference potential at the receiver nodes (row, m), m = mlo+1 ..
    mhi-1, is v there -- which pins the receiver index range against a closed form -- and those
    nodes are exactly the nodes of M+ in that row that are not on gamma."""
    sub = W.small_subdomain(33, 6.0, ap, 4)
    S = APSystem(sub)
    v = discrete_plane_wave(sub, 0.3)
    mlo, mhi, nlo, nhi = S.mplus_range()
    on_gamma = np.zeros_like(S.gs.Mp)
    on_gamma[S.gs.gamma_n, S.gs.gamma_m] = True
    for row in (nlo + 1, (nlo + nhi) // 2, nhi - 1):
        rec = S.receivers(row, xi=[S.trace(v)])[0]
        want = np.nonzero(S.gs.Mp[row] & ~on_gamma[row])[0]
        np.testing.assert_array_equal(want, np.arange(mlo + 1, mhi))
        assert np.abs(rec - v[row, want]).max() < 1e-11 * np.abs(v).max()


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
@pytest.mark.parametrize("kind", ["Q", "P"])
def test_receiver_adjoint_dot_product(ap, kind):
    """P9 with a receiver cotangent: <c, out(xi)> + <c_rec, receivers(xi)> = <grad_xi, xi>, and
    with the gamma cotangent zero, <c_rec, receivers(xi)> = <grad_xi, xi> alone (the receiver
    term R_rec^T c_rec of the adjoint right-hand side is the transpose of the forward gather)."""
    S = APSystem(W.small_subdomain(33, 6.0, ap, 4))
    ng = S.n_gamma
    _, _, nlo, nhi = S.mplus_range()
    row = (nlo + nhi) // 2 + 1
    xi = W.random_complex((3, ng), seed=12)
    c = W.random_complex((3, ng), seed=13)
    rec = S.receivers(row, xi=xi)
    c_rec = W.random_complex(rec.shape, seed=14)
    out = S.columns(xi=xi, kind=kind)
    gx, _ = S.adjoint(c, kind=kind, xi=xi, cot_rec=c_rec, rec_row=row)
    lhs = np.vdot(c, out) + np.vdot(c_rec, rec)
    assert abs(lhs - np.vdot(gx, xi)) < 1e-10 * abs(lhs)
    gx0, _ = S.adjoint(np.zeros_like(c), kind="Q", xi=xi, cot_rec=c_rec, rec_row=row)
    lhs0 = np.vdot(c_rec, rec)
    assert abs(lhs0 - np.vdot(gx0, xi)) < 1e-10 * abs(lhs0)


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
@pytest.mark.parametrize("basis", [True, False])
def test_receiver_wavenumber_gradient_matches_central_differences(ap, basis):
    """P9 with a receiver cotangent: dLoss/dk of Loss = Re <c_rec, receivers(k)> (the gamma
    cotangent zero, and then both together) from the adjoint equals a fourth-order central
    difference of the forward receivers in k; basis columns carry Ex's own k-dependence."""
    sub = W.small_subdomain(33, 6.0, ap, 3)
    S0 = APSystem(sub)
    _, _, nlo, nhi = S0.mplus_range()
    row = nlo + 3
    cols = [0, 5, 14, 23]
    ng = S0.n_gamma
    xi = None if basis else W.random_complex((len(cols), ng), seed=15)
    npx = S0.receivers(row, cols=[0]).shape[1]
    c_rec = W.random_complex((len(cols), npx), seed=16)
    c = W.random_complex((len(cols), ng), seed=17)

    def loss(k, with_gamma):
        S = APSystem(sub.with_k(k))
        rec = S.receivers(row, cols=cols) if basis else S.receivers(row, xi=xi)
        val = np.real(np.vdot(c_rec, rec))
        if with_gamma:
            out = S.columns(cols=cols) if basis else S.columns(xi=xi)
            val += np.real(np.vdot(c, out))
        return val

    d = 1e-4 * sub.k
    for with_gamma in (False, True):
        cot = c if with_gamma else np.zeros_like(c)
        _, gk = S0.adjoint(cot, xi=xi, cols=cols, cot_rec=c_rec, rec_row=row)
        f = lambda k: loss(k, with_gamma)   # noqa: E731
        fd = (8 * (f(sub.k + d) - f(sub.k - d)) - (f(sub.k + 2 * d) - f(sub.k - 2 * d))) / (12 * d)
        assert abs(gk - fd) < 1e-6 * max(abs(fd), 1e-30), (with_gamma, gk, fd)
