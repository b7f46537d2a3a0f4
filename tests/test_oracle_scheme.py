"""Pins for the oracle's compact scheme and discrete AP (Sections 3.1, 3.2.1)."""
import numpy as np
import pytest
import scipy.fft
from scipy.sparse.linalg import splu

import workloads as W
from oracle.grid import node_coordinates
from oracle.projection import APSystem
from oracle.scheme import apply_L, assemble


def discrete_plane_wave(sub, theta):
    """e^{i(alpha x + beta y)} with alpha = k cos(theta) and beta fixed by the scheme's
    discrete dispersion relation: for the separable symbol of the 9-point operator,
    (2cos(beta h) - 2) = -(a/h^2 + k^2 + k^2 a/12) / (1/h^2 + a/(6h^2) + k^2/12),
    a = 2cos(alpha h) - 2 (the operator acting on a Fourier mode)."""
    h, k = sub.h, sub.k
    alpha = k * np.cos(theta)
    a = 2 * np.cos(alpha * h) - 2
    b = -(a / h**2 + k**2 + k**2 * a / 12) / (1 / h**2 + a / (6 * h**2) + k**2 / 12)
    beta = np.arccos(1 + b / 2) / h
    x, y = node_coordinates(sub)
    X, Y = np.meshgrid(x, y)
    return np.exp(1j * (alpha * X + beta * Y))


@pytest.mark.parametrize("n,k", [(33, 3.0), (129, 10.0), (257, 30.0)])
def test_interior_stencil_annihilates_discrete_plane_wave(n, k):
    sub = W.small_subdomain(n, k, W.AP_DIRX_SOMMY, 4)
    v = discrete_plane_wave(sub, 0.3)
    r = apply_L(v, sub.h, k)[1:-1, 1:-1]
    assert np.abs(r).max() < 1e-12 / sub.h**2


@pytest.mark.parametrize("n,k", [(17, 3.0), (65, 10.0), (129, 10.0)])
def test_dirichlet_ap_matches_sine_transform_closed_form(n, k):
    """P1: with u = 0 on all four sides the AP is diagonalised by the 2-D DST-I:
    G g = IDST[ DST[g] / mu_pq ], mu_pq = (lp + lq)/h^2 + lp lq/(6h^2) + k^2 + k^2 (lp + lq)/12,
    lp = -4 sin^2(pi p / (2 N_c)). scipy.fft.dstn (type 1) is the library transform."""
    sub = W.small_subdomain(n, k, W.AP_DIRICHLET4, 4)
    S = APSystem(sub)
    nc = n - 1
    g = W.random_complex((n, n), seed=0)
    g[0, :] = g[-1, :] = g[:, 0] = g[:, -1] = 0
    u = S.solve(g)
    h = sub.h
    lam = -4 * np.sin(np.pi * np.arange(1, nc) / (2 * nc)) ** 2
    LP, LQ = np.meshgrid(lam, lam)
    mu = (LP + LQ) / h**2 + LP * LQ / (6 * h**2) + k**2 + k**2 * (LP + LQ) / 12
    ghat = scipy.fft.dstn(g[1:-1, 1:-1], type=1)
    u_cf = scipy.fft.idstn(ghat / mu, type=1)
    kappa = np.abs(mu).max() / np.abs(mu).min()
    err = np.abs(u[1:-1, 1:-1] - u_cf).max() / np.abs(u_cf).max()
    assert err < 50 * kappa * np.finfo(float).eps


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
@pytest.mark.parametrize("n", [9, 17])
def test_splu_matches_dense_solve_and_adjoint(ap, n):
    """P8: brute force on tiny grids -- SuperLU equals a dense solve, and the adjoint
    solve equals the conjugate transpose of the dense inverse."""
    sub = W.small_subdomain(n, 5.0, ap, 4)
    A, U, idx = assemble(sub)
    Ad = A.toarray()
    b = W.random_complex(A.shape[0], seed=1)
    x1 = splu(A).solve(b)
    x2 = np.linalg.solve(Ad, b)
    assert np.abs(x1 - x2).max() < 1e-11 * np.abs(x2).max()
    S = APSystem(sub)
    y = np.zeros(U.shape, complex)
    y[U] = b
    xa = S.solve_adjoint(y)[U]
    xd = np.linalg.inv(Ad).conj().T @ b
    assert np.abs(xa - xd).max() < 1e-11 * np.abs(xd).max()


def _sommerfeld_truncation(n, k, theta, top, ap=W.AP_DIRX_SOMMY):
    """Residual of the assembled Sommerfeld row on a continuous plane wave, minus the
    exact du/dn + i k u at the half node (n outward)."""
    sub = W.small_subdomain(n, k, ap, 4)
    A, U, idx = assemble(sub)
    x, y = node_coordinates(sub)
    X, Y = np.meshgrid(x, y)
    alpha, beta = k * np.cos(theta), k * np.sin(theta)
    u = np.exp(1j * (alpha * X + beta * Y))
    Au = np.zeros(U.shape, complex)
    Au[U] = A @ u[U]
    row = n - 1 if top else 0
    ms = np.arange(2, n - 2)  # rows whose neighbours are all unknowns
    yh = (y[n - 1] + y[n - 2]) / 2 if top else (y[0] + y[1]) / 2
    dudn = 1j * beta if top else -1j * beta
    exact = (dudn + 1j * k) * np.exp(1j * (alpha * x[ms] + beta * yh))
    return np.abs(Au[row, ms] - exact).max()


@pytest.mark.parametrize("top", [True, False])
def test_sommerfeld_rows_are_fourth_order(top):
    """The Sommerfeld rows approximate du/dn + i k u at the half node to O(h^4): the
    truncation error on a smooth Helmholtz solution falls ~16x per halving of h."""
    errs = [_sommerfeld_truncation(n, 10.0, 0.7, top) for n in (33, 65, 129, 257)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.7), rates


@pytest.mark.parametrize("top", [True, False])
def test_paper_sommerfeld_rows_are_second_order(top):
    """The Sommerfeld rows as printed (AP_DIRX_SOMMY_PAPER: D delta / 6 with a minus sign,
    -k^2 h^2 / 24, D abar / 2) are consistent with du/dn + i k u = 0 but only to O(h^2): the
    truncation error falls ~4x per halving of h. This is why the default rows are re-derived."""
    errs = [_sommerfeld_truncation(n, 10.0, 0.7, top, W.AP_DIRX_SOMMY_PAPER) for n in (33, 65, 129, 257)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.2), rates


@pytest.mark.parametrize("ap", [W.AP_DIRX_SOMMY, W.AP_DIRX_SOMMY_PAPER])
def test_dk_matrix_matches_finite_difference(ap):
    sub = W.small_subdomain(17, 7.0, ap, 4)
    dA = assemble(sub, deriv=True)[0].toarray()
    d = 1e-5
    fd = (assemble(sub, k=7.0 + d)[0].toarray() - assemble(sub, k=7.0 - d)[0].toarray()) / (2 * d)
    assert np.abs(dA - fd).max() < 1e-6 * np.abs(dA).max()
