"""Closed-form solutions used as test references (no method arithmetic of either side).

layered_exact: a plane wave normally incident on layers of piecewise-constant wavenumber
(Appendix A): in layer j, u_j(x) = A_j e^{i k_j x} + B_j e^{-i k_j x}, with the incident
amplitude A_0 = 1, no incoming wave from the right (B_last = 0), and u, du/dx continuous at
the interfaces. Solved as the small dense linear system of the interface conditions."""
import numpy as np


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
