"""Pins for the oracle's grid sets (Section 3.2.2) against brute force and counting."""
import numpy as np
import pytest

import workloads as W
from oracle.grid import grid_sets, node_coordinates


def brute_force_sets(sub):
    """Node-by-node restatement of Section 3.2.2 with explicit neighbourhood checks."""
    x, y = node_coordinates(sub)
    nx, ny = sub.nx, sub.ny
    M0 = {(n, m) for n in range(1, ny - 1) for m in range(1, nx - 1)}
    Mp = {(n, m) for (n, m) in M0 if sub.x0 < x[m] < sub.x1 and sub.y0 < y[n] < sub.y1}
    Mm = M0 - Mp

    def footprint(S):
        out = set()
        for (n, m) in S:
            for dn in (-1, 0, 1):
                for dm in (-1, 0, 1):
                    out.add((n + dn, m + dm))
        return out

    return Mp, Mm, footprint(Mp) & footprint(Mm)


@pytest.mark.parametrize("n", [9, 17, 33])
def test_grid_sets_match_brute_force(n):
    sub = W.small_subdomain(n, 3.0, W.AP_DIRX_SOMMY, 4)
    gs = grid_sets(sub)
    Mp, Mm, gamma = brute_force_sets(sub)
    assert {tuple(p) for p in np.argwhere(gs.Mp)} == Mp
    assert {tuple(p) for p in np.argwhere(gs.Mm)} == Mm
    got = list(zip(gs.gamma_n.tolist(), gs.gamma_m.tolist()))
    assert set(got) == gamma
    assert got == sorted(gamma)  # row-major (n, m) order


@pytest.mark.parametrize("n,expect", [(129, 856), (257, 1704), (513, 3416), (1025, 6824)])
def test_gamma_is_8P(n, expect):
    """gamma is the 2-node ring around M+: |gamma| = (P+2)^2 - (P-2)^2 = 8P with P the
    number of M+ nodes per side (P = 107/213/427/853 for the 129..1025 grids)."""
    sub = W.small_subdomain(n, 10.0, W.AP_DIRX_SOMMY, 4)
    x, _ = node_coordinates(sub)
    P = int(np.sum((x > 0.0) & (x < 1.0)))
    gs = grid_sets(sub)
    assert gs.gamma_n.size == 8 * P == expect
    assert gs.Mp.sum() == P * P


def test_ownership_and_parameters():
    sub = W.small_subdomain(129, 10.0, W.AP_DIRX_SOMMY, 4)
    gs = grid_sets(sub)
    x, y = node_coordinates(sub)
    counts = np.bincount(gs.owner, minlength=5)[1:]
    # corner ties go to the horizontal sides (lower index): symmetric counts
    assert counts[0] == counts[1] and counts[2] == counts[3]
    assert counts.sum() == gs.gamma_n.size
    gx, gy = x[gs.gamma_m], y[gs.gamma_n]
    for side, rho_exact, s_exact in ((1, -gy, 2 * gx - 1), (2, gy - 1, 2 * gx - 1),
                                     (3, -gx, 2 * gy - 1), (4, gx - 1, 2 * gy - 1)):
        sel = gs.owner == side
        np.testing.assert_allclose(gs.rho[sel], rho_exact[sel], atol=1e-15)
        np.testing.assert_allclose(gs.s[sel], s_exact[sel], atol=1e-14)
    # each gamma node is within 2h of the boundary and owned by a nearest side
    assert np.all(np.abs(gs.rho) < 2 * sub.h)
