"""Host model of the cooperative Householder QR (csrc/qr.cu, k_qr_cta): the column ownership,
the per-column count of reflectors applied, the choice of the next item (closest to forming its
matrix's next reflector, then matrix, then slot), the fused step on the critical column (norm
from the expansion ||a - s v||^2 = ||a||^2 - 2 Re(conj(s) v^H a) + |s|^2 ||v||^2 with
||v||^2 = 2 Re(tau) / |tau|^2, summed again when cancellation could cost more than two bits) and
the publication counters, run with the CTAs interleaved at random (each wait yields). It checks
that every interleaving ends (the waits are on published counters only) and that the result is
the least-squares factorisation (R^H R = A^H A, R^{-1} Q^H b = lstsq), on the CPU in numpy."""
import numpy as np
import pytest

N_SM = 152


def shape_of(batch, C, n_sm):
    """The launch shape of qr_shape: (G, Gb, slots)."""
    if batch <= n_sm:
        Gb = min(n_sm // batch, C)
        return batch * Gb, Gb, -(-C // Gb)
    return n_sm, 0, -(-batch // n_sm) * C


def reflector_of(a, xn2):
    """beta, tau, inv = 1/(alpha - beta), or H = I."""
    if xn2 == 0.0 and a.imag == 0.0:
        return a.real, 0j, 0j, False
    nrm = np.sqrt(abs(a) ** 2 + xn2)
    beta = -nrm if a.real >= 0 else nrm
    g = beta - a.real
    rd = 1.0 / (g * g + a.imag ** 2)
    return beta, complex(g / beta, -a.imag / beta), complex(-g * rd, -a.imag * rd), True


def cta(me, q, A, glob, tau, progress, stats):
    """One CTA as a generator; it yields whenever it would wait or has finished an item."""
    batch, m, n, C, G, Gb = q
    if Gb > 0:
        owned = [(me // Gb, me % Gb + s * Gb) for s in range(-(-(C - me % Gb) // Gb))]
    else:
        owned = [(me + (s // C) * G, s % C) for s in range(((batch - me + G - 1) // G) * C)]
    loc = {s: A[b][:, c].copy() for s, (b, c) in enumerate(owned)}
    nxt = {s: 0 for s in loc}

    def publish(b, c, x, t):
        glob[b][:, c] = x
        tau[b][c] = t
        assert progress[b] == c, "reflectors are published in order"
        progress[b] = c + 1

    for s, (b, c) in enumerate(owned):
        if c == 0:
            x = loc[s]
            beta, t, inv, refl = reflector_of(x[0], float(np.sum(np.abs(x[1:]) ** 2)))
            x[1:] = x[1:] * inv if refl else x[1:]
            x[0] = beta
            publish(b, 0, x.copy(), t)
    while True:
        best, pending = None, False
        for s, (b, c) in enumerate(owned):
            j, tg = nxt[s], min(c, n)
            if j < tg:
                pending = True
                if progress[b] > j:
                    key = (c - progress[b], b, s)
                    best = key if best is None or key < best else best
        if best is None:
            if not pending:
                break
            stats["waits"] += 1
            yield
            continue
        s0 = best[2]
        b, c = owned[s0]
        k = nxt[s0]
        v = glob[b][k:, k].copy()
        v[0] = 1.0
        t = tau[b][k]
        if c < n and k == c - 1:       # the fused step: apply H_k, form reflector c
            x = loc[s0]
            a = x[k:]
            w = np.vdot(v, a)           # conj(v) . a
            s_ = np.conj(t) * w
            d = np.vdot(v[2:], a[2:])
            s2 = float(np.sum(np.abs(a[2:]) ** 2))
            alpha = a[1] - v[1] * s_
            xn2, exact = s2, True
            if t != 0:
                vn2 = 2 * t.real / abs(t) ** 2 - 1 - abs(v[1]) ** 2
                xn2 = abs(s_) ** 2 * vn2 - 2 * (np.conj(s_) * d).real + s2
                exact = s2 > 0 and xn2 >= 0.25 * s2
            a_new = a - v * s_
            if not exact:
                stats["fallback"] += 1
                xn2 = float(np.sum(np.abs(a_new[2:]) ** 2))
            else:
                stats["estimate"] += 1
            beta, tn, inv, refl = reflector_of(alpha, xn2)
            x[k] = a_new[0]
            x[k + 1] = beta
            x[k + 2:] = a_new[2:] * inv if refl else a_new[2:]
            nxt[s0] = k + 1
            publish(b, c, x.copy(), tn)
        else:                            # up to 4 columns waiting for the same reflector
            chunk = [s0] + [s for s, (b2, c2) in enumerate(owned)
                            if s != s0 and b2 == b and nxt[s] == k and k < min(c2, n)
                            and not (c2 < n and k == c2 - 1)][:3]
            for s in chunk:
                if t != 0:
                    loc[s][k:] -= v * (np.conj(t) * np.vdot(v, loc[s][k:]))
                nxt[s] = k + 1
        yield
    for s, (b, c) in enumerate(owned):
        if c >= n:
            glob[b][:, c] = loc[s]


def run(batch, m, n, nrhs, n_sm, seed, near_dependent=False):
    rng = np.random.default_rng(seed)
    C = n + nrhs
    A = rng.standard_normal((batch, m, C)) + 1j * rng.standard_normal((batch, m, C))
    if near_dependent:            # columns nearly in the span of earlier ones: the norm estimate cancels
        for b in range(batch):
            for c in range(2, n, 3):
                A[b][:, c] = A[b][:, c - 1] * (1 + 1e-9) + 1e-7 * A[b][:, c]
    G, Gb, slots = shape_of(batch, C, n_sm)
    q = (batch, m, n, C, G, Gb)
    glob = [np.zeros((m, C), complex) for _ in range(batch)]
    tau = [np.zeros(n, complex) for _ in range(batch)]
    progress = [0] * batch
    stats = {"waits": 0, "fallback": 0, "estimate": 0}
    gens = [cta(me, q, A, glob, tau, progress, stats) for me in range(G)]
    live = list(range(G))
    steps = 0
    while live:
        i = live[rng.integers(len(live))]
        try:
            next(gens[i])
        except StopIteration:
            live.remove(i)
        steps += 1
        assert steps < 5_000_000, "no progress: a wait would never end"
    return A, glob, tau, stats


@pytest.mark.parametrize("batch,m,n,nrhs,n_sm", [(1, 40, 12, 1, 5), (1, 40, 12, 1, 152), (3, 30, 10, 2, 7),
                                                 (4, 25, 9, 1, 3), (2, 12, 12, 0, 4), (5, 20, 6, 1, 152)])
def test_every_interleaving_ends_with_the_least_squares_factorisation(batch, m, n, nrhs, n_sm):
    for seed in range(3):
        A, glob, tau, stats = run(batch, m, n, nrhs, n_sm, seed)
        for b in range(batch):
            R = np.triu(glob[b][:n, :n])
            An = A[b][:, :n]
            G_ = An.conj().T @ An
            assert np.abs(R.conj().T @ R - G_).max() <= 1e-12 * np.abs(G_).max()
            assert np.all(np.diag(R).imag == 0)
            if nrhs:
                x = np.linalg.solve(R, glob[b][:n, n])
                xr = np.linalg.lstsq(An, A[b][:, n], rcond=None)[0]
                assert np.abs(x - xr).max() <= 1e-9 * np.abs(xr).max()
        assert stats["estimate"] > 0


def test_cancellation_takes_the_exact_norm():
    """Nearly dependent columns make the norm expansion cancel: the fused step must fall back to
    summing the updated column, and the factorisation stays exact to rounding."""
    A, glob, tau, stats = run(1, 30, 12, 1, 5, 0, near_dependent=True)
    assert stats["fallback"] > 0
    R = np.triu(glob[0][:12, :12])
    An = A[0][:, :12]
    G_ = An.conj().T @ An
    assert np.abs(R.conj().T @ R - G_).max() <= 1e-10 * np.abs(G_).max()
