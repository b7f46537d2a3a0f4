"""Host logic of the structured least squares (linalg.structured_qr): the private/shared column
split, the placement of the blocks' factors in R, the stacking of the shared blocks and the
column permutation, checked on the CPU with the device QR launch and triangular solve replaced
by numpy's QR and solve on the same storage layout (garbage below the diagonal included, as the
reflectors leave there)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _fake_launch(M, batch, m, n, ldm, stride):
    """What mdp_householder_qr_batched leaves in M for one right-hand side: R in the upper triangle
    of the first n columns (column-major), noise below it, Q^H b in column n."""
    rng = np.random.default_rng(batch * 1000 + m)
    Mv = M.reshape(-1)
    for j in range(batch):
        blk = Mv[j * stride:j * stride + (n + 1) * ldm].reshape(n + 1, ldm)
        A = blk[:n, :m].T.numpy()
        b = blk[n, :m].numpy()
        Q, R = np.linalg.qr(A, mode="complete")
        noise = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
        cm = np.where(np.arange(m)[None, :] <= np.arange(n)[:, None], R[:, :n].T, noise)   # [col, row]
        blk[:n, :m] = torch.from_numpy(cm)
        blk[n, :m] = torch.from_numpy(Q.conj().T @ b)
    return None, torch.zeros(batch + 2, dtype=torch.int32)


def _fake_trsv(F, n, ldr, rhs, conj_trans=False):
    R = np.triu(F[:n, :n].numpy().T)
    Rop = R.conj().T if conj_trans else R
    return torch.from_numpy(np.linalg.solve(Rop, rhs.numpy()))


@pytest.fixture
def host_linalg(monkeypatch):
    from paper_2103_12172_gb300 import linalg
    monkeypatch.setattr(linalg, "_need_cuda", lambda *t: None)
    monkeypatch.setattr(linalg, "_qr_launch", _fake_launch)
    monkeypatch.setattr(linalg, "triangular_solve", _fake_trsv)
    return linalg


@pytest.mark.parametrize("layout", ["strip", "overlap3", "no_shared"])
def test_structured_qr_assembly_gives_the_least_squares_solution(host_linalg, layout):
    rng = np.random.default_rng(4)
    if layout == "strip":        # 4 blocks, interfaces shared by neighbours (the layered strip's pattern)
        n, rows = 40, [30, 34, 28, 31]
        cols = [list(range(0, 12)), list(range(8, 22)), list(range(18, 32)), list(range(28, 40))]
    elif layout == "overlap3":   # a column shared by three blocks, unsorted column lists
        n, rows = 20, [25, 22, 26]
        cols = [[5, 0, 1, 2, 3, 19], [4, 5, 6, 7, 8, 9, 19], [19, 10, 11, 12, 13, 14, 15, 16, 17, 18, 5]]
    else:                        # block diagonal: no shared column, no second stage
        n, rows = 15, [10, 12]
        cols = [list(range(0, 7)), list(range(7, 15))]
    A = np.zeros((sum(rows), n), complex)
    r0 = 0
    for g, cj in zip(rows, cols):
        A[r0:r0 + g, cj] = rng.standard_normal((g, len(cj))) + 1j * rng.standard_normal((g, len(cj)))
        r0 += g
    b = rng.standard_normal(sum(rows)) + 1j * rng.standard_normal(sum(rows))
    fac = host_linalg.structured_qr(torch.from_numpy(A), torch.from_numpy(b), rows, cols)
    perm = fac.perm.numpy()
    assert sorted(perm.tolist()) == list(range(n))
    R = fac.R().numpy()
    Ap = A[:, perm]
    G = Ap.conj().T @ Ap
    assert np.abs(R.conj().T @ R - G).max() <= 1e-12 * np.abs(G).max()
    xr = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.abs(fac.lstsq().numpy() - xr).max() <= 1e-11 * np.abs(xr).max()
    g = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = fac.gram_solve(torch.from_numpy(g)).numpy()
    assert np.abs((A.conj().T @ A) @ w - g).max() <= 1e-10 * np.abs(g).max()
    assert len(fac.works) == (1 if layout == "no_shared" else 2)
