"""The dense linear algebra of the coupled solve on the GPU (Section 3.5, steps 2(b)-(c)):
mdp_householder_qr (one cooperative launch, columns in shared memory or, for tall matrices, in
global memory), the structured two-stage QR, mdp_triangular_solve and mdp_complex_matmul,
against numpy's textbook routines on the same matrices; and the least squares' gradient
(LeastSquares on the GPU) against central differences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _qr_checks(A, b, fac):
    fac.check()
    R = fac.R().cpu().numpy()
    assert np.all(np.abs(np.diag(R).imag) == 0.0) and np.all(np.diag(R).real != 0.0)
    Ap = A if fac.perm is None else A[:, fac.perm.cpu().numpy()]
    G = Ap.conj().T @ Ap
    assert np.abs(R.conj().T @ R - G).max() <= 1e-12 * np.abs(G).max()
    xr = np.linalg.lstsq(A, b, rcond=None)[0]
    y = np.linalg.solve(R, fac.qb.cpu().numpy())
    x = y if fac.perm is None else np.empty_like(y)
    if fac.perm is not None:
        x[fac.perm.cpu().numpy()] = y
    assert np.abs(x - xr).max() <= 1e-10 * np.abs(xr).max()
    assert np.abs(fac.lstsq().cpu().numpy() - xr).max() <= 1e-10 * np.abs(xr).max()


@pytest.mark.parametrize("m,n", [(500, 60), (3424, 384), (64, 64), (1, 1), (37, 5), (9000, 40)])
def test_householder_qr_gram_identity_and_least_squares(mdp, m, n):
    """R^H R = A^H A, a real nonzero diagonal, and R^{-1} (Q^H b) is the least-squares solution;
    (9000, 40) keeps its columns in global memory, (3424, 384) takes three columns per CTA."""
    from paper_2103_12172_gb300.linalg import householder_qr
    rng = np.random.default_rng(m + n)
    A = _rand(rng, m, n)
    if n > 1 and m > 1:
        A[:, 1] = 0.0
        A[1, 1] = 2.0 + 0.0j        # column 1 below row 1 already zero (H = I after step 0 ... up to fill-in)
        A[0, 1] = 0.5
    b = _rand(rng, m)
    fac = householder_qr(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda())
    _qr_checks(A, b, fac)


def test_qr_of_an_already_triangular_matrix_keeps_its_columns(mdp):
    """Columns already of the form beta e_k with real beta get H = I (tau = 0)."""
    from paper_2103_12172_gb300.linalg import householder_qr
    rng = np.random.default_rng(3)
    n = 50
    A = np.triu(_rand(rng, n, n))
    A[np.arange(n), np.arange(n)] = -np.abs(A[np.arange(n), np.arange(n)]) - 1.0   # real negative diagonal
    b = _rand(rng, n)
    fac = householder_qr(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda())
    fac.check()
    assert np.abs(fac.R().cpu().numpy() - A).max() <= 1e-14 * np.abs(A).max()
    assert np.abs(fac.qb.cpu().numpy() - b).max() == 0.0


def test_batched_qr_with_several_right_hand_sides(mdp):
    """mdp_householder_qr_batched on 5 matrices with 3 right-hand sides each: every matrix's R and
    Q^H B match its own dense factorisation (numpy's QR up to the signs of the rows of R)."""
    import ctypes as C
    from paper_2103_12172_gb300 import _lib
    rng = np.random.default_rng(11)
    batch, m, n, nrhs = 5, 300, 70, 3
    As = _rand(rng, batch, m, n + nrhs)
    M = torch.from_numpy(np.ascontiguousarray(As.transpose(0, 2, 1))).cuda()   # column-major blocks
    tau = torch.empty((batch, n), dtype=torch.complex128, device="cuda")
    work = torch.empty(int(_lib.lib().mdp_householder_qr_work_ints(batch)), dtype=torch.int32, device="cuda")
    st = _lib.lib().mdp_householder_qr_batched(batch, m, n, nrhs, C.c_void_p(M.data_ptr()), m, (n + nrhs) * m,
                                               C.c_void_p(tau.data_ptr()), C.c_void_p(work.data_ptr()),
                                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert int(work[batch].item()) == 0
    out = M.cpu().numpy().transpose(0, 2, 1)
    for j in range(batch):
        A, B = As[j, :, :n], As[j, :, n:]
        R = np.triu(out[j, :n, :n])
        Q, Rn = np.linalg.qr(A)
        s = np.diag(Rn) / np.diag(R)                 # unit phases relating the two factorisations
        assert np.abs(np.abs(s) - 1).max() <= 1e-12
        assert np.abs(s[:, None] * R - Rn).max() <= 1e-12 * np.abs(Rn).max()
        assert np.abs(s[:, None] * out[j, :n, n:] - Q.conj().T @ B).max() <= 1e-12 * np.abs(B).max() * np.sqrt(m)


def test_structured_qr_equals_the_dense_least_squares(mdp):
    """Two-stage QR (a batched QR per row block on its own columns, then the stacked factors)
    gives the least-squares solution and the Gram matrix of the whole block-sparse system, in
    the order private columns of each block, then the shared ones; gram_solve inverts A^H A."""
    from paper_2103_12172_gb300.linalg import householder_qr, structured_qr
    rng = np.random.default_rng(7)
    n = 40
    rows = [90, 70, 110]
    cols = [list(range(0, 16)), list(range(10, 30)), list(range(24, 40)) + [2, 3]]
    A = np.zeros((sum(rows), n), complex)
    r0 = 0
    for g, cj in zip(rows, cols):
        A[r0:r0 + g, cj] = _rand(rng, g, len(cj))
        r0 += g
    b = _rand(rng, sum(rows))
    At, bt = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
    fac = structured_qr(At, bt, rows, [sorted(c) for c in cols])
    assert fac.perm is not None and len(fac.works) == 2   # two stages: the blocks, then the shared columns
    _qr_checks(A, b, fac)
    g = _rand(rng, n)
    w = fac.gram_solve(torch.from_numpy(g).cuda()).cpu().numpy()
    assert np.abs((A.conj().T @ A) @ w - g).max() <= 1e-10 * np.abs(g).max()


@pytest.mark.parametrize("n,nrhs", [(1, 1), (31, 2), (33, 1), (384, 3), (1000, 1)])
@pytest.mark.parametrize("conj_trans", [False, True])
def test_triangular_solve_matches_numpy(mdp, n, nrhs, conj_trans):
    """mdp_triangular_solve reads only the upper triangle of the column-major factor (garbage
    below it is ignored) and solves R X = B or R^H X = B to rounding."""
    from paper_2103_12172_gb300.linalg import triangular_solve
    rng = np.random.default_rng(n + 7 * nrhs)
    R = np.linalg.qr(_rand(rng, 2 * n, n))[1]      # well conditioned (a random triangle is not)
    ldr = n + 5
    F = _rand(rng, n, ldr)                          # F[j, i] = R(i, j) for i <= j, garbage elsewhere
    F[:, :n] = np.where(np.triu(np.ones((n, n), bool)).T, R.T, F[:, :n])
    B = _rand(rng, n, nrhs)
    X = triangular_solve(torch.from_numpy(F).cuda(), n, ldr, torch.from_numpy(B).cuda(), conj_trans).cpu().numpy()
    Rop = R.conj().T if conj_trans else R
    Xr = np.linalg.solve(Rop, B)
    assert np.abs(Rop @ X - B).max() <= 1e-15 * n * np.abs(R).max() * np.abs(X).max()   # backward error
    assert np.abs(X - Xr).max() <= 1e-11 * np.abs(Xr).max()
    xv = triangular_solve(torch.from_numpy(F).cuda(), n, ldr, torch.from_numpy(B[:, 0].copy()).cuda(), conj_trans)
    assert np.array_equal(xv.cpu().numpy(), X[:, 0])


def test_complex_matmul_strides_conjugation_and_empty_shapes(mdp):
    """mdp_complex_matmul against numpy: plain, transposed and conjugated views (the lazily
    conjugated torch view too), a matrix-vector product, ragged tiles, k = 0 and m = 0."""
    from paper_2103_12172_gb300.linalg import _matmul, matmul
    rng = np.random.default_rng(5)
    A = _rand(rng, 37, 21)
    B = _rand(rng, 21, 19)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    tol = 1e-13 * 21

    def close(x, y):
        return np.abs(x.cpu().numpy() - y).max() <= tol * max(1.0, np.abs(y).max())

    assert close(matmul(At, Bt), A @ B)
    assert close(matmul(Bt.transpose(0, 1), At.transpose(0, 1)), B.T @ A.T)
    assert close(_matmul(At, Bt, conj_a=True), A.conj() @ B)
    assert close(_matmul(At, Bt, conj_b=True), A @ B.conj())
    assert close(matmul(At.conj(), Bt), A.conj() @ B)
    assert close(matmul(At.transpose(0, 1).conj(), At), A.conj().T @ A)
    assert close(matmul(At, Bt[:, 4]), A @ B[:, 4])
    assert close(matmul(At[::2, ::3], Bt[::3, 1:]), A[::2, ::3] @ B[::3, 1:])
    assert close(matmul(torch.ones(4, 21, dtype=torch.float64, device="cuda"), Bt), np.ones((4, 21)) @ B)
    z = matmul(At[:, :0], Bt[:0, :])
    assert z.shape == (37, 19) and float(z.abs().max()) == 0.0
    assert matmul(At[:0], Bt).shape == (0, 19)


def test_matmul_gradient_matches_torch(mdp):
    """MatMul's backward (g B^H, A^H g) equals torch's own matmul gradient."""
    from paper_2103_12172_gb300.linalg import matmul
    g = torch.Generator().manual_seed(1)
    A = torch.randn(12, 7, dtype=torch.complex128, generator=g).cuda().requires_grad_(True)
    B = torch.randn(7, 5, dtype=torch.complex128, generator=g).cuda().requires_grad_(True)
    W = torch.randn(12, 5, dtype=torch.complex128, generator=g).cuda()
    (matmul(A, B) * W).real.sum().backward()
    gA, gB = A.grad.clone(), B.grad.clone()
    A.grad = B.grad = None
    ((A.cpu() @ B.cpu()) * W.cpu()).real.sum().backward()
    assert (gA - A.grad).abs().max().item() <= 1e-13 and (gB - B.grad).abs().max().item() <= 1e-13


def test_least_squares_on_the_gpu_and_its_gradient(mdp):
    """LeastSquares (equilibrated QR, triangular solves, closed-form backward, all on libmdp's
    kernels) against numpy's lstsq, and its gradient against central differences."""
    from paper_2103_12172_gb300.strip import LeastSquares
    rng = np.random.default_rng(2)
    A0 = _rand(rng, 60, 14)
    A0[:, 3] *= 1e3
    b0 = _rand(rng, 60)
    A = torch.from_numpy(A0).cuda()
    b = torch.from_numpy(b0).cuda()
    x = LeastSquares.apply(A, b).cpu().numpy()
    xr = np.linalg.lstsq(A0, b0, rcond=None)[0]
    assert np.abs(x - xr).max() <= 1e-11 * np.abs(xr).max()
    w = _rand(rng, 14)
    wt = torch.from_numpy(w).cuda()
    A.requires_grad_(True)
    b.requires_grad_(True)
    (LeastSquares.apply(A, b) * wt).real.sum().backward()
    gA, gb = A.grad.cpu().numpy(), b.grad.cpu().numpy()

    def f(Ap, bp):
        return (np.linalg.lstsq(Ap, bp, rcond=None)[0] * w).real.sum()

    eps = 1e-6
    for (i, j) in [(0, 0), (5, 3), (59, 13)]:
        E = np.zeros_like(A0)
        E[i, j] = eps
        d_re = (f(A0 + E, b0) - f(A0 - E, b0)) / (2 * eps)
        d_im = (f(A0 + 1j * E, b0) - f(A0 - 1j * E, b0)) / (2 * eps)
        assert abs(gA[i, j] - (d_re + 1j * d_im)) <= 1e-6 * max(1.0, abs(d_re + 1j * d_im))
    e = np.zeros_like(b0)
    e[7] = eps
    d = (f(A0, b0 + e) - f(A0, b0 - e)) / (2 * eps) + 1j * (f(A0, b0 + 1j * e) - f(A0, b0 - 1j * e)) / (2 * eps)
    assert abs(gb[7] - d) <= 1e-6 * max(1.0, abs(d))
