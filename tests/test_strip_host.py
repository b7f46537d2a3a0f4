"""Host-side pieces of the layered-strip glue: the closed-form backward of the least-squares
solve (strip.least_squares_grads), checked on the CPU with torch's own QR standing in for the
GPU factorisation (the GPU path is tested in test_gpu_linalg.py)."""
import pytest

torch = pytest.importorskip("torch")


class _HostLeastSquares(torch.autograd.Function):
    """x = argmin ||A x - b|| by torch.linalg.qr on the CPU, backward by least_squares_grads."""

    @staticmethod
    def forward(ctx, A, b):
        Q, R = torch.linalg.qr(A)
        x = torch.linalg.solve_triangular(R, (Q.conj().transpose(0, 1) @ b)[:, None], upper=True)[:, 0]
        ctx.save_for_backward(A, b, x, R)
        return x

    @staticmethod
    def backward(ctx, g):
        from paper_2103_12172_gb300.strip import least_squares_grads
        A, b, x, R = ctx.saved_tensors
        t = torch.linalg.solve_triangular(R.conj().transpose(0, 1), g[:, None], upper=False)
        w = torch.linalg.solve_triangular(R, t, upper=True)[:, 0]
        return least_squares_grads(A, b, x, w, lambda M, v: M @ v)


def test_least_squares_closed_form_gradient_passes_gradcheck():
    g = torch.Generator().manual_seed(0)
    A = torch.randn(40, 12, dtype=torch.complex128, generator=g)
    A[:, 3] *= 1e2                                   # unequal column scales
    b = torch.randn(40, dtype=torch.complex128, generator=g)
    x = _HostLeastSquares.apply(A, b)
    xr = torch.linalg.lstsq(A, b[:, None]).solution[:, 0]
    assert (x - xr).abs().max().item() <= 1e-12 * xr.abs().max().item()
    A.requires_grad_(True)
    b.requires_grad_(True)
    assert torch.autograd.gradcheck(lambda A, b: _HostLeastSquares.apply(A, b), (A, b), eps=1e-6, atol=1e-5)


def test_least_squares_refuses_host_tensors():
    """The product path has no CPU fallback: LeastSquares takes CUDA tensors only."""
    from paper_2103_12172_gb300.strip import LeastSquares
    A = torch.randn(8, 3, dtype=torch.complex128)
    with pytest.raises(TypeError):
        LeastSquares.apply(A, torch.randn(8, dtype=torch.complex128))
