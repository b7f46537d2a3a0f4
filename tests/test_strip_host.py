"""Host-side pieces of the layered-strip glue: the least-squares solve and its closed-form
backward (torch on the CPU; the GPU runs the same code on device tensors)."""
import pytest

torch = pytest.importorskip("torch")


def test_least_squares_matches_lstsq_and_its_gradient_passes_gradcheck():
    from paper_2103_12172_gb300.strip import LeastSquares
    g = torch.Generator().manual_seed(0)
    A = torch.randn(40, 12, dtype=torch.complex128, generator=g)
    A[:, 3] *= 1e4                                   # unequal column scales (equilibrated inside)
    b = torch.randn(40, dtype=torch.complex128, generator=g)
    x = LeastSquares.apply(A, b)
    xr = torch.linalg.lstsq(A, b[:, None]).solution[:, 0]
    assert (x - xr).abs().max().item() <= 1e-12 * xr.abs().max().item()
    A.requires_grad_(True)
    b.requires_grad_(True)
    assert torch.autograd.gradcheck(lambda A, b: LeastSquares.apply(A, b), (A, b), eps=1e-6, atol=1e-5)
