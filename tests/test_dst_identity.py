"""The identity behind the dense-row sine transforms of the GPU path: a DST-I of length N - 1
(complex data) from one complex FFT of length N of the twisted sequence
y_j = sin(pi j/N)(x_j + x_{N-j}) + (x_j - x_{N-j})/2, with the even outputs (i/2)(C_k - C_{N-k})
and the odd outputs the prefix sums of (C_k + C_{N-k})/2 (F_1 = C_0/2). Checked here in numpy
against the direct sine sums, for every power-of-2 length the kernels take."""
import numpy as np
import pytest


@pytest.mark.parametrize("N", [8, 16, 64, 256, 2048])
def test_dst1_from_a_length_n_fft(N):
    rng = np.random.default_rng(N)
    x = np.zeros(N + 1, complex)
    x[1:N] = rng.standard_normal(N - 1) + 1j * rng.standard_normal(N - 1)
    j = np.arange(1, N)
    direct = np.array([np.sum(x[1:N] * np.sin(np.pi * q * j / N)) for q in range(1, N)])
    s = np.sin(np.pi * np.arange(N) / N)
    y = np.zeros(N, complex)
    y[1:] = s[1:] * (x[1:N] + x[N - 1:0:-1]) + 0.5 * (x[1:N] - x[N - 1:0:-1])
    C = np.fft.fft(y)
    F = np.zeros(N, complex)
    k = np.arange(1, N // 2)
    F[2 * k] = 0.5j * (C[k] - C[N - k])
    terms = np.concatenate([[C[0] / 2], (C[k] + C[N - k]) / 2])
    F[1::2] = np.cumsum(terms)
    err = np.abs(F[1:] - direct).max() / np.abs(direct).max()
    assert err < 1e-12 * max(1.0, N / 256), err
