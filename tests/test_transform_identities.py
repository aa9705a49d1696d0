"""The identities behind the library's real transforms, checked in numpy against the oracle's dense
matrices (no GPU): two real lines packed into one complex line, one length-N complex DFT, and the
pre-/post-processing that turns it into the Hartley transform (periodic, Eq. PP), DST-I (Dirichlet,
Eq. PD) or weighted DCT-I (Neumann, Eq. PN) of both lines.  The CUDA kernels implement these steps;
the GPU tests check the kernels themselves.  This file pins the derivation they rest on: the DST-I
and DCT-I of N-interval lines from a length-N DFT of the pre-processed line (no 2N extension), the
even outputs read off directly and the odd outputs as a running sum (the classical sine and cosine
transforms by FFT, e.g. Numerical Recipes, 2nd ed., Sec. 12.3, restated here)."""
import numpy as np
import pytest

from tests.helpers import library_axis_matrix


def _packed_transform(bc, A, B, N):
    """Library transform of the real lines A and B (values at the unknowns) via one complex DFT."""
    j = np.arange(N)
    s = np.sin(np.pi * j / N)
    c = np.cos(np.pi * j / N)
    X = A + 1j * B
    anchor = 0.0
    if bc == "periodic":
        z = X
    elif bc == "dirichlet":                      # unknowns 1..N-1 stored at 0..N-2; x_0 = x_N = 0
        x = np.concatenate([[0.0], X, [0.0]])
        xj, xm = x[j], x[N - j]
        z = s * (xj + xm) + 0.5 * (xj - xm)
    else:                                        # unknowns 0..N
        xj, xm = X[j], X[N - j]
        z = 0.5 * (xj + xm) - s * (xj - xm)
        anchor = 0.5 * (X[0] - X[N]) + np.sum(X[1:N] * c[1:N])
    Z = np.fft.fft(z)                            # Z_k = sum_j z_j exp(-2 pi i j k / N)
    H = N // 2
    k = np.arange(H)
    zk, zm = Z[k], Z[(N - k) % N]
    R = 0.5 * (zk + zm)                          # real-line parts of the two packed lines
    I = 0.5j * (zk - zm)
    if bc == "periodic":
        out = np.empty(N, dtype=complex)
        out[k] = R + I                           # T_k
        out[(N - k[1:])] = (R - I)[1:]           # T_{N-k}
        out[H] = Z[H]
        return out
    if bc == "dirichlet":
        out = np.empty(N - 1, dtype=complex)     # index = unknown - 1
        out[2 * k[1:] - 1] = I[1:]               # T_{2k} = I_k
        d = R.copy()
        d[0] *= 0.5
        out[2 * k] = np.cumsum(d)                # T_{2k+1} = T_{2k-1} + R_k, T_1 = R_0 / 2
        return out
    out = np.empty(N + 1, dtype=complex)
    out[2 * k] = R                               # T_{2k} = R_k
    d = I.copy()
    d[0] = anchor                                # T_1 = (x_0 - x_N)/2 + sum_j x_j cos(j pi / N)
    out[2 * k + 1] = np.cumsum(d)                # T_{2k+1} = T_{2k-1} + I_k
    out[N] = Z[H]
    return out


@pytest.mark.parametrize("bc", ["periodic", "dirichlet", "neumann"])
@pytest.mark.parametrize("N", [4, 8, 16, 64, 256])
def test_packed_real_transform_equals_dense_transform(bc, N):
    n = {"periodic": N, "dirichlet": N - 1, "neumann": N + 1}[bc]
    rng = np.random.default_rng(N)
    A, B = rng.standard_normal(n), rng.standard_normal(n)
    T = library_axis_matrix(bc, N)
    got = _packed_transform(bc, A, B, N)
    scale = max(np.abs(T @ A).max(), np.abs(T @ B).max())
    np.testing.assert_allclose(got.real, T @ A, atol=1e-12 * scale)
    np.testing.assert_allclose(got.imag, T @ B, atol=1e-12 * scale)


@pytest.mark.parametrize("bc,const", [("periodic", lambda N: N), ("dirichlet", lambda N: N / 2),
                                      ("neumann", lambda N: N / 2)])
def test_library_transforms_are_involutions_up_to_a_constant(bc, const):
    """T^2 = C I with C = N (Hartley), N/2 (DST-I and weighted DCT-I): the inverse is T / C."""
    for N in (6, 8, 10):
        T = library_axis_matrix(bc, N)
        np.testing.assert_allclose(T @ T, const(N) * np.eye(T.shape[0]), atol=1e-12 * N)
