"""Test-side helpers: library-convention transforms built from the oracle's matrices,
and the shared workload -> GPU plan bridge."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402


def library_axis_matrix(bc, N):
    """The unnormalised real transform the library uses on one axis, written with the
    oracle's eigenvector matrices: Hartley = Re(P) - Im(P) for periodic (P = DFT of Eq. PP);
    P of Eq. PD for Dirichlet; C W = (N/2) W^{-1} F for Neumann (F = (2/N) W C W)."""
    F, _ = O.transform_pair(bc, N)
    if bc == O.PERIODIC:
        return F.real - F.imag
    if bc == O.DIRICHLET:
        return F
    w = np.ones(N + 1)
    w[0] = w[-1] = 0.5
    return (N / 2.0) * (F / w[:, None])


def library_forward(U, bc, Ns):
    """Apply the library transform along every axis of U (axes ordered z, y, x; Ns = (Nx, Ny, Nz))."""
    for d, N in enumerate(Ns):
        U = O.apply_along(library_axis_matrix(bc, N), U, U.ndim - 1 - d)
    return U


def rel_max(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.max(np.abs(x - y)) / np.max(np.abs(y)))


def rel_l2(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.linalg.norm((x - y).ravel()) / np.linalg.norm(y.ravel()))
