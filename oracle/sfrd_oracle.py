"""Plain FP64 CPU oracle for the compact-MTT ETDRK4-P13 solver of space-fractional
reaction-diffusion equations (arXiv 2003.13569, "Fast and accurate high-order method for high dimensional
space-fractional reaction-diffusion equation with general boundary conditions").

TEST INFRASTRUCTURE ONLY.  tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm are the only code allowed to import this module.  The
product path (the CUDA library under paper_2003_13569_gb300/ and its Python
binding) never imports it, and this module imports nothing from the product.

What it computes, in the paper's order and notation:

  * Section 3.1: per axis, the fourth-order compact Laplacian T = A^{-1} B
    (Eq. Lap), its closed-form eigenvalues and its eigenvector matrix P for
    periodic (Eq. PP), homogeneous Dirichlet (Eq. PD) and homogeneous Neumann
    (Eq. PN) boundary conditions.  Every transform is a dense matrix applied
    along one axis: O(n^2) per line, no fast transform anywhere.
  * Sections 3.2-3.3 (Eqs. E16-E18, E22): separable multi-D transform
    F(U) = P_z (z) P_y (y) P_x (x) U and the summed eigenvalue array
    Lambda = lambda_x + lambda_y (+ lambda_z), raised to alpha/2 (Def. 1, MTT).
  * Algorithm 1: L = kappa tau Lambda^{alpha/2}, the six Pade-(1,3) coefficient
    arrays, and the ETDRK4-P13 step exactly as listed there -- seven forward and
    four inverse transforms per species per step, including the re-transform of
    the stage value a_k.
  * Section 5: the maximum-norm error and the two manufactured-solution sources
    (Example 1, Example 2).
  * The discrete adjoint of that step (reverse-mode derivative of the same
    arithmetic), for gradient checks.
  * The Cox-Matthews variant of the step: the same stages with exact
    exponentials (e^{-L} in the place of R13(L)), its coefficients evaluated by
    the Cauchy contour integral.

Readings where the paper is garbled or silent (each pinned by a CPU test):
  R1  periodic eigenvalue angle: sin^2(pi k / N), k = 0..N-1 in DFT order (the
      printed (n-1) pi / (2N) angle does not diagonalise the circulant A^{-1}B);
  R2  multi-D: the summed eigenvalue is raised to alpha/2 (Def. 1, E16-E22);
  R3  Neumann: N+1 eigenvalues n = 0..N;
  R4  Neumann: T = C diag(lambda) C^{-1} with C_ij = cos(i j pi / N); the
      forward map (grid values -> eigen-coefficients) is C^{-1} = (2/N) W C W,
      W = diag(1/2, 1, ..., 1, 1/2);
  R5  c-stage uses a^k (Eq. ETDRK4P13 and Algorithm 1);
  R8  Example 1's source term carries a single kappa;
  R9  Table 1 uses kappa = 10, T = 1 and tau = h / (4 kappa);
  R10 Example 2: the third term of Phi is (40 pi^2)^{alpha/2};
  R12 a zero eigenvalue (L = 0) needs no special case: the rationals take their limits there;
  R14 Dirichlet conditions for Schnakenberg apply to the perturbation w about the homogeneous
      steady state u* (the reaction is evaluated at u* + w): a modelling choice, parity unpinned
      (the tests pin only that the perturbation form equals the reaction at u* + w);
  R16 the reaction is evaluated at t_k, t_k + tau/2, t_k + tau/2, t_k + tau in the four stages;
  R17 the Cox-Matthews variant puts e^{-L}, e^{-L/2} and the exponential phi-functions in the
      places of the Pade-(1,3) rationals.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Sequence

import numpy as np

PERIODIC = "periodic"
DIRICHLET = "dirichlet"
NEUMANN = "neumann"
BCS = (PERIODIC, DIRICHLET, NEUMANN)


# ---------------------------------------------------------------------------
# Section 3.1: one axis
# ---------------------------------------------------------------------------

def unknown_indices(bc: str, N: int) -> np.ndarray:
    """Grid indices n of the unknowns x_n = x_a + n h on an axis of N intervals.

    Periodic: u_1..u_N of the paper, i.e. nodes 0..N-1 (node N is node 0);
    Dirichlet: interior nodes 1..N-1; Neumann: all nodes 0..N (Section 3.1).
    """
    if bc == PERIODIC:
        return np.arange(0, N)
    if bc == DIRICHLET:
        return np.arange(1, N)
    if bc == NEUMANN:
        return np.arange(0, N + 1)
    raise ValueError(bc)


def compact_matrices(bc: str, N: int, h: float) -> tuple[np.ndarray, np.ndarray]:
    """The matrices A and B of the compact scheme as printed in Section 3.1.

    Periodic: N x N circulant tridiagonals; Dirichlet: (N-1) x (N-1)
    tridiagonals; Neumann: (N+1) x (N+1) with the 1/6 and -2 boundary rows.
    -Delta u ~ A^{-1} B u  (Eq. Lap).
    """
    n = len(unknown_indices(bc, N))
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    for i in range(n):
        A[i, i] = 5.0 / 6.0
        B[i, i] = 2.0
        if i > 0:
            A[i, i - 1] = 1.0 / 12.0
            B[i, i - 1] = -1.0
        if i < n - 1:
            A[i, i + 1] = 1.0 / 12.0
            B[i, i + 1] = -1.0
    if bc == PERIODIC:
        A[0, n - 1] = A[n - 1, 0] = 1.0 / 12.0
        B[0, n - 1] = B[n - 1, 0] = -1.0
    elif bc == NEUMANN:
        A[0, 1] = 1.0 / 6.0
        A[n - 1, n - 2] = 1.0 / 6.0
        B[0, 1] = -2.0
        B[n - 1, n - 2] = -2.0
    return A, B / (h * h)


def eigenvalues(bc: str, N: int, h: float) -> np.ndarray:
    """Closed-form eigenvalues of T = A^{-1}B, in the spectral order of transform_pair.

    lambda = 4 s / (h^2 (1 - s/3)) with
      periodic  s = sin^2(pi k / N),      k = 0..N-1   (reading R1)
      Dirichlet s = sin^2(n pi / (2N)),   n = 1..N-1
      Neumann   s = sin^2(n pi / (2N)),   n = 0..N     (reading R3)
    """
    if bc == PERIODIC:
        s = np.sin(np.pi * np.arange(N) / N) ** 2
    else:
        s = np.sin(np.pi * unknown_indices(bc, N) / (2.0 * N)) ** 2
    return 4.0 * s / (h * h * (1.0 - s / 3.0))


def transform_pair(bc: str, N: int) -> tuple[np.ndarray, np.ndarray]:
    """(F, Finv) with T = Finv diag(lambda) F: F takes grid values to eigen-coefficients.

    Periodic: F = P of Eq. PP, P_ij = exp(-2 pi sqrt(-1) i j / N), Finv = P^{-1}.
    Dirichlet: F = P of Eq. PD, P_ij = sin(i j pi / N), Finv = (2/N) P.
    Neumann (reading R4): C_ij = cos(i j pi / N) of Eq. PN holds the eigenvectors
    as columns, so F = C^{-1} = (2/N) W C W and Finv = C.

    The entries depend on the integer product i j only through its residue modulo the
    period (N for exp(-2 pi i ij/N), 2N for sin and cos of ij pi/N), so the product is
    reduced exactly in integers before the angle is formed: the angle then stays below
    2 pi and carries one rounding, instead of a relative rounding of a product that grows
    to N^2 (an absolute phase error of about 1e-13 at N = 384).
    """
    if bc == PERIODIC:
        j = np.arange(N)
        P = np.exp(-2j * np.pi * (np.outer(j, j) % N) / N)
        return P, np.conj(P) / N
    if bc == DIRICHLET:
        j = np.arange(1, N)
        S = np.sin(np.pi * (np.outer(j, j) % (2 * N)) / N)
        return S, (2.0 / N) * S
    if bc == NEUMANN:
        j = np.arange(0, N + 1)
        C = np.cos(np.pi * (np.outer(j, j) % (2 * N)) / N)
        w = np.ones(N + 1)
        w[0] = w[-1] = 0.5
        return (2.0 / N) * (w[:, None] * C * w[None, :]), C
    raise ValueError(bc)


# ---------------------------------------------------------------------------
# Sections 3.2-3.3: separable multi-D operators
# ---------------------------------------------------------------------------

def apply_along(M: np.ndarray, U: np.ndarray, axis: int) -> np.ndarray:
    """(M (axis) U): contract the matrix M with index `axis` of U (the circled-x/y/z products)."""
    return np.moveaxis(np.tensordot(M, U, axes=([1], [axis])), 0, axis)


@dataclass
class Grid:
    """Uniform grid: N[d] intervals on [lo[d], hi[d]] per axis, axes listed x, y, z.

    Fields are stored as numpy arrays of shape (n_z, n_y, n_x) in 3D, (n_y, n_x)
    in 2D and (n_x,) in 1D, so x is the last (fastest) array index.
    """
    N: tuple
    lo: tuple
    hi: tuple

    @property
    def dim(self) -> int:
        return len(self.N)

    def h(self, d: int) -> float:
        return (self.hi[d] - self.lo[d]) / self.N[d]

    def coords(self, bc: str, d: int) -> np.ndarray:
        return self.lo[d] + unknown_indices(bc, self.N[d]) * self.h(d)

    def shape(self, bc: str) -> tuple:
        return tuple(len(unknown_indices(bc, self.N[d])) for d in reversed(range(self.dim)))

    def mesh(self, bc: str) -> list:
        """Coordinate arrays [X, Y, (Z)] broadcast to the field shape."""
        axes = [self.coords(bc, d) for d in reversed(range(self.dim))]
        grids = np.meshgrid(*axes, indexing="ij")
        return list(reversed(grids))


class Spectral:
    """Per-axis transform pairs and the summed-eigenvalue array for one grid and BC."""

    def __init__(self, grid: Grid, bc: str):
        self.grid, self.bc = grid, bc
        self.pairs = [transform_pair(bc, grid.N[d]) for d in range(grid.dim)]
        self.lams = [eigenvalues(bc, grid.N[d], grid.h(d)) for d in range(grid.dim)]

    def forward(self, U: np.ndarray) -> np.ndarray:
        """F(U) = P_z (z) P_y (y) P_x (x) U  (Eqs. E19, E22)."""
        for d in range(self.grid.dim):
            U = apply_along(self.pairs[d][0], U, U.ndim - 1 - d)
        return U

    def inverse(self, U: np.ndarray) -> np.ndarray:
        """F^{-1}(U) = P_z^{-1} (z) P_y^{-1} (y) P_x^{-1} (x) U  (Eqs. E16-E18)."""
        for d in range(self.grid.dim):
            U = apply_along(self.pairs[d][1], U, U.ndim - 1 - d)
        return U

    def Lambda(self) -> np.ndarray:
        """Lambda_{n,m,l} = lambda_n + lambda_m + lambda_l on the field shape (reading R2)."""
        dim = self.grid.dim
        Lam = np.zeros(tuple(len(l) for l in reversed(self.lams)))
        for d in range(dim):
            shape = [1] * dim
            shape[dim - 1 - d] = len(self.lams[d])
            Lam = Lam + self.lams[d].reshape(shape)
        return Lam

    def Lambda_frac(self, alpha: float) -> np.ndarray:
        """Lambda^{alpha/2} with 0^{alpha/2} = 0 (MTT, Def. 1)."""
        return np.power(self.Lambda(), alpha / 2.0)

    def frac_laplacian(self, U: np.ndarray, alpha: float) -> np.ndarray:
        """(-Delta)^{alpha/2} U ~ F^{-1}(Lambda^{alpha/2} . F(U))  (Eqs. E16-E18)."""
        V = self.inverse(self.Lambda_frac(alpha) * self.forward(U))
        return V.real if self.bc == PERIODIC else V


# ---------------------------------------------------------------------------
# Section 4: Pade-(1,3) coefficients and the ETDRK4-P13 step
# ---------------------------------------------------------------------------

def pade13(z):
    """R_{1,3}(z) = (24 - 6z) / (24 + 18z + 6z^2 + z^3), the Pade-(1,3) approximant of e^{-z}."""
    return (24.0 - 6.0 * z) / (24.0 + 18.0 * z + 6.0 * z ** 2 + z ** 3)


def p13_coefficients(L, tau: float) -> dict:
    """The six arrays precomputed in Algorithm 1 from L = kappa tau Lambda^{alpha/2}."""
    D1 = 24.0 + 18.0 * L + 6.0 * L ** 2 + L ** 3
    D2 = 192.0 + 72.0 * L + 12.0 * L ** 2 + L ** 3
    return {
        "R13": (24.0 - 6.0 * L) / D1,
        "Q13": 24.0 * (8.0 - L) / D2,
        "phi": tau * (96.0 + 12.0 * L + L ** 2) / D2,
        "phi1": tau * (4.0 - L) / D1,
        "phi2": 2.0 * tau * (4.0 + L) / D1,
        "phi3": tau * (4.0 + 3.0 * L + L ** 2) / D1,
    }


def cox_matthews_coefficients(L, tau: float, npts: int = 64) -> dict:
    """The Cox-Matthews ETDRK4 coefficients (exact exponentials) in the places of Algorithm 1's six
    arrays, for the linear part u_t = -(L/tau) u, z = -L:
      R13 -> e^{z},  Q13 -> e^{z/2},  phi -> (tau/2) (e^{z/2} - 1)/(z/2),
      phi1 -> tau [-4 - z + e^{z}(4 - 3z + z^2)] / z^3,
      phi2 -> 2 tau [2 + z + e^{z}(z - 2)] / z^3,
      phi3 -> tau [-4 - 3z - z^2 + e^{z}(4 - z)] / z^3,
    i.e. Algorithm 1 with R13(L) replaced by e^{-L}.  These forms cancel as z -> 0.  For |z| < 2
    each function is evaluated as its mean over a circle centred at its argument (the trapezoidal
    rule of the Cauchy integral, npts points, as Kassam and Trefethen do for the ETDRK4
    coefficients), with radius |z| + 1 so that the circle never comes closer than 1 to the origin,
    where the forms cancel; for |z| >= 2 the forms are evaluated directly (they lose at most a factor
    of about 30 there).  This is the exponential-integrator scheme the P13 scheme approximates."""
    L = np.asarray(L, dtype=np.float64)
    z = -L
    unit = np.exp(2j * np.pi * (np.arange(npts) + 0.5) / npts)

    def phi_forms(Z):
        eZ = np.exp(Z)
        Z3 = Z ** 3
        return ((-4.0 - Z + eZ * (4.0 - 3.0 * Z + Z ** 2)) / Z3,
                (2.0 + Z + eZ * (Z - 2.0)) / Z3,
                (-4.0 - 3.0 * Z - Z ** 2 + eZ * (4.0 - Z)) / Z3)

    def psi1(Z):
        return (np.exp(Z) - 1.0) / Z

    def contour(f, w):
        pts = w[..., None] + (np.abs(w)[..., None] + 1.0) * unit
        return f(pts).mean(axis=-1).real

    near = np.abs(z) < 2.0
    zs = np.where(near, 3.0, z)          # any value with |zs| >= 2 where the direct forms are not used
    d1, d2, d3 = phi_forms(zs)
    w = z / 2
    ws = np.where(np.abs(w) < 2.0, 3.0, w)
    phi_w = np.where(np.abs(w) < 2.0, contour(psi1, w), psi1(ws))
    c1 = np.where(near, contour(lambda Z: phi_forms(Z)[0], z), d1)
    c2 = np.where(near, contour(lambda Z: phi_forms(Z)[1], z), d2)
    c3 = np.where(near, contour(lambda Z: phi_forms(Z)[2], z), d3)
    return {
        "R13": np.exp(z),
        "Q13": np.exp(w),
        "phi": tau / 2 * phi_w,
        "phi1": tau * c1,
        "phi2": 2.0 * tau * c2,
        "phi3": tau * c3,
    }


SCHEMES = {"p13": p13_coefficients, "cox_matthews": cox_matthews_coefficients}


Reaction = Callable[[list, float], list]


@dataclass
class Problem:
    """u_t = -kappa_s (-Delta)^{alpha_s/2} u_s + f_s(u, t) on a box (Eq. 1), one entry per species."""
    grid: Grid
    bc: str
    alpha: Sequence[float]
    kappa: Sequence[float]
    tau: float
    reaction: Reaction
    dreaction: Callable | None = None     # (u, t) -> Jacobian J[s][r] = d f_s / d u_r (arrays)
    nspecies: int = 2
    extra: dict = field(default_factory=dict)


class ETDRK4P13:
    """Algorithm 1 of the paper for any dimension, boundary condition and species count.
    scheme "cox_matthews" runs the same stages with the exact-exponential coefficients
    (cox_matthews_coefficients) instead of the Pade-(1,3) ones."""

    def __init__(self, prob: Problem, scheme: str = "p13"):
        self.prob = prob
        self.scheme = scheme
        self.sp = Spectral(prob.grid, prob.bc)
        self.L = [prob.kappa[s] * prob.tau * self.sp.Lambda_frac(prob.alpha[s])
                  for s in range(prob.nspecies)]
        self.coef = [SCHEMES[scheme](L, prob.tau) for L in self.L]

    def _real(self, V):
        return V.real if self.prob.bc == PERIODIC else V

    def step(self, u: list, t: float) -> list:
        """One step k -> k+1 (Algorithm 1, loop body), t = t_k."""
        F, Fi, tau, S = self.sp.forward, self.sp.inverse, self.prob.tau, self.prob.nspecies
        c = self.coef
        f = self.prob.reaction
        u_h = [F(u[s]) for s in range(S)]
        f_u = f(u, t)
        a = [self._real(Fi(c[s]["Q13"] * u_h[s] + c[s]["phi"] * F(f_u[s]))) for s in range(S)]
        f_a = f(a, t + tau / 2)
        b = [self._real(Fi(c[s]["Q13"] * u_h[s] + c[s]["phi"] * F(f_a[s]))) for s in range(S)]
        f_b = f(b, t + tau / 2)
        cc = [self._real(Fi(c[s]["Q13"] * F(a[s]) + c[s]["phi"] * F(2 * f_b[s] - f_u[s])))
              for s in range(S)]
        f_c = f(cc, t + tau)
        return [self._real(Fi(c[s]["R13"] * u_h[s] + c[s]["phi1"] * F(f_u[s])
                              + c[s]["phi2"] * F(f_a[s] + f_b[s]) + c[s]["phi3"] * F(f_c[s])))
                for s in range(S)]

    def run(self, u0: list, t0: float, nsteps: int) -> list:
        """M steps from t_0 (t_k = t_0 + k tau, Algorithm 1)."""
        u = [np.array(x, dtype=np.float64) for x in u0]
        for k in range(nsteps):
            u = self.step(u, t0 + k * self.prob.tau)
        return u

    # -- discrete adjoint ---------------------------------------------------
    #
    # The step above is u' = G(u; theta).  For a loss l(u'), the reverse-mode
    # derivative of the same arithmetic is taken operation by operation: each
    # linear map M (a transform, a diagonal scaling) contributes M^T to the
    # backward sweep, the reaction contributes its Jacobian transposed.  For the
    # periodic case the complex transforms are real-linear maps on real data,
    # and the real adjoint of  x -> Re(Fi(D F x))  is  y -> Re(F^H D^* Fi^H y),
    # with F^H = conj(F)^T.

    def _adj_F(self, Y):
        """Transpose (real-linear adjoint) of the forward transform."""
        for d in range(self.prob.grid.dim):
            Y = apply_along(np.conj(self.sp.pairs[d][0]).T, Y, Y.ndim - 1 - d)
        return Y

    def _adj_Fi(self, Y):
        for d in range(self.prob.grid.dim):
            Y = apply_along(np.conj(self.sp.pairs[d][1]).T, Y, Y.ndim - 1 - d)
        return Y

    def step_vjp(self, u: list, t: float, gbar: list, dcoef: dict | None = None,
                 dparams: Callable | None = None) -> tuple:
        """Reverse sweep of one step: returns (ubar, coefficient-bar dict, params-bar).

        gbar = dl/du' on the new state.  dcoef[s][name] receives dl/d(coefficient
        array) for each of the six arrays (used for dl/d alpha and dl/d kappa by the
        chain rule through L), and dparams(u_stage, t, wbar) -> dl/dtheta for the
        reaction parameters.
        """
        F, Fi, tau, S = self.sp.forward, self.sp.inverse, self.prob.tau, self.prob.nspecies
        aF, aFi = self._adj_F, self._adj_Fi
        c = self.coef
        f, J = self.prob.reaction, self.prob.dreaction
        R = self._real
        conj = np.conj
        # forward recomputation, keeping every intermediate
        u_h = [F(u[s]) for s in range(S)]
        f_u = f(u, t)
        Ffu = [F(f_u[s]) for s in range(S)]
        a = [R(Fi(c[s]["Q13"] * u_h[s] + c[s]["phi"] * Ffu[s])) for s in range(S)]
        f_a = f(a, t + tau / 2)
        Ffa = [F(f_a[s]) for s in range(S)]
        b = [R(Fi(c[s]["Q13"] * u_h[s] + c[s]["phi"] * Ffa[s])) for s in range(S)]
        f_b = f(b, t + tau / 2)
        Fa = [F(a[s]) for s in range(S)]
        Fbu = [F(2 * f_b[s] - f_u[s]) for s in range(S)]
        cc = [R(Fi(c[s]["Q13"] * Fa[s] + c[s]["phi"] * Fbu[s])) for s in range(S)]
        f_c = f(cc, t + tau)
        Fab = [F(f_a[s] + f_b[s]) for s in range(S)]
        Ffc = [F(f_c[s]) for s in range(S)]

        def cbar(s, name, X, Ybar):
            if dcoef is not None:
                dcoef[s][name] = dcoef[s].get(name, 0.0) + (conj(X) * Ybar).real

        zero = [np.zeros_like(u[s]) for s in range(S)]
        u_bar = [z.copy() for z in zero]
        fu_bar = [z.copy() for z in zero]
        fa_bar = [z.copy() for z in zero]
        fb_bar = [z.copy() for z in zero]
        fc_bar = [z.copy() for z in zero]
        a_bar = [z.copy() for z in zero]
        uh_bar = [0.0] * S
        p_bar = 0.0
        # u' = Re Fi( R13 uh + phi1 F fu + phi2 F(fa + fb) + phi3 F fc )
        for s in range(S):
            Z = aFi(gbar[s].astype(complex) if self.prob.bc == PERIODIC else gbar[s])
            uh_bar[s] = c[s]["R13"] * Z
            cbar(s, "R13", u_h[s], Z)
            cbar(s, "phi1", Ffu[s], Z)
            cbar(s, "phi2", Fab[s], Z)
            cbar(s, "phi3", Ffc[s], Z)
            fu_bar[s] = fu_bar[s] + R(aF(c[s]["phi1"] * Z))
            t2 = R(aF(c[s]["phi2"] * Z))
            fa_bar[s] = fa_bar[s] + t2
            fb_bar[s] = fb_bar[s] + t2
            fc_bar[s] = fc_bar[s] + R(aF(c[s]["phi3"] * Z))
        # f_c = f(c, t + tau)
        c_bar = self._react_vjp(J, cc, t + tau, fc_bar)
        if dparams is not None:
            p_bar = p_bar + dparams(cc, t + tau, fc_bar)
        # c = Re Fi( Q13 F a + phi F(2 fb - fu) )
        for s in range(S):
            Z = aFi(c_bar[s].astype(complex) if self.prob.bc == PERIODIC else c_bar[s])
            cbar(s, "Q13", Fa[s], Z)
            cbar(s, "phi", Fbu[s], Z)
            a_bar[s] = a_bar[s] + R(aF(c[s]["Q13"] * Z))
            t2 = R(aF(c[s]["phi"] * Z))
            fb_bar[s] = fb_bar[s] + 2 * t2
            fu_bar[s] = fu_bar[s] - t2
        # f_b = f(b, t + tau/2)
        b_bar = self._react_vjp(J, b, t + tau / 2, fb_bar)
        if dparams is not None:
            p_bar = p_bar + dparams(b, t + tau / 2, fb_bar)
        # b = Re Fi( Q13 uh + phi F fa )
        for s in range(S):
            Z = aFi(b_bar[s].astype(complex) if self.prob.bc == PERIODIC else b_bar[s])
            cbar(s, "Q13", u_h[s], Z)
            cbar(s, "phi", Ffa[s], Z)
            uh_bar[s] = uh_bar[s] + c[s]["Q13"] * Z
            fa_bar[s] = fa_bar[s] + R(aF(c[s]["phi"] * Z))
        # f_a = f(a, t + tau/2)
        ga = self._react_vjp(J, a, t + tau / 2, fa_bar)
        if dparams is not None:
            p_bar = p_bar + dparams(a, t + tau / 2, fa_bar)
        for s in range(S):
            a_bar[s] = a_bar[s] + ga[s]
        # a = Re Fi( Q13 uh + phi F fu )
        for s in range(S):
            Z = aFi(a_bar[s].astype(complex) if self.prob.bc == PERIODIC else a_bar[s])
            cbar(s, "Q13", u_h[s], Z)
            cbar(s, "phi", Ffu[s], Z)
            uh_bar[s] = uh_bar[s] + c[s]["Q13"] * Z
            fu_bar[s] = fu_bar[s] + R(aF(c[s]["phi"] * Z))
        # f_u = f(u, t)
        gu = self._react_vjp(J, u, t, fu_bar)
        if dparams is not None:
            p_bar = p_bar + dparams(u, t, fu_bar)
        # u_h = F u
        for s in range(S):
            u_bar[s] = gu[s] + R(aF(uh_bar[s]))
        return u_bar, p_bar

    @staticmethod
    def _react_vjp(J, u, t, wbar):
        Jm = J(u, t)
        S = len(u)
        return [sum(Jm[r][s] * wbar[r] for r in range(S)) for s in range(S)]


def coefficient_derivatives(L, tau: float) -> dict:
    """d(coefficient)/dL for the six arrays of Algorithm 1 (quotient rule on the printed rationals)."""
    D1 = 24.0 + 18.0 * L + 6.0 * L ** 2 + L ** 3
    D2 = 192.0 + 72.0 * L + 12.0 * L ** 2 + L ** 3
    dD1 = 18.0 + 12.0 * L + 3.0 * L ** 2
    dD2 = 72.0 + 24.0 * L + 3.0 * L ** 2

    def q(n, dn, d, dd):
        return (dn * d - n * dd) / (d * d)

    return {
        "R13": q(24.0 - 6.0 * L, -6.0, D1, dD1),
        "Q13": q(24.0 * (8.0 - L), -24.0, D2, dD2),
        "phi": tau * q(96.0 + 12.0 * L + L ** 2, 12.0 + 2.0 * L, D2, dD2),
        "phi1": tau * q(4.0 - L, -1.0, D1, dD1),
        "phi2": 2.0 * tau * q(4.0 + L, 1.0, D1, dD1),
        "phi3": tau * q(4.0 + 3.0 * L + L ** 2, 3.0 + 2.0 * L, D1, dD1),
    }


def cox_matthews_derivatives(L, tau: float, npts: int = 64) -> dict:
    """d(coefficient)/dL for the six Cox-Matthews arrays of cox_matthews_coefficients.

    Each coefficient is an entire function c(z) of z = -L (the forms' poles at 0 are removable), so
    its derivative is the Cauchy integral dc/dz = (1/2 pi i) [contour integral of] c(w) / (w - z)^2 dw, i.e. the mean
    of c(w) / (w - z) over a circle around z.  The radius is |z| + 1 for |z| < 2 (the circle keeps a
    distance of 1 from the origin, where the forms cancel) and 1 otherwise (every point then has
    |w| >= 1 and Re w <= -1: no cancellation beyond the forms' own, no overflow).  dc/dL = -dc/dz."""
    L = np.asarray(L, dtype=np.float64)
    z = -L
    unit = np.exp(2j * np.pi * (np.arange(npts) + 0.5) / npts)

    def forms(Z):
        eZ = np.exp(Z)
        Z3 = Z ** 3
        return {"R13": eZ,
                "Q13": np.exp(Z / 2),
                "phi": tau / 2 * (np.exp(Z / 2) - 1.0) / (Z / 2),
                "phi1": tau * (-4.0 - Z + eZ * (4.0 - 3.0 * Z + Z ** 2)) / Z3,
                "phi2": 2.0 * tau * (2.0 + Z + eZ * (Z - 2.0)) / Z3,
                "phi3": tau * (-4.0 - 3.0 * Z - Z ** 2 + eZ * (4.0 - Z)) / Z3}

    r = np.where(np.abs(z) < 2.0, np.abs(z) + 1.0, 1.0)
    pts = z[..., None] + r[..., None] * unit
    vals = forms(pts)
    return {k: -(v / (pts - z[..., None])).mean(axis=-1).real for k, v in vals.items()}


COEFFICIENT_DERIVATIVES = {"p13": coefficient_derivatives, "cox_matthews": cox_matthews_derivatives}


def adjoint_run(solver: ETDRK4P13, u0: list, t0: float, nsteps: int, dldu_T: list,
                dparams: Callable | None = None) -> dict:
    """Gradient of l(u_M) through M steps: dl/du0, dl/dalpha_s, dl/dkappa_s, dl/dtheta.

    Stores every state (no checkpointing) and sweeps the steps in reverse.
    dl/dkappa_s = sum dl/dC * dC/dL * tau Lambda^{alpha_s/2};
    dl/dalpha_s = sum dl/dC * dC/dL * kappa_s tau Lambda^{alpha_s/2} ln(Lambda)/2 (0 where Lambda = 0).
    """
    prob = solver.prob
    S = prob.nspecies
    states = [[np.array(x, dtype=np.float64) for x in u0]]
    for k in range(nsteps):
        states.append(solver.step(states[-1], t0 + k * prob.tau))
    gbar = [np.array(g, dtype=np.float64) for g in dldu_T]
    dcoef = [dict() for _ in range(S)]
    p_bar = 0.0
    for k in reversed(range(nsteps)):
        gbar, pb = solver.step_vjp(states[k], t0 + k * prob.tau, gbar, dcoef, dparams)
        p_bar = p_bar + pb
    Lam = solver.sp.Lambda()
    logLam = np.where(Lam > 0, np.log(np.where(Lam > 0, Lam, 1.0)), 0.0)
    dalpha, dkappa = [], []
    for s in range(S):
        dC = COEFFICIENT_DERIVATIVES[solver.scheme](solver.L[s], prob.tau)
        dLdC = sum((dcoef[s].get(n, 0.0) * dC[n]).sum() for n in dC) if dcoef[s] else 0.0
        g_L = sum(dcoef[s].get(n, 0.0) * dC[n] for n in dC) if dcoef[s] else 0.0
        Lf = solver.sp.Lambda_frac(prob.alpha[s])
        dkappa.append(float(np.sum(g_L * prob.tau * Lf)))
        dalpha.append(float(np.sum(g_L * prob.kappa[s] * prob.tau * Lf * 0.5 * logLam)))
        del dLdC
    return {"u0": gbar, "alpha": dalpha, "kappa": dkappa, "params": p_bar, "uT": states[-1]}


# ---------------------------------------------------------------------------
# Reaction terms (Section 5 and the workload definitions)
# ---------------------------------------------------------------------------

def fitzhugh_nagumo(mu=0.1, eps=0.01, beta=0.5, gamma=1.0, delta=0.0) -> tuple:
    """f_u = u(1-u)(u-mu) - v,  f_v = eps(beta u - gamma v - delta)  (Section 5.2, FHN)."""
    def f(w, t):
        u, v = w
        return [u * (1 - u) * (u - mu) - v, eps * (beta * u - gamma * v - delta)]

    def J(w, t):
        u, v = w
        return [[-3 * u * u + 2 * (1 + mu) * u - mu, -np.ones_like(u)],
                [eps * beta * np.ones_like(u), -eps * gamma * np.ones_like(u)]]

    def dmu(w, t, wbar):
        # d f_u / d mu = -u(1-u)
        u, v = w
        return float(np.sum(wbar[0] * (-u * (1 - u))))
    return f, J, dmu


def gray_scott(F=0.04, K=0.06) -> tuple:
    """f_u = -u v^2 + F(1-u),  f_v = u v^2 - (F+K) v  (Section 5.2, Gray-Scott)."""
    def f(w, t):
        u, v = w
        return [-u * v * v + F * (1 - u), u * v * v - (F + K) * v]

    def J(w, t):
        u, v = w
        return [[-v * v - F, -2 * u * v], [v * v, 2 * u * v - (F + K)]]
    return f, J


def schnakenberg(gamma=1000.0, a=0.1, b=0.9, ustar=(0.0, 0.0)) -> tuple:
    """f_u = gamma(a - U + U^2 V), f_v = gamma(b - U^2 V), U = u* + w_u, V = v* + w_v (Section 5.2)."""
    def f(w, t):
        U, V = w[0] + ustar[0], w[1] + ustar[1]
        return [gamma * (a - U + U * U * V), gamma * (b - U * U * V)]

    def J(w, t):
        U, V = w[0] + ustar[0], w[1] + ustar[1]
        return [[gamma * (-1 + 2 * U * V), gamma * U * U], [-gamma * 2 * U * V, -gamma * U * U]]
    return f, J


def gierer_meinhardt(c1=1.0, c2=1.0, c3=1.0, c4=1.0) -> tuple:
    """f_u = c1 u^2 / v - c2 u,  f_v = c3 u^2 - c4 v  (Eq. GM with its constants as parameters)."""
    def f(w, t):
        u, v = w
        return [c1 * u * u / v - c2 * u, c3 * u * u - c4 * v]

    def J(w, t):
        u, v = w
        return [[2 * c1 * u / v - c2, -c1 * u * u / (v * v)], [2 * c3 * u, -c4 * np.ones_like(u)]]
    return f, J


def linear(gamma: float) -> tuple:
    """f(u) = gamma u: the test equation of the linear stability analysis (Eq. TEq)."""
    def f(w, t):
        return [gamma * x for x in w]

    def J(w, t):
        S = len(w)
        return [[gamma * np.ones_like(w[0]) if r == s else np.zeros_like(w[0]) for s in range(S)]
                for r in range(S)]
    return f, J


def fisher_mms(grid: Grid, kappa: float, alpha: float):
    """Example 1: f(u,t) = -2e^{-t}s^3 + (kappa/4)e^{-t}(3(2pi)^a sin 2pi x - (6pi)^a sin 6pi x)
    + e^{-2t}s^6 + u - u^2, s = sin(2 pi x)  (reading R8: a single kappa)."""
    x = grid.mesh(DIRICHLET)[0]
    s = np.sin(2 * np.pi * x)
    src = (kappa / 4.0) * (3 * (2 * np.pi) ** alpha * np.sin(2 * np.pi * x)
                           - (6 * np.pi) ** alpha * np.sin(6 * np.pi * x))

    def f(w, t):
        u = w[0]
        e = math.exp(-t)
        return [-2 * e * s ** 3 + e * src + e * e * s ** 6 + u - u * u]

    def exact(t):
        return math.exp(-t) * s ** 3
    return f, exact


def huxley_mms(grid: Grid, bc: str, kappa: float, alpha: float):
    """Example 2: u(1-u)(u-1) + source with exact u = t^alpha cos^3(2pi x) cos^3(2pi y) (reading R10)."""
    X, Y = grid.mesh(bc)
    g = np.cos(2 * np.pi * X) ** 3 * np.cos(2 * np.pi * Y) ** 3
    c = np.cos
    Phi = (kappa / 16.0) * (9 * (8 * np.pi ** 2) ** (alpha / 2) * c(2 * np.pi * X) * c(2 * np.pi * Y)
                            + 3 * (40 * np.pi ** 2) ** (alpha / 2) * c(6 * np.pi * X) * c(2 * np.pi * Y)
                            + 3 * (40 * np.pi ** 2) ** (alpha / 2) * c(2 * np.pi * X) * c(6 * np.pi * Y)
                            + (72 * np.pi ** 2) ** (alpha / 2) * c(6 * np.pi * X) * c(6 * np.pi * Y))

    def f(w, t):
        u = w[0]
        ta = t ** alpha
        tam1 = alpha * t ** (alpha - 1) if t > 0 else 0.0
        src = tam1 * g + ta * Phi - ta * g * (1 - ta * g) * (ta * g - 1)
        return [u * (1 - u) * (u - 1) + src]

    def exact(t):
        return t ** alpha * g
    return f, exact


# ---------------------------------------------------------------------------
# Section 5: error norm, linear analysis
# ---------------------------------------------------------------------------

def max_error(u, v) -> float:
    """||u - v||_inf over the grid (Section 5)."""
    return float(np.max(np.abs(np.asarray(u) - np.asarray(v))))


def rel_max(x: Sequence, y: Sequence) -> float:
    """max|x - y| / max|y| over all unknowns of all species."""
    num = max(float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) for a, b in zip(x, y))
    den = max(float(np.max(np.abs(np.asarray(b)))) for b in y)
    return num / den


def rel_l2(x: Sequence, y: Sequence) -> float:
    """||x - y||_2 / ||y||_2 over all unknowns of all species."""
    num = sum(float(np.sum((np.asarray(a, dtype=np.float64) - np.asarray(b)) ** 2)) for a, b in zip(x, y))
    den = sum(float(np.sum(np.asarray(b) ** 2)) for b in y)
    return math.sqrt(num / den)
