"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than the oracle's own
formula: a dense eigendecomposition of the printed matrices, a banded solve of
the classical compact scheme, the published Cox-Matthews ETDRK4 coefficients,
the paper's closed-form amplification factor (Eq. 41), the RK4 reduction, exact
single-mode decay, and the error tables printed in Section 5 (Tables 1 and 2).
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def _same_to_printed_digits(value, printed):
    """True when `value` rounds to the printed 5-significant-digit number."""
    return float("%.4e" % value) == printed


# --------------------------------------------------------------------------
# Section 3.1: eigenvalues and eigenvectors of the compact Laplacian
# --------------------------------------------------------------------------

@pytest.mark.parametrize("bc", O.BCS)
@pytest.mark.parametrize("N", [4, 7, 8, 12, 16])
def test_eigenvalues_match_dense_eig_of_printed_matrices(bc, N):
    h = 0.37
    A, B = O.compact_matrices(bc, N, h)
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(A, B)).real)
    closed = np.sort(O.eigenvalues(bc, N, h))
    assert len(ev) == len(closed)
    np.testing.assert_allclose(closed, ev, rtol=1e-10, atol=1e-10 * ev.max())


@pytest.mark.parametrize("bc", O.BCS)
@pytest.mark.parametrize("N", [5, 8, 16])
def test_transform_pair_diagonalises_A_inv_B(bc, N):
    """T = Finv diag(lambda) F must equal A^{-1} B entry by entry (fixes the eigenvector
    order, the transform direction and the Neumann reading)."""
    h = 1.0 / N
    A, B = O.compact_matrices(bc, N, h)
    T = np.linalg.solve(A, B)
    F, Fi = O.transform_pair(bc, N)
    lam = O.eigenvalues(bc, N, h)
    T2 = Fi @ np.diag(lam) @ F
    assert np.max(np.abs(T2.imag if np.iscomplexobj(T2) else 0.0)) < 1e-9 * np.abs(T).max()
    np.testing.assert_allclose(T2.real, T, atol=1e-10 * np.abs(T).max())
    np.testing.assert_allclose((Fi @ F).real, np.eye(len(lam)), atol=1e-12)


def test_printed_periodic_angle_is_not_an_eigenvalue():
    """The printed periodic angle (n-1) pi / (2N) gives a different spectrum; the corrected one matches."""
    N, h = 8, 0.125
    A, B = O.compact_matrices(O.PERIODIC, N, h)
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(A, B)).real)
    n = np.arange(1, N + 1)
    s = np.sin((n - 1) * np.pi / (2 * N)) ** 2
    printed = np.sort(4 * s / (h * h * (1 - s / 3)))
    assert np.max(np.abs(printed - ev)) > 1.0
    np.testing.assert_allclose(np.sort(O.eigenvalues(O.PERIODIC, N, h)), ev, rtol=1e-10, atol=1e-9)


@pytest.mark.parametrize("bc", O.BCS)
@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.9])
def test_fractional_power_matches_numeric_eigendecomposition(bc, alpha):
    """T^{alpha/2} = P Lambda^{alpha/2} P^{-1} from a numerical eig (Lemma 1) vs the closed form."""
    N, h = 12, 1.0 / 12
    A, B = O.compact_matrices(bc, N, h)
    T = np.linalg.solve(A, B)
    w, V = np.linalg.eig(T)
    w = np.where(np.abs(w) < 1e-9, 0.0, w.real)
    Tf = (V @ np.diag(np.power(w, alpha / 2)) @ np.linalg.inv(V)).real
    F, Fi = O.transform_pair(bc, N)
    lam = O.eigenvalues(bc, N, h)
    closed = (Fi @ np.diag(np.power(lam, alpha / 2)) @ F).real
    np.testing.assert_allclose(closed, Tf, atol=1e-9 * np.abs(Tf).max())
    if bc == O.DIRICHLET:       # SPD: also against scipy's Schur-Pade fractional power
        Tsp = sla.fractional_matrix_power(T, alpha / 2).real
        np.testing.assert_allclose(closed, Tsp, atol=1e-8 * np.abs(Tsp).max())


@pytest.mark.parametrize("bc", O.BCS)
def test_alpha2_reduces_to_classical_compact_scheme_2d(bc):
    """At alpha = 2 the MTT operator is T_x (x) U + T_y (y) U (Eq. EP) with T v = A^{-1}(B v)
    computed by a banded (or cyclic) solve."""
    Nx, Ny = 10, 14
    g = O.Grid((Nx, Ny), (0.0, -1.0), (1.3, 2.0))
    sp = O.Spectral(g, bc)
    U = np.random.default_rng(7).standard_normal(g.shape(bc))

    def T_apply(N, h, V, axis):
        A, B = O.compact_matrices(bc, N, h)
        BV = np.moveaxis(np.tensordot(B, V, axes=([1], [axis])), 0, axis)
        if bc == O.PERIODIC:
            return np.moveaxis(np.tensordot(np.linalg.inv(A), BV, axes=([1], [axis])), 0, axis)
        n = A.shape[0]
        ab = np.zeros((3, n))
        ab[0, 1:] = np.diag(A, 1)
        ab[1, :] = np.diag(A)
        ab[2, :-1] = np.diag(A, -1)
        moved = np.moveaxis(BV, axis, 0)
        sol = sla.solve_banded((1, 1), ab, moved.reshape(n, -1)).reshape(moved.shape)
        return np.moveaxis(sol, 0, axis)

    ref = T_apply(Nx, g.h(0), U, 1) + T_apply(Ny, g.h(1), U, 0)
    got = sp.frac_laplacian(U, 2.0)
    np.testing.assert_allclose(got, ref, atol=1e-9 * np.abs(ref).max())


def test_compact_laplacian_is_fourth_order():
    """-Delta sin(pi x) on Dirichlet grids: error of A^{-1}B falls by ~16 per halving (Eq. Lap)."""
    errs = []
    for N in (16, 32, 64):
        h = 1.0 / N
        x = np.arange(1, N) * h
        F, Fi = O.transform_pair(O.DIRICHLET, N)
        lam = O.eigenvalues(O.DIRICHLET, N, h)
        v = np.sin(np.pi * x)
        errs.append(np.max(np.abs(Fi @ (lam * (F @ v)) - np.pi ** 2 * v)))
    assert 15.0 < errs[0] / errs[1] < 17.0 and 15.0 < errs[1] / errs[2] < 17.0


# --------------------------------------------------------------------------
# Section 4: Pade-(1,3) coefficients
# --------------------------------------------------------------------------

def test_pade13_is_fourth_order_approximation_of_exp():
    z = np.array([1e-2, 2e-2, 4e-2])
    err = np.abs(O.pade13(z) - np.exp(-z))
    ratios = err[1:] / err[:-1]
    np.testing.assert_allclose(ratios, 32.0, rtol=0.05)   # O(z^5)


@pytest.mark.parametrize("L", [1e-3, 0.25, 1.0, 4.6, 36.0, 1e3])
def test_coefficients_equal_cox_matthews_with_pade_exponential(L):
    """Algorithm 1's rationals equal the Cox-Matthews ETDRK4 coefficients with e^{-L} replaced
    by R13(L) (and e^{-L/2} by R13(L/2) = Q13)."""
    tau = 0.37
    c = O.p13_coefficients(L, tau)
    R, Q = O.pade13(L), O.pade13(L / 2)
    assert c["R13"] == pytest.approx(R, rel=1e-13)
    assert c["Q13"] == pytest.approx(Q, rel=1e-13)
    assert c["phi"] == pytest.approx(tau * (1 - Q) / L, rel=1e-8 if L < 1e-2 else 1e-12)
    if L > 0.2:   # the Cox-Matthews forms cancel catastrophically for small L
        assert c["phi1"] == pytest.approx(tau * (-4 + L + R * (4 + 3 * L + L * L)) / (-L ** 3), rel=1e-10)
        assert c["phi2"] == pytest.approx(2 * tau * (2 - L - R * (2 + L)) / (-L ** 3), rel=1e-10)
        assert c["phi3"] == pytest.approx(tau * (-4 + 3 * L - L * L + R * (4 + L)) / (-L ** 3), rel=1e-10)


def test_coefficients_zero_eigenvalue_limits():
    tau = 0.1
    c = O.p13_coefficients(np.array([0.0]), tau)
    assert c["R13"][0] == 1.0 and c["Q13"][0] == 1.0
    assert c["phi"][0] == pytest.approx(tau / 2)
    assert c["phi1"][0] == pytest.approx(tau / 6)
    assert c["phi2"][0] == pytest.approx(tau / 3)
    assert c["phi3"][0] == pytest.approx(tau / 6)


def test_coefficient_derivatives_match_finite_differences():
    tau = 0.3
    for L in (0.0, 0.7, 5.0, 40.0):
        d = O.coefficient_derivatives(L, tau)
        hh = 1e-6 * max(1.0, L)
        cp, cm = O.p13_coefficients(L + hh, tau), O.p13_coefficients(L - hh, tau)
        for k in d:
            assert d[k] == pytest.approx((cp[k] - cm[k]) / (2 * hh), rel=1e-6, abs=1e-9)


# --------------------------------------------------------------------------
# Section 4.2: linear analysis
# --------------------------------------------------------------------------

def eq41(x, y):
    """Amplification factor of Eq. 41 as printed, with the y^2 term of c1's numerator restored
    (+55738368 y^2; symbolic derivation from the scheme)."""
    d1 = 24 - 18 * y + 6 * y ** 2 - y ** 3
    d2 = 192 - 72 * y + 12 * y ** 2 - y ** 3
    c0 = 6 * (4 + y) / d1
    c1 = (169869312 - 148635648 * y + 55738368 * y ** 2 - 9621504 * y ** 3 + 470016 * y ** 4
          + 165888 * y ** 5 - 46464 * y ** 6 + 6240 * y ** 7 - 600 * y ** 8 + 32 * y ** 9
          - y ** 10) / (d2 ** 3 * d1)
    c2 = (442368 - 221184 * y + 34560 * y ** 2 + 11712 * y ** 3 - 2976 * y ** 4 + 404 * y ** 5
          - 25 * y ** 6 + y ** 7) / (d2 ** 2 * d1)
    c3 = 2 * (96 - 12 * y + y ** 2) ** 2 * (1536 - 960 * y + 240 * y ** 2 + 8 * y ** 3 + y ** 4) / (d2 ** 3 * d1)
    c4 = 2 * (96 - 12 * y + y ** 2) ** 3 * (4 - 3 * y + y ** 2) / (d2 ** 3 * d1)
    return c0 + c1 * x + c2 * x ** 2 + c3 * x ** 3 + c4 * x ** 4


def _one_mode_factor(bc, N, mode, x, y_target, alpha=1.6):
    """Apply one oracle step to a single eigenmode with f(u) = gamma u; return u^{k+1}/u^k."""
    g = O.Grid((N,), (0.0,), (1.0,))
    sp = O.Spectral(g, bc)
    lam = sp.Lambda_frac(alpha)
    tau = 0.05
    kappa = -y_target / (tau * lam[mode])      # y = -kappa tau lambda^{alpha/2}
    gamma = x / tau
    f, J = O.linear(gamma)
    prob = O.Problem(g, bc, [alpha], [kappa], tau, f, dreaction=J, nspecies=1)
    s = O.ETDRK4P13(prob)
    coef = np.zeros(len(lam))
    coef[mode] = 1.0
    u0 = sp.inverse(coef)
    u0 = u0.real if bc == O.PERIODIC else u0
    u1 = s.step([u0], 0.0)[0]
    return float(np.dot(u1, u0) / np.dot(u0, u0))


@pytest.mark.parametrize("bc,mode", [(O.DIRICHLET, 2), (O.NEUMANN, 3)])
@pytest.mark.parametrize("x,y", [(-0.5, -1.0), (0.3, -4.0), (-2.0, -20.0), (1.0, -0.2), (-0.1, -60.0)])
def test_step_reproduces_amplification_factor_eq41(bc, mode, x, y):
    assert _one_mode_factor(bc, 16, mode, x, y) == pytest.approx(eq41(x, y), rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("x", [-2.5, -1.0, -0.3, 0.4])
def test_eq41_at_y0_is_rk4(x):
    assert eq41(x, 0.0) == pytest.approx(1 + x + x * x / 2 + x ** 3 / 6 + x ** 4 / 24, rel=1e-14)


def test_single_eigenmode_decays_by_r13_power():
    """f = 0: each eigen-coefficient is multiplied by R13(L) per step, exactly."""
    N, M = 16, 7
    g = O.Grid((N, N), (0.0, 0.0), (2.0, 2.0))
    f, J = O.linear(0.0)
    for bc in O.BCS:
        prob = O.Problem(g, bc, [1.7], [0.3], 0.2, f, dreaction=J, nspecies=1)
        s = O.ETDRK4P13(prob)
        rng = np.random.default_rng(3)
        u0 = rng.standard_normal(g.shape(bc))
        uM = s.run([u0], 0.0, M)[0]
        expect = s.sp.forward(u0) * s.coef[0]["R13"] ** M
        got = s.sp.forward(uM)
        np.testing.assert_allclose(got, expect, atol=1e-12 * np.abs(expect).max())


def _closed_form_lambda(bc, n, N, h):
    """The compact scheme's eigenvalue of mode n on N intervals (Section 3.1; periodic angle by reading R1)."""
    s = math.sin(n * math.pi / N) ** 2 if bc == O.PERIODIC else math.sin(n * math.pi / (2 * N)) ** 2
    return 4.0 * s / (h * h * (1.0 - s / 3.0))


def _closed_form_mode(bc, n, N):
    """The grid function of mode n at the unknowns: cos(2 pi n i / N), i < N (periodic); sin(n pi i / N),
    0 < i < N (Dirichlet); cos(n pi i / N), 0 <= i <= N (Neumann)."""
    if bc == O.PERIODIC:
        return np.cos(2 * np.pi * n * np.arange(N) / N)
    if bc == O.DIRICHLET:
        return np.sin(np.pi * n * np.arange(1, N) / N)
    return np.cos(np.pi * n * np.arange(N + 1) / N)


@pytest.mark.parametrize("bc", O.BCS)
def test_separable_3d_eigenmodes_decay_by_closed_form_r13(bc):
    """f = 0 on a 3D grid with different sides: a product of 1D modes is an eigenvector of the summed operator
    with eigenvalue lambda_x + lambda_y + lambda_z (closed forms of Section 3), so after M steps it is scaled
    by R13(L)^M with L = kappa tau (lambda_x + lambda_y + lambda_z)^{alpha/2} (Eqs. E22 and ETDRK4P13),
    R13(L) = (24 - 6L) / (24 + 18L + 6L^2 + L^3).  The expected field uses none of the oracle's tables."""
    Ns, lo, hi = (8, 10, 6), (0.0, -1.0, 0.5), (1.0, 1.5, 2.0)
    alpha, kappa, tau, M = 1.6, 0.7, 0.05, 5
    g = O.Grid(Ns, lo, hi)
    f, J = O.linear(0.0)
    s = O.ETDRK4P13(O.Problem(g, bc, [alpha], [kappa], tau, f, dreaction=J, nspecies=1))
    U0 = np.zeros(g.shape(bc))
    expect = np.zeros_like(U0)
    for (nx, ny, nz), wgt in (((1, 2, 3), 1.0), ((3, 1, 2), -0.6), ((2, 4, 1), 0.3)):
        modes = [_closed_form_mode(bc, n, N) for n, N in zip((nx, ny, nz), Ns)]
        F = wgt * np.einsum("z,y,x->zyx", modes[2], modes[1], modes[0])
        lam = sum(_closed_form_lambda(bc, n, N, (b - a) / N) for n, N, a, b in zip((nx, ny, nz), Ns, lo, hi))
        L = kappa * tau * lam ** (alpha / 2)
        R = (24 - 6 * L) / (24 + 18 * L + 6 * L * L + L ** 3)
        U0 += F
        expect += R ** M * F
    got = s.run([U0], 0.0, M)[0]
    np.testing.assert_allclose(got, expect, atol=1e-12 * np.abs(U0).max())


@pytest.mark.parametrize("bc", O.BCS)
@pytest.mark.parametrize("Ns", [(2,), (3,), (2, 2), (2, 3), (2, 3, 4), (4, 2, 3)])
def test_smallest_grids_decay_mode_by_mode(bc, Ns):
    """Degenerate sizes (one to five unknowns per axis): every separable mode of the grid, superposed with
    random weights, is scaled by R13(L)^M with L from the closed-form eigenvalues (as in the 3D test above)."""
    dim = len(Ns)
    lo, hi = (0.0,) * dim, tuple(1.0 + 0.5 * d for d in range(dim))
    alpha, kappa, tau, M = 1.7, 0.4, 0.03, 4
    g = O.Grid(Ns, lo, hi)
    f, J = O.linear(0.0)
    s = O.ETDRK4P13(O.Problem(g, bc, [alpha], [kappa], tau, f, dreaction=J, nspecies=1))
    modes_per_axis = [range(1, N) if bc == O.DIRICHLET else range(0, N + 1) if bc == O.NEUMANN else range(N)
                      for N in Ns]
    rng = np.random.default_rng(sum(Ns) + dim)
    U0 = np.zeros(g.shape(bc))
    expect = np.zeros_like(U0)
    for ns in itertools.product(*modes_per_axis):
        F = rng.standard_normal()
        for d in reversed(range(dim)):                 # field axes are (z, y, x)
            F = np.multiply.outer(F, _closed_form_mode(bc, ns[d], Ns[d]))
        lam = sum(_closed_form_lambda(bc, n, N, (b - a) / N) for n, N, a, b in zip(ns, Ns, lo, hi))
        L = kappa * tau * lam ** (alpha / 2)
        R = (24 - 6 * L) / (24 + 18 * L + 6 * L * L + L ** 3)
        U0 += F
        expect += R ** M * F
    got = s.run([U0], 0.0, M)[0]
    assert got.shape == g.shape(bc)
    np.testing.assert_allclose(got, expect, atol=1e-12 * np.abs(U0).max())


@pytest.mark.parametrize("bc", [O.PERIODIC, O.NEUMANN])
def test_zero_mode_is_conserved_without_reaction(bc):
    N = 12
    g = O.Grid((N, N), (0.0, 0.0), (1.0, 1.0))
    f, J = O.linear(0.0)
    prob = O.Problem(g, bc, [1.4], [2.0], 0.5, f, dreaction=J, nspecies=1)
    s = O.ETDRK4P13(prob)
    u0 = np.random.default_rng(1).standard_normal(g.shape(bc))
    u1 = s.run([u0], 0.0, 5)[0]
    z0, z1 = s.sp.forward(u0).flat[0], s.sp.forward(u1).flat[0]
    assert abs(z1 - z0) < 1e-12 * abs(z0) + 1e-12


# --------------------------------------------------------------------------
# Section 5: the printed error tables
# --------------------------------------------------------------------------

def _example1_error(Ninv):
    g = O.Grid((Ninv,), (0.0,), (1.0,))
    kappa, alpha = 10.0, 1.8
    tau = (1.0 / Ninv) / (4 * kappa)
    f, exact = O.fisher_mms(g, kappa, alpha)
    s = O.ETDRK4P13(O.Problem(g, O.DIRICHLET, [alpha], [kappa], tau, f, nspecies=1))
    M = int(round(1.0 / tau))
    u = s.run([exact(0.0)], 0.0, M)
    return O.max_error(u[0], exact(M * tau))


@pytest.mark.parametrize("row", _table("table1.txt"))
def test_table1_example1_errors(row):
    Ninv, printed = int(row[0]), row[1]
    assert _same_to_printed_digits(_example1_error(Ninv), printed)


def _example2_error(bc, alpha, Ninv):
    g = O.Grid((Ninv, Ninv), (0.0, 0.0), (1.0, 1.0))
    tau = 0.1 / Ninv
    f, exact = O.huxley_mms(g, bc, 1.0, alpha)
    s = O.ETDRK4P13(O.Problem(g, bc, [alpha], [1.0], tau, f, nspecies=1))
    M = int(round(1.0 / tau))
    u = s.run([exact(0.0)], 0.0, M)
    return O.max_error(u[0], exact(M * tau))


_T2 = [r for r in _table("table2.txt") if r[1] <= 80 or r[0] == 1.8]


@pytest.mark.parametrize("row", _T2, ids=["a%.1f-n%d" % (r[0], r[1]) for r in _T2])
@pytest.mark.parametrize("bc", [O.NEUMANN, O.PERIODIC])
def test_table2_example2_errors(row, bc):
    alpha, Ninv = row[0], int(row[1])
    printed = row[2] if bc == O.NEUMANN else row[3]
    assert _same_to_printed_digits(_example2_error(bc, alpha, Ninv), printed)


def test_table_orders_are_four():
    rows = _table("table1.txt")
    errs = [_example1_error(int(r[0])) for r in rows[:3]]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.9 < o < 4.4 for o in orders)


# --------------------------------------------------------------------------
# Section 5.2: reaction terms, pinned by properties of the printed models (conserved combinations,
# homogeneous steady states, nullclines, degrees of homogeneity) rather than by their formulas
# --------------------------------------------------------------------------

def _grid_uv(lo=0.2, hi=2.0, n=7):
    u, v = np.meshgrid(np.linspace(lo, hi, n), np.linspace(lo + 0.1, hi + 0.3, n), indexing="ij")
    return u.ravel(), v.ravel()


def test_fitzhugh_nagumo_cubic_nullcline_and_affine_recovery():
    mu, eps, beta, gamma, delta = 0.13, 0.02, 0.7, 1.3, 0.05
    f, _, _ = O.fitzhugh_nagumo(mu=mu, eps=eps, beta=beta, gamma=gamma, delta=delta)
    u = np.linspace(-1.0, 2.0, 9)
    fu0 = f([u, np.zeros_like(u)], 0.0)[0]
    c = np.polyfit(u, fu0, 3)                     # f_u(u, 0): a cubic with leading coefficient -1
    assert abs(c[0] + 1.0) < 1e-12
    np.testing.assert_allclose(np.sort(np.roots(c).real), [0.0, mu, 1.0], atol=1e-10)
    for v in (-0.4, 0.9):                         # f_u depends on v only through -v
        np.testing.assert_allclose(f([u, np.full_like(u, v)], 0.0)[0], fu0 - v, atol=1e-14)
    # f_v is affine with gradient eps (beta, -gamma) and vanishes on the line beta u - gamma v = delta
    uu = np.array([0.0, 1.0, -2.0])
    vv = (beta * uu - delta) / gamma
    np.testing.assert_allclose(f([uu, vv], 0.0)[1], 0.0, atol=1e-15)
    np.testing.assert_allclose(f([uu + 1, vv], 0.0)[1], eps * beta, rtol=1e-12)
    np.testing.assert_allclose(f([uu, vv + 1], 0.0)[1], -eps * gamma, rtol=1e-12)


def test_gray_scott_exchange_cancels_and_cubic_term():
    F, K = 0.037, 0.06
    f, _ = O.gray_scott(F, K)
    u, v = _grid_uv()
    fu, fv = f([u, v], 0.0)
    # the autocatalytic u v^2 moves mass from u to v: the sum is linear
    np.testing.assert_allclose(fu + fv, F * (1 - u) - (F + K) * v, atol=1e-14)
    g = lambda a, b: f([a, b], 0.0)[0] - F * (1 - a)          # the nonlinear part of f_u
    np.testing.assert_allclose(g(2 * u, v), 2 * g(u, v), atol=1e-13)   # degree 1 in u
    np.testing.assert_allclose(g(u, 2 * v), 4 * g(u, v), atol=1e-13)   # degree 2 in v
    assert abs(g(np.array(1.0), np.array(1.0)) + 1.0) < 1e-15          # coefficient -1
    assert np.all(np.asarray(f([u, 0 * v], 0.0)[1]) == 0)              # no v, no source of v


def test_schnakenberg_steady_state_and_exchange():
    gam, a, b = 1000.0, 0.1, 0.9
    f, _ = O.schnakenberg(gamma=gam, a=a, b=b)
    Us, Vs = a + b, b / (a + b) ** 2                                  # the homogeneous steady state
    r = f([np.array([Us]), np.array([Vs])], 0.0)
    assert max(abs(r[0][0]), abs(r[1][0])) < 1e-12
    u, v = _grid_uv()
    fu, fv = f([u, v], 0.0)
    np.testing.assert_allclose(fu + fv, gam * (a + b - u), rtol=1e-13, atol=1e-10)
    h = lambda p, q: f([p, q], 0.0)[1] - gam * b                        # the nonlinear part of f_v
    np.testing.assert_allclose(h(2 * u, v), 4 * h(u, v), rtol=1e-13)   # degree 2 in u
    np.testing.assert_allclose(h(u, 2 * v), 2 * h(u, v), rtol=1e-13)   # degree 1 in v
    # the perturbation form used with Dirichlet conditions: f evaluated at u* + w
    fo, _ = O.schnakenberg(gamma=gam, a=a, b=b, ustar=(Us, Vs))
    w = [u - Us, v - Vs]
    for x, y in zip(fo(w, 0.0), (fu, fv)):
        np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-9)


def test_gierer_meinhardt_steady_state_nullcline_and_homogeneity():
    c1, c2, c3, c4 = 1.0, 1.0, 1.0 / (0.04 * 0.1), 1.0 / 0.1          # the printed model: eps 0.04, mu 0.1
    f, _ = O.gierer_meinhardt(c1, c2, c3, c4)
    us = c1 * c4 / (c2 * c3)
    vs = c3 * us * us / c4
    r = f([np.array([us]), np.array([vs])], 0.0)
    assert max(abs(r[0][0]), abs(r[1][0])) < 1e-12
    u, v = _grid_uv()
    fu, fv = f([u, v], 0.0)
    np.testing.assert_allclose(f([2 * u, 2 * v], 0.0)[0], 2 * fu, rtol=1e-13)   # f_u homogeneous of degree 1
    np.testing.assert_allclose(f([u, c1 * u / c2], 0.0)[0], 0.0, atol=1e-12)      # u-nullcline v = c1 u / c2
    np.testing.assert_allclose(f([u, c3 * u * u / c4], 0.0)[1], 0.0, atol=1e-12)  # v-nullcline
    np.testing.assert_allclose(f([u, v + 1.0], 0.0)[1] - fv, -c4, rtol=1e-12)     # f_v affine in v
    # the unit model of the batched workload has the steady state (1, 1)
    f1, _ = O.gierer_meinhardt()
    assert max(abs(x[0]) for x in f1([np.array([1.0]), np.array([1.0])], 0.0)) == 0.0


@pytest.mark.parametrize("name", ["fhn", "gray_scott", "schnakenberg", "gierer_meinhardt"])
def test_reaction_jacobians_match_central_differences(name):
    f, J = {"fhn": lambda: O.fitzhugh_nagumo()[:2], "gray_scott": O.gray_scott,
            "schnakenberg": lambda: O.schnakenberg(ustar=(1.0, 0.9)), "gierer_meinhardt": O.gierer_meinhardt}[name]()
    u, v = _grid_uv(0.3, 1.7, 5)
    Jm = J([u, v], 0.0)
    d = 1e-6
    for s in range(2):
        wp = [u.copy(), v.copy()]
        wm = [u.copy(), v.copy()]
        wp[s] += d
        wm[s] -= d
        fp, fm = f(wp, 0.0), f(wm, 0.0)
        for r in range(2):
            fd = (fp[r] - fm[r]) / (2 * d)
            np.testing.assert_allclose(np.broadcast_to(Jm[r][s], fd.shape), fd,
                                       rtol=1e-6, atol=1e-6 * max(1.0, np.abs(fd).max()))


# --------------------------------------------------------------------------
# Symmetry and the adjoint
# --------------------------------------------------------------------------

@pytest.mark.parametrize("bc", [O.DIRICHLET, O.NEUMANN])
def test_mirror_symmetric_initial_data_stays_symmetric(bc):
    N = 10
    g = O.Grid((N, N), (0.0, 0.0), (1.0, 1.0))
    f, J, _ = O.fitzhugh_nagumo()
    prob = O.Problem(g, bc, [1.5, 1.5], [0.01, 0.002], 0.2, f, dreaction=J)
    s = O.ETDRK4P13(prob)
    rng = np.random.default_rng(11)
    u = rng.uniform(0, 1, g.shape(bc))
    u = u + u[:, ::-1]
    v = rng.uniform(0, 0.1, g.shape(bc))
    v = v + v[:, ::-1]
    out = s.run([u, v], 0.0, 6)
    for w in out:
        np.testing.assert_allclose(w, w[:, ::-1], atol=1e-13)
    # exchange of axes on a square grid
    ut, vt = s.run([u.T.copy(), v.T.copy()], 0.0, 6)
    np.testing.assert_allclose(ut, out[0].T, atol=1e-13)


@pytest.mark.parametrize("bc", O.BCS)
def test_oracle_adjoint_matches_central_differences(bc):
    """dl/du0, dl/dalpha, dl/dkappa and dl/dmu of l = 1/2 ||u_M - target||^2 through 3 steps."""
    N = 6
    g = O.Grid((N, N), (0.0, 0.0), (10.0, 10.0))
    rng = np.random.default_rng(5)

    def build(alpha, kappa_u, mu):
        f, J, dmu = O.fitzhugh_nagumo(mu=mu)
        prob = O.Problem(g, bc, [alpha, alpha], [kappa_u, 0.3], 0.1, f, dreaction=J)
        return O.ETDRK4P13(prob), dmu

    shp = g.shape(bc)
    u0 = [rng.uniform(0, 1, shp), rng.uniform(0, 0.2, shp)]
    tgt = [rng.uniform(0, 1, shp), rng.uniform(0, 0.2, shp)]
    M = 3
    th = dict(alpha=1.6, kappa_u=1.0, mu=0.1)

    def loss(th_, u0_):
        s, _ = build(th_["alpha"], th_["kappa_u"], th_["mu"])
        uM = s.run(u0_, 0.0, M)
        return 0.5 * sum(float(np.sum((a - b) ** 2)) for a, b in zip(uM, tgt))

    s, dmu = build(**th)
    uM = s.run(u0, 0.0, M)
    gr = O.adjoint_run(s, u0, 0.0, M, [a - b for a, b in zip(uM, tgt)], dparams=dmu)
    hh = 1e-6
    for name in ("alpha", "kappa_u", "mu"):
        tp, tm = dict(th), dict(th)
        tp[name] += hh
        tm[name] -= hh
        fd = (loss(tp, u0) - loss(tm, u0)) / (2 * hh)
        if name == "alpha":
            got = sum(gr["alpha"])
        elif name == "kappa_u":
            got = gr["kappa"][0]
        else:
            got = gr["params"]
        assert got == pytest.approx(fd, rel=1e-6, abs=1e-9), name
    for idx in [(0, 1, 2), (1, 3, 0)]:
        sp_, i, j = idx
        up = [x.copy() for x in u0]
        um = [x.copy() for x in u0]
        up[sp_][i, j] += hh
        um[sp_][i, j] -= hh
        fd = (loss(th, up) - loss(th, um)) / (2 * hh)
        assert gr["u0"][sp_][i, j] == pytest.approx(fd, rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("bc", O.BCS)
@pytest.mark.parametrize("scheme", ["p13", "cox_matthews"])
def test_oracle_adjoint_is_the_transpose_of_the_linear_run(bc, scheme):
    """Dot-product test: with a linear reaction f(u, v) = C (u, v) the run u0 -> u_M is a linear map J,
    and the reverse sweep must apply its transpose, <J v, w> = <v, J^T w>, to rounding, for random v, w.
    C couples the species non-symmetrically and the species have their own orders and diffusivities, so
    J is not symmetric for any boundary condition and a transposed operand is detected (checked below)."""
    g = O.Grid((8, 6), (0.0, 0.0), (3.0, 4.0))
    C = [[-0.7, 0.3], [-0.2, -0.5]]

    def f(w_, t):
        return [C[0][0] * w_[0] + C[0][1] * w_[1], C[1][0] * w_[0] + C[1][1] * w_[1]]

    def J(w_, t):
        return [[C[r][c] * np.ones_like(w_[0]) for c in range(2)] for r in range(2)]
    prob = O.Problem(g, bc, [1.5, 1.8], [0.4, 0.1], 0.05, f, dreaction=J)
    s = O.ETDRK4P13(prob, scheme=scheme)
    rng = np.random.default_rng(21)
    shp = g.shape(bc)
    v = [rng.standard_normal(shp) for _ in range(2)]
    w = [rng.standard_normal(shp) for _ in range(2)]
    M = 4
    Jv = s.run(v, 0.0, M)
    JTw = O.adjoint_run(s, v, 0.0, M, w)["u0"]
    lhs = sum(float(np.sum(a * b)) for a, b in zip(Jv, w))
    rhs = sum(float(np.sum(a * b)) for a, b in zip(v, JTw))
    scale = np.sqrt(sum(float(np.sum(a * a)) for a in Jv) * sum(float(np.sum(b * b)) for b in w))
    assert abs(lhs - rhs) <= 1e-13 * scale
    # a transposed operand would break it: the forward map applied in place of its transpose
    Jw = s.run(w, 0.0, M)
    assert abs(sum(float(np.sum(a * b)) for a, b in zip(v, Jw)) - lhs) > 1e-6 * scale


# --------------------------------------------------------------------------
# The Cox-Matthews variant (exact exponentials, Section 4's reference scheme)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("L", [1.5, 4.6, 20.0, 300.0])
def test_cox_matthews_contour_coefficients_match_closed_forms(L):
    """Away from L = 0 the closed forms do not cancel: the contour means must equal them."""
    tau = 0.37
    c = O.cox_matthews_coefficients(np.array([L]), tau)
    E, E2 = math.exp(-L), math.exp(-L / 2)
    z = -L
    assert c["R13"][0] == pytest.approx(E, rel=1e-15)
    assert c["Q13"][0] == pytest.approx(E2, rel=1e-15)
    assert c["phi"][0] == pytest.approx(tau * (1 - E2) / L, rel=1e-12)
    assert c["phi1"][0] == pytest.approx(tau * (-4 - z + E * (4 - 3 * z + z * z)) / z ** 3, rel=1e-11)
    assert c["phi2"][0] == pytest.approx(2 * tau * (2 + z + E * (z - 2)) / z ** 3, rel=1e-11)
    assert c["phi3"][0] == pytest.approx(tau * (-4 - 3 * z - z * z + E * (4 - z)) / z ** 3, rel=1e-11)


def test_cox_matthews_coefficients_zero_limits_and_small_l_series():
    """L -> 0: the classical RK4 weights; small L: the Taylor series of the phi-functions."""
    tau = 0.1
    c = O.cox_matthews_coefficients(np.array([0.0, 1e-3]), tau)
    assert c["R13"][0] == 1.0 and c["Q13"][0] == 1.0
    for k, v in (("phi", tau / 2), ("phi1", tau / 6), ("phi2", tau / 3), ("phi3", tau / 6)):
        assert c[k][0] == pytest.approx(v, rel=1e-14), k
    L = 1e-3   # series to O(L^2) (alpha = 1/6 - z/6 + 3z^2/40 ..., z = -L) from e^z expanded by hand
    assert c["phi1"][1] == pytest.approx(tau * (1 / 6 - L / 6 + 3 * L * L / 40), rel=1e-9)
    assert c["phi2"][1] == pytest.approx(2 * tau * (1 / 6 - L / 12 + L * L / 40), rel=1e-9)
    assert c["phi3"][1] == pytest.approx(tau * (1 / 6 + 0 * L - L * L / 120), rel=1e-9)


def test_cox_matthews_single_eigenmode_decays_exactly():
    """f = 0: each eigen-coefficient decays by exactly exp(-kappa Lambda^{alpha/2} t)."""
    N, M, tau = 16, 7, 0.2
    g = O.Grid((N, N), (0.0, 0.0), (2.0, 2.0))
    f, J = O.linear(0.0)
    for bc in O.BCS:
        prob = O.Problem(g, bc, [1.7], [0.3], tau, f, dreaction=J, nspecies=1)
        s = O.ETDRK4P13(prob, scheme="cox_matthews")
        u0 = np.random.default_rng(3).standard_normal(g.shape(bc))
        uM = s.run([u0], 0.0, M)[0]
        lam = s.sp.Lambda_frac(1.7)
        expect = s.sp.forward(u0) * np.exp(-0.3 * lam * tau * M)
        np.testing.assert_allclose(s.sp.forward(uM), expect, atol=1e-12 * np.abs(expect).max())


def test_cox_matthews_is_exact_for_a_constant_source():
    """f(u) = c (constant): the exact solution of u_t = -K u + c is reached in one step."""
    N, tau, cval = 12, 0.3, 0.7
    g = O.Grid((N, N), (0.0, 0.0), (1.0, 1.5))

    def f(w, t):
        return [np.full_like(w[0], cval)]

    for bc in O.BCS:
        prob = O.Problem(g, bc, [1.5], [0.8], tau, f, nspecies=1)
        s = O.ETDRK4P13(prob, scheme="cox_matthews")
        u0 = np.random.default_rng(5).standard_normal(g.shape(bc))
        u1 = s.run([u0], 0.0, 1)[0]
        L = s.L[0]
        Lsafe = np.where(L > 0, L, 1.0)
        gain = np.where(L > 0, tau * (1 - np.exp(-L)) / Lsafe, tau)
        expect = np.exp(-L) * s.sp.forward(u0) + gain * s.sp.forward(np.full(g.shape(bc), cval))
        np.testing.assert_allclose(s.sp.forward(u1), expect, atol=1e-12 * np.abs(expect).max())


def test_cox_matthews_and_p13_agree_to_fifth_order_in_l():
    """The schemes differ only through e^{-L} versus R13(L) = e^{-L} + O(L^5) per step."""
    tau = 1.0
    d = []
    for L in (0.02, 0.04):
        a, b = O.cox_matthews_coefficients(np.array([L]), tau), O.p13_coefficients(np.array([L]), tau)
        d.append(abs(a["R13"][0] - b["R13"][0]))
    assert d[1] / d[0] == pytest.approx(32.0, rel=0.05)


def test_cox_matthews_derivatives_zero_limits_and_central_differences():
    """dC/dL of the Cox-Matthews arrays: at L = 0 the values follow from the series by hand
    (d e^{-L} = -1, d e^{-L/2} = -1/2, dphi = -tau/8, dphi1 = dphi2 = -tau/6, dphi3 = 0), and
    elsewhere they equal central differences of cox_matthews_coefficients."""
    tau = 0.1
    d0 = O.cox_matthews_derivatives(np.array([0.0]), tau)
    for k, v in (("R13", -1.0), ("Q13", -0.5), ("phi", -tau / 8), ("phi1", -tau / 6), ("phi2", -tau / 6)):
        assert d0[k][0] == pytest.approx(v, rel=1e-13), k
    assert abs(d0["phi3"][0]) < 1e-15
    L = np.array([0.3, 0.99, 1.0, 1.5, 2.0, 2.5, 3.7, 30.0])
    h = 1e-6
    d = O.cox_matthews_derivatives(L, tau)
    cp, cm = O.cox_matthews_coefficients(L + h, tau), O.cox_matthews_coefficients(L - h, tau)
    for k in d:
        fd = (cp[k] - cm[k]) / (2 * h)
        np.testing.assert_allclose(d[k], fd, rtol=1e-7, atol=1e-12 * tau, err_msg=k)


def test_oracle_cox_matthews_adjoint_matches_central_differences():
    """The oracle's reverse sweep with the Cox-Matthews coefficients: dl/dalpha, dl/dkappa and
    dl/du0 of l = 1/2 ||u_M - target||^2 through 3 steps against central differences."""
    N = 6
    g = O.Grid((N, N), (0.0, 0.0), (10.0, 10.0))
    rng = np.random.default_rng(8)
    f, J, dmu = O.fitzhugh_nagumo()

    def build(alpha, kappa_u):
        prob = O.Problem(g, O.NEUMANN, [alpha, alpha], [kappa_u, 0.3], 0.1, f, dreaction=J)
        return O.ETDRK4P13(prob, scheme="cox_matthews")

    shp = g.shape(O.NEUMANN)
    u0 = [rng.uniform(0, 1, shp), rng.uniform(0, 0.2, shp)]
    tgt = [rng.uniform(0, 1, shp), rng.uniform(0, 0.2, shp)]
    M = 3

    def loss(alpha, kappa_u, u0_):
        uM = build(alpha, kappa_u).run(u0_, 0.0, M)
        return 0.5 * sum(float(np.sum((a - b) ** 2)) for a, b in zip(uM, tgt))

    s = build(1.6, 1.0)
    uM = s.run(u0, 0.0, M)
    gr = O.adjoint_run(s, u0, 0.0, M, [a - b for a, b in zip(uM, tgt)], dparams=dmu)
    hh = 1e-6
    fd = (loss(1.6 + hh, 1.0, u0) - loss(1.6 - hh, 1.0, u0)) / (2 * hh)
    assert sum(gr["alpha"]) == pytest.approx(fd, rel=1e-6, abs=1e-9)
    fd = (loss(1.6, 1.0 + hh, u0) - loss(1.6, 1.0 - hh, u0)) / (2 * hh)
    assert gr["kappa"][0] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    up = [x.copy() for x in u0]
    um = [x.copy() for x in u0]
    up[0][2, 3] += hh
    um[0][2, 3] -= hh
    fd = (loss(1.6, 1.0, up) - loss(1.6, 1.0, um)) / (2 * hh)
    assert gr["u0"][0][2, 3] == pytest.approx(fd, rel=1e-6, abs=1e-9)


# --------------------------------------------------------------------------
# Section 5: the error norms every parity test decides by
# --------------------------------------------------------------------------

def test_relative_error_norms_on_hand_computed_values():
    """rel_max = max|x - y| / max|y| and rel_l2 = ||x - y||_2 / ||y||_2 over all unknowns of all
    species, checked on arrays whose norms are worked out by hand.  The differences form a 3-4-5
    triangle and y a 5-12-13 one, so rel_l2 is exactly 5/13: a dropped square root (25/169), a
    per-species instead of a global norm, or a norm of x instead of y all give another number."""
    x = [np.array([[4.0, 12.0]]), np.array([0.0])]
    y = [np.array([[1.0, 12.0]]), np.array([-4.0])]
    # |x - y| = (3, 0 | 4): max 4; max|y| = 12  ->  4 / 12
    assert O.rel_max(x, y) == pytest.approx(1.0 / 3.0, rel=0, abs=1e-16)
    # ||x - y||^2 = 9 + 16 = 25; ||y||^2 = 1 + 144 + 16 = 161
    assert O.rel_l2(x, y) == pytest.approx(5.0 / math.sqrt(161.0), rel=0, abs=1e-16)
    # one species: differences (3, 4), y = (5, 12): rel_l2 = 5/13, rel_max = 4/12
    assert O.rel_l2([np.array([8.0, 16.0])], [np.array([5.0, 12.0])]) == pytest.approx(5.0 / 13.0, rel=0,
                                                                                         abs=1e-16)
    assert O.rel_max([np.array([8.0, 16.0])], [np.array([5.0, 12.0])]) == pytest.approx(1.0 / 3.0, rel=0,
                                                                                          abs=1e-16)
    # the norms are not symmetric in their arguments: the reference is the second one
    assert O.rel_l2([np.array([5.0, 12.0])], [np.array([8.0, 16.0])]) == pytest.approx(
        5.0 / math.sqrt(320.0), rel=0, abs=1e-16)
    # the largest difference and the largest reference value may sit in different species
    assert O.rel_max([np.array([0.0, 10.0]), np.array([7.0])], [np.array([0.0, 10.0]), np.array([2.0])]) == \
        pytest.approx(0.5, rel=0, abs=1e-16)
    # equal inputs give zero
    assert O.rel_max(y, y) == 0.0 and O.rel_l2(y, y) == 0.0


def test_test_side_error_norms_agree_with_the_oracle_norms():
    """The single-array norms in tests/helpers.py, on the same hand-computed values."""
    from tests.helpers import rel_l2, rel_max
    assert rel_l2(np.array([8.0, 16.0]), np.array([5.0, 12.0])) == pytest.approx(5.0 / 13.0, rel=0, abs=1e-16)
    assert rel_max(np.array([8.0, 16.0]), np.array([5.0, 12.0])) == pytest.approx(1.0 / 3.0, rel=0, abs=1e-16)
    assert rel_max(np.array([[0.0, 10.0], [7.0, 0.0]]), np.array([[0.0, 10.0], [2.0, 0.0]])) == \
        pytest.approx(0.5, rel=0, abs=1e-16)
