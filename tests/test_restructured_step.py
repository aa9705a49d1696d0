"""The library's form of the step, written out in numpy on the oracle's transforms and coefficient
arrays, against the oracle's literal Algorithm 1 (no GPU).

Algorithm 1 takes seven forward and four inverse transforms per species and step, one of them the
re-transform of the stage value a_k.  The library takes four of each: by linearity of F,
F(a_k) = Q13 u_hat + phi F(f_u), F(f_a + f_b) = F(f_a) + F(f_b) and F(2 f_b - f_u) = 2 F(f_b) - F(f_u),
so the stage c combination and the update reuse the spectra F(f_u), F(f_a), F(f_b) kept from the
earlier stages.  This file checks that the two orders of work agree to rounding."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.bridge import solver as oracle_solver

_PARAMS = {"fhn": [0.1, 0.01, 0.5, 1.0, 0.0], "gray_scott": [0.04, 0.06], "schnakenberg": [5.0, 0.1, 0.9],
           "gierer_meinhardt": [1.0, 1.0, 1.0, 1.0]}
_OFFSET = {"schnakenberg": [1.0, 0.9], "gierer_meinhardt": [1.0, 1.0]}


def _cfg(dim, N, bc, kind, dt):
    return dict(dim=dim, N=tuple(N), lo=(0.0,) * dim, hi=tuple(2.0 + d for d in range(dim)), bc=bc,
                alpha=(1.5, 1.7), kappa=(0.7, 0.2), dt=dt, nsteps=1,
                reaction=dict(kind=kind, p=_PARAMS[kind], offset=_OFFSET.get(kind, [0.0, 0.0])),
                dtype="f64", seed=7)


def _rand_fields(cfg, seed, lo, hi):
    rng = np.random.default_rng(seed)
    return [rng.uniform(lo, hi, W.field_shape(cfg)) for _ in range(2)]


def _restructured_step(s, u, u_h, t):
    """One step from the physical state u and its spectrum u_h (kept from the previous step, as the
    library keeps it resident); returns both for the next step.  4 forward and 4 inverse transforms."""
    F, Fi, tau, S = s.sp.forward, s.sp.inverse, s.prob.tau, s.prob.nspecies
    c, f, re = s.coef, s.prob.reaction, s._real
    Fu = [F(x) for x in f(u, t)]                                      # forward 1
    a_h = [c[k]["Q13"] * u_h[k] + c[k]["phi"] * Fu[k] for k in range(S)]
    Fa = [F(x) for x in f([re(Fi(x)) for x in a_h], t + tau / 2)]     # inverse 1, forward 2
    b_h = [c[k]["Q13"] * u_h[k] + c[k]["phi"] * Fa[k] for k in range(S)]
    Fb = [F(x) for x in f([re(Fi(x)) for x in b_h], t + tau / 2)]     # inverse 2, forward 3
    c_h = [c[k]["Q13"] * a_h[k] + c[k]["phi"] * (2 * Fb[k] - Fu[k]) for k in range(S)]
    Fc = [F(x) for x in f([re(Fi(x)) for x in c_h], t + tau)]         # inverse 3, forward 4
    u_h = [c[k]["R13"] * u_h[k] + c[k]["phi1"] * Fu[k] + c[k]["phi2"] * (Fa[k] + Fb[k]) + c[k]["phi3"] * Fc[k]
           for k in range(S)]
    return [re(Fi(x)) for x in u_h], u_h                              # inverse 4: u for the next f_u


@pytest.mark.parametrize("dim,N,bc,kind", [(2, (12, 10), "periodic", "gray_scott"),
                                           (2, (12, 10), "dirichlet", "schnakenberg"),
                                           (2, (12, 10), "neumann", "fhn"),
                                           (3, (8, 6, 10), "periodic", "gray_scott"),
                                           (3, (8, 6, 10), "dirichlet", "gierer_meinhardt"),
                                           (3, (8, 6, 10), "neumann", "schnakenberg")])
def test_four_transform_step_equals_algorithm1(dim, N, bc, kind):
    cfg = _cfg(dim, N, bc, kind=kind, dt=0.05)
    lo, hi = (0.0, 1.0) if kind in ("fhn", "gray_scott") else (-0.05, 0.05)
    u = _rand_fields(cfg, seed=5, lo=lo, hi=hi)
    s = oracle_solver(cfg)
    lit, res = [x.copy() for x in u], [x.copy() for x in u]
    res_h = [s.sp.forward(x) for x in res]                            # the initial transform, once
    for k in range(3):
        lit = s.step(lit, k * cfg["dt"])
        res, res_h = _restructured_step(s, res, res_h, k * cfg["dt"])
    assert O.rel_max(res, lit) < 1e-12
