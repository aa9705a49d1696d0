"""Builds oracle problems from the shared workload descriptions (oracle side; test infrastructure only)."""
from . import sfrd_oracle as O


def reaction_fns(cfg):
    r = cfg["reaction"]
    k, p, off = r["kind"], r["p"], r.get("offset", [0.0, 0.0])
    if k == "fhn":
        f, J, dmu = O.fitzhugh_nagumo(*p)
        return f, J, dmu
    if k == "gray_scott":
        f, J = O.gray_scott(*p)
        return f, J, None
    if k == "schnakenberg":
        f, J = O.schnakenberg(p[0], p[1], p[2], ustar=tuple(off))
        return f, J, None
    if k == "gierer_meinhardt":
        f0, J0 = O.gierer_meinhardt(*p)

        def f(w, t):
            return f0([w[0] + off[0], w[1] + off[1]], t)

        def J(w, t):
            return J0([w[0] + off[0], w[1] + off[1]], t)
        return f, J, None
    if k == "linear":
        f, J = O.linear(p[0])
        return f, J, None
    if k == "none":
        f, J = O.linear(0.0)
        return f, J, None
    raise ValueError(k)


def problem(cfg):
    g = O.Grid(tuple(cfg["N"]), tuple(cfg["lo"]), tuple(cfg["hi"]))
    if cfg["reaction"]["kind"] == "fisher_mms":     # Example 1 (needs the grid)
        f, _ = O.fisher_mms(g, cfg["kappa"][0], cfg["alpha"][0])
        return O.Problem(g, cfg["bc"], list(cfg["alpha"]), list(cfg["kappa"]), cfg["dt"], f, nspecies=1)
    f, J, _ = reaction_fns(cfg)
    return O.Problem(g, cfg["bc"], list(cfg["alpha"]), list(cfg["kappa"]), cfg["dt"], f,
                     dreaction=J, nspecies=len(cfg["alpha"]))


def solver(cfg):
    return O.ETDRK4P13(problem(cfg), scheme=cfg.get("scheme", "p13"))
