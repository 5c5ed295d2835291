"""Chemical potential for a fixed mean particle number, plain FP64 CPU oracle
(test infrastructure only: only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may use it).

White & Chan, arXiv:2004.01729, fix the electron number of the grand
canonical calculation by choosing mu: the coupled-cluster system and the
reference each get their own chemical potential with N electrons (App. D,
the definition of E_xc; Sec. III.A fixes N to 1e-4 for every grid).  Here:

* the reference mu_0 solves sum_p n_p(mu) = N with the Fermi-Dirac
  occupations of the orbital energies (Sec. II.A), by bisection;
* the coupled-cluster mu_CC solves N(mu) = N, where N(mu) = -dOmega/dmu is
  the derivative of the converged FT-CCSD grand potential (App. B, evaluated
  by `ftccsd.response` through the lambda equations), by the secant method
  from mu_0, keeping a bracket once the target is straddled (regula falsi
  with the Illinois weighting), so that the search stays inside it.
"""
import math

import torch

from . import ftccsd as fc


def n_reference(eps, beta, mu):
    """sum_p n_p with n_p = 1 / (1 + exp(beta (eps_p - mu)))  (Sec. II.A)."""
    n, _ = fc.occupations(torch.as_tensor(eps, dtype=fc.DT), torch.as_tensor(beta, dtype=fc.DT),
                          torch.as_tensor(mu, dtype=fc.DT))
    return float(n.sum())


def mu_reference(eps, beta, n_target, tol=1e-14):
    """mu_0 with sum_p n_p(mu_0) = N, by bisection (the sum rises with mu)."""
    e = torch.as_tensor(eps, dtype=fc.DT)
    lo = float(e.min()) - 50.0 / beta - 1.0
    hi = float(e.max()) + 50.0 / beta + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if n_reference(e, beta, mid) < n_target:
            lo = mid
        else:
            hi = mid
        if hi - lo < tol:
            break
    return 0.5 * (lo + hi)


def n_cc(system, beta, mu, ngrid, thr=0.0, solve_kw=None):
    """N(mu) = -dOmega/dmu of the converged FT-CCSD grand potential (App. B)."""
    return fc.response(system, beta, mu, ngrid, thr, solve_kw)["N"]


def mu_for_n(system, beta, n_target, ngrid, mu0=None, dmu=0.05, tol_n=1e-10, max_iter=40, thr=0.0,
             solve_kw=None):
    """mu_CC with N(mu_CC) = n_target.

    Starts from mu0 (default: the reference mu_0 of the same N) and mu0 + dmu;
    secant steps until |N - n_target| < tol_n, regula falsi with the Illinois
    weighting once a bracket exists.  Returns mu, N and the number of N
    evaluations.
    """
    if mu0 is None:
        mu0 = mu_reference(system["eps"], beta, n_target)
    f = lambda m: n_cc(system, beta, m, ngrid, thr, solve_kw) - n_target  # noqa: E731
    a, fa = mu0, f(mu0)
    evals = 1
    if abs(fa) < tol_n:
        return {"mu": a, "N": fa + n_target, "evaluations": evals}
    b, fb = mu0 + (dmu if fa < 0 else -dmu), None
    fb = f(b)
    evals += 1
    bracket = fa * fb < 0
    side = 0
    for _ in range(max_iter):
        if abs(fb) < tol_n:
            break
        if fb == fa:
            raise RuntimeError("flat N(mu): no secant step")
        c = b - fb * (b - a) / (fb - fa)
        fc_ = f(c)
        evals += 1
        if bracket:
            # keep the pair that straddles the target; halve the weight of a
            # retained end point that is kept twice in a row (Illinois)
            if fc_ * fb < 0:
                a, fa = b, fb
                side = 0
            else:
                if side == -1:
                    fa *= 0.5
                side = -1
            b, fb = c, fc_
        else:
            a, fa, b, fb = b, fb, c, fc_
            bracket = fa * fb < 0
        if not math.isfinite(fb):
            raise RuntimeError("N(mu) not finite during the search")
    return {"mu": b, "N": fb + n_target, "evaluations": evals}
