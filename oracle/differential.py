"""Differential-form driver of the FT-CCSD amplitude equations, plain FP64 CPU
oracle (test infrastructure only: only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may use it).

Follows White & Chan, arXiv:2004.01729:

* the amplitudes obey ds_mu/dtau = -(Delta_mu s_mu(tau) + S_mu[s(tau)]) with
  s(0) = 0 (Eq. smud; the kernels S_mu are Eqs. ccS1 / ccS2, evaluated term
  by term by `ftccsd.S1` / `ftccsd.S2`);
* Alg. 1 marches them over the uniform grid tau_y = y h, h = beta/(ngrid-1),
  one explicit step per interval, and accumulates
  Omega_CC = beta^-1 sum_y g_y E[s(tau_y)] with the quadrature weights g of
  Sec. II.C (Eq. Ecc), so the grand potential keeps the h^4 quadrature error
  and the amplitudes carry the step's own error (Table I: RK1 h, RK2 h^2,
  RK4 h^4).

Reading R13: the paper names RK1, RK2 and RK4 without printing their
tableaux.  Taken here: RK1 = forward Euler, RK2 = Heun's method (the explicit
trapezoid rule), RK4 = the classical four-stage method.  The kernel S does not
depend on tau explicitly, so only the stage weights enter.
"""
import torch

from . import ftccsd as fc

# Butcher tableaux of the explicit methods (reading R13): A (strictly lower
# triangular, one row per stage) and the weights b
TABLEAU = {
    1: ([[]], [1.0]),
    2: ([[], [1.0]], [0.5, 0.5]),
    4: ([[], [0.5], [0.0, 0.5], [0.0, 0.0, 1.0]], [1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0]),
}


def derivative(prob, t1, t2):
    """ds/dtau = -(Delta s + S[s]) for one amplitude state (Eq. smud).

    t1 [i, a] and t2 [i, j, a, b]; returns the two derivatives in the same
    shapes.
    """
    s1 = fc.S1(prob, t1[None], t2[None])[0]
    s2 = fc.S2(prob, t1[None], t2[None])[0]
    return -(prob.D1 * t1 + s1), -(prob.D2 * t2 + s2)


def step(prob, t1, t2, h, order):
    """One explicit Runge-Kutta step of length h (reading R13)."""
    A, b = TABLEAU[order]
    k1, k2 = [], []
    for s, row in enumerate(A):
        y1, y2 = t1, t2
        for j, a in enumerate(row):
            if a != 0.0:
                y1 = y1 + h * a * k1[j]
                y2 = y2 + h * a * k2[j]
        d1, d2 = derivative(prob, y1, y2)
        k1.append(d1)
        k2.append(d2)
    n1, n2 = t1, t2
    for s, w in enumerate(b):
        n1 = n1 + h * w * k1[s]
        n2 = n2 + h * w * k2[s]
    return n1, n2


def march(prob, order):
    """Alg. 1: s(tau_0) = 0, then one step per grid interval.

    Returns the amplitudes at every grid point, t1 [ng, i, a] and
    t2 [ng, i, j, a, b].
    """
    if order not in TABLEAU:
        raise ValueError("order must be 1, 2 or 4")
    no, nv, ng = len(prob.iO), len(prob.iV), prob.ngrid
    h = prob.beta / (ng - 1)
    t1 = torch.zeros((no, nv), dtype=fc.DT)
    t2 = torch.zeros((no, no, nv, nv), dtype=fc.DT)
    out1, out2 = [t1], [t2]
    with torch.no_grad():
        for _ in range(1, ng):
            t1, t2 = step(prob, t1, t2, h, order)
            out1.append(t1)
            out2.append(t2)
    return torch.stack(out1), torch.stack(out2)


def solve_rk(prob, order):
    """Grand potential from the differential form (Alg. 1 with RK1/RK2/RK4).

    Same keys as `ftccsd.solve` where they apply; Omega_CC uses the grid's
    quadrature weights g (Eq. Ecc).
    """
    t1, t2 = march(prob, order)
    occ = fc.omega_cc(prob, t1, t2).item()
    om0 = prob.omega0.item()
    om1 = prob.omega1.item()
    return {"omega": om0 + om1 + occ, "omega0": om0, "omega1": om1, "omega_cc": occ, "t1": t1, "t2": t2,
            "order": order}


def omega_rk(system, beta, mu, ngrid, order, thr=0.0):
    """Omega of one (system, beta, mu, ngrid) from the RK driver."""
    return solve_rk(fc.Problem(system, beta, mu, ngrid, thr), order)["omega"]
