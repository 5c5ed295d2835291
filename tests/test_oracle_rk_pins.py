"""Pins of the oracle's differential-form driver (Eq. smud marched by Alg. 1
with RK1 / RK2 / RK4, reading R13) against values fixed by mathematics.

Each reference is a closed form (the grand potential of a one-body
Hamiltonian, which FT-CCSD reproduces exactly in the continuum limit), the
convergence order of the method (Table I: amplitude error h, h^2, h^4), or the
integral form's own converged value, which reaches the same continuum limit
through a different discretisation.
"""
import numpy as np
import pytest
import torch

from oracle import differential as df
from oracle import exact, ftccsd as fc, systems
from paper_2004_01729_gb300 import workloads as wl

# (order, grid sizes, accepted range of err(h) / err(h/2))
ORDERS = [(1, (17, 33, 65), (1.8, 2.3)), (2, (17, 33, 65), (3.6, 4.6)), (4, (17, 33, 65), (13.0, 19.0))]


@pytest.mark.parametrize("order,grids,ratio", ORDERS)
def test_rk_single_orbital_shift_converges_to_exact(order, grids, ratio):
    """One orbital with f - eps = delta: the singles equation is exact for a
    one-body perturbation, so Omega -> the non-interacting grand potential
    with the step's own order."""
    eps, dl, beta, mu = 0.3, 0.7, 2.0, 0.1
    s = systems.generic(torch.tensor([[eps + dl]]), torch.zeros(1, 1, 1, 1), torch.tensor([eps]))
    ex = exact.noninteracting_omega(np.array([[eps + dl]]), beta, mu)
    err = [df.omega_rk(s, beta, mu, ng, order) - ex for ng in grids]
    for a, b in zip(err, err[1:]):
        assert ratio[0] < a / b < ratio[1], (order, err)
    assert abs(err[-1]) < {1: 1e-3, 2: 1e-5, 4: 1e-9}[order]


@pytest.mark.parametrize("order,grids,ratio", [(1, (65, 129), (1.7, 2.3)), (2, (33, 65), (3.5, 4.6)),
                                               (4, (33, 65), (13.0, 19.0))])
def test_rk_general_one_body_perturbation_converges_to_exact(order, grids, ratio):
    """Off-diagonal one-body perturbation (Delta != 0 singles, coupled)."""
    rng = np.random.default_rng(3)
    a = rng.normal(size=(4, 4))
    h = 0.5 * (a + a.T)
    eps = np.diag(h) + 0.3 * rng.normal(size=4)
    s = systems.generic(torch.tensor(h), torch.zeros(4, 4, 4, 4), torch.tensor(eps))
    ex = exact.noninteracting_omega(h, 1.5, 0.2)
    err = [df.omega_rk(s, 1.5, 0.2, ng, order) - ex for ng in grids]
    assert ratio[0] < err[0] / err[1] < ratio[1], (order, err)


def test_rk_zero_interaction_gives_zero_correlation():
    """At U = 0 the k-space reference is exact: S[0] = 0, so s stays 0."""
    s = systems.hubbard_1d(6, 1.0, 0.0)
    for order in (1, 2, 4):
        sol = df.solve_rk(fc.Problem(s, 1.0, 0.0, 9), order)
        assert sol["omega_cc"] == 0.0
        assert torch.count_nonzero(sol["t2"]) == 0


@pytest.mark.parametrize("order,grids,ratio", [(2, (17, 33, 65), (3.2, 4.8)), (4, (17, 33, 65), (11.0, 20.0)),
                                               (1, (129, 257, 513), (1.6, 2.3))])
def test_rk_order_on_hubbard_6(order, grids, ratio):
    """Table I on an interacting system: successive differences of Omega
    shrink as h^p for RK_p (RK1 reaches its order only on fine grids)."""
    c = wl.HUBBARD_6
    s = systems.hubbard_1d(c["L"], c["t"], c["U"])
    om = [df.omega_rk(s, c["beta"], c["mu"], ng, order) for ng in grids]
    r = (om[0] - om[1]) / (om[1] - om[2])
    assert ratio[0] < r < ratio[1], (order, om)


def test_rk4_and_integral_form_share_the_continuum_limit():
    """RK4 (differential form) and the Simpson fixed point (integral form)
    carry O(h^4) errors of their own; at 65 points they agree far below
    either one's 17-point error."""
    c = wl.HUBBARD_6
    s = systems.hubbard_1d(c["L"], c["t"], c["U"])
    rk = df.omega_rk(s, c["beta"], c["mu"], 65, 4)
    simp = fc.omega_at(s, c["beta"], c["mu"], 65)
    coarse = abs(df.omega_rk(s, c["beta"], c["mu"], 17, 4) - simp)
    assert abs(rk - simp) < 1e-6
    assert abs(rk - simp) < coarse / 50.0
