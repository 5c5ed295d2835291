"""Pins of the oracle's fixed-N chemical potential search (App. D: mu chosen
so that the coupled-cluster system holds N electrons) against values fixed by
mathematics: the closed-form Fermi root of a non-interacting system, the
particle-hole symmetric point of the half-filled ring, and central
differences of the converged grand potential."""
import numpy as np
from scipy.optimize import brentq

from oracle import chemical_potential as cp
from oracle import ftccsd as fc
from oracle import systems

BETA, NG = 1.0, 16


def test_reference_mu_is_the_fermi_root():
    """mu_0 solves sum_p 1 / (1 + exp(beta (eps_p - mu))) = N."""
    s = systems.hubbard_1d(6, 1.0, 2.0)
    e = s["eps"].numpy()
    root = brentq(lambda m: np.sum(1.0 / (1.0 + np.exp(BETA * (e - m)))) - 5.0, -20.0, 20.0, xtol=1e-15)
    assert abs(cp.mu_reference(s["eps"], BETA, 5.0) - root) < 1e-12


def test_mu_search_without_interaction_lands_on_the_fermi_root():
    """At U = 0 the FT-CCSD N(mu) is the non-interacting Fermi sum, so the
    search (started away from the root) reaches its closed-form root."""
    s = systems.hubbard_1d(6, 1.0, 0.0)
    e = s["eps"].numpy()
    root = brentq(lambda m: np.sum(1.0 / (1.0 + np.exp(BETA * (e - m)))) - 5.0, -20.0, 20.0, xtol=1e-15)
    r = cp.mu_for_n(s, BETA, 5.0, NG, mu0=0.0)
    assert r["evaluations"] > 2
    assert abs(r["mu"] - root) < 1e-9


def test_mu_search_at_half_filling_is_particle_hole_symmetric():
    """N = L on the even ring is reached at mu = U / 2."""
    U = 2.0
    s = systems.hubbard_1d(6, 1.0, U)
    r = cp.mu_for_n(s, BETA, 6.0, NG, mu0=0.4)
    assert abs(r["mu"] - U / 2.0) < 1e-8


def test_mu_search_off_half_filling_matches_finite_differences():
    """At the mu found for N = 5 the particle number from central
    differences of Omega(mu) (no lambda equations) is 5."""
    s = systems.hubbard_1d(6, 1.0, 2.0)
    r = cp.mu_for_n(s, BETA, 5.0, NG)
    d = 1e-4
    om_p = fc.omega_at(s, BETA, r["mu"] + d, NG)
    om_m = fc.omega_at(s, BETA, r["mu"] - d, NG)
    assert abs(-(om_p - om_m) / (2 * d) - 5.0) < 1e-6
    assert abs(r["N"] - 5.0) < 1e-9
