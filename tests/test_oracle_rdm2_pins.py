"""Pins of the oracle's unrelaxed normal-ordered 2-RDM Gamma_N (reading R14:
the Lagrangian's derivative with respect to the integrals of the CC equations
and energy at a fixed reference) against finite differences of the converged
Omega_CC and against the exact zero of a non-interacting reference."""
import numpy as np
import torch

from oracle import ftccsd as fc
from oracle import systems
from paper_2004_01729_gb300 import workloads as wl


def _symmetric_perturbation(n, seed):
    """A random dV with the symmetries of <pq||rs> (antisymmetric in each
    pair, symmetric under (pq) <-> (rs))."""
    rng = np.random.default_rng(seed)
    d = torch.tensor(rng.normal(size=(n, n, n, n)))
    d = d - d.permute(1, 0, 2, 3)
    d = d - d.permute(0, 1, 3, 2)
    return 0.5 * (d + d.permute(2, 3, 0, 1))


def _richardson_derivative(s, beta, mu, ng, d, h, thr=0.0):
    def central(step):
        up = fc.omega_cc_frozen_reference(s, beta, mu, ng, s["eri"] + step * d, thr, tol=1e-14, tol_amp=1e-12)
        dn = fc.omega_cc_frozen_reference(s, beta, mu, ng, s["eri"] - step * d, thr, tol=1e-14, tol_amp=1e-12)
        return (up - dn) / (2.0 * step)
    return (4.0 * central(h / 2.0) - central(h)) / 3.0


def test_rdm2_matches_finite_differences_on_the_ring():
    s = systems.hubbard_1d(4, 1.0, 2.0)
    G = fc.rdm2_normal(s, 1.0, 1.0, 16)
    d = _symmetric_perturbation(s["eri"].shape[0], 5)
    fd = _richardson_derivative(s, 1.0, 1.0, 16, d, 4e-4)
    assert abs(float(torch.sum(G * d)) - fd) < 1e-10


def test_rdm2_matches_finite_differences_on_a_random_truncated_system():
    """A coupled random system with one orbital truncated from each space."""
    h, eri, eps = wl.random_generic_system(21, 7, v_scale=0.04)
    s = systems.generic(torch.tensor(h), torch.tensor(eri), torch.tensor(eps))
    beta, mu, thr, ng = 2.5, -0.1, 0.05, 12
    G = fc.rdm2_normal(s, beta, mu, ng, thr)
    d = _symmetric_perturbation(len(eps), 11)
    fd = _richardson_derivative(s, beta, mu, ng, d, 4e-4, thr)
    assert abs(float(torch.sum(G * d)) - fd) < 1e-10 * max(1.0, abs(fd))


def test_rdm2_vanishes_for_an_exact_reference():
    """At U = 0 the k-space reference is exact: s = 0, lambda = 0, Gamma_N = 0."""
    s = systems.hubbard_1d(4, 1.0, 0.0)
    assert float(fc.rdm2_normal(s, 1.0, 0.0, 16).abs().max()) == 0.0
