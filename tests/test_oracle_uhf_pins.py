"""Pins of the oracle's UHF reference for the site-basis Hubbard ring
(Sec. IV.A: FT-CCSD from a zero-temperature UHF reference, whose orbital
energies are the diagonal of the UHF Fock matrix) against values fixed by
mathematics: SCF invariants, the variational principle and the restricted
solution below the instability, unitary invariance of the many-body
spectrum, the atomic limit (where UHF is the Neel state), and exactness of
FT-CCSD for a one-body problem."""
import numpy as np
import torch

from oracle import exact
from oracle import ftccsd as fc
from oracle import systems


def _rhf_energy(L, t, U):
    """Closed-shell restricted energy at half filling: twice the lowest L/2
    hopping eigenvalues plus U L / 4 (uniform density 1/2 per spin)."""
    hs = systems.hubbard_1d_sites(L, t, U)["h"][:L, :L].numpy()
    w = np.linalg.eigvalsh(hs)
    return 2.0 * np.sum(w[:L // 2]) + U * L * 0.25


def test_uhf_scf_invariants():
    """The converged density commutes with its Fock matrix and is an
    idempotent projector onto n_sigma orbitals."""
    L, U = 6, 4.0
    u = systems.uhf_site_hubbard(L, 1.0, U)
    for sg in range(2):
        F = u["h_site"] + U * np.diag(u["n"][1 - sg])
        P = u["P"][sg]
        assert np.max(np.abs(F @ P - P @ F)) < 1e-9
        assert np.max(np.abs(P @ P - P)) < 1e-12
        assert abs(np.trace(P) - L / 2) < 1e-12


def test_uhf_restricted_below_and_broken_above_the_instability():
    """U = 0.5: the Neel guess relaxes to the restricted solution (no
    magnetisation, the restricted energy); U = 8: spin symmetry breaks and
    the energy falls below the restricted one (variational principle)."""
    L = 6
    lo = systems.uhf_site_hubbard(L, 1.0, 0.5)
    assert np.max(np.abs(lo["n"] - 0.5)) < 1e-8
    assert abs(lo["energy"] - _rhf_energy(L, 1.0, 0.5)) < 1e-10
    hi = systems.uhf_site_hubbard(L, 1.0, 8.0)
    ms = np.mean([(-1) ** i * (hi["n"][0, i] - hi["n"][1, i]) for i in range(L)])
    assert ms > 0.9
    assert hi["energy"] < _rhf_energy(L, 1.0, 8.0) - 1.0


def test_uhf_basis_leaves_the_many_body_spectrum_unchanged():
    """h and <pq||rs> transformed to the UHF orbitals describe the same
    Hamiltonian: the exact grand potential is the site-basis one."""
    for L, U in ((2, 3.0), (3, 5.0)):
        site = systems.hubbard_1d_sites(L, 1.0, U)
        uhf = systems.hubbard_1d_uhf(L, 1.0, U)
        a = exact.fock_space_omega(site["h"].numpy(), site["eri"].numpy(), 1.3, U / 2.0)
        b = exact.fock_space_omega(uhf["h"].numpy(), uhf["eri"].numpy(), 1.3, U / 2.0)
        assert abs(a - b) < 1e-10


def test_uhf_atomic_limit_is_the_neel_reference():
    """At t = 0 the UHF orbitals are sites and the UHF energies are the Neel
    reference energies, so FT-CCSD gives the Neel-reference Omega."""
    L, U = 2, 3.0
    uhf = systems.hubbard_1d_uhf(L, 0.0, U)
    neel = systems.hubbard_1d_neel(L, 0.0, U)
    for sg in range(2):
        assert torch.equal(torch.sort(uhf["eps"][sg * L:(sg + 1) * L]).values,
                           torch.sort(neel["eps"][sg * L:(sg + 1) * L]).values)
    a = fc.omega_at(uhf, 1.0, U / 2.0, 16)
    b = fc.omega_at(neel, 1.0, U / 2.0, 16)
    assert abs(a - b) < 1e-12


def test_uhf_reference_without_interaction_is_exact():
    """At U = 0 the UHF orbitals diagonalise the hopping, the reference is
    the exact non-interacting system and Omega_CC = 0."""
    s = systems.hubbard_1d_uhf(4, 1.0, 0.0)
    sol = fc.solve(fc.Problem(s, 1.0, 0.2, 16))
    ex = exact.noninteracting_omega(systems.hubbard_1d_sites(4, 1.0, 0.0)["h"].numpy(), 1.0, 0.2)
    assert abs(sol["omega_cc"]) < 1e-12
    assert abs(sol["omega"] - ex) < 1e-12
