"""Pins of the oracle with the Neel-state reference of the site-basis Hubbard
model (Sec. IV.A: the reference is the diagonal of the zero-temperature Fock
matrix of the Neel determinant) and of the staggered magnetisation of the
FT-CCSD 1-RDM (Fig. 5), against exact results."""
import math

import numpy as np
import torch

from oracle import exact
from oracle import ftccsd as fc
from oracle import systems


def test_neel_reference_energies():
    """eps_{i sigma} = U on the spin opposite to the Neel electron of site i."""
    s = systems.hubbard_1d_neel(4, 1.0, 3.0)
    assert torch.equal(s["eps"], torch.tensor([0.0, 3.0, 0.0, 3.0, 3.0, 0.0, 3.0, 0.0], dtype=torch.float64))


def test_neel_reference_without_interaction_is_exact():
    """At U = 0 every reference energy is 0 and hopping is a one-body
    perturbation, which FT-CCSD treats exactly: Omega -> the non-interacting
    grand potential with the quadrature's h^4 error."""
    s = systems.hubbard_1d_neel(4, 1.0, 0.0)
    ex = exact.noninteracting_omega(s["h"].numpy(), 1.0, 0.3)
    err = [fc.omega_at(s, 1.0, 0.3, ng) - ex for ng in (16, 32)]
    assert abs(err[-1]) < 1e-6
    assert 10.0 < err[0] / err[1] < 24.0


def test_neel_hubbard_atom_is_exact_and_unmagnetised():
    """The half-filled Hubbard atom from the spin-broken reference
    (eps_up = 0, eps_down = U): Omega -> -beta^-1 ln(2 + 2 exp(beta U / 2))
    and the 1-RDM's spin polarisation -> 0, the exact atom being spin
    symmetric; both errors fall as h^4."""
    U, beta = 4.0, 2.0
    s = systems.hubbard_1d_neel(1, 0.0, U)
    ex = -math.log(2.0 + 2.0 * math.exp(beta * U / 2.0)) / beta
    res = [fc.response(s, beta, U / 2.0, ng) for ng in (64, 128)]
    err = [r["omega"] - ex for r in res]
    ms = [systems.staggered_magnetisation(r["rdm1"], 1) for r in res]
    assert abs(err[-1]) < 5e-8 and 8.0 < err[0] / err[1] < 20.0
    assert abs(ms[-1]) < 1e-7 and 8.0 < ms[0] / ms[1] < 20.0
    assert abs(res[-1]["N"] - 1.0) < 1e-10


def test_staggered_magnetisation_of_a_neel_density():
    """m_s of the Neel determinant's own density is 1 (and -1 for the other
    sublattice assignment); a paramagnetic density gives 0."""
    L = 4
    d = np.zeros(2 * L)
    for i in range(L):
        d[i] = 1.0 if i % 2 == 0 else 0.0
        d[L + i] = 1.0 - d[i]
    assert systems.staggered_magnetisation(np.diag(d), L) == 1.0
    assert systems.staggered_magnetisation(np.diag(1.0 - d), L) == -1.0
    assert systems.staggered_magnetisation(np.diag(np.full(2 * L, 0.5)), L) == 0.0
