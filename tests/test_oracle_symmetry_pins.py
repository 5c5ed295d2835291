"""Conservation pins of the oracle's S kernel (Eqs. ccS1, ccS2, term by
term): with integrals that conserve crystal momentum and spin (the k-space
Hubbard ring, the plane-wave gas), amplitudes that conserve them are mapped
to residuals that conserve them.  An index moved between the two pairs of
an integral or an amplitude (e.g. <kb||cj> read as <kc||bj>) puts weight on
forbidden entries and fails here; a swap inside one antisymmetric pair only
flips a sign, keeps the conservation pattern, and is left to the exactness
and closed-form pins."""
import numpy as np
import pytest
import torch

from oracle import ftccsd as fc
from oracle import systems


def _labels(kind):
    """(system, momentum label per spin orbital as an integer vector, modulus
    for the momentum sum or None, spin per spin orbital)."""
    if kind == "hubbard":
        L = 6
        s = systems.hubbard_1d(L, 1.0, 3.0)
        mom = np.array([[p % L] for p in range(2 * L)])
        return s, mom, L, np.array([p // L for p in range(2 * L)])
    M = 7
    s = systems.ueg(2, 1.0, M)
    vec = systems.plane_wave_grid(M)
    mom = np.array([vec[p % M] for p in range(2 * M)])
    return s, mom, None, np.array([p // M for p in range(2 * M)])


def _zero(d, mod):
    """d = 0 (mod the lattice period when there is one)."""
    return bool(np.all((d % mod) == 0)) if mod else bool(np.all(d == 0))


@pytest.mark.parametrize("kind", ["hubbard", "ueg"])
def test_s_kernel_conserves_momentum_and_spin(kind):
    s, mom, mod, spin = _labels(kind)
    N = len(spin)
    prob = fc.Problem(s, 1.0, 0.3, 3)
    assert len(prob.iO) == N and len(prob.iV) == N   # no truncation: slot index = orbital
    ok1 = np.zeros((N, N), dtype=bool)
    for i in range(N):
        for a in range(N):
            ok1[i, a] = spin[i] == spin[a] and _zero(mom[i] - mom[a], mod)
    ok2 = np.zeros((N, N, N, N), dtype=bool)
    for i in range(N):
        for j in range(N):
            for a in range(N):
                for b in range(N):
                    ok2[i, j, a, b] = (spin[i] + spin[j] == spin[a] + spin[b]
                                       and _zero(mom[i] + mom[j] - mom[a] - mom[b], mod))
    assert 0 < ok1.sum() < N * N and 0 < ok2.sum() < N ** 4
    rng = np.random.default_rng(17)
    t1 = torch.tensor(np.where(ok1, rng.normal(scale=0.1, size=(N, N)), 0.0))[None]
    r2 = rng.normal(scale=0.1, size=(N, N, N, N))
    r2 = r2 - r2.transpose(1, 0, 2, 3)
    r2 = r2 - r2.transpose(0, 1, 3, 2)
    t2 = torch.tensor(np.where(ok2, r2, 0.0))[None]
    S1 = fc.S1(prob, t1, t2)[0].numpy()
    S2 = fc.S2(prob, t1, t2)[0].numpy()
    assert np.max(np.abs(S1[~ok1])) == 0.0
    assert np.max(np.abs(S2[~ok2])) == 0.0
    assert np.max(np.abs(S2[ok2])) > 1e-3   # the allowed part is not trivially empty
