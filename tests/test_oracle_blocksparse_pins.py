"""Pins of the momentum/spin block-sparse execution of the oracle
(oracle/blocksparse.py) and of the plane-wave gas integrals it is used on.

* The charge-stored integrals are the dense builders' integrals (every
  element, including the zeros outside the conserving set).
* S1, S2 and E of random charge-conserving amplitudes equal the dense
  oracle's term-by-term Eqs. ccS1, ccS2 and E to 1e-12 on 19-, 27- and
  33-plane-wave gases and on the k-space Hubbard ring.
* Converged solves equal the dense oracle's (same iterations, Omega to 1e-12).
* The gas's Coulomb prefactor and Hartree-Fock reference energies meet the
  textbook exchange energy of the homogeneous gas, -(3/4pi) k_F per
  electron, with the known finite-size correction of a Coulomb sum without
  its G = 0 term, xi / (2 L) with xi = 2.837297 the simple-cubic Madelung
  constant; a dropped (2 pi / L)^2, a wrong 4 pi or a sign slip in the
  exchange sum misses it by far more than the tolerance.
"""
import math

import numpy as np
import pytest
import torch

from oracle import blocksparse as bs, ftccsd as fc, systems
from paper_2004_01729_gb300 import workloads as wl


def _close(a, b, tol):
    scale = max(1.0, float(torch.max(torch.abs(b))))
    return float(torch.max(torch.abs(a - b))) <= tol * scale


@pytest.mark.parametrize("which", ["hubbard4", "hubbard6", "ueg7", "ueg19"])
def test_charge_stored_integrals_equal_dense_builders(which):
    if which.startswith("hubbard"):
        L = int(which[7:])
        sc, d = bs.hubbard_1d(L, 1.0, 2.5), systems.hubbard_1d(L, 1.0, 2.5)
    else:
        n = int(which[3:])
        sc, d = bs.ueg(14, 1.0, n), systems.ueg(14, 1.0, n)
    ex = bs.expand(sc)
    assert torch.equal(ex["eri"] == 0, d["eri"] == 0)       # same conserving set
    assert _close(ex["eri"], d["eri"], 1e-15)
    assert _close(ex["h"], d["h"], 1e-15)
    assert _close(ex["eps"], d["eps"], 1e-14)


def _kernels_match(sc, dense, beta, mu, ng, seed, sample=0):
    """Block-sparse vs dense S1, S2, E and propagation on random conserving
    amplitudes; with sample > 0 the dense terms are evaluated on that many
    random values of each output letter (every summed index in full)."""
    ch = sc["charges"]
    pb = bs.Problem(sc, beta, mu, ng)
    pd = fc.Problem(dense, beta, mu, ng)
    assert abs(pb.omega0.item() - pd.omega0.item()) < 1e-12
    assert abs(pb.omega1.item() - pd.omega1.item()) < 1e-12
    t1, t2 = bs.random_amplitudes(ch, seed, ng)
    d1, d2 = bs.dense_amplitudes(ch, t1, t2)
    S1b, S2b = bs.S1(pb, t1, t2), bs.S2(pb, t1, t2)
    g1, g2 = bs.dense_amplitudes(ch, S1b, S2b)
    assert _close(bs.energy(pb, t1, t2), fc.energy(pd, d1, d2), 1e-12)
    if sample:
        # random hole-like letters; particle-like letters chosen so that the
        # sampled block holds conserving elements (b balances i + j - a)
        rng = np.random.default_rng(seed)
        io = sorted(int(x) for x in rng.choice(ch.N, sample, replace=False))
        iv = set()
        while len(iv) < sample:
            i, j = rng.choice(io, 2, replace=False)
            a = int(rng.integers(ch.N))
            b = int(ch.find((ch.q[i] + ch.q[j] - ch.q[a])[None, :])[0])
            if b >= 0 and b != a and len(iv) <= sample - 2:
                iv.update((a, b))
            elif len(iv) == sample - 1:
                iv.add(a)
        io, iv = torch.tensor(io), torch.tensor(sorted(iv))
        r1 = fc.S1(pd, d1, d2, sel={"i": io, "a": iv})
        r2 = fc.S2(pd, d1, d2, sel={"i": io, "j": io, "a": iv, "b": iv})
        assert _close(g1[:, io][:, :, iv], r1, 1e-12)
        assert _close(g2[:, io][:, :, io][:, :, :, iv][:, :, :, :, iv], r2, 1e-12)
        assert float(torch.max(torch.abs(r2))) > 0
        return
    r1, r2 = fc.S1(pd, d1, d2), fc.S2(pd, d1, d2)
    assert _close(g1, r1, 1e-12)
    assert _close(g2, r2, 1e-12)
    # the propagation acts element by element: the stored elements propagate as the dense ones
    p2 = bs.dense_amplitudes(ch, t1, fc.propagate(pb, S2b, pb.D2))[1]
    assert _close(p2, fc.propagate(pd, r2, pd.D2), 1e-12)


@pytest.mark.parametrize("n_pw,sample", [(19, 0), (27, 6), (33, 6)])
def test_block_sparse_kernels_equal_dense_oracle_on_gas(n_pw, sample):
    _kernels_match(bs.ueg(14, 1.0, n_pw), systems.ueg(14, 1.0, n_pw), wl.ueg_beta(1.0, 0.5), 1.2, 3, n_pw,
                   sample)


def test_block_sparse_kernels_equal_dense_oracle_on_ring():
    _kernels_match(bs.hubbard_1d(6, 1.0, 3.0), systems.hubbard_1d(6, 1.0, 3.0), 1.3, 1.5, 4, 6)


@pytest.mark.parametrize("which", ["hubbard4", "ueg7"])
def test_block_sparse_solve_equals_dense_solve(which):
    if which == "hubbard4":
        sc, d, beta, mu, ng = bs.hubbard_1d(4, 1.0, 2.0), systems.hubbard_1d(4, 1.0, 2.0), 1.0, 1.0, 6
    else:
        sc, d, beta, mu, ng = bs.ueg(14, 1.0, 7), systems.ueg(14, 1.0, 7), 0.8, 0.6, 4
    a = bs.solve(bs.Problem(sc, beta, mu, ng), tol=1e-13, tol_amp=1e-11)
    b = fc.solve(fc.Problem(d, beta, mu, ng), tol=1e-13, tol_amp=1e-11)
    assert a["converged"] and b["converged"]
    assert a["iterations"] == b["iterations"]
    assert abs(a["omega"] - b["omega"]) < 1e-12
    assert abs(a["omega_cc"]) > 1e-3          # a correlated case
    g1, g2 = bs.dense_amplitudes(sc["charges"], a["t1"], a["t2"])
    assert _close(g2, b["t2"], 1e-11)


def test_truncating_threshold_is_refused():
    sc = bs.ueg(14, 1.0, 7)
    with pytest.raises(ValueError):
        bs.Problem(sc, 40.0, 0.0, 4, thr=0.3)


def test_gas_exchange_energy_meets_the_homogeneous_gas_limit():
    """E_x = 1/2 sum_occ (eps_p - |k_p|^2/2) of closed shells of 2 x 515
    electrons: (E_x/N - e_x) L -> xi/2 (finite size of a Coulomb sum without
    G = 0), e_x = -(3/4pi) k_F, k_F = (9pi/4)^(1/3) / rs."""
    xi = 2.837297
    for rs in (1.0, 4.0):
        ne, npw = 1030, 515
        eps, kin = systems.ueg_hf_energies(ne, rs, npw)
        ex = float(np.sum(eps[:npw] - kin[:npw]))          # two spins x 1/2
        L = (4.0 / 3.0 * math.pi * ne) ** (1.0 / 3.0) * rs
        e_tl = -3.0 / (4.0 * math.pi) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / rs
        assert abs((ex / ne - e_tl) * L - xi / 2) < 0.1, (rs, (ex / ne - e_tl) * L)
        # and the 14-electron shell of the workloads has the same prefactor:
        # its exchange energy scales exactly as 1/rs
    e1, k1 = systems.ueg_hf_energies(14, 1.0, 57)
    e4, k4 = systems.ueg_hf_energies(14, 4.0, 57)
    assert np.allclose(k4, k1 / 16.0, rtol=1e-14, atol=0)
    assert np.allclose(e4 - k4, (e1 - k1) / 4.0, rtol=1e-13, atol=0)
