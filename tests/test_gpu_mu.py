"""The chemical potential of the coupled-cluster system at a fixed mean
electron number on the GPU (ftcc_mu_for_n, App. D) against the oracle's
search and against values fixed by mathematics: the Fermi root of the
non-interacting ring and the particle-hole symmetric point of the
half-filled ring."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import chemical_potential as cp, systems

pytestmark = pytest.mark.gpu
BETA, NG = 1.0, 16


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_01729_gb300 import ftcc
    c = ftcc.Context(0)
    yield c
    c.close()


def test_noninteracting_ring_lands_on_the_fermi_root(ctx):
    ctx.build_hubbard(6, 1.0, 0.0)
    e = systems.hubbard_1d(6, 1.0, 0.0)["eps"].numpy()
    root = brentq(lambda m: np.sum(1.0 / (1.0 + np.exp(BETA * (e - m)))) - 5.0, -20.0, 20.0, xtol=1e-15)
    mu, n, ev, _ = ctx.mu_for_n(BETA, 5.0, NG, mu0=0.0, precision="fp64")
    assert ev > 2
    assert abs(mu - root) < 1e-9 and abs(n - 5.0) < 1e-10


def test_half_filled_ring_is_particle_hole_symmetric(ctx):
    U = 2.0
    ctx.build_hubbard(6, 1.0, U)
    mu, n, _, r = ctx.mu_for_n(BETA, 6.0, NG, mu0=0.4, precision="fp64")
    assert abs(mu - U / 2.0) < 1e-8 and r["converged"]


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_off_half_filling_matches_the_oracle(ctx, prec):
    s = systems.hubbard_1d(6, 1.0, 2.0)
    ref = cp.mu_for_n(s, BETA, 5.0, NG)
    ctx.build_hubbard(6, 1.0, 2.0)
    mu0 = cp.mu_reference(s["eps"], BETA, 5.0)
    mu, n, ev, r = ctx.mu_for_n(BETA, 5.0, NG, mu0=mu0, precision=prec)
    assert abs(n - 5.0) < 1e-10
    assert abs(mu - ref["mu"]) < 1e-8, (mu, ref["mu"])


def test_block_sparse_search_matches_the_oracle(ctx):
    """The same search on the k-space ring with the block-sparse storage
    (its adjoint supplies N at every step)."""
    s = systems.hubbard_1d(6, 1.0, 2.0)
    ref = cp.mu_for_n(s, BETA, 5.0, NG)
    ctx.build_hubbard(6, 1.0, 2.0)
    mu0 = cp.mu_reference(s["eps"], BETA, 5.0)
    mu, n, _, r = ctx.mu_for_n(BETA, 5.0, NG, mu0=mu0, precision="fp64", block_sparse=1)
    assert r["converged"] and abs(n - 5.0) < 1e-10
    assert abs(mu - ref["mu"]) < 1e-8, (mu, ref["mu"])


def test_ueg57_electron_number_is_fixed_at_full_size(ctx):
    """App. D on the 114-spin-orbital gas: mu_CC with <N> = 14 from the
    block-sparse solves and adjoints; a fresh solve and adjoint at that mu
    give N = 14, and mu_CC lies below mu_0 (N(mu_0) = 14.2068 > 14 and
    dN/dmu > 0)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_ueg57.json")))
    c = gold["config"]
    ctx.build_ueg(c["n_elec"], c["rs"], c["n_pw"])
    mu0 = gold["mu"]
    mu, n, ev, r = ctx.mu_for_n(c["beta"], 14.0, c["ngrid"], mu0=mu0, dmu=0.02, precision="fp64", block_sparse=1)
    assert r["converged"] and abs(n - 14.0) < 1e-9 and ev <= 12
    assert mu < mu0
    ctx.solve(c["beta"], mu, c["ngrid"], precision="fp64", block_sparse=1, tol_omega=1e-12, tol_amp=1e-10)
    d, _ = ctx.adjoint(with_rdm1=False)
    assert abs(d["N"] - 14.0) < 1e-8
