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
