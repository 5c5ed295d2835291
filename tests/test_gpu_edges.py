"""GPU edge cases of the sweep against the oracle and the exact limits:
the non-interacting ring (U = 0, where Omega_CC vanishes), the shortest
grid (three tau points: only the G^1 row and the first Simpson panel), odd
and even point counts (composite 1/3 only, or 1/3 then 3/8), a grid of
arbitrary length (ragged against every tile and chunk size), and tau
streaming with a window longer than the grid."""
import numpy as np
import pytest

from oracle import ftccsd as fc, systems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_01729_gb300 import ftcc
    c = ftcc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_noninteracting_ring_has_no_correlation(ctx, prec):
    L, beta, mu = 6, 1.3, 0.0
    ctx.build_hubbard(L, 1.0, 0.0)
    r = ctx.solve(beta, mu, 8, precision=prec, refine_max_iter=4)
    assert r["converged"]
    assert abs(r["omega_cc"]) < 1e-13
    eps = systems.hubbard_1d(L, 1.0, 0.0)["eps"].numpy()
    exact = -np.sum(np.log1p(np.exp(-beta * (eps - mu)))) / beta
    assert abs(r["omega"] - exact) < 1e-12


@pytest.mark.parametrize("ngrid", [3, 4, 5, 17, 23])
def test_grid_lengths_match_oracle(ctx, ngrid):
    L, U, beta, mu = 6, 2.0, 1.0, 1.0
    ref = fc.solve(fc.Problem(systems.hubbard_1d(L, 1.0, U), beta, mu, ngrid), tol=1e-13, tol_amp=1e-11)
    assert ref["converged"]
    ctx.build_hubbard(L, 1.0, U)
    r = ctx.solve(beta, mu, ngrid, precision="fp64", tol_omega=1e-12, tol_amp=1e-10)
    assert r["converged"]
    assert abs(r["omega"] - ref["omega"]) < 1e-8
    m = ctx.solve(beta, mu, ngrid, precision="bf16x3", refine_max_iter=60)
    assert m["converged"] and abs(m["omega"] - ref["omega"]) < 1e-6


def test_stream_window_longer_than_grid(ctx):
    L, U, beta, mu, ngrid = 6, 2.0, 1.0, 1.0, 5
    ctx.build_hubbard(L, 1.0, U)
    full = ctx.solve(beta, mu, ngrid, precision="fp64", tol_omega=1e-12, tol_amp=1e-10)
    got = ctx.solve(beta, mu, ngrid, precision="fp64", tol_omega=1e-12, tol_amp=1e-10, stream_tau=1, tau_chunk=9)
    assert got["converged"] and abs(got["omega"] - full["omega"]) < 1e-13
