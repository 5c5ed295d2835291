"""The site-basis references of the Hubbard ring (Sec. IV.A: the Neel state
and zero-temperature UHF) and the unrelaxed two-particle density Gamma_N
(App. B) on the GPU against the pinned oracle: grand potential, N, E, S, the
staggered magnetisation of the 1-RDM (Fig. 5) and Gamma_N element by
element."""
import numpy as np
import pytest
import torch

from oracle import ftccsd as fc, systems
from paper_2004_01729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_01729_gb300 import ftcc
    c = ftcc.Context(0)
    yield c
    c.close()


def test_neel_system_matches_the_oracle_builder(ctx):
    ref = systems.hubbard_1d_neel(4, 1.0, 3.0)
    ctx.build_hubbard(4, 1.0, 3.0, reference="neel")
    h, eri, eps = ctx.get_system()
    assert np.max(np.abs(h - ref["h"].numpy())) == 0.0
    assert np.max(np.abs(eri - ref["eri"].numpy())) == 0.0
    assert np.max(np.abs(eps - ref["eps"].numpy())) == 0.0


@pytest.mark.parametrize("L,U", [(4, 2.0), (6, 4.0)])
def test_neel_reference_response_matches_oracle(ctx, L, U):
    """Omega, N, E, S and the staggered magnetisation of the 1-RDM with the
    Neel reference at half filling (mu = U/2)."""
    beta, mu, ng = 1.0, U / 2.0, 8
    s = systems.hubbard_1d_neel(L, 1.0, U)
    ref = fc.response(s, beta, mu, ng, solve_kw=dict(tol=1e-13, tol_amp=1e-11))
    ctx.build_hubbard(L, 1.0, U, reference="neel")
    r = ctx.solve(beta, mu, ng, precision="fp64", tol_omega=1e-12, tol_amp=1e-10)
    assert r["converged"] and abs(r["omega"] - ref["omega"]) < 1e-8
    d, rdm = ctx.adjoint(with_rdm1=True)
    for key in ("N", "E", "S"):
        assert abs(d[key] - ref[key]) < 1e-8, (key, d[key], ref[key])
    assert np.max(np.abs(rdm - ref["rdm1"].numpy())) < 1e-8
    ms_gpu = systems.staggered_magnetisation(rdm, L)
    ms_ref = systems.staggered_magnetisation(ref["rdm1"], L)
    assert abs(ms_gpu - ms_ref) < 1e-8


@pytest.mark.parametrize("L,U,beta", [(4, 8.0, 0.5), (6, 6.0, 1.0)])
def test_uhf_reference_matches_oracle(ctx, L, U, beta):
    """The broken-symmetry UHF reference: its orbital energies, and Omega, N,
    E and S of the FT-CCSD solve (invariant under rotations among degenerate
    UHF orbitals, which the two eigen-solvers may pick differently).  (At
    U = 8 and beta = 1 the fixed-point iteration diverges from s = 0 in the
    oracle as on the GPU, so the 4-site case runs at beta = 0.5.)"""
    mu, ng = U / 2.0, 8
    s = systems.hubbard_1d_uhf(L, 1.0, U)
    ctx.build_hubbard(L, 1.0, U, reference="uhf")
    h, eri, eps = ctx.get_system()
    assert np.max(np.abs(eps - s["eps"].numpy())) < 1e-10
    assert abs(np.trace(h) - float(torch.trace(s["h"]))) < 1e-10
    ref = fc.response(s, beta, mu, ng, solve_kw=dict(tol=1e-13, tol_amp=1e-11, max_iter=400))
    assert ref["solve"]["converged"]
    r = ctx.solve(beta, mu, ng, precision="fp64", tol_omega=1e-12, tol_amp=1e-10, max_iter=400)
    assert r["converged"] and abs(r["omega"] - ref["omega"]) < 1e-8
    d, _ = ctx.adjoint(with_rdm1=False)
    for key in ("N", "E", "S"):
        assert abs(d[key] - ref[key]) < 1e-8, (key, d[key], ref[key])


def test_unknown_reference_is_rejected(ctx):
    from paper_2004_01729_gb300 import ftcc
    with pytest.raises(ftcc.FTCCError):
        ctx.build_hubbard(4, 1.0, 2.0, reference=7)


@pytest.mark.parametrize("which", ["kspace4", "neel4", "generic7_truncated"])
def test_rdm2_matches_oracle(ctx, which):
    """Gamma_N element by element against the oracle's derivative of the
    Lagrangian with respect to the integrals (itself pinned to central
    differences of the converged Omega_CC)."""
    if which == "kspace4":
        s, beta, mu, ng, thr = systems.hubbard_1d(4, 1.0, 2.0), 1.0, 1.0, 8, 0.0
        ctx.build_hubbard(4, 1.0, 2.0)
    elif which == "neel4":
        s, beta, mu, ng, thr = systems.hubbard_1d_neel(4, 1.0, 2.0), 1.0, 1.0, 8, 0.0
        ctx.build_hubbard(4, 1.0, 2.0, reference="neel")
    else:
        h, eri, eps = wl.random_generic_system(21, 7, v_scale=0.04)
        s = systems.generic(torch.tensor(h), torch.tensor(eri), torch.tensor(eps))
        beta, mu, ng, thr = 2.5, -0.1, 8, 0.05
        ctx.build_generic(h, eri, eps)
    G = fc.rdm2_normal(s, beta, mu, ng, thr, solve_kw=dict(tol=1e-13, tol_amp=1e-11)).numpy()
    G = 0.5 * (G + G.transpose(2, 3, 0, 1))   # the part seen by perturbations with the integrals' symmetries
    r = ctx.solve(beta, mu, ng, precision="fp64", trunc_thr=thr, tol_omega=1e-12, tol_amp=1e-10)
    assert r["converged"]
    ctx.adjoint(with_rdm1=False)
    g = ctx.rdm2()
    assert np.max(np.abs(G)) > 1e-4
    assert np.max(np.abs(g - G)) < 1e-9 * max(1.0, np.max(np.abs(G)))


def test_rdm2_before_the_adjoint_is_a_state_error(ctx):
    from paper_2004_01729_gb300 import ftcc
    ctx.build_hubbard(4, 1.0, 2.0)
    ctx.solve(1.0, 1.0, 6, precision="fp64")
    with pytest.raises(ftcc.FTCCError) as e:
        ctx.rdm2()
    assert e.value.status == ftcc.ERR_STATE
