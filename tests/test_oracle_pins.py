"""Pins of the FP64 oracle against results fixed by the paper and by mathematics.

None of these compares the oracle with itself: each reference value is a
closed form, an exact diagonalisation, a library eigen-solver, a finite
difference, or an invariant.
"""
import math

import numpy as np
import pytest
import torch

from oracle import exact, ftccsd as fc, systems
from paper_2004_01729_gb300 import workloads as wl


# ---------------------------------------------------------------- quadrature (Sec. II.C, R1)
@pytest.mark.parametrize("ng", [4, 7, 16, 17])
def test_simpson_tensors_integrate_polynomials(ng):
    beta = 1.7
    tau, G, g = fc.simpson_G(ng, beta)
    for y in range(1, ng):
        top = 2 if y == 1 else 3           # G^1 is the quadratic rule, the rest are cubic-exact
        for p in range(top + 1):
            lhs = torch.sum(G[y] * tau ** p).item()
            rhs = tau[y].item() ** (p + 1) / (p + 1)
            assert abs(lhs - rhs) < 1e-13 * max(1.0, abs(rhs))
    assert torch.equal(g, G[-1])
    assert torch.all(G[0] == 0)


# ---------------------------------------------------------------- reference quantities
def test_fermi_and_omega0_closed_forms():
    eps = torch.tensor([-50.0, -1.0, 0.0, 0.3, 2.0, 80.0], dtype=torch.float64)
    beta, mu = 3.0, 0.2
    n, nb = fc.occupations(eps, beta, mu)
    assert torch.allclose(n + nb, torch.ones_like(n), atol=0, rtol=1e-15)
    direct = -sum(math.log1p(math.exp(-beta * (e - mu))) if beta * (e - mu) > -30
                  else -beta * (e - mu) + math.log1p(math.exp(beta * (e - mu)))
                  for e in eps.tolist()) / beta
    assert abs(fc.omega0(eps, beta, mu).item() - direct) < 1e-12


def test_mean_field_part_is_exact_first_order():
    """Omega0 + Omega1 equals the non-interacting Omega plus first-order
    perturbation theory: dOmega1/dn_q = f_qq - eps_q (App. B)."""
    h, eri, eps = wl.random_generic_system(3, 5)
    n = torch.tensor(np.random.default_rng(0).uniform(0.1, 0.9, 5), requires_grad=True)
    o1 = fc.omega1(torch.tensor(h), torch.tensor(eri), torch.tensor(eps), n)
    (g,) = torch.autograd.grad(o1, n)
    f = fc.fock(torch.tensor(h), torch.tensor(eri), n.detach())
    assert torch.allclose(g, torch.diagonal(f) - torch.tensor(eps), atol=1e-13)


# ---------------------------------------------------------------- integrals
@pytest.mark.parametrize("n_pw", [1, 7, 19, 27, 33, 57, 81, 93, 123])
def test_plane_wave_shell_counts(n_pw):
    assert len(systems.plane_wave_grid(n_pw)) == n_pw


def test_plane_wave_open_shell_rejected():
    with pytest.raises(ValueError):
        systems.plane_wave_grid(20)


@pytest.mark.parametrize("build", [lambda: systems.hubbard_1d(6, 1.0, 2.0),
                                   lambda: systems.ueg(14, 1.0, 19)])
def test_integral_symmetries(build):
    s = build()
    g = s["eri"]
    assert torch.allclose(g, -g.permute(1, 0, 2, 3), atol=0)
    assert torch.allclose(g, -g.permute(0, 1, 3, 2), atol=0)
    assert torch.allclose(g, g.permute(2, 3, 0, 1), atol=0)
    assert torch.allclose(s["h"], s["h"].T, atol=0)


def test_ueg_momentum_and_spin_conservation():
    s = systems.ueg(14, 1.0, 19)
    nv = systems.plane_wave_grid(19)
    M = len(nv)
    g = s["eri"].numpy()
    nz = np.argwhere(np.abs(g) > 0)
    for p, q, r, t in nz[:: max(1, len(nz) // 2000)]:
        assert np.all(nv[p % M] + nv[q % M] == nv[r % M] + nv[t % M])
        assert (p // M + q // M) == (r // M + t // M)


def test_ueg_cell_and_fermi_energy():
    s = systems.ueg(14, 1.0, 7)
    assert abs(s["vol"] ** (1 / 3) - 3.8851) < 1e-4
    assert abs(systems.ueg_fermi_energy(1.0) - 1.84158) < 1e-5   # 50.11 eV at rs = 1
    assert abs(wl.UEG_57["beta"] - 1.0860) < 1e-4


@pytest.mark.parametrize("L", [2, 4])
def test_hubbard_k_space_equals_site_basis(L):
    """Same Fock-space spectrum from the k-space and the site-basis integrals."""
    a = systems.hubbard_1d(L, 1.0, 2.5)
    b = systems.hubbard_1d_sites(L, 1.0, 2.5)
    oa = exact.fock_space_omega(a["h"].numpy(), a["eri"].numpy(), 1.3, 0.7)
    ob = exact.fock_space_omega(b["h"].numpy(), b["eri"].numpy(), 1.3, 0.7)
    assert abs(oa - ob) < 1e-12


def test_hubbard_reference_is_thermal_hf_at_half_filling():
    s = systems.hubbard_1d(6, 1.0, 3.0)
    p = fc.Problem(s, 0.8, 1.5, 8)
    assert torch.max(torch.abs(p.Fbar)).item() < 1e-14


# ---------------------------------------------------------------- exact limits of the method
def test_zero_interaction_gives_zero_correlation():
    """P1: at U = 0 the k-space reference is exact: Omega_CC = 0 and Omega is
    the non-interacting grand potential."""
    s = systems.hubbard_1d(6, 1.0, 0.0)
    sol = fc.solve(fc.Problem(s, 1.0, 0.0, 16))
    assert sol["omega_cc"] == 0.0
    assert abs(sol["omega"] - exact.noninteracting_omega(s["h"].numpy(), 1.0, 0.0)) < 1e-12


def test_single_orbital_shift_is_exact_with_h4_error():
    """P2: one orbital with f - eps = delta; FT-CCSD singles are exact for a
    one-body perturbation, so Omega -> exact with O(h^4) quadrature error."""
    eps, dl, beta, mu = 0.3, 0.7, 2.0, 0.1
    s = systems.generic(torch.tensor([[eps + dl]]), torch.zeros(1, 1, 1, 1), torch.tensor([eps]))
    ex = exact.noninteracting_omega(np.array([[eps + dl]]), beta, mu)
    err = [fc.omega_at(s, beta, mu, ng) - ex for ng in (16, 32, 64)]
    assert abs(err[-1]) < 2e-10
    for a, b in zip(err, err[1:]):
        assert 8.0 < a / b < 24.0


def test_general_one_body_perturbation_is_exact():
    """P2': off-diagonal one-body perturbation (Delta != 0 singles)."""
    rng = np.random.default_rng(3)
    a = rng.normal(size=(4, 4))
    h = 0.5 * (a + a.T)
    eps = np.diag(h) + 0.3 * rng.normal(size=4)
    s = systems.generic(torch.tensor(h), torch.zeros(4, 4, 4, 4), torch.tensor(eps))
    ex = exact.noninteracting_omega(h, 1.5, 0.2)
    err = [fc.omega_at(s, 1.5, 0.2, ng) - ex for ng in (16, 32)]
    assert abs(err[-1]) < 1e-6
    assert 10.0 < err[0] / err[1] < 40.0


def test_hubbard_atom_is_exact():
    """P3: the half-filled Hubbard atom (2 spin orbitals, h = 0, eps = mu = U/2)
    has Omega = -beta^-1 ln(2 + 2 exp(beta U / 2)) and FT-CCSD reproduces it."""
    U, beta = 4.0, 2.0
    s = systems.hubbard_1d(1, 0.0, U)
    ex = -math.log(2.0 + 2.0 * math.exp(beta * U / 2.0)) / beta
    err = [fc.omega_at(s, beta, U / 2.0, ng) - ex for ng in (32, 64)]
    assert abs(err[-1]) < 2e-8
    assert 10.0 < err[0] / err[1] < 20.0


def _phi(delta, beta):
    """int_0^beta (1 - exp(-Delta tau)) / Delta dtau, with its series near 0 (R10)."""
    y = beta * delta
    out = np.empty_like(delta)
    small = np.abs(y) < 1e-2
    d = delta[~small]
    out[~small] = (beta * d - 1.0 + np.exp(-beta * d)) / d ** 2
    ys = y[small]
    out[small] = beta ** 2 * (0.5 - ys / 6.0 + ys ** 2 / 24.0 - ys ** 3 / 120.0)
    return out


def test_first_iteration_is_ft_mp2():
    """P4: from s = 0 the first iteration's linear energy integrates to the
    second-order grand potential (Sec. III.A; last term read with the square):
    Omega2 = -beta^-1 [1/4 sum |<ij||ab>|^2 + sum |f_ai|^2] phi(Delta)."""
    h, eri, eps = wl.random_generic_system(5, 5, v_scale=0.1)
    s = systems.generic(torch.tensor(h), torch.tensor(eri), torch.tensor(eps))
    beta, mu = 1.2, 0.1
    errs = []
    for ng in (16, 32, 64):
        p = fc.Problem(s, beta, mu, ng)
        z1 = torch.zeros((ng, 5, 5), dtype=torch.float64)
        z2 = torch.zeros((ng, 5, 5, 5, 5), dtype=torch.float64)
        t1, t2 = fc.fixed_point_map(p, z1, z2)
        e_lin = (torch.einsum("ia,xia->x", p.F("ia"), t1)
                 + 0.25 * torch.einsum("ijab,xijab->x", p.V("ijab"), t2))
        om = (torch.sum(p.g * e_lin) / beta).item()
        d1 = p.D1.numpy()
        d2 = p.D2.numpy()
        closed = -(0.25 * np.sum(p.V("ijab").numpy() ** 2 * _phi(d2, beta))
                   + np.sum(p.F("ai").numpy().T ** 2 * _phi(d1, beta))) / beta
        errs.append(om - closed)
    assert abs(errs[-1]) < 2e-8
    assert 13.0 < errs[0] / errs[1] < 19.0
    assert 13.0 < errs[1] / errs[2] < 19.0


def test_quadrature_order_on_hubbard_6():
    """P5 / Table I: the Simpson integral method converges as h^4."""
    c = wl.HUBBARD_6
    s = systems.hubbard_1d(c["L"], c["t"], c["U"])
    om = [fc.omega_at(s, c["beta"], c["mu"], ng) for ng in (16, 32, 64)]
    r = (om[0] - om[1]) / (om[1] - om[2])
    assert 11.0 < r < 22.0


def test_third_order_exact_against_fock_space():
    """P7: against exact diagonalisation of the 4-site ring the error falls as U^4
    (FT-CCSD is exact through third order in the interaction)."""
    errs = []
    for U in (0.5, 0.25):
        s = systems.hubbard_1d(4, 1.0, U)
        o1 = fc.omega_at(s, 1.0, U / 2, 24)
        o2 = fc.omega_at(s, 1.0, U / 2, 48)
        oinf = o2 + (o2 - o1) / 15.0
        errs.append(oinf - exact.fock_space_omega(s["h"].numpy(), s["eri"].numpy(), 1.0, U / 2))
    assert 13.0 < errs[0] / errs[1] < 19.0


@pytest.mark.slow
def test_two_electron_low_temperature_limit():
    """P6: at low T the kernel energy mid-grid, E(beta/2), tends to the
    ground-state CCSD correlation energy, and CCSD is exact for two electrons,
    so it equals E_FCI(2 e) - E_ref from diagonalisation.  Richardson over
    two grids removes the h^4 error."""
    rng = np.random.default_rng(11)
    N = 4
    a = rng.normal(size=(N, N))
    h = 0.3 * (a + a.T) / 2 + np.diag([-1.3, -1.0, 1.0, 1.3])
    b = rng.normal(size=(N, N, N, N))
    b = b + b.transpose(2, 3, 0, 1)
    b = b + b.transpose(1, 0, 3, 2)
    eri = 0.05 * (b - b.transpose(1, 0, 2, 3) - b.transpose(0, 1, 3, 2) + b.transpose(1, 0, 3, 2))
    occ = np.array([1.0, 1.0, 0.0, 0.0])
    eps = np.diag(h + np.einsum("prqr,r->pq", eri, occ)).copy()
    e, k = exact.fock_space_spectrum(h, eri)
    e0 = [e[k == kk].min() for kk in range(N + 1)]
    mu = 0.5 * ((e0[2] - e0[1]) + (e0[3] - e0[2]))
    eref = h[0, 0] + h[1, 1] + eri[0, 1, 0, 1]
    target = e0[2] - eref
    s = systems.generic(torch.tensor(h), torch.tensor(eri), torch.tensor(eps))
    mids = []
    for ng in (121, 241):
        p = fc.Problem(s, 10.0, mu, ng)
        sol = fc.solve(p, tol_amp=1e-9)
        mids.append(fc.energy(p, sol["t1"], sol["t2"])[ng // 2].item())
    extrap = mids[1] + (mids[1] - mids[0]) / 15.0
    assert abs(mids[1] - target) < 5e-6
    assert abs(extrap - target) < 5e-8


# ---------------------------------------------------------------- response (App. B)
def _fd(f, x, d):
    """Central difference with one Richardson step."""
    d1 = (f(x + d) - f(x - d)) / (2 * d)
    d2 = (f(x + d / 2) - f(x - d / 2)) / d
    return d2 + (d2 - d1) / 3.0


def test_adjoint_matches_finite_differences():
    """P8: dOmega/dmu, dOmega/dbeta and Tr p^cc = N against central differences
    of the converged discrete solution."""
    s = systems.hubbard_1d(4, 1.0, 3.0)
    beta, mu, ng = 1.3, 1.2, 10
    kw = dict(tol=1e-14, tol_amp=1e-13)
    r = fc.response(s, beta, mu, ng, solve_kw=kw)
    fm = _fd(lambda m: fc.omega_at(s, beta, m, ng, **kw), mu, 1e-3)
    fb = _fd(lambda b: fc.omega_at(s, b, mu, ng, **kw), beta, 1e-3)
    assert abs(r["dOmega_dmu"] - fm) < 1e-9
    assert abs(r["dOmega_dbeta"] - fb) < 1e-9
    assert abs(torch.trace(r["rdm1"]).item() - r["N"]) < 1e-12
    assert abs(r["S"] - beta * (r["E"] - mu * r["N"] - r["omega"])) < 1e-10


def test_rdm1_matches_finite_differences():
    """P8: p^cc_pq is the response to a symmetric one-body perturbation X_pq;
    diagonal entries also shift eps_q (App. B, type 1 + type 2 terms)."""
    h, eri, eps = wl.random_generic_system(9, 4, v_scale=0.08)
    s = systems.generic(torch.tensor(h), torch.tensor(eri), torch.tensor(eps))
    beta, mu, ng = 1.1, 0.05, 8
    kw = dict(tol=1e-14, tol_amp=1e-13)
    r = fc.response(s, beta, mu, ng, solve_kw=kw)

    def om(p, q, a):
        hh = s["h"].clone()
        ee = s["eps"].clone()
        hh[p, q] += a
        if p != q:
            hh[q, p] += a
        else:
            ee[p] += a
        return fc.omega_at(dict(s, h=hh, eps=ee), beta, mu, ng, **kw)

    for p, q in [(0, 0), (2, 2), (0, 1), (1, 3)]:
        fd = _fd(lambda a: om(p, q, a), 0.0, 1e-3)
        an = r["rdm1"][p, q].item() + (r["rdm1"][q, p].item() if p != q else 0.0)
        assert abs(an - fd) < 1e-9


def test_half_filling_particle_hole_symmetry():
    """P9: the even ring at mu = U/2 holds exactly L electrons."""
    s = systems.hubbard_1d(6, 1.0, 2.0)
    r = fc.response(s, 1.0, 1.0, 8)
    assert abs(r["N"] - 6.0) < 1e-10
