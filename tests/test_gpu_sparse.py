"""The momentum/spin block-sparse execution (option block_sparse) of the
plane-wave gas and the k-space Hubbard ring on the GPU: its S kernel on
random charge-conserving amplitudes element by element against the oracle's
printed terms of Eqs. ccS1/ccS2, converged solves against the dense FP64 GPU
path and the oracle, the 114- and 162-spin-orbital gases against the
block-sparse oracle's converged goldens, and the argument checks."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import blocksparse as bs, ftccsd as fc, systems

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_01729_gb300 import ftcc
    c = ftcc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n_elec,n_pw", [(6, 7), (14, 19)])
def test_sparse_s_kernel_matches_oracle_terms(ctx, n_elec, n_pw):
    """S1 and S2 of random amplitudes that conserve momentum and spin, from
    the block-sparse kernel, against the dense oracle's 45 terms, element by
    element (every element, including the ones that must vanish)."""
    rs, beta, ng = 1.0, 1.5, 4
    sysc = bs.ueg(n_elec, rs, n_pw)
    t1c, t2c = bs.random_amplitudes(sysc["charges"], 11, 2, 0.05)
    d1, d2 = bs.dense_amplitudes(sysc["charges"], t1c, t2c)
    ctx.build_ueg(n_elec, rs, n_pw)
    mu = ctx.reference_mu(beta, float(n_elec))
    ctx.prepare(beta, mu, ng, precision="fp64", block_sparse=1)
    s1, s2 = ctx.eval_s(d1, d2)
    prob = fc.Problem(systems.ueg(n_elec, rs, n_pw), beta, mu, ng, 0.0)
    r1 = fc.S1(prob, d1, d2)
    r2 = fc.S2(prob, d1, d2)
    e1 = torch.max(torch.abs(s1.cpu() - r1)).item()
    e2 = torch.max(torch.abs(s2.cpu() - r2)).item()
    assert torch.max(torch.abs(r2)).item() > 1e-3
    assert e1 < 1e-12 * max(1.0, torch.max(torch.abs(r1)).item()), e1
    assert e2 < 1e-12 * max(1.0, torch.max(torch.abs(r2)).item()), e2


@pytest.mark.parametrize("n_elec,n_pw,against", [(6, 7, "oracle"), (14, 19, "oracle"), (14, 33, "fp64")])
def test_sparse_s_kernel_fp32_elementwise(ctx, n_elec, n_pw, against):
    """The FP32 block-sparse S kernel of the mixed sweep (register-tiled
    sector products, FP32 reductions) element by element: against the
    oracle's printed terms on the 7- and 19-plane-wave gases, and against
    the FP64 block-sparse kernel on the 33-plane-wave gas, whose sectors of
    up to 66 pairs span two 48-wide tiles and two K chunks with a ragged
    tail.  Bound: 2e-6 of max |S| (FP32 rounding of sums over at most N^2
    terms of the rounded inputs)."""
    rs, beta, ng = 1.0, 1.5, 4
    sysc = bs.ueg(n_elec, rs, n_pw)
    t1c, t2c = bs.random_amplitudes(sysc["charges"], 17, 2, 0.05)
    d1, d2 = bs.dense_amplitudes(sysc["charges"], t1c, t2c)
    ctx.build_ueg(n_elec, rs, n_pw)
    mu = ctx.reference_mu(beta, float(n_elec))
    ctx.prepare(beta, mu, ng, precision="bf16x3", block_sparse=1)
    s1, s2 = ctx.eval_s(d1, d2, precision="bf16x3")
    if against == "oracle":
        prob = fc.Problem(systems.ueg(n_elec, rs, n_pw), beta, mu, ng, 0.0)
        r1, r2 = fc.S1(prob, d1, d2), fc.S2(prob, d1, d2)
    else:
        ctx.prepare(beta, mu, ng, precision="fp64", block_sparse=1)
        r1, r2 = ctx.eval_s(d1, d2)
        r1, r2 = r1.cpu(), r2.cpu()
    m1, m2 = torch.max(torch.abs(r1)).item(), torch.max(torch.abs(r2)).item()
    assert m2 > 1e-3
    e1 = torch.max(torch.abs(s1.cpu() - r1)).item()
    e2 = torch.max(torch.abs(s2.cpu() - r2)).item()
    assert e1 < 2e-6 * max(m1, m2), (e1, m1)
    assert e2 < 2e-6 * m2, (e2, m2)
    # and not exact: the FP32 path really ran
    assert e2 > 0.0


def test_sparse_s_kernel_matches_dense_gpu(ctx):
    """The same S evaluation through the dense FP64 engine: identical up to
    rounding order."""
    n_elec, rs, n_pw, beta, ng = 14, 1.0, 19, 2.0, 4
    sysc = bs.ueg(n_elec, rs, n_pw)
    t1c, t2c = bs.random_amplitudes(sysc["charges"], 3, 3, 0.05)
    d1, d2 = bs.dense_amplitudes(sysc["charges"], t1c, t2c)
    ctx.build_ueg(n_elec, rs, n_pw)
    mu = ctx.reference_mu(beta, float(n_elec))
    ctx.prepare(beta, mu, ng, precision="fp64", block_sparse=1)
    a1, a2 = ctx.eval_s(d1, d2)
    ctx.prepare(beta, mu, ng, precision="fp64")
    b1, b2 = ctx.eval_s(d1, d2)
    assert torch.max(torch.abs(a1 - b1)).item() < 1e-12 * max(1.0, torch.max(torch.abs(b1)).item())
    assert torch.max(torch.abs(a2 - b2)).item() < 1e-12 * max(1.0, torch.max(torch.abs(b2)).item())


@pytest.mark.parametrize("which", ["ueg7", "ueg19", "hubbard6", "hubbard10"])
def test_sparse_solve_matches_dense_and_oracle(ctx, which):
    """Converged Omega, its history and the amplitudes of the block-sparse
    solve against the dense FP64 GPU solve; Omega against the oracle."""
    if which.startswith("ueg"):
        n_pw = int(which[3:])
        n_elec, rs, beta, ng = (6 if n_pw == 7 else 14), 1.0, 2.0, 8
        sysd = systems.ueg(n_elec, rs, n_pw)
        build = lambda: ctx.build_ueg(n_elec, rs, n_pw)
        build()
        mu = ctx.reference_mu(beta, float(n_elec))
    else:
        L = int(which[7:])
        U, beta, ng = 2.0, 1.0, 8
        sysd = systems.hubbard_1d(L, 1.0, U)
        build = lambda: ctx.build_hubbard(L, 1.0, U)
        build()
        mu = U / 2.0
    rs_ = ctx.solve(beta, mu, ng, precision="fp64", block_sparse=1, tol_omega=1e-12, tol_amp=1e-10)
    s1s, s2s = ctx.amplitudes(ng, sysd["eps"].shape[0], sysd["eps"].shape[0])
    rd = ctx.solve(beta, mu, ng, precision="fp64", tol_omega=1e-12, tol_amp=1e-10)
    s1d, s2d = ctx.amplitudes(ng, sysd["eps"].shape[0], sysd["eps"].shape[0])
    assert rs_["converged"] and rd["converged"]
    assert rs_["iterations"] == rd["iterations"]
    assert abs(rs_["omega"] - rd["omega"]) < 1e-11, (rs_["omega"], rd["omega"])
    assert np.max(np.abs(s1s - s1d)) < 1e-11
    assert np.max(np.abs(s2s - s2d)) < 1e-11
    if which in ("ueg7", "hubbard6"):
        prob = fc.Problem(sysd, beta, mu, ng, 0.0)
        ref = fc.solve(prob, tol=1e-13, tol_amp=1e-11)
        assert abs(rs_["omega_cc"] - float(ref["omega_cc"])) < 1e-10


@pytest.mark.parametrize("name,tau_chunk", [("oracle_ueg57.json", 0), ("oracle_ueg57.json", 8),
                                            ("oracle_ueg81.json", 0)])
def test_sparse_converged_gases_match_goldens(ctx, name, tau_chunk):
    """The 114- and 162-spin-orbital gases solved in FP64 with the
    block-sparse storage against the block-sparse oracle's converged Omega
    (the oracle converged to |dOmega_CC| < 1e-11; the two run the same
    Jacobi fixed point, so the iteration counts agree too)."""
    gold = json.load(open(os.path.join(GOLD, name)))
    c = gold["config"]
    ctx.build_ueg(c["n_elec"], c["rs"], c["n_pw"])
    mu = ctx.reference_mu(c["beta"], float(c["n_elec"]))
    assert abs(mu - gold["mu"]) < 1e-10
    r = ctx.solve(c["beta"], gold["mu"], c["ngrid"], precision="fp64", block_sparse=1, tau_chunk=tau_chunk,
                  tol_omega=1e-11, tol_amp=1e-9, max_iter=80)
    assert r["converged"] and (r["n_occ"], r["n_vir"]) == (gold["n_orbitals"], gold["n_orbitals"])
    assert abs(r["omega0"] - gold["omega0"]) < 1e-10
    assert abs(r["omega1"] - gold["omega1"]) < 1e-10
    assert abs(r["omega"] - gold["omega"]) < 1e-9, (r["omega"], gold["omega"])


@pytest.mark.parametrize("name", ["oracle_ueg57.json", "oracle_ueg81.json"])
def test_sparse_mixed_precision_gases(ctx, name):
    """The mixed pipeline on the block-sparse storage: FP32 sweep (storage
    and SIMT sector products, FP64 propagator factors and energy sums)
    alone, then followed by FP64 residual corrections, against the
    block-sparse oracle's converged Omega; the FP32 phase within 1e-6 Ha,
    the corrected solve within 1e-8 Ha."""
    gold = json.load(open(os.path.join(GOLD, name)))
    c = gold["config"]
    ctx.build_ueg(c["n_elec"], c["rs"], c["n_pw"])
    kw = dict(precision="bf16x3", block_sparse=1, trunc_thr=c["thr"], max_iter=80)
    r = ctx.solve(c["beta"], gold["mu"], c["ngrid"], refine_max_iter=0, **kw)
    assert r["converged"] and r["refine_iterations"] == 0
    assert abs(r["omega"] - gold["omega"]) < 1e-6, (r["omega"], gold["omega"])
    r = ctx.solve(c["beta"], gold["mu"], c["ngrid"], refine_max_iter=3, tol_omega=1e-10, tol_amp=1e-8, **kw)
    assert r["converged"] and 1 <= r["refine_iterations"] <= 3
    assert abs(r["omega"] - gold["omega"]) < 1e-8, (r["omega"], gold["omega"])


def test_sparse_argument_checks(ctx):
    from paper_2004_01729_gb300 import ftcc
    ctx.build_ueg(6, 1.0, 7)
    ctx.prepare(1.0, 0.5, 4, precision="tf32", block_sparse=1)
    with pytest.raises(ftcc.FTCCError) as e:          # more slices than the grid holds
        ctx.eval_s(torch.zeros((5, 14, 14), dtype=torch.float64), torch.zeros((5, 14, 14, 14, 14), dtype=torch.float64),
                   precision="tf32")
    assert e.value.status == ftcc.ERR_INVALID_ARG
    with pytest.raises(ftcc.FTCCError) as e:          # Simpson integral form only
        ctx.solve(1.0, 0.5, 5, quad=ftcc.QUAD_RK4, precision="fp64", block_sparse=1)
    assert e.value.status == ftcc.ERR_UNSUPPORTED
    r = ctx.solve(1.0, 0.5, 6, precision="fp64", block_sparse=1)
    assert r["converged"]
    with pytest.raises(ftcc.FTCCError) as e:          # dense layouts only
        ctx.propagate_adjoint("ia", torch.zeros((6, 14, 14), dtype=torch.float64))
    assert e.value.status == ftcc.ERR_UNSUPPORTED
    rng = np.random.default_rng(0)
    N = 6
    h = np.diag(rng.standard_normal(N))
    eri = np.zeros((N, N, N, N))
    ctx.build_generic(h, eri, np.diag(h).copy())       # no conserved charges
    with pytest.raises(ftcc.FTCCError) as e:
        ctx.prepare(1.0, 0.0, 4, precision="fp64", block_sparse=1)
    assert e.value.status == ftcc.ERR_INVALID_ARG
    ctx.build_hubbard(4, 1.0, 2.0, reference="neel")   # site basis: no conserved momentum
    with pytest.raises(ftcc.FTCCError) as e:
        ctx.prepare(1.0, 1.0, 4, precision="fp64", block_sparse=1)
    assert e.value.status == ftcc.ERR_INVALID_ARG


def test_generic_system_with_charges(ctx):
    """A GENERIC system built from the gas's host Hamiltonian with its orbital
    charges (ftcc_get_charges) solves with block_sparse to the same Omega as
    the built-in gas; a non-unique charge set is refused."""
    from paper_2004_01729_gb300 import ftcc
    n_elec, rs, n_pw, beta, ng = 14, 1.0, 19, 2.0, 8
    ctx.build_ueg(n_elec, rs, n_pw)
    mu = ctx.reference_mu(beta, float(n_elec))
    ref = ctx.solve(beta, mu, ng, precision="fp64", block_sparse=1)
    h, eri, eps = ctx.get_system()
    ch, md = ctx.get_charges()
    assert ch.shape == (2 * n_pw, 4) and len({tuple(r) for r in ch}) == 2 * n_pw
    ctx.build_generic(h, eri, eps, ch, md)
    r = ctx.solve(beta, mu, ng, precision="fp64", block_sparse=1)
    assert abs(r["omega"] - ref["omega"]) < 1e-12
    ch2 = ch.copy()
    ch2[1] = ch2[0]
    ctx.build_generic(h, eri, eps, ch2, md)
    with pytest.raises(ftcc.FTCCError) as e:
        ctx.prepare(beta, mu, ng, precision="fp64", block_sparse=1)
    assert e.value.status == ftcc.ERR_INVALID_ARG
    ctx.build_generic(h, eri, eps)
    with pytest.raises(ftcc.FTCCError):
        ctx.get_charges()


def _conserving_antisym(ch, t1, t2):
    """Orthogonal projection of dense s1 [x,i,a] / s2 [x,i,j,a,b] onto the
    charge-conserving (s1 diagonal, q_i + q_j = q_a + q_b), antisymmetric
    elements."""
    q = np.asarray(ch.q)
    N = q.shape[0]
    keep1 = torch.eye(N, dtype=torch.float64)
    tot = q[:, None, :] + q[None, :, :]
    keep2 = torch.from_numpy(np.all(tot[:, :, None, None, :] == tot[None, None, :, :, :], axis=-1).astype(np.float64))
    a2 = 0.25 * (t2 - t2.transpose(1, 2) - t2.transpose(3, 4) + t2.transpose(1, 2).transpose(3, 4))
    return t1 * keep1, a2 * keep2


def test_sparse_vjp_matches_dense_gpu(ctx):
    """The transpose of the block-sparse S kernel against the dense engine's
    tape-replayed transpose on the conserving antisymmetric subspace
    (19-plane-wave gas, random amplitudes and cotangents), element by
    element."""
    n_elec, rs, n_pw, beta, ng = 14, 1.0, 19, 2.0, 4
    sysc = bs.ueg(n_elec, rs, n_pw)
    ch = sysc["charges"]
    t1c, t2c = bs.random_amplitudes(ch, 5, 2, 0.05)
    d1, d2 = bs.dense_amplitudes(ch, t1c, t2c)
    rng = np.random.default_rng(9)
    w1 = torch.tensor(rng.standard_normal(tuple(d1.shape)))
    w2 = torch.tensor(rng.standard_normal(tuple(d2.shape)))
    w1, w2 = _conserving_antisym(ch, w1, w2)
    ctx.build_ueg(n_elec, rs, n_pw)
    mu = ctx.reference_mu(beta, float(n_elec))
    ctx.prepare(beta, mu, ng, precision="fp64", block_sparse=1)
    a1, a2 = ctx.eval_s_vjp(d1, d2, w1, w2)
    ctx.prepare(beta, mu, ng, precision="fp64")
    b1, b2 = ctx.eval_s_vjp(d1, d2, w1, w2)
    a1, a2 = _conserving_antisym(ch, a1.cpu(), a2.cpu())
    b1, b2 = _conserving_antisym(ch, b1.cpu(), b2.cpu())
    s1 = torch.max(torch.abs(b1)).item()
    s2 = torch.max(torch.abs(b2)).item()
    assert s2 > 1e-3
    assert torch.max(torch.abs(a1 - b1)).item() < 1e-11 * max(1.0, s1)
    assert torch.max(torch.abs(a2 - b2)).item() < 1e-11 * max(1.0, s2)


@pytest.mark.parametrize("which", ["ueg19", "hubbard6"])
def test_sparse_adjoint_matches_dense(ctx, which):
    """N, E, S, the 1-RDM and Gamma_N from the block-sparse lambda sweep
    against the dense FP64 adjoint of the same converged solve."""
    if which == "ueg19":
        beta, ng = 2.0, 8
        ctx.build_ueg(14, 1.0, 19)
        mu = ctx.reference_mu(beta, 14.0)
    else:
        beta, ng, mu = 1.0, 8, 1.0
        ctx.build_hubbard(6, 1.0, 2.0)
    kw = dict(precision="fp64", tol_omega=1e-12, tol_amp=1e-10)
    ctx.solve(beta, mu, ng, block_sparse=1, **kw)
    ds, rs_ = ctx.adjoint(with_rdm1=True)
    gs = ctx.rdm2()
    ctx.solve(beta, mu, ng, **kw)
    dd, rd = ctx.adjoint(with_rdm1=True)
    gd = ctx.rdm2()
    for k in ("dOmega_dmu", "dOmega_dbeta", "N", "E", "S"):
        assert abs(ds[k] - dd[k]) < 1e-9 * max(1.0, abs(dd[k])), (k, ds[k], dd[k])
    assert np.max(np.abs(rs_ - rd)) < 1e-9
    assert np.max(np.abs(gs - gd)) < 1e-9 * max(1.0, np.max(np.abs(gd)))


def test_sparse_adjoint_ueg57_matches_oracle_differences(ctx):
    """N, E and S of the 114-spin-orbital gas from the block-sparse FP64
    lambda sweep against central differences (one Richardson step) of
    converged block-sparse oracle solves."""
    gold = json.load(open(os.path.join(GOLD, "oracle_ueg57.json")))
    gr = json.load(open(os.path.join(GOLD, "oracle_ueg57_response.json")))
    c = gold["config"]
    ctx.build_ueg(c["n_elec"], c["rs"], c["n_pw"])
    r = ctx.solve(c["beta"], gold["mu"], c["ngrid"], precision="fp64", block_sparse=1, tol_omega=1e-12,
                  tol_amp=1e-10)
    assert r["converged"]
    d, rdm = ctx.adjoint(with_rdm1=True)
    assert abs(d["N"] - gr["N"]) < 2e-7, (d["N"], gr["N"])
    assert abs(d["E"] - gr["E"]) < 2e-6, (d["E"], gr["E"])
    assert abs(d["S"] - gr["S"]) < 2e-6, (d["S"], gr["S"])
    assert abs(np.trace(rdm) - d["N"]) < 1e-8
    assert np.max(np.abs(rdm - np.diag(np.diag(rdm)))) == 0.0   # momentum conservation: diagonal


def test_sparse_adjoint_ueg81_matches_central_differences(ctx):
    """The 162-spin-orbital gas: dOmega/dmu and dOmega/dbeta from the
    block-sparse lambda sweep against central differences (one Richardson
    step, h = 1e-3) of converged block-sparse solves of the same gas."""
    gold = json.load(open(os.path.join(GOLD, "oracle_ueg81.json")))
    c = gold["config"]
    ctx.build_ueg(c["n_elec"], c["rs"], c["n_pw"])
    mu, beta, ng = gold["mu"], c["beta"], c["ngrid"]
    kw = dict(precision="fp64", block_sparse=1, trunc_thr=c["thr"], tol_omega=1e-13, tol_amp=1e-11, max_iter=100)
    r = ctx.solve(beta, mu, ng, **kw)
    assert r["converged"] and abs(r["omega"] - gold["omega"]) < 1e-9
    d, _ = ctx.adjoint(with_rdm1=False)

    def om(b, m):
        x = ctx.solve(b, m, ng, **kw)
        assert x["converged"]
        return x["omega"]

    def rich(f, h):
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
        return (4 * d1 - d2) / 3

    h = 1e-3
    dmu = rich(lambda e: om(beta, mu + e), h)
    dbeta = rich(lambda e: om(beta + e, mu), h)
    assert abs(d["dOmega_dmu"] - dmu) < 1e-7 * max(1.0, abs(dmu)), (d["dOmega_dmu"], dmu)
    assert abs(d["dOmega_dbeta"] - dbeta) < 1e-7 * max(1.0, abs(dbeta)), (d["dOmega_dbeta"], dbeta)
