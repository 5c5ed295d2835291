"""Adjoint (lambda) pieces on the GPU against the oracle: the S-kernel
vector-Jacobian product, the transposed propagation, and the converged
multipliers of the discrete Lagrangian (Eqs. Lagrangian, lmu, ltilde)."""
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


def _system(which):
    if which == "hubbard6":
        return systems.hubbard_1d(6, 1.0, 2.0), dict(kind="h", L=6, U=2.0), 1.0, 1.0, 0.0
    h, eri, eps = wl.random_generic_system(21, 7, v_scale=0.04)
    return (systems.generic(torch.tensor(h), torch.tensor(eri), torch.tensor(eps)),
            dict(kind="g", h=h, eri=eri, eps=eps), 2.5, -0.1, 0.05)


def _build(ctx, spec):
    if spec["kind"] == "h":
        ctx.build_hubbard(spec["L"], 1.0, spec["U"])
    else:
        ctx.build_generic(spec["h"], spec["eri"], spec["eps"])


def _rel(a, b):
    a = torch.as_tensor(a).double().cpu()
    b = torch.as_tensor(b).double().cpu()
    return (torch.max(torch.abs(a - b)) / torch.max(torch.abs(b))).item()


def _asym(t):
    """Projection onto amplitudes antisymmetric in (i, j) and in (a, b)."""
    t = t - t.transpose(1, 2)
    return 0.25 * (t - t.transpose(3, 4))


@pytest.mark.parametrize("which", ["hubbard6", "generic7_truncated"])
def test_s_kernel_vjp_matches_reverse_mode(ctx, which):
    """The factorised GPU schedule and the paper's terms are the same function
    only on antisymmetric doubles, so their gradients agree after projecting
    the doubles part onto that subspace; directional derivatives along
    admissible directions are also checked against central differences of
    the GPU S kernel itself."""
    sysd, spec, beta, mu, thr = _system(which)
    ng, nx = 6, 4
    _build(ctx, spec)
    ctx.prepare(beta, mu, ng, precision="fp64", trunc_thr=thr)
    prob = fc.Problem(sysd, beta, mu, ng, thr)
    no, nv = len(prob.iO), len(prob.iV)
    t1, t2 = [torch.tensor(a) for a in wl.random_amplitudes(8, nx, no, nv, 0.3)]
    w1, w2 = [torch.tensor(a) for a in wl.random_amplitudes(9, nx, no, nv, 1.0)]
    g1, g2 = ctx.eval_s_vjp(t1, t2, w1, w2)
    g1, g2 = g1.cpu(), g2.cpu()
    a1 = t1.clone().requires_grad_(True)
    a2 = t2.clone().requires_grad_(True)
    r1, r2 = torch.autograd.grad((fc.S1(prob, a1, a2), fc.S2(prob, a1, a2)), (a1, a2), grad_outputs=(w1, w2))
    v1, v2 = [torch.tensor(a) for a in wl.random_amplitudes(10, nx, no, nv, 1.0)]
    dir_gpu = (torch.sum(g1 * v1) + torch.sum(g2 * v2)).item()
    dir_ora = (torch.sum(r1 * v1) + torch.sum(r2 * v2)).item()
    eps = 1e-4
    sp = ctx.eval_s(t1 + eps * v1, t2 + eps * v2)
    sm = ctx.eval_s(t1 - eps * v1, t2 - eps * v2)
    fd = sum(torch.sum(w * (p.cpu() - m.cpu())).item() for w, p, m in zip((w1, w2), sp, sm)) / (2 * eps)
    assert abs(dir_gpu - dir_ora) < 1e-10 * max(1.0, abs(dir_ora)), (dir_gpu, dir_ora)
    assert abs(dir_gpu - fd) < 1e-6 * max(1.0, abs(fd)), (dir_gpu, fd)
    assert _rel(g1, r1) < 1e-11
    assert _rel(_asym(g2), _asym(r2)) < 1e-11


@pytest.mark.parametrize("slots", ["ia", "ijab"])
def test_transposed_propagation(ctx, slots):
    sysd, spec, beta, mu, thr = _system("generic7_truncated")
    ng = 11
    _build(ctx, spec)
    ctx.prepare(beta, mu, ng, trunc_thr=thr)
    prob = fc.Problem(sysd, beta, mu, ng, thr)
    no, nv = len(prob.iO), len(prob.iV)
    shape = (ng, no, nv) if slots == "ia" else (ng, no, no, nv, nv)
    rng = np.random.default_rng(2)
    m = torch.tensor(rng.standard_normal(shape))
    S = torch.zeros(shape, dtype=torch.float64, requires_grad=True)
    out = fc.propagate(prob, S, prob.D1 if slots == "ia" else prob.D2)      # = -sum_x G e S
    (ref,) = torch.autograd.grad(out, S, grad_outputs=m)
    got = ctx.propagate_adjoint(slots, m).cpu()
    assert _rel(got, -ref) < 1e-12


@pytest.mark.parametrize("which", ["hubbard6", "generic7_truncated"])
def test_lambda_matches_oracle(ctx, which):
    sysd, spec, beta, mu, thr = _system(which)
    ng = 8
    _build(ctx, spec)
    r = ctx.solve(beta, mu, ng, precision="fp64", trunc_thr=thr, tol_omega=1e-13, tol_amp=1e-11)
    assert r["converged"]
    d, _ = ctx.adjoint(allow_unsupported=True)
    assert d["iterations"] > 0
    prob = fc.Problem(sysd, beta, mu, ng, thr)
    sol = fc.solve(prob, tol=1e-13, tol_amp=1e-11)
    lam = fc.lambda_solve(prob, sol["t1"], sol["t2"], tol=1e-12)
    no, nv = len(prob.iO), len(prob.iV)
    m1, m2 = ctx.get_lambda(ng, no, nv)
    # the multipliers are fixed on the antisymmetric subspace (see above)
    assert _rel(m1, lam["m1"]) < 1e-8
    assert _rel(_asym(torch.tensor(m2)), _asym(lam["m2"])) < 1e-8


@pytest.mark.parametrize("which", ["hubbard6", "generic7_truncated"])
def test_response_matches_oracle(ctx, which):
    """dOmega/dmu, dOmega/dbeta, N, E, S and the partially relaxed 1-RDM from
    the GPU adjoint against the oracle's derivatives of the same discrete
    Lagrangian (App. B; both are exact for the discrete scheme)."""
    sysd, spec, beta, mu, thr = _system(which)
    ng = 8
    _build(ctx, spec)
    r = ctx.solve(beta, mu, ng, precision="fp64", trunc_thr=thr, tol_omega=1e-13, tol_amp=1e-11)
    assert r["converged"]
    d, rdm = ctx.adjoint()
    ref = fc.response(sysd, beta, mu, ng, thr, solve_kw=dict(tol=1e-13, tol_amp=1e-11))
    for k in ("dOmega_dmu", "dOmega_dbeta", "N", "E", "S"):
        assert abs(d[k] - ref[k]) < 1e-8 * max(1.0, abs(ref[k])), (k, d[k], ref[k])
    assert np.max(np.abs(rdm - ref["rdm1"].numpy())) < 1e-8
    assert abs(d["trace_rdm1"] - d["N"]) < 1e-9


def test_response_after_mixed_solve(ctx):
    """A TF32 solve is refined in FP64 before the adjoint; the response equals
    the FP64 one."""
    sysd, spec, beta, mu, thr = _system("hubbard6")
    ng = 8
    _build(ctx, spec)
    ctx.solve(beta, mu, ng, precision="tf32", refine_max_iter=30)
    d, rdm = ctx.adjoint()
    ref = fc.response(sysd, beta, mu, ng, thr, solve_kw=dict(tol=1e-13, tol_amp=1e-11))
    assert abs(d["dOmega_dbeta"] - ref["dOmega_dbeta"]) < 1e-7
    assert abs(d["N"] - ref["N"]) < 1e-7


def test_batched_adjoint_equals_single_instances():
    """ft_ccsd_adjoint on the members of a batched solve: the lambda sweep
    runs over the whole batch at once and every member gets the response of
    its own single-instance solve (dOmega/dmu, dOmega/dbeta, E, S, 1-RDM)."""
    from paper_2004_01729_gb300 import ftcc
    L, U, ng = 6, 2.0, 12
    betas, mus = [0.7, 1.0, 1.6], [1.0, 0.8, 1.2]
    ctxs = []
    for _ in betas:
        c = ftcc.Context(0)
        c.build_hubbard(L, 1.0, U)
        ctxs.append(c)
    res = ftcc.solve_batched(ctxs, betas, mus, ng, precision="fp64", tol_omega=1e-12, tol_amp=1e-10)
    assert all(r["converged"] for r in res)
    got = [c.adjoint(with_rdm1=True) for c in ctxs]
    one = ftcc.Context(0)
    one.build_hubbard(L, 1.0, U)
    for (d, rdm), b, m in zip(got, betas, mus):
        one.solve(b, m, ng, precision="fp64", tol_omega=1e-12, tol_amp=1e-10)
        e, erdm = one.adjoint(with_rdm1=True)
        for k in ("dOmega_dmu", "dOmega_dbeta", "N", "E", "S"):
            assert abs(d[k] - e[k]) < 1e-9, (k, d[k], e[k])
        assert np.max(np.abs(rdm - erdm)) < 1e-9
    for c in ctxs + [one]:
        c.close()


def test_autograd_omega_matches_adjoint_and_differences():
    """ftcc.omega: Omega as a torch function whose backward is the GPU lambda
    sweep; its beta, mu and one-body gradients agree with ft_ccsd_adjoint and
    with central differences of GPU solves."""
    from paper_2004_01729_gb300 import ftcc
    c = ftcc.Context(0)
    c.build_hubbard(6, 1.0, 2.0)
    N = c.num_orbitals()
    kw = dict(precision="fp64", tol_omega=1e-13, tol_amp=1e-11)
    beta = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(0.9, dtype=torch.float64, requires_grad=True)
    V = torch.zeros((N, N), dtype=torch.float64, requires_grad=True)
    om = ftcc.omega(c, beta, mu, 12, V=V, **kw)
    om.backward()
    d, rdm = c.adjoint(with_rdm1=True)
    assert abs(beta.grad.item() - d["dOmega_dbeta"]) < 1e-12
    assert abs(mu.grad.item() + d["N"]) < 1e-12
    assert np.max(np.abs(V.grad.numpy() - rdm.T)) < 1e-12
    step = 1e-4
    fd_b = (ftcc.omega(c, 1.0 + step, 0.9, 12, V=V.detach(), **kw).item()
            - ftcc.omega(c, 1.0 - step, 0.9, 12, V=V.detach(), **kw).item()) / (2 * step)
    assert abs(fd_b - beta.grad.item()) < 1e-6
    dv = torch.zeros((N, N), dtype=torch.float64)
    dv[0, 1] = dv[1, 0] = step          # a symmetric off-diagonal one-body change
    fd_v = (ftcc.omega(c, 1.0, 0.9, 12, V=dv, **kw).item() - ftcc.omega(c, 1.0, 0.9, 12, V=-dv, **kw).item()) / (2 * step)
    assert abs(fd_v - (V.grad[0, 1] + V.grad[1, 0]).item()) < 1e-6
    c.close()


def test_adjoint_of_live_members_beside_a_diverged_one():
    """In a batch where one member diverges from s = 0 (and is frozen), the
    other members still get their adjoint, equal to their single-instance
    response; the diverged member's call is refused."""
    from paper_2004_01729_gb300 import ftcc
    cb = wl.hubbard_batch()
    bad = cb[43]                          # 6 sites, U = 7.7, beta = 2.8: diverges from s = 0
    good = next(q for q in cb if q["L"] == bad["L"] and q is not bad)
    pair = [bad, good]
    ctxs = []
    for q in pair:
        c = ftcc.Context(0)
        c.build_hubbard(q["L"], q["t"], q["U"])
        ctxs.append(c)
    kw = dict(precision="tf32", refine_max_iter=30, max_iter=400)
    res = ftcc.solve_batched(ctxs, [q["beta"] for q in pair], [q["mu"] for q in pair], bad["ngrid"],
                             allow_unconverged=True, **kw)
    assert not res[0]["converged"] and res[1]["converged"]
    d, rdm = ctxs[1].adjoint(with_rdm1=True)
    with pytest.raises(ftcc.FTCCError):
        ctxs[0].adjoint(with_rdm1=False)
    one = ftcc.Context(0)
    one.build_hubbard(good["L"], good["t"], good["U"])
    one.solve(good["beta"], good["mu"], good["ngrid"], **kw)
    e, erdm = one.adjoint(with_rdm1=True)
    for k in ("dOmega_dmu", "dOmega_dbeta", "E", "S"):
        assert abs(d[k] - e[k]) < 1e-8, (k, d[k], e[k])
    assert np.max(np.abs(rdm - erdm)) < 1e-8
    for c in ctxs + [one]:
        c.close()


@pytest.mark.parametrize("k", [0, 1, 2])
def test_response_matches_golden_hubbard10(ctx, k):
    """N, E, S and dOmega/dbeta of the three 10-site temperatures (FP64 solve,
    GPU lambda sweep) against the oracle's golden values."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "oracle_hubbard10.json")))[k]
    c = wl.HUBBARD_10[k]
    ctx.build_hubbard(c["L"], c["t"], c["U"])
    r = ctx.solve(c["beta"], c["mu"], c["ngrid"], precision="fp64", tol_omega=1e-12, tol_amp=1e-10)
    assert r["converged"]
    d, rdm = ctx.adjoint(with_rdm1=True)
    for key in ("dOmega_dmu", "dOmega_dbeta", "N", "E", "S"):
        assert abs(d[key] - gold[key]) < 1e-8, (key, d[key], gold[key])
    assert np.max(np.abs(np.diag(rdm) - np.array(gold["rdm1_diag"]))) < 1e-8


@pytest.mark.parametrize("k", [0, 1, 2])
def test_mixed_adjoint_hubbard10(ctx, k):
    """The lambda sweep and the response in the mixed arithmetic (FP32
    multipliers, BF16X3 contractions, FP64 propagator factors and sums) after
    a BF16X3 solve without FP64 iterations: N, E and S of the three 10-site
    temperatures against the oracle's golden values."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "oracle_hubbard10.json")))[k]
    c = wl.HUBBARD_10[k]
    ctx.build_hubbard(c["L"], c["t"], c["U"])
    r = ctx.solve(c["beta"], c["mu"], c["ngrid"], precision="bf16x3", refine_max_iter=0, mixed_adjoint=1)
    assert r["converged"] and r["refine_iterations"] == 0
    d, rdm = ctx.adjoint(with_rdm1=True)
    for key in ("N", "E", "S"):
        assert abs(d[key] - gold[key]) < 2e-5 * max(1.0, abs(gold[key])), (key, d[key], gold[key])
    assert np.max(np.abs(np.diag(rdm) - np.array(gold["rdm1_diag"]))) < 2e-5
    from paper_2004_01729_gb300 import ftcc
    with pytest.raises(ftcc.FTCCError) as e:
        ctx.rdm2()
    assert e.value.status == ftcc.ERR_UNSUPPORTED
