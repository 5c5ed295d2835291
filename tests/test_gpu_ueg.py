"""Full-size parity for the warm dense electron gas workloads (114 and 162
spin orbitals): the GPU S kernel on seeded random amplitudes against the
oracle's Eqs. ccS1/ccS2 evaluated on a sampled block of output indices
(every summation over the full orbital range)."""
import numpy as np
import pytest
import torch

from oracle import ftccsd as fc, systems
from paper_2004_01729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# relative to the largest sampled |S|; sums run over up to N^2 = 26244 terms,
# so the bf16 hi/lo split (~2^-16 per product) is allowed a few 1e-4
TOL = {"fp64": 1e-11, "tf32": 5e-3, "bf16x3": 5e-4}


def _mu0(eps, beta, n_elec):
    lo, hi = float(eps.min()) - 60.0 / beta, float(eps.max()) + 60.0 / beta
    for _ in range(200):
        m = 0.5 * (lo + hi)
        n, _ = fc.occupations(eps, beta, m)
        if n.sum().item() < n_elec:
            lo = m
        else:
            hi = m
    return 0.5 * (lo + hi)


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_01729_gb300 import ftcc
    c = ftcc.Context(0)
    yield c
    c.close()


CASES = [("ueg57", wl.UEG_57, "fp64"), ("ueg57", wl.UEG_57, "tf32"), ("ueg57", wl.UEG_57, "bf16x3"),
         ("ueg81", wl.UEG_81, "tf32"), ("ueg81", wl.UEG_81, "bf16x3")]


@pytest.mark.parametrize("name,cfg,prec", CASES, ids=[f"{a}-{c}" for a, _, c in CASES])
def test_ueg_s_kernel_sampled(ctx, name, cfg, prec):
    sysd = systems.ueg(cfg["n_elec"], cfg["rs"], cfg["n_pw"])
    beta = cfg["beta"]
    ctx.build_ueg(cfg["n_elec"], cfg["rs"], cfg["n_pw"])
    mu = ctx.reference_mu(beta, float(cfg["n_elec"]))
    assert abs(mu - _mu0(sysd["eps"], beta, cfg["n_elec"])) < 1e-10
    ng = 4   # the S kernel is local in tau: a short grid keeps the amplitude buffers small
    info = ctx.prepare(beta, mu, ng, precision=prec, trunc_thr=cfg["thr"], tau_chunk=1)
    prob = fc.Problem(sysd, beta, mu, ng, cfg["thr"])
    no, nv = len(prob.iO), len(prob.iV)
    assert (info["n_occ"], info["n_vir"]) == (no, nv)
    t1, t2 = wl.random_amplitudes(17, 1, no, nv, 0.05)
    t1, t2 = torch.tensor(t1), torch.tensor(t2)
    s1, s2 = ctx.eval_s(t1, t2, precision=prec)
    rng = np.random.default_rng(5)
    io = torch.tensor(sorted(rng.choice(no, 4, replace=False)))
    iv = torch.tensor(sorted(rng.choice(nv, 4, replace=False)))
    # only the output letters are restricted; every summed index runs in full
    r1 = fc.S1(prob, t1, t2, sel={"i": io, "a": iv})
    r2 = fc.S2(prob, t1, t2, sel={"i": io, "j": io, "a": iv, "b": iv})
    g1 = s1.cpu()[:, io][:, :, iv]
    g2 = s2.cpu()[:, io][:, :, io][:, :, :, iv][:, :, :, :, iv]
    e1 = (torch.max(torch.abs(g1 - r1)) / torch.max(torch.abs(r1))).item()
    e2 = (torch.max(torch.abs(g2 - r2)) / torch.max(torch.abs(r2))).item()
    assert e1 < TOL[prec], e1
    assert e2 < TOL[prec], e2
