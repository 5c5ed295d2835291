"""Write the oracle's converged grand potentials of the plane-wave gases
(114 and 162 spin orbitals) with the momentum/spin block-sparse execution of
the oracle (``oracle/blocksparse.py``).

Calls only ``oracle/`` (plus the seeded parameters in workloads.py); the GPU
path never contributes to these files.  Run from the repository root:
    python tests/golden/make_golden_ueg.py ueg57      # about half an hour on 8 cores
    python tests/golden/make_golden_ueg.py ueg81      # a few hours
    python tests/golden/make_golden_ueg.py ueg57_response   # N, E, S by central differences
Each run writes tests/golden/oracle_<name>.json with mu (the reference mu_0
of the gas at 14 electrons, App. D), Omega, its parts and the Omega_CC
history of the fixed point; the *_response runs write
tests/golden/oracle_<name>_response.json with dOmega/dmu, dOmega/dbeta, N, E
and S.
"""
import json
import os
import sys
import time

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import blocksparse as bs, chemical_potential as cp  # noqa: E402
from paper_2004_01729_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden")


def run(name, cfg):
    t0 = time.time()
    sysc = bs.ueg(cfg["n_elec"], cfg["rs"], cfg["n_pw"])
    mu = cp.mu_reference(sysc["eps"], cfg["beta"], float(cfg["n_elec"]))
    prob = bs.Problem(sysc, cfg["beta"], mu, cfg["ngrid"], cfg["thr"])
    sol = bs.solve(prob, tol=1e-11, tol_amp=1e-9, max_iter=200, verbose=True)
    out = dict(config=cfg, mu=mu, omega=sol["omega"], omega0=sol["omega0"], omega1=sol["omega1"],
               omega_cc=sol["omega_cc"], iterations=sol["iterations"], converged=sol["converged"],
               history=sol["history"], n_orbitals=prob.ch.N, seconds=time.time() - t0,
               threads=torch.get_num_threads())
    with open(os.path.join(OUT, f"oracle_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "history"}), flush=True)


def response(name, cfg, hmu=2e-3, hbeta=2e-3):
    """N = -dOmega/dmu and dOmega/dbeta (hence E = Omega + beta dOmega/dbeta
    + mu N, S = beta^2 dOmega/dbeta) of the converged discrete scheme by
    central differences with one Richardson step (steps h and 2h), at the
    reference mu_0; each displaced solve starts from the converged amplitudes
    of the undisplaced one and converges to |dOmega_CC| < 1e-12."""
    t0 = time.time()
    sysc = bs.ueg(cfg["n_elec"], cfg["rs"], cfg["n_pw"])
    mu = cp.mu_reference(sysc["eps"], cfg["beta"], float(cfg["n_elec"]))
    beta = cfg["beta"]
    kw = dict(tol=1e-12, tol_amp=1e-10, max_iter=200)
    base = bs.solve(bs.Problem(sysc, beta, mu, cfg["ngrid"], cfg["thr"]), **kw)

    def omega(b, m):
        r = bs.solve(bs.Problem(sysc, b, m, cfg["ngrid"], cfg["thr"]), t1=base["t1"], t2=base["t2"], **kw)
        assert r["converged"]
        print(json.dumps({"beta": b, "mu": m, "omega": r["omega"], "iterations": r["iterations"]}), flush=True)
        return r["omega"]

    def deriv(f, h):
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
        return (4 * d1 - d2) / 3

    dmu = deriv(lambda d: omega(beta, mu + d), hmu)
    dbeta = deriv(lambda d: omega(beta + d, mu), hbeta)
    om = base["omega"]
    n = -dmu
    out = dict(config=cfg, mu=mu, omega=om, dOmega_dmu=dmu, dOmega_dbeta=dbeta, N=n, E=om + beta * dbeta + mu * n,
               S=beta * beta * dbeta, steps={"mu": hmu, "beta": hbeta},
               how="central differences of converged block-sparse oracle solves, one Richardson step",
               seconds=time.time() - t0, threads=torch.get_num_threads())
    with open(os.path.join(OUT, f"oracle_{name}_response.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    which = sys.argv[1:] or ["ueg57"]
    if "ueg57" in which:
        run("ueg57", wl.UEG_57)
    if "ueg81" in which:
        run("ueg81", wl.UEG_81)
    if "ueg57_response" in which:
        response("ueg57", wl.UEG_57)
    if "ueg81_response" in which:
        response("ueg81", wl.UEG_81)
