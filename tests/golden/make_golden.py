"""Write the oracle's converged values for the Hubbard workloads.

Calls only ``oracle/`` (plus the seeded parameters in workloads.py); the GPU
path never contributes to these files.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ftccsd as fc, systems  # noqa: E402
from paper_2004_01729_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden")


def run(cfg, with_response):
    s = systems.hubbard_1d(cfg["L"], cfg["t"], cfg["U"])
    t0 = time.time()
    kw = dict(tol=1e-13, tol_amp=1e-11, max_iter=1000)
    if with_response:
        r = fc.response(s, cfg["beta"], cfg["mu"], cfg["ngrid"], solve_kw=kw)
        sol = r["solve"]
        extra = {k: r[k] for k in ("dOmega_dmu", "dOmega_dbeta", "N", "E", "S")}
        extra["rdm1_diag"] = [float(v) for v in r["rdm1"].diagonal()]
    else:
        sol = fc.solve(fc.Problem(s, cfg["beta"], cfg["mu"], cfg["ngrid"]), **kw)
        extra = {}
    out = dict(config=cfg, omega=sol["omega"], omega0=sol["omega0"], omega1=sol["omega1"],
               omega_cc=sol["omega_cc"], iterations=sol["iterations"],
               converged=sol["converged"], seconds=time.time() - t0, **extra)
    print(json.dumps({k: v for k, v in out.items() if k != "rdm1_diag"}), flush=True)
    return out


if __name__ == "__main__":
    which = sys.argv[1:] or ["hubbard6", "hubbard10"]
    if "hubbard6" in which:
        res = run(wl.HUBBARD_6, True)
        with open(os.path.join(OUT, "oracle_hubbard6.json"), "w") as f:
            json.dump(res, f, indent=1)
    if "hubbard10" in which:
        res = [run(c, True) for c in wl.HUBBARD_10]
        with open(os.path.join(OUT, "oracle_hubbard10.json"), "w") as f:
            json.dump(res, f, indent=1)
