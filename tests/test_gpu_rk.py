"""GPU parity of the differential-form drivers (Eq. smud marched by Alg. 1
with RK1 / RK2 / RK4) against the oracle's own RK driver, through the C ABI."""
import pytest
import torch

from oracle import differential as df
from oracle import ftccsd as fc
from oracle import systems
from paper_2004_01729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_01729_gb300 import ftcc
    c = ftcc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("order,quad", [(1, 1), (2, 2), (4, 3)])
@pytest.mark.parametrize("ng", [3, 9, 17])
def test_rk_drivers_match_oracle(ctx, order, quad, ng):
    c = wl.HUBBARD_6
    ctx.build_hubbard(c["L"], c["t"], c["U"])
    r = ctx.solve(c["beta"], c["mu"], ng, quad=quad, precision="fp64")
    ref = df.solve_rk(fc.Problem(systems.hubbard_1d(c["L"], c["t"], c["U"]), c["beta"], c["mu"], ng), order)
    assert abs(r["omega"] - ref["omega"]) < 1e-10
    assert r["iterations"] == ng - 1
    assert r["converged"] == 1


def test_rk_batched_temperatures_match_single_solves(ctx):
    from paper_2004_01729_gb300 import ftcc
    cs = wl.HUBBARD_10
    ctxs = []
    for q in cs:
        x = ftcc.Context(0)
        x.build_hubbard(q["L"], q["t"], q["U"])
        ctxs.append(x)
    try:
        rb = ftcc.solve_batched(ctxs, [q["beta"] for q in cs], [q["mu"] for q in cs], 9, quad=3, precision="fp64")
        for q, r in zip(cs, rb):
            ref = df.solve_rk(fc.Problem(systems.hubbard_1d(q["L"], q["t"], q["U"]), q["beta"], q["mu"], 9), 4)
            assert abs(r["omega"] - ref["omega"]) < 1e-10
    finally:
        for x in ctxs:
            x.close()


def test_rk_rejects_what_it_does_not_build(ctx):
    from paper_2004_01729_gb300 import ftcc
    c = wl.HUBBARD_6
    ctx.build_hubbard(c["L"], c["t"], c["U"])
    with pytest.raises(ftcc.FTCCError):
        ctx.solve(c["beta"], c["mu"], 9, quad=3, precision="tf32")
    ctx.solve(c["beta"], c["mu"], 9, quad=3, precision="fp64")
    with pytest.raises(ftcc.FTCCError):
        ctx.adjoint(with_rdm1=False)
    with pytest.raises(ftcc.FTCCError):
        ctx.iterate(1)
