"""Failure detection through the C ABI, with every failure made on the host
(no kernel is made to fault, trap or wait): a NaN-poisoned integral, an
allocator that runs out, calls out of order, an iteration cap, arguments
out of range on a live context, and a device error flag written from the
host as a bounded in-kernel wait that gave up would write it.  After each
failure the same context still solves a valid problem."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2004_01729_gb300 import ftcc, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    c = ftcc.Context(0)
    yield c
    c.close()


def _still_works(c):
    c.build_hubbard(4, 1.0, 2.0)
    r = c.solve(1.0, 1.0, 6, precision="fp64")
    assert r["converged"] and np.isfinite(r["omega"])


def test_nan_in_an_integral_is_diverged(ctx):
    h, eri, eps = wl.random_generic_system(3, 6, v_scale=0.04)
    eri = eri.copy()
    eri[1, 2, 3, 4] = np.nan
    ctx.build_generic(h, eri, eps)
    for prec in ("fp64", "tf32"):
        o = ftcc.default_options(precision=ftcc.PRECISIONS[prec])
        res = ftcc.Result()
        s = ctx.lib.ft_ccsd_solve(ctx.h, 1.0, 0.0, 6, ftcc.QUAD_SIMPSON, ctypes.byref(o), ctypes.byref(res))
        assert s == ftcc.ERR_DIVERGED, (prec, s)
    _still_works(ctx)


def test_allocator_that_runs_out_gives_oom():
    """An allocator with a 2 MB budget: creating the context fits, the
    10-site ring's integrals (1.3 MB of <pq||rs>) too, the solve's buffers do
    not; the call returns FTCC_ERR_OOM instead of failing inside CUDA."""
    lib = ftcc.load()
    live = {}
    budget = [2 << 20]

    def _a(nbytes, user):
        if nbytes > budget[0]:
            return None
        try:
            p = torch.cuda.caching_allocator_alloc(int(nbytes), 0)
        except Exception:
            return None
        budget[0] -= nbytes
        live[p] = nbytes
        return p

    def _f(ptr, user):
        budget[0] += live.pop(ptr, 0)
        torch.cuda.caching_allocator_delete(ptr)

    al = ftcc.Allocator(ftcc.ALLOC_FN(_a), ftcc.FREE_FN(_f), None)
    stream = torch.cuda.Stream(0)
    h = ctypes.c_void_p()
    assert lib.ftcc_create(0, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(al), ctypes.byref(h)) == ftcc.OK
    sysd = ftcc.System(kind=ftcc.SYS_HUBBARD_1D, L=10, t=1.0, U=4.0, pbc=1)
    assert lib.build_integrals(h, ctypes.byref(sysd)) == ftcc.OK
    o = ftcc.default_options(precision=ftcc.PREC_FP64)
    res = ftcc.Result()
    s = lib.ft_ccsd_solve(h, 1.0, 2.0, 32, ftcc.QUAD_SIMPSON, ctypes.byref(o), ctypes.byref(res))
    assert s == ftcc.ERR_OOM, s
    assert b"allocation" in lib.ftcc_last_error(h)
    budget[0] += 1 << 40           # the same context recovers once memory is there
    s = lib.ft_ccsd_solve(h, 1.0, 2.0, 8, ftcc.QUAD_SIMPSON, ctypes.byref(o), ctypes.byref(res))
    assert s == ftcc.OK and res.converged
    lib.ftcc_destroy(h)
    torch.cuda.synchronize()
    assert not live


def test_adjoint_before_a_solve_is_a_state_error(ctx):
    ctx.build_hubbard(4, 1.0, 2.0)
    out = ftcc.AdjointResult()
    assert ctx.lib.ft_ccsd_adjoint(ctx.h, ctypes.byref(out), None) == ftcc.ERR_STATE
    _still_works(ctx)


def test_iteration_cap_is_not_converged_with_outputs(ctx):
    ctx.build_hubbard(6, 1.0, 2.0)
    r = ctx.solve(1.0, 1.0, 16, precision="fp64", max_iter=1, allow_unconverged=True)
    assert r["status"] == ftcc.ERR_NOT_CONVERGED
    assert r["iterations"] == 1 and not r["converged"] and np.isfinite(r["omega"])
    out = ftcc.AdjointResult()
    assert ctx.lib.ft_ccsd_adjoint(ctx.h, ctypes.byref(out), None) == ftcc.ERR_STATE
    _still_works(ctx)


@pytest.mark.parametrize("beta,mu,ngrid", [(0.0, 1.0, 8), (-1.0, 1.0, 8), (float("inf"), 1.0, 8),
                                           (float("nan"), 1.0, 8), (1.0, float("nan"), 8),
                                           (1.0, float("inf"), 8), (1.0, 1.0, 2), (1.0, 1.0, -4)])
def test_invalid_arguments_on_a_live_context(ctx, beta, mu, ngrid):
    ctx.build_hubbard(4, 1.0, 2.0)
    ctx.solve(1.0, 1.0, 6, precision="fp64")
    o = ftcc.default_options()
    res = ftcc.Result()
    s = ctx.lib.ft_ccsd_solve(ctx.h, beta, mu, ngrid, ftcc.QUAD_SIMPSON, ctypes.byref(o), ctypes.byref(res))
    assert s == ftcc.ERR_INVALID_ARG
    bad = ftcc.default_options(damping=0.0)
    s = ctx.lib.ft_ccsd_solve(ctx.h, 1.0, 1.0, 6, ftcc.QUAD_SIMPSON, ctypes.byref(bad), ctypes.byref(res))
    assert s == ftcc.ERR_INVALID_ARG
    _still_works(ctx)


def test_device_error_flag_becomes_timeout(ctx):
    """A device error flag set from the host (the code a bounded TMA wait
    writes when it gives up) turns the next solve into FTCC_ERR_TIMEOUT and
    is cleared by it; the context then solves normally."""
    ctx.build_hubbard(4, 1.0, 2.0)
    ctx.inject_device_error(1)
    o = ftcc.default_options(precision=ftcc.PREC_TF32)
    res = ftcc.Result()
    s = ctx.lib.ft_ccsd_solve(ctx.h, 1.0, 1.0, 6, ftcc.QUAD_SIMPSON, ctypes.byref(o), ctypes.byref(res))
    assert s == ftcc.ERR_TIMEOUT
    assert b"wait" in ctx.lib.ftcc_last_error(ctx.h)
    assert ctx.device_error() == 0
    with pytest.raises(ftcc.FTCCError):
        ctx.inject_device_error(0)
    _still_works(ctx)
