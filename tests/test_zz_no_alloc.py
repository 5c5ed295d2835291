"""The FP64 GEMM entry point that allocates nothing (ftcc_gemm_f64_static).

It exists for callers that cannot allocate device memory where they need the
contraction (code inside a device-memory allocator's own callback, where
allocating would re-enter the allocator, or programs whose device-memory
footprint is fixed at start-up): its split-K partial sums live in a static
device array instead of allocated scratch.  It is checked
through the C ABI against the regular FP64 GEMM entry point, on two calls in
a row with different data so that a stale partial left in the shared array
would show.  This file is collected last so that a failure here stops a
``-x`` run only after every other test has run.
"""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


def _static_gemm(lib, A, B, alpha):
    bt, M, K = A.shape
    N = B.shape[1]
    C = torch.empty((bt, M, N), dtype=torch.float64, device=A.device)
    st = torch.cuda.current_stream().cuda_stream
    s = lib.ftcc_gemm_f64_static(ctypes.c_void_p(st), bt, M, N, K, alpha, A.data_ptr(), K, M * K if bt > 1 else 0,
                                 B.data_ptr(), K, N * K if bt > 1 else 0, C.data_ptr(), N, M * N)
    torch.cuda.synchronize()
    return s, C


@pytest.mark.parametrize("shape", [(1, 64, 48, 8192), (3, 100, 90, 700)])
def test_static_scratch_gemm_matches_regular_gemm(shape):
    from paper_2004_01729_gb300 import ftcc
    lib = ftcc.load()
    ctx = ftcc.Context(0)
    bt, M, N, K = shape
    for call in range(2):
        g = torch.Generator(device="cuda").manual_seed(100 * call + M)
        A = torch.randn((bt, M, K), device="cuda", dtype=torch.float64, generator=g)
        B = torch.randn((bt, N, K), device="cuda", dtype=torch.float64, generator=g)
        ref = ctx.gemm(A, B, precision="fp64", alpha=0.75)
        s, C = _static_gemm(lib, A, B, 0.75)
        assert s == ftcc.OK
        err = (torch.linalg.norm(C - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-13, (call, err)
    ctx.close()


def test_static_scratch_gemm_rejects_outputs_beyond_the_array():
    from paper_2004_01729_gb300 import ftcc
    lib = ftcc.load()
    A = torch.zeros((1, 2048, 8), device="cuda", dtype=torch.float64)
    B = torch.zeros((1, 1024, 8), device="cuda", dtype=torch.float64)
    s, _ = _static_gemm(lib, A, B, 1.0)       # 2^21 outputs > 2^20
    assert s == ftcc.ERR_INVALID_ARG
