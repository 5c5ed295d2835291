"""Thin ctypes binding of libftcc (include/ftcc.h); argument marshalling only.

Every step of the FT-CCSD sweep runs inside the CUDA library.  PyTorch is
used for device memory (the library allocates through torch's caching
allocator) and for the CUDA stream.  There is no fallback: if the library or
a GPU is missing the calls raise.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libftcc.so")

OK, ERR_INVALID_ARG, ERR_NO_DEVICE, ERR_OOM, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_TIMEOUT, \
    ERR_UNSUPPORTED, ERR_STATE, ERR_CUDA = range(10)
QUAD_SIMPSON, QUAD_RK1, QUAD_RK2, QUAD_RK4 = range(4)
PREC_FP64, PREC_TF32, PREC_BF16X3 = range(3)
SYS_HUBBARD_1D, SYS_UEG, SYS_GENERIC = range(3)
REF_KSPACE_RHF, REF_NEEL_SITE, REF_UHF_SITE = range(3)
REFERENCES = {"kspace_rhf": REF_KSPACE_RHF, "neel": REF_NEEL_SITE, "uhf": REF_UHF_SITE}
PRECISIONS = {"fp64": PREC_FP64, "tf32": PREC_TF32, "bf16x3": PREC_BF16X3}


class System(C.Structure):
    _fields_ = [("kind", C.c_int), ("L", C.c_int), ("t", C.c_double), ("U", C.c_double), ("pbc", C.c_int),
                ("n_elec", C.c_int), ("rs", C.c_double), ("n_pw", C.c_int), ("N", C.c_int),
                ("h", C.POINTER(C.c_double)), ("eri", C.POINTER(C.c_double)), ("eps", C.POINTER(C.c_double)),
                ("reference", C.c_int), ("charge", C.POINTER(C.c_int)), ("charge_mod", C.POINTER(C.c_int))]


class Options(C.Structure):
    _fields_ = [("tol_omega", C.c_double), ("tol_amp", C.c_double), ("damping", C.c_double),
                ("trunc_thr", C.c_double), ("max_iter", C.c_int), ("precision", C.c_int),
                ("refine_max_iter", C.c_int), ("tol_mixed", C.c_double), ("tau_chunk", C.c_int),
                ("use_graph", C.c_int), ("stream_tau", C.c_int),
                ("autotune", C.c_int), ("polish_max_iter", C.c_int), ("fp64_propagation", C.c_int),
                ("tol_refine", C.c_double), ("mixed_adjoint", C.c_int), ("block_sparse", C.c_int)]


class Result(C.Structure):
    _fields_ = [("omega", C.c_double), ("omega0", C.c_double), ("omega1", C.c_double), ("omega_cc", C.c_double),
                ("d_omega", C.c_double), ("d_amp", C.c_double), ("iterations", C.c_int),
                ("refine_iterations", C.c_int), ("converged", C.c_int), ("n_occ", C.c_int), ("n_vir", C.c_int),
                ("ms_per_iter", C.c_double), ("kernels_per_iter", C.c_int), ("polish_iterations", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AdjointResult(C.Structure):
    _fields_ = [("dOmega_dmu", C.c_double), ("dOmega_dbeta", C.c_double), ("N", C.c_double), ("E", C.c_double),
                ("S", C.c_double), ("trace_rdm1", C.c_double), ("iterations", C.c_int)]


class KernelStats(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_longlong), ("ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", FREE_FN), ("user", C.c_void_p)]


_lib = None

# (name, restype, argtypes) for every entry point of include/ftcc.h
_SIGS = [
    ("ftcc_create", C.c_int, [C.c_int, C.c_void_p, C.POINTER(Allocator), C.POINTER(C.c_void_p)]),
    ("ftcc_destroy", None, [C.c_void_p]),
    ("ftcc_status_string", C.c_char_p, [C.c_int]),
    ("ftcc_last_error", C.c_char_p, [C.c_void_p]),
    ("build_integrals", C.c_int, [C.c_void_p, C.POINTER(System)]),
    ("ftcc_num_orbitals", C.c_int, [C.c_void_p]),
    ("ftcc_get_system", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ftcc_get_charges", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ftcc_reference_mu", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.POINTER(C.c_double)]),
    ("ftcc_mu_for_n", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int, C.POINTER(Options),
                                C.c_double, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(Result)]),
    ("ftcc_prepare", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int, C.POINTER(Options),
                               C.POINTER(Result)]),
    ("ft_ccsd_iterate", C.c_int, [C.c_void_p, C.c_int, C.POINTER(Result)]),
    ("ft_ccsd_solve", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int, C.POINTER(Options),
                                C.POINTER(Result)]),
    ("ft_ccsd_solve_batched", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.c_int, C.c_int, C.POINTER(Options),
                                        C.POINTER(Result)]),
    ("ftcc_prepare_batched", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.c_int, C.c_int, C.POINTER(Options)]),
    ("ft_ccsd_adjoint", C.c_int, [C.c_void_p, C.POINTER(AdjointResult), C.c_void_p]),
    ("ft_ccsd_adjoint_batched", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(AdjointResult),
                                          C.POINTER(C.c_int)]),
    ("ftcc_get_amplitudes", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ftcc_rdm2", C.c_int, [C.c_void_p, C.c_void_p]),
    ("ftcc_eval_s", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ftcc_propagate", C.c_int, [C.c_void_p, C.c_char_p, C.c_void_p, C.c_void_p]),
    ("ftcc_gemm", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                            C.c_void_p, C.c_longlong, C.c_longlong, C.c_void_p, C.c_longlong, C.c_longlong,
                            C.c_void_p, C.c_longlong, C.c_longlong]),
    ("ftcc_eval_s_vjp", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    ("ftcc_propagate_adjoint", C.c_int, [C.c_void_p, C.c_char_p, C.c_void_p, C.c_void_p]),
    ("ftcc_get_lambda", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ftcc_gemm_f64_static", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                       C.c_void_p, C.c_longlong, C.c_longlong, C.c_void_p, C.c_longlong,
                                       C.c_longlong, C.c_void_p, C.c_longlong, C.c_longlong]),
    ("ftcc_profile", C.c_int, [C.c_void_p, C.c_int]),
    ("ftcc_profile_read", C.c_int, [C.c_void_p, C.POINTER(KernelStats), C.c_int]),
    ("ftcc_device_error", C.c_int, [C.c_void_p]),
    ("ftcc_inject_device_error", C.c_int, [C.c_void_p, C.c_int]),
]


def load(path=LIB_PATH):
    """Load libftcc.so (raises OSError / FileNotFoundError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run __graft_entry__.build() first")
    lib = C.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FTCCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def default_options(**kw):
    o = Options(tol_omega=1e-10, tol_amp=1e-8, damping=1.0, trunc_thr=0.0, max_iter=200,
                precision=PREC_FP64, refine_max_iter=2, tol_mixed=1e-7, tau_chunk=0, use_graph=1, stream_tau=0,
                autotune=1, polish_max_iter=40, fp64_propagation=1, tol_refine=1e-6, mixed_adjoint=0,
                block_sparse=0)
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(o, k, v)
    return o


class Context:
    """One libftcc context on a CUDA device, allocating through torch."""

    def __init__(self, device=0, stream=None, torch_alloc=True):
        import torch
        self._torch = torch
        self.lib = load()
        self.device = device
        if stream is None:
            # a created stream: the per-iteration CUDA graph cannot capture the legacy stream
            stream = torch.cuda.Stream(device)
        self.stream = stream
        self._alloc = None
        alloc_p = None
        if torch_alloc:
            dev, st = device, stream

            def _a(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:
                    return None

            def _f(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc = Allocator(ALLOC_FN(_a), FREE_FN(_f), None)
            alloc_p = C.byref(self._alloc)
        h = C.c_void_p()
        s = self.lib.ftcc_create(device, C.c_void_p(stream.cuda_stream), alloc_p, C.byref(h))
        if s != OK:
            raise FTCCError(s, "ftcc_create: " + self.lib.ftcc_status_string(s).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.ftcc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _in(self):
        """Order the context stream after the caller's current stream."""
        cur = self._torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        return cur

    def _out(self, cur):
        """Order the caller's stream after the library's work."""
        cur.wait_stream(self.stream)

    def _check(self, s, what, allow=()):
        if s != OK and s not in allow:
            raise FTCCError(s, f"{what}: {self.lib.ftcc_status_string(s).decode()}: "
                               f"{self.lib.ftcc_last_error(self.h).decode()}")
        return s

    # -- systems
    def build_hubbard(self, L, t, U, reference="kspace_rhf"):
        ref = REFERENCES[reference] if isinstance(reference, str) else int(reference)
        sysd = System(kind=SYS_HUBBARD_1D, L=L, t=t, U=U, pbc=1, reference=ref)
        self._check(self.lib.build_integrals(self.h, C.byref(sysd)), "build_integrals")
        return self.num_orbitals()

    def build_ueg(self, n_elec, rs, n_pw):
        sysd = System(kind=SYS_UEG, n_elec=n_elec, rs=rs, n_pw=n_pw)
        self._check(self.lib.build_integrals(self.h, C.byref(sysd)), "build_integrals")
        return self.num_orbitals()

    def build_generic(self, h, eri, eps, charge=None, charge_mod=None):
        """GENERIC system from host arrays; charge [N, 4] (int) and charge_mod [4]
        optionally give every orbital's conserved charge (block_sparse)."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        eri = np.ascontiguousarray(eri, dtype=np.float64)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        sysd = System(kind=SYS_GENERIC, N=len(eps), h=_dptr(h), eri=_dptr(eri), eps=_dptr(eps))
        keep = []
        if charge is not None:
            ch = np.ascontiguousarray(charge, dtype=np.int32).reshape(len(eps), 4)
            keep.append(ch)
            sysd.charge = ch.ctypes.data_as(C.POINTER(C.c_int))
            if charge_mod is not None:
                md = np.ascontiguousarray(charge_mod, dtype=np.int32).reshape(4)
                keep.append(md)
                sysd.charge_mod = md.ctypes.data_as(C.POINTER(C.c_int))
        self._check(self.lib.build_integrals(self.h, C.byref(sysd)), "build_integrals")
        return self.num_orbitals()

    def get_charges(self):
        """ftcc_get_charges: (charge [N, 4], charge_mod [4]) of the built system."""
        N = self.num_orbitals()
        ch = np.empty((N, 4), dtype=np.int32)
        md = np.empty(4, dtype=np.int32)
        self._check(self.lib.ftcc_get_charges(self.h, ch.ctypes.data, md.ctypes.data), "ftcc_get_charges")
        return ch, md

    def build(self, cfg):
        if cfg["kind"] == "hubbard":
            return self.build_hubbard(cfg["L"], cfg["t"], cfg["U"])
        if cfg["kind"] == "ueg":
            return self.build_ueg(cfg["n_elec"], cfg["rs"], cfg["n_pw"])
        raise ValueError(cfg["kind"])

    def num_orbitals(self):
        return self.lib.ftcc_num_orbitals(self.h)

    def get_system(self, with_eri=True):
        N = self.num_orbitals()
        eps = np.empty(N)
        h = np.empty((N, N))
        eri = np.empty((N, N, N, N)) if with_eri else None
        self._check(self.lib.ftcc_get_system(self.h, eps.ctypes.data, h.ctypes.data,
                                             eri.ctypes.data if with_eri else None), "ftcc_get_system")
        return h, eri, eps

    def reference_mu(self, beta, n_elec):
        mu = C.c_double()
        self._check(self.lib.ftcc_reference_mu(self.h, beta, n_elec, C.byref(mu)), "ftcc_reference_mu")
        return mu.value

    def mu_for_n(self, beta, n_target, ngrid, mu0, dmu=0.05, tol_n=1e-10, max_evals=40, quad=QUAD_SIMPSON, **opts):
        """ftcc_mu_for_n: mu_CC with N(mu_CC) = n_target; returns (mu, N, evaluations, last solve)."""
        o = default_options(**opts)
        r = Result()
        mu, n, ev = C.c_double(), C.c_double(), C.c_int()
        self._check(self.lib.ftcc_mu_for_n(self.h, beta, n_target, ngrid, quad, C.byref(o), mu0, dmu, tol_n,
                                           max_evals, C.byref(mu), C.byref(n), C.byref(ev), C.byref(r)),
                    "ftcc_mu_for_n")
        return mu.value, n.value, ev.value, r.as_dict()

    # -- solves
    def prepare(self, beta, mu, ngrid, quad=QUAD_SIMPSON, **opts):
        o = default_options(**opts)
        r = Result()
        self._check(self.lib.ftcc_prepare(self.h, beta, mu, ngrid, quad, C.byref(o), C.byref(r)), "ftcc_prepare")
        return r.as_dict()

    def iterate(self, n):
        r = Result()
        self._check(self.lib.ft_ccsd_iterate(self.h, n, C.byref(r)), "ft_ccsd_iterate")
        return r.as_dict()

    def solve(self, beta, mu, ngrid, quad=QUAD_SIMPSON, allow_unconverged=False, **opts):
        o = default_options(**opts)
        r = Result()
        s = self.lib.ft_ccsd_solve(self.h, beta, mu, ngrid, quad, C.byref(o), C.byref(r))
        self._check(s, "ft_ccsd_solve", allow=(ERR_NOT_CONVERGED,) if allow_unconverged else ())
        d = r.as_dict()
        d["status"] = s
        return d

    def adjoint(self, with_rdm1=True, allow_unsupported=False):
        """ft_ccsd_adjoint: dOmega/dmu, dOmega/dbeta, N, E, S and the 1-RDM p^cc."""
        out = AdjointResult()
        N = self.num_orbitals()
        rdm = np.empty((N, N)) if with_rdm1 else None
        s = self.lib.ft_ccsd_adjoint(self.h, C.byref(out), rdm.ctypes.data if with_rdm1 else None)
        self._check(s, "ft_ccsd_adjoint", allow=(ERR_UNSUPPORTED,) if allow_unsupported else ())
        d = {k: getattr(out, k) for k, _ in out._fields_}
        d["status"] = s
        return d, rdm

    def rdm2(self):
        """ftcc_rdm2: the unrelaxed normal-ordered 2-RDM Gamma_N [N, N, N, N] after adjoint()."""
        N = self.num_orbitals()
        g = np.empty((N, N, N, N))
        self._check(self.lib.ftcc_rdm2(self.h, g.ctypes.data), "ftcc_rdm2")
        return g

    def amplitudes(self, ngrid, no, nv):
        s1 = np.empty((ngrid, no, nv))
        s2 = np.empty((ngrid, no, no, nv, nv))
        self._check(self.lib.ftcc_get_amplitudes(self.h, s1.ctypes.data, s2.ctypes.data), "ftcc_get_amplitudes")
        return s1, s2

    # -- kernels exposed for parity checks (torch CUDA tensors in and out)
    def eval_s(self, t1, t2, precision="fp64"):
        torch = self._torch
        t1 = t1.to(device=f"cuda:{self.device}", dtype=torch.float64).contiguous()
        t2 = t2.to(device=f"cuda:{self.device}", dtype=torch.float64).contiguous()
        s1 = torch.empty_like(t1)
        s2 = torch.empty_like(t2)
        cur = self._in()
        self._check(self.lib.ftcc_eval_s(self.h, t1.shape[0], PRECISIONS[precision], t1.data_ptr(),
                                         t2.data_ptr(), s1.data_ptr(), s2.data_ptr()), "ftcc_eval_s")
        self._out(cur)
        return s1, s2

    def eval_s_vjp(self, t1, t2, w1, w2):
        torch = self._torch
        dev = f"cuda:{self.device}"
        t1, t2, w1, w2 = [a.to(device=dev, dtype=torch.float64).contiguous() for a in (t1, t2, w1, w2)]
        b1 = torch.empty_like(t1)
        b2 = torch.empty_like(t2)
        cur = self._in()
        self._check(self.lib.ftcc_eval_s_vjp(self.h, t1.shape[0], t1.data_ptr(), t2.data_ptr(), w1.data_ptr(),
                                             w2.data_ptr(), b1.data_ptr(), b2.data_ptr()), "ftcc_eval_s_vjp")
        self._out(cur)
        return b1, b2

    def propagate_adjoint(self, slots, m):
        torch = self._torch
        m = m.to(device=f"cuda:{self.device}", dtype=torch.float64).contiguous()
        out = torch.empty_like(m)
        cur = self._in()
        self._check(self.lib.ftcc_propagate_adjoint(self.h, slots.encode(), m.data_ptr(), out.data_ptr()),
                    "ftcc_propagate_adjoint")
        self._out(cur)
        return out

    def get_lambda(self, ngrid, no, nv):
        m1 = np.empty((ngrid, no, nv))
        m2 = np.empty((ngrid, no, no, nv, nv))
        self._check(self.lib.ftcc_get_lambda(self.h, m1.ctypes.data, m2.ctypes.data), "ftcc_get_lambda")
        return m1, m2

    def propagate(self, slots, S):
        torch = self._torch
        S = S.to(device=f"cuda:{self.device}", dtype=torch.float64).contiguous()
        out = torch.empty_like(S)
        cur = self._in()
        self._check(self.lib.ftcc_propagate(self.h, slots.encode(), S.data_ptr(), out.data_ptr()),
                    "ftcc_propagate")
        self._out(cur)
        return out

    def gemm(self, A, B, precision="fp64", alpha=1.0, shared_b=False):
        """C[b] = alpha A[b] B[b]^T for A [batch, M, K], B [batch or 1, N, K] CUDA tensors."""
        torch = self._torch
        dt = torch.float64 if precision == "fp64" else torch.float32
        A = A.to(dt).contiguous()
        B = B.to(dt).contiguous()
        bt, M, K = A.shape
        N = B.shape[1]
        Cm = torch.empty((bt, M, N), dtype=dt, device=A.device)
        sb = 0 if (shared_b or B.shape[0] == 1) else N * K
        cur = self._in()
        self._check(self.lib.ftcc_gemm(self.h, PRECISIONS[precision], bt, M, N, K, alpha,
                                       A.data_ptr(), K, M * K if bt > 1 else 0, B.data_ptr(), K, sb,
                                       Cm.data_ptr(), N, M * N), "ftcc_gemm")
        self._out(cur)
        return Cm

    def profile(self, enable=True):
        self._check(self.lib.ftcc_profile(self.h, 1 if enable else 0), "ftcc_profile")

    def profile_read(self):
        out = (KernelStats * 8)()
        n = self.lib.ftcc_profile_read(self.h, out, 8)
        return [{"name": out[i].name.decode(), "launches": out[i].launches, "ms": out[i].ms,
                 "bytes": out[i].bytes, "flops": out[i].flops} for i in range(n)]

    def device_error(self):
        return self.lib.ftcc_device_error(self.h)

    def inject_device_error(self, code):
        self._check(self.lib.ftcc_inject_device_error(self.h, int(code)), "ftcc_inject_device_error")


def _batch_args(ctxs, betas, mus):
    n = len(ctxs)
    hs = (C.c_void_p * n)(*[c.h.value for c in ctxs])
    b = (C.c_double * n)(*[float(x) for x in betas])
    m = (C.c_double * n)(*[float(x) for x in mus])
    return n, hs, b, m


def solve_batched(ctxs, betas, mus, ngrid, quad=QUAD_SIMPSON, allow_unconverged=False, **opts):
    """ft_ccsd_solve_batched over Context objects; returns one result dict per instance."""
    lib = load()
    n, hs, b, m = _batch_args(ctxs, betas, mus)
    o = default_options(**opts)
    out = (Result * n)()
    for c in ctxs:
        c.stream.wait_stream(c._torch.cuda.current_stream(c.device))
    s = lib.ft_ccsd_solve_batched(hs, n, b, m, ngrid, quad, C.byref(o), out)
    if s != OK and not (allow_unconverged and s in (ERR_NOT_CONVERGED, ERR_DIVERGED)):
        raise FTCCError(s, "ft_ccsd_solve_batched: " + lib.ftcc_status_string(s).decode() + ": "
                        + lib.ftcc_last_error(ctxs[0].h).decode())
    res = [r.as_dict() for r in out]
    for r in res:
        r["status"] = s
    return res


def adjoint_batched(ctxs):
    """ft_ccsd_adjoint_batched: the adjoints of several contexts, their batches
    concurrently; one (result dict, status) pair per context, no exception
    for a failing member."""
    lib = load()
    n = len(ctxs)
    hs = (C.c_void_p * n)(*[c.h.value for c in ctxs])
    out = (AdjointResult * n)()
    st = (C.c_int * n)()
    for c in ctxs:
        c.stream.wait_stream(c._torch.cuda.current_stream(c.device))
    s = lib.ft_ccsd_adjoint_batched(hs, n, out, st)
    if s == ERR_INVALID_ARG and all(v == 0 for v in st):
        raise FTCCError(s, "ft_ccsd_adjoint_batched: invalid arguments")
    res = []
    for r, v in zip(out, st):
        d = {k: getattr(r, k) for k, _ in r._fields_}
        d["status"] = v
        res.append(d)
    return res


def prepare_batched(ctxs, betas, mus, ngrid, quad=QUAD_SIMPSON, **opts):
    """ftcc_prepare_batched: set up the batches (s = 0) without iterating."""
    lib = load()
    n, hs, b, m = _batch_args(ctxs, betas, mus)
    o = default_options(**opts)
    s = lib.ftcc_prepare_batched(hs, n, b, m, ngrid, quad, C.byref(o))
    if s != OK:
        raise FTCCError(s, "ftcc_prepare_batched: " + lib.ftcc_status_string(s).decode() + ": "
                        + lib.ftcc_last_error(ctxs[0].h).decode())


def _omega_function():
    """torch.autograd.Function for Omega(beta, mu, V) of a context's system
    (built on first use so that importing this module needs no torch)."""
    import torch

    class FTCCOmega(torch.autograd.Function):
        """Omega = Omega0 + Omega1 + Omega_CC of the system held by a Context,
        as a differentiable function of beta, mu and a one-body perturbation V
        (N x N, added to h with its diagonal also added to the reference
        energies).  forward runs ft_ccsd_solve; backward runs the GPU lambda
        sweep (ft_ccsd_adjoint) and returns dOmega/dbeta, dOmega/dmu (= -N)
        and dOmega/dV_pq = rdm1[q, p] (App. B).  V = None leaves the system
        as built; a V solves the perturbed system, rebuilt from the context's
        first (unperturbed) system."""

        @staticmethod
        def forward(fctx, beta, mu, V, context, ngrid, opts):
            if V is not None:
                if not hasattr(context, "_base_system"):
                    context._base_system = context.get_system()
                h, eri, eps = context._base_system
                v = V.detach().cpu().double().numpy()
                context.build_generic(h + v, eri, eps + np.diag(v))
            r = context.solve(float(beta), float(mu), int(ngrid), **(opts or {}))
            fctx.context = context
            fctx.has_v = V is not None
            return torch.tensor(r["omega"], dtype=torch.float64)

        @staticmethod
        def backward(fctx, g):
            d, rdm = fctx.context.adjoint(with_rdm1=True)
            gb = g * d["dOmega_dbeta"]
            gm = g * d["dOmega_dmu"]
            gv = g * torch.from_numpy(rdm.T.copy()) if fctx.has_v else None
            return gb, gm, gv, None, None, None

    return FTCCOmega


def omega(context, beta, mu, ngrid, V=None, **opts):
    """Differentiable Omega(beta, mu[, V]) (see _omega_function); beta and mu
    may be torch scalars with requires_grad."""
    import torch
    f = _omega_function()
    b = beta if torch.is_tensor(beta) else torch.tensor(float(beta), dtype=torch.float64)
    m = mu if torch.is_tensor(mu) else torch.tensor(float(mu), dtype=torch.float64)
    return f.apply(b, m, V, context, ngrid, opts)
