"""Benchmark of the FT-CCSD imaginary-time amplitude sweep on GB300.

Workload: the 10-site Hubbard ring (t=1, U=4, mu=U/2, 20 spin orbitals,
32 Simpson tau points) at beta = 2, 1 and 0.5, solved as one batch.  One
step = one application of the fixed-point map (S kernel at every tau point,
propagation, energy and Omega) to all three temperatures; the metric is
seconds per such iteration, mixed-precision path (TF32 tensor cores, FP32
storage, FP64 propagators and Omega) with the FP64 GPU path measured beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision tf32|bf16x3|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

With N > 1 (torchrun) each rank runs its own copy of the three problems
(independent instances, no collective on the data path: weak scaling); the
timing is the maximum over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2004_01729_gb300 import workloads as wl  # noqa: E402

METRIC = "FT-CCSD s/iteration & tensor TFLOP/s, mixed vs FP64 GPU at |dOmega|<=1e-6 Ha"
WORKLOAD = "hubbard_1d L=10 t=1 U=4 mu=2 N=20 spin orbitals, beta in {2,1,0.5}, ngrid=32 Simpson"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# nominal dense ratios of the recipe: tf32 1.1 PF vs bf16 2.25 PF
TF32_PER_BF16 = 1.1 / 2.25

# DRAM bytes (read + write) per launch of a kernel class in this step, from
# one ncu capture of the current kernels (profiles/ gives the command); a
# class missing here reports traffic null
MEASURED_TRAFFIC = {
    "gemm_tc_kernel": (78.6e6, "profiles/gemm_tc_kernel_hubbard10_tf32.md: mean over 327 launches"),
}


class Clocks:
    """Sample nvidia-smi during the timed region."""

    def __init__(self):
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", os.environ.get("LOCAL_RANK", "0")],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        # nvidia-smi takes longer to start than the timed loop lasts: wait
        # (at most 3 s) for its first sample so that the loop is covered
        t0 = time.time()
        while self.proc is not None and not self.samples and self.proc.poll() is None and time.time() - t0 < 3.0:
            time.sleep(0.01)
        self.first = len(self.samples)   # samples before the timed region
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples), "interval_ms": 50,
                "samples_before_timed_region": getattr(self, "first", 0)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend, init_method="env://")
    return rank, world


def barrier_max(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- CPU oracle arm
def oracle_iteration_seconds(cfg, n_iter=1):
    """Time n_iter oracle fixed-point iterations from s = 0 (bounded sample)."""
    import torch
    from oracle import ftccsd as fc, systems
    s = systems.hubbard_1d(cfg["L"], cfg["t"], cfg["U"])
    p = fc.Problem(s, cfg["beta"], cfg["mu"], cfg["ngrid"])
    no, nv, ng = len(p.iO), len(p.iV), cfg["ngrid"]
    t1 = torch.zeros((ng, no, nv), dtype=torch.float64)
    t2 = torch.zeros((ng, no, no, nv, nv), dtype=torch.float64)
    fc.fixed_point_map(p, t1, t2)   # warm caches
    t0 = time.perf_counter()
    with torch.no_grad():
        for _ in range(n_iter):
            t1, t2 = fc.fixed_point_map(p, t1, t2)
            fc.omega_cc(p, t1, t2)
    return (time.perf_counter() - t0) / n_iter


def run_reference(args, rank, world):
    if rank != 0:
        return
    import torch
    cores = torch.get_num_threads()
    cfgs = wl.HUBBARD_10
    for _ in range(args.warmup):
        pass
    times = []
    for _ in range(args.steps):
        times.append(sum(oracle_iteration_seconds(c, 1) for c in cfgs))
    step = statistics.mean(times)
    value = step / len(cfgs)
    line = {"metric": METRIC, "value": value, "unit": "s/iteration", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "s/iteration", "cores": cores, "kind": "oracle",
                             "sample": "one fixed-point iteration of each temperature per step, from s=0"},
            "e2e": {"value": value, "unit": "s/iteration", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def flops_per_iteration(no, nv, ng):
    """Algorithmic flops of the five O(N^6) contractions of one iteration
    (particle ladder o^2 v^4, hole ladder + W_mnij 2 o^4 v^2, ring + W_mbej 2 o^3 v^3)."""
    return 2.0 * ng * (no ** 2 * nv ** 4 + 2 * no ** 4 * nv ** 2 + 2 * no ** 3 * nv ** 3)


def run_gemm_only(args):
    """Time the tensor-core GEMM alone on one shape (for kernel profiles)."""
    import torch
    from paper_2004_01729_gb300 import ftcc
    b, M, N, K = [int(v) for v in args.gemm.split(",")]
    ctx = ftcc.Context(0)
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((b, M, K), device="cuda", dtype=torch.float32, generator=g)
    B = torch.randn((b, N, K), device="cuda", dtype=torch.float32, generator=g)
    prec = args.precision if args.precision != "fp64" else "tf32"
    for _ in range(args.warmup):
        ctx.gemm(A, B, precision=prec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.gemm(A, B, precision=prec)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # each call returns after a stream synchronise, so ms includes the host
    # work of the call; ncu's kernel duration is the device-only figure
    print(json.dumps({"gemm": [b, M, N, K], "precision": prec, "ms": ms,
                      "tflops": 2.0 * b * M * N * K / ms / 1e9}), flush=True)
    ctx.close()


def run_gpu(args, rank, world):
    import numpy as np
    import torch
    from paper_2004_01729_gb300 import ftcc
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cfgs = wl.HUBBARD_10
    gold_path = os.path.join(ROOT, "tests", "golden", "oracle_hubbard10.json")
    gold = json.load(open(gold_path)) if os.path.exists(gold_path) else None

    betas = [c["beta"] for c in cfgs]
    mus = [c["mu"] for c in cfgs]

    def built():
        out = []
        for c in cfgs:
            ctx = ftcc.Context(dev)
            ctx.build_hubbard(c["L"], c["t"], c["U"])
            out.append(ctx)
        return out

    # accuracy at convergence (untimed): batched full solves in both arithmetics
    acc = {}
    for prec in (() if args.quick else (args.precision, "fp64")):
        ctxs = built()
        res = ftcc.solve_batched(ctxs, betas, mus, cfgs[0]["ngrid"], precision=prec, refine_max_iter=20,
                                 max_iter=300, allow_unconverged=True)
        errs = [abs(r["omega"] - g["omega"]) for r, g in zip(res, gold)] if gold else []
        acc[prec] = {"max_abs_dOmega_vs_oracle": max(errs) if errs else None,
                     "iterations_total": res[0]["iterations"], "refine_iterations": res[0]["refine_iterations"],
                     "converged": all(r["converged"] for r in res)}
        for c in ctxs:
            c.close()

    def make_ctxs(prec):
        out = built()
        ftcc.prepare_batched(out, betas, mus, cfgs[0]["ngrid"], precision=prec)
        return out

    # L2 hygiene: a 256 MB buffer (twice the 129 MB L2) is rewritten on the
    # library stream before every timed step, outside the step's events
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(ctxs, steps, warmup):
        # one step = one batched iteration of all three temperatures, timed
        # with CUDA events on the stream the library launches on
        st = ctxs[0].stream
        for _ in range(warmup):
            ctxs[0].iterate(1)
        barrier(world)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            with torch.cuda.stream(st):
                flush.zero_()
            a.record(st)
            ctxs[0].iterate(1)
            b.record(st)
        torch.cuda.synchronize()
        barrier(world)
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    ctx_mixed = make_ctxs(args.precision)
    with Clocks() as clk:
        t_mixed = timed(ctx_mixed, args.steps, args.warmup)
    # the same steps again with per-kernel CUDA events inside the iteration graph
    ctx_mixed[0].profile(True)
    t_prof = timed(ctx_mixed, args.steps, 1)
    kstats = ctx_mixed[0].profile_read()
    ctx_mixed[0].profile(False)
    if args.quick:
        print(json.dumps({"quick": True, "s_per_iteration": t_mixed / args.steps,
                          "kernels_per_iter": ctx_mixed[0].iterate(0)["kernels_per_iter"],
                          "ms_per_step_by_class": {r["name"]: r["ms"] / args.steps for r in kstats}}), flush=True)
        for ctx in ctx_mixed:
            ctx.close()
        return
    ctx_fp64 = make_ctxs("fp64")
    t_fp64 = timed(ctx_fp64, max(1, min(args.steps, 3)), 1)
    k_mixed = ctx_mixed[0].iterate(0)["kernels_per_iter"]
    res0 = ctx_mixed[0].iterate(0)
    no, nv = res0["n_occ"], res0["n_vir"]
    n_prob = len(cfgs)
    t_mixed = barrier_max(t_mixed, world)
    t_fp64 = barrier_max(t_fp64, world)
    # one step = one batched fixed-point iteration of the three temperatures
    s_per_iter = t_mixed / (args.steps * world)
    fp64_s_per_iter = t_fp64 / (max(1, min(args.steps, 3)) * world)
    fl = n_prob * flops_per_iteration(no, nv, cfgs[0]["ngrid"])

    # e2e: the public API from pinned host Hamiltonian arrays: build_integrals
    # (host -> device) for the three instances + one batched solve to
    # convergence (per-iteration state read back) + results on the host
    ctx_e = built()
    h_np, eri_np, eps_np = ctx_e[0].get_system()
    pin = [torch.from_numpy(a).pin_memory() for a in (h_np, eri_np, eps_np)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ctx in ctx_e:
        ctx.build_generic(pin[0].numpy(), pin[1].numpy(), pin[2].numpy())
    res = ftcc.solve_batched(ctx_e, betas, mus, cfgs[0]["ngrid"], precision=args.precision, refine_max_iter=20,
                             max_iter=300, allow_unconverged=True)
    torch.cuda.synchronize()
    e2e_t = barrier_max(time.perf_counter() - t0, world)
    e2e_iters = res[0]["iterations"]
    h2d = len(ctx_e) * sum(a.numel() * 8 for a in pin)
    e2e = {"value": e2e_t / (e2e_iters * world), "unit": "s/iteration", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": e2e_iters * 8 * (8 + 256) * len(cfgs) + len(cfgs) * 112,
           "what": "build_integrals(host arrays) x3 + ft_ccsd_solve_batched to convergence; one step = the whole solve"}
    for ctx in ctx_e:
        ctx.close()

    # the 114-spin-orbital gas (UEG, 57 plane waves, 32 tau points): per-iteration time
    # of the same sweep where the O(N^6) contractions dominate
    ueg = {}
    if not args.no_ueg and world == 1:
        c = wl.UEG_57
        ctx_u = ftcc.Context(dev)
        ctx_u.build_ueg(c["n_elec"], c["rs"], c["n_pw"])
        mu_u = ctx_u.reference_mu(c["beta"], float(c["n_elec"]))
        for prec in ("tf32", "bf16x3"):
            ctx_u.prepare(c["beta"], mu_u, c["ngrid"], precision=prec, tau_chunk=8)
            ctx_u.iterate(1)
            st = ctx_u.stream
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ctx_u.iterate(2)
            e1.record(st)
            torch.cuda.synchronize()
            t_it = e0.elapsed_time(e1) / 2e3
            fl_u = flops_per_iteration(114, 114, c["ngrid"])
            ueg[prec] = {"s_per_iteration": t_it, "tensor_tflops": fl_u / t_it / 1e12,
                         "algorithmic_flops_per_iteration": fl_u}
            # the contractions alone: one more iteration with per-launch events
            ctx_u.profile(True)
            ctx_u.iterate(1)
            ks = ctx_u.profile_read()
            ctx_u.profile(False)
            g = [r for r in ks if r["name"] == "gemm_tc_kernel"]
            if g and g[0]["ms"] > 0:
                tf = g[0]["flops"] / (g[0]["ms"] * 1e-3) / 1e12
                pk = peaks()[1] * TF32_PER_BF16 if prec == "tf32" else peaks()[1] / 3.0
                ueg[prec]["tensor_core_gemm"] = {
                    "ms_per_iteration": g[0]["ms"], "tflops": tf, "peak_tflops": pk, "frac_of_peak": tf / pk,
                    "peak_source": "measured bf16 burst x nominal tf32/bf16" if prec == "tf32"
                    else "measured bf16 burst / 3 (three bf16 products per FP32-accurate one)",
                    "share_of_iteration": g[0]["ms"] / sum(r["ms"] for r in ks)}
        ctx_u.close()

    # the 162-orbital gas (UEG, 81 plane waves, 40 tau points), streamed over
    # tau (S kept for one window, Simpson chain carried): one TF32 iteration
    ueg81 = None
    if not args.no_ueg and not args.quick and world == 1:
        c = wl.UEG_81
        torch.cuda.empty_cache()
        torch.cuda.reset_peak_memory_stats()
        ctx_u = ftcc.Context(dev)
        ctx_u.build_ueg(c["n_elec"], c["rs"], c["n_pw"])
        mu_u = ctx_u.reference_mu(c["beta"], float(c["n_elec"]))
        ctx_u.prepare(c["beta"], mu_u, c["ngrid"], precision="tf32", trunc_thr=c["thr"], stream_tau=1, tau_chunk=1)
        st = ctx_u.stream
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        r81 = ctx_u.iterate(1)
        e1.record(st)
        torch.cuda.synchronize()
        t_it = e0.elapsed_time(e1) / 1e3
        fl_u = flops_per_iteration(r81["n_occ"], r81["n_vir"], c["ngrid"])
        ueg81 = {"tf32_streamed": {"s_per_iteration": t_it, "tensor_tflops": fl_u / t_it / 1e12,
                                   "algorithmic_flops_per_iteration": fl_u,
                                   "peak_device_memory_gb": torch.cuda.max_memory_allocated() / 1e9,
                                   "note": "first iteration from s = 0; S kept for one tau window"}}
        ctx_u.close()

    # the adjoint (lambda) sweep and response of the beta = 1 instance after an
    # FP64 solve: seconds per lambda iteration (ft_ccsd_adjoint, host timed)
    adj = None
    bat64 = None
    if not args.quick and world == 1:
        c = cfgs[1]
        ctx_a = ftcc.Context(dev)
        ctx_a.build_hubbard(c["L"], c["t"], c["U"])
        ctx_a.solve(c["beta"], c["mu"], c["ngrid"], precision="fp64", tol_omega=1e-12, tol_amp=1e-10)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ar, _ = ctx_a.adjoint(with_rdm1=True)
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        adj = {"workload": "hubbard_1d L=10 U=4 beta=1, ngrid=32, FP64 lambda sweep + response",
               "s_total": t_adj, "lambda_iterations": ar["iterations"],
               "s_per_lambda_iteration": t_adj / max(1, ar["iterations"]),
               "dOmega_dmu": ar["dOmega_dmu"], "N": ar["N"], "E": ar["E"], "S": ar["S"]}
        ctx_a.close()
        # the 64-instance batch (6-14 sites, U in [1,8], T in [0.25,4], ngrid=24):
        # one batched mixed solve with FP64 refinement, per size class
        cb = wl.hubbard_batch()
        ctx_b = []
        for q in cb:
            x = ftcc.Context(dev)
            x.build_hubbard(q["L"], q["t"], q["U"])
            ctx_b.append(x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rb = ftcc.solve_batched(ctx_b, [q["beta"] for q in cb], [q["mu"] for q in cb], cb[0]["ngrid"],
                                precision=args.precision, refine_max_iter=30, max_iter=400, allow_unconverged=True)
        torch.cuda.synchronize()
        t_b = time.perf_counter() - t0
        bat64 = {"workload": "64 hubbard_1d instances, L in {6..14}, ngrid=24, batched per size class",
                 "s_total": t_b, "instances": len(cb), "converged": int(sum(r["converged"] for r in rb)),
                 "iterations_max": int(max(r["iterations"] for r in rb))}
        # energies and entropies from the adjoint (one FP64 lambda sweep per
        # size-class batch; a batch with a diverged member has none), for the
        # 6- and 8-site classes, which keep the default run within minutes
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_adj = 0
        for x, q in zip(ctx_b, cb):
            if q["L"] > 8:
                continue
            try:
                x.adjoint(with_rdm1=False)
                n_adj += 1
            except ftcc.FTCCError:
                pass
        torch.cuda.synchronize()
        bat64["adjoint_s_total"] = time.perf_counter() - t0
        bat64["adjoint_instances"] = n_adj
        bat64["adjoint_scope"] = "instances with L <= 8 (12 and 16 spin orbitals)"
        for x in ctx_b:
            x.close()

    # (the two measurements below run last: a fault in either can only cost its own field)
    if not args.no_ueg and world == 1:
        # the dense O(N^6) contraction of that sweep on its own: the particle
        # ladder of one 8-point tau chunk, [8*12996 x 12996] . [12996 x 12996]^T,
        # through ftcc_gemm (host-timed between synchronisations; the call's
        # host work is negligible beside its ~40 ms); the class figure above
        # also holds the short-K, memory-bound products
        try:
            nn = 114 * 114
            ctx_g = ftcc.Context(dev)
            ga = torch.randn((1, 8 * nn, nn), device="cuda", dtype=torch.float32)
            gb = torch.randn((1, nn, nn), device="cuda", dtype=torch.float32)
            fl_g = 2.0 * 8 * nn * nn * nn
            for prec in ("tf32", "bf16x3"):
                ctx_g.gemm(ga, gb, precision=prec)   # warm
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(3):
                    ctx_g.gemm(ga, gb, precision=prec)   # output dropped at once
                torch.cuda.synchronize()
                t_g = (time.perf_counter() - t0) / 3
                pk = peaks()[1] * TF32_PER_BF16 if prec == "tf32" else peaks()[1] / 3.0
                ueg.setdefault(prec, {})["dense_ladder_gemm"] = {
                    "shape_bmnk": [1, 8 * nn, nn, nn], "ms": t_g * 1e3, "tflops": fl_g / t_g / 1e12,
                    "frac_of_peak": fl_g / t_g / 1e12 / pk}
            del ga, gb
            ctx_g.close()
        except Exception as e:   # noqa: BLE001 - reported, the headline line still prints
            ueg["dense_ladder_gemm_error"] = f"{type(e).__name__}: {e}"[:300]

    # the differential form (Eq. smud, Alg. 1): an RK4 / RK2 march of the same
    # batch in FP64, host-timed whole solves beside the FP64 Simpson fixed
    # point (the paper's Table II compares these costs); a failure here is
    # reported in the line, not raised
    rk = None
    if not args.quick and world == 1:
        rk = {"workload": WORKLOAD + ", FP64, one batched solve each (host-timed, synchronised)"}
        try:
            for name, quad, kw in (("simpson_fp64", ftcc.QUAD_SIMPSON, {"max_iter": 300}),
                                   ("rk4_fp64", ftcc.QUAD_RK4, {}), ("rk2_fp64", ftcc.QUAD_RK2, {})):
                ctxs = built()
                try:
                    ftcc.solve_batched(ctxs, betas, mus, cfgs[0]["ngrid"], quad=quad, precision="fp64", **kw)  # warm
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    res = ftcc.solve_batched(ctxs, betas, mus, cfgs[0]["ngrid"], quad=quad, precision="fp64", **kw)
                    torch.cuda.synchronize()
                    rk[name] = {"s_total": time.perf_counter() - t0, "iterations_or_steps": res[0]["iterations"],
                                "omega": [r["omega"] for r in res]}
                finally:
                    for c in ctxs:
                        c.close()
            rk["rk4_minus_simpson_omega"] = [a - b for a, b in zip(rk["rk4_fp64"]["omega"],
                                                                   rk["simpson_fp64"]["omega"])]
        except Exception as e:   # noqa: BLE001 - reported, the headline line still prints
            rk["error"] = f"{type(e).__name__}: {e}"[:300]

    # roofline of the dominant kernel class of the timed step (events inside the graph)
    hbm, bf16, bf16s, src = peaks()
    tf32_peak = bf16 * TF32_PER_BF16
    dom = max(kstats, key=lambda r: r["ms"]) if kstats else None
    total_ms = sum(r["ms"] for r in kstats) or 1.0
    kernels = [{"name": r["name"], "launches": r["launches"], "ms": r["ms"], "share": r["ms"] / total_ms,
                "GB_per_s": r["bytes"] / (r["ms"] * 1e-3) / 1e9 if r["ms"] > 0 else None,
                "TFLOP_per_s": r["flops"] / (r["ms"] * 1e-3) / 1e12 if r["ms"] > 0 and r["flops"] else None}
               for r in sorted(kstats, key=lambda r: -r["ms"])]
    # a contraction is tensor-bound only when its algorithmic intensity
    # (flops per algorithmic byte) is above the ridge point peak_flops / peak_bw;
    # below it the roofline ceiling is intensity x HBM bandwidth
    ridge = tf32_peak * 1e12 / (hbm * 1e9)
    intensity = dom["flops"] / dom["bytes"] if dom and dom["flops"] and dom["bytes"] else None
    if dom and dom["name"] == "gemm_tc_kernel" and intensity is not None and intensity >= ridge:
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s", "frac": ach / tf32_peak,
                "peak_source": f"bf16 burst {bf16} ({src}) x nominal tf32/bf16 {TF32_PER_BF16:.3f}"}
    elif dom:
        ach = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "peak_source": f"hbm copy {hbm} GB/s ({src})"}
    else:
        roof = {"bound": None}
    if dom:
        tr = MEASURED_TRAFFIC.get(dom["name"])
        roof.update({"traffic": tr[0] if tr else None, "traffic_source": tr[1] if tr else None,
                     "kernel": dom["name"],
                     "launches_per_step": dom["launches"] / args.steps,
                     "avg_launch_us": dom["ms"] * 1e3 / dom["launches"],
                     "algorithmic_bytes_per_launch": dom["bytes"] / dom["launches"],
                     "algorithmic_flops_per_launch": dom["flops"] / dom["launches"],
                     "intensity_flop_per_byte": intensity,
                     "ridge_flop_per_byte": ridge,
                     "tensor_frac": (dom["flops"] / (dom["ms"] * 1e-3) / 1e12 / tf32_peak
                                     if dom["flops"] else None),
                     "timed_with": "CUDA events around every launch inside the per-iteration graph, "
                                   "a second pass of the same steps"})
    for ctx in ctx_mixed + ctx_fp64:
        ctx.close()

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import torch as _t
            cpu_s = oracle_iteration_seconds(cfgs[1], 1)
            cpu = {"value": cpu_s, "unit": "s/iteration", "cores": _t.get_num_threads(), "kind": "oracle",
                   "sample": "one oracle fixed-point iteration at beta=1 (the middle temperature)"}
        line = {"metric": METRIC, "value": s_per_iter, "unit": "s/iteration", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_mixed / args.steps * 1e3,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "precision": args.precision,
                           "l2": "flushed: a 256 MB buffer is rewritten on the library stream before every "
                                 "timed step, outside the step's CUDA events"},
                "fp64_gpu_s_per_iteration": fp64_s_per_iter,
                "mixed_over_fp64_speedup": fp64_s_per_iter / s_per_iter,
                "tensor_tflops_per_iteration": fl / s_per_iter / 1e12,
                "accuracy": acc,
                "roofline": roof, "kernels": kernels, "profiled_step_ms": t_prof / args.steps * 1e3,
                "ueg57_114_spin_orbitals": ueg or None,
                "ueg81_162_spin_orbitals": ueg81,
                "adjoint_lambda_sweep": adj, "batched_64_instances": bat64, "differential_form": rk,
                "e2e": e2e, "gpu_launches": k_mixed * args.steps,
                "clocks": clk.summary()}
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32", choices=["tf32", "bf16x3", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ueg", action="store_true", help="skip the 114-spin-orbital gas timing")
    ap.add_argument("--quick", action="store_true", help="timed mixed loop only (for profiler launch lists)")
    ap.add_argument("--gemm", default=None, help="B,M,N,K: time the tensor-core GEMM alone on that shape")
    args = ap.parse_args()
    rank, world = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.gemm:
        run_gemm_only(args)
    else:
        run_gpu(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
