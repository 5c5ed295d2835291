"""Benchmark of the FT-CCSD imaginary-time amplitude sweep on GB300.

Headline workload: the warm dense electron gas of 14 electrons at rs = 1,
Theta = T/T_F = 0.5 in 57 plane waves (114 spin orbitals, no truncation),
32 Simpson tau points, mu = mu_0 (the reference chemical potential of 14
electrons).  One step = one iteration of the FP64 sweep with block-sparse
storage (every orbital carries its own momentum and S_z, so the integrals
and amplitudes live in charge sectors): the S kernel at all 32 tau points,
the propagation, the energy and Omega_CC.  value = seconds per step; the
line also carries the time to a solution within 1e-6 Ha of the oracle (the
block-sparse oracle's converged Omega), the roofline of the dominant kernel,
e2e through host buffers and the oracle on the host cores.  Extra fields:
the dense schedule on the same workload (the mixed-precision tcgen05 sweep,
its tensor TFLOP/s, time to 1e-6 Ha, adjoint and the dense FP64 estimate),
the 162-orbital gas (block-sparse solve; dense streamed iteration), the
10-site Hubbard ring at three temperatures (mixed vs FP64 time to 1e-6 Ha),
the adjoint, the 64-instance batch and the RK drivers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3|tf32] [--no-dense] [--quick]
  python bench.py --impl reference ...   # the CPU oracle on the host cores

With N > 1 (torchrun) each rank runs its own copy of the problem
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
C3 = wl.UEG_57
WORKLOAD = ("ueg 14 electrons rs=1 Theta=0.5, 57 plane waves = 114 spin orbitals, ngrid=32 Simpson, "
            "mu=mu_0(N=14)")
C2_WORKLOAD = "hubbard_1d L=10 t=1 U=4 mu=2 N=20 spin orbitals, beta in {2,1,0.5}, ngrid=32 Simpson, batched"
GOLD = os.path.join(ROOT, "tests", "golden")


def measured_peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


def measure_peaks(torch):
    """TF32 (burst and a 3 s loop) and FP64 dense matmul rates of this GPU
    (torch.matmul 8192^3, CUDA events); the bf16 and HBM figures come from
    the driver's measurement."""
    out = {}

    def rate(dt, tf32, reps, loop_s=0.0):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        n = 8192
        a = torch.randn(n, n, device="cuda", dtype=dt)
        b = torch.randn(n, n, device="cuda", dtype=dt)
        a @ b
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        r = {"burst": 2.0 * n ** 3 / best / 1e12}
        if loop_s > 0:
            k = max(1, int(loop_s / best))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(k):
                a @ b
            e1.record()
            torch.cuda.synchronize()
            r["sustained"] = 2.0 * n ** 3 * k / (e0.elapsed_time(e1) * 1e-3) / 1e12
        torch.backends.cuda.matmul.allow_tf32 = False
        del a, b
        return r

    out["tf32_tflops"] = rate(torch.float32, True, 5, 3.0)
    out["fp64_tflops"] = rate(torch.float64, False, 2)
    hbm, bf16, bf16s, src = measured_peaks_file()
    out.update({"bf16_tflops": {"burst": bf16, "sustained": bf16s}, "hbm_gbs": hbm, "bf16_hbm_source": src,
                "how": "torch.matmul 8192^3 with CUDA events: best of several (burst), a 3 s loop (sustained); "
                       "bf16 and HBM from the driver-written measured peaks"})
    return out


def cpu_info():
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"cpu_count": os.cpu_count(), "model": model or platform.machine()}


class Clocks:
    """Sample nvidia-smi during the timed region."""

    def __init__(self, interval_ms=200):
        self.samples = []
        self.proc = None
        self.interval_ms = interval_ms

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", str(self.interval_ms), "-i", os.environ.get("LOCAL_RANK", "0")],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        # wait (at most 3 s) for the first sample so that the loop is covered
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
        pw = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(self.samples),
                "interval_ms": self.interval_ms, "samples_before_timed_region": getattr(self, "first", 0)}


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


def c3_gold():
    p = os.path.join(GOLD, "oracle_ueg57.json")
    return json.load(open(p)) if os.path.exists(p) else None


# ---------------------------------------------------------------- CPU oracle
class OracleSample:
    """The block-sparse oracle (the oracle for the plane-wave gas: the same
    term tables restricted to momentum- and spin-allowed blocks) on a bounded
    sample of one fixed-point iteration of the headline workload: the S
    kernel, the propagation and the energy on n_tau of the 32 tau points,
    scaled to the whole grid (every part is linear in the tau points)."""

    def __init__(self, n_tau=4):
        import torch
        from oracle import blocksparse as bs, chemical_potential as cp
        self.torch, self.bs = torch, bs
        sysc = bs.ueg(C3["n_elec"], C3["rs"], C3["n_pw"])
        mu = cp.mu_reference(sysc["eps"], C3["beta"], float(C3["n_elec"]))
        self.prob = bs.Problem(sysc, C3["beta"], mu, C3["ngrid"])
        self.n_tau = n_tau
        N = self.prob.ch.N
        self.t1, self.t2 = bs.random_amplitudes(self.prob.ch, 1, n_tau, 0.01)
        self.cores = torch.get_num_threads()
        self.N = N

    def run(self):
        """Seconds for the sample and its scale factor to one iteration."""
        bs = self.bs
        t0 = time.perf_counter()
        with self.torch.no_grad():
            S1 = bs.S1(self.prob, self.t1, self.t2)
            S2 = bs.S2(self.prob, self.t1, self.t2)
            bs.energy(self.prob, self.t1, self.t2)
            # the propagation of the sample's tau points (same per-element work as in the sweep)
            for x in range(self.n_tau):
                _ = S2[x] * self.prob.D2
                _ = S1[x] * self.prob.D1
        return time.perf_counter() - t0, C3["ngrid"] / self.n_tau

    def describe(self):
        return (f"block-sparse oracle (FP64, torch CPU, {self.cores} threads): S1, S2, energy and propagation "
                f"of {self.n_tau} of the 32 tau points of the headline workload, scaled by {C3['ngrid'] // self.n_tau}")


def run_reference(args, rank, world):
    if rank != 0:
        return
    smp = OracleSample()
    smp.run()   # builds the contraction plans (untimed)
    for _ in range(args.warmup):
        smp.run()
    times = []
    for _ in range(args.steps):
        dt, scale = smp.run()
        times.append(dt * scale)
    value = statistics.mean(times)
    cpu = cpu_info()
    line = {"metric": METRIC, "value": value, "unit": "s/iteration", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "s/iteration", "cores": smp.cores, "kind": "oracle",
                             "sample": smp.describe(), "cpu_count": cpu["cpu_count"], "cpu_model": cpu["model"],
                             "step_spread_s": [min(times), max(times)]},
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
    prec = args.precision
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
    print(json.dumps({"gemm": [b, M, N, K], "precision": prec, "ms": ms,
                      "tflops": 2.0 * b * M * N * K / ms / 1e9}), flush=True)
    ctx.close()


def run_c3_iteration(args):
    """Prepare the headline workload and run W + K iterations (for the ncu
    launch list of one step)."""
    import torch
    from paper_2004_01729_gb300 import ftcc
    ctx = ftcc.Context(0)
    ctx.build_ueg(C3["n_elec"], C3["rs"], C3["n_pw"])
    mu = ctx.reference_mu(C3["beta"], float(C3["n_elec"]))
    if args.no_dense and args.sparse_precision == "fp64":   # the headline path: block-sparse FP64
        ctx.prepare(C3["beta"], mu, C3["ngrid"], **sparse_opts())
    elif args.no_dense:   # the FP32 sweep of the mixed block-sparse path
        ctx.prepare(C3["beta"], mu, C3["ngrid"], precision="bf16x3", block_sparse=1)
    else:
        ctx.prepare(C3["beta"], mu, C3["ngrid"], precision=args.precision, tau_chunk=8)
    ctx.iterate(args.warmup + args.steps)
    torch.cuda.synchronize()
    if args.c3_adjoint:   # the headline solve to convergence and its adjoint (lambda sweep + response)
        ctx.solve(C3["beta"], mu, C3["ngrid"], **sparse_opts())
        ctx.adjoint(with_rdm1=False)
        torch.cuda.synchronize()
    ctx.close()


def gemm_flops_per_step(kstats, steps):
    """Algorithmic flops (2MNK per product) summed over the contraction classes of one step."""
    return sum(r["flops"] for r in kstats if r["flops"]) / steps


def class_table(kstats, steps):
    total = sum(r["ms"] for r in kstats) or 1.0
    return [{"name": r["name"], "launches_per_step": r["launches"] / steps, "ms_per_step": r["ms"] / steps,
             "share": r["ms"] / total,
             "GB_per_s": r["bytes"] / (r["ms"] * 1e-3) / 1e9 if r["ms"] > 0 else None,
             "TFLOP_per_s": r["flops"] / (r["ms"] * 1e-3) / 1e12 if r["ms"] > 0 and r["flops"] else None}
            for r in sorted(kstats, key=lambda r: -r["ms"])]


def roofline(kstats, steps, prec, pk):
    """Roofline of the dominant kernel class: achieved = its algorithmic
    flops (2MNK per launch) / its device time summed over the launches,
    against the measured peak of its arithmetic; HBM-bound classes against
    the measured copy bandwidth."""
    dom = max(kstats, key=lambda r: r["ms"])
    hbm = pk["hbm_gbs"]
    if prec == "tf32":
        peak, psrc = pk["tf32_tflops"]["sustained"], "TF32 torch.matmul 8192^3, 3 s loop (measured live)"
    else:
        peak = pk["bf16_tflops"]["sustained"] / 3.0
        psrc = "bf16 sustained (driver-measured) / 3: three bf16 products per FP32-accurate one"
    intensity = dom["flops"] / dom["bytes"] if dom["flops"] and dom["bytes"] else None
    ridge = peak * 1e12 / (hbm * 1e9)
    if dom["name"] == "gemm_tc_kernel" and intensity and intensity >= ridge:
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        r = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
             "peak_source": psrc + " (of measured)"}
    else:
        ach = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
        r = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
             "peak_source": "HBM copy (of measured)"}
    r.update({"traffic": None,
              "traffic_note": "DRAM bytes per launch come from ncu captures kept with the kernel profiles; "
                              "not measurable inside this run",
              "kernel": dom["name"], "launches_per_step": dom["launches"] / steps,
              "avg_launch_ms": dom["ms"] / dom["launches"],
              "algorithmic_flops_per_launch": dom["flops"] / dom["launches"],
              "algorithmic_bytes_per_launch": dom["bytes"] / dom["launches"],
              "intensity_flop_per_byte": intensity, "ridge_flop_per_byte": ridge,
              "timed_with": "CUDA events around every launch inside the per-iteration graph "
                            "(a profiled pass after the timed steps)"})
    return r


def bench_dense_mixed(ftcc, torch, dev, world, args, pk, gold):
    """The dense schedule on the headline workload: the mixed-precision
    sweep (tcgen05 contractions over every element of the 114-orbital
    tensors), its solve, adjoint, timed iterations, kernel classes and
    roofline, the FP64 dense estimate and e2e."""
    prec = args.precision
    ctx = ftcc.Context(dev)
    ctx.build_ueg(C3["n_elec"], C3["rs"], C3["n_pw"])
    mu = gold["mu"] if gold else ctx.reference_mu(C3["beta"], float(C3["n_elec"]))
    opts = dict(precision=prec, refine_max_iter=0, tau_chunk=8, max_iter=80)
    # a solve to convergence (host-timed between synchronisations), in tau
    # chunks of 2 so that the adjoint that follows fits beside it
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sol = ctx.solve(C3["beta"], mu, C3["ngrid"], allow_unconverged=True, mixed_adjoint=1,
                    **dict(opts, tau_chunk=2))
    torch.cuda.synchronize()
    t_sol = time.perf_counter() - t0
    solve = {"s_total": t_sol, "iterations": sol["iterations"], "polish_iterations": sol["polish_iterations"],
             "fp64_iterations": sol["refine_iterations"], "converged": bool(sol["converged"]),
             "omega": sol["omega"], "abs_dOmega_vs_oracle": abs(sol["omega"] - gold["omega"]) if gold else None,
             "oracle": "block-sparse oracle, converged to |dOmega_CC| < 1e-11" if gold else None}
    # the response of that solve: the lambda sweep in the mixed arithmetic
    # (FP32 multipliers, BF16X3 VJP), N, E, S against the oracle's central
    # differences of converged solves
    adjoint = None
    if not args.no_adjoint and sol["converged"]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ad, _ = ctx.adjoint(with_rdm1=False)
        torch.cuda.synchronize()
        adjoint = {"s_total": time.perf_counter() - t0, "lambda_iterations": ad["iterations"],
                   "N": ad["N"], "E": ad["E"], "S": ad["S"], "dOmega_dbeta": ad["dOmega_dbeta"]}
        rp = os.path.join(GOLD, "oracle_ueg57_response.json")
        if os.path.exists(rp):
            gr = json.load(open(rp))
            adjoint["abs_diff_vs_oracle"] = {k: abs(ad[k] - gr[k]) for k in ("N", "E", "S")}
            adjoint["oracle"] = gr["how"]

    # timed steps: W warm-up iterations, then K iterations each bracketed by
    # CUDA events on the library stream; the amplitudes (21 GB) and integral
    # blocks are far larger than the 129 MB L2, so no flush is needed
    ctx.prepare(C3["beta"], mu, C3["ngrid"], **opts)
    st = ctx.stream
    ctx.iterate(max(1, args.warmup))
    barrier(world)
    torch.cuda.synchronize()
    dsteps = min(args.steps, 10)   # ~1.2 s per dense step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(dsteps)]
    with Clocks() as clk:
        for a, b in ev:
            a.record(st)
            ctx.iterate(1)
            b.record(st)
        torch.cuda.synchronize()
    barrier(world)
    t_steps = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    k_iter = ctx.iterate(0)["kernels_per_iter"]
    # the same iteration with per-launch events inside the graph
    ctx.profile(True)
    prof_steps = 2
    ctx.iterate(prof_steps)
    kstats = ctx.profile_read()
    ctx.profile(False)
    ctx.close()
    t_steps = barrier_max(t_steps, world)
    s_per_iter = t_steps / dsteps
    fl = flops_per_iteration(114, 114, C3["ngrid"])
    roof = roofline(kstats, prof_steps, prec, pk)

    # FP64 GPU path on the same workload: one tau point of the S kernel in
    # FP64 (SIMT: tcgen05 has no FP64 kind) through ftcc_eval_s, scaled to the
    # 32 points of an iteration (the S kernel is local in tau and takes all
    # but a few percent of an iteration)
    fp64 = None
    if not args.no_fp64:
        try:
            cf = ftcc.Context(dev)
            cf.build_ueg(C3["n_elec"], C3["rs"], C3["n_pw"])
            cf.prepare(C3["beta"], mu, 3, precision="fp64", tau_chunk=1)
            t1, t2 = wl.random_amplitudes(3, 1, 114, 114, 0.01)
            t1 = torch.tensor(t1, device="cuda")
            t2 = torch.tensor(t2, device="cuda")
            cf.eval_s(t1, t2, precision="fp64")   # sizes the workspaces
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cf.eval_s(t1, t2, precision="fp64")
            torch.cuda.synchronize()
            t_tau = time.perf_counter() - t0
            it_fp64 = gold["iterations"] if gold else sol["iterations"]
            fp64 = {"s_per_iteration": t_tau * C3["ngrid"], "s_one_tau_point": t_tau,
                    "tflops": fl / C3["ngrid"] / t_tau / 1e12,
                    "frac_of_measured_fp64_peak": fl / C3["ngrid"] / t_tau / 1e12 / pk["fp64_tflops"]["burst"],
                    "iterations_to_converge": it_fp64,
                    "estimated_s_to_solution": t_tau * C3["ngrid"] * it_fp64,
                    "how": "S kernel of one tau point in FP64 (ftcc_eval_s), host-timed, x 32 tau points; "
                           "iterations from the FP64 oracle's fixed point on the same grid"}
            del t1, t2
            cf.close()
        except Exception as e:   # noqa: BLE001 - reported, the headline line still prints
            fp64 = {"error": f"{type(e).__name__}: {e}"[:300]}

    # e2e through the public API with host buffers: build_integrals from the
    # pinned host Hamiltonian (h, <pq||rs> N^4, eps in FP64), the mixed solve
    # to convergence (the per-iteration state read back each iteration) and
    # the result on the host; value = that time / iterations
    e2e = None
    if not args.no_e2e:
        ce = ftcc.Context(dev)
        ce.build_ueg(C3["n_elec"], C3["rs"], C3["n_pw"])
        h_np, eri_np, eps_np = ce.get_system()
        pin = [torch.from_numpy(a).pin_memory() for a in (h_np, eri_np, eps_np)]
        del h_np, eri_np, eps_np
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ce.build_generic(pin[0].numpy(), pin[1].numpy(), pin[2].numpy())
        r = ce.solve(C3["beta"], mu, C3["ngrid"], allow_unconverged=True, **opts)
        torch.cuda.synchronize()
        t_e = barrier_max(time.perf_counter() - t0, world)
        h2d = sum(a.numel() * 8 for a in pin)
        e2e = {"value": t_e / r["iterations"], "unit": "s/iteration", "h2d_bytes_per_step": h2d / r["iterations"],
               "d2h_bytes_per_step": 8 * (8 + 256) + 112 / r["iterations"],
               "what": "build_integrals(GENERIC, pinned host h, <pq||rs>, eps) + ft_ccsd_solve (mixed, to "
                       "convergence) + result to the host, divided by the iterations of the solve",
               "s_total": t_e, "iterations": r["iterations"],
               "abs_dOmega_vs_oracle": abs(r["omega"] - gold["omega"]) if gold else None}
        del pin
        ce.close()

    return {"workload": WORKLOAD + "; dense storage (every element), " + prec + " tensor-core contractions",
            "s_per_iteration": s_per_iter, "steps": dsteps,
            "tensor_tflops_per_iteration": gemm_flops_per_step(kstats, prof_steps) / s_per_iter / 1e12,
            "algorithmic_flops_per_iteration": gemm_flops_per_step(kstats, prof_steps),
            "dense_schedule_flops_per_iteration": fl,
            "flops_note": "algorithmic = 2MNK summed over the contractions the iteration executes (the ladders "
                          "over unordered index pairs); dense_schedule = the five O(N^6) contractions of the "
                          "unpacked schedule",
            "time_to_1e-6": solve, "adjoint_mixed": adjoint, "fp64_gpu": fp64,
            "mixed_over_fp64_time_to_solution": (fp64["estimated_s_to_solution"] / t_sol
                                                 if fp64 and "estimated_s_to_solution" in fp64 else None),
            "roofline": roof, "kernels": class_table(kstats, prof_steps), "e2e": e2e,
            "gpu_launches_per_iteration": k_iter, "clocks": clk.summary()}


def roofline_sparse(kstats, steps, pk):
    """Roofline of the dominant kernel class of the block-sparse FP64
    iteration: the sector products against the FP64 rate of this GPU
    (cuBLAS DGEMM 8192^3 measured live; the FP64 FMA pipe, "alu"), an
    elementwise class against the measured HBM copy bandwidth."""
    dom = max(kstats, key=lambda r: r["ms"])
    if dom["flops"]:
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        peak = pk["fp64_tflops"]["burst"]
        r = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
             "peak_source": "FP64 FMA pipe: torch.matmul float64 8192^3 (cuBLAS DGEMM), measured live (of measured)"}
    else:
        ach = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
        r = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
             "peak_source": "HBM copy (of measured)"}
    r.update({"traffic": None,
              "traffic_note": "DRAM bytes per launch come from ncu captures kept with the kernel profiles; "
                              "not measurable inside this run",
              "kernel": dom["name"], "launches_per_step": dom["launches"] / steps,
              "avg_launch_ms": dom["ms"] / dom["launches"],
              "algorithmic_flops_per_launch": dom["flops"] / dom["launches"],
              "algorithmic_bytes_per_launch": dom["bytes"] / dom["launches"],
              "timed_with": "CUDA events around every launch inside the per-iteration graph "
                            "(a profiled pass after the timed steps)"})
    return r


def sparse_opts():
    return dict(precision="fp64", block_sparse=1, tol_omega=1e-11, tol_amp=1e-9, max_iter=100)


def run_gpu(args, rank, world):
    import torch
    from paper_2004_01729_gb300 import ftcc
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    pk = measure_peaks(torch)
    gold = c3_gold()
    extra = {}

    # ---- headline: the 114-spin-orbital gas with block-sparse storage, FP64
    ctx = ftcc.Context(dev)
    ctx.build_ueg(C3["n_elec"], C3["rs"], C3["n_pw"])
    mu = gold["mu"] if gold else ctx.reference_mu(C3["beta"], float(C3["n_elec"]))
    ctx.solve(C3["beta"], mu, C3["ngrid"], **sparse_opts())   # first solve: sizes and captures (untimed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sol = ctx.solve(C3["beta"], mu, C3["ngrid"], allow_unconverged=True, **sparse_opts())
    torch.cuda.synchronize()
    t_sol = time.perf_counter() - t0
    solve = {"s_total": t_sol, "iterations": sol["iterations"], "converged": bool(sol["converged"]),
             "omega": sol["omega"], "abs_dOmega_vs_oracle": abs(sol["omega"] - gold["omega"]) if gold else None,
             "oracle": "block-sparse oracle, converged to |dOmega_CC| < 1e-11" if gold else None,
             "how": "ft_ccsd_solve FP64 block-sparse from s = 0 to |dOmega_CC| < 1e-11, host-timed"}
    # the FP64 lambda sweep and response of that solve: N, E, S and the
    # 1-RDM against the oracle's central differences of converged solves
    adjoint = None
    if not args.no_adjoint and sol["converged"]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ad, rdm1 = ctx.adjoint(with_rdm1=True)
        torch.cuda.synchronize()
        adjoint = {"s_total": time.perf_counter() - t0, "lambda_iterations": ad["iterations"],
                   "N": ad["N"], "E": ad["E"], "S": ad["S"], "trace_rdm1": float(rdm1.trace()),
                   "how": "ft_ccsd_adjoint after the block-sparse solve: FP64 lambda sweep through the transpose "
                          "of the block-sparse S kernel, response (App. B), host-timed"}
        rp = os.path.join(GOLD, "oracle_ueg57_response.json")
        if os.path.exists(rp):
            gr = json.load(open(rp))
            adjoint["abs_diff_vs_oracle"] = {k: abs(ad[k] - gr[k]) for k in ("N", "E", "S")}
            adjoint["oracle"] = gr["how"]
    # timed steps: W warm-up iterations, then K iterations each bracketed by
    # CUDA events on the library stream (one captured graph per iteration);
    # the amplitudes (32 x 114^3 x 8 B = 379 MB each for s and S) exceed the
    # 129 MB L2, so no flush is needed
    ctx.prepare(C3["beta"], mu, C3["ngrid"], **sparse_opts())
    st = ctx.stream
    ctx.iterate(max(1, args.warmup))
    barrier(world)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(interval_ms=20) as clk:   # steps of ~13 ms: sample every 20 ms
        for a, b in ev:
            a.record(st)
            ctx.iterate(1)
            b.record(st)
        torch.cuda.synchronize()
    barrier(world)
    t_steps = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    k_iter = ctx.iterate(0)["kernels_per_iter"]
    ctx.profile(True)
    prof_steps = 3
    ctx.iterate(prof_steps)
    kstats = ctx.profile_read()
    ctx.profile(False)
    ctx.close()
    t_steps = barrier_max(t_steps, world)
    s_per_iter = t_steps / args.steps
    roof = roofline_sparse(kstats, prof_steps, pk)

    # the mixed pipeline on the same storage: FP32 sweep (SIMT sector
    # products, FP64 propagator factors and energy sums), then FP64 residual
    # corrections (refine_max_iter = 2, the default)
    mixed = None
    if not args.no_mixed:
        mopts = dict(precision="bf16x3", block_sparse=1, max_iter=100)
        cm = ftcc.Context(dev)
        cm.build_ueg(C3["n_elec"], C3["rs"], C3["n_pw"])
        cm.solve(C3["beta"], mu, C3["ngrid"], allow_unconverged=True, **mopts)   # sizing and captures
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rm = cm.solve(C3["beta"], mu, C3["ngrid"], allow_unconverged=True, **mopts)
        torch.cuda.synchronize()
        tm = time.perf_counter() - t0
        cm.prepare(C3["beta"], mu, C3["ngrid"], **mopts)
        cm.iterate(max(1, args.warmup))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cm.stream)
        cm.iterate(args.steps)
        e1.record(cm.stream)
        torch.cuda.synchronize()
        cm.profile(True)
        cm.iterate(3)
        km = cm.profile_read()
        cm.profile(False)
        cm.close()
        mixed = {"s_per_iteration": e0.elapsed_time(e1) / 1e3 / args.steps, "steps": args.steps,
                 "time_to_1e-6": {"s_total": tm, "iterations": rm["iterations"],
                                  "fp64_corrections": rm["refine_iterations"], "converged": bool(rm["converged"]),
                                  "omega": rm["omega"],
                                  "abs_dOmega_vs_oracle": abs(rm["omega"] - gold["omega"]) if gold else None},
                 "kernels": class_table(km, 3),
                 "how": "FP32 block-sparse sweep (storage and SIMT sector products; propagator factors and energy "
                        "sums in FP64) to |dOmega_CC| < tol_mixed, then up to 2 FP64 residual corrections; "
                        "iterations of the FP32 sweep timed with CUDA events"}
        mixed["fp64_over_mixed_time_to_solution"] = t_sol / tm if tm > 0 else None

    # e2e through the public API with host buffers: the gas's Hamiltonian and
    # its orbital charges from pinned host memory (build_integrals GENERIC
    # with charges), the block-sparse FP64 solve to convergence (the state
    # read back every iteration) and the result on the host
    e2e = None
    if not args.no_e2e:
        ce = ftcc.Context(dev)
        ce.build_ueg(C3["n_elec"], C3["rs"], C3["n_pw"])
        h_np, eri_np, eps_np = ce.get_system()
        ch_np, md_np = ce.get_charges()
        pin = [torch.from_numpy(a).pin_memory() for a in (h_np, eri_np, eps_np)]
        del h_np, eri_np, eps_np
        # first pass sizes the allocator and the graphs (untimed)
        ce.build_generic(pin[0].numpy(), pin[1].numpy(), pin[2].numpy(), ch_np, md_np)
        ce.solve(C3["beta"], mu, C3["ngrid"], allow_unconverged=True, **sparse_opts())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ce.build_generic(pin[0].numpy(), pin[1].numpy(), pin[2].numpy(), ch_np, md_np)
        r = ce.solve(C3["beta"], mu, C3["ngrid"], allow_unconverged=True, **sparse_opts())
        torch.cuda.synchronize()
        t_e = barrier_max(time.perf_counter() - t0, world)
        h2d = sum(a.numel() * 8 for a in pin) + ch_np.nbytes + md_np.nbytes
        e2e = {"value": t_e / r["iterations"], "unit": "s/iteration", "h2d_bytes_per_step": h2d / r["iterations"],
               "d2h_bytes_per_step": 8 * (8 + 256) + 112 / r["iterations"],
               "what": "build_integrals(GENERIC with charges: pinned host h, <pq||rs> N^4, eps) + ft_ccsd_solve "
                       "(FP64 block-sparse, to convergence) + result to the host, divided by the iterations",
               "s_total": t_e, "iterations": r["iterations"],
               "abs_dOmega_vs_oracle": abs(r["omega"] - gold["omega"]) if gold else None}
        del pin
        ce.close()

    # ---- the dense schedule on the same workload, the 162-orbital gas and the rest
    dense = None
    if not args.no_dense:
        dense = bench_dense_mixed(ftcc, torch, dev, world, args, pk, gold)
        extra["dense_mixed"] = dense
    if not args.quick:
        extra["ueg81_162_spin_orbitals"] = bench_ueg81(ftcc, torch, dev, world, args)
        extra["hubbard10"] = bench_hubbard10(ftcc, torch, dev, world, args)
        extra.update(bench_small_extras(ftcc, torch, dev, world, args))
        extra["dense_ladder_gemm"] = bench_dense_gemm(ftcc, torch, dev, world, pk)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            smp = OracleSample()
            smp.run()
            runs = [smp.run() for _ in range(3)]
            vals = [dt * sc for dt, sc in runs]
            ci = cpu_info()
            cpu = {"value": statistics.median(vals), "unit": "s/iteration", "cores": smp.cores, "kind": "oracle",
                   "sample": smp.describe() + "; median of 3", "samples_s_per_iteration": vals,
                   "cpu_count": ci["cpu_count"], "cpu_model": ci["model"]}
        dts = dense["time_to_1e-6"]["s_total"] if dense and dense.get("time_to_1e-6") else None
        line = {"metric": METRIC, "value": s_per_iter, "unit": "s/iteration", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_per_iter * 1e3,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "storage": "block-sparse: momentum/spin charge sectors, FP64",
                           "l2": "inputs larger than L2: s and S are 379 MB each (FP64, 32 x 114^3), the integral "
                                 "blocks 12 x 12 MB; L2 129 MB, no flush"},
                "algorithmic_flops_per_iteration": gemm_flops_per_step(kstats, prof_steps),
                "flops_note": "2 sum_s rows_s^3 over the charge sectors of the five products of two four-index "
                              "factors, every tau point; the dense schedule's 7.0e14 flops per iteration are in "
                              "extra.dense_mixed",
                "time_to_1e-6": solve, "adjoint": adjoint, "mixed_block_sparse": mixed,
                "fp64_block_sparse_vs_dense_mixed_time_to_solution": (dts / t_sol if dts else None),
                "peaks": pk, "roofline": roof, "kernels": class_table(kstats, prof_steps),
                "e2e": e2e, "gpu_launches": k_iter * args.steps, "clocks": clk.summary()}
        line.update(extra)
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)


def bench_hubbard10(ftcc, torch, dev, world, args):
    """The 10-site ring at three temperatures as one batch: time to a
    solution within 1e-6 Ha of the oracle for the mixed pipeline (TF32,
    BF16X3 polish, FP64 corrections) and for the FP64 path, plus the
    steady-state time of one batched TF32 iteration and its kernel classes."""
    cfgs = wl.HUBBARD_10
    gold = json.load(open(os.path.join(GOLD, "oracle_hubbard10.json")))
    betas, mus = [c["beta"] for c in cfgs], [c["mu"] for c in cfgs]

    def built():
        out = []
        for c in cfgs:
            x = ftcc.Context(dev)
            x.build_hubbard(c["L"], c["t"], c["U"])
            out.append(x)
        return out

    out = {"workload": C2_WORKLOAD}
    for name, kw in (("mixed", dict(precision="tf32")), ("fp64", dict(precision="fp64", max_iter=300)),
                     ("tf32_bf16x3_no_fp64", dict(precision="tf32", refine_max_iter=0)),
                     ("tf32_only", dict(precision="tf32", refine_max_iter=0, polish_max_iter=0, tol_mixed=1e-12))):
        ctxs = built()
        ftcc.solve_batched(ctxs, betas, mus, cfgs[0]["ngrid"], allow_unconverged=True, **kw)   # tile tuning
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ftcc.solve_batched(ctxs, betas, mus, cfgs[0]["ngrid"], allow_unconverged=True, **kw)
        torch.cuda.synchronize()
        out[name] = {"s_to_solution": time.perf_counter() - t0, "iterations": res[0]["iterations"],
                     "polish_iterations": res[0]["polish_iterations"], "fp64_iterations": res[0]["refine_iterations"],
                     "max_abs_dOmega_vs_oracle": max(abs(r["omega"] - g["omega"]) for r, g in zip(res, gold)),
                     "converged": all(r["converged"] for r in res)}
        for c in ctxs:
            c.close()
    out["mixed_over_fp64_time_to_solution"] = out["fp64"]["s_to_solution"] / out["mixed"]["s_to_solution"]
    # steady-state TF32 iteration (cold L2 each step)
    ctxs = built()
    ftcc.prepare_batched(ctxs, betas, mus, cfgs[0]["ngrid"], precision="tf32")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    st = ctxs[0].stream
    ctxs[0].iterate(3)
    torch.cuda.synchronize()
    n = 20
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for a, b in ev:
        with torch.cuda.stream(st):
            flush.zero_()
        a.record(st)
        ctxs[0].iterate(1)
        b.record(st)
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in ev) / 1e3 / n
    ctxs[0].profile(True)
    ctxs[0].iterate(n)
    ks = ctxs[0].profile_read()
    ctxs[0].profile(False)
    out["tf32_s_per_batched_iteration"] = t
    out["kernels"] = class_table(ks, n)
    for c in ctxs:
        c.close()
    # FP64 iteration
    ctxs = built()
    ftcc.prepare_batched(ctxs, betas, mus, cfgs[0]["ngrid"], precision="fp64")
    ctxs[0].iterate(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctxs[0].stream)
    ctxs[0].iterate(3)
    e1.record(ctxs[0].stream)
    torch.cuda.synchronize()
    out["fp64_s_per_batched_iteration"] = e0.elapsed_time(e1) / 3e3
    for c in ctxs:
        c.close()
    return out


def bench_ueg81(ftcc, torch, dev, world, args):
    """The 162-orbital gas (81 plane waves, 40 tau points): one dense mixed
    iteration from s = 0 streamed over tau (with the peak device memory),
    and the block-sparse FP64 iteration and solve."""
    if args.no_ueg81 or world != 1:
        return None
    c = wl.UEG_81
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    ctx = ftcc.Context(dev)
    ctx.build_ueg(c["n_elec"], c["rs"], c["n_pw"])
    mu = ctx.reference_mu(c["beta"], float(c["n_elec"]))
    ctx.prepare(c["beta"], mu, c["ngrid"], precision=args.precision, trunc_thr=c["thr"], stream_tau=1, tau_chunk=1)
    st = ctx.stream
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    r = ctx.iterate(1)
    e1.record(st)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    fl = flops_per_iteration(r["n_occ"], r["n_vir"], c["ngrid"])
    dense = {"precision": args.precision, "s_per_iteration": t, "tensor_tflops": fl / t / 1e12,
             "dense_schedule_flops_per_iteration": fl,
             "peak_device_memory_gb": torch.cuda.max_memory_allocated() / 1e9,
             "note": "dense storage, tau-streamed: first iteration from s = 0 (includes the tile autotuning of its "
                     "shapes); S kept for one tau window"}
    ctx.close()
    # block-sparse FP64: timed iterations and a solve to convergence against
    # the block-sparse oracle's converged Omega
    gp = os.path.join(GOLD, "oracle_ueg81.json")
    g81 = json.load(open(gp)) if os.path.exists(gp) else None
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    ctx = ftcc.Context(dev)
    ctx.build_ueg(c["n_elec"], c["rs"], c["n_pw"])
    ctx.solve(c["beta"], mu, c["ngrid"], trunc_thr=c["thr"], **sparse_opts())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rs = ctx.solve(c["beta"], mu, c["ngrid"], trunc_thr=c["thr"], allow_unconverged=True, **sparse_opts())
    torch.cuda.synchronize()
    t_sol = time.perf_counter() - t0
    ctx.prepare(c["beta"], mu, c["ngrid"], trunc_thr=c["thr"], **sparse_opts())
    st = ctx.stream
    ctx.iterate(3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    ctx.iterate(10)
    e1.record(st)
    torch.cuda.synchronize()
    # the lambda sweep and response of the converged solve (dOmega/dmu,
    # dOmega/dbeta, N, E, S)
    adj = None
    if not args.no_adjoint and rs["converged"]:
        ctx.solve(c["beta"], mu, c["ngrid"], trunc_thr=c["thr"], **sparse_opts())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ad, _ = ctx.adjoint(with_rdm1=True)
        torch.cuda.synchronize()
        adj = {"s_total": time.perf_counter() - t0, "lambda_iterations": ad["iterations"],
               "dOmega_dmu": ad["dOmega_dmu"], "dOmega_dbeta": ad["dOmega_dbeta"], "N": ad["N"], "E": ad["E"],
               "S": ad["S"],
               "check": "tests/test_gpu_sparse.py compares dOmega/dmu and dOmega/dbeta with central differences "
                        "(one Richardson step) of converged block-sparse solves to 1e-7"}
    sparse = {"s_per_iteration": e0.elapsed_time(e1) / 1e3 / 10, "solve_s_total": t_sol, "adjoint": adj,
              "iterations": rs["iterations"], "converged": bool(rs["converged"]), "omega": rs["omega"],
              "abs_dOmega_vs_oracle": abs(rs["omega"] - g81["omega"]) if g81 else None,
              "peak_device_memory_gb": torch.cuda.max_memory_allocated() / 1e9,
              "how": "FP64 block-sparse; 10 iterations timed with CUDA events after 3 warm-up; the solve from s = 0 "
                     "to |dOmega_CC| < 1e-11 host-timed"}
    ctx.close()
    return {"workload": "ueg 14 electrons rs=1 Theta=1, 81 plane waves = 162 spin orbitals, ngrid=40, mu=mu_0",
            "block_sparse_fp64": sparse, "dense_first_iteration": dense}


def bench_small_extras(ftcc, torch, dev, world, args):
    out = {}
    if world != 1:
        return out
    # the adjoint (lambda) sweep and response of the beta = 1 ring after an FP64 solve
    c = wl.HUBBARD_10[1]
    ca = ftcc.Context(dev)
    ca.build_hubbard(c["L"], c["t"], c["U"])
    ca.solve(c["beta"], c["mu"], c["ngrid"], precision="fp64", tol_omega=1e-12, tol_amp=1e-10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ar, _ = ca.adjoint(with_rdm1=True)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    out["adjoint_lambda_sweep"] = {"workload": "hubbard_1d L=10 U=4 beta=1, ngrid=32, FP64 lambda sweep + response",
                                   "s_total": t, "lambda_iterations": ar["iterations"],
                                   "s_per_lambda_iteration": t / max(1, ar["iterations"]),
                                   "N": ar["N"], "E": ar["E"], "S": ar["S"]}
    ca.close()
    if args.no_batch:
        return out
    # the 64-instance batch (6-14 sites, U in [1,8], T in [0.25,4], ngrid=24):
    # block-sparse FP64 (every k-space ring carries momentum and S_z), each
    # instance its own batch on its own stream, all iterating in lockstep; then
    # the adjoint of every converged instance; the dense mixed solve beside it
    cb = wl.hubbard_batch()

    def ring_contexts():
        out_ = []
        for q in cb:
            x = ftcc.Context(dev)
            x.build_hubbard(q["L"], q["t"], q["U"])
            out_.append(x)
        return out_

    betas_b, mus_b = [q["beta"] for q in cb], [q["mu"] for q in cb]
    ctx_b = ring_contexts()
    kw_sp = dict(precision="fp64", block_sparse=1, max_iter=300, allow_unconverged=True)
    ftcc.solve_batched(ctx_b, betas_b, mus_b, cb[0]["ngrid"], **kw_sp)   # sizing and captures
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rb = ftcc.solve_batched(ctx_b, betas_b, mus_b, cb[0]["ngrid"], **kw_sp)
    torch.cuda.synchronize()
    bat = {"workload": "64 hubbard_1d instances, L in {6..14}, U in [1,8], T in [0.25,4], half filling, ngrid=24; "
                       "block-sparse FP64, every instance its own batch; once each has captured its iteration, a step "
                       "of all unfinished instances is one graph launch (their iterations as child graphs)",
           "s_total": time.perf_counter() - t0, "instances": len(cb),
           "converged": int(sum(r["converged"] for r in rb)),
           "iterations_max": int(max(r["iterations"] for r in rb))}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    adjs = ftcc.adjoint_batched(ctx_b)   # the batches' lambda sweeps concurrently
    torch.cuda.synchronize()
    bat["adjoint_s_total"] = time.perf_counter() - t0
    bat["adjoint_instances"] = int(sum(a["status"] == ftcc.OK for a in adjs))
    bat["adjoint_how"] = "ft_ccsd_adjoint_batched: every converged instance's FP64 lambda sweep and response, " \
                         "the batches concurrently from a pool of host threads, each on its own stream"
    # the mixed pipeline on the same storage (FP32 sweep, then FP64 residual
    # corrections) and the adjoints after it, against the FP64 solves above
    kw_m = dict(precision="bf16x3", block_sparse=1, max_iter=300, refine_max_iter=3, tol_omega=1e-10,
                tol_amp=1e-8, allow_unconverged=True)
    ftcc.solve_batched(ctx_b, betas_b, mus_b, cb[0]["ngrid"], **kw_m)   # sizing and captures
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rm = ftcc.solve_batched(ctx_b, betas_b, mus_b, cb[0]["ngrid"], **kw_m)
    torch.cuda.synchronize()
    t_m = time.perf_counter() - t0
    t0 = time.perf_counter()
    am = ftcc.adjoint_batched(ctx_b)
    torch.cuda.synchronize()
    ok = [k for k, (x, y) in enumerate(zip(rm, rb)) if x["converged"] and y["converged"]]
    bat["block_sparse_mixed"] = {
        "s_total": t_m, "converged": int(sum(r["converged"] for r in rm)),
        "max_abs_dOmega_vs_fp64": max([abs(rm[k]["omega"] - rb[k]["omega"]) for k in ok], default=None),
        "fp64_corrections_max": int(max(r["refine_iterations"] for r in rm)),
        "adjoint_s_total": time.perf_counter() - t0,
        "adjoint_instances": int(sum(a["status"] == ftcc.OK for a in am)),
        "max_abs_dE_vs_fp64_adjoint": max([abs(am[k]["E"] - adjs[k]["E"]) for k in ok
                                           if am[k]["status"] == ftcc.OK and adjs[k]["status"] == ftcc.OK],
                                          default=None),
        "how": "precision bf16x3 with block_sparse: FP32 sweep, then up to 3 FP64 residual corrections; "
               "ft_ccsd_adjoint_batched after it (FP64 lambda sweeps from the corrected amplitudes)"}
    for x in ctx_b:
        x.close()
    # the dense schedule: one batch per size class, TF32, BF16X3 polish, FP64
    # corrections until the FP64 tolerances hold (at most 30)
    ctx_b = ring_contexts()
    kw_d = dict(precision="tf32", refine_max_iter=30, max_iter=400, allow_unconverged=True)
    ftcc.solve_batched(ctx_b, betas_b, mus_b, cb[0]["ngrid"], **kw_d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rd = ftcc.solve_batched(ctx_b, betas_b, mus_b, cb[0]["ngrid"], **kw_d)
    torch.cuda.synchronize()
    bat["dense_mixed"] = {"s_total": time.perf_counter() - t0, "converged": int(sum(r["converged"] for r in rd)),
                          "how": "one batch per size class (instance letter z), the five classes iterating together "
                                 "on their own streams; the dense adjoint is not timed here"}
    for x in ctx_b:
        x.close()
    out["batched_64_instances"] = bat
    # the differential form (Eq. smud, Alg. 1): RK4 / RK2 marches of the
    # three-temperature ring in FP64 beside the FP64 Simpson fixed point
    cfgs = wl.HUBBARD_10
    rk = {"workload": C2_WORKLOAD + ", FP64, one batched solve each (host-timed, synchronised)"}
    try:
        for name, quad, kw in (("simpson_fp64", ftcc.QUAD_SIMPSON, {"max_iter": 300}),
                               ("rk4_fp64", ftcc.QUAD_RK4, {}), ("rk2_fp64", ftcc.QUAD_RK2, {})):
            ctxs = []
            for q in cfgs:
                x = ftcc.Context(dev)
                x.build_hubbard(q["L"], q["t"], q["U"])
                ctxs.append(x)
            betas, mus = [q["beta"] for q in cfgs], [q["mu"] for q in cfgs]
            ftcc.solve_batched(ctxs, betas, mus, cfgs[0]["ngrid"], quad=quad, precision="fp64", **kw)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = ftcc.solve_batched(ctxs, betas, mus, cfgs[0]["ngrid"], quad=quad, precision="fp64", **kw)
            torch.cuda.synchronize()
            rk[name] = {"s_total": time.perf_counter() - t0, "iterations_or_steps": res[0]["iterations"],
                        "omega": [r["omega"] for r in res]}
            for x in ctxs:
                x.close()
        rk["rk4_minus_simpson_omega"] = [a - b for a, b in zip(rk["rk4_fp64"]["omega"], rk["simpson_fp64"]["omega"])]
    except Exception as e:   # noqa: BLE001 - reported, the headline line still prints
        rk["error"] = f"{type(e).__name__}: {e}"[:300]
    out["differential_form"] = rk
    return out


def bench_dense_gemm(ftcc, torch, dev, world, pk):
    """The dense particle-ladder product of one 8-point tau chunk of the
    headline workload, [8*12996 x 12996] . [12996 x 12996]^T, through
    ftcc_gemm alone (host-timed between synchronisations)."""
    if world != 1:
        return None
    out = {}
    try:
        nn = 114 * 114
        cg = ftcc.Context(dev)
        ga = torch.randn((1, 8 * nn, nn), device="cuda", dtype=torch.float32)
        gb = torch.randn((1, nn, nn), device="cuda", dtype=torch.float32)
        fl = 2.0 * 8 * nn * nn * nn
        for prec in ("tf32", "bf16x3"):
            cg.gemm(ga, gb, precision=prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                cg.gemm(ga, gb, precision=prec)
            torch.cuda.synchronize()
            t = (time.perf_counter() - t0) / 3
            peak = pk["tf32_tflops"]["burst"] if prec == "tf32" else pk["bf16_tflops"]["burst"] / 3.0
            out[prec] = {"shape_bmnk": [1, 8 * nn, nn, nn], "ms": t * 1e3, "tflops": fl / t / 1e12,
                         "frac_of_measured_peak": fl / t / 1e12 / peak}
        del ga, gb
        cg.close()
    except Exception as e:   # noqa: BLE001
        out["error"] = f"{type(e).__name__}: {e}"[:300]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "tf32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ueg81", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the lambda sweep of the headline workload")
    ap.add_argument("--quick", action="store_true", help="headline only, no extra workloads")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense mixed-precision sweep")
    ap.add_argument("--no-mixed", action="store_true", help="skip the FP32 block-sparse sweep")
    ap.add_argument("--c3-iterations", action="store_true",
                    help="prepare the headline workload and run W + K iterations (profiler launch lists)")
    ap.add_argument("--c3-adjoint", action="store_true",
                    help="with --c3-iterations --no-dense: then solve and run the adjoint (profiler launch lists)")
    ap.add_argument("--sparse-precision", default="fp64", choices=["fp64", "bf16x3"],
                    help="with --c3-iterations --no-dense: the block-sparse FP64 iteration or its FP32 sweep")
    ap.add_argument("--gemm", default=None, help="B,M,N,K: time the tensor-core GEMM alone on that shape")
    args = ap.parse_args()
    rank, world = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.gemm:
        run_gemm_only(args)
    elif args.c3_iterations:
        run_c3_iteration(args)
    else:
        run_gpu(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
