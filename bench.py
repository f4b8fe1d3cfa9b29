"""Benchmark of the sparse-grid isogeometric solve on GB300: learned/mixed
against plain per-grid FP64 PCG.

Workload (the learned-preconditioner configuration): 3D Poisson
-div(a grad u) = 1 on the unit cube mapped by a seeded cubic B-spline
perturbation (amplitude 0.1), log-normal coefficient a (std 0.5, correlation
length 0.2, 128 random Fourier features), p = 3 C^2 B-splines, combination
level w = 12 (199 component grids with 12 <= |i| <= 14, 3,026,945 DoFs),
every component solved to relative residual 1e-8, then evaluation of every
component on the 17^3 parametric lattice and the +-combination sum.

A step = load vector from f at the quadrature points (resident in HBM) +
batched solve (the faster of the mixed FP32/FP64 solve with fast
diagonalisation and the same with the learned scaling, chosen at set-up) +
evaluation + combination, through the C ABI. `value` is the whole job's DoF/s
(sum of component DoFs over all ranks / step time); each rank under torchrun
solves its own replica of the workload (weak scaling). The comparators of the
metric (plain per-grid FP64 PCG, batched FP64 PCG, mixed FD, learned + mixed,
and the network-free scaling) are timed once each beside it, with their error
against the oracle's stored combined values; the set-up is broken down by
phase. The earlier FP64 unit-cube line (w = 10) is kept under "cube_fp64".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sparse-grid IGA solve wall time & DoF/s at 1e-8 L2, learned/mixed vs plain PCG"
WORKLOAD = dict(d=3, p=3, w=12, nfeat=128, tol=1e-8, lattice=16, inner_tol=1e-3)
WORKLOAD_NAME = ("3D Poisson -div(a grad u) = 1 on the unit cube mapped by a seeded cubic B-spline perturbation "
                 "(amplitude 0.1), log-normal a (std 0.5, correlation length 0.2, 128 Fourier features), p=3 C^2 "
                 "B-splines, combination level w=12 (199 grids, 12<=|i|<=14, 3026945 DoFs), every component solved "
                 "to rel. residual 1e-8, eval+combine on the 17^3 parametric lattice")
GOLDEN = os.path.join(ROOT, "tests", "golden", "perturbed_p3_w12.txt")
# the earlier FP64 unit-cube line (kept beside the headline)
CUBE = dict(d=3, p=3, w=10, tol=1e-12, lattice=16)
CUBE_NAME = ("3D unit-cube Poisson, u=sin(pi x)sin(pi y)sin(pi z), p=3 C^2, w=10 (136 grids, 557030 DoFs), FP64 "
             "matrix-free apply + batched FD-PCG to rel. residual 1e-12, eval+combine on 17^3")
CUBE_GOLDEN = os.path.join(ROOT, "tests", "golden", "cube_p3_w10.txt")
# components of the workload solved by the CPU oracle in its bounded sample
# (assembly + sparse direct solve + evaluation); |i| = 12, the smallest grids
ORACLE_SAMPLE = [(10, 1, 1), (4, 4, 4)]
# the reference arm's one component per step, cycling
REFERENCE_SAMPLE = [(10, 1, 1), (1, 10, 1), (4, 4, 4), (1, 1, 10)]
# DRAM bytes (read + write) of one launch of the FP32 apply on this workload
# at the autotuned tiles (110 KB budget, 16,384-point cap, 256 threads, whole
# prefetch): the mean of three launches of one ncu capture of the current
# kernel (dram__bytes_read.sum + dram__bytes_write.sum)
APPLY_F32_DRAM_BYTES = 3192.9e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--host-loop", action="store_true",
                    help="run the CG loops from the host instead of the captured graph (same kernels; "
                         "profilers list the kernels of a device-side graph loop only this way)")
    ap.add_argument("--quick", action="store_true",
                    help="headline only: skip the comparators, the cube line and the CPU baselines")
    ap.add_argument("--oracle-parallel", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-list", default="", help=argparse.SUPPRESS)
    return ap.parse_args()


# ----------------------------------------------------------------------------
# CPU oracle sample (runs in a child process with one BLAS thread)
# ----------------------------------------------------------------------------

def oracle_task(lv):
    """One component of the workload through the oracle: assembly, sparse
    direct solve, evaluation on the lattice. Returns its DoFs."""
    from oracle import geometry, problems
    from oracle.galerkin import Component
    from paper_1707_09598_gb300.inputs import eval_points, lognormal_features, perturbed_cube_patch
    kn, cp = perturbed_cube_patch(1)
    om, ph, amp = lognormal_features(2, nfeat=WORKLOAD["nfeat"])
    geom = geometry.BSplinePatch([3, 3, 3], kn, cp)
    comp = Component(geom, lv, WORKLOAD["p"]).assemble(f=problems.get("one3").f,
                                                       diffusion=geometry.lognormal_coefficient(om, ph, amp))
    comp.evaluate(comp.solve(), eval_points(3, WORKLOAD["lattice"]))
    return comp.ndof


def oracle_sample_child(comps):
    dofs = 0
    t0 = time.perf_counter()
    for lv in comps:
        dofs += oracle_task(lv)
    dt = time.perf_counter() - t0
    print(json.dumps({"dofs": dofs, "seconds": dt, "components": len(comps)}))


def oracle_parallel_child(per_core):
    """The paper's parallelisation of the combination technique on the host:
    a pool of one-thread workers (spawned) over every core, components in LPT
    order (largest first), per_core tasks per core drawn from ORACLE_SAMPLE."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    tasks = [ORACLE_SAMPLE[i % len(ORACLE_SAMPLE)] for i in range(per_core * ncores)]
    tasks.sort(key=lambda lv: -(2 ** sum(lv)))
    ctx = mp.get_context("spawn")
    with ctx.Pool(ncores) as pool:
        pool.map(int, range(ncores))                    # workers up before timing
        t0 = time.perf_counter()
        dofs = sum(pool.imap_unordered(oracle_task, tasks, chunksize=1))
        dt = time.perf_counter() - t0
    print(json.dumps({"dofs": dofs, "seconds": dt, "components": len(tasks), "cores": ncores}))


def run_oracle_sample(n, parallel=False, comps=None):
    """Serial: the components `comps` (default ORACLE_SAMPLE) in one child;
    parallel: n tasks per core over a spawned pool."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    if parallel:
        argv = ["--oracle-parallel", str(n)]
    else:
        comps = ORACLE_SAMPLE if comps is None else comps
        argv = ["--oracle-list", ";".join(",".join(map(str, lv)) for lv in comps)]
    out = subprocess.run([sys.executable, os.path.abspath(__file__)] + argv,
                         env=env, capture_output=True, text=True, cwd=ROOT)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(v, world, device):
    """Largest v over all ranks (identity for one rank); every rank gets it."""
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed / the max-over-ranks time (weak scaling)."""
    return world * units_per_rank / seconds


class Clocks:
    """nvidia-smi clock/throttle sampling (200 ms) around the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


class NvmlClocks:
    """SM clock and clock-event reasons read through NVML (the driver's
    libnvidia-ml, ctypes) every `period` seconds in a background thread,
    between start() and stop(): dense enough for a timed region of tens of
    milliseconds. Read-only; the device is matched by PCI bus id."""

    # nvmlClocksEventReasons bits (nvml.h)
    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, torch, local, period=0.005):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        props = torch.cuda.get_device_properties(local)
        bus = None
        if all(hasattr(props, k) for k in ("pci_domain_id", "pci_bus_id", "pci_device_id")):
            bus = "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
        if bus is None or self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(self.h)) != 0:
            if self.lib.nvmlDeviceGetHandleByIndex_v2(local, ctypes.byref(self.h)) != 0:
                raise RuntimeError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.period = period
        self.sm, self.bits, self.stop_flag, self.thread = [], 0, False, None

    def _run(self):
        ct = self.ct
        mhz, rs = ct.c_uint(), ct.c_ulonglong()
        while not self.stop_flag:
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz)) == 0:   # NVML_CLOCK_SM
                self.sm.append(float(mhz.value))
            if self.reasons_fn(self.h, ct.byref(rs)) == 0:
                self.bits |= rs.value
            time.sleep(self.period)

    def start(self):
        import threading
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_flag = True
        self.thread.join(timeout=2)
        mx = self.ct.c_uint()
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, self.ct.byref(mx))
        if not self.sm:
            return None
        return {"sm_mhz": statistics.median(self.sm), "sm_max_mhz": float(mx.value),
                "reasons": sorted(n for b, n in self.BITS.items() if self.bits & b), "samples": len(self.sm),
                "source": "NVML, %g ms period, timed region only" % (self.period * 1e3)}


def clock_sampler(torch, local):
    """NVML sampler where the driver library loads, else nvidia-smi at 200 ms."""
    try:
        return NvmlClocks(torch, local)
    except Exception:
        return Clocks(local)


def apply_flops(plan):
    """Algorithmic FP64 flops of one operator apply: untiled sum factorisation
    (forward: 2(p+1) + 3(p+1) + 3(p+1) FMA per output of the three stages,
    pointwise 9 FMA per qp -- 3 when the metric is diagonal --, backward
    mirrored), best axis order per grid."""
    import itertools
    p = plan.info.p
    pw = 3 if plan.info.diag_metric else 9
    P1, Q = p + 1, p + 1
    total = 0.0
    for g in plan.grids:
        E = [2 ** g.levels[k] for k in range(3)]
        nf = [g.n[k] + 2 for k in range(3)]
        best = None
        for a, b, c in itertools.permutations(range(3)):
            s_c = 2 * P1 * nf[a] * nf[b] * Q * E[c]
            s_b = 3 * P1 * nf[a] * Q * E[b] * Q * E[c]
            s_a = 3 * P1 * Q * E[a] * Q * E[b] * Q * E[c]
            fma = 2 * (s_a + s_b + s_c) + pw * Q ** 3 * E[0] * E[1] * E[2]
            best = fma if best is None else min(best, fma)
        total += 2.0 * best
    return total


def fp64_peak_tflops(torch):
    """Measured FP64 dense peak: cuBLAS DGEMM 8192^3, best of 5 (TFLOP/s)."""
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


# ----------------------------------------------------------------------------
# reference arm: the CPU oracle, on host cores
# ----------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    k = 0
    for _ in range(args.warmup):
        run_oracle_sample(0, comps=[REFERENCE_SAMPLE[k % len(REFERENCE_SAMPLE)]])
        k += 1
    dofs, secs = 0, 0.0
    for _ in range(args.steps):
        r = run_oracle_sample(0, comps=[REFERENCE_SAMPLE[k % len(REFERENCE_SAMPLE)]])
        k += 1
        dofs += r["dofs"]
        secs += r["seconds"]
    value = dofs / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME},
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": "DoF/s", "cores": 1,
                         "sample": "per step: one component of the workload (cycling %s), assembly + sparse "
                                   "direct solve + evaluation on 17^3 points, FP64, one BLAS thread"
                                   % REFERENCE_SAMPLE},
        "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


class Workload:
    """Inputs of the perturbed-cube workload shared by every plan of the bench."""

    def __init__(self, sgiga, torch, stream):
        from paper_1707_09598_gb300.inputs import eval_points, lognormal_features, perturbed_cube_patch
        self.sg, self.torch, self.stream = sgiga, torch, stream
        self.kn, self.cp = perturbed_cube_patch(1)
        self.om, self.ph, self.amp = lognormal_features(2, nfeat=WORKLOAD["nfeat"])
        self.pts_h = eval_points(3, WORKLOAD["lattice"])
        self.pts = torch.as_tensor(self.pts_h, device="cuda")
        self.npts = len(self.pts_h)
        self.gold = np.loadtxt(GOLDEN)[:, 0]

    def plan(self, precision, precond, components=None, autotune=True, use_graph=True):
        """A plan with the coefficient set, the solver options of the workload
        (mixed plans: inner tolerance; set before the autotuner, whose probe
        solves use them) and (optionally) autotuned; returns (plan, set-up
        seconds, phase times, tuning)."""
        sg = self.sg
        t0 = time.perf_counter()
        kw = {} if components is None else {"components": components}
        P = sg.Plan(3, WORKLOAD["p"], WORKLOAD["w"], domain="patch", patch=([3, 3, 3], self.kn, self.cp),
                    precision=precision, precond=precond, stream=self.stream, **kw)
        sg.sgiga_set_coefficient(P.handle, self.om, self.ph, self.amp)
        if precision == "mixed":
            sg.sgiga_set_solver_options(P.handle, use_graph=use_graph, inner_tol=WORKLOAD["inner_tol"], inner_max=100)
        tune = sg.sgiga_autotune(P.handle, reps=2) if autotune else None
        return P, time.perf_counter() - t0, sg.sgiga_plan_times(P.handle), tune

    def combined(self, P):
        torch = self.torch
        uc = torch.zeros(P.info.ngrids * self.npts, dtype=torch.float64, device="cuda")
        self.sg.sgiga_eval(P.handle, self.pts, self.npts, uc)
        u = torch.zeros(self.npts, dtype=torch.float64, device="cuda")
        self.sg.sgiga_combine(P.handle, uc, self.npts, u)
        return u.cpu().numpy()

    def timed_solve(self, P, tol, maxit, reps=2):
        """Best of `reps` solves after one warm-up (CUDA events on the plan's stream)."""
        sg, torch = self.sg, self.torch
        sg.sgiga_solve(P.handle, tol, maxit, check=False)
        best, st = 1e30, None
        for _ in range(reps):
            e0, e1 = _events(torch)
            torch.cuda.synchronize()
            e0.record(self.stream)
            st, rc = sg.sgiga_solve(P.handle, tol, maxit, check=False)
            e1.record(self.stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return st, rc, best


def measure_comparators(W, args):
    """Plain per-grid FP64 PCG, batched FP64 PCG and mixed FD, each timed once
    (best of 2 after a warm-up) at the workload's tolerance, with the error of
    its combined values against the oracle. Returns (dict, mixed FD plan)."""
    sg, torch, tol = W.sg, W.torch, WORKLOAD["tol"]
    out = {}
    P, ps, pt, _ = W.plan("fp64", "fd")
    if args.host_loop:
        sg.sgiga_set_solver_options(P.handle, use_graph=False)
    sg.sgiga_set_rhs_builtin(P.handle, "one")
    st, rc, ms = W.timed_solve(P, tol, 2000)
    out["batched_fp64"] = {"ms": ms, "iterations": st.iterations, "rc": rc, "setup_s": ps,
                           "rel_l2_vs_oracle": _rel(W.combined(P), W.gold)}
    comps = [tuple(g.levels[:3]) for g in P.grids]
    coefs = [g.coeff for g in P.grids]
    P.close()
    # plain per-grid FP64 PCG: one plan per component, solved one after the other
    # on the stream with the host loop (no batching, no captured graph)
    t0 = time.perf_counter()
    singles = []
    for cl in comps:
        Q, _, _, _ = W.plan("fp64", "fd", components=[cl], autotune=False)
        sg.sgiga_set_rhs_builtin(Q.handle, "one")
        sg.sgiga_set_solver_options(Q.handle, use_graph=False)
        singles.append(Q)
    setup_s = time.perf_counter() - t0
    for Q in singles[:4]:
        sg.sgiga_solve(Q.handle, tol, 2000, check=False)
    e0, e1 = _events(torch)
    torch.cuda.synchronize()
    e0.record(W.stream)
    its = 0
    for Q in singles:
        st, _ = sg.sgiga_solve(Q.handle, tol, 2000, check=False)
        its = max(its, st.iterations)
    e1.record(W.stream)
    torch.cuda.synchronize()
    acc = np.zeros(W.npts)
    for Q, c in zip(singles, coefs):
        uq = torch.zeros(W.npts, dtype=torch.float64, device="cuda")
        sg.sgiga_eval(Q.handle, W.pts, W.npts, uq)
        acc += c * uq.cpu().numpy()
        Q.close()
    out["per_grid_fp64"] = {"ms": e0.elapsed_time(e1), "iterations": its, "plans": len(singles),
                            "setup_s": setup_s, "rel_l2_vs_oracle": _rel(acc, W.gold)}
    # mixed: FP32 inner FD-CG in FP64 refinement
    M, ps, pt, mt = W.plan("mixed", "fd", use_graph=not args.host_loop)
    sg.sgiga_set_rhs_builtin(M.handle, "one")
    st, rc, ms = W.timed_solve(M, tol, 50)
    out["mixed_fd"] = {"ms": ms, "outer": st.iterations, "inner": st.inner_iterations, "rc": rc, "setup_s": ps,
                       "plan_phases_s": pt, "rel_l2_vs_oracle": _rel(W.combined(M), W.gold),
                       "solve_precision": "fp64" if mt.solve_precision == 0 else "mixed",
                       "probe_solve_ms": {"fp64": mt.solve_ms_fp64, "fp64_fd32": mt.solve_ms_fp64_fd32,
                                          "mixed": mt.solve_ms_mixed}}
    return out, M


def train_learned(W, args):
    """The learned plan: set-up, the network trained on the plan's own CG
    pairs, and its solve. Returns (plan, dict, tuning)."""
    sg = W.sg
    L, ps, pt, tune = W.plan("mixed", "learned", use_graph=not args.host_loop)
    t0 = time.perf_counter()
    sg.sgiga_net_init(L.handle, 11)
    tr = sg.sgiga_train_net(L.handle, target_pairs=10000, max_iter_record=30, epochs=12, lr=5e-4, seed=100,
                            batch=2)
    train_s = time.perf_counter() - t0
    sg.sgiga_set_rhs_builtin(L.handle, "one")
    st, rc, ms = W.timed_solve(L, WORKLOAD["tol"], 50)
    out = {"ms": ms, "outer": st.iterations, "inner": st.inner_iterations, "rc": rc, "fallback": st.fallback,
           "setup_s": ps, "plan_phases_s": pt, "rel_l2_vs_oracle": _rel(W.combined(L), W.gold),
           "training": {"seconds": train_s, "pairs": tr.pairs, "samples": tr.samples, "adam_steps": tr.steps,
                        "loss_fd": tr.loss_fd, "loss_initial": tr.loss_initial,
                        "loss_epochs": [tr.loss_epoch[e] for e in range(min(12, 32))],
                        "best_epoch": tr.best_epoch, "log_s_range": [tr.logs_min, tr.logs_max],
                        "validation_inner_iterations": {"initial": tr.val_iters_initial, "kept": tr.val_iters_best}}}
    tuning = {"best": {"smem_budget": tune.budget[tune.best], "qp_cap": tune.qpcap[tune.best],
                       "threads": tune.nthreads[tune.best], "l2_prefetch_bytes_per_plane": tune.best_prefetch,
                       "apply_f32_ms": tune.best_ms, "ntiles": tune.ntiles},
              "candidates_ms": {"%d/%d/%d/%d" % (tune.budget[i], tune.qpcap[i], tune.nthreads[i], tune.prefetch[i]):
                                round(tune.ms[i], 4) for i in range(tune.ncand)},
              "precond": {"best_ks": tune.fd_ks[tune.fd_best],
                          "layout": "grouped" if tune.fd_grouped[tune.fd_best] else "per piece"}}
    return L, out, tuning


def network_free_scaling(W, L):
    """The learned plan with S = c^(-1/2) (no network), then the network's S restored."""
    sg, torch = W.sg, W.torch
    params = sg.sgiga_net_get_params(L.handle)
    phi = torch.zeros(L.info.ndof, dtype=torch.float32, device="cuda")
    sg.sgiga_net_features(L.handle, phi)
    sg.sgiga_net_set_scaling(L.handle, torch.exp(-0.5 * phi).contiguous())
    st, rc, ms = W.timed_solve(L, WORKLOAD["tol"], 50)
    out = {"ms": ms, "outer": st.iterations, "inner": st.inner_iterations, "rc": rc,
           "rel_l2_vs_oracle": _rel(W.combined(L), W.gold)}
    sg.sgiga_net_set_params(L.handle, params)
    return out


def cube_line(sgiga, torch, stream, steps, peak=None):
    """The FP64 unit-cube workload (w = 10): step = load vector + batched FD-PCG
    to 1e-12 + eval + combine; its FP64 operator apply against the FP64 rate
    (cuBLAS DGEMM, measured here)."""
    from paper_1707_09598_gb300.inputs import eval_points
    C = CUBE
    P = sgiga.Plan(C["d"], C["p"], C["w"], domain="unit", stream=stream)
    sgiga.sgiga_autotune(P.handle, reps=3)
    pts_h = eval_points(3, C["lattice"])
    npts = len(pts_h)
    pts = torch.as_tensor(pts_h, device="cuda")
    uc = torch.zeros(P.info.ngrids * npts, dtype=torch.float64, device="cuda")
    u = torch.zeros(npts, dtype=torch.float64, device="cuda")
    f = torch.zeros(P.info.nqp, dtype=torch.float64, device="cuda")
    sgiga.sgiga_source_at_qp(P.handle, "sine", f)

    def step():
        sgiga.sgiga_set_rhs(P.handle, f)
        sgiga.sgiga_solve(P.handle, C["tol"], 50)
        sgiga.sgiga_eval(P.handle, pts, npts, uc)
        sgiga.sgiga_combine(P.handle, uc, npts, u)

    for _ in range(3):
        step()
    e0, e1 = _events(torch)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    l2 = _rel(u.cpu().numpy(), np.loadtxt(CUBE_GOLDEN)[:, 0])
    x = torch.randn(P.info.ndof, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    for _ in range(3):
        sgiga.sgiga_apply(P.handle, x, y)
    a0, a1 = _events(torch)
    torch.cuda.synchronize()
    a0.record(stream)
    for _ in range(20):
        sgiga.sgiga_apply(P.handle, x, y)
    a1.record(stream)
    torch.cuda.synchronize()
    apply_s = a0.elapsed_time(a1) / 20 / 1e3
    flops = apply_flops(P)
    peak = peak if peak else fp64_peak_tflops(torch)
    # the same step on a MIXED plan: its autotuner times the mixed solve against
    # FP64 PCG (FD is exact on the cube) and keeps the faster
    M = sgiga.Plan(C["d"], C["p"], C["w"], domain="unit", stream=stream, precision="mixed")
    sgiga.sgiga_set_rhs(M.handle, f)
    mt = sgiga.sgiga_autotune(M.handle, reps=3)
    ucm = torch.zeros_like(uc)
    um = torch.zeros_like(u)

    def step_m():
        sgiga.sgiga_set_rhs(M.handle, f)
        sgiga.sgiga_solve(M.handle, C["tol"], 50)
        sgiga.sgiga_eval(M.handle, pts, npts, ucm)
        sgiga.sgiga_combine(M.handle, ucm, npts, um)

    for _ in range(3):
        step_m()
    m0, m1 = _events(torch)
    torch.cuda.synchronize()
    m0.record(stream)
    for _ in range(steps):
        step_m()
    m1.record(stream)
    torch.cuda.synchronize()
    mixed_plan = {"solve_precision": "fp64" if mt.solve_precision == 0 else "mixed",
                  "fp32_preconditioner": bool(mt.solve_fp32_precond),
                  "ms_per_step": m0.elapsed_time(m1) / steps,
                  "probe_solve_ms": {"fp64": mt.solve_ms_fp64, "fp64_fd32": mt.solve_ms_fp64_fd32,
                                     "mixed": mt.solve_ms_mixed},
                  "rel_l2_vs_oracle": _rel(um.cpu().numpy(), np.loadtxt(CUBE_GOLDEN)[:, 0])}
    M.close()
    out = {"workload": CUBE_NAME, "value": P.info.ndof / (ms / 1e3), "unit": "DoF/s", "ms_per_step": ms,
           "dtype": "f64", "rel_l2_vs_oracle": l2, "target": 1e-10,
           "apply_fp64": {"ms": apply_s * 1e3, "algorithmic_flops": flops, "TFLOPs": flops / apply_s / 1e12,
                          "fp64_peak_TFLOPs": peak, "frac": flops / apply_s / 1e12 / peak,
                          "peak_source": "measured cuBLAS DGEMM 8192^3 on this GPU"},
           "mixed_plan": mixed_plan}
    P.close()
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1707_09598_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    from paper_1707_09598_gb300 import sgiga

    stream = torch.cuda.Stream()
    # torch's fills and reads of the buffers handed to the plans run on the
    # plans' stream, in order with their calls
    torch.cuda.set_stream(stream)
    W = Workload(sgiga, torch, stream)
    tol = WORKLOAD["tol"]
    comparison = {}
    if not args.quick:
        comparison, M = measure_comparators(W, args)
    else:
        M, _, _, _ = W.plan("mixed", "fd", use_graph=not args.host_loop)
        sgiga.sgiga_set_rhs_builtin(M.handle, "one")
        st, rc, ms = W.timed_solve(M, tol, 50)
        comparison["mixed_fd"] = {"ms": ms, "outer": st.iterations, "inner": st.inner_iterations, "rc": rc}
    L, comparison["learned_mixed"], tuning = train_learned(W, args)
    if not args.quick:
        comparison["scaled_no_network"] = network_free_scaling(W, L)
    # the headline path: the faster of mixed FD and learned + mixed, at the tolerance
    use_learned = (comparison["learned_mixed"]["rc"] == 0 and
                   comparison["learned_mixed"]["ms"] <= comparison["mixed_fd"]["ms"])
    P = L if use_learned else M
    (M if use_learned else L).close()
    if "per_grid_fp64" in comparison:
        pg = comparison["per_grid_fp64"]["ms"]
        for k, v in comparison.items():
            if k != "per_grid_fp64":
                v["speedup_vs_per_grid_fp64"] = pg / v["ms"]
    ndof, ng, nqp, npts = P.info.ndof, P.info.ngrids, P.info.nqp, W.npts
    uc = torch.zeros(ng * npts, dtype=torch.float64, device="cuda")
    u = torch.zeros(npts, dtype=torch.float64, device="cuda")
    f_dev = torch.ones(nqp, dtype=torch.float64, device="cuda")     # f = 1 at every quadrature point
    stats = []

    def step():
        # an NVTX range per step, so that a profiler's launch list can be
        # restricted to the steps (ncu --nvtx --nvtx-include bench_step/)
        torch.cuda.nvtx.range_push("bench_step")
        sgiga.sgiga_set_rhs(P.handle, f_dev)
        st, _ = sgiga.sgiga_solve(P.handle, tol, 50)
        stats.append(st)
        sgiga.sgiga_eval(P.handle, W.pts, npts, uc)
        sgiga.sgiga_combine(P.handle, uc, npts, u)
        torch.cuda.nvtx.range_pop()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clock_sampler(torch, local)
    clocks.start()
    l0 = sgiga.sgiga_launch_count()
    e0, e1 = _events(torch)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = sgiga.sgiga_launch_count() - l0
    ck = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    if world > 1:
        torch.distributed.barrier()
    value = whole_job_rate(ndof, world, ms / 1e3)
    l2 = _rel(u.cpu().numpy(), W.gold)

    # per-phase times (one extra step, events between the calls)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    sgiga.sgiga_set_rhs(P.handle, f_dev)
    ev[1].record(stream)
    sgiga.sgiga_solve(P.handle, tol, 50)
    ev[2].record(stream)
    sgiga.sgiga_eval(P.handle, W.pts, npts, uc)
    sgiga.sgiga_combine(P.handle, uc, npts, u)
    ev[3].record(stream)
    torch.cuda.synchronize()
    phases = {"rhs_ms": ev[0].elapsed_time(ev[1]), "solve_ms": ev[1].elapsed_time(ev[2]),
              "eval_combine_ms": ev[2].elapsed_time(ev[3])}

    # dominant kernel of the mixed path: the FP32 operator apply, timed alone
    x = torch.randn(ndof, dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    for _ in range(3):
        sgiga.sgiga_apply_f32(P.handle, x, y)
    reps = 20
    a0, a1 = _events(torch)
    torch.cuda.synchronize()
    a0.record(stream)
    for _ in range(reps):
        sgiga.sgiga_apply_f32(P.handle, x, y)
    a1.record(stream)
    torch.cuda.synchronize()
    apply_s = a0.elapsed_time(a1) / reps / 1e3
    nplanes = 3 if P.info.diag_metric else 6
    g_bytes = nplanes * 4 * nqp + 2 * 4 * ndof
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    roofline = {"bound": "hbm", "achieved": g_bytes / apply_s / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": g_bytes / apply_s / 1e9 / hbm, "traffic": APPLY_F32_DRAM_BYTES,
                "kernel": "k_op3<float,3,0,false> (FP32 sum-factorised stiffness apply, general metric)",
                "apply_ms": apply_s * 1e3, "algorithmic_bytes": g_bytes,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"}

    # the refinement's FP64 residual apply (the largest time share of the
    # solve), against the FP64 rate measured here (cuBLAS DGEMM)
    fp64_peak = fp64_peak_tflops(torch)
    xd = torch.randn(ndof, dtype=torch.float64, device="cuda")
    yd = torch.zeros_like(xd)
    for _ in range(3):
        sgiga.sgiga_apply(P.handle, xd, yd)
    d0, d1 = _events(torch)
    torch.cuda.synchronize()
    d0.record(stream)
    for _ in range(10):
        sgiga.sgiga_apply(P.handle, xd, yd)
    d1.record(stream)
    torch.cuda.synchronize()
    apply64_s = d0.elapsed_time(d1) / 10 / 1e3
    flops64 = apply_flops(P)
    roofline_fp64 = {"bound": "alu", "achieved": flops64 / apply64_s / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": flops64 / apply64_s / 1e12 / fp64_peak, "traffic": None,
                     "kernel": "k_op3<double,3,0,false> (FP64 residual apply of the refinement, general metric)",
                     "apply_ms": apply64_s * 1e3, "algorithmic_flops": flops64,
                     "peak_source": "measured cuBLAS DGEMM 8192^3 on this GPU"}

    # end to end through the C ABI with host buffers (pinned): f, points in; u out
    f_h = torch.ones(nqp, dtype=torch.float64).pin_memory()
    pts_pin = torch.as_tensor(W.pts_h).pin_memory()
    u_pin = torch.zeros(npts, dtype=torch.float64).pin_memory()
    f_np, pts_np, u_np = f_h.numpy(), pts_pin.numpy(), u_pin.numpy()

    def step_e2e():
        sgiga.sgiga_set_rhs(P.handle, f_np)
        sgiga.sgiga_solve(P.handle, tol, 50)
        sgiga.sgiga_eval(P.handle, pts_np, npts, uc)
        sgiga.sgiga_combine(P.handle, uc, npts, u_np)

    step_e2e()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world, "cuda")
    l2_e2e = _rel(u_np, W.gold)
    setup = {"headline_plan_s": comparison["learned_mixed"]["setup_s"] if use_learned
             else comparison["mixed_fd"].get("setup_s"),
             "headline_plan_phases_s": sgiga.sgiga_plan_times(P.handle)}
    if use_learned:
        setup["training_s"] = comparison["learned_mixed"]["training"]["seconds"]
    setup["setup_plus_solve_s"] = (setup["headline_plan_s"] or 0.0) + setup.get("training_s", 0.0) + \
        phases["solve_ms"] / 1e3
    P.close()
    del f_h, pts_pin, u_pin
    torch.cuda.synchronize()

    cube = None if args.quick else cube_line(sgiga, torch, stream, 10, peak=fp64_peak)
    cpu = cpu_par = None
    if rank == 0 and not args.quick:
        r = run_oracle_sample(0)
        cpu = {"value": r["dofs"] / r["seconds"], "unit": "DoF/s", "cores": 1, "kind": "oracle",
               "sample": "%d components of the workload %s: assembly + sparse direct solve + evaluation "
                         "on 17^3 points, FP64, one BLAS thread, %.1f s" % (len(ORACLE_SAMPLE), ORACLE_SAMPLE,
                                                                            r["seconds"])}
        rp = run_oracle_sample(1, parallel=True)
        cpu_par = {"value": rp["dofs"] / rp["seconds"], "unit": "DoF/s", "cores": rp["cores"], "kind": "oracle",
                   "sample": "%d components (the serial sample's, one per core) over a spawned pool of %d "
                             "one-thread workers in LPT order (the paper's parallelisation), %.1f s"
                             % (rp["components"], rp["cores"], rp["seconds"])}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 inner solve, f64 residual/combination", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "ngrids": ng, "ndof": ndof, "nqp": nqp, "eval_points": npts,
                       "path": "learned + mixed" if use_learned else "mixed FD",
                       "inner_tol": WORKLOAD["inner_tol"],
                       "parallelism": "replica per GPU" if world > 1 else "single GPU",
                       "l2_policy": "inputs larger than L2 (FP32 geometry planes %.2f GB per inner apply)"
                                    % (nplanes * 4 * nqp / 1e9),
                       "cg_loop": "host loop" if args.host_loop else "captured graph with device-side while"},
            "accuracy": {"rel_l2_vs_oracle": l2, "rel_l2_vs_oracle_e2e": l2_e2e, "target": 1e-8,
                         "outer_iterations": max(s.iterations for s in stats),
                         "inner_iterations": max(s.inner_iterations for s in stats)},
            "phases_ms": phases, "setup": setup, "autotune": tuning, "comparison": comparison,
            "roofline": roofline, "roofline_fp64_residual": roofline_fp64,
            "cpu_baseline": cpu, "cpu_baseline_parallel": cpu_par,
            "e2e": {"value": whole_job_rate(ndof, world, e2e_s), "unit": "DoF/s",
                    "h2d_bytes_per_step": int(nqp * 8 + npts * 3 * 8), "d2h_bytes_per_step": int(npts * 8)},
            "gpu_launches": int(launches), "clocks": ck, "cube_fp64": cube,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.oracle_list:
        oracle_sample_child([tuple(int(v) for v in c.split(",")) for c in args.oracle_list.split(";")])
        return 0
    if args.oracle_parallel:
        oracle_parallel_child(args.oracle_parallel)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
