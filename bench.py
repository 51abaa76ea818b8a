"""Benchmark of the sparse-GP (GAP) fit on GB300: design rows per second of the
whole fit (assemble -> factor -> solve -> predict) on workload 2, the synthetic
stand-in for the paper's training sets (2000 configurations of 16-128 atoms,
d=512, M=4000, zeta=4, three force rows per atom; 441,968 design rows).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed_bf16]
                    [--impl ours|reference] [--fp64-steps 1] [--no-cpu-baseline]

One JSON line on stdout (rank 0).  `value` is device-timed with inputs resident
in HBM; `e2e` repeats the step through the C-ABI with pinned host buffers
(host-to-device copies and the read-back of c and the predictions inside the
timed region; the predictions are for the assembled problem, from its device
copies, so the inputs cross the host link once per step).  Several GPUs run independent replicas of the fit (the fit of
one problem is not sharded across GPUs here).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fit wall time and design rows/s, mixed vs FP64 on one GB300 at 1e-6 rel error"
UNIT = "design rows/s"
WORKLOAD = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed_bf16", choices=["mixed_bf16", "mixed_tf32", "mixed_fp16", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the plain FP64 GPU path (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--max-cfg", type=int, default=0,
                    help="profile a slice: the first N configurations of the workload, full sparse set")
    ap.add_argument("--force-walk", type=int, default=0,
                    help="consecutive tiles per step of the tensor-core force pass's tile walk (0: the library default)")
    ap.add_argument("--no-cur", action="store_true", help="skip the timing of the CUR choice of the sparse set")
    ap.add_argument("--no-other-precisions", action="store_true",
                    help="skip the timing of the other mixed precisions on the same inputs")
    ap.add_argument("--other-steps", type=int, default=3, help="timed steps of each other mixed precision")
    ap.add_argument("--host-register", type=int, default=0,
                    help="workload 5: page-lock J and X in place with cudaHostRegister (0: leave them pageable)")
    ap.add_argument("--j-ring-direct", type=int, default=0,
                    help="workload 5: the kernels read the page-locked host J in place (0: copies through FP64 slots)")
    ap.add_argument("--tol", type=float, default=0.0, help="option tol of the refinement (0: the library default)")
    ap.add_argument("--tsqr-shards", type=int, default=0,
                    help="factor the data rows as up to this many row blocks merged by a TSQR (0: one QR)")
    ap.add_argument("--autotune", default=None, metavar="CACHE",
                    help="workload 4: pick the fits in flight with the schedule autotuner before the "
                         "warm-up (a JSON cache file, or 'mem' for no file)")
    ap.add_argument("--workload", type=int, default=2, choices=[2, 4, 5],
                    help="4: the 64-fit sweep through one gap_fit_batched call per step (not the headline)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle samples taken during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(torch, device, max_cfg=0):
    """Workload 2 inputs: device tensors, pinned host tensors (e2e) and targets.
    max_cfg > 0 keeps the first max_cfg configurations (profiling slices)."""
    import gapgen
    import paper_2207_03803_gb300 as g
    r = gapgen.RECIPES[WORKLOAD]
    if max_cfg > 0:
        p = gapgen.make_problem(r, max_cfg=max_cfg)
        y = gapgen.load_targets_slice(p, WORKLOAD)
        J_pin = torch.from_numpy(p.J).pin_memory()
    else:
        n_atoms, n_pairs = gapgen.count_shape(r)
        J_pin = torch.empty((n_pairs, 3, r.d), dtype=torch.float64).pin_memory()
        p = gapgen.make_problem(r, J_out=J_pin.numpy())
        y = gapgen.load_targets(p, WORKLOAD)
    sigma = np.concatenate([p.sigma_e, p.sigma_f])
    host = {"cfg_ptr": p.cfg_ptr, "X": p.X, "Xs": p.Xs, "y": y, "sigma": sigma, "pair_ptr": p.pair_ptr,
            "pair_src": p.pair_src}
    pinned = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in host.items()}
    pinned["J"] = J_pin
    dev = {k: v.to(device, non_blocking=True) for k, v in pinned.items()}
    torch.cuda.synchronize()
    kw = dict(delta=r.delta, zeta=r.zeta, jitter=r.jitter)
    prob_dev = g.Problem(memory=g.GAP_MEM_DEVICE, **kw, **dev)
    prob_host = g.Problem(memory=g.GAP_MEM_HOST, **kw, **pinned)
    h2d = sum(int(t.numel() * t.element_size()) for t in pinned.values())
    return p, prob_dev, prob_host, h2d


ORACLE_FIT = os.path.join(ROOT, "tests", "golden", "workload2_oracle_fit.npz")
W5_ROWS = os.path.join(ROOT, "tests", "golden", "workload5_sampled_rows.npz")


def oracle_record(p):
    """The FP64 oracle's fit of the whole workload 2 (weights, every prediction, phase times
    and the machine it ran on), stored by tests/golden/make_workload2_fit.py; None for
    other inputs (a profiling slice) or when it has not been recorded."""
    import gapgen
    if not os.path.exists(ORACLE_FIT) or p.n_cfg != gapgen.RECIPES[WORKLOAD].n_cfg:
        return None
    z = np.load(ORACLE_FIT)
    if str(z["fingerprint"]) != gapgen.fingerprint(p):
        return None
    return z


def accuracy(rec, c, E, F):
    """Relative L2 errors of the weights and of the fitted model's predictions (energies,
    forces) against the oracle's full fit."""
    if rec is None:
        return None
    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"c": rel(c.cpu().numpy(), rec["c"]), "E": rel(E.cpu().numpy(), rec["E"]),
            "F": rel(F.cpu().numpy(), rec["F"]), "reference": "FP64 oracle fit of the full workload"}


def h2d_alone_ms(torch, prob_host, dev, stream, reps=2):
    """Device time of copying a host problem's pinned arrays to the device on their own
    (CUDA events on the copying stream), the best of a few repetitions."""
    src = [t for t in prob_host._keep if t is not None and hasattr(t, "is_pinned")]
    dst = [torch.empty_like(t, device=dev) for t in src]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(reps):
        torch.cuda.synchronize()
        ev0.record(stream)
        for d_, s_ in zip(dst, src):
            d_.copy_(s_, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        best = ms if best is None else min(best, ms)
    del dst
    return best


def fit_step(ctx, prob, c, E, F):
    """assemble + factor + solve + predict; the predictions are for the assembled
    problem, from its device copies (a host problem is copied to the device once)."""
    ctx.assemble(prob)
    ctx.factor()
    info = ctx.solve(c)
    ctx.predict(None, c, E, F)
    return info


def profile_traffic(kernel_src, per_unit_key):
    """DRAM traffic per unit recorded in a committed ncu summary under profiles/,
    if it was taken on the kernel source as it stands (sha256 prefix match)."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "paper_2207_03803_gb300", "csrc", kernel_src)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    pdir = os.path.join(here, "profiles")
    for fn in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        txt = open(os.path.join(pdir, fn)).read()
        if ("source_sha256_prefix: %s" % sha) in txt and per_unit_key in txt:
            for line in txt.splitlines():
                if line.strip().startswith(per_unit_key + ":"):
                    return float(line.split(":", 1)[1].split()[0]), fn
    return None, None


ASSEMBLY_PHASES = ("copy_in", "pack", "gemm_energy", "gemm_force")


def assembly_rate(phase_ms, n_rows):
    """Design rows per second of the assembly alone: the data rows over the device time per
    step of the kernel classes gap_assemble runs (staging of host inputs, packing, the energy
    and force passes).  The line's value divides the same rows by the whole step."""
    ms = sum(float(phase_ms.get(k, 0.0)) for k in ASSEMBLY_PHASES)
    return {"ms": round(ms, 3), "rows_per_s": n_rows / (ms * 1e-3) if ms > 0 else None,
            "phases": [k for k in ASSEMBLY_PHASES if float(phase_ms.get(k, 0.0)) > 0]}


def roofline(prof, p, precision, pk, step_ms, iterations):
    """Roofline of the kernel class with the largest device time per step."""
    cls = max(("gemm_force", "gemm_energy", "qr_update", "qr_panel", "refine", "predict", "pack", "kmm_chol"),
              key=lambda k: prof[k]["ms"])
    ms = prof[cls]["ms"]
    groups = max(prof[cls]["groups"], 1)
    M, d, N = p.n_sparse, p.d, p.n_rows
    rows = N + M
    out = {"kernel": cls, "share_of_step": ms / step_ms if step_ms else None}
    if cls in ("gemm_force", "gemm_energy"):
        R = 3 * p.n_pairs if cls == "gemm_force" else p.n_atoms
        flop = 2.0 * R * M * d  # one contraction per (row, sparse point): the method's products
        if precision == "mixed_tf32":
            peak = pk["bf16_tflops"] * 0.5
            note = "TF32 dense peak = measured BF16 burst peak x nominal TF32/BF16 ratio 1/2; 3 MMA passes"
        elif precision == "mixed_bf16":
            peak = pk["bf16_tflops"]
            note = "measured BF16 burst peak; 6 MMA passes (three-slice split products)"
        elif precision == "mixed_fp16" and cls == "gemm_force":
            peak = pk["bf16_tflops"]
            note = ("FP16 dense peak = measured BF16 burst peak (the same tensor-core rate); 3 MMA passes "
                    "(scaled two-slice FP16 split products)")
        elif precision == "mixed_fp16":
            peak = pk["bf16_tflops"]
            note = "measured BF16 burst peak; 6 MMA passes (three-slice split products)"
        else:
            peak = 152 * 2 * 2 * 2.07e9 / 1e12  # FP64 SIMT: 2 DFMA/clk/SM (GB300), max clock
            note = "FP64 ALU peak derived from unit counts"
        achieved = flop / (ms / groups * 1e-3) / 1e12
        traffic, src = (None, None)
        if cls == "gemm_force" and precision in ("mixed_bf16", "mixed_fp16"):
            key = "dram_bytes_per_jacobian_row" + ("_fp16" if precision == "mixed_fp16" else "")
            per_row, src = profile_traffic("k_tc.cu", key)
            traffic = per_row * R if per_row is not None else None
        out.update({"bound": "tensor" if precision != "fp64" else "alu", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic, "peak_note": note,
                    "algorithmic_flop_per_launch": flop, "algorithmic_unit": "2 d M flop per Jacobian row",
                    "traffic_source": src})
    elif cls in ("qr_update", "qr_panel"):
        # two-level QR, outer panels of 128 applied with plain-TF32 tensor-core GEMMs: each
        # outer panel reads the trailing columns once (Y = V^T C) and reads + writes them
        # once (C -= V W2): 12 bytes per (row, trailing column) per outer panel
        nbo = 128
        bytes_ = sum(12.0 * (rows - k0) * (M + 1 - min(M, k0 + nbo)) for k0 in range(0, M, nbo))
        achieved = bytes_ / (ms * 1e-3) / 1e9
        out.update({"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"], "traffic": None,
                    "peak_note": "algorithmic bytes of the outer trailing updates over the phase's time"})
    elif cls == "refine":
        # one fused pass over the FP32 residual matrix per CGLS iteration, plus the two
        # true-residual passes
        bytes_ = (iterations + 2) * rows * M * 4.0
        achieved = bytes_ / (ms * 1e-3) / 1e9
        out.update({"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"], "traffic": None})
    else:
        out.update({"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None})
    return out


def cpu_baseline(budget_s=25.0):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of
    workload 2 extrapolated to the whole fit by its operation counts."""
    import gapgen
    import oracle
    r = gapgen.RECIPES[WORKLOAD]
    n_atoms, n_pairs = gapgen.count_shape(r)
    N = r.n_cfg + 3 * n_atoms
    M = sum(r.n_sparse)
    cores = os.cpu_count()
    # (1) assembly of the first configurations at full M and d
    p = gapgen.make_problem(r, max_cfg=4)
    t0 = time.time()
    D = oracle.design(p)
    t_asm = time.time() - t0
    asm_rate = D.shape[0] / t_asm  # design rows per second
    # (2) Householder QR of a tall block with M' columns, scaled by (M/M')^2 per row; the
    # block (134 MB) exceeds the host caches, as the full fit's 14 GB matrix does (a
    # 4096 x 1024 block ran 24 % faster per flop than the full QR on the same cores)
    Mp = 1024
    rng = np.random.default_rng(0)
    B = rng.standard_normal((16 * Mp, Mp))
    t0 = time.time()
    oracle.householder_qr(B)
    t_qr = time.time() - t0
    qr_flop = 2.0 * B.shape[0] * Mp ** 2 - 2.0 / 3 * Mp ** 3
    qr_rate = qr_flop / t_qr
    full_qr_flop = 2.0 * (N + M) * M ** 2 - 2.0 / 3 * M ** 3
    est = N / asm_rate + full_qr_flop / qr_rate
    return {"value": N / est, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "oracle design rows of workload-2 configurations 0-3 (%d rows at M=%d, d=%d: %.1f s) and "
                      "Householder QR of a %dx%d block (%.1f s), extrapolated to the %d-row fit by operation count"
                      % (D.shape[0], M, r.d, t_asm, B.shape[0], Mp, t_qr, N),
            "est_fit_s": est}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import gapgen
    n_atoms, _ = gapgen.count_shape(gapgen.RECIPES[WORKLOAD])
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(budget_s=5.0)
    t0 = time.time()
    for _ in range(args.steps):
        vals.append(cpu_baseline())
    wall = time.time() - t0
    v = float(np.median([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator; paper datasets not available)",
            "config": {"workload": "workload 2: 2000 configurations, d=512, M=4000, zeta=4, energies+forces",
                       "method": "FP64 CPU oracle, bounded sample extrapolated by operation count"},
            "cpu_baseline": {k: vals[-1][k] for k in ("kind", "cores", "sample")} | {"value": v, "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """Workload 4: the seeded 64-fit sweep (d = 256; rows, M, zeta and sigma_E varying per
    fit), device-resident, fitted through one gap_fit_batched call per step.  With N
    ranks, whole fits are placed by greedy LPT (no exchange between ranks).  Prints one
    JSON line: design rows of all fits per second of the slowest rank's batched call."""
    import torch
    import gapgen
    import paper_2207_03803_gb300 as g
    g.build()
    g.load()
    import torch.distributed as dist
    from paper_2207_03803_gb300.sharding import fit_cost, lpt_assign
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    recs = gapgen.sweep_recipes()
    # whole fits per rank by greedy LPT on the estimated cost (no exchange between ranks);
    # the row counts come from the recipes' configuration sizes, drawn without the problems
    shape = [gapgen.count_shape(r) for r in recs]
    costs = [fit_cost(r.n_cfg + 3 * na, r.n_sparse[0]) for r, (na, _) in zip(recs, shape)]
    mine = lpt_assign(costs, world)[rank]
    probs, outs, rows, t0 = [], [], 0, time.time()
    for f in mine:
        p = gapgen.make_problem(recs[f])
        y = gapgen.load_sweep_targets(p, f)
        probs.append(g.problem_from_arrays(p, y, device="cuda"))
        outs.append(torch.empty(p.n_sparse, dtype=torch.float64, device=dev))
        rows += p.n_rows  # data rows, as the single-fit line counts them
    gen_s = time.time() - t0
    ctx = g.Context(args.precision)
    lanes = 4  # the library's default
    if args.autotune:
        from paper_2207_03803_gb300 import autotune
        cache = autotune.TuneCache(None if args.autotune == "mem" else args.autotune)
        lanes = int(autotune.tune_batched(ctx, probs, outs, cache)["batch_lanes"])
    for _ in range(max(args.warmup, 1)):
        infos = ctx.fit_batched(probs, outs)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    t = time.perf_counter()
    for _ in range(args.steps):
        infos = ctx.fit_batched(probs, outs)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = (time.perf_counter() - t) * 1e3 / args.steps
    clocks = sampler.stop()
    tot = torch.tensor([ms, float(rows), float(sum(1 for i in infos if i["converged"]))], dtype=torch.float64,
                       device=dev)
    if world > 1:
        mx = tot[:1].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        tot[0] = mx[0]
    ms, rows, n_conv = float(tot[0]), int(tot[1]), int(tot[2])
    if rank != 0:
        return
    out = {"metric": "design rows/s over a batched sweep of independent fits", "value": rows / (ms * 1e-3),
           "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
           "data": "synthetic (seeded generator)",
           "config": {"workload": "workload 4: 64 independent fits, rows ~ logU[2k, 40k], M ~ logU[200, 2000], "
                                  "d=256, zeta in {2,3,4}, sigma_E in {1e-4,1e-3,1e-2}; gap_fit_batched "
                                  "(assemble + factor + solve per fit, %d worker lanes%s)"
                                  % (lanes, ", picked by the autotuner" if args.autotune else ""),
                      "precision": args.precision, "fits": len(recs), "design_rows": rows,
                      "parallelism": "whole fits per GPU by greedy LPT" if world > 1 else "single GPU",
                      "timing": "host wall clock around the batched call (it synchronises), max over ranks"},
           "converged": n_conv, "generation_s": gen_s, "clocks": clocks}
    print(json.dumps(out))


RING_ROWS_W5 = 128 * 4096  # J ring of the workload-5 fit: 172,032 pairs (4.2 GB of FP64 J) per chunk


def host_mem_available():
    """MemAvailable of this host in bytes (0 if unknown)."""
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


def run_workload5(args):
    """Workload 5 at full size: 6000 configurations of 16-96 atoms in three species
    (335,097 atoms, 5,365,085 pairs), d = 1024, M = 5334 + 5333 + 5333 = 16,000 sparse
    points, 1,011,291 data rows.  Its 132 GB of FP64 Jacobians stay in host memory (pageable
    by default; --host-register 1 page-locks them in place) and reach the force pass through the J ring (option
    "j_ring_rows"); the design matrices, W and the factors fit in HBM.  A step is one fit
    (assemble + factor + solve) and the fitted model's predictions of the problem (its
    design rows times c: the Jacobians are not on the device; the predictions from the
    descriptors, J through the ring again, are timed once beside it); device-timed with
    CUDA events, so the host-to-device copies of J are inside it.  Checks at this size: design rows of sampled configurations against the
    oracle, the fit's normalised residual, and the other mixed precisions' fits against
    this one.  Prints one JSON line; one process only."""
    import torch
    import gapgen
    import paper_2207_03803_gb300 as g
    world = int(os.environ.get("WORLD_SIZE", "1"))
    base = {"metric": METRIC + " (workload 5 at full size)", "unit": UNIT, "impl": "ours"}
    if world > 1:
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(dict(base, unavailable="workload 5 holds 136 GB of host memory per fit: one process only")))
        return
    r = gapgen.RECIPES[5]
    n_atoms, n_pairs = gapgen.count_shape(r)
    need = (n_pairs * 3 + n_atoms) * r.d * 8 + 16e9
    avail = host_mem_available()
    if avail < need:
        print(json.dumps(dict(base, unavailable="workload 5 needs %.0f GB of host memory, %.0f GB available"
                                                % (need / 1e9, avail / 1e9))))
        return
    g.build()
    g.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    p = gapgen.make_problem(r)
    y = gapgen.load_targets(p, 5)
    gen_s = time.time() - t0
    # optionally page-lock the Jacobians and descriptors where they are
    cudart = torch.cuda.cudart()
    t0 = time.time()
    pinned = args.host_register and int(cudart.cudaHostRegister(p.J.ctypes.data, p.J.nbytes, 0)) == 0
    pinned_x = args.host_register and int(cudart.cudaHostRegister(p.X.ctypes.data, p.X.nbytes, 0)) == 0
    pin_s = time.time() - t0
    prob = g.problem_from_arrays(p, y, device="cpu")
    N, M = p.n_rows, p.n_sparse
    rows = N  # the data rows of the design matrix, as in the workload-2 line
    c = torch.empty(M, dtype=torch.float64, device=dev)
    E = torch.empty(p.n_cfg, dtype=torch.float64, device=dev)
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device=dev)
    c_h = torch.empty(M, dtype=torch.float64).pin_memory()
    E_h = torch.empty(p.n_cfg, dtype=torch.float64).pin_memory()
    F_h = torch.empty(3 * p.n_atoms, dtype=torch.float64).pin_memory()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step(ctx):
        ctx.assemble(prob)
        ctx.factor()
        inf = ctx.solve(c, check=False)  # a fit that stops at max_iter is reported, not raised
        if inf["status"] not in (g.GAP_OK, g.GAP_ERR_NOT_CONVERGED):
            ctx._check(inf["status"])
        ctx.predict(None, c, E, F)  # the assembled problem: its design rows times c (J is not on the device)
        c_h.copy_(c, non_blocking=True)
        E_h.copy_(E, non_blocking=True)
        F_h.copy_(F, non_blocking=True)
        return inf

    def fit_with(prec, warmup, steps):
        ctx = g.Context(prec)
        ctx.set_option("j_ring_rows", RING_ROWS_W5)
        ctx.set_option("j_ring_direct", 1 if (pinned and args.j_ring_direct) else 0)
        for _ in range(warmup):
            inf = step(ctx)
        torch.cuda.synchronize()
        free, total = torch.cuda.mem_get_info()
        sampler = ClockSampler(0)
        sampler.start()
        ev0.record(stream)
        for _ in range(steps):
            inf = step(ctx)
        ev1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = ev0.elapsed_time(ev1) / steps
        prof = ctx.profile()
        return ctx, inf, ms, prof, clocks, (total - free)

    ws = g.workspace_size(prob, args.precision, RING_ROWS_W5)
    ctx, info, step_ms, prof, clocks, used = fit_with(args.precision, max(args.warmup, 3), args.steps)
    E0, F0, c0 = E_h.numpy().copy(), F_h.numpy().copy(), c_h.numpy().copy()
    # one more step with events between the calls: where the step's time goes, host gaps
    # included (each call synchronises before it returns)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    evs[0].record(stream)
    ctx.assemble(prob)
    evs[1].record(stream)
    ctx.factor()
    evs[2].record(stream)
    ctx.solve(c, check=False)
    evs[3].record(stream)
    ctx.predict(None, c, E, F)
    evs[4].record(stream)
    torch.cuda.synchronize()
    call_ms = {k: evs[i].elapsed_time(evs[i + 1]) for i, k in enumerate(("assemble", "factor", "solve", "predict"))}
    # the host link on this machine: the copies a step makes, each timed alone with CUDA events
    def h2d_ms(src_t, reps=2):
        dst = torch.empty(src_t.shape, dtype=src_t.dtype, device=dev)
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            ev0.record(stream)
            dst.copy_(src_t, non_blocking=True)
            ev1.record(stream)
            torch.cuda.synchronize()
            best = ev0.elapsed_time(ev1) if best is None else min(best, ev0.elapsed_time(ev1))
        del dst
        return best
    slot_pairs = RING_ROWS_W5 // 128 * 42
    j_chunk = torch.from_numpy(p.J[:slot_pairs])
    x_t = torch.from_numpy(p.X)
    xs_t = torch.from_numpy(np.ascontiguousarray(p.Xs))
    pin_chunk = torch.empty(j_chunk.shape, dtype=torch.float64).pin_memory()
    pin_chunk.copy_(j_chunk)
    link = {"J_chunk_gbs": j_chunk.nbytes / h2d_ms(j_chunk) / 1e6, "X_gbs": x_t.nbytes / h2d_ms(x_t) / 1e6,
            "page_locked": bool(pinned),
            "J_chunk_pinned_alloc_gbs": pin_chunk.nbytes / h2d_ms(pin_chunk) / 1e6,
            "Xs_pageable_gbs": xs_t.nbytes / h2d_ms(xs_t) / 1e6,
            "bytes": {"J_chunk": int(j_chunk.nbytes), "X": int(x_t.nbytes), "Xs": int(xs_t.nbytes)}}
    del pin_chunk
    # the same predictions from the descriptors (Eqs. 1, 2), J through the ring once more
    ev0.record(stream)
    ctx.predict(prob, c, E, F)
    ev1.record(stream)
    torch.cuda.synchronize()

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    pred_ring = {"ms": ev0.elapsed_time(ev1), "E_vs_design_rows": rel(E.cpu().numpy(), E0),
                 "F_vs_design_rows": rel(F.cpu().numpy(), F0)}
    # design rows of sampled configurations (each one's energy row, then three force rows
    # per atom) against the oracle's rows stored by tests/golden/make_workload5_rows.py
    rows_check = None
    z = np.load(W5_ROWS) if os.path.exists(W5_ROWS) else None
    if z is not None and str(z["fingerprint"]) == gapgen.fingerprint(p):
        cols, ref = z["cols"], z["rows"]
        got, en = [], []
        for A in z["cfgs"]:
            a0, a1 = int(p.cfg_ptr[A]), int(p.cfg_ptr[A + 1])
            o = torch.empty((1 + 3 * (a1 - a0), M), dtype=torch.float64, device=dev)
            ctx.read_design(1, int(A), 1, o[:1])
            ctx.read_design(1, p.n_cfg + 3 * a0, 3 * (a1 - a0), o[1:])
            got.append(o.cpu().numpy()[:, cols])
            en += [True] + [False] * (3 * (a1 - a0))
        got, en = np.concatenate(got), np.array(en)
        scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-300
        rows_check = {"configurations": [int(a) for a in z["cfgs"]], "rows": int(ref.shape[0]), "columns": int(len(cols)),
                      "energy_rel": rel(got[en], ref[en]), "force_rel": rel(got[~en], ref[~en]),
                      "max_abs_over_row_scale": float(np.max(np.abs(got - ref) / scale)),
                      "reference": "FP64 oracle rows of the same configurations (tests/golden/make_workload5_rows.py)"}
    sig = np.concatenate([p.sigma_e, p.sigma_f])
    res = (y - np.concatenate([E0, F0])) / sig
    chi2 = float(res @ res) / (N - M)
    ctx.close()
    others = {}
    if not args.no_other_precisions:
        for prec in ("mixed_bf16", "mixed_fp16", "mixed_tf32"):
            if prec == args.precision:
                continue
            cx, inf_o, ms_o, pr_o, _, _ = fit_with(prec, 1, 1)
            others[prec] = {"ms_per_step": ms_o, "value": rows / (ms_o * 1e-3), "unit": UNIT, "steps": 1,
                            "warmup": 1, "iterations": inf_o["iterations"], "converged": inf_o["converged"],
                            "phase_ms": {kk: round(v["ms"], 3) for kk, v in pr_o.items() if v["ms"] > 0},
                            "vs_main_precision": {"E": rel(E_h.numpy(), E0), "F": rel(F_h.numpy(), F0),
                                                  "c": rel(c_h.numpy(), c0)}}
            cx.close()
    if pinned:
        cudart.cudaHostUnregister(p.J.ctypes.data)
    if pinned_x:
        cudart.cudaHostUnregister(p.X.ctypes.data)
    n_chunks = -(-(-(-n_pairs // 42) * 128) // RING_ROWS_W5)
    line = dict(base, **{
        "value": rows / (step_ms * 1e-3), "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed_bf16": "bf16", "mixed_tf32": "tf32", "mixed_fp16": "fp16"}[args.precision],
        "data": "synthetic (seeded generator; the paper's datasets are not available)",
        "config": {"workload": "workload 5: %d configurations of 16-96 atoms, 3 species, d=%d, M=%d (5334+5333+5333), "
                               "zeta=%d, energies + 3 force rows per atom (%d design rows, %d pairs)"
                               % (p.n_cfg, p.d, M, r.zeta, N, n_pairs),
                   "precision": args.precision, "step": "assemble + factor + solve (FP64 refinement) + predict (design rows x c), "
                   "J (%.1f GB FP64) from %s host memory through the J ring" % (p.J.nbytes / 1e9,
                                                                                 "page-locked" if pinned else "pageable"),
                   "j_ring_rows": RING_ROWS_W5, "ring_chunks": n_chunks,
                   "j_ring_direct": bool(pinned and args.j_ring_direct),
                   "l2": "inputs larger than L2 (J alone is %.0f GB)" % (p.J.nbytes / 1e9),
                   "timing": "CUDA events on the ctx stream around whole steps; the copies of J, and of c, E, F "
                             "back to pinned host memory, are inside the step"},
        "fit_info": {kk: info[kk] for kk in ("iterations", "converged", "rel_update", "residual_norm")},
        "phase_ms": {kk: round(v["ms"], 3) for kk, v in prof.items() if v["ms"] > 0},
        "accuracy": {"sampled_design_rows": rows_check, "chi2_per_dof": chi2},
        "predict_from_descriptors": pred_ring,
        "call_ms": call_ms,
        "link": link,
        "memory": {"workspace_size_gb": ws / 1e9, "device_used_gb": used / 1e9, "host_J_gb": p.J.nbytes / 1e9,
                   "pin_s": pin_s, "J_registered": bool(pinned), "X_registered": bool(pinned_x)},
        "e2e": {"value": rows / (step_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(p.J.nbytes + p.X.nbytes),
                "d2h_bytes_per_step": int((M + p.n_cfg + 3 * p.n_atoms) * 8),
                "note": "the device-timed step already reads its inputs from host memory"},
        "clocks": clocks, "generation_s": gen_s,
        "gpu_launches": kernel_launch_count(p, args.precision, info["iterations"], ring_chunks=n_chunks,
                                            predict_from_rows=True) * args.steps,
    })
    if others:
        line["other_precisions"] = others
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == 4:
        return run_sweep(args)
    if args.workload == 5:
        return run_workload5(args)
    import torch
    import torch.distributed as dist
    import paper_2207_03803_gb300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g.build()
    g.load()

    def barrier():
        if world > 1:
            dist.barrier()

    p, prob_dev, prob_host, h2d_bytes = make_inputs(torch, dev, args.max_cfg)
    N, M = p.n_rows, p.n_sparse
    c = torch.empty(M, dtype=torch.float64, device=dev)
    E = torch.empty(p.n_cfg, dtype=torch.float64, device=dev)
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device=dev)
    ctx = g.Context(args.precision)
    if args.tsqr_shards:
        ctx.set_option("tsqr_shards", args.tsqr_shards)
    if args.tol > 0:
        ctx.set_option("tol", args.tol)
    if args.force_walk > 0:
        ctx.set_option("force_walk", args.force_walk)
    stream = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 3)):
        info = fit_step(ctx, prob_dev, c, E, F)
    torch.cuda.synchronize()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        info = fit_step(ctx, prob_dev, c, E, F)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_ms = ev0.elapsed_time(ev1)
    prof = ctx.profile()  # kernel classes of the last step
    rec = oracle_record(p)
    acc = accuracy(rec, c, E, F)  # the last timed step's fit and predictions
    tsqr_used = ctx.tsqr_blocks()
    t_all = torch.tensor([t_ms], device=dev)
    if world > 1:
        dist.all_reduce(t_all, op=dist.ReduceOp.MAX)
    t_ms = float(t_all.item())
    step_ms = t_ms / args.steps
    value = world * N * args.steps / (t_ms * 1e-3)
    launches = sum(v["groups"] for v in prof.values())

    # end to end through the C-ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        c_h = torch.empty(M, dtype=torch.float64).pin_memory()
        E_h = torch.empty(p.n_cfg, dtype=torch.float64).pin_memory()
        F_h = torch.empty(3 * p.n_atoms, dtype=torch.float64).pin_memory()
        fit_step(ctx, prob_host, c, E, F)
        torch.cuda.synchronize()
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            fit_step(ctx, prob_host, c, E, F)
            c_h.copy_(c, non_blocking=True)
            E_h.copy_(E, non_blocking=True)
            F_h.copy_(F, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        te = torch.tensor([ev0.elapsed_time(ev1)], device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        d2h = (M + p.n_cfg + 3 * p.n_atoms) * 8
        e2e_ms = float(te.item()) / args.steps
        # the host-to-device copies of one step's inputs alone (the same pinned buffers, the
        # same link), to tell link time from its overlap with the fit
        copy_ms = h2d_alone_ms(torch, prob_host, dev, stream)
        e2e = {"value": world * N * args.steps / (float(te.item()) * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
               "h2d_alone_ms": copy_ms, "h2d_alone_gbs": h2d_bytes / (copy_ms * 1e-3) / 1e9,
               "device_step_ms": step_ms,
               # 1: the copies hide entirely under the fit; 0: copies and fit one after the other
               "overlap": (copy_ms + step_ms - e2e_ms) / min(copy_ms, step_ms)}

    # the other mixed precisions on the same inputs (the config's TF32 variant, and FP16),
    # each its own context, closed before the next
    others = {}
    if not args.no_other_precisions and world == 1 and args.precision in ("mixed_bf16", "mixed_tf32", "mixed_fp16"):
        for prec in ("mixed_bf16", "mixed_tf32", "mixed_fp16"):
            if prec == args.precision:
                continue
            cx = g.Context(prec)
            if args.force_walk > 0:
                cx.set_option("force_walk", args.force_walk)
            for _ in range(2):
                inf_o = fit_step(cx, prob_dev, c, E, F)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.other_steps):
                inf_o = fit_step(cx, prob_dev, c, E, F)
            ev1.record(stream)
            torch.cuda.synchronize()
            t_o = ev0.elapsed_time(ev1) / args.other_steps
            pr_o = cx.profile()
            others[prec] = {"ms_per_step": t_o, "value": N / (t_o * 1e-3), "unit": UNIT, "steps": args.other_steps,
                            "warmup": 2, "iterations": inf_o["iterations"],
                            "phase_ms": {k: round(v["ms"], 3) for k, v in pr_o.items() if v["ms"] > 0},
                            "accuracy": accuracy(rec, c, E, F)}
            cx.close()

    # CUR choice of the sparse set from the workload's own descriptors (timed apart from
    # the step: the step's sparse set is the seeded random subset)
    cur = None
    if not args.no_cur and args.workload == 2:
        cur = cur_measure(g, torch, prob_dev.X, p, stream, dev)

    # the plain FP64 GPU path on the same inputs (denominator of the mixed speedup)
    fp64 = None
    if args.fp64_steps > 0 and args.precision != "fp64":
        ctx64 = g.Context("fp64")
        if args.tsqr_shards:
            ctx64.set_option("tsqr_shards", args.tsqr_shards)
        fit_step(ctx64, prob_dev, c, E, F)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.fp64_steps):
            fit_step(ctx64, prob_dev, c, E, F)
        ev1.record(stream)
        torch.cuda.synchronize()
        t64 = ev0.elapsed_time(ev1) / args.fp64_steps
        prof64 = ctx64.profile()
        acc64 = accuracy(rec, c, E, F)
        fp64 = {"ms_per_step": t64, "value": N / (t64 * 1e-3), "unit": UNIT, "steps": args.fp64_steps,
                "warmup": 1, "speedup_of_mixed": t64 / step_ms,
                "phase_ms": {k: round(v["ms"], 3) for k, v in prof64.items() if v["ms"] > 0},
                "accuracy": acc64}
        ctx64.close()

    if rank != 0:
        return
    pk = peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"mixed_bf16": "bf16", "mixed_tf32": "tf32", "mixed_fp16": "fp16", "fp64": "f64"}[args.precision],
        "data": "synthetic (seeded generator; the paper's HEA/SiC datasets are not available)",
        "config": {"workload": ("slice: " if args.max_cfg else "") +
                               "workload 2: %d configurations of 16-128 atoms, d=%d, M=%d, zeta=%d, energies + "
                               "3 force rows per atom (%d design rows, %d pairs)"
                               % (p.n_cfg, p.d, M, p.recipe.zeta, N, p.n_pairs),
                   "precision": args.precision, "step": "assemble + factor + solve (FP64 refinement) + predict",
                   "l2": "inputs larger than L2 (J alone is %.1f GB)" % (p.J.nbytes / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "factorisation": ("TSQR: %d row blocks, then the QR of [R_1; ...; R_G; U]" % tsqr_used
                                     if tsqr_used else "one QR of the stacked matrix")},
        "fit_info": {k: info[k] for k in ("iterations", "converged", "rel_update", "residual_norm")},
        "accuracy": acc,
        "phase_ms": {k: round(v["ms"], 3) for k, v in prof.items() if v["ms"] > 0},
        "assembly": assembly_rate({k: v["ms"] for k, v in prof.items()}, N),
        "roofline": roofline(prof, p, args.precision, pk, step_ms, info["iterations"]),
        "gpu_launches": None, "clocks": clocks, "e2e": e2e, "fp64_path": fp64, "peaks": pk,
    }
    if others:
        line["other_precisions"] = others
    if cur is not None:
        line["cur_selection"] = cur
    line["roofline"]["peak_source"] = pk["source"]
    line["gpu_launches"] = kernel_launch_count(p, args.precision, info["iterations"], tsqr_used) * args.steps
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        if rec is not None:
            # the oracle's whole fit as recorded, beside this run's sampled estimate
            host = json.loads(str(rec["host"]))
            line["cpu_baseline"]["measured_full_s"] = host["fit_s"]
            line["cpu_baseline"]["measured_full"] = {
                "machine": host["machine"], "cores": host["cores"], "date": host["date"],
                "phase_s": dict(zip(("assembly", "kmm_cholesky", "qr", "solve", "predict"),
                                    [float(x) for x in rec["times"]]))}
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


CUR_K, CUR_L, CUR_Q = 64, 96, 2  # rank, range-finder width, power iterations of the CUR choice


def cur_measure(g, torch, X, p, stream, dev, reps=3):
    """gap_select_cur on the workload's descriptor rows, M points per species, timed with
    CUDA events (the call synchronises its stream once per species).  Its work is FP64
    products: Y = X Omega, per power iteration P = Q^T X and Y = X P^T, the final B = Q^T X
    (2 n d l each); three CholeskyQR passes per orthonormalisation (4 n l^2 each); the
    scores Q W_k (2 n l k)."""
    import gapgen
    n, d = int(X.shape[0]), int(X.shape[1])
    l, k, q = CUR_L, CUR_K, CUR_Q
    omega, u = gapgen.cur_draws(p.recipe.seed, n, d, l)
    om = torch.from_numpy(omega).to(dev)
    ud = torch.from_numpy(u).to(dev)
    sizes = list(p.recipe.n_sparse)
    sp = None if p.atom_species is None else torch.from_numpy(p.atom_species).to(dev)
    g.select_cur(X, sizes, k, l, om, ud, power_iters=q, atom_species=sp)  # warm-up
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        sel = g.select_cur(X, sizes, k, l, om, ud, power_iters=q, atom_species=sp)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    flop = 2.0 * n * d * l * (2 + 2 * q) + 3 * (q + 1) * 4.0 * n * l * l + 2.0 * d * l * l + 2.0 * n * l * k
    peak = 152 * 2 * 2 * 2.07e9 / 1e12  # FP64: 2 DFMA/clk/SM (GB300), maximum SM clock
    return {"ms": ms, "atoms": n, "d": d, "points": int(sel.shape[0]), "k": k, "l": l, "power_iters": q,
            "roofline": {"bound": "alu", "achieved": flop / (ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flop / (ms * 1e-3) / 1e12 / peak, "algorithmic_flop": flop,
                         "peak_note": "FP64 ALU peak derived from unit counts (152 SMs x 2 DFMA/clk x 2.07 GHz)"}}


def kernel_launch_count(p, precision, iterations, tsqr_blocks=0, ring_chunks=0, predict_from_rows=False):
    """Kernels of the library launched by one fit step, counted from its launch
    schedule.  The ncu launch list of a workload-2 mixed_bf16 step with 13 refinement
    iterations (2052 launches per step) matches it.  A TSQR factorisation over G row
    blocks runs G + 1 QRs of M columns (the panel and update schedule does not depend on
    the rows) and G + 1 copies into the merge stack; in FP64 its residual norm converts G
    more block tails."""
    M = p.n_sparse
    nb32 = (M + 31) // 32    # Cholesky panels and inner QR panels
    n_outer = (M + 127) // 128
    solve = 2 + (M + 63) // 64  # diagonal-block inverses, one step per 64-row block, copy-out
    if precision == "fp64":
        assemble, predict = 10, 4
        chol = 1 + 3 * nb32 - 2 + 1  # K_MM, potrf/trsm/syrk per panel, stacking U
        qr = nb32 * (1 + 32 + 5)     # column kernels per panel, then the block update
        refine = 0
    else:
        assemble, predict = 23, 8  # each centres its descriptors (two means launches)
        # split X_s, K_MM, split, potrf/trsm/syrk, merge, stacking U twice
        chol = 1 + 1 + 1 + 3 * nb32 - 2 + 1 + 2
        # inner panels: CholeskyQR (Gram, its sum, Cholesky, two row passes, reconstruction), and
        # an update of the rest of the outer panel (Y, W2, update; the panel kernels packed
        # the reflectors) except after the last inner panel of an outer panel
        qr = 6 * nb32 + 3 * (nb32 - n_outer)
        # outer panels in pairs: the first panel's update of the second (8 launches), then
        # the pair's update of the trailing columns (11); a lone last panel: 8
        K0 = 0
        while K0 < M:
            K1 = min(M, K0 + 128)
            if K1 - K0 == 128 and K1 < M:
                qr += 8 + 11
                K0 = min(M, K1 + 128)
            else:
                qr += 8
                K0 = K1
        # per refinement pass: the fused pass, its reduction, the vector split, and the FP64
        # head pass over the energy rows (rows, column slabs, slab sum; no column slabs in
        # the final residual-only pass); per iteration also three W products, three dots,
        # two axpys, one xpby and two splits; once: the two inverses of R's blocks
        refine = 29 + 16 * iterations
        # the force GEMM (over d) and the predictions' gradient product (over M) run in
        # K-chunks of at most 8 k-blocks of 128 bytes; both operands are padded to 64 columns
        esz = 2 if precision in ("mixed_bf16", "mixed_fp16") else 4
        kb_force = (-(-p.d // 64) * 64) * esz // 128
        kb_grad = (-(-M // 64) * 64) * esz // 128
        assemble += -(-kb_force // 8) - 1
        predict += -(-kb_grad // 8) - 1
        if ring_chunks:  # J ring: a packing and the force GEMM's K-chunks per chunk
            assemble += (ring_chunks - 1) * (1 + -(-kb_force // 8))
        if predict_from_rows:  # the design rows times c: energy rows, c split, force rows
            predict = 3
    if tsqr_blocks:
        qr = (tsqr_blocks + 1) * (qr + 1)
        if precision == "fp64":
            solve += tsqr_blocks
    return assemble + chol + qr + solve + refine + predict


if __name__ == "__main__":
    main()
