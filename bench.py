"""Benchmark: useful TFLOP/s of the irrep-aligned contraction, split-BF16 vs FP64.

Workload (default): the coupled-cluster particle-particle ladder under Z_8
symmetry, w[a,b,i,j] = sum_{c,d} v[a,b,c,d] t[c,d,i,j], virtual modes 8
sectors x 32, occupied modes 8 sectors x 8 (seeded synthetic reduced forms:
v ~ N(0,1)/16, 4.3 GB; t ~ N(0,1)*1e-2): one aligned GEMM batch of 8 irreps
with M = K = 8192, N = 512 (549.8 GFLOP of symmetry-reduced work).  One step =
the whole contraction, standard reduced forms in and out.
--workload mps: the MPS transfer step under Z_8, E'[g,d] = sum E[a,b] A[a,s,g]
A[b,s,d], as two aligned contractions X = einsum('ab,asg->bsg', E, A) and
E' = einsum('bsg,bsd->gd', X, A) (bond 8 sectors x 128, physical 8 x 2).

Metric: useful TFLOP/s = symmetry-reduced GEMM flops (2 * n_Q * M * N * K per
contraction) / device time of the step (median over the timed steps).  The
split-BF16 form is the headline value; the FP64 form and the relative errors
of both against the CPU float64 oracle are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload cc_ladder|mps|...] [--precision split_bf16|fp64|tf32]
Multi-GPU (torchrun): replicas only; each rank runs the whole workload.
"""
from __future__ import annotations

import os

_CORES = len(os.sched_getaffinity(0))
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(_CORES))

import argparse
import hashlib
import json
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as WL  # noqa: E402

L2_FLUSH_BYTES = 256 << 20


def spec(t):
    return (t.signs, t.charge, t.dims)


# ---------------------------------------------------------------------------
# workloads: list of (einsum, moduli, sym_u, sym_v) steps and input arrays
# ---------------------------------------------------------------------------

def mps_workload():
    E = WL.draw(WL.MPS_E, (WL.MPS_G,))
    A = WL.draw(WL.MPS_A, (WL.MPS_G,))
    name = "mps_transfer_Z8_bond8x128_phys8x2 (X=E.A, E'=X.A; two aligned contractions)"
    return name, E, A


def cc_contraction(args):
    if args.cc_dims:
        virt, occ = (int(x) for x in args.cc_dims.split(","))
        return WL.cc_ladder(8, virt, occ)
    return WL.CC_LADDER


def cc_workload(args):
    c = cc_contraction(args)
    g = c.moduli[0]
    # v[a,b,c,d] has four virtual modes; t[c,d,i,j] ends with the occupied ones
    name = f"cc_ladder_Z{g}_virt{g}x{c.u.dims[0]}_occ{g}x{c.v.dims[-1]} (w=v.t)"
    return name, WL.draw(c.u, c.moduli), WL.draw(c.v, c.moduli)


# ---------------------------------------------------------------------------
# oracle (CPU float64) -- cpu_baseline leg and the reference arm only
# ---------------------------------------------------------------------------

def oracle_step(workload, a, b, c=None):
    import oracle as O
    if workload == "mps":
        g = O.Group((WL.MPS_G,))
        p1 = O.plan(WL.MPS_STEP1, g, O.Sym(*spec(WL.MPS_E)), O.Sym(*spec(WL.MPS_A)))
        p2 = O.plan(WL.MPS_STEP2, g, p1.sym_w, O.Sym(*spec(WL.MPS_A)))

        def run():
            x = O.contract_blockloop(p1, a, b)
            return O.contract_blockloop(p2, x, b)
        return run
    c = c or WL.CC_LADDER
    p = O.plan(c.einsum, O.Group(c.moduli), O.Sym(*spec(c.u)), O.Sym(*spec(c.v)))
    # the whole block loop (its G^(s+t+v-2) block products are NumPy matmuls)
    return lambda: O.contract_blockloop(p, a, b)


def time_oracle(workload, a, b, budget_s=12.0, max_reps=50, c=None):
    run = oracle_step(workload, a, b, c)
    out = run()
    ts = []
    t_end = time.perf_counter() + budget_s
    while len(ts) < max_reps and (not ts or time.perf_counter() < t_end):
        t0 = time.perf_counter()
        run()
        ts.append(time.perf_counter() - t0)
    return out, statistics.median(ts), len(ts)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"symctr_clocks_{os.getpid()}.csv")
        self.dev = device_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}",
                                          f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1].split()[0]))
                mx.append(float(r[2].split()[0]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


# ---------------------------------------------------------------------------
# replicas: every rank runs the whole step on its own GPU (the contraction has
# no exchange step); the job time is the slowest rank's
# ---------------------------------------------------------------------------

def max_over_ranks(ms, world, device):
    """The largest per-step time over all ranks (every rank returns it)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.barrier()
    return float(t.item())


def replicas_value(flops_per_step, ms, world):
    """Whole-job useful TFLOP/s: every rank completes one step of
    `flops_per_step` in at most `ms` milliseconds."""
    return world * flops_per_step / (ms * 1e-3) / 1e12


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

# the sources that decide each kernel's code and launch shape (the launchers
# sit beside the kernels; the shared sizing rules are in the internal header)
KERNEL_SOURCES = {
    "prep_kernel": ("transforms.cu", "symctr_internal.h"),
    "rowtile_kernel": ("transforms.cu", "symctr_internal.h"),
    "rowstream_kernel": ("transforms.cu", "symctr_internal.h"),
    "gemm_tc_kernel": ("gemm_tc.cu", "symctr_internal.h"),
    "gemm_f64": ("gemm_f64.cu", "symctr_internal.h"),
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    files = []
    for k in kernel.split("+"):
        files += [f for f in KERNEL_SOURCES[k] if f not in files]
    for f in files:
        with open(os.path.join(ROOT, "paper_2007_08056_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(kernel, key):
    """DRAM bytes per launch (read + write) from the committed ncu summary
    profiles/traffic.json, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            e = json.load(f).get(key)
        if e and e.get("source_hash") == kernel_source_hash(kernel):
            return e.get("bytes_per_launch")
    except Exception:
        pass
    return None


def peaks():
    p = {"hbm_gbs": 6692.1, "bf16_tflops": 1925.9, "bf16_tflops_sustained": 1723.2, "src": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        p.update({k: d[k] for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained") if k in d})
        p["src"] = "measured"
    except Exception:
        pass
    return p


def prep_bytes(pl):
    """Algorithmic bytes of one operand-prep launch: every aligned operand
    element read once as float64 and written once in the GEMM's operand format
    (S BF16 slices, or one TF32 word), plus one int32 exponent per row."""
    i = pl.info
    elems = i.aligned_numel_u + i.aligned_numel_v
    if i.precision == 1:
        return elems * (8 + 2 * i.n_slices) + 4 * i.n_q * (i.M + i.N)
    return elems * (8 + 4)


def prep_kernels(pl):
    """The operand-preparation kernels a plan launches: per operand, bits 0/1 of
    info.single_read_prep mean rows streamed by bulk copies (rowstream_kernel),
    bits 2/3 whole short rows per CTA (rowtile_kernel), neither the two-phase
    prep_kernel (which also runs alone to zero split-K sums when no short-row
    kernel runs)."""
    i = pl.info
    if i.precision != 1:
        return ["prep_kernel"]
    names = []
    for op in (0, 1):
        if i.single_read_prep & (1 << op):
            names.append("rowstream_kernel")
        elif i.single_read_prep & (4 << op):
            names.append("rowtile_kernel")
        else:
            names.append("prep_kernel")
    if "rowtile_kernel" not in names:
        names.append("prep_kernel")
    return names


def rooflines(args, plans, prep, gemm, pk):
    """One roofline per kernel kind of the step: achieved = algorithmic work of
    its launches in one step / their CUDA-event time in that step."""
    out = []
    gemm_ms = sum(gemm)
    if args.precision == "split_bf16":
        pairs = [pl.info.n_slices * (pl.info.n_slices + 1) // 2 for pl in plans]
        work = sum(pl.useful_flops * k for pl, k in zip(plans, pairs))
        kernel, bound, unit, peak = "gemm_tc_kernel", "tensor", "TFLOP/s", pk["bf16_tflops"]
        peak_src = f"{pk['src']} bf16 burst"
    elif args.precision == "tf32":
        work = sum(pl.useful_flops for pl in plans)
        kernel, bound, unit, peak = "gemm_tc_kernel", "tensor", "TFLOP/s", pk["bf16_tflops"] / 2
        peak_src = f"{pk['src']} bf16 burst x 1/2 (nominal tf32:bf16 ratio)"
    else:
        work = sum(pl.useful_flops for pl in plans)
        kernel, bound, unit, peak = "gemm_f64", "alu", "TFLOP/s", 1.25
        peak_src = "1.25 TFLOP/s nominal FP64 (152 SMs x FP64 units x clock; cuBLAS DGEMM measured 1.1)"
    achieved = work / (gemm_ms * 1e-3) / 1e12
    key = f"{kernel}/{args.precision}/{args.workload}"
    out.append({"kernel": kernel, "bound": bound, "achieved": round(achieved, 3), "peak": peak,
                "unit": unit, "frac": round(achieved / peak, 4),
                "traffic": load_traffic(kernel, key), "peak_src": peak_src,
                "launches_per_step": len(plans), "ms_per_step": round(gemm_ms, 4),
                "work_per_launch": work / len(plans)})
    prep_ms = sum(prep)
    if args.precision != "fp64" and prep_ms > 0:
        nbytes = sum(prep_bytes(pl) for pl in plans)
        achieved = nbytes / (prep_ms * 1e-3) / 1e9
        names = []
        for pl in plans:
            for k in prep_kernels(pl):
                if k not in names:
                    names.append(k)
        label = "+".join(names)
        key = f"{label}/{args.precision}/{args.workload}"
        out.append({"kernel": label, "bound": "hbm", "achieved": round(achieved, 1),
                    "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4),
                    "traffic": load_traffic(label, key), "peak_src": f"{pk['src']} hbm copy",
                    "launches_per_step": len(plans), "ms_per_step": round(prep_ms, 4),
                    "work_per_launch": nbytes / len(plans)})
    return out


def run_ours(args, rank, world):
    import torch
    import paper_2007_08056_gb300 as sc

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = torch.device("cuda")
    ctr = None
    if args.workload == "mps":
        name, Eh, Ah = mps_workload()
        if args.chain:
            name += ", X kept aligned between the steps"
        E, A = torch.from_numpy(Eh).to(dev), torch.from_numpy(Ah).to(dev)

        def make(prec):
            p1 = sc.Plan(WL.MPS_STEP1, (WL.MPS_G,), spec(WL.MPS_E), spec(WL.MPS_A), prec)
            p2 = sc.Plan(WL.MPS_STEP2, (WL.MPS_G,), p1.sym_w, spec(WL.MPS_A), prec)
            if args.chain:
                # X stays in X = E.A's aligned layout and is read from there by E' = X.A
                p1.chain(w_aligned=True)
                p2.chain(u_from=p1)
            X = torch.empty(p1.shape_w, dtype=torch.float64, device=dev)
            out = torch.empty(p2.shape_w, dtype=torch.float64, device=dev)

            def step(e=E, a=A):
                p1.contract(e, a, out=X)
                p2.contract(X, a, out=out)
                return out
            return [p1, p2], step, out
        inputs_host = [Eh, Ah]
    else:
        name, Uh, Vh = cc_workload(args)
        U, V = torch.from_numpy(Uh).to(dev), torch.from_numpy(Vh).to(dev)
        c = ctr = cc_contraction(args)

        def make(prec):
            p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), prec)
            out = torch.empty(p.shape_w, dtype=torch.float64, device=dev)

            def step(a=U, b=V):
                p.contract(a, b, out=out)
                return out
            return [p], step, out
        inputs_host = [Uh, Vh]

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ev_s = torch.cuda.Event(enable_timing=True)
    ev_e = torch.cuda.Event(enable_timing=True)

    def timed(step, n, warm, per_plan=None):
        for _ in range(warm):
            step()
        torch.cuda.synchronize()
        times, phases = [], []
        for _ in range(n):
            flush.fill_(1)                       # L2 flush, outside the timed window
            ev_s.record()
            step()
            ev_e.record()
            ev_e.synchronize()
            times.append(ev_s.elapsed_time(ev_e))
            if per_plan:
                phases.append([pl.phase_times() for pl in per_plan])
        return times, phases

    plans, step, out = make(args.precision)
    flops = sum(pl.useful_flops for pl in plans)

    # The timed steps run without the library's phase events: an event recorded
    # between the prep kernel and the GEMM would end the programmatic launch
    # overlap between them.  Phase times come from separate profiled steps.
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as clk:
        times, _ = timed(step, args.steps, args.warmup)
    torch.cuda.synchronize()
    for pl in plans:
        pl.check_device_error()
    ms = max_over_ranks(statistics.median(times), world, dev)
    ms_mean = max_over_ranks(statistics.mean(times), world, dev)
    value = replicas_value(flops, ms, world)

    # per-kernel phases (averaged over profiled steps outside the timed region)
    for pl in plans:
        pl.profile(True)
    _, phases = timed(step, max(5, min(args.steps, 10)), 1, plans)
    for pl in plans:
        pl.profile(False)
    prep = [statistics.mean(ph[i][0] for ph in phases) for i in range(len(plans))]
    gemm = [statistics.mean(ph[i][1] for ph in phases) for i in range(len(plans))]
    launches_per_step = sum(phases[-1][i][2] for i in range(len(plans)))

    # accuracy of the forms against the oracle (outside any timed region)
    res = {}
    if rank == 0:
        ref = oracle_step(args.workload, *inputs_host, c=ctr)()
        got = step().cpu().numpy()
        res[args.precision] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    # the FP64 form beside it
    fp64 = None
    if args.precision != "fp64" and not args.no_fp64:
        plans64, step64, _ = make("fp64")
        t64, _ = timed(step64, max(2, min(args.steps, 5)), 1)
        ms64 = statistics.median(t64)
        fp64 = {"value": round(world * flops / (ms64 * 1e-3) / 1e12, 4), "ms_per_step": round(ms64, 4)}
        if rank == 0:
            got = step64().cpu().numpy()
            res["fp64"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))

    # end to end through the public API from pinned host buffers
    hin = [torch.from_numpy(x).pin_memory() for x in inputs_host]
    dins = [torch.empty(x.shape, dtype=torch.float64, device=dev) for x in inputs_host]
    hout = torch.empty(tuple(out.shape), dtype=torch.float64).pin_memory()

    def e2e_step():
        for h, d in zip(hin, dins):
            d.copy_(h, non_blocking=True)
        o = step(*dins)
        hout.copy_(o, non_blocking=True)
    t_e2e, _ = timed(e2e_step, args.steps, args.warmup)
    ms_e2e = max_over_ranks(statistics.median(t_e2e), world, dev)

    pk = peaks()
    roofs = rooflines(args, plans, prep, gemm, pk)
    dominant = max(roofs, key=lambda r: r["ms_per_step"])
    other = [r for r in roofs if r is not dominant]
    clocks = clk.summary()
    line = {
        "metric": "useful TFLOP/s, split-BF16 vs FP64 irrep-aligned contraction at stated rel err",
        "value": round(value, 4),
        "unit": "TFLOP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "ms_per_step_mean": round(ms_mean, 4),
        "timing": "median over the timed steps (CUDA events on the launching stream)",
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"split_bf16": "bf16 slices x5, fp32 accumulate, int64 combine, f64 out",
                  "tf32": "tf32, fp32 accumulate, f64 out", "fp64": "f64"}[args.precision],
        "data": "synthetic (seeded N(0,1) reduced forms)",
        "config": {"workload": name, "precision": args.precision,
                   "n_slices": plans[0].info.n_slices, "useful_gflop_per_step": flops / 1e9,
                   "l2": "flushed (256 MiB write) between timed steps, outside the events",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "rel_err_vs_oracle": {k: float(f"{v:.3e}") for k, v in res.items()},
        "fp64_form": fp64,
        "phases_ms": {"prep": [round(x, 4) for x in prep], "gemm": [round(x, 4) for x in gemm]},
        "roofline": dominant,
        "roofline_other": other[0] if other else None,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "e2e": {"value": round(replicas_value(flops, ms_e2e, world), 4), "unit": "TFLOP/s",
                "ms_per_step": round(ms_e2e, 4),
                "h2d_bytes_per_step": int(sum(x.nbytes for x in inputs_host)),
                "d2h_bytes_per_step": int(out.numel() * 8)},
    }
    if rank == 0 and not args.no_cpu_baseline:
        _, t_or, reps = time_oracle(args.workload, *inputs_host, budget_s=args.cpu_budget, c=ctr)
        line["cpu_baseline"] = {"value": round(flops / t_or / 1e12, 6), "unit": "TFLOP/s",
                                "cores": _CORES, "kind": "oracle",
                                "sample": f"whole step ({'both contractions' if args.workload == 'mps' else 'the contraction'}), "
                                          f"block-loop route, median of {reps} runs, {t_or * 1e3:.1f} ms each"}
    return line


def run_complex(args, rank, world):
    """The MPS transfer step with complex tensors, E' = sum E A conj(A): X = E.A,
    then E' = X.conj(A), conj(A) carrying A's negated law.  Useful flops count
    the four real products of each complex contraction."""
    import torch
    import oracle as O
    import paper_2007_08056_gb300 as sc

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = torch.device("cuda")
    g = WL.MPS_G
    sE, sA = spec(WL.MPS_E), spec(WL.MPS_A)
    negA = (tuple(-c for c in sA[0]), tuple(-z for z in sA[1]), sA[2])
    rng = np.random.default_rng(2101)
    shE = WL.reduced_shape((g,), WL.MPS_E.dims)
    shA = WL.reduced_shape((g,), WL.MPS_A.dims)
    Eh = rng.standard_normal(shE) + 1j * rng.standard_normal(shE)
    Ah = rng.standard_normal(shA) + 1j * rng.standard_normal(shA)
    p1 = sc.Plan(WL.MPS_STEP1, (g,), sE, sA, args.precision)
    p2 = sc.Plan(WL.MPS_STEP2, (g,), p1.sym_w, negA, args.precision)
    E, A = torch.from_numpy(Eh).to(dev), torch.from_numpy(Ah).to(dev)
    X = torch.empty(p1.shape_w, dtype=torch.complex128, device=dev)
    out = torch.empty(p2.shape_w, dtype=torch.complex128, device=dev)

    def step(e=E, a=A):
        p1.contract_complex(e, a, out=X)
        p2.contract_complex(X, a, out=out, conj_v=True)
        return out

    flops = 4 * (p1.useful_flops + p2.useful_flops)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ev_s, ev_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1)
            ev_s.record()
            fn()
            ev_e.record()
            ev_e.synchronize()
            ts.append(ev_s.elapsed_time(ev_e))
        return statistics.median(ts)

    ms = max_over_ranks(timed(step), world, dev)
    p2.check_device_error()
    G = O.Group((g,))
    o1 = O.plan(WL.MPS_STEP1, G, O.Sym(*sE), O.Sym(*sA))
    o2 = O.plan(WL.MPS_STEP2, G, o1.sym_w, O.Sym(*negA))
    want = O.contract_blockloop(o2, O.contract_blockloop(o1, Eh, Ah), np.conj(Ah))
    got = step().cpu().numpy()
    hin = [torch.from_numpy(x).pin_memory() for x in (Eh, Ah)]
    dins = [torch.empty(x.shape, dtype=torch.complex128, device=dev) for x in (Eh, Ah)]
    hout = torch.empty(tuple(out.shape), dtype=torch.complex128).pin_memory()

    def e2e_step():
        for h, d in zip(hin, dins):
            d.copy_(h, non_blocking=True)
        o = step(*dins)
        hout.copy_(o, non_blocking=True)
    ms_e2e = max_over_ranks(timed(e2e_step), world, dev)
    return {"workload": "mps_transfer_Z8_complex (X=E.A, E'=X.conj(A))", "precision": args.precision,
            "ms_per_step": round(ms, 4), "useful_tflops": round(replicas_value(flops, ms, world), 4),
            "useful_gflop_per_step": flops / 1e9,
            "rel_err_vs_oracle": float(f"{np.linalg.norm(got - want) / np.linalg.norm(want):.3e}"),
            "e2e": {"value": round(replicas_value(flops, ms_e2e, world), 4), "ms_per_step": round(ms_e2e, 4),
                    "h2d_bytes_per_step": int(Eh.nbytes + Ah.nbytes), "d2h_bytes_per_step": int(out.numel() * 16)}}


def run_device(args, rank, world):
    """Workloads whose operands are drawn on the device: config 5 (the
    CC-ladder contraction at virtual 512 / occupied 128 with sector dims 512/G
    and 128/G, up to 275 GB at G = 2; --sweep-dims 256,64 gives the secondary
    sweep at the CC ladder's dimensions), the Table-2 instances of the Table-1
    contraction families and the generic (s, t, v) contractions of Sec. 5.1.1
    (G = 4, about 80e9 useful flops each).  The error is taken on entries the
    oracle computes one by one.  Forward, and with --backward the adjoint pair
    as well.  Step times are medians over the timed steps."""
    import torch
    import oracle as O
    import paper_2007_08056_gb300 as sc

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = torch.device("cuda")
    if args.workload == "sweep":
        G = args.sweep_g
        virt, occ = (int(x) for x in args.sweep_dims.split(","))
        c = WL.cc_ladder(G, virt, occ)
        seed = 5000 + G if (virt, occ) == (512, 128) else 5100 + G
    elif args.workload == "generic":
        c = WL.generic_contraction(*args.stv_point)
        G = c.moduli[0]
        seed = c.u.seed
    else:
        c = WL.TABLE2[args.case]
        G = c.moduli[0]
        seed = c.u.seed
    probe = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "fp64")
    operand_bytes = 8 * (probe.info.numel_u + probe.info.numel_v + probe.info.numel_w)
    del probe
    if operand_bytes > torch.cuda.mem_get_info()[0] - (8 << 30):
        return {"workload": c.name, "precision": args.precision, "G": G,
                "unavailable": f"exceeds one GPU's HBM (u, v, w alone take {operand_bytes / 1e9:.0f} GB)"}
    gen = torch.Generator(device="cuda").manual_seed(seed)
    U = torch.randn(WL.reduced_shape(c.moduli, c.u.dims), generator=gen, device=dev,
                    dtype=torch.float64).mul_(c.u.scale)
    V = torch.randn(WL.reduced_shape(c.moduli, c.v.dims), generator=gen, device=dev,
                    dtype=torch.float64).mul_(c.v.scale)
    p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), args.precision)
    W = torch.empty(p.shape_w, dtype=torch.float64, device=dev)
    free, _ = torch.cuda.mem_get_info()
    want = int(p.info.workspace_bytes)
    budget = free - (8 << 30) - L2_FLUSH_BYTES
    nbytes = want if want <= budget else max(int(p.info.workspace_bytes_min), budget)
    if nbytes > budget:
        return {"workload": c.name, "unavailable": "exceeds one GPU's HBM"}
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ev_s, ev_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1)
            ev_s.record()
            fn()
            ev_e.record()
            ev_e.synchronize()
            ts.append(ev_s.elapsed_time(ev_e))
        return statistics.median(ts)

    ms = max_over_ranks(timed(lambda: p.contract(U, V, out=W, workspace=ws)), world, dev)
    # phase times from one profiled call outside the timed steps (the events
    # would end the programmatic launch overlap of prep and GEMM)
    p.profile(True)
    p.contract(U, V, out=W, workspace=ws)
    torch.cuda.synchronize()
    prep_ms, gemm_ms, _ = p.phase_times()
    p.profile(False)
    p.check_device_error(ws)
    o = O.plan(c.einsum, O.Group(c.moduli), O.Sym(*spec(c.u)), O.Sym(*spec(c.v)))
    rng = np.random.default_rng(seed + 500)
    idx = [tuple(int(rng.integers(0, d)) for d in p.shape_w) for _ in range(16)]
    want_e = [O.contract_element_lazy(o, lambda i: U[i].cpu().numpy(), lambda i: V[i].cpu().numpy(), ix)
              for ix in idx]
    got = [W[ix].item() for ix in idx]
    rel = float(np.linalg.norm(np.subtract(got, want_e)) / np.linalg.norm(want_e))
    line = {"workload": c.name, "einsum": c.einsum, "precision": args.precision, "G": G,
            "M_N_K": [int(p.info.M), int(p.info.N), int(p.info.K)], "n_q": int(p.info.n_q),
            "useful_tflop": p.useful_flops / 1e12, "ms": round(ms, 3),
            "useful_tflops": round(replicas_value(p.useful_flops, ms, world), 3),
            "phases_ms": {"prep": round(prep_ms, 3), "gemm": round(gemm_ms, 3)},
            "passes": "one" if nbytes >= want else f"Q-streaming, workspace {nbytes / 1e9:.1f} GB",
            "rel_err_sampled_16": float(f"{rel:.3e}")}
    pk = peaks()
    if nbytes >= want:
        line["rooflines"] = rooflines(args, [p], [prep_ms], [gemm_ms], pk)
    else:
        line["rooflines"] = ("not separable: with Q-streaming the passes interleave operand "
                             "preparation and GEMM, and the phase events bracket the first pass")
    if args.backward:
        del ws
        torch.cuda.empty_cache()
        gW = torch.randn(p.shape_w, generator=gen, device=dev, dtype=torch.float64)
        free, _ = torch.cuda.mem_get_info()
        need = int(p.info.workspace_bytes_backward) + 8 * (U.numel() + V.numel())
        if need > free - (8 << 30):
            line["backward"] = {"unavailable": "exceeds one GPU's HBM (the gradients add the size of u and v)"}
        else:
            wsb = torch.empty(int(p.info.workspace_bytes_backward), dtype=torch.uint8, device=dev)
            msb = max_over_ranks(timed(lambda: p.backward(gW, U, V, workspace=wsb)), world, dev)
            line["backward"] = {"ms": round(msb, 3),
                                "useful_tflops": round(replicas_value(2 * p.useful_flops, msb, world), 3)}
    return line


def run_small(args, rank, world):
    """Config 1 (the order-4 Z_3 contraction of Sec. 2, 6912-entry reduced
    forms: launch-latency bound) and config 4 (PEPS-style gradients under
    Z_2 x Z_3: forward y = T.Env, loss = sum y^2, hand-written backward through
    the autograd Function; HBM-bound, its GEMVs run in float64 on the CUDA
    cores in every form).  Whole-step device time, L2 flushed between steps,
    errors against the oracle."""
    import torch
    import oracle as O
    import paper_2007_08056_gb300 as sc

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = torch.device("cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ev_s, ev_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1)
            ev_s.record()
            fn()
            ev_e.record()
            ev_e.synchronize()
            ts.append(ev_s.elapsed_time(ev_e))
        return statistics.median(ts)

    def graphed(fn):
        """fn captured once as a CUDA graph: (replay, None), or (None, why)
        when the capture fails.  Warm-up and capture share one side stream, so
        the plans have seen it before the capture starts."""
        try:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for _ in range(3):
                    fn()
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                fn()
            torch.cuda.synchronize()
            return g.replay, None
        except Exception as e:
            torch.cuda.synchronize()
            return None, f"graph capture failed: {type(e).__name__}"

    if args.workload == "z3":
        c = WL.Z3_ORDER4
        uh, vh = WL.draw_pair(c)
        u, v = torch.from_numpy(uh).to(dev), torch.from_numpy(vh).to(dev)
        p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), args.precision)
        w = torch.empty(p.shape_w, dtype=torch.float64, device=dev)
        ms = max_over_ranks(timed(lambda: p.contract(u, v, out=w)), world, dev)
        want = O.contract_blockloop(O.plan(c.einsum, O.Group(c.moduli), O.Sym(*spec(c.u)),
                                           O.Sym(*spec(c.v))), uh, vh)
        got = w.cpu().numpy()
        return {"workload": "z3_order4 (config 1: G = 3, D = 4, reduced forms [3,3,3,4,4,4,4])",
                "precision": args.precision, "ms_per_step": round(ms, 4),
                "useful_flops_per_step": p.useful_flops,
                "useful_tflops": round(replicas_value(p.useful_flops, ms, world), 6),
                "bound": "launch latency (0.66 MFLOP per step)",
                "rel_err_vs_oracle": float(f"{np.linalg.norm(got - want) / np.linalg.norm(want):.3e}")}
    moduli = WL.PEPS_MODULI
    Th, Envh = WL.draw(WL.PEPS_T, moduli), WL.draw(WL.PEPS_ENV, moduli)
    T = torch.from_numpy(Th).to(dev).requires_grad_(True)
    Env = torch.from_numpy(Envh).to(dev).requires_grad_(True)
    py = sc.Plan(WL.PEPS_Y, moduli, spec(WL.PEPS_T), spec(WL.PEPS_ENV), args.precision)
    pl = sc.Plan(WL.PEPS_LOSS, moduli, py.sym_w, py.sym_w, args.precision)

    def step():
        T.grad = None
        Env.grad = None
        y = sc.contract(py, T, Env)
        sc.contract(pl, y, y).backward()

    # The step issues about a dozen launches through autograd; replayed as one
    # CUDA graph it no longer waits on the host between them.  The eager step
    # is timed too.
    ms_eager = max_over_ranks(timed(step), world, dev)
    replay, graph_note = graphed(step)
    ms = max_over_ranks(timed(replay), world, dev) if replay else ms_eager
    (replay or step)()
    torch.cuda.synchronize()
    oy = O.plan(WL.PEPS_Y, O.Group(moduli), O.Sym(*spec(WL.PEPS_T)), O.Sym(*spec(WL.PEPS_ENV)))
    y_ref = O.contract_blockloop(oy, Th, Envh)
    gT_ref = O.grad_u(oy, 2 * y_ref, Envh)
    gE_ref = O.grad_v(oy, Th, 2 * y_ref)
    gT, gE = T.grad.cpu().numpy(), Env.grad.cpu().numpy()
    rel = max(np.linalg.norm(gT - gT_ref) / np.linalg.norm(gT_ref),
              np.linalg.norm(gE - gE_ref) / np.linalg.norm(gE_ref))
    # algorithmic bytes: forward reads T's live sector and Env; the backward
    # writes all of gT (zeros outside the live sector), reads Env and T's live
    # sector again and writes gEnv
    live_t = py.info.aligned_numel_u * 8
    env_b = Envh.nbytes
    nbytes = (live_t + env_b) + (Th.nbytes + env_b) + (live_t + env_b)
    flops = 3 * py.useful_flops   # forward GEMV and the two adjoint products
    achieved = nbytes / (ms * 1e-3) / 1e9
    pk = peaks()
    return {"workload": "peps_grad (config 4: Z_2 x Z_3, T [6,6,6,6,16,16,16,16,2], Env [6,6,6,16,16,16,16])",
            "precision": args.precision, "ms_per_step": round(ms, 4),
            "step": "CUDA graph replay" if replay else f"eager ({graph_note})",
            "ms_per_step_eager": round(ms_eager, 4),
            "useful_tflops": round(replicas_value(flops, ms, world), 4),
            "roofline": {"kernel": "whole step (gemm_f64 GEMVs, fill, align)", "bound": "hbm",
                         "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": round(achieved / pk["hbm_gbs"], 4),
                         "algorithmic_bytes_per_step": nbytes},
            "rel_err_grad_vs_oracle": float(f"{rel:.3e}")}


def run_reference(args, rank, world):
    """The oracle on the host cores, on the same workload and metric: the
    block loop (Algorithm 1 generalised) of the whole step, one full step per
    timed step (about 1.5 s for the CC ladder on 16 cores, 10 ms for the MPS
    step)."""
    if rank != 0:
        return None
    import oracle as O
    if args.workload == "mps":
        name, a, b = mps_workload()
        g = WL.MPS_G
        p1 = O.plan(WL.MPS_STEP1, O.Group((g,)), O.Sym(*spec(WL.MPS_E)), O.Sym(*spec(WL.MPS_A)))
        p2 = O.plan(WL.MPS_STEP2, O.Group((g,)), p1.sym_w, O.Sym(*spec(WL.MPS_A)))
        plans = (p1, p2)
        c = None
    elif args.workload == "cc_ladder":
        name, a, b = cc_workload(args)
        c = cc_contraction(args)
        plans = (O.plan(c.einsum, O.Group(c.moduli), O.Sym(*spec(c.u)), O.Sym(*spec(c.v))),)
    else:
        return {"impl": "reference", "unavailable": f"reference arm times the cc_ladder and mps "
                                                    f"workloads only (asked: {args.workload})"}
    flops = 2.0 * sum(len(O.q_set(p)) * np.prod(O.aligned_dims(p)[1:]) for p in plans)
    run = oracle_step(args.workload, a, b, c=c)
    for _ in range(args.warmup):
        run()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        run()
        ts.append(time.perf_counter() - t0)
    ms = statistics.median(ts) * 1e3
    value = flops / (ms * 1e-3) / 1e12
    return {
        "impl": "reference",
        "metric": "useful TFLOP/s, split-BF16 vs FP64 irrep-aligned contraction at stated rel err",
        "value": round(value, 6), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "precision": "fp64 (CPU oracle, block loop)"},
        "cpu_baseline": {"value": round(value, 6), "unit": "TFLOP/s", "cores": _CORES,
                         "kind": "oracle", "sample": "one whole step per timed step, median"},
        "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 160 for the CC ladder, about 1 s of timed work; "
                         "20 otherwise and for the reference arm)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["cc_ladder", "mps", "sweep", "table", "generic", "z3",
                                           "peps"],
                    default="cc_ladder")
    ap.add_argument("--stv", default="all",
                    help="generic: S,T,V (free modes of U, of V, contracted modes) or 'all' (the 27 "
                         "points with s, t, v in 1..3), G = 4, about 80e9 useful flops each")
    ap.add_argument("--case", default="CC1_a", help="table: a Table-2 case (" + ", ".join(WL.TABLE2) + ")")
    ap.add_argument("--sweep-g", type=int, default=16, help="G of the sweep workload (config 5)")
    ap.add_argument("--sweep-dims", default="512,128",
                    help="VIRT,OCC of the sweep workload: 512,128 (config 5) or 256,64 (the "
                         "secondary sweep at the CC ladder's dimensions)")
    ap.add_argument("--backward", action="store_true", help="sweep: time the backward pair too")
    ap.add_argument("--chain", action="store_true",
                    help="mps: keep X aligned between the two contractions (symctr_plan_chain)")
    ap.add_argument("--complex", action="store_true",
                    help="mps: complex tensors, E' = sum E A conj(A) (four real products per contraction)")
    ap.add_argument("--precision", choices=["split_bf16", "fp64", "tf32"], default="split_bf16")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--cc-dims", default=None,
                    help="VIRT,OCC for the cc_ladder workload (default 256,64); smaller cases are "
                         "for profiling captures")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.steps is None:
        args.steps = 160 if (args.impl == "ours" and args.workload == "cc_ladder") else 20

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    if args.workload == "generic":
        points = WL.GENERIC_STV if args.stv == "all" else [tuple(int(x) for x in args.stv.split(","))]
        for pt in points:
            args.stv_point = pt
            line = run_device(args, rank, world)
            line["stv"] = list(pt)
            if rank == 0:
                print(json.dumps(line), flush=True)
            import torch
            torch.cuda.empty_cache()
        line = None
    elif args.workload in ("sweep", "table"):
        line = run_device(args, rank, world)
    elif args.workload in ("z3", "peps"):
        line = run_small(args, rank, world)
    elif args.complex:
        line = run_complex(args, rank, world)
    else:
        line = run_ours(args, rank, world)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
