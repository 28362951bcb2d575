#!/usr/bin/env python3
"""Benchmark: time-to-P and block-GEMM throughput of the mixed-precision sign
iteration against the plain FP64 one, on the 4,096-water synthetic Hamiltonian
with 23/7 atom blocks (N = 151,552, eps 1e-6, tol 1e-8; split-BF16 tensor-core
products until ||X^2 - 1||_F / N < 1e-4, FP64 after).

One step = one complete sign iteration from the resident H to the density matrix
P (every product, filter, trace of the path).  value = executed block-product
flops (2 m n k per product, unpadded) of the mixed iteration / device time
(TFLOP/s); ms_per_step = its time-to-P.  The FP64 iteration of the same H, the
1,024-water FP64 configuration (13/5 blocks, eps 1e-7, tol 1e-9) and its mixed
ladder are timed beside it.  With --gpus N > 1 (torchrun) every rank solves its
own replica (the path is not sharded across GPUs here: replicas only, weak
scaling).

--impl reference times the FP64 CPU oracle (plain C) on the host cores, each step
a bounded sample of the same workload: the oracle's first product X0.X0 of the
4,096-water iteration restricted to a fixed set of block rows of its left factor.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# nominal dense rates (TFLOP/s) used to carry a measured bf16 peak over to FP64
NOMINAL_BF16 = 2250.0
NOMINAL_FP64 = 1.25
FALLBACK_BF16_BURST, FALLBACK_BF16_SUSTAINED = 1900.0, 1700.0

# DRAM bytes per flop of the FP64 block-product kernels: dram__bytes_read.sum +
# dram__bytes_write.sum over three captured launches (7x7, 23x7 and 7x23 classes of one product
# of the 512-water 23/7 case) divided by their executed DFMA flops (2 x
# sm__sass_thread_inst_executed_op_dfma_pred_on.sum): 2.680 GB / 21.63 GFLOP.  A full launch's
# traffic is this ratio times its flops (the larger systems are assumed to re-read operands at the
# same rate per flop).  Reset to None whenever the kernel changes.
SMM_F64_BYTES_PER_FLOP = 0.1239


def bf16_peak():
    """Measured bf16 tensor peak (sustained: the low tier runs inside a seconds-long step)."""
    try:
        pk = json.load(open(PEAKS_FILE))
        return float(pk["bf16_tflops_sustained"]), "measured bf16 sustained"
    except Exception:
        return FALLBACK_BF16_SUSTAINED, "fallback bf16 sustained"


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s)."""
    try:
        return float(json.load(open(PEAKS_FILE))["hbm_gbs"]), "measured copy"
    except Exception:
        return 6800.0, "fallback copy"


def fp64_derived_peak():
    """The measured bf16 peak times the nominal FP64/bf16 ratio (context only)."""
    try:
        bf16 = float(json.load(open(PEAKS_FILE))["bf16_tflops_sustained"])
    except Exception:
        bf16 = FALLBACK_BF16_SUSTAINED
    return bf16 * NOMINAL_FP64 / NOMINAL_BF16


def fp64_peak(gb, torch):
    """FP64 roofline peak: the higher of the library's DFMA and DMMA (m8n8k4) loops, measured
    on this GPU with every SM busy (MEASURED_PEAKS.json holds no FP64 figure)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    dfma = gb.lib().dbcsr_bench_peak(0, 4096, sms * 8, 256) / 1e3
    dmma = gb.lib().dbcsr_bench_peak(1, 4096, sms * 8, 256) / 1e3
    peak = max(dfma, dmma)
    return peak, {"peak_source": "measured FP64 (max of the DFMA and DMMA loops, dbcsr_bench_peak)",
                  "fp64_dfma_measured_tflops": dfma, "fp64_dmma_measured_tflops": dmma,
                  "fp64_derived_tflops": fp64_derived_peak(), "sms": sms}


class Clocks:
    """nvidia-smi samples during the timed region (median SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as f:
            out = parse_clock_samples(f)
        os.unlink(self.path)
        return out


def parse_clock_samples(lines):
    """Median SM clock, the largest max clock and the throttle reasons seen, from
    nvidia-smi lines of Clocks.Q (csv, noheader, nounits); None without samples."""
    rows = []
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            rows.append((float(f[1]), float(f[2]), f[5:9]))
        except ValueError:
            continue
    if not rows:
        return None
    sm = sorted(r[0] for r in rows)
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
            "samples": len(rows)}


def oracle_sample(h, w, steps: int):
    """The oracle's FP64 sign iteration on the same H, stopped after ``steps``
    Newton-Schulz steps (2 products each), with the library's norm-bound prescreen: a bounded
    sample of the workload."""
    from oracle import bsr, sign
    Ho = bsr.Mat.of(h.H)
    t0 = time.perf_counter()
    r = sign.sign_iterate(Ho, h.mu, w.eps_filter, w.tol, max_iter=steps, prescreen=True)
    dt = time.perf_counter() - t0
    return r.flops, dt, bsr.num_threads()


def sample_text(steps, flops, dt):
    return (f"first {steps} Newton-Schulz steps ({2 * steps} products) of the oracle's FP64 sign iteration "
            f"on the full H ({flops / 1e9:.0f} GFLOP executed in {dt:.1f} s, prescreen and norms included; the "
            f"oracle forms the blocks whose norm bound reaches eps, as the library does)")


class RowsSample:
    """A bounded sample of the sign iteration's first product for the oracle: X0 = (H - mu)/alpha
    (alpha the Gershgorin bound), and the product of its first ``rows`` block rows with the whole
    X0, filtered at eps, as the oracle computes it with the library's exact norm-bound prescreen
    (the candidate blocks whose bound reaches eps are formed, the same product list)."""

    def __init__(self, h, w, frac: float):
        from oracle import bsr, sign
        self.bsr = bsr
        Ho = bsr.Mat.of(h.H)
        alpha = sign.gershgorin(Ho, h.mu)
        self.X0 = bsr.add_identity(Ho, 1.0 / alpha, -h.mu / alpha)
        X = self.X0
        self.rows = max(1, int(round(frac * X.nblk)))
        nz = int(X.rp[self.rows])
        rp = X.rp.copy()
        rp[self.rows + 1:] = nz
        self.A = bsr.Mat(X.bs, rp, X.col[:nz].copy(), X.data[:int(X.boff[nz])].copy())
        self.eps = w.eps_filter

    def run(self):
        t0 = time.perf_counter()
        _, info = self.bsr.multiply(1.0, self.A, self.X0, eps=self.eps, info=True, prescreen=True)
        return float(info.flops), time.perf_counter() - t0, self.bsr.num_threads()

    def text(self, flops, dt):
        return (f"the oracle's first product X0.X0 of the iteration restricted to block rows 0..{self.rows - 1} "
                f"of {self.X0.nblk} ({flops / 1e9:.0f} GFLOP executed in {dt:.1f} s, prescreen and norms "
                f"included; the oracle forms the blocks whose norm bound reaches eps, as the library does)")


def one_core_sample(h, w):
    """The oracle's rows sample of the first product on one host thread (the thread count is
    restored afterwards)."""
    from oracle import bsr
    n0 = bsr.num_threads()
    bsr.set_num_threads(1)
    try:
        smp = RowsSample(h, w, CPU_1CORE_ROWS_FRAC)
        f, dt, cores = smp.run()
    finally:
        bsr.set_num_threads(n0)
    return {"value": f / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": smp.text(f, dt)}


# block rows of the 4,096-water X0 in one oracle sample (the prescreened product): a
# reference-arm step (about 6 s on 16 host cores) and the CPU baseline of the main line (the
# whole product, about 11 s)
REF_ROWS_FRAC, CPU_ROWS_FRAC = 1.0 / 2, 1.0
# the same sample on one host core: block rows of X0 in that sample (about 11 s)
CPU_1CORE_ROWS_FRAC = 1.0 / 16
HEADLINE_METRIC = "block-GEMM TFLOP/s & time-to-P at 1e-6 Ha/atom, mixed vs FP64 on GB300"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import synth
    w = synth.SIGN_4096
    h = synth.build_hamiltonian(w)
    smp = RowsSample(h, w, REF_ROWS_FRAC)
    for _ in range(args.warmup):
        smp.run()
    tot_f, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        f, dt, cores = smp.run()
        tot_f += f
        tot_t += dt
    value = tot_f / tot_t / 1e12
    sample = smp.text(f, dt) + ", one per step"
    out = {"metric": HEADLINE_METRIC, "value": value, "unit": "TFLOP/s",
           "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "sign-4096h2o-23-7-mixed-vs-fp64", "n_mol": w.n_mol, "N": w.n,
                      "blocks": {"O": w.basis[0], "H": w.basis[1]}, "eps_filter": w.eps_filter, "tol": w.tol,
                      "sample": sample},
           "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_batch(args, gb, synth, torch, barrier, small=False):
    """64 uneven water systems (n_mol log-uniform in [100, 2000], or in [20, 100] with small,
    O/H blocks per system): one batched sign iteration vs the same systems solved one after
    the other, in FP64 and with the mixed-precision ladder, with the FP64 block products
    launched per shape and with one work-queue launch per product."""
    from paper_2003_03868_gb300 import ranks
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    dist = None
    if world > 1:
        import torch.distributed as dist
    # every rank solves its own 64 systems (independent problems: weak scaling, no data exchange)
    ws = (synth.batch_systems(seed=synth.batch_seed(rank), lo=20, hi=100) if small
          else synth.batch_systems(seed=synth.batch_seed(rank)))
    hs = [synth.build_hamiltonian(w) for w in ws]
    stream = torch.cuda.current_stream()
    Hs = [gb.Matrix.of(h.H, stream=stream.cuda_stream) for h in hs]
    eps, tol = ws[0].eps_filter, ws[0].tol

    def leg(prec):
        for _ in range(args.warmup):
            gb.sign_iterate_batched(Hs, [0.0] * len(Hs), eps, tol, prec=prec)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            Ps, reps, st = gb.sign_iterate_batched(Hs, [0.0] * len(Hs), eps, tol, prec=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_b, flops_all = ranks.job_timing(e0.elapsed_time(e1) / args.steps, reps[0].flops, dist, "cuda")
        # the same systems one by one
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        seq = [gb.sign_iterate(H, 0.0, eps, tol, prec=prec) for H in Hs]
        s1.record(stream)
        torch.cuda.synchronize()
        ms_s = s0.elapsed_time(s1)
        de = max(abs(r.e_band - g.report.e_band) / h.n_atoms for r, g, h in zip(reps, seq, hs))
        its = [r.iterations for r in reps]
        return {"ms_per_step": ms_b, "value": flops_all / (ms_b * 1e-3) / 1e12, "unit": "TFLOP/s",
                "sequential_ms": ms_s, "speedup_vs_sequential": ms_s / ms_b,
                "systems_converged": sum(int(r.converged) for r in reps),
                "systems_stalled": sum(int(r.stalled) for r in reps),
                "max_de_band_per_atom_vs_sequential": de, "iterations_min": min(its), "iterations_max": max(its),
                "ms_multiply": reps[0].ms_multiply, "ms_low": reps[0].ms_low}, reps

    gb.set_fp64_schedule(gb.DBCSR_SCHEDULE_PER_SHAPE)
    f64, reps64 = leg(gb.DBCSR_FP64)
    mixed = None
    if not args.no_mixed:
        mixed, repsm = leg(gb.DBCSR_MIXED)
        mixed["speedup_vs_fp64_batched"] = f64["ms_per_step"] / mixed["ms_per_step"]
        mixed["max_de_band_per_atom_vs_fp64"] = max(abs(a.e_band - b.e_band) / h.n_atoms
                                                    for a, b, h in zip(repsm, reps64, hs))
        mixed["dtype"] = "bf16x3 (split bf16 hi+lo operands, fp32 accumulate), then f64"
    # the same legs with one work-queue launch per FP64 product (every shape of up to 9 slots
    # per lane in one launch)
    gb.set_fp64_schedule(gb.DBCSR_SCHEDULE_QUEUE)
    f64q, _ = leg(gb.DBCSR_FP64)
    mixedq = None if args.no_mixed else leg(gb.DBCSR_MIXED)[0]
    gb.set_fp64_schedule(gb.DBCSR_SCHEDULE_PER_SHAPE)
    queue = {"fp64": f64q, "mixed": mixedq,
             "fp64_queue_over_per_shape_time": f64q["ms_per_step"] / f64["ms_per_step"],
             "note": "DBCSR_SCHEDULE_QUEUE: one work-queue launch per FP64 product for the small shapes"}
    name = "batch-64-small" if small else "batch-64"
    out = {"metric": "block-GEMM TFLOP/s (batched sign iteration)", "value": f64["value"],
           "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": f64["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": name, "systems_per_rank": len(ws), "molecules_rank0": sum(w.n_mol for w in ws),
                      "atoms_rank0": sum(w.n_atoms for w in ws), "eps_filter": eps, "tol": tol,
                      "parallelism": f"independent systems, 64 per rank x{world}"},
           **{k: v for k, v in f64.items() if k not in ("value", "ms_per_step", "unit")}, "mixed": mixed,
           "queue_schedule": queue}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


# matrix products per iteration of the sign iteration of each order (the last iteration of a
# converged run forms only X X)
PRODUCTS_PER_ITERATION = {2: 2, 3: 3, 4: 4, 5: 4, 6: 5, 7: 5}


def run_orders(args, gb, synth, torch, barrier, w, h):
    """The sign iteration of every order from 2 (Newton-Schulz) to 7 on one system:
    time-to-P, iterations, products and flops in FP64, and with the mixed-precision ladder."""
    from paper_2003_03868_gb300 import ranks
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
    stream = torch.cuda.current_stream()
    H = gb.Matrix.of(h.H, stream=stream.cuda_stream)
    orders = [int(o) for o in args.orders.split(",")]
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = gb.lib().dbcsr_launch_count()

    def leg(order, prec):
        def one():
            return gb.sign_iterate(H, h.mu, w.eps_filter, w.tol, prec=prec, switch_tol=w.switch or 1e-4,
                                   order=order, verbose=args.verbose)
        for _ in range(args.warmup):
            one()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = ms_mult = ms_sym = ms_low = 0.0
        for _ in range(args.steps):
            r = one()
            flops += r.report.flops
            ms_mult += r.report.ms_multiply
            ms_sym += r.report.ms_symbolic
            ms_low += r.report.ms_low
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms, flops_all = ranks.job_timing(e0.elapsed_time(e1) / args.steps, flops / args.steps, dist, "cuda")
        it = r.report.iterations
        return {"order": order, "time_to_p_ms": ms, "iterations": it,
                # a run that converged or stalled ended on the X X of its last iteration
                "products": (PRODUCTS_PER_ITERATION[order] * (it - 1) + 1
                             if (r.report.converged or r.report.stalled) else None),
                "converged": bool(r.report.converged), "stalled": bool(r.report.stalled),
                "residual": r.report.residual, "flops_per_step": flops / args.steps,
                "value": flops_all / (ms * 1e-3) / 1e12,
                "kernel_tflops": flops / (ms_mult * 1e-3) / 1e12 if ms_mult > 0 else None,
                "ms_multiply": ms_mult / args.steps, "ms_symbolic": ms_sym / args.steps,
                "ms_low": ms_low / args.steps, "fp64_from_step": r.report.fp64_from,
                "trace_p": r.report.trace_p, "e_band": r.report.e_band}

    f64 = [leg(o, gb.DBCSR_FP64) for o in orders]
    mixed = [] if args.no_mixed else [leg(o, gb.DBCSR_MIXED) for o in orders]
    launches = gb.lib().dbcsr_launch_count() - l0

    # the block-sparse add of the even orders, A <- A + c B, on matrices of the iteration's size:
    # A = H (the pattern of X_0) and B = filter(H H) (the pattern of X^2), so that the union
    # is B's pattern grown by H's.  Bound by HBM: A and B read once, the sum written once.
    B = gb.Matrix(H.blk_size, stream.cuda_stream)
    gb.multiply(1.0, H, H, 0.0, B, w.eps_filter)
    def nel(M):
        return int(M.info()[2])
    ms_add, bytes_add = 0.0, 0.0
    for k in range(args.warmup + args.steps):
        A = H.copy()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        a0.record(stream)
        gb.add(1.0, A, 0.375, B)
        a1.record(stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            ms_add += a0.elapsed_time(a1)
            bytes_add += 8.0 * (nel(H) + nel(B) + nel(A))
        A.close()
    hp, hp_src = hbm_peak()
    gbs = bytes_add / (ms_add * 1e-3) / 1e9
    add = {"kernel": "dbcsr_add (k_union_rows x2, k_add_values)", "ms_per_call": ms_add / args.steps,
           "blocks": {"A": H.nnzb, "B": B.nnzb},
           "algorithmic_bytes_per_call": bytes_add / args.steps,
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hp, "unit": "GB/s", "frac": gbs / hp,
                        "peak_source": hp_src,
                        "note": "8 bytes per element of A, B and the sum; call time including its two "
                                "host readbacks of the union size"}}
    B.close()
    clk = clocks.stop()
    ref = next((x for x in f64 if x["order"] == 2), f64[0])
    for x in f64 + mixed:
        x["de_band_per_atom_vs_fp64_order2"] = abs(x["e_band"] - ref["e_band"]) / h.n_atoms
        x["speedup_vs_fp64_order2"] = ref["time_to_p_ms"] / x["time_to_p_ms"]
    best = min(f64, key=lambda x: x["time_to_p_ms"])
    out = {"metric": "time-to-P by sign-iteration order (FP64; best order)", "value": best["time_to_p_ms"],
           "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": best["time_to_p_ms"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name + "-orders", "n_mol": w.n_mol, "N": w.n,
                      "blocks": {"O": w.basis[0], "H": w.basis[1]}, "eps_filter": w.eps_filter, "tol": w.tol,
                      "orders": orders, "mixed_switch": w.switch or 1e-4,
                      "l2": "inputs larger than L2 (H alone is %.0f MB; 129 MB L2)" % (h.H.data.nbytes / 1e6),
                      "parallelism": f"replicas x{world}"},
           "best_order": best["order"], "fp64": f64, "mixed": mixed, "add": add, "gpu_launches": launches,
           "clocks": clk}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def run_nonorth(args, gb, synth, torch, barrier, w, h):
    """The density matrix in a non-orthogonal basis, P = (1 - sign(S^-1 K - mu 1)) S^-1 / 2,
    on the workload's water box with its synthetic overlap S: the square root S^-1/2, the
    congruences and the sign iteration, FP64 and mixed, for each order of --orders."""
    from paper_2003_03868_gb300 import ranks
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
    s_bm = synth.build_overlap(w)
    stream = torch.cuda.current_stream()
    K = gb.Matrix.of(h.H, stream=stream.cuda_stream)
    S = gb.Matrix.of(s_bm, stream=stream.cuda_stream)
    orders = [int(o) for o in args.orders.split(",")]
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = gb.lib().dbcsr_launch_count()

    def leg(order, prec):
        def one():
            return gb.sign_iterate_nonorth(K, S, h.mu, w.eps_filter, w.tol, prec=prec,
                                           switch_tol=w.switch or 1e-4, order=order, verbose=args.verbose)
        for _ in range(args.warmup):
            one()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = ms_mult = ms_sqrt = 0.0
        for _ in range(args.steps):
            r = one()
            flops += r.report.flops + r.report_sqrt.flops
            ms_mult += r.report.ms_multiply + r.report_sqrt.ms_multiply
            ms_sqrt += r.report_sqrt.ms_total
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms, flops_all = ranks.job_timing(e0.elapsed_time(e1) / args.steps, flops / args.steps, dist, "cuda")
        rr, rs = r.report, r.report_sqrt
        return {"order": order, "time_to_p_ms": ms, "sqrt_ms": ms_sqrt / args.steps,
                "value": flops_all / (ms * 1e-3) / 1e12,
                "kernel_tflops": flops / (ms_mult * 1e-3) / 1e12 if ms_mult > 0 else None,
                "flops_per_step": flops / args.steps,
                "sqrt": {"iterations": rs.iterations, "converged": bool(rs.converged), "stalled": bool(rs.stalled),
                         "residual": rs.residual, "scale": rs.alpha, "fp64_from_step": rs.fp64_from},
                "sign": {"iterations": rr.iterations, "converged": bool(rr.converged), "stalled": bool(rr.stalled),
                         "residual": rr.residual, "fp64_from_step": rr.fp64_from},
                "trace_ps": rr.trace_p, "trace_ps_error": rr.trace_p - h.n_occ, "e_band": rr.e_band}

    f64 = [leg(o, gb.DBCSR_FP64) for o in orders]
    mixed = [] if args.no_mixed else [leg(o, gb.DBCSR_MIXED) for o in orders]
    launches = gb.lib().dbcsr_launch_count() - l0
    clk = clocks.stop()
    ref = f64[0]
    for x in f64 + mixed:
        x["de_band_per_atom_vs_fp64_first"] = abs(x["e_band"] - ref["e_band"]) / h.n_atoms
    best = min(f64 + mixed, key=lambda x: x["time_to_p_ms"])
    out = {"metric": "time-to-P, non-orthogonal basis (S^-1/2, congruences, sign iteration)",
           "value": f64[0]["time_to_p_ms"], "unit": "ms", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": f64[0]["time_to_p_ms"], "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name + "-nonorth", "n_mol": w.n_mol, "N": w.n,
                      "blocks": {"O": w.basis[0], "H": w.basis[1]}, "eps_filter": w.eps_filter, "tol": w.tol,
                      "orders": orders, "overlap": "1 + 0.9 |D| / max row sum (synthetic; eigenvalues in [0.1, 1.9])",
                      "l2": "inputs larger than L2 (K alone is %.0f MB; 129 MB L2)" % (h.H.data.nbytes / 1e6),
                      "parallelism": f"replicas x{world}"},
           "fp64": f64, "mixed": mixed, "fastest": {"order": best["order"], "time_to_p_ms": best["time_to_p_ms"]},
           "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def run_purify(args, gb, synth, torch, barrier, w, h):
    """Canonical density matrices without a known mu: TC2 and TRS4 purification, and the sign
    method with mu bisected on H + 1.0 (the shift moves the gap off mu = 0) in the bracket
    [0.3, 5.0], next to the sign method at the known mid-gap mu.  The bracket's lower end
    lies just above the occupied band, as an estimate from an earlier step would: a trial
    mu inside a band makes sign(H - mu) non-local, and the filtered X then fills in toward
    a dense matrix (on 1,024 waters it passed a million blocks within ten steps)."""
    from paper_2003_03868_gb300 import ranks
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
    stream = torch.cuda.current_stream()
    H = gb.Matrix.of(h.H, stream=stream.cuda_stream)
    shift = 1.0
    Hs = H.copy()
    Hs.scale_shift(1.0, shift)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = gb.lib().dbcsr_launch_count()

    def leg(run):
        for _ in range(args.warmup):
            run()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = ms_mult = 0.0
        for _ in range(args.steps):
            r = run()
            flops += r.report.flops
            ms_mult += r.report.ms_multiply
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms, flops_all = ranks.job_timing(e0.elapsed_time(e1) / args.steps, flops / args.steps, dist, "cuda")
        return r, {"time_to_p_ms": ms, "value": flops_all / (ms * 1e-3) / 1e12, "flops_per_step": flops / args.steps,
                   "kernel_tflops": flops / (ms_mult * 1e-3) / 1e12 if ms_mult > 0 else None,
                   "iterations": r.report.iterations, "converged": bool(r.report.converged),
                   "trace_p": r.report.trace_p, "trace_p_error": r.report.trace_p - h.n_occ,
                   "e_band": r.report.e_band}

    rs, ref = leg(lambda: gb.sign_iterate(H, h.mu, w.eps_filter, w.tol))
    ref["residual"] = rs.report.residual
    legs = {"sign_known_mu": ref}
    for m in ("tc2", "trs4"):
        r, x = leg(lambda: gb.purify(H, h.n_occ, w.eps_filter, w.tol, method=m))
        x["idempotency"] = r.report.residual
        legs[m] = x
    bracket = (shift - 0.7, shift + 4.0)
    rm, x = leg(lambda: gb.sign_mu_search(Hs, h.n_occ, w.eps_filter, w.tol, mu_lo=bracket[0], mu_hi=bracket[1]))
    x.update({"mu": rm.mu, "evaluations": rm.evaluations, "shift": shift, "bracket": bracket,
              "e_band": rm.report.e_band - shift * h.n_occ})      # back to H's energy
    legs["sign_mu_search"] = x
    for k, x in legs.items():
        x["de_band_per_atom_vs_sign"] = abs(x["e_band"] - ref["e_band"]) / h.n_atoms
        x["speedup_vs_sign_known_mu"] = ref["time_to_p_ms"] / x["time_to_p_ms"]
    launches = gb.lib().dbcsr_launch_count() - l0
    clk = clocks.stop()
    best = min(("tc2", "trs4", "sign_mu_search"), key=lambda k: legs[k]["time_to_p_ms"])
    out = {"metric": "time-to-P without a known chemical potential (FP64; fastest canonical method)",
           "value": legs[best]["time_to_p_ms"], "unit": "ms", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": legs[best]["time_to_p_ms"], "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name + "-purify", "n_mol": w.n_mol, "N": w.n, "n_occ": h.n_occ,
                      "blocks": {"O": w.basis[0], "H": w.basis[1]}, "eps_filter": w.eps_filter, "tol": w.tol,
                      "mu_search_on": f"H + {shift} 1",
                      "l2": "inputs larger than L2 (H alone is %.0f MB; 129 MB L2)" % (h.H.data.nbytes / 1e6),
                      "parallelism": f"replicas x{world}"},
           "fastest": best, "legs": legs, "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def run_submatrix(args, gb, synth, torch, barrier):
    """The submatrix method against the sparse Newton-Schulz iteration on 6,192 waters with
    a minimal basis (SZV, N = 37,152): time-to-P and band-energy error per atom against a
    tight reference (Newton-Schulz at eps_filter 1e-9), as the paper compares them."""
    from paper_2003_03868_gb300 import ranks
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
    w = synth.SUBMATRIX_6192
    h = synth.build_hamiltonian(w)
    stream = torch.cuda.current_stream()
    H = gb.Matrix.of(h.H, stream=stream.cuda_stream)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = gb.lib().dbcsr_launch_count()
    ref = gb.sign_iterate(H, h.mu, 1e-9, 1e-10)
    e_ref = ref.report.e_band

    def leg(run):
        for _ in range(args.warmup):
            run()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            r = run()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms, flops_all = ranks.job_timing(e0.elapsed_time(e1) / args.steps, r.report.flops, dist, "cuda")
        return {"time_to_p_ms": ms, "iterations": r.report.iterations, "converged": bool(r.report.converged),
                "stalled": bool(r.report.stalled), "residual": r.report.residual, "gflop": r.report.flops * 1e-9,
                "trace_p_error": r.report.trace_p - h.n_occ,
                "de_band_per_atom": abs(r.report.e_band - e_ref) / h.n_atoms,
                "rel_energy_error": abs(r.report.e_band - e_ref) / abs(e_ref)}

    legs = {}
    for eps in (1e-5, 1e-6, 1e-7):
        legs[f"newton_schulz_eps{eps:g}"] = leg(lambda: gb.sign_iterate(H, h.mu, eps, 1e-9))
    x = leg(lambda: gb.submatrix_sign(H, h.mu, 1e-5, prec=gb.DBCSR_MIXED))
    x["dtype"] = "f32 (tf32 tensor-core GEMMs while r >= 1e-3, then fp32 GEMMs)"
    legs["submatrix_tf32_fp32"] = x
    launches = gb.lib().dbcsr_launch_count() - l0
    clk = clocks.stop()
    out = {"metric": "time-to-P and band-energy error, submatrix method vs Newton-Schulz (6,192 H2O, SZV)",
           "value": legs["submatrix_tf32_fp32"]["time_to_p_ms"], "unit": "ms", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": legs["submatrix_tf32_fp32"]["time_to_p_ms"],
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
           "data": "synthetic",
           "config": {"workload": w.name, "n_mol": w.n_mol, "N": w.n, "blocks": {"O": w.basis[0], "H": w.basis[1]},
                      "reference": "Newton-Schulz FP64, eps_filter 1e-9, tol 1e-10",
                      "e_band_reference": e_ref, "reference_iterations": ref.report.iterations,
                      "l2": "inputs larger than L2 (H alone is %.0f MB; 129 MB L2)" % (h.H.data.nbytes / 1e6),
                      "parallelism": f"replicas x{world}"},
           "legs": legs, "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def run_mult32(args, gb, synth, torch, barrier):
    """The single product C = A A of the 32-water decay matrix (N = 736, eps 1e-6): one-off
    products (stack builder, block products, filter, with their host round trips) against
    replays of a planned product (one CUDA graph of the numeric phase on fixed patterns)."""
    w = synth.DECAY_32
    a = synth.build_decay(w)
    stream = torch.cuda.current_stream()
    A = gb.Matrix.of(a, stream=stream.cuda_stream)
    C1 = gb.Matrix(A.blk_size, stream.cuda_stream)
    reps = max(20, 50 * args.steps)

    def timed(fn, n):
        for _ in range(args.warmup):
            fn()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    st = gb.multiply(1.0, A, A, 0.0, C1, w.eps_filter)
    ms_once = timed(lambda: gb.multiply(1.0, A, A, 0.0, C1, w.eps_filter, stats=False), reps)
    C2 = gb.Matrix(A.blk_size, stream.cuda_stream)
    plan = gb.Plan(1.0, A, A, C2, w.eps_filter)
    l0 = gb.lib().dbcsr_launch_count()
    ms_plan = timed(plan.execute, reps * 10)
    launches = (gb.lib().dbcsr_launch_count() - l0) // (args.warmup + reps * 10)
    out = {"metric": "block-GEMM GFLOP/s (single product C = A A, planned and replayed as a CUDA graph)",
           "value": st.flops / (ms_plan * 1e-3) / 1e9, "unit": "GFLOP/s", "n_gpus": 1, "steps": reps * 10,
           "warmup": args.warmup, "ms_per_step": ms_plan, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "n_mol": w.n_mol, "N": w.n, "blocks": {"O": 13, "H": 5},
                      "eps_filter": w.eps_filter, "l2": "inputs smaller than L2 (4.3 MB): a launch-bound case"},
           "flops_per_product": st.flops, "products": st.n_products, "blocks_formed": st.n_formed,
           "blocks_kept": st.n_kept, "one_off_ms": ms_once, "one_off_gflops": st.flops / (ms_once * 1e-3) / 1e9,
           "planned_speedup": ms_once / ms_plan, "gpu_launches": launches}
    plan.close()
    print(json.dumps(out))
    return 0


def run_predictor(args, gb, synth, torch, barrier):
    """Learned launch configurations on the 20,736-water mixed sign iteration (O/H = 23/7,
    N = 767,232): the MLP is trained on autotuner timings of triples drawn from {4..32}^3
    (the workload's own triples held out), predicts configurations for the workload's
    block shapes, and the mixed iteration runs with the default, the predicted and the
    exhaustively tuned configurations."""
    import numpy as np
    w = synth.SIGN_20736 if args.predictor_waters == synth.SIGN_20736.n_mol else synth.Workload(
        f"sign-{args.predictor_waters}h2o-23-7-mixed", args.predictor_waters, (23, 7), synth.configs.BASE_SEED + 14,
        1e-6, 1e-8, 1e-4)
    bo, bh = w.basis
    target = [(m, n, max(w.basis)) for m in (bo, bh) for n in (bo, bh)]
    rng = np.random.default_rng(20736)
    train = []
    while len(train) < args.train_triples:
        t = tuple(int(v) for v in rng.integers(4, 33, 3))
        if t not in target and t not in train:
            train.append(t)
    # the per-shape kernels are the FP64 ones (the BF16 products run on the tensor-core tier,
    # one tile shape for every block shape)
    precs = {"fp64": gb.DBCSR_FP64}
    gb.tune_clear()
    t0 = time.time()
    recs_train = {k: gb.autotune(train, p, stack_len=args.tune_stack, reps=3) for k, p in precs.items()}
    tune_train_s = time.time() - t0
    models, mlp_rep = {}, {}
    for k, p in precs.items():
        models[k], rep = gb.train_predictor(recs_train[k], p)
        mlp_rep[k] = {"loss_first": rep.loss_first, "loss_last": rep.loss_last, "ms": rep.ms,
                      "samples": len(recs_train[k])}
    pred = {k: gb.mlp_predict_best(models[k], target, p) for k, p in precs.items()}
    gb.tune_clear()
    t0 = time.time()
    recs_target = {k: gb.autotune(target, p, stack_len=args.tune_stack, reps=3) for k, p in precs.items()}
    tune_target_s = time.time() - t0
    best = {k: {t: gb.tune_get(p, *t)[0] for t in target} for k, p in precs.items()}
    gb.tune_clear()
    default = {k: gb.tune_get(p, 1, 1, 1)[0] for k, p in precs.items()}

    def key(c):
        return (c.tpb, c.ctas_per_sm, c.colmajor, c.prefetch2, c.split)

    # synthetic-stack time of the predicted and default configurations relative to the best
    ratios = {}
    for k in precs:
        rs = []
        for t, c in zip(target, pred[k]):
            tm = {key(r.cfg): r.ms for r in recs_target[k] if (r.m, r.n, r.k) == t}
            bt = min(tm.values())
            td = gb.time_configs(*t, [default[k]], stack_len=args.tune_stack, reps=3)[0]
            rs.append({"mnk": list(t), "predicted_over_best": tm[key(c)] / bt, "default_over_best": td / bt})
        ratios[k] = rs

    h = synth.build_hamiltonian(w)
    stream = torch.cuda.current_stream()
    H = gb.Matrix.of(h.H, stream=stream.cuda_stream)

    # the prediction checked by measured time, with the exhaustive search as its fallback
    gb.tune_clear()
    t0 = time.time()
    fallback = {k: gb.tune_predicted(models[k], target, p, stack_len=args.tune_stack, reps=3, tolerance=0.02)
                for k, p in precs.items()}
    fallback_s = time.time() - t0
    guarded = {k: {t: gb.tune_get(p, *t)[0] for t in target} for k, p in precs.items()}

    def install(which):
        gb.tune_clear()
        if which == "default":
            return
        for k, p in precs.items():
            chosen = {"mlp": dict(zip(target, pred[k])), "exhaustive": best[k], "mlp_fallback": guarded[k]}[which]
            for t, c in chosen.items():
                gb.tune_set(p, *t, c)

    def timed(prec):
        for _ in range(args.warmup):
            gb.sign_iterate(H, h.mu, w.eps_filter, w.tol, prec=prec, switch_tol=w.switch)
        barrier()
        l0 = gb.lib().dbcsr_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = 0.0
        for _ in range(args.steps):
            r = gb.sign_iterate(H, h.mu, w.eps_filter, w.tol, prec=prec, switch_tol=w.switch)
            fl += r.report.flops
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        return {"time_to_p_ms": ms, "gpu_launches": gb.lib().dbcsr_launch_count() - l0, "tflops": fl / args.steps / (ms * 1e-3) / 1e12, "iterations": r.report.iterations,
                "fp64_from_step": r.report.fp64_from, "converged": bool(r.report.converged),
                "stalled": bool(r.report.stalled), "e_band": r.report.e_band, "trace_p": r.report.trace_p,
                "ms_low": r.report.ms_low, "ms_multiply": r.report.ms_multiply}

    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    runs = {}
    for which in ("default", "mlp", "mlp_fallback", "exhaustive"):
        install(which)
        runs[which] = timed(gb.DBCSR_MIXED)
    install("exhaustive")
    fp64 = timed(gb.DBCSR_FP64)
    clk = clocks.stop()
    for v in runs.values():
        v["de_band_per_atom_vs_fp64"] = abs(v["e_band"] - fp64["e_band"]) / h.n_atoms
    out = {"metric": "block-GEMM TFLOP/s (mixed sign iteration, MLP-predicted launch configurations)",
           "value": runs["mlp"]["tflops"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": runs["mlp"]["time_to_p_ms"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 then f64", "data": "synthetic",
           "config": {"workload": w.name, "n_mol": w.n_mol, "N": w.n, "blocks": {"O": bo, "H": bh},
                      "eps_filter": w.eps_filter, "tol": w.tol, "switch": w.switch,
                      "l2": "inputs larger than L2 (H alone is %.0f MB)" % (h.H.data.nbytes / 1e6)},
           "runs": runs, "fp64_exhaustive": fp64,
           "mlp_over_exhaustive_time": runs["mlp"]["time_to_p_ms"] / runs["exhaustive"]["time_to_p_ms"],
           "default_over_exhaustive_time": runs["default"]["time_to_p_ms"] / runs["exhaustive"]["time_to_p_ms"],
           "mixed_speedup_vs_fp64": fp64["time_to_p_ms"] / runs["mlp"]["time_to_p_ms"],
           "synthetic_ratios": ratios, "mlp": mlp_rep,
           "tuning": {"train_triples": len(train), "stack_len": args.tune_stack, "train_s": tune_train_s,
                      "target_s": tune_target_s, "fallback_s": fallback_s,
                      "fell_back": {k: [list(t) for t, f in zip(target, v) if f] for k, v in fallback.items()},
                      "fallback_tolerance": 0.02},
           "clocks": clk, "gpu_launches": runs["mlp"]["gpu_launches"]}
    print(json.dumps(out))
    return 0


def sign_leg(gb, torch, barrier, H, h, w, steps, warmup, prec, **kw):
    """``steps`` timed sign iterations of H (after ``warmup`` untimed ones) on the current stream:
    device time-to-P from CUDA events around the timed calls, and the reports' work counters."""
    stream = torch.cuda.current_stream()

    def one():
        return gb.sign_iterate(H, h.mu, w.eps_filter, w.tol, prec=prec, switch_tol=w.switch or 1e-4, **kw)

    for _ in range(warmup):
        one()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    acc = {k: 0.0 for k in ("flops", "flops_low", "ms_low", "ms_multiply", "ms_symbolic", "ms_filter",
                            "bytes_min_fp64", "launches_fp64", "flops_tensor", "bytes_tensor")}
    for _ in range(steps):
        r = one()
        for k in acc:
            acc[k] += float(getattr(r.report, k))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    return r, ms, acc


def fp64_roofline(acc, ms, steps, peak, peak_info):
    """k_smm_f64 in a step: executed FP64 flops over the FP64 block-product kernels' own time
    (CUDA events the library records around them on the launching stream)."""
    f = acc["flops"] - acc["flops_low"]
    t = acc["ms_multiply"] - acc["ms_low"]
    nl = acc["launches_fp64"]
    achieved = f / (t * 1e-3) / 1e12 if t > 0 else 0.0
    return {"bound": "fp64", "kernel": "k_smm_f64", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": SMM_F64_BYTES_PER_FLOP * f / nl if SMM_F64_BYTES_PER_FLOP and nl else None,
            "traffic_note": "DRAM bytes per launch: bytes per flop of a small-case capture x flops per launch",
            "kernel_share_of_step": t / ms if ms > 0 else None, "launches_per_step": nl / steps,
            "compulsory_bytes_per_launch": acc["bytes_min_fp64"] / nl if nl else None,
            "ms_per_step": t / steps, **peak_info}


def low_roofline(acc, ms, steps):
    """The low tier's split-BF16 block-product kernel against the measured sustained bf16 peak."""
    bpk, bpk_src = bf16_peak()
    low_alg = acc["flops_low"] / (acc["ms_low"] * 1e-3) / 1e12 if acc["ms_low"] > 0 else 0.0
    t = acc["ms_low"] * 1e-3
    return {"bound": "tensor", "kernel": LOW_TIER_KERNEL, "achieved": 3 * low_alg, "unit": "TFLOP/s",
            "peak": bpk, "frac": 3 * low_alg / bpk, "peak_source": bpk_src, "algorithmic_tflops": low_alg,
            "executed_tflops": acc["flops_tensor"] / t / 1e12 if t > 0 else None,
            "padding_factor": acc["flops_tensor"] / (3 * acc["flops_low"]) if acc["flops_low"] > 0 else None,
            "copy_gbs": acc["bytes_tensor"] / t / 1e9 if t > 0 else None,
            "kernel_share_of_step": acc["ms_low"] / ms if ms > 0 else None, "ms_per_step": acc["ms_low"] / steps,
            "note": "achieved counts the three bf16 products (hi*hi, hi*lo, lo*hi) of every unpadded 2mnk "
                    "block product; executed_tflops counts every issued MMA (group-tile padding included); "
                    "the time is k_lowtier's own (CUDA events around its launch); the operand packing is "
                    "timed with the symbolic phase"}


LOW_TIER_KERNEL = "k_lowtier"


def run_headline(args, gb, synth, torch, barrier, dist, rank, world, local):
    """The metric's own configuration: mixed vs FP64 sign iteration on 4,096 waters (23/7 blocks),
    with the 1,024-water FP64 configuration (13/5) and its mixed ladder beside it."""
    import numpy as np
    from paper_2003_03868_gb300 import ranks
    w = synth.SIGN_4096
    h = synth.build_hamiltonian(w)
    stream = torch.cuda.current_stream()
    H = gb.Matrix.of(h.H, stream=stream.cuda_stream)
    side_steps = max(1, min(args.steps, args.side_steps))
    peak, peak_info = fp64_peak(gb, torch)
    # the FP64 kernels' configurations for the block shapes of both workloads, picked by the
    # autotuner (untimed setup, like a tuned parameter table shipped with the library)
    tuning = None
    gb.tune_clear()
    if not args.no_tune:
        t0 = time.time()
        triples = [(m, n, max(b)) for b in ((23, 7), (13, 5)) for m in b for n in b]
        recs = gb.autotune(triples, gb.DBCSR_FP64, stack_len=args.tune_stack, reps=3)
        d = gb.tune_get(gb.DBCSR_FP64, 1, 1, 1)[0]
        tuning = {"seconds": time.time() - t0, "stack_len": args.tune_stack, "configs_timed": len(recs),
                  "triples": [{"mnk": list(t), "best_ms": min(r.ms for r in recs if (r.m, r.n, r.k) == t),
                               "default_ms": float(gb.time_configs(*t, [d], stack_len=args.tune_stack, reps=3)[0]),
                               "split": gb.tune_get(gb.DBCSR_FP64, *t)[0].split} for t in triples]}

    # main leg: the mixed ladder (split BF16 while r >= 1e-4, then FP64), args.steps timed steps
    clocks = Clocks(local)
    l0 = gb.lib().dbcsr_launch_count()
    for _ in range(args.warmup):
        gb.sign_iterate(H, h.mu, w.eps_filter, w.tol, prec=gb.DBCSR_MIXED, switch_tol=w.switch)
    barrier()
    clocks.start()
    l1 = gb.lib().dbcsr_launch_count()
    rm, ms_m, acc_m = sign_leg(gb, torch, barrier, H, h, w, args.steps, 0, gb.DBCSR_MIXED)
    launches = gb.lib().dbcsr_launch_count() - l1
    clk = clocks.stop()
    ms_all, flops_all = ranks.job_timing(ms_m, acc_m["flops"], dist, "cuda")
    value = flops_all / (ms_all * 1e-3) / 1e12

    fp64 = low_correction = c2 = None
    de_vs_fp64 = speedup = None
    if not args.main_only:
        fp64, low_correction, de_vs_fp64, speedup = headline_side_legs(args, gb, torch, barrier, dist, H, h, w,
                                                                       side_steps, peak, peak_info, rm, ms_all)

    # end to end through the public API: H from pinned host memory each step, P exported to pinned
    # host memory each step (row pointers, block columns, values), the report read back
    e2e = None
    if not args.no_e2e:
        e2e = headline_e2e(args, gb, torch, barrier, stream, h, w, rm)

    # the 1,024-water configuration beside it: FP64 (eps 1e-7, tol 1e-9) and the mixed ladder
    if not args.main_only:
        c2 = headline_sign1024(gb, synth, torch, barrier, stream, side_steps, peak, peak_info)

    f_roof = fp64_roofline(acc_m, ms_m, args.steps, peak, peak_info)
    l_roof = low_roofline(acc_m, ms_m, args.steps)
    dominant = f_roof if f_roof["kernel_share_of_step"] >= (l_roof["kernel_share_of_step"] or 0.0) else l_roof
    out = {"metric": HEADLINE_METRIC, "value": value, "unit": "TFLOP/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3+f64",
           "data": "synthetic",
           "config": {"workload": "sign-4096h2o-23-7-mixed-vs-fp64", "n_mol": w.n_mol, "N": w.n,
                      "blocks": {"O": w.basis[0], "H": w.basis[1]}, "eps_filter": w.eps_filter, "tol": w.tol,
                      "switch": w.switch, "mu": h.mu,
                      "l2": "inputs larger than L2 (H alone is %.0f MB; 129 MB L2)" % (h.H.data.nbytes / 1e6),
                      "parallelism": f"replicas x{world}"},
           "time_to_p_ms": ms_all / args.steps, "iterations": rm.report.iterations,
           "fp64_from_step": rm.report.fp64_from, "converged": bool(rm.report.converged),
           "stalled": bool(rm.report.stalled), "residual": rm.report.residual, "trace_p": rm.report.trace_p,
           "n_occ": h.n_occ, "e_band": rm.report.e_band, "e_band_both_spins": 2.0 * rm.report.e_band,
           "de_band_per_atom_vs_fp64": de_vs_fp64, "speedup_vs_fp64": speedup,
           "ms_per_step_phases": {k: acc_m[k] / args.steps for k in ("ms_low", "ms_multiply", "ms_symbolic",
                                                                      "ms_filter")},
           "gpu_launches": launches, "clocks": clk, "roofline": dominant,
           "fp64_tail_roofline": f_roof, "low_tier_roofline": l_roof,
           "fp64": fp64, "low_correction": low_correction, "e2e": e2e, "sign_1024h2o": c2, "tuning": tuning}
    if not args.main_only:
        shapes = [(23, 23, 23), (23, 7, 23), (7, 23, 23), (7, 7, 23)]
        out["vendor_small_gemm"] = {
            "fp64": vendor_small_gemm(torch, shapes, torch.float64),
            "bf16": vendor_small_gemm(torch, shapes, torch.bfloat16),
            "note": "torch.bmm (cuBLAS) on 131,072 independent products per block shape, untimed by the step; "
                    "compare k_smm_f64 (roofline.achieved) and k_lowtier (low_tier_roofline.algorithmic_tflops)"}
    if rank == 0 and world == 1 and not args.no_cpu:
        smp = RowsSample(h, w, CPU_ROWS_FRAC)
        f, dt, cores = smp.run()
        out["cpu_baseline"] = {"value": f / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                               "sample": smp.text(f, dt), "single_core": one_core_sample(h, w)}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def vendor_small_gemm(torch, shapes, dtype, nprod=131072, reps=5):
    """Context for the block-product kernels: the vendor library's batched GEMM (torch.bmm, which
    calls cuBLAS) on independent products of the block shapes, nprod per batch, timed with CUDA
    events after a warm-up.  Not the same work as a block-sparse product (no accumulation of a
    stack into one C block, no prescreen): a rate for the small shapes, nothing more."""
    out = []
    for (m, n, k) in shapes:
        a = torch.rand(nprod, m, k, dtype=dtype, device="cuda")
        b = torch.rand(nprod, k, n, dtype=dtype, device="cuda")
        c = torch.empty(nprod, m, n, dtype=dtype, device="cuda")
        torch.bmm(a, b, out=c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.bmm(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out.append({"mnk": [m, n, k], "tflops": 2.0 * m * n * k * nprod / (ms * 1e-3) / 1e12, "ms": ms})
        del a, b, c
    return out


def headline_side_legs(args, gb, torch, barrier, dist, H, h, w, side_steps, peak, peak_info, rm, ms_all):
    """The plain FP64 iteration of the headline H and the low-correction option beside the mixed leg."""
    from paper_2003_03868_gb300 import ranks
    rf, ms_f, acc_f = sign_leg(gb, torch, barrier, H, h, w, side_steps, 1, gb.DBCSR_FP64)
    ms_f_all, flops_f_all = ranks.job_timing(ms_f, acc_f["flops"], dist, "cuda")
    fp64 = {"time_to_p_ms": ms_f_all / side_steps, "value": flops_f_all / (ms_f_all * 1e-3) / 1e12,
            "unit": "TFLOP/s", "steps": side_steps, "iterations": rf.report.iterations,
            "converged": bool(rf.report.converged), "stalled": bool(rf.report.stalled),
            "residual": rf.report.residual, "trace_p": rf.report.trace_p, "e_band": rf.report.e_band,
            "roofline": fp64_roofline(acc_f, ms_f, side_steps, peak, peak_info),
            "ms_per_step": {k: acc_f[k] / side_steps for k in ("ms_multiply", "ms_symbolic", "ms_filter")}}

    # option: the FP64 tail's update correction in split BF16
    rc, ms_c, _ = sign_leg(gb, torch, barrier, H, h, w, side_steps, 1, gb.DBCSR_MIXED, low_correction=True)
    low_correction = {"time_to_p_ms": ms_c / side_steps, "speedup_vs_fp64": ms_f / ms_c * 1.0,
                      "steps": side_steps, "iterations": rc.report.iterations, "converged": bool(rc.report.converged),
                      "de_band_per_atom_vs_fp64": abs(rc.report.e_band - rf.report.e_band) / h.n_atoms,
                      "note": "DBCSR_SIGN_LOW_CORRECTION: X*X, residual, test, filter and traces in FP64; "
                              "the update's correction product in split BF16"}
    return fp64, low_correction, abs(rm.report.e_band - rf.report.e_band) / h.n_atoms, \
        fp64["time_to_p_ms"] / (ms_all / args.steps)


def headline_e2e(args, gb, torch, barrier, stream, h, w, rm):
    """The mixed sign iteration end to end: H from pinned host memory, P exported to pinned host memory."""
    import numpy as np
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    data_pin = torch.from_numpy(np.ascontiguousarray(h.H.data)).pin_memory()
    rows_pin = torch.from_numpy(np.ascontiguousarray(
        np.repeat(np.arange(h.H.blk_size.shape[0], dtype=np.int32), np.diff(h.H.row_ptr)))).pin_memory()
    cols_pin = torch.from_numpy(np.ascontiguousarray(h.H.col, dtype=np.int32)).pin_memory()
    nb, nzp, nep = rm.P.info()
    cap_z, cap_e = int(nzp * 1.25) + 1024, int(nep * 1.25) + 65536
    p_rp = torch.empty(nb + 1, dtype=torch.int64).pin_memory()
    p_col = torch.empty(cap_z, dtype=torch.int32).pin_memory()
    p_dat = torch.empty(cap_e, dtype=torch.float64).pin_memory()
    h2d = int(data_pin.numel() * 8 + rows_pin.numel() * 4 + cols_pin.numel() * 4)
    barrier()
    f0 = time.perf_counter()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    fl, d2h = 0.0, 0
    for _ in range(e2e_steps):
        Hs = gb.Matrix.from_pinned(h.H.blk_size, rows_pin.data_ptr(), cols_pin.data_ptr(), cols_pin.numel(),
                                   data_pin.data_ptr(), stream=stream.cuda_stream)
        rr = gb.sign_iterate(Hs, h.mu, w.eps_filter, w.tol, prec=gb.DBCSR_MIXED, switch_tol=w.switch)
        d2h += rr.P.export_to(p_rp.data_ptr(), p_col.data_ptr(), cap_z, p_dat.data_ptr(), cap_e)
        fl += rr.report.flops
        d2h += 3 * 8                                                # trace, band energy, residual
        _ = (float(rr.report.e_band), float(rr.report.trace_p), float(rr.report.residual))
        rr.P.close()
        Hs.close()
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms2 = ev[0].elapsed_time(ev[1])
    e2e = {"value": fl / (ms2 * 1e-3) / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h // e2e_steps, "ms_per_step": ms2 / e2e_steps, "steps": e2e_steps,
           "wall_s": time.perf_counter() - f0,
           "note": "dbcsr_put_blocks + dbcsr_finalize from pinned host buffers, the mixed sign iteration, "
                   "dbcsr_export of P into pinned host buffers"}
    return e2e


def headline_sign1024(gb, synth, torch, barrier, stream, side_steps, peak, peak_info):
    """The 1,024-water configuration (13/5): FP64 and the mixed ladder."""
    w2 = synth.SIGN_1024
    h2 = synth.build_hamiltonian(w2)
    H2 = gb.Matrix.of(h2.H, stream=stream.cuda_stream)
    r2f, ms2f, acc2f = sign_leg(gb, torch, barrier, H2, h2, w2, side_steps, 1, gb.DBCSR_FP64)
    r2m, ms2m, acc2m = sign_leg(gb, torch, barrier, H2, h2, w2, side_steps, 1, gb.DBCSR_MIXED)
    c2 = {"workload": w2.name, "n_mol": w2.n_mol, "N": w2.n, "blocks": {"O": w2.basis[0], "H": w2.basis[1]},
          "eps_filter": w2.eps_filter, "tol": w2.tol, "steps": side_steps,
          "fp64": {"time_to_p_ms": ms2f / side_steps, "value": acc2f["flops"] / (ms2f * 1e-3) / 1e12,
                   "iterations": r2f.report.iterations, "converged": bool(r2f.report.converged),
                   "stalled": bool(r2f.report.stalled), "residual": r2f.report.residual,
                   "trace_p": r2f.report.trace_p, "e_band": r2f.report.e_band,
                   "roofline": fp64_roofline(acc2f, ms2f, side_steps, peak, peak_info)},
          "mixed": {"time_to_p_ms": ms2m / side_steps, "value": acc2m["flops"] / (ms2m * 1e-3) / 1e12,
                    "speedup_vs_fp64": ms2f / ms2m, "iterations": r2m.report.iterations,
                    "fp64_from_step": r2m.report.fp64_from, "converged": bool(r2m.report.converged),
                    "stalled": bool(r2m.report.stalled),
                    "de_band_per_atom_vs_fp64": abs(r2m.report.e_band - r2f.report.e_band) / h2.n_atoms,
                    "low_tier_roofline": low_roofline(acc2m, ms2m, side_steps)},
          "unit": "TFLOP/s", "unit_time": "ms"}
    H2.close()
    return c2


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision leg")
    ap.add_argument("--ref-steps", type=int, default=1, help="Newton-Schulz steps per oracle sample (reference arm)")
    ap.add_argument("--cpu-steps", type=int, default=2, help="Newton-Schulz steps in the oracle CPU baseline")
    ap.add_argument("--side-steps", type=int, default=3, help="timed steps of the side legs of the default run")
    ap.add_argument("--e2e-steps", type=int, default=5, help="timed steps of the end-to-end leg")
    ap.add_argument("--no-tune", action="store_true", help="default run: skip the autotuning of the block shapes")
    ap.add_argument("--main-only", action="store_true",
                    help="default run: the mixed leg alone (no FP64, low-correction or 1,024-water legs), "
                         "for launch lists whose kernel shares match the headline step")
    ap.add_argument("--workload", default="sign-4096h2o-mixed",
                    choices=["sign-4096h2o-mixed", "sign-1024h2o", "sign-512h2o", "sign-512h2o-23-7", "sign-4096h2o", "batch-64", "batch-64-small",
                             "sign-20736h2o-mlp", "mult-32h2o", "sign-1024h2o-orders", "sign-4096h2o-orders",
                             "sign-1024h2o-nonorth", "sign-4096h2o-nonorth", "sign-1024h2o-purify",
                             "sign-4096h2o-purify", "submatrix-6192h2o-szv"],
                    help="sign-4096h2o-mixed (default): the mixed vs FP64 sign iteration on 4,096 waters (23/7) "
                         "with the 1,024-water configuration beside it; sign-1024h2o: the FP64 iteration on "
                         "1,024 waters (13/5) with its ladders; sign-512h2o, sign-512h2o-23-7: smaller cases for profiler captures; sign-4096h2o: "
                         "4,096 waters with O/H blocks 23/7 (FP64 and mixed); batch-64: 64 uneven systems "
                         "batched vs one by one; sign-20736h2o-mlp: the mixed iteration on 20,736 waters with "
                         "default, MLP-predicted and exhaustively tuned launch configurations; mult-32h2o: the "
                         "32-water product, one-off vs planned (CUDA graph); sign-1024h2o-orders, "
                         "sign-4096h2o-orders: the sign iteration of orders 2 to 7 (--orders), FP64 and mixed; "
                         "sign-1024h2o-nonorth, sign-4096h2o-nonorth: the density matrix with an overlap matrix S; "
                         "sign-1024h2o-purify, sign-4096h2o-purify: TC2, TRS4 and the mu search; "
                         "submatrix-6192h2o-szv: the submatrix method against Newton-Schulz")
    ap.add_argument("--orders", default="2,3,4,5,6,7", help="sign-*-orders: the orders to time")
    ap.add_argument("--train-triples", type=int, default=48, help="sign-20736h2o-mlp: autotuned training triples")
    ap.add_argument("--tune-stack", type=int, default=500000, help="products of the autotuner's synthetic stacks")
    ap.add_argument("--predictor-waters", type=int, default=20736, help="sign-20736h2o-mlp: waters of the system")
    ap.add_argument("--verbose", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    import paper_2003_03868_gb300 as gb
    try:
        gb.lib()
    except ImportError:
        from paper_2003_03868_gb300 import build
        build.build()
        gb.lib()
    import synth

    if args.workload == "sign-4096h2o-mixed":
        return run_headline(args, gb, synth, torch, barrier, dist, rank, world, local)
    if args.workload in ("batch-64", "batch-64-small"):
        return run_batch(args, gb, synth, torch, barrier, small=args.workload == "batch-64-small")
    if args.workload == "submatrix-6192h2o-szv":
        return run_submatrix(args, gb, synth, torch, barrier)
    if args.workload in ("sign-20736h2o-mlp", "mult-32h2o"):
        # one-GPU studies: under torchrun rank 0 alone runs them
        if rank != 0:
            if dist:
                dist.destroy_process_group()
            return 0
        return (run_predictor if args.workload == "sign-20736h2o-mlp" else run_mult32)(args, gb, synth, torch,
                                                                                         lambda: torch.cuda.synchronize())
    w = {"sign-1024h2o": synth.SIGN_1024, "sign-4096h2o": synth.SIGN_4096,
         "sign-1024h2o-orders": synth.SIGN_1024, "sign-4096h2o-orders": synth.SIGN_4096,
         "sign-1024h2o-nonorth": synth.SIGN_1024, "sign-4096h2o-nonorth": synth.SIGN_4096,
         "sign-1024h2o-purify": synth.SIGN_1024, "sign-4096h2o-purify": synth.SIGN_4096,
         "sign-512h2o": synth.Workload("sign-512h2o-dzvp-fp64", 512, (13, 5), synth.configs.BASE_SEED + 12, 1e-7, 1e-9),
         "sign-512h2o-23-7": synth.Workload("sign-512h2o-23-7", 512, (23, 7), synth.configs.BASE_SEED + 13, 1e-6, 1e-8,
                                            1e-4)}[args.workload]
    h = synth.build_hamiltonian(w)
    if args.workload.endswith("-orders"):
        return run_orders(args, gb, synth, torch, barrier, w, h)
    if args.workload.endswith("-nonorth"):
        return run_nonorth(args, gb, synth, torch, barrier, w, h)
    if args.workload.endswith("-purify"):
        return run_purify(args, gb, synth, torch, barrier, w, h)
    stream = torch.cuda.current_stream()
    H = gb.Matrix.of(h.H, stream=stream.cuda_stream)

    def step():
        return gb.sign_iterate(H, h.mu, w.eps_filter, w.tol, verbose=args.verbose)

    for _ in range(args.warmup):
        r = step()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = gb.lib().dbcsr_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    flops, ms_mult, iters, ebands, trp, conv = 0.0, 0.0, [], [], [], []
    bytes_min, smm_launches = 0.0, 0
    for _ in range(args.steps):
        r = step()
        flops += r.report.flops
        ms_mult += r.report.ms_multiply
        bytes_min += r.report.bytes_min_fp64
        smm_launches += r.report.launches_fp64
        iters.append(r.report.iterations)
        ebands.append(r.report.e_band)
        trp.append(r.report.trace_p)
        conv.append(bool(r.report.converged))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = gb.lib().dbcsr_launch_count() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    from paper_2003_03868_gb300 import ranks
    ms_all, flops_all = ranks.job_timing(ms, flops, dist, "cuda")
    value = flops_all / (ms_all * 1e-3) / 1e12

    # the same workload with the precision ladder: split-BF16 tensor-core products while r >= 1e-4,
    # then FP64 (and, for comparison, the ladder with plain BF16 products)
    mixed = None
    if not args.no_mixed:
        def time_mixed(low, correction=False):
            def one():
                return gb.sign_iterate(H, h.mu, w.eps_filter, w.tol, prec=gb.DBCSR_MIXED, switch_tol=1e-4,
                                       low=low, low_correction=correction, verbose=args.verbose)
            for _ in range(args.warmup):
                one()
            barrier()
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            acc = {"flops": 0.0, "flops_low": 0.0, "ms_low": 0.0, "ms_multiply": 0.0, "ms_symbolic": 0.0,
                   "ms_filter": 0.0, "flops_tensor": 0.0, "bytes_tensor": 0.0}
            for _ in range(args.steps):
                rm = one()
                for k in acc:
                    acc[k] += getattr(rm.report, k)
            m1.record(stream)
            torch.cuda.synchronize()
            barrier()
            return rm, m0.elapsed_time(m1), acc

        rm, mms, acc = time_mixed(gb.DBCSR_BF16X3)
        mixed = {"time_to_p_ms": mms / args.steps, "value": acc["flops"] / (mms * 1e-3) / 1e12, "unit": "TFLOP/s",
                 "speedup_vs_fp64": (ms_all / args.steps) / (mms / args.steps),
                 "iterations": rm.report.iterations, "fp64_from_step": rm.report.fp64_from,
                 "converged": bool(rm.report.converged), "stalled": bool(rm.report.stalled),
                 "residual": rm.report.residual, "trace_p": rm.report.trace_p, "e_band": rm.report.e_band,
                 "de_band_per_atom_vs_fp64": abs(rm.report.e_band - ebands[-1]) / h.n_atoms,
                 "switch": 1e-4,
                 "dtype": "bf16x3 (split bf16 hi+lo operands, fp32 accumulate), then f64",
                 "ms_per_step": {k: acc[k] / args.steps for k in ("ms_low", "ms_multiply", "ms_symbolic", "ms_filter")},
                 "low_tier_roofline": low_roofline(acc, mms, args.steps)}
        rp_, mps, _ = time_mixed(gb.DBCSR_BF16)
        mixed["plain_bf16"] = {"time_to_p_ms": mps / args.steps, "iterations": rp_.report.iterations,
                               "fp64_from_step": rp_.report.fp64_from,
                               "de_band_per_atom_vs_fp64": abs(rp_.report.e_band - ebands[-1]) / h.n_atoms}
        # option beyond the FP64 tail: its update correction X (X^2 - 1) in split BF16
        rc_, mcs, _ = time_mixed(gb.DBCSR_BF16X3, correction=True)
        mixed["low_correction"] = {"time_to_p_ms": mcs / args.steps,
                                   "speedup_vs_fp64": (ms_all / args.steps) / (mcs / args.steps),
                                   "iterations": rc_.report.iterations, "converged": bool(rc_.report.converged),
                                   "stalled": bool(rc_.report.stalled), "residual": rc_.report.residual,
                                   "de_band_per_atom_vs_fp64": abs(rc_.report.e_band - ebands[-1]) / h.n_atoms,
                                   "note": "DBCSR_SIGN_LOW_CORRECTION: X*X, residual, test, filter and traces "
                                           "in FP64; the update's correction product in split BF16"}

    # end to end through the public API: inputs from pinned host memory, report read back
    e2e = None
    if not args.no_e2e:
        data_pin = torch.from_numpy(np.ascontiguousarray(h.H.data)).pin_memory()
        h2d = int(h.H.data.nbytes + 2 * 4 * h.H.col.shape[0])
        barrier()
        f0 = time.perf_counter()
        e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e2[0].record(stream)
        fl = 0.0
        for _ in range(args.steps):
            Hs = gb.Matrix.from_blocks(h.H.blk_size, h.H.row_ptr, h.H.col, None, stream=stream.cuda_stream,
                                       data_ptr=data_pin.data_ptr())
            rr = gb.sign_iterate(Hs, h.mu, w.eps_filter, w.tol)
            fl += rr.report.flops
            _ = float(rr.report.e_band)
            Hs.close()
        e2[1].record(stream)
        torch.cuda.synchronize()
        ms2 = e2[0].elapsed_time(e2[1])
        e2e = {"value": fl / (ms2 * 1e-3) / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 8 * 3, "ms_per_step": ms2 / args.steps,
               "wall_s": time.perf_counter() - f0}

    peak, peak_info = fp64_peak(gb, torch)
    achieved = flops / (ms_mult * 1e-3) / 1e12 if ms_mult > 0 else 0.0
    roofline = {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "kernel": "k_smm_f64",
                "traffic": (SMM_F64_BYTES_PER_FLOP * flops / smm_launches
                            if SMM_F64_BYTES_PER_FLOP and smm_launches else None),
                "kernel_share_of_step": ms_mult / ms if ms > 0 else None,
                "launches_per_step": smm_launches / args.steps,
                "compulsory_bytes_per_launch": bytes_min / smm_launches if smm_launches else None, **peak_info}

    out = {"metric": "block-GEMM TFLOP/s (FP64 sign iteration, time-to-P)", "value": value, "unit": "TFLOP/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": w.name, "n_mol": w.n_mol, "N": w.n, "blocks": {"O": w.basis[0], "H": w.basis[1]},
                      "eps_filter": w.eps_filter, "tol": w.tol, "mu": h.mu,
                      "l2": "inputs larger than L2 (H alone is %.0f MB; 129 MB L2)" % (h.H.data.nbytes / 1e6),
                      "parallelism": f"replicas x{world}"},
           "time_to_p_ms": ms_all / args.steps,
           "iterations": iters[-1], "converged": all(conv), "trace_p": trp[-1], "n_occ": h.n_occ,
           "e_band": ebands[-1], "e_band_both_spins": 2.0 * ebands[-1],
           "residual": r.report.residual, "stalled": bool(r.report.stalled),
           "gpu_launches": launches, "clocks": clk, "roofline": roofline, "e2e": e2e, "mixed": mixed}

    if rank == 0 and world == 1 and not args.no_cpu:
        f, dt, cores = oracle_sample(h, w, args.cpu_steps)
        out["cpu_baseline"] = {"value": f / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                               "sample": sample_text(args.cpu_steps, f, dt)}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
