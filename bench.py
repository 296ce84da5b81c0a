"""Benchmark of the reaction-field matvec (Mtargets/s) on synthetic inputs.

Default workload: four layers (interfaces z = 0, -1, -2, k = (1, 1.5, 2, 2.5)
+ 0.02i), N = 2^20 points in 64 Gaussian clusters (sigma 0.05) in layers 1-2,
complex currents, truncation p = 12.  One step = one full matvec
Phi = A J (P2M, M2M, M2L, L2L, L2P, near field) with the tree and tables
built beforehand.  The mixed form runs M2L, M2M and L2L on the tensor cores
(--tensor-cores 3); its error against the oracle's direct sum is measured on
sampled targets in the same run.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp64|mixed] [--tensor-cores 0|1|2|3]
                  [--workload four_layer|three_layer|two_layer|four_layer_small|three_layer_small
                              |paper_2layer|paper_3layer]

Multi-GPU: every rank runs an independent replica of the workload (the
reaction components are independent FMMs, no data exchange is needed);
value = targets processed by all ranks / max-over-ranks time (weak scaling).
--impl reference times the CPU oracle (direct FP64 Sommerfeld sum) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# ALU peaks from unit counts and the maximum SM clock (152 SMs, 2070 MHz):
# FP32 128 FMA/clk/SM, FP64 2 FMA/clk/SM (the nominal 1.25 TFLOP/s).
SM_COUNT, SM_MHZ = 152, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * 128 * 2 * SM_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = SM_COUNT * 2 * 2 * SM_MHZ * 1e6 / 1e12
# dense TF32 tensor peak: the measured bf16 burst peak times the nominal
# TF32 / bf16 ratio (1.1 / 2.25 PFLOP/s); fallback 1.9 PFLOP/s bf16
TF32_PER_BF16 = 1.1 / 2.25


def tensor_peak(tf32):
    """Dense tensor peak of the kernel's operand type: the measured bf16 burst,
    times the nominal tf32/bf16 ratio for a TF32 kernel."""
    r, tag = (TF32_PER_BF16, " x nominal tf32/bf16 1.1/2.25") if tf32 else (1.0, "")
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
        return bf16 * r, "of measured: bf16 burst %.1f TFLOP/s%s" % (bf16, tag)
    except (OSError, KeyError, ValueError):
        return 1900.0 * r, "of fallback: bf16 1900 TFLOP/s%s" % tag


def workload(name, seed_shift=0):
    from paper_2507_18491_gb300 import workloads as W
    if name == "four_layer":
        # leaf level from the depth tuner (host-side cost model over depths 5-7)
        return W.four_layer_clusters(seed=1005 + seed_shift), dict(depth="auto", depths=(5, 6, 7), theta=0.5)
    if name == "three_layer":
        return W.three_layer(seed=1002 + seed_shift), dict(depth=5, theta=0.45)
    if name == "four_layer_small":
        return W.four_layer_clusters(n=131072, seed=1005 + seed_shift), dict(depth=4, theta=0.55)
    if name == "three_layer_small":
        return W.three_layer(n=8192, seed=1002 + seed_shift, p=8), dict(depth=4, theta=0.55)
    if name == "two_layer":
        return W.two_layer_small(seed=1001 + seed_shift), dict(depth=2, theta=0.4)
    if name in ("paper_2layer", "paper_3layer"):
        # Section 4 efficiency test: 10^6 uniform points per layer in unit cubes, p = 8
        layers = 2 if name == "paper_2layer" else 3
        return W.paper_table_uniform(m=10 ** 6, layers=layers, seed=1006 + seed_shift, p=8), \
            dict(depth=5, theta=0.55)
    raise SystemExit("unknown workload " + name)


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch.distributed as dist
    import torch
    rank, lrank = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(lrank)
    dist.init_process_group("nccl")
    return rank, ws, lrank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, ws):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, idx):
        self.proc = None
        import tempfile
        self.out = os.path.join(tempfile.gettempdir(), "lmfmm_clocks_%d.csv" % os.getpid())
        try:
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(idx), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.out):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None, "reasons": sorted(reasons)}


def cpu_baseline(w, sample_sources=1500, sample_targets=8, threads=0):
    """The oracle (direct FP64 Sommerfeld sum) on a bounded sample; returns
    targets/s extrapolated to all N sources."""
    import oracle
    rng = np.random.default_rng(0)
    src = rng.choice(w.N, min(sample_sources, w.N), replace=False)
    tg = rng.choice(w.N, sample_targets, replace=False)
    t0 = time.time()
    oracle.direct(w.d, w.k, w.xyz, w.J, targets=tg, sources=src, nthreads=threads)
    dt = time.time() - t0
    pairs_per_s = tg.size * src.size / dt
    cores = threads or os.cpu_count()
    return {"value": pairs_per_s / w.N / 1e6, "unit": "Mtargets/s", "cores": cores,
            "kind": "oracle",
            "sample": "%d targets x %d of %d sources (direct FP64 Sommerfeld sum), "
                      "%.1f s wall; targets/s = pairs/s / N" % (tg.size, src.size, w.N, dt)}


SAMPLE_OF = {"four_layer_clusters_n1048576": "four_layer_n1048576", "three_layer_n65536": "three_layer_n65536",
             "two_layer_n512": "two_layer_n512", "paper_table_2layer_m1000000": "paper_2layer_m1000000",
             "paper_table_3layer_m1000000": "paper_3layer_m1000000"}

# The paper's own timings of the reaction part on this workload (Table Cputime_N_p8,
# M = 10^6 per layer, p = 8, one Xeon E5-2699 v4 core, setup and all passes included):
# sum of the Phi^r rows -> 2 x 10^6 targets in 94.39 s, 3 x 10^6 in 417.90 s.
PAPER_MTARGETS = {"paper_table_2layer_m1000000": 2e6 / 94.39 / 1e6,
                  "paper_table_3layer_m1000000": 3e6 / 417.90 / 1e6}


def _samples():
    """The stored-oracle reader (tests/golden/make_oracle_samples.py): oracle
    values for seeded target/source samples, recomputed if the inputs differ."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_oracle_samples", os.path.join(ROOT, "tests", "golden", "make_oracle_samples.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def accuracy(op, w, dtype):
    """Err_2 and Err_max (Section 4) of the matvec against the oracle's direct
    sum on the workload's stored sample (J kept on the sampled sources, zero
    elsewhere; targets half next to an interface), else on 16 random targets
    x 400 random sources computed now."""
    import torch
    import oracle
    name = SAMPLE_OF.get(w.name)
    if name is not None:
        _, tg, src, J, ref = _samples().reference(name)
        how = "stored oracle sample %s" % name
    else:
        rng = np.random.default_rng(11)
        src = rng.choice(w.N, min(400, w.N), replace=False)
        tg = rng.choice(w.N, min(16, w.N), replace=False)
        J = np.zeros_like(w.J)
        J[src] = w.J[src]
        ref, _ = oracle.direct(w.d, w.k, w.xyz, J, targets=tg, sources=src)
        how = "oracle now"
    got = op.matvec(torch.from_numpy(J).to("cuda", dtype)).cpu().numpy().astype(np.complex128)
    op.check()
    e2 = float(np.linalg.norm(got[tg] - ref) / np.linalg.norm(ref))
    em = float(np.max(np.linalg.norm(got[tg] - ref, axis=1) / np.linalg.norm(ref, axis=1)))
    return {"err_2": e2, "err_max": em, "targets": int(tg.size),
            "sources": int(w.N if src is None else src.size), "reference": how}


def run_reference(args):
    rank, ws, _ = dist_init()
    if rank != 0:
        return
    w, _ = workload(args.workload)
    per = []
    for _ in range(args.warmup):
        cpu_baseline(w, sample_sources=200, sample_targets=2)
    for _ in range(args.steps):
        per.append(cpu_baseline(w, sample_sources=600, sample_targets=4))
    v = float(np.mean([c["value"] for c in per]))
    cb = dict(per[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mtargets/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * w.N / (v * 1e6), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "p": w.p, "layers": int(w.d.size + 1)},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "Mtargets/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = "layered Maxwell FMM matvec Mtargets/s at N=1M vs FP64 form at rel err <=1e-6"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip the FP64-form comparison run of the default (mixed) bench")
    ap.add_argument("--workload", default="four_layer")
    ap.add_argument("--p", type=int, default=0)
    ap.add_argument("--theta", type=float, default=0.0, help="admissibility (default: the workload's)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tensor-cores", type=int, default=3,
                    help="tensor_cores option of the mixed form: 3 = M2L, M2M and L2L on the "
                         "tensor cores (default), 1 = M2L only, 0 = none")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2507_18491_gb300 import build as B
    from paper_2507_18491_gb300 import lmfmm
    rank, ws, lrank = dist_init()
    dev = lrank if ws > 1 else 0
    torch.cuda.set_device(dev)
    B.build()
    w, opt = workload(args.workload, seed_shift=rank)
    if args.theta:
        opt["theta"] = args.theta
    p = args.p or w.p
    prec = lmfmm.FP64 if args.precision == "fp64" else lmfmm.MIXED
    tuner = None
    if opt["depth"] == "auto":
        # predicted matvec times of the mixed tensor-core form from the host-built
        # structures' counts (lmfmm_plan_depth), before anything runs on the device
        best, pred = lmfmm.plan_depth(w.d, w.k, w.xyz, p=p, depths=opt["depths"], theta=opt["theta"])
        opt["depth"] = best
        tuner = {"choice": best, "predicted_ms": {str(k): round(v, 3) for k, v in pred.items()},
                 "model": "lmfmm_plan_depth default unit costs (measured on GB300, mixed form, p = 12)"}
    t0 = time.time()
    tck = {"tensor_cores": args.tensor_cores} if prec == lmfmm.MIXED else {}
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=p, depth=opt["depth"], theta=opt["theta"],
                        precision=prec, device=dev, **tck).build()
    setup_s = time.time() - t0
    stream = torch.cuda.current_stream()
    # currents in the workload's own type (the four-layer workload draws complex64)
    cdt = torch.complex64 if w.dtype == "c64" else torch.complex128
    ndt = np.complex64 if w.dtype == "c64" else np.complex128
    J = torch.from_numpy(w.J.astype(ndt)).to("cuda")
    out = torch.empty_like(J)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    op.matvec(J, out)
    a1.record(stream)
    torch.cuda.synchronize()
    first_ms = a0.elapsed_time(a1)
    for _ in range(args.warmup):
        op.matvec(J, out)
    op.check()
    clocks = Clocks(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    m2l_ms = []
    barrier(ws)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(i & 0xff)        # L2 flush between timed steps (outside the events)
        ev[i][0].record(stream)
        op.matvec(J, out)
        ev[i][1].record(stream)
        torch.cuda.synchronize()
        m2l_ms.append(op.stats()["ms_stage"]["m2l"])
    torch.cuda.synchronize()
    barrier(ws)
    ck = clocks.stop()
    op.check()                       # no device wait of the timed matvecs gave up
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    total_ms = allmax(total_ms, ws)
    ms = total_ms / args.steps
    value = ws * w.N / (ms * 1e-3) / 1e6
    st = op.stats()
    # end to end through the host-buffer entry point (pinned host memory, the
    # workload's element type; the call copies in, applies, copies out, checks)
    Jh = torch.from_numpy(w.J.astype(ndt)).pin_memory().numpy()
    Ph = torch.empty((w.N, 3), dtype=cdt).pin_memory().numpy()
    lmfmm.matvec_host(op.ctx, Jh, Ph)
    barrier(ws)
    t1 = time.time()
    for _ in range(args.steps):
        lmfmm.matvec_host(op.ctx, Jh, Ph)
    e2e_ms = allmax((time.time() - t1) * 1e3 / args.steps, ws)
    P = (p + 1) ** 2
    flops = 8.0 * P * P * st["m2l_columns"]
    m2l_s = float(np.mean(m2l_ms)) * 1e-3
    achieved = flops / m2l_s / 1e12
    kern = {0: "k_m2l<double>", 1: "k_m2l<float>", 2: "k_m2l_tc", 3: "k_m2l_tc2"}[st["m2l_kernel"]]
    # DRAM bytes per launch of k_m2l_tc2: the table image times the read + write / image
    # ratio of an ncu capture of the same kernel (dram__bytes_read.sum 2.780 GB +
    # dram__bytes_write.sum 0.042 GB for a 2.622 GB image, three-layer N = 8192,
    # p = 12, depth 4, theta 0.55).  The image, read once per launch, is most of it; the
    # multipole expansions fit in L2 in that case but not at N = 2^20 (152 MB), so the
    # scaled figure is a lower bound there.  Other kernels: not captured
    traffic = st["bytes_tables"] * (2.8226 / 2.6224) if st["m2l_kernel"] == 3 else None
    bound = "tensor" if st["m2l_kernel"] >= 2 else "alu"
    if prec == lmfmm.FP64:
        peak, peak_src = FP64_PEAK_TFLOPS, "derived (not measured) FP64 ALU: 152 SM x 2 FMA/clk x 2 x 2070 MHz"
    elif bound == "tensor":
        peak, peak_src = tensor_peak(tf32=st["m2l_kernel"] == 2)
    else:
        peak, peak_src = FP32_PEAK_TFLOPS, "derived (not measured) FP32 ALU: 152 SM x 128 FMA/clk x 2 x 2070 MHz"
    line = {
        "metric": METRIC, "value": value, "unit": "Mtargets/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": (value / PAPER_MTARGETS[w.name]) if w.name in PAPER_MTARGETS else None,
        "dtype": "f64" if prec == lmfmm.FP64 else "f32", "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "layers": int(w.d.size + 1), "p": p,
                   "depth": st["depth"], "depth_tuner": tuner, "theta": opt["theta"],
                   "precision": args.precision,
                   "tensor_cores": int(args.tensor_cores) if prec == lmfmm.MIXED else 0,
                   "components": st["n_components"], "m2l_pairs": st["n_m2l_pairs"],
                   "geometries": st["n_geometries"],
                   "geometries_same_layer": st["n_geometries_same_layer"],
                   "table_bytes": st["bytes_tables"],
                   "near_point_pairs": st["n_near_point_pairs"], "io_dtype": w.dtype,
                   "setup_s": round(setup_s, 3), "cold_s": round(setup_s + first_ms * 1e-3, 3),
                   "tabulation": {"ms": round(st["ms_tabulate"], 3), "gflop": st["tab_flops"] / 1e9,
                                  "tflops": st["tab_flops"] / max(st["ms_tabulate"], 1e-9) / 1e9,
                                  "frac_of_fp64_peak": st["tab_flops"] / max(st["ms_tabulate"], 1e-9) / 1e9
                                  / FP64_PEAK_TFLOPS,
                                  "peak": "derived FP64 ALU %.2f TFLOP/s: 152 SM x 2 FMA/clk x 2 x 2070 MHz"
                                          % FP64_PEAK_TFLOPS},
                   "l2": "flushed (256 MiB write) between steps",
                   "stage_ms": {k: round(v, 3) for k, v in st["ms_stage"].items()},
                   "parallelism": "replicas" if ws > 1 else "single"},
        "clocks": ck,
        "e2e": {"value": ws * w.N / (e2e_ms * 1e-3) / 1e6, "unit": "Mtargets/s",
                "h2d_bytes_per_step": int(Jh.nbytes), "d2h_bytes_per_step": int(Ph.nbytes)},
        "gpu_launches": int(st["launches"]) * args.steps,
        "roofline": {"kernel": kern, "bound": bound, "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_src, "flops_per_launch": flops,
                     "flops_definition": "algorithmic: 8 P^2 real flops per M2L column (complex P x P "
                                         "product); the tensor path executes more: 6 bf16 products of "
                                         "three-piece splits (k_m2l_tc2) or 3 TF32 terms (k_m2l_tc)"},
    }
    if rank == 0 and not args.no_cpu:
        acc = accuracy(op, w, cdt)
        line["config"]["rel_err_vs_oracle"] = acc["err_2"]
        line["config"]["accuracy"] = acc
    op.close()
    if prec == lmfmm.MIXED and not args.no_fp64_form:
        # the same matvec in the FP64 form on the same GPU (fewer steps: ~1.2 s each)
        op64 = lmfmm.Operator(w.d, w.k, w.xyz, p=p, depth=opt["depth"], theta=opt["theta"],
                              precision=lmfmm.FP64, device=dev).build()
        for _ in range(3):
            op64.matvec(J, out)
        op64.check()
        t64 = []
        for i in range(10):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(i & 0xff)
            a.record(stream)
            op64.matvec(J, out)
            b.record(stream)
            torch.cuda.synchronize()
            t64.append(a.elapsed_time(b))
        op64.check()
        ms64 = allmax(float(np.median(t64)), ws)
        line["fp64_form"] = {"value": ws * w.N / (ms64 * 1e-3) / 1e6, "unit": "Mtargets/s",
                             "ms_per_step": ms64, "steps": 10, "statistic": "median of 10 after 3 warm-up",
                             "stage_ms": {k: round(v, 3) for k, v in op64.stats()["ms_stage"].items()}}
        if rank == 0 and not args.no_cpu:
            acc64 = accuracy(op64, w, cdt)
            line["fp64_form"]["rel_err_vs_oracle"] = acc64["err_2"]
            line["fp64_form"]["accuracy"] = acc64
        op64.close()
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
