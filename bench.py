"""Benchmark: Wilson Dslash GFlop/s and fraction of the HBM roofline on one GB300.

Workload (default): the 32^4 lattice (V = 1,048,576, m = 0.01) with smooth
SU(3) links U = exp(0.3 i H), even-odd preconditioned.  One step applies the
even-odd normal operator Mhat^dag Mhat (four even-odd hops: H_oe, H_eo with
the Schur diagonal, and the same with the dagger) to a Gaussian even-parity
spinor, in the storage precision --prec (FP16 with per-site FP32 norms by
default, FP32 arithmetic).  This is the operator the inner mixed-precision
CG iterates.  GFlop/s count 1320 flop per output site per hop.

Output: one JSON line (rank 0).  `roofline` is for the hop kernel: the
algorithmic bytes of one launch over its CUDA-event duration on the launch
stream, against the measured HBM copy bandwidth.  `cpu_baseline` is the FP64
CPU oracle applying the same operator on this host.  --impl reference times
that oracle alone, as the reference arm.

N > 1 (torchrun): independent replicas, one per GPU (no data-path exchange),
value = all ranks' flops / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOP_PER_SITE = 1320
METRIC = "Dslash GFlop/s & % HBM roofline; mixed vs FP64 CG time to 1e-10 residual"
PREC_NAMES = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
CONFIGS = {
    # name: dims, mass, link seed
    "wilson_eo_32x4": ((32, 32, 32, 32), 0.01, 1002),
    "wilson_eo_16x3x32": ((16, 16, 16, 32), 0.05, 1001),
}


# single solves for profiling: 24^3x48, m = 0.02, smooth links (18-real), the 12 point sources of one
# site, to 1e-10 (full D^dag D or the even-odd normal equations; block CG over the 12, or FP64 CG on
# the first); the uneven batch 8^4..20^4 x 4 (even-odd, FP16 inner) batched or one lattice after another
SOLVES = ("eo_block_24x3x48", "full_block_24x3x48", "eo_fp64_24x3x48", "full_fp64_24x3x48",
          "batch_uneven_8x4_to_20x4", "seq_uneven_8x4_to_20x4")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="wilson_eo_32x4", choices=sorted(CONFIGS))
    ap.add_argument("--prec", default="f16", choices=sorted(PREC_NAMES))
    ap.add_argument("--compress12", type=int, default=0)
    ap.add_argument("--su3-only", action="store_true",
                    help="time only the lattice-wide SU(3) product sweep (the workload of its ncu capture)")
    ap.add_argument("--hops-only", action="store_true",
                    help="time only the 12-RHS and domain-wall hops (the workload of their ncu captures)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the CPU baseline, e2e and per-precision table (for profiler runs)")
    ap.add_argument("--solve", choices=sorted(SOLVES),
                    help="run only this solve, --steps times, one JSON line each (the workload of its ncu captures)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """SM clock and throttle reasons sampled every ~2 ms during the timed region
    through NVML (libnvidia-ml, read-only queries); nvidia-smi at 200 ms if
    NVML cannot be loaded."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index):
        self.cuda_index = cuda_index
        self.samples = []
        self.max_mhz = None
        self.stop = threading.Event()
        self.nvml = None
        self.proc = None
        self.lines = []

    def _nvml_handle(self):
        import ctypes

        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        handle = ctypes.c_void_p()
        ok = False
        try:
            import torch

            uuid = str(torch.cuda.get_device_properties(self.cuda_index).uuid)
            u = ("GPU-" + uuid).encode()
            ok = lib.nvmlDeviceGetHandleByUUID(ctypes.c_char_p(u), ctypes.byref(handle)) == 0
        except Exception:
            ok = False
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.cuda_index), ctypes.byref(handle)) != 0:
            raise RuntimeError("no NVML handle")
        mx = ctypes.c_uint(0)
        if lib.nvmlDeviceGetMaxClockInfo(handle, ctypes.c_int(1), ctypes.byref(mx)) == 0:
            self.max_mhz = float(mx.value)
        return lib, handle

    def _poll_nvml(self):
        import ctypes

        lib, handle = self.nvml
        clk = ctypes.c_uint(0)
        mask = ctypes.c_ulonglong(0)
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop.is_set():
            if lib.nvmlDeviceGetClockInfo(handle, ctypes.c_int(1), ctypes.byref(clk)) == 0:
                r = reasons_fn(handle, ctypes.byref(mask))
                self.samples.append((float(clk.value), int(mask.value) if r == 0 else 0))
            time.sleep(0.002)

    def _read_smi(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __enter__(self):
        try:
            self.nvml = self._nvml_handle()
            self.t = threading.Thread(target=self._poll_nvml, daemon=True)
            self.t.start()
            time.sleep(0.01)
        except Exception:
            self.nvml = None
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.cuda_index), "--query-gpu=clocks.sm,clocks.max.sm,"
                     "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                     "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                     "--format=csv,noheader,nounits", "-lms", "200"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.t = threading.Thread(target=self._read_smi, daemon=True)
                self.t.start()
                time.sleep(0.3)
            except Exception:
                self.proc = None
        return self

    def __exit__(self, *a):
        if self.nvml:
            self.stop.set()
            self.t.join(timeout=1)
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        reasons = set()
        if self.nvml:
            sm = [c for c, _ in self.samples]
            for _, m in self.samples:
                for bit, name in self.REASONS.items():
                    if m & bit:
                        reasons.add(name)
            src = "nvml"
        else:
            sm = []
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for line in self.lines:
                f = [x.strip() for x in line.split(",")]
                try:
                    sm.append(float(f[0]))
                    self.max_mhz = float(f[1])
                except (ValueError, IndexError):
                    continue
                for n, v in zip(names, f[2:6]):
                    if v.lower() == "active":
                        reasons.add(n)
            src = "nvidia-smi"
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"], "source": src}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.max_mhz, "reasons": sorted(reasons),
                "samples": len(sm), "source": src}


def hop_source_hash():
    import hashlib

    h = hashlib.sha256()
    for f in ("hop_async.cuh", "lqcd_internal.cuh", "hop.cuh", "pdl.cuh"):
        with open(os.path.join(ROOT, "paper_2001_07557_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(config, prec, r12):
    """DRAM bytes per hop launch from profiles/traffic.txt, if measured on the current kernel sources."""
    try:
        cur = hop_source_hash()
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            for line in f:
                p = line.split()
                if len(p) == 5 and not line.startswith("#") and p[0] == config and p[1] == prec and \
                        int(p[2]) == r12 and p[3] == cur:
                    return float(p[4])
    except Exception:
        return None
    return None


# FP64 on GB300: 152 SMs x 2 DFMA / clock x 2 flop x 2.07 GHz (the nominal 1.25 TFLOP/s; a DFMA loop
# measured 1.21 TFLOP/s on this machine)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def roofline_entry(prec, bytes_launch, launch_ms, Vh, hbm, peak_kind, traffic):
    if prec == 0:
        # the FP64 hop is bound by FP64 arithmetic, not by HBM
        tf = FLOP_PER_SITE * Vh / (launch_ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tf / FP64_PEAK_TFLOPS, "peak_kind": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz",
                "traffic": traffic, "kernel": "wilson_hop_kernel (FP64)", "launch_ms": launch_ms}
    achieved = bytes_launch / (launch_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "peak_kind": peak_kind, "traffic": traffic, "kernel": "wilson_hop_async_kernel",
            "bytes_per_launch": bytes_launch, "launch_ms": launch_ms}


def algorithmic_bytes_per_site(prec, r12, diag):
    """Minimum DRAM bytes of one even-odd hop per output site: 8 links, the
    input spinor once, the output once (+ the diagonal input)."""
    link = {0: (144, 96), 1: (72, 48), 2: (36, 24), 3: (36, 24)}[prec][1 if r12 else 0]
    sp = {0: 192, 1: 96, 2: 52, 3: 52}[prec]
    return 8 * link + 2 * sp + (sp if diag else 0)


def setup(cfg, seed_src=2002):
    from paper_2001_07557_gb300 import inputs

    dims, mass, lseed = CONFIGS[cfg]
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=lseed)
    psi_e = inputs.gaussian_spinor(V // 2, seed=seed_src)
    return dims, mass, U, psi_e


def oracle_normal_op(dims, mass, U, psi_e):
    """Mhat^dag Mhat psi_e by the FP64 CPU oracle; returns (seconds, result)."""
    import oracle

    prm = oracle.params(dims, mass=mass)
    t0 = time.perf_counter()
    out = oracle.apply_normal(oracle.OP_WILSON_EO, psi_e, U, prm)
    return time.perf_counter() - t0, out


def oracle_timed(fn, *a, **k):
    """CPU-baseline leg: one call of an oracle function, wall seconds and result."""
    t0 = time.perf_counter()
    r = fn(*a, **k)
    return time.perf_counter() - t0, r


def host_cpu():
    """The host CPU's model name (lscpu), else the machine architecture."""
    import platform
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip() + " (" + platform.machine() + ")"
    except Exception:
        pass
    return platform.machine()


def host_cores():
    try:
        import oracle

        oracle.build()
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    except Exception:
        return os.cpu_count() or 1


def workload_config(args, dims, mass, world):
    """The `config` of the bench line: the workload both arms run (the GPU arm in the storage precision
    --prec, the reference arm in the oracle's FP64)."""
    prec = PREC_NAMES[args.prec]
    return {"workload": f"{args.config}: even-odd Wilson Mhat^dag Mhat, {args.prec} storage"
                        f"{' + per-site norms' if prec >= 2 else ''}, {'12' if args.compress12 else '18'}-real links",
            "dims": list(dims), "mass": mass, "links": "smooth exp(0.3iH), seed " + str(CONFIGS[args.config][2]),
            "l2": "inputs larger than L2 (links + 3 half spinors > 129 MB); no flush",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle applying the bench's own step (Mhat^dag Mhat on the full
    lattice of the workload, the same generator and source) on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dims, mass, U, psi_e = setup(args.config)
    Vh = int(np.prod(dims)) // 2
    for _ in range(args.warmup):
        oracle_normal_op(dims, mass, U, psi_e)
    t = 0.0
    for _ in range(args.steps):
        dt, _ = oracle_normal_op(dims, mass, U, psi_e)
        t += dt
    flops = 4 * FLOP_PER_SITE * Vh * args.steps
    val = flops / t / 1e9
    cores = host_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GFlop/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, dims, mass, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": val, "unit": "GFlop/s", "cores": cores, "cpu": host_cpu(), "kind": "oracle",
                         "sample": f"Mhat^dag Mhat on the full {list(dims)} lattice per step, FP64 oracle "
                                   "(dense gamma matrices, OpenMP over sites)"},
        "e2e": {"value": val, "unit": "GFlop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.hops_only:
        hops_only(args)
        return
    if args.su3_only:
        su3_only(args)
        return
    if args.solve:
        solve_only(args)
        return

    import torch
    import torch.distributed as dist

    from paper_2001_07557_gb300 import build as lqbuild
    from paper_2001_07557_gb300 import dist as lqdist
    from paper_2001_07557_gb300 import lqcd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    lqbuild.build()

    prec = PREC_NAMES[args.prec]
    r12 = bool(args.compress12)
    nat = lqcd.LQ_NATIVE | prec
    dims, mass, U, psi_e = setup(args.config)
    V = int(np.prod(dims))
    Vh = V // 2
    prm = lqcd.make_params(dims, mass=mass, compress12=r12)
    Ud = torch.from_numpy(U).cuda()
    h = lqcd.lq_create(prm, Ud, lqcd.LQ_F64)
    del Ud
    torch.cuda.empty_cache()
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream

    def nbuf(subset=lqcd.LQ_EVEN, p=prec):
        return torch.empty(lqcd.lq_field_bytes(h, lqcd.LQ_NATIVE | p, subset, 1), dtype=torch.uint8,
                           device="cuda")

    x64 = torch.from_numpy(psi_e).cuda()
    x = nbuf()
    y = nbuf()
    z = nbuf()
    lqcd.lq_convert(h, x, nat, x64, lqcd.LQ_F64, lqcd.LQ_EVEN, stream=sh)

    def step():
        # Mhat^dag Mhat x: two Schur applications (2 hops each, the second with the diagonal)
        lqcd.dslash_apply(h, y, x, nat, lqcd.LQ_SCHUR_EVEN, stream=sh)
        lqcd.dslash_dag_apply(h, z, y, nat, lqcd.LQ_SCHUR_EVEN, stream=sh)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
    stream.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t0 = time.perf_counter()
        for k in range(args.steps):
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    # replicas: the job's time is the slowest rank's timed region
    total_ms = lqdist.job_time(total_ms)
    flops_step = 4 * FLOP_PER_SITE * Vh
    value = flops_step * args.steps * world / (total_ms * 1e-3) / 1e9

    # the hop kernel: 4 launches per step (2 plain hops, 2 with the diagonal input)
    bytes_launch = Vh * (algorithmic_bytes_per_site(prec, r12, False) + algorithmic_bytes_per_site(prec, r12, True)) / 2
    launch_ms = statistics.median(step_ms) / 4
    hbm, peak_kind = peaks()
    traffic = measured_traffic(args.config, args.prec, int(r12))
    line = {
        "metric": METRIC, "value": value, "unit": "GFlop/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32", "data": "synthetic",
        "config": workload_config(args, dims, mass, world),
        "roofline": roofline_entry(prec, bytes_launch, launch_ms, Vh, hbm, peak_kind, traffic),
        "gpu_launches": 4 * args.steps,
        "clocks": clocks.summary(),
        "wall_s_timed": wall,
    }

    if rank == 0 and not args.no_extras:
        z64 = torch.empty_like(x64)  # the timed step's output, for its error against the oracle
        lqcd.lq_convert(h, z64, lqcd.LQ_F64, z, nat, lqcd.LQ_EVEN, stream=sh)
        stream.synchronize()
        step_out = z64.cpu().numpy()
        del z64
        lqcd.lq_destroy(h)
        h = lqcd.lq_create(prm, torch.from_numpy(U).cuda(), lqcd.LQ_F64)
        line["cg"] = cg_compare(h, lqcd, torch, psi_e, prec)
        line["e2e"] = e2e(h, lqcd, torch, dims, psi_e, prec, args, world)
        line["per_precision"] = precision_table(h, lqcd, torch, psi_e, Vh, args, U, dims, mass)
        line["cpu_baseline"], want = cpu_baseline(dims, mass, U, psi_e, Vh)
        line["error_vs_oracle"] = {
            "rel_norm": float(np.linalg.norm(step_out - want) / np.linalg.norm(want)),
            "max_abs_over_max": float(np.max(np.abs(step_out - want)) / np.max(np.abs(want))),
            "what": f"the timed step's output ({args.prec} storage) against the FP64 oracle's Mhat^dag Mhat "
                    "of the same source"}
        line["configs"] = other_configs(lqcd, torch)
        # last key of the line, so that a reader of the line's tail sees the metric's CG half
        line["summary"] = summary(line)
    lqcd.lq_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def summary(line):
    """The metric's second half and the other headline figures in a few hundred bytes:
    time to a 1e-10 FP64 true residual of the mixed and the plain FP64 CG (32^4), the
    12-source comparison on 24^3x48 (one FP64 single-RHS solve against the 12-source
    batched mixed and block solves, full D^dag D and even-odd), the FP64 hop of 32^4 (the
    paper's precision), and the link-sharing hops' fractions of the HBM roofline."""
    def r(v, d=4):
        return None if v is None else float(f"{v:.{d}g}")

    out = {}
    cg = line.get("cg", {})
    if cg:
        out["cg_32x4_1e-10"] = {"fp64_s": r(cg["fp64"]["seconds"]), "mixed_s": r(cg["mixed"]["seconds"]),
                                "speedup": r(cg["speedup"], 3), "fp64_res": r(cg["fp64"]["true_rel_residual"], 2),
                                "mixed_res": r(cg["mixed"]["true_rel_residual"], 2),
                                "inner": cg.get("inner_precision")}
    c4 = line.get("configs", {}).get("wilson_24x3x48_12rhs", {})
    if c4:
        def sec(k):
            return r(c4[k]["seconds"]) if k in c4 else None

        def ok(k):
            return k in c4 and c4[k]["status"] == 0 and c4[k]["max_true_rel_residual"] < 1e-10
        out["cg_24x3x48_12src_1e-10"] = {
            "full": {"fp64_1rhs_s": sec("fp64_cg_1rhs"), "mixed_12rhs_s": sec("mixed_cg_12rhs_batched_f16"),
                     "block_12rhs_s": sec("block_cg_12rhs_f32"), "fp64_12rhs_s": sec("fp64_cg_12rhs_batched")},
            "eo": {"fp64_1rhs_s": sec("eo_fp64_cg_1rhs"), "mixed_12rhs_s": sec("eo_mixed_cg_12rhs_batched_f16"),
                   "block_12rhs_s": sec("eo_block_cg_12rhs_f32")},
            "all_reached_1e-10": all(ok(k) for k in ("fp64_cg_1rhs", "mixed_cg_12rhs_batched_f16",
                                                     "block_cg_12rhs_f32", "eo_fp64_cg_1rhs",
                                                     "eo_mixed_cg_12rhs_batched_f16", "eo_block_cg_12rhs_f32"))}
        out["hop_24x3x48_12rhs_frac_hbm"] = {k[4:]: r(v["frac_hbm"], 3) for k, v in c4.items()
                                             if k.startswith("hop_") and "frac_hbm" in v}
    f64 = line.get("per_precision", {}).get("f64_r18")
    if f64:
        out["hop_32x4_f64"] = {"gflops": r(f64["gflops"]), "us": r(f64["ms"] * 1e3),
                               "frac_fp64_alu": r(f64["gflops"] / (FP64_PEAK_TFLOPS * 1e3), 3)}
    dwf = line.get("configs", {}).get("dwf_16x4_ls16", {})
    if dwf:
        out["dwf_16x4_ls16_frac_hbm"] = {k[4:]: r(v["frac_hbm"], 3) for k, v in dwf.items()
                                         if k.startswith("dwf_") and isinstance(v, dict) and "frac_hbm" in v}
    ub = line.get("configs", {}).get("uneven_batch_8x4_to_20x4", {})
    if ub and "batched_one_graph" in ub:
        out["uneven_batch_s"] = {"one_graph": r(ub["batched_one_graph"]["seconds"]),
                                 "sequential": r(ub["sequential_per_lattice"]["seconds"])}
        shape = ub.get("autotuned_shape")
        if shape:
            out["uneven_batch_s"]["sites_per_item"] = list(shape["sites_per_item"].values())
    return out


def e2e(h, lqcd, torch, dims, psi_e, prec, args, world):
    """Same operator through the public calls with pinned host buffers, every
    step: H2D of the site-major FP32 source, conversion to the storage format,
    Mhat^dag Mhat, conversion back, D2H of the result.  Steps are pipelined
    two deep: the upload of step k+1 and the download of step k-1 run on their
    own streams (copy engines) while step k computes.  (lq_convert can also
    address the pinned host buffers directly, but its host reads are slower
    than the copy engines: 3.0 against 0.34 ms per step on 32^4.)"""
    Vh = psi_e.shape[0]
    nat = lqcd.LQ_NATIVE | prec
    nbuf = 2
    hx = [torch.from_numpy(psi_e.astype(np.complex64)).pin_memory() for _ in range(nbuf)]
    hy = [torch.empty_like(hx[0]).pin_memory() for _ in range(nbuf)]
    dx = [torch.empty(hx[0].shape, dtype=hx[0].dtype, device="cuda") for _ in range(nbuf)]
    dy = [torch.empty_like(dx[0]) for _ in range(nbuf)]
    nb = lqcd.lq_field_bytes(h, nat, lqcd.LQ_EVEN, 1)
    a, b, c = (torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(3))
    s_in, s_c, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()  # noqa: E731
    up = [ev() for _ in range(nbuf)]  # upload of buffer k done
    used = [ev() for _ in range(nbuf)]  # compute done with dx[k] (may be overwritten)
    done = [ev() for _ in range(nbuf)]  # result in dy[k]
    down = [ev() for _ in range(nbuf)]  # download of dy[k] done (may be overwritten)
    for k in range(nbuf):
        used[k].record(s_c)
        down[k].record(s_out)

    def one(k):
        i = k % nbuf
        s_in.wait_event(used[i])
        with torch.cuda.stream(s_in):
            dx[i].copy_(hx[i], non_blocking=True)
        up[i].record(s_in)
        s_c.wait_event(up[i])
        lqcd.lq_convert(h, a, nat, dx[i], lqcd.LQ_F32, lqcd.LQ_EVEN, stream=s_c)
        used[i].record(s_c)
        lqcd.dslash_apply(h, b, a, nat, lqcd.LQ_SCHUR_EVEN, stream=s_c)
        lqcd.dslash_dag_apply(h, c, b, nat, lqcd.LQ_SCHUR_EVEN, stream=s_c)
        s_c.wait_event(down[i])
        lqcd.lq_convert(h, dy[i], lqcd.LQ_F32, c, nat, lqcd.LQ_EVEN, stream=s_c)
        done[i].record(s_c)
        s_out.wait_event(done[i])
        with torch.cuda.stream(s_out):
            hy[i].copy_(dy[i], non_blocking=True)
        down[i].record(s_out)

    for k in range(3):
        one(k)
    torch.cuda.synchronize()
    n = max(5, args.steps // 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for k in range(n):
        one(k)
    s_in.wait_stream(s_out)
    e1.record(s_in)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    ok = bool(torch.equal(dy[(n - 1) % nbuf].cpu(), hy[(n - 1) % nbuf]))  # the last step's result reached the host
    nbytes = hx[0].numel() * hx[0].element_size()
    return {"value": 4 * FLOP_PER_SITE * Vh / (ms * 1e-3) / 1e9 * world, "unit": "GFlop/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": ms,
            "host_format": "site-major FP32, pinned", "pipelined": "two deep: upload, compute, download overlap",
            "host_result_checked": ok}


def precision_table(h, lqcd, torch, psi_e, Vh, args, U, dims, mass):
    """Single even-odd hop H_eo (one launch) per storage precision, 18- and 12-real links."""
    out = {}
    hbm, _ = peaks()
    x64 = torch.from_numpy(inputs_odd(psi_e)).cuda()
    st = torch.cuda.Stream()
    for pname, p in PREC_NAMES.items():
        for r12 in ((0,) if p == 0 else (0, 1)):  # FP64 always keeps 18-real links
            prm = lqcd.make_params(dims, mass=mass, compress12=bool(r12))
            hh = lqcd.lq_create(prm, torch.from_numpy(U).cuda(), lqcd.LQ_F64)
            nat = lqcd.LQ_NATIVE | p
            nb = lqcd.lq_field_bytes(hh, nat, lqcd.LQ_EVEN, 1)
            a = torch.empty(nb, dtype=torch.uint8, device="cuda")
            b = torch.empty(nb, dtype=torch.uint8, device="cuda")
            lqcd.lq_convert(hh, a, nat, x64, lqcd.LQ_F64, lqcd.LQ_ODD, stream=st)
            reps = 20 if p == 0 else 100
            for _ in range(5):
                lqcd.dslash_apply(hh, b, a, nat, lqcd.LQ_EVEN, stream=st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                lqcd.dslash_apply(hh, b, a, nat, lqcd.LQ_EVEN, stream=st)
            e1.record(st)
            st.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = Vh * algorithmic_bytes_per_site(p, r12, False) / (ms * 1e-3) / 1e9
            y64 = torch.empty_like(x64)
            lqcd.lq_convert(hh, y64, lqcd.LQ_F64, b, nat, lqcd.LQ_EVEN, stream=st)
            st.synchronize()
            if p == 0:
                ref = y64  # the FP64 hop, itself within 1e-15 of the oracle in the parity tests
            key = f"{pname}_r{12 if r12 else 18}"
            out[key] = {"gflops": FLOP_PER_SITE * Vh / (ms * 1e-3) / 1e9, "ms": ms, "model_gbs": gbs,
                        "frac_hbm": gbs / hbm,
                        "rel_err_vs_fp64": float(torch.linalg.vector_norm(y64 - ref) / torch.linalg.vector_norm(ref))}
            lqcd.lq_destroy(hh)
    return out


def cg_compare(h, lqcd, torch, psi_e, prec):
    """Time to |b - A x| / |b| < 1e-10 on the even-odd normal equations, b = the
    Gaussian even source: plain FP64 CG against FP64 defect correction with the
    inner CG in the benchmark's storage precision (FP32 arithmetic)."""
    out = {}
    b = torch.from_numpy(psi_e).cuda()
    inner = prec if prec != 0 else lqcd.LQ_F32
    for name, mode in (("fp64", lqcd.LQ_CG_PLAIN), ("mixed", lqcd.LQ_CG_MIXED)):
        x = torch.zeros_like(b)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, mode, lqcd.LQ_F64, tol=1e-10, maxiter=20000,
                                 inner=inner)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = lqcd.cg_solve(h, x, b, cp, check=False)
        wall = time.perf_counter() - t0
        out[name] = {"status": rc, "seconds": wall, "iters": st[0].iters, "outer": st[0].outer_iters,
                     "true_rel_residual": st[0].true_rel_residual}
        if name == "fp64":
            x64 = x.clone()
        else:
            out[name]["rel_diff_vs_fp64"] = float((x - x64).norm() / x64.norm())
    out["inner_precision"] = {0: "f64", 1: "f32", 2: "f16", 3: "bf16"}[inner]
    out["speedup"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    return out


def _time(fn, st, reps, torch):
    for _ in range(3):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    st.synchronize()
    return e0.elapsed_time(e1) / reps


def mrhs_hops(lqcd, torch, st, hbm, U, reps, variants=((False, 1), (True, 1), (False, 2), (False, 3))):
    """24^3x48, m = 0.02: the full-lattice hop on 12 point sources in one launch, on the CUDA
    cores (the default); FP16/BF16 also with the tensor-core kernel."""
    from paper_2001_07557_gb300 import inputs

    dims = (24, 24, 24, 48)
    V = int(np.prod(dims))
    res = {}
    for r12, hp in variants:
        h = lqcd.lq_create(lqcd.make_params(dims, mass=0.02, compress12=r12), torch.from_numpy(U).cuda())
        nat = lqcd.LQ_NATIVE | hp
        pts = torch.from_numpy(inputs.point_sources(V).astype(np.complex64)).cuda()
        nb = lqcd.lq_field_bytes(h, nat, lqcd.LQ_FULL, 12)
        a_, b_ = (torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2))
        lqcd.lq_convert(h, a_, nat, pts, lqcd.LQ_F32, lqcd.LQ_FULL, 12, stream=st)
        pname = {1: "f32", 2: "f16", 3: "bf16"}[hp]
        del pts
        link = 4 * {(1, True): 48, (1, False): 72, (2, False): 36, (3, False): 36}[(hp, r12)]
        byts = V * (link + 12 * 2 * {1: 96, 2: 52, 3: 52}[hp])
        kinds = [(lqcd.LQ_HOP_CUDA_CORES, "")] + ([(lqcd.LQ_HOP_TENSOR_CORES, "_tensor_cores")] if hp > 1 else [])
        for kind, suffix in kinds:
            lqcd.lq_set_hop_kernel(h, kind)
            ms = _time(lambda: lqcd.dslash_apply(h, b_, a_, nat, lqcd.LQ_FULL, nrhs=12, stream=st), st, reps, torch)
            res[f"hop_{pname}_12rhs_r{12 if r12 else 18}{suffix}"] = {
                "gflops": FLOP_PER_SITE * V * 12 / (ms * 1e-3) / 1e9, "ms": ms,
                "model_gbs": byts / (ms * 1e-3) / 1e9, "frac_hbm": byts / (ms * 1e-3) / 1e9 / hbm,
                "bytes_model": "links once per site (4 x link) + 12 x (in + out)",
                "kernel": "tensor cores (mma.sync m16n8k8)" if kind == lqcd.LQ_HOP_TENSOR_CORES else "CUDA cores"}
        lqcd.lq_destroy(h)
        del a_, b_
    return res


def dwf_hops(lqcd, torch, st, hbm, U, reps, precs=(("f32", 1), ("f16", 2), ("bf16", 3))):
    """16^4 x Ls = 16, M5 = 1.8, mf = 0.01: the domain-wall operator on a Gaussian 5-d field."""
    from paper_2001_07557_gb300 import inputs

    dims = (16, 16, 16, 16)
    Ls = 16
    V = int(np.prod(dims))
    res = {}
    for pname, p in precs:
        # 18-real links: the Ls = 16 slices share every link load
        h = lqcd.lq_create(lqcd.make_params(dims, Ls=Ls, M5=1.8, mf=0.01, compress12=False),
                           torch.from_numpy(U).cuda())
        nat = lqcd.LQ_NATIVE | p
        nb = lqcd.lq_field_bytes(h, nat, five_d=True)
        a_, b_ = (torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2))
        lqcd.lq_convert(h, a_, nat, torch.from_numpy(inputs.gaussian_spinor(V, seed=2004, nrhs=Ls)).cuda(),
                        lqcd.LQ_F64, five_d=True, stream=st)
        sp = {1: 96, 2: 52, 3: 52}[p]
        byts = V * (4 * {1: 72, 2: 36, 3: 36}[p] + Ls * 2 * sp)  # minimum: links once per 4-d site, 5-d in once, out once
        kinds = [(lqcd.LQ_HOP_CUDA_CORES, "")] + ([(lqcd.LQ_HOP_TENSOR_CORES, "_tensor_cores")] if p > 1 else [])
        for kind, suffix in kinds:
            lqcd.lq_set_hop_kernel(h, kind)
            ms = _time(lambda: lqcd.dwf_dslash_apply(h, b_, a_, nat, False, stream=st), st, reps, torch)
            res[f"dwf_{pname}_r18{suffix}"] = {
                "gflops_4d": FLOP_PER_SITE * V * Ls / (ms * 1e-3) / 1e9, "ms": ms,
                "model_gbs": byts / (ms * 1e-3) / 1e9, "frac_hbm": byts / (ms * 1e-3) / 1e9 / hbm,
                "extra_5d_flop_per_site": 96,
                "kernel": "tensor cores (mma.sync m16n8k8)" if kind == lqcd.LQ_HOP_TENSOR_CORES else "CUDA cores"}
        lqcd.lq_destroy(h)
    return res


def su3_sweep(lqcd, torch, st, hbm, reps, sides=(8, 16, 24, 32, 48)):
    """The paper's SU(3) matrix-matrix benchmark (Sec. 3.3, Fig. 4a-c): C(x) =
    A(x) B(x) on one colour matrix per site of an L^4 lattice, FP32 and FP64,
    random SU(3) factors.  198 flop per product (27 complex multiplies, 18
    complex adds); 3 x 72 B (FP32) or 3 x 144 B (FP64) of algorithmic traffic."""
    from paper_2001_07557_gb300 import inputs

    base = inputs.gauge_field((4, 4, 4, 4), "random", seed=1000).reshape(-1, 3, 3)  # 1024 SU(3) matrices
    out = {}
    for pname, fmt, dt, mb in (("f32", lqcd.LQ_F32, torch.complex64, 72), ("f64", lqcd.LQ_F64, torch.complex128, 144)):
        for L in sides:
            n = L ** 4
            reps_src = (n + len(base) - 1) // len(base)
            a = torch.from_numpy(np.tile(base, (reps_src, 1, 1))[:n].copy()).to(dt).cuda()
            b = torch.roll(a, 1, 0).contiguous()
            c = torch.empty_like(a)
            ms = _time(lambda: lqcd.lq_su3_mul(c, a, b, n, fmt, stream=st), st, reps, torch)
            gbs = 3 * mb * n / (ms * 1e-3) / 1e9
            e = {"n": n, "us": ms * 1e3, "gflops": 198 * n / (ms * 1e-3) / 1e9, "model_gbs": gbs}
            if 3 * mb * n < 129e6:
                e["note"] = "working set fits in L2"
            if fmt == lqcd.LQ_F32:
                e["frac_hbm"] = gbs / hbm
            else:
                e["frac_fp64_alu"] = e["gflops"] / (FP64_PEAK_TFLOPS * 1e3)
            out[f"{pname}_L{L}"] = e
            del a, b, c
    out["timeouts"] = lqcd.lq_wait_timeouts()
    return out


def su3_only(args):
    """The SU(3) product sweep alone (the workload of its ncu capture)."""
    import torch

    from paper_2001_07557_gb300 import build as lqbuild
    from paper_2001_07557_gb300 import lqcd

    lqbuild.build()
    hbm, _ = peaks()
    st = torch.cuda.Stream()
    print(json.dumps({"su3_mul": su3_sweep(lqcd, torch, st, hbm, args.steps)}))


def hops_only(args):
    """The 12-RHS and domain-wall hops alone (FP32 and FP16, 18-real links), each
    run args.steps times after 3 warm-up launches: the workload of their ncu captures."""
    import torch

    from paper_2001_07557_gb300 import build as lqbuild
    from paper_2001_07557_gb300 import inputs, lqcd

    lqbuild.build()
    hbm, _ = peaks()
    st = torch.cuda.Stream()
    U4 = inputs.gauge_field((24, 24, 24, 48), "smooth", seed=1003)
    out = mrhs_hops(lqcd, torch, st, hbm, U4, args.steps, variants=((False, 1), (False, 2)))
    del U4
    U5 = inputs.gauge_field((16, 16, 16, 16), "smooth", seed=1004)
    out.update(dwf_hops(lqcd, torch, st, hbm, U5, args.steps, precs=(("f32", 1), ("f16", 2))))
    print(json.dumps({"hops_only": out}))


def solve_only(args):
    """One named solve (SOLVES), run args.steps times: the workload of the solver profiles."""
    import torch

    from paper_2001_07557_gb300 import build as lqbuild
    from paper_2001_07557_gb300 import inputs, lqcd

    lqbuild.build()
    name = args.solve
    if "uneven" in name:
        shapes = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (20, 20, 20, 20)]
        hs, bs, xs = [], [], []
        for i, dd in enumerate(shapes):
            Vd = int(np.prod(dd))
            hs.append(lqcd.lq_create(lqcd.make_params(dd, mass=0.02, compress12=True),
                                     torch.from_numpy(inputs.gauge_field(dd, "smooth", seed=1300 + i)).cuda()))
            bs.append(torch.from_numpy(inputs.gaussian_spinor(Vd // 2, seed=2300 + i, nrhs=4)).cuda())
            xs.append(torch.zeros_like(bs[-1]))
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=4, tol=1e-10,
                                 inner=lqcd.LQ_F16)

        def run():
            if name.startswith("batch"):
                return lqcd.lq_batch_cg_solve(hs, xs, bs, cp, check=False)
            rc, st = 0, []
            for h, x, b in zip(hs, xs, bs):
                r, s_ = lqcd.cg_solve(h, x, b, cp, check=False)
                rc, st = rc or r, st + list(s_)
            return rc, st
    else:
        dims = (24, 24, 24, 48)
        V = int(np.prod(dims))
        U = inputs.gauge_field(dims, "smooth", seed=1003)
        h = lqcd.lq_create(lqcd.make_params(dims, mass=0.02, compress12=False), torch.from_numpy(U).cuda())
        eo = name.startswith("eo")
        src = inputs.point_sources(V)
        if eo:
            src = np.ascontiguousarray(inputs.to_half(src, dims, 0))
        src = torch.from_numpy(src).cuda()
        b = torch.empty_like(src)
        lqcd.dslash_dag_apply(h, b, src, lqcd.LQ_F64, lqcd.LQ_SCHUR_EVEN if eo else lqcd.LQ_FULL, nrhs=12)
        del src
        n = 12 if "block" in name else 1
        b = b[:n].contiguous()
        xs = [torch.zeros_like(b)]
        op = lqcd.LQ_OP_WILSON_EO_NORMAL if eo else lqcd.LQ_OP_WILSON_NORMAL
        mode = lqcd.LQ_CG_BLOCK if n == 12 else lqcd.LQ_CG_PLAIN
        cp = lqcd.make_cg_params(op, mode, lqcd.LQ_F64, nrhs=n, tol=1e-10, inner=lqcd.LQ_F32)

        def run():
            return lqcd.cg_solve(h, xs[0], b, cp, check=False)
    for _ in range(args.steps):
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = run()
        sec = time.perf_counter() - t0
        print(json.dumps({"solve": name, "status": rc, "seconds": sec, "max_iters": max(z.iters for z in st),
                          "max_outer": max(z.outer_iters for z in st),
                          "max_true_rel_residual": max(z.true_rel_residual for z in st)}), flush=True)
        if rc:
            sys.exit(1)


def halo_emulation(lqcd, torch, hbm, reps=20):
    """Time-slab decomposition of the full-lattice FP16 Wilson hop on 32^4 into
    two ranks on one GPU: each rank a 32^3 x 18 lattice (16 own slices + two
    ghosts); per hop, 4 face copies (the antiperiodic sign folded into the
    copy at the global boundary) on one stream while the interior slices run on
    another, then the edge slices.  Compared with the single-domain hop."""
    from paper_2001_07557_gb300 import inputs

    dims, R, mass = (32, 32, 32, 32), 2, 0.01
    L3, V3 = dims[3], dims[0] * dims[1] * dims[2]
    Lt = L3 // R
    U = inputs.gauge_field((32, 32, 32, 4), "smooth", seed=1002)  # 4 time slices of links, tiled in t
    Ug = np.tile(U.reshape(4, V3, 4, 3, 3), (L3 // 4, 1, 1, 1, 1))
    nat = lqcd.LQ_NATIVE | lqcd.LQ_F16
    src = torch.randn(L3 * V3 * 12, dtype=torch.complex64, device="cuda").reshape(-1, 4, 3)
    # single domain
    h = lqcd.lq_create(lqcd.make_params(dims, mass=mass), torch.from_numpy(Ug.reshape(-1, 4, 3, 3)).cuda())
    nb = lqcd.lq_field_bytes(h, nat, lqcd.LQ_FULL, 1)
    a_, b_ = (torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2))
    lqcd.lq_convert(h, a_, nat, src, lqcd.LQ_F32)
    st = torch.cuda.Stream()
    single = _time(lambda: lqcd.dslash_apply(h, b_, a_, nat, lqcd.LQ_FULL, stream=st), st, reps, torch)
    lqcd.lq_destroy(h)
    del a_, b_
    # two slabs with ghosts
    hs, ins, outs = [], [], []
    srcg = src.reshape(L3, V3, 4, 3)
    for r in range(R):
        ts = [(r * Lt + tp - 1) % L3 for tp in range(Lt + 2)]
        hr = lqcd.lq_create(lqcd.make_params((32, 32, 32, Lt + 2), mass=mass, bc=(1, 1, 1, 1)),
                            torch.from_numpy(np.ascontiguousarray(Ug[ts]).reshape(-1, 4, 3, 3)).cuda())
        n = lqcd.lq_field_bytes(hr, nat, lqcd.LQ_FULL, 1)
        i_, o_ = torch.empty(n, dtype=torch.uint8, device="cuda"), torch.zeros(n, dtype=torch.uint8, device="cuda")
        loc = torch.zeros((Lt + 2, V3, 4, 3), dtype=torch.complex64, device="cuda")
        loc[1:Lt + 1] = srcg[r * Lt:(r + 1) * Lt]
        lqcd.lq_convert(hr, i_, nat, loc.reshape(-1, 4, 3), lqcd.LQ_F32)
        hs.append(hr)
        ins.append(i_)
        outs.append(o_)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ev = torch.cuda.Event()

    def step():
        ev.record(sa)
        sb.wait_event(ev)
        for r in range(R):
            lqcd.dslash_apply_slices(hs[r], outs[r], ins[r], nat, 2, Lt, stream=sa)
        for r in range(R):
            lo, hi = (r - 1) % R, (r + 1) % R
            lqcd.lq_face_copy(hs[r], ins[r], 0, hs[lo], ins[lo], Lt, nat, -1.0 if r == 0 else 1.0, sb)
            lqcd.lq_face_copy(hs[r], ins[r], Lt + 1, hs[hi], ins[hi], 1, nat, -1.0 if r == R - 1 else 1.0, sb)
        for r in range(R):
            lqcd.dslash_apply_slices(hs[r], outs[r], ins[r], nat, 1, 2, stream=sb)
            lqcd.dslash_apply_slices(hs[r], outs[r], ins[r], nat, Lt, Lt + 1, stream=sb)
        ev.record(sb)
        sa.wait_event(ev)

    split = _time(step, sa, reps, torch)
    # spin-projected faces: each rank packs h = psi_up +- psi_dn of its edge slices, a device copy
    # moves each message to the neighbour (where NCCL would send it), the neighbour unpacks its ghosts
    nw = lqcd.lq_face_wire_bytes(hs[0], nat)
    send = [[torch.empty(nw, dtype=torch.uint8, device="cuda") for _ in range(2)] for _ in range(R)]
    recv = [[torch.empty(nw, dtype=torch.uint8, device="cuda") for _ in range(2)] for _ in range(R)]

    def step_projected():
        ev.record(sa)
        sb.wait_event(ev)
        for r in range(R):
            lqcd.dslash_apply_slices(hs[r], outs[r], ins[r], nat, 2, Lt, stream=sa)
        with torch.cuda.stream(sb):
            for r in range(R):
                lqcd.lq_face_pack(hs[r], send[r][0], ins[r], Lt, nat, 1, -1.0 if r == R - 1 else 1.0, sb)
                lqcd.lq_face_pack(hs[r], send[r][1], ins[r], 1, nat, -1, -1.0 if r == 0 else 1.0, sb)
            for r in range(R):
                recv[r][0].copy_(send[(r - 1) % R][0], non_blocking=True)
                recv[r][1].copy_(send[(r + 1) % R][1], non_blocking=True)
            for r in range(R):
                lqcd.lq_face_unpack(hs[r], ins[r], 0, recv[r][0], nat, 1, sb)
                lqcd.lq_face_unpack(hs[r], ins[r], Lt + 1, recv[r][1], nat, -1, sb)
        for r in range(R):
            lqcd.dslash_apply_slices(hs[r], outs[r], ins[r], nat, 1, 2, stream=sb)
            lqcd.dslash_apply_slices(hs[r], outs[r], ins[r], nat, Lt, Lt + 1, stream=sb)
        ev.record(sb)
        sa.wait_event(ev)

    split_p = _time(step_projected, sa, reps, torch)
    for hr in hs:
        lqcd.lq_destroy(hr)
    face = 2 * R * V3 * 52  # bytes of the four faces (FP16 + norms, full spinors)
    return {"single_domain_us": single * 1e3, "two_slabs_us": split * 1e3,
            "two_slabs_projected_us": split_p * 1e3,
            "gflops_single": FLOP_PER_SITE * L3 * V3 / (single * 1e-3) / 1e9,
            "gflops_two_slabs": FLOP_PER_SITE * L3 * V3 / (split * 1e-3) / 1e9,
            "gflops_two_slabs_projected": FLOP_PER_SITE * L3 * V3 / (split_p * 1e-3) / 1e9,
            "face_bytes_per_hop": face, "projected_message_bytes_per_hop": 2 * R * nw,
            "ghost_compute": "none (only own slices are computed)",
            "note": "both ranks on one GPU; interior slices overlap the face exchange on a second stream; "
                    "projected: pack, one device copy per message, unpack"}


def other_configs(lqcd, torch):
    """The other workloads of the method, one short measurement each."""
    from paper_2001_07557_gb300 import inputs

    hbm, _ = peaks()
    out = {}
    st = torch.cuda.Stream()

    # 4^4, random SU(3), m = 0.1: FP64 CG on D^dag D to 1e-12 (latency bound)
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, "random", seed=1000)
    h = lqcd.lq_create(lqcd.make_params(dims, mass=0.1), torch.from_numpy(U).cuda())
    eta = torch.from_numpy(inputs.gaussian_spinor(256, seed=2000)).cuda()
    b = torch.empty_like(eta)
    lqcd.dslash_dag_apply(h, b, eta, lqcd.LQ_F64, lqcd.LQ_FULL)
    x = torch.zeros_like(b)
    cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F64, tol=1e-12)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, stt = lqcd.cg_solve(h, x, b, cp, check=False)
    out["wilson_4x4_fp64_cg"] = {"status": rc, "seconds": time.perf_counter() - t0, "iters": stt[0].iters,
                             "true_rel_residual": stt[0].true_rel_residual}
    import oracle  # CPU-baseline leg: the oracle timed on the host cores beside each GPU figure

    cores = host_cores()
    prm = oracle.params(dims, mass=0.1)
    dt, (xo, it, _, _) = oracle_timed(oracle.cg, oracle.OP_WILSON, b.cpu().numpy(), U, prm, 1e-12)
    out["wilson_4x4_fp64_cg"]["cpu_baseline"] = {"seconds": dt, "iters": it, "cores": cores, "kind": "oracle"}
    lqcd.lq_destroy(h)

    # 16^3x32 even-odd, smooth links, m = 0.05: FP64 and FP32 hops; FP64 and mixed CG to 1e-10
    dims = (16, 16, 16, 32)
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1001)
    h = lqcd.lq_create(lqcd.make_params(dims, mass=0.05), torch.from_numpy(U).cuda())
    src = inputs.gaussian_spinor(V // 2, seed=2001)
    res = {}
    for pname, p in (("f64", 0), ("f32", 1)):
        nat = lqcd.LQ_NATIVE | p
        nb = lqcd.lq_field_bytes(h, nat, lqcd.LQ_EVEN, 1)
        a_, b_ = (torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2))
        lqcd.lq_convert(h, a_, nat, torch.from_numpy(src).cuda(), lqcd.LQ_F64, lqcd.LQ_ODD, stream=st)
        ms = _time(lambda: lqcd.dslash_apply(h, b_, a_, nat, lqcd.LQ_EVEN, stream=st), st, 50, torch)
        gbs = (V // 2) * algorithmic_bytes_per_site(p, False, False) / (ms * 1e-3) / 1e9
        res[f"{pname}_eo_hop"] = {"gflops": FLOP_PER_SITE * (V // 2) / (ms * 1e-3) / 1e9, "ms": ms, "model_gbs": gbs,
                                  "frac_hbm": gbs / hbm, "note": "working set fits in L2"}
    bd = torch.from_numpy(src).cuda()
    for name, mode in (("fp64_cg", lqcd.LQ_CG_PLAIN), ("mixed_cg_f16", lqcd.LQ_CG_MIXED)):
        x = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, mode, lqcd.LQ_F64, tol=1e-10, inner=lqcd.LQ_F16)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, stt = lqcd.cg_solve(h, x, bd, cp, check=False)
        res[name] = {"status": rc, "seconds": time.perf_counter() - t0, "iters": stt[0].iters,
                     "true_rel_residual": stt[0].true_rel_residual}
    dt, _ = oracle_timed(oracle.wilson_hop_eo, src, U, dims, 0)
    prm = oracle.params(dims, mass=0.05)
    dt_cg, (_, it, _, _) = oracle_timed(oracle.cg, oracle.OP_WILSON_EO, src, U, prm, 1e-10, maxiter=10)
    res["cpu_baseline"] = {"eo_hop_gflops": FLOP_PER_SITE * (V // 2) / dt / 1e9,
                           "cg_seconds_per_iteration": dt_cg / max(it, 1),
                           "cg_seconds_projected": dt_cg / max(it, 1) * res["fp64_cg"]["iters"],
                           "cores": cores, "kind": "oracle",
                           "sample": "one FP64 eo hop; 10 CG iterations, projected to the GPU FP64 CG's count"}
    out["wilson_eo_16x3x32_solves"] = res
    lqcd.lq_destroy(h)

    # 24^3x48, m = 0.02, 12 point sources: multi-RHS full-lattice hop (FP32) and solves
    dims = (24, 24, 24, 48)
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1003)
    res = mrhs_hops(lqcd, torch, st, hbm, U, 10)
    dt, _ = oracle_timed(oracle.wilson_dslash, inputs.point_sources(V), U, dims, 0.02)
    res["cpu_baseline"] = {"hop_12rhs_gflops": FLOP_PER_SITE * V * 12 / dt / 1e9, "seconds": dt, "cores": cores,
                           "kind": "oracle", "sample": "one 12-source full-lattice D application in FP64"}
    # solves to 1e-10 on D^dag D x = D^dag (point source): one FP64 CG, 12 FP64 CGs in one batch,
    # 12 mixed CGs in one batch (FP16 inner), and block CG over the 12 (FP32 inner)
    # 18-real links: with 12 right-hand sides sharing every link load, rebuilding row 3 costs more than it saves
    h = lqcd.lq_create(lqcd.make_params(dims, mass=0.02, compress12=False), torch.from_numpy(U).cuda())
    pts = torch.from_numpy(inputs.point_sources(V)).cuda()
    b = torch.empty_like(pts)
    lqcd.dslash_dag_apply(h, b, pts, lqcd.LQ_F64, lqcd.LQ_FULL, nrhs=12)
    del pts
    runs = [("fp64_cg_1rhs", lqcd.LQ_CG_PLAIN, 1, lqcd.LQ_F32), ("fp64_cg_12rhs_batched", lqcd.LQ_CG_PLAIN, 12, lqcd.LQ_F32),
            ("mixed_cg_12rhs_batched_f16", lqcd.LQ_CG_MIXED, 12, lqcd.LQ_F16),
            ("block_cg_12rhs_f32", lqcd.LQ_CG_BLOCK, 12, lqcd.LQ_F32)]
    for name, mode, n, inner in runs:
        x = torch.zeros_like(b[:n])
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, mode, lqcd.LQ_F64, nrhs=n, tol=1e-10, inner=inner)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, stt = lqcd.cg_solve(h, x, b[:n].contiguous(), cp, check=False)
        res[name] = {"status": rc, "seconds": time.perf_counter() - t0, "max_iters": max(z.iters for z in stt),
                     "max_outer": max(z.outer_iters for z in stt),
                     "max_true_rel_residual": max(z.true_rel_residual for z in stt)}
        del x
    # the same comparison on the even-odd preconditioned system: the point sources sit on an
    # even site, so b_hat_e = eta_e and the normal equations read Mhat^dag Mhat x_e = Mhat^dag eta_e
    pts_e = torch.from_numpy(np.ascontiguousarray(inputs.to_half(inputs.point_sources(V), dims, 0))).cuda()
    be = torch.empty_like(pts_e)
    lqcd.dslash_dag_apply(h, be, pts_e, lqcd.LQ_F64, lqcd.LQ_SCHUR_EVEN, nrhs=12)
    del pts_e
    for name, mode, n, inner in [("eo_fp64_cg_1rhs", lqcd.LQ_CG_PLAIN, 1, lqcd.LQ_F32),
                                 ("eo_mixed_cg_12rhs_batched_f16", lqcd.LQ_CG_MIXED, 12, lqcd.LQ_F16),
                                 ("eo_block_cg_12rhs_f32", lqcd.LQ_CG_BLOCK, 12, lqcd.LQ_F32)]:
        x = torch.zeros_like(be[:n])
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, mode, lqcd.LQ_F64, nrhs=n, tol=1e-10, inner=inner)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, stt = lqcd.cg_solve(h, x, be[:n].contiguous(), cp, check=False)
        res[name] = {"status": rc, "seconds": time.perf_counter() - t0, "max_iters": max(z.iters for z in stt),
                     "max_outer": max(z.outer_iters for z in stt),
                     "max_true_rel_residual": max(z.true_rel_residual for z in stt)}
        del x
    lqcd.lq_destroy(h)
    res["note"] = ("full-lattice D^dag D, m = 0.02, smooth links, 18-real links; b = D^dag (point source); "
                   "eo_*: the even-odd normal equations Mhat^dag Mhat x_e = Mhat^dag eta_e")
    out["wilson_24x3x48_12rhs"] = res

    # uneven batch: 8^4, 12^4, 16^4, 20^4 x 4 right-hand sides, one persistent graph-captured solve
    # (even-odd normal equations, m = 0.02, FP16 inner, FP64 defect correction to 1e-10),
    # against the same four solves one after another
    res = {}
    shapes = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (20, 20, 20, 20)]
    hs_, bs_, xs_ = [], [], []
    for i, dd in enumerate(shapes):
        Vd = int(np.prod(dd))
        hs_.append(lqcd.lq_create(lqcd.make_params(dd, mass=0.02, compress12=True),
                                  torch.from_numpy(inputs.gauge_field(dd, "smooth", seed=1300 + i)).cuda()))
        bs_.append(torch.from_numpy(inputs.gaussian_spinor(Vd // 2, seed=2300 + i, nrhs=4)).cuda())
        xs_.append(torch.zeros_like(bs_[-1]))
    cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=4, tol=1e-10,
                             inner=lqcd.LQ_F16)
    # the autotuner's choices come back through its cache file (read by the library at its first tuning)
    import tempfile
    tune_file = os.path.join(tempfile.mkdtemp(), "lqcd_tune.txt")
    os.environ["LQCD_TUNE_CACHE"] = tune_file
    for rep in range(2):  # the first call also autotunes the persistent launch
        for x_ in xs_:
            x_.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, stt = lqcd.lq_batch_cg_solve(hs_, xs_, bs_, cp, check=False)
        sec = time.perf_counter() - t0
        key = "batched_one_graph" + ("" if rep else "_first_call_with_tuning")
        res[key] = {"status": rc, "seconds": sec, "max_iters": max(z.iters for z in stt),
                    "max_true_rel_residual": max(z.true_rel_residual for z in stt)}
    flops = sum(4 * FLOP_PER_SITE * (int(np.prod(dd)) // 2) * 4 for dd in shapes) * res["batched_one_graph"]["max_iters"]
    res["batched_one_graph"]["hop_gflops_upper"] = flops / res["batched_one_graph"]["seconds"] / 1e9
    t0 = time.perf_counter()
    worst = 0.0
    for h_, x_, b_ in zip(hs_, xs_, bs_):
        x_.zero_()
        rc, stt = lqcd.cg_solve(h_, x_, b_, cp, check=False)
        worst = max([worst] + [z.true_rel_residual for z in stt])
    res["sequential_per_lattice"] = {"seconds": time.perf_counter() - t0, "max_true_rel_residual": worst}
    for h_ in hs_:
        lqcd.lq_destroy(h_)
    res["autotuned_shape"] = read_tune_file(tune_file, shapes)
    out["uneven_batch_8x4_to_20x4"] = res

    # 16^4 x Ls=16 domain wall, FP32
    dims = (16, 16, 16, 16)
    Ls = 16
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1004)
    res = dwf_hops(lqcd, torch, st, hbm, U, 20)
    psi5 = inputs.gaussian_spinor(V, seed=2004, nrhs=Ls)
    dt, _ = oracle_timed(oracle.dwf_dslash, psi5, U, dims, Ls, 1.8, 0.01)
    dt_s, _ = oracle_timed(oracle.dwf_schur, psi5[:, : V // 2], U, dims, Ls, 1.8, 0.01)
    res["cpu_baseline"] = {"dwf_gflops_4d": FLOP_PER_SITE * V * Ls / dt / 1e9, "dwf_seconds": dt,
                           "eo_schur_seconds": dt_s, "cores": cores, "kind": "oracle",
                           "sample": "one D_dw and one Mhat application in FP64"}
    del psi5
    # CG on D_dw^dag D_dw: FP32 alone to 1e-8, and FP64 refinement around FP32 inner solves to 1e-10
    h = lqcd.lq_create(lqcd.make_params(dims, Ls=Ls, M5=1.8, mf=0.01, compress12=False), torch.from_numpy(U).cuda())
    eta = torch.from_numpy(inputs.gaussian_spinor(V, seed=2004, nrhs=Ls)).cuda()
    b = torch.empty_like(eta)
    lqcd.dwf_dslash_apply(h, b, eta, lqcd.LQ_F64, True)
    Dpsi = torch.empty_like(eta)

    def full_residual(psi):  # |D_dw psi - eta| / |eta| in FP64
        lqcd.dwf_dslash_apply(h, Dpsi, psi, lqcd.LQ_F64, False)
        return float(torch.linalg.vector_norm(Dpsi - eta) / torch.linalg.vector_norm(eta))

    b32 = b.to(torch.complex64)
    x32 = torch.zeros_like(b32)
    cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F32, tol=1e-8, maxiter=20000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, stt = lqcd.cg_solve(h, x32, b32, cp, check=False)
    res["fp32_cg_1e-8"] = {"status": rc, "seconds": time.perf_counter() - t0, "iters": stt[0].iters,
                           "true_rel_residual_fp64": stt[0].true_rel_residual}
    x = torch.zeros_like(b)
    cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10, maxiter=40000,
                             inner=lqcd.LQ_F32, inner_tol=1e-6)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, stt = lqcd.cg_solve(h, x, b, cp, check=False)
    res["fp64_refined_fp32_inner_1e-10"] = {"status": rc, "seconds": time.perf_counter() - t0,
                                            "iters": stt[0].iters, "outer": stt[0].outer_iters,
                                            "true_rel_residual": stt[0].true_rel_residual,
                                            "full_system_rel_residual": full_residual(x)}
    # the same system through the even-odd (4-d parity) Schur complement: prepare the source,
    # CG on Mhat^dag Mhat (FP64 outer, FP32 inner) to 1e-10, reconstruct the odd half
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bh = torch.empty((Ls, V // 2, 4, 3), dtype=eta.dtype, device="cuda")
    lqcd.dwf_eo_prepare(h, bh, eta, lqcd.LQ_F64)
    be = torch.empty_like(bh)
    lqcd.dwf_schur_apply(h, be, bh, lqcd.LQ_F64, True)
    xe = torch.zeros_like(be)
    cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_EO_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10, maxiter=40000,
                             inner=lqcd.LQ_F32, inner_tol=1e-6)
    rc, stt = lqcd.cg_solve(h, xe, be, cp, check=False)
    psi = torch.empty_like(eta)
    lqcd.dwf_eo_reconstruct(h, psi, xe, eta, lqcd.LQ_F64)
    torch.cuda.synchronize()
    res["eo_fp64_refined_fp32_inner_1e-10"] = {"status": rc, "seconds": time.perf_counter() - t0,
                                               "iters": stt[0].iters, "outer": stt[0].outer_iters,
                                               "true_rel_residual": stt[0].true_rel_residual,
                                               "full_system_rel_residual": full_residual(psi),
                                               "note": "includes source preparation and reconstruction"}
    # one application of the Schur complement, FP32 native (2 half-lattice hops + M5^-1 + M5)
    nat = lqcd.LQ_NATIVE | lqcd.LQ_F32
    nb = lqcd.lq_field_bytes(h, nat, lqcd.LQ_EVEN, Ls)
    a_, b_ = (torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2))
    lqcd.lq_convert(h, a_, nat, bh, lqcd.LQ_F64, lqcd.LQ_EVEN, Ls, stream=st)
    ms = _time(lambda: lqcd.dwf_schur_apply(h, b_, a_, nat, False, stream=st), st, 20, torch)
    res["eo_schur_f32"] = {"ms": ms, "gflops_hops": 2 * FLOP_PER_SITE * (V // 2) * Ls / (ms * 1e-3) / 1e9,
                           "note": "flops of the two half-lattice 4-d hops only"}
    lqcd.lq_destroy(h)
    # Moebius (b5 = 1.5, c5 = 0.5, b5 - c5 = 1): one FP32 operator application and the FP64-refined solve
    hm = lqcd.lq_create(lqcd.make_params(dims, Ls=Ls, M5=1.8, mf=0.01, mobius=True, b5=1.5, c5=0.5),
                        torch.from_numpy(U).cuda())
    nat = lqcd.LQ_NATIVE | lqcd.LQ_F32
    nb = lqcd.lq_field_bytes(hm, nat, five_d=True)
    a_, b_ = (torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2))
    lqcd.lq_convert(hm, a_, nat, eta, lqcd.LQ_F64, five_d=True, stream=st)
    ms = _time(lambda: lqcd.dwf_dslash_apply(hm, b_, a_, nat, False, stream=st), st, 20, torch)
    bm = torch.empty_like(eta)
    lqcd.dwf_dslash_apply(hm, bm, eta, lqcd.LQ_F64, True)
    x = torch.zeros_like(bm)
    cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10, maxiter=40000,
                             inner=lqcd.LQ_F32, inner_tol=1e-6)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, stt = lqcd.cg_solve(hm, x, bm, cp, check=False)
    res["mobius_b1.5_c0.5"] = {"dslash_f32_ms": ms, "gflops_4d": FLOP_PER_SITE * V * Ls / (ms * 1e-3) / 1e9,
                               "cg_status": rc, "cg_seconds": time.perf_counter() - t0, "cg_iters": stt[0].iters,
                               "cg_true_rel_residual": stt[0].true_rel_residual,
                               "note": "two 5th-dimension passes + one Wilson hop launch per application"}
    # the same Moebius system through its even-odd Schur complement (FP64 outer, FP32 inner)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bh = torch.empty((Ls, V // 2, 4, 3), dtype=eta.dtype, device="cuda")
    lqcd.dwf_eo_prepare(hm, bh, eta, lqcd.LQ_F64)
    be = torch.empty_like(bh)
    lqcd.dwf_schur_apply(hm, be, bh, lqcd.LQ_F64, True)
    xe = torch.zeros_like(be)
    cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_EO_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10, maxiter=40000,
                             inner=lqcd.LQ_F32, inner_tol=1e-6)
    rc, stt = lqcd.cg_solve(hm, xe, be, cp, check=False)
    psi = torch.empty_like(eta)
    lqcd.dwf_eo_reconstruct(hm, psi, xe, eta, lqcd.LQ_F64)
    torch.cuda.synchronize()
    t_eo = time.perf_counter() - t0
    lqcd.dwf_dslash_apply(hm, Dpsi, psi, lqcd.LQ_F64, False)
    # read before any launch on the timing stream: the handle's workspace serves one stream at a time
    full_eo = float(torch.linalg.vector_norm(Dpsi - eta) / torch.linalg.vector_norm(eta))
    torch.cuda.synchronize()
    nbe = lqcd.lq_field_bytes(hm, nat, lqcd.LQ_EVEN, Ls)
    ae, be_ = (torch.empty(nbe, dtype=torch.uint8, device="cuda") for _ in range(2))
    lqcd.lq_convert(hm, ae, nat, bh, lqcd.LQ_F64, lqcd.LQ_EVEN, Ls, stream=st)
    ms_eo = _time(lambda: lqcd.dwf_schur_apply(hm, be_, ae, nat, False, stream=st), st, 20, torch)
    res["mobius_b1.5_c0.5"]["eo"] = {
        "status": rc, "seconds": t_eo, "iters": stt[0].iters, "outer": stt[0].outer_iters,
        "true_rel_residual": stt[0].true_rel_residual,
        "full_system_rel_residual": full_eo,
        "schur_f32_ms": ms_eo, "gflops_hops": 2 * FLOP_PER_SITE * (V // 2) * Ls / (ms_eo * 1e-3) / 1e9,
        "note": "solve includes source preparation and reconstruction; Schur complement = one 5th-dimension "
                "pass, two half-lattice hops and one inverse-and-B sweep"}
    del ae, be_
    lqcd.lq_destroy(hm)
    del a_, b_
    out["dwf_16x4_ls16"] = res
    out["halo_2rank_32x4"] = halo_emulation(lqcd, torch, hbm)
    out["su3_mul"] = su3_sweep(lqcd, torch, st, hbm, 20)
    A = inputs.gauge_field((16, 16, 16, 16), "random", seed=1000).reshape(-1, 3, 3)  # 262,144 matrices
    dt, _ = oracle_timed(oracle.su3_mul, A, np.roll(A, 1, axis=0))
    out["su3_mul"]["cpu_baseline"] = {"gflops": 198 * len(A) / dt / 1e9, "n": len(A), "cores": cores,
                                      "kind": "oracle", "sample": "one FP64 product over 16^4 x 4 link matrices"}
    return out


def read_tune_file(path, shapes):
    """The batch autotuner's choice for the lattices `shapes` from its cache file: resident
    blocks and 128-site tiles per work item of each lattice."""
    want = ":" + ":".join("x".join(str(d) for d in dd) for dd in shapes)
    try:
        with open(path) as f:
            for line in f:
                tok = line.split()
                if len(tok) >= 3 and tok[0].endswith(want) and int(tok[2]) == len(shapes):
                    mult = [int(v) for v in tok[3:3 + len(shapes)]]
                    return {"blocks": int(tok[1]),
                            "sites_per_item": {"x".join(str(d) for d in dd): 128 * m for dd, m in zip(shapes, mult)},
                            "key": tok[0]}
    except OSError:
        pass
    return None


def inputs_odd(psi_e):
    return psi_e  # any Gaussian half field serves as the odd-parity input


def cpu_baseline(dims, mass, U, psi_e, Vh):
    """Repeat the oracle's Mhat^dag Mhat on the full lattice until >= 10 s (at most 6 times); returns the
    timing entry and the oracle's output."""
    cores = host_cores()
    total, n = 0.0, 0
    while total < 10.0 and n < 6:
        dt, out = oracle_normal_op(dims, mass, U, psi_e)
        total += dt
        n += 1
    return ({"value": 4 * FLOP_PER_SITE * Vh * n / total / 1e9, "unit": "GFlop/s", "cores": cores, "cpu": host_cpu(),
             "kind": "oracle",
             "sample": f"{n} Mhat^dag Mhat applications on the full {list(dims)} lattice, {total:.1f} s"}, out)


if __name__ == "__main__":
    main()
