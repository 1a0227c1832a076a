"""Benchmark of the chi0 hot path (one JSON line on rank 0).

A step is one pass of the whole path over one synthetic q-point: band setup of the
valence and conduction sets (a1), then pair elements, energy factor, contraction,
diagonal-free symmetrisation (a2-a7), chunked over pairs.  Default workload: 48^3
grid, 128 valence + 1024 conduction bands on a 6000-G wavefunction sphere,
N_G = 2000, chunks of 8192 pairs, omega = 0 (about 4.2 TFLOP in the contraction
by the 8 N_G^2 P convention).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|ozaki] [--impl ours|reference]

Multi-GPU: the path has no exchange step; N ranks run N independent q-points
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

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
sys.path.insert(0, ROOT)

import gwgen  # noqa: E402

METRIC = "chi0 TFLOP/s & ms/q-point, FP64 DMMA vs Ozaki-split at stated err, % of roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "ozaki"])
    ap.add_argument("--nslices", type=int, default=6)
    ap.add_argument("--mtxel", default=None, choices=["fp64", "twofloat"],
                    help="stage (a) arithmetic; default fp64 with --prec fp64, twofloat with --prec ozaki")
    ap.add_argument("--config", default="c2_48cube", choices=sorted(gwgen.CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-pairs", type=int, default=4096)
    ap.add_argument("--no-check", action="store_true", help="skip the sampled error check against the oracle")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def conv_flops(cfg, nw=1):
    return 8.0 * cfg.ng ** 2 * cfg.npairs * nw


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, index):
        self.index = index
        self.p = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.p is None:
            return out
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        self.f.close()
        os.unlink(self.f.name)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ---------------------------------------------------------------- oracle baseline
def cpu_baseline(cfg, prob, sample_pairs):
    """The oracle, as it stands, on a bounded sample: sample_pairs pairs x the full sphere."""
    import oracle
    nv_s = max(1, sample_pairs // cfg.nc)
    nc_s = min(cfg.nc, sample_pairs)
    t0 = time.perf_counter()
    M = oracle.m_conv(prob.gpsi, prob.cv[:nv_s], prob.gpsi, prob.cc[:nc_s], prob.gchi)
    dl = oracle.delta(prob.ev[:nv_s], prob.ec[:nc_s], 0.0)
    oracle.chi0(M, dl)
    dt = time.perf_counter() - t0
    P = nv_s * nc_s
    return {"value": 8.0 * cfg.ng ** 2 * P / dt * 1e-12, "unit": "TFLOP/s", "cores": oracle.threads(),
            "kind": "oracle",
            "sample": f"{P} pairs ({nv_s} valence x {nc_s} conduction) x the full N_G={cfg.ng} sphere: "
                      f"M by G-space convolution + compensated chi0 sum, {dt:.1f} s",
            "seconds": dt}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfg = gwgen.CONFIGS[args.config]
    prob = gwgen.config_problem(cfg)
    for _ in range(args.warmup):
        cpu_baseline(cfg, prob, max(16, args.cpu_sample_pairs // 4))
    vals, secs = [], []
    for _ in range(args.steps):
        r = cpu_baseline(cfg, prob, args.cpu_sample_pairs)
        vals.append(r["value"])
        secs.append(r["seconds"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "ms_per_step": 1e3 * statistics.median(secs), "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.name, "grid": list(cfg.grid), "nv": cfg.nv, "nc": cfg.nc,
                       "ngpsi": cfg.ngpsi, "ng": cfg.ng, "sample_pairs": args.cpu_sample_pairs},
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
# DRAM bytes per launch of the dominant kernel, from one ncu capture of an identical launch
# (8192 pairs, N_G = 2000); set to None whenever that kernel changes.
TRAFFIC = {
    "contract_f64": {"bytes_per_launch": 1.941011e9 + 0.034306e9,
                     "source": "ncu dram__bytes_read+write, contract_f64_kernel, p1_48cube_onechunk"},
}


def sampled_error(cfg, prob, chi, nsample=12, seed=3):
    """Relative Frobenius error of a sampled nsample x nsample block of chi against the oracle."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(cfg.ng, nsample, replace=False))
    M = oracle.m_conv(prob.gpsi, prob.cv, prob.gpsi, prob.cc, prob.gchi[idx])
    ref = oracle.chi0(M, oracle.delta(prob.ev, prob.ec, 0.0))
    got = chi[np.ix_(idx, idx)]
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref)), f"{nsample}x{nsample} sampled entries, all pairs"


def peak_for(prec):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    pk = json.load(open(path)) if os.path.exists(path) else {}
    src = "measured" if pk else "fallback"
    bf16_burst = pk.get("bf16_tflops", 1900.0)
    bf16_sus = pk.get("bf16_tflops_sustained", 1700.0)
    if prec == "fp64":
        # FP64 tensor peak = measured bf16 (sustained: the kernel runs inside a long step)
        # x nominal FP64/bf16 dense ratio 1.25 / 2250
        return bf16_sus * 1.25 / 2250.0, f"of {src} bf16 sustained x nominal fp64/bf16 ratio (1.25/2250)"
    return bf16_sus, f"of {src} bf16 sustained"


def ours(args):
    import torch
    import torch.distributed as dist
    import paper_2509_23018_gb300 as gw
    from paper_2509_23018_gb300.shard import max_over_ranks

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    cfg = gwgen.CONFIGS[args.config]
    seed = gwgen.BASE_SEED + cfg.index + 1000 * rank  # each rank: its own q-point
    prob = gwgen.config_problem(cfg, seed=seed)
    dev = torch.device("cuda", local)
    gpsi = torch.as_tensor(prob.gpsi, device=dev)
    cv, cc = torch.as_tensor(prob.cv, device=dev), torch.as_tensor(prob.cc, device=dev)
    ev, ec = torch.as_tensor(prob.ev, device=dev), torch.as_tensor(prob.ec, device=dev)
    gchi = torch.as_tensor(prob.gchi, device=dev)
    omega = [0.0]
    mtxel = args.mtxel or ("fp64" if args.prec == "fp64" else "twofloat")
    h = gw.Chi0(cfg.grid, nq=1, prec=args.prec, nslices=args.nslices, pair_chunk=cfg.pair_chunk, mtxel=mtxel)
    chi = torch.empty(cfg.ng * cfg.ng, dtype=torch.complex128, device=dev)
    h.ng[0] = cfg.ng

    def step():
        h.set_bands(0, 1, gpsi, cc, ec)
        h.set_bands(0, 0, gpsi, cv, ev)
        h.set_gsphere(0, gchi)
        h.compute(0, omega, out=chi)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    h.sync()
    h.set_timing(True)
    h.timing(reset=True)
    clk = Clocks(local)
    clk.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    tim = h.timing(reset=True)
    h.set_timing(False)
    h.sync()
    ms = max_over_ranks(ms, device=dev)
    ms_step = ms / args.steps
    value = conv_flops(cfg) * world * args.steps / (ms * 1e-3) * 1e-12
    launches = int(sum(v[1] for v in tim.values()))

    # dominant kernel: the contraction
    kname = "contract_f64" if args.prec == "fp64" else "ozaki_gemm"
    kms, kn = tim.get(kname, (0.0, 0))
    nchunk = -(-cfg.npairs // cfg.pair_chunk)
    per_launch_flops = 4.0 * cfg.ng * (cfg.ng + 1) * cfg.npairs / nchunk
    if args.prec == "ozaki":
        # low-precision flops of the kept slice pairs: s(s+1)/2 x 4 N_G^2 P per chunk and frequency
        per_launch_flops = args.nslices * (args.nslices + 1) / 2 * 4.0 * cfg.ng ** 2 * cfg.npairs / nchunk
    peak, peak_src = peak_for(args.prec)
    achieved = per_launch_flops / (kms / kn * 1e-3) * 1e-12 if kn else None
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": None, "kernel": kname,
                "launches": kn, "ms_per_launch": kms / kn if kn else None,
                "flops_per_launch": per_launch_flops, "peak_source": peak_src,
                "share_of_step": kms / ms if ms else None,
                "fp64_probe_peaks_tflops": {"dmma": 1.055, "dfma": 1.204},
                "traffic_source": TRAFFIC.get(kname, {}).get("source")}
    roofline["traffic"] = TRAFFIC.get(kname, {}).get("bytes_per_launch")

    # end to end through the public API with host buffers (pinned), H2D inputs + D2H result
    e2e = None
    if not args.no_e2e:
        hcv, hcc = cv.cpu().pin_memory(), cc.cpu().pin_memory()
        hev, hec = ev.cpu().pin_memory(), ec.cpu().pin_memory()
        hg, hgc = gpsi.cpu().pin_memory(), gchi.cpu().pin_memory()
        hout = torch.empty(cfg.ng * cfg.ng, dtype=torch.complex128).pin_memory()

        def e2e_step():
            d = [x.to(dev, non_blocking=True) for x in (hg, hcv, hcc, hev, hec, hgc)]
            h.set_bands(0, 1, d[0], d[2], d[4])
            h.set_bands(0, 0, d[0], d[1], d[3])
            h.set_gsphere(0, d[5])
            h.compute(0, omega, out=chi)
            hout.copy_(chi, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        es = t1 - t0
        es = max_over_ranks(es, device=dev)
        h2d = sum(x.numel() * x.element_size() for x in (hg, hcv, hcc, hev, hec, hgc))
        e2e = {"value": conv_flops(cfg) * world * args.steps / es * 1e-12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(hout.numel() * hout.element_size()),
               "ms_per_step": 1e3 * es / args.steps}

    err = None
    if rank == 0 and not args.no_check:
        e, how = sampled_error(cfg, prob, chi.view(cfg.ng, cfg.ng).cpu().numpy())
        err = {"rel_frobenius_vs_oracle": e, "sample": how}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg, prob, args.cpu_sample_pairs)
        cpu.pop("seconds", None)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "ms_per_q": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "bf16-split/f64",
                "data": "synthetic",
                "config": {"workload": f"{cfg.name}: grid {cfg.grid[0]}^3, {cfg.nv}+{cfg.nc} bands, "
                                       f"N_Gpsi={cfg.ngpsi}, N_G={cfg.ng}, chunks of {cfg.pair_chunk} pairs, omega=0",
                           "prec": args.prec, "nslices": args.nslices if args.prec == "ozaki" else None,
                           "mtxel": mtxel,
                           "pairs": cfg.npairs, "conv_tflop_per_step": conv_flops(cfg) * 1e-12,
                           "l2": "inputs larger than L2 (psi grids 2.0 GB, M chunks 262 MB)",
                           "parallelism": f"replicas x{world} (independent q-points)"},
                "error": err, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "kernel_ms": {k: v[0] for k, v in tim.items()}, "clocks": clocks}
        print(json.dumps(line), flush=True)
    h.destroy()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
