"""Benchmark of the chi0 hot path (one JSON line on rank 0).

A step is one pass of the whole path over one synthetic q-point: band setup of the
valence and conduction sets (a1), then pair elements, energy factor, contraction,
diagonal-free symmetrisation (a2-a7), chunked over pairs.  Default workload: 48^3
grid, 128 valence + 1024 conduction bands on a 6000-G wavefunction sphere,
N_G = 2000, chunks of 8192 pairs, omega = 0 (about 4.2 TFLOP in the contraction
by the 8 N_G^2 P convention).

The headline mode is the split-precision contraction (7 BF16 slices, two-float stage
(a)) with its error against the oracle stated on sampled entries; the same line carries
the native FP64 tensor-core path on the same input under "fp64_dmma".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|ozaki] [--impl ours|reference]
    python bench.py --sweep      slice-count sweep on one 72^3 chunk (error and throughput)
    python bench.py --batch      64 q-points x 16 frequencies in one graph (40^3)
    python bench.py --adjoint    adjoint of Re Tr(W chi) on 40^3, 96+768 bands, N_G = 1500

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
    ap.add_argument("--prec", default="ozaki", choices=["fp64", "ozaki"])
    ap.add_argument("--nslices", type=int, default=7)
    ap.add_argument("--path", default="stream", choices=["batch", "stream"],
                    help="batch: resident M, persistent contraction, CUDA graph (gw_chi0_compute_batch); "
                         "stream: chunk-by-chunk launches (gw_chi0_compute)")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the native FP64 DMMA run on the same input (split-precision mode only)")
    ap.add_argument("--mtxel", default=None, choices=["fp64", "twofloat"],
                    help="stage (a) arithmetic; default fp64 with --prec fp64, twofloat with --prec ozaki")
    ap.add_argument("--config", default="c2_48cube", choices=sorted(gwgen.CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-pairs", type=int, default=4096)
    ap.add_argument("--no-check", action="store_true", help="skip the sampled error check against the oracle")
    ap.add_argument("--peaks", action="store_true", help="measure the pipe peaks, write profiles/peaks_gb300.json")
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--sweep-fp64", action="store_true", help="with --sweep --config c3_72cube: also native FP64")
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--subspace", action="store_true")
    ap.add_argument("--epsilon", action="store_true")
    ap.add_argument("--extras", action="store_true", help="real-axis chi and the forward derivative")
    ap.add_argument("--sigma", action="store_true", help="off-diagonal plasmon-pole self-energy")
    ap.add_argument("--sigma-ng", type=int, default=11075)
    ap.add_argument("--sigma-nsig", type=int, default=512)
    ap.add_argument("--sigma-ne", type=int, default=16, help="energies per step (the default workload: 16)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def conv_flops(cfg, nw=1):
    return 8.0 * cfg.ng ** 2 * cfg.npairs * nw


def gpp_offdiag_flops(nb, ne, nsig, ng):
    """FLOP count of the off-diagonal GPP kernel as Eq. flop_count_fullmat states it:
    2 N_b N_E x 8 (N_Sigma N_G^2 + N_G N_Sigma^2).  The paper's printed throughputs use this
    count (the Si998 rows of its best-throughput table)."""
    return 2.0 * nb * ne * 8.0 * (nsig * ng * ng + ng * nsig * nsig)


def gpp_products_flops(nb, ne, nsig, ng):
    """ZGEMM flops of the products this path runs: one pair per (n, E), X^T = P^T conj(M_n)^T
    (8 N_Sigma N_G^2) and Sigma^T += M_n X^T (8 N_G N_Sigma^2), half of the count above."""
    return nb * ne * 8.0 * (nsig * ng * ng + ng * nsig * nsig)


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


def oracle_block(cfg, prob, nsample=24, seed=3):
    """Reference values for the error check, from the oracle on a bounded sample: the
    nsample x nsample block of chi(0) at sampled G, all pairs.  Runs only with the CPU baseline."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(cfg.ng, nsample, replace=False))
    M = oracle.m_conv(prob.gpsi, prob.cv, prob.gpsi, prob.cc, prob.gchi[idx])
    ref = oracle.chi0(M, oracle.delta(prob.ev, prob.ec, 0.0))
    return idx, ref, cfg.ng


def block_error(chi, blk):
    """Error of chi against the oracle's sampled block, as an estimate of the relative Frobenius
    error over the whole N_G x N_G matrix.  The diagonal (sums of squares) carries a small share
    of the matrix's entries but most of a small block's norm, and far smaller relative errors
    than the off-diagonal entries; so the two strata are weighted by their shares of the whole
    matrix: N_G diagonal and N_G (N_G - 1) off-diagonal entries."""
    idx, ref, ng = blk
    n = len(idx)
    d = chi[np.ix_(idx, idx)] - ref
    on = np.eye(n, dtype=bool)
    e_d, r_d = float(np.sum(np.abs(d[on]) ** 2)), float(np.sum(np.abs(ref[on]) ** 2))
    e_o, r_o = float(np.sum(np.abs(d[~on]) ** 2)), float(np.sum(np.abs(ref[~on]) ** 2))
    wd, wo = ng / n, ng * (ng - 1.0) / (n * (n - 1.0))
    return {"rel_frobenius_vs_oracle": ((wd * e_d + wo * e_o) / (wd * r_d + wo * r_o)) ** 0.5,
            "offdiag_rel": (e_o / r_o) ** 0.5, "diag_rel": (e_d / r_d) ** 0.5,
            "block_rel": ((e_d + e_o) / (r_d + r_o)) ** 0.5,
            "sample": f"oracle on the {n}x{n} block of chi at {n} sampled G (all pairs); the full-matrix "
                      f"estimate weights its {n} diagonal and {n * (n - 1)} off-diagonal entries by their "
                      f"shares of the {ng}x{ng} matrix"}


def oracle_sigma_rows(p, n0, eidx, rows):
    """Oracle Sigma rows for one (n, E) of the plasmon-pole workload (P formed once), timed as the
    CPU baseline of that mode: the oracle's rate on this sample in the same flop convention."""
    import oracle
    t0 = time.perf_counter()
    P = oracle.gpp_pole_matrix(p.omega2, p.wtilde, p.vcoul, float(p.E[eidx] - p.En[n0]), n0 < p.nocc)
    ref = (p.M[n0][rows].conj() @ P) @ p.M[n0].T
    dt = time.perf_counter() - t0
    ng, nsig = P.shape[0], p.M.shape[1]
    fl = 8.0 * (len(rows) * ng * ng + ng * len(rows) * nsig)
    return ref, {"value": fl / dt * 1e-12, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
                 "sample": f"one (n, E): P^n(E) formed and {len(rows)} rows of Sigma, {dt:.1f} s"}


def oracle_adjoint_sample(prob, W, nvs):
    """The oracle adjoint on nvs valence bands x all conduction bands, scaled to every pair."""
    import oracle
    t0 = time.perf_counter()
    oracle.adjoint(prob.gpsi, prob.cv[:nvs], prob.ev[:nvs], prob.gpsi, prob.cc, prob.ec, prob.gchi, W, 0.0)
    dt = time.perf_counter() - t0
    nv, nc = len(prob.ev), len(prob.ec)
    return {"value": dt * nv / nvs, "unit": "s per adjoint", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{nvs} valence x {nc} conduction bands ({nvs * nc} of {nv * nc} pairs): {dt:.1f} s, "
                      "scaled by the pair count"}


def oracle_chi_sample(prob, npairs, omegas, basis=None, eta=None):
    """The oracle on npairs pairs x the full sphere: M by the G-space convolution, then chi at the
    given frequencies (in the subspace when basis is given, on the real axis when eta is given).
    Returns (seconds for M, seconds per frequency, description)."""
    import oracle
    nc = len(prob.ec)
    nvs = max(1, npairs // nc)
    ncs = min(nc, npairs)
    t0 = time.perf_counter()
    M = oracle.m_conv(prob.gpsi, prob.cv[:nvs], prob.gpsi, prob.cc[:ncs], prob.gchi)
    t1 = time.perf_counter()
    for w in omegas:
        if eta is not None:
            oracle.chi0_real(M, oracle.delta_real(prob.ev[:nvs], prob.ec[:ncs], w, eta))
        elif basis is not None:
            oracle.chi0_subspace(M, oracle.delta(prob.ev[:nvs], prob.ec[:ncs], w), basis)
        else:
            oracle.chi0(M, oracle.delta(prob.ev[:nvs], prob.ec[:ncs], w))
    t2 = time.perf_counter()
    return (t1 - t0, (t2 - t1) / max(1, len(omegas)),
            f"{nvs * ncs} pairs x the full sphere, {len(omegas)} frequencies", oracle.threads())


def oracle_epsilon_sample(chi, v):
    import oracle
    t0 = time.perf_counter()
    oracle.epsilon_inverse(chi, v)
    return time.perf_counter() - t0, oracle.threads()


def workload_name(cfg):
    """The workload both arms name in their config."""
    return (f"{cfg.name}: grid {cfg.grid[0]}^3, {cfg.nv}+{cfg.nc} bands, N_Gpsi={cfg.ngpsi}, N_G={cfg.ng}, "
            f"chunks of {cfg.pair_chunk} pairs, omega=0")


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
            "config": {"workload": workload_name(cfg), "grid": list(cfg.grid), "nv": cfg.nv, "nc": cfg.nc,
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
    # the FFT route of stage (a) (fp64 and pre-tensor-core paths): taken before the tensor-core
    # route existed; the kernel is unchanged since
    "pair_mtxel": {"bytes_per_launch": 3.112e9 + 1.486e9,
                   "source": "ncu dram__bytes_read+write, pair_kernel_tf_ct<48>, p1_48cube_onechunk"},
    # the tensor-core route of the 48^3 workload: one 8192-pair chunk (128 valence x 64
    # conduction bands), the launch shape the bench's step repeats 16 times
    "zdft": {"bytes_per_launch": 0.477185e9 + 4.482903e9,
             "source": "ncu dram__bytes_read+write, zd_gemm_kernel (128-column tiles), p2_48cube_chunk"},
    "pair_from_f": {"bytes_per_launch": 5.504037e9 + 1.240109e9,
                    "source": "ncu dram__bytes_read+write, pair_kernel_tf_from_f<48> (TMA-fed), p2_48cube_chunk"},
    # the single-stream launch (4-deep TMA ring) the tensor-core route runs
    "ozaki_gemm": {"bytes_per_launch": 5.176667e9 + 0.212558e9,
                   "source": "ncu dram__bytes_read+write, oz_gemm_kernel<240,0,4> (s = 7), p2_48cube_chunk"},
    "ozaki_gemm_single_stream": {"bytes_per_launch": 5.176667e9 + 0.212558e9,
                                 "source": "ncu dram__bytes_read+write, oz_gemm_kernel<240,0,4> (s = 7), "
                                           "p2_48cube_chunk"},
}


# the launch shape of every capture above: 48^3 grid, N_G = 2000, 8192 pairs per launch
TRAFFIC_SHAPE = ((48, 48, 48), 2000, 8192)


def traffic_for(key, cfg):
    """(DRAM bytes per launch, source) of a kernel, or (None, why) when the captures were taken
    on another launch shape than cfg's."""
    t = TRAFFIC.get(key) or {}
    if t.get("bytes_per_launch") is None:
        return None, None
    if (tuple(cfg.grid), cfg.ng, min(cfg.pair_chunk, cfg.npairs)) != TRAFFIC_SHAPE:
        return None, "no ncu capture of this launch shape (captures: 48^3, N_G = 2000, 8192 pairs per launch)"
    return t["bytes_per_launch"], t["source"]


# ---------------------------------------------------------------- pipe peaks
# Rates of the arithmetic pipes, measured by the library's probes (gw_chi0_probe) on this GPU:
# filled by measure_peaks() at the start of a run; profiles/peaks_gb300.json (written by
# `bench.py --peaks`) is the record of one such measurement and the fallback.
PEAKS_JSON = os.path.join(ROOT, "profiles", "peaks_gb300.json")
PROBE_KINDS = ["ffma", "ffma2", "fadd2", "dfma", "dmma_m8n8k4", "dmma_m16n8k16", "bf16_mma_sync", "int8_mma_sync",
               "tcgen05_n64", "tcgen05_n128", "tcgen05_n256"]
LIVE_PEAKS = {}


def probe_rates(kinds, target_ms=25.0, reps=3):
    """Peak rate (T operations/s; an FMA counts 2) of each probe kind: one calibration launch
    sizes the chain length for about target_ms, then the best of `reps` timed launches (CUDA
    events on the launching stream)."""
    import ctypes

    import torch
    from paper_2509_23018_gb300 import _lib

    lib = _lib.load()
    sink = torch.zeros(256, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    out = {}
    def launch(k, iters):
        ops = ctypes.c_double()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc = lib.gw_chi0_probe(_lib.PROBES[k], iters, ctypes.c_void_p(st.cuda_stream),
                               ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops))
        e1.record(st)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError(f"gw_chi0_probe({k}) failed: {rc}")
        return e0.elapsed_time(e1), ops.value

    for k in kinds:
        iters, ms = 64, 0.0
        while True:  # calibration: grow the chains until a launch takes a good part of target_ms
            ms, _ = launch(k, iters)
            if ms >= 0.3 * target_ms or iters > (1 << 30):
                break
            iters = int(iters * min(64.0, max(2.0, target_ms / max(ms, 1e-3))))
        iters = max(64, int(iters * target_ms / max(ms, 1e-3)))
        best = 0.0
        for _ in range(reps):
            ms, ops = launch(k, iters)
            best = max(best, ops / (ms * 1e-3) * 1e-12)
        out[k] = {"tops": best, "iters": iters, "ms": ms}
    return out


def measure_peaks(kinds=("ffma", "ffma2", "dfma", "dmma_m8n8k4", "dmma_m16n8k16")):
    """Fill LIVE_PEAKS from the probes on this GPU (falls back to the committed record)."""
    try:
        LIVE_PEAKS.update({k: v["tops"] for k, v in probe_rates(list(kinds)).items()})
        LIVE_PEAKS["_source"] = "measured in this run (gw_chi0_probe)"
    except Exception as e:  # noqa: BLE001
        if os.path.exists(PEAKS_JSON):
            rec = json.load(open(PEAKS_JSON))
            LIVE_PEAKS.update({k: v["tops"] for k, v in rec.get("probes", {}).items()})
            LIVE_PEAKS["_source"] = f"profiles/peaks_gb300.json ({rec.get('when')}); live probe failed: {e}"


def fp64_tensor_peak():
    """FP64 tensor peak (TFLOP/s): the faster of the two measured DMMA shapes."""
    r = [LIVE_PEAKS.get(k) for k in ("dmma_m8n8k4", "dmma_m16n8k16") if LIVE_PEAKS.get(k)]
    if r:
        return max(r), f"measured DMMA (gw_chi0_probe; {LIVE_PEAKS.get('_source')})"
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    pk = json.load(open(path)) if os.path.exists(path) else {}
    return pk.get("bf16_tflops_sustained", 1700.0) * 1.25 / 2250.0, "bf16 sustained x nominal fp64/bf16 ratio"


def fp32_lane_peak():
    """FP32 operations per second (T; one FMA = one operation) of the FP32 pipes: the faster of
    the scalar and the packed two-lane FMA probes, else lanes x max clock."""
    r = [LIVE_PEAKS.get(k) for k in ("ffma", "ffma2") if LIVE_PEAKS.get(k)]
    if r:
        return max(r) / 2.0, f"measured FFMA/FFMA2 (gw_chi0_probe; {LIVE_PEAKS.get('_source')})"
    return FP32_PEAK_TOPS, "152 SMs x 128 FP32 lanes x 2070 MHz (one operation per lane per clock)"


def peak_for(prec):
    if prec == "fp64":
        return fp64_tensor_peak()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    pk = json.load(open(path)) if os.path.exists(path) else {}
    src = "measured" if pk else "fallback"
    return pk.get("bf16_tflops_sustained", 1700.0), f"of {src} bf16 sustained (cuBLAS)"


def run_mode(args, cfg, prob, dev, prec, nslices, mtxel, steps, warmup, with_e2e, world, single_stream=False):
    """Time `steps` passes of the whole path in one precision mode; returns a result dict."""
    import torch
    import paper_2509_23018_gb300 as gw
    from paper_2509_23018_gb300.shard import max_over_ranks

    gpsi = torch.as_tensor(prob.gpsi, device=dev)
    cv, cc = torch.as_tensor(prob.cv, device=dev), torch.as_tensor(prob.cc, device=dev)
    ev, ec = torch.as_tensor(prob.ev, device=dev), torch.as_tensor(prob.ec, device=dev)
    gchi = torch.as_tensor(prob.gchi, device=dev)
    omega = [0.0]
    h = gw.Chi0(cfg.grid, nq=1, prec=prec, nslices=nslices, pair_chunk=cfg.pair_chunk, mtxel=mtxel,
                single_stream=single_stream)
    chi = torch.empty(cfg.ng * cfg.ng, dtype=torch.complex128, device=dev)
    h.ng[0] = cfg.ng

    run = h.compute_batch if args.path == "batch" else h.compute

    def step():
        h.set_bands(0, 1, gpsi, cc, ec)
        h.set_bands(0, 0, gpsi, cv, ev)
        h.set_gsphere(0, gchi)
        run([0], omega, out=chi)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    h.sync()
    h.set_timing(True)
    h.timing(reset=True)
    clk = Clocks(dev.index)
    clk.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), device=dev)
    tim = h.timing(reset=True)
    h.set_timing(False)
    h.sync()
    res = {"ms_per_step": ms / steps, "value": conv_flops(cfg) * world * steps / (ms * 1e-3) * 1e-12,
           "launches": int(sum(v[1] for v in tim.values())), "kernel_ms": {k: v[0] for k, v in tim.items()},
           "clocks": clocks, "timing": tim, "total_ms": ms, "streams": h.streams(0)}

    e2e = None
    if with_e2e:
        hcv, hcc = cv.cpu().pin_memory(), cc.cpu().pin_memory()
        hev, hec = ev.cpu().pin_memory(), ec.cpu().pin_memory()
        hg, hgc = gpsi.cpu().pin_memory(), gchi.cpu().pin_memory()
        hout = torch.empty(cfg.ng * cfg.ng, dtype=torch.complex128).pin_memory()

        def e2e_step():
            d = [x.to(dev, non_blocking=True) for x in (hg, hcv, hcc, hev, hec, hgc)]
            h.set_bands(0, 1, d[0], d[2], d[4])
            h.set_bands(0, 0, d[0], d[1], d[3])
            h.set_gsphere(0, d[5])
            run([0], omega, out=chi)
            hout.copy_(chi, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            e2e_step()
        torch.cuda.synchronize()
        es = max_over_ranks(time.perf_counter() - t0, device=dev)
        h2d = sum(x.numel() * x.element_size() for x in (hg, hcv, hcc, hev, hec, hgc))
        e2e = {"value": conv_flops(cfg) * world * steps / es * 1e-12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(hout.numel() * hout.element_size()),
               "ms_per_step": 1e3 * es / steps}
    res["e2e"] = e2e
    res["chi"] = chi.view(cfg.ng, cfg.ng).cpu().numpy()
    h.destroy()
    return res


# FP32 operations of the two-float arithmetic as the kernels implement it (fft_tf.cuh):
# tf_addl 8, tf_norm 3, tf_add 11, tf_mul 7, tf_dot2 19, tf_dot2l 16, tf_acc2 24; a complex
# multiply is 2 tf_dot2 (38), a lazy twiddle multiply 2 tf_dot2l (32), an accumulation 2 tf_acc2.
_CMUL = 38
_CMUL_L = 32
_ACC = 48


def _rad_plan(n):
    """Radix order of the transforms (3s, 5s, 4s, one 8 from a 2 and a 4, 2)."""
    m, n4, n2, n3, n5 = n, 0, 0, 0, 0
    while m % 4 == 0:
        n4, m = n4 + 1, m // 4
    while m % 2 == 0:
        n2, m = n2 + 1, m // 2
    while m % 3 == 0:
        n3, m = n3 + 1, m // 3
    while m % 5 == 0:
        n5, m = n5 + 1, m // 5
    n8 = 0
    if n2 and n4:
        n2, n4, n8 = 0, n4 - 1, 1
    return [3] * n3 + [5] * n5 + [4] * n4 + [8] * n8 + [2] * n2


def _prune_radix(n):
    return 3 if n % 3 == 0 else (2 if n % 2 == 0 else 5)


def _bfly_ops(r, twiddled, lazy=False):
    """One butterfly: the radix-r sums (a lazy radix-4 skips its 4 renormalisations) plus
    r - 1 lazy twiddle products."""
    base = {2: 2 * 2 * 11, 3: 12 * 8 + 2 * 7 + 4 + 6 * 3, 4: 16 * 8 + 8 * 3,
            5: 8 * 11 + 2 * 11 + 2 * (4 * 7 + 2 * 11) * 2 + 4 * 2 * 11,
            8: 2 * 128 + 2 * (2 * 8 + 2 * 7) + 16 * 8 + 16 * 3}[r]
    if lazy and r == 4:
        base -= 8 * 3
    return base + ((r - 1) * _CMUL_L if twiddled else 0)


def _head_ops(n, lazy=False):
    """All stages but the pruned last one of the pruned plan, per line."""
    ops, ns = 0, 1
    for r in _rad_plan(n // _prune_radix(n)):
        ops += (n // r) * _bfly_ops(r, ns > 1, lazy)
        ns *= r
    return ops


def _prune_out_ops(n):
    """One output of the pruned last stage: R - 1 lazy twiddle products and sums, one renormalisation."""
    return (_prune_radix(n) - 1) * (_CMUL_L + 16) + 6


def twofloat_ops_per_pair(cfg, k2, k12):
    """FP32 operations of the two-float pair kernel per pair: the lazy product, i2 transform of
    every line (lazy butterflies, pruned to the k2 kept columns), i1 transform of those columns
    (pruned to the k12 cells of the sphere), i0 transform of the k12 cell columns (pruned
    to the sphere points)."""
    n0, n1, n2 = cfg.grid
    i2 = n1 * (_head_ops(n2, lazy=True) + k2 * _prune_out_ops(n2))
    i1 = k2 * _head_ops(n1, lazy=True) + k12 * _prune_out_ops(n1)
    i0 = k12 * _head_ops(n0, lazy=True) + cfg.ng * _prune_out_ops(n0)
    return n0 * (n1 * n2 * _CMUL_L + i2 + i1) + i0


def cells(prob, n):
    """Number of (k1, k2) cells of the sphere."""
    return len(set((int(g[1]) % n[1], int(g[2]) % n[2]) for g in prob.gchi))


def kept_columns(prob, n2):
    return len(set(int(g) % n2 for g in prob.gchi[:, 2]))


FP32_PEAK_TOPS = 152 * 128 * 2.070e9 * 1e-12  # lanes x max SM clock: FP32 operations per second, in T


def _full_ops(n):
    """A full two-float line transform of n points, every stage renormalised."""
    ops, ns = 0, 1
    for r in _rad_plan(n):
        ops += (n // r) * _bfly_ops(r, ns > 1)
        ns *= r
    return ops


def backprojection_ops_per_pair(cfg, k2):
    """FP32 operations of the two-float adjoint back-projection per pair: per i0 slab the sphere's
    sums per (k1, k2) cell (a complex product and a complex sum per point), K2 lines along i1,
    N1 lines along i2, the scaled conjugate of the slab."""
    n0, n1, n2 = cfg.grid
    return n0 * (cfg.ng * (_CMUL + 22) + k2 * _full_ops(n1) + n1 * _full_ops(n2) + n1 * n2 * 14)


def _hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    pk = json.load(open(path)) if os.path.exists(path) else {}
    return (pk["hbm_gbs"], "measured") if "hbm_gbs" in pk else (6800.0, "fallback")


def oz_kpad(ka):
    """Real K extent of a general split product with ka complex inner entries (padded to 64)."""
    return (2 * ka + 63) // 64 * 64


def mode_roofline(bound, kernel, work, ms, unit_of_work, prec="ozaki"):
    """Roofline object of one kernel in a side mode: work (FP32 operations, low-precision flops or
    bytes) over its measured time."""
    if not ms:
        return None
    if bound == "alu":
        peak, src = fp32_lane_peak()
        unit = "FP32 Tops/s"
        ach = work / (ms * 1e-3) * 1e-12
    elif bound == "hbm":
        peak, src = _hbm_peak()
        unit, src = "GB/s", f"{src} copy bandwidth"
        ach = work / (ms * 1e-3) * 1e-9
    else:
        peak, src = peak_for(prec)
        unit = "TFLOP/s"
        ach = work / (ms * 1e-3) * 1e-12
    return {"bound": bound, "kernel": kernel, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
            "traffic": None, "ms": ms, "work": work, "unit_of_work": unit_of_work, "peak_source": src}




def method_stage_a(cfg):
    """Stage (a)'s method-level work per step: the algorithmic bytes (read every band grid once,
    write M once) and the FFT flops of the pruned transforms (half of 5 N_r log2 N_r per pair)
    plus the pair product (6 flops per point)."""
    n0, n1, n2 = cfg.grid
    nr = n0 * n1 * n2
    nbytes = (cfg.nv + cfg.nc) * nr * 16 + cfg.npairs * cfg.ng * 16
    flops = cfg.npairs * (0.5 * 5 * nr * np.log2(nr) + 6 * nr)
    return float(nbytes), float(flops)


ZD_SLICES, ZD_TILE_N, ZD_TILE_M = 6, 128, 128


def zd_ops(cfg, prob):
    """Work of stage (a) on the tensor-core route per chunk: the low-precision flops the last-axis
    split product executes (21 kept slice products of 128 x 128 x 2N tiles, padding included) and
    the useful share, and the FP32 operations of the middle/first-axis kernel per pair."""
    n0, n1, n2 = cfg.grid
    k2 = kept_columns(prob, n2)
    ct = min(4, ZD_TILE_N // (2 * k2))
    cb = max(1, cfg.pair_chunk // cfg.nv)
    tiles = n0 * n1 * -(-cfg.nv // ZD_TILE_M) * -(-cb // ct)
    prods = ZD_SLICES * (ZD_SLICES + 1) // 2
    flops = prods * 2.0 * ZD_TILE_M * ZD_TILE_N * 2 * n2 * tiles
    useful = prods * 8.0 * n2 * k2 * cfg.nv * cb * n0 * n1  # complex MACs of the kept outputs
    k12 = cells(prob, cfg.grid)
    i1 = k2 * _head_ops(n1, lazy=True) + k12 * _prune_out_ops(n1)
    i0 = k12 * _head_ops(n0, lazy=True) + cfg.ng * _prune_out_ops(n0)
    return flops, useful, n0 * i1 + i0, cb


def roofline_zd(cfg, prob, res):
    """Rooflines of the tensor-core stage (a): the last-axis split product (tensor) and the
    middle/first-axis kernel (FP32 issue), each per launch; plus the method-level stage (a)
    numbers over both."""
    flops, useful, ops_pair, cb = zd_ops(cfg, prob)
    out = {}
    kms, kn = res["timing"].get("zdft", (0.0, 0))
    if kn:
        peak, src = peak_for("ozaki")
        ach = flops / (kms / kn * 1e-3) * 1e-12
        out["zdft"] = {"bound": "tensor", "kernel": "zd_gemm_kernel", "achieved": ach, "peak": peak,
                       "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic_for("zdft", cfg)[0],
                       "traffic_source": traffic_for("zdft", cfg)[1], "launches": kn,
                       "ms_per_launch": kms / kn, "flops_per_launch": flops, "useful_share": useful / flops,
                       "peak_source": src, "share_of_step": kms / res["total_ms"],
                       "unit_of_work": "BF16 flops of the 21 kept slice products (128 x 128 tiles, K = 2N)"}
    kms2, kn2 = res["timing"].get("pair_from_f", (0.0, 0))
    if kn2:
        peak, src = fp32_lane_peak()
        per_launch = ops_pair * cfg.nv * cb
        ach = per_launch / (kms2 / kn2 * 1e-3) * 1e-12
        out["pair_from_f"] = {"bound": "alu", "kernel": "pair_kernel_tf_from_f", "achieved": ach, "peak": peak,
                              "unit": "FP32 Tops/s", "frac": ach / peak,
                              "traffic": traffic_for("pair_from_f", cfg)[0],
                              "traffic_source": traffic_for("pair_from_f", cfg)[1], "launches": kn2,
                              "ms_per_launch": kms2 / kn2, "ops_per_launch": per_launch, "ops_per_pair": ops_pair,
                              "peak_source": src, "share_of_step": kms2 / res["total_ms"],
                              "unit_of_work": "FP32 operations of the two-float i1 and i0 transforms as implemented"}
    if kn and kn2:
        mbytes, mflops = method_stage_a(cfg)
        hbm, hbm_src = _hbm_peak()
        nchunk = -(-cfg.nc // cb)
        t_step = (kms / kn + kms2 / kn2) * 1e-3 * nchunk
        dfma = LIVE_PEAKS.get("dfma")
        out["stage_a_method"] = {"bytes_per_step": mbytes, "flops_per_step": mflops,
                                 "hbm_frac": mbytes / t_step * 1e-9 / hbm, "hbm_peak_gbs": hbm,
                                 "hbm_peak_source": hbm_src, "fp64_equiv_tflops": mflops / t_step * 1e-12,
                                 "fp64_alu_peak_tflops": dfma,
                                 "fp64_alu_frac": mflops / t_step * 1e-12 / dfma if dfma else None,
                                 "note": "bytes: every band grid read once + M written once; flops: half of "
                                         "5 N_r log2 N_r per pair (output-pruned FFT) + 6 N_r for the product"}
    return out


def roofline_pair(cfg, prob, res):
    kms, kn = res["timing"].get("pair_mtxel", (0.0, 0))
    nchunk = -(-cfg.npairs // cfg.pair_chunk)
    per_pair = twofloat_ops_per_pair(cfg, kept_columns(prob, cfg.grid[2]), cells(prob, cfg.grid))
    per_launch = per_pair * cfg.npairs / nchunk
    ms_launch = kms / kn if kn else None
    achieved = per_launch / (ms_launch * 1e-3) * 1e-12 if kn else None
    peak, peak_src = fp32_lane_peak()
    # the method-level bound of stage (a): max(HBM bytes, FP64 ALU flops)
    mbytes, mflops = method_stage_a(cfg)
    hbm, hbm_src = _hbm_peak()
    dfma = LIVE_PEAKS.get("dfma")
    t_step = kms * 1e-3 * nchunk / kn if kn else None
    traffic = traffic_for("pair_mtxel", cfg)[0]
    method = {"bytes_per_step": mbytes, "flops_per_step": mflops,
              "hbm_frac": (mbytes / t_step * 1e-9 / hbm) if t_step else None, "hbm_peak_gbs": hbm,
              "hbm_peak_source": hbm_src,
              "fp64_equiv_tflops": (mflops / t_step * 1e-12) if t_step else None,
              "fp64_alu_peak_tflops": dfma, "fp64_alu_frac": (mflops / t_step * 1e-12 / dfma) if t_step and dfma
              else None,
              "dram_bytes_per_step_ncu": traffic * nchunk if traffic else None,
              "dram_over_method_bytes": traffic * nchunk / mbytes if traffic else None,
              "note": "bytes: every band grid read once + M written once; flops: half of 5 N_r log2 N_r per "
                      "pair (output-pruned FFT) + 6 N_r for the product, FP64 arithmetic"}
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "FP32 Tops/s",
            "frac": achieved / peak if achieved else None,
            "traffic": traffic, "kernel": "pair_kernel_tf_ct",
            "launches": kn, "ms_per_launch": ms_launch, "ops_per_launch": per_launch,
            "ops_per_pair": per_pair, "peak_source": peak_src,
            "unit_of_work": "FP32 operations of the two-float transforms as implemented (issue efficiency)",
            "share_of_step": kms / res["total_ms"] if res["total_ms"] else None,
            "traffic_source": traffic_for("pair_mtxel", cfg)[1], "method": method,
            "method_bytes": mbytes, "method_flops": mflops, "hbm_frac": method["hbm_frac"]}


def roofline_for(cfg, prec, nslices, res, single_stream=False):
    kname = "contract_f64" if prec == "fp64" else "ozaki_gemm"
    tkey = kname + ("_single_stream" if single_stream and prec != "fp64" else "")
    kms, kn = res["timing"].get(kname, (0.0, 0))
    nchunk = -(-cfg.npairs // cfg.pair_chunk)
    per_launch_flops = 4.0 * cfg.ng * (cfg.ng + 1) * cfg.npairs / nchunk
    if prec == "ozaki":
        # low-precision flops of the kept slice pairs: s(s+1)/2 x 4 N_G^2 P per chunk and frequency
        per_launch_flops = nslices * (nslices + 1) / 2 * 4.0 * cfg.ng ** 2 * cfg.npairs / nchunk
    peak, peak_src = peak_for(prec)
    achieved = per_launch_flops / (kms / kn * 1e-3) * 1e-12 if kn else None
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic_for(tkey, cfg)[0], "kernel": kname,
            "launches": kn, "ms_per_launch": kms / kn if kn else None, "flops_per_launch": per_launch_flops,
            "peak_source": peak_src, "share_of_step": kms / res["total_ms"] if res["total_ms"] else None,
            "traffic_source": traffic_for(tkey, cfg)[1],
            "probe_peaks_tops": {k: v for k, v in LIVE_PEAKS.items() if not k.startswith("_")}}


def ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    cfg = gwgen.CONFIGS[args.config]
    seed = gwgen.BASE_SEED + cfg.index + 1000 * rank  # each rank: its own q-point
    prob = gwgen.config_problem(cfg, seed=seed)
    dev = torch.device("cuda", local)
    mtxel = args.mtxel or ("fp64" if args.prec == "fp64" else "twofloat")
    main = run_mode(args, cfg, prob, dev, args.prec, args.nslices, mtxel, args.steps, args.warmup,
                    not args.no_e2e, world)
    roofline = roofline_for(cfg, args.prec, args.nslices, main)
    # the dominant kernel of the step carries the "roofline" key; every kernel's is under "rooflines"
    rooflines = {roofline["kernel"]: roofline}
    if "zdft" in main["timing"]:
        rooflines.update(roofline_zd(cfg, prob, main))
    elif mtxel == "twofloat":
        rooflines["pair_mtxel"] = roofline_pair(cfg, prob, main)
    kernel_ms = {"ozaki_gemm": "ozaki_gemm", "contract_f64": "contract_f64", "zdft": "zdft",
                 "pair_from_f": "pair_from_f", "pair_mtxel": "pair_mtxel"}
    dom = max((k for k in rooflines if k in kernel_ms),
              key=lambda k: main["timing"].get(kernel_ms[k], (0.0, 0))[0])
    roofline = rooflines[dom]
    roofline_other = rooflines.get("ozaki_gemm") if dom != "ozaki_gemm" else None
    # In split precision the step runs each chunk's contraction on a second stream beside the
    # next chunk's pair elements, so the kernels above share the SMs; a short single-stream
    # pass gives each kernel's rate when it runs alone.
    alone = None
    if args.prec == "ozaki" and args.path == "stream" and mtxel == "twofloat" and main.get("streams", 1) == 2:
        a = run_mode(args, cfg, prob, dev, args.prec, args.nslices, mtxel, 2, 1, False, world, single_stream=True)
        alone = {"ms_per_step": a["ms_per_step"], "value": a["value"],
                 "pair": roofline_zd(cfg, prob, a) if "zdft" in a["timing"] else roofline_pair(cfg, prob, a),
                 "contraction": roofline_for(cfg, args.prec, args.nslices, a, single_stream=True)}
    # the CPU baseline leg (rank 0): the oracle timed on a bounded sample, and its reference block
    # for the error check
    err, blk = None, None
    if rank == 0 and not args.no_cpu_baseline and not args.no_check:
        blk = oracle_block(cfg, prob)
        err = block_error(main["chi"], blk)
    # the native FP64 tensor-core path on the same input, for the FP64-vs-split comparison
    other = None
    if args.prec == "ozaki" and not args.no_fp64_compare:
        f = run_mode(args, cfg, prob, dev, "fp64", 0, "fp64", max(1, min(2, args.steps)), 1, False, world)
        other = {"value": f["value"], "unit": "TFLOP/s", "ms_per_q": f["ms_per_step"], "mtxel": "fp64",
                 "roofline": roofline_for(cfg, "fp64", 0, f), "kernel_ms_per_step":
                     {k: v / max(1, min(2, args.steps)) for k, v in f["kernel_ms"].items()}}
        if blk is not None:
            other["error"] = block_error(f["chi"], blk)
        if err is not None:
            # the whole matrix against the library's FP64 mode (FP64 stage (a) and DMMA, no shared
            # arithmetic with the split path; itself within 1e-15 of the oracle's block)
            d = main["chi"] - f["chi"]
            err["rel_frobenius_full_vs_fp64_mode"] = float(np.linalg.norm(d) / np.linalg.norm(f["chi"]))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg, prob, args.cpu_sample_pairs)
        cpu.pop("seconds", None)
    if rank == 0:
        line = {"metric": METRIC, "value": main["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "ms_per_q": main["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.prec == "fp64" else "bf16-split/f64", "data": "synthetic",
                "config": {"workload": workload_name(cfg),
                           "prec": args.prec, "nslices": args.nslices if args.prec == "ozaki" else None,
                           "mtxel": mtxel, "path": args.path, "pairs": cfg.npairs,
                           "conv_tflop_per_step": conv_flops(cfg) * 1e-12,
                           "l2": "inputs larger than L2 (psi grids 2.0 GB, M chunks 262 MB)",
                           "parallelism": f"replicas x{world} (independent q-points)",
                           "streams": main.get("streams", 1)},
                "error": err, "roofline": roofline, "roofline_contraction": roofline_other, "rooflines": rooflines,
                "single_stream": alone, "fp64_dmma": other, "cpu_baseline": cpu, "e2e": main["e2e"],
                "gpu_launches": main["launches"], "kernel_ms": main["kernel_ms"], "clocks": main["clocks"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Pairs per chunk of the precision workload: chunks sized to 40 GB of M (N_G = 6000 complex128
# rows of 96 kB), a whole number of conduction rows: 204 x 2048 = 417792 pairs (40.1 GB).
C3_CHUNK_40GB = 204 * 2048


def sweep(args):
    """Slice-count sweep with the error against the oracle per slice count.  --config c3_72cube:
    the precision workload as configured (72^3, 256 + 2048 bands, N_G = 6000, pair chunks sized to
    40 GB of M, s = 4..7, one q-point per step); otherwise one 8192-pair chunk of it (s = 4..8 and
    native FP64)."""
    import dataclasses

    import torch
    import paper_2509_23018_gb300 as gw  # noqa: F401
    full = args.config == "c3_72cube"
    cfg = gwgen.CONFIGS["c3_72cube" if full else "p3_72cube_onechunk"]
    if full:
        cfg = dataclasses.replace(cfg, pair_chunk=C3_CHUNK_40GB)
    prob = gwgen.config_problem(cfg)
    dev = torch.device("cuda", 0)
    blk = oracle_block(cfg, prob)
    out = {"metric": METRIC, "mode": "slice-count sweep",
           "workload": f"{cfg.name}: grid 72^3, {cfg.nv}+{cfg.nc} bands, N_Gpsi={cfg.ngpsi}, N_G={cfg.ng}, "
                       f"pair chunks of {cfg.pair_chunk} pairs ({cfg.pair_chunk * cfg.ng * 16 / 1e9:.1f} GB of M)",
           "unit": "TFLOP/s (8 N_G^2 P convention) and ms per q-point", "slices": {}}
    steps, warm = (1, 1) if full else (2, 1)
    for s_ in ((4, 5, 6, 7) if full else (4, 5, 6, 7, 8)):
        r = run_mode(args, cfg, prob, dev, "ozaki", s_, "twofloat", steps, warm, False, 1)
        rf = roofline_for(cfg, "ozaki", s_, r)
        e = block_error(r["chi"], blk)
        out["sample"] = e.pop("sample")
        out["slices"][s_] = {"rel_err": e["rel_frobenius_vs_oracle"], "error": e, "ms_per_q": r["ms_per_step"], "value": r["value"], "gemm_tflops": rf["achieved"],
                             "gemm_frac": rf["frac"], "gemm_ms": rf["ms_per_launch"], "clocks": r["clocks"]}
        if s_ == 7:
            out["roofline"] = rf
            out["roofline_pair"] = roofline_pair(cfg, prob, r)
    if not full or args.sweep_fp64:
        r = run_mode(args, cfg, prob, dev, "fp64", 0, "fp64", 1, 1 if not full else 0, False, 1)
        e = block_error(r["chi"], blk)
        rf = roofline_for(cfg, "fp64", 0, r)
        out["fp64_dmma"] = {"rel_err": e["rel_frobenius_vs_oracle"],
                            "contract_tflops": rf["achieved"], "contract_ms": rf["ms_per_launch"],
                            "ms_per_q": r["ms_per_step"], "value": r["value"], "roofline": rf}
    if not args.no_cpu_baseline:
        # at N_G = 6000 the oracle takes about 47 ms a pair on 16 cores: 512 pairs stay near 25 s
        cpu = cpu_baseline(cfg, prob, min(args.cpu_sample_pairs, 512))
        cpu.pop("seconds", None)
        out["cpu_baseline"] = cpu
    print(json.dumps(out), flush=True)


def batch(args):
    """64 q-points (4x4x4 grid), N_G uniform in [300, 3000], 16 frequencies, one graph per call."""
    import torch
    import paper_2509_23018_gb300 as gw
    cfg = gwgen.CONFIGS["c4_batch"]
    b = gwgen.make_batch(cfg.grid, cfg.nv, cfg.nc, cfg.ngpsi, 300, 3000, 4, 16, seed=gwgen.BASE_SEED + cfg.index)
    dev = torch.device("cuda", 0)
    h = gw.Chi0(cfg.grid, nq=len(b.qs), prec="ozaki", nslices=args.nslices, mtxel="twofloat")
    g = torch.as_tensor(b.gpsi, device=dev)
    h.set_bands(0, 1, g, torch.as_tensor(b.cc, device=dev), torch.as_tensor(b.ec, device=dev))
    for iq in range(len(b.qs)):
        h.set_bands(iq, 0, g, torch.as_tensor(b.cv[iq], device=dev), torch.as_tensor(b.ev[iq], device=dev))
        h.set_gsphere(iq, torch.as_tensor(b.gchi[iq], device=dev))
    slots = list(range(len(b.qs)))
    ngs = [len(x) for x in b.gchi]
    out = torch.empty(sum(16 * n * n for n in ngs), dtype=torch.complex128, device=dev)
    t0 = time.perf_counter()
    h.compute_batch(slots, list(b.omega), out=out)  # tunes, captures, runs
    torch.cuda.synchronize()
    first = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.set_timing(True)
    h.timing(reset=True)
    e0.record()
    for _ in range(args.steps):
        h.compute_batch(slots, list(b.omega), out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    P = cfg.nv * cfg.nc
    conv = sum(8.0 * n * n * P * 16 for n in ngs)
    s = args.nslices
    # a graph replay has no per-kernel timing: the contraction's rate over the whole call (stage (a)
    # and the per-frequency slicing included) bounds it from below
    roof = mode_roofline("tensor", "oz_gemm_kernel (16 per-frequency launches over all q), whole replay",
                         sum(s * (s + 1) / 2 * 4.0 * n * n * P * 16 for n in ngs), ms,
                         "low-precision flops of the kept slice pairs over the whole replay time")
    cpu = None
    if not args.no_cpu_baseline:
        import types
        q0 = types.SimpleNamespace(gpsi=b.gpsi, cv=b.cv[0], ev=b.ev[0], cc=b.cc, ec=b.ec, gchi=b.gchi[0])
        tm, tw, how, cores = oracle_chi_sample(q0, 1024, list(b.omega[:2]))
        npair = (1024 // cfg.nc) * cfg.nc
        # M scales with pairs x N_G, chi with pairs x N_G^2: scale by the slots' sphere sizes
        n0 = len(b.gchi[0])
        est = sum((tm * n / n0 + tw * 16 * (n / n0) ** 2) * P / npair for n in ngs)
        cpu = {"value": 1e3 * est, "unit": "ms per call", "cores": cores, "kind": "oracle",
               "sample": f"q-point 0 (N_G = {n0}), {how}: M {tm:.1f} s, {tw:.1f} s per frequency, scaled by "
                         "pairs, frequencies and each slot's N_G (M ~ N_G, chi ~ N_G^2)"}
    print(json.dumps({"workload": "64 q (4^3 grid) x 16 imaginary frequencies (Gauss-Legendre on [0,100] eV), "
                                  "40^3, 64+512 bands, N_Gpsi=8000, N_G in [300,3000]",
                      "prec": "ozaki", "nslices": args.nslices, "ms_per_call": ms, "ms_per_q": ms / len(b.qs),
                      "conv_tflops": conv / (ms * 1e-3) * 1e-12, "first_call_s": first,
                      "tuning": h.tuning(), "timing_ms": {k: v[0] / args.steps for k, v in h.timing().items()},
                      "roofline": roof, "cpu_baseline": cpu}),
          flush=True)


def adjoint(args):
    """Adjoint of L = Re Tr(W chi0) on 40^3, 96+768 bands, N_G = 1500 (M recomputed per chunk)."""
    import torch
    import paper_2509_23018_gb300 as gw
    cfg = gwgen.CONFIGS["c5_adjoint"]
    prob = gwgen.config_problem(cfg)
    W = gwgen.hermitian(np.random.default_rng(gwgen.BASE_SEED + 4), cfg.ng)
    dev = torch.device("cuda", 0)
    h = gw.from_problem(prob, prec=args.prec, nslices=args.nslices, mtxel=args.mtxel or "twofloat")
    Wd = torch.as_tensor(W, device=dev)
    h.adjoint(0, Wd)
    torch.cuda.synchronize()
    h.set_timing(True)
    h.timing(reset=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L, dEv, dEc, dcv, dcc = h.adjoint(0, Wd)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / args.steps
    kms = {k: v[0] / args.steps for k, v in h.timing().items()}
    P, nr = cfg.nv * cfg.nc, cfg.grid[0] * cfg.grid[1] * cfg.grid[2]
    s = args.nslices
    roofs = {}
    if (args.mtxel or "twofloat") == "twofloat":
        roofs["back_projection"] = mode_roofline(
            "alu", "adj_pair_tf_kernel", backprojection_ops_per_pair(cfg, kept_columns(prob, cfg.grid[2])) * P,
            kms.get("adj_pair"), "FP32 operations of the two-float back-projection (bench.backprojection_ops_per_pair) x pairs")
        roofs["products"] = mode_roofline("hbm", "adj_cond_tf_kernel + adj_val_tf_kernel", 2 * 16.0 * P * nr,
                                          kms.get("adj_products"), "H read once by each product kernel, 16 B per point")
    if args.prec == "ozaki":
        roofs["y_mw"] = mode_roofline("tensor", "oz_gemm_kernel (general product Y = M W)",
                                      s * (s + 1) / 2 * 2.0 * P * (2 * cfg.ng) * oz_kpad(cfg.ng), kms.get("adj_zgemm"),
                                      "low-precision flops of the kept slice pairs")
    dom = max(roofs, key=lambda k: roofs[k]["ms"] if roofs[k] else 0.0) if roofs else None
    cpu = None if args.no_cpu_baseline else oracle_adjoint_sample(prob, W, 1)
    print(json.dumps({"workload": "L = Re Tr(W chi0), 40^3, 96+768 bands, N_Gpsi=4500, N_G=1500",
                      "prec": args.prec, "nslices": args.nslices, "s_per_adjoint": sec, "L": L,
                      "timing_ms": kms, "roofline": roofs.get(dom) if dom else None, "rooflines": roofs,
                      "cpu_baseline": cpu}), flush=True)


def subspace(args):
    """Static subspace on the 48^3 workload: chi(0) in the full basis (pair elements kept resident),
    the N_Eig = 20 % basis, then 19 imaginary frequencies in the subspace from the resident pair
    elements, against the same 19 in the full basis."""
    import torch
    import paper_2509_23018_gb300 as gw
    cfg = gwgen.CONFIGS["c2_48cube"]
    prob = gwgen.config_problem(cfg)
    neig = cfg.ng // 5
    om19 = [float(w) for w in gwgen.gl_freqs(19)]
    mtxel = args.mtxel or "twofloat"
    h = gw.from_problem(prob, prec=args.prec, nslices=args.nslices, mtxel=mtxel, pair_chunk=cfg.pair_chunk)
    # chi(0) keeps its pair elements resident (4.2 GB) and the subspace call reuses them
    h.keep_pair_elements(True)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    (chi0,), _ = timed(lambda: h.compute(0, [0.0]))  # warm-up (tuning, buffers)
    (chi0,), t0 = timed(lambda: h.compute(0, [0.0]))
    (C, lam), tb_first = timed(lambda: h.subspace_basis(chi0[0], neig))  # loads the solver
    (C, lam), tb = timed(lambda: h.subspace_basis(chi0[0], neig))
    _ = h.compute_subspace(0, C, om19)
    h.set_timing(True)
    h.timing(reset=True)
    sub, ts = timed(lambda: h.compute_subspace(0, C, om19))
    kms = {k: v[0] for k, v in h.timing(reset=True).items()}
    h.set_timing(False)
    sub0, _ = timed(lambda: h.compute_subspace(0, C, [0.0]))
    full, tf = timed(lambda: h.compute(0, om19)[0])
    h.sync()
    Cn = C.cpu().numpy()
    # identities at full size: chi_BB'(0) = diag(lambda); chi_BB'(w) = C^H chi(w) C
    d0 = float(np.linalg.norm(sub0[0].cpu().numpy() - np.diag(lam.cpu().numpy()))
               / np.linalg.norm(lam.cpu().numpy()))
    k = len(om19) // 2
    fk = full[k].cpu().numpy()
    proj = Cn.conj().T @ fk @ Cn
    dk = float(np.linalg.norm(sub[k].cpu().numpy() - proj) / np.linalg.norm(proj))
    approx = float(np.linalg.norm(Cn @ sub[k].cpu().numpy() @ Cn.conj().T - fk) / np.linalg.norm(fk))
    P = cfg.npairs
    s = args.nslices
    k2, k12 = kept_columns(prob, cfg.grid[2]), cells(prob, cfg.grid)
    roofs = {"pair_elements": mode_roofline("alu", "pair_kernel_tf_ct<48>", twofloat_ops_per_pair(cfg, k2, k12) * P,
                                            kms.get("pair_mtxel"), "FP32 operations of the pair kernel x pairs")}
    if args.prec == "ozaki":
        roofs["contraction"] = mode_roofline("tensor", "oz_gemm_kernel (N_Eig columns)",
                                             s * (s + 1) / 2 * 4.0 * neig ** 2 * P * len(om19),
                                             kms.get("ozaki_gemm"), "low-precision flops of the kept slice pairs")
        roofs["projection"] = mode_roofline("tensor", "oz_gemm_kernel (general product M C_s)",
                                            s * (s + 1) / 2 * 2.0 * P * (2 * neig) * oz_kpad(cfg.ng),
                                            kms.get("subspace_projection"), "low-precision flops of the kept slice pairs")
    cpu = None
    if not args.no_cpu_baseline:
        tm, tw, how, cores = oracle_chi_sample(prob, 1024, om19[:2], basis=Cn)
        npair = (1024 // cfg.nc) * cfg.nc
        cpu = {"value": 1e3 * (tm + tw * len(om19)) * P / npair, "unit": "ms for 19 frequencies in the subspace",
               "cores": cores, "kind": "oracle",
               "sample": f"{how}: M {tm:.1f} s, {tw:.1f} s per frequency, scaled by the pair count"}
    print(json.dumps({
        "roofline": max((r for r in roofs.values() if r), key=lambda r: r["ms"], default=None), "rooflines": roofs,
        "cpu_baseline": cpu,
        "workload": f"{cfg.name}: 48^3, {cfg.nv}+{cfg.nc} bands, N_G={cfg.ng}, N_Eig={neig} (20 %), "
                    "19 Gauss-Legendre imaginary frequencies on [0,100] eV",
        "prec": args.prec, "nslices": args.nslices, "mtxel": mtxel,
        "ms_chi0_full": t0, "ms_basis": tb, "ms_basis_first_call": tb_first, "ms_19_subspace": ts,
        "ms_19_full": tf, "kernel_ms_19_subspace": kms,
        "speedup_19": tf / ts, "subspace_19_over_chi0_full": ts / t0,
        "conv_tflops_19_subspace": 8.0 * neig * neig * P * 19 / (ts * 1e-3) * 1e-12,
        "rel_err_chi_sub0_vs_diag_lambda": d0, "rel_err_chi_sub_vs_projected_full": dk,
        "subspace_approximation_error": approx, "omega_checked": om19[k]}), flush=True)


def epsilon(args):
    """Inverse dielectric matrix [I - v chi(w)]^-1 on the 48^3 workload (N_G = 2000) for chi(0) and
    chi at two imaginary frequencies, v_G = 4 pi / |G|^2."""
    import torch
    import paper_2509_23018_gb300 as gw
    cfg = gwgen.CONFIGS["c2_48cube"]
    prob = gwgen.config_problem(cfg)
    om = [0.0, 5.0, 20.0]
    h = gw.from_problem(prob, prec=args.prec, nslices=args.nslices, mtxel=args.mtxel or "twofloat",
                        pair_chunk=cfg.pair_chunk)
    (chi,) = h.compute(0, om)
    v = torch.as_tensor(gwgen.coulomb(prob.gchi), device="cuda")
    h.epsilon_inverse(chi, v)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.set_timing(True)
    h.timing(reset=True)
    e0.record()
    einv = h.epsilon_inverse(chi, v)
    e1.record()
    torch.cuda.synchronize()
    tm = h.timing(reset=True)
    kms = {k: val[0] for k, val in tm.items()}
    h_launches = {k: val[1] for k, val in tm.items()}
    ms = e0.elapsed_time(e1)
    eye = torch.eye(cfg.ng, dtype=torch.complex128, device="cuda")
    res = [float(torch.linalg.norm((eye - v[:, None] * chi[i]) @ einv[i] - eye) / cfg.ng ** 0.5)
           for i in range(len(om))]
    steps = h_launches.get("eps_products", 0)
    s = args.nslices
    n = cfg.ng
    if args.prec == "ozaki":
        per_step = 2 * s * (s + 1) / 2 * 2.0 * n * (2 * n) * oz_kpad(n)
        roof = mode_roofline("tensor", "oz_gemm_kernel (general products of the Newton-Schulz steps)",
                             per_step * steps, kms.get("eps_products"), "low-precision flops of the kept slice pairs")
    else:
        roof = mode_roofline("tensor", "zgemm_kernel (DMMA)", 2 * 8.0 * n ** 3 * steps, kms.get("eps_products"),
                             "FP64 flops of the two complex products per step", prec="fp64")
    cpu = None
    if not args.no_cpu_baseline:
        dt, cores = oracle_epsilon_sample(chi[0].cpu().numpy(), v.cpu().numpy())
        cpu = {"value": 1e3 * dt, "unit": "ms per frequency block", "cores": cores, "kind": "oracle",
               "sample": f"one {n} x {n} block, dense inverse"}
    print(json.dumps({"workload": f"{cfg.name}: eps^-1 = [I - v chi(w)]^-1, N_G={cfg.ng}, w = {om} eV, "
                                  "v_G = 4 pi/|G|^2, chi from the 48^3 workload",
                      "prec": args.prec, "nslices": args.nslices, "ms_per_block": ms / len(om),
                      "newton_schulz_steps": steps, "kernel_ms": kms, "residual_rms": res, "roofline": roof,
                      "cpu_baseline": cpu}), flush=True)


def extras(args):
    """Real-axis chi (3 frequencies, eta = 0.1 eV) and the forward derivative (JVP, 1 frequency)
    on the 48^3 workload; times through CUDA events on the handle's stream."""
    import torch
    import paper_2509_23018_gb300 as gw
    cfg = gwgen.CONFIGS["c2_48cube"]
    prob = gwgen.config_problem(cfg)
    h = gw.from_problem(prob, prec=args.prec, nslices=args.nslices, mtxel=args.mtxel or "twofloat",
                        pair_chunk=cfg.pair_chunk)
    rng = np.random.default_rng(5)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    dcv = t((rng.standard_normal(prob.cv.shape) + 1j * rng.standard_normal(prob.cv.shape)) / np.sqrt(cfg.ngpsi))
    dcc = t((rng.standard_normal(prob.cc.shape) + 1j * rng.standard_normal(prob.cc.shape)) / np.sqrt(cfg.ngpsi))
    dev, dec = t(rng.standard_normal(cfg.nv)), t(rng.standard_normal(cfg.nc))

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    h.set_timing(True)
    h.timing(reset=True)
    real, tr = timed(lambda: h.compute_real(0, [2.0, 15.0, 40.0], 0.1))
    kr = h.timing(reset=True)  # warm-up call and timed call
    d, tj = timed(lambda: h.jvp(0, [0.0], dcv, dcc, dev, dec))
    h.set_timing(False)
    (chi,), tc = timed(lambda: h.compute(0, [0.0]))
    # the same calls reusing chi(0)'s resident pair elements
    h.keep_pair_elements(True)
    h.compute(0, [0.0])
    _, trr = timed(lambda: h.compute_real(0, [2.0, 15.0, 40.0], 0.1))
    _, tjr = timed(lambda: h.jvp(0, [0.0], dcv, dcc, dev, dec))
    h.keep_pair_elements(False)
    h.sync()
    ci = (real[1] - real[1].conj().T) / 2j
    s = args.nslices
    P = cfg.npairs
    nchunk = -(-P // cfg.pair_chunk)
    k2, k12 = kept_columns(prob, cfg.grid[2]), cells(prob, cfg.grid)
    half = lambda k: (kr[k][0] / 2, kr[k][1] // 2) if k in kr else (None, 0)
    gms, gl = half("ozaki_gemm")
    pms, _ = half("pair_mtxel")
    roofs = {"pair_elements": mode_roofline("alu", "pair_kernel_tf_ct<48>", twofloat_ops_per_pair(cfg, k2, k12) * P,
                                            pms, "FP32 operations of the pair kernel x pairs")}
    if args.prec == "ozaki":
        roofs["contraction"] = mode_roofline("tensor", "oz_gemm_kernel (sign-split real-axis contractions)",
                                             s * (s + 1) / 2 * 4.0 * cfg.ng ** 2 * P / nchunk * gl, gms,
                                             "low-precision flops of the kept slice pairs, per chunk contraction")
    cpu = None
    if not args.no_cpu_baseline:
        tm, tw, how, cores = oracle_chi_sample(prob, 1024, [15.0], eta=0.1)
        npair = (1024 // cfg.nc) * cfg.nc
        cpu = {"value": 1e3 * (tm / 3 + tw) * P / npair, "unit": "ms per real-axis frequency (three share M)",
               "cores": cores, "kind": "oracle",
               "sample": f"{how}: M {tm:.1f} s, {tw:.1f} s per frequency, scaled by the pair count"}
    print(json.dumps({"workload": f"{cfg.name}: 48^3, {cfg.nv}+{cfg.nc} bands, N_G={cfg.ng}",
                      "prec": args.prec, "nslices": args.nslices, "ms_chi_imag_axis_1w": tc,
                      "ms_chi_real_axis_per_w": tr / 3, "ms_jvp_1w": tj,
                      "ms_chi_real_axis_per_w_resident_m": trr / 3, "ms_jvp_1w_resident_m": tjr,
                      "kernel_ms_real_axis_3w": {k: v[0] / 2 for k, v in kr.items()},
                      "roofline": max((r for r in roofs.values() if r), key=lambda r: r["ms"], default=None),
                      "rooflines": roofs, "cpu_baseline": cpu,
                      "chi_I_max_eig_over_norm": float(torch.linalg.eigvalsh(ci).max() / torch.linalg.norm(ci)),
                      "jvp_hermitian": bool(torch.equal(d[0], d[0].conj().T))}), flush=True)


def sigma(args):
    """Off-diagonal plasmon-pole self-energy (section on the off-diagonal GPP kernel): N_Sigma = 512
    self-energy bands (the paper's Si998 full-matrix runs), N_G = 11,075 (the Si214 dielectric
    sphere of Table 2), per step 4 summed bands (2 occupied, 2 empty) x 16 energies of the grid.
    TFLOP/s counts the ZGEMM flops of the two products run per (n, E) over the whole kernel time
    including the prep. step; the line also carries the rate by Eq. flop_count_fullmat's count,
    which is twice that.  Inputs from the seeded plasmon-pole recipe."""
    import torch
    import paper_2509_23018_gb300 as gw
    ng, nsig, nb, nocc, ne = args.sigma_ng, args.sigma_nsig, 4, 2, args.sigma_ne
    p = gwgen.make_gpp(nb, nocc, nsig, ng, ne, seed=gwgen.BASE_SEED + 50)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    M, o2, wt, v = t(p.M), t(p.omega2), t(p.wtilde), t(p.vcoul)
    h = gw.Chi0((8, 8, 8), prec=args.prec, nslices=args.nslices)
    out = torch.empty((ne, nsig, nsig), dtype=torch.complex128, device="cuda")
    flops = gpp_products_flops(nb, ne, nsig, ng)
    steps, warm = max(1, min(args.steps, 3)), 1
    for _ in range(warm):
        h.sigma_gpp(M, p.En, nocc, o2, wt, v, p.E, out=out)
    torch.cuda.synchronize()
    clk = Clocks(torch.cuda.current_device())
    clk.start()
    h.set_timing(True)
    h.timing(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        h.sigma_gpp(M, p.En, nocc, o2, wt, v, p.E, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    kt = h.timing(reset=True)
    h.set_timing(False)
    clocks = clk.stop()
    kms = {k: val[0] / steps for k, val in kt.items()}
    s = args.nslices
    issued_x = s * (s + 1) / 2 * 8.0 * nsig * ng * ng * nb * ne      # slice pairs x real flops, first product
    pk, pk_src = peak_for("ozaki")
    roof = None
    if args.prec == "ozaki" and "gpp_gemm_x" in kms:
        ach = issued_x / (kms["gpp_gemm_x"] * 1e-3) * 1e-12
        roof = {"bound": "tensor", "kernel": "oz_gemm_kernel (X = conj(M_n) P)", "achieved": ach, "peak": pk,
                "unit": "TFLOP/s", "frac": ach / pk, "peak_source": pk_src}
    # error: one (n, E) against the oracle on 8 sampled rows l (P formed once on the host)
    n0, eidx = 0, min(5, ne - 1)
    one = h.sigma_gpp(M[n0:n0 + 1], p.En[n0:n0 + 1], 1 if n0 < nocc else 0, o2, wt, v, p.E[eidx:eidx + 1])
    got = one[0].cpu().numpy()
    h.sync()
    rows = np.random.default_rng(1).choice(nsig, 8, replace=False)
    err, cpu = None, None
    if not args.no_cpu_baseline:
        ref, cpu = oracle_sigma_rows(p, n0, eidx, rows)
        err = float(np.linalg.norm(got[rows] - ref) / np.linalg.norm(ref))
    print(json.dumps({
        "metric": "gpp_offdiag_tflops", "value": flops / (ms * 1e-3) * 1e-12,
        "unit": "TFLOP/s (ZGEMM flops of the products run, whole kernel time)", "ms_per_step": ms,
        "value_eq_flop_count_fullmat": gpp_offdiag_flops(nb, ne, nsig, ng) / (ms * 1e-3) * 1e-12,
        "workload": f"GPP off-diag. Sigma: N_Sigma={nsig}, N_G={ng}, {nb} summed bands ({nocc} occupied) x "
                    f"{ne} energies per step, plasmon-pole recipe (wp = 16.6 eV, eta = 0.25 eV)",
        "prec": args.prec, "nslices": s, "kernel_ms": kms, "roofline": roof, "clocks": clocks,
        "rel_err_sampled_rows_one_nE": err, "cpu_baseline": cpu}), flush=True)


def peaks(args):
    """Measure the pipe peaks of this GPU (the library's probes, cuBLAS bf16, cuBLASLt int8, a
    device copy) and write them to profiles/peaks_gb300.json; one JSON line on stdout."""
    import torch

    clk = Clocks(torch.cuda.current_device())
    clk.start()
    rates = probe_rates(PROBE_KINDS)
    lib = {}

    def best_of(fn, flops, reps=5):
        fn()
        torch.cuda.synchronize()
        b = 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            b = max(b, flops / (e0.elapsed_time(e1) * 1e-3) * 1e-12)
        return b

    n = 8192
    a = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)
    lib["bf16_cublas_tflops"] = best_of(lambda: a @ a, 2.0 * n ** 3)
    try:
        i8 = torch.randint(-8, 8, (n, n), device="cuda", dtype=torch.int8)
        lib["int8_cublaslt_tops"] = best_of(lambda: torch._int_mm(i8, i8), 2.0 * n ** 3)
    except Exception as e:  # noqa: BLE001
        lib["int8_cublaslt_tops"] = None
        lib["int8_error"] = str(e)[:200]
    del a
    x = torch.empty(1 << 30, dtype=torch.bfloat16, device="cuda")
    y = torch.empty_like(x)
    lib["hbm_copy_gbs"] = best_of(lambda: y.copy_(x), 4.0 * (1 << 30)) * 1e3  # 2 GiB read + 2 GiB written
    del x, y
    clocks = clk.stop()
    rec = {"what": "peak rates of this GPU's pipes (T operations/s, an FMA counts 2)",
           "command": "python bench.py --peaks", "gpu": torch.cuda.get_device_name(),
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "probes": rates, "library": lib, "clocks": clocks,
           "notes": {"ffma2": "fma.rn.f32x2: two FP32 lanes per instruction",
                     "dmma": "FP64 tensor rate; the FP64 contraction issues m8n8k4",
                     "bf16_mma_sync/int8_mma_sync": "warp-level (legacy) tensor instructions, not tcgen05"}}
    os.makedirs(os.path.dirname(PEAKS_JSON), exist_ok=True)
    with open(PEAKS_JSON, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if args.peaks:
        peaks(args)
        return
    measure_peaks()
    if args.sweep:
        sweep(args)
    elif args.batch:
        batch(args)
    elif args.subspace:
        subspace(args)
    elif args.epsilon:
        epsilon(args)
    elif args.extras:
        extras(args)
    elif args.sigma:
        sigma(args)
    elif args.adjoint:
        adjoint(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
