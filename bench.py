#!/usr/bin/env python
"""Benchmark of the GB300 pCMD forward model.

One step = one full likelihood evaluation of the plain full model (256x256 image, 2 bands,
7 SFH bins x 7 [Fe/H] x 300 masses, log10 Npix = 2, log-normal dust, 25x25 PSF, sky + photon
noise, 100x100 Hess, Eq. 2-4 likelihood) through the C ABI: host table build, draws, dust,
PSF, noise, magnitudes, Hess, likelihood; the likelihood value is read back every step.
Every step uses a new RNG set id (a new realisation of the model).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on the host cores on
a bounded pixel sample of the same workload.  Under torchrun every rank evaluates its own
models (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = ("plain full model: 256x256, 2 bands, 7 SFH x 7 [Fe/H] x 300 masses (14700 points), "
            "log10 Npix 2, log-normal dust F_dust 0.5, 25x25 Moffat PSF, sky + photon noise, "
            "100x100 Hess, Eq. 2-4 likelihood")
METRIC = "model pixels/s (plain full model, one likelihood evaluation per step)"
# Each step evaluates a new parameter point (a sampler-like random walk) with a new RNG set id.
PEAK_ISSUE_PER_SM_CLK = 128          # 4 schedulers x 32 lanes: thread-instructions per clock
# dram__bytes_read.sum + dram__bytes_write.sum of one draw launch on the headline workload
# (ncu, launch shape 256/4/128): the point tables are read once, the image stays in L2
DRAW_TRAFFIC_BYTES = 846848 + 0
OPS_PER_INV_DRAW = 3.5               # 1/16 Philox4x32-10 block (40 instr) + one byte compare
OPS_PER_PTRS_DRAW = 60.0             # 1/2 Philox block + ~40 FP32 ops of the squeeze test


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", type=int, default=1, help="also time the batched path")
    ap.add_argument("--launch", default="", help="block,split,chunk: skip the autotuner")
    ap.add_argument("--surrogate-sims", type=int, default=1 << 20,
                    help="simulations the surrogate is trained on in the extras")
    ap.add_argument("--only", default="", choices=["", "batched", "large", "surrogate", "mlp", "lmax", "psf_grid", "pool", "npix"],
                    help="run one extra section alone and print its JSON (profiling runs)")
    ap.add_argument("--large-n-im", type=int, default=1024, help="image edge of the large-Npix line")
    return ap.parse_args()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != self.idx:
                    continue
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ---------------------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline key)
# ---------------------------------------------------------------------------------------
def oracle_step(w, mock, set_id: int, n_threads: int) -> float:
    """One whole step of the workload through the oracle: the full forward model of the whole
    image (draws, dust, PSF, noise, magnitudes, Hess; OpenMP over pixels for the draws) and the
    Eq. 2-4 likelihood against the mock.  Returns seconds."""
    import oracle as O
    t0 = time.perf_counter()
    r = O.model(w, 0, set_id, n_threads=n_threads)
    O.loglike(r["hist"], r["moments"], r["n_pix"], mock["hist"], mock["moments"], mock["n_pix"])
    return time.perf_counter() - t0


def _oracle_mock(w, n_threads: int):
    import oracle as O
    small = W_full_crop(w, 32)
    return O.model(small, 0, 424_242, n_threads=n_threads)


def W_full_crop(w, n: int):
    import dataclasses
    return dataclasses.replace(w, n_im=n, n_ims=[n])


def cpu_baseline(w, steps: int = 3):
    """The oracle on the host cores: `steps` whole-image evaluations of the headline workload."""
    import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    mock = _oracle_mock(w, cores)
    t = [oracle_step(w, mock, 10 + k, cores) for k in range(steps)]
    npix = w.n_im * w.n_im
    v = steps * npix / sum(t)
    return {"value": v, "unit": "model pixels/s", "cores": cores, "kind": "oracle",
            "sample": "%d whole-image evaluations of the headline workload (%dx%d: draws with OpenMP "
                      "over pixels on %d threads, FP64 PSF, noise, magnitudes, Hess, Eq. 2-4), "
                      "%.2f s each" % (steps, w.n_im, w.n_im, cores, sum(t) / steps)}


def run_reference(args, world, rank):
    """The reference arm: the oracle, whole 256x256 evaluations of the headline workload per step
    (the warm-up steps run a 32x32 crop: the CPU path has nothing to warm)."""
    if rank != 0:
        return
    from paper_1904_00011_gb300 import workloads as W
    import oracle as O
    O.build()
    w = W.full()
    cores = os.cpu_count() or 1
    mock = _oracle_mock(w, cores)
    small = W_full_crop(w, 32)
    for i in range(args.warmup):
        oracle_step(small, mock, 100 + i, cores)
    t = [oracle_step(w, mock, 200 + i, cores) for i in range(args.steps)]
    total = sum(t)
    npix = w.n_im * w.n_im
    value = args.steps * npix / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "model pixels/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_im": 256, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "model pixels/s", "cores": cores, "kind": "oracle",
                             "sample": "each step one whole 256x256 evaluation (forward model and "
                                       "likelihood) on %d threads" % cores},
            "e2e": {"value": value, "unit": "model pixels/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# the GB300 arm
# ---------------------------------------------------------------------------------------
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12   # FMA lanes x 2 FLOP x max SM clock


def hess_roofline(hess_ms: float, n_bands: int, npix: int, psf: int, nbins: int,
                  psf_grid: bool = False) -> dict:
    """PSF / noise / magnitude / Hess kernel: 2 KS^2 FLOP per pixel and band (the stencil) against
    the FP32 FMA peak, and its algorithmic bytes (raw image read once, histogram flush) against
    the measured HBM copy bandwidth."""
    s = hess_ms / 1e3
    flop = 2.0 * psf * psf * n_bands * npix
    byts = 4.0 * n_bands * npix + 4.0 * nbins
    hbm = _measured_peak("hbm_gbs", 6800.0)
    # a single 25x25 PSF runs the band-split kernel, other sizes and PSF grids the tiled one
    name = ("hess_bs_kernel<%d>" % n_bands if psf == 25 and not psf_grid
            else "hess_kernel<%d,%d>" % (n_bands, psf))
    return {"kernel": name, "avg_launch_ms": hess_ms,
            "fp32": {"bound": "fp32", "achieved": flop / s / 1e12, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": flop / s / 1e12 / FP32_PEAK_TFLOPS,
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"},
            "hbm": {"bound": "hbm", "achieved": byts / s / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": byts / s / 1e9 / hbm, "bytes_per_launch": byts}}


def issue_roofline(instr: float, seconds: float, what: str) -> dict:
    peak = 152 * PEAK_ISSUE_PER_SM_CLK * 2070e6 / 1e12
    a = instr / seconds / 1e12
    return {"bound": "alu", "achieved": a, "peak": peak, "unit": "Tinstr/s", "frac": a / peak,
            "algorithmic": what, "peak_basis": "152 SMs x 128 issue slots/clk x 2070 MHz"}


INV_LIMIT = 640.0                    # inversion below this mean, transformed rejection at/above
DENSE_LAM = 0.08                     # slots from this mean on are drawn in dense groups


def algorithmic_ops(sim, params):
    lam, _, _ = sim.tables(params)
    inv = int(((lam > 0) & (lam < INV_LIMIT)).sum())
    ptrs = int((lam >= INV_LIMIT).sum())
    return inv * OPS_PER_INV_DRAW + ptrs * OPS_PER_PTRS_DRAW, inv, ptrs


def run_gb300(args, world, rank, local):
    import torch
    import paper_1904_00011_gb300 as P
    from paper_1904_00011_gb300 import build as B
    from paper_1904_00011_gb300 import workloads as W

    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    w = W.full()
    n = w.n_im
    npix = n * n
    sim = P.Simulator(w, max_sets=1)
    # the data: another realisation of the model (set ids far from the timed ones)
    sim.simulate(w.params, [n], 1_000_000 + rank)
    mh, mm, mc, _ = sim.hess(1, [n])
    torch.cuda.synchronize()
    mock_hess = mh[0].clone()
    mock_mom = mm[0].cpu().numpy().copy()
    mock_host = mock_hess.cpu().pin_memory()
    mode = W.LL_PAPER
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    base_id = rank * 10_000_000

    from paper_1904_00011_gb300 import autotune
    if args.launch:
        b_, s_, c_ = (int(v) for v in args.launch.split(","))
        sim.set_launch(b_, s_, c_)
        tuned = {"block": b_, "split": s_, "chunk": c_, "sweep": None}
    else:
        tuned = autotune.tune(sim, w.params, [n], use_cache=False)
    # a sampler-like sequence of parameter points: small seeded steps around the mock's values
    rng = np.random.default_rng(1234 + rank)
    p0 = w.params[0]

    def proposal():
        return [W.Params(log_sfh=p0.log_sfh + rng.normal(0, 0.05, size=p0.log_sfh.size),
                         feh_mean=p0.feh_mean + rng.normal(0, 0.02), feh_sigma=p0.feh_sigma,
                         log_ebv=p0.log_ebv + rng.normal(0, 0.02), dust_sigma=p0.dust_sigma,
                         dmod=p0.dmod + rng.normal(0, 0.02))]

    for i in range(args.warmup):
        sim.evaluate(proposal(), [n], mock_hess, mock_mom, npix, mode, first_set_id=base_id + i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                    if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local)
    clocks.start()
    sim.profile(True)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    lls = []
    props = [proposal() for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()                      # L2 flush between timed steps (outside the interval)
        ev0[i].record(stream)
        ll = sim.evaluate(props[i], [n], mock_hess, mock_mom, npix, mode,
                          first_set_id=base_id + args.warmup + i)
        ev1[i].record(stream)
        lls.append(float(ll[0]))
    torch.cuda.synchronize()
    kt = sim.kernel_times()
    sim.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = sum(step_ms)
    # end to end through the ABI from host buffers: mock Hess H2D from pinned memory each step
    e2e_ms = []
    for i in range(max(3, args.steps // 3)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mock_hess.copy_(mock_host, non_blocking=True)
        ll = sim.evaluate(proposal(), [n], mock_hess, mock_mom, npix, mode,
                          first_set_id=base_id + 5_000_000 + i)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([total_ms, sum(e2e_ms) / len(e2e_ms)], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms, e2e_step = float(t[0]), float(t[1])
    else:
        e2e_step = sum(e2e_ms) / len(e2e_ms)

    extras = {}
    if args.extras and rank == 0:
        extras["batched"] = run_batched(sim, P, W, torch)
        extras["large_npix"] = run_large(P, W, torch, n_im=args.large_n_im)
        extras["npix_range"] = run_npix_range(P, W, torch)
        extras["lmax"] = run_lmax(P, W, torch)
        extras["psf_grid"] = run_psf_grid(P, W, torch)
        extras["pool"] = run_pool(P, W, torch)
        extras["surrogate"] = run_surrogate(torch, n_sims=args.surrogate_sims)

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return
    value = world * args.steps * npix / (total_ms / 1e3)
    evals = world * args.steps / (total_ms / 1e3)
    draw_ms, draw_n = kt["draw"]
    ops, n_inv, n_ptrs = algorithmic_ops(sim, w.params[0])
    per_launch = ops * npix
    avg_draw_s = (draw_ms / max(draw_n, 1)) / 1e3
    peak = 152 * PEAK_ISSUE_PER_SM_CLK * 2070e6 / 1e12   # Tinstr/s at the maximum SM clock
    # (MEASURED_PEAKS.json holds copy bandwidth and cuBLAS BF16 only; the issue-slot peak is
    # derived from the SM count and the maximum clock)
    achieved = per_launch / avg_draw_s / 1e12
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w)
    launches_per_step = {k: c / args.steps for k, (ms, c) in kt.items() if c}
    line = {
        "metric": METRIC, "value": value, "unit": "model pixels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_im": n, "points": w.iso.n_points,
                   "draw_entries_per_pixel": n_inv + n_ptrs, "ptrs_entries_per_pixel": n_ptrs,
                   "l2": "flushed between timed steps (256 MB write outside the timed interval)",
                   "launch": {k: tuned[k] for k in ("block", "split", "chunk")},
                   "autotune_sweep_ms": tuned.get("sweep")},
        "loglike_evals_per_s": evals,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinstr/s",
                     "frac": achieved / peak, "traffic": DRAW_TRAFFIC_BYTES,
                     "traffic_unit": "bytes per launch (DRAM read + write, ncu capture of this kernel on this workload)",
                     "kernel": "draw_kernel<2,false,IMAGE,sparse>",
                     "avg_launch_ms": avg_draw_s * 1e3,
                     "algorithmic": "%g instr/pixel = %d inversion draws x %g + %d PTRS draws x %g"
                                    % (ops, n_inv, OPS_PER_INV_DRAW, n_ptrs, OPS_PER_PTRS_DRAW),
                     "peak_basis": "152 SMs x 128 issue slots/clk x 2070 MHz (issue-slot roofline)"},
        "secondary_rooflines": {"hess": hess_roofline(kt["hess"][0] / max(1, kt["hess"][1]), w.n_bands,
                                                      npix, 25 if w.psf is not None else 0,
                                                      w.hess_nx * w.hess_ny)},
        "kernel_ms_per_step": {k: ms / args.steps for k, (ms, c) in kt.items() if c},
        # the table builder's timer brackets its three kernels (count, scan, write)
        "gpu_launches": int(round(sum(c * (3 if k == "tables" else 1) for k, (ms, c) in kt.items()))),
        "launches_per_step": launches_per_step,
        "e2e": {"value": world * npix / (e2e_step / 1e3), "unit": "model pixels/s",
                "h2d_bytes_per_step": int(mock_hess.numel() * 4 + 168),
                "d2h_bytes_per_step": 8},
        "clocks": clk,
        "loglike_sample": lls[:3],
    }
    if cpu:
        line["cpu_baseline"] = cpu
    line.update(extras)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()


def run_batched(sim_plain, P, W, torch):
    """The batched path: 512 sampler live points with uneven images (128..512) and log10 Npix
    1..6 in one graph-replayed persistent launch, Poisson likelihood against a mock."""
    w = W.batch()
    sim = P.Simulator(w, max_sets=w.n_sets)
    mp = W.batch_mock_params()
    wm = W.with_params(w, [mp], [256])
    ms = P.Simulator(wm, max_sets=1, max_im=256)
    ms.simulate([mp], [256], 777_777)
    h, m, c, _ = ms.hess(1, [256])
    torch.cuda.synchronize()
    mock = h[0].clone()
    mom = m[0].cpu().numpy().copy()
    from paper_1904_00011_gb300 import autotune
    tuned = autotune.tune(sim, w.params, w.n_ims, fused=True, reps=1, use_cache=False,
                          candidates=[(256, 4, 64), (256, 2, 64), (256, 1, 64), (256, 8, 64),
                                      (128, 1, 64), (128, 2, 64)],
                          mock=(mock, mom, 256 * 256, W.LL_POISSON))
    for i in range(2):
        sim.evaluate(w.params, w.n_ims, mock, mom, 256 * 256, W.LL_POISSON, first_set_id=i * 1000)
    torch.cuda.synchronize()
    sim.profile(True)
    t = []
    reps = 5
    for i in range(reps):
        t0 = time.perf_counter()
        sim.evaluate(w.params, w.n_ims, mock, mom, 256 * 256, W.LL_POISSON, first_set_id=10_000 + i * 1000)
        t.append(time.perf_counter() - t0)
    kt = sim.kernel_times()
    sim.profile(False)
    step = statistics.median(t)
    # the same 512 sets (same set ids) through the plain per-model path: one pcmd_evaluate per set
    # on a one-set context (its graphs are cached per image size, as a sampler loop would see)
    one = P.Simulator(w, max_sets=1, max_im=max(w.n_ims))
    one.set_launch(tuned["block"], tuned["split"], tuned["chunk"])
    for k in range(8):
        one.evaluate([w.params[k]], [w.n_ims[k]], mock, mom, 256 * 256, W.LL_POISSON, first_set_id=10 + k)
    torch.cuda.synchronize()
    per_model = []
    ll_one = np.zeros(w.n_sets)
    for i in range(2):
        t0 = time.perf_counter()
        for k in range(w.n_sets):
            ll_one[k] = one.evaluate([w.params[k]], [w.n_ims[k]], mock, mom, 256 * 256, W.LL_POISSON,
                                     first_set_id=10_000 + i * 1000 + k)[0]
        per_model.append(time.perf_counter() - t0)
    one.close()
    ll_b = sim.evaluate(w.params, w.n_ims, mock, mom, 256 * 256, W.LL_POISSON, first_set_id=11_000)
    ll_rel = float(np.max(np.abs(ll_b - ll_one) / np.maximum(np.abs(ll_b), 1e-300)))
    per_model_s = min(per_model)
    pix = sum(n * n for n in w.n_ims)
    instr = 0.0
    for p_, n_ in zip(w.params, w.n_ims):
        ops, _, _ = algorithmic_ops(sim, p_)
        instr += ops * n_ * n_
    graph_ms = kt["graph"][0] / max(1, kt["graph"][1])
    return {"workload": "512 sets, images 128..512 (step 16), log10 Npix U[1,6], dmod U[22,26], "
                        "log E(B-V) U[-1,0], 200-point isochrone, Poisson likelihood",
            "evals_per_s": w.n_sets / step, "model_pixels_per_s": pix / step, "ms_per_batch": 1e3 * step,
            "graph_ms_per_batch": graph_ms,
            "vs_per_model": {"per_model_evals_per_s": w.n_sets / per_model_s,
                             "per_model_ms_for_512": 1e3 * per_model_s,
                             "batched_over_per_model": per_model_s / step,
                             "max_rel_likelihood_difference": ll_rel,
                             "how": "the same 512 sets and set ids, one pcmd_evaluate call per set on a "
                                    "one-set context (best of 2 passes)"},
            "launch": {k: tuned[k] for k in ("block", "split", "chunk")},
            "roofline": issue_roofline(instr, graph_ms / 1e3,
                                       "%.3g instr per batch: inversion draws x %g + PTRS draws x %g "
                                       "(draw, noise, magnitudes and histogram in one graph replay)"
                                       % (instr, OPS_PER_INV_DRAW, OPS_PER_PTRS_DRAW))}


LARGE_CANDIDATES = [(256, 1, 32), (256, 2, 32), (256, 4, 32), (256, 1, 64), (256, 2, 64), (256, 4, 64),
                    (128, 1, 32), (128, 2, 32)]


def run_line(P, W, torch, w, label: str, reps: int = 3, candidates=None, tune_reps: int = 1) -> dict:
    """One workload evaluated through pcmd_evaluate (the image + PSF path, or the fused graph
    without a PSF): launch shape tuned on the workload itself, `reps` timed evaluations with a new
    RNG set id each, the library's CUDA-event kernel times, the draw kernel's issue roofline
    (entries per pixel: inversion draws x OPS_PER_INV_DRAW + transformed-rejection draws x
    OPS_PER_PTRS_DRAW) and, with a PSF, the PSF / Hess kernel's rooflines."""
    n = w.n_im
    sim = P.Simulator(w, max_sets=1)
    from paper_1904_00011_gb300 import autotune
    tuned = autotune.tune(sim, w.params, [n], reps=tune_reps, use_cache=False, candidates=candidates)
    sim.simulate(w.params, [n], 2_000_000)
    h, m, c, _ = sim.hess(1, [n])
    torch.cuda.synchronize()
    mock, mom = h[0].clone(), m[0].cpu().numpy().copy()
    sim.evaluate(w.params, [n], mock, mom, n * n, W.LL_PAPER, first_set_id=1)
    torch.cuda.synchronize()
    sim.profile(True)
    t0 = time.perf_counter()
    for i in range(reps):
        sim.evaluate(w.params, [n], mock, mom, n * n, W.LL_PAPER, first_set_id=10 + i)
    dt = (time.perf_counter() - t0) / reps
    kt = sim.kernel_times()
    sim.profile(False)
    lam, _, _ = sim.tables(w.params[0])
    inv = int(((lam > 0) & (lam < INV_LIMIT)).sum())
    dense = int(((lam >= DENSE_LAM) & (lam < INV_LIMIT)).sum())
    ptrs = int((lam >= INV_LIMIT).sum())
    fused = w.psf is None
    draw_ms = (kt["graph"] if fused else kt["draw"])[0] / max(1, (kt["graph"] if fused else kt["draw"])[1])
    instr = (inv * OPS_PER_INV_DRAW + ptrs * OPS_PER_PTRS_DRAW) * n * n
    out = {"workload": label, "n_im": n, "log10_npix": round(math.log10(sum(10.0 ** np.asarray(w.params[0].log_sfh))), 3),
           "model_pixels_per_s": n * n / dt, "evals_per_s": 1.0 / dt, "ms_per_eval": 1e3 * dt,
           ("graph_ms" if fused else "draw_ms"): draw_ms,
           "kernel_ms": {k: v[0] / max(1, v[1]) for k, v in kt.items() if v[1]},
           "entries_per_pixel": inv + ptrs, "dense_entries_per_pixel": dense,
           "ptrs_entries_per_pixel": ptrs,
           "launch": {k: tuned[k] for k in ("block", "split", "chunk")},
           "draws_per_s": (inv + ptrs) * n * n / (draw_ms / 1e3),
           "roofline": issue_roofline(instr, draw_ms / 1e3,
                                      "%d inversion draws x %g + %d PTRS draws x %g per pixel%s"
                                      % (inv, OPS_PER_INV_DRAW, ptrs, OPS_PER_PTRS_DRAW,
                                         " (draw, noise, magnitudes, Hess in one graph)" if fused else ""))}
    if not fused:
        out["hess_ms"] = kt["hess"][0] / max(1, kt["hess"][1])
        out["hess_roofline"] = hess_roofline(out["hess_ms"], w.n_bands, n * n, w.psf.shape[-1],
                                             w.hess_nx * w.hess_ny)
    sim.close()
    return out


def run_large(P, W, torch, log_npix: float = 6.0, reps: int = 3, n_im: int = 1024):
    """Large-Npix regime: 1024x1024, 3 bands, 10 ages x 9 [Fe/H] x 400 masses, dense inversion
    groups dominant (transformed rejection from log10 Npix ~6), Kahan sums; full evaluation (PSF
    path) per step."""
    w = W.large(log_npix=log_npix, n_im=n_im)
    return run_line(P, W, torch, w, "%dx%d, 3 bands, 10 ages x 9 [Fe/H] x 400 masses, log10 Npix %.1f, "
                    "dust, 25x25 PSF, noise, Kahan sums" % (n_im, n_im, log_npix), reps=reps,
                    candidates=LARGE_CANDIDATES, tune_reps=2)


def run_npix_range(P, W, torch) -> dict:
    """The plain full model over its stated log10 Npix range (2 is the headline) and the
    large-Npix model over its range, each with its own roofline and draw-entry counts, and the
    tiny model."""
    out = {"full_256": [], "large_1024": []}
    for lg in (3.0, 4.0, 5.0):
        w = W.full(log_npix=lg)
        out["full_256"].append(run_line(P, W, torch, w, "plain full model 256x256, log10 Npix %.0f "
                                        "(distance modulus %.1f)" % (lg, w.params[0].dmod), reps=5))
    for lg in (5.0, 5.5, 6.5):
        out["large_1024"].append(run_large(P, W, torch, log_npix=lg))
    wt = W.tiny()
    out["tiny_64"] = run_line(P, W, torch, wt, "tiny model 64x64, one isochrone of 200 masses, Npix 100, "
                              "no dust / PSF / noise (fused graph)", reps=50, tune_reps=3)
    return out


# Inference batch of the surrogate lines: 96 rows per SM, i.e. three 128-row tiles per SM on the
# 1024-wide layers and whole waves of tiles on every layer (152 SMs).
INFER_BATCH = 152 * 96


def run_surrogate(torch, n_sims: int = 1 << 20, infer_batch: int = INFER_BATCH, reps: int = 10):
    """Surrogate: train on fresh simulations, report held-out accuracy against the exact
    simulator, inference throughput (tensor-core GEMMs) and the nested-sampling pre-screen gain."""
    from paper_1904_00011_gb300.surrogate import Surrogate
    from paper_1904_00011_gb300.sampler import nested_sampling
    S = Surrogate(batch=512, seed=0, infer_batch=infer_batch)
    info = S.train(n_sims=n_sims)
    d_mock, mom, npix = S.exact_mock(S.box.mean(axis=1).astype(np.float32))
    err = S.errors(n_test=512, seed=43, d_mock=d_mock, mock_moments=mom, mock_n_pix=npix)
    # inference: forward + likelihood of infer_batch parameter points
    th = S.sample_theta(infer_batch, np.random.default_rng(7)).astype(np.float32)
    th_d = torch.from_numpy(th).cuda()
    st = torch.cuda.current_stream()
    S.net.forward(th_d)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        S.net.forward(th_d)
    e1.record(st)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        S.loglike(th, d_mock, npix)
    ll_s = (time.perf_counter() - t0) / reps
    # the same with the parameters already on the device (fused forward + likelihood)
    scale = float(S.exact_n_im ** 2) / float(S.n_im ** 2)
    ratio = npix / float(S.exact_n_im ** 2)
    S.net.forward_loglike(th_d, d_mock.reshape(-1), scale, ratio)
    t0 = time.perf_counter()
    for _ in range(reps):
        S.net.forward_loglike(th_d, d_mock.reshape(-1), scale, ratio)
    fused_s = (time.perf_counter() - t0) / reps
    dims = S.net.dims
    flop = 2.0 * sum(dims[l] * dims[l + 1] for l in range(len(dims) - 1)) * infer_batch
    tflops = flop / (fwd_ms / 1e3) / 1e12
    peak = _measured_peak("bf16_tflops", 1900.0)
    scatter = S.scatter_calibration(d_mock, mom, npix, n_theta=32, n_rep=16)
    # pre-screen gain in short nested-sampling runs, several sampler seeds
    offset, margin = err["ll_offset"], 2.0 * err["ll_spread_p90"]
    exact = lambda t: S.exact_loglike(t, d_mock, mom, npix)  # noqa: E731
    sur = lambda t: S.loglike(t, d_mock, npix) + offset  # noqa: E731
    prior = lambda k, rng: S.sample_theta(k, rng).astype(np.float32)  # noqa: E731
    runs = []
    for seed in (3, 4, 5, 6, 7):
        plain = nested_sampling(exact, prior, n_live=32, n_iter=96, seed=seed)
        fast = nested_sampling(exact, prior, n_live=32, n_iter=96, seed=seed, surrogate_ll=sur,
                               margin=margin)
        runs.append((plain, fast))
    gains = [p_.exact_calls_per_replacement / max(1e-9, f_.exact_calls_per_replacement) for p_, f_ in runs]
    return {"workload": "12 parameters -> 100x100 log expected Hess counts (64x64 image, full "
                        "physics), MLP 64(12)-4x1024 GELU-10000, BF16 weights, FP32 accumulation",
            "train": info, "errors": err,
            "evals_per_s": infer_batch / ll_s, "evals_per_s_device_inputs": infer_batch / fused_s,
            "fused_ms_batch": 1e3 * fused_s, "forward_ms_batch": fwd_ms, "batch": infer_batch,
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "kernel": "gemm_bf16_kernel (5 layers)"},
            "scatter": scatter,
            "prescreen": {"seeds": [3, 4, 5, 6, 7],
                          "exact_calls_per_replacement_plain": [p_.exact_calls_per_replacement for p_, _ in runs],
                          "exact_calls_per_replacement_surrogate": [f_.exact_calls_per_replacement for _, f_ in runs],
                          "gain": gains, "gain_mean": float(np.mean(gains)),
                          "gain_sd": float(np.std(gains, ddof=1)),
                          "l_min_final_plain": [p_.l_min_final for p_, _ in runs],
                          "l_min_final_surrogate": [f_.l_min_final for _, f_ in runs],
                          "judge": "exact simulator, 256x256 images, Poisson likelihood"}}


def run_lmax(P, W, torch, reps: int = 100):
    """Appendix A workload: the best fit of the full model (here the mock's own parameters)
    recomputed `reps` times with distinct RNG set ids in one batched call; L_max = median."""
    from paper_1904_00011_gb300 import sampler as S
    w = W.full()
    n = w.n_im
    sim = P.Simulator(w, max_sets=reps)
    sim.simulate(w.params, [n], 3_000_000)
    h, m, _, _ = sim.hess(1, [n])
    torch.cuda.synchronize()
    mock, mom = h[0].clone(), m[0].cpu().numpy().copy()
    p = w.params[0]
    sim.evaluate([p] * reps, [n] * reps, mock, mom, n * n, W.LL_PAPER, first_set_id=10)
    torch.cuda.synchronize()
    sim.profile(True)
    t0 = time.perf_counter()
    ll = sim.evaluate([p] * reps, [n] * reps, mock, mom, n * n, W.LL_PAPER, first_set_id=1000)
    dt = time.perf_counter() - t0
    kt = sim.kernel_times()
    sim.profile(False)
    return {"workload": "full model 256x256, best fit recomputed %d times in one batched call "
                        "(Appendix A ceiling)" % reps,
            "ms": 1e3 * dt, "evals_per_s": reps / dt, "model_pixels_per_s": reps * n * n / dt,
            "kernel_ms": {k: v[0] for k, v in kt.items() if v[1]},
            "l_max": S.lmax_from_repeats(ll), "ll_std": float(np.std(ll)),
            "ll_min": float(np.min(ll)), "ll_max": float(np.max(ll))}


def run_psf_grid(P, W, torch, reps: int = 10):
    """The full model with the 4x4 grid of sub-pixel-shifted PSFs (Section 2.2): per-evaluation
    time and the PSF / Hess kernel's rooflines."""
    w = W.full(psf_grid=True)
    n = w.n_im
    sim = P.Simulator(w, max_sets=1)
    from paper_1904_00011_gb300 import autotune
    autotune.tune(sim, w.params, [n], reps=2, use_cache=False)
    sim.simulate(w.params, [n], 4_000_000)
    h, m, _, _ = sim.hess(1, [n])
    torch.cuda.synchronize()
    mock, mom = h[0].clone(), m[0].cpu().numpy().copy()
    sim.evaluate(w.params, [n], mock, mom, n * n, W.LL_PAPER, first_set_id=1)
    sim.profile(True)
    t0 = time.perf_counter()
    for i in range(reps):
        sim.evaluate(w.params, [n], mock, mom, n * n, W.LL_PAPER, first_set_id=10 + i)
    dt = (time.perf_counter() - t0) / reps
    kt = sim.kernel_times()
    sim.profile(False)
    hess_ms = kt["hess"][0] / max(1, kt["hess"][1])
    return {"workload": "full model 256x256 with a 4x4 grid of sub-pixel-shifted 25x25 Moffat PSFs",
            "ms_per_eval": 1e3 * dt, "model_pixels_per_s": n * n / dt, "hess_ms": hess_ms,
            "hess_roofline": hess_roofline(hess_ms, w.n_bands, n * n, 25, w.hess_nx * w.hess_ny, psf_grid=True)}


def run_pool(P, W, torch, reps: int = 20):
    """The full model (256x256, log10 Npix 2) with the total-count sampler for the points below
    the sampler boundary (lambda 640): per pixel and half one Poisson total and ~Npix / 2 star assignments instead of
    14 700 per-point draws; same law of the image, another RNG stream."""
    import dataclasses
    w0 = W.full()
    w = dataclasses.replace(w0, flags=w0.flags | W.FLAG_POOL)
    n = w.n_im
    sim = P.Simulator(w, max_sets=1)
    from paper_1904_00011_gb300 import autotune
    tuned = autotune.tune(sim, w.params, [n], reps=3, use_cache=False)
    sim.simulate(w.params, [n], 5_000_000)
    h, m, _, _ = sim.hess(1, [n])
    torch.cuda.synchronize()
    mock, mom = h[0].clone(), m[0].cpu().numpy().copy()
    for i in range(3):
        sim.evaluate(w.params, [n], mock, mom, n * n, W.LL_PAPER, first_set_id=1 + i)
    torch.cuda.synchronize()
    sim.profile(True)
    t0 = time.perf_counter()
    for i in range(reps):
        sim.evaluate(w.params, [n], mock, mom, n * n, W.LL_PAPER, first_set_id=10 + i)
    dt = (time.perf_counter() - t0) / reps
    kt = sim.kernel_times()
    sim.profile(False)
    return {"workload": "full model 256x256, log10 Npix 2, total-count sampler (PCMD_FLAG_POOL)",
            "ms_per_eval": 1e3 * dt, "model_pixels_per_s": n * n / dt,
            "kernel_ms": {k: v[0] / max(1, v[1]) for k, v in kt.items() if v[1]},
            "launch": {k: tuned[k] for k in ("block", "split", "chunk")}}


def run_mlp(torch, batch: int = INFER_BATCH, reps: int = 20):
    """Surrogate network alone (random init, no training): the 5-layer inference forward and the
    fused forward + likelihood on a batch of parameter points; GEMM roofline."""
    from paper_1904_00011_gb300.surrogate import Mlp
    dims = [64, 1024, 1024, 1024, 1024, 10000]
    net = Mlp(dims, 12, -np.ones(12), np.ones(12), max_batch=batch, seed=1)
    net.set_loss(True)
    rng = np.random.default_rng(0)
    th = torch.from_numpy(rng.uniform(-1, 1, size=(batch, 12)).astype(np.float32)).cuda()
    data = torch.from_numpy(rng.poisson(3.0, size=dims[-1]).astype(np.int32)).cuda()
    st = torch.cuda.current_stream()
    for _ in range(3):
        net.forward(th)
        net.forward_loglike(th, data, 16.0, 1.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        net.forward(th)
    e1.record(st)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        net.forward_loglike(th, data, 16.0, 1.0)
    fused_ms = 1e3 * (time.perf_counter() - t0) / reps
    flop = 2.0 * sum(dims[l] * dims[l + 1] for l in range(len(dims) - 1)) * batch
    tflops = flop / (fwd_ms / 1e3) / 1e12
    peak = _measured_peak("bf16_tflops", 1900.0)
    return {"workload": "MLP 64(12)-4x1024 GELU-10000, BF16, batch %d, random weights" % batch,
            "forward_ms": fwd_ms, "fused_loglike_ms": fused_ms, "evals_per_s": batch / (fused_ms / 1e3),
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "kernel": "gemm_bf16_kernel (5 layers)"}}


def _measured_peak(key: str, fallback: float) -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, ValueError, KeyError):
        return fallback


def main():
    args = _args()
    world, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.only:
        import torch
        import paper_1904_00011_gb300 as P
        from paper_1904_00011_gb300 import build as B
        from paper_1904_00011_gb300 import workloads as W
        B.build()
        torch.cuda.set_device(local)
        if args.only == "large":
            out = run_large(P, W, torch, n_im=args.large_n_im)
        elif args.only == "batched":
            out = run_batched(None, P, W, torch)
        elif args.only == "mlp":
            out = run_mlp(torch)
        elif args.only == "lmax":
            out = run_lmax(P, W, torch)
        elif args.only == "psf_grid":
            out = run_psf_grid(P, W, torch)
        elif args.only == "pool":
            out = run_pool(P, W, torch)
        elif args.only == "npix":
            out = run_npix_range(P, W, torch)
        else:
            out = run_surrogate(torch, n_sims=args.surrogate_sims)
        print(json.dumps({"section": args.only, **out}), flush=True)
        return
    run_gb300(args, world, rank, local)


if __name__ == "__main__":
    main()
