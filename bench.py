"""Benchmark of the ITA hot path on the 8192 x 8192 spaceborne workload.

One step = one iteration of Algorithm 1 (Eq. (25)) on an 8192 x 8192 complex64
scene: spaceborne C-band geometry, 2000 3x3 lognormal targets over -25 dB
clutter, echo = G(X), 40% Bernoulli sampling, K = 20000, fixed mu = 1, soft
threshold.  The echo, mask and iterate stay resident in HBM across the timed
iterations (each array is 512 MiB, larger than the 129 MB L2, so no flush is
needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun, one rank per GPU) solve
independent scenes (weak scaling, no collective on the data path).
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

import synth  # noqa: E402

N_AZ = N_RG = 8192
K_SPARSITY = 20000
RATE = 0.4
ITERS_PER_SOLVE = 100   # I of the workload (one user call of csar_solve_host)
METRIC = "ITA iterations/s at 8192x8192 c64 (spaceborne, K=20000, 40% sampling)"
UNIT = "iterations/s"
WORKLOAD = ("spaceborne C-band 8192x8192 complex64 ITA: 2000 3x3 lognormal(2,0.5) targets over "
            "-25 dB Rayleigh clutter, echo G(X), 40% Bernoulli sampling, K=20000, fixed mu=1, "
            "soft threshold")
# Algorithmic HBM bytes per element per pass (five passes forced by two separable
# 2-D operators, echo read compacted at 8 s B, mask 1/8 B, K-sparse iterate).  The
# residue's echo term is subtracted by the range pass of M, so its 8 s B sit there.
ALG_BYTES = {"C1_sparse_fft": 8.0, "R1_range_G": 16.0, "C2_residue": 8.0 + 0.125 + 8.0,
             "R2_range_M": 16.0 + 8.0 * RATE, "C3_select": 8.0}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def scene_seed(rank: int) -> int:
    """Each rank solves its own scene (weak scaling, no data exchange between ranks)."""
    return 1234 + rank


def max_over_ranks(value: float, pg=None, device="cpu") -> float:
    """Max of a per-rank float over the process group (the slowest rank's time)."""
    if pg is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps: int, ms: float, world: int) -> float:
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    return world * steps / (ms / 1e3)


def make_inputs(csar, plan, seed: int):
    """Scene X (numpy, seeded), echo G(X) on the GPU, Bernoulli mask."""
    import torch
    rng = np.random.default_rng(seed)
    x = synth.targets_over_clutter(rng, N_AZ, N_RG).astype(np.complex64)
    mask = synth.bernoulli_mask(rng, N_AZ, N_RG, RATE)
    bits = synth.pack_mask(mask)
    xd = torch.from_numpy(x).cuda()
    y = csar.csar_G(plan, xd)
    del xd
    md = torch.from_numpy(bits.view(np.int32)).cuda()
    torch.cuda.synchronize()
    return x, y, md, bits


def cpu_baseline_oracle(x_scene: np.ndarray, bits: np.ndarray, iters: int = 1, workers_list=(0,)):
    """The FP64 oracle on the host cores: `iters` ITA iterations of the same workload for
    each FFT worker count in workers_list (0: every core).  Returns [(seconds per
    iteration, workers)]."""
    from oracle import csa, ita
    g = synth.spaceborne(N_AZ, N_RG)
    mask = np.unpackbits(bits.view(np.uint8), bitorder="little").astype(bool).reshape(N_AZ, N_RG)
    y = csa.observe_G(g, x_scene.astype(np.complex128))
    y *= mask
    out = []
    saved = csa._WORKERS
    try:
        for w in workers_list:
            csa._WORKERS = w or (os.cpu_count() or 1)
            x = np.zeros((N_AZ, N_RG), np.complex128)
            t0 = time.perf_counter()
            for _ in range(iters):
                x, _ = ita.ita_iteration(g, y, mask, x, K_SPARSITY)
            out.append(((time.perf_counter() - t0) / iters, csa._WORKERS))
    finally:
        csa._WORKERS = saved
    return out


def cufft_comparison(csar, plan, y, md, steps: int):
    """The cuFFT-based comparison build (paper_1302_3120_gb300/compare/cufft_ita.cu: the
    same iteration in dense form with cuFFT C2C transforms, elementwise phase kernels and a
    three-round radix select), timed on the same GPU and inputs, plus its agreement with
    the library after 20 iterations.  Never part of the library's path."""
    import ctypes
    import torch
    path = os.path.join(ROOT, "paper_1302_3120_gb300", "libcsar_cufft.so")
    if not os.path.exists(path):
        return {"unavailable": "libcsar_cufft.so was not built"}
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.csar_cufft_create.argtypes = [ctypes.POINTER(csar.Params), ctypes.POINTER(vp)]
    lib.csar_cufft_solve.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, vp]
    lib.csar_cufft_destroy.argtypes = [vp]
    lib.csar_cufft_last_error.restype = ctypes.c_char_p
    p = csar.params_of(synth.spaceborne(N_AZ, N_RG))
    h = vp()
    if lib.csar_cufft_create(ctypes.byref(p), ctypes.byref(h)) != 0:
        return {"unavailable": lib.csar_cufft_last_error().decode()}
    stream = torch.cuda.current_stream()
    sp = vp(stream.cuda_stream)
    xc = torch.empty_like(y)

    def solve(iters):
        st = lib.csar_cufft_solve(h, vp(y.data_ptr()), vp(md.data_ptr()), vp(xc.data_ptr()),
                                  K_SPARSITY, iters, 1.0, sp)
        if st != 0:
            raise RuntimeError(lib.csar_cufft_last_error().decode())
    try:
        solve(3)
        ms = _event_ms(lambda: solve(steps), stream)
        solve(20)
        torch.cuda.synchronize()
        x_cmp = xc.cpu().numpy()
        x_lib = csar.csar_solve(plan, y, md, K_SPARSITY, 20).cpu().numpy()
    finally:
        lib.csar_cufft_destroy(h)
    d = np.linalg.norm(x_cmp - x_lib) / max(np.linalg.norm(x_lib), 1e-30)
    same = int(np.count_nonzero((x_cmp != 0) == (x_lib != 0)))
    return {"value": steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "rel_l2_vs_library_20_iters": float(d),
            "support_agreement_20_iters": same / x_lib.size,
            "what": "same inputs and GPU; dense ITA with cuFFT C2C (8 transforms), 6 phase, "
                    "residue, step+histogram, 2 histogram, 3 pick, threshold kernels per "
                    "iteration, captured in one CUDA graph"}


def run_reference(args, world, rank):
    """The oracle as the reference arm (CPU, rank 0 only)."""
    if rank != 0:
        return
    rng = np.random.default_rng(1234)
    x = synth.targets_over_clutter(rng, N_AZ, N_RG)
    mask = synth.bernoulli_mask(rng, N_AZ, N_RG, RATE)
    from oracle import csa, ita
    g = synth.spaceborne(N_AZ, N_RG)
    y = csa.observe_G(g, x) * mask
    del x
    xk = np.zeros((N_AZ, N_RG), np.complex128)
    for _ in range(min(args.warmup, 1)):
        xk, _ = ita.ita_iteration(g, y, mask, xk, K_SPARSITY)
    budget = 150.0
    done = 0
    t0 = time.perf_counter()
    while done < args.steps:
        xk, _ = ita.ita_iteration(g, y, mask, xk, K_SPARSITY)
        done += 1
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    value = done / dt
    cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": done, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * dt / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_az": N_AZ, "n_rg": N_RG,
                                           "K": K_SPARSITY, "sampling": RATE},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{done} full ITA iterations of the 8192x8192 workload "
                                       f"(numpy/scipy complex128, scipy.fft workers={cores}), "
                                       f"bounded to ~{int(budget)} s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _event_ms(fn, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_batched(args, world, rank, local):
    """64 airborne patches of uneven size (each axis from {512, 1024, 2048, 4096}), 1%
    Rayleigh scenes, 50% sampling, K_p = 1% of each patch: iterations/s of the batched
    solve (one graph launch per iteration) against the per-patch loop."""
    import torch
    torch.cuda.set_device(local)
    from paper_1302_3120_gb300 import build
    build.build()
    from paper_1302_3120_gb300 import csar
    rng = np.random.default_rng(2024 + rank)
    shapes = synth.batch_shapes(rng, 64)
    geoms = [synth.airborne(a, r) for a, r in shapes]
    Ys, Ms, Ks = [], [], []
    for g in geoms:
        plan = csar.csar_plan_create(g)
        x = synth.sparse_rayleigh(rng, g.n_az, g.n_rg, 0.01).astype(np.complex64)
        Ys.append(csar.csar_G(plan, torch.from_numpy(x).cuda()))
        Ms.append(torch.from_numpy(synth.pack_mask(synth.bernoulli_mask(rng, g.n_az, g.n_rg, 0.5))
                                   .view(np.int32)).cuda())
        Ks.append(int(round(0.01 * g.n_az * g.n_rg)))
        plan.close()
    for g in {(a, r) for a, r in shapes}:
        csar.csar_autotune(synth.airborne(*g), iters=3)
    batch = csar.csar_batch_create(geoms)
    plans = [csar.csar_plan_create(g) for g in geoms]
    Xs = [torch.empty_like(y) for y in Ys]
    stream = torch.cuda.current_stream()
    csar.csar_solve_batched(batch, Ys, Ms, Ks, max(args.warmup, 3), Xs=Xs)
    for i, p in enumerate(plans):
        csar.csar_solve(p, Ys[i], Ms[i], Ks[i], max(args.warmup, 3), X=Xs[i])
    steps = args.steps
    with ClockSampler(local) as clk:
        ms_b = _event_ms(lambda: csar.csar_solve_batched(batch, Ys, Ms, Ks, steps, Xs=Xs, stream=stream), stream)
    ms_l = _event_ms(lambda: [csar.csar_solve(p, Ys[i], Ms[i], Ks[i], steps, X=Xs[i], stream=stream)
                              for i, p in enumerate(plans)], stream)
    csar.csar_batch_check(batch)
    elems = sum(a * r for a, r in shapes)
    line = {"metric": "batched ITA iterations/s (64 uneven airborne patches)", "value": steps / (ms_b / 1e3),
            "unit": "iterations/s", "n_gpus": world, "steps": steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms_b / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64", "data": "synthetic",
            "config": {"workload": "64 patches, axes from {512,1024,2048,4096}, 1% Rayleigh, 50% mask, "
                                   "K_p = 1% of each patch, fixed mu = 1, soft", "elements": elems,
                       "shapes": shapes},
            "per_patch_loop": {"value": steps / (ms_l / 1e3), "ms_per_step": ms_l / steps},
            "speedup_vs_loop": ms_l / ms_b, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_autofocus(args, world, rank, local):
    """4096^2 airborne, 0.5% scene, 50% sampling, theta = 3 sinusoids, K = 83886:
    forward (50-iteration unroll with checkpoints) + loss + backward per step."""
    import torch
    torch.cuda.set_device(local)
    from paper_1302_3120_gb300 import build
    build.build()
    from paper_1302_3120_gb300 import csar
    na = nr = 4096
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(5 + rank)
    x = synth.sparse_rayleigh(rng, na, nr, 0.005).astype(np.complex64)
    th_true = synth.theta_sinusoids(rng, na)
    mask = synth.bernoulli_mask(rng, na, nr, 0.5)
    plan = csar.csar_plan_create(g)
    yg = csar.csar_G(plan, torch.from_numpy(x).cuda())
    Y = (yg * torch.from_numpy(np.exp(1j * th_true).astype(np.complex64)).cuda()[:, None]).contiguous()
    md = torch.from_numpy(synth.pack_mask(mask).view(np.int32)).cuda()
    theta = torch.from_numpy((th_true + 0.05 * synth.theta_sinusoids(rng, na, peak=1.0)).astype(np.float32)).cuda()
    K, iters = 83886, 50
    stream = torch.cuda.current_stream()

    def step():
        th = theta.clone().requires_grad_(True)
        L = csar.autofocus_loss(plan, Y, md, th, K, iters)
        L.backward()
        return L

    for _ in range(max(args.warmup, 3)):
        step()
    steps = max(1, min(args.steps, 20))
    fwd = _event_ms(lambda: csar.csar_af_solve(plan, Y, md, theta, K, iters), stream)
    tot = _event_ms(lambda: [step() for _ in range(steps)], stream) / steps
    line = {"metric": "autofocus forward+backward steps/s (4096^2, 50-iteration unroll)",
            "value": 1e3 / tot, "unit": "steps/s", "n_gpus": world, "steps": steps,
            "warmup": max(args.warmup, 3), "ms_per_step": tot, "forward_ms": fwd,
            "forward_iterations_per_s": iters / (fwd / 1e3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "airborne 4096x4096, 0.5% Rayleigh, 50% mask, theta = 3 sinusoids "
                                   "(peak 2 pi), K = 83886, 50 iterations, soft, mu = 1"}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_operators(args, world, rank, local):
    """Standalone operators on the 8192^2 spaceborne grid: one step = one G and one M
    application (chirp-scaling pair, or the range-Doppler pair with sinc RCMC)."""
    import torch
    torch.cuda.set_device(local)
    from paper_1302_3120_gb300 import build
    build.build()
    from paper_1302_3120_gb300 import csar
    g = synth.spaceborne(N_AZ, N_RG)
    rda = args.op == "rda"
    plan = csar.csar_plan_create(g, flags=csar.PLAN_RDA if rda else 0)
    rng = np.random.default_rng(7 + rank)
    x = torch.from_numpy(synth.targets_over_clutter(rng, N_AZ, N_RG).astype(np.complex64)).cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        csar.csar_G(plan, x, y, stream=stream)
        csar.csar_M(plan, y, x, stream=stream)
    steps = args.steps
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e[0].record(stream)
        for _ in range(steps):
            csar.csar_G(plan, x, y, stream=stream)
        e[1].record(stream)
        for _ in range(steps):
            csar.csar_M(plan, y, x, stream=stream)
        e[2].record(stream)
        torch.cuda.synchronize()
    ms_g, ms_m = e[0].elapsed_time(e[1]) / steps, e[1].elapsed_time(e[2]) / steps
    n = N_AZ * N_RG
    # algorithmic bytes per application: column, range and column pass each read and
    # write every element once (both pairs)
    alg = 48.0 * n
    peak, peak_kind = peaks()
    gbs = alg / ((ms_g + ms_m) / 2 * 1e-3) / 1e9
    line = {"metric": f"{'RDA' if rda else 'CSA'} operator applications/s (G and M, 8192x8192 c64)",
            "value": 2 * steps / ((ms_g + ms_m) * steps / 1e3), "unit": "applications/s",
            "n_gpus": world, "steps": steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms_g + ms_m, "G_ms": ms_g, "M_ms": ms_m, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "spaceborne 8192x8192, targets over clutter; one step = G then M",
                       "operator": "range-Doppler, 8-tap sinc RCMC" if rda else "chirp scaling"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": gbs / peak, "alg_bytes_per_application": alg},
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="spaceborne8192",
                    choices=["spaceborne8192", "batched", "autofocus", "operators"],
                    help="spaceborne8192 (default, the headline), the batched / autofocus rows, "
                         "or standalone G/M applications")
    ap.add_argument("--op", default="csa", choices=["csa", "rda"],
                    help="operator pair of --workload operators and of the ITA workload "
                         "(rda: CS-RDA; no CPU baseline)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison build")
    ap.add_argument("--cpu-iters", type=int, default=1)
    ap.add_argument("--size", type=int, default=8192,
                    help="profiling only: azimuth size of a smaller case of the same workload")
    ap.add_argument("--n-rg", type=int, default=0,
                    help="profiling only: range size of a smaller case (default: --size)")
    args = ap.parse_args()
    world, rank, local = dist_env()
    global N_AZ, N_RG, K_SPARSITY
    if args.size != 8192 or args.n_rg:
        N_AZ = args.size
        N_RG = args.n_rg or args.size
        K_SPARSITY = max(1, int(round(20000 * N_AZ * N_RG / 8192 ** 2)))

    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batched":
        run_batched(args, world, rank, local)
        return
    if args.workload == "autofocus":
        run_autofocus(args, world, rank, local)
        return
    if args.workload == "operators":
        run_operators(args, world, rank, local)
        return

    import torch
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_1302_3120_gb300 import build
    build.build()
    from paper_1302_3120_gb300 import csar

    g = synth.spaceborne(N_AZ, N_RG)
    rda = args.op == "rda"     # Algorithm 1 over the range-Doppler pair (CS-RDA)
    plan = csar.csar_plan_create(g, flags=csar.PLAN_RDA if rda else 0)
    x_scene, y, md, bits = make_inputs(csar, plan, seed=scene_seed(rank))
    X = torch.empty_like(y)

    # warm-up (captures the iteration graphs)
    csar.csar_solve(plan, y, md, K_SPARSITY, max(args.warmup, 3), X=X)
    torch.cuda.synchronize()

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        csar.csar_solve(plan, y, md, K_SPARSITY, args.steps, X=X, stream=stream)
        ev1.record(stream)
        barrier()
    clocks = clk.summary()
    ms = max_over_ranks(ev0.elapsed_time(ev1), pg, "cuda")
    csar.csar_plan_check(plan)
    value = job_rate(args.steps, ms, world)

    # per-pass device times (CUDA events on the launching stream, same workload)
    prof_iters = min(args.steps, 200)
    _, pass_ms = csar.csar_solve_profile(plan, y, md, K_SPARSITY, prof_iters, X=X, stream=stream)
    n = N_AZ * N_RG
    peak, peak_kind = peaks()
    passes = {}
    for name, tot in pass_ms.items():
        avg = tot / prof_iters
        entry = {"ms": avg}
        if name in ALG_BYTES:
            gbs = ALG_BYTES[name] * n / (avg * 1e-3) / 1e9
            entry.update({"alg_bytes": ALG_BYTES[name] * n, "gbs": gbs, "frac": gbs / peak})
        passes[name] = entry
    dominant = max((k for k in passes if k in ALG_BYTES), key=lambda k: passes[k]["ms"])
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath) and not rda:     # counters of the chirp-scaling passes
        try:
            traffic = json.load(open(tpath)).get(dominant)
        except Exception:
            traffic = None
    alg_iter = sum(ALG_BYTES.values()) * n
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": passes[dominant]["gbs"],
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": passes[dominant]["gbs"] / peak, "traffic": traffic,
                "iteration_alg_gbs": alg_iter * args.steps / (ms * 1e-3) / 1e9 / world,
                "iteration_frac": alg_iter * args.steps / (ms * 1e-3) / 1e9 / world / peak}

    # end to end through the host-buffer entry point, as the workload is run: solves of
    # I = 100 iterations from pinned host buffers (H2D of echo + mask, the iterations,
    # D2H of the image, all inside the timed region), repeated to cover `steps` iterations
    y_h = torch.empty(n, dtype=torch.complex64, pin_memory=True)
    y_h.copy_(y.reshape(-1))
    m_h = torch.from_numpy(bits.view(np.int32)).pin_memory()
    x_h = torch.empty(n, dtype=torch.complex64, pin_memory=True)
    y_np, m_np, x_np = y_h.numpy(), m_h.numpy().view(np.uint32), x_h.numpy()
    per_call = min(ITERS_PER_SOLVE, args.steps)
    calls = max(1, args.steps // per_call)
    barrier()
    t0 = time.perf_counter()
    for _ in range(calls):
        csar.csar_solve_host(plan, y_np, m_np, K_SPARSITY, per_call, X=x_np, stream=stream)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, pg, "cuda")
    e2e = {"value": job_rate(calls * per_call, e2e_s * 1e3, world), "unit": UNIT,
           "h2d_bytes_per_step": (y_np.nbytes + m_np.nbytes) / per_call,
           "d2h_bytes_per_step": x_np.nbytes / per_call,
           "note": f"{calls} csar_solve_host calls of {per_call} iterations each (echo and "
                   "mask copied in, image copied out once per call)"}

    cmp = None
    if rank == 0 and world == 1 and not rda and not args.no_cufft:
        cmp = cufft_comparison(csar, plan, y, md, min(args.steps, 200))

    cpu = cpu1 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not rda:
        del y, X
        torch.cuda.empty_cache()
        res = cpu_baseline_oracle(x_scene, bits, args.cpu_iters, (0, 1))
        (dt, cores), (dt1, _) = res
        cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_iters} ITA iteration(s) of the same 8192x8192 workload from "
                         f"X=0 (numpy/scipy complex128, scipy.fft workers={cores}, elementwise "
                         "numpy on one thread); echo built by the oracle's own G"}
        cpu1 = {"value": 1.0 / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"the same {args.cpu_iters} iteration(s) with scipy.fft workers=1"}

    # kernels of one fixed-step iteration (direct sparse DFT, sparse-FFT path, R1, C2, R2,
    # C3, check, 3 x (round, pick), count, scan, scatter, finish; the re-passes are
    # conditional graph nodes that launch only when the predicted cut was too high) and
    # of the per-solve set-up / output (mask transpose, masked echo, its azimuth FFT,
    # control init, list->dense)
    kernels_per_iter, kernels_per_solve = 17, 5
    line = {"metric": METRIC.replace("ITA", "CS-RDA ITA") if rda else METRIC, "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_az": N_AZ, "n_rg": N_RG, "K": K_SPARSITY,
                       "sampling": RATE, "mu": "fixed 1.0", "threshold": "soft",
                       "operator": "range-Doppler, 8-tap sinc RCMC" if rda else "chirp scaling",
                       "l2": "no flush: every array (512 MiB) exceeds the 129 MB L2",
                       "parallelism": f"independent scenes x{world}"},
            "roofline": roofline, "passes": passes, "clocks": clocks, "e2e": e2e,
            "gpu_launches": kernels_per_iter * args.steps + kernels_per_solve, "cpu_baseline": cpu,
            "cpu_baseline_1core": cpu1, "cufft_comparison": cmp}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
