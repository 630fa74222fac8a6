#!/usr/bin/env python
"""PnP-FB imaging throughput on one GB300 (iterations per second), learned vs plain.

Workload (default): 4096^2 float32 image, 8192^2 complex64 grid, M = 2e7
synthetic MeerKAT-like visibilities in 64 radial data blocks, w folded into G
with J in {7, 9, 12, 16} by |w| quartile (complex64 weights, int32 columns),
40 dB input SNR.  A step is one full PnP-FB iteration (forward FFT with padding
and grid correction, fused de-gridding + residual + gridding pass, adjoint FFT
with the fused gradient step, denoiser, positivity and FP64 norms), replayed as
a captured CUDA graph.  The timed loop is the learned one: the problem divided
by the dirty-image peak bound alpha, the faceted residual CNN (4x4 uneven facets,
32 px halo, BF16 tensor-core convolutions) trained by the library's kernels at
the heuristic noise level.  The plain loop (one-level Haar soft threshold
tau/sqrt(2L) + positivity) is timed beside it, and its SNR after 200
iterations is the target of the learned loop's time-to-SNR.

``--gpus N`` under torchrun runs N independent replicas (the path does not
shard across GPUs here); ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "PnP-FB iter/s (4096² img, 2e7 vis), learned vs plain at equal SNR (dB)"
UNIT = "iter/s"
WORKLOADS = {
    "C3": dict(name="C3", desc="4096^2 img, 8192^2 grid, 2e7 vis in 64 blocks, Briggs r0, w-folded G J7-16 c64"),
    "C1": dict(name="C1", desc="2048^2 img, 4096^2 grid, 2e7 vis, w-folded G J7-16 c64"),
    "C0": dict(name="C0", desc="256^2 img, 512^2 grid, 2e5 vis, KB J7"),
    "C4": dict(name="C4", desc="8192^2 img, 16384^2 grid, 2.5e7 vis (one band), Briggs r0, w-folded G J7-9 bf16",
               facets="8x8"),
}
BLOCKS = {"C3": 64, "C1": 1, "C0": 1, "C4": 1}
CPU_SAMPLE_ROWS = 4000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="C3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-bf16-g", dest="bf16_g", action="store_false",
                    help="skip timing the plain loop with BF16 weights in G")
    ap.add_argument("--wstacks", type=int, default=8,
                    help="w-stacks of the stacked-operator comparison line (0 skips it)")
    ap.add_argument("--holo-rows", type=int, default=20_000_000,
                    help="rows of the 256^2 / 512^2 holographic comparison line (0 skips it)")
    ap.add_argument("--usara-prox-iters", type=int, default=10,
                    help="dual-FB iterations per uSARA denoise in its comparison line (0 skips it)")
    ap.add_argument("--usara-iters", type=int, default=300, help="uSARA iterations for its SNR trace")
    ap.add_argument("--usara-reweight-every", type=int, default=100,
                    help="FB iterations per weighted-l1 surrogate of uSARA (log-sum reweighting)")
    ap.add_argument("--converge-iters", type=int, default=2000,
                    help="iterations of the plain loop whose final SNR (minus 0.5 dB) is the time-to-SNR target")
    ap.add_argument("--no-l1", dest="l1", action="store_false",
                    help="skip the learned loop with the network trained without the penalty")
    ap.add_argument("--weights", default=None, help="network of the learned loop (default: the committed one)")
    ap.add_argument("--band-mhz", type=float, default=1053.0,
                    help="frequency band of the 8192^2 workload (C4): 1053 or 1399")
    ap.add_argument("--weights-l1", default=None, help="network of the learned_l1 comparison line")
    ap.add_argument("--train-batch", type=int, default=16,
                    help="batch of 256^2 images of the timed denoiser training steps (0 skips them)")
    ap.add_argument("--kernel-case", choices=["gridding", "cnn", "fft"], default=None,
                    help="run a small profiling case of one kernel (for ncu) instead of the benchmark")
    ap.add_argument("--cnn-side", type=int, default=4096,
                    help="image side of the cnn kernel case (4x4 facets scaled with it, 32 px halo)")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_aggregate(ms: float, steps: int, dist, ws: int, device: str = "cpu"):
    """(max over ranks of the timed milliseconds, whole-job iterations per second).

    Replicas run the same loop independently (the path is not sharded), so the
    job's throughput is ws * steps over the slowest rank's time."""
    if dist is not None and ws > 1:
        import torch
        tt = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    return ms, ws * steps / (ms / 1e3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([s.strip() for s in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 5 + i and s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def measured_bf16_peak():
    """Dense BF16 TFLOP/s for a kernel timed alone (burst), from the measured peaks file."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), "measured (burst)"
    return 1900.0, "fallback"


CNN_FLOP_PER_PX = 2 * 9 * 64 + 6 * 2 * 9 * 64 * 64 + 2 * 9 * 64   # 1->64, 6 x 64->64, 64->1 (3x3)


def _facet_pixels(n, facet_rows, facet_cols, halo):
    """Pixels the faceted denoiser processes: every facet extended by the halo, clipped at the border."""
    er = np.concatenate([[0], np.cumsum(facet_rows)])
    ec = np.concatenate([[0], np.cumsum(facet_cols)])
    px = 0
    for a0, a1 in zip(er[:-1], er[1:]):
        for b0, b1 in zip(ec[:-1], ec[1:]):
            px += (min(n, a1 + halo) - max(0, a0 - halo)) * (min(n, b1 + halo) - max(0, b0 - halo))
    return int(px)


def src_hash(*names):
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_2207_11336_gb300", "csrc", nm), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_file: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(f"{kernel_file}:{workload}")
    if not e or e.get("src_sha") != src_hash(kernel_file):
        return None
    return e.get("dram_bytes_per_launch")


# ---------------------------------------------------------------- CPU oracle sample
CNN_TILE = 96   # side of the image tile the FP64 oracle network is timed on


def oracle_sample(prob, rows, x, y_rows, gamma, t, cnn=None, row_scale=None):
    """Time one oracle PnP-FB iteration on a row sample of G; returns (s/iter estimate, parts).

    With ``cnn`` = (params, pixels) the denoiser is the FP64 oracle network, timed on a
    CNN_TILE^2 tile of the iterate and scaled to ``pixels`` (the facets with their halos);
    otherwise the Haar prox on the whole image."""
    from oracle import fb as ofb
    from oracle import nufft as onu
    n, K, M = prob["n"], prob["K"], prob["M"]
    gs = onu.GridSpec(n, K)
    G = onu.degridding_matrix(gs, prob["omega"], prob["w"], prob["dl"], prob["J_per_row"], rows, row_scale)
    GH = G.conj().T.tocsr()
    t0 = time.perf_counter()
    Xh = onu.dft2(onu.zero_pad(gs, x)).ravel()
    t1 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        r = G @ Xh - y_rows
        grid = GH @ r
    t2 = time.perf_counter()
    z = x - gamma * onu.zero_pad_adjoint(gs, onu.dft2_adjoint(grid.reshape(K, K))).real
    t3 = time.perf_counter()
    if cnn is None:
        ofb.haar_denoise(z, t)
        den = time.perf_counter() - t3
    else:
        from oracle import cnn as ocnn
        params, pixels = cnn
        ocnn.denoise(params, z[:CNN_TILE, :CNN_TILE], bf16=False)
        den = (time.perf_counter() - t3) * pixels / CNN_TILE ** 2
    g_full = (t2 - t1) / reps * (M / rows.size)
    est = (t1 - t0) + g_full + (t3 - t2) + den
    return est, dict(fft_and_pad_s=(t1 - t0) + (t3 - t2), g_pass_scaled_s=g_full,
                     g_sample_s=(t2 - t1) / reps, denoiser_s=den)


def cpu_sample_inputs(prob, x_dev_np, y_np):
    rng = np.random.default_rng(1234)
    rows = np.sort(rng.choice(prob["M"], CPU_SAMPLE_ROWS, replace=False))
    return rows, y_np[rows]


# ---------------------------------------------------------------- reference arm
def workload_desc(wl, learned):
    """The workload's description with the denoiser the timed loop applies (one string for both arms)."""
    return wl["desc"] + ((", CNN %s facets" % wl.get("facets", "4x4")) if learned else ", Haar")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    wl = dict(WORKLOADS[args.workload])
    if wl["name"] == "C4":
        prob = synth.make_problem("C4", freq_hz=args.band_mhz * 1e6)
        wl["desc"] = wl["desc"].replace("(one band)", "at %.0f MHz" % args.band_mhz)
    else:
        prob = synth.make_problem(wl["name"])
    from oracle import nufft as onu
    n, K, M = prob["n"], prob["K"], prob["M"]
    x = np.zeros((n, n))
    # the oracle's y on the sampled rows (noise-free sky model + scaled noise)
    rows, _ = cpu_sample_inputs(prob, None, np.zeros(M, complex))
    gs = onu.GridSpec(n, K)
    wimg = prob.get("imaging_weight")
    d = None if wimg is None else np.sqrt(wimg)
    Xt = onu.dft2(onu.zero_pad(gs, prob["x_true"])).ravel()
    G = onu.degridding_matrix(gs, prob["omega"], prob["w"], prob["dl"], prob["J_per_row"], rows, d)
    y_rows = G @ Xt + 1e-3 * prob["noise"][rows]
    gamma, t = 1.0 / M, 1e-6
    cnn, desc = None, workload_desc(wl, False)
    if os.path.exists(WEIGHTS) and "facet_rows" in prob:   # the same loop as the GPU arm times
        from paper_2207_11336_gb300.train_denoiser import load as load_weights
        params, _ = load_weights(WEIGHTS)
        cnn = (params, _facet_pixels(n, prob["facet_rows"], prob["facet_cols"], prob["halo"]))
        desc = workload_desc(wl, True)
    times = []
    for i in range(args.warmup + args.steps):
        est, _ = oracle_sample(prob, rows, x, y_rows, gamma, t, cnn, d)
        if i >= args.warmup:
            times.append(est)
    total = sum(times)
    val = len(times) / total
    sample = (f"per step: one FP64 oracle iteration with the full-size FFT pair (scipy.fft on {os.cpu_count()} "
              f"threads), G restricted to {CPU_SAMPLE_ROWS} seeded rows (scipy CSR, one thread; time scaled by "
              f"M/{CPU_SAMPLE_ROWS})"
              + (f" and the FP64 network on a {CNN_TILE}^2 tile (time scaled to the facets' pixels)" if cnn else ""))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc,
                                            "l2": "inputs larger than L2 (G %.1f GB)"
                                                  % ((prob["J_per_row"].astype(np.int64) ** 2).sum() * 10 / 1e9)},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
# the learned loop's network: trained on the l1 loss, then fine-tuned with the soft firm
# non-expansiveness penalty of Eq. training_loss (the convergence safeguard of App. C)
WEIGHTS = os.path.join(ROOT, "paper_2207_11336_gb300", "weights", "dncnn_C3_fne.npz")
# the same network before the penalised fine-tuning (l1 loss only), a comparison line
WEIGHTS_L1 = os.path.join(ROOT, "paper_2207_11336_gb300", "weights", "dncnn_C3.npz")
SNR_CHUNK = 10           # loops are run in chunks of this many iterations between SNR readings
TARGET_MARGIN_DB = 0.5   # time-to-SNR target: the plain loop's converged SNR minus this margin


def _snr_db(x_true, x):
    import torch
    xt = x_true.double()
    return float(20.0 * torch.log10(torch.linalg.vector_norm(xt) / torch.linalg.vector_norm(xt - x.double())))


def _timed_loop(plan, den, y, x, gamma, L, steps, stream, alpha=1.0):
    """ms for ``steps`` graph-replayed iterations (x updated in place), kernel launches inside."""
    import torch
    import paper_2207_11336_gb300 as pnp
    k0 = pnp.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    plan.fb_run(den, y, x0=x, gamma=gamma, L=L, max_iter=steps, check_every=steps, use_graph=True,
                inplace=True, alpha=alpha)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), pnp.kernel_launches() - k0


def _time_training(params, batch, stream, size=256, reps=10, fne_reps=3):
    """Milliseconds per denoiser training step on the GPU (App. C): the l1 step (forward, back-propagation,
    weight gradients, Adam) and the step with the soft firm non-expansiveness penalty of Eq. training_loss
    (20 power iterations on J_Q^T J_Q, lambda 10, the last fine-tuning stage's settings), on a batch of
    ``batch`` synthetic size^2 training images; CUDA events on the trainer's stream.  A separate trainer
    starting from the benchmark's network: its updates are discarded."""
    import torch
    import paper_2207_11336_gb300 as pnp
    import synth
    rng = np.random.default_rng(17)
    u = torch.from_numpy(np.stack([synth.training_image(size, rng) for _ in range(batch)]).astype(np.float32)).cuda()
    nz = torch.from_numpy(rng.standard_normal((batch, size, size)).astype(np.float32)).cuda()
    v0 = torch.from_numpy(rng.standard_normal((batch, size, size)).astype(np.float32)).cuda()
    sigma = 0.05
    tr = pnp.CnnTrainer(params, batch, size, lr=1e-6, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, k):
        fn()
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    ms_l1 = timed(lambda: tr.step(u, nz, sigma), reps)
    ms_fne = timed(lambda: tr.step_fne(u, nz, sigma, v0, 20, 10.0, 0.05), fne_reps)
    tr.close()
    flop = 3 * batch * size * size * CNN_FLOP_PER_PX   # forward, data gradients, weight gradients
    return {"batch": f"{batch} x {size}^2 synthetic training images", "l1_ms_per_step": ms_l1,
            "l1_images_per_s": batch / ms_l1 * 1e3, "l1_TFLOPs": flop / (ms_l1 * 1e-3) / 1e12,
            "fne_ms_per_step": ms_fne, "fne_power_iterations": 20}


def _run_to_snr(plan, den, y, gamma, L, x_true, alpha, target, max_iters):
    """Run the loop from x = 0 in chunks of SNR_CHUNK iterations until SNR >= target (or max_iters);
    returns (iterations to the target or None, [(iterations, SNR dB)], final iterate)."""
    import torch
    n = x_true.shape[0]
    x = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    trace, it = [], 0
    while it < max_iters:
        plan.fb_run(den, y, x0=x, gamma=gamma, L=L, max_iter=SNR_CHUNK, check_every=SNR_CHUNK,
                    use_graph=True, inplace=True, alpha=alpha)
        it += SNR_CHUNK
        snr = _snr_db(x_true, x)
        trace.append((it, snr))
        if target is not None and snr >= target:
            return it, trace, x
    return None, trace, x


def _first_at(trace, target):
    for it, snr in trace:
        if snr >= target:
            return it
    return None


def _thin(trace, every):
    return [(i, round(s, 3)) for i, s in trace if i % every == 0 or i == trace[-1][0]]


def run_gpu(args):
    global WEIGHTS, WEIGHTS_L1
    WEIGHTS = args.weights or WEIGHTS
    WEIGHTS_L1 = args.weights_l1 or WEIGHTS_L1
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2207_11336_gb300 as pnp
    from paper_2207_11336_gb300 import heuristics
    from paper_2207_11336_gb300.train_denoiser import load as load_weights
    import synth

    wl = dict(WORKLOADS[args.workload])
    wide = wl["name"] == "C4"   # the wide-field scale: one band of two, BF16 G, 8 x 8 facets
    if wide:
        prob = synth.make_problem("C4", freq_hz=args.band_mhz * 1e6)
        wl["desc"] = wl["desc"].replace("(one band)", "at %.0f MHz" % args.band_mhz)
        for k in ("bf16_g", "wstacks", "holo_rows", "usara_prox_iters"):   # comparison lines of the 4096^2 case
            setattr(args, k, 0)
    else:
        prob = synth.make_problem(wl["name"])
    n, K, M = prob["n"], prob["K"], prob["M"]
    stream = torch.cuda.current_stream()
    wimg = prob.get("imaging_weight")
    d = None if wimg is None else np.sqrt(wimg)   # Sec. 3: Briggs-weighted data, rows of G scaled by sqrt(w)
    plan = pnp.Plan(n, K, prob["omega"], prob["w"], prob["dl"], prob["J_per_row"], weight_dtype="bf16" if wide else "c64",
                    block=prob["block"], nblocks=BLOCKS[wl["name"]], stream=stream, row_scale=d)
    tune = plan.autotune(reps=2)   # run cap x unit size of the gridding pass, timed on this GPU
    info = plan.info
    x_true = torch.from_numpy(prob["x_true"].astype(np.float32)).cuda()
    y0 = plan.phi_forward(x_true)                       # weighted model data D Phi x
    y0_raw = y0 if d is None else y0 / torch.from_numpy(d.astype(np.float32)).cuda()
    norm_y0 = float(torch.linalg.vector_norm(y0_raw.to(torch.complex128)).item())
    tau = synth.noise_std_for_isnr(norm_y0, M, prob["isnr_db"])   # 40 dB input SNR of the raw data
    noise = plan.scale_data(torch.from_numpy(prob["noise"].astype(np.complex64)).cuda())
    y = (y0 + tau * noise).contiguous()
    tau_w = tau * (1.0 if wimg is None else float(np.sqrt(np.mean(wimg))))   # RMS of the weighted noise
    v0 = torch.from_numpy(synth.rng_for("power").standard_normal((n, n)).astype(np.float32)).cuda()
    hp = heuristics.imaging_parameters(plan, y, tau_w, v0)
    L, gamma, t = hp["L"], hp["gamma"], hp["noise_level"]
    haar = pnp.HaarDenoiser(t, stream=stream)

    learned = os.path.exists(WEIGHTS) and "facet_rows" in prob
    alpha = 1.0
    cnn_tune = None
    if learned:
        params, wmeta = load_weights(WEIGHTS)
        cnn = pnp.CnnDenoiser(params, n, facet_rows=prob["facet_rows"], facet_cols=prob["facet_cols"],
                              halo=prob["halo"], stream=stream)
        cnn_tune = cnn.autotune(x_true, reps=2)   # strip height of the convolution work lists, timed here
        # App. C, F: rescale by an upper bound on the peak that also matches the data's noise level to
        # the one the network was trained at (Eq. sigma); the library applies it (Eq. invpb2)
        alpha_match = heuristics.alpha_for_denoiser(tau_w, L, float(wmeta["sigma"]))
        alpha = max(hp["alpha"], alpha_match)
    den = cnn if learned else haar

    def barrier():
        if dist is not None:
            dist.barrier()

    steps = args.steps + (args.steps & 1)  # the graph replays iteration pairs
    # ---- timed region: the benchmark loop (learned if weights are present, else plain)
    x = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    plan.fb_run(den, y, x0=x, gamma=gamma, L=L, max_iter=max(args.warmup, 3), check_every=2,
                use_graph=True, inplace=True, alpha=alpha)
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(local) as clk:
        ms, launches = _timed_loop(plan, den, y, x, gamma, L, steps, stream, alpha)
    barrier()
    ms, value = replica_aggregate(ms, steps, dist, ws, "cuda")

    # ---- the plain loop: timed the same way, then run to convergence (a fixed budget) for the SNR target
    xp = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    plan.fb_run(haar, y, x0=xp, gamma=gamma, L=L, max_iter=4, check_every=2, use_graph=True, inplace=True)
    ms_plain, _ = _timed_loop(plan, haar, y, xp, gamma, L, steps, stream)
    _, trace_plain, xp = _run_to_snr(plan, haar, y, gamma, L, x_true, 1.0, None, args.converge_iters)
    snr_conv = trace_plain[-1][1]
    target = snr_conv - TARGET_MARGIN_DB
    it_plain = _first_at(trace_plain, target)
    plain = {"iter_per_s": ws * steps / (ms_plain / 1e3), "ms_per_iter": ms_plain / steps,
             "snr_db_converged": snr_conv, "converge_iters": args.converge_iters,
             "iters_to_target": it_plain, "time_to_target_s": it_plain * ms_plain / steps / 1e3,
             "snr_trace": _thin(trace_plain, 100)}
    comparison = {"snr_target_db": target,
                  "snr_target": "the plain loop's SNR after %d iterations minus %.1f dB"
                                % (args.converge_iters, TARGET_MARGIN_DB),
                  "plain": plain}
    if args.bf16_g:
        # mixed precision: the same operator with G stored as BF16 complex weights (FP32 accumulation)
        plan_bf = pnp.Plan(n, K, prob["omega"], prob["w"], prob["dl"], prob["J_per_row"], weight_dtype="bf16",
                           block=prob["block"], nblocks=BLOCKS[wl["name"]], stream=stream, row_scale=d)
        tune_bf = plan_bf.autotune(reps=2)
        y_bf = plan_bf.phi_forward(x_true)
        err = float(torch.linalg.vector_norm((y_bf - y0).to(torch.complex128)) /
                    torch.linalg.vector_norm(y0.to(torch.complex128)))
        xb = torch.zeros((n, n), dtype=torch.float32, device="cuda")
        plan_bf.fb_run(haar, y, x0=xb, gamma=gamma, L=L, max_iter=4, check_every=2, use_graph=True, inplace=True)
        ms_bf, _ = _timed_loop(plan_bf, haar, y, xb, gamma, L, steps, stream)
        comparison["plain_bf16_G"] = {"iter_per_s": ws * steps / (ms_bf / 1e3), "ms_per_iter": ms_bf / steps,
                                      "phi_rel_l2_vs_c64_G": err, "gridding_autotune": tune_bf,
                                      "G_bytes": plan_bf.info["nnz"] * 6}
        plan_bf.close()
        del plan_bf, y_bf, xb
    if args.wstacks > 1 and prob["dl"] > 0 and prob["J_per_row"] is not None:
        # the w-stacking hybrid (App. E): P stacks with the centre chirps in Z_p and the residual w in G
        supports = synth.CONFIGS[wl["name"]]["supports"]
        stk, cen = synth.w_stacks_min_taps(prob["w"], args.wstacks, supports)
        jr_s = synth.j_per_row_stacked(prob["w"], stk, cen, prob["w"], supports)
        t_plan = time.perf_counter()
        plan_ws = pnp.Plan(n, K, prob["omega"], prob["w"], prob["dl"], jr_s, block=prob["block"],
                           nblocks=BLOCKS[wl["name"]], stream=stream, stack=stk, w_centres=cen, row_scale=d)
        t_plan = time.perf_counter() - t_plan
        tune_ws = plan_ws.autotune(reps=2)
        y_ws = plan_ws.phi_forward(x_true)
        err = float(torch.linalg.vector_norm((y_ws - y0).to(torch.complex128)) /
                    torch.linalg.vector_norm(y0.to(torch.complex128)))
        xw = torch.zeros((n, n), dtype=torch.float32, device="cuda")
        plan_ws.fb_run(haar, y, x0=xw, gamma=gamma, L=L, max_iter=4, check_every=2, use_graph=True, inplace=True)
        ms_ws, _ = _timed_loop(plan_ws, haar, y, xw, gamma, L, steps, stream)
        plan_ws.set_timing(True)
        plan_ws.fb_run(haar, y, x0=xw, gamma=gamma, L=L, max_iter=5, check_every=5, use_graph=False, inplace=True)
        tw = plan_ws.read_timing()
        plan_ws.set_timing(False)
        comparison["plain_wstacked"] = {
            "stacks": args.wstacks, "w_centres": [round(float(v), 1) for v in cen],
            "iter_per_s": ws * steps / (ms_ws / 1e3), "ms_per_iter": ms_ws / steps,
            "nnz": plan_ws.info["nnz"], "G_bytes": plan_ws.info["nnz"] * 10,
            "G_bytes_unstacked": info["nnz"] * 10,
            "gridding_ms_per_iter": tw["gridding"][0] / 5, "fft_ms_per_iter": (tw["fft_forward"][0] + tw["fft_adjoint"][0]) / 5,
            "phi_rel_l2_vs_unstacked": err, "plan_build_s": t_plan, "gridding_autotune": tune_ws}
        plan_ws.close()
        del plan_ws, y_ws, xw
    if args.usara_prox_iters > 0:
        # uSARA (App. B) on the same operator: the SARA prox by dual FB, gamma lambda = rho = tau / sqrt(2L),
        # reweighted every usara_reweight_every iterations (the log-sum majoriser)
        try:
            sara = pnp.SaraDenoiser(n, t, t, args.usara_prox_iters, levels=4, stream=stream)
            xu = torch.zeros((n, n), dtype=torch.float32, device="cuda")
            plan.fb_run(sara, y, x0=xu, gamma=gamma, L=L, max_iter=4, check_every=2, use_graph=True, inplace=True)
            ms_u, _ = _timed_loop(plan, sara, y, xu, gamma, L, steps, stream)
            sara.close()
            sara = pnp.SaraDenoiser(n, t, t, args.usara_prox_iters, levels=4, stream=stream)
            xu.zero_()
            trace_u, it, rw = [], 0, args.usara_reweight_every
            while it < args.usara_iters:
                k = min(rw, args.usara_iters - it)
                # the library re-forms the weights after every rw iterations (Eq. B1's surrogates)
                plan.fb_run(sara, y, x0=xu, gamma=gamma, L=L, max_iter=k, check_every=k, use_graph=True,
                            inplace=True, reweight_every=rw)
                it += k
                trace_u.append((it, _snr_db(x_true, xu)))
            comparison["usara"] = {
                "prox_iters": args.usara_prox_iters, "reweight_every": rw,
                "iter_per_s": ws * steps / (ms_u / 1e3), "ms_per_iter": ms_u / steps,
                "iters_run": it, "snr_db_final": trace_u[-1][1], "iters_to_target": _first_at(trace_u, target),
                "snr_trace": _thin(trace_u, 100)}
            sara.close()
            del xu
        except Exception as e:  # a comparison line; the headline above stands without it
            comparison["usara"] = {"error": f"{type(e).__name__}: {e}"}
    if args.holo_rows > 0:
        # App. E, Eq. phidagphi: with many rows per grid cell the holographic H = G^H G is far smaller
        # than G; the 256^2 image / 512^2 grid layout with M rows (KB J = 7), plain loop with G vs with H
        ph = synth.make_problem("C0", M=args.holo_rows)
        nh, Kh = ph["n"], ph["K"]
        plan_h = pnp.Plan(nh, Kh, ph["omega"], stream=stream)
        xth = torch.from_numpy(ph["x_true"].astype(np.float32)).cuda()
        y0h = plan_h.phi_forward(xth)
        tauh = synth.noise_std_for_isnr(float(torch.linalg.vector_norm(y0h.to(torch.complex128)).item()),
                                        ph["M"], ph["isnr_db"])
        yh = (y0h + tauh * torch.from_numpy(ph["noise"].astype(np.complex64)).cuda()).contiguous()
        Lh, _ = plan_h.op_norm(None, 200, 1e-6)
        haar_h = pnp.HaarDenoiser(tauh / np.sqrt(2.0 * Lh), stream=stream)
        res_h = {}
        for mode in ("G", "H"):
            if mode == "H":
                t_b = time.perf_counter()
                plan_h.set_holographic(True)
                res_h["H_build_s"] = time.perf_counter() - t_b
            xh = torch.zeros((nh, nh), dtype=torch.float32, device="cuda")
            plan_h.fb_run(haar_h, yh, x0=xh, L=Lh, max_iter=4, check_every=2, use_graph=True, inplace=True)
            ms_h, _ = _timed_loop(plan_h, haar_h, yh, xh, 1.98 / Lh, Lh, steps, stream)
            res_h[mode] = {"iter_per_s": ws * steps / (ms_h / 1e3), "ms_per_iter": ms_h / steps}
            res_h["x_" + mode] = xh
        res_h["x_rel_diff_H_vs_G"] = float(torch.linalg.vector_norm((res_h.pop("x_H") - res_h["x_G"]).double()) /
                                           torch.linalg.vector_norm(res_h.pop("x_G").double()))
        comparison["plain_holographic"] = dict(
            workload="256^2 image, 512^2 grid, M=%.0e vis, KB J=7, Haar prox" % args.holo_rows,
            G_bytes=plan_h.info["nnz"] * 10, H_bytes=plan_h.info["holographic_bytes"], **res_h)
        plan_h.close()
        del plan_h, yh, y0h, xth
    xl = None
    if learned:
        it_l, trace_l, xl = _run_to_snr(plan, cnn, y, gamma, L, x_true, alpha, target, args.converge_iters)
        comparison["learned"] = {
            "weights": "l1 loss, then fine-tuned with the firm non-expansiveness penalty (last stage: lambda %g, "
                       "%d power iterations per step, %d steps)" % (
                float(wmeta.get("fne_lambda", 0.0)), int(wmeta.get("fne_iters", 0)), int(wmeta.get("steps", 0))),
            "iter_per_s": value, "ms_per_iter": ms / steps, "alpha": alpha, "alpha_dirty_peak": hp["alpha"],
            "alpha_matched_to_sigma": alpha_match, "sigma_trained": float(wmeta["sigma"]),
            "sigma_heuristic_at_dirty_peak": hp["sigma"], "iters_to_target": it_l,
            "time_to_target_s": None if it_l is None else it_l * ms / steps / 1e3,
            "snr_db_final": trace_l[-1][1], "iters_run": trace_l[-1][0],
            "snr_trace": _thin(trace_l, 100)}
        if os.path.exists(WEIGHTS_L1) and args.l1:
            # the learned loop with the network trained without the penalty (same cost per iteration)
            params_f, meta_f = load_weights(WEIGHTS_L1)
            cnn_f = pnp.CnnDenoiser(params_f, n, facet_rows=prob["facet_rows"], facet_cols=prob["facet_cols"],
                                    halo=prob["halo"], stream=stream)
            cnn_f.set_strip_rows(cnn_tune["strip_rows"])
            alpha_f = max(hp["alpha"], heuristics.alpha_for_denoiser(tau_w, L, float(meta_f["sigma"])))
            it_f, trace_f, _ = _run_to_snr(plan, cnn_f, y, gamma, L, x_true, alpha_f, target, args.converge_iters)
            comparison["learned_l1"] = {
                "weights": "l1 loss only, %d steps" % int(meta_f.get("steps", 0)), "alpha": alpha_f,
                "iters_to_target": it_f, "time_to_target_s": None if it_f is None else it_f * ms / steps / 1e3,
                "snr_db_final": trace_f[-1][1], "iters_run": trace_f[-1][0],
                "snr_trace": _thin(trace_f, 100)}
            cnn_f.close()
        if args.train_batch > 0:
            comparison["training"] = _time_training(params, args.train_batch, stream)

    # ---- kernel timing: eager replay with CUDA events around each operator stage
    plan.set_timing(True)
    kt = min(steps, 10)
    xk = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    plan.fb_run(haar, y, x0=xk, gamma=gamma, L=L, max_iter=kt, check_every=kt, use_graph=False, inplace=True)
    tim = plan.read_timing()
    # the same stages with the gridding flush's compensated summation switched off (the fast option)
    comp = bool(info["compensated"])
    plan.set_compensated(not comp)
    plan.fb_run(haar, y, x0=xk, gamma=gamma, L=L, max_iter=kt, check_every=kt, use_graph=False, inplace=True)
    tim_other = plan.read_timing()
    plan.set_compensated(comp)
    plan.set_timing(False)
    g_ms, g_cnt = tim["gridding"]
    g_ms_launch = g_ms / max(g_cnt, 1)
    # algorithmic bytes of one fused pass: G read once as complex64 weight + int32 column per tap, the
    # data y, and the grid read and written (12 B per tap, 8 B per row, 16 B per cell)
    wbytes = 4 if wide else 8   # BF16 or complex64 weight per tap
    alg_bytes = info["nnz"] * (wbytes + 4) + M * 8 + 2 * K * K * 8
    moved_bytes = info["nnz"] * (wbytes + 2) + M * 8 + 2 * K * K * 8   # what the pass stores: 16-bit cells
    hbm, peak_kind = measured_peaks()
    achieved = alg_bytes / (g_ms_launch * 1e-3) / 1e9
    roof_cnn = None
    if learned:
        zin = (x_true / alpha).contiguous()
        zout = torch.empty_like(zin)
        for _ in range(2):
            cnn.denoise(zin, zout)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            cnn.denoise(zin, zout)
        e1.record(stream)
        torch.cuda.synchronize()
        d_ms = e0.elapsed_time(e1) / 5
        px = _facet_pixels(n, prob["facet_rows"], prob["facet_cols"], prob["halo"])
        flop = px * CNN_FLOP_PER_PX
        bf16_peak, bf16_kind = measured_bf16_peak()
        roof_cnn = {"bound": "tensor", "kernel": "faceted CNN denoiser (cnn_first + 6 x conv64_rows + cnn_last)",
                    "achieved": flop / (d_ms * 1e-3) / 1e12, "peak": bf16_peak, "peak_kind": bf16_kind,
                    "unit": "TFLOP/s", "frac": flop / (d_ms * 1e-3) / 1e12 / bf16_peak, "traffic": None,
                    "flop_per_launch": flop, "ms_per_launch": d_ms}

    # ---- end to end through the public API with host buffers: every step copies its y in from pinned
    # host memory and its image out to pinned host memory.  The copies run on a second stream, double
    # buffered: step i + 1's y is uploaded while step i computes, and step i's image (a device snapshot
    # taken at the end of the step) is read back while step i + 1 computes; the timed region ends when
    # the last image has reached the host.
    y_host = y.cpu().pin_memory()
    x_host = torch.empty((n, n), dtype=torch.float32).pin_memory()
    y_dev = [torch.empty_like(y), torch.empty_like(y)]
    x_snap = torch.empty_like(x)
    copy_stream = torch.cuda.Stream()
    up = [torch.cuda.Event(), torch.cuda.Event()]
    snap_ready, snap_free = torch.cuda.Event(), torch.cuda.Event()
    torch.cuda.synchronize()
    e2e_steps = max(1, args.e2e_steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start = time.perf_counter()
    e0.record(stream)
    copy_stream.wait_event(e0)
    with torch.cuda.stream(copy_stream):
        y_dev[0].copy_(y_host, non_blocking=True)
        up[0].record(copy_stream)
        snap_free.record(copy_stream)
    for i in range(e2e_steps):
        if i + 1 < e2e_steps:
            copy_stream.wait_stream(stream)   # step i - 1, the last reader of this buffer, is complete
            with torch.cuda.stream(copy_stream):
                y_dev[(i + 1) % 2].copy_(y_host, non_blocking=True)
                up[(i + 1) % 2].record(copy_stream)
        stream.wait_event(up[i % 2])
        plan.fb_run(den, y_dev[i % 2], x0=x, gamma=gamma, L=L, max_iter=1, check_every=1, use_graph=False,
                    inplace=True, alpha=alpha)   # reads the FP64 norms back
        stream.wait_event(snap_free)             # the previous image has left x_snap
        x_snap.copy_(x, non_blocking=True)
        snap_ready.record(stream)
        copy_stream.wait_event(snap_ready)
        with torch.cuda.stream(copy_stream):
            x_host.copy_(x_snap, non_blocking=True)
            snap_free.record(copy_stream)
    stream.wait_stream(copy_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t_start)
    e2e_val = ws * e2e_steps / e2e_s

    out = None
    if rank == 0:
        desc = workload_desc(wl, learned)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps,
               "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16" if learned else "f32",
               "data": "synthetic", "impl": "gpu",
               "config": {"workload": desc, "parallelism": f"replicas{ws}",
                          "l2": "inputs larger than L2 (G %.1f GB)" % (info["nnz"] * (wbytes + 2) / 1e9),
                          "nnz": info["nnz"], "denoiser": "cnn" if learned else "haar", "graph": True,
                          "gridding_autotune": tune, "region_pitch": info["region_pitch"],
                          "cnn_autotune": cnn_tune},
               "clocks": clk.summary(),
               "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": M * 8,
                       "d2h_bytes_per_step": n * n * 4 + 16},
               "gpu_launches": launches,
               "roofline": {"bound": "hbm", "kernel": "gpass<G_FUSED> (degrid+residual+grid)",
                            "achieved": achieved, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                            "frac": achieved / hbm, "traffic": profiled_traffic("gridding.cu", wl["name"]),
                            "alg_bytes_per_launch": alg_bytes, "ms_per_launch": g_ms_launch,
                            "moved_bytes_per_launch": moved_bytes,
                            "frac_of_moved_bytes": moved_bytes / (g_ms_launch * 1e-3) / 1e9 / hbm,
                            "stage_ms_per_iter": {k: v[0] / max(v[1], 1) for k, v in tim.items()},
                            "compensated_gridding": comp,
                            ("stage_ms_per_iter_uncompensated" if comp else "stage_ms_per_iter_compensated"):
                                {k: v[0] / max(v[1], 1) for k, v in tim_other.items()}},
               "roofline_denoiser": roof_cnn,
               "comparison": comparison,
               "fb": {k: (float(v) if isinstance(v, (int, float, np.floating)) else v) for k, v in hp.items()}}
        out["fb"]["tau_raw"] = tau
        if ws == 1 and not args.no_cpu_baseline:
            rows, y_rows = cpu_sample_inputs(prob, None, y.cpu().numpy().astype(np.complex128))
            if learned:
                xs = xl.cpu().numpy().astype(np.float64) / alpha
                cnn_arg = (params, _facet_pixels(n, prob["facet_rows"], prob["facet_cols"], prob["halo"]))
                ys = y_rows / alpha
            else:
                xs, cnn_arg, ys = xp.cpu().numpy().astype(np.float64), None, y_rows
            est, parts = oracle_sample(prob, rows, xs, ys, gamma, t, cnn_arg, d)
            out["cpu_baseline"] = {"value": 1.0 / est, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                   "sample": f"one FP64 oracle iteration of the timed loop: full-size FFT pair "
                                             f"(scipy.fft on {os.cpu_count()} threads), G restricted to "
                                             f"{CPU_SAMPLE_ROWS} seeded rows (scipy CSR, one thread; time scaled by "
                                             f"M/{CPU_SAMPLE_ROWS})"
                                             + (f", the FP64 network on a {CNN_TILE}^2 tile (time scaled to the "
                                                f"facets' pixels)" if learned else ", Haar prox"),
                                   "parts_s": parts, "host_cores": os.cpu_count()}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_kernel_case(args):
    """Small case of the fused gridding pass for ncu: 1024^2 image, 2048^2 grid, M = 2e6
    (same row density per grid cell and J mix as the benchmark workload, G = 3.2 GB)."""
    import torch
    import paper_2207_11336_gb300 as pnp
    import synth
    n, K, M = 1024, 2048, 2_000_000
    prob = synth.make_problem("C1", M=M, n=n, K=K)
    plan = pnp.Plan(n, K, prob["omega"], prob["w"], prob["dl"], prob["J_per_row"])
    x = torch.from_numpy(prob["x_true"].astype(np.float32)).cuda()
    y = torch.from_numpy(prob["noise"].astype(np.complex64)).cuda()
    out = torch.empty_like(x)
    for _ in range(max(args.warmup, 1)):
        plan.grad_step(x, y, 1e-6, out)
    plan.set_timing(True)
    for _ in range(max(args.steps, 1)):
        plan.grad_step(x, y, 1e-6, out)
    t = plan.read_timing()
    info = plan.info
    ms = t["gridding"][0] / max(t["gridding"][1], 1)
    alg = info["nnz"] * 10 + M * 8 + 2 * K * K * 8
    print(json.dumps({"case": "gridding 1024^2/2048^2 M=2e6", "nnz": info["nnz"], "units": info["n_units"],
                      "gridding_ms": ms, "alg_bytes": alg, "GBps": alg / ms / 1e6,
                      "stage_ms": {k: v[0] / max(v[1], 1) for k, v in t.items()}}))
    return 0


def fft_case(args):
    """The FFT passes of the 4096^2 / 8192^2 operator with 2e5 visibilities of the benchmark's uv
    distribution (1.7 GB on the device): enough rows that the uv support the passes are pruned to is
    the benchmark's (the disc of the longest baselines)."""
    import torch
    import paper_2207_11336_gb300 as pnp
    import synth
    prob = synth.make_problem("C3", M=200_000)
    plan = pnp.Plan(prob["n"], prob["K"], prob["omega"], prob["w"], prob["dl"], prob["J_per_row"])
    x = torch.from_numpy(prob["x_true"].astype(np.float32)).cuda()
    y = torch.from_numpy(prob["noise"].astype(np.complex64)).cuda()
    out = torch.empty_like(x)
    for _ in range(max(args.warmup, 1)):
        plan.grad_step(x, y, 1e-10, out)
    plan.set_timing(True)
    for _ in range(max(args.steps, 1)):
        plan.grad_step(x, y, 1e-10, out)
    t = plan.read_timing()
    print(json.dumps({"case": "fft passes 4096^2 / 8192^2", "stage_ms": {k: v[0] / max(v[1], 1) for k, v in t.items()}}))
    return 0


def cnn_case(args):
    """The faceted CNN denoiser on the 4096^2 workload (or --cnn-side): 16 uneven facets, 32 px halo."""
    import torch
    import paper_2207_11336_gb300 as pnp
    import synth
    prob = synth.make_problem("C3", M=16, n=args.cnn_side, with_sky=True)
    n = prob["n"]
    params = synth.cnn_init(synth.rng_for("train"), 64, 8, 0.1)
    den = pnp.CnnDenoiser(params, n, facet_rows=prob["facet_rows"], facet_cols=prob["facet_cols"], halo=32)
    z = torch.from_numpy(prob["x_true"].astype(np.float32)).cuda()
    out = torch.empty_like(z)
    for _ in range(max(args.warmup, 1)):
        den.denoise(z, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed():
        torch.cuda.synchronize()
        e0.record()
        for _ in range(max(args.steps, 1)):
            den.denoise(z, out)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / max(args.steps, 1)

    ms = timed()
    by_rows = {}
    for rows in (16, 24, 32, 48, 64, 96):   # the strip heights the autotuner chooses among
        den.set_strip_rows(rows)
        den.denoise(z, out)
        by_rows[rows] = timed()
    den.set_strip_rows(32)
    px = _facet_pixels(n, prob["facet_rows"], prob["facet_cols"], 32)
    flop = px * CNN_FLOP_PER_PX
    print(json.dumps({"case": f"cnn {n}^2, 16 facets, halo 32", "ms": ms, "pixels_with_halo": int(px),
                      "TFLOP_per_call": flop / 1e12, "TFLOPs": flop / ms / 1e9, "ms_by_strip_rows": by_rows,
                      "status": den.device_status()}))
    return 0


def main():
    args = parse()
    if args.kernel_case == "cnn":
        return cnn_case(args)
    if args.kernel_case == "fft":
        return fft_case(args)
    if args.kernel_case:
        return run_kernel_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
