"""Train the residual CNN denoiser of the learned loop on the GPU (App. C).

The training noise level follows the heuristic sigma = tau / (alpha sqrt(2L))
(Eq. sigma) of the imaging problem the denoiser is meant for: the workload's
operator and noisy data are built on the GPU and L, beta and alpha come from
``heuristics.imaging_parameters``.  The training images are seeded synthetic
peak-normalised skies (points and Gaussian blobs with log-uniform intensities
down to 1e-5, ``synth.training_image``), standing in for the paper's training
database, with random dihedral transforms.  Each step draws z = u + sigma n with
n from ``torch.randn`` (passed in as an input) and takes one Adam step on the
l1 loss through the library's own forward and backward kernels
(``CnnTrainer``); the step size follows a cosine decay.

Noise units.  The heuristic sigma can sit far below the image peak (a dynamic
range of ~1e6 for the 4096^2 workload), below what BF16 hidden activations
resolve next to biases of the size Adam's steps give them.  The network is
therefore trained on u / s at noise level sigma / s with s = 2^round(log2 sigma),
i.e. in units of the noise, and s is folded back into the first and last layers
(W1 / s, s W8, s b8), so the saved network acts on images at their own scale:
z - s N(z / s).  With s a power of two the folding is exact in binary floating
point, including the BF16 rounding of the weights, so inference and the oracle
use the folded weights unchanged.

    python -m paper_2207_11336_gb300.train_denoiser --workload C3 \\
        --out paper_2207_11336_gb300/weights/dncnn_C3.npz
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _pool_chunk(args):
    size, count, seed = args
    import synth
    rng = np.random.default_rng(seed)
    return np.stack([synth.training_image(size, rng) for _ in range(count)]).astype(np.float32)


def image_pool(count: int, size: int, seed: int = 0, workers: int | None = None) -> np.ndarray:
    """count seeded training images (float32, count x size x size), built in a spawn pool."""
    chunk = 250
    seeds = np.random.SeedSequence([seed, 0x7A11]).spawn((count + chunk - 1) // chunk)
    jobs = [(size, min(chunk, count - i * chunk), s) for i, s in enumerate(seeds)]
    workers = workers or max(1, min(len(jobs), (os.cpu_count() or 2)))
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_pool_chunk, jobs)
    return np.concatenate(parts)


def noisy_problem(name: str, stream=None):
    """(problem dict, plan, x_true, y, tau) for a benchmark workload: y = D (Phi x_true + tau_raw n) with
    the workload's data weights D (Sec. 3: Briggs; none for natural weighting), the raw noise level set
    by the input SNR, and tau the RMS of the weighted noise D tau_raw n."""
    import torch
    import synth
    import paper_2207_11336_gb300 as pnp
    prob = synth.make_problem(name)
    nblocks = int(prob["block"].max()) + 1
    wimg = prob.get("imaging_weight")
    d = None if wimg is None else np.sqrt(wimg)
    plan = pnp.Plan(prob["n"], prob["K"], prob["omega"], prob["w"], prob["dl"], prob["J_per_row"],
                    block=prob["block"], nblocks=nblocks, stream=stream, row_scale=d)
    x_true = torch.from_numpy(prob["x_true"].astype(np.float32)).cuda()
    y0 = plan.phi_forward(x_true)
    y0_raw = y0 if d is None else y0 / torch.from_numpy(d.astype(np.float32)).cuda()
    norm_y0 = float(torch.linalg.vector_norm(y0_raw.to(torch.complex128)).item())
    tau = synth.noise_std_for_isnr(norm_y0, prob["M"], prob["isnr_db"])
    y = (y0 + tau * plan.scale_data(torch.from_numpy(prob["noise"].astype(np.complex64)).cuda())).contiguous()
    tau_w = tau * (1.0 if wimg is None else float(np.sqrt(np.mean(wimg))))
    return prob, plan, x_true, y, tau_w


def noise_unit(sigma: float) -> float:
    """s = 2^round(log2 sigma): the power of two nearest the training noise level."""
    return float(2.0 ** np.round(np.log2(sigma)))


def fold_scale(params, s: float):
    """Weights of z -> s N(z / s) for the network N given by params (exact for s a power of two)."""
    out = [(np.array(W, dtype=np.float64), np.array(b, dtype=np.float64)) for W, b in params]
    out[0] = (out[0][0] / s, out[0][1])
    out[-1] = (out[-1][0] * s, out[-1][1] * s)
    return out


def train(pool, sigma: float, steps: int, batch: int = 16, lr: float = 5e-4, lr_min: float = 1e-5,
          seed: int = 0, params=None, log_every: int = 200, log=print, scale: float = 1.0,
          fne_lambda: float = 0.0, fne_iters: int = 4, fne_eps: float = 0.05):
    """Adam on the l1 loss over random dihedral transforms of pool images; returns (params, history).

    With ``scale`` s the images are divided by s and the noise level is sigma / s (noise units); the
    returned parameters are those of the network in those units (see ``fold_scale``).
    With ``fne_lambda`` > 0 every step adds the soft firm non-expansiveness penalty of
    Eq. training_loss, fne_lambda / B sum_b max(||grad(2D - I)(z_b) v_b||^2, 1 - fne_eps), v_b from
    ``fne_iters`` power iterations from Gaussian draws (the Jacobian of D does not change with the
    noise-unit scaling)."""
    import torch
    import synth
    import paper_2207_11336_gb300 as pnp
    N, s, _ = pool.shape
    if params is None:
        params = synth.cnn_init(synth.rng_for("train"), 64, 8, last_scale=0.01)
    tr = pnp.CnnTrainer(params, batch, s, lr=lr)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    hist = []
    t0 = time.perf_counter()
    for it in range(steps):
        cur = lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * it / max(steps - 1, 1)))
        tr.set_lr(cur)
        idx = torch.randint(0, N, (batch,), device="cuda", generator=gen)
        u = pool[idx]
        k = int(torch.randint(0, 8, (1,), generator=gen, device="cuda").item())
        if k & 4:
            u = u.transpose(1, 2)
        u = torch.rot90(u, k & 3, dims=(1, 2))
        if scale != 1.0:
            u = u * (1.0 / scale)
        u = u.contiguous()
        noise = torch.randn((batch, s, s), device="cuda", generator=gen)
        want = (it + 1) % log_every == 0 or it == steps - 1
        pen = None
        if fne_lambda > 0:
            v0 = torch.randn((batch, s, s), device="cuda", generator=gen)
            vals = tr.step_fne(u, noise, sigma / scale, v0, fne_iters, fne_lambda, fne_eps, update=True,
                               want_values=want)
            loss, pen = vals if want else (None, None)
        else:
            loss = tr.step(u, noise, sigma / scale, update=True, want_loss=want)
        if want:
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            hist.append((it + 1, loss * scale, el))
            extra = "" if pen is None else f"  penalty {pen:.4e}"
            log(f"step {it + 1:6d}  loss {loss * scale:.4e} (image units){extra}  lr {cur:.2e}  {el:7.1f} s")
    out, _ = tr.read()
    tr.close()
    return out, hist


def save(path: str, params, meta: dict):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    arrs = {}
    for i, (W, b) in enumerate(params):
        arrs[f"W{i}"] = np.asarray(W, dtype=np.float32)
        arrs[f"b{i}"] = np.asarray(b, dtype=np.float32)
    for k, v in meta.items():
        arrs[f"meta_{k}"] = np.asarray(v)
    np.savez_compressed(path, **arrs)


def load(path: str):
    """(params as float64 (W, b) pairs, metadata dict) from ``save``'s file."""
    d = np.load(path)
    depth = sum(1 for k in d.files if k.startswith("W"))
    params = [(d[f"W{i}"].astype(np.float64), d[f"b{i}"].astype(np.float64)) for i in range(depth)]
    meta = {k[5:]: d[k].item() if d[k].ndim == 0 else d[k] for k in d.files if k.startswith("meta_")}
    return params, meta


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="C3", help="imaging problem whose heuristic sets sigma")
    ap.add_argument("--sigma", type=float, default=None, help="override the heuristic noise level")
    ap.add_argument("--images", type=int, default=20000)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--image-units", action="store_true",
                    help="train at the images' own scale instead of in noise units")
    ap.add_argument("--init", default=None, help="start from these weights (fine-tuning)")
    ap.add_argument("--fne-lambda", type=float, default=0.0,
                    help="weight of the soft firm non-expansiveness penalty (0: l1 loss only)")
    ap.add_argument("--fne-iters", type=int, default=4, help="power iterations per penalised step")
    ap.add_argument("--fne-eps", type=float, default=0.05, help="penalty floor 1 - eps on ||grad(2D - I)||^2")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                                  "dncnn_C3.npz"))
    a = ap.parse_args(argv)
    t0 = time.perf_counter()
    pool_np = image_pool(a.images, a.size, a.seed)   # before any CUDA call (spawned workers)
    print(f"pool: {pool_np.shape} in {time.perf_counter() - t0:.1f} s", flush=True)
    import torch
    meta = dict(workload=a.workload, images=a.images, size=a.size, batch=a.batch, steps=a.steps, lr=a.lr,
                seed=a.seed, fne_lambda=a.fne_lambda, fne_iters=a.fne_iters, fne_eps=a.fne_eps)
    if a.sigma is None:
        from paper_2207_11336_gb300 import heuristics
        import synth
        prob, plan, _, y, tau = noisy_problem(a.workload)
        v0 = torch.from_numpy(synth.rng_for("power").standard_normal((prob["n"],) * 2).astype(np.float32)).cuda()
        hp = heuristics.imaging_parameters(plan, y, tau, v0)
        plan.close()
        del plan, y
        torch.cuda.empty_cache()
        sigma = hp["sigma"]
        meta.update({f"heuristic_{k}": v for k, v in hp.items()})
        print("heuristics:", {k: float(v) for k, v in hp.items()}, flush=True)
    else:
        sigma = a.sigma
    meta["sigma"] = sigma
    scale = 1.0 if a.image_units else noise_unit(sigma)
    meta["noise_unit"] = scale
    pool = torch.from_numpy(pool_np).cuda()
    init = None
    if a.init:
        # fine-tuning: the saved network acts at image scale; train() works in noise units
        init = fold_scale(load(a.init)[0], 1.0 / scale)
    params, hist = train(pool, sigma, a.steps, a.batch, a.lr, seed=a.seed, params=init,
                         log=lambda s: print(s, flush=True), scale=scale, fne_lambda=a.fne_lambda,
                         fne_iters=a.fne_iters, fne_eps=a.fne_eps)
    params = fold_scale(params, scale)
    meta["loss_history"] = np.array([h[1] for h in hist])
    meta["train_seconds"] = hist[-1][2] if hist else 0.0
    save(a.out, params, meta)
    print("saved", a.out, flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
