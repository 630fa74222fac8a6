"""The five imaging workloads (C0..C4) as seeded synthetic problems.

C0  plain PnP-FB: 256^2 image, 512^2 grid, KB J=7, M=2e5, no w, Haar, 200 its.
C1  gradient step only: 2048^2 image, 4096^2 grid, M=2e7, 12 h track,
    w folded into G with J in {7,9,12,16} by |w| quartile.
C2  learned residual CNN denoiser used on C1's operator (512^2 facets, 32 px halo).
C3  4096^2 image, 8192^2 grid, M=2e7 in 64 radial blocks, 16 uneven facets.
C4  8192^2 image, 16384^2 grid, M=2.5e7 per band (1053 and 1399 MHz),
    J in {7,8,8,9}, BF16 weights.
"""
from __future__ import annotations

import numpy as np

from . import meerkat as mk

CONFIGS = {
    "C0": dict(n=256, K=512, M=200_000, hours=8.0, supports=None, w_spread=0.0,
               isnr_db=40.0, n_blocks=1, facets=None, halo=0, iters=200),
    "C1": dict(n=2048, K=4096, M=20_000_000, hours=12.0, supports=(7, 9, 12, 16),
               w_spread=4.0, isnr_db=40.0, n_blocks=1, facets=(4, 512, 512), halo=32, iters=200),
    "C3": dict(n=4096, K=8192, M=20_000_000, hours=12.0, supports=(7, 9, 12, 16),
               w_spread=4.0, isnr_db=40.0, n_blocks=64, facets=(4, 768, 1280), halo=32, iters=200,
               robust=0.0),
    "C4": dict(n=8192, K=16384, M=25_000_000, hours=12.0, supports=(7, 8, 8, 9),
               w_spread=2.0, isnr_db=40.0, n_blocks=1, facets=(8, 1024, 1024), halo=32, iters=500,
               robust=0.0, ref_freq_hz=1.399e9),
}


def make_problem(name: str, M: int | None = None, n: int | None = None, K: int | None = None,
                 freq_hz: float = 1.399e9, root_seed: int = 0, with_sky: bool = True,
                 n_stacks: int = 1) -> dict:
    """Seeded inputs for one workload (sizes may be overridden for small cases).

    Returns a dict with n, K, M, omega (M, 2) rad/px, w (M,) wavelengths, dl,
    J_per_row (int8 or None for a single J=7), x_true (n, n) float64 sky,
    imaging_weight (M,) Briggs weights (robust 0, Sec. 3) for the wide-field workloads
    (None for the others: natural weighting),
    noise (M,) standard complex normal draws, block (M,) int32, facet widths,
    and the w-stack layout: stack (M,) int32 ids and w_centres (n_stacks,).  With
    n_stacks > 1 (w-stacking hybrid, App. E) the stacks are the minimum-taps
    partition of w and the supports follow the residual |w - centre| against the
    unstacked |w| quartile edges.
    """
    cfg = dict(CONFIGS[name])
    if M is not None:
        cfg["M"] = int(M)
    if n is not None:
        cfg["n"] = int(n)
        cfg["K"] = int(K if K is not None else 2 * n)
    m, nn, kk = cfg["M"], cfg["n"], cfg["K"]
    enu = mk.antenna_layout(mk.rng_for("uv", root_seed))
    # the pixel size is fixed by a reference band (both bands of the 8192^2 workload share one image
    # grid, as in Sec. 3): its longest baseline sits at 0.8 of Nyquist, another band's (u, v, w) in
    # wavelengths scale with its frequency
    ref = cfg.get("ref_freq_hz", freq_hz)
    uvw = mk.uvw_track(enu, m, cfg["hours"], freq_hz=ref)
    omega, w, dl = mk.imaging_geometry(uvw, nn, kk, 0.8, cfg["w_spread"])
    omega, w = omega * (freq_hz / ref), w * (freq_hz / ref)
    out = dict(name=name, n=nn, K=kk, M=m, omega=omega, w=w, dl=dl,
               isnr_db=cfg["isnr_db"], iters=cfg["iters"], halo=cfg["halo"])
    out["J_per_row"] = (mk.j_per_row_by_w_quartile(w, cfg["supports"])
                        if cfg["supports"] is not None else None)
    if n_stacks > 1:
        if cfg["supports"] is None or dl == 0.0:
            raise ValueError(f"{name} has no w-terms to stack")
        out["stack"], out["w_centres"] = mk.w_stacks_min_taps(w, n_stacks, cfg["supports"])
        out["J_per_row"] = mk.j_per_row_stacked(w, out["stack"], out["w_centres"], w, cfg["supports"])
    else:
        out["stack"], out["w_centres"] = np.zeros(m, dtype=np.int32), np.zeros(1)
    if with_sky:
        scale = nn / 256.0
        out["x_true"] = mk.sky_model(nn, mk.rng_for("sky", root_seed),
                                     n_points=int(round(200 * scale)), n_blobs=5)
    out["noise"] = mk.complex_normal(m, mk.rng_for("noise", root_seed))
    robust = cfg.get("robust")
    out["imaging_weight"] = None if robust is None else mk.briggs_weights(omega, nn, robust)
    out["block"] = (mk.radial_blocks(omega, cfg["n_blocks"], mk.rng_for("blocks", root_seed))
                    if cfg["n_blocks"] > 1 else np.zeros(m, dtype=np.int32))
    if cfg["facets"] is not None:
        nf, lo, hi = cfg["facets"]
        lo, hi = lo * nn // CONFIGS[name]["n"], hi * nn // CONFIGS[name]["n"]
        rf = mk.rng_for("facets", root_seed)
        out["facet_rows"] = mk.facet_layout(nn, nf, rf, lo, hi)
        out["facet_cols"] = mk.facet_layout(nn, nf, rf, lo, hi)
    return out
