"""MeerKAT-like synthetic measurement geometry and skies (seeded).

Every generator takes a numpy ``Generator`` or a seed-stream name; the named
streams are spawned from ``SeedSequence(0)`` so each kind of draw (uv, sky,
noise, blocks, facets, power-iteration start, training) is reproducible on its
own.
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299_792_458.0

SEED_STREAMS = ("uv", "sky", "noise", "blocks", "facets", "power", "train", "misc")


def rng_for(name: str, root_seed: int = 0) -> np.random.Generator:
    """Generator for one named stream spawned from SeedSequence(root_seed)."""
    idx = SEED_STREAMS.index(name)
    child = np.random.SeedSequence(root_seed).spawn(len(SEED_STREAMS))[idx]
    return np.random.default_rng(child)


def antenna_layout(rng: np.random.Generator, n_core: int = 48, n_outer: int = 16,
                   core_sigma_m: float = 300.0, outer_radius_m: float = 4000.0) -> np.ndarray:
    """East/North antenna positions [m], shape (n_core + n_outer, 2).

    A Gaussian core (sigma per axis) plus antennas uniform in area out to a
    radius, giving baselines up to ~8 km like the array of Sec. 3.
    """
    core = rng.normal(0.0, core_sigma_m, size=(n_core, 2))
    r = outer_radius_m * np.sqrt(rng.random(n_outer))
    th = 2.0 * np.pi * rng.random(n_outer)
    outer = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    return np.concatenate([core, outer], axis=0)


def uvw_track(enu: np.ndarray, n_rows: int, hours: float, dec_deg: float = -60.0,
              lat_deg: float = -30.7, freq_hz: float = 1.399e9) -> np.ndarray:
    """(u, v, w) in wavelengths for all antenna pairs over a symmetric hour-angle track.

    Rows are ordered (time, baseline) and truncated to ``n_rows``.  The number of
    time samples is ceil(n_rows / n_baselines), spread uniformly over
    [-hours/2, +hours/2].
    """
    lat = np.deg2rad(lat_deg)
    dec = np.deg2rad(dec_deg)
    east, north = enu[:, 0], enu[:, 1]
    # local horizontal plane -> equatorial XYZ (antennas on a flat plane, up = 0)
    X = -np.sin(lat) * north
    Y = east
    Z = np.cos(lat) * north
    ii, jj = np.triu_indices(len(enu), k=1)
    bx, by, bz = X[jj] - X[ii], Y[jj] - Y[ii], Z[jj] - Z[ii]
    nb = len(ii)
    nt = -(-n_rows // nb)
    ha = np.deg2rad(15.0) * np.linspace(-hours / 2.0, hours / 2.0, nt)
    sh, ch = np.sin(ha)[:, None], np.cos(ha)[:, None]
    u = sh * bx + ch * by
    v = -np.sin(dec) * ch * bx + np.sin(dec) * sh * by + np.cos(dec) * bz
    w = np.cos(dec) * ch * bx - np.cos(dec) * sh * by + np.sin(dec) * bz
    lam = C_LIGHT / freq_hz
    uvw = np.stack([u.ravel(), v.ravel(), w.ravel()], axis=1)[:n_rows] / lam
    return uvw


def imaging_geometry(uvw_lambda: np.ndarray, n: int, K: int, nyquist_frac: float = 0.8,
                     w_spread_bins: float = 0.0):
    """Map physical (u, v, w) to the imaging problem's inputs.

    Returns ``(omega, w, dl)``: ``omega`` (M, 2) float64 angular frequencies in
    rad/pixel (column 0 pairs with image axis 0, column 1 with axis 1), scaled
    so the longest uv baseline sits at ``nyquist_frac * pi``; ``w`` in
    wavelengths; ``dl`` the pixel size in radians used for the w-term, chosen so
    that the largest |w| spreads its image-edge chirp over ``w_spread_bins``
    grid cells (``w * dl**2 * n * K = w_spread_bins``).  ``w_spread_bins = 0``
    gives ``dl = 0`` (no w-term).
    """
    uv = uvw_lambda[:, :2]
    bmax = np.max(np.hypot(uv[:, 0], uv[:, 1]))
    omega = uv * (nyquist_frac * np.pi / bmax)
    w = uvw_lambda[:, 2].copy()
    if w_spread_bins > 0:
        wmax = np.max(np.abs(w))
        dl = float(np.sqrt(w_spread_bins / (wmax * n * K)))
    else:
        dl = 0.0
    return omega, w, dl


def briggs_weights(omega: np.ndarray, n: int, robust: float) -> np.ndarray:
    """Briggs (robust) imaging weights of the visibilities (Briggs 1995), float64 (M,).

    Sec. 3 images data weighted by this scheme with robust parameter 0; the weights are a
    property of the data set, fixed before imaging, and reach the imaging problem as an
    input like the uv coverage.  Each row (natural weight 1) falls in a cell of the n x n uv
    grid whose spacing is the inverse field of view (cell = 2 pi / n rad/px in omega); W_k
    counts the rows in cell k together with the rows whose conjugate (-u, -v) lands there
    (each baseline samples both).  With f^2 = (5 * 10^-robust)^2 / (sum_m W_k(m) / M), the
    mean cell occupancy seen by a visibility, a row in cell k gets 1 / (1 + W_k f^2):
    robust -> +inf gives natural weighting (all 1), robust -> -inf uniform weighting (1 / W_k
    up to a constant).
    """
    omega = np.asarray(omega, dtype=np.float64)
    k = np.rint(omega * (n / (2.0 * np.pi))).astype(np.int64) % n
    cell = k[:, 0] * n + k[:, 1]
    conj = ((-k[:, 0]) % n) * n + ((-k[:, 1]) % n)
    W = (np.bincount(cell, minlength=n * n) + np.bincount(conj, minlength=n * n)).astype(np.float64)
    Wm = W[cell]
    if Wm.size == 0:
        return np.zeros(0)
    f2 = (5.0 * 10.0 ** (-robust)) ** 2 / (Wm.sum() / Wm.size)
    return 1.0 / (1.0 + Wm * f2)


def j_per_row_by_w_quartile(w: np.ndarray, supports=(7, 9, 12, 16)) -> np.ndarray:
    """Per-row kernel support J (int8): the q-th |w| quartile gets supports[q]."""
    aw = np.abs(w)
    edges = np.quantile(aw, [0.25, 0.5, 0.75])
    q = np.searchsorted(edges, aw, side="right")
    return np.asarray(supports, dtype=np.int8)[q]


def w_stacks(w: np.ndarray, n_stacks: int) -> tuple[np.ndarray, np.ndarray]:
    """w-stack id (int32) per row and the stack centres (float64, wavelengths).

    The rows are binned into n_stacks equal-count bins of w (quantile edges);
    each centre is the midpoint of its bin's w range, which minimises the
    largest residual |w - centre| left to the row kernels.
    """
    w = np.asarray(w, dtype=np.float64)
    if n_stacks < 1:
        raise ValueError("n_stacks must be >= 1")
    edges = np.quantile(w, np.linspace(0.0, 1.0, n_stacks + 1)[1:-1]) if w.size else np.zeros(n_stacks - 1)
    stack = np.searchsorted(edges, w, side="right").astype(np.int32)
    centres = np.zeros(n_stacks)
    for s in range(n_stacks):
        ws = w[stack == s]
        if ws.size:
            centres[s] = 0.5 * (ws.min() + ws.max())
    return stack, centres


def w_stacks_min_taps(w: np.ndarray, n_stacks: int, supports=(7, 9, 12, 16), bins: int = 512):
    """w-stack layout (stack ids int32, centres float64) that minimises the taps of G.

    A planning rule for the w-stacking hybrid (App. E leaves the binning to a cost model of
    the operator): w is cut into ``bins`` equal-count bins (fine where the rows are dense),
    and dynamic programming splits them into n_stacks contiguous stacks minimising the sum
    over rows of J^2 with J given by ``j_per_row_stacked``'s rule (residual |w - centre|
    against the unstacked |w| quartile edges, taken at the bin's edge farther from the
    centre).  Each stack takes the best of three centres: the midpoint of its w range, its
    median, and its point nearest w = 0 (so a stack holding w = 0 can keep the central rows
    on the unstacked supports).  Rows are then assigned by the chosen w edges.
    """
    w = np.asarray(w, dtype=np.float64)
    if n_stacks < 1:
        raise ValueError("n_stacks must be >= 1")
    if w.size == 0 or n_stacks == 1:
        return np.zeros(w.size, dtype=np.int32), np.array([0.5 * (w.min() + w.max()) if w.size else 0.0])
    qe = np.quantile(np.abs(w), [0.25, 0.5, 0.75])
    sq = np.asarray(supports, dtype=np.float64) ** 2
    edges = np.unique(np.quantile(w, np.linspace(0.0, 1.0, bins + 1)))
    bins = edges.size - 1
    if bins < 1:
        return np.zeros(w.size, dtype=np.int32), np.full(n_stacks, w[0])
    cnt, _ = np.histogram(w, edges)
    cost = np.full((bins + 1, bins + 1), np.inf)
    centre = np.zeros((bins + 1, bins + 1))
    for i in range(bins):
        j = np.arange(i + 1, bins + 1)
        outside = np.arange(i, bins)[None, :] >= j[:, None]
        best_c, best_t = None, None
        for c in (0.5 * (edges[i] + edges[j]), edges[(i + j) // 2], np.clip(0.0, edges[i], edges[j])):
            r = np.maximum(np.abs(edges[None, i:-1] - c[:, None]), np.abs(edges[None, i + 1:] - c[:, None]))
            taps = sq[np.searchsorted(qe, r, side="right")] * cnt[None, i:]
            taps[outside] = 0.0
            t = taps.sum(axis=1)
            if best_t is None:
                best_c, best_t = c.copy(), t
            else:
                better = t < best_t
                best_c[better], best_t[better] = c[better], t[better]
        cost[i, i + 1:] = best_t
        centre[i, i + 1:] = best_c
    best = np.full((n_stacks + 1, bins + 1), np.inf)
    best[0, 0] = 0.0
    arg = np.zeros((n_stacks + 1, bins + 1), dtype=np.int64)
    for p in range(1, n_stacks + 1):
        for j in range(1, bins + 1):
            v = best[p - 1, :j] + cost[:j, j]
            k = int(np.argmin(v))
            best[p, j], arg[p, j] = v[k], k
    cuts = [bins]
    for p in range(n_stacks, 0, -1):
        cuts.append(int(arg[p, cuts[-1]]))
    cuts = np.asarray(cuts[::-1])
    we = edges[cuts]
    stack = np.clip(np.searchsorted(we[1:-1], w, side="right"), 0, n_stacks - 1).astype(np.int32)
    return stack, centre[cuts[:-1], cuts[1:]].astype(np.float64)


def j_per_row_stacked(w: np.ndarray, stack: np.ndarray, centres: np.ndarray, w_ref: np.ndarray,
                      supports=(7, 9, 12, 16)) -> np.ndarray:
    """Per-row support J (int8) of a w-stacked operator: the |w| quartile edges of the
    unstacked rows w_ref, applied to each row's residual |w - centre of its stack|, so a
    row gets the support an unstacked row with that |w| would get."""
    edges = np.quantile(np.abs(np.asarray(w_ref, dtype=np.float64)), [0.25, 0.5, 0.75])
    resid = np.abs(np.asarray(w, dtype=np.float64) - np.asarray(centres)[stack])
    q = np.searchsorted(edges, resid, side="right")
    return np.asarray(supports, dtype=np.int8)[q]


def _add_blobs(img, rng, n_blobs, sigma_lo, sigma_hi, peak_lo, peak_hi):
    n0, n1 = img.shape
    ya, xa = np.mgrid[0:n0, 0:n1]
    for _ in range(n_blobs):
        cy, cx = rng.uniform(0, n0), rng.uniform(0, n1)
        s = rng.uniform(sigma_lo, sigma_hi)
        peak = 10.0 ** rng.uniform(np.log10(peak_lo), np.log10(peak_hi))
        img += peak * np.exp(-((ya - cy) ** 2 + (xa - cx) ** 2) / (2.0 * s * s))


def sky_model(n: int, rng: np.random.Generator, n_points: int = 200, n_blobs: int = 5,
              flux_lo: float = 1e-4, flux_hi: float = 1.0) -> np.ndarray:
    """Ground-truth sky [Jy/pixel], float64 n x n, non-negative.

    ``n_points`` point sources with log-uniform flux in [flux_lo, flux_hi] at
    uniform pixels, plus ``n_blobs`` Gaussian blobs (width U[2, 8] * n/256 px,
    peak log-U[1e-3, 1e-1]); clipped at zero.
    """
    img = np.zeros((n, n))
    ia = rng.integers(0, n, n_points)
    ib = rng.integers(0, n, n_points)
    flux = 10.0 ** rng.uniform(np.log10(flux_lo), np.log10(flux_hi), n_points)
    np.add.at(img, (ia, ib), flux)
    sc = n / 256.0
    _add_blobs(img, rng, n_blobs, 2.0 * sc, 8.0 * sc, 1e-3, 1e-1)
    return np.clip(img, 0.0, None)


def training_image(n: int, rng: np.random.Generator, flux_lo: float = 1e-5) -> np.ndarray:
    """One normalised high-dynamic-range training image (peak exactly 1).

    Points and Gaussian blobs with log-uniform intensities in [flux_lo, 1],
    standing in for the paper's training database (Sec. C), which is not
    available.
    """
    img = np.zeros((n, n))
    npts = int(rng.integers(20, 200))
    ia = rng.integers(0, n, npts)
    ib = rng.integers(0, n, npts)
    np.add.at(img, (ia, ib), 10.0 ** rng.uniform(np.log10(flux_lo), 0.0, npts))
    _add_blobs(img, rng, int(rng.integers(1, 8)), 1.0, n / 16.0, flux_lo, 1.0)
    img = np.clip(img, 0.0, None)
    return img / img.max()


def complex_normal(m: int, rng: np.random.Generator) -> np.ndarray:
    """Standard complex Gaussian draws (a + ib)/sqrt(2), E|n|^2 = 1, complex128."""
    return (rng.standard_normal(m) + 1j * rng.standard_normal(m)) / np.sqrt(2.0)


def noise_std_for_isnr(norm_clean: float, m: int, isnr_db: float) -> float:
    """tau such that ||Phi x|| / (sqrt(M) tau) = 10^(iSNR/20)."""
    return float(norm_clean / (np.sqrt(m) * 10.0 ** (isnr_db / 20.0)))


def radial_blocks(omega: np.ndarray, n_blocks: int, rng: np.random.Generator,
                  lo: float = 1e5, hi: float = 2e6) -> np.ndarray:
    """Block id (int32) per row: consecutive radial uv slices of log-uniform sizes.

    Block sizes are drawn log-U[lo, hi] and rescaled/clipped until they sum to M;
    rows are ordered by uv angle and cut into those consecutive slices.
    """
    m = omega.shape[0]
    sizes = 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), n_blocks)
    lo_c, hi_c = min(lo, m / n_blocks), max(hi, m / n_blocks)
    for _ in range(100):
        sizes = np.clip(sizes * (m / sizes.sum()), lo_c, hi_c)
        if abs(sizes.sum() - m) < 0.5:
            break
    cnt = np.floor(sizes).astype(np.int64)
    cnt[np.argsort(-(sizes - cnt))[: m - cnt.sum()]] += 1
    if cnt.sum() != m:  # tiny m: fall back to near-equal slices
        cnt = np.full(n_blocks, m // n_blocks, dtype=np.int64)
        cnt[: m - cnt.sum()] += 1
    ang = np.arctan2(omega[:, 1], omega[:, 0])
    order = np.argsort(ang, kind="stable")
    block = np.empty(m, dtype=np.int32)
    block[order] = np.repeat(np.arange(n_blocks, dtype=np.int32), cnt)
    return block


def facet_layout(n: int, nf: int, rng: np.random.Generator, lo: int, hi: int) -> np.ndarray:
    """Facet side widths along one axis: nf integers drawn U[lo, hi], renormalised to sum n."""
    wdt = rng.uniform(lo, hi, nf)
    wdt = wdt * (n / wdt.sum())
    out = np.floor(wdt).astype(np.int64)
    out[np.argsort(-(wdt - out))[: n - out.sum()]] += 1
    return out
