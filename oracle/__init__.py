"""Plain, slow FP64 CPU oracle for the PnP forward-backward imaging path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA product path never calls it, and it never calls the CUDA path: the two
share no code.  Inputs come from the separate ``synth`` package.

Each function cites the passage of arXiv 2207.11336 (Dabbech et al. 2022) it
follows.  Where the paper is silent the function states the reading it takes.

Modules
-------
nufft   measurement operator Phi = G F Z (Eq. 1), w-folded rows (App. E),
        direct non-uniform DFT used as ground truth.
fb      data-fidelity gradient and Lipschitz constant (App. A), power
        iteration, Haar soft-threshold prox (App. B, one-level form),
        forward-backward iteration (Eq. fb), parameter heuristics
        (Eqs. lambda, sigma; App. F).
cnn     residual CNN denoiser (App. C): forward, backward, l1 training loss,
        Adam, faceted inference (App. D).

Parity status: every function is pinned by a ``-m "not gpu"`` test against
something other than itself (a library routine, a closed form, an invariant
or brute force): ``fb.snr_db`` by closed-form cases of its definition and
``fb.pnp_fb`` by its limits with the identity and positivity denoisers
(numpy's least squares and scipy's NNLS on the dense system).  The paper
prints no reconstruction SNR for synthetic data, so the SNR values the loops
reach on the synthetic skies are comparative, not pinned to the paper.
"""
