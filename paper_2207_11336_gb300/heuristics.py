"""Parameter heuristics of PnP-FB imaging, evaluated with the library's GPU operator.

* L = ||Re{Phi^H Phi}||_S by power iteration (App. A) and gamma = 1.98 / L (App. B);
* the image-domain noise level tau / sqrt(2L) (Eq. lambda), which is also the
  soft threshold gamma*lambda of the plain Haar prox;
* beta = max_i (Re{Phi^H Phi} delta)_i with delta the unit image at the phase
  centre, the peak of the dirty beam (App. F, footnote on the normalisation);
* alpha = max(Re{Phi^H y}) / beta, the peak of the normalised dirty image, an
  upper bound on the sky's peak by which the problem is rescaled before a
  learned denoiser trained on peak-normalised images is applied (App. C, F);
* sigma = tau / (alpha sqrt(2L)), the noise level a denoiser must be trained
  for to act on the rescaled problem (Eq. sigma), and conversely the alpha that
  matches a problem to a denoiser trained at a given sigma (App. F: one
  denoiser for several data sets, each rescaled by its own alpha).

Every operator application runs in the library's kernels; only scalars are
combined here.
"""
from __future__ import annotations

import numpy as np


def psf_peak(plan) -> float:
    """beta: the dirty beam Re{Phi^H Phi} delta at the phase centre (pixel (n/2, n/2))."""
    import torch
    n = plan.n
    d = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    d[n // 2, n // 2] = 1.0
    psf = plan.phi_adjoint(plan.phi_forward(d))
    return float(psf.max().item())


def dirty_peak(plan, y, beta: float) -> float:
    """alpha: peak of the dirty image Re{Phi^H y} normalised by the dirty-beam peak beta."""
    return float(plan.phi_adjoint(y).max().item()) / beta


def imaging_parameters(plan, y, tau: float, v0=None, max_it: int = 1000, tol: float = 1e-6) -> dict:
    """All scalars of the plain and the learned loop for data y with noise std tau."""
    L, it = plan.op_norm(v0, max_it, tol)
    beta = psf_peak(plan)
    alpha = dirty_peak(plan, y, beta)
    noise = tau / np.sqrt(2.0 * L)
    return dict(L=L, power_iters=it, gamma=1.98 / L, tau=tau, noise_level=noise, beta=beta, alpha=alpha,
                sigma=noise / alpha)


def alpha_for_denoiser(tau: float, L: float, sigma_train: float) -> float:
    """alpha with tau / (alpha sqrt(2L)) = sigma_train: Eq. sigma solved for alpha (App. F).

    A valid rescaling needs alpha >= the peak of the sought image; callers take the larger of this
    and the dirty-peak bound."""
    return tau / (sigma_train * np.sqrt(2.0 * L))
