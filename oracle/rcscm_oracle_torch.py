"""FP64 PyTorch restatement of the accelerated estimator, for gradients.

TEST INFRASTRUCTURE ONLY (imported by the tests; never by the product path).
Plain CPU torch ops in complex128/float64, differentiated by autograd, give the
oracle gradient of a loss of the extracted target image with respect to x, a
and R'.  The forward follows the same steps as ``rcscm_oracle.run`` with the
second-stage rule (Algorithm 2, Sec. III-C-2) and the multichannel Wiener
filter (posterior mean); lambda_i starts from a given lambda0 (held constant),
and the initial variances are constants.  Its outputs are pinned to the numpy
oracle and its gradients to central finite differences of the numpy oracle
(tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import torch


def _h(A):
    return A.conj().transpose(-1, -2)


def forward(x, a, Rp, rh0, ru0, lam0, n_iter: int, alpha: float = 1.1, beta: float = 1e-16):
    """x [I,J,M], a [I,M], Rp [I,M,M] complex128; rh0, ru0 [I,J], lam0 [I] float64.

    Returns the Wiener estimate h [I,J,M] and the final (rh, ru, lam)."""
    M = x.shape[-1]
    A = 0.5 * (Rp + _h(Rp))                                    # symmetrised R'
    mu, E = torch.linalg.eigh(A)                               # ascending
    b = E[..., :, 0]
    En = E[..., :, 1:]
    P = (En / mu[..., None, 1:].to(En.dtype)) @ _h(En)        # (R')^+, Eq. (eq:riinv)
    tau_aa = torch.einsum("im,imn,in->i", a.conj(), P, a).real
    sigma_ab = torch.einsum("im,im->i", a.conj(), b)
    tau_ax = torch.einsum("im,imn,ijn->ij", a.conj(), P, x)
    tau_xx = torch.einsum("ijm,imn,ijn->ij", x.conj(), P, x).real
    sigma_bx = torch.einsum("im,ijm->ij", b.conj(), x)
    sab = sigma_ab[:, None]
    sab2 = sigma_ab.abs() ** 2
    rh, ru, lam = rh0, ru0, lam0
    for _ in range(n_iter):                                    # Algorithm 2
        rho_aa_t = tau_aa + sab2 / lam
        rho_ax_t = tau_ax + sab * sigma_bx / lam[:, None]
        gamma = rh / (ru + rh * rho_aa_t[:, None])
        rh_new = (gamma * (ru + gamma * rho_ax_t.abs() ** 2) + beta) / (alpha + 2.0)
        ell = gamma * sab2[:, None] + (sigma_bx - gamma * sab.conj() * rho_ax_t).abs() ** 2 / ru
        lam_new = ell.mean(dim=1)
        rho_aa = tau_aa + sab2 / lam_new
        rho_ax = tau_ax + sab * sigma_bx / lam_new[:, None]
        rho_xx = tau_xx + sigma_bx.abs() ** 2 / lam_new[:, None]
        ru = (gamma * rho_aa[:, None] * (ru + gamma * rho_ax_t.abs() ** 2)
              + rho_xx - 2.0 * gamma * (rho_ax_t * rho_ax.conj()).real) / M
        rh, lam = rh_new, lam_new
    rho_aa = tau_aa + sab2 / lam
    rho_ax = tau_ax + sab * sigma_bx / lam[:, None]
    w = rh * rho_ax / (ru + rh * rho_aa[:, None])
    h = w[..., None] * a[:, None, :]
    return h, (rh, ru, lam)


def loss_and_grads(x, a, Rp, rh0, ru0, lam0, n_iter, h_true, alpha=1.1, beta=1e-16):
    """L = sum |h - h_true|^2 and its gradients (PyTorch convention for complex
    inputs: dL/dRe + i dL/dIm) with respect to x, a and R'."""
    x = torch.as_tensor(x, dtype=torch.complex128).clone().requires_grad_(True)
    a = torch.as_tensor(a, dtype=torch.complex128).clone().requires_grad_(True)
    Rp = torch.as_tensor(Rp, dtype=torch.complex128).clone().requires_grad_(True)
    args = [torch.as_tensor(v, dtype=torch.float64) for v in (rh0, ru0, lam0)]
    h, _ = forward(x, a, Rp, *args, n_iter, alpha, beta)
    loss = ((h - torch.as_tensor(h_true, dtype=torch.complex128)).abs() ** 2).sum()
    loss.backward()
    return float(loss.detach()), x.grad.numpy(), a.grad.numpy(), Rp.grad.numpy()
