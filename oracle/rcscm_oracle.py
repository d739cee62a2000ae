"""FP64 CPU oracle for rank-constrained SCM estimation (Kubo et al., 2019).

TEST INFRASTRUCTURE ONLY.  This module is imported by the tests, by the smoke
check in ``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``; the
product path never calls it.  It shares no code with the CUDA path: it uses
numpy (complex128 / float64) and takes each step of the paper in the paper's
order and notation.  Inputs are the boundary tensors of one utterance:

    x   [I, J, M] complex   observed STFT x_ij
    a   [I, M]    complex   target steering vector a_i^(h)
    Rp  [I, M, M] complex   rank-(M-1) noise SCM R'_i^(u)
    rh, ru [I, J] real      variances r_ij^(h), r_ij^(u)
    lam [I]       real      lambda_i

Index conventions: i = frequency bin, j = frame, m = microphone (Sec. II-A; the
sentence there that lists the indices swaps "microphones" and "sources"; the
vectors it defines fix m as the microphone index).  The target index n_h is the
first demixing row.

Readings where the paper is silent (each also listed in the design notes):
  * Setup: R' is symmetrised, and exactly one eigenvalue (the smallest) is taken
    as the zero eigenvalue of Sec. II-B-1 (and set to zero in the R' that the
    naive rule, the first-stage rule, the Wiener filter and the objective use);
    b_i is its unit eigenvector and lambda_i starts at the next eigenvalue
    (Sec. II-B-3, "minimum nonzero").
  * Real quantities formed from complex products (tau_aa, tau_xx, rho_aa,
    rho_xx, b^H R^u b, tr(.)) take the real part.
  * Update order inside one pass of the repeat loop follows Algorithms 1 and 2:
    gamma~ and rho~ use the previous (r_h, r_u, lambda); lambda uses the previous
    r_u; r_u uses the NEW lambda with the previous gamma~, rho~, r~_u.
  * The multichannel Wiener filter (named in Sec. II-A and Sec. IV-B without a
    formula) is the posterior mean E[h_ij | x_ij] = r_h a a^H (R_x)^{-1} x with
    the final parameters.
  * The objective is the observed-data log posterior of the generative model of
    Sec. II-B-1 (constants dropped), which every EM pass must not decrease.
Every function here has a pin in tests/test_oracle_pins.py (ilrma_init: in
tests/test_oracle_ilrma.py).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _herm(A):
    return np.conj(np.swapaxes(A, -1, -2))


@dataclass
class Setup:
    """Per-frequency quantities fixed during the iteration."""
    Rp: np.ndarray        # symmetrised R'            [I, M, M]
    mu: np.ndarray        # ascending eigenvalues     [I, M]
    b: np.ndarray         # unit null eigenvector b_i [I, M]
    Rp_pinv: np.ndarray   # (R')^+                    [I, M, M]
    lam0: np.ndarray      # initial lambda_i          [I]
    tau_aa: np.ndarray    # Eq. (eq:taa)              [I]
    sigma_ab: np.ndarray  # Eq. (eq:sap)              [I]


def setup(a, Rp, lambda0=None) -> Setup:
    """Per-frequency setup (Sec. II-B-1, Sec. II-B-3, Eq. (eq:riinv), (eq:taa), (eq:sap)).

    b_i: unit eigenvector of R'_i for its zero eigenvalue.  (R')^+ from the
    eigendecomposition.  lambda_i: smallest nonzero eigenvalue unless given.
    The returned R' has its smallest eigenvalue set to exactly zero, so that
    R_i = R' + lambda b b^H and R_i^{-1} = (R')^+ + b b^H / lambda hold for any
    Hermitian input (for a rank-(M-1) input this changes nothing).
    """
    a = np.asarray(a, np.complex128)
    Rp = np.asarray(Rp, np.complex128)
    Rp = 0.5 * (Rp + _herm(Rp))
    mu, E = np.linalg.eigh(Rp)                       # ascending, orthonormal columns
    b = E[:, :, 0]
    # the smallest eigenvalue is the zero one: R' is used with it set to zero exactly
    Rp = Rp - mu[:, 0, None, None] * np.einsum("im,in->imn", b, np.conj(b))
    En = E[:, :, 1:]
    Rp_pinv = np.einsum("imk,ik,ink->imn", En, 1.0 / mu[:, 1:], np.conj(En))
    lam0 = mu[:, 1].copy() if lambda0 is None else np.asarray(lambda0, np.float64).copy()
    tau_aa = np.real(np.einsum("im,imn,in->i", np.conj(a), Rp_pinv, a))
    sigma_ab = np.einsum("im,im->i", np.conj(a), b)
    return Setup(Rp=Rp, mu=mu, b=b, Rp_pinv=Rp_pinv, lam0=lam0, tau_aa=tau_aa, sigma_ab=sigma_ab)


@dataclass
class IlrmaInit:
    a: np.ndarray         # a_i = column n_h of W_i^{-1}   [I, M]
    Rp: np.ndarray        # Eq. (eq:rit)                   [I, M, M]
    rh0: np.ndarray       # Eq. (eq:rhinit)                [I, J]
    ru0: np.ndarray       # Eq. (eq:ruinit)                [I, J]


def ilrma_init(x, W, T, V, n_h=0) -> IlrmaInit:
    """Inputs of the estimator from the outputs of the ILRMA stage.

    W_i = (w_{i,1} ... w_{i,M})^H is ILRMA's demixing matrix, so W_i = A_i^{-1}
    and the target's steering vector is column n_h of W_i^{-1} (Sec. II-A;
    Sec. II-B-1 names it a_i).  R'_i is the back-projection of the M-1 noise
    outputs w_{i,n}^H x_ij, n != n_h, averaged over the frames (Eq. (eq:rit),
    Sec. II-B-1).  The initial variances follow Sec. II-B-3: r_h from the
    target's NMF bases T (t_{ik,n_h}, [I, K]) and activations V (v_{kj,n_h},
    [K, J]) (Eq. (eq:rhinit)), and r_u = (1/M) y^H (R'_i)^+ y with y the
    back-projected noise image W_i^{-1} (w_1^H x, ..., 0 at n_h, ..., w_M^H x)^T
    (Eq. (eq:ruinit)).  lambda_i starts at the minimum nonzero eigenvalue of
    R'_i, which setup() computes.
    """
    x = np.asarray(x, np.complex128)
    W = np.asarray(W, np.complex128)
    I, J, M = x.shape
    Winv = np.linalg.inv(W)                                      # A_i = W_i^{-1}
    a = Winv[:, :, n_h].copy()
    y = np.einsum("inm,ijm->ijn", W, x)                          # y_ijn = w_{i,n}^H x_ij
    keep = np.ones(M)
    keep[n_h] = 0.0                                              # the target output is left out
    P = np.abs(y) ** 2 * keep                                    # |w_{i,n}^H x_ij|^2, 0 at n_h
    Rp = np.einsum("imn,ijn,ikn->imk", Winv, P, np.conj(Winv)) / J
    rh0 = np.asarray(T, np.float64) @ np.asarray(V, np.float64)  # sum_k t_ik v_kj
    yu = np.einsum("imn,ijn->ijm", Winv, y * keep)               # back-projected noise image
    # (R'_i)^+ of the rank-(M-1) R'_i: its smallest eigenvalue is the zero one (the
    # reading of setup()); a relative cutoff would keep a rounding-level eigenvalue
    # and swamp the quadratic form with its inverse
    mu, E = np.linalg.eigh(0.5 * (Rp + np.conj(np.transpose(Rp, (0, 2, 1)))))
    En = E[:, :, 1:]
    Rp_pinv = np.einsum("imk,ik,ink->imn", En, 1.0 / mu[:, 1:], np.conj(En))
    ru0 = np.real(np.einsum("ijm,imn,ijn->ij", np.conj(yu), Rp_pinv, yu)) / M
    return IlrmaInit(a=a, Rp=Rp, rh0=rh0, ru0=ru0)


@dataclass
class Invariants:
    tau_ax: np.ndarray    # Eq. (eq:tax)  [I, J] complex
    tau_xx: np.ndarray    # Eq. (eq:txx)  [I, J] real
    sigma_bx: np.ndarray  # Eq. (eq:spx)  [I, J] complex


def invariants(x, a, st: Setup) -> Invariants:
    """Quadratic forms that do not change during the iteration (Algorithm 2, before the loop)."""
    x = np.asarray(x, np.complex128)
    tau_ax = np.einsum("im,imn,ijn->ij", np.conj(a), st.Rp_pinv, x)
    tau_xx = np.real(np.einsum("ijm,imn,ijn->ij", np.conj(x), st.Rp_pinv, x))
    sigma_bx = np.einsum("im,ijm->ij", np.conj(st.b), x)
    return Invariants(tau_ax=tau_ax, tau_xx=tau_xx, sigma_bx=sigma_bx)


def iterate_accel2(rh, ru, lam, inv: Invariants, st: Setup, M, alpha, beta):
    """One pass of the repeat loop of Algorithm 2 (second-stage rule, Sec. III-C-2).

    Scalar forms of the updates as printed in Sec. III-C-2 for r_h, lambda_i, r_u.
    Returns (rh, ru, lam).
    """
    rh_t, ru_t, lam_t = rh, ru, lam                                   # tilde copies
    sab = st.sigma_ab[:, None]
    sab2 = np.abs(st.sigma_ab) ** 2
    rho_aa_t = st.tau_aa + sab2 / lam_t                               # Eq. (eq:traa_accel)
    rho_ax_t = inv.tau_ax + sab * inv.sigma_bx / lam_t[:, None]       # rho~^(ax)
    gamma = rh_t / (ru_t + rh_t * rho_aa_t[:, None])                  # Eq. (eq:tal)
    rh_new = (gamma * (ru_t + gamma * np.abs(rho_ax_t) ** 2) + beta) / (alpha + 2.0)
    ell = gamma * sab2[:, None] + np.abs(inv.sigma_bx - gamma * np.conj(sab) * rho_ax_t) ** 2 / ru_t
    lam_new = np.mean(ell, axis=1)                                    # Eq. (eq:1st_li) via (eq:traa_accel)
    rho_aa = st.tau_aa + sab2 / lam_new
    rho_ax = inv.tau_ax + sab * inv.sigma_bx / lam_new[:, None]
    rho_xx = inv.tau_xx + np.abs(inv.sigma_bx) ** 2 / lam_new[:, None]
    ru_new = (gamma * rho_aa[:, None] * (ru_t + gamma * np.abs(rho_ax_t) ** 2)
              + rho_xx - 2.0 * gamma * np.real(rho_ax_t * np.conj(rho_ax))) / M
    return rh_new, ru_new, lam_new


def iterate_accel1(rh, ru, lam, x, a, st: Setup, alpha, beta):
    """One pass of the repeat loop of Algorithm 1 (first-stage rule, Sec. III-C-1).

    Uses explicit per-frequency inverses of R~_i and R_i with Eqs. (eq:raa)-(eq:tal),
    (eq:1st_rh), (eq:1st_li), (eq:1st_ru).
    """
    x = np.asarray(x, np.complex128)
    M = x.shape[-1]
    bbH = np.einsum("im,in->imn", st.b, np.conj(st.b))
    rh_t, ru_t, lam_t = rh, ru, lam
    Rt_inv = np.linalg.inv(st.Rp + lam_t[:, None, None] * bbH)        # (R~_i)^{-1}
    rho_aa_t = np.real(np.einsum("im,imn,in->i", np.conj(a), Rt_inv, a))        # (eq:traa)
    rho_ax_t = np.einsum("im,imn,ijn->ij", np.conj(a), Rt_inv, x)                # (eq:trax)
    sab = st.sigma_ab[:, None]
    sbx = np.einsum("im,ijm->ij", np.conj(st.b), x)                             # (eq:spx)
    gamma = rh_t / (ru_t + rh_t * rho_aa_t[:, None])                            # (eq:tal)
    rh_new = (gamma * (ru_t + gamma * np.abs(rho_ax_t) ** 2) + beta) / (alpha + 2.0)
    lam_new = np.mean(gamma * np.abs(sab) ** 2
                      + np.abs(sbx - gamma * np.conj(sab) * rho_ax_t) ** 2 / ru_t, axis=1)
    R_inv = np.linalg.inv(st.Rp + lam_new[:, None, None] * bbH)       # up-to-date R_i
    rho_aa = np.real(np.einsum("im,imn,in->i", np.conj(a), R_inv, a))           # (eq:raa)
    rho_ax = np.einsum("im,imn,ijn->ij", np.conj(a), R_inv, x)                   # (eq:rax)
    rho_xx = np.real(np.einsum("ijm,imn,ijn->ij", np.conj(x), R_inv, x))         # (eq:rxx)
    ru_new = (gamma * rho_aa[:, None] * (ru_t + gamma * np.abs(rho_ax_t) ** 2)
              + rho_xx - 2.0 * gamma * np.real(rho_ax_t * np.conj(rho_ax))) / M
    return rh_new, ru_new, lam_new


def e_step_naive(rh_t, ru_t, lam_t, x, a, st: Setup, dtype=np.complex128):
    """E-step of Sec. II-B-2 with an explicit M x M inverse per slot.

    Returns (rhat_h [I, J], Rhat_u [I, J, M, M]).  Eqs. (eq:rijx), (eq:E_hrh), (eq:E_hru).
    ``dtype`` is the precision of the arithmetic: complex128 for the oracle;
    the tests also evaluate the same formulas in complex64 to measure the
    accuracy that single precision allows for this rule.
    """
    rdt = np.float32 if dtype == np.complex64 else np.float64
    x = np.asarray(x, dtype)
    a = np.asarray(a, dtype)
    rh_t, ru_t, lam_t = (np.asarray(v, rdt) for v in (rh_t, ru_t, lam_t))
    st = Setup(Rp=np.asarray(st.Rp, dtype), mu=st.mu, b=np.asarray(st.b, dtype), Rp_pinv=st.Rp_pinv,
               lam0=st.lam0, tau_aa=st.tau_aa, sigma_ab=st.sigma_ab)
    bbH = np.einsum("im,in->imn", st.b, np.conj(st.b))
    Rt = st.Rp + lam_t[:, None, None] * bbH                                     # R~_i
    aaH = np.einsum("im,in->imn", a, np.conj(a))
    Rx = rh_t[..., None, None] * aaH[:, None] + ru_t[..., None, None] * Rt[:, None]   # (eq:rijx)
    P = np.linalg.inv(Rx)                                                        # (R~^(x)_ij)^{-1}
    aPa = np.einsum("im,ijmn,in->ij", np.conj(a), P, a)
    xPa = np.einsum("ijm,ijmn,in->ij", np.conj(x), P, a)
    rhat_h = np.real(rh_t - rh_t ** 2 * aPa + np.abs(rh_t * xPa) ** 2)          # (eq:E_hrh)
    RtP = np.einsum("imk,ijkn->ijmn", Rt, P)
    RtPRt = np.einsum("ijmk,ikn->ijmn", RtP, Rt)
    RtPx = np.einsum("ijmn,ijn->ijm", RtP, x)
    Rhat_u = (ru_t[..., None, None] * Rt[:, None]
              - (ru_t ** 2)[..., None, None] * RtPRt
              + (ru_t ** 2)[..., None, None] * np.einsum("ijm,ijn->ijmn", RtPx, np.conj(RtPx)))  # (eq:E_hru)
    return rhat_h, Rhat_u


def m_step_naive(rhat_h, Rhat_u, ru_t, st: Setup, M, alpha, beta, dtype=np.complex128):
    """M-step of Sec. II-B-2: Eqs. (eq:M_rh), (eq:M_li), R_i update, (eq:M_ru)."""
    rdt = np.float32 if dtype == np.complex64 else np.float64
    ru_t, alpha, beta = np.asarray(ru_t, rdt), rdt(alpha), rdt(beta)
    st = Setup(Rp=np.asarray(st.Rp, dtype), mu=st.mu, b=np.asarray(st.b, dtype), Rp_pinv=st.Rp_pinv,
               lam0=st.lam0, tau_aa=st.tau_aa, sigma_ab=st.sigma_ab)
    rh_new = (rhat_h + beta) / (alpha + 2.0)                                     # (eq:M_rh)
    bRb = np.real(np.einsum("im,ijmn,in->ij", np.conj(st.b), Rhat_u, st.b))
    lam_new = np.mean(bRb / ru_t, axis=1)                                        # (eq:M_li)
    bbH = np.einsum("im,in->imn", st.b, np.conj(st.b))
    R = st.Rp + lam_new[:, None, None] * bbH                                     # R_i <- R' + lambda b b^H
    R_inv = np.linalg.inv(R)
    ru_new = np.real(np.einsum("imn,ijnm->ij", R_inv, Rhat_u)) / M               # (eq:M_ru)
    return rh_new, ru_new, lam_new


def iterate_naive(rh, ru, lam, x, a, st: Setup, alpha, beta, dtype=np.complex128):
    """One EM pass of the naive rule (Sec. II-B-2), frequency by frequency."""
    M = np.asarray(x).shape[-1]
    rdt = np.float32 if dtype == np.complex64 else np.float64
    out_rh = np.empty(np.shape(rh), rdt)
    out_ru = np.empty(np.shape(ru), rdt)
    out_lam = np.empty(np.shape(lam), rdt)
    for i in range(rh.shape[0]):
        sub = Setup(Rp=st.Rp[i:i + 1], mu=st.mu[i:i + 1], b=st.b[i:i + 1],
                    Rp_pinv=st.Rp_pinv[i:i + 1], lam0=st.lam0[i:i + 1],
                    tau_aa=st.tau_aa[i:i + 1], sigma_ab=st.sigma_ab[i:i + 1])
        rhat_h, Rhat_u = e_step_naive(rh[i:i + 1], ru[i:i + 1], lam[i:i + 1], x[i:i + 1], a[i:i + 1], sub, dtype)
        r1, r2, l = m_step_naive(rhat_h, Rhat_u, ru[i:i + 1], sub, M, alpha, beta, dtype)
        out_rh[i], out_ru[i], out_lam[i] = r1[0], r2[0], l[0]
    return out_rh, out_ru, out_lam


def model_cov(rh, ru, lam, a, st: Setup):
    """R^(x)_ij = r_h a a^H + r_u (R' + lambda b b^H)  [I, J, M, M] (Sec. II-B-1)."""
    bbH = np.einsum("im,in->imn", st.b, np.conj(st.b))
    R = st.Rp + lam[:, None, None] * bbH
    aaH = np.einsum("im,in->imn", a, np.conj(a))
    return rh[..., None, None] * aaH[:, None] + ru[..., None, None] * R[:, None]


def wiener(rh, ru, lam, x, a, st: Setup):
    """Multichannel Wiener filter: h_ij = r_h a a^H (R^(x)_ij)^{-1} x_ij (posterior mean)."""
    x = np.asarray(x, np.complex128)
    Rx = model_cov(rh, ru, lam, a, st)
    Px = np.linalg.solve(Rx, x[..., None])[..., 0]
    aPx = np.einsum("im,ijm->ij", np.conj(a), Px)
    return (rh * aPx)[..., None] * a[:, None, :]


def objective(rh, ru, lam, x, a, st: Setup, alpha, beta):
    """Observed-data log posterior, constants dropped (Sec. II-B-1).

    sum_ij [ -log det R^(x)_ij - x^H (R^(x)_ij)^{-1} x - (alpha+1) log r_h - beta / r_h ].
    """
    x = np.asarray(x, np.complex128)
    Rx = model_cov(rh, ru, lam, a, st)
    _, logdet = np.linalg.slogdet(Rx)
    quad = np.real(np.einsum("ijm,ijm->ij", np.conj(x), np.linalg.solve(Rx, x[..., None])[..., 0]))
    return float(np.sum(-logdet - quad - (alpha + 1.0) * np.log(rh) - beta / rh))


RULES = ("accel2", "accel1", "naive")


def run(prob: dict, n_iter: int, rule: str = "accel2", alpha: float = 1.1, beta: float = 1e-16,
        lambda0=None, rows=None, history=None):
    """Run n_iter passes of one rule on one utterance and return the final state.

    ``prob`` holds x, a, Rp, rh0, ru0 (as produced by the input generator).
    ``rows`` restricts the run to a subset of frequency bins (rows are independent).
    ``history``: optional list that receives (rh, ru, lam) after each pass.
    """
    sel = slice(None) if rows is None else np.asarray(rows)
    x = np.asarray(prob["x"])[sel].astype(np.complex128)
    a = np.asarray(prob["a"])[sel].astype(np.complex128)
    Rp = np.asarray(prob["Rp"])[sel].astype(np.complex128)
    rh = np.asarray(prob["rh0"])[sel].astype(np.float64)
    ru = np.asarray(prob["ru0"])[sel].astype(np.float64)
    lam0 = None if lambda0 is None else np.asarray(lambda0, np.float64)[sel]
    st = setup(a, Rp, lam0)
    lam = st.lam0.copy()
    M = x.shape[-1]
    inv = invariants(x, a, st) if rule == "accel2" else None
    for _ in range(n_iter):
        if rule == "accel2":
            rh, ru, lam = iterate_accel2(rh, ru, lam, inv, st, M, alpha, beta)
        elif rule == "accel1":
            rh, ru, lam = iterate_accel1(rh, ru, lam, x, a, st, alpha, beta)
        elif rule == "naive":
            rh, ru, lam = iterate_naive(rh, ru, lam, x, a, st, alpha, beta)
        else:
            raise ValueError(rule)
        if history is not None:
            history.append((rh.copy(), ru.copy(), lam.copy()))
    h = wiener(rh, ru, lam, x, a, st)
    return dict(rh=rh, ru=ru, lam=lam, h=h, setup=st, x=x, a=a)
