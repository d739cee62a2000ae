"""The algebra the accelerated CUDA kernel evaluates, restated in FP64 numpy and
checked against the oracle's printed second-stage forms (Sec. III-C-2).

The kernel evaluates per slot (old r~_h, r~_u, lambda~):
  rho~_ax = tau_ax + sigma_ab sigma_bx / lambda~,  gamma = r~_h / (r~_u + r~_h rho~_aa)
  c = gamma rho~_ax,  Q = gamma r~_u
  r_h = (Q + |c|^2 + beta) / (alpha + 2)
  d = sigma_bx - c conj(sigma_ab),  B = Q |sigma_ab|^2 + |d|^2,  ell = B / r~_u
  A = Q tau_aa + kappa + tau_aa |c - tau_ax / tau_aa|^2
  lambda = mean_j ell,  r_u = (A + B / lambda) / M
which must equal the printed forms exactly in exact arithmetic."""
import numpy as np
import pytest

from oracle import rcscm_oracle as O
from paper_1908_01964_gb300 import synth

ALPHA, BETA = 1.1, 1e-16


def kernel_form(rh, ru, lam, inv, st, M):
    sab = st.sigma_ab[:, None]
    sab2 = np.abs(st.sigma_ab)[:, None] ** 2
    taa = st.tau_aa[:, None]
    kappa = inv.tau_xx - np.abs(inv.tau_ax) ** 2 / taa
    rtaa = taa + sab2 / lam[:, None]
    rax = inv.tau_ax + sab * inv.sigma_bx / lam[:, None]
    g = rh / (ru + rh * rtaa)
    c = g * rax
    Q = g * ru
    rh_new = (Q + np.abs(c) ** 2 + BETA) / (ALPHA + 2)
    d = inv.sigma_bx - c * np.conj(sab)
    B = Q * sab2 + np.abs(d) ** 2
    lam_new = np.mean(B / ru, axis=1)
    A = Q * taa + kappa + taa * np.abs(c - inv.tau_ax / taa) ** 2
    ru_new = (A + B / lam_new[:, None]) / M
    return rh_new, ru_new, lam_new


@pytest.mark.parametrize("M", [2, 3, 4, 8])
def test_kernel_algebra_equals_printed_second_stage_rule(M):
    p = synth.tiny(M=M, I=9, J=40, K=3, seed=100 + M)
    x = p["x"].astype(complex)
    st = O.setup(p["a"], p["Rp"])
    inv = O.invariants(x, p["a"], st)
    rh, ru, lam = p["rh0"].astype(float), p["ru0"].astype(float), st.lam0.copy()
    for _ in range(8):
        want = O.iterate_accel2(rh, ru, lam, inv, st, M, ALPHA, BETA)
        got = kernel_form(rh, ru, lam, inv, st, M)
        for u, v in zip(got, want):
            assert np.linalg.norm(u - v) < 1e-12 * np.linalg.norm(v)
            np.testing.assert_allclose(u, v, rtol=1e-8)   # elementwise: the printed r_u form cancels
        rh, ru, lam = want


def test_kernel_algebra_terms_are_non_negative():
    p = synth.tiny(M=4, I=9, J=40, K=3, seed=7)
    x = p["x"].astype(complex)
    st = O.setup(p["a"], p["Rp"])
    inv = O.invariants(x, p["a"], st)
    kappa = inv.tau_xx - np.abs(inv.tau_ax) ** 2 / st.tau_aa[:, None]
    assert np.all(kappa >= -1e-12 * inv.tau_xx)           # Cauchy-Schwarz in the R'^+ inner product


@pytest.mark.parametrize("M", [3, 4, 6, 8])
def test_kappa_fp32_bound_holds_for_any_complement_basis(M):
    # the tolerance of the invariants' kappa: an FP32 projection through an exact basis of
    # the whitened complement of a, rounded once, stays within kappa_fp32_bound in any basis
    from parity_util import kappa_fp32_bound
    p = synth.make_problem(synth.ProblemSpec(M=M, I=11, J=300, K=4, spacing=0.03), 10 + M)
    x = p["x"].astype(complex)
    a = p["a"].astype(complex)
    st = O.setup(p["a"], p["Rp"])
    inv = O.invariants(x, a, st)
    kappa = inv.tau_xx - np.abs(inv.tau_ax) ** 2 / st.tau_aa[:, None]
    bound = kappa_fp32_bound(x, a, st, kappa)
    rng = np.random.default_rng(M)
    worst = 0.0
    for i in range(x.shape[0]):
        mu, E = np.linalg.eigh(st.Rp[i])
        L = E[:, 1:] / np.sqrt(mu[1:])                       # R'^+ = L L^H
        v = L.conj().T @ a[i]
        Q, _ = np.linalg.qr(np.column_stack([v, rng.standard_normal((M - 1, M - 2))
                                             + 1j * rng.standard_normal((M - 1, M - 2))]))
        for basis in (Q[:, 1:], Q[:, 1:] @ np.linalg.qr(rng.standard_normal((M - 2, M - 2))
                                                          + 1j * rng.standard_normal((M - 2, M - 2)))[0]):
            P = (L @ basis).conj().T.astype(np.complex64)   # rows orthogonal to L^H a, FP32
            z = x[i].astype(np.complex64) @ P.T
            k32 = np.sum(z.real.astype(np.float32) ** 2 + z.imag.astype(np.float32) ** 2, axis=1, dtype=np.float32)
            err = np.abs(k32.astype(float) - kappa[i])
            assert np.all(err <= bound[i]), (i, np.max(err / bound[i]))
            worst = max(worst, float(np.max(err / inv.tau_xx[i])))
    assert worst > 1e-6                                       # the DC bin's floor is well above FP32 rounding


@pytest.mark.parametrize("M,n_h", [(2, 0), (4, 0), (4, 3), (8, 5)])
def test_ilrma_fp32_bounds_hold_for_an_fp32_evaluation(M, n_h):
    # the tolerances of the GPU initialisation from ILRMA outputs: an FP32 evaluation
    # of y = W x (W rounded once), powers and ratios stays within ilrma_fp32_bounds
    from parity_util import ilrma_fp32_bounds
    p = synth.make_problem(synth.ProblemSpec(M=M, I=9, J=300, K=6, spacing=0.03), 60 + M)
    x, W = p["x"], p["W"]
    ref = O.ilrma_init(x, W, p["T"], p["V"], n_h)
    dR, dru = ilrma_fp32_bounds(x, W, n_h)
    y = np.einsum("inm,ijm->ijn", W.astype(np.complex64), x.astype(np.complex64))
    P = (y.real.astype(np.float32) ** 2 + y.imag.astype(np.float32) ** 2).astype(np.float64)
    keep = np.ones(M)
    keep[n_h] = 0.0
    d = (P * keep).mean(axis=1)
    Winv = np.linalg.inv(W)
    Rp = np.einsum("imn,in,ikn->imk", Winv, d, np.conj(Winv))
    ru = np.sum(keep * P / np.where(keep > 0, d, 1.0)[:, None, :], axis=2) / M
    assert np.all(np.linalg.norm(Rp - ref.Rp, axis=(1, 2)) <= dR)
    assert np.all(np.abs(ru - ref.ru0) <= dru)
