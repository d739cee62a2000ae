"""Pins for the FP64 oracle: each check ties an oracle function to something
other than itself (a textbook identity, a library routine used on a different
route, brute force on tiny inputs, an invariance, or a value printed in the
paper), so that a dropped term, a wrong sign or a transposed operand fails.
CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats
from scipy.special import gammaln

from oracle import rcscm_oracle as O
from paper_1908_01964_gb300 import synth

ALPHA, BETA = 1.1, 1e-16
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prob(M=3, I=6, J=9, K=3, seed=5, **kw):
    return synth.tiny(M=M, I=I, J=J, K=K, seed=seed, **kw)


def _start(p):
    x = p["x"].astype(np.complex128)
    a = p["a"]
    st = O.setup(a, p["Rp"])
    return x, a, st, p["rh0"].astype(float), p["ru0"].astype(float), st.lam0.copy()


def _conditioning(rh, ru, Rt, a, x):
    """Generic Gaussian conditioning of z = (s, u) on x = [a | I] z.

    Prior z ~ N_c(0, blockdiag(rh, ru Rt)).  Returns E|s|^2 | x and E[u u^H | x]
    (the sufficient statistics of the E-step, Sec. II-B-2) without using the
    paper's closed forms."""
    M = a.shape[0]
    Sz = np.zeros((M + 1, M + 1), complex)
    Sz[0, 0] = rh
    Sz[1:, 1:] = ru * Rt
    H = np.concatenate([a[:, None], np.eye(M)], axis=1)
    Sx = H @ Sz @ H.conj().T
    Szx = Sz @ H.conj().T
    K = np.linalg.solve(Sx, Szx.conj().T).conj().T          # Szx Sx^{-1}
    m = K @ x
    C = Sz - K @ Szx.conj().T
    return np.real(abs(m[0]) ** 2 + C[0, 0]), np.outer(m[1:], m[1:].conj()) + C[1:, 1:], m


# ---------------------------------------------------------------- golden / paper

def test_paper_constants_and_worked_size():
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    assert synth.ALPHA == g["alpha"]["value"] and synth.BETA == g["beta"]["value"]
    assert synth.FS == g["fs_hz"]["value"]
    nfft = g["fs_hz"]["value"] * g["stft_window_ms"]["value"] // 1000
    ws = g["worked_size"]
    assert nfft // 2 + 1 == ws["I"]                      # 64 ms at 16 kHz -> I = 513
    assert ws["I"] * ws["J"] == ws["IJ"]                 # 141075 inversions per naive pass
    spec = synth.ProblemSpec(M=ws["M"], I=ws["I"], J=ws["J"])
    assert spec.nfft == nfft


# ---------------------------------------------------------------- setup

def test_setup_pinv_and_riinv_identity():
    p = _prob(M=4, I=5)
    st = O.setup(p["a"], p["Rp"])
    for i in range(5):
        Rp = st.Rp[i]
        # pseudo-inverse against numpy's SVD-based pinv
        np.testing.assert_allclose(st.Rp_pinv[i], np.linalg.pinv(Rp, rcond=1e-12), atol=1e-10 * np.abs(st.Rp_pinv[i]).max())
        # Eq. (eq:riinv): (R' + lam b b^H)^{-1} = R'^+ + b b^H / lam, for any lam > 0
        b = st.b[i]
        for lam in (st.lam0[i], 0.37, 5.0):
            lhs = np.linalg.inv(Rp + lam * np.outer(b, b.conj()))
            rhs = st.Rp_pinv[i] + np.outer(b, b.conj()) / lam
            np.testing.assert_allclose(lhs, rhs, atol=1e-10 * np.abs(lhs).max())
        # b is a unit null vector: R' b = 0, ||b|| = 1 (Sec. II-B-1)
        assert abs(np.linalg.norm(b) - 1) < 1e-12
        assert np.linalg.norm(Rp @ b) < 1e-12 * np.linalg.norm(Rp)
        # tau_aa (eq:taa), sigma_ab (eq:sap) by direct products
        a = p["a"][i]
        assert abs(st.tau_aa[i] - np.real(a.conj() @ np.linalg.pinv(Rp, rcond=1e-12) @ a)) < 1e-9 * st.tau_aa[i]
        assert abs(st.sigma_ab[i] - a.conj() @ b) < 1e-12


def test_setup_b_is_target_demixing_row():
    # R' = W^{-1} diag(p, p_nh = 0) W^{-H} annihilates w_nh (Eq. (eq:rit)), so b is parallel to it.
    p = _prob(M=4, I=7)
    st = O.setup(p["a"], p["Rp"])
    w0 = np.conj(p["W"][:, 0, :])                      # target row of W is w_0^H
    cosang = np.abs(np.einsum("im,im->i", np.conj(st.b), w0)) / np.linalg.norm(w0, axis=1)
    np.testing.assert_allclose(cosang, 1.0, atol=1e-12)


def test_setup_m2_lambda_is_trace():
    p = _prob(M=2, I=8)
    st = O.setup(p["a"], p["Rp"])
    np.testing.assert_allclose(st.lam0, np.real(np.trace(st.Rp, axis1=1, axis2=2)), rtol=1e-12)


# ---------------------------------------------------------------- E-step / identities

def test_sherman_morrison_expansion():
    # Eq. (eq:rijxinv) against an explicit inverse
    p = _prob(M=4, I=3, J=4)
    x, a, st, rh, ru, lam = _start(p)
    for i in range(3):
        Rt = st.Rp[i] + lam[i] * np.outer(st.b[i], st.b[i].conj())
        Rti = np.linalg.inv(Rt)
        for j in range(4):
            Rx = rh[i, j] * np.outer(a[i], a[i].conj()) + ru[i, j] * Rt
            sm = (Rti - rh[i, j] / (ru[i, j] + rh[i, j] * np.real(a[i].conj() @ Rti @ a[i]))
                  * Rti @ np.outer(a[i], a[i].conj()) @ Rti) / ru[i, j]
            np.testing.assert_allclose(sm, np.linalg.inv(Rx), atol=1e-11 * np.abs(sm).max())


def test_e_step_matches_gaussian_conditioning():
    p = _prob(M=3, I=4, J=5)
    x, a, st, rh, ru, lam = _start(p)
    rhat, Rhat = O.e_step_naive(rh, ru, lam, x, a, st)
    for i in range(4):
        Rt = st.Rp[i] + lam[i] * np.outer(st.b[i], st.b[i].conj())
        for j in range(5):
            r_ref, R_ref, _ = _conditioning(rh[i, j], ru[i, j], Rt, a[i], x[i, j])
            assert abs(rhat[i, j] - r_ref) < 1e-10 * abs(r_ref)
            np.testing.assert_allclose(Rhat[i, j], R_ref, atol=1e-10 * np.abs(R_ref).max())


def _inv2(A):
    """2 x 2 inverse by the adjugate formula, written out element by element."""
    det = A[0][0] * A[1][1] - A[0][1] * A[1][0]
    return [[A[1][1] / det, -A[0][1] / det], [-A[1][0] / det, A[0][0] / det]]


def test_naive_iteration_bruteforce_loops():
    """One naive EM pass for M = 2 written with scalar loops only (Sec. II-B-2)."""
    p = _prob(M=2, I=3, J=4, seed=9)
    x, a, st, rh, ru, lam = _start(p)
    ref = O.iterate_naive(rh, ru, lam, x, a, st, ALPHA, BETA)
    I, J, M = x.shape
    for i in range(I):
        b = [complex(v) for v in st.b[i]]
        av = [complex(v) for v in a[i]]
        Rt = [[complex(st.Rp[i][m][n]) + lam[i] * b[m] * b[n].conjugate() for n in range(M)] for m in range(M)]
        rh_new, ells, Rus = [], [], []
        for j in range(J):
            xv = [complex(v) for v in x[i, j]]
            Rx = [[rh[i, j] * av[m] * av[n].conjugate() + ru[i, j] * Rt[m][n] for n in range(M)] for m in range(M)]
            P = _inv2(Rx)
            aPa = sum(av[m].conjugate() * P[m][n] * av[n] for m in range(M) for n in range(M))
            xPa = sum(xv[m].conjugate() * P[m][n] * av[n] for m in range(M) for n in range(M))
            rhat = (rh[i, j] - rh[i, j] ** 2 * aPa + abs(rh[i, j] * xPa) ** 2).real
            RtP = [[sum(Rt[m][k] * P[k][n] for k in range(M)) for n in range(M)] for m in range(M)]
            RtPRt = [[sum(RtP[m][k] * Rt[k][n] for k in range(M)) for n in range(M)] for m in range(M)]
            y = [sum(RtP[m][n] * xv[n] for n in range(M)) for m in range(M)]
            Ru = [[ru[i, j] * Rt[m][n] - ru[i, j] ** 2 * RtPRt[m][n] + ru[i, j] ** 2 * y[m] * y[n].conjugate()
                   for n in range(M)] for m in range(M)]
            rh_new.append((rhat + BETA) / (ALPHA + 2))
            ells.append(sum(b[m].conjugate() * Ru[m][n] * b[n] for m in range(M) for n in range(M)).real / ru[i, j])
            Rus.append(Ru)
        lam_new = sum(ells) / J
        R = [[complex(st.Rp[i][m][n]) + lam_new * b[m] * b[n].conjugate() for n in range(M)] for m in range(M)]
        Ri = _inv2(R)
        for j in range(J):
            tr = sum(Ri[m][n] * Rus[j][n][m] for m in range(M) for n in range(M)).real
            assert abs(ref[1][i, j] - tr / M) < 1e-10 * abs(tr / M)
            assert abs(ref[0][i, j] - rh_new[j]) < 1e-10 * abs(rh_new[j])
        assert abs(ref[2][i] - lam_new) < 1e-10 * lam_new


def test_invariants_bruteforce_loops():
    p = _prob(M=3, I=2, J=3)
    x, a, st, *_ = _start(p)
    inv = O.invariants(x, a, st)
    P = st.Rp_pinv
    for i in range(2):
        for j in range(3):
            tax = sum(a[i, m].conjugate() * P[i, m, n] * x[i, j, n] for m in range(3) for n in range(3))
            txx = sum(x[i, j, m].conjugate() * P[i, m, n] * x[i, j, n] for m in range(3) for n in range(3)).real
            sbx = sum(st.b[i, m].conjugate() * x[i, j, m] for m in range(3))
            assert abs(inv.tau_ax[i, j] - tax) < 1e-12 * max(1, abs(tax))
            assert abs(inv.tau_xx[i, j] - txx) < 1e-12 * max(1, abs(txx))
            assert abs(inv.sigma_bx[i, j] - sbx) < 1e-12 * max(1, abs(sbx))


# ---------------------------------------------------------------- rule agreement (central claim)

@pytest.mark.parametrize("M", [2, 3, 4, 6])
def test_three_rules_agree(M):
    p = _prob(M=M, I=6, J=12, seed=M)
    h2, h1, hn = [], [], []
    O.run(p, 15, "accel2", history=h2)
    O.run(p, 15, "accel1", history=h1)
    O.run(p, 15, "naive", history=hn)
    for k in range(15):
        for q in range(3):
            ref = hn[k][q]
            for other in (h1, h2):
                err = np.linalg.norm(other[k][q] - ref) / np.linalg.norm(ref)
                assert err < 1e-10, (k, q, err)


# ---------------------------------------------------------------- M-step stationarity

def _q_slot(rh, ru, lam, rhat, Rhat, Rp, b, M):
    """One slot's term of the Q function (Sec. II-B-2), constants dropped."""
    R = Rp + lam * np.outer(b, b.conj())
    _, logdet = np.linalg.slogdet(R)
    return (-(ALPHA + 2) * np.log(rh) - (rhat + BETA) / rh - M * np.log(ru) - logdet
            - np.real(np.trace(np.linalg.solve(R, Rhat))) / ru)


def test_m_step_is_stationary_point_of_q():
    p = _prob(M=3, I=3, J=6, seed=21)
    x, a, st, rh, ru, lam = _start(p)
    I, J, M = x.shape
    inv = O.invariants(x, a, st)
    rh1, ru1, lam1 = O.iterate_accel2(rh, ru, lam, inv, st, M, ALPHA, BETA)
    for i in range(I):
        Rt = st.Rp[i] + lam[i] * np.outer(st.b[i], st.b[i].conj())
        stats_ = [_conditioning(rh[i, j], ru[i, j], Rt, a[i], x[i, j])[:2] for j in range(J)]
        # d/d lambda at r_u = r~_u (the lambda step conditions on the old r_u)
        def q_lam(l):
            return sum(_q_slot(rh1[i, j], ru[i, j], l, *stats_[j], st.Rp[i], st.b[i], M) for j in range(J))
        h = 1e-6 * lam1[i]
        g = (q_lam(lam1[i] + h) - q_lam(lam1[i] - h)) / (2 * h)
        scale = abs(q_lam(lam1[i])) / lam1[i]
        assert abs(g) < 1e-5 * scale, (i, g, scale)
        for j in range(J):
            def q_rh(r):
                return _q_slot(r, ru1[i, j], lam1[i], *stats_[j], st.Rp[i], st.b[i], M)

            def q_ru(r):
                return _q_slot(rh1[i, j], r, lam1[i], *stats_[j], st.Rp[i], st.b[i], M)
            for fn, v in ((q_rh, rh1[i, j]), (q_ru, ru1[i, j])):
                h = 1e-5 * v
                g = (fn(v + h) - fn(v - h)) / (2 * h)
                assert abs(g) * v < 1e-5 * (1 + abs(fn(v))), (i, j, g)


def test_m_step_moves_off_stationarity_when_mutated():
    """A planted mistake (r_u without the 1/M) breaks the stationarity check."""
    p = _prob(M=3, I=2, J=5, seed=21)
    x, a, st, rh, ru, lam = _start(p)
    M = 3
    inv = O.invariants(x, a, st)
    rh1, ru1, lam1 = O.iterate_accel2(rh, ru, lam, inv, st, M, ALPHA, BETA)
    bad = ru1 * M
    Rt = st.Rp[0] + lam[0] * np.outer(st.b[0], st.b[0].conj())
    s = _conditioning(rh[0, 0], ru[0, 0], Rt, a[0], x[0, 0])[:2]

    def q_ru(r):
        return _q_slot(rh1[0, 0], r, lam1[0], *s, st.Rp[0], st.b[0], M)
    v = bad[0, 0]
    g = (q_ru(v * (1 + 1e-5)) - q_ru(v * (1 - 1e-5))) / (2e-5 * v)
    assert abs(g) * v > 1e-3


# ---------------------------------------------------------------- objective

def _complex_gauss_logpdf(x, R):
    """log N_c(x; 0, R) through scipy's real 2M-dimensional normal."""
    M = x.shape[0]
    Rr = 0.5 * np.block([[R.real, -R.imag], [R.imag, R.real]])
    return stats.multivariate_normal(mean=np.zeros(2 * M), cov=Rr).logpdf(np.concatenate([x.real, x.imag]))


def test_objective_equals_library_log_densities():
    p = _prob(M=3, I=2, J=3, seed=4)
    x, a, st, rh, ru, lam = _start(p)
    I, J, M = x.shape
    ours = O.objective(rh, ru, lam, x, a, st, ALPHA, BETA)
    Rx = O.model_cov(rh, ru, lam, a, st)
    lib = 0.0
    for i in range(I):
        for j in range(J):
            lib += _complex_gauss_logpdf(x[i, j], Rx[i, j])
            lib += stats.invgamma(ALPHA, scale=BETA).logpdf(rh[i, j])
    # the constants the oracle drops, per slot: -M log(pi) from the complex Gaussian
    # density and alpha log(beta) - log Gamma(alpha) from the inverse-gamma density
    const = I * J * (-M * math.log(math.pi) + ALPHA * math.log(BETA) - gammaln(ALPHA))
    assert abs((lib - const) - ours) < 1e-9 * abs(ours)


def test_objective_closed_form():
    # log det R_x = M log r_u + log lam + log pdet R' + log(1 + r_h rho_aa / r_u), and
    # x^H R_x^{-1} x = (rho_xx - r_h |rho_ax|^2 / (r_u + r_h rho_aa)) / r_u
    p = _prob(M=4, I=3, J=5, seed=8)
    x, a, st, rh, ru, lam = _start(p)
    inv = O.invariants(x, a, st)
    sab2 = np.abs(st.sigma_ab) ** 2
    rho_aa = st.tau_aa + sab2 / lam
    rho_ax = inv.tau_ax + st.sigma_ab[:, None] * inv.sigma_bx / lam[:, None]
    rho_xx = inv.tau_xx + np.abs(inv.sigma_bx) ** 2 / lam[:, None]
    logpdet = np.sum(np.log(st.mu[:, 1:]), axis=1)
    ld = 4 * np.log(ru) + (np.log(lam) + logpdet)[:, None] + np.log1p(rh * rho_aa[:, None] / ru)
    qd = (rho_xx - rh * np.abs(rho_ax) ** 2 / (ru + rh * rho_aa[:, None])) / ru
    closed = np.sum(-ld - qd - (ALPHA + 1) * np.log(rh) - BETA / rh)
    assert abs(closed - O.objective(rh, ru, lam, x, a, st, ALPHA, BETA)) < 1e-9 * abs(closed)


@pytest.mark.parametrize("rule", O.RULES)
def test_objective_monotone_and_model_pd(rule):
    p = _prob(M=4, I=5, J=20, seed=13)
    x, a, st, rh, ru, lam = _start(p)
    hist = []
    O.run(p, 25, rule, history=hist)
    objs = [O.objective(rh, ru, lam, x, a, st, ALPHA, BETA)]
    for rh_k, ru_k, lam_k in hist:
        objs.append(O.objective(rh_k, ru_k, lam_k, x, a, st, ALPHA, BETA))
        Rx = O.model_cov(rh_k, ru_k, lam_k, a, st)
        np.testing.assert_allclose(Rx, np.conj(np.swapaxes(Rx, -1, -2)), atol=1e-12 * np.abs(Rx).max())
        assert np.linalg.eigvalsh(Rx).min() > 0
    d = np.diff(objs)
    assert np.all(d >= -1e-12 * np.abs(objs[1:])), d


# ---------------------------------------------------------------- Wiener filter

def test_wiener_is_posterior_mean_and_closed_form():
    p = _prob(M=3, I=3, J=4, seed=17)
    x, a, st, rh, ru, lam = _start(p)
    h = O.wiener(rh, ru, lam, x, a, st)
    inv = O.invariants(x, a, st)
    sab2 = np.abs(st.sigma_ab) ** 2
    rho_aa = st.tau_aa + sab2 / lam
    rho_ax = inv.tau_ax + st.sigma_ab[:, None] * inv.sigma_bx / lam[:, None]
    w = rh * rho_ax / (ru + rh * rho_aa[:, None])
    np.testing.assert_allclose(h, w[..., None] * a[:, None, :], atol=1e-12 * np.abs(h).max())
    for i in range(3):
        R = st.Rp[i] + lam[i] * np.outer(st.b[i], st.b[i].conj())
        for j in range(4):
            m = _conditioning(rh[i, j], ru[i, j], R, a[i], x[i, j])[2]
            np.testing.assert_allclose(h[i, j], m[0] * a[i], atol=1e-11 * np.abs(h[i, j]).max())


# ---------------------------------------------------------------- invariances

def test_b_phase_invariance():
    p = _prob(M=4, I=4, J=8, seed=2)
    r0 = O.run(p, 6, "accel2")
    st = O.setup(p["a"], p["Rp"])
    x, a = p["x"].astype(complex), p["a"]
    st.b = st.b * np.exp(1j * np.linspace(0.3, 2.0, 4))[:, None]
    st.sigma_ab = np.einsum("im,im->i", np.conj(a), st.b)
    inv = O.invariants(x, a, st)
    rh, ru, lam = p["rh0"].astype(float), p["ru0"].astype(float), st.lam0.copy()
    for _ in range(6):
        rh, ru, lam = O.iterate_accel2(rh, ru, lam, inv, st, 4, ALPHA, BETA)
    for u, v in ((rh, r0["rh"]), (ru, r0["ru"]), (lam, r0["lam"])):
        np.testing.assert_allclose(u, v, rtol=1e-10)
    np.testing.assert_allclose(O.wiener(rh, ru, lam, x, a, st), r0["h"], atol=1e-10 * np.abs(r0["h"]).max())


def test_rows_are_independent():
    p = _prob(M=3, I=8, J=10, seed=6)
    full = O.run(p, 7, "accel2")
    rows = [1, 4, 6]
    sub = O.run(p, 7, "accel2", rows=rows)
    for k in ("rh", "ru", "lam"):
        np.testing.assert_allclose(sub[k], full[k][rows], rtol=1e-13)


def test_scale_equivariance_beta_zero():
    # With beta = 0: (x, R', lam, r_h, r_u) -> (c x, |c|^2 R', |c|^2 lam, |c|^2 r_h, r_u) maps h -> c h.
    p = _prob(M=3, I=4, J=6, seed=12)
    c = 1.7 - 0.4j
    q = dict(p)
    q["x"] = p["x"].astype(np.complex128) * c
    q["Rp"] = p["Rp"] * abs(c) ** 2
    q["rh0"] = p["rh0"].astype(float) * abs(c) ** 2
    q["ru0"] = p["ru0"].astype(float)
    r1 = O.run(p, 5, "accel2", beta=0.0)
    r2 = O.run(q, 5, "accel2", beta=0.0)
    np.testing.assert_allclose(r2["h"], c * r1["h"], atol=1e-10 * np.abs(r2["h"]).max())
    np.testing.assert_allclose(r2["rh"], abs(c) ** 2 * r1["rh"], rtol=1e-10)
    np.testing.assert_allclose(r2["ru"], r1["ru"], rtol=1e-10)
    np.testing.assert_allclose(r2["lam"], abs(c) ** 2 * r1["lam"], rtol=1e-10)


# ---------------------------------------------------------------- planted mistakes

@pytest.mark.parametrize("mutant", ["drop_gamma_term_in_lambda", "stale_lambda_in_ru", "conj_sigma_ab"])
def test_planted_mistakes_break_rule_agreement(mutant, monkeypatch):
    """Mistakes planted in the oracle's second-stage rule are caught by naive agreement."""
    orig = O.iterate_accel2

    def bad(rh, ru, lam, inv, st, M, alpha, beta):
        if mutant == "drop_gamma_term_in_lambda":
            rh2, ru2, lam2 = orig(rh, ru, lam, inv, st, M, alpha, beta)
            sab = st.sigma_ab[:, None]
            rho_aa_t = st.tau_aa + np.abs(st.sigma_ab) ** 2 / lam
            rho_ax_t = inv.tau_ax + sab * inv.sigma_bx / lam[:, None]
            g = rh / (ru + rh * rho_aa_t[:, None])
            lam2 = np.mean(np.abs(inv.sigma_bx - g * np.conj(sab) * rho_ax_t) ** 2 / ru, axis=1)
            return rh2, ru2, lam2
        if mutant == "stale_lambda_in_ru":
            rh2, _, lam2 = orig(rh, ru, lam, inv, st, M, alpha, beta)
            # recompute r_u with the OLD lambda
            sab = st.sigma_ab[:, None]
            sab2 = np.abs(st.sigma_ab) ** 2
            rho_aa_t = st.tau_aa + sab2 / lam
            rho_ax_t = inv.tau_ax + sab * inv.sigma_bx / lam[:, None]
            g = rh / (ru + rh * rho_aa_t[:, None])
            rho_xx = inv.tau_xx + np.abs(inv.sigma_bx) ** 2 / lam[:, None]
            ru2 = (g * rho_aa_t[:, None] * (ru + g * np.abs(rho_ax_t) ** 2) + rho_xx
                   - 2 * g * np.abs(rho_ax_t) ** 2) / M
            return rh2, ru2, lam2
        st2 = O.Setup(**{**st.__dict__, "sigma_ab": np.conj(st.sigma_ab)})
        return orig(rh, ru, lam, inv, st2, M, alpha, beta)

    monkeypatch.setattr(O, "iterate_accel2", bad)
    p = _prob(M=3, I=4, J=10, seed=31)
    h2, hn = [], []
    O.run(p, 3, "accel2", history=h2)
    O.run(p, 3, "naive", history=hn)
    worst = max(np.linalg.norm(h2[k][q] - hn[k][q]) / np.linalg.norm(hn[k][q]) for k in range(3) for q in range(3))
    assert worst > 1e-6
