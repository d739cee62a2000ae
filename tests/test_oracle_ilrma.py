"""Pins of oracle.ilrma_init, the estimator's inputs from the ILRMA stage
(Sec. II-A: W_i = A_i^{-1}; Sec. II-B-1: Eq. (eq:rit); Sec. II-B-3: Eqs.
(eq:rhinit), (eq:ruinit)).  Each pin is independent of the oracle's code: plain
loops with an explicit (Cramer) inverse on tiny inputs, a noise-free mixture
whose sources and mixing matrix are known, the closed form of Eq. (eq:ruinit)
for a back-projected rank-(M-1) SCM, and the scale invariance of
back-projection."""
import itertools

import numpy as np
import pytest

from oracle import rcscm_oracle as O


def _cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _det(A):
    # Leibniz formula (tiny M only)
    M = A.shape[0]
    total = 0j
    for perm in itertools.permutations(range(M)):
        sign = 1
        for p in range(M):
            for q in range(p + 1, M):
                if perm[p] > perm[q]:
                    sign = -sign
        prod = 1 + 0j
        for r in range(M):
            prod *= A[r, perm[r]]
        total += sign * prod
    return total


def _inv_cramer(A):
    M = A.shape[0]
    d = _det(A)
    out = np.zeros((M, M), complex)
    for r in range(M):
        for c in range(M):
            minor = np.delete(np.delete(A, c, axis=0), r, axis=1)
            out[r, c] = (-1) ** (r + c) * (_det(minor) if M > 1 else 1.0) / d
    return out


@pytest.mark.parametrize("M,n_h", [(2, 0), (3, 1), (3, 2)])
def test_ilrma_init_equals_loops_on_tiny_inputs(M, n_h):
    rng = np.random.default_rng(10 * M + n_h)
    I, J, K = 2, 5, 3
    x = _cplx(rng, I, J, M)
    W = _cplx(rng, I, M, M)
    T = rng.gamma(1.0, 1.0, (I, K))
    V = rng.gamma(1.0, 1.0, (K, J))
    got = O.ilrma_init(x, W, T, V, n_h)
    for i in range(I):
        A = _inv_cramer(W[i])
        np.testing.assert_allclose(got.a[i], A[:, n_h], rtol=1e-12, atol=1e-12)
        Rp = np.zeros((M, M), complex)
        for j in range(J):
            for n in range(M):
                if n == n_h:
                    continue
                yn = sum(W[i, n, m] * x[i, j, m] for m in range(M))     # row n of W is w_n^H
                for r in range(M):
                    for c in range(M):
                        Rp[r, c] += abs(yn) ** 2 * A[r, n] * np.conj(A[c, n]) / J
        np.testing.assert_allclose(got.Rp[i], Rp, rtol=1e-12, atol=1e-12)
        Rp_pinv = np.linalg.pinv(Rp, hermitian=True, rcond=1e-10)      # rank M-1: the zero eigenvalue dropped
        for j in range(J):
            rh = sum(T[i, k] * V[k, j] for k in range(K))
            assert abs(got.rh0[i, j] - rh) <= 1e-12 * rh
            yu = np.zeros(M, complex)
            for n in range(M):
                if n != n_h:
                    yu += sum(W[i, n, m] * x[i, j, m] for m in range(M)) * A[:, n]
            ru = np.real(np.conj(yu) @ Rp_pinv @ yu) / M
            assert abs(got.ru0[i, j] - ru) <= 1e-9 * ru


@pytest.mark.parametrize("M,n_h", [(2, 1), (4, 0), (6, 3)])
def test_noise_free_mixture_gives_the_sum_of_the_noise_outputs(M, n_h):
    # x = A s with W = A^{-1}: y = s, so R' is the power-weighted sum of the other
    # columns of A (Sec. II-A), a is A's target column and the null vector of R'
    # is the target row w_{n_h} of W
    rng = np.random.default_rng(M + 7 * n_h)
    I, J = 3, 40
    A = _cplx(rng, I, M, M)
    s = _cplx(rng, I, J, M)
    x = np.einsum("imn,ijn->ijm", A, s)
    W = np.linalg.inv(A)
    got = O.ilrma_init(x, W, np.ones((I, 1)), np.ones((1, J)), n_h)
    for i in range(I):
        want = sum(np.mean(np.abs(s[i, :, n]) ** 2) * np.outer(A[i, :, n], np.conj(A[i, :, n]))
                   for n in range(M) if n != n_h)
        np.testing.assert_allclose(got.Rp[i], want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
        np.testing.assert_allclose(got.a[i], A[i, :, n_h], rtol=1e-9)
        w = np.conj(W[i, n_h])                                   # the vector w_{n_h}
        assert np.linalg.norm(got.Rp[i] @ w) <= 1e-9 * np.linalg.norm(got.Rp[i]) * np.linalg.norm(w)
        assert np.linalg.matrix_rank(got.Rp[i], tol=1e-8 * np.abs(got.Rp[i]).max()) == M - 1
        d = [np.mean(np.abs(s[i, :, n]) ** 2) for n in range(M)]
        ru = sum(np.abs(s[i, :, n]) ** 2 / d[n] for n in range(M) if n != n_h) / M
        np.testing.assert_allclose(got.ru0[i], ru, rtol=1e-9)


@pytest.mark.parametrize("M,n_h", [(3, 0), (4, 2), (8, 5)])
def test_ruinit_closed_form(M, n_h):
    # with R' = sum_{n != n_h} d_n q_n q_n^H (q_n the columns of W^{-1}, d_n the mean
    # output powers), y^H R'^+ y = sum_{n != n_h} |w_n^H x|^2 / d_n
    rng = np.random.default_rng(M * 3 + n_h)
    I, J = 4, 30
    x = _cplx(rng, I, J, M)
    W = _cplx(rng, I, M, M)
    got = O.ilrma_init(x, W, np.ones((I, 1)), np.ones((1, J)), n_h)
    y = np.einsum("inm,ijm->ijn", W, x)
    d = np.mean(np.abs(y) ** 2, axis=1)
    terms = np.abs(y) ** 2 / d[:, None, :]
    terms[:, :, n_h] = 0.0
    np.testing.assert_allclose(got.ru0, terms.sum(axis=2) / M, rtol=1e-8)


def test_back_projection_is_scale_invariant():
    # ILRMA fixes W only up to a per-output scale: W -> diag(g) W leaves the
    # back-projected R' and r_u0 unchanged (the reason for back-projection)
    rng = np.random.default_rng(3)
    I, J, M = 3, 25, 4
    x = _cplx(rng, I, J, M)
    W = _cplx(rng, I, M, M)
    g = _cplx(rng, I, M)
    ref = O.ilrma_init(x, W, np.ones((I, 1)), np.ones((1, J)), 1)
    got = O.ilrma_init(x, g[:, :, None] * W, np.ones((I, 1)), np.ones((1, J)), 1)
    np.testing.assert_allclose(got.Rp, ref.Rp, rtol=1e-10, atol=1e-12 * np.abs(ref.Rp).max())
    np.testing.assert_allclose(got.ru0, ref.ru0, rtol=1e-9)
    np.testing.assert_allclose(got.a * g[:, 1:2], ref.a, rtol=1e-10)


def test_ruinit_at_full_size_rows_equals_the_closed_form():
    # at some rows of the single-utterance workload (M = 4, I = 1025, J = 1000) the null
    # eigenvalue of R' rounds to about 1.2e-15 of the largest (row 700), above a relative
    # pseudo-inverse cutoff of M eps; (R')^+ must still drop it (R' has rank M-1)
    from paper_1908_01964_gb300 import synth
    p = synth.make_workload(synth.workload("single-m4"))[0]
    rows = np.array([0, 1, 300, 699, 700, 701, 1024])
    got = O.ilrma_init(p["x"][rows], p["W"][rows], p["T"][rows], p["V"], 0)
    y = np.einsum("inm,ijm->ijn", p["W"][rows], p["x"][rows].astype(complex))
    d = np.mean(np.abs(y) ** 2, axis=1)
    cf = (np.abs(y[:, :, 1:]) ** 2 / d[:, None, 1:]).sum(axis=2) / 4
    np.testing.assert_allclose(got.ru0, cf, rtol=1e-8)
