"""Pins of the front-end oracle (oracle/ilrma_oracle.py): the STFT against the
DFT written as loops, perfect reconstruction of the inverse STFT, the sphering,
and the ILRMA updates against what their definitions fix -- the cost never
increases, the IP update is the exact minimiser over its row (brute force),
the NMF updates leave a stationary point unchanged, the scale normalisation
leaves the cost unchanged, and a noise-free determined mixture is separated.
CPU only."""
import numpy as np
import pytest

from oracle import ilrma_oracle as F
from paper_1908_01964_gb300 import synth


# ----------------------------------------------------------------------------- STFT

def test_stft_equals_dft_loops():
    rng = np.random.default_rng(0)
    sig = rng.standard_normal((2, 45))
    n_fft, shift = 16, 8
    X = F.stft(sig, n_fft, shift)
    I, J, M = X.shape
    assert (I, M) == (9, 2) and J == 1 + -(-(45 - 16) // 8)
    for m in range(M):
        for j in range(J):
            for i in range(I):
                acc = 0j
                for n in range(n_fft):
                    t = j * shift + n
                    v = sig[m, t] if t < 45 else 0.0
                    w = 0.54 - 0.46 * np.cos(2 * np.pi * n / n_fft)
                    acc += w * v * np.exp(-2j * np.pi * i * n / n_fft)
                assert abs(X[i, j, m] - acc) < 1e-12


@pytest.mark.parametrize("n_fft,shift,T", [(64, 32, 1000), (64, 16, 777), (1024, 512, 16000), (32, 32, 100)])
def test_istft_inverts_stft(n_fft, shift, T):
    sig = np.random.default_rng(n_fft + shift).standard_normal((3, T))
    X = F.stft(sig, n_fft, shift)
    back = F.istft(X, n_fft, shift, T)
    assert np.max(np.abs(back - sig)) < 1e-12 * np.max(np.abs(sig)) * n_fft


def test_istft_is_least_squares_for_modified_spectra():
    # for an arbitrary X (not an STFT of anything) the output is the signal whose STFT
    # is closest to X: the residual X - STFT(istft(X)) is orthogonal to every STFT
    rng = np.random.default_rng(5)
    n_fft, shift, T = 32, 16, 200
    J = F.n_frames(T, n_fft, shift)
    L = (J - 1) * shift + n_fft
    X = rng.standard_normal((17, J, 1)) + 1j * rng.standard_normal((17, J, 1))
    X[0].imag = 0
    X[-1].imag = 0
    y = F.istft(X, n_fft, shift, L)
    res = X - F.stft(y, n_fft, shift)
    for _ in range(5):
        z = rng.standard_normal((1, L))
        Z = F.stft(z, n_fft, shift)
        # real inner product of one-sided spectra, weighting the bins that stand for two
        wts = np.full(17, 2.0)
        wts[0] = wts[-1] = 1.0
        ip = np.sum(wts[:, None, None] * np.real(np.conj(res) * Z))
        assert abs(ip) < 1e-9 * np.linalg.norm(X) * np.linalg.norm(Z)


def test_hamming_window_values():
    w = F.hamming(8)
    np.testing.assert_allclose(w[[0, 2, 4]], [0.08, 0.54, 1.0], atol=1e-15)


# ----------------------------------------------------------------------------- sphering

def test_sphering_whitens_in_descending_order():
    b = synth.make_bss_mixture(4, 7, 300, 3, 11)
    X = b["x"].astype(np.complex128)
    Q = F.sphering(X)
    Xs = np.einsum("imn,ijn->ijm", Q, X)
    C = np.einsum("ijm,ijn->imn", Xs, np.conj(Xs)) / X.shape[1]
    np.testing.assert_allclose(C, np.broadcast_to(np.eye(4), C.shape), atol=1e-10)
    # row k of Q is e_k^H / sqrt(mu_k) with mu descending: row norms ascending
    nrm = np.linalg.norm(Q, axis=2)
    assert np.all(np.diff(nrm, axis=1) >= -1e-12)


# ----------------------------------------------------------------------------- ILRMA updates

def _state(M=3, I=6, J=40, K=3, seed=21):
    b = synth.make_bss_mixture(M, I, J, K, seed)
    X = b["x"].astype(np.complex128)
    Q = F.sphering(X)
    Xs = np.einsum("imn,ijn->ijm", Q, X)
    rng = np.random.default_rng(seed)
    W = np.eye(M)[None] + 0.3 * (rng.standard_normal((I, M, M)) + 1j * rng.standard_normal((I, M, M)))
    return Xs, W, b["T0"].copy(), b["V0"].copy()


def test_each_update_does_not_increase_the_cost():
    Xs, W, T, V = _state()
    N = W.shape[1]
    c = F.cost(Xs, W, T, V)
    for _ in range(5):
        for n in range(N):
            P = np.abs(np.einsum("inm,ijm->ijn", W, Xs)) ** 2
            F.update_T(P, T, V, n)
            c1 = F.cost(Xs, W, T, V)
            F.update_V(P, T, V, n)
            c2 = F.cost(Xs, W, T, V)
            F.update_w(Xs, W, T, V, n)
            c3 = F.cost(Xs, W, T, V)
            for a, b in ((c, c1), (c1, c2), (c2, c3)):
                assert b <= a + 1e-9 * abs(a)
            c = c3
        F.normalise(Xs, W, T)
        c4 = F.cost(Xs, W, T, V)
        assert abs(c4 - c) <= 1e-9 * abs(c)           # the scale normalisation changes nothing
        c = c4


def test_iteration_cost_is_monotone_over_a_run():
    b = synth.make_bss_mixture(4, 9, 120, 4, 31)
    hist = []
    F.ilrma(b["x"], b["T0"], b["V0"], 40, history=hist)
    d = np.diff(hist)
    assert np.all(d <= 1e-9 * np.abs(np.array(hist[1:])))


@pytest.mark.parametrize("n", [0, 1, 2])
def test_ip_update_is_the_minimiser_of_its_row(n):
    """With the source models and the other rows fixed the cost is a function of w_n
    alone, and the IP update minimises it: no perturbation of the updated row,
    large or small, does better (brute force)."""
    Xs, W, T, V = _state(seed=40 + n)
    F.update_w(Xs, W, T, V, n)
    c0 = F.cost(Xs, W, T, V)
    rng = np.random.default_rng(n)
    for scale in (1e-3, 1e-2, 1e-1, 1.0):
        for _ in range(20):
            W2 = W.copy()
            W2[:, n, :] += scale * (rng.standard_normal(W[:, n, :].shape) + 1j * rng.standard_normal(W[:, n, :].shape))
            assert F.cost(Xs, W2, T, V) >= c0 - 1e-10 * abs(c0)


def test_nmf_updates_fix_a_stationary_point():
    # |y|^2 = r exactly makes the gradient of the cost in T and V vanish; the
    # multiplicative updates must then leave T and V unchanged
    rng = np.random.default_rng(3)
    N, I, K, J = 2, 5, 3, 11
    T = rng.uniform(0.5, 2.0, (N, I, K))
    V = rng.uniform(0.5, 2.0, (N, K, J))
    P = np.einsum("nik,nkj->ijn", T, V)
    T1, V1 = T.copy(), V.copy()
    for n in range(N):
        F.update_T(P, T1, V1, n)
        F.update_V(P, T1, V1, n)
    np.testing.assert_allclose(T1, T, rtol=1e-13)
    np.testing.assert_allclose(V1, V, rtol=1e-13)


def test_nmf_update_moves_towards_the_data():
    # if every |y|^2 is scaled by c, one T update scales T by exactly sqrt(c)
    rng = np.random.default_rng(4)
    T = rng.uniform(0.5, 2.0, (1, 4, 2))
    V = rng.uniform(0.5, 2.0, (1, 2, 9))
    P = 4.0 * np.einsum("nik,nkj->ijn", T, V)
    T1 = T.copy()
    F.update_T(P, T1, V, 0)
    np.testing.assert_allclose(T1, 2.0 * T, rtol=1e-13)


def test_ilrma_separates_a_noise_free_determined_mixture():
    M = 3
    b = synth.make_bss_mixture(M, 17, 400, 3, 55)
    res = F.ilrma(b["x"], b["T0"], b["V0"], 60)
    G = np.einsum("imn,ink->imk", res.W, b["A"])          # global system W A per frequency
    P = np.abs(G) ** 2
    sir = 10 * np.log10(P.max(axis=2) / (P.sum(axis=2) - P.max(axis=2)))   # per output
    assert np.median(sir) > 20.0, np.median(sir)
