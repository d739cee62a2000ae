"""FP64 CPU oracle of the front end that feeds rank-constrained SCM estimation:
STFT / inverse STFT and ILRMA (independent low-rank matrix analysis).

TEST INFRASTRUCTURE ONLY, like rcscm_oracle.py: imported by the tests, by the
smoke check and by bench.py's CPU-baseline leg, never by the product path, and
sharing no code with the CUDA path (numpy complex128 / float64).

The paper (Sec. II-A, Sec. IV-A, Table II) runs ILRMA before the estimator and
fixes its settings but does not print its update rules: sampling frequency
16 kHz, STFT with a 64 ms Hamming window and a 32 ms shift, K = 10 NMF bases
per source, 50 iterations, the observation sphered by principal component
analysis, the demixing matrix initialised to the identity and the NMF
variables to non-negative random values.  The updates below are those of the
published ILRMA algorithm (Kitamura, Ono, Sawada, Kameoka, Saruwatari, IEEE/ACM
TASLP 24(9), 2016), written here from their definition:

  model      y_ijn = w_in^H x_ij,  y_ijn ~ N_c(0, r_ijn),  r_ijn = sum_k t_ikn v_kjn
  cost       L = sum_ijn (|y_ijn|^2 / r_ijn + log r_ijn) - 2 J sum_i log |det W_i|
  NMF (MM)   t_ikn <- t_ikn sqrt( sum_j |y_ijn|^2 v_kjn / r_ijn^2 / sum_j v_kjn / r_ijn )
             v_kjn <- v_kjn sqrt( sum_i |y_ijn|^2 t_ikn / r_ijn^2 / sum_i t_ikn / r_ijn )
  IP         U_in = (1/J) sum_j x_ij x_ij^H / r_ijn
             w_in <- (W_i U_in)^{-1} e_n,  w_in <- w_in / sqrt(w_in^H U_in w_in)
  scale      lambda_n = sqrt( (1/(IJ)) sum_ij |y_ijn|^2 ):  w_in <- w_in / lambda_n,
             t_ikn <- t_ikn / lambda_n^2 (leaves L unchanged up to a constant)

Each update does not increase L (majorisation-minimisation); the tests pin
this, and brute-force minimality of each update, on small inputs.  Readings
where the paper is silent (listed in the design notes): the window is the
periodic Hamming window w[n] = 0.54 - 0.46 cos(2 pi n / N), frames start at
j * shift from the first sample with zeros after the end; the inverse is the
least-squares overlap-add (each output sample is sum_j w y_j / sum_j w^2); the
sphering keeps all M principal components (N = M), in descending order of
their variance; within an iteration source n's T, then V, then w_n are
updated, for n = 0..N-1, then the scales are normalised; T and V are floored at
NMF_FLOOR after each update, as published implementations do, so that every
r_ijn stays positive where the separation is exact (a floor that binds can
raise the cost by a rounding-level amount).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


# ----------------------------------------------------------------------------- STFT

def hamming(n_fft: int) -> np.ndarray:
    """Periodic Hamming window of length n_fft (Table II: Hamming)."""
    n = np.arange(n_fft)
    return 0.54 - 0.46 * np.cos(2.0 * np.pi * n / n_fft)


def n_frames(n_samples: int, n_fft: int, shift: int) -> int:
    """Frames that cover n_samples with frames starting at j * shift (at least one)."""
    if n_samples <= n_fft:
        return 1
    return 1 + -(-(n_samples - n_fft) // shift)


def stft(sig, n_fft: int, shift: int):
    """STFT of a multichannel signal sig [M, T] (real) -> X [I, J, M] complex, I = n_fft/2 + 1:
    X[i, j, m] = sum_n w[n] sig[m, j shift + n] exp(-2 pi i i n / n_fft) (zeros past the end)."""
    sig = np.asarray(sig, np.float64)
    M, T = sig.shape
    J = n_frames(T, n_fft, shift)
    pad = np.zeros((M, (J - 1) * shift + n_fft))
    pad[:, :T] = sig
    w = hamming(n_fft)
    idx = np.arange(J)[:, None] * shift + np.arange(n_fft)[None, :]
    frames = pad[:, idx] * w                                        # [M, J, n_fft]
    X = np.fft.rfft(frames, axis=-1)                                # [M, J, I]
    return np.transpose(X, (2, 1, 0)).copy()


def istft(X, n_fft: int, shift: int, n_samples: int):
    """Least-squares inverse of stft(): every frame is inverse-transformed, windowed and
    overlap-added, and each sample is divided by the sum of the squared windows that
    cover it.  X [I, J, M] -> sig [M, n_samples]."""
    X = np.asarray(X, np.complex128)
    I, J, M = X.shape
    w = hamming(n_fft)
    frames = np.fft.irfft(np.transpose(X, (2, 1, 0)), n=n_fft, axis=-1) * w   # [M, J, n_fft]
    L = (J - 1) * shift + n_fft
    out = np.zeros((M, L))
    den = np.zeros(L)
    for j in range(J):
        out[:, j * shift:j * shift + n_fft] += frames[:, j]
        den[j * shift:j * shift + n_fft] += w ** 2
    return (out / np.where(den > 0, den, 1.0))[:, :n_samples]


# ----------------------------------------------------------------------------- ILRMA

def sphering(X):
    """Principal component sphering per frequency (Sec. IV-A): C_i = (1/J) sum_j x x^H =
    E diag(mu) E^H, Q_i = diag(mu)^{-1/2} E^H with the eigenvalues in descending order,
    so (1/J) sum_j (Q_i x)(Q_i x)^H = I.  Returns Q [I, M, M]."""
    X = np.asarray(X, np.complex128)
    J = X.shape[1]
    C = np.einsum("ijm,ijn->imn", X, np.conj(X)) / J
    mu, E = np.linalg.eigh(0.5 * (C + np.conj(np.transpose(C, (0, 2, 1)))))
    mu, E = mu[:, ::-1], E[:, :, ::-1]                              # descending
    return np.conj(np.transpose(E, (0, 2, 1))) / np.sqrt(mu)[:, :, None]


def cost(Xs, W, T, V):
    """ILRMA negative log-likelihood (constants dropped) of the sphered observation
    Xs [I, J, M], demixing W [I, N, N] (row n = w_n^H), bases T [N, I, K], activations
    V [N, K, J]."""
    Y = np.einsum("inm,ijm->ijn", W, Xs)
    R = np.einsum("nik,nkj->ijn", T, V)
    J = Xs.shape[1]
    logdet = np.log(np.abs(np.linalg.det(W)))
    return float(np.sum(np.abs(Y) ** 2 / R + np.log(R)) - 2.0 * J * np.sum(logdet))


# Floor of the NMF variables after each update: where the separation is exact some
# |y|^2 vanish and the multiplicative updates would drive t, v (and so r) to zero.
# With the scale normalisation keeping the mean output power at 1, t, v >= 1e-6 keeps
# r >= 1e-12 and 1 / r^2 within the range of single precision.
NMF_FLOOR = 1e-6


def update_T(P, T, V, n):
    """Multiplicative update of source n's bases (in place); P = |y|^2 [I, J, N]."""
    R = T[n] @ V[n]
    T[n] = np.maximum(T[n] * np.sqrt(((P[:, :, n] / R ** 2) @ V[n].T) / ((1.0 / R) @ V[n].T)), NMF_FLOOR)


def update_V(P, T, V, n):
    """Multiplicative update of source n's activations (in place)."""
    R = T[n] @ V[n]
    V[n] = np.maximum(V[n] * np.sqrt((T[n].T @ (P[:, :, n] / R ** 2)) / (T[n].T @ (1.0 / R))), NMF_FLOOR)


def update_w(Xs, W, T, V, n):
    """Iterative-projection update of demixing row n of every frequency (in place)."""
    I, J, M = Xs.shape
    R = T[n] @ V[n]                                                 # [I, J]
    U = np.einsum("ijm,ijk->imk", Xs / R[:, :, None], np.conj(Xs)) / J
    e = np.zeros(M)
    e[n] = 1.0
    w = np.linalg.solve(W @ U, np.broadcast_to(e, (I, M)).astype(np.complex128)[..., None])[..., 0]
    w = w / np.sqrt(np.real(np.einsum("im,imk,ik->i", np.conj(w), U, w)))[:, None]
    W[:, n, :] = np.conj(w)


def normalise(Xs, W, T):
    """Per-source scale: lambda_n^2 = mean |y_n|^2; w_n /= lambda_n, t_n /= lambda_n^2."""
    Y = np.einsum("inm,ijm->ijn", W, Xs)
    lam = np.sqrt(np.mean(np.abs(Y) ** 2, axis=(0, 1)))            # [N]
    W /= lam[None, :, None]
    T /= (lam ** 2)[:, None, None]


def iterate(Xs, W, T, V):
    """One ILRMA iteration on the sphered observation (in place): for each source n,
    the bases, the activations and the demixing row; then the scale normalisation."""
    N = W.shape[1]
    for n in range(N):
        P = np.abs(np.einsum("inm,ijm->ijn", W, Xs)) ** 2
        update_T(P, T, V, n)
        update_V(P, T, V, n)
        update_w(Xs, W, T, V, n)
    normalise(Xs, W, T)


@dataclass
class IlrmaResult:
    W: np.ndarray      # [I, M, M] demixing matrices of the original observation (row n = w_n^H)
    T: np.ndarray      # [N, I, K] bases
    V: np.ndarray      # [N, K, J] activations
    Q: np.ndarray      # [I, M, M] sphering


def ilrma(X, T0, V0, n_iter: int, history=None) -> IlrmaResult:
    """ILRMA on the observation X [I, J, M] with initial NMF variables T0 [N, I, K],
    V0 [N, K, J] (non-negative, drawn by the caller) and W = I in the sphered
    coordinates.  Returns the demixing matrices of X itself (W Q), T and V.
    history, when a list, receives the cost after every iteration."""
    X = np.asarray(X, np.complex128)
    I, J, M = X.shape
    Q = sphering(X)
    Xs = np.einsum("imn,ijn->ijm", Q, X)
    W = np.broadcast_to(np.eye(M, dtype=np.complex128), (I, M, M)).copy()
    T = np.array(T0, np.float64)
    V = np.array(V0, np.float64)
    for _ in range(n_iter):
        iterate(Xs, W, T, V)
        if history is not None:
            history.append(cost(Xs, W, T, V))
    return IlrmaResult(W=W @ Q, T=T, V=V, Q=Q)
