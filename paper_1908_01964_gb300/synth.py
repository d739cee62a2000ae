"""Seeded synthetic inputs for rank-constrained SCM estimation.

This module only draws random numbers and assembles the method's INPUTS; it
contains none of the estimator's arithmetic (no setup, no EM update, no Wiener
filter).  Both the CUDA path and the FP64 oracle consume what it returns.

The paper's data (JNAS speech convolved with measured room impulse responses,
Sec. IV-A) is not available, so seeded draws with the same STFT scale stand in
for it (fs = 16 kHz, Table II):

* target direction: a plane wave from a random direction of arrival,
  a_true[i, m] = exp(-j 2 pi f_i tau_m) / sqrt(M) (unit norm);
* diffuse noise SCM: spherically isotropic coherence sin(z)/z with
  z = 2 pi f_i d_mn / c, plus 1e-3 I (full rank);
* target variance: rank-K NMF, r_h = T V with T, V ~ Gamma(1, 1);
* noise variance: r_u ~ Gamma(shape 2, scale 0.5), i.i.d. per slot;
* x = a_true s + u, s ~ N_c(0, r_h), u ~ N_c(0, r_u R_true) (Sec. II-B-1).

A stand-in for the ILRMA stage (Sec. II-A) gives the boundary inputs: the true
demixing matrix W_true = Q^H (Q unitary, first column a_true) perturbed by 1 %
complex Gaussian noise; a is the target column of W~^{-1}; R' is the
back-projected rank-(M-1) noise SCM of Eq. (eq:rit); r_u0 follows Eq.
(eq:ruinit) and r_h0 is the true NMF product with 1 % multiplicative noise
(stands in for Eq. (eq:rhinit)).  The target index n_h is 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

FS = 16000.0          # sampling frequency [Hz] (Table II)
C_SOUND = 343.0       # speed of sound [m/s]
BASE_SEED = 190801964
ALPHA = 1.1           # inverse-gamma shape (Table II)
BETA = 1e-16          # inverse-gamma scale (Table II)


@dataclass
class ProblemSpec:
    """Shape and geometry of one utterance (one STFT tensor I x J x M)."""
    M: int
    I: int
    J: int
    K: int = 10
    geometry: str = "linear"     # "linear" (spacing) or "circular" (radius)
    spacing: float = 0.04        # [m]: mic spacing, or radius if circular

    @property
    def nfft(self) -> int:
        return 2 * (self.I - 1)


@dataclass
class Workload:
    """A named set of utterances solved together, plus the iteration count."""
    name: str
    specs: List[ProblemSpec]
    n_iter: int
    seed: int
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def slots(self) -> int:
        return int(sum(s.I * s.J for s in self.specs))


def _mic_positions(spec: ProblemSpec) -> np.ndarray:
    M = spec.M
    if spec.geometry == "linear":
        xs = (np.arange(M) - (M - 1) / 2.0) * spec.spacing
        return np.stack([xs, np.zeros(M)], axis=1)
    if spec.geometry == "circular":
        ang = 2.0 * np.pi * np.arange(M) / M
        return spec.spacing * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    raise ValueError(f"unknown geometry {spec.geometry!r}")


def make_problem(spec: ProblemSpec, seed: int) -> dict:
    """Draw one utterance.

    Returns a dict with the boundary inputs
      x   complex64  [I, J, M]   observed STFT
      a   complex128 [I, M]      target steering vector (back-projected)
      Rp  complex128 [I, M, M]   rank-(M-1) noise SCM R'
      rh0 float32    [I, J]      initial target variance
      ru0 float32    [I, J]      initial noise variance
    and the ground truth  a_true, h_true (complex64 [I, J, M], target image),
    rh_true, ru_true; and the ILRMA stand-in's own outputs W (perturbed
    demixing matrices, complex128 [I, M, M]), T (float32 [I, K]) and V
    (float32 [K, J]) (the target's NMF factors with 1 % noise) and n_h = 0.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    M, I, J, K = spec.M, spec.I, spec.J, spec.K
    f = np.arange(I) * FS / spec.nfft                       # [I]

    pos = _mic_positions(spec)                               # [M, 2]
    if spec.geometry == "linear":
        theta = rng.uniform(0.0, np.pi)
    else:
        theta = rng.uniform(0.0, 2.0 * np.pi)
    direction = np.array([np.cos(theta), np.sin(theta)])
    delay = -(pos @ direction) / C_SOUND                     # [M]
    a_true = np.exp(-2j * np.pi * f[:, None] * delay[None, :]) / np.sqrt(M)

    dist = np.linalg.norm(pos[:, None, :] - pos[None, :, :], axis=-1)  # [M, M]
    # np.sinc(v) = sin(pi v)/(pi v); the coherence is sin(z)/z, z = 2 pi f d / c
    R_true = np.sinc(2.0 * f[:, None, None] * dist[None] / C_SOUND) + 1e-3 * np.eye(M)
    L_true = np.linalg.cholesky(R_true)                      # [I, M, M]

    T = rng.gamma(1.0, 1.0, size=(I, K))
    V = rng.gamma(1.0, 1.0, size=(K, J))
    rh_true = T @ V                                          # [I, J]
    ru_true = rng.gamma(2.0, 0.5, size=(I, J))

    s = np.sqrt(rh_true / 2.0) * (rng.standard_normal((I, J)) + 1j * rng.standard_normal((I, J)))
    nse = (rng.standard_normal((I, J, M)) + 1j * rng.standard_normal((I, J, M))) / np.sqrt(2.0)
    u = np.sqrt(ru_true)[..., None] * np.einsum("imn,ijn->ijm", L_true, nse)
    h_true = a_true[:, None, :] * s[..., None]
    x = (h_true + u).astype(np.complex64)
    xd = x.astype(np.complex128)

    # ILRMA stand-in: W_true = Q^H with Q unitary and Q[:, 0] = a_true.
    Z = rng.standard_normal((I, M, M)) + 1j * rng.standard_normal((I, M, M))
    Z[:, :, 0] = a_true
    Q, Rq = np.linalg.qr(Z)
    ph = Rq[:, 0, 0] / np.abs(Rq[:, 0, 0])
    Q[:, :, 0] *= ph[:, None]
    W_true = np.conj(np.transpose(Q, (0, 2, 1)))
    G = (rng.standard_normal((I, M, M)) + 1j * rng.standard_normal((I, M, M))) / np.sqrt(2.0)
    W = W_true + 0.01 * (np.sqrt(M) / M) * G                # ||W_true||_F = sqrt(M)
    Winv = np.linalg.inv(W)
    a = Winv[:, :, 0].copy()                                 # back-projected target column

    # Eq. (eq:rit): back-projection of the M-1 noise outputs, averaged over j.
    y = np.einsum("imn,ijn->ijm", W, xd)                     # y_n = w_n^H x
    p = np.mean(np.abs(y) ** 2, axis=1)                      # [I, M]
    p[:, 0] = 0.0
    Rp = np.einsum("imk,ik,ink->imn", Winv, p, np.conj(Winv))
    Rp = 0.5 * (Rp + np.conj(np.transpose(Rp, (0, 2, 1))))

    # Eq. (eq:ruinit): r_u = y_u^H R'^+ y_u / M with the back-projected noise image.
    y[:, :, 0] = 0.0
    yu = np.einsum("imn,ijn->ijm", Winv, y)
    Rp_pinv = np.linalg.pinv(Rp, hermitian=True, rcond=1e-10)
    ru0 = np.real(np.einsum("ijm,imn,ijn->ij", np.conj(yu), Rp_pinv, yu)) / M
    ru0 = np.maximum(ru0, 1e-6 * np.mean(ru0))

    # Eq. (eq:rhinit) stand-in: the true NMF factors with 1 % multiplicative noise.
    That = T * np.maximum(1.0 + 0.01 * rng.standard_normal(T.shape), 1e-3)
    Vhat = V * np.maximum(1.0 + 0.01 * rng.standard_normal(V.shape), 1e-3)
    rh0 = That @ Vhat

    return dict(
        x=x, a=a, Rp=Rp,
        rh0=rh0.astype(np.float32), ru0=ru0.astype(np.float32),
        a_true=a_true, h_true=h_true.astype(np.complex64),
        rh_true=rh_true, ru_true=ru_true, W=W, spec=spec, seed=seed,
        T=That.astype(np.float32), V=Vhat.astype(np.float32), n_h=0,
    )


# --------------------------------------------------------------------------
# Named workloads (sizes of the paper's STFT scale; Table II gives fs, alpha,
# beta; the iteration counts and sizes below are the workloads measured here).
# --------------------------------------------------------------------------

def workload(name: str, n_utt: Optional[int] = None) -> Workload:
    """Return a named workload.

    plain-m2     M=2, I=257 (nfft 512), J=250, linear 4 cm, K=10, 50 iterations
    single-m4    M=4, I=1025 (nfft 2048), J=1000, linear 3 cm, K=20, 100 iterations
    batch-256    256 utterances, I=513, J ~ U[200, 2000], M in {2, 4, 6},
                 linear 4 cm, K=10, 100 iterations
    adjoint-16   16 utterances of M=4, I=513, J=500, linear 3 cm, K=10, 20 iterations
    scale-m8     M=8 circular (radius 5 cm), I=2049 (nfft 4096), J=4000, K=10, 200 iterations
    """
    if name == "plain-m2":
        specs = [ProblemSpec(M=2, I=257, J=250, K=10, spacing=0.04)]
        return Workload(name, specs, 50, BASE_SEED + 0)
    if name == "single-m4":
        specs = [ProblemSpec(M=4, I=1025, J=1000, K=20, spacing=0.03)]
        return Workload(name, specs, 100, BASE_SEED + 1)
    if name == "batch-256":
        n = 256 if n_utt is None else n_utt
        rng = np.random.Generator(np.random.PCG64(BASE_SEED + 2))
        Js = rng.integers(200, 2001, size=256)
        Ms = rng.choice([2, 4, 6], size=256)
        specs = [ProblemSpec(M=int(Ms[u]), I=513, J=int(Js[u]), K=10, spacing=0.04)
                 for u in range(n)]
        return Workload(name, specs, 100, BASE_SEED + 2)
    if name == "adjoint-16":
        n = 16 if n_utt is None else n_utt
        specs = [ProblemSpec(M=4, I=513, J=500, K=10, spacing=0.03) for _ in range(n)]
        return Workload(name, specs, 20, BASE_SEED + 3, extra={"ckpt_stride": 5})
    if name == "scale-m8":
        specs = [ProblemSpec(M=8, I=2049, J=4000, K=10, geometry="circular", spacing=0.05)]
        return Workload(name, specs, 200, BASE_SEED + 4)
    raise KeyError(name)


def utterance_seed(wl: Workload, u: int) -> int:
    """Seed of utterance u of a workload (independent PCG64 streams)."""
    return int(np.random.SeedSequence([wl.seed, u]).generate_state(1, dtype=np.uint64)[0] >> 1)


_INPUT_KEYS = ("x", "a", "Rp", "rh0", "ru0", "spec", "seed", "W", "T", "V", "n_h")


def _make_inputs_only(args):
    spec, seed = args
    p = make_problem(spec, seed)
    return {k: p[k] for k in _INPUT_KEYS}


def make_workload(wl: Workload, workers: int = 1, inputs_only: bool = False) -> List[dict]:
    """Draw every utterance of a workload (optionally in `workers` spawned processes;
    `inputs_only` drops the ground-truth arrays to save memory)."""
    jobs = [(s, utterance_seed(wl, u)) for u, s in enumerate(wl.specs)]
    if workers <= 1 or len(jobs) <= 1:
        if inputs_only:
            return [_make_inputs_only(j) for j in jobs]
        return [make_problem(s, seed) for s, seed in jobs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    fn = _make_inputs_only if inputs_only else _make_full
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, jobs, chunksize=1))


def _make_full(args):
    spec, seed = args
    return make_problem(spec, seed)


def tiny(M: int = 3, I: int = 5, J: int = 7, K: int = 3, seed: int = 7, **kw) -> dict:
    """A tiny problem for brute-force checks."""
    return make_problem(ProblemSpec(M=M, I=I, J=J, K=K, **kw), seed)


# --------------------------------------------------------------------------
# Inputs of the front end (STFT and ILRMA).  Random draws and signal synthesis
# only: no STFT, no ILRMA update and no estimator arithmetic.
# --------------------------------------------------------------------------

def ilrma_init_values(I: int, J: int, N: int, K: int, seed: int):
    """Non-negative random initial NMF variables of ILRMA (Sec. IV-A: "initialized by
    nonnegative random values"): T0 [N, I, K], V0 [N, K, J], uniform in [0.1, 1.1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    T0 = rng.uniform(0.1, 1.1, size=(N, I, K))
    V0 = rng.uniform(0.1, 1.1, size=(N, K, J))
    return T0, V0


def make_bss_mixture(M: int, I: int, J: int, K: int, seed: int) -> dict:
    """A determined, noise-free instantaneous mixture per frequency: x_ij = A_i s_ij with
    M sources whose variances are rank-K NMF products (Gamma(1, 1) bases and
    activations, one set per source) and a random mixing matrix A_i (complex Gaussian
    entries, each column scaled to unit norm).  Returns x (complex64 [I, J, M]), A
    (complex128 [I, M, M]), s (complex128 [I, J, M]) and ILRMA's initial T0, V0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Tn = rng.gamma(1.0, 1.0, size=(M, I, K))
    Vn = rng.gamma(1.0, 1.0, size=(M, K, J)) ** 2          # sparse-ish activations
    r = np.einsum("nik,nkj->ijn", Tn, Vn)
    s = np.sqrt(r / 2.0) * (rng.standard_normal((I, J, M)) + 1j * rng.standard_normal((I, J, M)))
    A = rng.standard_normal((I, M, M)) + 1j * rng.standard_normal((I, M, M))
    A /= np.linalg.norm(A, axis=1, keepdims=True)
    x = np.einsum("imn,ijn->ijm", A, s).astype(np.complex64)
    T0, V0 = ilrma_init_values(I, J, M, K, seed + 1)
    return dict(x=x, A=A, s=s, T0=T0, V0=V0)


def make_time_mixture(M: int, n_samples: int, seed: int, spacing: float = 0.04, snr_db: float = 0.0,
                      target_deg: float = 30.0, n_noise: int = 19) -> dict:
    """Multichannel time-domain mixture at fs = 16 kHz in the paper's arrangement
    (Sec. IV-A): a directional target 30 degrees from the array normal and a diffuse
    babble stand-in made of n_noise independent sources at 10-degree intervals, mixed
    at the given speech-to-noise ratio, on a linear array.  Each source signal is
    white noise shaped by a random two-pole resonance and a slowly varying random
    envelope (a speech-like, non-stationary spectrum); propagation to each microphone
    is a plane-wave delay applied as a phase shift of the source's whole-signal
    spectrum.  Returns sig (float64 [M, n_samples]), target (the target's image at the
    microphones, float64 [M, n_samples]) and the target direction."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = (np.arange(M) - (M - 1) / 2.0) * spacing
    n = n_samples
    freqs = np.fft.rfftfreq(n, d=1.0 / FS)

    def source():
        e = rng.standard_normal(n + 2)
        f0 = rng.uniform(200.0, 3000.0)
        rho = rng.uniform(0.85, 0.98)
        a1, a2 = 2.0 * rho * np.cos(2.0 * np.pi * f0 / FS), -rho * rho
        y = np.zeros(n + 2)
        for t in range(2, n + 2):
            y[t] = e[t] + a1 * y[t - 1] + a2 * y[t - 2]
        env = np.repeat(rng.gamma(1.0, 1.0, size=n // 800 + 2), 800)[:n]
        kern = np.hanning(801)
        env = np.convolve(env, kern / kern.sum(), mode="same")
        sig = y[2:] * env
        return sig / np.sqrt(np.mean(sig ** 2))

    def image(sig, deg):
        th = np.deg2rad(deg)
        delay = xs * np.sin(th) / C_SOUND                     # [M] seconds
        S = np.fft.rfft(sig)
        return np.fft.irfft(S[None, :] * np.exp(-2j * np.pi * freqs[None, :] * delay[:, None]), n=n, axis=1)

    target = image(source(), target_deg)
    angles = -90.0 + 10.0 * np.arange(n_noise)
    noise = sum(image(source(), d) for d in angles)
    g = np.sqrt(np.mean(target ** 2) / np.mean(noise ** 2) / 10.0 ** (snr_db / 10.0))
    return dict(sig=target + g * noise, target=target, target_deg=target_deg, spacing=spacing)
