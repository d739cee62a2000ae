"""Parity of the front end on the GPU (STFT, inverse STFT, ILRMA; called through
the C ABI) with the FP64 oracle of oracle/ilrma_oracle.py on the same seeded
inputs, and the whole chain from a time signal to the extracted target's time
signal against the oracle's chain.  Needs a GPU; marked `gpu`.

Bars: the STFT and inverse STFT are FP32 FFTs of log2(n_fft) stages, within
1e-5 relative of the FP64 transforms (about log2(n_fft) units of rounding of
the signal's norm); ILRMA after one iteration within 1e-5 and after a full run
within 1e-3 relative (W, T, V), the bars of the estimator; the chain's output
signal at least 60 dB SNR against the oracle's."""
import numpy as np
import pytest

from oracle import ilrma_oracle as F
from oracle import rcscm_oracle as O
from paper_1908_01964_gb300 import synth
from parity_util import ALPHA, BETA, SDR_MIN_DB, TOL_FULL_RUN, TOL_ONE_ITER, rel, report, sdr_db

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1908_01964_gb300 import build, rcscm
    build.build()
    rcscm.lib()
    torch.cuda.init()


def rel_rows(Wg, Wo):
    """Relative error of demixing matrices up to a unit factor per row: the sphering's
    eigenvectors, and so each row of W_i Q_i, are defined up to a phase, which no
    output of the chain depends on (the back-projection and R' are invariant)."""
    Wg = np.asarray(Wg, np.complex128)
    d = np.einsum("inm,inm->in", Wg, np.conj(Wo))
    d = np.where(np.abs(d) > 0, d / np.abs(d), 1.0)
    return rel(Wg * np.conj(d)[..., None], Wo)


def _t(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


@pytest.mark.parametrize("M,T,n_fft,shift", [(2, 4000, 64, 32), (3, 1000, 16, 8), (4, 16000 * 2, 1024, 512),
                                             (5, 3333, 256, 64), (8, 20000, 4096, 2048), (4, 100, 512, 256)])
def test_stft_and_inverse_match_oracle(M, T, n_fft, shift):
    from paper_1908_01964_gb300 import rcscm as R
    sig = np.random.default_rng(M * 1000 + n_fft).standard_normal((M, T)).astype(np.float32)
    with R.Front(M, T, n_fft, shift, K=2) as fe:
        X = fe.stft(_t(sig, np.float32)).cpu().numpy()
        Xo = F.stft(sig.astype(np.float64), n_fft, shift)
        assert X.shape == Xo.shape
        e_fwd = rel(X, Xo)
        back = fe.istft(_t(X, np.complex64)).cpu().numpy()
        e_inv = rel(back, sig)
        # a spectrum that is no STFT of anything (the estimator's outputs are not):
        # the least-squares inverse against the oracle's
        Y = (Xo * np.exp(1j * np.random.default_rng(1).uniform(0, 2 * np.pi, Xo.shape))).astype(np.complex64)
        y = fe.istft(_t(Y, np.complex64)).cpu().numpy()
        e_ls = rel(y, F.istft(Y.astype(np.complex128), n_fft, shift, T))
    report("stft", M=M, T=T, n_fft=n_fft, shift=shift, forward=e_fwd, roundtrip=e_inv, inverse=e_ls)
    assert e_fwd < 1e-5 and e_inv < 1e-5 and e_ls < 1e-5, (e_fwd, e_inv, e_ls)


@pytest.mark.parametrize("case", ["bss-m2", "bss-m3", "bss-m4", "mixture-m4"])
def test_ilrma_matches_oracle(case):
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    if case.startswith("bss"):
        M = int(case[-1])
        b = synth.make_bss_mixture(M, 33, 200, 5, 70 + M)
        X, T0, V0, K, n_fft = b["x"], b["T0"], b["V0"], 5, 64
        T = (200 - 1) * 32 + 64
    else:
        M, n_fft, shift, K = 4, 1024, 512, 10
        d = synth.make_time_mixture(M, 16000 * 3, 81)
        X = F.stft(d["sig"], n_fft, shift).astype(np.complex64)
        T = d["sig"].shape[1]
        T0, V0 = synth.ilrma_init_values(X.shape[0], X.shape[1], M, K, 82)
    I, J, _ = X.shape
    shift = n_fft // 2
    with R.Front(M, T, n_fft, shift, K=K) as fe:
        assert (fe.I, fe.J) == (I, J)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        for n_iter, tol in ((1, TOL_ONE_ITER), (50, TOL_FULL_RUN)):
            W, Tg, Vg = fe.ilrma(_t(X, np.complex64), _t(T0, np.float32), _t(V0, np.float32), n_iter, status=st)
            o = F.ilrma(X.astype(np.complex128), T0, V0, n_iter)
            e = dict(W=rel_rows(W.cpu().numpy(), o.W), T=rel(Tg.cpu().numpy(), o.T), V=rel(Vg.cpu().numpy(), o.V))
            report("ilrma", case=case, n_iter=n_iter, gpu=e)
            assert int(st.item()) == 0
            assert max(e.values()) < tol, (n_iter, e)


def test_front_to_back_chain_matches_oracle():
    """Time signal -> STFT -> ILRMA (50 iterations) -> estimator inputs (Sec. II-B-1,
    II-B-3) -> 100 passes of Algorithm 2 -> Wiener filter -> inverse STFT, on the GPU
    through the C ABI and in the FP64 oracle, in the paper's arrangement (M = 4,
    16 kHz, 64 ms / 32 ms, K = 10, 30-degree target, 19-source babble, 0 dB)."""
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    M, n_fft, shift, K, n_ilrma, n_em = 4, 1024, 512, 10, 50, 100
    d = synth.make_time_mixture(M, 16000 * 4, 91)
    sig = d["sig"].astype(np.float32)
    T = sig.shape[1]
    with R.Front(M, T, n_fft, shift, K=K) as fe:
        I, J = fe.I, fe.J
        T0, V0 = synth.ilrma_init_values(I, J, M, K, 92)
        X = fe.stft(_t(sig, np.float32))
        W, Tg, Vg = fe.ilrma(X, _t(T0, np.float32), _t(V0, np.float32), n_ilrma)
        # oracle chain
        Xo = F.stft(sig.astype(np.float64), n_fft, shift)
        o = F.ilrma(Xo, T0, V0, n_ilrma)
        # target output: the demixing column whose back-projected steering vector is
        # closest to the plane wave from the target direction (known to the test)
        f = np.arange(I) * 16000.0 / n_fft
        xs = (np.arange(M) - (M - 1) / 2.0) * d["spacing"]
        a_true = np.exp(-2j * np.pi * f[:, None] * (xs * np.sin(np.deg2rad(d["target_deg"])) / 343.0)[None, :])
        A = np.linalg.inv(o.W)
        score = [np.sum(np.abs(np.einsum("im,im->i", np.conj(a_true[1:]), A[1:, :, n])) /
                        np.linalg.norm(A[1:, :, n], axis=1)) for n in range(M)]
        n_h = int(np.argmax(score))
        utt = dict(x=X, W=W, T=Tg[n_h].contiguous(), V=Vg[n_h].contiguous(), n_h=n_h)
        (init,) = R.ilrma_init([utt])
        prob = dict(x=X, a=init["a"], Rp=init["Rp"], rh0=init["rh0"], ru0=init["ru0"])
        with R.Solver([prob]) as s:
            s.setup()
            s.iterate(n_em)
            h = s.extract().view(I, J, M)
            assert s.status() in (R.OK, R.ECLAMP)
        out = fe.istft(h.contiguous()).cpu().numpy()
        oi = O.ilrma_init(Xo, o.W, o.T[n_h], o.V[n_h], n_h)
        po = dict(x=Xo, a=oi.a, Rp=oi.Rp, rh0=oi.rh0, ru0=oi.ru0)
        ro = O.run(po, n_em, "accel2", alpha=ALPHA, beta=BETA)
        out_o = F.istft(ro["h"], n_fft, shift, T)
    snr = sdr_db(out, out_o)
    diag = dict(X=rel(X.cpu().numpy(), Xo), W=rel_rows(W.cpu().numpy(), o.W), T=rel(Tg.cpu().numpy(), o.T),
                V=rel(Vg.cpu().numpy(), o.V), rh0=rel(init["rh0"].cpu().numpy(), oi.rh0),
                ru0=rel(init["ru0"].cpu().numpy(), oi.ru0), Rp=rel(init["Rp"].cpu().numpy(), oi.Rp),
                h_stft=sdr_db(h.cpu().numpy(), ro["h"]))
    # the GPU solver on the oracle's estimator inputs: isolates the estimator's share
    with R.Solver([R.to_device(dict(x=Xo.astype(np.complex64), a=oi.a, Rp=oi.Rp, rh0=oi.rh0, ru0=oi.ru0))]) as s:
        s.setup()
        s.iterate(n_em)
        h2 = s.extract().view(I, J, M).cpu().numpy()
    diag["h_from_oracle_inputs"] = sdr_db(h2, ro["h"])
    report("front_to_back_diag", **diag)
    # separation quality against the target image (a sanity figure, not a parity bar)
    gain = sdr_db(out_o[0], d["target"][0]) - sdr_db(sig[0], d["target"][0])
    report("front_to_back_chain", snr_vs_oracle=snr, n_h=n_h, oracle_gain_db=gain)
    assert snr > SDR_MIN_DB, snr
    assert gain > 0.0, gain
