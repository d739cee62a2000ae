"""Pins for the FP64 gradient oracle (torch autograd of oracle/rcscm_oracle_torch.py):
its forward equals the numpy oracle, and its gradients equal central finite
differences of the numpy oracle's loss.  CPU only."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rcscm_oracle as O  # noqa: E402
from oracle import rcscm_oracle_torch as OT  # noqa: E402
from paper_1908_01964_gb300 import synth  # noqa: E402


def _case(M, I=3, J=6, seed=1, K=4):
    p = synth.tiny(M=M, I=I, J=J, K=2, seed=seed)
    st = O.setup(p["a"], p["Rp"])
    p["lambda0"] = st.lam0 * 1.3          # a given lambda0 (held constant in the gradient)
    return p, K


def _numpy_loss(p, K, x=None, a=None, Rp=None):
    q = dict(p)
    if x is not None:
        q["x"] = x
    if a is not None:
        q["a"] = a
    if Rp is not None:
        q["Rp"] = Rp
    r = O.run(q, K, "accel2", lambda0=p["lambda0"])
    return float(np.sum(np.abs(r["h"] - p["h_true"].astype(np.complex128)) ** 2))


@pytest.mark.parametrize("M", [2, 3, 4])
def test_torch_forward_equals_numpy_oracle(M):
    p, K = _case(M)
    h, (rh, ru, lam) = OT.forward(*(torch.as_tensor(p[k].astype(np.complex128)) for k in ("x", "a", "Rp")),
                                  *(torch.as_tensor(np.asarray(p[k], np.float64)) for k in ("rh0", "ru0", "lambda0")), K)
    r = O.run(p, K, "accel2", lambda0=p["lambda0"])
    np.testing.assert_allclose(h.numpy(), r["h"], atol=1e-12 * np.abs(r["h"]).max())
    np.testing.assert_allclose(rh.numpy(), r["rh"], rtol=1e-11)
    np.testing.assert_allclose(ru.numpy(), r["ru"], rtol=1e-11)
    np.testing.assert_allclose(lam.numpy(), r["lam"], rtol=1e-11)


@pytest.mark.parametrize("M", [2, 3])
def test_gradients_equal_central_finite_differences(M):
    p, K = _case(M, seed=M + 10)
    L, gx, ga, gR = OT.loss_and_grads(p["x"], p["a"], p["Rp"], p["rh0"], p["ru0"], p["lambda0"], K, p["h_true"])
    assert abs(L - _numpy_loss(p, K)) < 1e-10 * abs(L)
    rng = np.random.default_rng(3)
    base = dict(x=p["x"].astype(np.complex128), a=p["a"].astype(np.complex128), Rp=p["Rp"].astype(np.complex128))
    for name, g in (("x", gx), ("a", ga), ("Rp", gR)):
        for _ in range(3):
            v = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
            if name == "Rp":
                v = 0.1 * v * np.abs(base["Rp"]).max()
            h = 1e-6
            lp = _numpy_loss(p, K, **{name: base[name] + h * v})
            lm = _numpy_loss(p, K, **{name: base[name] - h * v})
            fd = (lp - lm) / (2 * h)
            an = float(np.sum(np.real(np.conj(g) * v)))      # dL = Re <grad, v>
            assert abs(fd - an) <= 1e-5 * max(abs(fd), 1e-3 * abs(L)), (name, fd, an)


def test_loss_is_invariant_to_the_phase_of_b():
    # the gradient of R' is well defined because nothing depends on the phase of b
    p, K = _case(3, seed=5)
    L1 = _numpy_loss(p, K)
    q = dict(p)
    st = O.setup(p["a"], p["Rp"])
    st.b = st.b * np.exp(0.7j)
    st.sigma_ab = np.einsum("im,im->i", np.conj(p["a"]), st.b)
    x = p["x"].astype(np.complex128)
    inv = O.invariants(x, p["a"], st)
    rh, ru, lam = p["rh0"].astype(float), p["ru0"].astype(float), p["lambda0"].copy()
    for _ in range(K):
        rh, ru, lam = O.iterate_accel2(rh, ru, lam, inv, st, 3, 1.1, 1e-16)
    h = O.wiener(rh, ru, lam, x, p["a"], st)
    L2 = float(np.sum(np.abs(h - q["h_true"]) ** 2))
    assert abs(L1 - L2) < 1e-10 * abs(L1)
