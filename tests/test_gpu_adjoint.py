"""Parity of the CUDA adjoint (rcscm_backward and the autograd wrapper) with
the FP64 oracle gradient (torch autograd of oracle/rcscm_oracle_torch.py, itself
pinned to finite differences of the numpy oracle) and with central finite
differences of the numpy oracle's loss.  Loss: L = sum |h - h_true|^2.
Tolerance: 1e-3 relative (2-norm over each gradient)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rcscm_oracle as O  # noqa: E402
from oracle import rcscm_oracle_torch as OT  # noqa: E402
from paper_1908_01964_gb300 import synth  # noqa: E402

from parity_util import rel, report  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3


def _prob(M, I, J, seed, lam_scale=1.3):
    p = synth.tiny(M=M, I=I, J=J, K=4, seed=seed)
    st = O.setup(p["a"], p["Rp"])
    p["lambda0"] = st.lam0 * lam_scale          # given, held constant by both sides
    return p


def _gpu_grads(probs, K, stride, block=0, iters_per_launch=0):
    """Forward + backward on the GPU; L = sum |h - h_true|^2 with g_h = 2 (h - h_true)."""
    from paper_1908_01964_gb300 import rcscm as R
    dev = [R.to_device(p) for p in probs]
    with R.Solver(dev, ckpt_stride=stride, ckpt_max_iters=max(K, 1), block=block,
                  iters_per_launch=iters_per_launch) as s:
        s.setup()
        s.iterate(K)
        h = s.extract()
        ht = torch.cat([torch.from_numpy(np.ascontiguousarray(p["h_true"], np.complex64)).reshape(-1)
                        for p in probs]).cuda()
        gh = (2.0 * (h - ht)).contiguous()
        grads = [tuple(g.cpu().numpy() for g in gs) for gs in s.split_grads(*s.backward(gh))]
        torch.cuda.synchronize()
    return grads


def _oracle_grads(p, K, rows=None):
    q = {k: (v[rows] if rows is not None and k in ("x", "a", "Rp", "rh0", "ru0", "lambda0", "h_true") else v)
         for k, v in p.items()}
    _, gx, ga, gR = OT.loss_and_grads(q["x"], q["a"], q["Rp"], q["rh0"], q["ru0"], q["lambda0"], K, q["h_true"])
    return gx, ga, gR


@pytest.mark.parametrize("M", [2, 3, 4, 6, 8])
def test_adjoint_matches_oracle_gradient(M):
    p = _prob(M, I=6, J=40, seed=100 + M)
    K = 7                                           # checkpoints at passes 0 and 5
    (gx, ga, gR), = _gpu_grads([p], K, stride=5)
    ox, oa, oR = _oracle_grads(p, K)
    e = dict(x=rel(gx, ox), a=rel(ga, oa), Rp=rel(gR, oR))
    report(f"adjoint M={M}", **e)
    assert max(e.values()) < TOL_GRAD, e


def test_adjoint_equals_central_finite_differences():
    # M = 2, I = 8, J = 16: directional derivatives of the FP64 numpy loss
    p = _prob(2, I=8, J=16, seed=21)
    K = 6
    (gx, ga, gR), = _gpu_grads([p], K, stride=5)

    def loss(**kw):
        q = dict(p)
        q.update(kw)
        r = O.run(q, K, "accel2", lambda0=p["lambda0"])
        return float(np.sum(np.abs(r["h"] - p["h_true"].astype(np.complex128)) ** 2))

    rng = np.random.default_rng(5)
    base = dict(x=p["x"].astype(np.complex128), a=p["a"].astype(np.complex128), Rp=p["Rp"].astype(np.complex128))
    L0 = loss()
    for name, g in (("x", gx), ("a", ga), ("Rp", gR)):
        for _ in range(3):
            v = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
            if name == "Rp":
                v = 0.1 * v * np.abs(base["Rp"]).max()
            h = 1e-6
            fd = (loss(**{name: base[name] + h * v}) - loss(**{name: base[name] - h * v})) / (2 * h)
            an = float(np.sum(np.real(np.conj(g.astype(np.complex128)) * v)))
            assert abs(fd - an) <= TOL_GRAD * max(abs(fd), 1e-3 * L0), (name, fd, an)


def test_adjoint_is_independent_of_the_checkpoint_stride():
    # recomputation from checkpoints reproduces the forward states bit for bit
    p = _prob(3, I=5, J=300, seed=8)
    K = 11
    ref = _gpu_grads([p], K, stride=1, block=128)
    for stride in (3, 5, 11, 40):
        got = _gpu_grads([p], K, stride=stride, block=128)
        for a, b in zip(ref[0], got[0]):
            assert np.array_equal(a, b), stride


def test_checkpoints_from_the_streaming_kernel_give_the_same_gradients():
    # one pass per launch runs the streaming kernel, which writes the checkpoints itself
    p = _prob(4, I=4, J=700, seed=9)
    K = 8
    a = _gpu_grads([p], K, stride=3, block=256)
    b = _gpu_grads([p], K, stride=3, block=256, iters_per_launch=1)
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("block", [128, 256])
def test_adjoint_batch_mixed_shapes(block):
    # one context: mixed M and ragged J spanning one to four chunk pairs
    Js = [40, 300, 700, 1500] if block == 256 else [40, 130, 300, 512]
    probs = [_prob(M, I=3, J=J, seed=40 + k) for k, (M, J) in enumerate(zip([2, 3, 4, 5], Js))]
    K = 6
    grads = _gpu_grads(probs, K, stride=5, block=block)
    for k, p in enumerate(probs):
        ox, oa, oR = _oracle_grads(p, K)
        e = dict(x=rel(grads[k][0], ox), a=rel(grads[k][1], oa), Rp=rel(grads[k][2], oR))
        report(f"adjoint batch block={block} J={p['x'].shape[1]}", **e)
        assert max(e.values()) < TOL_GRAD, (k, e)


def test_adjoint_zero_passes_is_the_wiener_and_setup_gradient():
    p = _prob(4, I=4, J=33, seed=3)
    (gx, ga, gR), = _gpu_grads([p], 0, stride=5)
    ox, oa, oR = _oracle_grads(p, 0)
    assert max(rel(gx, ox), rel(ga, oa), rel(gR, oR)) < TOL_GRAD


def test_autograd_function_matches_solver_backward():
    from paper_1908_01964_gb300 import rcscm as R
    from paper_1908_01964_gb300.autograd import wiener_estimate
    p = _prob(3, I=4, J=50, seed=12)
    d = R.to_device(p)
    x = d["x"].clone().requires_grad_(True)
    a = d["a"].clone().requires_grad_(True)
    Rp = d["Rp"].clone().requires_grad_(True)
    ht = torch.from_numpy(p["h_true"]).cuda()
    h = wiener_estimate(x, a, Rp, d["rh0"], d["ru0"], 8, lambda0=d["lambda0"], ckpt_stride=5)
    loss = ((h - ht).abs() ** 2).sum()
    loss.backward()
    ox, oa, oR = _oracle_grads(p, 8)
    e = dict(x=rel(x.grad.cpu().numpy(), ox), a=rel(a.grad.cpu().numpy(), oa), Rp=rel(Rp.grad.cpu().numpy(), oR))
    assert max(e.values()) < TOL_GRAD, e


def test_backward_call_contract():
    from paper_1908_01964_gb300 import rcscm as R
    p = _prob(2, I=3, J=20, seed=2)
    d = R.to_device(p)
    gh = torch.zeros(3 * 20 * 2, dtype=torch.complex64, device="cuda")
    with R.Solver([d]) as s:                        # no checkpoints
        s.setup()
        s.iterate(2)
        with pytest.raises(R.RcscmError) as ei:
            s.backward(gh)
        assert ei.value.code == R.EINVAL
    with R.Solver([d], ckpt_stride=2, ckpt_max_iters=4) as s:
        s.setup()
        s.iterate(3)
        with pytest.raises(R.RcscmError) as ei:     # beyond ckpt_max_iters
            s.iterate(2)
        assert ei.value.code == R.EINVAL
        with pytest.raises(R.RcscmError) as ei:     # graphs need host bookkeeping
            s.graph_create(2, torch.empty(120, dtype=torch.complex64, device="cuda"))
        assert ei.value.code == R.EINVAL
        s.backward(gh)                              # still usable
        torch.cuda.synchronize()
    with pytest.raises(R.RcscmError):               # adjoint block shapes only
        R.Solver([d], ckpt_stride=2, ckpt_max_iters=4, block=512)


def test_adjoint_full_size_sampled_rows():
    # the adjoint workload's utterance shape (M = 4, I = 513, J = 500, 20 passes,
    # stride 5), two utterances in one context; sampled rows against the oracle
    wl = synth.workload("adjoint-16", n_utt=2)
    probs = synth.make_workload(wl)
    for p in probs:
        p["lambda0"] = O.setup(p["a"], p["Rp"]).lam0
    grads = _gpu_grads(probs, wl.n_iter, stride=wl.extra["ckpt_stride"])
    rows = np.array([0, 17, 256, 511])
    for k, p in enumerate(probs):
        ox, oa, oR = _oracle_grads(p, wl.n_iter, rows=rows)
        gx, ga, gR = (g[rows] for g in grads[k])
        e = dict(x=rel(gx, ox), a=rel(ga, oa), Rp=rel(gR, oR))
        report(f"adjoint full-size utt {k}", **e)
        assert max(e.values()) < TOL_GRAD, (k, e)
        assert all(np.isfinite(g).all() for g in grads[k])
