"""Parity of rcscm_ilrma_init (the estimator's inputs from the outputs of the
ILRMA stage: Sec. II-A, Sec. II-B-1 Eq. (eq:rit), Sec. II-B-3 Eqs. (eq:rhinit),
(eq:ruinit)) with the FP64 oracle, called through the C ABI.

Tolerances: a_i (an FP64 inverse) 1e-10 relative per row; r_h0 (K positive FP32
products) 2 (K + 1) u relative per slot; R'_i and r_u0 within the forward error
bounds of their FP32 frame sums (tests/parity_util.ilrma_fp32_bounds, checked on
the CPU in tests/test_formulation.py).  End to end, the initialisation followed by
the accelerated solve meets the bars of the solve itself against the oracle run
from the oracle's own initialisation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rcscm_oracle as O  # noqa: E402
from paper_1908_01964_gb300 import synth  # noqa: E402

from parity_util import (SDR_MIN_DB, TOL_FULL_RUN, TOL_ONE_ITER, compare, ilrma_fp32_bounds,  # noqa: E402
                         oracle_run, rel, report)

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def _raw(M, I, J, K, seed, n_h=0):
    p = synth.make_problem(synth.ProblemSpec(M=M, I=I, J=J, K=K, spacing=0.03), seed)
    p["n_h"] = n_h
    return p


def _gpu_init(probs, status=None):
    from paper_1908_01964_gb300 import rcscm as R
    outs = R.ilrma_init([R.ilrma_to_device(p) for p in probs], status=status)
    torch.cuda.synchronize()
    return [{k: v.cpu().numpy() for k, v in o.items()} for o in outs]


def _check_init(p, g, name):
    o = O.ilrma_init(p["x"], p["W"], p["T"], p["V"], p["n_h"])
    K = p["T"].shape[1]
    ea = np.max(np.linalg.norm(g["a"] - o.a, axis=1) / np.linalg.norm(o.a, axis=1))
    erh = np.max(np.abs(g["rh0"] - o.rh0) / o.rh0)
    dR, dru = ilrma_fp32_bounds(p["x"], p["W"], p["n_h"])
    eR = np.linalg.norm(g["Rp"] - o.Rp, axis=(1, 2))
    eru = np.abs(g["ru0"] - o.ru0)
    report(name, a=float(ea), rh0=float(erh), Rp=float(np.max(eR / np.linalg.norm(o.Rp, axis=(1, 2)))),
           ru0=float(np.max(eru / o.ru0)), Rp_of_bound=float(np.max(eR / dR)), ru0_of_bound=float(np.max(eru / dru)))
    assert ea < 1e-10, ea
    assert erh <= 2 * (K + 1) * U, erh
    assert np.all(eR <= dR + 1e-12 * np.linalg.norm(o.Rp, axis=(1, 2))), np.max(eR / dR)
    assert np.all(eru <= dru + 1e-12 * o.ru0), np.max(eru / dru)
    # R'_i comes out exactly Hermitian (upper triangle mirrored)
    assert np.array_equal(g["Rp"], np.conj(np.transpose(g["Rp"], (0, 2, 1))))


def test_ilrma_init_matches_oracle_mixed_batch():
    # one call over utterances with M = 2..8, n_h inside and at the ends, K = 1..20 and
    # ragged J (1 frame up to several thread strides with a tail)
    cases = [(2, 1, 1, 0), (2, 37, 3, 1), (3, 300, 7, 2), (4, 1000, 20, 0), (5, 129, 5, 4),
             (6, 97, 11, 3), (7, 300, 2, 6), (8, 400, 9, 5)]
    probs = [_raw(M, I=5, J=J, K=K, seed=200 + k, n_h=nh) for k, (M, J, K, nh) in enumerate(cases)]
    outs = _gpu_init(probs)
    for p, g, (M, J, K, nh) in zip(probs, outs, cases):
        _check_init(p, g, f"ilrma_init M={M} J={J} K={K} n_h={nh}")


def test_ilrma_init_full_size_sampled_rows():
    # the single-utterance shape (M = 4, I = 1025, J = 1000, K = 20); rows sampled for the oracle
    wl = synth.workload("single-m4")
    p = synth.make_workload(wl)[0]
    p["n_h"] = 0
    (g,) = _gpu_init([p])
    rows = np.array([0, 1, 2, 300, 700, 1023, 1024])
    q = dict(x=p["x"][rows], W=p["W"][rows], T=p["T"][rows], V=p["V"], n_h=0)
    _check_init(q, {k: v[rows] for k, v in g.items()}, "ilrma_init single-m4 sampled rows")


@pytest.mark.parametrize("M,n_iter", [(2, 1), (4, 1), (4, 20)])
def test_ilrma_init_then_solve_matches_oracle(M, n_iter):
    from paper_1908_01964_gb300 import rcscm as R
    p = _raw(M, I=17, J=300, K=10, seed=300 + M)
    (g,) = _gpu_init([p])
    dev = dict(x=R.to_device(p)["x"], a=torch.from_numpy(g["a"]).cuda(), Rp=torch.from_numpy(g["Rp"]).cuda(),
               rh0=torch.from_numpy(g["rh0"]).cuda(), ru0=torch.from_numpy(g["ru0"]).cuda())
    with R.Solver([dev]) as s:
        h = s.solve(n_iter).cpu().numpy().reshape(p["x"].shape)
        rh, ru, lam = (t.cpu().numpy() for t in s.get_state(0))
        st = s.status()
    o_in = O.ilrma_init(p["x"], p["W"], p["T"], p["V"], 0)
    q = dict(p, a=o_in.a, Rp=o_in.Rp, rh0=o_in.rh0, ru0=o_in.ru0)
    o = oracle_run(q, n_iter)
    e = compare(dict(rh=rh, ru=ru, lam=lam, h=h), o)
    report(f"ilrma_init + solve M={M} passes={n_iter}", gpu=e, status=st)
    assert st == 0, st
    tol = TOL_ONE_ITER if n_iter == 1 else TOL_FULL_RUN
    assert max(e["rh"], e["ru"], e["lam"]) < tol, e
    assert e["sdr"] > SDR_MIN_DB, e


def test_ilrma_init_status_and_refusals():
    from paper_1908_01964_gb300 import rcscm as R
    p = _raw(3, I=4, J=50, K=4, seed=9)
    d = R.ilrma_to_device(p)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    outs = R.ilrma_init([d], status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.isfinite(torch.view_as_real(outs[0]["Rp"])).all()
    Ws = d["W"].clone()
    Ws[2, 1, :] = 0                                   # row 2: W singular
    R.ilrma_init([dict(d, W=Ws)], status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & (1 << (R.ENULLSPACE - 1))
    with pytest.raises(R.RcscmError) as ei:           # n_h outside 0..M-1
        R.ilrma_init([dict(d, n_h=3)])
    assert ei.value.code == R.EINVAL
    with pytest.raises(TypeError):                    # pageable host memory: refused by the binding
        R.ilrma_init([dict(d, x=d["x"].cpu())])


def test_ilrma_plan_reruns_reproduce_the_call():
    # a prepared call run again over its own outputs gives the one-shot call's
    # results bit for bit
    from paper_1908_01964_gb300 import rcscm as R
    probs = [_raw(4, 9, 300, 5, 61, n_h=1), _raw(3, 5, 77, 2, 62, n_h=2)]
    utts = [R.ilrma_to_device(p) for p in probs]
    ref = [{k: v.cpu().numpy() for k, v in o.items()} for o in R.ilrma_init(utts)]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    plan = R.IlrmaPlan(utts, status=status)
    for _ in range(3):
        outs = plan.run()
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            for k in r:
                np.testing.assert_array_equal(o[k].cpu().numpy(), r[k], err_msg=k)
    assert int(status.item()) == 0
