"""The fused entry points (rcscm_setup_freq / rcscm_run / rcscm_solve) against the
separate calls (rcscm_setup, rcscm_iterate, rcscm_extract): outputs, state and
invariants must be bitwise equal, for every launch shape, plus the oracle on
the fused output."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1908_01964_gb300 import synth  # noqa: E402

from parity_util import SDR_MIN_DB, TOL_FULL_RUN, compare, oracle_run  # noqa: E402

pytestmark = pytest.mark.gpu


def _probs(shapes, seed=0):
    return [synth.tiny(M=M, I=I, J=J, K=4, seed=seed + k) for k, (M, I, J) in enumerate(shapes)]


def _snapshot(s):
    out = []
    for k in range(len(s.shapes)):
        rh, ru, lam = s.get_state(k)
        inv = s.get_invariants(k)
        out.append([t.cpu().numpy() for t in (rh, ru, lam, inv["tau_ax"], inv["sigma_bx"], inv["kappa"])])
    return out


def _separate(dev, K, **opts):
    from paper_1908_01964_gb300 import rcscm as R
    with R.Solver(dev, **opts) as s:
        s.setup()
        s.iterate(K)
        h = s.extract().cpu().numpy()
        snap = _snapshot(s)
        st = s.status()
    return h, snap, st


def _fused(dev, K, **opts):
    from paper_1908_01964_gb300 import rcscm as R
    with R.Solver(dev, **opts) as s:
        h = s.solve(K).cpu().numpy()
        snap = _snapshot(s)
        st = s.status()
    return h, snap, st


def _assert_same(a, b):
    ha, sa, sta = a
    hb, sb, stb = b
    assert sta == stb
    np.testing.assert_array_equal(ha, hb)
    for xa, xb in zip(sa, sb):
        for u, v in zip(xa, xb):
            np.testing.assert_array_equal(u, v)


CASES = [
    ([(2, 7, 250)], dict()),
    ([(4, 5, 1000)], dict()),
    ([(4, 5, 1000)], dict(block=128)),
    ([(4, 5, 1000)], dict(block=256)),
    ([(4, 5, 1000)], dict(block=128, persistent=1)),
    ([(3, 4, 130), (6, 3, 700), (8, 2, 2049), (2, 3, 1)], dict()),
    ([(3, 4, 130), (6, 3, 700), (8, 2, 2049), (2, 3, 1)], dict(persistent=1)),
    ([(5, 3, 4096), (2, 2, 33)], dict(block=1024)),
    ([(7, 3, 63), (4, 2, 64), (2, 2, 65)], dict(block=32)),
]


@pytest.mark.parametrize("shapes,opts", CASES)
def test_solve_is_bitwise_the_separate_calls(shapes, opts):
    from paper_1908_01964_gb300 import rcscm as R
    dev = [R.to_device(p) for p in _probs(shapes)]
    K = 9
    _assert_same(_separate(dev, K, **opts), _fused(dev, K, **opts))


def test_run_starts_from_the_initial_state_every_time():
    from paper_1908_01964_gb300 import rcscm as R
    dev = [R.to_device(p) for p in _probs([(4, 6, 300)], seed=3)]
    with R.Solver(dev) as s:
        s.setup_freq()
        h1 = s.run(7).cpu().numpy()
        s.iterate(5)                                # moves the state on
        h2 = s.run(7).cpu().numpy()
        h3 = s.solve(7).cpu().numpy()
        torch.cuda.synchronize()
    np.testing.assert_array_equal(h1, h2)
    np.testing.assert_array_equal(h1, h3)


def test_solve_zero_passes_is_the_initial_wiener_filter():
    from paper_1908_01964_gb300 import rcscm as R
    dev = [R.to_device(p) for p in _probs([(3, 4, 90)], seed=5)]
    _assert_same(_separate(dev, 0), _fused(dev, 0))


@pytest.mark.parametrize("opts", [dict(rule="naive64"), dict(iters_per_launch=3),
                                  dict(ckpt_stride=4, ckpt_max_iters=9)])
def test_solve_in_other_configurations_runs_the_separate_calls(opts):
    from paper_1908_01964_gb300 import rcscm as R
    dev = [R.to_device(p) for p in _probs([(4, 3, 200)], seed=7)]
    _assert_same(_separate(dev, 9, **opts), _fused(dev, 9, **opts))
    with R.Solver(dev, **opts) as s:               # rcscm_run itself needs the fused configuration
        s.setup()
        with pytest.raises(R.RcscmError) as ei:
            s.run(2)
        assert ei.value.code == R.EINVAL


def test_solve_matches_the_oracle():
    from paper_1908_01964_gb300 import rcscm as R
    p = _probs([(4, 9, 500)], seed=11)[0]
    with R.Solver([R.to_device(p)]) as s:
        h = s.solve(40).view(p["x"].shape).cpu().numpy()
        rh, ru, lam = (t.cpu().numpy() for t in s.get_state(0))
        torch.cuda.synchronize()
    e = compare(dict(rh=rh, ru=ru, lam=lam, h=h), oracle_run(p, 40))
    assert max(e["rh"], e["ru"], e["lam"]) < TOL_FULL_RUN and e["sdr"] > SDR_MIN_DB, e
