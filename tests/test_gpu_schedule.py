"""Batched schedule (persistent launch, CUDA graph, autotuner) and the objective
kernel, against the one-CTA-per-row path and the FP64 oracle.  Needs a GPU."""
import numpy as np
import pytest

from oracle import rcscm_oracle as O
from paper_1908_01964_gb300 import synth
from parity_util import ALPHA, BETA, SDR_MIN_DB, TOL_FULL_RUN, compare, gpu_run, oracle_run, rel, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1908_01964_gb300 import build, rcscm
    build.build()
    rcscm.lib()


def _batch(n=6, I=33, seed=700, max_j=2000):
    rng = np.random.default_rng(seed)
    specs = [synth.ProblemSpec(M=int(rng.choice([2, 4, 6])), I=I, J=int(rng.integers(100, max_j + 1)), K=5,
                               spacing=0.04)
             for _ in range(n)]
    return [synth.make_problem(s, seed + k) for k, s in enumerate(specs)]


@pytest.mark.parametrize("block", [128, 256, 512])
def test_persistent_launch_equals_one_cta_per_row(block):
    probs = _batch(max_j=8 * block)                 # rows of up to 8 * block frames
    a, _ = gpu_run(probs, 12, block=block, persistent=0)
    b, _ = gpu_run(probs, 12, block=block, persistent=1)
    for x, y in zip(a, b):
        for k in ("rh", "ru", "lam", "h"):
            np.testing.assert_array_equal(x[k], y[k])


def test_graph_replay_equals_direct_calls():
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    probs = _batch(n=4, seed=710)
    dev = [R.to_device(p) for p in probs]
    with R.Solver(dev, persistent=1) as s:
        s.setup()
        s.iterate(15)
        ref = s.extract().clone()
        ref_state = [t.clone() for t in s.get_state(2)]
        out = torch.empty_like(ref)
        s.graph_create(15, out)
        for _ in range(2):                    # replays restart from the inputs each time
            out.zero_()
            s.graph_launch()
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
            for u, v in zip(s.get_state(2), ref_state):
                assert torch.equal(u, v)
        assert s.status() == R.OK


def test_autotune_keeps_state_and_results_stay_within_tolerance():
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    probs = _batch(n=5, seed=720)
    dev = [R.to_device(p) for p in probs]
    with R.Solver(dev) as s:
        s.setup()
        s.iterate(3)
        before = [[t.clone() for t in s.get_state(k)] for k in range(len(probs))]
        block, pers = s.autotune(n_iter_probe=5)
        assert block in (32, 64, 128, 256, 512, 1024) and pers in (0, 1)
        for k in range(len(probs)):
            for u, v in zip(s.get_state(k), before[k]):
                assert torch.equal(u, v)
        s.iterate(17)
        h = s.split(s.extract())
        for k, p in enumerate(probs):
            rh, ru, lam = (t.cpu().numpy() for t in s.get_state(k))
            e = compare(dict(rh=rh, ru=ru, lam=lam, h=h[k].cpu().numpy()), oracle_run(p, 20))
            assert max(e["rh"], e["ru"], e["lam"]) < TOL_FULL_RUN, e
            assert e["sdr"] > SDR_MIN_DB, e
    report("autotune_choice", block=block, persistent=pers)


def test_objective_matches_oracle_at_the_same_state():
    from paper_1908_01964_gb300 import rcscm as R
    probs = _batch(n=3, I=17, seed=730)
    dev = [R.to_device(p) for p in probs]
    with R.Solver(dev) as s:
        s.setup()
        for n in (0, 4):
            s.iterate(n)
            got = s.objective()
            for k, p in enumerate(probs):
                rh, ru, lam = (t.cpu().numpy().astype(np.float64) for t in s.get_state(k))
                st = O.setup(p["a"], p["Rp"])
                want = O.objective(rh, ru, lam, p["x"].astype(np.complex128), p["a"], st, ALPHA, BETA)
                report("objective", n_iter=n, gpu=got[k], oracle=want)
                assert abs(got[k] - want) <= 1e-5 * abs(want), (got[k], want)


def test_objective_is_non_decreasing_on_gpu():
    from paper_1908_01964_gb300 import rcscm as R
    p = synth.make_workload(synth.workload("plain-m2"))[0]
    with R.Solver([R.to_device(p)]) as s:
        s.setup()
        vals = [s.objective()[0]]
        for _ in range(30):
            s.iterate(1)
            vals.append(s.objective()[0])
    d = np.diff(vals)
    # FP32 per-slot terms summed in FP64: allow rounding-level decreases only
    assert np.all(d >= -2e-6 * np.abs(vals[1:])), d


def test_batch_subset_of_batch_256_sampled_rows():
    """24 utterances of the batch workload (uneven J, mixed M) in one persistent,
    autotuned launch; the oracle runs on sampled rows of every utterance."""
    wl = synth.workload("batch-256", n_utt=24)
    probs = synth.make_workload(wl)
    outs, st = gpu_run(probs, wl.n_iter, persistent=1)
    assert st == 0
    rng = np.random.default_rng(1)
    for p, g in zip(probs, outs):
        rows = sorted(set([0, p["x"].shape[0] - 1] + list(rng.choice(p["x"].shape[0], 3, replace=False))))
        e = compare(g, oracle_run(p, wl.n_iter, rows=rows), rows=rows)
        assert max(e["rh"], e["ru"], e["lam"]) < TOL_FULL_RUN, e
        assert e["sdr"] > SDR_MIN_DB, e


def test_sharded_batch_equals_unsharded():
    # the shards two ranks would solve, run one after another on this GPU, give bit for
    # bit the per-utterance results of the whole batch (same block size)
    import bench
    probs = _batch(n=7, seed=900, max_j=2048)
    whole, _ = gpu_run(probs, 10, block=256)
    weights = [p["x"].shape[0] * p["x"].shape[1] for p in probs]
    for rank in range(2):
        mine = bench.shard(weights, rank, 2)
        part, _ = gpu_run([probs[i] for i in mine], 10, block=256)
        for i, out in zip(mine, part):
            for k in ("rh", "ru", "lam", "h"):
                np.testing.assert_array_equal(out[k], whole[i][k])


def test_frequency_ranges_equal_unsharded():
    # one utterance split into the contiguous frequency ranges that two ranks would
    # solve, run one after another on this GPU: bit for bit the rows of the whole
    # utterance (rows are independent; every range runs the same kernel shape)
    import bench
    p = synth.make_problem(synth.ProblemSpec(M=4, I=37, J=1000, K=5, spacing=0.03), 950)
    (whole,), _ = gpu_run([p], 12)
    for rank in range(2):
        i0, i1 = bench.freq_range(37, rank, 2)
        (part,), st = gpu_run([bench.slice_rows(p, i0, i1)], 12)
        assert st == 0
        for k in ("rh", "ru", "lam", "h"):
            np.testing.assert_array_equal(part[k], whole[k][i0:i1])
