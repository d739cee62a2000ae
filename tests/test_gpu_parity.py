"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle on
the same seeded inputs.  Needs a GPU; marked `gpu`."""
import numpy as np
import pytest

from oracle import rcscm_oracle as O
from paper_1908_01964_gb300 import synth
from parity_util import (ALPHA, BETA, ELEM_FULL_RUN, ELEM_ONE_ITER, SDR_MIN_DB, TOL_FULL_RUN, TOL_ONE_ITER, compare,
                         elem_max, elementwise, gpu_run, kappa_fp32_bound, norm_max, oracle_run, rel, report, sdr_db)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1908_01964_gb300 import build, rcscm
    build.build()
    rcscm.lib()
    torch.cuda.init()


def _tiny(M, I=7, J=37, seed=3, K=4):
    return synth.make_problem(synth.ProblemSpec(M=M, I=I, J=J, K=K, spacing=0.03), seed)


# ------------------------------------------------------------------ A0 setup

@pytest.mark.parametrize("M", [2, 3, 4, 5, 6, 7, 8])
def test_setup_matches_oracle(M):
    from paper_1908_01964_gb300 import rcscm as R
    p = _tiny(M, I=9, seed=M)
    st = O.setup(p["a"], p["Rp"])
    with R.Solver([R.to_device(p)]) as s:
        s.setup()
        g = {k: v.cpu().numpy() for k, v in s.get_setup(0).items()}
        assert s.status() == R.OK
    muM = st.mu[:, -1:]
    assert np.max(np.abs(g["mu"] - st.mu) / muM) < 1e-12
    np.testing.assert_allclose(g["lambda0"], st.lam0, rtol=1e-9)
    np.testing.assert_allclose(g["tau_aa"], st.tau_aa, rtol=1e-9)
    # b is defined up to a phase: compare |b_gpu^H b_oracle| and phase-free products
    overlap = np.abs(np.einsum("im,im->i", np.conj(g["b"]), st.b))
    np.testing.assert_allclose(overlap, 1.0, atol=1e-10)
    np.testing.assert_allclose(np.abs(g["sigma_ab"]), np.abs(st.sigma_ab), rtol=1e-9)
    np.testing.assert_allclose(g["sigma_ab"], np.einsum("im,im->i", np.conj(p["a"]), g["b"]), atol=1e-12)


@pytest.mark.parametrize("M,ratio", [(2, 1e-7), (4, 1e-6), (4, 2e-7), (6, 5e-7), (8, 1e-7)])
def test_setup_resolves_close_small_eigenvalues(M, ratio):
    """R' whose two smallest eigenvalues (the null one and mu_2) are ratio * |R'| apart, as
    ILRMA's noise estimate gives at low frequencies: a few FP32 units of |R'|, below what
    the FP32 Jacobi resolves; the setup must still return the FP64 null vector and the
    estimator the oracle's result."""
    from paper_1908_01964_gb300 import rcscm as R
    p = _tiny(M, I=6, J=200, seed=90 + M)
    rng = np.random.default_rng(M)
    I = p["x"].shape[0]
    Rp = np.empty((I, M, M), np.complex128)
    for i in range(I):
        Z = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
        E, _ = np.linalg.qr(Z)
        mu = np.concatenate([[0.0, ratio * (1 + i)], np.sort(rng.uniform(0.2, 1.0, M - 2))])
        Rp[i] = (E * mu) @ np.conj(E.T)
    p["Rp"] = 0.5 * (Rp + np.conj(np.transpose(Rp, (0, 2, 1))))
    st = O.setup(p["a"], p["Rp"])
    with R.Solver([R.to_device(p)]) as s:
        s.setup()
        g = {k: v.cpu().numpy() for k, v in s.get_setup(0).items()}
        assert s.status() == R.OK
    overlap = np.abs(np.einsum("im,im->i", np.conj(g["b"]), st.b))
    report("setup_close_eigenvalues", M=M, ratio=ratio, b_angle=float(np.max(1 - overlap)),
           tau_aa=float(np.max(np.abs(g["tau_aa"] / st.tau_aa - 1))))
    np.testing.assert_allclose(overlap, 1.0, atol=1e-10)
    # lambda_0 = mu_2 is ratio * |R'|: its attainable absolute accuracy is a small multiple of
    # the FP64 rounding of |R'| (the largest eigenvalue), not of mu_2 itself
    assert np.max(np.abs(g["lambda0"] - st.lam0) / st.mu[:, -1]) < 1e-10
    np.testing.assert_allclose(g["tau_aa"], st.tau_aa, rtol=1e-8)
    (o,), code = gpu_run([p], 3)
    e = compare(o, oracle_run(p, 3))
    report("solve_close_eigenvalues", M=M, ratio=ratio, gpu=e)
    assert code == 0 and norm_max(e) < 1e-4 and e["sdr"] > SDR_MIN_DB, e


def test_setup_uses_given_lambda0():
    from paper_1908_01964_gb300 import rcscm as R
    p = _tiny(4)
    p["lambda0"] = np.linspace(0.3, 2.0, p["x"].shape[0])
    with R.Solver([R.to_device(p)]) as s:
        s.setup()
        lam0 = s.get_setup(0)["lambda0"].cpu().numpy()
        lam = s.get_state(0)[2].cpu().numpy()
    np.testing.assert_array_equal(lam0, p["lambda0"])
    np.testing.assert_allclose(lam, p["lambda0"], rtol=1e-7)


# ------------------------------------------------------------------ A1 invariants

@pytest.mark.parametrize("M", [2, 4, 6, 8])
def test_invariants_match_oracle(M):
    from paper_1908_01964_gb300 import rcscm as R
    p = _tiny(M, I=11, J=300, seed=10 + M)
    x = p["x"].astype(np.complex128)
    st = O.setup(p["a"], p["Rp"])
    inv = O.invariants(x, p["a"], st)
    with R.Solver([R.to_device(p)]) as s:
        s.setup()
        g = {k: v.cpu().numpy() for k, v in s.get_invariants(0).items()}
        b_gpu = s.get_setup(0)["b"].cpu().numpy()
        sab_gpu = s.get_setup(0)["sigma_ab"].cpu().numpy()
    assert rel(g["tau_ax"], inv.tau_ax) < 1e-5
    kappa = inv.tau_xx - np.abs(inv.tau_ax) ** 2 / st.tau_aa[:, None]
    assert np.all(g["kappa"] >= 0)
    # 1e-5 of tau_xx, or the FP32 forward error bound of the projection where that is larger
    tol = np.maximum(1e-5 * inv.tau_xx, kappa_fp32_bound(x, p["a"], st, kappa))
    assert np.all(np.abs(g["kappa"] - kappa) <= tol), np.max(np.abs(g["kappa"] - kappa) / tol)
    # sigma_bx follows the GPU's b; the product sigma_ab sigma_bx is phase free
    assert rel(sab_gpu[:, None] * g["sigma_bx"], st.sigma_ab[:, None] * inv.sigma_bx) < 1e-5
    assert rel(g["sigma_bx"], np.einsum("im,ijm->ij", np.conj(b_gpu), x)) < 1e-5


# ------------------------------------------------------------------ A2-A4 accelerated iteration

@pytest.mark.parametrize("name", ["plain-m2", "m4-small"])
def test_accel_one_iteration(name):
    if name == "plain-m2":
        p = synth.make_workload(synth.workload("plain-m2"))[0]
    else:
        p = synth.make_problem(synth.ProblemSpec(M=4, I=129, J=333, K=20, spacing=0.03), 77)
    (g,), st = gpu_run([p], 1)
    o = oracle_run(p, 1)
    e = compare(g, o)
    report("accel_one_iter", case=name, gpu=e)
    assert st == 0, st
    assert max(e["rh"], e["ru"], e["lam"]) < TOL_ONE_ITER, e
    assert e["sdr"] > SDR_MIN_DB, e
    assert elem_max(e, 0) < ELEM_ONE_ITER[0] and elem_max(e, 1) < ELEM_ONE_ITER[1], e


def test_accel_full_run_plain_m2():
    wl = synth.workload("plain-m2")
    p = synth.make_workload(wl)[0]
    (g,), st = gpu_run([p], wl.n_iter)
    o = oracle_run(p, wl.n_iter)
    e = compare(g, o)
    report("accel_full_run_plain_m2", gpu=e)
    assert st == 0
    assert max(e["rh"], e["ru"], e["lam"]) < TOL_FULL_RUN, e
    assert e["sdr"] > SDR_MIN_DB, e
    assert elem_max(e, 0) < ELEM_FULL_RUN[0] and elem_max(e, 1) < ELEM_FULL_RUN[1], e


@pytest.mark.parametrize("M,J,block", [(2, 1, 0), (3, 2, 128), (4, 31, 0), (5, 129, 128), (6, 257, 256),
                                       (7, 1000, 256), (8, 1023, 1024), (4, 2049, 512), (4, 4096, 0),
                                       (2, 4096, 1024), (4, 700, 512)])
def test_accel_edge_shapes(M, J, block):
    p = synth.make_problem(synth.ProblemSpec(M=M, I=5, J=J, K=3, spacing=0.04), 1000 + J + M)
    (g,), st = gpu_run([p], 3, block=block)
    o = oracle_run(p, 3)
    e = compare(g, o)
    assert max(e["rh"], e["ru"], e["lam"]) < 1e-5, e
    assert e["sdr"] > SDR_MIN_DB, e


def test_batch_mixed_m_and_j():
    specs = [synth.ProblemSpec(M=M, I=33, J=J, K=5, spacing=0.04)
             for M, J in ((2, 200), (4, 1999), (6, 731), (4, 256), (3, 17), (8, 1500))]
    probs = [synth.make_problem(s, 500 + k) for k, s in enumerate(specs)]
    outs, st = gpu_run(probs, 10)
    assert st == 0
    for p, g in zip(probs, outs):
        e = compare(g, oracle_run(p, 10))
        assert max(e["rh"], e["ru"], e["lam"]) < 1e-4, e
        assert e["sdr"] > SDR_MIN_DB, e


def test_streaming_launches_equal_resident_bitwise():
    p = _tiny(4, I=17, J=900, seed=4)
    (g0,), _ = gpu_run([p], 7)
    (g1,), _ = gpu_run([p], 7, iters_per_launch=1)
    (g2,), _ = gpu_run([p], 7, iters_per_launch=3)
    for k in ("rh", "ru", "lam", "h"):
        np.testing.assert_array_equal(g0[k], g1[k])
        np.testing.assert_array_equal(g0[k], g2[k])


def test_resume_is_bitwise_and_deterministic():
    p = _tiny(4, I=17, J=900, seed=5)
    (a,), _ = gpu_run([p], 10)
    (b,), _ = gpu_run([p], 10, chunks=[4, 6])
    (c,), _ = gpu_run([p], 10)
    for k in ("rh", "ru", "lam", "h"):
        np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a[k], c[k])


def test_get_set_state_roundtrip():
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    p = _tiny(3, I=6, J=50)
    with R.Solver([R.to_device(p)]) as s:
        s.setup()
        s.iterate(3)
        rh, ru, lam = s.get_state(0)
        s.iterate(2)
        ref = [t.clone() for t in s.get_state(0)]
        s.set_state(0, rh, ru, lam)
        s.iterate(2)
        got = s.get_state(0)
        for u, v in zip(got, ref):
            assert torch.equal(u, v)


def test_rows_independent_in_batch():
    # the same utterance alone and inside a batch gives bitwise-equal results
    p = _tiny(4, I=9, J=400, seed=8)
    q = _tiny(6, I=5, J=1200, seed=9)
    (alone,), _ = gpu_run([p], 6, block=256)           # same block size -> same reduction tree
    (first, _), _ = gpu_run([p, q], 6, block=256)
    for k in ("rh", "ru", "lam", "h"):
        np.testing.assert_array_equal(alone[k], first[k])


# ------------------------------------------------------------------ A5 naive rule

def _naive_printed_fp32_error(p, n_iter):
    """Error of the naive rule evaluated with the oracle's own formulas, in the
    printed coordinates, in single precision (numpy complex64 / float32) against
    the FP64 oracle: the accuracy FP32 arithmetic allows for the literal E-step,
    whose difference r~_h - r~_h^2 a^H P a cancels when r~_h rho~ >> r~_u and
    whose per-slot inverse inherits the condition number of R~_i."""
    st = O.setup(p["a"], p["Rp"])
    rh, ru, lam = p["rh0"], p["ru0"], st.lam0.astype(np.float32)
    for _ in range(n_iter):
        rh, ru, lam = O.iterate_naive(rh, ru, lam, p["x"], p["a"], st, ALPHA, BETA, dtype=np.complex64)
    o = oracle_run(p, n_iter, rule="naive")
    return dict(rh=rel(rh, o["rh"]), ru=rel(ru, o["ru"]), lam=rel(lam, o["lam"])), o


@pytest.mark.parametrize("M", [2, 3, 4, 5, 6, 7, 8])
def test_naive_fp32_one_iteration(M):
    """The FP32 naive rule (per-slot explicit inverse in the whitened coordinates of
    R~_i) after one pass: the same bars as the accelerated rule."""
    p = synth.make_problem(synth.ProblemSpec(M=M, I=33, J=301, K=10, spacing=0.03), 40 + M)
    (g,), st = gpu_run([p], 1, rule="naive")
    o = oracle_run(p, 1, rule="naive")
    e = compare(g, o)
    report("naive_one_iter", M=M, gpu=e, status=st)
    assert st == 0, st
    assert norm_max(e) < TOL_ONE_ITER, e
    assert e["sdr"] > SDR_MIN_DB, e
    assert elem_max(e, 0) < ELEM_ONE_ITER[0] and elem_max(e, 1) < ELEM_ONE_ITER[1], e


@pytest.mark.parametrize("M,n_iter", [(2, 50), (4, 20), (6, 20), (8, 10)])
def test_naive_fp32_full_runs(M, n_iter):
    p = synth.make_problem(synth.ProblemSpec(M=M, I=65, J=250, K=10, spacing=0.04), 60 + M)
    (g,), st = gpu_run([p], n_iter, rule="naive")
    o = oracle_run(p, n_iter, rule="naive")
    e = compare(g, o)
    report("naive_fp32_full_run", M=M, n_iter=n_iter, gpu=e, status=st)
    assert st == 0, st
    assert norm_max(e) < TOL_FULL_RUN, e
    assert e["sdr"] > SDR_MIN_DB, e
    assert elem_max(e, 0) < ELEM_FULL_RUN[0] and elem_max(e, 1) < ELEM_FULL_RUN[1], e


def test_naive_fp32_full_run_plain_m2():
    """The plain M = 2 workload over its 50 passes, whose low bins are the worst
    conditioned (the printed-coordinates FP32 rule leaves 1e-2 there)."""
    wl = synth.workload("plain-m2")
    p = synth.make_workload(wl)[0]
    (g,), st = gpu_run([p], wl.n_iter, rule="naive")
    o = oracle_run(p, wl.n_iter, rule="naive")
    e = compare(g, o)
    report("naive_fp32_full_run_plain_m2", gpu=e, status=st)
    assert st == 0, st
    assert norm_max(e) < TOL_FULL_RUN, e
    assert e["sdr"] > SDR_MIN_DB, e
    assert elem_max(e, 0) < ELEM_FULL_RUN[0] and elem_max(e, 1) < ELEM_FULL_RUN[1], e


def test_naive_fp32_single_m4_full_size_sampled_rows():
    """The benchmarked workload with the FP32 naive rule (100 passes), as the
    accelerated-vs-naive ratio times it, on sampled rows including the lowest
    bins and the Nyquist bin."""
    wl = synth.workload("single-m4")
    p = synth.make_workload(wl)[0]
    (g,), st = gpu_run([p], wl.n_iter, rule="naive")
    I = p["x"].shape[0]
    rows = [0, 1, 2, 3, 300, 700, I - 1]
    o = oracle_run(p, wl.n_iter, rule="naive", rows=rows)
    e = compare(g, o, rows=rows)
    report("naive_fp32_single_m4_full_size", rows=len(rows), gpu=e, status=st)
    assert st == 0, st
    assert norm_max(e) < TOL_FULL_RUN, e
    assert e["sdr"] > SDR_MIN_DB, e
    assert elem_max(e, 0) < ELEM_FULL_RUN[0] and elem_max(e, 1) < ELEM_FULL_RUN[1], e


def test_naive_fp32_agrees_with_accel_gpu_plain_m2():
    """Two GPU rules that share no per-slot arithmetic agree over a full run."""
    wl = synth.workload("plain-m2")
    p = synth.make_workload(wl)[0]
    (gn,), sn = gpu_run([p], wl.n_iter, rule="naive")
    (ga,), _ = gpu_run([p], wl.n_iter)
    e = {k: rel(ga[k], gn[k]) for k in ("rh", "ru", "lam")}
    e["sdr"] = sdr_db(ga["h"], gn["h"])
    report("accel_vs_naive_fp32_plain_m2", gpu=e, status=sn)
    assert sn == 0
    assert max(e["rh"], e["ru"], e["lam"]) < TOL_FULL_RUN, e
    assert e["sdr"] > SDR_MIN_DB, e


@pytest.mark.parametrize("M", [2, 4, 8])
def test_naive_printed_fp32_one_iteration_within_its_accuracy(M):
    """The naive rule in FP32 in the printed coordinates (kept for timing the
    literal form): within 10x of what the same formulas give in numpy complex64."""
    p = synth.make_problem(synth.ProblemSpec(M=M, I=33, J=301, K=10, spacing=0.03), 40 + M)
    e32, o = _naive_printed_fp32_error(p, 1)
    (g,), st = gpu_run([p], 1, rule="naive_printed")
    e = compare(g, o)
    report("naive_printed_one_iter", M=M, gpu=e, fp32_emulation=e32)
    for k in ("rh", "ru", "lam"):
        assert e[k] < max(TOL_ONE_ITER, 10 * e32[k]), (k, e, e32)


def test_naive_printed_fp32_plain_m2_stays_valid():
    """On the plain M=2 workload the printed-coordinates FP32 rule hits its
    projections (status ECLAMP) and drifts from the FP64 result; it must still
    return a valid model."""
    wl = synth.workload("plain-m2")
    p = synth.make_workload(wl)[0]
    (gn,), sn = gpu_run([p], 5, rule="naive_printed")
    o = oracle_run(p, 5, rule="naive")
    e = compare(gn, o)
    report("naive_printed_fp32_plain_m2_5iter", gpu=e, status=sn)
    assert sn in (0, 4), sn
    for k in ("rh", "ru", "lam", "h"):
        assert np.all(np.isfinite(gn[k])), k
    assert np.all(gn["rh"] > 0) and np.all(gn["ru"] > 0) and np.all(gn["lam"] > 0)


@pytest.mark.parametrize("M", [2, 3, 4, 6, 8])
def test_naive_f64_one_iteration(M):
    p = synth.make_problem(synth.ProblemSpec(M=M, I=33, J=301, K=10, spacing=0.03), 40 + M)
    (g,), st = gpu_run([p], 1, rule="naive64")
    o = oracle_run(p, 1, rule="naive")
    e = compare(g, o)
    report("naive_f64_one_iter", M=M, gpu=e, status=st)
    assert st == 0, st
    assert max(e["rh"], e["ru"], e["lam"]) < TOL_ONE_ITER, e
    assert e["sdr"] > SDR_MIN_DB, e


def test_naive_f64_full_run_plain_m2():
    wl = synth.workload("plain-m2")
    p = synth.make_workload(wl)[0]
    (g,), st = gpu_run([p], wl.n_iter, rule="naive64")
    o = oracle_run(p, wl.n_iter, rule="naive")
    e = compare(g, o)
    report("naive_f64_full_run_plain_m2", gpu=e, status=st)
    assert st == 0, st
    assert max(e["rh"], e["ru"], e["lam"]) < TOL_FULL_RUN, e
    assert e["sdr"] > SDR_MIN_DB, e


def test_naive_f64_single_m4_full_size_sampled_rows():
    wl = synth.workload("single-m4")
    p = synth.make_workload(wl)[0]
    (g,), st = gpu_run([p], wl.n_iter, rule="naive64")
    I = p["x"].shape[0]
    rows = [0, 1, 2, 300, 700, I - 1]
    o = oracle_run(p, wl.n_iter, rule="naive", rows=rows)
    e = compare(g, o, rows=rows)
    report("naive_f64_single_m4_full_size", rows=len(rows), gpu=e, status=st)
    assert st == 0, st
    assert max(e["rh"], e["ru"], e["lam"]) < TOL_FULL_RUN, e
    assert e["sdr"] > SDR_MIN_DB, e


def test_naive_f64_gpu_agrees_with_accel_gpu_plain_m2():
    """Two GPU rules that share no per-slot arithmetic agree over a full run."""
    wl = synth.workload("plain-m2")
    p = synth.make_workload(wl)[0]
    (gn,), sn = gpu_run([p], wl.n_iter, rule="naive64")
    (ga,), _ = gpu_run([p], wl.n_iter)
    e = {k: rel(ga[k], gn[k]) for k in ("rh", "ru", "lam")}
    e["sdr"] = sdr_db(ga["h"], gn["h"])
    report("accel_vs_naive_f64_plain_m2", gpu=e, status=sn)
    assert sn == 0
    assert max(e["rh"], e["ru"], e["lam"]) < TOL_FULL_RUN, e
    assert e["sdr"] > SDR_MIN_DB, e


# ------------------------------------------------------------------ status and host API

def test_status_flags_full_rank_noise_scm():
    from paper_1908_01964_gb300 import rcscm as R
    p = _tiny(4)
    p["Rp"] = p["Rp"] + 0.5 * np.eye(4)[None]          # not rank M-1 any more
    with R.Solver([R.to_device(p)]) as s:
        s.setup()
        assert s.status() == R.ENULLSPACE
        assert s.status() == R.OK                       # the word is cleared by the read


def test_status_flags_nonfinite_input():
    from paper_1908_01964_gb300 import rcscm as R
    p = _tiny(4, J=64)
    p["x"] = p["x"].copy()
    p["x"][2, 5, 1] = np.nan
    with R.Solver([R.to_device(p)]) as s:
        s.setup()
        s.iterate(2)
        assert s.status() == R.ENONFINITE


def test_solve_host_matches_device_path():
    from paper_1908_01964_gb300 import rcscm as R
    p = _tiny(4, I=13, J=250, seed=12)
    r = R.solve_host(p["x"], p["a"], p["Rp"], p["rh0"], p["ru0"], 8)
    (g,), _ = gpu_run([p], 8)
    for k in ("rh", "ru", "lam", "h"):
        np.testing.assert_array_equal(r[k], g[k])


@pytest.mark.parametrize("n_chunks,rule", [(1, "accel"), (3, "accel"), (8, "accel"), (4, "naive64")])
def test_host_plan_equals_device_path(n_chunks, rule):
    """rcscm_host_run (chunked host pipeline) returns bit for bit what the
    device-resident context returns: rows are independent and every chunk uses
    the same kernel shape."""
    from paper_1908_01964_gb300 import rcscm as R
    p = _tiny(4, I=29, J=700, seed=14)
    plan = R.HostPlan(*p["x"].shape, n_chunks=n_chunks, rule=rule)
    for _ in range(2):                          # the plan is reusable
        r = plan.run(p, 9)
        (g,), _ = gpu_run([p], 9, rule=rule)
        for k in ("rh", "ru", "lam", "h"):
            np.testing.assert_array_equal(r[k], g[k])
    plan.close()


def test_host_plan_graph_follows_addresses_and_contents():
    """The host pipeline replays a captured graph while the host addresses stay the
    same: new contents in the same page-locked buffers give the new results, and
    switching to other buffers captures again (bitwise equal to the device path)."""
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    probs = [_tiny(4, I=21, J=300, seed=s) for s in (61, 62)]
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).pin_memory()  # noqa: E731

    def buffers(p):
        return dict(x=pin(p["x"], np.complex64), a=pin(p["a"], np.complex128), Rp=pin(p["Rp"], np.complex128),
                    rh0=pin(p["rh0"], np.float32), ru0=pin(p["ru0"], np.float32),
                    h=torch.empty(p["x"].shape, dtype=torch.complex64).pin_memory())

    def run(plan, b):
        code = plan.run_ptrs(b["x"].data_ptr(), b["a"].data_ptr(), b["Rp"].data_ptr(), b["rh0"].data_ptr(),
                             b["ru0"].data_ptr(), 7, b["h"].data_ptr())
        assert code in (R.OK, R.ECLAMP), R.strerror(code)
        return b["h"].numpy().copy()

    want = [gpu_run([p], 7)[0][0]["h"] for p in probs]
    plan = R.HostPlan(*probs[0]["x"].shape, n_chunks=3)
    bufs = [buffers(p) for p in probs]
    for k in (0, 1, 0, 1):                        # other addresses: capture again
        np.testing.assert_array_equal(run(plan, bufs[k]), want[k])
    for k in (1, 0):                              # same addresses (buffer set 0), new contents: replay
        for name, dt in (("x", np.complex64), ("a", np.complex128), ("Rp", np.complex128), ("rh0", np.float32),
                         ("ru0", np.float32)):
            bufs[0][name].copy_(torch.from_numpy(np.ascontiguousarray(probs[k][name], dt)))
        np.testing.assert_array_equal(run(plan, bufs[0]), want[k])
    plan.close()


# ------------------------------------------------------------------ full-size workload (sampled rows)

def test_single_m4_full_size_sampled_rows():
    """The benchmarked workload (M=4, I=1025, J=1000, 100 passes, then the
    Wiener filter) in the bench's launch configuration; the oracle runs on a
    sample of rows (rows are independent), including the ill-conditioned
    lowest bins and the Nyquist bin."""
    wl = synth.workload("single-m4")
    p = synth.make_workload(wl)[0]
    (g,), st = gpu_run([p], wl.n_iter)
    assert st == 0
    I = p["x"].shape[0]
    rows = sorted(set([0, 1, 2, 3, I - 1] + list(np.random.default_rng(0).choice(I, 11, replace=False))))
    o = oracle_run(p, wl.n_iter, rows=rows)
    e = compare(g, o, rows=rows)
    report("accel_single_m4_full_size", rows=len(rows), gpu=e)
    assert max(e["rh"], e["ru"], e["lam"]) < TOL_FULL_RUN, e
    assert e["sdr"] > SDR_MIN_DB, e
    assert elem_max(e, 0) < ELEM_FULL_RUN[0] and elem_max(e, 1) < ELEM_FULL_RUN[1], e
    assert np.all(np.isfinite(g["h"])) and np.all(g["ru"] > 0) and np.all(g["rh"] > 0)


def test_scale_m8_precision_at_1_10_200_passes():
    """Precision at scale: M = 8 circular array, I = 2049, J = 4000 (8.2 M slots),
    200 passes.  Relative errors of r_h, r_u, lambda after passes 1, 10 and 200
    and of the extracted target, on sampled rows against the FP64 oracle."""
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    wl = synth.workload("scale-m8")
    p = synth.make_workload(wl)[0]
    I = p["x"].shape[0]
    rows = sorted(set([0, 1, 2, I // 2, I - 2, I - 1] + list(np.random.default_rng(1).choice(I, 6, replace=False))))
    hist = []
    o = O.run(p, wl.n_iter, "accel2", alpha=ALPHA, beta=BETA, rows=rows, history=hist)
    d = R.to_device(p)
    errs = {}
    with R.Solver([d]) as s:
        s.setup()
        done = 0
        for k in (1, 10, 200):
            s.iterate(k - done)
            done = k
            rh, ru, lam = (t.cpu().numpy()[rows] for t in s.get_state(0))
            orh, oru, olam = hist[k - 1]
            errs[k] = dict(rh=rel(rh, orh), ru=rel(ru, oru), lam=rel(lam, olam),
                           elem={"rh": elementwise(rh, orh), "ru": elementwise(ru, oru),
                                 "lam": elementwise(lam, olam)})
        h = s.extract().view(p["x"].shape).cpu().numpy()[rows]
        st = s.status()
        torch.cuda.synchronize()
    errs["sdr_200"] = sdr_db(h, o["h"])
    report("scale_m8_precision", rows=len(rows), errors=errs, status=st)
    assert st == 0
    assert norm_max(errs[1]) < TOL_ONE_ITER, errs
    assert norm_max(errs[10]) < TOL_FULL_RUN and norm_max(errs[200]) < TOL_FULL_RUN, errs
    assert errs["sdr_200"] > SDR_MIN_DB, errs
    assert elem_max(errs[1], 0) < ELEM_ONE_ITER[0] and elem_max(errs[1], 1) < ELEM_ONE_ITER[1], errs
    for k in (10, 200):
        assert elem_max(errs[k], 0) < ELEM_FULL_RUN[0] and elem_max(errs[k], 1) < ELEM_FULL_RUN[1], errs


# ------------------------------------------------------------------ first-stage rule (Algorithm 1)

@pytest.mark.parametrize("M,J", [(2, 300), (3, 300), (4, 300), (5, 1500), (6, 300), (7, 33), (8, 3000)])
def test_first_stage_one_pass_and_full_run(M, J):
    p = _tiny(M, I=9, J=J, seed=60 + M)
    for n_iter, tol in ((1, TOL_ONE_ITER), (30, TOL_FULL_RUN)):
        (g,), st = gpu_run([p], n_iter, rule="accel1")
        e = compare(g, oracle_run(p, n_iter, rule="accel1"))
        report("first_stage", M=M, n_iter=n_iter, gpu=e, status=st)
        assert st == 0 and max(e["rh"], e["ru"], e["lam"]) < tol and e["sdr"] > SDR_MIN_DB, (n_iter, e)


def test_first_stage_agrees_with_second_stage_gpu():
    # Algorithm 1 and Algorithm 2 compute the same updates (Sec. III-C); the two kernels
    # share no per-slot arithmetic (explicit per-row inverses against the fixed
    # projection), so agreement over many passes cross-checks both
    probs = [_tiny(M, I=6, J=J, seed=70 + M) for M, J in ((2, 100), (4, 1000), (6, 2048), (8, 3000))]
    a, sa = gpu_run(probs, 30, rule="accel1")
    b, sb = gpu_run(probs, 30, rule="accel")
    assert sa == sb == 0
    for x, y in zip(a, b):
        e = {k: rel(x[k], y[k]) for k in ("rh", "ru", "lam")}
        assert max(e.values()) < TOL_FULL_RUN and sdr_db(x["h"], y["h"]) > SDR_MIN_DB, e


def test_first_stage_single_m4_full_size_sampled_rows():
    """Algorithm 1 on the benchmarked workload (100 passes), on sampled rows
    including the lowest bins, against the oracle's Algorithm 1 with explicit FP64
    inverses."""
    wl = synth.workload("single-m4")
    p = synth.make_workload(wl)[0]
    (g,), st = gpu_run([p], wl.n_iter, rule="accel1")
    I = p["x"].shape[0]
    rows = [0, 1, 2, 3, 200, 600, I - 1]
    o = oracle_run(p, wl.n_iter, rule="accel1", rows=rows)
    e = compare(g, o, rows=rows)
    report("first_stage_single_m4_full_size", rows=len(rows), gpu=e, status=st)
    assert st == 0, st
    assert norm_max(e) < TOL_FULL_RUN and e["sdr"] > SDR_MIN_DB, e
    assert elem_max(e, 0) < ELEM_FULL_RUN[0] and elem_max(e, 1) < ELEM_FULL_RUN[1], e
