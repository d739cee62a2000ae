"""Boundary options of rcscm_create, called through the C ABI: a caller-supplied
null vector b_i of R'_i (Sec. II-B-1; validated by the setup) and R'_i given as
complex64.  Needs a GPU; marked `gpu`."""
import numpy as np
import pytest

from oracle import rcscm_oracle as O
from paper_1908_01964_gb300 import synth
from parity_util import SDR_MIN_DB, TOL_ONE_ITER, compare, norm_max, oracle_run, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1908_01964_gb300 import build, rcscm
    build.build()
    rcscm.lib()
    torch.cuda.init()


def _problem(M, seed, I=17, J=200):
    return synth.make_problem(synth.ProblemSpec(M=M, I=I, J=J, K=5, spacing=0.03), seed)


def _solve(dev_prob, n_iter):
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    with R.Solver([dev_prob]) as s:
        s.setup()
        s.iterate(n_iter)
        h = s.extract()
        code = s.status()
        rh, ru, lam = s.get_state(0)
        out = dict(rh=rh.cpu().numpy(), ru=ru.cpu().numpy(), lam=lam.cpu().numpy(),
                   h=h.view(dev_prob["x"].shape).cpu().numpy())
        torch.cuda.synchronize()
    return out, code


@pytest.mark.parametrize("M", [2, 4, 7])
def test_caller_b_accepted_and_results_unchanged(M):
    """A correct b (any phase) passes the validation and changes nothing: the
    estimator uses the eigenvector of the smallest eigenvalue either way."""
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    p = _problem(M, 300 + M)
    st = O.setup(p["a"], p["Rp"])
    phase = np.exp(1j * np.random.default_rng(M).uniform(0, 2 * np.pi, size=(st.b.shape[0], 1)))
    d = R.to_device(p)
    ref, code0 = _solve(d, 4)
    d["b"] = torch.from_numpy(np.ascontiguousarray(st.b * phase)).cuda()
    got, code1 = _solve(d, 4)
    assert code0 == code1 == R.OK
    for k in ("rh", "ru", "lam", "h"):
        np.testing.assert_array_equal(got[k], ref[k])


@pytest.mark.parametrize("M", [2, 4, 7])
def test_caller_b_not_in_the_null_space_is_refused(M):
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    p = _problem(M, 310 + M)
    st = O.setup(p["a"], p["Rp"])
    bad = st.b.copy()
    bad[5] = st.b[5] + 0.01 * np.roll(st.b[5], 1)              # one row off its null vector
    d = R.to_device(p)
    d["b"] = torch.from_numpy(np.ascontiguousarray(bad)).cuda()
    _, code = _solve(d, 1)
    assert code == R.ENULLSPACE
    d["b"] = torch.from_numpy(np.ascontiguousarray(st.b)).cuda()
    _, code = _solve(d, 1)
    assert code == R.OK


@pytest.mark.parametrize("M", [2, 4, 8])
def test_complex64_noise_scm(M):
    """R' given as complex64 is widened exactly, so the result equals the complex128
    run on the same rounded values bit for bit, and it meets the one-pass bar
    against the oracle on those values."""
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    p = _problem(M, 320 + M, I=33, J=300)
    rp32 = np.ascontiguousarray(p["Rp"], np.complex64)
    q = dict(p, Rp=rp32.astype(np.complex128))
    d64 = R.to_device(q)
    d32 = dict(d64, Rp=torch.from_numpy(rp32).cuda())
    a, ca = _solve(d64, 1)
    b, cb = _solve(d32, 1)
    assert ca == cb == R.OK
    for k in ("rh", "ru", "lam", "h"):
        np.testing.assert_array_equal(a[k], b[k])
    e = compare(b, oracle_run(q, 1))
    report("complex64_noise_scm_one_iter", M=M, gpu=e)
    assert norm_max(e) < TOL_ONE_ITER and e["sdr"] > SDR_MIN_DB, e
