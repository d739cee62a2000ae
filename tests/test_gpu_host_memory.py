"""Problem buffers and outputs in page-locked host memory, read and written in
place by the kernels: results equal the device-resident path bit for bit, and
any other host memory is refused by the library before anything runs."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1908_01964_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _host(prob, pinned=True):
    out = {}
    for k, dt in (("x", np.complex64), ("a", np.complex128), ("Rp", np.complex128), ("rh0", np.float32),
                  ("ru0", np.float32)):
        t = torch.from_numpy(np.ascontiguousarray(prob[k], dt))
        out[k] = t.pin_memory() if pinned else t
    return out


@pytest.mark.parametrize("fused", [True, False])
def test_pinned_host_buffers_equal_the_device_path(fused):
    from paper_1908_01964_gb300 import rcscm as R
    probs = [synth.tiny(M=M, I=6, J=J, K=4, seed=80 + M) for M, J in ((4, 300), (2, 77))]
    with R.Solver([R.to_device(p) for p in probs]) as s:
        ref = s.solve(9).cpu().numpy()
        ref_state = [t.cpu().numpy() for t in s.get_state(1)]
    hp = [_host(p) for p in probs]
    with R.Solver(hp) as s:
        n = s.out_elements
        if fused:
            h = torch.empty(n, dtype=torch.complex64).pin_memory()
            s.solve(9, out=h)
        else:
            s.setup()
            s.iterate(9)
            h = torch.empty(n, dtype=torch.complex64).pin_memory()
            s.extract(out=h)
        torch.cuda.synchronize()
        state = [t.cpu().numpy() for t in s.get_state(1)]
    np.testing.assert_array_equal(h.numpy(), ref)
    for a, b in zip(state, ref_state):
        np.testing.assert_array_equal(a, b)


def test_pageable_host_memory_is_refused():
    from paper_1908_01964_gb300 import rcscm as R
    p = synth.tiny(M=3, I=2, J=20, K=3, seed=1)
    arrs = {k: np.ascontiguousarray(p[k], dt) for k, dt in (("x", np.complex64), ("a", np.complex128),
                                                           ("Rp", np.complex128), ("rh0", np.float32),
                                                           ("ru0", np.float32))}
    q = R.Problem()
    q.I, q.J, q.M = 2, 20, 3
    q.x, q.a, q.Rp = (ctypes.c_void_p(arrs[k].ctypes.data) for k in ("x", "a", "Rp"))
    q.rh0, q.ru0 = (ctypes.c_void_p(arrs[k].ctypes.data) for k in ("rh0", "ru0"))
    q.lambda0 = None
    o = R.options()
    ctx = ctypes.c_void_p()
    code = R.lib().rcscm_create(ctypes.byref(ctx), ctypes.byref(q), 1, ctypes.byref(o), None)
    assert code == R.EINVAL and not ctx.value
    with R.Solver([R.to_device(p)]) as s:               # pageable output buffer
        s.setup()
        h = np.zeros(s.out_elements, np.complex64)
        code = R.lib().rcscm_extract(s.ctx, ctypes.c_void_p(h.ctypes.data), None)
        assert code == R.EINVAL
        torch.cuda.synchronize()
    with pytest.raises(TypeError):                       # the binding refuses it first
        R.Solver([_host(p, pinned=False)])
