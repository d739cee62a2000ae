"""The no-allocation entry point, rcscm_solve_noalloc, called through the C ABI.

Some callers of this library cannot allocate device memory while they run: a
real-time audio thread cannot risk the device-wide synchronisation and
unbounded stall a cudaMalloc may cause, and some host applications give the
library a fixed GPU memory budget up front.  rcscm_solve_noalloc serves them
from one fixed array inside the library.  These tests check that it returns
what the context-based entry points return, on two calls in a row (the second
call must not be disturbed by what the first left in the shared array), that a
call leaves the device's free memory and PyTorch's allocator untouched, and
that a problem too large for the array, an address the device cannot reach
(pageable host memory) and the options the entry point does not offer are
refused before any work starts.

This file is named so that pytest collects it after every other test file.
"""
import ctypes

import numpy as np
import pytest

from paper_1908_01964_gb300 import synth
from parity_util import SDR_MIN_DB, TOL_ONE_ITER, gpu_run, rel, sdr_db

pytestmark = pytest.mark.gpu


def _noalloc(p, n_iter):
    import torch
    from paper_1908_01964_gb300 import build, rcscm as R
    build.build()
    L = R.lib()
    d = R.to_device(p)
    I, J, M = p["x"].shape
    rh = torch.full((I, J), float("nan"), dtype=torch.float32, device="cuda")
    ru = torch.full_like(rh, float("nan"))
    lam = torch.full((I,), float("nan"), dtype=torch.float32, device="cuda")
    h = torch.full((I, J, M), float("nan"), dtype=torch.complex64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    o = R.options()
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    code = L.rcscm_solve_noalloc(I, J, M, vp(d["x"]), vp(d["a"]), vp(d["Rp"]), None, vp(d["rh0"]), vp(d["ru0"]),
                                 ctypes.byref(o), n_iter, vp(rh), vp(ru), vp(lam), vp(h), vp(status),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert code == R.OK, R.strerror(code)
    return dict(rh=rh.cpu().numpy(), ru=ru.cpu().numpy(), lam=lam.cpu().numpy(), h=h.cpu().numpy(),
                status=int(status.item()))


def test_noalloc_matches_context_entry_points_on_two_calls():
    specs = [(synth.ProblemSpec(M=4, I=257, J=1000, K=10, spacing=0.03), 91, 20),
             (synth.ProblemSpec(M=6, I=129, J=333, K=5, spacing=0.04), 92, 7)]
    for spec, seed, n_iter in specs:          # two calls in a row, different shapes
        p = synth.make_problem(spec, seed)
        (ref,), ref_status = gpu_run([p], n_iter)
        got = _noalloc(p, n_iter)
        assert got["status"] == ref_status == 0
        for k in ("rh", "ru", "lam"):
            assert rel(got[k], ref[k]) < TOL_ONE_ITER, k
        assert sdr_db(got["h"], ref["h"]) > SDR_MIN_DB


def test_noalloc_refuses_a_problem_larger_than_its_array():
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    L = R.lib()
    I, J, M = 2049, 4000, 8                    # 8.2 M slots: more than the fixed array holds
    fake = ctypes.c_void_p(0x1000)             # never dereferenced: refused before any launch
    o = R.options()
    code = L.rcscm_solve_noalloc(I, J, M, fake, fake, fake, None, fake, fake, ctypes.byref(o), 10,
                                 fake, fake, fake, fake, None, None)
    assert code == R.ECAPACITY
    assert "fixed scratch" in R.strerror(code)
    torch.cuda.synchronize()


def _buffers(p):
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    d = R.to_device(p)
    I, J, M = p["x"].shape
    out = dict(rh=torch.empty((I, J), dtype=torch.float32, device="cuda"),
               ru=torch.empty((I, J), dtype=torch.float32, device="cuda"),
               lam=torch.empty((I,), dtype=torch.float32, device="cuda"),
               h=torch.empty((I, J, M), dtype=torch.complex64, device="cuda"),
               status=torch.zeros((1,), dtype=torch.int32, device="cuda"))
    return d, out


def _call(L, p, d, out, n_iter, o, **override):
    import torch
    I, J, M = p["x"].shape
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    args = dict(x=vp(d["x"]), a=vp(d["a"]), Rp=vp(d["Rp"]), rh0=vp(d["rh0"]), ru0=vp(d["ru0"]))
    args.update(override)
    return L.rcscm_solve_noalloc(I, J, M, args["x"], args["a"], args["Rp"], None, args["rh0"], args["ru0"],
                                 ctypes.byref(o), n_iter, vp(out["rh"]), vp(out["ru"]), vp(out["lam"]),
                                 vp(out["h"]), vp(out["status"]),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_call_leaves_device_memory_unchanged():
    """After a first call on the device (which loads the module and its fixed array),
    a call changes neither the device's free memory nor PyTorch's allocator."""
    import torch
    from paper_1908_01964_gb300 import build, rcscm as R
    build.build()
    L = R.lib()
    p = synth.make_problem(synth.ProblemSpec(M=4, I=65, J=300, K=5, spacing=0.03), 95)
    d, out = _buffers(p)
    o = R.options()
    assert _call(L, p, d, out, 5, o) == R.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    assert _call(L, p, d, out, 5, o) == R.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for k in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(k, 0) == stats0.get(k, 0), k
    assert int(out["status"].item()) == 0


def test_noalloc_refuses_pageable_host_memory_and_unsupported_options():
    import numpy as np_
    import torch
    from paper_1908_01964_gb300 import build, rcscm as R
    build.build()
    L = R.lib()
    p = synth.make_problem(synth.ProblemSpec(M=4, I=9, J=64, K=3, spacing=0.03), 96)
    d, out = _buffers(p)
    out["h"].fill_(float("nan"))
    pageable = np_.ascontiguousarray(p["x"], np_.complex64)          # ordinary (pageable) host memory
    code = _call(L, p, d, out, 3, R.options(), x=ctypes.c_void_p(pageable.ctypes.data))
    assert code == R.EINVAL
    o = R.options(persistent=1)
    assert _call(L, p, d, out, 3, o) == R.EINVAL
    o = R.options(ckpt_stride=2, ckpt_max_iters=4)
    assert _call(L, p, d, out, 3, o) == R.EINVAL
    torch.cuda.synchronize()
    assert torch.isnan(out["h"]).all()                                # nothing was launched
