"""Runs one fixed set of small, oddly shaped cases through every kernel path of
one build of the library and saves what they return (used by
test_gpu_debug_build.py to compare the debug build, whose kernels check their
row, slot and shape indexes, with the normal build).

    python tests/debug_cases.py <library path> <output .npz>

Every case records its outputs and the status code the library returned."""
import ctypes
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(lib_path, out_path):
    import torch
    from paper_1908_01964_gb300 import rcscm as R, synth
    R.LIB_PATH = lib_path
    out, codes = {}, {}

    def tiny(M, I, J, seed, K=3):
        return synth.make_problem(synth.ProblemSpec(M=M, I=I, J=J, K=K, spacing=0.03), seed)

    batch = [tiny(M, 3, J, 40 + k) for k, (M, J) in enumerate(((2, 1), (3, 33), (5, 257), (8, 1000), (4, 64)))]
    dev = [R.to_device(p) for p in batch]
    for name, opts in (("fused", {}), ("stream", dict(iters_per_launch=1)), ("persistent", dict(persistent=1)),
                       ("block256", dict(block=256)), ("accel1", dict(rule="accel1")),
                       ("naive", dict(rule="naive")), ("naive64", dict(rule="naive64"))):
        with R.Solver(dev if name not in ("naive", "naive64") else dev[:3], **opts) as s:
            if name == "fused":
                h = s.solve(6)
            else:
                s.setup()
                s.iterate(6)
                h = s.extract()
            out[f"{name}_h"] = h.cpu().numpy()
            out[f"{name}_lam"] = s.get_state(0)[2].cpu().numpy()
            out[f"{name}_obj"] = s.objective()
            codes[name] = s.status()
    adj = [tiny(3, 4, 300, 7), tiny(2, 3, 40, 8)]
    with R.Solver([R.to_device(p) for p in adj], ckpt_stride=2, ckpt_max_iters=5) as s:
        s.setup()
        s.iterate(5)
        h = s.extract()
        for k, g in enumerate(s.split_grads(*s.backward(h))[0]):
            out[f"adjoint_g{k}"] = g.cpu().numpy()
        codes["adjoint"] = s.status()
    u = tiny(4, 5, 77, 11)
    (gi,) = R.ilrma_init([R.ilrma_to_device(u)])
    for k, v in gi.items():
        out[f"ilrma_{k}"] = v.cpu().numpy()
    plan = R.HostPlan(*u["x"].shape, n_chunks=2)
    res = plan.run(u, 4)
    out["host_h"] = res["h"]
    codes["host"] = R.OK
    plan.close()
    # the no-allocation entry point
    d = R.to_device(u)
    I, J, M = u["x"].shape
    rh = torch.zeros((I, J), dtype=torch.float32, device="cuda")
    ru, lam = torch.zeros_like(rh), torch.zeros((I,), dtype=torch.float32, device="cuda")
    h = torch.zeros((I, J, M), dtype=torch.complex64, device="cuda")
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    codes["noalloc"] = R.lib().rcscm_solve_noalloc(
        I, J, M, vp(d["x"]), vp(d["a"]), vp(d["Rp"]), None, vp(d["rh0"]), vp(d["ru0"]), ctypes.byref(R.options()),
        4, vp(rh), vp(ru), vp(lam), vp(h), vp(status), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    out["noalloc_h"] = h.cpu().numpy()
    codes["noalloc_status"] = int(status.item())
    np.savez(out_path, codes=np.array([[k, v] for k, v in codes.items()], dtype=object), **out)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
