"""Python binding of librcscm.so (the C ABI declared in include/rcscm.h).

Argument marshalling only: tensors are checked for device, dtype and layout and
their addresses are handed to the library, which runs every step of the
estimator in its CUDA kernels.  PyTorch provides device memory and streams.
There is no fallback: if the library is missing or fails to load, every entry
point raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, c_double, c_float, c_int, c_int64, c_void_p
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librcscm.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "rcscm.h")

OK, EINVAL, ENULLSPACE, ENONFINITE, ECLAMP, ECUDA, ENOMEM, ETIMEOUT, ECAPACITY, EBOUNDS = range(10)
RULE_ACCEL, RULE_NAIVE, RULE_NAIVE_F64, RULE_ACCEL1, RULE_NAIVE_PRINTED = 0, 1, 2, 3, 4
RULES = {"accel": RULE_ACCEL, "naive": RULE_NAIVE, "naive64": RULE_NAIVE_F64, "accel1": RULE_ACCEL1,
         "naive_printed": RULE_NAIVE_PRINTED}
MAX_M = 8
MAX_J_ACCEL = 4096
FLT_MIN = float(np.finfo(np.float32).tiny)


class Problem(ctypes.Structure):
    _fields_ = [("I", c_int64), ("J", c_int64), ("M", c_int64),
                ("x", c_void_p), ("a", c_void_p), ("Rp", c_void_p),
                ("lambda0", c_void_p), ("rh0", c_void_p), ("ru0", c_void_p),
                ("b", c_void_p), ("rp_c64", c_int)]


class Options(ctypes.Structure):
    _fields_ = [("rule", c_int), ("alpha", c_double), ("beta", c_double),
                ("ru_floor", c_float), ("null_tol", c_double), ("block", c_int),
                ("iters_per_launch", c_int), ("persistent", c_int),
                ("ckpt_stride", c_int), ("ckpt_max_iters", c_int)]


class Ilrma(ctypes.Structure):
    _fields_ = [("I", c_int64), ("J", c_int64), ("M", c_int64), ("K", c_int64), ("n_h", c_int64),
                ("x", c_void_p), ("W", c_void_p), ("T", c_void_p), ("V", c_void_p),
                ("a", c_void_p), ("Rp", c_void_p), ("rh0", c_void_p), ("ru0", c_void_p)]


class RcscmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: rcscm error {code}: {strerror(code)}")


_LIB = None


def header_symbols() -> List[str]:
    """Names of every function the public headers (include/*.h) declare."""
    import glob
    src = "".join(open(h).read() for h in sorted(glob.glob(os.path.join(os.path.dirname(HEADER), "*.h"))))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rcscm_[a-z_0-9]+)\s*\(", src)))


def lib():
    """Load librcscm.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1908_01964_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64p = c_void_p, POINTER(c_int64)
    sig = {
        "rcscm_default_options": (None, [POINTER(Options)]),
        "rcscm_strerror": (ctypes.c_char_p, [c_int]),
        "rcscm_create": (c_int, [POINTER(vp), POINTER(Problem), c_int, POINTER(Options), vp]),
        "rcscm_setup": (c_int, [vp, vp]),
        "rcscm_iterate": (c_int, [vp, c_int, vp]),
        "rcscm_extract": (c_int, [vp, vp, vp]),
        "rcscm_get_state": (c_int, [vp, c_int, vp, vp, vp, vp]),
        "rcscm_set_state": (c_int, [vp, c_int, vp, vp, vp, vp]),
        "rcscm_get_setup": (c_int, [vp, c_int, vp, vp, vp, vp, vp, vp]),
        "rcscm_get_invariants": (c_int, [vp, c_int, vp, vp, vp, vp]),
        "rcscm_status": (c_int, [vp, POINTER(c_int), vp]),
        "rcscm_info": (c_int, [vp, i64p, i64p, i64p]),
        "rcscm_destroy": (None, [vp]),
        "rcscm_solve_host": (c_int, [c_int64, c_int64, c_int64, vp, vp, vp, vp, vp, vp,
                                     POINTER(Options), c_int, vp, vp, vp, vp]),
        "rcscm_solve_noalloc": (c_int, [c_int64, c_int64, c_int64, vp, vp, vp, vp, vp, vp,
                                        POINTER(Options), c_int, vp, vp, vp, vp, vp, vp]),
        "rcscm_objective": (c_int, [vp, POINTER(c_double), vp]),
        "rcscm_autotune": (c_int, [vp, c_int, POINTER(c_int), POINTER(c_int), vp]),
        "rcscm_graph_create": (c_int, [vp, c_int, vp]),
        "rcscm_graph_launch": (c_int, [vp, vp]),
        "rcscm_backward": (c_int, [vp, vp, vp, vp, vp, vp]),
        "rcscm_setup_freq": (c_int, [vp, vp]),
        "rcscm_run": (c_int, [vp, c_int, vp, vp]),
        "rcscm_solve": (c_int, [vp, c_int, vp, vp]),
        "rcscm_host_create": (c_int, [POINTER(vp), c_int64, c_int64, c_int64, POINTER(Options), c_int]),
        "rcscm_host_run": (c_int, [vp, vp, vp, vp, vp, vp, vp, c_int, vp, vp, vp, vp]),
        "rcscm_host_destroy": (None, [vp]),
        "rcscm_ilrma_init": (c_int, [POINTER(Ilrma), c_int, vp, vp]),
        "rcscm_probe_fma": (c_int, [c_int, c_int, ctypes.c_longlong, vp, vp, POINTER(c_double)]),
        "rcscm_front_create": (c_int, [POINTER(vp), c_int64, c_int64, c_int, c_int, c_int]),
        "rcscm_front_shape": (c_int, [vp, i64p, i64p]),
        "rcscm_front_destroy": (None, [vp]),
        "rcscm_front_stft": (c_int, [vp, vp, vp, vp]),
        "rcscm_front_istft": (c_int, [vp, vp, vp, vp]),
        "rcscm_front_ilrma": (c_int, [vp, vp, vp, vp, c_int, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def strerror(code: int) -> str:
    return lib().rcscm_strerror(code).decode()


def _check(code: int, where: str, allow=(OK,)):
    if code not in allow:
        raise RcscmError(code, where)
    return code


def options(rule: str = "accel", alpha: float = 1.1, beta: float = 1e-16, ru_floor: float = FLT_MIN,
            null_tol: float = 1e-6, block: int = 0, iters_per_launch: int = 0, persistent: int = 0,
            ckpt_stride: int = 0, ckpt_max_iters: int = 0) -> Options:
    o = Options()
    lib().rcscm_default_options(ctypes.byref(o))
    o.rule = RULES[rule]
    o.alpha, o.beta, o.ru_floor, o.null_tol = alpha, beta, ru_floor, null_tol
    o.block, o.iters_per_launch, o.persistent = block, iters_per_launch, int(persistent)
    o.ckpt_stride, o.ckpt_max_iters = int(ckpt_stride), int(ckpt_max_iters)
    return o


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return c_void_p(s.cuda_stream)


def _dev(t, dtype, shape, name):
    """Address of a CUDA tensor, or of a page-locked CPU tensor (which the library
    reads or writes in place; it refuses any other host memory)."""
    import torch
    if not isinstance(t, torch.Tensor) or not (t.is_cuda or t.is_pinned()):
        raise TypeError(f"{name} must be a CUDA tensor or a page-locked CPU tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return c_void_p(t.data_ptr())


class Solver:
    """A context over one or more utterances held in CUDA tensors.

    Each problem is a dict with x (complex64 [I, J, M]), a (complex128 [I, M]),
    Rp (complex128, or complex64, [I, M, M]), rh0, ru0 (float32 [I, J]) and
    optionally lambda0 (float64 [I]) and b (complex128 [I, M], the caller's null
    vector of R', validated by the setup).  The tensors must stay alive and
    unchanged while the Solver exists (it keeps references to them).
    """

    def __init__(self, problems: Sequence[dict], rule: str = "accel", stream=None, **opts):
        import torch
        self._keep = []
        arr = (Problem * len(problems))()
        self.shapes = []
        for k, p in enumerate(problems):
            I, J, M = p["x"].shape
            q = arr[k]
            q.I, q.J, q.M = I, J, M
            q.x = _dev(p["x"], torch.complex64, (I, J, M), "x")
            q.a = _dev(p["a"], torch.complex128, (I, M), "a")
            rp_c64 = p["Rp"].dtype == torch.complex64
            q.Rp = _dev(p["Rp"], torch.complex64 if rp_c64 else torch.complex128, (I, M, M), "Rp")
            q.rp_c64 = int(rp_c64)
            b = p.get("b")
            q.b = _dev(b, torch.complex128, (I, M), "b") if b is not None else None
            q.rh0 = _dev(p["rh0"], torch.float32, (I, J), "rh0")
            q.ru0 = _dev(p["ru0"], torch.float32, (I, J), "ru0")
            lam0 = p.get("lambda0")
            q.lambda0 = _dev(lam0, torch.float64, (I,), "lambda0") if lam0 is not None else None
            self._keep.append(p)
            self.shapes.append((I, J, M))
        dev0 = problems[0]["x"].device
        self.device = dev0 if dev0.type == "cuda" else torch.device("cuda", torch.cuda.current_device())
        self.opt = options(rule=rule, **opts)
        self.rule = rule
        ctx = c_void_p()
        _check(lib().rcscm_create(ctypes.byref(ctx), arr, len(problems), ctypes.byref(self.opt), _stream(stream)),
               "rcscm_create")
        self.ctx = ctx

    # -- lifecycle -------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            lib().rcscm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- estimator steps -------------------------------------------------------
    def setup(self, stream=None):
        _check(lib().rcscm_setup(self.ctx, _stream(stream)), "rcscm_setup")

    def iterate(self, n_iter: int, stream=None):
        _check(lib().rcscm_iterate(self.ctx, int(n_iter), _stream(stream)), "rcscm_iterate")

    @property
    def out_elements(self) -> int:
        return int(sum(I * J * M for I, J, M in self.shapes))

    def extract(self, out=None, stream=None):
        """Wiener-filtered target images, all utterances concatenated (complex64)."""
        import torch
        if out is None:
            out = torch.empty(self.out_elements, dtype=torch.complex64, device=self.device)
        elif out.dtype != torch.complex64 or out.numel() != self.out_elements or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex64 tensor with one element per output")
        _check(lib().rcscm_extract(self.ctx, c_void_p(out.data_ptr()), _stream(stream)), "rcscm_extract")
        return out

    def _out(self, out):
        import torch
        if out is None:
            return torch.empty(self.out_elements, dtype=torch.complex64, device=self.device)
        if out.dtype != torch.complex64 or out.numel() != self.out_elements or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex64 tensor with one element per output")
        if not (out.is_cuda or out.is_pinned()):
            raise TypeError("out must be a CUDA tensor or a page-locked CPU tensor")
        return out

    def setup_freq(self, stream=None):
        """Per-frequency setup only (rcscm_setup_freq)."""
        _check(lib().rcscm_setup_freq(self.ctx, _stream(stream)), "rcscm_setup_freq")

    def run(self, n_iter: int, out=None, stream=None):
        """Invariants + n_iter passes + Wiener output from the initial state, one launch."""
        out = self._out(out)
        _check(lib().rcscm_run(self.ctx, int(n_iter), c_void_p(out.data_ptr()), _stream(stream)), "rcscm_run")
        return out

    def solve(self, n_iter: int, out=None, stream=None):
        """setup + n_iter passes + Wiener output (rcscm_solve)."""
        out = self._out(out)
        _check(lib().rcscm_solve(self.ctx, int(n_iter), c_void_p(out.data_ptr()), _stream(stream)), "rcscm_solve")
        return out

    def split(self, flat):
        """Views of a concatenated extract() result, one [I, J, M] tensor per utterance."""
        outs, o = [], 0
        for I, J, M in self.shapes:
            outs.append(flat[o:o + I * J * M].view(I, J, M))
            o += I * J * M
        return outs

    def get_state(self, p: int = 0, stream=None):
        import torch
        I, J, _ = self.shapes[p]
        rh = torch.empty((I, J), dtype=torch.float32, device=self.device)
        ru = torch.empty_like(rh)
        lam = torch.empty((I,), dtype=torch.float32, device=self.device)
        _check(lib().rcscm_get_state(self.ctx, p, c_void_p(rh.data_ptr()), c_void_p(ru.data_ptr()),
                                     c_void_p(lam.data_ptr()), _stream(stream)), "rcscm_get_state")
        return rh, ru, lam

    def set_state(self, p: int, rh=None, ru=None, lam=None, stream=None):
        import torch
        I, J, _ = self.shapes[p]
        ptr = lambda t, shp, nm: _dev(t, torch.float32, shp, nm) if t is not None else None  # noqa: E731
        _check(lib().rcscm_set_state(self.ctx, p, ptr(rh, (I, J), "rh"), ptr(ru, (I, J), "ru"),
                                     ptr(lam, (I,), "lam"), _stream(stream)), "rcscm_set_state")

    def get_setup(self, p: int = 0, stream=None) -> dict:
        import torch
        I, _, M = self.shapes[p]
        kw = dict(device=self.device)
        out = dict(b=torch.empty((I, M), dtype=torch.complex128, **kw),
                   lambda0=torch.empty((I,), dtype=torch.float64, **kw),
                   tau_aa=torch.empty((I,), dtype=torch.float64, **kw),
                   sigma_ab=torch.empty((I,), dtype=torch.complex128, **kw),
                   mu=torch.empty((I, M), dtype=torch.float64, **kw))
        _check(lib().rcscm_get_setup(self.ctx, p, *(c_void_p(out[k].data_ptr()) for k in
                                                    ("b", "lambda0", "tau_aa", "sigma_ab", "mu")),
                                     _stream(stream)), "rcscm_get_setup")
        return out

    def get_invariants(self, p: int = 0, stream=None) -> dict:
        import torch
        I, J, _ = self.shapes[p]
        kw = dict(device=self.device)
        out = dict(tau_ax=torch.empty((I, J), dtype=torch.complex64, **kw),
                   sigma_bx=torch.empty((I, J), dtype=torch.complex64, **kw),
                   kappa=torch.empty((I, J), dtype=torch.float32, **kw))
        _check(lib().rcscm_get_invariants(self.ctx, p, *(c_void_p(out[k].data_ptr()) for k in
                                                         ("tau_ax", "sigma_bx", "kappa")),
                                          _stream(stream)), "rcscm_get_invariants")
        return out

    def objective(self, stream=None) -> np.ndarray:
        """Observed-data log posterior per utterance (constants dropped), FP64."""
        out = (c_double * len(self.shapes))()
        _check(lib().rcscm_objective(self.ctx, out, _stream(stream)), "rcscm_objective")
        return np.array(out[:], dtype=np.float64)

    def autotune(self, n_iter_probe: int = 10, stream=None):
        """Pick the fastest launch shape of the accelerated kernel for this work list."""
        b, p = c_int(0), c_int(0)
        _check(lib().rcscm_autotune(self.ctx, int(n_iter_probe), ctypes.byref(b), ctypes.byref(p), _stream(stream)),
               "rcscm_autotune")
        return b.value, p.value

    def graph_create(self, n_iter: int, out):
        """Capture setup + n_iter passes + extraction into `out` as a CUDA graph."""
        import torch
        if out.dtype != torch.complex64 or out.numel() != self.out_elements or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex64 tensor with one element per output")
        self._graph_out = out
        _check(lib().rcscm_graph_create(self.ctx, int(n_iter), c_void_p(out.data_ptr())), "rcscm_graph_create")

    def backward(self, grad_h, stream=None):
        """Gradients of a real loss of extract()'s output (grad_h: complex64, one
        element per output, dL/dRe h + i dL/dIm h) with respect to x, a and R',
        through the passes run since setup.  Returns flat concatenations
        (grad_x complex64 like the outputs, grad_a complex128 [sum I*M],
        grad_Rp complex128 [sum I*M*M]); split_grads() gives per-utterance views.
        Needs a Solver created with ckpt_stride > 0."""
        import torch
        if grad_h.dtype != torch.complex64 or grad_h.numel() != self.out_elements or not grad_h.is_contiguous():
            raise ValueError("grad_h must be a contiguous complex64 tensor with one element per output")
        kw = dict(device=self.device)
        gx = torch.empty(self.out_elements, dtype=torch.complex64, **kw)
        ga = torch.empty(int(sum(I * M for I, _, M in self.shapes)), dtype=torch.complex128, **kw)
        gR = torch.empty(int(sum(I * M * M for I, _, M in self.shapes)), dtype=torch.complex128, **kw)
        _check(lib().rcscm_backward(self.ctx, c_void_p(grad_h.data_ptr()), c_void_p(gx.data_ptr()),
                                    c_void_p(ga.data_ptr()), c_void_p(gR.data_ptr()), _stream(stream)),
               "rcscm_backward")
        return gx, ga, gR

    def split_grads(self, gx, ga, gR):
        """Per-utterance views ([I,J,M], [I,M], [I,M,M]) of backward()'s results."""
        out, ox, oa, orp = [], 0, 0, 0
        for I, J, M in self.shapes:
            out.append((gx[ox:ox + I * J * M].view(I, J, M), ga[oa:oa + I * M].view(I, M),
                        gR[orp:orp + I * M * M].view(I, M, M)))
            ox, oa, orp = ox + I * J * M, oa + I * M, orp + I * M * M
        return out

    def graph_launch(self, stream=None):
        _check(lib().rcscm_graph_launch(self.ctx, _stream(stream)), "rcscm_graph_launch")

    def status(self, stream=None) -> int:
        flags = c_int(0)
        code = lib().rcscm_status(self.ctx, ctypes.byref(flags), _stream(stream))
        if code == ECUDA:
            raise RcscmError(code, "rcscm_status")
        return code

    def info(self) -> dict:
        r, s, b = c_int64(), c_int64(), c_int64()
        _check(lib().rcscm_info(self.ctx, ctypes.byref(r), ctypes.byref(s), ctypes.byref(b)), "rcscm_info")
        return dict(rows=r.value, slots=s.value, device_bytes=b.value)


class IlrmaPlan:
    """rcscm_ilrma_init with its arguments marshalled once: the output tensors and
    the argument array are made at construction, and run() enqueues the call on
    `stream` (the same outputs are overwritten by every run).  Inputs and status
    as for ilrma_init; they must stay alive while the plan is used."""

    def __init__(self, utts, status=None):
        import torch
        self._arr = (Ilrma * len(utts))()
        self._keep = list(utts)
        self.outs = []
        for k, u in enumerate(utts):
            I, J, M = u["x"].shape
            K = u["T"].shape[1]
            dev = u["x"].device if u["x"].is_cuda else torch.device("cuda", torch.cuda.current_device())
            o = dict(a=torch.empty((I, M), dtype=torch.complex128, device=dev),
                     Rp=torch.empty((I, M, M), dtype=torch.complex128, device=dev),
                     rh0=torch.empty((I, J), dtype=torch.float32, device=dev),
                     ru0=torch.empty((I, J), dtype=torch.float32, device=dev))
            q = self._arr[k]
            q.I, q.J, q.M, q.K, q.n_h = I, J, M, K, int(u.get("n_h", 0))
            q.x = _dev(u["x"], torch.complex64, (I, J, M), "x")
            q.W = _dev(u["W"], torch.complex128, (I, M, M), "W")
            q.T = _dev(u["T"], torch.float32, (I, K), "T")
            q.V = _dev(u["V"], torch.float32, (K, J), "V")
            q.a, q.Rp, q.rh0, q.ru0 = (c_void_p(o[n].data_ptr()) for n in ("a", "Rp", "rh0", "ru0"))
            self.outs.append(o)
        self._status = status
        self._st = None if status is None else _dev(status, torch.int32, (1,), "status")

    def run(self, stream=None) -> list:
        _check(lib().rcscm_ilrma_init(self._arr, len(self.outs), self._st, _stream(stream)), "rcscm_ilrma_init")
        return self.outs


def ilrma_init(utts, status=None, stream=None) -> list:
    """Estimator inputs from the outputs of the ILRMA stage (rcscm_ilrma_init).

    Each element of `utts` is a dict with x (complex64 [I, J, M]), W (complex128
    [I, M, M], row n = w_{i,n}^H), T (float32 [I, K]), V (float32 [K, J]) as CUDA
    or page-locked CPU tensors and n_h (int, default 0).  Returns one dict per
    utterance with a (complex128 [I, M]), Rp (complex128 [I, M, M]), rh0 and ru0
    (float32 [I, J]) as CUDA tensors on the inputs' device, in the layouts
    Solver takes.  `status` (an int32 CUDA tensor of one element, or None)
    receives the status bits.  Enqueued on `stream`; does not synchronise."""
    return IlrmaPlan(utts, status).run(stream)


def ilrma_to_device(prob: dict, device="cuda") -> dict:
    """The ILRMA-stage outputs of a generator problem (synth: x, W, T, V, n_h) as CUDA tensors."""
    import torch
    return dict(
        x=torch.from_numpy(np.ascontiguousarray(prob["x"], np.complex64)).to(device),
        W=torch.from_numpy(np.ascontiguousarray(prob["W"], np.complex128)).to(device),
        T=torch.from_numpy(np.ascontiguousarray(prob["T"], np.float32)).to(device),
        V=torch.from_numpy(np.ascontiguousarray(prob["V"], np.float32)).to(device),
        n_h=int(prob.get("n_h", 0)),
    )


def to_device(prob: dict, device="cuda") -> dict:
    """Move a generator problem (numpy arrays) to CUDA tensors in the ABI's dtypes."""
    import torch
    out = dict(
        x=torch.from_numpy(np.ascontiguousarray(prob["x"], np.complex64)).to(device),
        a=torch.from_numpy(np.ascontiguousarray(prob["a"], np.complex128)).to(device),
        Rp=torch.from_numpy(np.ascontiguousarray(prob["Rp"], np.complex128)).to(device),
        rh0=torch.from_numpy(np.ascontiguousarray(prob["rh0"], np.float32)).to(device),
        ru0=torch.from_numpy(np.ascontiguousarray(prob["ru0"], np.float32)).to(device),
    )
    if prob.get("lambda0") is not None:
        out["lambda0"] = torch.from_numpy(np.ascontiguousarray(prob["lambda0"], np.float64)).to(device)
    return out


class HostPlan:
    """rcscm_host_*: solves utterances of one shape from host (numpy) arrays with
    chunked copy/compute overlap.  Use page-locked arrays for overlap."""

    def __init__(self, I: int, J: int, M: int, n_chunks: int = 4, rule: str = "accel", **opts):
        self.shape = (I, J, M)
        self.opt = options(rule=rule, **opts)
        plan = c_void_p()
        _check(lib().rcscm_host_create(ctypes.byref(plan), I, J, M, ctypes.byref(self.opt), int(n_chunks)),
               "rcscm_host_create")
        self.plan = plan

    def run_ptrs(self, x, a, Rp, rh0, ru0, n_iter, h_out, rh=None, ru=None, lam=None) -> int:
        """Run on raw host addresses (ints); returns the status code."""
        v = lambda p: None if p is None else c_void_p(p)  # noqa: E731
        return lib().rcscm_host_run(self.plan, v(x), v(a), v(Rp), None, v(rh0), v(ru0), int(n_iter), v(h_out),
                                    v(rh), v(ru), v(lam))

    def run(self, prob: dict, n_iter: int, want_state: bool = True) -> dict:
        I, J, M = self.shape
        arrs = dict(x=np.ascontiguousarray(prob["x"], np.complex64), a=np.ascontiguousarray(prob["a"], np.complex128),
                    Rp=np.ascontiguousarray(prob["Rp"], np.complex128),
                    rh0=np.ascontiguousarray(prob["rh0"], np.float32), ru0=np.ascontiguousarray(prob["ru0"], np.float32))
        out = dict(h=np.empty((I, J, M), np.complex64))
        if want_state:
            out.update(rh=np.empty((I, J), np.float32), ru=np.empty((I, J), np.float32), lam=np.empty((I,), np.float32))
        ad = lambda k, d: d[k].ctypes.data if k in d else None  # noqa: E731
        code = self.run_ptrs(ad("x", arrs), ad("a", arrs), ad("Rp", arrs), ad("rh0", arrs), ad("ru0", arrs), n_iter,
                             out["h"].ctypes.data, ad("rh", out), ad("ru", out), ad("lam", out))
        _check(code, "rcscm_host_run", allow=(OK, ECLAMP))
        return out

    def close(self):
        if getattr(self, "plan", None) is not None and self.plan.value:
            lib().rcscm_host_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_host(x, a, Rp, rh0, ru0, n_iter: int, lambda0=None, want_state: bool = True, **opts):
    """One-shot solve from host (numpy) arrays through rcscm_solve_host."""
    x = np.ascontiguousarray(x, np.complex64)
    a = np.ascontiguousarray(a, np.complex128)
    Rp = np.ascontiguousarray(Rp, np.complex128)
    rh0 = np.ascontiguousarray(rh0, np.float32)
    ru0 = np.ascontiguousarray(ru0, np.float32)
    I, J, M = x.shape
    h = np.empty_like(x)
    rh = np.empty((I, J), np.float32) if want_state else None
    ru = np.empty((I, J), np.float32) if want_state else None
    lam = np.empty((I,), np.float32) if want_state else None
    l0 = None if lambda0 is None else np.ascontiguousarray(lambda0, np.float64)
    ptr = lambda v: None if v is None else c_void_p(v.ctypes.data)  # noqa: E731
    o = options(**opts)
    code = lib().rcscm_solve_host(I, J, M, ptr(x), ptr(a), ptr(Rp), ptr(l0), ptr(rh0), ptr(ru0),
                                  ctypes.byref(o), int(n_iter), ptr(h), ptr(rh), ptr(ru), ptr(lam))
    _check(code, "rcscm_solve_host", allow=(OK, ECLAMP))
    return dict(h=h, rh=rh, ru=ru, lam=lam)


class Front:
    """rcscm_front_*: STFT, ILRMA and inverse STFT for signals of one shape (the front
    end of the estimator; include/rcscm_frontend.h).  Tensors are CUDA tensors."""

    def __init__(self, M: int, n_samples: int, n_fft: int = 1024, shift: int = 512, K: int = 10):
        h = c_void_p()
        _check(lib().rcscm_front_create(ctypes.byref(h), M, n_samples, n_fft, shift, K), "rcscm_front_create")
        self.h = h
        self.M, self.n_samples, self.n_fft, self.shift, self.K = M, n_samples, n_fft, shift, K
        I, J = c_int64(), c_int64()
        _check(lib().rcscm_front_shape(h, ctypes.byref(I), ctypes.byref(J)), "rcscm_front_shape")
        self.I, self.J = I.value, J.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().rcscm_front_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stft(self, sig, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.I, self.J, self.M), dtype=torch.complex64, device=sig.device)
        _check(lib().rcscm_front_stft(self.h, _dev(sig, torch.float32, (self.M, self.n_samples), "sig"),
                                      _dev(out, torch.complex64, (self.I, self.J, self.M), "X"), _stream(stream)),
               "rcscm_front_stft")
        return out

    def istft(self, X, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.M, self.n_samples), dtype=torch.float32, device=X.device)
        _check(lib().rcscm_front_istft(self.h, _dev(X, torch.complex64, (self.I, self.J, self.M), "X"),
                                       _dev(out, torch.float32, (self.M, self.n_samples), "out"), _stream(stream)),
               "rcscm_front_istft")
        return out

    def ilrma(self, X, T0, V0, n_iter: int, status=None, stream=None):
        """Returns (W complex128 [I, M, M] for X itself, T float32 [N, I, K], V float32 [N, K, J])."""
        import torch
        dev = X.device
        N, I, J, K = self.M, self.I, self.J, self.K
        W = torch.empty((I, N, N), dtype=torch.complex128, device=dev)
        T = torch.empty((N, I, K), dtype=torch.float32, device=dev)
        V = torch.empty((N, K, J), dtype=torch.float32, device=dev)
        st = status if status is not None else None
        _check(lib().rcscm_front_ilrma(self.h, _dev(X, torch.complex64, (I, J, N), "X"),
                                       _dev(T0, torch.float32, (N, I, K), "T0"),
                                       _dev(V0, torch.float32, (N, K, J), "V0"), int(n_iter),
                                       _dev(W, torch.complex128, (I, N, N), "W"), _dev(T, torch.float32, (N, I, K), "T"),
                                       _dev(V, torch.float32, (N, K, J), "V"),
                                       _dev(st, torch.int32, (1,), "status") if st is not None else None,
                                       _stream(stream)), "rcscm_front_ilrma")
        return W, T, V
