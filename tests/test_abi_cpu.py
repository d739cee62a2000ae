"""C-ABI checks that need no GPU: the library builds and loads, exports every
function the public header declares, the ctypes structs match the C layout, and
host-side validation rejects bad arguments before any CUDA call."""
import ctypes
import os
import subprocess

import pytest

from paper_1908_01964_gb300 import build as B
from paper_1908_01964_gb300 import rcscm as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return R.lib()


def test_header_declares_the_boundary():
    syms = R.header_symbols()
    for name in ("rcscm_create", "rcscm_setup", "rcscm_iterate", "rcscm_extract", "rcscm_get_state",
                 "rcscm_set_state", "rcscm_status", "rcscm_destroy", "rcscm_strerror", "rcscm_solve_host"):
        assert name in syms


def test_library_exports_every_header_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [s for s in R.header_symbols() if s not in exported]
    assert not missing, missing
    for s in R.header_symbols():
        assert hasattr(L, s)


def test_header_is_plain_c_and_struct_layout_matches(tmp_path, L):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "rcscm.h"
#include "rcscm_probe.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(rcscm_problem), offsetof(rcscm_problem, x),
         offsetof(rcscm_problem, ru0), offsetof(rcscm_problem, b), offsetof(rcscm_problem, rp_c64),
         sizeof(rcscm_options), offsetof(rcscm_options, iters_per_launch));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(R.Problem), R.Problem.x.offset, R.Problem.ru0.offset, R.Problem.b.offset,
            R.Problem.rp_c64.offset, ctypes.sizeof(R.Options), R.Options.iters_per_launch.offset]
    assert got == want


def test_strerror_and_defaults(L):
    for code in range(8):
        assert len(R.strerror(code)) > 3
    assert "unknown" in R.strerror(99)
    o = R.options()
    assert o.rule == R.RULE_ACCEL and o.alpha == 1.1 and o.beta == 1e-16
    assert o.null_tol == 1e-6 and o.block == 0 and o.iters_per_launch == 0


def _problem(I=4, J=8, M=4, ptr=0x1000):
    p = R.Problem()
    p.I, p.J, p.M = I, J, M
    p.x = p.a = p.Rp = p.rh0 = p.ru0 = ptr
    p.lambda0 = None
    return p


@pytest.mark.parametrize("bad", ["M1", "M9", "J0", "I0", "nullx", "longJ", "rule", "block", "npro"])
def test_create_rejects_bad_arguments_without_cuda(L, bad):
    p = _problem()
    o = R.options()
    n = 1
    if bad == "M1":
        p.M = 1
    elif bad == "M9":
        p.M = 9
    elif bad == "J0":
        p.J = 0
    elif bad == "I0":
        p.I = 0
    elif bad == "nullx":
        p.x = None
    elif bad == "longJ":
        p.J = R.MAX_J_ACCEL + 1
    elif bad == "rule":
        o.rule = 7
    elif bad == "block":
        o.block = 100
    elif bad == "npro":
        n = 0
    ctx = ctypes.c_void_p()
    code = L.rcscm_create(ctypes.byref(ctx), ctypes.byref(p), n, ctypes.byref(o), None)
    assert code == R.EINVAL
    assert not ctx.value


def test_null_context_calls_are_rejected(L):
    assert L.rcscm_setup(None, None) == R.EINVAL
    assert L.rcscm_iterate(None, 3, None) == R.EINVAL
    assert L.rcscm_extract(None, None, None) == R.EINVAL
    assert L.rcscm_status(None, None, None) == R.EINVAL
    L.rcscm_destroy(None)


def test_status_codes_match_the_header():
    import re
    from paper_1908_01964_gb300 import rcscm as R
    src = open(R.HEADER).read()
    codes = dict((m.group(1), int(m.group(2))) for m in re.finditer(r"#define RCSCM_(E[A-Z]+|OK)\s+(\d+)", src))
    for name, value in codes.items():
        assert getattr(R, name) == value, name
    assert codes["EBOUNDS"] == 9
