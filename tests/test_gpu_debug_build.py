"""The debug build (compiled with RCSCM_DEBUG; compute-sanitizer is not
available): every kernel checks its row, slot and shape indexes and reports
RCSCM_EBOUNDS instead of touching memory out of range.  Run on small, oddly
shaped inputs through every kernel path (fused, streaming, persistent, other
block sizes, first-stage, naive FP32 and FP64, adjoint, objective, ILRMA
initialisation, host pipeline, no-allocation entry point), no check fails and
the results equal the normal build's bit for bit (the checks do not touch the
arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(lib, out):
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_cases.py"), lib, out], capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out, allow_pickle=True)


def test_debug_build_checks_pass_and_results_match(tmp_path):
    from paper_1908_01964_gb300 import build as B, rcscm as R
    normal = _run(B.build(), str(tmp_path / "normal.npz"))
    debug = _run(B.build(debug=True), str(tmp_path / "debug.npz"))
    bounds_bit = 1 << (R.EBOUNDS - 1)
    for res in (normal, debug):
        for name, code in res["codes"]:
            if name == "noalloc_status":
                assert not int(code) & bounds_bit, name
            else:
                assert int(code) in (R.OK, R.ECLAMP), (name, R.strerror(int(code)))
    assert sorted(normal.files) == sorted(debug.files)
    for k in normal.files:
        if k != "codes":
            np.testing.assert_array_equal(debug[k], normal[k], err_msg=k)
