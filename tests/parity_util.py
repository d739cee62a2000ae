"""Helpers shared by the parity tests: error metrics and runners for the CUDA
path (through the C ABI) and the FP64 oracle on the same seeded inputs."""
import json
import os

import numpy as np

from oracle import rcscm_oracle as O

ALPHA, BETA = 1.1, 1e-16

# Tolerances (relative 2-norm error over all slots of a parameter; SNR for h).
TOL_ONE_ITER = 1e-5      # parameters after one pass
TOL_FULL_RUN = 1e-3      # parameters after a full run
SDR_MIN_DB = 60.0        # extracted target against the oracle's


def rel(a, b):
    a = np.asarray(a, np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def sdr_db(est, ref):
    ref = np.asarray(ref, np.complex128).ravel()
    err = np.asarray(est, np.complex128).ravel() - ref
    return float(10 * np.log10(np.vdot(ref, ref).real / max(np.vdot(err, err).real, 1e-300)))


def gpu_run(probs, n_iter, rule="accel", chunks=None, **opts):
    """Run the CUDA path on a list of generator problems; returns per-problem dicts."""
    import torch
    from paper_1908_01964_gb300 import rcscm as R
    dev = [R.to_device(p) for p in probs]
    with R.Solver(dev, rule=rule, **opts) as s:
        s.setup()
        for k in (chunks or [n_iter]):
            s.iterate(k)
        h = s.extract()
        st = s.status()
        out = []
        for k, hk in enumerate(s.split(h)):
            rh, ru, lam = s.get_state(k)
            out.append(dict(rh=rh.cpu().numpy(), ru=ru.cpu().numpy(), lam=lam.cpu().numpy(),
                            h=hk.cpu().numpy()))
        torch.cuda.synchronize()
    return out, st


def oracle_run(prob, n_iter, rule="accel2", rows=None):
    return O.run(prob, n_iter, rule=rule, alpha=ALPHA, beta=BETA, rows=rows)


def compare(gpu, ora, rows=None):
    sel = slice(None) if rows is None else np.asarray(rows)
    g = {k: np.asarray(gpu[k])[sel] for k in ("rh", "ru", "lam", "h")}
    return dict(rh=rel(g["rh"], ora["rh"]), ru=rel(g["ru"], ora["ru"]), lam=rel(g["lam"], ora["lam"]),
                sdr=sdr_db(g["h"], ora["h"]))


def report(name, **kw):
    """Append measured errors to the JSON-lines file named by RCSCM_PARITY_REPORT (if set)."""
    path = os.environ.get("RCSCM_PARITY_REPORT")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps({"case": name, **kw}, default=float) + "\n")
