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
# Ceilings on the elementwise relative error of every slot (max over slots, and the
# 99.9th percentile).  FP32 rounding of a slot's own quadratic forms bounds each
# slot's error by a few hundred units of rounding times the slot's conditioning; the
# ceilings leave room for the slots where r_h is small against r_u (its relative
# error grows as the posterior variance dominates).
ELEM_ONE_ITER = (1e-2, 1e-3)     # (max, 99.9th percentile) after one pass
ELEM_FULL_RUN = (1e-1, 1e-2)     # after a full run


def rel(a, b):
    a = np.asarray(a, np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def kappa_fp32_bound(x, a, st, kappa):
    """Forward error bound of kappa_ij = sum_k |Phi_k x_ij|^2 (k = 1..M-2) formed in FP32
    from an FP32 copy of any orthonormal-complement basis Phi (Sec. III-C-2, the
    invariants of Algorithm 2).  With unit roundoff u = 2^-24, rounding Phi once and
    accumulating M fused products gives |dz_k| <= (M + 1) u sum_n |Phi_kn| |x_n|; by
    Cauchy-Schwarz the whole error E = (sum_k |dz_k|^2)^(1/2) is at most
    (M + 1) u |x| (sum_k |Phi_k|^2)^(1/2), and sum_k |Phi_k|^2 = tr(R'^+) - |R'^+ a|^2 / tau_aa
    does not depend on the basis.  Then |kappa^ - kappa| <= 2 kappa^(1/2) E + E^2 + M u kappa.
    Where x is almost parallel to a (the DC bin), this floor is far above 1e-5 tau_xx."""
    x = np.asarray(x, np.complex128)
    M = x.shape[-1]
    u = 2.0 ** -24
    P = st.Rp_pinv
    ga = np.einsum("imn,in->im", P, np.asarray(a, np.complex128))
    rows2 = np.real(np.trace(P, axis1=1, axis2=2)) - np.sum(np.abs(ga) ** 2, axis=1) / st.tau_aa
    E = (M + 1) * u * np.linalg.norm(x, axis=-1) * np.sqrt(np.maximum(rows2, 0.0))[:, None]
    k = np.maximum(kappa, 0.0)
    return 2.0 * np.sqrt(k) * E + E ** 2 + M * u * k


def ilrma_fp32_bounds(x, W, n_h):
    """Forward error bounds of the FP32 frame sums of the initialisation from the
    ILRMA stage (Sec. II-B-1 Eq. (eq:rit), Sec. II-B-3 Eq. (eq:ruinit)).  With
    unit roundoff u = 2^-24, y = W x formed from W rounded once and M fused
    products has |dy_n| <= e_n = (M + 1) u sum_m |w_nm| |x_m|, so the output power
    P_n = |y_n|^2 is off by at most dP_n = 2 |y_n| e_n + e_n^2; the frame mean d_n,
    summed with compensation, by dd_n = mean_j dP_n + 4 u d_n.  Then
    |R'^ - R'|_F <= sum_{n != n_h} dd_n |q_n|^2 (q_n the columns of W^{-1}) and
    r_u0 = (1/M) sum_{n != n_h} P_n / d_n is off by at most
    (1/M) sum_{n != n_h} (dP_n / d_n + P_n dd_n / d_n^2 + 3 u P_n / d_n).
    Returns (bound on |dR'|_F per row [I], bound on |dr_u0| per slot [I, J])."""
    u = 2.0 ** -24
    x = np.asarray(x, np.complex128)
    W = np.asarray(W, np.complex128)
    M = x.shape[-1]
    y = np.einsum("inm,ijm->ijn", W, x)
    e = (M + 1) * u * np.einsum("inm,ijm->ijn", np.abs(W), np.abs(x))
    P = np.abs(y) ** 2
    dP = 2.0 * np.abs(y) * e + e ** 2
    keep = np.ones(M)
    keep[n_h] = 0.0
    d = P.mean(axis=1)
    dd = dP.mean(axis=1) + 4.0 * u * d
    q2 = np.sum(np.abs(np.linalg.inv(W)) ** 2, axis=1)            # |q_n|^2, [I, M]
    dR = np.sum(keep * dd * q2, axis=1)
    ds = np.where(keep > 0, d, 1.0)[:, None, :]
    dru = np.sum(keep * (dP / ds + P * dd[:, None, :] / ds ** 2 + 3.0 * u * P / ds), axis=2) / M
    return dR, dru


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


def elementwise(a, b):
    """Elementwise relative errors |a - b| / |b| of a parameter: (max, 99.9th percentile).
    The 2-norm of rel() can hide a few badly wrong slots; these two cannot."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    e = np.abs(a - b) / np.maximum(np.abs(b), np.finfo(np.float64).tiny)
    return float(e.max()), float(np.quantile(e, 0.999))


def compare(gpu, ora, rows=None):
    """Errors of a GPU result against the oracle's: the relative 2-norm of each
    parameter (rh, ru, lam), the SNR of the extracted target (sdr) and, under
    "elem", the elementwise (max, 99.9th percentile) relative error of each
    parameter."""
    sel = slice(None) if rows is None else np.asarray(rows)
    g = {k: np.asarray(gpu[k])[sel] for k in ("rh", "ru", "lam", "h")}
    return dict(rh=rel(g["rh"], ora["rh"]), ru=rel(g["ru"], ora["ru"]), lam=rel(g["lam"], ora["lam"]),
                sdr=sdr_db(g["h"], ora["h"]),
                elem={k: elementwise(g[k], ora[k]) for k in ("rh", "ru", "lam")})


def norm_max(e):
    """Largest relative 2-norm error of the three parameters of a compare() result."""
    return max(e["rh"], e["ru"], e["lam"])


def elem_max(e, q=0):
    """Largest elementwise error over the parameters: q = 0 the maximum, q = 1 the 99.9th percentile."""
    return max(v[q] for v in e["elem"].values())


def report(name, **kw):
    """Append measured errors to the JSON-lines file named by RCSCM_PARITY_REPORT (if set)."""
    path = os.environ.get("RCSCM_PARITY_REPORT")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps({"case": name, **kw}, default=float) + "\n")
