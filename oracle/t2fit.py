"""Mono-exponential T2 fitting of a recovered image series (TEST INFRASTRUCTURE ONLY).

Sec. IV-A: after reconstruction, T2 maps are estimated by fitting a mono-exponential model to
every pixel. The paper does not state the fitting method; this module uses: magnitude data
|x_n(r)| ~ A(r) exp(-t_n / T2(r)), a log-linear least-squares initial guess, then at most 20
Gauss-Newton steps on the un-logged residual, over foreground pixels |x_0| > 0.1 max |x_0|.
The same CPU fitter is applied to the oracle's and to the CUDA path's series.
"""

from __future__ import annotations

import numpy as np


def foreground(x: np.ndarray, frac: float = 0.1) -> np.ndarray:
    a0 = np.abs(x[0])
    return a0 > frac * a0.max()


def fit_t2(x: np.ndarray, times_ms, fg: np.ndarray | None = None, n_gn: int = 20,
           t2_max: float = 1e4) -> np.ndarray:
    """T2 map (ms) of shape (P, Q); NaN outside the foreground."""
    t = np.asarray(times_ms, dtype=np.float64)
    mag = np.abs(np.asarray(x, dtype=np.complex128))          # (T, P, Q)
    if fg is None:
        fg = foreground(x)
    y = mag[:, fg]                                            # (T, n)
    # log-linear initial guess: log y = log A - t / T2
    ly = np.log(np.maximum(y, 1e-30))
    tm = t.mean()
    slope = ((t - tm)[:, None] * (ly - ly.mean(0))).sum(0) / ((t - tm) ** 2).sum()
    R = np.clip(-slope, 1.0 / t2_max, None)                  # relaxation rate 1/T2
    Aamp = np.exp(ly.mean(0) + R * tm)
    for _ in range(n_gn):
        e = np.exp(-t[:, None] * R[None])
        model = Aamp[None] * e
        res = model - y
        jA = e
        jR = -t[:, None] * model
        # 2x2 normal equations per pixel
        a11 = (jA * jA).sum(0)
        a12 = (jA * jR).sum(0)
        a22 = (jR * jR).sum(0)
        g1 = (jA * res).sum(0)
        g2 = (jR * res).sum(0)
        det = a11 * a22 - a12 * a12
        ok = np.abs(det) > 1e-300
        dA = np.where(ok, (a22 * g1 - a12 * g2) / np.where(ok, det, 1.0), 0.0)
        dR = np.where(ok, (-a12 * g1 + a11 * g2) / np.where(ok, det, 1.0), 0.0)
        Aamp = Aamp - dA
        R = np.clip(R - dR, 1.0 / t2_max, None)
    out = np.full(fg.shape, np.nan)
    out[fg] = 1.0 / R
    return out


def t2_rel_l2(t2_ref: np.ndarray, t2_test: np.ndarray) -> float:
    """||T2_test - T2_ref|| / ||T2_ref|| over the pixels where both are defined."""
    ok = np.isfinite(t2_ref) & np.isfinite(t2_test)
    return float(np.linalg.norm(t2_test[ok] - t2_ref[ok]) / np.linalg.norm(t2_ref[ok]))
