"""Seeded generators for damped-exponential image series and their undersampled k-space.

Signal model (Sec. II-B, Eq. signal-model): every pixel r of frame n holds
    x[n, r] = rho(r) * sum_i f_i(r) * exp(-t_n / T2_i(r)),
i.e. a sum of L damped exponentials whose decay rates vary smoothly in space.

Measurement model (Sec. II-A, Eq. measurement-model, single coil): frame n is observed as
    b_n = mask_n * (F x_n + eta_n),
with F the unitary 2-D DFT (forward sign e^{-2 pi i}, natural frequency order, no fftshift),
mask_n in {0,1} a per-frame Cartesian point mask, and eta_n complex white Gaussian noise.

Layouts: image series and k-space are complex arrays of shape (T, P, Q) (Q fastest);
masks are uint8 arrays of the same shape.

Seeds (base seed S): rho uses S+1, relaxation/fraction fields S+2, mask of frame n S+10+n,
noise S+99, served request i S+1000*i.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic reconstruction problem and the solver settings it is run with."""

    name: str
    P: int
    Q: int
    T: int
    times_ms: tuple            # echo / spin-lock times t_n, length T
    n_ellipses: int
    t2_ranges: tuple           # ((lo, hi), ...) one range per exponential component, ms
    frac_range: tuple          # (lo, hi) of the first component's fraction (two components only)
    R: float                   # undersampling factor: P*Q/R samples per frame
    N1: int
    N2: int
    M: int
    lam: float
    p: float
    n_irls: int
    n_cg: int
    snr_db: float = 30.0
    seed: int = 0
    n_coils: int = 1           # receiver coils (Eq. measurement-ij); 1 = single channel
    depth: int = 1             # slices of a 3-D volume (1 = 2-D images)
    N3: int = 1                # filter taps along the depth
    mask: str = "vd"           # "vd": variable density (vd_mask); "uniform": uniform_mask

    @property
    def shape(self):
        return (self.T, self.P, self.Q)

    @property
    def taps(self):
        return self.N1 * self.N2 * self.M


def _tiny():
    return Workload(
        name="tiny_32x32x8", P=32, Q=32, T=8,
        times_ms=tuple(5.0 + 5.0 * n for n in range(8)),
        n_ellipses=6, t2_ranges=((20.0, 120.0),), frac_range=(1.0, 1.0),
        R=4.0, N1=5, N2=5, M=2, lam=1e-3, p=0.0, n_irls=20, n_cg=10)


def _perf():
    return Workload(
        name="perf_256x256x16", P=256, Q=256, T=16,
        times_ms=tuple(1.0 + 59.0 * n / 15.0 for n in range(16)),
        n_ellipses=10, t2_ranges=((10.0, 40.0), (50.0, 150.0)), frac_range=(0.2, 0.8),
        R=8.0, N1=9, N2=9, M=3, lam=1e-3, p=0.0, n_irls=30, n_cg=15)


def _coils():
    # the paper's in-vivo series (Sec. IV-A): 128 x 128, 12 echoes at 10 .. 120 ms, 12 coils.
    # lam: with 12 coils at 6x the data term alone is a noisy SENSE-type fit; 0.1 lets IRLS halve
    # the adjoint's error (the paper picks its weight by an SNR sweep, not reproduced here)
    return Workload(
        name="coils_128x128x12", P=128, Q=128, T=12,
        times_ms=tuple(10.0 * (n + 1) for n in range(12)),
        n_ellipses=8, t2_ranges=((20.0, 120.0),), frac_range=(1.0, 1.0),
        R=6.0, N1=9, N2=9, M=3, lam=0.1, p=0.0, n_irls=20, n_cg=10, n_coils=12)


def _vol():
    # 3-D volumes: 128 x 128 x 64 slices, 12 frames, one exponential, 6x 3-D variable-density
    # sampling, filter 7 x 7 x 3 spatial taps x 2 frame taps (s = 294)
    return Workload(
        name="vol_128x128x64x12", P=128, Q=128, T=12, depth=64, N3=3,
        times_ms=tuple(10.0 * (n + 1) for n in range(12)),
        n_ellipses=12, t2_ranges=((20.0, 120.0),), frac_range=(1.0, 1.0),
        R=6.0, N1=7, N2=7, M=2, lam=1e-3, p=0.0, n_irls=25, n_cg=15)


def _cmp():
    # the paper's comparison of the approximations (Sec. IV-A, Fig. 2 / Fig. 3): a single-channel
    # 128 x 128 series of 12 echoes at 10 .. 120 ms from 30 % uniform random Fourier samples
    return Workload(
        name="cmp_128x128x12", P=128, Q=128, T=12,
        times_ms=tuple(10.0 * (n + 1) for n in range(12)),
        n_ellipses=8, t2_ranges=((20.0, 120.0),), frac_range=(1.0, 1.0),
        R=1.0 / 0.3, N1=9, N2=9, M=3, lam=1e-3, p=0.0, n_irls=20, n_cg=10, mask="uniform")


WORKLOADS = {w.name: w for w in (_tiny(), _perf(), _coils(), _vol(), _cmp())}


def workload(name: str, **overrides) -> Workload:
    """Named workload, optionally with fields replaced (e.g. smaller iteration counts)."""
    return dataclasses.replace(WORKLOADS[name], **overrides)


def ellipse_phantom(P: int, Q: int, n: int, rng: np.random.Generator) -> np.ndarray:
    """Additive sum of n random filled ellipses (centres in the central 60 %, semi-axes
    3-12 px at 32x32 scaled with the grid, angle U[0, pi), intensity U[0.2, 1])."""
    scale = min(P, Q) / 32.0
    yy, xx = np.meshgrid(np.arange(P, dtype=np.float64), np.arange(Q, dtype=np.float64),
                         indexing="ij")
    img = np.zeros((P, Q), dtype=np.float64)
    for _ in range(n):
        cy = rng.uniform(0.2 * P, 0.8 * P)
        cx = rng.uniform(0.2 * Q, 0.8 * Q)
        a = rng.uniform(3.0, 12.0) * scale
        b = rng.uniform(3.0, 12.0) * scale
        th = rng.uniform(0.0, math.pi)
        amp = rng.uniform(0.2, 1.0)
        dy, dx = yy - cy, xx - cx
        u = (dx * math.cos(th) + dy * math.sin(th)) / a
        v = (-dx * math.sin(th) + dy * math.cos(th)) / b
        img += amp * ((u * u + v * v) <= 1.0)
    return img


def smooth_field(P: int, Q: int, sigma: float, lo: float, hi: float,
                 rng: np.random.Generator) -> np.ndarray:
    """White N(0,1) noise blurred by a periodic Gaussian of width sigma (px), then min-max
    mapped onto [lo, hi]."""
    w = rng.standard_normal((P, Q))
    f1 = np.fft.fftfreq(P)[:, None]
    f2 = np.fft.fftfreq(Q)[None, :]
    g = np.exp(-2.0 * (math.pi * sigma) ** 2 * (f1 * f1 + f2 * f2))
    s = np.real(np.fft.ifft2(np.fft.fft2(w) * g))
    s = (s - s.min()) / max(s.max() - s.min(), 1e-300)
    return lo + (hi - lo) * s


def vd_mask(P: int, Q: int, R: float, rng: np.random.Generator) -> np.ndarray:
    """Variable-density Cartesian point mask with round(P*Q/R) samples, natural FFT order.

    A c x c block around DC is fully sampled (c = max(4, P//32)); the remaining samples are drawn
    without replacement with probability proportional to 1 / (1 + (|k| / (P/8))^2), |k| the
    centred frequency radius in grid units."""
    n_target = int(round(P * Q / R))
    k1 = np.fft.fftfreq(P) * P
    k2 = np.fft.fftfreq(Q) * Q
    K1, K2 = np.meshgrid(k1, k2, indexing="ij")
    c = max(4, P // 32)
    centre = (K1 >= -c // 2) & (K1 < c - c // 2) & (K2 >= -c // 2) & (K2 < c - c // 2)
    mask = centre.copy()
    need = n_target - int(mask.sum())
    if need > 0:
        rad = np.sqrt(K1 * K1 + K2 * K2)
        wgt = 1.0 / (1.0 + (rad / (P / 8.0)) ** 2)
        wgt[mask] = 0.0
        flat = wgt.ravel() / wgt.sum()
        pick = rng.choice(P * Q, size=need, replace=False, p=flat)
        mask.ravel()[pick] = True
    return mask.astype(np.uint8)


def uniform_mask(P: int, Q: int, R: float, rng: np.random.Generator) -> np.ndarray:
    """Uniform random Cartesian point mask with round(P*Q/R) samples: the DC sample plus
    draws without replacement, every other position equally likely."""
    n_target = int(round(P * Q / R))
    mask = np.zeros(P * Q, dtype=bool)
    mask[0] = True
    pick = rng.choice(np.arange(1, P * Q), size=n_target - 1, replace=False)
    mask[pick] = True
    return mask.reshape(P, Q).astype(np.uint8)


def make_series(w: Workload) -> np.ndarray:
    """Ground-truth image series x_true, complex128 of shape (T, P, Q)."""
    S = w.seed
    rho = ellipse_phantom(w.P, w.Q, w.n_ellipses, np.random.default_rng(S + 1))
    rng = np.random.default_rng(S + 2)
    sigma = 3.0 * w.P / 32.0
    t = np.asarray(w.times_ms, dtype=np.float64)[:, None, None]
    if len(w.t2_ranges) == 1:
        lo, hi = w.t2_ranges[0]
        t2 = smooth_field(w.P, w.Q, sigma, lo, hi, rng)
        x = rho[None] * np.exp(-t / t2[None])
    else:
        (alo, ahi), (blo, bhi) = w.t2_ranges
        t2a = smooth_field(w.P, w.Q, sigma, alo, ahi, rng)
        t2b = smooth_field(w.P, w.Q, sigma, blo, bhi, rng)
        f = rng.uniform(w.frac_range[0], w.frac_range[1], size=(w.P, w.Q))
        x = rho[None] * (f[None] * np.exp(-t / t2a[None]) + (1.0 - f[None]) * np.exp(-t / t2b[None]))
    return x.astype(np.complex128)


def coil_maps(n_coils: int, P: int, Q: int, rng: np.random.Generator) -> np.ndarray:
    """Smooth complex receiver sensitivities (n_coils, P, Q): coils spaced on a circle of radius
    0.6 P around the image centre, Gaussian magnitude fall-off (sigma 0.4 P, periodic distance),
    a random constant phase plus a small random linear phase ramp each, normalised so that
    sum_c |C_c|^2 = 1 at every pixel."""
    yy, xx = np.meshgrid(np.arange(P, dtype=np.float64), np.arange(Q, dtype=np.float64),
                         indexing="ij")
    maps = []
    for c in range(n_coils):
        ang = 2.0 * np.pi * c / n_coils
        cy = P / 2.0 + 0.6 * P * np.sin(ang)
        cx = Q / 2.0 + 0.6 * Q * np.cos(ang)
        dy = (yy - cy + P / 2.0) % P - P / 2.0
        dx = (xx - cx + Q / 2.0) % Q - Q / 2.0
        mag = np.exp(-(dy * dy + dx * dx) / (2.0 * (0.4 * P) ** 2))
        ky, kx = rng.uniform(-1.0, 1.0, size=2)
        ph = rng.uniform(0.0, 2.0 * np.pi) + 2.0 * np.pi * (ky * yy / P + kx * xx / Q)
        maps.append(mag * np.exp(1j * ph))
    C = np.stack(maps)
    return C / np.sqrt((np.abs(C) ** 2).sum(0))[None]


def ellipsoid_phantom(D: int, P: int, Q: int, n: int, rng: np.random.Generator) -> np.ndarray:
    """Additive sum of n random filled ellipsoids (centres in the central 60 % of each axis,
    semi-axes 3-12 px scaled with the grid per axis, a random rotation about the depth axis,
    intensity U[0.2, 1]); shape (D, P, Q)."""
    sp, sd = min(P, Q) / 32.0, D / 32.0
    zz, yy, xx = np.meshgrid(np.arange(D, dtype=np.float64), np.arange(P, dtype=np.float64),
                             np.arange(Q, dtype=np.float64), indexing="ij")
    vol = np.zeros((D, P, Q), dtype=np.float64)
    for _ in range(n):
        cz = rng.uniform(0.2 * D, 0.8 * D)
        cy = rng.uniform(0.2 * P, 0.8 * P)
        cx = rng.uniform(0.2 * Q, 0.8 * Q)
        a = rng.uniform(3.0, 12.0) * sp
        b = rng.uniform(3.0, 12.0) * sp
        c = rng.uniform(3.0, 12.0) * sd
        th = rng.uniform(0.0, math.pi)
        amp = rng.uniform(0.2, 1.0)
        dz, dy, dx = zz - cz, yy - cy, xx - cx
        u = (dx * math.cos(th) + dy * math.sin(th)) / a
        v = (-dx * math.sin(th) + dy * math.cos(th)) / b
        wv = dz / c
        vol += amp * ((u * u + v * v + wv * wv) <= 1.0)
    return vol


def smooth_field3(D: int, P: int, Q: int, sigma: float, sigma_d: float, lo: float, hi: float,
                  rng: np.random.Generator) -> np.ndarray:
    """White N(0,1) noise blurred by a periodic Gaussian (sigma px in-plane, sigma_d px in
    depth), min-max mapped onto [lo, hi]; shape (D, P, Q)."""
    w = rng.standard_normal((D, P, Q))
    f0 = np.fft.fftfreq(D)[:, None, None]
    f1 = np.fft.fftfreq(P)[None, :, None]
    f2 = np.fft.fftfreq(Q)[None, None, :]
    g = np.exp(-2.0 * math.pi ** 2 * (sigma_d ** 2 * f0 * f0 + sigma ** 2 * (f1 * f1 + f2 * f2)))
    s = np.real(np.fft.ifftn(np.fft.fftn(w) * g))
    s = (s - s.min()) / max(s.max() - s.min(), 1e-300)
    return lo + (hi - lo) * s


def vd_mask3(D: int, P: int, Q: int, R: float, rng: np.random.Generator) -> np.ndarray:
    """3-D variable-density Cartesian mask with exactly D*P*Q/R samples: a c x c x cd block around
    DC fully sampled (c = max(4, P//32), cd = max(2, D//32)), the rest drawn without replacement
    with probability proportional to 1 / (1 + (|k| / (P/8))^2), |k| the centred frequency radius
    with the depth frequencies scaled by P / D."""
    n_target = int(round(D * P * Q / R))
    k0 = np.fft.fftfreq(D) * D
    k1 = np.fft.fftfreq(P) * P
    k2 = np.fft.fftfreq(Q) * Q
    K0, K1, K2 = np.meshgrid(k0, k1, k2, indexing="ij")
    c, cd = max(4, P // 32), max(2, D // 32)
    centre = ((K1 >= -c // 2) & (K1 < c - c // 2) & (K2 >= -c // 2) & (K2 < c - c // 2) &
              (K0 >= -cd // 2) & (K0 < cd - cd // 2))
    mask = centre.copy()
    need = n_target - int(mask.sum())
    if need > 0:
        rad = np.sqrt(K1 * K1 + K2 * K2 + (K0 * P / D) ** 2)
        wgt = 1.0 / (1.0 + (rad / (P / 8.0)) ** 2)
        wgt[mask] = 0.0
        flat = wgt.ravel() / wgt.sum()
        pick = rng.choice(D * P * Q, size=need, replace=False, p=flat)
        mask.ravel()[pick] = True
    return mask.astype(np.uint8)


def make_problem3(w: Workload) -> dict:
    """Seeded 3-D problem: x_true (T, D, P, Q) complex128 = rho exp(-t / T2) on random ellipsoids
    with a T2 field smooth in 3-D (sigma 3 P / 32 px in-plane, 3 D / 32 px in depth); masks
    (T, D, P, Q) uint8 (seed S + 10 + n); kspace = mask * (F3 x_true + eta) at w.snr_db
    (noise seed S + 99), F3 the unitary 3-D DFT."""
    S, D = w.seed, w.depth
    rho = ellipsoid_phantom(D, w.P, w.Q, w.n_ellipses, np.random.default_rng(S + 1))
    lo, hi = w.t2_ranges[0]
    t2 = smooth_field3(D, w.P, w.Q, 3.0 * w.P / 32.0, 3.0 * D / 32.0, lo, hi,
                       np.random.default_rng(S + 2))
    t = np.asarray(w.times_ms, dtype=np.float64)[:, None, None, None]
    x = (rho[None] * np.exp(-t / t2[None])).astype(np.complex128)
    masks = np.stack([vd_mask3(D, w.P, w.Q, w.R, np.random.default_rng(S + 10 + n))
                      for n in range(w.T)])
    clean = masks * np.fft.fftn(x, axes=(1, 2, 3), norm="ortho")
    rng = np.random.default_rng(S + 99)
    eta = (rng.standard_normal(clean.shape) + 1j * rng.standard_normal(clean.shape)) * masks
    scale = np.linalg.norm(clean) * 10.0 ** (-w.snr_db / 20.0) / max(np.linalg.norm(eta), 1e-300)
    return {"x_true": x, "masks": masks, "kspace": clean + scale * eta, "workload": w}


def make_problem(w: Workload) -> dict:
    """Seeded problem: x_true (T,P,Q) complex128, masks (T,P,Q) uint8, kspace (T,P,Q) complex128.

    kspace = mask * (F x_true + eta); eta is complex Gaussian on the sampled entries, scaled so
    that 20 log10(||mask * F x_true|| / ||eta||) equals w.snr_db exactly. With w.n_coils > 1 the
    k-space is coil-major (Nc, T, P, Q), kspace[c, n] = mask_n * (F (C_c x_n) + eta), and the
    sensitivities (Nc, P, Q) are returned as "coils" (seed S + 20). Volumes (w.depth > 1) come
    from make_problem3."""
    if w.depth > 1:
        return make_problem3(w)
    S = w.seed
    x = make_series(w)
    draw = uniform_mask if w.mask == "uniform" else vd_mask
    masks = np.stack([draw(w.P, w.Q, w.R, np.random.default_rng(S + 10 + n))
                      for n in range(w.T)])
    if w.n_coils > 1:
        coils = coil_maps(w.n_coils, w.P, w.Q, np.random.default_rng(S + 20))
        clean = np.stack([masks * np.fft.fft2(coils[c][None] * x, norm="ortho")
                          for c in range(w.n_coils)])
    else:
        coils = None
        clean = masks * np.fft.fft2(x, norm="ortho")
    rng = np.random.default_rng(S + 99)
    eta = (rng.standard_normal(clean.shape) + 1j * rng.standard_normal(clean.shape)) * masks
    scale = np.linalg.norm(clean) * 10.0 ** (-w.snr_db / 20.0) / max(np.linalg.norm(eta), 1e-300)
    kspace = clean + scale * eta
    out = {"x_true": x, "masks": masks, "kspace": kspace, "workload": w}
    if coils is not None:
        out["coils"] = coils
    return out


def served_mix(n_requests: int = 512, rate_hz: float = 20.0, seed: int = 0,
               sizes=(64, 128, 192, 256)) -> list:
    """Served-mix request list: Poisson arrivals and seeded per-request workloads.

    Each entry is (arrival_s, Workload). Sizes uniform over `sizes`, frames U{8..24},
    1-2 components, undersampling U[4, 10], filter N1=N2 in {5,7,9}, M in {2,3}."""
    rng = np.random.default_rng(seed + 7)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    t_arr = np.cumsum(gaps)
    out = []
    for i in range(n_requests):
        r = np.random.default_rng(seed + 1000 * i)
        P = int(r.choice(sizes))
        T = int(r.integers(8, 25))
        L = int(r.integers(1, 3))
        R = float(r.uniform(4.0, 10.0))
        N = int(r.choice([5, 7, 9]))
        M = int(r.choice([2, 3]))
        times = tuple(1.0 + 59.0 * n / (T - 1) for n in range(T))
        ranges = ((20.0, 120.0),) if L == 1 else ((10.0, 40.0), (50.0, 150.0))
        w = Workload(name=f"req{i}", P=P, Q=P, T=T, times_ms=times, n_ellipses=8,
                     t2_ranges=ranges, frac_range=(0.2, 0.8), R=R, N1=N, N2=N, M=M,
                     lam=1e-3, p=0.0, n_irls=30, n_cg=15, seed=seed + 1000 * i)
        out.append((float(t_arr[i]), w))
    return out
