"""FP64 oracle of the comparison methods of Sec. IV (TEST INFRASTRUCTURE ONLY).

Three variants of the least-squares / weight alternation of Algorithm 1, each written from the
paper's description in plain NumPy, on the same forward model (oracle/slr.py: x (T, P, Q),
x_hat = F x unitary, A = mask * F):

  * GIRAF, fully circulant (Sec. III-A: the GIRAF scheme approximates every linear convolution,
    the one along the parameter axis included, by a circular one). The lifting has T windows
    instead of k = T - M + 1; window j, column (l, m) holds x_hat[(j + M - 1 - m) mod T][c - l].
    Everything else is the proposed method's arithmetic.
  * HLR-Voxel (Sec. II-D, Eq. MORASA-objective; Sec. IV-B names it): one k x M Toeplitz matrix of
    the temporal signal per pixel, T_r[j, m] = x_{j+M-1-m}(r), image domain, no spatial coupling;
    IRLS with one M x M Gram G_r = T_r^H T_r and one weight H_r = (G_r + eps I)^(p/2-1) per
    pixel. The penalty sum_r ||T_r||_p is one objective smoothed by one eps, scheduled as in
    Sec. III-C: eps^(0) = eps0_frac * max_r lambda_max(G_r(x0)), eps <- eps / gamma.
  * IRLS-direct (Sec. IV-A: Eq. x-update and Eq. weight-update solved without the FFT
    approximations): the exact multi-fold Toeplitz matrix, valid linear convolution in all three
    dimensions (rows Gamma:Lambda of Sec. II-B; slr.lift_linear), its Gram G = T^H T, the weight
    H, and the penalty gradient F^H C^H T^*(T(C F x) H) with T^* the adjoint of the lifting. The
    exact lifting is not shift invariant, so it is taken on the centred k-space C F x (C =
    fftshift, DC at (P/2, Q/2)): the grid Gamma of Sec. II-B holds the Fourier samples around
    k = 0, and its boundaries, where the circulant approximation is justified by the decay of
    the coefficients, are the highest frequencies. (For the circulant liftings the centring
    changes nothing.)

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use it.
"""

from __future__ import annotations

import numpy as np

from . import slr


# ----------------------------------------------------------------------------------------------
# GIRAF: circular in time as well (Sec. III-A)
# ----------------------------------------------------------------------------------------------

def lift_circ(x_hat: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    """Fully circulant lifting: T windows, Tm[(j, c), (l, m)] = x_hat[(j + M - 1 - m) % T][c - l]."""
    T, P, Q = x_hat.shape
    Tm = np.zeros((T * P * Q, N1 * N2 * M), dtype=np.complex128)
    for j in range(T):
        rows = slice(j * P * Q, (j + 1) * P * Q)
        for m in range(M):
            frame = x_hat[(j + M - 1 - m) % T]
            for l1 in range(N1):
                for l2 in range(N2):
                    Tm[rows, slr.col_index(l1, l2, m, N1, N2)] = \
                        np.roll(frame, (l1, l2), axis=(0, 1)).ravel()
    return Tm


def pair_products_circ(x: np.ndarray, M: int) -> np.ndarray:
    """q[m, m'](r) = sum_{j < T} conj(x_{(j+M-1-m) % T}(r)) x_{(j+M-1-m') % T}(r)."""
    T = x.shape[0]
    q = np.zeros((M, M) + x.shape[1:], dtype=np.complex128)
    for m in range(M):
        for mp in range(M):
            for j in range(T):
                q[m, mp] += np.conj(x[(j + M - 1 - m) % T]) * x[(j + M - 1 - mp) % T]
    return q


def gram_circ(x: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    """G = Tm^H Tm of the fully circulant lifting of F x: the lags of the circular pair products
    (unnormalised 2-D DFT read out around zero lag) filled as in slr.gram_fft."""
    P, Q = x.shape[1:]
    g = np.fft.fft2(pair_products_circ(x, M))
    s = N1 * N2 * M
    G = np.zeros((s, s), dtype=np.complex128)
    for m in range(M):
        for mp in range(M):
            for l1 in range(N1):
                for l2 in range(N2):
                    for lp1 in range(N1):
                        for lp2 in range(N2):
                            G[slr.col_index(l1, l2, m, N1, N2), slr.col_index(lp1, lp2, mp, N1, N2)] = \
                                g[m, mp, (l1 - lp1) % P, (l2 - lp2) % Q]
    return G


def apply_W_circ(x: np.ndarray, S: np.ndarray) -> np.ndarray:
    """(W x) = sum_{j < T} E_j^T S(r) E_j x(r) with (E_j x)[m] = x_{(j+M-1-m) % T}."""
    M = S.shape[0]
    T = x.shape[0]
    out = np.zeros_like(x)
    for j in range(T):
        v = np.stack([x[(j + M - 1 - m) % T] for m in range(M)])
        w = np.einsum("ab...,b...->a...", S, v)
        for a in range(M):
            out[(j + M - 1 - a) % T] += w[a]
    return out


def weight_from_x_circ(x, N1, N2, M, eps, p):
    G = gram_circ(x, N1, N2, M)
    H, _ = slr.weight_H(G, eps, p)
    return slr.weight_S(slr.diag_sums(H, N1, N2, M), x.shape[1], x.shape[2])


def irls_giraf(kspace, masks, N1, N2, M, lam, p, n_irls, n_cg, gamma=1.4, eps_frac=0.01):
    """Algorithm 1 with the fully circulant lifting (same schedule and warm start)."""
    rhs = slr.AH(kspace, masks)
    x = rhs.copy()
    eps = eps_frac * float(np.linalg.eigvalsh(gram_circ(x, N1, N2, M))[-1])
    for _ in range(n_irls):
        S = weight_from_x_circ(x, N1, N2, M, eps, p)
        x = slr.cg(lambda v: slr.AH(slr.A(v, masks), masks) + lam * apply_W_circ(v, S), rhs, x,
                   n_cg)
        eps = eps / gamma
    return x


# ----------------------------------------------------------------------------------------------
# HLR-Voxel: one Toeplitz matrix of the temporal signal per pixel (Sec. II-D)
# ----------------------------------------------------------------------------------------------

def voxel_toeplitz(x: np.ndarray, M: int, r: tuple) -> np.ndarray:
    """T_r (k x M): T_r[j, m] = x_{j+M-1-m}(r)."""
    T = x.shape[0]
    k = T - M + 1
    return np.array([[x[j + M - 1 - m][r] for m in range(M)] for j in range(k)])


def voxel_grams(x: np.ndarray, M: int) -> np.ndarray:
    """G_r = T_r^H T_r for every pixel, shape (P, Q, M, M): G_r[m, m'] = sum_j
    conj(x_{j+M-1-m}(r)) x_{j+M-1-m'}(r) (the image-domain pair products, not transformed)."""
    return np.moveaxis(slr.pair_products(x, M), (0, 1), (2, 3))


def voxel_weights(Gv: np.ndarray, eps, p: float) -> np.ndarray:
    """H_r = U diag((lambda + eps_r)^(p/2-1)) U^H per pixel (batched eigh). eps: one value for
    every pixel, or (P, Q)."""
    lam, U = np.linalg.eigh(Gv)
    alpha = (lam + np.asarray(eps, dtype=np.float64)[..., None]) ** (p / 2.0 - 1.0)
    return np.einsum("...im,...m,...jm->...ij", U, alpha, U.conj())


def voxel_S(Hv: np.ndarray) -> np.ndarray:
    """The per-pixel M x M matrix of the banded W that gives Re <x, W x> = sum_r Tr(H_r G_r):
    Tr(H T^H T) = sum_j v_j^T H conj(v_j) = sum_j v_j^H H^T v_j with v_j = E_j x(r), so
    S(r) = H_r^T. Returned as (M, M, P, Q) like slr.weight_S."""
    return np.moveaxis(np.swapaxes(Hv, -1, -2), (2, 3), (0, 1))


def voxel_penalty(x: np.ndarray, Hv: np.ndarray, M: int) -> float:
    """sum_r Tr(H_r T_r^H T_r) with the explicit per-pixel Toeplitz matrices."""
    P, Q = x.shape[1:]
    tot = 0.0
    for r1 in range(P):
        for r2 in range(Q):
            Tr = voxel_toeplitz(x, M, (r1, r2))
            tot += float(np.trace(Hv[r1, r2] @ (Tr.conj().T @ Tr)).real)
    return tot


def voxel_initial_eps(x0: np.ndarray, M: int, frac: float = 0.01) -> float:
    """eps^(0) = frac * the largest lambda_max(G_r(x0)) over the pixels (Sec. III-C)."""
    return frac * float(np.max(np.linalg.eigvalsh(voxel_grams(x0, M))[..., -1]))


def irls_hlr_voxel(kspace, masks, M, lam, p, n_irls, n_cg, gamma=1.4, eps_frac=0.01):
    """IRLS on sum_r ||T_r||_p: x0 = A^H b, one eps for the whole penalty (Sec. III-C schedule),
    n_cg CG steps per iteration on (A^H A + lam W) with W built from S(r) = H_r^T."""
    rhs = slr.AH(kspace, masks)
    x = rhs.copy()
    eps = voxel_initial_eps(x, M, eps_frac)
    for _ in range(n_irls):
        S = voxel_S(voxel_weights(voxel_grams(x, M), eps, p))
        x = slr.cg(lambda v: slr.normal_op(v, masks, S, lam), rhs, x, n_cg)
        eps = eps / gamma
    return x


# ----------------------------------------------------------------------------------------------
# IRLS-direct: the exact (valid) multi-fold Toeplitz matrix, no FFT approximation (Sec. IV-A)
# ----------------------------------------------------------------------------------------------

def lift_direct(x_hat: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    """Rows (j, c1, c2) with c in [N1-1, P-1] x [N2-1, Q-1]: Tm[(j, c), (l, m)] =
    x_hat[j + M - 1 - m][c - l] (slr.lift_linear)."""
    return slr.lift_linear(x_hat, N1, N2, M)


def unlift_direct(Y: np.ndarray, T: int, P: int, Q: int, N1: int, N2: int, M: int) -> np.ndarray:
    """T^*(Y): the adjoint of lift_direct, every entry of Y added back to the x_hat sample it was
    copied from."""
    k = T - M + 1
    nr1, nr2 = P - N1 + 1, Q - N2 + 1
    z = np.zeros((T, P, Q), dtype=np.complex128)
    for j in range(k):
        blk_rows = slice(j * nr1 * nr2, (j + 1) * nr1 * nr2)
        for m in range(M):
            for l1 in range(N1):
                for l2 in range(N2):
                    col = Y[blk_rows, slr.col_index(l1, l2, m, N1, N2)].reshape(nr1, nr2)
                    z[j + M - 1 - m, N1 - 1 - l1: N1 - 1 - l1 + nr1,
                      N2 - 1 - l2: N2 - 1 - l2 + nr2] += col
    return z


def centred_kspace(x: np.ndarray) -> np.ndarray:
    """C F x: the unitary 2-D DFT of every frame with DC moved to (P/2, Q/2)."""
    return np.fft.fftshift(slr.F2(x), axes=(-2, -1))


def gram_direct(x: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    Tm = lift_direct(centred_kspace(x), N1, N2, M)
    return Tm.conj().T @ Tm


def apply_W_direct(x: np.ndarray, H: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    """Gradient of Tr(H T(C F x)^H T(C F x)) with respect to conj(x):
    F^H C^H T^*(T(C F x) H)."""
    T, P, Q = x.shape
    Tm = lift_direct(centred_kspace(x), N1, N2, M)
    z = unlift_direct(Tm @ H, T, P, Q, N1, N2, M)
    return slr.F2H(np.fft.ifftshift(z, axes=(-2, -1)))


def normal_op_direct(x, masks, H, lam, N1, N2, M):
    return slr.AH(slr.A(x, masks), masks) + lam * apply_W_direct(x, H, N1, N2, M)


def irls_direct(kspace, masks, N1, N2, M, lam, p, n_irls, n_cg, gamma=1.4, eps_frac=0.01):
    rhs = slr.AH(kspace, masks)
    x = rhs.copy()
    eps = eps_frac * float(np.linalg.eigvalsh(gram_direct(x, N1, N2, M))[-1])
    for _ in range(n_irls):
        H, _ = slr.weight_H(gram_direct(x, N1, N2, M), eps, p)
        x = slr.cg(lambda v: normal_op_direct(v, masks, H, lam, N1, N2, M), rhs, x, n_cg)
        eps = eps / gamma
    return x
