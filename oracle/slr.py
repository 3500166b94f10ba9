"""FP64 oracle for the IRLS recovery of damped exponentials (TEST INFRASTRUCTURE ONLY).

Plain NumPy restatement of the method of Sec. III (Algorithm 1). Nothing here is blocked, fused
or reordered beyond what the equations state; numpy.fft and numpy.linalg.eigh are used as library
primitives. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use it.

Conventions (readings of the paper, each stated where it is used):
  * The unknown is the image series x, shape (T, P, Q), complex. Its k-space is x_hat = F x with F
    the unitary 2-D DFT, forward sign e^{-2 pi i}, natural frequency order.
  * A_n = mask_n * F (single coil, Eq. measurement-ij with C_j = I). With coils (Eq.
    measurement-ij): b[c, n] = mask_n * F (C_c * x_n) for coil sensitivities C_c (P, Q); the
    paper's F C_j F^* acting on the k-space x_hat is the multiplication of the image by C_j.
  * Filter support Lambda = N1 x N2 spatial taps x M frame taps, s = N1*N2*M columns. A column of
    the lifted matrix is indexed a = (m*N1 + l1)*N2 + l2.
  * Lifting (Sec. II-B, Eq. annihil-compact, with the hybrid approximation of Sec. III-A): space is
    circular (Eq. Toeplitz-circ-rep, circulant of size L = P*Q), frames are a *valid* linear
    convolution, k = T - M + 1 windows. Row (j, c) = window j, k-space position c:
        Tm[(j, c), (l, m)] = x_hat[j + M - 1 - m][c - l  (mod P, Q)].
    so Tm @ d is the 3-D convolution d (*) x_hat evaluated at frames M-1 .. T-1.
  * Gram matrix G = Tm^H Tm (s x s). The paper writes R = T T^* with the transposed lifting
    (Sec. III-B, Eq. gram-matrix: M x M blocks of N1N2 x N1N2); both are the same s x s matrix.
  * Weight H = (G + eps I)^(p/2 - 1) (Eq. weight-update); its square root's rows are the filters
    h_i = sqrt(alpha_i) u_i^*, alpha_i = (lambda_i + eps)^(p/2-1) (Sec. III-B).
  * Least-squares step: J(x) = ||A x - b||^2 + lam * Tr(H G(x)), whose normal equations are
    (A^H A + lam W) x = A^H b (Eq. grad-ls; the paper's mu p / 2 weighting is folded into lam).
"""

from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------------------------
# Forward model (Sec. II-A, Eq. measurement-ij / measurement-model-compact, one coil)
# ----------------------------------------------------------------------------------------------

def F2(x: np.ndarray) -> np.ndarray:
    """Unitary forward 2-D DFT over the last two axes (sign e^{-2 pi i k.r})."""
    return np.fft.fft2(x, norm="ortho")


def F2H(y: np.ndarray) -> np.ndarray:
    """Adjoint (= inverse) of F2."""
    return np.fft.ifft2(y, norm="ortho")


def A(x: np.ndarray, masks: np.ndarray) -> np.ndarray:
    """A x = mask * F x, frame by frame."""
    return masks * F2(x)


def AH(b: np.ndarray, masks: np.ndarray) -> np.ndarray:
    """A^H b = F^H (mask * b), frame by frame."""
    return F2H(masks * b)


def A_coils(x: np.ndarray, masks: np.ndarray, C: np.ndarray) -> np.ndarray:
    """b[c, n] = mask_n * F (C_c * x_n) (Eq. measurement-ij): coil-major (Nc, T, P, Q)."""
    return np.stack([masks * F2(C[c][None] * x) for c in range(C.shape[0])])


def AH_coils(b: np.ndarray, masks: np.ndarray, C: np.ndarray) -> np.ndarray:
    """A^H b = sum_c conj(C_c) * F^H (mask_n * b[c, n])."""
    return sum(np.conj(C[c])[None] * F2H(masks * b[c]) for c in range(C.shape[0]))


# ----------------------------------------------------------------------------------------------
# Explicit lifting (Sec. II-B, Eq. annihil-compact; Sec. III-A, Eq. expand-first-term and
# Eq. Toeplitz-circ-rep). Only for tiny problems: it has k*P*Q rows and s columns.
# ----------------------------------------------------------------------------------------------

def col_index(l1: int, l2: int, m: int, N1: int, N2: int) -> int:
    return (m * N1 + l1) * N2 + l2


def lift(x_hat: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    """Hybrid (spatially circular, temporally valid) multi-fold Toeplitz matrix of x_hat."""
    T, P, Q = x_hat.shape
    k = T - M + 1
    Tm = np.zeros((k * P * Q, N1 * N2 * M), dtype=np.complex128)
    for j in range(k):
        rows = slice(j * P * Q, (j + 1) * P * Q)
        for m in range(M):
            frame = x_hat[j + M - 1 - m]
            for l1 in range(N1):
                for l2 in range(N2):
                    # np.roll(f, (l1, l2))[c] = f[c - l]
                    Tm[rows, col_index(l1, l2, m, N1, N2)] = np.roll(frame, (l1, l2), axis=(0, 1)).ravel()
    return Tm


def lift_linear(x_hat: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    """Exact multi-fold Toeplitz matrix: valid linear convolution in all three dimensions
    (rows = the valid shifts Gamma:Lambda of Sec. II-B). Used only to report the size of the
    hybrid approximation, never as a parity reference."""
    T, P, Q = x_hat.shape
    k = T - M + 1
    nr1, nr2 = P - N1 + 1, Q - N2 + 1
    Tm = np.zeros((k * nr1 * nr2, N1 * N2 * M), dtype=np.complex128)
    for j in range(k):
        for m in range(M):
            frame = x_hat[j + M - 1 - m]
            for l1 in range(N1):
                for l2 in range(N2):
                    # row (j, c1, c2), c in [N-1, P-1]: value x_hat[c - l]
                    blk = frame[N1 - 1 - l1: N1 - 1 - l1 + nr1, N2 - 1 - l2: N2 - 1 - l2 + nr2]
                    Tm[j * nr1 * nr2:(j + 1) * nr1 * nr2, col_index(l1, l2, m, N1, N2)] = blk.ravel()
    return Tm


def gram_brute(x: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    """G = Tm^H Tm from the explicit lifting of x_hat = F x."""
    Tm = lift(F2(x), N1, N2, M)
    return Tm.conj().T @ Tm


# ----------------------------------------------------------------------------------------------
# Gram matrix through FFT autocorrelation (Sec. III-B, Eq. block-expression-for-R and
# Eq. P-ij-modified)
# ----------------------------------------------------------------------------------------------

def pair_products(x: np.ndarray, M: int) -> np.ndarray:
    """q[m, m'](r) = sum_{j<k} conj(x_{j+M-1-m}(r)) x_{j+M-1-m'}(r) for all m, m' < M.

    This is the image-domain product summed over the k windows of the block formula
    R_{p,q} = sum_i T(x_{p+i-1}) T(x_{q+i-1})^* (Eq. block-expression-for-R)."""
    T = x.shape[0]
    k = T - M + 1
    q = np.zeros((M, M) + x.shape[1:], dtype=np.complex128)
    for m in range(M):
        for mp in range(M):
            for j in range(k):
                q[m, mp] += np.conj(x[j + M - 1 - m]) * x[j + M - 1 - mp]
    return q


def gram_lags(x: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    """lag[m, m', d1, d2] = sum_r q[m, m'](r) e^{-2 pi i (d1 r1 / P + d2 r2 / Q)} for
    d1 in [-(N1-1), N1-1], d2 in [-(N2-1), N2-1], stored at offset (N1-1, N2-1).

    The paper obtains these entries from the DFT of the product image (Eq. P-ij-modified); here the
    full unnormalised FFT is taken and the (2N1-1) x (2N2-1) neighbourhood around zero lag is
    read out."""
    P, Q = x.shape[1:]
    g = np.fft.fft2(pair_products(x, M))       # unnormalised forward DFT
    L1, L2 = 2 * N1 - 1, 2 * N2 - 1
    lag = np.zeros((M, M, L1, L2), dtype=np.complex128)
    for i1 in range(L1):
        for i2 in range(L2):
            lag[:, :, i1, i2] = g[:, :, (i1 - (N1 - 1)) % P, (i2 - (N2 - 1)) % Q]
    return lag


def gram_fft(x: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    """G[(l, m), (l', m')] = lag[m, m'](l - l'), the sliding-window fill of Eq. P-ij-modified."""
    lag = gram_lags(x, N1, N2, M)
    s = N1 * N2 * M
    G = np.zeros((s, s), dtype=np.complex128)
    for m in range(M):
        for mp in range(M):
            for l1 in range(N1):
                for l2 in range(N2):
                    for lp1 in range(N1):
                        for lp2 in range(N2):
                            G[col_index(l1, l2, m, N1, N2), col_index(lp1, lp2, mp, N1, N2)] = \
                                lag[m, mp, l1 - lp1 + N1 - 1, l2 - lp2 + N2 - 1]
    return G


# ----------------------------------------------------------------------------------------------
# Weight update (Eq. weight-update; Sec. III-B; epsilon schedule of Sec. III-C)
# ----------------------------------------------------------------------------------------------

def weight_H(G: np.ndarray, eps: float, p: float):
    """H = U diag((lambda_i + eps)^(p/2 - 1)) U^H from the eigendecomposition G = U Lambda U^H.
    Returns (H, eigenvalues ascending)."""
    lam, U = np.linalg.eigh(G)
    alpha = (lam + eps) ** (p / 2.0 - 1.0)
    return (U * alpha) @ U.conj().T, lam


def filters_from_H(G: np.ndarray, eps: float, p: float) -> np.ndarray:
    """Rows of H^{1/2}: h_i = sqrt(alpha_i) u_i^* (Sec. III-B). Returns an (s, s) array whose
    row i is h_i."""
    lam, U = np.linalg.eigh(G)
    alpha = (lam + eps) ** (p / 2.0 - 1.0)
    return np.sqrt(alpha)[:, None] * U.conj().T


def diag_sums(H: np.ndarray, N1: int, N2: int, M: int) -> np.ndarray:
    """d[a, b, d1, d2] = sum_{l - l' = d} H[(l', b), (l, a)], lags at offset (N1-1, N2-1).

    These are the summed diagonals of the blocks of H that the precomputed weight operator of
    Eq. grad-ls needs (Sec. III-A: the product (E E^*) summed over shifted copies)."""
    L1, L2 = 2 * N1 - 1, 2 * N2 - 1
    d = np.zeros((M, M, L1, L2), dtype=np.complex128)
    for a in range(M):
        for b in range(M):
            for l1 in range(N1):
                for l2 in range(N2):
                    for lp1 in range(N1):
                        for lp2 in range(N2):
                            d[a, b, l1 - lp1 + N1 - 1, l2 - lp2 + N2 - 1] += \
                                H[col_index(lp1, lp2, b, N1, N2), col_index(l1, l2, a, N1, N2)]
    return d


def weight_S(d: np.ndarray, P: int, Q: int) -> np.ndarray:
    """S[a, b](r) = sum_d d[a, b, d] e^{-2 pi i (d1 r1/P + d2 r2/Q)}: the lag array placed on the
    P x Q grid (negative lags wrapped, aliases added) and transformed by an unnormalised forward
    FFT. Shape (M, M, P, Q)."""
    M, _, L1, L2 = d.shape
    N1, N2 = (L1 + 1) // 2, (L2 + 1) // 2
    pad = np.zeros((M, M, P, Q), dtype=np.complex128)
    for i1 in range(L1):
        for i2 in range(L2):
            pad[:, :, (i1 - (N1 - 1)) % P, (i2 - (N2 - 1)) % Q] += d[:, :, i1, i2]
    return np.fft.fft2(pad)


def apply_W(x: np.ndarray, S: np.ndarray) -> np.ndarray:
    """(W x)(r) = sum_j E_j^T S(r) E_j x(r) with (E_j x)(r)[m] = x_{j+M-1-m}(r):
    the sum over the k windows of per-pixel M x M products (Eq. grad-ls, the operator
    Q G Q^* with G = sum_i D(h_i)^* D(h_i))."""
    M = S.shape[0]
    T = x.shape[0]
    k = T - M + 1
    out = np.zeros_like(x)
    for j in range(k):
        v = np.stack([x[j + M - 1 - m] for m in range(M)])
        w = np.einsum("abpq,bpq->apq", S, v)
        for a in range(M):
            out[j + M - 1 - a] += w[a]
    return out


def penalty_filters(x: np.ndarray, Hh: np.ndarray, N1: int, N2: int, M: int) -> float:
    """sum_i ||Tm h_i^*||^2 evaluated with the explicit lifting (the quadratic form whose
    FFT restatement is Eq. ls-update-mod). Hh holds one filter per row (filters_from_H)."""
    Tm = lift(F2(x), N1, N2, M)
    tot = 0.0
    for h in Hh:
        tot += float(np.sum(np.abs(Tm @ h.conj()) ** 2))
    return tot


# ----------------------------------------------------------------------------------------------
# Least-squares step (Eq. x-update / grad-ls) by conjugate gradients (Algorithm 1, step 2)
# ----------------------------------------------------------------------------------------------

def normal_op(x: np.ndarray, masks: np.ndarray, S: np.ndarray, lam: float,
              coils: np.ndarray | None = None) -> np.ndarray:
    """(A^H A + lam W) x, single coil or with coil sensitivities `coils` (Nc, P, Q)."""
    if coils is None:
        return AH(A(x, masks), masks) + lam * apply_W(x, S)
    return AH_coils(A_coils(x, masks, coils), masks, coils) + lam * apply_W(x, S)


def vdot(u: np.ndarray, v: np.ndarray) -> complex:
    return complex(np.vdot(u.ravel(), v.ravel()))


def cg(op, rhs: np.ndarray, x0: np.ndarray, n_iter: int) -> np.ndarray:
    """Plain (Hestenes-Stiefel) conjugate gradients for a Hermitian positive-definite operator,
    warm-started at x0, fixed iteration count, no preconditioner, no early exit."""
    x = x0.copy()
    r = rhs - op(x)
    p = r.copy()
    rr = vdot(r, r).real
    for _ in range(n_iter):
        q = op(p)
        alpha = rr / vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = vdot(r, r).real
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    return x


# ----------------------------------------------------------------------------------------------
# IRLS (Algorithm 1, epsilon schedule of Sec. III-C)
# ----------------------------------------------------------------------------------------------

def weight_from_x(x: np.ndarray, N1: int, N2: int, M: int, eps: float, p: float) -> np.ndarray:
    """Step 1 of Algorithm 1: Gram of x, eigendecomposition, weight, per-pixel S (M, M, P, Q)."""
    G = gram_fft(x, N1, N2, M)
    H, _ = weight_H(G, eps, p)
    return weight_S(diag_sums(H, N1, N2, M), x.shape[1], x.shape[2])


def initial_eps(x0: np.ndarray, N1: int, N2: int, M: int, frac: float = 0.01) -> float:
    """eps^(0) = lambda_max(G(x^(0))) / 100 (Sec. III-C)."""
    return frac * float(np.linalg.eigvalsh(gram_fft(x0, N1, N2, M))[-1])


def irls(kspace: np.ndarray, masks: np.ndarray, N1: int, N2: int, M: int, lam: float, p: float,
         n_irls: int, n_cg: int, gamma: float = 1.4, eps_frac: float = 0.01,
         history: list | None = None, coils: np.ndarray | None = None) -> np.ndarray:
    """Algorithm 1 with x^(0) = A^H b, eps^(0) = lambda_max / 100, eps <- eps / gamma.

    Iteration n uses the weight from x^(n-1) and eps^(n-1), then n_cg CG steps warm-started at
    x^(n-1). If `history` is a list, (eps, x) after each iteration is appended. With `coils`
    (Nc, P, Q) the k-space is coil-major (Nc, T, P, Q) and A is the multi-coil operator."""
    rhs = AH(kspace, masks) if coils is None else AH_coils(kspace, masks, coils)
    x = rhs.copy()
    eps = initial_eps(x, N1, N2, M, eps_frac)
    for _ in range(n_irls):
        S = weight_from_x(x, N1, N2, M, eps, p)
        x = cg(lambda v: normal_op(v, masks, S, lam, coils), rhs, x, n_cg)
        if history is not None:
            history.append((eps, x.copy()))
        eps = eps / gamma
    return x


def snr_db(x_true: np.ndarray, x_rec: np.ndarray) -> float:
    """SNR = 20 log10(||X_g|| / ||X_g - X_r||) (Sec. III-C)."""
    return 20.0 * np.log10(np.linalg.norm(x_true) / np.linalg.norm(x_true - x_rec))
