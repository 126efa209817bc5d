"""Plain FP64 CPU oracle of the FFT-Galerkin (GaNi) homogenization hot path.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct
restatement of what the GPU path computes.  Only the test suite, the smoke
check and the benchmark's CPU-baseline / reference arm may import it; the
product path (the C-ABI library and its Python binding) never does, and
shares no code, table or helper with it.

Every function follows one passage of Vondrejc, Zeman & Marek, "An FFT-based
Galerkin method for homogenization of periodic media" (arXiv:1311.0089):

  * Sec. 2 (Eq. FT_def)        frequencies xi(k) = (k_a / Y_a)_a
  * Sec. 4.1 (Eq. A4)          odd grids, Z_N^d = {-N_a/2 <= m_a < N_a/2}
  * Sec. 4.1 (Eq. DFT_def)     forward DFT carries 1/|N|, inverse unnormalised
  * Sec. 3 (Eq. Gamma_hat)     Gamma_hat(k) = xi (x) xi / (A0 xi . xi), 0 at k=0
  * Sec. 5.1 (Eq. FFT_matrices) Gamma_N = F^-1 Gamma_hat F,  G_N = Gamma_N A0
  * Sec. 5.1                   scalar product (u,v) = 1/|N| sum_k u^k . v^k
  * Sec. 5.2 (Eq. LSD, final_system)  [I + Gamma_N(A_N - A0)] e = E and
                               G_N A_N e~ = -G_N A_N E for A0 = lambda I
  * Sec. 5.3 (Lemma on CG)     CG on the non-symmetric G_N A_N from e~_0 in E_N
  * Sec. 5.3                   Moulinec-Suquet fixed point (Neumann series)
  * Sec. 5.1 (Eq. Helmholtz_discrete) R^{dN} = U_N (+) E_N (+) J_N; the dual
                               (flux) problem on J_N that Sec. 6 announces
  * Sec. 4.2 (Ga)              Galerkin approximation with exact integration,
                               for coefficients constant on the pixels of a grid
  * Sec. 3 (Eq. forms_def1)    energy a(e,e) -> homogenized matrix A_H
                               (A_H itself is not defined in the paper; the
                               energy reading is stated in the project notes)

Array conventions: a field is float64 of shape (d, *N) (component first,
spatial C order, first index slowest); a coefficient field is (d, d, *N).
The FFT is numpy's (a library primitive used as one step); `dft_naive`
writes the definition out as a dense sum and pins it on small grids.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "check_grid", "freq_index", "xi_axes", "dft", "idft", "dft_naive",
    "idft_naive", "gamma_hat", "apply_gamma", "apply_G", "apply_A", "apply_K",
    "inner", "ZERO_RHS", "cg", "homogenized_energy", "homogenized_flux", "solve_AH",
    "dense_gamma_matrix", "solve_lsd_dense", "moulinec_suquet",
    "apply_gamma_J", "invert_coeffs", "cg_dual", "solve_AH_dual", "solve_dual_dense",
    "cg_ref", "solve_AH_ref",
    "pixel_fourier_coeffs", "ga_quadrature_grid", "ga_coefficients", "apply_gamma_band", "solve_AH_ga",
    "solve_ga_dense",
]


# ---------------------------------------------------------------------------
# grid and frequencies (Sec. 4.1, Eq. A4; Sec. 2, Eq. FT_def)
# ---------------------------------------------------------------------------
def check_grid(N: Sequence[int]) -> Tuple[int, ...]:
    """Assumption (A4): every N_a is odd (Sec. 4.1)."""
    N = tuple(int(n) for n in N)
    if len(N) < 1 or any(n < 1 or n % 2 == 0 for n in N):
        raise ValueError(f"grid {N} violates (A4): every N_a must be odd")
    return N


def freq_index(n: int) -> np.ndarray:
    """Integer frequency m of storage bin j on an odd axis of length n.

    The grid Z_N = {-n/2 <= m < n/2} (Sec. 4.1) is stored 0-based; bin j holds
    m = j for j <= (n-1)/2 and m = j - n otherwise.  Since the DFT kernel
    omega^{km} (Eq. DFT_def) depends on k*m mod n only, this storage changes
    nothing in the transform itself; it fixes which xi multiplies each bin.
    """
    j = np.arange(n)
    return np.where(j <= (n - 1) // 2, j, j - n)


def xi_axes(N: Sequence[int], Y: Optional[Sequence[float]] = None) -> List[np.ndarray]:
    """xi_a(k) = k_a / Y_a per axis (Sec. 2, definition below Eq. FT_def)."""
    N = check_grid(N)
    if Y is None:
        Y = [1.0] * len(N)
    return [freq_index(n).astype(np.float64) / float(y) for n, y in zip(N, Y)]


def _xi_field(N, Y) -> np.ndarray:
    """The vector xi(k) on the whole grid, shape (d, *N)."""
    axes = xi_axes(N, Y)
    return np.stack(np.meshgrid(*axes, indexing="ij"))


# ---------------------------------------------------------------------------
# discrete Fourier transform (Sec. 4.1, Eq. DFT_def)
# ---------------------------------------------------------------------------
def dft(u: np.ndarray, d: Optional[int] = None) -> np.ndarray:
    """Forward DFT over the trailing d axes, normalised by 1/|N| (Eq. DFT_def)."""
    d = u.ndim if d is None else d
    axes = tuple(range(u.ndim - d, u.ndim))
    M = int(np.prod(u.shape[u.ndim - d:]))
    return np.fft.fftn(u, axes=axes) / M


def idft(U: np.ndarray, d: Optional[int] = None) -> np.ndarray:
    """Inverse DFT over the trailing d axes, unnormalised (Eq. DFT_def)."""
    d = U.ndim if d is None else d
    axes = tuple(range(U.ndim - d, U.ndim))
    M = int(np.prod(U.shape[U.ndim - d:]))
    return np.fft.ifftn(U, axes=axes) * M


def _dft_matrix(N: Sequence[int], sign: int) -> np.ndarray:
    """Dense matrix omega_N^{sign k m} over all multi-indices (Eq. DFT_def)."""
    N = tuple(N)
    ks = np.array(list(itertools.product(*[range(n) for n in N])), dtype=np.int64)
    phase = np.zeros((ks.shape[0], ks.shape[0]))
    for a, n in enumerate(N):
        phase += np.outer(ks[:, a], ks[:, a]) / n
    return np.exp(sign * 2j * np.pi * phase)


def dft_naive(u: np.ndarray, N: Sequence[int]) -> np.ndarray:
    """The forward DFT written out as the dense sum of Eq. DFT_def (small |N|).

    u has shape (..., *N); returns (1/|N|) sum_m u(x_m) omega^{-k m}."""
    N = tuple(N)
    M = int(np.prod(N))
    W = _dft_matrix(N, -1)
    lead = u.shape[: u.ndim - len(N)]
    flat = u.reshape(lead + (M,))
    return (flat @ W.T / M).reshape(lead + N)


def idft_naive(U: np.ndarray, N: Sequence[int]) -> np.ndarray:
    """Inverse of Eq. DFT_def as a dense sum: sum_m U(m) omega^{k m}."""
    N = tuple(N)
    M = int(np.prod(N))
    W = _dft_matrix(N, +1)
    lead = U.shape[: U.ndim - len(N)]
    flat = U.reshape(lead + (M,))
    return (flat @ W.T).reshape(lead + N)


# ---------------------------------------------------------------------------
# Green operator and projection (Sec. 3 Eq. Gamma_hat; Sec. 5.1 Eq. FFT_matrices)
# ---------------------------------------------------------------------------
def gamma_hat(N: Sequence[int], Y=None, A0: Optional[np.ndarray] = None) -> np.ndarray:
    """Gamma_hat(k) = xi(k) (x) xi(k) / (A0 xi(k) . xi(k)), zero at k = 0.

    Eq. Gamma_hat (Sec. 3) evaluated on Z_N^d (Sec. 5.1).  Returns (d, d, *N)."""
    N = check_grid(N)
    d = len(N)
    A0 = np.eye(d) if A0 is None else np.asarray(A0, dtype=np.float64)
    xi = _xi_field(N, Y)
    denom = np.einsum("ab,a...,b...->...", A0, xi, xi)
    G = np.einsum("a...,b...->ab...", xi, xi)
    zero = denom == 0.0
    denom = np.where(zero, 1.0, denom)
    G = G / denom
    G[(slice(None), slice(None)) + np.nonzero(zero)] = 0.0
    return G


def apply_gamma(u: np.ndarray, N, Y=None, A0=None) -> np.ndarray:
    """Gamma_N u = F^-1 Gamma_hat F u (Eq. FFT_matrices); u is (d, *N) real."""
    N = check_grid(N)
    d = len(N)
    Gh = gamma_hat(N, Y, A0)
    uh = dft(u, d)
    vh = np.einsum("ab...,b...->a...", Gh, uh)
    return idft(vh, d).real


def apply_G(u: np.ndarray, N, Y=None, A0=None) -> np.ndarray:
    """G_N u = Gamma_N A0 u (Eq. FFT_matrices)."""
    N = check_grid(N)
    d = len(N)
    A0m = np.eye(d) if A0 is None else np.asarray(A0, dtype=np.float64)
    return apply_gamma(np.einsum("ab,b...->a...", A0m, u), N, Y, A0)


def apply_A(A: np.ndarray, u: np.ndarray) -> np.ndarray:
    """A_N u: the block-diagonal coefficient matrix of Sec. 5.1 acting pointwise."""
    return np.einsum("ab...,b...->a...", A, u)


def apply_K(A: np.ndarray, u: np.ndarray, N, Y=None) -> np.ndarray:
    """K u = G_N A_N u with A0 = I, the system matrix of Eq. final_system."""
    return apply_G(apply_A(A, u), N, Y, None)


def inner(u: np.ndarray, v: np.ndarray) -> float:
    """(u, v) = 1/|N| sum_k u^k . v^k, the scalar product of Sec. 5.1."""
    M = u[0].size
    return float(np.sum(u * v)) / M


# ---------------------------------------------------------------------------
# conjugate gradients on Eq. final_system (Sec. 5.3)
# ---------------------------------------------------------------------------
ZERO_RHS = 1e-13   # ||b|| / ||A_N E|| below this is roundoff of an exact zero

def cg(A: np.ndarray, E: np.ndarray, N, Y=None, tol: float = 1e-10,
       maxiter: int = 10000, x0: Optional[np.ndarray] = None) -> Dict:
    """Solve G_N A_N x = -G_N A_N E by conjugate gradients (Sec. 5.3 Lemma).

    The paper proves that plain CG works on this non-symmetric system from
    any start in E_N.  The steps are the textbook Hestenes-Stiefel recursion:
      b = -K E;  r_0 = b - K x_0;  p_0 = r_0;
      q = K p;  alpha = (r,r)/(p,q);  x += alpha p;  r -= alpha q;
      beta = (r,r)_new/(r,r)_old;  p = r + beta p.
    Stop when ||r_i|| / ||b|| <= tol (relative recursive residual; the paper
    gives no criterion).  The sign of r follows Eq. final_system (r = b - K x),
    reading the printed r_0 = G A (e~_0 + E) as its negative.

    A right-hand side that vanishes in exact arithmetic (G kills constants,
    Lemma FD_projection (iv)) is roundoff in floating point; since G is an
    orthogonal projection, ||b|| <= ||A_N E||, and b is taken as zero when
    ||b|| <= ZERO_RHS * ||A_N E||.  Then x = x_0 and no iteration is made.
    """
    N = check_grid(N)
    d = len(N)
    Evec = np.asarray(E, dtype=np.float64).reshape((d,) + (1,) * d) * np.ones((d,) + N)
    b = -apply_K(A, Evec, N, Y)
    x = np.zeros((d,) + N) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_K(A, x, N, Y) if x0 is not None else b.copy()
    p = r.copy()
    rr = inner(r, r)
    bnorm = np.sqrt(inner(b, b))
    AE = apply_A(A, Evec)
    if bnorm <= ZERO_RHS * np.sqrt(inner(AE, AE)):
        bnorm = 0.0
    hist = [np.sqrt(rr) / bnorm if bnorm > 0 else 0.0]
    it = 0
    if bnorm == 0.0 or hist[0] <= tol:
        return {"x": x, "iters": 0, "rel_res": hist[0], "hist": hist,
                "true_rel_res": 0.0 if bnorm == 0 else hist[0], "b": b}
    while it < maxiter:
        q = apply_K(A, p, N, Y)
        alpha = rr / inner(p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rr_new = inner(r, r)
        hist.append(np.sqrt(rr_new) / bnorm)
        if hist[-1] <= tol:
            break
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    true_r = b - apply_K(A, x, N, Y)
    return {"x": x, "iters": it, "rel_res": hist[-1], "hist": hist,
            "true_rel_res": np.sqrt(inner(true_r, true_r)) / bnorm, "b": b}


# ---------------------------------------------------------------------------
# homogenized matrix (energy of the macroscopic loads, Eq. forms_def1)
# ---------------------------------------------------------------------------
def homogenized_energy(A: np.ndarray, e: Sequence[np.ndarray]) -> np.ndarray:
    """A_H[i][j] = (A_N e_j, e_i) with e_j = E_j + e~_j (energy form)."""
    d = len(e)
    AH = np.zeros((d, d))
    for i in range(d):
        for j in range(d):
            AH[i, j] = inner(apply_A(A, e[j]), e[i])
    return AH


def homogenized_flux(A: np.ndarray, e: Sequence[np.ndarray]) -> np.ndarray:
    """A_H[i][j] = <A_N e_j>_i, the mean flux of load j (equal to the energy
    form at convergence by Galerkin orthogonality, Eq. GaNiD with v = e~_i)."""
    d = len(e)
    AH = np.zeros((d, d))
    for j in range(d):
        flux = apply_A(A, e[j])
        for i in range(d):
            AH[i, j] = float(np.mean(flux[i]))
    return AH


def solve_AH(A: np.ndarray, N, Y=None, tol: float = 1e-10, maxiter: int = 10000,
             loads: Optional[Sequence[int]] = None) -> Dict:
    """Solve the cell problem for E = e_1..e_d and assemble A_H (Sec. 5.2-5.3)."""
    N = check_grid(N)
    d = len(N)
    loads = list(range(d)) if loads is None else list(loads)
    res = {"iters": [], "rel_res": [], "true_rel_res": [], "x": []}
    es = []
    for j in range(d):
        E = np.zeros(d)
        E[j] = 1.0
        out = cg(A, E, N, Y, tol, maxiter)
        res["iters"].append(out["iters"])
        res["rel_res"].append(out["rel_res"])
        res["true_rel_res"].append(out["true_rel_res"])
        res["x"].append(out["x"])
        es.append(E.reshape((d,) + (1,) * d) + out["x"])
    res["AH"] = homogenized_energy(A, es)
    res["AH_flux"] = homogenized_flux(A, es)
    return res


# ---------------------------------------------------------------------------
# dense discrete Lippmann-Schwinger solve (Sec. 5.2, Eq. LSD) for tiny grids
# ---------------------------------------------------------------------------
def dense_gamma_matrix(N, Y=None, A0=None) -> np.ndarray:
    """Gamma_N = F^-1 Gamma_hat F as a dense real (d|N|) x (d|N|) matrix.

    Built from the dense DFT matrices of Eq. FFT_matrices (not from an FFT),
    with index order (component, flat grid index)."""
    N = check_grid(N)
    d = len(N)
    M = int(np.prod(N))
    F = _dft_matrix(N, -1) / M
    Fi = _dft_matrix(N, +1)
    Gh = gamma_hat(N, Y, A0).reshape(d, d, M)
    out = np.zeros((d * M, d * M), dtype=np.complex128)
    for a in range(d):
        for b in range(d):
            out[a * M:(a + 1) * M, b * M:(b + 1) * M] = Fi @ (Gh[a, b][:, None] * F)
    return out.real


def solve_lsd_dense(A: np.ndarray, E: np.ndarray, N, Y=None, lam: float = 1.0,
                    A0: Optional[np.ndarray] = None) -> np.ndarray:
    """Solve [I + Gamma_N (A_N - A0)] e = E by LU (Eq. LSD) with A0 = lam I, or
    the given SPD A0; returns e (d, *N)."""
    N = check_grid(N)
    d = len(N)
    M = int(np.prod(N))
    A0m = lam * np.eye(d) if A0 is None else np.asarray(A0, dtype=np.float64)
    Gam = dense_gamma_matrix(N, Y, A0m)
    Ad = np.zeros((d * M, d * M))
    Af = A.reshape(d, d, M)
    idx = np.arange(M)
    for a in range(d):
        for b in range(d):
            Ad[a * M + idx, b * M + idx] = Af[a, b] - A0m[a, b]
    sysm = np.eye(d * M) + Gam @ Ad
    rhs = np.repeat(np.asarray(E, dtype=np.float64), M)
    e = np.linalg.solve(sysm, rhs)
    return e.reshape((d,) + N)


# ---------------------------------------------------------------------------
# Moulinec-Suquet fixed point (Sec. 5.3, Neumann series for Eq. LSD)
# ---------------------------------------------------------------------------
def moulinec_suquet(A: np.ndarray, E: np.ndarray, N, Y=None, lam: float = 1.0,
                    tol: float = 1e-10, maxiter: int = 100000) -> Dict:
    """e_i = -Gamma_N (A_N - lam I) e_{i-1} + E, from e_0 = E (Sec. 5.3).

    Stops when ||e_i - e_{i-1}|| / ||E|| <= tol (the paper gives no criterion).
    """
    N = check_grid(N)
    d = len(N)
    A0 = lam * np.eye(d)
    Evec = np.asarray(E, dtype=np.float64).reshape((d,) + (1,) * d) * np.ones((d,) + N)
    e = Evec.copy()
    Enorm = np.sqrt(inner(Evec, Evec))
    it = 0
    step = np.inf
    while it < maxiter:
        tau = apply_A(A, e) - np.einsum("ab,b...->a...", A0, e)
        e_new = Evec - apply_gamma(tau, N, Y, A0)
        step = np.sqrt(inner(e_new - e, e_new - e)) / Enorm
        e = e_new
        it += 1
        if step <= tol:
            break
    return {"e": e, "iters": it, "step": step}


# ---------------------------------------------------------------------------
# dual (flux) formulation on J_N (Eq. Helmholtz_discrete; announced in Sec. 6)
# ---------------------------------------------------------------------------
def apply_gamma_J(u: np.ndarray, N, Y=None) -> np.ndarray:
    """Orthogonal projection onto J_N (zero-mean divergence-free grid fields).

    Eq. Helmholtz_discrete splits R^{dN} into the mutually orthogonal U_N
    (constants), E_N and J_N, so the projection onto J_N is the identity minus
    the projection onto U_N (the grid mean) minus Gamma_N (the orthogonal
    projection onto E_N for A0 = I, Lemma FD_projection)."""
    N = check_grid(N)
    d = len(N)
    mean = u.reshape(d, -1).mean(axis=1).reshape((d,) + (1,) * d)
    return u - mean - apply_gamma(u, N, Y)


def invert_coeffs(A: np.ndarray) -> np.ndarray:
    """A(x_k)^-1 per voxel, (d, d, *N) -> (d, d, *N)."""
    d = A.shape[0]
    m = np.moveaxis(A.reshape(d, d, -1), 2, 0)
    inv = np.linalg.inv(m)
    return np.moveaxis(inv, 0, 2).reshape(A.shape)


def cg_dual(A: np.ndarray, S: np.ndarray, N, Y=None, tol: float = 1e-10,
            maxiter: int = 10000) -> Dict:
    """Dual GaNi problem: the flux s = S + s~ with s~ in J_N and
    (A_N^-1 s, t) = 0 for all t in J_N, i.e. G_J A_N^-1 s~ = -G_J A_N^-1 S
    with G_J the projection onto J_N.  G_J A_N^-1 is symmetric positive
    definite on J_N, so the CG steps of `cg` apply unchanged (same stopping
    rule and zero right-hand-side rule)."""
    N = check_grid(N)
    d = len(N)
    Ainv = invert_coeffs(A)
    K = lambda u: apply_gamma_J(apply_A(Ainv, u), N, Y)
    Svec = np.asarray(S, dtype=np.float64).reshape((d,) + (1,) * d) * np.ones((d,) + N)
    b = -K(Svec)
    x = np.zeros((d,) + N)
    r = b.copy()
    p = r.copy()
    rr = inner(r, r)
    bnorm = np.sqrt(rr)
    AS = apply_A(Ainv, Svec)
    if bnorm <= ZERO_RHS * np.sqrt(inner(AS, AS)):
        bnorm = 0.0
    if bnorm == 0.0:
        return {"x": x, "iters": 0, "rel_res": 0.0}
    it = 0
    rel = 1.0
    while it < maxiter and rel > tol:
        q = K(p)
        alpha = rr / inner(p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rr_new = inner(r, r)
        rel = np.sqrt(rr_new) / bnorm
        p = r + (rr_new / rr) * p
        rr = rr_new
    return {"x": x, "iters": it, "rel_res": rel}


def solve_AH_dual(A: np.ndarray, N, Y=None, tol: float = 1e-10, maxiter: int = 10000) -> Dict:
    """Unit flux loads S = e_j: the homogenized compliance
    C_H[i][j] = (A_N^-1 s_j, s_i) (energy form) and <A_N^-1 s_j>_i (mean
    field, flux form), and A_H = C_H^-1 from each."""
    N = check_grid(N)
    d = len(N)
    Ainv = invert_coeffs(A)
    ss, iters, xs = [], [], []
    for j in range(d):
        S = np.zeros(d)
        S[j] = 1.0
        out = cg_dual(A, S, N, Y, tol, maxiter)
        iters.append(out["iters"])
        xs.append(out["x"])
        ss.append(S.reshape((d,) + (1,) * d) + out["x"])
    CH = homogenized_energy(Ainv, ss)
    CH_flux = homogenized_flux(Ainv, ss)
    return {"CH": CH, "CH_flux": CH_flux, "AH": np.linalg.inv(CH), "AH_flux": np.linalg.inv(CH_flux),
            "iters": iters, "x": xs}


def solve_dual_dense(A: np.ndarray, S: np.ndarray, N, Y=None) -> np.ndarray:
    """Dense route to s~ for tiny grids: with P_J the projection onto J_N
    assembled from the dense DFT matrices (identity minus mean minus dense
    Gamma_N), solve [P_J A^-1 P_J + (I - P_J)] s~ = -P_J A^-1 S by LU (the
    second term makes the matrix regular off J_N without touching J_N)."""
    N = check_grid(N)
    d = len(N)
    M = int(np.prod(N))
    Gam = dense_gamma_matrix(N, Y, None)
    Pu = np.kron(np.eye(d), np.full((M, M), 1.0 / M))
    PJ = np.eye(d * M) - Pu - Gam
    Ai = invert_coeffs(A).reshape(d, d, M)
    Ad = np.zeros((d * M, d * M))
    idx = np.arange(M)
    for a in range(d):
        for b in range(d):
            Ad[a * M + idx, b * M + idx] = Ai[a, b]
    sysm = PJ @ Ad @ PJ + (np.eye(d * M) - PJ)
    rhs = -PJ @ (Ad @ np.repeat(np.asarray(S, dtype=np.float64), M))
    return np.linalg.solve(sysm, rhs).reshape((d,) + N)


# ---------------------------------------------------------------------------
# CG with a general reference medium A0 (Lemma FD_projection (ii)-(iii))
# ---------------------------------------------------------------------------
def cg_ref(A: np.ndarray, E: np.ndarray, N, A0: np.ndarray, Y=None, tol: float = 1e-10,
           maxiter: int = 10000) -> Dict:
    """The discrete Lippmann-Schwinger equation (Eq. LSD) with a general SPD
    reference medium A0, on the fluctuation x = e - E in E_N:

        Gamma_N A_N x = -Gamma_N A_N E,   Gamma_N = F^-1 Gamma_hat(A0) F,

    (Gamma_N A0 x = x on E_N, since G_N = Gamma_N A0 projects onto E_N, Lemma
    FD_projection (iii)).  By Lemma FD_projection (ii) Gamma_N is symmetric,
    so K = Gamma_N A_N satisfies (A0 K x, y) = (A_N x, y) for x, y in E_N:
    K is symmetric positive definite in the scalar product (u, v)_A0 =
    (A0 u, v), and CG runs in that product.  Stops on ||r||_A0 / ||b||_A0.
    For A0 = lam I the iterates are those of `cg`."""
    N = check_grid(N)
    d = len(N)
    A0 = np.asarray(A0, dtype=np.float64)
    K = lambda u: apply_gamma(apply_A(A, u), N, Y, A0)
    ip = lambda u, v: inner(np.einsum("ab,b...->a...", A0, u), v)
    Evec = np.asarray(E, dtype=np.float64).reshape((d,) + (1,) * d) * np.ones((d,) + N)
    b = -K(Evec)
    x = np.zeros((d,) + N)
    r = b.copy()
    p = r.copy()
    rr = ip(r, r)
    bnorm = np.sqrt(rr)
    # zero right-hand side: ||b||_A0 <= sqrt(lmax) ||b|| <= sqrt(lmax)/lmin ||A E||
    ev = np.linalg.eigvalsh(A0)
    AE = apply_A(A, Evec)
    if bnorm <= ZERO_RHS * np.sqrt(ev[-1]) / ev[0] * np.sqrt(inner(AE, AE)):
        return {"x": x, "iters": 0, "rel_res": 0.0}
    it, rel = 0, 1.0
    while it < maxiter and rel > tol:
        q = K(p)
        alpha = rr / ip(p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rr_new = ip(r, r)
        rel = np.sqrt(rr_new) / bnorm
        p = r + (rr_new / rr) * p
        rr = rr_new
    return {"x": x, "iters": it, "rel_res": rel}


def solve_AH_ref(A: np.ndarray, N, A0: np.ndarray, Y=None, tol: float = 1e-10,
                 maxiter: int = 10000) -> Dict:
    """`solve_AH` with the general reference medium A0 (same A_H: the GaNi
    solution does not depend on A0)."""
    N = check_grid(N)
    d = len(N)
    es, iters, xs = [], [], []
    for j in range(d):
        E = np.zeros(d)
        E[j] = 1.0
        out = cg_ref(A, E, N, A0, Y, tol, maxiter)
        iters.append(out["iters"])
        xs.append(out["x"])
        es.append(E.reshape((d,) + (1,) * d) + out["x"])
    return {"AH": homogenized_energy(A, es), "AH_flux": homogenized_flux(A, es), "iters": iters, "x": xs}


# ---------------------------------------------------------------------------
# Galerkin approximation with exact integration (Sec. 4.2, Ga) for
# coefficients constant on the pixels of a grid P
# ---------------------------------------------------------------------------
def pixel_fourier_coeffs(A_pix: np.ndarray, N: Sequence[int]) -> np.ndarray:
    """Fourier coefficients A_hat(l), |l_a| <= N_a - 1, of A constant on the
    pixels of the grid P = A_pix.shape[2:] (pixel k centred at x_k = k h,
    width h = 2 Y / P).  Integrating exp(-i pi xi(l) . x) over a pixel gives
    its centre value times prod_a sinc(l_a / P_a) (sinc(t) = sin(pi t)/(pi t)),
    so A_hat(l) = DFT_P(A)(l mod P) prod_a sinc(l_a / P_a).
    Returns (d, d, 2N_1 - 1, ...), index l + N - 1."""
    P = A_pix.shape[2:]
    nd = len(P)
    Ah = dft(A_pix, nd)
    idx = np.ix_(*[np.arange(-(n - 1), n) % p for n, p in zip(N, P)])
    out = Ah[(slice(None), slice(None)) + idx]
    for a, (n, p) in enumerate(zip(N, P)):
        shape = [1] * (nd + 2)
        shape[2 + a] = 2 * n - 1
        out = out * np.sinc(np.arange(-(n - 1), n) / p).reshape(shape)
    return out


def ga_quadrature_grid(N: Sequence[int]) -> Tuple[int, ...]:
    """The smallest odd M_a >= 2 N_a - 1 (a product of two trigonometric
    polynomials of the trial space Z_N then integrates exactly on M)."""
    return tuple(2 * n - 1 for n in N)


def ga_coefficients(A_pix: np.ndarray, N: Sequence[int], M: Sequence[int]) -> np.ndarray:
    """Values on the grid M of the Fourier series of A truncated to |l_a| <=
    N_a - 1: the frequencies a product of two trial functions reaches, so for
    u, v of the trial space mean_M(A_M u . v) is the exact integral of
    A u . v (for M_a >= 2 N_a - 1).  Not SPD pointwise in general."""
    Ahat = pixel_fourier_coeffs(A_pix, N)
    spec = np.zeros(A_pix.shape[:2] + tuple(M), dtype=np.complex128)
    idx = np.ix_(*[np.arange(-(n - 1), n) % m for n, m in zip(N, M)])
    spec[(slice(None), slice(None)) + idx] = Ahat
    return idft(spec, len(M)).real


def apply_gamma_band(u: np.ndarray, M, N, Y=None, dual: bool = False) -> np.ndarray:
    """Gamma_N (or the projection onto J_N for dual) on the grid M, followed by
    the removal of every frequency outside the trial space Z_N."""
    M = check_grid(M)
    d = len(M)
    uh = dft(u, d)
    if dual:
        xi = _xi_field(M, Y)
        den = np.einsum("a...,a...->...", xi, xi)
        num = np.einsum("a...,a...->...", xi, uh)
        zero = den == 0
        vh = uh - xi * np.where(zero, 0.0, num / np.where(zero, 1.0, den))
        vh[(slice(None),) + tuple([0] * d)] = 0.0
    else:
        vh = np.einsum("ab...,b...->a...", gamma_hat(M, Y), uh)
    band = np.ones(M, dtype=bool)
    for a, (m, n) in enumerate(zip(M, N)):
        shape = [1] * d
        shape[a] = m
        band &= (np.abs(freq_index(m)) <= (n - 1) // 2).reshape(shape)
    vh = vh * band
    return idft(vh, d).real


def solve_AH_ga(A_pix: np.ndarray, N, M=None, Y=None, tol: float = 1e-12, maxiter: int = 10000,
                dual: bool = False) -> Dict:
    """Ga on the trial space Z_N for pixel-constant A: CG (the steps of `cg`)
    on the grid M with the band-limited projection and the coefficients
    `ga_coefficients`; A_H from the exact energy.  Ga minimises the energy over
    a subspace of the continuous problem's fields, so its A_H bounds the
    homogenized matrix of the pixelated medium from above; the dual (fluxes on
    the band-limited J_N, coefficients A^-1) bounds it from below."""
    N = check_grid(N)
    d = len(N)
    M = check_grid(ga_quadrature_grid(N) if M is None else M)
    C = invert_coeffs(A_pix) if dual else A_pix
    AM = ga_coefficients(C, N, M)
    K = lambda u: apply_gamma_band(apply_A(AM, u), M, N, Y, dual)
    es, iters = [], []
    for j in range(d):
        E = np.zeros(d)
        E[j] = 1.0
        Evec = E.reshape((d,) + (1,) * d) * np.ones((d,) + M)
        b = -K(Evec)
        x = np.zeros((d,) + M)
        r = b.copy()
        p = r.copy()
        rr = inner(r, r)
        bnorm = np.sqrt(rr)
        AE = apply_A(AM, Evec)
        it = 0
        if bnorm > ZERO_RHS * np.sqrt(inner(AE, AE)):
            rel = 1.0
            while it < maxiter and rel > tol:
                q = K(p)
                alpha = rr / inner(p, q)
                x = x + alpha * p
                r = r - alpha * q
                it += 1
                rr_new = inner(r, r)
                rel = np.sqrt(rr_new) / bnorm
                p = r + (rr_new / rr) * p
                rr = rr_new
        iters.append(it)
        es.append(Evec + x)
    H = homogenized_energy(AM, es)
    out = {"iters": iters, "M": M}
    if dual:
        out["CH"] = H
        out["AH"] = np.linalg.inv(H)
    else:
        out["AH"] = H
    return out


def solve_ga_dense(A_pix: np.ndarray, N, Y=None) -> np.ndarray:
    """Ga assembled in Fourier space for tiny trial spaces: e = E + e~ with
    e~_hat(m) = xi(m) c(m) (curl-free), and the exact energy
    sum_{m,n} conj(e_hat(n)) . A_hat(n - m) e_hat(m); its minimiser solves
    sum_{m != 0} xi(n)^T A_hat(n - m) xi(m) c(m) = -xi(n)^T A_hat(n) E for
    n != 0.  Returns A_H (d x d)."""
    N = check_grid(N)
    d = len(N)
    Ahat = pixel_fourier_coeffs(A_pix, N)
    grids = np.meshgrid(*[freq_index(n) for n in N], indexing="ij")
    ms = np.stack([g.ravel() for g in grids], axis=1)
    Yv = [1.0] * d if Y is None else Y
    xi = ms / np.asarray(Yv, dtype=np.float64)
    nz = [i for i in range(len(ms)) if np.any(ms[i] != 0)]
    off = np.asarray(N) - 1

    def Ah(l):
        return Ahat[(slice(None), slice(None)) + tuple(l + off)]

    AH = np.zeros((d, d))
    es = []
    for j in range(d):
        E = np.zeros(d)
        E[j] = 1.0
        K = np.zeros((len(nz), len(nz)), dtype=np.complex128)
        rhs = np.zeros(len(nz), dtype=np.complex128)
        for a, n in enumerate(nz):
            rhs[a] = -xi[n] @ Ah(ms[n]) @ E
            for b, m in enumerate(nz):
                K[a, b] = xi[n] @ Ah(ms[n] - ms[m]) @ xi[m]
        c = np.linalg.solve(K, rhs)
        eh = {tuple(ms[n]): xi[n] * c[a] for a, n in enumerate(nz)}
        eh[tuple([0] * d)] = E.astype(np.complex128)
        es.append(eh)
    for i in range(d):
        for j in range(d):
            tot = 0.0
            for kn, en in es[i].items():
                for km, em in es[j].items():
                    tot += np.conj(en) @ Ah(np.array(kn) - np.array(km)) @ em
            AH[i, j] = tot.real
    return AH
