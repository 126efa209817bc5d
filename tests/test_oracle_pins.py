"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a lemma of the paper, a dense direct solve built from the matrix
definitions, or an exact homogenization result.  A dropped 1/|N|, a flipped
sign in the DFT kernel, a wrong frequency map, a transposed operand or a
missing term in the projection fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

RNG = np.random.default_rng(1311)


def rand_field(N, d=None, rng=RNG):
    d = len(N) if d is None else d
    return rng.standard_normal((d,) + tuple(N))


# ----------------------------------------------------------------- DFT (Eq. DFT_def)
@pytest.mark.parametrize("N", [(3,), (5,), (3, 5), (5, 3, 7), (9, 5)])
def test_dft_matches_dense_definition(N):
    u = RNG.standard_normal(N) + 1j * RNG.standard_normal(N)
    np.testing.assert_allclose(O.dft(u), O.dft_naive(u, N), atol=1e-13)
    np.testing.assert_allclose(O.idft(u), O.idft_naive(u, N), atol=1e-12)


def test_freq_index_symmetric_range():
    # Z_N = {-N/2 <= m < N/2} for odd N (Sec. 4.1)
    assert list(O.freq_index(5)) == [0, 1, 2, -2, -1]
    assert list(O.freq_index(1)) == [0]
    assert sorted(O.freq_index(7)) == list(range(-3, 4))


@pytest.mark.parametrize("N,m0", [((5, 7), (2, -3)), ((9,), (-4,)), ((3, 5, 3), (1, 2, -1))])
def test_dft_single_exponential_closed_form(N, m0):
    # u(x_k) = exp(2 pi i k.m0/N) is the basis function of frequency m0, so
    # its forward DFT (with 1/|N|) is exactly 1 at bin m0 and 0 elsewhere.
    ks = np.meshgrid(*[np.arange(n) for n in N], indexing="ij")
    ph = sum(k * m / n for k, m, n in zip(ks, m0, N))
    u = np.exp(2j * np.pi * ph)
    U = O.dft(u)
    idx = tuple(m % n for m, n in zip(m0, N))
    assert abs(U[idx] - 1.0) < 1e-13
    U[idx] = 0
    assert np.max(np.abs(U)) < 1e-13


def test_dft_constant_and_parseval():
    N = (7, 5)
    u = 3.25 * np.ones(N)
    U = O.dft(u)
    assert abs(U[0, 0] - 3.25) < 1e-14
    U[0, 0] = 0
    assert np.max(np.abs(U)) < 1e-13
    # Plancherel / Eq. scal_trig_pol: 1/|N| sum u v = sum_k U(k) conj(V(k))
    a, b = RNG.standard_normal(N), RNG.standard_normal(N)
    lhs = np.mean(a * b)
    rhs = np.sum(O.dft(a) * np.conj(O.dft(b))).real
    assert abs(lhs - rhs) < 1e-13


# ------------------------------------------------- projection (Lemma FD_projection)
def trig_gradient(N, m, Y=None, phase=0.3):
    """Grid values of grad f, f(x) = cos(pi xi(m).x + phase), on x_k = k h."""
    d = len(N)
    Y = [1.0] * d if Y is None else Y
    ks = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in N], indexing="ij")
    # pi xi(m).x_k with x_k = k h, h = 2Y/N:  = 2 pi sum m_a k_a / N_a
    arg = sum(2 * np.pi * m[a] * ks[a] / N[a] for a in range(d)) + phase
    return np.stack([-np.pi * m[a] / Y[a] * np.sin(arg) for a in range(d)])


@pytest.mark.parametrize("N,m,Y", [((7, 5), (2, -1), None), ((9, 7), (-3, 3), (1.0, 2.5)),
                                   ((5, 5, 7), (1, -2, 3), (1.0, 0.5, 2.0))])
def test_gamma_is_identity_on_gradients(N, m, Y):
    g = trig_gradient(N, m, Y)
    np.testing.assert_allclose(O.apply_gamma(g, N, Y), g, atol=1e-12)
    # also for a general SPD reference medium: G = Gamma A0 keeps E_N fixed
    d = len(N)
    A0 = np.eye(d) * 2.0 + 0.3
    np.testing.assert_allclose(O.apply_G(g, N, Y, A0), g, atol=1e-12)


@pytest.mark.parametrize("N,m,Y", [((7, 5), (2, -1), (1.0, 3.0)), ((5, 5, 7), (1, -2, 3), None)])
def test_gamma_kills_divergence_free(N, m, Y):
    g = trig_gradient(N, m, Y)
    d = len(N)
    if d == 2:
        v = np.stack([g[1], -g[0]])      # rotated gradient: divergence free
    else:
        c = np.array([0.3, -1.1, 0.7])
        # xi x c times the same scalar wave: divergence free by construction
        Yv = [1.0] * d if Y is None else Y
        xi = np.array([m[a] / Yv[a] for a in range(d)])
        w = np.cross(xi, c)
        s = g[0] / (-np.pi * xi[0])
        v = np.stack([w[a] * s for a in range(d)])
    np.testing.assert_allclose(O.apply_gamma(v, N, Y), 0.0, atol=1e-12)


@pytest.mark.parametrize("N", [(5, 7), (9, 9), (3, 5, 7)])
def test_gamma_projection_lemma(N):
    u, v = rand_field(N), rand_field(N)
    Gu = O.apply_gamma(u, N)
    np.testing.assert_allclose(O.apply_gamma(Gu, N), Gu, atol=1e-12)          # (iii)
    assert abs(O.inner(Gu, v) - O.inner(u, O.apply_gamma(v, N))) < 1e-12      # (v)
    const = np.ones((len(N),) + N) * np.arange(1, len(N) + 1).reshape((-1,) + (1,) * len(N))
    np.testing.assert_allclose(O.apply_gamma(const, N), 0.0, atol=1e-13)      # (iv)
    # zero mean output
    assert np.max(np.abs(Gu.reshape(len(N), -1).mean(axis=1))) < 1e-13
    # lambda independence (v)
    d = len(N)
    np.testing.assert_allclose(O.apply_G(u, N, None, 3.7 * np.eye(d)), Gu, atol=1e-12)
    # the complex result of F^-1 Gamma_hat F on real data is real
    uh = O.dft(u, d)
    vh = np.einsum("ab...,b...->a...", O.gamma_hat(N), uh)
    assert np.max(np.abs(O.idft(vh, d).imag)) < 1e-12


def test_general_reference_medium_projection_not_orthogonal():
    N = (7, 9)
    A0 = np.array([[3.0, 1.0], [1.0, 2.0]])
    u, v = rand_field(N), rand_field(N)
    Gu = O.apply_G(u, N, None, A0)
    np.testing.assert_allclose(O.apply_G(Gu, N, None, A0), Gu, atol=1e-12)
    # Lemma (ii): G^* A0 = A0 G, i.e. (G u, A0 v) = (A0 u, G v)
    lhs = O.inner(Gu, np.einsum("ab,b...->a...", A0, v))
    rhs = O.inner(np.einsum("ab,b...->a...", A0, u), O.apply_G(v, N, None, A0))
    assert abs(lhs - rhs) < 1e-12
    # ... but G is not self-adjoint in the plain scalar product
    assert abs(O.inner(Gu, v) - O.inner(u, O.apply_G(v, N, None, A0))) > 1e-6


def test_dense_gamma_equals_fft_gamma():
    N = (5, 3)
    u = rand_field(N)
    Gd = O.dense_gamma_matrix(N)
    np.testing.assert_allclose((Gd @ u.reshape(-1)).reshape(u.shape),
                               O.apply_gamma(u, N), atol=1e-12)


# ---------------------------------------- CG vs dense LU of the discrete L-S equation
@pytest.mark.parametrize("N,kind", [((3, 3), "phase"), ((5, 3), "spd"), ((5, 5), "phase"),
                                    ((3, 3, 3), "spd"), ((3, 5, 3), "phase")])
def test_cg_matches_dense_lsd(N, kind):
    rng = np.random.default_rng(7)
    d = len(N)
    if kind == "phase":
        ph = (rng.random(N) < 0.4).astype(np.uint8)
        ms = W.Microstructure(N, ph, W.isotropic_table([1.0, 25.0], d))
        A = ms.full_field()
    else:
        A = W.random_spd_field(N, rng, 1.0, 30.0)
    for j in range(d):
        E = np.zeros(d)
        E[j] = 1.0
        sol = O.cg(A, E, N, tol=1e-13, maxiter=500)
        for lam in (1.0, 4.0):
            e = O.solve_lsd_dense(A, E, N, lam=lam)
            x_lu = e - E.reshape((d,) + (1,) * d)
            err = np.sqrt(O.inner(sol["x"] - x_lu, sol["x"] - x_lu))
            ref = np.sqrt(O.inner(x_lu, x_lu)) + 1e-300
            assert err / ref < 1e-10, (lam, err / ref)


def test_cg_independent_of_start_in_EN():
    N = (9, 7)
    rng = np.random.default_rng(3)
    A = W.random_spd_field(N, rng, 1.0, 50.0)
    E = np.array([1.0, 0.0])
    a = O.cg(A, E, N, tol=1e-13)
    x0 = O.apply_gamma(rand_field(N, rng=rng), N)       # a start inside E_N
    b = O.cg(A, E, N, tol=1e-13, x0=x0)
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-10)
    # iterates stay in E_N
    np.testing.assert_allclose(O.apply_gamma(a["x"], N), a["x"], atol=1e-12)


# ------------------------------------------------------------------ A_H closed forms
def test_homogeneous_medium_exact():
    N = (7, 5, 3)
    A0 = np.array([[4.0, 1.0, 0.5], [1.0, 3.0, 0.2], [0.5, 0.2, 2.0]])
    A = np.broadcast_to(A0[:, :, None, None, None], (3, 3) + N).copy()
    res = O.solve_AH(A, N)
    # b = -G A E is zero in exact arithmetic (G kills constants, Lemma
    # FD_projection (iv)); its roundoff is recognised and no step is taken.
    assert res["iters"] == [0, 0, 0]
    np.testing.assert_allclose(res["AH"], A0, atol=1e-13)


@pytest.mark.parametrize("N,axis", [((9, 5), 0), ((7, 9), 1), ((7, 3, 5), 0), ((3, 5, 7), 2)])
def test_laminate_exact(N, axis):
    # A(x) = a(x_axis) I: A_H = harmonic mean across the layers and the
    # arithmetic mean along them, exactly for the grid values.
    rng = np.random.default_rng(11 + axis)
    d = len(N)
    a = np.exp(rng.uniform(0, np.log(100.0), size=N[axis]))
    shape = [1] * d
    shape[axis] = N[axis]
    af = np.broadcast_to(a.reshape(shape), N)
    A = np.einsum("ab,...->ab...", np.eye(d), af)
    res = O.solve_AH(A, N, tol=1e-14)
    harm = 1.0 / np.mean(1.0 / a)
    arith = np.mean(a)
    expect = np.eye(d) * arith
    expect[axis, axis] = harm
    np.testing.assert_allclose(res["AH"], expect, rtol=1e-11, atol=1e-12)
    # loads along the layers see b = -G A E = 0 (xi . t_hat vanishes on the
    # Fourier line of a field that varies along `axis` only): no real iteration
    assert all(res["iters"][j] == 0 for j in range(d) if j != axis)


@pytest.mark.parametrize("N,seed", [((15, 15), 1), ((9, 11), 2), ((7, 5, 9), 3)])
def test_voigt_reuss_bounds_and_symmetry(N, seed):
    rng = np.random.default_rng(seed)
    d = len(N)
    A = W.random_spd_field(N, rng, 1.0, 200.0)
    res = O.solve_AH(A, N, tol=1e-12)
    AH = res["AH"]
    np.testing.assert_allclose(AH, AH.T, atol=1e-12)
    np.testing.assert_allclose(res["AH_flux"], AH, rtol=1e-8, atol=1e-9)
    voigt = A.reshape(d, d, -1).mean(axis=2)
    Ainv = np.linalg.inv(np.moveaxis(A.reshape(d, d, -1), 2, 0))
    reuss = np.linalg.inv(Ainv.mean(axis=0))
    assert np.min(np.linalg.eigvalsh(voigt - AH)) > -1e-10
    assert np.min(np.linalg.eigvalsh(AH - reuss)) > -1e-10
    # strictly inside for a genuinely heterogeneous medium
    assert np.max(np.linalg.eigvalsh(voigt - AH)) > 1e-3


def test_keller_duality_2d():
    # For scalar isotropic a(x) in 2D, a' = c / a gives A_H' = c R A_H^-1 R^T.
    ms = W.circles_2d(n=45, count=6, r_lo=3, r_hi=8, contrast=20.0, seed=5)
    a1, a2 = 1.0, 20.0
    A = ms.full_field()
    dual = W.Microstructure(ms.N, ms.phase, W.isotropic_table([a2, a1], 2))
    Ad = dual.full_field()
    r1 = O.solve_AH(A, ms.N, tol=1e-13)
    r2 = O.solve_AH(Ad, ms.N, tol=1e-13)
    R = np.array([[0.0, -1.0], [1.0, 0.0]])
    predicted = a1 * a2 * R @ np.linalg.inv(r1["AH"]) @ R.T
    np.testing.assert_allclose(r2["AH"], predicted, rtol=1e-9)


def test_square_inclusion_symmetry():
    ms = W.square_inclusion_15()
    res = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)
    AH = res["AH"]
    assert abs(AH[0, 0] - AH[1, 1]) < 1e-12 * AH[0, 0]
    assert abs(AH[0, 1]) < 1e-12
    assert 1.0 < AH[0, 0] < 10.0


# -------------------------------------------------------------- convergence claims
def test_cg_iterations_grow_like_sqrt_contrast_and_ms_like_contrast():
    base = W.circles_2d(n=45, count=8, r_lo=3, r_hi=7, contrast=10.0, seed=9)
    its_cg, its_ms = [], []
    rhos = [10.0, 100.0, 1000.0]
    for rho in rhos:
        A = W.Microstructure(base.N, base.phase, W.isotropic_table([1.0, rho], 2)).full_field()
        its_cg.append(O.cg(A, np.array([1.0, 0.0]), base.N, tol=1e-8)["iters"])
        if rho <= 100.0:
            lam = 0.5 * (1.0 + rho)          # optimal reference medium
            its_ms.append(O.moulinec_suquet(A, np.array([1.0, 0.0]), base.N, lam=lam,
                                            tol=1e-8)["iters"])
    slope_cg = np.polyfit(np.log(rhos), np.log(its_cg), 1)[0]
    slope_ms = np.log(its_ms[1] / its_ms[0]) / np.log(10.0)
    assert slope_cg < 0.6, its_cg          # ~ sqrt(rho) or better
    assert slope_ms > 0.7, its_ms          # ~ rho
    assert its_ms[1] > 3 * its_cg[1]


def test_moulinec_suquet_reaches_the_same_solution():
    N = (15, 15)
    ms = W.square_inclusion_15()
    A = ms.full_field()
    E = np.array([1.0, 0.0])
    cg = O.cg(A, E, N, tol=1e-13)
    msr = O.moulinec_suquet(A, E, N, lam=5.5, tol=1e-14)
    np.testing.assert_allclose(msr["e"] - E.reshape(2, 1, 1), cg["x"], atol=1e-10)


def test_rejects_even_grid():
    with pytest.raises(ValueError):
        O.check_grid((4, 5))


def test_golden_laminate_fixture():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "laminate_9x7.json")))
    ms = W.laminate(tuple(g["N"]), g["layers_axis0"])
    res = O.solve_AH(ms.full_field(), ms.N, tol=1e-14)
    np.testing.assert_allclose(res["AH"], np.array(g["AH"]), rtol=1e-12, atol=1e-13)


def _smooth_field(N, a_of_x):
    """Isotropic a(x) I sampled at x_k = 2 k / N (one period of the cell
    [-1, 1]^d, up to a shift, which leaves A_H unchanged)."""
    d = len(N)
    xs = np.meshgrid(*[2.0 * np.arange(n) / n for n in N], indexing="ij")
    a = a_of_x(*xs)
    A = np.zeros((d, d) + tuple(N))
    for i in range(d):
        A[i, i] = a
    return A


def test_smooth_laminate_converges_to_continuous_closed_form():
    """Prop. GaNi (Sec. 4.3): for smooth coefficients the GaNi solution
    converges to the continuous one.  For a(x) = 2 + sin(pi x_1) the cell
    problem is a laminate: continuous A_H = diag(harmonic mean, arithmetic
    mean) = diag(sqrt(3), 2), since (1/2pi) int dt / (2 + sin t) = 1/sqrt(3).
    The error falls geometrically with N (trapezoidal rule on an analytic
    periodic integrand)."""
    errs = []
    for n in (3, 5, 9, 15):
        A = _smooth_field((n, 7), lambda x, y: 2.0 + np.sin(np.pi * x))
        AH = O.solve_AH(A, (n, 7), tol=1e-13)["AH"]
        assert abs(AH[1, 1] - 2.0) < 1e-12 and abs(AH[0, 1]) < 1e-12
        errs.append(abs(AH[0, 0] - np.sqrt(3.0)))
    assert errs[-1] < 1e-8
    assert all(e2 < 0.5 * e1 for e1, e2 in zip(errs, errs[1:]) if e1 > 1e-14)


def test_smooth_2d_medium_grid_refinement_is_cauchy():
    """Prop. GaNi (Sec. 4.3): a smooth, genuinely 2D medium; A_H(N) forms a
    Cauchy sequence as the grid is refined (differences between successive
    odd grids shrink rapidly), stays symmetric and between the Voigt and
    Reuss bounds of the sampled medium."""
    a = lambda x, y: 3.0 + np.sin(np.pi * x) * np.cos(np.pi * y) + 0.5 * np.cos(2 * np.pi * x)
    AHs = []
    for n in (9, 15, 27, 45):
        A = _smooth_field((n, n), a)
        AH = O.solve_AH(A, (n, n), tol=1e-13)["AH"]
        np.testing.assert_allclose(AH, AH.T, atol=1e-12)
        av = A[0, 0]
        assert np.mean(av) - 1e-12 >= AH[0, 0] >= 1.0 / np.mean(1.0 / av) - 1e-12
        AHs.append(AH)
    diffs = [np.max(np.abs(b - a_)) for a_, b in zip(AHs, AHs[1:])]
    assert diffs[-1] < 1e-9
    assert diffs[1] < 0.1 * diffs[0] and diffs[2] < 0.1 * diffs[1]


def _two_phase_field(N, rho, seed):
    """Isotropic two-phase medium 1*I / rho*I on a random voxel set."""
    rng = np.random.default_rng(seed)
    d = len(N)
    a = np.where(rng.random(N) < 0.4, rho, 1.0)
    A = np.zeros((d, d) + tuple(N))
    for i in range(d):
        A[i, i] = a
    return A


def _energy_norm(A, u):
    return math.sqrt(O.inner(O.apply_A(A, u), u))


@pytest.mark.parametrize("rho", [10.0, 100.0])
def test_cg_error_obeys_the_conditioning_bound(rho):
    """Sec. 5.3: on E_N the system is SPD in the energy product (A_N u, v) with
    spectrum in [c_A, C_A], so the CG error contracts as the textbook bound
    ||x_i - x*||_A <= 2 ((sqrt(rho) - 1) / (sqrt(rho) + 1))^i ||x*||_A
    (x_0 = 0); the exact x* from the dense solve of Eq. LSD."""
    N = (9, 7)
    A = _two_phase_field(N, rho, 3)
    E = np.array([1.0, 0.0])
    xstar = O.solve_lsd_dense(A, E, N) - E.reshape(2, 1, 1)
    q = (math.sqrt(rho) - 1.0) / (math.sqrt(rho) + 1.0)
    e0 = _energy_norm(A, xstar)
    for i in range(1, 16):
        x = O.cg(A, E, N, tol=0.0, maxiter=i)["x"]
        err = _energy_norm(A, x - xstar)
        assert err <= 2.0 * q ** i * e0 + 1e-12 * e0, (i, err / e0, 2 * q ** i)


@pytest.mark.parametrize("rho", [10.0, 100.0])
def test_moulinec_suquet_contracts_at_the_optimal_rate(rho):
    """Sec. 5.3: with A0 = lambda I, lambda = (c_A + C_A) / 2, the fixed point
    e_i = E - Gamma_N (A_N - lambda I) e_{i-1} contracts the error in the
    plain norm by at most (rho - 1) / (rho + 1) per step.  On this small
    random medium the observed factor (about 0.82 per step at rho = 100)
    stays below that bound but is of its order: the iteration neither
    diverges nor converges in one step."""
    N = (9, 7)
    A = _two_phase_field(N, rho, 4)
    E = np.array([1.0, 0.0])
    estar = O.solve_lsd_dense(A, E, N)
    lam = 0.5 * (1.0 + rho)
    q = (rho - 1.0) / (rho + 1.0)
    d0 = math.sqrt(O.inner(E.reshape(2, 1, 1) - estar, E.reshape(2, 1, 1) - estar))
    errs = []
    for i in range(1, 13):
        e = O.moulinec_suquet(A, E, N, lam=lam, tol=0.0, maxiter=i)["e"]
        errs.append(math.sqrt(O.inner(e - estar, e - estar)))
        assert errs[-1] <= q ** i * d0 * (1 + 1e-9) + 1e-13, (i, errs[-1] / d0, q ** i)
    assert errs[-1] / errs[-2] > 0.5 * q


@pytest.mark.parametrize("N,Y,perm", [((9, 15), (1.0, 2.5), (1, 0)),
                                      ((5, 9, 7), (1.0, 0.5, 2.0), (2, 0, 1)),
                                      ((5, 9, 7), (1.0, 1.0, 1.0), (1, 2, 0))])
def test_axis_permutation_equivariance(N, Y, perm):
    """Relabelling the axes of the cell (grid, cell sizes Y and tensor
    components together) relabels A_H: A_H' = P A_H P^T.  Exact for GaNi
    (Sec. 4.1 grid, xi_a = m_a / Y_a of Sec. 2); catches an axis mixed up in
    the frequency map, in Y or in the component order."""
    d = len(N)
    A = W.random_spd_field(N, np.random.default_rng(sum(N)), 1.0, 20.0)
    AH = O.solve_AH(A, N, Y=Y, tol=1e-13)["AH"]
    Np = tuple(N[p] for p in perm)
    Yp = tuple(Y[p] for p in perm)
    Ap = np.transpose(A, (0, 1) + tuple(2 + p for p in perm))       # grid axes
    Ap = Ap[np.ix_(perm, perm)]                                       # components
    AHp = O.solve_AH(np.ascontiguousarray(Ap), Np, Y=Yp, tol=1e-13)["AH"]
    np.testing.assert_allclose(AHp, AH[np.ix_(perm, perm)], atol=1e-10 * np.max(np.abs(AH)))


def test_reflection_equivariance_and_scalings():
    """x_a -> -x_a (grid index k -> -k mod N_a) with A -> R A R, R = diag(+-1),
    gives A_H -> R A_H R; c A gives c A_H; a common factor on every Y_a leaves
    A_H unchanged (Gamma_hat depends on xi only through its direction)."""
    N = (9, 7)
    A = W.random_spd_field(N, np.random.default_rng(21), 1.0, 20.0)
    AH = O.solve_AH(A, N, tol=1e-13)["AH"]
    R = np.diag([-1.0, 1.0])
    idx = (-np.arange(9)) % 9
    Ar = A[:, :, idx, :] * np.outer(np.diag(R), np.diag(R))[:, :, None, None]
    AHr = O.solve_AH(np.ascontiguousarray(Ar), N, tol=1e-13)["AH"]
    np.testing.assert_allclose(AHr, R @ AH @ R, atol=1e-10 * np.max(np.abs(AH)))
    np.testing.assert_allclose(O.solve_AH(3.5 * A, N, tol=1e-13)["AH"], 3.5 * AH,
                               atol=1e-10 * np.max(np.abs(AH)))
    np.testing.assert_allclose(O.solve_AH(A, N, Y=(1.7, 1.7), tol=1e-13)["AH"], AH,
                               atol=1e-10 * np.max(np.abs(AH)))
    # an anisotropic cell is not a common factor: A_H changes
    assert np.max(np.abs(O.solve_AH(A, N, Y=(1.0, 3.0), tol=1e-13)["AH"] - AH)) > 1e-4
