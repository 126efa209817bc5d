"""Pins of the oracle's dual (flux) formulation on J_N.

The projection onto J_N is checked on analytic divergence-free fields and
gradients (Eq. Helmholtz_discrete), the CG dual solve against a dense LU solve
assembled from the DFT matrices, and the dual homogenized matrix against the
primal one, which it equals exactly for GaNi: the primal e = E + e~ has
A e in U_N (+) J_N (Galerkin orthogonality), so s = A e solves the dual
problem and A^-1 s = e lies in U_N (+) E_N.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

RNG = np.random.default_rng(1789)


def trig_gradient(N, m, Y=None, phase=0.3):
    """Grid values of grad f, f(x) = cos(pi xi(m).x + phase), on x_k = k h."""
    d = len(N)
    Y = [1.0] * d if Y is None else Y
    ks = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in N], indexing="ij")
    arg = sum(2 * np.pi * m[a] * ks[a] / N[a] for a in range(d)) + phase
    return np.stack([-np.pi * m[a] / Y[a] * np.sin(arg) for a in range(d)])


def divergence_free(N, m, Y=None):
    """A zero-mean divergence-free trigonometric field: in 2D the rotated
    gradient, in 3D (xi x c) times a scalar wave."""
    g = trig_gradient(N, m, Y)
    d = len(N)
    if d == 2:
        return np.stack([g[1], -g[0]])
    Yv = [1.0] * d if Y is None else Y
    xi = np.array([m[a] / Yv[a] for a in range(d)])
    w = np.cross(xi, np.array([0.3, -1.1, 0.7]))
    s = g[0] / (-np.pi * xi[0])
    return np.stack([w[a] * s for a in range(d)])


@pytest.mark.parametrize("N,m,Y", [((7, 5), (2, -1), None), ((9, 7), (-3, 3), (1.0, 2.5)),
                                   ((5, 5, 7), (1, -2, 3), (1.0, 0.5, 2.0))])
def test_gamma_J_keeps_divergence_free_and_kills_gradients(N, m, Y):
    v = divergence_free(N, m, Y)
    np.testing.assert_allclose(O.apply_gamma_J(v, N, Y), v, atol=1e-12)
    g = trig_gradient(N, m, Y)
    np.testing.assert_allclose(O.apply_gamma_J(g, N, Y), 0.0, atol=1e-12)
    c = np.ones((len(N),) + N) * 2.5
    np.testing.assert_allclose(O.apply_gamma_J(c, N, Y), 0.0, atol=1e-12)


@pytest.mark.parametrize("N", [(5, 7), (3, 5, 7)])
def test_gamma_J_is_an_orthogonal_projection(N):
    d = len(N)
    u = RNG.standard_normal((d,) + N)
    w = RNG.standard_normal((d,) + N)
    Pu = O.apply_gamma_J(u, N)
    np.testing.assert_allclose(O.apply_gamma_J(Pu, N), Pu, atol=1e-12)
    assert abs(O.inner(Pu, w) - O.inner(u, O.apply_gamma_J(w, N))) < 1e-12
    # orthogonal to E_N
    assert abs(O.inner(Pu, O.apply_gamma(w, N))) < 1e-12


@pytest.mark.parametrize("N,kind", [((3, 3), "phase"), ((5, 3), "spd"), ((3, 3, 3), "spd"),
                                    ((3, 5, 3), "phase")])
def test_cg_dual_matches_dense_solve(N, kind):
    rng = np.random.default_rng(17)
    d = len(N)
    if kind == "phase":
        ph = (rng.random(N) < 0.4).astype(np.uint8)
        A = W.Microstructure(N, ph, W.isotropic_table([1.0, 25.0], d)).full_field()
    else:
        A = W.random_spd_field(N, rng, 1.0, 30.0)
    for j in range(d):
        S = np.zeros(d)
        S[j] = 1.0
        sol = O.cg_dual(A, S, N, tol=1e-13, maxiter=500)
        x_lu = O.solve_dual_dense(A, S, N)
        err = np.sqrt(O.inner(sol["x"] - x_lu, sol["x"] - x_lu))
        ref = np.sqrt(O.inner(x_lu, x_lu)) + 1e-300
        assert err / ref < 1e-10, err / ref


@pytest.mark.parametrize("N,seed", [((15, 15), 1), ((9, 11), 2), ((7, 5, 9), 3)])
def test_dual_A_H_equals_primal(N, seed):
    rng = np.random.default_rng(seed)
    A = W.random_spd_field(N, rng, 1.0, 200.0)
    p = O.solve_AH(A, N, tol=1e-13)
    q = O.solve_AH_dual(A, N, tol=1e-13)
    np.testing.assert_allclose(q["AH"], p["AH"], rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(q["AH_flux"], p["AH"], rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(q["CH"], q["CH"].T, atol=1e-13)


def test_dual_laminate_and_homogeneous_exact():
    N = (9, 7)
    rng = np.random.default_rng(4)
    a = np.exp(rng.uniform(0, np.log(100.0), size=N[0]))
    af = np.broadcast_to(a[:, None], N)
    A = np.einsum("ab,...->ab...", np.eye(2), af)
    q = O.solve_AH_dual(A, N, tol=1e-14)
    expect = np.diag([1.0 / np.mean(1.0 / a), np.mean(a)])
    np.testing.assert_allclose(q["AH"], expect, rtol=1e-11, atol=1e-12)
    # the flux across the layers is constant already: that load takes no step
    assert q["iters"][0] == 0
    A0 = np.array([[3.0, 1.0], [1.0, 2.0]])
    H = np.broadcast_to(A0[:, :, None, None], (2, 2) + N).copy()
    h = O.solve_AH_dual(H, N)
    assert h["iters"] == [0, 0]
    np.testing.assert_allclose(h["AH"], A0, atol=1e-13)
