"""Pins of the oracle's CG with a general reference medium A0.

Checked against the dense LU solve of Eq. LSD with the same A0 (assembled from
the DFT matrices), against the A0 = I solution (the GaNi solution does not
depend on A0), and, for A0 = lam I, against the iterates of the plain CG.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.mark.parametrize("N,kind", [((5, 3), "spd"), ((5, 5), "phase"), ((3, 3, 3), "spd")])
def test_cg_ref_matches_dense_lsd_with_the_same_A0(N, kind):
    rng = np.random.default_rng(31)
    d = len(N)
    if kind == "phase":
        ph = (rng.random(N) < 0.4).astype(np.uint8)
        A = W.Microstructure(N, ph, W.isotropic_table([1.0, 25.0], d)).full_field()
    else:
        A = W.random_spd_field(N, rng, 1.0, 30.0)
    A0 = W.random_spd_field((1,) * d, rng, 0.5, 8.0).reshape(d, d)
    for j in range(d):
        E = np.zeros(d)
        E[j] = 1.0
        sol = O.cg_ref(A, E, N, A0, tol=1e-13, maxiter=500)
        e = O.solve_lsd_dense(A, E, N, A0=A0)
        x_lu = e - E.reshape((d,) + (1,) * d)
        err = np.sqrt(O.inner(sol["x"] - x_lu, sol["x"] - x_lu))
        assert err / (np.sqrt(O.inner(x_lu, x_lu)) + 1e-300) < 1e-10
        # and the GaNi solution itself does not depend on A0
        plain = O.cg(A, E, N, tol=1e-13, maxiter=500)
        err2 = np.sqrt(O.inner(sol["x"] - plain["x"], sol["x"] - plain["x"]))
        assert err2 / (np.sqrt(O.inner(x_lu, x_lu)) + 1e-300) < 1e-10


def test_scalar_reference_medium_reproduces_plain_cg_iterates():
    ms = W.circles_2d(n=45, count=5, r_lo=3, r_hi=8, contrast=30.0, seed=3)
    A = ms.full_field()
    E = np.array([1.0, 0.0])
    a = O.cg(A, E, ms.N, tol=1e-9)
    b = O.cg_ref(A, E, ms.N, 4.0 * np.eye(2), tol=1e-9)
    assert a["iters"] == b["iters"]
    np.testing.assert_allclose(b["x"], a["x"], atol=1e-12)


def test_reference_medium_A_H_and_anisotropic_speedup():
    # strongly anisotropic laminate-like medium: a reference medium with the
    # same anisotropy conditions the A0-weighted system better than I
    rng = np.random.default_rng(8)
    N = (27, 27)
    ph = (rng.random(N) < 0.35).astype(np.uint8)
    tab = np.array([[[1.0, 0.0], [0.0, 50.0]], [[20.0, 0.0], [0.0, 1000.0]]])
    A = W.Microstructure(N, ph, tab).full_field()
    plain = O.solve_AH(A, N, tol=1e-10)
    A0 = np.diag([5.0, 250.0])
    ref = O.solve_AH_ref(A, N, A0, tol=1e-10)
    np.testing.assert_allclose(ref["AH"], plain["AH"], rtol=1e-8)
    assert sum(ref["iters"]) < sum(plain["iters"])
