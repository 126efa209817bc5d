"""Pins of the oracle's Galerkin scheme with exact integration (Sec. 4.2, Ga)
for coefficients constant on pixels.

The CG solve on the quadrature grid with the band-limited projection is
checked against a dense Galerkin solve assembled directly in Fourier space from
the pixels' exact Fourier coefficients; the result is checked to be
independent of the quadrature grid once M >= 2N - 1; closed forms for
homogeneous media and laminates; and the bounds: Ga minimises the energy over
a subspace of the continuous problem's fields, so its A_H decreases on nested
trial spaces and stays above the dual's, which increases.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def two_phase(P, seed, contrast=10.0):
    rng = np.random.default_rng(seed)
    d = len(P)
    ph = (rng.random(P) < 0.4).astype(np.uint8)
    return W.Microstructure(P, ph, W.isotropic_table([1.0, contrast], d)).full_field()


@pytest.mark.parametrize("P,N", [((3, 3), (3, 3)), ((5, 5), (3, 3)), ((5, 5), (5, 5)), ((3, 3, 3), (3, 3, 3))])
def test_ga_cg_matches_dense_fourier_galerkin(P, N):
    A = two_phase(P, 3)
    ga = O.solve_AH_ga(A, N, tol=1e-14)
    dense = O.solve_ga_dense(A, N)
    np.testing.assert_allclose(ga["AH"], dense, rtol=1e-11, atol=1e-12)


def test_ga_sinc_coefficients_of_a_single_pixel():
    # one pixel of value 1 at the origin on P: A_hat(l) = prod sinc(l / P) / |P|
    P = (5, 7)
    A = np.zeros((1, 1) + P)
    A[0, 0, 0, 0] = 1.0
    c = O.pixel_fourier_coeffs(A, (3, 4))[0, 0]
    l0 = np.arange(-2, 3)[:, None]
    l1 = np.arange(-3, 4)[None, :]
    expect = np.sinc(l0 / 5.0) * np.sinc(l1 / 7.0) / 35.0
    np.testing.assert_allclose(c, expect, atol=1e-15)


def test_ga_independent_of_quadrature_grid_beyond_2N_minus_1():
    A = two_phase((5, 5), 8)
    N = (5, 5)
    a = O.solve_AH_ga(A, N, M=(9, 9), tol=1e-13)
    b = O.solve_AH_ga(A, N, M=(15, 11), tol=1e-13)
    np.testing.assert_allclose(a["AH"], b["AH"], rtol=1e-11)
    # one point short of 2N - 1 aliases the product into the trial band
    c = O.solve_AH_ga(A, N, M=(7, 7), tol=1e-13)
    assert np.max(np.abs(c["AH"] - a["AH"])) > 1e-6


def test_ga_homogeneous_and_laminate_closed_forms():
    P = (7, 5)
    A0 = np.array([[3.0, 1.0], [1.0, 2.0]])
    H = np.broadcast_to(A0[:, :, None, None], (2, 2) + P).copy()
    for dual in (False, True):
        r = O.solve_AH_ga(H, (5, 5), dual=dual)
        assert r["iters"] == [0, 0]
        np.testing.assert_allclose(r["AH"], A0, atol=1e-13)
    rng = np.random.default_rng(2)
    a = np.exp(rng.uniform(0, np.log(50.0), size=P[0]))
    L = np.einsum("ab,...->ab...", np.eye(2), np.broadcast_to(a[:, None], P))
    harm, arith = 1.0 / np.mean(1.0 / a), np.mean(a)
    up = O.solve_AH_ga(L, (7, 5), tol=1e-13)
    lo = O.solve_AH_ga(L, (7, 5), tol=1e-13, dual=True)
    # along the layers the primal field is E itself; across, the dual flux is S itself
    assert up["iters"][1] == 0 and abs(up["AH"][1, 1] - arith) < 1e-12 * arith
    assert lo["iters"][0] == 0 and abs(lo["AH"][0, 0] - harm) < 1e-12 * harm
    assert up["AH"][0, 0] >= harm * (1 - 1e-12)
    assert lo["AH"][1, 1] <= arith * (1 + 1e-12)


def test_ga_bounds_and_monotonicity_on_nested_trial_spaces():
    A = two_phase((5, 5), 3)
    up5 = O.solve_AH_ga(A, (5, 5), tol=1e-13)["AH"]
    up15 = O.solve_AH_ga(A, (15, 15), tol=1e-12)["AH"]
    lo5 = O.solve_AH_ga(A, (5, 5), tol=1e-13, dual=True)["AH"]
    lo15 = O.solve_AH_ga(A, (15, 15), tol=1e-12, dual=True)["AH"]
    for big, small in ((up5, up15), (up15, lo15), (lo15, lo5)):
        assert np.min(np.linalg.eigvalsh(big - small)) > -1e-9
    # strictly: the refinement tightens both bounds
    assert np.trace(up5 - up15) > 1e-3 and np.trace(lo15 - lo5) > 1e-3
