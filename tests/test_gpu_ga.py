"""Galerkin scheme with exact integration (Sec. 4.2, Ga) on the GPU against the
oracle's `solve_AH_ga`.

The grid of the solve is the quadrature grid M >= 2N - 1; the coefficients are
the pixels' Fourier series truncated to the band the energy of two trial fields
reaches, and the projection is limited to the trial space Z_N.  The primal gives
the upper bound, the dual (coefficients (A^-1)_M, fluxes on the band-limited
J_N) the lower bound.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hg):
    c = hg.Context(0)
    yield c
    c.close()


def pixels(P, seed, contrast=10.0, n_phases=2):
    rng = np.random.default_rng(seed)
    d = len(P)
    ph = rng.integers(0, n_phases, size=P).astype(np.uint8)
    vals = np.exp(np.linspace(0.0, np.log(contrast), n_phases))
    return ph, W.isotropic_table(list(vals), d)


def oracle_ga(ph, table, N, M, dual, tol=1e-12):
    A = W.Microstructure(ph.shape, ph, table).full_field()
    return O.solve_AH_ga(A, N, M=M, tol=tol, dual=dual)


def gpu_ga(hg, ctx, ph, table, N, M, dual, **kw):
    g = ctx.grid(M)
    try:
        g.set_coeffs_exact(N, ph, table)
        o = hg.default_opts(formulation=hg.HG_DUAL if dual else hg.HG_PRIMAL, **kw)
        return g.solve(o)
    finally:
        g.close()


def close(a, b, rel):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) <= rel * np.max(np.abs(b))


@pytest.mark.parametrize("dual", [False, True])
@pytest.mark.parametrize("P,N,M", [
    ((5, 5), (5, 5), (9, 9)),
    ((7, 5), (5, 3), (15, 5)),
    ((15, 15), (15, 15), (35, 35)),
    ((45, 27), (9, 5), (25, 9)),
    ((3, 3, 3), (3, 3, 3), (5, 5, 5)),
    ((5, 5, 5), (5, 5, 5), (9, 9, 9)),
])
def test_ga_fp64_matches_oracle(hg, ctx, P, N, M, dual):
    ph, table = pixels(P, 11, contrast=20.0)
    ref = oracle_ga(ph, table, N, M, dual)
    r = gpu_ga(hg, ctx, ph, table, N, M, dual, tol=1e-12)
    assert r["status"] == 0
    assert close(r["AH"], ref["AH"], 1e-9)
    assert abs(r["iters"][0] - ref["iters"][0]) <= max(2, ref["iters"][0] // 10)


@pytest.mark.parametrize("dual", [False, True])
def test_ga_mixed_precision_matches_oracle(hg, ctx, dual):
    ph, table = pixels((27, 27), 4, contrast=100.0, n_phases=3)
    N, M = (15, 15), (35, 35)
    ref = oracle_ga(ph, table, N, M, dual)
    r = gpu_ga(hg, ctx, ph, table, N, M, dual, tol=1e-9, prec=hg.HG_MIXED)
    assert r["status"] == 0
    assert close(r["AH"], ref["AH"], 1e-7)


def test_ga_result_independent_of_quadrature_grid(hg, ctx):
    ph, table = pixels((5, 5), 8)
    a = gpu_ga(hg, ctx, ph, table, (5, 5), (9, 9), False, tol=1e-12)["AH"]
    b = gpu_ga(hg, ctx, ph, table, (5, 5), (15, 21), False, tol=1e-12)["AH"]
    assert close(b, a, 1e-10)


def test_ga_bounds_bracket_and_tighten(hg, ctx):
    ph, table = pixels((15, 15), 3, contrast=50.0)
    up5 = gpu_ga(hg, ctx, ph, table, (5, 5), (9, 9), False, tol=1e-12)["AH"]
    up15 = gpu_ga(hg, ctx, ph, table, (15, 15), (35, 35), False, tol=1e-12)["AH"]
    lo15 = gpu_ga(hg, ctx, ph, table, (15, 15), (35, 35), True, tol=1e-12)["AH"]
    lo5 = gpu_ga(hg, ctx, ph, table, (5, 5), (9, 9), True, tol=1e-12)["AH"]
    for big, small in ((up5, up15), (up15, lo15), (lo15, lo5)):
        assert np.min(np.linalg.eigvalsh(big - small)) > -1e-9
    assert np.trace(up5 - up15) > 1e-3 and np.trace(lo15 - lo5) > 1e-3


def test_ga_homogeneous_and_laminate(hg, ctx):
    A0 = np.array([[3.0, 1.0], [1.0, 2.0]])
    for dual in (False, True):
        r = gpu_ga(hg, ctx, np.zeros((7, 5), np.uint8), A0[None], (5, 5), (9, 9), dual, tol=1e-12)
        assert r["iters"] == [0, 0]
        np.testing.assert_allclose(r["AH"], A0, atol=1e-13)
    # layers across axis 0: the primal's second load and the dual's first need no iteration
    rng = np.random.default_rng(2)
    ph = np.broadcast_to(rng.integers(0, 4, size=7)[:, None], (7, 5)).astype(np.uint8).copy()
    table = W.isotropic_table(list(np.exp(rng.uniform(0, np.log(50.0), size=4))), 2)
    a = table[ph[:, 0], 0, 0]
    harm, arith = 1.0 / np.mean(1.0 / a), np.mean(a)
    up = gpu_ga(hg, ctx, ph, table, (7, 5), (15, 9), False, tol=1e-12)
    lo = gpu_ga(hg, ctx, ph, table, (7, 5), (15, 9), True, tol=1e-12)
    assert up["iters"][1] == 0 and abs(up["AH"][1, 1] - arith) < 1e-11 * arith
    assert lo["iters"][0] == 0 and abs(lo["AH"][0, 0] - harm) < 1e-11 * harm


def test_ga_grid_reset_by_other_coefficients(hg, ctx):
    # after set_coeffs_phase the same grid solves GaNi again (no band, no A_M)
    ph, table = pixels((9, 9), 5)
    g = ctx.grid((9, 9))
    g.set_coeffs_exact((5, 5), pixels((5, 5), 1)[0], table)
    g.set_coeffs_phase(ph, table)
    r = g.solve(hg.default_opts(tol=1e-12))
    A = W.Microstructure((9, 9), ph, table).full_field()
    assert close(r["AH"], O.solve_AH(A, (9, 9), tol=1e-12)["AH"], 1e-9)
    g.close()


def test_ga_argument_errors(hg, ctx):
    ph, table = pixels((5, 5), 1)
    g = ctx.grid((9, 9))
    for N in [(7, 5), (4, 5), (0, 5)]:          # M < 2N - 1, even N, empty
        with pytest.raises(hg.HGError) as e:
            g.set_coeffs_exact(N, ph, table)
        assert e.value.status == hg.HG_ERR_ARG
    with pytest.raises(hg.HGError) as e:
        g.set_coeffs_exact((5, 5), np.full((5, 5), 2, np.uint8), table)
    assert e.value.status == hg.HG_ERR_ARG
    bad = table.copy()
    bad[1] = -bad[1]
    with pytest.raises(hg.HGError) as e:
        g.set_coeffs_exact((5, 5), ph, bad)
    assert e.value.status == hg.HG_ERR_NOT_SPD
    g.set_coeffs_exact((5, 5), ph, table)
    assert g.solve(hg.default_opts(method=hg.HG_MS), raise_on_error=False)["status"] == hg.HG_ERR_ARG
    assert g.solve(hg.default_opts(A0=2.0 * np.eye(2)), raise_on_error=False)["status"] == hg.HG_ERR_ARG
    g.close()
