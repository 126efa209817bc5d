"""Moulinec-Suquet fixed point on the GPU (Sec. 5.3 comments) against the oracle.

The CUDA path runs the fixed point as the CG kernels with the step fixed to
1 / lambda and beta = 0; the oracle runs the Neumann-series recursion
e_i = E - Gamma_N (A_N - lambda I) e_{i-1} as the paper writes it.  Both stop on
||e_i - e_{i-1}|| / ||E|| <= tol, so iteration counts agree exactly.
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


def eig_bounds(A):
    """(c_A, C_A) of a (d, d, *N) field: extreme eigenvalues over the voxels."""
    d = A.shape[0]
    m = np.moveaxis(A.reshape(d, d, -1), 2, 0)
    ev = np.linalg.eigvalsh(m)
    return float(ev.min()), float(ev.max())


def ms_opts(hg, **kw):
    kw.setdefault("method", hg.HG_MS)
    return hg.default_opts(**kw)


@pytest.mark.parametrize("case", ["square15", "spd_field_27x15", "two_phase_3d"])
def test_ms_fp64_matches_oracle_iterates(hg, ctx, case):
    rng = np.random.default_rng(11)
    if case == "square15":
        ms = W.square_inclusion_15()
        N, A = ms.N, ms.full_field()
    elif case == "spd_field_27x15":
        N = (27, 15)
        A = W.random_spd_field(N, rng, 1.0, 20.0)
    else:
        N = (15, 9, 15)
        phase = (rng.random(N) < 0.3).astype(np.uint8)
        tab = np.stack([np.eye(3), W.random_spd_pair(3, rng, 1.0, 30.0)[1]])
        A = W.Microstructure(N, phase, tab).full_field()
    d = len(N)
    c, C = eig_bounds(A)
    lam = 0.5 * (c + C)
    g = ctx.grid(N)
    g.set_coeffs_field(A)
    tol = 1e-11
    r = g.solve(ms_opts(hg, tol=tol, lambda_ref=lam, max_iter=20000))
    assert r["status"] == 0
    assert r["lambda_ref"] == lam
    for l in range(d):
        E = np.eye(d)[l]
        ref = O.moulinec_suquet(A, E, N, lam=lam, tol=tol)
        x_ref = ref["e"] - E.reshape((d,) + (1,) * d)
        assert r["iters"][l] == ref["iters"], (l, r["iters"], ref["iters"])
        x = g.field(l)
        assert np.max(np.abs(x - x_ref)) <= 1e-10 * max(1.0, np.max(np.abs(x_ref)))
    # the fixed point is the GaNi solution: A_H agrees with the oracle's CG
    AH_cg = O.solve_AH(A, N, tol=1e-13)["AH"]
    assert np.max(np.abs(r["AH"] - AH_cg)) <= 1e-9 * np.max(np.abs(AH_cg))
    g.close()


def test_ms_default_lambda_is_the_optimal_reference(hg, ctx):
    rng = np.random.default_rng(3)
    N = (15, 27)
    A = W.random_spd_field(N, rng, 2.0, 50.0)
    c, C = eig_bounds(A)
    g = ctx.grid(N)
    g.set_coeffs_field(A)
    r = g.solve(ms_opts(hg, tol=1e-9, max_iter=20000))
    assert abs(r["c_A"] - c) <= 1e-12 * C
    assert abs(r["C_A"] - C) <= 1e-12 * C
    assert abs(r["lambda_ref"] - 0.5 * (c + C)) <= 1e-12 * C
    # new coefficients: bounds recomputed
    g.set_coeffs_field(2.0 * A)
    r2 = g.solve(ms_opts(hg, tol=1e-9, max_iter=20000))
    assert abs(r2["C_A"] - 2.0 * C) <= 1e-12 * C
    assert np.max(np.abs(r2["AH"] - 2.0 * r["AH"])) <= 1e-7 * np.max(np.abs(r2["AH"]))
    # phase-map coefficients: bounds over the phases present
    ms = W.square_inclusion_15()
    tab = np.concatenate([ms.table, 1e3 * np.eye(2)[None]])      # phase 2 unused
    g2 = ctx.grid(ms.N)
    g2.set_coeffs_phase(ms.phase, tab)
    r3 = g2.solve(ms_opts(hg, tol=1e-9))
    assert (r3["c_A"], r3["C_A"], r3["lambda_ref"]) == (1.0, 10.0, 5.5)
    g.close()
    g2.close()


def test_ms_lambda_below_half_the_upper_bound_is_rejected(hg, ctx):
    ms = W.square_inclusion_15()
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    r = g.solve(ms_opts(hg, lambda_ref=4.9), raise_on_error=False)     # C_A / 2 = 5
    assert r["status"] == -1
    r = g.solve(ms_opts(hg, lambda_ref=7.0, tol=1e-10))                # converges, slower
    r_opt = g.solve(ms_opts(hg, tol=1e-10))
    assert r["iters"][0] > r_opt["iters"][0]
    assert np.max(np.abs(r["AH"] - r_opt["AH"])) <= 1e-8 * np.max(np.abs(r_opt["AH"]))
    bad = hg.default_opts(method=7)
    assert g.solve(bad, raise_on_error=False)["status"] == -1
    g.close()


def test_ms_iterations_grow_like_contrast_cg_like_its_root(hg, ctx):
    """Sec. 5.3 comments: MS iterations ~ rho_A, CG iterations ~ sqrt(rho_A) at most."""
    base = W.circles_2d(n=45, count=8, r_lo=3, r_hi=7, contrast=10.0, seed=9)
    g = ctx.grid(base.N)
    rhos = [10.0, 100.0, 1000.0]
    its_ms, its_cg = [], []
    for rho in rhos:
        g.set_coeffs_phase(base.phase, W.isotropic_table([1.0, rho], 2))
        its_ms.append(g.solve(ms_opts(hg, tol=1e-6, max_iter=50000))["iters"][0])
        its_cg.append(g.solve(hg.default_opts(tol=1e-6))["iters"][0])
    slope_ms = np.polyfit(np.log(rhos), np.log(its_ms), 1)[0]
    slope_cg = np.polyfit(np.log(rhos), np.log(its_cg), 1)[0]
    assert 0.8 < slope_ms < 1.2, its_ms
    assert slope_cg < 0.6, its_cg
    # the contraction (rho - 1) / (rho + 1) bounds the MS count from above
    for rho, n in zip(rhos, its_ms):
        q = (rho - 1.0) / (rho + 1.0)
        assert n <= np.log(1e-6 / 10.0) / np.log(q) + 10
    g.close()


def test_ms_mixed_precision_reaches_the_fp64_A_H(hg, ctx):
    ms = W.circles_2d(n=135, count=12, r_lo=5, r_hi=15, contrast=100.0, seed=21)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    ref = g.solve(hg.default_opts(tol=1e-11))
    r = g.solve(ms_opts(hg, prec=hg.HG_MIXED, tol=1e-8, max_iter=100000))
    assert r["status"] == 0
    assert max(r["outer"]) >= 1
    err = np.max(np.abs(r["AH"] - ref["AH"])) / np.max(np.abs(ref["AH"]))
    assert err <= 1e-6, err
    r64 = g.solve(ms_opts(hg, tol=1e-8, max_iter=100000))
    assert np.max(np.abs(r64["AH"] - ref["AH"])) / np.max(np.abs(ref["AH"])) <= 1e-6
    g.close()


def test_ms_through_the_scheduler_matches_blocking(hg, ctx):
    ms = W.square_inclusion_15()
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    blocking = g.solve(ms_opts(hg, tol=1e-10))
    t = ctx.submit(g, ms_opts(hg, tol=1e-10))
    res = None
    while res is None:
        res = ctx.poll(t, 100000)
    assert res["iters"] == blocking["iters"]
    np.testing.assert_array_equal(res["AH"], blocking["AH"])
    assert res["lambda_ref"] == 5.5
    g.close()


def test_ms_homogeneous_medium_needs_no_iteration(hg, ctx):
    N = (15, 9)
    A0 = np.array([[3.0, 1.0], [1.0, 2.0]])
    g = ctx.grid(N)
    g.set_coeffs_phase(np.zeros(N, np.uint8), A0[None])
    r = g.solve(ms_opts(hg))
    assert r["iters"] == [0, 0]
    assert np.max(np.abs(r["AH"] - A0)) <= 1e-14 * 3.0
    g.close()
