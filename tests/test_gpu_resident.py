"""The resident FP32 CG solver (one cooperative launch per inner solve, r and p
kept in shared memory) against the CPU oracle and against the pass kernels.

The method is the CG of Sec. 5.3 on Eq. final_system; the resident kernel only
changes where the iteration's vectors live, so its A_H must meet the same
bounds as the pass kernels' (1e-6 relative for the mixed path) and its
iteration counts must agree with theirs up to rounding of the partial sums.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def ctx(hg):
    c = hg.Context(0)
    yield c
    c.close()


def _phase_problem(n, seed, contrast=100.0):
    ms = W.circles_2d(n=n, count=max(3, n // 20), r_lo=max(1.5, n / 30), r_hi=max(3.0, n / 10),
                      contrast=contrast, seed=seed)
    return ms


@pytest.mark.parametrize("n", [45, 75, 81, 135, 243, 375])
def test_resident_matches_oracle_and_pass_kernels(hg, ctx, n):
    ms = _phase_problem(n, seed=n)
    ref = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    res = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, resident=-1))
    plain = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, resident=0))
    assert res["status"] == 0 and plain["status"] == 0
    assert res["resident_ctas"] > 0 and plain["resident_ctas"] == 0
    assert rel_max(res["AH"], ref["AH"]) < 1e-6
    assert rel_max(res["AH"], plain["AH"]) < 1e-6
    # same iterates up to the rounding of the partial sums
    for a, b in zip(res["iters"], plain["iters"]):
        assert abs(a - b) <= max(3, 0.05 * b)
    assert max(res["rel_res"]) <= 1e-9
    # e~ against the oracle's
    for j in range(2):
        e = g.field(j)
        err = np.sqrt(O.inner(e - ref["x"][j], e - ref["x"][j]))
        assert err <= 1e-6 * max(1.0, np.sqrt(O.inner(ref["x"][j], ref["x"][j])))
    g.close()


def test_resident_full_size_729_against_golden(hg, ctx):
    """The 729x729 workload at bench.py's settings (tol 1e-5) and tight."""
    gold = json.load(open(os.path.join(HERE, "golden", "circles_729_AH.json")))
    ref = np.array(gold["AH"])
    ms = W.circles_2d()
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    res = g.solve(hg.default_opts(tol=1e-5, prec=hg.HG_MIXED, inner_tol=5e-6))
    assert res["status"] == 0 and res["resident_ctas"] > 0
    assert rel_max(res["AH"], ref) < 1e-6
    tight = g.solve(hg.default_opts(tol=1e-10, prec=hg.HG_MIXED))
    assert tight["status"] == 0 and tight["resident_ctas"] > 0
    assert rel_max(tight["AH"], ref) < 1e-8
    g.close()


@pytest.mark.parametrize("n,T", [(45, 1), (81, 2), (81, 7), (81, 40), (81, 10000)])
def test_resident_team_sizes_give_the_same_solution(hg, ctx, n, T):
    """Any team size (one CTA, uneven splits of rows and columns, more CTAs
    than the device has SMs requested) solves the same system."""
    ms = _phase_problem(n, seed=3)
    ref = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)["AH"]
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    res = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, resident=T))
    assert res["status"] == 0
    # at most one CTA per SM, per grid row of a load and per column of the half spectrum
    assert 1 <= res["resident_ctas"] <= min(T, 2 * n, 2 * ((n + 1) // 2))
    assert rel_max(res["AH"], ref) < 1e-6
    g.close()


def test_resident_falls_back_when_the_state_does_not_fit(hg, ctx):
    """A team too small to hold r and p in shared memory (one CTA for 81^2)
    runs the pass kernels instead, with the same result."""
    ms = _phase_problem(81, seed=3)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    res = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, resident=1))
    plain = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, resident=0))
    assert res["status"] == 0 and res["resident_ctas"] == 0
    np.testing.assert_array_equal(res["AH"], plain["AH"])
    g.close()


def test_resident_packed_field_anisotropic_cell(hg, ctx):
    """Random SPD field (packed coefficients, read from global memory) on an
    anisotropic cell Y = (1, 2.5)."""
    N, Y = (45, 45), (1.0, 2.5)
    rng = np.random.default_rng(9)
    A = W.random_spd_field(N, rng, 1.0, 50.0)
    ref = O.solve_AH(A, N, Y, tol=1e-12)["AH"]
    g = ctx.grid(N, Y)
    g.set_coeffs_field(A)
    res = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED))
    assert res["status"] == 0 and res["resident_ctas"] > 0
    assert rel_max(res["AH"], ref) < 1e-6
    g.close()


def test_resident_dual_ms_and_reference_medium(hg, ctx):
    """The variants the resident kernel carries: the dual formulation (J_N
    projection, A^-1), Moulinec-Suquet (fixed step 1/lambda) and a general
    reference medium A0 (Gamma_hat(A0), (A0 r, r))."""
    ms = _phase_problem(75, seed=12, contrast=30.0)
    A = ms.full_field()
    N = ms.N
    g = ctx.grid(N)
    g.set_coeffs_phase(ms.phase, ms.table)
    dual = O.solve_AH_dual(A, N, tol=1e-12)
    r = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, formulation=hg.HG_DUAL))
    assert r["status"] == 0 and r["resident_ctas"] > 0
    assert rel_max(r["CH"], dual["CH"]) < 1e-6
    primal = O.solve_AH(A, N, tol=1e-12)["AH"]
    r = g.solve(hg.default_opts(tol=1e-8, prec=hg.HG_MIXED, method=hg.HG_MS, max_iter=5000))
    assert r["status"] == 0 and r["resident_ctas"] > 0
    assert rel_max(r["AH"], primal) < 1e-6
    A0 = np.array([[2.0, 0.5], [0.5, 1.0]])
    r = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, A0=A0))
    assert r["status"] == 0 and r["resident_ctas"] > 0
    assert rel_max(r["AH"], primal) < 1e-6
    g.close()


def test_resident_zero_rhs_and_single_load(hg, ctx):
    """A homogeneous medium (b = 0: no iteration) and a solve of one load only."""
    N = (81, 81)
    g = ctx.grid(N)
    g.set_coeffs_phase(np.zeros(N, np.uint8), W.isotropic_table([3.0], 2))
    r = g.solve(hg.default_opts(prec=hg.HG_MIXED))
    assert r["status"] == 0
    np.testing.assert_allclose(r["AH"], 3.0 * np.eye(2), atol=1e-12)
    ms = _phase_problem(81, seed=21)
    ref = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)["AH"]
    g.set_coeffs_phase(ms.phase, ms.table)
    r = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, loads_mask=2))
    assert r["status"] == 0 and r["resident_ctas"] > 0
    assert abs(r["AH"][1, 1] - ref[1, 1]) < 1e-6 * abs(ref[1, 1])
    g.close()


def test_resident_bounded_wait_reports_timeout_and_context_survives(hg, ctx):
    """One CTA of the resident launch leaves at once: the others' barrier
    waits run out (0.1 s), the solve returns HG_ERR_DEVICE_TIMEOUT, and the
    same grid then solves normally."""
    ms = _phase_problem(81, seed=5)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    st = g.test_resident_timeout(1, hg.default_opts(tol=1e-8, prec=hg.HG_MIXED))
    assert st == hg.HG_ERR_DEVICE_TIMEOUT
    r = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED))
    assert r["status"] == 0 and r["resident_ctas"] > 0
    ref = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)["AH"]
    assert rel_max(r["AH"], ref) < 1e-6
    g.close()


def test_resident_time_pass_times_the_launch(hg, ctx):
    ms = _phase_problem(243, seed=8)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    r = g.solve(hg.default_opts(tol=1e-6, prec=hg.HG_MIXED, time_pass=0))
    assert r["status"] == 0 and r["resident_ctas"] > 0
    assert r["pass_launches"] >= 1 and r["pass_ms_total"] > 0.0
    g.close()


@pytest.mark.parametrize("N,prec", [((15, 15), 0), ((45, 75), 0), ((15, 15), 1), ((45, 75), 1), ((81, 81), 1)])
def test_true_residual_matches_oracle(hg, ctx, N, prec):
    """hg_result.true_rel_res = ||b - G A x|| / ||b|| recomputed in FP64 at exit
    (the stopping rule of Sec. 5.3 is the paper's open point): it equals the
    oracle's recomputation of that residual from the returned e~ (hg_get_field),
    and for the FP64 path with the oracle's own iteration count also the
    oracle's true residual of its own iterate."""
    rng = np.random.default_rng(N[0] * 7 + prec)
    ph = (rng.random(N) < 0.3).astype(np.uint8)
    table = W.isotropic_table([1.0, 20.0], 2)
    ms = W.Microstructure(N, ph, table)
    A = ms.full_field()
    tol = 1e-7
    ref = O.solve_AH(A, N, tol=tol)
    g = ctx.grid(N)
    g.set_coeffs_phase(ph, table)
    r = g.solve(hg.default_opts(tol=tol, prec=prec))
    assert r["status"] == 0
    for j in range(2):
        E = np.zeros((2,) + (1,) * 2)
        E[j] = 1.0
        b = -O.apply_K(A, E * np.ones((2,) + N), N)
        x = g.field(j)
        res = b - O.apply_K(A, x, N)
        want = np.sqrt(O.inner(res, res) / O.inner(b, b))
        got = r["true_rel_res"][j]
        assert 0.0 < got <= 2 * tol
        assert abs(got - want) <= 1e-10 + 1e-3 * want
        if prec == 0 and r["iters"][j] == ref["iters"][j]:
            # the same FP64 iterate up to rounding: the oracle's own residual
            assert abs(got - ref["true_rel_res"][j]) <= 1e-3 * ref["true_rel_res"][j]
            # and the FP64 recursion has not drifted from it
            assert abs(got - r["rel_res"][j]) <= 1e-3 * r["rel_res"][j]
    g.close()
