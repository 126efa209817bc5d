"""Dual (flux) formulation on the GPU against the oracle's dual and the primal.

The CUDA path solves G_J A^-1 s~ = -G_J A^-1 S with the CG kernels, the
inverse coefficients and the projection onto J_N in the projection pass; the
oracle runs the same CG steps with its FFT projection (pinned against the
dense solve and analytic fields).  For GaNi the dual homogenized matrix
equals the primal one exactly.
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


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("case", ["square15", "spd_field_27x15", "phase_3d", "spd_field_3d"])
def test_dual_fp64_matches_oracle(hg, ctx, case):
    rng = np.random.default_rng(23)
    if case == "square15":
        ms = W.square_inclusion_15()
        N, A, phase = ms.N, ms.full_field(), ms
    elif case == "spd_field_27x15":
        N = (27, 15)
        A, phase = W.random_spd_field(N, rng, 1.0, 40.0), None
    elif case == "phase_3d":
        N = (15, 9, 15)
        ph = (rng.random(N) < 0.3).astype(np.uint8)
        tab = np.stack([np.eye(3), W.random_spd_pair(3, rng, 1.0, 30.0)[1]])
        phase = W.Microstructure(N, ph, tab)
        A = phase.full_field()
    else:
        N = (9, 15, 5)
        A, phase = W.random_spd_field(N, rng, 1.0, 20.0), None
    d = len(N)
    g = ctx.grid(N)
    if phase is not None:
        g.set_coeffs_phase(phase.phase, phase.table)
    else:
        g.set_coeffs_field(A)
    r = g.solve(hg.default_opts(tol=1e-12, formulation=hg.HG_DUAL))
    assert r["status"] == 0
    ref = O.solve_AH_dual(A, N, tol=1e-12)
    assert rel(r["CH"], ref["CH"]) <= 1e-9
    assert rel(r["AH"], ref["AH"]) <= 1e-9
    assert rel(r["AH_flux"], ref["AH_flux"]) <= 1e-8
    for l in range(d):
        x = g.field(l)
        assert np.max(np.abs(x - ref["x"][l])) <= 1e-8 * max(1.0, np.max(np.abs(ref["x"][l])))
        assert abs(r["iters"][l] - ref["iters"][l]) <= 2
    # GaNi: the dual A_H is the primal A_H
    p = g.solve(hg.default_opts(tol=1e-12))
    assert rel(r["AH"], p["AH"]) <= 1e-9
    g.close()


def test_dual_mixed_precision_and_moulinec_suquet(hg, ctx):
    ms = W.circles_2d(n=135, count=12, r_lo=5, r_hi=15, contrast=100.0, seed=21)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    ref = g.solve(hg.default_opts(tol=1e-11))
    dm = g.solve(hg.default_opts(tol=1e-7, prec=hg.HG_MIXED, formulation=hg.HG_DUAL))
    assert dm["status"] == 0 and max(dm["outer"]) >= 1
    assert rel(dm["AH"], ref["AH"]) <= 1e-6
    msd = g.solve(hg.default_opts(tol=1e-9, method=hg.HG_MS, formulation=hg.HG_DUAL, max_iter=100000))
    # Moulinec-Suquet on the dual iterates with A^-1: bounds 1/100 .. 1
    assert abs(msd["c_A"] - 0.01) < 1e-15 and abs(msd["C_A"] - 1.0) < 1e-15
    assert rel(msd["AH"], ref["AH"]) <= 1e-6
    # the primal afterwards is unaffected by the dual state of the grid
    p2 = g.solve(hg.default_opts(tol=1e-11))
    np.testing.assert_array_equal(p2["AH"], ref["AH"])
    g.close()


def test_dual_laminate_homogeneous_and_errors(hg, ctx):
    N = (9, 7)
    rng = np.random.default_rng(4)
    a = np.exp(rng.uniform(0, np.log(100.0), size=N[0]))
    A = np.einsum("ab,...->ab...", np.eye(2), np.broadcast_to(a[:, None], N))
    g = ctx.grid(N)
    g.set_coeffs_field(A)
    r = g.solve(hg.default_opts(tol=1e-14, formulation=hg.HG_DUAL))
    expect = np.diag([1.0 / np.mean(1.0 / a), np.mean(a)])
    np.testing.assert_allclose(r["AH"], expect, rtol=1e-11, atol=1e-12)
    assert r["iters"][0] == 0
    # every load is needed to invert the compliance
    bad = g.solve(hg.default_opts(formulation=hg.HG_DUAL, loads_mask=1), raise_on_error=False)
    assert bad["status"] == -1
    assert g.solve(hg.default_opts(formulation=5), raise_on_error=False)["status"] == -1
    g.close()
    A0 = np.array([[3.0, 1.0], [1.0, 2.0]])
    h = ctx.grid(N)
    h.set_coeffs_phase(np.zeros(N, np.uint8), A0[None])
    r = h.solve(hg.default_opts(formulation=hg.HG_DUAL))
    assert r["iters"] == [0, 0]
    np.testing.assert_allclose(r["AH"], A0, atol=1e-13)
    np.testing.assert_allclose(r["CH"], np.linalg.inv(A0), atol=1e-14)
    h.close()


def test_dual_through_the_scheduler(hg, ctx):
    ms = W.square_inclusion_15()
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    o = hg.default_opts(tol=1e-10, formulation=hg.HG_DUAL)
    blocking = g.solve(o)
    t = ctx.submit(g, o)
    res = None
    while res is None:
        res = ctx.poll(t, 100000)
    np.testing.assert_array_equal(res["AH"], blocking["AH"])
    np.testing.assert_array_equal(res["CH"], blocking["CH"])
    g.close()
