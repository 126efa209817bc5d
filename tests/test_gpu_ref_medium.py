"""CG with a general reference medium A0 on the GPU against the oracle.

The iteration runs on Gamma_N(A0) A_N in the scalar product (A0 u, v); its
solution is the GaNi solution for every SPD A0, so A_H matches the A0 = I
solve, while the iterates and the count follow the oracle's `cg_ref`.
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


def aniso_medium(N, seed=8):
    rng = np.random.default_rng(seed)
    ph = (rng.random(N) < 0.35).astype(np.uint8)
    tab = np.array([[[1.0, 0.0], [0.0, 50.0]], [[20.0, 0.0], [0.0, 1000.0]]])
    return W.Microstructure(N, ph, tab)


def test_ref_medium_fp64_matches_oracle_and_A0_free_solution(hg, ctx):
    ms = aniso_medium((27, 27))
    A = ms.full_field()
    A0 = np.array([[5.0, 1.0], [1.0, 250.0]])
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    r = g.solve(hg.default_opts(tol=1e-11, A0=A0))
    ref = O.solve_AH_ref(A, ms.N, A0, tol=1e-11)
    for l in range(2):
        assert abs(r["iters"][l] - ref["iters"][l]) <= 2, (r["iters"], ref["iters"])
        x = g.field(l)
        assert np.max(np.abs(x - ref["x"][l])) <= 1e-8 * np.max(np.abs(ref["x"][l]))
    plain = g.solve(hg.default_opts(tol=1e-11))
    err = np.max(np.abs(r["AH"] - plain["AH"])) / np.max(np.abs(plain["AH"]))
    assert err <= 1e-9, err
    # an anisotropic reference medium close to the medium's conditions it better
    assert sum(r["iters"]) < 0.5 * sum(plain["iters"])
    g.close()


def test_ref_medium_3d_field_and_mixed(hg, ctx):
    rng = np.random.default_rng(5)
    N = (15, 9, 15)
    A = W.random_spd_field(N, rng, 1.0, 40.0)
    A0 = W.random_spd_field((1, 1, 1), rng, 2.0, 20.0).reshape(3, 3)
    g = ctx.grid(N)
    g.set_coeffs_field(A)
    r = g.solve(hg.default_opts(tol=1e-11, A0=A0))
    ref = O.solve_AH_ref(A, N, A0, tol=1e-11)
    assert max(abs(a - b) for a, b in zip(r["iters"], ref["iters"])) <= 2
    assert np.max(np.abs(r["AH"] - ref["AH"])) <= 1e-9 * np.max(np.abs(ref["AH"]))
    m = g.solve(hg.default_opts(tol=1e-8, prec=hg.HG_MIXED, A0=A0))
    assert m["status"] == 0
    assert np.max(np.abs(m["AH"] - ref["AH"])) <= 1e-6 * np.max(np.abs(ref["AH"]))
    g.close()


def test_ref_medium_scalar_case_and_errors(hg, ctx):
    ms = W.square_inclusion_15()
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    plain = g.solve(hg.default_opts(tol=1e-12))
    lam = g.solve(hg.default_opts(tol=1e-12, A0=4.0 * np.eye(2)))
    assert lam["iters"] == plain["iters"]
    assert np.max(np.abs(lam["AH"] - plain["AH"])) <= 1e-12
    bad = g.solve(hg.default_opts(A0=np.array([[1.0, 2.0], [2.0, 1.0]])), raise_on_error=False)
    assert bad["status"] == -3      # not SPD
    bad = g.solve(hg.default_opts(A0=np.eye(2) * 2, method=hg.HG_MS), raise_on_error=False)
    assert bad["status"] == -1
    bad = g.solve(hg.default_opts(A0=np.eye(2) * 2, formulation=hg.HG_DUAL), raise_on_error=False)
    assert bad["status"] == -1
    # the grid's next plain solve is unaffected by the reference-medium state
    again = g.solve(hg.default_opts(tol=1e-12))
    np.testing.assert_array_equal(again["AH"], plain["AH"])
    # homogeneous medium: zero right-hand side under the A0 scalar product too
    A0 = np.array([[3.0, 1.0], [1.0, 2.0]])
    h = ctx.grid((9, 7))
    h.set_coeffs_phase(np.zeros((9, 7), np.uint8), A0[None])
    r = h.solve(hg.default_opts(A0=np.array([[7.0, -1.0], [-1.0, 0.5]])))
    assert r["iters"] == [0, 0]
    np.testing.assert_allclose(r["AH"], A0, atol=1e-13)
    g.close()
    h.close()
