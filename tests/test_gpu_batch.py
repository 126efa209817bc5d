"""Batched solves (hg_solve_batch: every pass one launch for all problems of a
shape, one CUDA graph for all shapes) against single solves and the oracle.

A batched launch runs, for each problem, the same tile bodies with the same
tile-to-CTA map and fixed-order reductions as that problem's own launch, so
each problem's iterates, iteration counts and A_H equal its single solve
bitwise (single solves with the pass kernels, resident = 0: a mixed single
solve of a square 2D grid otherwise runs the resident kernel, whose partial
sums are grouped differently).
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


def problems(n, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        vf = rng.uniform(0.1, 0.5)
        contrast = float(np.exp(rng.uniform(np.log(10.0), np.log(1e4))))
        out.append(W.ellipses_2d(n, vf, contrast, np.random.default_rng(seed + 17 * k)))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_single_solves(hg, ctx, prec):
    pr = hg.HG_MIXED if prec == "mixed" else hg.HG_FP64
    ms = problems(45, 9, 5)
    grids = []
    for m in ms:
        g = ctx.grid(m.N)
        g.set_coeffs_phase(m.phase, m.table)
        grids.append(g)
    o = hg.default_opts(tol=1e-7, prec=pr, max_iter=20000, batch_tiles=0, resident=0)
    batch = ctx.solve_batch(grids, o)
    fields = [g.field(1) for g in grids]
    for g, b, f in zip(grids, batch, fields):
        single = g.solve(o)
        assert b["status"] == 0
        assert b["iters"] == single["iters"] and b["outer"] == single["outer"]
        np.testing.assert_array_equal(b["AH"], single["AH"])
        np.testing.assert_array_equal(f, g.field(1))
    for g in grids:
        g.close()


def test_batch_against_oracle_3d_and_runtime_sizes(hg, ctx):
    rng = np.random.default_rng(2)
    for N in [(15, 9, 15), (7, 9, 5), (45, 75)]:
        As = [W.random_spd_field(N, rng, 1.0, 20.0) for _ in range(3)]
        grids = []
        for A in As:
            g = ctx.grid(N)
            g.set_coeffs_field(A)
            grids.append(g)
        res = ctx.solve_batch(grids, hg.default_opts(tol=1e-11))
        for A, r in zip(As, res):
            ref = O.solve_AH(A, N, tol=1e-11)["AH"]
            assert np.max(np.abs(r["AH"] - ref)) <= 1e-8 * np.max(np.abs(ref))
        resm = ctx.solve_batch(grids, hg.default_opts(tol=1e-9, prec=hg.HG_MIXED))
        for A, r in zip(As, resm):
            ref = O.solve_AH(A, N, tol=1e-11)["AH"]
            assert np.max(np.abs(r["AH"] - ref)) <= 1e-6 * np.max(np.abs(ref))
        for g in grids:
            g.close()


def test_batch_with_a_homogeneous_problem_and_loads_mask(hg, ctx):
    ms = problems(27, 3, 9)
    N = ms[0].N
    grids = []
    for m in ms:
        g = ctx.grid(N)
        g.set_coeffs_phase(m.phase, m.table)
        grids.append(g)
    A0 = np.array([[3.0, 1.0], [1.0, 2.0]])
    h = ctx.grid(N)
    h.set_coeffs_phase(np.zeros(N, np.uint8), A0[None])
    grids.append(h)
    o = hg.default_opts(tol=1e-8, prec=hg.HG_MIXED, batch_tiles=0, resident=0)
    res = ctx.solve_batch(grids, o)
    assert res[-1]["iters"] == [0, 0]
    np.testing.assert_allclose(res[-1]["AH"], A0, atol=1e-13)
    for g, r in zip(grids[:-1], res[:-1]):
        single = g.solve(o)
        np.testing.assert_array_equal(r["AH"], single["AH"])
    only2 = ctx.solve_batch(grids, hg.default_opts(tol=1e-8, prec=hg.HG_MIXED, loads_mask=2))
    for r in only2:
        assert r["iters"][0] == 0 and r["AH"][0, 0] == 0.0
    for g in grids:
        g.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_of_mixed_shapes_equals_single_solves(hg, ctx, prec):
    """2D and 3D problems of five shapes (compile-time and run-time FFT
    lengths) in one call: one CUDA graph per chunk with a branch per shape.
    Each problem's result equals its single solve bitwise and the oracle
    within the path's tolerance."""
    pr = hg.HG_MIXED if prec == "mixed" else hg.HG_FP64
    rng = np.random.default_rng(31)
    shapes = [(45, 45), (27, 27, 27), (75, 75), (15, 9, 15), (63, 35)]
    probs = []
    for k in range(10):
        N = shapes[k % len(shapes)]
        if len(N) == 2 and k < 5:
            m = W.ellipses_2d(N[0], 0.3, 50.0, np.random.default_rng(100 + k))
            probs.append((N, ("phase", m.phase, m.table)))
        else:
            probs.append((N, ("field", W.random_spd_field(N, rng, 1.0, 30.0))))
    grids = []
    for N, c in probs:
        g = ctx.grid(N)
        if c[0] == "phase":
            g.set_coeffs_phase(c[1], c[2])
        else:
            g.set_coeffs_field(c[1])
        grids.append(g)
    o = hg.default_opts(tol=1e-8, prec=pr, max_iter=20000, batch_tiles=0, resident=0)
    batch = ctx.solve_batch(grids, o)
    for g, b, (N, c) in zip(grids, batch, probs):
        assert b["status"] == 0 and b["AH"].shape == (len(N), len(N))
        single = g.solve(o)
        assert b["iters"] == single["iters"] and b["outer"] == single["outer"]
        np.testing.assert_array_equal(b["AH"], single["AH"])
    # batch row tiles (the default): the same solutions up to rounding
    tiled = ctx.solve_batch(grids, hg.default_opts(tol=1e-8, prec=pr, max_iter=20000))
    bound = 1e-6 if prec == "mixed" else 1e-7
    for g, b, t, (N, c) in zip(grids, batch, tiled, probs):
        assert t["status"] == 0
        assert np.max(np.abs(t["AH"] - b["AH"])) <= bound * np.max(np.abs(b["AH"]))
        assert all(abs(x - y) <= 3 for x, y in zip(t["iters"], b["iters"]))
    for g, b, (N, c) in list(zip(grids, tiled, probs))[5:8]:
        ref = O.solve_AH(c[1], N, tol=1e-11)["AH"]
        assert np.max(np.abs(b["AH"] - ref)) <= bound * np.max(np.abs(ref))
    for g in grids:
        g.close()


def test_batch_errors(hg, ctx):
    a = ctx.grid((15, 15))
    m = W.square_inclusion_15()
    a.set_coeffs_phase(m.phase, m.table)
    import ctypes
    lib = hg.load()
    res = (hg.Result * 2)()
    hs = (ctypes.c_void_p * 2)(a.h, a.h)
    assert lib.hg_solve_batch(hs, 2, ctypes.byref(hg.default_opts()), res) == -1
    hs1 = (ctypes.c_void_p * 1)(a.h)
    assert lib.hg_solve_batch(hs1, 1, ctypes.byref(hg.default_opts(method=hg.HG_MS)), res) == -1
    assert lib.hg_solve_batch(hs1, 1, ctypes.byref(hg.default_opts(formulation=hg.HG_DUAL)), res) == -1
    assert lib.hg_solve_batch(hs1, 1, ctypes.byref(hg.default_opts(A0=2.0 * np.eye(2))), res) == -1
    assert lib.hg_solve_batch(hs1, 0, ctypes.byref(hg.default_opts()), res) == -1
    assert lib.hg_solve_batch(hs1, 1, ctypes.byref(hg.default_opts(batch_tiles=2)), res) == -1
    other = hg.Context(0)
    b = other.grid((15, 15))
    b.set_coeffs_phase(m.phase, m.table)
    hs = (ctypes.c_void_p * 2)(a.h, b.h)   # grids of two contexts
    assert lib.hg_solve_batch(hs, 2, ctypes.byref(hg.default_opts()), res) == -1
    a.close()
    b.close()
    other.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_tiles_many_problems_against_oracle(hg, ctx, prec):
    """Default batch row tiles on groups large enough to take them (24 x 45^2,
    12 x 75^2, 6 x 27^3): every A_H within the path's tolerance of the oracle,
    iteration counts within 3 of the single solves."""
    pr = hg.HG_MIXED if prec == "mixed" else hg.HG_FP64
    bound = 1e-6 if prec == "mixed" else 1e-8
    rng = np.random.default_rng(77)
    probs = [((45, 45), W.random_spd_field((45, 45), rng, 1.0, 40.0)) for _ in range(24)]
    probs += [((75, 75), W.random_spd_field((75, 75), rng, 1.0, 40.0)) for _ in range(12)]
    probs += [((27, 27, 27), W.random_spd_field((27, 27, 27), rng, 1.0, 40.0)) for _ in range(6)]
    grids = []
    for N, A in probs:
        g = ctx.grid(N)
        g.set_coeffs_field(A)
        grids.append(g)
    o = hg.default_opts(tol=1e-10, prec=pr)
    res = ctx.solve_batch(grids, o)
    for k, ((N, A), g, r) in enumerate(zip(probs, grids, res)):
        assert r["status"] == 0
        if k % 6 == 0:
            ref = O.solve_AH(A, N, tol=1e-11)["AH"]
            assert np.max(np.abs(r["AH"] - ref)) <= bound * np.max(np.abs(ref)), (N, k)
            single = g.solve(o)
            assert all(abs(x - y) <= 3 for x, y in zip(r["iters"], single["iters"]))
    for g in grids:
        g.close()
