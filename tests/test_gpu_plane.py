"""The 3D plane passes of the FP32 CG iteration (axes 1 and 2 transformed in
shared memory, one CTA per plane and component) against the CPU oracle and
against the pass kernels.

The method is the CG of Sec. 5.3 on Eq. final_system with Gamma_hat of
Eq. Gamma_hat; the plane passes only regroup the transforms of an iteration,
so their A_H meets the same bounds as the pass kernels' (1e-6 relative for
the mixed path) and their iteration counts agree up to the rounding of the
partial sums.  A plane iteration is three launches, the pass kernels' five.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def ctx(hg):
    c = hg.Context(0)
    yield c
    c.close()


def _balls(N, seed, contrast=100.0, vf=0.2):
    return W.balls_to_vf(N, vf, np.random.default_rng(seed), contrast)


def _launches_per_iter(r):
    # the loads of a grid share every launch
    return r["launches"] / max(1, max(r["iters"]))


# cubic and N0 != N1 = N2 grids of every plane length (N odd, H odd and even);
# N0 = 21 and 35 take the run-time FFT plan in the axis-0 pass
@pytest.mark.parametrize("N", [(15, 15, 15), (27, 27, 27), (45, 45, 45), (81, 27, 27), (27, 45, 45),
                               (45, 81, 81), (15, 135, 135), (21, 27, 27), (35, 45, 45)])
def test_plane_matches_oracle_and_pass_kernels(hg, ctx, N):
    ms = _balls(N, seed=sum(N))
    ref = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    res = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED))
    plain = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, resident=0))
    assert res["status"] == 0 and plain["status"] == 0
    assert rel_max(res["AH"], ref["AH"]) < 1e-6
    assert rel_max(res["AH"], plain["AH"]) < 1e-6
    for a, b in zip(res["iters"], plain["iters"]):
        assert abs(a - b) <= max(3, 0.05 * b)
    # three launches per iteration instead of five (set-up launches aside)
    assert _launches_per_iter(res) < _launches_per_iter(plain) - 1.0
    assert max(res["rel_res"]) <= 1e-9
    for j in range(3):
        e = g.field(j)
        err = np.sqrt(O.inner(e - ref["x"][j], e - ref["x"][j]))
        assert err <= 1e-6 * max(1.0, np.sqrt(O.inner(ref["x"][j], ref["x"][j])))
    g.close()


def test_plane_packed_field_anisotropic_cell(hg, ctx):
    """A full symmetric coefficient field (packed layout, every entry of a row
    of A(x) from its own array) on a cell with unequal sides."""
    N = (27, 45, 45)
    rng = np.random.default_rng(7)
    A = W.random_spd_field(N, rng, 1.0, 30.0)
    Y = (1.0, 0.7, 1.3)
    ref = O.solve_AH(A, N, Y=Y, tol=1e-12)
    g = ctx.grid(N, Y=Y)
    g.set_coeffs_field(A)
    res = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED))
    plain = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, resident=0))
    assert res["status"] == 0
    assert _launches_per_iter(res) < _launches_per_iter(plain) - 1.0
    assert rel_max(res["AH"], ref["AH"]) < 1e-6
    g.close()


def test_plane_dual_formulation_and_loads_mask(hg, ctx):
    """The dual formulation (projection onto J_N in the axis-0 pass, inverse
    coefficients in the plane passes) and a single active load (the other
    loads' CTAs publish zeros)."""
    N = (27, 27, 27)
    ms = _balls(N, seed=3, contrast=50.0)
    # (the oracle's dual CG reaches about 1.6e-12 on loads 0 and 2 of this
    # grid before rounding takes its iterates out of J_N: 1e-10 is attainable)
    ref_d = O.solve_AH_dual(ms.full_field(), ms.N, tol=1e-10)
    ref = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    r = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, formulation=hg.HG_DUAL))
    assert r["status"] == 0
    assert rel_max(r["AH"], ref_d["AH"]) < 1e-6
    # GaNi: the dual homogenized matrix is the primal one
    assert rel_max(r["AH"], ref["AH"]) < 1e-6
    r1 = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, loads_mask=0b010))
    assert r1["status"] == 0
    assert r1["iters"][0] == 0 and r1["iters"][2] == 0 and r1["iters"][1] > 0
    assert abs(r1["AH"][1, 1] - ref["AH"][1, 1]) < 1e-6 * ref["AH"][1, 1]
    g.close()


def test_plane_batch_equals_single_solves_bitwise(hg, ctx):
    """hg_solve_batch runs the batched plane kernels (grid z = problem) with the
    same tiles and reductions as a single solve: the same A_H to the bit."""
    shapes = [(27, 27, 27), (27, 27, 27), (45, 45, 45), (81, 27, 27)]
    grids, singles = [], []
    # batch_tiles = 0: the batch's row passes (right-hand side, refinement) take
    # the single solve's tiles
    o = hg.default_opts(tol=1e-8, prec=hg.HG_MIXED, batch_tiles=0)
    for k, N in enumerate(shapes):
        ms = _balls(N, seed=100 + k, contrast=10.0 ** (1 + k))
        g = ctx.grid(ms.N)
        g.set_coeffs_phase(ms.phase, ms.table)
        singles.append(g.solve(o))
        grids.append(g)
    res = ctx.solve_batch(grids, o)
    for a, b in zip(res, singles):
        assert a["status"] == 0
        assert np.array_equal(a["AH"], b["AH"])
        assert list(a["iters"]) == list(b["iters"])
    for g in grids:
        g.close()


def test_plane_scheduler_alone_and_in_a_mix(hg, ctx):
    """3D requests through hg_submit: the rolling batch's plane launches give
    each request the result it gets alone."""
    shapes = [(27, 27, 27), (45, 45, 45), (45, 45, 45), (27, 45, 45)]
    o = hg.default_opts(tol=1e-8, prec=hg.HG_MIXED)
    probs = [_balls(N, seed=200 + k) for k, N in enumerate(shapes)]
    grids = []
    for ms in probs:
        g = ctx.grid(ms.N)
        g.set_coeffs_phase(ms.phase, ms.table)
        grids.append(g)
    alone = [ctx.poll(ctx.submit(g, o), timeout_us=-1) for g in grids]
    tickets = [ctx.submit(g, o) for g in grids]
    mixed = [ctx.poll(t, timeout_us=-1) for t in tickets]
    for a, b in zip(alone, mixed):
        assert a["status"] == 0 and b["status"] == 0
        assert np.array_equal(a["AH"], b["AH"])
    ref = O.solve_AH(probs[0].full_field(), probs[0].N, tol=1e-12)
    assert rel_max(alone[0]["AH"], ref["AH"]) < 1e-6
    for g in grids:
        g.close()


def test_plane_time_pass_and_pass_count(hg, ctx):
    """hg_num_iter_passes gives the schedule's launches per iteration (3 for
    the plane passes, the pass kernels' 5 otherwise), and time_pass brackets
    each of the three plane launches without changing the result."""
    N = (27, 27, 27)
    ms = _balls(N, seed=11)
    g = ctx.grid(N)
    g.set_coeffs_phase(ms.phase, ms.table)
    o = hg.default_opts(tol=1e-8, prec=hg.HG_MIXED)
    assert g.num_iter_passes(o) == 3
    assert g.num_iter_passes(hg.default_opts(tol=1e-8, prec=hg.HG_MIXED, resident=0)) == 5
    assert g.num_iter_passes(hg.default_opts(tol=1e-8, prec=hg.HG_FP64)) == 5
    base = g.solve(o)
    for p in range(3):
        r = g.solve(hg.default_opts(tol=1e-8, prec=hg.HG_MIXED, time_pass=p))
        assert r["status"] == 0 and r["pass_launches"] > 0 and r["pass_ms_total"] > 0.0
        assert np.array_equal(r["AH"], base["AH"])
    with pytest.raises(hg.HGError):
        g.solve(hg.default_opts(tol=1e-8, prec=hg.HG_MIXED, time_pass=3))
    g.close()
