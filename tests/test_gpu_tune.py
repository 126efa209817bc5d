"""Launch geometry and its autotuner (hg_set_launch_cfg, hg_tune) on the GPU.

Every tiling the kernels accept must give the solution of Eq. final_system:
the A_H of each admissible geometry is compared with the oracle's, for
compile-time and run-time FFT lengths in 2D and 3D, FP64 and mixed precision.
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


def admissible(hg, g, prec):
    """Every (rb, lb, lanes) the library accepts for grid g (probed through
    hg_set_launch_cfg, which validates on the host)."""
    d = g.d
    lane_sets = [[0, 0]]
    if d == 2:
        lane_sets = [[c, 0] for c in (1, 2, 4, 8, 16, 32)]
    else:
        lane_sets = [[c0, c1] for c0 in (1, 2, 4, 8) for c1 in (1, 2, 4, 8)]
    out = []
    for lb in range(1, d + 1):
        for rb in range(1, 65):
            try:
                g.set_launch_cfg(prec, rb, lb, lane_sets[0])
            except hg.HGError:
                continue
            out.append((rb, lb, None))
    lanes_ok = []
    rb0, lb0 = out[0][0], out[0][1]
    for ln in lane_sets:
        try:
            g.set_launch_cfg(prec, rb0, lb0, ln)
            lanes_ok.append(ln)
        except hg.HGError:
            pass
    return [(rb, lb) for rb, lb, _ in out], lanes_ok


CASES = [
    ((45, 45), "ct 2D"),
    ((63, 35), "runtime 2D"),
    ((27, 27, 27), "ct 3D"),
    ((15, 21, 25), "runtime 3D"),
]


@pytest.mark.parametrize("N,kind", CASES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_geometry_gives_the_oracle_solution(hg, ctx, N, kind, prec):
    pr = hg.HG_MIXED if prec == "mixed" else hg.HG_FP64
    rng = np.random.default_rng(sum(N))
    A = W.random_spd_field(N, rng, 1.0, 50.0)
    ref = O.solve_AH(A, N, tol=1e-11)["AH"]
    bound = 1e-6 if prec == "mixed" else 1e-8
    g = ctx.grid(N)
    g.set_coeffs_field(A)
    default = g.launch_cfg(pr)
    tiles, lanes = admissible(hg, g, pr)
    assert (default["row_rb"], default["row_lb"]) in tiles
    assert default["lanes"] in lanes
    assert len(tiles) >= 2 and len(lanes) >= 1
    # every tile with the default lanes, every lane set with the default tile
    cfgs = [(rb, lb, default["lanes"]) for rb, lb in tiles]
    cfgs += [(default["row_rb"], default["row_lb"], ln) for ln in lanes]
    o = hg.default_opts(tol=1e-10, prec=pr)
    iters0 = None
    for rb, lb, ln in cfgs:
        g.set_launch_cfg(pr, rb, lb, ln)
        got = g.launch_cfg(pr)
        assert (got["row_rb"], got["row_lb"], got["lanes"]) == (rb, lb, list(ln))
        r = g.solve(o)
        assert r["status"] == 0
        err = np.max(np.abs(r["AH"] - ref)) / np.max(np.abs(ref))
        assert err <= bound, (rb, lb, ln, err)
        if iters0 is None:
            iters0 = r["iters"]
        assert all(abs(a - b) <= 2 for a, b in zip(r["iters"], iters0)), (rb, lb, ln)
    g.close()


def test_invalid_geometries_are_rejected(hg, ctx):
    g = ctx.grid((45, 45))
    m = W.ellipses_2d(45, 0.3, 100.0, np.random.default_rng(3))
    g.set_coeffs_phase(m.phase, m.table)
    before = g.launch_cfg(hg.HG_MIXED)
    for rb, lb, ln in [(0, 1, [1, 0]), (1, 0, [1, 0]), (1, 3, [1, 0]), (1, 1, [3, 0]),
                       (1, 1, [1, 1]), (46, 1, [1, 0]), (1, 1, [0, 0]), (64, 2, [1, 0])]:
        with pytest.raises(hg.HGError) as e:
            g.set_launch_cfg(hg.HG_MIXED, rb, lb, ln)
        assert e.value.status == hg.HG_ERR_ARG
    assert g.launch_cfg(hg.HG_MIXED) == before
    g.close()


@pytest.mark.parametrize("N", [(243, 243), (27, 27, 27)])
def test_tune_then_solve_and_cache(hg, ctx, N, tmp_path):
    cache = str(tmp_path / "tune.txt")
    if len(N) == 2:
        m = W.ellipses_2d(N[0], 0.3, 100.0, np.random.default_rng(8))
        set_c = lambda g: g.set_coeffs_phase(m.phase, m.table)
        A = m.table[m.phase.astype(np.intp)]                      # (*N, d, d)
        A = np.moveaxis(np.moveaxis(A, -1, 0), -1, 0)             # (d, d, *N)
    else:
        A = W.random_spd_field(N, np.random.default_rng(8), 1.0, 100.0)
        set_c = lambda g: g.set_coeffs_field(A)
    ref = O.solve_AH(A, N, tol=1e-11)["AH"]
    g = ctx.grid(N)
    set_c(g)
    for pr, bound in [(hg.HG_MIXED, 1e-6), (hg.HG_FP64, 1e-8)]:
        t = g.tune(pr, reps=4, cache_path=cache)
        assert not t["from_cache"] and t["candidates"] >= 2
        assert t["ms_chosen"] > 0 and t["ms_heuristic"] > 0
        assert g.launch_cfg(pr) == t["chosen"]
        r = g.solve(hg.default_opts(tol=1e-10, prec=pr))
        assert np.max(np.abs(r["AH"] - ref)) <= bound * np.max(np.abs(ref))
    lines = open(cache).read().splitlines()
    assert len(lines) == 2 and all(ln.startswith("hg-tune-v2 ") for ln in lines)
    # a second grid of the same shape takes the cached geometry without timing
    g2 = ctx.grid(N)
    set_c(g2)
    t2 = g2.tune(hg.HG_MIXED, reps=4, cache_path=cache)
    assert t2["from_cache"] and t2["candidates"] == 0
    assert t2["chosen"] == g.launch_cfg(hg.HG_MIXED) == g2.launch_cfg(hg.HG_MIXED)
    fields = lines[0].split()
    found = hg.tune_cache_find(cache, fields[1], int(fields[2]), hg.HG_MIXED, N)
    assert found is not None and found[0] == t2["chosen"]
    r = g2.solve(hg.default_opts(tol=1e-10, prec=hg.HG_MIXED))
    assert np.max(np.abs(r["AH"] - ref)) <= 1e-6 * np.max(np.abs(ref))
    g.close()
    g2.close()


def test_batch_runs_a_tuned_lead_geometry_on_untuned_problems(hg, ctx):
    """A group runs its first grid's geometry; the other grids' reduction slots
    are sized for it.  The lead is forced to one row per CTA (the most CTAs)."""
    N = (75, 75)
    ms = [W.ellipses_2d(75, 0.3, 300.0, np.random.default_rng(40 + k)) for k in range(4)]
    grids = []
    for m in ms:
        g = ctx.grid(N)
        g.set_coeffs_phase(m.phase, m.table)
        grids.append(g)
    grids[0].set_launch_cfg(hg.HG_MIXED, 1, 1, [1, 0])
    grids[0].set_launch_cfg(hg.HG_FP64, 1, 1, [1, 0])
    o = hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, batch_tiles=0)
    res = ctx.solve_batch(grids, o)
    for m, r in zip(ms, res):
        A = np.moveaxis(np.moveaxis(m.table[m.phase.astype(np.intp)], -1, 0), -1, 0)
        ref = O.solve_AH(A, N, tol=1e-11)["AH"]
        assert r["status"] == 0
        assert np.max(np.abs(r["AH"] - ref)) <= 1e-6 * np.max(np.abs(ref))
    for g in grids:
        g.close()


def test_default_row_tile_fits_the_offset_table_3d_runtime_length(hg, ctx):
    """A 3D grid with a run-time last-axis length and many rows: the default
    row tile stays within the 64 real rows a row-pass CTA can index, and the
    mixed solve matches the oracle."""
    N = (49, 63, 25)
    A = W.random_spd_field(N, np.random.default_rng(12), 1.0, 20.0)
    g = ctx.grid(N)
    g.set_coeffs_field(A)
    for pr in (hg.HG_MIXED, hg.HG_FP64):
        c = g.launch_cfg(pr)
        assert c["row_rb"] * c["row_lb"] * 3 <= 64, c
    ref = O.solve_AH(A, N, tol=1e-11)["AH"]
    r = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED))
    assert np.max(np.abs(r["AH"] - ref)) <= 1e-6 * np.max(np.abs(ref))
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_radix_order_gives_the_oracle_solution(hg, ctx, prec):
    """Run-time FFT plans: every order of the radix-3/5/7 stages along each
    axis (105 = 3 5 7 and 63 = 3 3 7 in 2D; 3D with 25 = 5 5 and 21 = 3 7)."""
    import itertools
    pr = hg.HG_MIXED if prec == "mixed" else hg.HG_FP64
    bound = 1e-6 if prec == "mixed" else 1e-8
    for N in [(105, 63), (21, 15, 25)]:
        A = W.random_spd_field(N, np.random.default_rng(5), 1.0, 30.0)
        ref = O.solve_AH(A, N, tol=1e-11)["AH"]
        g = ctx.grid(N)
        g.set_coeffs_field(A)
        c = g.launch_cfg(pr)
        default = c["radix"]
        assert [sorted(o) for o in default[:len(N)]] == [o for o in default[:len(N)]]   # ascending
        o = hg.default_opts(tol=1e-10, prec=pr)
        for a in range(len(N)):
            for order in sorted(set(itertools.permutations(default[a]))):
                radix = [list(x) for x in default]
                radix[a] = list(order)
                g.set_launch_cfg(pr, c["row_rb"], c["row_lb"], c["lanes"], radix)
                assert g.launch_cfg(pr)["radix"][a] == list(order)
                r = g.solve(o)
                err = np.max(np.abs(r["AH"] - ref)) / np.max(np.abs(ref))
                assert r["status"] == 0 and err <= bound, (N, a, order, err)
            g.set_launch_cfg(pr, c["row_rb"], c["row_lb"], c["lanes"], default)
        g.close()


def test_radix_orders_are_validated(hg, ctx):
    g = ctx.grid((105, 45))     # 105 has a run-time plan, 45 a compile-time kernel
    g.set_coeffs_field(W.random_spd_field((105, 45), np.random.default_rng(2), 1.0, 5.0))
    c = g.launch_cfg(hg.HG_MIXED)
    assert c["radix"][0] == [3, 5, 7] and c["radix"][1] == []
    for bad in ([[3, 5], [], []], [[3, 5, 5], [], []], [[3, 5, 7], [3, 3, 5], []], [[2, 5, 7], [], []],
                [[3, 5, 7], [], [3]]):
        with pytest.raises(hg.HGError) as e:
            g.set_launch_cfg(hg.HG_MIXED, c["row_rb"], c["row_lb"], c["lanes"], bad)
        assert e.value.status == hg.HG_ERR_ARG
    g.set_launch_cfg(hg.HG_MIXED, c["row_rb"], c["row_lb"], c["lanes"], [[7, 3, 5], [], []])
    # the order is the grid's: both precisions see it
    assert g.launch_cfg(hg.HG_FP64)["radix"][0] == [7, 3, 5]
    t = g.tune(hg.HG_MIXED, reps=2)
    assert t["heuristic"]["radix"][0] == [3, 5, 7]
    assert sorted(t["chosen"]["radix"][0]) == [3, 5, 7]
    assert t["candidates"] >= 6
    g.close()
