"""Parity of the CUDA path (through the C ABI) with the CPU oracle."""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))

GRIDS_2D = [(3, 3), (5, 3), (15, 15), (45, 75), (135, 27), (81, 243), (7, 49), (1, 5), (9, 1), (625, 9),
            (729, 9), (9, 729), (375, 27), (27, 375), (243, 15), (75, 45)]
GRIDS_3D = [(3, 3, 3), (5, 3, 7), (15, 9, 25), (27, 45, 21), (1, 3, 5), (7, 1, 9), (45, 27, 81),
            (135, 15, 27), (15, 81, 135)]


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def ctx(hg):
    c = hg.Context(0)
    yield c
    c.close()


# ---------------------------------------------------------------- DFT (Eq. DFT_def)
@pytest.mark.parametrize("N", GRIDS_2D + GRIDS_3D)
def test_spectrum_fp64_matches_oracle_dft(hg, ctx, N):
    rng = np.random.default_rng(abs(hash(N)) % 2**32)
    d = len(N)
    u = rng.standard_normal((d,) + N)
    g = ctx.grid(N)
    S = g.spectrum(u, hg.HG_FP64)
    ref = O.dft(u, d)[..., : (N[-1] + 1) // 2]
    assert S.shape == ref.shape
    assert rel_max(S, ref) < 1e-12
    g.close()


@pytest.mark.parametrize("N", [(45, 75), (15, 9, 25), (729, 15), (15, 729), (375, 243), (45, 27, 81),
                               (135, 15, 27)])
def test_spectrum_fp32_matches_oracle_dft(hg, ctx, N):
    rng = np.random.default_rng(5)
    d = len(N)
    u = rng.standard_normal((d,) + N)
    g = ctx.grid(N)
    S = g.spectrum(u, hg.HG_MIXED)
    ref = O.dft(u, d)[..., : (N[-1] + 1) // 2]
    assert rel_max(S, ref) < 2e-6
    g.close()


# ------------------------------------------------------- projection and matvec
@pytest.mark.parametrize("N", GRIDS_2D[:8] + GRIDS_3D)
def test_apply_G_and_GA_fp64(hg, ctx, N):
    rng = np.random.default_rng(11)
    d = len(N)
    u = rng.standard_normal((d,) + N)
    A = W.random_spd_field(N, rng, 1.0, 20.0)
    g = ctx.grid(N)
    g.set_coeffs_field(A)
    np.testing.assert_allclose(g.apply(u, with_A=False), O.apply_gamma(u, N), atol=1e-12)
    np.testing.assert_allclose(g.apply(u, with_A=True), O.apply_K(A, u, N), atol=1e-11)
    g.close()


def test_apply_general_reference_medium_and_cell(hg, ctx):
    N, Y = (15, 21), (1.0, 2.5)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((2,) + N)
    A0 = np.array([[3.0, 1.0], [1.0, 2.0]])
    g = ctx.grid(N, Y)
    np.testing.assert_allclose(g.apply(u, with_A=False, A0=A0), O.apply_G(u, N, Y, A0), atol=1e-12)
    np.testing.assert_allclose(g.apply(u, with_A=False), O.apply_gamma(u, N, Y), atol=1e-12)
    g.close()
    N3, Y3 = (9, 5, 7), (1.0, 0.5, 2.0)
    u3 = rng.standard_normal((3,) + N3)
    A03 = np.array([[2.0, 0.3, 0.1], [0.3, 1.5, 0.2], [0.1, 0.2, 1.0]])
    g3 = ctx.grid(N3, Y3)
    np.testing.assert_allclose(g3.apply(u3, with_A=False, A0=A03), O.apply_G(u3, N3, Y3, A03), atol=1e-12)
    g3.close()


@pytest.mark.parametrize("N", [(45, 75), (27, 45, 21)])
def test_apply_fp32(hg, ctx, N):
    rng = np.random.default_rng(3)
    d = len(N)
    u = rng.standard_normal((d,) + N)
    ms = W.Microstructure(N, (rng.random(N) < 0.3).astype(np.uint8), W.isotropic_table([1.0, 50.0], d))
    g = ctx.grid(N)
    g.set_coeffs_phase(ms.phase, ms.table)
    ref = O.apply_K(ms.full_field(), u, N)
    assert rel_max(g.apply(u, prec=hg.HG_MIXED), ref) < 2e-5
    g.close()


# ------------------------------------------------------------------ CG and A_H
def solve_both(hg, ctx, ms_or_A, N, tol=1e-10, prec=0, table=None, **kw):
    g = ctx.grid(N)
    if table is not None:
        g.set_coeffs_phase(ms_or_A, table)
        A = W.Microstructure(N, ms_or_A, table).full_field()
    else:
        g.set_coeffs_field(ms_or_A)
        A = ms_or_A
    res = g.solve(hg.default_opts(tol=tol, prec=prec, **kw))
    ref = O.solve_AH(A, N, tol=tol)
    fields = [g.field(j) for j in range(len(N))]
    g.close()
    return res, ref, fields


def test_square_inclusion_fp64_against_golden_and_oracle(hg, ctx):
    gold = json.load(open(os.path.join(HERE, "golden", "square_inclusion_15.json")))
    ms = W.square_inclusion_15()
    res, ref, fields = solve_both(hg, ctx, ms.phase, ms.N, tol=1e-12, table=ms.table)
    assert rel_max(res["AH"], np.array(gold["AH"])) < 1e-10
    assert rel_max(res["AH"], ref["AH"]) < 1e-10
    assert all(abs(a - b) <= 1 for a, b in zip(res["iters"], ref["iters"]))
    for j in range(2):
        np.testing.assert_allclose(fields[j], ref["x"][j], atol=1e-9)
    np.testing.assert_allclose(res["AH_flux"], res["AH"], atol=1e-9)


@pytest.mark.parametrize("N,kind", [((15, 21), "spd"), ((45, 45), "phase"), ((9, 7, 15), "spd"),
                                    ((15, 15, 15), "phase"), ((81, 5), "phase"), ((3, 3), "spd"),
                                    ((5, 3, 3), "phase")])
def test_solve_fp64_parity(hg, ctx, N, kind):
    rng = np.random.default_rng(sum(N))
    d = len(N)
    if kind == "spd":
        A = W.random_spd_field(N, rng, 1.0, 80.0)
        res, ref, fields = solve_both(hg, ctx, A, N)
    else:
        ph = (rng.random(N) < 0.35).astype(np.uint8)
        res, ref, fields = solve_both(hg, ctx, ph, N, table=W.isotropic_table([1.0, 100.0], d))
    assert res["status"] == 0
    assert rel_max(res["AH"], ref["AH"]) < 1e-8
    assert all(abs(a - b) <= 2 for a, b in zip(res["iters"], ref["iters"]))
    for j in range(d):
        err = np.sqrt(O.inner(fields[j] - ref["x"][j], fields[j] - ref["x"][j]))
        assert err <= 1e-7 * max(1.0, np.sqrt(O.inner(ref["x"][j], ref["x"][j])))


def test_solve_mixed_parity(hg, ctx):
    ms = W.circles_2d(n=135, count=10, r_lo=5, r_hi=12, contrast=100.0, seed=4)
    res, ref, _ = solve_both(hg, ctx, ms.phase, ms.N, tol=1e-10, prec=1, table=ms.table)
    assert res["status"] == 0
    assert rel_max(res["AH"], ref["AH"]) < 1e-6
    assert max(res["rel_res"]) <= 1e-10
    ms3 = W.spheres_3d(n=27, count=6, r_lo=2, r_hi=5, seed=8)
    res3, ref3, _ = solve_both(hg, ctx, ms3.phase, ms3.N, tol=1e-10, prec=1, table=ms3.table)
    assert res3["status"] == 0
    assert rel_max(res3["AH"], ref3["AH"]) < 1e-6


def test_laminate_and_homogeneous_exact(hg, ctx):
    gold = json.load(open(os.path.join(HERE, "golden", "laminate_9x7.json")))
    ms = W.laminate(tuple(gold["N"]), gold["layers_axis0"])
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    res = g.solve(hg.default_opts(tol=1e-14))
    np.testing.assert_allclose(res["AH"], np.array(gold["AH"]), rtol=1e-11, atol=1e-12)
    assert res["iters"][1] == 0
    g.close()
    N = (7, 5, 3)
    A0 = np.array([[4.0, 1.0, 0.5], [1.0, 3.0, 0.2], [0.5, 0.2, 2.0]])
    g = ctx.grid(N)
    g.set_coeffs_phase(np.zeros(N, np.uint8), A0[None])
    res = g.solve()
    assert res["iters"] == [0, 0, 0]
    np.testing.assert_allclose(res["AH"], A0, atol=1e-13)
    # mixed precision: the FP32 right-hand side is roundoff, too small to decide
    # the zero test, so the solve takes the FP64 one and does no iteration
    res = g.solve(hg.default_opts(prec=hg.HG_MIXED))
    assert res["iters"] == [0, 0, 0] and res["outer"] == [0, 0, 0]
    np.testing.assert_allclose(res["AH"], A0, atol=1e-13)
    g.close()
    # a laminate whose along-layer loads have b = 0 exactly and the across-layer
    # load not: the FP64 recheck decides per load, the mixed solve still
    # reaches the harmonic mean
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    res = g.solve(hg.default_opts(prec=hg.HG_MIXED, tol=1e-12))
    np.testing.assert_allclose(res["AH"], np.array(gold["AH"]), rtol=1e-11, atol=1e-12)
    assert res["iters"][1] == 0
    g.close()


def test_loads_mask_and_packed_layout(hg, ctx):
    N = (25, 15)
    rng = np.random.default_rng(9)
    A = W.random_spd_field(N, rng, 1.0, 10.0)
    g = ctx.grid(N)
    pk = np.stack([A[0, 0].ravel(), A[1, 1].ravel(), A[0, 1].ravel()])
    g.set_coeffs(pk, hg.HG_COEFF_PACKED)
    full = g.solve(hg.default_opts(tol=1e-12))
    only1 = g.solve(hg.default_opts(tol=1e-12, loads_mask=2))
    assert only1["iters"][0] == 0
    assert abs(only1["AH"][1, 1] - full["AH"][1, 1]) < 1e-12 * full["AH"][1, 1]
    assert only1["AH"][0, 0] == 0.0
    g.close()


# ------------------------------------------------------------------ errors
def test_error_codes(hg, ctx):
    with pytest.raises(hg.HGError) as e:
        ctx.grid((4, 5))
    assert e.value.status == -2
    with pytest.raises(hg.HGError) as e:
        ctx.grid((11, 5))          # prime factor 11
    assert e.value.status == -2
    g = ctx.grid((5, 5))
    with pytest.raises(hg.HGError) as e:
        g.solve()
    assert e.value.status == -11
    bad = np.array([[[1.0, 2.0], [2.0, 1.0]]])      # indefinite
    with pytest.raises(hg.HGError) as e:
        g.set_coeffs_phase(np.zeros((5, 5), np.uint8), bad)
    assert e.value.status == -3
    with pytest.raises(hg.HGError) as e:
        g.set_coeffs_phase(np.ones((5, 5), np.uint8), np.eye(2)[None])   # phase out of range
    assert e.value.status == -1
    g.set_coeffs_phase(np.zeros((5, 5), np.uint8), np.eye(2)[None] * 2.0)
    res = g.solve(hg.default_opts(max_iter=1), raise_on_error=False)
    assert res["status"] == 0           # homogeneous: zero right-hand side
    g.close()


def test_not_converged_status(hg, ctx):
    ms = W.circles_2d(n=45, count=5, r_lo=4, r_hi=8, contrast=1000.0, seed=2)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    res = g.solve(hg.default_opts(tol=1e-12, max_iter=3, check_every=2), raise_on_error=False)
    assert res["status"] == -5
    assert max(res["iters"]) == 3
    g.close()


# ------------------------------------------------------------------ serving
def test_submit_poll_matches_blocking(hg, ctx):
    probs = [W.circles_2d(n=45, count=4, r_lo=3, r_hi=8, contrast=c, seed=int(c)) for c in (10.0, 100.0)]
    probs.append(W.spheres_3d(n=15, count=3, r_lo=2, r_hi=4, seed=3, anisotropic=False, contrast=30.0))
    blocking, grids = [], []
    for ms in probs:
        g = ctx.grid(ms.N)
        g.set_coeffs_phase(ms.phase, ms.table)
        blocking.append(g.solve(hg.default_opts(tol=1e-10)))
        grids.append(g)
    tickets = [ctx.submit(g, hg.default_opts(tol=1e-10)) for g in grids]
    with pytest.raises(hg.HGError):
        ctx.submit(grids[0], hg.default_opts())        # borrowed
    out = [ctx.poll(t, timeout_us=-1) for t in tickets]
    for a, b in zip(out, blocking):
        assert a["status"] == 0
        # the scheduler batches requests with per-shape launch tiles: the same
        # iteration up to the rounding of the partial sums
        assert rel_max(a["AH"], b["AH"]) < 1e-10
    for g in grids:
        g.close()


def test_time_pass_in_graph(hg, ctx):
    ms = W.circles_2d(n=45, count=4, r_lo=3, r_hi=8, contrast=50.0, seed=3)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    plain = g.solve(hg.default_opts(tol=1e-8))
    for p in range(g.num_passes()):
        r = g.solve(hg.default_opts(tol=1e-8, time_pass=p, check_every=8))
        # one timed launch per graph chunk of 8 iterations that started active
        assert r["pass_launches"] == -(-max(r["iters"]) // 8)
        assert r["pass_ms_total"] > 0.0
        np.testing.assert_allclose(r["AH"], plain["AH"], rtol=1e-13)
    with pytest.raises(hg.HGError):
        g.solve(hg.default_opts(time_pass=g.num_passes()))
    g.close()


def test_scheduler_admission_by_memory_budget(hg):
    # A context whose budget holds the solver state of one 135x135 grid at a
    # time: the second request waits for the first, then reuses its memory.
    ms = [W.circles_2d(n=135, count=6, r_lo=5, r_hi=12, contrast=c, seed=int(c)) for c in (20.0, 40.0)]
    probe = hg.Context(0, use_torch_stream=False)
    g = probe.grid(ms[0].N)
    g.set_coeffs_phase(ms[0].phase, ms[0].table)
    want = [None, None]
    for k in range(2):
        g.set_coeffs_phase(ms[k].phase, ms[k].table)
        want[k] = g.solve(hg.default_opts(tol=1e-9, prec=hg.HG_MIXED))["AH"]
    g.close()
    probe.close()
    budget = 7 << 20           # one grid's FP64 + FP32 state at 135^2 is ~4.7 MiB
    ctx = hg.Context(0, mem_budget=budget, use_torch_stream=False)
    gs = []
    for m in ms:
        gg = ctx.grid(m.N)
        gg.set_coeffs_phase(m.phase, m.table)
        gs.append(gg)
    ts = [ctx.submit(gg, hg.default_opts(tol=1e-9, prec=hg.HG_MIXED)) for gg in gs]
    out = [ctx.poll(t, timeout_us=-1) for t in ts]
    for k in range(2):
        assert out[k]["status"] == 0
        # blocking mixed solves of square grids run the resident kernel, the
        # scheduler the batched pass kernels: equal to the method's tolerance
        assert rel_max(out[k]["AH"], want[k]) < 1e-6
    big = ctx.grid((405, 405))
    big.set_coeffs_phase(np.zeros((405, 405), np.uint8), np.eye(2)[None])
    t = ctx.submit(big, hg.default_opts())
    r = ctx.poll(t, timeout_us=-1)
    assert r["status"] == -4            # can never fit the budget
    ctx.close()


def test_cancel_queued_ticket(hg):
    ctx = hg.Context(0, use_torch_stream=False)
    ms = W.circles_2d(n=81, count=4, r_lo=4, r_hi=9, contrast=30.0, seed=1)
    gs = []
    for _ in range(3):
        g = ctx.grid(ms.N)
        g.set_coeffs_phase(ms.phase, ms.table)
        gs.append(g)
    ts = [ctx.submit(g, hg.default_opts(tol=1e-10)) for g in gs]
    ctx.cancel(ts[2])
    outs = [ctx.poll(t, timeout_us=-1) for t in ts]
    assert outs[0]["status"] == 0 and outs[1]["status"] == 0
    assert outs[2]["status"] in (0, -9)
    ctx.close()


# ------------------------------------------------------------ full-size workloads
def test_full_size_729_against_oracle_golden(hg, ctx):
    """The 729x729 workload in the configuration bench.py times (tol 1e-5,
    mixed and FP64) against the oracle's A_H at tol 1e-12."""
    gold = json.load(open(os.path.join(HERE, "golden", "circles_729_AH.json")))
    ref = np.array(gold["AH"])
    ms = W.circles_2d()
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    # the launch geometry bench.py runs: autotuned for each precision
    g.tune(hg.HG_MIXED, reps=20)
    g.tune(hg.HG_FP64, reps=4)
    mixed = g.solve(hg.default_opts(tol=1e-5, prec=hg.HG_MIXED, inner_tol=5e-6))
    fp64 = g.solve(hg.default_opts(tol=1e-5, prec=hg.HG_FP64))
    tight = g.solve(hg.default_opts(tol=1e-12, prec=hg.HG_FP64))
    assert rel_max(mixed["AH"], ref) < 1e-6
    assert rel_max(fp64["AH"], ref) < 1e-6
    assert rel_max(tight["AH"], ref) < 1e-8
    assert abs(tight["iters"][0] - gold["iters"][0]) <= 2
    g.close()


def test_full_size_135_cubed_sampled_and_properties(hg, ctx):
    """The 135^3 workload: one operator application against the oracle, and
    A_H symmetry, Voigt/Reuss bounds and energy = flux at full size."""
    ms = W.spheres_3d()
    N, d = ms.N, 3
    g = ctx.grid(N)
    g.set_coeffs_phase(ms.phase, ms.table)
    A = ms.full_field()
    u = np.random.default_rng(5).standard_normal((d,) + N)
    Ku = O.apply_K(A, u, N)
    np.testing.assert_allclose(g.apply(u, with_A=True), Ku, atol=1e-9)
    g.tune(hg.HG_MIXED, reps=4)   # the launch geometry bench.py runs
    assert rel_max(g.apply(u, with_A=True, prec=hg.HG_MIXED), Ku) < 1e-4
    res = g.solve(hg.default_opts(tol=1e-6, prec=hg.HG_MIXED, inner_tol=5e-7))
    assert res["status"] == 0
    AH = res["AH"]
    np.testing.assert_allclose(AH, AH.T, atol=1e-9 * np.max(np.abs(AH)))
    np.testing.assert_allclose(res["AH_flux"], AH, rtol=1e-4, atol=1e-6 * np.max(np.abs(AH)))
    f = ms.phase.mean()
    voigt = (1 - f) * ms.table[0] + f * ms.table[1]
    reuss = np.linalg.inv((1 - f) * np.linalg.inv(ms.table[0]) + f * np.linalg.inv(ms.table[1]))
    assert np.min(np.linalg.eigvalsh(voigt - AH)) > -1e-8 * np.max(np.abs(AH))
    assert np.min(np.linalg.eigvalsh(AH - reuss)) > -1e-8 * np.max(np.abs(AH))
    g.close()


def test_full_size_135_cubed_against_oracle_golden(hg, ctx):
    """The 135^3 workload (60 spheres, two random SPD phases, contrast 1000)
    against the oracle's A_H at tol 1e-12 (tests/golden/spheres_135_AH.json,
    written by make_golden.py --large3d): every entry of the FP64 path at tol
    1e-10 within 1e-8 and of the mixed path at bench.py's settings (tol 1e-5)
    within 1e-6, both relative to max |A_H| (Sec. 5.2 Eq. final_system)."""
    gold = json.load(open(os.path.join(HERE, "golden", "spheres_135_AH.json")))
    ref = np.array(gold["AH"])
    ms = W.spheres_3d()
    assert list(ms.N) == gold["N"] and abs(ms.meta["vf"] - gold["vf"]) < 1e-12
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    g.tune(hg.HG_MIXED, reps=4)    # the launch geometry bench.py runs
    fp64 = g.solve(hg.default_opts(tol=1e-10, prec=hg.HG_FP64))
    mixed = g.solve(hg.default_opts(tol=1e-5, prec=hg.HG_MIXED, inner_tol=5e-6))
    assert fp64["status"] == 0 and mixed["status"] == 0
    assert rel_max(fp64["AH"], ref) < 1e-8
    assert rel_max(mixed["AH"], ref) < 1e-6
    # the oracle's iteration counts at tol 1e-12 bound the FP64 path's at 1e-10
    assert all(a <= b + 2 for a, b in zip(fp64["iters"], gold["iters"]))
    g.close()


def test_mixed_high_contrast_accuracy(hg, ctx):
    """Contrast ~5e3: the mixed path (FP32 CG, FP64 refinement with the
    projection onto E_N) meets 1e-6 in A_H at tol 1e-5."""
    probs = W.batch_2d(count=40)
    ms = max((p for p in probs if p.N[0] <= 135), key=lambda p: p.meta["contrast"])
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    ref = g.solve(hg.default_opts(tol=1e-11))["AH"]
    mixed = g.solve(hg.default_opts(tol=1e-5, prec=hg.HG_MIXED, inner_tol=5e-6))
    assert ms.meta["contrast"] > 1e3
    assert rel_max(mixed["AH"], ref) < 1e-6
    g.close()
    # and against the oracle itself on one small batched problem
    small = next(p for p in probs if p.N[0] == 45)
    g = ctx.grid(small.N)
    g.set_coeffs_phase(small.phase, small.table)
    mixed = g.solve(hg.default_opts(tol=1e-8, prec=hg.HG_MIXED))
    oref = O.solve_AH(small.full_field(), small.N, tol=1e-12)["AH"]
    assert rel_max(mixed["AH"], oref) < 1e-6
    g.close()


def test_resetting_coefficients_between_solves(hg, ctx):
    # every change of the coefficient storage (phase map <-> field, another
    # phase count) drops the cached CG graphs that point at the old buffers
    N = (27, 27)
    rng = np.random.default_rng(31)
    m2 = W.Microstructure(N, (rng.random(N) < 0.3).astype(np.uint8), W.isotropic_table([1.0, 30.0], 2))
    m3 = W.Microstructure(N, rng.integers(0, 3, size=N).astype(np.uint8), W.isotropic_table([1.0, 5.0, 80.0], 2))
    A = W.random_spd_field(N, rng, 1.0, 20.0)
    g = ctx.grid(N)
    for prec in (hg.HG_FP64, hg.HG_MIXED):
        o = hg.default_opts(tol=1e-10, prec=prec)
        for kind, src in (("phase", m2), ("field", A), ("phase", m3), ("phase", m2), ("field", A)):
            if kind == "phase":
                g.set_coeffs_phase(src.phase, src.table)
                ref = O.solve_AH(src.full_field(), N, tol=1e-11)["AH"]
            else:
                g.set_coeffs_field(src)
                ref = O.solve_AH(src, N, tol=1e-11)["AH"]
            r = g.solve(o)
            assert rel_max(r["AH"], ref) <= (1e-8 if prec == hg.HG_FP64 else 1e-6)
    g.close()


def test_smooth_laminate_continuous_closed_form(hg, ctx):
    """a(x) = 2 + sin(pi x_1): the GaNi A_H on a 15 x 7 grid equals the
    continuous laminate's diag(sqrt(3), 2) to roundoff (Prop. GaNi, Sec. 4.3;
    the trapezoidal rule is exact to 2e-16 here), FP64 and mixed."""
    N = (15, 7)
    x = np.meshgrid(2.0 * np.arange(15) / 15, 2.0 * np.arange(7) / 7, indexing="ij")[0]
    A = np.zeros((2, 2) + N)
    A[0, 0] = A[1, 1] = 2.0 + np.sin(np.pi * x)
    g = ctx.grid(N)
    g.set_coeffs_field(A)
    exact = np.diag([np.sqrt(3.0), 2.0])
    r = g.solve(hg.default_opts(tol=1e-12))
    np.testing.assert_allclose(r["AH"], exact, atol=1e-11)
    r = g.solve(hg.default_opts(tol=1e-10, prec=hg.HG_MIXED))
    np.testing.assert_allclose(r["AH"], exact, atol=1e-7)
    g.close()


@pytest.mark.parametrize("N,Y", [((45, 27), (1.0, 2.5)), ((15, 9, 25), (1.0, 0.5, 2.0))])
def test_anisotropic_cell_solve_and_axis_relabelling(hg, ctx, N, Y):
    """Solves on a cell with unequal Y_a (xi_a = m_a / Y_a, Sec. 2) against the
    oracle, FP64 and mixed, and the same medium with its axes relabelled
    (grid, Y and tensor components together) giving P A_H P^T."""
    d = len(N)
    A = W.random_spd_field(N, np.random.default_rng(sum(N) + 1), 1.0, 20.0)
    ref = O.solve_AH(A, N, Y=Y, tol=1e-12)["AH"]
    g = ctx.grid(N, Y)
    g.set_coeffs_field(A)
    r64 = g.solve(hg.default_opts(tol=1e-11))
    r32 = g.solve(hg.default_opts(tol=1e-10, prec=hg.HG_MIXED))
    g.close()
    assert rel_max(r64["AH"], ref) < 1e-8
    assert rel_max(r32["AH"], ref) < 1e-6
    perm = tuple(range(1, d)) + (0,)
    Np = tuple(N[p] for p in perm)
    Yp = tuple(Y[p] for p in perm)
    Ap = np.ascontiguousarray(np.transpose(A, (0, 1) + tuple(2 + p for p in perm))[np.ix_(perm, perm)])
    gp = ctx.grid(Np, Yp)
    gp.set_coeffs_field(Ap)
    rp = gp.solve(hg.default_opts(tol=1e-11))
    gp.close()
    assert rel_max(rp["AH"], r64["AH"][np.ix_(perm, perm)]) < 1e-8
