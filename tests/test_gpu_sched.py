"""The request scheduler's cross-request batching (hg_submit / hg_poll).

Requests for the standard CG (Sec. 5.3 on Eq. final_system) join a rolling
batch: every tick steps all of them together, one launch per pass and grid
shape.  The contract tested here: a request's result is the same alone and in
any mix (bitwise, since each shape's launch tiles are fixed and a batched
launch computes every request's tiles as alone), it meets the oracle's A_H at
the method's tolerance, and requests that arrive while others run are admitted
between ticks.
"""
import time

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _mix():
    """2D and 3D two-phase requests of several sizes and contrasts."""
    probs = []
    for k, (n, c) in enumerate([(45, 20.0), (81, 300.0), (45, 1000.0), (135, 50.0), (81, 10.0)]):
        probs.append(W.circles_2d(n=n, count=max(3, n // 20), r_lo=n / 30, r_hi=n / 10, contrast=c, seed=100 + k))
    for k, (n, c) in enumerate([(15, 40.0), (27, 200.0)]):
        probs.append(W.spheres_3d(n=n, count=4, r_lo=n / 10, r_hi=n / 5, seed=200 + k, anisotropic=k == 1,
                                  contrast=c))
    return probs


def _solve_alone(hg, ms, opts):
    ctx = hg.Context(0, use_torch_stream=False)
    g = ctx.grid(ms.N)
    g.set_coeffs_phase(ms.phase, ms.table)
    r = ctx.poll(ctx.submit(g, opts), timeout_us=-1)
    ctx.close()
    return r


@pytest.mark.parametrize("prec", [1, 0])
def test_same_result_alone_and_in_the_mix(hg, prec):
    opts = hg.default_opts(tol=1e-8, prec=prec)
    probs = _mix()
    alone = [_solve_alone(hg, ms, opts) for ms in probs]
    ctx = hg.Context(0, use_torch_stream=False)
    grids = []
    for ms in probs + probs[:3]:      # the mix holds copies of some requests as well
        g = ctx.grid(ms.N)
        g.set_coeffs_phase(ms.phase, ms.table)
        grids.append(g)
    tickets = [ctx.submit(g, opts) for g in grids]
    out = [ctx.poll(t, timeout_us=-1) for t in tickets]
    for k, ms in enumerate(probs):
        assert out[k]["status"] == 0 and alone[k]["status"] == 0
        np.testing.assert_array_equal(out[k]["AH"], alone[k]["AH"])
        assert out[k]["iters"] == alone[k]["iters"]
    for k in range(3):
        np.testing.assert_array_equal(out[len(probs) + k]["AH"], alone[k]["AH"])
    # and each meets the oracle at the method's tolerance
    for k in (0, 2, 5):
        ms = probs[k]
        ref = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)["AH"]
        assert rel_max(out[k]["AH"], ref) < (1e-6 if prec else 1e-8)
    ctx.close()


def test_requests_arriving_while_others_run(hg):
    """A large request runs; small 2D and 3D mixed requests arrive while it is
    on the GPU and join its ticks; all results equal their solo ones."""
    opts = hg.default_opts(tol=1e-9, prec=hg.HG_MIXED)
    big = W.circles_2d(n=243, count=12, r_lo=8, r_hi=24, contrast=500.0, seed=9)
    small = _mix()
    ref_big = _solve_alone(hg, big, opts)["AH"]
    ref_small = [_solve_alone(hg, ms, opts)["AH"] for ms in small]
    ctx = hg.Context(0, use_torch_stream=False)
    gb = ctx.grid(big.N)
    gb.set_coeffs_phase(big.phase, big.table)
    gs = []
    for ms in small:
        g = ctx.grid(ms.N)
        g.set_coeffs_phase(ms.phase, ms.table)
        gs.append(g)
    tb = ctx.submit(gb, opts)
    tickets = []
    for g in gs:
        time.sleep(0.0003)
        tickets.append(ctx.submit(g, opts))
    outs = [ctx.poll(t, timeout_us=-1) for t in tickets]
    rb = ctx.poll(tb, timeout_us=-1)
    assert rb["status"] == 0
    np.testing.assert_array_equal(rb["AH"], ref_big)
    for o, r in zip(outs, ref_small):
        assert o["status"] == 0
        np.testing.assert_array_equal(o["AH"], r)
    ctx.close()


def test_batched_and_per_request_jobs_together(hg):
    """Requests the rolling batch does not take (Moulinec-Suquet, the dual
    formulation, a general A0) run as per-request jobs beside it."""
    ms = W.circles_2d(n=45, count=4, r_lo=3, r_hi=8, contrast=30.0, seed=5)
    A = ms.full_field()
    ref = O.solve_AH(A, ms.N, tol=1e-12)["AH"]
    ctx = hg.Context(0, use_torch_stream=False)
    kinds = [hg.default_opts(tol=1e-9, prec=hg.HG_MIXED),
             hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, method=hg.HG_MS, max_iter=20000),
             hg.default_opts(tol=1e-9, prec=hg.HG_MIXED, formulation=hg.HG_DUAL),
             hg.default_opts(tol=1e-9, prec=hg.HG_FP64, A0=np.array([[2.0, 0.3], [0.3, 1.0]])),
             hg.default_opts(tol=1e-9, prec=hg.HG_FP64)]
    grids, tickets = [], []
    for o in kinds:
        g = ctx.grid(ms.N)
        g.set_coeffs_phase(ms.phase, ms.table)
        grids.append(g)
        tickets.append(ctx.submit(g, o))
    for t in tickets:
        r = ctx.poll(t, timeout_us=-1)
        assert r["status"] == 0
        assert rel_max(r["AH"], ref) < 1e-6
    ctx.close()


def test_cancel_a_running_batched_request(hg):
    opts = hg.default_opts(tol=1e-12, prec=hg.HG_MIXED)
    probs = _mix()[:4]
    ctx = hg.Context(0, use_torch_stream=False)
    grids = []
    for ms in probs:
        g = ctx.grid(ms.N)
        g.set_coeffs_phase(ms.phase, ms.table)
        grids.append(g)
    ts = [ctx.submit(g, opts) for g in grids]
    ctx.cancel(ts[1])
    outs = [ctx.poll(t, timeout_us=-1) for t in ts]
    assert outs[1]["status"] in (0, -9)
    for k in (0, 2, 3):
        assert outs[k]["status"] == 0
    # the cancelled request's grid is free again
    r = ctx.poll(ctx.submit(grids[1], opts), timeout_us=-1)
    assert r["status"] == 0
    ctx.close()
