"""hg_apply_noalloc: the operator G_N A_N u without device allocation.

Some callers cannot allocate device memory when they need the operator
(plug-ins whose device memory belongs to their host application's allocator,
real-time loops where cudaMalloc/cudaFree and their synchronisation are not
allowed).  The entry point keeps its scratch in a fixed static device array;
this test calls it twice in a row through the C ABI and checks both results
against hg_apply, the allocating entry point, at the tolerance of the other
FP64 operator tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _dev(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("N", [(45, 75), (15, 9, 25), (729, 243)])
def test_noalloc_matches_apply_twice(hg, N):
    import torch
    lib = hg.load()
    rng = np.random.default_rng(77)
    d = len(N)
    ms = W.Microstructure(N, (rng.random(N) < 0.3).astype(np.uint8), W.isotropic_table([1.0, 40.0], d))
    u = rng.standard_normal((d,) + N)
    ctx = hg.Context(0)
    g = ctx.grid(N)
    g.set_coeffs_phase(ms.phase, ms.table)
    ref = g.apply(u, with_A=True)
    g.close()
    ctx.close()

    dev = torch.device("cuda", 0)
    phase = torch.from_numpy(ms.phase).to(dev)
    table = torch.from_numpy(ms.table).to(dev)
    u_d = torch.from_numpy(u).to(dev)
    Narr = (ctypes.c_int * d)(*N)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for call in range(2):
        out = torch.full((d,) + N, float("nan"), dtype=torch.float64, device=dev)
        st = lib.hg_apply_noalloc(d, Narr, _dev(phase), ms.table.shape[0], _dev(table), _dev(u_d),
                                  _dev(out), stream)
        assert st == 0, hg.STATUS.get(st, st)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-11, err_msg=f"call {call}")


def test_noalloc_rejects_oversize_grid(hg):
    import torch
    lib = hg.load()
    dev = torch.device("cuda", 0)
    N = (135, 135, 135)
    d = 3
    dummy = torch.zeros(8, dtype=torch.float64, device=dev)
    ph = torch.zeros(8, dtype=torch.uint8, device=dev)
    Narr = (ctypes.c_int * d)(*N)
    st = lib.hg_apply_noalloc(d, Narr, _dev(ph), 1, _dev(dummy), _dev(dummy), _dev(dummy), None)
    assert st == -12
    assert "16 MiB" in lib.hg_strerror(st).decode()
    st = lib.hg_apply_noalloc(2, (ctypes.c_int * 2)(4, 5), _dev(ph), 1, _dev(dummy), _dev(dummy),
                              _dev(dummy), None)
    assert st == -2


def test_noalloc_out_of_range_phase_reads_last_entry(hg):
    """The phase map of hg_apply_noalloc is a device buffer the library does not
    read back: a byte >= n_phases must not read past the table; it is read as the
    last phase, so the result equals the one with that byte set to n_phases - 1."""
    import torch
    lib = hg.load()
    rng = np.random.default_rng(5)
    N = (45, 75)
    d = 2
    phase = (rng.random(N) < 0.3).astype(np.uint8)
    table = W.isotropic_table([1.0, 40.0], d)
    bad = phase.copy()
    bad[3, 7] = 200                      # out of range for a 2-entry table
    fixed = phase.copy()
    fixed[3, 7] = 1
    u = rng.standard_normal((d,) + N)
    dev = torch.device("cuda", 0)
    tab_d = torch.from_numpy(table).to(dev)
    u_d = torch.from_numpy(u).to(dev)
    Narr = (ctypes.c_int * d)(*N)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    outs = []
    for ph in (bad, fixed):
        ph_d = torch.from_numpy(ph).to(dev)
        out = torch.full((d,) + N, float("nan"), dtype=torch.float64, device=dev)
        st = lib.hg_apply_noalloc(d, Narr, _dev(ph_d), 2, _dev(tab_d), _dev(u_d), _dev(out), stream)
        assert st == 0, hg.STATUS.get(st, st)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    assert np.all(np.isfinite(outs[0]))
    np.testing.assert_array_equal(outs[0], outs[1])
