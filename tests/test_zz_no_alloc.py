"""nb_regular_force_noalloc: the allocation-free entry point for callers that cannot
allocate device memory while they integrate (a host code whose own memory manager owns
the device, or a step loop that must not reach cudaMalloc/cudaFree).

It is called here through the C ABI (ctypes) and compared with the FP64 oracle directly and
with the context-based nb_regular_force (FP64) on the same inputs, with the FP64 parity bar
of the other GPU tests (1e-12 relative per row).  Two calls in a row on different inputs
check that the shared scratch array carries nothing stale from one call into the next.  The
cases reach every launch shape the entry point has: a few splits (small n), many splits
over a handful of rows (the wide reduction), one split at the 65536-row limit (the scratch
bound), and rows whose index is outside [0, n) (zeros).  This file is named so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def noalloc(lib, xp, vp, m, idx):
    n_i = idx.shape[0]
    acc = torch.empty((n_i, 3), dtype=torch.float64, device=DEV)
    jerk = torch.empty_like(acc)
    pot = torch.empty((n_i,), dtype=torch.float64, device=DEV)
    err = ctypes.create_string_buffer(256)
    s = lib.nb_regular_force_noalloc(xp.shape[0], xp.data_ptr(), vp.data_ptr(), m.data_ptr(), n_i, idx.data_ptr(),
                                     acc.data_ptr(), jerk.data_ptr(), pot.data_ptr(),
                                     torch.cuda.current_stream(DEV).cuda_stream, err, 256)
    assert s == 0, err.value.decode()
    return acc, jerk, pot


def with_context(cl, idx):
    from paper_1504_03687_gb300 import Context
    ctx = Context(cl.n, precision="fp64", nb_cap=8)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    res = ctx.regular_force(T(idx), 0.0, neighbours=False)
    ctx.sync()
    out = res.acc.cpu().numpy(), res.jerk.cpu().numpy(), res.pot.cpu().numpy()
    ctx.close()
    return out


def assert_rows_close(got, ref, tol=1e-12):
    g, r = got.reshape(len(got), -1), ref.reshape(len(ref), -1)
    d = np.linalg.norm(g - r, axis=1)
    s = np.linalg.norm(r, axis=1)
    assert np.all(d <= tol * np.maximum(s, 1e-3 * s.max())), float((d / s).max())


def oracle_rows(cl, idx):
    import oracle
    a, j, p, _, _ = oracle.regular_force(cl.x, cl.v, cl.m, idx, 0.0, cap=1, lists=False)
    return a, j, p


def test_noalloc_matches_regular_force_on_two_calls_in_a_row():
    from paper_1504_03687_gb300 import api
    lib = api.load_library()
    cases = []
    cl = W.plummer(4096, 71, masses="kroupa")
    cases.append((cl, np.random.default_rng(1).permutation(cl.n)[:700].astype(np.int32)))
    cl = W.plummer(3000, 72)
    cases.append((cl, np.random.default_rng(2).permutation(cl.n)[:33].astype(np.int32)))
    outs = [noalloc(lib, T(c.x), T(c.v), T(c.m), T(i)) for c, i in cases]  # two calls back to back
    torch.cuda.synchronize()
    for (c, i), got in zip(cases, outs):
        ref = with_context(c, i)
        orc = oracle_rows(c, i)
        for g, r, o in zip(got, ref, orc):
            assert_rows_close(g.cpu().numpy(), r)
            assert_rows_close(g.cpu().numpy(), o)


def test_noalloc_many_splits_and_the_row_limit():
    """n = 65536: 8 rows (64 source splits, the wide fixed-order reduction) and then all
    65536 rows (the 4 MiB scratch allows one split), back to back; against the context path
    on every row and the oracle on sampled rows."""
    from paper_1504_03687_gb300 import api
    lib = api.load_library()
    cl = W.plummer(65536, 73, masses="kroupa")
    few = np.random.default_rng(3).permutation(cl.n)[:8].astype(np.int32)
    full = np.random.default_rng(4).permutation(cl.n).astype(np.int32)
    xd, vd, md = T(cl.x), T(cl.v), T(cl.m)
    out_few = noalloc(lib, xd, vd, md, T(few))
    out_full = noalloc(lib, xd, vd, md, T(full))
    torch.cuda.synchronize()
    sel = np.sort(np.random.default_rng(5).choice(cl.n, 48, replace=False))
    for rows, got, sub in ((few, out_few, np.arange(8)), (full, out_full, sel)):
        ref = with_context(cl, rows)
        orc = oracle_rows(cl, rows[sub])
        for g, r, o in zip(got, ref, orc):
            g = g.cpu().numpy()
            assert_rows_close(g, r)
            assert_rows_close(g[sub], o)


def test_noalloc_out_of_range_rows_are_zero():
    from paper_1504_03687_gb300 import api
    lib = api.load_library()
    cl = W.plummer(2000, 74)
    idx = np.array([5, -1, 17, 2000, 1999, 0], np.int32)
    got = [g.cpu().numpy() for g in noalloc(lib, T(cl.x), T(cl.v), T(cl.m), T(idx))]
    torch.cuda.synchronize()
    ok = np.array([0, 2, 4, 5])
    orc = oracle_rows(cl, idx[ok])
    for g, o in zip(got, orc):
        assert not np.any(g[[1, 3]])
        assert_rows_close(g[ok], o)


def test_noalloc_rejects_blocks_beyond_its_scratch():
    from paper_1504_03687_gb300 import api
    lib = api.load_library()
    err = ctypes.create_string_buffer(256)
    s = lib.nb_regular_force_noalloc(100000, None, None, None, 65537, None, None, None, None, None, err, 256)
    assert s == api.NB_ERR_ARG
    assert b"65536" in err.value
