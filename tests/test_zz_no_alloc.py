"""nb_regular_force_noalloc: the allocation-free entry point for callers that cannot
allocate device memory while they integrate (a host code whose own memory manager owns
the device, or a step loop that must not reach cudaMalloc/cudaFree).

It is called here through the C ABI (ctypes) and compared with the context-based
nb_regular_force (FP64) on the same inputs, with the FP64 parity bar of the other GPU
tests (1e-12 relative per row).  Two calls in a row on different inputs check that the
shared scratch array carries nothing stale from one call into the next.  This file is
named so that pytest collects it last.
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
        for g, r in zip(got, ref):
            assert_rows_close(g.cpu().numpy(), r)


def test_noalloc_rejects_blocks_beyond_its_scratch():
    from paper_1504_03687_gb300 import api
    lib = api.load_library()
    err = ctypes.create_string_buffer(256)
    s = lib.nb_regular_force_noalloc(100000, None, None, None, 65537, None, None, None, None, None, err, 256)
    assert s == api.NB_ERR_ARG
    assert b"65536" in err.value
