"""The device Ahmad-Cohen integrator (nb_ac_*) against the reference AC integrator of the
oracle (orc_ac_run), both started from the same cluster and run for the same block steps.

Bars: FP64 context — block times, steps, regular-step times, list lengths and lists
identical, r_s^2 to 1e-12 relative (one library power function each side), positions and
velocities to 1e-9 relative after 300 block steps (the predictor and the summation order
differ at rounding level and the differences grow with the orbits); mixed context — energy
conserved to 2e-5 at t = 1/4 and within a factor 4 of the reference run's own error, or
below 2e-6."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def make(n, prec, cap):
    from paper_1504_03687_gb300 import Context
    return Context(n, precision=prec, nb_cap=cap)


def test_ac_fp64_follows_the_reference_step_for_step(gpu_lib):
    from paper_1504_03687_gb300 import ACIntegrator
    cl, rs2 = W.plummer_1k_equal()
    K = 300
    kw = dict(eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=0.125, nb_opt=50)
    ox, ov, ors2, info = oracle.ac_run(cl.m, cl.x, cl.v, rs2, 100.0, cap=256, max_blocks=K, **kw)
    assert info["rc"] == -2 and info["blocks"] == K
    ctx = make(cl.n, "fp64", 256)
    ac = ACIntegrator(ctx, cl.m, cl.x, cl.v, rs2, level_max=40, **kw)
    n_act = n_reg = 0
    for _ in range(K):
        t, na, nr = ac.step()
        n_act += na
        n_reg += nr
    g = ac.get()
    assert n_act == info["irregular_steps"] and n_reg == info["regular_steps"]
    for k in ("t", "dt", "DT", "T"):
        np.testing.assert_array_equal(g[k], info[k], err_msg=k)
    np.testing.assert_array_equal(g["nb_count"], info["nb_count"])
    for i in range(cl.n):
        np.testing.assert_array_equal(g["nb_lists"][i, :g["nb_count"][i]], info["nb_lists"][i])
    np.testing.assert_allclose(g["rs2"], ors2, rtol=1e-12)
    np.testing.assert_allclose(g["x"], ox, rtol=1e-9, atol=1e-9 * np.abs(ox).max())
    np.testing.assert_allclose(g["v"], ov, rtol=1e-9, atol=1e-9 * np.abs(ov).max())
    ac.close()
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ac_device_driven_run_equals_step_by_step(gpu_lib, prec):
    """nb_ac_run drives the block steps without a regular subset from the device, in batches
    the host enqueues without synchronising in between; stepping one block at a time through
    nb_ac_step (the host path) for the same number of block steps gives bit-identical
    positions, velocities, times, steps, lists and counters."""
    from paper_1504_03687_gb300 import ACIntegrator
    cl = W.plummer(4096, 105, masses="kroupa")
    rs2 = W.neighbour_radius2(cl.x, 50, seed=105)
    kw = dict(eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=1.0 / 16, nb_opt=50)
    ctx = make(cl.n, prec, 128)
    a = ACIntegrator(ctx, cl.m, cl.x, cl.v, rs2, **kw)
    sa = a.run(1.0 / 16, max_blocks=1000000)
    ga = a.get()
    a.close()
    assert sa["blocks"] > 100 and sa["regular_steps"] > 0
    b = ACIntegrator(ctx, cl.m, cl.x, cl.v, rs2, **kw)
    n_act = n_reg = 0
    for _ in range(sa["blocks"]):
        _, na, nr = b.step()
        n_act += na
        n_reg += nr
    gb = b.get()
    b.close()
    ctx.close()
    assert n_act == sa["irregular_steps"] and n_reg == sa["regular_steps"]
    for k in ("x", "v", "t", "dt", "DT", "T", "rs2", "nb_count"):
        np.testing.assert_array_equal(ga[k], gb[k], err_msg=k)
    for i in range(cl.n):
        c = ga["nb_count"][i]
        np.testing.assert_array_equal(ga["nb_lists"][i, :c], gb["nb_lists"][i, :c])
    assert np.all(ga["t"] == 1.0 / 16)


def test_ac_every_particle_a_neighbour_is_plain_hermite(gpu_lib):
    """r_s covering the system, fixed: the device AC run is the plain block-step Hermite run
    (the reference's reduction, pinned against the Kepler orbit), to rounding."""
    import ctypes
    from paper_1504_03687_gb300 import ACIntegrator
    cl = W.plummer(256, 102)
    xh, vh = cl.x.copy(), cl.v.copy()
    st = np.zeros(4)
    lib = oracle._load()
    assert lib.orc_hermite_run(256, cl.m.ctypes.data, xh.ctypes.data, vh.ctypes.data, ctypes.c_double(0.125),
                               ctypes.c_double(0.02), ctypes.c_double(0.01), ctypes.c_double(0.125),
                               ctypes.c_double(0.0), ctypes.c_int64(0), st.ctypes.data) == 0
    ctx = make(256, "fp64", 256)
    ac = ACIntegrator(ctx, cl.m, cl.x, cl.v, 1e300, eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=0.125, nb_opt=0)
    s = ac.run(0.125, max_blocks=20000)
    g = ac.get()
    assert s["blocks"] == int(st[0]) and s["irregular_steps"] == int(st[1])
    assert np.all(g["t"] == 0.125)
    np.testing.assert_allclose(g["x"], xh, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(g["v"], vh, rtol=1e-10, atol=1e-12)
    ac.close()
    ctx.close()


def test_ac_mixed_conserves_energy(gpu_lib):
    from paper_1504_03687_gb300 import ACIntegrator
    cl = W.plummer(4096, 103)
    rs2 = W.neighbour_radius2(cl.x, 50, seed=103)
    kw = dict(eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=0.125, nb_opt=50)
    E0 = sum(oracle.energy(cl.m, cl.x, cl.v))
    ox, ov, _, info = oracle.ac_run(cl.m, cl.x, cl.v, rs2, 0.25, cap=256, **kw)
    e_ref = abs(sum(oracle.energy(cl.m, ox, ov)) - E0) / abs(E0)
    ctx = make(cl.n, "mixed", 256)
    ac = ACIntegrator(ctx, cl.m, cl.x, cl.v, rs2, **kw)
    s = ac.run(0.25, max_blocks=200000)
    g = ac.get()
    assert np.all(g["t"] == 0.25) and np.all(g["dt"] <= g["DT"])
    e = abs(sum(oracle.energy(cl.m, g["x"], g["v"])) - E0) / abs(E0)
    assert e < 2e-5 and (e < 4 * e_ref or e < 2e-6), (e, e_ref)
    assert s["regular_steps"] < 0.5 * s["irregular_steps"]
    assert 35 <= np.median(g["nb_count"]) <= 70
    ac.close()
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ac_checkpoint_resume_is_bitwise(gpu_lib, prec):
    """Run 120 block steps, checkpoint, run 150 more; resume the checkpoint on a fresh
    context and run the same 150: every output identical bit for bit."""
    from paper_1504_03687_gb300 import ACIntegrator
    cl = W.plummer(3000, 105, masses="kroupa")
    rs2 = W.neighbour_radius2(cl.x, 40, seed=105)
    kw = dict(eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=0.125, nb_opt=40)
    ctx = make(cl.n, prec, 128)
    ac = ACIntegrator(ctx, cl.m, cl.x, cl.v, rs2, **kw)
    for _ in range(120):
        ac.step()
    blob = ac.save()
    times = [ac.step()[0] for _ in range(150)]
    a = ac.get()
    ac.close()
    ctx.close()
    ctx2 = make(cl.n + 7, prec, 128)  # any context with room, the same precision and cap
    ac2 = ACIntegrator.restore(ctx2, blob)
    times2 = [ac2.step()[0] for _ in range(150)]
    b = ac2.get()
    assert times == times2
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    ac2.close()
    ctx2.close()


def test_hermite_run_to_t1_energy_drift(gpu_lib):
    """The 1024-body Plummer sphere (equal masses) integrated to t = 1 with eta = 0.02 on the
    device (the AC integrator with r_s covering everything is the plain block-step Hermite
    integrator): the FP64 drift stays below 1e-6 and within a factor 2 of the oracle run's
    own drift; the mixed-precision drift is below 1e-6 too."""
    import ctypes
    from paper_1504_03687_gb300 import ACIntegrator
    cl, _ = W.plummer_1k_equal()
    E0 = sum(oracle.energy(cl.m, cl.x, cl.v))
    xh, vh = cl.x.copy(), cl.v.copy()
    st = np.zeros(4)
    lib = oracle._load()
    assert lib.orc_hermite_run(cl.n, cl.m.ctypes.data, xh.ctypes.data, vh.ctypes.data, ctypes.c_double(1.0),
                               ctypes.c_double(0.02), ctypes.c_double(0.01), ctypes.c_double(0.125),
                               ctypes.c_double(0.0), ctypes.c_int64(0), st.ctypes.data) == 0
    e_ref = abs(sum(oracle.energy(cl.m, xh, vh)) - E0) / abs(E0)
    for prec in ("fp64", "mixed"):
        ctx = make(cl.n, prec, cl.n)
        ac = ACIntegrator(ctx, cl.m, cl.x, cl.v, 1e300, eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=0.125,
                          nb_opt=0)
        ac.run(1.0, max_blocks=100000)
        g = ac.get()
        assert np.all(g["t"] == 1.0)
        e = abs(sum(oracle.energy(cl.m, g["x"], g["v"])) - E0) / abs(E0)
        assert e < 1e-6, (prec, e, e_ref)
        if prec == "fp64":
            assert e < 2 * e_ref + 1e-9, (e, e_ref)
        ac.close()
        ctx.close()


def test_context_irregular_force_sees_the_integrated_state(gpu_lib):
    """The integrator rewrites the context's state arrays in place: the context's own irregular
    force (predict-on-load form, which caches per-particle state records) must use the state
    after the steps, whether or not it was called before them. Two identical runs, one with a
    call before the steps that fills the cache, give identical results after them (FP64)."""
    from paper_1504_03687_gb300 import ACIntegrator
    cl = W.plummer(2000, 107, masses="kroupa")
    rs2 = W.neighbour_radius2(cl.x, 40, seed=107)
    kw = dict(eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=0.125, nb_opt=40)
    idx = np.arange(0, 2000, 200, dtype=np.int32)  # 10 rows: 10 x 128 < N, the cached-record form

    def csr(g):
        cnt = g["nb_count"][idx]
        off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
        flat = np.concatenate([g["nb_lists"][i, :c] for i, c in zip(idx, cnt)]).astype(np.int32)
        return off, flat

    out = []
    for warm in (True, False):
        ctx = make(cl.n, "fp64", 128)
        ac = ACIntegrator(ctx, cl.m, cl.x, cl.v, rs2, **kw)
        if warm:
            ctx.irregular_force(0.0, idx, *csr(ac.get()))
        t = 0.0
        for _ in range(60):
            t = ac.step()[0]
        res = ctx.irregular_force(t, idx, *csr(ac.get()))
        out.append(res)
        ac.close()
        ctx.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
