"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (written here, per particle i):
  FP64 path   e_i = |q_gpu - q_ref| / |q_ref| <= 1e-12 for acc, jerk (vector 2-norm)
              and pot, OR |q_gpu - q_ref| <= 1e-12 * sum_j |term_ij| (summation order
              differs, so particles whose sum cancels are bounded by the term sum);
              neighbour lists identical (same FP64 distance arithmetic).
  mixed path  median e_i <= 2e-6 and max e_i <= 1e-4 for acc, jerk and pot;
              neighbour sets identical outside a 1e-6 relative band around r_s.
  predictor   within 4 ulp of the sum of the term magnitudes of the oracle's term-by-term
              Taylor sum (the GPU evaluates the same polynomial in Horner form with FMA).
"""
import math
import warnings

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def rel_err(got, ref):
    if got.ndim == 2:
        return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    return np.abs(got - ref) / np.abs(ref)


def term_sums(xp, vp, m, idx):
    """sum_j |acc term|, sum_j |jerk term| and sum_j |pot term| for the rows idx."""
    out = np.zeros((len(idx), 3))
    for k, i in enumerate(idx):
        r = xp - xp[i]
        w = vp - vp[i]
        r2 = (r * r).sum(1)
        r2[i] = np.inf
        d = np.sqrt(r2)
        out[k, 0] = (m / r2).sum()
        out[k, 1] = (m * (np.linalg.norm(w, axis=1) / d ** 3 + 3 * np.abs((r * w).sum(1)) / d ** 4)).sum()
        out[k, 2] = (m / d).sum()
    return out


def check_fp64(res, ref, xp, vp, m, idx, tol=1e-12):
    acc, jerk, pot = (res.acc.cpu().numpy(), res.jerk.cpu().numpy(), res.pot.cpu().numpy()) \
        if torch.is_tensor(res.acc) else (res.acc, res.jerk, res.pot)
    errs = [rel_err(acc, ref[0]), rel_err(jerk, ref[1]), rel_err(pot, ref[2])]
    bad = np.nonzero((errs[0] > tol) | (errs[1] > tol) | (errs[2] > tol))[0]
    if bad.size:
        ts = term_sums(xp, vp, m, idx[bad])
        da = np.linalg.norm(acc[bad] - ref[0][bad], axis=1)
        dj = np.linalg.norm(jerk[bad] - ref[1][bad], axis=1)
        dp = np.abs(pot[bad] - ref[2][bad])
        assert np.all(da <= tol * ts[:, 0]), (bad, da / ts[:, 0])
        assert np.all(dj <= tol * ts[:, 1]), (bad, dj / ts[:, 1])
        assert np.all(dp <= tol * ts[:, 2])
    return bad.size


def check_mixed(res, ref):
    acc, jerk, pot = res.acc.cpu().numpy(), res.jerk.cpu().numpy(), res.pot.cpu().numpy()
    stats = {}
    for name, g, r in (("acc", acc, ref[0]), ("jerk", jerk, ref[1]), ("pot", pot, ref[2])):
        e = rel_err(g, r)
        stats[name] = (float(np.median(e)), float(e.max()))
        assert np.median(e) <= 2e-6, (name, stats[name])
        assert e.max() <= 1e-4, (name, stats[name])
    return stats


def lists_of(res):
    return res.neighbour_lists()


def check_lists_exact(res, ref_cnt, ref_lists, cap):
    cnt = res.nb_count.cpu().numpy()
    assert np.array_equal(cnt, ref_cnt)
    got = lists_of(res)
    for k, (a, b) in enumerate(zip(got, ref_lists)):
        assert np.array_equal(a, b[:cap]), k


def check_lists_band(res, xp, idx, rs2, ref_cnt, ref_lists, cap, band=1e-6):
    got = lists_of(res)
    cnt = res.nb_count.cpu().numpy()
    rs = math.sqrt(rs2)
    for k, i in enumerate(idx):
        a, b = set(got[k].tolist()), set(ref_lists[k].tolist())
        if a == b and cnt[k] == ref_cnt[k]:
            continue
        d = np.sqrt(((xp[list(a ^ b)] - xp[i]) ** 2).sum(1)) if (a ^ b) else np.zeros(0)
        assert np.all(np.abs(d - rs) <= band * rs), (k, d, rs)
        assert abs(int(cnt[k]) - int(ref_cnt[k])) <= len(a ^ b) + 2 * int(cnt[k] > cap)
        assert list(got[k]) == sorted(got[k])


def make_ctx(n, prec, cap=512):
    from paper_1504_03687_gb300 import Context
    return Context(n, precision=prec, nb_cap=cap)


# ------------------------------------------------------------------ predictor
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_predictor_within_rounding(gpu_lib, prec):
    """The GPU predictor (Horner, FMA) agrees with the oracle's term-by-term Taylor sum to
    within 4 ulp of the sum of the magnitudes of its terms."""
    cl, _ = W.plummer_1k_equal()
    steps = W.block_steps(cl, seed=0)
    a0, j0, tl = W.hermite_state(cl, seed=1, t_block=0.5, steps=steps)
    ctx = make_ctx(cl.n, prec)
    ctx.set_particles(T(cl.x), T(cl.v), T(a0), T(j0), T(cl.m), T(tl))
    ctx.predict(0.5)
    xp, vp = ctx.get_predicted()
    rx, rv = oracle.predict(0.5, cl.x, cl.v, a0, j0, tl)
    dt = (0.5 - tl)[:, None]
    eps = np.finfo(float).eps
    bx = np.abs(cl.x) + np.abs(cl.v * dt) + np.abs(a0 * dt ** 2 / 2) + np.abs(j0 * dt ** 3 / 6)
    bv = np.abs(cl.v) + np.abs(a0 * dt) + np.abs(j0 * dt ** 2 / 2)
    assert np.all(np.abs(xp.cpu().numpy() - rx) <= 4 * eps * bx)
    assert np.all(np.abs(vp.cpu().numpy() - rv) <= 4 * eps * bv)
    assert (xp.cpu().numpy() != rx).mean() < 0.5  # mostly bit-identical anyway


def expected_records(xp, vp, m, prec):
    """The j-records as the header defines them, from the FP64 predicted state, with numpy's
    FP64 -> FP32 conversion (round to nearest, ties to even)."""
    if prec == "fp64":
        out = np.zeros((len(m), 8))
        out[:, 0:3], out[:, 3], out[:, 4:7] = xp, m, vp
        return out.view(np.uint64)
    hi = (xp.view(np.uint64) & ~np.uint64(0x1FFFFFFF)).view(np.float64)
    with np.errstate(over="ignore"):
        out = np.zeros((len(m), 12), np.float32)
        out[:, 0:3], out[:, 3] = hi.astype(np.float32), m.astype(np.float32)
        out[:, 4:7] = (xp - hi).astype(np.float32)
        out[:, 8:11] = vp.astype(np.float32)
    return out.view(np.uint32)


def edge_values(rng, k):
    """FP64 values that take every branch of the record's rounding: zeros, values exact in
    FP32, ties and near-ties at the rounding bit of x (v, m) and of x - hi, remainders of
    every length, carries into the exponent, magnitudes outside the normal FP32 range."""
    e = rng.integers(1023 - 40, 1023 + 40, k).astype(np.uint64)
    mant = rng.integers(0, 1 << 52, k, dtype=np.uint64)
    sign = rng.integers(0, 2, k).astype(np.uint64) << np.uint64(63)
    kind = np.arange(k) % 6
    low = mant & np.uint64(0x1FFFFFFF)
    sh = rng.integers(1, 6, k).astype(np.uint64)
    tie_lo = ((rng.integers(0, 1 << 24, k, dtype=np.uint64) | np.uint64(1 << 23)) << sh) | (np.uint64(1) << (sh - np.uint64(1)))
    low = np.where(kind == 0, np.uint64(0x10000000), low)                       # tie of x -> float
    low = np.where(kind == 1, tie_lo & np.uint64(0x1FFFFFFF), low)             # tie of lo
    low = np.where(kind == 2, low >> rng.integers(0, 29, k).astype(np.uint64), low)  # short remainders
    low = np.where(kind == 3, np.uint64(0), low)                               # exact in FP32
    mant = (mant & ~np.uint64(0x1FFFFFFF)) | low
    mant = np.where(kind == 4, np.uint64(0xFFFFFF0000000) | (mant & np.uint64(0xFFFFFFF)), mant)  # carries
    b = sign | (e << np.uint64(52)) | mant
    v = b.view(np.float64).copy()
    special = np.array([0.0, -0.0, 1.5, -3.25, 1e-40, -1e-40, 1e-30, 3e-39, 3.4028235677973366e38, 1e39,
                        -1e39, 2.0 ** -126, 2.0 ** 127 * 1.9999999, 5e-324])
    v[:len(special)] = special
    return v


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_records_are_the_rounded_predicted_state(gpu_lib, prec):
    """The j-records the force kernels stream, bit for bit: from the predictor's output
    (Plummer 1k with a Hermite state) and from chosen edge values loaded as a predicted state
    (mixed: the hi/lo split and the FP32 roundings of v and m; fp64: plain copies)."""
    cl, _ = W.plummer_1k_equal()
    steps = W.block_steps(cl, seed=0)
    a0, j0, tl = W.hermite_state(cl, seed=1, t_block=0.5, steps=steps)
    ctx = make_ctx(cl.n, prec)
    ctx.set_particles(T(cl.x), T(cl.v), T(a0), T(j0), T(cl.m), T(tl))
    ctx.predict(0.5)
    xp, vp = (q.cpu().numpy() for q in ctx.get_predicted())
    got = ctx.get_records().cpu().numpy()
    assert np.array_equal(got.view(np.uint32 if prec == "mixed" else np.uint64), expected_records(xp, vp, cl.m, prec))
    rng = np.random.default_rng(11)
    n = 3000
    xq = edge_values(rng, 3 * n).reshape(n, 3)
    vq = edge_values(rng, 3 * n).reshape(n, 3)[rng.permutation(n)]
    mq = np.abs(edge_values(rng, n))
    ctx2 = make_ctx(n, prec)
    ctx2.set_predicted(T(xq), T(vq), T(mq))
    got = ctx2.get_records().cpu().numpy()
    assert np.array_equal(got.view(np.uint32 if prec == "mixed" else np.uint64), expected_records(xq, vq, mq, prec))
    ctx.close()
    ctx2.close()


# ------------------------------------------------------------------ Plummer 1024, full block
@pytest.fixture(scope="module")
def p1k():
    cl, rs2 = W.plummer_1k_equal()
    idx = np.arange(cl.n, dtype=np.int32)
    ref = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=512)
    return cl, rs2, idx, ref


def test_fp64_full_block_1k(gpu_lib, p1k):
    cl, rs2, idx, ref = p1k
    ctx = make_ctx(cl.n, "fp64")
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    res = ctx.regular_force(T(idx), rs2)
    assert ctx.sync() == 0
    check_fp64(res, ref, cl.x, cl.v, cl.m, idx)
    check_lists_exact(res, ref[3], ref[4], 512)


def test_mixed_full_block_1k(gpu_lib, p1k):
    cl, rs2, idx, ref = p1k
    ctx = make_ctx(cl.n, "mixed")
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    res = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    check_mixed(res, ref)
    check_lists_band(res, cl.x, idx, rs2, ref[3], ref[4], 512)


def test_host_buffers_match_device_buffers(gpu_lib, p1k):
    cl, rs2, idx, ref = p1k
    for prec in ("fp64", "mixed"):
        ctx = make_ctx(cl.n, prec)
        ctx.set_predicted(cl.x, cl.v, cl.m)  # host arrays
        host = ctx.regular_force(idx, rs2)
        dev = ctx.regular_force(T(idx), rs2)
        ctx.sync()
        np.testing.assert_array_equal(host.acc, dev.acc.cpu().numpy())
        np.testing.assert_array_equal(host.pot, dev.pot.cpu().numpy())
        np.testing.assert_array_equal(host.nb_off, dev.nb_off.cpu().numpy())
        tot = host.nb_off[-1]
        np.testing.assert_array_equal(host.nb_idx[:tot], dev.nb_idx[:tot].cpu().numpy())


# ------------------------------------------------------------------ Plummer 128k Kroupa
@pytest.fixture(scope="module")
def p128k():
    cl, rs2 = W.plummer_128k_kroupa()
    steps = W.block_steps(cl, seed=1)
    return cl, rs2, steps


@pytest.mark.parametrize("n_i", [1, 7, 16, 31, 33, 128, 1000, 1024])
def test_fp64_and_mixed_128k_blocks(gpu_lib, p128k, n_i):
    cl, rs2, steps = p128k
    idx = W.active_block(steps, n_i)
    ref = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=512)
    for prec in ("fp64", "mixed"):
        ctx = make_ctx(cl.n, prec)
        ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
        res = ctx.regular_force(T(idx), rs2)
        ctx.sync()
        if prec == "fp64":
            check_fp64(res, ref, cl.x, cl.v, cl.m, idx)
            check_lists_exact(res, ref[3], ref[4], 512)
        else:
            check_mixed(res, ref)
            check_lists_band(res, cl.x, idx, rs2, ref[3], ref[4], 512)
        ctx.close()


@pytest.mark.slow
def test_mixed_128k_large_block(gpu_lib, p128k):
    cl, rs2, steps = p128k
    idx = W.active_block(steps, 16384)
    ctx = make_ctx(cl.n, "mixed")
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    res = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    # oracle on a sample of the rows
    sel = np.random.default_rng(0).choice(idx.size, 512, replace=False)
    ref = oracle.regular_force(cl.x, cl.v, cl.m, idx[sel], rs2, cap=512)

    class Sub:
        pass
    sub = Sub()
    sub.acc, sub.jerk, sub.pot = res.acc[sel], res.jerk[sel], res.pot[sel]
    check_mixed(sub, ref)
    got = res.neighbour_lists()
    cnt = res.nb_count.cpu().numpy()
    for q, k in enumerate(sel):
        a, b = set(got[k].tolist()), set(ref[4][q].tolist())
        if a != b:
            d = np.sqrt(((cl.x[list(a ^ b)] - cl.x[idx[k]]) ** 2).sum(1))
            assert np.all(np.abs(d - math.sqrt(rs2)) <= 1e-6 * math.sqrt(rs2))
        assert abs(int(cnt[k]) - int(ref[3][q])) <= len(a ^ b)


# ------------------------------------------------------------------ neighbour caps and capacity
def test_cap_truncation_keeps_smallest_indices(gpu_lib, p1k):
    cl, rs2, idx, _ = p1k
    big = 9 * rs2  # many neighbours per particle
    ref = oracle.regular_force(cl.x, cl.v, cl.m, idx, big, cap=16)
    assert (ref[3] > 16).sum() > 100
    for prec in ("fp64", "mixed"):
        ctx = make_ctx(cl.n, prec, cap=16)
        ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
        res = ctx.regular_force(T(idx), big)
        with pytest.warns(Warning):
            ctx.sync()
        if prec == "fp64":
            check_lists_exact(res, ref[3], ref[4], 16)
        else:
            check_lists_band(res, cl.x, idx, big, ref[3], ref[4], 16)


def test_csr_capacity_too_small_is_reported(gpu_lib, p1k):
    from paper_1504_03687_gb300 import api
    cl, rs2, idx, ref = p1k
    ctx = make_ctx(cl.n, "fp64")
    ctx.set_predicted(cl.x, cl.v, cl.m)
    with pytest.warns(api.NBOverflow):
        res = ctx.regular_force(idx, rs2, nb_capacity=100)
    assert res.nb_off[-1] == sum(min(c, 512) for c in ref[3])
    flat = np.concatenate(ref[4])[:100]
    np.testing.assert_array_equal(res.nb_idx[:100], flat)


# ------------------------------------------------------------------ tiny blocks (one-launch epilogue)
@pytest.mark.parametrize("prec,plan", [("fp64", (0, 0, 20)), ("fp64", (0, 0, 8)), ("mixed", (1, 4, 24)),
                                       ("mixed", (1, 4, 5))])
def test_tiny_block_epilogue_is_bit_identical(gpu_lib, p128k, prec, plan):
    """Blocks of at most 8 rows take one launch for the partial-sum reduction and the
    neighbour CSR.  With a forced plan whose per-row partial sums do not depend on the other
    rows of the block, the rows of a 6-row block must carry the same bits (sums, counts,
    offsets within the row, lists) as the same rows inside a 100-row block, which takes the
    separate reduction and CSR kernels; the split counts reach both reduction orders (more
    than 16 splits: lanes over the splits and a butterfly; up to 16: split order)."""
    cl, rs2, steps = p128k
    idx = W.active_block(steps, 100)
    ctx = make_ctx(cl.n, prec)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    ctx.set_plan_override(*plan)
    big = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    small = ctx.regular_force(T(idx[:6]), rs2)
    ctx.sync()
    for a, b in ((small.acc, big.acc[:6]), (small.jerk, big.jerk[:6]), (small.pot, big.pot[:6]),
                 (small.nb_count, big.nb_count[:6])):
        assert torch.equal(a, b)
    ls, lb = lists_of(small), lists_of(big)
    for k in range(6):
        assert np.array_equal(ls[k], lb[k]), k
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tiny_block_cap_truncation_and_capacity(gpu_lib, p1k, prec):
    """A 5-row block with many neighbours a row, cap 16: lists keep the smallest indices and
    the true counts are reported; then a CSR buffer too small for the kept entries is
    reported, its offsets still those of the full lists and its first entries the lists'."""
    from paper_1504_03687_gb300 import api
    cl, rs2, idx, _ = p1k
    big = 9 * rs2
    sel = idx[[3, 100, 511, 700, 1023]]
    ref = oracle.regular_force(cl.x, cl.v, cl.m, sel, big, cap=16)
    assert (ref[3] > 16).all()
    ctx = make_ctx(cl.n, prec, cap=16)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    res = ctx.regular_force(T(sel), big)
    with pytest.warns(Warning):
        ctx.sync()
    if prec == "fp64":
        check_lists_exact(res, ref[3], ref[4], 16)
    else:
        check_lists_band(res, cl.x, sel, big, ref[3], ref[4], 16)
    with pytest.warns(api.NBOverflow):
        small = ctx.regular_force(T(sel), big, nb_capacity=40)
        ctx.sync()
    assert int(small.nb_off[-1]) == 5 * 16
    assert torch.equal(small.nb_off, res.nb_off)
    assert torch.equal(small.nb_idx[:40], res.nb_idx[:40])
    ctx.close()


def test_tiny_block_counts_only(gpu_lib, p1k):
    """Through the C ABI with no list buffer: a 7-row block gets the true counts and the
    offsets of the kept counts, as the oracle's lists give them, and no capacity report."""
    import ctypes
    cl, rs2, idx, _ = p1k
    sel = idx[::113][:7].astype(np.int32)
    ref = oracle.regular_force(cl.x, cl.v, cl.m, sel, rs2, cap=512)
    ctx = make_ctx(cl.n, "fp64")
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    d_idx, d_rs2 = T(sel), T(np.array([rs2]))
    acc = torch.empty((7, 3), dtype=torch.float64, device=DEV)
    jerk, pot = torch.empty_like(acc), torch.empty(7, dtype=torch.float64, device=DEV)
    off = torch.full((8,), -7, dtype=torch.int64, device=DEV)
    cnt = torch.full((7,), -7, dtype=torch.int32, device=DEV)
    ctx._bind_stream()
    s = ctx.lib.nb_regular_force(ctx.h, 7, d_idx.data_ptr(), d_rs2.data_ptr(), 1, acc.data_ptr(), jerk.data_ptr(),
                                 pot.data_ptr(), off.data_ptr(), None, 0, cnt.data_ptr(), 1)
    assert s == 0
    assert ctx.sync(allow_overflow=False) == 0
    np.testing.assert_array_equal(cnt.cpu().numpy(), ref[3])
    assert ref[3].max() <= 512
    kept = ref[3]
    np.testing.assert_array_equal(off.cpu().numpy(), np.concatenate([[0], np.cumsum(kept)]))
    check_fp64(type("R", (), {"acc": acc.cpu().numpy(), "jerk": jerk.cpu().numpy(), "pot": pot.cpu().numpy()}),
               ref, cl.x, cl.v, cl.m, sel)
    ctx.close()


def test_per_particle_rs2(gpu_lib, p1k):
    cl, rs2, idx, _ = p1k
    sel = idx[::5]
    rs2v = np.linspace(0.0, 2 * rs2, sel.size)
    ref = oracle.regular_force(cl.x, cl.v, cl.m, sel, rs2v, cap=512)
    ctx = make_ctx(cl.n, "fp64")
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    res = ctx.regular_force(T(sel), rs2v)
    ctx.sync()
    check_lists_exact(res, ref[3], ref[4], 512)


# ------------------------------------------------------------------ edge cases
def test_degenerate_sizes(gpu_lib):
    from paper_1504_03687_gb300 import api
    for prec in ("fp64", "mixed"):
        # n = 1: the only particle feels nothing
        ctx = make_ctx(4, prec)
        x = np.array([[0.1, 0.2, 0.3]])
        ctx.set_predicted(x, np.zeros((1, 3)), np.array([1.0]))
        res = ctx.regular_force(np.array([0], np.int32), 1.0)
        assert np.all(res.acc == 0) and np.all(res.pot == 0) and res.nb_count[0] == 0
        # n = 2: closed form
        x = np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 1.2]])
        v = np.array([[0.1, 0.0, 0.0], [0.0, 0.2, -0.1]])
        m = np.array([0.25, 0.75])
        ctx.set_predicted(x, v, m)
        res = ctx.regular_force(np.array([1, 0], np.int32), 10.0)
        ref = oracle.regular_force(x, v, m, np.array([1, 0], np.int32), 10.0)
        tol = 1e-14 if prec == "fp64" else 1e-6
        np.testing.assert_allclose(res.acc, ref[0], rtol=tol)
        np.testing.assert_allclose(res.jerk, ref[1], rtol=tol)
        np.testing.assert_allclose(res.pot, ref[2], rtol=tol)
        assert res.nb_off.tolist() == [0, 1, 2] and res.nb_idx[:2].tolist() == [0, 1]
        # n_i = 0
        res = ctx.regular_force(np.zeros(0, np.int32), 1.0)
        assert res.nb_off.tolist() == [0]
        # out-of-range index: rejected on the host immediately
        with pytest.raises(api.NBError) as e:
            ctx.regular_force(np.array([0, 2], np.int32), 1.0)
        assert e.value.status == api.NB_ERR_ARG
        # ... and by the device check (deferred to nb_sync) for device buffers
        ctx.regular_force(T(np.array([0, 5], np.int32)), 1.0)
        with pytest.raises(api.NBError) as e:
            ctx.sync()
        assert e.value.status == api.NB_ERR_ARG
        ctx.sync()  # the deferred status was consumed
        ctx.close()


def test_two_particles_1e_12_apart(gpu_lib):
    """Two distinct particles 1e-12 length units apart inside a 64-body Plummer sphere (the
    self-exclusion reading: distinct particles are never skipped, only j = i is).  FP64: every
    row, the close pair's included, within the FP64 bar of the oracle.  Mixed: the positions
    carry 2^-48 |x| in double-single, so the pair's separation (|x| about 0.6) is known to a few
    parts in 1e3 and its two rows are bounded by 1e-2; every other row keeps the mixed bars.
    Both find each other as neighbours; with the whole block (tiled kernels) and with just the
    pair (the j-streamed kernel)."""
    cl = W.plummer(64, 79)
    d = np.array([0.6, -0.48, 0.64]) * 1e-12
    x = np.concatenate([cl.x, cl.x[:1] + d])
    v = np.concatenate([cl.v, cl.v[:1] + np.array([[0.01, 0.02, -0.01]])])
    m = np.concatenate([cl.m, cl.m[:1]])
    n, close = x.shape[0], np.array([0, 64])
    assert 0 < np.linalg.norm(x[64] - x[0]) < 2e-12
    rs2 = float(W.neighbour_radius2(x, 8, seed=79))
    for rows in (np.arange(n, dtype=np.int32), close.astype(np.int32)):
        ref = oracle.regular_force(x, v, m, rows, rs2, cap=64)
        for prec in ("fp64", "mixed"):
            ctx = make_ctx(n, prec, cap=64)
            ctx.set_predicted(T(x), T(v), T(m))
            res = ctx.regular_force(T(rows), rs2)
            ctx.sync()
            if prec == "fp64":
                check_fp64(res, ref, x, v, m, rows)
            else:
                for g, r in ((res.acc, ref[0]), (res.jerk, ref[1]), (res.pot, ref[2])):
                    e = rel_err(g.cpu().numpy(), r)
                    pair = np.isin(rows, close)
                    assert e[pair].max() <= 1e-2, float(e[pair].max())
                    if (~pair).any():
                        assert np.median(e[~pair]) <= 2e-6 and e[~pair].max() <= 1e-4
            got = res.neighbour_lists()
            for k, i in enumerate(rows):
                if i in close:
                    assert (64 if i == 0 else 0) in set(got[k].tolist())
            ctx.close()


def test_call_order_and_argument_errors(gpu_lib):
    from paper_1504_03687_gb300 import api
    ctx = make_ctx(8, "mixed")
    with pytest.raises(api.NBError) as e:
        ctx.predict(0.0)
    assert e.value.status == api.NB_ERR_STATE
    with pytest.raises(api.NBError) as e:
        ctx.regular_force(np.zeros(1, np.int32), 1.0)
    assert e.value.status == api.NB_ERR_STATE
    with pytest.raises(api.NBError) as e:
        ctx.set_predicted(np.zeros((9, 3)), np.zeros((9, 3)), np.ones(9))
    assert e.value.status == api.NB_ERR_ARG
    ctx.close()


def test_duplicate_indices_give_identical_rows(gpu_lib, p1k):
    cl, rs2, _, _ = p1k
    idx = np.array([5, 17, 5, 900, 17], np.int32)
    ctx = make_ctx(cl.n, "mixed")
    ctx.set_predicted(cl.x, cl.v, cl.m)
    res = ctx.regular_force(idx, rs2)
    np.testing.assert_array_equal(res.acc[0], res.acc[2])
    np.testing.assert_array_equal(res.jerk[1], res.jerk[4])
    lists = res.neighbour_lists()
    np.testing.assert_array_equal(lists[0], lists[2])


def test_bitwise_reproducible(gpu_lib, p128k):
    cl, rs2, steps = p128k
    idx = T(W.active_block(steps, 4096))
    ctx = make_ctx(cl.n, "mixed")
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    a = ctx.regular_force(idx, rs2)
    b = ctx.regular_force(idx, rs2)
    ctx.sync()
    assert torch.equal(a.acc, b.acc) and torch.equal(a.jerk, b.jerk) and torch.equal(a.pot, b.pot)
    assert torch.equal(a.nb_off, b.nb_off)
    tot = int(a.nb_off[-1])
    assert torch.equal(a.nb_idx[:tot], b.nb_idx[:tot])


# ------------------------------------------------------------------ full size, 2^20
@pytest.fixture(scope="module")
def king1m():
    cl, rs2 = W.king_1m_binaries()
    steps = W.block_steps(cl, seed=2)
    return cl, rs2, steps


class _Rows:
    """Sampled rows of a force result: sums and the CSR lists of those rows only."""

    def __init__(self, res, sel):
        off = res.nb_off.cpu().numpy()
        self.acc, self.jerk, self.pot = res.acc[sel], res.jerk[sel], res.pot[sel]
        self.nb_count = res.nb_count[sel]
        self._lists = [res.nb_idx[off[k]:off[k + 1]].cpu().numpy() for k in sel]

    def neighbour_lists(self):
        return self._lists


@pytest.mark.slow
def test_million_body_sampled_rows(gpu_lib, king1m):
    """King W0=6, 2^20 bodies, the headline configuration: the mixed full block (all 2^20 rows,
    CSR sized so that no list is cut) and the FP64 2^10 block against the oracle on sampled
    rows, sums and neighbour lists (mixed: identical outside the 1e-6 band; FP64: identical)."""
    cl, rs2, steps = king1m
    n = cl.n
    rng = np.random.default_rng(7)
    for prec, n_i, n_s in (("mixed", n, 192), ("fp64", 1024, 96)):
        idx = np.arange(n, dtype=np.int32) if n_i == n else W.active_block(steps, n_i)
        ctx = make_ctx(n, prec)
        ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
        res = ctx.regular_force(T(idx), rs2, nb_capacity=n_i * 512)
        with warnings.catch_warnings(record=True) as caught:
            warnings.simplefilter("always")
            ctx.sync()
        # rows with more than nb_cap neighbours are cut at the cap (allowed); the CSR never is
        assert not any("capacity" in str(w.message) for w in caught), [str(w.message) for w in caught]
        assert int(res.nb_off[-1]) == int(torch.minimum(res.nb_count, torch.tensor(512, device=DEV)).sum())
        sel = np.sort(rng.choice(n_i, n_s, replace=False))
        ref = oracle.regular_force(cl.x, cl.v, cl.m, idx[sel], rs2, cap=512)
        sub = _Rows(res, sel)
        if prec == "mixed":
            check_mixed(sub, ref)
            check_lists_band(sub, cl.x, idx[sel], rs2, ref[3], ref[4], 512)
        else:
            sub.acc, sub.jerk, sub.pot = sub.acc.cpu().numpy(), sub.jerk.cpu().numpy(), sub.pot.cpu().numpy()
            check_fp64(sub, ref, cl.x, cl.v, cl.m, idx[sel])
            check_lists_exact(sub, ref[3], ref[4], 512)
        ctx.close()


# ------------------------------------------------------------------ every tiled kernel variant
@pytest.mark.parametrize("variant", list(range(20)))
def test_each_mixed_tiled_variant(gpu_lib, p128k, variant):
    """Every variant of the mixed tiled kernel (scalar and packed FP32x2, forced through the plan
    override) meets the mixed bar against the oracle and gives the same neighbour lists."""
    cl, rs2, steps = p128k
    idx = W.active_block(steps, 1000)
    ref = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=512)
    ctx = make_ctx(cl.n, "mixed")
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    ctx.set_plan_override(1, variant, 3)
    assert ctx.plan(cl.n, idx.size)["variant"] == variant
    res = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    check_mixed(res, ref)
    check_lists_band(res, cl.x, idx, rs2, ref[3], ref[4], 512)
    ctx.set_plan_override(-1)
    base = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    assert torch.equal(base.nb_off, res.nb_off)  # same FP32 distance arithmetic in every variant
    tot = int(base.nb_off[-1])
    assert torch.equal(base.nb_idx[:tot], res.nb_idx[:tot])
    ctx.close()


@pytest.mark.parametrize("variant", list(range(20)))
def test_each_mixed_tiled_variant_dense_lists(gpu_lib, p1k, variant):
    """Dense neighbourhoods (r_s^2 x 9, hundreds of neighbours a row) with nb_cap 16: many hits
    in every 32-j chunk of the packed kernels' interaction loop and lists cut at the cap inside a
    chunk, for every variant; the kept entries are the smallest indices, as the oracle's."""
    cl, rs2, idx, _ = p1k
    big = 9 * rs2
    ref = oracle.regular_force(cl.x, cl.v, cl.m, idx, big, cap=16)
    assert (ref[3] > 64).sum() > 100
    ctx = make_ctx(cl.n, "mixed", cap=16)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    ctx.set_plan_override(1, variant, 3)
    res = ctx.regular_force(T(idx), big)
    with pytest.warns(Warning):
        ctx.sync()
    check_mixed(res, ref)
    check_lists_band(res, cl.x, idx, big, ref[3], ref[4], 16)
    ctx.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("n_i,splits", [(1, 37), (3, 37), (6, 152), (16, 37), (21, 5)])
def test_jstream_variants(gpu_lib, p128k, variant, n_i, splits):
    """The j-streamed kernels of tiny blocks (1, 4, 8 and 2 rows a CTA, the last batch ragged;
    the 2-, 4- and 8-row forms packed FP32x2), forced at several j-split counts: the mixed bars
    against the oracle on every row, lists within the 1e-6 band of the oracle's, and lists
    identical to those of the packed tiled kernel with one split."""
    cl, rs2, steps = p128k
    idx = W.active_block(steps, n_i)
    ref = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=512)
    ctx = make_ctx(cl.n, "mixed")
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    ctx.set_plan_override(2, variant, splits)
    assert ctx.plan(cl.n, n_i)["kernel"] == 2
    res = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    check_mixed(res, ref)
    check_lists_band(res, cl.x, idx, rs2, ref[3], ref[4], 512)
    ctx.set_plan_override(1, 4, 1)
    one = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    assert torch.equal(one.nb_off, res.nb_off) and torch.equal(one.nb_count, res.nb_count)
    tot = int(one.nb_off[-1])
    assert torch.equal(one.nb_idx[:tot], res.nb_idx[:tot])
    ctx.close()


@pytest.mark.parametrize("prec,variant", [("mixed", 4), ("mixed", 10), ("mixed", 15), ("fp64", 0)])
@pytest.mark.parametrize("n_i,splits", [(2000, 40), (600, 40), (6000, 24)])
def test_many_splits(gpu_lib, p128k, prec, variant, n_i, splits):
    """Many j-splits (the partial-sum reductions of more than 16 splits: a warp per component
    for up to 1024 rows, a warp per row up to 4096, a thread per row above), over kernels that
    write their partial sums and segments at the row index and at the spatial-order position:
    the bars against the oracle, and lists identical to the one-split call's."""
    cl, rs2, steps = p128k
    idx = W.active_block(steps, n_i)
    sel = np.sort(np.random.default_rng(n_i).choice(n_i, 96, replace=False))
    ref = oracle.regular_force(cl.x, cl.v, cl.m, idx[sel], rs2, cap=512)
    ctx = make_ctx(cl.n, prec)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    kernel = 1 if prec == "mixed" else 0
    ctx.set_plan_override(kernel, variant, splits)
    assert ctx.plan(cl.n, n_i)["splits"] == splits
    res = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    ctx.set_plan_override(kernel, variant, 1)
    one = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    assert torch.equal(one.nb_off, res.nb_off) and torch.equal(one.nb_count, res.nb_count)
    tot = int(one.nb_off[-1])
    assert torch.equal(one.nb_idx[:tot], res.nb_idx[:tot])

    class _Rows:
        pass
    sub = _Rows()
    sub.acc, sub.jerk, sub.pot = res.acc[sel], res.jerk[sel], res.pot[sel]
    if prec == "mixed":
        check_mixed(sub, ref)
    else:
        sub.acc, sub.jerk, sub.pot = sub.acc.cpu().numpy(), sub.jerk.cpu().numpy(), sub.pot.cpu().numpy()
        check_fp64(sub, ref, cl.x, cl.v, cl.m, idx[sel])
    ctx.close()


def test_mixed_far_from_the_origin(gpu_lib):
    """The cluster translated by (1e4, -2e4, 3e3) length units (a star cluster far from the
    coordinate origin): forces do not change, but single-precision coordinates would lose about
    four digits of every separation there. The double-single differences (and the anchored
    kernel's separations from an anchor among the rows) keep the mixed path within its bars
    against the oracle of the shifted state, with the same neighbour lists."""
    cl = W.plummer(4096, 77, masses="kroupa")
    rs2 = float(W.neighbour_radius2(cl.x, 50, seed=77))
    x = cl.x + np.array([1.0e4, -2.0e4, 3.0e3])
    idx = np.arange(0, 4096, 3, dtype=np.int32)
    ref = oracle.regular_force(x, cl.v, cl.m, idx, rs2, cap=512)
    ctx = make_ctx(cl.n, "mixed")
    ctx.set_predicted(T(x), T(cl.v), T(cl.m))
    for variant in (None, 4, 10):  # the automatic plan, the packed and the anchored kernel
        if variant is not None:
            ctx.set_plan_override(1, variant, 0)
        res = ctx.regular_force(T(idx), rs2)
        ctx.sync()
        check_mixed(res, ref)
        check_lists_band(res, x, idx, rs2, ref[3], ref[4], 512)
    ctx.close()
