"""Error handling under injected host-side failures (nb_inject_fault / NB_FAULT): a failed
scratch allocation is reported as NB_ERR_OOM and the call can be retried; a failed stream
synchronisation or status read is reported as NB_ERR_CUDA and leaves the context unusable
(NB_ERR_STATE) until it is freed, after which a new context computes correct results.  The
failures are simulated by the library's host layer; nothing faults, traps or hangs the GPU."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def setup(n=3000):
    from paper_1504_03687_gb300 import Context
    cl = W.plummer(n, 111)
    rs2 = float(W.neighbour_radius2(cl.x, 30, seed=111))
    ctx = Context(n, precision="fp64", nb_cap=64)
    ctx.set_predicted(cl.x, cl.v, cl.m)
    return cl, rs2, ctx


def check(cl, rs2, idx, res):
    ref = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=64, lists=False)
    e = np.linalg.norm(res.acc - ref[0], axis=1) / np.linalg.norm(ref[0], axis=1)
    assert e.max() < 1e-12
    np.testing.assert_array_equal(res.nb_count, ref[3])


def test_allocation_failure_is_reported_and_retryable(gpu_lib):
    from paper_1504_03687_gb300 import NBError
    from paper_1504_03687_gb300.api import NB_ERR_OOM, NB_FAULT_ALLOC
    cl, rs2, ctx = setup()
    idx = np.arange(0, 3000, 7, dtype=np.int32)
    ctx.inject_fault(NB_FAULT_ALLOC, 0)
    with pytest.raises(NBError) as e:
        ctx.regular_force(idx, rs2)
    assert e.value.status == NB_ERR_OOM and "out of memory" in str(e.value)
    check(cl, rs2, idx, ctx.regular_force(idx, rs2))  # the fault fired once: the retry works
    # countdown: the second allocation after arming fails (a larger block grows the scratch)
    ctx.inject_fault(NB_FAULT_ALLOC, 1)
    big = np.arange(3000, dtype=np.int32)
    with pytest.raises(NBError) as e:
        ctx.regular_force(big, rs2)
    assert e.value.status == NB_ERR_OOM
    check(cl, rs2, big, ctx.regular_force(big, rs2))
    ctx.close()


@pytest.mark.parametrize("kind", ["sync", "status"])
def test_sync_and_status_failures_poison_the_context(gpu_lib, kind):
    from paper_1504_03687_gb300 import NBError
    from paper_1504_03687_gb300.api import NB_ERR_CUDA, NB_ERR_STATE, NB_FAULT_STATUS, NB_FAULT_SYNC
    cl, rs2, ctx = setup()
    idx = np.arange(0, 3000, 5, dtype=np.int32)
    check(cl, rs2, idx, ctx.regular_force(idx, rs2))
    ctx.inject_fault(NB_FAULT_SYNC if kind == "sync" else NB_FAULT_STATUS, 0)
    with pytest.raises(NBError) as e:
        ctx.regular_force(idx, rs2)  # host mode: synchronises, then reads the status
    assert e.value.status == NB_ERR_CUDA
    with pytest.raises(NBError) as e:
        ctx.regular_force(idx, rs2)
    assert e.value.status == NB_ERR_STATE and "unusable" in str(e.value)
    ctx.close()
    cl, rs2, ctx2 = setup()
    check(cl, rs2, idx, ctx2.regular_force(idx, rs2))
    ctx2.close()


def test_fault_armed_from_the_environment(gpu_lib):
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import numpy as np, workloads as W\n"
        "from paper_1504_03687_gb300 import Context, NBError\n"
        "cl = W.plummer(500, 3)\n"
        "ctx = Context(500, precision='mixed', nb_cap=32)\n"
        "ctx.set_predicted(cl.x, cl.v, cl.m)\n"
        "try:\n"
        "    ctx.regular_force(np.arange(50, dtype=np.int32), 0.01)\n"
        "    print('no fault')\n"
        "except NBError as e:\n"
        "    print('status', e.status)\n" % ROOT)
    env = dict(os.environ, NB_FAULT="alloc:0")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "status 3" in out.stdout  # NB_ERR_OOM
