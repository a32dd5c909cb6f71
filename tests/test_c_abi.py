"""The boundary used from C, without Python: tests/abi_example.c compiles with -std=c11
-Wall -Wextra -Werror against include/nbgpu.h and links to libnbgpu.so (CPU); on a GPU it
predicts a seeded Plummer state and runs the regular force on an active block, and the
results agree with the oracle (FP64: 1e-12, lists exact)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import workloads as W
from paper_1504_03687_gb300 import _build, api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_example(tmp_path):
    api.load_library()  # builds libnbgpu.so in-tree if needed
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_example")
    libdir = os.path.dirname(_build.LIB)
    cmd = [cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "abi_example.c"), "-L", libdir, "-l:" + os.path.basename(_build.LIB),
           "-Wl,-rpath," + libdir, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_consumer_compiles_and_links(tmp_path):
    assert os.path.exists(build_example(tmp_path))


@pytest.mark.gpu
def test_c_consumer_matches_the_oracle(gpu_lib, tmp_path):
    exe = build_example(tmp_path)
    cl = W.plummer(3000, 41, masses="kroupa")
    a0, j0, tl = W.hermite_state(cl, seed=41, t_block=0.25)
    rs2 = float(W.neighbour_radius2(cl.x, 30, seed=41))
    idx = np.arange(0, 3000, 7, dtype=np.int32)
    t, cap = 0.25, 64
    src, dst = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(src, "wb") as f:
        f.write(np.int64(cl.n).tobytes())
        for q in (cl.x, cl.v, a0, j0, cl.m, tl):
            f.write(np.ascontiguousarray(q, dtype=np.float64).tobytes())
        f.write(np.int64(idx.size).tobytes())
        f.write(idx.tobytes())
        f.write(np.float64(rs2).tobytes() + np.float64(t).tobytes())
        f.write(np.int32(0).tobytes() + np.int32(cap).tobytes())  # FP64 context
    r = subprocess.run([exe, src, dst], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stderr
    raw = open(dst, "rb").read()
    k = idx.size
    o = 0
    acc = np.frombuffer(raw, np.float64, 3 * k, o).reshape(k, 3); o += 24 * k
    jerk = np.frombuffer(raw, np.float64, 3 * k, o).reshape(k, 3); o += 24 * k
    pot = np.frombuffer(raw, np.float64, k, o); o += 8 * k
    off = np.frombuffer(raw, np.int64, k + 1, o); o += 8 * (k + 1)
    cnt = np.frombuffer(raw, np.int32, k, o); o += 4 * k
    lists = np.frombuffer(raw, np.int32, int(off[-1]), o)
    xp, vp = oracle.predict(t, cl.x, cl.v, a0, j0, tl)
    ref = oracle.regular_force(xp, vp, cl.m, idx, rs2, cap=cap)
    for g, rf in ((acc, ref[0]), (jerk, ref[1])):
        e = np.linalg.norm(g - rf, axis=1) / np.linalg.norm(rf, axis=1)
        assert e.max() < 1e-12
    assert np.max(np.abs(pot - ref[2]) / np.abs(ref[2])) < 1e-12
    np.testing.assert_array_equal(cnt, ref[3])
    for q in range(k):
        np.testing.assert_array_equal(lists[off[q]:off[q + 1]], ref[4][q])
