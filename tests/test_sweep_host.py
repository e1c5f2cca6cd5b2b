"""Host checks of the fused sweep subtrees (hdd_set_sweep_fusion): the plan's subtree
tables against the index arithmetic of the fused sweep kernels, compiled from
tests/sweep_tables_check.cpp with the host plan code (no GPU); the height in use as the
limit and the shared-memory budget allow; the launch count of an evaluation."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workload as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1708_02207_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("sweep") / "sweep_tables_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "sweep_tables_check.cpp"), os.path.join(CSRC, "plan.cpp"), "-o", exe],
                   check=True)
    return exe


@pytest.fixture(scope="module")
def hdd():
    from paper_1708_02207_gb300 import build, hdd as binding
    build.build()
    return binding


# (N, leaf, precision, fp64_top_levels, max_height): the benched grids, FP64 plans,
# irregular trees (N - 1 not a power of two), leaves that are not condensed
CASES = [(513, 4, 1, 0, 2), (513, 4, 1, 0, 6), (513, 4, 0, 0, 6), (513, 4, 1, 2, 3), (1025, 4, 1, 0, 2),
         (257, 4, 1, 0, 4), (129, 6, 1, 0, 6), (65, 3, 0, 0, 6), (50, 5, 0, 0, 6), (50, 5, 1, 0, 2),
         (33, 4, 1, 0, 1), (9, 2, 0, 0, 6), (100, 7, 1, 0, 6), (33, 8, 0, 0, 6)]


@pytest.mark.parametrize("N,leaf,prec,top,maxh", CASES)
def test_subtree_tables_match_the_kernels_indexing(checker, N, leaf, prec, top, maxh):
    out = subprocess.run([checker, str(N), str(leaf), str(prec), str(top), str(maxh)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    h = int(out.stdout.split()[1])
    assert 0 <= h <= maxh


def test_height_follows_the_limit(hdd):
    obs = w.obs_vertices(513, 16)
    plan = hdd.Plan(513, 4, None, obs, 0.01, device=-1, precision=hdd.HDD_MIXED_FP32, ir_max_iter=2)
    assert plan.info()["sweep_fuse_height"] == 2
    launches = {}
    for h in range(0, 7):
        plan.set_sweep_fusion(h)
        got = plan.info()["sweep_fuse_height"]
        assert got <= h
        launches[h] = plan.info()["launches_evaluate"]
    assert launches[0] > launches[1] > launches[2]   # each fused level saves a launch per full sweep
    with pytest.raises(hdd.HDDError):
        plan.set_sweep_fusion(7)
    with pytest.raises(hdd.HDDError):
        plan.set_sweep_fusion(-1)
    # 8 x 8-cell leaves keep their factors (49 interior vertices): no subtree qualifies
    p8 = hdd.Plan(65, 8, None, w.obs_vertices(65, 4), 0.01, device=-1)
    assert p8.info()["sweep_fuse_height"] == 0
