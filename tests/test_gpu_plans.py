"""The plan search space of the 1D step and the tuned-plan cache.

Every plan of the wide set -- four values per thread (n <= 1024) and the
alternative radix orders with sixteen (radix 8 throughout at n = 4096, the
small radix first otherwise) -- on a mixed-size batch against the FP64
oracle, in the resident and streaming modes (bitwise equal), with and without
the norm projection; the autotuner's cache: a miss runs the search and
records it, a second context with the same key reads the same plans without
timing anything and reproduces the tuned run bit for bit; plan validation."""
import json

import numpy as np
import pytest

from oracle import oracle as O
from paper_1007_3470_gb300 import workloads as W
from tests.gpu_helpers import TOL_C64, budget, need_gpu

pytestmark = pytest.mark.gpu

SIZES = (128, 256, 512, 1024, 2048, 4096)


def _solve(insts, psis, steps, plans, mode=None, project=False, occupancy=0):
    from paper_1007_3470_gb300 import hfs
    s = hfs.Solver(insts, precision="c64", chunk_steps=64)
    s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    s.set_norm_projection(project)
    for n, p in plans.items():
        s.set_plan(n, p)
    if mode is not None:
        s.set_mode(*mode)
    hfs.hfs_set_occupancy(s.h, occupancy)
    s.set_psi(psis)
    s.step(steps)
    out = s.get_psi()
    assert s.status() == hfs.HFS_OK
    s.close()
    return out


@pytest.mark.parametrize("project", [False, True])
@pytest.mark.parametrize("family", ["four", "alt"])
def test_wide_plans_match_oracle(family, project):
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=60, seed=11)
    steps = 24
    if family == "four":
        plans = {n: 4 for n in SIZES if n <= 1024}
    else:
        plans = {n: 16 | hfs.HFS_PLAN_ALT_ORDER for n in SIZES}
    res = _solve(insts, psis, steps, plans, project=project)
    stream = _solve(insts, psis, steps, plans, mode=(hfs.HFS_MODE_STREAMING, 5), project=project)
    one_cta = _solve(insts, psis, steps, plans, project=project, occupancy=1)
    assert np.array_equal(res, stream) and np.array_equal(res, one_cta)
    refs = O.run_batch([O.Problem(**i.as_dict()) for i in insts], psis, steps)
    off = np.concatenate([[0], np.cumsum([i.n[0] for i in insts])])
    worst = max(O.rel_l2(res[off[i]:off[i + 1]], r) for i, r in enumerate(refs))
    assert worst <= budget(TOL_C64, steps * 0.005), worst


def test_autotune_cache_hit_reproduces_tuned_run(tmp_path):
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=200, seed=12)
    path = str(tmp_path / "plans.json")
    runs = []
    for expect_hit in (False, True):
        s = hfs.Solver(insts, precision="c64", chunk_steps=32)
        s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
        s.set_norm_projection(True)
        plans = s.autotune(4, cache=path)
        assert s.tune_cache_hit == expect_hit
        s.set_psi(psis)
        s.step(32)
        runs.append((plans, s.get_psi()))
        s.close()
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])
    text = open(path).read()
    entry = json.loads(text)["entries"][0]
    assert entry["plans"] == runs[0][0] and "src=" in entry["key"] and "proj=1" in entry["key"]
    # a different key (projection off) misses and adds a second entry
    s = hfs.Solver(insts, precision="c64", chunk_steps=32)
    s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    s.autotune(4, cache=path)
    assert not s.tune_cache_hit
    s.close()
    assert len(json.loads(open(path).read())["entries"]) == 2


def test_plan_validation():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, _, _ = W.batch_1d(count=4, seed=13)
    s = hfs.Solver(insts, precision="c64")
    for n, p in ((2048, 4), (4096, 8), (512, 8 | hfs.HFS_PLAN_ALT_ORDER), (256, 12), (300, 16), (128, 0x200 | 16)):
        with pytest.raises(hfs.HfsError) as ei:
            s.set_plan(n, p)
        assert ei.value.code == 2, (n, p)
    s.close()
    d = hfs.Solver(insts, precision="c128")
    for p in (4, 16 | hfs.HFS_PLAN_ALT_ORDER):
        with pytest.raises(hfs.HfsError):
            d.set_plan(256, p)
    d.set_plan(256, 8)
    d.close()


def test_autotune_cache_unwritable_path_still_tunes(tmp_path):
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=64, seed=14)
    path = str(tmp_path / "missing_dir" / "plans.json")
    s = hfs.Solver(insts, precision="c64", chunk_steps=8)
    s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    plans = s.autotune(4, cache=path)
    assert not s.tune_cache_hit and any(plans)
    s.set_psi(psis)
    s.step(8)
    assert s.status() == hfs.HFS_OK
    s.close()
    import os
    assert not os.path.exists(path)
