"""GPU checks of the autotuner (lb_autotune): every candidate runs, the winner is
the fastest timed candidate, the heuristic's pick is timed first, the winner's
plan and y agree with the oracle, and the cache returns the same choice."""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import assert_within_bound, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbmod():
    import paper_2301_04792_gb300 as lb
    lb.build()
    lb.autotune_cache_clear()
    return lb


def test_autotune_powerlaw_picks_fastest_and_matches_oracle(lbmod):
    m = W.powerlaw(50_000, 50_000, 1_000_000, lmax=40_000, plant_long=False, seed=21)
    x = W.x_for(m)
    y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
    rp, ci, v, xd = to_dev(m.rp, m.ci, m.v, x)
    plan, rep = lbmod.autotune(rp, ci, v, xd, num_cols=m.num_cols, reps=3, use_cache=False)
    cands = rep["candidates"]
    # merge-path warp x3 static + x2 row-weighted + x2 look-back, CTA x4 (buffers are aligned),
    # thread-mapped as printed and staged, group-mapped x7
    assert len(cands) == 20
    assert all(c["status"] == 0 for c in cands), cands
    assert all(c["ms"] > 0 and c["reps"] in (1, 3) for c in cands)
    assert rep["heuristic"] == "merge_path_ipt8_v0" and cands[0]["name"] == "merge_path_ipt8_v0"
    best_ms = min(c["ms"] for c in cands)
    assert rep["best"] == next(c["name"] for c in cands if c["ms"] == best_ms)
    assert not rep["from_cache"]
    info = plan.info()
    assert info["schedule"] == rep["best_schedule"]
    assert_within_bound(rep["y"].cpu().numpy(), y64, b, "autotune y")
    y2 = plan.spmv(ci, v, xd)
    assert_within_bound(y2.cpu().numpy(), y64, b, "winner plan y")
    # algorithmic bytes / time
    c0 = cands[0]
    nbytes = 8 * m.nnz + 4 * (m.num_rows + 1) + 4 * m.num_cols + 4 * m.num_rows
    assert abs(c0["gbps"] - nbytes / (c0["ms"] * 1e-3) / 1e9) <= 1e-3 * c0["gbps"]


def test_autotune_cache_hit_returns_same_choice(lbmod):
    m = W.powerlaw(20_000, 20_000, 300_000, lmax=10_000, plant_long=False, seed=22)
    x = W.x_for(m)
    y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
    rp, ci, v, xd = to_dev(m.rp, m.ci, m.v, x)
    _, r1 = lbmod.autotune(rp, ci, v, xd, num_cols=m.num_cols, reps=2)
    p2, r2 = lbmod.autotune(rp, ci, v, xd, num_cols=m.num_cols, reps=2)
    assert not r1["from_cache"] and r2["from_cache"]
    assert r1["best"] == r2["best"] and r1["best_opts"] == r2["best_opts"]
    assert_within_bound(r2["y"].cpu().numpy(), y64, b, "cached winner y")
    # another column pattern on the same rows is another key
    ci2 = ci.flip(0).contiguous()
    _, r3 = lbmod.autotune(rp, ci2, v, xd, num_cols=m.num_cols, reps=2)
    assert not r3["from_cache"]
    lbmod.autotune_cache_clear()
    _, r4 = lbmod.autotune(rp, ci, v, xd, num_cols=m.num_cols, reps=2)
    assert not r4["from_cache"]


def test_autotune_small_matrix_prior_is_thread_mapped(lbmod):
    m = W.plain(400, 400, 10, seed=1)  # 4,000 nonzeros, 400 rows: the Sec. 6.2 rule picks thread-mapped
    x = W.x_for(m)
    y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
    rp, ci, v, xd = to_dev(m.rp, m.ci, m.v, x)
    _, rep = lbmod.autotune(rp, ci, v, xd, num_cols=m.num_cols, use_cache=False)
    assert rep["candidates"][0]["name"] == "thread_mapped" and rep["heuristic"] == "thread_mapped"
    assert_within_bound(rep["y"].cpu().numpy(), y64, b, "small autotune y")


def test_autotune_family_mask_and_edge_cases(lbmod):
    import torch
    from paper_2301_04792_gb300 import _lib
    m = W.powerlaw(5000, 4000, 60_000, lmax=3000, plant_long=False, seed=23)
    x = W.x_for(m)
    y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
    rp, ci, v, xd = to_dev(m.rp, m.ci, m.v, x)
    _, rep = lbmod.autotune(rp, ci, v, xd, num_cols=m.num_cols, families=_lib.TUNE_GROUP, use_cache=False)
    assert [c["group_size"] for c in rep["candidates"]] == [4, 8, 16, 32, 64, 128, 256]
    assert_within_bound(rep["y"].cpu().numpy(), y64, b, "group-only y")
    # unaligned buffers: the bulk-copy variant is not a candidate
    ci_u = torch.empty(m.nnz + 1, dtype=torch.int32, device="cuda")[1:]
    v_u = torch.empty(m.nnz + 1, dtype=torch.float32, device="cuda")[1:]
    ci_u.copy_(ci)
    v_u.copy_(v)
    _, rep = lbmod.autotune(rp, ci_u, v_u, xd, num_cols=m.num_cols, families=_lib.TUNE_MP_CTA, use_cache=False)
    assert [c["mp_variant"] for c in rep["candidates"]] == [1, 1]
    assert_within_bound(rep["y"].cpu().numpy(), y64, b, "unaligned y")
    # all rows empty: every candidate runs, y = 0
    e = W.from_lengths(np.zeros(300, np.int64), 200, seed=2)
    rp_e = torch.from_numpy(e.rp).cuda()
    ci_e = torch.zeros(0, dtype=torch.int32, device="cuda")
    v_e = torch.zeros(0, dtype=torch.float32, device="cuda")
    x_e = torch.ones(200, device="cuda")
    _, rep = lbmod.autotune(rp_e, ci_e, v_e, x_e, num_cols=200, use_cache=False)
    assert torch.equal(rep["y"].cpu(), torch.zeros(300))
    # num_cols missing with atoms present: refused before any launch
    with pytest.raises(_lib.LBError):
        lbmod.autotune(rp, ci, v, xd, num_cols=0, use_cache=False)


_CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
import torch, workloads as W, paper_2301_04792_gb300 as lb
m = W.powerlaw(30_000, 30_000, 500_000, lmax=20_000, plant_long=False, seed=24)
rp, ci, v, x = (torch.from_numpy(a).cuda() for a in (m.rp, m.ci, m.v, W.x_for(m)))
_, rep = lb.autotune(rp, ci, v, x, num_cols=m.num_cols, reps=2)
print(json.dumps({{"from_cache": rep["from_cache"], "best": rep["best"], "ms": [c["ms"] for c in rep["candidates"]],
                  "size": lb.autotune_cache_size()}}))
"""


def test_autotune_cache_file_skips_timing_in_a_second_process(lbmod, tmp_path):
    """With LB_AUTOTUNE_CACHE set, the first process times every candidate and
    writes the file; a second process finds the entry and times nothing, with
    the same winner and the same table."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = tmp_path / "tune.jsonl"
    env = dict(os.environ, LB_AUTOTUNE_CACHE=str(path))
    runs = []
    for _ in range(2):
        out = subprocess.run([sys.executable, "-c", _CHILD.format(root=root)], env=env, capture_output=True, text=True,
                             timeout=600)
        assert out.returncode == 0, out.stderr[-2000:]
        runs.append(json.loads(out.stdout.strip().splitlines()[-1]))
    assert path.exists() and len(path.read_text().splitlines()) == 1
    assert not runs[0]["from_cache"] and runs[1]["from_cache"]
    assert runs[0]["best"] == runs[1]["best"]
    assert runs[0]["ms"] == runs[1]["ms"]
    assert runs[1]["size"] == 1
