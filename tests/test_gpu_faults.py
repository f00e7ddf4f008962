"""Failure detection on the GPU without a GPU fault.

* The tensor-core sampler bounds every mbarrier wait.  The host-side injector
  HM_FAULT_TC_STALL_AFTER=k makes one launch withhold its bulk copies and wait
  at most 1 ms: hm_compress must return HM_ETIMEOUT (its tensor memory freed,
  no copy left in flight), the same context must compress correctly
  afterwards, and a fresh context must give the same operator.
* Allocation failures: HM_FAULT_ALLOC_AFTER=k makes the library's device
  allocation after k successful ones fail once (before any CUDA call is made
  for it).  For allocation indices spread over a whole job (tree, compression,
  apply), the failing call returns HM_ENOMEM, the context is destroyable, and a
  fresh job afterwards gives the same result as an uninjected run.

Each case runs in a child process so that the injector (read when the library
is loaded) starts from a known count.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

JOB = r'''
import json, sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import hm_workloads as W
import paper_2205_03406_gb300 as hm

w = W.torus_laplace(n=6000, tol=1e-6, r=32)
pts = torch.from_numpy(w.points).cuda()
x = torch.from_numpy(np.random.default_rng(0).standard_normal((w.n, 2))).cuda()
op = hm.kernel_op(w.kernel)

def settings():
    return hm.Settings(d=3, leaf_size=w.leaf_size, r=w.r, oversample=w.oversample, tol=w.tol,
                       precision=hm.HM_MIXED_BF16X6, seed=w.seed)

def job(comp=None):
    comp = comp or hm.Compressor(settings())
    comp.tree_build(pts)
    info = comp.compress(op)
    return comp, comp.apply(x), info
'''


def run_child(body: str, env_extra: dict) -> dict:
    code = JOB.format(root=ROOT) + body
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_tc_wait_timeout_reported_and_context_recovers():
    res = run_child(r'''
comp = hm.Compressor(settings())
comp.tree_build(pts)
try:
    comp.compress(op)
    status, msg = 0, ""
except hm.HMError as e:
    status, msg = e.status, str(e)
_, y1, info = job(comp)          # the same context, after the timeout
c2, y2, _ = job()                 # a fresh context
d = float(torch.linalg.norm(y1 - y2) / torch.linalg.norm(y2))
print(json.dumps({"status": status, "msg": msg, "diff": d, "tc": info.bb_tc_levels,
                  "finite": bool(torch.isfinite(y1).all())}))
''', {"HM_FAULT_TC_STALL_AFTER": "0"})
    import paper_2205_03406_gb300 as hm
    assert res["status"] == hm.HM_ETIMEOUT, res
    assert "wait expired" in res["msg"], res
    assert res["tc"] > 0 and res["finite"] and res["diff"] <= 1e-12, res


def test_allocation_fault_sweep_over_a_whole_job():
    import paper_2205_03406_gb300 as hm
    base = run_child(r'''
a0 = hm.hm_get_info(hm.Compressor(settings()).ctx).device_allocs
comp, y, info = job()
print(json.dumps({"allocs": comp.info().device_allocs - a0, "y": y[:4, 0].tolist()}))
''', {})
    total = base["allocs"]
    assert total > 20, base
    ks = sorted(set([0, 1, 2, 5] + [int(total * f) for f in (0.1, 0.25, 0.4, 0.55, 0.7, 0.85)] + [total - 1]))
    for k in ks:
        res = run_child(r'''
comp = hm.Compressor(settings())
status, msg = 0, ""
try:
    comp.tree_build(pts)
    comp.compress(op)
    comp.apply(x)
except hm.HMError as e:
    status, msg = e.status, str(e)
rc = hm.hm_destroy(comp.ctx); comp.ctx = None
_, y, _ = job()
print(json.dumps({"status": status, "msg": msg, "destroy": rc, "y": y[:4, 0].tolist()}))
''', {"HM_FAULT_ALLOC_AFTER": str(k)})
        assert res["status"] == hm.HM_ENOMEM and "injected" in res["msg"], (k, res)
        assert res["destroy"] == hm.HM_OK, (k, res)
        assert res["y"] == base["y"], (k, res["y"], base["y"])
