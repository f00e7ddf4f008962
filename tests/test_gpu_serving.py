"""Serving (hm_server_*): jobs of differing size, geometry and kernel admitted
by device-memory footprint, compressed concurrently and kept resident.

* Every job's operator from the server equals the same job compressed alone
  with hm_compress (the kernels are deterministic; checked to 1e-12).
* Admission respects the byte budget: with a budget for one job at a time
  the jobs run one by one; with room for several they overlap.
* A job larger than the whole budget is refused; released jobs give their
  reservation back; matvec latencies are recorded.
"""
import numpy as np
import pytest

import hm_workloads as W

from gpu_helpers import hm

pytestmark = pytest.mark.gpu

MIXED = 1


def settings(w):
    m = hm()
    return m.Settings(d=w.d, leaf_size=w.leaf_size, r=w.r, oversample=w.oversample, tol=w.tol,
                      precision=MIXED, seed=w.seed)


def alone(w, x):
    import torch
    m = hm()
    comp = m.Compressor(settings(w))
    comp.tree_build(torch.from_numpy(w.points).cuda())
    comp.compress(m.kernel_op(w.kernel))
    y0, y1 = comp.apply(x, 0), comp.apply(x, 1)
    comp.close()
    return y0, y1


def test_jobs_in_the_mix_equal_jobs_alone():
    import torch
    m = hm()
    jobs = W.serving_jobs(9, n_min=3000, n_max=20000)
    srv = m.Server(slots=4)
    ids = [srv.submit(w.points, settings(w), m.kernel_op(w.kernel)) for w in jobs]
    for jid in ids:
        st = srv.wait(jid, timeout=300.0)
        assert st.state == m.HM_JOB_READY and st.info.bb_tc_levels > 0
    info = srv.info()
    assert info.completed == len(jobs) and info.failed == 0
    assert info.max_running >= 2, "no two jobs were compressed at the same time"
    for w, jid in zip(jobs, ids):
        x = torch.from_numpy(np.random.default_rng(w.seed).standard_normal((w.n, 2))).cuda()
        r0, r1 = alone(w, x)
        for trans, ref in ((0, r0), (1, r1)):
            y = srv.apply(jid, x, trans)
            e = float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref))
            assert e <= 1e-12, (w.name, trans, e)
    info = srv.info()
    assert info.applies == 2 * len(jobs) and info.apply_p99_s >= info.apply_p50_s > 0
    assert info.job_p99_s >= info.job_p50_s > 0 and info.jobs_per_s > 0
    for jid in ids:
        srv.release(jid)
    info = srv.info()
    assert info.reserved == 0 and info.released == len(jobs)
    srv.close()


def test_admission_by_footprint():
    m = hm()
    w = W.torus_laplace(n=8000, tol=1e-6, r=32)
    probe = m.Server(slots=2)
    est = probe.wait(probe.submit(w.points, settings(w), m.kernel_op(w.kernel)), 300.0).estimate_bytes
    probe.close()
    # room for one job's estimate only: the four jobs are compressed one at a time
    srv = m.Server(slots=4, hbm_budget=int(1.5 * est))
    ids = [srv.submit(w.points, settings(w), m.kernel_op(w.kernel)) for _ in range(4)]
    for jid in ids:
        assert srv.wait(jid, 300.0).state == m.HM_JOB_READY
    info = srv.info()
    assert info.max_running == 1 and info.max_reserved <= info.budget, (info.max_running, info.max_reserved)
    # a job whose estimate exceeds the whole budget is refused
    big = W.torus_laplace(n=200_000, tol=1e-6, r=32)
    with pytest.raises(m.HMError) as ei:
        srv.submit(big.points, settings(big), m.kernel_op(big.kernel))
    assert ei.value.status == m.HM_ENOTSUP
    # a queued or running job cannot be released; an unknown id is an error
    with pytest.raises(m.HMError):
        srv.release(12345)
    srv.close()
