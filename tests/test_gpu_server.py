"""The continuous-batching server: results identical alone and in a mix,
FIFO admission under the HBM budget, oversized jobs, cancellation, and
injected allocation refusals (host-side fault injection)."""
import time

import numpy as np
import pytest

from paper_2602_13553_gb300 import inputs
from tests._gpu import assert_split_close, pimd  # noqa: F401
from tests.test_gpu_batch import MIX

pytestmark = pytest.mark.gpu


def submit(srv, r, nsteps):
    return srv.submit(r["x0"], r["mass"], T=r["T"], dt=r["dt"], nsteps=nsteps, ff=r["ff"], box=r["box"],
                      seed=r["seed"])


def wait(srv, jobs, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(jobs):
        for j in jobs:
            if j not in out:
                res = srv.poll(j)
                if res is not None:
                    out[j] = res
        assert time.time() - t0 < timeout, "jobs did not finish"
        time.sleep(0.005)
    return out


def test_result_same_alone_and_in_mix(pimd):
    srv = pimd.Server(8 << 30, max_replicas=16, chunk_steps=25)
    ja = submit(srv, MIX[2], 130)
    alone = wait(srv, [ja])[ja]
    srv.close()
    srv = pimd.Server(8 << 30, max_replicas=16, chunk_steps=25)
    early = [submit(srv, MIX[0], 300), submit(srv, MIX[4], 90)]
    time.sleep(0.05)                      # the mix is already running when the job arrives
    jb = submit(srv, MIX[2], 130)
    late = [submit(srv, r, 60 + 10 * i) for i, r in enumerate(MIX[3:])]
    res = wait(srv, early + [jb] + late)
    mixed = res[jb]
    assert mixed["step"] == alone["step"] == 130
    for k in ("H", "K_CV", "P_CV", "K_PR", "T_ring"):
        assert abs(mixed[k] - alone[k]) <= 1e-12 * abs(alone[k]), k
    st = srv.stats()
    assert st["completed"] == 2 + 1 + len(late) and st["failed"] == 0
    srv.close()


def test_served_job_agrees_with_oracle(orc, pimd):
    """A job submitted into a running mix is served to completion; its final
    state and every estimator are compared with the oracle run of the same
    inputs for the same number of steps, at the split-precision bars."""
    srv = pimd.Server(8 << 30, max_replicas=16, chunk_steps=25, keep_state=True)
    early = [submit(srv, MIX[0], 300), submit(srv, MIX[5], 200)]
    time.sleep(0.05)
    jobs = {submit(srv, MIX[2], 60): MIX[2], submit(srv, MIX[3], 45): MIX[3]}
    res = wait(srv, early + list(jobs))
    for j, r in jobs.items():
        x, v, st = srv.get_state(j)
        n = 60 if r is MIX[2] else 45
        assert st == n and res[j]["step"] == n
        c = orc.Sim(r["x0"], r["mass"], T=r["T"], dt=r["dt"], potential=1, ff=r["ff"], box=r["box"],
                    seed=r["seed"])
        c.run(n)
        assert_split_close(x, v, res[j], c, c.estimators(), "served job %d" % j)
        with pytest.raises(pimd.PimdError) as ei:   # the kept copy is released once fetched
            srv.get_state(j)
        assert ei.value.status == 7
    srv.close()


def test_serving_trace_jobs_agree_with_oracle(orc, pimd):
    """Jobs of the serving workload itself (the Poisson trace's boxes, drawn
    on the perturbed lattice, its temperatures, seeds and bead counts),
    served together at a reduced step count, against the oracle: the
    trace's first jobs small enough for the oracle to follow in seconds."""
    trace = inputs.serving_trace(2000, 50.0, seed=1)
    picks = [j for j in trace if j.nmol <= 160 and j.P <= 32][:5]
    assert len(picks) == 5
    srv = pimd.Server(8 << 30, max_replicas=8, chunk_steps=10, keep_state=True)
    jobs = {}
    for j in picks:
        L = inputs.box_length(j.nmol)
        x0, mass = inputs.water_lattice_box(j.nmol, L, j.P, j.seed % (2 ** 31), jitter=0.02)
        kw = dict(T=j.T, dt=5e-4, ff=inputs.water_ff_for_box(L), box=(L, L, L), seed=j.seed)
        jobs[srv.submit(x0, mass, nsteps=25, **kw)] = (x0, mass, kw)
    res = wait(srv, list(jobs))
    for jid, (x0, mass, kw) in jobs.items():
        x, v, st = srv.get_state(jid)
        assert st == 25
        c = orc.Sim(x0, mass, potential=1, **kw)
        c.run(25)
        assert_split_close(x, v, res[jid], c, c.estimators(), "trace job %d (P = %d)" % (jid, x0.shape[0]))
    srv.close()


def test_small_jobs_pass_a_head_job_that_does_not_fit(pimd):
    """A head job that must wait for memory does not idle the budget: a later
    job that fits is admitted while the head waits."""
    big, small = MIX[2], MIX[0]
    nb = pimd.replica_bytes(big["x0"].shape[1], big["x0"].shape[0])
    ns = pimd.replica_bytes(small["x0"].shape[1], small["x0"].shape[0])
    assert ns < nb
    srv = pimd.Server(nb + ns, max_replicas=8, chunk_steps=20)
    first = submit(srv, big, 2000)      # holds nb of the budget for a while
    head = submit(srv, big, 20)         # cannot fit until the first finishes
    later = submit(srv, small, 20)      # fits beside the first
    wait(srv, [first, head, later])
    t_first, t_head, t_later = srv.times(first), srv.times(head), srv.times(later)
    assert t_later[1] < t_first[2] <= t_head[1] + 1e-9
    srv.close()


def test_fifo_admission_under_budget(pimd):
    r = MIX[1]
    need = pimd.replica_bytes(r["x0"].shape[1], r["x0"].shape[0])
    srv = pimd.Server(int(need * 1.5), max_replicas=8, chunk_steps=20)
    jobs = [submit(srv, r, 40) for _ in range(3)]
    wait(srv, jobs)
    times = [srv.times(j) for j in jobs]
    for (s0, a0, f0), (s1, a1, f1) in zip(times, times[1:]):
        assert a1 >= f0 - 1e-9          # one job at a time fits the budget
    srv.close()


def test_oversized_job_and_cancel(pimd):
    r = MIX[0]
    need = pimd.replica_bytes(r["x0"].shape[1], r["x0"].shape[0])
    srv = pimd.Server(need // 2, max_replicas=4, chunk_steps=20)
    with pytest.raises(pimd.PimdError) as ei:
        submit(srv, r, 10)
    assert ei.value.status == 8        # PIMD_EBUDGET
    srv.close()
    srv = pimd.Server(8 << 30, max_replicas=4, chunk_steps=20)
    j = submit(srv, MIX[1], 10 ** 7)
    time.sleep(0.1)
    srv.cancel(j)
    time.sleep(0.2)
    with pytest.raises(pimd.PimdError) as ei:
        srv.poll(j)
    assert ei.value.status == 7        # PIMD_ENOTFOUND once cancelled
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_allocation_refusal_fails_only_that_job(pimd):
    """Fault injection on the host: an allocator hook that refuses large
    requests makes that job fail with ENOMEM; the server keeps serving."""
    import ctypes
    import torch
    big = MIX[4]
    limit = pimd.replica_bytes(big["x0"].shape[1], big["x0"].shape[0]) - 1

    def alloc(nbytes, stream, ctx):
        if nbytes > limit:
            return None
        return int(torch.cuda.caching_allocator_alloc(int(nbytes)))

    def free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = pimd.ALLOC_FN(alloc), pimd.FREE_FN(free)
    pimd.lib().pimd_set_allocator(fa, ff, None)
    try:
        srv = pimd.Server(8 << 30, max_replicas=4, chunk_steps=20)
        jbad = submit(srv, big, 40)
        jok = submit(srv, MIX[0], 40)
        t0 = time.time()
        while True:
            try:
                r = srv.poll(jbad)
            except pimd.PimdError as e:
                assert e.status == 2   # PIMD_ENOMEM
                break
            assert r is None and time.time() - t0 < 60
            time.sleep(0.01)
        assert wait(srv, [jok])[jok]["step"] == 40
        srv.close()
    finally:
        pimd.reset_allocator()
