"""Continuous-batching server: results equal the single-job solver and the FP64 oracle,
each job's result is the same alone and in a mix, admission follows the memory budget,
and jobs arriving mid-flight join running ones."""
import numpy as np
import pytest

import synth
from oracle import marchenko as omar
from oracle import solvers
from test_gpu_marchenko import problem, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make_jobs(cfg, G, specs, seed=0):
    """Jobs: (nv, niter, tol) with random focusing points at z = 200 m on the problem's grid."""
    rng = np.random.default_rng(seed)
    jobs = []
    for nv, niter, tol in specs:
        c = cfg.with_(nv=nv, point_grid=0, z_point=200.0)
        d = synth.draw(c)
        d.points = rng.uniform(0, synth.GRID_DX * (cfg.n_side - 1), size=(nv, 2))
        jobs.append({"nv": nv, "niter": niter, "tol": tol, "cut": synth.window_cutoffs(c, d),
                     "fd": synth.direct_focusing(c, d)})
    return jobs


def outputs(cfg, nv):
    return [np.zeros((cfg.nt, cfg.ns, nv), np.float32) for _ in range(4)]


def run_server(m, lo, ref, cfg, jobs, schedule, budget=1 << 34, max_cols=64, nref=0, niter_ref=0):
    """schedule: {step_index: [job indices submitted before that step]}; runs until all done."""
    srv = m.srv_create(lo.h, ref.h if ref is not None else None, budget, max_cols, nref, niter_ref)
    outs, ids, step = {}, {}, 0
    try:
        while True:
            for i in schedule.get(step, []):
                o = outputs(cfg, jobs[i]["nv"])
                outs[i] = o
                ids[i] = m.srv_submit(srv, jobs[i]["cut"], jobs[i]["fd"], jobs[i]["nv"], jobs[i]["niter"],
                                      jobs[i]["tol"], o)
            m.srv_step(srv)
            step += 1
            polls = {i: m.srv_poll(srv, ids[i]) for i in ids}
            if len(ids) == sum(len(v) for v in schedule.values()) and all(
                    p["state"] == m.JOB_DONE for p in polls.values()):
                return outs, polls, step
            assert step < 500
    finally:
        m.srv_destroy(srv)


@pytest.fixture(scope="module")
def small():
    cfg, G, cut, fd = problem(11, 256, 60, 1, 200.0)
    return cfg, G


def test_server_matches_single_job_solver_and_oracle(small):
    """complex64 kernel, no refinement: every job equals marchenko_lsqr and the FP64 oracle."""
    import paper_2011_11120_gb300 as m
    cfg, G = small
    jobs = make_jobs(cfg, G, [(3, 12, 0.0), (1, 8, 0.0), (5, 10, 1e-4), (2, 6, 0.0)], seed=1)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    outs, polls, _ = run_server(m, op, None, cfg, jobs, {0: [0, 1], 2: [2], 3: [3]})
    for i, job in enumerate(jobs):
        ref = omar.Marchenko(G, cfg.dt, cfg.dr, job["cut"], cfg.nt)
        res = solvers.lsqr(ref.matvec, ref.rmatvec, ref.data(job["fd"]), niter=job["niter"], tol=job["tol"])
        gm, _, gp = ref.greens(res.x[0], res.x[1], job["fd"])
        assert polls[i]["iters"] == res.iters
        assert rel(outs[i][0], res.x[0]) <= 1e-5 and rel(outs[i][1], res.x[1]) <= 1e-5
        assert rel(outs[i][2], gm) <= 1e-5 and rel(outs[i][3], gp) <= 1e-5
        single = op.marchenko(torch.from_numpy(job["cut"]).cuda(), torch.from_numpy(job["fd"]).cuda(),
                              job["niter"], tol=job["tol"])
        assert rel(outs[i][0], single["f_minus"].cpu().numpy()) <= 1e-6
    op.close()


def test_server_solo_equals_mix_fp16_with_refinement(small):
    """FP16 kernel in LSQR + float32 refinement: a job's result alone equals its result in a mix."""
    import paper_2011_11120_gb300 as m
    cfg, G = small
    jobs = make_jobs(cfg, G, [(3, 12, 0.0), (4, 9, 0.0), (1, 14, 0.0), (6, 7, 0.0)], seed=2)
    Gt = torch.from_numpy(G.astype(np.complex64)).cuda()
    lo = m.MDC(Gt, cfg.nt, cfg.dt, cfg.dr, storage="c16f")
    ref = m.MDC(Gt, cfg.nt, cfg.dt, cfg.dr, storage="c64")
    solo, _, _ = run_server(m, lo, ref, cfg, jobs, {0: [0]}, nref=1, niter_ref=5)
    mix, polls, _ = run_server(m, lo, ref, cfg, jobs, {0: [1, 2], 1: [0], 4: [3]}, nref=1, niter_ref=5)
    for k in range(4):
        d = rel(mix[0][k], solo[0][k])
        print(f"output {k}: solo vs mix rel L2 {d:.2e}")
        assert d <= 1e-6
    # accuracy of every mixed job against the converged FP64 solution
    for i, job in enumerate(jobs):
        o = omar.Marchenko(G, cfg.dt, cfg.dr, job["cut"], cfg.nt)
        res = solvers.lsqr(o.matvec, o.rmatvec, o.data(job["fd"]), niter=200, tol=1e-13)
        e = rel(mix[i][0], res.x[0])
        print(f"job {i}: rel L2 vs converged FP64 {e:.2e}, final residual {polls[i]['final_residual']:.2e}")
        assert e <= 1e-3
        assert polls[i]["iters"] == job["niter"] + 5
    lo.close()
    ref.close()


def test_server_admission_by_budget_and_mid_flight_arrivals(small):
    import paper_2011_11120_gb300 as m
    cfg, G = small
    jobs = make_jobs(cfg, G, [(2, 10, 0.0), (2, 10, 0.0), (2, 10, 0.0)], seed=3)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    per_job = 12 * cfg.nt * cfg.ns * 2 * 4 + 4 * cfg.ns * 2 * 8 + cfg.ns * 2 * 4 + (1 << 20)
    srv = m.srv_create(op.h, None, int(1.5 * per_job), 64)      # room for one job at a time
    try:
        ids = [m.srv_submit(srv, j["cut"], j["fd"], j["nv"], j["niter"]) for j in jobs]
        m.srv_step(srv)
        st = m.srv_stats(srv)
        assert st["running"] == 1 and st["queued"] == 2
        steps = 1
        while any(m.srv_poll(srv, i)["state"] != m.JOB_DONE for i in ids):
            m.srv_step(srv)
            steps += 1
            assert m.srv_stats(srv)["running"] <= 1
            assert steps < 100
        assert steps >= 30          # three jobs of 10 iterations, one at a time
        q = [m.srv_poll(srv, i)["queue_s"] for i in ids]
        assert q[0] <= q[1] <= q[2]
        with pytest.raises(m.MDCError):
            big = make_jobs(cfg, G, [(40, 5, 0.0)], seed=4)[0]
            m.srv_submit(srv, big["cut"], big["fd"], 40, 5)          # can never fit the budget
    finally:
        m.srv_destroy(srv)
    # mid-flight arrival: the second job starts while the first is still running
    srv = m.srv_create(op.h, None, 1 << 34, 64)
    try:
        a = m.srv_submit(srv, jobs[0]["cut"], jobs[0]["fd"], 2, 10)
        for _ in range(3):
            m.srv_step(srv)
        b = m.srv_submit(srv, jobs[1]["cut"], jobs[1]["fd"], 2, 10)
        m.srv_step(srv)
        assert m.srv_poll(srv, a)["state"] == m.JOB_RUNNING and m.srv_poll(srv, b)["state"] == m.JOB_RUNNING
        while m.srv_poll(srv, b)["state"] != m.JOB_DONE:
            m.srv_step(srv)
        assert m.srv_poll(srv, a)["latency_s"] < m.srv_poll(srv, b)["latency_s"] + 1.0
    finally:
        m.srv_destroy(srv)
    op.close()


def test_server_retires_a_non_finite_job_alone(small):
    """A job whose data holds NaN fails with MDC_ERR_NUMERIC; its batch mates are unaffected."""
    import paper_2011_11120_gb300 as m
    cfg, G = small
    jobs = make_jobs(cfg, G, [(2, 8, 0.0), (3, 8, 0.0), (2, 8, 0.0)], seed=5)
    bad = dict(jobs[1])
    bad["fd"] = jobs[1]["fd"].copy()
    bad["fd"][3, 5, 1] = np.nan
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    solo, _, _ = run_server(m, op, None, cfg, [jobs[0]], {0: [0]})
    srv = m.srv_create(op.h, None, 1 << 34, 64)
    try:
        outs = [outputs(cfg, j["nv"]) for j in (jobs[0], bad, jobs[2])]
        ids = [m.srv_submit(srv, j["cut"], j["fd"], j["nv"], j["niter"], 0.0, o)
               for j, o in zip((jobs[0], bad, jobs[2]), outs)]
        for _ in range(30):
            m.srv_step(srv)
            if all(m.srv_poll(srv, i)["state"] >= m.JOB_DONE for i in ids):
                break
        polls = [m.srv_poll(srv, i) for i in ids]
        assert polls[1]["state"] == m.JOB_FAILED and polls[1]["status"] == -5
        assert polls[0]["state"] == m.JOB_DONE and polls[2]["state"] == m.JOB_DONE
        assert rel(outs[0][0], solo[0][0]) <= 1e-6
        assert np.isfinite(outs[2][0]).all()
    finally:
        m.srv_destroy(srv)
    op.close()


@pytest.mark.parametrize("storage,nref", [("c64", 0), ("c16f", 1)])
def test_checkpoint_resume_continues_bit_for_bit(small, storage, nref):
    """A server checkpointed mid-flight (jobs running, one still queued) and resumed on a new
    server finishes with the same outputs, iteration counts and residuals as the uninterrupted
    server, bit for bit; resumed jobs wait for srv_bind; a checkpoint does not fit a server of
    another kernel shape."""
    import paper_2011_11120_gb300 as m
    cfg, G = small
    jobs = make_jobs(cfg, G, [(3, 12, 0.0), (2, 9, 0.0), (4, 10, 1e-4)], seed=5)
    Gt = torch.from_numpy(G.astype(np.complex64)).cuda()
    op = m.MDC(Gt, cfg.nt, cfg.dt, cfg.dr, storage=storage)
    ref = m.MDC(Gt, cfg.nt, cfg.dt, cfg.dr, storage="c64") if nref else None
    niter_ref = 3 if nref else 0
    max_cols = 12   # jobs 0 and 1 run together (10 columns); job 2 (8 columns) waits in the queue

    def submit_all(srv):
        outs, ids = [], []
        for job in jobs:
            o = outputs(cfg, job["nv"])
            outs.append(o)
            ids.append(m.srv_submit(srv, job["cut"], job["fd"], job["nv"], job["niter"], job["tol"], o))
        return outs, ids

    def drain(srv, ids):
        for _ in range(500):
            if all(m.srv_poll(srv, i)["state"] == m.JOB_DONE for i in ids):
                return {i: m.srv_poll(srv, i) for i in ids}
            m.srv_step(srv)
        raise AssertionError("server did not drain")

    srv = m.srv_create(op.h, ref.h if ref else None, 1 << 34, max_cols, nref, niter_ref)
    outs_a, ids_a = submit_all(srv)
    polls_a = drain(srv, ids_a)
    m.srv_destroy(srv)

    srv = m.srv_create(op.h, ref.h if ref else None, 1 << 34, max_cols, nref, niter_ref)
    outs_b, ids_b = submit_all(srv)
    for _ in range(5):
        m.srv_step(srv)
    st = m.srv_stats(srv)
    assert st["running"] == 2 and st["queued"] == 1
    blob = m.srv_checkpoint(srv)
    m.srv_destroy(srv)                       # the first server is gone: its host buffers are not reused

    srv = m.srv_create(op.h, ref.h if ref else None, 1 << 34, max_cols, nref, niter_ref)
    try:
        got = m.srv_resume(srv, blob)
        assert got == ids_b
        with pytest.raises(m.MDCError):
            m.srv_step(srv)                  # no outputs bound yet
        outs_c = [outputs(cfg, job["nv"]) for job in jobs]
        for i, o in zip(got, outs_c):
            m.srv_bind(srv, i, o)
        polls_c = drain(srv, got)
        with pytest.raises(m.MDCError):
            m.srv_resume(srv, blob)          # ids already known to this server
    finally:
        m.srv_destroy(srv)
    for q, (ia, ic) in enumerate(zip(ids_a, got)):
        assert polls_c[ic]["iters"] == polls_a[ia]["iters"]
        assert polls_c[ic]["final_residual"] == polls_a[ia]["final_residual"]
        for k in range(4):
            assert np.array_equal(outs_c[q][k], outs_a[q][k]), (q, k)

    other = m.MDC(torch.zeros((cfg.nf, 9, 9), dtype=torch.complex64, device="cuda"), cfg.nt, cfg.dt, cfg.dr,
                  storage=storage)
    srv = m.srv_create(other.h, None, 1 << 34, max_cols, 0, 0)
    try:
        with pytest.raises(m.MDCError):
            m.srv_resume(srv, blob)
        with pytest.raises(m.MDCError):
            m.srv_resume(srv, b"not a checkpoint" * 4)
    finally:
        m.srv_destroy(srv)
    other.close()
    op.close()
    if ref:
        ref.close()


def test_kept_results_match_submitted_buffers(small):
    """srv_result returns, for a job submitted without output buffers (results kept by the
    server), exactly what a job with buffers received; without keep_results it is refused."""
    import paper_2011_11120_gb300 as m
    cfg, G = small
    job = make_jobs(cfg, G, [(2, 6, 0.0)], seed=9)[0]
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    srv = m.srv_create(op.h, None, 1 << 34, 64)
    try:
        o_a = outputs(cfg, 2)
        ja = m.srv_submit(srv, job["cut"], job["fd"], 2, job["niter"], 0.0, o_a)
        jb = m.srv_submit(srv, job["cut"], job["fd"], 2, job["niter"], 0.0)         # dropped results
        m.srv_keep_results(srv, True)
        jc = m.srv_submit(srv, job["cut"], job["fd"], 2, job["niter"], 0.0)         # kept results
        with pytest.raises(m.MDCError):
            m.srv_result(srv, jc, outputs(cfg, 2))                                   # still queued
        while any(m.srv_poll(srv, j)["state"] < m.JOB_DONE for j in (ja, jb, jc)):
            m.srv_step(srv)
        o_c = outputs(cfg, 2)
        m.srv_result(srv, jc, o_c)
        o_a2 = outputs(cfg, 2)
        m.srv_result(srv, ja, o_a2)
        for k in range(4):
            assert np.array_equal(o_c[k], o_a[k]) and np.array_equal(o_a2[k], o_a[k])
        with pytest.raises(m.MDCError):
            m.srv_result(srv, jb, outputs(cfg, 2))                                   # was dropped
    finally:
        m.srv_destroy(srv)
    op.close()
