"""Request loop: mixed solve/apply jobs on different meshes and degrees, admitted as slots and
memory free up, overlapping on the device. Each result must equal the same job run alone (mixed
solves on channels run as block solves: alone means a block of one column)."""
import time

import numpy as np
import pytest

from paper_1705_08813_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = {
    "a": I.Workload("a", 6, 4, 4, 2, 180.0, 1.0 / 3250.0, seed=31),
    "b": I.Workload("b", 8, 6, 4, 3, 395.0, 1.0 / 6000.0, seed=32),
    "c": I.Workload("c", 4, 4, 4, 4, 590.0, 1.0 / 12000.0, seed=33),
    "d": I.Workload("d", 4, 4, 2, 5, 180.0, 1.0 / 3250.0, seed=34),
}
# (kind, workload, prec, solve mode)
JOBS = [(0, "a", 0, 1), (0, "b", 0, 1), (1, "c", 0, 0), (3, "a", 0, 0), (4, "b", 0, 0), (2, "c", 0, 0),
        (0, "d", 0, 0), (1, "d", 1, 0), (0, "a", 0, 1), (4, "d", 1, 0), (3, "c", 1, 0), (0, "c", 0, 1)]


@pytest.fixture(scope="module")
def dgw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_08813_gb300 import dgw as d
    return d


def _inputs(dgw, kind, w, prec, j):
    m = dgw.mesh_for(w)
    dt = torch.float64 if prec == 0 else torch.float32
    if kind == 0:
        inp = torch.tensor(I.pressure_rhs(m.n_p, 100 + j), device="cuda")
        out = torch.zeros(m.n_p, dtype=torch.float64, device="cuda")
    elif kind == 1:
        inp = torch.tensor(I.pressure_field(m.n_p, 100 + j), device="cuda", dtype=dt)
        out = torch.zeros(m.n_p, dtype=dt, device="cuda")
    else:
        u = I.velocity_field(m.node_coords(), m.n_e, w)
        inp = torch.tensor(u, device="cuda", dtype=torch.float64 if kind == 2 else dt)
        out = torch.zeros(m.n_p if kind == 2 else m.n_u, dtype=torch.float64 if kind == 2 else dt, device="cuda")
    return m, inp, out


def _alone(m, kind, inp, out, mode, aux=None):
    if kind == 0 and mode == 1:
        # the request loop runs mixed solves on channels as block solves: alone is a block of one
        from paper_1705_08813_gb300 import dgw
        dgw.pressure_solve_batch(m, [inp], [out], rtol=1e-10, max_iter=500)
    elif kind == 0:
        m.pressure_solve(inp, out, rtol=1e-10, max_iter=500, mode=mode)
    elif kind == 1:
        m.laplace(inp, out)
    elif kind == 2:
        m.divergence(inp, out)
    elif kind == 3:
        m.convective(inp, out)
    else:
        m.update_eddy_viscosity(aux)
        m.viscous(inp, out)
    torch.cuda.synchronize()
    return out.clone()


def _wait(srv, tickets, timeout=120.0):
    res, t0 = {}, time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
        assert time.time() - t0 < timeout, "jobs did not complete"
        time.sleep(0.001)
    return res


def test_mixed_jobs_equal_alone(dgw):
    refs, bufs = [], []
    for j, (kind, wn, prec, mode) in enumerate(JOBS):
        m, inp, out = _inputs(dgw, kind, W[wn], prec, j)
        aux = inp.double().contiguous() if kind == 4 else None
        refs.append(_alone(m, kind, inp, out, mode, aux))
        bufs.append((inp, torch.zeros_like(out), aux))
        del m
    srv = dgw.Server(16 << 30, max_inflight=4)
    tickets = []
    for j, (kind, wn, prec, mode) in enumerate(JOBS):
        inp, out, aux = bufs[j]
        tickets.append(srv.submit(kind, dgw.mesh_params(W[wn]), inp, out, prec=prec, mode=mode, aux=aux))
    res = _wait(srv, tickets)
    for j, t in enumerate(tickets):
        assert res[t]["status"] == 0, (j, res[t])
        got, ref = bufs[j][1].double().cpu().numpy(), refs[j].double().cpu().numpy()
        assert np.array_equal(got, ref) or np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max(), j
        if JOBS[j][0] == 0:
            assert res[t]["rel_residual"] <= 1e-10
        assert res[t]["latency_ms"] > 0
    st = srv.stats()
    assert st["queued"] == 0 and st["running"] == 0 and st["meshes"] >= 4
    srv.close()


def test_admission_by_memory_budget(dgw):
    """A budget that holds one small mesh: jobs on three meshes still complete (idle meshes are
    evicted), and a job that can never fit fails with DGW_ENOMEM."""
    srv = dgw.Server(24 << 20, max_inflight=2)
    tickets, outs = [], []
    for j, wn in enumerate(["a", "c", "a"]):
        m, inp, out = _inputs(dgw, 1, W[wn], 0, j)
        tickets.append(srv.submit(1, dgw.mesh_params(W[wn]), inp, out))
        outs.append((inp, out, m))
    big = I.Workload("big", 32, 24, 24, 4, 590.0, 1.0 / 12000.0, seed=2)
    xb = torch.zeros(32 * 24 * 24 * 125, dtype=torch.float64, device="cuda")   # full-size buffers
    yb = torch.zeros_like(xb)
    tb = srv.submit(0, dgw.mesh_params(big), xb, yb)
    res = _wait(srv, tickets + [tb])
    for t in tickets:
        assert res[t]["status"] == 0
    assert res[tb]["status"] == -2
    for inp, out, m in outs:
        y = torch.empty_like(out)
        m.laplace(inp, y)
        assert torch.equal(y, out)
    assert srv.stats()["reserved_bytes"] <= 24 << 20
    srv.close()


def test_stream_of_block_solves_on_two_meshes(dgw):
    """Solves arrive one by one on two meshes of the same degree while finished ones are polled (and
    their records freed) as soon as they complete: a block keeps admitting only solves of its own
    mesh, and every solve meets its tolerance with the result it has alone."""
    wx = I.Workload("x", 8, 6, 4, 3, 395.0, 1.0 / 6000.0, seed=51)
    wy = I.Workload("y", 6, 6, 4, 3, 395.0, 1.0 / 6000.0, seed=52)
    jobs = []
    for j in range(24):
        w = wx if j % 3 else wy
        m, inp, out = _inputs(dgw, 0, w, 0, 200 + j)
        jobs.append((w, m, inp, out))
    refs = [_alone(m, 0, inp, torch.zeros_like(out), 1) for (w, m, inp, out) in jobs]
    srv = dgw.Server(16 << 30, max_inflight=4)
    tickets, res = {}, {}
    t0 = time.time()
    for j, (w, m, inp, out) in enumerate(jobs):
        tickets[srv.submit(0, dgw.mesh_params(w), inp, out, mode=1)] = j
        for t in list(tickets):
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
        time.sleep(0.002)
    while len(res) < len(tickets):
        for t in list(tickets):
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
        assert time.time() - t0 < 120.0, "jobs did not complete"
        time.sleep(0.001)
    srv.close()
    for t, j in tickets.items():
        assert res[t]["status"] == 0, (j, res[t])
        assert res[t]["rel_residual"] <= 1e-10
        got, ref = jobs[j][3].cpu().numpy(), refs[j].cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max(), j
