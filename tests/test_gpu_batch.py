"""Block mixed-precision solves (dgw_pressure_solve_batch) and continuous batching in the request
loop: every column reaches the 1e-10 residual checked with the oracle's own operator, and a column's
result is the same bits alone, in a block of any composition and when it joins a running block."""
import time

import numpy as np
import pytest

import oracle as O
from paper_1705_08813_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dgw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_08813_gb300 import dgw as d
    assert torch.cuda.is_available()
    return d


def _rhs(m, seeds):
    return [torch.tensor(I.pressure_rhs(m.n_p, s), device="cuda") for s in seeds]


def _oracle_residual(om, b, p):
    bh = b.cpu().numpy()
    bh = bh - bh.mean()
    return np.linalg.norm(bh - om.laplace(p.cpu().numpy())) / np.linalg.norm(bh)


@pytest.mark.parametrize("wname,ncols", [("channel_q2_8x8x8", 5), ("channel_q2_8x8x8", 11)])
def test_block_columns_converge_and_equal_alone(dgw, wname, ncols):
    """ncols = 11 > 8 columns: the last three join the block as the first ones finish."""
    w = I.WORKLOADS[wname]
    m = dgw.mesh_for(w)
    om = O.Mesh(**w.mesh_kwargs())
    bs = _rhs(m, range(50, 50 + ncols))
    ps = [torch.full_like(b, 7.0) for b in bs]      # stale output contents must not matter
    infos = dgw.pressure_solve_batch(m, bs, ps)
    for c in range(ncols):
        assert infos[c]["rel_residual"] <= 1e-10, (c, infos[c])
        assert _oracle_residual(om, bs[c], ps[c]) <= 1.5e-10, c
        assert abs(ps[c].mean().item()) <= 1e-14 * ps[c].abs().max().item()
    # each column alone (a block of one), and two columns in another order
    for c in (0, ncols - 1):
        p1 = torch.zeros_like(bs[c])
        dgw.pressure_solve_batch(m, [bs[c]], [p1])
        assert torch.equal(p1, ps[c]), c
    q = [torch.zeros_like(bs[0]) for _ in range(2)]
    dgw.pressure_solve_batch(m, [bs[2], bs[1]], q)
    assert torch.equal(q[0], ps[2]) and torch.equal(q[1], ps[1])


def test_block_matches_the_single_solve(dgw):
    """Same problem as dgw_pressure_solve mode 1: both solutions satisfy the 1e-10 residual, so they
    agree to the conditioning-limited accuracy."""
    w = I.Workload("bq3", 8, 6, 4, 3, 395.0, 1.0 / 6000.0, seed=5)
    m = dgw.mesh_for(w)
    b = _rhs(m, [9])[0]
    p_single = torch.zeros_like(b)
    info = m.pressure_solve(b, p_single, rtol=1e-10, max_iter=500, mode=1)
    p_block = torch.zeros_like(b)
    [binfo] = dgw.pressure_solve_batch(m, [b], [p_block])
    assert info["rel_residual"] <= 1e-10 and binfo["rel_residual"] <= 1e-10
    diff = (p_single - p_block).norm().item() / p_single.norm().item()
    assert diff < 1e-6, diff


def test_block_rejections(dgw):
    bump = dgw.mesh_for(I.bump_workload("b", 4, 4, 2, 2, seed=3))
    b = torch.zeros(bump.n_p, dtype=torch.float64, device="cuda")
    with pytest.raises(dgw.DGWError):
        dgw.pressure_solve_batch(bump, [b], [torch.zeros_like(b)])
    with pytest.raises(ValueError):
        dgw.pressure_solve_batch(bump, [], [])


def test_request_loop_batches_solves_that_arrive_while_others_run(dgw):
    """Solves on one channel submitted over time, with applies and solves on another mesh between
    them: every solve is the same bits as its column alone, so joining a running block (or not)
    changes nothing; the loop uses fewer blocks than solves."""
    wa = I.Workload("sa", 8, 8, 8, 3, 395.0, 1.0 / 6000.0, seed=61)
    wb = I.Workload("sb", 6, 4, 4, 2, 180.0, 1.0 / 3250.0, seed=62)
    ma, mb = dgw.mesh_for(wa), dgw.mesh_for(wb)
    ba = _rhs(ma, range(70, 82))
    refs = []
    for b in ba:
        p = torch.zeros_like(b)
        dgw.pressure_solve_batch(ma, [b], [p])
        refs.append(p)
    pb = torch.tensor(I.pressure_field(mb.n_p, 3), device="cuda")
    yb_ref = torch.empty_like(pb)
    mb.laplace(pb, yb_ref)
    torch.cuda.synchronize()
    srv = dgw.Server(16 << 30, max_inflight=3)
    outs = [torch.full_like(b, 3.0) for b in ba]
    yb = torch.zeros_like(pb)
    tickets = []
    for j, b in enumerate(ba):
        tickets.append(srv.submit(0, dgw.mesh_params(wa), b, outs[j], mode=1))
        if j == 4:
            tickets.append(srv.submit(1, dgw.mesh_params(wb), pb, yb))
        if j % 4 == 3:
            time.sleep(0.002)   # some arrive while the block is running
    res, t0 = {}, time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
        assert time.time() - t0 < 120, "jobs did not complete"
        time.sleep(0.001)
    assert all(r["status"] == 0 for r in res.values())
    for j in range(len(ba)):
        assert torch.equal(outs[j], refs[j]), j
    assert torch.equal(yb, yb_ref)
    st = srv.stats()
    assert st["queued"] == 0 and st["running"] == 0
    srv.close()
