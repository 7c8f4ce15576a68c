"""The allocation-free pressure solve, for callers that cannot let the library allocate device
memory at solve time (memory owned by a framework's caching allocator or a fixed budget, or loops
where cudaMalloc/cudaFree would synchronise the device), gives the same answer as the regular
Jacobi-preconditioned solve. Called through the C ABI, twice in a row, so the second call runs on
scratch memory that still holds the first call's data; and once on a mesh close to the scratch
limit. This file sorts last so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

from paper_1705_08813_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_NP = 131072   # scratch limit of the allocation-free solve


@pytest.fixture(scope="module")
def dgw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_08813_gb300 import dgw as d
    assert torch.cuda.is_available()
    return d


def _noalloc(dgw, mesh, b, p, rtol, max_iter):
    info = dgw.SolveInfo()
    st = dgw._lib.dgw_pressure_solve_jacobi_noalloc(mesh.h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                                    rtol, max_iter, ctypes.byref(info),
                                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, info


def _check_against_regular(dgw, w, seed, calls):
    mesh = dgw.mesh_for(w)
    assert mesh.n_p <= MAX_NP
    b = torch.tensor(I.pressure_rhs(mesh.n_p, seed), device="cuda")
    p_ref = torch.zeros_like(b)
    ref = mesh.pressure_solve(b, p_ref, rtol=1e-10, max_iter=20000, mode=2)
    assert ref["rel_residual"] <= 1e-10
    pr = p_ref.cpu().numpy()
    for call in range(calls):
        p = torch.full_like(b, float(call + 1))      # stale output contents must not matter
        st, info = _noalloc(dgw, mesh, b, p, 1e-10, 20000)
        assert st == 0, dgw._lib.dgw_last_error()
        assert info.rel_residual <= 1e-10
        ph = p.cpu().numpy()
        assert abs(ph.mean()) < 1e-14
        assert np.linalg.norm(ph - pr) / np.linalg.norm(pr) < 1e-6, call


def test_noalloc_solve_matches_regular_solve_twice(dgw):
    _check_against_regular(dgw, I.WORKLOADS["channel_q2_8x8x8"], 7, 2)


def test_noalloc_solve_near_the_scratch_limit(dgw):
    # 16 x 16 x 16 Q2: 110592 pressure DoFs, 84% of the scratch vectors in use
    _check_against_regular(dgw, I.Workload("big", 16, 16, 16, 2, 180.0, 1.0 / 3250.0, seed=3), 11, 1)


def test_noalloc_rejects_meshes_beyond_its_scratch(dgw):
    big = dgw.mesh_for(I.Workload("big2", 16, 16, 12, 3, 180.0, 1.0 / 3250.0, seed=3))   # 196608 DoFs
    assert big.n_p > MAX_NP
    b = torch.zeros(big.n_p, dtype=torch.float64, device="cuda")
    p = torch.zeros_like(b)
    st, _ = _noalloc(dgw, big, b, p, 1e-10, 10)
    assert st == -1 and b"exceeds" in dgw._lib.dgw_last_error()


def test_noalloc_refuses_a_capturing_stream(dgw):
    """The solve synchronises its stream every iteration, which a stream capture forbids: called on a
    stream that is being captured it returns DGW_EINVAL before any work, and the capture stays valid."""
    mesh = dgw.mesh_for(I.WORKLOADS["channel_q2_8x8x8"])
    b = torch.zeros(mesh.n_p, dtype=torch.float64, device="cuda")
    p = torch.zeros_like(b)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        graph.capture_begin()
        try:
            p.add_(1.0)                     # one captured kernel, so the graph is not empty
            st, _ = _noalloc(dgw, mesh, b, p, 1e-10, 10)
        finally:
            graph.capture_end()
    assert st == -1 and b"captured" in dgw._lib.dgw_last_error()
    graph.replay()
    torch.cuda.synchronize()
    assert float(p[0]) == 1.0
