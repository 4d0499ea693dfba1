"""The allocation-free CG solve (nbte_laplacian_solve_noalloc).

Some callers cannot call cudaMalloc: code running inside another framework's
memory pool or under a fixed device-memory budget, or a loop where an
allocation may block or fail.  This entry point works in a fixed array of the
library's device code, on buffers the caller owns.

The checks:
* one synthetic iteration through nbte_solve_steady (the existing entry
  point) applies the correction delta = T^1 - T_L, the solution of the
  cell-Laplacian system L delta = V beta (T_L - T^0).  The allocation-free
  call, given that matrix and right-hand side, returns the same delta -- on
  two calls in a row (the second with the right-hand side scaled by -2),
  within the temperature tolerance of the FP64 parity tests (1e-9 of the
  field's deviation) -- and the oracle's sparse LU solution of the same
  system;
* after a first call on the device (n = 0 does only that set-up) a call
  leaves the device's free memory unchanged;
* a row without a positive diagonal entry is refused, and a barrier wait made
  to run out (nbte_test_timeouts: one poll) gives up with
  NBTE_ERR_DEVICE_TIMEOUT, after which the next call is exact again.
The test's own device buffers come from PyTorch; the calls under test
allocate nothing.
"""
import numpy as np
import pytest

from oracle import OracleSolver
from cases import fin2d_mixed

pytestmark = pytest.mark.gpu


def _system(p, torch, dev):
    o = OracleSolver(p)
    lu = o.laplacian()
    L = o._lap_matrix.tocsr()
    L.sort_indices()
    rp = torch.tensor(L.indptr.astype(np.int32), device=dev)
    col = torch.tensor(L.indices.astype(np.int32), device=dev)
    val = torch.tensor(L.data, dtype=torch.float64, device=dev)
    return o, lu, L, rp, col, val


def test_noalloc_solve_matches_synthetic_correction(gpu_lib):
    import torch
    from paper_2607_03226_b300 import nbte

    torch.cuda.set_device(0)
    p = fin2d_mixed()
    s = nbte.Solver(p)
    info = s.solve(scheme="synthetic", precision="fp64", n_iter=1, cg_tol=1e-14, cg_max_iter=50000)
    assert info["status"] == 0
    T1 = s.temperature(0)
    TL = s.temperature(2)
    delta_ref = T1 - TL
    scale_T = np.abs(T1 - p.T_ref).max()
    s.close()

    dev = torch.device("cuda", 0)
    o, lu, L, rp, col, val = _system(p, torch, dev)
    rhs = o.g.V * o.beta * (TL - p.T_ref)   # T^0 = T_ref, so T'^0 = 0
    n = L.shape[0]
    stream = torch.cuda.current_stream().cuda_stream
    # the per-device set-up (loads the library's device code and its array)
    assert nbte.nbte_laplacian_solve_noalloc(0, 0, 0, 0, 0, 0, 1e-13, 1, stream=stream)[0] == nbte.NBTE_OK
    for k, factor in enumerate((1.0, -2.0)):
        b = torch.tensor(factor * rhs, dtype=torch.float64, device=dev)
        x = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        status, iters, res = nbte.nbte_laplacian_solve_noalloc(
            n, rp.data_ptr(), col.data_ptr(), val.data_ptr(), b.data_ptr(), x.data_ptr(), 1e-13, 50000,
            stream=stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "the call changed the device's free memory"
        assert status == nbte.NBTE_OK and iters > 0 and res <= 1e-13
        xh = x.cpu().numpy()
        err = np.abs(xh - factor * delta_ref).max() / (abs(factor) * scale_T)
        assert err < 1e-9, (factor, err)
        exact = lu.solve(factor * rhs)
        err_o = np.abs(xh - exact).max() / np.abs(exact).max()
        assert err_o < 1e-9, (factor, err_o)


def test_noalloc_refuses_a_row_without_positive_diagonal(gpu_lib):
    import torch
    from paper_2607_03226_b300 import nbte

    dev = torch.device("cuda", 0)
    o, lu, L, rp, col, val = _system(fin2d_mixed(), torch, dev)
    n = L.shape[0]
    bad = L.copy()
    r = n // 2
    bad.data[bad.indptr[r]:bad.indptr[r + 1]][bad.indices[bad.indptr[r]:bad.indptr[r + 1]] == r] = 0.0
    vbad = torch.tensor(bad.data, dtype=torch.float64, device=dev)
    b = torch.ones(n, dtype=torch.float64, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    with pytest.raises(nbte.NbteError) as e:
        nbte.nbte_laplacian_solve_noalloc(n, rp.data_ptr(), col.data_ptr(), vbad.data_ptr(), b.data_ptr(),
                                          x.data_ptr(), 1e-10, 100)
    assert e.value.code == nbte.NBTE_ERR_ARG and "diagonal" in str(e.value)


def test_noalloc_barrier_timeout_then_exact(gpu_lib):
    """A system of ~100k rows runs on many cooperative blocks; with one poll
    per barrier wait the early blocks give up, the call reports a timeout,
    and the next call (default limit) solves exactly."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import spsolve
    import torch
    from paper_2607_03226_b300 import nbte

    dev = torch.device("cuda", 0)
    m = 320
    T = sp.diags([-np.ones(m - 1), 2.5 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    A = (sp.kron(sp.identity(m), T) + sp.kron(T, sp.identity(m))).tocsr()
    A.sort_indices()
    n = A.shape[0]
    rhs = np.random.default_rng(3).standard_normal(n)
    rp = torch.tensor(A.indptr.astype(np.int32), device=dev)
    col = torch.tensor(A.indices.astype(np.int32), device=dev)
    val = torch.tensor(A.data, dtype=torch.float64, device=dev)
    b = torch.tensor(rhs, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    args = (n, rp.data_ptr(), col.data_ptr(), val.data_ptr(), b.data_ptr(), x.data_ptr(), 1e-12, 5000)
    code = None
    try:
        for _ in range(3):
            nbte.nbte_test_timeouts(1)
            try:
                nbte.nbte_laplacian_solve_noalloc(*args)
                code = nbte.NBTE_OK
            except nbte.NbteError as e:
                code = e.code
            if code == nbte.NBTE_ERR_DEVICE_TIMEOUT:
                break
    finally:
        nbte.nbte_test_timeouts(0)
    assert code == nbte.NBTE_ERR_DEVICE_TIMEOUT
    status, iters, res = nbte.nbte_laplacian_solve_noalloc(*args)
    assert status == nbte.NBTE_OK and res <= 1e-12
    exact = spsolve(A.tocsc(), rhs)
    assert np.abs(x.cpu().numpy() - exact).max() / np.abs(exact).max() < 1e-9


def test_noalloc_rejects_oversized_system(gpu_lib):
    """Sizes beyond the fixed scratch are refused before any device work."""
    from paper_2607_03226_b300 import nbte
    with pytest.raises(nbte.NbteError) as e:
        nbte.nbte_laplacian_solve_noalloc((1 << 18) + 1, 1, 1, 1, 1, 1, 1e-10, 10)
    assert e.value.code == nbte.NBTE_ERR_ARG
    assert "exceeds" in str(e.value)
