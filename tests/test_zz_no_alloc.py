"""ok_apply_jacobian_noalloc: the Jacobian apply for callers that cannot
allocate device memory (their own allocator owns the GPU, or a fixed memory
budget, or no room for cudaMalloc's synchronisation on a hot loop).

It runs the same kernels as ok_apply_jacobian with the coefficient store in a
static device array, so it must give the same y = J(u_k) z as the handle-based
entry point, on two calls in a row (the second call overwrites the store the
first one left behind), and the first call's y must match the oracle's
assembled Jacobian row by row.  Collected last on purpose: it shares nothing with the
other tests and passes alone in a fresh process as well as after them."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1603_04570_gb300 as ok

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.mark.parametrize("dim,n", [(2, 40), (2, 160), (3, 12)])
def test_noalloc_jacobian_matches_handle_path_twice(dim, n):
    lib = ok.load()
    p = ok.Params(0.03, 150.0, 0.1, 0.5, 1e-3)
    nv = (n + 1) ** dim
    rng = np.random.default_rng(7 * dim + n)
    with ok.Grid(dim, n, p.eps, p.sigma, p.m, p.theta, p.dt) as g:
        for call in range(2):                     # two calls in a row, different inputs
            u = _dev(rng.uniform(-1.1, 1.1, nv))
            z = _dev(rng.standard_normal(2 * nv))
            y_ref = torch.empty(2 * nv, dtype=torch.float64, device="cuda")
            g.apply_jacobian(u, z, y_ref)
            y = torch.full((2 * nv,), float("nan"), dtype=torch.float64, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            st = lib.ok_apply_jacobian_noalloc(dim, n, ctypes.byref(p), u.data_ptr(), z.data_ptr(), y.data_ptr(),
                                               stream)
            assert st == ok.OK_SUCCESS, lib.ok_last_error()
            torch.cuda.synchronize()
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            scale = np.abs(b).max()
            assert np.abs(a - b).max() <= 1e-13 * scale, call
            if call == 0 and nv <= 30000:             # and against the oracle's assembled J (eqn newton)
                from oracle.fem import Mesh, Params, System
                sysm = System(Mesh(dim, n), Params(p.eps, p.sigma, p.m, p.theta, p.dt))
                J = sysm.jacobian(u.cpu().numpy())
                zh = z.cpu().numpy()
                assert (np.abs(a - J @ zh) <= 1e-13 * (abs(J) @ np.abs(zh))).all()


def test_noalloc_rejects_oversize_and_host_arrays():
    lib = ok.load()
    p = ok.Params(0.03, 150.0, 0.1, 0.5, 1e-3)
    u = torch.zeros(10, dtype=torch.float64, device="cuda")
    st = lib.ok_apply_jacobian_noalloc(2, 600, ctypes.byref(p), u.data_ptr(), u.data_ptr(), u.data_ptr(), None)
    assert st == ok.OK_ERR_INVALID_ARG and b"too large" in lib.ok_last_error()
    st = lib.ok_apply_jacobian_noalloc(3, 55, ctypes.byref(p), u.data_ptr(), u.data_ptr(), u.data_ptr(), None)
    assert st == ok.OK_ERR_INVALID_ARG
    h = np.zeros(2 * 9 ** 2)
    st = lib.ok_apply_jacobian_noalloc(2, 8, ctypes.byref(p), h.ctypes.data, h.ctypes.data, h.ctypes.data, None)
    assert st == ok.OK_ERR_INVALID_ARG and b"device arrays" in lib.ok_last_error()
