"""The no-allocation solve (ot_assoc_solve_cost_noalloc) against the context-based solve.

Some callers cannot allocate device memory at solve time -- a scheduler loop that must not
stall on cudaMalloc/cudaFree, or a process held to a fixed memory pool -- so the library
offers a solve whose scratch is a fixed device array inside the library image.  This file is
collected last on purpose.  It calls the entry point through the C ABI twice in a row, on
two different instances (the array keeps whatever the previous call left in it), and checks
each result against ot_assoc_solve_cost on the same inputs with the parity tolerances of the
other GPU tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_PI = 2e-5      # per plan entry, as for the iterate parity tests
RTOL_COST = 1e-6


def _instance(seed, I, J):
    rng = np.random.Generator(np.random.PCG64(seed))
    C = rng.uniform(0.0, 1.0, (I, J)).astype(np.float32)
    p = rng.lognormal(0.0, 1.0, I)
    q = rng.uniform(0.5, 1.5, J)
    p = (p / p.sum()).astype(np.float32)
    q = (q / q.sum()).astype(np.float32)
    return C, p, q


def _noalloc(L, binding, Ct, pt, qt, eps, tol, max_iter):
    I, J = Ct.shape
    f = torch.empty(I, dtype=torch.float64, device="cuda")
    g = torch.empty(J, dtype=torch.float64, device="cuda")
    pi = torch.empty((I, J), dtype=torch.float32, device="cuda")
    load = torch.empty(J, dtype=torch.float64, device="cuda")
    r = binding.ot_assoc_result()
    r.pi, r.pi_ld, r.f, r.g, r.rrh_load = pi.data_ptr(), J, f.data_ptr(), g.data_ptr(), load.data_ptr()
    st = L.ot_assoc_solve_cost_noalloc(ctypes.c_void_p(Ct.data_ptr()), Ct.stride(0), ctypes.c_void_p(pt.data_ptr()),
                                       ctypes.c_void_p(qt.data_ptr()), I, J, eps, tol, max_iter, 0, ctypes.byref(r),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, r, pi, f, g, load


def test_noalloc_solve_matches_context_solve_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_01559_gb300 import binding
    L = binding.lib()
    ctx = binding.Context(0)
    try:
        # second instance: J = 257 inside rows padded to 260 floats (the entry point reads C in
        # place, so its leading dimension must be a multiple of 4)
        for seed, (I, J, ld), eps in ((1, (20000, 800, 800), 0.05), (2, (3001, 257, 260), 0.1)):
            C, p, q = _instance(seed, I, J)
            Cpad = np.zeros((I, ld), np.float32)
            Cpad[:, :J] = C
            Ct = torch.from_numpy(Cpad).cuda()[:, :J]
            pt, qt = (torch.from_numpy(a).cuda() for a in (p, q))
            st, r, pi, f, g, load = _noalloc(L, binding, Ct, pt, qt, eps, 1e-6, 2000)
            assert st == binding.OT_OK, binding._status_name(st)
            ref = ctx.solve_cost(Ct, pt, qt, eps, tol=1e-6, max_iter=2000, want_pi=True)
            assert ref.status == binding.OT_OK
            assert abs(r.iters - ref.iters) <= 1
            assert abs(r.transport_cost - ref.transport_cost) <= RTOL_COST * ref.transport_cost
            a, b = pi.cpu().numpy().astype(np.float64), ref.pi.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(a - b) <= RTOL_PI * b + 1e-12)
            np.testing.assert_allclose(load.cpu().numpy(), ref.rrh_load.cpu().numpy(), rtol=1e-5)
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limits_and_unaligned_rows():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_01559_gb300 import binding
    L = binding.lib()
    for I, J in ((8, 1025), (131073, 4)):
        C = torch.ones((I, J), dtype=torch.float32, device="cuda")
        p = torch.full((I,), 1.0 / I, dtype=torch.float32, device="cuda")
        q = torch.full((J,), 1.0 / J, dtype=torch.float32, device="cuda")
        st, *_ = _noalloc(L, binding, C, p, q, 0.1, 1e-6, 10)
        assert st == binding.OT_EUNSUPPORTED
    # rows that are not 16-byte aligned cannot be read in place and are refused
    C = torch.ones((16, 7), dtype=torch.float32, device="cuda")
    p = torch.full((16,), 1.0 / 16, dtype=torch.float32, device="cuda")
    q = torch.full((7,), 1.0 / 7, dtype=torch.float32, device="cuda")
    st, *_ = _noalloc(L, binding, C, p, q, 0.1, 1e-6, 10)
    assert st == binding.OT_EINVAL
