"""The allocation-free transform entry point (pt_dst_forward_noalloc).

It serves callers that cannot let the library allocate device memory (another allocator owns
the device, or allocation latency is not acceptable in their loop).  Through the C ABI its
output must match the allocating pt_dst_forward of a problem on the same data, on two calls in
a row (the shared scratch array keeps the previous call's contents), and sizes beyond its
fixed scratch must be refused before any work is launched.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_matches_allocating_transform_on_two_calls():
    import paper_1802_08126_gb300 as ptu
    from paper_1802_08126_gb300 import _lib, build
    build.build()
    L = _lib.load()
    rng = np.random.default_rng(11)
    for prob in (S.heat2d_uniform(15, 16), S.heat1d_mms(31, 64)):
        with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, S.source(prob), None) as P:
            for call in range(2):
                r = torch.from_numpy(rng.standard_normal((prob.N, prob.ns))).cuda()
                ref = torch.empty_like(r)
                P.dst_forward(r, ref)
                out = torch.full_like(r, float("nan"))
                st = L.pt_dst_forward_noalloc(ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                              prob.N, prob.ns, None)
                assert st == 0, L.pt_last_error()
                torch.cuda.synchronize()
                a, b = out.cpu().numpy(), ref.cpu().numpy()
                assert np.isfinite(a).all()
                assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max() * np.log2(prob.N), (prob.name, call)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1802_08126_gb300 import _lib, build
    build.build()
    L = _lib.load()
    r = torch.zeros(8, dtype=torch.float64, device="cuda")
    # N_t * ceil32(ncols) = 4096 * 544 > 2^21: refused on the host, nothing launched
    st = L.pt_dst_forward_noalloc(ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(r.data_ptr()), 4096, 513, None)
    assert st == _lib.PT_EINVAL
    assert b"exceeds" in L.pt_last_error()
    st = L.pt_dst_forward_noalloc(ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(r.data_ptr()), 12, 4, None)
    assert st == _lib.PT_EINVAL
