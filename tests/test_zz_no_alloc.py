"""The allocation-free transform entry point (pt_dst_forward_noalloc).

It serves callers that cannot let the library allocate device memory (another allocator owns
the device, or allocation latency is not acceptable in their loop).  Through the C ABI its
output must equal the sine sums of the forward change of basis of §4 (rhat_k = sum_n r_n
sin((2k-1) n pi / (2N)), the oracle's dense definition) and the allocating pt_dst_forward of a
problem on the same data, on two calls in a row (the shared scratch array keeps the previous
call's contents), at the sizes its fixed scratch admits, up to N_t = 8192 and N_t * ceil32(ncols)
= 2^21 exactly; sizes beyond it must be refused before any work is launched.  This file is
collected last.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S
from oracle import spacetime as st

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1802_08126_gb300 import _lib as lib, build
    build.build()
    return lib.load()


def _call(L, r, out, N, ncols):
    return L.pt_dst_forward_noalloc(ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(out.data_ptr()), N, ncols, None)


def _tol(ref, N):
    # radix-2 FFT in FP64: error grows like log2(N) eps relative to the largest output
    return 1e-12 * np.abs(ref).max() * max(1.0, np.log2(N))


# (N_t, ncols): the one-slot transform, ragged column counts, and both edges of the scratch
# limit N_t * ceil32(ncols) = 2^21 (N_t = 1024 with 2043 columns padded to 2048; N_t = 8192,
# the largest N_t, with 256 columns)
SIZES = [(1, 7), (16, 1000), (64, 961), (1024, 2043), (8192, 256)]


@pytest.mark.parametrize("N,ncols", SIZES, ids=lambda v: str(v))
def test_noalloc_matches_oracle_sine_sums_on_two_calls(N, ncols):
    L = _lib()
    rng = np.random.default_rng(N + ncols)
    for call in range(2):
        r = rng.standard_normal((N, ncols))
        ref = st.dst_forward(r)
        rd = torch.from_numpy(r).cuda()
        out = torch.full_like(rd, float("nan"))
        assert _call(L, rd, out, N, ncols) == 0, L.pt_last_error()
        torch.cuda.synchronize()
        a = out.cpu().numpy()
        assert np.isfinite(a).all()
        assert np.abs(a - ref).max() <= _tol(ref, N), (N, ncols, call)


def test_noalloc_matches_allocating_transform_on_two_calls():
    import paper_1802_08126_gb300 as ptu
    L = _lib()
    rng = np.random.default_rng(11)
    for prob in (S.heat2d_uniform(15, 16), S.heat1d_mms(31, 64), S.heat2d_uniform(31, 1024)):
        with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, S.source(prob), None) as P:
            for call in range(2):
                r = torch.from_numpy(rng.standard_normal((prob.N, prob.ns))).cuda()
                ref = torch.empty_like(r)
                P.dst_forward(r, ref)
                out = torch.full_like(r, float("nan"))
                assert _call(L, r, out, prob.N, prob.ns) == 0, L.pt_last_error()
                torch.cuda.synchronize()
                a, b = out.cpu().numpy(), ref.cpu().numpy()
                assert np.isfinite(a).all()
                assert np.abs(a - b).max() <= _tol(b, prob.N), (prob.name, call)


def test_noalloc_on_a_second_device():
    """The scratch address and the kernels' shared-memory limits are set up per device."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one visible GPU")
    L = _lib()
    N, ncols = 1024, 300
    r = np.random.default_rng(2).standard_normal((N, ncols))
    ref = st.dst_forward(r)
    for dev in (0, 1):
        with torch.cuda.device(dev):
            rd = torch.from_numpy(r).cuda()
            out = torch.full_like(rd, float("nan"))
            assert _call(L, rd, out, N, ncols) == 0, L.pt_last_error()
            torch.cuda.synchronize()
            assert np.abs(out.cpu().numpy() - ref).max() <= _tol(ref, N)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1802_08126_gb300 import _lib as lib
    L = _lib()
    r = torch.zeros(8, dtype=torch.float64, device="cuda")
    # N_t * ceil32(ncols) = 4096 * 544 > 2^21: refused on the host, nothing launched
    assert _call(L, r, r, 4096, 513) == lib.PT_EINVAL
    assert b"exceeds" in L.pt_last_error()
    # N_t not a power of two, N_t above 8192, no columns
    assert _call(L, r, r, 12, 4) == lib.PT_EINVAL
    assert _call(L, r, r, 16384, 1) == lib.PT_EINVAL
    assert _call(L, r, r, 16, 0) == lib.PT_EINVAL
