"""The no-allocation residual check (mss_residual_norm_noalloc) against the
allocating one (mss_residual_norm), through the C-ABI.

The no-allocation entry point serves callers that cannot allocate device
memory when they make the call (a device pool reserved by another framework,
a region where an allocation call is not allowed, a loop that must not enter
the allocator). This file is collected last so that a run stopping at its
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-12     # the relative tolerance of the FP64 parity tests


def _counting_handle(mss):
    """A handle whose allocation hooks count calls (and use cudaMalloc-like
    memory from torch's allocator)."""
    calls = {"alloc": 0, "free": 0}
    stream = torch.cuda.current_stream()

    def _alloc(nbytes, ctx):
        calls["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                  stream)

    def _free(ptr, ctx):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    a, f = mss.ALLOC_FN(_alloc), mss.FREE_FN(_free)
    h = C.c_void_p()
    lib = mss.load()
    assert lib.mss_create(C.byref(h), C.c_void_p(stream.cuda_stream), a, f, None) == 0
    return lib, h, calls, (a, f)


def test_noalloc_matches_allocating_call_twice():
    from paper_1912_04385_gb300 import build, mss
    from paper_1912_04385_gb300 import synthetic as sy
    build.build()
    lib, h, calls, keep = _counting_handle(mss)
    try:
        s = sy.make_system(45, 37, 6, pe=10.0, sigma=1.0, band=True, seed=5)
        rp = torch.from_numpy(s.row_ptr).cuda()
        ci = torch.from_numpy(s.col_idx).cuda()
        v = torch.from_numpy(s.vals.reshape(-1)).cuda()
        b = torch.from_numpy(s.b).cuda()
        J = mss.Bsr(s.n_cells, s.nnzb, rp.data_ptr(), ci.data_ptr(), v.data_ptr())
        rng = np.random.default_rng(11)
        for call in range(2):   # two calls in a row: the shared scratch is reused
            x = torch.from_numpy(rng.standard_normal(s.n_cells * 6)).cuda()
            ref = torch.empty(2, dtype=torch.float64, device="cuda")
            out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
            assert lib.mss_residual_norm(h, C.byref(J), 6, b.data_ptr(), x.data_ptr(),
                                         ref.data_ptr()) == 0
            before = dict(calls)
            st = lib.mss_residual_norm_noalloc(h, C.byref(J), 6, b.data_ptr(), x.data_ptr(),
                                               out.data_ptr())
            assert st == 0, lib.mss_last_error(h)
            torch.cuda.synchronize()
            assert calls == before, "the no-allocation call used the allocation hooks"
            r, o = ref.cpu().numpy(), out.cpu().numpy()
            assert np.all(np.abs(o - r) <= TOL * np.abs(r)), (call, o, r)
        assert calls["alloc"] >= 2      # the allocating call did allocate
    finally:
        lib.mss_destroy(h)


def test_noalloc_rejects_sizes_beyond_the_limit():
    from paper_1912_04385_gb300 import build, mss
    build.build()
    lib, h, calls, keep = _counting_handle(mss)
    try:
        tiny_i = torch.zeros(4, dtype=torch.int32, device="cuda")
        tiny_d = torch.zeros(4, dtype=torch.float64, device="cuda")
        too_many = (1 << 20) + 1
        # sizes are checked on the host before any device work
        J = mss.Bsr(too_many, too_many, tiny_i.data_ptr(), tiny_i.data_ptr(), tiny_d.data_ptr())
        st = lib.mss_residual_norm_noalloc(h, C.byref(J), 6, tiny_d.data_ptr(),
                                           tiny_d.data_ptr(), tiny_d.data_ptr())
        assert st == mss.ERR_INVALID_ARG
        assert b"no-allocation limit" in lib.mss_last_error(h)
        assert calls["alloc"] == 0
    finally:
        lib.mss_destroy(h)


def test_noalloc_at_the_limit():
    # exactly MSS_NOALLOC_MAX_CELLS cells (the 1024 x 1024 grid): the kernels
    # write and read the whole static array; a diagonal-only BSR with nb = 2
    # keeps the inputs small (about 40 MB)
    from paper_1912_04385_gb300 import build, mss
    build.build()
    lib, h, calls, keep = _counting_handle(mss)
    try:
        n = 1 << 20
        nb = 2
        rp = torch.arange(n + 1, dtype=torch.int32, device="cuda")
        ci = torch.arange(n, dtype=torch.int32, device="cuda")
        g = torch.Generator(device="cpu").manual_seed(3)
        v = torch.randn(n * nb * nb, generator=g, dtype=torch.float64).cuda()
        b = torch.randn(n * nb, generator=g, dtype=torch.float64).cuda()
        x = torch.randn(n * nb, generator=g, dtype=torch.float64).cuda()
        J = mss.Bsr(n, n, rp.data_ptr(), ci.data_ptr(), v.data_ptr())
        ref = torch.empty(2, dtype=torch.float64, device="cuda")
        out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        assert lib.mss_residual_norm(h, C.byref(J), nb, b.data_ptr(), x.data_ptr(),
                                     ref.data_ptr()) == 0
        before = dict(calls)
        st = lib.mss_residual_norm_noalloc(h, C.byref(J), nb, b.data_ptr(), x.data_ptr(),
                                           out.data_ptr())
        assert st == 0, lib.mss_last_error(h)
        torch.cuda.synchronize()
        assert calls == before
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.abs(o - r) <= TOL * np.abs(r)), (o, r)
        # and against the definition, block by block on the host
        blocks = v.view(n, nb, nb).cpu().numpy()
        res = b.cpu().numpy().reshape(n, nb) - np.einsum("kij,kj->ki", blocks,
                                                         x.cpu().numpy().reshape(n, nb))
        assert abs(o[0] - np.linalg.norm(res)) <= TOL * np.linalg.norm(res)
    finally:
        lib.mss_destroy(h)
