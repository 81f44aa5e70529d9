"""The allocation-free rescale (fe_rescale_noalloc) against the regular one.

Callers that cannot allocate device memory -- a serving process with a fixed
device footprint, a host framework that owns all device memory, latency-critical
code that cannot afford an allocation -- use fe_rescale_noalloc, whose scratch is
a fixed static device array.  This test calls it through the C ABI twice in a
row (the second call reuses the array left over from the first) and requires the
same residues as fe_rescale, bit for bit.  Around a warmed-up call it also
checks the property the entry point exists for: the device's stream-ordered
memory pool (which fe_rescale draws on) sees no allocation -- its used-memory
high watermark stays at the current use -- and PyTorch's allocator makes none
either; fe_rescale, under the same watch, does raise the watermark.  It lives
in its own file, collected last, and creates its own context so that it passes
alone or after other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402


class PoolWatch:
    """Used-memory high watermark of the current device's default stream-ordered
    pool (cudaMallocAsync draws on it), reset to the current use on entry."""

    def __init__(self):
        from cuda.bindings import driver, runtime
        self.rt, self.drv = runtime, driver
        err, self.pool = runtime.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
        assert err == runtime.cudaError_t.cudaSuccess

    def _get(self, attr):
        err, v = self.rt.cudaMemPoolGetAttribute(self.pool, attr)
        assert err == self.rt.cudaError_t.cudaSuccess
        return int(v)

    def __enter__(self):
        A = self.rt.cudaMemPoolAttr
        torch.cuda.synchronize()
        self.used0 = self._get(A.cudaMemPoolAttrUsedMemCurrent)
        err, = self.rt.cudaMemPoolSetAttribute(self.pool, A.cudaMemPoolAttrUsedMemHigh, self.drv.cuuint64_t(0))
        assert err == self.rt.cudaError_t.cudaSuccess
        self.torch0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        return self

    def __exit__(self, *exc):
        torch.cuda.synchronize()
        A = self.rt.cudaMemPoolAttr
        self.high = self._get(A.cudaMemPoolAttrUsedMemHigh)
        self.torch_allocs = torch.cuda.memory_stats().get("allocation.all.allocated", 0) - self.torch0
        return False


def _u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


def _noalloc(ctx, ct, level, out=None):
    out = ctx.empty_ct(ct.shape[0], level - 1) if out is None else out
    rc = fe.load().fe_rescale_noalloc(ctx.handle, ctypes.c_void_p(ct.data_ptr()), ct.shape[0], level,
                                      ctypes.c_void_p(out.data_ptr()), fe._stream())
    fe.check(rc)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("args,n_ct,level", [((13, 3, 1, 30, 50), 4, 2), ((16, 24, 4, 36, 36), 1, 23)])
def test_rescale_noalloc_matches_rescale_on_two_calls(args, n_ct, level):
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(*args)
        sk = ctx.sk_gen(5)
        rng = np.random.default_rng(level)
        outs = []
        for call in range(2):
            z = torch.from_numpy(rng.uniform(-1, 1, (n_ct, ctx.N // 2)))
            ct = ctx.encrypt(sk, z, level, 2.0 ** 25, seed=10 + call)
            want = _u64(ctx.rescale(ct, level))
            got = _u64(_noalloc(ctx, ct, level))
            assert np.array_equal(got, want), f"call {call}"
            outs.append(got)
        assert not np.array_equal(outs[0], outs[1])
        # a warmed-up call allocates nothing; the regular rescale does, under the same watch
        out = ctx.empty_ct(n_ct, level - 1)
        with PoolWatch() as w:
            _noalloc(ctx, ct, level, out)
        assert w.high == w.used0 and w.torch_allocs == 0
        assert np.array_equal(_u64(out), outs[1])
        with PoolWatch() as w:
            fe.check(fe.load().fe_rescale(ctx.handle, ctypes.c_void_p(ct.data_ptr()), n_ct, level,
                                          ctypes.c_void_p(out.data_ptr()), fe._stream()))
        assert w.high > w.used0


def test_rescale_noalloc_rejects_oversized_requests():
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(16, 24, 4, 36, 36)
        ct = ctx.empty_ct(2, 23)
        out = ctx.empty_ct(2, 22)
        rc = fe.load().fe_rescale_noalloc(ctx.handle, ctypes.c_void_p(ct.data_ptr()), 2, 23,
                                          ctypes.c_void_p(out.data_ptr()), fe._stream())
        assert rc == fe.FE_ENOMEM
        assert b"32" in fe.load().fe_last_error() or b"static" in fe.load().fe_last_error()
