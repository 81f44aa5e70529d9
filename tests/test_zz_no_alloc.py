"""The allocation-free rescale (fe_rescale_noalloc) against the regular one.

Callers that cannot allocate device memory -- a serving process with a fixed
device footprint, a host framework that owns all device memory, latency-critical
code that cannot afford an allocation -- use fe_rescale_noalloc, whose scratch is
a fixed static device array.  This test calls it through the C ABI twice in a
row (the second call reuses the array left over from the first) and requires the
same residues as fe_rescale, bit for bit.  It lives in its own file, collected
last, and creates its own context so that it passes alone or after other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402


def _u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


def _noalloc(ctx, ct, level):
    out = ctx.empty_ct(ct.shape[0], level - 1)
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
