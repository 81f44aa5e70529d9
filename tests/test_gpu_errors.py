"""The C ABI's error contract on a GPU.

Every call validates its arguments before it launches anything and returns an
int status (FE_EINVAL, FE_ELEVEL, FE_EKEY, FE_ENOMEM, ...) with a message in
fe_last_error(); no kernel traps.  After a rejected call the context, its keys
and the stream stay usable, and the device status word stays clear.  Calls on
an empty batch (n_ct = 0) succeed and touch nothing.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402
from oracle import plain  # noqa: E402

P = fe._ptr


@pytest.fixture(scope="module")
def g():
    return fe.Context(10, 3, 1, 30, 50)


@pytest.fixture(scope="module")
def keys(g):
    sk = g.sk_gen(21)
    return sk, g.evk_gen(sk, 21, [1])


def _slots(g, n, seed):
    return torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, (n, g.N // 2)))


def test_empty_batches_succeed_and_touch_nothing(g, keys):
    sk, evk = keys
    lib, s = fe.load(), fe._stream()
    src = g.encrypt(sk, _slots(g, 1, 1), g.L, 2.0 ** 25, seed=1)
    out = g.empty_ct(1, g.L)
    out.fill_(7)
    slots = torch.full((1, g.N // 2), 3.0, dtype=torch.float64, device="cuda")
    assert lib.fe_rescale(g.handle, P(src), 0, g.L, P(out), s) == fe.FE_OK
    assert lib.fe_rescale_noalloc(g.handle, P(src), 0, g.L, P(out), s) == fe.FE_OK
    assert lib.fe_rotate(g.handle, evk.handle, P(src), 0, g.L, 1, P(out), s) == fe.FE_OK
    assert lib.fe_pmult(g.handle, P(src), P(src), 0, g.L, P(out), s) == fe.FE_OK
    assert lib.fe_add(g.handle, P(src), P(src), 0, g.L, P(out), s) == fe.FE_OK
    assert lib.fe_encode_encrypt(g.handle, P(sk), P(slots), 0, g.L, 2.0 ** 25, 5, 0, P(out), s) == fe.FE_OK
    assert lib.fe_decrypt_decode(g.handle, P(sk), P(src), 0, g.L, 2.0 ** 25, P(slots), s) == fe.FE_OK
    ws = g.workspace(1 << 16)
    sc = ctypes.c_double()
    assert lib.fe_he_poly_act(g.handle, evk.handle, 0.0, 0.5, 0.25, P(src), 0, g.L, 2.0 ** 25, P(out),
                              ctypes.byref(sc), P(ws), ws.numel() * 8, s) == fe.FE_OK
    lay = g.layout(4, 4, 1, 1, 1)
    assert lib.fe_compress_masked(g.handle, evk.handle, ctypes.byref(lay), 1, 2.0 ** 20, P(src), 0, g.L, 2.0 ** 25,
                                  P(out), ctypes.byref(sc), P(ws), ws.numel() * 8, s) == fe.FE_OK
    torch.cuda.synchronize()
    assert bool((out == 7).all()) and bool((slots == 3.0).all())
    assert g.device_status() == 0


def test_rejected_calls_return_their_status_and_leave_the_context_usable(g, keys):
    sk, evk = keys
    lib, s = fe.load(), fe._stream()
    z = _slots(g, 1, 2)
    ct = g.encrypt(sk, z, g.L, 2.0 ** 25, seed=2)
    out = g.empty_ct(1, g.L)
    misaligned = ctypes.c_void_p(ct.data_ptr() + 8)
    cases = [
        ("rescale at level 0", lambda: lib.fe_rescale(g.handle, P(ct), 1, 0, P(out), s), fe.FE_ELEVEL),
        ("rescale above L", lambda: lib.fe_rescale(g.handle, P(ct), 1, g.L + 1, P(out), s), fe.FE_ELEVEL),
        ("rotation without its key", lambda: lib.fe_rotate(g.handle, evk.handle, P(ct), 1, g.L, 2, P(out), s),
         fe.FE_EKEY),
        ("misaligned input", lambda: lib.fe_rotate(g.handle, evk.handle, misaligned, 1, g.L, 1, P(out), s),
         fe.FE_EINVAL),
        ("misaligned rescale", lambda: lib.fe_rescale(g.handle, misaligned, 1, g.L, P(out), s), fe.FE_EINVAL),
        ("null context", lambda: lib.fe_rescale(None, P(ct), 1, g.L, P(out), s), fe.FE_EINVAL),
        ("no-alloc rescale at level 0", lambda: lib.fe_rescale_noalloc(g.handle, P(ct), 1, 0, P(out), s),
         fe.FE_ELEVEL),
        ("hoisted rotations in place", lambda: lib.fe_rotate_many(g.handle, evk.handle, P(ct), 1, g.L,
                                                                  (ctypes.c_int32 * 2)(1, 1), 2, P(ct), s),
         fe.FE_EINVAL),
        ("hoisted rotation without its key", lambda: lib.fe_rotate_many(g.handle, evk.handle, P(ct), 1, g.L,
                                                                        (ctypes.c_int32 * 2)(1, 2), 2, P(out), s),
         fe.FE_EKEY),
    ]
    # every call that takes device buffers rejects a misaligned one before launching
    slots = torch.zeros((2, g.N // 2), dtype=torch.float64, device="cuda")
    bad_slots = ctypes.c_void_p(slots.data_ptr() + 8)
    lay = g.layout(4, 4, 1, 1, 2)
    out_lay = fe.FeLayout()
    cases += [
        ("misaligned pmult", lambda: lib.fe_pmult(g.handle, misaligned, P(ct), 1, g.L, P(out), s), fe.FE_EINVAL),
        ("misaligned add", lambda: lib.fe_add(g.handle, P(ct), misaligned, 1, g.L, P(out), s), fe.FE_EINVAL),
        ("misaligned encode", lambda: lib.fe_encode(g.handle, bad_slots, 1, g.L, 2.0 ** 25, P(out), s), fe.FE_EINVAL),
        ("misaligned encrypt", lambda: lib.fe_encode_encrypt(g.handle, P(sk), bad_slots, 1, g.L, 2.0 ** 25, 5, 0,
                                                             P(out), s), fe.FE_EINVAL),
        ("misaligned decrypt", lambda: lib.fe_decrypt_decode(g.handle, P(sk), P(ct), 1, g.L, 2.0 ** 25, bad_slots, s),
         fe.FE_EINVAL),
        ("misaligned pack", lambda: lib.fe_fragment_pack(g.handle, ctypes.byref(lay), bad_slots, P(slots), s),
         fe.FE_EINVAL),
        ("misaligned unpack", lambda: lib.fe_fragment_unpack(g.handle, ctypes.byref(lay), bad_slots, P(slots), s),
         fe.FE_EINVAL),
        ("misaligned pool", lambda: lib.fe_he_avgpool(g.handle, ctypes.byref(lay), misaligned, g.L, P(out),
                                                      ctypes.byref(out_lay), s), fe.FE_EINVAL),
    ]
    for name, call, code in cases:
        assert call() == code, name
        assert lib.fe_last_error(), name
    assert lib.fe_rotate(g.handle, evk.handle, P(ct), 1, g.L, 2, P(out), s) == fe.FE_EKEY
    assert b"step 2" in lib.fe_last_error()
    torch.cuda.synchronize()
    assert g.device_status() == 0
    # the context, its keys and the stream still work: Rot(z, 1) decrypts to z shifted left by one slot
    y = g.decrypt(sk, g.rotate(evk, ct, g.L, 1), g.L, 2.0 ** 25).cpu().numpy()
    assert np.abs(y - np.roll(z.numpy(), -1, axis=1)).max() < 1e-3


def test_layer_planning_and_evaluation_errors(g, keys):
    sk, evk = keys
    lay = g.layout(6, 6, 2, 1, 4)
    for kw, code in [(dict(Cout=3, K=7), fe.FE_EINVAL),               # kernel larger than the map
                     (dict(Cout=3, K=0), fe.FE_EINVAL),               # empty kernel
                     (dict(Cout=3, K=3, stride=3), fe.FE_EINVAL),     # stride other than 1 or 2
                     (dict(Cout=5, K=3, depthwise=True), fe.FE_EINVAL),  # depthwise changes C
                     (dict(Cout=3, K=3, level=0), fe.FE_ELEVEL)]:     # no level to rescale
        with pytest.raises(fe.FencError) as e:
            g.plan_conv(lay, **kw)
        assert e.value.code == code, kw
    with pytest.raises(fe.FencError) as e:
        g.plan_conv(g.layout(6, 6, 2, 1, 3), 3, 3, stride=2)           # stride 2 needs an even S
    assert e.value.code == fe.FE_EINVAL
    plan = g.plan_conv(lay, 3, 3)
    w = np.random.default_rng(3).normal(0, 0.3, (3, 2, 3, 3))
    pt = g.load_weights(plan, w, float(g.moduli[g.L]))
    ct = g.encrypt(sk, g.pack(lay, torch.from_numpy(np.random.default_rng(4).uniform(0, 1, (1, 2, 6, 6)))),
                   g.L, 2.0 ** 25, seed=3)
    # the evk holds only step 1; the plan needs others
    with pytest.raises(fe.FencError) as e:
        g.he_conv(evk, plan, pt, ct)
    assert e.value.code == fe.FE_EKEY
    full = g.evk_gen(sk, 21, plan.steps)
    with pytest.raises(fe.FencError) as e:
        g.he_conv(full, plan, pt, ct, ws=g.workspace(64))
    assert e.value.code == fe.FE_ENOMEM
    with pytest.raises(fe.FencError) as e:
        g.he_conv(full, plan, pt, ct, mode=3)
    assert e.value.code == fe.FE_EINVAL
    torch.cuda.synchronize()
    assert g.device_status() == 0
    # and the same plan runs once its keys and workspace are there
    y = g.unpack(plan.out_layout, g.decrypt(sk, g.he_conv(full, plan, pt, ct), g.L - 1, 2.0 ** 25)).cpu().numpy()
    x = np.random.default_rng(4).uniform(0, 1, (1, 2, 6, 6))
    assert np.abs(y - plain.conv2d(x, w)).max() < 1e-3


def test_mac_wait_expiry_sets_the_status_and_leaves_the_context_usable(g, keys):
    """The PMult-MAC's bounded waits, made to run out on purpose: every MAC item
    announces the bytes of its first term but no copy for it is issued, so that
    stage never fills.  With a 1 ms limit the consumers give up, set bit 0 of the
    status word and stop; the producer waits (bounded) for the copies it did
    issue.  Afterwards, with the default limit back, the same layer on the same
    context and stream gives the residues of a clean run, and a rotation
    decrypts correctly."""
    sk, evk = keys
    lay = g.layout(6, 6, 2, 1, 2)
    plan = g.plan_conv(lay, 3, 3)
    w = np.random.default_rng(5).normal(0, 0.3, (3, 2, 3, 3))
    pt = g.load_weights(plan, w, float(g.moduli[g.L]))
    x = np.random.default_rng(6).uniform(0, 1, (1, 2, 6, 6))
    ct = g.encrypt(sk, g.pack(lay, torch.from_numpy(x)), g.L, 2.0 ** 25, seed=4)
    full = g.evk_gen(sk, 22, plan.steps)
    clean = g.he_conv(full, plan, pt, ct).cpu().numpy().view(np.uint64).copy()
    torch.cuda.synchronize()
    assert g.device_status() == 0
    try:
        g.set_mac_wait(1_000_000, 0)
        g.he_conv(full, plan, pt, ct)
        assert g.device_status(reset=True) & 1 == 1
    finally:
        g.set_mac_wait()
    assert g.device_status() == 0
    again = g.he_conv(full, plan, pt, ct).cpu().numpy().view(np.uint64)
    assert np.array_equal(again, clean)
    y = g.unpack(plan.out_layout, g.decrypt(sk, g.he_conv(full, plan, pt, ct), g.L - 1, 2.0 ** 25)).cpu().numpy()
    assert np.abs(y - plain.conv2d(x, w)).max() < 1e-3
    z = _slots(g, 1, 9)
    zc = g.encrypt(sk, z, g.L, 2.0 ** 25, seed=8)
    yr = g.decrypt(sk, g.rotate(evk, zc, g.L, 1), g.L, 2.0 ** 25).cpu().numpy()
    assert np.abs(yr - np.roll(z.numpy(), -1, axis=1)).max() < 1e-3
    assert g.device_status() == 0
    with pytest.raises(fe.FencError):
        g.set_mac_wait(0, -1)


def test_error_contract_of_the_layers_added_around_the_convolution(g, keys):
    """The activation, masked AAC, scale rule, block-size change, token layout
    and attention calls return their status before any launch, and the
    context stays usable."""
    sk, evk = keys
    lib, s = fe.load(), fe._stream()
    ct = g.encrypt(sk, _slots(g, 1, 12), g.L, 2.0 ** 25, seed=12)
    out = g.empty_ct(1, g.L)
    ws = g.workspace(1 << 20)
    sc = ctypes.c_double()
    # activation: level 0, non-finite coefficient, a != 0 without a relinearisation key
    assert lib.fe_he_poly_act(g.handle, evk.handle, 1.0, 0.0, 0.0, P(ct), 1, 0, 2.0 ** 25, P(out), ctypes.byref(sc),
                              P(ws), ws.numel() * 8, s) == fe.FE_ELEVEL
    assert lib.fe_he_poly_act(g.handle, evk.handle, float("nan"), 0.0, 0.0, P(ct), 1, g.L, 2.0 ** 25, P(out),
                              ctypes.byref(sc), P(ws), ws.numel() * 8, s) == fe.FE_EINVAL
    assert lib.fe_he_poly_act(g.handle, evk.handle, 1.0, 0.0, 0.0, P(ct), 1, g.L, 2.0 ** 25, P(out),
                              ctypes.byref(sc), P(ws), ws.numel() * 8, s) == fe.FE_EKEY
    # masked AAC: a mask scale below 1
    lay = g.layout(4, 4, 1, 1, 1)
    assert lib.fe_compress_masked(g.handle, evk.handle, ctypes.byref(lay), 1, 0.5, P(ct), 1, g.L, 2.0 ** 25, P(out),
                                  ctypes.byref(sc), P(ws), ws.numel() * 8, s) == fe.FE_EINVAL
    # scale rule and plan scales
    assert lib.fe_weight_scale(g.handle, 0, 1.0, 1.0, 0.0, ctypes.byref(sc)) == fe.FE_ELEVEL
    assert lib.fe_poly_act_scale(g.handle, g.L, -1.0, 1.0, ctypes.byref(sc)) == fe.FE_EINVAL
    plan = g.plan_conv(g.layout(6, 6, 2, 1, 2), 3, 3)
    assert lib.fe_plan_out_scale(plan.handle, 1.0, ctypes.byref(sc)) == fe.FE_EINVAL  # weights not loaded
    # block-size change between layouts of different maps
    h = ctypes.c_void_p()
    la, lb = g.layout(6, 6, 2, 1, 2), g.layout(6, 6, 3, 1, 1)
    assert lib.fe_plan_repack(g.handle, ctypes.byref(la), ctypes.byref(lb), g.L, ctypes.byref(h)) == fe.FE_EINVAL
    # token layout that does not fit, attention without its keys
    bad = fe.FeTokenLayout(4, 4000, 2, 0, 0, 0)
    assert lib.fe_token_layout_make(g.handle, ctypes.byref(bad)) == fe.FE_EINVAL
    tl = g.token_layout(4, 16, 2)
    relin_only = g.evk_gen(sk, 21, [1], relin=True)
    assert lib.fe_he_attention_scores(g.handle, relin_only.handle, ctypes.byref(tl), P(ct), P(ct), g.L, 1.0, 1.0,
                                      P(out), ctypes.byref(sc), s) == fe.FE_EKEY
    # wait limits out of range
    assert lib.fe_ctx_set_mac_wait(g.handle, 0, -1) == fe.FE_EINVAL
    assert lib.fe_ctx_set_mac_wait(g.handle, 1000, -2) == fe.FE_EINVAL
    torch.cuda.synchronize()
    assert g.device_status() == 0
    # still usable: the affine case a = 0 needs no relinearisation key
    z = _slots(g, 1, 13)
    c2 = g.encrypt(sk, z, g.L, 2.0 ** 25, seed=13)
    o, osc = g.he_poly_act(evk, c2, g.L, 2.0 ** 25, 0.0, 0.5, 0.25)
    y = g.decrypt(sk, o, g.L - 1, osc).cpu().numpy()
    assert np.abs(y - (0.5 * z.numpy() + 0.25)).max() < 1e-3
