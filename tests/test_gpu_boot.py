"""GPU parity of the ciphertext refresh (bootstrapping; Sec. 5, Evaluation
Methodology) against the oracle (oracle/boot.py): the sparse secret, the
conjugation, ModRaise and the plaintext-matrix product bit for bit, the whole
refresh bit for bit at N = 2^10, and a full-size refresh (N = 2^16, 24 primes of
50 bits) checked by decryption against the message."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402
from oracle import boot, ckks  # noqa: E402


def u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


def oracle_ct(pr, ct):
    return np.stack([ct.c0, ct.c1])


def to_gpu(cts):
    a = np.stack([oracle_ct(None, c) for c in cts]).view(np.int64)
    return torch.from_numpy(a.copy()).cuda()


@pytest.fixture(scope="module")
def small():
    """N = 2^10, 20 primes of 50 bits and 4 special primes, secret weight 32."""
    logN, n_q, k, bits, h = 10, 20, 4, 50, 32
    pr = ckks.Params(logN, n_q, k, bits)
    bp = boot.BootParams(pr, 3, 3, 6)  # default schedule: baby ratio 4, double hoisting
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(logN, n_q, k, bits)
        assert ctx.moduli == pr.moduli
        sk = ctx.sk_gen_sparse(11, h)
        torch.cuda.synchronize()
    keys = boot.SparseKeySet(pr, 11, h, rot_steps=boot.boot_rotation_steps(pr, bp), relin=True, conj=True)
    return pr, bp, ctx, sk, keys, s


def test_sparse_secret_equals_the_oracle(small):
    pr, bp, ctx, sk, keys, s = small
    assert np.array_equal(u64(sk), keys.sk.ntt)
    assert np.count_nonzero(keys.sk.coef) == 32


def test_mod_raise_and_conjugation_bit_exact(small):
    pr, bp, ctx, sk, keys, s = small
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, (2, pr.N // 2))
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, z[i], 0, 2.0 ** 45), 3, i) for i in range(2)]
    with torch.cuda.stream(s):
        evk = ctx.evk_gen(sk, 11, [fe.FE_STEP_CONJ], relin=False)
        raised = ctx.mod_raise(to_gpu(octs), 9)
        cj = ctx.conjugate(evk, raised, 9)
        torch.cuda.synchronize()
    want_r = [boot.mod_raise(pr, c, 9) for c in octs]
    assert np.array_equal(u64(raised), np.stack([oracle_ct(pr, c) for c in want_r]))
    want_c = [boot.conjugate(pr, keys, c) for c in want_r]
    assert np.array_equal(u64(cj), np.stack([oracle_ct(pr, c) for c in want_c]))


def test_plaintext_matrix_product_bit_exact(small):
    """Two inputs, two outputs, negative and positive offsets, a giant step of 0."""
    pr, bp, ctx, sk, keys, s = small
    n = pr.N // 2
    rng = np.random.default_rng(2)
    diags = {}
    for (o, i) in ((0, 0), (0, 1), (1, 0), (1, 1)):
        for r in (-12, -4, 0, 4, 8, 20):
            if (o + i + r) % 3:
                diags[(o, i, r)] = rng.uniform(-1, 1, n)
    n1, lv = 2, 7
    steps = boot.lintrans_steps(diags, n, n1)
    for st in steps:
        keys.add_rotation(st)
    zs = rng.uniform(-1, 1, (3, 2, n))
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, zs[q][i], lv, 2.0 ** 40), 5, 2 * q + i)
            for q in range(3) for i in range(2)]
    order = list(diags)
    with torch.cuda.stream(s):
        evk = ctx.evk_gen(sk, 11, steps, relin=False)
        plan = ctx.plan_lintrans(order, 2, 2, lv, n1=n1)
        assert sorted(x % n for x in plan.steps) == steps
        pt = ctx.lintrans_load(plan, np.stack([diags[k] for k in order]))
        got = u64(ctx.he_lintrans(evk, plan, pt, to_gpu(octs), n_req=3))
        torch.cuda.synchronize()
    for q in range(3):
        want = boot.he_lintrans(pr, keys, octs[2 * q:2 * q + 2], diags, 2, n1)
        assert np.array_equal(got[2 * q:2 * q + 2], np.stack([oracle_ct(pr, c) for c in want])), q


def test_refresh_bit_exact_against_the_oracle(small):
    """Two level-0 ciphertexts refreshed in one call equal the oracle's refresh of
    each, residue for residue, and decrypt to the messages."""
    pr, bp, ctx, sk, keys, s = small
    s_in = 2.0 ** 45
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, (2, pr.N // 2))
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, z[i], 0, s_in), 7, i) for i in range(2)]
    with torch.cuda.stream(s):
        b = ctx.boot_create(s_in, 3, 3, 6)
        assert sorted(x for x in b.steps if x != fe.FE_STEP_CONJ) == boot.boot_rotation_steps(pr, bp)
        assert fe.FE_STEP_CONJ in b.steps
        evk = ctx.evk_gen(sk, 11, b.steps, relin=True)
        out = ctx.bootstrap(evk, b, to_gpu(octs))
        got = u64(out)
        dec = ctx.decrypt(sk, out, b.out_level, b.out_scale).cpu().numpy()
        torch.cuda.synchronize()
    assert b.out_level == pr.L - bp.depth
    for i in range(2):
        want = boot.bootstrap(pr, keys, octs[i], bp)
        assert want.scale == b.out_scale and want.level == b.out_level
        assert np.array_equal(got[i], oracle_ct(pr, want)), i
    assert np.abs(dec - z).max() < 1e-4


@pytest.mark.parametrize("form", ["complex", "real"])
def test_refresh_graph_replays_the_direct_refresh(small, form):
    """fe_boot_graph_capture: one captured graph of the refresh of two
    ciphertexts (either transform form), replayed on two batches copied into its
    input buffer, gives the direct call's residues for each batch, and the
    oracle's."""
    pr, _, ctx, sk, keys, s = small
    bp = boot.BootParams(pr, 3, 3, 6, form=form)
    for st in boot.boot_rotation_steps(pr, bp):
        keys.add_rotation(st)
    s_in = 2.0 ** 45
    rng = np.random.default_rng(12)
    z = rng.uniform(-1, 1, (2, 2, pr.N // 2))
    octs = [[ckks.encrypt(pr, keys.sk, ckks.encode(pr, z[j][i], 0, s_in), 7, 10 + 2 * j + i) for i in range(2)]
            for j in range(2)]
    with torch.cuda.stream(s):
        b = ctx.boot_create(s_in, 3, 3, 6, form=form)
        evk = ctx.evk_gen(sk, 11, b.steps, relin=True)
        ws = ctx.workspace(b.workspace_bytes(2))
        x = to_gpu(octs[0])
        out = ctx.empty_ct(2, b.out_level)
        g = ctx.boot_graph_capture(evk, b, x, out, ws)
        (ib,), (ob,) = g.io()
        assert ib == x.numel() * 8 and ob == out.numel() * 8
        replayed = []
        for j in range(2):
            x.copy_(to_gpu(octs[j]))
            g.launch()
            replayed.append(u64(out).copy())
        direct = [u64(ctx.bootstrap(evk, b, to_gpu(octs[j]))) for j in range(2)]
        torch.cuda.synchronize()
    for j in range(2):
        assert np.array_equal(replayed[j], direct[j]), j
    want = boot.bootstrap(pr, keys, octs[1][0], bp)
    assert np.array_equal(replayed[1][0], oracle_ct(pr, want))


def test_caller_capture_of_the_refresh_replays_it(small):
    """A caller's own stream capture (torch.cuda.CUDAGraph) of fe_he_bootstrap:
    the per-call item tables travel in the graph by value, so replays on new
    inputs give the direct call's residues."""
    pr, bp, ctx, sk, keys, s = small
    s_in = 2.0 ** 45
    z = np.random.default_rng(13).uniform(-1, 1, (2, 1, pr.N // 2))
    with torch.cuda.stream(s):
        b = ctx.boot_create(s_in, 3, 3, 6)
        evk = ctx.evk_gen(sk, 11, b.steps, relin=True)
        ws = ctx.workspace(b.workspace_bytes(1))
        cts = [ctx.encrypt(sk, z[j], 0, s_in, seed=14 + j) for j in range(2)]
        direct = [ctx.bootstrap(evk, b, cts[j]).clone() for j in range(2)]
        x = cts[0].clone()
        out = ctx.empty_ct(1, b.out_level)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        g.capture_begin()
        ctx.bootstrap(evk, b, x, ws=ws, out=out)
        g.capture_end()
        replayed = []
        for j in range(2):
            x.copy_(cts[j])
            g.replay()
            replayed.append(out.clone())
        torch.cuda.synchronize()
    for j in range(2):
        assert torch.equal(replayed[j], direct[j]), j


@pytest.mark.parametrize("form", ["real", "complex"])
def test_refresh_full_size(form):
    """N = 2^16 with 24 primes of 50 bits and 4 special primes, secret weight 64:
    the refresh (both forms) returns at level 23 - 17 = 6 with every slot within
    1e-3 of the message (decrypted on the GPU), and its time is reported."""
    logN, n_q, k, bits = 16, 24, 4, 50
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(logN, n_q, k, bits)
        sk = ctx.sk_gen_sparse(21, 64)
        s_in = 2.0 ** 45
        b = ctx.boot_create(s_in, 3, 3, 6, form=form)
        evk = ctx.evk_gen(sk, 21, b.steps, relin=True)
        rng = np.random.default_rng(4)
        z = rng.uniform(-1, 1, (1, ctx.N // 2))
        ct = ctx.encrypt(sk, z, 0, s_in, seed=5)
        ws = ctx.workspace(b.workspace_bytes(1))
        out = ctx.bootstrap(evk, b, ct, ws=ws)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s)
        for _ in range(3):
            ctx.bootstrap(evk, b, ct, ws=ws, out=out)
        t1.record(s)
        torch.cuda.synchronize()
        dec = ctx.decrypt(sk, out, b.out_level, b.out_scale).cpu().numpy()
    assert b.out_level == 6
    err = float(np.abs(dec - z).max())
    print(f"refresh N=2^16 ({form} form): {t0.elapsed_time(t1) / 3:.2f} ms, max error {err:.2e}")
    assert err < 1e-3


@pytest.mark.parametrize("groups,r,ratio,double,form", [(3, 6, 1, False, "real"), (3, 6, 2, False, "real"),
                                                      (2, 5, 4, True, "real"), (3, 6, 4, True, "complex"),
                                                      (2, 5, 4, True, "complex"), (3, 6, 1, False, "complex")])
def test_refresh_schedules_bit_exact(small, groups, r, ratio, double, form):
    """Other baby / giant splits (n1^2 >= ratio x the offsets of each group),
    single-hoisted groups, and the 14-level refresh (two groups each way, five
    double angles) change every group's composition; the residues still equal
    the oracle's."""
    pr, bp, ctx, sk, keys, s = small
    bp2 = boot.BootParams(pr, groups, groups, r, baby_ratio=ratio, double_hoist=double, form=form)
    for st in boot.boot_rotation_steps(pr, bp2):
        keys.add_rotation(st)
    s_in = 2.0 ** 45
    z = np.random.default_rng(8).uniform(-1, 1, (1, pr.N // 2))
    oct_ = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z[0], 0, s_in), 9, 0)
    with torch.cuda.stream(s):
        b = ctx.boot_create(s_in, groups, groups, r, baby_ratio=ratio, double_hoist=double, form=form)
        assert sorted(x for x in b.steps if x != fe.FE_STEP_CONJ) == boot.boot_rotation_steps(pr, bp2)
        evk = ctx.evk_gen(sk, 11, b.steps, relin=True)
        got = u64(ctx.bootstrap(evk, b, to_gpu([oct_])))
        torch.cuda.synchronize()
    want = boot.bootstrap(pr, keys, oct_, bp2)
    assert b.out_level == want.level == pr.L - bp2.depth
    assert np.array_equal(got[0], oracle_ct(pr, want))


def _oracle_chain(pr, keys, cts, lay, w, act, delta, bp, scale_in):
    """The oracle's composition of RefreshChain: block, then (prepare, refresh,
    block) for each further block."""
    from oracle import henn
    a, b, c = act

    def block(h, lay_, wd, wp):
        lv = h[0].level
        h, l1 = henn.he_conv(pr, keys, h, lay_, wd, depthwise=True,
                             w_scale=henn.weight_scale(pr, lv, h[0].scale, delta, a))
        h = henn.he_poly_act(pr, keys, h, a, b, c)
        h, l2 = henn.he_conv(pr, keys, h, l1, wp, w_scale=henn.weight_scale(pr, lv - 2, h[0].scale, delta, a))
        return henn.he_poly_act(pr, keys, h, a, b, c), l2

    h, ly = block(cts, lay, *w[0])
    for wd, wp in w[1:]:
        h = [boot.bootstrap(pr, keys, boot.prepare(pr, ct, scale_in), bp) for ct in h]
        h, ly = block(h, ly, wd, wp)
    return h, ly


@pytest.mark.parametrize("n_blocks,n_q,H", [(2, 22, 6), (3, 23, 8)])
def test_refresh_chain_bit_exact_small(n_blocks, n_q, H):
    """Block (dw 3x3, activation, pw, activation), then prepare, refresh and
    block again, at N = 2^10 with n_q primes of 50 bits (two blocks and one
    refresh; three blocks and two refreshes, which need a fifth level after the
    refresh): every output residue equals the oracle's composition of the same
    steps, and the decryption matches FP64.  Each unpadded 3x3 depthwise
    convolution shrinks the H x H map by 2."""
    from oracle import fragment, henn, plain
    from paper_2606_16359_b300 import net
    logN, k, bits, h, C = 10, 4, 50, 32, 4
    pr = ckks.Params(logN, n_q, k, bits)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(logN, n_q, k, bits)
        ch = net.RefreshChain(ctx, H, C, h=h, key_seed=41, seed=5, n_blocks=n_blocks)
        assert len(ch.w) == n_blocks
        out = ch.forward()
        got = u64(out)
        y = ch.decrypt(out)
        torch.cuda.synchronize()
    bp = boot.BootParams(pr, 3, 3, 6)
    lay = fragment.Layout(pr.N, H, H, C, 1, 1)
    steps = set(boot.boot_rotation_steps(pr, bp))
    ly = lay
    for _ in range(n_blocks):
        steps |= set(henn.conv_rotation_steps(ly, C, C, 3, depthwise=True))
        ly = henn.out_layout_conv(ly, C, 3, 1)
        steps |= set(henn.conv_rotation_steps(ly, C, C, 1))
        ly = henn.out_layout_conv(ly, C, 1, 1)
    keys = boot.SparseKeySet(pr, 41, h, rot_steps=sorted(steps), relin=True, conj=True)
    slots = fragment.pack(lay, ch.x)
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, ch.delta), 7, i) for i in range(lay.n_ct)]
    want, lo = _oracle_chain(pr, keys, cts, lay, ch.w, ch.act, ch.delta, bp, 2.0 ** 44)
    assert want[0].level == ch.out_level and want[0].scale == ch.out_scale
    assert np.array_equal(got, np.stack([oracle_ct(pr, c) for c in want]))
    ref = ch.x
    for wd, wp in ch.w:
        ref = plain.poly_act(plain.conv2d(plain.poly_act(plain.conv2d(ref, wd, depthwise=True), *ch.act), wp),
                             *ch.act)
    assert np.abs(y - ref).max() < 1e-3


@pytest.mark.parametrize("encapsulate,n_blocks", [(False, 2), (True, 2), (True, 3)])
def test_refresh_chain_full_size(encapsulate, n_blocks):
    """The same chain at N = 2^16 (24 primes of 50 bits) on a 14 x 14 x 32 map,
    under a sparse secret of weight 64, or under a dense secret with the sparse
    one borrowed by the refresh; two blocks, or three with two refreshes (12
    convolution and activation levels on a 23-level chain): decrypted within
    1e-3 of the FP64 network."""
    from paper_2606_16359_b300 import net
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(16, 24, 4, 50)
        ch = net.RefreshChain(ctx, 14, 32, h=64, encapsulate=encapsulate, n_blocks=n_blocks)
        out = ch.forward()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s)
        out = ch.forward()
        t1.record(s)
        torch.cuda.synchronize()
        y = ch.decrypt(out)
    err = float(np.abs(y - ch.reference()).max())
    print(f"{n_blocks} blocks, {n_blocks - 1} refreshes at N=2^16 (encapsulated: {encapsulate}): "
          f"{t0.elapsed_time(t1):.1f} ms, max error {err:.2e}")
    assert ch.out_level == 2 and err < 1e-3


def test_refresh_chain_captured_as_one_graph():
    """The whole block-refresh-block network at N = 2^16 (dense secret,
    encapsulated refresh) captured by the caller as one CUDA graph
    (torch.cuda.CUDAGraph around RefreshChain.forward): every library call in it
    carries its per-call tables in the graph, so the replay gives the direct
    forward pass's residues; both times are reported."""
    from paper_2606_16359_b300 import net
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(16, 24, 4, 50)
        ch = net.RefreshChain(ctx, 14, 32, h=64, encapsulate=True)
        want = ch.forward()
        for _ in range(2):
            ch.forward()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s)
        for _ in range(3):
            ch.forward()
        t1.record(s)
        torch.cuda.synchronize()
        ms_direct = t0.elapsed_time(t1) / 3
        g = torch.cuda.CUDAGraph()
        g.capture_begin()
        got = ch.forward()
        g.capture_end()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        t0.record(s)
        for _ in range(3):
            g.replay()
        t1.record(s)
        torch.cuda.synchronize()
        ms_graph = t0.elapsed_time(t1) / 3
        assert torch.equal(got, want)
    print(f"block + refresh + block at N=2^16, dense secret: {ms_direct:.1f} ms direct, {ms_graph:.1f} ms as one graph")


def test_refresh_steps_bit_exact_at_full_size():
    """At the refresh's full parameter set (N = 2^16, 24 + 4 primes of 50 bits,
    secret weight 64), the steps the oracle can afford there are compared
    residue for residue: the sparse secret on all 28 moduli, ModRaise of a
    level-0 ciphertext to level 23, and its conjugation (one key switch)."""
    logN, n_q, k, bits, h = 16, 24, 4, 50, 64
    pr = ckks.Params(logN, n_q, k, bits)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(logN, n_q, k, bits)
        assert ctx.moduli == pr.moduli
        sk = ctx.sk_gen_sparse(51, h)
        evk = ctx.evk_gen(sk, 51, [fe.FE_STEP_CONJ], relin=False)
        torch.cuda.synchronize()
    keys = boot.SparseKeySet(pr, 51, h, conj=True)
    assert np.array_equal(u64(sk), keys.sk.ntt)
    z = np.random.default_rng(13).uniform(-1, 1, pr.N // 2)
    oct_ = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 0, 2.0 ** 45), 14, 0)
    with torch.cuda.stream(s):
        raised = ctx.mod_raise(to_gpu([oct_]), pr.L)
        cj = ctx.conjugate(evk, raised, pr.L)
        torch.cuda.synchronize()
    want_r = boot.mod_raise(pr, oct_, pr.L)
    assert np.array_equal(u64(raised)[0], oracle_ct(pr, want_r))
    assert np.array_equal(u64(cj)[0], oracle_ct(pr, boot.conjugate(pr, keys, want_r)))


def test_encapsulated_refresh_bit_exact():
    """Sparse-secret encapsulation at N = 2^10: a dense secret (fe_sk_gen) for the
    ciphertext and the refresh's keys, a sparse one (weight 32) borrowed for
    ModRaise; the generic key switch and the refresh equal the oracle's, and so
    does the refresh captured as one graph and run through host buffers."""
    logN, n_q, k, bits, h = 10, 20, 4, 50, 32
    pr = ckks.Params(logN, n_q, k, bits)
    bp = boot.BootParams(pr, 3, 3, 6)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(logN, n_q, k, bits)
        sk = ctx.sk_gen(61)
        sp = ctx.sk_gen_sparse(62, h)
        b = ctx.boot_create(2.0 ** 45)
        ctx.boot_encapsulate(b, sk, sp, 61)
        evk = ctx.evk_gen(sk, 61, b.steps, relin=True)
        torch.cuda.synchronize()
    keys = ckks.KeySet(pr, 61, rot_steps=boot.boot_rotation_steps(pr, bp), relin=True)
    boot.add_conjugation(keys)
    enc = boot.Encapsulation(keys, 62, h)
    z = np.random.default_rng(15).uniform(-1, 1, pr.N // 2)
    oct_ = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 0, 2.0 ** 45), 16, 0)
    lv = 5
    octs5 = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, lv, 2.0 ** 45), 17, 0)
    with torch.cuda.stream(s):
        ks = u64(ctx.key_switch(b.encaps_keys[:b.encaps_keys.numel() // 2], to_gpu([octs5]), lv))
        got = u64(ctx.bootstrap(evk, b, to_gpu([oct_])))
        # the same refresh as one captured graph (its two key switches carry their
        # tables in the graph), run through host buffers
        x = to_gpu([oct_])
        y = ctx.empty_ct(1, b.out_level)
        g = ctx.boot_graph_capture(evk, b, x, y, ctx.workspace(b.workspace_bytes(1)))
        h_in = x.cpu().pin_memory()
        h_out = torch.empty(y.numel(), dtype=torch.int64).pin_memory()
        x.zero_()
        g.launch_host([h_in], [h_out])
        torch.cuda.synchronize()
        got_graph = h_out.numpy().view(np.uint64).reshape(got.shape)
    assert np.array_equal(ks[0], oracle_ct(pr, boot.key_switch(pr, octs5, enc.to_sparse)))
    want = boot.bootstrap(pr, keys, oct_, bp, encaps=enc)
    assert np.array_equal(got[0], oracle_ct(pr, want))
    assert np.array_equal(got_graph, got)
    assert np.abs(ckks.decrypt(pr, keys.sk, want) - z).max() < 1e-4
