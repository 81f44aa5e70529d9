"""Encrypted layers under the fragment encoding: HE convolution (Sec. 3.1, Eq. 2
with inner and outer rotations), x^2 activation, 2x2 average pooling, fully
connected layers, Arch-aware Ciphertext Compression (AAC), and the LeNet-shaped
network built from them.

Test infrastructure only (see oracle/__init__.py).

HE convolution (the algorithm, in the order it is evaluated here):
 1. Inner rotations (spatial dependency, Sec. 3.1 inner rotations, Eq. 3):
    output pixel (h, w) = (bi S + u', bj S + v') sits in the slot of input pixel
    (h, w).  Tap (i, j) reads input pixel (h + i, w + j), which lives in input
    fragment u = (u' + i) mod S at block row bi + a, a = (u' + i) div S (same for
    columns).  Every input ciphertext is therefore rotated by
    r = (a m + b) BS for each needed block offset (a, b) != (0, 0); the ModUp of
    its c1 is computed once and shared by all of its rotations (hoisting).
 2. PMult-MAC over fragment masks (Fig. 2): for output ciphertext (group h,
    fragment (u', v')) and diagonal d, P_d = sum_g sum_taps R ⊙ pt, where pt
    holds W[o][c][i][j] in the slots of input channel position c_loc for output
    channel position o_loc = (c_loc - d) mod cpc, and zero at every output
    position that is not a valid output of the (strided) valid convolution.
 3. Outer rotations (channel dependency, Eq. 4): out = P_0 + sum_{d != 0}
    Rot(P_d, d m^2 BS), before any rescale; all-zero diagonals are skipped.
    An output with no nonzero term at all (its fragment holds no valid output
    position, or every weight it reads is zero) is an empty sum: the zero
    ciphertext.
 4. One rescale.
Weights are encoded at scale q_level by default, so the output scale equals the
input scale.  Stride 2 keeps the output fragments with even (u', v') and halves S
(Sec. 5, Implementation paragraph: stride by discarding ciphertexts).
"""
import math

import numpy as np

from . import _core as C
from . import ckks
from . import counts
from .fragment import Layout, TokenLayout


class Counters:
    def __init__(self):
        self.rot = 0
        self.keyswitch = 0
        self.pmult = 0
        self.cmult = 0
        self.rescale = 0
        self.modup = 0
        self.moddown = 0  # ModDowns of partial sums under double hoisting

    def as_dict(self):
        return dict(self.__dict__)


def _add(pr, acc, x):
    if acc is None:
        return x.copy()
    return ckks.add(pr, acc, x)


def _empty_sum(pr, level, scale):
    """An output ciphertext none of whose terms has a nonzero plaintext (its
    fragment holds no valid output position, or every weight it reads is zero):
    the sum of step 3 is empty, so the output is the zero ciphertext, at the
    level and scale that the rescaled sum would have had."""
    z = np.zeros((level, pr.N), dtype=np.uint64)
    return ckks.Ciphertext(z, z.copy(), level - 1, scale / pr.moduli[level])


def out_layout_conv(lay, Cout, K, stride):
    if lay.S % stride and lay.S != 1:
        raise ValueError("stride must divide S")
    if stride != 1 and lay.S == 1:
        raise ValueError("stride > 1 needs S >= 2 (stride by discarding fragments)")
    Ho = (lay.H - K) // stride + 1
    Wo = (lay.W - K) // stride + 1
    return Layout(lay.N, Ho, Wo, Cout, lay.BS, lay.S // stride, m=lay.m)


def conv_diagonals(lay, Cin, Cout, h, depthwise, in_period):
    cpc = lay.cpc
    if depthwise:
        return [0]
    if in_period is not None:
        return list(range(in_period))
    ds = set()
    for c in range(Cin):
        for o_loc in range(cpc):
            if h * cpc + o_loc < Cout:
                ds.add(((c % cpc) - o_loc) % cpc)
    return sorted(ds)


def bsgs_split(lay, n1, depthwise=False, in_period=None):
    """Baby-step count actually used: n1 clipped to cpc; 0 (linear outer
    rotations) for depthwise or replicated-input layers and for cpc = 1."""
    if not n1 or depthwise or in_period is not None or lay.cpc <= 1:
        return 0
    return min(n1, lay.cpc)


def conv_rotation_steps(lay, Cin, Cout, K, stride=1, depthwise=False, in_period=None, bsgs_n1=0):
    offs = counts.inner_offsets(lay.S, K, stride)
    G_out = lay.groups if depthwise else -(-Cout // lay.cpc)
    n1 = bsgs_split(lay, bsgs_n1, depthwise, in_period)
    babies = {0}
    if n1:
        for h in range(G_out):
            babies |= {d % n1 for d in conv_diagonals(lay, Cin, Cout, h, depthwise, in_period)}
    steps = set()
    for u in range(lay.S):
        for v in range(lay.S):
            for a in offs[u]:
                for b in offs[v]:
                    for i in babies:
                        if (a, b, i) != (0, 0, 0):
                            steps.add((a * lay.m + b) * lay.BS + i * lay.blk)
    for h in range(G_out):
        for d in conv_diagonals(lay, Cin, Cout, h, depthwise, in_period):
            if n1:
                if d >= n1:
                    steps.add((d // n1) * n1 * lay.blk)
            elif d:
                steps.add(d * lay.blk)
    return sorted(steps)


def conv_weight_slots(lay, W, h, up, vp, d, g, i, j, *, stride, depthwise, in_period, wmul, Cout):
    """Slot vector of the plaintext for output (group h, fragment (up, vp)),
    diagonal d, input group g, tap (i, j)."""
    K = W.shape[-1]
    Cin = W.shape[1] if not depthwise else W.shape[0]
    z = np.zeros(lay.N // 2, dtype=np.float64)
    cpc = lay.cpc
    for c_loc in range(cpc):
        if in_period is not None:
            c = c_loc % in_period
        else:
            c = g * cpc + c_loc
            if c >= Cin:
                continue
        o_loc = (c_loc - d) % cpc
        o = h * cpc + o_loc
        if o >= Cout:
            continue
        if depthwise:
            if o != c:
                continue
            wv = W[c, 0, i, j]
        else:
            wv = W[o, c, i, j]
        wv = wv * wmul
        for bi in range(lay.m):
            hp = bi * lay.S + up
            if hp > lay.H - K:
                break
            if hp % stride:
                continue
            for bj in range(lay.m):
                wp = bj * lay.S + vp
                if wp > lay.W - K:
                    break
                if wp % stride:
                    continue
                base = lay.slot(c_loc, bi, bj, 0)
                z[base:base + lay.BS] = wv
    return z


def he_conv(pr, keys, cts, lay, W, *, stride=1, depthwise=False, in_period=None, wmul=1.0,
            w_scale=None, cnt=None, bsgs_n1=0, hoist="single"):
    """Encrypted convolution of the fragment-packed input `cts` (list in (g, u, v)
    order).  Returns (output ciphertexts in (h, u'', v'') order, output layout).
    bsgs_n1 > 0 selects the baby-step / giant-step schedule of the outer
    rotations (he_conv_bsgs).  hoist="double" keeps the inner rotations on the
    key-switching basis Q_level * P and performs one ModDown per partial sum
    P_d instead of one per rotation (double hoisting): P_d = ModDown(sum of
    V (x) pt) with V = sigma((P c0, 0) + key inner product) for a rotated source
    and V = P x for an unrotated one, plaintexts encoded on Q_level * P.
    hoist="double_fused": as "double", and when the layer has no outer rotation
    every output is its one partial sum divided by q_level P in one step
    (ckks.mod_down_rescale) instead of ModDown then rescale."""
    if bsgs_split(lay, bsgs_n1, depthwise, in_period):
        return he_conv_bsgs(pr, keys, cts, lay, W, stride=stride, wmul=wmul, w_scale=w_scale, cnt=cnt,
                            n1=bsgs_n1, hoist=hoist)
    double = hoist in ("double", "double_fused")
    cnt = cnt if cnt is not None else Counters()
    level = cts[0].level
    Cout = W.shape[0]
    Cin = W.shape[0] if depthwise else W.shape[1]
    K = W.shape[-1]
    olay = out_layout_conv(lay, Cout, K, stride)
    S, m, BS = lay.S, lay.m, lay.BS
    dw = float(pr.moduli[level]) if w_scale is None else w_scale
    G_in = 1 if in_period is not None else lay.groups
    G_out = olay.groups

    # 1. inner rotations, hoisted per input ciphertext
    offs = counts.inner_offsets(S, K, stride)
    R = {}
    for g in range(G_in):
        for u in range(S):
            for v in range(S):
                ct = cts[lay.ct_index(g, u, v)]
                pairs = [(a, b) for a in offs[u] for b in offs[v]]
                if any(p != (0, 0) for p in pairs):
                    ext = ckks.mod_up(pr, ct.c1, ct.level)
                    cnt.modup += 1
                for (a, b) in pairs:
                    if (a, b) == (0, 0):
                        R[(g, u, v, a, b)] = ckks.lift_qp(pr, ct) if double else ct
                    else:
                        rot = ckks.rotate_ext_qp if double else ckks.rotate_ext
                        R[(g, u, v, a, b)] = rot(pr, keys, ct, ext, (a * m + b) * BS)
                        cnt.rot += 1
                        cnt.keyswitch += 1

    # 2-4. MAC per diagonal, outer rotations, rescale
    fused = hoist == "double_fused" and not any(
        d for h in range(G_out) for d in conv_diagonals(lay, Cin, Cout, h, depthwise, in_period))
    out = [None] * olay.n_ct
    for h in range(G_out):
        diags = conv_diagonals(lay, Cin, Cout, h, depthwise, in_period)
        for up in range(0, S, stride):
            for vp in range(0, S, stride):
                total = None
                for d in diags:
                    acc, terms = None, []
                    for g in range(G_in):
                        for i in range(K):
                            u, a = (up + i) % S, (up + i) // S
                            for j in range(K):
                                v, b = (vp + j) % S, (vp + j) // S
                                z = conv_weight_slots(lay, W, h, up, vp, d, g, i, j, stride=stride,
                                                      depthwise=depthwise, in_period=in_period,
                                                      wmul=wmul, Cout=Cout)
                                if not z.any():
                                    continue
                                if double:
                                    terms.append((R[(g, u, v, a, b)], ckks.encode_qp(pr, z, level, dw)))
                                else:
                                    pt = ckks.encode(pr, z, level, dw)
                                    acc = _add(pr, acc, ckks.pmult(pr, R[(g, u, v, a, b)], pt))
                                cnt.pmult += 1
                    if double and terms and fused:
                        ab, aa = ckks.mac_qp(pr, level, terms)
                        total = ckks.mod_down_rescale_ct(pr, ab, aa, level, cts[0].scale * dw)
                        cnt.moddown += 1
                        cnt.rescale += 1
                        continue
                    if double and terms:
                        ab, aa = ckks.mac_qp(pr, level, terms)
                        acc = ckks.mod_down_ct(pr, ab, aa, level, cts[0].scale * dw)
                        cnt.moddown += 1
                    if acc is None:
                        continue
                    if d:
                        acc = ckks.rotate(pr, keys, acc, d * lay.blk)
                        cnt.rot += 1
                        cnt.keyswitch += 1
                        cnt.modup += 1
                    total = _add(pr, total, acc)
                if total is None:
                    res = _empty_sum(pr, level, cts[0].scale * dw)
                elif fused:
                    res = total
                else:
                    res = ckks.rescale(pr, total)
                    cnt.rescale += 1
                out[olay.ct_index(h, up // stride, vp // stride)] = res
    return out, olay


def he_conv_bsgs(pr, keys, cts, lay, W, *, stride=1, wmul=1.0, w_scale=None, cnt=None, n1=4, hoist="single"):
    """Encrypted convolution with baby-step / giant-step outer rotations (the
    schedule the paper assumes for the channel diagonals, Sec. 3.1).

    Diagonal d = j n1 + i.  Rot(P_d, d blk) = Rot(Q, j n1 blk) with
    Q = sum over taps of Rot(R_tap, i blk) (x) Rot(pt_d, i blk), because a slot-wise
    product commutes with a rotation.  So:
      1. every input ciphertext is rotated, from one hoisted ModUp, by
         tap_step + i blk for every needed block offset and baby index i
         (one key switch each, the inner and baby rotations together);
      2. for each output and giant index j, Q_j = sum_{i, g, taps} of those
         rotations times the plaintexts of diagonal j n1 + i rotated left by
         i blk slots;
      3. out = Q_0 + sum_{j > 0} Rot(Q_j, j n1 blk), before the one rescale.
    hoist="double": the inner and baby rotations stay on Q_level * P and each Q_j
    takes one ModDown (see he_conv); "double_fused" as in he_conv."""
    cnt = cnt if cnt is not None else Counters()
    double = hoist in ("double", "double_fused")
    level = cts[0].level
    Cout, Cin, K = W.shape[0], W.shape[1], W.shape[-1]
    olay = out_layout_conv(lay, Cout, K, stride)
    S, m, BS, blk, cpc = lay.S, lay.m, lay.BS, lay.blk, lay.cpc
    n1 = min(n1, cpc)
    n2 = -(-cpc // n1)
    dw = float(pr.moduli[level]) if w_scale is None else w_scale
    G_in, G_out = lay.groups, olay.groups
    diags = {h: conv_diagonals(lay, Cin, Cout, h, False, None) for h in range(G_out)}
    babies = sorted({0} | {d % n1 for h in diags for d in diags[h]})
    offs = counts.inner_offsets(S, K, stride)

    # 1. inner + baby rotations, hoisted per input ciphertext
    R = {}
    for g in range(G_in):
        for u in range(S):
            for v in range(S):
                ct = cts[lay.ct_index(g, u, v)]
                keys_needed = [(a, b, i) for a in offs[u] for b in offs[v] for i in babies]
                ext = None
                for (a, b, i) in keys_needed:
                    if (a, b, i) == (0, 0, 0):
                        R[(g, u, v, a, b, i)] = ckks.lift_qp(pr, ct) if double else ct
                        continue
                    if ext is None:
                        ext = ckks.mod_up(pr, ct.c1, ct.level)
                        cnt.modup += 1
                    rot = ckks.rotate_ext_qp if double else ckks.rotate_ext
                    R[(g, u, v, a, b, i)] = rot(pr, keys, ct, ext, (a * m + b) * BS + i * blk)
                    cnt.rot += 1
                    cnt.keyswitch += 1

    # 2-4. MAC per giant step, giant rotations, rescale
    fused = hoist == "double_fused" and not any(d >= n1 for h in diags for d in diags[h])
    out = [None] * olay.n_ct
    for h in range(G_out):
        dset = set(diags[h])
        for up in range(0, S, stride):
            for vp in range(0, S, stride):
                total = None
                for j in range(n2):
                    acc, terms = None, []
                    for i in range(n1):
                        d = j * n1 + i
                        if d >= cpc or d not in dset:
                            continue
                        for g in range(G_in):
                            for ti in range(K):
                                u, a = (up + ti) % S, (up + ti) // S
                                for tj in range(K):
                                    v, b = (vp + tj) % S, (vp + tj) // S
                                    z = conv_weight_slots(lay, W, h, up, vp, d, g, ti, tj, stride=stride,
                                                          depthwise=False, in_period=None, wmul=wmul, Cout=Cout)
                                    if not z.any():
                                        continue
                                    z = np.roll(z, -i * blk)  # Rot(z, i blk)[l] = z[l + i blk]
                                    if double:
                                        terms.append((R[(g, u, v, a, b, i)], ckks.encode_qp(pr, z, level, dw)))
                                    else:
                                        pt = ckks.encode(pr, z, level, dw)
                                        acc = _add(pr, acc, ckks.pmult(pr, R[(g, u, v, a, b, i)], pt))
                                    cnt.pmult += 1
                    if double and terms and fused:
                        ab, aa = ckks.mac_qp(pr, level, terms)
                        total = ckks.mod_down_rescale_ct(pr, ab, aa, level, cts[0].scale * dw)
                        cnt.moddown += 1
                        cnt.rescale += 1
                        continue
                    if double and terms:
                        ab, aa = ckks.mac_qp(pr, level, terms)
                        acc = ckks.mod_down_ct(pr, ab, aa, level, cts[0].scale * dw)
                        cnt.moddown += 1
                    if acc is None:
                        continue
                    if j:
                        acc = ckks.rotate(pr, keys, acc, j * n1 * blk)
                        cnt.rot += 1
                        cnt.keyswitch += 1
                        cnt.modup += 1
                    total = _add(pr, total, acc)
                if total is None:
                    res = _empty_sum(pr, level, cts[0].scale * dw)
                elif fused:
                    res = total
                else:
                    res = ckks.rescale(pr, total)
                    cnt.rescale += 1
                out[olay.ct_index(h, up // stride, vp // stride)] = res
    return out, olay


def he_square(pr, keys, cts, cnt=None):
    """x^2 activation: CMult with relinearisation, then rescale."""
    cnt = cnt if cnt is not None else Counters()
    out = []
    for ct in cts:
        out.append(ckks.rescale(pr, ckks.cmult_relin(pr, keys, ct, ct)))
        cnt.cmult += 1
        cnt.keyswitch += 1
        cnt.modup += 1
        cnt.rescale += 1
    return out


def he_avgpool2(pr, cts, lay):
    """2x2 average pooling by summing fragment ciphertexts (S even): output fragment
    (u'', v'') = sum of input fragments (2u''+di, 2v''+dj).  The 1/4 is left to the
    next linear layer (its weights are multiplied by 1/4)."""
    if lay.S % 2:
        raise ValueError("pooling by fragment sums needs an even S")
    olay = Layout(lay.N, lay.H // 2, lay.W // 2, lay.C, lay.BS, lay.S // 2, m=lay.m)
    out = []
    for g in range(lay.groups):
        for u in range(olay.S):
            for v in range(olay.S):
                acc = None
                for di in range(2):
                    for dj in range(2):
                        acc = _add(pr, acc, cts[lay.ct_index(g, 2 * u + di, 2 * v + dj)])
                out.append(acc)
    return out, olay


def aac_compress(pr, keys, cts, lay, c_valid, cnt=None):
    """Arch-aware Ciphertext Compression: a ciphertext whose first c_valid channel
    positions are valid and the rest empty is filled by rotate-and-add doubling,
    ct <- ct + Rot(ct, -s m^2 BS) for s = c_valid, 2 c_valid, ..., cpc/2, so that
    position c_loc holds channel c_loc mod c_valid (Fig. 6).  No plaintext mask is
    needed because the empty positions hold zeros (the preceding layer's weight
    plaintexts are zero there, which merges the mask into those weights at their
    single scale).  Consumes no level."""
    cnt = cnt if cnt is not None else Counters()
    if lay.cpc % c_valid:
        raise ValueError("c_valid must divide cpc")
    out = []
    for ct in cts:
        acc = ct.copy()
        s = c_valid
        while s < lay.cpc:
            acc = ckks.add(pr, acc, ckks.rotate(pr, keys, acc, -s * lay.blk))
            cnt.rot += 1
            cnt.keyswitch += 1
            cnt.modup += 1
            s *= 2
        out.append(acc)
    return out


def aac_rotation_steps(lay, c_valid):
    steps = []
    s = c_valid
    while s < lay.cpc:
        steps.append(-s * lay.blk)
        s *= 2
    return steps


# ---------------------------------------------------------------------------
# Fully connected layers: diagonal method with baby-step / giant-step over the
# P = cpc m^2 block positions of a ciphertext (rotation by one position is a
# rotation by BS slots).
# ---------------------------------------------------------------------------

def fc_bsgs_split(P):
    k = P.bit_length() - 1
    n1 = 1 << ((k + 1) // 2)
    return n1, P // n1


def fc_rotation_steps(P, BS):
    n1, n2 = fc_bsgs_split(P)
    return sorted({b * BS for b in range(1, n1)} | {n1 * g * BS for g in range(1, n2)})


def he_fc(pr, keys, cts, feat_of, P, BS, Wfc, *, w_scale=None, cnt=None, n1=None):
    """y = Wfc x.  cts: input ciphertexts; feat_of(c, p) -> feature index or -1 for
    position p of input ciphertext c.  Output neuron n sits in ciphertext n // P at
    position n % P (for every batch slot).  n1: baby steps (default fc_bsgs_split)."""
    cnt = cnt if cnt is not None else Counters()
    level = cts[0].level
    dw = float(pr.moduli[level]) if w_scale is None else w_scale
    F_out = Wfc.shape[0]
    T = -(-F_out // P)
    if n1 is None:
        n1, n2 = fc_bsgs_split(P)
    else:
        n2 = P // n1

    def diag(t, c, delta):
        z = np.zeros(P)
        for p in range(P):
            n = t * P + p
            f = feat_of(c, (p + delta) % P)
            if n < F_out and f >= 0:
                z[p] = Wfc[n, f]
        return z

    # plaintext diagonals, rotated for the giant steps
    pts = {}
    for t in range(T):
        for c in range(len(cts)):
            for gam in range(n2):
                for beta in range(n1):
                    dz = diag(t, c, n1 * gam + beta)
                    dz = np.roll(dz, n1 * gam)  # dz'[p] = diag[(p - n1 gam) mod P]
                    if dz.any():
                        pts[(t, c, gam, beta)] = np.repeat(dz, BS)
    # baby steps, hoisted per input ciphertext
    baby = {}
    for c, ct in enumerate(cts):
        need = sorted({k[3] for k in pts if k[1] == c})
        ext = None
        for beta in need:
            if beta == 0:
                baby[(c, 0)] = ct
            else:
                if ext is None:
                    ext = ckks.mod_up(pr, ct.c1, ct.level)
                    cnt.modup += 1
                baby[(c, beta)] = ckks.rotate_ext(pr, keys, ct, ext, beta * BS)
                cnt.rot += 1
                cnt.keyswitch += 1
    out = []
    for t in range(T):
        total = None
        for gam in range(n2):
            acc = None
            for c in range(len(cts)):
                for beta in range(n1):
                    key = (t, c, gam, beta)
                    if key not in pts:
                        continue
                    pt = ckks.encode(pr, pts[key], level, dw)
                    acc = _add(pr, acc, ckks.pmult(pr, baby[(c, beta)], pt))
                    cnt.pmult += 1
            if acc is None:
                continue
            if gam:
                acc = ckks.rotate(pr, keys, acc, n1 * gam * BS)
                cnt.rot += 1
                cnt.keyswitch += 1
                cnt.modup += 1
            total = _add(pr, total, acc)
        if total is None:  # every weight of these outputs is zero: an empty sum
            out.append(_empty_sum(pr, level, cts[0].scale * dw))
            continue
        out.append(ckks.rescale(pr, total))
        cnt.rescale += 1
    return out


# ---------------------------------------------------------------------------
# Fragment-size change between layers (Sec. 5, Implementation paragraph: the
# rot-mask-add adjustment of the block size S when a later layer's optimal S
# differs)
# ---------------------------------------------------------------------------

def element_id(lay, c, h, w):
    return (c * lay.H + h) * lay.W + w


def layout_position(lay, c, h, w):
    """(ciphertext, position) of element (c, h, w) under Algorithm 1's slot map;
    the element's BS batch entries occupy slots position * BS + b."""
    g, c_loc = divmod(c, lay.cpc)
    ct = lay.ct_index(g, h % lay.S, w % lay.S)
    return ct, (c_loc * lay.m + h // lay.S) * lay.m + w // lay.S


def repack_map(la, lb):
    """Source (ct, position) under layout la and target (ct, position) under lb
    of every element (c, h, w) of the map both layouts describe."""
    assert (la.C, la.H, la.W, la.BS, la.N) == (lb.C, lb.H, lb.W, lb.BS, lb.N)
    out = []
    for c in range(la.C):
        for h in range(la.H):
            for w in range(la.W):
                out.append((layout_position(la, c, h, w), layout_position(lb, c, h, w)))
    return out


def repack_shifts(la, lb):
    """{(target ct, source ct): set of position shifts d = source - target mod P}."""
    P = la.cpc * la.m * la.m
    sh = {}
    for (cs, ps), (ct, pt) in repack_map(la, lb):
        sh.setdefault((ct, cs), set()).add((ps - pt) % P)
    return sh


def repack_bsgs_n1(la, lb):
    """Baby-step count of the repack: the power of two n1 <= P that minimises the
    rotations of the diagonal method, sum over source ciphertexts of their
    distinct nonzero baby steps (d mod n1) plus sum over target ciphertexts of
    their distinct nonzero giant steps (d div n1); ties to the smaller n1."""
    P = la.cpc * la.m * la.m
    sh = repack_shifts(la, lb)
    best = None
    n1 = 1
    while n1 <= P:
        baby, giant = {}, {}
        for (ct, cs), ds in sh.items():
            for d in ds:
                if d % n1:
                    baby.setdefault(cs, set()).add(d % n1)
                if d // n1:
                    giant.setdefault(ct, set()).add(d // n1)
        cost = sum(map(len, baby.values())) + sum(map(len, giant.values()))
        if best is None or cost < best[1]:
            best = (n1, cost)
        n1 *= 2
    return best[0]


def he_repack(pr, keys, cts, la, lb, cnt=None):
    """Re-encode ciphertexts from fragment layout la to layout lb (same map, other
    S or block grid): each target position receives its element from its
    source position, target_t = sum_{source s} sum_d Rot(ct_s, d BS) (x) M_{t,s,d},
    M_{t,s,d} the 0/1 mask of the target positions whose element sits d positions
    further in source s -- the diagonal method of a permutation matrix, with
    baby-step / giant-step rotations (repack_bsgs_n1) and the masks at scale
    q_level, so one rescale follows and the scale is kept.  Written as the FC
    layer whose weight matrix is that permutation."""
    P = la.cpc * la.m * la.m
    n_out = lb.n_ct
    F_in = la.C * la.H * la.W
    W = np.zeros((n_out * P, F_in))
    feat = {}
    for (c, h, w), ((cs, ps), (ct, pt)) in zip(
            ((c, h, w) for c in range(la.C) for h in range(la.H) for w in range(la.W)), repack_map(la, lb)):
        f = element_id(la, c, h, w)
        feat[(cs, ps)] = f
        W[ct * P + pt, f] = 1.0
    return he_fc(pr, keys, cts, lambda c, p: feat.get((c, p), -1), P, la.BS, W, cnt=cnt,
                 n1=repack_bsgs_n1(la, lb))


def repack_rotation_steps(la, lb):
    """Rotation steps (slots) the repack needs keys for."""
    P = la.cpc * la.m * la.m
    n1 = repack_bsgs_n1(la, lb)
    steps = set()
    for (ct, cs), ds in repack_shifts(la, lb).items():
        for d in ds:
            if d % n1:
                steps.add((d % n1) * la.BS)
            if d // n1:
                steps.add((d // n1) * n1 * la.BS)
    return sorted(steps)


# ---------------------------------------------------------------------------
# Transformer extension (Sec. 7): a linear layer on fragmented token embeddings
# ---------------------------------------------------------------------------

def he_token_linear(pr, keys, cts, tl, W, *, w_scale=None, cnt=None):
    """Y = X W^T for the tokens of layout tl (W: E_out x E), output in the
    fragmented layout of E_out with the same S and token count: output element
    k = f' S + s' of every token sits in ciphertext s' at position f'.  It is
    the FC layer of Sec. 5 (diagonals with baby-step / giant-step) on the
    fragment feature table, with its output neuron s' P + f' taking row k of W."""
    E_out = W.shape[0]
    tlo = TokenLayout(tl.N, tl.n_tok, E_out, tl.S)
    P = tl.P
    Wfc = np.zeros((tl.S * P, tl.E))
    for k in range(E_out):
        f, s = divmod(k, tl.S)
        Wfc[s * P + f] = W[k]
    out = he_fc(pr, keys, cts, tl.feature, P, tl.n_tok, Wfc, w_scale=w_scale, cnt=cnt)
    return out, tlo


def drop_level(ct):
    """The same ciphertext modulo Q_{l-1}: its first l limbs (exact; scale kept)."""
    return ckks.Ciphertext(ct.c0[:ct.level].copy(), ct.c1[:ct.level].copy(), ct.level - 1, ct.scale)


def mask_scale_pow2(pr, level):
    """Scale of the 0/1 token masks: the power of two 2^floor(log2 q_level).  The
    masks are periodic in the slots, so their coefficients are rationals with
    denominators dividing N; at an odd scale (a prime) some land exactly on a
    rounding tie, at 2^k >= N none does."""
    return 2.0 ** (int(pr.moduli[level]).bit_length() - 1)


def token_masks(tl, r):
    """0/1 slot vectors of the tokens t < n - r and t >= n - r, in every position
    block of n_tok slots (the two halves of a token-wise rotation by r)."""
    n = tl.n_tok
    lo = np.tile((np.arange(n) < n - r).astype(float), tl.P)
    return lo, 1.0 - lo


def token_rotate(pr, keys, ct, tl, r, mask_scale):
    """Rotation of every position block of n_tok token slots by r tokens, t <- t + r
    mod n: M_lo (x) Rot(ct, r) + M_hi (x) Rot(ct, r - n) with the masks at
    mask_scale (a power of two), then one rescale: scale (s mask_scale) / q_l.
    r = 0: the ciphertext times the integer mask_scale, rescaled, which gives
    the same level and scale as the rotated ones."""
    if r == 0:
        x = ckks.mul_int(pr, ct, int(mask_scale))
        x.scale = ct.scale * mask_scale
        return ckks.rescale(pr, x)
    lo, hi = token_masks(tl, r)
    a = ckks.pmult(pr, ckks.rotate(pr, keys, ct, r), ckks.encode(pr, lo, ct.level, mask_scale))
    b = ckks.pmult(pr, ckks.rotate(pr, keys, ct, r - tl.n_tok), ckks.encode(pr, hi, ct.level, mask_scale))
    return ckks.rescale(pr, ckks.add(pr, a, b))  # scale (s mask_scale) / q_l


def position_sum(pr, keys, ct, tl):
    """Sum over the P positions of a ciphertext, replicated into every position:
    ct += Rot(ct, 2^k n_tok) for k = 0 .. log2(P) - 1."""
    acc = ct
    step = tl.n_tok
    while step < tl.N // 2:
        acc = ckks.add(pr, acc, ckks.rotate(pr, keys, acc, step))
        step *= 2
    return acc


def attention_rotation_steps(tl):
    """Rotation steps (slots) of the attention products."""
    n = tl.n_tok
    steps = set()
    for r in range(1, n):
        steps |= {r, r - n}
    step = n
    while step < tl.N // 2:
        steps.add(step)
        step *= 2
    return sorted(steps)


def he_attention_scores(pr, keys, q_cts, k_cts, tl, mask_scale=None):
    """A = Q K^T of the tokens of the fragmented layout tl (Sec. 7: token-wise
    aggregation for the attention products), as its n diagonals:
    D_r[i] = A[i][(i + r) mod n] = sum_e Q[i][e] K[(i + r) mod n][e], r < n.
    For each r: K's fragment ciphertexts rotated token-wise by r (token_rotate,
    one level), each multiplied by Q's matching fragment (one level dropped to
    meet them), the S products summed before relinearisation (one
    relinearisation per diagonal), rescaled, and summed over the positions
    (position_sum), so D_r holds A[i][(i + r) mod n] at slot f n + i of every
    position f.  Two levels; the output scale is s_q s_k' / q_{l-1}, s_k' the
    rotated K's scale."""
    level = q_cts[0].level
    ms = mask_scale_pow2(pr, level) if mask_scale is None else mask_scale
    qd = [drop_level(q) for q in q_cts]
    out = []
    for r in range(tl.n_tok):
        acc = None
        for q, k in zip(qd, k_cts):
            t = ckks.tensor(pr, q, token_rotate(pr, keys, k, tl, r, ms))
            acc = t if acc is None else ckks.tensor_add(pr, acc, t)
        d = ckks.rescale(pr, ckks.relinearize(pr, keys, acc))
        out.append(position_sum(pr, keys, d, tl))
    return out


def he_attention_apply(pr, keys, d_cts, v_cts, tl, mask_scale=None):
    """O = A V from the n diagonals of A (as he_attention_scores leaves them,
    replicated over positions) and V in the fragmented layout tl:
    O[i][e] = sum_r D_r[i] V[(i + r) mod n][e].  For each fragment ciphertext of V
    and each r: V rotated token-wise by r (one level), multiplied by D_r after
    the higher of the two has limbs dropped to meet the other; the n products
    are summed before one relinearisation, then rescaled once.  Output in V's
    layout, one level below the lower of V's rotated copies and D's."""
    level = v_cts[0].level
    ms = mask_scale_pow2(pr, level) if mask_scale is None else mask_scale
    out = []
    for v in v_cts:
        acc = None
        for r, d in enumerate(d_cts):
            vr = token_rotate(pr, keys, v, tl, r, ms)
            dr = d
            while dr.level > vr.level:
                dr = drop_level(dr)
            while vr.level > dr.level:
                vr = drop_level(vr)
            t = ckks.tensor(pr, dr, vr)
            acc = t if acc is None else ckks.tensor_add(pr, acc, t)
        out.append(ckks.rescale(pr, ckks.relinearize(pr, keys, acc)))
    return out


# ---------------------------------------------------------------------------
# Polynomial activation a x^2 + b x + c (Sec. 5, Implementation paragraph)
# ---------------------------------------------------------------------------

def poly_act_constants(s, a, b, c):
    """The integer constants of he_poly_act for input scale s and a != 0:
    (K1, sign, K2) with beta = b / (2a), gamma = c / a - beta^2,
    K1 = nearest(beta s), sign = sign(a), K2 = sign nearest(gamma (s s)).
    Every quotient and product is one IEEE double operation in the order
    written; nearest() rounds to the nearest integer, ties away from zero."""
    if a == 0:
        raise ValueError("a == 0 has no square term")
    beta = b / (2.0 * a)
    gamma = c / a - beta * beta
    sign = 1 if a > 0 else -1
    return ckks.nearest_int(beta * s), sign, sign * ckks.nearest_int(gamma * (s * s))


def he_poly_act(pr, keys, cts, a, b, c, cnt=None):
    """The activation a x^2 + b x + c that replaces ReLU (Sec. 5, Implementation),
    in one level, as the library computes it.

    a != 0 (completing the square): a x^2 + b x + c = a [(x + beta)^2 + gamma],
      1. u = ct + K1, K1 = nearest(beta s)          (scale s)
      2. w = relin(u (x) u)                          (scale s^2)
      3. v = sign(a) w + K2, K2 = sign(a) nearest(gamma s^2)
      4. rescale by q_l: the output decrypts to sign(a) [(x+beta)^2 + gamma]
         at scale s^2 / q_l, i.e. to a x^2 + b x + c at scale s^2 / (q_l |a|).
    a == 0 (affine): v = ct B + K with B = nearest(b q_l), K = nearest(c s q_l)
      (scale s q_l), rescaled by q_l to scale s.
    With a = 1, b = c = 0 every step is the identity but the square and the
    rescale, so the residues are those of he_square."""
    cnt = cnt if cnt is not None else Counters()
    out = []
    for ct in cts:
        lv, s = ct.level, ct.scale
        ql = float(pr.moduli[lv])
        if a != 0:
            K1, sign, K2 = poly_act_constants(s, a, b, c)
            u = ckks.add_int(pr, ct, K1)
            w = ckks.cmult_relin(pr, keys, u, u)
            cnt.cmult += 1
            cnt.keyswitch += 1
            v = ckks.add_int(pr, ckks.mul_int(pr, w, sign), K2)
            r = ckks.rescale(pr, v)
            r.scale = (s * s) / (ql * abs(a))
        else:
            B = ckks.nearest_int(b * ql)
            K = ckks.nearest_int(c * (s * ql))
            r = ckks.rescale(pr, ckks.add_int(pr, ckks.mul_int(pr, ct, B), K))
            r.scale = s
        cnt.rescale += 1
        out.append(r)
    return out


def aac_mask_slots(lay, c_valid):
    """0/1 slot vector of the valid channel blocks: 1 where c_loc < c_valid."""
    mask = np.zeros(lay.N // 2)
    per = lay.m * lay.m * lay.BS
    mask[:c_valid * per] = 1.0
    return mask


def aac_compress_masked(pr, keys, cts, lay, c_valid, mask_scale, cnt=None):
    """AAC with its plaintext mask (Sec. 4.3, last paragraph): the 0/1 mask of the
    valid channel blocks, encoded at scale Delta_2 = mask_scale, zeroes whatever
    the empty blocks hold (e.g. the constant of an activation with c != 0); the
    rotate-and-add replication follows on the masked ciphertexts.  No rescale
    here: the output scale is s Delta_2, and the next layer's weights are
    encoded at Delta_1 = q_l t / (s Delta_2), so that one rescale follows both
    multiplications (Delta_1 Delta_2 = q_l t / s)."""
    cnt = cnt if cnt is not None else Counters()
    mask = ckks.encode(pr, aac_mask_slots(lay, c_valid), cts[0].level, mask_scale)
    masked = []
    for ct in cts:
        masked.append(ckks.pmult(pr, ct, mask))
        cnt.pmult += 1
    return aac_compress(pr, keys, masked, lay, c_valid, cnt)


# ---------------------------------------------------------------------------
# Scale rule for a chain of layers and the LeNet-shaped network
# ---------------------------------------------------------------------------

def weight_scale(pr, level, s_in, delta, act_a):
    """Scale at which a linear layer at `level` encodes its weights: the output
    scale after its rescale is delta, or sqrt(delta q_{level-1} |a|) when an
    activation with leading coefficient a follows (x^2: a = 1; a bool True
    counts as 1), so that the activation's rescale (scale s^2 / (q_{level-1} |a|),
    he_poly_act) lands back on delta.  act_a = 0 / False: no activation follows.
    Evaluated as written, in IEEE double arithmetic."""
    t = math.sqrt(delta * float(pr.moduli[level - 1]) * abs(act_a)) if act_a else delta
    return (t / s_in) * float(pr.moduli[level])


def lenet_layouts(N, BS, S=4):
    l0 = Layout(N, 28, 28, 1, BS, S)
    return l0


def lenet_rotation_steps(N, BS, S=4):
    """Every rotation step the LeNet-shaped network uses (for key generation)."""
    l0 = lenet_layouts(N, BS, S)
    steps = set(conv_rotation_steps(l0, 1, 6, 5))
    l1 = out_layout_conv(l0, 6, 5, 1)
    l1p = Layout(N, l1.H // 2, l1.W // 2, 6, BS, l1.S // 2, m=l1.m)
    steps |= set(conv_rotation_steps(l1p, 6, 16, 5))
    P = l1p.cpc * l1p.m * l1p.m
    steps |= set(fc_rotation_steps(P, BS))
    return sorted(steps)


def he_lenet(pr, keys, cts, lay, weights, delta, cnt=None, act=None):
    """conv5x5 1->6, act, avgpool2, conv5x5 6->16, act, avgpool2, FC 256->120->84->10,
    act = x^2 (he_square) or, given act = (a, b, c), a x^2 + b x + c (he_poly_act).
    Returns the output ciphertexts (neuron n at position n of the FC layout)."""
    cnt = cnt if cnt is not None else Counters()
    a = 1.0 if act is None else act[0]

    def activation(h):
        return he_square(pr, keys, h, cnt) if act is None else he_poly_act(pr, keys, h, *act, cnt=cnt)

    lv = cts[0].level
    h, l1 = he_conv(pr, keys, cts, lay, weights["conv1"],
                    w_scale=weight_scale(pr, lv, cts[0].scale, delta, a), cnt=cnt)
    h = activation(h)
    h, l1 = he_avgpool2(pr, h, l1)
    lv = h[0].level
    h, l2 = he_conv(pr, keys, h, l1, weights["conv2"], wmul=0.25,
                    w_scale=weight_scale(pr, lv, h[0].scale, delta, a), cnt=cnt)
    h = activation(h)
    h, l2 = he_avgpool2(pr, h, l2)
    assert l2.S == 1
    P = l2.cpc * l2.m * l2.m
    m = l2.m

    def feat_conv(c_ct, p):
        c_loc, k = divmod(p, m * m)
        c = c_ct * l2.cpc + c_loc
        bi, bj = divmod(k, m)
        if c >= l2.C or bi >= l2.H or bj >= l2.W:
            return -1
        return (c * l2.H + bi) * l2.W + bj

    BS = l2.BS
    Wf1 = weights["fc1"] * 0.25
    lv = h[0].level
    h = he_fc(pr, keys, h, feat_conv, P, BS, Wf1,
              w_scale=weight_scale(pr, lv, h[0].scale, delta, False), cnt=cnt)
    for name in ("fc2", "fc3"):
        F_in = weights[name].shape[1]

        def feat_fc(c_ct, p, F_in=F_in):
            f = c_ct * P + p
            return f if f < F_in else -1

        lv = h[0].level
        h = he_fc(pr, keys, h, feat_fc, P, BS, weights[name],
                  w_scale=weight_scale(pr, lv, h[0].scale, delta, False), cnt=cnt)
    return h, P


def lenet_decode_logits(slots_list, P, BS, n_out=10):
    """Read the FC output layout back: logits[b, n] = slot (n mod P) * BS + b of ct n // P."""
    y = np.zeros((BS, n_out))
    for n in range(n_out):
        t, p = divmod(n, P)
        y[:, n] = slots_list[t][p * BS:(p + 1) * BS]
    return y
