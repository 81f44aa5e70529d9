"""Conv-aware fragment encoding (Algorithm 1) and its slot map.

Test infrastructure only (see oracle/__init__.py).

Algorithm 1: zero-pad X (BS x C x H x W) to M x M, cut each map into an m x m
grid of S x S blocks (m = M / S), and for every intra-block position (u, v)
gather element (u, v) of every block into one ciphertext, slot
    l = (c_loc * m^2 + k) * BS + b,   k = bi * m + bj  (block row-major),
with batch innermost and channel outermost.

Readings (the paper leaves these open or prints them garbled):
* pad(): M = S * 2^ceil(log2(ceil(max(H, W) / S))), so m is a power of two and
  cpc * m^2 * BS = N/2 exactly (cpc = channels per ciphertext); rotating by a
  multiple of m^2 * BS then permutes whole channel blocks cyclically.
* The slot map of Algorithm 1 is printed with ceilings on 0-based indices; the
  floor form above is used (i = l // (BS m^2), j = l mod BS, k = (l // BS) mod m^2).
* Channels beyond cpc go to further ciphertexts: channel c sits in group
  g = c // cpc at position c_loc = c mod cpc.  Ciphertexts are listed in the
  order (g, u, v).
"""
import numpy as np


class Layout:
    """Fragment layout of a BS x C x H x W activation for ring degree N.

    m may be given explicitly: a layer's output keeps its input's block grid
    (only S and the valid region H x W change)."""

    def __init__(self, N, H, W, C, BS, S, m=None):
        if S < 1:
            raise ValueError("S must be >= 1")
        if m is None:
            side = -(-max(H, W) // S)
            m = 1
            while m < side:
                m *= 2
        elif S * m < max(H, W):
            raise ValueError("block grid too small for the map")
        slots = N // 2
        if m * m * BS > slots or slots % (m * m * BS):
            raise ValueError("one channel block does not fit the ciphertext")
        self.N, self.H, self.W, self.C, self.BS, self.S = N, H, W, C, BS, S
        self.m = m
        self.M = S * m
        self.cpc = slots // (m * m * BS)
        self.groups = -(-C // self.cpc)
        self.blk = m * m * BS  # slots per channel block

    @property
    def n_ct(self):
        return self.groups * self.S * self.S

    def ct_index(self, g, u, v):
        return (g * self.S + u) * self.S + v

    def slot(self, c_loc, bi, bj, b):
        return (c_loc * self.m * self.m + bi * self.m + bj) * self.BS + b

    def utilisation(self):
        """Fraction of slots holding valid activations."""
        used = self.C * self.H * self.W * self.BS
        return used / (self.n_ct * (self.N // 2))

    def describe(self):
        return dict(S=self.S, M=self.M, m=self.m, BS=self.BS, cpc=self.cpc, n_ct=self.n_ct)


def pack(lay, x):
    """Algorithm 1, steps 1-3: x (BS, C, H, W) -> slot vectors (n_ct, N/2), zero padded."""
    BS, Cc, H, W = x.shape
    assert (BS, Cc, H, W) == (lay.BS, lay.C, lay.H, lay.W)
    out = np.zeros((lay.n_ct, lay.N // 2), dtype=np.float64)
    for g in range(lay.groups):
        for u in range(lay.S):
            for v in range(lay.S):
                vec = out[lay.ct_index(g, u, v)]
                for c_loc in range(lay.cpc):
                    c = g * lay.cpc + c_loc
                    if c >= Cc:
                        break
                    for bi in range(lay.m):
                        h = bi * lay.S + u
                        if h >= H:
                            break
                        for bj in range(lay.m):
                            w = bj * lay.S + v
                            if w >= W:
                                break
                            for b in range(BS):
                                vec[lay.slot(c_loc, bi, bj, b)] = x[b, c, h, w]
    return out


def unpack(lay, slots):
    """Inverse of pack on the valid region: (n_ct, N/2) -> (BS, C, H, W)."""
    y = np.zeros((lay.BS, lay.C, lay.H, lay.W), dtype=np.float64)
    for g in range(lay.groups):
        for u in range(lay.S):
            for v in range(lay.S):
                vec = slots[lay.ct_index(g, u, v)]
                for c_loc in range(lay.cpc):
                    c = g * lay.cpc + c_loc
                    if c >= lay.C:
                        break
                    for bi in range(lay.m):
                        h = bi * lay.S + u
                        if h >= lay.H:
                            break
                        for bj in range(lay.m):
                            w = bj * lay.S + v
                            if w >= lay.W:
                                break
                            for b in range(lay.BS):
                                y[b, c, h, w] = vec[lay.slot(c_loc, bi, bj, b)]
    return y


def slot_map(lay):
    """Index-slot mapping returned to the client: for every (b, c, h, w) the pair
    (ciphertext index, slot)."""
    ct = np.empty((lay.BS, lay.C, lay.H, lay.W), dtype=np.int64)
    sl = np.empty_like(ct)
    for b in range(lay.BS):
        for c in range(lay.C):
            g, c_loc = divmod(c, lay.cpc)
            for h in range(lay.H):
                bi, u = divmod(h, lay.S)
                for w in range(lay.W):
                    bj, v = divmod(w, lay.S)
                    ct[b, c, h, w] = lay.ct_index(g, u, v)
                    sl[b, c, h, w] = lay.slot(c_loc, bi, bj, b)
    return ct, sl


class TokenLayout:
    """Fragmented token-embedding layout (Sec. 7): n_tok tokens with embedding
    dimension E; element e = f S + s of token t sits in ciphertext s at
    position f, slot f n_tok + t (tokens innermost, like the batch of
    Algorithm 1).  Each ciphertext holds E / S elements of every token, so an
    embedding-wise sum needs rotations over E / S positions, and P = N / (2
    n_tok) positions must hold them."""

    def __init__(self, N, n_tok, E, S):
        if (N // 2) % n_tok:
            raise ValueError("n_tok must divide N / 2")
        self.N, self.n_tok, self.E, self.S = N, n_tok, E, S
        self.P = N // 2 // n_tok
        self.F = -(-E // S)  # positions used
        if self.F > self.P:
            raise ValueError("E / S positions do not fit a ciphertext")
        self.n_ct = S

    def feature(self, c, p):
        """Embedding index held at position p of ciphertext c, or -1."""
        e = p * self.S + c
        return e if p < self.F and e < self.E else -1


def pack_tokens(tl, x):
    """x: (n_tok, E) -> (S, N/2) slot vectors."""
    out = np.zeros((tl.n_ct, tl.N // 2))
    for e in range(tl.E):
        f, s = divmod(e, tl.S)
        out[s, f * tl.n_tok:(f + 1) * tl.n_tok] = x[:, e]
    return out


def unpack_tokens(tl, slots):
    x = np.zeros((tl.n_tok, tl.E))
    for e in range(tl.E):
        f, s = divmod(e, tl.S)
        x[:, e] = slots[s, f * tl.n_tok:(f + 1) * tl.n_tok]
    return x
