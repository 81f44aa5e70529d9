"""Rotation-complexity model of the fragment encoding (Eq. 3 - Eq. 8) and the
analytic block-size choice (Theorem, Eq. 8).

Test infrastructure only (see oracle/__init__.py).

Readings, each fixed so that the printed numbers of Table 6 come out:
* alpha = N / (2 M^2) with the padded side M (equals N / (2 H W) when M = H).
* Eq. 3 / Eq. 5 inner term for K > S is (ceil(K/S)^2 - 1) per input ciphertext
  (the printed parentheses are garbled); for K <= S the "formula" count is 0 as
  in Table 6, while the edge rotations that an implementation executes are
  counted separately (executed_inner).
* Eq. 4 carries the BS factor of Eq. 5: (BS/alpha) (alpha S^2 / BS - 1) N_out.
* Theorem / Eq. 8: S*^4 = K^2 N_in BS / (alpha N_out) (the BS factor is needed
  to reproduce the worked value 3.57); the decision is the argmin of Eq. 5 over
  the admissible S of Eq. 7, ties to the smaller S.
"""
import math


def alpha(N, M):
    return N / (2 * M * M)


def inner_eq3(N_in, K, S, alpha_, M=None):
    """Eq. 3 per layer (ciphertexts N_in / alpha), Table 6 convention for K <= S."""
    if M is not None and S == M:
        return 0.0
    if K > S:
        return (math.ceil(K / S) ** 2 - 1) * N_in / alpha_
    return 0.0


def inner_eq3_case2(N_in, S, alpha_):
    """Eq. 3 as printed for K <= S < M: 4(S-1)/S^2 * N_in / alpha."""
    return 4 * (S - 1) / (S * S) * N_in / alpha_


def outer_eq4(N_out, S, BS, alpha_):
    """Eq. 4 with the BS factor of Eq. 5."""
    return (BS / alpha_) * (alpha_ * S * S / BS - 1) * N_out


def total_eq5(N_in, N_out, K, S, BS, alpha_):
    """Eq. 5: (BS/alpha) [inner(S) N_in + (alpha S^2 / BS - 1) N_out]."""
    inner = (math.ceil(K / S) ** 2 - 1) if K > S else 0
    return (BS / alpha_) * (inner * N_in + (alpha_ * S * S / BS - 1) * N_out)


def amortized_eq6(N_in, K, S, alpha_):
    """Eq. 6 (large batch, no outer rotations): rotations per sample."""
    if S < K:
        return (math.ceil(K / S) ** 2 - 1) * N_in / alpha_
    return 4 * (S - 1) / (S * S) * N_in / alpha_


def s_bound_eq7(BS, N_in, alpha_):
    """Eq. 7: S <= sqrt(BS N_in / alpha)."""
    return math.sqrt(BS * N_in / alpha_)


def s_star_eq8(K, N_in, N_out, BS, alpha_):
    """Theorem (Eq. 8) with the BS factor: (K^2 N_in BS / (alpha N_out))^(1/4), unrounded."""
    return (K * K * N_in * BS / (alpha_ * N_out)) ** 0.25


def choose_S(N, H, K, N_in, N_out, BS, candidates=(1, 2, 4, 8, 16, 32)):
    """Analytic fragment-size choice: argmin of Eq. 5 over admissible S (Eq. 7),
    alpha recomputed from each S's padded side; ties go to the smaller S."""
    best = None
    for S in candidates:
        side = -(-H // S)
        m = 1
        while m < side:
            m *= 2
        M = S * m
        if m * m * BS > N // 2:
            continue
        a = alpha(N, M)
        if S > 1 and S > s_bound_eq7(BS, N_in, a):
            continue
        cost = total_eq5(N_in, N_out, K, S, BS, a)
        if best is None or cost < best[1]:
            best = (S, cost)
    return best


def inner_offsets(S, K, stride=1):
    """Executed inner rotations of the fragment conv: for each source fragment
    row u, the block offsets a with u + a S = u' + i for a kept output row u'
    (u' % stride == 0) and a tap 0 <= i < K.  Returns {u: sorted offsets}."""
    res = {}
    for u in range(S):
        offs = set()
        for up in range(0, S, stride):
            for i in range(K):
                if (up + i) % S == u:
                    offs.add((up + i) // S)
        res[u] = sorted(offs)
    return res


def executed_inner(S, K, n_groups, stride=1):
    """Inner rotations executed per layer: sum over input fragments of
    (#row offsets x #column offsets - 1)."""
    offs = inner_offsets(S, K, stride)
    total = 0
    for u in range(S):
        for v in range(S):
            total += sum(1 for a in offs[u] for b in offs[v] if (a, b) != (0, 0))
    return total * n_groups


# ---------------------------------------------------------------------------
# Transformer extension (Sec. 7): token embeddings split into fragments of size
# S; embedding-wise rotations fall as E / S, token-wise ones grow as S.
# ---------------------------------------------------------------------------

def transformer_rotations(E, n, gamma, S):
    """The rotation complexity of Sec. 7 taken as a count: gamma E / S for the
    FFN and projections (embedding aggregation over E / S positions) plus 2 n S
    for the token-wise aggregation of the attention products."""
    return gamma * E / S + 2 * n * S


def choose_S_transformer(E, n, gamma, candidates=(1, 2, 4, 8, 16, 32, 64)):
    """Argmin of transformer_rotations over the candidate S that divide E
    (ties to the smaller S)."""
    best = None
    for S in candidates:
        if E % S:
            continue
        cost = transformer_rotations(E, n, gamma, S)
        if best is None or cost < best[1]:
            best = (S, cost)
    return best


def s_star_transformer(E, n, gamma):
    """Continuous optimum of gamma E / S + 2 n S: S* = sqrt(gamma E / (2 n))."""
    return math.sqrt(gamma * E / (2 * n))
