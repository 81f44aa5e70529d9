// Rotation-complexity model of the fragment encoding (Eq. 3 - Eq. 8) and the
// analytic fragment-size choice (Theorem).  Host code only: no device, no
// context, so a planner (or the learned proposer, as its fallback and judge)
// can call it anywhere.
//
//   alpha = N / (2 M^2), M = S m with m = 2^ceil(log2 ceil(max(H, W) / S))
//   Eq. 3 (inner, per layer) = (ceil(K/S)^2 - 1) N_in / alpha      for K > S, else 0
//   Eq. 4 (outer, per layer) = (BS / alpha) (alpha S^2 / BS - 1) N_out
//   Eq. 5 (total)            = (BS / alpha) [inner(S) N_in + (alpha S^2 / BS - 1) N_out]
//   Eq. 7 (admissible S)     = S <= sqrt(BS N_in / alpha)  (S = 1 always admissible)
//   Eq. 8 (closed form)      = S*^4 = K^2 N_in BS / (alpha N_out)
// The choice is the argmin of Eq. 5 over the admissible power-of-two S whose
// channel block fits one ciphertext (m^2 BS <= N/2); ties go to the smaller S.
// Depthwise layers have no outer rotations (one diagonal), so only the inner
// term counts.
#include <algorithm>
#include <cmath>
#include <set>

#include "common.h"

namespace {

uint32_t pow2_at_least(uint32_t x) {
    uint32_t m = 1;
    while (m < x) m *= 2;
    return m;
}

struct Geometry {
    uint32_t m, M;
    double alpha;
    bool fits;
};

Geometry geometry(uint32_t N, uint32_t H, uint32_t W, uint32_t BS, uint32_t S) {
    Geometry g;
    const uint32_t side = (std::max(H, W) + S - 1) / S;
    g.m = pow2_at_least(side);
    g.M = S * g.m;
    g.alpha = (double)N / (2.0 * g.M * (double)g.M);
    g.fits = (uint64_t)g.m * g.m * BS <= N / 2;
    return g;
}

double inner_term(uint32_t K, uint32_t S) {
    if (K <= S) return 0.0;
    const double a = std::ceil((double)K / S);
    return a * a - 1.0;
}

// executed inner rotations per input channel group: for each source fragment
// (u, v), the block offsets (a, b) != (0, 0) that some kept output and tap read
uint64_t executed_inner_per_group(uint32_t S, uint32_t K, uint32_t stride) {
    std::vector<std::set<int>> offs(S);
    for (uint32_t u = 0; u < S; u++)
        for (uint32_t up = 0; up < S; up += stride)
            for (uint32_t i = 0; i < K; i++)
                if ((up + i) % S == u) offs[u].insert((int)((up + i) / S));
    uint64_t n = 0;
    for (uint32_t u = 0; u < S; u++)
        for (uint32_t v = 0; v < S; v++)
            for (int a : offs[u])
                for (int b : offs[v]) n += (a != 0 || b != 0);
    return n;
}

}  // namespace

extern "C" int fe_rotation_model(uint32_t N, uint32_t H, uint32_t W, uint32_t Cin, uint32_t Cout, uint32_t K,
                                 uint32_t S, uint32_t BS, uint32_t stride, int depthwise, fe_rotation_model_t* out) {
    if (!out) return fe::fail(FE_EINVAL, "null argument");
    if (!N || (N & (N - 1)) || !H || !W || !Cin || !Cout || !K || !S || !BS || (stride != 1 && stride != 2))
        return fe::fail(FE_EINVAL, "fe_rotation_model: zero extent, N not a power of two, or stride not 1 or 2");
    const Geometry g = geometry(N, H, W, BS, S);
    if (!g.fits) return fe::fail(FE_EINVAL, "fe_rotation_model: one channel block does not fit a ciphertext");
    const double in = inner_term(K, S), a = g.alpha;
    out->m = g.m;
    out->M = g.M;
    out->cpc = (uint32_t)((N / 2) / ((uint64_t)g.m * g.m * BS));
    out->alpha = a;
    out->eq3_inner = (S == g.M) ? 0.0 : in * Cin / a;
    out->eq4_outer = depthwise ? 0.0 : (BS / a) * (a * S * S / BS - 1.0) * Cout;
    out->eq5_total = (BS / a) * (in * Cin + (depthwise ? 0.0 : (a * S * S / BS - 1.0) * Cout));
    out->s_bound_eq7 = std::sqrt(BS * (double)Cin / a);
    out->s_star_eq8 = depthwise ? 0.0 : std::pow((double)K * K * Cin * BS / (a * Cout), 0.25);
    const uint32_t groups = (Cin + out->cpc - 1) / out->cpc;
    out->executed_inner = executed_inner_per_group(S, K, stride) * groups;
    return FE_OK;
}

extern "C" int fe_choose_fragment(uint32_t N, uint32_t H, uint32_t W, uint32_t Cin, uint32_t Cout, uint32_t K,
                                  uint32_t BS, int depthwise, uint32_t max_S, fe_fragment_choice* out) {
    if (!out) return fe::fail(FE_EINVAL, "null argument");
    if (!N || (N & (N - 1)) || !H || !W || !Cin || !Cout || !K || !BS)
        return fe::fail(FE_EINVAL, "fe_choose_fragment: zero extent or N not a power of two");
    if (max_S == 0) max_S = 32;
    bool found = false;
    uint32_t n_adm = 0;
    for (uint32_t S = 1; S <= max_S; S *= 2) {
        const Geometry g = geometry(N, H, W, BS, S);
        if (!g.fits) continue;
        if (S > 1 && S > std::sqrt(BS * (double)Cin / g.alpha)) continue;
        n_adm++;
        fe_rotation_model_t r;
        if (fe_rotation_model(N, H, W, Cin, Cout, K, S, BS, 1, depthwise, &r) != FE_OK) continue;
        if (!found || r.eq5_total < out->eq5) {
            found = true;
            out->S = S;
            out->m = r.m;
            out->M = r.M;
            out->cpc = r.cpc;
            out->alpha = r.alpha;
            out->eq5 = r.eq5_total;
            out->s_star = r.s_star_eq8;
        }
    }
    out->n_admissible = n_adm;
    if (!found) return fe::fail(FE_EINVAL, "fe_choose_fragment: no admissible fragment size (the map does not fit)");
    return FE_OK;
}

// Transformer extension (Sec. 7): the rotation complexity gamma E / S + 2 n S
// (embedding-wise aggregation over E / S positions in the FFN and projections,
// token-wise aggregation over S times more tokens per ciphertext in the
// attention products), taken as a count, and its argmin over the power-of-two
// S <= max_S that divide E (ties to the smaller S).
extern "C" int fe_choose_token_fragment(uint32_t E, uint32_t n_tok, double gamma, uint32_t max_S, uint32_t* S_out,
                                        double* rotations, double* s_star) {
    if (!S_out || !E || !n_tok || !(gamma > 0)) return fe::fail(FE_EINVAL, "fe_choose_token_fragment: bad argument");
    if (max_S == 0) max_S = 64;
    bool found = false;
    double best = 0;
    for (uint32_t S = 1; S <= max_S; S *= 2) {
        if (E % S) continue;
        const double r = gamma * E / S + 2.0 * n_tok * S;
        if (!found || r < best) {
            found = true;
            best = r;
            *S_out = S;
        }
    }
    if (!found) return fe::fail(FE_EINVAL, "fe_choose_token_fragment: no candidate S divides E");
    if (rotations) *rotations = best;
    if (s_star) *s_star = std::sqrt(gamma * E / (2.0 * n_tok));
    return FE_OK;
}
