// Layer plans shared by the planner (henn.cu) and the graph / layer helpers.
#pragma once

#include <vector>

#include "ops.h"

struct fe_plan {
    fe_ctx* c;
    int kind;  // 0 conv, 1 fc
    int level;
    int n_in, n_out;
    fe_layout lin, lout;
    int Cin, Cout, K, stride, depthwise, in_period;
    int P, BS, F_in, F_out, n1, n2;
    std::vector<int> feat;
    struct Inner {
        int ci;
        int32_t step;
    };
    std::vector<Inner> inner;     // rotated inputs ("R slots")
    std::vector<int> modup_cts;   // input ciphertexts that are rotated (sorted)
    std::vector<int> modup_slot;  // [n_in] -> position in modup_cts or -1
    struct Term {
        int src;  // >= 0: R slot, < 0: input -(src + 1)
        int pt;
    };
    struct Group {
        int32_t step;  // 0: no rotation
        int t0, nt;
    };
    struct Out {
        std::vector<Group> groups;
    };
    std::vector<Term> terms;
    std::vector<Out> outs;
    struct ConvPt {
        int h, up, vp, d, g, i, j;
        int rot;  // left rotation of the slot vector (baby step i: i m^2 BS)
    };
    std::vector<ConvPt> cpts;
    struct FcPt {
        int t, c, gam, beta;
    };
    std::vector<FcPt> fpts;
    int n_pt = 0;
    int n_outer = 0;
    int bsgs_n1 = 0;  // baby steps of the outer rotations, 0: linear
    int mac_ways = 4;  // outputs sharing one MAC item (ciphertext loads), 1, 2 or 4
    int dhoist = 0;    // 1: double hoisting (rotations and MAC on Q_l * P, one ModDown per sum)
    int lift_mac = 1;  // double hoisting, depthwise: the MAC forms the rotated copies on the fly
    std::vector<int32_t> steps;
    double w_scale = 0;  // scale of the loaded weights (0 until fe_plan_load_weights)
    int repack = 0;      // 1: an FC-kind plan whose weights are the permutation from lin to lout
    std::vector<int> rowmap;  // FC-kind: output neuron -> row of the caller's weight matrix (-1: none)
    int w_rows = 0;           // rows of the caller's weight matrix when rowmap is used
    // FC-kind plaintext-matrix product given by its diagonals (fe_plan_lintrans):
    // plaintext k is diagonal lt_src[k].first rotated by -lt_src[k].second
    int lintrans = 0;
    std::vector<std::pair<int, int32_t>> lt_src;
    size_t lt_ndiag = 0;
};

namespace fe {
int layout_fill(int N, fe_layout* l);
size_t plan_workspace(const fe_plan* p, size_t chunk, size_t n_req = 1);
// fills steps, n_outer, modup_cts and modup_slot from inner / outs
void finish_plan(fe_plan* p);
size_t plan_data_bytes(const fe_plan* p, size_t chunk, size_t n_req);
size_t plan_table_bytes(const fe_plan* p, size_t chunk, size_t n_req);
size_t plan_chunk(const fe_plan* p, size_t n_req, int mode, size_t data_bytes, bool data_only);
// phase bit 1: upload item tables; bit 2: launch kernels.  n_req requests laid
// out contiguously (inputs [n_req][n_in] ct, outputs [n_req][n_out] ct).
int run_plan(fe_ctx* c, const fe_evk* evk, const fe_plan* p, const u64* in, const u64* pt, u64* out,
             void* ws, size_t ws_bytes, int mode, cudaStream_t st, int phase, int n_req = 1, int pt_pool = 0,
             void* data_ws = nullptr, size_t data_ws_bytes = 0);
}  // namespace fe
