// Host-side LocPIR circuit builder shared by the batch entry points and the server:
// Algorithms 2-5 of the paper as a gate DAG over numbered wires (see circuit.cu).
#pragma once
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace lp {

struct Sig {
    int32_t w = -1;
    bool neg = false;
};

struct Node {
    int op;
    Sig in[3];
    int32_t out;
};

struct Circuit {
    std::vector<int> depth;   // per wire
    std::vector<Node> nodes;
    int zero_w = -1;

    int wire(int d)
    {
        depth.push_back(d);
        return (int)depth.size() - 1;
    }
    // k consecutive input wires.
    int inputs(int k)
    {
        const int first = (int)depth.size();
        for (int i = 0; i < k; i++) wire(0);
        return first;
    }
    Sig zero()
    {
        if (zero_w < 0) zero_w = wire(0);
        return Sig{zero_w, false};
    }
    static Sig NOT(Sig a) { return Sig{a.w, !a.neg}; }
    Sig gate(int op, Sig a, Sig b, Sig c = Sig{})
    {
        int d = std::max(depth[a.w], depth[b.w]);
        if (op == LP_MUX) d = std::max(d, depth[c.w]);
        const int w = wire(d + 1);
        Node nd;
        nd.op = op;
        nd.in[0] = a;
        nd.in[1] = b;
        nd.in[2] = c;
        nd.out = w;
        nodes.push_back(nd);
        return Sig{w, false};
    }
};

// HomCompS (Algorithm 2): t0 = Enc(0); with is_signed, both MSBs are flipped (lines 2-3);
// for i = 0 .. l-1 (LSB first): t1 = XNOR(c1[i], c2[i]); t0 = MUX(t1, t0, c2[i]).
inline Sig comp_s(Circuit &C, int c1, int c2, int l, bool is_signed)
{
    Sig t0 = C.zero();
    for (int i = 0; i < l; i++) {
        Sig a{c1 + i, false}, b{c2 + i, false};
        if (is_signed && i == l - 1) {
            a = Circuit::NOT(a);
            b = Circuit::NOT(b);
        }
        Sig t1 = C.gate(LP_XNOR, a, b);
        t0 = C.gate(LP_MUX, t1, t0, b);
    }
    return t0;
}

// HomCompLE(a, b) = a <= b = NOT HomCompS(b, a).
inline Sig comp_le(Circuit &C, int a, int b, int l, bool is_signed)
{
    return Circuit::NOT(comp_s(C, b, a, l, is_signed));
}

// Comparator x < K with K known in the clear (beyond the paper): Algorithm 2 with c2's bits
// known.  XNOR(a, k) is a (k = 1) or NOT a (k = 0); MUX(t1, t0, k) = t1 ? t0 : k becomes
// AND(NOT a, t0) for k = 0 and OR(NOT a, t0) for k = 1.  While t0 is a known constant c, a
// step keeps c when k = c and yields NOT a otherwise, without a gate.
inline Sig comp_s_known(Circuit &C, int c1, uint64_t K, int l, bool is_signed)
{
    const int cst = 0;
    bool known = true;
    Sig t0;
    for (int i = 0; i < l; i++) {
        Sig a{c1 + i, false};
        int k = (int)((K >> i) & 1u);
        if (is_signed && i == l - 1) {
            a = Circuit::NOT(a);
            k ^= 1;
        }
        const Sig na = Circuit::NOT(a);
        if (known) {
            if (k != cst) {
                t0 = na;
                known = false;
            }
        } else {
            t0 = C.gate(k ? LP_OR : LP_AND, na, t0);
        }
    }
    return known ? Sig{C.zero().w, cst != 0} : t0;
}

// The combine of the per-box services (Algorithm 4): XOR chain as printed, or a pairwise
// XOR / OR tree over boxes.
inline std::vector<Sig> build_locpir_rows(Circuit &C, std::vector<std::vector<Sig>> &rows, int m, int comb)
{
    if (comb == LP_XOR_CHAIN) {  // Algorithm 4 as printed (its S_i[j] target read as S[j])
        std::vector<Sig> S(m, C.zero());
        for (auto &Si : rows)
            for (int j = 0; j < m; j++) S[j] = C.gate(LP_XOR, S[j], Si[j]);
        return S;
    }
    const int op = comb == LP_OR_TREE ? LP_OR : LP_XOR;
    while (rows.size() > 1) {
        std::vector<std::vector<Sig>> next;
        for (size_t i = 0; i + 1 < rows.size(); i += 2) {
            std::vector<Sig> r(m);
            for (int j = 0; j < m; j++) r[j] = C.gate(op, rows[i][j], rows[i + 1][j]);
            next.push_back(std::move(r));
        }
        if (rows.size() % 2) next.push_back(std::move(rows.back()));
        rows.swap(next);
    }
    return rows[0];
}

// LocPIR (Algorithm 3) with known bounds [n_boxes][4] = (X1, X2, Y1, Y2): X1 <= x is
// NOT(x < X1), x < X2 is comp_s_known; validation, bitwiseAND and combine as build_locpir.
inline std::vector<Sig> build_locpir_known(Circuit &C, int l, bool is_signed, int x, int y, int n_boxes,
                                           const uint64_t *bounds, int m, int services, int comb)
{
    std::vector<std::vector<Sig>> rows;
    rows.reserve(n_boxes);
    for (int i = 0; i < n_boxes; i++) {
        const uint64_t *b = bounds + 4 * (size_t)i;
        Sig xl = Circuit::NOT(comp_s_known(C, x, b[0], l, is_signed));
        Sig xr = comp_s_known(C, x, b[1], l, is_signed);
        Sig yl = Circuit::NOT(comp_s_known(C, y, b[2], l, is_signed));
        Sig yr = comp_s_known(C, y, b[3], l, is_signed);
        Sig v1 = C.gate(LP_AND, xl, xr);
        Sig v2 = C.gate(LP_AND, yl, yr);
        Sig f = C.gate(LP_AND, v1, v2);
        std::vector<Sig> Si(m);
        for (int j = 0; j < m; j++) Si[j] = C.gate(LP_AND, f, Sig{services + i * m + j, false});  // Algorithm 5
        rows.push_back(std::move(Si));
    }
    return build_locpir_rows(C, rows, m, comb);
}

// LocPIR (Algorithm 3) for one query; x, y, boxes, services are first input wires.
inline std::vector<Sig> build_locpir(Circuit &C, int l, bool is_signed, int x, int y, int n_boxes, int boxes, int m,
                                     int services, int comb)
{
    std::vector<std::vector<Sig>> rows;
    rows.reserve(n_boxes);
    for (int i = 0; i < n_boxes; i++) {
        const int X1 = boxes + (4 * i + 0) * l, X2 = boxes + (4 * i + 1) * l;
        const int Y1 = boxes + (4 * i + 2) * l, Y2 = boxes + (4 * i + 3) * l;
        Sig xl = comp_le(C, X1, x, l, is_signed);
        Sig xr = comp_s(C, x, X2, l, is_signed);
        Sig yl = comp_le(C, Y1, y, l, is_signed);
        Sig yr = comp_s(C, y, Y2, l, is_signed);
        Sig v1 = C.gate(LP_AND, xl, xr);
        Sig v2 = C.gate(LP_AND, yl, yr);
        Sig f = C.gate(LP_AND, v1, v2);
        std::vector<Sig> Si(m);
        for (int j = 0; j < m; j++) Si[j] = C.gate(LP_AND, f, Sig{services + i * m + j, false});  // Algorithm 5
        rows.push_back(std::move(Si));
    }
    return build_locpir_rows(C, rows, m, comb);
}

// Pre-combination of a two-input gate (LocPIR Section 2.2; the TFHE gates it refers to).
inline void gate_base(int op, uint32_t &cst, int &ca, int &cb)
{
    switch (op) {
    case LP_AND: cst = 0u - T_EIGHTH; ca = 1; cb = 1; break;
    case LP_NAND: cst = T_EIGHTH; ca = -1; cb = -1; break;
    case LP_OR: cst = T_EIGHTH; ca = 1; cb = 1; break;
    case LP_XOR: cst = T_QUARTER; ca = 2; cb = 2; break;
    default: cst = 0u - T_QUARTER; ca = -2; cb = -2; break;  // XNOR
    }
}

// Append the blind-rotation jobs and the key-switch job of one gate; wires are offset by
// `base` (the gate's circuit position in a shared pool) and e1/e2 index the pass's jobs.
inline void append_gate_jobs(const Node &nd, int base, size_t pass_br, std::vector<BrJob> &br, std::vector<KsJob> &ks)
{
    auto sgn = [](const Sig &s, int coef) { return s.neg ? -coef : coef; };
    KsJob kj;
    kj.out = base + nd.out;
    kj.e1 = (int)pass_br;
    if (nd.op == LP_MUX) {
        BrJob j1{}, j2{};
        j1.in[0] = base + nd.in[0].w; j1.coef[0] = sgn(nd.in[0], 1);
        j1.in[1] = base + nd.in[1].w; j1.coef[1] = sgn(nd.in[1], 1);
        j1.bconst = 0u - T_EIGHTH;
        j2.in[0] = base + nd.in[0].w; j2.coef[0] = sgn(nd.in[0], -1);
        j2.in[1] = base + nd.in[2].w; j2.coef[1] = sgn(nd.in[2], 1);
        j2.bconst = 0u - T_EIGHTH;
        br.push_back(j1);
        br.push_back(j2);
        kj.e2 = (int)pass_br + 1;
        kj.bconst = T_EIGHTH;
    } else {
        uint32_t cst; int ca, cb;
        gate_base(nd.op, cst, ca, cb);
        BrJob j{};
        j.in[0] = base + nd.in[0].w; j.coef[0] = sgn(nd.in[0], ca);
        j.in[1] = base + nd.in[1].w; j.coef[1] = sgn(nd.in[1], cb);
        j.bconst = cst;
        br.push_back(j);
        kj.e2 = -1;
        kj.bconst = 0u;
    }
    ks.push_back(kj);
}

// Gates grouped by the bootstrap depth of their output (index 0 unused), in creation order.
inline std::vector<std::vector<int>> levels_of(const Circuit &C)
{
    int maxd = 0;
    for (const Node &nd : C.nodes) maxd = std::max(maxd, C.depth[nd.out]);
    std::vector<std::vector<int>> lv(maxd + 1);
    for (size_t i = 0; i < C.nodes.size(); i++) lv[C.depth[C.nodes[i].out]].push_back((int)i);
    return lv;
}

// One ciphertext copied entry (pool <-> caller), optionally negated.
cudaError_t launch_copy_entries(const CopyEntry *e, size_t cnt, int n, int num_sms, cudaStream_t st);

// Argument checks of one LocPIR query (LP_EINVAL with a message).
int check_query(const lp_query &q);

}  // namespace lp
