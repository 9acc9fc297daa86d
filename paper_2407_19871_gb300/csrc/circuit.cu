// LocPIR circuits on the GPU: a host-side circuit builder (Algorithms 2-5 of the paper)
// and a level scheduler that runs all gates of one bootstrap level -- across every
// comparison, box and query of a call -- as one shared pre-combination / blind-rotation
// / key-switch pass.
//
// NOT gates cost nothing: a signal is (wire, negated) and a negation folds into the
// signs of the pre-combination coefficients of every gate that reads it (exactly equal
// mod 2^32 to negating the ciphertext first).  Trivial constants live in one pool slot.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "runtime.h"

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
static Sig comp_s(Circuit &C, int c1, int c2, int l, bool is_signed)
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
static Sig comp_le(Circuit &C, int a, int b, int l, bool is_signed)
{
    return Circuit::NOT(comp_s(C, b, a, l, is_signed));
}

// LocPIR (Algorithm 3) for one query; x, y, boxes, services are first input wires.
static std::vector<Sig> build_locpir(Circuit &C, int l, bool is_signed, int x, int y, int n_boxes, int boxes, int m,
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

// ---------------------------------------------------------------------------------
// Execution.
// ---------------------------------------------------------------------------------
struct InputCopy {
    int first_wire;
    const uint32_t *src;
    int count;
};
struct OutputCopy {
    Sig sig;
    uint32_t *dst;
};
struct CopyEntry {
    const uint32_t *src;
    uint32_t *dst;
    int32_t neg;
    int32_t pad;
};

__global__ void copy_entries_kernel(const CopyEntry *e, size_t cnt, int n)
{
    const int lane = threadIdx.x & 31;
    const size_t warps = (size_t)gridDim.x * (blockDim.x / 32);
    for (size_t g = (size_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); g < cnt; g += warps) {
        const CopyEntry E = e[g];
        for (int w = lane; w <= n; w += 32) {
            const uint32_t v = E.src[w];
            E.dst[w] = E.neg ? 0u - v : v;
        }
    }
}

static void gate_base(int op, uint32_t &cst, int &ca, int &cb)
{
    switch (op) {
    case LP_AND: cst = 0u - T_EIGHTH; ca = 1; cb = 1; break;
    case LP_NAND: cst = T_EIGHTH; ca = -1; cb = -1; break;
    case LP_OR: cst = T_EIGHTH; ca = 1; cb = 1; break;
    case LP_XOR: cst = T_QUARTER; ca = 2; cb = 2; break;
    default: cst = 0u - T_QUARTER; ca = -2; cb = -2; break;  // XNOR
    }
}

struct Pass {
    size_t br_off, br_cnt, ks_off, ks_cnt;
};

static int execute(lp_ctx *c, const Circuit &C, const std::vector<InputCopy> &ins, const std::vector<OutputCopy> &outs,
                   cudaStream_t st)
{
    const int n = c->params.n;
    const size_t W = (size_t)n + 1;
    const size_t nw = C.depth.size();
    int rc = ensure_buf(c->pool, nw * W * 4, "ciphertext pool");
    if (rc) return rc;
    uint32_t *pool = static_cast<uint32_t *>(c->pool.ptr);

    // Levels: nodes grouped by the bootstrap depth of their output, in creation order.
    int maxd = 0;
    for (const Node &nd : C.nodes) maxd = std::max(maxd, C.depth[nd.out]);
    std::vector<std::vector<int>> levels(maxd + 1);
    for (size_t i = 0; i < C.nodes.size(); i++) levels[C.depth[C.nodes[i].out]].push_back((int)i);

    const size_t MAXJ = 131072;
    std::vector<BrJob> br;
    std::vector<KsJob> ks;
    std::vector<Pass> passes;
    size_t max_pass = 1;
    for (int d = 1; d <= maxd; d++) {
        Pass ps{br.size(), 0, ks.size(), 0};
        for (int idx : levels[d]) {
            const Node &nd = C.nodes[idx];
            const size_t need = nd.op == LP_MUX ? 2 : 1;
            if (ps.br_cnt + need > MAXJ) {
                passes.push_back(ps);
                max_pass = std::max(max_pass, ps.br_cnt);
                ps = Pass{br.size(), 0, ks.size(), 0};
            }
            auto sgn = [](const Sig &s, int coef) { return s.neg ? -coef : coef; };
            KsJob kj;
            kj.out = nd.out;
            kj.e1 = (int)ps.br_cnt;
            if (nd.op == LP_MUX) {
                BrJob j1{}, j2{};
                j1.in[0] = nd.in[0].w; j1.coef[0] = sgn(nd.in[0], 1);
                j1.in[1] = nd.in[1].w; j1.coef[1] = sgn(nd.in[1], 1);
                j1.in[2] = 0;          j1.coef[2] = 0;
                j1.bconst = 0u - T_EIGHTH;
                j2.in[0] = nd.in[0].w; j2.coef[0] = sgn(nd.in[0], -1);
                j2.in[1] = nd.in[2].w; j2.coef[1] = sgn(nd.in[2], 1);
                j2.in[2] = 0;          j2.coef[2] = 0;
                j2.bconst = 0u - T_EIGHTH;
                br.push_back(j1);
                br.push_back(j2);
                kj.e2 = (int)ps.br_cnt + 1;
                kj.bconst = T_EIGHTH;
            } else {
                uint32_t cst; int ca, cb;
                gate_base(nd.op, cst, ca, cb);
                BrJob j{};
                j.in[0] = nd.in[0].w; j.coef[0] = sgn(nd.in[0], ca);
                j.in[1] = nd.in[1].w; j.coef[1] = sgn(nd.in[1], cb);
                j.in[2] = 0;          j.coef[2] = 0;
                j.bconst = cst;
                br.push_back(j);
                kj.e2 = -1;
                kj.bconst = 0u;
            }
            ks.push_back(kj);
            ps.br_cnt += need;
            ps.ks_cnt += 1;
        }
        if (ps.ks_cnt) {
            passes.push_back(ps);
            max_pass = std::max(max_pass, ps.br_cnt);
        }
    }

    std::vector<CopyEntry> outc;
    outc.reserve(outs.size());
    for (const OutputCopy &o : outs) outc.push_back(CopyEntry{pool + (size_t)o.sig.w * W, o.dst, o.sig.neg ? 1 : 0, 0});

    const size_t br_bytes = br.size() * sizeof(BrJob), ks_bytes = ks.size() * sizeof(KsJob);
    const size_t out_off = (br_bytes + ks_bytes + 255) & ~(size_t)255;
    rc = ensure_buf(c->jobs, out_off + outc.size() * sizeof(CopyEntry) + 256, "job records");
    if (!rc) rc = ensure_scratch(c, max_pass);
    if (rc) return rc;
    char *jb = static_cast<char *>(c->jobs.ptr);
    cudaError_t e = cudaSuccess;
    if (br_bytes) e = cudaMemcpyAsync(jb, br.data(), br_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && ks_bytes) e = cudaMemcpyAsync(jb + br_bytes, ks.data(), ks_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !outc.empty())
        e = cudaMemcpyAsync(jb + out_off, outc.data(), outc.size() * sizeof(CopyEntry), cudaMemcpyHostToDevice, st);
    for (const InputCopy &in : ins) {
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(pool + (size_t)in.first_wire * W, in.src, (size_t)in.count * W * 4,
                            cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess && C.zero_w >= 0) {
        e = launch_trivial(pool + (size_t)C.zero_w * W, n, 0u - T_EIGHTH, st);
        c->launches++;
    }
    if (e != cudaSuccess) return cuda_fail(e, "circuit setup");

    const BrJob *dbr = reinterpret_cast<const BrJob *>(jb);
    const KsJob *dks = reinterpret_cast<const KsJob *>(jb + br_bytes);
    for (const Pass &ps : passes) {
        e = launch_precomb_indexed(dbr + ps.br_off, ps.br_cnt, pool, n, static_cast<uint16_t *>(c->abar.ptr),
                                   abar_stride(c), c->num_sms, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "pre-combination launch");
        if ((rc = run_br(c, ps.br_cnt, T_EIGHTH, st))) return rc;
        if ((rc = run_ks(c, dks + ps.ks_off, ps.ks_cnt, 0, pool, st))) return rc;
    }
    if (!outc.empty()) {
        int grid = (int)std::min<size_t>((outc.size() + 7) / 8, (size_t)c->num_sms * 16);
        copy_entries_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const CopyEntry *>(jb + out_off), outc.size(), n);
        c->launches++;
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "output copy launch");
    }
    return LP_OK;
}

}  // namespace lp

using namespace lp;

static int check_ready(lp_ctx *c)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (!c->have_bsk || !c->have_ksk) return fail(LP_ENOKEY, "load the bootstrapping and key-switching keys first");
    cudaSetDevice(c->device);
    return LP_OK;
}

extern "C" int lp_compare_batch(lp_ctx *c, int kind, int is_signed, int l, const uint32_t *x1, const uint32_t *x2,
                                uint32_t *out, size_t count, void *stream)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (kind != LP_LT && kind != LP_LE) return fail(LP_EINVAL, "unknown comparison %d", kind);
    if (l < 1 || l > 64) return fail(LP_EINVAL, "bit width l=%d outside [1, 64]", l);
    if (count == 0) return LP_OK;
    if (!x1 || !x2 || !out) return fail(LP_EINVAL, "null pointer");
    const size_t W = (size_t)c->params.n + 1;
    Circuit C;
    std::vector<InputCopy> ins;
    std::vector<OutputCopy> outs;
    const int a = C.inputs((int)(count * l));
    const int b = C.inputs((int)(count * l));
    ins.push_back(InputCopy{a, x1, (int)(count * l)});
    ins.push_back(InputCopy{b, x2, (int)(count * l)});
    for (size_t g = 0; g < count; g++) {
        const int u = a + (int)g * l, v = b + (int)g * l;
        Sig s = kind == LP_LT ? comp_s(C, u, v, l, is_signed != 0) : comp_le(C, u, v, l, is_signed != 0);
        outs.push_back(OutputCopy{s, out + g * W});
    }
    return execute(c, C, ins, outs, static_cast<cudaStream_t>(stream));
}

static int check_query(const lp_query &q)
{
    if (q.l < 1 || q.l > 64) return fail(LP_EINVAL, "bit width l=%d outside [1, 64]", q.l);
    if (q.n_boxes < 1) return fail(LP_EINVAL, "n_boxes=%d < 1", q.n_boxes);
    if (q.m < 1) return fail(LP_EINVAL, "service length m=%d < 1", q.m);
    if (q.comb < LP_XOR_TREE || q.comb > LP_OR_TREE) return fail(LP_EINVAL, "unknown combine %d", q.comb);
    if (!q.x || !q.y || !q.boxes || !q.services || !q.out_service) return fail(LP_EINVAL, "null pointer in query");
    return LP_OK;
}

extern "C" int lp_locpir_batch(lp_ctx *c, const lp_query *q, size_t nq, void *stream)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (nq == 0) return LP_OK;
    if (!q) return fail(LP_EINVAL, "null query array");
    const size_t W = (size_t)c->params.n + 1;
    Circuit C;
    std::vector<InputCopy> ins;
    std::vector<OutputCopy> outs;
    for (size_t i = 0; i < nq; i++) {
        if ((rc = check_query(q[i]))) return rc;
        const lp_query &Q = q[i];
        const int x = C.inputs(Q.l), y = C.inputs(Q.l);
        const int bx = C.inputs(4 * Q.l * Q.n_boxes);
        const int sv = C.inputs(Q.m * Q.n_boxes);
        ins.push_back(InputCopy{x, Q.x, Q.l});
        ins.push_back(InputCopy{y, Q.y, Q.l});
        ins.push_back(InputCopy{bx, Q.boxes, 4 * Q.l * Q.n_boxes});
        ins.push_back(InputCopy{sv, Q.services, Q.m * Q.n_boxes});
        std::vector<Sig> S = build_locpir(C, Q.l, Q.is_signed != 0, x, y, Q.n_boxes, bx, Q.m, sv, Q.comb);
        for (int j = 0; j < Q.m; j++) outs.push_back(OutputCopy{S[j], Q.out_service + (size_t)j * W});
    }
    return execute(c, C, ins, outs, static_cast<cudaStream_t>(stream));
}

extern "C" int lp_locpir_query(lp_ctx *c, int l, int is_signed, const uint32_t *x, const uint32_t *y, int n_boxes,
                               const uint32_t *boxes, int m, const uint32_t *services, int comb, uint32_t *out_service,
                               void *stream)
{
    lp_query q{l, is_signed, n_boxes, m, comb, x, y, boxes, services, out_service};
    return lp_locpir_batch(c, &q, 1, stream);
}
