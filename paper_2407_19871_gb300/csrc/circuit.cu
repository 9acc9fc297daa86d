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

#include "circuit.h"
#include "common.cuh"
#include "kernels.h"
#include "runtime.h"

namespace lp {

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

struct Pass {
    size_t br_off, br_cnt, ks_off, ks_cnt;
};

// A levelled schedule: job records of every pass, in bootstrap-level order, plus the copies
// in and out of the ciphertext pool.  Pool addresses in `outc` are offsets (in words) until
// the pool is known.
struct Schedule {
    std::vector<BrJob> br;
    std::vector<KsJob> ks;
    std::vector<Pass> passes;
    std::vector<CopyEntry> outc;
    std::vector<InputCopy> ins;
    std::vector<ExecPass> xpass;   // the passes for the persistent executor
    size_t max_pass = 1, nwires = 0, br_bytes = 0, ks_bytes = 0, out_off = 0, xpass_off = 0, ctl_off = 0,
           job_bytes = 0;
    int zero_w = -1;
};

static void schedule(const Circuit &C, const std::vector<InputCopy> &ins, const std::vector<OutputCopy> &outs, int n,
                     Schedule &S)
{
    const size_t W = (size_t)n + 1;
    const std::vector<std::vector<int>> levels = levels_of(C);
    const int maxd = (int)levels.size() - 1;
    const size_t MAXJ = 131072;
    for (int d = 1; d <= maxd; d++) {
        Pass ps{S.br.size(), 0, S.ks.size(), 0};
        for (int idx : levels[d]) {
            const Node &nd = C.nodes[idx];
            const size_t need = nd.op == LP_MUX ? 2 : 1;
            if (ps.br_cnt + need > MAXJ) {
                S.passes.push_back(ps);
                S.max_pass = std::max(S.max_pass, ps.br_cnt);
                ps = Pass{S.br.size(), 0, S.ks.size(), 0};
            }
            append_gate_jobs(nd, 0, ps.br_cnt, S.br, S.ks);
            ps.br_cnt += need;
            ps.ks_cnt += 1;
        }
        if (ps.ks_cnt) {
            S.passes.push_back(ps);
            S.max_pass = std::max(S.max_pass, ps.br_cnt);
        }
    }
    for (const OutputCopy &o : outs)
        S.outc.push_back(CopyEntry{reinterpret_cast<const uint32_t *>((size_t)o.sig.w * W), o.dst, o.sig.neg ? 1 : 0, 0});
    S.ins = ins;
    S.zero_w = C.zero_w;
    S.nwires = C.depth.size();
    for (const Pass &ps : S.passes)
        S.xpass.push_back(ExecPass{(uint32_t)ps.br_off, (uint32_t)ps.br_cnt, (uint32_t)ps.ks_off, (uint32_t)ps.ks_cnt});
    S.br_bytes = S.br.size() * sizeof(BrJob);
    S.ks_bytes = S.ks.size() * sizeof(KsJob);
    S.out_off = (S.br_bytes + S.ks_bytes + 255) & ~(size_t)255;
    S.xpass_off = (S.out_off + S.outc.size() * sizeof(CopyEntry) + 255) & ~(size_t)255;
    S.ctl_off = (S.xpass_off + S.xpass.size() * sizeof(ExecPass) + 255) & ~(size_t)255;
    S.job_bytes = S.ctl_off + exec_ctl_words((int)S.xpass.size()) * sizeof(uint32_t) + 256;
}

// Buffers a schedule runs on.
struct RunBufs {
    uint32_t *pool;
    char *jobs;
    uint16_t *abar;
    uint32_t *ext;
};

// Upload the job records (host -> device, on st).
static cudaError_t upload_schedule(Schedule &S, const RunBufs &B, cudaStream_t st)
{
    for (CopyEntry &e : S.outc)
        e.src = B.pool + reinterpret_cast<size_t>(e.src);   // offsets -> pool addresses
    cudaError_t e = cudaSuccess;
    if (S.br_bytes) e = cudaMemcpyAsync(B.jobs, S.br.data(), S.br_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && S.ks_bytes)
        e = cudaMemcpyAsync(B.jobs + S.br_bytes, S.ks.data(), S.ks_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !S.outc.empty())
        e = cudaMemcpyAsync(B.jobs + S.out_off, S.outc.data(), S.outc.size() * sizeof(CopyEntry),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !S.xpass.empty())
        e = cudaMemcpyAsync(B.jobs + S.xpass_off, S.xpass.data(), S.xpass.size() * sizeof(ExecPass),
                            cudaMemcpyHostToDevice, st);
    return e;
}

// Enqueue the whole evaluation: inputs into the pool, every level's passes, outputs out.
// Only stream-ordered work: the same sequence is captured into a CUDA graph by plans.
static int enqueue_schedule(lp_ctx *c, const Schedule &S, const RunBufs &B, cudaStream_t st, bool timed)
{
    const int n = c->params.n;
    const size_t W = (size_t)n + 1;
    cudaError_t e = cudaSuccess;
    for (const InputCopy &in : S.ins) {
        e = cudaMemcpyAsync(B.pool + (size_t)in.first_wire * W, in.src, (size_t)in.count * W * 4,
                            cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "circuit input copy");
    }
    if (S.zero_w >= 0) {
        e = launch_trivial(B.pool + (size_t)S.zero_w * W, n, 0u - T_EIGHTH, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "trivial constant");
    }
    const BrJob *dbr = reinterpret_cast<const BrJob *>(B.jobs);
    const KsJob *dks = reinterpret_cast<const KsJob *>(B.jobs + S.br_bytes);
    int *err = static_cast<int *>(c->err.ptr);
    if (c->executor == LP_EXEC_PERSISTENT) {
        // One persistent launch runs every pass and the output copies; its control words start
        // at zero on every run (a memset node when captured into a plan's graph).
        uint32_t *ctl = reinterpret_cast<uint32_t *>(B.jobs + S.ctl_off);
        e = cudaMemsetAsync(ctl, 0, exec_ctl_words((int)S.xpass.size()) * sizeof(uint32_t), st);
        if (e != cudaSuccess) return cuda_fail(e, "executor control words");
        ExecArgs x{reinterpret_cast<const ExecPass *>(B.jobs + S.xpass_off), (int)S.xpass.size(), dbr, dks,
                   reinterpret_cast<const CopyEntry *>(B.jobs + S.out_off), (uint32_t)S.outc.size(), B.pool, B.abar,
                   abar_stride(c), B.ext, static_cast<const uint32_t *>(c->bsk_hat.ptr),
                   static_cast<const uint2 *>(c->tw_lane.ptr), static_cast<const uint32_t *>(c->ksk.ptr), n,
                   c->ks_slice_max, err, ctl, 0};
        cudaEvent_t ev0 = nullptr;
        if (timed) timer_begin(c, "exec", st, &ev0);
        e = launch_exec(x, c->num_sms, st);
        if (timed) timer_end(c, "exec", st, ev0);
        c->launches++;
        return e == cudaSuccess ? LP_OK : cuda_fail(e, "persistent executor launch");
    }
    for (const Pass &ps : S.passes) {
        e = launch_precomb_indexed(dbr + ps.br_off, ps.br_cnt, B.pool, n, B.abar, abar_stride(c), c->num_sms, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "pre-combination launch");
        cudaEvent_t ev0 = nullptr;
        if (timed) timer_begin(c, "br", st, &ev0);
        int launched = 0;
        e = launch_br(B.abar, abar_stride(c), B.ext, static_cast<const uint32_t *>(c->bsk_hat.ptr),
                      static_cast<const uint2 *>(c->tw_lane.ptr), n, (int)ps.br_cnt, T_EIGHTH, err, c->num_sms, st,
                      BR_VARIANT_AUTO, c->br_split_max, c->br_tail_split, br_pair_limit(c), br_quad_limit(c), &launched);
        if (timed) timer_end(c, "br", st, ev0);
        c->launches += launched;
        if (e != cudaSuccess) return cuda_fail(e, "blind rotation launch");
        if (timed) timer_begin(c, "ks", st, &ev0);
        e = launch_ks(B.ext, dks + ps.ks_off, ps.ks_cnt, 0, B.pool, static_cast<const uint32_t *>(c->ksk.ptr), n, err,
                      c->num_sms, st, c->ks_slice_max, &launched);
        if (timed) timer_end(c, "ks", st, ev0);
        c->launches += launched;
        if (e != cudaSuccess) return cuda_fail(e, "key switch launch");
    }
    if (!S.outc.empty()) {
        e = launch_copy_entries(reinterpret_cast<const CopyEntry *>(B.jobs + S.out_off), S.outc.size(), n, c->num_sms, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "output copy launch");
    }
    return LP_OK;
}

static int execute(lp_ctx *c, const Circuit &C, const std::vector<InputCopy> &ins, const std::vector<OutputCopy> &outs,
                   cudaStream_t st)
{
    const int n = c->params.n;
    const size_t W = (size_t)n + 1;
    Schedule S;
    schedule(C, ins, outs, n, S);
    int rc = ensure_buf(c->pool, S.nwires * W * 4, "ciphertext pool");
    if (!rc) rc = ensure_buf(c->jobs, S.job_bytes, "job records");
    if (!rc) rc = ensure_scratch(c, S.max_pass);
    if (rc) return rc;
    RunBufs B{static_cast<uint32_t *>(c->pool.ptr), static_cast<char *>(c->jobs.ptr),
              static_cast<uint16_t *>(c->abar.ptr), static_cast<uint32_t *>(c->ext.ptr)};
    cudaError_t e = upload_schedule(S, B, st);
    if (e != cudaSuccess) return cuda_fail(e, "upload job records");
    return enqueue_schedule(c, S, B, st, c->timing);
}

cudaError_t launch_copy_entries(const CopyEntry *e, size_t cnt, int n, int num_sms, cudaStream_t st)
{
    if (!cnt) return cudaSuccess;
    const int grid = (int)std::min<size_t>((cnt + 7) / 8, (size_t)num_sms * 16);
    copy_entries_kernel<<<grid, 256, 0, st>>>(e, cnt, n);
    return cudaGetLastError();
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

int lp::check_query(const lp_query &q)
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

// Device bytes a built circuit needs while it runs: its ciphertext pool and its job records
// (the pass scratch is bounded separately by the largest pass).
static size_t circuit_bytes(const Circuit &C, size_t outputs, int n)
{
    const size_t W = (size_t)n + 1;
    size_t br = 0;
    for (const Node &nd : C.nodes) br += nd.op == LP_MUX ? 2 : 1;
    return C.depth.size() * W * 4 + br * sizeof(BrJob) + C.nodes.size() * sizeof(KsJob) + outputs * sizeof(CopyEntry);
}

extern "C" int lp_locpir_batch_waves(lp_ctx *c, const lp_query *q, size_t nq, size_t mem_budget, size_t *waves_out,
                                     void *stream)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (waves_out) *waves_out = 0;
    if (nq == 0) return LP_OK;
    if (!q) return fail(LP_EINVAL, "null query array");
    for (size_t i = 0; i < nq; i++)
        if ((rc = check_query(q[i]))) return rc;
    const int n = c->params.n;
    const size_t W = (size_t)n + 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    size_t next = 0, waves = 0;
    while (next < nq) {
        // Grow the wave query by query; a query that takes it over the budget is taken back
        // (the builder only appends, so truncating restores the circuit) and opens the next wave.
        Circuit C;
        std::vector<InputCopy> ins;
        std::vector<OutputCopy> outs;
        size_t first = next;
        while (next < nq) {
            const size_t nw = C.depth.size(), nn = C.nodes.size(), ni = ins.size(), no = outs.size();
            const int zw = C.zero_w;
            const lp_query &Q = q[next];
            const int x = C.inputs(Q.l), y = C.inputs(Q.l);
            const int bx = C.inputs(4 * Q.l * Q.n_boxes);
            const int sv = C.inputs(Q.m * Q.n_boxes);
            ins.push_back(InputCopy{x, Q.x, Q.l});
            ins.push_back(InputCopy{y, Q.y, Q.l});
            ins.push_back(InputCopy{bx, Q.boxes, 4 * Q.l * Q.n_boxes});
            ins.push_back(InputCopy{sv, Q.services, Q.m * Q.n_boxes});
            std::vector<Sig> S = build_locpir(C, Q.l, Q.is_signed != 0, x, y, Q.n_boxes, bx, Q.m, sv, Q.comb);
            for (int j = 0; j < Q.m; j++) outs.push_back(OutputCopy{S[j], Q.out_service + (size_t)j * W});
            if (circuit_bytes(C, outs.size(), n) > mem_budget) {
                if (next == first)
                    return fail(LP_ENOMEM, "query %zu alone needs %zu bytes, above the memory budget of %zu", next,
                                circuit_bytes(C, outs.size(), n), mem_budget);
                C.depth.resize(nw);
                C.nodes.resize(nn);
                C.zero_w = zw;
                ins.resize(ni);
                outs.resize(no);
                break;
            }
            next++;
        }
        if ((rc = execute(c, C, ins, outs, st))) return rc;
        waves++;
    }
    if (waves_out) *waves_out = waves;
    return LP_OK;
}

extern "C" int lp_locpir_query(lp_ctx *c, int l, int is_signed, const uint32_t *x, const uint32_t *y, int n_boxes,
                               const uint32_t *boxes, int m, const uint32_t *services, int comb, uint32_t *out_service,
                               void *stream)
{
    lp_query q{l, is_signed, n_boxes, m, comb, x, y, boxes, services, out_service};
    return lp_locpir_batch(c, &q, 1, stream);
}

// ---------------------------------------------------------------------------------
// Server-known bounds (beyond the paper).
// ---------------------------------------------------------------------------------
extern "C" int lp_compare_known_batch(lp_ctx *c, int kind, int is_signed, int l, const uint32_t *x, const uint64_t *k,
                                      uint32_t *out, size_t count, void *stream)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (kind != LP_LT && kind != LP_LE) return fail(LP_EINVAL, "unknown comparison %d", kind);
    if (l < 1 || l > 64) return fail(LP_EINVAL, "bit width l=%d outside [1, 64]", l);
    if (count == 0) return LP_OK;
    if (!x || !k || !out) return fail(LP_EINVAL, "null pointer");
    const size_t W = (size_t)c->params.n + 1;
    Circuit C;
    std::vector<InputCopy> ins;
    std::vector<OutputCopy> outs;
    const int a = C.inputs((int)(count * l));
    ins.push_back(InputCopy{a, x, (int)(count * l)});
    for (size_t g = 0; g < count; g++) {
        const Sig s = comp_s_known(C, a + (int)g * l, k[g], l, is_signed != 0);
        outs.push_back(OutputCopy{kind == LP_LT ? s : Circuit::NOT(s), out + g * W});
    }
    return execute(c, C, ins, outs, static_cast<cudaStream_t>(stream));
}

extern "C" int lp_locpir_known_batch(lp_ctx *c, const lp_query_known *q, size_t nq, void *stream)
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
        const lp_query_known &Q = q[i];
        // Same argument rules as an encrypted-bounds query (the bounds pointer stands in for boxes).
        lp_query chk{Q.l, Q.is_signed, Q.n_boxes, Q.m, Q.comb, Q.x, Q.y, reinterpret_cast<const uint32_t *>(Q.bounds),
                     Q.services, Q.out_service};
        if ((rc = check_query(chk))) return rc;
        const int x = C.inputs(Q.l), y = C.inputs(Q.l);
        const int sv = C.inputs(Q.m * Q.n_boxes);
        ins.push_back(InputCopy{x, Q.x, Q.l});
        ins.push_back(InputCopy{y, Q.y, Q.l});
        ins.push_back(InputCopy{sv, Q.services, Q.m * Q.n_boxes});
        std::vector<Sig> S = build_locpir_known(C, Q.l, Q.is_signed != 0, x, y, Q.n_boxes, Q.bounds, Q.m, sv, Q.comb);
        for (int j = 0; j < Q.m; j++) outs.push_back(OutputCopy{S[j], Q.out_service + (size_t)j * W});
    }
    return execute(c, C, ins, outs, static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------------
// Gate statistics of one query's circuit, host only (no context, no device call).
extern "C" int lp_circuit_info(int l, int is_signed, int n_boxes, int m, int comb, const uint64_t *bounds,
                               lp_circuit_stats *out)
{
    if (!out) return fail(LP_EINVAL, "null output pointer");
    if (l < 1 || l > 64) return fail(LP_EINVAL, "bit width l=%d outside [1, 64]", l);
    if (n_boxes < 1) return fail(LP_EINVAL, "n_boxes=%d < 1", n_boxes);
    if (m < 1) return fail(LP_EINVAL, "service length m=%d < 1", m);
    if (comb < LP_XOR_TREE || comb > LP_OR_TREE) return fail(LP_EINVAL, "unknown combine %d", comb);
    Circuit C;
    const int x = C.inputs(l), y = C.inputs(l);
    if (bounds) {
        const int sv = C.inputs(m * n_boxes);
        build_locpir_known(C, l, is_signed != 0, x, y, n_boxes, bounds, m, sv, comb);
    } else {
        const int bx = C.inputs(4 * l * n_boxes);
        const int sv = C.inputs(m * n_boxes);
        build_locpir(C, l, is_signed != 0, x, y, n_boxes, bx, m, sv, comb);
    }
    lp_circuit_stats st{};
    for (const Node &nd : C.nodes) {
        st.gates_by_op[nd.op]++;
        st.blind_rotations += nd.op == LP_MUX ? 2 : 1;
    }
    st.key_switches = C.nodes.size();
    const std::vector<std::vector<int>> lv = levels_of(C);
    for (size_t d = 1; d < lv.size(); d++) {
        uint64_t br = 0;
        for (int g : lv[d]) br += C.nodes[g].op == LP_MUX ? 2 : 1;
        if (!lv[d].empty()) st.levels++;
        st.widest_level = std::max(st.widest_level, br);
    }
    st.wires = C.depth.size();
    *out = st;
    return LP_OK;
}

// Plans: a LocPIR batch scheduled once and captured into a CUDA graph.
// ---------------------------------------------------------------------------------
struct lp_plan {
    lp_ctx *c = nullptr;
    Schedule S;
    DevBuf pool, jobs, abar, ext;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0, blind_rotations = 0, key_switches = 0;
};

static void plan_free(lp_plan *P)
{
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    for (DevBuf *b : {&P->pool, &P->jobs, &P->abar, &P->ext}) free_buf(*b);
    delete P;
}

// Schedule a built circuit once, allocate the plan's pool and scratch, and capture the whole
// evaluation into a CUDA graph.
static int make_plan(lp_ctx *c, const Circuit &C, const std::vector<InputCopy> &ins,
                     const std::vector<OutputCopy> &outs, lp_plan **out)
{
    const int n = c->params.n;
    const size_t W = (size_t)n + 1;
    int rc = LP_OK;
    lp_plan *P = new lp_plan();
    P->c = c;
    schedule(C, ins, outs, n, P->S);
    for (const Pass &ps : P->S.passes) {
        P->blind_rotations += ps.br_cnt;
        P->key_switches += ps.ks_cnt;
    }
    rc = ensure_buf(P->pool, P->S.nwires * W * 4, "plan pool");
    if (!rc) rc = ensure_buf(P->jobs, P->S.job_bytes, "plan job records");
    if (!rc) rc = ensure_buf(P->abar, P->S.max_pass * abar_stride(c) * sizeof(uint16_t), "plan scratch");
    if (!rc) rc = ensure_buf(P->ext, P->S.max_pass * EXT_STRIDE * sizeof(uint32_t), "plan scratch");
    if (rc) {
        plan_free(P);
        return rc;
    }
    RunBufs B{static_cast<uint32_t *>(P->pool.ptr), static_cast<char *>(P->jobs.ptr),
              static_cast<uint16_t *>(P->abar.ptr), static_cast<uint32_t *>(P->ext.ptr)};
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = upload_schedule(P->S, B, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        plan_free(P);
        return cuda_fail(e, "plan setup");
    }
    const uint64_t l0 = c->launches;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        rc = enqueue_schedule(c, P->S, B, st, false);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(st, &g);
        P->graph = g;
        if (!rc && e2 != cudaSuccess) rc = cuda_fail(e2, "end graph capture");
    } else {
        rc = cuda_fail(e, "begin graph capture");
    }
    P->kernels = c->launches - l0;
    c->launches = l0;
    if (!rc) {
        e = cudaGraphInstantiate(&P->exec, P->graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "instantiate graph");
    }
    cudaStreamDestroy(st);
    if (rc) {
        plan_free(P);
        return rc;
    }
    *out = P;
    return LP_OK;
}

extern "C" int lp_plan_locpir(lp_ctx *c, const lp_query *q, size_t nq, lp_plan **out)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (!q || !out || nq == 0) return fail(LP_EINVAL, "empty or null query list");
    *out = nullptr;
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
        std::vector<Sig> Sv = build_locpir(C, Q.l, Q.is_signed != 0, x, y, Q.n_boxes, bx, Q.m, sv, Q.comb);
        for (int j = 0; j < Q.m; j++) outs.push_back(OutputCopy{Sv[j], Q.out_service + (size_t)j * W});
    }
    return make_plan(c, C, ins, outs, out);
}

extern "C" int lp_plan_locpir_known(lp_ctx *c, const lp_query_known *q, size_t nq, lp_plan **out)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (!q || !out || nq == 0) return fail(LP_EINVAL, "empty or null query list");
    *out = nullptr;
    const size_t W = (size_t)c->params.n + 1;
    Circuit C;
    std::vector<InputCopy> ins;
    std::vector<OutputCopy> outs;
    for (size_t i = 0; i < nq; i++) {
        const lp_query_known &Q = q[i];
        lp_query chk{Q.l, Q.is_signed, Q.n_boxes, Q.m, Q.comb, Q.x, Q.y, reinterpret_cast<const uint32_t *>(Q.bounds),
                     Q.services, Q.out_service};
        if ((rc = check_query(chk))) return rc;
        const int x = C.inputs(Q.l), y = C.inputs(Q.l);
        const int sv = C.inputs(Q.m * Q.n_boxes);
        ins.push_back(InputCopy{x, Q.x, Q.l});
        ins.push_back(InputCopy{y, Q.y, Q.l});
        ins.push_back(InputCopy{sv, Q.services, Q.m * Q.n_boxes});
        std::vector<Sig> Sv = build_locpir_known(C, Q.l, Q.is_signed != 0, x, y, Q.n_boxes, Q.bounds, Q.m, sv, Q.comb);
        for (int j = 0; j < Q.m; j++) outs.push_back(OutputCopy{Sv[j], Q.out_service + (size_t)j * W});
    }
    return make_plan(c, C, ins, outs, out);
}

extern "C" int lp_plan_run(lp_plan *P, void *stream)
{
    if (!P) return fail(LP_EINVAL, "null plan");
    cudaSetDevice(P->c->device);
    cudaError_t e = cudaGraphLaunch(P->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    P->c->launches += P->kernels;
    return LP_OK;
}

extern "C" int lp_plan_info(const lp_plan *P, uint64_t *blind_rotations, uint64_t *key_switches, uint64_t *kernels)
{
    if (!P) return fail(LP_EINVAL, "null plan");
    if (blind_rotations) *blind_rotations = P->blind_rotations;
    if (key_switches) *key_switches = P->key_switches;
    if (kernels) *kernels = P->kernels;
    return LP_OK;
}

extern "C" int lp_plan_destroy(lp_plan *P)
{
    if (!P) return LP_OK;
    cudaSetDevice(P->c->device);
    cudaDeviceSynchronize();
    plan_free(P);
    return LP_OK;
}
