// Query server with continuous batching.
//
// A server thread owns a device pool of resident ciphertexts bounded by a memory budget.
// Submitted LocPIR queries (Algorithm 3) wait in FIFO order until their circuit's wires fit
// in the pool; admission copies their input ciphertexts into the pool, where they stay until
// the result is ready.  Every scheduler tick takes the next bootstrap level of EVERY admitted
// query -- queries at different depths, with different l, B_x and m -- and runs all those
// gates as one shared pre-combination / blind-rotation / key-switch pass.  A query that
// finishes its last level has its service ciphertexts copied out, its pool range freed, and
// its latency (submit -> result on the device) recorded.
//
// A gate's output depends only on its input ciphertexts and the keys, so every result is
// bit-identical to the same query evaluated alone.  lp_server_stop ends the loop after the tick
// in flight; queries not finished by then are abandoned (their results are never written).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "circuit.h"
#include "common.cuh"
#include "kernels.h"
#include "runtime.h"

namespace lp {

using Clock = std::chrono::steady_clock;

struct SrvQuery {
    uint64_t ticket = 0;
    lp_query q{};                   // for known bounds, q.boxes is unused
    bool known = false;             // server-known (plaintext) bounds
    std::vector<uint64_t> bounds;   // [n_boxes][4] when known
    Circuit C;
    std::vector<std::vector<int>> levels;
    std::vector<Sig> outs;
    int inputs[4] = {0, 0, 0, 0};   // first wire of x, y, boxes, services
    int next_level = 1;
    size_t pool_off = 0, nwires = 0;
    Clock::time_point t_submit, t_done;
    bool admitted = false, done = false;
};

struct Server {
    lp_ctx *c = nullptr;
    size_t budget_words = 0;        // pool capacity in 32-bit words
    int policy = LP_SERVER_QUEUE;
    DevBuf pool, abar, ext, jobs;
    cudaStream_t st = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<SrvQuery *> waiting;
    std::vector<SrvQuery *> active;
    std::map<uint64_t, SrvQuery *> all;
    std::vector<std::pair<size_t, size_t>> free_list;   // (offset, words), sorted by offset
    // statistics
    uint64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, ticks = 0, bootstraps = 0;
    std::vector<double> latencies_ms;
    Clock::time_point t_start;
    int error = LP_OK;
};

static size_t query_words(const lp_ctx *c, size_t nwires) { return nwires * (size_t)(c->params.n + 1); }

static bool pool_alloc(Server &S, size_t words, size_t *off)
{
    for (size_t i = 0; i < S.free_list.size(); i++) {
        auto &f = S.free_list[i];
        if (f.second >= words) {
            *off = f.first;
            f.first += words;
            f.second -= words;
            if (f.second == 0) S.free_list.erase(S.free_list.begin() + i);
            return true;
        }
    }
    return false;
}

static void pool_free(Server &S, size_t off, size_t words)
{
    S.free_list.emplace_back(off, words);
    std::sort(S.free_list.begin(), S.free_list.end());
    std::vector<std::pair<size_t, size_t>> merged;
    for (auto &f : S.free_list) {
        if (!merged.empty() && merged.back().first + merged.back().second == f.first) merged.back().second += f.second;
        else merged.push_back(f);
    }
    S.free_list.swap(merged);
}

// Release the host-side circuit of a query (a waiting query keeps only its arguments, so that
// a long queue costs little host memory; admission builds the circuit again).
static void drop_circuit(SrvQuery &Q)
{
    Q.C = Circuit();
    std::vector<std::vector<int>>().swap(Q.levels);
    std::vector<Sig>().swap(Q.outs);
}

// Build the circuit of one query (host only).
static void build_query(lp_ctx *c, SrvQuery &Q)
{
    const lp_query &q = Q.q;
    Q.inputs[0] = Q.C.inputs(q.l);
    Q.inputs[1] = Q.C.inputs(q.l);
    Q.inputs[2] = Q.C.inputs(Q.known ? 0 : 4 * q.l * q.n_boxes);
    Q.inputs[3] = Q.C.inputs(q.m * q.n_boxes);
    if (Q.known)
        Q.outs = build_locpir_known(Q.C, q.l, q.is_signed != 0, Q.inputs[0], Q.inputs[1], q.n_boxes, Q.bounds.data(),
                                    q.m, Q.inputs[3], q.comb);
    else
        Q.outs = build_locpir(Q.C, q.l, q.is_signed != 0, Q.inputs[0], Q.inputs[1], q.n_boxes, Q.inputs[2], q.m,
                              Q.inputs[3], q.comb);
    Q.levels = levels_of(Q.C);
    Q.nwires = Q.C.depth.size();
    (void)c;
}

// Wires of an encrypted-bounds query's circuit without building it: the inputs
// (2l + 4l B_x + m B_x), per box 4 comparators of l XNOR + l MUX, 3 validation ANDs and m
// service ANDs, the combine (B_x m XORs as a chain, (B_x - 1) m as a tree), and the shared
// constant wire.  build_locpir makes exactly these (checked again at admission).
static size_t encrypted_query_wires(const lp_query &q)
{
    const size_t l = (size_t)q.l, nb = (size_t)q.n_boxes, m = (size_t)q.m;
    const size_t combine = q.comb == LP_XOR_CHAIN ? nb * m : (nb - 1) * m;
    return 2 * l + 4 * l * nb + m * nb + nb * (8 * l + 3 + m) + combine + 1;
}

// Admission: reserve pool space and copy the inputs in (server stream).
static int admit(Server &S, SrvQuery &Q)
{
    lp_ctx *c = S.c;
    const size_t W = (size_t)c->params.n + 1;
    uint32_t *pool = static_cast<uint32_t *>(S.pool.ptr) + Q.pool_off;
    const lp_query &q = Q.q;
    const uint32_t *srcs[4] = {q.x, q.y, q.boxes, q.services};
    const size_t cnts[4] = {(size_t)q.l, (size_t)q.l, Q.known ? 0 : (size_t)4 * q.l * q.n_boxes,
                            (size_t)q.m * q.n_boxes};
    for (int k = 0; k < 4; k++) {
        if (!cnts[k]) continue;
        cudaError_t e = cudaMemcpyAsync(pool + (size_t)Q.inputs[k] * W, srcs[k], cnts[k] * W * 4,
                                        cudaMemcpyDeviceToDevice, S.st);
        if (e != cudaSuccess) return cuda_fail(e, "server: copy query inputs");
    }
    if (Q.C.zero_w >= 0) {
        cudaError_t e = launch_trivial(pool + (size_t)Q.C.zero_w * W, c->params.n, 0u - T_EIGHTH, S.st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "server: trivial constant");
    }
    Q.admitted = true;
    return LP_OK;
}

// One scheduler tick: the next level of every active query, as shared passes.
static int tick(Server &S)
{
    lp_ctx *c = S.c;
    const int n = c->params.n;
    const size_t W = (size_t)n + 1;
    const size_t MAXJ = 131072;
    struct Pass {
        size_t br_off, br_cnt, ks_off, ks_cnt;
    };
    std::vector<BrJob> br;
    std::vector<KsJob> ks;
    std::vector<Pass> passes;
    Pass ps{0, 0, 0, 0};
    size_t max_pass = 1;
    uint64_t tick_bootstraps = 0;
    for (SrvQuery *Q : S.active) {
        if (Q->next_level >= (int)Q->levels.size()) continue;
        const int base = (int)(Q->pool_off / W);
        for (int idx : Q->levels[Q->next_level]) {
            const Node &nd = Q->C.nodes[idx];
            const size_t need = nd.op == LP_MUX ? 2 : 1;
            if (ps.br_cnt + need > MAXJ) {
                passes.push_back(ps);
                max_pass = std::max(max_pass, ps.br_cnt);
                ps = Pass{br.size(), 0, ks.size(), 0};
            }
            append_gate_jobs(nd, base, ps.br_cnt, br, ks);
            ps.br_cnt += need;
            ps.ks_cnt += 1;
        }
    }
    if (ps.ks_cnt) {
        passes.push_back(ps);
        max_pass = std::max(max_pass, ps.br_cnt);
    }
    // Queries whose last level runs in this tick: their services are copied out after it.
    uint32_t *pool = static_cast<uint32_t *>(S.pool.ptr);
    std::vector<CopyEntry> outc;
    std::vector<SrvQuery *> finishing;
    for (SrvQuery *Q : S.active) {
        if (Q->next_level + 1 >= (int)Q->levels.size()) {
            finishing.push_back(Q);
            for (int j = 0; j < Q->q.m; j++)
                outc.push_back(CopyEntry{pool + Q->pool_off + (size_t)Q->outs[j].w * W, Q->q.out_service + (size_t)j * W,
                                         Q->outs[j].neg ? 1 : 0, 0});
        }
    }
    const size_t br_bytes = br.size() * sizeof(BrJob), ks_bytes = ks.size() * sizeof(KsJob);
    const size_t out_off = (br_bytes + ks_bytes + 255) & ~(size_t)255;
    int rc = ensure_buf(S.jobs, out_off + outc.size() * sizeof(CopyEntry) + 256, "server: job records");
    if (!rc) rc = ensure_buf(S.abar, max_pass * abar_stride(c) * sizeof(uint16_t), "server: scratch");
    if (!rc) rc = ensure_buf(S.ext, max_pass * EXT_STRIDE * sizeof(uint32_t), "server: scratch");
    if (rc) return rc;
    char *jb = static_cast<char *>(S.jobs.ptr);
    cudaError_t e = cudaSuccess;
    if (br_bytes) e = cudaMemcpyAsync(jb, br.data(), br_bytes, cudaMemcpyHostToDevice, S.st);
    if (e == cudaSuccess && ks_bytes) e = cudaMemcpyAsync(jb + br_bytes, ks.data(), ks_bytes, cudaMemcpyHostToDevice, S.st);
    if (e == cudaSuccess && !outc.empty())
        e = cudaMemcpyAsync(jb + out_off, outc.data(), outc.size() * sizeof(CopyEntry), cudaMemcpyHostToDevice, S.st);
    if (e != cudaSuccess) return cuda_fail(e, "server: upload jobs");
    const BrJob *dbr = reinterpret_cast<const BrJob *>(jb);
    const KsJob *dks = reinterpret_cast<const KsJob *>(jb + br_bytes);
    for (const Pass &p : passes) {
        e = launch_precomb_indexed(dbr + p.br_off, p.br_cnt, pool, n, static_cast<uint16_t *>(S.abar.ptr),
                                   abar_stride(c), c->num_sms, S.st);
        int lb = 0, lk = 0;
        if (e == cudaSuccess)
            e = launch_br(static_cast<const uint16_t *>(S.abar.ptr), abar_stride(c), static_cast<uint32_t *>(S.ext.ptr),
                          static_cast<const uint32_t *>(c->bsk_hat.ptr), static_cast<const uint2 *>(c->tw_lane.ptr), n,
                          (int)p.br_cnt, T_EIGHTH, static_cast<int *>(c->err.ptr), c->num_sms, S.st,
                          BR_VARIANT_AUTO, c->br_split_max, c->br_tail_split, br_pair_limit(c), br_quad_limit(c), &lb);
        if (e == cudaSuccess)
            e = launch_ks(static_cast<const uint32_t *>(S.ext.ptr), dks + p.ks_off, p.ks_cnt, 0, pool,
                          static_cast<const uint32_t *>(c->ksk.ptr), n, static_cast<int *>(c->err.ptr), c->num_sms,
                          S.st, c->ks_slice_max, &lk);
        c->launches += 1 + lb + lk;
        if (e != cudaSuccess) return cuda_fail(e, "server: pass launch");
        tick_bootstraps += p.br_cnt;
    }
    if (!outc.empty()) {
        e = launch_copy_entries(reinterpret_cast<const CopyEntry *>(jb + out_off), outc.size(), n, c->num_sms, S.st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "server: output copy");
    }
    for (SrvQuery *Q : S.active) Q->next_level++;
    e = cudaStreamSynchronize(S.st);
    if (e != cudaSuccess) return cuda_fail(e, "server: tick");
    const auto now = Clock::now();
    // Counters that lp_server_stats reads are updated under the lock.
    std::lock_guard<std::mutex> lock(S.mu);
    S.ticks++;
    S.bootstraps += tick_bootstraps;
    for (SrvQuery *Q : finishing) {
        Q->done = true;
        Q->t_done = now;
        S.completed++;
        S.latencies_ms.push_back(std::chrono::duration<double, std::milli>(now - Q->t_submit).count());
        pool_free(S, Q->pool_off, query_words(c, Q->nwires));
        drop_circuit(*Q);
    }
    S.active.erase(std::remove_if(S.active.begin(), S.active.end(), [](SrvQuery *Q) { return Q->done; }),
                   S.active.end());
    S.done_cv.notify_all();
    return LP_OK;
}

static void server_loop(Server *Sp)
{
    Server &S = *Sp;
    cudaSetDevice(S.c->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(S.mu);
            // Admit waiting queries in FIFO order while their wires fit in the pool.
            while (!S.waiting.empty()) {
                SrvQuery *Q = S.waiting.front();
                size_t off;
                if (!pool_alloc(S, query_words(S.c, Q->nwires), &off)) break;
                Q->pool_off = off;
                S.waiting.pop_front();
                const size_t reserved = Q->nwires;
                if (Q->levels.empty()) build_query(S.c, *Q);   // not built, or dropped while it waited
                int rc = Q->nwires == reserved
                             ? admit(S, *Q)
                             : fail(LP_ECUDA, "server: query circuit has %zu wires, %zu were reserved", Q->nwires,
                                    reserved);
                if (rc) {
                    S.error = rc;
                    S.stop = true;
                    break;
                }
                S.active.push_back(Q);
                S.admitted++;
            }
            if (S.stop) break;
            if (S.active.empty()) {
                S.cv.wait_for(lock, std::chrono::milliseconds(20));
                continue;
            }
        }
        int rc = tick(S);
        if (rc) {
            std::lock_guard<std::mutex> lock(S.mu);
            S.error = rc;
            S.stop = true;
            S.done_cv.notify_all();
            break;
        }
    }
}

}  // namespace lp

using namespace lp;

extern "C" int lp_server_start(lp_ctx *c, size_t mem_budget, int policy)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (c->server) return fail(LP_EBUSY, "a server is already running on this context");
    if (!c->have_bsk || !c->have_ksk) return fail(LP_ENOKEY, "load the bootstrapping and key-switching keys first");
    if (policy != LP_SERVER_QUEUE && policy != LP_SERVER_REJECT) return fail(LP_EINVAL, "unknown policy %d", policy);
    const size_t W = (size_t)c->params.n + 1;
    if (mem_budget < W * 4 * 64) return fail(LP_EINVAL, "memory budget %zu B is too small", mem_budget);
    cudaSetDevice(c->device);
    Server *S = new Server();
    S->c = c;
    S->policy = policy;
    S->budget_words = (mem_budget / 4 / W) * W;
    int rc = ensure_buf(S->pool, S->budget_words * 4, "server pool");
    if (rc) {
        delete S;
        return rc;
    }
    S->free_list.emplace_back(0, S->budget_words);
    cudaError_t e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_buf(S->pool);
        delete S;
        return cuda_fail(e, "server stream");
    }
    S->t_start = Clock::now();
    c->server = S;
    S->th = std::thread(server_loop, S);
    return LP_OK;
}

// Queue a built query (FIFO) or reject it against the budget; takes ownership of Q.
static int submit_query(lp_ctx *c, SrvQuery *Q, uint64_t *ticket)
{
    Server *S = c->server;
    // Encrypted-bounds circuits have a closed-form size, so submitting one costs O(1); the
    // size of a known-bounds circuit depends on the bound bits, so it is built here.
    if (Q->known) build_query(c, *Q);
    else Q->nwires = encrypted_query_wires(Q->q);
    const size_t need = query_words(c, Q->nwires);
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) {
        delete Q;
        return fail(S->error ? S->error : LP_EINVAL, "server stopped");
    }
    if (need > S->budget_words) {
        delete Q;
        S->rejected++;
        return fail(LP_EBUSY, "query needs %zu B of resident ciphertexts, more than the %zu B budget", need * 4,
                    S->budget_words * 4);
    }
    if (S->policy == LP_SERVER_REJECT) {
        size_t largest = 0;
        for (auto &f : S->free_list) largest = std::max(largest, f.second);
        if (!S->waiting.empty() || largest < need) {
            delete Q;
            S->rejected++;
            return fail(LP_EBUSY, "memory budget exhausted");
        }
    }
    Q->ticket = S->next_ticket++;
    Q->t_submit = Clock::now();
    // Only its size was needed here; the circuit is built again at admission.
    drop_circuit(*Q);
    S->all[Q->ticket] = Q;
    S->waiting.push_back(Q);
    S->submitted++;
    *ticket = Q->ticket;
    S->cv.notify_all();
    return LP_OK;
}

extern "C" int lp_server_submit(lp_ctx *c, const lp_query *q, uint64_t *ticket)
{
    if (!c || !q || !ticket) return fail(LP_EINVAL, "null argument");
    if (!c->server) return fail(LP_EINVAL, "no server running on this context");
    int rc = check_query(*q);
    if (rc) return rc;
    SrvQuery *Q = new SrvQuery();
    Q->q = *q;
    return submit_query(c, Q, ticket);
}

extern "C" int lp_server_submit_known(lp_ctx *c, const lp_query_known *q, uint64_t *ticket)
{
    if (!c || !q || !ticket) return fail(LP_EINVAL, "null argument");
    if (!c->server) return fail(LP_EINVAL, "no server running on this context");
    lp_query chk{q->l, q->is_signed, q->n_boxes, q->m, q->comb, q->x, q->y,
                 reinterpret_cast<const uint32_t *>(q->bounds), q->services, q->out_service};
    int rc = check_query(chk);
    if (rc) return rc;
    SrvQuery *Q = new SrvQuery();
    Q->q = chk;
    Q->q.boxes = nullptr;
    Q->known = true;
    Q->bounds.assign(q->bounds, q->bounds + 4 * (size_t)q->n_boxes);   // the caller's array may go away
    return submit_query(c, Q, ticket);
}

extern "C" int lp_server_poll(lp_ctx *c, uint64_t ticket, int *done)
{
    if (!c || !done) return fail(LP_EINVAL, "null argument");
    Server *S = c->server;
    if (!S) return fail(LP_EINVAL, "no server running on this context");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(LP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    *done = it->second->done ? 1 : 0;
    return S->error ? fail(S->error, "server failed") : LP_OK;
}

extern "C" int lp_server_wait(lp_ctx *c, uint64_t ticket, uint32_t timeout_ms)
{
    if (!c) return fail(LP_EINVAL, "null context");
    Server *S = c->server;
    if (!S) return fail(LP_EINVAL, "no server running on this context");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(LP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    SrvQuery *Q = it->second;
    const bool ok = S->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                                        [&] { return Q->done || S->error != LP_OK; });
    if (S->error) return fail(S->error, "server failed");
    if (!ok) return fail(LP_ETIMEOUT, "query %llu not finished within %u ms", (unsigned long long)ticket, timeout_ms);
    return LP_OK;
}

extern "C" int lp_server_stats(lp_ctx *c, lp_stats *out)
{
    if (!c || !out) return fail(LP_EINVAL, "null argument");
    Server *S = c->server;
    if (!S) return fail(LP_EINVAL, "no server running on this context");
    std::lock_guard<std::mutex> lock(S->mu);
    lp_stats st{};
    st.submitted = S->submitted;
    st.admitted = S->admitted;
    st.completed = S->completed;
    st.rejected = S->rejected;
    st.waiting = S->waiting.size();
    st.active = S->active.size();
    st.ticks = S->ticks;
    st.bootstraps = S->bootstraps;
    st.elapsed_s = std::chrono::duration<double>(Clock::now() - S->t_start).count();
    if (!S->latencies_ms.empty()) {
        std::vector<double> v = S->latencies_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            size_t k = (size_t)(p * (v.size() - 1) + 0.5);
            return v[std::min(k, v.size() - 1)];
        };
        st.p50_ms = pct(0.50);
        st.p99_ms = pct(0.99);
        double s = 0;
        for (double x : v) s += x;
        st.mean_ms = s / v.size();
    }
    st.queries_per_s = st.elapsed_s > 0 ? st.completed / st.elapsed_s : 0.0;
    st.bootstraps_per_s = st.elapsed_s > 0 ? st.bootstraps / st.elapsed_s : 0.0;
    *out = st;
    return LP_OK;
}

extern "C" int lp_server_stop(lp_ctx *c)
{
    if (!c) return fail(LP_EINVAL, "null context");
    Server *S = c->server;
    if (!S) return LP_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    S->th.join();
    const int err = S->error;
    cudaStreamSynchronize(S->st);
    cudaStreamDestroy(S->st);
    for (DevBuf *b : {&S->pool, &S->abar, &S->ext, &S->jobs}) free_buf(*b);
    for (auto &kv : S->all) delete kv.second;
    c->server = nullptr;
    delete S;
    return err ? fail(err, "server stopped after an error") : LP_OK;
}
