// Host side of liblocpir: context, key loading, the C-ABI entry points, NTT tables.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "runtime.h"

using namespace lp;

// ---------------------------------------------------------------------------------
// Errors.
// ---------------------------------------------------------------------------------
static thread_local std::string g_last_error;

int lp::fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int lp::cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) return fail(LP_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(LP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *lp_strerror(int code)
{
    switch (code) {
    case LP_OK: return "ok";
    case LP_EINVAL: return "invalid argument";
    case LP_ENOMEM: return "device out of memory";
    case LP_ECUDA: return "CUDA error";
    case LP_ENOKEY: return "keys not loaded";
    case LP_ETIMEOUT: return "device wait timed out";
    case LP_EBUSY: return "busy: memory budget exhausted";
    case LP_ECORRUPT: return "key checksum mismatch";
    default: return "unknown error";
    }
}

extern "C" const char *lp_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------------
// NTT tables (host arithmetic on 64-bit integers).
// ---------------------------------------------------------------------------------
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (a * b) % p; }
static uint64_t powmod(uint64_t b, uint64_t e, uint64_t p)
{
    uint64_t r = 1;
    b %= p;
    while (e) {
        if (e & 1) r = mulmod(r, b, p);
        b = mulmod(b, b, p);
        e >>= 1;
    }
    return r;
}
static uint32_t bitrev10(uint32_t x)
{
    uint32_t r = 0;
    for (int i = 0; i < 10; i++) r |= ((x >> i) & 1u) << (9 - i);
    return r;
}
static uint2 shoup_pair(uint64_t w, uint64_t p) { return make_uint2((uint32_t)w, (uint32_t)((w << 32) / p)); }

void lp::build_ntt_tables(NttTables &t)
{
    const uint64_t primes[2] = {PRIME0, PRIME1};
    for (int pi = 0; pi < 2; pi++) {
        const uint64_t p = primes[pi];
        t.prime[pi] = (uint32_t)p;
        t.red_one[pi] = (uint32_t)((1ull << 32) / p);
        // psi = g^((p-1)/2048) has order exactly 2048 iff psi^1024 = -1; take the first g
        // that gives one.
        uint64_t psi = 0;
        for (uint64_t g = 2; g < 1000; g++) {
            psi = powmod(g, (p - 1) / 2048, p);
            if (powmod(psi, 1024, p) == p - 1) break;
        }
        std::vector<uint64_t> zeta(RING_N), izeta(RING_N);
        for (uint32_t z = 0; z < (uint32_t)RING_N; z++) {
            zeta[z] = powmod(psi, bitrev10(z), p);
            izeta[z] = powmod(zeta[z], p - 2, p);
        }
        for (int z = 0; z < 32; z++) {
            t.ctw[pi][0][z] = shoup_pair(zeta[z], p);
            t.ctw[pi][1][z] = shoup_pair(izeta[z], p);
        }
        for (int s = 5; s < 10; s++) {
            const int L = 512 >> s, base = (1 << (s - 5)) - 1;
            for (int b = 0; b < 16 / L; b++)
                for (int lane = 0; lane < 32; lane++) {
                    const int z = (1 << s) + lane * (16 / L) + b;
                    t.lane[pi][0][(base + b) * 32 + lane] = shoup_pair(zeta[z], p);
                    t.lane[pi][1][(base + b) * 32 + lane] = shoup_pair(izeta[z], p);
                }
        }
        // -p^-1 mod 2^32 by Newton iteration (p odd).
        uint32_t inv = (uint32_t)p;
        for (int i = 0; i < 5; i++) inv *= 2u - (uint32_t)p * inv;
        t.pinv_neg[pi] = 0u - inv;
        // N^-1 2^32 mod p.
        const uint64_t ninv = powmod(RING_N, p - 2, p);
        t.bsk_scale[pi] = (uint32_t)mulmod(ninv, (1ull << 32) % p, p);
    }
    const uint64_t cinv = powmod(PRIME0 % PRIME1, PRIME1 - 2, PRIME1);
    t.crt = shoup_pair(cinv, PRIME1);
}

// ---------------------------------------------------------------------------------
// Context.
// ---------------------------------------------------------------------------------
int lp::ensure_buf(DevBuf &b, size_t bytes, const char *what)
{
    if (b.bytes >= bytes) return LP_OK;
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.ptr, bytes);
    if (e != cudaSuccess) return cuda_fail(e, what);
    b.bytes = bytes;
    return LP_OK;
}

void lp::free_buf(DevBuf &b)
{
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
}

extern "C" int lp_params_default(lp_params *p)
{
    if (!p) return fail(LP_EINVAL, "null params");
    p->n = 630;
    p->N = 1024;
    p->k = 1;
    p->Bgbit = 10;
    p->lg = 3;
    p->basebit = 2;
    p->t = 8;
    return LP_OK;
}

static int check_params(const lp_params *p)
{
    if (!p) return fail(LP_EINVAL, "null params");
    if (p->N != RING_N || p->k != 1 || p->Bgbit != BGBIT || p->lg != LG || p->basebit != KS_BASEBIT ||
        p->t != KS_T)
        return fail(LP_EINVAL, "unsupported parameters (this build: N=1024 k=1 Bgbit=10 lg=3 basebit=2 t=8)");
    if (p->n < 1 || p->n > MAX_LWE_N) return fail(LP_EINVAL, "LWE dimension n=%d outside [1, %d]", p->n, MAX_LWE_N);
    return LP_OK;
}

extern "C" int lp_create(const lp_params *p, int device, lp_ctx **out)
{
    if (!out) return fail(LP_EINVAL, "null output pointer");
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(LP_EINVAL, "device %d not present (%d devices)", device, ndev);
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    if ((size_t)prop.sharedMemPerBlockOptin < br_smem_bytes())
        return fail(LP_EINVAL, "device offers %zu B shared memory per block, blind rotation needs %zu",
                    (size_t)prop.sharedMemPerBlockOptin, br_smem_bytes());
    lp_ctx *c = new lp_ctx();
    c->params = *p;
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    c->br_pair_clusters = br_pair_clusters(c->num_sms);
    c->br_quad_clusters = br_quad_clusters(c->num_sms);
    build_ntt_tables(c->tables);
    if ((e = upload_constants(c->tables)) != cudaSuccess) {
        delete c;
        return cuda_fail(e, "upload constants");
    }
    rc = ensure_buf(c->tw_lane, sizeof(c->tables.lane), "twiddle tables");
    if (!rc) rc = ensure_buf(c->err, sizeof(int), "error word");
    if (rc) {
        lp_destroy(c);
        return rc;
    }
    cudaMemcpy(c->tw_lane.ptr, c->tables.lane, sizeof(c->tables.lane), cudaMemcpyHostToDevice);
    cudaMemset(c->err.ptr, 0, sizeof(int));
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        lp_destroy(c);
        return cuda_fail(e, "context init");
    }
    *out = c;
    return LP_OK;
}

extern "C" int lp_destroy(lp_ctx *c)
{
    if (!c) return LP_OK;
    if (c->server) lp_server_stop(c);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto &t : c->timers) {
        for (auto &ev : t.second.pending) {
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
    }
    tc_release(c);
    for (cudaStream_t st : {c->st_h2d, c->st_run, c->st_d2h})
        if (st) cudaStreamDestroy(st);
    for (int k = 0; k < lp_ctx::HOST_CHUNKS; k++) {
        if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
        if (c->ev_run[k]) cudaEventDestroy(c->ev_run[k]);
    }
    for (DevBuf *b : {&c->tw_lane, &c->err, &c->bsk_hat, &c->bsk_coef, &c->ksk, &c->abar, &c->ext, &c->pool,
                      &c->jobs, &c->tmp_in, &c->tmp_out})
        free_buf(*b);
    delete c;
    return LP_OK;
}

int lp::ctx_check_err(lp_ctx *c)
{
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, c->err.ptr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read device error word");
    if (h) {
        cudaMemset(c->err.ptr, 0, sizeof(int));
        if (h & DEV_ERR_TIMEOUT) return fail(LP_ETIMEOUT, "a device-side wait timed out");
        return fail(LP_ECUDA, "device error word 0x%x", h);
    }
    return LP_OK;
}

extern "C" int lp_sync(lp_ctx *c)
{
    if (!c) return fail(LP_EINVAL, "null context");
    cudaSetDevice(c->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    return ctx_check_err(c);
}

// ---------------------------------------------------------------------------------
// Timing of library kernels with CUDA events on the launching stream.
// ---------------------------------------------------------------------------------
void lp::timer_begin(lp_ctx *c, const char *name, cudaStream_t st, cudaEvent_t *ev0)
{
    *ev0 = nullptr;
    if (!c->timing) return;
    cudaEventCreate(ev0);
    cudaEventRecord(*ev0, st);
    (void)name;
}

void lp::timer_end(lp_ctx *c, const char *name, cudaStream_t st, cudaEvent_t ev0)
{
    if (!c->timing || !ev0) return;
    cudaEvent_t ev1;
    cudaEventCreate(&ev1);
    cudaEventRecord(ev1, st);
    c->timers[name].pending.emplace_back(ev0, ev1);
}

extern "C" int lp_set_timing(lp_ctx *c, int enable)
{
    if (!c) return fail(LP_EINVAL, "null context");
    c->timing = enable != 0;
    return LP_OK;
}

extern "C" int lp_kernel_time(lp_ctx *c, const char *kernel, double *ms_total, uint64_t *launches)
{
    if (!c || !kernel || !ms_total || !launches) return fail(LP_EINVAL, "null argument");
    cudaSetDevice(c->device);
    auto it = c->timers.find(kernel);
    *ms_total = 0.0;
    *launches = 0;
    if (it == c->timers.end()) return LP_OK;
    KernelTimer &t = it->second;
    for (auto &ev : t.pending) {
        cudaError_t e = cudaEventSynchronize(ev.second);
        if (e != cudaSuccess) return cuda_fail(e, "event synchronize");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev.first, ev.second);
        t.ms += ms;
        t.count += 1;
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    t.pending.clear();
    *ms_total = t.ms;
    *launches = t.count;
    return LP_OK;
}

extern "C" int lp_reset_timing(lp_ctx *c)
{
    if (!c) return fail(LP_EINVAL, "null context");
    double ms;
    uint64_t n;
    for (auto &kv : c->timers) lp_kernel_time(c, kv.first.c_str(), &ms, &n);
    c->timers.clear();
    return LP_OK;
}

extern "C" uint64_t lp_launch_count(const lp_ctx *c) { return c ? c->launches.load() : 0; }

// ---------------------------------------------------------------------------------
// Keys.
// ---------------------------------------------------------------------------------
static size_t bsk_words(const lp_params &p) { return (size_t)p.n * ROWS * 2 * RING_N; }
static size_t ksk_words(const lp_params &p) { return (size_t)RING_N * KS_T * KS_BASE * (p.n + 1); }

static int load_bsk_common(lp_ctx *c, const uint32_t *src, bool on_device, size_t words, cudaStream_t st)
{
    if (!c || !src) return fail(LP_EINVAL, "null argument");
    if (words != bsk_words(c->params))
        return fail(LP_EINVAL, "bootstrapping key has %zu words, expected %zu", words, bsk_words(c->params));
    cudaSetDevice(c->device);
    int rc = ensure_buf(c->bsk_hat, words * 2 * sizeof(uint32_t), "bootstrapping key");
    // The coefficient-domain key stays resident (31 MB) for the Toeplitz engines.
    if (!rc) rc = ensure_buf(c->bsk_coef, words * sizeof(uint32_t), "bootstrapping key (coefficients)");
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(c->bsk_coef.ptr, src, words * 4,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy bootstrapping key");
    e = launch_bsk_to_ntt(static_cast<const uint32_t *>(c->bsk_coef.ptr), static_cast<uint32_t *>(c->bsk_hat.ptr),
                          c->params.n, static_cast<const uint2 *>(c->tw_lane.ptr), c->tables.bsk_scale[0],
                          c->tables.bsk_scale[1], c->num_sms, st);
    c->launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "convert bootstrapping key");
    c->have_bsk = true;
    return LP_OK;
}

extern "C" int lp_load_bsk(lp_ctx *c, const uint32_t *bsk, size_t words)
{
    return load_bsk_common(c, bsk, false, words, 0);
}

extern "C" int lp_load_bsk_device(lp_ctx *c, const uint32_t *bsk, size_t words, void *stream)
{
    return load_bsk_common(c, bsk, true, words, static_cast<cudaStream_t>(stream));
}

static int load_ksk_common(lp_ctx *c, const uint32_t *src, bool on_device, size_t words, cudaStream_t st)
{
    if (!c || !src) return fail(LP_EINVAL, "null argument");
    if (words != ksk_words(c->params))
        return fail(LP_EINVAL, "key-switching key has %zu words, expected %zu", words, ksk_words(c->params));
    cudaSetDevice(c->device);
    // The context keeps only the digit-pair table the key switch reads (see keyswitch.cu).
    int rc = ensure_buf(c->ksk, ks_table_words(c->params.n) * sizeof(uint32_t), "key-switching table");
    if (rc) return rc;
    DevBuf staging;
    const uint32_t *dsrc = src;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        rc = ensure_buf(staging, words * sizeof(uint32_t), "key-switching key staging");
        if (rc) return rc;
        e = cudaMemcpyAsync(staging.ptr, src, words * 4, cudaMemcpyHostToDevice, st);
        dsrc = static_cast<const uint32_t *>(staging.ptr);
    }
    if (e == cudaSuccess) {
        e = launch_ks_table(dsrc, static_cast<uint32_t *>(c->ksk.ptr), c->params.n, c->num_sms, st);
        c->launches++;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    free_buf(staging);
    if (e != cudaSuccess) return cuda_fail(e, "build key-switching table");
    c->have_ksk = true;
    if (c->ks_engine == LP_KS_TENSOR_INT8) {
        if ((rc = ks_tensor_prepare(c, st))) return rc;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "build one-hot key");
    }
    return LP_OK;
}

extern "C" int lp_load_ksk(lp_ctx *c, const uint32_t *ksk, size_t words)
{
    return load_ksk_common(c, ksk, false, words, 0);
}

extern "C" int lp_load_ksk_device(lp_ctx *c, const uint32_t *ksk, size_t words, void *stream)
{
    return load_ksk_common(c, ksk, true, words, static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------------
// Bootstrap pipeline pieces shared by the batch and circuit entry points.
// ---------------------------------------------------------------------------------
int lp::abar_stride(const lp_ctx *c) { return ((c->params.n + 1) + 7) & ~7; }

int lp::ensure_scratch(lp_ctx *c, size_t br_jobs)
{
    int rc = ensure_buf(c->abar, br_jobs * abar_stride(c) * sizeof(uint16_t), "mod-switched scratch");
    if (!rc) rc = ensure_buf(c->ext, br_jobs * EXT_STRIDE * sizeof(uint32_t), "extracted-sample scratch");
    return rc;
}

int lp::br_variant(const lp_ctx *c)
{
    switch (c->br_engine) {
    case LP_BR_NTT_BATCHED: return BR_VARIANT_BATCHED;
    case LP_BR_NTT_SPLIT: return BR_VARIANT_SPLIT;
    case LP_BR_NTT_PAIR: return BR_VARIANT_PAIR;
    case LP_BR_NTT_QUAD: return BR_VARIANT_QUAD;
    default: return BR_VARIANT_AUTO;
    }
}

int lp::run_br(lp_ctx *c, size_t jobs, uint32_t mu, cudaStream_t st)
{
    cudaEvent_t ev0;
    timer_begin(c, "br", st, &ev0);
    if (c->br_engine == LP_BR_TENSOR_BF16 || c->br_engine == LP_BR_TENSOR_INT8) {
        const int rc = run_br_tensor(c, jobs, mu, st);
        timer_end(c, "br", st, ev0);
        return rc;
    }
    const int variant = br_variant(c);
    int launched = 0;
    cudaError_t e = launch_br(static_cast<const uint16_t *>(c->abar.ptr), abar_stride(c),
                              static_cast<uint32_t *>(c->ext.ptr), static_cast<const uint32_t *>(c->bsk_hat.ptr),
                              static_cast<const uint2 *>(c->tw_lane.ptr), c->params.n, (int)jobs, mu,
                              static_cast<int *>(c->err.ptr), c->num_sms, st, variant, c->br_split_max,
                              c->br_tail_split, br_pair_limit(c), br_quad_limit(c), &launched);
    timer_end(c, "br", st, ev0);
    c->launches += launched;
    if (e != cudaSuccess) return cuda_fail(e, "blind rotation launch");
    return LP_OK;
}

int lp::run_ks(lp_ctx *c, const KsJob *jobs, size_t njobs, int dense_mux, uint32_t *out, cudaStream_t st)
{
    cudaEvent_t ev0;
    timer_begin(c, "ks", st, &ev0);
    if (c->ks_engine != LP_KS_TABLE) {
        const int rc = run_ks_tensor(c, jobs, njobs, dense_mux, out, st);
        timer_end(c, "ks", st, ev0);
        return rc;
    }
    int launched = 0;
    cudaError_t e = launch_ks(static_cast<const uint32_t *>(c->ext.ptr), jobs, njobs, dense_mux, out,
                              static_cast<const uint32_t *>(c->ksk.ptr), c->params.n,
                              static_cast<int *>(c->err.ptr), c->num_sms, st, c->ks_slice_max, &launched);
    timer_end(c, "ks", st, ev0);
    c->launches += launched;
    if (e != cudaSuccess) return cuda_fail(e, "key switch launch");
    return LP_OK;
}

extern "C" int lp_set_engines(lp_ctx *c, int br_engine, int ks_engine)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (br_engine < LP_BR_NTT || br_engine > LP_BR_NTT_QUAD)
        return fail(LP_EINVAL, "unknown blind-rotation engine %d", br_engine);
    if (ks_engine < LP_KS_TABLE || ks_engine > LP_KS_TENSOR_INT8)
        return fail(LP_EINVAL, "unknown key-switch engine %d", ks_engine);
    cudaSetDevice(c->device);
    if (ks_engine == LP_KS_TENSOR_INT8 && c->have_ksk && !c->ks_A.ptr) {
        int rc = ks_tensor_prepare(c, 0);
        if (rc) return rc;
        const cudaError_t e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) return cuda_fail(e, "build one-hot key");
    }
    c->br_engine = br_engine;
    c->ks_engine = ks_engine;
    return LP_OK;
}

// Median of three timed launches (after one untimed) of fn on the default stream, in ms.
template <class F>
static cudaError_t time_median(F fn, float *ms)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float t[3] = {};
    cudaError_t e = fn();
    for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
        cudaEventRecord(e0, 0);
        e = fn();
        cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) cudaEventElapsedTime(&t[rep], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::sort(t, t + 3);
    *ms = t[1];
    return e;
}

// Measure the launch policy on this device: the blind rotation's split/batched crossing (which
// also decides whether a wider level's partial last wave runs split) and the key switch's
// slicing crossing.  Synthetic inputs; every choice gives the same bits.
static int measure_tuning(lp_ctx *c, lp_tuning *t)
{
    const int S = c->num_sms, maxw = 4 * S, stride = abar_stride(c), n = c->params.n;
    int rc = ensure_scratch(c, (size_t)maxw);
    if (rc) return rc;
    // Mod-switched inputs: every coefficient in [0, 2N) from a fixed LCG, so that no CMux step is
    // skipped.
    std::vector<uint16_t> h((size_t)maxw * stride);
    uint32_t x = 12345u;
    for (uint16_t &v : h) {
        x = x * 1664525u + 1013904223u;
        v = (uint16_t)(x >> 21);
    }
    cudaError_t e = cudaMemcpy(c->abar.ptr, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "autotune inputs");
    float tb[5][2] = {};
    for (int k = 1; k <= 4 && e == cudaSuccess; k++)
        for (int v = 0; v < 2 && e == cudaSuccess; v++) {
            const int variant = v ? BR_VARIANT_SPLIT : BR_VARIANT_BATCHED;
            e = time_median(
                [&] {
                    c->launches++;
                    return launch_br(static_cast<const uint16_t *>(c->abar.ptr), stride,
                                     static_cast<uint32_t *>(c->ext.ptr), static_cast<const uint32_t *>(c->bsk_hat.ptr),
                                     static_cast<const uint2 *>(c->tw_lane.ptr), n, k * S, T_EIGHTH,
                                     static_cast<int *>(c->err.ptr), S, 0, variant);
                },
                &tb[k][v]);
        }
    if (e != cudaSuccess) return cuda_fail(e, "autotune blind rotation");
    // Levels below one wave always favour the split kernel; widen while it stays faster.  The
    // same crossing bounds the partial last wave that a wider level may run split.
    int best = S;
    for (int k = 2; k <= 4 && tb[k][1] < tb[k][0]; k++) best = k * S;
    t->split_max = best;
    t->tail_split = tb[1][1] < tb[1][0] ? 1 : 0;
    // Paired against split at one ciphertext per resident cluster (half the SMs at most).
    t->pair_max = -1;
    const int pc = c->br_pair_clusters;
    if (pc > 0) {
        float tp[2] = {};
        for (int v = 0; v < 2 && e == cudaSuccess; v++) {
            const int variant = v ? BR_VARIANT_PAIR : BR_VARIANT_SPLIT;
            e = time_median(
                [&] {
                    c->launches++;
                    return launch_br(static_cast<const uint16_t *>(c->abar.ptr), stride,
                                     static_cast<uint32_t *>(c->ext.ptr), static_cast<const uint32_t *>(c->bsk_hat.ptr),
                                     static_cast<const uint2 *>(c->tw_lane.ptr), n, pc, T_EIGHTH,
                                     static_cast<int *>(c->err.ptr), S, 0, variant);
                },
                &tp[v]);
        }
        if (e != cudaSuccess) return cuda_fail(e, "autotune paired blind rotation");
        if (tp[1] < tp[0]) t->pair_max = pc;
    }
    // Quad against the faster of paired and split at one ciphertext per resident cluster of four.
    t->quad_max = -1;
    const int qc = c->br_quad_clusters;
    if (qc > 0) {
        float tq[2] = {};
        for (int v = 0; v < 2 && e == cudaSuccess; v++) {
            const int variant = v ? BR_VARIANT_QUAD : (t->pair_max > 0 ? BR_VARIANT_PAIR : BR_VARIANT_SPLIT);
            e = time_median(
                [&] {
                    c->launches++;
                    return launch_br(static_cast<const uint16_t *>(c->abar.ptr), stride,
                                     static_cast<uint32_t *>(c->ext.ptr), static_cast<const uint32_t *>(c->bsk_hat.ptr),
                                     static_cast<const uint2 *>(c->tw_lane.ptr), n, qc, T_EIGHTH,
                                     static_cast<int *>(c->err.ptr), S, 0, variant);
                },
                &tq[v]);
        }
        if (e != cudaSuccess) return cuda_fail(e, "autotune quad blind rotation");
        if (tq[1] < tq[0]) t->quad_max = qc;
    }
    // Key switch: sliced against whole-table CTAs at 1/4 .. 1 batch per SM (64 outputs each),
    // on the extracted samples the blind rotations just wrote.
    DevBuf out;
    const int kmax = 4;
    rc = ensure_buf(out, (size_t)S * 64 * (n + 1) * sizeof(uint32_t), "autotune key-switch output");
    if (rc) return rc;
    if ((size_t)S * 64 > (size_t)maxw) rc = ensure_scratch(c, (size_t)S * 64);
    if (rc) {
        free_buf(out);
        return rc;
    }
    int slice_max = 0;
    for (int k = 1; k <= kmax && e == cudaSuccess; k++) {
        const size_t nb = (size_t)S * k / kmax, jobs = nb * 64;
        float ts[2] = {};
        for (int v = 0; v < 2 && e == cudaSuccess; v++)
            e = time_median(
                [&] {
                    c->launches++;
                    return launch_ks_forced(static_cast<const uint32_t *>(c->ext.ptr), jobs,
                                            static_cast<uint32_t *>(out.ptr), static_cast<const uint32_t *>(c->ksk.ptr),
                                            n, static_cast<int *>(c->err.ptr), S, 0, v);
                },
                &ts[v]);
        if (e == cudaSuccess && ts[1] < ts[0] && (size_t)slice_max == nb - (size_t)S / kmax) slice_max = (int)nb;
    }
    free_buf(out);
    if (e != cudaSuccess) return cuda_fail(e, "autotune key switch");
    t->ks_slice_max = slice_max > 0 ? slice_max : -1;   // -1: never slice
    return ctx_check_err(c);
}

static void apply_tuning(lp_ctx *c, const lp_tuning &t)
{
    c->br_split_max = t.split_max;
    c->br_tail_split = t.tail_split;
    c->ks_slice_max = t.ks_slice_max;
    c->br_pair_max = t.pair_max;
    c->br_quad_max = t.quad_max;
}

extern "C" int lp_autotune(lp_ctx *c, int *split_max_out)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (!c->have_bsk || !c->have_ksk) return fail(LP_ENOKEY, "load the bootstrapping and key-switching keys first");
    cudaSetDevice(c->device);
    lp_tuning t{};
    int rc = measure_tuning(c, &t);
    if (rc) return rc;
    apply_tuning(c, t);
    if (split_max_out) *split_max_out = t.split_max;
    return LP_OK;
}

// The cache key: what the measured choices depend on.
static std::string tuning_key(const lp_ctx *c)
{
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, c->device);
    char buf[320];
    snprintf(buf, sizeof buf, "%s|sms=%d|n=%d|schema=%d", prop.name, c->num_sms, c->params.n, LP_TUNING_SCHEMA);
    return buf;
}

// A flat JSON object of one string field and integer fields, written and read by this library.
static bool read_tuning(const char *path, const std::string &key, lp_tuning *t)
{
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    std::string txt;
    char chunk[4096];
    size_t got;
    while ((got = fread(chunk, 1, sizeof chunk, f)) > 0) txt.append(chunk, got);
    fclose(f);
    auto field = [&](const char *name, std::string *str, long *num) -> bool {
        const std::string pat = std::string("\"") + name + "\":";
        size_t p = txt.find(pat);
        if (p == std::string::npos) return false;
        p += pat.size();
        while (p < txt.size() && txt[p] == ' ') p++;
        if (str) {
            if (p >= txt.size() || txt[p] != '"') return false;
            const size_t q = txt.find('"', p + 1);
            if (q == std::string::npos) return false;
            *str = txt.substr(p + 1, q - p - 1);
            return true;
        }
        char *end = nullptr;
        *num = strtol(txt.c_str() + p, &end, 10);
        return end != txt.c_str() + p;
    };
    std::string k;
    long sm = 0, ts = 0, ks = 0, pm = 0, qm = 0;
    if (!field("key", &k, nullptr) || k != key) return false;
    if (!field("split_max", nullptr, &sm) || !field("tail_split", nullptr, &ts) || !field("ks_slice_max", nullptr, &ks) ||
        !field("pair_max", nullptr, &pm) || !field("quad_max", nullptr, &qm))
        return false;
    if (sm < 1 || sm > 1 << 20 || (ts != 0 && ts != 1) || ks < -1 || ks > 1 << 20 || pm < -1 || pm > 1 << 20 ||
        qm < -1 || qm > 1 << 20)
        return false;
    t->split_max = (int)sm;
    t->tail_split = (int)ts;
    t->ks_slice_max = (int)ks;
    t->pair_max = (int)pm;
    t->quad_max = (int)qm;
    return true;
}

static int write_tuning(const char *path, const std::string &key, const lp_tuning &t)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(LP_EINVAL, "cannot write the tuning cache %s", tmp.c_str());
    std::string k;
    for (char ch : key) k += (ch == '"' || ch == '\\') ? '_' : ch;
    fprintf(f,
            "{\"key\": \"%s\", \"split_max\": %d, \"tail_split\": %d, \"ks_slice_max\": %d, \"pair_max\": %d, "
            "\"quad_max\": %d}\n",
            k.c_str(), t.split_max, t.tail_split, t.ks_slice_max, t.pair_max, t.quad_max);
    const bool ok = fclose(f) == 0;
    if (!ok || rename(tmp.c_str(), path) != 0) return fail(LP_EINVAL, "cannot write the tuning cache %s", path);
    return LP_OK;
}

extern "C" int lp_autotune_cached(lp_ctx *c, const char *cache_path, int force, lp_tuning *out)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (!c->have_bsk || !c->have_ksk) return fail(LP_ENOKEY, "load the bootstrapping and key-switching keys first");
    cudaSetDevice(c->device);
    std::string key = tuning_key(c);
    for (char &ch : key)
        if (ch == '"' || ch == '\\') ch = '_';
    lp_tuning t{};
    if (cache_path && !force && read_tuning(cache_path, key, &t)) {
        t.from_cache = 1;
    } else {
        int rc = measure_tuning(c, &t);
        if (rc) return rc;
        t.from_cache = 0;
        if (cache_path && (rc = write_tuning(cache_path, key, t))) return rc;
    }
    apply_tuning(c, t);
    if (out) *out = t;
    return LP_OK;
}

extern "C" int lp_set_executor(lp_ctx *c, int executor)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (executor != LP_EXEC_LEVELS && executor != LP_EXEC_PERSISTENT)
        return fail(LP_EINVAL, "unknown executor %d", executor);
    if (executor == LP_EXEC_PERSISTENT) {
        cudaSetDevice(c->device);
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
        if (!coop) return fail(LP_EINVAL, "device %d does not support cooperative launches", c->device);
    }
    c->executor = executor;
    return LP_OK;
}

extern "C" int lp_set_tuning(lp_ctx *c, const lp_tuning *t)
{
    if (!c || !t) return fail(LP_EINVAL, "null argument");
    if (t->split_max < 0 || (t->tail_split != 0 && t->tail_split != 1) || t->ks_slice_max < -1 || t->pair_max < -1 ||
        t->quad_max < -1)
        return fail(LP_EINVAL, "invalid tuning (split_max %d, tail_split %d, ks_slice_max %d, pair_max %d, quad_max %d)",
                    t->split_max, t->tail_split, t->ks_slice_max, t->pair_max, t->quad_max);
    apply_tuning(c, *t);
    return LP_OK;
}

extern "C" int lp_get_tuning(const lp_ctx *c, lp_tuning *t)
{
    if (!c || !t) return fail(LP_EINVAL, "null argument");
    *t = lp_tuning{};
    t->split_max = c->br_split_max;
    t->tail_split = c->br_tail_split;
    t->ks_slice_max = c->ks_slice_max;
    t->pair_max = c->br_pair_max;
    t->quad_max = c->br_quad_max;
    return LP_OK;
}

// Largest number of blind-rotation jobs one pass handles (bounds the scratch to ~0.6 GB).
static const size_t MAX_PASS_JOBS = 131072;

extern "C" int lp_gate_batch(lp_ctx *c, int op, const uint32_t *a, const uint32_t *b, const uint32_t *cc,
                             uint32_t *out, size_t count, void *stream)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (op < LP_NAND || op > LP_MUX) return fail(LP_EINVAL, "unknown gate %d", op);
    if (count == 0) return LP_OK;
    if (!a || !out || (op != LP_NOT && !b) || (op == LP_MUX && !cc)) return fail(LP_EINVAL, "null ciphertext pointer");
    cudaSetDevice(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = c->params.n;
    const size_t W = (size_t)n + 1;
    if (op == LP_NOT) {
        cudaError_t e = launch_negate(a, out, count * W, c->num_sms, st);
        c->launches++;
        return e == cudaSuccess ? LP_OK : cuda_fail(e, "negate launch");
    }
    if (!c->have_bsk || !c->have_ksk) return fail(LP_ENOKEY, "load the bootstrapping and key-switching keys first");
    const size_t halves = op == LP_MUX ? 2 : 1;
    const size_t per_pass = MAX_PASS_JOBS / halves;
    int rc = ensure_scratch(c, (count < per_pass ? count : per_pass) * halves);
    if (rc) return rc;
    for (size_t off = 0; off < count; off += per_pass) {
        const size_t cnt = count - off < per_pass ? count - off : per_pass;
        cudaError_t e = launch_precomb_dense(op, a + off * W, b + off * W, op == LP_MUX ? cc + off * W : nullptr, n,
                                             cnt, static_cast<uint16_t *>(c->abar.ptr), abar_stride(c),
                                             c->num_sms, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "pre-combination launch");
        if ((rc = run_br(c, cnt * halves, T_EIGHTH, st))) return rc;
        if ((rc = run_ks(c, nullptr, cnt, op == LP_MUX, out + off * W, st))) return rc;
    }
    return LP_OK;
}

extern "C" int lp_gate_batch_host(lp_ctx *c, int op, const uint32_t *a, const uint32_t *b, const uint32_t *cc,
                                  uint32_t *out, size_t count)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (count == 0) return LP_OK;
    if (op < LP_NAND || op > LP_MUX) return fail(LP_EINVAL, "unknown gate %d", op);
    if (!a || !out || (op != LP_NOT && !b) || (op == LP_MUX && !cc)) return fail(LP_EINVAL, "null ciphertext pointer");
    cudaSetDevice(c->device);
    const size_t W = (size_t)c->params.n + 1, bytes = count * W * 4;
    const int nin = op == LP_NOT ? 1 : (op == LP_MUX ? 3 : 2);
    int rc = ensure_buf(c->tmp_in, bytes * nin, "host-batch input staging");
    if (!rc) rc = ensure_buf(c->tmp_out, bytes, "host-batch output staging");
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (!c->st_h2d) {
        e = cudaStreamCreateWithFlags(&c->st_h2d, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->st_run, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->st_d2h, cudaStreamNonBlocking);
        for (int k = 0; k < lp_ctx::HOST_CHUNKS && e == cudaSuccess; k++) {
            e = cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_run[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "host-batch streams");
    }
    // Pipeline: the batch in up to HOST_CHUNKS chunks (each still many waves of the GPU); all
    // uploads queue on one copy stream, each chunk's gates wait for its upload, and each
    // download waits for its gates on the other copy direction, so transfers overlap compute.
    const size_t nch = count >= (size_t)lp_ctx::HOST_CHUNKS * 8192 ? lp_ctx::HOST_CHUNKS : 1;
    const size_t per = (count + nch - 1) / nch;
    uint32_t *din = static_cast<uint32_t *>(c->tmp_in.ptr);
    uint32_t *dout = static_cast<uint32_t *>(c->tmp_out.ptr);
    const uint32_t *srcs[3] = {a, b, cc};
    for (size_t k = 0; k < nch && e == cudaSuccess; k++) {
        const size_t off = k * per, cnt = std::min(per, count - off);
        for (int i = 0; i < nin && e == cudaSuccess; i++)
            e = cudaMemcpyAsync(din + i * count * W + off * W, srcs[i] + off * W, cnt * W * 4, cudaMemcpyHostToDevice,
                                c->st_h2d);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_in[k], c->st_h2d);
    }
    if (e != cudaSuccess) return cuda_fail(e, "copy inputs");
    for (size_t k = 0; k < nch; k++) {
        const size_t off = k * per, cnt = std::min(per, count - off);
        e = cudaStreamWaitEvent(c->st_run, c->ev_in[k], 0);
        if (e != cudaSuccess) return cuda_fail(e, "host-batch ordering");
        rc = lp_gate_batch(c, op, din + off * W, nin > 1 ? din + count * W + off * W : nullptr,
                           nin > 2 ? din + 2 * count * W + off * W : nullptr, dout + off * W, cnt, c->st_run);
        if (rc) return rc;
        e = cudaEventRecord(c->ev_run[k], c->st_run);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->st_d2h, c->ev_run[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out + off * W, dout + off * W, cnt * W * 4, cudaMemcpyDeviceToHost, c->st_d2h);
        if (e != cudaSuccess) return cuda_fail(e, "copy outputs");
    }
    e = cudaStreamSynchronize(c->st_d2h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st_run);
    if (e != cudaSuccess) return cuda_fail(e, "host batch");
    return ctx_check_err(c);
}

extern "C" int lp_bootstrap_extract(lp_ctx *c, const uint32_t *lwe, uint32_t mu, uint32_t *ext, size_t count,
                                    void *stream)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (count == 0) return LP_OK;
    if (!lwe || !ext) return fail(LP_EINVAL, "null pointer");
    if (!c->have_bsk) return fail(LP_ENOKEY, "load the bootstrapping key first");
    cudaSetDevice(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = c->params.n;
    int rc = ensure_scratch(c, count < MAX_PASS_JOBS ? count : MAX_PASS_JOBS);
    if (rc) return rc;
    for (size_t off = 0; off < count; off += MAX_PASS_JOBS) {
        const size_t cnt = count - off < MAX_PASS_JOBS ? count - off : MAX_PASS_JOBS;
        cudaError_t e = launch_modswitch(lwe + off * (n + 1), n, cnt, static_cast<uint16_t *>(c->abar.ptr),
                                         abar_stride(c), c->num_sms, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "modulus switch launch");
        if ((rc = run_br(c, cnt, mu, st))) return rc;
        e = cudaMemcpy2DAsync(ext + off * (RING_N + 1), (RING_N + 1) * 4, c->ext.ptr, EXT_STRIDE * 4,
                              (RING_N + 1) * 4, cnt, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy extracted samples");
    }
    return LP_OK;
}

extern "C" int lp_key_switch(lp_ctx *c, const uint32_t *ext, uint32_t *out, size_t count, void *stream)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (count == 0) return LP_OK;
    if (!ext || !out) return fail(LP_EINVAL, "null pointer");
    if (!c->have_ksk) return fail(LP_ENOKEY, "load the key-switching key first");
    cudaSetDevice(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = c->params.n;
    int rc = ensure_scratch(c, count < MAX_PASS_JOBS ? count : MAX_PASS_JOBS);
    if (rc) return rc;
    for (size_t off = 0; off < count; off += MAX_PASS_JOBS) {
        const size_t cnt = count - off < MAX_PASS_JOBS ? count - off : MAX_PASS_JOBS;
        cudaError_t e = cudaMemcpy2DAsync(c->ext.ptr, EXT_STRIDE * 4, ext + off * (RING_N + 1), (RING_N + 1) * 4,
                                          (RING_N + 1) * 4, cnt, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "stage extracted samples");
        if ((rc = run_ks(c, nullptr, cnt, 0, out + off * (n + 1), st))) return rc;
    }
    return LP_OK;
}

// ---------------------------------------------------------------------------------
// Client side.
// ---------------------------------------------------------------------------------
static int device_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

extern "C" int lp_client_lwe_encrypt(int n, const uint8_t *s, const uint32_t *mask, const uint32_t *noise,
                                     const uint32_t *mu, uint32_t *out, size_t count, void *stream)
{
    if (n < 1 || n > MAX_LWE_N) return fail(LP_EINVAL, "bad n=%d", n);
    if (count == 0) return LP_OK;
    if (!s || !mask || !noise || !mu || !out) return fail(LP_EINVAL, "null pointer");
    cudaError_t e = launch_lwe_encrypt(n, s, mask, noise, mu, out, count, device_sms(), static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LP_OK : cuda_fail(e, "encrypt launch");
}

extern "C" int lp_client_lwe_phase(int n, const uint8_t *s, const uint32_t *ct, uint32_t *phase, size_t count,
                                   void *stream)
{
    if (n < 1 || n > MAX_LWE_N) return fail(LP_EINVAL, "bad n=%d", n);
    if (count == 0) return LP_OK;
    if (!s || !ct || !phase) return fail(LP_EINVAL, "null pointer");
    cudaError_t e = launch_lwe_phase(n, s, ct, phase, count, device_sms(), static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LP_OK : cuda_fail(e, "phase launch");
}

extern "C" int lp_client_keygen_bsk(const lp_params *p, const uint8_t *s, const uint8_t *S, const uint32_t *mask,
                                    const uint32_t *noise, uint32_t *bsk, void *stream)
{
    int rc = check_params(p);
    if (rc) return rc;
    if (!s || !S || !mask || !noise || !bsk) return fail(LP_EINVAL, "null pointer");
    cudaError_t e = launch_keygen_bsk(p->n, s, S, mask, noise, bsk, device_sms(), static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LP_OK : cuda_fail(e, "keygen_bsk launch");
}

extern "C" int lp_client_keygen_ksk(const lp_params *p, const uint8_t *s, const uint8_t *S, const uint32_t *mask,
                                    const uint32_t *noise, uint32_t *ksk, void *stream)
{
    int rc = check_params(p);
    if (rc) return rc;
    if (!s || !S || !mask || !noise || !ksk) return fail(LP_EINVAL, "null pointer");
    cudaError_t e = launch_keygen_ksk(p->n, s, S, mask, noise, ksk, device_sms(), static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LP_OK : cuda_fail(e, "keygen_ksk launch");
}

extern "C" int lp_preprocess_services(int n, const uint32_t *zero, const uint8_t *bits, uint32_t *out, size_t count,
                                      void *stream)
{
    if (n < 1 || n > MAX_LWE_N) return fail(LP_EINVAL, "bad n=%d", n);
    if (count == 0) return LP_OK;
    if (!zero || !bits || !out) return fail(LP_EINVAL, "null pointer");
    cudaError_t e = launch_preprocess(n, zero, bits, out, count, device_sms(), static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LP_OK : cuda_fail(e, "preprocess launch");
}

extern "C" int lp_selftest_exec_timeout(lp_ctx *c, void *stream)
{
    if (!c) return fail(LP_EINVAL, "null context");
    cudaSetDevice(c->device);
    // One empty pass; CTA 0 leaves at once, so the other CTAs' first grid barrier sees no
    // progress and gives up after 2 s, raising LP_ETIMEOUT.  No copy is in flight at any point.
    DevBuf ctl, pass;
    int rc = ensure_buf(ctl, exec_ctl_words(1) * sizeof(uint32_t), "self-test control words");
    if (!rc) rc = ensure_buf(pass, sizeof(ExecPass), "self-test pass");
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(ctl.ptr, 0, exec_ctl_words(1) * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pass.ptr, 0, sizeof(ExecPass), st);
    ExecArgs x{};
    x.passes = static_cast<const ExecPass *>(pass.ptr);
    x.npasses = 1;
    x.n = c->params.n;
    x.abar_stride = abar_stride(c);
    x.err = static_cast<int *>(c->err.ptr);
    x.ctl = static_cast<uint32_t *>(ctl.ptr);
    x.selftest_stall = 1;
    if (e == cudaSuccess) e = launch_exec(x, c->num_sms, st);
    c->launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    free_buf(ctl);
    free_buf(pass);
    return e == cudaSuccess ? LP_OK : cuda_fail(e, "executor self-test");
}

extern "C" int lp_selftest_pair_timeout(lp_ctx *c, void *stream)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (!c->have_bsk) return fail(LP_ENOKEY, "load the bootstrapping key first");
    cudaSetDevice(c->device);
    int rc = ensure_scratch(c, 1);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // One ciphertext whose mod-switched inputs are all 0: every step still waits for its key
    // rows and exchanges residues.
    cudaError_t e = cudaMemsetAsync(c->abar.ptr, 0, (size_t)abar_stride(c) * sizeof(uint16_t), st);
    if (e == cudaSuccess)
        e = launch_pair_selftest(static_cast<const uint16_t *>(c->abar.ptr), abar_stride(c),
                                 static_cast<uint32_t *>(c->ext.ptr), static_cast<const uint32_t *>(c->bsk_hat.ptr),
                                 static_cast<const uint2 *>(c->tw_lane.ptr), c->params.n,
                                 static_cast<int *>(c->err.ptr), c->num_sms, st);
    c->launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? LP_OK : cuda_fail(e, "paired-kernel self-test");
}

extern "C" int lp_selftest_quad_timeout(lp_ctx *c, void *stream)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (!c->have_bsk) return fail(LP_ENOKEY, "load the bootstrapping key first");
    cudaSetDevice(c->device);
    int rc = ensure_scratch(c, 1);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(c->abar.ptr, 0, (size_t)abar_stride(c) * sizeof(uint16_t), st);
    if (e == cudaSuccess)
        e = launch_quad_selftest(static_cast<const uint16_t *>(c->abar.ptr), abar_stride(c),
                                 static_cast<uint32_t *>(c->ext.ptr), static_cast<const uint32_t *>(c->bsk_hat.ptr),
                                 static_cast<const uint2 *>(c->tw_lane.ptr), c->params.n,
                                 static_cast<int *>(c->err.ptr), c->num_sms, st);
    c->launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? LP_OK : cuda_fail(e, "quad-kernel self-test");
}

extern "C" int lp_selftest_wait_timeout(lp_ctx *c, uint32_t limit_ms, void *stream)
{
    if (!c) return fail(LP_EINVAL, "null context");
    if (limit_ms == 0 || limit_ms > 10000) return fail(LP_EINVAL, "limit_ms=%u outside [1, 10000]", limit_ms);
    cudaSetDevice(c->device);
    cudaError_t e = launch_wait_probe(static_cast<int *>(c->err.ptr), (uint64_t)limit_ms * 1000000ull,
                                      static_cast<cudaStream_t>(stream));
    c->launches++;
    return e == cudaSuccess ? LP_OK : cuda_fail(e, "wait probe launch");
}
