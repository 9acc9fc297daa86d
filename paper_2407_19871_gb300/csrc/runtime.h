// Context structure and host helpers of liblocpir (internal).
#pragma once
#include <atomic>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/locpir.h"
#include "kernels.h"

namespace lp {

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct Server;

struct KernelTimer {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    double ms = 0.0;
    uint64_t count = 0;
};

}  // namespace lp

struct lp_ctx {
    lp_params params{};
    int device = 0;
    int num_sms = 1;
    lp::NttTables tables{};
    lp::DevBuf tw_lane, err;        // lane twiddles, device error word
    lp::DevBuf bsk_hat, ksk;        // keys (transform-domain BSK, coefficient KSK)
    lp::DevBuf abar, ext;           // per-pass scratch: mod-switched inputs, extracted samples
    lp::DevBuf pool, jobs;          // circuit ciphertext pool and job records
    lp::DevBuf tmp_in, tmp_out;     // staging of the host-pointer entry points
    bool have_bsk = false, have_ksk = false;
    bool timing = false;
    std::atomic<uint64_t> launches{0};   // incremented by the server thread too
    std::map<std::string, lp::KernelTimer> timers;
    lp::Server *server = nullptr;   // query server (lp_server_start), if running
    // Alternative tensor-core engines (tensor_engine.cu) and their state.
    int br_engine = LP_BR_NTT, ks_engine = LP_KS_TABLE;
    int br_split_max = 0;           // widest level run split (0: the default rule; lp_autotune)
    int br_tail_split = 0;          // a wider level's partial last wave runs split (lp_autotune)
    int br_pair_max = 0;            // paired-kernel limit as set (0: resident clusters, -1: never)
    int br_pair_clusters = 0;       // clusters of the paired kernel resident at once
    int br_quad_max = 0;            // quad-kernel limit as set (0: resident clusters, -1: never)
    int br_quad_clusters = 0;       // clusters of the quad kernel resident at once
    int ks_slice_max = 0;           // key switches of at most this many batches run sliced (0: rule)
    int executor = LP_EXEC_LEVELS;  // circuits: per-level kernels or the persistent executor
    void *blas = nullptr;           // cuBLAS handle, created on first use
    lp::DevBuf bsk_coef;            // coefficient-domain BSK (Toeplitz engine)
    lp::DevBuf tc_T, tc_D, tc_C, tc_acc, ks_A, ks_H, ks_C, ks_aux;
    // Pipelined host-pointer batches (lp_gate_batch_host): copy and compute streams, events.
    static constexpr int HOST_CHUNKS = 4;
    cudaStream_t st_h2d = nullptr, st_run = nullptr, st_d2h = nullptr;
    cudaEvent_t ev_in[HOST_CHUNKS] = {}, ev_run[HOST_CHUNKS] = {};
};

namespace lp {

int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
int ensure_buf(DevBuf &b, size_t bytes, const char *what);
void free_buf(DevBuf &b);
int ctx_check_err(lp_ctx *c);
int abar_stride(const lp_ctx *c);
int ensure_scratch(lp_ctx *c, size_t br_jobs);
int run_br(lp_ctx *c, size_t jobs, uint32_t mu, cudaStream_t st);
// The blind-rotation kernel choice (BR_VARIANT_*) of an NTT engine selection.
int br_variant(const lp_ctx *c);
// Widest level (or remainder) that runs on the paired kernel; 0 = none.
inline int br_pair_limit(const lp_ctx *c)
{
    return c->br_pair_max == 0 ? c->br_pair_clusters : c->br_pair_max < 0 ? 0 : c->br_pair_max;
}
// Widest level (or remainder) that runs on the quad kernel; 0 = none.
inline int br_quad_limit(const lp_ctx *c)
{
    return c->br_quad_max == 0 ? c->br_quad_clusters : c->br_quad_max < 0 ? 0 : c->br_quad_max;
}
int run_ks(lp_ctx *c, const KsJob *jobs, size_t njobs, int dense_mux, uint32_t *out, cudaStream_t st);
int run_br_tensor(lp_ctx *c, size_t jobs, uint32_t mu, cudaStream_t st);
int run_ks_tensor(lp_ctx *c, const KsJob *jobs, size_t njobs, int dense_mux, uint32_t *out, cudaStream_t st);
int ks_tensor_prepare(lp_ctx *c, cudaStream_t st);
void tc_release(lp_ctx *c);
void timer_begin(lp_ctx *c, const char *name, cudaStream_t st, cudaEvent_t *ev0);
void timer_end(lp_ctx *c, const char *name, cudaStream_t st, cudaEvent_t ev0);

}  // namespace lp
