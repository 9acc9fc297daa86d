// Internal launcher declarations of liblocpir (not part of the public C-ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace lp {

// One blind-rotation job of a circuit level: pre-combination sum_k coef_k pool[in[k]] +
// (0, bconst); coef 0 marks an unused operand.
struct BrJob {
    int32_t in[3];
    int32_t coef[3];
    uint32_t bconst;
    int32_t pad;
};

// One key-switch job: ext rows e1 (+ e2 when e2 >= 0, for MUX) + (0, bconst) -> out row.
struct KsJob {
    int32_t e1, e2;
    uint32_t bconst;
    int32_t out;
};

// One copy of a ciphertext out of the circuit pool, negated when neg != 0.
struct CopyEntry {
    const uint32_t *src;
    uint32_t *dst;
    int32_t neg;
    int32_t pad;
};

// Persistent circuit executor (blind_rotate.cu): one launch runs every pass of a levelled
// schedule.  A pass is the pre-combination + blind rotation of br_cnt jobs from br_off and the
// key switch of ks_cnt jobs from ks_off.
struct ExecPass {
    uint32_t br_off, br_cnt, ks_off, ks_cnt;
};
struct ExecArgs {
    const ExecPass *passes;
    int npasses;
    const BrJob *br;
    const KsJob *ks;
    const CopyEntry *outc;
    uint32_t nout;
    uint32_t *pool;
    uint16_t *abar;
    int abar_stride;
    uint32_t *ext;
    const uint32_t *bsk_hat;
    const uint2 *tw_lane;
    const uint32_t *T;
    int n;
    int ks_slice_max;
    int *err;
    uint32_t *ctl;   // exec_ctl_words(npasses) words, zero before the launch
    int selftest_stall;   // self-test only: CTA 0 leaves before the first barrier, so the others' wait runs out
};
// Control words: barrier count, barrier generation, progress, abort flag, then per pass the
// blind-rotation and key-switch work counters.
__host__ __device__ __forceinline__ size_t exec_ctl_words(int npasses) { return 4 + 2 * (size_t)npasses; }
size_t exec_smem_bytes();
// Cooperative launch over one CTA per SM (every CTA must be resident: the phases meet at
// grid-wide barriers whose waits give up, with LP_ETIMEOUT, after 2 s without progress).
cudaError_t launch_exec(const ExecArgs &x, int num_sms, cudaStream_t st);

size_t br_smem_bytes();
size_t ks_smem_bytes();
size_t br_split_smem_bytes();
// Blind-rotation kernel choice: AUTO runs levels of at most split_max ciphertexts split
// (br_split_kernel, one ciphertext per CTA over 12 warps) and larger ones batched
// (br_kernel, BR_SLOTS ciphertexts per CTA); split_max <= 0 means the measured GB300 rule,
// two ciphertexts per SM (lp_autotune measures it on the device at hand).  The other two
// variants force one kernel.
constexpr int BR_VARIANT_AUTO = 0;
constexpr int BR_VARIANT_BATCHED = 1;
constexpr int BR_VARIANT_SPLIT = 2;
constexpr int BR_VARIANT_PAIR = 3;
constexpr int BR_VARIANT_QUAD = 4;
// tail_split: with AUTO, a level wider than split_max runs its full batched waves batched and
// the remainder split when the remainder is at most split_max.  pair_max: with AUTO, a level (or
// remainder) run split that has at most pair_max ciphertexts runs on br_pair_kernel instead
// (one ciphertext per cluster of two CTAs, one per prime), and one of at most quad_max on
// br_quad_kernel (four CTAs: prime x ACC component); 0 never.  *launched (may be null)
// receives the number of kernels launched.
cudaError_t launch_br(const uint16_t *abar, int abar_stride, uint32_t *ext, const uint32_t *bsk_hat,
                      const uint2 *tw_lane, int n, int jobs, uint32_t mu, int *err, int num_sms, cudaStream_t st,
                      int variant = BR_VARIANT_AUTO, int split_max = 0, int tail_split = 0, int pair_max = 0,
                      int quad_max = 0, int *launched = nullptr);
// The paired kernel's stop self-test: one ciphertext (abar: one row), CTA rank 1 of its cluster
// issues no key copy, so its first wait runs out after 2 s and both CTAs stop after the same
// exchange with DEV_ERR_TIMEOUT; nothing is in flight when they leave.
cudaError_t launch_pair_selftest(const uint16_t *abar, int abar_stride, uint32_t *ext, const uint32_t *bsk_hat,
                                 const uint2 *tw_lane, int n, int *err, int num_sms, cudaStream_t st);
// The same for the quad kernel (CTA rank 1 of its cluster of four issues no key copy).
cudaError_t launch_quad_selftest(const uint16_t *abar, int abar_stride, uint32_t *ext, const uint32_t *bsk_hat,
                                 const uint2 *tw_lane, int n, int *err, int num_sms, cudaStream_t st);
// Clusters of br_pair_kernel that are resident at once on this device (0 when the query fails).
int br_pair_clusters(int num_sms);
int br_quad_clusters(int num_sms);
size_t br_quad_smem_bytes();
size_t br_pair_smem_bytes();
cudaError_t launch_bsk_to_ntt(const uint32_t *bsk, uint32_t *bsk_hat, int n, const uint2 *tw_lane, uint32_t scale0,
                              uint32_t scale1, int num_sms, cudaStream_t st);
cudaError_t launch_precomb_dense(int op, const uint32_t *a, const uint32_t *b, const uint32_t *c, int n,
                                 size_t count, uint16_t *abar, int abar_stride, int num_sms, cudaStream_t st);
cudaError_t launch_modswitch(const uint32_t *lwe, int n, size_t jobs, uint16_t *abar, int abar_stride, int num_sms,
                             cudaStream_t st);
cudaError_t launch_precomb_indexed(const BrJob *jobs, size_t njobs, const uint32_t *pool, int n, uint16_t *abar,
                                   int abar_stride, int num_sms, cudaStream_t st);
// Key switch from the digit-pair table T (built by launch_ks_table at key load).  Batches of
// KS_CT outputs; when there are at most slice_max batches (0: fewer than half the SMs), the
// input coefficients are split across CTAs (see keyswitch.cu).  *launched as for launch_br.
cudaError_t launch_ks(const uint32_t *ext, const KsJob *jobs, size_t njobs, int dense_mux, uint32_t *out,
                      const uint32_t *T, int n, int *err, int num_sms, cudaStream_t st, int slice_max = 0,
                      int *launched = nullptr);
// Sliced (1) or whole-table (0) key switch regardless of the batch count (autotuner).
cudaError_t launch_ks_forced(const uint32_t *ext, size_t njobs, uint32_t *out, const uint32_t *T, int n, int *err,
                             int num_sms, cudaStream_t st, int sliced);
cudaError_t launch_ks_table(const uint32_t *ksk, uint32_t *T, int n, int num_sms, cudaStream_t st);
// Words per key-switch table row and per output ciphertext buffer row: n + 1 rounded up to 4.
__host__ __device__ __forceinline__ int ks_row_words(int n) { return ((n + 1) + 3) & ~3; }
__host__ __device__ size_t ks_table_words(int n);
cudaError_t launch_negate(const uint32_t *in, uint32_t *out, size_t words, int num_sms, cudaStream_t st);
cudaError_t launch_gather(const uint32_t *pool, const int *slots, const uint8_t *neg, size_t cnt, int n,
                          uint32_t *out, int num_sms, cudaStream_t st);
cudaError_t launch_trivial(uint32_t *dst, int n, uint32_t b, cudaStream_t st);
cudaError_t launch_lwe_encrypt(int n, const uint8_t *s, const uint32_t *mask, const uint32_t *noise,
                               const uint32_t *mu, uint32_t *out, size_t count, int num_sms, cudaStream_t st);
cudaError_t launch_lwe_phase(int n, const uint8_t *s, const uint32_t *ct, uint32_t *phase, size_t count,
                             int num_sms, cudaStream_t st);
cudaError_t launch_keygen_bsk(int n, const uint8_t *s, const uint8_t *S, const uint32_t *mask,
                              const uint32_t *noise, uint32_t *bsk, int num_sms, cudaStream_t st);
cudaError_t launch_keygen_ksk(int n, const uint8_t *s, const uint8_t *S, const uint32_t *mask,
                              const uint32_t *noise, uint32_t *ksk, int num_sms, cudaStream_t st);

cudaError_t launch_wait_probe(int *err, uint64_t limit_ns, cudaStream_t st);
cudaError_t launch_preprocess(int n, const uint32_t *zero, const uint8_t *bits, uint32_t *out, size_t count,
                              int num_sms, cudaStream_t st);

// Twiddle and constant tables (host side) uploaded at context creation.
struct NttTables {
    uint32_t prime[2];                  // the two NTT primes
    uint2 ctw[2][2][32];                // warp-uniform stages
    uint2 lane[2][2][31 * 32];          // lane-dependent stages
    uint32_t pinv_neg[2];               // Montgomery constants -p^-1 mod 2^32
    uint32_t red_one[2];                // floor(2^32 / p): lazy reduction by 1
    uint2 crt;                          // p0^-1 mod p1 and its Shoup companion
    uint32_t bsk_scale[2];              // N^-1 2^32 mod p
};
void build_ntt_tables(NttTables &t);
cudaError_t upload_constants(const NttTables &t);

}  // namespace lp
