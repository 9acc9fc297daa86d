/*
 * locpir.h -- C-ABI of liblocpir.so: TFHE gate bootstrapping and the LocPIR circuits
 * (LocPIR: Fast Private Location-based Information Retrieval over the Torus,
 * arXiv 2407.19871) on one GB300 GPU.
 *
 * Conventions (every entry point):
 *   - Torus32: uint32_t, the torus value x / 2^32 mod 1 (two's-complement wrap).
 *   - LWE ciphertext: uint32_t[n + 1] = a[0 .. n-1], b; phase = b - <a, s>.  A batch is
 *     [count][n + 1], contiguous.  Encoding f(m) = m/4 - 1/8: bit 1 -> 2^29, bit 0 -> -2^29
 *     (Section 2.2, Encrypt / Decrypt).
 *   - A coordinate is l ciphertexts, least significant bit first (index l-1 is the MSB that
 *     Algorithm 2 flips).  A box is [4][l][n + 1] in the order X1, X2, Y1, Y2; the point
 *     (x, y) is inside iff X1 <= x < X2 and Y1 <= y < Y2.  A service is [m][n + 1], bit 0
 *     first.
 *   - Pointers named *_dev and every ciphertext pointer of the batch calls are DEVICE
 *     pointers on the context's device; `stream` is a cudaStream_t (NULL = legacy default
 *     stream).  Calls that take a stream are asynchronous: they return once the work is
 *     enqueued; lp_sync() waits and returns a sticky device error (e.g. LP_ETIMEOUT).
 *     Entry points named *_host take host pointers and are synchronous.
 *   - Ownership: the caller owns every input and output buffer; the library never frees
 *     caller memory.  The context owns the device memory it allocates (keys in the
 *     transform domain, scratch) and frees it in lp_destroy.
 *   - Outputs may not alias inputs.  Calls on one context must be issued from one host
 *     thread at a time and on one stream at a time (they share the context's scratch).
 *   - Return value: LP_OK (0) or a negative LP_E* code; lp_last_error() gives a
 *     thread-local message for the last failure.  Nothing throws across this ABI.
 */
#ifndef LOCPIR_H
#define LOCPIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define LP_OK 0
#define LP_EINVAL (-1)   /* bad argument: size, null pointer, unsupported parameter   */
#define LP_ENOMEM (-2)   /* device allocation failed                                    */
#define LP_ECUDA (-3)    /* a CUDA runtime call failed                                  */
#define LP_ENOKEY (-4)   /* an evaluation was requested before both keys were loaded    */
#define LP_ETIMEOUT (-5) /* a device-side wait gave up (bounded waits, ~2 s)            */
#define LP_EBUSY (-6)    /* the server's memory budget is exhausted                     */
#define LP_ECORRUPT (-7) /* key data failed its checksum                                */

/* ---- parameters ---------------------------------------------------------------------
 * TFHE parameters: LWE dimension n, ring degree N, TRLWE dimension k, gadget base 2^Bgbit
 * with lg levels, key-switch base 2^basebit with t digits.  The paper fixes n (Section 5,
 * TFHE Parameters: 630 for the 128-bit set, 540 for the 80-bit set) and defers the rest to
 * TFHE; this build supports N = 1024, k = 1, Bgbit = 10, lg = 3, basebit = 2, t = 8 and
 * any n in [1, 639]. */
typedef struct lp_params {
    int n, N, k, Bgbit, lg, basebit, t;
} lp_params;

/* Gate identifiers.  HomAND is Bootstrap((0, -1/8) + c1 + c2) (Section 2.2, EvalGate); the
 * other gates are the TFHE gate constructions the paper refers to (Section 2.2): NAND
 * (0, 1/8) - c1 - c2, OR (0, 1/8) + c1 + c2, XOR (0, 1/4) + 2c1 + 2c2, XNOR
 * (0, -1/4) - 2c1 - 2c2, NOT = -c1 (no bootstrap), MUX(a, b, c) = a ? b : c from two
 * blind rotations of (0, -1/8) + a + b and (0, -1/8) - a + c summed with (0, 1/8) in
 * dimension N and one key switch. */
enum lp_op { LP_NAND = 0, LP_AND = 1, LP_OR = 2, LP_XOR = 3, LP_XNOR = 4, LP_NOT = 5, LP_MUX = 6 };

/* Comparator kinds: LP_LT = HomCompS(x1, x2) (Algorithm 2, x1 < x2); LP_LE = HomCompLE(x1,
 * x2) = NOT HomCompS(x2, x1) (x1 <= x2; Section 4.2 defines HomCompLE as the negation of
 * HomCompS, read with swapped operands so that it is the inclusive bound Algorithm 3 uses). */
enum lp_cmp { LP_LT = 0, LP_LE = 1 };

/* Combination of the per-box services (Algorithm 3, last line; Algorithm 4).
 * LP_XOR_TREE: pairwise XOR over boxes level by level (box 2i with 2i+1, an odd last row
 * carried up); LP_XOR_CHAIN: Algorithm 4 as printed, S = Enc(0)^m then S[j] ^= S_i[j] box by
 * box; LP_OR_TREE: the tree with OR (correct also for overlapping boxes). */
enum lp_combine { LP_XOR_TREE = 0, LP_XOR_CHAIN = 1, LP_OR_TREE = 2 };

typedef struct lp_ctx lp_ctx;

/* Fill *p with n = 630, N = 1024, k = 1, Bgbit = 10, lg = 3, basebit = 2, t = 8. */
int lp_params_default(lp_params *p);

/* Create a context on CUDA device `device`.  Fails with LP_EINVAL for unsupported
 * parameters, LP_ECUDA if the device cannot be used. */
int lp_create(const lp_params *p, int device, lp_ctx **out);
int lp_destroy(lp_ctx *ctx);

/* Wait for all work the context enqueued; returns LP_ETIMEOUT if a device wait gave up
 * since the last lp_sync (the flag is then cleared), LP_ECUDA on a CUDA error. */
int lp_sync(lp_ctx *ctx);

const char *lp_strerror(int code);
const char *lp_last_error(void);

/* ---- keys (KeyGen, Section 2.2: PK = {bootstrapping key, key-switching key}) ----------
 * Bootstrapping key, coefficient domain, layout [n][2 lg][2][N] uint32 (words =
 * n * 2 lg * 2 * N): row r = c lg + p of BSK_i is a TRLWE sample (component 0 = mask,
 * 1 = body) with s_i 2^(32 - Bgbit (p+1)) added to coefficient 0 of component c.  The
 * library converts it to its transform domain (two NTT primes) on the device and keeps
 * only that copy.  LP_EINVAL if words does not match. */
int lp_load_bsk(lp_ctx *ctx, const uint32_t *bsk, size_t words);
int lp_load_bsk_device(lp_ctx *ctx, const uint32_t *bsk_dev, size_t words, void *stream);

/* Key-switching key, layout [N][t][2^basebit][n + 1] uint32: entry [i][j][v] is an LWE
 * sample of v S_i 2^(32 - basebit (j+1)) under s.  Entries with v = 0 are never read.  The
 * library keeps it as a table of digit-pair sums (16 rows per coefficient and pair of digits,
 * about 166 MB at n = 630) built on the device at load. */
int lp_load_ksk(lp_ctx *ctx, const uint32_t *ksk, size_t words);
int lp_load_ksk_device(lp_ctx *ctx, const uint32_t *ksk_dev, size_t words, void *stream);

/* Key files (the keys are the only persistent state; this is their checkpoint format):
 * header "LPKEYS01", version, the 7 parameters, both word counts and the SHA-256 (FIPS 180-4) of
 * the two key arrays, then the bootstrapping key and the key-switching key in the layouts above.
 * lp_save_keys_file writes one from host arrays (no context).  lp_verify_keys_file checks a file
 * without loading it (LP_ECORRUPT on a bad header, a short file or a checksum mismatch).
 * lp_load_keys_file verifies and loads into a context whose parameters must match.
 * lp_sha256: the hash itself (host). */
int lp_save_keys_file(const lp_params *p, const uint32_t *bsk, const uint32_t *ksk, const char *path);
int lp_verify_keys_file(const char *path, lp_params *params_out);
int lp_load_keys_file(lp_ctx *ctx, const char *path);
int lp_sha256(const void *data, size_t bytes, uint8_t out[32]);

/* ---- gate bootstrapping ----------------------------------------------------------------
 * lp_gate_batch: count independent gates out[g] = op(a[g], b[g]) (MUX: a[g] ? b[g] : c[g];
 * NOT reads a only; c is read by MUX only and may be NULL otherwise).  All pointers device,
 * [count][n + 1].  Each bootstrapped gate is: linear pre-combination, modulus switch to
 * Z_2N, blind rotation (n CMux external products with the bootstrapping key), sample
 * extraction, key switch.  LP_ENOKEY before both keys are loaded.  count = 0 is a no-op. */
int lp_gate_batch(lp_ctx *ctx, int op, const uint32_t *a, const uint32_t *b, const uint32_t *c,
                  uint32_t *out, size_t count, void *stream);

/* Same, host pointers; copies in and out and synchronises. */
int lp_gate_batch_host(lp_ctx *ctx, int op, const uint32_t *a, const uint32_t *b, const uint32_t *c,
                       uint32_t *out, size_t count);

/* lp_gate_batch_noalloc: the same gates as lp_gate_batch, bit for bit, for
 * callers that must not allocate device memory while they evaluate -- e.g. a server whose
 * device memory is handed out up front by its own allocator and budget, or a latency-critical
 * loop that cannot absorb the device-wide synchronisation of cudaMalloc / cudaFree.  (The
 * paper has no counterpart; this is a deployment variant of the gate batch.)
 * It allocates nothing: no cudaMalloc, cudaFree or allocating library call.  Its scratch (the
 * mod-switched inputs and the extracted samples) is a fixed array of about 1.5 MiB compiled
 * into the library, held by every GPU that loads the library until the process exits.
 * Limit: at most 256 blind rotations per call (count <= 256 for two-input gates, <= 128 for
 * MUX; NOT uses no scratch); larger counts return LP_EINVAL.  The first call on a device looks
 * up the array's device address with that device current (a one-time set-up per device); make
 * that first call before any stream capture.  All calls share the array and it keeps the last
 * call's contents (nothing in it needs clearing: every word read is written earlier in the same
 * call), so calls that overlap on the GPU race: issue them in order on one stream.  Keys must be
 * loaded (LP_ENOKEY otherwise); pointers and layout as in lp_gate_batch.
 * Kernels: always the NTT blind rotation and the table key switch.  A forced split or batched
 * NTT choice (lp_set_engines) is honoured; a tensor-core engine selection is ignored here,
 * because those engines allocate their scratch.  The per-phase timers are not recorded.
 * A device reset (cudaDeviceReset) after the first call invalidates the looked-up address:
 * the entry point then stays unusable on that device until the process restarts. */
int lp_gate_batch_noalloc(lp_ctx *ctx, int op, const uint32_t *a, const uint32_t *b, const uint32_t *c,
                          uint32_t *out, size_t count, void *stream);

/* The two halves of a bootstrap, exposed for step-level parity checks.
 * lp_bootstrap_extract: count LWEs [count][n + 1] -> modulus switch, blind rotation with
 * test vector v_j = mu for all j, sample extraction -> [count][N + 1] N-LWEs under S.
 * lp_key_switch: count N-LWEs [count][N + 1] -> [count][n + 1] LWEs under s. */
int lp_bootstrap_extract(lp_ctx *ctx, const uint32_t *lwe, uint32_t mu, uint32_t *ext, size_t count,
                         void *stream);
int lp_key_switch(lp_ctx *ctx, const uint32_t *ext, uint32_t *out, size_t count, void *stream);

/* ---- circuits ---------------------------------------------------------------------------
 * lp_compare_batch: count comparisons of l-bit values, x1 and x2 [count][l][n + 1] (LSB
 * first), out [count][n + 1] encrypting x1 < x2 (LP_LT) or x1 <= x2 (LP_LE); is_signed
 * selects two's-complement order (Algorithm 2 with its MSB flip) or unsigned order (the
 * same loop without the flip).  Gates of all comparisons run in shared batches, level by
 * level: l + 1 bootstrap levels. */
int lp_compare_batch(lp_ctx *ctx, int kind, int is_signed, int l, const uint32_t *x1, const uint32_t *x2,
                     uint32_t *out, size_t count, void *stream);

/* One LocPIR query (Algorithm 3): point x, y [l][n + 1] each, n_boxes boxes
 * [n_boxes][4][l][n + 1], services [n_boxes][m][n + 1]; out_service [m][n + 1] encrypts the
 * combination (comb) of the services of the boxes that contain the point. */
int lp_locpir_query(lp_ctx *ctx, int l, int is_signed, const uint32_t *x, const uint32_t *y, int n_boxes,
                    const uint32_t *boxes, int m, const uint32_t *services, int comb, uint32_t *out_service,
                    void *stream);

/* Several LocPIR queries with their own l, n_boxes, m and pointers (uneven shapes); all
 * their gates are scheduled together by bootstrap level.  Pointers as in lp_locpir_query. */
typedef struct lp_query {
    int l, is_signed, n_boxes, m, comb;
    const uint32_t *x, *y, *boxes, *services;
    uint32_t *out_service;
} lp_query;
int lp_locpir_batch(lp_ctx *ctx, const lp_query *q, size_t nq, void *stream);

/* The same queries in memory-budgeted waves: queries are taken in order into a wave while its
 * circuit's device memory (ciphertext pool and job records: one (n + 1)-word ciphertext per wire
 * of the levelled circuit, Algorithms 2-5) stays within mem_budget bytes; each wave is scheduled
 * by bootstrap level as in lp_locpir_batch, and the waves run one after another on the stream.
 * The pass scratch (at most 131,072 blind rotations: ~0.7 GB) comes on top of the budget.
 * *waves_out (may be null) receives the number of waves.  LP_ENOMEM if one query alone exceeds
 * the budget.  Outputs are bit-identical to lp_locpir_batch over the same queries. */
int lp_locpir_batch_waves(lp_ctx *ctx, const lp_query *q, size_t nq, size_t mem_budget, size_t *waves_out,
                          void *stream);

/* ---- server-known box bounds (beyond the paper) ------------------------------------------
 * When the server holds the box bounds in the clear, Algorithm 2's second operand is a known
 * bit string: XNOR with a known bit is the point bit or its negation (no bootstrap), and the
 * MUX with a known arm is one AND (bound bit 0) or one OR (bound bit 1) of the negated point
 * bit with the running result, so a comparator costs at most l - 1 bootstraps instead of 3l.
 * While the running result is still a known constant no gate is made.
 *
 * lp_compare_known_batch: x [count][l][n + 1] (LSB first, device), k [count] plaintext
 * bounds (host, low l bits used as the bit pattern; with is_signed they are two's
 * complement); out [count][n + 1] encrypts x < k (LP_LT) or k <= x (LP_LE, the negation).
 * A comparison whose result is known without a gate (e.g. unsigned x < 0) is written as
 * the trivial encryption of that bit. */
int lp_compare_known_batch(lp_ctx *ctx, int kind, int is_signed, int l, const uint32_t *x, const uint64_t *k,
                           uint32_t *out, size_t count, void *stream);

/* LocPIR queries with known bounds: as lp_query, but bounds [n_boxes][4] (X1, X2, Y1, Y2;
 * host memory, read during the call) replace the encrypted boxes.  The point is inside a box
 * iff X1 <= x < X2 and Y1 <= y < Y2; validation, bitwiseAND and the combine are Algorithm 3's. */
typedef struct lp_query_known {
    int l, is_signed, n_boxes, m, comb;
    const uint32_t *x, *y;
    const uint64_t *bounds;
    const uint32_t *services;
    uint32_t *out_service;
} lp_query_known;
int lp_locpir_known_batch(lp_ctx *ctx, const lp_query_known *q, size_t nq, void *stream);

/* ---- alternative product engines (measured against the defaults; beyond the paper) -------
 * lp_set_engines selects the engines of lp_gate_batch, lp_gate_batch_host,
 * lp_bootstrap_extract and lp_key_switch (circuits, plans and the server always use the
 * defaults).  Every engine computes the same exact integers, so outputs are bit-identical.
 *   LP_BR_NTT          two-prime NTT external products in shared memory (default): a level
 *                      of at most one ciphertext per four SMs runs on the quad kernel (one
 *                      ciphertext per cluster of four CTAs: prime x ACC component, exchanging
 *                      partial sums and residues through distributed shared memory), one of at
 *                      most one per two SMs paired (clusters of two CTAs, one per prime), one
 *                      of at most two per SM split (one ciphertext per CTA, its 12
 *                      digit-and-prime transforms on 12 warps), a larger one batched (4
 *                      ciphertexts per CTA sharing each key row);
 *   LP_BR_NTT_BATCHED  the NTT engine, always batched;
 *   LP_BR_NTT_SPLIT    the NTT engine, always split (one CTA per ciphertext);
 *   LP_BR_NTT_PAIR     the NTT engine, always paired;
 *   LP_BR_NTT_QUAD     the NTT engine, always on the quad kernel;
 *   LP_BR_TENSOR_BF16  per step one Toeplitz(BSK_i) x digit-matrix GEMM on the bf16 tensor
 *                      cores (cuBLAS), factors split into 6-bit limbs so fp32 sums stay exact;
 *   LP_BR_TENSOR_INT8  the same with 8-bit limbs on the int8 tensor cores, int32 sums;
 *   LP_KS_TABLE        digit-pair table gather (default);
 *   LP_KS_TENSOR_INT8  one-hot digits x KSK limbs as one int8 GEMM per batch.
 * Returns LP_EINVAL for an unknown engine.  May be called before or after the keys are loaded;
 * the key layouts an engine needs are built when both are available. */
#define LP_BR_NTT 0
#define LP_BR_TENSOR_BF16 1
#define LP_BR_TENSOR_INT8 2
#define LP_BR_NTT_BATCHED 3
#define LP_BR_NTT_SPLIT 4
#define LP_BR_NTT_PAIR 5
#define LP_BR_NTT_QUAD 6
#define LP_KS_TABLE 0
#define LP_KS_TENSOR_INT8 1
int lp_set_engines(lp_ctx *ctx, int br_engine, int ks_engine);

/* Launch policy of a context, chosen by the autotuner (no counterpart in the paper, whose
 * gates run one per call on a CPU):
 *   split_max     the widest level the blind rotation runs on the split kernel (one ciphertext
 *                 per CTA); 0 = the built-in rule, two ciphertexts per SM;
 *   tail_split    1: a wider level runs its full batched waves batched and its partial last
 *                 wave split, when that remainder is at most split_max; 0: all batched;
 *   ks_slice_max  key switches of at most this many 64-output batches split their input
 *                 coefficients across CTAs; 0 = the built-in rule (fewer than half the SMs),
 *                 -1 = never;
 *   from_cache    (output only) 1 when lp_autotune_cached read the choices from its cache;
 *   pair_max      a level (or partial last wave) that would run split and has at most this many
 *                 ciphertexts runs on the paired kernel (one ciphertext per two SMs); 0 = the
 *                 built-in rule (as many as clusters of two CTAs fit on the device at once),
 *                 -1 = never;
 *   quad_max      the same for the quad kernel (one ciphertext per four SMs), checked first.
 * Every policy gives the same output bits. */
#define LP_TUNING_SCHEMA 3
typedef struct lp_tuning {
    int split_max, tail_split, ks_slice_max, from_cache, pair_max, quad_max;
} lp_tuning;

/* lp_autotune: measures the policy on this device (synthetic inputs, CUDA events, about 0.5 s):
 * both NTT blind-rotation kernels at levels of 1-4 ciphertexts per SM (split_max: the largest
 * multiple of the SM count up to which the split kernel is still faster, never below one per
 * SM; tail_split when the split kernel beats a batched wave at one per SM), and the key switch
 * sliced against whole-table CTAs at 1/4 to 1 batch per SM (ks_slice_max: the widest batch
 * count of the leading run where slicing is faster), the paired kernel against the split
 * kernel at one ciphertext per resident cluster (pair_max: that count when paired is faster,
 * else -1), and the quad kernel against the faster of those two at one ciphertext per
 * resident cluster of four (quad_max, likewise).  Applies it to the context.
 * *split_max_out (may be NULL) receives split_max.  Needs both keys (LP_ENOKEY); uses the
 * context's scratch, so call it while no other work of this context is in flight (not while a
 * server runs). */
int lp_autotune(lp_ctx *ctx, int *split_max_out);
/* lp_autotune_cached: as lp_autotune, but reads the choices from the JSON file cache_path when
 * it holds an entry for this device (GPU name, SM count, LWE dimension n, LP_TUNING_SCHEMA) and
 * force is 0; otherwise measures and writes the file (replacing it; cache_path NULL: no file).
 * *out (may be NULL) receives the applied policy.  LP_EINVAL if the file cannot be written. */
int lp_autotune_cached(lp_ctx *ctx, const char *cache_path, int force, lp_tuning *out);
/* Circuit executor of a context (lp_compare_batch, lp_locpir_*, plans; not the server):
 *   LP_EXEC_LEVELS      per bootstrap level, three kernels (pre-combination, blind rotation, key
 *                       switch) queued on the stream; plans capture them into one CUDA graph;
 *   LP_EXEC_PERSISTENT  one persistent kernel (one CTA per SM, cooperative launch) runs every
 *                       level: its CTAs take the level's gate groups and key-switch batches from
 *                       device-side counters and meet at grid-wide barriers between phases; a
 *                       barrier wait that sees no progress for 2 s ends the run with LP_ETIMEOUT.
 * Both give the same output bits.  LP_EINVAL for another value. */
#define LP_EXEC_LEVELS 0
#define LP_EXEC_PERSISTENT 1
int lp_set_executor(lp_ctx *ctx, int executor);

/* Apply a policy explicitly (e.g. the built-in rules: all fields 0) / read the current one. */
int lp_set_tuning(lp_ctx *ctx, const lp_tuning *t);
int lp_get_tuning(const lp_ctx *ctx, lp_tuning *t);

/* lp_circuit_info: the gate statistics of one LocPIR query's circuit (Algorithms 2-5; the
 * comparators of Algorithm 2, validation, bitwiseAND of Algorithm 5, the combine `comb`) as
 * the library builds and levels it for the batch entry points, plans and the server.  With
 * bounds == NULL the box bounds are encrypted inputs; otherwise bounds [n_boxes][4] (X1, X2,
 * Y1, Y2; host memory, read during the call) are server-known, as in lp_query_known.  Host
 * only: needs no context and no GPU.  *out receives:
 *   gates_by_op[op]   bootstrapped gates per lp_op code (NOT is free and never counted);
 *   blind_rotations   one per gate, two per MUX;  key_switches  one per gate;
 *   levels            bootstrap depth = the number of levels the scheduler runs;
 *   widest_level      blind rotations of the widest level;  wires  circuit wires incl. inputs.
 * LP_EINVAL for l outside [1, 64], n_boxes < 1, m < 1, an unknown comb or a null out. */
typedef struct lp_circuit_stats {
    uint64_t gates_by_op[8];
    uint64_t blind_rotations, key_switches, levels, widest_level, wires;
} lp_circuit_stats;
int lp_circuit_info(int l, int is_signed, int n_boxes, int m, int comb, const uint64_t *bounds,
                    lp_circuit_stats *out);

/* Plans: lp_plan_locpir schedules a batch of queries once (levels, job records, a plan-owned
 * pool and scratch) and captures the whole evaluation -- input copies from the queries' pointers,
 * every level's pre-combination / blind-rotation / key-switch pass, output copies -- into one
 * CUDA graph.  lp_plan_run replays it on a stream (asynchronous; the queries' pointers must stay
 * valid while the plan exists, their contents may change between runs).  lp_plan_info reports the
 * plan's blind rotations, key switches and kernels per run. */
typedef struct lp_plan lp_plan;
int lp_plan_locpir(lp_ctx *ctx, const lp_query *q, size_t nq, lp_plan **out);
/* The same for queries with server-known bounds (lp_query_known; the bounds are read during
 * the call and fixed in the plan's circuit). */
int lp_plan_locpir_known(lp_ctx *ctx, const lp_query_known *q, size_t nq, lp_plan **out);
int lp_plan_run(lp_plan *plan, void *stream);
int lp_plan_info(const lp_plan *plan, uint64_t *blind_rotations, uint64_t *key_switches, uint64_t *kernels);
int lp_plan_destroy(lp_plan *plan);

/* ---- query server (continuous batching) ---------------------------------------------------
 * lp_server_start: start a server thread on the context.  Queries are admitted in arrival order
 * while their circuit's ciphertexts ((wires) x (n + 1) x 4 B: inputs, gate outputs, one trivial
 * constant) fit in a device pool of mem_budget bytes; admission copies the inputs into the pool,
 * where they stay resident until the result is written.  Each scheduler tick evaluates the next
 * bootstrap level of every admitted query as one shared batch (pre-combination, blind rotation,
 * key switch), so queries of different shapes and depths share batches.  policy LP_SERVER_QUEUE
 * keeps queries that do not fit waiting; LP_SERVER_REJECT refuses them with LP_EBUSY.  Scratch for
 * the shared batches is allocated outside the budget.  Results are bit-identical to
 * lp_locpir_query on the same query.  While a server runs, call no other evaluation entry point
 * on its context (other contexts may be used from other threads); submit, poll, wait and stats
 * are safe from any thread.
 * lp_server_submit: the query's device pointers (inputs and out_service) must stay valid until the
 * query is done; *ticket identifies it.  A query larger than the whole budget returns LP_EBUSY.
 * lp_server_poll: *done = 1 once out_service holds the result.  lp_server_wait: block up to
 * timeout_ms (LP_ETIMEOUT).  lp_server_stats: counters and latency percentiles of completed
 * queries (submit -> result on the device).  lp_server_stop: stop after the tick in flight,
 * abandoning unfinished queries (their out_service is not written; poll keeps reporting not
 * done), join the thread and free the pool. */
#define LP_SERVER_QUEUE 0
#define LP_SERVER_REJECT 1
typedef struct lp_stats {
    uint64_t submitted, admitted, completed, rejected, waiting, active, ticks, bootstraps;
    double p50_ms, p99_ms, mean_ms, elapsed_s, queries_per_s, bootstraps_per_s;
} lp_stats;
int lp_server_start(lp_ctx *ctx, size_t mem_budget, int policy);
int lp_server_submit(lp_ctx *ctx, const lp_query *q, uint64_t *ticket);
/* The same for a query with server-known bounds (lp_query_known; its bounds array is copied
 * during the call, the device pointers must stay valid until the result is written). */
int lp_server_submit_known(lp_ctx *ctx, const lp_query_known *q, uint64_t *ticket);
int lp_server_poll(lp_ctx *ctx, uint64_t ticket, int *done);
int lp_server_wait(lp_ctx *ctx, uint64_t ticket, uint32_t timeout_ms);
int lp_server_stats(lp_ctx *ctx, lp_stats *out);
int lp_server_stop(lp_ctx *ctx);

/* ---- client-side helpers on the device (no context) -------------------------------------
 * Encrypt (Section 2.2) and the zero-phase samples of Algorithm 1: out[g] = (a_g,
 * <a_g, s> + e_g + mu_g) with the caller's uniform masks mask [count][n], noise [count]
 * and messages mu [count] (torus32).  s: [n] uint8 key bits.  Device pointers. */
int lp_client_lwe_encrypt(int n, const uint8_t *s, const uint32_t *mask, const uint32_t *noise,
                          const uint32_t *mu, uint32_t *out, size_t count, void *stream);
/* phase[g] = b_g - <a_g, s> (Decrypt rounds it: bit = (int32)phase > 0). */
int lp_client_lwe_phase(int n, const uint8_t *s, const uint32_t *ct, uint32_t *phase, size_t count,
                        void *stream);
/* Bootstrapping key from its randomness: S [N] key bits, mask and noise [n][2 lg][N];
 * row r = c lg + p is (a, a S + e) with s_i 2^(32 - Bgbit (p+1)) added to coefficient 0 of
 * component c.  Output [n][2 lg][2][N].  Device pointers. */
int lp_client_keygen_bsk(const lp_params *p, const uint8_t *s, const uint8_t *S, const uint32_t *mask,
                         const uint32_t *noise, uint32_t *bsk, void *stream);
/* Key-switching key: mask [N][t][2^basebit][n], noise [N][t][2^basebit]; output
 * [N][t][2^basebit][n + 1], entry [i][j][v] = (a, <a, s> + e + v S_i 2^(32 - basebit (j+1))). */
int lp_client_keygen_ksk(const lp_params *p, const uint8_t *s, const uint8_t *S, const uint32_t *mask,
                         const uint32_t *noise, uint32_t *ksk, void *stream);

/* Algorithm 1 (Preprocess): out[g] = zero[g] + (0, f(bits[g])), turning the client's zero-phase
 * samples zero [count][n + 1] (b = <a, s> + e, sent with the public key) into encryptions of the
 * service bits bits [count] (uint8, 0 or 1).  The paper's text says the samples encrypt "0";
 * their printed form b = a K + e has phase 0, which is the reading used (adding f(1) = +1/8 or
 * f(0) = -1/8 then gives a valid encryption).  Device pointers. */
int lp_preprocess_services(int n, const uint32_t *zero, const uint8_t *bits, uint32_t *out, size_t count,
                           void *stream);

/* ---- introspection -------------------------------------------------------------------- */
/* Kernel launches this context has issued since creation (every launch of the library's
 * own kernels counts one). */
uint64_t lp_launch_count(const lp_ctx *ctx);
/* Average device time (ms) of the blind-rotation kernel over the launches timed since the
 * last reset, measured with CUDA events on the launching stream; *launches receives the
 * number of timed launches.  Timing is enabled by lp_set_timing(ctx, 1). */
int lp_set_timing(lp_ctx *ctx, int enable);
int lp_kernel_time(lp_ctx *ctx, const char *kernel, double *ms_total, uint64_t *launches);
int lp_reset_timing(lp_ctx *ctx);

/* Failure-detection self-test: launches a kernel that waits on a barrier nothing completes,
 * with the library's bounded wait (limit_ms, 1..10000).  The wait gives up, the kernel records
 * a timeout and returns; the next lp_sync reports LP_ETIMEOUT and the context stays usable.
 * Every wait inside the library's kernels uses the same bounded routine (2 s limit). */
int lp_selftest_wait_timeout(lp_ctx *ctx, uint32_t limit_ms, void *stream);
/* lp_selftest_exec_timeout: launches the persistent executor on one empty pass with one CTA
 * leaving at once, so the others' grid-barrier wait runs out after 2 s; synchronous.  The
 * device error word then holds LP_ETIMEOUT (lp_sync returns it) and the context stays usable. */
int lp_selftest_exec_timeout(lp_ctx *ctx, void *stream);
/* lp_selftest_pair_timeout: runs the paired blind rotation on one ciphertext with CTA rank 1 of
 * its cluster issuing no key copy.  Its first key wait gives up after 2 s, it tells its
 * partner through the residue exchange's status word, and both CTAs stop after that exchange
 * (the partner's exchange wait would itself give up after 8 s); synchronous, about 4 s.  The
 * device error word then holds LP_ETIMEOUT (lp_sync returns it) and the context stays usable.
 * LP_ENOKEY before lp_load_bsk. */
int lp_selftest_pair_timeout(lp_ctx *ctx, void *stream);
/* lp_selftest_quad_timeout: the same for the quad blind rotation (a cluster of four CTAs; rank 1
 * issues no key copy).  Its stop decision reaches the CTA of the same prime in the partial-sum
 * exchange and the other prime's CTAs in the residue exchange of the same step, so all four
 * stop together; synchronous, about 4 s; LP_ETIMEOUT afterwards, the context stays usable. */
int lp_selftest_quad_timeout(lp_ctx *ctx, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LOCPIR_H */
