// Blind rotation + sample extraction (the hot loop of gate bootstrapping) and the
// conversion of the bootstrapping key to the transform domain.
//
// TFHE gate bootstrapping (Chillotti et al., J. Cryptology 2020; LocPIR Section 2.2
// defers to it): ACC = (0, X^-bbar v); for i < n: ACC += BSK_i [x] ((X^abar_i - 1) ACC);
// then extract coefficient 0 as an N-LWE.  Every ciphertext of a batch reads the same
// BSK_i at step i, so one CTA runs BR_SLOTS ciphertexts in lock step and streams each
// BSK_i slice from L2 into shared memory once for all of them.
//
// CTA layout (BR_THREADS = 8 warps, two per SM sub-partition so that each thread may
// hold up to 255 registers):
//   Warp w serves ciphertext slot w / 2 and NTT prime w % 2; the two warps of a slot (a
//   "pair") split the external product by prime and meet twice per step (named barrier
//   1 + slot, 64 threads).  Both primes run the same code (the prime is a runtime value),
//   which keeps the kernel inside the instruction caches.
//   Key chunks (one chunk = row r of BSK_i for one prime, both TRLWE components, 8 KB)
//   flow through a ring of BR_RING shared-memory slots per prime.  Lane 0 of the slot-0
//   warp of each prime is also that prime's producer: it issues cp.async.bulk copies
//   (TMA engine) completing on "full" mbarriers.  After consuming chunk q it issues chunk
//   q + BR_LOOKAHEAD into the slot of chunk q + BR_LOOKAHEAD - BR_RING = q - 2, which is
//   free once all BR_SLOTS consumers have arrived on its "empty" mbarrier: the producer
//   waits only for a slot that is more than one chunk behind it.  All waits are bounded
//   (LP_ETIMEOUT on expiry).
//
// Per step and pair: both warps rotate/subtract ACC (shared memory) and decompose it;
// each warp forward-transforms the 6 digit polynomials modulo its prime and multiplies
// them with the key chunk, accumulating both output components in 64-bit registers
// (key stored as NTT(b) N^-1 2^32 mod p, one Montgomery reduction per coefficient);
// it inverse-transforms the 2 sums together (their butterflies interleaved).  The pair then
// swaps half of its residues through shared memory: the prime-0 warp recombines component 0
// (centred CRT) and adds it to ACC, the prime-1 warp component 1.
//
// The file also holds the kernels for levels too small to fill the GPU (see their sections):
// br_split_kernel spreads one ciphertext over 12 warps, br_pair_kernel over a cluster of two
// CTAs and br_quad_kernel over a cluster of four; launch_br picks one per level.
#include "common.cuh"
#include "kernels.h"
#include "ks_device.cuh"
#include "ntt.cuh"

namespace lp {

constexpr int BR_SLOTS = 4;
constexpr int BR_RING = 3;
constexpr int BR_LOOKAHEAD = 1;                          // chunks issued ahead of the one consumed
static_assert(BR_LOOKAHEAD >= 1 && BR_LOOKAHEAD < BR_RING, "chunk q + L reuses the slot of chunk q + L - R < q");
constexpr int BR_COMPUTE_WARPS = 2 * BR_SLOTS;
constexpr int BR_THREADS = BR_COMPUTE_WARPS * 32;
constexpr int CHUNK_WORDS = 2 * RING_N;                 // one (i, prime, row) chunk
constexpr uint32_t CHUNK_BYTES = CHUNK_WORDS * 4u;
constexpr int ABAR_STRIDE_MAX = 1024;                    // u16 entries per job (>= n + 1)

struct __align__(16) BrSmem {
    uint32_t ring[2][BR_RING][CHUNK_WORDS];              // 48 KB
    uint32_t ubuf[BR_COMPUTE_WARPS][RING_N];             // 32 KB: rounded differences, per warp
    uint32_t acc[BR_SLOTS][2][RING_N];                   // 32 KB
    uint32_t xch[BR_SLOTS][2][RING_N];                   // 32 KB
    uint32_t tbuf[BR_COMPUTE_WARPS][32 * 33];            // 33 KB
    uint2 tw[2][2][LANE_TW * 32];                        // 31 KB [prime][dir]
    uint16_t abar[BR_SLOTS][ABAR_STRIDE_MAX];            // 8 KB
    uint64_t full_bar[2][BR_RING];
    uint64_t empty_bar[2][BR_RING];
    int abort;
    int claim;                                           // group handed to this CTA (persistent executor)
};

struct BrArgs {
    const uint16_t *abar;      // [jobs][abar_stride]: abar_0 .. abar_{n-1}, bbar at index n
    uint32_t *ext;             // [jobs][EXT_STRIDE]: extracted a'_0 .. a'_{N-1}, b' at index N
    const uint32_t *bsk_hat;   // [n][2 primes][ROWS][2][N] (transform domain, chunk layout)
    const uint2 *tw_lane;      // [2][2][LANE_TW * 32]
    int n;
    int abar_stride;
    int jobs;
    uint32_t mu;               // test-vector value (1/8)
    int *err;
};

size_t br_smem_bytes() { return sizeof(BrSmem); }

// Chunk stream of one prime: chunk q of a CTA is row q % ROWS of BSK_((q / ROWS) % n),
// for q < total (= the CTA's groups * n * ROWS).
struct Producer {
    const uint32_t *bsk_hat;
    uint32_t total;
    uint32_t issued;
    int n;
    int pi;
};

__device__ __forceinline__ void produce(BrSmem &sm, Producer &pr, uint32_t upto)
{
    // Issue chunks [pr.issued, min(upto, total)) into their ring slots; the slot of chunk q
    // is free once chunk q - BR_RING was released by all consumers.
    while (pr.issued < upto && pr.issued < pr.total) {
        const uint32_t q = pr.issued;
        const uint32_t s = q % BR_RING;
        if (q >= (uint32_t)BR_RING) {
            const uint32_t par = ((q - BR_RING) / BR_RING) & 1u;
            if (!mbar_wait_bounded(&sm.empty_bar[pr.pi][s], par, &sm.abort)) {
                *reinterpret_cast<volatile int *>(&sm.abort) = 1;
                return;
            }
        }
        const int r = (int)(q % ROWS);
        const int i = (int)((q / ROWS) % (uint32_t)pr.n);
        mbar_arrive_expect_tx(&sm.full_bar[pr.pi][s], CHUNK_BYTES);
        const uint32_t *src = pr.bsk_hat + ((size_t)(i * 2 + pr.pi) * ROWS + r) * CHUNK_WORDS;
        bulk_copy_g2s(sm.ring[pr.pi][s], src, CHUNK_BYTES, &sm.full_bar[pr.pi][s]);
        pr.issued++;
    }
}

// Wait (bounded) until every chunk issued by this producer has landed in shared memory.
__device__ __forceinline__ bool drain(BrSmem &sm, const Producer &pr)
{
    bool ok = true;
    const uint32_t first = pr.issued > (uint32_t)BR_RING ? pr.issued - BR_RING : 0u;
    volatile int never = 0;
    for (uint32_t q = first; q < pr.issued; q++)
        ok &= mbar_wait_bounded(&sm.full_bar[pr.pi][q % BR_RING], (q / BR_RING) & 1u, &never);
    return ok;
}

// Wait for the next key chunk of this prime, multiply-accumulate the transformed digit x into
// both output components (64-bit sums), release the chunk, and (producer lane) refill the ring.
__device__ __forceinline__ void mac_chunk(BrSmem &sm, int pi, int lane, bool work, bool &ok, uint32_t &cseq,
                                          const uint32_t (&x)[32], unsigned long long (&acc0)[32],
                                          unsigned long long (&acc1)[32], Producer &pr, bool producer)
{
    const uint32_t rs = cseq % BR_RING;
    const uint32_t par = (cseq / BR_RING) & 1u;
    if (ok && !mbar_wait_bounded(&sm.full_bar[pi][rs], par, &sm.abort)) {
        ok = false;
        if (lane == 0) *reinterpret_cast<volatile int *>(&sm.abort) = 1;
    }
    if (work && ok) {
        // x in [0, 22p), key in [0, p): six products sum below 132 p^2 < 2^64.
        const uint4 *ch0 = reinterpret_cast<const uint4 *>(sm.ring[pi][rs]);
        const uint4 *ch1 = reinterpret_cast<const uint4 *>(sm.ring[pi][rs] + RING_N);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint4 b0 = ch0[q * 32 + lane];
            const uint4 b1 = ch1[q * 32 + lane];
            const uint32_t bb0[4] = {b0.x, b0.y, b0.z, b0.w};
            const uint32_t bb1[4] = {b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int k = 4 * q + e;
                acc0[k] += (unsigned long long)x[k] * bb0[e];
                acc1[k] += (unsigned long long)x[k] * bb1[e];
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        mbar_arrive(&sm.empty_bar[pi][rs]);
        // Issue chunk cseq + BR_LOOKAHEAD (its slot held chunk cseq + BR_LOOKAHEAD - BR_RING).
        if (producer) produce(sm, pr, cseq + 1 + BR_LOOKAHEAD);
    }
    __syncwarp();
    cseq++;
}

// One external-product half for prime pi: rotate/decompose ACC, 6 forward NTTs each
// followed by the 64-bit multiply-accumulate with the streamed key chunk, 2 inverse NTTs.
// On return `mine` holds component pi of the product mod p (in [0, p), layout A) and
// component 1 - pi has been written to xch for the partner warp.
__device__ __forceinline__ bool external_product(BrSmem &sm, int slot, int lane, int pi, const PrimeK &K, int ab,
                                                 bool work, uint32_t &cseq, uint32_t (&mine)[32], uint32_t *tbuf,
                                                 Producer &pr, bool producer)
{
    const uint2 *twf = sm.tw[pi][0];
    const uint2 *twi = sm.tw[pi][1];
    bool ok = true;
    uint32_t *U = sm.ubuf[2 * slot + pi];
    uint32_t x[32];
    unsigned long long acc0[32], acc1[32];
#pragma unroll
    for (int k = 0; k < 32; k++) {
        acc0[k] = 0ull;
        acc1[k] = 0ull;
    }
#pragma unroll 1
    for (int c = 0; c < 2; c++) {
        if (work) {
            const uint32_t *A = sm.acc[slot][c];
#pragma unroll
            for (int k = 0; k < 32; k++) {
                const int j = lane + 32 * k;
                const int idx = (j - ab) & (2 * RING_N - 1);
                uint32_t v = A[idx & (RING_N - 1)];
                v = (idx & RING_N) ? (0u - v) : v;
                U[j] = v - A[j] + GADGET_OFF;
            }
        }
        // digit + 512 in [0, 1024), shifted by p - 512 into [p - 512, p + 512) = digit mod p.
#pragma unroll 1
        for (int p = 0; p < LG; p++) {
            const int sh = 22 - BGBIT * p;
            if (work) {
#pragma unroll
                for (int k = 0; k < 32; k++) x[k] = ((U[lane + 32 * k] >> sh) & 1023u) + (K.p - 512u);
                ntt_fwd<false>(x, tbuf, twf, lane, pi, K);
            }
            mac_chunk(sm, pi, lane, work, ok, cseq, x, acc0, acc1, pr, producer);
        }
    }
    if (work && ok) {
        // Montgomery reduction of sums below 132 p^2 leaves [0, 132 p^2 / 2^32 + p) within [0, 7p)
        // (p < 2^32 / 22); two conditional subtractions (ALU pipe, not the multiplier) bring
        // it into [0, 2p).  Both components are then inverse-transformed together.
        uint32_t y[2][32];
#pragma unroll
        for (int k = 0; k < 32; k++) {
#pragma unroll
            for (int q = 0; q < 2; q++) {
                uint32_t v = redc64(q == 0 ? acc0[k] : acc1[k], K);
                v = umin_u32(v, v - 2u * K.p2);
                y[q][k] = umin_u32(v, v - K.p2);
            }
        }
        ntt_inv_multi<2>(y, tbuf, twi, lane, pi, K);
#pragma unroll
        for (int k = 0; k < 32; k++) {
            const uint32_t r0 = umin_u32(y[0][k], y[0][k] - K.p), r1 = umin_u32(y[1][k], y[1][k] - K.p);
            mine[k] = pi == 0 ? r0 : r1;
            sm.xch[slot][1 - pi][lane + 32 * k] = pi == 0 ? r1 : r0;
        }
    }
    return ok;
}

__device__ __forceinline__ uint32_t crt_lift(uint32_t x0, uint32_t x1)
{
    // V = x0 + p0 t, t = (x1 - x0) p0^-1 mod p1, V in [0, p0 p1); centred lift mod 2^32.
    constexpr uint64_t PP = (uint64_t)PRIME0 * (uint64_t)PRIME1;
    const uint2 inv = c_crt;
    const uint32_t x0r = umin_u32(x0, x0 - PRIME1);
    const uint32_t d = x1 - x0r + PRIME1;
    uint32_t t = shoup_mul_r(d, inv.x, inv.y, PRIME1);
    t = umin_u32(t, t - PRIME1);
    const uint64_t V = (uint64_t)PRIME0 * t + x0;
    uint32_t r = (uint32_t)V;
    if (V > (PP - 1) / 2) r -= (uint32_t)PP;
    return r;
}

// Next group of a CTA that pulls its work from a device-side counter (all threads call it at
// the same point; the counter hands each group to exactly one CTA).
__device__ __forceinline__ int claim_group(BrSmem &sm, uint32_t *ctr)
{
    __syncthreads();
    if (threadIdx.x == 0) sm.claim = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    return sm.claim;
}

// Loop of one compute warp over its CTA's ciphertext groups: groups blockIdx.x, + gridDim.x, ...
// (Dyn = false), or groups claimed one at a time from *claim (Dyn = true: the persistent
// executor).  A claimed group's key stream starts when it is claimed; an abort is then decided
// CTA-wide at the group boundary.  Returns false after an abort.
template <bool Dyn>
__device__ __forceinline__ bool compute_warp(BrSmem &sm, const BrArgs &a, int warp, int lane, int ngroups,
                                             uint32_t *claim = nullptr, uint32_t *progress = nullptr)
{
    const int slot = warp >> 1;
    const int pi = warp & 1;
    const int bar_id = 1 + slot;
    const int n = a.n;
    const PrimeK K = prime_k(pi);
    uint32_t *tbuf = sm.tbuf[warp];
    uint32_t cseq = 0;
    uint32_t mine[32];
    const bool producer = slot == 0 && lane == 0;
    Producer pr;
    pr.bsk_hat = a.bsk_hat;
    pr.n = n;
    pr.pi = pi;
    pr.issued = 0;
    int g;
    if (Dyn) {
        pr.total = 0;
        g = claim_group(sm, claim);
    } else {
        const int my_groups = (int)blockIdx.x < ngroups ? (ngroups - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
        pr.total = (uint32_t)my_groups * (uint32_t)n * ROWS;
        if (producer) produce(sm, pr, BR_RING);
        g = blockIdx.x;
    }
    bool failed = false;
    while (g < ngroups) {
        if (Dyn) {
            pr.total += (uint32_t)n * ROWS;
            if (producer) produce(sm, pr, cseq + BR_RING);
        }
        const int job = g * BR_SLOTS + slot;
        const bool active = job < a.jobs;
        if (pi == 1 && active) {
            const uint16_t *src = a.abar + (size_t)job * a.abar_stride;
            for (int i = lane; i <= n; i += 32) sm.abar[slot][i] = src[i];
            __syncwarp();
            const int bb = sm.abar[slot][n];
            // ACC = (0, X^-bbar v): coefficient j of X^-k v is v (j + k < N) or -v.
            for (int j = lane; j < RING_N; j += 32) {
                sm.acc[slot][0][j] = 0u;
                const int e = (j + bb) & (2 * RING_N - 1);
                sm.acc[slot][1][j] = (e & RING_N) ? (0u - a.mu) : a.mu;
            }
        }
        bool aborted = bar_red_or(bar_id, 64, false);
        for (int i = 0; i < n && !aborted; i++) {
            const int ab = active ? (int)sm.abar[slot][i] : 0;
            const bool work = ab != 0;
            const bool ok = external_product(sm, slot, lane, pi, K, ab, work, cseq, mine, tbuf, pr, producer);
            aborted = bar_red_or(bar_id, 64, !ok || *reinterpret_cast<volatile int *>(&sm.abort) != 0);
            if (aborted) break;
            if (work) {
                // Component pi: residue mod p_pi in `mine`, the other prime's residue in xch.
                uint32_t *A = sm.acc[slot][pi];
                const uint32_t *X = sm.xch[slot][pi];
#pragma unroll
                for (int k = 0; k < 32; k++) {
                    const int j = lane + 32 * k;
                    const uint32_t x0 = pi == 0 ? mine[k] : X[j];
                    const uint32_t x1 = pi == 0 ? X[j] : mine[k];
                    A[j] += crt_lift(x0, x1);
                }
            }
            aborted = bar_red_or(bar_id, 64, false);
        }
        if (aborted) {
            if (lane == 0 && pi == 1) atomicOr(a.err, DEV_ERR_TIMEOUT);
        } else if (pi == 1 && active) {
            // Sample extraction: a'_0 = A_0, a'_j = -A_{N-j}, b' = B_0.
            uint32_t *dst = a.ext + (size_t)job * EXT_STRIDE;
            for (int j = lane; j < RING_N; j += 32)
                dst[j] = j == 0 ? sm.acc[slot][0][0] : 0u - sm.acc[slot][0][RING_N - j];
            if (lane == 0) dst[RING_N] = sm.acc[slot][1][0];
        }
        if (Dyn) {
            if (__syncthreads_or(aborted)) {
                failed = true;
                break;
            }
            if (threadIdx.x == 0 && progress) atomicAdd(progress, 1u);
            g = claim_group(sm, claim);
        } else {
            if (aborted) {
                failed = true;
                break;
            }
            g += gridDim.x;
        }
    }
    // No bulk copy may still be in flight when the CTA exits.
    if (producer && !drain(sm, pr)) {
        atomicOr(a.err, DEV_ERR_TIMEOUT);
        failed = true;
    }
    return !failed;
}

__global__ void __launch_bounds__(BR_THREADS, 1) br_kernel(BrArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    BrSmem &sm = *reinterpret_cast<BrSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    for (int i = threadIdx.x; i < 2 * 2 * LANE_TW * 32; i += blockDim.x) (&sm.tw[0][0][0])[i] = a.tw_lane[i];
    if (threadIdx.x == 0) {
        for (int p = 0; p < 2; p++)
            for (int s = 0; s < BR_RING; s++) {
                mbar_init(&sm.full_bar[p][s], 1);
                mbar_init(&sm.empty_bar[p][s], BR_SLOTS);
            }
        sm.abort = 0;
        mbar_fence_init();
    }
    __syncthreads();
    const int ngroups = (a.jobs + BR_SLOTS - 1) / BR_SLOTS;
    compute_warp<false>(sm, a, warp, lane, ngroups);
}

// ---------------------------------------------------------------------------------
// Split blind rotation: one ciphertext per CTA, its external product spread over
// SPLIT_WARPS = 12 warps, one per (prime, digit row).  It shortens one CMux step about four
// times against br_kernel (whose warp pair runs all 6 forward and 2 inverse transforms of a
// ciphertext in sequence), for levels too small to fill the GPU with groups of BR_SLOTS.
//
// Per step: every warp rotates/decomposes its own digit row r of ACC, forward-transforms it
// modulo its prime and parks the transformed row (lazy, in [0, 22p)) in its transpose buffer.
// After a barrier, warps (pi, c, h) for the 8 combinations of prime, output component and half
// of the transform's registers sum the six rows' products with their key rows in 64 bits
// (x < 22p and key < p: six products stay below 132 p^2 < 2^64) and reduce each sum once
// (Montgomery, then two conditional subtractions: [0, 2p)), keeping it in registers.  After a
// second barrier, each warp refills its key buffer with the next step's row (cp.async.bulk,
// bounded mbarrier wait at the next step), and the two warps of each (pi, c) inverse-transform
// component c modulo prime pi together (ntt_inv_2warp); after a third, all threads recombine
// both primes (centred CRT) into ACC.  Steps with abar_i = 0 leave ACC unchanged and are
// skipped (CTA-uniform), as in br_kernel.
// ---------------------------------------------------------------------------------
constexpr int SPLIT_WARPS = 2 * ROWS;
constexpr int SPLIT_THREADS = SPLIT_WARPS * 32;

struct __align__(16) SplitSmem {
    uint32_t key[SPLIT_WARPS][CHUNK_WORDS];             // 96 KB: this step's row per warp
    uint32_t tbuf[SPLIT_WARPS][32 * 33];                 // 50 KB: transposes, then the parked row
    uint2 tw[2][2][LANE_TW * 32];                        // 31 KB [prime][dir]
    uint32_t part[2][2][RING_N];                         // 16 KB [prime][component]
    uint32_t acc[2][RING_N];                             // 8 KB
    uint16_t abar[ABAR_STRIDE_MAX];                      // 2 KB
    uint64_t bar[SPLIT_WARPS];
    int abort;
};

size_t br_split_smem_bytes() { return sizeof(SplitSmem); }

__device__ __forceinline__ void split_issue(SplitSmem &sm, const uint32_t *bsk_hat, int w, int pi, int r, int i)
{
    mbar_arrive_expect_tx(&sm.bar[w], CHUNK_BYTES);
    bulk_copy_g2s(sm.key[w], bsk_hat + ((size_t)(i * 2 + pi) * ROWS + r) * CHUNK_WORDS, CHUNK_BYTES, &sm.bar[w]);
}

// Inverse transform of one polynomial by two warps: warp h holds registers 16 h .. 16 h + 15
// of layout B (lane t, register k = index 32 t + k), 16 values y[i] per lane, in [0, 2p).
// Stages 9..6 pair registers within a half; stage 5 (pairs k, k + 16) and stage 0 (layout A,
// pairs k', k' + 16) cross the halves, so the warps swap 8 values per lane through X (512
// words) and each computes half of those butterflies; the layout B -> A transpose goes through
// TB (32 x 33 words).  The warps meet at named barrier bar_id (64 threads).  On return y[i],
// in [0, 2p), is the natural-order coefficient lane + 32 k' with k' = 8 h + i (i < 8) or
// 16 + 8 h + (i - 8).
__device__ __forceinline__ void ntt_inv_2warp(uint32_t (&y)[16], int h, int lane, int pi, const PrimeK &K,
                                              const uint2 *twi, uint32_t *TB, uint32_t *X, int bar_id)
{
#pragma unroll
    for (int s = 9; s >= 6; s--) {
        const int L = 16 >> (s - 5);
        const int base = (1 << (s - 5)) - 1;
#pragma unroll
        for (int bl = 0; bl < 16 / (2 * L); bl++) {
            const uint2 z = twi[(base + (16 * h) / (2 * L) + bl) * 32 + lane];
#pragma unroll
            for (int o = 0; o < L; o++) bfly_inv(y[bl * 2 * L + o], y[bl * 2 * L + o + L], z.x, z.y, K);
        }
    }
    // Stage 5: warp 0 computes the pairs (k, k + 16) for k < 8, warp 1 those for 8 <= k < 16.
    uint32_t *out = X + h * 256;
    const uint32_t *in = X + (1 - h) * 256;
#pragma unroll
    for (int i = 0; i < 8; i++) out[i * 32 + lane] = h == 0 ? y[8 + i] : y[i];
    bar_red_or(bar_id, 64, false);
    {
        const uint2 z = twi[lane];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            uint32_t a = h == 0 ? y[i] : in[i * 32 + lane];
            uint32_t b = h == 0 ? in[i * 32 + lane] : y[8 + i];
            bfly_inv(a, b, z.x, z.y, K);
            y[i] = a;
            y[8 + i] = b;
        }
    }
    // Layout B -> A: values at registers 8 h + i and 16 + 8 h + i of lane t.
#pragma unroll
    for (int i = 0; i < 8; i++) {
        TB[lane * 33 + 8 * h + i] = y[i];
        TB[lane * 33 + 16 + 8 * h + i] = y[8 + i];
    }
    bar_red_or(bar_id, 64, false);
#pragma unroll
    for (int i = 0; i < 16; i++) y[i] = TB[(16 * h + i) * 33 + lane];
    // Stages 4..1 within the half (registers k' = 16 h + i of layout A).
#pragma unroll
    for (int s = 4; s >= 1; s--) {
        const int D = 16 >> s;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            if (i & D) continue;
            const uint2 z = c_tw[pi][1][(1 << s) + ((16 * h + i) >> (5 - s))];
            bfly_inv(y[i], y[i + D], z.x, z.y, K);
        }
    }
    // Stage 0 (pairs k', k' + 16), split as stage 5.  X was last read before the transpose's
    // barrier, so it may be written again.
#pragma unroll
    for (int i = 0; i < 8; i++) out[i * 32 + lane] = h == 0 ? y[8 + i] : y[i];
    bar_red_or(bar_id, 64, false);
    {
        const uint2 z = c_tw[pi][1][1];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            uint32_t a = h == 0 ? y[i] : in[i * 32 + lane];
            uint32_t b = h == 0 ? in[i * 32 + lane] : y[8 + i];
            bfly_inv(a, b, z.x, z.y, K);
            y[i] = a;
            y[8 + i] = b;
        }
    }
}

// Forward transform of one polynomial by two warps (the mirror of ntt_inv_2warp).  Warp h holds
// the layout-A registers k = 2 i + h (i < 16), values in [0, 2p).  Stages 0..3 pair registers of
// the same parity, inside the warp; stage 4 pairs 2 i with 2 i + 1 across the warps, which swap
// 8 values per lane through X (512 words) and compute its butterflies i < 8 (warp 0) and i >= 8
// (warp 1), leaving warp h with registers 16 h .. 16 h + 15.  The layout A -> B transpose goes
// through TB (32 x 33 words, written by both warps), after which warp h holds the layout-B
// registers k' = 2 i + h: stages 5..8 are local and stage 9 crosses as stage 4 did.  The warps
// meet at named barrier bar_id (64 threads).  On return y[m], in [0, 22p), is layout-B register
// 16 h + m; TB and X are free for the caller once both warps have returned.
__device__ __forceinline__ void ntt_fwd_2warp(uint32_t (&y)[16], int h, int lane, int pi, const PrimeK &K,
                                              const uint2 *twf, uint32_t *TB, uint32_t *X, int bar_id)
{
#pragma unroll
    for (int s = 0; s < 4; s++) {
        const int D2 = 8 >> s;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            if (i & D2) continue;
            const uint2 z = c_tw[pi][0][(1 << s) + (i >> (4 - s))];
            bfly_fwd(y[i], y[i + D2], z.x, z.y, K);
        }
    }
    uint32_t *out = X + h * 256;
    const uint32_t *in = X + (1 - h) * 256;
    uint32_t t[16];
    // Stage 4: butterfly ii pairs register 2 ii (warp 0's y[ii]) with 2 ii + 1 (warp 1's y[ii]).
#pragma unroll
    for (int i = 0; i < 8; i++) out[i * 32 + lane] = h == 0 ? y[8 + i] : y[i];
    bar_red_or(bar_id, 64, false);
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint2 z = c_tw[pi][0][16 + 8 * h + i];
        uint32_t a = h == 0 ? y[i] : in[i * 32 + lane];
        uint32_t b = h == 0 ? in[i * 32 + lane] : y[8 + i];
        bfly_fwd(a, b, z.x, z.y, K);
        t[2 * i] = a;
        t[2 * i + 1] = b;
    }
    // Layout A -> B: registers 16 h + m of layout A in, registers 2 i + h of layout B out.
#pragma unroll
    for (int m = 0; m < 16; m++) TB[(16 * h + m) * 33 + lane] = t[m];
    bar_red_or(bar_id, 64, false);
#pragma unroll
    for (int i = 0; i < 16; i++) y[i] = TB[lane * 33 + 2 * i + h];
#pragma unroll
    for (int s = 5; s < 9; s++) {
        const int L = 16 >> (s - 5), L2 = L / 2;
        const int base = (1 << (s - 5)) - 1;
#pragma unroll
        for (int b = 0; b < 16 / L; b++) {
            const uint2 z = twf[(base + b) * 32 + lane];
#pragma unroll
            for (int o = 0; o < L2; o++) bfly_fwd(y[b * L + o], y[b * L + o + L2], z.x, z.y, K);
        }
    }
    // Stage 9, split as stage 4.  X was last read before the transpose's barrier.
#pragma unroll
    for (int i = 0; i < 8; i++) out[i * 32 + lane] = h == 0 ? y[8 + i] : y[i];
    bar_red_or(bar_id, 64, false);
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint2 z = twf[(15 + 8 * h + i) * 32 + lane];
        uint32_t a = h == 0 ? y[i] : in[i * 32 + lane];
        uint32_t b = h == 0 ? in[i * 32 + lane] : y[8 + i];
        bfly_fwd(a, b, z.x, z.y, K);
        t[2 * i] = a;
        t[2 * i + 1] = b;
    }
#pragma unroll
    for (int m = 0; m < 16; m++) y[m] = t[m];
}

// One stage of a four-warp transform whose pairs cross two warps (this one, w, and `partner`):
// each holds 8 values, the low-side warp (low) the pairs' first operands; they swap 4 values per
// lane through R (4 warps x 128 words) and compute 4 butterflies each, the low side the pairs
// of its registers 0..3, with twiddle z[j] for its butterfly j.  On return registers 0..3 hold
// the pairs' first outputs, 4..7 the second.
template <bool Fwd>
__device__ __forceinline__ void cross4(uint32_t (&y)[8], int w, int partner, bool low, int lane, const uint2 (&z)[4],
                                       const PrimeK &K, uint32_t *R, int bar_id)
{
    uint32_t *out = R + w * 128;
    const uint32_t *in = R + partner * 128;
#pragma unroll
    for (int j = 0; j < 4; j++) out[j * 32 + lane] = low ? y[4 + j] : y[j];
    bar_red_or(bar_id, 128, false);
    uint32_t t[8];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        uint32_t a = low ? y[j] : in[j * 32 + lane];
        uint32_t b = low ? in[j * 32 + lane] : y[4 + j];
        if (Fwd)
            bfly_fwd(a, b, z[j].x, z[j].y, K);
        else
            bfly_inv(a, b, z[j].x, z[j].y, K);
        t[j] = a;
        t[4 + j] = b;
    }
#pragma unroll
    for (int m = 0; m < 8; m++) y[m] = t[m];
}

// Forward transform of one polynomial by four warps.  Warp w = 2 hb + w0 holds the layout-A
// registers 4 i + w (i < 8), values in [0, 2p).  Stages 0..2 are local; stage 3 (pairs k, k + 2)
// crosses warps w and w ^ 2 and stage 4 (k, k + 1) warps w and w ^ 1 (cross4, each through its
// own half of X, 1024 words), after which warp w holds registers 16 hb + 4 j + 2 w0 + e at
// y[4 e + j].  The layout A -> B transpose goes through TB (32 x 33 words, all four warps),
// giving warp w the layout-B registers 4 i + w; stages 5..7 are local and stages 8 and 9 cross
// as 3 and 4 did.  The warps meet at named barrier bar_id (128 threads).  On return y[4 e + j],
// in [0, 22p), is layout-B register 16 hb + 4 j + 2 w0 + e; TB and X are free for the caller
// once all four warps have returned.
__device__ __forceinline__ void ntt_fwd_4warp(uint32_t (&y)[8], int w, int lane, int pi, const PrimeK &K,
                                              const uint2 *twf, uint32_t *TB, uint32_t *X, int bar_id)
{
    const int hb = w >> 1, w0 = w & 1;
#pragma unroll
    for (int s = 0; s < 3; s++) {
        const int D4 = 4 >> s;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            if (i & D4) continue;
            const uint2 z = c_tw[pi][0][(1 << s) + (i >> (3 - s))];
            bfly_fwd(y[i], y[i + D4], z.x, z.y, K);
        }
    }
    uint2 z[4];
#pragma unroll
    for (int j = 0; j < 4; j++) z[j] = c_tw[pi][0][8 + 4 * hb + j];
    cross4<true>(y, w, w ^ 2, hb == 0, lane, z, K, X, bar_id);
#pragma unroll
    for (int j = 0; j < 4; j++) z[j] = c_tw[pi][0][16 + 8 * hb + 2 * j + w0];
    cross4<true>(y, w, w ^ 1, w0 == 0, lane, z, K, X + 512, bar_id);
#pragma unroll
    for (int e = 0; e < 2; e++)
#pragma unroll
        for (int j = 0; j < 4; j++) TB[(16 * hb + 4 * j + 2 * w0 + e) * 33 + lane] = y[4 * e + j];
    bar_red_or(bar_id, 128, false);
#pragma unroll
    for (int i = 0; i < 8; i++) y[i] = TB[lane * 33 + 4 * i + w];
#pragma unroll
    for (int s = 5; s < 8; s++) {
        const int L = 16 >> (s - 5), L2 = L / 2, L4 = L / 4;
        const int base = (1 << (s - 5)) - 1;
#pragma unroll
        for (int b = 0; b < 8 / L2; b++) {
            const uint2 zz = twf[(base + b) * 32 + lane];
#pragma unroll
            for (int o = 0; o < L4; o++) bfly_fwd(y[b * L2 + o], y[b * L2 + o + L4], zz.x, zz.y, K);
        }
    }
    // Each half of X was last read before the barrier that follows its next writer's barrier.
#pragma unroll
    for (int j = 0; j < 4; j++) z[j] = twf[(7 + 4 * hb + j) * 32 + lane];
    cross4<true>(y, w, w ^ 2, hb == 0, lane, z, K, X, bar_id);
#pragma unroll
    for (int j = 0; j < 4; j++) z[j] = twf[(15 + 8 * hb + 2 * j + w0) * 32 + lane];
    cross4<true>(y, w, w ^ 1, w0 == 0, lane, z, K, X + 512, bar_id);
}

// Inverse transform of one polynomial by four warps.  Warp w = 2u + v holds layout-B registers
// 8 w .. 8 w + 7 (bit 4 of the register index is u, bit 3 is v), values in [0, 2p).  Stages
// 9..7 are local; stage 6 (pairs k, k + 8) crosses warps w and w ^ 1, stage 5 (k, k + 16) warps
// w and w ^ 2 (cross4, each through its own half of X, 1024 words), after which warp w holds
// registers 16 c + 8 u + 4 v + j at y[4 c + j].  The layout B -> A transpose goes through TB
// (32 x 33 words, all four warps), giving warp w the layout-A registers 8 w .. 8 w + 7 again;
// stages 4..2 are local and stages 1 and 0 cross as 6 and 5 did.  The warps meet at named
// barrier bar_id (128 threads).  On return y[4 c + j], in [0, 2p), is the natural-order
// coefficient lane + 32 (16 c + 8 u + 4 v + j).
__device__ __forceinline__ void ntt_inv_4warp(uint32_t (&y)[8], int w, int lane, int pi, const PrimeK &K,
                                              const uint2 *twi, uint32_t *TB, uint32_t *X, int bar_id)
{
    const int u = w >> 1, v = w & 1;
#pragma unroll
    for (int s = 9; s >= 7; s--) {
        const int L = 16 >> (s - 5);
        const int base = (1 << (s - 5)) - 1;
#pragma unroll
        for (int b = 0; b < 8 / (2 * L); b++) {
            const uint2 zz = twi[(base + 4 * w / L + b) * 32 + lane];
#pragma unroll
            for (int o = 0; o < L; o++) bfly_inv(y[b * 2 * L + o], y[b * 2 * L + o + L], zz.x, zz.y, K);
        }
    }
    uint2 z[4];
#pragma unroll
    for (int j = 0; j < 4; j++) z[j] = twi[(1 + u) * 32 + lane];
    cross4<false>(y, w, w ^ 1, v == 0, lane, z, K, X, bar_id);
#pragma unroll
    for (int j = 0; j < 4; j++) z[j] = twi[lane];
    cross4<false>(y, w, w ^ 2, u == 0, lane, z, K, X + 512, bar_id);
#pragma unroll
    for (int m = 0; m < 8; m++) TB[lane * 33 + 16 * (m >> 2) + 8 * u + 4 * v + (m & 3)] = y[m];
    bar_red_or(bar_id, 128, false);
#pragma unroll
    for (int i = 0; i < 8; i++) y[i] = TB[(8 * w + i) * 33 + lane];
#pragma unroll
    for (int s = 4; s >= 2; s--) {
        const int D = 16 >> s;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            if (i & D) continue;
            const uint2 zz = c_tw[pi][1][(1 << s) + ((8 * w + i) >> (5 - s))];
            bfly_inv(y[i], y[i + D], zz.x, zz.y, K);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) z[j] = c_tw[pi][1][2 + u];
    cross4<false>(y, w, w ^ 1, v == 0, lane, z, K, X, bar_id);
#pragma unroll
    for (int j = 0; j < 4; j++) z[j] = c_tw[pi][1][1];
    cross4<false>(y, w, w ^ 2, u == 0, lane, z, K, X + 512, bar_id);
}

// Sums are stored in transform (layout B) order, index 32 lane + k swizzled to
// 32 lane + (k ^ lane) so that a warp's 32 lanes hit 32 different banks.
__device__ __forceinline__ int split_pos(int lane, int k) { return lane * 32 + (k ^ lane); }

__global__ void __launch_bounds__(SPLIT_THREADS, 1) br_split_kernel(BrArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    SplitSmem &sm = *reinterpret_cast<SplitSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pi = warp / ROWS, r = warp % ROWS;
    const int c_in = r / LG, p_dig = r % LG;
    const int n = a.n;
    const PrimeK K = prime_k(pi);
    // Roles after the forward transforms: warp 4 mpi + 2 mc + mh (< 8) sums the products of
    // (prime mpi, output component mc) for half mh of the registers, then inverse-transforms
    // that half together with its partner warp.
    const int mpi = (warp >> 2) & 1, mc = (warp >> 1) & 1, mh = warp & 1;
    const PrimeK MK = prime_k(mpi);

    for (int i = threadIdx.x; i < 2 * 2 * LANE_TW * 32; i += blockDim.x) (&sm.tw[0][0][0])[i] = a.tw_lane[i];
    if (threadIdx.x == 0) {
        for (int w = 0; w < SPLIT_WARPS; w++) mbar_init(&sm.bar[w], 1);
        sm.abort = 0;
        mbar_fence_init();
    }
    __syncthreads();

    uint32_t *tbuf = sm.tbuf[warp];
    uint32_t phase = 0;          // completed uses of this warp's barrier
    bool pending = false;        // a copy into this warp's key buffer is in flight
    bool aborted = false;
    for (int job = blockIdx.x; job < a.jobs && !aborted; job += gridDim.x) {
        const uint16_t *src = a.abar + (size_t)job * a.abar_stride;
        for (int i = threadIdx.x; i <= n; i += blockDim.x) sm.abar[i] = src[i];
        __syncthreads();
        const int bb = sm.abar[n];
        for (int j = threadIdx.x; j < RING_N; j += blockDim.x) {
            sm.acc[0][j] = 0u;
            const int e = (j + bb) & (2 * RING_N - 1);
            sm.acc[1][j] = (e & RING_N) ? (0u - a.mu) : a.mu;
        }
        if (n > 0) {
            if (lane == 0) split_issue(sm, a.bsk_hat, warp, pi, r, 0);
            pending = true;   // every lane tracks the barrier phase
        }
        __syncthreads();
        for (int i = 0; i < n; i++) {
            const int ab = sm.abar[i];
            // This step's key row has landed (bounded wait); the refill comes after the sums.
            bool ok = true;
            if (pending) {
                ok = mbar_wait_bounded(&sm.bar[warp], phase & 1u, &sm.abort);
                if (ok) {
                    phase++;
                    pending = false;   // else the copy stays pending for the drain at exit
                }
            }
            if (!ok && lane == 0) *reinterpret_cast<volatile int *>(&sm.abort) = 1;
            if (ab != 0 && ok) {
                const uint32_t *A = sm.acc[c_in];
                const int sh = 32 - BGBIT * (p_dig + 1);
                uint32_t x[32];
#pragma unroll
                for (int k = 0; k < 32; k++) {
                    const int j = lane + 32 * k;
                    const int idx = (j - ab) & (2 * RING_N - 1);
                    uint32_t v = A[idx & (RING_N - 1)];
                    v = (idx & RING_N) ? (0u - v) : v;
                    const uint32_t u = v - A[j] + GADGET_OFF;
                    x[k] = ((u >> sh) & 1023u) + (K.p - 512u);
                }
                ntt_fwd<false>(x, tbuf, sm.tw[pi][0], lane, pi, K);
                // Park the row: register k of lane t at [k][t] (the transform's last transpose
                // read is behind the warp's synchronisation at its end).
#pragma unroll
                for (int k = 0; k < 32; k++) tbuf[k * 33 + lane] = x[k];
            }
            if (__syncthreads_or(!ok || *reinterpret_cast<volatile int *>(&sm.abort) != 0)) {
                aborted = true;
                break;
            }
            // Sums for (prime mpi, component mc), registers k = 16 mh + i of layout B (blocks of 4),
            // kept in registers for this pair of warps' inverse transform.
            uint32_t ys[16];
            if (ab != 0 && warp < 8) {
                const uint32_t *rows = sm.tbuf[mpi * ROWS];
#pragma unroll
                for (int qq = 0; qq < 4; qq++) {
                    const int q = 4 * mh + qq;
                    unsigned long long s4[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
                    for (int rr = 0; rr < ROWS; rr++) {
                        const uint4 kv = reinterpret_cast<const uint4 *>(sm.key[mpi * ROWS + rr] + mc * RING_N)[q * 32 + lane];
                        const uint32_t kk[4] = {kv.x, kv.y, kv.z, kv.w};
                        const uint32_t *xr = rows + rr * 32 * 33;
#pragma unroll
                        for (int e = 0; e < 4; e++) s4[e] += (unsigned long long)xr[(4 * q + e) * 33 + lane] * kk[e];
                    }
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        uint32_t v = redc64(s4[e], MK);
                        v = umin_u32(v, v - 2u * MK.p2);
                        ys[4 * qq + e] = umin_u32(v, v - MK.p2);
                    }
                }
            }
            __syncthreads();
            // Refill this warp's key buffer with the next step's row (every read of it is done).
            if (lane == 0 && i + 1 < n) {
                fence_proxy_async_smem();
                split_issue(sm, a.bsk_hat, warp, pi, r, i + 1);
            }
            pending = i + 1 < n;
            if (ab == 0) continue;   // CTA-uniform: ACC unchanged
            if (warp < 8) {
                // Component mc modulo prime mpi by warps (mpi, mc, 0) and (mpi, mc, 1), through the
                // transpose buffers of that warp pair (the parked rows are all read).
                const int w0 = 4 * mpi + 2 * mc;
                ntt_inv_2warp(ys, mh, lane, mpi, MK, sm.tw[mpi][1], sm.tbuf[w0], sm.tbuf[w0 + 1], 1 + 2 * mpi + mc);
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const int kk = i < 8 ? 8 * mh + i : 16 + 8 * mh + (i - 8);
                    sm.part[mpi][mc][lane + 32 * kk] = umin_u32(ys[i], ys[i] - MK.p);
                }
            }
            __syncthreads();
            // ACC += CRT(residues) for both components.
            for (int t = threadIdx.x; t < 2 * RING_N; t += blockDim.x) {
                const int c = t / RING_N, j = t % RING_N;
                sm.acc[c][j] += crt_lift(sm.part[0][c][j], sm.part[1][c][j]);
            }
            __syncthreads();
        }
        if (aborted) break;
        // Sample extraction: a'_0 = A_0, a'_j = -A_{N-j}, b' = B_0.
        uint32_t *dst = a.ext + (size_t)job * EXT_STRIDE;
        for (int j = threadIdx.x; j < RING_N; j += blockDim.x)
            dst[j] = j == 0 ? sm.acc[0][0] : 0u - sm.acc[0][RING_N - j];
        if (threadIdx.x == 0) dst[RING_N] = sm.acc[1][0];
        __syncthreads();
    }
    if (aborted && threadIdx.x == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
    // No bulk copy may still be in flight when the CTA exits (only possible after an abort).
    if (lane == 0 && pending) {
        volatile int never = 0;
        if (!mbar_wait_bounded(&sm.bar[warp], phase & 1u, &never)) atomicOr(a.err, DEV_ERR_TIMEOUT);
    }
}

// ---------------------------------------------------------------------------------
// Paired split blind rotation: one ciphertext per cluster of two CTAs on two SMs, for levels
// of at most one ciphertext per two SMs.  CTA rank q of the cluster computes modulo NTT prime
// q only, on 12 warps: warps 2 r and 2 r + 1 rotate and decompose digit row r (16 coefficients
// per lane each), forward-transform it together (ntt_fwd_2warp) and park it; warps (mc, mh) < 4
// sum the six rows' products with the key rows of output component mc for half mh of the
// registers (64-bit sums, one reduction each) and inverse-transform component mc together
// (ntt_inv_2warp).  Each CTA writes its residues of both components into its own shared memory
// and, with st.async, into its partner's, so that after one exchange per step both CTAs hold
// all four residue polynomials and each recombines both components (centred CRT) into its own
// copy of ACC; the two copies stay equal.
//
// Exchange s lands in buffer set s & 1 and completes on the receiver's mbarrier xbar[s & 1]:
// the receiver arms it once per exchange (one arrival, PAIR_XCHG_BYTES expected), and every
// st.async of the sender counts its bytes on it (release at cluster scope); the receiver's
// bounded wait acquires at cluster scope.  A sender reaches exchange s + 1 only after it has
// received exchange s, so it is at most one exchange ahead: the other set and the other
// barrier.  The sender's status word (1: a key copy timed out) is part of each exchange, so a
// CTA that stops makes its partner stop after the same exchange; a stopping CTA still sends
// every byte, which keeps the count exact.  The exchange waits allow four times the key
// waits' limit.  The hardware cluster barrier is used only at entry (the partner's barriers
// are initialised before the first st.async) and at exit (no CTA leaves while its partner may
// still write to it), both reached unconditionally.
// ---------------------------------------------------------------------------------
constexpr int PAIR_WARPS = 2 * ROWS;
constexpr int PAIR_THREADS = PAIR_WARPS * 32;
constexpr uint64_t PAIR_XCHG_LIMIT_NS = 4 * WAIT_LIMIT_NS;
constexpr uint32_t PAIR_XCHG_BYTES = 2u * RING_N * 4u + 4u;   // both components + status word

struct __align__(16) PairSmem {
    uint32_t key[ROWS][CHUNK_WORDS];                     // 48 KB: this step's rows for this CTA's prime
    uint32_t tbuf[ROWS][32 * 33];                         // 24.8 KB: transposes, then the parked rows
    uint32_t xbuf[ROWS][512];                             // 12 KB: the forward pairs' cross-warp swaps
    uint2 tw[2][LANE_TW * 32];                            // 15.5 KB [dir] for this CTA's prime
    uint32_t res[2][2][2][RING_N];                        // 32 KB [exchange set][prime][component]
    uint32_t acc[2][RING_N];                              // 8 KB
    uint16_t abar[ABAR_STRIDE_MAX];                       // 2 KB
    uint64_t bar[ROWS];                                   // key copies, one per row
    uint64_t xbar[2];                                     // exchanges, by set
    uint32_t status[2];                                   // the partner's status, by set
    int abort;                                            // a key wait of this CTA gave up
};

size_t br_pair_smem_bytes() { return sizeof(PairSmem); }

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// The address of the same shared-memory location in CTA `rank` of this cluster.
__device__ __forceinline__ uint32_t mapa_shared(const void *p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

// Store to another CTA's shared memory that counts its 4 bytes on that CTA's mbarrier.
__device__ __forceinline__ void st_async_u32(uint32_t addr, uint32_t v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.u32 [%0], %1, [%2];" ::"r"(addr), "r"(v),
                 "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void hw_cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\tselp.u32 "
        "%0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

__device__ __forceinline__ bool pair_wait_xchg(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((it & 255u) == 0u && global_timer_ns() - t0 > PAIR_XCHG_LIMIT_NS) return false;
    }
}

__device__ __forceinline__ void pair_issue(PairSmem &sm, const uint32_t *bsk_hat, int pi, int r, int i)
{
    mbar_arrive_expect_tx(&sm.bar[r], CHUNK_BYTES);
    bulk_copy_g2s(sm.key[r], bsk_hat + ((size_t)(i * 2 + pi) * ROWS + r) * CHUNK_WORDS, CHUNK_BYTES, &sm.bar[r]);
}

// selftest_stall (self-test only): CTA rank 1 issues no key copy, so its first wait runs out.
__global__ void __launch_bounds__(PAIR_THREADS, 1) br_pair_kernel(BrArgs a, int selftest_stall)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    PairSmem &sm = *reinterpret_cast<PairSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pi = (int)cluster_ctarank();   // this CTA's prime
    const uint32_t peer = 1u - (uint32_t)pi;
    const int r = warp >> 1, fh = warp & 1;   // forward: digit row r, half fh of its registers
    const int c_in = r / LG, p_dig = r % LG;
    const int n = a.n;
    const PrimeK K = prime_k(pi);
    const int mc = warp >> 1, mh = warp & 1;   // warps 0..3 after the forward transforms
    const uint32_t peer_res = mapa_shared(&sm.res[0][0][0][0], peer);
    const uint32_t peer_xbar = mapa_shared(&sm.xbar[0], peer);
    const uint32_t peer_status = mapa_shared(&sm.status[0], peer);

    for (int i = threadIdx.x; i < 2 * LANE_TW * 32; i += blockDim.x)
        (&sm.tw[0][0])[i] = a.tw_lane[(size_t)pi * 2 * LANE_TW * 32 + i];
    if (threadIdx.x == 0) {
        for (int w = 0; w < ROWS; w++) mbar_init(&sm.bar[w], 1);
        mbar_init(&sm.xbar[0], 1);
        mbar_init(&sm.xbar[1], 1);
        sm.abort = 0;
        mbar_fence_init();
    }
    __syncthreads();
    hw_cluster_sync();   // both CTAs' barriers are initialised

    uint32_t phase = 0;        // completed uses of this warp's key barrier
    uint32_t xs = 0;           // exchanges done
    bool pending = false;      // a copy into this row's key buffer is in flight
    bool aborted = false;
    const int clusters = (int)(gridDim.x >> 1);
    for (int job = (int)(blockIdx.x >> 1); job < a.jobs && !aborted; job += clusters) {
        const uint16_t *src = a.abar + (size_t)job * a.abar_stride;
        for (int i = threadIdx.x; i <= n; i += blockDim.x) sm.abar[i] = src[i];
        __syncthreads();
        const int bb = sm.abar[n];
        for (int j = threadIdx.x; j < RING_N; j += blockDim.x) {
            sm.acc[0][j] = 0u;
            const int e = (j + bb) & (2 * RING_N - 1);
            sm.acc[1][j] = (e & RING_N) ? (0u - a.mu) : a.mu;
        }
        if (n > 0) {
            // (In the stop self-test CTA 1 issues nothing, so its first key wait runs out.)
            if (lane == 0 && fh == 0 && !(selftest_stall && pi == 1)) pair_issue(sm, a.bsk_hat, pi, r, 0);
            pending = true;   // both warps of the row track its barrier
        }
        __syncthreads();
        for (int i = 0; i < n; i++) {
            const int ab = sm.abar[i];   // both CTAs run the same job: the same decisions
            const int set = (int)(xs & 1u);
            // Arm this exchange's barrier (its previous phase completed two exchanges ago).
            if (threadIdx.x == 0) mbar_arrive_expect_tx(&sm.xbar[set], PAIR_XCHG_BYTES);
            bool ok = true;
            if (pending) {
                ok = mbar_wait_bounded(&sm.bar[r], phase & 1u, &sm.abort);
                if (ok) {
                    phase++;
                    pending = false;   // else the copy stays pending for the drain at exit
                }
            }
            if (!ok && lane == 0) *reinterpret_cast<volatile int *>(&sm.abort) = 1;
            // The two warps of a row agree before their transform meets at its barriers.
            const bool row_ok = !bar_red_or(1 + r, 64, !ok);
            if (ab != 0 && row_ok) {
                const uint32_t *A = sm.acc[c_in];
                const int sh = 32 - BGBIT * (p_dig + 1);
                uint32_t x[16];
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    const int j = lane + 32 * (2 * k + fh);   // layout-A register 2 k + fh
                    const int idx = (j - ab) & (2 * RING_N - 1);
                    uint32_t v = A[idx & (RING_N - 1)];
                    v = (idx & RING_N) ? (0u - v) : v;
                    const uint32_t u = v - A[j] + GADGET_OFF;
                    x[k] = ((u >> sh) & 1023u) + (K.p - 512u);
                }
                ntt_fwd_2warp(x, fh, lane, pi, K, sm.tw[0], sm.tbuf[r], sm.xbuf[r], 1 + r);
                // Park the row: layout-B register k of lane t at [k][t].
#pragma unroll
                for (int m = 0; m < 16; m++) sm.tbuf[r][(16 * fh + m) * 33 + lane] = x[m];
            }
            const bool bad = __syncthreads_or(!row_ok || *reinterpret_cast<volatile int *>(&sm.abort) != 0);
            const bool work = !bad && ab != 0;
            uint32_t ys[16];
#pragma unroll
            for (int t = 0; t < 16; t++) ys[t] = 0u;
            if (work && warp < 4) {
#pragma unroll
                for (int qq = 0; qq < 4; qq++) {
                    const int q = 4 * mh + qq;
                    unsigned long long s4[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
                    for (int rr = 0; rr < ROWS; rr++) {
                        const uint4 kv = reinterpret_cast<const uint4 *>(sm.key[rr] + mc * RING_N)[q * 32 + lane];
                        const uint32_t kk[4] = {kv.x, kv.y, kv.z, kv.w};
                        const uint32_t *xr = sm.tbuf[rr];
#pragma unroll
                        for (int e = 0; e < 4; e++) s4[e] += (unsigned long long)xr[(4 * q + e) * 33 + lane] * kk[e];
                    }
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        uint32_t v = redc64(s4[e], K);
                        v = umin_u32(v, v - 2u * K.p2);
                        ys[4 * qq + e] = umin_u32(v, v - K.p2);
                    }
                }
            }
            __syncthreads();
            // Refill this warp's key buffer with the next step's row (every read of it is done).
            if (!bad && lane == 0 && fh == 0 && i + 1 < n) {
                fence_proxy_async_smem();
                pair_issue(sm, a.bsk_hat, pi, r, i + 1);
            }
            if (!bad && i + 1 < n) pending = true;
            if (warp < 4) {
                // Component mc modulo this CTA's prime by warps (mc, 0) and (mc, 1), through the
                // transpose buffers of rows 2 mc and 2 mc + 1 (all parked rows are read).
                if (work)
                    ntt_inv_2warp(ys, mh, lane, pi, K, sm.tw[1], sm.tbuf[2 * mc], sm.tbuf[2 * mc + 1], 1 + ROWS + mc);
                const int off = ((set * 2 + pi) * 2 + mc) * RING_N;
                uint32_t *dst = &sm.res[0][0][0][0] + off;
                const uint32_t rdst = peer_res + 4u * (uint32_t)off;
                const uint32_t rbar = peer_xbar + 8u * (uint32_t)set;
#pragma unroll
                for (int t = 0; t < 16; t++) {
                    const int kk = t < 8 ? 8 * mh + t : 16 + 8 * mh + (t - 8);
                    const int j = lane + 32 * kk;
                    const uint32_t v = umin_u32(ys[t], ys[t] - K.p);
                    dst[j] = v;
                    st_async_u32(rdst + 4u * (uint32_t)j, v, rbar);
                }
                if (threadIdx.x == 0)
                    st_async_u32(peer_status + 4u * (uint32_t)set, bad ? 1u : 0u, rbar);
            }
            const bool arrived = pair_wait_xchg(&sm.xbar[set], (xs >> 1) & 1u);
            xs++;
            const bool stop =
                __syncthreads_or(bad || !arrived || *reinterpret_cast<volatile uint32_t *>(&sm.status[set]) != 0u);
            if (stop) {
                aborted = true;
                break;
            }
            if (ab != 0) {
                // ACC += CRT(residues) for both components, from this exchange's set.
                for (int t = threadIdx.x; t < 2 * RING_N; t += blockDim.x) {
                    const int c = t / RING_N, j = t % RING_N;
                    sm.acc[c][j] += crt_lift(sm.res[set][0][c][j], sm.res[set][1][c][j]);
                }
            }
            __syncthreads();
        }
        if (aborted) break;
        // Sample extraction (both copies of ACC are equal; CTA 0 writes the sample).
        if (pi == 0) {
            uint32_t *dst = a.ext + (size_t)job * EXT_STRIDE;
            for (int j = threadIdx.x; j < RING_N; j += blockDim.x)
                dst[j] = j == 0 ? sm.acc[0][0] : 0u - sm.acc[0][RING_N - j];
            if (threadIdx.x == 0) dst[RING_N] = sm.acc[1][0];
        }
        __syncthreads();
    }
    if (aborted && threadIdx.x == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
    // No bulk copy may still be in flight when the CTA exits (only possible after an abort).
    if (lane == 0 && pending) {
        volatile int never = 0;
        if (!mbar_wait_bounded(&sm.bar[r], phase & 1u, &never)) atomicOr(a.err, DEV_ERR_TIMEOUT);
    }
    hw_cluster_sync();   // the partner no longer writes to this CTA's shared memory
}

// ---------------------------------------------------------------------------------
// Quad split blind rotation: one ciphertext per cluster of four CTAs on four SMs, for levels
// of at most one ciphertext per four SMs.  CTA rank 2 g + q computes modulo NTT prime q and
// owns ACC component g; because digit rows 3 g .. 3 g + 2 decompose component g, it needs no
// other part of ACC.  On 12 warps:
//   * warps 4 r' .. 4 r' + 3 decompose digit row 3 g + r' (8 coefficients per lane each),
//     forward-transform it together (ntt_fwd_4warp) and park it;
//   * warps 4 mc + w (mc, w < 2, 4) sum the three parked rows' products with the key rows of
//     output component mc for registers 8 w .. 8 w + 7 (64-bit sums, one reduction each);
//   * exchange P: the partial sums of component 1 - g go to the CTA of the same prime that owns
//     it (rank ^ 2), whose partial sums of component g arrive here; warps 4 g .. 4 g + 3 add
//     them and inverse-transform component g together (ntt_inv_4warp);
//   * exchange R: the residues of component g modulo this prime go to the CTA of the other
//     prime that owns the same component (rank ^ 1), whose residues arrive here; all warps
//     recombine component g (centred CRT) into ACC.
// Both exchanges work as in br_pair_kernel (st.async stores that count their bytes on the
// receiver's mbarrier of the exchange's parity, bounded acquire waits, one status word each).
// A CTA's status in exchange R is its stop decision after exchange P (its own key wait or its
// P partner's status), so a stop reaches all four CTAs by the end of the same step, and every
// CTA still sends every byte of both exchanges.  CTA 0 writes the extracted a', CTA 2 b'.
// ---------------------------------------------------------------------------------
constexpr int QUAD_ROWS = LG;                          // digit rows per CTA
constexpr int QUAD_WARPS = 4 * QUAD_ROWS;
constexpr int QUAD_THREADS = QUAD_WARPS * 32;
constexpr uint32_t QUAD_XCHG_BYTES = RING_N * 4u + 4u;   // one polynomial + status word
// Dynamic shared memory of at least this size keeps two CTAs of a cluster off one SM.
constexpr size_t QUAD_SMEM_MIN = 116 * 1024;

struct __align__(16) QuadSmem {
    uint32_t key[QUAD_ROWS][CHUNK_WORDS];                 // 24 KB: this step's rows for this prime
    uint32_t tbuf[QUAD_ROWS][32 * 33];                     // 12.4 KB: transposes, then the parked rows
    uint32_t xbuf[QUAD_ROWS][1024];                        // 12 KB: the four-warp transforms' swaps
    uint2 tw[2][LANE_TW * 32];                             // 15.5 KB [dir] for this CTA's prime
    uint32_t psum[2][RING_N];                              // 8 KB: partner's partial sums, by set
    uint32_t res[2][2][RING_N];                            // 16 KB [set][prime]: component g residues
    uint32_t acc[RING_N];                                  // 4 KB: ACC component g
    uint16_t abar[ABAR_STRIDE_MAX];                        // 2 KB
    uint64_t bar[QUAD_ROWS];                               // key copies, one per row
    uint64_t xp[2], xr[2];                                 // exchanges P and R, by set
    uint32_t status_p[2], status_r[2];                     // the partners' status words, by set
    int abort;                                             // a key wait of this CTA gave up
};

size_t br_quad_smem_bytes() { return sizeof(QuadSmem) > QUAD_SMEM_MIN ? sizeof(QuadSmem) : QUAD_SMEM_MIN; }

__device__ __forceinline__ void quad_issue(QuadSmem &sm, const uint32_t *bsk_hat, int pi, int g, int rl, int i)
{
    mbar_arrive_expect_tx(&sm.bar[rl], CHUNK_BYTES);
    bulk_copy_g2s(sm.key[rl], bsk_hat + ((size_t)(i * 2 + pi) * ROWS + LG * g + rl) * CHUNK_WORDS, CHUNK_BYTES,
                  &sm.bar[rl]);
}

// selftest_stall (self-test only): CTA rank 1 issues no key copy, so its first wait runs out.
__global__ void __launch_bounds__(QUAD_THREADS, 1) br_quad_kernel(BrArgs a, int selftest_stall)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    QuadSmem &sm = *reinterpret_cast<QuadSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const int pi = (int)(rank & 1u), g = (int)(rank >> 1);   // prime, owned component
    const int rl = warp >> 2, fw = warp & 3;                   // forward: local row, warp in row
    const int mc = warp >> 2, mw = warp & 3;                   // products (warps 0..7)
    const int n = a.n;
    const PrimeK K = prime_k(pi);
    const uint32_t half_peer = rank ^ 2u, prime_peer = rank ^ 1u;
    const uint32_t peer_psum = mapa_shared(&sm.psum[0][0], half_peer);
    const uint32_t peer_xp = mapa_shared(&sm.xp[0], half_peer);
    const uint32_t peer_status_p = mapa_shared(&sm.status_p[0], half_peer);
    const uint32_t peer_res = mapa_shared(&sm.res[0][0][0], prime_peer);
    const uint32_t peer_xr = mapa_shared(&sm.xr[0], prime_peer);
    const uint32_t peer_status_r = mapa_shared(&sm.status_r[0], prime_peer);

    for (int i = threadIdx.x; i < 2 * LANE_TW * 32; i += blockDim.x)
        (&sm.tw[0][0])[i] = a.tw_lane[(size_t)pi * 2 * LANE_TW * 32 + i];
    if (threadIdx.x == 0) {
        for (int w = 0; w < QUAD_ROWS; w++) mbar_init(&sm.bar[w], 1);
        for (int s = 0; s < 2; s++) {
            mbar_init(&sm.xp[s], 1);
            mbar_init(&sm.xr[s], 1);
        }
        sm.abort = 0;
        mbar_fence_init();
    }
    __syncthreads();
    hw_cluster_sync();   // all four CTAs' barriers are initialised

    uint32_t phase = 0;        // completed uses of this warp's key barrier
    uint32_t xs = 0;           // steps exchanged (each step: one P and one R exchange)
    bool pending = false;      // a copy into this row's key buffer is in flight
    bool aborted = false;
    const int clusters = (int)(gridDim.x >> 2);
    for (int job = (int)(blockIdx.x >> 2); job < a.jobs && !aborted; job += clusters) {
        const uint16_t *src = a.abar + (size_t)job * a.abar_stride;
        for (int i = threadIdx.x; i <= n; i += blockDim.x) sm.abar[i] = src[i];
        __syncthreads();
        const int bb = sm.abar[n];
        for (int j = threadIdx.x; j < RING_N; j += blockDim.x) {
            const int e = (j + bb) & (2 * RING_N - 1);
            sm.acc[j] = g == 0 ? 0u : ((e & RING_N) ? (0u - a.mu) : a.mu);
        }
        if (n > 0) {
            if (lane == 0 && fw == 0 && !(selftest_stall && rank == 1u)) quad_issue(sm, a.bsk_hat, pi, g, rl, 0);
            pending = true;   // the row's four warps track its barrier
        }
        __syncthreads();
        for (int i = 0; i < n; i++) {
            const int ab = sm.abar[i];   // all four CTAs run the same job: the same decisions
            const int set = (int)(xs & 1u);
            const uint32_t par = (xs >> 1) & 1u;
            if (threadIdx.x == 0) {
                mbar_arrive_expect_tx(&sm.xp[set], QUAD_XCHG_BYTES);
                mbar_arrive_expect_tx(&sm.xr[set], QUAD_XCHG_BYTES);
            }
            bool ok = true;
            if (pending) {
                ok = mbar_wait_bounded(&sm.bar[rl], phase & 1u, &sm.abort);
                if (ok) {
                    phase++;
                    pending = false;   // else the copy stays pending for the drain at exit
                }
            }
            if (!ok && lane == 0) *reinterpret_cast<volatile int *>(&sm.abort) = 1;
            // The four warps of a row agree before their transform meets at its barriers.
            const bool row_ok = !bar_red_or(1 + rl, 128, !ok);
            if (ab != 0 && row_ok) {
                const uint32_t *A = sm.acc;
                const int sh = 32 - BGBIT * (rl + 1);
                uint32_t x[8];
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const int j = lane + 32 * (4 * k + fw);   // layout-A register 4 k + fw
                    const int idx = (j - ab) & (2 * RING_N - 1);
                    uint32_t v = A[idx & (RING_N - 1)];
                    v = (idx & RING_N) ? (0u - v) : v;
                    const uint32_t u = v - A[j] + GADGET_OFF;
                    x[k] = ((u >> sh) & 1023u) + (K.p - 512u);
                }
                ntt_fwd_4warp(x, fw, lane, pi, K, sm.tw[0], sm.tbuf[rl], sm.xbuf[rl], 1 + rl);
                // Park the row: layout-B register k of lane t at [k][t].
#pragma unroll
                for (int e = 0; e < 2; e++)
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        sm.tbuf[rl][(16 * (fw >> 1) + 4 * j + 2 * (fw & 1) + e) * 33 + lane] = x[4 * e + j];
            }
            const bool bad = __syncthreads_or(!row_ok || *reinterpret_cast<volatile int *>(&sm.abort) != 0);
            const bool work = !bad && ab != 0;
            uint32_t ys[8];
#pragma unroll
            for (int t = 0; t < 8; t++) ys[t] = 0u;
            if (work && warp < 8) {
                // Partial sums of component mc over this CTA's three rows, registers 8 mw + 4 qq + e.
#pragma unroll
                for (int qq = 0; qq < 2; qq++) {
                    const int q = 2 * mw + qq;
                    unsigned long long s4[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
                    for (int rr = 0; rr < QUAD_ROWS; rr++) {
                        const uint4 kv = reinterpret_cast<const uint4 *>(sm.key[rr] + mc * RING_N)[q * 32 + lane];
                        const uint32_t kk[4] = {kv.x, kv.y, kv.z, kv.w};
                        const uint32_t *xr = sm.tbuf[rr];
#pragma unroll
                        for (int e = 0; e < 4; e++) s4[e] += (unsigned long long)xr[(4 * q + e) * 33 + lane] * kk[e];
                    }
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        uint32_t v = redc64(s4[e], K);
                        v = umin_u32(v, v - 2u * K.p2);
                        ys[4 * qq + e] = umin_u32(v, v - K.p2);
                    }
                }
            }
            __syncthreads();
            // Refill the key buffers with the next step's rows (every read of them is done).
            if (!bad && lane == 0 && fw == 0 && i + 1 < n) {
                fence_proxy_async_smem();
                quad_issue(sm, a.bsk_hat, pi, g, rl, i + 1);
            }
            if (!bad && i + 1 < n) pending = true;
            bool stop_p = false;   // known to warps 4 g .. 4 g + 3
            if (warp < 8 && mc != g) {
                // Exchange P out: component 1 - g to the CTA of this prime that owns it.
                const uint32_t rdst = peer_psum + 4u * (uint32_t)(set * RING_N);
                const uint32_t rbar = peer_xp + 8u * (uint32_t)set;
#pragma unroll
                for (int t = 0; t < 8; t++) st_async_u32(rdst + 4u * (uint32_t)((8 * mw + t) * 32 + lane), ys[t], rbar);
                if (mw == 0 && lane == 0) st_async_u32(peer_status_p + 4u * (uint32_t)set, bad ? 1u : 0u, rbar);
            } else if (warp < 8) {
                // Exchange P in, then component g modulo this prime: add, inverse-transform, and
                // exchange R out to the other prime's CTA of this component.
                const bool arrived = pair_wait_xchg(&sm.xp[set], par);
                stop_p = bad || !arrived || *reinterpret_cast<volatile uint32_t *>(&sm.status_p[set]) != 0u;
#pragma unroll
                for (int t = 0; t < 8; t++) {
                    const uint32_t v = ys[t] + sm.psum[set][(8 * mw + t) * 32 + lane];
                    ys[t] = umin_u32(v, v - K.p2);
                }
                if (work)
                    ntt_inv_4warp(ys, mw, lane, pi, K, sm.tw[1], sm.tbuf[0], sm.tbuf[1], 1 + QUAD_ROWS);
                uint32_t *dst = &sm.res[set][pi][0];
                const uint32_t rdst = peer_res + 4u * (uint32_t)((set * 2 + pi) * RING_N);
                const uint32_t rbar = peer_xr + 8u * (uint32_t)set;
#pragma unroll
                for (int t = 0; t < 8; t++) {
                    const int j = lane + 32 * (16 * (t >> 2) + 8 * (mw >> 1) + 4 * (mw & 1) + (t & 3));
                    const uint32_t v = umin_u32(ys[t], ys[t] - K.p);
                    dst[j] = v;
                    st_async_u32(rdst + 4u * (uint32_t)j, v, rbar);
                }
                if (mw == 0 && lane == 0) st_async_u32(peer_status_r + 4u * (uint32_t)set, stop_p ? 1u : 0u, rbar);
            }
            const bool arrived_r = pair_wait_xchg(&sm.xr[set], par);
            xs++;
            const bool stop = __syncthreads_or(stop_p || bad || !arrived_r ||
                                               *reinterpret_cast<volatile uint32_t *>(&sm.status_r[set]) != 0u);
            if (stop) {
                aborted = true;
                break;
            }
            if (ab != 0) {
                // ACC_g += CRT(residues), from this step's set.
                for (int j = threadIdx.x; j < RING_N; j += blockDim.x)
                    sm.acc[j] += crt_lift(sm.res[set][0][j], sm.res[set][1][j]);
            }
            __syncthreads();
        }
        if (aborted) break;
        // Sample extraction: CTA 0 (prime 0, component 0) writes a', CTA 2 (component 1) b'.
        uint32_t *dst = a.ext + (size_t)job * EXT_STRIDE;
        if (rank == 0u)
            for (int j = threadIdx.x; j < RING_N; j += blockDim.x)
                dst[j] = j == 0 ? sm.acc[0] : 0u - sm.acc[RING_N - j];
        if (rank == 2u && threadIdx.x == 0) dst[RING_N] = sm.acc[0];
        __syncthreads();
    }
    if (aborted && threadIdx.x == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
    // No bulk copy may still be in flight when the CTA exits (only possible after an abort).
    if (lane == 0 && pending) {
        volatile int never = 0;
        if (!mbar_wait_bounded(&sm.bar[rl], phase & 1u, &never)) atomicOr(a.err, DEV_ERR_TIMEOUT);
    }
    hw_cluster_sync();   // no partner writes to this CTA's shared memory any more
}

// ---------------------------------------------------------------------------------
// Bootstrapping key -> transform domain.  One warp per (i, prime, row, component)
// polynomial: centred lift mod p, forward NTT, scale by N^-1 2^32 mod p, store in the
// chunk layout the blind rotation reads (component c, then [q][lane][4] so that lane t
// finds registers k = 4q .. 4q+3 of layout B in one 16-byte load).
// ---------------------------------------------------------------------------------
struct ConvSmem {
    uint32_t tbuf[8][32 * 33];
    uint2 tw[2][LANE_TW * 32];   // forward tables of both primes
};

__global__ void __launch_bounds__(256) bsk_to_ntt_kernel(const uint32_t *bsk, uint32_t *bsk_hat, int n,
                                                         const uint2 *tw_lane, uint32_t scale0, uint32_t scale1)
{
    __shared__ ConvSmem sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < LANE_TW * 32; i += blockDim.x) {
        sm.tw[0][i] = tw_lane[(0 * 2 + 0) * LANE_TW * 32 + i];
        sm.tw[1][i] = tw_lane[(1 * 2 + 0) * LANE_TW * 32 + i];
    }
    __syncthreads();
    const long total = (long)n * 2 * ROWS * 2;
    for (long poly = (long)blockIdx.x * 8 + warp; poly < total; poly += (long)gridDim.x * 8) {
        const int c = (int)(poly % 2);
        const int r = (int)((poly / 2) % ROWS);
        const int pi = (int)((poly / (2 * ROWS)) % 2);
        const long i = poly / (4 * ROWS);
        const uint32_t *src = bsk + ((i * ROWS + r) * 2 + c) * RING_N;
        const PrimeK K = prime_k(pi);
        uint32_t x[32];
#pragma unroll
        for (int k = 0; k < 32; k++) {
            const int32_t v = (int32_t)src[lane + 32 * k];
            int64_t m = (int64_t)v % (int64_t)K.p;
            if (m < 0) m += K.p;
            x[k] = (uint32_t)m;
        }
        ntt_fwd<true>(x, sm.tbuf[warp], sm.tw[pi], lane, pi, K);
        const uint64_t sc = pi == 0 ? scale0 : scale1;   // N^-1 2^32 mod p
        uint32_t *dst = bsk_hat + ((i * 2 + pi) * ROWS + r) * CHUNK_WORDS + c * RING_N;
#pragma unroll
        for (int k = 0; k < 32; k++) {
            const uint64_t y = (uint64_t)(x[k] % K.p) * sc % K.p;
            dst[(k >> 2) * 128 + lane * 4 + (k & 3)] = (uint32_t)y;
        }
    }
}

// ---------------------------------------------------------------------------------
// Persistent circuit executor: one launch runs a whole levelled schedule (every pass of
// pre-combination + modulus switch, blind rotation + extraction, key switch, then the output
// copies).  One CTA per SM, all resident (cooperative launch).  Within a phase the CTAs pull
// their work from device-side counters -- groups of BR_SLOTS blind rotations, key-switch
// units of one batch (and one coefficient slice) -- so no host step sits between the levels;
// phases meet at grid-wide barriers whose waits give up after 2 s without progress (a shared
// progress counter moves with every finished unit), raise a global abort flag and report
// LP_ETIMEOUT.  Shared memory holds the blind rotation's state or the key switch's, one after
// the other: each phase initialises its barriers and invalidates them when it ends.
// ---------------------------------------------------------------------------------
constexpr uint64_t EXEC_WAIT_NS = 2000000000ull;

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier over ctl[0] (arrivals) and ctl[1] (generation); ctl[2] counts progress,
// ctl[3] is the abort flag.  Returns false (CTA-uniformly) when the executor is aborting.
__device__ bool exec_barrier(uint32_t *ctl, int *err, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = ld_acquire_gpu(&ctl[3]) == 0u;
        const uint32_t gen = ld_acquire_gpu(&ctl[1]);
        __threadfence();
        atomicAdd(&ctl[2], 1u);
        if (atomicAdd(&ctl[0], 1u) == gridDim.x - 1) {
            atomicExch(&ctl[0], 0u);
            __threadfence();
            atomicAdd(&ctl[1], 1u);
        } else {
            uint32_t prog = ld_acquire_gpu(&ctl[2]);
            uint64_t t0 = global_timer_ns();
            for (uint32_t it = 1; ld_acquire_gpu(&ctl[1]) == gen; ++it) {
                if ((it & 63u) != 0u) continue;
                if (ld_acquire_gpu(&ctl[3]) != 0u) break;
                const uint32_t p = ld_acquire_gpu(&ctl[2]);
                const uint64_t t = global_timer_ns();
                if (p != prog) {
                    prog = p;
                    t0 = t;
                } else if (t - t0 > EXEC_WAIT_NS) {
                    atomicExch(&ctl[3], 1u);
                    atomicOr(err, DEV_ERR_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
        ok = ok && ld_acquire_gpu(&ctl[3]) == 0u;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

__global__ void __launch_bounds__(BR_THREADS, 1) exec_kernel(ExecArgs x)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    BrSmem &bs = *reinterpret_cast<BrSmem *>(smem_raw);
    KsSmem &ks = *reinterpret_cast<KsSmem *>(smem_raw);
    __shared__ int s_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = x.n, V = n + 1;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nthr = (size_t)gridDim.x * blockDim.x;
    if (x.selftest_stall && blockIdx.x == 0) return;   // nothing in flight: the wait self-test
    bool ok = true;
    for (int p = 0; p < x.npasses && ok; p++) {
        const ExecPass P = x.passes[p];
        // Pre-combination + modulus switch of the pass's blind-rotation jobs (every thread).
        const BrJob *jobs = x.br + P.br_off;
        for (size_t idx = tid; idx < (size_t)P.br_cnt * V; idx += nthr) {
            const size_t jb = idx / V;
            const int w = (int)(idx % V);
            const BrJob J = jobs[jb];
            uint32_t v = 0u;
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (J.coef[k] != 0) v += (uint32_t)J.coef[k] * x.pool[(size_t)J.in[k] * V + w];
            if (w == n) v += J.bconst;
            x.abar[jb * x.abar_stride + w] = modswitch_2048(v);
        }
        if (!(ok = exec_barrier(x.ctl, x.err, &s_flag))) break;
        // Blind rotation + extraction: groups pulled from the pass's counter.
        if (P.br_cnt > 0) {
            for (int i = threadIdx.x; i < 2 * 2 * LANE_TW * 32; i += blockDim.x) (&bs.tw[0][0][0])[i] = x.tw_lane[i];
            if (threadIdx.x == 0) {
                for (int q = 0; q < 2; q++)
                    for (int r = 0; r < BR_RING; r++) {
                        mbar_init(&bs.full_bar[q][r], 1);
                        mbar_init(&bs.empty_bar[q][r], BR_SLOTS);
                    }
                bs.abort = 0;
                mbar_fence_init();
            }
            __syncthreads();
            BrArgs a{x.abar, x.ext, x.bsk_hat, x.tw_lane, n, x.abar_stride, (int)P.br_cnt, T_EIGHTH, x.err};
            const bool good = compute_warp<true>(bs, a, warp, lane, (int)((P.br_cnt + BR_SLOTS - 1) / BR_SLOTS),
                                                 &x.ctl[4 + 2 * p], &x.ctl[2]);
            if (__syncthreads_or(!good) && threadIdx.x == 0) atomicExch(&x.ctl[3], 1u);
            if (threadIdx.x == 0)
                for (int q = 0; q < 2; q++)
                    for (int r = 0; r < BR_RING; r++) {
                        mbar_inval(&bs.full_bar[q][r]);
                        mbar_inval(&bs.empty_bar[q][r]);
                    }
        }
        if (!(ok = exec_barrier(x.ctl, x.err, &s_flag))) break;
        // Key switch: units of one batch of KS_CT outputs, split into coefficient slices when the
        // batches are too few for the SMs (outputs first set to (0, b'), then added into).
        const KsJob *kj = x.ks + P.ks_off;
        const size_t nb = ((size_t)P.ks_cnt + KS_CT - 1) / KS_CT;
        const bool sliced = x.ks_slice_max > 0 ? nb <= (size_t)x.ks_slice_max
                                               : x.ks_slice_max < 0 ? false : 2 * nb < (size_t)gridDim.x;
        const int slices = sliced ? ks_slices(nb, gridDim.x) : 1;
        if (sliced) {
            ks_init_rows(x.ext, kj, P.ks_cnt, 0, x.pool, n, tid, nthr);
            if (!(ok = exec_barrier(x.ctl, x.err, &s_flag))) break;
        }
        if (P.ks_cnt > 0) {
            KsProducer pr;
            ks_setup(ks, pr, x.T, n);
            __syncthreads();
            uint32_t cseq = 0;
            bool good = true;
            const int nblk = RING_N / KS_ICH;
            for (;;) {
                __syncthreads();
                if (threadIdx.x == 0) s_flag = (int)atomicAdd(&x.ctl[5 + 2 * p], 1u);
                __syncthreads();
                const size_t u = (size_t)s_flag;
                if (u >= nb * slices) break;
                const size_t bt = u / slices;
                const int sl = (int)(u % slices);
                const int i_begin = sliced ? (sl * nblk / slices) * KS_ICH : 0;
                const int i_end = sliced ? ((sl + 1) * nblk / slices) * KS_ICH : RING_N;
                good = sliced ? ks_unit<true>(ks, pr, cseq, x.ext, kj, P.ks_cnt, 0, x.pool, n, bt, i_begin, i_end)
                              : ks_unit<false>(ks, pr, cseq, x.ext, kj, P.ks_cnt, 0, x.pool, n, bt, i_begin, i_end);
                if (!good) break;
                if (threadIdx.x == 0) atomicAdd(&x.ctl[2], 1u);
            }
            if (threadIdx.x == 0 && !ks_drain(ks, pr)) good = false;
            if (__syncthreads_or(!good) && threadIdx.x == 0) {
                atomicExch(&x.ctl[3], 1u);
                atomicOr(x.err, DEV_ERR_TIMEOUT);
            }
            if (threadIdx.x == 0)
                for (int r = 0; r < KS_RING; r++) {
                    mbar_inval(&ks.full_bar[r]);
                    mbar_inval(&ks.empty_bar[r]);
                }
        }
        ok = exec_barrier(x.ctl, x.err, &s_flag);
    }
    if (!ok) return;
    // Outputs out of the pool (negated where the output signal is).
    for (size_t idx = tid; idx < (size_t)x.nout * V; idx += nthr) {
        const CopyEntry E = x.outc[idx / V];
        const uint32_t v = E.src[idx % V];
        E.dst[idx % V] = E.neg ? 0u - v : v;
    }
}

size_t exec_smem_bytes() { return sizeof(BrSmem) > sizeof(KsSmem) ? sizeof(BrSmem) : sizeof(KsSmem); }

cudaError_t launch_exec(const ExecArgs &x, int num_sms, cudaStream_t st)
{
    const size_t smem = exec_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(exec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)num_sms);
    cfg.blockDim = dim3(BR_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, exec_kernel, x);
}

// ---------------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------------
cudaError_t upload_constants(const NttTables &t)
{
    uint4 prm[2];
    for (int pi = 0; pi < 2; pi++)
        prm[pi] = make_uint4(t.prime[pi], 2u * t.prime[pi], t.pinv_neg[pi], t.red_one[pi]);
    cudaError_t e = cudaMemcpyToSymbol(c_tw, t.ctw, sizeof(t.ctw));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_prm, prm, sizeof(prm));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_crt, &t.crt, sizeof(t.crt));
    return e;
}

cudaError_t launch_bsk_to_ntt(const uint32_t *bsk, uint32_t *bsk_hat, int n, const uint2 *tw_lane,
                              uint32_t scale0, uint32_t scale1, int num_sms, cudaStream_t st)
{
    const long polys = (long)n * 2 * ROWS * 2;
    long grid = (polys + 7) / 8;
    if (grid > 4L * num_sms) grid = 4L * num_sms;
    bsk_to_ntt_kernel<<<(int)grid, 256, 0, st>>>(bsk, bsk_hat, n, tw_lane, scale0, scale1);
    return cudaGetLastError();
}

static cudaError_t launch_split(const BrArgs &a, int num_sms, cudaStream_t st)
{
    const size_t smem = sizeof(SplitSmem);
    cudaError_t e = cudaFuncSetAttribute(br_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = a.jobs < num_sms ? a.jobs : num_sms;
    br_split_kernel<<<grid, SPLIT_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// Launch configuration of a cluster kernel: `csize` CTAs per cluster, `clusters` clusters.
static cudaError_t cluster_config(const void *kernel, int threads, size_t smem, int csize, int clusters,
                                  cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3((unsigned)(csize * clusters));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaSuccess;
}

static cudaError_t pair_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr, int clusters, cudaStream_t st)
{
    return cluster_config((const void *)br_pair_kernel, PAIR_THREADS, sizeof(PairSmem), 2, clusters, cfg, attr, st);
}

static cudaError_t quad_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr, int clusters, cudaStream_t st)
{
    return cluster_config((const void *)br_quad_kernel, QUAD_THREADS, br_quad_smem_bytes(), 4, clusters, cfg, attr,
                          st);
}

int br_pair_clusters(int num_sms)
{
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    if (pair_config(cfg, attr, num_sms / 2, nullptr) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, br_pair_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// Resident clusters of four per device, recorded by br_quad_clusters (the GPCs' SM counts need
// not be multiples of 4, so fewer than num_sms / 4 may fit at once); launch_quad launches no
// more clusters than that, so none waits for another to finish.
constexpr int QUAD_MAX_DEVICES = 64;
static int g_quad_resident[QUAD_MAX_DEVICES];   // read and written with __atomic builtins

int br_quad_clusters(int num_sms)
{
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    if (quad_config(cfg, attr, num_sms / 4, nullptr) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, br_quad_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < QUAD_MAX_DEVICES)
        __atomic_store_n(&g_quad_resident[dev], n, __ATOMIC_RELAXED);
    return n;
}

static cudaError_t launch_pair(const BrArgs &a, int num_sms, cudaStream_t st, int selftest_stall = 0)
{
    const int clusters = a.jobs < num_sms / 2 ? a.jobs : num_sms / 2;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = pair_config(cfg, attr, clusters, st);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, br_pair_kernel, a, selftest_stall);
}

static cudaError_t launch_quad(const BrArgs &a, int num_sms, cudaStream_t st, int selftest_stall = 0)
{
    int cap = num_sms / 4, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < QUAD_MAX_DEVICES) {
        const int r = __atomic_load_n(&g_quad_resident[dev], __ATOMIC_RELAXED);
        if (r > 0 && r < cap) cap = r;
    }
    const int clusters = a.jobs < cap ? a.jobs : cap;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = quad_config(cfg, attr, clusters, st);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, br_quad_kernel, a, selftest_stall);
}

cudaError_t launch_pair_selftest(const uint16_t *abar, int abar_stride, uint32_t *ext, const uint32_t *bsk_hat,
                                 const uint2 *tw_lane, int n, int *err, int num_sms, cudaStream_t st)
{
    BrArgs a{abar, ext, bsk_hat, tw_lane, n, abar_stride, 1, T_EIGHTH, err};
    return launch_pair(a, num_sms, st, 1);
}

cudaError_t launch_quad_selftest(const uint16_t *abar, int abar_stride, uint32_t *ext, const uint32_t *bsk_hat,
                                 const uint2 *tw_lane, int n, int *err, int num_sms, cudaStream_t st)
{
    BrArgs a{abar, ext, bsk_hat, tw_lane, n, abar_stride, 1, T_EIGHTH, err};
    return launch_quad(a, num_sms, st, 1);
}

// Levels (or remainders) small enough for one CTA, CTA pair or CTA quad per ciphertext: on four
// SMs when they fit quad_max clusters, on two when they fit pair_max, else split.
static cudaError_t launch_small(const BrArgs &a, int num_sms, cudaStream_t st, int pair_max, int quad_max)
{
    if (a.jobs <= quad_max) return launch_quad(a, num_sms, st);
    return a.jobs <= pair_max ? launch_pair(a, num_sms, st) : launch_split(a, num_sms, st);
}

static cudaError_t launch_batched(const BrArgs &a, int num_sms, cudaStream_t st)
{
    const size_t smem = sizeof(BrSmem);
    cudaError_t e = cudaFuncSetAttribute(br_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int groups = (a.jobs + BR_SLOTS - 1) / BR_SLOTS;
    const int grid = groups < num_sms ? groups : num_sms;
    br_kernel<<<grid, BR_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_br(const uint16_t *abar, int abar_stride, uint32_t *ext, const uint32_t *bsk_hat,
                      const uint2 *tw_lane, int n, int jobs, uint32_t mu, int *err, int num_sms,
                      cudaStream_t st, int variant, int split_max, int tail_split, int pair_max, int quad_max,
                      int *launched)
{
    if (launched) *launched = 0;
    if (jobs <= 0) return cudaSuccess;
    BrArgs a{abar, ext, bsk_hat, tw_lane, n, abar_stride, jobs, mu, err};
    if (variant == BR_VARIANT_PAIR || variant == BR_VARIANT_QUAD) {
        if (launched) *launched = 1;
        return variant == BR_VARIANT_PAIR ? launch_pair(a, num_sms, st) : launch_quad(a, num_sms, st);
    }
    // Policy (measured on GB300): a split CTA finishes one ciphertext in about 4 ms, a batched
    // wave of up to 4 per SM takes 13.3-14.3 ms, so levels of up to two ciphertexts per SM run
    // split (one or two split waves) and larger ones batched, unless lp_autotune measured
    // another crossing on this device.  Levels that fit quad_max clusters of four SMs, or
    // pair_max clusters of two, run on the quad or paired kernel instead.
    const int smax = split_max > 0 ? split_max : 2 * num_sms;
    const int pmax = variant == BR_VARIANT_AUTO ? pair_max : 0;
    const int qmax = variant == BR_VARIANT_AUTO ? quad_max : 0;
    const bool split = variant == BR_VARIANT_SPLIT || (variant == BR_VARIANT_AUTO && jobs <= smax);
    if (split) {
        if (launched) *launched = 1;
        return launch_small(a, num_sms, st, pmax, qmax);
    }
    // A wider level whose last batched wave would be partial: with tail_split (chosen by the
    // autotuner), the full waves run batched and the remainder, when it is within the split
    // crossing, on the split (or paired) kernel, which finishes it in a fraction of a batched wave.
    const int wave = BR_SLOTS * num_sms;
    const int rem = jobs % wave;
    if (variant == BR_VARIANT_AUTO && tail_split && rem > 0 && rem <= smax && jobs > rem) {
        BrArgs head = a, tail = a;
        head.jobs = jobs - rem;
        tail.jobs = rem;
        tail.abar = abar + (size_t)head.jobs * abar_stride;
        tail.ext = ext + (size_t)head.jobs * EXT_STRIDE;
        cudaError_t e = launch_batched(head, num_sms, st);
        if (e == cudaSuccess) e = launch_small(tail, num_sms, st, pmax, qmax);
        if (launched) *launched = 2;
        return e;
    }
    if (launched) *launched = 1;
    return launch_batched(a, num_sms, st);
}

}  // namespace lp
