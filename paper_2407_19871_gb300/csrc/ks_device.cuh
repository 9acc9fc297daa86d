// Device side of the batched key switch, shared by the stand-alone key-switch kernel
// (keyswitch.cu) and the persistent circuit executor (blind_rotate.cu).  The algorithm and the
// digit-pair table are described in keyswitch.cu.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace lp {

constexpr int KS_CT = 64;          // outputs per batch (per CTA at a time)
constexpr int KS_THREADS = 256;    // 8 warps x 8 outputs
constexpr int KS_CPW = 8;          // outputs per warp
constexpr int KS_CPT = 20;         // words per lane (32 * 20 = 640 >= W)
constexpr int KS_WMAX = 640;
constexpr int KS_PAIRS = KS_T / 2; // digit pairs per coefficient
constexpr int KS_CROWS = 16;       // table rows per pair
constexpr int KS_RING = 3;
constexpr int KS_ICH = 32;         // input coefficients staged at a time

struct __align__(16) KsSmem {
    uint32_t ring[KS_RING][KS_CROWS * KS_WMAX];   // 120 KB
    uint32_t xs[KS_CT][KS_ICH + 1];
    uint32_t body[KS_CT];
    int src[KS_CT][2];
    int dst[KS_CT];
    uint64_t full_bar[KS_RING];
    uint64_t empty_bar[KS_RING];
    int abort;
};

// Table-chunk stream of one CTA: chunk q (a running count over the CTA's units) is table chunk
// base + (q - unit_start), one (i, jp) slice of 16 rows, for q < total (the current unit's end).
struct KsProducer {
    const uint32_t *T;
    uint32_t total, issued, chunk_words;
    uint32_t base, unit_start;
};

__device__ __forceinline__ void ks_produce(KsSmem &sm, KsProducer &pr, uint32_t upto)
{
    while (pr.issued < upto && pr.issued < pr.total) {
        const uint32_t q = pr.issued;
        const uint32_t s = q % KS_RING;
        if (q >= (uint32_t)KS_RING) {
            if (!mbar_wait_bounded(&sm.empty_bar[s], ((q - KS_RING) / KS_RING) & 1u, &sm.abort)) {
                *reinterpret_cast<volatile int *>(&sm.abort) = 1;
                return;
            }
        }
        const uint32_t chunk = pr.base + (q - pr.unit_start);   // (i, jp) of this chunk
        mbar_arrive_expect_tx(&sm.full_bar[s], pr.chunk_words * 4u);
        bulk_copy_g2s(sm.ring[s], pr.T + (size_t)chunk * pr.chunk_words, pr.chunk_words * 4u, &sm.full_bar[s]);
        pr.issued++;
    }
}

// Barriers and producer state of a CTA (thread 0 initialises; the caller synchronises after).
__device__ __forceinline__ void ks_setup(KsSmem &sm, KsProducer &pr, const uint32_t *T, int n)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < KS_RING; s++) {
            mbar_init(&sm.full_bar[s], 1);
            mbar_init(&sm.empty_bar[s], KS_THREADS / 32);
        }
        sm.abort = 0;
        mbar_fence_init();
    }
    pr.T = T;
    pr.chunk_words = (uint32_t)(KS_CROWS * ks_row_words(n));
    pr.total = pr.issued = pr.base = pr.unit_start = 0;
}

// One unit of key switching: the outputs of batch bt (jobs bt * KS_CT ...), over the input
// coefficients [i_begin, i_end) (a multiple of KS_ICH).  Not Sliced: the unit covers all N
// coefficients and writes the outputs.  Sliced: adds the unit's partial sums into outputs that
// hold (0, b') already (global atomics, exact mod 2^32 in any order).  Every thread of the CTA
// calls it; cseq (chunks consumed) and the producer's count run on across units.  Returns false,
// CTA-uniformly, once a wait has given up.
template <bool Sliced>
__device__ bool ks_unit(KsSmem &sm, KsProducer &pr, uint32_t &cseq, const uint32_t *ext, const KsJob *jobs,
                        size_t njobs, int dense_mux, uint32_t *out, int n, size_t bt, int i_begin, int i_end)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W = ks_row_words(n);
    const int V = n + 1;
    const bool producer = tid == 0;
    bool ok = true;
    // This unit's chunk stream: (i_end - i_begin) * KS_PAIRS chunks from table chunk i_begin * KS_PAIRS.
    pr.unit_start = pr.issued;
    pr.base = (uint32_t)i_begin * KS_PAIRS;
    pr.total = pr.issued + (uint32_t)(i_end - i_begin) * KS_PAIRS;
    if (producer) ks_produce(sm, pr, cseq + KS_RING);

    const size_t first = bt * KS_CT;
    if (tid < KS_CT) {
        const size_t g = first + tid;
        int e1 = -1, e2 = -1, o = -1;
        uint32_t bc = 0u, bsum = 0u;
        if (g < njobs) {
            if (jobs) {
                const KsJob J = jobs[g];
                e1 = J.e1; e2 = J.e2; bc = J.bconst; o = J.out;
            } else {
                e1 = (int)g; o = (int)g;
                if (dense_mux) { e2 = (int)(g + njobs); bc = T_EIGHTH; }
            }
            bsum = ext[(size_t)e1 * EXT_STRIDE + RING_N] + bc;
            if (e2 >= 0) bsum += ext[(size_t)e2 * EXT_STRIDE + RING_N];
        }
        sm.body[tid] = bsum;
        sm.src[tid][0] = e1;
        sm.src[tid][1] = e2;
        sm.dst[tid] = o;
    }
    __syncthreads();
    uint32_t acc[KS_CPW][KS_CPT];
#pragma unroll
    for (int c = 0; c < KS_CPW; c++)
#pragma unroll
        for (int q = 0; q < KS_CPT; q++)
            acc[c][q] = (!Sliced && lane + 32 * q == n) ? sm.body[warp * KS_CPW + c] : 0u;

    for (int i0 = i_begin; i0 < i_end; i0 += KS_ICH) {
        // Every decision to stop is taken CTA-wide, so that all threads meet the same barriers.
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        for (int e = tid; e < KS_CT * KS_ICH; e += KS_THREADS) {
            const int ct = e / KS_ICH, ii = e % KS_ICH;
            const int e1 = sm.src[ct][0], e2 = sm.src[ct][1];
            uint32_t v = 0u;
            if (e1 >= 0) {
                v = ext[(size_t)e1 * EXT_STRIDE + i0 + ii];
                if (e2 >= 0) v += ext[(size_t)e2 * EXT_STRIDE + i0 + ii];
            }
            sm.xs[ct][ii] = v + (1u << 15);
        }
        __syncthreads();
#pragma unroll 1
        for (int ii = 0; ii < KS_ICH; ii++) {
            uint32_t x[KS_CPW];
#pragma unroll
            for (int c = 0; c < KS_CPW; c++) x[c] = sm.xs[warp * KS_CPW + c][ii];
#pragma unroll 1
            for (int jp = 0; jp < KS_PAIRS; jp++) {
                const uint32_t rs = cseq % KS_RING;
                if (ok && !mbar_wait_bounded(&sm.full_bar[rs], (cseq / KS_RING) & 1u, &sm.abort)) {
                    ok = false;
                    if (lane == 0) *reinterpret_cast<volatile int *>(&sm.abort) = 1;
                }
                if (ok) {
                    const uint32_t *Tr = sm.ring[rs];
#pragma unroll
                    for (int c = 0; c < KS_CPW; c++) {
                        const uint32_t *row = Tr + ((x[c] >> (28 - 4 * jp)) & 15u) * W + lane;
#pragma unroll
                        for (int q = 0; q < KS_CPT; q++) acc[c][q] -= row[32 * q];
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&sm.empty_bar[rs]);
                    if (producer) ks_produce(sm, pr, cseq + KS_RING);
                }
                __syncwarp();
                cseq++;
            }
        }
    }
    ok = !__syncthreads_or(!ok);
    if (!ok) return false;
#pragma unroll
    for (int c = 0; c < KS_CPW; c++) {
        const int o = sm.dst[warp * KS_CPW + c];
        if (o < 0) continue;
#pragma unroll
        for (int q = 0; q < KS_CPT; q++) {
            const int col = lane + 32 * q;
            if (col >= V) continue;
            if (Sliced) atomicAdd(&out[(size_t)o * V + col], acc[c][q]);
            else out[(size_t)o * V + col] = acc[c][q];
        }
    }
    __syncthreads();
    return true;
}

// No bulk copy may still be in flight when the CTA exits: wait (bounded) for the last chunks
// the producer issued.  Returns false if a wait gave up.
__device__ __forceinline__ bool ks_drain(KsSmem &sm, const KsProducer &pr)
{
    bool ok = true;
    const uint32_t firstq = pr.issued > (uint32_t)KS_RING ? pr.issued - KS_RING : 0u;
    volatile int never = 0;
    for (uint32_t q = firstq; q < pr.issued; q++)
        ok &= mbar_wait_bounded(&sm.full_bar[q % KS_RING], (q / KS_RING) & 1u, &never);
    return ok;
}

// Sliced key switch: every output row starts as (0, b') (b' of its summed inputs plus bconst).
// Words [t0, total) by stride `step` (a grid-stride loop of the caller's threads).
__device__ __forceinline__ void ks_init_rows(const uint32_t *ext, const KsJob *jobs, size_t njobs, int dense_mux,
                                             uint32_t *out, int n, size_t t0, size_t step)
{
    const int V = n + 1;
    const size_t total = njobs * (size_t)V;
    for (size_t idx = t0; idx < total; idx += step) {
        const size_t g = idx / V;
        const int w = (int)(idx % V);
        int e1, e2 = -1, o;
        uint32_t bc = 0u;
        if (jobs) {
            const KsJob J = jobs[g];
            e1 = J.e1; e2 = J.e2; bc = J.bconst; o = J.out;
        } else {
            e1 = (int)g; o = (int)g;
            if (dense_mux) { e2 = (int)(g + njobs); bc = T_EIGHTH; }
        }
        uint32_t v = 0u;
        if (w == n) {
            v = ext[(size_t)e1 * EXT_STRIDE + RING_N] + bc;
            if (e2 >= 0) v += ext[(size_t)e2 * EXT_STRIDE + RING_N];
        }
        out[(size_t)o * V + w] = v;
    }
}

// Slices of the input coefficients for a key switch of nb batches on num_sms SMs (1 = none).
__host__ __device__ __forceinline__ int ks_slices(size_t nb, int num_sms)
{
    size_t s = (size_t)num_sms / (nb ? nb : 1);
    if (s > (size_t)(RING_N / KS_ICH)) s = RING_N / KS_ICH;
    return s < 1 ? 1 : (int)s;
}

}  // namespace lp
