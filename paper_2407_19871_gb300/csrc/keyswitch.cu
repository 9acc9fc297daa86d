// Batched key switching.
//
// For an N-LWE (a', b') under S the key switch returns the n-LWE
//   out = (0, b') - sum_{i < N} sum_{j < t} KSK[i][j][v_ij],   v_ij = ((a'_i + 2^15) >> (30 - 2j)) & 3,
// where KSK[i][j][v] encrypts v S_i 2^(32 - 2(j+1)) under s and v = 0 contributes nothing
// (TFHE, Chillotti et al., J. Cryptology 2020; the paper defers the bootstrap to it).
//
// GB300 layout.  At key load the library folds each pair of digits (j, j+1) = (2 jp,
// 2 jp + 1) into one table row: T[i][jp][c] = KSK[i][2jp][c >> 2] + KSK[i][2jp+1][c & 3]
// (with the v = 0 rows read as zero) for the 16 values of c = 4 v_2jp + v_2jp+1, rows
// padded to W = n + 1 rounded up to 4 words.  A key switch then subtracts, per input
// coefficient i and digit pair jp, the single row T[i][jp][(x >> (28 - 4 jp)) & 15]: one
// shared-memory read and one subtraction per output word and digit pair, instead of a
// select chain per word and digit.  Addition mod 2^32 is exact, so the result equals the
// digit-by-digit sum bit for bit.
//
// A CTA takes KS_CT outputs and all W words.  Table chunks (one (i, jp): 16 rows, 40 KB at
// n = 630) stream L2 -> shared memory through cp.async.bulk into a KS_RING-slot ring with
// full / empty mbarriers; thread 0 is the producer.  Each warp owns 8 outputs; lane l owns
// words l + 32 q (q < KS_CPT), so every shared-memory read of the warp is conflict-free.
// 64 outputs per CTA (160 accumulators per thread, 255 registers, no spills) halve the
// table traffic from L2 against 32: a full batch of 65,536 takes 24.4 ms instead of 36.7.
// MUX jobs sum their two extracted samples and (0, 1/8) while their inputs are staged.
//
// Small batches.  A CTA streams the whole 165.7 MB table once per batch of KS_CT outputs,
// which takes about 2.5 ms however few outputs there are.  When the batches cannot fill
// half of the SMs, the input coefficients are split into up to 32 slices (grid.y): every
// CTA streams only its slice of the table and adds its partial sum into the output words
// with global atomics (exact mod 2^32 in any order), after ks_init_kernel has written (0, b').
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lp {

constexpr int KS_CT = 64;          // outputs per CTA
constexpr int KS_THREADS = 256;    // 8 warps x 8 outputs
constexpr int KS_CPW = 8;          // outputs per warp
constexpr int KS_CPT = 20;         // words per lane (32 * 20 = 640 >= W)
constexpr int KS_WMAX = 640;
constexpr int KS_PAIRS = KS_T / 2; // digit pairs per coefficient
constexpr int KS_CROWS = 16;       // table rows per pair
constexpr int KS_RING = 3;
constexpr int KS_ICH = 32;         // input coefficients staged at a time

__host__ __device__ size_t ks_table_words(int n) { return (size_t)RING_N * KS_PAIRS * KS_CROWS * ks_row_words(n); }

// Table from the key-switching key [N][t][4][n+1].
__global__ void ks_table_kernel(const uint32_t *ksk, uint32_t *T, int n)
{
    const int W = ks_row_words(n), V = n + 1;
    const size_t total = ks_table_words(n);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int col = (int)(idx % W);
        const size_t row = idx / W;              // (i * KS_PAIRS + jp) * 16 + c
        const int c = (int)(row % KS_CROWS);
        const size_t ijp = row / KS_CROWS;
        const int jp = (int)(ijp % KS_PAIRS);
        const size_t i = ijp / KS_PAIRS;
        uint32_t v = 0u;
        if (col < V) {
            const int hi = c >> 2, lo = c & 3;
            if (hi) v += ksk[((i * KS_T + 2 * jp) * KS_BASE + hi) * V + col];
            if (lo) v += ksk[((i * KS_T + 2 * jp + 1) * KS_BASE + lo) * V + col];
        }
        T[idx] = v;
    }
}

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

struct KsProducer {
    const uint32_t *T;
    uint32_t total, issued, chunk_words;
    uint32_t base, per_batch;   // first (i, jp) chunk of this CTA's slice, chunks per batch
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
        const uint32_t chunk = pr.base + q % pr.per_batch;   // (i, jp) of this chunk
        mbar_arrive_expect_tx(&sm.full_bar[s], pr.chunk_words * 4u);
        bulk_copy_g2s(sm.ring[s], pr.T + (size_t)chunk * pr.chunk_words, pr.chunk_words * 4u, &sm.full_bar[s]);
        pr.issued++;
    }
}

// Sliced: the grid.y slices of the input coefficients add into pre-initialised outputs.
template <bool Sliced>
__global__ void __launch_bounds__(KS_THREADS, 1) ks_kernel(const uint32_t *ext, const KsJob *jobs, size_t njobs,
                                                           int dense_mux, uint32_t *out, const uint32_t *T, int n,
                                                           int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    KsSmem &sm = *reinterpret_cast<KsSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W = ks_row_words(n);
    const int V = n + 1;
    const uint32_t chunk_words = (uint32_t)(KS_CROWS * W);
    const size_t nbatches = (njobs + KS_CT - 1) / KS_CT;
    // Input-coefficient slice of this CTA (the whole range unless grid.y > 1), in blocks of
    // KS_ICH coefficients.
    const int nblk = RING_N / KS_ICH;
    const int i_begin = Sliced ? (int)(blockIdx.y * nblk / gridDim.y) * KS_ICH : 0;
    const int i_end = Sliced ? (int)((blockIdx.y + 1) * nblk / gridDim.y) * KS_ICH : RING_N;
    const uint32_t per_batch = (uint32_t)(i_end - i_begin) * KS_PAIRS;

    if (tid == 0) {
        for (int s = 0; s < KS_RING; s++) {
            mbar_init(&sm.full_bar[s], 1);
            mbar_init(&sm.empty_bar[s], KS_THREADS / 32);
        }
        sm.abort = 0;
        mbar_fence_init();
    }
    __syncthreads();

    const bool producer = tid == 0;
    KsProducer pr;
    pr.T = T;
    pr.chunk_words = chunk_words;
    pr.issued = 0;
    pr.base = (uint32_t)i_begin * KS_PAIRS;
    pr.per_batch = per_batch;
    const size_t my_batches = blockIdx.x < nbatches ? (nbatches - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    pr.total = (uint32_t)(my_batches * per_batch);
    if (producer) ks_produce(sm, pr, KS_RING);

    uint32_t cseq = 0;
    bool ok = true;
    for (size_t bt = blockIdx.x; bt < nbatches; bt += gridDim.x) {
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
        // Every decision to stop is taken CTA-wide, so that all threads meet the same barriers.
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        uint32_t acc[KS_CPW][KS_CPT];
#pragma unroll
        for (int c = 0; c < KS_CPW; c++)
#pragma unroll
            for (int q = 0; q < KS_CPT; q++)
                acc[c][q] = (!Sliced && lane + 32 * q == n) ? sm.body[warp * KS_CPW + c] : 0u;

        for (int i0 = i_begin; i0 < i_end; i0 += KS_ICH) {
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
        if (!ok) break;
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
    }
    if (!ok && lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
    if (producer) {
        // No bulk copy may still be in flight when the CTA exits.
        const uint32_t firstq = pr.issued > (uint32_t)KS_RING ? pr.issued - KS_RING : 0u;
        volatile int never = 0;
        for (uint32_t q = firstq; q < pr.issued; q++)
            if (!mbar_wait_bounded(&sm.full_bar[q % KS_RING], (q / KS_RING) & 1u, &never))
                atomicOr(err, DEV_ERR_TIMEOUT);
    }
}

// Sliced key switch: every output row starts as (0, b') (b' of its summed inputs plus bconst).
__global__ void ks_init_kernel(const uint32_t *ext, const KsJob *jobs, size_t njobs, int dense_mux, uint32_t *out, int n)
{
    const int V = n + 1;
    const size_t total = njobs * (size_t)V;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
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

cudaError_t launch_ks_table(const uint32_t *ksk, uint32_t *T, int n, int num_sms, cudaStream_t st)
{
    ks_table_kernel<<<num_sms * 8, 256, 0, st>>>(ksk, T, n);
    return cudaGetLastError();
}

cudaError_t launch_ks(const uint32_t *ext, const KsJob *jobs, size_t njobs, int dense_mux, uint32_t *out,
                      const uint32_t *T, int n, int *err, int num_sms, cudaStream_t st)
{
    if (!njobs) return cudaSuccess;
    const size_t smem = sizeof(KsSmem);
    cudaError_t e = cudaFuncSetAttribute(ks_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ks_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const size_t nb = (njobs + KS_CT - 1) / KS_CT;
    if (2 * nb < (size_t)num_sms) {
        // Too few batches to fill the GPU: split the input coefficients (see above).
        const int slices = (int)std::min<size_t>((size_t)(RING_N / KS_ICH), (size_t)num_sms / nb);
        const size_t total = njobs * (size_t)(n + 1);
        const int ig = (int)std::min<size_t>((total + 255) / 256, (size_t)num_sms * 8);
        ks_init_kernel<<<ig, 256, 0, st>>>(ext, jobs, njobs, dense_mux, out, n);
        ks_kernel<true><<<dim3((unsigned)nb, (unsigned)slices), KS_THREADS, smem, st>>>(ext, jobs, njobs, dense_mux,
                                                                                        out, T, n, err);
        return cudaGetLastError();
    }
    const int grid = (int)(nb < (size_t)num_sms ? nb : (size_t)num_sms);
    ks_kernel<false><<<grid, KS_THREADS, smem, st>>>(ext, jobs, njobs, dense_mux, out, T, n, err);
    return cudaGetLastError();
}

}  // namespace lp
