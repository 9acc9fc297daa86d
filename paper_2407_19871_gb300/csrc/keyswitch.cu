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

#include "ks_device.cuh"

namespace lp {

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

// Stand-alone key switch: CTA b takes batches b, b + gridDim.x, ...; with Sliced, the
// grid.y slices of the input coefficients add into pre-initialised outputs.
template <bool Sliced>
__global__ void __launch_bounds__(KS_THREADS, 1) ks_kernel(const uint32_t *ext, const KsJob *jobs, size_t njobs,
                                                           int dense_mux, uint32_t *out, const uint32_t *T, int n,
                                                           int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    KsSmem &sm = *reinterpret_cast<KsSmem *>(smem_raw);
    const size_t nbatches = (njobs + KS_CT - 1) / KS_CT;
    // Input-coefficient slice of this CTA (the whole range unless grid.y > 1), in blocks of
    // KS_ICH coefficients.
    const int nblk = RING_N / KS_ICH;
    const int i_begin = Sliced ? (int)(blockIdx.y * nblk / gridDim.y) * KS_ICH : 0;
    const int i_end = Sliced ? (int)((blockIdx.y + 1) * nblk / gridDim.y) * KS_ICH : RING_N;
    KsProducer pr;
    ks_setup(sm, pr, T, n);
    __syncthreads();
    uint32_t cseq = 0;
    bool ok = true;
    for (size_t bt = blockIdx.x; bt < nbatches && ok; bt += gridDim.x)
        ok = ks_unit<Sliced>(sm, pr, cseq, ext, jobs, njobs, dense_mux, out, n, bt, i_begin, i_end);
    if (!ok && threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
    if (threadIdx.x == 0 && !ks_drain(sm, pr)) atomicOr(err, DEV_ERR_TIMEOUT);
}

__global__ void ks_init_kernel(const uint32_t *ext, const KsJob *jobs, size_t njobs, int dense_mux, uint32_t *out, int n)
{
    ks_init_rows(ext, jobs, njobs, dense_mux, out, n, (size_t)blockIdx.x * blockDim.x + threadIdx.x,
                 (size_t)gridDim.x * blockDim.x);
}

cudaError_t launch_ks_table(const uint32_t *ksk, uint32_t *T, int n, int num_sms, cudaStream_t st)
{
    ks_table_kernel<<<num_sms * 8, 256, 0, st>>>(ksk, T, n);
    return cudaGetLastError();
}

size_t ks_smem_bytes() { return sizeof(KsSmem); }

static cudaError_t ks_run(const uint32_t *ext, const KsJob *jobs, size_t njobs, int dense_mux, uint32_t *out,
                          const uint32_t *T, int n, int *err, int num_sms, cudaStream_t st, bool sliced, int *launched)
{
    const size_t smem = sizeof(KsSmem);
    cudaError_t e = cudaFuncSetAttribute(ks_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ks_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const size_t nb = (njobs + KS_CT - 1) / KS_CT;
    if (sliced) {
        // Too few batches to fill the GPU: split the input coefficients (see above).
        const int slices = ks_slices(nb, num_sms);
        const size_t total = njobs * (size_t)(n + 1);
        const int ig = (int)std::min<size_t>((total + 255) / 256, (size_t)num_sms * 8);
        ks_init_kernel<<<ig, 256, 0, st>>>(ext, jobs, njobs, dense_mux, out, n);
        ks_kernel<true><<<dim3((unsigned)nb, (unsigned)slices), KS_THREADS, smem, st>>>(ext, jobs, njobs, dense_mux,
                                                                                        out, T, n, err);
        if (launched) *launched = 2;
        return cudaGetLastError();
    }
    const int grid = (int)(nb < (size_t)num_sms ? nb : (size_t)num_sms);
    ks_kernel<false><<<grid, KS_THREADS, smem, st>>>(ext, jobs, njobs, dense_mux, out, T, n, err);
    if (launched) *launched = 1;
    return cudaGetLastError();
}

cudaError_t launch_ks(const uint32_t *ext, const KsJob *jobs, size_t njobs, int dense_mux, uint32_t *out,
                      const uint32_t *T, int n, int *err, int num_sms, cudaStream_t st, int slice_max, int *launched)
{
    if (launched) *launched = 0;
    if (!njobs) return cudaSuccess;
    const size_t nb = (njobs + KS_CT - 1) / KS_CT;
    const bool sliced = slice_max > 0 ? nb <= (size_t)slice_max : slice_max < 0 ? false : 2 * nb < (size_t)num_sms;
    return ks_run(ext, jobs, njobs, dense_mux, out, T, n, err, num_sms, st, sliced, launched);
}

cudaError_t launch_ks_forced(const uint32_t *ext, size_t njobs, uint32_t *out, const uint32_t *T, int n, int *err,
                             int num_sms, cudaStream_t st, int sliced)
{
    if (!njobs) return cudaSuccess;
    return ks_run(ext, nullptr, njobs, 0, out, T, n, err, num_sms, st, sliced != 0, nullptr);
}

}  // namespace lp
