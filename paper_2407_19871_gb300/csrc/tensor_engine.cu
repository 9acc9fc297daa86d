// Alternative product engines on the tensor cores (row "alternative product engine" of the
// design: measured head to head against the NTT engine, not the default).  Both compute the
// same exact integers as the NTT engine and the key-switch table, so their outputs are the
// same bits.
//
// Blind rotation as a Toeplitz GEMM.  At step i every ciphertext of a batch multiplies its
// 6 digit polynomials by the same key rows BSK_i[r][c], so the external product of a batch
// of B ciphertexts is one matrix product
//     C [2N x B] = T_i [2N x 6N] . D [6N x B],
// T_i[c N + jo][r N + j] = the negacyclic matrix entry of BSK_i[r][c] (b[jo - j] for
// j <= jo, -b[N + jo - j] otherwise), D[r N + j][b] = digit r, coefficient j of ciphertext b.
// Products are kept exact by splitting both factors into small balanced limbs:
//   * bf16 engine: key words into 6 limbs of 6 bits ([-32, 32)), digits into 2 limbs
//     (d = 64 hi + lo, lo in [-32, 32), hi in [-8, 8]); every limb is an integer a bf16 holds
//     exactly, every product is exact in fp32, and every partial sum stays below
//     6144 (32 8 + 32 32) < 2^23, so the fp32 accumulation is exact in any order;
//   * int8 engine: key words into 4 limbs of 8 bits, digits into 2 limbs (d = 256 hi + lo,
//     hi in [-2, 2]); int32 accumulation, |sum| < 6144 (128 2 + 128 128) < 2^27.
// The limb pairs of equal weight 2^(s w) share one GEMM over a doubled K: with the key limbs
// stored in ascending order along K and D = [D_hi ; D_lo], C_w = [T_(w-1) | T_w] . D, so
// w = 1 .. W-1 is one strided-batched GEMM and w = 0 one more.  The pair whose weight is
// 2^32 or more vanishes mod 2^32.  A recombination kernel adds sum_w C_w 2^(s w) to ACC mod 2^32.
// T_i is rebuilt for each step (151 MB bf16, 50 MB int8), D and C live for one step.
//
// Key switch as a one-hot GEMM (int8).  H[(i, j, v - 1)][g] = 1 iff digit v_ij of output g
// equals v (v = 1, 2, 3); KSK words are split into 4 balanced 8-bit limbs stacked along M;
// C [4 W x G] = A . H with int32 sums (at most 8192 ones per column, |sum| < 2^20), and
// out = (0, b') - sum_limb C_limb 2^(8 limb) mod 2^32.  A is built from the digit-pair table
// (KSK[i][2jp][v] is table row 4v, KSK[i][2jp+1][v] table row v).
//
// The GEMMs are cuBLAS calls (plain library GEMMs); decomposition, Toeplitz construction,
// one-hot encoding and recombination are this file's kernels.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "runtime.h"

namespace lp {

constexpr int TC_BR_BATCH = 8192;   // ciphertexts per Toeplitz GEMM pass
constexpr int TC_KS_BATCH = 16384;  // outputs per one-hot GEMM pass
constexpr int TC_K = 6 * RING_N;    // digit rows
constexpr int TC_M = 2 * RING_N;    // output rows
constexpr int KS_K = RING_N * KS_T * (KS_BASE - 1);   // one-hot rows (v = 1..3)

template <typename E>
__device__ __forceinline__ E to_limb(int v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_limb<__nv_bfloat16>(int v) { return __int2bfloat16_rn(v); }
template <>
__device__ __forceinline__ int8_t to_limb<int8_t>(int v) { return (int8_t)v; }

__device__ __forceinline__ int acc_to_int(float v) { return __float2int_rn(v); }
__device__ __forceinline__ int acc_to_int(int v) { return v; }

// Balanced digit of x in base 2^S: x = lo + 2^S hi with lo in [-2^(S-1), 2^(S-1)).
template <int S>
__device__ __forceinline__ int balanced_low(long long x)
{
    constexpr long long H = 1LL << (S - 1);
    return (int)(((x + H) & ((1LL << S) - 1)) - H);
}

// ACC = (0, X^-bbar mu) per job.
__global__ void tc_init_kernel(uint32_t *acc, const uint16_t *abar, int abar_stride, int n, int jobs, uint32_t mu)
{
    const size_t total = (size_t)jobs * RING_N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx % RING_N);
        const size_t b = idx / RING_N;
        const int bb = abar[b * abar_stride + n];
        acc[b * TC_M + j] = 0u;
        const int e = (j + bb) & (2 * RING_N - 1);
        acc[b * TC_M + RING_N + j] = (e & RING_N) ? (0u - mu) : mu;
    }
}

// D = [D_hi ; D_lo] [2K x jobs] (column b contiguous): the gadget digits of X^abar_i ACC - ACC.
template <typename E, int S>
__global__ void tc_decompose_kernel(const uint32_t *acc, const uint16_t *abar, int abar_stride, int step, int jobs,
                                    E *D)
{
    const size_t total = (size_t)jobs * 2 * RING_N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx % RING_N);
        const int c = (int)((idx / RING_N) % 2);
        const size_t b = idx / (2 * RING_N);
        const int ab = abar[b * abar_stride + step];
        const uint32_t *A = acc + b * TC_M + (size_t)c * RING_N;
        const int ri = (j - ab) & (2 * RING_N - 1);
        uint32_t v = A[ri & (RING_N - 1)];
        v = (ri & RING_N) ? (0u - v) : v;
        const uint32_t u = v - A[j] + GADGET_OFF;
        E *col = D + b * (2 * (size_t)TC_K);
#pragma unroll
        for (int p = 0; p < LG; p++) {
            const int d = (int)((u >> (32 - BGBIT * (p + 1))) & 1023u) - 512;
            const int lo = balanced_low<S>(d);
            const int hi = (d - lo) >> S;
            const int row = (3 * c + p) * RING_N + j;
            col[row] = to_limb<E>(hi);
            col[TC_K + row] = to_limb<E>(lo);
        }
    }
}

// Stored A^T of step i: [L K x M] column-major, element (limb l, row r N + j) of output row m.
template <typename E, int S, int L>
__global__ void tc_toeplitz_kernel(const uint32_t *bsk, int step, E *T)
{
    const size_t total = (size_t)TC_M * TC_K;
    const size_t ktot = (size_t)L * TC_K;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx % RING_N);
        const int r = (int)((idx / RING_N) % ROWS);
        const int m = (int)(idx / TC_K);
        const int c = m / RING_N, jo = m % RING_N;
        const uint32_t *b = bsk + (((size_t)step * ROWS + r) * 2 + c) * RING_N;
        const uint32_t v = j <= jo ? b[jo - j] : 0u - b[RING_N + jo - j];
        long long x = v;
        E *dst = T + (size_t)m * ktot + (size_t)r * RING_N + j;
#pragma unroll
        for (int l = 0; l < L; l++) {
            const int d = balanced_low<S>(x);
            dst[(size_t)l * TC_K] = to_limb<E>(d);
            x = (x - d) >> S;
        }
    }
}

// ACC += sum_w C_w 2^(S w) (mod 2^32); C_w [M x jobs] column-major, stride M jobs.
template <typename CT, int S, int W>
__global__ void tc_recombine_kernel(const CT *C, uint32_t *acc, int jobs)
{
    const size_t total = (size_t)jobs * TC_M;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        uint32_t s = 0u;
#pragma unroll
        for (int w = 0; w < W; w++) s += (uint32_t)acc_to_int(C[(size_t)w * total + idx]) << (S * w);
        acc[idx] += s;
    }
}

// a'_0 = A_0, a'_j = -A_{N-j}, b' = B_0.
__global__ void tc_extract_kernel(const uint32_t *acc, uint32_t *ext, int jobs)
{
    const size_t total = (size_t)jobs * (RING_N + 1);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx % (RING_N + 1));
        const size_t b = idx / (RING_N + 1);
        const uint32_t *A = acc + b * TC_M;
        uint32_t v;
        if (j == RING_N) v = A[RING_N];
        else v = j == 0 ? A[0] : 0u - A[RING_N - j];
        ext[b * EXT_STRIDE + j] = v;
    }
}

// ---------------------------------------------------------------------------------
// Key switch: one-hot GEMM.
// ---------------------------------------------------------------------------------
// A [KS_K x 4 Wp] column-major from the digit-pair table.
__global__ void ks_onehot_key_kernel(const uint32_t *table, int8_t *A, int n)
{
    const int Wp = ks_row_words(n), V = n + 1;
    const size_t total = (size_t)KS_K * Wp;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % KS_K);
        const int w = (int)(idx / KS_K);
        const int v = k % 3 + 1, jj = (k / 3) % KS_T, i = k / (3 * KS_T);
        const int jp = jj / 2;
        const int row = (jj & 1) ? v : 4 * v;
        const uint32_t val = w < V ? table[(((size_t)i * (KS_T / 2) + jp) * 16 + row) * Wp + w] : 0u;
        long long x = val;
#pragma unroll
        for (int l = 0; l < 4; l++) {
            const int d = balanced_low<8>(x);
            A[(size_t)(l * Wp + w) * KS_K + k] = (int8_t)d;
            x = (x - d) >> 8;
        }
    }
}

// H [KS_K x G] one-hot digits of each output's N-LWE input; body and destination per output.
__global__ void ks_onehot_kernel(const uint32_t *ext, const KsJob *jobs, size_t first, size_t cnt, size_t njobs,
                                 int dense_mux, int8_t *H, uint32_t *body, int *dst)
{
    const size_t total = cnt * RING_N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % RING_N);
        const size_t gl = idx / RING_N, g = first + gl;
        int e1, e2 = -1, o;
        uint32_t bc = 0u;
        if (jobs) {
            const KsJob J = jobs[g];
            e1 = J.e1; e2 = J.e2; bc = J.bconst; o = J.out;
        } else {
            e1 = (int)g; o = (int)g;
            if (dense_mux) { e2 = (int)(g + njobs); bc = T_EIGHTH; }
        }
        uint32_t y = ext[(size_t)e1 * EXT_STRIDE + i];
        if (e2 >= 0) y += ext[(size_t)e2 * EXT_STRIDE + i];
        const uint32_t x = y + (1u << 15);
        uint32_t words[6];
#pragma unroll
        for (int q = 0; q < 6; q++) words[q] = 0u;
#pragma unroll
        for (int j = 0; j < KS_T; j++) {
            const uint32_t v = (x >> (30 - 2 * j)) & 3u;
            if (v) {
                const int k = j * 3 + (int)v - 1;     // 0 .. 23 within this coefficient
                words[k >> 2] |= 1u << (8 * (k & 3));
            }
        }
        uint32_t *h = reinterpret_cast<uint32_t *>(H + gl * KS_K + (size_t)i * 24);
#pragma unroll
        for (int q = 0; q < 6; q++) h[q] = words[q];
        if (i == 0) {
            uint32_t bs = ext[(size_t)e1 * EXT_STRIDE + RING_N] + bc;
            if (e2 >= 0) bs += ext[(size_t)e2 * EXT_STRIDE + RING_N];
            body[gl] = bs;
            dst[gl] = o;
        }
    }
}

// out[dst][w] = (w == n ? body : 0) - sum_l C[l Wp + w] 2^(8 l).
__global__ void ks_combine_kernel(const int *C, const uint32_t *body, const int *dst, uint32_t *out, int n, size_t cnt)
{
    const int Wp = ks_row_words(n), V = n + 1;
    const size_t total = cnt * V;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(idx % V);
        const size_t g = idx / V;
        const int *col = C + g * (size_t)(4 * Wp);
        uint32_t s = 0u;
#pragma unroll
        for (int l = 0; l < 4; l++) s += (uint32_t)col[l * Wp + w] << (8 * l);
        out[(size_t)dst[g] * V + w] = (w == n ? body[g] : 0u) - s;
    }
}

// ---------------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------------
static int grid_for(size_t total, int num_sms)
{
    const size_t g = (total + 255) / 256;
    const size_t cap = (size_t)num_sms * 16;
    return (int)(g < cap ? (g ? g : 1) : cap);
}

static int blas_fail(cublasStatus_t s, const char *what)
{
    return fail(LP_ECUDA, "%s: cuBLAS status %d", what, (int)s);
}

int tc_blas(lp_ctx *c, cudaStream_t st)
{
    if (!c->blas) {
        cublasHandle_t h;
        const cublasStatus_t s = cublasCreate(&h);
        if (s != CUBLAS_STATUS_SUCCESS) return blas_fail(s, "cublasCreate");
        c->blas = h;
    }
    const cublasStatus_t s = cublasSetStream(static_cast<cublasHandle_t>(c->blas), st);
    return s == CUBLAS_STATUS_SUCCESS ? LP_OK : blas_fail(s, "cublasSetStream");
}

void tc_release(lp_ctx *c)
{
    if (c->blas) cublasDestroy(static_cast<cublasHandle_t>(c->blas));
    c->blas = nullptr;
    for (DevBuf *b : {&c->tc_T, &c->tc_D, &c->tc_C, &c->tc_acc, &c->ks_A, &c->ks_H, &c->ks_C, &c->ks_aux})
        free_buf(*b);
}

template <typename E, typename CT, int S, int L>
static int br_tensor_pass(lp_ctx *c, const uint16_t *abar, int stride, uint32_t *ext, int jobs, uint32_t mu,
                          cudaDataType et, cudaDataType ct, cublasComputeType_t comp, cudaStream_t st)
{
    constexpr int W = L;   // weights 0 .. L-1 (the pair of weight 2^(S L) >= 2^32 vanishes)
    const int n = c->params.n;
    const size_t ktot = (size_t)L * TC_K;
    int rc = ensure_buf(c->tc_T, (size_t)TC_M * ktot * sizeof(E), "Toeplitz key limbs");
    if (!rc) rc = ensure_buf(c->tc_D, (size_t)TC_BR_BATCH * 2 * TC_K * sizeof(E), "digit limbs");
    if (!rc) rc = ensure_buf(c->tc_C, (size_t)W * TC_M * TC_BR_BATCH * sizeof(CT), "limb products");
    if (!rc) rc = ensure_buf(c->tc_acc, (size_t)TC_BR_BATCH * TC_M * sizeof(uint32_t), "accumulators");
    if (!rc) rc = tc_blas(c, st);
    if (rc) return rc;
    cublasHandle_t h = static_cast<cublasHandle_t>(c->blas);
    E *T = static_cast<E *>(c->tc_T.ptr);
    E *D = static_cast<E *>(c->tc_D.ptr);
    CT *C = static_cast<CT *>(c->tc_C.ptr);
    uint32_t *acc = static_cast<uint32_t *>(c->tc_acc.ptr);
    const uint32_t *bsk = static_cast<const uint32_t *>(c->bsk_coef.ptr);
    const CT one = (CT)1, zero = (CT)0;
    for (int off = 0; off < jobs; off += TC_BR_BATCH) {
        const int B = jobs - off < TC_BR_BATCH ? jobs - off : TC_BR_BATCH;
        const uint16_t *ab = abar + (size_t)off * stride;
        tc_init_kernel<<<grid_for((size_t)B * RING_N, c->num_sms), 256, 0, st>>>(acc, ab, stride, n, B, mu);
        c->launches++;
        for (int i = 0; i < n; i++) {
            tc_toeplitz_kernel<E, S, L><<<grid_for((size_t)TC_M * TC_K, c->num_sms), 256, 0, st>>>(bsk, i, T);
            tc_decompose_kernel<E, S><<<grid_for((size_t)B * 2 * RING_N, c->num_sms), 256, 0, st>>>(acc, ab, stride,
                                                                                                      i, B, D);
            c->launches += 2;
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "tensor-engine decomposition");
            // w = 0: T_0 . D_lo
            cublasStatus_t s = cublasGemmEx(h, CUBLAS_OP_T, CUBLAS_OP_N, TC_M, B, TC_K, &one, T, et, (int)ktot,
                                            D + TC_K, et, 2 * TC_K, &zero, C, ct, TC_M, comp, CUBLAS_GEMM_DEFAULT);
            if (s != CUBLAS_STATUS_SUCCESS) return blas_fail(s, "Toeplitz GEMM (weight 0)");
            // w = 1 .. W-1: [T_(w-1) | T_w] . [D_hi ; D_lo]
            s = cublasGemmStridedBatchedEx(h, CUBLAS_OP_T, CUBLAS_OP_N, TC_M, B, 2 * TC_K, &one, T, et, (int)ktot,
                                           (long long)TC_K, D, et, 2 * TC_K, 0LL, &zero, C + (size_t)TC_M * B, ct, TC_M,
                                           (long long)TC_M * B, W - 1, comp, CUBLAS_GEMM_DEFAULT);
            if (s != CUBLAS_STATUS_SUCCESS) return blas_fail(s, "Toeplitz GEMM (weights 1..)");
            tc_recombine_kernel<CT, S, W><<<grid_for((size_t)B * TC_M, c->num_sms), 256, 0, st>>>(C, acc, B);
            c->launches++;
        }
        tc_extract_kernel<<<grid_for((size_t)B * (RING_N + 1), c->num_sms), 256, 0, st>>>(
            acc, ext + (size_t)off * EXT_STRIDE, B);
        c->launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "tensor-engine blind rotation");
    }
    return LP_OK;
}

int run_br_tensor(lp_ctx *c, size_t jobs, uint32_t mu, cudaStream_t st)
{
    if (!c->bsk_coef.ptr) return fail(LP_ENOKEY, "the coefficient-domain bootstrapping key is not loaded");
    const uint16_t *abar = static_cast<const uint16_t *>(c->abar.ptr);
    uint32_t *ext = static_cast<uint32_t *>(c->ext.ptr);
    if (c->br_engine == LP_BR_TENSOR_BF16)
        return br_tensor_pass<__nv_bfloat16, float, 6, 6>(c, abar, abar_stride(c), ext, (int)jobs, mu, CUDA_R_16BF,
                                                          CUDA_R_32F, CUBLAS_COMPUTE_32F, st);
    return br_tensor_pass<int8_t, int, 8, 4>(c, abar, abar_stride(c), ext, (int)jobs, mu, CUDA_R_8I, CUDA_R_32I,
                                             CUBLAS_COMPUTE_32I, st);
}

int ks_tensor_prepare(lp_ctx *c, cudaStream_t st)
{
    const int n = c->params.n;
    int rc = ensure_buf(c->ks_A, (size_t)KS_K * 4 * ks_row_words(n), "one-hot key limbs");
    if (rc) return rc;
    ks_onehot_key_kernel<<<grid_for((size_t)KS_K * ks_row_words(n), c->num_sms), 256, 0, st>>>(
        static_cast<const uint32_t *>(c->ksk.ptr), static_cast<int8_t *>(c->ks_A.ptr), n);
    c->launches++;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LP_OK : cuda_fail(e, "one-hot key build");
}

int run_ks_tensor(lp_ctx *c, const KsJob *jobs, size_t njobs, int dense_mux, uint32_t *out, cudaStream_t st)
{
    const int n = c->params.n;
    const int Wp = ks_row_words(n), M = 4 * Wp;
    if (!c->ks_A.ptr) return fail(LP_ENOKEY, "the one-hot key is not built");
    int rc = ensure_buf(c->ks_H, (size_t)TC_KS_BATCH * KS_K, "one-hot digits");
    if (!rc) rc = ensure_buf(c->ks_C, (size_t)TC_KS_BATCH * M * sizeof(int), "one-hot products");
    if (!rc) rc = ensure_buf(c->ks_aux, (size_t)TC_KS_BATCH * 2 * sizeof(uint32_t), "one-hot bodies");
    if (!rc) rc = tc_blas(c, st);
    if (rc) return rc;
    cublasHandle_t h = static_cast<cublasHandle_t>(c->blas);
    int8_t *H = static_cast<int8_t *>(c->ks_H.ptr);
    int *C = static_cast<int *>(c->ks_C.ptr);
    uint32_t *body = static_cast<uint32_t *>(c->ks_aux.ptr);
    int *dst = reinterpret_cast<int *>(body + TC_KS_BATCH);
    const int one = 1, zero = 0;
    for (size_t off = 0; off < njobs; off += TC_KS_BATCH) {
        const size_t G = njobs - off < (size_t)TC_KS_BATCH ? njobs - off : (size_t)TC_KS_BATCH;
        ks_onehot_kernel<<<grid_for(G * RING_N, c->num_sms), 256, 0, st>>>(
            static_cast<const uint32_t *>(c->ext.ptr), jobs, off, G, njobs, dense_mux, H, body, dst);
        c->launches++;
        const cublasStatus_t s = cublasGemmEx(h, CUBLAS_OP_T, CUBLAS_OP_N, M, (int)G, KS_K, &one, c->ks_A.ptr,
                                              CUDA_R_8I, KS_K, H, CUDA_R_8I, KS_K, &zero, C, CUDA_R_32I, M,
                                              CUBLAS_COMPUTE_32I, CUBLAS_GEMM_DEFAULT);
        if (s != CUBLAS_STATUS_SUCCESS) return blas_fail(s, "one-hot key-switch GEMM");
        ks_combine_kernel<<<grid_for(G * (n + 1), c->num_sms), 256, 0, st>>>(C, body, dst, out, n, G);
        c->launches++;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "one-hot key switch");
    }
    return LP_OK;
}

}  // namespace lp
