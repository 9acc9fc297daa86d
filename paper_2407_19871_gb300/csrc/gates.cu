// Gate pre-combination + modulus switch, small helpers, and the client-side
// kernels (encryption, phase, key generation from given randomness).
#include "common.cuh"
#include "kernels.h"

namespace lp {

// ---------------------------------------------------------------------------------
// Pre-combination + modulus switch.
// A bootstrapped gate first forms the linear combination (0, const) + sum_k coef_k c_k
// (LocPIR Section 2.2, EvalGate: HomAND uses (0, -1/8) + c1 + c2), then rounds every
// coefficient to Z_2N: abar = ((x + 2^20) mod 2^32) >> 21 (half up).
// ---------------------------------------------------------------------------------

__device__ __forceinline__ void gate_coefs(int op, int half, uint32_t &cst, int &ca, int &cb, int &cc)
{
    cc = 0;
    switch (op) {
    case LP_AND: cst = 0u - T_EIGHTH; ca = 1; cb = 1; break;
    case LP_NAND: cst = T_EIGHTH; ca = -1; cb = -1; break;
    case LP_OR: cst = T_EIGHTH; ca = 1; cb = 1; break;
    case LP_XOR: cst = T_QUARTER; ca = 2; cb = 2; break;
    case LP_XNOR: cst = 0u - T_QUARTER; ca = -2; cb = -2; break;
    default:  // MUX: half 0 = (0,-1/8) + a + b, half 1 = (0,-1/8) - a + c
        cst = 0u - T_EIGHTH;
        if (half == 0) { ca = 1; cb = 1; }
        else { ca = -1; cb = 0; cc = 1; }
        break;
    }
}

// Dense gate batch: job jb < count * halves; gate g = jb % count, half = jb / count.
__global__ void precomb_dense_kernel(int op, const uint32_t *a, const uint32_t *b, const uint32_t *c, int n,
                                     size_t count, size_t jobs, uint16_t *abar, int abar_stride)
{
    const size_t total = jobs * (size_t)(n + 1);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t jb = idx / (n + 1);
        const int w = (int)(idx % (n + 1));
        const size_t g = jb % count;
        const int half = (int)(jb / count);
        uint32_t cst; int ca, cb, cc;
        gate_coefs(op, half, cst, ca, cb, cc);
        const size_t off = g * (size_t)(n + 1) + w;
        uint32_t x = (uint32_t)ca * a[off];
        if (cb) x += (uint32_t)cb * b[off];
        if (cc) x += (uint32_t)cc * c[off];
        if (w == n) x += cst;
        abar[jb * abar_stride + w] = modswitch_2048(x);
    }
}

// Plain modulus switch of given LWEs (lp_bootstrap_extract).
__global__ void modswitch_kernel(const uint32_t *lwe, int n, size_t jobs, uint16_t *abar, int abar_stride)
{
    const size_t total = jobs * (size_t)(n + 1);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t jb = idx / (n + 1);
        const int w = (int)(idx % (n + 1));
        abar[jb * abar_stride + w] = modswitch_2048(lwe[idx]);
    }
}

// Circuit mode: job records index a ciphertext pool [slots][n + 1].
__global__ void precomb_indexed_kernel(const BrJob *jobs, size_t njobs, const uint32_t *pool, int n,
                                       uint16_t *abar, int abar_stride)
{
    const size_t total = njobs * (size_t)(n + 1);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t jb = idx / (n + 1);
        const int w = (int)(idx % (n + 1));
        const BrJob J = jobs[jb];
        uint32_t x = 0u;
#pragma unroll
        for (int k = 0; k < 3; k++)
            if (J.coef[k] != 0) x += (uint32_t)J.coef[k] * pool[(size_t)J.in[k] * (n + 1) + w];
        if (w == n) x += J.bconst;
        abar[jb * abar_stride + w] = modswitch_2048(x);
    }
}

// ---------------------------------------------------------------------------------
// Small helpers: negated copy (NOT), trivial constants, pool gather with negation.
// ---------------------------------------------------------------------------------
__global__ void negate_kernel(const uint32_t *in, uint32_t *out, size_t words)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x)
        out[i] = 0u - in[i];
}

__global__ void gather_kernel(const uint32_t *pool, const int *slots, const uint8_t *neg, size_t cnt, int n,
                              uint32_t *out)
{
    const size_t total = cnt * (size_t)(n + 1);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t g = idx / (n + 1);
        const int w = (int)(idx % (n + 1));
        const uint32_t v = pool[(size_t)slots[g] * (n + 1) + w];
        out[idx] = neg[g] ? 0u - v : v;
    }
}

__global__ void trivial_kernel(uint32_t *dst, int n, uint32_t b)
{
    for (int w = threadIdx.x; w <= n; w += blockDim.x) dst[w] = (w == n) ? b : 0u;
}

// ---------------------------------------------------------------------------------
// Client side (device): Encrypt and phase, one warp per ciphertext; key generation.
// ---------------------------------------------------------------------------------
__global__ void lwe_encrypt_kernel(int n, const uint8_t *s, const uint32_t *mask, const uint32_t *noise,
                                   const uint32_t *mu, uint32_t *out, size_t count)
{
    const size_t warps = (size_t)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    for (size_t g = (size_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); g < count; g += warps) {
        const uint32_t *a = mask + g * (size_t)n;
        uint32_t *c = out + g * (size_t)(n + 1);
        uint32_t dot = 0u;
        for (int i = lane; i < n; i += 32) {
            const uint32_t ai = a[i];
            c[i] = ai;
            dot += s[i] ? ai : 0u;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0) c[n] = dot + noise[g] + mu[g];
    }
}

__global__ void lwe_phase_kernel(int n, const uint8_t *s, const uint32_t *ct, uint32_t *phase, size_t count)
{
    const size_t warps = (size_t)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    for (size_t g = (size_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); g < count; g += warps) {
        const uint32_t *c = ct + g * (size_t)(n + 1);
        uint32_t dot = 0u;
        for (int i = lane; i < n; i += 32) dot += s[i] ? c[i] : 0u;
#pragma unroll
        for (int o = 16; o; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0) phase[g] = c[n] - dot;
    }
}

// One CTA per TRGSW row (i, r): body = mask * S + noise (negacyclic, S binary), gadget
// term s_i 2^(32 - Bgbit (p+1)) on coefficient 0 of component c = r / lg.
__global__ void __launch_bounds__(256) keygen_bsk_kernel(int n, const uint8_t *s, const uint8_t *S,
                                                         const uint32_t *mask, const uint32_t *noise,
                                                         uint32_t *bsk)
{
    __shared__ uint32_t A[RING_N];
    __shared__ uint8_t Sk[RING_N];
    for (int j = threadIdx.x; j < RING_N; j += blockDim.x) Sk[j] = S[j];
    for (long ir = blockIdx.x; ir < (long)n * ROWS; ir += gridDim.x) {
        const int i = (int)(ir / ROWS), r = (int)(ir % ROWS);
        __syncthreads();
        for (int j = threadIdx.x; j < RING_N; j += blockDim.x) A[j] = mask[ir * RING_N + j];
        __syncthreads();
        uint32_t o[RING_N / 256];
#pragma unroll
        for (int q = 0; q < RING_N / 256; q++) o[q] = noise[ir * RING_N + threadIdx.x + 256 * q];
        for (int k = 0; k < RING_N; k++) {
            if (!Sk[k]) continue;
#pragma unroll
            for (int q = 0; q < RING_N / 256; q++) {
                const int j = threadIdx.x + 256 * q;
                const int d = j - k;
                o[q] += d >= 0 ? A[d] : 0u - A[d + RING_N];
            }
        }
        const int c = r / LG, p = r % LG;
        const uint32_t g = s[i] ? (1u << (32 - BGBIT * (p + 1))) : 0u;
        uint32_t *oa = bsk + (ir * 2 + 0) * RING_N;
        uint32_t *ob = bsk + (ir * 2 + 1) * RING_N;
#pragma unroll
        for (int q = 0; q < RING_N / 256; q++) {
            const int j = threadIdx.x + 256 * q;
            oa[j] = A[j] + ((c == 0 && j == 0) ? g : 0u);
            ob[j] = o[q] + ((c == 1 && j == 0) ? g : 0u);
        }
    }
}

__global__ void keygen_ksk_kernel(int n, const uint8_t *s, const uint8_t *S, const uint32_t *mask,
                                  const uint32_t *noise, uint32_t *ksk)
{
    const size_t total = (size_t)RING_N * KS_T * KS_BASE;
    const size_t warps = (size_t)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    for (size_t e = (size_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); e < total; e += warps) {
        const int i = (int)(e / (KS_T * KS_BASE));
        const int j = (int)((e / KS_BASE) % KS_T);
        const uint32_t v = (uint32_t)(e % KS_BASE);
        const uint32_t *a = mask + e * (size_t)n;
        uint32_t *c = ksk + e * (size_t)(n + 1);
        uint32_t dot = 0u;
        for (int w = lane; w < n; w += 32) {
            const uint32_t aw = a[w];
            c[w] = aw;
            dot += s[w] ? aw : 0u;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0) c[n] = dot + noise[e] + v * (uint32_t)S[i] * (1u << (32 - KS_BASEBIT * (j + 1)));
    }
}

// ---------------------------------------------------------------------------------
// Failure-detection self-test: a wait on an mbarrier that nothing completes.  The bounded
// wait gives up after limit_ns, the kernel records LP_ETIMEOUT in the error word and
// returns; no fault, no trap, and the context stays usable.
// ---------------------------------------------------------------------------------
__global__ void wait_probe_kernel(int *err, uint64_t limit_ns)
{
    __shared__ uint64_t bar;
    __shared__ int abort;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, &abort, limit_ns)) atomicOr(err, DEV_ERR_TIMEOUT);
}

// Algorithm 1 (Preprocess): the cloud turns the client's zero-phase samples into
// encryptions of its service bits by adding the encoding (0, f(bit)) to each.
__global__ void preprocess_kernel(int n, const uint32_t *zero, const uint8_t *bits, uint32_t *out, size_t count)
{
    const size_t total = count * (size_t)(n + 1);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t g = idx / (n + 1);
        const int w = (int)(idx % (n + 1));
        uint32_t v = zero[idx];
        if (w == n) v += bits[g] ? T_EIGHTH : 0u - T_EIGHTH;
        out[idx] = v;
    }
}

// ---------------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------------
static int grid_for(size_t work, int threads, int num_sms)
{
    size_t g = (work + threads - 1) / threads;
    const size_t cap = (size_t)num_sms * 16;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

cudaError_t launch_precomb_dense(int op, const uint32_t *a, const uint32_t *b, const uint32_t *c, int n,
                                 size_t count, uint16_t *abar, int abar_stride, int num_sms, cudaStream_t st)
{
    const size_t jobs = count * (op == LP_MUX ? 2 : 1);
    precomb_dense_kernel<<<grid_for(jobs * (n + 1), 256, num_sms), 256, 0, st>>>(op, a, b, c, n, count, jobs,
                                                                                  abar, abar_stride);
    return cudaGetLastError();
}

cudaError_t launch_modswitch(const uint32_t *lwe, int n, size_t jobs, uint16_t *abar, int abar_stride, int num_sms,
                             cudaStream_t st)
{
    modswitch_kernel<<<grid_for(jobs * (n + 1), 256, num_sms), 256, 0, st>>>(lwe, n, jobs, abar, abar_stride);
    return cudaGetLastError();
}

cudaError_t launch_precomb_indexed(const BrJob *jobs, size_t njobs, const uint32_t *pool, int n, uint16_t *abar,
                                   int abar_stride, int num_sms, cudaStream_t st)
{
    if (!njobs) return cudaSuccess;
    precomb_indexed_kernel<<<grid_for(njobs * (n + 1), 256, num_sms), 256, 0, st>>>(jobs, njobs, pool, n, abar,
                                                                                     abar_stride);
    return cudaGetLastError();
}

cudaError_t launch_negate(const uint32_t *in, uint32_t *out, size_t words, int num_sms, cudaStream_t st)
{
    if (!words) return cudaSuccess;
    negate_kernel<<<grid_for(words, 256, num_sms), 256, 0, st>>>(in, out, words);
    return cudaGetLastError();
}

cudaError_t launch_gather(const uint32_t *pool, const int *slots, const uint8_t *neg, size_t cnt, int n,
                          uint32_t *out, int num_sms, cudaStream_t st)
{
    if (!cnt) return cudaSuccess;
    gather_kernel<<<grid_for(cnt * (n + 1), 256, num_sms), 256, 0, st>>>(pool, slots, neg, cnt, n, out);
    return cudaGetLastError();
}

cudaError_t launch_trivial(uint32_t *dst, int n, uint32_t b, cudaStream_t st)
{
    trivial_kernel<<<1, 256, 0, st>>>(dst, n, b);
    return cudaGetLastError();
}

cudaError_t launch_lwe_encrypt(int n, const uint8_t *s, const uint32_t *mask, const uint32_t *noise,
                               const uint32_t *mu, uint32_t *out, size_t count, int num_sms, cudaStream_t st)
{
    if (!count) return cudaSuccess;
    lwe_encrypt_kernel<<<grid_for(count * 32, 256, num_sms), 256, 0, st>>>(n, s, mask, noise, mu, out, count);
    return cudaGetLastError();
}

cudaError_t launch_lwe_phase(int n, const uint8_t *s, const uint32_t *ct, uint32_t *phase, size_t count,
                             int num_sms, cudaStream_t st)
{
    if (!count) return cudaSuccess;
    lwe_phase_kernel<<<grid_for(count * 32, 256, num_sms), 256, 0, st>>>(n, s, ct, phase, count);
    return cudaGetLastError();
}

cudaError_t launch_keygen_bsk(int n, const uint8_t *s, const uint8_t *S, const uint32_t *mask,
                              const uint32_t *noise, uint32_t *bsk, int num_sms, cudaStream_t st)
{
    int grid = n * ROWS;
    if (grid > num_sms * 8) grid = num_sms * 8;
    keygen_bsk_kernel<<<grid, 256, 0, st>>>(n, s, S, mask, noise, bsk);
    return cudaGetLastError();
}

cudaError_t launch_keygen_ksk(int n, const uint8_t *s, const uint8_t *S, const uint32_t *mask,
                              const uint32_t *noise, uint32_t *ksk, int num_sms, cudaStream_t st)
{
    const size_t total = (size_t)RING_N * KS_T * KS_BASE;
    keygen_ksk_kernel<<<grid_for(total * 32, 256, num_sms), 256, 0, st>>>(n, s, S, mask, noise, ksk);
    return cudaGetLastError();
}

cudaError_t launch_wait_probe(int *err, uint64_t limit_ns, cudaStream_t st)
{
    wait_probe_kernel<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_preprocess(int n, const uint32_t *zero, const uint8_t *bits, uint32_t *out, size_t count,
                              int num_sms, cudaStream_t st)
{
    if (!count) return cudaSuccess;
    preprocess_kernel<<<grid_for(count * (n + 1), 256, num_sms), 256, 0, st>>>(n, zero, bits, out, count);
    return cudaGetLastError();
}

}  // namespace lp
