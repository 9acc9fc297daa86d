// Integer-pipe throughput microbenchmark (stand-alone program).
//
// Measures, per SM and clock, the issue rate of the integer instructions the blind rotation
// is built from: 32-bit multiply-add (low half), 32-bit multiply high, 32x32 -> 64-bit
// multiply-add, one lazy Shoup modular product (mul.hi + 2 mul.lo), and a plain integer add.
// Every thread runs 8 independent dependency chains so that latency is hidden; 8 warps per
// SM sub-partition.  The results are the measured denominators behind the "alu" roofline.
//
// Build and run: python bench.py --int-peaks   (prints one JSON object)
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

constexpr int CHAINS = 8;
constexpr int ITERS = 4096;
constexpr int THREADS = 1024;

template <int OP>
__global__ void __launch_bounds__(THREADS) probe(uint32_t *out, uint32_t seed, long long *cycles)
{
    uint32_t v[CHAINS];
    unsigned long long w[CHAINS];
    const uint32_t a = seed * 2654435761u + threadIdx.x, b = seed ^ 0x9e3779b9u, p = 195198977u, wp = 3u * seed + 7u;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        v[c] = a + c * 7919u;
        w[c] = v[c];
    }
    __syncthreads();
    const long long t0 = clock64();
#pragma unroll 4
    for (int it = 0; it < ITERS; it++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) {
            if (OP == 0) v[c] = v[c] * b + a;                                   // IMAD (lo)
            if (OP == 1) v[c] = __umulhi(v[c], b) + a;                          // mul.hi (+ add)
            if (OP == 2) w[c] += (unsigned long long)(uint32_t)w[c] * b;        // 32x32 -> 64 multiply-add
            if (OP == 3) v[c] = v[c] * b - __umulhi(v[c], wp) * p;              // lazy Shoup product
            if (OP == 4) v[c] = v[c] + b + (uint32_t)c;                         // plain add
        }
    }
    const long long t1 = clock64();
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) r ^= v[c] ^ (uint32_t)w[c] ^ (uint32_t)(w[c] >> 32);
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int OP>
static double run(int sms, uint32_t *out, long long *cyc_d)
{
    probe<OP><<<sms, THREADS>>>(out, 1u, cyc_d);   // warm-up
    probe<OP><<<sms, THREADS>>>(out, 3u, cyc_d);
    cudaDeviceSynchronize();
    long long cyc[1024];
    cudaMemcpy(cyc, cyc_d, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
    double mean = 0;
    for (int i = 0; i < sms; i++) mean += (double)cyc[i];
    mean /= sms;
    // operations per SM per clock (one CTA per SM, THREADS threads)
    return (double)THREADS * ITERS * CHAINS / mean;
}

int main()
{
    int dev = 0, sms = 0, clk = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    uint32_t *out;
    long long *cyc;
    if (cudaMalloc(&out, sizeof(uint32_t) * sms * THREADS) != cudaSuccess) return 1;
    if (cudaMalloc(&cyc, sizeof(long long) * sms) != cudaSuccess) return 1;
    const double imad = run<0>(sms, out, cyc);
    const double mulhi = run<1>(sms, out, cyc);
    const double wide = run<2>(sms, out, cyc);
    const double shoup = run<3>(sms, out, cyc);
    const double add = run<4>(sms, out, cyc);
    const cudaError_t e = cudaGetLastError();
    printf("{\"sms\": %d, \"max_clock_mhz\": %.0f, \"per_sm_per_clock\": {\"imad_lo\": %.2f, \"mulhi_plus_add\": %.2f, "
           "\"mad_wide_u32\": %.2f, \"shoup_modmul\": %.2f, \"iadd\": %.2f}, \"error\": \"%s\"}\n",
           sms, clk / 1000.0, imad, mulhi, wide, shoup, add, cudaGetErrorString(e));
    cudaFree(out);
    cudaFree(cyc);
    return e == cudaSuccess ? 0 : 2;
}
