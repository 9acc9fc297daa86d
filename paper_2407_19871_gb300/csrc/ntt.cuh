// Warp-level negacyclic NTT of length 1024 modulo one of the two NTT primes.
//
// One warp holds one polynomial, 32 coefficients per lane, in one of two layouts:
//   layout A: lane t, register k holds index j = t + 32 k;
//   layout B: lane t, register k holds index j = 32 t + k.
// The forward transform is the Cooley-Tukey negacyclic NTT (psi a primitive 2048-th root
// of unity mod p, zeta[z] = psi^bitrev10(z)): stage s (s = 0..9) pairs indices j, j + L
// with L = 512 >> s and twiddle zeta[2^s + j / (2L)].  Stages 0..4 pair registers of the
// same lane in layout A and use warp-uniform twiddles (constant memory); the warp then
// transposes to layout B through shared memory and runs stages 5..9 on registers again,
// with lane-dependent twiddles from a shared table.  The output stays in layout B in the
// transform's own (bit-reversed) order; pointwise products only need both operands in
// the same order.  The inverse runs the Gentleman-Sande butterflies in the opposite order
// (layout B, transpose, layout A) with inverse twiddles, leaving natural order in layout A.
// Its 1/N factor is folded into the transform-domain bootstrapping key.
//
// The prime is a runtime (warp-uniform) value, so both primes share one copy of the code.
//
// Value ranges.  Forward: no reduction inside the transform.  A Cooley-Tukey butterfly
// maps (x, y) with x, y < B to x + t, x - t + 2p with t = y w mod p in [0, 2p) (lazy Shoup
// product, valid for any y < 2^32), so the bound grows by 2p per stage: inputs in [0, 2p)
// leave the 10 stages below 22p < 2^32 (p < 2^32 / 22), and one lazy Shoup reduction by 1
// brings the output back to [0, 2p).  Inverse (Harvey): inputs and outputs in [0, 2p).
#pragma once
#include "common.cuh"

namespace lp {

// Twiddles of the five register-local (warp-uniform) stages: [prime][dir][zeta index 1..31]
// as (w, floor(w 2^32 / p)); dir 0 = forward, 1 = inverse.  Only blind_rotate.cu includes
// this header, so these constant-memory objects exist once.
__constant__ uint2 c_tw[2][2][32];
// Per prime: p, 2p, -p^-1 mod 2^32 (Montgomery), floor(2^32 / p) (reduction by 1).
__constant__ uint4 c_prm[2];
// CRT: p0^-1 mod p1 with its Shoup companion modulo p1.
__constant__ uint2 c_crt;

struct PrimeK {
    uint32_t p, p2, pinv_neg, rp;
};

__device__ __forceinline__ PrimeK prime_k(int pi)
{
    const uint4 v = c_prm[pi];
    return PrimeK{v.x, v.y, v.z, v.w};
}

// Lazy Shoup product with a runtime modulus: y w mod p in [0, 2p) for any y < 2^32.
__device__ __forceinline__ uint32_t shoup_mul_r(uint32_t y, uint32_t w, uint32_t wp, uint32_t p)
{
    return y * w - __umulhi(y, wp) * p;
}

__device__ __forceinline__ void bfly_fwd(uint32_t &x, uint32_t &y, uint32_t w, uint32_t wp, const PrimeK &k)
{
    const uint32_t t = shoup_mul_r(y, w, wp, k.p);
    y = x - t + k.p2;
    x = x + t;
}

__device__ __forceinline__ void bfly_inv(uint32_t &x, uint32_t &y, uint32_t w, uint32_t wp, const PrimeK &k)
{
    uint32_t s = x + y;
    s = umin_u32(s, s - k.p2);
    const uint32_t d = x - y + k.p2;
    x = s;
    y = shoup_mul_r(d, w, wp, k.p);
}

// tbuf: this warp's 32 x 33 word transpose buffer; tw: the lane table of this prime and
// direction ([LANE_TW][32] (w, w')); slot base + b of stage s is block b of the lane's
// 16 / L blocks (base = 2^(s-5) - 1).  Input in [0, 2p) (layout A); output (layout B) in
// [0, 2p) with Reduce, else in [0, 22p) (the caller reduces later, more cheaply).
template <bool Reduce>
__device__ __forceinline__ void ntt_fwd(uint32_t (&x)[32], uint32_t *tbuf, const uint2 *tw, int lane, int pi,
                                        const PrimeK &K)
{
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const int D = 16 >> s;
#pragma unroll
        for (int k = 0; k < 32; k++) {
            if (k & D) continue;
            const uint2 z = c_tw[pi][0][(1 << s) + (k >> (5 - s))];
            bfly_fwd(x[k], x[k + D], z.x, z.y, K);
        }
    }
#pragma unroll
    for (int k = 0; k < 32; k++) tbuf[k * 33 + lane] = x[k];
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 32; k++) x[k] = tbuf[lane * 33 + k];
    __syncwarp();
#pragma unroll
    for (int s = 5; s < 10; s++) {
        const int L = 16 >> (s - 5);
        const int base = (1 << (s - 5)) - 1;
#pragma unroll
        for (int b = 0; b < (16 / L); b++) {
            const uint2 z = tw[(base + b) * 32 + lane];
#pragma unroll
            for (int o = 0; o < L; o++) {
                const int k = b * 2 * L + o;
                bfly_fwd(x[k], x[k + L], z.x, z.y, K);
            }
        }
    }
    if (Reduce) {
#pragma unroll
        for (int k = 0; k < 32; k++) x[k] -= __umulhi(x[k], K.rp) * K.p;
    }
}

// Inverse transform of NP polynomials together (butterflies of the same position interleaved,
// for instruction-level parallelism).  Input in [0, 2p) (layout B), output in [0, 2p) (layout A).
template <int NP>
__device__ __forceinline__ void ntt_inv_multi(uint32_t (&x)[NP][32], uint32_t *tbuf, const uint2 *tw, int lane,
                                              int pi, const PrimeK &K)
{
#pragma unroll
    for (int s = 9; s >= 5; s--) {
        const int L = 16 >> (s - 5);
        const int base = (1 << (s - 5)) - 1;
#pragma unroll
        for (int b = 0; b < (16 / L); b++) {
            const uint2 z = tw[(base + b) * 32 + lane];
#pragma unroll
            for (int o = 0; o < L; o++) {
                const int k = b * 2 * L + o;
#pragma unroll
                for (int q = 0; q < NP; q++) bfly_inv(x[q][k], x[q][k + L], z.x, z.y, K);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NP; q++) {
#pragma unroll
        for (int k = 0; k < 32; k++) tbuf[lane * 33 + k] = x[q][k];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 32; k++) x[q][k] = tbuf[k * 33 + lane];
        __syncwarp();
    }
#pragma unroll
    for (int s = 4; s >= 0; s--) {
        const int D = 16 >> s;
#pragma unroll
        for (int k = 0; k < 32; k++) {
            if (k & D) continue;
            const uint2 z = c_tw[pi][1][(1 << s) + (k >> (5 - s))];
#pragma unroll
            for (int q = 0; q < NP; q++) bfly_inv(x[q][k], x[q][k + D], z.x, z.y, K);
        }
    }
}

// Montgomery reduction: T 2^-32 mod p, as the exact value (T + m p) / 2^32 < T / 2^32 + p
// (m = -T p^-1 mod 2^32); in [0, 2p) for T < 2^32 p.  The caller keeps it below 2^32.
__device__ __forceinline__ uint32_t redc64(unsigned long long T, const PrimeK &K)
{
    const uint32_t lo = (uint32_t)T, hi = (uint32_t)(T >> 32);
    const uint32_t m = lo * K.pinv_neg;
    return hi + __umulhi(m, K.p) + (lo != 0u ? 1u : 0u);
}

}  // namespace lp
