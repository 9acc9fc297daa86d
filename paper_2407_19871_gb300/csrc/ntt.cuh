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
// Values are kept lazily reduced (Harvey): forward inputs and outputs in [0, 4p), inverse
// inputs and outputs in [0, 2p).
#pragma once
#include "common.cuh"

namespace lp {

// Twiddles of the five register-local (warp-uniform) stages: [prime][dir][zeta index 1..31]
// as (w, floor(w 2^32 / p)); dir 0 = forward, 1 = inverse.  Only blind_rotate.cu includes
// this header, so these constant-memory objects exist once.
__constant__ uint2 c_tw[2][2][32];
// Montgomery constants -p^-1 mod 2^32, per prime.
__constant__ uint32_t c_pinv_neg[2];
// CRT: p0^-1 mod p1 with its Shoup companion modulo p1.
__constant__ uint2 c_crt;

// Lane-twiddle table in shared memory: [LANE_TW][32] (w, w') per prime and direction;
// slot q of stage s covers block (q - (2^(s-5) - 1)) of the lane's 16 / L blocks.
template <int PI>
__device__ __forceinline__ void bfly_fwd(uint32_t &x, uint32_t &y, uint32_t w, uint32_t wp)
{
    constexpr uint32_t P = Prime<PI>::p;
    uint32_t X = umin_u32(x, x - 2u * P);
    uint32_t T = shoup_mul<P>(y, w, wp);
    x = X + T;
    y = X - T + 2u * P;
}

template <int PI>
__device__ __forceinline__ void bfly_inv(uint32_t &x, uint32_t &y, uint32_t w, uint32_t wp)
{
    constexpr uint32_t P = Prime<PI>::p;
    uint32_t S = x + y;
    S = umin_u32(S, S - 2u * P);
    uint32_t D = x - y + 2u * P;
    x = S;
    y = shoup_mul<P>(D, w, wp);
}

// tbuf: this warp's 32 x 33 word transpose buffer; tw: the lane table of this prime and
// direction ([LANE_TW][32] uint2).
template <int PI>
__device__ __forceinline__ void ntt_fwd(uint32_t (&x)[32], uint32_t *tbuf, const uint2 *tw, int lane)
{
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const int D = 16 >> s;
#pragma unroll
        for (int k = 0; k < 32; k++) {
            if (k & D) continue;
            const uint2 z = c_tw[PI][0][(1 << s) + (k >> (5 - s))];
            bfly_fwd<PI>(x[k], x[k + D], z.x, z.y);
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
                bfly_fwd<PI>(x[k], x[k + L], z.x, z.y);
            }
        }
    }
}

template <int PI>
__device__ __forceinline__ void ntt_inv(uint32_t (&x)[32], uint32_t *tbuf, const uint2 *tw, int lane)
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
                bfly_inv<PI>(x[k], x[k + L], z.x, z.y);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 32; k++) tbuf[lane * 33 + k] = x[k];
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 32; k++) x[k] = tbuf[k * 33 + lane];
    __syncwarp();
#pragma unroll
    for (int s = 4; s >= 0; s--) {
        const int D = 16 >> s;
#pragma unroll
        for (int k = 0; k < 32; k++) {
            if (k & D) continue;
            const uint2 z = c_tw[PI][1][(1 << s) + (k >> (5 - s))];
            bfly_inv<PI>(x[k], x[k + D], z.x, z.y);
        }
    }
}

}  // namespace lp
