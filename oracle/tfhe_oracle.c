/*
 * Plain CPU TFHE oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this library.  It shares no code with the CUDA path: it is a slow, literal
 * statement of what gate bootstrapping computes, against which every GPU output
 * ciphertext is compared bit for bit.
 *
 * All torus values are uint32_t (torus32: x / 2^32 mod 1, two's-complement wrap).
 * An LWE ciphertext is uint32_t[n+1] = a[0..n-1], b.  A TRLWE ciphertext (k = 1) is
 * two polynomials of degree < N: component 0 (mask a) and component 1 (body b).
 *
 * Sources: the paper (LocPIR, arXiv 2407.19871) fixes the encoding f(m) = m/4 - 1/8,
 * Encrypt, Decrypt (Section 2.2), HomAND as Bootstrap((0,-1/8) + c1 + c2) (Section 2.2),
 * and leaves the bootstrap itself to TFHE (Chillotti, Gama, Georgieva, Izabachene,
 * J. Cryptology 2020).  The bootstrap below follows that paper's gate bootstrapping:
 * modulus switch, blind rotation by CMux external products with the TRGSW
 * bootstrapping key, sample extraction, key switching.  The rounding offsets and
 * digit conventions are the ones this project fixes (see the design notes); the
 * paper prints none of them.
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_N 4096

/* ------------------------------------------------------------------------ */
/* Negacyclic products in Z_{2^32}[X]/(X^N + 1).                           */
/* ------------------------------------------------------------------------ */

/* Textbook definition: X^N = -1, so a term landing on degree i + k >= N wraps
 * to degree i + k - N with its sign flipped. */
void or_poly_mul_schoolbook(int N, const uint32_t *a, const uint32_t *b, uint32_t *out)
{
    uint32_t tmp[OR_MAX_N];
    memset(tmp, 0, sizeof(uint32_t) * (size_t)N);
    for (int i = 0; i < N; i++)
        for (int k = 0; k < N; k++) {
            uint32_t prod = a[i] * b[k];
            int d = i + k;
            if (d < N) tmp[d] += prod;
            else tmp[d - N] -= prod;
        }
    memcpy(out, tmp, sizeof(uint32_t) * (size_t)N);
}

#define KARA_BASE 16

/* Full (non-reduced) product r[0 .. 2n-1] of two length-n polynomials over
 * Z_{2^32}, by Karatsuba: (a0 + a1 Y)(b0 + b1 Y) with Y = X^h, middle term
 * (a0+a1)(b0+b1) - a0 b0 - a1 b1.  Only ring operations are used (no division),
 * so the identity holds exactly modulo 2^32.  ws needs 4n words. */
static void kara_full(const uint32_t *a, const uint32_t *b, uint32_t *r, int n, uint32_t *ws)
{
    if (n <= KARA_BASE) {
        for (int i = 0; i < 2 * n; i++) r[i] = 0;
        for (int i = 0; i < n; i++) {
            uint32_t ai = a[i];
            for (int k = 0; k < n; k++) r[i + k] += ai * b[k];
        }
        return;
    }
    int h = n / 2;
    kara_full(a, b, r, h, ws);             /* a0 b0 -> r[0 .. n-1]   */
    kara_full(a + h, b + h, r + n, h, ws); /* a1 b1 -> r[n .. 2n-1]  */
    uint32_t *sa = ws, *sb = ws + h, *m = ws + n, *wn = ws + 2 * n;
    for (int i = 0; i < h; i++) {
        sa[i] = a[i] + a[i + h];
        sb[i] = b[i] + b[i + h];
    }
    kara_full(sa, sb, m, h, wn);           /* (a0+a1)(b0+b1) -> m[0 .. n-1] */
    for (int i = 0; i < n; i++) m[i] -= r[i] + r[n + i];
    for (int i = 0; i < n; i++) r[h + i] += m[i];
}

/* out += a * b mod (X^N + 1), via the full Karatsuba product folded with X^N = -1. */
static void poly_mul_add_karatsuba(int N, const uint32_t *a, const uint32_t *b, uint32_t *out,
                                   uint32_t *ws /* 6N words */)
{
    uint32_t *full = ws;
    kara_full(a, b, full, N, ws + 2 * N);
    for (int j = 0; j < N; j++) out[j] += full[j] - full[j + N];
}

void or_poly_mul_karatsuba(int N, const uint32_t *a, const uint32_t *b, uint32_t *out)
{
    uint32_t *ws = (uint32_t *)malloc(sizeof(uint32_t) * 6 * (size_t)N);
    uint32_t *acc = (uint32_t *)calloc((size_t)N, sizeof(uint32_t));
    poly_mul_add_karatsuba(N, a, b, acc, ws);
    memcpy(out, acc, sizeof(uint32_t) * (size_t)N);
    free(acc);
    free(ws);
}

/* Multiply a polynomial by the monomial X^e (e taken mod 2N): coefficient j of
 * X^e * v is v[j - e] for j >= e, and -v[j - e + N] for j < e (when e < N); a
 * shift by e >= N is the shift by e - N negated. */
void or_poly_mul_monomial(int N, const uint32_t *v, int e, uint32_t *out)
{
    int twoN = 2 * N;
    e %= twoN;
    if (e < 0) e += twoN;
    for (int j = 0; j < N; j++) {
        int src = j - e;          /* in (-2N, N) */
        uint32_t sign_neg = 0;
        while (src < 0) { src += N; sign_neg ^= 1u; }
        out[j] = sign_neg ? (0u - v[src]) : v[src];
    }
}

/* ------------------------------------------------------------------------ */
/* Decompositions and modulus switch.                                       */
/* ------------------------------------------------------------------------ */

/* Signed gadget decomposition of a torus32 value into lg digits of base
 * Bg = 2^Bgbit, digit p (1-based) weighting 2^(32 - Bgbit p), each digit in
 * [-Bg/2, Bg/2).  Adding OFF = sum_p (Bg/2) 2^(32 - Bgbit p) + 2^(31 - Bgbit lg)
 * rounds to the nearest multiple of 2^(32 - Bgbit lg) and recentres every digit. */
void or_gadget_digits(int lg, int Bgbit, uint32_t x, int32_t *dig)
{
    uint32_t half = 1u << (Bgbit - 1);
    uint32_t off = 0;
    for (int p = 1; p <= lg; p++) off += half << (32 - Bgbit * p);
    if (Bgbit * lg < 32) off += 1u << (31 - Bgbit * lg);
    uint32_t u = x + off;
    uint32_t mask = (1u << Bgbit) - 1;
    for (int p = 1; p <= lg; p++)
        dig[p - 1] = (int32_t)((u >> (32 - Bgbit * p)) & mask) - (int32_t)half;
}

/* Key-switch digits: x rounded to t base-2^basebit digits (unsigned), digit j
 * (0-based) weighting 2^(32 - basebit (j+1)). */
void or_ks_digits(int t, int basebit, uint32_t x, uint32_t *v)
{
    uint32_t prec = 1u << (32 - basebit * t - 1);
    uint32_t y = x + prec;
    uint32_t mask = (1u << basebit) - 1;
    for (int j = 0; j < t; j++) v[j] = (y >> (32 - basebit * (j + 1))) & mask;
}

/* Round a torus32 value to Z_{2N}: nearest multiple of 1/(2N), half rounded up. */
uint32_t or_modswitch(uint32_t x, int N)
{
    int lg2 = 0;
    while ((1 << lg2) < 2 * N) lg2++;
    int shift = 32 - lg2;
    return (x + (1u << (shift - 1))) >> shift;
}

/* ------------------------------------------------------------------------ */
/* Client side: keys, encryption, phase.                                    */
/* ------------------------------------------------------------------------ */

/* phase(c) = b - <a, s> for LWE ciphertexts [count][n+1]. */
void or_lwe_phase(int n, size_t count, const uint8_t *s, const uint32_t *ct, uint32_t *phase)
{
    for (size_t g = 0; g < count; g++) {
        const uint32_t *c = ct + g * (size_t)(n + 1);
        uint32_t dot = 0;
        for (int i = 0; i < n; i++) dot += s[i] ? c[i] : 0u;
        phase[g] = c[n] - dot;
    }
}

/* Encrypt: (a, <a, s> + e + mu) with the given uniform masks a [count][n], noise
 * e [count] and messages mu [count] (torus32). */
void or_lwe_encrypt(int n, size_t count, const uint8_t *s, const uint32_t *mask,
                    const uint32_t *noise, const uint32_t *mu, uint32_t *out)
{
    for (size_t g = 0; g < count; g++) {
        const uint32_t *a = mask + g * (size_t)n;
        uint32_t *c = out + g * (size_t)(n + 1);
        uint32_t dot = 0;
        for (int i = 0; i < n; i++) {
            c[i] = a[i];
            dot += s[i] ? a[i] : 0u;
        }
        c[n] = dot + noise[g] + mu[g];
    }
}

/* Bootstrapping key: BSK[i] = TRGSW_S(s_i), rows r = c lg + p (c = 0 mask part,
 * c = 1 body part, p = 0 .. lg-1).  Row r is the zero-phase TRLWE sample
 * (a_r, a_r S + e_r) with s_i 2^(32 - Bgbit (p+1)) added to coefficient 0 of
 * component c.  Output layout [n][(k+1) lg][2][N]. */
void or_keygen_bsk(int n, int N, int lg, int Bgbit, const uint8_t *s, const uint8_t *S,
                   const uint32_t *mask, const uint32_t *noise, uint32_t *bsk)
{
    int rows = 2 * lg;
    uint32_t *Sp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    for (int j = 0; j < N; j++) Sp[j] = S[j];
    long long total = (long long)n * rows;
#pragma omp parallel
    {
        uint32_t *ws = (uint32_t *)malloc(sizeof(uint32_t) * 6 * (size_t)N);
#pragma omp for schedule(static)
        for (long long ir = 0; ir < total; ir++) {
            int i = (int)(ir / rows), r = (int)(ir % rows);
            const uint32_t *a = mask + (size_t)ir * N;
            const uint32_t *e = noise + (size_t)ir * N;
            uint32_t *out_a = bsk + ((size_t)ir * 2 + 0) * N;
            uint32_t *out_b = bsk + ((size_t)ir * 2 + 1) * N;
            for (int j = 0; j < N; j++) {
                out_a[j] = a[j];
                out_b[j] = e[j];
            }
            poly_mul_add_karatsuba(N, a, Sp, out_b, ws); /* b = a S + e */
            int c = r / lg, p = r % lg;
            uint32_t g = s[i] ? (1u << (32 - Bgbit * (p + 1))) : 0u;
            if (c == 0) out_a[0] += g;
            else out_b[0] += g;
        }
        free(ws);
    }
    free(Sp);
}

/* Key-switching key KSK[i][j][v] = LWE_s(v S_i 2^(32 - basebit (j+1))), layout
 * [N][t][2^basebit][n+1]; masks [N][t][2^basebit][n], noise [N][t][2^basebit]. */
void or_keygen_ksk(int n, int N, int t, int basebit, const uint8_t *s, const uint8_t *S,
                   const uint32_t *mask, const uint32_t *noise, uint32_t *ksk)
{
    int B = 1 << basebit;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < t; j++)
            for (int v = 0; v < B; v++) {
                size_t idx = ((size_t)i * t + j) * B + v;
                uint32_t mu = (uint32_t)v * (uint32_t)S[i] * (1u << (32 - basebit * (j + 1)));
                or_lwe_encrypt(n, 1, s, mask + idx * n, noise + idx, &mu, ksk + idx * (n + 1));
            }
}

/* ------------------------------------------------------------------------ */
/* Gate bootstrapping.                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n, N, lg, Bgbit, t, basebit;
} or_params;

/* Blind rotation of the mod-switched LWE bar[0 .. n] (bar[n] = switched body):
 * ACC = (0, X^(-bar_n) v) with v_j = mu for all j; for i = 0 .. n-1,
 * ACC <- ACC + BSK_i [x] ((X^(bar_i) - 1) ACC), the CMux external product.
 * A step with bar_i = 0 leaves ACC unchanged (its difference is 0, all digits 0)
 * and is skipped.  acc: [2][N]. */
static void blind_rotate(const or_params *P, const uint32_t *bsk, const uint32_t *bar,
                         uint32_t mu, uint32_t *acc, uint32_t *ws)
{
    int N = P->N, lg = P->lg, rows = 2 * lg;
    uint32_t *tv = ws;                       /* N   */
    uint32_t *rot = ws + N;                  /* N   */
    uint32_t *digp = ws + 2 * N;             /* rows * N */
    uint32_t *kws = ws + (2 + rows) * N;     /* 6N  */
    int32_t dig[32];

    for (int j = 0; j < N; j++) tv[j] = mu;
    memset(acc, 0, sizeof(uint32_t) * (size_t)N);
    or_poly_mul_monomial(N, tv, 2 * N - (int)bar[P->n], acc + N);

    for (int i = 0; i < P->n; i++) {
        int ab = (int)bar[i];
        if (ab == 0) continue;
        /* D = X^ab ACC - ACC, decomposed coefficient-wise into digit polynomials. */
        for (int c = 0; c < 2; c++) {
            or_poly_mul_monomial(N, acc + c * N, ab, rot);
            for (int j = 0; j < N; j++) {
                or_gadget_digits(lg, P->Bgbit, rot[j] - acc[c * N + j], dig);
                for (int p = 0; p < lg; p++) digp[(size_t)(c * lg + p) * N + j] = (uint32_t)dig[p];
            }
        }
        /* ACC += sum_r digit_r(X) * BSK_i[r]  (both components). */
        const uint32_t *bi = bsk + (size_t)i * rows * 2 * N;
        for (int r = 0; r < rows; r++)
            for (int c = 0; c < 2; c++)
                poly_mul_add_karatsuba(N, digp + (size_t)r * N, bi + ((size_t)r * 2 + c) * N,
                                       acc + c * N, kws);
    }
}

/* Sample extraction of coefficient 0: a'_0 = A_0, a'_j = -A_(N-j), b' = B_0. */
static void sample_extract(int N, const uint32_t *acc, uint32_t *out /* N+1 */)
{
    out[0] = acc[0];
    for (int j = 1; j < N; j++) out[j] = 0u - acc[N - j];
    out[N] = acc[N];
}

/* Key switch an N-LWE (a', b') to an n-LWE: out = (0, b') - sum_{i,j} KSK[i][j][v_ij]
 * with v_ij the base-2^basebit digits of a'_i; digit value 0 contributes nothing. */
static void key_switch(const or_params *P, const uint32_t *ksk, const uint32_t *in, uint32_t *out)
{
    int n = P->n, B = 1 << P->basebit;
    uint32_t v[32];
    memset(out, 0, sizeof(uint32_t) * (size_t)(n + 1));
    out[n] = in[P->N];
    for (int i = 0; i < P->N; i++) {
        or_ks_digits(P->t, P->basebit, in[i], v);
        for (int j = 0; j < P->t; j++) {
            if (v[j] == 0) continue;
            const uint32_t *row = ksk + (((size_t)i * P->t + j) * B + v[j]) * (n + 1);
            for (int w = 0; w <= n; w++) out[w] -= row[w];
        }
    }
}

/* blind_rotate scratch (2 + 2 lg + 6) N plus the accumulator 2N of bootstrap_extract. */
static size_t ws_words(const or_params *P) { return (size_t)(4 + 2 * P->lg + 6) * P->N + 64; }

/* One bootstrap of a (pre-combined) LWE up to the extracted N-LWE. */
static void bootstrap_extract(const or_params *P, const uint32_t *bsk, const uint32_t *lwe,
                              uint32_t mu, uint32_t *ext, uint32_t *ws)
{
    uint32_t bar[OR_MAX_N + 1];
    uint32_t *acc = ws;
    for (int i = 0; i <= P->n; i++) bar[i] = or_modswitch(lwe[i], P->N);
    blind_rotate(P, bsk, bar, mu, acc, ws + 2 * P->N);
    sample_extract(P->N, acc, ext);
}

/* Exported single steps (for pins). */
void or_blind_rotate(int n, int N, int lg, int Bgbit, const uint32_t *bsk,
                     const uint32_t *bar, uint32_t mu, uint32_t *acc)
{
    or_params P = {n, N, lg, Bgbit, 0, 0};
    uint32_t *ws = (uint32_t *)malloc(sizeof(uint32_t) * ws_words(&P));
    blind_rotate(&P, bsk, bar, mu, acc, ws);
    free(ws);
}

void or_sample_extract(int N, const uint32_t *acc, uint32_t *out) { sample_extract(N, acc, out); }

void or_key_switch(int n, int N, int t, int basebit, const uint32_t *ksk, const uint32_t *in,
                   uint32_t *out)
{
    or_params P = {n, N, 0, 0, t, basebit};
    key_switch(&P, ksk, in, out);
}

/* Gate identifiers (the same numbering as the library's public header). */
enum { OR_NAND = 0, OR_AND = 1, OR_OR = 2, OR_XOR = 3, OR_XNOR = 4, OR_NOT = 5, OR_MUX = 6 };

#define T_EIGHTH 0x20000000u   /* 1/8 */
#define T_QUARTER 0x40000000u  /* 1/4 */

/* Linear pre-combination of a two-input gate: (0, const) + ca * c1 + cb * c2. */
static int gate_lin(int op, uint32_t *cst, int *ca, int *cb)
{
    switch (op) {
    case OR_AND:  *cst = 0u - T_EIGHTH;  *ca = 1;  *cb = 1;  return 0;
    case OR_NAND: *cst = T_EIGHTH;       *ca = -1; *cb = -1; return 0;
    case OR_OR:   *cst = T_EIGHTH;       *ca = 1;  *cb = 1;  return 0;
    case OR_XOR:  *cst = T_QUARTER;      *ca = 2;  *cb = 2;  return 0;
    case OR_XNOR: *cst = 0u - T_QUARTER; *ca = -2; *cb = -2; return 0;
    default: return -1;
    }
}

static void lin_comb(int n, uint32_t cst, int ca, const uint32_t *c1, int cb, const uint32_t *c2,
                     uint32_t *out)
{
    for (int w = 0; w <= n; w++) out[w] = (uint32_t)ca * c1[w] + (uint32_t)cb * c2[w];
    out[n] += cst;
}

/* Evaluate count independent gates.  a, b, c, out: [count][n+1].  c is read by MUX
 * only (out = a ? b : c); NOT reads a only.  Independent gates run on nthreads
 * OpenMP threads.  bsk: [n][2 lg][2][N]; ksk: [N][t][2^basebit][n+1]. */
int or_gate_batch(int n, int N, int lg, int Bgbit, int t, int basebit, const uint32_t *bsk,
                  const uint32_t *ksk, int op, const uint32_t *a, const uint32_t *b,
                  const uint32_t *c, uint32_t *out, size_t count, int nthreads)
{
    or_params P = {n, N, lg, Bgbit, t, basebit};
    if (N > OR_MAX_N || n > OR_MAX_N) return -1;
    if (op < 0 || op > OR_MUX) return -1;
    if (op == OR_NOT) {
        for (size_t g = 0; g < count; g++)
            for (int w = 0; w <= n; w++) out[g * (n + 1) + w] = 0u - a[g * (n + 1) + w];
        return 0;
    }
    long long cnt = (long long)count;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        uint32_t *ws = (uint32_t *)malloc(sizeof(uint32_t) * (ws_words(&P) + 4 * (size_t)(N + 1) + 2 * (size_t)(n + 1)));
        uint32_t *ext1 = ws + ws_words(&P);
        uint32_t *ext2 = ext1 + (N + 1);
        uint32_t *sum = ext2 + (N + 1);
        uint32_t *lin = sum + 2 * (N + 1);
        uint32_t *lin2 = lin + (n + 1);
#pragma omp for schedule(dynamic, 1)
        for (long long g = 0; g < cnt; g++) {
            const uint32_t *ga = a + (size_t)g * (n + 1);
            const uint32_t *gb = b + (size_t)g * (n + 1);
            uint32_t *go = out + (size_t)g * (n + 1);
            if (op == OR_MUX) {
                const uint32_t *gc = c + (size_t)g * (n + 1);
                /* u1 = BR((0,-1/8) + a + b), u2 = BR((0,-1/8) - a + c);
                 * out = KS((0, 1/8) + u1 + u2) in dimension N. */
                lin_comb(n, 0u - T_EIGHTH, 1, ga, 1, gb, lin);
                lin_comb(n, 0u - T_EIGHTH, -1, ga, 1, gc, lin2);
                bootstrap_extract(&P, bsk, lin, T_EIGHTH, ext1, ws);
                bootstrap_extract(&P, bsk, lin2, T_EIGHTH, ext2, ws);
                for (int w = 0; w <= N; w++) sum[w] = ext1[w] + ext2[w];
                sum[N] += T_EIGHTH;
                key_switch(&P, ksk, sum, go);
            } else {
                uint32_t cst = 0; int ca = 0, cb = 0;
                gate_lin(op, &cst, &ca, &cb);
                lin_comb(n, cst, ca, ga, cb, gb, lin);
                bootstrap_extract(&P, bsk, lin, T_EIGHTH, ext1, ws);
                key_switch(&P, ksk, ext1, go);
            }
        }
        free(ws);
    }
    return 0;
}

/* Bootstrap only (no key switch): count pre-combined LWEs -> extracted N-LWEs. */
void or_bootstrap_extract_batch(int n, int N, int lg, int Bgbit, const uint32_t *bsk,
                                const uint32_t *lwe, uint32_t mu, uint32_t *ext, size_t count,
                                int nthreads)
{
    or_params P = {n, N, lg, Bgbit, 0, 0};
    long long cnt = (long long)count;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        uint32_t *ws = (uint32_t *)malloc(sizeof(uint32_t) * ws_words(&P));
#pragma omp for schedule(dynamic, 1)
        for (long long g = 0; g < cnt; g++)
            bootstrap_extract(&P, bsk, lwe + (size_t)g * (n + 1), mu, ext + (size_t)g * (N + 1), ws);
        free(ws);
    }
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
