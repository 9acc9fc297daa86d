// Key files: the bootstrapping and key-switching keys with a SHA-256 checksum.
//
// Layout (little endian):
//   "LPKEYS01" | u32 version = 1 | 7 x i32 parameters (n, N, k, Bgbit, lg, basebit, t) |
//   u64 bsk words | u64 ksk words | 32-byte SHA-256 of the two key arrays | bsk | ksk
// SHA-256 is the hash of FIPS 180-4, written here from that specification.
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "runtime.h"

namespace {

struct Sha256 {
    uint32_t h[8];
    uint64_t len = 0;
    uint8_t buf[64];
    size_t fill = 0;

    static uint32_t rotr(uint32_t x, int r) { return (x >> r) | (x << (32 - r)); }

    Sha256()
    {
        static const uint32_t h0[8] = {0x6a09e667u, 0xbb67ae85u, 0x3c6ef372u, 0xa54ff53au,
                                       0x510e527fu, 0x9b05688cu, 0x1f83d9abu, 0x5be0cd19u};
        memcpy(h, h0, sizeof h);
    }

    void block(const uint8_t *p)
    {
        static const uint32_t K[64] = {
            0x428a2f98u, 0x71374491u, 0xb5c0fbcfu, 0xe9b5dba5u, 0x3956c25bu, 0x59f111f1u, 0x923f82a4u, 0xab1c5ed5u,
            0xd807aa98u, 0x12835b01u, 0x243185beu, 0x550c7dc3u, 0x72be5d74u, 0x80deb1feu, 0x9bdc06a7u, 0xc19bf174u,
            0xe49b69c1u, 0xefbe4786u, 0x0fc19dc6u, 0x240ca1ccu, 0x2de92c6fu, 0x4a7484aau, 0x5cb0a9dcu, 0x76f988dau,
            0x983e5152u, 0xa831c66du, 0xb00327c8u, 0xbf597fc7u, 0xc6e00bf3u, 0xd5a79147u, 0x06ca6351u, 0x14292967u,
            0x27b70a85u, 0x2e1b2138u, 0x4d2c6dfcu, 0x53380d13u, 0x650a7354u, 0x766a0abbu, 0x81c2c92eu, 0x92722c85u,
            0xa2bfe8a1u, 0xa81a664bu, 0xc24b8b70u, 0xc76c51a3u, 0xd192e819u, 0xd6990624u, 0xf40e3585u, 0x106aa070u,
            0x19a4c116u, 0x1e376c08u, 0x2748774cu, 0x34b0bcb5u, 0x391c0cb3u, 0x4ed8aa4au, 0x5b9cca4fu, 0x682e6ff3u,
            0x748f82eeu, 0x78a5636fu, 0x84c87814u, 0x8cc70208u, 0x90befffau, 0xa4506cebu, 0xbef9a3f7u, 0xc67178f2u};
        uint32_t w[64];
        for (int i = 0; i < 16; i++)
            w[i] = (uint32_t)p[4 * i] << 24 | (uint32_t)p[4 * i + 1] << 16 | (uint32_t)p[4 * i + 2] << 8 | p[4 * i + 3];
        for (int i = 16; i < 64; i++) {
            const uint32_t s0 = rotr(w[i - 15], 7) ^ rotr(w[i - 15], 18) ^ (w[i - 15] >> 3);
            const uint32_t s1 = rotr(w[i - 2], 17) ^ rotr(w[i - 2], 19) ^ (w[i - 2] >> 10);
            w[i] = w[i - 16] + s0 + w[i - 7] + s1;
        }
        uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
        for (int i = 0; i < 64; i++) {
            const uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
            const uint32_t ch = (e & f) ^ (~e & g);
            const uint32_t t1 = hh + S1 + ch + K[i] + w[i];
            const uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
            const uint32_t mj = (a & b) ^ (a & c) ^ (b & c);
            const uint32_t t2 = S0 + mj;
            hh = g; g = f; f = e; e = d + t1; d = c; c = b; b = a; a = t1 + t2;
        }
        h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
    }

    void update(const void *data, size_t n)
    {
        const uint8_t *p = static_cast<const uint8_t *>(data);
        len += n;
        while (n) {
            const size_t take = std::min(n, 64 - fill);
            memcpy(buf + fill, p, take);
            fill += take;
            p += take;
            n -= take;
            if (fill == 64) {
                block(buf);
                fill = 0;
            }
        }
    }

    void final(uint8_t out[32])
    {
        const uint64_t bits = len * 8;
        const uint8_t one = 0x80, zero = 0;
        update(&one, 1);
        while (fill != 56) update(&zero, 1);
        uint8_t L[8];
        for (int i = 0; i < 8; i++) L[i] = (uint8_t)(bits >> (56 - 8 * i));
        update(L, 8);
        for (int i = 0; i < 8; i++)
            for (int j = 0; j < 4; j++) out[4 * i + j] = (uint8_t)(h[i] >> (24 - 8 * j));
    }
};

const char MAGIC[8] = {'L', 'P', 'K', 'E', 'Y', 'S', '0', '1'};

struct Header {
    char magic[8];
    uint32_t version;
    int32_t params[7];
    uint64_t bsk_words, ksk_words;
    uint8_t sha[32];
};

size_t bsk_words_of(const lp_params &p) { return (size_t)p.n * 2 * p.lg * 2 * p.N; }
size_t ksk_words_of(const lp_params &p) { return (size_t)p.N * p.t * (1u << p.basebit) * (p.n + 1); }

// Read and verify a key file; on success fills params and the two key arrays.
int read_keys(const char *path, lp_params *P, std::vector<uint32_t> *bsk, std::vector<uint32_t> *ksk)
{
    FILE *f = fopen(path, "rb");
    if (!f) return lp::fail(LP_EINVAL, "cannot open key file %s", path);
    Header h;
    if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, MAGIC, 8) != 0 || h.version != 1) {
        fclose(f);
        return lp::fail(LP_ECORRUPT, "%s is not a version-1 key file", path);
    }
    lp_params p{h.params[0], h.params[1], h.params[2], h.params[3], h.params[4], h.params[5], h.params[6]};
    if (p.n < 1 || p.n > 4096 || p.N < 1 || p.N > 65536 || p.lg < 1 || p.lg > 8 || p.t < 1 || p.t > 32 ||
        p.basebit < 1 || p.basebit > 8 || h.bsk_words != bsk_words_of(p) || h.ksk_words != ksk_words_of(p)) {
        fclose(f);
        return lp::fail(LP_ECORRUPT, "%s: header sizes do not match its parameters", path);
    }
    if (bsk) bsk->resize(h.bsk_words);
    if (ksk) ksk->resize(h.ksk_words);
    std::vector<uint32_t> tmp;
    std::vector<uint32_t> *B = bsk ? bsk : &tmp;
    if (!bsk) B->resize(h.bsk_words);
    bool ok = fread(B->data(), 4, h.bsk_words, f) == h.bsk_words;
    Sha256 sh;
    sh.update(B->data(), h.bsk_words * 4);
    if (!bsk) B->clear();
    std::vector<uint32_t> tmp2;
    std::vector<uint32_t> *K = ksk ? ksk : &tmp2;
    if (!ksk) K->resize(h.ksk_words);
    ok = ok && fread(K->data(), 4, h.ksk_words, f) == h.ksk_words;
    fclose(f);
    if (!ok) return lp::fail(LP_ECORRUPT, "%s is truncated", path);
    sh.update(K->data(), h.ksk_words * 4);
    uint8_t d[32];
    sh.final(d);
    if (memcmp(d, h.sha, 32) != 0) return lp::fail(LP_ECORRUPT, "%s: SHA-256 of the keys does not match", path);
    *P = p;
    return LP_OK;
}

}  // namespace

extern "C" int lp_sha256(const void *data, size_t bytes, uint8_t out[32])
{
    if ((!data && bytes) || !out) return lp::fail(LP_EINVAL, "null pointer");
    Sha256 sh;
    sh.update(data, bytes);
    sh.final(out);
    return LP_OK;
}

extern "C" int lp_save_keys_file(const lp_params *p, const uint32_t *bsk, const uint32_t *ksk, const char *path)
{
    if (!p || !bsk || !ksk || !path) return lp::fail(LP_EINVAL, "null argument");
    Header h;
    memcpy(h.magic, MAGIC, 8);
    h.version = 1;
    const int32_t prm[7] = {p->n, p->N, p->k, p->Bgbit, p->lg, p->basebit, p->t};
    memcpy(h.params, prm, sizeof prm);
    h.bsk_words = bsk_words_of(*p);
    h.ksk_words = ksk_words_of(*p);
    Sha256 sh;
    sh.update(bsk, h.bsk_words * 4);
    sh.update(ksk, h.ksk_words * 4);
    sh.final(h.sha);
    FILE *f = fopen(path, "wb");
    if (!f) return lp::fail(LP_EINVAL, "cannot create %s", path);
    bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(bsk, 4, h.bsk_words, f) == h.bsk_words &&
              fwrite(ksk, 4, h.ksk_words, f) == h.ksk_words;
    ok = (fclose(f) == 0) && ok;
    return ok ? LP_OK : lp::fail(LP_EINVAL, "write to %s failed", path);
}

extern "C" int lp_verify_keys_file(const char *path, lp_params *params_out)
{
    if (!path) return lp::fail(LP_EINVAL, "null path");
    lp_params p;
    int rc = read_keys(path, &p, nullptr, nullptr);
    if (rc) return rc;
    if (params_out) *params_out = p;
    return LP_OK;
}

extern "C" int lp_load_keys_file(lp_ctx *c, const char *path)
{
    if (!c || !path) return lp::fail(LP_EINVAL, "null argument");
    lp_params p;
    std::vector<uint32_t> bsk, ksk;
    int rc = read_keys(path, &p, &bsk, &ksk);
    if (rc) return rc;
    const lp_params &q = c->params;
    if (p.n != q.n || p.N != q.N || p.k != q.k || p.Bgbit != q.Bgbit || p.lg != q.lg || p.basebit != q.basebit ||
        p.t != q.t)
        return lp::fail(LP_EINVAL, "%s holds keys for other parameters (n=%d) than the context's (n=%d)", path, p.n,
                        q.n);
    rc = lp_load_bsk(c, bsk.data(), bsk.size());
    if (!rc) rc = lp_load_ksk(c, ksk.data(), ksk.size());
    return rc;
}
