// lp_gate_batch_noalloc: the gate-batch pipeline (pre-combination + modulus switch,
// blind rotation + extraction, key switch) with its scratch in a fixed, file-scope device
// array instead of memory the context allocates.
//
// Who needs this: callers that must not allocate device memory at evaluation time --
// for example a serving process whose device memory is handed out up front by its own
// allocator and budget (so a cudaMalloc inside the call could fail or exceed the budget),
// or a latency-critical loop where cudaMalloc / cudaFree would add their device-wide
// synchronisation to every request.  This entry point calls no cudaMalloc, cudaFree or
// allocating library routine; the caller still provides inputs and outputs, and the
// context's keys must already be loaded.
//
// The scratch array below is part of the library's device image: every GPU that loads the
// library holds it (NOALLOC_SCRATCH_BYTES, about 1.5 MiB) until the process exits.  All
// calls on a device share it, so calls that overlap on the GPU (for instance on two streams
// without ordering between them) race on it; issue them in order on one stream.  Every
// word the kernels read from the scratch is written earlier in the same call, so nothing
// has to be cleared between calls, although the array keeps the previous call's contents.
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "runtime.h"

namespace {

// At most this many blind rotations per call: 256 two-input gates or 128 MUX gates.
constexpr size_t NOALLOC_MAX_JOBS = 256;
constexpr size_t NOALLOC_ABAR_BYTES = NOALLOC_MAX_JOBS * 1024 * sizeof(uint16_t);  // stride <= 1024 entries
constexpr size_t NOALLOC_EXT_BYTES = NOALLOC_MAX_JOBS * lp::EXT_STRIDE * sizeof(uint32_t);
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_ABAR_BYTES + NOALLOC_EXT_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device.  In host code the array's name is only
// a host-side stand-in, so the address is looked up once per device with that device
// current.  A device reset (cudaDeviceReset) unloads the module and invalidates the cached
// address; the entry point is then unusable on that device until the process restarts.
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

int scratch_address(int device, void **out)
{
    if (device < 0 || device >= NOALLOC_MAX_DEVICES)
        return lp::fail(LP_EINVAL, "device %d outside the %d devices the no-alloc scratch table covers", device,
                        NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return lp::cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_addr[device] = p;
    }
    *out = g_noalloc_addr[device];
    return LP_OK;
}

}  // namespace

extern "C" int lp_gate_batch_noalloc(lp_ctx *c, int op, const uint32_t *a, const uint32_t *b, const uint32_t *cc,
                                     uint32_t *out, size_t count, void *stream)
{
    using namespace lp;
    if (!c) return fail(LP_EINVAL, "null context");
    if (op < LP_NAND || op > LP_MUX) return fail(LP_EINVAL, "unknown gate %d", op);
    if (count == 0) return LP_OK;
    if (!a || !out || (op != LP_NOT && !b) || (op == LP_MUX && !cc)) return fail(LP_EINVAL, "null ciphertext pointer");
    const size_t halves = op == LP_MUX ? 2 : 1;
    if (op != LP_NOT && count * halves > NOALLOC_MAX_JOBS)
        return fail(LP_EINVAL,
                    "lp_gate_batch_noalloc handles at most %zu blind rotations per call (%zu two-input gates or %zu "
                    "MUX gates); got %zu gates",
                    NOALLOC_MAX_JOBS, NOALLOC_MAX_JOBS, NOALLOC_MAX_JOBS / 2, count);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = c->params.n;
    if (op == LP_NOT) {
        e = launch_negate(a, out, count * ((size_t)n + 1), c->num_sms, st);
        c->launches++;
        return e == cudaSuccess ? LP_OK : cuda_fail(e, "negate launch");
    }
    if (!c->have_bsk || !c->have_ksk) return fail(LP_ENOKEY, "load the bootstrapping and key-switching keys first");
    void *base = nullptr;
    int rc = scratch_address(c->device, &base);
    if (rc) return rc;
    uint16_t *abar = static_cast<uint16_t *>(base);
    uint32_t *ext = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(base) + NOALLOC_ABAR_BYTES);
    e = launch_precomb_dense(op, a, b, op == LP_MUX ? cc : nullptr, n, count, abar, abar_stride(c), c->num_sms, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "pre-combination launch");
    // The NTT kernels only: a forced batched, split, paired or quad choice is honoured, and a
    // tensor-core engine selection falls back to the automatic NTT choice (those engines
    // allocate).
    const int variant = br_variant(c);
    e = launch_br(abar, abar_stride(c), ext, static_cast<const uint32_t *>(c->bsk_hat.ptr),
                  static_cast<const uint2 *>(c->tw_lane.ptr), n, (int)(count * halves), T_EIGHTH,
                  static_cast<int *>(c->err.ptr), c->num_sms, st, variant, c->br_split_max, 0, br_pair_limit(c),
                  br_quad_limit(c));
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "blind rotation launch");
    e = launch_ks(ext, nullptr, count, op == LP_MUX, out, static_cast<const uint32_t *>(c->ksk.ptr), n,
                  static_cast<int *>(c->err.ptr), c->num_sms, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "key switch launch");
    return LP_OK;
}
