"""lp_gate_batch_noalloc -- the gate batch for callers that cannot allocate device memory
while they evaluate (a server whose device memory is pre-assigned by its own allocator, or
a latency-critical loop that cannot take cudaMalloc's device-wide synchronisation) -- gives
the same ciphertexts as lp_gate_batch, on two calls in a row that reuse its fixed scratch
array.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu


def _enc(keys, seed, count, offset=0):
    bits = synth.bits(seed, 1, count)
    return oracle.encrypt(keys.s, bits, synth.lwe_draws(seed, count, offset=offset))


def _both(gpu_ctx, keys, op, count, seed):
    """(lp_gate_batch output, lp_gate_batch_noalloc output) on the same fresh inputs."""
    n = keys.params.n
    a, b, c = (to_dev(_enc(keys, seed, count, k * count)) for k in range(3))
    cc = c if op == oracle.MUX else None
    ref = empty_dev(count, n + 1)
    got = empty_dev(count, n + 1)
    gpu_ctx.lp_gate_batch(op, a, b, cc, ref, count)
    gpu_ctx.lp_gate_batch_noalloc(op, a, b, cc, got, count)
    gpu_ctx.lp_sync()
    return to_host(ref), to_host(got)


@pytest.mark.parametrize("op,count", [(oracle.NAND, 37), (oracle.MUX, 128), (oracle.XOR, 256)])
def test_noalloc_matches_gate_batch_on_consecutive_calls(gpu_ctx, keys, op, count):
    for call in range(2):
        ref, got = _both(gpu_ctx, keys, op, count, 700 + 10 * op + call)
        # Bit-exact, the tolerance of every ciphertext test here.
        assert_same(got, ref, f"noalloc op={op} call={call}")


def test_noalloc_shrinking_batch_and_not(gpu_ctx, keys):
    """A full 256-rotation call followed by a single gate, a MUX and a NOT: every scratch word
    the smaller calls read must come from their own call, not the larger one before."""
    for op, count, seed in ((oracle.AND, 256, 801), (oracle.OR, 1, 802), (oracle.MUX, 3, 803),
                            (oracle.NOT, 5, 804), (oracle.NAND, 2, 805)):
        ref, got = _both(gpu_ctx, keys, op, count, seed)
        assert_same(got, ref, f"noalloc op={op} count={count}")


def test_noalloc_adds_no_device_allocation(gpu_ctx, keys):
    """After a warm-up call (which loads the library's module and looks up the scratch address),
    a call leaves the device's free memory unchanged."""
    import torch
    n = keys.params.n
    count = 64
    a, b = (to_dev(_enc(keys, 811, count, k * count)) for k in range(2))
    out = empty_dev(count, n + 1)
    gpu_ctx.lp_gate_batch_noalloc(oracle.NAND, a, b, None, out, count)
    gpu_ctx.lp_sync()
    free0, _ = torch.cuda.mem_get_info()
    gpu_ctx.lp_gate_batch_noalloc(oracle.NAND, a, b, None, out, count)
    gpu_ctx.lp_sync()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_batches_above_its_limit(gpu_ctx, keys):
    from paper_2407_19871_gb300.locpir import LP_EINVAL, LocpirError
    n = keys.params.n
    t = empty_dev(129, n + 1)
    with pytest.raises(LocpirError) as e:
        gpu_ctx.lp_gate_batch_noalloc(oracle.MUX, t, t, t, empty_dev(129, n + 1), 129)
    assert e.value.code == LP_EINVAL and "at most 256" in str(e.value)


def test_noalloc_needs_keys(keys):
    from paper_2407_19871_gb300 import build
    from paper_2407_19871_gb300.locpir import LP_ENOKEY, Context, LocpirError
    build.build()
    n = keys.params.n
    t = empty_dev(2, n + 1)
    with Context(0) as bare:
        with pytest.raises(LocpirError) as e:
            bare.lp_gate_batch_noalloc(oracle.NAND, t, t, None, empty_dev(2, n + 1), 2)
    assert e.value.code == LP_ENOKEY
