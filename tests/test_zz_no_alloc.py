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


@pytest.mark.parametrize("op,count", [(oracle.NAND, 37), (oracle.MUX, 128), (oracle.XOR, 256)])
def test_noalloc_matches_gate_batch_on_consecutive_calls(gpu_ctx, keys, op, count):
    n = keys.params.n
    for call in range(2):
        seed = 700 + 10 * op + call
        a, b, c = (to_dev(_enc(keys, seed, count, k * count)) for k in range(3))
        cc = c if op == oracle.MUX else None
        ref = empty_dev(count, n + 1)
        got = empty_dev(count, n + 1)
        gpu_ctx.lp_gate_batch(op, a, b, cc, ref, count)
        gpu_ctx.lp_gate_batch_noalloc(op, a, b, cc, got, count)
        gpu_ctx.lp_sync()
        # Bit-exact, the tolerance of every ciphertext test here.
        assert_same(to_host(got), to_host(ref), f"noalloc op={op} call={call}")


def test_noalloc_rejects_batches_above_its_limit(gpu_ctx, keys):
    from paper_2407_19871_gb300.locpir import LP_EINVAL, LocpirError
    n = keys.params.n
    t = empty_dev(129, n + 1)
    with pytest.raises(LocpirError) as e:
        gpu_ctx.lp_gate_batch_noalloc(oracle.MUX, t, t, t, empty_dev(129, n + 1), 129)
    assert e.value.code == LP_EINVAL and "at most 256" in str(e.value)
