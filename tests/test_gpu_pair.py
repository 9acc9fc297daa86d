"""The paired blind rotation (br_pair_kernel): one ciphertext per cluster of two CTAs, CTA q
computing modulo NTT prime q, the two exchanging their residue polynomials through distributed
shared memory at every CMux step of TFHE's gate bootstrapping (to which Section 2.2 defers).
Bit-exact against the oracle at small counts, and word for word against the split kernel
(itself pinned to the oracle) where each cluster runs several ciphertexts in turn."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu

EIGHTH = 1 << 29


def _random_lwes(seed, count, n):
    return synth.uniform_u32(seed, 900, count * (n + 1)).reshape(count, n + 1)


@pytest.fixture
def engine_ctx(gpu_ctx):
    yield gpu_ctx
    from paper_2407_19871_gb300.locpir import LP_BR_NTT
    gpu_ctx.lp_set_engines(LP_BR_NTT, 0)


def _extract(ctx, engine, lwe, mu=EIGHTH):
    ctx.lp_set_engines(engine, 0)
    ext = empty_dev(lwe.shape[0], 1025)
    ctx.lp_bootstrap_extract(to_dev(lwe), mu, ext, lwe.shape[0])
    ctx.lp_sync()
    return to_host(ext)


@pytest.mark.parametrize("count", [1, 2, 5])
def test_pair_matches_oracle(engine_ctx, keys, count):
    from paper_2407_19871_gb300.locpir import LP_BR_NTT_PAIR
    lwe = _random_lwes(301 + count, count, keys.params.n)
    assert_same(_extract(engine_ctx, LP_BR_NTT_PAIR, lwe), oracle.bootstrap_extract(keys, lwe),
                f"paired x{count}")


def test_pair_several_ciphertexts_per_cluster(engine_ctx, keys):
    """More ciphertexts than SM pairs: clusters loop over jobs (and the exchange parity carries
    over from one job to the next).  Word for word against the split kernel, three samples
    (first, first of a cluster's second round, last) against the oracle."""
    import torch
    from paper_2407_19871_gb300.locpir import LP_BR_NTT_PAIR, LP_BR_NTT_SPLIT
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    count = 2 * (sms // 2) + 3
    lwe = _random_lwes(311, count, keys.params.n)
    got = _extract(engine_ctx, LP_BR_NTT_PAIR, lwe)
    assert_same(got, _extract(engine_ctx, LP_BR_NTT_SPLIT, lwe), f"paired vs split x{count}")
    idx = [0, sms // 2, count - 1]
    assert_same(got[idx], oracle.bootstrap_extract(keys, lwe[idx]), "paired samples vs oracle")


@pytest.mark.parametrize("op", [oracle.NAND, oracle.MUX])
def test_pair_gates_match_oracle(engine_ctx, keys, op):
    """Whole gates (pre-combination, paired blind rotation, key switch); MUX runs two blind
    rotations per gate."""
    from paper_2407_19871_gb300.locpir import LP_BR_NTT_PAIR
    n, cnt = keys.params.n, 6
    A, B, Cb = (synth.bits(320, k, cnt) for k in (1, 2, 3))
    a, b, c = (oracle.encrypt(keys.s, X, synth.lwe_draws(321, cnt, offset=k * cnt)) for k, X in enumerate((A, B, Cb)))
    engine_ctx.lp_set_engines(LP_BR_NTT_PAIR, 0)
    out = empty_dev(cnt, n + 1)
    engine_ctx.lp_gate_batch(op, to_dev(a), to_dev(b), to_dev(c) if op == oracle.MUX else None, out, cnt)
    engine_ctx.lp_sync()
    assert_same(to_host(out), oracle.gate_batch(keys, op, a, b, c if op == oracle.MUX else None), f"paired op={op}")


def test_default_policy_pairs_narrow_levels(engine_ctx, keys):
    """The default engine runs a level of a few ciphertexts on the paired kernel (pair_max is
    the number of co-resident clusters unless the autotuner found the split kernel faster) and
    gives the forced kernels' bits."""
    from paper_2407_19871_gb300.locpir import LP_BR_NTT, LP_BR_NTT_BATCHED
    assert engine_ctx.lp_get_tuning()["pair_max"] >= -1
    lwe = _random_lwes(331, 3, keys.params.n)
    assert_same(_extract(engine_ctx, LP_BR_NTT, lwe), _extract(engine_ctx, LP_BR_NTT_BATCHED, lwe), "auto vs batched")


def test_pair_stop_protocol_times_out_cleanly(engine_ctx, keys):
    """One CTA of a cluster never gets its first key rows: its wait gives up after 2 s, it passes
    its stop decision to the partner in the residue exchange, both leave after that exchange and
    the call reports LP_ETIMEOUT.  The context then bootstraps normally (oracle parity)."""
    from paper_2407_19871_gb300.locpir import LP_BR_NTT_PAIR, LP_ETIMEOUT, LocpirError
    engine_ctx.lp_selftest_pair_timeout()
    with pytest.raises(LocpirError) as e:
        engine_ctx.lp_sync()
    assert e.value.code == LP_ETIMEOUT
    lwe = _random_lwes(341, 2, keys.params.n)
    assert_same(_extract(engine_ctx, LP_BR_NTT_PAIR, lwe), oracle.bootstrap_extract(keys, lwe), "paired after the stop")
