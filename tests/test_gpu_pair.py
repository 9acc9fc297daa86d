"""The cluster blind rotations, in TFHE's gate bootstrapping (to which Section 2.2 defers):
  * paired (br_pair_kernel): one ciphertext per cluster of two CTAs, CTA q computing modulo NTT
    prime q, the two exchanging their residue polynomials through distributed shared memory at
    every CMux step;
  * quad (br_quad_kernel): one ciphertext per cluster of four CTAs, CTA (q, g) computing modulo
    prime q with ACC component g, exchanging partial sums with the other CTA of its prime and
    residues with the other CTA of its component.
Bit-exact against the oracle at small counts, and word for word against the split kernel
(itself pinned to the oracle) where each cluster runs several ciphertexts in turn."""
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu

EIGHTH = 1 << 29
CLUSTER = {"pair": 2, "quad": 4}


def _engine(name):
    from paper_2407_19871_gb300.locpir import LP_BR_NTT_PAIR, LP_BR_NTT_QUAD
    return {"pair": LP_BR_NTT_PAIR, "quad": LP_BR_NTT_QUAD}[name]


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


@pytest.mark.parametrize("kernel", ["pair", "quad"])
@pytest.mark.parametrize("count", [1, 2, 5])
def test_cluster_kernel_matches_oracle(engine_ctx, keys, kernel, count):
    lwe = _random_lwes(301 + count, count, keys.params.n)
    assert_same(_extract(engine_ctx, _engine(kernel), lwe), oracle.bootstrap_extract(keys, lwe), f"{kernel} x{count}")


@pytest.mark.parametrize("kernel", ["pair", "quad"])
def test_several_ciphertexts_per_cluster(engine_ctx, keys, kernel):
    """More ciphertexts than clusters: clusters loop over jobs (and the exchange parity carries
    over from one job to the next).  Word for word against the split kernel, three samples
    (first, first of a cluster's second round, last) against the oracle."""
    import torch
    from paper_2407_19871_gb300.locpir import LP_BR_NTT_SPLIT
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clusters = sms // CLUSTER[kernel]
    count = 2 * clusters + 3
    lwe = _random_lwes(311, count, keys.params.n)
    got = _extract(engine_ctx, _engine(kernel), lwe)
    assert_same(got, _extract(engine_ctx, LP_BR_NTT_SPLIT, lwe), f"{kernel} vs split x{count}")
    idx = [0, clusters, count - 1]
    assert_same(got[idx], oracle.bootstrap_extract(keys, lwe[idx]), f"{kernel} samples vs oracle")


@pytest.mark.parametrize("kernel", ["pair", "quad"])
@pytest.mark.parametrize("op", [oracle.NAND, oracle.MUX])
def test_cluster_kernel_gates_match_oracle(engine_ctx, keys, kernel, op):
    """Whole gates (pre-combination, cluster blind rotation, key switch); MUX runs two blind
    rotations per gate."""
    n, cnt = keys.params.n, 6
    A, B, Cb = (synth.bits(320, k, cnt) for k in (1, 2, 3))
    a, b, c = (oracle.encrypt(keys.s, X, synth.lwe_draws(321, cnt, offset=k * cnt)) for k, X in enumerate((A, B, Cb)))
    engine_ctx.lp_set_engines(_engine(kernel), 0)
    out = empty_dev(cnt, n + 1)
    engine_ctx.lp_gate_batch(op, to_dev(a), to_dev(b), to_dev(c) if op == oracle.MUX else None, out, cnt)
    engine_ctx.lp_sync()
    assert_same(to_host(out), oracle.gate_batch(keys, op, a, b, c if op == oracle.MUX else None), f"{kernel} op={op}")


def test_default_policy_runs_narrow_levels_on_clusters(engine_ctx, keys):
    """The default engine runs a level of a few ciphertexts on a cluster kernel (pair_max and
    quad_max are the resident cluster counts unless the autotuner found another kernel faster)
    and gives the forced kernels' bits."""
    from paper_2407_19871_gb300.locpir import LP_BR_NTT, LP_BR_NTT_BATCHED
    t = engine_ctx.lp_get_tuning()
    assert t["pair_max"] >= -1 and t["quad_max"] >= -1
    lwe = _random_lwes(331, 3, keys.params.n)
    assert_same(_extract(engine_ctx, LP_BR_NTT, lwe), _extract(engine_ctx, LP_BR_NTT_BATCHED, lwe), "auto vs batched")


@pytest.mark.parametrize("kernel", ["pair", "quad"])
def test_cluster_stop_protocol_times_out_cleanly(engine_ctx, keys, kernel):
    """One CTA of a cluster never gets its first key rows: its wait gives up after 2 s, its stop
    decision travels with the exchanges of that step, every CTA of the cluster leaves after
    them and the call reports LP_ETIMEOUT.  The context then bootstraps normally (oracle
    parity)."""
    from paper_2407_19871_gb300.locpir import LP_ETIMEOUT, LocpirError
    if kernel == "pair":
        engine_ctx.lp_selftest_pair_timeout()
    else:
        engine_ctx.lp_selftest_quad_timeout()
    with pytest.raises(LocpirError) as e:
        engine_ctx.lp_sync()
    assert e.value.code == LP_ETIMEOUT
    lwe = _random_lwes(341, 2, keys.params.n)
    assert_same(_extract(engine_ctx, _engine(kernel), lwe), oracle.bootstrap_extract(keys, lwe), f"{kernel} after the stop")
