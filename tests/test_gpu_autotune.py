"""The launch-policy autotuner (lp_autotune_cached): its JSON cache per device, and that every
policy it can choose gives the same ciphertexts as the built-in rules, bit for bit.  The paths
a policy switches between: a level's partial last wave on the split blind rotation instead of
a batched wave, and the sliced key switch instead of whole-table CTAs."""
import json

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture
def tuned_ctx(gpu_ctx):
    saved = gpu_ctx.lp_get_tuning()
    yield gpu_ctx
    gpu_ctx.lp_set_tuning(**saved)


def test_cache_roundtrip(tuned_ctx, tmp_path):
    path = tmp_path / "tuning.json"
    first = tuned_ctx.lp_autotune_cached(str(path))
    assert first["from_cache"] == 0 and path.exists()
    rec = json.loads(path.read_text())
    assert "sms=" in rec["key"] and "n=630" in rec["key"]
    assert rec["split_max"] == first["split_max"] >= 1
    second = tuned_ctx.lp_autotune_cached(str(path))
    assert second == dict(first, from_cache=1)
    assert tuned_ctx.lp_get_tuning() == {k: first[k] for k in ("split_max", "tail_split", "ks_slice_max", "pair_max",
                                                                "quad_max")}
    assert rec["pair_max"] == first["pair_max"] >= -1 and rec["quad_max"] == first["quad_max"] >= -1
    # an entry for another device is not used: the call measures again and rewrites the file
    rec["key"] = "another GPU|sms=1|n=630|schema=3"
    path.write_text(json.dumps(rec))
    third = tuned_ctx.lp_autotune_cached(str(path))
    assert third["from_cache"] == 0
    assert json.loads(path.read_text())["key"] != rec["key"]


def test_policies_give_identical_bits(tuned_ctx, keys):
    """NAND gates over 4 ciphertexts per SM plus a 200-wide remainder: all batched under the
    built-in rules, the remainder split (or paired, or quad, each cluster taking several
    ciphertexts in turn) under tail splitting; and key switches of 1-4 batches per SM whole-table and sliced.
    Every output word is the same; a sample is the oracle's."""
    from paper_2407_19871_gb300.locpir import LP_NAND
    p = keys.params
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    count = 4 * sms + 200
    A, B = synth.bits(820, 1, count), synth.bits(820, 2, count)
    a = to_dev(oracle.encrypt(keys.s, A, synth.lwe_draws(821, count)))
    b = to_dev(oracle.encrypt(keys.s, B, synth.lwe_draws(822, count)))
    outs = []
    for policy in (dict(split_max=0, tail_split=0, ks_slice_max=0),        # built-in rules
                   dict(split_max=2 * sms, tail_split=1, ks_slice_max=0, pair_max=-1),  # remainder split
                   dict(split_max=2 * sms, tail_split=1, ks_slice_max=-1, pair_max=200, quad_max=-1),  # paired
                   dict(split_max=2 * sms, tail_split=1, ks_slice_max=0, pair_max=-1, quad_max=200),  # quad
                   dict(split_max=sms, tail_split=0, ks_slice_max=sms)):   # always slice here
        tuned_ctx.lp_set_tuning(**policy)
        out = empty_dev(count, p.n + 1)
        tuned_ctx.lp_gate_batch(LP_NAND, a, b, None, out, count)
        tuned_ctx.lp_sync()
        outs.append(to_host(out))
    for k in range(1, len(outs)):
        assert_same(outs[k], outs[0], f"policy {k} vs built-in rules")
    assert (oracle.decrypt(keys.s, outs[0]) == 1 - (A & B)).all()
    idx = np.array([0, 4 * sms - 1, 4 * sms, count - 1])   # last batched, first and last of the remainder
    ha, hb = to_host(a), to_host(b)
    assert_same(outs[1][idx], oracle.gate_batch(keys, oracle.NAND, ha[idx], hb[idx]), "sampled vs oracle")
