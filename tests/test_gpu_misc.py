"""Other device paths through the C-ABI: Algorithm 1 preprocessing, the failure-detection
self-test, and the 80-bit parameter set's LWE dimension (n = 540, Section 5)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, make_context, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_preprocess_services_matches_oracle(keys):
    import torch
    from paper_2407_19871_gb300 import build, locpir
    build.build()
    n, cnt = keys.params.n, 77
    bits = synth.bits(82, 1, cnt)
    zero = oracle.zero_samples(keys.s, synth.lwe_draws(82, cnt))
    out = empty_dev(cnt, n + 1)
    locpir.lp_preprocess_services(n, to_dev(zero), to_dev(bits), out, cnt)
    torch.cuda.synchronize()
    got = to_host(out)
    assert_same(got, oracle.preprocess(zero, bits), "preprocess")
    np.testing.assert_array_equal(oracle.decrypt(keys.s, got), bits)


def test_wait_timeout_is_reported_and_context_survives(gpu_ctx, keys):
    """A device wait that nothing completes gives up after its limit; lp_sync reports
    LP_ETIMEOUT once, and the context keeps working afterwards."""
    from paper_2407_19871_gb300.locpir import LP_ETIMEOUT, LocpirError
    gpu_ctx.lp_selftest_wait_timeout(200)
    with pytest.raises(LocpirError) as e:
        gpu_ctx.lp_sync()
    assert e.value.code == LP_ETIMEOUT
    gpu_ctx.lp_sync()  # flag cleared
    n = keys.params.n
    A, B = synth.bits(83, 1, 3), synth.bits(83, 2, 3)
    a = oracle.encrypt(keys.s, A, synth.lwe_draws(83, 3))
    b = oracle.encrypt(keys.s, B, synth.lwe_draws(83, 3, offset=3))
    out = empty_dev(3, n + 1)
    gpu_ctx.lp_gate_batch(oracle.AND, to_dev(a), to_dev(b), None, out, 3)
    gpu_ctx.lp_sync()
    assert_same(to_host(out), oracle.gate_batch(keys, oracle.AND, a, b), "AND after timeout")


def test_lambda80_dimension_matches_oracle():
    """n = 540 (the 80-bit set's LWE dimension; its other TFHE parameters are not printed,
    so the rest of the set is kept) runs the same kernels bit-exactly."""
    from paper_2407_19871_gb300 import locpir
    p = synth.Params(n=540)
    keys80 = oracle.keygen(synth.key_draws(5, p))
    lp = locpir.params_default()
    lp.n = 540
    ctx = locpir.Context(0, lp)
    try:
        ctx.lp_load_bsk(np.ascontiguousarray(keys80.bsk.reshape(-1)))
        ctx.lp_load_ksk(np.ascontiguousarray(keys80.ksk.reshape(-1)))
        cnt = 6
        A, B, Cb = (synth.bits(84, k, cnt) for k in (1, 2, 3))
        a, b, c = (oracle.encrypt(keys80.s, X, synth.lwe_draws(84, cnt, p, offset=k * cnt))
                   for k, X in enumerate((A, B, Cb)))
        for op in (oracle.NAND, oracle.MUX):
            out = empty_dev(cnt, p.n + 1)
            ctx.lp_gate_batch(op, to_dev(a), to_dev(b), to_dev(c) if op == oracle.MUX else None, out, cnt)
            ctx.lp_sync()
            assert_same(to_host(out), oracle.gate_batch(keys80, op, a, b, c if op == oracle.MUX else None),
                        f"n=540 op={op}")
    finally:
        ctx.close()


@pytest.mark.parametrize("n", [1, 7, 639])
def test_lwe_dimension_edges_match_oracle(n):
    """The smallest, an odd and the largest supported LWE dimension (n + 1 = 640 words fills
    the key switch's 20 words per lane exactly), on each blind-rotation kernel."""
    from paper_2407_19871_gb300 import locpir
    p = synth.Params(n=n)
    kn = oracle.keygen(synth.key_draws(6, p))
    lp = locpir.params_default()
    lp.n = n
    ctx = locpir.Context(0, lp)
    try:
        ctx.lp_load_bsk(np.ascontiguousarray(kn.bsk.reshape(-1)))
        ctx.lp_load_ksk(np.ascontiguousarray(kn.ksk.reshape(-1)))
        cnt = 5
        A, B, Cb = (synth.bits(85, k, cnt) for k in (1, 2, 3))
        a, b, c = (oracle.encrypt(kn.s, X, synth.lwe_draws(85, cnt, p, offset=k * cnt))
                   for k, X in enumerate((A, B, Cb)))
        for op in (oracle.AND, oracle.MUX):
            want = oracle.gate_batch(kn, op, a, b, c if op == oracle.MUX else None)
            for variant in (locpir.LP_BR_NTT_BATCHED, locpir.LP_BR_NTT_SPLIT, locpir.LP_BR_NTT_PAIR,
                            locpir.LP_BR_NTT_QUAD):
                ctx.lp_set_engines(variant, 0)
                out = empty_dev(cnt, p.n + 1)
                ctx.lp_gate_batch(op, to_dev(a), to_dev(b), to_dev(c) if op == oracle.MUX else None, out, cnt)
                ctx.lp_sync()
                assert_same(to_host(out), want, f"n={n} op={op} variant={variant}")
    finally:
        ctx.close()


def _mkquery(keys, seed, l, boxes, services, px, py, comb=0):
    n = keys.params.n
    bits = lambda v: synth.int_to_bits(v, l)
    enc = lambda b, off: oracle.encrypt(keys.s, b, synth.lwe_draws(seed, len(b), offset=off))
    bb = np.concatenate([bits(v) for box in boxes for v in box])
    sv = np.concatenate([np.asarray(s, np.uint8) for s in services])
    m = len(services[0])
    return dict(l=l, is_signed=0, n_boxes=len(boxes), m=m, comb=comb, x=to_dev(enc(bits(px), 0)),
                y=to_dev(enc(bits(py), l)), boxes=to_dev(enc(bb, 2 * l)), services=to_dev(enc(sv, 2 * l + len(bb))),
                out_service=empty_dev(m, n + 1))


def test_plan_graph_replay_matches_batch(gpu_ctx, keys):
    """A CUDA-graph plan gives the same ciphertexts as lp_locpir_batch, also after the contents
    of its input buffers change between runs."""
    n = keys.params.n
    specs = [(4, [(1, 9, 2, 12)], [[1, 1]], 5, 6), (5, [(3, 20, 0, 31), (20, 30, 5, 25)], [[1, 0], [0, 1]], 22, 9)]
    qs = [_mkquery(keys, 600 + k, *sp) for k, sp in enumerate(specs)]
    plan = gpu_ctx.lp_plan_locpir(qs)
    info = plan.lp_plan_info()
    assert info["blind_rotations"] == sum(len(b) * (12 * l + 3 + len(s[0])) + (len(b) - 1) * len(s[0])
                                          for (l, b, s, _, _) in specs)
    for rnd in range(2):
        if rnd == 1:  # new point for query 0: overwrite its input buffers in place
            fresh = _mkquery(keys, 650, *specs[0][:3], 2, 3)
            qs[0]["x"].copy_(fresh["x"])
            qs[0]["y"].copy_(fresh["y"])
        plan.lp_plan_run()
        gpu_ctx.lp_sync()
        ref = [dict(q, out_service=empty_dev(q["m"], n + 1)) for q in qs]
        gpu_ctx.lp_locpir_batch(ref)
        gpu_ctx.lp_sync()
        for k in range(len(qs)):
            assert_same(to_host(qs[k]["out_service"]), to_host(ref[k]["out_service"]), f"plan run {rnd} query {k}")
    assert oracle.decrypt(keys.s, to_host(qs[0]["out_service"])).tolist() == [1, 1]  # (2, 3) is inside box 0
    plan.lp_plan_destroy()


def test_load_keys_file(keys, tmp_path):
    from paper_2407_19871_gb300 import locpir
    p = locpir.params_default()
    path = str(tmp_path / "k.lpk")
    locpir.lp_save_keys_file(p, np.ascontiguousarray(keys.bsk.reshape(-1)), np.ascontiguousarray(keys.ksk.reshape(-1)),
                             path)
    ctx = locpir.Context(0)
    try:
        ctx.lp_load_keys_file(path)
        A, B = synth.bits(85, 1, 5), synth.bits(85, 2, 5)
        a = oracle.encrypt(keys.s, A, synth.lwe_draws(85, 5))
        b = oracle.encrypt(keys.s, B, synth.lwe_draws(85, 5, offset=5))
        out = empty_dev(5, p.n + 1)
        ctx.lp_gate_batch(oracle.OR, to_dev(a), to_dev(b), None, out, 5)
        ctx.lp_sync()
        assert_same(to_host(out), oracle.gate_batch(keys, oracle.OR, a, b), "OR with keys from file")
        raw = bytearray(open(path, "rb").read())
        raw[200] ^= 1
        open(path, "wb").write(bytes(raw))
        with pytest.raises(locpir.LocpirError) as e:
            ctx.lp_load_keys_file(path)
        assert e.value.code == locpir.LP_ECORRUPT
    finally:
        ctx.close()
