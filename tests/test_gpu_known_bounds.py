"""Server-known box bounds (beyond the paper) on the GPU: comparators and LocPIR queries whose
bounds are plaintext.  Every output ciphertext equals the oracle's known-bounds circuit
evaluation bit for bit and decrypts to the plaintext truth."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host
from oracle import circuits as C

pytestmark = pytest.mark.gpu


def _enc_bits(keys, bits, seed, offset):
    return oracle.encrypt(keys.s, bits, synth.lwe_draws(seed, len(bits), offset=offset))


def _bits(v, l):
    return synth.int_to_bits(v, l)


@pytest.mark.parametrize("signed", [0, 1])
def test_compare_known_matches_oracle(gpu_ctx, keys, signed):
    """All 16 bounds against 4 encrypted 4-bit points, both kinds; includes the bounds
    whose result needs no gate (a trivial constant) and those that are a negated input."""
    l = 4
    xs = [0, 5, 8, 15]
    pairs = [(x, K) for x in xs for K in range(16)]
    n = keys.params.n
    bits = np.concatenate([_bits(x, l) for x, _ in pairs])
    cx = _enc_bits(keys, bits, 500 + signed, 0)
    ks = [K for _, K in pairs]
    sv = lambda v: v - 16 if signed and v >= 8 else v
    for kind in (0, 1):
        out = empty_dev(len(pairs), n + 1)
        gpu_ctx.lp_compare_known_batch(kind, signed, l, to_dev(cx), ks, out, len(pairs))
        gpu_ctx.lp_sync()
        got = to_host(out)
        net = C.Netlist()
        ins, outs = {}, []
        for g, (_, K) in enumerate(pairs):
            a = net.inputs(l)
            ins.update(zip(a, cx[g * l:(g + 1) * l]))
            s = C.comp_s_known(net, a, K, bool(signed))
            outs.append(s if kind == 0 else net.NOT(s))
        val = C.eval_encrypted(net, keys, ins)
        assert_same(got, val[outs], f"compare-known kind={kind} signed={signed}")
        truth = [int(sv(x) < sv(K)) if kind == 0 else int(sv(K) <= sv(x)) for x, K in pairs]
        assert oracle.decrypt(keys.s, got).tolist() == truth


def _oracle_known(keys, l, x, y, bounds, sc, m, comb, signed):
    net = C.Netlist()
    xw, yw = net.inputs(l), net.inputs(l)
    sw = [net.inputs(m) for _ in bounds]
    out = C.locpir_known(net, xw, yw, bounds, sw, comb, bool(signed))
    ins = dict(zip(xw, x))
    ins.update(zip(yw, y))
    ins.update(zip([w for s in sw for w in s], sc))
    return C.eval_encrypted(net, keys, ins)[out]


@pytest.mark.parametrize("comb", [C.XOR_TREE, C.XOR_CHAIN, C.OR_TREE])
def test_locpir_known_matches_oracle(gpu_ctx, keys, comb):
    """Two uneven queries in one call (l = 4 and l = 6, 3 and 2 boxes); one bound of 0 and
    one of 2^l - 1 make gate-free comparators."""
    n = keys.params.n
    specs = [
        (4, 10, 5, [(2, 9, 1, 7), (9, 15, 3, 12), (0, 3, 10, 15)], [[1, 0, 1], [0, 1, 1], [1, 1, 0]]),
        (6, 40, 33, [(0, 63, 30, 34), (41, 50, 0, 63)], [[1, 1, 0], [0, 1, 0]]),
    ]
    queries, wants, truths = [], [], []
    for q, (l, px, py, bounds, services) in enumerate(specs):
        m = len(services[0])
        x = _enc_bits(keys, _bits(px, l), 600 + 10 * comb + q, 0)
        y = _enc_bits(keys, _bits(py, l), 600 + 10 * comb + q, l)
        sc = _enc_bits(keys, np.concatenate([np.asarray(s, np.uint8) for s in services]), 600 + 10 * comb + q,
                       2 * l)
        wants.append(_oracle_known(keys, l, x, y, bounds, sc, m, comb, 0))
        t = [0] * m
        for (x1, x2, y1, y2), s in zip(bounds, services):
            if x1 <= px < x2 and y1 <= py < y2:
                t = [(u | v) if comb == C.OR_TREE else (u ^ v) for u, v in zip(t, s)]
        truths.append(t)
        queries.append(dict(l=l, is_signed=0, n_boxes=len(bounds), m=m, comb=comb, x=to_dev(x), y=to_dev(y),
                            bounds=bounds, services=to_dev(sc), out_service=empty_dev(m, n + 1)))
    gpu_ctx.lp_locpir_known_batch(queries)
    gpu_ctx.lp_sync()
    for k, (q, w, t) in enumerate(zip(queries, wants, truths)):
        got = to_host(q["out_service"])
        assert_same(got, w, f"known-bounds query {k}")
        assert oracle.decrypt(keys.s, got).tolist() == t


def test_locpir_known_agrees_with_encrypted_bounds(gpu_ctx, keys):
    """The same city-shaped query (l = 16, one box, m = 8) with its bounds encrypted and in
    the clear decrypts to the same service (half of the points lie inside)."""
    n = keys.params.n
    l, m = 16, 8
    qs = synth.city_batch(7, 4, l, m)
    for k, q in enumerate(qs):
        x = _enc_bits(keys, _bits(q.x, l), 700 + k, 0)
        y = _enc_bits(keys, _bits(q.y, l), 700 + k, l)
        bx = _enc_bits(keys, np.concatenate([_bits(v, l) for v in q.box]), 700 + k, 2 * l)
        sc = _enc_bits(keys, q.service, 700 + k, 6 * l)
        out_e, out_k = empty_dev(m, n + 1), empty_dev(m, n + 1)
        gpu_ctx.lp_locpir_query(l, 0, to_dev(x), to_dev(y), 1, to_dev(bx), m, to_dev(sc), C.XOR_TREE, out_e)
        gpu_ctx.lp_locpir_known_batch([dict(l=l, is_signed=0, n_boxes=1, m=m, comb=C.XOR_TREE, x=to_dev(x),
                                            y=to_dev(y), bounds=[q.box], services=to_dev(sc), out_service=out_k)])
        gpu_ctx.lp_sync()
        x1, x2, y1, y2 = q.box
        want = q.service if (x1 <= q.x < x2 and y1 <= q.y < y2) else np.zeros(m, np.uint8)
        assert oracle.decrypt(keys.s, to_host(out_e)).tolist() == want.tolist()
        assert oracle.decrypt(keys.s, to_host(out_k)).tolist() == want.tolist()


def test_known_bounds_argument_errors(gpu_ctx):
    from paper_2407_19871_gb300.locpir import LocpirError
    n = gpu_ctx.n
    x = empty_dev(65, n + 1)
    with pytest.raises(LocpirError):
        gpu_ctx.lp_compare_known_batch(7, 0, 4, x, [1], empty_dev(1, n + 1), 1)
    with pytest.raises(LocpirError):
        gpu_ctx.lp_compare_known_batch(0, 0, 65, x, [1], empty_dev(1, n + 1), 1)
    with pytest.raises(LocpirError):
        gpu_ctx.lp_locpir_known_batch([dict(l=4, n_boxes=0, m=1, x=x, y=x, bounds=[], services=x,
                                            out_service=empty_dev(1, n + 1))])


def test_known_bounds_plan_replays_match_batch(gpu_ctx, keys):
    """A known-bounds batch captured into a CUDA-graph plan gives, on every replay, the
    ciphertexts lp_locpir_known_batch gives."""
    n = keys.params.n
    l, m = 8, 4
    qs = synth.city_batch(9, 6, l, m)
    queries, refs = [], []
    for k, q in enumerate(qs):
        x = _enc_bits(keys, _bits(q.x, l), 800 + k, 0)
        y = _enc_bits(keys, _bits(q.y, l), 800 + k, l)
        sc = _enc_bits(keys, q.service, 800 + k, 2 * l)
        base = dict(l=l, is_signed=0, n_boxes=1, m=m, comb=C.XOR_TREE, x=to_dev(x), y=to_dev(y), bounds=[q.box],
                    services=to_dev(sc))
        queries.append(dict(base, out_service=empty_dev(m, n + 1)))
        refs.append(dict(base, out_service=empty_dev(m, n + 1)))
    gpu_ctx.lp_locpir_known_batch(refs)
    plan = gpu_ctx.lp_plan_locpir_known(queries)
    try:
        for rep in range(2):
            plan.lp_plan_run()
            gpu_ctx.lp_sync()
            for k, (q, r) in enumerate(zip(queries, refs)):
                assert_same(to_host(q["out_service"]), to_host(r["out_service"]), f"replay {rep} query {k}")
    finally:
        plan.lp_plan_destroy()
    for k, q in enumerate(qs):
        x1, x2, y1, y2 = q.box
        want = q.service if (x1 <= q.x < x2 and y1 <= q.y < y2) else np.zeros(m, np.uint8)
        assert oracle.decrypt(keys.s, to_host(queries[k]["out_service"])).tolist() == want.tolist()
