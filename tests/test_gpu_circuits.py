"""Comparator and LocPIR circuits on the GPU: every output ciphertext equals the oracle's
circuit evaluation (Algorithms 2-5) bit for bit, and decrypts to the plaintext truth."""
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
def test_compare_batch_matches_oracle(gpu_ctx, keys, signed):
    l = 4
    pairs = [(3, 11), (11, 3), (7, 7), (0, 15), (9, 8)]
    n = keys.params.n
    x1 = np.concatenate([_bits(a, l) for a, _ in pairs])
    x2 = np.concatenate([_bits(b, l) for _, b in pairs])
    c1 = _enc_bits(keys, x1, 300 + signed, 0)
    c2 = _enc_bits(keys, x2, 300 + signed, len(x1))
    for kind, name in ((0, "lt"), (1, "le")):
        out = empty_dev(len(pairs), n + 1)
        gpu_ctx.lp_compare_batch(kind, signed, l, to_dev(c1), to_dev(c2), out, len(pairs))
        gpu_ctx.lp_sync()
        got = to_host(out)
        net = C.Netlist()
        ins, outs = {}, []
        for g in range(len(pairs)):
            a, b = net.inputs(l), net.inputs(l)
            ins.update(zip(a, c1[g * l:(g + 1) * l]))
            ins.update(zip(b, c2[g * l:(g + 1) * l]))
            outs.append(C.comp_s(net, a, b, bool(signed)) if kind == 0 else C.comp_le(net, a, b, bool(signed)))
        val = C.eval_encrypted(net, keys, ins)
        assert_same(got, val[outs], f"compare {name} signed={signed}")
        sv = lambda v: v - 16 if signed and v >= 8 else v
        truth = [int(sv(a) < sv(b)) if kind == 0 else int(sv(a) <= sv(b)) for a, b in pairs]
        assert oracle.decrypt(keys.s, got).tolist() == truth


def _query_inputs(keys, seed, l, px, py, boxes, services):
    x = _enc_bits(keys, _bits(px, l), seed, 0)
    y = _enc_bits(keys, _bits(py, l), seed, l)
    bb = np.concatenate([_bits(v, l) for box in boxes for v in box])
    bx = _enc_bits(keys, bb, seed, 2 * l)
    sv = np.concatenate([np.asarray(s, np.uint8) for s in services])
    sc = _enc_bits(keys, sv, seed, 2 * l + len(bb))
    return x, y, bx, sc


def _oracle_locpir(keys, l, x, y, bx, sc, nbox, m, comb, signed):
    net = C.Netlist()
    xw, yw = net.inputs(l), net.inputs(l)
    bw = [tuple(net.inputs(l) for _ in range(4)) for _ in range(nbox)]
    sw = [net.inputs(m) for _ in range(nbox)]
    out = C.locpir(net, xw, yw, bw, sw, comb, bool(signed))
    ins = dict(zip(xw, x))
    ins.update(zip(yw, y))
    flat_b = [w for box in bw for part in box for w in part]
    ins.update(zip(flat_b, bx))
    ins.update(zip([w for s in sw for w in s], sc))
    return C.eval_encrypted(net, keys, ins)[out]


@pytest.mark.parametrize("comb", [C.XOR_TREE, C.XOR_CHAIN, C.OR_TREE])
def test_locpir_small_multibox_matches_oracle(gpu_ctx, keys, comb):
    l, m = 4, 3
    boxes = [(2, 9, 1, 7), (9, 15, 3, 12), (0, 3, 10, 15)]
    services = [[1, 0, 1], [0, 1, 1], [1, 1, 0]]
    px, py = 10, 5  # inside box 1 only
    x, y, bx, sc = _query_inputs(keys, 400 + comb, l, px, py, boxes, services)
    out = empty_dev(m, keys.params.n + 1)
    gpu_ctx.lp_locpir_query(l, 0, to_dev(x), to_dev(y), len(boxes), to_dev(bx), m, to_dev(sc), comb, out)
    gpu_ctx.lp_sync()
    got = to_host(out)
    assert_same(got, _oracle_locpir(keys, l, x, y, bx, sc, len(boxes), m, comb, 0), f"locpir comb={comb}")
    assert oracle.decrypt(keys.s, got).tolist() == services[1]


def test_locpir_single_query_paper_shape(gpu_ctx, keys):
    """One query of the single-query workload: 16-bit unsigned coordinates (Seoul's
    Table 1 box shifted by +90 / +180 degrees, 7 fraction bits), one box, a 64-bit
    service holding 427; the point lies inside, so the service comes back."""
    l, m = 16, 64
    enc = lambda deg: int(np.floor(deg * 128 + 0.5))
    box = (enc(37.4758 + 90), enc(37.6195 + 90), enc(126.8831 + 180), enc(127.1331 + 180))
    px, py = enc(37.55 + 90), enc(127.0 + 180)
    svc = _bits(427, m)
    x, y, bx, sc = _query_inputs(keys, 0, l, px, py, [box], [svc])
    out = empty_dev(m, keys.params.n + 1)
    gpu_ctx.lp_locpir_query(l, 0, to_dev(x), to_dev(y), 1, to_dev(bx), m, to_dev(sc), C.XOR_TREE, out)
    gpu_ctx.lp_sync()
    got = to_host(out)
    assert_same(got, _oracle_locpir(keys, l, x, y, bx, sc, 1, m, C.XOR_TREE, 0), "locpir single query")
    dec = oracle.decrypt(keys.s, got)
    assert sum(int(b) << j for j, b in enumerate(dec)) == 427


def test_locpir_batch_uneven_equals_single(gpu_ctx, keys):
    """Queries of different l, B_x and m scheduled together give the same ciphertexts as
    each query alone."""
    n = keys.params.n
    specs = [(4, [(1, 9, 2, 12)], 2, [[1, 1]], 5, 6),
             (6, [(3, 40, 0, 63), (40, 60, 5, 30)], 3, [[1, 0, 1], [0, 1, 1]], 45, 20),
             (5, [(0, 31, 0, 31)], 1, [[1]], 7, 7)]
    qs, singles = [], []
    for k, (l, boxes, m, services, px, py) in enumerate(specs):
        x, y, bx, sc = _query_inputs(keys, 500 + k, l, px, py, boxes, services)
        d = dict(l=l, is_signed=0, n_boxes=len(boxes), m=m, comb=0, x=to_dev(x), y=to_dev(y), boxes=to_dev(bx),
                 services=to_dev(sc), out_service=empty_dev(m, n + 1))
        qs.append(d)
        alone = empty_dev(m, n + 1)
        gpu_ctx.lp_locpir_query(l, 0, d["x"], d["y"], len(boxes), d["boxes"], m, d["services"], 0, alone)
        singles.append(alone)
    gpu_ctx.lp_locpir_batch(qs)
    gpu_ctx.lp_sync()
    for k, (q, s) in enumerate(zip(qs, singles)):
        assert_same(to_host(q["out_service"]), to_host(s), f"query {k}")
    # and the first query against the oracle
    l, boxes, m, services, px, py = specs[1]
    x, y, bx, sc = _query_inputs(keys, 501, l, px, py, boxes, services)
    assert_same(to_host(qs[1]["out_service"]), _oracle_locpir(keys, l, x, y, bx, sc, 2, m, 0, 0), "batch vs oracle")
