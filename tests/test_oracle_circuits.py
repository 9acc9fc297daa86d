"""Pins of the oracle's LocPIR circuits: integer truth by brute force, the paper's
worked example and Table 1, gate counts, and a few encrypted runs."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import circuits as C

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _bits(v, l):
    return [int(b) for b in synth.int_to_bits(v, l)]


def _signed(v, l):
    v &= (1 << l) - 1
    return v - (1 << l) if v >> (l - 1) else v


@pytest.mark.parametrize("signed", [False, True])
def test_comp_s_and_le_brute_force_l4(signed):
    l = 4
    net = C.Netlist()
    a, b = net.inputs(l), net.inputs(l)
    lt = C.comp_s(net, a, b, signed)
    le = C.comp_le(net, a, b, signed)
    for x1, x2 in itertools.product(range(16), repeat=2):
        vals = C.eval_plain(net, dict(zip(a + b, _bits(x1, l) + _bits(x2, l))))
        v1, v2 = (_signed(x1, l), _signed(x2, l)) if signed else (x1, x2)
        assert vals[lt] == int(v1 < v2), (x1, x2)
        assert vals[le] == int(v1 <= v2), (x1, x2)


def test_unflipped_loop_is_unsigned_less_than():
    """Without the MSB flip the loop alone already orders unsigned values; the flip
    turns it into the signed two's-complement order (reading of Section 4.2)."""
    l = 4
    net = C.Netlist()
    a, b = net.inputs(l), net.inputs(l)
    t0 = net.const(0)
    for i in range(l):
        t1 = net.gate(oracle.XNOR, a[i], b[i])
        t0 = net.gate(oracle.MUX, t1, t0, b[i])
    for x1, x2 in itertools.product(range(16), repeat=2):
        vals = C.eval_plain(net, dict(zip(a + b, _bits(x1, l) + _bits(x2, l))))
        assert vals[t0] == int(x1 < x2)


def _locpir_net(l, boxes, m, comb, signed):
    net = C.Netlist()
    x, y = net.inputs(l), net.inputs(l)
    bw = [tuple(net.inputs(l) for _ in range(4)) for _ in boxes]
    sw = [net.inputs(m) for _ in boxes]
    out = C.locpir(net, x, y, bw, sw, comb, signed)
    return net, x, y, bw, sw, out


def _assign(l, m, x, y, bw, sw, px, py, boxes, services):
    inp = dict(zip(x, _bits(px, l)))
    inp.update(zip(y, _bits(py, l)))
    for (X1, X2, Y1, Y2), box, w in zip(bw, boxes, sw):
        for wires, v in zip((X1, X2, Y1, Y2), box):
            inp.update(zip(wires, _bits(v, l)))
    for w, s in zip(sw, services):
        inp.update(zip(w, s))
    return inp


@pytest.mark.parametrize("comb", [C.XOR_TREE, C.XOR_CHAIN, C.OR_TREE])
def test_locpir_brute_force_l4(comb):
    l, m = 4, 4
    boxes = [(2, 9, 1, 7), (9, 15, 3, 12), (0, 3, 10, 16 - 1)]
    services = [[1, 0, 1, 1], [0, 1, 1, 0], [1, 1, 0, 1]]
    net, x, y, bw, sw, out = _locpir_net(l, boxes, m, comb, False)
    for px, py in itertools.product(range(16), repeat=2):
        vals = C.eval_plain(net, _assign(l, m, x, y, bw, sw, px, py, boxes, services))
        want = [0] * m
        for (X1, X2, Y1, Y2), s in zip(boxes, services):
            if X1 <= px < X2 and Y1 <= py < Y2:
                want = [(w | v) if comb == C.OR_TREE else (w ^ v) for w, v in zip(want, s)]
        assert [vals[o] for o in out] == want, (px, py)


def _fixed(deg, frac=7):
    """Fixed-point encoding of Section 4.1 (9 integer bits, 7 fraction bits), rounded
    half away from zero."""
    v = deg * (1 << frac)
    return int(math.floor(abs(v) + 0.5)) * (1 if v >= 0 else -1)


def test_paper_illustrative_example():
    g = json.load(open(os.path.join(GOLD, "example.json")))
    l, m = 16, 3
    box = [_fixed(g["box"][k]) for k in ("lat1", "lat2", "lon1", "lon2")]
    svc = [int(c) for c in reversed(g["service_bits_msb_first"])]
    net, x, y, bw, sw, out = _locpir_net(l, [box], m, C.XOR_TREE, True)
    # Expose the comparator results too.
    vals = C.eval_plain(net, _assign(l, m, x, y, bw, sw, _fixed(g["x"]), _fixed(g["y"]), [box], [svc]))
    res = "".join(str(vals[o]) for o in reversed(out))
    assert res == g["expected_msb_first"]


def test_table1_cities_return_their_service():
    g = json.load(open(os.path.join(GOLD, "table1.json")))
    rows = g["rows"]
    l, m = 16, 9
    boxes = [tuple(_fixed(r[k]) for k in ("lat1", "lat2", "lon1", "lon2")) for r in rows]
    services = [[int(b) for b in synth.int_to_bits(r["service"], m)] for r in rows]
    net, x, y, bw, sw, out = _locpir_net(l, boxes, m, C.XOR_TREE, True)
    assert max(r["service"] for r in rows) < 1 << m
    for r in rows:
        px = _fixed((r["lat1"] + r["lat2"]) / 2)
        py = _fixed((r["lon1"] + r["lon2"]) / 2)
        vals = C.eval_plain(net, _assign(l, m, x, y, bw, sw, px, py, boxes, services))
        got = sum(vals[o] << j for j, o in enumerate(out))
        assert got == r["service"], r["city"]
    vals = C.eval_plain(net, _assign(l, m, x, y, bw, sw, _fixed(37.5), _fixed(130.1), boxes, services))
    assert sum(vals[o] for o in out) == 0
    # Negative coordinates (southern / western hemisphere) order correctly too.
    vals = C.eval_plain(net, _assign(l, m, x, y, bw, sw, _fixed(-37.5), _fixed(-127.0), boxes, services))
    assert sum(vals[o] for o in out) == 0


@pytest.mark.parametrize("l,bx,m", [(4, 1, 4), (16, 1, 64), (32, 1, 256), (16, 9, 9), (24, 5, 8)])
def test_gate_counts(l, bx, m):
    """Comparator = l XNOR + l MUX = 3l bootstraps (Section 6.2); per box 12l + 3 + m
    blind rotations and 8l + 3 + m key switches; the XOR tree adds (B_x - 1) m."""
    net = C.Netlist()
    x, y = net.inputs(l), net.inputs(l)
    bw = [tuple(net.inputs(l) for _ in range(4)) for _ in range(bx)]
    sw = [net.inputs(m) for _ in range(bx)]
    C.locpir(net, x, y, bw, sw, C.XOR_TREE, False)
    br, ks = net.bootstraps()
    assert br == bx * (12 * l + 3 + m) + (bx - 1) * m
    assert ks == bx * (8 * l + 3 + m) + (bx - 1) * m
    depth = max(C.depths(net))
    assert depth == l + 1 + 2 + 1 + math.ceil(math.log2(bx))


@pytest.mark.slow
def test_comparator_encrypted_l4(keys_noiseless):
    """Encrypted HomCompS/HomCompLE at l = 4 decrypt to integer truth."""
    k = keys_noiseless
    l = 4
    pairs = [(3, 11), (11, 3), (7, 7)]
    net = C.Netlist()
    wires = []
    for _ in pairs:
        a, b = net.inputs(l), net.inputs(l)
        wires.append((a, b, C.comp_s(net, a, b, False), C.comp_le(net, a, b, False)))
    inputs = {}
    seq = 0
    for (x1, x2), (a, b, _, _) in zip(pairs, wires):
        bits_ = _bits(x1, l) + _bits(x2, l)
        ct = oracle.encrypt(k.s, bits_, synth.lwe_draws(70, len(bits_), offset=seq))
        seq += len(bits_)
        inputs.update(zip(a + b, ct))
    val = C.eval_encrypted(net, k, inputs)
    for (x1, x2), (_, _, lt, le) in zip(pairs, wires):
        assert oracle.decrypt(k.s, val[lt])[0] == int(x1 < x2)
        assert oracle.decrypt(k.s, val[le])[0] == int(x1 <= x2)


# ---------------------------------------------------------------------------
# Server-known bounds (beyond the paper).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("signed", [False, True])
@pytest.mark.parametrize("l", [1, 2, 4])
def test_comp_s_known_brute_force(signed, l):
    """x < K for every encrypted x and known K of l bits, and the gate count: one
    AND/OR per step after the first step whose bit differs from the running constant."""
    for K in range(1 << l):
        net = C.Netlist()
        a = net.inputs(l)
        lt = C.comp_s_known(net, a, K, signed)
        kv = _signed(K, l) if signed else K
        for x in range(1 << l):
            vals = C.eval_plain(net, dict(zip(a, _bits(x, l))))
            xv = _signed(x, l) if signed else x
            assert vals[lt] == int(xv < kv), (x, K)
        kb = _bits(K, l)
        if signed:
            kb[l - 1] ^= 1
        first = next((i for i, b in enumerate(kb) if b != 0), None)
        assert net.bootstraps()[0] == (0 if first is None else l - 1 - first)


@pytest.mark.parametrize("comb", [C.XOR_TREE, C.XOR_CHAIN, C.OR_TREE])
def test_locpir_known_matches_encrypted_bounds_l4(comb):
    """The known-bounds circuit computes what Algorithm 3 computes with the same bounds
    encrypted, for every point of a 4-bit grid."""
    l, m = 4, 3
    boxes = [(2, 9, 0, 16 - 1), (5, 6, 3, 12), (0, 1, 8, 9)]
    services = [[1, 0, 1], [0, 1, 1], [1, 1, 0]]
    net = C.Netlist()
    x, y = net.inputs(l), net.inputs(l)
    sw = [net.inputs(m) for _ in boxes]
    out = C.locpir_known(net, x, y, boxes, sw, comb, False)
    for px, py in itertools.product(range(16), repeat=2):
        inputs = dict(zip(x, _bits(px, l)))
        inputs.update(zip(y, _bits(py, l)))
        for w, sv in zip(sw, services):
            inputs.update(zip(w, sv))
        vals = C.eval_plain(net, inputs)
        want = [0] * m
        for (x1, x2, y1, y2), sv in zip(boxes, services):
            if x1 <= px < x2 and y1 <= py < y2:
                want = [(u | v) if comb == C.OR_TREE else (u ^ v) for u, v in zip(want, sv)]
        assert [vals[o] for o in out] == want, (px, py)


def test_locpir_known_bootstrap_count():
    """Per box the known-bounds circuit needs at most 4(l - 1) + 3 + m blind rotations,
    against 12l + 3 + m with encrypted bounds."""
    l, m = 16, 8
    rng = np.random.default_rng(5)
    bounds = [tuple(int(v) for v in rng.integers(0, 1 << l, 4)) for _ in range(5)]
    net = C.Netlist()
    x, y = net.inputs(l), net.inputs(l)
    sw = [net.inputs(m) for _ in bounds]
    C.locpir_known(net, x, y, bounds, sw, C.XOR_TREE, False)
    br, ks = net.bootstraps()
    assert br == ks
    assert br <= 5 * (4 * (l - 1) + 3 + m) + 4 * m


@pytest.mark.slow
def test_comparator_known_encrypted_l4(keys_noiseless):
    """Encrypted x against known K at l = 4 (signed and unsigned) decrypts to truth."""
    k = keys_noiseless
    l = 4
    cases = [(3, 11, False), (11, 3, False), (7, 7, False), (12, 3, True), (3, 12, True)]
    net = C.Netlist()
    wires = []
    for _ in cases:
        wires.append(net.inputs(l))
    outs = [C.comp_s_known(net, a, K, sg) for a, (_, K, sg) in zip(wires, cases)]
    inputs = {}
    for j, ((x, _, _), a) in enumerate(zip(cases, wires)):
        ct = oracle.encrypt(k.s, _bits(x, l), synth.lwe_draws(71, l, offset=j * l))
        inputs.update(zip(a, ct))
    val = C.eval_encrypted(net, k, inputs)
    for (x, K, sg), o in zip(cases, outs):
        xv, kv = (_signed(x, l), _signed(K, l)) if sg else (x, K)
        assert oracle.decrypt(k.s, val[o])[0] == int(xv < kv)
