"""The query server (continuous batching): queries of different shapes arriving over time
share bootstrap batches, wait for pool memory when the budget is full, and each result is
bit-identical to the same query evaluated alone."""
import time

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu


def _enc(keys, bits, seed, offset):
    return oracle.encrypt(keys.s, bits, synth.lwe_draws(seed, len(bits), offset=offset))


def _query(keys, seed, l, boxes, services, px, py, comb=0):
    n = keys.params.n
    bits = lambda v: synth.int_to_bits(v, l)
    x = _enc(keys, bits(px), seed, 0)
    y = _enc(keys, bits(py), seed, l)
    bb = np.concatenate([bits(v) for box in boxes for v in box])
    bx = _enc(keys, bb, seed, 2 * l)
    sv = np.concatenate([np.asarray(s, np.uint8) for s in services])
    sc = _enc(keys, sv, seed, 2 * l + len(bb))
    m = len(services[0])
    return dict(l=l, is_signed=0, n_boxes=len(boxes), m=m, comb=comb, x=to_dev(x), y=to_dev(y), boxes=to_dev(bx),
                services=to_dev(sc), out_service=empty_dev(m, n + 1))


SPECS = [
    (4, [(1, 9, 2, 12)], [[1, 0]], 5, 6),
    (6, [(3, 40, 0, 63), (40, 60, 5, 30)], [[1, 0, 1], [0, 1, 1]], 45, 20),
    (5, [(0, 31, 0, 31)], [[1]], 7, 7),
    (3, [(1, 5, 1, 5), (5, 7, 0, 7), (0, 2, 0, 2)], [[1, 1], [0, 1], [1, 0]], 6, 3),
    (4, [(0, 15, 0, 15)], [[0, 1, 1, 0]], 9, 2),
]


def _wires(l, nb, m):
    # inputs + gates (+1 constant): 2l + 4 l nb + m nb inputs, per box 8l + 3 + m gates, tree (nb - 1) m
    return 2 * l + 4 * l * nb + m * nb + nb * (8 * l + 3 + m) + (nb - 1) * m + 1


def test_server_mixed_arrivals_match_single_queries(gpu_ctx, keys):
    n = keys.params.n
    qs = [_query(keys, 900 + k, l, boxes, svc, px, py, comb=k % 2) for k, (l, boxes, svc, px, py) in enumerate(SPECS)]
    # Each query alone, through the batch entry point.
    alone = []
    for q in qs:
        out = empty_dev(q["m"], n + 1)
        gpu_ctx.lp_locpir_query(q["l"], 0, q["x"], q["y"], q["n_boxes"], q["boxes"], q["m"], q["services"],
                                q["comb"], out)
        alone.append(out)
    gpu_ctx.lp_sync()
    # A budget that holds the two largest queries at once, so later arrivals wait for memory.
    sizes = [_wires(l, len(b), len(s[0])) * (n + 1) * 4 for (l, b, s, _, _) in SPECS]
    budget = sorted(sizes)[-1] + sorted(sizes)[-2]
    gpu_ctx.lp_server_start(budget)
    try:
        tickets = []
        for k, q in enumerate(qs):
            tickets.append(gpu_ctx.lp_server_submit(q))
            if k % 2 == 1:
                time.sleep(0.05)  # staggered arrivals: later queries join batches already in flight
        for t in tickets:
            gpu_ctx.lp_server_wait(t, 300000)
            assert gpu_ctx.lp_server_poll(t)
        st = gpu_ctx.lp_server_stats()
    finally:
        gpu_ctx.lp_server_stop()
    for k, (q, a) in enumerate(zip(qs, alone)):
        assert_same(to_host(q["out_service"]), to_host(a), f"query {k} in the mix vs alone")
    assert st["completed"] == len(qs) and st["admitted"] == len(qs)
    # Per box 12l + 3 + m blind rotations; the combine adds (B_x - 1) m XORs as a tree (even
    # k) or B_x m as the printed chain (odd k).
    assert st["bootstraps"] == sum(
        len(bx) * (12 * l + 3 + len(s[0])) + (len(bx) - (k % 2 == 0)) * len(s[0])
        for k, (l, bx, s, _, _) in enumerate(SPECS))
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    # Fewer ticks than evaluating the queries one after another: levels were shared.
    depth = lambda l, nb: l + 4 + int(np.ceil(np.log2(nb)))
    assert st["ticks"] < sum(depth(l, len(b)) for (l, b, _, _, _) in SPECS)
    # and the result decrypts to the plaintext truth for the query inside box 1 of spec 1
    dec = oracle.decrypt(keys.s, to_host(qs[1]["out_service"]))
    assert dec.tolist() == [0, 1, 1]


def test_server_budget_refusals(gpu_ctx, keys):
    from paper_2407_19871_gb300.locpir import LP_EBUSY, LP_SERVER_REJECT, LocpirError
    n = keys.params.n
    l, boxes, svc, px, py = SPECS[0]
    one = _wires(l, len(boxes), len(svc[0])) * (n + 1) * 4
    q1 = _query(keys, 950, l, boxes, svc, px, py)
    q2 = _query(keys, 951, l, boxes, svc, px, py)
    big = _query(keys, 952, *SPECS[1][:3], *SPECS[1][3:])
    gpu_ctx.lp_server_start(one + (n + 1) * 4 * 8, LP_SERVER_REJECT)
    try:
        with pytest.raises(LocpirError) as e:
            gpu_ctx.lp_server_submit(big)   # larger than the whole budget
        assert e.value.code == LP_EBUSY
        t1 = gpu_ctx.lp_server_submit(q1)
        with pytest.raises(LocpirError) as e:
            gpu_ctx.lp_server_submit(q2)    # budget held by q1 (reject policy)
        assert e.value.code == LP_EBUSY
        gpu_ctx.lp_server_wait(t1, 300000)
        st = gpu_ctx.lp_server_stats()
        assert st["rejected"] == 2 and st["completed"] == 1
    finally:
        gpu_ctx.lp_server_stop()


def test_server_mixes_known_and_encrypted_bounds(gpu_ctx, keys):
    """Known-bounds queries (lp_server_submit_known) and encrypted-bounds queries share the
    server's ticks; each known-bounds result equals lp_locpir_known_batch on the same query
    alone, bit for bit, and each encrypted one equals lp_locpir_query alone."""
    n = keys.params.n
    enc = [_query(keys, 950 + k, l, boxes, svc, px, py) for k, (l, boxes, svc, px, py) in enumerate(SPECS[:3])]
    known = []
    for k, (l, boxes, svc, px, py) in enumerate(SPECS[1:]):
        q = _query(keys, 970 + k, l, boxes, svc, px, py, comb=k % 3)
        known.append(dict(l=q["l"], is_signed=0, n_boxes=q["n_boxes"], m=q["m"], comb=q["comb"], x=q["x"], y=q["y"],
                          bounds=boxes, services=q["services"], out_service=empty_dev(q["m"], n + 1)))
    alone_enc = []
    for q in enc:
        out = empty_dev(q["m"], n + 1)
        gpu_ctx.lp_locpir_query(q["l"], 0, q["x"], q["y"], q["n_boxes"], q["boxes"], q["m"], q["services"],
                                q["comb"], out)
        alone_enc.append(out)
    alone_known = []
    for q in known:
        qa = dict(q, out_service=empty_dev(q["m"], n + 1))
        gpu_ctx.lp_locpir_known_batch([qa])
        alone_known.append(qa["out_service"])
    gpu_ctx.lp_sync()
    gpu_ctx.lp_server_start(1 << 30)
    try:
        tickets = []
        for k in range(max(len(enc), len(known))):
            if k < len(known):
                tickets.append(gpu_ctx.lp_server_submit_known(known[k]))
            if k < len(enc):
                tickets.append(gpu_ctx.lp_server_submit(enc[k]))
        for t in tickets:
            gpu_ctx.lp_server_wait(t, 300000)
    finally:
        gpu_ctx.lp_server_stop()
    for k, (q, a) in enumerate(zip(known, alone_known)):
        assert_same(to_host(q["out_service"]), to_host(a), f"known-bounds query {k} in the mix vs alone")
    for k, (q, a) in enumerate(zip(enc, alone_enc)):
        assert_same(to_host(q["out_service"]), to_host(a), f"encrypted-bounds query {k} in the mix vs alone")
    # spec 1's point (45, 20) lies in its second box only
    assert oracle.decrypt(keys.s, to_host(known[0]["out_service"])).tolist() == [0, 1, 1]
