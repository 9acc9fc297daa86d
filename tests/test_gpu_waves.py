"""Uneven LocPIR queries in memory-budgeted waves (lp_locpir_batch_waves), the multi-box
workload's shape at reduced size: per-query box counts and coordinate widths 16 / 24 / 32 bits
differ, per-box results combined by an encrypted OR tree (Algorithms 3-5).

* A budget below the batch's need splits it into several waves, and every output ciphertext
  equals the single-call lp_locpir_batch over the same queries word for word.
* One query of each width (16, 24 and 32 bits) equals the oracle's circuit evaluation word for
  word, and every output decrypts to the plaintext truth."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host
from oracle import circuits as C

pytestmark = pytest.mark.gpu

M = 4           # service bits per box (the full workload has 512)


def _inputs(keys, q, seed):
    bits = np.concatenate([synth.int_to_bits(q.x, q.l), synth.int_to_bits(q.y, q.l)] +
                          [synth.int_to_bits(v, q.l) for b in q.boxes for v in b] +
                          [np.asarray(q.services, np.uint8).reshape(-1)])
    return oracle.encrypt(keys.s, bits, synth.lwe_draws(seed, len(bits)))


def _truth(q):
    want = np.zeros(M, np.uint8)
    for (x1, x2, y1, y2), sv in zip(q.boxes, np.asarray(q.services, np.uint8).reshape(-1, M)):
        if x1 <= q.x < x2 and y1 <= q.y < y2:
            want |= sv
    return want


def _oracle_query(keys, q, ct):
    l, nb = q.l, len(q.boxes)
    net = C.Netlist()
    xw, yw = net.inputs(l), net.inputs(l)
    bw = [tuple(net.inputs(l) for _ in range(4)) for _ in range(nb)]
    sw = [net.inputs(M) for _ in range(nb)]
    out = C.locpir(net, xw, yw, bw, sw, C.OR_TREE, False)
    wires = xw + yw + [w for box in bw for part in box for w in part] + [w for s in sw for w in s]
    return C.eval_encrypted(net, keys, dict(zip(wires, ct)))[out]


def test_waves_match_single_batch_and_oracle(gpu_ctx, keys):
    from paper_2407_19871_gb300.locpir import LP_OR_TREE
    n = keys.params.n
    W = n + 1
    qs = synth.multibox_batch(5, 4, m=M, max_boxes=2)      # widths 24, 32, 16, 16; 1, 1, 2, 2 boxes
    assert {q.l for q in qs} == {16, 24, 32}
    cts = [_inputs(keys, q, 600 + k) for k, q in enumerate(qs)]

    def queries(outs):
        res = []
        for q, ct, o in zip(qs, cts, outs):
            l, nb = q.l, len(q.boxes)
            d = to_dev(ct)
            res.append(dict(l=l, is_signed=0, n_boxes=nb, m=M, comb=LP_OR_TREE, x=d[:l], y=d[l:2 * l],
                            boxes=d[2 * l:2 * l + 4 * l * nb], services=d[2 * l + 4 * l * nb:], out_service=o))
        return res

    one = [empty_dev(M, W) for _ in qs]
    gpu_ctx.lp_locpir_batch(queries(one))
    waved = [empty_dev(M, W) for _ in qs]
    # Each query's circuit needs 0.9-1.2 MB here (348-460 wires of 2,524 bytes plus job records),
    # 4.3 MB together: a 2.5 MB budget fits at most two queries per wave.
    waves = gpu_ctx.lp_locpir_batch_waves(queries(waved), 5 << 19)
    gpu_ctx.lp_sync()
    assert waves >= 2
    for k, (a, b) in enumerate(zip(one, waved)):
        assert_same(to_host(b), to_host(a), f"query {k}: waves vs one batch")
    for k, q in enumerate(qs):
        assert oracle.decrypt(keys.s, to_host(waved[k])).tolist() == _truth(q).tolist(), f"query {k}"
    for k in (0, 1, 2):                                      # l = 24, 32, 16
        assert_same(to_host(waved[k]), _oracle_query(keys, qs[k], cts[k]), f"query {k} (l={qs[k].l}) vs oracle")


def test_waves_reject_a_query_above_the_budget(gpu_ctx, keys):
    from paper_2407_19871_gb300.locpir import LP_ENOMEM, LocpirError
    n = keys.params.n
    t = empty_dev(2 * 16 + 4 * 16 + M, n + 1)
    q = dict(l=16, is_signed=0, n_boxes=1, m=M, comb=0, x=t[:16], y=t[16:32], boxes=t[32:96], services=t[96:],
             out_service=empty_dev(M, n + 1))
    with pytest.raises(LocpirError) as e:
        gpu_ctx.lp_locpir_batch_waves([q], 1 << 16)
    assert e.value.code == LP_ENOMEM
