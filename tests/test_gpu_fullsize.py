"""Parity at the workloads' full sizes, in the launch configurations the bench times.

* 65,536 NAND gates (the gate-bootstrapping microbenchmark): one batched launch over every SM.
  Sampled outputs, at CTA-group and wave boundaries, equal the oracle's word for word, and
  every output decrypts to the plaintext truth.
* 4,096 city-shaped LocPIR queries (l = 32 unsigned, one box, 256-bit service) in one
  CUDA-graph plan.  Sampled queries' output ciphertexts equal the oracle's circuit
  evaluation of those queries, word for word.  With this parameter set the comparators'
  chained MUX decides wrongly with probability about 1.9e-5 per decision (the selector's and
  the previous MUX output's noise add up to sigma ~ 0.030 against a 1/8 margin), and a wrong
  decision changes a comparison only when every more significant bit of the operands agrees:
  about 1.5e-4 per query, 0.6 flipped queries per batch on average.  Every query whose
  service does not decrypt to the truth must therefore be reproduced word for word by the
  oracle: the flip is then the parameters' noise, identical on both sides, and not a fault
  of the GPU path."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host
from oracle import circuits as C

pytestmark = pytest.mark.gpu


def test_nand_65536_sampled(gpu_ctx, keys):
    count = 65536
    A, B = synth.nand_pairs(1, count)
    a = oracle.encrypt(keys.s, A, synth.lwe_draws(1, count))
    b = oracle.encrypt(keys.s, B, synth.lwe_draws(1, count, offset=count))
    out = empty_dev(count, keys.params.n + 1)
    gpu_ctx.lp_gate_batch(oracle.NAND, to_dev(a), to_dev(b), None, out, count)
    gpu_ctx.lp_sync()
    got = to_host(out)
    # 256 outputs: 200 spread evenly over the batch, plus the first and last slots of CTA
    # groups (6 ciphertexts per CTA) and of waves (152 CTAs: 912 ciphertexts) at the start,
    # the middle and the tail; plus any output that decrypts wrongly (fresh inputs make that
    # very unlikely here; it would have to be the parameters' noise, reproduced by the oracle).
    bad = np.flatnonzero(oracle.decrypt(keys.s, got) != 1 - (A & B))
    assert len(bad) <= 2, f"{len(bad)} NAND outputs decrypt wrongly"
    edges = [0, 1, 4, 5, 6, 7, 11, 12, 905, 911, 912, 913, 917, 918, 1823, 1824, 32766, 32767, 32768, 32769,
             count - 913, count - 912, count - 911, count - 7, count - 6, count - 5, count - 2, count - 1]
    spread = np.linspace(0, count - 1, 256 - len(edges)).astype(np.int64)
    idx = np.unique(np.concatenate([edges, spread, bad]).astype(np.int64))
    assert len(idx) >= 250
    assert_same(got[idx], oracle.gate_batch(keys, oracle.NAND, a[idx], b[idx]), "NAND 65,536 sampled")


def test_city_4096_plan_sampled(gpu_ctx, keys):
    from paper_2407_19871_gb300.locpir import LP_XOR_TREE
    nq, l, m = 4096, 32, 256
    n = keys.params.n
    qs = synth.city_batch(2, nq, l, m)
    per_q = 2 * l + 4 * l + m
    bits = np.concatenate([np.concatenate([synth.int_to_bits(q.x, l), synth.int_to_bits(q.y, l)] +
                                          [synth.int_to_bits(v, l) for v in q.box] + [q.service]) for q in qs])
    # Encrypted in chunks (the draws of 1.8 M ciphertexts at once would need ~14 GB of host memory).
    ct = np.empty((len(bits), n + 1), np.uint32)
    step = 256 * per_q
    for o in range(0, len(bits), step):
        e = min(o + step, len(bits))
        ct[o:e] = oracle.encrypt(keys.s, bits[o:e], synth.lwe_draws(2, e - o, offset=o))
    dct = to_dev(ct)
    out = empty_dev(nq * m, n + 1)
    queries = []
    for k in range(nq):
        b0 = k * per_q
        queries.append(dict(l=l, is_signed=0, n_boxes=1, m=m, comb=LP_XOR_TREE, x=dct[b0:b0 + l],
                            y=dct[b0 + l:b0 + 2 * l], boxes=dct[b0 + 2 * l:b0 + 6 * l],
                            services=dct[b0 + 6 * l:b0 + per_q], out_service=out[k * m:(k + 1) * m]))
    plan = gpu_ctx.lp_plan_locpir(queries)
    try:
        plan.lp_plan_run()
        gpu_ctx.lp_sync()
    finally:
        plan.lp_plan_destroy()
    got = to_host(out)
    dec = oracle.decrypt(keys.s, got).reshape(nq, m)
    wrong = []
    for k, q in enumerate(qs):
        x1, x2, y1, y2 = q.box
        want = q.service if (x1 <= q.x < x2 and y1 <= q.y < y2) else np.zeros(m, np.uint8)
        if dec[k].tolist() != want.tolist():
            wrong.append(k)
    # Poisson(0.6): more than 4 flipped queries has probability < 5e-4.
    assert len(wrong) <= 4, f"{len(wrong)} queries decrypt wrongly: {wrong[:10]}"

    def oracle_query(k):
        b0 = k * per_q
        net = C.Netlist()
        xw, yw = net.inputs(l), net.inputs(l)
        bw = tuple(net.inputs(l) for _ in range(4))
        sw = net.inputs(m)
        outs = C.locpir(net, xw, yw, [bw], [sw], C.XOR_TREE, False)
        ins = dict(zip(xw, ct[b0:b0 + l]))
        ins.update(zip(yw, ct[b0 + l:b0 + 2 * l]))
        ins.update(zip([w for part in bw for w in part], ct[b0 + 2 * l:b0 + 6 * l]))
        ins.update(zip(sw, ct[b0 + 6 * l:b0 + per_q]))
        return C.eval_encrypted(net, keys, ins)[outs]

    # The first and last queries, one in the middle, the last one inside its box, and every
    # query that decrypted wrongly, against the oracle.
    sample = [0, 2049, nq - 1, max(i for i in range(nq) if i % 2 == 0)]
    for k in sorted(set(sample + wrong)):
        assert_same(got[k * m:(k + 1) * m], oracle_query(k), f"city query {k} of 4,096")
