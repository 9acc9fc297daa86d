"""The persistent circuit executor (LP_EXEC_PERSISTENT): one kernel runs every bootstrap level of
a scheduled LocPIR batch (Algorithms 2-5), its CTAs taking each level's gate groups and
key-switch batches from device-side counters.  Its outputs equal the per-level executor's word
for word (and a sampled query the oracle's), in direct calls and in a plan's CUDA graph; a
barrier wait that sees no progress gives up with LP_ETIMEOUT and leaves the context usable."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host
from oracle import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture
def exec_ctx(gpu_ctx):
    yield gpu_ctx
    from paper_2407_19871_gb300.locpir import LP_EXEC_LEVELS
    gpu_ctx.lp_set_executor(LP_EXEC_LEVELS)


def _city(keys, nq, l, m, seed):
    qs = synth.city_batch(seed, nq, l, m)
    per_q = 6 * l + m
    bits = np.concatenate([np.concatenate([synth.int_to_bits(q.x, l), synth.int_to_bits(q.y, l)] +
                                          [synth.int_to_bits(v, l) for v in q.box] + [q.service]) for q in qs])
    ct = oracle.encrypt(keys.s, bits, synth.lwe_draws(seed, len(bits)))
    return qs, ct, per_q


def _queries(ct_dev, qs, l, m, per_q, out):
    from paper_2407_19871_gb300.locpir import LP_XOR_TREE
    res = []
    for k in range(len(qs)):
        b0 = k * per_q
        res.append(dict(l=l, is_signed=0, n_boxes=1, m=m, comb=LP_XOR_TREE, x=ct_dev[b0:b0 + l],
                        y=ct_dev[b0 + l:b0 + 2 * l], boxes=ct_dev[b0 + 2 * l:b0 + 6 * l],
                        services=ct_dev[b0 + 6 * l:b0 + per_q], out_service=out[k * m:(k + 1) * m]))
    return res


@pytest.mark.parametrize("nq,l,m", [(3, 4, 3), (80, 6, 64)])
def test_persistent_matches_levels(exec_ctx, keys, nq, l, m):
    """3 tiny queries (sliced key switches, a single group per level); 80 queries with 64-bit
    services (5,120-output key switches over whole-table CTAs, 1,280 blind-rotation groups)."""
    from paper_2407_19871_gb300.locpir import LP_EXEC_LEVELS, LP_EXEC_PERSISTENT
    n = keys.params.n
    qs, ct, per_q = _city(keys, nq, l, m, 830 + nq)
    d = to_dev(ct)
    outs = {}
    for ex in (LP_EXEC_LEVELS, LP_EXEC_PERSISTENT):
        exec_ctx.lp_set_executor(ex)
        out = empty_dev(nq * m, n + 1)
        exec_ctx.lp_locpir_batch(_queries(d, qs, l, m, per_q, out))
        exec_ctx.lp_sync()
        outs[ex] = to_host(out)
    assert_same(outs[LP_EXEC_PERSISTENT], outs[LP_EXEC_LEVELS], "persistent vs per-level executor")
    got = oracle.decrypt(keys.s, outs[LP_EXEC_PERSISTENT]).reshape(nq, m)
    for k, q in enumerate(qs):
        x1, x2, y1, y2 = q.box
        want = q.service if (x1 <= q.x < x2 and y1 <= q.y < y2) else np.zeros(m, np.uint8)
        assert got[k].tolist() == want.tolist(), f"query {k}"
    if nq == 3:   # one query against the oracle's circuit
        net = C.Netlist()
        xw, yw = net.inputs(l), net.inputs(l)
        bw = tuple(net.inputs(l) for _ in range(4))
        sw = net.inputs(m)
        res = C.locpir(net, xw, yw, [bw], [sw], C.XOR_TREE, False)
        wires = xw + yw + [w for part in bw for w in part] + sw
        want = C.eval_encrypted(net, keys, dict(zip(wires, ct[:per_q])))[res]
        assert_same(outs[LP_EXEC_PERSISTENT][:m], want, "persistent query 0 vs oracle")


def test_persistent_plan_replays(exec_ctx, keys):
    from paper_2407_19871_gb300.locpir import LP_EXEC_LEVELS, LP_EXEC_PERSISTENT
    n = keys.params.n
    nq, l, m = 6, 5, 4
    qs, ct, per_q = _city(keys, nq, l, m, 840)
    d = to_dev(ct)
    ref = empty_dev(nq * m, n + 1)
    exec_ctx.lp_set_executor(LP_EXEC_LEVELS)
    exec_ctx.lp_locpir_batch(_queries(d, qs, l, m, per_q, ref))
    exec_ctx.lp_set_executor(LP_EXEC_PERSISTENT)
    out = empty_dev(nq * m, n + 1)
    plan = exec_ctx.lp_plan_locpir(_queries(d, qs, l, m, per_q, out))
    try:
        for _ in range(2):
            out.zero_()
            plan.lp_plan_run()
            exec_ctx.lp_sync()
            assert_same(to_host(out), to_host(ref), "persistent plan replay")
    finally:
        plan.lp_plan_destroy()


def test_persistent_barrier_wait_times_out(exec_ctx, keys):
    """A CTA that never reaches the first barrier: the others give up after 2 s without
    progress and report LP_ETIMEOUT; the context then evaluates gates normally."""
    from paper_2407_19871_gb300.locpir import LP_ETIMEOUT, LP_NAND, LocpirError
    exec_ctx.lp_selftest_exec_timeout()
    with pytest.raises(LocpirError) as e:
        exec_ctx.lp_sync()
    assert e.value.code == LP_ETIMEOUT
    n = keys.params.n
    A, B = synth.bits(850, 1, 3), synth.bits(850, 2, 3)
    a = oracle.encrypt(keys.s, A, synth.lwe_draws(851, 3))
    b = oracle.encrypt(keys.s, B, synth.lwe_draws(852, 3))
    out = empty_dev(3, n + 1)
    exec_ctx.lp_gate_batch(LP_NAND, to_dev(a), to_dev(b), None, out, 3)
    exec_ctx.lp_sync()
    assert_same(to_host(out), oracle.gate_batch(keys, oracle.NAND, a, b), "gates after the timeout")
