"""Gate batches through the C-ABI: bit-exact parity with the oracle's gates."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu

OPS = ["NAND", "AND", "OR", "XOR", "XNOR", "MUX"]


def _inputs(keys, seed, count):
    A = synth.bits(seed, 1, count)
    B = synth.bits(seed, 2, count)
    Cb = synth.bits(seed, 3, count)
    a = oracle.encrypt(keys.s, A, synth.lwe_draws(seed, count))
    b = oracle.encrypt(keys.s, B, synth.lwe_draws(seed, count, offset=count))
    c = oracle.encrypt(keys.s, Cb, synth.lwe_draws(seed, count, offset=2 * count))
    return (A, B, Cb), (a, b, c)


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("count", [1, 7])
def test_gate_batch_matches_oracle(gpu_ctx, keys, op, count):
    code = oracle.OP_NAMES[op]
    (A, B, Cb), (a, b, c) = _inputs(keys, 200 + count + code, count)
    out = empty_dev(count, keys.params.n + 1)
    gpu_ctx.lp_gate_batch(code, to_dev(a), to_dev(b), to_dev(c) if op == "MUX" else None, out, count)
    gpu_ctx.lp_sync()
    want = oracle.gate_batch(keys, code, a, b, c if op == "MUX" else None)
    got = to_host(out)
    assert_same(got, want, op)
    truth = {"NAND": 1 - (A & B), "AND": A & B, "OR": A | B, "XOR": A ^ B, "XNOR": 1 - (A ^ B),
             "MUX": np.where(A == 1, B, Cb)}[op]
    np.testing.assert_array_equal(oracle.decrypt(keys.s, got), truth)


def test_not_is_negation(gpu_ctx, keys):
    (A, _, _), (a, _, _) = _inputs(keys, 250, 5)
    out = empty_dev(5, keys.params.n + 1)
    gpu_ctx.lp_gate_batch(oracle.NOT, to_dev(a), None, None, out, 5)
    gpu_ctx.lp_sync()
    assert_same(to_host(out), oracle.gate_batch(keys, oracle.NOT, a), "NOT")


def test_host_entry_point_matches_device(gpu_ctx, keys):
    count = 5
    (_, _, _), (a, b, _) = _inputs(keys, 260, count)
    out = np.empty_like(a)
    gpu_ctx.lp_gate_batch_host(oracle.NAND, a, b, None, out, count)
    assert_same(out, oracle.gate_batch(keys, oracle.NAND, a, b), "host NAND")


def test_many_ctas_sampled(gpu_ctx, keys):
    """A batch over many CTAs (more groups than one persistent wave of the GPU):
    sampled outputs equal the oracle's; every output decrypts to the truth."""
    import torch
    count = 4 * 200 + 3
    p = keys.params
    (A, B, _), (a, b, _) = _inputs(keys, 270, count)
    out = empty_dev(count, p.n + 1)
    gpu_ctx.lp_gate_batch(oracle.NAND, to_dev(a), to_dev(b), None, out, count)
    gpu_ctx.lp_sync()
    got = to_host(out)
    idx = np.array([0, 1, 2, 3, 4, 401, 607, count - 1])
    assert_same(got[idx], oracle.gate_batch(keys, oracle.NAND, a[idx], b[idx]), "NAND sampled")
    np.testing.assert_array_equal(oracle.decrypt(keys.s, got), 1 - (A & B))


def test_host_entry_point_pipelined_chunks(gpu_ctx, keys):
    """A host batch large enough to be pipelined in chunks (uploads, gates and downloads on
    separate streams) returns exactly what the device entry point returns; sampled rows
    equal the oracle's."""
    count = 4 * 8192 + 5
    (A, B, _), (a, b, _) = _inputs(keys, 280, count)
    out = np.empty_like(a)
    gpu_ctx.lp_gate_batch_host(oracle.AND, a, b, None, out, count)
    dev = empty_dev(count, keys.params.n + 1)
    gpu_ctx.lp_gate_batch(oracle.AND, to_dev(a), to_dev(b), None, dev, count)
    gpu_ctx.lp_sync()
    assert_same(out, to_host(dev), "pipelined host batch vs device batch")
    idx = np.array([0, 8193, 16387, 24581, count - 1])
    assert_same(out[idx], oracle.gate_batch(keys, oracle.AND, a[idx], b[idx]), "pipelined host batch sampled")
