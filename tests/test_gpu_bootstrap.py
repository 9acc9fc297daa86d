"""Parity of the CUDA bootstrap pieces with the oracle, through the C-ABI.

Bit-exact: every output word of the blind rotation + extraction and of the key
switch equals the oracle's on the same keys and inputs."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu

EIGHTH = 1 << 29


def _random_lwes(seed, count, n):
    return synth.uniform_u32(seed, 900, count * (n + 1)).reshape(count, n + 1)


@pytest.mark.parametrize("count", [1, 7])
def test_bootstrap_extract_matches_oracle(gpu_ctx, keys, count):
    """count = 7: one full group of 4 ciphertexts and a ragged group of 3."""
    p = keys.params
    lwe = _random_lwes(101 + count, count, p.n)
    ext = empty_dev(count, p.N + 1)
    gpu_ctx.lp_bootstrap_extract(to_dev(lwe), EIGHTH, ext, count)
    gpu_ctx.lp_sync()
    assert_same(to_host(ext), oracle.bootstrap_extract(keys, lwe), "bootstrap_extract")


def test_bootstrap_closed_form_trivial_keys(gpu_ctx_trivial, keys_trivial):
    """Under trivial keys the extracted sample is (0, +-1/8), sign by the switched phase."""
    p = keys_trivial.params
    cnt = 9
    lwe = _random_lwes(7, cnt, p.n)
    ext = empty_dev(cnt, p.N + 1)
    gpu_ctx_trivial.lp_bootstrap_extract(to_dev(lwe), EIGHTH, ext, cnt)
    gpu_ctx_trivial.lp_sync()
    got = to_host(ext)
    s = keys_trivial.s.astype(np.int64)
    for g in range(cnt):
        bar = ((lwe[g].astype(np.int64) + (1 << 20)) % (1 << 32)) >> 21
        phi = int(bar[p.n] - (bar[:p.n] * s).sum()) % (2 * p.N)
        assert not got[g, :p.N].any()
        # coefficient 0 of X^-phi v: +v for phi in [0, N), -v otherwise
        assert got[g, p.N] == (EIGHTH if phi < p.N else (1 << 32) - EIGHTH)


@pytest.mark.parametrize("count", [1, 17, 40])
def test_key_switch_matches_oracle(gpu_ctx, keys, count):
    """17 = one full tile of 16 outputs and a ragged tail; 40 spans three tiles."""
    p = keys.params
    ext = synth.uniform_u32(55 + count, 901, count * (p.N + 1)).reshape(count, p.N + 1)
    out = empty_dev(count, p.n + 1)
    gpu_ctx.lp_key_switch(to_dev(ext), out, count)
    gpu_ctx.lp_sync()
    want = np.stack([oracle.key_switch(p, keys.ksk, ext[g]) for g in range(count)])
    assert_same(to_host(out), want, "key_switch")


def test_bootstrap_test_vector_value(gpu_ctx, keys):
    """mu is the test-vector value: a bootstrap with mu = 1/4 equals the oracle's too."""
    p = keys.params
    lwe = _random_lwes(8, 2, p.n)
    ext = empty_dev(2, p.N + 1)
    gpu_ctx.lp_bootstrap_extract(to_dev(lwe), 1 << 30, ext, 2)
    gpu_ctx.lp_sync()
    assert_same(to_host(ext), oracle.bootstrap_extract(keys, lwe, mu=1 << 30), "mu=1/4")


def test_zero_count_is_noop(gpu_ctx, keys):
    p = keys.params
    t = empty_dev(1, p.n + 1)
    gpu_ctx.lp_gate_batch(0, t, t, None, t, 0)
    gpu_ctx.lp_bootstrap_extract(t, EIGHTH, empty_dev(1, p.N + 1), 0)
    gpu_ctx.lp_sync()


# ---------------------------------------------------------------------------------------
# The edge of the product engine's exactness (tests/crt_edge.py): key words at -2^31 and
# body digits at -512 drive the first external product to 3 * 2^50 ~ 2^51.6 (random inputs
# reach ~2^46), near the 2^52.6 bound the centred two-prime CRT must cover.  TFHE's external
# product (J. Cryptology 2020), to which the paper's EvalGate (Section 2.2) defers.
# ---------------------------------------------------------------------------------------
@pytest.fixture(scope="module", params=[0, 24], ids=["key-0x80000000", "key-low-bits-24"])
def edge_case(request):
    from crt_edge import crafted_bsk
    from paper_2407_19871_gb300 import build
    from paper_2407_19871_gb300.locpir import Context
    p = synth.DEFAULT
    bsk = crafted_bsk(p, low_bits=request.param, seed=17)
    keys = oracle.Keys(p, np.zeros(p.n, np.uint8), np.zeros(p.N, np.uint8), bsk, np.zeros(1, np.uint32))
    build.build()
    ctx = Context(0)
    ctx.lp_load_bsk(np.ascontiguousarray(bsk.reshape(-1)))
    yield ctx, keys
    ctx.close()


@pytest.mark.parametrize("engine", ["batched", "split", "pair", "quad"])
@pytest.mark.parametrize("count", [1, 7])
def test_bootstrap_at_the_crt_edge_matches_oracle(edge_case, engine, count):
    """count = 7: one full group of 4 and a ragged group of 3 on the batched kernel; sample 0
    has one edge step, sample 1 all 630, the others a random subset."""
    from crt_edge import MU_EDGE, crafted_lwes
    from paper_2407_19871_gb300.locpir import (LP_BR_NTT, LP_BR_NTT_BATCHED, LP_BR_NTT_PAIR, LP_BR_NTT_QUAD,
                                               LP_BR_NTT_SPLIT)
    ctx, keys = edge_case
    p = keys.params
    lwe = crafted_lwes(p, count, seed=40 + count)
    ctx.lp_set_engines({"batched": LP_BR_NTT_BATCHED, "split": LP_BR_NTT_SPLIT, "pair": LP_BR_NTT_PAIR,
                        "quad": LP_BR_NTT_QUAD}[engine], 0)
    try:
        ext = empty_dev(count, p.N + 1)
        ctx.lp_bootstrap_extract(to_dev(lwe), MU_EDGE, ext, count)
        ctx.lp_sync()
    finally:
        ctx.lp_set_engines(LP_BR_NTT, 0)
    assert_same(to_host(ext), oracle.bootstrap_extract(keys, lwe, mu=MU_EDGE), f"edge {engine} x{count}")
