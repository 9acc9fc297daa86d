"""Device-side client helpers (key generation, Encrypt, phase) equal the oracle's on
the same random draws."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_device_keygen_matches_oracle(keys):
    import torch
    from paper_2407_19871_gb300 import build, locpir
    build.build()
    d = synth.key_draws(0)
    p = locpir.params_default()
    bsk = empty_dev(p.n, 6, 2, p.N)
    locpir.lp_client_keygen_bsk(p, to_dev(d.s), to_dev(d.S), to_dev(d.bsk_mask), to_dev(d.bsk_noise), bsk)
    ksk = empty_dev(p.N, p.t, 4, p.n + 1)
    locpir.lp_client_keygen_ksk(p, to_dev(d.s), to_dev(d.S), to_dev(d.ksk_mask), to_dev(d.ksk_noise), ksk)
    torch.cuda.synchronize()
    assert_same(to_host(bsk), keys.bsk, "bsk")
    assert_same(to_host(ksk), keys.ksk, "ksk")


def test_device_encrypt_and_phase_match_oracle(keys):
    import torch
    from paper_2407_19871_gb300 import build, locpir
    build.build()
    n, cnt = keys.params.n, 37
    bits = synth.bits(5, 9, cnt)
    dr = synth.lwe_draws(5, cnt)
    mu = oracle.encode(bits)
    out = empty_dev(cnt, n + 1)
    locpir.lp_client_lwe_encrypt(n, to_dev(keys.s), to_dev(dr.mask), to_dev(dr.noise), to_dev(mu), out, cnt)
    ph = empty_dev(cnt)
    locpir.lp_client_lwe_phase(n, to_dev(keys.s), out, ph, cnt)
    torch.cuda.synchronize()
    want = oracle.encrypt(keys.s, bits, dr)
    assert_same(to_host(out), want, "encrypt")
    assert_same(to_host(ph), oracle.phase(keys.s, want), "phase")
