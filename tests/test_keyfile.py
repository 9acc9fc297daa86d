"""Key files and their SHA-256 checksum (host only, no GPU)."""
import hashlib
import os

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def lp():
    from paper_2407_19871_gb300 import build, locpir
    build.build()
    return locpir


@pytest.mark.parametrize("size", [0, 1, 55, 56, 63, 64, 65, 1000, 4096 + 7])
def test_sha256_matches_hashlib(lp, size):
    data = bytes((synth.uniform_u32(3, size, max(size, 1)) & 0xFF).astype(np.uint8))[:size]
    assert lp.lp_sha256(data) == hashlib.sha256(data).digest()


def test_key_file_round_trip_and_corruption(lp, tmp_path, keys):
    p = lp.params_default()
    bsk = np.ascontiguousarray(keys.bsk.reshape(-1))
    ksk = np.ascontiguousarray(keys.ksk.reshape(-1))
    path = str(tmp_path / "keys.lpk")
    lp.lp_save_keys_file(p, bsk, ksk, path)
    q = lp.lp_verify_keys_file(path)
    assert (q.n, q.N, q.lg, q.t) == (630, 1024, 3, 8)
    raw = open(path, "rb").read()
    assert raw[:8] == b"LPKEYS01"
    hdr = 8 + 4 + 7 * 4 + 8 + 8
    assert raw[hdr:hdr + 32] == hashlib.sha256(bsk.tobytes() + ksk.tobytes()).digest()
    # flip one bit of the key-switching key: the checksum catches it
    bad = bytearray(raw)
    bad[-5] ^= 0x10
    bad_path = str(tmp_path / "bad.lpk")
    open(bad_path, "wb").write(bytes(bad))
    with pytest.raises(lp.LocpirError) as e:
        lp.lp_verify_keys_file(bad_path)
    assert e.value.code == lp.LP_ECORRUPT
    # a truncated file too
    open(bad_path, "wb").write(raw[:-100])
    with pytest.raises(lp.LocpirError) as e:
        lp.lp_verify_keys_file(bad_path)
    assert e.value.code == lp.LP_ECORRUPT
