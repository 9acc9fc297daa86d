import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for _p in (ROOT, os.path.dirname(os.path.abspath(__file__))):
    if _p not in sys.path:
        sys.path.insert(0, _p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (parity tests through the C-ABI)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture(scope="session")
def params():
    import synth
    return synth.DEFAULT


@pytest.fixture(scope="session")
def keys():
    """Keys of the parameter set n=630, N=1024, Bgbit=10, lg=3, basebit=2, t=8 from seed 0."""
    import oracle
    import synth
    return oracle.keygen(synth.key_draws(0))


@pytest.fixture(scope="session")
def keys_noiseless():
    """Random masks, zero noise: bootstraps decide every gate correctly."""
    import oracle
    import synth
    return oracle.keygen(synth.key_draws(7, noiseless=True))


@pytest.fixture(scope="session")
def keys_trivial():
    """Zero masks and zero noise: the bootstrap has the closed form (0, X^-phi v)."""
    import oracle
    import synth
    return oracle.keygen(synth.key_draws(11, noiseless=True, zero_masks=True))


@pytest.fixture(scope="session")
def gpu_ctx(keys):
    """Library context on cuda:0 with the seed-0 keys (generated by the oracle) loaded."""
    from gpu_util import make_context
    ctx = make_context(keys)
    yield ctx
    ctx.close()


@pytest.fixture(scope="session")
def gpu_ctx_trivial(keys_trivial):
    from gpu_util import make_context
    ctx = make_context(keys_trivial)
    yield ctx
    ctx.close()
