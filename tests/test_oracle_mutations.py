"""The pins catch plausible slips: each mutation below plants one mistake in a copy of the
oracle's C source (on the CPU), and the quick pin tests run against that build must fail,
while the same tests against an unmodified build of the copy pass.

The mistakes are the kinds a reader checking the oracle against the paper and TFHE would look
for: a sign in the sample extraction, the rounding of the gadget decomposition, of the modulus
switch and of the key-switch digits, the direction of the rotation, a gate constant, the MUX
post-sum constant and the placement of the gadget in the TRGSW rows."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tfhe_oracle.c")
PINS = ["tests/test_oracle_decomp.py", "tests/test_oracle_bootstrap.py", "tests/test_oracle_keys.py"]

MUTATIONS = {
    "extraction sign": ("out[j] = 0u - acc[N - j];", "out[j] = acc[N - j];"),
    "gadget rounding": ("if (Bgbit * lg < 32) off += 1u << (31 - Bgbit * lg);", ""),
    "modulus-switch rounding": ("return (x + (1u << (shift - 1))) >> shift;", "return x >> shift;"),
    "rotation direction": ("or_poly_mul_monomial(N, acc + c * N, ab, rot);",
                           "or_poly_mul_monomial(N, acc + c * N, 2 * N - ab, rot);"),
    "key-switch rounding": ("uint32_t y = x + prec;", "uint32_t y = x;"),
    "XNOR constant": ("case OR_XNOR: *cst = 0u - T_QUARTER;", "case OR_XNOR: *cst = T_QUARTER;"),
    "MUX post-sum constant": ("sum[N] += T_EIGHTH;", "sum[N] -= T_EIGHTH;"),
    "TRGSW row placement": ("if (c == 0) out_a[0] += g;", "if (c == 1) out_a[0] += g;"),
}


def _build(src_text: str, path: str) -> None:
    c_path = path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", path, c_path])


def test_every_planted_mistake_fails_a_pin(tmp_path):
    text = open(SRC).read()
    libs = {"control": str(tmp_path / "control.so")}
    _build(text, libs["control"])
    for k, (name, (orig, mutated)) in enumerate(MUTATIONS.items()):
        assert text.count(orig) == 1, f"mutation site of {name!r} not found exactly once"
        libs[name] = str(tmp_path / f"m{k}.so")
        _build(text.replace(orig, mutated), libs[name])
    procs = {}
    for name, so in libs.items():
        env = dict(os.environ, ORACLE_LIB=so, OMP_NUM_THREADS="2")
        cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not slow and not gpu"] + PINS
        procs[name] = subprocess.Popen(cmd, cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    out = {name: (p.communicate()[0], p.returncode) for name, p in procs.items()}
    log, rc = out.pop("control")
    assert rc == 0, f"the pins fail on an unmodified copy of the oracle:\n{log[-2000:]}"
    for name, (log, rc) in out.items():
        # exit code 1: tests ran and at least one failed (not a collection or usage error)
        assert rc == 1, f"no pin caught the planted {name!r} mistake (pytest exit {rc}):\n{log[-1500:]}"
