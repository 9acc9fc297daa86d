"""Error behaviour of the C-ABI without a GPU: every entry point that takes a context returns
LP_EINVAL for a null one (the destroy calls, like free, accept it) and leaves a message in
lp_last_error; client and key-file calls reject null pointers the same way.  Nothing throws
or crashes across the ABI.  The calls run in a child process, so a crash fails the test
instead of ending the test session."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, json, sys
sys.path.insert(0, sys.argv[1])
from paper_2407_19871_gb300 import build, locpir
build.build()
L = locpir.lib()
out = {}
for name in locpir.EXPORTS:
    f = getattr(L, name)
    args = f.argtypes or []
    if not args or args[0] is not ctypes.c_void_p:
        continue
    vals = [1 if a in (ctypes.c_int, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_uint64) else None for a in args]
    code = f(*vals)
    out[name] = [int(code), (L.lp_last_error() or b"").decode()]
p = locpir.lp_params()
L.lp_params_default(ctypes.byref(p))
P = ctypes.byref(p)
calls = {
    "lp_client_lwe_encrypt": lambda: L.lp_client_lwe_encrypt(630, None, None, None, None, None, 1, None),
    "lp_client_lwe_phase": lambda: L.lp_client_lwe_phase(630, None, None, None, 1, None),
    "lp_client_keygen_bsk": lambda: L.lp_client_keygen_bsk(P, None, None, None, None, None, None),
    "lp_client_keygen_ksk": lambda: L.lp_client_keygen_ksk(P, None, None, None, None, None, None),
    "lp_preprocess_services": lambda: L.lp_preprocess_services(630, None, None, None, 1, None),
    "lp_save_keys_file": lambda: L.lp_save_keys_file(P, None, None, b"unused.lpk"),
    "lp_verify_keys_file": lambda: L.lp_verify_keys_file(b"", None),
    "lp_create": lambda: L.lp_create(None, 0, None),
    "lp_params_default": lambda: L.lp_params_default(None),
}
for name, call in calls.items():
    code = call()
    out[name] = [int(code), (L.lp_last_error() or b"").decode()]
print(json.dumps(out))
"""


def test_null_arguments_are_rejected_with_a_message():
    from paper_2407_19871_gb300 import locpir
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    ctx_calls = [n for n in locpir.EXPORTS if n in res and n not in (
        "lp_client_lwe_encrypt", "lp_client_lwe_phase", "lp_client_keygen_bsk", "lp_client_keygen_ksk",
        "lp_preprocess_services", "lp_save_keys_file", "lp_verify_keys_file", "lp_create", "lp_params_default")]
    assert len(ctx_calls) >= 30
    for name, (code, msg) in res.items():
        if name in ("lp_destroy", "lp_plan_destroy"):
            assert code == locpir.LP_OK, name                  # like free(NULL)
        elif name == "lp_launch_count":
            assert code == 0, name                             # a counter, not a status
        else:
            assert code == locpir.LP_EINVAL, (name, code)
            assert msg, name
