"""Thin ctypes binding of liblocpir.so (include/locpir.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes pointers and
sizes straight through; all arithmetic runs in the library's CUDA kernels.  Device
ciphertext arguments are torch tensors on the context's CUDA device (int32 or uint32,
contiguous, [count][n + 1]); host arguments of the *_host / key-loading calls are numpy
uint32 arrays.  A missing library raises immediately: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblocpir.so")

LP_OK, LP_EINVAL, LP_ENOMEM, LP_ECUDA, LP_ENOKEY, LP_ETIMEOUT, LP_EBUSY, LP_ECORRUPT = 0, -1, -2, -3, -4, -5, -6, -7
LP_NAND, LP_AND, LP_OR, LP_XOR, LP_XNOR, LP_NOT, LP_MUX = range(7)
LP_LT, LP_LE = 0, 1
LP_XOR_TREE, LP_XOR_CHAIN, LP_OR_TREE = 0, 1, 2

# Every symbol the header declares (checked by the ABI test).
EXPORTS = [
    "lp_params_default", "lp_create", "lp_destroy", "lp_sync", "lp_strerror", "lp_last_error",
    "lp_load_bsk", "lp_load_bsk_device", "lp_load_ksk", "lp_load_ksk_device",
    "lp_gate_batch", "lp_gate_batch_host", "lp_gate_batch_noalloc", "lp_bootstrap_extract", "lp_key_switch",
    "lp_compare_batch", "lp_locpir_query", "lp_locpir_batch", "lp_locpir_batch_waves", "lp_compare_known_batch",
    "lp_locpir_known_batch",
    "lp_client_lwe_encrypt", "lp_client_lwe_phase", "lp_client_keygen_bsk", "lp_client_keygen_ksk",
    "lp_launch_count", "lp_set_timing", "lp_kernel_time", "lp_reset_timing",
    "lp_preprocess_services", "lp_selftest_wait_timeout",
    "lp_server_start", "lp_server_submit", "lp_server_submit_known", "lp_server_poll", "lp_server_wait", "lp_server_stats", "lp_server_stop",
    "lp_save_keys_file", "lp_verify_keys_file", "lp_load_keys_file", "lp_sha256",
    "lp_plan_locpir", "lp_plan_run", "lp_plan_info", "lp_plan_destroy", "lp_set_engines", "lp_autotune",
    "lp_plan_locpir_known", "lp_circuit_info", "lp_autotune_cached", "lp_set_tuning", "lp_get_tuning",
    "lp_set_executor", "lp_selftest_exec_timeout", "lp_selftest_pair_timeout", "lp_selftest_quad_timeout",
]
LP_BR_NTT, LP_BR_TENSOR_BF16, LP_BR_TENSOR_INT8, LP_BR_NTT_BATCHED, LP_BR_NTT_SPLIT, LP_BR_NTT_PAIR, LP_BR_NTT_QUAD = range(7)
LP_KS_TABLE, LP_KS_TENSOR_INT8 = 0, 1
LP_SERVER_QUEUE, LP_SERVER_REJECT = 0, 1
LP_EXEC_LEVELS, LP_EXEC_PERSISTENT = 0, 1


class lp_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("n", "N", "k", "Bgbit", "lg", "basebit", "t")]


class lp_query(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int), ("is_signed", ctypes.c_int), ("n_boxes", ctypes.c_int), ("m", ctypes.c_int),
                ("comb", ctypes.c_int), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("boxes", ctypes.c_void_p),
                ("services", ctypes.c_void_p), ("out_service", ctypes.c_void_p)]


class lp_query_known(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int), ("is_signed", ctypes.c_int), ("n_boxes", ctypes.c_int), ("m", ctypes.c_int),
                ("comb", ctypes.c_int), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("bounds", ctypes.c_void_p),
                ("services", ctypes.c_void_p), ("out_service", ctypes.c_void_p)]


class lp_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "admitted", "completed", "rejected", "waiting", "active",
                                               "ticks", "bootstraps")] + \
               [(k, ctypes.c_double) for k in ("p50_ms", "p99_ms", "mean_ms", "elapsed_s", "queries_per_s",
                                               "bootstraps_per_s")]


class lp_circuit_stats(ctypes.Structure):
    _fields_ = [("gates_by_op", ctypes.c_uint64 * 8)] + \
               [(k, ctypes.c_uint64) for k in ("blind_rotations", "key_switches", "levels", "widest_level", "wires")]


class lp_tuning(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("split_max", "tail_split", "ks_slice_max", "from_cache", "pair_max",
                                            "quad_max")]


class LocpirError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load liblocpir.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2407_19871_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, i, u32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32
        P = ctypes.POINTER(lp_params)
        sig = {
            "lp_params_default": (i, [P]),
            "lp_create": (i, [P, i, ctypes.POINTER(vp)]),
            "lp_destroy": (i, [vp]),
            "lp_sync": (i, [vp]),
            "lp_strerror": (ctypes.c_char_p, [i]),
            "lp_last_error": (ctypes.c_char_p, []),
            "lp_load_bsk": (i, [vp, vp, sz]),
            "lp_load_bsk_device": (i, [vp, vp, sz, vp]),
            "lp_load_ksk": (i, [vp, vp, sz]),
            "lp_load_ksk_device": (i, [vp, vp, sz, vp]),
            "lp_gate_batch": (i, [vp, i, vp, vp, vp, vp, sz, vp]),
            "lp_gate_batch_host": (i, [vp, i, vp, vp, vp, vp, sz]),
            "lp_gate_batch_noalloc": (i, [vp, i, vp, vp, vp, vp, sz, vp]),
            "lp_bootstrap_extract": (i, [vp, vp, u32, vp, sz, vp]),
            "lp_key_switch": (i, [vp, vp, vp, sz, vp]),
            "lp_compare_batch": (i, [vp, i, i, i, vp, vp, vp, sz, vp]),
            "lp_locpir_query": (i, [vp, i, i, vp, vp, i, vp, i, vp, i, vp, vp]),
            "lp_locpir_batch": (i, [vp, ctypes.POINTER(lp_query), sz, vp]),
            "lp_locpir_batch_waves": (i, [vp, ctypes.POINTER(lp_query), sz, sz, ctypes.POINTER(sz), vp]),
            "lp_compare_known_batch": (i, [vp, i, i, i, vp, vp, vp, sz, vp]),
            "lp_locpir_known_batch": (i, [vp, ctypes.POINTER(lp_query_known), sz, vp]),
            "lp_client_lwe_encrypt": (i, [i, vp, vp, vp, vp, vp, sz, vp]),
            "lp_client_lwe_phase": (i, [i, vp, vp, vp, sz, vp]),
            "lp_client_keygen_bsk": (i, [P, vp, vp, vp, vp, vp, vp]),
            "lp_client_keygen_ksk": (i, [P, vp, vp, vp, vp, vp, vp]),
            "lp_launch_count": (ctypes.c_uint64, [vp]),
            "lp_set_timing": (i, [vp, i]),
            "lp_kernel_time": (i, [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_uint64)]),
            "lp_reset_timing": (i, [vp]),
            "lp_preprocess_services": (i, [i, vp, vp, vp, sz, vp]),
            "lp_selftest_wait_timeout": (i, [vp, u32, vp]),
            "lp_server_start": (i, [vp, sz, i]),
            "lp_server_submit": (i, [vp, ctypes.POINTER(lp_query), ctypes.POINTER(ctypes.c_uint64)]),
            "lp_server_submit_known": (i, [vp, ctypes.POINTER(lp_query_known), ctypes.POINTER(ctypes.c_uint64)]),
            "lp_server_poll": (i, [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
            "lp_server_wait": (i, [vp, ctypes.c_uint64, u32]),
            "lp_server_stats": (i, [vp, ctypes.POINTER(lp_stats)]),
            "lp_server_stop": (i, [vp]),
            "lp_save_keys_file": (i, [P, vp, vp, ctypes.c_char_p]),
            "lp_verify_keys_file": (i, [ctypes.c_char_p, P]),
            "lp_load_keys_file": (i, [vp, ctypes.c_char_p]),
            "lp_sha256": (i, [vp, sz, ctypes.c_char_p]),
            "lp_plan_locpir": (i, [vp, ctypes.POINTER(lp_query), sz, ctypes.POINTER(vp)]),
            "lp_plan_locpir_known": (i, [vp, ctypes.POINTER(lp_query_known), sz, ctypes.POINTER(vp)]),
            "lp_plan_run": (i, [vp, vp]),
            "lp_plan_info": (i, [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(ctypes.c_uint64)]),
            "lp_plan_destroy": (i, [vp]),
            "lp_set_engines": (i, [vp, i, i]),
            "lp_autotune": (i, [vp, ctypes.POINTER(ctypes.c_int)]),
            "lp_autotune_cached": (i, [vp, ctypes.c_char_p, i, ctypes.POINTER(lp_tuning)]),
            "lp_set_tuning": (i, [vp, ctypes.POINTER(lp_tuning)]),
            "lp_set_executor": (i, [vp, i]),
            "lp_selftest_exec_timeout": (i, [vp, vp]),
            "lp_selftest_pair_timeout": (i, [vp, vp]),
            "lp_selftest_quad_timeout": (i, [vp, vp]),
            "lp_get_tuning": (i, [vp, ctypes.POINTER(lp_tuning)]),
            "lp_circuit_info": (i, [i, i, i, i, i, vp, ctypes.POINTER(lp_circuit_stats)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int, where: str) -> None:
    if code != LP_OK:
        raise LocpirError(code, where, lib().lp_last_error().decode())


def _dptr(t, words: int | None = None, name: str = "tensor") -> int | None:
    """Device pointer of a contiguous CUDA tensor of 32-bit (or 8-bit key) elements."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if words is not None and t.numel() < words:
        raise ValueError(f"{name} has {t.numel()} elements, the call reads {words}")
    return t.data_ptr()


def _hptr(a: np.ndarray) -> int:
    if not (a.flags["C_CONTIGUOUS"] and a.dtype == np.uint32):
        raise ValueError("host arrays must be C-contiguous uint32")
    return a.ctypes.data


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def params_default() -> lp_params:
    p = lp_params()
    _check(lib().lp_params_default(ctypes.byref(p)), "lp_params_default")
    return p


def lp_circuit_info(l, is_signed, n_boxes, m, comb=LP_XOR_TREE, bounds=None) -> dict:
    """Gate statistics of one LocPIR query's circuit as the library builds and levels it (host
    only).  bounds: None (encrypted bounds) or [n_boxes][4] server-known (X1, X2, Y1, Y2)."""
    st = lp_circuit_stats()
    b = None
    if bounds is not None:
        b = np.ascontiguousarray(np.asarray(bounds, dtype=np.uint64).reshape(n_boxes, 4))
    _check(lib().lp_circuit_info(l, int(is_signed), n_boxes, m, comb, None if b is None else b.ctypes.data,
                                 ctypes.byref(st)), "lp_circuit_info")
    return {"gates_by_op": list(st.gates_by_op), "blind_rotations": st.blind_rotations,
            "key_switches": st.key_switches, "levels": st.levels, "widest_level": st.widest_level,
            "wires": st.wires}


def lp_client_lwe_encrypt(n, s, mask, noise, mu, out, count, stream=None):
    _check(lib().lp_client_lwe_encrypt(n, _dptr(s), _dptr(mask), _dptr(noise), _dptr(mu), _dptr(out), count,
                                       _stream(stream)), "lp_client_lwe_encrypt")


def lp_client_lwe_phase(n, s, ct, phase, count, stream=None):
    _check(lib().lp_client_lwe_phase(n, _dptr(s), _dptr(ct), _dptr(phase), count, _stream(stream)),
           "lp_client_lwe_phase")


def lp_client_keygen_bsk(params, s, S, mask, noise, bsk, stream=None):
    _check(lib().lp_client_keygen_bsk(ctypes.byref(params), _dptr(s), _dptr(S), _dptr(mask), _dptr(noise),
                                      _dptr(bsk), _stream(stream)), "lp_client_keygen_bsk")


def lp_client_keygen_ksk(params, s, S, mask, noise, ksk, stream=None):
    _check(lib().lp_client_keygen_ksk(ctypes.byref(params), _dptr(s), _dptr(S), _dptr(mask), _dptr(noise),
                                      _dptr(ksk), _stream(stream)), "lp_client_keygen_ksk")


def lp_sha256(data: bytes) -> bytes:
    out = ctypes.create_string_buffer(32)
    _check(lib().lp_sha256(data, len(data), out), "lp_sha256")
    return out.raw


def lp_save_keys_file(params: lp_params, bsk: np.ndarray, ksk: np.ndarray, path: str) -> None:
    _check(lib().lp_save_keys_file(ctypes.byref(params), _hptr(bsk), _hptr(ksk), path.encode()), "lp_save_keys_file")


def lp_verify_keys_file(path: str) -> lp_params:
    p = lp_params()
    _check(lib().lp_verify_keys_file(path.encode(), ctypes.byref(p)), "lp_verify_keys_file")
    return p


def lp_preprocess_services(n, zero, bits, out, count, stream=None):
    _check(lib().lp_preprocess_services(n, _dptr(zero), _dptr(bits), _dptr(out), count, _stream(stream)),
           "lp_preprocess_services")


class Plan:
    """An lp_plan (a LocPIR batch captured in a CUDA graph); keeps its query tensors alive."""

    def __init__(self, h, queries):
        self.h = h
        self.queries = queries

    def lp_plan_run(self, stream=None) -> None:
        _check(lib().lp_plan_run(self.h, _stream(stream)), "lp_plan_run")

    def lp_plan_info(self) -> dict:
        a, b, k = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().lp_plan_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(k)), "lp_plan_info")
        return {"blind_rotations": a.value, "key_switches": b.value, "kernels": k.value}

    def lp_plan_destroy(self) -> None:
        if self.h:
            lib().lp_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.lp_plan_destroy()
        except Exception:
            pass


class Context:
    """An lp_ctx: keys and scratch on one device.  Methods mirror the lp_* entry points."""

    def __init__(self, device: int = 0, params: lp_params | None = None):
        self.params = params or params_default()
        h = ctypes.c_void_p()
        _check(lib().lp_create(ctypes.byref(self.params), device, ctypes.byref(h)), "lp_create")
        self.h = h
        self.device = device
        self.n = self.params.n
        self.N = self.params.N

    def close(self) -> None:
        if self.h:
            lib().lp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- keys
    def lp_load_bsk(self, bsk: np.ndarray) -> None:
        _check(lib().lp_load_bsk(self.h, _hptr(bsk), bsk.size), "lp_load_bsk")

    def lp_load_ksk(self, ksk: np.ndarray) -> None:
        _check(lib().lp_load_ksk(self.h, _hptr(ksk), ksk.size), "lp_load_ksk")

    def lp_load_bsk_device(self, bsk, stream=None) -> None:
        _check(lib().lp_load_bsk_device(self.h, _dptr(bsk), bsk.numel(), _stream(stream)), "lp_load_bsk_device")

    def lp_load_keys_file(self, path: str) -> None:
        _check(lib().lp_load_keys_file(self.h, path.encode()), "lp_load_keys_file")

    def lp_load_ksk_device(self, ksk, stream=None) -> None:
        _check(lib().lp_load_ksk_device(self.h, _dptr(ksk), ksk.numel(), _stream(stream)), "lp_load_ksk_device")

    # ---- bootstrapping
    def lp_gate_batch(self, op: int, a, b, c, out, count: int, stream=None) -> None:
        W = count * (self.n + 1)
        _check(lib().lp_gate_batch(self.h, op, _dptr(a, W, "a"), _dptr(b, W, "b") if b is not None else None,
                                   _dptr(c, W, "c") if c is not None else None, _dptr(out, W, "out"), count,
                                   _stream(stream)), "lp_gate_batch")

    def lp_gate_batch_host(self, op: int, a: np.ndarray, b, c, out: np.ndarray, count: int) -> None:
        _check(lib().lp_gate_batch_host(self.h, op, _hptr(a), _hptr(b) if b is not None else None,
                                        _hptr(c) if c is not None else None, _hptr(out), count),
               "lp_gate_batch_host")

    def lp_gate_batch_noalloc(self, op: int, a, b, c, out, count: int, stream=None) -> None:
        """lp_gate_batch without device allocation: scratch in the library's fixed array
        (at most 256 blind rotations per call)."""
        W = count * (self.n + 1)
        _check(lib().lp_gate_batch_noalloc(self.h, op, _dptr(a, W, "a"), _dptr(b, W, "b") if b is not None else None,
                                           _dptr(c, W, "c") if c is not None else None, _dptr(out, W, "out"), count,
                                           _stream(stream)), "lp_gate_batch_noalloc")

    def lp_bootstrap_extract(self, lwe, mu: int, ext, count: int, stream=None) -> None:
        _check(lib().lp_bootstrap_extract(self.h, _dptr(lwe, count * (self.n + 1), "lwe"), mu & 0xFFFFFFFF,
                                          _dptr(ext, count * (self.N + 1), "ext"), count, _stream(stream)),
               "lp_bootstrap_extract")

    def lp_key_switch(self, ext, out, count: int, stream=None) -> None:
        _check(lib().lp_key_switch(self.h, _dptr(ext, count * (self.N + 1), "ext"),
                                   _dptr(out, count * (self.n + 1), "out"), count, _stream(stream)), "lp_key_switch")

    # ---- circuits
    def lp_compare_batch(self, kind: int, is_signed: int, l: int, x1, x2, out, count: int, stream=None) -> None:
        W = self.n + 1
        _check(lib().lp_compare_batch(self.h, kind, is_signed, l, _dptr(x1, count * l * W, "x1"),
                                      _dptr(x2, count * l * W, "x2"), _dptr(out, count * W, "out"), count,
                                      _stream(stream)), "lp_compare_batch")

    def lp_locpir_query(self, l, is_signed, x, y, n_boxes, boxes, m, services, comb, out_service, stream=None):
        W = self.n + 1
        _check(lib().lp_locpir_query(self.h, l, is_signed, _dptr(x, l * W, "x"), _dptr(y, l * W, "y"), n_boxes,
                                     _dptr(boxes, n_boxes * 4 * l * W, "boxes"), m,
                                     _dptr(services, n_boxes * m * W, "services"), comb,
                                     _dptr(out_service, m * W, "out_service"), _stream(stream)), "lp_locpir_query")

    def _query_struct(self, q: dict) -> lp_query:
        W = self.n + 1
        l, nb, m = q["l"], q["n_boxes"], q["m"]
        return lp_query(l, q.get("is_signed", 0), nb, m, q.get("comb", LP_XOR_TREE),
                        _dptr(q["x"], l * W, "x"), _dptr(q["y"], l * W, "y"),
                        _dptr(q["boxes"], nb * 4 * l * W, "boxes"), _dptr(q["services"], nb * m * W, "services"),
                        _dptr(q["out_service"], m * W, "out_service"))

    def lp_locpir_batch(self, queries: list[dict], stream=None) -> None:
        """queries: dicts with l, is_signed, n_boxes, m, comb and tensors x, y, boxes,
        services, out_service (shapes as in lp_locpir_query)."""
        arr = (lp_query * len(queries))()
        for i, q in enumerate(queries):
            arr[i] = self._query_struct(q)
        _check(lib().lp_locpir_batch(self.h, arr, len(queries), _stream(stream)), "lp_locpir_batch")

    def lp_locpir_batch_waves(self, queries: list[dict], mem_budget: int, stream=None) -> int:
        """As lp_locpir_batch, in waves whose circuits fit mem_budget bytes; returns the number
        of waves."""
        arr = (lp_query * len(queries))()
        for i, q in enumerate(queries):
            arr[i] = self._query_struct(q)
        waves = ctypes.c_size_t()
        _check(lib().lp_locpir_batch_waves(self.h, arr, len(queries), int(mem_budget), ctypes.byref(waves),
                                           _stream(stream)), "lp_locpir_batch_waves")
        return waves.value

    # ---- alternative product engines
    def lp_set_engines(self, br_engine: int = LP_BR_NTT, ks_engine: int = LP_KS_TABLE) -> None:
        _check(lib().lp_set_engines(self.h, br_engine, ks_engine), "lp_set_engines")

    def lp_autotune(self) -> int:
        """Measure the split/batched blind-rotation crossing on this GPU; returns the widest
        level (ciphertexts) the default engine now runs split."""
        v = ctypes.c_int()
        _check(lib().lp_autotune(self.h, ctypes.byref(v)), "lp_autotune")
        return v.value

    def lp_autotune_cached(self, cache_path=None, force: bool = False) -> dict:
        """Measure (or read from the JSON cache file) the launch policy and apply it; returns it."""
        t = lp_tuning()
        path = None if cache_path is None else os.fsencode(cache_path)
        _check(lib().lp_autotune_cached(self.h, path, int(force), ctypes.byref(t)), "lp_autotune_cached")
        return {k: getattr(t, k) for k, _ in lp_tuning._fields_}

    def lp_set_tuning(self, split_max: int = 0, tail_split: int = 0, ks_slice_max: int = 0, pair_max: int = 0,
                      quad_max: int = 0) -> None:
        t = lp_tuning(split_max, tail_split, ks_slice_max, 0, pair_max, quad_max)
        _check(lib().lp_set_tuning(self.h, ctypes.byref(t)), "lp_set_tuning")

    def lp_selftest_exec_timeout(self, stream=None) -> None:
        _check(lib().lp_selftest_exec_timeout(self.h, _stream(stream)), "lp_selftest_exec_timeout")

    def lp_selftest_pair_timeout(self, stream=None) -> None:
        _check(lib().lp_selftest_pair_timeout(self.h, _stream(stream)), "lp_selftest_pair_timeout")

    def lp_selftest_quad_timeout(self, stream=None) -> None:
        _check(lib().lp_selftest_quad_timeout(self.h, _stream(stream)), "lp_selftest_quad_timeout")

    def lp_set_executor(self, executor: int) -> None:
        _check(lib().lp_set_executor(self.h, executor), "lp_set_executor")

    def lp_get_tuning(self) -> dict:
        t = lp_tuning()
        _check(lib().lp_get_tuning(self.h, ctypes.byref(t)), "lp_get_tuning")
        return {k: getattr(t, k) for k, _ in lp_tuning._fields_ if k != "from_cache"}

    # ---- server-known bounds (beyond the paper)
    def lp_compare_known_batch(self, kind: int, is_signed: int, l: int, x, k, out, count: int, stream=None) -> None:
        """x: device ciphertexts [count][l][n+1]; k: plaintext bounds (sequence of count ints)."""
        W = self.n + 1
        kb = np.ascontiguousarray(np.asarray(k, dtype=np.uint64).reshape(-1))
        if kb.size < count:
            raise ValueError(f"k has {kb.size} bounds, the call reads {count}")
        _check(lib().lp_compare_known_batch(self.h, kind, is_signed, l, _dptr(x, count * l * W, "x"),
                                            kb.ctypes.data, _dptr(out, count * W, "out"), count, _stream(stream)),
               "lp_compare_known_batch")

    def _query_known_struct(self, q: dict):
        """(lp_query_known, bounds array to keep alive) for a known-bounds query dict."""
        W = self.n + 1
        l, nb, m = q["l"], q["n_boxes"], q["m"]
        b = np.ascontiguousarray(np.asarray(q["bounds"], dtype=np.uint64).reshape(-1))
        if b.size < 4 * nb:
            raise ValueError(f"bounds has {b.size} values, the query reads {4 * nb}")
        return lp_query_known(l, q.get("is_signed", 0), nb, m, q.get("comb", LP_XOR_TREE),
                              _dptr(q["x"], l * W, "x"), _dptr(q["y"], l * W, "y"), b.ctypes.data,
                              _dptr(q["services"], nb * m * W, "services"),
                              _dptr(q["out_service"], m * W, "out_service")), b

    def lp_locpir_known_batch(self, queries: list[dict], stream=None) -> None:
        """queries: dicts with l, is_signed, n_boxes, m, comb, bounds ([n_boxes][4] ints
        X1, X2, Y1, Y2) and tensors x, y, services, out_service."""
        arr = (lp_query_known * len(queries))()
        keep = []
        for i, q in enumerate(queries):
            arr[i], b = self._query_known_struct(q)
            keep.append(b)
        _check(lib().lp_locpir_known_batch(self.h, arr, len(queries), _stream(stream)), "lp_locpir_known_batch")

    # ---- plans (CUDA graphs)
    def lp_plan_locpir_known(self, queries: list[dict]) -> "Plan":
        arr = (lp_query_known * len(queries))()
        keep = []
        for i, q in enumerate(queries):
            arr[i], b = self._query_known_struct(q)
            keep.append(b)
        h = ctypes.c_void_p()
        _check(lib().lp_plan_locpir_known(self.h, arr, len(queries), ctypes.byref(h)), "lp_plan_locpir_known")
        return Plan(h, queries)

    def lp_plan_locpir(self, queries: list[dict]) -> "Plan":
        arr = (lp_query * len(queries))()
        for i, q in enumerate(queries):
            arr[i] = self._query_struct(q)
        h = ctypes.c_void_p()
        _check(lib().lp_plan_locpir(self.h, arr, len(queries), ctypes.byref(h)), "lp_plan_locpir")
        return Plan(h, queries)

    # ---- server (continuous batching)
    def lp_server_start(self, mem_budget: int, policy: int = LP_SERVER_QUEUE) -> None:
        self._server_refs = {}
        _check(lib().lp_server_start(self.h, mem_budget, policy), "lp_server_start")

    def lp_server_submit(self, q: dict) -> int:
        """Submit a query dict (as in lp_locpir_batch); its tensors are kept referenced here
        until lp_server_stop, since the server reads them asynchronously."""
        t = ctypes.c_uint64()
        qs = self._query_struct(q)
        _check(lib().lp_server_submit(self.h, ctypes.byref(qs), ctypes.byref(t)), "lp_server_submit")
        self._server_refs[t.value] = q
        return t.value

    def lp_server_submit_known(self, q: dict) -> int:
        """Submit a known-bounds query dict (as in lp_locpir_known_batch); its bounds are copied
        by the call, its tensors are kept referenced until lp_server_stop."""
        t = ctypes.c_uint64()
        qs, _ = self._query_known_struct(q)
        _check(lib().lp_server_submit_known(self.h, ctypes.byref(qs), ctypes.byref(t)), "lp_server_submit_known")
        self._server_refs[t.value] = q
        return t.value

    def lp_server_poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(lib().lp_server_poll(self.h, ticket, ctypes.byref(d)), "lp_server_poll")
        return bool(d.value)

    def lp_server_wait(self, ticket: int, timeout_ms: int = 600000) -> None:
        _check(lib().lp_server_wait(self.h, ticket, timeout_ms), "lp_server_wait")

    def lp_server_stats(self) -> dict:
        st = lp_stats()
        _check(lib().lp_server_stats(self.h, ctypes.byref(st)), "lp_server_stats")
        return {k: getattr(st, k) for k, _ in lp_stats._fields_}

    def lp_server_stop(self) -> None:
        try:
            _check(lib().lp_server_stop(self.h), "lp_server_stop")
        finally:
            self._server_refs = {}

    # ---- runtime
    def lp_sync(self) -> None:
        _check(lib().lp_sync(self.h), "lp_sync")

    def lp_launch_count(self) -> int:
        return int(lib().lp_launch_count(self.h))

    def lp_set_timing(self, enable: bool) -> None:
        _check(lib().lp_set_timing(self.h, int(bool(enable))), "lp_set_timing")

    def lp_kernel_time(self, kernel: str) -> tuple[float, int]:
        ms, cnt = ctypes.c_double(), ctypes.c_uint64()
        _check(lib().lp_kernel_time(self.h, kernel.encode(), ctypes.byref(ms), ctypes.byref(cnt)), "lp_kernel_time")
        return ms.value, cnt.value

    def lp_reset_timing(self) -> None:
        _check(lib().lp_reset_timing(self.h), "lp_reset_timing")

    def lp_selftest_wait_timeout(self, limit_ms: int, stream=None) -> None:
        _check(lib().lp_selftest_wait_timeout(self.h, limit_ms, _stream(stream)), "lp_selftest_wait_timeout")
