"""ctypes binding of libhelrm.so (argument marshalling only).

Every function mirrors the C entry point of the same name in include/helrm.h;
all computation runs in the CUDA library.  Handles are wrapped in objects that
release themselves (helrm_free) when garbage-collected, and keep their context
alive.  A non-OK status raises HelrmError with the library's message.  If the
shared library has not been built the import of any function raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhelrm.so")

STATUS = {0: "HELRM_OK", -1: "HELRM_E_INVAL", -2: "HELRM_E_PARAM", -3: "HELRM_E_LEVEL",
          -4: "HELRM_E_SCALE", -5: "HELRM_E_NOKEY", -6: "HELRM_E_NOMEM", -7: "HELRM_E_CUDA",
          -8: "HELRM_E_TIMEOUT"}


class HelrmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Params(C.Structure):
    _fields_ = [("log_n", C.c_uint32), ("n_q", C.c_uint32), ("q_bits", C.POINTER(C.c_uint32)),
                ("n_p", C.c_uint32), ("p_bits", C.c_uint32), ("alpha", C.c_uint32),
                ("log2_scale", C.c_double)]


class BootDesc(C.Structure):
    _fields_ = [("n_s", C.c_uint32), ("K", C.c_uint32), ("r", C.c_uint32), ("degree", C.c_uint32),
                ("log2_boost", C.c_uint32), ("cts_levels", C.c_uint32), ("s_ref", C.c_double),
                ("eval_scale", C.c_double), ("coeffs", C.POINTER(C.c_double))]


class ServeStats(C.Structure):
    _fields_ = [("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_ms", C.c_double),
                ("makespan_s", C.c_double), ("throughput", C.c_double), ("n_batches", C.c_uint32),
                ("max_batch", C.c_uint32), ("max_inflight", C.c_uint32), ("mean_batch", C.c_double)]


class ModelDesc(C.Structure):
    _fields_ = [("n_dense", C.c_uint32), ("n_bottom", C.c_uint32),
                ("bottom_widths", C.POINTER(C.c_uint32)),
                ("bottom_W", C.POINTER(C.POINTER(C.c_double))), ("bottom_b", C.POINTER(C.POINTER(C.c_double))),
                ("n_top", C.c_uint32), ("top_widths", C.POINTER(C.c_uint32)),
                ("top_W", C.POINTER(C.POINTER(C.c_double))), ("top_b", C.POINTER(C.POINTER(C.c_double))),
                ("n_tables", C.c_uint32), ("cards", C.POINTER(C.c_uint64)), ("base_p", C.c_uint32),
                ("dim", C.c_uint32), ("tables", C.POINTER(C.POINTER(C.c_float))),
                ("interaction", C.c_int32), ("threshold", C.c_uint64),
                ("act_degree", C.c_uint32), ("act_coeffs", C.POINTER(C.c_double)),
                ("boot_bottom", C.c_uint32), ("boot_z", C.c_uint32), ("boot_top", C.c_uint32),
                ("boot_coeffs", C.POINTER(C.c_double))]


_lib = None
_vp = C.c_void_p
_pp = C.POINTER(C.c_void_p)
_u64p = C.POINTER(C.c_uint64)
_i64p = C.POINTER(C.c_int64)
_u32p = C.POINTER(C.c_uint32)
_i32p = C.POINTER(C.c_int32)
_dp = C.POINTER(C.c_double)

_SIGS = {
    "helrm_ctx_create": [C.POINTER(Params), C.c_int, _vp, _pp],
    "helrm_ctx_primes": [_vp, _u64p, _u64p],
    "helrm_ctx_dims": [_vp, _u32p],
    "helrm_ctx_set_memory_cap": [_vp, C.c_uint64],
    "helrm_ctx_memory_in_use": [_vp, _u64p],
    "helrm_ctx_synchronize": [_vp],
    "helrm_ctx_launch_count": [_vp, _u64p],
    "helrm_ntt": [_vp, _vp, C.c_uint32, C.c_uint32, C.c_int],
    "helrm_alu_peak": [_vp, C.c_int32, C.c_uint32, C.c_uint32, _dp],
    "helrm_keygen": [_vp, C.c_uint64, _i32p, C.c_uint32, _pp, _pp],
    "helrm_evk_add_rotations": [_vp, _vp, _vp, _i32p, C.c_uint32],
    "helrm_model_keygen": [_vp, _vp, C.c_uint64, _pp, _pp],
    "helrm_evk_bytes": [_vp, _u64p],
    "helrm_encode": [_vp, _dp, C.c_uint32, C.c_int32, C.c_double, _pp],
    "helrm_pt_import": [_vp, _i64p, C.c_int32, C.c_double, _pp],
    "helrm_pt_export": [_vp, _vp, _i64p],
    "helrm_encrypt": [_vp, _vp, _vp, C.c_uint64, _pp],
    "helrm_decrypt": [_vp, _vp, _vp, _dp, C.c_uint32],
    "helrm_ct_export": [_vp, _vp, _u64p, _i32p, _dp],
    "helrm_ct_import": [_vp, _u64p, C.c_int32, C.c_double, _pp],
    "helrm_ct_info": [_vp, _i32p, _dp],
    "helrm_add": [_vp, _vp, _vp, _pp],
    "helrm_sub": [_vp, _vp, _vp, _pp],
    "helrm_add_pt": [_vp, _vp, _vp, _pp],
    "helrm_mul_pt": [_vp, _vp, _vp, _pp],
    "helrm_mul": [_vp, _vp, _vp, _vp, _pp],
    "helrm_rescale": [_vp, _vp, _pp],
    "helrm_drop_level": [_vp, _vp, C.c_int32, _pp],
    "helrm_rotate": [_vp, _vp, _vp, C.c_int32, _pp],
    "helrm_rotate_hoisted": [_vp, _vp, _vp, _i32p, C.c_uint32, _pp],
    "helrm_ptmat_prepare": [_vp, _dp, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int32,
                            C.c_double, C.c_double, _pp],
    "helrm_ptmat_info": [_vp, _u32p],
    "helrm_ptmat_rotations": [_vp, _i32p, _u32p],
    "helrm_ptmat_import": [_vp, _vp, _i64p, C.c_uint32],
    "helrm_ptct_matvec": [_vp, _vp, _vp, _vp, C.c_uint32, _pp],
    "helrm_emb_prepare": [_vp, C.c_uint32, _u64p, C.c_uint32, C.c_uint64, C.c_uint32, C.POINTER(C.POINTER(C.c_float)),
                          C.c_uint32, C.c_uint32, C.c_int32, C.c_double, C.c_double, _pp],
    "helrm_query_pack": [_vp, _u64p, _dp, C.c_uint32],
    "helrm_emb_info": [_vp, _u32p, _u32p],
    "helrm_embedding_lookup": [_vp, _vp, _vp, _vp, C.c_uint32, _pp],
    "helrm_emb_chunks": [_vp, _u32p],
    "helrm_emb_matrix": [_vp, C.c_uint32, _pp],
    "helrm_embedding_lookup_multi": [_vp, _vp, _vp, _pp, C.c_uint32, _pp],
    "helrm_model_create": [_vp, C.POINTER(ModelDesc), _pp],
    "helrm_model_info": [_vp, _u32p],
    "helrm_model_rotations": [_vp, _i32p, _u32p],
    "helrm_model_import_plaintexts": [_vp, _vp, _i64p, C.c_uint32],
    "helrm_model_export_plaintexts": [_vp, _vp, _i64p, C.c_uint32],
    "helrm_encrypt_query": [_vp, _vp, _vp, _dp, _u64p, C.c_uint64, _pp, _pp],
    "helrm_infer": [_vp, _vp, _vp, _vp, _vp, _pp],
    "helrm_infer_multi": [_vp, _vp, _vp, _vp, _pp, C.c_uint32, _pp],
    "helrm_decrypt_logit": [_vp, _vp, _vp, _dp, _dp],
    "helrm_infer_e2e": [_vp, _vp, _vp, _vp, _dp, _u64p, C.c_uint32, C.c_uint64, _dp, _dp],
    "helrm_infer_e2e_device": [_vp, _vp, _vp, _vp, _vp, _vp, C.c_uint32, C.c_uint64, _vp, _vp],
    "helrm_rescale_noalloc": [_vp, _vp, _vp, C.c_int32, C.c_uint32],
    "helrm_poly_eval": [_vp, _vp, _vp, _dp, C.c_uint32, C.c_double, _pp],
    "helrm_batch_create": [_vp, _vp, C.c_uint32, _pp, _pp],
    "helrm_infer_batch": [_vp, _vp, _pp, _pp, _pp],
    "helrm_batch_set_graph": [_vp, _vp, C.c_int],
    "helrm_infer_batch_e2e_device": [_vp, _vp, _pp, _vp, _vp, C.c_uint64, _vp],
    "helrm_infer_batch_e2e": [_vp, _vp, _pp, _vp, _vp, C.c_uint64, _vp],
    "helrm_server_create": [_vp, C.c_uint32, C.c_uint32, C.c_uint64, _pp],
    "helrm_server_add_client": [_vp, _vp, _vp, _vp, _u32p],
    "helrm_server_run": [_vp, _vp, C.c_uint32, _dp, _u32p, _pp, _pp, _pp, _dp, C.c_void_p],
    "helrm_ctx_profile": [_vp, C.c_int],
    "helrm_ctx_ntt_tuning": [_vp, _u32p],
    "helrm_ctx_wait_selftest": [_vp, C.c_uint32],
    "helrm_ctx_profile_report": [_vp, C.c_char_p, C.c_uint64, _u64p],
    "helrm_ctx_profile_records": [_vp, C.c_char_p, C.c_uint64, _u64p],
    "helrm_keygen_ex": [_vp, C.c_uint64, C.c_uint32, _i32p, C.c_uint32, C.c_int, _pp, _pp],
    "helrm_conjugate": [_vp, _vp, _vp, _pp],
    "helrm_ptmat_export": [_vp, _vp, _i64p, C.c_uint32],
    "helrm_boot_create": [_vp, C.POINTER(BootDesc), _pp],
    "helrm_boot_info": [_vp, _u32p],
    "helrm_boot_rotations": [_vp, _i32p, _u32p],
    "helrm_boot_coeffs": [_vp, _dp, C.c_uint32],
    "helrm_boot_matrix": [_vp, C.c_uint32, _pp],
    "helrm_bootstrap": [_vp, _vp, _vp, _vp, _pp, _pp],
}


def lib():
    """Load libhelrm.so; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.helrm_free.argtypes = [_vp]
        L.helrm_free.restype = None
        L.helrm_last_error.argtypes = [_vp]
        L.helrm_last_error.restype = C.c_char_p
        L.helrm_status_string.argtypes = [C.c_int]
        L.helrm_status_string.restype = C.c_char_p
        _lib = L
    return _lib


def declared_symbols():
    """Entry points this binding expects (all declared in include/helrm.h)."""
    return sorted(list(_SIGS) + ["helrm_free", "helrm_last_error", "helrm_status_string"])


def _owning_context(keep):
    if isinstance(keep, Context):
        return keep
    if isinstance(keep, (tuple, list)):
        for k in keep:
            c = _owning_context(k)
            if c is not None:
                return c
    return None


class Handle:
    """An owned library handle; freed on garbage collection.

    A handle that depends on a context is counted on it, and the context is
    released only after the last of them: the library requires that order,
    and the cyclic garbage collector finalises the members of a cycle (a
    context and its handles held by a traceback, say) in no particular order.
    """

    def __init__(self, ptr, keep=None):
        self.ptr = C.c_void_p(ptr)
        self._keep = keep
        self._ctx = _owning_context(keep)
        if self._ctx is not None and self.ptr:
            self._ctx._live += 1
        else:
            self._ctx = None

    def __del__(self):
        try:
            if self.ptr and _lib is not None:
                _lib.helrm_free(self.ptr)
                self.ptr = C.c_void_p()
            ctx, self._ctx = self._ctx, None
            if ctx is not None:
                ctx._live -= 1
                ctx._release_if_done()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.ptr


class Context(Handle):
    """The context: freed when it is collected and no handle of it is left."""

    def __init__(self, ptr):
        self._live = 0
        self._closing = False
        super().__init__(ptr)

    def _release_if_done(self):
        if self._closing and self._live == 0 and self.ptr and _lib is not None:
            _lib.helrm_free(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self._closing = True
            self._release_if_done()
        except Exception:
            pass


class Borrowed(Handle):
    """A handle owned by another object (kept alive by it); never freed here."""

    def __del__(self):
        pass


def _check(ctx, st):
    if st != 0:
        msg = lib().helrm_last_error(ctx.ptr if ctx is not None else None)
        raise HelrmError(st, msg.decode() if msg else "")


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(_u64p)


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_i64p)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_i32p)


# ------------------------------------------------------------------ context
def helrm_ctx_create(log_n, q_bits, n_p, p_bits, alpha, log2_scale, device=0, stream=0) -> Context:
    qb = (C.c_uint32 * len(q_bits))(*q_bits)
    p = Params(log_n, len(q_bits), qb, n_p, p_bits, alpha, log2_scale)
    out = C.c_void_p()
    st = lib().helrm_ctx_create(C.byref(p), device, C.c_void_p(stream), C.byref(out))
    if st != 0:
        raise HelrmError(st, "helrm_ctx_create failed (see parameters)")
    return Context(out.value)


def helrm_ctx_primes(ctx):
    d = helrm_ctx_dims(ctx)
    n = d[2] + 1 + d[3]
    pr = np.zeros(n, dtype=np.uint64)
    psi = np.zeros(n, dtype=np.uint64)
    _check(ctx, lib().helrm_ctx_primes(ctx.ptr, pr.ctypes.data_as(_u64p), psi.ctypes.data_as(_u64p)))
    return [int(x) for x in pr], [int(x) for x in psi]


def helrm_ctx_dims(ctx):
    d = (C.c_uint32 * 6)()
    _check(ctx, lib().helrm_ctx_dims(ctx.ptr, d))
    return list(d)


def helrm_ctx_set_memory_cap(ctx, nbytes: int):
    _check(ctx, lib().helrm_ctx_set_memory_cap(ctx.ptr, nbytes))


def helrm_ctx_memory_in_use(ctx) -> int:
    v = C.c_uint64()
    _check(ctx, lib().helrm_ctx_memory_in_use(ctx.ptr, C.byref(v)))
    return v.value


def helrm_ctx_synchronize(ctx):
    _check(ctx, lib().helrm_ctx_synchronize(ctx.ptr))


def helrm_ctx_launch_count(ctx) -> int:
    v = C.c_uint64()
    _check(ctx, lib().helrm_ctx_launch_count(ctx.ptr, C.byref(v)))
    return v.value


def helrm_ntt(ctx, d_ptr: int, n_limbs: int, first_prime: int, inverse: bool):
    _check(ctx, lib().helrm_ntt(ctx.ptr, C.c_void_p(d_ptr), n_limbs, first_prime, int(inverse)))


def helrm_alu_peak(ctx, kind: int, blocks_per_sm: int = 4, iters: int = 4096) -> float:
    out = C.c_double()
    _check(ctx, lib().helrm_alu_peak(ctx.ptr, kind, blocks_per_sm, iters, C.byref(out)))
    return out.value


# ------------------------------------------------------------------ keys / pts / cts
def helrm_keygen(ctx, seed: int, rot_steps=()):
    st_arr, st_p = _i32(list(rot_steps) or [0])
    sk, evk = C.c_void_p(), C.c_void_p()
    _check(ctx, lib().helrm_keygen(ctx.ptr, seed, st_p, len(rot_steps), C.byref(sk), C.byref(evk)))
    return Handle(sk.value, ctx), Handle(evk.value, ctx)


def helrm_model_keygen(ctx, m, seed: int):
    """(sk, evk) with the model's keys, each truncated to the highest level it is used at."""
    sk, evk = C.c_void_p(), C.c_void_p()
    _check(ctx, lib().helrm_model_keygen(ctx.ptr, m.ptr, seed, C.byref(sk), C.byref(evk)))
    return Handle(sk.value, ctx), Handle(evk.value, ctx)


def helrm_evk_add_rotations(ctx, sk, evk, rot_steps):
    a, p = _i32(list(rot_steps) or [0])
    _check(ctx, lib().helrm_evk_add_rotations(ctx.ptr, sk.ptr, evk.ptr, p, len(rot_steps)))


def helrm_evk_bytes(ctx, evk) -> int:
    v = C.c_uint64()
    _check(ctx, lib().helrm_evk_bytes(evk.ptr, C.byref(v)))
    return v.value


def helrm_encode(ctx, slots, level: int, scale: float):
    a, p = _f64(slots)
    out = C.c_void_p()
    _check(ctx, lib().helrm_encode(ctx.ptr, p, len(a), level, scale, C.byref(out)))
    return Handle(out.value, ctx)


def helrm_pt_import(ctx, coeffs, level: int, scale: float):
    a, p = _i64(coeffs)
    out = C.c_void_p()
    _check(ctx, lib().helrm_pt_import(ctx.ptr, p, level, scale, C.byref(out)))
    return Handle(out.value, ctx)


def helrm_pt_export(ctx, pt):
    n = helrm_ctx_dims(ctx)[0]
    out = np.zeros(n, dtype=np.int64)
    _check(ctx, lib().helrm_pt_export(ctx.ptr, pt.ptr, out.ctypes.data_as(_i64p)))
    return out


def helrm_encrypt(ctx, evk, pt, seed: int):
    out = C.c_void_p()
    _check(ctx, lib().helrm_encrypt(ctx.ptr, evk.ptr, pt.ptr, seed, C.byref(out)))
    return Handle(out.value, ctx)


def helrm_decrypt(ctx, sk, ct, n_slots: int):
    out = np.zeros(max(n_slots, 1))
    _check(ctx, lib().helrm_decrypt(ctx.ptr, sk.ptr, ct.ptr, out.ctypes.data_as(_dp), n_slots))
    return out[:n_slots]


def helrm_ct_info(ctx, ct):
    lv, sc = C.c_int32(), C.c_double()
    _check(ctx, lib().helrm_ct_info(ct.ptr, C.byref(lv), C.byref(sc)))
    return lv.value, sc.value


def helrm_ct_export(ctx, ct):
    """(coeffs [2, level+1, N] uint64 coefficient domain, level, scale)."""
    lv, sc = helrm_ct_info(ctx, ct)
    n = helrm_ctx_dims(ctx)[0]
    out = np.zeros((2, lv + 1, n), dtype=np.uint64)
    _check(ctx, lib().helrm_ct_export(ctx.ptr, ct.ptr, out.ctypes.data_as(_u64p), None, None))
    return out, lv, sc


def helrm_ct_import(ctx, coeffs, level: int, scale: float):
    a, p = _u64(coeffs)
    out = C.c_void_p()
    _check(ctx, lib().helrm_ct_import(ctx.ptr, p, level, scale, C.byref(out)))
    return Handle(out.value, ctx)


def _ct_op(name, ctx, *args):
    out = C.c_void_p()
    _check(ctx, getattr(lib(), name)(ctx.ptr, *args, C.byref(out)))
    return Handle(out.value, ctx)


def helrm_add(ctx, a, b):
    return _ct_op("helrm_add", ctx, a.ptr, b.ptr)


def helrm_sub(ctx, a, b):
    return _ct_op("helrm_sub", ctx, a.ptr, b.ptr)


def helrm_add_pt(ctx, a, pt):
    return _ct_op("helrm_add_pt", ctx, a.ptr, pt.ptr)


def helrm_mul_pt(ctx, a, pt):
    return _ct_op("helrm_mul_pt", ctx, a.ptr, pt.ptr)


def helrm_mul(ctx, evk, a, b):
    return _ct_op("helrm_mul", ctx, evk.ptr, a.ptr, b.ptr)


def helrm_poly_eval(ctx, evk, x, coeffs, target_scale: float):
    """sum_k coeffs[k] x^k slot-wise (coeffs: a_0 .. a_d)."""
    cf = np.ascontiguousarray(coeffs, dtype=np.float64)
    out = C.c_void_p()
    _check(ctx, lib().helrm_poly_eval(ctx.ptr, evk.ptr, x.ptr, cf.ctypes.data_as(_dp), len(cf), target_scale,
                                      C.byref(out)))
    return Handle(out.value, ctx)


def helrm_rescale(ctx, a):
    return _ct_op("helrm_rescale", ctx, a.ptr)


def helrm_drop_level(ctx, a, level: int):
    return _ct_op("helrm_drop_level", ctx, a.ptr, level)


def helrm_rotate(ctx, evk, a, step: int):
    return _ct_op("helrm_rotate", ctx, evk.ptr, a.ptr, step)


def helrm_rotate_hoisted(ctx, evk, a, steps):
    arr, p = _i32(list(steps))
    outs = (C.c_void_p * len(steps))()
    _check(ctx, lib().helrm_rotate_hoisted(ctx.ptr, evk.ptr, a.ptr, p, len(steps), outs))
    return [Handle(o, ctx) for o in outs]


# ------------------------------------------------------------------ matvec / embeddings
def helrm_ptmat_prepare(ctx, W, in_pad, out_pad, level, ct_scale, target_scale):
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = C.c_void_p()
    _check(ctx, lib().helrm_ptmat_prepare(ctx.ptr, W.ctypes.data_as(_dp), W.shape[0], W.shape[1], in_pad,
                                          out_pad, level, ct_scale, target_scale, C.byref(out)))
    return Handle(out.value, ctx)


def helrm_ptmat_info(ctx, m):
    o = (C.c_uint32 * 6)()
    _check(ctx, lib().helrm_ptmat_info(m.ptr, o))
    return dict(zip(["D", "n1", "n2", "nonzero", "folds", "level"], list(o)))


def _steps(fn, ctx, h):
    n = C.c_uint32(0)
    _check(ctx, fn(h.ptr, None, C.byref(n)))
    arr = (C.c_int32 * max(n.value, 1))()
    _check(ctx, fn(h.ptr, arr, C.byref(n)))
    return list(arr)[: n.value]


def helrm_ptmat_rotations(ctx, m):
    return _steps(lib().helrm_ptmat_rotations, ctx, m)


def helrm_ptmat_import(ctx, m, coeffs):
    a, p = _i64(coeffs)
    _check(ctx, lib().helrm_ptmat_import(ctx.ptr, m.ptr, p, a.shape[0]))


def helrm_ptct_matvec(ctx, evk, m, ct):
    return _ct_op("helrm_ptct_matvec", ctx, evk.ptr, m.ptr, ct.ptr, 1)


def _float_tables(tables):
    """tables[t] = list of digit tables (rows x dim) -> stacked float32 arrays + pointer array."""
    arrs = [np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float32) for x in t], axis=0))
            for t in tables]
    ptrs = (C.POINTER(C.c_float) * len(arrs))(*[a.ctypes.data_as(C.POINTER(C.c_float)) for a in arrs])
    return arrs, ptrs


def helrm_emb_prepare(ctx, cards, base_p, threshold, dim, tables, out_offset, out_pad, level, ct_scale,
                      target_scale):
    """threshold: tables with more rows are digit-decomposed (0 = base_p)."""
    c_arr, c_p = _u64(cards)
    arrs, ptrs = _float_tables(tables)
    out = C.c_void_p()
    _check(ctx, lib().helrm_emb_prepare(ctx.ptr, len(cards), c_p, base_p, threshold, dim, ptrs, out_offset, out_pad,
                                        level, ct_scale, target_scale, C.byref(out)))
    return Handle(out.value, ctx)


def helrm_emb_info(ctx, emb):
    w, p = C.c_uint32(), C.c_uint32()
    _check(ctx, lib().helrm_emb_info(emb.ptr, C.byref(w), C.byref(p)))
    return w.value, p.value


def helrm_query_pack(ctx, emb, indices, n_slots):
    a, p = _u64(indices)
    out = np.zeros(n_slots)
    _check(ctx, lib().helrm_query_pack(emb.ptr, p, out.ctypes.data_as(_dp), n_slots))
    return out


def helrm_emb_chunks(ctx, emb) -> int:
    n = C.c_uint32()
    _check(ctx, lib().helrm_emb_chunks(emb.ptr, C.byref(n)))
    return n.value


def helrm_emb_matrix(ctx, emb, chunk: int):
    """The embedding's own matrix of ciphertext `chunk` (not freed by this handle)."""
    out = C.c_void_p()
    _check(ctx, lib().helrm_emb_matrix(emb.ptr, chunk, C.byref(out)))
    return Borrowed(out.value, emb)


def helrm_embedding_lookup_multi(ctx, evk, emb, sels):
    out = C.c_void_p()
    _check(ctx, lib().helrm_embedding_lookup_multi(ctx.ptr, evk.ptr, emb.ptr, _ptrs(sels), len(sels), C.byref(out)))
    return Handle(out.value, ctx)


def helrm_embedding_lookup(ctx, evk, emb, sel):
    return _ct_op("helrm_embedding_lookup", ctx, evk.ptr, emb.ptr, sel.ptr, 1)


# ------------------------------------------------------------------ model
def helrm_model_create(ctx, spec, w):
    """spec: synthetic.DLRMSpec-like object; w: synthetic.DLRMWeights-like object."""
    keep = []

    def dptrs(mats):
        arrs = [np.ascontiguousarray(m, dtype=np.float64) for m in mats]
        keep.extend(arrs)
        return (C.POINTER(C.c_double) * len(arrs))(*[a.ctypes.data_as(_dp) for a in arrs])

    bw = (C.c_uint32 * len(spec.bottom))(*spec.bottom)
    tw = (C.c_uint32 * len(spec.top))(*spec.top)
    cards = np.ascontiguousarray(spec.cards, dtype=np.uint64)
    tarrs, tptrs = _float_tables(w.tables)
    keep += [bw, tw, cards, tarrs, tptrs]
    d = ModelDesc(spec.n_dense, len(w.bottom_W), bw, dptrs(w.bottom_W), dptrs(w.bottom_b),
                  len(w.top_W), tw, dptrs(w.top_W), dptrs(w.top_b), len(spec.cards),
                  cards.ctypes.data_as(_u64p), spec.base, spec.dim, tptrs,
                  0 if spec.interaction == "dot" else 1, getattr(spec, "threshold", 0) or 0)
    act = getattr(spec, "act", None)
    if act is not None:
        acts = np.ascontiguousarray(act, dtype=np.float64)
        keep.append(acts)
        d.act_degree = len(acts) - 1
        d.act_coeffs = acts.ctypes.data_as(_dp)
    for pt in getattr(spec, "boot", ()) or ():
        if pt == "z":
            d.boot_z = 1
        elif pt[0] == "b":
            d.boot_bottom |= 1 << int(pt[1:])
        elif pt[0] == "t":
            d.boot_top |= 1 << int(pt[1:])
        else:
            raise ValueError(f"unknown bootstrap point {pt}")
    bc = getattr(spec, "boot_coeffs", None)
    if bc is not None:
        bca = np.ascontiguousarray(bc, dtype=np.float64)
        keep.append(bca)
        d.boot_coeffs = bca.ctypes.data_as(_dp)
    out = C.c_void_p()
    _check(ctx, lib().helrm_model_create(ctx.ptr, C.byref(d), C.byref(out)))
    return Handle(out.value, ctx)


def helrm_model_info(ctx, m):
    o = (C.c_uint32 * 10)()
    _check(ctx, lib().helrm_model_info(m.ptr, o))
    keys = ["lvl_dense", "lvl_sel", "lvl_z", "lvl_u", "p_dense", "p_sel", "W_z", "W_u", "n_plaintexts", "n_sel"]
    return dict(zip(keys, list(o)))


def helrm_model_rotations(ctx, m):
    return _steps(lib().helrm_model_rotations, ctx, m)


def helrm_model_import_plaintexts(ctx, m, coeffs):
    a, p = _i64(coeffs)
    _check(ctx, lib().helrm_model_import_plaintexts(ctx.ptr, m.ptr, p, a.shape[0]))


def helrm_model_export_plaintexts(ctx, m):
    n = helrm_ctx_dims(ctx)[0]
    cnt = helrm_model_info(ctx, m)["n_plaintexts"]
    out = np.zeros((cnt, n), dtype=np.int64)
    _check(ctx, lib().helrm_model_export_plaintexts(ctx.ptr, m.ptr, out.ctypes.data_as(_i64p), cnt))
    return out


def helrm_encrypt_query(ctx, evk, m, dense, indices, seed: int):
    """(ct_dense, ct_sel): ct_sel is one handle when the model's n_sel is 1, else a list of n_sel."""
    d, dp = _f64(dense)
    i, ip = _u64(indices)
    ns = helrm_model_info(ctx, m)["n_sel"]
    a, b = C.c_void_p(), (C.c_void_p * ns)()
    _check(ctx, lib().helrm_encrypt_query(ctx.ptr, evk.ptr, m.ptr, dp, ip, seed, C.byref(a), b))
    sel = [Handle(b[k], ctx) for k in range(ns)]
    return Handle(a.value, ctx), (sel[0] if ns == 1 else sel)


def helrm_infer(ctx, evk, m, ct_dense, ct_sel):
    return _ct_op("helrm_infer", ctx, evk.ptr, m.ptr, ct_dense.ptr, ct_sel.ptr)


def helrm_infer_multi(ctx, evk, m, ct_dense, cts_sel):
    out = C.c_void_p()
    _check(ctx, lib().helrm_infer_multi(ctx.ptr, evk.ptr, m.ptr, ct_dense.ptr, _ptrs(cts_sel), len(cts_sel),
                                        C.byref(out)))
    return Handle(out.value, ctx)


def helrm_decrypt_logit(ctx, sk, ct):
    lg, pr = C.c_double(), C.c_double()
    _check(ctx, lib().helrm_decrypt_logit(ctx.ptr, sk.ptr, ct.ptr, C.byref(lg), C.byref(pr)))
    return lg.value, pr.value


def helrm_infer_e2e_device(ctx, sk, evk, m, d_dense: int, d_indices: int, n_queries: int, seed: int,
                           d_logits: int, d_probs: int = 0):
    """All buffers are device pointers (ints); stream-ordered, no synchronisation."""
    _check(ctx, lib().helrm_infer_e2e_device(ctx.ptr, sk.ptr, evk.ptr, m.ptr, C.c_void_p(d_dense),
                                             C.c_void_p(d_indices), n_queries, seed, C.c_void_p(d_logits),
                                             C.c_void_p(d_probs or None)))


def _ptrs(handles):
    return (C.c_void_p * len(handles))(*[h.ptr.value for h in handles])


def helrm_batch_create(ctx, m, evks):
    """A lockstep batch of len(evks) queries of model m; evks[q] = the key set of query q's client."""
    arr = _ptrs(evks)
    out = C.c_void_p()
    _check(ctx, lib().helrm_batch_create(ctx.ptr, m.ptr, len(evks), arr, C.byref(out)))
    return Handle(out.value, (ctx, m, list(evks)))


def helrm_batch_set_graph(ctx, batch, enable: bool):
    _check(ctx, lib().helrm_batch_set_graph(ctx.ptr, batch.ptr, int(enable)))


def helrm_infer_batch(ctx, batch, cts_dense, cts_sel):
    """cts_sel: n x n_sel handles, query-major (a flat list, or one list per query)."""
    n = len(cts_dense)
    cts_sel = [x for s in cts_sel for x in (s if isinstance(s, (list, tuple)) else [s])]
    outs = (C.c_void_p * n)()
    _check(ctx, lib().helrm_infer_batch(ctx.ptr, batch.ptr, _ptrs(cts_dense), _ptrs(cts_sel), outs))
    return [Handle(outs[q], ctx) for q in range(n)]


def helrm_infer_batch_e2e_device(ctx, batch, sks, d_dense: int, d_indices: int, seed: int, d_logits: int):
    """Device pointers (ints): d_dense n x n_dense f64, d_indices n x n_tables u64, d_logits n f64."""
    _check(ctx, lib().helrm_infer_batch_e2e_device(ctx.ptr, batch.ptr, _ptrs(sks), C.c_void_p(d_dense),
                                                   C.c_void_p(d_indices), seed, C.c_void_p(d_logits)))


def helrm_infer_batch_e2e(ctx, batch, sks, dense, indices, seed: int):
    """Host arrays: dense n x n_dense, indices n x n_tables; returns the n logits."""
    d = np.ascontiguousarray(dense, dtype=np.float64)
    i = np.ascontiguousarray(np.asarray(indices).astype(np.uint64))
    out = np.zeros(d.shape[0])
    _check(ctx, lib().helrm_infer_batch_e2e(ctx.ptr, batch.ptr, _ptrs(sks), C.c_void_p(d.ctypes.data),
                                            C.c_void_p(i.ctypes.data), seed, C.c_void_p(out.ctypes.data)))
    return out


def helrm_server_create(ctx, n_slots: int, max_batch: int, mem_budget: int = 0):
    out = C.c_void_p()
    _check(ctx, lib().helrm_server_create(ctx.ptr, n_slots, max_batch, mem_budget, C.byref(out)))
    return Handle(out.value, ctx)


def helrm_server_add_client(ctx, server, m, evk) -> int:
    cid = C.c_uint32()
    _check(ctx, lib().helrm_server_add_client(ctx.ptr, server.ptr, m.ptr, evk.ptr, C.byref(cid)))
    server._keep = (server._keep, m, evk) if server._keep is not None else (m, evk)
    return cid.value


def helrm_server_run(ctx, server, arrival_s, clients, cts_dense, cts_sel):
    """Replay a trace; returns (logit ciphertexts, latencies in ms, stats dict).
    cts_sel[r]: request r's selector handle, or the list of them when its
    model's selector spans several ciphertexts (flattened request by request)."""
    n = len(arrival_s)
    cts_sel = [x for s in cts_sel for x in (s if isinstance(s, (list, tuple)) else [s])]
    arr, ap = _f64(arrival_s)
    cl = np.ascontiguousarray(clients, dtype=np.uint32)
    outs = (C.c_void_p * n)()
    lat = np.zeros(n)
    stt = ServeStats()
    _check(ctx, lib().helrm_server_run(ctx.ptr, server.ptr, n, ap, cl.ctypes.data_as(_u32p), _ptrs(cts_dense),
                                       _ptrs(cts_sel), outs, lat.ctypes.data_as(_dp), C.byref(stt)))
    stats = {f: getattr(stt, f) for f, _ in ServeStats._fields_}
    return [Handle(outs[r], ctx) for r in range(n)], lat, stats


def helrm_rescale_noalloc(ctx, d_in: int, d_out: int, level: int, n_polys: int):
    """Rescale without allocating: device pointers in (n_polys x (level+1) x N) and
    out (n_polys x level x N), NTT domain; scratch is a static 1 MiB device array."""
    _check(ctx, lib().helrm_rescale_noalloc(ctx.ptr, C.c_void_p(d_in), C.c_void_p(d_out), level, n_polys))


def helrm_ctx_wait_selftest(ctx, polls: int):
    """Raises HelrmError(HELRM_E_TIMEOUT): a bounded device wait that ran out."""
    _check(ctx, lib().helrm_ctx_wait_selftest(ctx.ptr, polls))


def helrm_ctx_ntt_tuning(ctx):
    """{limb bucket: (tile words, CTA multiple of the SM count, elements per thread)} chosen at context creation."""
    out = (C.c_uint32 * 12)()
    _check(ctx, lib().helrm_ctx_ntt_tuning(ctx.ptr, out))
    return {b: (out[3 * i], out[3 * i + 1], out[3 * i + 2]) for i, b in enumerate(["<=4", "<=16", "<=64", ">64"])}


def helrm_ctx_profile(ctx, enable: bool):
    _check(ctx, lib().helrm_ctx_profile(ctx.ptr, int(enable)))


def helrm_ctx_profile_report(ctx):
    """{kernel name: (launches, total_ms, algorithmic_bytes)}"""
    need = C.c_uint64(0)
    _check(ctx, lib().helrm_ctx_profile_report(ctx.ptr, None, 0, C.byref(need)))
    buf = C.create_string_buffer(need.value + 1)
    _check(ctx, lib().helrm_ctx_profile_report(ctx.ptr, buf, need.value + 1, None))
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms, b = line.split()
        out[name] = (int(n), float(ms), float(b))
    return out


def helrm_ctx_profile_records(ctx):
    """[(kernel name, ms, algorithmic_bytes)] per recorded launch, in order"""
    need = C.c_uint64(0)
    _check(ctx, lib().helrm_ctx_profile_records(ctx.ptr, None, 0, C.byref(need)))
    buf = C.create_string_buffer(need.value + 1)
    _check(ctx, lib().helrm_ctx_profile_records(ctx.ptr, buf, need.value + 1, None))
    out = []
    for line in buf.value.decode().splitlines():
        name, ms, b = line.split()
        out.append((name, float(ms), float(b)))
    return out


def helrm_infer_e2e(ctx, sk, evk, m, dense, indices, seed: int):
    d, dp = _f64(dense)
    i, ip = _u64(indices)
    nq = d.shape[0]
    lg = np.zeros(nq)
    pr = np.zeros(nq)
    _check(ctx, lib().helrm_infer_e2e(ctx.ptr, sk.ptr, evk.ptr, m.ptr, dp, ip, nq, seed,
                                      lg.ctypes.data_as(_dp), pr.ctypes.data_as(_dp)))
    return lg, pr


# ------------------------------------------------------------------ bootstrapping
def helrm_keygen_ex(ctx, seed: int, hamming_weight: int = 0, rot_steps=(), conj: bool = False):
    """(sk, evk): hamming_weight 0 is helrm_keygen's dense secret, h > 0 a sparse one;
    conj adds the key of X -> X^(2N-1)."""
    st_arr, st_p = _i32(list(rot_steps) or [0])
    sk, evk = C.c_void_p(), C.c_void_p()
    _check(ctx, lib().helrm_keygen_ex(ctx.ptr, seed, hamming_weight, st_p, len(rot_steps), 1 if conj else 0,
                                      C.byref(sk), C.byref(evk)))
    return Handle(sk.value, ctx), Handle(evk.value, ctx)


def helrm_conjugate(ctx, evk, a):
    return _ct_op("helrm_conjugate", ctx, evk.ptr, a.ptr)


def helrm_ptmat_export(ctx, m, count: int, n: int):
    out = np.zeros((count, n), dtype=np.int64)
    _check(ctx, lib().helrm_ptmat_export(ctx.ptr, m.ptr, out.ctypes.data_as(_i64p), count))
    return out


def helrm_boot_create(ctx, n_s: int, K: int = 24, r: int = 6, degree: int = 16, log2_boost: int = 10,
                      cts_levels: int = 1, s_ref: float = 2.0**40, eval_scale: float = 2.0**60, coeffs=None):
    cf = None if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
    d = BootDesc(n_s, K, r, degree, log2_boost, cts_levels, s_ref, eval_scale,
                 cf.ctypes.data_as(_dp) if cf is not None else None)
    out = C.c_void_p()
    _check(ctx, lib().helrm_boot_create(ctx.ptr, C.byref(d), C.byref(out)))
    return Handle(out.value, ctx)


def helrm_boot_info(ctx, b):
    o = (C.c_uint32 * 6)()
    _check(ctx, lib().helrm_boot_info(b.ptr, o))
    return dict(zip(["n_s", "level_top", "level_stc", "level_out", "n_plaintexts", "degree"], list(o)))


def helrm_boot_rotations(ctx, b):
    return _steps(lib().helrm_boot_rotations, ctx, b)


def helrm_boot_coeffs(ctx, b):
    n = helrm_boot_info(ctx, b)["degree"] + 1
    out = (C.c_double * n)()
    _check(ctx, lib().helrm_boot_coeffs(b.ptr, out, n))
    return list(out)


def helrm_boot_matrix(ctx, b, which: int):
    """0: CoeffToSlot, 1: SlotToCoeff (not freed by this handle)."""
    out = C.c_void_p()
    _check(ctx, lib().helrm_boot_matrix(b.ptr, which, C.byref(out)))
    return Borrowed(out.value, b)


def helrm_bootstrap(ctx, evk, b, ct, stages: bool = False):
    """The refreshed ciphertext; with stages, (out, [raised, subsum, cts, evalmod, out copy])."""
    out = C.c_void_p()
    st = (C.c_void_p * 5)() if stages else None
    _check(ctx, lib().helrm_bootstrap(ctx.ptr, evk.ptr, b.ptr, ct.ptr, C.byref(out), st))
    if stages:
        return Handle(out.value, ctx), [Handle(v, ctx) for v in st]
    return Handle(out.value, ctx)
