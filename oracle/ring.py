"""ctypes wrappers around oracle/ring.c (test infrastructure only).

Polynomials are numpy uint64 arrays shaped [limbs, N] (coefficient or
evaluation values, canonical residues in [0, q)).  ``moduli`` is a sequence of
Python ints, one per limb.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ring.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libhelrm_oracle.so")
_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile ring.c into oracle/_build/libhelrm_oracle.so with gcc."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u64 = ctypes.c_uint64
            L.orc_mul_mod.argtypes = [u64, u64, u64]
            L.orc_mul_mod.restype = u64
            L.orc_pow_mod.argtypes = [u64, u64, u64]
            L.orc_pow_mod.restype = u64
            L.orc_negacyclic_schoolbook.argtypes = [_u64p, _u64p, _u64p, u64, u64]
            L.orc_ntt_batch.argtypes = [_u64p, u64, u64, _u64p, _u64p, ctypes.c_int]
            L.orc_polymul_batch.argtypes = [_u64p, _u64p, _u64p, u64, u64, _u64p, _u64p]
            L.orc_mul_batch.argtypes = [_u64p, _u64p, _u64p, u64, u64, _u64p]
            L.orc_mul_scalar_batch.argtypes = [_u64p, _u64p, _u64p, u64, u64, _u64p]
            L.orc_reduce128_batch.argtypes = [_u64p, _u64p, _u64p, u64, u64, _u64p]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u64p)


def _mods(moduli) -> np.ndarray:
    return np.ascontiguousarray(np.array([int(m) for m in moduli], dtype=np.uint64))


def _as2d(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a.reshape(1, -1) if a.ndim == 1 else a


def mul_mod(a: int, b: int, q: int) -> int:
    return int(lib().orc_mul_mod(a % q, b % q, q))


def schoolbook(a: np.ndarray, b: np.ndarray, q: int) -> np.ndarray:
    """Negacyclic product of two length-N residue vectors, O(N^2)."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.empty_like(a)
    lib().orc_negacyclic_schoolbook(_p(a), _p(b), _p(out), a.shape[-1], q)
    return out


def ntt(a: np.ndarray, moduli, psis, inverse: bool = False) -> np.ndarray:
    """Negacyclic NTT per limb: forward ahat[k] = a(psi^(2k+1)), natural order."""
    out = _as2d(a).copy()
    m, r = _mods(moduli), _mods(psis)
    assert out.shape[0] == len(m)
    lib().orc_ntt_batch(_p(out), out.shape[1], out.shape[0], _p(m), _p(r), int(inverse))
    return out


def polymul(a: np.ndarray, b: np.ndarray, moduli, psis) -> np.ndarray:
    a2, b2 = _as2d(a), _as2d(b)
    assert a2.shape == b2.shape
    out = np.empty_like(a2)
    m, r = _mods(moduli), _mods(psis)
    lib().orc_polymul_batch(_p(a2), _p(b2), _p(out), a2.shape[1], a2.shape[0], _p(m), _p(r))
    return out


def mul(a: np.ndarray, b: np.ndarray, moduli) -> np.ndarray:
    a2, b2 = _as2d(a), _as2d(b)
    out = np.empty_like(a2)
    m = _mods(moduli)
    lib().orc_mul_batch(_p(a2), _p(b2), _p(out), a2.shape[1], a2.shape[0], _p(m))
    return out


def mul_scalar(a: np.ndarray, scalars, moduli) -> np.ndarray:
    """out[l] = a[l] * scalars[l] mod moduli[l]; a may hold values >= q."""
    a2 = _as2d(a)
    out = np.empty_like(a2)
    c = _mods([int(s) % int(q) for s, q in zip(scalars, moduli)])
    m = _mods(moduli)
    lib().orc_mul_scalar_batch(_p(a2), _p(c), _p(out), a2.shape[1], a2.shape[0], _p(m))
    return out


def reduce128(hi: np.ndarray, lo: np.ndarray, moduli) -> np.ndarray:
    h2, l2 = _as2d(hi), _as2d(lo)
    out = np.empty_like(h2)
    m = _mods(moduli)
    lib().orc_reduce128_batch(_p(h2), _p(l2), _p(out), h2.shape[1], h2.shape[0], _p(m))
    return out


def add(a: np.ndarray, b: np.ndarray, moduli) -> np.ndarray:
    q = _mods(moduli)[:, None]
    return (_as2d(a) + _as2d(b)) % q          # residues < 2^62: no overflow


def sub(a: np.ndarray, b: np.ndarray, moduli) -> np.ndarray:
    q = _mods(moduli)[:, None]
    return (_as2d(a) + (q - _as2d(b))) % q


def neg(a: np.ndarray, moduli) -> np.ndarray:
    q = _mods(moduli)[:, None]
    return (q - _as2d(a)) % q


def from_signed(v: np.ndarray, moduli) -> np.ndarray:
    """Reduce a vector of signed integers (int64 or Python ints) mod every q."""
    v = np.asarray(v)
    rows = []
    for q in moduli:
        q = int(q)
        if v.dtype == object:
            rows.append(np.array([int(x) % q for x in v], dtype=np.uint64))
        else:
            rows.append((v.astype(np.int64) % np.int64(q)).astype(np.uint64)
                        if q < 2**63 else None)
    return np.ascontiguousarray(np.stack(rows))
