"""ctypes wrapper for the plain CPU oracle (oracle/ks_oracle.cpp).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference leg may import this module; the product package never
does. The oracle is schoolbook ``unsigned __int128 %`` arithmetic that follows
the KeySwitch steps of the paper's Sec. II-A / Fig. 1 in order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ks_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libks_oracle.so")
_lock = threading.Lock()
_lib = None

u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libks_oracle.so (g++, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            l.orc_is_prime.restype = ctypes.c_int
            l.orc_is_prime.argtypes = [ctypes.c_uint64]
            l.orc_find_psi.restype = ctypes.c_uint64
            l.orc_find_psi.argtypes = [ctypes.c_uint64, ctypes.c_int]
            for f in (l.orc_ntt_fwd, l.orc_ntt_inv):
                f.restype = None
                f.argtypes = [u64p, u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            l.orc_bconv.restype = None
            l.orc_bconv.argtypes = [u64p, u64p, ctypes.c_int, u64p, ctypes.c_int, u64p,
                                    ctypes.c_int, ctypes.c_int]
            l.orc_moddown.restype = ctypes.c_int
            l.orc_moddown.argtypes = [ctypes.c_int] * 3 + [u64p, ctypes.c_int, u64p, ctypes.c_int,
                                                           u64p, u64p, ctypes.c_int]
            l.orc_keyswitch.restype = ctypes.c_int
            l.orc_keyswitch.argtypes = [ctypes.c_int] * 3 + [u64p, ctypes.c_int, u64p, ctypes.c_int,
                                                             u64p, u64p, u64p, u64p, u64p,
                                                             ctypes.c_int]
            l.orc_keygen.restype = ctypes.c_int
            l.orc_keygen.argtypes = [ctypes.c_int] * 3 + [
                u64p, ctypes.c_int, u64p, ctypes.c_int,
                ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_int8), u64p,
                ctypes.POINTER(ctypes.c_int32), u64p, ctypes.c_int]
            l.orc_keygen_poly.restype = ctypes.c_int
            l.orc_keygen_poly.argtypes = [ctypes.c_int] * 3 + [
                u64p, ctypes.c_int, u64p, ctypes.c_int,
                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int8), u64p,
                ctypes.POINTER(ctypes.c_int32), u64p, ctypes.c_int]
            l.orc_keyswitch_level.restype = ctypes.c_int
            l.orc_keyswitch_level.argtypes = [ctypes.c_int] * 3 + [
                u64p, ctypes.c_int, u64p, ctypes.c_int, ctypes.c_int, u64p, u64p, u64p,
                ctypes.c_int]
            l.orc_hmul.restype = ctypes.c_int
            l.orc_hmul.argtypes = [ctypes.c_int] * 3 + [
                u64p, ctypes.c_int, u64p, ctypes.c_int, ctypes.c_int, u64p, u64p, u64p, u64p,
                ctypes.c_int]
            l.orc_hrot.restype = ctypes.c_int
            l.orc_hrot.argtypes = [ctypes.c_int] * 3 + [
                u64p, ctypes.c_int, u64p, ctypes.c_int, ctypes.c_int, u64p, ctypes.c_uint64,
                u64p, u64p, ctypes.c_int]
            l.orc_automorph_ntt.restype = None
            l.orc_automorph_ntt.argtypes = [u64p, u64p, u64p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_uint64, ctypes.c_int]
            i64p = ctypes.POINTER(ctypes.c_int64)
            l.orc_negacyclic_mul_i64.restype = None
            l.orc_negacyclic_mul_i64.argtypes = [i64p, i64p, i64p, ctypes.c_int]
            l.orc_automorphism_i64.restype = None
            l.orc_automorphism_i64.argtypes = [i64p, i64p, ctypes.c_int, ctypes.c_uint64]
            _lib = l
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.uint64:
        return a.ctypes.data_as(u64p)
    if a.dtype == np.int8:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    if a.dtype == np.int32:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    if a.dtype == np.int64:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    raise TypeError(a.dtype)


def _u64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint64))


def is_prime(n: int) -> bool:
    return bool(lib().orc_is_prime(n))


def find_psi(q: int, logn: int) -> int:
    return int(lib().orc_find_psi(q, logn))


def ntt_fwd(a: np.ndarray, mods, logn: int, nthreads: int | None = None) -> np.ndarray:
    """Forward negacyclic NTT of limbs a[count][N] (copy); slot k = a(psi^(2 brv(k)+1))."""
    out = _u64(a).copy()
    mods = _u64(mods)
    lib().orc_ntt_fwd(_p(out), _p(mods), len(mods), logn, nthreads or default_threads())
    return out


def ntt_inv(a: np.ndarray, mods, logn: int, nthreads: int | None = None) -> np.ndarray:
    out = _u64(a).copy()
    mods = _u64(mods)
    lib().orc_ntt_inv(_p(out), _p(mods), len(mods), logn, nthreads or default_threads())
    return out


def bconv(x: np.ndarray, src, dst, logn: int, nthreads: int | None = None) -> np.ndarray:
    """Fast basis conversion of coefficient-form limbs x[len(src)][N] onto dst."""
    x = _u64(x)
    src, dst = _u64(src), _u64(dst)
    y = np.zeros((len(dst), 1 << logn), dtype=np.uint64)
    lib().orc_bconv(_p(x), _p(src), len(src), _p(dst), len(dst), _p(y), logn,
                    nthreads or default_threads())
    return y


def moddown(prm, acc: np.ndarray, nthreads: int | None = None) -> np.ndarray:
    """ModDown of acc[QP][N] (NTT form over Q u P) to out[L+1][N] (NTT form over Q)."""
    q, p = _u64(prm.q), _u64(prm.p)
    acc = _u64(acc)
    out = np.zeros((len(q), prm.N), dtype=np.uint64)
    rc = lib().orc_moddown(prm.dnum, prm.logn, prm.L, _p(q), len(q), _p(p), len(p), _p(acc),
                           _p(out), nthreads or default_threads())
    if rc:
        raise ValueError("orc_moddown: bad parameters")
    return out


def keyswitch(prm, d: np.ndarray, evk: np.ndarray, trace: bool = False,
              nthreads: int | None = None):
    """Hybrid KeySwitch of d[L+1][N] with evk[beta][2][QP][N]; returns out[2][L+1][N]
    (and, with trace=True, also ext[beta][QP][N] and acc[2][QP][N])."""
    q, p = _u64(prm.q), _u64(prm.p)
    d, evk = _u64(d), _u64(evk)
    out = np.zeros((2, len(q), prm.N), dtype=np.uint64)
    ext = np.zeros((prm.beta, prm.QP, prm.N), dtype=np.uint64) if trace else None
    acc = np.zeros((2, prm.QP, prm.N), dtype=np.uint64) if trace else None
    null = ctypes.cast(None, u64p)
    rc = lib().orc_keyswitch(prm.dnum, prm.logn, prm.L, _p(q), len(q), _p(p), len(p), _p(d),
                             _p(evk), _p(out), _p(ext) if trace else null,
                             _p(acc) if trace else null, nthreads or default_threads())
    if rc:
        raise ValueError("orc_keyswitch: bad parameters")
    return (out, ext, acc) if trace else out


def keygen(prm, s_from: np.ndarray, s_to: np.ndarray, a: np.ndarray, e: np.ndarray,
           nthreads: int | None = None) -> np.ndarray:
    """evk[beta][2][QP][N] from ternary keys, uniform a (NTT form) and small errors e."""
    q, p = _u64(prm.q), _u64(prm.p)
    s_from = np.ascontiguousarray(s_from, dtype=np.int8)
    s_to = np.ascontiguousarray(s_to, dtype=np.int8)
    a = _u64(a)
    e = np.ascontiguousarray(e, dtype=np.int32)
    evk = np.zeros((prm.beta, 2, prm.QP, prm.N), dtype=np.uint64)
    rc = lib().orc_keygen(prm.dnum, prm.logn, prm.L, _p(q), len(q), _p(p), len(p), _p(s_from),
                          _p(s_to), _p(a), _p(e), _p(evk), nthreads or default_threads())
    if rc:
        raise ValueError("orc_keygen: bad parameters")
    return evk


def keygen_poly(prm, s_from: np.ndarray, s_to: np.ndarray, a: np.ndarray, e: np.ndarray,
                nthreads: int | None = None) -> np.ndarray:
    """keygen with s_from any int64 polynomial (s^2 for relinearisation, sigma_k(s) for
    rotation)."""
    q, p = _u64(prm.q), _u64(prm.p)
    s_from = np.ascontiguousarray(s_from, dtype=np.int64)
    s_to = np.ascontiguousarray(s_to, dtype=np.int8)
    a = _u64(a)
    e = np.ascontiguousarray(e, dtype=np.int32)
    evk = np.zeros((prm.beta, 2, prm.QP, prm.N), dtype=np.uint64)
    rc = lib().orc_keygen_poly(prm.dnum, prm.logn, prm.L, _p(q), len(q), _p(p), len(p),
                               _p(s_from), _p(s_to), _p(a), _p(e), _p(evk),
                               nthreads or default_threads())
    if rc:
        raise ValueError("orc_keygen_poly: bad parameters")
    return evk


def keyswitch_level(prm, level: int, d: np.ndarray, evk: np.ndarray,
                    nthreads: int | None = None) -> np.ndarray:
    """KeySwitch at level `level` of d[level+1][N] with the level-L key of prm."""
    q, p = _u64(prm.q), _u64(prm.p)
    d, evk = _u64(d), _u64(evk)
    out = np.zeros((2, level + 1, prm.N), dtype=np.uint64)
    rc = lib().orc_keyswitch_level(prm.dnum, prm.logn, prm.L, _p(q), len(q), _p(p), len(p),
                                   level, _p(d), _p(evk), _p(out), nthreads or default_threads())
    if rc:
        raise ValueError("orc_keyswitch_level: bad parameters")
    return out


def hmul(prm, level: int, ct1: np.ndarray, ct2: np.ndarray, rlk: np.ndarray,
         nthreads: int | None = None) -> np.ndarray:
    """HMUL of ciphertexts [2][level+1][N] (NTT form) under the relinearisation key."""
    q, p = _u64(prm.q), _u64(prm.p)
    ct1, ct2, rlk = _u64(ct1), _u64(ct2), _u64(rlk)
    out = np.zeros((2, level + 1, prm.N), dtype=np.uint64)
    rc = lib().orc_hmul(prm.dnum, prm.logn, prm.L, _p(q), len(q), _p(p), len(p), level,
                        _p(ct1), _p(ct2), _p(rlk), _p(out), nthreads or default_threads())
    if rc:
        raise ValueError("orc_hmul: bad parameters")
    return out


def hrot(prm, level: int, ct: np.ndarray, k: int, rtk: np.ndarray,
         nthreads: int | None = None) -> np.ndarray:
    """HROT of ct [2][level+1][N] (NTT form) by the Galois element k under rtk."""
    q, p = _u64(prm.q), _u64(prm.p)
    ct, rtk = _u64(ct), _u64(rtk)
    out = np.zeros((2, level + 1, prm.N), dtype=np.uint64)
    rc = lib().orc_hrot(prm.dnum, prm.logn, prm.L, _p(q), len(q), _p(p), len(p), level,
                        _p(ct), k, _p(rtk), _p(out), nthreads or default_threads())
    if rc:
        raise ValueError("orc_hrot: bad parameters")
    return out


def automorph_ntt(a: np.ndarray, mods, logn: int, k: int,
                  nthreads: int | None = None) -> np.ndarray:
    """sigma_k of NTT-form limbs a[count][N] (through the coefficient domain)."""
    a, mods = _u64(a), _u64(mods)
    out = np.zeros_like(a)
    lib().orc_automorph_ntt(_p(a), _p(out), _p(mods), len(mods), logn, k,
                            nthreads or default_threads())
    return out


def negacyclic_mul_i64(a: np.ndarray, b: np.ndarray, logn: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int64)
    b = np.ascontiguousarray(b, dtype=np.int64)
    out = np.zeros(1 << logn, dtype=np.int64)
    lib().orc_negacyclic_mul_i64(_p(a), _p(b), _p(out), logn)
    return out


def automorphism_i64(a: np.ndarray, logn: int, k: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int64)
    out = np.zeros(1 << logn, dtype=np.int64)
    lib().orc_automorphism_i64(_p(a), _p(out), logn, k)
    return out
