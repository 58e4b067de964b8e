"""CPU oracle for the FDSC hot path -- TEST INFRASTRUCTURE ONLY.

A thin ctypes/numpy front end over ``fdsc_oracle.c`` (plain C, exact integer
arithmetic, single-threaded).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module; the product
library under ``paper_2003_05328_gb300/`` never does and shares no code with
it.  Every function is pinned by CPU tests against the paper's printed
parameters, closed forms, brute force or library routines.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "fdsc_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, no tuning)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fdsc_oracle.h")))
    if force or stale:
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [("n", C.c_uint32), ("logn", C.c_uint32), ("p", C.c_uint32), ("S", C.c_uint32),
                ("logS", C.c_uint32), ("d", C.c_uint32), ("g_p", C.c_uint32), ("psi_p", C.c_uint32),
                ("pad0", C.c_uint32), ("q", C.c_uint64), ("g_q", C.c_uint64), ("psi_q", C.c_uint64),
                ("delta", C.c_uint64), ("r_q", C.c_uint64)]


class Layer(C.Structure):
    _fields_ = [(k, C.c_uint32) for k in ("B", "Ci", "Co", "H", "W", "g_c", "g_b", "HW", "T", "GB",
                                          "beta", "n_in", "n_out")]


_P = C.POINTER(Params)
_L = C.POINTER(Layer)
_u32p = C.POINTER(C.c_uint32)
_u64p = C.POINTER(C.c_uint64)
_i64p = C.POINTER(C.c_int64)
_i8p = C.POINTER(C.c_int8)

_SIGS = {
    "orc_set_tier": (None, [C.c_int]),
    "orc_get_tier": (C.c_int, []),
    "orc_is_prime": (C.c_int, [C.c_uint64]),
    "orc_powmod": (C.c_uint64, [C.c_uint64, C.c_uint64, C.c_uint64]),
    "orc_primitive_root": (C.c_uint64, [C.c_uint64]),
    "orc_min_prime_1mod": (C.c_uint64, [C.c_uint64, C.c_uint64]),
    "orc_find_q": (C.c_uint64, [C.c_uint32]),
    "orc_brv": (C.c_uint32, [C.c_uint32, C.c_uint32]),
    "orc_params_init": (C.c_int, [C.c_uint32, C.c_uint32, _P]),
    "orc_layer_init": (C.c_int, [_P] + [C.c_uint32] * 7 + [_L]),
    "orc_noise_bound_log2": (C.c_double, [_P, C.c_uint32]),
    "orc_noise_ok": (C.c_int, [_P, C.c_uint32]),
    "orc_noise_ok_flood": (C.c_int, [_P, C.c_uint32, C.c_uint32]),
    "orc_rng": (C.c_uint64, [C.c_uint64, C.c_uint64, C.c_uint64]),
    "orc_cdt": (None, [_u64p]),
    "orc_gauss": (C.c_int64, [C.c_uint64, _u64p]),
    "orc_uniform_q": (C.c_uint64, [_P, C.c_uint64, C.c_uint64]),
    "orc_uniform_p": (C.c_uint32, [C.c_uint32, C.c_uint64]),
    "orc_ntt2d": (None, [C.c_uint32, C.c_uint32, C.c_uint32, _u32p, _u32p, C.c_uint64, C.c_int]),
    "orc_slot_decode": (None, [_P, _u32p, _u32p]),
    "orc_slot_encode": (None, [_P, _u32p, _u32p]),
    "orc_ntt_q": (None, [_P, _u64p, _u64p]),
    "orc_intt_q": (None, [_P, _u64p, _u64p]),
    "orc_keygen": (None, [_P, C.c_uint64, _i64p, _u64p]),
    "orc_pack_input": (None, [_P, _L, _u32p, _u32p]),
    "orc_encrypt": (None, [_P, _L, _u64p, _u32p, C.c_uint64, _u64p]),
    "orc_homrec": (None, [_P, _L, _u64p, _u32p]),
    "orc_filter_spectra": (None, [_P, _L, _i8p, C.c_uint32, C.c_uint32, _u32p]),
    "orc_filter_prepare": (None, [_P, _L, _i8p, C.c_uint32, C.c_uint32, _u64p]),
    "orc_mask_prepare": (None, [_P, _L, C.c_uint64, _u64p, _u32p]),
    "orc_mask_prepare_flooded": (None, [_P, _L, C.c_uint64, C.c_uint32, _u64p, _u32p]),
    "orc_homconv": (None, [_P, _L, _u64p, _u64p, _u64p, _u64p]),
    "orc_decrypt": (None, [_P, _L, _u64p, _u64p, _u32p, _i64p]),
    "orc_decrypt_raw": (None, [_P, _u64p, _u64p, _u32p, _i64p]),
    "orc_conv_plain": (None, [C.c_uint32] * 6 + [_u32p, _i8p, C.c_uint32, C.c_uint32, _u32p]),
    "orc_pool2x2_sum": (None, [C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32, _u32p, _u32p]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            h = C.CDLL(build())
            for name, (res, args) in _SIGS.items():
                f = getattr(h, name)
                f.restype, f.argtypes = res, args
            _lib = h
    return _lib


def _ptr(a: np.ndarray | None, ct):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ct)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


class tier:
    """Context manager selecting the transform tier (0 = O(N^2) definition)."""

    def __init__(self, t: int):
        self.t, self.old = t, None

    def __enter__(self):
        self.old = lib().orc_get_tier()
        lib().orc_set_tier(self.t)

    def __exit__(self, *a):
        lib().orc_set_tier(self.old)


def params(n: int, p: int) -> Params:
    P = Params()
    if lib().orc_params_init(n, p, C.byref(P)) != 0:
        raise ValueError(f"unsupported (n, p) = ({n}, {p})")
    return P


def layer(P: Params, B, Ci, Co, H, W, g_c=None, g_b=1) -> Layer:
    HW = H * W
    if g_c is None:
        g_c = max(1, min(Ci, P.S // HW)) if HW <= P.S else 1
        while HW <= P.S and g_c * g_b * HW > P.S:
            g_c -= 1
    L = Layer()
    if lib().orc_layer_init(C.byref(P), B, Ci, Co, H, W, g_c, g_b, C.byref(L)) != 0:
        raise ValueError("unsupported layer / packing")
    return L


def noise_bound_log2(P, T):
    return lib().orc_noise_bound_log2(C.byref(P), T)


def noise_ok(P, T, flood_bits=0):
    return bool(lib().orc_noise_ok_flood(C.byref(P), T, flood_bits))


def rng(seed, domain, idx):
    return int(lib().orc_rng(seed, domain, idx))


def cdt():
    out = np.zeros(19, np.uint64)
    lib().orc_cdt(_ptr(out, _u64p))
    return out


def gauss(r, table=None):
    table = cdt() if table is None else _u64(table)
    return int(lib().orc_gauss(r, _ptr(table, _u64p)))


def uniform_q(P, r1, r2):
    return int(lib().orc_uniform_q(C.byref(P), r1, r2))


def uniform_p(p, r):
    return int(lib().orc_uniform_p(p, r))


def ntt2d(x, p, inverse=False):
    x = _u32(x)
    H, W = x.shape[-2:]
    out = np.empty_like(x)
    lib().orc_ntt2d(p, H, W, _ptr(x, _u32p), _ptr(out, _u32p), x.size // (H * W), int(inverse))
    return out


def slot_decode(P, m):
    m = _u32(m)
    s = np.empty(P.S, np.uint32)
    lib().orc_slot_decode(C.byref(P), _ptr(m, _u32p), _ptr(s, _u32p))
    return s


def slot_encode(P, s):
    s = _u32(s)
    m = np.empty(P.S, np.uint32)
    lib().orc_slot_encode(C.byref(P), _ptr(s, _u32p), _ptr(m, _u32p))
    return m


def ntt_q(P, a):
    a = _u64(a)
    out = np.empty(P.n, np.uint64)
    lib().orc_ntt_q(C.byref(P), _ptr(a, _u64p), _ptr(out, _u64p))
    return out


def intt_q(P, A):
    A = _u64(A)
    out = np.empty(P.n, np.uint64)
    lib().orc_intt_q(C.byref(P), _ptr(A, _u64p), _ptr(out, _u64p))
    return out


def keygen(P, seed):
    t = np.empty(P.n, np.int64)
    t_hat = np.empty(P.n, np.uint64)
    lib().orc_keygen(C.byref(P), seed, _ptr(t, _i64p), _ptr(t_hat, _u64p))
    return t, t_hat


def pack_input(P, L, X):
    X = _u32(X)
    out = np.empty((L.n_in, P.n), np.uint32)
    lib().orc_pack_input(C.byref(P), C.byref(L), _ptr(X, _u32p), _ptr(out, _u32p))
    return out


def encrypt(P, L, t_hat, X, seed):
    X, t_hat = _u32(X), _u64(t_hat)
    ct = np.empty((L.n_in, 2, P.n), np.uint64)
    lib().orc_encrypt(C.byref(P), C.byref(L), _ptr(t_hat, _u64p), _ptr(X, _u32p), seed, _ptr(ct, _u64p))
    return ct


def homrec(P, L, ct, XB):
    ct = _u64(ct).copy()
    XB = _u32(XB)
    lib().orc_homrec(C.byref(P), C.byref(L), _ptr(ct, _u64p), _ptr(XB, _u32p))
    return ct


def _check_filter(L, w):
    w = np.ascontiguousarray(w, dtype=np.int8)
    Co, Ci, fh, fw = w.shape
    if (Co, Ci) != (L.Co, L.Ci) or fh > L.H or fw > L.W:
        raise ValueError("filter shape does not match the layer")
    return w, fh, fw


def filter_spectra(P, L, w):
    w, fh, fw = _check_filter(L, w)
    out = np.empty((L.Co, L.Ci, L.HW), np.uint32)
    lib().orc_filter_spectra(C.byref(P), C.byref(L), _ptr(w, _i8p), fh, fw, _ptr(out, _u32p))
    return out


def filter_prepare(P, L, w):
    w, fh, fw = _check_filter(L, w)
    out = np.empty((L.Co * L.T * L.beta, P.n), np.uint64)
    lib().orc_filter_prepare(C.byref(P), C.byref(L), _ptr(w, _i8p), fh, fw, _ptr(out, _u64p))
    return out


def mask_prepare(P, L, seed, flood_bits=0):
    M = np.empty((L.n_out, P.n), np.uint64)
    sB = np.empty((L.B, L.Co, L.HW), np.uint32)
    lib().orc_mask_prepare_flooded(C.byref(P), C.byref(L), seed, flood_bits, _ptr(M, _u64p), _ptr(sB, _u32p))
    return M, sB


def homconv(P, L, ct_in, Phat, Mhat=None):
    ct_in, Phat = _u64(ct_in), _u64(Phat)
    Mhat = None if Mhat is None else _u64(Mhat)
    out = np.empty((L.n_out, 2, P.n), np.uint64)
    lib().orc_homconv(C.byref(P), C.byref(L), _ptr(ct_in, _u64p), _ptr(Phat, _u64p),
                      _ptr(Mhat, _u64p), _ptr(out, _u64p))
    return out


def decrypt(P, L, t_hat, ct):
    t_hat, ct = _u64(t_hat), _u64(ct)
    SA = np.empty((L.B, L.Co, L.HW), np.uint32)
    noise = np.empty(L.n_out, np.int64)
    lib().orc_decrypt(C.byref(P), C.byref(L), _ptr(t_hat, _u64p), _ptr(ct, _u64p), _ptr(SA, _u32p),
                      _ptr(noise, _i64p))
    return SA, noise


def decrypt_raw(P, t_hat, ct):
    t_hat, ct = _u64(t_hat), _u64(ct)
    m = np.empty(P.n, np.uint32)
    noise = C.c_int64(0)
    lib().orc_decrypt_raw(C.byref(P), _ptr(t_hat, _u64p), _ptr(ct, _u64p), _ptr(m, _u32p), C.byref(noise))
    return m, int(noise.value)


def conv_plain(p, x, w):
    x = _u32(x)
    w = np.ascontiguousarray(w, dtype=np.int8)
    B, Ci, H, W = x.shape
    Co, Ci2, fh, fw = w.shape
    assert Ci == Ci2
    y = np.empty((B, Co, H, W), np.uint32)
    lib().orc_conv_plain(p, B, Ci, Co, H, W, _ptr(x, _u32p), _ptr(w, _i8p), fh, fw, _ptr(y, _u32p))
    return y


def pool2x2_sum(p, x):
    """Appendix average pooling on a share (2x2 sum mod p): [..., H, W] -> [..., H/2, W/2]."""
    x = _u32(x)
    H, W = x.shape[-2:]
    planes = x.size // (H * W)
    y = np.empty(x.shape[:-2] + (H // 2, W // 2), np.uint32)
    lib().orc_pool2x2_sum(p, planes, H, W, _ptr(x, _u32p), _ptr(y, _u32p))
    return y


def round_trip(P, L, xA, xB, w, key_seed, enc_seed, srv_seed, with_homrec=True, flood_bits=0):
    """One FDSC layer (the one-layer protocol of Fig. 2, with HomRec of Bob's
    share, Eq. 3; optionally HomShare noise flooding): returns every stage
    boundary for parity checks."""
    H, W = L.H, L.W
    out = {}
    t, t_hat = keygen(P, key_seed)
    out["t_hat"] = t_hat
    XA = ntt2d(xA, P.p).reshape(L.B, L.Ci, L.HW)
    out["XA"] = XA
    ct = encrypt(P, L, t_hat, XA, enc_seed)
    out["ct_enc"] = ct
    if with_homrec:
        XB = ntt2d(xB, P.p).reshape(L.B, L.Ci, L.HW)
        out["XB"] = XB
        ct = homrec(P, L, ct, XB)
        out["ct_rec"] = ct
    Phat = filter_prepare(P, L, w)
    out["Phat"] = Phat
    Mhat, sB = mask_prepare(P, L, srv_seed, flood_bits)
    out["Mhat"], out["sB_hat"] = Mhat, sB
    ct_out = homconv(P, L, ct, Phat, Mhat)
    out["ct_out"] = ct_out
    SA, noise = decrypt(P, L, t_hat, ct_out)
    out["SA_hat"], out["noise"] = SA, noise
    out["yA"] = ntt2d(SA.reshape(L.B, L.Co, H, W), P.p, inverse=True)
    out["yB"] = ntt2d(sB.reshape(L.B, L.Co, H, W), P.p, inverse=True)
    return out
