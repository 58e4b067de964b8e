"""Python binding of libfdsc (argument marshalling only).

Every function here forwards to the entry point of the same name in
``include/fdsc.h``: it checks shapes and dtypes, allocates outputs with
PyTorch when the caller gives none, and passes raw device pointers and the
current CUDA stream.  All arithmetic runs in the CUDA kernels of libfdsc;
there is no CPU path, and every call raises if the library is missing or
returns an error.

Dtype mapping: Z_p data (uint32 in the C ABI) travels in torch.int32
tensors and Z_q data (uint64) in torch.int64 tensors; every value is
non-negative and below 2^60, so the bit patterns are identical.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfdsc.so")

FDSC_OK = 0
ERR_NAMES = {-1: "FDSC_ERR_ARG", -2: "FDSC_ERR_NOISE", -3: "FDSC_ERR_OOM", -4: "FDSC_ERR_CUDA",
             -5: "FDSC_ERR_UNSUPPORTED", -6: "FDSC_ERR_TIMEOUT", -7: "FDSC_ERR_BUDGET"}


class FdscError(RuntimeError):
    def __init__(self, code: int, fn: str, msg: str):
        super().__init__(f"{fn}: {ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class ParamsInfo(C.Structure):
    _fields_ = [(k, C.c_uint32) for k in ("n", "logn", "p", "S", "logS", "d", "g_p", "psi_p")] + \
               [(k, C.c_uint64) for k in ("q", "g_q", "psi_q", "delta", "r_q")]


class Layer(C.Structure):
    _fields_ = [(k, C.c_uint32) for k in ("B", "Ci", "Co", "H", "W", "g_c", "g_b")]


class Layout(C.Structure):
    _fields_ = [(k, C.c_uint32) for k in ("HW", "T", "GB", "beta", "n_in", "n_out")] + \
               [(k, C.c_uint64) for k in ("ct_in_words", "ct_out_words", "filter_words", "mask_words",
                                          "in_spectra_words", "out_spectra_words")]


_vp = C.c_void_p
_PI = C.POINTER(ParamsInfo)
_PL = C.POINTER(Layer)
_PO = C.POINTER(Layout)
_SIGS = {
    "fdsc_last_error": (C.c_char_p, []),
    "fdsc_params_query": (C.c_int, [C.c_uint32, C.c_uint32, _PI]),
    "fdsc_params_create": (C.c_int, [C.c_uint32, C.c_uint32, C.c_uint32, C.POINTER(_vp)]),
    "fdsc_params_destroy": (C.c_int, [_vp]),
    "fdsc_params_get_info": (C.c_int, [_vp, _PI]),
    "fdsc_gauss_table": (C.c_int, [_vp]),
    "fdsc_layout_query": (C.c_int, [C.c_uint32, C.c_uint32, _PL, _PO]),
    "fdsc_ntt2d": (C.c_int, [_vp, C.c_uint32, C.c_uint32, _vp, _vp, C.c_uint64, _vp]),
    "fdsc_intt2d": (C.c_int, [_vp, C.c_uint32, C.c_uint32, _vp, _vp, C.c_uint64, _vp]),
    "fdsc_pool2x2_sum": (C.c_int, [_vp, C.c_uint32, C.c_uint32, _vp, _vp, C.c_uint64, _vp]),
    "fdsc_keygen": (C.c_int, [_vp, C.c_uint64, _vp, _vp]),
    "fdsc_filter_prepare": (C.c_int, [_vp, _PL, _vp, C.c_uint32, C.c_uint32, _vp, _vp]),
    "fdsc_mask_prepare": (C.c_int, [_vp, _PL, C.c_uint64, _vp, _vp, _vp]),
    "fdsc_mask_prepare_flooded": (C.c_int, [_vp, _PL, C.c_uint64, C.c_uint32, _vp, _vp, _vp]),
    "fdsc_flood_bits_max": (C.c_int, [C.c_uint32, C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32)]),
    "fdsc_encrypt": (C.c_int, [_vp, _PL, _vp, _vp, C.c_uint64, _vp, _vp]),
    "fdsc_homrec": (C.c_int, [_vp, _PL, _vp, _vp, _vp]),
    "fdsc_homconv": (C.c_int, [_vp, _PL, _vp, _vp, _vp, _vp, _vp]),
    "fdsc_decrypt": (C.c_int, [_vp, _PL, _vp, _vp, _vp, _vp]),
    "fdsc_set_homconv_variant": (C.c_int, [C.c_int]),
    "fdsc_set_launch_overlap": (C.c_int, [C.c_int]),
    "fdsc_set_decrypt_pair": (C.c_int, [C.c_int]),
    "fdsc_calibrate": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "fdsc_encrypt_constants": (C.c_int, [_vp, _PL, _vp, C.c_uint64, _vp, _vp]),
    "fdsc_encode_share": (C.c_int, [_vp, _PL, _vp, _vp, _vp]),
    "fdsc_homrec_share": (C.c_int, [_vp, _PL, _vp, _vp, _vp]),
    "fdsc_online_produce": (C.c_int, [_vp, _PL, _vp, C.c_uint64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fdsc_homconv_sum": (C.c_int, [_vp, _PL, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fdsc_filter_tc_words": (C.c_int, [C.c_uint32, C.c_uint32, _PL, C.POINTER(C.c_uint64)]),
    "fdsc_filter_tc": (C.c_int, [_vp, _PL, _vp, _vp, _vp]),
    "fdsc_homconv_tc": (C.c_int, [_vp, _PL, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fdsc_homconv_tc_status": (C.c_int, [C.POINTER(C.c_uint32)]),
    "fdsc_encrypt_constants_seeded": (C.c_int, [_vp, _PL, _vp, C.c_uint64, _vp, _vp]),
    "fdsc_homconv_seeded": (C.c_int, [_vp, _PL, C.c_uint64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fdsc_decrypt_share": (C.c_int, [_vp, _PL, _vp, _vp, _vp, _vp]),
    "fdsc_encrypt_constants_multi": (C.c_int, [_vp, _PL, _vp, C.c_uint64, _vp, _vp, _vp]),
    "fdsc_mask_prepare_multi": (C.c_int, [_vp, _PL, _vp, _vp, _vp, _vp]),
    "fdsc_decrypt_share_multi": (C.c_int, [_vp, _PL, _vp, C.c_uint64, _vp, _vp, _vp]),
    "fdsc_plan_create": (C.c_int, [_vp, C.c_uint32, C.c_uint32, _vp, C.POINTER(_vp)]),
    "fdsc_plan_launch": (C.c_int, [_vp, _vp]),
    "fdsc_plan_layer_info_get": (C.c_int, [_vp, C.c_uint32, _vp]),
    "fdsc_plan_destroy": (C.c_int, [_vp]),
    "fdsc_server_create": (C.c_int, [_vp, C.POINTER(_vp)]),
    "fdsc_server_add_type": (C.c_int, [_vp, _vp, _PL, _vp, C.c_uint32, C.c_uint32, _vp, C.c_uint32,
                                       C.POINTER(C.c_uint32)]),
    "fdsc_server_start": (C.c_int, [_vp]),
    "fdsc_server_submit": (C.c_int, [_vp, _vp, C.POINTER(C.c_uint64)]),
    "fdsc_server_wait": (C.c_int, [_vp, C.c_uint64, C.c_uint32, C.POINTER(C.c_double)]),
    "fdsc_server_stats_get": (C.c_int, [_vp, _vp]),
    "fdsc_server_destroy": (C.c_int, [_vp]),
    "fdsc_layer_online_noalloc": (C.c_int, [_vp, _PL, _vp, C.c_uint64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
}
# entry points declared in include/fdsc.h (checked against the library's exports by the tests)
EXPORTS = tuple(_SIGS)

_lib = None


def lib() -> C.CDLL:
    """Load libfdsc.so (built by ``paper_2003_05328_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2003_05328_gb300.build.build()")
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype, f.argtypes = res, args
        _lib = h
    return _lib


def _call(name: str, *args) -> None:
    rc = getattr(lib(), name)(*args)
    if rc != FDSC_OK:
        raise FdscError(rc, name, (lib().fdsc_last_error() or b"").decode())


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor, dtype, numel: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


# ---------------------------------------------------------------- parameters
def params_query(n: int, p: int) -> ParamsInfo:
    info = ParamsInfo()
    _call("fdsc_params_query", n, p, C.byref(info))
    return info


def layout_query(n: int, p: int, layer: "LayerSpec") -> Layout:
    out = Layout()
    _call("fdsc_layout_query", n, p, C.byref(layer.c()), C.byref(out))
    return out


def gauss_table():
    import numpy as np

    out = np.zeros(19, np.uint64)
    _call("fdsc_gauss_table", out.ctypes.data)
    return out


class Params:
    """Owner of an ``fdsc_params`` object created on the current device."""

    def __init__(self, n: int, p: int, max_T: int = 256):
        h = _vp()
        _call("fdsc_params_create", n, p, max_T, C.byref(h))
        self.handle = h
        self.device = torch.cuda.current_device()
        self.info = ParamsInfo()
        _call("fdsc_params_get_info", h, C.byref(self.info))

    @property
    def n(self):
        return self.info.n

    @property
    def p(self):
        return self.info.p

    def close(self):
        if self.handle:
            lib().fdsc_params_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass(frozen=True)
class LayerSpec:
    B: int
    Ci: int
    Co: int
    H: int
    W: int
    g_c: int = 1
    g_b: int = 1

    def c(self) -> Layer:
        return Layer(self.B, self.Ci, self.Co, self.H, self.W, self.g_c, self.g_b)


def layout(P: Params, L: LayerSpec) -> Layout:
    return layout_query(P.n, P.p, L)


# ---------------------------------------------------------------- transforms
def _ntt2d(name, P, x, out, stream):
    H, W = x.shape[-2:]
    planes = x.numel() // (H * W)
    if out is None:
        out = torch.empty_like(x)
    _call(name, P.handle, H, W, _ptr(x, torch.int32, x.numel(), "x"), _ptr(out, torch.int32, x.numel(), "out"),
          planes, _stream(stream))
    return out


def ntt2d(P: Params, x: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """Cyclic NTT2D mod p of int32 [..., H, W] planes (Eq. 12, 2-D)."""
    return _ntt2d("fdsc_ntt2d", P, x, out, stream)


def intt2d(P: Params, X: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    return _ntt2d("fdsc_intt2d", P, X, out, stream)


def pool2x2_sum(P: Params, x: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """2 x 2 sum pooling mod p of a share [..., H, W] -> [..., H/2, W/2]."""
    H, W = x.shape[-2], x.shape[-1]
    planes = x.numel() // (H * W)
    if out is None:
        out = torch.empty(x.shape[:-2] + (H // 2, W // 2), dtype=torch.int32, device="cuda")
    _call("fdsc_pool2x2_sum", P.handle, H, W, _ptr(x, torch.int32, x.numel(), "x"),
          _ptr(out, torch.int32, planes * (H // 2) * (W // 2), "y"), planes, _stream(stream))
    return out


# ---------------------------------------------------------------- setup
def keygen(P: Params, seed: int, out=None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(P.n, dtype=torch.int64, device="cuda")
    _call("fdsc_keygen", P.handle, seed, _ptr(out, torch.int64, P.n, "t_hat"), _stream(stream))
    return out


def filter_prepare(P: Params, L: LayerSpec, w: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    lay = layout(P, L)
    Co, Ci, fh, fw = w.shape
    if (Co, Ci) != (L.Co, L.Ci):
        raise ValueError("filter shape does not match the layer")
    if out is None:
        out = torch.empty(lay.filter_words, dtype=torch.int64, device="cuda")
    _call("fdsc_filter_prepare", P.handle, C.byref(L.c()), _ptr(w, torch.int8, w.numel(), "w"), fh, fw,
          _ptr(out, torch.int64, lay.filter_words, "P_hat"), _stream(stream))
    return out


def mask_prepare(P: Params, L: LayerSpec, seed: int, M_hat=None, sB_hat=None, stream=None):
    lay = layout(P, L)
    if M_hat is None:
        M_hat = torch.empty(lay.mask_words, dtype=torch.int64, device="cuda")
    if sB_hat is None:
        sB_hat = torch.empty(lay.out_spectra_words, dtype=torch.int32, device="cuda")
    _call("fdsc_mask_prepare", P.handle, C.byref(L.c()), seed, _ptr(M_hat, torch.int64, lay.mask_words, "M_hat"),
          _ptr(sB_hat, torch.int32, lay.out_spectra_words, "sB_hat"), _stream(stream))
    return M_hat, sB_hat


def mask_prepare_flooded(P: Params, L: LayerSpec, seed: int, flood_bits: int, M_hat=None, sB_hat=None, stream=None):
    """HomShare masks with noise flooding of 2^flood_bits per coefficient."""
    lay = layout(P, L)
    if M_hat is None:
        M_hat = torch.empty(lay.mask_words, dtype=torch.int64, device="cuda")
    if sB_hat is None:
        sB_hat = torch.empty(lay.out_spectra_words, dtype=torch.int32, device="cuda")
    _call("fdsc_mask_prepare_flooded", P.handle, C.byref(L.c()), seed, flood_bits,
          _ptr(M_hat, torch.int64, lay.mask_words, "M_hat"), _ptr(sB_hat, torch.int32, lay.out_spectra_words, "sB_hat"),
          _stream(stream))
    return M_hat, sB_hat


def flood_bits_max(n: int, p: int, T: int) -> int:
    out = C.c_uint32(0)
    _call("fdsc_flood_bits_max", n, p, T, C.byref(out))
    return out.value


def set_homconv_variant(v: int) -> None:
    """Kernel variant for HomConv (0 automatic; results are identical)."""
    _call("fdsc_set_homconv_variant", v)


def calibrate(P: Params, which: int):
    """(ops/s, ops per clock per SM) of primitive `which`: 0 HomConv's exact
    MAC, 1 the 64-bit Shoup mulmod, 2 the 32-bit one."""
    a, b = C.c_double(0), C.c_double(0)
    _call("fdsc_calibrate", P.handle, which, C.byref(a), C.byref(b))
    return a.value, b.value


def set_launch_overlap(on: bool) -> bool:
    """Programmatic dependent launch of the online kernels (default off);
    returns the previous setting."""
    return bool(lib().fdsc_set_launch_overlap(1 if on else 0))


def set_decrypt_pair(on: bool) -> bool:
    """One image's decryption on CTA pairs (default on; off: one CTA per
    ciphertext, fewer instructions); returns the previous setting."""
    return bool(lib().fdsc_set_decrypt_pair(1 if on else 0))


# ---------------------------------------------------------------- online
def encrypt(P: Params, L: LayerSpec, t_hat, X, seed: int, out=None, stream=None) -> torch.Tensor:
    lay = layout(P, L)
    if out is None:
        out = torch.empty(lay.ct_in_words, dtype=torch.int64, device="cuda")
    _call("fdsc_encrypt", P.handle, C.byref(L.c()), _ptr(t_hat, torch.int64, P.n, "t_hat"),
          _ptr(X, torch.int32, lay.in_spectra_words, "X"), seed, _ptr(out, torch.int64, lay.ct_in_words, "ct"),
          _stream(stream))
    return out


def homrec(P: Params, L: LayerSpec, XB, ct, stream=None) -> torch.Tensor:
    lay = layout(P, L)
    _call("fdsc_homrec", P.handle, C.byref(L.c()), _ptr(XB, torch.int32, lay.in_spectra_words, "XB"),
          _ptr(ct, torch.int64, lay.ct_in_words, "ct"), _stream(stream))
    return ct


def homconv(P: Params, L: LayerSpec, ct_in, P_hat, M_hat=None, out=None, stream=None) -> torch.Tensor:
    lay = layout(P, L)
    if out is None:
        out = torch.empty(lay.ct_out_words, dtype=torch.int64, device="cuda")
    m = None if M_hat is None else _ptr(M_hat, torch.int64, lay.mask_words, "M_hat")
    _call("fdsc_homconv", P.handle, C.byref(L.c()), _ptr(ct_in, torch.int64, lay.ct_in_words, "ct_in"),
          _ptr(P_hat, torch.int64, lay.filter_words, "P_hat"), m, _ptr(out, torch.int64, lay.ct_out_words, "ct_out"),
          _stream(stream))
    return out


def decrypt(P: Params, L: LayerSpec, t_hat, ct, out=None, stream=None) -> torch.Tensor:
    lay = layout(P, L)
    if out is None:
        out = torch.empty(lay.out_spectra_words, dtype=torch.int32, device="cuda")
    _call("fdsc_decrypt", P.handle, C.byref(L.c()), _ptr(t_hat, torch.int64, P.n, "t_hat"),
          _ptr(ct, torch.int64, lay.ct_out_words, "ct"), _ptr(out, torch.int32, lay.out_spectra_words, "SA_hat"),
          _stream(stream))
    return out


# ---------------------------------------------------------------- fused online path
def encrypt_constants(P: Params, L: LayerSpec, t_hat, seed: int, out=None, stream=None) -> torch.Tensor:
    """Enc(0) in the NTT_q domain: the RLWE constants of one encryption."""
    lay = layout(P, L)
    if out is None:
        out = torch.empty(lay.ct_in_words, dtype=torch.int64, device="cuda")
    _call("fdsc_encrypt_constants", P.handle, C.byref(L.c()), _ptr(t_hat, torch.int64, P.n, "t_hat"), seed,
          _ptr(out, torch.int64, lay.ct_in_words, "ct"), _stream(stream))
    return out


def encode_share(P: Params, L: LayerSpec, x, out=None, stream=None) -> torch.Tensor:
    """NTT_q(Delta * encode(pack(NTT2D(x)))) for a spatial share x."""
    lay = layout(P, L)
    if out is None:
        out = torch.empty(lay.n_in * P.n, dtype=torch.int64, device="cuda")
    _call("fdsc_encode_share", P.handle, C.byref(L.c()), _ptr(x, torch.int32, lay.in_spectra_words, "x"),
          _ptr(out, torch.int64, lay.n_in * P.n, "A"), _stream(stream))
    return out


def online_produce(P: Params, L: LayerSpec, t_hat, seed: int, xA, xB, ct=None, A=None, R=None, P_hat=None,
                   M_hat=None, stream=None):
    """Encryption constants, Alice's and Bob's share encodings in one launch
    (the words of encrypt_constants, encode_share(xA), encode_share(xB));
    P_hat / M_hat, if given, are prefetched into L2 for the HomConv that
    follows.  Returns (ct, A, R)."""
    lay = layout(P, L)
    na = lay.n_in * P.n
    ct = torch.empty(lay.ct_in_words, dtype=torch.int64, device="cuda") if ct is None else ct
    A = torch.empty(na, dtype=torch.int64, device="cuda") if A is None else A
    R = torch.empty(na, dtype=torch.int64, device="cuda") if R is None else R
    ph = None if P_hat is None else _ptr(P_hat, torch.int64, lay.filter_words, "P_hat")
    mh = None if M_hat is None else _ptr(M_hat, torch.int64, lay.mask_words, "M_hat")
    _call("fdsc_online_produce", P.handle, C.byref(L.c()), _ptr(t_hat, torch.int64, P.n, "t_hat"), seed,
          _ptr(xA, torch.int32, lay.in_spectra_words, "xA"), _ptr(xB, torch.int32, lay.in_spectra_words, "xB"),
          _ptr(ct, torch.int64, lay.ct_in_words, "ct"), _ptr(A, torch.int64, na, "A"), _ptr(R, torch.int64, na, "R"),
          ph, mh, _stream(stream))
    return ct, A, R


def homrec_share(P: Params, L: LayerSpec, xB, ct, stream=None) -> torch.Tensor:
    lay = layout(P, L)
    _call("fdsc_homrec_share", P.handle, C.byref(L.c()), _ptr(xB, torch.int32, lay.in_spectra_words, "xB"),
          _ptr(ct, torch.int64, lay.ct_in_words, "ct"), _stream(stream))
    return ct


def homconv_sum(P: Params, L: LayerSpec, ct_in, A1, A2, P_hat, M_hat=None, out=None, stream=None) -> torch.Tensor:
    lay = layout(P, L)
    if out is None:
        out = torch.empty(lay.ct_out_words, dtype=torch.int64, device="cuda")
    na = lay.n_in * P.n
    a1 = None if A1 is None else _ptr(A1, torch.int64, na, "A1")
    a2 = None if A2 is None else _ptr(A2, torch.int64, na, "A2")
    m = None if M_hat is None else _ptr(M_hat, torch.int64, lay.mask_words, "M_hat")
    _call("fdsc_homconv_sum", P.handle, C.byref(L.c()), _ptr(ct_in, torch.int64, lay.ct_in_words, "ct_in"), a1, a2,
          _ptr(P_hat, torch.int64, lay.filter_words, "P_hat"), m, _ptr(out, torch.int64, lay.ct_out_words, "ct_out"),
          _stream(stream))
    return out


def filter_tc_words(n: int, p: int, L: LayerSpec) -> int:
    """Words of the digit-ready filter of the tensor-core HomConv (host only)."""
    out = C.c_uint64()
    _call("fdsc_filter_tc_words", n, p, C.byref(L.c()), C.byref(out))
    return out.value


def filter_tc(P: Params, L: LayerSpec, P_hat, out=None, stream=None) -> torch.Tensor:
    """P_hat [Co][T][beta][n] -> the tensor-core layout [beta n][ceil(T/16)][Co][16] (biased words)."""
    lay = layout(P, L)
    words = filter_tc_words(P.n, P.p, L)
    if out is None:
        out = torch.empty(words, dtype=torch.int64, device="cuda")
    _call("fdsc_filter_tc", P.handle, C.byref(L.c()), _ptr(P_hat, torch.int64, lay.filter_words, "P_hat"),
          _ptr(out, torch.int64, words, "P_tc"), _stream(stream))
    return out


def homconv_tc(P: Params, L: LayerSpec, ct_in, A1, A2, P_tc, M_hat=None, out=None, stream=None) -> torch.Tensor:
    """homconv_sum on the tensor cores (exact digit products, fp32 accumulation below 2^24)."""
    lay = layout(P, L)
    if out is None:
        out = torch.empty(lay.ct_out_words, dtype=torch.int64, device="cuda")
    na = lay.n_in * P.n
    a1 = None if A1 is None else _ptr(A1, torch.int64, na, "A1")
    a2 = None if A2 is None else _ptr(A2, torch.int64, na, "A2")
    m = None if M_hat is None else _ptr(M_hat, torch.int64, lay.mask_words, "M_hat")
    _call("fdsc_homconv_tc", P.handle, C.byref(L.c()), _ptr(ct_in, torch.int64, lay.ct_in_words, "ct_in"), a1, a2,
          _ptr(P_tc, torch.int64, filter_tc_words(P.n, P.p, L), "P_tc"), m,
          _ptr(out, torch.int64, lay.ct_out_words, "ct_out"), _stream(stream))
    return out


def homconv_tc_status() -> int:
    """0 if no tensor-core HomConv CTA gave up a bounded wait since the last call (raises otherwise)."""
    code = C.c_uint32()
    _call("fdsc_homconv_tc_status", C.byref(code))
    return code.value


def encrypt_constants_seeded(P: Params, L: LayerSpec, t_hat, seed: int, out=None, stream=None) -> torch.Tensor:
    """c1 of Enc(0) alone ([n_in][n]): the seeded ciphertext form."""
    lay = layout(P, L)
    if out is None:
        out = torch.empty(lay.n_in * P.n, dtype=torch.int64, device="cuda")
    _call("fdsc_encrypt_constants_seeded", P.handle, C.byref(L.c()), _ptr(t_hat, torch.int64, P.n, "t_hat"), seed,
          _ptr(out, torch.int64, lay.n_in * P.n, "c1"), _stream(stream))
    return out


def homconv_seeded(P: Params, L: LayerSpec, seed: int, c1, A1, A2, P_hat, M_hat=None, out=None,
                   stream=None) -> torch.Tensor:
    """homconv_sum on seeded ciphertexts: c0 drawn again from the encryption seed."""
    lay = layout(P, L)
    if out is None:
        out = torch.empty(lay.ct_out_words, dtype=torch.int64, device="cuda")
    na = lay.n_in * P.n
    a1 = None if A1 is None else _ptr(A1, torch.int64, na, "A1")
    a2 = None if A2 is None else _ptr(A2, torch.int64, na, "A2")
    m = None if M_hat is None else _ptr(M_hat, torch.int64, lay.mask_words, "M_hat")
    _call("fdsc_homconv_seeded", P.handle, C.byref(L.c()), seed, _ptr(c1, torch.int64, na, "c1"), a1, a2,
          _ptr(P_hat, torch.int64, lay.filter_words, "P_hat"), m, _ptr(out, torch.int64, lay.ct_out_words, "ct_out"),
          _stream(stream))
    return out


def decrypt_share(P: Params, L: LayerSpec, t_hat, ct, out=None, stream=None) -> torch.Tensor:
    """Decrypt, decode, fold and INTT2D: Alice's spatial share int32 [B][Co][H][W]."""
    lay = layout(P, L)
    if out is None:
        out = torch.empty((L.B, L.Co, L.H, L.W), dtype=torch.int32, device="cuda")
    _call("fdsc_decrypt_share", P.handle, C.byref(L.c()), _ptr(t_hat, torch.int64, P.n, "t_hat"),
          _ptr(ct, torch.int64, lay.ct_out_words, "ct"), _ptr(out, torch.int32, lay.out_spectra_words, "y"),
          _stream(stream))
    return out


# ---------------------------------------------------------------- several clients in one call
def encrypt_constants_multi(P: Params, L: LayerSpec, t_hats, seeds, key_stride=None, out=None, stream=None):
    """Enc(0) with a key and a seed per image group (t_hats [GB][n] or one key, seeds int64 [GB] on the device)."""
    lay = layout(P, L)
    if key_stride is None:
        key_stride = P.n if t_hats.numel() > P.n else 0
    if out is None:
        out = torch.empty(lay.ct_in_words, dtype=torch.int64, device="cuda")
    _call("fdsc_encrypt_constants_multi", P.handle, C.byref(L.c()), _ptr(t_hats, torch.int64, t_hats.numel(), "t_hats"),
          key_stride, _ptr(seeds, torch.int64, lay.GB, "seeds"), _ptr(out, torch.int64, lay.ct_in_words, "ct"),
          _stream(stream))
    return out


def mask_prepare_multi(P: Params, L: LayerSpec, seeds, M_hat=None, sB_hat=None, stream=None):
    lay = layout(P, L)
    if M_hat is None:
        M_hat = torch.empty(lay.mask_words, dtype=torch.int64, device="cuda")
    if sB_hat is None:
        sB_hat = torch.empty(lay.out_spectra_words, dtype=torch.int32, device="cuda")
    _call("fdsc_mask_prepare_multi", P.handle, C.byref(L.c()), _ptr(seeds, torch.int64, lay.GB, "seeds"),
          _ptr(M_hat, torch.int64, lay.mask_words, "M_hat"), _ptr(sB_hat, torch.int32, lay.out_spectra_words, "sB_hat"),
          _stream(stream))
    return M_hat, sB_hat


def decrypt_share_multi(P: Params, L: LayerSpec, t_hats, ct, key_stride=None, out=None, stream=None):
    lay = layout(P, L)
    if key_stride is None:
        key_stride = P.n if t_hats.numel() > P.n else 0
    if out is None:
        out = torch.empty((L.B, L.Co, L.H, L.W), dtype=torch.int32, device="cuda")
    _call("fdsc_decrypt_share_multi", P.handle, C.byref(L.c()), _ptr(t_hats, torch.int64, t_hats.numel(), "t_hats"),
          key_stride, _ptr(ct, torch.int64, lay.ct_out_words, "ct"), _ptr(out, torch.int32, lay.out_spectra_words, "y"),
          _stream(stream))
    return out


# ---------------------------------------------------------------- batched plan
class PlanLayerC(C.Structure):
    _fields_ = [("params", _vp), ("layer", Layer), ("fh", C.c_uint32), ("fw", C.c_uint32), ("w", _vp),
                ("t_hat", _vp), ("enc_seed", C.c_uint64), ("mask_seed", C.c_uint64), ("xA", _vp), ("xB", _vp),
                ("yA", _vp), ("yB", _vp), ("pA", _vp), ("pB", _vp), ("flood_bits", C.c_uint32),
                ("pad0", C.c_uint32)]


class PlanLayerInfo(C.Structure):
    _fields_ = [(k, C.c_uint32) for k in ("g_c", "g_b", "homconv_variant", "fused", "candidates", "pad0")] + \
               [("tuned_step_us", C.c_double)]


PLAN_TUNE = 1
PLAN_CHAIN = 2
PLAN_TENSOR = 4


class Plan:
    """Many layers' online paths recorded as one CUDA graph (setup at creation).

    ``layers``: dicts with keys params, layer (LayerSpec; g_c = 0 lets the plan
    choose), w (int8 [Co][Ci][fh][fw]), t_hat, enc_seed, mask_seed, xA, xB, yA,
    yB (device tensors)."""

    def __init__(self, layers, tune=False, stream=None, chain=False, tensor=False):
        arr = (PlanLayerC * len(layers))()
        self._keep = layers
        for i, d in enumerate(layers):
            L, w = d["layer"], d["w"]
            Co, Ci, fh, fw = w.shape
            arr[i] = PlanLayerC(d["params"].handle, L.c(), fh, fw, _ptr(w, torch.int8, w.numel(), "w"),
                                _ptr(d["t_hat"], torch.int64, d["params"].n, "t_hat"), d["enc_seed"], d["mask_seed"],
                                d["xA"].data_ptr(), d["xB"].data_ptr(), d["yA"].data_ptr(), d["yB"].data_ptr(),
                                d["pA"].data_ptr() if d.get("pA") is not None else None,
                                d["pB"].data_ptr() if d.get("pB") is not None else None,
                                d.get("flood_bits", 0), 0)
        h = _vp()
        flags = (PLAN_TUNE if tune else 0) | (PLAN_CHAIN if chain else 0) | (PLAN_TENSOR if tensor else 0)
        _call("fdsc_plan_create", C.addressof(arr), len(layers), flags, _stream(stream), C.byref(h))
        self.handle = h

    def launch(self, stream=None):
        _call("fdsc_plan_launch", self.handle, _stream(stream))

    def info(self, i) -> PlanLayerInfo:
        out = PlanLayerInfo()
        _call("fdsc_plan_layer_info_get", self.handle, i, C.byref(out))
        return out

    def close(self):
        if self.handle:
            lib().fdsc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving
class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_batch", C.c_uint32), ("lanes", C.c_uint32)]


class Request(C.Structure):
    _fields_ = [("type", C.c_uint32), ("key", C.c_uint32), ("enc_seed", C.c_uint64), ("mask_seed", C.c_uint64),
                ("xA", _vp), ("xB", _vp), ("yA", _vp), ("yB", _vp)]


class ServerStats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("submitted", "completed", "batches", "peak_inflight_bytes")] + \
               [(k, C.c_double) for k in ("mean_batch", "p50_us", "p99_us", "mean_us", "max_us")] + \
               [("tensor_batches", C.c_uint64), ("reserved_bytes", C.c_uint64), ("lanes", C.c_uint32),
                ("lane_capacity", C.c_uint32)]


class Server:
    """Continuous-batching server (a scheduling thread inside libfdsc).
    Request buffers are host numpy arrays (uint32) kept alive by the caller
    until the request is done."""

    def __init__(self, hbm_budget_bytes, max_batch=16, lanes=4):
        cfg = ServerConfig(hbm_budget_bytes, max_batch, lanes)
        h = _vp()
        _call("fdsc_server_create", C.byref(cfg), C.byref(h))
        self.handle = h
        self._keep = []

    def add_type(self, P: Params, L: LayerSpec, w, keys) -> int:
        Co, Ci, fh, fw = w.shape
        tid = C.c_uint32()
        nkeys = keys.numel() // P.n
        self._keep += [w, keys]
        _call("fdsc_server_add_type", self.handle, P.handle, C.byref(L.c()), _ptr(w, torch.int8, w.numel(), "w"), fh,
              fw, _ptr(keys, torch.int64, keys.numel(), "keys"), nkeys, C.byref(tid))
        return tid.value

    def start(self):
        _call("fdsc_server_start", self.handle)

    def submit(self, type_id, key, enc_seed, mask_seed, xA, xB, yA, yB) -> int:
        r = Request(type_id, key, enc_seed, mask_seed, xA.ctypes.data, xB.ctypes.data, yA.ctypes.data,
                    yB.ctypes.data)
        t = C.c_uint64()
        _call("fdsc_server_submit", self.handle, C.byref(r), C.byref(t))
        return t.value

    def wait(self, ticket, timeout_ms=60000) -> float:
        lat = C.c_double()
        _call("fdsc_server_wait", self.handle, ticket, timeout_ms, C.byref(lat))
        return lat.value

    def stats(self) -> ServerStats:
        out = ServerStats()
        _call("fdsc_server_stats_get", self.handle, C.byref(out))
        return out

    def close(self):
        if self.handle:
            lib().fdsc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- one layer, no device allocation
def layer_online_noalloc(P: Params, L: LayerSpec, t_hat, enc_seed: int, P_hat, M_hat, sB_hat, xA, xB, yA, yB,
                         stream=None) -> None:
    """The fused online path of one layer with its intermediate ciphertexts
    in the library's fixed device array: for callers that must not allocate
    device memory (the outputs yA, yB are the caller's buffers)."""
    lay = layout(P, L)
    _call("fdsc_layer_online_noalloc", P.handle, C.byref(L.c()), _ptr(t_hat, torch.int64, P.n, "t_hat"), enc_seed,
          _ptr(P_hat, torch.int64, lay.filter_words, "P_hat"), _ptr(M_hat, torch.int64, lay.mask_words, "M_hat"),
          _ptr(sB_hat, torch.int32, lay.out_spectra_words, "sB_hat"),
          _ptr(xA, torch.int32, lay.in_spectra_words, "xA"), _ptr(xB, torch.int32, lay.in_spectra_words, "xB"),
          _ptr(yA, torch.int32, lay.out_spectra_words, "yA"), _ptr(yB, torch.int32, lay.out_spectra_words, "yB"),
          _stream(stream))
