"""CPU-side checks of libfdsc: the library loads, exports every entry point
declared in include/fdsc.h, and its host-side parameter / layout / sampler
logic agrees with the oracle (no GPU needed: these calls touch no device)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_2003_05328_gb300 import build

    build.build()
    from paper_2003_05328_gb300 import fdsc

    return fdsc


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fdsc_\w+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_entry_point(F):
    lib = C.CDLL(F.LIB_PATH)
    names = declared_entry_points()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding covers them all
    assert set(names) <= set(F.EXPORTS), set(names) - set(F.EXPORTS)


@pytest.mark.parametrize("n,p", [(1024, 65537), (2048, 65537), (4096, 65537), (2048, 12289), (4096, 12289),
                                 (64, 65537), (256, 12289), (2048, 147457), (4096, 786433)])
def test_params_query_matches_oracle(F, n, p):
    info = F.params_query(n, p)
    ref = O.params(n, p)
    for k in ("n", "p", "S", "d", "g_p", "psi_p", "q", "g_q", "psi_q", "delta", "r_q"):
        assert getattr(info, k) == getattr(ref, k), k


def test_params_query_rejects(F):
    for n, p in [(1000, 65537), (8192, 65537), (2048, 65535), (2048, 7), (2048, 1 << 21)]:
        with pytest.raises(F.FdscError) as e:
            F.params_query(n, p)
        assert e.value.code == -1


@pytest.mark.parametrize("n,p,shape", [
    (2048, 65537, (1, 64, 64, 32, 32, 2, 1)),
    (2048, 65537, (16, 128, 128, 16, 16, 8, 1)),
    (4096, 65537, (16, 256, 256, 8, 8, 64, 1)),
    (4096, 65537, (16, 256, 256, 8, 8, 16, 4)),
    (4096, 12289, (8, 128, 128, 64, 64, 1, 1)),
    (256, 65537, (3, 5, 3, 8, 8, 2, 2)),
    (1024, 65537, (2, 3, 2, 64, 64, 1, 1)),
])
def test_layout_matches_oracle(F, n, p, shape):
    B, Ci, Co, H, W, g_c, g_b = shape
    lay = F.layout_query(n, p, F.LayerSpec(B, Ci, Co, H, W, g_c, g_b))
    OP = O.params(n, p)
    ref = O.layer(OP, B, Ci, Co, H, W, g_c, g_b)
    for k in ("HW", "T", "GB", "beta", "n_in", "n_out"):
        assert getattr(lay, k) == getattr(ref, k), k
    # one filter word per group of d evaluation indices (w_0(x^d) plaintexts)
    assert lay.ct_in_words == ref.n_in * 2 * n and lay.filter_words == Co * ref.T * ref.beta * n // OP.d


def test_layout_rejects_bad_packing(F):
    with pytest.raises(F.FdscError):
        F.layout_query(2048, 65537, F.LayerSpec(1, 64, 64, 32, 32, 4, 1))  # 4 blocks of 1024 > S
    with pytest.raises(F.FdscError):
        F.layout_query(1024, 65537, F.LayerSpec(1, 4, 4, 64, 64, 2, 1))  # HW > S needs g_c = 1
    with pytest.raises(F.FdscError):
        F.layout_query(2048, 65537, F.LayerSpec(0, 4, 4, 16, 16, 1, 1))  # empty batch
    with pytest.raises(F.FdscError):
        F.layout_query(2048, 65537, F.LayerSpec(1, 4, 4, 12, 16, 1, 1))  # not a power of two


def test_gauss_table_matches_oracle(F):
    assert np.array_equal(F.gauss_table(), O.cdt())


@pytest.mark.parametrize("n,p,T", [(1024, 65537, 1), (2048, 65537, 32), (4096, 12289, 128), (2048, 65537, 64)])
def test_flood_bits_max_matches_oracle_bound(F, n, p, T):
    """The largest admissible HomShare flooding (host arithmetic, no GPU)
    against the oracle's independent noise bound."""
    P = O.params(n, p)
    f = F.flood_bits_max(n, p, T)
    assert O.noise_ok(P, T, f) and not O.noise_ok(P, T, f + 1)


@pytest.mark.parametrize("n,p,shape", [
    (2048, 65537, (1, 64, 64, 32, 32, 2, 1)),
    (4096, 12289, (8, 128, 128, 64, 64, 1, 1)),
    (256, 65537, (5, 34, 130, 8, 8, 1, 1)),
])
def test_filter_tc_words(F, n, p, shape):
    """Size of the tensor-core filter layout: per group of d evaluation
    indices (one filter value each) and block of 16 input ciphertexts, 8 fp16
    digit planes of 16 values for every row, the rows of the last
    128-channel tile rounded up to a multiple of 8."""
    B, Ci, Co, H, W, g_c, g_b = shape
    L = F.LayerSpec(B, Ci, Co, H, W, g_c, g_b)
    OP = O.params(n, p)
    ref = O.layer(OP, B, Ci, Co, H, W, g_c, g_b)
    co_pad = 128 * ((Co - 1) // 128) + -(-(Co - 128 * ((Co - 1) // 128)) // 8) * 8
    assert F.filter_tc_words(n, p, L) * 8 == ref.beta * (n // OP.d) * (-(-ref.T // 16)) * co_pad * 8 * 16 * 2


def test_filter_tc_rejects_large_T(F):
    with pytest.raises(F.FdscError) as e:  # T = 129 > 128: a diagonal could reach 2^24
        F.filter_tc_words(256, 65537, F.LayerSpec(1, 129, 4, 8, 8, 1, 1))
    assert e.value.code == -5
