"""The seeded synthetic inputs follow the stated recipe (CPU only): shares
uniform in [0, p) on the image support and zero on the padding, 4-bit
weights in [-8, 7] (or +-1 for the binarized layer), the same arrays for the
same seed and different ones for different streams."""
import numpy as np
import pytest

import fdsc_inputs as FI


@pytest.mark.parametrize("cfg", sorted(FI.CONFIGS))
def test_shares_and_weights_follow_the_recipe(cfg):
    c = FI.CONFIGS[cfg]
    for li, ls in enumerate(c.layers):
        B = min(ls.B, 2)  # the recipe does not depend on the batch; keep the arrays small
        ls2 = FI.LayerShape(B, ls.Ci, ls.Co, ls.H, ls.W, ls.fh, ls.fw, ls.n, ls.p, ls.h, ls.w, ls.binary)
        xA, xB = FI.shares(ls2, c.cid, li)
        h, w = ls2.support
        for x in (xA, xB):
            assert x.dtype == np.uint32 and x.shape == (B, ls.Ci, ls.H, ls.W)
            assert x.max() < ls.p and not x[:, :, h:, :].any() and not x[:, :, :, w:].any()
            body = x[:, :, :h, :w].astype(np.float64)
            # uniform on [0, p): the mean is (p - 1) / 2 within 6 standard errors
            assert abs(body.mean() - (ls.p - 1) / 2) < 6 * ls.p / np.sqrt(12 * body.size)
        assert not np.array_equal(xA, xB)
        a2, b2 = FI.shares(ls2, c.cid, li)
        assert np.array_equal(xA, a2) and np.array_equal(xB, b2)
        wt = FI.weights(ls, c.cid, li)
        assert wt.dtype == np.int8 and wt.shape == (ls.Co, ls.Ci, ls.fh, ls.fw)
        vals = set(np.unique(wt).tolist())
        if ls.binary:
            assert vals == {-1, 1}
        else:
            assert vals <= set(range(-8, 8)) and {-8, 7} <= vals
        assert np.array_equal(wt, FI.weights(ls, c.cid, li))


def test_seeds_and_packing():
    got = [FI.seeds(c.cid, s) for c in FI.CONFIGS.values() for s in range(3)]
    flat = [v for t in got for v in t]
    assert len(set(flat)) == len(flat)  # every stream its own seed
    for c in FI.CONFIGS.values():
        for ls in c.layers:
            S = min(ls.n, 2048 if ls.p == 12289 else ls.n)
            g_c, g_b = FI.default_pack(ls, S)
            assert g_b == 1 and 1 <= g_c <= ls.Ci
            assert ls.H * ls.W > S or g_c * ls.H * ls.W <= S
