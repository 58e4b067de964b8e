"""Pins for the oracle's protocol steps (CPU only).

Decryption correctness (Sec. 3.1), the homomorphic Hadamard product against
a schoolbook ring product, HomRec / HomShare identities (Eq. 2, 3), and the
end-to-end result s_A + s_B = u * w mod p (Eqs. 9-11) against a brute-force
cyclic convolution and, for the 28x28 (*) 5x5 layer padded to 32x32, against
scipy's full linear convolution.
"""
import numpy as np
import pytest
import scipy.signal

import fdsc_inputs as FI
from oracle import oracle as O


def negacyclic_schoolbook(a, b, m):
    L = len(a)
    out = [0] * L
    for i in range(L):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(L):
            k = i + j
            if k < L:
                out[k] += ai * int(b[j])
            else:
                out[k - L] -= ai * int(b[j])
    return [v % m for v in out]


def test_conv_plain_matches_bruteforce_and_scipy():
    p = 65537
    g = np.random.default_rng(0)
    x = np.zeros((1, 2, 32, 32), np.uint32)
    x[:, :, :28, :28] = g.integers(0, p, (1, 2, 28, 28))
    w = g.integers(-8, 8, (3, 2, 5, 5)).astype(np.int8)
    y = O.conv_plain(p, x, w)
    for co in range(3):
        full = sum(scipy.signal.convolve2d(x[0, ci, :28, :28].astype(np.int64), w[co, ci].astype(np.int64),
                                           mode="full") for ci in range(2))
        assert full.shape == (32, 32)
        assert np.array_equal(y[0, co], (full % p).astype(np.uint32))
    # wrap-around case: 8x8 plane, 3x3 filter, against np.roll brute force
    x = g.integers(0, p, (1, 1, 8, 8))
    w = g.integers(-8, 8, (1, 1, 3, 3)).astype(np.int8)
    ref = np.zeros((8, 8), dtype=object)
    for a in range(3):
        for c in range(3):
            ref = ref + int(w[0, 0, a, c]) * np.roll(np.roll(x[0, 0].astype(object), a, 0), c, 1)
    assert np.array_equal(O.conv_plain(p, x, w)[0, 0], (ref % p).astype(np.uint32))


@pytest.mark.parametrize("n,p,H,W", [(1024, 65537, 32, 32), (2048, 12289, 32, 64), (256, 65537, 16, 16)])
def test_decrypt_encrypt_roundtrip_and_fresh_noise(n, p, H, W):
    P = O.params(n, p)
    L = O.layer(P, 1, 1, 1, H, W, 1, 1)
    _, t_hat = O.keygen(P, 99)
    X = np.random.default_rng(n).integers(0, p, (1, 1, H * W)).astype(np.uint32)
    ct = O.encrypt(P, L, t_hat, X, 1234)
    assert ct.shape == (L.n_in, 2, n)
    for u in range(L.n_in):
        m, noise = O.decrypt_raw(P, t_hat, ct[u])
        assert noise <= 19
        slots = np.concatenate([O.slot_decode(P, m[r::P.d]) for r in range(P.d)]) if P.d > 1 else O.slot_decode(P, m)
        assert np.array_equal(slots, O.pack_input(P, L, X)[u])
    SA, noise = O.decrypt(P, L, t_hat, ct[:, :, :]) if L.n_in == L.n_out else (None, None)
    if SA is not None:
        assert np.array_equal(SA, X)


def test_hadamard_is_ring_product_and_homrec_adds():
    # n = 64: the decrypted HomConv output's coefficients are the schoolbook
    # negacyclic product of the message and the (centred) filter polynomial.
    n, p = 64, 65537
    P = O.params(n, p)
    L = O.layer(P, 1, 1, 1, 8, 8, 1, 1)
    _, t_hat = O.keygen(P, 5)
    g = np.random.default_rng(1)
    XA = g.integers(0, p, (1, 1, 64)).astype(np.uint32)
    XB = g.integers(0, p, (1, 1, 64)).astype(np.uint32)
    w = g.integers(-8, 8, (1, 1, 3, 3)).astype(np.int8)
    ct = O.encrypt(P, L, t_hat, XA, 77)
    ct = O.homrec(P, L, ct, XB)
    m, _ = O.decrypt_raw(P, t_hat, ct[0])
    assert np.array_equal(O.slot_decode(P, m), (XA[0, 0].astype(np.int64) + XB[0, 0]) % p)
    Phat = O.filter_prepare(P, L, w)
    out = O.homconv(P, L, ct, Phat, None)
    m_out, _ = O.decrypt_raw(P, t_hat, out[0])
    m_u = O.slot_encode(P, (XA[0, 0].astype(np.int64) + XB[0, 0]) % p)
    Wspec = O.filter_spectra(P, L, w)[0, 0]
    m_w = O.slot_encode(P, Wspec)
    assert [int(v) for v in m_out] == negacyclic_schoolbook(m_u, m_w, p)
    # the filter plaintext is the centred lift of m_w
    wpoly = O.intt_q(P, Phat[0])
    cent = [int(v) if int(v) <= (p - 1) // 2 else int(v) - p for v in m_w]
    assert [int(v) if int(v) < P.q // 2 else int(v) - P.q for v in wpoly] == cent


def _e2e(n, p, B, Ci, Co, H, W, fh, g_c=None, g_b=1, seed=0, homrec=True, support=None):
    P = O.params(n, p)
    L = O.layer(P, B, Ci, Co, H, W, g_c, g_b)
    g = np.random.default_rng(seed)
    h, w_ = support or (H, W)
    xA = np.zeros((B, Ci, H, W), np.uint32)
    xB = np.zeros((B, Ci, H, W), np.uint32)
    xA[:, :, :h, :w_] = g.integers(0, p, (B, Ci, h, w_))
    xB[:, :, :h, :w_] = g.integers(0, p, (B, Ci, h, w_))
    if not homrec:
        xB[:] = 0
    w = g.integers(-8, 8, (Co, Ci, fh, fh)).astype(np.int8)
    out = O.round_trip(P, L, xA, xB, w, 11 + seed, 22 + seed, 33 + seed, with_homrec=homrec)
    y = O.conv_plain(p, (xA.astype(np.int64) + xB) % p, w)
    assert np.array_equal((out["yA"].astype(np.int64) + out["yB"]) % p, y)
    assert out["noise"].max() < 2 ** O.noise_bound_log2(P, L.T)
    assert O.noise_ok(P, L.T)
    return P, L, out


@pytest.mark.parametrize("args", [
    dict(n=1024, p=65537, B=1, Ci=4, Co=4, H=16, W=16, fh=3),                       # the 16x16x4 layer's shape
    dict(n=256, p=65537, B=3, Ci=5, Co=3, H=8, W=8, fh=3, g_c=2, g_b=2),            # ragged Ci, B
    dict(n=256, p=65537, B=2, Ci=3, Co=2, H=32, W=16, fh=3),                       # halves (HW > S)
    dict(n=512, p=12289, B=3, Ci=3, Co=2, H=8, W=8, fh=3, g_c=2, g_b=2),            # p = 12289
    dict(n=4096, p=12289, B=3, Ci=2, Co=2, H=64, W=64, fh=3),                      # d = 2 with halves
    dict(n=4096, p=12289, B=5, Ci=3, Co=2, H=16, W=16, fh=3, g_c=2, g_b=3),         # d = 2 with blocks
    dict(n=2048, p=65537, B=1, Ci=1, Co=4, H=32, W=32, fh=5, support=(28, 28)),    # MNIST-shaped
    dict(n=2048, p=147457, B=1, Ci=6, Co=3, H=32, W=32, fh=3),                     # Table 2 "Medium" prime
    dict(n=256, p=786433, B=3, Ci=3, Co=2, H=8, W=8, fh=3, g_c=2, g_b=2),           # p = 3 2^18 + 1, near 2^20
])
def test_end_to_end_shares_reconstruct_convolution(args):
    _e2e(**args)


def test_first_round_without_homrec():
    _e2e(1024, 65537, 1, 4, 4, 16, 16, 3, homrec=False)


def test_packing_invariance_of_final_shares():
    res = {}
    for g_c, g_b in [(1, 1), (2, 1), (4, 1), (2, 2), (1, 4), (3, 1)]:
        P, L, out = _e2e(256, 65537, 4, 5, 3, 8, 8, 3, g_c=g_c, g_b=g_b, seed=4)
        res[(g_c, g_b)] = (out["yA"], out["yB"])
    ref = res[(1, 1)]
    for k, (yA, yB) in res.items():
        assert np.array_equal(yA, ref[0]) and np.array_equal(yB, ref[1]), k


def test_tier0_and_tier1_pipelines_agree_bitwise():
    P = O.params(64, 65537)
    L = O.layer(P, 2, 3, 2, 4, 4, 2, 2)
    g = np.random.default_rng(8)
    xA, xB = g.integers(0, 65537, (2, 2, 3, 4, 4))
    w = g.integers(-8, 8, (2, 3, 3, 3)).astype(np.int8)
    o1 = O.round_trip(P, L, xA, xB, w, 1, 2, 3)
    with O.tier(0):
        o0 = O.round_trip(P, L, xA, xB, w, 1, 2, 3)
    for k in o1:
        assert np.array_equal(o0[k], o1[k]), k


def test_homshare_fold_gives_product_minus_mask():
    n, p = 256, 65537
    P = O.params(n, p)
    L = O.layer(P, 2, 5, 3, 8, 8, 2, 2)
    g = np.random.default_rng(3)
    xA = g.integers(0, p, (2, 5, 8, 8))
    w = g.integers(-8, 8, (3, 5, 3, 3)).astype(np.int8)
    out = O.round_trip(P, L, xA, np.zeros_like(xA), w, 1, 2, 3, with_homrec=False)
    Wh = O.filter_spectra(P, L, w).astype(object)
    X = out["XA"].astype(object)
    Y = np.einsum("bcf,ocf->bof", X, Wh) % p
    assert np.array_equal((out["SA_hat"].astype(object) + out["sB_hat"]) % p, Y)


@pytest.mark.parametrize("cfg", ["layer_16x16x4_b1", "cifar_32x32x64_b1"])
def test_config_round_trip(cfg):
    c = FI.CONFIGS[cfg]
    ls = c.layers[0]
    P = O.params(ls.n, ls.p)
    g_c, g_b = FI.default_pack(ls, P.S)
    L = O.layer(P, ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
    xA, xB = FI.shares(ls, c.cid)
    w = FI.weights(ls, c.cid)
    ks, es, ss = FI.seeds(c.cid)
    out = O.round_trip(P, L, xA, xB, w, ks, es, ss)
    y = O.conv_plain(ls.p, (xA.astype(np.int64) + xB) % ls.p, w)
    assert np.array_equal((out["yA"].astype(np.int64) + out["yB"]) % ls.p, y)
    assert np.log2(out["noise"].max()) < O.noise_bound_log2(P, L.T) < np.log2(P.delta / 2)


def test_pool2x2_sum_pins():
    """The appendix's average pooling on shares (a 2x2 sum mod p): a delta
    goes to a delta, every window sum is kept, and pooling commutes with
    adding the shares (so each party pools its own)."""
    p = 65537
    x = np.zeros((1, 8, 6), np.uint32)
    x[0, 5, 2] = 7
    y = O.pool2x2_sum(p, x)
    assert y.shape == (1, 4, 3) and y[0, 2, 1] == 7 and y.sum() == 7
    g = np.random.default_rng(4)
    a = g.integers(0, p, (3, 2, 16, 16)).astype(np.uint32)
    b = g.integers(0, p, (3, 2, 16, 16)).astype(np.uint32)
    ya, yb = O.pool2x2_sum(p, a), O.pool2x2_sum(p, b)
    assert int(ya.astype(object).sum()) % p == int(a.astype(object).sum()) % p
    both = O.pool2x2_sum(p, ((a.astype(np.int64) + b) % p).astype(np.uint32))
    assert np.array_equal((ya.astype(np.int64) + yb) % p, both)
    win = a[1, 1, 6:8, 10:12].astype(np.int64).sum() % p  # one window by hand
    assert ya[1, 1, 3, 5] == win


def test_two_layer_chain_with_pooling_reconstructs_the_network():
    """A chain of FDSC layers (Fig. 2's layer to layer steps, the activation protocol
    left out): layer 2 takes layer 1's output shares after sum pooling; the
    final shares add up to conv2(pool(conv1(x))) computed directly."""
    p, n = 65537, 1024
    g = np.random.default_rng(9)
    P = O.params(n, p)
    xA = g.integers(0, p, (1, 3, 16, 16)).astype(np.uint32)
    xB = g.integers(0, p, (1, 3, 16, 16)).astype(np.uint32)
    w1 = g.integers(-8, 8, (4, 3, 3, 3)).astype(np.int8)
    w2 = g.integers(-8, 8, (2, 4, 3, 3)).astype(np.int8)
    o1 = O.round_trip(P, O.layer(P, 1, 3, 4, 16, 16), xA, xB, w1, 1, 2, 3)
    pA, pB = O.pool2x2_sum(p, o1["yA"]), O.pool2x2_sum(p, o1["yB"])
    o2 = O.round_trip(P, O.layer(P, 1, 4, 2, 8, 8), pA, pB, w2, 4, 5, 6)
    x = (xA.astype(np.int64) + xB) % p
    h1 = np.zeros((1, 4, 16, 16), dtype=object)  # brute-force cyclic convolution
    for co in range(4):
        for ci in range(3):
            for a in range(3):
                for c in range(3):
                    h1[0, co] += int(w1[co, ci, a, c]) * np.roll(np.roll(x[0, ci].astype(object), a, 0), c, 1)
    h1 = h1 % p
    pooled = (h1[:, :, 0::2, 0::2] + h1[:, :, 1::2, 0::2] + h1[:, :, 0::2, 1::2] + h1[:, :, 1::2, 1::2]) % p
    h2 = np.zeros((1, 2, 8, 8), dtype=object)
    for co in range(2):
        for ci in range(4):
            for a in range(3):
                for c in range(3):
                    h2[0, co] += int(w2[co, ci, a, c]) * np.roll(np.roll(pooled[0, ci], a, 0), c, 1)
    h2 = (h2 % p).astype(np.int64)
    assert np.array_equal((o2["yA"].astype(np.int64) + o2["yB"]) % p, h2)


def _max_flood(P, T):
    f = 0
    while f < 62 and O.noise_ok(P, T, f + 1):
        f += 1
    return f


def test_noise_flooding_keeps_the_shares_and_stays_in_the_bound():
    """HomShare noise flooding (circuit privacy, not in the paper): the mask
    plaintext carries a uniform error of 2^f per coefficient.  At the largest
    f the noise bound admits, decryption still rounds it away: the final
    shares are those of the unflooded run, the ciphertexts differ, and the
    decryption noise grows to the flood's size but stays under the bound."""
    p, n = 65537, 1024
    P = O.params(n, p)
    L = O.layer(P, 1, 4, 4, 16, 16)
    f = _max_flood(P, L.T)
    assert 40 <= f <= 43 and not O.noise_ok(P, L.T, f + 1)
    g = np.random.default_rng(12)
    xA = g.integers(0, p, (1, 4, 16, 16)).astype(np.uint32)
    xB = g.integers(0, p, (1, 4, 16, 16)).astype(np.uint32)
    w = g.integers(-8, 8, (4, 4, 3, 3)).astype(np.int8)
    plain = O.round_trip(P, L, xA, xB, w, 1, 2, 3)
    flood = O.round_trip(P, L, xA, xB, w, 1, 2, 3, flood_bits=f)
    assert np.array_equal(plain["yA"], flood["yA"]) and np.array_equal(plain["yB"], flood["yB"])
    assert not np.array_equal(plain["ct_out"], flood["ct_out"])
    assert flood["noise"].max() > 2 ** (f - 1)  # the flood dominates the noise
    assert flood["noise"].max() < 2 ** O.noise_bound_log2(P, L.T) + 2 ** f


def test_flood_error_is_uniform_on_its_interval():
    """INTT_q of (flooded mask - plain mask) is the flood error itself: every
    coefficient in [-2^f, 2^f), the interval's two halves about equally hit."""
    p, n, f = 65537, 1024, 20
    P = O.params(n, p)
    L = O.layer(P, 1, 4, 8, 16, 16)
    M0, s0 = O.mask_prepare(P, L, 77)
    M1, s1 = O.mask_prepare(P, L, 77, f)
    assert np.array_equal(s0, s1)
    d = ((M1.astype(object) - M0.astype(object)) % P.q).astype(np.uint64)
    e = np.array([[int(v) if v < P.q // 2 else int(v) - P.q for v in O.intt_q(P, row)] for row in d], dtype=np.int64)
    assert e.min() >= -(1 << f) and e.max() < (1 << f)
    assert e.min() < -(1 << (f - 1)) and e.max() > (1 << (f - 1))
    assert abs(np.mean(e >= 0) - 0.5) < 0.02


@pytest.mark.parametrize("n,p,B,Ci,Co,H,W,g_c,g_b", [(4096, 12289, 2, 3, 2, 64, 64, 1, 1),
                                                    (4096, 12289, 4, 5, 3, 16, 16, 2, 2),
                                                    (1024, 7681, 2, 3, 2, 16, 16, 1, 1)])
def test_filter_plaintexts_take_one_value_per_group_of_d_indices(n, p, B, Ci, Co, H, W, g_c, g_b):
    """With d = n/S slot sets the filter plaintexts are w_0(x^d) (Sec. 3.1's
    SIMDScMult over several slot sets): in the bit-reversed NTT_q order the d
    consecutive evaluation indices of a group are the points x times the d-th
    roots of unity, where x^d -- and so the filter -- takes one value.  This
    is what lets the filter be stored once per group.  Checked on the
    oracle's plaintexts, and the group's points checked directly."""
    P = O.params(n, p)
    assert P.d > 1
    L = O.layer(P, B, Ci, Co, H, W, g_c, g_b)
    w = np.random.default_rng(n + p).integers(-8, 8, (Co, Ci, 3, 3)).astype(np.int8)
    Ph = O.filter_prepare(P, L, w).reshape(-1, n)
    for r in range(1, P.d):
        assert np.array_equal(Ph[:, r::P.d], Ph[:, 0::P.d])
    # the points: psi^(2 brv(j) + 1) for the j of a group, raised to d, agree
    q, psi, logn = P.q, P.psi_q, n.bit_length() - 1
    brv = lambda j: int(format(j, "0%db" % logn)[::-1], 2)
    for g0 in range(0, n, P.d * 37):
        pts = {pow(pow(psi, 2 * brv(j) + 1, q), P.d, q) for j in range(g0, g0 + P.d)}
        assert len(pts) == 1
