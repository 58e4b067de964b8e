"""GPU parity: every stage of the CUDA path is bit-identical to the CPU
oracle on the same seeded inputs (exact integer arithmetic, tolerance zero).

Stage-by-stage checks run at sizes the oracle finishes in seconds (the full
32x32x64 layer, reduced-batch versions of the other workloads, ragged and
degenerate shapes); at full batch sizes the composed result is checked with a
property that holds at any size, s_A + s_B = u * w mod p, on sampled planes
against the oracle's plain convolution.
"""
import numpy as np
import pytest
import torch

import fdsc_inputs as FI
from fdsc_harness import compare_all, dev, gpu_round_trip, u32, u64
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_05328_gb300 import build

    build.build()
    from paper_2003_05328_gb300 import fdsc

    torch.cuda.set_device(0)
    return fdsc


def _inputs(seed, B, Ci, Co, H, W, fh, fw, p, support=None):
    g = np.random.default_rng(seed)
    h, w_ = support or (H, W)
    xA = np.zeros((B, Ci, H, W), np.uint32)
    xB = np.zeros((B, Ci, H, W), np.uint32)
    xA[:, :, :h, :w_] = g.integers(0, p, (B, Ci, h, w_))
    xB[:, :, :h, :w_] = g.integers(0, p, (B, Ci, h, w_))
    w = g.integers(-8, 8, (Co, Ci, fh, fw)).astype(np.int8)
    return xA, xB, w


def _check_layer(F, n, p, B, Ci, Co, H, W, fh, fw=None, g_c=None, g_b=1, seed=0, homrec=True, support=None,
                 xA=None, xB=None, w=None):
    fw = fw or fh
    OP = O.params(n, p)
    OL = O.layer(OP, B, Ci, Co, H, W, g_c, g_b)
    P = F.Params(n, p, max_T=max(OL.T, 1))
    L = F.LayerSpec(B, Ci, Co, H, W, OL.g_c, OL.g_b)
    if xA is None:
        xA, xB, w = _inputs(seed, B, Ci, Co, H, W, fh, fw, p, support)
    if not homrec:
        xB = np.zeros_like(xA)
    ks, es, ss = 1000 + seed, 2000 + seed, 3000 + seed
    got = gpu_round_trip(P, L, xA, xB, w, ks, es, ss, homrec=homrec)
    ref = O.round_trip(OP, OL, xA, xB, w, ks, es, ss, with_homrec=homrec)
    compare_all(got, ref)
    y = O.conv_plain(p, (xA.astype(np.int64) + xB) % p, w)
    assert np.array_equal((got["yA"].reshape(y.shape).astype(np.int64) + got["yB"].reshape(y.shape)) % p, y)
    P.close()
    return got, ref


# ---------------------------------------------------------------- transforms
@pytest.mark.parametrize("p", [65537, 12289, 147457, 786433])  # 786433 2^10 < 2^32: lazy sums still fit
@pytest.mark.parametrize("H,W,planes", [(2, 2, 3), (4, 64, 5), (64, 4, 2), (8, 8, 7), (16, 16, 64), (16, 16, 5),
                                        (32, 32, 1), (32, 32, 64), (64, 64, 9), (2, 2048, 2), (32, 32, 2500)])
def test_ntt2d_intt2d_match_oracle(F, p, H, W, planes):
    P = F.Params(1024, p, max_T=8)  # the default T = 256 fails the noise bound at p = 786433
    x = np.random.default_rng(H * 131 + W + planes).integers(0, p, (planes, H, W)).astype(np.uint32)
    X = F.ntt2d(P, dev(x, np.int32))
    assert np.array_equal(u32(X).reshape(x.shape), O.ntt2d(x, p))
    back = F.intt2d(P, X)
    assert np.array_equal(u32(back).reshape(x.shape), x)
    # in place
    t = dev(x, np.int32)
    F.ntt2d(P, t, out=t)
    assert np.array_equal(u32(t).reshape(x.shape), O.ntt2d(x, p))
    # a delta transforms to all ones; the inverse of the oracle spectrum is x
    d = np.zeros((1, H, W), np.uint32)
    d[0, 0, 0] = 1
    assert np.all(u32(F.ntt2d(P, dev(d, np.int32))) == 1)
    assert np.array_equal(u32(F.intt2d(P, dev(O.ntt2d(x, p), np.int32))).reshape(x.shape), x)
    # the largest inputs (every word p - 1), where unreduced sums grow the most
    m = np.full((2, H, W), p - 1, np.uint32)
    assert np.array_equal(u32(F.ntt2d(P, dev(m, np.int32))).reshape(m.shape), O.ntt2d(m, p))
    assert np.array_equal(u32(F.intt2d(P, dev(m, np.int32))).reshape(m.shape), O.ntt2d(m, p, inverse=True))
    P.close()


def test_ntt2d_empty_batch_is_noop(F):
    P = F.Params(1024, 65537)
    x = torch.empty((0, 16, 16), dtype=torch.int32, device="cuda")
    out = F.ntt2d(P, x)
    assert out.numel() == 0
    P.close()


@pytest.mark.parametrize("n,p", [(1024, 65537), (2048, 65537), (4096, 65537), (4096, 12289), (16, 65537)])
def test_keygen_matches_oracle(F, n, p):
    P = F.Params(n, p)
    t_hat = F.keygen(P, 424242)
    _, ref = O.keygen(O.params(n, p), 424242)
    assert np.array_equal(u64(t_hat), ref)
    P.close()


# ---------------------------------------------------------------- whole layer, every stage
@pytest.mark.parametrize("cfg", ["layer_16x16x4_b1", "cifar_32x32x64_b1"])
def test_config_layer_bit_exact(F, cfg):
    c = FI.CONFIGS[cfg]
    ls = c.layers[0]
    S = O.params(ls.n, ls.p).S
    g_c, g_b = FI.default_pack(ls, S)
    xA, xB = FI.shares(ls, c.cid)
    w = FI.weights(ls, c.cid)
    _check_layer(F, ls.n, ls.p, ls.B, ls.Ci, ls.Co, ls.H, ls.W, ls.fh, ls.fw, g_c, g_b, seed=c.cid, xA=xA, xB=xB,
                 w=w)


@pytest.mark.parametrize("args", [
    dict(n=256, p=65537, B=3, Ci=5, Co=3, H=8, W=8, fh=3, g_c=2, g_b=2),          # ragged Ci and B
    dict(n=256, p=65537, B=2, Ci=3, Co=2, H=32, W=16, fh=3),                     # halves (HW > S)
    dict(n=512, p=12289, B=3, Ci=3, Co=2, H=8, W=8, fh=3, g_c=2, g_b=2),          # p = 12289
    dict(n=4096, p=12289, B=3, Ci=2, Co=3, H=64, W=64, fh=3),                    # d = 2 slot sets, halves
    dict(n=4096, p=12289, B=5, Ci=3, Co=2, H=16, W=16, fh=3, g_c=2, g_b=3),       # d = 2 with blocks
    dict(n=2048, p=65537, B=1, Ci=1, Co=16, H=32, W=32, fh=5, support=(28, 28)), # MNIST-shaped layer
    dict(n=1024, p=65537, B=2, Ci=7, Co=5, H=16, W=16, fh=3, g_c=3, g_b=1),       # g_c not a power of two
    dict(n=64, p=65537, B=1, Ci=1, Co=1, H=2, W=2, fh=2),                        # smallest plane, full filter
    dict(n=1024, p=65537, B=1, Ci=3, Co=2, H=32, W=32, fh=1),                    # 1x1 filter
    dict(n=1024, p=65537, B=1, Ci=2, Co=2, H=4, W=256, fh=3, fw=5),              # wide plane, fh != fw
    dict(n=2048, p=65537, B=2, Ci=64, Co=8, H=32, W=32, fh=3, homrec=False),     # first round, no HomRec
    dict(n=2048, p=147457, B=1, Ci=16, Co=4, H=32, W=32, fh=3),                  # Table 2 "Medium" prime
    dict(n=1024, p=786433, B=3, Ci=6, Co=3, H=16, W=16, fh=3, g_c=2, g_b=2),      # p = 3 2^18 + 1, near 2^20
])
def test_layer_variants_bit_exact(F, args):
    _check_layer(F, **args)


def _sweep_cases():
    """A seeded sweep of small layers over the property ranges: n in {64,
    128, 256}, H, W in {4, 8, 16} with H W <= S (S = n for these n and both
    primes), Ci, Co in {1, 2, 3, 5}, 1 to 3 images, and random packings of
    channel and image blocks."""
    g = np.random.default_rng(2024)
    cases = []
    while len(cases) < 12:
        n, p = int(g.choice([64, 128, 256])), int(g.choice([65537, 12289]))
        H, W = int(g.choice([4, 8, 16])), int(g.choice([4, 8, 16]))
        if H * W > n:
            continue
        Ci, Co, B = int(g.choice([1, 2, 3, 5])), int(g.choice([1, 2, 3, 5])), int(g.integers(1, 4))
        blocks = n // (H * W)
        g_c = int(g.integers(1, min(blocks, Ci) + 1))
        g_b = int(g.integers(1, blocks // g_c + 1))
        cases.append(dict(n=n, p=p, B=B, Ci=Ci, Co=Co, H=H, W=W, g_c=g_c, g_b=g_b))
    return cases


@pytest.mark.parametrize("i,case", list(enumerate(_sweep_cases())))
def test_small_layer_sweep_with_edge_values(F, i, case):
    """Every stage word-exact on the sweep, with shares drawn from the edge
    values {0, 1, p - 1} and 3x3 weights from {-8, -1, 0, 7}."""
    g = np.random.default_rng(100 + i)
    n, p, B, Ci, Co, H, W = (case[k] for k in ("n", "p", "B", "Ci", "Co", "H", "W"))
    xA = g.choice(np.array([0, 1, p - 1], np.uint32), (B, Ci, H, W))
    xB = g.choice(np.array([0, 1, p - 1], np.uint32), (B, Ci, H, W))
    w = g.choice(np.array([-8, -1, 0, 7], np.int8), (Co, Ci, 3, 3))
    _check_layer(F, n, p, B, Ci, Co, H, W, 3, g_c=case["g_c"], g_b=case["g_b"], seed=200 + i, xA=xA, xB=xB, w=w)


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_batched_stack_layers_reduced_batch_bit_exact(F, layer):
    ls = FI.CONFIGS["stack_16img_32x32x64_16x16x128_8x8x256"].layers[layer]
    S = O.params(ls.n, ls.p).S
    g_c, g_b = FI.default_pack(ls, S)
    _check_layer(F, ls.n, ls.p, 2, ls.Ci, ls.Co, ls.H, ls.W, ls.fh, ls.fw, g_c, g_b, seed=20 + layer)


def test_binarized_layer_reduced_channels_bit_exact(F):
    ls = FI.CONFIGS["binarized_64x64x128_b8"].layers[0]
    g = np.random.default_rng(44)
    B, Ci, Co = 2, 8, 8
    xA, xB, _ = _inputs(44, B, Ci, Co, ls.H, ls.W, 3, 3, ls.p)
    w = (g.integers(0, 2, (Co, Ci, 3, 3)) * 2 - 1).astype(np.int8)
    _check_layer(F, ls.n, ls.p, B, Ci, Co, ls.H, ls.W, 3, 3, 1, 1, xA=xA, xB=xB, w=w)


def test_degenerate_values(F):
    n, p, B, Ci, Co, H, W = 1024, 65537, 1, 4, 3, 16, 16
    zeros = np.zeros((B, Ci, H, W), np.uint32)
    top = np.full((B, Ci, H, W), p - 1, np.uint32)
    w = np.full((Co, Ci, 3, 3), -8, np.int8)
    _check_layer(F, n, p, B, Ci, Co, H, W, 3, g_c=4, xA=zeros, xB=zeros.copy(), w=w)
    _check_layer(F, n, p, B, Ci, Co, H, W, 3, g_c=4, xA=top, xB=top.copy(), w=w)
    _check_layer(F, n, p, B, Ci, Co, H, W, 3, g_c=4, xA=top, xB=zeros.copy(), w=np.zeros_like(w))


def test_homconv_without_mask_and_determinism(F):
    n, p, B, Ci, Co, H, W = 2048, 65537, 1, 64, 64, 32, 32
    OP = O.params(n, p)
    OL = O.layer(OP, B, Ci, Co, H, W, 2, 1)
    P = F.Params(n, p)
    L = F.LayerSpec(B, Ci, Co, H, W, 2, 1)
    g = np.random.default_rng(5)
    ct = np.array(g.integers(0, OP.q, (OL.n_in, 2, n), dtype=np.uint64))
    Ph = np.array(g.integers(0, OP.q, (Co * OL.T, n), dtype=np.uint64))
    ct[0, 0, :8] = OP.q - 1  # extremes
    Ph[0, :8] = OP.q - 1
    ref = O.homconv(OP, OL, ct, Ph, None)
    a = F.homconv(P, L, dev(ct.view(np.int64), np.int64), dev(Ph.view(np.int64), np.int64))
    b = F.homconv(P, L, dev(ct.view(np.int64), np.int64), dev(Ph.view(np.int64), np.int64))
    assert np.array_equal(u64(a).reshape(ref.shape), ref)
    assert torch.equal(a, b)
    P.close()


def test_homconv_many_terms_folds_accumulator(F):
    # T = 300 > 256: the 128-bit accumulator must be reduced part way.
    n, p, B, Ci, Co, H, W = 64, 65537, 1, 300, 2, 8, 8
    OP = O.params(n, p)
    OL = O.layer(OP, B, Ci, Co, H, W, 1, 1)
    P = F.Params(n, p, max_T=300)
    L = F.LayerSpec(B, Ci, Co, H, W, 1, 1)
    ct = np.full((OL.n_in, 2, n), OP.q - 1, np.uint64)
    Ph = np.full((Co * OL.T, n), OP.q - 1, np.uint64)
    ref = O.homconv(OP, OL, ct, Ph, None)
    try:  # the default kernel, and the Karatsuba-column kernel folding every 256 terms
        for v in (0, 8):
            F.set_homconv_variant(v)
            got = F.homconv(P, L, dev(ct.view(np.int64), np.int64), dev(Ph.view(np.int64), np.int64))
            assert np.array_equal(u64(got).reshape(ref.shape), ref), v
    finally:
        F.set_homconv_variant(0)
    P.close()


# ---------------------------------------------------------------- full sizes (property checks)
def _full_size_property(F, ls, cid, g_c, g_b, sample_planes):
    P = F.Params(ls.n, ls.p, max_T=256)
    L = F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
    xA, xB = FI.shares(ls, cid)
    w = FI.weights(ls, cid)
    ks, es, ss = FI.seeds(cid)
    got = gpu_round_trip(P, L, xA, xB, w, ks, es, ss)
    y = (got["yA"].reshape(ls.B, ls.Co, ls.H, ls.W).astype(np.int64) +
         got["yB"].reshape(ls.B, ls.Co, ls.H, ls.W)) % ls.p
    x = (xA.astype(np.int64) + xB) % ls.p
    rng = np.random.default_rng(cid)
    for _ in range(sample_planes):
        b, co = int(rng.integers(ls.B)), int(rng.integers(ls.Co))
        ref = O.conv_plain(ls.p, x[b:b + 1], w[co:co + 1])
        assert np.array_equal(y[b, co], ref[0, 0]), (b, co)
    # Bob's mask is uniform and Alice's share alone is not the result
    assert not np.array_equal(got["yA"].reshape(y.shape), y)
    P.close()


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_batched_stack_full_batch_property(F, layer):
    ls = FI.CONFIGS["stack_16img_32x32x64_16x16x128_8x8x256"].layers[layer]
    g_c, g_b = FI.default_pack(ls, O.params(ls.n, ls.p).S)
    _full_size_property(F, ls, 2, g_c, g_b, 6)


def test_binarized_layer_full_size_property(F):
    ls = FI.CONFIGS["binarized_64x64x128_b8"].layers[0]
    _full_size_property(F, ls, 4, 1, 1, 4)


# ---------------------------------------------------------------- errors
def test_argument_errors_are_reported(F):
    P = F.Params(2048, 65537, max_T=16)
    L = F.LayerSpec(1, 64, 64, 32, 32, 2, 1)  # T = 32 > max_T
    lay = F.layout(P, L)
    ct = torch.zeros(lay.ct_in_words, dtype=torch.int64, device="cuda")
    Ph = torch.zeros(lay.filter_words, dtype=torch.int64, device="cuda")
    with pytest.raises(F.FdscError) as e:
        F.homconv(P, L, ct, Ph)
    assert e.value.code == -2
    L2 = F.LayerSpec(1, 32, 64, 32, 32, 2, 1)
    lay2 = F.layout(P, L2)
    big = torch.zeros(lay2.ct_in_words + lay2.ct_out_words, dtype=torch.int64, device="cuda")
    with pytest.raises(F.FdscError) as e:  # output overlapping the input
        F._call("fdsc_homconv", P.handle, F.C.byref(L2.c()), big.data_ptr(), Ph.data_ptr(), None,
                     big.data_ptr() + 8 * 16, 0)
    assert e.value.code == -1
    x = torch.zeros(2 * 16 * 16 + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(F.FdscError) as e:  # misaligned
        F._call("fdsc_ntt2d", P.handle, 16, 16, x.data_ptr() + 4, x.data_ptr(), 2, 0)
    assert e.value.code == -1
    with pytest.raises(F.FdscError) as e:  # bad plane
        F._call("fdsc_ntt2d", P.handle, 12, 16, x.data_ptr(), x.data_ptr(), 1, 0)
    assert e.value.code == -1
    with pytest.raises(F.FdscError) as e:  # noise bound at creation
        F.Params(4096, 65537, max_T=100000)
    assert e.value.code == -2
    P.close()


@pytest.mark.parametrize("shape", [(2048, 1, 64, 64, 32, 32, 2, 1), (4096, 2, 256, 8, 8, 8, 64, 1),
                                   (1024, 3, 5, 7, 16, 16, 2, 2), (64, 1, 300, 3, 8, 8, 1, 1),
                                   (256, 2, 3, 5, 32, 16, 1, 1),
                                   # many image groups per CTA (tile slots recycled), T not a multiple of 8
                                   (2048, 16, 50, 8, 32, 32, 2, 1),
                                   # beta = 4 halves per plane, Co not a multiple of 8
                                   (1024, 2, 12, 12, 64, 64, 1, 1),
                                   # fewer evaluation indices than one tile, ragged channel tile
                                   (16, 2, 8, 9, 4, 4, 1, 1)])
def test_homconv_variants_identical(F, shape):
    """Every HomConv kernel variant (accumulation scheme, tiling, fused c1
    addends) gives the oracle's words."""
    n, B, Ci, Co, H, W, g_c, g_b = shape
    OP = O.params(n, 65537)
    OL = O.layer(OP, B, Ci, Co, H, W, g_c, g_b)
    P = F.Params(n, 65537, max_T=max(OL.T, 1))
    L = F.LayerSpec(B, Ci, Co, H, W, g_c, g_b)
    g = np.random.default_rng(n + Ci)
    ct = np.array(g.integers(0, OP.q, (OL.n_in, 2, n), dtype=np.uint64))
    A1 = np.array(g.integers(0, OP.q, (OL.n_in, n), dtype=np.uint64))
    A2 = np.array(g.integers(0, OP.q, (OL.n_in, n), dtype=np.uint64))
    Ph = np.array(g.integers(0, OP.q, (Co * OL.T * OL.beta, n), dtype=np.uint64))
    Mh = np.array(g.integers(0, OP.q, (OL.n_out, n), dtype=np.uint64))
    ct[:, :, :4] = OP.q - 1
    Ph[:, :4] = OP.q - 1
    summed = ct.astype(object)
    summed[:, 1] = (summed[:, 1] + A1.astype(object) + A2.astype(object)) % OP.q
    ref = O.homconv(OP, OL, summed.astype(np.uint64), Ph, Mh)
    d = lambda a: dev(a.view(np.int64), np.int64)
    try:
        for v in (1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 12, 13, 14, 15):
            F.set_homconv_variant(v)
            out = F.homconv_sum(P, L, d(ct), d(A1), d(A2), d(Ph), d(Mh))
            assert np.array_equal(u64(out).reshape(ref.shape), ref), v
            out = F.homconv_sum(P, L, d(ct), d(A1), None, d(Ph), None)
            part = ct.astype(object)
            part[:, 1] = (part[:, 1] + A1.astype(object)) % OP.q
            assert np.array_equal(u64(out).reshape(ref.shape), O.homconv(OP, OL, part.astype(np.uint64), Ph, None)), v
            out = F.homconv_sum(P, L, d(summed.astype(np.uint64)), None, None, d(Ph), d(Mh))
            assert np.array_equal(u64(out).reshape(ref.shape), ref), v
    finally:
        F.set_homconv_variant(0)
    P.close()


@pytest.mark.parametrize("shape", [(2048, 1, 64, 64, 32, 32, 2, 1), (1024, 3, 5, 7, 16, 16, 2, 2),
                                   (1024, 2, 12, 12, 64, 64, 1, 1)])
def test_seeded_ciphertexts(F, shape):
    """Seeded input ciphertexts (seed + c1): the c1 words are those of the
    oracle's encryption, and HomConv drawing c0 = -a again from the seed
    gives the oracle's HomConv of the full ciphertexts."""
    n, B, Ci, Co, H, W, g_c, g_b = shape
    OP = O.params(n, 65537)
    OL = O.layer(OP, B, Ci, Co, H, W, g_c, g_b)
    P = F.Params(n, 65537, max_T=max(OL.T, 1))
    L = F.LayerSpec(B, Ci, Co, H, W, g_c, g_b)
    es = 0x5EED + n
    _, t_hat_o = O.keygen(OP, 7)
    ct_o = O.encrypt(OP, OL, t_hat_o, np.zeros((B, Ci, H * W), np.uint32), es)
    c1 = F.encrypt_constants_seeded(P, L, F.keygen(P, 7), es)
    torch.cuda.synchronize()
    assert np.array_equal(u64(c1).reshape(OL.n_in, n), ct_o[:, 1])
    g = np.random.default_rng(n + Co)
    A1 = np.array(g.integers(0, OP.q, (OL.n_in, n), dtype=np.uint64))
    A2 = np.array(g.integers(0, OP.q, (OL.n_in, n), dtype=np.uint64))
    Ph = np.array(g.integers(0, OP.q, (Co * OL.T * OL.beta, n), dtype=np.uint64))
    Mh = np.array(g.integers(0, OP.q, (OL.n_out, n), dtype=np.uint64))
    d = lambda a: dev(a.view(np.int64), np.int64)
    out = F.homconv_seeded(P, L, es, c1, d(A1), d(A2), d(Ph), d(Mh))
    full = ct_o.astype(object)
    full[:, 1] = (full[:, 1] + A1.astype(object) + A2.astype(object)) % OP.q
    ref = O.homconv(OP, OL, full.astype(np.uint64), Ph, Mh)
    assert np.array_equal(u64(out).reshape(ref.shape), ref)
    P.close()


# ---------------------------------------------------------------- tensor-core HomConv
def _worst_digit_word(q):
    """The largest word below q whose balanced base-256 digits 0..6 are all
    -128: (w + 0x80..80) has bytes 0..6 equal to zero."""
    low = (1 << 56) - 0x80808080808080  # w = low mod 2^56
    t = (q - 1 - low) >> 56
    return low + (t << 56)


@pytest.mark.parametrize("shape", [
    (2048, 1, 64, 64, 32, 32, 2, 1),    # the 32x32x64 layer at batch 1: T = 32, Co = 64 (half an M tile)
    (1024, 3, 5, 7, 16, 16, 2, 2),      # T = 3: one ragged block of 16 input ciphertexts; 2 image groups
    (1024, 2, 12, 12, 64, 64, 1, 1),    # beta = 4 ciphertexts per spectrum, Co not a multiple of 8
    (2048, 16, 50, 8, 32, 32, 2, 1),    # 16 image groups: two passes of 8; T = 25
    (256, 5, 34, 130, 8, 8, 1, 1),      # Co = 130: a full and a 2-channel tile; T = 34: 3 blocks; 5 groups: 4 + 1
    (1024, 1, 128, 128, 32, 32, 1, 1),  # T = 128, the largest the fp32 bound admits
    # d > 1: an item holds the d evaluation indices that share a filter word
    (4096, 3, 5, 9, 32, 32, 2, 1, 12289),     # d = 2, two image groups (the second half empty)
    (4096, 8, 16, 130, 64, 64, 1, 1, 12289),  # d = 2, beta = 2, four image groups, two channel tiles
    (1024, 9, 20, 12, 16, 16, 1, 1, 7681),    # d = 4: two groups per pass, the second pass ragged; T = 20
])
def test_homconv_tc_matches_oracle(F, shape):
    """The tensor-core HomConv (digit planes in fp16, exact fp32 sums of the
    15 weight classes) gives the oracle's words, with and without the fused
    c1 addends and the HomShare mask."""
    n, B, Ci, Co, H, W, g_c, g_b = shape[:8]
    p = shape[8] if len(shape) > 8 else 65537
    OP = O.params(n, p)
    OL = O.layer(OP, B, Ci, Co, H, W, g_c, g_b)
    P = F.Params(n, p, max_T=max(OL.T, 1))
    L = F.LayerSpec(B, Ci, Co, H, W, g_c, g_b)
    g = np.random.default_rng(n + Ci + Co)
    ct = np.array(g.integers(0, OP.q, (OL.n_in, 2, n), dtype=np.uint64))
    A1 = np.array(g.integers(0, OP.q, (OL.n_in, n), dtype=np.uint64))
    A2 = np.array(g.integers(0, OP.q, (OL.n_in, n), dtype=np.uint64))
    dd = OP.d  # the library stores one filter word per group of d indices; the oracle takes all n
    Ph = np.array(g.integers(0, OP.q, (Co * OL.T * OL.beta, n // dd), dtype=np.uint64))
    Mh = np.array(g.integers(0, OP.q, (OL.n_out, n), dtype=np.uint64))
    ct[:, :, :4] = OP.q - 1
    Ph[:, :4] = OP.q - 1
    ct[:, :, 4:8] = 0
    Ph_full = np.repeat(Ph, dd, axis=1)
    summed = ct.astype(object)
    summed[:, 1] = (summed[:, 1] + A1.astype(object) + A2.astype(object)) % OP.q
    ref = O.homconv(OP, OL, summed.astype(np.uint64), Ph_full, Mh)
    d = lambda a: dev(a.view(np.int64), np.int64)
    Ptc = F.filter_tc(P, L, d(Ph))
    assert Ptc.numel() == F.filter_tc_words(n, p, L)
    out = F.homconv_tc(P, L, d(ct), d(A1), d(A2), Ptc, d(Mh))
    torch.cuda.synchronize()
    assert F.homconv_tc_status() == 0
    assert np.array_equal(u64(out).reshape(ref.shape), ref)
    out = F.homconv_tc(P, L, d(ct), None, None, Ptc, None)
    assert np.array_equal(u64(out).reshape(ref.shape), O.homconv(OP, OL, ct, Ph_full, None))
    # identical to the CUDA-core kernel on the same inputs
    assert torch.equal(F.homconv_tc(P, L, d(ct), d(A1), d(A2), Ptc, d(Mh)),
                       F.homconv_sum(P, L, d(ct), d(A1), d(A2), d(Ph), d(Mh)))
    torch.cuda.synchronize()
    assert F.homconv_tc_status() == 0
    P.close()


def test_homconv_tc_worst_case_digits(F):
    """T = 128 words whose low seven digits are all -128 on both sides: the
    weight class 256^6 then sums 128 x 7 products of +2^14 (14.7 M, the
    largest partial sum the bound allows below 2^24), and q - 1 / 0 words
    exercise the top digit and the zero digits."""
    n, B, Ci, Co, H, W = 1024, 2, 128, 128, 32, 32
    OP = O.params(n, 65537)
    OL = O.layer(OP, B, Ci, Co, H, W, 1, 1)
    P = F.Params(n, 65537, max_T=128)
    L = F.LayerSpec(B, Ci, Co, H, W, 1, 1)
    wbad = _worst_digit_word(OP.q)
    assert wbad < OP.q and all(((wbad + 0x8080808080808080) >> (8 * a)) & 255 == 0 for a in range(7))
    ct = np.full((OL.n_in, 2, n), wbad, np.uint64)
    Ph = np.full((Co * OL.T, n), wbad, np.uint64)
    ct[:, :, 1::3] = OP.q - 1
    Ph[:, 2::5] = 0
    ref = O.homconv(OP, OL, ct, Ph, None)
    d = lambda a: dev(a.view(np.int64), np.int64)
    out = F.homconv_tc(P, L, d(ct), None, None, F.filter_tc(P, L, d(Ph)), None)
    torch.cuda.synchronize()
    assert F.homconv_tc_status() == 0
    assert np.array_equal(u64(out).reshape(ref.shape), ref)
    P.close()


def test_homconv_tc_full_size_binarized_layer(F):
    """The binarized 64x64x128 layer at batch 8 (n = 4096, p = 12289, two
    ciphertexts per spectrum): the tensor-core words equal the CUDA-core
    kernel's at full size, and sampled output words equal the oracle's
    per-word sum."""
    ls = FI.CONFIGS["binarized_64x64x128_b8"].layers[0]
    OP = O.params(ls.n, ls.p)
    OL = O.layer(OP, ls.B, ls.Ci, ls.Co, ls.H, ls.W, 1, 1)
    P = F.Params(ls.n, ls.p, max_T=OL.T)
    L = F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, 1, 1)
    gen = torch.Generator(device="cuda").manual_seed(44)
    q = OP.q
    ct = torch.randint(0, q, (OL.n_in * 2 * ls.n,), dtype=torch.int64, device="cuda", generator=gen)
    dd = OP.d  # one filter word per group of d evaluation indices
    assert F.layout(P, L).filter_words == ls.Co * OL.T * OL.beta * ls.n // dd
    Ph = torch.randint(0, q, (ls.Co * OL.T * OL.beta * ls.n // dd,), dtype=torch.int64, device="cuda", generator=gen)
    Mh = torch.randint(0, q, (OL.n_out * ls.n,), dtype=torch.int64, device="cuda", generator=gen)
    a = F.homconv_tc(P, L, ct, None, None, F.filter_tc(P, L, Ph), Mh)
    b = F.homconv_sum(P, L, ct, None, None, Ph, Mh)
    torch.cuda.synchronize()
    assert F.homconv_tc_status() == 0
    assert torch.equal(a, b)
    ctn, Phn, Mhn, outn = (u64(t) for t in (ct, Ph, Mh, a))
    ctn = ctn.reshape(OL.GB, OL.T, OL.beta, 2, ls.n)
    Phn = Phn.reshape(ls.Co, OL.T, OL.beta, ls.n // dd)
    outn = outn.reshape(OL.GB, ls.Co, OL.beta, 2, ls.n)
    Mhn = Mhn.reshape(OL.GB, ls.Co, OL.beta, ls.n)
    rng = np.random.default_rng(4)
    for _ in range(64):
        bb, co, h, c, j = (int(rng.integers(m)) for m in (OL.GB, ls.Co, OL.beta, 2, ls.n))
        s = sum(int(ctn[bb, k, h, c, j]) * int(Phn[co, k, h, j // dd]) for k in range(OL.T)) % q
        if c == 1:
            s = (s - int(Mhn[bb, co, h, j])) % q
        assert int(outn[bb, co, h, c, j]) == s, (bb, co, h, c, j)
    P.close()


def test_homconv_tc_argument_errors(F):
    """T > 128 is refused (a weight class could reach 2^24), as are outputs
    overlapping an input and misaligned buffers; nothing is launched."""
    P = F.Params(256, 65537, max_T=256)
    L = F.LayerSpec(1, 129, 4, 8, 8, 1, 1)  # T = 129
    lay = F.layout(P, L)
    ct = torch.zeros(lay.ct_in_words, dtype=torch.int64, device="cuda")
    Ph = torch.zeros(lay.filter_words, dtype=torch.int64, device="cuda")
    with pytest.raises(F.FdscError) as e:
        F._call("fdsc_filter_tc", P.handle, F.C.byref(L.c()), Ph.data_ptr(), Ph.data_ptr() + 8 * lay.filter_words, 0)
    assert e.value.code == -5
    with pytest.raises(F.FdscError) as e:
        F._call("fdsc_homconv_tc", P.handle, F.C.byref(L.c()), ct.data_ptr(), None, None, Ph.data_ptr(), None,
                ct.data_ptr() + 8 * lay.ct_in_words, 0)
    assert e.value.code == -5
    L2 = F.LayerSpec(1, 32, 4, 8, 8, 1, 1)
    lay2 = F.layout(P, L2)
    Ptc = torch.zeros(F.filter_tc_words(256, 65537, L2), dtype=torch.int64, device="cuda")
    big = torch.zeros(lay2.ct_in_words + lay2.ct_out_words, dtype=torch.int64, device="cuda")
    with pytest.raises(F.FdscError) as e:  # output overlapping the input
        F._call("fdsc_homconv_tc", P.handle, F.C.byref(L2.c()), big.data_ptr(), None, None, Ptc.data_ptr(), None,
                big.data_ptr() + 8 * 16, 0)
    assert e.value.code == -1
    out = torch.zeros(lay2.ct_out_words + 2, dtype=torch.int64, device="cuda")
    with pytest.raises(F.FdscError) as e:  # misaligned output
        F._call("fdsc_homconv_tc", P.handle, F.C.byref(L2.c()), big.data_ptr(), None, None, Ptc.data_ptr(), None,
                out.data_ptr() + 8, 0)
    assert e.value.code == -1
    torch.cuda.synchronize()
    assert F.homconv_tc_status() == 0
    P.close()
