"""GPU parity of the fused online path: encryption constants, spatial share
encoding, HomRec from a spatial share, HomConv over summed c1 addends and the
fused decrypt + INTT2D produce exactly the words of the step-by-step oracle
(Fig. 2; Enc(m) = Enc(0) + (0, NTT_q(Delta m)) by linearity of NTT_q)."""
import numpy as np
import pytest
import torch

import fdsc_inputs as FI
from fdsc_harness import dev, u32, u64
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


CASES = [
    dict(n=1024, p=65537, B=1, Ci=4, Co=4, H=16, W=16, fh=3),                      # single small layer
    dict(n=2048, p=65537, B=1, Ci=64, Co=64, H=32, W=32, fh=3),                    # CIFAR-shaped layer
    dict(n=2048, p=65537, B=1, Ci=1, Co=16, H=32, W=32, fh=5, support=(28, 28)),   # MNIST-shaped layer
    dict(n=2048, p=65537, B=2, Ci=128, Co=8, H=16, W=16, fh=3),                    # 16x16, g_c = 8
    dict(n=4096, p=65537, B=2, Ci=256, Co=4, H=8, W=8, fh=3),                      # 8x8, g_c = 64
    dict(n=4096, p=65537, B=3, Ci=40, Co=3, H=8, W=8, fh=3, g_c=16, g_b=4),        # image blocks, ragged B
    dict(n=4096, p=12289, B=5, Ci=3, Co=2, H=16, W=16, fh=3, g_c=2, g_b=3),        # two slot sets (d = 2)
    dict(n=256, p=65537, B=3, Ci=5, Co=3, H=8, W=8, fh=3, g_c=2, g_b=2),           # small ring, ragged
    dict(n=1024, p=65537, B=1, Ci=2, Co=2, H=8, W=128, fh=3, fw=5),                # wide plane
    dict(n=2048, p=147457, B=1, Ci=64, Co=64, H=32, W=32, fh=3),                   # Table 2 "Medium" prime
    dict(n=1024, p=786433, B=3, Ci=6, Co=3, H=16, W=16, fh=3, g_c=2, g_b=2),       # p = 3 2^18 + 1, near 2^20
    # spectra spanning several ciphertexts (H W > S)
    dict(n=4096, p=12289, B=3, Ci=3, Co=2, H=64, W=64, fh=3, g_c=1),              # d = 2, beta = 2, ragged B
    dict(n=1024, p=65537, B=1, Ci=2, Co=2, H=64, W=64, fh=3, g_c=1),              # d = 1, beta = 4
    dict(n=2048, p=65537, B=2, Ci=3, Co=2, H=32, W=128, fh=3, fw=5, g_c=1),        # beta = 2, wide plane
]


@pytest.mark.parametrize("args", CASES)
def test_fused_path_bit_exact(F, args):
    args = dict(args)
    n, p, B, Ci, Co, H, W, fh = (args.pop(k) for k in ("n", "p", "B", "Ci", "Co", "H", "W", "fh"))
    fw = args.pop("fw", fh)
    g_c, g_b, support = args.pop("g_c", None), args.pop("g_b", 1), args.pop("support", None)
    OP = O.params(n, p)
    OL = O.layer(OP, B, Ci, Co, H, W, g_c, g_b)
    P = F.Params(n, p, max_T=max(OL.T, 1))
    L = F.LayerSpec(B, Ci, Co, H, W, OL.g_c, OL.g_b)
    g = np.random.default_rng(n + Ci + 7 * B)
    h, w_ = support or (H, W)
    xA = np.zeros((B, Ci, H, W), np.uint32)
    xB = np.zeros((B, Ci, H, W), np.uint32)
    xA[:, :, :h, :w_] = g.integers(0, p, (B, Ci, h, w_))
    xB[:, :, :h, :w_] = g.integers(0, p, (B, Ci, h, w_))
    w = g.integers(-8, 8, (Co, Ci, fh, fw)).astype(np.int8)
    ks, es, ss = 71, 72, 73
    ref = O.round_trip(OP, OL, xA, xB, w, ks, es, ss)
    q = OP.q

    t_hat = F.keygen(P, ks)
    Phat = F.filter_prepare(P, L, dev(w, np.int8))
    Mhat, sB = F.mask_prepare(P, L, ss)
    C0 = F.encrypt_constants(P, L, t_hat, es)
    zero = np.zeros((B, Ci, H * W), np.uint32)
    assert np.array_equal(u64(C0).reshape(OL.n_in, 2, n), O.encrypt(OP, OL, ref["t_hat"], zero, es))
    dA, dB = dev(xA, np.int32), dev(xB, np.int32)
    A = F.encode_share(P, L, dA)
    Bsh = F.encode_share(P, L, dB)
    # constants + message = encryption; + Bob's plaintext = HomRec
    got_enc = u64(C0).reshape(OL.n_in, 2, n).astype(object)
    got_enc[:, 1] = (got_enc[:, 1] + u64(A).reshape(OL.n_in, n).astype(object)) % q
    assert np.array_equal(got_enc.astype(np.uint64), ref["ct_enc"])
    ct = F.encrypt_constants(P, L, t_hat, es)
    F.homrec_share(P, L, dA, ct)
    F.homrec_share(P, L, dB, ct)
    assert np.array_equal(u64(ct).reshape(ref["ct_rec"].shape), ref["ct_rec"])
    out = F.homconv_sum(P, L, C0, A, Bsh, Phat, Mhat)
    assert np.array_equal(u64(out).reshape(ref["ct_out"].shape), ref["ct_out"])
    out1 = F.homconv_sum(P, L, ct, None, None, Phat, Mhat)
    assert torch.equal(out, out1)
    yA = F.decrypt_share(P, L, t_hat, out)
    assert np.array_equal(u32(yA).reshape(ref["yA"].shape), ref["yA"])
    # the three producers in one launch (with the L2 prefetch of HomConv's
    # operands, and without): the same words as the separate calls
    for pf in ((Phat, Mhat), (None, None)):
        ct3, A3, R3 = F.online_produce(P, L, t_hat, es, dA, dB, P_hat=pf[0], M_hat=pf[1])
        assert torch.equal(ct3, C0) and torch.equal(A3, A) and torch.equal(R3, Bsh)
    torch.cuda.synchronize()
    P.close()


def test_fused_path_rejects_unsupported_shapes(F):
    P = F.Params(1024, 65537)
    L2 = F.LayerSpec(1, 2, 2, 4, 64, 1, 1)  # H = 4 < 8: no radix-8 column passes
    with pytest.raises(F.FdscError) as e:
        F.encode_share(P, L2, torch.zeros(2 * 4 * 64, dtype=torch.int32, device="cuda"))
    assert e.value.code == -5
    P.close()


def test_multi_client_batch_equals_single_requests(F):
    """Three clients (own key, encryption seed and HomShare seed) in one
    launch: every client's ciphertexts and shares are the words of the oracle
    run on that client alone."""
    n, p, Ci, Co, H, W, G = 2048, 65537, 64, 8, 32, 32, 3
    OP = O.params(n, p)
    OL1 = O.layer(OP, 1, Ci, Co, H, W, 2, 1)
    P = F.Params(n, p, max_T=OL1.T)
    LB = F.LayerSpec(G, Ci, Co, H, W, 2, 1)
    g = np.random.default_rng(99)
    xA = g.integers(0, p, (G, Ci, H, W)).astype(np.uint32)
    xB = g.integers(0, p, (G, Ci, H, W)).astype(np.uint32)
    w = g.integers(-8, 8, (Co, Ci, 3, 3)).astype(np.int8)
    ks = [11, 12, 13]
    es = [int(v) for v in g.integers(0, 2**62, G)]
    ss = [int(v) for v in g.integers(0, 2**62, G)]
    t_hats = torch.stack([F.keygen(P, k) for k in ks]).reshape(-1)
    seeds_e = torch.tensor(es, dtype=torch.int64, device="cuda")
    seeds_s = torch.tensor(ss, dtype=torch.int64, device="cuda")
    Phat = F.filter_prepare(P, LB, dev(w, np.int8))
    C0 = F.encrypt_constants_multi(P, LB, t_hats, seeds_e)
    M, sB = F.mask_prepare_multi(P, LB, seeds_s)
    A = F.encode_share(P, LB, dev(xA, np.int32))
    R = F.encode_share(P, LB, dev(xB, np.int32))
    out = F.homconv_sum(P, LB, C0, A, R, Phat, M)
    yA = F.decrypt_share_multi(P, LB, t_hats, out)
    yB = F.intt2d(P, sB.view(G, Co, H, W))
    yA_n, yB_n = u32(yA).reshape(G, Co, H, W), u32(yB).reshape(G, Co, H, W)
    C0_n = u64(C0).reshape(G, OL1.n_in, 2, n)
    for i in range(G):
        ref = O.round_trip(OP, OL1, xA[i:i + 1], xB[i:i + 1], w, ks[i], es[i], ss[i])
        zero = np.zeros((1, Ci, H * W), np.uint32)
        assert np.array_equal(C0_n[i], O.encrypt(OP, OL1, ref["t_hat"], zero, es[i])), i
        assert np.array_equal(yA_n[i], ref["yA"][0]), i
        assert np.array_equal(yB_n[i], ref["yB"][0]), i
        y = O.conv_plain(p, (xA[i:i + 1].astype(np.int64) + xB[i:i + 1]) % p, w)[0]
        assert np.array_equal((yA_n[i].astype(np.int64) + yB_n[i]) % p, y)
    P.close()


def test_binarized_layer_full_size_fused_path(F):
    """The binarized 64x64x128 layer at batch 8 (n = 4096, p = 12289: two
    slot sets per ciphertext, each spectrum over two ciphertexts) through the
    fused kernels at full size, HomConv on the tensor cores and on the CUDA
    cores: both give the same words, and s_A + s_B is the convolution of
    x_A + x_B with the filters on sampled planes."""
    ls = FI.CONFIGS["binarized_64x64x128_b8"].layers[0]
    cid = FI.CONFIGS["binarized_64x64x128_b8"].cid
    P = F.Params(ls.n, ls.p, max_T=ls.Ci)
    L = F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, 1, 1)
    xA, xB = FI.shares(ls, cid)
    w = FI.weights(ls, cid)
    ks, es, ss = FI.seeds(cid)
    t_hat = F.keygen(P, ks)
    Phat = F.filter_prepare(P, L, dev(w, np.int8))
    Mhat, sB = F.mask_prepare(P, L, ss)
    ct, A, R = F.online_produce(P, L, t_hat, es, dev(xA, np.int32), dev(xB, np.int32), P_hat=Phat, M_hat=Mhat)
    out = F.homconv_tc(P, L, ct, A, R, F.filter_tc(P, L, Phat), Mhat)
    assert torch.equal(out, F.homconv_sum(P, L, ct, A, R, Phat, Mhat))
    yA = F.decrypt_share(P, L, t_hat, out)
    yB = F.intt2d(P, sB.view(ls.B, ls.Co, ls.H, ls.W))
    torch.cuda.synchronize()
    assert F.homconv_tc_status() == 0
    y = (u32(yA).reshape(ls.B, ls.Co, ls.H, ls.W).astype(np.int64) +
         u32(yB).reshape(ls.B, ls.Co, ls.H, ls.W)) % ls.p
    x = (xA.astype(np.int64) + xB) % ls.p
    rng = np.random.default_rng(cid)
    for _ in range(4):
        b, co = int(rng.integers(ls.B)), int(rng.integers(ls.Co))
        assert np.array_equal(y[b, co], O.conv_plain(ls.p, x[b:b + 1], w[co:co + 1])[0, 0]), (b, co)
    P.close()


def test_decrypt_pair_switch_gives_the_same_words(F):
    """One image's decryption on CTA pairs (the default) and on one CTA per
    ciphertext (fdsc_set_decrypt_pair(0)) write the same shares."""
    n, p, Ci, Co, H, W = 2048, 65537, 64, 64, 32, 32
    P = F.Params(n, p, max_T=64)
    L = F.LayerSpec(1, Ci, Co, H, W, 2, 1)
    lay = F.layout(P, L)
    g = torch.Generator(device="cuda").manual_seed(3)
    q = P.info.q
    ct = torch.randint(0, q, (lay.ct_out_words,), dtype=torch.int64, device="cuda", generator=g)
    t_hat = F.keygen(P, 5)
    a = F.decrypt_share(P, L, t_hat, ct)
    old = F.set_decrypt_pair(False)
    try:
        b = F.decrypt_share(P, L, t_hat, ct)
    finally:
        F.set_decrypt_pair(old)
    torch.cuda.synchronize()
    assert old and torch.equal(a, b)
    P.close()


_PIPELINE_REFS = {}


@pytest.mark.parametrize("pair", [False, True])
def test_stage_pipelined_steps_match_the_oracle(F, pair):
    """The timed schedule of the one-image 32x32x64 layer: consecutive steps
    (three instances with their own weights, keys, seeds and shares, cycled
    over seven steps) pipelined by stage -- every step's producers in one
    launch on a producer stream, its HomConv on one of two HomConv streams,
    its decryption on one of two decryption streams, Bob's INTT2D on a
    stream of its own -- with programmatic dependent launch, run eagerly and
    as one CUDA graph replayed twice: every step's two output shares are the
    oracle's words for its instance (pair: decryption on CTA pairs)."""
    c = FI.CONFIGS["cifar_32x32x64_b1"]
    ls = c.layers[0]
    OP = O.params(ls.n, ls.p)
    info = F.params_query(ls.n, ls.p)
    g_c, g_b = FI.default_pack(ls, info.S)
    OL = O.layer(OP, ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
    P = F.Params(ls.n, ls.p, max_T=OL.T)
    L = F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
    lay = F.layout(P, L)
    R, G = 3, 7
    insts, refs = [], []
    for r in range(R):
        xA, xB = FI.shares(ls, c.cid, r)
        w = FI.weights(ls, c.cid, r)
        ks, es, ss = FI.seeds(c.cid, r)
        if r not in _PIPELINE_REFS:  # the oracle takes a few seconds per instance
            _PIPELINE_REFS[r] = O.round_trip(OP, OL, xA, xB, w, ks, es, ss)
        refs.append(_PIPELINE_REFS[r])
        d = dict(es=es, t_hat=F.keygen(P, ks), Phat=F.filter_prepare(P, L, dev(w, np.int8)),
                 xA=dev(xA, np.int32), xB=dev(xB, np.int32))
        d["Mhat"], sB = F.mask_prepare(P, L, ss)
        d["sB4"] = sB.view(ls.B, ls.Co, ls.H, ls.W)
        insts.append(d)

    def buffers():
        return dict(ct=torch.empty(lay.ct_in_words, dtype=torch.int64, device="cuda"),
                    A=torch.empty(lay.n_in * ls.n, dtype=torch.int64, device="cuda"),
                    R=torch.empty(lay.n_in * ls.n, dtype=torch.int64, device="cuda"),
                    out=torch.empty(lay.ct_out_words, dtype=torch.int64, device="cuda"),
                    yA=torch.zeros((ls.B, ls.Co, ls.H, ls.W), dtype=torch.int32, device="cuda"),
                    yB=torch.zeros((ls.B, ls.Co, ls.H, ls.W), dtype=torch.int32, device="cuda"))

    bufs = [buffers() for _ in range(G)]
    s_prod = torch.cuda.Stream()
    s_hc = [torch.cuda.Stream(), torch.cuda.Stream()]
    s_dec = [torch.cuda.Stream(), torch.cuda.Stream()]
    s_bob = torch.cuda.Stream()
    streams = [s_prod, s_bob] + s_hc + s_dec

    def steps():
        main = torch.cuda.current_stream()
        for st in streams:
            st.wait_stream(main)
        for i, o in enumerate(bufs):
            d = insts[i % R]
            with torch.cuda.stream(s_prod):
                F.online_produce(P, L, d["t_hat"], d["es"], d["xA"], d["xB"], o["ct"], o["A"], o["R"])
                produced = torch.cuda.Event()
                produced.record(s_prod)
            with torch.cuda.stream(s_bob):
                F.intt2d(P, d["sB4"], out=o["yB"])
            sh, sd = s_hc[i % 2], s_dec[i % 2]
            with torch.cuda.stream(sh):
                sh.wait_event(produced)
                F.homconv_sum(P, L, o["ct"], o["A"], o["R"], d["Phat"], d["Mhat"], out=o["out"])
                convolved = torch.cuda.Event()
                convolved.record(sh)
            with torch.cuda.stream(sd):
                sd.wait_event(convolved)
                F.decrypt_share(P, L, d["t_hat"], o["out"], out=o["yA"])
        for st in streams:
            main.wait_stream(st)

    def check():
        torch.cuda.synchronize()
        for i, o in enumerate(bufs):
            ref = refs[i % R]
            assert np.array_equal(u32(o["yA"]).reshape(ref["yA"].shape), ref["yA"]), i
            assert np.array_equal(u32(o["yB"]).reshape(ref["yB"].shape), ref["yB"]), i
            o["yA"].zero_()
            o["yB"].zero_()
        torch.cuda.synchronize()

    prev_overlap = F.set_launch_overlap(True)
    prev_pair = F.set_decrypt_pair(pair)
    try:
        steps()
        check()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(graph, stream=s):
                steps()
        torch.cuda.current_stream().wait_stream(s)
        for _ in range(2):
            graph.replay()
            check()
    finally:
        F.set_launch_overlap(prev_overlap)
        F.set_decrypt_pair(prev_pair)
    P.close()
