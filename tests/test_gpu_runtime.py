"""GPU tests of the batching runtime: a plan of several uneven layers in one
graph launch (fused and step-by-step layers, default and autotuned packing)
and the continuous-batching server.  Results are compared word for word with
the oracle; the final shares do not depend on the packing, so the oracle runs
with its default packing."""
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


LAYERS = [  # (n, p, B, Ci, Co, H, W, fh)
    (2048, 65537, 2, 64, 16, 32, 32, 3),
    (2048, 65537, 2, 128, 8, 16, 16, 3),
    (4096, 65537, 2, 256, 4, 8, 8, 3),
    (4096, 12289, 2, 3, 2, 64, 64, 3),   # spectra span two ciphertexts (fused)
    (1024, 65537, 3, 4, 4, 16, 16, 5),
    (512, 65537, 2, 3, 2, 4, 16, 3),     # H = 4 < 8: step-by-step path
]


def _make_layers(F, seed):
    g = np.random.default_rng(seed)
    specs, refs, params = [], [], []
    for i, (n, p, B, Ci, Co, H, W, fh) in enumerate(LAYERS):
        P = F.Params(n, p, max_T=256)
        params.append(P)
        xA = g.integers(0, p, (B, Ci, H, W)).astype(np.uint32)
        xB = g.integers(0, p, (B, Ci, H, W)).astype(np.uint32)
        w = g.integers(-8, 8, (Co, Ci, fh, fh)).astype(np.int8)
        ks, es, ss = 100 + i, 200 + i, 300 + i
        specs.append(dict(params=P, layer=F.LayerSpec(B, Ci, Co, H, W, 0, 0), w=dev(w, np.int8),
                          t_hat=F.keygen(P, ks), enc_seed=es, mask_seed=ss, xA=dev(xA, np.int32),
                          xB=dev(xB, np.int32),
                          yA=torch.empty((B, Co, H, W), dtype=torch.int32, device="cuda"),
                          yB=torch.empty((B, Co, H, W), dtype=torch.int32, device="cuda")))
        OP = O.params(n, p)
        refs.append(O.round_trip(OP, O.layer(OP, B, Ci, Co, H, W), xA, xB, w, ks, es, ss))
    return specs, refs, params


@pytest.mark.parametrize("tune,tensor", [(False, False), (True, False), (False, True)])
def test_plan_of_uneven_layers_matches_oracle(F, tune, tensor):
    """tensor: every layer's HomConv on the tensor cores (all have T <= 128)."""
    specs, refs, params = _make_layers(F, 5 + tune)
    plan = F.Plan(specs, tune=tune, tensor=tensor)
    for rep in range(2):
        for d in specs:
            d["yA"].zero_()
            d["yB"].zero_()
        plan.launch()
        torch.cuda.synchronize()
        for i, (d, ref) in enumerate(zip(specs, refs)):
            assert np.array_equal(u32(d["yA"]).reshape(ref["yA"].shape), ref["yA"]), (i, rep)
            assert np.array_equal(u32(d["yB"]).reshape(ref["yB"].shape), ref["yB"]), (i, rep)
    infos = [plan.info(i) for i in range(len(LAYERS))]
    assert [x.fused for x in infos] == [1, 1, 1, 1, 1, 0]
    if tune:
        assert all(x.candidates > 0 for x, f in zip(infos, [1, 1, 1, 1, 1, 0]) if f)
    if tensor:
        assert [x.homconv_variant for x in infos] == [7] * len(LAYERS)
        assert F.homconv_tc_status() == 0
    plan.close()
    for P in params:
        P.close()


def _server_case(F, g, S, types, pools, OPs):
    t = int(g.integers(len(types)))
    (n, p, Ci, Co, H, W, fh), w = types[t]
    key = int(g.integers(4))
    xA = g.integers(0, p, (Ci, H, W)).astype(np.uint32)
    xB = g.integers(0, p, (Ci, H, W)).astype(np.uint32)
    es, ss = int(g.integers(2**62)), int(g.integers(2**62))
    return dict(t=t, key=key, xA=xA, xB=xB, es=es, ss=ss, yA=np.zeros((Co, H, W), np.uint32),
                yB=np.zeros((Co, H, W), np.uint32))


def test_server_results_same_alone_and_in_the_mix(F):
    g = np.random.default_rng(17)
    types_def = [(2048, 65537, 64, 8, 32, 32, 3), (2048, 65537, 8, 4, 16, 16, 3), (2048, 65537, 1, 4, 32, 32, 5)]
    P = F.Params(2048, 65537, max_T=64)
    OP = O.params(2048, 65537)
    key_seeds = [7, 8, 9, 10]
    keys = torch.stack([F.keygen(P, k) for k in key_seeds]).reshape(-1)
    types = []
    for (n, p, Ci, Co, H, W, fh) in types_def:
        w = g.integers(-8, 8, (Co, Ci, fh, fh)).astype(np.int8)
        types.append(((n, p, Ci, Co, H, W, fh), w))

    def make_server(max_batch, lanes):
        S = F.Server(hbm_budget_bytes=8 << 30, max_batch=max_batch, lanes=lanes)
        ids = [S.add_type(P, F.LayerSpec(1, d[2], d[3], d[4], d[5], 0, 1), dev(w, np.int8), keys)
               for d, w in types]
        S.start()
        return S, ids

    reqs = [_server_case(F, g, None, types, None, None) for _ in range(14)]
    # all at once: batched and overlapped
    S, ids = make_server(max_batch=4, lanes=3)
    tickets = [S.submit(ids[r["t"]], r["key"], r["es"], r["ss"], r["xA"], r["xB"], r["yA"], r["yB"]) for r in reqs]
    for tk in tickets:
        assert S.wait(tk) > 0
    st = S.stats()
    assert st.completed == len(reqs) and st.batches < len(reqs)  # some batches held several requests
    assert st.p99_us >= st.p50_us > 0
    S.close()
    mixed = [(r["yA"].copy(), r["yB"].copy()) for r in reqs]
    # one at a time: every request alone
    S, ids = make_server(max_batch=1, lanes=1)
    for r, (yA_m, yB_m) in zip(reqs, mixed):
        r["yA"][:] = 0
        r["yB"][:] = 0
        S.wait(S.submit(ids[r["t"]], r["key"], r["es"], r["ss"], r["xA"], r["xB"], r["yA"], r["yB"]))
        assert np.array_equal(r["yA"], yA_m) and np.array_equal(r["yB"], yB_m)
    S.close()
    # and both are the oracle's shares for that request alone
    for r in reqs[:5]:
        (n, p, Ci, Co, H, W, fh), w = types[r["t"]]
        OL = O.layer(OP, 1, Ci, Co, H, W)
        ref = O.round_trip(OP, OL, r["xA"][None], r["xB"][None], w, key_seeds[r["key"]], r["es"], r["ss"])
        assert np.array_equal(r["yA"], ref["yA"][0]) and np.array_equal(r["yB"], ref["yB"][0])
    P.close()


def test_server_large_batches_use_the_tensor_cores(F):
    """Batches of 4 or more requests run HomConv on the tensor cores; every
    result is still the oracle's shares for that request alone."""
    g = np.random.default_rng(23)
    types_def = [(2048, 65537, 64, 8, 32, 32, 3), (2048, 65537, 8, 4, 16, 16, 3)]
    P = F.Params(2048, 65537, max_T=64)
    OP = O.params(2048, 65537)
    key_seeds = [11, 12, 13, 14]
    keys = torch.stack([F.keygen(P, k) for k in key_seeds]).reshape(-1)
    types = []
    for (n, p, Ci, Co, H, W, fh) in types_def:
        w = g.integers(-8, 8, (Co, Ci, fh, fh)).astype(np.int8)
        types.append(((n, p, Ci, Co, H, W, fh), w))
    S = F.Server(hbm_budget_bytes=8 << 30, max_batch=8, lanes=1)
    ids = [S.add_type(P, F.LayerSpec(1, d[2], d[3], d[4], d[5], 0, 1), dev(w, np.int8), keys) for d, w in types]
    S.start()
    reqs = []
    for t in (0, 1):
        for _ in range(12):
            r = _server_case(F, g, None, types, None, None)
            (n, p, Ci, Co, H, W, fh), _ = types[t]
            r.update(t=t, xA=g.integers(0, p, (Ci, H, W)).astype(np.uint32),
                     xB=g.integers(0, p, (Ci, H, W)).astype(np.uint32), yA=np.zeros((Co, H, W), np.uint32),
                     yB=np.zeros((Co, H, W), np.uint32))
            reqs.append(r)
    tickets = [S.submit(ids[r["t"]], r["key"], r["es"], r["ss"], r["xA"], r["xB"], r["yA"], r["yB"]) for r in reqs]
    for tk in tickets:
        assert S.wait(tk) > 0
    st = S.stats()
    assert st.completed == len(reqs) and st.tensor_batches >= 1, (st.batches, st.tensor_batches)
    S.close()
    torch.cuda.synchronize()
    assert F.homconv_tc_status() == 0
    for r in reqs:
        (n, p, Ci, Co, H, W, fh), w = types[r["t"]]
        ref = O.round_trip(OP, O.layer(OP, 1, Ci, Co, H, W), r["xA"][None], r["xB"][None], w,
                           key_seeds[r["key"]], r["es"], r["ss"])
        assert np.array_equal(r["yA"], ref["yA"][0]) and np.array_equal(r["yB"], ref["yB"][0])
    P.close()


def _served_mix_refs():
    """The served mix's three layer types at full size, with the requests of
    the full-size server test and the oracle's shares for each alone."""
    c = FI.CONFIGS["served_mix_28x28x1_32x32x64_16x16x128"]
    OP = O.params(2048, 65537)
    key_seeds = [31, 32, 33]
    types = []
    for ti, ls in enumerate(c.layers):
        xA, xB = FI.shares(ls, c.cid, ti)
        types.append((ls, FI.weights(ls, c.cid, ti), np.ascontiguousarray(xA[0], dtype=np.uint32),
                      np.ascontiguousarray(xB[0], dtype=np.uint32)))
    reqs = []
    for i, t in enumerate([1, 1, 1, 0, 2, 1, 2]):
        ls, w, xA, xB = types[t]
        ref = O.round_trip(OP, O.layer(OP, 1, ls.Ci, ls.Co, ls.H, ls.W), xA[None], xB[None], w, key_seeds[i % 3],
                           100 + i, 200 + i)
        reqs.append(dict(t=t, key=i % 3, es=100 + i, ss=200 + i, xA=xA, xB=xB, ref=ref,
                         yA=np.zeros((ls.Co, ls.H, ls.W), np.uint32), yB=np.zeros((ls.Co, ls.H, ls.W), np.uint32)))
    return c, key_seeds, types, reqs


def test_server_served_mix_types_at_full_size(F):
    """The served mix's layer types at their full sizes (28x28 padded to
    32x32, 1 -> 16, 5x5; 32x32x64 -> 64, 3x3; 16x16x128 -> 128, 3x3) through
    the server as the bench runs it (batches of up to 16 on 4 lanes, every
    request its own key and seeds): each result is the oracle's pair of
    shares for that request alone."""
    c, key_seeds, types, reqs = _served_mix_refs()
    P = F.Params(2048, 65537, max_T=64)
    keys = torch.stack([F.keygen(P, k) for k in key_seeds]).reshape(-1)
    S = F.Server(hbm_budget_bytes=c.extra["hbm_budget_bytes"], max_batch=16, lanes=4)
    ids = []
    for ls, w, _, _ in types:
        g_c, _ = FI.default_pack(ls, P.info.S)
        ids.append(S.add_type(P, F.LayerSpec(1, ls.Ci, ls.Co, ls.H, ls.W, g_c, 1), dev(w, np.int8), keys))
    S.start()
    tickets = [S.submit(ids[r["t"]], r["key"], r["es"], r["ss"], r["xA"], r["xB"], r["yA"], r["yB"]) for r in reqs]
    for tk in tickets:
        assert S.wait(tk) > 0
    assert S.stats().completed == len(reqs)
    S.close()
    for r in reqs:
        assert np.array_equal(r["yA"], r["ref"]["yA"][0]) and np.array_equal(r["yB"], r["ref"]["yB"][0]), r["t"]
    P.close()


def test_server_budget_and_timeouts(F):
    P = F.Params(2048, 65537, max_T=64)
    keys = F.keygen(P, 1)
    w = dev(np.ones((8, 64, 3, 3), np.int8), np.int8)
    S = F.Server(hbm_budget_bytes=1 << 20, max_batch=4, lanes=2)  # 1 MiB: less than one request needs
    S.add_type(P, F.LayerSpec(1, 64, 8, 32, 32, 0, 1), w, keys)
    with pytest.raises(F.FdscError) as e:
        S.start()
    assert e.value.code == -7
    S.close()
    S = F.Server(hbm_budget_bytes=1 << 30, max_batch=4, lanes=2)
    tid = S.add_type(P, F.LayerSpec(1, 64, 8, 32, 32, 0, 1), w, keys)
    S.start()
    x = np.zeros((64, 32, 32), np.uint32)
    y = np.zeros((8, 32, 32), np.uint32)
    with pytest.raises(F.FdscError) as e:
        S.wait(12345, timeout_ms=20)  # a ticket nobody submitted
    assert e.value.code == -6
    with pytest.raises(F.FdscError) as e:
        S.submit(tid, 5, 1, 2, x, x, y, y)  # key outside the pool
    assert e.value.code == -1
    S.close()
    P.close()


def test_server_budget_bounds_device_memory(F):
    """The budget sizes the lanes' device buffers: with room for 2.5
    requests and 4 lanes asked, two lanes of one request each are made and
    the device memory fdsc_server_start takes stays within the budget (plus
    the recorded graphs); a large budget gives lanes x max_batch requests'
    worth.  Requests under the small budget give the same shares."""
    P = F.Params(2048, 65537, max_T=64)
    keys = torch.stack([F.keygen(P, k) for k in (3, 4)]).reshape(-1)
    g = np.random.default_rng(9)
    w = g.integers(-8, 8, (16, 64, 3, 3)).astype(np.int8)
    L = F.LayerSpec(1, 64, 16, 32, 32, 0, 1)

    def started(budget, lanes, max_batch):
        S = F.Server(hbm_budget_bytes=budget, max_batch=max_batch, lanes=lanes)
        tid = S.add_type(P, L, dev(w, np.int8), keys)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        S.start()
        torch.cuda.synchronize()
        return S, tid, free0 - torch.cuda.mem_get_info()[0]

    big, tid_b, drop_big = started(8 << 30, 4, 16)
    stb = big.stats()
    assert (stb.lanes, stb.lane_capacity) == (4, 16)
    assert drop_big >= stb.reserved_bytes > 0
    per = stb.reserved_bytes / 64  # one request slot of one lane
    budget = int(2.5 * per)
    small, tid_s, drop_small = started(budget, 4, 16)
    st = small.stats()
    assert (st.lanes, st.lane_capacity) == (2, 1) and st.reserved_bytes <= budget
    assert drop_small <= budget + (32 << 20) < drop_big
    outs = {}
    for name, S, tid in (("big", big, tid_b), ("small", small, tid_s)):
        rng = np.random.default_rng(21)
        res = []
        tickets = []
        for i in range(6):
            xa = rng.integers(0, 65537, (64, 32, 32)).astype(np.uint32)
            xb = rng.integers(0, 65537, (64, 32, 32)).astype(np.uint32)
            ya, yb = np.zeros((16, 32, 32), np.uint32), np.zeros((16, 32, 32), np.uint32)
            res.append((xa, xb, ya, yb))
            tickets.append(S.submit(tid, i % 2, 40 + i, 50 + i, xa, xb, ya, yb))
        for tk in tickets:
            S.wait(tk)
        outs[name] = [(ya.copy(), yb.copy()) for _, _, ya, yb in res]
        assert S.stats().completed == 6
        S.close()
    for (a1, b1), (a2, b2) in zip(outs["big"], outs["small"]):
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    P.close()


def test_server_latency_histogram_percentiles(F):
    """The latency record is a fixed histogram: its percentiles lie within a
    bin (0.45 %) of the sorted latencies the waiters saw."""
    P = F.Params(2048, 65537, max_T=64)
    keys = F.keygen(P, 2)
    w = dev(np.ones((4, 4, 3, 3), np.int8), np.int8)
    S = F.Server(hbm_budget_bytes=1 << 30, max_batch=4, lanes=2)
    tid = S.add_type(P, F.LayerSpec(1, 4, 4, 16, 16, 0, 1), w, keys)
    S.start()
    x = np.ones((4, 16, 16), np.uint32)
    lat = []
    for i in range(200):
        y1, y2 = np.zeros((4, 16, 16), np.uint32), np.zeros((4, 16, 16), np.uint32)
        lat.append(S.wait(S.submit(tid, 0, i, i, x, x, y1, y2)))
    st = S.stats()
    v = np.sort(lat)
    for q, got in ((0.50, st.p50_us), (0.99, st.p99_us)):
        ref = v[min(len(v) - 1, int(q * (len(v) - 1) + 0.5))]
        assert abs(got - ref) <= 0.005 * ref, (q, got, ref)
    assert abs(st.max_us - v[-1]) < 1e-6 * v[-1] and abs(st.mean_us - v.mean()) < 1e-6 * v.mean()
    S.close()
    P.close()


def test_launch_overlap_gives_identical_results(F):
    """Programmatic dependent launch changes when kernels start, not what
    they compute: a plan captured with and without it, and eager calls in
    one stream, give the same words."""
    specs, refs, params = _make_layers(F, 11)
    prev = F.set_launch_overlap(False)
    try:
        plan_off = F.Plan(specs[:3])
        F.set_launch_overlap(True)
        plan_on = F.Plan(specs[:3])
        for plan in (plan_off, plan_on, plan_off, plan_on):
            for d in specs[:3]:
                d["yA"].zero_()
                d["yB"].zero_()
            plan.launch()
            torch.cuda.synchronize()
            for d, ref in zip(specs[:3], refs[:3]):
                assert np.array_equal(u32(d["yA"]).reshape(ref["yA"].shape), ref["yA"])
                assert np.array_equal(u32(d["yB"]).reshape(ref["yB"].shape), ref["yB"])
        plan_off.close()
        plan_on.close()
    finally:
        F.set_launch_overlap(prev)
    for P in params:
        P.close()


def test_pool2x2_sum_matches_oracle(F):
    P = F.Params(1024, 65537, max_T=8)
    g = np.random.default_rng(21)
    x = g.integers(0, 65537, (3, 5, 16, 12)).astype(np.uint32)
    y = F.pool2x2_sum(P, dev(x, np.int32))
    torch.cuda.synchronize()
    assert np.array_equal(u32(y).reshape(3, 5, 8, 6), O.pool2x2_sum(65537, x))
    with pytest.raises(F.FdscError):
        F.pool2x2_sum(P, dev(np.zeros((1, 3, 5), np.uint32), np.int32))  # odd plane
    P.close()


@pytest.mark.parametrize("tensor", [False, True])
def test_chained_plan_of_a_network_matches_oracle(F, tensor):
    """The appendix network's pattern at reduced width: conv, sum pooling,
    conv, 1x1 conv, run as one chained plan (each layer reads the shares the
    previous one wrote) and compared with the oracle run layer by layer;
    tensor: every layer's HomConv on the tensor cores."""
    p, n = 65537, 1024
    P = F.Params(n, p, max_T=64)
    OP = O.params(n, p)
    g = np.random.default_rng(31)
    shapes = [(3, 8, 16, 3, True), (8, 8, 8, 3, False), (8, 4, 8, 1, False)]  # (Ci, Co, H, fh, pool after)
    xA = g.integers(0, p, (1, 3, 16, 16)).astype(np.uint32)
    xB = g.integers(0, p, (1, 3, 16, 16)).astype(np.uint32)
    specs, ws, seeds = [], [], []
    inA, inB = dev(xA, np.int32), dev(xB, np.int32)
    for i, (Ci, Co, H, fh, pool) in enumerate(shapes):
        w = g.integers(-8, 8, (Co, Ci, fh, fh)).astype(np.int8)
        ks, es, ss = 40 + i, 50 + i, 60 + i
        d = dict(params=P, layer=F.LayerSpec(1, Ci, Co, H, H, 0, 0), w=dev(w, np.int8), t_hat=F.keygen(P, ks),
                 enc_seed=es, mask_seed=ss, xA=inA, xB=inB,
                 yA=torch.zeros((1, Co, H, H), dtype=torch.int32, device="cuda"),
                 yB=torch.zeros((1, Co, H, H), dtype=torch.int32, device="cuda"))
        if pool:
            d["pA"] = torch.zeros((1, Co, H // 2, H // 2), dtype=torch.int32, device="cuda")
            d["pB"] = torch.zeros_like(d["pA"])
        inA, inB = (d["pA"], d["pB"]) if pool else (d["yA"], d["yB"])
        specs.append(d)
        ws.append(w)
        seeds.append((ks, es, ss))
    plan = F.Plan(specs, chain=True, tensor=tensor)
    if tensor:
        assert [plan.info(i).homconv_variant for i in range(len(shapes))] == [7] * len(shapes)
    for _ in range(2):
        plan.launch()
        torch.cuda.synchronize()
        a, b = xA, xB
        for (Ci, Co, H, fh, pool), w, (ks, es, ss), d in zip(shapes, ws, seeds, specs):
            ref = O.round_trip(OP, O.layer(OP, 1, Ci, Co, H, H), a, b, w, ks, es, ss)
            assert np.array_equal(u32(d["yA"]).reshape(ref["yA"].shape), ref["yA"])
            assert np.array_equal(u32(d["yB"]).reshape(ref["yB"].shape), ref["yB"])
            a, b = ref["yA"], ref["yB"]
            if pool:
                a, b = O.pool2x2_sum(p, a), O.pool2x2_sum(p, b)
                assert np.array_equal(u32(d["pA"]).reshape(a.shape), a)
                assert np.array_equal(u32(d["pB"]).reshape(b.shape), b)
    plan.close()
    P.close()


def test_noise_flooding_masks_and_shares(F):
    """HomShare flooding: the mask words are the oracle's, and the final
    shares of the fused path and of a plan equal the unflooded oracle run."""
    n, p = 1024, 65537
    P = F.Params(n, p, max_T=8)
    OP = O.params(n, p)
    B, Ci, Co, H = 1, 4, 4, 16
    OL = O.layer(OP, B, Ci, Co, H, H)
    L = F.LayerSpec(B, Ci, Co, H, H, OL.g_c, OL.g_b)
    f = F.flood_bits_max(n, p, OL.T)
    M, sB = F.mask_prepare_flooded(P, L, 33, f)
    Mo, sBo = O.mask_prepare(OP, OL, 33, f)
    torch.cuda.synchronize()
    assert np.array_equal(u64(M).reshape(Mo.shape), Mo) and np.array_equal(u32(sB).reshape(sBo.shape), sBo)
    with pytest.raises(F.FdscError) as e:
        F.mask_prepare_flooded(P, L, 33, f + 1)
    assert e.value.code == -2
    g = np.random.default_rng(5)
    xA = g.integers(0, p, (B, Ci, H, H)).astype(np.uint32)
    xB = g.integers(0, p, (B, Ci, H, H)).astype(np.uint32)
    w = g.integers(-8, 8, (Co, Ci, 3, 3)).astype(np.int8)
    ref = O.round_trip(OP, OL, xA, xB, w, 1, 2, 33)
    t_hat = F.keygen(P, 1)
    Ph = F.filter_prepare(P, L, dev(w, np.int8))
    ct = F.encrypt_constants(P, L, t_hat, 2)
    out = F.homconv_sum(P, L, ct, F.encode_share(P, L, dev(xA, np.int32)), F.encode_share(P, L, dev(xB, np.int32)),
                        Ph, M)
    yA = F.decrypt_share(P, L, t_hat, out)
    torch.cuda.synchronize()
    assert np.array_equal(u32(yA).reshape(ref["yA"].shape), ref["yA"])
    d = dict(params=P, layer=F.LayerSpec(B, Ci, Co, H, H, 0, 0), w=dev(w, np.int8), t_hat=t_hat, enc_seed=2,
             mask_seed=33, xA=dev(xA, np.int32), xB=dev(xB, np.int32), flood_bits=f,
             yA=torch.zeros((B, Co, H, H), dtype=torch.int32, device="cuda"),
             yB=torch.zeros((B, Co, H, H), dtype=torch.int32, device="cuda"))
    plan = F.Plan([d], tune=True)
    plan.launch()
    torch.cuda.synchronize()
    assert np.array_equal(u32(d["yA"]).reshape(ref["yA"].shape), ref["yA"])
    assert np.array_equal(u32(d["yB"]).reshape(ref["yB"].shape), ref["yB"])
    plan.close()
    P.close()


def test_calibration_rates_are_plausible(F):
    """The measured rates of the exact primitives: positive, below the
    SM's issue rate (128 thread-instructions per clock), the 128-bit MAC
    slower than a 32-bit modular multiply."""
    P = F.Params(2048, 65537, max_T=8)
    rates = [F.calibrate(P, i) for i in range(3)]
    for per_s, per_clk in rates:
        assert per_s > 0 and 0 < per_clk < 128
    assert rates[0][1] < rates[2][1]
    with pytest.raises(F.FdscError):
        F.calibrate(P, 3)
    P.close()


def test_new_entry_points_reject_bad_arguments(F):
    """Argument checks of the seeded, pooling and flooding calls: errors
    come back as status codes, nothing is launched."""
    P = F.Params(64, 65537, max_T=400)
    L = F.LayerSpec(1, 300, 3, 8, 8, 1, 1)  # T = 300 input ciphertexts: more than the seeded HomConv stages
    lay = F.layout(P, L)
    c1 = torch.zeros(lay.n_in * 64, dtype=torch.int64, device="cuda")
    Ph = torch.zeros(lay.filter_words, dtype=torch.int64, device="cuda")
    with pytest.raises(F.FdscError) as e:
        F.homconv_seeded(P, L, 1, c1, None, None, Ph)
    assert e.value.code == -5
    x = torch.zeros((2, 8, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(F.FdscError) as e:
        F.pool2x2_sum(P, x, out=x.view(-1)[: 2 * 16].view(2, 4, 4))  # output inside the input
    assert e.value.code == -1
    xin = torch.zeros((1, 3, 8, 8), dtype=torch.int32, device="cuda")
    yout = torch.zeros((1, 2, 8, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(F.FdscError) as e:  # a plan layer whose flooding breaks the bound
        F.Plan([dict(params=P, layer=F.LayerSpec(1, 3, 2, 8, 8, 0, 0),
                     w=dev(np.ones((2, 3, 3, 3), np.int8), np.int8), t_hat=F.keygen(P, 1), enc_seed=1, mask_seed=2,
                     xA=xin, xB=xin, yA=yout, yB=yout.clone(), flood_bits=60)])
    assert e.value.code == -2
    P.close()
