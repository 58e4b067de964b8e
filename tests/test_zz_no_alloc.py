"""The allocation-free layer entry point (for callers that must not let the
library allocate device memory: applications whose device memory belongs to
their own pooling allocator, and request threads that must never enter the
CUDA allocator).  Called through the C ABI, it must give exactly the words of
the existing fused entry points, on two calls in a row that share the fixed
device array.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

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


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()


@pytest.mark.parametrize("n,p,B,Ci,Co,H,W,g_c,g_b", [
    (2048, 65537, 1, 64, 64, 32, 32, 2, 1),   # the 32x32x64 layer
    (1024, 65537, 1, 4, 4, 16, 16, 4, 1),     # the 16x16 4 -> 4 layer
    (2048, 65537, 3, 16, 24, 16, 16, 4, 2),   # Ci != Co, several images per slot set, a ragged last group
    (4096, 12289, 4, 3, 5, 16, 16, 2, 2),     # two slot sets per ciphertext
])
def test_noalloc_layer_matches_existing_entry_points_twice(F, n, p, B, Ci, Co, H, W, g_c, g_b):
    P = F.Params(n, p, max_T=64)
    L = F.LayerSpec(B, Ci, Co, H, W, g_c, g_b)
    g = np.random.default_rng(2024)
    w = _dev(g.integers(-8, 8, (Co, Ci, 3, 3)), np.int8)
    t_hat = F.keygen(P, 31)
    Phat = F.filter_prepare(P, L, w)
    results = []
    for call in range(2):  # two calls in a row, different inputs, seeds and masks
        xA = _dev(g.integers(0, p, (B, Ci, H, W)), np.int32)
        xB = _dev(g.integers(0, p, (B, Ci, H, W)), np.int32)
        es, ss = 1000 + call, 2000 + call
        Mhat, sB = F.mask_prepare(P, L, ss)
        # existing entry points, caller-allocated intermediates
        ct = F.encrypt_constants(P, L, t_hat, es)
        A = F.encode_share(P, L, xA)
        R = F.encode_share(P, L, xB)
        out = F.homconv_sum(P, L, ct, A, R, Phat, Mhat)
        yA_ref = F.decrypt_share(P, L, t_hat, out)
        yB_ref = F.intt2d(P, sB.view(B, Co, H, W))
        # the allocation-free entry point
        yA = torch.empty((B, Co, H, W), dtype=torch.int32, device="cuda")
        yB = torch.empty_like(yA)
        F.layer_online_noalloc(P, L, t_hat, es, Phat, Mhat, sB, xA, xB, yA, yB)
        torch.cuda.synchronize()
        assert torch.equal(yA, yA_ref), call
        assert torch.equal(yB, yB_ref), call
        results.append((yA.clone(), yB.clone()))
    assert not torch.equal(results[0][0], results[1][0])  # the second call really recomputed
    P.close()


def test_noalloc_rejects_layers_beyond_the_fixed_array(F):
    P = F.Params(2048, 65537, max_T=64)
    L = F.LayerSpec(16, 64, 64, 32, 32, 2, 1)  # 16 images: 64 MiB of intermediate ciphertexts
    lay = F.layout(P, L)
    z32 = lambda k: torch.zeros(k, dtype=torch.int32, device="cuda")
    z64 = lambda k: torch.zeros(k, dtype=torch.int64, device="cuda")
    with pytest.raises(F.FdscError) as e:
        F.layer_online_noalloc(P, L, z64(P.n), 1, z64(lay.filter_words), z64(lay.mask_words),
                               z32(lay.out_spectra_words), z32(lay.in_spectra_words), z32(lay.in_spectra_words),
                               z32(lay.out_spectra_words), z32(lay.out_spectra_words))
    assert e.value.code == -5 and "fixed array" in str(e.value)
    P.close()
