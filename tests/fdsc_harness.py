"""Shared helpers for the GPU parity tests: run one layer through the CUDA
path (via the Python binding of the C ABI) and through the CPU oracle on the
same seeded inputs, returning every stage boundary as numpy arrays."""
import numpy as np
import torch

from oracle import oracle as O
from paper_2003_05328_gb300 import fdsc as F


def dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def gpu_round_trip(P, L, xA, xB, w, ks, es, ss, homrec=True):
    out = {}
    H, W = L.H, L.W
    out["t_hat"] = t_hat = F.keygen(P, ks)
    out["Phat"] = Phat = F.filter_prepare(P, L, dev(w, np.int8))
    Mhat, sB = F.mask_prepare(P, L, ss)
    out["Mhat"], out["sB_hat"] = Mhat, sB
    out["XA"] = XA = F.ntt2d(P, dev(xA, np.int32))
    out["ct_enc"] = ct = F.encrypt(P, L, t_hat, XA, es)
    out["ct_enc"] = ct.clone()
    if homrec:
        out["XB"] = XB = F.ntt2d(P, dev(xB, np.int32))
        F.homrec(P, L, XB, ct)
        out["ct_rec"] = ct
    out["ct_out"] = ct_out = F.homconv(P, L, ct, Phat, Mhat)
    out["SA_hat"] = SA = F.decrypt(P, L, t_hat, ct_out)
    out["yA"] = F.intt2d(P, SA.view(L.B, L.Co, H, W))
    out["yB"] = F.intt2d(P, sB.view(L.B, L.Co, H, W))
    torch.cuda.synchronize()
    res = {k: (u64(v) if v.dtype == torch.int64 else u32(v)) for k, v in out.items()}
    # filter plaintexts are stored once per group of d evaluation indices
    # (w_0(x^d) takes one value on each group): expand to the oracle's layout
    d = P.info.d
    res["Phat"] = np.repeat(res["Phat"].reshape(-1, P.n // d), d, axis=1).reshape(-1)
    return res


def compare_all(got, ref, keys=None):
    keys = keys or [k for k in ref if k in got and k != "noise"]
    for k in keys:
        g, r = got[k].reshape(-1), np.asarray(ref[k]).reshape(-1)
        assert g.shape == r.shape, (k, g.shape, r.shape)
        if not np.array_equal(g, r):
            bad = np.nonzero(g != r)[0]
            raise AssertionError(f"stage {k}: {bad.size} of {g.size} words differ, first at {bad[:5]}: "
                                 f"gpu {g[bad[:5]]} oracle {r[bad[:5]]}")
