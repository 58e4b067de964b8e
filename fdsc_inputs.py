"""Seeded synthetic workloads for the FDSC hot path.

This module only draws inputs: it holds none of the method's arithmetic and
is the one piece of Python shared by the CPU oracle's callers and the GPU
library's callers (tests, benchmark, smoke check).

The workloads stand in for the paper's CIFAR-10 / MNIST-scale convolution
layers (Sec. 6.2, Table 4, the appendix architectures): secret shares are
uniform in Z_p on the image support and zero on the padding, filters are
int8 uniform in [-8, 7] (4-bit, like the "Medium" filter width of Table 1)
or uniform in {-1, +1} for the binarized layer.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 0xE45E10000


@dataclass(frozen=True)
class LayerShape:
    """One convolution layer: B images of Ci x (h x w) zero-padded to H x W,
    Co filters of fh x fw."""

    B: int
    Ci: int
    Co: int
    H: int
    W: int
    fh: int
    fw: int
    n: int
    p: int
    h: int = 0  # image support (0 = the whole padded plane)
    w: int = 0
    binary: bool = False

    @property
    def support(self):
        return (self.h or self.H, self.w or self.W)


@dataclass(frozen=True)
class Config:
    name: str
    cid: int
    layers: tuple
    note: str = ""
    extra: dict = field(default_factory=dict)


CONFIGS = {
    "layer_16x16x4_b1": Config("single layer 16x16x4->4, 3x3, n=1024", 0,
                   (LayerShape(1, 4, 4, 16, 16, 3, 3, 1024, 65537),)),
    "cifar_32x32x64_b1": Config("CIFAR-shaped layer 32x32x64->64, 3x3, batch 1, n=2048", 1,
                   (LayerShape(1, 64, 64, 32, 32, 3, 3, 2048, 65537),)),
    "stack_16img_32x32x64_16x16x128_8x8x256": Config("batched uneven stack, 16 images: 32x32x64->64, 16x16x128->128, 8x8x256->256", 2,
                   (LayerShape(16, 64, 64, 32, 32, 3, 3, 2048, 65537),
                    LayerShape(16, 128, 128, 16, 16, 3, 3, 2048, 65537),
                    LayerShape(16, 256, 256, 8, 8, 3, 3, 4096, 65537))),
    "served_mix_28x28x1_32x32x64_16x16x128": Config("served mix: 28x28 (pad 32)x1->16 5x5, 32x32x64->64 3x3, 16x16x128->128 3x3", 3,
                   (LayerShape(1, 1, 16, 32, 32, 5, 5, 2048, 65537, h=28, w=28),
                    LayerShape(1, 64, 64, 32, 32, 3, 3, 2048, 65537),
                    LayerShape(1, 128, 128, 16, 16, 3, 3, 2048, 65537)),
                   extra={"rate_per_s": 2000.0, "requests": 20000, "hbm_budget_bytes": 120 * 10**9}),
    "binarized_64x64x128_b8": Config("binarized layer 64x64x128->128, batch 8, p=12289, n=4096", 4,
                   (LayerShape(8, 128, 128, 64, 64, 3, 3, 4096, 12289, binary=True),)),
}


def _rng(cid: int, tag: int, sub: int = 0) -> np.random.Generator:
    return np.random.default_rng([SEED_BASE + cid, tag, sub])


def shares(ls: LayerShape, cid: int, sub: int = 0):
    """Alice's and Bob's additive shares x_A, x_B of a zero-padded input:
    uint32 [B][Ci][H][W], uniform in [0, p) on the h x w support, 0 elsewhere."""
    h, w = ls.support
    out = []
    for tag in (1, 2):
        x = np.zeros((ls.B, ls.Ci, ls.H, ls.W), np.uint32)
        x[:, :, :h, :w] = _rng(cid, tag, sub).integers(0, ls.p, (ls.B, ls.Ci, h, w), dtype=np.uint32)
        out.append(x)
    return out[0], out[1]


def weights(ls: LayerShape, cid: int, sub: int = 0) -> np.ndarray:
    """Bob's filters: int8 [Co][Ci][fh][fw]."""
    g = _rng(cid, 3, sub)
    if ls.binary:
        return (g.integers(0, 2, (ls.Co, ls.Ci, ls.fh, ls.fw)) * 2 - 1).astype(np.int8)
    return g.integers(-8, 8, (ls.Co, ls.Ci, ls.fh, ls.fw)).astype(np.int8)


def seeds(cid: int, sub: int = 0):
    """(key_seed, enc_seed, server_seed) for the method's own randomness."""
    g = _rng(cid, 4, sub)
    return tuple(int(v) for v in g.integers(0, 2**63, 3, dtype=np.uint64))


def default_pack(ls: LayerShape, S: int):
    """Channel blocks per slot set when an image plane fits in one slot set:
    as many input channels as fit, one image per block row."""
    HW = ls.H * ls.W
    if HW > S:
        return 1, 1
    return max(1, min(ls.Ci, S // HW)), 1

