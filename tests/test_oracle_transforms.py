"""Pins for the oracle's transforms (CPU only).

NTT2D is checked against the convolution theorem (Eq. 6) with a brute-force
cyclic convolution, closed forms (delta, constants) and its own inverse; the
negacyclic transforms against schoolbook ring products in Python integers and
the root structure of x^L + 1.  Tier 1 (radix-2) is checked against tier 0
(the O(N^2) definition).
"""
import numpy as np
import pytest

from oracle import oracle as O


def cyclic_conv_bruteforce(x, w, p):
    """y[i][j] = sum_{a,c} w[a][c] x[(i-a) mod H][(j-c) mod W] with np.roll."""
    H, W = x.shape
    y = np.zeros((H, W), dtype=object)
    for a in range(w.shape[0]):
        for c in range(w.shape[1]):
            y = y + int(w[a, c]) * np.roll(np.roll(x.astype(object), a, axis=0), c, axis=1)
    return (y % p).astype(np.uint32)


def negacyclic_schoolbook(a, b, m):
    L = len(a)
    out = [0] * L
    for i in range(L):
        for j in range(L):
            k = i + j
            if k < L:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - L] -= int(a[i]) * int(b[j])
    return [v % m for v in out]


@pytest.mark.parametrize("p", [65537, 12289, 147457, 786433])
@pytest.mark.parametrize("H,W", [(4, 4), (8, 16), (16, 8), (2, 32)])
def test_ntt2d_tier1_equals_definition(p, H, W):
    x = np.random.default_rng(H * W).integers(0, p, (3, H, W))
    X1 = O.ntt2d(x, p)
    with O.tier(0):
        X0 = O.ntt2d(x, p)
    assert np.array_equal(X0, X1)


@pytest.mark.parametrize("p", [65537, 12289, 147457, 786433])
@pytest.mark.parametrize("H,W", [(8, 8), (16, 16), (32, 32), (4, 64)])
def test_convolution_theorem(p, H, W):
    g = np.random.default_rng(3 + H)
    x = g.integers(0, p, (H, W))
    w = np.zeros((H, W), np.int64)
    w[:3, :3] = g.integers(-8, 8, (3, 3))
    X = O.ntt2d(x, p).astype(object)
    Wh = O.ntt2d(w % p, p).astype(object)
    y = O.ntt2d(((X * Wh) % p).astype(np.uint32), p, inverse=True)
    assert np.array_equal(y, cyclic_conv_bruteforce(x, w[:3, :3], p))


@pytest.mark.parametrize("p", [65537, 12289, 147457, 786433])
def test_ntt2d_closed_forms_and_inverse(p):
    H, W = 16, 32
    delta = np.zeros((H, W), np.uint32)
    delta[0, 0] = 1
    assert np.all(O.ntt2d(delta, p) == 1)
    const = np.full((H, W), 7, np.uint32)
    Xc = O.ntt2d(const, p)
    assert Xc[0, 0] == (7 * H * W) % p and np.count_nonzero(Xc) == 1
    x = np.random.default_rng(1).integers(0, p, (5, H, W))
    assert np.array_equal(O.ntt2d(O.ntt2d(x, p), p, inverse=True), x)
    # linearity
    y = np.random.default_rng(2).integers(0, p, (5, H, W))
    lhs = O.ntt2d((x + y) % p, p)
    rhs = (O.ntt2d(x, p).astype(np.int64) + O.ntt2d(y, p)) % p
    assert np.array_equal(lhs, rhs)
    # an impulse at (i0, j0) gives w_H^(i0 k1) w_W^(j0 k2): its spectrum's row 1
    # column 0 is a primitive H-th root of unity
    imp = np.zeros((H, W), np.uint32)
    imp[1, 0] = 1
    r = int(O.ntt2d(imp, p)[1, 0])
    assert pow(r, H, p) == 1 and pow(r, H // 2, p) == p - 1


@pytest.mark.parametrize("n,p", [(64, 65537), (256, 65537), (1024, 12289), (4096, 12289), (128, 147457),
                                 (2048, 147457), (256, 786433)])
def test_slot_transform_is_ring_homomorphism(n, p):
    P = O.params(n, p)
    S = P.S
    g = np.random.default_rng(S)
    a, b = g.integers(0, p, S), g.integers(0, p, S)
    if S <= 256:
        prod = negacyclic_schoolbook(a, b, p)
        lhs = O.slot_decode(P, np.array(prod))
        rhs = (O.slot_decode(P, a).astype(np.int64) * O.slot_decode(P, b)) % p
        assert np.array_equal(lhs, rhs)
    s = g.integers(0, p, S)
    assert np.array_equal(O.slot_decode(P, O.slot_encode(P, s)), s)


@pytest.mark.parametrize("n,p", [(64, 65537), (128, 12289), (64, 147457), (128, 786433)])
def test_slot_order_is_bit_reversed_roots(n, p):
    P = O.params(n, p)
    S = P.S
    mono = np.zeros(S, np.uint32)
    mono[1] = 1  # m(x) = x  -> slot i holds the root itself
    roots = [int(v) for v in O.slot_decode(P, mono)]
    assert len(set(roots)) == S
    assert all(pow(r, S, p) == p - 1 for r in roots)
    # bit-reversed order: slots 2m and 2m+1 are negatives of one another,
    # slot 0 is psi itself
    assert roots[0] == P.psi_p
    assert all((roots[2 * m] + roots[2 * m + 1]) % p == 0 for m in range(S // 2))
    with O.tier(0):
        assert [int(v) for v in O.slot_decode(P, mono)] == roots


@pytest.mark.parametrize("n,p", [(16, 65537), (64, 65537), (256, 65537), (64, 12289), (64, 147457), (64, 786433)])
def test_ntt_q_ring_product_and_tiers(n, p):
    P = O.params(n, p)
    q = P.q
    g = np.random.default_rng(n)
    a = [int(v) for v in g.integers(0, 2**62, n, dtype=np.uint64) % np.uint64(q)]
    b = [int(v) for v in g.integers(0, 2**62, n, dtype=np.uint64) % np.uint64(q)]
    A, Bh = O.ntt_q(P, a), O.ntt_q(P, b)
    prod = O.intt_q(P, [(int(x) * int(y)) % q for x, y in zip(A, Bh)])
    assert [int(v) for v in prod] == negacyclic_schoolbook(a, b, q)
    assert [int(v) for v in O.intt_q(P, A)] == a
    with O.tier(0):
        assert np.array_equal(O.ntt_q(P, a), A)
        assert [int(v) for v in O.intt_q(P, A)] == a
    mono = [0] * n
    mono[1] = 1
    roots = [int(v) for v in O.ntt_q(P, mono)]
    assert roots[0] == P.psi_q and all(pow(r, n, q) == q - 1 for r in roots)
    assert all((roots[2 * m] + roots[2 * m + 1]) % q == 0 for m in range(n // 2))


def test_ntt_q_full_size_inverse():
    for n in (1024, 2048, 4096):
        P = O.params(n, 65537)
        a = np.random.default_rng(n).integers(0, 2**62, n, dtype=np.uint64) % np.uint64(P.q)
        assert np.array_equal(O.intt_q(P, O.ntt_q(P, a)), a)
