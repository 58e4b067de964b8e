"""The bounds behind two single-step reductions of the device code, checked
with Python integers for every ciphertext modulus q the library derives (no
GPU): the key products a t + b of encryption and decryption (one Barrett
reduction of a 121-bit value) and decryption's rounding round(p v / q) mod p
(one correction of a quotient estimate).  Each step below is the device
code's, in 64-bit wrapping arithmetic; the asserts are the ranges that make
one conditional subtraction enough."""
import random

import pytest

M64 = (1 << 64) - 1
PRIMES = (65537, 12289, 147457, 786433, 7681)


@pytest.fixture(scope="module")
def F():
    from paper_2003_05328_gb300 import build

    build.build()
    from paper_2003_05328_gb300 import fdsc

    return fdsc


def moduli(F):
    out = []
    for p in PRIMES:
        for n in (1024, 2048, 4096):
            info = F.params_query(n, p)
            out.append((p, info.q))
    return out


def muladd(a, b, c, q, mu):
    """(a b + c) mod q: x' = floor(x / 2^58), estimate floor(x' mu / 2^64)."""
    x = a * b + c
    lo, hi = x & M64, x >> 64
    assert hi < (1 << 58)  # x < 2^122: the shifted value fits 64 bits
    est = ((((hi << 6) & M64) | (lo >> 58)) * mu) >> 64
    assert x // q - 1 <= est <= x // q
    r = (lo - est * q) & M64
    assert r < 2 * q
    return r - q if r >= q else r


def round_pq(v, p, q, round_k):
    """round(p v / q) mod p through the remainder p v - z q."""
    z = (v * round_k) >> 64
    assert (p * v) // q - 1 <= z <= (p * v) // q
    rem = (p * v - z * q) & M64
    assert rem < 2 * q
    if rem >= q:
        rem -= q
        z += 1
    z += 2 * rem >= q
    return z - p if z >= p else z


def test_every_derived_q_admits_the_single_step_reductions(F):
    for p, q in moduli(F):
        assert (1 << 59) < q < (1 << 60), (p, q)
        assert q % 2 == 1  # odd: 2 p v + q is never a multiple of 2 q, no ties


def test_barrett_key_product_is_exact(F):
    rng = random.Random(5)
    for p, q in moduli(F)[::3]:
        mu = (1 << 122) // q
        assert (1 << 62) < mu < (1 << 63)
        edge = [0, 1, 2, q - 1, q - 2, q // 2, (1 << 32) - 1, 1 << 32]
        cases = [(a, b, c) for a in edge for b in edge for c in edge]
        cases += [(rng.randrange(q), rng.randrange(q), rng.randrange(q)) for _ in range(20000)]
        for a, b, c in cases:
            assert muladd(a, b, c, q, mu) == (a * b + c) % q


def test_remainder_rounding_is_exact(F):
    rng = random.Random(6)
    for p, q in moduli(F)[::3]:
        round_k = (p << 64) // q
        vs = [0, 1, q - 1, q - 2, q // 2]
        for m in list(range(40)) + [p // 2, p - 2, p - 1]:
            half = ((2 * m + 1) * q) // (2 * p)  # next to the rounding boundary m + 1/2
            vs += [v for v in (half - 1, half, half + 1, half + 2) if 0 <= v < q]
        vs += [rng.randrange(q) for _ in range(20000)]
        for v in vs:
            assert round_pq(v, p, q, round_k) == ((2 * p * v + q) // (2 * q)) % p
