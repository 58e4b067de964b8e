"""The arithmetic the tensor-core HomConv rests on, checked on the CPU with
Python integers: balanced base-256 digits of words below q reconstruct them,
the products summed per weight class 256^kappa (the diagonals the MMAs
accumulate in fp32) recombine into the exact product sum, and no partial sum
of a diagonal reaches 2^24 for up to 128 input ciphertexts, which is what
makes the fp32 accumulation exact."""
import numpy as np
import pytest

from oracle import oracle as O

BIAS = 0x8080808080808080


def digits(w):
    """d_a = byte_a(w + 0x80..80) - 128, a < 8."""
    v = w + BIAS
    return [((v >> (8 * a)) & 255) - 128 for a in range(8)]


@pytest.mark.parametrize("p", [65537, 12289])
def test_digits_reconstruct_words_below_q(p):
    q = O.params(2048 if p == 65537 else 4096, p).q
    g = np.random.default_rng(p)
    words = [0, 1, q - 1, q - 2, 2**56 - 1, 2**56, (q - 1) & ~0xFF] + [int(x) for x in g.integers(0, q, 2000, dtype=np.uint64)]
    for w in words:
        d = digits(w)
        assert sum(x * 256**a for a, x in enumerate(d)) == w
        assert all(-128 <= x <= 127 for x in d)
        assert 0 <= d[7] <= 16  # the top digit of a word below 2^60


def test_diagonals_recombine_the_product_sum():
    q = O.params(2048, 65537).q
    g = np.random.default_rng(3)
    T = 32
    P = [int(x) for x in g.integers(0, q, T, dtype=np.uint64)]
    X = [int(x) for x in g.integers(0, q, T, dtype=np.uint64)]
    D = [0] * 15
    for pk, xk in zip(P, X):
        dp, dx = digits(pk), digits(xk)
        for a in range(8):
            for b in range(8):
                D[a + b] += dp[a] * dx[b]
    assert sum(Dk * 256**k for k, Dk in enumerate(D)) == sum(pk * xk for pk, xk in zip(P, X))


def test_diagonal_bound_below_2_24_for_128_terms():
    """Largest possible |partial sum| of a diagonal: sum of |products| over
    its pairs, the top digit (a = 7 or b = 7) being at most 16."""
    worst = 0
    for kap in range(15):
        s = 0
        for a in range(8):
            b = kap - a
            if 0 <= b < 8:
                ma = 16 if a == 7 else 128
                mb = 16 if b == 7 else 128
                s += ma * mb
        worst = max(worst, s)
    assert worst == 7 * 2**14  # diagonal 6: seven products of (-128)(-128)
    assert 128 * worst < 2**24 < 147 * worst  # T = 128 fits; the bound would break above T = 146
    # the magic-number conversion (one fp32 add of 1.5 * 2^23) needs |D| < 2^22: T <= 32
    assert 32 * worst < 2**22 < 37 * worst


def test_worst_case_words_reach_the_bound():
    """Words with digits 0..6 all -128 (the GPU test's worst case) make
    diagonal 6 equal T * 7 * 2^14 exactly."""
    q = O.params(2048, 65537).q
    low = (1 << 56) - 0x80808080808080
    w = low + (((q - 1 - low) >> 56) << 56)
    assert w < q and digits(w)[:7] == [-128] * 7
    T = 128
    D6 = sum(digits(w)[a] * digits(w)[6 - a] for a in range(7)) * T
    assert D6 == T * 7 * 2**14 < 2**24
