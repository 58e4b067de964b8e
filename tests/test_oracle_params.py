"""Pins for the oracle's parameter arithmetic and randomness (CPU only).

Each check compares the oracle with something other than itself: numbers the
paper prints (Table 2, Sec. 5.2), sympy's number theory, published generator
output, or exact distributions.
"""
import math
import os

import numpy as np
import pytest
import sympy

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_table2_pE_is_minimal_prime_splitting_xn_plus_1():
    # Sec. 6.4: p_E is the minimal prime >= p_N with p_E = 1 mod n (n = 2048),
    # and Table 2 prints the resulting p_E and its bit length.
    for name, pN, _lg_pN, pE, lg_pE, _lg_q in _rows("table2_moduli.txt"):
        pN, pE = int(pN), int(pE)
        assert O.lib().orc_min_prime_1mod(pN, 2048) == pE, name
        assert math.ceil(math.log2(pE)) == int(lg_pE)
        assert sympy.isprime(pE)


def test_decoupled_moduli_do_not_reconstruct_mod_pN():
    """Table 2's Binary and High rows pair an NTT modulus p_N with a larger
    encryption modulus p_E (Sec. 5.2 asks p_E >= p_A >= p_N).  Shares taken
    mod p_E do not give the result mod p_N: the appendix's step
    x mod p_A mod p_N = x mod p_N fails as soon as x passes p_A, and one
    Hadamard product of two spectra below p_N already passes p_E.  Only rows
    with p_N = p_E (Table 2's Medium row) run as one prime; the library takes
    any such prime below 2^20."""
    rows = {r[0]: (int(r[1]), int(r[3])) for r in _rows("table2_moduli.txt")}
    assert rows["Medium"][0] == rows["Medium"][1]
    for name in ("Binary", "High"):
        pN, pE = rows[name]
        assert pN < pE
        x = (pN - 1) * (pN - 1)  # one product of two spectra words
        assert x >= pE and x % pE % pN != x % pN, name
        # smallest counterexample to the appendix identity: x = p_E
        assert pE % pE % pN == 0 != pE % pN, name
    P = O.params(2048, rows["Medium"][0])
    assert P.S == 2048 and O.noise_ok(P, 32)


def test_no_share_conversion_exists_at_table2_decoupled_moduli():
    """Why Table 2's Binary and High rows are not built (Sec. 5.2, Sec. 6.4).

    1. Information is lost, so no rule -- interactive or not -- can work on
       HomConv's output: a slot of the decrypted, masked result is a
       function of Y mod p_E, Y the integer Hadamard sum; two spectrum pairs
       with the same product mod p_E but different products mod p_N give
       the same output distribution and different wanted results.
    2. A correct variant keeps the integer Y below p_E and masks it with
       r < 2^kappa Y_max (statistical hiding), so Alice lifts Y - r exactly
       and both parties reduce mod p_N: it needs p_E > (2^kappa + 1) Y_max
       with Y_max = Ci (2 p_N - 2)(p_N - 1) (HomRec adds Bob's spectrum
       without a reduction mod p_N), and a ciphertext modulus q whose
       worst-case noise bound (fresh error times filter, T n 20 p_E / 2, at
       p_E's scale Delta = q / p_E) holds.  Even with kappa = 0 and a single
       input channel, q needs more than 60 bits at n = 2048.
    3. p_N - 1 has a single factor 2 for both rows, so no power-of-two
       plane transform exists mod p_N (only mixed-radix lengths)."""
    rows = {r[0]: (int(r[1]), int(r[3]), int(r[5])) for r in _rows("table2_moduli.txt")}
    n = 2048
    for name in ("Binary", "High"):
        pN, pE, lg_q = rows[name]
        # 1: a collision of products mod p_E that differs mod p_N
        x = pE + 1  # = 1 * (pE + 1) as a product of two spectrum values below p_N
        a = next(d for d in range(2, pN) if x % d == 0 and x // d < pN)
        u1, w1, u2, w2 = 1, 1, a, x // a
        assert max(u1, w1, u2, w2) < pN
        assert (u1 * w1) % pE == (u2 * w2) % pE and (u1 * w1) % pN != (u2 * w2) % pN, name
        # 2: the smallest plaintext modulus that keeps Y exact at Ci = 1, kappa = 0, and the q it needs
        y_max = 1 * (2 * pN - 2) * (pN - 1)
        pE_min = sympy.nextprime(y_max)
        while (pE_min - 1) % (2 * n):
            pE_min = sympy.nextprime(pE_min)
        T = 1
        eta = T * n * 20 * (pE_min // 2)  # fresh error and HomRec carry (r_q = 1 at best), times the filter
        q_min = 2 * (pE_min * eta + (pE_min - 1))  # p_E |eta| + r_q (p_E - 1) < q / 2, with r_q = 1
        assert pE_min > pE and math.log2(q_min) > 60 and int(lg_q) <= 60, name
        # 3: no power-of-two transform lengths beyond 2
        assert (pN - 1) % 2 == 0 and (pN - 1) % 4 != 0, name


def test_smallest_prime_splitting_x2048_plus_1_is_12289():
    # Sec. 5.2: "for n = 2048, p_E >= 12289" -- x^n + 1 splits completely mod
    # a prime iff 2n | p - 1.
    assert O.lib().orc_min_prime_1mod(2, 4096) == 12289


@pytest.mark.parametrize("p", [65537, 12289])
def test_q_is_largest_60bit_prime_1_mod_8192p(p):
    q = O.lib().orc_find_q(p)
    M = 8192 * p
    assert sympy.isprime(q) and q < 2**60 and q % M == 1 and q > 2**59
    # no larger candidate below 2^60 is prime (independent search)
    k = (2**60 - 2) // M
    cand = [k2 * M + 1 for k2 in range(k, (q - 1) // M, -1)]
    assert not any(sympy.isprime(c) for c in cand)


def test_is_prime_matches_sympy():
    lib = O.lib()
    g = np.random.default_rng(7)
    nums = [int(v) for v in g.integers(2, 2**63, 300, dtype=np.uint64)]
    nums += [int(v) | 1 for v in g.integers(2**40, 2**62, 300, dtype=np.uint64)]
    # strong pseudoprimes to several small bases and Carmichael numbers
    nums += [2047, 1373653, 25326001, 3215031751, 2152302898747, 3474749660383, 341550071728321,
             3825123056546413051, 561, 1105, 1729, 2465, 2821, 6601, 8911]
    nums += [65537, 12289, 2**61 - 1, 2**31 - 1, 1152921497895862273]
    for v in nums:
        assert bool(lib.orc_is_prime(v)) == sympy.isprime(v), v


@pytest.mark.parametrize("m", [65537, 12289, 147457, 2363393, 1152921497895862273, 1152921504107839489])
def test_primitive_root_matches_sympy(m):
    assert O.lib().orc_primitive_root(m) == sympy.primitive_root(m)


@pytest.mark.parametrize("n,p", [(1024, 65537), (2048, 65537), (4096, 65537), (2048, 12289), (4096, 12289)])
def test_params_roots_orders(n, p):
    P = O.params(n, p)
    q = P.q
    # psi_q has order exactly 2n: psi^n = -1
    assert pow(P.psi_q, n, q) == q - 1
    assert sympy.n_order(P.psi_q, q) == 2 * n
    # slot sets: S = largest power of two with 2S | p-1, capped at n
    v = sympy.multiplicity(2, p - 1)
    assert P.S == min(n, 2 ** (v - 1)) and P.d * P.S == n
    assert sympy.n_order(P.psi_p, p) == 2 * P.S
    assert P.delta == q // p and P.r_q == q % p == 1


def test_params_reject_bad_inputs():
    with pytest.raises(ValueError):
        O.params(1000, 65537)  # not a power of two
    with pytest.raises(ValueError):
        O.params(2048, 65535)  # not prime
    with pytest.raises(ValueError):
        O.params(8192, 65537)  # beyond the q = 1 mod 8192 p design


def test_noise_bound_admits_all_configs_and_rejects_huge_T():
    for n, p, T in [(1024, 65537, 1), (2048, 65537, 32), (2048, 65537, 16), (4096, 65537, 4),
                    (4096, 12289, 128), (2048, 65537, 128)]:
        P = O.params(n, p)
        assert O.noise_ok(P, T)
    P = O.params(4096, 65537)
    assert not O.noise_ok(P, 1 << 12)  # 4096 input ciphertexts overflow Delta/2


def test_splitmix64_published_first_output():
    # orc_rng(0, 0, 0) = mix(mix(0) + gamma) = mix(gamma): the first output of
    # SplitMix64 started from state 0.
    (_state, out), = _rows("splitmix64.txt")
    assert O.rng(0, 0, 0) == int(out, 16)


def test_uniform_p_and_q_ranges_and_mean():
    P = O.params(2048, 65537)
    vals_q = [O.uniform_q(P, O.rng(5, 2, 2 * i), O.rng(5, 2, 2 * i + 1)) for i in range(4000)]
    assert all(0 <= v < P.q for v in vals_q)
    assert abs(np.mean(np.array(vals_q, dtype=np.float64)) / P.q - 0.5) < 0.02
    vals_p = np.array([O.uniform_p(65537, O.rng(9, 4, i)) for i in range(20000)])
    assert vals_p.min() >= 0 and vals_p.max() < 65537
    # chi-square on 16 equal bins
    hist = np.histogram(vals_p, bins=16, range=(0, 65537))[0]
    chi2 = ((hist - 1250) ** 2 / 1250).sum()
    assert chi2 < 40
    # extremes of the multiply-high map
    assert O.uniform_p(65537, 0) == 0 and O.uniform_p(65537, 2**64 - 1) == 65536
    assert O.uniform_q(P, 2**64 - 1, 2**64 - 1) == P.q - 1 and O.uniform_q(P, 0, 0) == 0


def test_gaussian_cdt_matches_exact_distribution():
    table = O.cdt()
    sigma = 3.2
    rho = np.array([math.exp(-k * k / (2 * sigma * sigma)) for k in range(20)])
    Z = rho[0] + 2 * rho[1:].sum()
    probs = np.concatenate([[rho[0] / Z], 2 * rho[1:] / Z])
    cum = np.cumsum(probs)[:19]
    assert np.all(np.abs(table.astype(np.float64) / 2.0**63 - cum) < 1e-12)
    assert np.all(np.diff(table.astype(np.float64)) > 0)
    # sampling: exact support and moments
    xs = np.array([O.gauss(O.rng(11, 3, i), table) for i in range(40000)])
    assert xs.min() >= -19 and xs.max() <= 19
    assert abs(xs.mean()) < 0.06
    assert abs(xs.var() - sigma**2) < 0.35
    # boundary behaviour: u = 0 -> 0, all-ones -> -19
    assert O.gauss(0, table) == 0 and O.gauss(2**64 - 1, table) == -19 and O.gauss(2**63 - 1, table) == 19


def test_ternary_secret_is_balanced():
    P = O.params(2048, 65537)
    t, _ = O.keygen(P, 1234)
    assert set(np.unique(t)) <= {-1, 0, 1}
    counts = [(t == v).sum() for v in (-1, 0, 1)]
    assert min(counts) > 600
