"""The oracle's worst-case decryption bound (Sec. 3.1 decryption, after
HomRec, HomConv and HomShare, Fig. 2), pinned by a construction that reaches
it rather than by the formula itself.

Construction: T input ciphertexts (c0 = 0, so decryption reads c1 alone)
whose fresh error is -19 in every coefficient and whose message is Alice's
plaintext p-1 plus Bob's HomRec plaintext p-1 in every coefficient (so every
coefficient carries past p: Delta (2p - 2) = Delta (p - 2) + q - r_q); a
filter whose plaintext coefficients are all floor(p/2).  In the negacyclic
ring every product of two constant polynomials has coefficient
i -> c (2 i + 2 - n), so the HomConv output's error and message are known in
closed form:

    M_i   = T (p-2) floor(p/2) (2i + 2 - n)                 (the message product)
    eta_i = -T (19 + r_q) floor(p/2) (2i + 2 - n) - r_q floor(M_i / p)

largest at i = n-1.  Its two parts are exactly the two terms of the bound
(fresh error plus HomRec carry, times the filter; and r_q times the
plaintext product's multiples of p), so dropping either term of the bound
leaves the measured noise above it.  With a second 60-bit prime q = 1 mod 2n
whose residue r_q = q mod p is near p/2 the carry term alone exceeds
Delta / 2 at T = 32: decryption then really fails, and the bound says so."""
import random

import numpy as np
import pytest
import sympy

from oracle import oracle as O


def _worst_case(P, T):
    n, p, q, delta = P.n, P.p, P.q, P.delta
    L = O.layer(P, 1, T, 1, 32, 32, 1, 1)
    assert (L.T, L.n_in, L.n_out, L.beta) == (T, T, 1, 1)
    c1 = (q - 19 + 2 * delta * (p - 1)) % q  # error -19, messages p-1 (Alice) and p-1 (Bob's HomRec)
    ct = np.zeros((T, 2, n), np.uint64)
    ct[:, 1] = O.ntt_q(P, np.full(n, c1, np.uint64))
    Phat = np.tile(O.ntt_q(P, np.full(n, p // 2, np.uint64)), (T, 1))
    out = O.homconv(P, L, ct, Phat, None)
    m, noise = O.decrypt_raw(P, np.zeros(n, np.uint64), out[0])
    return m, noise


def _closed_form(P, T):
    n, p, r = P.n, P.p, P.r_q
    h = p // 2
    M = [T * (p - 2) * h * (2 * i + 2 - n) for i in range(n)]
    eta = [-T * (19 + r) * h * (2 * i + 2 - n) - r * (Mi // p) for i, Mi in zip(range(n), M)]
    return [Mi % p for Mi in M], max(abs(e) for e in eta), abs(eta[n - 1])


@pytest.mark.parametrize("n,p,T", [(2048, 65537, 32), (2048, 65537, 1), (1024, 65537, 4), (4096, 12289, 128)])
def test_worst_case_reaches_the_bound(n, p, T):
    P = O.params(n, p)
    assert P.r_q == 1
    m, noise = _worst_case(P, T)
    m_ref, eta_max, eta_last = _closed_form(P, T)
    assert eta_max == eta_last  # the extreme coefficient is the last one
    assert noise == eta_max  # the oracle's decryption measures exactly the constructed noise
    assert np.array_equal(m, np.array(m_ref, np.uint32))  # and still decrypts correctly
    bound = 2.0 ** O.noise_bound_log2(P, T)
    assert bound >= noise
    # tight: the bound exceeds this worst case only by the last coefficient's
    # rounding of the carry count and the HomShare borrow
    assert bound - noise <= 2 * P.r_q * (1 + T * n * (p // 2) // p) + 1e-9 * bound
    # dropping the HomRec carry (19 + r_q -> 19) or the plaintext-carry term
    # would leave the bound below what the construction measures
    h = p // 2
    without_homrec_carry = T * n * 19 * h + P.r_q * -(-T * n * (p - 1) * h // p) + P.r_q
    without_plain_carries = T * n * (19 + P.r_q) * h + P.r_q
    assert noise > without_homrec_carry and noise > without_plain_carries
    assert O.noise_ok(P, T)


def _params_with_q(n, p, want_r):
    """Oracle params for (n, p) with another 60-bit prime q = 1 mod 2n whose
    residue q mod p is near want_r (not 1 mod p)."""
    P = O.params(n, p)
    k = ((1 << 60) - 1) // (2 * n)
    while True:
        q = k * 2 * n + 1
        if abs(q % p - want_r) < p // 8 and sympy.isprime(q):
            break
        k -= 1
    rnd = random.Random(q)
    while True:  # an element of order exactly 2n: its n-th power is -1
        psi = pow(rnd.randrange(2, q - 1), (q - 1) // (2 * n), q)
        if pow(psi, n, q) == q - 1:
            break
    P.q, P.psi_q, P.g_q, P.delta, P.r_q = q, psi, 0, q // p, q % p
    assert (1 << 59) < q < (1 << 60)
    return P


def test_large_r_q_breaks_decryption_exactly_where_the_bound_says():
    n, p = 2048, 65537
    P = _params_with_q(n, p, p // 2)
    assert P.r_q > p // 4
    # one input ciphertext: the carries stay below Delta/2 and decryption is correct
    m, noise = _worst_case(P, 1)
    m_ref, eta_max, _ = _closed_form(P, 1)
    assert O.noise_ok(P, 1) and noise == eta_max and np.array_equal(m, np.array(m_ref, np.uint32))
    # 32 input ciphertexts: r_q times the plaintext carries alone exceeds Delta/2
    assert P.r_q * (32 * n * (p - 2) * (p // 2) // p) > P.delta // 2
    m, _ = _worst_case(P, 32)
    m_ref, _, _ = _closed_form(P, 32)
    assert not np.array_equal(m, np.array(m_ref, np.uint32))
    assert not O.noise_ok(P, 32)
