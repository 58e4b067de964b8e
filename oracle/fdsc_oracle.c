/*
 * fdsc_oracle.c -- TEST INFRASTRUCTURE ONLY (see fdsc_oracle.h).
 *
 * A plain CPU statement of the frequency-domain secure convolution (FDSC)
 * protocol of ENSEI (Bian et al., CVPR 2020), written from the paper:
 *   Sec. 3.1 / Eq. 1   BFV encryption c0 = -a, c1 = a*t + (q/p)u + e, and
 *                      decryption round(p/q (c0 t + c1));
 *   Sec. 3.1           homomorphic add and Hadamard product (SIMDScMult);
 *   Eq. 2 / Eq. 3      HomShare and HomRec;
 *   Eq. 5, 6, 12       the (number theoretic) DFT and the convolution theorem;
 *   Fig. 2             the protocol: NTT2D -> Enc -> Hadamard -> HomShare ->
 *                      Dec -> INTT2D, with HomRec between layers;
 *   Sec. 5.1           ciphertexts kept in the NTT domain, RLWE constants
 *                      drawn there;
 *   Sec. 5.2, 6.4      moduli and parameter instantiation.
 *
 * Every modular product is an unsigned __int128 followed by '%'.  No lazy
 * reduction, no precomputed-quotient tricks, no blocking: a reader can check
 * each function against the section it cites.  Transforms come in two tiers:
 * tier 0 evaluates the O(N^2) definition, tier 1 uses the textbook iterative
 * radix-2 cyclic transform (bit-reversal permutation + butterflies), and the
 * tests pin tier 1 to tier 0 and both to brute force.
 *
 * Where the paper is silent or inconsistent, the readings taken are stated at
 * the point of use (single prime p for p_N = p_A = p_E; transform length = the
 * padded plane; ciphertexts in the NTT_q domain with `a` drawn there; slot
 * sets for primes with few roots of unity; packing; randomness).
 */
#include "fdsc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef uint64_t u64;
typedef uint32_t u32;

static int g_tier = 1;
void orc_set_tier(int tier) { g_tier = tier; }
int orc_get_tier(void) { return g_tier; }

/* ------------------------------------------------------------------------ */
/* modular arithmetic: operands are already reduced mod m                    */
/* ------------------------------------------------------------------------ */
static u64 mulm(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }
static u64 addm(u64 a, u64 b, u64 m) { return (u64)(((u128)a + b) % m); }
static u64 subm(u64 a, u64 b, u64 m) { return (u64)(((u128)a + m - b) % m); }

u64 orc_powmod(u64 b, u64 e, u64 m) {
    u64 r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = mulm(r, b, m);
        b = mulm(b, b, m);
        e >>= 1;
    }
    return r;
}

static u64 invm(u64 a, u64 m) { return orc_powmod(a, m - 2, m); } /* m prime */

/* Deterministic Miller-Rabin: the first twelve primes as witnesses decide
 * primality for every m < 3.3e24 (Sorenson & Webster 2015), so for all u64. */
int orc_is_prime(u64 m) {
    static const u64 wit[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (m < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (m == wit[i]) return 1;
        if (m % wit[i] == 0) return 0;
    }
    u64 dd = m - 1;
    int s = 0;
    while ((dd & 1) == 0) { dd >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = orc_powmod(wit[i], dd, m);
        if (x == 1 || x == m - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; r++) {
            x = mulm(x, x, m);
            if (x == m - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* Smallest generator of the multiplicative group of the prime field Z_m:
 * g is a generator iff g^((m-1)/r) != 1 for every prime r dividing m-1. */
u64 orc_primitive_root(u64 m) {
    u64 fac[64];
    int nf = 0;
    u64 r = m - 1;
    if ((r & 1) == 0) {
        fac[nf++] = 2;
        while ((r & 1) == 0) r >>= 1;
    }
    for (u64 dv = 3; dv <= r / dv; dv += 2) {
        if (r % dv == 0) {
            fac[nf++] = dv;
            while (r % dv == 0) r /= dv;
        }
    }
    if (r > 1) fac[nf++] = r;
    for (u64 g = 2; g < m; g++) {
        int ok = 1;
        for (int i = 0; i < nf && ok; i++)
            if (orc_powmod(g, (m - 1) / fac[i], m) == 1) ok = 0;
        if (ok) return g;
    }
    return 0;
}

/* Smallest prime >= lower that is 1 mod `modulus` (Sec. 6.4: the smallest
 * p_E >= p_N splitting x^n + 1). */
u64 orc_min_prime_1mod(u64 lower, u64 modulus) {
    u64 k = (lower <= 1) ? 0 : (lower - 1 + modulus - 1) / modulus;
    for (;; k++) {
        u64 x = k * modulus + 1;
        if (x >= lower && orc_is_prime(x)) return x;
    }
}

/* Ciphertext modulus (Sec. 6.4 says q is "adjusted to tolerate the error
 * growth"; the reading taken): the largest prime below 2^60 with
 * q = 1 mod 8192*p.  q = 1 mod 2n gives negacyclic NTTs for every n <= 4096
 * and q = 1 mod p makes q mod p = 1, which keeps plaintext carries small. */
u64 orc_find_q(u32 p) {
    u64 M = 8192ull * p;
    u64 k = ((1ull << 60) - 2) / M;
    while (k > 0 && !orc_is_prime(k * M + 1)) k--;
    return k * M + 1;
}

u32 orc_brv(u32 i, u32 logL) {
    u32 r = 0;
    for (u32 b = 0; b < logL; b++) r |= ((i >> b) & 1u) << (logL - 1 - b);
    return r;
}

static u32 ilog2(u64 x) {
    u32 l = 0;
    while ((1ull << l) < x) l++;
    return l;
}
static int is_pow2(u64 x) { return x && !(x & (x - 1)); }

int orc_params_init(u32 n, u32 p, orc_params* P) {
    memset(P, 0, sizeof(*P));
    if (!is_pow2(n) || n < 4 || n > 4096) return -1;
    if (p < 3 || p >= (1u << 20) || !orc_is_prime(p)) return -1;
    u32 v = 0;
    while (((p - 1) >> v & 1u) == 0) v++;
    if (v < 2) return -1;
    /* Slot sets: x^n + 1 splits into linear factors mod p only if 2n | p-1.
     * For a prime with fewer roots (12289 with n = 4096) the ring is read as
     * d = n/S interleaved length-S negacyclic slot sets, y = x^d, y^S = -1. */
    u32 S = n;
    if (S > (1u << (v - 1))) S = 1u << (v - 1);
    P->n = n;
    P->logn = ilog2(n);
    P->p = p;
    P->S = S;
    P->logS = ilog2(S);
    P->d = n / S;
    P->g_p = (u32)orc_primitive_root(p);
    P->psi_p = (u32)orc_powmod(P->g_p, (p - 1) / (2ull * S), p);
    P->q = orc_find_q(p);
    if (P->q < (1ull << 59)) return -1;
    P->g_q = orc_primitive_root(P->q);
    P->psi_q = orc_powmod(P->g_q, (P->q - 1) / (2ull * n), P->q);
    P->delta = P->q / p;
    P->r_q = P->q % p;
    return 0;
}

int orc_layer_init(const orc_params* P, u32 B, u32 Ci, u32 Co, u32 H, u32 W, u32 g_c,
                   u32 g_b, orc_layer* L) {
    memset(L, 0, sizeof(*L));
    if (!B || !Ci || !Co || !g_c || !g_b) return -1;
    if (!is_pow2(H) || !is_pow2(W) || (P->p - 1) % H || (P->p - 1) % W) return -1;
    L->B = B; L->Ci = Ci; L->Co = Co; L->H = H; L->W = W;
    L->g_c = g_c; L->g_b = g_b;
    L->HW = H * W;
    if (L->HW <= P->S) {
        if ((u64)g_c * g_b * L->HW > P->S) return -1;
        L->beta = 1;
        L->T = (Ci + g_c - 1) / g_c;
        L->GB = (B + P->d * g_b - 1) / (P->d * g_b);
    } else {
        if (g_c != 1 || g_b != 1 || L->HW % P->S) return -1;
        L->beta = L->HW / P->S;
        L->T = Ci;
        L->GB = (B + P->d - 1) / P->d;
    }
    L->n_in = L->GB * L->T * L->beta;
    L->n_out = L->GB * Co * L->beta;
    return 0;
}

/* Worst-case decryption noise of one HomConv output ciphertext with T input
 * ciphertexts, each carrying fresh error |e| <= 19 plus one HomRec carry:
 *   |eta| <= T n (19 + r_q) floor(p/2) + r_q ceil(T n (p-1) floor(p/2) / p) + r_q,
 * where the second term is the plaintext product's multiples of p (Delta p =
 * q - r_q) and the last one the HomShare borrow.  Decryption rounds correctly
 * when p |eta| + r_q (p-1) < q/2. */
static long double noise_max(const orc_params* P, u32 T) {
    long double Tn = (long double)T * P->n, h = (long double)(P->p / 2);
    long double carries = ceill(Tn * (P->p - 1) * h / P->p);
    return Tn * (19.0L + P->r_q) * h + (long double)P->r_q * carries + P->r_q;
}
double orc_noise_bound_log2(const orc_params* P, u32 T) { return (double)log2l(noise_max(P, T)); }
int orc_noise_ok(const orc_params* P, u32 T) { return orc_noise_ok_flood(P, T, 0); }
/* With HomShare noise flooding of `flood_bits` (every mask coefficient
 * carries an extra error in [-2^f, 2^f)), |eta| grows by at most 2^f. */
int orc_noise_ok_flood(const orc_params* P, u32 T, u32 flood_bits) {
    long double eta = noise_max(P, T) + (flood_bits ? ldexpl(1.0L, (int)flood_bits) : 0.0L);
    return eta * P->p + (long double)P->r_q * (P->p - 1) < (long double)P->q / 2;
}

/* ------------------------------------------------------------------------ */
/* randomness                                                                */
/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the generator's state after
 * k steps from s is s + k*gamma and its output is mix(state).  Used here as a
 * counter-based generator: a stream key from (seed, domain), then the
 * (idx+1)-th output of the stream keyed by it. */
static const u64 GAMMA = 0x9E3779B97F4A7C15ull;
static u64 splitmix_out(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
u64 orc_rng(u64 seed, u64 domain, u64 idx) {
    u64 key = splitmix_out(seed + domain * GAMMA);
    return splitmix_out(key + (idx + 1) * GAMMA);
}

enum { DOM_T = 1, DOM_A = 2, DOM_E = 3, DOM_MASK = 4, DOM_MASK_SPLIT = 5, DOM_FLOOD = 6 };

/* floor(r * m / 2^64): uniform on [0, m) from one 64-bit word. */
u32 orc_uniform_p(u32 p, u64 r) { return (u32)(((u128)r * p) >> 64); }

/* floor((r1 2^64 + r2) q / 2^128): uniform on [0, q) from two words.  With
 * A = r1 q and B = r2 q = Bh 2^64 + Bl, (A 2^64 + B) / 2^128 has floor
 * floor((A + Bh) / 2^64) because Bl < 2^64. */
u64 orc_uniform_q(const orc_params* P, u64 r1, u64 r2) {
    u128 A = (u128)r1 * P->q;
    u128 Bh = ((u128)r2 * P->q) >> 64;
    return (u64)((A + Bh) >> 64);
}

/* Discrete Gaussian, sigma = 3.2, support |x| <= 19 (Sec. 3.1 draws e from a
 * discrete Gaussian; the sigma and tail cut are readings).  Cumulative table
 * over |x|: P(0) = rho(0)/Z, P(k) = 2 rho(k)/Z, rho(k) = exp(-k^2/(2 sigma^2)),
 * accumulated in double in increasing k and scaled by 2^63. */
void orc_cdt(u64* cdt) {
    const double sigma = 3.2;
    double rho[20];
    for (int k = 0; k < 20; k++) rho[k] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
    double Z = rho[0];
    for (int k = 1; k < 20; k++) Z += 2.0 * rho[k];
    double cum = 0.0;
    for (int k = 0; k < 19; k++) {
        cum += (k == 0 ? rho[0] : 2.0 * rho[k]) / Z;
        cdt[k] = (u64)ldexp(cum, 63);
    }
}
/* Sign from the top bit; |x| = number of table entries the low 63 bits reach. */
int64_t orc_gauss(u64 r, const u64* cdt) {
    u64 u = r & 0x7FFFFFFFFFFFFFFFull;
    int64_t a = 0;
    for (int k = 0; k < 19; k++)
        if (u >= cdt[k]) a++;
    return (r >> 63) ? -a : a;
}

/* ------------------------------------------------------------------------ */
/* transforms                                                                */
/* ------------------------------------------------------------------------ */
/* Textbook in-place cyclic DFT over Z_m of length L (power of two):
 * out[k] = sum_j a[j] w^(jk), w a primitive L-th root.  Bit-reversal
 * permutation followed by log2(L) rounds of butterflies. */
static void cyclic_radix2(u64* a, u32 L, u64 w, u64 m) {
    u32 lg = ilog2(L);
    for (u32 i = 0; i < L; i++) {
        u32 j = orc_brv(i, lg);
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (u32 len = 2; len <= L; len <<= 1) {
        u64 wl = orc_powmod(w, L / len, m);
        for (u32 s = 0; s < L; s += len) {
            u64 tw = 1;
            for (u32 j = 0; j < len / 2; j++) {
                u64 x = a[s + j], y = mulm(a[s + j + len / 2], tw, m);
                a[s + j] = addm(x, y, m);
                a[s + j + len / 2] = subm(x, y, m);
                tw = mulm(tw, wl, m);
            }
        }
    }
}

/* Definition: out[k] = sum_j a[j] w^(jk) mod m. */
static void cyclic_direct(u64* a, u32 L, u64 w, u64 m) {
    u64* o = (u64*)calloc(L, sizeof(u64));
    for (u32 k = 0; k < L; k++) {
        u64 s = 0;
        for (u32 j = 0; j < L; j++) s = addm(s, mulm(a[j], orc_powmod(w, (u64)j * k % L, m), m), m);
        o[k] = s;
    }
    memcpy(a, o, L * sizeof(u64));
    free(o);
}

static void cyclic(u64* a, u32 L, u64 w, u64 m) {
    if (g_tier == 0) cyclic_direct(a, L, w, m);
    else cyclic_radix2(a, L, w, m);
}

/* Eq. 12 in two dimensions over the padded H x W plane (the paper's n_f is
 * read as the padded plane size, since Alice pads before transforming):
 *   X[k1][k2] = sum_{i,j} x[i][j] w_H^(i k1) w_W^(j k2) mod p,
 * w_L = g_p^((p-1)/L).  The inverse uses w^-1 and multiplies by (HW)^-1. */
static void ntt2d_plane_direct(u32 p, u32 H, u32 W, const u32* x, u32* X, int inverse) {
    u64 g = orc_primitive_root(p);
    u64 wH = orc_powmod(g, (p - 1) / H, p), wW = orc_powmod(g, (p - 1) / W, p);
    if (inverse) { wH = invm(wH, p); wW = invm(wW, p); }
    u64 scale = inverse ? invm((u64)H * W % p, p) : 1;
    for (u32 k1 = 0; k1 < H; k1++)
        for (u32 k2 = 0; k2 < W; k2++) {
            u64 s = 0;
            for (u32 i = 0; i < H; i++)
                for (u32 j = 0; j < W; j++) {
                    u64 tw = mulm(orc_powmod(wH, (u64)i * k1 % H, p), orc_powmod(wW, (u64)j * k2 % W, p), p);
                    s = addm(s, mulm(x[i * W + j], tw, p), p);
                }
            X[k1 * W + k2] = (u32)mulm(s, scale, p);
        }
}

static void ntt2d_plane_rowcol(u32 p, u32 H, u32 W, const u32* x, u32* X, int inverse) {
    u64 g = orc_primitive_root(p);
    u64 wH = orc_powmod(g, (p - 1) / H, p), wW = orc_powmod(g, (p - 1) / W, p);
    if (inverse) { wH = invm(wH, p); wW = invm(wW, p); }
    u64 scale = inverse ? invm((u64)H * W % p, p) : 1;
    u64* buf = (u64*)malloc((size_t)H * W * sizeof(u64));
    u64* col = (u64*)malloc(H * sizeof(u64));
    for (u32 i = 0; i < H * W; i++) buf[i] = x[i] % p;
    for (u32 i = 0; i < H; i++) cyclic(buf + (size_t)i * W, W, wW, p);
    for (u32 j = 0; j < W; j++) {
        for (u32 i = 0; i < H; i++) col[i] = buf[(size_t)i * W + j];
        cyclic(col, H, wH, p);
        for (u32 i = 0; i < H; i++) buf[(size_t)i * W + j] = col[i];
    }
    for (u32 i = 0; i < H * W; i++) X[i] = (u32)mulm(buf[i], scale, p);
    free(col);
    free(buf);
}

void orc_ntt2d(u32 p, u32 H, u32 W, const u32* x, u32* X, u64 planes, int inverse) {
    for (u64 pl = 0; pl < planes; pl++) {
        const u32* src = x + pl * H * W;
        u32* dst = X + pl * H * W;
        if (g_tier == 0) ntt2d_plane_direct(p, H, W, src, dst, inverse);
        else ntt2d_plane_rowcol(p, H, W, src, dst, inverse);
    }
}

/* Negacyclic transform of length L over Z_m with psi a primitive 2L-th root:
 *   out[i] = a(psi^(2 brv(i) + 1)) = sum_j a[j] psi^((2 brv(i) + 1) j),
 * i.e. evaluation of a(x) in Z_m[x]/(x^L + 1) at the L roots of x^L + 1, the
 * root for output i being psi^(2 brv_L(i) + 1) (the "bit-reversed evaluation
 * order").  Computed as twist a[j] psi^j, cyclic DFT with w = psi^2 (giving
 * index k = brv(i)), then the bit-reversal permutation. */
static void negacyclic_fwd(u64* a, u32 L, u64 psi, u64 m) {
    u32 lg = ilog2(L);
    if (g_tier == 0) {
        u64* o = (u64*)calloc(L, sizeof(u64));
        for (u32 i = 0; i < L; i++) {
            u64 e = 2ull * orc_brv(i, lg) + 1, s = 0;
            for (u32 j = 0; j < L; j++) s = addm(s, mulm(a[j], orc_powmod(psi, e * j % (2ull * L), m), m), m);
            o[i] = s;
        }
        memcpy(a, o, L * sizeof(u64));
        free(o);
        return;
    }
    u64 pw = 1;
    for (u32 j = 0; j < L; j++) { a[j] = mulm(a[j], pw, m); pw = mulm(pw, psi, m); }
    cyclic_radix2(a, L, mulm(psi, psi, m), m);
    for (u32 i = 0; i < L; i++) {
        u32 j = orc_brv(i, lg);
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

/* Inverse of negacyclic_fwd: a[j] = L^-1 sum_i out[i] psi^(-(2 brv(i)+1) j). */
static void negacyclic_inv(u64* a, u32 L, u64 psi, u64 m) {
    u32 lg = ilog2(L);
    u64 psi_inv = invm(psi, m), Linv = invm(L % m, m);
    if (g_tier == 0) {
        u64* o = (u64*)calloc(L, sizeof(u64));
        for (u32 j = 0; j < L; j++) {
            u64 s = 0;
            for (u32 i = 0; i < L; i++) {
                u64 e = (2ull * orc_brv(i, lg) + 1) * j % (2ull * L);
                s = addm(s, mulm(a[i], orc_powmod(psi_inv, e, m), m), m);
            }
            o[j] = mulm(s, Linv, m);
        }
        memcpy(a, o, L * sizeof(u64));
        free(o);
        return;
    }
    for (u32 i = 0; i < L; i++) {
        u32 j = orc_brv(i, lg);
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    cyclic_radix2(a, L, invm(mulm(psi, psi, m), m), m);
    u64 pw = Linv;
    for (u32 j = 0; j < L; j++) { a[j] = mulm(a[j], pw, m); pw = mulm(pw, psi_inv, m); }
}

/* Slot decode (SIMD packing, Smart-Vercaueren): slot i of a length-S slot set
 * is the plaintext polynomial evaluated at psi_p^(2 brv_S(i) + 1). */
void orc_slot_decode(const orc_params* P, const u32* m, u32* s) {
    u64* a = (u64*)malloc(P->S * sizeof(u64));
    for (u32 i = 0; i < P->S; i++) a[i] = m[i] % P->p;
    negacyclic_fwd(a, P->S, P->psi_p, P->p);
    for (u32 i = 0; i < P->S; i++) s[i] = (u32)a[i];
    free(a);
}
void orc_slot_encode(const orc_params* P, const u32* s, u32* m) {
    u64* a = (u64*)malloc(P->S * sizeof(u64));
    for (u32 i = 0; i < P->S; i++) a[i] = s[i] % P->p;
    negacyclic_inv(a, P->S, P->psi_p, P->p);
    for (u32 i = 0; i < P->S; i++) m[i] = (u32)a[i];
    free(a);
}
/* Ring products in R_q = Z_q[x]/(x^n + 1) become pointwise products after
 * this transform (Sec. 3.1: polynomial products are negacyclic convolutions;
 * Sec. 5.1: ciphertexts stay in this domain). */
void orc_ntt_q(const orc_params* P, const u64* a, u64* A) {
    if (A != a) memcpy(A, a, P->n * sizeof(u64));
    negacyclic_fwd(A, P->n, P->psi_q, P->q);
}
void orc_intt_q(const orc_params* P, const u64* A, u64* a) {
    if (A != a) memcpy(a, A, P->n * sizeof(u64));
    negacyclic_inv(a, P->n, P->psi_q, P->q);
}

/* Plaintext polynomial from d slot sets: m(x) = sum_r x^r m_r(x^d), each m_r
 * the slot encoding of slot set r.  `slots` holds d consecutive sets of S. */
static void encode_sets(const orc_params* P, const u32* slots, u32* m) {
    u32* mr = (u32*)malloc(P->S * sizeof(u32));
    for (u32 r = 0; r < P->d; r++) {
        orc_slot_encode(P, slots + (size_t)r * P->S, mr);
        for (u32 i = 0; i < P->S; i++) m[r + (size_t)P->d * i] = mr[i];
    }
    free(mr);
}
static void decode_sets(const orc_params* P, const u32* m, u32* slots) {
    u32* mr = (u32*)malloc(P->S * sizeof(u32));
    for (u32 r = 0; r < P->d; r++) {
        for (u32 i = 0; i < P->S; i++) mr[i] = m[r + (size_t)P->d * i];
        orc_slot_decode(P, mr, slots + (size_t)r * P->S);
    }
    free(mr);
}

/* ------------------------------------------------------------------------ */
/* protocol steps                                                            */
/* ------------------------------------------------------------------------ */
/* Secret key: ternary t (coefficients uniform on {-1, 0, 1}), stored as its
 * NTT_q image (Eq. 1 names a small secret t; its distribution is a reading). */
void orc_keygen(const orc_params* P, u64 seed, int64_t* t, u64* t_hat) {
    for (u32 i = 0; i < P->n; i++) {
        int64_t ti = (int64_t)(((u128)orc_rng(seed, DOM_T, i) * 3) >> 64) - 1;
        if (t) t[i] = ti;
        t_hat[i] = ti < 0 ? P->q - 1 : (u64)ti;
    }
    orc_ntt_q(P, t_hat, t_hat);
}

/* Packing (the paper flattens one spectrum per ciphertext; several blocks per
 * slot set is the reading taken).  Slot s of slot set r of input ciphertext
 * (bb, k, h):
 *   HW <= S: block = s / HW, f = s % HW; block < g_c g_b holds image
 *            b = (bb d + r) g_b + block / g_c, channel ci = k g_c + block % g_c;
 *   HW >  S: half h of image b = bb d + r, channel k, f = h S + s.
 * Absent images / channels give 0. */
static u32 input_slot(const orc_params* P, const orc_layer* L, const u32* X, u32 bb, u32 k, u32 h,
                      u32 r, u32 s) {
    u32 b, ci, f;
    if (L->HW <= P->S) {
        u32 blk = s / L->HW;
        if (blk >= L->g_c * L->g_b) return 0;
        f = s % L->HW;
        b = (bb * P->d + r) * L->g_b + blk / L->g_c;
        ci = k * L->g_c + blk % L->g_c;
    } else {
        f = h * P->S + s;
        b = bb * P->d + r;
        ci = k;
    }
    if (b >= L->B || ci >= L->Ci) return 0;
    return X[((size_t)b * L->Ci + ci) * L->HW + f];
}

void orc_pack_input(const orc_params* P, const orc_layer* L, const u32* X, u32* slots) {
    for (u32 bb = 0; bb < L->GB; bb++)
        for (u32 k = 0; k < L->T; k++)
            for (u32 h = 0; h < L->beta; h++) {
                u32* sl = slots + ((size_t)(bb * L->T + k) * L->beta + h) * P->n;
                for (u32 r = 0; r < P->d; r++)
                    for (u32 s = 0; s < P->S; s++) sl[r * P->S + s] = input_slot(P, L, X, bb, k, h, r, s);
            }
}

/* Eq. 1 with the ciphertext kept in the NTT_q domain (Sec. 5.1: the RLWE
 * constants a-hat and a-hat * t-hat are produced in that domain, so only the
 * message and error pass through NTT_q):
 *   c0-hat = -a-hat,  c1-hat = a-hat o t-hat + NTT_q(Delta m + e),
 * with m the slot encoding of the packed spectra and Delta = floor(q/p). */
void orc_encrypt(const orc_params* P, const orc_layer* L, const u64* t_hat, const u32* X, u64 seed,
                 u64* ct) {
    u64 cdt[19];
    orc_cdt(cdt);
    u32* slots = (u32*)malloc((size_t)P->n * sizeof(u32));
    u32* m = (u32*)malloc((size_t)P->n * sizeof(u32));
    u64* c = (u64*)malloc((size_t)P->n * sizeof(u64));
    for (u32 u = 0; u < L->n_in; u++) {
        u32 h = u % L->beta, k = (u / L->beta) % L->T, bb = u / (L->beta * L->T);
        for (u32 r = 0; r < P->d; r++)
            for (u32 s = 0; s < P->S; s++) slots[r * P->S + s] = input_slot(P, L, X, bb, k, h, r, s);
        encode_sets(P, slots, m);
        for (u32 i = 0; i < P->n; i++) {
            int64_t e = orc_gauss(orc_rng(seed, DOM_E, (u64)u * P->n + i), cdt);
            u64 em = e < 0 ? P->q - (u64)(-e) : (u64)e;
            c[i] = addm(mulm(P->delta, m[i], P->q), em, P->q);
        }
        orc_ntt_q(P, c, c);
        u64* c0 = ct + (size_t)u * 2 * P->n;
        u64* c1 = c0 + P->n;
        for (u32 j = 0; j < P->n; j++) {
            u64 idx = 2 * ((u64)u * P->n + j);
            u64 a = orc_uniform_q(P, orc_rng(seed, DOM_A, idx), orc_rng(seed, DOM_A, idx + 1));
            c0[j] = subm(0, a, P->q);
            c1[j] = addm(mulm(a, t_hat[j], P->q), c[j], P->q);
        }
    }
    free(c);
    free(m);
    free(slots);
}

/* Eq. 3 / Fig. 2 (Bob's reconstruction): [s_A] (+) s_B, a plaintext added to
 * c1 as NTT_q(Delta m_B), m_B the slot encoding of the packed NTT2D(s_B). */
void orc_homrec(const orc_params* P, const orc_layer* L, u64* ct, const u32* XB) {
    u32* slots = (u32*)malloc((size_t)P->n * sizeof(u32));
    u32* m = (u32*)malloc((size_t)P->n * sizeof(u32));
    u64* c = (u64*)malloc((size_t)P->n * sizeof(u64));
    for (u32 u = 0; u < L->n_in; u++) {
        u32 h = u % L->beta, k = (u / L->beta) % L->T, bb = u / (L->beta * L->T);
        for (u32 r = 0; r < P->d; r++)
            for (u32 s = 0; s < P->S; s++) slots[r * P->S + s] = input_slot(P, L, XB, bb, k, h, r, s);
        encode_sets(P, slots, m);
        for (u32 i = 0; i < P->n; i++) c[i] = mulm(P->delta, m[i], P->q);
        orc_ntt_q(P, c, c);
        u64* c1 = ct + (size_t)u * 2 * P->n + P->n;
        for (u32 j = 0; j < P->n; j++) c1[j] = addm(c1[j], c[j], P->q);
    }
    free(c);
    free(m);
    free(slots);
}

/* Fig. 2 (Bob): pad each filter to the H x W plane with the taps at
 * [0, fh) x [0, fw), map the signed weights mod p, NTT2D. */
void orc_filter_spectra(const orc_params* P, const orc_layer* L, const int8_t* w, u32 fh, u32 fw,
                        u32* What) {
    if (fh > L->H || fw > L->W) return; /* the filter must fit the padded plane */
    u32* plane = (u32*)malloc((size_t)L->HW * sizeof(u32));
    for (u32 co = 0; co < L->Co; co++)
        for (u32 ci = 0; ci < L->Ci; ci++) {
            memset(plane, 0, (size_t)L->HW * sizeof(u32));
            for (u32 a = 0; a < fh; a++)
                for (u32 c = 0; c < fw; c++) {
                    int v = w[(((size_t)co * L->Ci + ci) * fh + a) * fw + c];
                    plane[a * L->W + c] = (u32)((v % (int)P->p + (int)P->p) % (int)P->p);
                }
            orc_ntt2d(P->p, L->H, L->W, plane, What + ((size_t)co * L->Ci + ci) * L->HW, 1, 0);
        }
    free(plane);
}

/* Plaintext filter operand of SIMDScMult (Sec. 3.1): slot set 0 of filter
 * plaintext (co, k, h) holds, in each input block, the spectrum of channel
 * ci = k g_c + block % g_c of filter co (replicated over image blocks; half h
 * when HW > S).  Encoded, lifted to the centred range (-p/2, p/2] and placed
 * at the coefficients x^(d i) so that w(x) = w_0(x^d) multiplies every slot
 * set by the same slots; then NTT_q. */
void orc_filter_prepare(const orc_params* P, const orc_layer* L, const int8_t* w, u32 fh, u32 fw,
                        u64* Phat) {
    u32* What = (u32*)malloc((size_t)L->Co * L->Ci * L->HW * sizeof(u32));
    orc_filter_spectra(P, L, w, fh, fw, What);
    u32* slots = (u32*)malloc(P->S * sizeof(u32));
    u32* w0 = (u32*)malloc(P->S * sizeof(u32));
    for (u32 co = 0; co < L->Co; co++)
        for (u32 k = 0; k < L->T; k++)
            for (u32 h = 0; h < L->beta; h++) {
                for (u32 s = 0; s < P->S; s++) {
                    u32 v = 0;
                    if (L->HW <= P->S) {
                        u32 blk = s / L->HW, ci = k * L->g_c + blk % L->g_c;
                        if (blk < L->g_c * L->g_b && ci < L->Ci)
                            v = What[((size_t)co * L->Ci + ci) * L->HW + s % L->HW];
                    } else {
                        v = What[((size_t)co * L->Ci + k) * L->HW + h * P->S + s];
                    }
                    slots[s] = v;
                }
                orc_slot_encode(P, slots, w0);
                u64* out = Phat + ((size_t)(co * L->T + k) * L->beta + h) * P->n;
                memset(out, 0, P->n * sizeof(u64));
                for (u32 i = 0; i < P->S; i++) {
                    u32 v = w0[i];
                    out[(size_t)P->d * i] = (v <= (P->p - 1) / 2) ? v : P->q - (P->p - v);
                }
                orc_ntt_q(P, out, out);
            }
    free(w0);
    free(slots);
    free(What);
}

/* Eq. 2 (HomShare): Bob draws his share s_B-hat[b][co][f] uniform mod p and
 * subtracts it from the encrypted product.  With g_c channel blocks per slot
 * set the mask is split so that the client-side fold (sum over blocks)
 * yields y-hat - s_B-hat whatever the packing: block ic >= 1 gets a fresh
 * uniform r_ic, block 0 gets s_B-hat - sum r_ic.  M-hat = NTT_q(Delta m_s). */
static u32 mask_slot(const orc_params* P, const orc_layer* L, u64 seed, u32 bb, u32 co, u32 h, u32 r,
                     u32 s) {
    const u32 p = P->p;
    if (L->HW <= P->S) {
        u32 blk = s / L->HW;
        if (blk >= L->g_c * L->g_b) return 0;
        u32 f = s % L->HW, ic = blk % L->g_c;
        u32 b = (bb * P->d + r) * L->g_b + blk / L->g_c;
        if (b >= L->B) return 0;
        u64 base = (u64)b * L->Co + co;
        if (ic > 0) return orc_uniform_p(p, orc_rng(seed, DOM_MASK_SPLIT, (base * L->g_c + ic) * L->HW + f));
        u64 v = orc_uniform_p(p, orc_rng(seed, DOM_MASK, base * L->HW + f));
        for (u32 j = 1; j < L->g_c; j++)
            v = subm(v, orc_uniform_p(p, orc_rng(seed, DOM_MASK_SPLIT, (base * L->g_c + j) * L->HW + f)), p);
        return (u32)v;
    }
    u32 b = bb * P->d + r, f = h * P->S + s;
    if (b >= L->B) return 0;
    return orc_uniform_p(p, orc_rng(seed, DOM_MASK, ((u64)b * L->Co + co) * L->HW + f));
}

/* Noise flooding for circuit privacy (not in the paper; it leaves the
 * filter-dependent noise of HomConv in Bob's output ciphertext): the mask
 * plaintext Delta m_s gets, coefficient by coefficient, an error drawn
 * uniformly from [-2^f, 2^f), so that c1 - M_hat carries it too.  Decryption
 * rounds it away while the bound of orc_noise_ok_flood holds. */
static int64_t flood_error(u64 seed, u32 f, u64 idx) {
    return (int64_t)(orc_rng(seed, DOM_FLOOD, idx) >> (63 - f)) - ((int64_t)1 << f);
}

void orc_mask_prepare_flooded(const orc_params* P, const orc_layer* L, u64 seed, u32 flood_bits, u64* Mhat,
                              u32* sB) {
    for (u32 b = 0; b < L->B; b++)
        for (u32 co = 0; co < L->Co; co++)
            for (u32 f = 0; f < L->HW; f++)
                sB[((size_t)b * L->Co + co) * L->HW + f] =
                    orc_uniform_p(P->p, orc_rng(seed, DOM_MASK, ((u64)b * L->Co + co) * L->HW + f));
    u32* slots = (u32*)malloc(P->n * sizeof(u32));
    u32* m = (u32*)malloc(P->n * sizeof(u32));
    for (u32 v = 0; v < L->n_out; v++) {
        u32 h = v % L->beta, co = (v / L->beta) % L->Co, bb = v / (L->beta * L->Co);
        for (u32 r = 0; r < P->d; r++)
            for (u32 s = 0; s < P->S; s++) slots[r * P->S + s] = mask_slot(P, L, seed, bb, co, h, r, s);
        encode_sets(P, slots, m);
        u64* out = Mhat + (size_t)v * P->n;
        for (u32 i = 0; i < P->n; i++) {
            out[i] = mulm(P->delta, m[i], P->q);
            if (flood_bits) {
                int64_t e = flood_error(seed, flood_bits, (u64)v * P->n + i);
                out[i] = e >= 0 ? addm(out[i], (u64)e, P->q) : subm(out[i], (u64)(-e), P->q);
            }
        }
        orc_ntt_q(P, out, out);
    }
    free(m);
    free(slots);
}

void orc_mask_prepare(const orc_params* P, const orc_layer* L, u64 seed, u64* Mhat, u32* sB) {
    orc_mask_prepare_flooded(P, L, seed, 0, Mhat, sB);
}

/* Fig. 2 (Bob): [u-hat o w-hat] = [u-hat] (.) w-hat, summed over input
 * ciphertexts (the sum over input channels is implicit in the paper), then
 * HomShare subtracts the mask from c1.  In the NTT_q domain each ring
 * product is pointwise:
 *   out[bb][co][h][c][j] = sum_k in[bb][k][h][c][j] * P-hat[co][k][h][j] mod q,
 *   out[..][1][j] -= M-hat[bb][co][h][j]. */
void orc_homconv(const orc_params* P, const orc_layer* L, const u64* ct_in, const u64* Phat,
                 const u64* Mhat, u64* ct_out) {
    const u64 q = P->q;
    for (u32 bb = 0; bb < L->GB; bb++)
        for (u32 co = 0; co < L->Co; co++)
            for (u32 h = 0; h < L->beta; h++) {
                u32 v = (bb * L->Co + co) * L->beta + h;
                for (u32 c = 0; c < 2; c++)
                    for (u32 j = 0; j < P->n; j++) {
                        u64 acc = 0;
                        for (u32 k = 0; k < L->T; k++) {
                            u64 x = ct_in[(((size_t)(bb * L->T + k) * L->beta + h) * 2 + c) * P->n + j];
                            u64 w = Phat[((size_t)(co * L->T + k) * L->beta + h) * P->n + j];
                            acc = addm(acc, mulm(x, w, q), q);
                        }
                        if (c == 1 && Mhat) acc = subm(acc, Mhat[(size_t)v * P->n + j], q);
                        ct_out[((size_t)v * 2 + c) * P->n + j] = acc;
                    }
            }
}

/* Decryption of one ciphertext (Sec. 3.1): v = INTT_q(c0-hat o t-hat + c1-hat),
 * m_i = round(p v_i / q) mod p = floor((2 p v_i + q) / (2 q)) mod p (no ties:
 * q is an odd prime larger than p).  noise = max_i |centred(v_i - Delta m_i)|. */
void orc_decrypt_raw(const orc_params* P, const u64* t_hat, const u64* ct, u32* m, int64_t* noise) {
    const u64 q = P->q;
    u64* v = (u64*)malloc(P->n * sizeof(u64));
    for (u32 j = 0; j < P->n; j++) v[j] = addm(mulm(ct[j], t_hat[j], q), ct[P->n + j], q);
    orc_intt_q(P, v, v);
    int64_t worst = 0;
    for (u32 i = 0; i < P->n; i++) {
        u128 num = (u128)2 * P->p * v[i] + q;
        u64 z = (u64)(num / ((u128)2 * q)) % P->p;
        m[i] = (u32)z;
        u64 eta = subm(v[i], mulm(P->delta, z, q), q);
        int64_t c = eta > q / 2 ? -(int64_t)(q - eta) : (int64_t)eta;
        if (c < 0) c = -c;
        if (c > worst) worst = c;
    }
    if (noise) *noise = worst;
    free(v);
}

/* Fig. 2 (Alice): decrypt, decode the slots, and fold the channel blocks of
 * each image back onto one spectrum: S_A-hat[b][co][f] = sum_ic slot mod p.
 * With HomShare this is y-hat - s_B-hat for every packing. */
void orc_decrypt(const orc_params* P, const orc_layer* L, const u64* t_hat, const u64* ct, u32* SA,
                 int64_t* noise) {
    const u32 p = P->p;
    memset(SA, 0, (size_t)L->B * L->Co * L->HW * sizeof(u32));
    u32* m = (u32*)malloc(P->n * sizeof(u32));
    u32* slots = (u32*)malloc(P->n * sizeof(u32));
    for (u32 v = 0; v < L->n_out; v++) {
        u32 h = v % L->beta, co = (v / L->beta) % L->Co, bb = v / (L->beta * L->Co);
        int64_t nz;
        orc_decrypt_raw(P, t_hat, ct + (size_t)v * 2 * P->n, m, &nz);
        if (noise) noise[v] = nz;
        decode_sets(P, m, slots);
        for (u32 r = 0; r < P->d; r++)
            for (u32 s = 0; s < P->S; s++) {
                u32 val = slots[r * P->S + s], b, f;
                if (L->HW <= P->S) {
                    u32 blk = s / L->HW;
                    if (blk >= L->g_c * L->g_b) continue;
                    b = (bb * P->d + r) * L->g_b + blk / L->g_c;
                    f = s % L->HW;
                } else {
                    b = bb * P->d + r;
                    f = h * P->S + s;
                }
                if (b >= L->B) continue;
                u32* dst = SA + ((size_t)b * L->Co + co) * L->HW + f;
                *dst = (u32)addm(*dst, val, p);
            }
    }
    free(slots);
    free(m);
}

/* The result the protocol computes (Eq. 6 with Eqs. 9-11: s_A + s_B = u * w):
 * cyclic 2D convolution of the summed shares with the filters, summed over
 * input channels, mod p:
 *   y[b][co][i][j] = sum_ci sum_{a<fh, c<fw} w[co][ci][a][c] x[b][ci][(i-a) mod H][(j-c) mod W]. */
/* Appendix, "Average Pooling" layers: each 2x2 window of a share summed mod p
   (the 1/4 of the average belongs to the next layer's weights). */
void orc_pool2x2_sum(u32 p, u64 planes, u32 H, u32 W, const u32* x, u32* y) {
    for (u64 pl = 0; pl < planes; pl++)
        for (u32 i = 0; i < H / 2; i++)
            for (u32 j = 0; j < W / 2; j++) {
                u64 acc = 0;
                for (u32 a = 0; a < 2; a++)
                    for (u32 c = 0; c < 2; c++) acc += x[(pl * H + 2 * i + a) * W + 2 * j + c];
                y[(pl * (H / 2) + i) * (W / 2) + j] = (u32)(acc % p);
            }
}

void orc_conv_plain(u32 p, u32 B, u32 Ci, u32 Co, u32 H, u32 W, const u32* x, const int8_t* w, u32 fh,
                    u32 fw, u32* y) {
    for (u32 b = 0; b < B; b++)
        for (u32 co = 0; co < Co; co++)
            for (u32 i = 0; i < H; i++)
                for (u32 j = 0; j < W; j++) {
                    u64 acc = 0;
                    for (u32 ci = 0; ci < Ci; ci++)
                        for (u32 a = 0; a < fh; a++)
                            for (u32 c = 0; c < fw; c++) {
                                int wv = w[(((size_t)co * Ci + ci) * fh + a) * fw + c];
                                u64 wm = (u64)((wv % (int)p + (int)p) % (int)p);
                                u32 ii = (i + H - a % H) % H, jj = (j + W - c % W) % W;
                                acc = (acc + wm * x[(((size_t)b * Ci + ci) * H + ii) * W + jj]) % p;
                            }
                    y[(((size_t)b * Co + co) * H + i) * W + j] = (u32)acc;
                }
}
