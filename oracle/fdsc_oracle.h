/*
 * fdsc_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded CPU statement of what the frequency-domain
 * secure convolution (FDSC) of ENSEI computes (Bian, Wang, Hiromoto, Shi,
 * Sato, "ENSEI: Efficient Secure Inference via Frequency-Domain Homomorphic
 * Convolution for Privacy-Preserving Visual Recognition", CVPR 2020).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this code.  It shares no source with the CUDA library and includes none
 * of its headers.  All arithmetic is exact: every modular product goes through
 * an unsigned __int128 and the C '%' operator.
 *
 * Parity status: every function here is pinned by a CPU test against
 * something other than itself (paper-printed parameters, closed forms,
 * brute force on tiny inputs, library routines); see tests/test_oracle_*.py.
 */
#ifndef FDSC_ORACLE_H
#define FDSC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Scheme parameters for one (n, p) pair (Sec. 3.1 BFV triple (n, p_E, q);
 * Sec. 5.2 moduli; Sec. 6.4 instantiation).  One prime p plays the roles of
 * p_N, p_A and p_E. */
typedef struct {
    uint32_t n, logn;       /* ring degree, power of two                         */
    uint32_t p;             /* plaintext / sharing / NTT prime                    */
    uint32_t S, logS, d;    /* slot-set size S = min(n, 2^(v2(p-1)-1)), d = n/S   */
    uint32_t g_p;           /* smallest primitive root mod p                      */
    uint32_t psi_p;         /* primitive 2S-th root of unity mod p                */
    uint32_t pad0;
    uint64_t q;             /* largest prime < 2^60 with q = 1 mod 8192*p         */
    uint64_t g_q;           /* smallest primitive root mod q                      */
    uint64_t psi_q;         /* primitive 2n-th root of unity mod q                */
    uint64_t delta;         /* floor(q/p)                                         */
    uint64_t r_q;           /* q mod p                                            */
} orc_params;

/* One convolution layer and its ciphertext packing. */
typedef struct {
    uint32_t B, Ci, Co, H, W;   /* images, channels, padded plane               */
    uint32_t g_c, g_b;          /* channel blocks x image blocks per slot-set     */
    uint32_t HW, T, GB, beta;   /* derived: T = ceil(Ci/g_c), GB = ceil(B/g_b),
                                   beta = spectrum halves per channel (HW > S)    */
    uint32_t n_in, n_out;       /* input / output ciphertext counts               */
} orc_layer;

/* tier 0: every transform is its O(N^2) definition; tier 1: radix-2. */
void     orc_set_tier(int tier);
int      orc_get_tier(void);

/* arithmetic helpers exposed for pinning */
int      orc_is_prime(uint64_t m);
uint64_t orc_powmod(uint64_t b, uint64_t e, uint64_t m);
uint64_t orc_primitive_root(uint64_t m);
uint64_t orc_min_prime_1mod(uint64_t lower, uint64_t modulus);
uint64_t orc_find_q(uint32_t p);
uint32_t orc_brv(uint32_t i, uint32_t logL);

int      orc_params_init(uint32_t n, uint32_t p, orc_params* P);
int      orc_layer_init(const orc_params* P, uint32_t B, uint32_t Ci, uint32_t Co,
                        uint32_t H, uint32_t W, uint32_t g_c, uint32_t g_b, orc_layer* L);
double   orc_noise_bound_log2(const orc_params* P, uint32_t T);
int      orc_noise_ok(const orc_params* P, uint32_t T);
int      orc_noise_ok_flood(const orc_params* P, uint32_t T, uint32_t flood_bits);

/* counter-based randomness (SplitMix64 output function) */
uint64_t orc_rng(uint64_t seed, uint64_t domain, uint64_t idx);
void     orc_cdt(uint64_t* cdt /* [19] */);
int64_t  orc_gauss(uint64_t r, const uint64_t* cdt);
uint64_t orc_uniform_q(const orc_params* P, uint64_t r1, uint64_t r2);
uint32_t orc_uniform_p(uint32_t p, uint64_t r);

/* transforms */
void orc_ntt2d(uint32_t p, uint32_t H, uint32_t W, const uint32_t* x, uint32_t* X,
               uint64_t planes, int inverse);
void orc_slot_decode(const orc_params* P, const uint32_t* m, uint32_t* s);   /* length S */
void orc_slot_encode(const orc_params* P, const uint32_t* s, uint32_t* m);
void orc_ntt_q(const orc_params* P, const uint64_t* a, uint64_t* A);        /* length n */
void orc_intt_q(const orc_params* P, const uint64_t* A, uint64_t* a);

/* protocol steps */
void orc_keygen(const orc_params* P, uint64_t seed, int64_t* t /*nullable [n]*/, uint64_t* t_hat);
void orc_pack_input(const orc_params* P, const orc_layer* L, const uint32_t* X, uint32_t* slots);
void orc_encrypt(const orc_params* P, const orc_layer* L, const uint64_t* t_hat,
                 const uint32_t* X, uint64_t seed, uint64_t* ct);
void orc_homrec(const orc_params* P, const orc_layer* L, uint64_t* ct, const uint32_t* XB);
void orc_filter_spectra(const orc_params* P, const orc_layer* L, const int8_t* w,
                        uint32_t fh, uint32_t fw, uint32_t* What);
void orc_filter_prepare(const orc_params* P, const orc_layer* L, const int8_t* w,
                        uint32_t fh, uint32_t fw, uint64_t* Phat);
void orc_mask_prepare(const orc_params* P, const orc_layer* L, uint64_t seed,
                      uint64_t* Mhat, uint32_t* sB);
/* the same mask with noise flooding of 2^flood_bits (0: none) */
void orc_mask_prepare_flooded(const orc_params* P, const orc_layer* L, uint64_t seed, uint32_t flood_bits,
                              uint64_t* Mhat, uint32_t* sB);
void orc_homconv(const orc_params* P, const orc_layer* L, const uint64_t* ct_in,
                 const uint64_t* Phat, const uint64_t* Mhat, uint64_t* ct_out);
void orc_decrypt(const orc_params* P, const orc_layer* L, const uint64_t* t_hat,
                 const uint64_t* ct, uint32_t* SA, int64_t* noise /*nullable [n_out]*/);
void orc_decrypt_raw(const orc_params* P, const uint64_t* t_hat, const uint64_t* ct,
                     uint32_t* m, int64_t* noise);

/* the appendix networks' average pooling on a share, as a 2x2 sum pool mod p:
   y[pl][i][j] = sum_{a,b<2} x[pl][2i+a][2j+b] mod p */
void orc_pool2x2_sum(uint32_t p, uint64_t planes, uint32_t H, uint32_t W, const uint32_t* x, uint32_t* y);

/* the result the protocol must reproduce: cyclic 2D convolution mod p */
void orc_conv_plain(uint32_t p, uint32_t B, uint32_t Ci, uint32_t Co, uint32_t H, uint32_t W,
                    const uint32_t* x, const int8_t* w, uint32_t fh, uint32_t fw, uint32_t* y);

#ifdef __cplusplus
}
#endif
#endif
