/*
 * fdsc.h -- C ABI of libfdsc, the GB300 (sm_103a) implementation of the
 * frequency-domain secure convolution (FDSC) of ENSEI (Bian, Wang, Hiromoto,
 * Shi, Sato, CVPR 2020).
 *
 * One convolution layer, Fig. 2 of the paper, runs as:
 *   Alice  fdsc_ntt2d(x_A) -> fdsc_encrypt               (transform, encrypt)
 *   Bob    fdsc_ntt2d(x_B) -> fdsc_homrec               (HomRec, Eq. 3)
 *   Bob    fdsc_homconv (Hadamard product summed over input channels,
 *          fused with HomShare)                          (Eq. 2)
 *   Alice  fdsc_decrypt -> fdsc_intt2d;  Bob fdsc_intt2d(s_B-hat)
 *                                                        (decrypt, inverse transform)
 * with setup (no user input): fdsc_params_create, fdsc_keygen,
 * fdsc_filter_prepare, fdsc_mask_prepare.
 *
 * Conventions
 *  - Every call returns an int status: FDSC_OK (0) or a negative FDSC_ERR_*.
 *    fdsc_last_error() returns a message for the calling thread's last
 *    failure.  No C++ exception crosses this boundary.
 *  - Tensor arguments are DEVICE pointers owned by the caller (allocated on
 *    the device that was current when the params object was created); the
 *    library never frees them and keeps no reference after the call.  The
 *    only library-owned memory is the params object's constant tables.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All compute calls are asynchronous on that stream; argument
 *    errors are reported before anything is enqueued, launch errors after.
 *  - Element types: Z_p data uint32 in [0, p); Z_q data uint64 in [0, q);
 *    weights int8.  All arrays are dense, row-major, with the shapes given.
 *  - Z_q arrays must be 16-byte aligned and Z_p arrays 16-byte aligned
 *    (the kernels use 128-bit loads); FDSC_ERR_ARG otherwise.
 *  - Transform orders: NTT2D / INTT2D spectra are in natural order
 *    (k1, k2), f = k1 W + k2.  Ciphertext words index j holds the evaluation
 *    of the ring element at psi_q^(2 brv_n(j) + 1); slot i of a slot set is
 *    the plaintext evaluated at psi_p^(2 brv_S(i) + 1).
 */
#ifndef FDSC_H
#define FDSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FDSC_OK = 0,
    FDSC_ERR_ARG = -1,         /* invalid argument, shape or alignment            */
    FDSC_ERR_NOISE = -2,       /* the decryption noise bound fails (q too small)  */
    FDSC_ERR_OOM = -3,         /* device or host allocation failed                */
    FDSC_ERR_CUDA = -4,        /* a CUDA runtime call or kernel launch failed     */
    FDSC_ERR_UNSUPPORTED = -5, /* valid but outside what this library implements  */
    FDSC_ERR_TIMEOUT = -6,     /* a bounded wait ran out                          */
    FDSC_ERR_BUDGET = -7       /* a request can never fit the server's HBM budget */
};

/* Message for the calling thread's most recent failure ("" if none). */
const char* fdsc_last_error(void);

/* ---------------------------------------------------------------------- */
/* Parameters (Sec. 3.1 BFV triple (n, p_E, q); Sec. 5.2 moduli; Sec. 6.4) */
/* ---------------------------------------------------------------------- */
/* One prime p serves as NTT, sharing and plaintext modulus.  q is the
 * largest prime below 2^60 with q = 1 mod 8192 p, Delta = floor(q / p).
 * S = min(n, 2^(v2(p-1)-1)) slots per slot set, d = n / S slot sets per
 * ciphertext (d > 1 when x^n + 1 does not split into linear factors mod p). */
typedef struct {
    uint32_t n, logn, p, S, logS, d;
    uint32_t g_p, psi_p;        /* smallest primitive root mod p; 2S-th root  */
    uint64_t q, g_q, psi_q;     /* modulus; smallest primitive root; 2n-th root */
    uint64_t delta, r_q;        /* floor(q/p), q mod p                          */
} fdsc_params_info;

typedef struct fdsc_params fdsc_params; /* opaque */

/* Host-only derivation of the parameters for ring degree n (power of two,
 * 16 <= n <= 4096) and prime p (< 2^20, p = 1 mod 4).  Touches no device.
 * FDSC_ERR_ARG for unsupported (n, p). */
int fdsc_params_query(uint32_t n, uint32_t p, fdsc_params_info* out);

/* Creates the params object on the CURRENT device: derives the parameters
 * and uploads the twiddle tables (about 40 n bytes).  max_T is the largest
 * number of input ciphertexts a HomConv output will sum; the worst-case
 * decryption noise
 *   T n (19 + r_q) floor(p/2) + r_q ceil(T n (p-1) floor(p/2) / p) + r_q
 * must keep p |noise| + r_q (p-1) < q/2, else FDSC_ERR_NOISE. */
int fdsc_params_create(uint32_t n, uint32_t p, uint32_t max_T, fdsc_params** out);
int fdsc_params_destroy(fdsc_params* P);
int fdsc_params_get_info(const fdsc_params* P, fdsc_params_info* out);

/* The Gaussian sampler's cumulative table (sigma = 3.2, |e| <= 19; 2^63
 * scaled), for cross-checking; 19 entries. */
int fdsc_gauss_table(uint64_t* out19);

/* ---------------------------------------------------------------------- */
/* Layer shape and ciphertext packing                                      */
/* ---------------------------------------------------------------------- */
/* B images of Ci channels on an H x W plane (powers of two, H W <= 4096,
 * H and W dividing p-1), Co filters.  When H W <= S, one slot set holds
 * g_c x g_b blocks of H W slots (g_c channels of g_b images;
 * g_c g_b H W <= S); when H W > S, one channel spectrum spans
 * beta = H W / S ciphertexts ("halves") and g_c = g_b = 1. */
typedef struct {
    uint32_t B, Ci, Co, H, W, g_c, g_b;
} fdsc_layer;

typedef struct {
    uint32_t HW, T, GB, beta;   /* T = ceil(Ci/g_c) (or Ci); GB = ceil(B/(d g_b)) */
    uint32_t n_in, n_out;       /* input ciphertexts GB T beta; outputs GB Co beta */
    uint64_t ct_in_words;       /* n_in  * 2 * n   (uint64)                       */
    uint64_t ct_out_words;      /* n_out * 2 * n                                  */
    uint64_t filter_words;      /* Co * T * beta * n / d (one word per group of d) */
    uint64_t mask_words;        /* n_out * n                                      */
    uint64_t in_spectra_words;  /* B * Ci * H W    (uint32)                       */
    uint64_t out_spectra_words; /* B * Co * H W                                   */
} fdsc_layout;

int fdsc_layout_query(uint32_t n, uint32_t p, const fdsc_layer* L, fdsc_layout* out);

/* ---------------------------------------------------------------------- */
/* Transforms                                                              */
/* ---------------------------------------------------------------------- */
/* Eq. 12 in two dimensions (the cyclic NTT over the padded H x W plane,
 * Fig. 2, both parties' forward transforms): X[k1][k2] = sum_{i,j} x[i][j] w_H^(i k1) w_W^(j k2)
 * mod p, w_L = g_p^((p-1)/L).  x, X: uint32 [planes][H][W]; x may equal X. */
int fdsc_ntt2d(const fdsc_params* P, uint32_t H, uint32_t W, const uint32_t* x, uint32_t* X,
               uint64_t planes, void* stream);
/* Fig. 2's final inverse transform, x = (HW)^-1 sum X w^-(...). */
int fdsc_intt2d(const fdsc_params* P, uint32_t H, uint32_t W, const uint32_t* X, uint32_t* x,
                uint64_t planes, void* stream);

/* The average-pooling layers of the paper's appendix networks, on a share:
 * y[pl][i][j] = sum_{a,b < 2} x[pl][2i+a][2j+b] mod p (H, W even; x in
 * [0, p)).  It is linear mod p, so each party pools its own share and the
 * pooled shares add up to the pooled value; the 1/4 of the average is left
 * to the next layer's weights (a sum pool).  x: [planes][H][W], y:
 * [planes][H/2][W/2], both device, not overlapping. */
int fdsc_pool2x2_sum(const fdsc_params* P, uint32_t H, uint32_t W, const uint32_t* x, uint32_t* y,
                     uint64_t planes, void* stream);

/* ---------------------------------------------------------------------- */
/* Setup                                                                   */
/* ---------------------------------------------------------------------- */
/* Secret key of Eq. 1: ternary t (uniform on {-1,0,1}, drawn from `seed`),
 * written as t_hat = NTT_q(t): uint64 [n]. */
int fdsc_keygen(const fdsc_params* P, uint64_t seed, uint64_t* t_hat, void* stream);

/* Fig. 2, Bob's filter transform: w_hat = flatten(NTT2D(W)) packed into plaintext
 * polynomials and lifted to NTT_q.  w: int8 [Co][Ci][fh][fw] (taps at the
 * top-left of the padded plane, fh <= H, fw <= W); P_hat: uint64
 * [Co][T][beta][n / d] -- plaintext (co, k, h) holds the spectra of channels
 * k g_c .. k g_c + g_c - 1 in its blocks, centred-lifted, at x^(d i), so it
 * is a polynomial w_0(x^d) and takes one value on each group of d
 * consecutive NTT_q indices (the points x times the d-th roots of unity):
 * word i is the value of indices i d .. i d + d - 1 (with d = 1, one word per
 * index). */
int fdsc_filter_prepare(const fdsc_params* P, const fdsc_layer* L, const int8_t* w, uint32_t fh,
                        uint32_t fw, uint64_t* P_hat, void* stream);

/* Eq. 2 (HomShare) randomness, drawn from `seed`: Bob's share
 * sB_hat: uint32 [B][Co][H W], uniform mod p, and the encrypted-domain mask
 * M_hat: uint64 [GB][Co][beta][n] = NTT_q(Delta * encode(mask slots)), the
 * mask split over the g_c channel blocks so that the decrypt-side fold
 * gives y_hat - sB_hat for every packing. */
int fdsc_mask_prepare(const fdsc_params* P, const fdsc_layer* L, uint64_t seed, uint64_t* M_hat,
                      uint32_t* sB_hat, void* stream);

/* HomShare with noise flooding for circuit privacy (not in the paper, whose
 * HomShare leaves the filter-dependent noise of HomConv in Bob's output
 * ciphertext): as fdsc_mask_prepare, but every coefficient of the mask
 * plaintext Delta m_s also carries an error drawn from `seed` uniformly in
 * [-2^flood_bits, 2^flood_bits), which c1 - M_hat then carries too.
 * Decryption rounds it away, so the final shares are those of
 * fdsc_mask_prepare with the same seed.  FDSC_ERR_NOISE when the layer's
 * noise bound (T input ciphertexts) plus 2^flood_bits fails; 0 gives
 * fdsc_mask_prepare's words. */
int fdsc_mask_prepare_flooded(const fdsc_params* P, const fdsc_layer* L, uint64_t seed, uint32_t flood_bits,
                              uint64_t* M_hat, uint32_t* sB_hat, void* stream);
/* The largest flood_bits the noise bound admits for T input ciphertexts at
 * (n, p); FDSC_ERR_NOISE if T alone breaks it. */
int fdsc_flood_bits_max(uint32_t n, uint32_t p, uint32_t T, uint32_t* out);

/* ---------------------------------------------------------------------- */
/* Online path                                                             */
/* ---------------------------------------------------------------------- */
/* Eq. 1 in the NTT_q domain (Sec. 5.1): X: uint32 [B][Ci][H W] spectra
 * (NTT2D of Alice's share); ct: uint64 [GB][T][beta][2][n] with
 * c0_hat = -a_hat, c1_hat = a_hat o t_hat + NTT_q(Delta m + e); a_hat
 * uniform mod q and e ~ D_{3.2}, |e| <= 19, both drawn from `seed`. */
int fdsc_encrypt(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat, const uint32_t* X,
                 uint64_t seed, uint64_t* ct, void* stream);

/* Eq. 3 (HomRec): ct (in place) += the plaintext encoding of XB, Bob's share
 * spectra uint32 [B][Ci][H W] packed like the ciphertext. */
int fdsc_homrec(const fdsc_params* P, const fdsc_layer* L, const uint32_t* XB, uint64_t* ct,
                void* stream);

/* Fig. 2, Bob's HomConv and HomShare (Eq. 2): ct_out[bb][co][h][c][j] = sum_k ct_in[bb][k][h][c][j]
 * P_hat[co][k][h][j / d] mod q, then c1 -= M_hat[bb][co][h] (HomShare; skipped
 * when M_hat is NULL).  ct_out: uint64 [GB][Co][beta][2][n]; must not alias
 * ct_in.  Exact: the sum is formed in 128 bits and reduced once per 256
 * terms. */
int fdsc_homconv(const fdsc_params* P, const fdsc_layer* L, const uint64_t* ct_in,
                 const uint64_t* P_hat, const uint64_t* M_hat, uint64_t* ct_out, void* stream);

/* Fig. 2, Alice's decryption (Sec. 3.1): v = INTT_q(c0_hat o t_hat + c1_hat),
 * m = floor((2 p v + q) / (2 q)) mod p, slots = decode(m), and the g_c
 * channel blocks of each image folded: SA_hat: uint32 [B][Co][H W]. */
int fdsc_decrypt(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat,
                 const uint64_t* ct, uint32_t* SA_hat, void* stream);

/* ---------------------------------------------------------------------- */
/* Fused online path: the same words as the step-by-step calls, in fewer   */
/* kernels, with the input-independent work separable from the rest.      */
/* ---------------------------------------------------------------------- */
/* Eq. 1 with a zero message, in the NTT_q domain: for every input
 * ciphertext u, ct[u] = (-a_hat, a_hat o t_hat + NTT_q(e)), a_hat and e
 * drawn from `seed` exactly as fdsc_encrypt draws them.  These are the RLWE
 * constants of Sec. 5.1 (no user input).  Because NTT_q is linear,
 *   fdsc_encrypt(X = NTT2D(x), seed) = this + (0, fdsc_encode_share(x)). */
int fdsc_encrypt_constants(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat, uint64_t seed,
                           uint64_t* ct, void* stream);

/* The message part of Alice's encryption in Fig. 2 (and of Bob's HomRec
 * plaintext) from a SPATIAL share
 * x: uint32 [B][Ci][H][W] -> NTT2D -> flatten and pack -> slot encode ->
 * times Delta -> NTT_q, written to A: uint64 [n_in][n].  Needs
 * 8 <= H, W <= 512 (FDSC_ERR_UNSUPPORTED otherwise; use fdsc_ntt2d +
 * fdsc_encrypt).  When H W > S the spectrum of a channel spans beta
 * ciphertexts: the kernel of ciphertext (bb, k, h) transforms the d image
 * planes of its slot sets and keeps half h. */
int fdsc_encode_share(const fdsc_params* P, const fdsc_layer* L, const uint32_t* x, uint64_t* A, void* stream);

/* The three input-side producers of one online layer in ONE launch, with the
 * words of the separate calls: ct <- fdsc_encrypt_constants(t_hat, seed)
 * (Alice's RLWE constants of Eq. 1, Sec. 5.1), A <- fdsc_encode_share(xA)
 * (her message plaintext) and R <- fdsc_encode_share(xB) (Bob's HomRec
 * plaintext of Eq. 3); one CTA per (producer, input ciphertext).  ct:
 * [n_in][2][n], A, R: [n_in][n], none overlapping.  P_hat and M_hat (either
 * may be NULL) are the filter plaintexts [Co][T][beta][n] and HomShare masks
 * [GB][Co][beta][n] of the HomConv that follows: the launch asks the L2
 * cache to fetch them while its transforms run, so that the HomConv finds
 * them on chip.  The kernel lets the next kernel in the stream start early
 * (programmatic dependent launch).  Same restrictions as fdsc_encode_share. */
int fdsc_online_produce(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat, uint64_t seed,
                        const uint32_t* xA, const uint32_t* xB, uint64_t* ct, uint64_t* A, uint64_t* R,
                        const uint64_t* P_hat, const uint64_t* M_hat, void* stream);

/* Eq. 3 (HomRec) from Bob's SPATIAL share: ct.c1 += fdsc_encode_share(xB).
 * Same restrictions as fdsc_encode_share. */
int fdsc_homrec_share(const fdsc_params* P, const fdsc_layer* L, const uint32_t* xB, uint64_t* ct, void* stream);

/* fdsc_homconv applied to the ciphertexts (c0, c1 + A1 + A2): the message and
 * HomRec plaintexts of fdsc_encode_share are added to c1 as it is read.  A1,
 * A2: uint64 [n_in][n] or NULL.  ct_out must not overlap any input. */
int fdsc_homconv_sum(const fdsc_params* P, const fdsc_layer* L, const uint64_t* ct_in, const uint64_t* A1,
                     const uint64_t* A2, const uint64_t* P_hat, const uint64_t* M_hat, uint64_t* ct_out,
                     void* stream);

/* HomConv on the tensor cores (the same words as fdsc_homconv_sum).  For
 * every evaluation index the contraction over the T input ciphertexts is a
 * matrix product of 60-bit words; each word is split into eight balanced
 * base-256 digits (held exactly in fp16), the digit products are summed by
 * tcgen05 MMAs in fp32 into the 15 weight classes 256^kappa (exact: every
 * partial sum stays below 2^24 for T <= 128), and the classes are combined
 * into the 128-bit sum and reduced mod q once.
 * fdsc_filter_tc_words: the size in uint64 words of the digit-plane filter
 * for layer L at (n, p) (host only); FDSC_ERR_UNSUPPORTED if T > 128.
 * fdsc_filter_tc: P_hat uint64 [Co][T][beta][n / d] (fdsc_filter_prepare) ->
 * P_tc: per group of d evaluation indices (beta n / d), block of 16 input ciphertexts and
 * tile of up to 128 output channels (rows rounded up to a multiple of 8),
 * the eight fp16 digit planes of the filter words in the canonical layout of
 * a tcgen05 A operand (256 bytes per row); twice the bytes of P_hat.  Setup,
 * once per filter.
 * fdsc_homconv_tc: as fdsc_homconv_sum with P_tc in place of P_hat; ct_out
 * must not overlap any input.  Launches one persistent CTA per SM.
 * fdsc_homconv_tc_status: after synchronizing, 0 in *code if no CTA of the
 * tensor-core kernel gave up a bounded wait since the last call; otherwise
 * the role that did (1 loader, 2 MMA, 3 epilogue, 4 converter) and
 * FDSC_ERR_TIMEOUT (that launch's output is not valid).  Resets the flag. */
int fdsc_filter_tc_words(uint32_t n, uint32_t p, const fdsc_layer* L, uint64_t* words);
int fdsc_filter_tc(const fdsc_params* P, const fdsc_layer* L, const uint64_t* P_hat, uint64_t* P_tc,
                   void* stream);
int fdsc_homconv_tc(const fdsc_params* P, const fdsc_layer* L, const uint64_t* ct_in, const uint64_t* A1,
                    const uint64_t* A2, const uint64_t* P_tc, const uint64_t* M_hat, uint64_t* ct_out,
                    void* stream);
int fdsc_homconv_tc_status(uint32_t* code);

/* Seeded ciphertexts.  In Eq. 1 `a` is uniform and public, so a fresh
 * ciphertext can travel as its encryption seed and c1 alone: half the
 * client-to-server bytes, and half the input words HomConv reads.
 * fdsc_encrypt_constants_seeded writes the c1 of fdsc_encrypt_constants,
 * c1: uint64 [n_in][n] (the message and HomRec plaintexts are then added as
 * A1 / A2 below, or into c1).  fdsc_homconv_seeded is fdsc_homconv_sum with
 * c0 = -a drawn again from `seed` (the encryption's) instead of read: the
 * same output words as fdsc_homconv_sum on the full ciphertexts.  Needs
 * T <= 256 (FDSC_ERR_UNSUPPORTED otherwise). */
int fdsc_encrypt_constants_seeded(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat, uint64_t seed,
                                  uint64_t* c1, void* stream);
int fdsc_homconv_seeded(const fdsc_params* P, const fdsc_layer* L, uint64_t seed, const uint64_t* c1,
                        const uint64_t* A1, const uint64_t* A2, const uint64_t* P_hat, const uint64_t* M_hat,
                        uint64_t* ct_out, void* stream);

/* Alice's last two steps of Fig. 2 in one kernel: decrypt, decode, fold the channel
 * blocks and INTT2D, giving her SPATIAL share y: uint32 [B][Co][H][W]
 * (= fdsc_intt2d(fdsc_decrypt(...))).  Same restrictions as
 * fdsc_encode_share. */
int fdsc_decrypt_share(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat, const uint64_t* ct,
                       uint32_t* y, void* stream);

/* ---------------------------------------------------------------------- */
/* Several clients in one call                                             */
/* ---------------------------------------------------------------------- */
/* The same as fdsc_encrypt_constants, fdsc_mask_prepare and
 * fdsc_decrypt_share, but image group g (GB groups; one image per group when
 * d = g_b = 1) uses its own key t_hats + g * key_stride (uint64 words; 0 = one
 * key for all; even) and its own seed seeds[g] (DEVICE array of GB uint64),
 * with its randomness indexed from 0 inside the group.  Each group's words are
 * therefore exactly those of a call with that group alone (B = its images,
 * that key, that seed), whatever else shares the launch -- what batching
 * independent requests needs. */
int fdsc_encrypt_constants_multi(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hats,
                                 uint64_t key_stride, const uint64_t* seeds, uint64_t* ct, void* stream);
int fdsc_mask_prepare_multi(const fdsc_params* P, const fdsc_layer* L, const uint64_t* seeds, uint64_t* M_hat,
                            uint32_t* sB_hat, void* stream);
int fdsc_decrypt_share_multi(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hats, uint64_t key_stride,
                             const uint64_t* ct, uint32_t* y, void* stream);

/* ---------------------------------------------------------------------- */
/* Batched plan: many layers and images in one graph launch                */
/* ---------------------------------------------------------------------- */
/* Not in the paper (a batching runtime around its per-layer protocol).  A
 * plan holds, for every layer, the filter plaintexts and HomShare masks
 * (prepared at creation, i.e. setup) and its intermediate ciphertext buffers,
 * and records the whole online path of every layer (the one-layer protocol
 * of Fig. 2 with HomRec) as one CUDA graph in which independent layers and the
 * input-independent steps run concurrently.  The masks and encryption seeds
 * are fixed at creation; a protocol run must not reuse them, so a new plan
 * (or new seeds) is needed per inference. */
typedef struct {
    const fdsc_params* params;  /* created for this layer's (n, p), max_T >= T */
    fdsc_layer layer;           /* g_c = 0: the plan chooses the packing       */
    uint32_t fh, fw;
    const int8_t* w;            /* device [Co][Ci][fh][fw]                     */
    const uint64_t* t_hat;      /* device [n]: the client's key                */
    uint64_t enc_seed, mask_seed;
    const uint32_t* xA;         /* device [B][Ci][H][W]: Alice's share         */
    const uint32_t* xB;         /* device [B][Ci][H][W]: Bob's share (HomRec)  */
    uint32_t* yA;               /* device [B][Co][H][W]: Alice's output share  */
    uint32_t* yB;               /* device [B][Co][H][W]: Bob's output share    */
    uint32_t* pA;               /* NULL, or device [B][Co][H/2][W/2]: yA after
                                   fdsc_pool2x2_sum (H, W even)                */
    uint32_t* pB;               /* NULL, or the same for yB                    */
    uint32_t flood_bits;        /* HomShare noise flooding (0: none), as in
                                   fdsc_mask_prepare_flooded                   */
    uint32_t pad0;
} fdsc_plan_layer;

typedef struct {
    uint32_t g_c, g_b;          /* packing used                                */
    uint32_t homconv_variant;   /* as in fdsc_set_homconv_variant, or 7: the
                                   tensor-core kernel (fdsc_homconv_tc)        */
    uint32_t fused;             /* 1: fused online kernels; 0: step by step    */
    uint32_t candidates;        /* candidates the tuner timed (0: not tuned)   */
    uint32_t pad0;
    double tuned_step_us;       /* the chosen candidate's median step time     */
} fdsc_plan_layer_info;

enum {
    FDSC_PLAN_TUNE = 1,         /* time packings x HomConv variants (the tensor-core
                                   kernel among them where T <= 128), keep the fastest */
    FDSC_PLAN_CHAIN = 2,        /* layer i starts once layer i-1 (and its pooling) has
                                   finished, so it may read the shares layer i-1 wrote:
                                   a network's convolution stack (Fig. 2's layer to layer steps,
                                   with the activation protocol left to the caller) */
    FDSC_PLAN_TENSOR = 4        /* untuned layers with T <= 128 use the tensor-core
                                   HomConv (the words do not change) */
};

typedef struct fdsc_plan fdsc_plan;

/* Builds the plan on the current device: allocates its buffers, prepares
 * filters and masks, runs every layer once and records the graph; with
 * FDSC_PLAN_TUNE it first times every candidate packing x HomConv variant.
 * All of this runs on the plan's own streams and has finished on return
 * (`stream` is reserved).  Layers with H or W outside [8, 512] use
 * the step-by-step kernels. */
int fdsc_plan_create(const fdsc_plan_layer* layers, uint32_t count, uint32_t flags, void* stream, fdsc_plan** out);
/* One launch of the recorded graph: every layer's online path. */
int fdsc_plan_launch(fdsc_plan* plan, void* stream);
/* Layer i's packing (g_c, g_b), HomConv variant (7: tensor cores), whether
 * it runs the fused kernels, and the tuner's candidates and best time;
 * FDSC_ERR_ARG if i >= count. */
int fdsc_plan_layer_info_get(const fdsc_plan* plan, uint32_t i, fdsc_plan_layer_info* out);
/* Frees the plan's buffers, streams, events and graph; its launches must have
 * completed (synchronize their stream first). */
int fdsc_plan_destroy(fdsc_plan* plan);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of single-image requests                  */
/* ---------------------------------------------------------------------- */
/* Not in the paper.  A host thread inside the library admits requests (one
 * image of one registered layer type, from one client) into batches while
 * earlier batches are still on the GPU: each lane is a stream with its own
 * buffers, a batch holds up to lane_capacity requests of one type, and a
 * batch is launched only when the bytes of all requests in flight stay within
 * hbm_budget_bytes.  The budget also sizes the lanes' device buffers (the
 * memory requests in flight occupy): fdsc_server_start gives every lane room
 * for min(max_batch, budget / (lanes x the largest request)) requests, with
 * fewer lanes when not one request per lane fits, so the lanes never hold
 * more device memory than the budget.  Filter plaintexts (per type) and the
 * callers' key pools are resident state outside it.  Every request carries its own key and seeds and is
 * computed with the multi-client kernels, so its shares are bit-identical
 * whether it runs alone or batched with others. */
typedef struct {
    uint64_t hbm_budget_bytes;  /* device bytes requests in flight may use     */
    uint32_t max_batch;         /* requests per launch (>= 1)                  */
    uint32_t lanes;             /* batches in flight at once (>= 1)            */
} fdsc_server_config;

typedef struct {
    uint32_t type;              /* from fdsc_server_add_type                   */
    uint32_t key;               /* index into the type's key pool              */
    uint64_t enc_seed, mask_seed;
    const uint32_t* xA;         /* HOST [Ci][H][W]; valid until the request is done */
    const uint32_t* xB;         /* HOST [Ci][H][W]                              */
    uint32_t* yA;               /* HOST [Co][H][W], written when done          */
    uint32_t* yB;               /* HOST [Co][H][W]                              */
} fdsc_request;

typedef struct {
    uint64_t submitted, completed, batches;
    uint64_t peak_inflight_bytes;
    double mean_batch;
    double p50_us, p99_us, mean_us, max_us; /* submit-to-completion latency   */
    uint64_t tensor_batches;    /* batches whose HomConv ran on the tensor cores
                                   (batches of 4 or more requests, when the
                                   layer admits fdsc_homconv_tc)               */
    uint64_t reserved_bytes;    /* device bytes of the lanes' request buffers
                                   (at most hbm_budget_bytes)                  */
    uint32_t lanes;             /* lanes made (fewer than asked when the budget
                                   holds less than one request per lane)       */
    uint32_t lane_capacity;     /* requests one lane's buffers hold: at most
                                   max_batch, and budget / (lanes x the largest
                                   request's bytes)                            */
} fdsc_server_stats;

typedef struct fdsc_server fdsc_server;

/* A server for cfg on the current device (max_batch >= 1 and lanes >= 1,
 * FDSC_ERR_ARG otherwise); device memory is taken at fdsc_server_start. */
int fdsc_server_create(const fdsc_server_config* cfg, fdsc_server** out);
/* Registers a layer type (B is ignored; fused shapes with H W <= S and one
 * slot set per ciphertext, d = 1, since a batch packs one client per image
 * group): prepares its filter plaintexts from device weights w and keeps
 * a pointer to its key pool (device [nkeys][n]). */
int fdsc_server_add_type(fdsc_server* s, const fdsc_params* P, const fdsc_layer* L, const int8_t* w, uint32_t fh,
                         uint32_t fw, const uint64_t* keys, uint32_t nkeys, uint32_t* type_id);
/* Allocates the lanes' buffers within the budget (see above), records every
 * lane's batch of every type and size (1 .. lane_capacity) as a CUDA graph
 * (after one run per type on zero inputs), and starts the scheduling thread.
 * Types must all be added before; FDSC_ERR_BUDGET if the budget holds no
 * request, FDSC_ERR_CUDA if a recording fails. */
int fdsc_server_start(fdsc_server* s);
/* Queues a request (thread-safe); FDSC_ERR_BUDGET if it can never fit.  The
 * latency statistics are kept in a fixed histogram (0.45 % bins between 1 us
 * and 100 s): the server's memory does not grow with the requests served. */
int fdsc_server_submit(fdsc_server* s, const fdsc_request* r, uint64_t* ticket);
/* Waits at most timeout_ms for a ticket; FDSC_ERR_TIMEOUT if not done. */
int fdsc_server_wait(fdsc_server* s, uint64_t ticket, uint32_t timeout_ms, double* latency_us);
/* Counters, and latencies from submission until both output shares are in
 * the caller's buffers, over the requests completed so far; returns the
 * server's first failure, if any. */
int fdsc_server_stats_get(fdsc_server* s, fdsc_server_stats* out);
/* Stops the thread after the batches in flight finish and frees everything. */
int fdsc_server_destroy(fdsc_server* s);

/* ---------------------------------------------------------------------- */
/* One layer without any device allocation                                 */
/* ---------------------------------------------------------------------- */
/* The paper has no counterpart: this serves callers that cannot let a
 * library allocate device memory -- applications whose device memory is
 * entirely reserved by their own pooling allocator, and latency-critical
 * request threads that must never enter the CUDA allocator (its calls can
 * block on device-wide synchronisation).
 *
 * Runs the fused online path of one layer -- the same kernels as
 * fdsc_encrypt_constants(t_hat, enc_seed), fdsc_encode_share(xA),
 * fdsc_encode_share(xB), fdsc_homconv_sum(P_hat, M_hat),
 * fdsc_decrypt_share(t_hat) -> yA and fdsc_intt2d(sB_hat) -> yB -- and
 * writes exactly their words, but keeps the intermediate ciphertexts in one
 * fixed device array of FDSC_NOALLOC_SCRATCH_BYTES compiled into the library
 * (every device that loads the library holds it until the process exits).  It
 * calls no allocator.  Inputs and outputs are the caller's device buffers,
 * with the shapes of those calls (t_hat [n], P_hat [Co][T][n / d], M_hat
 * [GB][Co][n], sB_hat, yA, yB [B][Co][H][W], xA, xB [B][Ci][H][W]).
 *
 *  - The first call in a CUDA context (per device, and again after a device
 *    reset) looks up the array's device address; make that first call before
 *    any stream capture.
 *  - Layers whose intermediate ciphertexts need more than the array
 *    (8 (2 n_in + 2 n_in + 2 n_out) n bytes, each part rounded up to 256)
 *    are rejected with FDSC_ERR_UNSUPPORTED; so are shapes the fused kernels do
 *    not take (H W > S, H or W outside [8, 512]).
 *  - Every call uses the same array and leaves its last contents there; each
 *    call writes every word before reading it, so nothing needs clearing.
 *    Calls whose work overlaps on the GPU (other streams, other threads) race
 *    on the array: serialise them. */
#define FDSC_NOALLOC_SCRATCH_BYTES (8u << 20)
int fdsc_layer_online_noalloc(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat, uint64_t enc_seed,
                              const uint64_t* P_hat, const uint64_t* M_hat, const uint32_t* sB_hat, const uint32_t* xA,
                              const uint32_t* xB, uint32_t* yA, uint32_t* yB, void* stream);

/* ---------------------------------------------------------------------- */
/* Tuning                                                                  */
/* ---------------------------------------------------------------------- */
/* Selects the HomConv kernel variant for later fdsc_homconv calls in this
 * process (all variants give identical results): 0 automatic (default),
 * 1 limb-column accumulation with one image group per thread, 2 the same
 * with two image groups per thread, 3 carry-chained 128-bit accumulation,
 * 4 input tile staged in shared memory with carry-chained accumulation,
 * 5 staged tile with limb columns, 6 staged tile with lazy 32-bit-limb
 * columns, 8 / 9 staged tile with Karatsuba limb columns and one / two image
 * groups per CTA, 10 staged tile with two evaluation indices per lane
 * (T a multiple of 4 and at most 128, else 4), 11 / 12 the same with the
 * filter streamed through a shared-memory ring of 16 / 8 terms (T <= 64,
 * else 10), 13 / 14 variant 12 with 2 / 4 partial sums per output word,
 * 15 variant 12 reading its first filter terms before it waits for the
 * kernel before it: with launch overlap on (fdsc_set_launch_overlap) that
 * kernel must not write P_hat.  A variant that does not fit a layer falls
 * back as stated.  7 and values outside 0-15: FDSC_ERR_ARG (the tensor-core
 * kernel is fdsc_homconv_tc).  Not synchronised with concurrent calls. */
int fdsc_set_homconv_variant(int variant);

/* Launch overlap for the online kernels (on = 1; off = 0, the default):
 * each online kernel (NTT2D/INTT2D, encryption, HomRec, HomConv, masks,
 * decryption, and the fused kernels) is launched with programmatic stream
 * serialisation, so it may start while the kernel before it in the stream
 * finishes.  It stages the params' twiddle tables, and the encryption
 * constants draw and transform their error polynomial from the seed, before
 * it waits for that kernel; it touches caller memory only after the wait.
 * Results are identical either way.  Off by default: measured on GB300, the
 * early start saved under 1 us per layer step and made graph replays of
 * consecutive steps slower.  Returns the previous setting.  Applies to
 * launches issued after the call, process-wide. */
int fdsc_set_launch_overlap(int on);

/* The fused decryption of a layer whose output ciphertexts fill less than half
 * the SMs (one image) splits every ciphertext over a cluster of two CTAs, one
 * coefficient parity each (on = 1, the default): a lower latency for that
 * image, for about 45 % more instructions in all.  Off (0): one CTA per
 * ciphertext, the better choice when consecutive layers overlap on the GPU
 * and the SMs, not one layer's latency, are the bound.  The words are the same
 * either way.  Returns the previous setting; process-wide, for launches issued
 * after the call. */
int fdsc_set_decrypt_pair(int on);

/* Measured throughput of the exact arithmetic primitives on the current
 * device (the ALU side of the roofline): which = 0, the 60 x 60 -> 128-bit
 * multiply-accumulate of HomConv; 1, the 64-bit Shoup multiplication mod q
 * of the NTT_q butterflies; 2, the 32-bit Shoup multiplication mod p of the
 * NTT2D and slot transforms.  Register-resident, loop-carried chains on every
 * SM; returns operations per second and per clock per SM (SM count and clock
 * from the device attributes).  Synchronous; a few milliseconds. */
int fdsc_calibrate(const fdsc_params* P, int which, double* ops_per_s, double* ops_per_clk_sm);

#ifdef __cplusplus
}
#endif
#endif /* FDSC_H */
