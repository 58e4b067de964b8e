// modarith.cuh -- device arithmetic of libfdsc: exact modular products mod q
// (60-bit) and mod p (< 2^20), the counter-based sampler, and the
// block-cooperative transforms that run on shared memory.
//
// Products by a fixed operand w use Shoup's precomputed quotient
// w' = floor(w 2^k / m): for any a < 2^k, a w - floor(a w' / 2^k) m lies in
// [0, 2m) and is computed exactly in wrapping k-bit arithmetic (V. Shoup, NTL;
// D. Harvey, "Faster arithmetic for number-theoretic transforms", 2014).
// Butterflies keep values lazily in [0, 4m) (Harvey), which needs 4q < 2^64.
#pragma once
#include <utility>

#include "fdsc_internal.h"

// ------------------------------------------------------------------ mod q
__device__ __forceinline__ u64 shoup_mul(u64 a, u64 w, u64 ws, u64 q) {
    return a * w - __umul64hi(a, ws) * q;  // [0, 2q)
}

// (hi 2^64 + lo) mod q for any hi, lo < 2^64: hi 2^64 = hi (2^64 mod q) and
// lo = lo * 1, each by a Shoup product, then two conditional subtractions.
__device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const DevParams& P) {
    u64 r = shoup_mul(hi, P.r64, P.r64_s, P.q) + (lo - __umul64hi(lo, P.one_s) * P.q);
    r = r >= P.twoq ? r - P.twoq : r;
    return r >= P.q ? r - P.q : r;
}

// (a b + c) mod q for a, b, c in [0, q), q in (2^59, 2^60): one Barrett
// reduction (P. Barrett, CRYPTO '86) of the 121-bit x = a b + c.  With
// x' = floor(x / 2^58) < 2^63 and mu = floor(2^122 / q), the estimate
// floor(x' mu / 2^64) lies between x/q - 1.75 and x/q, so it is floor(x/q)
// or one less, and x minus it times q, taken mod 2^64, is in [0, 2q).
__device__ __forceinline__ u64 muladd_q(u64 a, u64 b, u64 c, const DevParams& P) {
    u64 lo = a * b, hi = __umul64hi(a, b);
    lo += c;
    hi += lo < c;
    const u64 est = __umul64hi((hi << 6) | (lo >> 58), P.mu);
    const u64 r = lo - est * P.q;
    return r >= P.q ? r - P.q : r;
}
// Decryption's rounding, round(p v / q) mod p = floor((2 p v + q) / (2 q))
// mod p for v in [0, q): z = floor(v floor(p 2^64 / q) / 2^64) is
// floor(p v / q) or one less, so the remainder p v - z q, taken mod 2^64,
// lies in [0, 2q); one conditional step makes it p v mod q, and the value
// rounds up when twice that remainder passes q (q is odd: no ties).
__device__ __forceinline__ u32 round_pq(u64 v, const DevParams& P) {
    u64 z = __umul64hi(v, P.round_k);
    u64 rem = (u64)P.p * v - z * P.q;
    if (rem >= P.q) {
        rem -= P.q;
        z++;
    }
    z += 2 * rem >= P.q;
    return (u32)(z >= P.p ? z - P.p : z);
}
// The same value from the same estimate z, stepped up while
// 2 q (z + 1) <= 2 p v + q in 128-bit arithmetic (at most twice).  Slower
// alone, but the fused decryptions of one ciphertext per CTA or CTA pair
// keep it: in the pipelined one-image step their CTAs share SMs with the
// producers that bound the step, and with the remainder form there the step
// took 18.6 instead of 18.2 us (same GPU, alternating runs); the pair kernel
// then compiled to 64 registers with spills and took 15.7 instead of 13.7 us.
__device__ __forceinline__ u32 round_pq_wide(u64 v, const DevParams& P) {
    u64 z = __umul64hi(v, P.round_k);
    const unsigned __int128 num = (unsigned __int128)(2ull * P.p) * v + P.q;
    const unsigned __int128 q2 = (unsigned __int128)2 * P.q;
#pragma unroll
    for (int it = 0; it < 3; it++)
        if (q2 * (z + 1) <= num) z++;
    return (u32)(z >= P.p ? z - P.p : z);
}
__device__ __forceinline__ u64 addmod_q(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 submod_q(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// ------------------------------------------------------------------ mod p
__device__ __forceinline__ u32 shoup_mul32(u32 a, u32 w, u32 ws, u32 p) {
    return a * w - __umulhi(a, ws) * p;  // [0, 2p)
}
__device__ __forceinline__ u32 addmod_p(u32 a, u32 b, u32 p) {
    u32 s = a + b;
    return s >= p ? s - p : s;
}
__device__ __forceinline__ u32 submod_p(u32 a, u32 b, u32 p) { return a >= b ? a - b : a + p - b; }

// ------------------------------------------------------------------ sampler
// SplitMix64 output function (Steele, Lea & Flood 2014) used as a counter
// generator: stream key = out(seed + domain gamma); value idx = out(key +
// (idx + 1) gamma).
#define FDSC_GAMMA 0x9E3779B97F4A7C15ull
enum { DOM_T = 1, DOM_A = 2, DOM_E = 3, DOM_MASK = 4, DOM_MASK_SPLIT = 5, DOM_FLOOD = 6 };

__device__ __forceinline__ u64 splitmix_out(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ u64 stream_key(u64 seed, u64 dom) { return splitmix_out(seed + dom * FDSC_GAMMA); }
__device__ __forceinline__ u64 stream_at(u64 key, u64 idx) { return splitmix_out(key + (idx + 1) * FDSC_GAMMA); }

// floor((r1 2^64 + r2) q / 2^128): the top word of r1 q + hi(r2 q).
__device__ __forceinline__ u64 uniform_q(u64 r1, u64 r2, u64 q) {
    u64 lo = r1 * q, hi = __umul64hi(r1, q);
    u64 s = lo + __umul64hi(r2, q);
    return hi + (s < lo);
}
__device__ __forceinline__ u32 uniform_p(u64 r, u32 p) { return (u32)__umul64hi(r, (u64)p); }

// Discrete Gaussian from one word: sign bit 63, magnitude = number of table
// entries the low 63 bits reach.
__device__ __forceinline__ int gauss_sample(u64 r, const u64* cdt) {
    u64 u = r & 0x7FFFFFFFFFFFFFFFull;
    int a = 0;
#pragma unroll
    for (int k = 0; k < 19; k++) a += (u >= cdt[k]);
    return (r >> 63) ? -a : a;
}

// ------------------------------------------------------------------ transforms
// All run with the whole CTA on a shared-memory array and end synchronised.

// Negacyclic NTT mod q, natural order in, bit-reversed evaluation order out
// (Cooley-Tukey butterflies with twiddles psi^brv(m+i)).  In: [0, 4q); out [0, q).
__device__ __forceinline__ void ntt_q_fwd(u64* a, const DevParams& P) {
    const u32 half = P.n >> 1;
    u32 logt = P.logn - 1;
    for (u32 m = 1; m < P.n; m <<= 1, logt--) {
        const u32 t = 1u << logt;
        for (u32 b = threadIdx.x; b < half; b += blockDim.x) {
            const u32 i = b >> logt, j = (i << (logt + 1)) + (b & (t - 1));
            const u64 w = P.qfw[m + i], ws = P.qfw_s[m + i];
            u64 x = a[j];
            x = x >= P.twoq ? x - P.twoq : x;
            const u64 y = shoup_mul(a[j + t], w, ws, P.q);
            a[j] = x + y;
            a[j + t] = x - y + P.twoq;
        }
        __syncthreads();
    }
    for (u32 j = threadIdx.x; j < P.n; j += blockDim.x) {
        u64 x = a[j];
        x = x >= P.twoq ? x - P.twoq : x;
        a[j] = x >= P.q ? x - P.q : x;
    }
    __syncthreads();
}

// Inverse: bit-reversed in, natural out, Gentleman-Sande butterflies with
// psi^-brv(h+i), then the factor n^-1.  In: [0, 2q); out [0, q).
__device__ __forceinline__ void ntt_q_inv(u64* a, const DevParams& P) {
    const u32 half = P.n >> 1;
    u32 logt = 0;
    for (u32 h = half; h >= 1; h >>= 1, logt++) {
        const u32 t = 1u << logt;
        for (u32 b = threadIdx.x; b < half; b += blockDim.x) {
            const u32 i = b >> logt, j = (i << (logt + 1)) + (b & (t - 1));
            const u64 w = P.qinv[h + i], ws = P.qinv_s[h + i];
            const u64 x = a[j], y = a[j + t];
            u64 s = x + y;
            a[j] = s >= P.twoq ? s - P.twoq : s;
            a[j + t] = shoup_mul(x - y + P.twoq, w, ws, P.q);
        }
        __syncthreads();
    }
    for (u32 j = threadIdx.x; j < P.n; j += blockDim.x) {
        u64 x = shoup_mul(a[j], P.ninv, P.ninv_s, P.q);
        a[j] = x >= P.q ? x - P.q : x;
    }
    __syncthreads();
}

// Slot decode on `cnt` consecutive length-S sets: negacyclic NTT mod p,
// natural in, bit-reversed out.  In [0, p); out [0, p).
__device__ __forceinline__ void ntt_p_fwd(u32* a, u32 cnt, const DevParams& P) {
    const u32 half = P.S >> 1, p = P.p;
    u32 logt = P.logS - 1;
    for (u32 m = 1; m < P.S; m <<= 1, logt--) {
        const u32 t = 1u << logt;
        for (u32 g = threadIdx.x; g < half * cnt; g += blockDim.x) {
            const u32 set = g >> (P.logS - 1), b = g & (half - 1);
            const u32 i = b >> logt, j = set * P.S + (i << (logt + 1)) + (b & (t - 1));
            u32 x = a[j], y = shoup_mul32(a[j + t], P.pfw[m + i], P.pfw_s[m + i], p);
            y = y >= p ? y - p : y;
            a[j] = addmod_p(x, y, p);
            a[j + t] = submod_p(x, y, p);
        }
        __syncthreads();
    }
}

// Slot encode: the inverse (bit-reversed in, natural out, times S^-1).
__device__ __forceinline__ void ntt_p_inv(u32* a, u32 cnt, const DevParams& P) {
    const u32 half = P.S >> 1, p = P.p;
    u32 logt = 0;
    for (u32 h = half; h >= 1; h >>= 1, logt++) {
        const u32 t = 1u << logt;
        for (u32 g = threadIdx.x; g < half * cnt; g += blockDim.x) {
            const u32 set = g >> (P.logS - 1), b = g & (half - 1);
            const u32 i = b >> logt, j = set * P.S + (i << (logt + 1)) + (b & (t - 1));
            const u32 x = a[j], y = a[j + t];
            a[j] = addmod_p(x, y, p);
            u32 d = shoup_mul32(submod_p(x, y, p), P.pinv[h + i], P.pinv_s[h + i], p);
            a[j + t] = d >= p ? d - p : d;
        }
        __syncthreads();
    }
    for (u32 j = threadIdx.x; j < P.S * cnt; j += blockDim.x) {
        u32 x = shoup_mul32(a[j], P.Sinv, P.Sinv_s, p);
        a[j] = x >= p ? x - p : x;
    }
    __syncthreads();
}

// Cyclic 2D NTT of one H x W plane held in shared memory in bit-reversed
// order along both axes (x[brv(i)][brv(j)]); leaves the natural-order
// spectrum.  Radix-2 decimation in time along rows, then columns, with
// twiddles w_L^k = w_lmax^(k lmax / L).  `inverse` selects w^-1 (no scaling).
__device__ __forceinline__ void ntt2d_plane(u32* x, u32 logH, u32 logW, bool inverse, const DevParams& P) {
    const u32 p = P.p, H = 1u << logH, W = 1u << logW, nb = (H * W) >> 1;
    const u32* tw = inverse ? P.w2di : P.w2d;
    const u32* tws = inverse ? P.w2di_s : P.w2d_s;
    // rows
    for (u32 ls = 1; ls <= logW; ls++) {
        const u32 hl = 1u << (ls - 1), shift = P.loglmax - ls;
        for (u32 b = threadIdx.x; b < nb; b += blockDim.x) {
            const u32 row = b >> (logW - 1), k = b & ((W >> 1) - 1);
            const u32 j = k & (hl - 1), idx = (row << logW) + ((k >> (ls - 1)) << ls) + j;
            const u32 tk = j << shift;
            u32 u = x[idx], v = shoup_mul32(x[idx + hl], tw[tk], tws[tk], p);
            v = v >= p ? v - p : v;
            x[idx] = addmod_p(u, v, p);
            x[idx + hl] = submod_p(u, v, p);
        }
        __syncthreads();
    }
    // columns
    for (u32 ls = 1; ls <= logH; ls++) {
        const u32 hl = 1u << (ls - 1), shift = P.loglmax - ls;
        for (u32 b = threadIdx.x; b < nb; b += blockDim.x) {
            const u32 col = b & (W - 1), k = b >> logW;
            const u32 j = k & (hl - 1), r = ((k >> (ls - 1)) << ls) + j;
            const u32 idx = (r << logW) + col, tk = j << shift;
            u32 u = x[idx], v = shoup_mul32(x[idx + (hl << logW)], tw[tk], tws[tk], p);
            v = v >= p ? v - p : v;
            x[idx] = addmod_p(u, v, p);
            x[idx + (hl << logW)] = submod_p(u, v, p);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ u32 brv_bits(u32 x, u32 bits) { return bits ? __brev(x) >> (32 - bits) : 0; }

// ------------------------------------------------------------------ radix-8 register passes
// A length-L transform (L = 2^logL >= 8) is run as passes of up to three
// butterfly stages: in each pass a thread holds 8 elements whose indices
// differ in one 3-bit window [wlo, wlo+3), does the stages of that window in
// registers, and exchanges through shared memory (one barrier per pass
// instead of one per stage).  Thread tl of a vector owns the elements
// win_index(tl, r, wlo), r < 8; L/8 threads serve one vector.
__device__ __forceinline__ u32 win_index(u32 tl, u32 r, u32 wlo) {
    return ((tl >> wlo) << (wlo + 3)) | (r << wlo) | (tl & ((1u << wlo) - 1u));
}

// Harvey butterflies mod q.  CT: x in [0,4q), y < 2^64 -> both in [0,4q).
__device__ __forceinline__ void bfly_ct_q(u64& x, u64& y, u64 w, u64 ws, const DevParams& P) {
    const u64 a = x >= P.twoq ? x - P.twoq : x;
    const u64 t = shoup_mul(y, w, ws, P.q);
    x = a + t;
    y = a - t + P.twoq;
}
// GS: x, y in [0,2q) -> both in [0,2q).
__device__ __forceinline__ void bfly_gs_q(u64& x, u64& y, u64 w, u64 ws, const DevParams& P) {
    const u64 s = x + y;
    const u64 d = shoup_mul(x - y + P.twoq, w, ws, P.q);
    x = s >= P.twoq ? s - P.twoq : s;
    y = d;
}
__device__ __forceinline__ void bfly_ct_p(u32& x, u32& y, u32 w, u32 ws, u32 p) {
    u32 t = shoup_mul32(y, w, ws, p);
    t = t >= p ? t - p : t;
    const u32 a = x;
    x = addmod_p(a, t, p);
    y = submod_p(a, t, p);
}
__device__ __forceinline__ void bfly_gs_p(u32& x, u32& y, u32 w, u32 ws, u32 p) {
    const u32 a = x, b = y;
    x = addmod_p(a, b, p);
    u32 d = shoup_mul32(submod_p(a, b, p), w, ws, p);
    y = d >= p ? d - p : d;
}

// Stage with bit b = wlo + RB on the 8 registers; twiddle of the pair whose
// lower index is i: table[(L + i) >> (b + 1)] (psi^brv for CT, psi^-brv for GS).
template <int RB, bool CT, typename T>
__device__ __forceinline__ void r8_stage(T (&x)[8], u32 tl, u32 wlo, u32 L, const T* tw, const T* tws,
                                         const DevParams& P) {
    const u32 b = wlo + RB;
#pragma unroll
    for (int r = 0; r < 8; r++) {
        if (r & (1 << RB)) continue;
        const u32 k = (L + win_index(tl, r, wlo)) >> (b + 1);
        const T w = tw[k], ws = tws[k];  // generic loads: tables may live in shared or global memory
        if constexpr (sizeof(T) == 8) {
            if (CT) bfly_ct_q(x[r], x[r | (1 << RB)], w, ws, P);
            else bfly_gs_q(x[r], x[r | (1 << RB)], w, ws, P);
        } else {
            if (CT) bfly_ct_p(x[r], x[r | (1 << RB)], w, ws, P.p);
            else bfly_gs_p(x[r], x[r | (1 << RB)], w, ws, P.p);
        }
    }
}

// Forward negacyclic transform of `cnt` contiguous length-L vectors in a:
// natural order in, bit-reversed evaluation order out.  mod q: in [0,4q),
// out [0,q).  mod p: in and out [0,p).  Every thread of the CTA must call it.
template <typename T>
__device__ __forceinline__ void ntt_fwd_r8(T* a, u32 logL, u32 cnt, const T* tw, const T* tws, const DevParams& P) {
    const u32 L = 1u << logL, lper = logL - 3;
    const bool active = threadIdx.x < (cnt << lper);
    const u32 vec = threadIdx.x >> lper, tl = threadIdx.x & ((1u << lper) - 1u);
    T* v = a + (u64)vec * L;
    for (int hi = (int)logL - 1; hi >= 0; hi -= 3) {
        const u32 wlo = hi >= 2 ? (u32)hi - 2 : 0u;
        const int lo = hi - 2 > 0 ? hi - 2 : 0;  // lowest stage bit of this pass
        if (active) {
            T x[8];
#pragma unroll
            for (int r = 0; r < 8; r++) x[r] = v[win_index(tl, r, wlo)];
            if ((int)wlo + 2 <= hi && (int)wlo + 2 >= lo) r8_stage<2, true>(x, tl, wlo, L, tw, tws, P);
            if ((int)wlo + 1 <= hi && (int)wlo + 1 >= lo) r8_stage<1, true>(x, tl, wlo, L, tw, tws, P);
            if ((int)wlo <= hi && (int)wlo >= lo) r8_stage<0, true>(x, tl, wlo, L, tw, tws, P);
            if (hi < 3) {  // last pass: canonical residues
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    if constexpr (sizeof(T) == 8) {
                        T y = x[r] >= P.twoq ? x[r] - P.twoq : x[r];
                        x[r] = y >= P.q ? y - P.q : y;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 8; r++) v[win_index(tl, r, wlo)] = x[r];
        }
        __syncthreads();
    }
}

// Inverse: bit-reversed in, natural out, times L^-1 (inv, inv_s).
template <typename T>
__device__ __forceinline__ void ntt_inv_r8(T* a, u32 logL, u32 cnt, const T* tw, const T* tws, T inv, T inv_s,
                                           const DevParams& P) {
    const u32 L = 1u << logL, lper = logL - 3;
    const bool active = threadIdx.x < (cnt << lper);
    const u32 vec = threadIdx.x >> lper, tl = threadIdx.x & ((1u << lper) - 1u);
    T* v = a + (u64)vec * L;
    for (u32 lo = 0; lo < logL; lo += 3) {
        const u32 top = lo + 3 < logL ? lo + 3 : logL;  // stage bits [lo, top)
        const u32 wlo = lo + 3 <= logL ? lo : logL - 3;
        if (active) {
            T x[8];
#pragma unroll
            for (int r = 0; r < 8; r++) x[r] = v[win_index(tl, r, wlo)];
            if (wlo >= lo && wlo < top) r8_stage<0, false>(x, tl, wlo, L, tw, tws, P);
            if (wlo + 1 >= lo && wlo + 1 < top) r8_stage<1, false>(x, tl, wlo, L, tw, tws, P);
            if (wlo + 2 >= lo && wlo + 2 < top) r8_stage<2, false>(x, tl, wlo, L, tw, tws, P);
            if (top == logL) {
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    if constexpr (sizeof(T) == 8) {
                        T y = shoup_mul(x[r], inv, inv_s, P.q);
                        x[r] = y >= P.q ? y - P.q : y;
                    } else {
                        T y = shoup_mul32(x[r], inv, inv_s, P.p);
                        x[r] = y >= P.p ? y - P.p : y;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 8; r++) v[win_index(tl, r, wlo)] = x[r];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void ntt_q_fwd8(u64* a, const DevParams& P) { ntt_fwd_r8<u64>(a, P.logn, 1, P.qfw, P.qfw_s, P); }
__device__ __forceinline__ void ntt_q_inv8(u64* a, const DevParams& P) {
    ntt_inv_r8<u64>(a, P.logn, 1, P.qinv, P.qinv_s, P.ninv, P.ninv_s, P);
}
__device__ __forceinline__ void ntt_p_fwd8(u32* a, u32 cnt, const DevParams& P) {
    ntt_fwd_r8<u32>(a, P.logS, cnt, P.pfw, P.pfw_s, P);
}
__device__ __forceinline__ void ntt_p_inv8(u32* a, u32 cnt, const DevParams& P) {
    ntt_inv_r8<u32>(a, P.logS, cnt, P.pinv, P.pinv_s, P.Sinv, P.Sinv_s, P);
}

// Cyclic decimation-in-frequency transform mod p of the lines of an H x W
// plane in shared memory (rows: lines H, length W, stride 1; columns: lines
// W, length H, stride W): natural order in, bit-reversed order out; twiddle
// of stage t = 2^b at in-line index i: w_lmax^((i mod t) lmax / (2t)).
// Needs L >= 8 and HW / 8 threads.
__device__ __forceinline__ void dif_lines_r8(u32* pl, u32 logL, u32 lines_log, bool rows, u32 logW, const u32* tw,
                                             const u32* tws, const DevParams& P) {
    const u32 lper = logL - 3;
    const bool active = threadIdx.x < (1u << (lines_log + lper));
    u32 line, tl;
    if (rows) {
        line = threadIdx.x >> lper;
        tl = threadIdx.x & ((1u << lper) - 1u);
    } else {  // consecutive threads on consecutive columns
        line = threadIdx.x & ((1u << lines_log) - 1u);
        tl = threadIdx.x >> lines_log;
    }
    const u32 p = P.p;
    for (int hi = (int)logL - 1; hi >= 0; hi -= 3) {
        const u32 wlo = hi >= 2 ? (u32)hi - 2 : 0u;
        const int lo = hi - 2 > 0 ? hi - 2 : 0;
        if (active) {
            u32 off[8], x[8];
#pragma unroll
            for (int r = 0; r < 8; r++) {
                const u32 i = win_index(tl, r, wlo);
                off[r] = rows ? (line << logW) + i : (i << logW) + line;
                x[r] = pl[off[r]];
            }
#pragma unroll
            for (int RB = 2; RB >= 0; RB--) {
                const int b = (int)wlo + RB;
                if (b > hi || b < lo) continue;
                const u32 t = 1u << b, shift = P.loglmax - 1 - b;
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    if (r & (1 << RB)) continue;
                    const u32 i = win_index(tl, r, wlo);
                    const u32 k = (i & (t - 1)) << shift;
                    const u32 u = x[r], v = x[r | (1 << RB)];
                    x[r] = addmod_p(u, v, p);
                    u32 d = shoup_mul32(submod_p(u, v, p), __ldg(tw + k), __ldg(tws + k), p);
                    x[r | (1 << RB)] = d >= p ? d - p : d;
                }
            }
#pragma unroll
            for (int r = 0; r < 8; r++) pl[off[r]] = x[r];
        }
        __syncthreads();
    }
}

// NTT2D (or its unscaled inverse) of a natural-order plane in shared memory,
// leaving X[k1][k2] at pl[brv(k1) W + brv(k2)].  H, W >= 8; HW/8 threads.
__device__ __forceinline__ void ntt2d_plane_dif(u32* pl, u32 logH, u32 logW, bool inverse, const DevParams& P) {
    const u32* tw = inverse ? P.w2di : P.w2d;
    const u32* tws = inverse ? P.w2di_s : P.w2d_s;
    dif_lines_r8(pl, logW, logH, true, logW, tw, tws, P);
    dif_lines_r8(pl, logH, logW, false, logW, tw, tws, P);
}

// ------------------------------------------------------------------ staging and multi-plane 2D transforms
// Asynchronous global -> shared copy of `bytes` (a multiple of 16, both
// addresses 16-byte aligned) by the whole CTA; stage_wait() completes every
// copy this thread issued and synchronises the CTA.
__device__ __forceinline__ void stage_async(void* smem, const void* g, u32 bytes) {
    const u32 base = (u32)__cvta_generic_to_shared(smem);
    const char* src = reinterpret_cast<const char*>(g);
    for (u32 o = threadIdx.x * 16; o < bytes; o += blockDim.x * 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(base + o), "l"(src + o) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void stage_wait() {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
}
// Completes every copy group but the N most recently committed ones (each
// stage_async call commits one group) and synchronises the CTA.
template <int N>
__device__ __forceinline__ void stage_wait_groups() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
    __syncthreads();
}

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation may start while the kernel before it in the stream is still
// running; griddep_wait() returns once that kernel has completed and its
// writes are visible (at once when there is none).  Every online kernel calls
// griddep_wait() before its first access to caller memory, read or write, so
// only work that depends on the params alone (twiddle tables, randomness
// from a seed argument) runs ahead.  griddep_release() lets the next kernel
// in the stream start its own launch early.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Cyclic radix-8 line transforms over `planes` stacked H x W planes in
// shared memory (plane stride HW).  Rows: planes*H lines of length W; columns:
// planes*W lines of length H.  `tw` holds w_T^k (k < T/2) for T = 2^logT >=
// the line length: stage t = 2^b uses w_{2t}^j = tw[j << (logT - 1 - b)].
//  dif: natural order in, bit-reversed out (Gentleman-Sande);
//  dit: bit-reversed in, natural order out (Cooley-Tukey).
// Needs line length >= 8 and planes * HW / 8 threads.
template <bool kDif>
__device__ __forceinline__ void lines_r8(u32* buf, u32 planes, bool rows, u32 logH, u32 logW, const u32* tw,
                                         const u32* tws, u32 logT, u32 p) {
    const u32 logL = rows ? logW : logH, lper = logL - 3;
    const u32 nlines = planes << (rows ? logH : logW);
    const bool active = threadIdx.x < (nlines << lper);
    u32 line, tl;
    if (rows) {
        line = threadIdx.x >> lper;
        tl = threadIdx.x & ((1u << lper) - 1u);
    } else {  // consecutive threads on consecutive columns: conflict-free shared accesses
        line = threadIdx.x % nlines;
        tl = threadIdx.x / nlines;
    }
    const u32 base = rows ? line << logW : ((line >> logW) << (logH + logW)) + (line & ((1u << logW) - 1u));
    const u32 stride_log = rows ? 0u : logW;
    const int npass = ((int)logL + 2) / 3;
    for (int ps = 0; ps < npass; ps++) {
        // dif: stage bits descending from logL-1; dit: ascending from 0
        int hi, lo;
        if (kDif) {
            hi = (int)logL - 1 - 3 * ps;
            lo = hi - 2 > 0 ? hi - 2 : 0;
        } else {
            lo = 3 * ps;
            hi = lo + 2 < (int)logL - 1 ? lo + 2 : (int)logL - 1;
        }
        const u32 wlo = kDif ? (hi >= 2 ? (u32)hi - 2 : 0u) : ((u32)lo + 3 <= logL ? (u32)lo : logL - 3);
        if (active) {
            u32 x[8];
#pragma unroll
            for (int r = 0; r < 8; r++) x[r] = buf[base + (win_index(tl, r, wlo) << stride_log)];
#pragma unroll
            for (int s = 0; s < 3; s++) {
                const int RB = kDif ? 2 - s : s;
                const int b = (int)wlo + RB;
                if (b > hi || b < lo) continue;
                const u32 t = 1u << b, shift = logT - 1 - b;
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    if (r & (1 << RB)) continue;
                    const u32 k = (win_index(tl, r, wlo) & (t - 1)) << shift;
                    const u32 w = tw[k], ws = tws[k];
                    const u32 u = x[r], v = x[r | (1 << RB)];
                    if (kDif) {
                        x[r] = addmod_p(u, v, p);
                        u32 d = shoup_mul32(submod_p(u, v, p), w, ws, p);
                        x[r | (1 << RB)] = d >= p ? d - p : d;
                    } else {
                        u32 m = shoup_mul32(v, w, ws, p);
                        m = m >= p ? m - p : m;
                        x[r] = addmod_p(u, m, p);
                        x[r | (1 << RB)] = submod_p(u, m, p);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 8; r++) buf[base + (win_index(tl, r, wlo) << stride_log)] = x[r];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ padded radix-8 passes
// Shared arrays of the fused kernels hold element i at padx(i): one word of
// padding every 32 keeps the strided windows of the last passes (stride 4
// and 1) from piling onto a few banks.
__device__ __forceinline__ u32 padx(u32 i) { return i + (i >> 5); }
// Words a padded array of n elements occupies (even, so that what follows
// stays 8-byte aligned).
__host__ __device__ inline u32 padded_len(u32 n) { return (n + (n >> 5) + 2) & ~1u; }

template <typename T>
struct Pair;
template <>
struct Pair<u64> {
    using type = ulonglong2;
};
template <>
struct Pair<u32> {
    using type = uint2;
};

template <bool kFwd, typename T>
__device__ __forceinline__ void bfly_pair(T& x, T& y, typename Pair<T>::type w, const DevParams& P) {
    if constexpr (sizeof(T) == 8) {
        if (kFwd) bfly_ct_q(x, y, w.x, w.y, P);
        else bfly_gs_q(x, y, w.x, w.y, P);
    } else {
        if (kFwd) bfly_ct_p(x, y, w.x, w.y, P.p);
        else bfly_gs_p(x, y, w.x, w.y, P.p);
    }
}

// `cnt` consecutive length-2^logL vectors (logL >= 3) in a padded shared
// array.  kFwd: natural in, bit-reversed evaluation order out (CT); else
// bit-reversed in, natural out, times L^-1 (GS).  mod q: forward input in
// [0, 4q), every output canonical.  Twiddles are (value, companion) pairs:
// stage bit b, pair with lower index i uses tw[(L + i) >> (b + 1)].  The pass
// loop stays a loop (compact code); per pass each thread computes one base
// and per stage one twiddle base, the rest are constant offsets.
template <bool kFwd, typename T>
__device__ __forceinline__ void ntt_r8p(T* a, u32 logL, u32 cnt, const typename Pair<T>::type* tw, T inv, T inv_s,
                                        const DevParams& P) {
    const u32 L = 1u << logL, lper = logL - 3;
    const bool active = threadIdx.x < (cnt << lper);
    const u32 tl = threadIdx.x & ((1u << lper) - 1u), voff = (threadIdx.x >> lper) << logL;
    const int npass = ((int)logL + 2) / 3;
    for (int ps = 0; ps < npass; ps++) {
        int hi, lo;
        u32 wlo;
        if (kFwd) {
            hi = (int)logL - 1 - 3 * ps;
            lo = hi - 2 > 0 ? hi - 2 : 0;
            wlo = hi >= 2 ? (u32)hi - 2 : 0u;
        } else {
            lo = 3 * ps;
            hi = lo + 2 < (int)logL - 1 ? lo + 2 : (int)logL - 1;
            wlo = (u32)lo + 3 <= logL ? (u32)lo : logL - 3;
        }
        if (active) {
            const u32 hb = (tl >> wlo) << (wlo + 3);
            const u32 base = voff + (hb | (tl & ((1u << wlo) - 1u)));
            T x[8];
#pragma unroll
            for (int r = 0; r < 8; r++) x[r] = a[padx(base + ((u32)r << wlo))];
#pragma unroll
            for (int s = 0; s < 3; s++) {
                const int RB = kFwd ? 2 - s : s;
                const int b = (int)wlo + RB;
                if (b > hi || b < lo) continue;
                const u32 tb = (L + hb) >> (b + 1);
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    if (r & (1 << RB)) continue;
                    bfly_pair<kFwd>(x[r], x[r | (1 << RB)], tw[tb + (r >> (RB + 1))], P);
                }
            }
            if (ps == npass - 1) {
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    if constexpr (sizeof(T) == 8) {
                        T y = kFwd ? x[r] : shoup_mul(x[r], inv, inv_s, P.q);
                        if (kFwd) y = y >= P.twoq ? y - P.twoq : y;
                        x[r] = y >= P.q ? y - P.q : y;
                    } else if (!kFwd) {
                        T y = shoup_mul32(x[r], inv, inv_s, P.p);
                        x[r] = y >= P.p ? y - P.p : y;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 8; r++) a[padx(base + ((u32)r << wlo))] = x[r];
        }
        __syncthreads();
    }
}

// Cyclic radix-8 line passes on stacked H x W planes in a padded shared
// array (rows: planes*H lines of W; columns: planes*W lines of H).  `tw`
// holds (w_L^k, companion) pairs for k < L/2, L the line length: stage t = 2^b
// uses tw[(i mod t) << (logL - 1 - b)].  kDif: natural in, bit-reversed out;
// else bit-reversed in, natural out.  Needs L >= 8 and planes*HW/8 threads.
template <bool kDif>
__device__ __forceinline__ void lines_r8p(u32* buf, u32 planes, bool rows, u32 logH, u32 logW, const uint2* tw,
                                          u32 p) {
    const u32 logL = rows ? logW : logH, lper = logL - 3;
    const u32 nlines = planes << (rows ? logH : logW);
    const bool active = threadIdx.x < (nlines << lper);
    u32 line, tl;
    if (rows) {
        line = threadIdx.x >> lper;
        tl = threadIdx.x & ((1u << lper) - 1u);
    } else {
        line = threadIdx.x % nlines;
        tl = threadIdx.x / nlines;
    }
    const u32 lbase = rows ? line << logW : ((line >> logW) << (logH + logW)) + (line & ((1u << logW) - 1u));
    const u32 sl = rows ? 0u : logW;
    const int npass = ((int)logL + 2) / 3;
    for (int ps = 0; ps < npass; ps++) {
        int hi, lo;
        u32 wlo;
        if (kDif) {
            hi = (int)logL - 1 - 3 * ps;
            lo = hi - 2 > 0 ? hi - 2 : 0;
            wlo = hi >= 2 ? (u32)hi - 2 : 0u;
        } else {
            lo = 3 * ps;
            hi = lo + 2 < (int)logL - 1 ? lo + 2 : (int)logL - 1;
            wlo = (u32)lo + 3 <= logL ? (u32)lo : logL - 3;
        }
        if (active) {
            const u32 low = tl & ((1u << wlo) - 1u);
            const u32 ib = ((tl >> wlo) << (wlo + 3)) | low;
            u32 off[8], x[8];
#pragma unroll
            for (int r = 0; r < 8; r++) {
                off[r] = padx(lbase + ((ib + ((u32)r << wlo)) << sl));
                x[r] = buf[off[r]];
            }
#pragma unroll
            for (int s = 0; s < 3; s++) {
                const int RB = kDif ? 2 - s : s;
                const int b = (int)wlo + RB;
                if (b > hi || b < lo) continue;
                const u32 sh = logL - 1 - (u32)b, tlow = low << sh;
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    if (r & (1 << RB)) continue;
                    const uint2 w = tw[tlow + (((u32)(r & ((1 << RB) - 1)) << wlo) << sh)];
                    const u32 u = x[r], v = x[r | (1 << RB)];
                    if (kDif) {
                        x[r] = addmod_p(u, v, p);
                        u32 d = shoup_mul32(submod_p(u, v, p), w.x, w.y, p);
                        x[r | (1 << RB)] = d >= p ? d - p : d;
                    } else {
                        u32 m = shoup_mul32(v, w.x, w.y, p);
                        m = m >= p ? m - p : m;
                        x[r] = addmod_p(u, m, p);
                        x[r | (1 << RB)] = submod_p(u, m, p);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 8; r++) buf[off[r]] = x[r];
        }
        __syncthreads();
    }
}

// Asynchronous copy of the (w_L^k, companion) pairs, k < L/2 (L = 2^logL
// >= 4), into dst (16-byte aligned); completed by stage_wait().
__device__ __forceinline__ void stage_pairs_for_length(uint2* dst, u32 logL, bool inverse, const DevParams& P) {
    const u32 half = 1u << (logL - 1);
    stage_async(dst, (inverse ? P.lpi : P.lpf) + half, half * 8);
}

