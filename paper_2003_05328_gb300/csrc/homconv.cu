// homconv.cu -- K4: HomConv fused with HomShare (Fig. 2, Eq. 2).
//
// In the NTT_q domain the homomorphic Hadamard product of an input
// ciphertext with a plaintext filter polynomial is a pointwise product, so
// for every evaluation index j the layer is a small modular matrix-vector
// product over the input ciphertexts k:
//   out[bb][co][h][c][j] = sum_k in[bb][k][h][c][j] * P[co][k][h][j]  (mod q)
// followed by the HomShare mask subtraction on c = 1.
//
// Work split: a CTA has 4 warps, one output channel per warp, and covers 64
// consecutive evaluation indices (2 per lane, so every operand row is read
// with 16-byte loads, fully coalesced).  Each thread also serves NB image
// groups, reusing every filter word from registers NB times.  The k loop is
// unrolled so that each thread keeps several 16-byte loads in flight; the
// input words are shared by the 4 warps through L1.
//
// Exact accumulation (both variants keep the true integer sum, reduced to
// [0, q) only at the end and every 256 terms, since 256 (q-1)^2 < 2^128):
//  - kWide:  operands split into 30-bit limbs (q < 2^60), the four limb
//            products accumulated with 32x32+64-bit multiply-adds into 64-bit
//            columns that are carried forward every 8 terms;
//  - !kWide: a 128-bit accumulator updated with carry-chained 32-bit
//            multiply-adds (10 per product).
#include <type_traits>

#include "modarith.cuh"

namespace {

constexpr u32 kWarps = 4;           // output channels per CTA
constexpr u32 kJT = 64;             // evaluation indices per CTA
constexpr u32 kThreads = 32 * kWarps;
constexpr u32 kUnroll = 4;          // k terms per load batch
constexpr u64 kM30 = (1ull << 30) - 1;

// ---- 128-bit carry-chain accumulator
struct Acc128 {
    u32 w[4];
};
__device__ __forceinline__ void acc_zero(Acc128& a) { a.w[0] = a.w[1] = a.w[2] = a.w[3] = 0; }
__device__ __forceinline__ void acc_mac(Acc128& acc, u64 a, u64 b) {
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
    asm("mad.lo.cc.u32  %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.u32    %3, %5, %7, %3;\n\t"
        "mad.lo.cc.u32  %1, %4, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
        "addc.u32       %3, %3, 0;\n\t"
        "mad.lo.cc.u32  %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "addc.u32       %3, %3, 0;"
        : "+r"(acc.w[0]), "+r"(acc.w[1]), "+r"(acc.w[2]), "+r"(acc.w[3])
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
}
__device__ __forceinline__ u64 acc_reduce(const Acc128& a, const DevParams& P) {
    return reduce128(((u64)a.w[3] << 32) | a.w[2], ((u64)a.w[1] << 32) | a.w[0], P);
}
// a += b (128-bit, carry-chained)
__device__ __forceinline__ void acc_add(Acc128& a, const Acc128& b) {
    asm("add.cc.u32  %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32    %3, %3, %7;"
        : "+r"(a.w[0]), "+r"(a.w[1]), "+r"(a.w[2]), "+r"(a.w[3])
        : "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]));
}
__device__ __forceinline__ void acc_set(Acc128& a, u64 r) {
    a.w[0] = (u32)r;
    a.w[1] = (u32)(r >> 32);
    a.w[2] = a.w[3] = 0;
}

// ---- 30-bit limb columns: value = c0 + c1 2^30 + c2 2^60 + c3 2^92
struct AccLimb {
    u64 c0, c1, c2, c3;
};
__device__ __forceinline__ void acc_zero(AccLimb& a) { a.c0 = a.c1 = a.c2 = a.c3 = 0; }
__device__ __forceinline__ void acc_mac_limbs(AccLimb& A, u32 x0, u32 x1, u32 w0, u32 w1) {
    A.c0 += (u64)x0 * w0;
    A.c1 += (u64)x0 * w1;
    A.c1 += (u64)x1 * w0;
    A.c2 += (u64)x1 * w1;
}
// Carry the columns forward: afterwards c0, c1 < 2^30, c2 < 2^32.  With at
// most 8 products per column between calls no column overflows 64 bits.
__device__ __forceinline__ void acc_normalize(AccLimb& A) {
    A.c1 += A.c0 >> 30;
    A.c0 &= kM30;
    A.c2 += A.c1 >> 30;
    A.c1 &= kM30;
    A.c3 += A.c2 >> 32;
    A.c2 &= 0xFFFFFFFFull;
}
__device__ __forceinline__ u64 acc_reduce(AccLimb A, const DevParams& P) {
    acc_normalize(A);
    const u64 t = A.c0 + (A.c1 << 30);
    const u64 lo = t + (A.c2 << 60);
    const u64 hi = (A.c2 >> 4) + (A.c3 << 28) + (lo < t ? 1 : 0);
    return reduce128(hi, lo, P);
}
__device__ __forceinline__ void acc_set(AccLimb& a, u64 r) {
    a.c0 = r & kM30;
    a.c1 = r >> 30;
    a.c2 = a.c3 = 0;
}

// ---- lazy 32-bit-limb columns.  With a = a1 2^32 + a0, b = b1 2^32 + b0
// (a1, b1 < 2^28 since q < 2^60): the low products a0 b0 go into a 96-bit
// word (one add-with-carry chain), the middle products a0 b1 + a1 b0 (each
// < 2^60) into a 64-bit column folded into `mh` every 4 terms, the high
// products a1 b1 (< 2^56) into a 64-bit column that cannot overflow within
// 256 terms.  Four 32x32+64-bit multiply-adds and three adds per product.
struct AccLazy {
    u32 l0, l1, l2;
    u64 mid, mh, hi;
};
__device__ __forceinline__ void acc_zero(AccLazy& a) {
    a.l0 = a.l1 = a.l2 = 0;
    a.mid = a.mh = a.hi = 0;
}
__device__ __forceinline__ void acc_mac(AccLazy& A, u64 a, u64 b) {
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
    const u64 p = (u64)a0 * b0;
    asm("add.cc.u32  %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32    %2, %2, 0;"
        : "+r"(A.l0), "+r"(A.l1), "+r"(A.l2)
        : "r"((u32)p), "r"((u32)(p >> 32)));
    A.mid += (u64)a0 * b1;
    A.mid += (u64)a1 * b0;
    A.hi += (u64)a1 * b1;
}
// Fold the middle column: afterwards mid < 2^32; between folds at most 4
// products (8 middle terms < 2^60 each) are added, so mid stays below 2^64.
__device__ __forceinline__ void acc_normalize(AccLazy& A) {
    A.mh += A.mid >> 32;
    A.mid &= 0xFFFFFFFFull;
}
__device__ __forceinline__ u64 acc_reduce(AccLazy A, const DevParams& P) {
    acc_normalize(A);
    const u64 L = ((u64)A.l1 << 32) | A.l0;
    const u64 lo = L + (A.mid << 32);
    const u64 hi = (u64)A.l2 + A.mh + A.hi + (lo < L ? 1 : 0);
    return reduce128(hi, lo, P);
}
__device__ __forceinline__ void acc_set(AccLazy& a, u64 r) {
    acc_zero(a);
    a.l0 = (u32)r;
    a.l1 = (u32)(r >> 32);
}

__device__ __forceinline__ ulonglong2 ldg2(const u64* p) { return __ldg(reinterpret_cast<const ulonglong2*>(p)); }
// The filter words of two consecutive evaluation indices (the first even):
// a pair when every index has its own word (d = 1), else the one word the
// group of d shares (filter plaintexts are w_0(x^d)).
__device__ __forceinline__ ulonglong2 ldgw2(const u64* p, u32 d) {
    if (d == 1) return ldg2(p);
    const u64 w = __ldg(p);
    return make_ulonglong2(w, w);
}

// kAdd extra c1 addends A1, A2 ([n_in][n] words) are added to every input
// ciphertext's c1 as it is loaded (HomRec of Bob's encoded share, and the
// message part of an encryption whose constants were drawn separately).
template <int NB, bool kWide, int kAdd>
__global__ void __launch_bounds__(kThreads) homconv_kernel(DevParams P, DevLayer L, const u64* __restrict__ ct_in,
                                                           const u64* __restrict__ A1, const u64* __restrict__ A2,
                                                           const u64* __restrict__ Phat,
                                                           const u64* __restrict__ Mhat, u64* __restrict__ ct_out,
                                                           u32 btiles, u32 jtiles) {
    using Acc = typename std::conditional<kWide, AccLimb, Acc128>::type;
    griddep_release();
    griddep_wait();
    u32 blk = blockIdx.x;
    const u32 bt = blk % btiles;
    blk /= btiles;
    const u32 jt = blk % jtiles, ct = blk / jtiles;
    const u32 co = ct * kWarps + (threadIdx.x >> 5);
    const u32 J = jt * kJT + 2 * (threadIdx.x & 31);
    const u32 nJ = L.beta * P.n;
    if (co >= L.Co || J >= nJ) return;
    const u32 h = J >> P.logn, j = J & (P.n - 1);
    const u64 n = P.n, beta = L.beta, T = L.T;
    const u32 bb0 = bt * NB;
    const u32 nbv = L.GB - bb0 < (u32)NB ? L.GB - bb0 : (u32)NB;

    Acc acc[NB][2][2];  // [image group][j offset][component]
#pragma unroll
    for (int b = 0; b < NB; b++)
#pragma unroll
        for (int e = 0; e < 2; e++) {
            acc_zero(acc[b][e][0]);
            acc_zero(acc[b][e][1]);
        }

    const u64 nd = n / P.d, w_step = beta * nd, x_step = beta * 2 * n;
    const u64* wp = Phat + ((u64)co * T * beta + h) * nd + j / P.d;
    const u64* xp[NB];
    u64 ap[NB];
#pragma unroll
    for (int b = 0; b < NB; b++) {
        const u64 u0 = (u64)(bb0 + (b < (int)nbv ? b : 0)) * T * beta + h;
        xp[b] = ct_in + u0 * 2 * n + j;
        ap[b] = u0 * n + j;
    }

    for (u32 k0 = 0; k0 < L.T; k0 += kUnroll) {
        ulonglong2 wv[kUnroll], xv[NB][kUnroll][2];
#pragma unroll
        for (int u = 0; u < (int)kUnroll; u++) {
            if (k0 + u < L.T) {
                wv[u] = ldgw2(wp + (k0 + u) * w_step, P.d);
#pragma unroll
                for (int b = 0; b < NB; b++) {
                    xv[b][u][0] = ldg2(xp[b] + (k0 + u) * x_step);
                    xv[b][u][1] = ldg2(xp[b] + (k0 + u) * x_step + n);
                    if constexpr (kAdd >= 1) {
                        const u64 off = (u64)ap[b] + (k0 + u) * w_step;
                        const ulonglong2 a1 = ldg2(A1 + off);
                        xv[b][u][1].x = addmod_q(xv[b][u][1].x, a1.x, P.q);
                        xv[b][u][1].y = addmod_q(xv[b][u][1].y, a1.y, P.q);
                        if constexpr (kAdd >= 2) {
                            const ulonglong2 a2 = ldg2(A2 + off);
                            xv[b][u][1].x = addmod_q(xv[b][u][1].x, a2.x, P.q);
                            xv[b][u][1].y = addmod_q(xv[b][u][1].y, a2.y, P.q);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < (int)kUnroll; u++) {
            if (k0 + u >= L.T) break;
            const u64 w2[2] = {wv[u].x, wv[u].y};
#pragma unroll
            for (int e = 0; e < 2; e++) {
                if constexpr (kWide) {
                    const u32 w0 = (u32)(w2[e] & kM30), w1 = (u32)(w2[e] >> 30);
#pragma unroll
                    for (int b = 0; b < NB; b++) {
#pragma unroll
                        for (int c = 0; c < 2; c++) {
                            const u64 x = e ? xv[b][u][c].y : xv[b][u][c].x;
                            acc_mac_limbs(acc[b][e][c], (u32)(x & kM30), (u32)(x >> 30), w0, w1);
                        }
                    }
                } else {
#pragma unroll
                    for (int b = 0; b < NB; b++)
#pragma unroll
                        for (int c = 0; c < 2; c++)
                            acc_mac(acc[b][e][c], e ? xv[b][u][c].y : xv[b][u][c].x, w2[e]);
                }
            }
        }
        if constexpr (kWide) {
            if (((k0 / kUnroll) & 1) || k0 + kUnroll >= L.T) {  // every 8 terms
#pragma unroll
                for (int b = 0; b < NB; b++)
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        acc_normalize(acc[b][e][0]);
                        acc_normalize(acc[b][e][1]);
                    }
            }
        }
        if (((k0 + kUnroll) & 255u) == 0 && k0 + kUnroll < L.T) {  // keep 256 (q-1)^2 < 2^128 headroom
#pragma unroll
            for (int b = 0; b < NB; b++)
#pragma unroll
                for (int e = 0; e < 2; e++)
#pragma unroll
                    for (int c = 0; c < 2; c++) acc_set(acc[b][e][c], acc_reduce(acc[b][e][c], P));
        }
    }

#pragma unroll
    for (int b = 0; b < NB; b++) {
        if (b >= (int)nbv) break;
        const u64 v = ((u64)(bb0 + b) * L.Co + co) * beta + h;
        ulonglong2 r0, r1;
        r0.x = acc_reduce(acc[b][0][0], P);
        r0.y = acc_reduce(acc[b][1][0], P);
        r1.x = acc_reduce(acc[b][0][1], P);
        r1.y = acc_reduce(acc[b][1][1], P);
        if (Mhat) {
            const ulonglong2 m = ldg2(Mhat + v * n + j);
            r1.x = submod_q(r1.x, m.x, P.q);
            r1.y = submod_q(r1.y, m.y, P.q);
        }
        *reinterpret_cast<ulonglong2*>(ct_out + v * 2 * n + j) = r0;
        *reinterpret_cast<ulonglong2*>(ct_out + v * 2 * n + n + j) = r1;
    }
}

template <int NB, bool W, int kAdd>
cudaError_t launch_variant(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                           const u64* Phat, const u64* Mhat, u64* ct_out, cudaStream_t s) {
    const u32 nJ = L.beta * P.n;
    const u32 jtiles = (nJ + kJT - 1) / kJT;
    const u32 ctiles = (L.Co + kWarps - 1) / kWarps;
    const u32 btiles = (L.GB + NB - 1) / NB;
    const u64 grid = (u64)jtiles * ctiles * btiles;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    return launch_online(homconv_kernel<NB, W, kAdd>, (u32)grid, kThreads, 0, s, P, L, ct_in, A1, A2, Phat, Mhat,
                         ct_out, btiles, jtiles);
}


// ---------------------------------------------------------------- v3: staged input tile
// A CTA covers kJ3 consecutive evaluation indices (one per lane) and kW3
// output channels (one per warp).  Its input tile -- every ciphertext k of
// the image group at those indices, with the c1 addends already summed -- is
// staged once in shared memory; the warps then stream only filter words from
// HBM, prefetching the next kPF3 terms while the current ones are multiplied.
constexpr u32 kJ3 = 32, kW3 = 8, kThreads3 = 32 * kW3, kPF3 = 8;

// kAcc: 0 carry-chained 128-bit, 1 30-bit limb columns, 2 lazy 32-bit-limb columns
template <int kAcc>
__global__ void __launch_bounds__(kThreads3) homconv3_kernel(DevParams P, DevLayer L, const u64* __restrict__ ct_in,
                                                             const u64* __restrict__ A1, const u64* __restrict__ A2,
                                                             const u64* __restrict__ Phat,
                                                             const u64* __restrict__ Mhat, u64* __restrict__ ct_out,
                                                             u32 jtiles, u32 ctiles, u64 seed, int seeded) {
    // seeded: ct_in holds c1 alone ([n_in][n]); c0 = -a is drawn again from
    // the encryption seed exactly as the encryption constants drew it
    extern __shared__ __align__(16) u64 xs[];  // [T][2][kJ3] canonical words, or 30-bit limb pairs
    constexpr bool kWide = kAcc == 1;
    using Acc = typename std::conditional<kAcc == 1, AccLimb,
                                          typename std::conditional<kAcc == 2, AccLazy, Acc128>::type>::type;
    u32 blk = blockIdx.x;
    const u32 jt = blk % jtiles;
    blk /= jtiles;
    const u32 ct = blk % ctiles, bb = blk / ctiles;
    const u32 nJ = L.beta * P.n, T = L.T;
    const u64 n = P.n, beta = L.beta;
    griddep_release();
    griddep_wait();
    const u64 keyA = stream_key(seed, DOM_A);
    // stage the input tile (all threads)
    for (u32 e = threadIdx.x; e < T * kJ3; e += kThreads3) {
        const u32 k = e / kJ3, jj = e % kJ3, J = jt * kJ3 + jj;
        u64 x0 = 0, x1 = 0;
        if (J < nJ) {
            const u32 h = J >> P.logn, j = J & (P.n - 1);
            const u64 u = ((u64)bb * T + k) * beta + h;
            if (seeded) {
                const u64 idx = 2 * (u * n + j);
                const u64 a = uniform_q(stream_at(keyA, idx), stream_at(keyA, idx + 1), P.q);
                x0 = a ? P.q - a : 0;
                x1 = __ldg(ct_in + u * n + j);
            } else {
                x0 = __ldg(ct_in + u * 2 * n + j);
                x1 = __ldg(ct_in + u * 2 * n + n + j);
            }
            if (A1) x1 = addmod_q(x1, __ldg(A1 + u * n + j), P.q);
            if (A2) x1 = addmod_q(x1, __ldg(A2 + u * n + j), P.q);
        }
        if constexpr (kWide) {
            x0 = (x0 & kM30) | ((x0 >> 30) << 32);
            x1 = (x1 & kM30) | ((x1 >> 30) << 32);
        }
        xs[(k * 2 + 0) * kJ3 + jj] = x0;
        xs[(k * 2 + 1) * kJ3 + jj] = x1;
    }
    __syncthreads();
    const u32 lane = threadIdx.x & 31, co = ct * kW3 + (threadIdx.x >> 5), J = jt * kJ3 + lane;
    if (co >= L.Co || J >= nJ) return;
    const u32 h = J >> P.logn, j = J & (P.n - 1);
    const u64 nd = n / P.d;
    const u64* wp = Phat + ((u64)co * T * beta + h) * nd + j / P.d;
    const u64 w_step = beta * nd;

    Acc acc0, acc1;
    acc_zero(acc0);
    acc_zero(acc1);
    u64 wbuf[kPF3];
#pragma unroll
    for (u32 u = 0; u < kPF3; u++) wbuf[u] = u < T ? __ldg(wp + u * w_step) : 0;
    for (u32 k0 = 0; k0 < T; k0 += kPF3) {
        u64 wcur[kPF3];
#pragma unroll
        for (u32 u = 0; u < kPF3; u++) {
            wcur[u] = wbuf[u];
            const u32 kn = k0 + kPF3 + u;
            if (kn < T) wbuf[u] = __ldg(wp + kn * w_step);
        }
#pragma unroll
        for (u32 u = 0; u < kPF3; u++) {
            const u32 k = k0 + u;
            if (k >= T) break;
            const u64 xa = xs[(k * 2 + 0) * kJ3 + lane], xb = xs[(k * 2 + 1) * kJ3 + lane];
            if constexpr (kWide) {
                const u32 w0 = (u32)(wcur[u] & kM30), w1 = (u32)(wcur[u] >> 30);
                acc_mac_limbs(acc0, (u32)xa, (u32)(xa >> 32), w0, w1);
                acc_mac_limbs(acc1, (u32)xb, (u32)(xb >> 32), w0, w1);
            } else {
                acc_mac(acc0, xa, wcur[u]);
                acc_mac(acc1, xb, wcur[u]);
            }
            if constexpr (kAcc == 2) {
                if ((u & 3) == 3) {
                    acc_normalize(acc0);
                    acc_normalize(acc1);
                }
            }
        }
        if constexpr (kAcc != 0) {
            acc_normalize(acc0);
            acc_normalize(acc1);
        }
        if (((k0 + kPF3) & 255u) == 0 && k0 + kPF3 < T) {
            acc_set(acc0, acc_reduce(acc0, P));
            acc_set(acc1, acc_reduce(acc1, P));
        }
    }
    const u64 v = ((u64)bb * L.Co + co) * beta + h;
    const u64 r0 = acc_reduce(acc0, P);
    u64 r1 = acc_reduce(acc1, P);
    if (Mhat) r1 = submod_q(r1, __ldg(Mhat + v * n + j), P.q);
    ct_out[v * 2 * n + j] = r0;
    ct_out[v * 2 * n + n + j] = r1;
}

template <int W>
cudaError_t launch_v3(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                      const u64* Phat, const u64* Mhat, u64* ct_out, cudaStream_t s, u64 seed = 0, int seeded = 0) {
    const u32 nJ = L.beta * P.n;
    const u32 jtiles = (nJ + kJ3 - 1) / kJ3, ctiles = (L.Co + kW3 - 1) / kW3;
    const u64 grid = (u64)jtiles * ctiles * L.GB;
    const size_t smem = (size_t)L.T * 2 * kJ3 * 8;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    if (smem + 1024 > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(homconv3_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_online(homconv3_kernel<W>, (u32)grid, kThreads3, smem, s, P, L, ct_in, A1, A2, Phat, Mhat, ct_out,
                         jtiles, ctiles, seed, seeded);
}

// ---------------------------------------------------------------- v4: Karatsuba limb columns
// Words below q < 2^60 split into 30-bit limbs, x = x1 2^30 + x0 and
// w = w1 2^30 + w0, and Karatsuba's identity
//   x w = x0 w0 + ((x0 + x1)(w0 + w1) - x0 w0 - x1 w1) 2^30 + x1 w1 2^60
// needs three 32 x 32 -> 64-bit multiply-adds per product (the carry chain
// needs ten 32-bit multiply steps, the plain limb columns four wide ones).
// Over k the three column sums lo = sum x0 w0, hi = sum x1 w1 (terms below
// 2^60) and mid = sum (x0 + x1)(w0 + w1) (terms below 2^62) live in 64-bit
// registers whose high words move into 64-bit carry registers every 4 terms
// (mid) or 8 terms (lo, hi), so no column overflows.  The 128-bit sum
// lo + (mid - lo - hi) 2^30 + hi 2^60 is assembled once per output word in
// wrapping 128-bit arithmetic -- exact, because the true sum (at most 256
// products of words below q, plus a residue) is below 2^128 -- and reduced
// mod q; longer sums are folded every 256 terms.
//
// Tiling as v3 (32 evaluation indices x 8 output channels per CTA, the input
// tile staged in shared memory as limb pairs), with NB image groups per CTA:
// each filter word, split once, serves the NB groups from registers.
constexpr u32 kJ4 = 32, kW4 = 8, kThreads4 = 32 * kW4, kPF4 = 8;
constexpr u32 kMaxStage4 = 160 * 1024;  // shared-memory cap of the staged tiles

struct AccK {
    u64 lo, lo_c, mid, mid_c, hi, hi_c;
};
__device__ __forceinline__ void acck_zero(AccK& a) { a.lo = a.lo_c = a.mid = a.mid_c = a.hi = a.hi_c = 0; }
// x: limb pair (x0 | x1 << 32); w0, w1 the filter word's limbs, ws = w0 + w1
__device__ __forceinline__ void acck_mac(AccK& a, u64 x, u32 w0, u32 w1, u32 ws) {
    const u32 x0 = (u32)x, x1 = (u32)(x >> 32);
    a.lo += (u64)x0 * w0;
    a.hi += (u64)x1 * w1;
    a.mid += (u64)(x0 + x1) * ws;
}
// mid < 2^32 afterwards; 4 more terms keep it below 2^32 + 4 (2^31 - 2)^2 < 2^64
__device__ __forceinline__ void acck_norm_mid(AccK& a) {
    a.mid_c += a.mid >> 32;
    a.mid &= 0xFFFFFFFFull;
}
// lo, hi < 2^32 afterwards; 8 more terms keep them below 2^32 + 8 2^60 < 2^64
__device__ __forceinline__ void acck_norm_lh(AccK& a) {
    a.lo_c += a.lo >> 32;
    a.lo &= 0xFFFFFFFFull;
    a.hi_c += a.hi >> 32;
    a.hi &= 0xFFFFFFFFull;
}
// (sum of the window's products + base) mod q
__device__ __forceinline__ u64 acck_reduce(const AccK& a, u64 base, const DevParams& P) {
    typedef unsigned __int128 u128;
    const u128 lo = ((u128)a.lo_c << 32) + a.lo, hi = ((u128)a.hi_c << 32) + a.hi;
    const u128 mid = ((u128)a.mid_c << 32) + a.mid;
    const u128 t = lo + ((mid - lo - hi) << 30) + (hi << 60) + base;
    return reduce128((u64)(t >> 64), (u64)t, P);
}
__device__ __forceinline__ u64 split30(u64 x) { return (x & kM30) | ((x >> 30) << 32); }

template <int NB, bool kFold>
__global__ void __launch_bounds__(kThreads4, NB == 1 ? 4 : 2)
    homconv4_kernel(DevParams P, DevLayer L, const u64* __restrict__ ct_in, const u64* __restrict__ A1,
                    const u64* __restrict__ A2, const u64* __restrict__ Phat, const u64* __restrict__ Mhat,
                    u64* __restrict__ ct_out, u32 jtiles, u32 ctiles) {
    extern __shared__ __align__(16) u64 xs4[];  // [NB][T][2][kJ4] limb pairs
    u32 blk = blockIdx.x;
    const u32 jt = blk % jtiles;
    blk /= jtiles;
    const u32 ct = blk % ctiles, bb0 = (blk / ctiles) * NB;
    const u32 nJ = L.beta * P.n, T = L.T;
    const u64 n = P.n, beta = L.beta;
    griddep_release();
    griddep_wait();
    const u32 per_g = T * kJ4;
    for (u32 e = threadIdx.x; e < NB * per_g; e += kThreads4) {
        const u32 g = e / per_g, r = e - g * per_g, k = r / kJ4, jj = r % kJ4, J = jt * kJ4 + jj;
        u64 x0 = 0, x1 = 0;
        if (J < nJ && bb0 + g < L.GB) {
            const u32 h = J >> P.logn, j = J & (P.n - 1);
            const u64 u = ((u64)(bb0 + g) * T + k) * beta + h;
            x0 = __ldg(ct_in + u * 2 * n + j);
            x1 = __ldg(ct_in + u * 2 * n + n + j);
            if (A1) x1 = addmod_q(x1, __ldg(A1 + u * n + j), P.q);
            if (A2) x1 = addmod_q(x1, __ldg(A2 + u * n + j), P.q);
        }
        xs4[((g * T + k) * 2 + 0) * kJ4 + jj] = split30(x0);
        xs4[((g * T + k) * 2 + 1) * kJ4 + jj] = split30(x1);
    }
    __syncthreads();
    const u32 lane = threadIdx.x & 31, co = ct * kW4 + (threadIdx.x >> 5), J = jt * kJ4 + lane;
    if (co >= L.Co || J >= nJ) return;
    const u32 h = J >> P.logn, j = J & (P.n - 1);
    const u64 nd = n / P.d;
    const u64* wp = Phat + ((u64)co * T * beta + h) * nd + j / P.d;
    const u64 w_step = beta * nd;

    AccK acc[NB][2];
    u64 base[kFold ? NB : 1][2];  // residues of the folded 256-term windows (kFold only)
#pragma unroll
    for (int g = 0; g < NB; g++) {
        acck_zero(acc[g][0]);
        acck_zero(acc[g][1]);
    }
#pragma unroll
    for (int g = 0; g < (kFold ? NB : 1); g++) base[g][0] = base[g][1] = 0;
    // a ring of kPF4 filter words in flight: the word for term k is replaced
    // by the one for term k + kPF4 as soon as it is used
    u64 wbuf[kPF4];
#pragma unroll
    for (u32 u = 0; u < kPF4; u++) wbuf[u] = u < T ? __ldg(wp + u * w_step) : 0;
    for (u32 k0 = 0; k0 < T; k0 += kPF4) {
#pragma unroll
        for (u32 u = 0; u < kPF4; u++) {
            const u32 k = k0 + u;
            if (k < T) {
                const u64 w = wbuf[u];
                if (k + kPF4 < T) wbuf[u] = __ldg(wp + (k + kPF4) * w_step);
                const u32 w0 = (u32)w & (u32)kM30, w1 = (u32)(w >> 30), ws = w0 + w1;
#pragma unroll
                for (int g = 0; g < NB; g++) {
                    const u64* xg = xs4 + (((u32)g * T + k) * 2) * kJ4 + lane;
                    acck_mac(acc[g][0], xg[0], w0, w1, ws);
                    acck_mac(acc[g][1], xg[kJ4], w0, w1, ws);
                }
            }
            if ((u & 3) == 3) {
#pragma unroll
                for (int g = 0; g < NB; g++) {
                    acck_norm_mid(acc[g][0]);
                    acck_norm_mid(acc[g][1]);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < NB; g++) {
            acck_norm_lh(acc[g][0]);
            acck_norm_lh(acc[g][1]);
        }
        if constexpr (kFold) {
            if (((k0 + kPF4) & 255u) == 0 && k0 + kPF4 < T) {  // fold every 256 terms
#pragma unroll
                for (int g = 0; g < NB; g++)
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        base[g][c] = acck_reduce(acc[g][c], base[g][c], P);
                        acck_zero(acc[g][c]);
                    }
            }
        }
    }
#pragma unroll
    for (int g = 0; g < NB; g++) {
        if (bb0 + g >= L.GB) break;
        const u64 v = ((u64)(bb0 + g) * L.Co + co) * beta + h;
        const u64 r0 = acck_reduce(acc[g][0], kFold ? base[kFold ? g : 0][0] : 0, P);
        u64 r1 = acck_reduce(acc[g][1], kFold ? base[kFold ? g : 0][1] : 0, P);
        if (Mhat) r1 = submod_q(r1, __ldg(Mhat + v * n + j), P.q);
        ct_out[v * 2 * n + j] = r0;
        ct_out[v * 2 * n + n + j] = r1;
    }
}

// ---------------------------------------------------------------- v5: lean staged tile, two indices per lane
// The carry-chained 128-bit accumulation of v3 with less work around each
// product: a CTA covers kJ5 = 64 consecutive evaluation indices (two per
// lane, so filter words, input words and outputs move as 16-byte pairs) and
// kW5 = 8 output channels (one per warp); the k loop is unrolled kTU terms
// deep with a ring of kTU filter-word pairs in flight per thread, whose
// first kTU loads are issued before the input tile is staged (the filter
// does not depend on the kernels before HomConv).  Needs T a multiple of
// kTU and T <= 128 (the staged tile, T KiB, stays in shared memory; no
// 256-term fold is needed).  (Under programmatic dependent launch the filter
// loads still wait for the previous kernel, like every access to caller
// memory.)
constexpr u32 kJ5 = 64, kW5 = 8, kThreads5 = 32 * kW5, kMaxT5 = 128;

template <int kTU>
__global__ void __launch_bounds__(kThreads5, 2)
    homconv5_kernel(DevParams P, DevLayer L, const u64* __restrict__ ct_in, const u64* __restrict__ A1,
                    const u64* __restrict__ A2, const u64* __restrict__ Phat, const u64* __restrict__ Mhat,
                    u64* __restrict__ ct_out, u32 jtiles, u32 ctiles) {
    extern __shared__ __align__(16) ulonglong2 xs5[];  // [T][2][kJ5 / 2] pairs of canonical words
    constexpr u32 kPairs = kJ5 / 2;
    u32 blk = blockIdx.x;
    const u32 jt = blk % jtiles;
    blk /= jtiles;
    const u32 ct = blk % ctiles, bb = blk / ctiles;
    const u32 nJ = L.beta * P.n, T = L.T;
    const u64 n = P.n, beta = L.beta;
    const u32 lane = threadIdx.x & 31, co = ct * kW5 + (threadIdx.x >> 5);
    const u32 J = jt * kJ5 + 2 * lane;  // J and J + 1 lie in the same half (n even)
    const bool active = co < L.Co && J < nJ;
    const u32 h = J >> P.logn, j = J & (P.n - 1);
    const u64 nd = n / P.d;
    const u64* wp = Phat + ((u64)(active ? co : 0) * T * beta + (active ? h : 0)) * nd + (active ? j / P.d : 0);
    const u64 w_step = beta * nd;
    griddep_release();
    griddep_wait();
    ulonglong2 ring[kTU];
#pragma unroll
    for (int u = 0; u < kTU; u++) ring[u] = active ? ldgw2(wp + (u64)u * w_step, P.d) : make_ulonglong2(0, 0);
    for (u32 e = threadIdx.x; e < T * kPairs; e += kThreads5) {
        const u32 k = e / kPairs, jp = e % kPairs, Jx = jt * kJ5 + 2 * jp;
        ulonglong2 x0 = make_ulonglong2(0, 0), x1 = make_ulonglong2(0, 0);
        if (Jx < nJ) {
            const u32 hx = Jx >> P.logn, jx = Jx & (P.n - 1);
            const u64 u = ((u64)bb * T + k) * beta + hx;
            x0 = ldg2(ct_in + u * 2 * n + jx);
            x1 = ldg2(ct_in + u * 2 * n + n + jx);
            if (A1) {
                const ulonglong2 a = ldg2(A1 + u * n + jx);
                x1.x = addmod_q(x1.x, a.x, P.q);
                x1.y = addmod_q(x1.y, a.y, P.q);
            }
            if (A2) {
                const ulonglong2 a = ldg2(A2 + u * n + jx);
                x1.x = addmod_q(x1.x, a.x, P.q);
                x1.y = addmod_q(x1.y, a.y, P.q);
            }
        }
        xs5[(k * 2 + 0) * kPairs + jp] = x0;
        xs5[(k * 2 + 1) * kPairs + jp] = x1;
    }
    __syncthreads();
    if (!active) return;
    Acc128 acc[2][2];  // [index J + e][component]
#pragma unroll
    for (int e = 0; e < 2; e++) {
        acc_zero(acc[e][0]);
        acc_zero(acc[e][1]);
    }
    for (u32 k0 = 0; k0 < T; k0 += kTU) {
#pragma unroll
        for (int u = 0; u < kTU; u++) {
            const u32 k = k0 + u;
            const ulonglong2 w = ring[u];
            if (k + kTU < T) ring[u] = ldgw2(wp + (u64)(k + kTU) * w_step, P.d);
            const ulonglong2 xa = xs5[(k * 2 + 0) * kPairs + lane], xb = xs5[(k * 2 + 1) * kPairs + lane];
            acc_mac(acc[0][0], xa.x, w.x);
            acc_mac(acc[1][0], xa.y, w.y);
            acc_mac(acc[0][1], xb.x, w.x);
            acc_mac(acc[1][1], xb.y, w.y);
        }
    }
    const u64 v = ((u64)bb * L.Co + co) * beta + h;
    ulonglong2 r0, r1;
    r0.x = acc_reduce(acc[0][0], P);
    r0.y = acc_reduce(acc[1][0], P);
    r1.x = acc_reduce(acc[0][1], P);
    r1.y = acc_reduce(acc[1][1], P);
    if (Mhat) {
        const ulonglong2 m = ldg2(Mhat + v * n + j);
        r1.x = submod_q(r1.x, m.x, P.q);
        r1.y = submod_q(r1.y, m.y, P.q);
    }
    *reinterpret_cast<ulonglong2*>(ct_out + v * 2 * n + j) = r0;
    *reinterpret_cast<ulonglong2*>(ct_out + v * 2 * n + n + j) = r1;
}

bool v5_supported(const DevLayer& L) { return L.T <= kMaxT5 && L.T % 4 == 0; }

// ---------------------------------------------------------------- v6: filter stream through shared memory
// v5's tile and accumulation, with the filter words streamed by cp.async
// into a per-thread ring of kD slots in shared memory instead of registers:
// every thread copies exactly the 16-byte filter pairs it multiplies (its
// output channel, its two indices), so the ring needs no barrier, and kD
// pairs per thread stay in flight without holding registers (kD = 16:
// 128 KiB of filter in flight per SM at two CTAs per SM).  One copy group is
// committed per term (empty past the end), so waiting for all but the kD - 1
// newest groups completes exactly the term about to be used.
constexpr u32 kMaxT6 = 64;

__device__ __forceinline__ void cp_async16(void* smem, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((u32)__cvta_generic_to_shared(smem)), "l"(g)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// A thread's filter pair: 16 bytes, or the 8 bytes both indices share
__device__ __forceinline__ void cp_async_w(void* smem, const void* g, bool shared_w) {
    if (shared_w)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((u32)__cvta_generic_to_shared(smem)), "l"(g)
                     : "memory");
    else
        cp_async16(smem, g);
}

// kS: independent partial sums per output word (term k goes to sum k mod kS),
// so that each thread has 4 kS carry chains in flight instead of 4: the
// chains' dependent latency, not the multiply pipe, bounds the kernel at one
// image, where a scheduler has only about four warps.
template <int kD, int kS, bool kEarly>
__global__ void __launch_bounds__(kThreads5, 2)
    homconv6_kernel(DevParams P, DevLayer L, const u64* __restrict__ ct_in, const u64* __restrict__ A1,
                    const u64* __restrict__ A2, const u64* __restrict__ Phat, const u64* __restrict__ Mhat,
                    u64* __restrict__ ct_out, u32 jtiles, u32 ctiles) {
    extern __shared__ __align__(16) ulonglong2 sm6[];  // [kD][kThreads5] filter ring, then [T][2][kJ5 / 2] inputs
    constexpr u32 kPairs = kJ5 / 2;
    ulonglong2* ring = sm6 + threadIdx.x;  // slot s at ring[s * kThreads5]
    ulonglong2* xs = sm6 + kD * kThreads5;
    u32 blk = blockIdx.x;
    const u32 jt = blk % jtiles;
    blk /= jtiles;
    const u32 ct = blk % ctiles, bb = blk / ctiles;
    const u32 nJ = L.beta * P.n, T = L.T;
    const u64 n = P.n, beta = L.beta;
    const u32 lane = threadIdx.x & 31, co = ct * kW5 + (threadIdx.x >> 5);
    const u32 J = jt * kJ5 + 2 * lane;  // J and J + 1 lie in the same half (n even)
    const bool active = co < L.Co && J < nJ;
    const u32 h = J >> P.logn, j = J & (P.n - 1);
    const u64 nd = n / P.d;
    const u64* wp = Phat + ((u64)(active ? co : 0) * T * beta + (active ? h : 0)) * nd + (active ? j / P.d : 0);
    const u64 w_step = beta * nd;
    const bool shared_w = P.d > 1;  // both indices use one filter word (copied as 8 bytes)
    griddep_release();
    // the first kD filter terms: before the grid-dependency wait when the
    // caller guarantees the kernel before this one does not write P_hat
    if (!kEarly) griddep_wait();
#pragma unroll
    for (int u = 0; u < kD; u++) {
        if (active && (u32)u < T) cp_async_w(ring + u * kThreads5, wp + (u64)u * w_step, shared_w);
        cp_commit();
    }
    if (kEarly) griddep_wait();
    ulonglong2 m = make_ulonglong2(0, 0);
    if (active && Mhat) m = ldg2(Mhat + (((u64)bb * L.Co + co) * beta + h) * n + j);
    // the input tile: every thread's loads (kSU pairs at a time) are issued
    // before any is used, so the tile costs one memory latency, not kSU
    constexpr u32 kSU = 4;
    for (u32 e0 = threadIdx.x; e0 < T * kPairs; e0 += kSU * kThreads5) {
        ulonglong2 x0[kSU], x1[kSU], a1[kSU], a2[kSU];
#pragma unroll
        for (u32 i = 0; i < kSU; i++) {
            const u32 e = e0 + i * kThreads5, k = e / kPairs, jp = e % kPairs, Jx = jt * kJ5 + 2 * jp;
            x0[i] = x1[i] = a1[i] = a2[i] = make_ulonglong2(0, 0);
            if (e < T * kPairs && Jx < nJ) {
                const u32 hx = Jx >> P.logn, jx = Jx & (P.n - 1);
                const u64 u = ((u64)bb * T + k) * beta + hx;
                x0[i] = ldg2(ct_in + u * 2 * n + jx);
                x1[i] = ldg2(ct_in + u * 2 * n + n + jx);
                if (A1) a1[i] = ldg2(A1 + u * n + jx);
                if (A2) a2[i] = ldg2(A2 + u * n + jx);
            }
        }
#pragma unroll
        for (u32 i = 0; i < kSU; i++) {
            const u32 e = e0 + i * kThreads5, k = e / kPairs, jp = e % kPairs;
            if (e >= T * kPairs) break;
            ulonglong2 c1 = x1[i];
            c1.x = addmod_q(addmod_q(c1.x, a1[i].x, P.q), a2[i].x, P.q);
            c1.y = addmod_q(addmod_q(c1.y, a1[i].y, P.q), a2[i].y, P.q);
            xs[(k * 2 + 0) * kPairs + jp] = x0[i];
            xs[(k * 2 + 1) * kPairs + jp] = c1;
        }
    }
    __syncthreads();
    if (!active) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        return;
    }
    Acc128 acc[kS][2][2];  // [partial sum][index J + e][component]
#pragma unroll
    for (int s = 0; s < kS; s++)
#pragma unroll
        for (int e = 0; e < 2; e++) {
            acc_zero(acc[s][e][0]);
            acc_zero(acc[s][e][1]);
        }
    for (u32 k0 = 0; k0 < T; k0 += kD) {
#pragma unroll
        for (int u = 0; u < kD; u++) {
            const u32 k = k0 + u;
            if (k < T) {
                asm volatile("cp.async.wait_group %0;" ::"n"(kD - 1) : "memory");
                ulonglong2 w = ring[u * kThreads5];
                if (shared_w) w.y = w.x;
                const ulonglong2 xa = xs[(k * 2 + 0) * kPairs + lane], xb = xs[(k * 2 + 1) * kPairs + lane];
                Acc128(&a)[2][2] = acc[u % kS];  // kD is a multiple of kS: term k -> sum k mod kS
                acc_mac(a[0][0], xa.x, w.x);
                acc_mac(a[1][0], xa.y, w.y);
                acc_mac(a[0][1], xb.x, w.x);
                acc_mac(a[1][1], xb.y, w.y);
                // the slot is refilled only after its words were used
                if (k + kD < T) cp_async_w(ring + u * kThreads5, wp + (u64)(k + kD) * w_step, shared_w);
                cp_commit();
            }
        }
    }
#pragma unroll
    for (int s = 1; s < kS; s++)  // T <= 64 products in all: the sums stay below 2^128
#pragma unroll
        for (int e = 0; e < 2; e++) {
            acc_add(acc[0][e][0], acc[s][e][0]);
            acc_add(acc[0][e][1], acc[s][e][1]);
        }
    const u64 v = ((u64)bb * L.Co + co) * beta + h;
    ulonglong2 r0, r1;
    r0.x = acc_reduce(acc[0][0][0], P);
    r0.y = acc_reduce(acc[0][1][0], P);
    r1.x = acc_reduce(acc[0][0][1], P);
    r1.y = acc_reduce(acc[0][1][1], P);
    if (Mhat) {
        r1.x = submod_q(r1.x, m.x, P.q);
        r1.y = submod_q(r1.y, m.y, P.q);
    }
    *reinterpret_cast<ulonglong2*>(ct_out + v * 2 * n + j) = r0;
    *reinterpret_cast<ulonglong2*>(ct_out + v * 2 * n + n + j) = r1;
}

bool v6_supported(const DevLayer& L) { return L.T <= kMaxT6; }

template <int kD, int kS, bool kEarly = false>
cudaError_t launch_v6(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                      const u64* Phat, const u64* Mhat, u64* ct_out, cudaStream_t s) {
    const u32 nJ = L.beta * P.n;
    const u32 jtiles = (nJ + kJ5 - 1) / kJ5, ctiles = (L.Co + kW5 - 1) / kW5;
    const u64 grid = (u64)jtiles * ctiles * L.GB;
    const size_t smem = (size_t)kD * kThreads5 * 16 + (size_t)L.T * 2 * kJ5 * 8;
    if (grid > 0x7FFFFFFFull || !v6_supported(L)) return cudaErrorInvalidConfiguration;
    if (smem + 1024 > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(homconv6_kernel<kD, kS, kEarly>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_online(homconv6_kernel<kD, kS, kEarly>, (u32)grid, kThreads5, smem, s, P, L, ct_in, A1, A2, Phat, Mhat, ct_out,
                         jtiles, ctiles);
}

cudaError_t launch_v5(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                      const u64* Phat, const u64* Mhat, u64* ct_out, cudaStream_t s) {
    const u32 nJ = L.beta * P.n;
    const u32 jtiles = (nJ + kJ5 - 1) / kJ5, ctiles = (L.Co + kW5 - 1) / kW5;
    const u64 grid = (u64)jtiles * ctiles * L.GB;
    const size_t smem = (size_t)L.T * 2 * kJ5 * 8;
    if (grid > 0x7FFFFFFFull || !v5_supported(L)) return cudaErrorInvalidConfiguration;
    void (*kern)(DevParams, DevLayer, const u64*, const u64*, const u64*, const u64*, const u64*, u64*, u32, u32) =
        L.T % 8 == 0 ? homconv5_kernel<8> : homconv5_kernel<4>;
    if (smem + 1024 > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_online(kern, (u32)grid, kThreads5, smem, s, P, L, ct_in, A1, A2, Phat, Mhat, ct_out, jtiles,
                         ctiles);
}

// NB image groups per CTA (the caller checks that the staged tiles fit)
template <int NB>
cudaError_t launch_v4(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                      const u64* Phat, const u64* Mhat, u64* ct_out, cudaStream_t s) {
    const u32 nJ = L.beta * P.n;
    const u32 jtiles = (nJ + kJ4 - 1) / kJ4, ctiles = (L.Co + kW4 - 1) / kW4, btiles = (L.GB + NB - 1) / NB;
    const u64 grid = (u64)jtiles * ctiles * btiles;
    const size_t smem = (size_t)NB * L.T * 2 * kJ4 * 8;
    if (grid > 0x7FFFFFFFull || smem > kMaxStage4) return cudaErrorInvalidConfiguration;
    const bool fold = L.T > 256;
    void (*kern)(DevParams, DevLayer, const u64*, const u64*, const u64*, const u64*, const u64*, u64*, u32, u32) =
        fold ? homconv4_kernel<NB, true> : homconv4_kernel<NB, false>;
    if (smem + 1024 > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_online(kern, (u32)grid, kThreads4, smem, s, P, L, ct_in, A1, A2, Phat, Mhat, ct_out, jtiles,
                         ctiles);
}


}  // namespace

// Variant selection: 0 = automatic, 1 = limb columns NB=1, 2 = limb columns
// NB=2, 3 = carry chain NB=1, 4 = staged tile with carry chain, 5 = staged
// tile with limb columns, 6 = staged tile with lazy 32-bit-limb columns,
// 8 / 9 = staged tile with Karatsuba limb columns and 1 / 2 image groups per
// CTA, 10 = lean staged tile with two indices per lane (T a multiple of 4,
// at most 128; 4 otherwise), 11 / 12 = the same with the filter streamed
// through a shared-memory ring of 16 / 8 terms (T <= 64; 10 otherwise), 13 /
// 14 = 12 with 2 / 4 independent partial sums per output word.  7 is the
// tensor-core kernel, a plan-only choice.
static int g_homconv_variant = 0;
bool homconv_variant_valid(int v) { return v >= 0 && v <= 15 && v != 7; }
extern "C" int fdsc_set_homconv_variant(int v) {
    if (!homconv_variant_valid(v)) return FDSC_ERR_ARG;
    g_homconv_variant = v;
    return FDSC_OK;
}

template <int NB, bool W>
cudaError_t launch_adds(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                        const u64* Phat, const u64* Mhat, u64* ct_out, cudaStream_t s) {
    if (!A1 && A2) {
        A1 = A2;
        A2 = nullptr;
    }
    if (!A1) return launch_variant<NB, W, 0>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
    if (!A2) return launch_variant<NB, W, 1>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
    return launch_variant<NB, W, 2>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
}

// Measured on GB300 (32x32x64 layer at 1 and 16 images): the shared-memory
// filter ring (12) is the fastest up to T = 64 (equal at one image, 12 %
// faster at 16); beyond that the staged carry-chain kernel (4), and past 256
// terms the unstaged one (3).
int homconv_default_variant(const DevLayer& L) { return L.T <= kMaxT6 ? 12 : (L.T <= 256 ? 4 : 3); }

// The variant launch_homconv_v runs when asked for v (the fallbacks below).
int homconv_effective_variant(const DevLayer& L, int v) {
    if (v <= 0 || v > 15 || v == 7) v = homconv_default_variant(L);
    if (v >= 11 && v <= 15 && !v6_supported(L)) v = 10;
    if (v == 10 && !v5_supported(L)) v = L.T <= 256 ? 4 : 3;
    if (v >= 8 && v <= 9 && (u64)L.T * 2 * kJ4 * 8 > kMaxStage4) v = 3;
    if (v >= 4 && v <= 6 && L.T > 256) v = 3;
    return v;
}

cudaError_t launch_homconv_v(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                             const u64* Phat, const u64* Mhat, u64* ct_out, int v, cudaStream_t s) {
    if (v <= 0 || v > 15 || v == 7) v = homconv_default_variant(L);
    if (v >= 11 && v <= 15) {
        if (v6_supported(L)) switch (v) {
                case 11: return launch_v6<16, 1>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
                case 12: return launch_v6<8, 1>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
                case 13: return launch_v6<8, 2>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
                case 14: return launch_v6<8, 4>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
                default: return launch_v6<8, 1, true>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
            }
        v = 10;
    }
    if (v == 10) {
        if (v5_supported(L)) return launch_v5(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
        v = L.T <= 256 ? 4 : 3;
    }
    if (v >= 8) {  // Karatsuba columns: as many image groups per CTA as the staged tiles allow
        const u64 tile = (u64)L.T * 2 * kJ4 * 8;
        if (v >= 9 && 2 * tile <= kMaxStage4 && L.GB >= 2)
            return launch_v4<2>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
        if (tile <= kMaxStage4) return launch_v4<1>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
        v = 3;
    }
    // the staged tile must fit in shared memory (T <= 256 words x 2 x 32 lanes)
    if (v >= 4 && L.T > 256) v = 3;
    switch (v) {
        case 4: return launch_v3<0>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
        case 5: return launch_v3<1>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
        case 6: return launch_v3<2>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
        case 1: return launch_adds<1, true>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
        case 2: return launch_adds<2, true>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
        default: return launch_adds<1, false>(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, s);
    }
}

cudaError_t launch_homconv(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                           const u64* Phat, const u64* Mhat, u64* ct_out, cudaStream_t s) {
    return launch_homconv_v(P, L, ct_in, A1, A2, Phat, Mhat, ct_out, g_homconv_variant, s);
}

// HomConv of seeded input ciphertexts (c1 alone, c0 from the encryption seed):
// the staged-tile kernel, which draws c0 once per tile while staging it.
cudaError_t launch_homconv_seeded(const DevParams& P, const DevLayer& L, u64 seed, const u64* c1, const u64* A1,
                                  const u64* A2, const u64* Phat, const u64* Mhat, u64* ct_out, cudaStream_t s) {
    if (L.T > 256) return cudaErrorInvalidValue;
    return launch_v3<0>(P, L, c1, A1, A2, Phat, Mhat, ct_out, s, seed, 1);
}

// ---------------------------------------------------------------- throughput of the exact primitives
// Register-resident loops of the arithmetic the hot kernels are built from,
// each chain loop-carried (an operand depends on the previous result) so
// nothing is hoisted: 0 = the 60 x 60 -> 128-bit multiply-accumulate of
// HomConv (acc_mac), 1 = the 64-bit Shoup multiplication of the NTT_q
// butterflies, 2 = the 32-bit Shoup multiplication of the mod-p transforms.
// Four independent chains per thread.
namespace {
__global__ void __launch_bounds__(256) calib_kernel(int which, u32 iters, u64 w, u64 ws, u64 q, u64* sink, int store) {
    u64 r = threadIdx.x;
    if (which == 0) {
        Acc128 acc[4];
#pragma unroll
        for (int i = 0; i < 4; i++) acc_zero(acc[i]);
        u64 x[4] = {w ^ threadIdx.x, w + 1, w + 2, w + 3};
        for (u32 it = 0; it < iters; it++) {
#pragma unroll
            for (int i = 0; i < 4; i++) {
                acc_mac(acc[i], x[i], ws);
                x[i] ^= acc[i].w[1];
            }
        }
#pragma unroll
        for (int i = 0; i < 4; i++) r ^= acc[i].w[0] ^ acc[i].w[3];
    } else if (which == 1) {
        u64 x[4] = {w ^ threadIdx.x, w + 1, w + 2, w + 3};
        for (u32 it = 0; it < iters; it++) {
#pragma unroll
            for (int i = 0; i < 4; i++) x[i] = shoup_mul(x[i], w, ws, q);
        }
        r ^= x[0] ^ x[1] ^ x[2] ^ x[3];
    } else {
        u32 x[4] = {(u32)w ^ threadIdx.x, (u32)w + 1, (u32)w + 2, (u32)w + 3};
        for (u32 it = 0; it < iters; it++) {
#pragma unroll
            for (int i = 0; i < 4; i++) x[i] = shoup_mul32(x[i], (u32)w, (u32)ws, (u32)q);
        }
        r ^= x[0] ^ x[1] ^ x[2] ^ x[3];
    }
    if (store) sink[blockIdx.x * blockDim.x + threadIdx.x] = r;  // a run-time flag (0): the loops stay
}
}  // namespace

extern "C" int fdsc_calibrate(const fdsc_params* P, int which, double* ops_per_s, double* ops_per_clk_sm) {
    if (!P || which < 0 || which > 2 || !ops_per_s || !ops_per_clk_sm) return fdsc_set_error(FDSC_ERR_ARG, "bad arguments");
    int dev = 0, sms = 0, khz = 0;
    cudaGetDevice(&dev);
    if (dev != P->device) return fdsc_set_error(FDSC_ERR_ARG, "params belong to another device");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    const DevParams& D = P->dev;
    u64 w, ws, q;
    if (which == 2) {
        q = D.p;
        w = 3;  // any residue below p; its companion follows
        ws = ((u64)w << 32) / q;
    } else {
        q = D.q;
        w = D.delta % q;
        ws = (u64)(((unsigned __int128)w << 64) / q);
    }
    u64* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, (size_t)sms * 8 * 256 * sizeof(u64));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const u32 blocks = (u32)sms * 8, threads = 256, iters = which == 0 ? 2000 : 8000;
    float ms = 0;
    for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {  // the first run warms up
        cudaEventRecord(e0);
        calib_kernel<<<blocks, threads>>>(which, iters, w, ws, q, sink, 0);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return fdsc_set_error(FDSC_ERR_CUDA, "calibrate: %s", cudaGetErrorString(e));
    const double ops = (double)blocks * threads * iters * 4;
    *ops_per_s = ops / (ms * 1e-3);
    *ops_per_clk_sm = *ops_per_s / ((double)khz * 1e3) / sms;
    return FDSC_OK;
}
