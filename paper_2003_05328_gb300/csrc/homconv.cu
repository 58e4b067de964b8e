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

    const u64 w_step = beta * n, x_step = beta * 2 * n;
    const u64* wp = Phat + ((u64)co * T * beta + h) * n + j;
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
                wv[u] = ldg2(wp + (k0 + u) * w_step);
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
    const u64* wp = Phat + ((u64)co * T * beta + h) * n + j;
    const u64 w_step = beta * n;

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


}  // namespace

// Variant selection: 0 = automatic, 1 = limb columns NB=1, 2 = limb columns
// NB=2, 3 = carry chain NB=1, 4 = staged tile with carry chain, 5 = staged
// tile with limb columns, 6 = staged tile with lazy 32-bit-limb columns.
static int g_homconv_variant = 0;
extern "C" int fdsc_set_homconv_variant(int v) {
    if (v < 0 || v > 6) return FDSC_ERR_ARG;
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

int homconv_default_variant(const DevLayer& L) { return L.T <= 256 ? 4 : 3; }

cudaError_t launch_homconv_v(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                             const u64* Phat, const u64* Mhat, u64* ct_out, int v, cudaStream_t s) {
    if (v <= 0 || v > 6) v = homconv_default_variant(L);
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
