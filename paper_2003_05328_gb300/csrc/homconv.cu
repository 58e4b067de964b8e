// homconv.cu -- K4: HomConv fused with HomShare (Fig. 2 lines 3-4, Eq. 2).
//
// In the NTT_q domain the homomorphic Hadamard product of an input
// ciphertext with a plaintext filter polynomial is a pointwise product, so
// for every evaluation index j the layer is a small modular matrix-vector
// product over the input ciphertexts k:
//   out[bb][co][h][c][j] = sum_k in[bb][k][h][c][j] * P[co][k][h][j]  (mod q)
// followed by the HomShare mask subtraction on c = 1.
//
// Each thread owns one index J = (h, j) and a chunk of output channels; the
// 60-bit x 60-bit products are accumulated exactly in 128 bits with
// carry-chained 32-bit multiply-adds and reduced once per output (and every
// 256 terms, so that T (q-1)^2 < 2^128 always holds).  A warp reads 32
// consecutive uint64 of every operand row: fully coalesced.
#include "modarith.cuh"

namespace {

// acc += a * b as 128-bit integers.  With a = a1 2^32 + a0 and b likewise:
// a0 b0 + a1 b1 2^64 in one carry chain, then a0 b1 2^32 and a1 b0 2^32.
__device__ __forceinline__ void mac128(u32 (&acc)[4], u64 a, u64 b) {
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
        : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2]), "+r"(acc[3])
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
}

__device__ __forceinline__ u64 reduce_acc(const u32 (&acc)[4], const DevParams& P) {
    const u64 lo = ((u64)acc[1] << 32) | acc[0], hi = ((u64)acc[3] << 32) | acc[2];
    return reduce128(hi, lo, P);
}

__device__ __forceinline__ void set_acc(u32 (&acc)[4], u64 v) {
    acc[0] = (u32)v;
    acc[1] = (u32)(v >> 32);
    acc[2] = 0;
    acc[3] = 0;
}

constexpr u32 kThreads = 128;

template <int CB>
__global__ void __launch_bounds__(kThreads) homconv_kernel(DevParams P, DevLayer L, const u64* __restrict__ ct_in,
                                                           const u64* __restrict__ Phat,
                                                           const u64* __restrict__ Mhat, u64* __restrict__ ct_out,
                                                           u32 jblocks, u32 cchunks) {
    const u32 nJ = L.beta * P.n;
    u32 blk = blockIdx.x;
    const u32 jb = blk % jblocks;
    blk /= jblocks;
    const u32 cc = blk % cchunks, bb = blk / cchunks;
    const u32 J = jb * kThreads + threadIdx.x;
    if (J >= nJ) return;
    const u32 h = J >> P.logn, j = J & (P.n - 1);
    const u32 co0 = cc * CB;
    const u64 n = P.n, beta = L.beta, T = L.T;

    u32 acc[CB][2][4];
#pragma unroll
    for (int cb = 0; cb < CB; cb++)
#pragma unroll
        for (int c = 0; c < 2; c++) set_acc(acc[cb][c], 0);

    const u64* in_p = ct_in + ((u64)bb * T * beta + h) * 2 * n + j;  // + k beta 2n + c n
    const u64* w_p = Phat + ((u64)co0 * T * beta + h) * n + j;       // + (cb T + k) beta n
    const u64 in_step = beta * 2 * n, w_step = beta * n, w_cb = T * beta * n;
    const u32 cb_valid = L.Co - co0 < (u32)CB ? L.Co - co0 : (u32)CB;

    for (u32 k = 0; k < L.T; k++) {
        const u64 x0 = in_p[k * in_step], x1 = in_p[k * in_step + n];
#pragma unroll
        for (int cb = 0; cb < CB; cb++) {
            if ((u32)cb < cb_valid) {
                const u64 w = w_p[cb * w_cb + k * w_step];
                mac128(acc[cb][0], x0, w);
                mac128(acc[cb][1], x1, w);
            }
        }
        if ((k & 255u) == 255u) {
#pragma unroll
            for (int cb = 0; cb < CB; cb++)
#pragma unroll
                for (int c = 0; c < 2; c++) set_acc(acc[cb][c], reduce_acc(acc[cb][c], P));
        }
    }
#pragma unroll
    for (int cb = 0; cb < CB; cb++) {
        if ((u32)cb >= cb_valid) continue;
        const u32 co = co0 + cb;
        const u64 v = ((u64)bb * L.Co + co) * beta + h;
        u64 r0 = reduce_acc(acc[cb][0], P), r1 = reduce_acc(acc[cb][1], P);
        if (Mhat) r1 = submod_q(r1, Mhat[v * n + j], P.q);
        ct_out[v * 2 * n + j] = r0;
        ct_out[v * 2 * n + n + j] = r1;
    }
}

}  // namespace

cudaError_t launch_homconv(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* Phat, const u64* Mhat,
                           u64* ct_out, cudaStream_t s) {
    constexpr int CB = 4;
    const u32 nJ = L.beta * P.n;
    const u32 jblocks = (nJ + kThreads - 1) / kThreads;
    const u32 cchunks = (L.Co + CB - 1) / CB;
    const u64 grid = (u64)jblocks * cchunks * L.GB;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    homconv_kernel<CB><<<(u32)grid, kThreads, 0, s>>>(P, L, ct_in, Phat, Mhat, ct_out, jblocks, cchunks);
    return cudaGetLastError();
}
