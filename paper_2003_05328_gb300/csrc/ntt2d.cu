// ntt2d.cu -- K1 / K2: batched cyclic NTT2D / INTT2D mod p over padded
// H x W planes (Eq. 12 in two dimensions; Fig. 2's forward and inverse transforms).
//
// One CTA transforms one plane at a time in shared memory: the plane is read
// with coalesced loads and scattered into bit-reversed order, rows and then
// columns run radix-2 decimation-in-time butterflies, and the natural-order
// spectrum is written back with coalesced stores.
#include "modarith.cuh"

// Small planes (H or W < 8): bit-reversed load, radix-2 DIT stages.
__global__ void __launch_bounds__(256) ntt2d_small_kernel(DevParams P, u32 logH, u32 logW, const u32* x, u32* X,
                                                          u64 planes, int inverse, u32 scale, u32 scale_s) {
    extern __shared__ u32 plane[];
    const u32 HW = 1u << (logH + logW), W = 1u << logW;
    griddep_release();
    griddep_wait();
    for (u64 pl = blockIdx.x; pl < planes; pl += gridDim.x) {
        const uint4* src = reinterpret_cast<const uint4*>(x + pl * HW);
        for (u32 e4 = threadIdx.x; e4 < HW / 4; e4 += blockDim.x) {
            const uint4 v = src[e4];
            const u32 vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (u32 t = 0; t < 4; t++) {
                const u32 e = e4 * 4 + t;
                plane[(brv_bits(e >> logW, logH) << logW) + brv_bits(e & (W - 1), logW)] = vals[t];
            }
        }
        __syncthreads();
        ntt2d_plane(plane, logH, logW, inverse != 0, P);
        uint4* dst = reinterpret_cast<uint4*>(X + pl * HW);
        for (u32 e4 = threadIdx.x; e4 < HW / 4; e4 += blockDim.x) {
            uint4 v = reinterpret_cast<const uint4*>(plane)[e4];
            if (inverse) {
                u32 t;
                t = shoup_mul32(v.x, scale, scale_s, P.p); v.x = t >= P.p ? t - P.p : t;
                t = shoup_mul32(v.y, scale, scale_s, P.p); v.y = t >= P.p ? t - P.p : t;
                t = shoup_mul32(v.z, scale, scale_s, P.p); v.z = t >= P.p ? t - P.p : t;
                t = shoup_mul32(v.w, scale, scale_s, P.p); v.w = t >= P.p ? t - P.p : t;
            }
            dst[e4] = v;
        }
        __syncthreads();
    }
}

// H, W >= 8: one CTA of HW/8 threads per plane; coalesced natural-order load,
// radix-8 DIF passes on rows and columns, and a store that reads the
// bit-reversed result back into natural order (scaled for the inverse).
__global__ void __launch_bounds__(512) ntt2d_kernel(DevParams P, u32 logH, u32 logW, const u32* x, u32* X, u64 planes,
                                                    int inverse, u32 scale, u32 scale_s) {
    extern __shared__ u32 plane[];
    const u32 HW = 1u << (logH + logW), W = 1u << logW;
    griddep_release();
    griddep_wait();
    for (u64 pl = blockIdx.x; pl < planes; pl += gridDim.x) {
        const uint4* src = reinterpret_cast<const uint4*>(x + pl * HW);
        for (u32 e4 = threadIdx.x; e4 < HW / 4; e4 += blockDim.x) reinterpret_cast<uint4*>(plane)[e4] = src[e4];
        __syncthreads();
        ntt2d_plane_dif(plane, logH, logW, inverse != 0, P);
        uint4* dst = reinterpret_cast<uint4*>(X + pl * HW);
        for (u32 e4 = threadIdx.x; e4 < HW / 4; e4 += blockDim.x) {
            u32 vals[4];
#pragma unroll
            for (u32 t = 0; t < 4; t++) {
                const u32 e = e4 * 4 + t;
                u32 v = plane[(brv_bits(e >> logW, logH) << logW) + brv_bits(e & (W - 1), logW)];
                if (inverse) {
                    v = shoup_mul32(v, scale, scale_s, P.p);
                    v = v >= P.p ? v - P.p : v;
                }
                vals[t] = v;
            }
            dst[e4] = make_uint4(vals[0], vals[1], vals[2], vals[3]);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- square planes up to 32 x 32
// One warp owns 32/N planes of N x N (N = 8, 16, 32); lane j of a plane
// holds column j in registers, read with coalesced row loads.  Columns, then
// rows, run unrolled radix-2 DIF (Gentleman-Sande) butterflies with lazy
// reduction (only the Shoup products reduce; a final Shoup product by 1 makes
// the words canonical; needs p 2^(2 LOG) < 2^32); the twiddles w_32^k, k < 16, and
// their Shoup companions are kernel parameters, so every multiply takes its
// twiddle straight from the constant bank.  The bit-reversed order the DIF
// leaves is a fixed register permutation, undone while the plane is
// transposed through padded shared memory (conflict-free) between the two
// directions and before the coalesced row stores.
struct Tw32 {
    u32 w[16];   // w_32^k (forward) or w_32^-k (inverse)
    u32 ws[16];  // floor(w 2^32 / p)
};

template <int LOG>
__host__ __device__ constexpr int brv_c(int i) {
    int r = 0;
    for (int b = 0; b < LOG; b++) r |= ((i >> b) & 1) << (LOG - 1 - b);
    return r;
}

__device__ __forceinline__ u32 lazy_mul(u32 x, u32 w, u32 ws, u32 p) {  // x < 2^32 -> [0, 2p)
    return x * w - __umulhi(x, ws) * p;
}
__device__ __forceinline__ u32 sub_if_ge(u32 x, u32 m) {  // x < 2m -> [0, m)
    return min(x, x - m);
}

// Unrolled DIF on N = 2^LOG registers whose values are below p 2^s0.  Sums
// and twiddle-1 differences are not reduced (a level doubles the bound, so
// after both directions of a 32 x 32 plane it is p 2^10 < 2^27); every other
// difference is offset by the level's bound and leaves a lazy Shoup product
// in [0, 2p).  The result is below p 2^(s0 + LOG).
template <int LOG>
__device__ __forceinline__ void dif_regs(u32 (&a)[1 << LOG], u32 p, u32 s0, const Tw32& tw) {
    constexpr int N = 1 << LOG;
#pragma unroll
    for (int len = N / 2, lvl = 0; len >= 1; len >>= 1, lvl++) {
        const u32 bound = p << (s0 + lvl);  // every input of this level is below it
#pragma unroll
        for (int st = 0; st < N; st += 2 * len) {
#pragma unroll
            for (int j = 0; j < len; j++) {
                const u32 u = a[st + j], v = a[st + j + len];
                a[st + j] = u + v;
                const u32 d = u - v + bound;
                const int k = j * (16 / len);  // w_{2 len}^j = w_32^(j 32 / (2 len))
                a[st + j + len] = j == 0 ? d : lazy_mul(d, tw.w[k], tw.ws[k], p);
            }
        }
    }
}

template <int LOG, bool kInv>
__global__ void __launch_bounds__(256, 4) ntt2d_reg_kernel(u32 p, Tw32 tw, u32 scale, u32 scale_s,
                                                        const u32* x, u32* X, u64 planes) {
    // x may equal X: a warp reads its planes whole before it writes them
    constexpr int N = 1 << LOG, PPW = 32 / N, STR = N + 1;
    __shared__ u32 sm[8][PPW * N * STR];
    griddep_release();
    griddep_wait();
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const u32 sub = lane / N, col = lane % N;
    const u32 one_s = (u32)(0x100000000ull / p);  // Shoup companion of 1
    u32* tr = sm[wid] + sub * N * STR;
    const u64 nwarps = (u64)gridDim.x * 8;
    for (u64 g = (u64)blockIdx.x * 8 + wid; g * PPW < planes; g += nwarps) {
        const u64 pl = g * PPW + sub;
        const bool valid = pl < planes;
        const u32* src = x + pl * N * N + col;
        u32 a[N];
#pragma unroll
        for (int r = 0; r < N; r++) a[r] = valid ? src[r * N] : 0u;
        dif_regs<LOG>(a, p, 0, tw);  // column col: a[i] = spectrum at row frequency brv(i), below p 2^LOG
#pragma unroll
        for (int i = 0; i < N; i++) tr[brv_c<LOG>(i) * STR + col] = a[i];
        __syncwarp();
#pragma unroll
        for (int c = 0; c < N; c++) a[c] = tr[col * STR + c];  // row col
        __syncwarp();
        dif_regs<LOG>(a, p, LOG, tw);  // a[i] = X[col][brv(i)], below p 2^(2 LOG)
#pragma unroll
        for (int i = 0; i < N; i++) tr[col * STR + brv_c<LOG>(i)] = a[i];
        __syncwarp();
        u32* dst = X + pl * N * N + col;
#pragma unroll
        for (int r = 0; r < N; r++) {
            u32 v = tr[r * STR + col];
            v = kInv ? lazy_mul(v, scale, scale_s, p) : lazy_mul(v, 1, one_s, p);  // [0, 2p)
            v = sub_if_ge(v, p);
            if (valid) dst[r * N] = v;
        }
        __syncwarp();
    }
}

template <int LOG, bool kInv>
cudaError_t launch_reg(const DevParams& P, const Tw32& tw, u32 scale, u32 scale_s, const u32* x, u32* X, u64 planes,
                       cudaStream_t s) {
    static int per_sm[2] = {0, 0};  // resident CTAs per SM, looked up once per process
    int& occ = per_sm[kInv ? 1 : 0];
    if (occ == 0) {
        int b = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ntt2d_reg_kernel<LOG, kInv>, 256, 0);
        if (e != cudaSuccess) return e;
        occ = b > 0 ? b : 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    constexpr u64 PPW = 32 >> LOG;
    const u64 ctas = (planes + 8 * PPW - 1) / (8 * PPW), cap = (u64)sms * occ;
    return launch_online(ntt2d_reg_kernel<LOG, kInv>, (u32)(ctas < cap ? ctas : cap), 256, 0, s, P.p, tw, scale,
                         scale_s, x, X, planes);
}

cudaError_t launch_ntt2d(const DevParams& P, u32 H, u32 W, const u32* x, u32* X, u64 planes, bool inverse,
                         cudaStream_t s) {
    if (planes == 0) return cudaSuccess;
    const u32 logH = __builtin_ctz(H), logW = __builtin_ctz(W), HW = H * W;
    u32 scale = 1, scale_s = 0;
    if (inverse) {
        scale = fdsc_powmod32(HW % P.p, P.p - 2, P.p);
        scale_s = fdsc_shoup32(scale, P.p);
    }
    if (logH == logW && logH >= 3 && logH <= 5 && (P.p - 1) % 32 == 0 && (u64)P.p << (2 * logH) < (1ull << 32)) {
        Tw32 tw;
        const u32 w32 = fdsc_powmod32(P.g_p, (P.p - 1) / 32, P.p);
        const u32 w = inverse ? fdsc_powmod32(w32, P.p - 2, P.p) : w32;
        u32 t = 1;
        for (int k = 0; k < 16; k++, t = (u32)((u64)t * w % P.p)) {
            tw.w[k] = t;
            tw.ws[k] = fdsc_shoup32(t, P.p);
        }
        if (logH == 5) return inverse ? launch_reg<5, true>(P, tw, scale, scale_s, x, X, planes, s)
                                      : launch_reg<5, false>(P, tw, scale, scale_s, x, X, planes, s);
        if (logH == 4) return inverse ? launch_reg<4, true>(P, tw, scale, scale_s, x, X, planes, s)
                                      : launch_reg<4, false>(P, tw, scale, scale_s, x, X, planes, s);
        return inverse ? launch_reg<3, true>(P, tw, scale, scale_s, x, X, planes, s)
                       : launch_reg<3, false>(P, tw, scale, scale_s, x, X, planes, s);
    }
    const u64 grid = planes < 152ull * 16 ? planes : 152ull * 16;
    if (logH >= 3 && logW >= 3) {
        const u32 threads = HW / 8 < 32 ? 32 : HW / 8;
        return launch_online(ntt2d_kernel, (u32)grid, threads, HW * sizeof(u32), s, P, logH, logW, x, X, planes,
                             inverse ? 1 : 0, scale, scale_s);
    } else {
        u32 threads = HW / 2 < 256 ? HW / 2 : 256;
        if (threads < 32) threads = 32;
        return launch_online(ntt2d_small_kernel, (u32)grid, threads, HW * sizeof(u32), s, P, logH, logW, x, X,
                             planes, inverse ? 1 : 0, scale, scale_s);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- 2 x 2 sum pooling of a share
__global__ void __launch_bounds__(256) pool2x2_kernel(u32 p, u32 H, u32 W, const u32* __restrict__ x,
                                                      u32* __restrict__ y, u64 planes) {
    griddep_release();
    griddep_wait();
    const u32 Wo = W / 2, HWo = (H / 2) * Wo;
    const u64 total = planes * HWo;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (u64)gridDim.x * blockDim.x) {
        const u64 pl = e / HWo;
        const u32 r = (u32)(e % HWo) / Wo, c = (u32)(e % HWo) % Wo;
        const u32* src = x + pl * H * W + (u64)(2 * r) * W + 2 * c;
        u32 a = src[0] + src[1], b = src[W] + src[W + 1];  // each < 2p
        a = a >= p ? a - p : a;
        b = b >= p ? b - p : b;
        a += b;
        y[e] = a >= p ? a - p : a;
    }
}

cudaError_t launch_pool2x2(const DevParams& P, u32 H, u32 W, const u32* x, u32* y, u64 planes, cudaStream_t s) {
    const u64 total = planes * (H / 2) * (W / 2);
    if (total == 0) return cudaSuccess;
    const u64 blocks = (total + 255) / 256, cap = 152ull * 8;
    return launch_online(pool2x2_kernel, (u32)(blocks < cap ? blocks : cap), 256, 0, s, P.p, H, W, x, y, planes);
}
