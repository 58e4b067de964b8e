// ntt2d.cu -- K1 / K2: batched cyclic NTT2D / INTT2D mod p over padded
// H x W planes (Eq. 12 in two dimensions; Fig. 2 lines 1, 6, 9).
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

cudaError_t launch_ntt2d(const DevParams& P, u32 H, u32 W, const u32* x, u32* X, u64 planes, bool inverse,
                         cudaStream_t s) {
    if (planes == 0) return cudaSuccess;
    const u32 logH = __builtin_ctz(H), logW = __builtin_ctz(W), HW = H * W;
    u32 scale = 1, scale_s = 0;
    if (inverse) {
        scale = fdsc_powmod32(HW % P.p, P.p - 2, P.p);
        scale_s = fdsc_shoup32(scale, P.p);
    }
    const u64 grid = planes < 152ull * 16 ? planes : 152ull * 16;
    if (logH >= 3 && logW >= 3) {
        const u32 threads = HW / 8 < 32 ? 32 : HW / 8;
        ntt2d_kernel<<<(u32)grid, threads, HW * sizeof(u32), s>>>(P, logH, logW, x, X, planes, inverse ? 1 : 0,
                                                                  scale, scale_s);
    } else {
        u32 threads = HW / 2 < 256 ? HW / 2 : 256;
        if (threads < 32) threads = 32;
        ntt2d_small_kernel<<<(u32)grid, threads, HW * sizeof(u32), s>>>(P, logH, logW, x, X, planes,
                                                                        inverse ? 1 : 0, scale, scale_s);
    }
    return cudaGetLastError();
}
