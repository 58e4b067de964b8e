// crypt.cu -- the per-ciphertext kernels of libfdsc.  Each CTA owns one
// ring element of degree n and walks it through slot packing, the slot
// transform mod p, the lift to Z_q and the negacyclic NTT mod q entirely in
// shared memory, so every ciphertext word is read and written once.
//
//   K9 keygen          Eq. 1 secret t, stored as NTT_q(t)
//   K3 encrypt         Eq. 1 in the NTT_q domain (Sec. 5.1)
//   K6 homrec          Eq. 3 (HomRec): add Bob's encoded share to c1
//   K7 filter_prepare  Fig. 2, Bob's filter: w_hat packed, lifted, NTT_q
//   K8 mask_prepare    Eq. 2 (HomShare) randomness and its NTT_q image
//   K5 decrypt         Sec. 3.1 decryption, slot decode, channel-block fold
#include <map>
#include <mutex>
#include <utility>

#include "modarith.cuh"

namespace {

constexpr u32 kMaxThreads = 512;

// One CTA per ring element: n/8 threads (8 coefficients each in the radix-8
// passes), at least one warp.
inline u32 threads_for(u32 n, u32 hw = 0) {
    u32 t = n / 8 > hw / 8 ? n / 8 : hw / 8;
    return t < 32 ? 32 : t;
}

// Packed input slot: slot s of slot set r of input ciphertext (bb, k, h).
// HW <= S: block s / HW holds image (bb d + r) g_b + blk / g_c and channel
// k g_c + blk % g_c; HW > S: half h of image bb d + r, channel k.
__device__ __forceinline__ u32 input_slot(const DevParams& P, const DevLayer& L, const u32* X, u32 bb, u32 k,
                                          u32 h, u32 r, u32 s) {
    u32 b, ci, f;
    if (L.beta == 1) {
        const u32 blk = s >> (L.logH + L.logW);
        if (blk >= L.g_c * L.g_b) return 0;
        f = s & (L.HW - 1);
        b = (bb * P.d + r) * L.g_b + blk / L.g_c;
        ci = k * L.g_c + blk % L.g_c;
    } else {
        f = h * P.S + s;
        b = bb * P.d + r;
        ci = k;
    }
    if (b >= L.B || ci >= L.Ci) return 0;
    return X[((u64)b * L.Ci + ci) * L.HW + f];
}

__device__ __forceinline__ u64 add_signed_mod_q(u64 v, int e, u64 q) {
    if (e >= 0) return addmod_q(v, (u64)e, q);
    return submod_q(v, (u64)(-e), q);
}

// ---------------------------------------------------------------- keygen
__global__ void __launch_bounds__(kMaxThreads) keygen_kernel(DevParams P, u64 seed, u64* t_hat) {
    extern __shared__ u64 c[];
    const u64 key = stream_key(seed, DOM_T);
    for (u32 i = threadIdx.x; i < P.n; i += blockDim.x) {
        const u32 t3 = (u32)__umul64hi(stream_at(key, i), 3ull);  // {0,1,2} -> t + 1
        c[i] = t3 == 0 ? P.q - 1 : (u64)(t3 - 1);
    }
    __syncthreads();
    ntt_q_fwd8(c, P);
    for (u32 j = threadIdx.x; j < P.n; j += blockDim.x) t_hat[j] = c[j];
}

// ---------------------------------------------------------------- encrypt / homrec
// mode 0: encrypt X into ct; mode 1: HomRec, add the encoding of X to c1.
template <int kMode>
__global__ void __launch_bounds__(kMaxThreads) encode_kernel(DevParams P, DevLayer L, const u64* __restrict__ t_hat,
                                                          const u32* __restrict__ X, u64 seed, u64* ct) {
    extern __shared__ u64 smem[];
    u64* c = smem;                                       // [n]
    u32* slots = reinterpret_cast<u32*>(smem + P.n);     // [n]
    __shared__ u64 cdt[19];
    const u32 u = blockIdx.x;
    const u32 h = u % L.beta, k = (u / L.beta) % L.T, bb = u / (L.beta * L.T);
    griddep_release();
    griddep_wait();
    if (kMode == 0 && threadIdx.x < 19) cdt[threadIdx.x] = P.cdt[threadIdx.x];
    for (u32 sg = threadIdx.x; sg < P.n; sg += blockDim.x)
        slots[sg] = input_slot(P, L, X, bb, k, h, sg >> P.logS, sg & (P.S - 1));
    __syncthreads();
    ntt_p_inv8(slots, P.d, P);  // slot encode, per slot set
    const u64 keyE = stream_key(seed, DOM_E);
    for (u32 sg = threadIdx.x; sg < P.n; sg += blockDim.x) {
        const u32 r = sg >> P.logS, i = sg & (P.S - 1), coef = r + P.d * i;
        u64 v = P.delta * slots[sg];  // < q since slots < p
        if (kMode == 0) v = add_signed_mod_q(v, gauss_sample(stream_at(keyE, (u64)u * P.n + coef), cdt), P.q);
        c[coef] = v;
    }
    __syncthreads();
    ntt_q_fwd8(c, P);
    u64* c0 = ct + (u64)u * 2 * P.n;
    u64* c1 = c0 + P.n;
    if (kMode == 0) {
        const u64 keyA = stream_key(seed, DOM_A);
        for (u32 j = threadIdx.x; j < P.n; j += blockDim.x) {
            const u64 idx = 2 * ((u64)u * P.n + j);
            const u64 a = uniform_q(stream_at(keyA, idx), stream_at(keyA, idx + 1), P.q);
            c0[j] = a ? P.q - a : 0;
            c1[j] = muladd_q(a, t_hat[j], c[j], P);
        }
    } else {
        for (u32 j = threadIdx.x; j < P.n; j += blockDim.x) c1[j] = addmod_q(c1[j], c[j], P.q);
    }
}

// ---------------------------------------------------------------- filter prepare
// One CTA per filter plaintext (co, k, h).  The channel spectra it needs are
// computed here with the shared NTT2D plane routine.
__global__ void __launch_bounds__(kMaxThreads) filter_kernel(DevParams P, DevLayer L, const int8_t* __restrict__ w,
                                                          u32 fh, u32 fw, u64* __restrict__ Phat) {
    extern __shared__ u64 smem[];
    const u32 cbytes = P.n * 8, pbytes = L.HW * 4;
    u64* c = smem;                                        // [n]       (aliases plane)
    u32* plane = reinterpret_cast<u32*>(smem);            // [HW]
    u32* slots = reinterpret_cast<u32*>(reinterpret_cast<unsigned char*>(smem) + (cbytes > pbytes ? cbytes : pbytes));
    const u32 v = blockIdx.x;
    const u32 h = v % L.beta, k = (v / L.beta) % L.T, co = v / (L.beta * L.T);
    for (u32 s = threadIdx.x; s < P.S; s += blockDim.x) slots[s] = 0;
    const u32 nch = L.beta == 1 ? L.g_c : 1;
    for (u32 ic = 0; ic < nch; ic++) {
        const u32 ci = L.beta == 1 ? k * L.g_c + ic : k;
        if (ci >= L.Ci) break;
        __syncthreads();
        for (u32 e = threadIdx.x; e < L.HW; e += blockDim.x) plane[e] = 0;
        __syncthreads();
        // DIF (natural in, both axes bit-reversed out) when the plane allows
        // radix-8 lines; otherwise bit-reversed in, natural out.
        const bool dif = L.logH >= 3 && L.logW >= 3;
        const int8_t* wf = w + ((u64)co * L.Ci + ci) * fh * fw;
        for (u32 e = threadIdx.x; e < fh * fw; e += blockDim.x) {
            const u32 a = e / fw, b = e % fw;
            const int wv = wf[e];
            const u32 pos = dif ? (a << L.logW) + b : (brv_bits(a, L.logH) << L.logW) + brv_bits(b, L.logW);
            plane[pos] = (u32)(wv < 0 ? (int)P.p + wv : wv);
        }
        __syncthreads();
        if (dif) ntt2d_plane_dif(plane, L.logH, L.logW, false, P);
        else ntt2d_plane(plane, L.logH, L.logW, false, P);
        auto at = [&](u32 f) {
            return dif ? plane[(brv_bits(f >> L.logW, L.logH) << L.logW) + brv_bits(f & (L.W - 1), L.logW)] : plane[f];
        };
        if (L.beta == 1) {
            for (u32 e = threadIdx.x; e < L.g_b * L.HW; e += blockDim.x) {
                const u32 ib = e >> (L.logH + L.logW), f = e & (L.HW - 1);
                slots[(ib * L.g_c + ic) * L.HW + f] = at(f);
            }
        } else {
            for (u32 s = threadIdx.x; s < P.S; s += blockDim.x) slots[s] = at(h * P.S + s);
        }
    }
    __syncthreads();
    ntt_p_inv8(slots, 1, P);
    for (u32 j = threadIdx.x; j < P.n; j += blockDim.x) c[j] = 0;
    __syncthreads();
    for (u32 i = threadIdx.x; i < P.S; i += blockDim.x) {
        const u32 m = slots[i];
        c[(u64)P.d * i] = m <= (P.p - 1) / 2 ? (u64)m : P.q - (P.p - m);  // centred lift
    }
    __syncthreads();
    ntt_q_fwd8(c, P);
    // w(x) = w_0(x^d): the d consecutive evaluation indices of one group
    // (the points x times the d-th roots of unity) share one value, stored once
    const u32 nd = P.n / P.d;
    u64* out = Phat + (u64)v * nd;
    for (u32 i = threadIdx.x; i < nd; i += blockDim.x) out[i] = c[(u64)i * P.d];
}

// ---------------------------------------------------------------- mask prepare
__device__ __forceinline__ u32 mask_value(const DevParams& P, const DevLayer& L, u64 kMask, u64 kSplit, u32 b,
                                          u32 co, u32 ic, u32 f) {
    const u64 base = (u64)b * L.Co + co;
    if (ic > 0) return uniform_p(stream_at(kSplit, (base * L.g_c + ic) * L.HW + f), P.p);
    u32 v = uniform_p(stream_at(kMask, base * L.HW + f), P.p);
    for (u32 j = 1; j < L.g_c; j++)
        v = submod_p(v, uniform_p(stream_at(kSplit, (base * L.g_c + j) * L.HW + f), P.p), P.p);
    return v;
}

// seeds == nullptr: one seed for the call, randomness indexed by the global
// image number.  Otherwise image group bb draws from seeds[bb] with images
// numbered from 0 inside the group, exactly as if it were a call of its own.
__global__ void __launch_bounds__(kMaxThreads) mask_kernel(DevParams P, DevLayer L, u64 seed,
                                                        const u64* __restrict__ seeds, u32 flood_bits,
                                                        u64* __restrict__ Mhat, u32* __restrict__ sB) {
    extern __shared__ u64 smem[];
    u64* c = smem;
    u32* slots = reinterpret_cast<u32*>(smem + P.n);
    const u32 v = blockIdx.x;
    const u32 h = v % L.beta, co = (v / L.beta) % L.Co, bb = v / (L.beta * L.Co);
    const u32 b_off = seeds ? bb * P.d * L.g_b : 0;  // first image of the group, for indexing randomness
    griddep_release();
    griddep_wait();
    if (seeds) seed = seeds[bb];
    const u64 kMask = stream_key(seed, DOM_MASK), kSplit = stream_key(seed, DOM_MASK_SPLIT);
    for (u32 sg = threadIdx.x; sg < P.n; sg += blockDim.x) {
        const u32 r = sg >> P.logS, s = sg & (P.S - 1);
        u32 val = 0;
        if (L.beta == 1) {
            const u32 blk = s >> (L.logH + L.logW);
            if (blk < L.g_c * L.g_b) {
                const u32 ic = blk % L.g_c, f = s & (L.HW - 1);
                const u32 b = (bb * P.d + r) * L.g_b + blk / L.g_c;
                if (b < L.B) {
                    const u32 br = b - b_off;
                    val = mask_value(P, L, kMask, kSplit, br, co, ic, f);
                    if (ic == 0)
                        sB[((u64)b * L.Co + co) * L.HW + f] =
                            uniform_p(stream_at(kMask, ((u64)br * L.Co + co) * L.HW + f), P.p);
                }
            }
        } else {
            const u32 b = bb * P.d + r, f = h * P.S + s;
            if (b < L.B) {
                val = uniform_p(stream_at(kMask, ((u64)(b - b_off) * L.Co + co) * L.HW + f), P.p);
                sB[((u64)b * L.Co + co) * L.HW + f] = val;
            }
        }
        slots[sg] = val;
    }
    __syncthreads();
    ntt_p_inv8(slots, P.d, P);
    // noise flooding: coefficient i of mask ciphertext v carries an error
    // uniform in [-2^f, 2^f), from the top f + 1 bits of its random word
    const u64 kFlood = stream_key(seed, DOM_FLOOD);
    for (u32 sg = threadIdx.x; sg < P.n; sg += blockDim.x) {
        const u32 r = sg >> P.logS, i = sg & (P.S - 1), coef = r + P.d * i;
        u64 m = P.delta * slots[sg];
        if (flood_bits) {
            const u64 t = stream_at(kFlood, (u64)v * P.n + coef) >> (63 - flood_bits), half = 1ull << flood_bits;
            m = t >= half ? addmod_q(m, t - half, P.q) : submod_q(m, half - t, P.q);
        }
        c[coef] = m;
    }
    __syncthreads();
    ntt_q_fwd8(c, P);
    u64* out = Mhat + (u64)v * P.n;
    for (u32 j = threadIdx.x; j < P.n; j += blockDim.x) out[j] = c[j];
}

// ---------------------------------------------------------------- decrypt
__global__ void __launch_bounds__(kMaxThreads) decrypt_kernel(DevParams P, DevLayer L, const u64* __restrict__ t_hat,
                                                           const u64* __restrict__ ct, u32* __restrict__ SA) {
    extern __shared__ u64 smem[];
    u64* c = smem;
    u32* slots = reinterpret_cast<u32*>(smem + P.n);
    const u32 v = blockIdx.x;
    const u32 h = v % L.beta, co = (v / L.beta) % L.Co, bb = v / (L.beta * L.Co);
    const u64* c0 = ct + (u64)v * 2 * P.n;
    const u64* c1 = c0 + P.n;
    griddep_release();
    griddep_wait();
    for (u32 j = threadIdx.x; j < P.n; j += blockDim.x) c[j] = muladd_q(c0[j], t_hat[j], c1[j], P);
    __syncthreads();
    ntt_q_inv8(c, P);
    for (u32 coef = threadIdx.x; coef < P.n; coef += blockDim.x) {
        const u32 r = coef & (P.d - 1), i = coef / P.d;
        slots[r * P.S + i] = round_pq(c[coef], P);
    }
    __syncthreads();
    ntt_p_fwd8(slots, P.d, P);  // slot decode
    if (L.beta == 1) {
        const u32 per_set = L.g_b * L.HW;
        for (u32 e = threadIdx.x; e < P.d * per_set; e += blockDim.x) {
            const u32 r = e / per_set, rem = e % per_set;
            const u32 ib = rem >> (L.logH + L.logW), f = rem & (L.HW - 1);
            const u32 b = (bb * P.d + r) * L.g_b + ib;
            if (b >= L.B) continue;
            u32 acc = 0;
            for (u32 ic = 0; ic < L.g_c; ic++) acc = addmod_p(acc, slots[r * P.S + (ib * L.g_c + ic) * L.HW + f], P.p);
            SA[((u64)b * L.Co + co) * L.HW + f] = acc;
        }
    } else {
        for (u32 sg = threadIdx.x; sg < P.n; sg += blockDim.x) {
            const u32 r = sg >> P.logS, s = sg & (P.S - 1), b = bb * P.d + r;
            if (b < L.B) SA[((u64)b * L.Co + co) * L.HW + h * P.S + s] = slots[sg];
        }
    }
}

// Opt a kernel in to more than the default 48 KiB of dynamic shared memory
// (leaving room for its static shared arrays); done once per kernel and size.
template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes + 1024 <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = done[{reinterpret_cast<const void*>(kernel), dev}];
    if (have >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

}  // namespace

cudaError_t launch_keygen(const DevParams& P, u64 seed, u64* t_hat, cudaStream_t s) {
    const size_t sm = (size_t)P.n * 8;
    cudaError_t e = set_smem(keygen_kernel, sm);
    if (e != cudaSuccess) return e;
    keygen_kernel<<<1, threads_for(P.n), sm, s>>>(P, seed, t_hat);
    return cudaGetLastError();
}

cudaError_t launch_encrypt(const DevParams& P, const DevLayer& L, const u64* t_hat, const u32* X, u64 seed, u64* ct,
                           cudaStream_t s) {
    const size_t sm = (size_t)P.n * 12;
    cudaError_t e = set_smem(encode_kernel<0>, sm);
    if (e != cudaSuccess) return e;
    return launch_online(encode_kernel<0>, L.n_in, threads_for(P.n), sm, s, P, L, t_hat, X, seed, ct);
}

cudaError_t launch_homrec(const DevParams& P, const DevLayer& L, const u32* XB, u64* ct, cudaStream_t s) {
    const size_t sm = (size_t)P.n * 12;
    cudaError_t e = set_smem(encode_kernel<1>, sm);
    if (e != cudaSuccess) return e;
    return launch_online(encode_kernel<1>, L.n_in, threads_for(P.n), sm, s, P, L, (const u64*)nullptr, XB, (u64)0, ct);
}

cudaError_t launch_filter_prepare(const DevParams& P, const DevLayer& L, const int8_t* w, u32 fh, u32 fw, u64* Phat,
                                  cudaStream_t s) {
    const size_t cb = (size_t)P.n * 8, pb = (size_t)L.HW * 4;
    const size_t sm = (cb > pb ? cb : pb) + (size_t)P.S * 4;
    cudaError_t e = set_smem(filter_kernel, sm);
    if (e != cudaSuccess) return e;
    const u32 grid = L.Co * L.T * L.beta;
    filter_kernel<<<grid, threads_for(P.n, L.HW), sm, s>>>(P, L, w, fh, fw, Phat);
    return cudaGetLastError();
}

cudaError_t launch_mask_prepare(const DevParams& P, const DevLayer& L, u64 seed, const u64* seeds, u32 flood_bits, u64* Mhat, u32* sB,
                                cudaStream_t s) {
    const size_t sm = (size_t)P.n * 12;
    cudaError_t e = set_smem(mask_kernel, sm);
    if (e != cudaSuccess) return e;
    return launch_online(mask_kernel, L.n_out, threads_for(P.n), sm, s, P, L, seed, seeds, flood_bits, Mhat, sB);
}

cudaError_t launch_decrypt(const DevParams& P, const DevLayer& L, const u64* t_hat, const u64* ct, u32* SA,
                           cudaStream_t s) {
    const size_t sm = (size_t)P.n * 12;
    cudaError_t e = set_smem(decrypt_kernel, sm);
    if (e != cudaSuccess) return e;
    return launch_online(decrypt_kernel, L.n_out, threads_for(P.n), sm, s, P, L, t_hat, ct, SA);
}
