// pipeline.cu -- the fused kernels of one online FDSC layer (Fig. 2), split
// so that the input-independent work runs concurrently with the rest:
//
//   constants_kernel   Eq. 1 with a zero message: ct = (-a_hat,
//                      a_hat o t_hat + NTT_q(e)) -- Sec. 5.1's RLWE
//                      constants, needing no user input;
//   share_kernel       a spatial share x (Alice's u or Bob's s_B) through
//                      NTT2D -> flatten/pack -> slot encode -> x Delta ->
//                      NTT_q: the plaintext that encryption (Eq. 1) or
//                      HomRec (Eq. 3) adds to c1;
//   decrypt_share      decryption, slot decode, channel-block fold and
//                      INTT2D in one pass: ct -> Alice's spatial share s_A.
//
// Because NTT_q is linear, Enc(m) = constants + (0, NTT_q(Delta m)) and
// HomRec adds (0, NTT_q(Delta m_B)): the composed ciphertext is word for word
// the one the one-shot entry points produce.  Each CTA owns one ring element
// and keeps it in shared memory; the twiddle tables it needs are staged into
// shared memory with asynchronous copies issued before the first global load
// of its data, so their latency overlaps.
#include "modarith.cuh"

namespace {

constexpr u32 kMaxThreads = 512;

inline u32 threads_for(u32 n) { return n / 8 < 32 ? 32 : n / 8; }

// Compact table of w_L^k, k < L/2, L = max(H, W) (a strided gather of the
// params' w_lmax table), loaded with plain loads.
__device__ __forceinline__ void load_line_table(u32* tw, u32* tws, u32 logT, bool inverse, const DevParams& P) {
    const u32* g = inverse ? P.w2di : P.w2d;
    const u32* gs = inverse ? P.w2di_s : P.w2d_s;
    const u32 half = 1u << (logT - 1), sh = P.loglmax - logT;
    for (u32 k = threadIdx.x; k < half; k += blockDim.x) {
        tw[k] = __ldg(g + (k << sh));
        tws[k] = __ldg(gs + (k << sh));
    }
}

// ---------------------------------------------------------------- encryption constants
__global__ void __launch_bounds__(kMaxThreads) constants_kernel(DevParams P, const u64* __restrict__ t_hat, u64 seed,
                                                                u64* __restrict__ ct) {
    extern __shared__ __align__(16) unsigned char sm[];
    const u32 n = P.n;
    u64* tq = reinterpret_cast<u64*>(sm);  // [n] psi^brv
    u64* tqs = tq + n;                     // [n]
    u64* c = tqs + n;                      // [n]
    __shared__ u64 cdt[19];
    stage_async(tq, P.qfw, n * 8);
    stage_async(tqs, P.qfw_s, n * 8);
    if (threadIdx.x < 19) cdt[threadIdx.x] = P.cdt[threadIdx.x];
    __syncthreads();
    const u32 u = blockIdx.x;
    const u64 keyE = stream_key(seed, DOM_E);
    for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
        const int e = gauss_sample(stream_at(keyE, (u64)u * n + i), cdt);
        c[i] = e >= 0 ? (u64)e : P.q - (u64)(-e);
    }
    stage_wait();
    ntt_fwd_r8<u64>(c, P.logn, 1, tq, tqs, P);
    const u64 keyA = stream_key(seed, DOM_A);
    u64* c0 = ct + (u64)u * 2 * n;
    u64* c1 = c0 + n;
    for (u32 j = threadIdx.x; j < n; j += blockDim.x) {
        const u64 idx = 2 * ((u64)u * n + j);
        const u64 a = uniform_q(stream_at(keyA, idx), stream_at(keyA, idx + 1), P.q);
        c0[j] = a ? P.q - a : 0;
        c1[j] = addmod_q(mulmod_q(a, __ldg(t_hat + j), P), c[j], P.q);
    }
}

// ---------------------------------------------------------------- share encoding
// One CTA per input ciphertext u = (bb, k) (beta = 1).  kMode 0: write
// A[u] = NTT_q(Delta m); kMode 1: add it to ct[u].c1.
template <int kMode>
__global__ void __launch_bounds__(kMaxThreads) share_kernel(DevParams P, DevLayer L, const u32* __restrict__ x,
                                                            u64* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    const u32 n = P.n, S = P.S;
    u64* tq = reinterpret_cast<u64*>(sm);
    u64* tqs = tq + n;
    u64* c = tqs + n;
    u32* tp = reinterpret_cast<u32*>(c + n);  // [S] psi_p^-brv
    u32* tps = tp + S;
    u32* slots = tps + S;                       // [n] = d slot sets
    u32* t2 = slots + n;                        // [T/2] line twiddles
    const u32 logT = L.logH > L.logW ? L.logH : L.logW;
    u32* t2s = t2 + (1u << (logT - 1));
    stage_async(tq, P.qfw, n * 8);
    stage_async(tqs, P.qfw_s, n * 8);
    stage_async(tp, P.pinv, S * 4);
    stage_async(tps, P.pinv_s, S * 4);
    load_line_table(t2, t2s, logT, false, P);

    const u32 u = blockIdx.x, k = u % L.T, bb = u / L.T;
    const u32 HW = L.HW, logHW = L.logH + L.logW, blocks = L.g_c * L.g_b;
    // planes of the packed slot vector, loaded in bit-reversed order along both axes
    for (u32 e = threadIdx.x; e < n; e += blockDim.x) {
        const u32 r = e >> P.logS, s = e & (S - 1), blk = s >> logHW, f = s & (HW - 1);
        u32 v = 0;
        if (blk < blocks) {
            const u32 b = (bb * P.d + r) * L.g_b + blk / L.g_c, ci = k * L.g_c + blk % L.g_c;
            if (b < L.B && ci < L.Ci) v = __ldg(x + ((u64)b * L.Ci + ci) * HW + f);
        }
        const u32 pos = (e & ~(HW - 1)) + (brv_bits(f >> L.logW, L.logH) << L.logW) + brv_bits(f & (L.W - 1), L.logW);
        slots[pos] = v;
    }
    __syncthreads();
    // NTT2D of every plane (zero planes included): rows, then columns
    lines_r8<false>(slots, n >> logHW, true, L.logH, L.logW, t2, t2s, logT, P.p);
    lines_r8<false>(slots, n >> logHW, false, L.logH, L.logW, t2, t2s, logT, P.p);
    stage_wait();
    ntt_inv_r8<u32>(slots, P.logS, P.d, tp, tps, P.Sinv, P.Sinv_s, P);  // slot encode
    for (u32 e = threadIdx.x; e < n; e += blockDim.x) {
        const u32 r = e >> P.logS, i = e & (S - 1);
        c[r + P.d * i] = P.delta * slots[e];
    }
    __syncthreads();
    ntt_fwd_r8<u64>(c, P.logn, 1, tq, tqs, P);
    if (kMode == 0) {
        u64* A = out + (u64)u * n;
        for (u32 j = threadIdx.x; j < n; j += blockDim.x) A[j] = c[j];
    } else {
        u64* c1 = out + (u64)u * 2 * n + n;
        for (u32 j = threadIdx.x; j < n; j += blockDim.x) c1[j] = addmod_q(c1[j], c[j], P.q);
    }
}

// ---------------------------------------------------------------- decrypt + fold + INTT2D
__device__ __forceinline__ u32 round_pq2(u64 v, const DevParams& P) {
    u64 z = __umul64hi(v, P.round_k);
    const unsigned __int128 num = (unsigned __int128)(2ull * P.p) * v + P.q;
    const unsigned __int128 q2 = (unsigned __int128)2 * P.q;
#pragma unroll
    for (int it = 0; it < 3; it++)
        if (q2 * (z + 1) <= num) z++;
    return (u32)(z >= P.p ? z - P.p : z);
}

__global__ void __launch_bounds__(kMaxThreads) decrypt_share_kernel(DevParams P, DevLayer L, const u64* __restrict__ t_hat,
                                                                    const u64* __restrict__ ct, u32* __restrict__ y,
                                                                    u32 scale, u32 scale_s) {
    extern __shared__ __align__(16) unsigned char sm[];
    const u32 n = P.n, S = P.S;
    u64* tq = reinterpret_cast<u64*>(sm);
    u64* tqs = tq + n;
    u64* c = tqs + n;
    u32* tp = reinterpret_cast<u32*>(c + n);
    u32* tps = tp + S;
    u32* slots = tps + S;
    u32* planes = slots + n;                    // [d g_b HW]
    const u32 logT = L.logH > L.logW ? L.logH : L.logW;
    const u32 HW = L.HW, logHW = L.logH + L.logW;
    const u32 nplanes = P.d * L.g_b;
    u32* t2 = planes + nplanes * HW;
    u32* t2s = t2 + (1u << (logT - 1));
    stage_async(tq, P.qinv, n * 8);
    stage_async(tqs, P.qinv_s, n * 8);
    stage_async(tp, P.pfw, S * 4);
    stage_async(tps, P.pfw_s, S * 4);
    load_line_table(t2, t2s, logT, true, P);

    const u32 v = blockIdx.x, co = v % L.Co, bb = v / L.Co;
    const u64* c0 = ct + (u64)v * 2 * n;
    const u64* c1 = c0 + n;
    for (u32 j = threadIdx.x; j < n; j += blockDim.x)
        c[j] = addmod_q(mulmod_q(__ldg(c0 + j), __ldg(t_hat + j), P), __ldg(c1 + j), P.q);
    stage_wait();
    ntt_inv_r8<u64>(c, P.logn, 1, tq, tqs, P.ninv, P.ninv_s, P);
    for (u32 coef = threadIdx.x; coef < n; coef += blockDim.x) {
        const u32 r = coef & (P.d - 1), i = coef / P.d;
        slots[r * S + i] = round_pq2(c[coef], P);
    }
    __syncthreads();
    ntt_fwd_r8<u32>(slots, P.logS, P.d, tp, tps, P);  // slot decode
    // fold the g_c channel blocks of every image block: plane (r, ib)
    for (u32 e = threadIdx.x; e < nplanes * HW; e += blockDim.x) {
        const u32 pl = e >> logHW, f = e & (HW - 1), r = pl / L.g_b, ib = pl % L.g_b;
        const u32* src = slots + r * S + ib * L.g_c * HW + f;
        u32 acc = 0;
        for (u32 ic = 0; ic < L.g_c; ic++) acc = addmod_p(acc, src[ic * HW], P.p);
        planes[e] = acc;
    }
    __syncthreads();
    lines_r8<true>(planes, nplanes, true, L.logH, L.logW, t2, t2s, logT, P.p);
    lines_r8<true>(planes, nplanes, false, L.logH, L.logW, t2, t2s, logT, P.p);
    for (u32 e = threadIdx.x; e < nplanes * HW; e += blockDim.x) {
        const u32 pl = e >> logHW, f = e & (HW - 1), r = pl / L.g_b, ib = pl % L.g_b;
        const u32 b = (bb * P.d + r) * L.g_b + ib;
        if (b >= L.B) continue;
        u32 val = planes[(pl << logHW) + (brv_bits(f >> L.logW, L.logH) << L.logW) + brv_bits(f & (L.W - 1), L.logW)];
        val = shoup_mul32(val, scale, scale_s, P.p);
        y[((u64)b * L.Co + co) * HW + f] = val >= P.p ? val - P.p : val;
    }
}

template <typename K>
cudaError_t opt_in(K kernel, size_t bytes) {
    if (bytes + 1024 <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

u32 line_log(const DevLayer& L) { return L.logH > L.logW ? L.logH : L.logW; }

}  // namespace

size_t share_smem_bytes(const DevParams& P, const DevLayer& L) {
    return (size_t)P.n * 8 * 3 + (size_t)P.S * 8 + (size_t)P.n * 4 + (size_t)8 * (1u << (line_log(L) - 1));
}
size_t decrypt_share_smem_bytes(const DevParams& P, const DevLayer& L) {
    return (size_t)P.n * 8 * 3 + (size_t)P.S * 8 + (size_t)P.n * 4 + (size_t)P.d * L.g_b * L.HW * 4 +
           (size_t)8 * (1u << (line_log(L) - 1));
}
size_t constants_smem_bytes(const DevParams& P) { return (size_t)P.n * 24; }

cudaError_t launch_constants(const DevParams& P, const DevLayer& L, const u64* t_hat, u64 seed, u64* ct,
                             cudaStream_t s) {
    const size_t sm = constants_smem_bytes(P);
    cudaError_t e = opt_in(constants_kernel, sm);
    if (e != cudaSuccess) return e;
    constants_kernel<<<L.n_in, threads_for(P.n), sm, s>>>(P, t_hat, seed, ct);
    return cudaGetLastError();
}

cudaError_t launch_share(const DevParams& P, const DevLayer& L, const u32* x, u64* out, bool add_to_ct,
                         cudaStream_t s) {
    const size_t sm = share_smem_bytes(P, L);
    cudaError_t e = add_to_ct ? opt_in(share_kernel<1>, sm) : opt_in(share_kernel<0>, sm);
    if (e != cudaSuccess) return e;
    if (add_to_ct) share_kernel<1><<<L.n_in, threads_for(P.n), sm, s>>>(P, L, x, out);
    else share_kernel<0><<<L.n_in, threads_for(P.n), sm, s>>>(P, L, x, out);
    return cudaGetLastError();
}

cudaError_t launch_decrypt_share(const DevParams& P, const DevLayer& L, const u64* t_hat, const u64* ct, u32* y,
                                 cudaStream_t s) {
    const size_t sm = decrypt_share_smem_bytes(P, L);
    cudaError_t e = opt_in(decrypt_share_kernel, sm);
    if (e != cudaSuccess) return e;
    const u32 scale = fdsc_powmod32(L.HW % P.p, P.p - 2, P.p);
    decrypt_share_kernel<<<L.n_out, threads_for(P.n), sm, s>>>(P, L, t_hat, ct, y, scale, fdsc_shoup32(scale, P.p));
    return cudaGetLastError();
}
