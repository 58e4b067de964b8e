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
//                      INTT2D in one pass: ct -> Alice's spatial share s_A;
//   decrypt_share_pair the same for a single image on a cluster of two CTAs
//                      per ciphertext, one coefficient parity each.
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

// The NTT_q twiddle pairs (16 n bytes) are staged in shared memory up to
// n = 2048; at n = 4096 the kernels are instantiated with kGTw = true and read
// them from global memory (L1-resident after the first pass), so that two
// CTAs fit on an SM.
inline bool global_qtw(u32 n) { return n > 2048; }
inline u32 qtw_entries(u32 n) { return global_qtw(n) ? 0u : n; }

// ---------------------------------------------------------------- L2 prefetch of a later kernel's operands
// Up to two device ranges (16-byte aligned, whole multiples of 16 bytes)
// split evenly over `slices` CTAs; the CTA `slice` asks the L2 cache for its
// part in 4 KiB bulk prefetches (no data reaches the SM).
struct L2Prefetch {
    const void* p[2];
    u64 bytes[2];
    u32 slice, slices;
    __device__ __forceinline__ void issue() const {
        constexpr u64 kChunk = 4096;
        for (int r = 0; r < 2; r++) {
            if (!p[r] || !bytes[r] || !slices) continue;
            const u64 chunks = (bytes[r] + kChunk - 1) / kChunk;
            const u64 c0 = chunks * slice / slices, c1 = chunks * (slice + 1) / slices;
            for (u64 c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
                const u64 off = c * kChunk, len = bytes[r] - off < kChunk ? bytes[r] - off : kChunk;
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const char*>(p[r]) + off),
                             "r"((u32)len)
                             : "memory");
            }
        }
    }
};

// ---------------------------------------------------------------- encryption constants
// Image group g = u / per_group uses the key t_hat + g key_stride; with
// seeds != nullptr it draws from seeds[g] with ciphertexts numbered from 0
// inside the group (as if it were a call of its own).
// c1_only: write c1 alone ([n_in][n]; the seeded form, c0 = -a being
// recomputable from the seed).
// The work of ciphertext u (one CTA); sm: constants_smem_bytes of dynamic
// shared memory.
template <bool kGTw>
__device__ __forceinline__ void constants_body(unsigned char* sm, const DevParams& P, const u64* __restrict__ t_hat,
                                               u64 key_stride, u32 per_group, u64 seed,
                                               const u64* __restrict__ seeds, u64* __restrict__ ct, int c1_only,
                                               u32 u, const L2Prefetch* pf = nullptr) {
    const u32 n = P.n;
    ulonglong2* tq_s = reinterpret_cast<ulonglong2*>(sm);  // [n] (psi^brv, companion), unless kGTw
    u64* c = reinterpret_cast<u64*>(tq_s + (kGTw ? 0 : n));  // padded [n]
    u64* key = c + padded_len(n);                        // [n], the key's NTT_q words
    const ulonglong2* tq = kGTw ? P.qfw2 : tq_s;
    __shared__ u64 cdt[19];
    const u32 grp = u / per_group;
    stage_async(tq_s, P.qfw2, kGTw ? 0 : n * 16);
    if (threadIdx.x < 19) cdt[threadIdx.x] = P.cdt[threadIdx.x];
    __syncthreads();
    const u32 ur = seeds ? u - grp * per_group : u;  // ciphertext number for the randomness
    if (seeds) {
        griddep_wait();
        seed = seeds[grp];
    }
    // NTT_q(e) needs the seed alone: it runs while the previous kernel finishes
    // The same discrete Gaussian as gauss_sample (sign bit 63, magnitude = the
    // table entries the low 63 bits reach), eight coefficients at a time, so
    // that each table entry is read from shared memory once per eight draws
    const u64 keyE = stream_key(seed, DOM_E);
    for (u32 i0 = 0; i0 < n; i0 += 8 * blockDim.x) {
        u64 r[8];
        int a[8];
#pragma unroll
        for (int t = 0; t < 8; t++) {
            r[t] = stream_at(keyE, (u64)ur * n + i0 + threadIdx.x + (u32)t * blockDim.x);
            a[t] = 0;
        }
#pragma unroll
        for (int kk = 0; kk < 19; kk++) {
            const u64 ck = cdt[kk];
#pragma unroll
            for (int t = 0; t < 8; t++) a[t] += ((r[t] & 0x7FFFFFFFFFFFFFFFull) >= ck);
        }
#pragma unroll
        for (int t = 0; t < 8; t++) {
            const u32 i = i0 + threadIdx.x + (u32)t * blockDim.x;
            if (i < n) c[padx(i)] = (r[t] >> 63) ? (a[t] ? P.q - (u64)a[t] : 0) : (u64)a[t];
        }
    }
    stage_wait();
    if (pf) pf->issue();
    ntt_r8p<true, u64>(c, P.logn, 1, tq, 0, 0, P);
    if (!seeds) griddep_wait();
    stage_async(key, t_hat + (u64)grp * key_stride, n * 8);
    const u64 keyA = stream_key(seed, DOM_A);
    u64* c0 = ct + (u64)u * 2 * n;
    u64* c1 = c1_only ? ct + (u64)u * n : c0 + n;
    // c0 = -a while the key arrives; a stays in registers for c1
    for (u32 j0 = 0; j0 < n; j0 += 8 * blockDim.x) {
        u64 a[8];
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const u32 j = j0 + threadIdx.x + (u32)r * blockDim.x;
            if (j < n) {
                const u64 idx = 2 * ((u64)ur * n + j);
                a[r] = uniform_q(stream_at(keyA, idx), stream_at(keyA, idx + 1), P.q);
                if (!c1_only) c0[j] = a[r] ? P.q - a[r] : 0;
            }
        }
        stage_wait();
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const u32 j = j0 + threadIdx.x + (u32)r * blockDim.x;
            if (j < n) c1[j] = muladd_q(a[r], key[j], c[padx(j)], P);
        }
    }
}

template <bool kGTw>
__global__ void __launch_bounds__(kMaxThreads) constants_kernel(DevParams P, const u64* __restrict__ t_hat, u64 key_stride,
                                                                u32 per_group, u64 seed, const u64* __restrict__ seeds,
                                                                u64* __restrict__ ct, int c1_only) {
    extern __shared__ __align__(16) unsigned char sm[];
    griddep_release();
    constants_body<kGTw>(sm, P, t_hat, key_stride, per_group, seed, seeds, ct, c1_only, blockIdx.x);
}

// ---------------------------------------------------------------- slot encode fused with the lift
// The slot encode of the d slot sets in `a` (bit-reversed in, natural out,
// times S^-1: the radix-8 passes of ntt_r8p) whose last pass, instead of
// storing the slots, writes coefficient i of slot set r straight into the
// NTT_q input as c[r + d i] = Delta m (< q).  Every thread of the CTA calls it;
// it ends synchronised.
__device__ __forceinline__ void slot_encode_lift(u32* a, u64* c, const uint2* tw, const DevParams& P) {
    const u32 logL = P.logS, L = 1u << logL, lper = logL - 3;
    const bool active = threadIdx.x < (P.d << lper);
    const u32 vec = threadIdx.x >> lper, tl = threadIdx.x & ((1u << lper) - 1u), voff = vec << logL;
    const int npass = ((int)logL + 2) / 3;
    for (int ps = 0; ps < npass; ps++) {
        const int lo = 3 * ps;
        const int hi = lo + 2 < (int)logL - 1 ? lo + 2 : (int)logL - 1;
        const u32 wlo = (u32)lo + 3 <= logL ? (u32)lo : logL - 3;
        if (active) {
            const u32 hb = (tl >> wlo) << (wlo + 3);
            const u32 base = hb | (tl & ((1u << wlo) - 1u));
            u32 x[8];
#pragma unroll
            for (int r = 0; r < 8; r++) x[r] = a[padx(voff + base + ((u32)r << wlo))];
#pragma unroll
            for (int st = 0; st < 3; st++) {
                const int b = (int)wlo + st;
                if (b > hi || b < lo) continue;
                const u32 tb = (L + hb) >> (b + 1);
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    if (r & (1 << st)) continue;
                    bfly_pair<false>(x[r], x[r | (1 << st)], tw[tb + (r >> (st + 1))], P);
                }
            }
            if (ps == npass - 1) {
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    u32 y = shoup_mul32(x[r], P.Sinv, P.Sinv_s, P.p);
                    y = y >= P.p ? y - P.p : y;
                    c[padx(vec + P.d * (base + ((u32)r << wlo)))] = P.delta * y;
                }
            } else {
#pragma unroll
                for (int r = 0; r < 8; r++) a[padx(voff + base + ((u32)r << wlo))] = x[r];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- share encoding
// beta = 1: one CTA per input ciphertext u = (bb, k).  beta > 1: one CTA per
// spectrum u = (bb, k), writing its beta ciphertexts (bb, k, h) from one
// transform of the planes.  kMode 0: write A = NTT_q(Delta m); kMode 1: add
// it to the ciphertexts' c1.
template <int kMode, bool kGTw>
__device__ __forceinline__ void share_body(unsigned char* sm, const DevParams& P, const DevLayer& L,
                                           const u32* __restrict__ x, u64* __restrict__ out, u32 u,
                                           const L2Prefetch* pf = nullptr) {
    const u32 n = P.n, S = P.S;
    const u32 np = padded_len(n);                        // padded length (even)
    ulonglong2* tq_s = reinterpret_cast<ulonglong2*>(sm);  // [n] (psi^brv, companion), unless kGTw
    uint2* tp = reinterpret_cast<uint2*>(tq_s + (kGTw ? 0 : n));  // [S] (psi_p^-brv, companion)
    uint2* tw_row = tp + S;                              // [W/2]
    uint2* tw_col = tw_row + (L.W >> 1);                 // [H/2]
    u64* c = reinterpret_cast<u64*>(tw_col + (L.H >> 1));  // padded [n]
    u32* slots = reinterpret_cast<u32*>(c + np);         // padded [n] = d slot sets
    u32* planes = slots + np;                            // beta > 1: padded [d][HW], the d images' planes
    const ulonglong2* tq = kGTw ? P.qfw2 : tq_s;
    const u32 HW = L.HW, logHW = L.logH + L.logW, blocks = L.g_c * L.g_b;
    if (L.beta > 1) {
        // a spectrum spans beta ciphertexts (H W > S, g_c = g_b = 1): slot set r
        // of ciphertext (bb, k, h) holds part h of the spectrum of channel k of
        // image bb d + r, so the CTA transforms the d whole planes once and
        // encodes the beta parts one after the other
        const u32 k = u % L.T, bb = u / L.T;
        for (u32 e = threadIdx.x; e < P.d * HW; e += blockDim.x) {
            const u32 r = e >> logHW, f = e & (HW - 1), b = bb * P.d + r;
            const u32 pos = (r << logHW) + (brv_bits(f >> L.logW, L.logH) << L.logW) + brv_bits(f & (L.W - 1), L.logW);
            planes[padx(pos)] = b < L.B ? __ldg(x + ((u64)b * L.Ci + k) * HW + f) : 0u;
        }
        stage_pairs_for_length(tw_row, L.logW, false, P);  // group 3
        stage_pairs_for_length(tw_col, L.logH, false, P);  // group 2
        stage_async(tp, P.pinv2, S * 8);                    // group 1
        stage_async(tq_s, P.qfw2, kGTw ? 0 : n * 16);  // group 0
        if (pf) pf->issue();
        stage_wait_groups<2>();
        for (u32 r = 0; r < P.d; r++) {  // one plane per pass: H W / 8 <= blockDim threads
            lines_r8p<false>(planes + padx(r * HW), 1, true, L.logH, L.logW, tw_row, P.p);
            lines_r8p<false>(planes + padx(r * HW), 1, false, L.logH, L.logW, tw_col, P.p);
        }
        stage_wait_groups<0>();  // every table in place
#pragma unroll 1
        for (u32 h = 0; h < L.beta; h++) {
            for (u32 e = threadIdx.x; e < n; e += blockDim.x) {
                const u32 r = e >> P.logS, s = e & (S - 1);
                slots[padx(e)] = planes[padx((r << logHW) + h * S + s)];
            }
            __syncthreads();
            slot_encode_lift(slots, c, tp, P);  // slot encode, then Delta m into c
            ntt_r8p<true, u64>(c, P.logn, 1, tq, 0, 0, P);
            const u64 uh = (u64)u * L.beta + h;  // ciphertext (bb, k, h)
            if (kMode == 0) {
                u64* A = out + uh * n;
                for (u32 j = threadIdx.x; j < n; j += blockDim.x) A[j] = c[padx(j)];
            } else {
                u64* c1 = out + uh * 2 * n + n;
                for (u32 j = threadIdx.x; j < n; j += blockDim.x) c1[j] = addmod_q(c1[j], c[padx(j)], P.q);
            }
            // the next part's slot copy writes slots only: c is rewritten after
            // the slot transform's barriers
        }
        return;
    } else {
    const u32 k = u % L.T, bb = u / L.T;
    // every load is issued before anything waits: the share's words (eight
    // per thread), then the twiddle tables in the order they are needed
    // (the block's image and channel are divided out only when the block
    // changes: a warp's words share one block, since H W >= 64)
    auto load8 = [&](u32 e0, u32 (&v)[8]) {
        u32 last = ~0u, bq = 0, br = 0;
#pragma unroll
        for (int t = 0; t < 8; t++) {
            const u32 e = e0 + threadIdx.x + (u32)t * blockDim.x;
            const u32 r = e >> P.logS, s = e & (S - 1), blk = s >> logHW, f = s & (HW - 1);
            v[t] = 0;
            if (e < n && blk < blocks) {
                if (blk != last) {
                    last = blk;
                    bq = blk / L.g_c;
                    br = blk - bq * L.g_c;
                }
                const u32 b = (bb * P.d + r) * L.g_b + bq, ci = k * L.g_c + br;
                if (b < L.B && ci < L.Ci) v[t] = __ldg(x + ((u64)b * L.Ci + ci) * HW + f);
            }
        }
    };
    // planes of the packed slot vector, in bit-reversed order along both axes
    auto store8 = [&](u32 e0, const u32 (&v)[8]) {
#pragma unroll
        for (int t = 0; t < 8; t++) {
            const u32 e = e0 + threadIdx.x + (u32)t * blockDim.x, f = e & (HW - 1);
            const u32 pos = (e & ~(HW - 1)) + (brv_bits(f >> L.logW, L.logH) << L.logW) + brv_bits(f & (L.W - 1), L.logW);
            if (e < n) slots[padx(pos)] = v[t];
        }
    };
    u32 v[8];
    load8(0, v);
    stage_pairs_for_length(tw_row, L.logW, false, P);  // group 3
    stage_pairs_for_length(tw_col, L.logH, false, P);  // group 2
    stage_async(tp, P.pinv2, S * 8);                    // group 1
    stage_async(tq_s, P.qfw2, kGTw ? 0 : n * 16);  // group 0
    store8(0, v);
    for (u32 e0 = 8 * blockDim.x; e0 < n; e0 += 8 * blockDim.x) {
        load8(e0, v);
        store8(e0, v);
    }
    if (pf) pf->issue();
    stage_wait_groups<2>();  // line twiddles (and the planes) in place
    // NTT2D of every plane (zero planes included): rows, then columns
    lines_r8p<false>(slots, n >> logHW, true, L.logH, L.logW, tw_row, P.p);
    lines_r8p<false>(slots, n >> logHW, false, L.logH, L.logW, tw_col, P.p);
    }
    stage_wait_groups<1>();
    slot_encode_lift(slots, c, tp, P);  // slot encode, then Delta m into c
    stage_wait_groups<0>();
    ntt_r8p<true, u64>(c, P.logn, 1, tq, 0, 0, P);
    if (kMode == 0) {
        u64* A = out + (u64)u * n;
        for (u32 j = threadIdx.x; j < n; j += blockDim.x) A[j] = c[padx(j)];
    } else {
        u64* c1 = out + (u64)u * 2 * n + n;
        for (u32 j = threadIdx.x; j < n; j += blockDim.x) c1[j] = addmod_q(c1[j], c[padx(j)], P.q);
    }
}

template <int kMode, bool kGTw>
__global__ void __launch_bounds__(kMaxThreads) share_kernel(DevParams P, DevLayer L, const u32* __restrict__ x,
                                                            u64* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    griddep_release();
    griddep_wait();
    share_body<kMode, kGTw>(sm, P, L, x, out, blockIdx.x);
}

// ---------------------------------------------------------------- the three producers in one launch
// CTAs [0, n_in) draw the encryption constants of ciphertext u, CTAs
// [n_in, 2 n_in) encode Alice's share x_A into A, CTAs [2 n_in, 3 n_in)
// encode Bob's share x_B into R -- the words of constants_kernel and
// share_kernel<0>.  Every CTA lets the next kernel in the stream launch at
// once (programmatic dependent launch), and, once its own loads have been
// issued, asks the L2 cache for its slice of two device ranges (the next
// kernel's input-independent operands: filter plaintexts and masks), so
// that those bytes stream from HBM while the transforms run.
template <bool kGTw>
__global__ void __launch_bounds__(kMaxThreads, kGTw ? 2 : 0) produce_kernel(DevParams P, DevLayer L, const u64* __restrict__ t_hat,
                                                              u64 seed, const u32* __restrict__ xA,
                                                              const u32* __restrict__ xB, u64* __restrict__ ct,
                                                              u64* __restrict__ A, u64* __restrict__ R, L2Prefetch pf) {
    extern __shared__ __align__(16) unsigned char sm[];
    griddep_release();
    griddep_wait();
    // CTAs [0, n_in): constants of ciphertext u; then n_in / beta CTAs per
    // share encoding, one per spectrum
    const u32 nsh = L.n_in / L.beta;
    u32 role = 0, u = blockIdx.x;
    if (blockIdx.x >= L.n_in) {
        const u32 b = blockIdx.x - L.n_in;
        role = 1 + b / nsh;
        u = b % nsh;
    }
    pf.slice = blockIdx.x;
    pf.slices = gridDim.x;
    if (role == 0) constants_body<kGTw>(sm, P, t_hat, 0, L.n_in, seed, nullptr, ct, 0, u, &pf);
    else share_body<0, kGTw>(sm, P, L, role == 1 ? xA : xB, role == 1 ? A : R, u, &pf);
}

// ---------------------------------------------------------------- decrypt + fold + INTT2D
// kMulti: a spectrum spans L.beta > 1 ciphertexts (H W > S); otherwise one.
template <bool kMulti, bool kGTw>
__global__ void __launch_bounds__(kMaxThreads, kMulti ? 2 : 0) decrypt_share_kernel(DevParams P, DevLayer L, const u64* __restrict__ t_hat,
                                                                    u64 key_stride, const u64* __restrict__ ct,
                                                                    u32* __restrict__ y, u32 scale, u32 scale_s) {
    extern __shared__ __align__(16) unsigned char sm[];
    const u32 n = P.n, S = P.S;
    const u32 np = padded_len(n);
    ulonglong2* tq_s = reinterpret_cast<ulonglong2*>(sm);  // [n] (psi^-brv, companion), unless kGTw
    uint2* tp = reinterpret_cast<uint2*>(tq_s + (kGTw ? 0 : n));  // [S] (psi_p^brv, companion)
    uint2* tw_row = tp + S;                              // [W/2]
    uint2* tw_col = tw_row + (L.W >> 1);                 // [H/2]
    u64* c = reinterpret_cast<u64*>(tw_col + (L.H >> 1));  // padded [n]
    u32* slots = reinterpret_cast<u32*>(c + np);         // padded [n]
    const u32 HW = L.HW, logHW = L.logH + L.logW;
    const u32 nplanes = P.d * L.g_b;
    u32* planes = slots + np;                            // padded [d g_b HW]
    const ulonglong2* tq = kGTw ? P.qinv2 : tq_s;
    griddep_release();
    griddep_wait();

    // one CTA per (image group, output channel): with H W > S its spectrum
    // spans beta ciphertexts (g_b = 1), decrypted one after the other into
    // the halves of the d planes
    const u32 vv = blockIdx.x, co = vv % L.Co, bb = vv / L.Co;
    const u32 beta = kMulti ? L.beta : 1u;
    t_hat += (u64)bb * key_stride;
#pragma unroll 1
    for (u32 h = 0; h < beta; h++) {
        const u64* c0 = ct + ((u64)vv * beta + h) * 2 * n;
        const u64* c1 = c0 + n;
        // v = c0 t + c1: all of a thread's words (n / blockDim <= 8 of each) are
        // requested at once, before the twiddle tables, which are copied in the
        // order they are needed; with several ciphertexts per spectrum, four at
        // a time (fewer registers: two CTAs share an SM)
        if constexpr (kMulti) {
#pragma unroll
            for (int r0 = 0; r0 < 8; r0 += 4) {
                u64 a[4], t[4], b[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const u32 j = threadIdx.x + (u32)(r0 + r) * blockDim.x;
                    if (j < n) {
                        a[r] = __ldg(c0 + j);
                        t[r] = __ldg(t_hat + j);
                        b[r] = __ldg(c1 + j);
                    }
                }
                if (h == 0 && r0 == 0) {
                    stage_async(tq_s, P.qinv2, kGTw ? 0 : n * 16);    // group 3
                    stage_async(tp, P.pfw2, S * 8);                    // group 2
                    stage_pairs_for_length(tw_row, L.logW, true, P);  // group 1
                    stage_pairs_for_length(tw_col, L.logH, true, P);  // group 0
                }
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const u32 j = threadIdx.x + (u32)(r0 + r) * blockDim.x;
                    if (j < n) c[padx(j)] = muladd_q(a[r], t[r], b[r], P);
                }
            }
        } else {
            u64 a[8], t[8], b[8];
#pragma unroll
            for (int r = 0; r < 8; r++) {
                const u32 j = threadIdx.x + (u32)r * blockDim.x;
                if (j < n) {
                    a[r] = __ldg(c0 + j);
                    t[r] = __ldg(t_hat + j);
                    b[r] = __ldg(c1 + j);
                }
            }
            if (h == 0) {
                stage_async(tq_s, P.qinv2, kGTw ? 0 : n * 16);    // group 3
                stage_async(tp, P.pfw2, S * 8);                    // group 2
                stage_pairs_for_length(tw_row, L.logW, true, P);  // group 1
                stage_pairs_for_length(tw_col, L.logH, true, P);  // group 0
            }
#pragma unroll
            for (int r = 0; r < 8; r++) {
                const u32 j = threadIdx.x + (u32)r * blockDim.x;
                if (j < n) c[padx(j)] = muladd_q(a[r], t[r], b[r], P);
            }
        }
        stage_wait_groups<3>();
        ntt_r8p<false, u64>(c, P.logn, 1, tq, P.ninv, P.ninv_s, P);
        for (u32 coef = threadIdx.x; coef < n; coef += blockDim.x) {
            const u32 r = coef & (P.d - 1), i = coef / P.d;
            slots[padx(r * S + i)] = kMulti ? round_pq(c[padx(coef)], P) : round_pq_wide(c[padx(coef)], P);
        }
        stage_wait_groups<2>();
        ntt_r8p<true, u32>(slots, P.logS, P.d, tp, 0, 0, P);  // slot decode
        if (!kMulti) {
            // fold the g_c channel blocks of every image block: plane (r, ib)
            for (u32 e = threadIdx.x; e < nplanes * HW; e += blockDim.x) {
                const u32 pl = e >> logHW, f = e & (HW - 1), r = pl / L.g_b, ib = pl % L.g_b;
                const u32 src = r * S + ib * L.g_c * HW + f;
                u32 acc = 0;
                for (u32 ic = 0; ic < L.g_c; ic++) acc = addmod_p(acc, slots[padx(src + ic * HW)], P.p);
                planes[padx(e)] = acc;
            }
        } else {
            // slot set r holds half h of image bb d + r's spectrum
            for (u32 e = threadIdx.x; e < n; e += blockDim.x) {
                const u32 r = e >> P.logS, s = e & (S - 1);
                planes[padx((r << logHW) + h * S + s)] = slots[padx(e)];
            }
        }
        __syncthreads();
    }
    stage_wait_groups<0>();
    if (!kMulti) {
        lines_r8p<true>(planes, nplanes, true, L.logH, L.logW, tw_row, P.p);
        lines_r8p<true>(planes, nplanes, false, L.logH, L.logW, tw_col, P.p);
    } else {
        for (u32 r = 0; r < nplanes; r++) {  // one plane per pass: H W / 8 <= blockDim threads
            lines_r8p<true>(planes + padx(r * HW), 1, true, L.logH, L.logW, tw_row, P.p);
            lines_r8p<true>(planes + padx(r * HW), 1, false, L.logH, L.logW, tw_col, P.p);
        }
    }
    for (u32 e = threadIdx.x; e < nplanes * HW; e += blockDim.x) {
        const u32 pl = e >> logHW, f = e & (HW - 1), r = pl / L.g_b, ib = pl % L.g_b;
        const u32 b = (bb * P.d + r) * L.g_b + ib;
        if (b >= L.B) continue;
        u32 val = planes[padx((pl << logHW) + (brv_bits(f >> L.logW, L.logH) << L.logW) + brv_bits(f & (L.W - 1), L.logW))];
        val = shoup_mul32(val, scale, scale_s, P.p);
        y[((u64)b * L.Co + co) * HW + f] = val >= P.p ? val - P.p : val;
    }
}

// The same decryption + decode + fold + INTT2D split between the two CTAs of
// a cluster by coefficient parity (one slot set, d = 1).  Rank r computes the
// coefficients v_{2i+r} only: with the NTT_q words in bit-reversed order,
// words 2t and 2t+1 are the evaluations at psi^(2k+1) and -psi^(2k+1)
// (k = brv_{n/2}(t)), so
//   v_{2i}   = n^-1 INTT_{n/2}(c_{2t} + c_{2t+1})_i,
//   v_{2i+1} = n^-1 INTT_{n/2}(psi^-(2k+1) (c_{2t} - c_{2t+1}))_i,
// half-length transforms with psi^2, whose bit-reversed twiddles are the first
// half of the length-n table (psi^-(2k+1) = psi^-brv_n(t) * psi^-1, psi^-1 =
// the table's entry n/2).  Rounding is per coefficient.  The rest is linear:
// the slot vector of the even coefficients is Y[u] at slots 2u and 2u+1 (Y the
// half-length NTT_p), that of the odd ones psi_p^(2k+1) Z[u] at 2u and its
// negation at 2u+1; each CTA folds and INTT2Ds its part and the two partial
// shares are added through distributed shared memory.
__device__ __forceinline__ u32 cluster_rank() {
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ u32 ld_peer_u32(const u32* local, u32 peer) {
    u32 a = (u32)__cvta_generic_to_shared(local), ra, v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(peer));
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
    return v;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kMaxThreads)
    decrypt_share_pair_kernel(DevParams P, DevLayer L, const u64* __restrict__ t_hat, u64 key_stride,
                              const u64* __restrict__ ct, u32* __restrict__ y, u32 scale, u32 scale_s) {
    extern __shared__ __align__(16) unsigned char sm[];
    const u32 n = P.n, S = P.S, hn = n >> 1, hS = S >> 1;
    const u32 np = padded_len(n);
    ulonglong2* tq = reinterpret_cast<ulonglong2*>(sm);  // [n] (psi^-brv, companion)
    uint2* tp = reinterpret_cast<uint2*>(tq + n);        // [S] (psi_p^brv, companion)
    uint2* tw_row = tp + S;                              // [W/2]
    uint2* tw_col = tw_row + (L.W >> 1);                 // [H/2]
    u64* c = reinterpret_cast<u64*>(tw_col + (L.H >> 1));  // padded [n]
    u32* slots = reinterpret_cast<u32*>(c + np);         // padded [n]
    const u32 HW = L.HW, logHW = L.logH + L.logW;
    const u32 nplanes = L.g_b;
    u32* planes = slots + np;                            // padded [g_b HW]
    u32* xs = reinterpret_cast<u32*>(c);                 // the part's slot vector, padded [S] (c is free by then)
    griddep_release();
    griddep_wait();

    const u32 rank = cluster_rank();
    const u32 v = blockIdx.x >> 1, co = v % L.Co, bb = v / L.Co;
    t_hat += (u64)bb * key_stride;
    const u64* c0 = ct + (u64)v * 2 * n;
    const u64* c1 = c0 + n;
    // all of a thread's words (n / blockDim <= 8 of each) are requested at once,
    // before the twiddle tables: one memory latency instead of two
    u64 a[8], t[8], b[8];
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const u32 j = threadIdx.x + (u32)r * blockDim.x;
        if (j < n) {
            a[r] = __ldg(c0 + j);
            t[r] = __ldg(t_hat + j);
            b[r] = __ldg(c1 + j);
        }
    }
    stage_async(tq, P.qinv2, n * 16);                  // group 3
    stage_async(tp, P.pfw2, S * 8);                    // group 2
    stage_pairs_for_length(tw_row, L.logW, true, P);  // group 1
    stage_pairs_for_length(tw_col, L.logH, true, P);  // group 0
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const u32 j = threadIdx.x + (u32)r * blockDim.x;
        if (j < n) c[padx(j)] = muladd_q(a[r], t[r], b[r], P);
    }
    stage_wait_groups<3>();
    // this part's half-length input: h_t = c_{2t} + c_{2t+1}, or psi^-(2k+1) (c_{2t} - c_{2t+1})
    {
        const ulonglong2 pinv1 = tq[hn];  // psi^-1
        u64 hv[4];  // n/2 words over at least n/8 threads
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const u32 tt = threadIdx.x + (u32)r * blockDim.x;
            if (tt >= hn) continue;
            const u64 x0 = c[padx(2 * tt)], x1 = c[padx(2 * tt + 1)];
            u64 h;
            if (rank == 0) {
                h = addmod_q(x0, x1, P.q);
            } else {
                h = shoup_mul(submod_q(x0, x1, P.q), tq[tt].x, tq[tt].y, P.q);
                h = h >= P.q ? h - P.q : h;
                h = shoup_mul(h, pinv1.x, pinv1.y, P.q);
                h = h >= P.q ? h - P.q : h;
            }
            hv[r] = h;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const u32 tt = threadIdx.x + (u32)r * blockDim.x;
            if (tt < hn) c[padx(tt)] = hv[r];
        }
        __syncthreads();
    }
    ntt_r8p<false, u64>(c, P.logn - 1, 1, tq, P.ninv, P.ninv_s, P);  // v_{2i+rank}, i < n/2, times n^-1
    for (u32 i = threadIdx.x; i < hn; i += blockDim.x) slots[padx(i)] = round_pq_wide(c[padx(i)], P);
    stage_wait_groups<2>();
    ntt_r8p<true, u32>(slots, P.logS - 1, 1, tp, 0, 0, P);  // half-length slot decode
    {
        const uint2 psip = tp[hS];  // psi_p
        for (u32 u = threadIdx.x; u < hS; u += blockDim.x) {
            u32 w = slots[padx(u)];
            if (rank == 1) {
                w = shoup_mul32(w, tp[u].x, tp[u].y, P.p);
                w = w >= P.p ? w - P.p : w;
                w = shoup_mul32(w, psip.x, psip.y, P.p);
                w = w >= P.p ? w - P.p : w;
            }
            xs[padx(2 * u)] = w;
            xs[padx(2 * u + 1)] = rank == 1 ? (w ? P.p - w : 0u) : w;
        }
    }
    __syncthreads();
    // fold the g_c channel blocks of every image block
    for (u32 e = threadIdx.x; e < nplanes * HW; e += blockDim.x) {
        const u32 ib = e >> logHW, f = e & (HW - 1);
        const u32 src = ib * L.g_c * HW + f;
        u32 acc = 0;
        for (u32 ic = 0; ic < L.g_c; ic++) acc = addmod_p(acc, xs[padx(src + ic * HW)], P.p);
        planes[padx(e)] = acc;
    }
    stage_wait_groups<0>();
    lines_r8p<true>(planes, nplanes, true, L.logH, L.logW, tw_row, P.p);
    lines_r8p<true>(planes, nplanes, false, L.logH, L.logW, tw_col, P.p);
    // this part's share in natural order, then the two parts added across the pair
    u32* part = slots;  // [g_b HW], free after the decode
    for (u32 e = threadIdx.x; e < nplanes * HW; e += blockDim.x) {
        const u32 pl = e >> logHW, f = e & (HW - 1);
        u32 val = planes[padx((pl << logHW) + (brv_bits(f >> L.logW, L.logH) << L.logW) + brv_bits(f & (L.W - 1), L.logW))];
        val = shoup_mul32(val, scale, scale_s, P.p);
        part[e] = val >= P.p ? val - P.p : val;
    }
    cluster_sync_all();
    const u32 half = (nplanes * HW) >> 1;
    for (u32 e = rank * half + threadIdx.x; e < (rank + 1) * half; e += blockDim.x) {
        const u32 pl = e >> logHW, f = e & (HW - 1);
        const u32 bi = bb * L.g_b + pl;
        if (bi >= L.B) continue;
        y[((u64)bi * L.Co + co) * HW + f] = addmod_p(part[e], ld_peer_u32(part + e, rank ^ 1), P.p);
    }
    cluster_sync_all();  // the peer's part stays in place until both halves are read
}

template <typename K>
cudaError_t opt_in(K kernel, size_t bytes) {
    if (bytes + 1024 <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}


}  // namespace

size_t share_smem_bytes(const DevParams& P, const DevLayer& L) {
    const size_t np = padded_len(P.n), npl = L.beta > 1 ? padded_len(P.d * L.HW) : 0;
    return (size_t)qtw_entries(P.n) * 16 + np * 8 + (size_t)P.S * 8 + np * 4 + npl * 4 + (size_t)4 * (L.W + L.H);
}
size_t decrypt_share_smem_bytes(const DevParams& P, const DevLayer& L) {
    const size_t np = padded_len(P.n), npl = padded_len(P.d * L.g_b * L.HW);
    return (size_t)qtw_entries(P.n) * 16 + np * 8 + (size_t)P.S * 8 + np * 4 + npl * 4 + (size_t)4 * (L.W + L.H);
}
// Threads of the fused kernels: n / 8 for the length-n passes, and at least
// H W / 8 for the line passes of one plane (more than n / 8 only when a
// spectrum spans several ciphertexts).
u32 fused_threads(const DevParams& P, const DevLayer& L) {
    const u32 t = threads_for(P.n), tl = L.HW / 8;
    return t > tl ? t : tl;
}
size_t constants_smem_bytes(const DevParams& P) {
    return (size_t)qtw_entries(P.n) * 16 + (size_t)P.n * 8 + (size_t)padded_len(P.n) * 8;
}

cudaError_t launch_constants(const DevParams& P, const DevLayer& L, const u64* t_hat, u64 key_stride, u64 seed,
                             const u64* seeds, u64* ct, cudaStream_t s, bool c1_only) {
    const size_t sm = constants_smem_bytes(P);
    auto kern = global_qtw(P.n) ? constants_kernel<true> : constants_kernel<false>;
    cudaError_t e = opt_in(kern, sm);
    if (e != cudaSuccess) return e;
    return launch_online(kern, L.n_in, threads_for(P.n), sm, s, P, t_hat, key_stride, L.T * L.beta, seed,
                         seeds, ct, c1_only ? 1 : 0);
}

cudaError_t launch_share(const DevParams& P, const DevLayer& L, const u32* x, u64* out, bool add_to_ct,
                         cudaStream_t s) {
    const size_t sm = share_smem_bytes(P, L);
    const bool g = global_qtw(P.n);
    auto kern = add_to_ct ? (g ? share_kernel<1, true> : share_kernel<1, false>)
                          : (g ? share_kernel<0, true> : share_kernel<0, false>);
    cudaError_t e = opt_in(kern, sm);
    if (e != cudaSuccess) return e;
    return launch_online(kern, L.n_in / L.beta, fused_threads(P, L), sm, s, P, L, x, out);
}

size_t produce_smem_bytes(const DevParams& P, const DevLayer& L) {
    const size_t a = share_smem_bytes(P, L), b = constants_smem_bytes(P);
    return a > b ? a : b;
}

cudaError_t launch_produce(const DevParams& P, const DevLayer& L, const u64* t_hat, u64 seed, const u32* xA,
                           const u32* xB, u64* ct, u64* A, u64* R, const void* pf0, u64 pf0_bytes, const void* pf1,
                           u64 pf1_bytes, cudaStream_t s) {
    const size_t sm = produce_smem_bytes(P, L);
    auto kern = global_qtw(P.n) ? produce_kernel<true> : produce_kernel<false>;
    cudaError_t e = opt_in(kern, sm);
    if (e != cudaSuccess) return e;
    L2Prefetch pf = {{pf0, pf1}, {pf0_bytes, pf1_bytes}, 0, 0};
    return launch_online(kern, L.n_in + 2 * (L.n_in / L.beta), fused_threads(P, L), sm, s, P, L, t_hat, seed, xA, xB, ct, A,
                         R, pf);
}

cudaError_t launch_decrypt_share(const DevParams& P, const DevLayer& L, const u64* t_hat, u64 key_stride, const u64* ct,
                                 u32* y, cudaStream_t s) {
    const size_t sm = decrypt_share_smem_bytes(P, L);
    const u32 scale = fdsc_powmod32(L.HW % P.p, P.p - 2, P.p);
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (fdsc_decrypt_pair_allowed() && P.d == 1 && L.beta == 1 && P.n >= 32 && 2ull * L.n_out <= (u64)sms) {
        // one slot set and fewer output ciphertexts than half the SMs (a single
        // image): the two CTAs of a cluster take one parity of the coefficients
        // each, on SMs that would otherwise idle; batched work keeps one CTA per
        // ciphertext (the pair repeats the loads and the first products)
        const size_t sm2 = sm + (size_t)(P.n - qtw_entries(P.n)) * 16;  // the pair stages the NTT_q twiddles at any n
        cudaError_t e = opt_in(decrypt_share_pair_kernel, sm2);
        if (e != cudaSuccess) return e;
        return launch_online(decrypt_share_pair_kernel, 2 * L.n_out, threads_for(P.n), sm2, s, P, L, t_hat, key_stride,
                             ct, y, scale, fdsc_shoup32(scale, P.p));
    }
    const bool g = global_qtw(P.n);
    auto kern = L.beta > 1 ? (g ? decrypt_share_kernel<true, true> : decrypt_share_kernel<true, false>)
                           : (g ? decrypt_share_kernel<false, true> : decrypt_share_kernel<false, false>);
    cudaError_t e = opt_in(kern, sm);
    if (e != cudaSuccess) return e;
    return launch_online(kern, L.n_out / L.beta, fused_threads(P, L), sm, s, P, L, t_hat, key_stride, ct, y, scale,
                         fdsc_shoup32(scale, P.p));
}
