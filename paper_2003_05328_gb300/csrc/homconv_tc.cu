// homconv_tc.cu -- HomConv + HomShare (Fig. 2, Eq. 2) on the
// tensor cores, exact.
//
// For every evaluation index J = (h, j) of the NTT_q domain the layer is a
// modular matrix product over the input ciphertexts k,
//   out[co][col] = sum_k P[co][k] X[k][col]  (mod q),   col = (bb, c),
// of 60-bit words.  A word w < 2^60 is written in balanced base-256 digits,
//   w = sum_{a<8} d_a 256^a,   d_a = byte_a(w + 0x8080808080808080) - 128,
// so d_a lies in [-128, 127] (the top digit in [0, 16]) and is held exactly
// by fp16.  Then
//   sum_k P X = sum_{kappa<15} 256^kappa D_kappa,
//   D_kappa[co][col] = sum_{a+b=kappa} sum_k P_a[co][k] X_b[k][col],
// and every partial sum of D_kappa is an integer of magnitude at most
// T * 7 * 2^14 < 2^24 for T <= 128, so the fp32 accumulation of the tensor
// cores is exact.  The epilogue converts the 15 diagonals to integers,
// combines them into the 128-bit value of the sum and reduces it mod q once.
//
// MMA mapping (tcgen05.mma kind::f16, M = 128 output channels in the TMEM
// lanes, K = 16 input ciphertexts per instruction): the B operand stacks the
// eight digit planes of X along N (rows (b, col), N = 8 NB), and the MMA of
// filter digit plane a accumulates into a TMEM column window shifted by a NB
// columns: column block kappa then receives exactly the products with
// a + b = kappa.  One MMA with a zero A operand clears the upper part of the
// window before the first accumulation.  The filter arrives as fp16 digit
// planes already in the A operand layout (fdsc_filter_tc, setup).
//
// Roles in a persistent CTA of 16 warps (one CTA per SM):
//   warps 0-7   epilogue: TMEM -> diagonals -> 128-bit sum -> mod q -> HomShare
//   warp 8      TMEM allocation; lane 0 issues the MMAs
//   warp 9      loader: one bulk copy per unit of the filter digit planes into
//               the unit's operand slot (lane 0)
//   warps 10-15 converters of the input words, NC of them (as many as operand
//               slots fit): each stages the ciphertext words (and the fused c1
//               addends) of its next unit with cp.async while it converts the
//               current one into fp16 digit planes.
// Unit u uses operand slot u mod NC and converter u mod NC, so every slot is
// filled, converted and consumed in unit order and no waiter can run two
// phases ahead of the mbarrier it polls (a parity wait cannot tell phase k
// from phase k - 2).
// A unit is (item, 16 input ciphertexts); an item is (J, 128 output channels,
// up to 8 image groups; with d slot sets per ciphertext, the d evaluation
// indices sharing a filter word and up to 8 / d image groups).  Up to 8 TMEM
// accumulators let the MMAs of later items run while the epilogue drains
// earlier ones.  Every wait is bounded: on
// a timeout the CTA records an error, stops, lets its copies and MMAs finish,
// frees its TMEM and returns.
#include <cuda_fp16.h>

#include <mutex>

#include "modarith.cuh"

namespace {

constexpr u32 kThreadsTC = 512;
constexpr u32 kEpiWarps = 8;
constexpr u32 kMmaWarp = 8;
constexpr u32 kLoadWarp = 9;
constexpr u32 kConvWarp0 = 10;
constexpr u32 kMaxConv = 6;   // converter warps at most
constexpr u32 kMaxSlots = 8;  // barrier slots reserved per ring
constexpr u64 kDigitBias = 0x8080808080808080ull;
constexpr u64 kWaitNs = 2000000000ull;  // a wait gives up after 2 s

struct TcGeom {
    u32 NB;       // B columns (r, bb, c) per item: 2 x image groups per pass x evaluation indices per item
    u32 dj;       // evaluation indices per item: d (the group sharing one filter word) or 1
    u32 lgbt;     // log2 gbt
    u32 KB;       // 16-ciphertext blocks: ceil(T / 16)
    u32 n_ct;     // 128-channel tiles
    u32 n_gbg;    // image-group passes
    u32 gbt;      // image groups per pass (NB / 2)
    u32 n_items;  // nJ * n_ct * n_gbg
    u32 NC;       // converter warps = operand slots
    u32 co_pad;   // filter rows stored per unit group: tiles of 128, the last rounded up to 8
    u32 az;       // bytes of a slot's A operand region
    u32 ssz;      // bytes of one slot (A, input digit planes, input-word buffers)
    u32 off_slot; // first slot
};

// Rows of 128-channel tile ct, rounded up to a multiple of 8.
__host__ __device__ inline u32 tile_rows8(u32 Co, u32 ct) {
    const u32 r = Co - 128 * ct < 128 ? Co - 128 * ct : 128;
    return (r + 7) & ~7u;
}

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ u64 sdesc(u32 addr, u32 lbo, u32 sbo) {
    // no-swizzle K-major: LBO = byte stride between the two 8-element K halves,
    // SBO = byte stride between 8-row groups; bit 46 = descriptor version 1
    return (u64)((addr & 0x3FFFF) >> 4) | ((u64)(lbo >> 4) << 16) | ((u64)(sbo >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ u32 idesc_f16(u32 M, u32 N) {
    // D f32 (bits 4-5 = 1), A and B f16 (0), both K-major, N >> 3 at 17, M >> 4 at 24
    return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(u32 d, u64 a, u64 b, u32 idesc, u32 acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(u32 bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(u32 bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(u32 bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u32 bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// try_wait with a suspend-time hint: a waiting warp sleeps in hardware until
// the phase completes (or about 20 us pass) instead of spinning on issue slots
__device__ __forceinline__ bool mbar_try(u32 bar, u32 parity) {
    u32 ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ u64 gtime_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: false after kWaitNs or once *abort is set.
__device__ __forceinline__ bool mbar_wait(u32 bar, u32 parity, const volatile u32* abort) {
    if (mbar_try(bar, parity)) return true;
    const u64 t0 = gtime_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort || gtime_ns() - t0 > kWaitNs) return false;
    }
}
// Bounded wait that ignores the abort flag (used to drain copies in flight).
__device__ __forceinline__ void mbar_drain(u32 bar, u32 parity) {
    const u64 t0 = gtime_ns();
    while (!mbar_try(bar, parity) && gtime_ns() - t0 <= kWaitNs) {
    }
}
__device__ __forceinline__ void bulk_g2s(u32 dst, const void* src, u32 bytes, u32 bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(u32 dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
template <int N>
__device__ __forceinline__ void tmem_ld(u32 addr, u32 (&r)[N]);
template <>
__device__ __forceinline__ void tmem_ld<1>(u32 addr, u32 (&r)[1]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[0]) : "r"(addr));
}
template <>
__device__ __forceinline__ void tmem_ld<2>(u32 addr, u32 (&r)[2]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}
template <>
__device__ __forceinline__ void tmem_ld<4>(u32 addr, u32 (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
template <>
__device__ __forceinline__ void tmem_ld<8>(u32 addr, u32 (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- digit planes
// Eight biased words (w + 0x80..80) -> for each digit a, the eight fp16 values
// d_a(w_0..w_7) in word order (one 16-byte row of a core matrix).  A byte u
// becomes the fp16 with bit pattern 0x64uu = 1024 + u; subtracting 1152
// leaves u - 128 = d_a exactly.
__device__ __forceinline__ u32 hsub1152(u32 h2) {
    __half2 v = *reinterpret_cast<__half2*>(&h2);
    v = __hsub2(v, __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480)));  // 1152
    return *reinterpret_cast<u32*>(&v);
}
__device__ __forceinline__ void digit_rows(const u64 (&w)[8], uint4 (&row)[8]) {
#pragma unroll
    for (int half = 0; half < 2; half++) {
        u32 v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = half ? (u32)(w[k] >> 32) : (u32)w[k];
        u32 o[4][4];  // [digit within half][word pair]
#pragma unroll
        for (int kp = 0; kp < 4; kp++) {
            const u32 t01 = __byte_perm(v[2 * kp], v[2 * kp + 1], 0x5140);  // x0 y0 x1 y1
            const u32 t23 = __byte_perm(v[2 * kp], v[2 * kp + 1], 0x7362);  // x2 y2 x3 y3
            o[0][kp] = hsub1152(__byte_perm(t01, 0x64646464u, 0x4140));
            o[1][kp] = hsub1152(__byte_perm(t01, 0x64646464u, 0x4342));
            o[2][kp] = hsub1152(__byte_perm(t23, 0x64646464u, 0x4140));
            o[3][kp] = hsub1152(__byte_perm(t23, 0x64646464u, 0x4342));
        }
#pragma unroll
        for (int a = 0; a < 4; a++) row[4 * half + a] = make_uint4(o[a][0], o[a][1], o[a][2], o[a][3]);
    }
}

// Walks the units of one CTA: unit u -> item blockIdx.x + (u / KB) * grid,
// ciphertext block u % KB; item -> (J fastest, channel tile, image-group
// pass).  Advancing by d units costs a few adds (no divisions).
struct UnitIter {
    u32 grid, nJ, n_ct, KB;
    u32 kb, J, ct, gbg;
    __device__ UnitIter(u32 cta, u32 grid_, u32 nJ_, u32 n_ct_, u32 KB_, u32 u0)
        : grid(grid_), nJ(nJ_), n_ct(n_ct_), KB(KB_) {
        const u32 item = cta + (u0 / KB) * grid;
        kb = u0 % KB;
        J = item % nJ;
        const u32 rest = item / nJ;
        ct = rest % n_ct;
        gbg = rest / n_ct;
    }
    __device__ void next(u32 d) {
        kb += d;
        while (kb >= KB) {
            kb -= KB;
            J += grid;
            while (J >= nJ) {
                J -= nJ;
                if (++ct == n_ct) {
                    ct = 0;
                    gbg++;
                }
            }
        }
    }
};

// ---------------------------------------------------------------- the kernel
template <int NBH>
__global__ void __launch_bounds__(kThreadsTC, 1)
    homconv_tc_kernel(DevParams P, DevLayer L, TcGeom G, const u64* __restrict__ ct_in, const u64* __restrict__ A1,
                      const u64* __restrict__ A2, const unsigned char* __restrict__ Ptc,
                      const u64* __restrict__ Mhat, u64* __restrict__ ct_out, u32* __restrict__ err) {
    constexpr u32 NB = 2 * NBH;
    constexpr u32 BUFC = 16 * NB;               // TMEM columns of one accumulator: 16 blocks of NB
    constexpr u32 NBUF = 512 / BUFC > 8 ? 8 : 512 / BUFC;  // accumulators in flight
    extern __shared__ __align__(1024) unsigned char sm[];
    // barriers: a_full[8] x_full[8] s_empty[8] tfull[8] tempty[8] drain
    const u32 b_afull = smem_u32(sm), b_xfull = b_afull + 64, b_sempty = b_xfull + 64, b_tfull = b_sempty + 64,
              b_tempty = b_tfull + 64, b_drain = b_tempty + 64;
    volatile u32* tmem_slot = reinterpret_cast<volatile u32*>(sm + 400);
    volatile u32* abort = reinterpret_cast<volatile u32*>(sm + 408);
    unsigned char* zero_blk = sm + 1024;
    const u32 tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const u32 nJ = L.beta * P.n / G.dj;  // items per (channel tile, image-group pass): groups of dj indices
    const u32 my_items = blockIdx.x < G.n_items ? (G.n_items - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const u32 total_units = my_items * G.KB;

    // ---- setup: zero block and operand slots, barriers, TMEM
    for (u32 e = tid; e < (G.off_slot + G.NC * G.ssz - 1024) / 16; e += kThreadsTC)
        reinterpret_cast<uint4*>(sm + 1024)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (u32 s = 0; s < kMaxSlots; s++) {
            mbar_init(b_afull + 8 * s, 1);   // the loader's expect_tx; the bulk copy completes the bytes
            mbar_init(b_xfull + 8 * s, 1);   // the slot's converter
            mbar_init(b_sempty + 8 * s, 1);  // tcgen05.commit after the slot's MMAs
            mbar_init(b_tfull + 8 * s, 1);
            mbar_init(b_tempty + 8 * s, kEpiWarps);
        }
        mbar_init(b_drain, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(
                         (const void*)tmem_slot)),
                     "r"(NBUF * BUFC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const u32 tmem = *tmem_slot;

    if (warp == kLoadWarp) {
        // ================================================================ loader (lane 0)
        if (lane == 0) {
            UnitIter it(blockIdx.x, gridDim.x, nJ, G.n_ct, G.KB, 0);
            u32 u = 0;
            for (; u < total_units; u++, it.next(1)) {
                const u32 s = u % G.NC, bar = b_afull + 8 * s;
                if (!mbar_wait(b_sempty + 8 * s, ((u / G.NC) & 1) ^ 1, abort)) break;
                const u32 rp = tile_rows8(L.Co, it.ct), bytes = 256 * rp;
                mbar_expect_tx(bar, bytes);
                // indices J of one group of d share their filter unit (w_0(x^d) plaintexts)
                bulk_g2s(smem_u32(sm + G.off_slot + s * G.ssz),
                         Ptc + ((u64)((it.J * G.dj / P.d) * G.KB + it.kb) * G.co_pad + it.ct * 128) * 256, bytes,
                         bar);
            }
            if (u < total_units) {
                *abort = 1;
                atomicExch(err, 1u);
            }
            // copies still in flight land before the CTA may exit (the last NC units at most)
            for (u32 v = u > G.NC ? u - G.NC : 0; v < u; v++) mbar_drain(b_afull + 8 * (v % G.NC), (v / G.NC) & 1);
        }
        __syncwarp();
    } else if (warp >= kConvWarp0) {
        // ================================================================ converters (input words)
        const u32 cw = warp - kConvWarp0, s = cw;  // this converter's own slot
        if (cw < G.NC && cw < total_units) {
            // input words of a unit, staged by this warp's lanes with cp.async:
            // [16][NB] ciphertext words, then [16][NB/2] A1 and [16][NB/2] A2 words of
            // the c1 columns; double-buffered so the next unit's copies fly while
            // this one is converted.  Column col = 2 (r gbt + bbi) + c: index
            // r of the item's dj evaluation indices, image group bbi of the pass,
            // ciphertext part c.
            u64* xbuf = reinterpret_cast<u64*>(sm + G.off_slot + s * G.ssz + G.az + 256 * NB);
            auto stage_x = [&](const UnitIter& t, u64* xr) {
                const u32 Jb = t.J * G.dj, h = Jb >> P.logn, j = Jb & (P.n - 1), bb0 = t.gbg * G.gbt;
#pragma unroll 2
                for (u32 e = lane; e < 32 * NB; e += 32) {
                    u32 plane, kk, col;
                    if (e < 16 * NB) {
                        plane = 0, kk = e / NB, col = e % NB;
                    } else {
                        const u32 ra = (e - 16 * NB) % (8 * NB);
                        plane = 1 + (e - 16 * NB) / (8 * NB), kk = ra / NBH, col = 2 * (ra % NBH) + 1;
                    }
                    const u32 c = col & 1, k = t.kb * 16 + kk, hc2 = col >> 1;
                    const u32 r = hc2 >> G.lgbt, bb = bb0 + (hc2 & (G.gbt - 1));
                    const u64* base = plane == 0 ? ct_in : (plane == 1 ? A1 : A2);
                    if (k < L.T && bb < L.GB && base) {
                        const u64 uin = ((u64)bb * L.T + k) * L.beta + h;
                        cp_async8(smem_u32(xr + e), base + (plane == 0 ? uin * 2 + c : uin) * P.n + j + r);
                    } else {
                        xr[e] = 0;
                    }
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
            UnitIter it(blockIdx.x, gridDim.x, nJ, G.n_ct, G.KB, cw);
            stage_x(it, xbuf);
            u32 par = 0;
            for (u32 u = cw; u < total_units; u += G.NC, par ^= 1) {
                UnitIter nx = it;
                nx.next(G.NC);
                if (u + G.NC < total_units)
                    stage_x(nx, xbuf + (par ^ 1) * 32 * NB);
                else
                    asm volatile("cp.async.commit_group;" ::: "memory");
                if (!__all_sync(0xffffffffu, mbar_wait(b_sempty + 8 * s, ((u / G.NC) & 1) ^ 1, abort))) {
                    *abort = 1;
                    atomicExch(err, 4u);
                    break;
                }
                asm volatile("cp.async.wait_group 1;" ::: "memory");  // this unit's input words
                __syncwarp();
                unsigned char* fX = sm + G.off_slot + s * G.ssz + G.az;
                const u64* xr = xbuf + par * 32 * NB;
                // task (col, k8): ciphertexts k8*8 .. k8*8+7 of column col; c1 gets the addends mod q
                for (u32 t = lane; t < 2 * NB; t += 32) {
                    u64 w[8];
                    uint4 row[8];
                    const u32 col = t >> 1, k8 = t & 1;
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const u32 kk = k8 * 8 + i;
                        u64 x = xr[kk * NB + col];
                        if (col & 1) {
                            x = addmod_q(x, xr[16 * NB + kk * NBH + (col >> 1)], P.q);
                            x = addmod_q(x, xr[24 * NB + kk * NBH + (col >> 1)], P.q);
                        }
                        w[i] = x + kDigitBias;
                    }
                    digit_rows(w, row);
#pragma unroll
                    for (int b = 0; b < 8; b++)
                        *reinterpret_cast<uint4*>(fX + k8 * (8 * NB * 16) + (b * NB + col) * 16) = row[b];
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(b_xfull + 8 * s);
                it = nx;
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
    } else if (warp == kMmaWarp) {
        // ================================================================ MMA issue
        if (lane == 0) {
            const u32 idesc = idesc_f16(128, 8 * NB);
            const u64 zdesc = sdesc(smem_u32(zero_blk), 128, 256);
            UnitIter it(blockIdx.x, gridDim.x, nJ, G.n_ct, G.KB, 0);
            u32 u = 0;
            bool ok = true;
            for (u32 li = 0; li < my_items && ok; li++) {
                const u32 b = li % NBUF;
                if (!mbar_wait(b_tempty + 8 * b, ((li / NBUF) & 1) ^ 1, abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const u32 dbuf = tmem + b * BUFC;
                for (u32 kb = 0; kb < G.KB; kb++, u++, it.next(1)) {
                    const u32 s = u % G.NC, par = (u / G.NC) & 1;
                    if (!mbar_wait(b_afull + 8 * s, par, abort) || !mbar_wait(b_xfull + 8 * s, par, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const u32 fA = smem_u32(sm + G.off_slot + s * G.ssz), ablk = 32 * tile_rows8(L.Co, it.ct);
                    const u64 xdesc = sdesc(fA + G.az, 8 * NB * 16, 128);
#pragma unroll
                    for (u32 a = 0; a < 8; a++) {
                        // digit plane a of the filter accumulates into the window shifted by a blocks
                        mma_f16(dbuf + a * NB, sdesc(fA + a * ablk, 128, 256), xdesc, idesc, (kb | a) ? 1u : 0u);
                        if (kb == 0 && a == 0) mma_f16(dbuf + 8 * NB, zdesc, xdesc, idesc, 0u);
                    }
                    mma_commit(b_sempty + 8 * s);
                }
                if (ok) mma_commit(b_tfull + 8 * b);
            }
            if (!ok) {
                *abort = 1;
                atomicExch(err, 2u);
            }
            // every MMA issued has completed before the TMEM may be freed
            mma_commit(b_drain);
            mbar_drain(b_drain, 0);
        }
        __syncwarp();
    } else {
        // ================================================================ epilogue
        const u32 quarter = warp & 3, hc = warp >> 2;
        const u32 r = quarter * 32 + lane;
        const u32 lane_addr = (quarter * 32) << 16;
        const u32 col0 = hc * NBH;
        // diagonals are read as biased integers B = D + 0x4B400000 (positive, below 2^31):
        // for T <= 32 every |D| < 2^22 and the bits of D + 1.5 * 2^23 (one fp32 add) are B;
        // otherwise B = rint(D) + 0x4B400000.  The bias of all 15 diagonals is removed once.
        const bool magic = L.T <= 32;
        unsigned __int128 bias = 0;
#pragma unroll
        for (int k = 0; k < 15; k++) bias += (unsigned __int128)0x4B400000u << (8 * k);
        const u64 out_bb = (u64)L.Co * L.beta * 2 * P.n;  // output stride of one image group
        const u64 msk_bb = (u64)L.Co * L.beta * P.n;      // mask stride of one image group
        UnitIter it(blockIdx.x, gridDim.x, nJ, G.n_ct, G.KB, 0);
        for (u32 li = 0; li < my_items; li++, it.next(G.KB)) {
            const u32 b = li % NBUF;
            const u32 Jb = it.J * G.dj, h = Jb >> P.logn, j = Jb & (P.n - 1);
            const u32 co = it.ct * 128 + r, bb0 = it.gbg * G.gbt;
            const u64 vbase = ((u64)bb0 * L.Co + co) * L.beta + h;
            const u64 obase = vbase * 2 * P.n + j, mbase = vbase * P.n + j;
            // the HomShare mask words of this thread's c1 outputs, fetched while the MMAs run
            u64 mk[NBH];
#pragma unroll
            for (int i = 0; i < NBH; i++) {
                const u32 col = col0 + i, hc2 = col >> 1, bbi = hc2 & (G.gbt - 1), ri = hc2 >> G.lgbt;
                mk[i] = 0;
                if ((col & 1) && Mhat && co < L.Co && bb0 + bbi < L.GB)
                    mk[i] = __ldg(Mhat + mbase + (u64)bbi * msk_bb + ri);
            }
            if (!__all_sync(0xffffffffu, mbar_wait(b_tfull + 8 * b, (li / NBUF) & 1, abort))) {
                *abort = 1;
                atomicExch(err, 3u);
                break;
            }
            tc_fence_after();
            if (quarter * 32 >= L.Co - it.ct * 128) {
                // this warp's lanes hold only the padding rows of a narrower tile
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(b_tempty + 8 * b);
                continue;
            }
            const u32 base = tmem + lane_addr + b * BUFC + col0;
            unsigned __int128 V[NBH];  // the biased sum mod 2^128
#pragma unroll
            for (int i = 0; i < NBH; i++) V[i] = 0;
#pragma unroll
            for (u32 m = 0; m < 4; m++) {
                u32 d[4][NBH];
#pragma unroll
                for (u32 rr = 0; rr < 4; rr++)
                    if (4 * m + rr < 15) tmem_ld<NBH>(base + (4 * m + rr) * NB, d[rr]);
                tmem_wait_ld();
#pragma unroll
                for (u32 rr = 0; rr < 4; rr++)
#pragma unroll
                    for (int i = 0; i < NBH; i++)
                        if (4 * m + rr < 15) asm volatile("" : "+r"(d[rr][i]));
#pragma unroll
                for (int i = 0; i < NBH; i++) {
                    u64 cm = 0;  // sum of B 2^(8 rr): below 2^56
#pragma unroll
                    for (u32 rr = 0; rr < 4; rr++) {
                        if (4 * m + rr >= 15) continue;
                        const float f = __uint_as_float(d[rr][i]);
                        const u32 bv = magic ? __float_as_uint(f + 12582912.0f)
                                             : (u32)(__float2int_rn(f) + 0x4B400000);
                        cm += (u64)bv << (8 * rr);
                    }
                    V[i] += (unsigned __int128)cm << (32 * m);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_tempty + 8 * b);
            if (co < L.Co) {
#pragma unroll
                for (int i = 0; i < NBH; i++) {
                    const u32 col = col0 + i, c = col & 1, hc2 = col >> 1, bbi = hc2 & (G.gbt - 1);
                    if (bb0 + bbi >= L.GB) continue;
                    const unsigned __int128 v = V[i] - bias;  // the exact sum, in [0, 2^127)
                    u64 res = reduce128((u64)(v >> 64), (u64)v, P);
                    if (c == 1) res = submod_q(res, mk[i], P.q);
                    ct_out[obase + (u64)bbi * out_bb + c * P.n + (hc2 >> G.lgbt)] = res;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NBUF * BUFC));
    }
}

// Phat [Co][T][beta][n/d] -> Ptc: per (group of d evaluation indices J' = J / d,
// 16-ciphertext block kb, 128-channel tile of R rows, R rounded up to rp, a
// multiple of 8) one contiguous unit of
// 256 rp bytes holding the eight fp16 digit planes of the filter words in the
// canonical no-swizzle K-major layout of a tcgen05 A operand: plane a at
// 32 rp a bytes, row r / k in the plane at (r / 8) 256 + (k / 8) 128 +
// (r mod 8) 16 + (k mod 8) 2.  Ciphertexts past T and rows past R are zero.
__global__ void filter_tc_kernel(const DevParams P, const DevLayer L, u32 KB, u32 co_pad,
                                 const u64* __restrict__ Phat, unsigned char* __restrict__ Ptc) {
    __shared__ u64 tile[16][65];
    const u32 nJ = L.beta * P.n / P.d;  // distinct filter words per (co, k)
    const u32 J0 = blockIdx.x * 64, kb = blockIdx.y, co = blockIdx.z;
    const u32 ct = co / 128, rl = co % 128, rp = tile_rows8(L.Co, ct);
    for (u32 e = threadIdx.x; e < 16 * 64; e += blockDim.x) {
        const u32 kk = e / 64, jj = e % 64, k = kb * 16 + kk, J = J0 + jj;
        u64 v = kDigitBias;
        if (k < L.T && J < nJ) v = Phat[((u64)co * L.T + k) * nJ + J] + kDigitBias;
        tile[kk][jj] = v;
    }
    __syncthreads();
    for (u32 e = threadIdx.x; e < 2 * 64; e += blockDim.x) {
        const u32 jj = e / 2, k8 = e % 2, J = J0 + jj;
        if (J >= nJ) continue;
        u64 w[8];
        uint4 row[8];
#pragma unroll
        for (int i = 0; i < 8; i++) w[i] = tile[k8 * 8 + i][jj];
        digit_rows(w, row);
        unsigned char* unit = Ptc + ((u64)(J * KB + kb) * co_pad + ct * 128) * 256;
        const u32 off = (rl >> 3) * 256 + k8 * 128 + (rl & 7) * 16;
#pragma unroll
        for (int a = 0; a < 8; a++) *reinterpret_cast<uint4*>(unit + a * 32 * rp + off) = row[a];
    }
}

__device__ u32 g_tc_err;  // nonzero after a CTA gave up waiting (1 loader, 2 MMA, 3 epilogue, 4 converter)

}  // namespace

// Geometry of the tensor-core path for a layer of ring degree n with d slot
// sets; false if it does not apply (T > 128 would let a diagonal reach 2^24).
// An item covers the d evaluation indices that share one filter word (d <= 8)
// and up to 8 / d image groups, so that one filter unit in shared memory
// serves B columns N = 8 NB <= 128 (the MMA costs the same per instruction up
// to N = 128).
static bool tc_geom(u32 n, u32 d, const DevLayer& L, TcGeom& G, size_t& smem) {
    if (L.T == 0 || L.T > 128 || L.GB == 0 || L.Co == 0 || d == 0 || n % d) return false;
    const u32 dj = d <= 8 ? d : 1, gmax = 8 / dj;
    u32 gbt = 1, lg = 0;
    while (2 * gbt <= gmax && 2 * gbt <= L.GB) gbt *= 2, lg++;
    G.dj = dj;
    G.gbt = gbt;
    G.lgbt = lg;
    G.NB = 2 * gbt * dj;
    G.KB = (L.T + 15) / 16;
    G.n_ct = (L.Co + 127) / 128;
    G.n_gbg = (L.GB + gbt - 1) / gbt;
    G.co_pad = 128 * (G.n_ct - 1) + tile_rows8(L.Co, G.n_ct - 1);
    const u64 items = (u64)L.beta * (n / dj) * G.n_ct * G.n_gbg;
    if (items > 0x7FFFFFFFull) return false;
    G.n_items = (u32)items;
    const u32 rp = tile_rows8(L.Co, 0);  // the widest tile
    // the A operand region: the digit planes, and room for the 128-row reads of the last plane
    G.az = 256 * rp > 7 * 32 * rp + 4096 ? 256 * rp : 7 * 32 * rp + 4096;
    G.ssz = G.az + 256 * G.NB + 2 * 32 * G.NB * 8;  // A, the input digit planes, two input-word buffers
    G.off_slot = 1024 + 4096;
    const size_t budget = 227 * 1024;
    size_t nc = (budget - G.off_slot) / G.ssz;
    if (nc < 2) return false;
    G.NC = (u32)(nc > kMaxConv ? kMaxConv : nc);
    smem = G.off_slot + (size_t)G.NC * G.ssz;
    return smem <= budget;
}

bool homconv_tc_supported(u32 n, const DevLayer& L) {
    TcGeom G;
    size_t smem;
    return tc_geom(n, 1, L, G, smem);  // the shared-memory need depends on NB <= 16 alone
}

// Words (u64) of the tensor-core filter layout: 256 bytes per row per
// (group of d evaluation indices, ciphertext block), rows padded per tile to
// a multiple of 8.
u64 filter_tc_words(u32 n, u32 d, const DevLayer& L) {
    const u32 n_ct = (L.Co + 127) / 128, co_pad = 128 * (n_ct - 1) + tile_rows8(L.Co, n_ct - 1);
    return (u64)L.beta * (n / d) * ((L.T + 15) / 16) * co_pad * 32;
}

cudaError_t launch_filter_tc(const DevParams& P, const DevLayer& L, const u64* Phat, u64* Ptc, cudaStream_t s) {
    const u32 nJ = L.beta * P.n / P.d, KB = (L.T + 15) / 16;
    const u32 n_ct = (L.Co + 127) / 128, co_pad = 128 * (n_ct - 1) + tile_rows8(L.Co, n_ct - 1);
    cudaError_t e = cudaMemsetAsync(Ptc, 0, filter_tc_words(P.n, P.d, L) * 8, s);  // padding rows stay zero
    if (e != cudaSuccess) return e;
    dim3 grid((nJ + 63) / 64, KB, L.Co);
    filter_tc_kernel<<<grid, 128, 0, s>>>(P, L, KB, co_pad, Phat, reinterpret_cast<unsigned char*>(Ptc));
    return cudaGetLastError();
}

template <int NBH>
static cudaError_t launch_tc(const DevParams& P, const DevLayer& L, const TcGeom& G, size_t smem, const u64* ct_in,
                             const u64* A1, const u64* A2, const u64* Ptc, const u64* Mhat, u64* ct_out,
                             cudaStream_t s) {
    // once per instantiation (thread-safe: the server's worker launches too): the
    // SM count, the shared-memory opt-in at the largest size any layer uses, and
    // the address of the error word
    static std::once_flag once;
    static cudaError_t init = cudaSuccess;
    static int sms = 0;
    static u32* errp = nullptr;
    std::call_once(once, [] {
        int dev = 0;
        init = cudaGetDevice(&dev);
        if (init == cudaSuccess) init = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (init == cudaSuccess)
            init = cudaFuncSetAttribute(homconv_tc_kernel<NBH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        227 * 1024);
        if (init == cudaSuccess) init = cudaGetSymbolAddress((void**)&errp, g_tc_err);
    });
    if (init != cudaSuccess) return init;
    const u32 grid = G.n_items < (u32)sms ? G.n_items : (u32)sms;
    homconv_tc_kernel<NBH><<<grid, kThreadsTC, smem, s>>>(P, L, G, ct_in, A1, A2,
                                                         reinterpret_cast<const unsigned char*>(Ptc), Mhat, ct_out,
                                                         errp);
    return cudaGetLastError();
}

cudaError_t launch_homconv_tc(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                              const u64* Ptc, const u64* Mhat, u64* ct_out, cudaStream_t s) {
    TcGeom G;
    size_t smem;
    if (!tc_geom(P.n, P.d, L, G, smem)) return cudaErrorInvalidValue;
    switch (G.NB / 2) {
        case 1: return launch_tc<1>(P, L, G, smem, ct_in, A1, A2, Ptc, Mhat, ct_out, s);
        case 2: return launch_tc<2>(P, L, G, smem, ct_in, A1, A2, Ptc, Mhat, ct_out, s);
        case 4: return launch_tc<4>(P, L, G, smem, ct_in, A1, A2, Ptc, Mhat, ct_out, s);
        default: return launch_tc<8>(P, L, G, smem, ct_in, A1, A2, Ptc, Mhat, ct_out, s);
    }
}

// The error word of the tensor-core kernel (0: no CTA gave up waiting).
u32 homconv_tc_error(bool reset) {
    u32 v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_err, sizeof(u32)) != cudaSuccess) return 0;
    if (reset && v) {
        const u32 z = 0;
        cudaMemcpyToSymbol(g_tc_err, &z, sizeof(u32));
    }
    return v;
}
