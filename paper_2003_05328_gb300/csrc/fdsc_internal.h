// fdsc_internal.h -- shared host/device definitions of libfdsc.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fdsc.h"

typedef uint64_t u64;
typedef uint32_t u32;

// Largest cyclic transform length the NTT2D tables cover (H, W <= LMAX).
#define FDSC_LMAX 4096u
// Largest padded plane a CTA transforms in shared memory.
#define FDSC_MAX_HW 4096u

// Everything a kernel needs about (n, p, q): passed by value.
struct DevParams {
    u32 n, logn, p, S, logS, d;
    u32 Sinv, Sinv_s;      // S^-1 mod p and its 32-bit Shoup companion
    u32 lmax, loglmax;     // NTT2D twiddle table covers w_lmax^k, k < lmax/2
    u32 g_p;               // the primitive root of p the roots of unity come from
    u64 q, twoq, delta;
    u64 r64, r64_s;        // 2^64 mod q, floor(r64 2^64 / q)
    u64 one_s;             // floor(2^64 / q): Shoup companion of 1
    u64 round_k;           // floor(p 2^64 / q)
    u64 mu;                // floor(2^122 / q): Barrett constant of muladd_q
    u64 ninv, ninv_s;      // n^-1 mod q and companion
    const u64* qfw;        // psi_q^brv_n(k), k < n
    const u64* qfw_s;
    const u64* qinv;       // psi_q^-brv_n(k)
    const u64* qinv_s;
    const u32* pfw;        // psi_p^brv_S(k), k < S
    const u32* pfw_s;
    const u32* pinv;
    const u32* pinv_s;
    const u32* w2d;        // w_lmax^k, k < lmax/2
    const u32* w2d_s;
    const u32* w2di;       // w_lmax^-k
    const u32* w2di_s;
    const u64* cdt;        // [19] Gaussian cumulative table
    // the same twiddles interleaved with their Shoup companions
    const ulonglong2* qfw2;  // (psi^brv(k), companion), k < n
    const ulonglong2* qinv2;
    const uint2* pfw2;       // k < S
    const uint2* pinv2;
    const uint2* lpf;        // line twiddles: (w_L^k, companion) at L/2 + k, L <= lmax
    const uint2* lpi;        // the same for w_L^-k
};

// A layer with its packing, derived (all counts fit in 32 bits).
struct DevLayer {
    u32 B, Ci, Co, H, W, HW, logH, logW;
    u32 g_c, g_b, T, GB, beta, n_in, n_out;
};

struct fdsc_params {
    fdsc_params_info info;
    DevParams dev;
    u32 max_T;
    int device;
    void* table_mem;  // one device allocation holding every table
};

// ---- host helpers (params.cu) ----
int fdsc_set_error(int code, const char* fmt, ...);
// Argument checks shared by the entry points (api.cu): the params object
// belongs to the current device; a layer fits the fused online kernels
// (H W <= S, 8 <= H, W <= 512, `smem` bytes of shared memory per CTA).
int fdsc_check_params(const fdsc_params* P);
int fdsc_check_fused(const fdsc_params* P, const DevLayer& D, size_t smem, const char* what);

// Whether online kernels are launched with programmatic stream serialisation
// (fdsc_set_launch_overlap; off by default).
bool fdsc_launch_overlap();
// Whether one image's decryption may split each ciphertext over a CTA pair
// (fdsc_set_decrypt_pair; on by default).
bool fdsc_decrypt_pair_allowed();

#ifdef __CUDACC__
// Launches an online kernel (one that calls griddep_wait() before touching
// caller memory) so that it may start while its predecessor in the stream
// finishes.
template <typename... KArgs, typename... Args>
cudaError_t launch_online(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = fdsc_launch_overlap() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
#endif
int fdsc_derive(u32 n, u32 p, fdsc_params_info* out);
int fdsc_make_layer(const fdsc_params_info& I, const fdsc_layer* L, DevLayer* out, fdsc_layout* lay);
void fdsc_host_cdt(u64* cdt19);
bool fdsc_noise_ok(const fdsc_params_info& I, u32 T);
bool fdsc_noise_ok_flood(const fdsc_params_info& I, u32 T, u32 flood_bits);
constexpr u32 FDSC_MAX_FLOOD_BITS = 62;
u32 fdsc_shoup32(u32 w, u32 p);
u32 fdsc_powmod32(u32 b, u64 e, u32 p);

// ---- kernel launchers (return cudaError_t of the launch) ----
cudaError_t launch_ntt2d(const DevParams& P, u32 H, u32 W, const u32* x, u32* X, u64 planes, bool inverse,
                         cudaStream_t s);
cudaError_t launch_keygen(const DevParams& P, u64 seed, u64* t_hat, cudaStream_t s);
cudaError_t launch_encrypt(const DevParams& P, const DevLayer& L, const u64* t_hat, const u32* X, u64 seed,
                           u64* ct, cudaStream_t s);
cudaError_t launch_homrec(const DevParams& P, const DevLayer& L, const u32* XB, u64* ct, cudaStream_t s);
cudaError_t launch_filter_prepare(const DevParams& P, const DevLayer& L, const int8_t* w, u32 fh, u32 fw,
                                  u64* Phat, cudaStream_t s);
cudaError_t launch_mask_prepare(const DevParams& P, const DevLayer& L, u64 seed, const u64* seeds, u32 flood_bits, u64* Mhat, u32* sB,
                                cudaStream_t s);
cudaError_t launch_homconv_seeded(const DevParams& P, const DevLayer& L, u64 seed, const u64* c1, const u64* A1,
                                  const u64* A2, const u64* Phat, const u64* Mhat, u64* ct_out, cudaStream_t s);
cudaError_t launch_homconv(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                           const u64* Phat, const u64* Mhat, u64* ct_out, cudaStream_t s);
cudaError_t launch_homconv_v(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                             const u64* Phat, const u64* Mhat, u64* ct_out, int variant, cudaStream_t s);
int homconv_default_variant(const DevLayer& L);
int homconv_effective_variant(const DevLayer& L, int variant);
// tensor-core HomConv (homconv_tc.cu)
bool homconv_tc_supported(u32 n, const DevLayer& L);
u64 filter_tc_words(u32 n, u32 d, const DevLayer& L);
cudaError_t launch_filter_tc(const DevParams& P, const DevLayer& L, const u64* Phat, u64* Ptc, cudaStream_t s);
cudaError_t launch_homconv_tc(const DevParams& P, const DevLayer& L, const u64* ct_in, const u64* A1, const u64* A2,
                              const u64* Ptc, const u64* Mhat, u64* ct_out, cudaStream_t s);
u32 homconv_tc_error(bool reset);
cudaError_t launch_pool2x2(const DevParams& P, u32 H, u32 W, const u32* x, u32* y, u64 planes, cudaStream_t s);
cudaError_t launch_constants(const DevParams& P, const DevLayer& L, const u64* t_hat, u64 key_stride, u64 seed,
                             const u64* seeds, u64* ct, cudaStream_t s, bool c1_only = false);
cudaError_t launch_share(const DevParams& P, const DevLayer& L, const u32* x, u64* out, bool add_to_ct,
                         cudaStream_t s);
cudaError_t launch_decrypt_share(const DevParams& P, const DevLayer& L, const u64* t_hat, u64 key_stride, const u64* ct,
                                 u32* y, cudaStream_t s);
cudaError_t launch_produce(const DevParams& P, const DevLayer& L, const u64* t_hat, u64 seed, const u32* xA,
                           const u32* xB, u64* ct, u64* A, u64* R, const void* pf0, u64 pf0_bytes, const void* pf1,
                           u64 pf1_bytes, cudaStream_t s);
size_t produce_smem_bytes(const DevParams& P, const DevLayer& L);
size_t share_smem_bytes(const DevParams& P, const DevLayer& L);
size_t decrypt_share_smem_bytes(const DevParams& P, const DevLayer& L);
cudaError_t launch_decrypt(const DevParams& P, const DevLayer& L, const u64* t_hat, const u64* ct, u32* SA,
                           cudaStream_t s);
