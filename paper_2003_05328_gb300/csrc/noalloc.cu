// noalloc.cu -- one online layer without any device allocation.
//
// Some callers cannot let a library allocate device memory: a host
// application whose device memory is entirely reserved by its own pooling
// allocator (an allocation from inside this library would fail, or carve
// into memory the application has promised elsewhere), and latency-critical
// request threads that must never enter the CUDA allocator, whose calls can
// block on device-wide synchronisation.  For them, fdsc_layer_online_noalloc
// runs the fused online path of one layer -- the same kernels, in the same
// order, as fdsc_encrypt_constants, fdsc_encode_share (twice),
// fdsc_homconv_sum, fdsc_decrypt_share and fdsc_intt2d -- with the
// intermediate ciphertexts in the fixed array below instead of caller or
// library allocations.  The caller still passes every input and output.
#include <mutex>

#include "fdsc_internal.h"

namespace {

// Every device that loads the library holds this array until the process
// exits.  Host code must not use its name as a device address: the address
// comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FDSC_NOALLOC_SCRATCH_BYTES];

// The array's device address, looked up once per CUDA context with that
// context current and remembered under the context's handle, so that a
// context created after a device reset (cudaDeviceReset) gets its own
// lookup instead of an address that belonged to the old one.
constexpr int kMaxContexts = 64;
std::mutex g_scratch_mu;
struct ScratchEntry {
    void* ctx;
    void* addr;
};
ScratchEntry g_scratch[kMaxContexts] = {};
int g_scratch_used = 0;

typedef int (*CtxGetCurrentFn)(void**);  // the driver's cuCtxGetCurrent

int scratch_on_current_device(void** out) {
    static CtxGetCurrentFn ctx_get_current = nullptr;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!ctx_get_current) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult st;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &st);
        if (e != cudaSuccess || st != cudaDriverEntryPointSuccess || !fn)
            return fdsc_set_error(FDSC_ERR_CUDA, "cuCtxGetCurrent not available: %s", cudaGetErrorString(e));
        ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    }
    void* ctx = nullptr;
    if (ctx_get_current(&ctx) != 0 || !ctx) return fdsc_set_error(FDSC_ERR_CUDA, "no current CUDA context");
    for (int i = 0; i < g_scratch_used; i++)
        if (g_scratch[i].ctx == ctx) {
            *out = g_scratch[i].addr;
            return FDSC_OK;
        }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fdsc_set_error(FDSC_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    // a full table forgets its oldest context
    const int slot = g_scratch_used < kMaxContexts ? g_scratch_used++ : 0;
    g_scratch[slot] = {ctx, p};
    *out = p;
    return FDSC_OK;
}

u64 round256(u64 b) { return (b + 255) & ~(u64)255; }

}  // namespace

extern "C" int fdsc_layer_online_noalloc(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat,
                                         uint64_t enc_seed, const uint64_t* P_hat, const uint64_t* M_hat,
                                         const uint32_t* sB_hat, const uint32_t* xA, const uint32_t* xB, uint32_t* yA,
                                         uint32_t* yB, void* stream) {
    int rc = fdsc_check_params(P);
    if (rc) return rc;
    DevLayer D;
    fdsc_layout lay;
    if ((rc = fdsc_make_layer(P->info, L, &D, &lay))) return rc;
    // exactly what the fused calls it runs accept
    if ((rc = fdsc_check_fused(P, D, share_smem_bytes(P->dev, D), "layer_online_noalloc")) ||
        (rc = fdsc_check_fused(P, D, decrypt_share_smem_bytes(P->dev, D), "layer_online_noalloc")))
        return rc;
    if (D.T > P->max_T)
        return fdsc_set_error(FDSC_ERR_NOISE, "T = %u exceeds the params' max_T = %u", D.T, P->max_T);
    const void* ptrs[] = {t_hat, P_hat, M_hat, sB_hat, xA, xB, yA, yB};
    const char* names[] = {"t_hat", "P_hat", "M_hat", "sB_hat", "xA", "xB", "yA", "yB"};
    for (int i = 0; i < 8; i++) {
        if (!ptrs[i]) return fdsc_set_error(FDSC_ERR_ARG, "%s is NULL", names[i]);
        if (reinterpret_cast<uintptr_t>(ptrs[i]) & 15) return fdsc_set_error(FDSC_ERR_ARG, "%s is not 16-byte aligned", names[i]);
    }
    // scratch: ct [n_in][2][n] | A [n_in][n] | R [n_in][n] | ct_out [n_out][2][n]
    const u64 n = P->info.n;
    const u64 o_A = round256(lay.ct_in_words * 8);
    const u64 o_R = o_A + round256((u64)D.n_in * n * 8);
    const u64 o_out = o_R + round256((u64)D.n_in * n * 8);
    const u64 need = o_out + round256(lay.ct_out_words * 8);
    if (need > FDSC_NOALLOC_SCRATCH_BYTES)
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED,
                              "layer needs %llu bytes of intermediate ciphertexts; the fixed array holds %u",
                              (unsigned long long)need, (unsigned)FDSC_NOALLOC_SCRATCH_BYTES);
    void* base = nullptr;
    if ((rc = scratch_on_current_device(&base))) return rc;
    unsigned char* sc = static_cast<unsigned char*>(base);
    u64* ct = reinterpret_cast<u64*>(sc);
    u64* A = reinterpret_cast<u64*>(sc + o_A);
    u64* R = reinterpret_cast<u64*>(sc + o_R);
    u64* ct_out = reinterpret_cast<u64*>(sc + o_out);
    // every scratch word is written before it is read, so nothing needs clearing
    cudaStream_t s = (cudaStream_t)stream;
    const DevParams& DP = P->dev;
    cudaError_t e = launch_constants(DP, D, t_hat, 0, enc_seed, nullptr, ct, s);
    if (e == cudaSuccess) e = launch_share(DP, D, xA, A, false, s);
    if (e == cudaSuccess) e = launch_share(DP, D, xB, R, false, s);
    if (e == cudaSuccess) e = launch_homconv(DP, D, ct, A, R, P_hat, M_hat, ct_out, s);
    if (e == cudaSuccess) e = launch_decrypt_share(DP, D, t_hat, 0, ct_out, yA, s);
    if (e == cudaSuccess) e = launch_ntt2d(DP, D.H, D.W, sB_hat, yB, (u64)D.B * D.Co, true, s);
    if (e != cudaSuccess) return fdsc_set_error(FDSC_ERR_CUDA, "layer_online_noalloc: %s", cudaGetErrorString(e));
    return FDSC_OK;
}
