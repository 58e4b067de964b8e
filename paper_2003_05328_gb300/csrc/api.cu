// api.cu -- the compute entry points of the libfdsc C ABI: argument checks,
// then one kernel launch each on the caller's stream.
#include "fdsc_internal.h"

int fdsc_check_params(const fdsc_params* P) {
    if (!P) return fdsc_set_error(FDSC_ERR_ARG, "params is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fdsc_set_error(FDSC_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev != P->device)
        return fdsc_set_error(FDSC_ERR_ARG, "params were created on device %d but device %d is current", P->device,
                              dev);
    return FDSC_OK;
}

namespace {

int check_params(const fdsc_params* P) { return fdsc_check_params(P); }

int check_ptr(const void* p, const char* name, bool align16 = true) {
    if (!p) return fdsc_set_error(FDSC_ERR_ARG, "%s is NULL", name);
    if (align16 && (reinterpret_cast<uintptr_t>(p) & 15))
        return fdsc_set_error(FDSC_ERR_ARG, "%s is not 16-byte aligned", name);
    return FDSC_OK;
}

int launched(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return FDSC_OK;
    return fdsc_set_error(FDSC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool overlap(const void* a, u64 abytes, const void* b, u64 bbytes) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + bbytes && y < x + abytes;
}

int ntt2d_common(const fdsc_params* P, uint32_t H, uint32_t W, const uint32_t* x, uint32_t* X, uint64_t planes,
                 void* stream, bool inverse) {
    int rc = check_params(P);
    if (rc) return rc;
    if (H < 2 || W < 2 || (H & (H - 1)) || (W & (W - 1)))
        return fdsc_set_error(FDSC_ERR_ARG, "H = %u, W = %u: powers of two >= 2 required", H, W);
    if (H > P->dev.lmax || W > P->dev.lmax || (u64)H * W > FDSC_MAX_HW)
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED, "plane %ux%u exceeds H, W <= %u, HW <= %u", H, W, P->dev.lmax,
                              FDSC_MAX_HW);
    if (planes == 0) return FDSC_OK;
    if ((rc = check_ptr(x, "x")) || (rc = check_ptr(X, "X"))) return rc;
    return launched(launch_ntt2d(P->dev, H, W, x, X, planes, inverse, (cudaStream_t)stream),
                    inverse ? "intt2d" : "ntt2d");
}

}  // namespace

extern "C" int fdsc_ntt2d(const fdsc_params* P, uint32_t H, uint32_t W, const uint32_t* x, uint32_t* X,
                          uint64_t planes, void* stream) {
    return ntt2d_common(P, H, W, x, X, planes, stream, false);
}

extern "C" int fdsc_intt2d(const fdsc_params* P, uint32_t H, uint32_t W, const uint32_t* X, uint32_t* x,
                           uint64_t planes, void* stream) {
    return ntt2d_common(P, H, W, X, x, planes, stream, true);
}

extern "C" int fdsc_pool2x2_sum(const fdsc_params* P, uint32_t H, uint32_t W, const uint32_t* x, uint32_t* y,
                                uint64_t planes, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    if (H < 2 || W < 2 || (H & 1) || (W & 1)) return fdsc_set_error(FDSC_ERR_ARG, "pooling needs even H, W >= 2");
    if ((rc = check_ptr(x, "x")) || (rc = check_ptr(y, "y"))) return rc;
    const u64 in_bytes = planes * H * W * 4, out_bytes = planes * (H / 2) * (W / 2) * 4;
    if (overlap(x, in_bytes, y, out_bytes)) return fdsc_set_error(FDSC_ERR_ARG, "x and y overlap");
    return launched(launch_pool2x2(P->dev, H, W, x, y, planes, (cudaStream_t)stream), "pool2x2_sum");
}

extern "C" int fdsc_keygen(const fdsc_params* P, uint64_t seed, uint64_t* t_hat, void* stream) {
    int rc = check_params(P);
    if (rc || (rc = check_ptr(t_hat, "t_hat"))) return rc;
    return launched(launch_keygen(P->dev, seed, t_hat, (cudaStream_t)stream), "keygen");
}

extern "C" int fdsc_encrypt(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat, const uint32_t* X,
                            uint64_t seed, uint64_t* ct, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_ptr(t_hat, "t_hat")) || (rc = check_ptr(X, "X")) || (rc = check_ptr(ct, "ct"))) return rc;
    return launched(launch_encrypt(P->dev, D, t_hat, X, seed, ct, (cudaStream_t)stream), "encrypt");
}

extern "C" int fdsc_homrec(const fdsc_params* P, const fdsc_layer* L, const uint32_t* XB, uint64_t* ct,
                           void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_ptr(XB, "XB")) || (rc = check_ptr(ct, "ct"))) return rc;
    return launched(launch_homrec(P->dev, D, XB, ct, (cudaStream_t)stream), "homrec");
}

extern "C" int fdsc_filter_prepare(const fdsc_params* P, const fdsc_layer* L, const int8_t* w, uint32_t fh,
                                   uint32_t fw, uint64_t* P_hat, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if (fh == 0 || fw == 0 || fh > D.H || fw > D.W)
        return fdsc_set_error(FDSC_ERR_ARG, "filter %ux%u must fit the %ux%u plane", fh, fw, D.H, D.W);
    if ((rc = check_ptr(w, "w", false)) || (rc = check_ptr(P_hat, "P_hat"))) return rc;
    return launched(launch_filter_prepare(P->dev, D, w, fh, fw, P_hat, (cudaStream_t)stream), "filter_prepare");
}

extern "C" int fdsc_mask_prepare(const fdsc_params* P, const fdsc_layer* L, uint64_t seed, uint64_t* M_hat,
                                 uint32_t* sB_hat, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_ptr(M_hat, "M_hat")) || (rc = check_ptr(sB_hat, "sB_hat"))) return rc;
    return launched(launch_mask_prepare(P->dev, D, seed, nullptr, 0, M_hat, sB_hat, (cudaStream_t)stream), "mask_prepare");
}

extern "C" int fdsc_mask_prepare_flooded(const fdsc_params* P, const fdsc_layer* L, uint64_t seed, uint32_t flood_bits,
                                         uint64_t* M_hat, uint32_t* sB_hat, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if (flood_bits > FDSC_MAX_FLOOD_BITS || !fdsc_noise_ok_flood(P->info, D.T, flood_bits))
        return fdsc_set_error(FDSC_ERR_NOISE, "flooding of 2^%u breaks the noise bound at T = %u", flood_bits, D.T);
    if ((rc = check_ptr(M_hat, "M_hat")) || (rc = check_ptr(sB_hat, "sB_hat"))) return rc;
    return launched(launch_mask_prepare(P->dev, D, seed, nullptr, flood_bits, M_hat, sB_hat, (cudaStream_t)stream),
                    "mask_prepare_flooded");
}

extern "C" int fdsc_flood_bits_max(uint32_t n, uint32_t p, uint32_t T, uint32_t* out) {
    if (!out) return fdsc_set_error(FDSC_ERR_ARG, "out is NULL");
    fdsc_params_info I;
    int rc = fdsc_params_query(n, p, &I);
    if (rc) return rc;
    if (!fdsc_noise_ok(I, T)) return fdsc_set_error(FDSC_ERR_NOISE, "noise bound fails for T = %u", T);
    u32 f = 0;
    while (f < FDSC_MAX_FLOOD_BITS && fdsc_noise_ok_flood(I, T, f + 1)) f++;
    *out = f;
    return FDSC_OK;
}

extern "C" int fdsc_homconv(const fdsc_params* P, const fdsc_layer* L, const uint64_t* ct_in, const uint64_t* P_hat,
                            const uint64_t* M_hat, uint64_t* ct_out, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    fdsc_layout lay;
    if ((rc = fdsc_make_layer(P->info, L, &D, &lay))) return rc;
    if (D.T > P->max_T)
        return fdsc_set_error(FDSC_ERR_NOISE, "T = %u input ciphertexts exceed the params' noise budget (max_T = %u)",
                              D.T, P->max_T);
    if ((rc = check_ptr(ct_in, "ct_in")) || (rc = check_ptr(P_hat, "P_hat")) || (rc = check_ptr(ct_out, "ct_out")))
        return rc;
    if (M_hat && (rc = check_ptr(M_hat, "M_hat"))) return rc;
    if (overlap(ct_in, lay.ct_in_words * 8, ct_out, lay.ct_out_words * 8))
        return fdsc_set_error(FDSC_ERR_ARG, "ct_out overlaps ct_in");
    return launched(launch_homconv(P->dev, D, ct_in, nullptr, nullptr, P_hat, M_hat, ct_out, (cudaStream_t)stream),
                    "homconv");
}

extern "C" int fdsc_decrypt(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat, const uint64_t* ct,
                            uint32_t* SA_hat, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_ptr(t_hat, "t_hat")) || (rc = check_ptr(ct, "ct")) || (rc = check_ptr(SA_hat, "SA_hat")))
        return rc;
    return launched(launch_decrypt(P->dev, D, t_hat, ct, SA_hat, (cudaStream_t)stream), "decrypt");
}

// ---------------------------------------------------------------- fused online path
// The fused spatial-domain kernels need radix-8 lines (8 <= H, W <= 512)
// and their shared memory to fit (a spectrum spanning several ciphertexts,
// H W > S, keeps the d whole planes of its images on chip).
int fdsc_check_fused(const fdsc_params* P, const DevLayer& D, size_t smem, const char* what) {
    if (D.logH < 3 || D.logW < 3 || D.logH > 9 || D.logW > 9)
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED,
                              "%s needs 8 <= H, W <= 512; use fdsc_ntt2d/fdsc_encrypt/fdsc_decrypt", what);
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
    if (e != cudaSuccess) return fdsc_set_error(FDSC_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    if (smem + 1024 > (size_t)optin)
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED, "%s needs %zu bytes of shared memory", what, smem);
    return FDSC_OK;
}

namespace {
int check_fused(const fdsc_params* P, const DevLayer& D, size_t smem, const char* what) {
    return fdsc_check_fused(P, D, smem, what);
}
}  // namespace

extern "C" int fdsc_encrypt_constants(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat, uint64_t seed,
                                      uint64_t* ct, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_ptr(t_hat, "t_hat")) || (rc = check_ptr(ct, "ct"))) return rc;
    return launched(launch_constants(P->dev, D, t_hat, 0, seed, nullptr, ct, (cudaStream_t)stream), "encrypt_constants");
}

extern "C" int fdsc_encode_share(const fdsc_params* P, const fdsc_layer* L, const uint32_t* x, uint64_t* A,
                                 void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_fused(P, D, share_smem_bytes(P->dev, D), "encode_share"))) return rc;
    if ((rc = check_ptr(x, "x")) || (rc = check_ptr(A, "A"))) return rc;
    return launched(launch_share(P->dev, D, x, A, false, (cudaStream_t)stream), "encode_share");
}

extern "C" int fdsc_online_produce(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat, uint64_t seed,
                                   const uint32_t* xA, const uint32_t* xB, uint64_t* ct, uint64_t* A, uint64_t* R,
                                   const uint64_t* P_hat, const uint64_t* M_hat, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    fdsc_layout lay;
    if ((rc = fdsc_make_layer(P->info, L, &D, &lay))) return rc;
    if ((rc = check_fused(P, D, produce_smem_bytes(P->dev, D), "online_produce"))) return rc;
    if ((rc = check_ptr(t_hat, "t_hat")) || (rc = check_ptr(xA, "xA")) || (rc = check_ptr(xB, "xB")) ||
        (rc = check_ptr(ct, "ct")) || (rc = check_ptr(A, "A")) || (rc = check_ptr(R, "R")))
        return rc;
    if ((P_hat && (rc = check_ptr(P_hat, "P_hat"))) || (M_hat && (rc = check_ptr(M_hat, "M_hat")))) return rc;
    const u64 cb = lay.ct_in_words * 8, ab = (u64)D.n_in * P->info.n * 8;
    if (overlap(ct, cb, A, ab) || overlap(ct, cb, R, ab) || overlap(A, ab, R, ab))
        return fdsc_set_error(FDSC_ERR_ARG, "ct, A and R must not overlap");
    return launched(launch_produce(P->dev, D, t_hat, seed, xA, xB, ct, A, R, P_hat, P_hat ? lay.filter_words * 8 : 0,
                                   M_hat, M_hat ? lay.mask_words * 8 : 0, (cudaStream_t)stream),
                    "online_produce");
}

extern "C" int fdsc_homrec_share(const fdsc_params* P, const fdsc_layer* L, const uint32_t* xB, uint64_t* ct,
                                 void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_fused(P, D, share_smem_bytes(P->dev, D), "homrec_share"))) return rc;
    if ((rc = check_ptr(xB, "xB")) || (rc = check_ptr(ct, "ct"))) return rc;
    return launched(launch_share(P->dev, D, xB, ct, true, (cudaStream_t)stream), "homrec_share");
}

extern "C" int fdsc_homconv_sum(const fdsc_params* P, const fdsc_layer* L, const uint64_t* ct_in, const uint64_t* A1,
                                const uint64_t* A2, const uint64_t* P_hat, const uint64_t* M_hat, uint64_t* ct_out,
                                void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    fdsc_layout lay;
    if ((rc = fdsc_make_layer(P->info, L, &D, &lay))) return rc;
    if (D.T > P->max_T)
        return fdsc_set_error(FDSC_ERR_NOISE, "T = %u input ciphertexts exceed the params' noise budget (max_T = %u)",
                              D.T, P->max_T);
    if ((rc = check_ptr(ct_in, "ct_in")) || (rc = check_ptr(P_hat, "P_hat")) || (rc = check_ptr(ct_out, "ct_out")))
        return rc;
    if ((A1 && (rc = check_ptr(A1, "A1"))) || (A2 && (rc = check_ptr(A2, "A2"))) ||
        (M_hat && (rc = check_ptr(M_hat, "M_hat"))))
        return rc;
    const u64 ob = lay.ct_out_words * 8, ab = (u64)D.n_in * P->info.n * 8;
    if (overlap(ct_in, lay.ct_in_words * 8, ct_out, ob) || (A1 && overlap(A1, ab, ct_out, ob)) ||
        (A2 && overlap(A2, ab, ct_out, ob)))
        return fdsc_set_error(FDSC_ERR_ARG, "ct_out overlaps an input");
    return launched(launch_homconv(P->dev, D, ct_in, A1, A2, P_hat, M_hat, ct_out, (cudaStream_t)stream),
                    "homconv_sum");
}

// ---------------------------------------------------------------- tensor-core HomConv
extern "C" int fdsc_filter_tc_words(uint32_t n, uint32_t p, const fdsc_layer* L, uint64_t* words) {
    if (!L || !words) return fdsc_set_error(FDSC_ERR_ARG, "layer or words is NULL");
    fdsc_params_info I;
    int rc = fdsc_derive(n, p, &I);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(I, L, &D, nullptr))) return rc;
    if (!homconv_tc_supported(n, D))
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED, "the tensor-core HomConv needs T <= 128 (T = %u)", D.T);
    *words = filter_tc_words(n, I.d, D);
    return FDSC_OK;
}

extern "C" int fdsc_filter_tc(const fdsc_params* P, const fdsc_layer* L, const uint64_t* P_hat, uint64_t* P_tc,
                              void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    fdsc_layout lay;
    if ((rc = fdsc_make_layer(P->info, L, &D, &lay))) return rc;
    if (!homconv_tc_supported(P->info.n, D))
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED, "the tensor-core HomConv needs T <= 128 (T = %u)", D.T);
    if ((rc = check_ptr(P_hat, "P_hat")) || (rc = check_ptr(P_tc, "P_tc"))) return rc;
    if (overlap(P_hat, lay.filter_words * 8, P_tc, filter_tc_words(P->info.n, P->info.d, D) * 8))
        return fdsc_set_error(FDSC_ERR_ARG, "P_tc overlaps P_hat");
    return launched(launch_filter_tc(P->dev, D, P_hat, P_tc, (cudaStream_t)stream), "filter_tc");
}

extern "C" int fdsc_homconv_tc(const fdsc_params* P, const fdsc_layer* L, const uint64_t* ct_in, const uint64_t* A1,
                               const uint64_t* A2, const uint64_t* P_tc, const uint64_t* M_hat, uint64_t* ct_out,
                               void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    fdsc_layout lay;
    if ((rc = fdsc_make_layer(P->info, L, &D, &lay))) return rc;
    if (D.T > P->max_T)
        return fdsc_set_error(FDSC_ERR_NOISE, "T = %u input ciphertexts exceed the params' noise budget (max_T = %u)",
                              D.T, P->max_T);
    if (!homconv_tc_supported(P->info.n, D))
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED, "the tensor-core HomConv needs T <= 128 (T = %u)", D.T);
    if ((rc = check_ptr(ct_in, "ct_in")) || (rc = check_ptr(P_tc, "P_tc")) || (rc = check_ptr(ct_out, "ct_out")))
        return rc;
    if ((A1 && (rc = check_ptr(A1, "A1"))) || (A2 && (rc = check_ptr(A2, "A2"))) ||
        (M_hat && (rc = check_ptr(M_hat, "M_hat"))))
        return rc;
    const u64 ob = lay.ct_out_words * 8, ab = (u64)D.n_in * P->info.n * 8;
    if (overlap(ct_in, lay.ct_in_words * 8, ct_out, ob) || (A1 && overlap(A1, ab, ct_out, ob)) ||
        (A2 && overlap(A2, ab, ct_out, ob)) || overlap(P_tc, filter_tc_words(P->info.n, P->info.d, D) * 8, ct_out, ob))
        return fdsc_set_error(FDSC_ERR_ARG, "ct_out overlaps an input");
    return launched(launch_homconv_tc(P->dev, D, ct_in, A1, A2, P_tc, M_hat, ct_out, (cudaStream_t)stream),
                    "homconv_tc");
}

extern "C" int fdsc_homconv_tc_status(uint32_t* code) {
    if (!code) return fdsc_set_error(FDSC_ERR_ARG, "code is NULL");
    *code = homconv_tc_error(true);
    if (*code) return fdsc_set_error(FDSC_ERR_TIMEOUT, "a tensor-core HomConv CTA gave up waiting (role %u)", *code);
    return FDSC_OK;
}

extern "C" int fdsc_encrypt_constants_seeded(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat,
                                             uint64_t seed, uint64_t* c1, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_ptr(t_hat, "t_hat")) || (rc = check_ptr(c1, "c1"))) return rc;
    return launched(launch_constants(P->dev, D, t_hat, 0, seed, nullptr, c1, (cudaStream_t)stream, true),
                    "encrypt_constants_seeded");
}

extern "C" int fdsc_homconv_seeded(const fdsc_params* P, const fdsc_layer* L, uint64_t seed, const uint64_t* c1,
                                   const uint64_t* A1, const uint64_t* A2, const uint64_t* P_hat,
                                   const uint64_t* M_hat, uint64_t* ct_out, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    fdsc_layout lay;
    if ((rc = fdsc_make_layer(P->info, L, &D, &lay))) return rc;
    if (D.T > P->max_T)
        return fdsc_set_error(FDSC_ERR_NOISE, "T = %u input ciphertexts exceed the params' noise budget (max_T = %u)",
                              D.T, P->max_T);
    if (D.T > 256) return fdsc_set_error(FDSC_ERR_UNSUPPORTED, "seeded HomConv stages T <= 256 input ciphertexts");
    if ((rc = check_ptr(c1, "c1")) || (rc = check_ptr(P_hat, "P_hat")) || (rc = check_ptr(ct_out, "ct_out")))
        return rc;
    if ((A1 && (rc = check_ptr(A1, "A1"))) || (A2 && (rc = check_ptr(A2, "A2"))) ||
        (M_hat && (rc = check_ptr(M_hat, "M_hat"))))
        return rc;
    const u64 ob = lay.ct_out_words * 8, ab = (u64)D.n_in * P->info.n * 8;
    if (overlap(c1, ab, ct_out, ob) || (A1 && overlap(A1, ab, ct_out, ob)) || (A2 && overlap(A2, ab, ct_out, ob)))
        return fdsc_set_error(FDSC_ERR_ARG, "ct_out overlaps an input");
    return launched(launch_homconv_seeded(P->dev, D, seed, c1, A1, A2, P_hat, M_hat, ct_out, (cudaStream_t)stream),
                    "homconv_seeded");
}

extern "C" int fdsc_decrypt_share(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hat,
                                  const uint64_t* ct, uint32_t* y, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_fused(P, D, decrypt_share_smem_bytes(P->dev, D), "decrypt_share"))) return rc;
    if ((rc = check_ptr(t_hat, "t_hat")) || (rc = check_ptr(ct, "ct")) || (rc = check_ptr(y, "y"))) return rc;
    return launched(launch_decrypt_share(P->dev, D, t_hat, 0, ct, y, (cudaStream_t)stream), "decrypt_share");
}

// ---------------------------------------------------------------- several clients in one call
extern "C" int fdsc_encrypt_constants_multi(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hats,
                                            uint64_t key_stride, const uint64_t* seeds, uint64_t* ct, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_ptr(t_hats, "t_hats")) || (rc = check_ptr(seeds, "seeds", false)) || (rc = check_ptr(ct, "ct")))
        return rc;
    if (key_stride % 2) return fdsc_set_error(FDSC_ERR_ARG, "key_stride must keep keys 16-byte aligned");
    return launched(launch_constants(P->dev, D, t_hats, key_stride, 0, seeds, ct, (cudaStream_t)stream),
                    "encrypt_constants_multi");
}

extern "C" int fdsc_mask_prepare_multi(const fdsc_params* P, const fdsc_layer* L, const uint64_t* seeds,
                                       uint64_t* M_hat, uint32_t* sB_hat, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_ptr(seeds, "seeds", false)) || (rc = check_ptr(M_hat, "M_hat")) ||
        (rc = check_ptr(sB_hat, "sB_hat")))
        return rc;
    return launched(launch_mask_prepare(P->dev, D, 0, seeds, 0, M_hat, sB_hat, (cudaStream_t)stream),
                    "mask_prepare_multi");
}

extern "C" int fdsc_decrypt_share_multi(const fdsc_params* P, const fdsc_layer* L, const uint64_t* t_hats,
                                        uint64_t key_stride, const uint64_t* ct, uint32_t* y, void* stream) {
    int rc = check_params(P);
    if (rc) return rc;
    DevLayer D;
    if ((rc = fdsc_make_layer(P->info, L, &D, nullptr))) return rc;
    if ((rc = check_fused(P, D, decrypt_share_smem_bytes(P->dev, D), "decrypt_share_multi"))) return rc;
    if ((rc = check_ptr(t_hats, "t_hats")) || (rc = check_ptr(ct, "ct")) || (rc = check_ptr(y, "y"))) return rc;
    if (key_stride % 2) return fdsc_set_error(FDSC_ERR_ARG, "key_stride must keep keys 16-byte aligned");
    return launched(launch_decrypt_share(P->dev, D, t_hats, key_stride, ct, y, (cudaStream_t)stream),
                    "decrypt_share_multi");
}
