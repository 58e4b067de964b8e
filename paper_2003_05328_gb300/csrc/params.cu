// params.cu -- host side of libfdsc: parameter derivation (Sec. 3.1, 5.2,
// 6.4), twiddle tables, layer validation, error reporting, and the params /
// layout entry points of the C ABI.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "fdsc_internal.h"

typedef unsigned __int128 u128;

// ---------------------------------------------------------------- errors
static thread_local char g_err[512] = "";

int fdsc_set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

extern "C" const char* fdsc_last_error(void) { return g_err; }

// ---------------------------------------------------------------- launch overlap
#include <atomic>
static std::atomic<int> g_launch_overlap{0};
bool fdsc_launch_overlap() { return g_launch_overlap.load(std::memory_order_relaxed) != 0; }
extern "C" int fdsc_set_launch_overlap(int on) { return g_launch_overlap.exchange(on ? 1 : 0); }

static std::atomic<int> g_decrypt_pair{1};
bool fdsc_decrypt_pair_allowed() { return g_decrypt_pair.load(std::memory_order_relaxed) != 0; }
extern "C" int fdsc_set_decrypt_pair(int on) { return g_decrypt_pair.exchange(on ? 1 : 0); }

// ---------------------------------------------------------------- number theory
static u64 mul_mod(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }

static u64 pow_mod(u64 base, u64 e, u64 m) {
    u64 acc = 1 % m;
    for (base %= m; e; e >>= 1, base = mul_mod(base, base, m))
        if (e & 1) acc = mul_mod(acc, base, m);
    return acc;
}

u32 fdsc_powmod32(u32 b, u64 e, u32 p) { return (u32)pow_mod(b, e, p); }

// Strong-probable-prime test to the twelve smallest prime bases, which is a
// proof of primality below 3.3e24 (Sorenson & Webster).
static bool is_prime_u64(u64 m) {
    const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (m < 2) return false;
    for (u64 b : bases)
        if (m % b == 0) return m == b;
    int r = __builtin_ctzll(m - 1);
    u64 odd = (m - 1) >> r;
    for (u64 b : bases) {
        u64 x = pow_mod(b, odd, m);
        if (x == 1 || x == m - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; i++) {
            x = mul_mod(x, x, m);
            if (x == m - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// Smallest primitive root of a prime m (distinct prime factors of m-1 by
// trial division; g generates iff no g^((m-1)/f) is 1).
static u64 smallest_generator(u64 m) {
    std::vector<u64> f;
    u64 rest = m - 1;
    for (u64 d = 2; d * d <= rest; d += (d == 2 ? 1 : 2)) {
        if (rest % d) continue;
        f.push_back(d);
        while (rest % d == 0) rest /= d;
    }
    if (rest > 1) f.push_back(rest);
    for (u64 g = 2; g < m; g++) {
        bool gen = true;
        for (u64 fi : f)
            if (pow_mod(g, (m - 1) / fi, m) == 1) { gen = false; break; }
        if (gen) return g;
    }
    return 0;
}

static u64 shoup64(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
u32 fdsc_shoup32(u32 w, u32 p) { return (u32)(((u64)w << 32) / p); }

int fdsc_derive(u32 n, u32 p, fdsc_params_info* I) {
    memset(I, 0, sizeof *I);
    if (n < 16 || n > 4096 || (n & (n - 1)))
        return fdsc_set_error(FDSC_ERR_ARG, "n = %u: need a power of two in [16, 4096]", n);
    if (p < 5 || p >= (1u << 20) || !is_prime_u64(p) || (p & 3) != 1)
        return fdsc_set_error(FDSC_ERR_ARG, "p = %u: need a prime < 2^20 with p = 1 mod 4", p);
    u32 v = __builtin_ctz(p - 1);
    u32 S = n < (1u << (v - 1)) ? n : (1u << (v - 1));
    I->n = n;
    I->logn = __builtin_ctz(n);
    I->p = p;
    I->S = S;
    I->logS = __builtin_ctz(S);
    I->d = n / S;
    I->g_p = (u32)smallest_generator(p);
    I->psi_p = (u32)pow_mod(I->g_p, (p - 1) / (2ull * S), p);
    // q: the largest prime below 2^60 that is 1 mod 8192 p.
    const u64 step = 8192ull * p;
    u64 k = ((1ull << 60) - 2) / step;
    while (k && !is_prime_u64(k * step + 1)) k--;
    I->q = k * step + 1;
    if (I->q <= (1ull << 59)) return fdsc_set_error(FDSC_ERR_ARG, "no 60-bit q for p = %u", p);
    I->g_q = smallest_generator(I->q);
    I->psi_q = pow_mod(I->g_q, (I->q - 1) / (2ull * n), I->q);
    I->delta = I->q / p;
    I->r_q = I->q % p;
    return FDSC_OK;
}

// Worst-case noise of a HomConv output summing T inputs (fresh error 19 plus
// a HomRec carry, the plaintext product's multiples of p, HomShare borrow).
// Worst-case decryption noise of a HomConv output with T input ciphertexts
// (fresh Gaussian noise times filter words, plaintext carries past p, the
// HomRec and HomShare carries), plus 2^flood_bits of HomShare flooding;
// decryption rounds correctly while p |eta| + r_q (p - 1) < q / 2.
bool fdsc_noise_ok_flood(const fdsc_params_info& I, u32 T, u32 flood_bits) {
    long double Tn = (long double)T * I.n, half = (long double)(I.p / 2);
    long double carry = ceill(Tn * (I.p - 1) * half / I.p);
    long double eta = Tn * (19.0L + I.r_q) * half + (long double)I.r_q * carry + I.r_q;
    if (flood_bits) eta += ldexpl(1.0L, (int)flood_bits);
    return eta * I.p + (long double)I.r_q * (I.p - 1) < (long double)I.q / 2;
}
bool fdsc_noise_ok(const fdsc_params_info& I, u32 T) { return fdsc_noise_ok_flood(I, T, 0); }

// Discrete Gaussian sigma = 3.2 on |x| <= 19: running sums of
// rho(0)/Z, 2 rho(k)/Z (rho(k) = exp(-k^2 / (2 sigma^2))) scaled by 2^63.
void fdsc_host_cdt(u64* cdt19) {
    const double sigma = 3.2;
    double rho[20], Z;
    for (int k = 0; k < 20; k++) rho[k] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
    Z = rho[0];
    for (int k = 1; k < 20; k++) Z += 2.0 * rho[k];
    double run = 0.0;
    for (int k = 0; k < 19; k++) {
        run += (k == 0 ? rho[0] : 2.0 * rho[k]) / Z;
        cdt19[k] = (u64)ldexp(run, 63);
    }
}

static u32 bitrev(u32 x, u32 bits) {
    u32 r = 0;
    for (u32 b = 0; b < bits; b++, x >>= 1) r = (r << 1) | (x & 1u);
    return r;
}

int fdsc_make_layer(const fdsc_params_info& I, const fdsc_layer* L, DevLayer* D, fdsc_layout* lay) {
    if (!L) return fdsc_set_error(FDSC_ERR_ARG, "layer is NULL");
    DevLayer d{};
    d.B = L->B; d.Ci = L->Ci; d.Co = L->Co; d.H = L->H; d.W = L->W; d.g_c = L->g_c; d.g_b = L->g_b;
    if (!d.B || !d.Ci || !d.Co || !d.g_c || !d.g_b)
        return fdsc_set_error(FDSC_ERR_ARG, "layer sizes and packing must be positive");
    if ((d.H & (d.H - 1)) || (d.W & (d.W - 1)) || d.H < 2 || d.W < 2)
        return fdsc_set_error(FDSC_ERR_ARG, "H = %u, W = %u: powers of two >= 2 required", d.H, d.W);
    u32 lmax = 1u << __builtin_ctz(I.p - 1);
    if (lmax > FDSC_LMAX) lmax = FDSC_LMAX;
    if (d.H > lmax || d.W > lmax || (u64)d.H * d.W > FDSC_MAX_HW)
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED, "plane %ux%u: need H, W <= %u and HW <= %u", d.H, d.W, lmax,
                              FDSC_MAX_HW);
    d.HW = d.H * d.W;
    d.logH = __builtin_ctz(d.H);
    d.logW = __builtin_ctz(d.W);
    if (d.HW <= I.S) {
        if ((u64)d.g_c * d.g_b * d.HW > I.S)
            return fdsc_set_error(FDSC_ERR_ARG, "packing g_c=%u g_b=%u needs %llu slots > S=%u", d.g_c, d.g_b,
                                  (unsigned long long)d.g_c * d.g_b * d.HW, I.S);
        d.beta = 1;
        d.T = (d.Ci + d.g_c - 1) / d.g_c;
        d.GB = (u32)((d.B + (u64)I.d * d.g_b - 1) / ((u64)I.d * d.g_b));
    } else {
        if (d.g_c != 1 || d.g_b != 1)
            return fdsc_set_error(FDSC_ERR_ARG, "HW = %u > S = %u: packing must be g_c = g_b = 1", d.HW, I.S);
        d.beta = d.HW / I.S;
        d.T = d.Ci;
        d.GB = (d.B + I.d - 1) / I.d;
    }
    u64 n_in = (u64)d.GB * d.T * d.beta, n_out = (u64)d.GB * d.Co * d.beta;
    if (n_in > (1u << 24) || n_out > (1u << 24) || (u64)d.B * d.Ci > (1u << 24) || (u64)d.B * d.Co > (1u << 24))
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED, "layer too large for one call");
    d.n_in = (u32)n_in;
    d.n_out = (u32)n_out;
    if (D) *D = d;
    if (lay) {
        lay->HW = d.HW; lay->T = d.T; lay->GB = d.GB; lay->beta = d.beta;
        lay->n_in = d.n_in; lay->n_out = d.n_out;
        lay->ct_in_words = n_in * 2 * I.n;
        lay->ct_out_words = n_out * 2 * I.n;
        lay->filter_words = (u64)d.Co * d.T * d.beta * (I.n / I.d);
        lay->mask_words = n_out * I.n;
        lay->in_spectra_words = (u64)d.B * d.Ci * d.HW;
        lay->out_spectra_words = (u64)d.B * d.Co * d.HW;
    }
    return FDSC_OK;
}

// ---------------------------------------------------------------- C ABI
extern "C" int fdsc_params_query(uint32_t n, uint32_t p, fdsc_params_info* out) {
    if (!out) return fdsc_set_error(FDSC_ERR_ARG, "out is NULL");
    return fdsc_derive(n, p, out);
}

extern "C" int fdsc_layout_query(uint32_t n, uint32_t p, const fdsc_layer* L, fdsc_layout* out) {
    fdsc_params_info I;
    int rc = fdsc_derive(n, p, &I);
    if (rc) return rc;
    if (!out) return fdsc_set_error(FDSC_ERR_ARG, "out is NULL");
    return fdsc_make_layer(I, L, nullptr, out);
}

extern "C" int fdsc_gauss_table(uint64_t* out19) {
    if (!out19) return fdsc_set_error(FDSC_ERR_ARG, "out is NULL");
    fdsc_host_cdt(out19);
    return FDSC_OK;
}

extern "C" int fdsc_params_create(uint32_t n, uint32_t p, uint32_t max_T, fdsc_params** out) {
    if (!out) return fdsc_set_error(FDSC_ERR_ARG, "out is NULL");
    *out = nullptr;
    fdsc_params_info I;
    int rc = fdsc_derive(n, p, &I);
    if (rc) return rc;
    if (max_T == 0) max_T = 1;
    if (!fdsc_noise_ok(I, max_T))
        return fdsc_set_error(FDSC_ERR_NOISE, "noise bound fails for T = %u at n = %u, p = %u", max_T, n, p);

    const u64 q = I.q;
    const u32 S = I.S;
    u32 lmax = 1u << __builtin_ctz(p - 1);
    if (lmax > FDSC_LMAX) lmax = FDSC_LMAX;
    const u32 half = lmax / 2;

    std::vector<u64> qfw(n), qfw_s(n), qinv(n), qinv_s(n);
    const u64 psi_inv = pow_mod(I.psi_q, q - 2, q);
    for (u32 k = 0; k < n; k++) {
        qfw[k] = pow_mod(I.psi_q, bitrev(k, I.logn), q);
        qinv[k] = pow_mod(psi_inv, bitrev(k, I.logn), q);
        qfw_s[k] = shoup64(qfw[k], q);
        qinv_s[k] = shoup64(qinv[k], q);
    }
    std::vector<u32> pfw(S), pfw_s(S), pinv(S), pinv_s(S);
    const u32 psip_inv = (u32)pow_mod(I.psi_p, p - 2, p);
    for (u32 k = 0; k < S; k++) {
        pfw[k] = (u32)pow_mod(I.psi_p, bitrev(k, I.logS), p);
        pinv[k] = (u32)pow_mod(psip_inv, bitrev(k, I.logS), p);
        pfw_s[k] = fdsc_shoup32(pfw[k], p);
        pinv_s[k] = fdsc_shoup32(pinv[k], p);
    }
    std::vector<u32> w2(half), w2s(half), w2i(half), w2is(half);
    const u32 wl = (u32)pow_mod(I.g_p, (p - 1) / lmax, p), wli = (u32)pow_mod(wl, p - 2, p);
    for (u32 k = 0; k < half; k++) {
        w2[k] = (u32)pow_mod(wl, k, p);
        w2i[k] = (u32)pow_mod(wli, k, p);
        w2s[k] = fdsc_shoup32(w2[k], p);
        w2is[k] = fdsc_shoup32(w2i[k], p);
    }
    u64 cdt[19];
    fdsc_host_cdt(cdt);
    std::vector<u64> qfw2(2ull * n), qinv2(2ull * n);
    for (u32 k = 0; k < n; k++) {
        qfw2[2 * k] = qfw[k];
        qfw2[2 * k + 1] = qfw_s[k];
        qinv2[2 * k] = qinv[k];
        qinv2[2 * k + 1] = qinv_s[k];
    }
    // line twiddles of every length L <= lmax, (w_L^k, companion) at entry
    // L/2 + k (k < L/2): a length's pairs are contiguous and 16-byte aligned
    std::vector<u32> lpf(2ull * lmax, 0), lpi(2ull * lmax, 0);
    for (u32 Ll = 2; Ll <= lmax; Ll *= 2)
        for (u32 k = 0; k < Ll / 2; k++) {
            const u32 idx = Ll / 2 + k, src = k * (lmax / Ll);
            lpf[2 * idx] = w2[src];
            lpf[2 * idx + 1] = w2s[src];
            lpi[2 * idx] = w2i[src];
            lpi[2 * idx + 1] = w2is[src];
        }
    std::vector<u32> pfw2(2ull * S), pinv2(2ull * S);
    for (u32 k = 0; k < S; k++) {
        pfw2[2 * k] = pfw[k];
        pfw2[2 * k + 1] = pfw_s[k];
        pinv2[2 * k] = pinv[k];
        pinv2[2 * k + 1] = pinv_s[k];
    }

    // one allocation: [qfw | qfw_s | qinv | qinv_s] [cdt] [pfw .. pinv_s] [w2 .. w2is]
    const size_t bytes_q = 4ull * n * 8, bytes_cdt = 19 * 8 + 8, bytes_p = 4ull * S * 4, bytes_w = 4ull * half * 4;
    const size_t total = 2 * bytes_q + bytes_cdt + 2 * bytes_p + bytes_w + 16ull * lmax + 256;
    fdsc_params* P = new (std::nothrow) fdsc_params();
    if (!P) return fdsc_set_error(FDSC_ERR_OOM, "host allocation failed");
    P->info = I;
    P->max_T = max_T;
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = cudaMalloc(&P->table_mem, total);
    if (e != cudaSuccess) {
        delete P;
        return fdsc_set_error(e == cudaErrorMemoryAllocation ? FDSC_ERR_OOM : FDSC_ERR_CUDA,
                              "params tables: %s", cudaGetErrorString(e));
    }
    std::vector<unsigned char> host(total, 0);
    unsigned char* h = host.data();
    size_t off = 0;
    auto put = [&](const void* src, size_t b) {
        if (off + b <= total) memcpy(h + off, src, b);
        size_t o = off;
        off += (b + 15) & ~size_t(15);
        return o;
    };
    size_t o_qfw = put(qfw.data(), 8ull * n), o_qfw_s = put(qfw_s.data(), 8ull * n);
    size_t o_qinv = put(qinv.data(), 8ull * n), o_qinv_s = put(qinv_s.data(), 8ull * n);
    size_t o_cdt = put(cdt, sizeof cdt);
    size_t o_pfw = put(pfw.data(), 4ull * S), o_pfw_s = put(pfw_s.data(), 4ull * S);
    size_t o_pinv = put(pinv.data(), 4ull * S), o_pinv_s = put(pinv_s.data(), 4ull * S);
    size_t o_w2 = put(w2.data(), 4ull * half), o_w2s = put(w2s.data(), 4ull * half);
    size_t o_w2i = put(w2i.data(), 4ull * half), o_w2is = put(w2is.data(), 4ull * half);
    size_t o_qfw2 = put(qfw2.data(), 16ull * n), o_qinv2 = put(qinv2.data(), 16ull * n);
    size_t o_pfw2 = put(pfw2.data(), 8ull * S), o_pinv2 = put(pinv2.data(), 8ull * S);
    size_t o_lpf = put(lpf.data(), 8ull * lmax), o_lpi = put(lpi.data(), 8ull * lmax);
    if (off > total) {  // layout bookkeeping error: never write past the allocation
        cudaFree(P->table_mem);
        delete P;
        return fdsc_set_error(FDSC_ERR_ARG, "internal: table layout %zu > %zu bytes", off, total);
    }
    e = cudaMemcpy(P->table_mem, h, off, cudaMemcpyHostToDevice);
    // a copy from pageable memory may return before it lands; kernels on
    // other streams (and those that read the tables before their
    // programmatic wait) must see the finished tables
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(P->table_mem);
        delete P;
        return fdsc_set_error(FDSC_ERR_CUDA, "params upload: %s", cudaGetErrorString(e));
    }
    unsigned char* dbase = (unsigned char*)P->table_mem;
    DevParams& D = P->dev;
    D.n = n; D.logn = I.logn; D.p = p; D.S = S; D.logS = I.logS; D.d = I.d; D.g_p = I.g_p;
    D.Sinv = (u32)pow_mod(S, p - 2, p);
    D.Sinv_s = fdsc_shoup32(D.Sinv, p);
    D.lmax = lmax;
    D.loglmax = __builtin_ctz(lmax);
    D.q = q; D.twoq = 2 * q; D.delta = I.delta;
    D.r64 = (u64)(((u128)1 << 64) % q);
    D.r64_s = shoup64(D.r64, q);
    D.one_s = shoup64(1, q);
    D.round_k = (u64)(((u128)p << 64) / q);
    D.mu = (u64)(((u128)1 << 122) / q);
    D.ninv = pow_mod(n, q - 2, q);
    D.ninv_s = shoup64(D.ninv, q);
    D.qfw = (const u64*)(dbase + o_qfw); D.qfw_s = (const u64*)(dbase + o_qfw_s);
    D.qinv = (const u64*)(dbase + o_qinv); D.qinv_s = (const u64*)(dbase + o_qinv_s);
    D.cdt = (const u64*)(dbase + o_cdt);
    D.pfw = (const u32*)(dbase + o_pfw); D.pfw_s = (const u32*)(dbase + o_pfw_s);
    D.pinv = (const u32*)(dbase + o_pinv); D.pinv_s = (const u32*)(dbase + o_pinv_s);
    D.w2d = (const u32*)(dbase + o_w2); D.w2d_s = (const u32*)(dbase + o_w2s);
    D.w2di = (const u32*)(dbase + o_w2i); D.w2di_s = (const u32*)(dbase + o_w2is);
    D.qfw2 = (const ulonglong2*)(dbase + o_qfw2); D.qinv2 = (const ulonglong2*)(dbase + o_qinv2);
    D.pfw2 = (const uint2*)(dbase + o_pfw2); D.pinv2 = (const uint2*)(dbase + o_pinv2);
    D.lpf = (const uint2*)(dbase + o_lpf); D.lpi = (const uint2*)(dbase + o_lpi);
    *out = P;
    return FDSC_OK;
}

extern "C" int fdsc_params_destroy(fdsc_params* P) {
    if (!P) return FDSC_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != P->device) cudaSetDevice(P->device);
    cudaError_t e = cudaFree(P->table_mem);
    if (prev >= 0 && prev != P->device) cudaSetDevice(prev);
    delete P;
    return e == cudaSuccess ? FDSC_OK : fdsc_set_error(FDSC_ERR_CUDA, "params free: %s", cudaGetErrorString(e));
}

extern "C" int fdsc_params_get_info(const fdsc_params* P, fdsc_params_info* out) {
    if (!P || !out) return fdsc_set_error(FDSC_ERR_ARG, "NULL argument");
    *out = P->info;
    return FDSC_OK;
}
