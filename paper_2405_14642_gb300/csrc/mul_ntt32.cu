// Batched multiplication through three 32-bit prime fields (BN_OP_MUL_NTT3),
// a variant of Section 4's transform product.
//
// Section 4 multiplies in one "good" field Z_p, p = k 2^n + 1.  Here the
// convolution of the 32-bit limbs (digits) is taken modulo three good primes
// below 2^30,
//     p0 = 7 * 2^26 + 1,   p1 = 45 * 2^24 + 1,   p2 = 119 * 2^23 + 1,
// each with a root of order 2^n found by Section 4.1's search, and the three
// residues of every coefficient are recombined by Garner's mixed-radix CRT.
// p0 p1 p2 ~ 2^88 exceeds the largest coefficient N (2^32 - 1)^2 < 2^78, so
// the recombined coefficients are exact.
//
// Why 32-bit primes on this GPU: a field element is one 32-bit word, so a
// product by a constant (twiddles, the digit reduction, the 1/N scale) is
// three 32x32 multiplies by Shoup's method and a product of two variables
// (pointwise) four by Montgomery's (R = 2^32), where the 64-bit fields take
// six 32x32->64 multiply-adds; and both spectra of a 16384-point transform
// fit in shared memory, so every size up to 256K-bit operands runs as one
// transform (no split).  Elements are kept lazily in [0, 2p): with p < 2^30,
// 4p < 2^32 leaves room for the DIF butterfly's unreduced difference
// u - v + 2p.
//
// Work mapping as in mul_ntt.cu: one CTA per integer pair at a time (a
// persistent grid), forward transforms decimation-in-frequency and the
// inverse decimation-in-time (no bit-reversal pass), radix-8 register passes.
// For each prime: digits -> A, B (reduced into the field), forward transforms,
// pointwise product, inverse, scale by 1/N.  The residues modulo p0 and p1 go
// to a per-CTA scratch slot (L2-resident), the residues modulo p2 stay in
// shared memory, and the normalisation recombines and carries them into
// limbs.  The kernels are instantiated for every transform length (log2 N =
// 1 .. 14; ntt3_device.cuh and mul_ntt32_k*.cu), so the passes run with
// compile-time strides; this file holds the host side: tables, plans and
// launches.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "bn_internal.h"
#include "ntt3_device.cuh"

namespace bn {

namespace {

using namespace ntt3;

ntt3::Kernels3 kernels_for(uint32_t log_n) {
    if (log_n >= 1 && log_n <= 10) return ntt3_kernels_small(log_n);
    if (log_n >= 11 && log_n <= 12) return ntt3_kernels_mid(log_n);
    if (log_n >= 13 && log_n <= 14) return ntt3_kernels_large(log_n);
    return {nullptr, nullptr};
}

// ---- host side ---------------------------------------------------------------

uint32_t mulmod(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)((uint64_t)a * b % p); }

uint32_t powmod(uint32_t a, uint64_t e, uint32_t p) {
    uint32_t r = 1 % p;
    a %= p;
    while (e) {
        if (e & 1) r = mulmod(r, a, p);
        a = mulmod(a, a, p);
        e >>= 1;
    }
    return r;
}

uint32_t invmod(uint32_t a, uint32_t p) { return powmod(a, p - 2, p); }

// Montgomery form x R mod p, the form in which the device keeps constants.
uint32_t form(uint32_t x, uint32_t p) { return (uint32_t)(((uint64_t)(x % p) << 32) % p); }

struct HostField32 {
    uint32_t p, k, n, g;  // p = k 2^n + 1, g of order exactly 2^n
};

// Section 4.1's search: the first a >= 2 whose a^k has order exactly 2^n.
HostField32 make_field(uint32_t k, uint32_t n) {
    HostField32 f{k * (1u << n) + 1, k, n, 0};
    for (uint32_t a = 2; a < 1000 && !f.g; ++a) {
        const uint32_t g = powmod(a, k, f.p);
        if (powmod(g, 1ull << (n - 1), f.p) != 1) f.g = g;
    }
    return f;
}

// Shoup pair (w, floor(w 2^32 / p)) of a canonical w.
uint2 shoup(uint32_t w, uint32_t p) { return make_uint2(w, (uint32_t)(((uint64_t)w << 32) / p)); }

void make_tables3(const HostField32 &f, uint32_t N, uint2 *twf, uint2 *twi, uint2 &scale) {
    const uint32_t w = powmod(f.g, (1ull << f.n) / N, f.p), wi = invmod(w, f.p);
    twf[0] = twi[0] = make_uint2(0, 0);
    for (uint32_t h = 1; h < N; h <<= 1) {
        const uint32_t s = powmod(w, N / (2 * h), f.p), si = powmod(wi, N / (2 * h), f.p);
        uint32_t x = 1, xi = 1;
        for (uint32_t j = 0; j < h; ++j) {
            twf[h + j] = shoup(x, f.p);
            twi[h + j] = shoup(xi, f.p);
            x = mulmod(x, s, f.p);
            xi = mulmod(xi, si, f.p);
        }
    }
    const uint32_t r = (uint32_t)((1ull << 32) % f.p);
    scale = shoup(mulmod(invmod(N % f.p, f.p), r, f.p), f.p);
}

uint32_t next_pow2_u32(uint32_t x) {
    uint32_t t = 1;
    while (t < x) t <<= 1;
    return t;
}

}  // namespace

struct Ntt3Plan {
    uint32_t na = 0, nb = 0, nout = 0, N = 0, logN = 0, threads = 0, smem = 0, max_grid = 0;
    ntt3::Kernels3 kern{nullptr, nullptr};
    uint64_t scratch_stride = 0;
    size_t scratch_bytes = 0;
    uint32_t *dev = nullptr;      // tables followed by scratch
    uint32_t *scratch = nullptr;
    Tab3 t[3]{};
    uint32_t g01 = 0, g02 = 0, g12 = 0;
};

bn_status ntt3_create(Ntt3Plan **out, uint32_t na, uint32_t nb, const bn_tuning *tun) {
    *out = nullptr;
    if (na == 0 || nb == 0) return BN_EINVAL;
    if (na > BN_MUL_MAX_LIMBS || nb > BN_MUL_MAX_LIMBS) return BN_EUNSUPPORTED;
    uint32_t cta = 0;
    if (tun) {
        if (tun->reserved || tun->variant || tun->limbs_per_thread) return BN_EINVAL;
        if (tun->cta_threads && (tun->cta_threads % 32 || tun->cta_threads > 1024)) return BN_EINVAL;
        cta = tun->cta_threads;
    }
    const HostField32 fs[3] = {make_field(7, 26), make_field(45, 24), make_field(119, 23)};
    static const uint32_t device_p[3] = {F0::P_VALUE, F1::P_VALUE, F2::P_VALUE};
    for (int i = 0; i < 3; ++i)
        if (fs[i].p != device_p[i] || !fs[i].g) return BN_EUNSUPPORTED;
    Ntt3Plan *p = new (std::nothrow) Ntt3Plan();
    if (!p) return BN_ENOMEM;
    p->na = na;
    p->nb = nb;
    p->nout = na + nb;
    p->N = next_pow2_u32(p->nout < 2 ? 2 : p->nout);
    if (p->N > kMaxLength3) {
        delete p;
        return BN_EUNSUPPORTED;
    }
    while ((1u << p->logN) < p->N) ++p->logN;
    // The kernels of this length have a compile-time thread count (one per
    // radix-8 group, 32 .. 1024); a tuning request for another count is refused.
    uint32_t T = p->N / 8;
    if (T < 32) T = 32;
    if (T > 1024) T = 1024;
    p->kern = kernels_for(p->logN);
    if (!p->kern.plain || (cta && cta != T)) {
        delete p;
        return p->kern.plain ? BN_EINVAL : BN_EUNSUPPORTED;
    }
    p->threads = T;
    const uint32_t Np = (phys4_words(p->N) + 3) & ~3u;
    p->smem = 4u * 2u * Np + 8u * T + 4u * 32u;

    cudaError_t e = allow_max_smem(p->kern.plain);
    if (e == cudaSuccess) e = allow_max_smem(p->kern.batch);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->kern.plain, (int)T, p->smem);
    if (e != cudaSuccess || per_sm == 0) {
        delete p;
        return e == cudaSuccess ? BN_EUNSUPPORTED : BN_ECUDA;
    }
    p->max_grid = (uint32_t)(sms * per_sm);
    p->scratch_stride = 2ull * p->N;

    const size_t table_words = ((size_t)12 * p->N + 63) & ~size_t(63);  // 3 primes x 2 tables x N pairs
    p->scratch_bytes = (size_t)p->max_grid * p->scratch_stride * 4u;
    e = cudaMalloc(&p->dev, table_words * 4u + p->scratch_bytes);
    if (e != cudaSuccess) {
        delete p;
        return e == cudaErrorMemoryAllocation ? BN_ENOMEM : BN_ECUDA;
    }
    std::vector<uint32_t> host(table_words, 0);
    for (int i = 0; i < 3; ++i) {
        uint2 *twf = reinterpret_cast<uint2 *>(host.data()) + (size_t)2 * i * p->N, *twi = twf + p->N;
        make_tables3(fs[i], p->N, twf, twi, p->t[i].scale);
        p->t[i].twf = reinterpret_cast<const uint2 *>(p->dev) + (size_t)2 * i * p->N;
        p->t[i].twi = p->t[i].twf + p->N;
    }
    e = cudaMemcpy(p->dev, host.data(), table_words * 4u, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->dev);
        delete p;
        return BN_ECUDA;
    }
    p->scratch = p->dev + table_words;
    p->g01 = form(invmod(fs[0].p % fs[1].p, fs[1].p), fs[1].p);
    p->g02 = form(invmod(fs[0].p % fs[2].p, fs[2].p), fs[2].p);
    p->g12 = form(invmod(fs[1].p % fs[2].p, fs[2].p), fs[2].p);
    *out = p;
    return BN_OK;
}

void ntt3_destroy(Ntt3Plan *p) {
    if (!p) return;
    cudaFree(p->dev);
    delete p;
}

size_t ntt3_scratch_bytes(const Ntt3Plan *p) { return p ? p->scratch_bytes : 0; }

uint32_t ntt3_length(const Ntt3Plan *p) { return p ? p->N : 0; }

namespace {

Ntt3Args plan_args3(const Ntt3Plan *p) {
    Ntt3Args args{};
    args.na = p->na;
    args.nb = p->nb;
    args.nout = p->nout;
    args.N = p->N;
    args.logN = p->logN;
    args.scratch = p->scratch;
    args.scratch_stride = p->scratch_stride;
    for (int i = 0; i < 3; ++i) args.t[i] = p->t[i];
    args.g01 = p->g01;
    args.g02 = p->g02;
    args.g12 = p->g12;
    return args;
}

}  // namespace

bn_status ntt3_batch_plan(Ntt3Plan **out, uint32_t N) {
    // A plan whose transform length is exactly N: na + nb = N.
    if (N < 2 || (N & (N - 1))) return BN_EINVAL;
    if (N / 2 > BN_MUL_MAX_LIMBS) return BN_EUNSUPPORTED;
    return ntt3_create(out, N / 2, N / 2, nullptr);
}

cudaError_t ntt3_batch_launch(Ntt3Plan *p, const BatchItem *items, uint32_t count, uint32_t *queue,
                              const BatchBinding *bind, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    Ntt3Args args = plan_args3(p);
    const uint32_t grid = count < p->max_grid ? count : p->max_grid;
    void *params[] = {&args, &items, &count, &queue, &bind};
    return cudaLaunchKernel(p->kern.batch, dim3(grid), dim3(p->threads), params, p->smem, st);
}

cudaError_t ntt3_launch_sized(Ntt3Plan *p, uint32_t na, uint32_t nb, const uint32_t *a, const uint32_t *b,
                              uint32_t *c, cudaStream_t st) {
    Ntt3Args args = plan_args3(p);
    args.a = a;
    args.b = b;
    args.c = c;
    args.na = na;
    args.nb = nb;
    args.nout = na + nb;
    args.batch = 1;
    void *params[] = {&args};
    return cudaLaunchKernel(p->kern.plain, dim3(1), dim3(p->threads), params, p->smem, st);
}

cudaError_t ntt3_launch(Ntt3Plan *p, const uint32_t *a, const uint32_t *b, uint32_t *c, uint64_t batch,
                        cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    Ntt3Args args = plan_args3(p);
    args.a = a;
    args.b = b;
    args.c = c;
    args.batch = batch;
    const uint64_t grid = batch < p->max_grid ? batch : p->max_grid;
    void *params[] = {&args};
    return cudaLaunchKernel(p->kern.plain, dim3((unsigned)grid), dim3(p->threads), params, p->smem, st);
}

}  // namespace bn
