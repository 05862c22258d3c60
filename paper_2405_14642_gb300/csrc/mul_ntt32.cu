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
// Montgomery product (R = 2^32) is two 32x32 multiplies for the product and
// two for the reduction (the 64-bit fields take six 32x32->64 multiply-adds),
// and both spectra of a 16384-point transform fit in shared memory, so every
// size up to 256K-bit operands runs as one transform (no split).  Elements are
// kept lazily in [0, 2p): with p < 2^30, 4p < 2^32 leaves room for the DIF
// butterfly's unreduced difference u - v + 2p.
//
// Work mapping as in mul_ntt.cu: one CTA per integer pair at a time (a
// persistent grid), forward transforms decimation-in-frequency and the
// inverse decimation-in-time (no bit-reversal pass), radix-8 register passes.
// For each prime: digits -> A, B (reduced into the field), forward transforms,
// pointwise product, inverse, scale by 1/N.  The residues modulo p0 and p1 go
// to a per-CTA scratch slot (L2-resident), the residues modulo p2 stay in
// shared memory, and the normalisation recombines and carries them into
// limbs.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "bn_internal.h"
#include "ntt_device.cuh"

namespace bn {

namespace {

using namespace ntt;

constexpr uint32_t kMaxLength3 = 16384;  // both u32 spectra in shared memory

// Z_P for a prime P < 2^30 in Montgomery form with R = 2^32; NINV = -P^-1
// mod 2^32.  Elements are kept lazily in [0, 2P); canon() maps to [0, P).
//   mul(a, b): t = a b < 4P^2 (a, b < 2P); the quotient
//   m = t_lo NINV makes t + m P divisible by 2^32, and (t + m P) / 2^32 =
//   t_hi + hi(m P) + (t_lo != 0) < 4P^2 / 2^32 + P < 2P.
template <uint32_t P, uint32_t NINV>
struct MontField32 {
    using Elem = uint32_t;
    static constexpr uint32_t P_VALUE = P;
    static constexpr uint32_t TWO_P = 2 * P;
    static constexpr uint32_t R_MOD_P = (uint32_t)((1ull << 32) % P);
    static_assert(P < (1u << 30), "4P < 2^32");
    static_assert((uint32_t)(P * NINV) == 0xffffffffu, "NINV = -P^-1 mod 2^32");
    // Reductions as unsigned minima: for r < 4P, r - 2P wraps above r exactly
    // when r < 2P, so min(r, r - 2P) is r mod-reduced into [0, 2P) (one
    // min and one subtract instead of a compare, a select and a subtract).
    __device__ static __forceinline__ uint32_t add(uint32_t a, uint32_t b) {
        const uint32_t r = a + b;
        return min(r, r - TWO_P);
    }
    __device__ static __forceinline__ uint32_t sub(uint32_t a, uint32_t b) {
        const uint32_t r = a + TWO_P - b;
        return min(r, r - TWO_P);
    }
    __device__ static __forceinline__ uint32_t canon(uint32_t a) { return min(a, a - P); }
    __device__ static __forceinline__ uint32_t mul(uint32_t a, uint32_t b) {
        const uint32_t lo = a * b, hi = __umulhi(a, b);
        const uint32_t m = lo * NINV;
        return hi + __umulhi(m, P) + (lo != 0u);
    }
    // Any 32-bit digit d into the field: d (R mod P) / R = d (mod P), < 2P.
    __device__ static __forceinline__ uint32_t from_digit(uint32_t d) { return mul(d, R_MOD_P); }
    // Twiddles by Shoup's method: an entry is (w, w' = floor(w 2^32 / P)) with
    // w < P, and for any a < 2^32, q = hi(a w') gives a w - q P in [0, 2P),
    // exact in 32-bit arithmetic.  One high and two low multiplies, against
    // Montgomery's two high, two low and a correction.
    using Tw = uint2;
    __device__ static __forceinline__ uint32_t twiddle(uint32_t a, uint2 w) {
        const uint32_t q = __umulhi(a, w.y);
        return a * w.x - q * P;
    }
    __device__ static __forceinline__ uint32_t twiddle_lazy(uint32_t a, uint2 w) { return twiddle(a, w); }
};

using F0 = MontField32<469762049u, 0x1bffffffu>;  // 7 * 2^26 + 1
using F1 = MontField32<754974721u, 0x2cffffffu>;  // 45 * 2^24 + 1
using F2 = MontField32<998244353u, 0x3b7fffffu>;  // 119 * 2^23 + 1
static_assert(F0::P_VALUE < F1::P_VALUE && F1::P_VALUE < F2::P_VALUE, "Garner order");

struct Tab3 {
    const uint2 *twf;     // [N]: twf[h + j] = Shoup pair of w_{2h}^j
    const uint2 *twi;     // [N]: Shoup pair of w_{2h}^-j
    uint32_t scale;       // N^-1 R^2 mod p: mul(x, scale) undoes the 1/R of the pointwise product
};

struct Ntt3Args {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t na, nb, nout, N, logN;
    uint64_t batch;
    uint32_t *scratch;        // per CTA: residues mod p0 [N], mod p1 [N]
    uint64_t scratch_stride;  // u32 words per CTA
    Tab3 t[3];
    uint32_t g01, g02, g12;   // form(p0^-1 mod p1), form(p0^-1 mod p2), form(p1^-1 mod p2)
};

// Coefficients 0 .. nout-1 of a*b mod F's prime (canonical) to dest, or, with
// dest == nullptr, to B (padded layout).  Ends with a barrier.
template <class F>
__device__ void prime_product3(const Ntt3Args &p, const Tab3 &tb, const uint32_t *arow,
                               const uint32_t *brow, uint32_t *A, uint32_t *B, uint32_t *dest) {
    for (uint32_t j = threadIdx.x; j < p.N; j += blockDim.x) {  // n1: digits
        A[phys4(j)] = j < p.na ? F::from_digit(__ldg(arow + j)) : 0u;
        B[phys4(j)] = j < p.nb ? F::from_digit(__ldg(brow + j)) : 0u;
    }
    __syncthreads();
    forward2<F>(p.N, p.logN, tb.twf, A, B);                       // n2: forward transforms
    for (uint32_t j = threadIdx.x; j < p.N; j += blockDim.x)      // n3: pointwise
        B[phys4(j)] = F::mul(A[phys4(j)], B[phys4(j)]);
    __syncthreads();
    inverse<F>(p.N, p.logN, tb.twi, B);                           // n4: inverse (unscaled)
    for (uint32_t j = threadIdx.x; j < p.nout; j += blockDim.x) {
        const uint32_t v = F::canon(F::mul(B[phys4(j)], tb.scale));
        if (dest) dest[j] = v;
        else B[phys4(j)] = v;
    }
    __syncthreads();
}

// n5: the coefficient with residues r0, r1, r2 (canonical): c = v0 + v1 p0 +
// v2 p0 p1 with v0 = r0, v1 = (r1 - v0) / p0 mod p1, v2 = ((r2 - v0) / p0 -
// v1) / p1 mod p2 (Garner), exact since c < p0 p1 p2.
__device__ __forceinline__ u128 garner3(const Ntt3Args &p, uint32_t r0, uint32_t r1, uint32_t r2) {
    uint32_t d = r1 >= r0 ? r1 - r0 : r1 + F1::P_VALUE - r0;  // r0 < p0 < p1
    const uint32_t v1 = F1::canon(F1::mul(d, p.g01));
    d = r2 >= r0 ? r2 - r0 : r2 + F2::P_VALUE - r0;            // r0 < p0 < p2
    uint32_t e = F2::canon(F2::mul(d, p.g02));
    e = e >= v1 ? e - v1 : e + F2::P_VALUE - v1;                // v1 < p1 < p2
    const uint32_t v2 = F2::canon(F2::mul(e, p.g12));
    constexpr uint64_t P01 = (uint64_t)F0::P_VALUE * F1::P_VALUE;
    return (u128)((uint64_t)r0 + (uint64_t)v1 * F0::P_VALUE) + (u128)v2 * P01;
}

__global__ void __launch_bounds__(1024) k_mul_ntt3(Ntt3Args p) {
    extern __shared__ __align__(16) uint32_t sm32[];
    const uint32_t Np = (phys4_words(p.N) + 3) & ~3u;  // B stays 16-byte aligned
    uint32_t *A = sm32;
    uint32_t *B = sm32 + Np;
    uint64_t *spill = reinterpret_cast<uint64_t *>(B + Np);
    uint32_t *flags = reinterpret_cast<uint32_t *>(spill + blockDim.x);
    uint32_t *R0 = p.scratch + blockIdx.x * p.scratch_stride;
    uint32_t *R1 = R0 + p.N;
    for (uint64_t inst = blockIdx.x; inst < p.batch; inst += gridDim.x) {
        const uint32_t *arow = p.a + inst * p.na, *brow = p.b + inst * p.nb;
        prime_product3<F0>(p, p.t[0], arow, brow, A, B, R0);
        prime_product3<F1>(p, p.t[1], arow, brow, A, B, R1);
        prime_product3<F2>(p, p.t[2], arow, brow, A, B, nullptr);
        // n6: recombine and carry into limbs (A's words serve as the staging row)
        normalize_limbs(p.nout, p.c + inst * p.nout, A, spill, flags,
                        [&](uint32_t k) { return garner3(p, R0[k], R1[k], B[phys4(k)]); });
    }
}

// Mixed-size batch of products sharing the transform length N (the plan's):
// the CTA takes the next item from the work queue (largest first) and uses
// that item's sizes and rows.
__global__ void __launch_bounds__(1024)
    k_mul_ntt3_batch(Ntt3Args p, const BatchItem *items, uint32_t count, uint32_t *queue,
                     const BatchBinding *bind) {
    extern __shared__ __align__(16) uint32_t sm32[];
    __shared__ uint32_t next;
    const uint32_t Np = (phys4_words(p.N) + 3) & ~3u;  // B stays 16-byte aligned
    uint32_t *A = sm32;
    uint32_t *B = sm32 + Np;
    uint64_t *spill = reinterpret_cast<uint64_t *>(B + Np);
    uint32_t *flags = reinterpret_cast<uint32_t *>(spill + blockDim.x);
    uint32_t *R0 = p.scratch + blockIdx.x * p.scratch_stride;
    uint32_t *R1 = R0 + p.N;
    for (;;) {
        __syncthreads();  // the previous item is stored before `next` moves on
        if (threadIdx.x == 0) next = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t i = next;
        if (i >= count) break;
        const BatchItem it = items[i];
        p.na = it.na;
        p.nb = it.nb;
        p.nout = it.na + it.nb;
        const uint32_t *arow = bind->a + it.off_a, *brow = bind->b + it.off_b;
        uint32_t *crow = bind->c + it.off_c;
        prime_product3<F0>(p, p.t[0], arow, brow, A, B, R0);
        prime_product3<F1>(p, p.t[1], arow, brow, A, B, R1);
        prime_product3<F2>(p, p.t[2], arow, brow, A, B, nullptr);
        normalize_limbs(p.nout, crow, A, spill, flags,
                        [&](uint32_t k) { return garner3(p, R0[k], R1[k], B[phys4(k)]); });
    }
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

void make_tables3(const HostField32 &f, uint32_t N, uint2 *twf, uint2 *twi, uint32_t &scale) {
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
    scale = mulmod(invmod(N % f.p, f.p), mulmod(r, r, f.p), f.p);
}

uint32_t next_pow2_u32(uint32_t x) {
    uint32_t t = 1;
    while (t < x) t <<= 1;
    return t;
}

}  // namespace

struct Ntt3Plan {
    uint32_t na = 0, nb = 0, nout = 0, N = 0, logN = 0, threads = 0, smem = 0, max_grid = 0;
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
    uint32_t T = p->N / 8;
    if (T < 32) T = 32;
    if (T > 1024) T = 1024;
    if (cta) T = cta;
    p->threads = T;
    const uint32_t Np = (phys4_words(p->N) + 3) & ~3u;
    p->smem = 4u * 2u * Np + 8u * T + 4u * 32u;

    cudaError_t e = allow_max_smem((const void *)k_mul_ntt3);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mul_ntt3, (int)T, p->smem);
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
    if (allow_max_smem((const void *)k_mul_ntt3_batch) != cudaSuccess) return BN_ECUDA;
    return ntt3_create(out, N / 2, N / 2, nullptr);
}

cudaError_t ntt3_batch_launch(Ntt3Plan *p, const BatchItem *items, uint32_t count, uint32_t *queue,
                              const BatchBinding *bind, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    if (cudaError_t e = allow_max_smem((const void *)k_mul_ntt3_batch)) return e;
    const uint32_t grid = count < p->max_grid ? count : p->max_grid;
    k_mul_ntt3_batch<<<grid, p->threads, p->smem, st>>>(plan_args3(p), items, count, queue, bind);
    return cudaGetLastError();
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
    k_mul_ntt3<<<1, p->threads, p->smem, st>>>(args);
    return cudaGetLastError();
}

cudaError_t ntt3_launch(Ntt3Plan *p, const uint32_t *a, const uint32_t *b, uint32_t *c, uint64_t batch,
                        cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    Ntt3Args args{};
    args.a = a;
    args.b = b;
    args.c = c;
    args.na = p->na;
    args.nb = p->nb;
    args.nout = p->nout;
    args.N = p->N;
    args.logN = p->logN;
    args.batch = batch;
    args.scratch = p->scratch;
    args.scratch_stride = p->scratch_stride;
    for (int i = 0; i < 3; ++i) args.t[i] = p->t[i];
    args.g01 = p->g01;
    args.g02 = p->g02;
    args.g12 = p->g12;
    const uint64_t grid = batch < p->max_grid ? batch : p->max_grid;
    k_mul_ntt3<<<(unsigned)grid, p->threads, p->smem, st>>>(args);
    return cudaGetLastError();
}

}  // namespace bn
