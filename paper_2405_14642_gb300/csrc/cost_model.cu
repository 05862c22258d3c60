// Built-in cost model for choosing between the multiplication kernels, shared
// by mixed-size batches and the serving loop.  Figures measured on GB300 with
// the size-sweep batches (64 MiB of operands per side), CUDA events.
#include "bn_internal.h"

namespace bn {

double default_quad_rate(uint32_t key) {
    // Schoolbook word products per microsecond by ceil(log2(longer operand)).
    static const double r[14] = {1.0e6, 1.0e6, 1.0e6, 1.0e6, 1.0e6, 3.12e6, 3.88e6, 4.41e6, 4.72e6,
                                 5.12e6, 5.34e6, 5.45e6, 5.51e6, 5.33e6};
    return r[key < 14 ? key : 13];
}

double default_ntt_us(bool crt, uint32_t logN) {
    // Microseconds per item by log2(N); below 2^11 (2^10 for CRT) a transform
    // is not considered: one small transform per CTA underuses the GPU.
    static const double t64[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0.0727, 0.159, 0.348, 0.882, 2.08};
    static const double tcrt[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0.076, 0.148, 0.323, 0.70, 1.79, 0};
    const double v = logN < 16 ? (crt ? tcrt[logN] : t64[logN]) : 0;
    return v > 0 ? v : 1e30;
}

double default_ntt3_us(uint32_t logN) {
    // Three 32-bit primes, microseconds per item by log2(N) (N = next power
    // of two >= na + nb), from 2^6 (1K-bit operands) to 2^14 (256K bits).
    static const double t3[15] = {0, 0, 0, 0, 0, 0, 0.00286, 0.00390, 0.00583, 0.01191, 0.02588,
                                  0.05375, 0.1188, 0.2545, 0.5270};
    const double v = logN < 15 ? t3[logN] : 0;
    return v > 0 ? v : 1e30;
}

namespace {
uint32_t clog2(uint32_t x) {
    uint32_t l = 0;
    while ((1u << l) < x) ++l;
    return l;
}
}  // namespace

MulChoice choose_mul(uint32_t na, uint32_t nb) {
    MulChoice c;
    const uint32_t mx = na > nb ? na : nb;
    c.quad_key = clog2(mx);
    const uint32_t d64 = 2 * (na + nb), dcrt = na + nb;
    c.log_n64 = clog2(d64 < 2 ? 2 : d64);
    c.log_ncrt = clog2(dcrt < 2 ? 2 : dcrt);
    const double q = (double)na * nb / default_quad_rate(c.quad_key);
    const double t64 = default_ntt_us(false, c.log_n64), tc = default_ntt_us(true, c.log_ncrt);
    c.kind = 1;
    c.est_us = q;
    if (t64 < c.est_us) { c.kind = 2; c.est_us = t64; }
    if (tc < c.est_us) { c.kind = 3; c.est_us = tc; }
    const double t3 = default_ntt3_us(c.log_ncrt);
    if (t3 < c.est_us) { c.kind = 4; c.est_us = t3; }
    return c;
}

}  // namespace bn
