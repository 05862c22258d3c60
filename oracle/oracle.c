/*
 * CPU oracle for batched midsize unsigned-integer addition and multiplication.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no code, header or constant with the
 * CUDA path.
 *
 * What it computes (plain definitions, no blocking, fusion or reordering):
 *   - oracle_add: c = a + b, written as max(na,nb)+1 little-endian u32 limbs.
 *     This is the sequential add-with-carry of Section 2 (the iterative
 *     procedure that adds corresponding words in a double-width type and
 *     carries the quotient), carried out on 64-bit words with a 128-bit sum.
 *   - oracle_sub: c = a - b mod 2^(32*na) (na >= nb) with the final borrow,
 *     used only to check the invariant (a + b) - b = a.
 *   - oracle_mul: c = a * b, written as na+nb little-endian u32 limbs.  This
 *     is the classical product of Section 3, Eq. (1), C_k = sum_{i+j=k} A_i B_j,
 *     evaluated row by row on 64-bit words: t = A_i*B_j + C_{i+j} + carry in
 *     128 bits, which cannot overflow since (2^64-1)^2 + 2(2^64-1) = 2^128-1.
 *     The paper truncates results to the input length; the full-width product
 *     is returned here and the truncated form is its low limbs.
 *   - oracle_mod_u64: a mod q for one integer and a modulus q < 2^63
 *     (Horner's rule), for residue checks of products.
 *
 * Layout: instance i of an operand with n limbs starts at limb i*n.  Limbs are
 * u32, little-endian within the integer.  The batch is split statically over
 * POSIX threads; each thread handles a contiguous range of instances.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* u32 limbs -> u64 limbs; an odd count is zero-padded at the top. */
static void to_u64(const uint32_t *src, uint32_t n, uint64_t *dst, uint32_t m)
{
    for (uint32_t w = 0; w < m; ++w) {
        uint64_t lo = (2 * w < n) ? src[2 * w] : 0;
        uint64_t hi = (2 * w + 1 < n) ? src[2 * w + 1] : 0;
        dst[w] = lo | (hi << 32);
    }
}

/* u64 limbs -> the first n u32 limbs. */
static void from_u64(const uint64_t *src, uint32_t n, uint32_t *dst)
{
    for (uint32_t k = 0; k < n; ++k)
        dst[k] = (uint32_t)(src[k / 2] >> (32 * (k % 2)));
}

/* ---- one instance --------------------------------------------------- */

static void add_one(const uint32_t *a, uint32_t na, const uint32_t *b, uint32_t nb,
                    uint32_t *c, uint64_t *wa, uint64_t *wb, uint64_t *wc)
{
    uint32_t n = na > nb ? na : nb;
    uint32_t m = (n + 1 + 1) / 2;          /* words holding n+1 u32 limbs */
    to_u64(a, na, wa, m);
    to_u64(b, nb, wb, m);
    uint64_t carry = 0;
    for (uint32_t w = 0; w < m; ++w) {
        u128 s = (u128)wa[w] + wb[w] + carry;
        wc[w] = (uint64_t)s;
        carry = (uint64_t)(s >> 64);
    }
    /* The true sum has at most n+1 limbs, so nothing is carried out of m words. */
    from_u64(wc, n + 1, c);
}

static uint32_t sub_one(const uint32_t *a, uint32_t na, const uint32_t *b, uint32_t nb,
                        uint32_t *c, uint64_t *wa, uint64_t *wb, uint64_t *wc)
{
    uint32_t m = (na + 1) / 2;
    to_u64(a, na, wa, m);
    to_u64(b, nb < na ? nb : na, wb, m);
    uint64_t borrow = 0;
    for (uint32_t w = 0; w < m; ++w) {
        u128 d = (u128)wa[w] - wb[w] - borrow;
        wc[w] = (uint64_t)d;
        borrow = (uint64_t)(d >> 64) ? 1 : 0;
    }
    /* Both pad halves are zero, so a borrow into the pad propagates out of
     * the top word: borrow == 1 exactly when a < b. */
    from_u64(wc, na, c);
    return (uint32_t)borrow;
}

static void mul_one(const uint32_t *a, uint32_t na, const uint32_t *b, uint32_t nb,
                    uint32_t *c, uint64_t *wa, uint64_t *wb, uint64_t *wc)
{
    uint32_t ma = (na + 1) / 2, mb = (nb + 1) / 2;
    to_u64(a, na, wa, ma);
    to_u64(b, nb, wb, mb);
    memset(wc, 0, sizeof(uint64_t) * (ma + mb));
    for (uint32_t i = 0; i < ma; ++i) {
        uint64_t carry = 0;
        for (uint32_t j = 0; j < mb; ++j) {
            u128 t = (u128)wa[i] * wb[j] + wc[i + j] + carry;
            wc[i + j] = (uint64_t)t;
            carry = (uint64_t)(t >> 64);
        }
        wc[i + mb] = carry;
    }
    from_u64(wc, na + nb, c);
}

/* ---- batch driver ---------------------------------------------------- */

enum { OP_ADD = 0, OP_SUB = 1, OP_MUL = 2 };

typedef struct {
    int op;
    const uint32_t *a, *b;
    uint32_t *c, *borrow;
    uint32_t na, nb, nc;
    uint64_t lo, hi;     /* instance range [lo, hi) */
    int status;
} job_t;

static void *run_job(void *arg)
{
    job_t *j = (job_t *)arg;
    uint32_t ma = (j->na + 2) / 2 + 1, mb = (j->nb + 2) / 2 + 1;
    uint32_t mm = ma > mb ? ma : mb;
    uint64_t *wa = (uint64_t *)malloc(sizeof(uint64_t) * mm);
    uint64_t *wb = (uint64_t *)malloc(sizeof(uint64_t) * mm);
    uint64_t *wc = (uint64_t *)malloc(sizeof(uint64_t) * (ma + mb));
    if (!wa || !wb || !wc) {
        free(wa); free(wb); free(wc);
        j->status = -1;
        return NULL;
    }
    for (uint64_t i = j->lo; i < j->hi; ++i) {
        const uint32_t *ai = j->a + i * j->na, *bi = j->b + i * j->nb;
        uint32_t *ci = j->c + i * j->nc;
        if (j->op == OP_ADD)
            add_one(ai, j->na, bi, j->nb, ci, wa, wb, wc);
        else if (j->op == OP_SUB) {
            uint32_t br = sub_one(ai, j->na, bi, j->nb, ci, wa, wb, wc);
            if (j->borrow) j->borrow[i] = br;
        } else
            mul_one(ai, j->na, bi, j->nb, ci, wa, wb, wc);
    }
    free(wa); free(wb); free(wc);
    j->status = 0;
    return NULL;
}

static int run_batch(int op, const uint32_t *a, const uint32_t *b, uint32_t *c,
                     uint32_t *borrow, uint32_t na, uint32_t nb, uint32_t nc,
                     uint64_t batch, int nthreads)
{
    if (na == 0 || nb == 0) return -2;
    if (batch == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > batch) nthreads = (int)batch;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tids) { free(jobs); free(tids); return -1; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (job_t){op, a, b, c, borrow, na, nb, nc,
                          batch * (uint64_t)t / (uint64_t)nthreads,
                          batch * (uint64_t)(t + 1) / (uint64_t)nthreads, 0};
    }
    int started = 0, rc = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&tids[t], NULL, run_job, &jobs[t]) != 0) { rc = -1; break; }
        started = t;
    }
    if (rc == 0) run_job(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(tids[t], NULL);
    for (int t = 0; t < nthreads && rc == 0; ++t) rc = jobs[t].status;
    free(jobs); free(tids);
    return rc;
}

int oracle_add(const uint32_t *a, const uint32_t *b, uint32_t *c,
               uint32_t na, uint32_t nb, uint64_t batch, int nthreads)
{
    uint32_t n = na > nb ? na : nb;
    return run_batch(OP_ADD, a, b, c, NULL, na, nb, n + 1, batch, nthreads);
}

int oracle_sub(const uint32_t *a, const uint32_t *b, uint32_t *c, uint32_t *borrow,
               uint32_t na, uint32_t nb, uint64_t batch, int nthreads)
{
    if (nb > na) return -2;
    return run_batch(OP_SUB, a, b, c, borrow, na, nb, na, batch, nthreads);
}

int oracle_mul(const uint32_t *a, const uint32_t *b, uint32_t *c,
               uint32_t na, uint32_t nb, uint64_t batch, int nthreads)
{
    return run_batch(OP_MUL, a, b, c, NULL, na, nb, na + nb, batch, nthreads);
}

uint64_t oracle_mod_u64(const uint32_t *a, uint32_t n, uint64_t q)
{
    if (q == 0) return 0;
    u128 r = 0;
    for (uint32_t k = n; k-- > 0;)
        r = ((r << 32) | a[k]) % q;
    return (uint64_t)r;
}
