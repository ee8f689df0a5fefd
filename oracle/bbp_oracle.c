/*
 * Oracle O2: BBP digit extraction of pi in plain C (C99 + unsigned __int128 + pthreads).
 *
 * TEST INFRASTRUCTURE ONLY.  Loaded by oracle/__init__.py for tests/,
 * __graft_entry__.smoke() and the CPU-baseline leg of bench.py.  It shares no
 * code with the CUDA library: it is a direct, slow restatement of the same
 * definition as the Python oracle O1 (oracle/bbp_oracle.py).
 *
 * Definition (Sze, "The Two Quadrillionth Bit of pi is 0!", Sec. 3, Eq. 3-5):
 *   d = n - 1; for series j with modulus m = a*k + b, exponent e = d + c - step*k:
 *     e >= 0 :  t = floor((2^e mod m) * 2^W / m)     (A_k: modexp, then division)
 *     e <  0 :  t = floor(2^(W+e) / m)               (B_k: shift, then division)
 *   S_j = sign_j * sum_k (-1)^(alt*k) t  (mod 2^W), summed until the natural end
 *   (first tail term that truncates to 0).
 * Modular exponentiation is right-to-left square-and-multiply with the
 * compiler's 128-bit '%'; the division is schoolbook long division, one 32-bit
 * quotient digit at a time.  Moduli must stay below 2^62.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef unsigned __int128 u128;

typedef struct { uint64_t a, b; int sign; int c; } series_t;
typedef struct { int step; int alternating; int count; series_t s[7]; } formula_t;

/* Eq. 2 (Bellard) and Eq. 1 in the form of Eq. 3 (BBP); same table as stated in
 * the paper, written out here independently of every other file. */
static const formula_t FORMULAS[2] = {
    {10, 1, 7, {{10, 1, +1, 2}, {10, 3, -1, 0}, {10, 5, -1, -4}, {10, 7, -1, -4},
                {10, 9, +1, -6}, {4, 1, -1, -1}, {4, 3, -1, -6}}},
    {4, 0, 4, {{8, 1, +1, 2}, {2, 1, -1, -1}, {8, 5, -1, 0}, {4, 3, -1, -1}}},
};

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ERANGE = -6 };

static uint64_t pow2_mod(uint64_t e, uint64_t m) {
    uint64_t result = 1 % m, base = 2 % m;
    while (e) {
        if (e & 1) result = (uint64_t)(((u128)result * base) % m);
        base = (uint64_t)(((u128)base * base) % m);
        e >>= 1;
    }
    return result;
}

/* q[0..L) = floor(r * 2^(32L) / m) for r < m: long division, top digit first. */
static void long_div_fraction(uint64_t r, uint64_t m, uint32_t *q, int L) {
    u128 rem = r;
    for (int i = L - 1; i >= 0; --i) {
        rem <<= 32;
        q[i] = (uint32_t)(rem / m);
        rem %= m;
    }
}

/* q[0..L) = floor(2^p / m) for p < 32L: long division of a lone 1 bit. */
static void long_div_power(uint64_t p, uint64_t m, uint32_t *q, int L) {
    memset(q, 0, sizeof(uint32_t) * (size_t)L);
    int top = (int)(p / 32);
    u128 rem = (u128)1 << (p % 32);
    for (int i = top; i >= 0; --i) {
        if (i != top) rem <<= 32;
        q[i] = (uint32_t)(rem / m);
        rem %= m;
    }
}

static void add_limbs(uint32_t *acc, const uint32_t *t, int L) {
    uint64_t carry = 0;
    for (int i = 0; i < L; ++i) {
        uint64_t s = (uint64_t)acc[i] + t[i] + carry;
        acc[i] = (uint32_t)s;
        carry = s >> 32;
    }
}

static void sub_limbs(uint32_t *acc, const uint32_t *t, int L) {
    uint64_t borrow = 0;
    for (int i = 0; i < L; ++i) {
        uint64_t s = (uint64_t)acc[i] - t[i] - borrow;
        acc[i] = (uint32_t)s;
        borrow = (s >> 32) & 1;
    }
}

static int64_t exponent_of(const formula_t *f, const series_t *s, uint64_t d, uint64_t k) {
    return (int64_t)d + s->c - (int64_t)(f->step * k);
}

uint64_t bbp_oracle_head_end(int formula, unsigned j, uint64_t n) {
    const formula_t *f = &FORMULAS[formula];
    int64_t top = (int64_t)(n - 1) + f->s[j].c;
    return top < 0 ? 0 : (uint64_t)top / (uint64_t)f->step + 1;
}

uint64_t bbp_oracle_natural_end(int formula, unsigned j, uint64_t n, unsigned W) {
    const formula_t *f = &FORMULAS[formula];
    const series_t *s = &f->s[j];
    uint64_t k = bbp_oracle_head_end(formula, j, n);
    for (;; ++k) {
        int64_t p = (int64_t)W + exponent_of(f, s, n - 1, k);
        uint64_t m = s->a * k + s->b;
        if (p < 0) return k;
        if (p < 64 && ((uint64_t)1 << p) < m) return k;   /* floor(2^p / m) == 0 */
    }
}

typedef struct {
    const formula_t *f;
    const series_t *s;
    uint64_t d, k_lo, k_hi;
    int L;
    uint32_t *acc;
    int status;
} job_t;

static void *run_job(void *arg) {
    job_t *jb = (job_t *)arg;
    const int L = jb->L;
    const uint64_t W = 32u * (uint64_t)L;
    uint32_t *t = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)L);
    if (!t) { jb->status = ORC_ENOMEM; return NULL; }
    memset(jb->acc, 0, sizeof(uint32_t) * (size_t)L);
    for (uint64_t k = jb->k_lo; k < jb->k_hi; ++k) {
        int64_t e = exponent_of(jb->f, jb->s, jb->d, k);
        uint64_t m = jb->s->a * k + jb->s->b;
        if (e >= 0) {
            long_div_fraction(pow2_mod((uint64_t)e, m), m, t, L);
        } else if ((int64_t)W + e >= 0) {
            long_div_power((uint64_t)((int64_t)W + e), m, t, L);
        } else {
            continue;
        }
        if (jb->f->alternating && (k & 1)) sub_limbs(jb->acc, t, L);
        else add_limbs(jb->acc, t, L);
    }
    free(t);
    jb->status = ORC_OK;
    return NULL;
}

static unsigned thread_count(unsigned threads) {
    if (threads) return threads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (unsigned)c : 1u;
}

/* out_limbs[0..W/32) = sign_j * sum_{k in [k_begin, min(k_end, end_j))} (-1)^k t  mod 2^W.
 * k_end = UINT64_MAX means the natural end.  threads = 0 uses every online core. */
int bbp_oracle_partial_sum(int formula, unsigned j, uint64_t k_begin, uint64_t k_end,
                           uint64_t n, unsigned W, uint32_t *out_limbs, unsigned threads) {
    if (formula < 0 || formula > 1 || n == 0 || W == 0 || W % 32 || !out_limbs) return ORC_EINVAL;
    const formula_t *f = &FORMULAS[formula];
    if (j >= (unsigned)f->count || k_begin > k_end) return ORC_EINVAL;
    const series_t *s = &f->s[j];
    const int L = (int)(W / 32);
    uint64_t end = bbp_oracle_natural_end(formula, j, n, W);
    uint64_t hi = k_end < end ? k_end : end;
    memset(out_limbs, 0, sizeof(uint32_t) * (size_t)L);
    if (k_begin >= hi) return ORC_OK;
    if (s->a * (hi - 1) + s->b >= ((uint64_t)1 << 62)) return ORC_ERANGE;

    unsigned T = thread_count(threads);
    uint64_t span = hi - k_begin;
    if ((uint64_t)T > span) T = (unsigned)span;
    job_t *jobs = (job_t *)calloc(T, sizeof(job_t));
    pthread_t *tid = (pthread_t *)calloc(T, sizeof(pthread_t));
    uint32_t *accs = (uint32_t *)calloc((size_t)T * (size_t)L, sizeof(uint32_t));
    if (!jobs || !tid || !accs) { free(jobs); free(tid); free(accs); return ORC_ENOMEM; }
    for (unsigned i = 0; i < T; ++i) {
        jobs[i].f = f;
        jobs[i].s = s;
        jobs[i].d = n - 1;
        jobs[i].k_lo = k_begin + span * i / T;
        jobs[i].k_hi = k_begin + span * (i + 1) / T;
        jobs[i].L = L;
        jobs[i].acc = accs + (size_t)i * (size_t)L;
        jobs[i].status = ORC_EINVAL;
    }
    for (unsigned i = 1; i < T; ++i)
        if (pthread_create(&tid[i], NULL, run_job, &jobs[i]) != 0) jobs[i].status = 1;
    run_job(&jobs[0]);
    int status = ORC_OK;
    for (unsigned i = 1; i < T; ++i) {
        if (jobs[i].status == 1) run_job(&jobs[i]);    /* thread could not start */
        else pthread_join(tid[i], NULL);
    }
    uint32_t *total = (uint32_t *)calloc((size_t)L, sizeof(uint32_t));
    for (unsigned i = 0; i < T && total; ++i) {
        if (jobs[i].status != ORC_OK) status = jobs[i].status;
        add_limbs(total, jobs[i].acc, L);
    }
    if (!total) status = ORC_ENOMEM;
    if (status == ORC_OK) {
        if (s->sign < 0) sub_limbs(out_limbs, total, L);   /* 0 - total */
        else memcpy(out_limbs, total, sizeof(uint32_t) * (size_t)L);
    }
    free(total);
    free(accs);
    free(tid);
    free(jobs);
    return status;
}

/* Full sum S = sum_j S_j mod 2^W over every series, and N = number of evaluated terms. */
int bbp_oracle_accumulate(int formula, uint64_t n, unsigned W, uint32_t *out_limbs,
                          uint64_t *n_terms, unsigned threads) {
    if (formula < 0 || formula > 1 || n == 0 || W == 0 || W % 32 || !out_limbs) return ORC_EINVAL;
    const formula_t *f = &FORMULAS[formula];
    const int L = (int)(W / 32);
    uint32_t *part = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)L);
    if (!part) return ORC_ENOMEM;
    memset(out_limbs, 0, sizeof(uint32_t) * (size_t)L);
    uint64_t N = 0;
    for (int j = 0; j < f->count; ++j) {
        int st = bbp_oracle_partial_sum(formula, (unsigned)j, 0, UINT64_MAX, n, W, part, threads);
        if (st != ORC_OK) { free(part); return st; }
        add_limbs(out_limbs, part, L);
        N += bbp_oracle_natural_end(formula, (unsigned)j, n, W);
    }
    free(part);
    if (n_terms) *n_terms = N;
    return ORC_OK;
}
