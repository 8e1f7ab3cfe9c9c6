/*
 * synth_gen.c -- fast seeded generator of sparse l2-logistic instances for
 * the batch workload (many instances of uneven n, d and density, as in a
 * regularisation path).  Data preparation only: it makes CSR matrices and
 * labels and holds none of the solver's arithmetic, so the CUDA path and
 * the float64 CPU checker consume the same inputs.
 *
 * Determinism across hosts (x86-64 here, aarch64 on the GPU machines): every
 * random number comes from an integer hash of (seed, stream, counter), and
 * the only floating-point operations are +, -, *, /, sqrt and exact scaling
 * by powers of two, evaluated in a fixed order (built with
 * -ffp-contract=off); log and exp are this file's own series, not libm's,
 * whose last bit may differ between C libraries.  The output is therefore the
 * same bits on every host and for every thread count.
 *
 * Instance (row i, columns v):
 *   row length   k_i = clamp(round(kmean + sqrt(kmean) z_i), kmin, kmax), z_i ~ N(0,1);
 *   columns      k_i distinct columns drawn with replacement from Zipf(s) over
 *                ranks 1..d mapped through a seeded permutation of the columns
 *                (rank 1 = the most frequent), first k_i distinct draws kept,
 *                sorted increasingly;
 *   values       |N(0,1)|, each row scaled to unit l2 norm, then rounded to
 *                the storage grid (float32 or bfloat16, round to nearest even);
 *   labels       sign(a_i . w* + 0.1 eps_i), w* ~ N(0, I), eps_i ~ N(0, 1),
 *                sign(0) = +1.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- random numbers */

/* The 64-bit finaliser of MurmurHash3 (Appleby): a bijective mix of a
 * 64-bit word. */
static uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

/* Random 64-bit word number `ctr` of stream `stream` of generator `seed`. */
static uint64_t rnd(uint64_t seed, uint64_t stream, uint64_t ctr) {
    uint64_t h = fmix64(seed * 0x9FB21C651E98DF25ULL + 0x2545F4914F6CDD1DULL);
    h = fmix64(h ^ (stream * 0xD6E8FEB86659FD93ULL));
    return fmix64(h + ctr * 0xC2B2AE3D27D4EB4FULL);
}

/* Uniform double in [0, 1) with 53 random bits. */
static double u01(uint64_t w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }

static const double kLn2 = 0.69314718055994530942;

/* Natural logarithm of x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)),
 * log m = 2 atanh(t), t = (m - 1)/(m + 1), |t| <= 0.172, by its series to
 * t^25 (truncation below 1e-19 relative). */
static double det_log(double x) {
    int e = 0;
    double m = frexp(x, &e); /* m in [0.5, 1) */
    if (m < 0.70710678118654752440) {
        m *= 2.0;
        e -= 1;
    }
    const double t = (m - 1.0) / (m + 1.0);
    const double t2 = t * t;
    double sum = 0.0;
    for (int j = 25; j >= 1; j -= 2) sum = sum * t2 + 1.0 / (double)j;
    return 2.0 * t * sum + (double)e * kLn2;
}

/* exp(x): x = k ln2 + r, |r| <= ln2 / 2 (+ rounding), exp(r) by its Taylor
 * series to r^24 (truncation below 1e-30 relative), scaled by 2^k. */
static double det_exp(double x) {
    const double k = floor(x / kLn2 + 0.5);
    const double r = x - k * kLn2;
    double sum = 1.0;
    for (int j = 24; j >= 1; --j) sum = 1.0 + sum * r / (double)j;
    return ldexp(sum, (int)k);
}

/* N(0,1) by the polar method (Marsaglia and Bray, 1964), drawing words
 * ctr, ctr+1, ... of the stream; advances *ctr past the words used. */
static double gauss(uint64_t seed, uint64_t stream, uint64_t *ctr) {
    for (;;) {
        const double u = 2.0 * u01(rnd(seed, stream, (*ctr)++)) - 1.0;
        const double v = 2.0 * u01(rnd(seed, stream, (*ctr)++)) - 1.0;
        const double s = u * u + v * v;
        if (s > 0.0 && s < 1.0) return u * sqrt(-2.0 * det_log(s) / s);
    }
}

/* ---------------------------------------------------------------- storage grids */

static double to_f32_grid(double v) { return (double)(float)v; }

static uint16_t bf16_bits(double v) {
    float f = (float)v;
    uint32_t b;
    memcpy(&b, &f, 4);
    b = (b + 0x7FFFu + ((b >> 16) & 1u)) >> 16; /* round to nearest even on the top 16 bits */
    return (uint16_t)b;
}

static double bf16_value(uint16_t h) {
    const uint32_t b = (uint32_t)h << 16;
    float f;
    memcpy(&f, &b, 4);
    return (double)f;
}

/* ---------------------------------------------------------------- instance */

enum { kStreamLen = 1, kStreamCol = 2, kStreamVal = 3, kStreamW = 4, kStreamEps = 5, kStreamPerm = 6 };

typedef struct {
    uint64_t seed;
    int64_t n, d;
    double kmean;
    int64_t kmin, kmax;
    double zipf_s;
    int storage; /* 1 float32, 2 bfloat16 */
    const double *cdf;     /* d: Zipf CDF over ranks */
    const int32_t *guide;  /* 16 d + 1: first rank whose CDF exceeds j / (16 d) */
    const int32_t *perm;   /* d: column of each rank */
    const double *w;       /* d: w* */
    int64_t *row_ptr;      /* n + 1 */
    int32_t *col;          /* nnz */
    double *val64;         /* nnz or NULL */
    uint16_t *val16;       /* nnz or NULL (bfloat16 bits) */
    double *labels;        /* n */
    uint64_t *row_hash;    /* n or NULL */
} Instance;

static int64_t row_length(const Instance *I, int64_t i) {
    uint64_t ctr = 0;
    const double z = gauss(I->seed, (uint64_t)kStreamLen << 56 | (uint64_t)i, &ctr);
    double k = floor(I->kmean + sqrt(I->kmean) * z + 0.5);
    if (k < (double)I->kmin) k = (double)I->kmin;
    if (k > (double)I->kmax) k = (double)I->kmax;
    if (k > (double)I->d) k = (double)I->d;
    return (int64_t)k;
}

static int32_t zipf_rank(const Instance *I, double u) {
    const int64_t m = 16 * I->d;
    int64_t g = (int64_t)(u * (double)m);
    if (g >= m) g = m - 1;
    int32_t k = I->guide[g];
    while (k < I->d - 1 && I->cdf[k] <= u) ++k;
    return k;
}

static int cmp_i32(const void *a, const void *b) {
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Fills row i (its range of row_ptr already set); table: scratch open-
 * addressing set of at least 2 kmax slots (stamped by row). */
static void fill_row(const Instance *I, int64_t i, int64_t *table_key, int64_t table_size) {
    const int64_t a = I->row_ptr[i], k = I->row_ptr[i + 1] - a;
    int32_t *cols = I->col + a;
    const uint64_t cstream = (uint64_t)kStreamCol << 56 | (uint64_t)i;
    uint64_t ctr = 0;
    int64_t got = 0;
    const uint64_t mask = (uint64_t)table_size - 1;
    while (got < k) {
        const int32_t c = I->perm[zipf_rank(I, u01(rnd(I->seed, cstream, ctr++)))];
        const int64_t want = ((int64_t)i + 1) << 32 | (int64_t)(uint32_t)c; /* row stamp and column */
        uint64_t h = fmix64((uint64_t)c) & mask;
        int dup = 0;
        for (;;) {
            const int64_t key = table_key[h];
            if (key == want) {
                dup = 1;
                break;
            }
            if ((key >> 32) != (int64_t)i + 1) break; /* empty, or a slot of an earlier row */
            h = (h + 1) & mask;
        }
        if (dup) continue;
        table_key[h] = want;
        cols[got++] = c;
    }
    qsort(cols, (size_t)k, sizeof(int32_t), cmp_i32);
    /* values: |N(0,1)|, unit row norm, storage grid */
    const uint64_t vstream = (uint64_t)kStreamVal << 56 | (uint64_t)i;
    uint64_t vctr = 0;
    double *tmp = (double *)malloc((size_t)(k > 0 ? k : 1) * sizeof(double));
    double ss = 0.0;
    for (int64_t j = 0; j < k; ++j) {
        const double g = fabs(gauss(I->seed, vstream, &vctr));
        tmp[j] = g;
        ss += g * g;
    }
    const double norm = sqrt(ss);
    double dot = 0.0;
    for (int64_t j = 0; j < k; ++j) {
        const double v = tmp[j] / norm;
        double q;
        if (I->storage == 2) {
            const uint16_t h = bf16_bits(v);
            q = bf16_value(h);
            if (I->val16) I->val16[a + j] = h;
        } else {
            q = to_f32_grid(v);
        }
        if (I->val64) I->val64[a + j] = q;
        dot += q * I->w[cols[j]];
    }
    free(tmp);
    uint64_t ectr = 0;
    const double eps = gauss(I->seed, (uint64_t)kStreamEps << 56 | (uint64_t)i, &ectr);
    I->labels[i] = (dot + 0.1 * eps) >= 0.0 ? 1.0 : -1.0;
    if (I->row_hash) { /* a checksum of the row: length, columns, stored values, label */
        uint64_t h = fmix64(0x5851F42D4C957F2DULL ^ (uint64_t)k);
        for (int64_t j = 0; j < k; ++j) {
            float f = I->val64 ? (float)I->val64[a + j] : (float)bf16_value(I->val16[a + j]);
            uint32_t b;
            memcpy(&b, &f, 4);
            h = fmix64(h ^ (uint64_t)(uint32_t)cols[j]);
            h = fmix64(h ^ ((uint64_t)b << 1));
        }
        I->row_hash[i] = fmix64(h ^ (I->labels[i] > 0.0 ? 1u : 2u));
    }
}

typedef struct {
    Instance *I;
    int64_t lo, hi;
    int pass; /* 0: row lengths into row_ptr[i + 1]; 1: rows */
} Task;

static void *worker(void *arg) {
    Task *t = (Task *)arg;
    Instance *I = t->I;
    if (t->pass == 0) {
        for (int64_t i = t->lo; i < t->hi; ++i) I->row_ptr[i + 1] = row_length(I, i);
        return NULL;
    }
    int64_t size = 64;
    while (size < 2 * I->kmax + 2) size <<= 1;
    int64_t *table = (int64_t *)malloc((size_t)size * sizeof(int64_t));
    if (!table) return (void *)1;
    for (int64_t j = 0; j < size; ++j) table[j] = 0;
    for (int64_t i = t->lo; i < t->hi; ++i) fill_row(I, i, table, size);
    free(table);
    return NULL;
}

static int run_pass(Instance *I, int pass, int threads) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t th[256];
    Task task[256];
    const int64_t chunk = (I->n + threads - 1) / threads;
    int started = 0, bad = 0;
    for (int t = 0; t < threads; ++t) {
        task[t].I = I;
        task[t].lo = (int64_t)t * chunk;
        task[t].hi = task[t].lo + chunk < I->n ? task[t].lo + chunk : I->n;
        task[t].pass = pass;
        if (task[t].lo >= task[t].hi) break;
        if (pthread_create(&th[t], NULL, worker, &task[t]) != 0) {
            if (worker(&task[t])) bad = 1; /* no thread: run it here */
            task[t].lo = task[t].hi;
            continue;
        }
        started = t + 1;
    }
    for (int t = 0; t < started; ++t) {
        if (task[t].lo >= task[t].hi) continue;
        void *r = NULL;
        pthread_join(th[t], &r);
        if (r) bad = 1;
    }
    return bad ? -1 : 0;
}

/* Shared per-instance tables: Zipf CDF and guide, column permutation, w*. */
static int setup(Instance *I, double **cdf, int32_t **guide, int32_t **perm, double **w) {
    const int64_t d = I->d;
    *cdf = (double *)malloc((size_t)d * sizeof(double));
    *guide = (int32_t *)malloc((size_t)(16 * d + 1) * sizeof(int32_t));
    *perm = (int32_t *)malloc((size_t)d * sizeof(int32_t));
    *w = (double *)malloc((size_t)d * sizeof(double));
    if (!*cdf || !*guide || !*perm || !*w) return -1;
    double total = 0.0;
    for (int64_t r = 0; r < d; ++r) {
        total += det_exp(-I->zipf_s * det_log((double)(r + 1)));
        (*cdf)[r] = total;
    }
    for (int64_t r = 0; r < d; ++r) (*cdf)[r] /= total;
    (*cdf)[d - 1] = 1.0;
    const int64_t m = 16 * d;
    int64_t k = 0;
    for (int64_t g = 0; g <= m; ++g) {
        const double u = (double)g / (double)m;
        while (k < d - 1 && (*cdf)[k] <= u) ++k;
        (*guide)[g] = (int32_t)k;
    }
    for (int64_t v = 0; v < d; ++v) (*perm)[v] = (int32_t)v;
    for (int64_t v = d - 1; v > 0; --v) { /* Fisher-Yates, j uniform in [0, v] by multiply-high */
        const uint64_t x = rnd(I->seed, (uint64_t)kStreamPerm << 56, (uint64_t)v);
        const int64_t j = (int64_t)(((__uint128_t)x * (__uint128_t)(uint64_t)(v + 1)) >> 64);
        const int32_t t = (*perm)[v];
        (*perm)[v] = (*perm)[j];
        (*perm)[j] = t;
    }
    for (int64_t v = 0; v < d; ++v) {
        uint64_t ctr = 0;
        (*w)[v] = gauss(I->seed, (uint64_t)kStreamW << 56 | (uint64_t)v, &ctr);
    }
    I->cdf = *cdf;
    I->guide = *guide;
    I->perm = *perm;
    I->w = *w;
    return 0;
}

/* Row pointers only: row_ptr[n + 1]; returns nnz, or -1 on bad arguments. */
int64_t synth_gen_rows(uint64_t seed, int64_t n, int64_t d, double kmean, int64_t kmin, int64_t kmax,
                       int64_t *row_ptr, int threads) {
    if (n < 1 || d < 1 || !(kmean >= 1.0) || kmin < 1 || kmax < kmin || !row_ptr) return -1;
    Instance I;
    memset(&I, 0, sizeof(I));
    I.seed = seed;
    I.n = n;
    I.d = d;
    I.kmean = kmean;
    I.kmin = kmin;
    I.kmax = kmax;
    I.row_ptr = row_ptr;
    row_ptr[0] = 0;
    if (run_pass(&I, 0, threads) != 0) return -1;
    for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
    return row_ptr[n];
}

/* Columns, values and labels for the row pointers of synth_gen_rows (same
 * arguments).  val64 (float64 on the storage grid) and val16 (bfloat16 bits,
 * storage 2 only) may each be NULL, not both.  row_hash (n, may be NULL)
 * receives a checksum of each row (length, columns, values, label).
 * Returns 0, or -1. */
int synth_gen_fill(uint64_t seed, int64_t n, int64_t d, double kmean, int64_t kmin, int64_t kmax, double zipf_s,
                   int storage, const int64_t *row_ptr, int32_t *col, double *val64, uint16_t *val16, double *labels,
                   uint64_t *row_hash, int threads) {
    if (n < 1 || d < 1 || d > 0x7fffffff || !row_ptr || !col || !labels || (storage != 1 && storage != 2) ||
        (val16 && storage != 2) || (!val64 && !val16) || !(zipf_s > 0.0))
        return -1;
    Instance I;
    memset(&I, 0, sizeof(I));
    I.seed = seed;
    I.n = n;
    I.d = d;
    I.kmean = kmean;
    I.kmin = kmin;
    I.kmax = kmax;
    I.zipf_s = zipf_s;
    I.storage = storage;
    I.row_ptr = (int64_t *)row_ptr;
    I.col = col;
    I.val64 = val64;
    I.val16 = val16;
    I.labels = labels;
    I.row_hash = row_hash;
    double *cdf = NULL, *w = NULL;
    int32_t *guide = NULL, *perm = NULL;
    int rc = setup(&I, &cdf, &guide, &perm, &w);
    if (rc == 0) rc = run_pass(&I, 1, threads);
    free(cdf);
    free(guide);
    free(perm);
    free(w);
    return rc;
}

/* The generator's own log and exp, exposed for the tests that check them
 * against the C library. */
double synth_gen_log(double x) { return det_log(x); }
double synth_gen_exp(double x) { return det_exp(x); }
