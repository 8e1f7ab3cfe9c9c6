/*
 * Lock-free asynchronous Sparse SAGA on the host's cores (ASAGA, Algorithm 2)
 * -- a CPU timing baseline for the GPU solver, in the style of the paper's
 * own multi-core implementation.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of this directory: only the tests
 * and the benchmark's CPU-baseline leg may load it.  It is not a checker
 * (its result depends on the thread interleaving); the serial saga_ref.c is.
 *
 * What it computes: T threads share x, abar and alpha (float64).  Each
 * thread repeatedly samples a row i, reads x^ on S_i and alpha_i without any
 * lock (the inconsistent read of Sec. 3.1), forms delta = phi'_i(a_i.x^) -
 * alpha^_i, and adds
 *     x_v    += -gamma (delta a_iv + D_v abar^_v + lambda D_v x^_v),
 *     abar_v += delta a_iv / n          (v in S_i),
 *     alpha_i += delta,
 * each as an atomic compare-and-swap loop on the 64-bit word, which is what
 * App. G.2 found necessary for convergence to high precision.  Rows are the
 * SplitMix64 stream of the solver (update t takes output t+1 of the stream
 * seeded with `seed`, row floor(u n / 2^64)); thread j takes updates
 * j, j + T, j + 2T, ...
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <string.h>

#define CPU_LOSS_LOGISTIC 0

static double cpu_phi_prime(int loss, double z, double b)
{
    if (loss == CPU_LOSS_LOGISTIC) {
        double t = b * z;
        if (t >= 0.0) {
            double e = exp(-t);
            return -b * e / (1.0 + e);
        }
        return -b / (1.0 + exp(t));
    }
    return z - b;
}

static uint64_t cpu_splitmix(uint64_t seed, uint64_t t)
{
    uint64_t z = seed + (t + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double load_relaxed(const double *p)
{
    uint64_t bits = __atomic_load_n((const uint64_t *)p, __ATOMIC_RELAXED);
    double v;
    memcpy(&v, &bits, sizeof v);
    return v;
}

static void cas_add(double *p, double inc)
{
    uint64_t *q = (uint64_t *)p;
    uint64_t old = __atomic_load_n(q, __ATOMIC_RELAXED), next;
    do {
        double v;
        memcpy(&v, &old, sizeof v);
        v += inc;
        memcpy(&next, &v, sizeof next);
    } while (!__atomic_compare_exchange_n(q, &old, next, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED));
}

typedef struct {
    int64_t n, d;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const double *val, *labels, *D;
    int loss;
    double lambda, gamma;
    double *x, *alpha, *abar;
    uint64_t seed, t_begin;
    int64_t count;
    int threads, id;
    double *zbuf;  /* per-thread scratch of max-row-length entries: x^ on S_i */
} cpu_job;

static void *cpu_worker(void *arg)
{
    cpu_job *J = (cpu_job *)arg;
    for (int64_t t = J->id; t < J->count; t += J->threads) {
        uint64_t u = cpu_splitmix(J->seed, J->t_begin + (uint64_t)t);
        int64_t i = (int64_t)(((unsigned __int128)u * (uint64_t)J->n) >> 64);
        int64_t lo = J->row_ptr[i], hi = J->row_ptr[i + 1];
        double z = 0.0;
        for (int64_t k = lo; k < hi; ++k) {
            double xv = load_relaxed(J->x + J->col_idx[k]);
            J->zbuf[k - lo] = xv;
            z += J->val[k] * xv;
        }
        double delta = cpu_phi_prime(J->loss, z, J->labels[i]) - load_relaxed(J->alpha + i);
        for (int64_t k = lo; k < hi; ++k) {
            int32_t v = J->col_idx[k];
            double a = J->val[k];
            double Dv = J->D[v];
            double step = delta * a + Dv * load_relaxed(J->abar + v) + J->lambda * Dv * J->zbuf[k - lo];
            cas_add(J->x + v, -J->gamma * step);
            cas_add(J->abar + v, delta * a / (double)J->n);
        }
        cas_add(J->alpha + i, delta);
    }
    return NULL;
}

/*
 * Runs `count` asynchronous updates numbered t_begin .. t_begin+count-1 on
 * `threads` threads (1..256).  zbuf: threads * max_row_len doubles of
 * scratch.  Returns 0, or -1 if a thread could not be started (the updates
 * of the started threads have run).
 */
int cpu_asaga(int64_t n, int64_t d, const int64_t *row_ptr, const int32_t *col_idx, const double *val,
              const double *labels, int loss, double lambda, double gamma, const double *D, double *x,
              double *alpha, double *abar, uint64_t seed, uint64_t t_begin, int64_t count, int threads,
              double *zbuf, int64_t max_row_len)
{
    enum { kMaxThreads = 256 };
    pthread_t tid[kMaxThreads];
    cpu_job jobs[kMaxThreads];
    int started = 0, rc = 0;
    (void)d;
    if (threads < 1)
        threads = 1;
    if (threads > kMaxThreads)
        threads = kMaxThreads;
    for (int j = 0; j < threads; ++j) {
        cpu_job J = {n, d, row_ptr, col_idx, val, labels, D, loss, lambda, gamma, x, alpha, abar,
                     seed, t_begin, count, threads, j, zbuf + (int64_t)j * max_row_len};
        jobs[j] = J;
        if (pthread_create(&tid[j], NULL, cpu_worker, &jobs[j]) != 0) {
            rc = -1;
            break;
        }
        ++started;
    }
    for (int j = 0; j < started; ++j)
        pthread_join(tid[j], NULL);
    return rc;
}
