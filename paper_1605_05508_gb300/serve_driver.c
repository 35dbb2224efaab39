/*
 * serve_driver.c -- drives the serving loop of libkf (kf_serve_start,
 * kf_submit, kf_poll) through its C ABI from native threads, so that served
 * events/s and latencies measure the library and not a scripting harness.
 *
 * usage: kf_serve_driver POOL REQUESTS RATE SUBMIT_THREADS SEED [REFIT [BUILD_SCAN LIST_WIDTH]]
 *   POOL            event pool file (format below)
 *   REQUESTS        requests to submit; request i is pool event i mod P
 *   RATE            mean arrival rate in events/s (Poisson arrivals), or 0 to
 *                   submit back to back (saturation)
 *   SUBMIT_THREADS  submitting threads (request i goes to thread i mod T and
 *                   is submitted at its arrival time, or when the queue has room)
 *   SEED            seed of the arrival times
 *   REFIT           1: each request also re-fits its best candidates (default 0)
 *   BUILD_SCAN,     the build's thread layout and child-list width in the
 *   LIST_WIDTH      context's launch parameters (kf_tuning; default 4 and 8)
 * One line of JSON on stdout: events/s over the whole run (first submit to
 * last result), p50 / p99 / mean latency (kf_submit to results on the host, as
 * the library measures it), and the loop's counters over the run (launches,
 * iterations, the scheduler thread's busy / GPU-wait / idle time).
 *
 * Pool file (little-endian): "KFSP", int32 version (1), float bz_tesla,
 * int32 n_layers, float radius[n_layers], float sigma_xy, float sigma_z,
 * float chi2_cut, int32 n_seed_layers, int32 n_build_layers, int32 max_cands,
 * int32 max_slots, int64 device_arena_bytes, int64 host_arena_bytes,
 * int32 n_events; then per event: int32 n_seeds, int64 n_hits, and the arrays
 * of kf_event in order -- seed_par [6][n] f32, seed_cov [21][n] f32,
 * seed_charge [n] i8, seed_hits [Ls][3][n] f32, seed_valid [Ls][n] u8,
 * layer_xyz [3][n_hits] f32, layer_off [Lb + 1] i64.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "kf.h"

typedef struct {
    int32_t n;
    int64_t nh;
    float *par, *cov, *shits, *xyz;
    int8_t *q;
    uint8_t *sval;
    int64_t *off;
    kf_event ev;
    kf_event_result res;
} PoolEvent;

static kf_ctx *g_ctx;
static PoolEvent *g_pool;
static int g_np, g_m, g_threads, g_ls, g_lb;
static double *g_due;          /* arrival time of request i (s after start) */
static uint64_t *g_ticket;
static volatile int *g_submitted;
static double *g_lat;
static double g_t0;
static int g_fail;

static double now_s(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

static void sleep_s(double s)
{
    if (s <= 0) return;
    struct timespec ts;
    ts.tv_sec = (time_t)s;
    ts.tv_nsec = (long)((s - (double)ts.tv_sec) * 1e9);
    nanosleep(&ts, NULL);
}

static void *read_n(FILE *f, size_t bytes)
{
    void *p = malloc(bytes ? bytes : 1);
    if (!p || fread(p, 1, bytes, f) != bytes) {
        fprintf(stderr, "pool file truncated\n");
        exit(2);
    }
    return p;
}

#define READ(f, x)                                         \
    do {                                                   \
        if (fread(&(x), sizeof(x), 1, f) != 1) {           \
            fprintf(stderr, "pool file truncated\n");      \
            exit(2);                                       \
        }                                                  \
    } while (0)

static int submit_one(int i)
{
    PoolEvent *e = &g_pool[i % g_np];
    for (;;) {
        uint64_t t;
        const int rc = kf_submit(g_ctx, &e->ev, &t);
        if (rc == KF_OK) {
            g_ticket[i] = t;
            __atomic_store_n(&g_submitted[i], 1, __ATOMIC_RELEASE);
            return 0;
        }
        if (rc != KF_EAGAIN) {
            fprintf(stderr, "kf_submit: %s\n", kf_strerror(rc));
            return rc;
        }
        sleep_s(50e-6); /* queue or host arena full: retry */
    }
}

static void *submitter(void *arg)
{
    const int t = (int)(intptr_t)arg;
    for (int i = t; i < g_m; i += g_threads) {
        sleep_s(g_t0 + g_due[i] - now_s());
        if (submit_one(i)) {
            g_fail = 1;
            return NULL;
        }
    }
    return NULL;
}

static int cmp_d(const void *a, const void *b)
{
    const double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : x > y;
}

int main(int argc, char **argv)
{
    if (argc < 6) {
        fprintf(stderr, "usage: %s POOL REQUESTS RATE SUBMIT_THREADS SEED [REFIT [BUILD_SCAN LIST_WIDTH]]\n",
                argv[0]);
        return 2;
    }
    g_m = atoi(argv[2]);
    const double rate = atof(argv[3]);
    g_threads = atoi(argv[4]);
    uint64_t rng = (uint64_t)strtoull(argv[5], NULL, 10) * 0x9E3779B97F4A7C15ull + 1;
    const int refit = argc > 6 ? atoi(argv[6]) : 0;
    const int build_scan = argc > 7 ? atoi(argv[7]) : 4, list_width = argc > 8 ? atoi(argv[8]) : 8;
    if (g_m < 1 || g_threads < 1 || rate < 0) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) {
        perror("pool");
        return 2;
    }
    char magic[4];
    int32_t version, nl, ls, lb, mc, slots, ne;
    float bz, sxy, sz, cut;
    int64_t darena, harena;
    if (fread(magic, 1, 4, f) != 4 || memcmp(magic, "KFSP", 4)) {
        fprintf(stderr, "not a pool file\n");
        return 2;
    }
    READ(f, version);
    READ(f, bz);
    READ(f, nl);
    if (version != 1 || nl < 1 || nl > 64) return 2;
    float *radius = (float *)read_n(f, sizeof(float) * nl);
    READ(f, sxy);
    READ(f, sz);
    READ(f, cut);
    READ(f, ls);
    READ(f, lb);
    READ(f, mc);
    READ(f, slots);
    READ(f, darena);
    READ(f, harena);
    READ(f, ne);
    if (ne < 1 || ls < 1 || lb < 1) return 2;
    g_ls = ls;
    g_lb = lb;
    g_np = ne;
    g_pool = (PoolEvent *)calloc(ne, sizeof(PoolEvent));
    for (int e = 0; e < ne; ++e) {
        PoolEvent *p = &g_pool[e];
        READ(f, p->n);
        READ(f, p->nh);
        const size_t n = (size_t)p->n;
        p->par = (float *)read_n(f, 6 * n * 4);
        p->cov = (float *)read_n(f, 21 * n * 4);
        p->q = (int8_t *)read_n(f, n);
        p->shits = (float *)read_n(f, (size_t)ls * 3 * n * 4);
        p->sval = (uint8_t *)read_n(f, (size_t)ls * n);
        p->xyz = (float *)read_n(f, 3 * (size_t)p->nh * 4);
        p->off = (int64_t *)read_n(f, (size_t)(lb + 1) * 8);
        p->ev = (kf_event){p->n, p->par, p->cov, p->q, p->shits, p->sval, p->xyz, p->off};
        memset(&p->res, 0, sizeof p->res);
        p->res.best_par = (float *)malloc(6 * n * 4);
        p->res.chi2_tot = (float *)malloc(n * 4);
        p->res.n_hits = (int32_t *)malloc(n * 4);
        p->res.status = (int32_t *)malloc(n * 4);
        p->res.hit_idx = (int32_t *)malloc((size_t)lb * n * 4);
        if (refit) {
            p->res.refit_par = (float *)malloc(6 * n * 4);
            p->res.refit_status = (int32_t *)malloc(n * 4);
        }
    }
    fclose(f);

    kf_config cfg = {bz, nl, radius, sxy, sz, cut, mc, NULL, 0.13957f};
    int rc = kf_create(&g_ctx, &cfg, 0, 0);
    if (rc) {
        fprintf(stderr, "kf_create: %s\n", kf_strerror(rc));
        return 1;
    }
    kf_tuning tune;
    kf_get_tuning(g_ctx, &tune);
    tune.build_scan = build_scan;
    tune.build_list_width = list_width;
    tune.bin_unordered = 1;
    rc = kf_set_tuning(g_ctx, &tune);
    if (rc) {
        fprintf(stderr, "kf_set_tuning: %s\n", kf_strerror(rc));
        return 1;
    }
    kf_serve_config sc = {ls, lb, mc, slots, 1 << 16, refit, (size_t)darena, (size_t)harena, 0};
    rc = kf_serve_start(g_ctx, &sc);
    if (rc) {
        fprintf(stderr, "kf_serve_start: %s\n", kf_strerror(rc));
        return 1;
    }
    /* warm-up: a few events one at a time */
    for (int i = 0; i < 4 && i < ne; ++i) {
        uint64_t t;
        if (kf_submit(g_ctx, &g_pool[i].ev, &t) || kf_poll(g_ctx, t, &g_pool[i].res, -1)) return 1;
    }
    g_due = (double *)malloc(sizeof(double) * g_m);
    g_ticket = (uint64_t *)calloc(g_m, sizeof(uint64_t));
    g_submitted = (volatile int *)calloc(g_m, sizeof(int));
    g_lat = (double *)malloc(sizeof(double) * g_m);
    double t = 0;
    for (int i = 0; i < g_m; ++i) { /* exponential gaps (xorshift64*) */
        if (rate > 0) {
            rng ^= rng >> 12;
            rng ^= rng << 25;
            rng ^= rng >> 27;
            const double u = ((rng * 0x2545F4914F6CDD1Dull) >> 11) * (1.0 / 9007199254740992.0);
            t += -log(1.0 - u) / rate;
        }
        g_due[i] = t;
    }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * g_threads);
    kf_serve_stats st0;
    kf_serve_stats_get(g_ctx, &st0);
    g_t0 = now_s();
    for (int k = 0; k < g_threads; ++k) pthread_create(&th[k], NULL, submitter, (void *)(intptr_t)k);
    /* this thread polls the requests in order */
    for (int i = 0; i < g_m && !g_fail; ++i) {
        while (!__atomic_load_n(&g_submitted[i], __ATOMIC_ACQUIRE) && !g_fail) sleep_s(20e-6);
        if (g_fail) break;
        kf_event_result *r = &g_pool[i % g_np].res;
        rc = kf_poll(g_ctx, g_ticket[i], r, -1);
        if (rc) {
            fprintf(stderr, "kf_poll: %s\n", kf_strerror(rc));
            g_fail = 1;
            break;
        }
        g_lat[i] = r->latency_ms;
    }
    const double wall = now_s() - g_t0;
    for (int k = 0; k < g_threads; ++k) pthread_join(th[k], NULL);
    if (g_fail) return 1;
    kf_serve_stats st;
    kf_serve_stats_get(g_ctx, &st);
    kf_serve_stop(g_ctx);
    kf_destroy(g_ctx);
    double mean = 0;
    for (int i = 0; i < g_m; ++i) mean += g_lat[i];
    mean /= g_m;
    qsort(g_lat, g_m, sizeof(double), cmp_d);
    const double p50 = g_lat[(int)(0.50 * (g_m - 1))], p99 = g_lat[(int)(0.99 * (g_m - 1))];
    printf("{\"requests\": %d, \"offered_events_per_s\": %.3f, \"submit_threads\": %d, \"wall_s\": %.6f, "
           "\"events_per_s\": %.3f, \"p50_ms\": %.4f, \"p99_ms\": %.4f, \"mean_ms\": %.4f, "
           "\"max_resident\": %d, \"step_launches\": %llu, \"iterations\": %llu, \"sched_busy_ms\": %.3f, "
           "\"sched_gpu_wait_ms\": %.3f, \"sched_idle_ms\": %.3f}\n",
           g_m, rate, g_threads, wall, g_m / wall, p50, p99, mean, st.max_resident,
           (unsigned long long)(st.step_launches - st0.step_launches),
           (unsigned long long)(st.iterations - st0.iterations), st.sched_busy_ms - st0.sched_busy_ms,
           st.sched_gpu_wait_ms - st0.sched_gpu_wait_ms, st.sched_idle_ms - st0.sched_idle_ms);
    return 0;
}
