/*
 * rt_oracle_threads.c -- the oracle's forward march on several host threads.
 *
 * TEST INFRASTRUCTURE ONLY (like rt_oracle.c): used by the tests and by the CPU-baseline /
 * reference legs of the benchmark, never by the product path.
 *
 * Nothing here changes what is computed. The field of Sec. 2 is a sum over sources and rays,
 * so the (source, block of rays) items are independent: each thread runs oracle_advance on its
 * share of the items into a private FP64 partial field, and the partial fields are added to the
 * output in thread order (the cells split into slices, one per thread, each slice adding the
 * partial fields 0, 1, ... in turn). The result is therefore the same for every run with the
 * same thread count, and differs from the one-thread result only by the order of FP64
 * additions.
 */
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

int oracle_advance(const double *j, const double *kappa, int nf, int n0, int n1, int n2,
                   const double *src, int nsrc, int num_rays, double ds, int ns,
                   int geom_mode, int kappa_mode, int ray_begin, int ray_end, double *out);

typedef struct work {
    const double *j, *kappa, *src;
    int nf, n0, n1, n2, nsrc, num_rays, ns, geom_mode, kappa_mode, ray_begin, ray_end, block;
    double ds;
    int thread, nthreads, status;
    size_t field;
    double *partial;
    struct work *all;   /* every thread's record (for the reduction phase) */
    double *out;
} work_t;

static void *run_items(void *arg)
{
    work_t *w = (work_t *)arg;
    /* the owning thread clears its partial field, so its pages are first touched in parallel */
    memset(w->partial, 0, w->field * sizeof(double));
    const int blocks = (w->ray_end - w->ray_begin + w->block - 1) / w->block;
    const long items = (long)w->nsrc * blocks;
    for (long it = w->thread; it < items; it += w->nthreads) {
        const int s = (int)(it / blocks), b = (int)(it % blocks);
        const int rb = w->ray_begin + b * w->block;
        const int re = rb + w->block < w->ray_end ? rb + w->block : w->ray_end;
        if (oracle_advance(w->j, w->kappa, w->nf, w->n0, w->n1, w->n2, w->src + 3 * (long)s, 1, w->num_rays,
                           w->ds, w->ns, w->geom_mode, w->kappa_mode, rb, re, w->partial) != 0) {
            w->status = -1;
            return NULL;
        }
    }
    return NULL;
}

/* Reduction phase: thread t adds, for its slice of the cells, the partial fields of threads
 * 0, 1, ..., nthreads-1 in that order (the same order for every cell). */
static void *reduce_slice(void *arg)
{
    work_t *w = (work_t *)arg;
    const size_t lo = w->field * (size_t)w->thread / (size_t)w->nthreads;
    const size_t hi = w->field * (size_t)(w->thread + 1) / (size_t)w->nthreads;
    for (int t = 0; t < w->nthreads; ++t) {
        const double *p = w->all[t].partial;
        for (size_t i = lo; i < hi; ++i) w->out[i] += p[i];
    }
    return NULL;
}

/* Same arguments and result as oracle_advance (out ACCUMULATED), traced by nthreads threads
 * over items of (one source, ray_block rays). Returns 0, or -1 on invalid arguments or an
 * allocation / thread failure. */
int oracle_advance_threads(const double *j, const double *kappa, int nf, int n0, int n1, int n2,
                           const double *src, int nsrc, int num_rays, double ds, int ns,
                           int geom_mode, int kappa_mode, int ray_begin, int ray_end, int nthreads,
                           int ray_block, double *out)
{
    if (nthreads < 1 || nthreads > 1024 || ray_block < 1 || nf < 1 || n0 < 1 || n1 < 1 || n2 < 1 || nsrc < 0 ||
        ray_begin < 0 || ray_end < ray_begin || ray_end > num_rays)
        return -1;
    if (nsrc == 0 || ray_end == ray_begin || ns == 0)
        return oracle_advance(j, kappa, nf, n0, n1, n2, src, nsrc, num_rays, ds, ns, geom_mode, kappa_mode,
                              ray_begin, ray_end, out);
    const size_t field = (size_t)nf * n0 * n1 * n2;
    work_t *w = (work_t *)calloc((size_t)nthreads, sizeof(work_t));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int rc = (w && tid) ? 0 : -1;
    int started = 0;
    for (int t = 0; t < nthreads && rc == 0; ++t) {
        work_t *x = &w[t];
        x->j = j; x->kappa = kappa; x->src = src;
        x->nf = nf; x->n0 = n0; x->n1 = n1; x->n2 = n2; x->nsrc = nsrc; x->num_rays = num_rays; x->ns = ns;
        x->geom_mode = geom_mode; x->kappa_mode = kappa_mode; x->ray_begin = ray_begin; x->ray_end = ray_end;
        x->block = ray_block; x->ds = ds; x->thread = t; x->nthreads = nthreads; x->status = 0;
        x->field = field; x->all = w; x->out = out;
        x->partial = (double *)malloc(field * sizeof(double));
        if (!x->partial || pthread_create(&tid[t], NULL, run_items, x) != 0) {
            rc = -1;
            break;
        }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    for (int t = 0; t < started && rc == 0; ++t)
        if (w[t].status != 0) rc = -1;
    if (rc == 0) {
        int running = 0;
        for (int t = 0; t < nthreads; ++t) {
            if (pthread_create(&tid[t], NULL, reduce_slice, &w[t]) != 0) break;
            ++running;
        }
        for (int t = 0; t < running; ++t) pthread_join(tid[t], NULL);
        /* a slice whose thread could not start is added here, in the same order */
        for (int t = running; t < nthreads; ++t) reduce_slice(&w[t]);
    }
    if (w)
        for (int t = 0; t < nthreads; ++t) free(w[t].partial);
    free(w);
    free(tid);
    return rc;
}
