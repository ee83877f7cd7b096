/*
 * rt_oracle.c -- plain, slow FP64 CPU oracle for the Ray-trax emission-absorption march.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load this file;
 * only the tests, the smoke check and the CPU baseline leg of the benchmark do. It shares no
 * code, header or table with the CUDA library.
 *
 * What it computes (paper Sec. 2, "Method and code structure"):
 *   - Eq. 2, applied per substep k -> k+1 along every ray:
 *         x_{k+1}   = x_k + n * ds
 *         tau_{k+1} = tau_k + kappa(x_k) ds
 *         I_{k+1}   = I_k exp(-kappa(x_k) ds) + j(x_k) exp(-tau_k) ds
 *   - N_s = ceil(c dt / ds) substeps, or an optional cap (Sec. 2, text after Eq. 2; App. A).
 *   - N_Omega directions on a Fibonacci (golden-angle) lattice; per-ray deposits are summed and
 *     scaled by 4 pi / N_Omega (Sec. 2).
 *   - j read by trilinear interpolation, kappa by nearest neighbour at the cell index of the
 *     previous position x_k, the post-attenuation I_{k+1} deposited with the same trilinear
 *     weights, indices clamped to the box (Sec. 2).
 *   - several sources: loop and sum (Sec. 2); frequency bins: an independent batch axis
 *     (Sec. 2, "Frequency-bin agnosticism").
 *
 * Readings taken where the paper is silent (each mirrored, independently, by the CUDA path):
 *   R1 lattice: z_i = 1 - (2i+1)/N, rho_i = sqrt(1 - z_i^2), phi_i = i * pi (3 - sqrt 5) mod 2 pi,
 *      n_i = (rho cos phi, rho sin phi, z); components (x, y, z) index array axes (0, 1, 2).
 *   R2 grid coordinates are node-centred (voxel v sits at coordinate v). Per axis:
 *      f = floor(x), i0 = clamp(f, 0, N-1), i1 = clamp(f+1, 0, N-1), t = x - f (unclamped),
 *      weights (1-t, t). Rays that leave the box keep marching and deposit on the boundary.
 *   R3 kappa_mode 0: kappa at (i0, i0, i0) = clamped floor of x_k ("the cell index used for the
 *      previous position"); kappa_mode 1: clamped floor(x_k + 1/2) (round to nearest).
 *      The paper does not fix which; this choice is parity unpinned by the paper.
 *   R4 N_s = ceil(c dt / ds) evaluated in FP64 with a relative guard of 1e-9 against roundoff,
 *      then min(N_s, cap) when cap > 0. Substeps k = 0 .. N_s-1.
 *   R5 deposit at x_k (the point where j was read), value I_{k+1}.
 *   R6 geometry precision. geom_mode 0 ("parity"): direction rounded to FP32, d = fl32(n ds),
 *      x_{k+1} = fl32(x_k + d), floor and t = fl32(x - floor x) in FP32, so that cell indices
 *      are those an FP32 implementation must produce; everything radiometric (weights,
 *      exponentials, I, tau, sums) is FP64. geom_mode 1 ("pure"): geometry in FP64 too.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared rt_oracle.c -lm   (no fast-math).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

/* ---- R4: substep count (Sec. 2 after Eq. 2; App. A "N_s") ---------------------------- */
int oracle_num_substeps(double ds, double c, double dt, int cap)
{
    if (!(ds > 0.0) || !(c > 0.0) || !(dt >= 0.0)) return -1;
    double q = c * dt / ds;
    double ns = ceil(q - 1e-9 * q);
    if (ns < 0.0) ns = 0.0;
    if (ns > 2147483647.0) return -1;
    int n = (int)ns;
    if (cap > 0 && n > cap) n = cap;
    return n;
}

/* ---- R1: Fibonacci / golden-angle lattice (Sec. 2) ----------------------------------- */
void oracle_fibonacci_dirs(int n, double *out)
{
    const double golden = ORACLE_PI * (3.0 - sqrt(5.0));
    for (int i = 0; i < n; ++i) {
        double z = 1.0 - (2.0 * i + 1.0) / (double)n;
        double rho = sqrt(fmax(0.0, 1.0 - z * z));
        double phi = fmod((double)i * golden, 2.0 * ORACLE_PI);
        out[3 * i + 0] = rho * cos(phi);
        out[3 * i + 1] = rho * sin(phi);
        out[3 * i + 2] = z;
    }
}

/* FP32 copy of the lattice: each FP64 component rounded once to the nearest float. */
void oracle_fibonacci_dirs_f32(int n, float *out)
{
    double *tmp = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    oracle_fibonacci_dirs(n, tmp);
    for (int i = 0; i < 3 * n; ++i) out[i] = (float)tmp[i];
    free(tmp);
}

/* ---- R2/R3: one sample point on the grid -------------------------------------------- */
typedef struct {
    long cell[8];   /* flat indices of the 8 trilinear corners */
    double w[8];    /* their weights */
    long nn;        /* flat index of the kappa cell */
    double t[3];    /* fractions x - floor(x) per axis (the weights are products of t, 1 - t) */
} sample_t;

static long clamp_index(double f, int n)
{
    if (f < 0.0) return 0;
    if (f > (double)(n - 1)) return n - 1;
    return (long)f;
}

/* Corner c = (c0, c1, c2) bits: bit 2 -> axis 0, bit 1 -> axis 1, bit 0 -> axis 2. */
static void make_sample(const double f[3], const double t[3], const double fnn[3],
                        int n0, int n1, int n2, sample_t *s)
{
    const int ext[3] = {n0, n1, n2};
    long lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = clamp_index(f[a], ext[a]);
        hi[a] = clamp_index(f[a] + 1.0, ext[a]);
    }
    for (int c = 0; c < 8; ++c) {
        int b0 = (c >> 2) & 1, b1 = (c >> 1) & 1, b2 = c & 1;
        long i = b0 ? hi[0] : lo[0];
        long jj = b1 ? hi[1] : lo[1];
        long k = b2 ? hi[2] : lo[2];
        s->cell[c] = (i * n1 + jj) * n2 + k;
        s->w[c] = (b0 ? t[0] : 1.0 - t[0]) * (b1 ? t[1] : 1.0 - t[1]) * (b2 ? t[2] : 1.0 - t[2]);
    }
    long m0 = clamp_index(fnn[0], n0), m1 = clamp_index(fnn[1], n1), m2 = clamp_index(fnn[2], n2);
    s->nn = (m0 * n1 + m1) * n2 + m2;
    for (int a = 0; a < 3; ++a) s->t[a] = t[a];
}

/* Geometry of one ray: positions x_0 .. x_{ns-1} turned into samples (R2, R3, R6). */
static void ray_samples(const double src[3], const double n64[3], double ds, int ns,
                        int geom_mode, int kappa_mode, int n0, int n1, int n2, sample_t *out)
{
    if (geom_mode == 0) {
        float x[3], d[3];
        float ds32 = (float)ds;
        for (int a = 0; a < 3; ++a) {
            float na = (float)n64[a];
            d[a] = na * ds32;              /* one FP32 product per component */
            x[a] = (float)src[a];
        }
        for (int k = 0; k < ns; ++k) {
            double f[3], t[3], fnn[3];
            for (int a = 0; a < 3; ++a) {
                float fl = floorf(x[a]);
                float tf = x[a] - fl;      /* FP32 subtraction */
                f[a] = (double)fl;
                t[a] = (double)tf;
                fnn[a] = kappa_mode ? (double)floorf(x[a] + 0.5f) : (double)fl;
            }
            make_sample(f, t, fnn, n0, n1, n2, &out[k]);
            for (int a = 0; a < 3; ++a) x[a] = x[a] + d[a];   /* FP32 addition */
        }
    } else {
        double x[3], d[3];
        for (int a = 0; a < 3; ++a) { d[a] = n64[a] * ds; x[a] = src[a]; }
        for (int k = 0; k < ns; ++k) {
            double f[3], t[3], fnn[3];
            for (int a = 0; a < 3; ++a) {
                f[a] = floor(x[a]);
                t[a] = x[a] - f[a];
                fnn[a] = kappa_mode ? floor(x[a] + 0.5) : f[a];
            }
            make_sample(f, t, fnn, n0, n1, n2, &out[k]);
            for (int a = 0; a < 3; ++a) x[a] = x[a] + d[a];
        }
    }
}

static int check_args(int nf, int n0, int n1, int n2, int nsrc, int num_rays, double ds, int ns,
                      int ray_begin, int ray_end)
{
    if (nf < 1 || n0 < 1 || n1 < 1 || n2 < 1 || nsrc < 0 || num_rays < 1 || !(ds > 0.0) || ns < 0)
        return -1;
    if (ray_begin < 0 || ray_end > num_rays || ray_begin > ray_end) return -1;
    return 0;
}

/* ---- Forward march: Eq. 2 per substep, deposit R5, sum over rays/sources/bins (Sec. 2) --
 * j, kappa: [nf][n0][n1][n2]; src: [nsrc][3] grid coordinates; out: [nf][n0][n1][n2],
 * ACCUMULATED (the caller zeroes it). Rays ray_begin .. ray_end-1 of the lattice are traced
 * (a shard of the direction set; the full set is 0 .. num_rays), each weighted 4 pi / num_rays.
 * Returns 0, or -1 on invalid arguments / allocation failure. */
int oracle_advance(const double *j, const double *kappa, int nf, int n0, int n1, int n2,
                   const double *src, int nsrc, int num_rays, double ds, int ns,
                   int geom_mode, int kappa_mode, int ray_begin, int ray_end, double *out)
{
    if (check_args(nf, n0, n1, n2, nsrc, num_rays, ds, ns, ray_begin, ray_end)) return -1;
    if (ns == 0 || nsrc == 0 || ray_end == ray_begin) return 0;
    const long ncell = (long)n0 * n1 * n2;
    const double scale = 4.0 * ORACLE_PI / (double)num_rays;
    const double dsr = geom_mode == 0 ? (double)(float)ds : ds;
    double *dirs = (double *)malloc(sizeof(double) * 3 * (size_t)num_rays);
    sample_t *smp = (sample_t *)malloc(sizeof(sample_t) * (size_t)ns);
    if (!dirs || !smp) { free(dirs); free(smp); return -1; }
    oracle_fibonacci_dirs(num_rays, dirs);

    for (int s = 0; s < nsrc; ++s) {
        for (int r = ray_begin; r < ray_end; ++r) {
            ray_samples(&src[3 * s], &dirs[3 * r], ds, ns, geom_mode, kappa_mode, n0, n1, n2, smp);
            for (int b = 0; b < nf; ++b) {
                const double *jb = j + (long)b * ncell;
                const double *kb = kappa + (long)b * ncell;
                double *ob = out + (long)b * ncell;
                double I = 0.0, tau = 0.0;
                for (int k = 0; k < ns; ++k) {
                    const sample_t *q = &smp[k];
                    double jk = 0.0;
                    for (int c = 0; c < 8; ++c) jk += q->w[c] * jb[q->cell[c]];
                    double kk = kb[q->nn];
                    double att = exp(-kk * dsr);
                    double emis = jk * exp(-tau) * dsr;
                    I = I * att + emis;                    /* Eq. 2, I update   */
                    tau = tau + kk * dsr;                  /* Eq. 2, tau update */
                    for (int c = 0; c < 8; ++c) ob[q->cell[c]] += scale * q->w[c] * I;
                }
            }
        }
    }
    free(dirs);
    free(smp);
    return 0;
}

/* ---- Reverse-mode adjoint of oracle_advance ------------------------------------------
 * For a loss L with G = dL/d(out), accumulates dL/dj into dj and dL/dkappa into dkappa.
 * Derived from Eq. 2 by the chain rule with, per ray and bin,
 *   g_k       = scale * sum_c w_{k,c} G[c_{k,c}]            (deposit of I_{k+1})
 *   lam_{k+1} = g_k + a_{k+1} lam_{k+2},  lam_{N_s+1} = 0,   a_k = exp(-kappa_k ds)
 *   mu_k      = mu_{k+1} + lam_{k+1} j_k E_k ds,  mu_{N_s} = 0,  E_k = exp(-tau_k)
 *   dL/dj_k   = lam_{k+1} E_k ds        -> spread to the 8 corners with w_{k,c}
 *   dL/dkap_k = -ds (lam_{k+1} I_k a_k + mu_{k+1})  -> the kappa cell of substep k.
 * The forward state of each ray is kept in full (no checkpointing). */
int oracle_backward(const double *j, const double *kappa, int nf, int n0, int n1, int n2,
                    const double *src, int nsrc, int num_rays, double ds, int ns,
                    int geom_mode, int kappa_mode, int ray_begin, int ray_end,
                    const double *G, double *dj, double *dkappa)
{
    if (check_args(nf, n0, n1, n2, nsrc, num_rays, ds, ns, ray_begin, ray_end)) return -1;
    if (ns == 0 || nsrc == 0 || ray_end == ray_begin) return 0;
    const long ncell = (long)n0 * n1 * n2;
    const double scale = 4.0 * ORACLE_PI / (double)num_rays;
    const double dsr = geom_mode == 0 ? (double)(float)ds : ds;
    double *dirs = (double *)malloc(sizeof(double) * 3 * (size_t)num_rays);
    sample_t *smp = (sample_t *)malloc(sizeof(sample_t) * (size_t)ns);
    double *Ik = (double *)malloc(sizeof(double) * (size_t)ns);   /* I_k   */
    double *Ek = (double *)malloc(sizeof(double) * (size_t)ns);   /* E_k   */
    double *ak = (double *)malloc(sizeof(double) * (size_t)ns);   /* a_k   */
    double *jv = (double *)malloc(sizeof(double) * (size_t)ns);   /* j_k   */
    if (!dirs || !smp || !Ik || !Ek || !ak || !jv) {
        free(dirs); free(smp); free(Ik); free(Ek); free(ak); free(jv);
        return -1;
    }
    oracle_fibonacci_dirs(num_rays, dirs);

    for (int s = 0; s < nsrc; ++s) {
        for (int r = ray_begin; r < ray_end; ++r) {
            ray_samples(&src[3 * s], &dirs[3 * r], ds, ns, geom_mode, kappa_mode, n0, n1, n2, smp);
            for (int b = 0; b < nf; ++b) {
                const double *jb = j + (long)b * ncell;
                const double *kb = kappa + (long)b * ncell;
                const double *Gb = G + (long)b * ncell;
                double *djb = dj + (long)b * ncell;
                double *dkb = dkappa + (long)b * ncell;
                /* forward sweep, Eq. 2, storing the state each reverse step needs */
                double I = 0.0, tau = 0.0;
                for (int k = 0; k < ns; ++k) {
                    const sample_t *q = &smp[k];
                    double jk = 0.0;
                    for (int c = 0; c < 8; ++c) jk += q->w[c] * jb[q->cell[c]];
                    double kk = kb[q->nn];
                    Ik[k] = I;
                    jv[k] = jk;
                    ak[k] = exp(-kk * dsr);
                    Ek[k] = exp(-tau);
                    I = I * ak[k] + jk * Ek[k] * dsr;
                    tau = tau + kk * dsr;
                }
                /* reverse sweep */
                double lam_next = 0.0;   /* lam_{k+2} */
                double a_next = 0.0;     /* a_{k+1}   */
                double mu = 0.0;         /* mu_{k+1}  */
                for (int k = ns - 1; k >= 0; --k) {
                    const sample_t *q = &smp[k];
                    double g = 0.0;
                    for (int c = 0; c < 8; ++c) g += q->w[c] * Gb[q->cell[c]];
                    g *= scale;
                    double lam = g + a_next * lam_next;                 /* lam_{k+1} */
                    double djk = lam * Ek[k] * dsr;
                    for (int c = 0; c < 8; ++c) djb[q->cell[c]] += djk * q->w[c];
                    dkb[q->nn] += -dsr * (lam * Ik[k] * ak[k] + mu);
                    mu = mu + lam * jv[k] * Ek[k] * dsr;                 /* mu_k */
                    lam_next = lam;
                    a_next = ak[k];
                }
            }
        }
    }
    free(dirs); free(smp); free(Ik); free(Ek); free(ak); free(jv);
    return 0;
}

/* ---- Per-ray record for the tests -----------------------------------------------------
 * For ray r of source src, bin 0 of the given maps: writes the base trilinear corner of each
 * substep (flat index of (i0, i0, i0), clamped), the kappa cell, and I_{k+1}. Any of the
 * output pointers may be NULL. */
int oracle_trace_ray(const double *j, const double *kappa, int n0, int n1, int n2,
                     const double src[3], int num_rays, int r, double ds, int ns,
                     int geom_mode, int kappa_mode, long *base_cell, long *nn_cell, double *I_out)
{
    if (r < 0 || r >= num_rays || ns < 0 || n0 < 1 || n1 < 1 || n2 < 1) return -1;
    if (ns == 0) return 0;
    double *dirs = (double *)malloc(sizeof(double) * 3 * (size_t)num_rays);
    sample_t *smp = (sample_t *)malloc(sizeof(sample_t) * (size_t)ns);
    if (!dirs || !smp) { free(dirs); free(smp); return -1; }
    oracle_fibonacci_dirs(num_rays, dirs);
    ray_samples(src, &dirs[3 * r], ds, ns, geom_mode, kappa_mode, n0, n1, n2, smp);
    const double dsr = geom_mode == 0 ? (double)(float)ds : ds;
    double I = 0.0, tau = 0.0;
    for (int k = 0; k < ns; ++k) {
        const sample_t *q = &smp[k];
        if (base_cell) base_cell[k] = q->cell[0];
        if (nn_cell) nn_cell[k] = q->nn;
        if (j && kappa && I_out) {
            double jk = 0.0;
            for (int c = 0; c < 8; ++c) jk += q->w[c] * j[q->cell[c]];
            double kk = kappa[q->nn];
            I = I * exp(-kk * dsr) + jk * exp(-tau) * dsr;
            tau += kk * dsr;
            I_out[k] = I;
        }
    }
    free(dirs);
    free(smp);
    return 0;
}

/* ---- Stateful advance: the march continued across calls (time integration with a fixed dt, Sec. 3) ----
 * Same march as oracle_advance, but each ray starts where the previous call left it: from the
 * position pos, with the intensity I and optical depth tau it had, and after ns substeps its new
 * position, I and tau are written back. With restart != 0 the input state is ignored and every
 * ray starts at its source with I = tau = 0 (oracle_advance exactly). j and kappa may change
 * between calls; each call deposits its own substeps. Consecutive calls therefore add up to one
 * call over the summed substeps.
 *   pos: [nsrc][num_rays][3] (in / out; with geom_mode 0 the positions are FP32 values)
 *   I, tau: [nf][nsrc][num_rays] (in / out)
 *   out: [nf][n0][n1][n2], ACCUMULATED.
 * Returns 0, or -1 on invalid arguments / allocation failure. */
int oracle_advance_state(const double *j, const double *kappa, int nf, int n0, int n1, int n2,
                         const double *src, int nsrc, int num_rays, double ds, int ns,
                         int geom_mode, int kappa_mode, int restart,
                         double *pos, double *I_state, double *tau_state, double *out)
{
    if (check_args(nf, n0, n1, n2, nsrc, num_rays, ds, ns, 0, num_rays)) return -1;
    if (!pos || !I_state || !tau_state) return -1;
    const long ncell = (long)n0 * n1 * n2;
    const long lanes = (long)nsrc * num_rays;
    const double scale = 4.0 * ORACLE_PI / (double)num_rays;
    const double dsr = geom_mode == 0 ? (double)(float)ds : ds;
    double *dirs = (double *)malloc(sizeof(double) * 3 * (size_t)num_rays);
    sample_t *smp = (sample_t *)malloc(sizeof(sample_t) * (size_t)(ns > 0 ? ns : 1));
    if (!dirs || !smp) { free(dirs); free(smp); return -1; }
    oracle_fibonacci_dirs(num_rays, dirs);

    for (int s = 0; s < nsrc; ++s) {
        for (int r = 0; r < num_rays; ++r) {
            const long lane = (long)s * num_rays + r;
            double *p = &pos[3 * lane];
            if (restart)
                for (int a = 0; a < 3; ++a) p[a] = src[3 * s + a];
            ray_samples(p, &dirs[3 * r], ds, ns, geom_mode, kappa_mode, n0, n1, n2, smp);
            for (int b = 0; b < nf; ++b) {
                const double *jb = j + (long)b * ncell;
                const double *kb = kappa + (long)b * ncell;
                double *ob = out + (long)b * ncell;
                double I = restart ? 0.0 : I_state[(long)b * lanes + lane];
                double tau = restart ? 0.0 : tau_state[(long)b * lanes + lane];
                for (int k = 0; k < ns; ++k) {
                    const sample_t *q = &smp[k];
                    double jk = 0.0;
                    for (int c = 0; c < 8; ++c) jk += q->w[c] * jb[q->cell[c]];
                    double kk = kb[q->nn];
                    I = I * exp(-kk * dsr) + jk * exp(-tau) * dsr;   /* Eq. 2, I update   */
                    tau = tau + kk * dsr;                             /* Eq. 2, tau update */
                    for (int c = 0; c < 8; ++c) ob[q->cell[c]] += scale * q->w[c] * I;
                }
                I_state[(long)b * lanes + lane] = I;
                tau_state[(long)b * lanes + lane] = tau;
            }
            /* the position after ns substeps, by the same additions ray_samples makes */
            if (geom_mode == 0) {
                const float ds32 = (float)ds;
                for (int a = 0; a < 3; ++a) {
                    const float d = (float)dirs[3 * r + a] * ds32;
                    float x = (float)p[a];
                    for (int k = 0; k < ns; ++k) x = x + d;
                    p[a] = (double)x;
                }
            } else {
                for (int a = 0; a < 3; ++a) {
                    const double d = dirs[3 * r + a] * ds;
                    double x = p[a];
                    for (int k = 0; k < ns; ++k) x = x + d;
                    p[a] = x;
                }
            }
        }
    }
    free(dirs);
    free(smp);
    return 0;
}

/* ---- Gradient with respect to the source positions ------------------------------------
 * Every position of a ray from source s is x_k = src_s + k n ds, so dL/dsrc_s is the sum over
 * the source's rays and substeps of dL/dx_k with everything else held fixed. x_k enters twice,
 * through trilinear weights: the deposit of I_{k+1} (scale w_c G[c] I_{k+1}) and the gather of
 * j (dL/dj_k = lam_{k+1} E_k ds, as in oracle_backward). With V_c = scale I_{k+1} G[c] +
 * lam_{k+1} E_k ds j[c] at the 8 corners,
 *     dL/dx_k,a = sum_c (dw_c / dt_a) V_c,   dw_c/dt_a = +-prod_{a' != a} (t or 1 - t),
 * + for the corners on the floor+1 side of axis a. The kappa cell is piecewise constant in x
 * and contributes nothing; on a clamped axis both corners are the same cell, so its terms
 * cancel. dsrc: [nsrc][3], ACCUMULATED. Returns 0, or -1 on invalid arguments. */
int oracle_source_gradient(const double *j, const double *kappa, int nf, int n0, int n1, int n2,
                           const double *src, int nsrc, int num_rays, double ds, int ns,
                           int geom_mode, int kappa_mode, const double *G, double *dsrc)
{
    if (check_args(nf, n0, n1, n2, nsrc, num_rays, ds, ns, 0, num_rays)) return -1;
    if (ns == 0 || nsrc == 0) return 0;
    const long ncell = (long)n0 * n1 * n2;
    const double scale = 4.0 * ORACLE_PI / (double)num_rays;
    const double dsr = geom_mode == 0 ? (double)(float)ds : ds;
    double *dirs = (double *)malloc(sizeof(double) * 3 * (size_t)num_rays);
    sample_t *smp = (sample_t *)malloc(sizeof(sample_t) * (size_t)ns);
    double *Ik = (double *)malloc(sizeof(double) * (size_t)(ns + 1));   /* I_0 .. I_ns */
    double *Ek = (double *)malloc(sizeof(double) * (size_t)ns);
    double *ak = (double *)malloc(sizeof(double) * (size_t)ns);
    if (!dirs || !smp || !Ik || !Ek || !ak) {
        free(dirs); free(smp); free(Ik); free(Ek); free(ak);
        return -1;
    }
    oracle_fibonacci_dirs(num_rays, dirs);
    for (int s = 0; s < nsrc; ++s) {
        for (int r = 0; r < num_rays; ++r) {
            ray_samples(&src[3 * s], &dirs[3 * r], ds, ns, geom_mode, kappa_mode, n0, n1, n2, smp);
            for (int b = 0; b < nf; ++b) {
                const double *jb = j + (long)b * ncell;
                const double *kb = kappa + (long)b * ncell;
                const double *Gb = G + (long)b * ncell;
                double tau = 0.0;
                Ik[0] = 0.0;
                for (int k = 0; k < ns; ++k) {
                    const sample_t *q = &smp[k];
                    double jk = 0.0;
                    for (int c = 0; c < 8; ++c) jk += q->w[c] * jb[q->cell[c]];
                    double kk = kb[q->nn];
                    ak[k] = exp(-kk * dsr);
                    Ek[k] = exp(-tau);
                    Ik[k + 1] = Ik[k] * ak[k] + jk * Ek[k] * dsr;      /* Eq. 2 */
                    tau = tau + kk * dsr;
                }
                double lam_next = 0.0, a_next = 0.0;
                for (int k = ns - 1; k >= 0; --k) {
                    const sample_t *q = &smp[k];
                    double g = 0.0;
                    for (int c = 0; c < 8; ++c) g += q->w[c] * Gb[q->cell[c]];
                    const double lam = scale * g + a_next * lam_next;   /* lam_{k+1} */
                    for (int a = 0; a < 3; ++a) {
                        double d = 0.0;
                        for (int c = 0; c < 8; ++c) {
                            double dw = 1.0;
                            for (int e = 0; e < 3; ++e) {
                                const int bit = (c >> (2 - e)) & 1;
                                if (e == a) dw *= bit ? 1.0 : -1.0;
                                else dw *= bit ? q->t[e] : 1.0 - q->t[e];
                            }
                            const double V = scale * Ik[k + 1] * Gb[q->cell[c]] + lam * Ek[k] * dsr * jb[q->cell[c]];
                            d += dw * V;
                        }
                        dsrc[3 * s + a] += d;
                    }
                    lam_next = lam;
                    a_next = ak[k];
                }
            }
        }
    }
    free(dirs); free(smp); free(Ik); free(Ek); free(ak);
    return 0;
}
