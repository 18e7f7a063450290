/*
 * md_oracle.c -- plain, slow, FP64 CPU oracle for the molecular-dynamics step
 * of Colberg & Hoefling, "Highly accelerated simulations of glassy dynamics
 * using GPUs: caveats on limited floating-point precision" (arXiv:0912.3824).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA library
 * is checked against.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA path and includes none of its files.
 *
 * Everything is IEEE double, evaluated one operation at a time: the build
 * passes -ffp-contract=off so that no multiply-add is fused and the results
 * are identical on x86_64 and aarch64 hosts.
 *
 * What is computed, and where the paper defines it:
 *   - the 12-6 Lennard-Jones pair potential V(r) = 4 eps [(r/sig)^-12 - (r/sig)^-6]
 *     cut at r_c (Sec. 3, performance measurements), optionally shifted so that
 *     V(r_c) = 0; the Kob-Andersen A/B parameter table (Sec. 5); optionally
 *     multiplied by the smoothing function g((r - r_c) / (h sigma)),
 *     g(x) = x^4 / (1 + x^4), of Sec. 4 (purely repulsive WCA is the shifted
 *     potential cut at its minimum, r_c = 2^(1/6) sigma, also Sec. 4);
 *   - the force on each particle as the plain sum over all partners within the
 *     cutoff (Sec. 2.2: neighbour lists and cells only make that sum cheaper,
 *     they do not change it) -- once by brute force over all pairs and once by
 *     an independently written cell list;
 *   - the velocity-Verlet integrator (Sec. 2.2) with periodic wrapping and
 *     image counters;
 *   - the per-step reductions named in Sec. 2.2: potential energy, kinetic
 *     energy (temperature), centre-of-mass momentum and the virial tensor.
 *
 * Geometry: cubic periodic box of edge L, positions kept in [0, L), minimum
 * image  d - L * rint(d / L)  (rint rounds half to even).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Pair-potential description.  Index [a*2+b] for species a, b in {0, 1}. */
typedef struct {
    int n_species;       /* 1 (monatomic LJ) or 2 (binary mixture)          */
    int shift;           /* 1: truncated and shifted, 0: truncated only     */
    double eps[4];       /* epsilon_ab                                      */
    double sigma[4];     /* sigma_ab                                        */
    double rcut[4];      /* absolute cutoff radius r_c,ab                   */
    double mass[2];      /* particle mass per species                       */
    double smooth_h;     /* h of the smoothing function (Sec. 4); 0 = none  */
} orc_pot;

/* Per-step observables recorded by orc_vv_run. */
typedef struct {
    long long step;
    double e_pot;        /* sum_{i<j} V(r_ij)                                */
    double e_kin;        /* sum_i m_i v_i^2 / 2                              */
    double virial;       /* sum_{i<j} r_ij . F_ij                            */
    double w[6];         /* virial tensor xx, yy, zz, xy, xz, yz             */
    double p[3];         /* total momentum sum_i m_i v_i                     */
} orc_obs;

/* ------------------------------------------------------------------------ */
/* Pair potential (Sec. 3 definition of V_LJ; Sec. 5 KA parameters).        */
/* ------------------------------------------------------------------------ */

/* Unshifted 12-6 potential at squared distance r2. */
static double lj_raw(double eps, double sig, double r2)
{
    double sr2 = (sig * sig) / r2;
    double sr6 = sr2 * sr2 * sr2;
    return 4.0 * eps * (sr6 * sr6 - sr6);
}

/*
 * Potential and force factor for one pair of species (a, b) at squared
 * separation r2.  Returns 1 if r < r_c,ab (strict), else 0 and zeros.
 * *v  = V_ab(r) - S_ab, with S_ab = V_ab(r_c) when shifting, else 0;
 * *fr = -V'(r) / r, so that the force on i from j is  fr * (r_i - r_j).
 *   -V'(r)/r = 48 eps / r^2 * [(sig/r)^12 - (sig/r)^6 / 2]
 * With smoothing (h > 0, Sec. 4) the potential is U(r) = V(r) g(x) with
 * x = (r - r_c) / (h sigma_ab) and g(x) = x^4 / (1 + x^4), so that
 *   *v  = V g
 *   *fr = -U'(r) / r = (-V'(r)/r) g - V g'(x) / (h sigma_ab r),
 *   g'(x) = 4 x^3 / (1 + x^4)^2.
 */
int orc_pair(const orc_pot *p, int a, int b, double r2, double *v, double *fr)
{
    int ab = a * 2 + b;
    double eps = p->eps[ab], sig = p->sigma[ab], rc = p->rcut[ab];
    *v = 0.0;
    *fr = 0.0;
    if (!(r2 < rc * rc))
        return 0;
    double sr2 = (sig * sig) / r2;
    double sr6 = sr2 * sr2 * sr2;
    double shift = p->shift ? lj_raw(eps, sig, rc * rc) : 0.0;
    *v = 4.0 * eps * (sr6 * sr6 - sr6) - shift;
    *fr = 48.0 * eps / r2 * (sr6 * sr6 - 0.5 * sr6);
    if (p->smooth_h > 0.0) {
        double hs = p->smooth_h * sig;
        double r = sqrt(r2);
        double x = (r - rc) / hs;
        double x4 = x * x * x * x;
        double g = x4 / (1.0 + x4);
        double dg = 4.0 * x * x * x / ((1.0 + x4) * (1.0 + x4));
        *fr = *fr * g - *v * dg / (hs * r);
        *v = *v * g;
    }
    return 1;
}

/* Minimum-image component of the separation d = x_i - x_j. */
static double min_image(double d, double L)
{
    return d - L * rint(d / L);
}

/* Accumulate one pair (i<j) into the outputs.  dx is r_i - r_j (minimum image). */
static void add_pair(const orc_pot *p, const int *type, long i, long j,
                     const double dx[3], double *f, double *e, double *w7)
{
    double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    double v, fr;
    if (!orc_pair(p, type[i], type[j], r2, &v, &fr))
        return;
    for (int k = 0; k < 3; ++k) {
        f[3 * i + k] += fr * dx[k];
        f[3 * j + k] -= fr * dx[k];
    }
    e[i] += 0.5 * v;
    e[j] += 0.5 * v;
    /* w7: [0] scalar virial, [1..6] tensor xx yy zz xy xz yz */
    w7[0] += fr * r2;
    w7[1] += fr * dx[0] * dx[0];
    w7[2] += fr * dx[1] * dx[1];
    w7[3] += fr * dx[2] * dx[2];
    w7[4] += fr * dx[0] * dx[1];
    w7[5] += fr * dx[0] * dx[2];
    w7[6] += fr * dx[1] * dx[2];
}

/*
 * Brute force O(N^2): every unordered pair once, minimum image.
 * f[n][3], e[n] (half of each pair energy to each partner), w7[7].
 * Requires L > 2 r_c,max so that at most one image of a pair is in range.
 */
void orc_forces_brute(const orc_pot *p, long n, double L, const int *type,
                      const double *pos, double *f, double *e, double *w7)
{
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    memset(e, 0, sizeof(double) * (size_t)n);
    memset(w7, 0, sizeof(double) * 7);
    for (long i = 0; i < n; ++i) {
        for (long j = i + 1; j < n; ++j) {
            double dx[3];
            for (int k = 0; k < 3; ++k)
                dx[k] = min_image(pos[3 * i + k] - pos[3 * j + k], L);
            add_pair(p, type, i, j, dx, f, e, w7);
        }
    }
}

/*
 * Force f3[3] and energy share *e (half of each pair energy) on the single
 * particle i, summed over every other particle by brute force.  Used to
 * check large systems on a sample of particles.
 */
void orc_force_one(const orc_pot *p, long n, double L, const int *type,
                   const double *pos, long i, double *f3, double *e)
{
    double fx = 0.0, fy = 0.0, fz = 0.0, ei = 0.0;
    for (long j = 0; j < n; ++j) {
        if (j == i)
            continue;
        double dx = min_image(pos[3 * i + 0] - pos[3 * j + 0], L);
        double dy = min_image(pos[3 * i + 1] - pos[3 * j + 1], L);
        double dz = min_image(pos[3 * i + 2] - pos[3 * j + 2], L);
        double v, fr;
        if (orc_pair(p, type[i], type[j], dx * dx + dy * dy + dz * dz, &v, &fr)) {
            fx += fr * dx;
            fy += fr * dy;
            fz += fr * dz;
            ei += 0.5 * v;
        }
    }
    f3[0] = fx;
    f3[1] = fy;
    f3[2] = fz;
    *e = ei;
}

/*
 * Cell-list version, written independently of the brute-force loop:
 * textbook linked cells (head / next arrays), cell edge >= r_c,max,
 * each unordered pair visited once by only taking partners j > i.
 * Along an axis with fewer than 3 cells the distinct neighbour cells are
 * deduplicated so that no pair is visited twice.
 */
void orc_forces_cells(const orc_pot *p, long n, double L, const int *type,
                      const double *pos, double *f, double *e, double *w7)
{
    double rmax = 0.0;
    int ns = p->n_species;
    for (int a = 0; a < ns; ++a)
        for (int b = 0; b < ns; ++b)
            if (p->rcut[a * 2 + b] > rmax)
                rmax = p->rcut[a * 2 + b];
    /* a 1e-9 relative margin keeps rounding in the binning below from
       placing two particles closer than r_c,max two cells apart */
    int nc = (int)floor(L / (rmax * (1.0 + 1e-9)));
    if (nc < 1)
        nc = 1;
    long ncell = (long)nc * nc * nc;
    long *head = (long *)malloc(sizeof(long) * (size_t)ncell);
    long *next = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    for (long c = 0; c < ncell; ++c)
        head[c] = -1;
    for (long i = n - 1; i >= 0; --i) {
        int c3[3];
        for (int k = 0; k < 3; ++k) {
            int c = (int)floor(pos[3 * i + k] / L * nc);
            if (c < 0) c = 0;
            if (c >= nc) c = nc - 1;
            c3[k] = c;
        }
        long c = ((long)c3[2] * nc + c3[1]) * nc + c3[0];
        next[i] = head[c];
        head[c] = i;
    }
    /* distinct neighbour offsets along one axis */
    int offs[3], noff;
    if (nc >= 3) { offs[0] = -1; offs[1] = 0; offs[2] = 1; noff = 3; }
    else if (nc == 2) { offs[0] = 0; offs[1] = 1; noff = 2; }
    else { offs[0] = 0; noff = 1; }

    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    memset(e, 0, sizeof(double) * (size_t)n);
    memset(w7, 0, sizeof(double) * 7);
    for (int cz = 0; cz < nc; ++cz)
    for (int cy = 0; cy < nc; ++cy)
    for (int cx = 0; cx < nc; ++cx) {
        long c = ((long)cz * nc + cy) * nc + cx;
        for (int oz = 0; oz < noff; ++oz)
        for (int oy = 0; oy < noff; ++oy)
        for (int ox = 0; ox < noff; ++ox) {
            int nx = (cx + offs[ox] + nc) % nc;
            int ny = (cy + offs[oy] + nc) % nc;
            int nz = (cz + offs[oz] + nc) % nc;
            long d = ((long)nz * nc + ny) * nc + nx;
            for (long i = head[c]; i >= 0; i = next[i])
                for (long j = head[d]; j >= 0; j = next[j]) {
                    if (j <= i)
                        continue;
                    double dx[3];
                    for (int k = 0; k < 3; ++k)
                        dx[k] = min_image(pos[3 * i + k] - pos[3 * j + k], L);
                    add_pair(p, type, i, j, dx, f, e, w7);
                }
        }
    }
    free(head);
    free(next);
}

/* Kinetic energy and total momentum (Sec. 2.2 reductions). */
void orc_kinetic(const orc_pot *p, long n, const int *type, const double *vel,
                 double *e_kin, double *mom)
{
    double ek = 0.0, px = 0.0, py = 0.0, pz = 0.0;
    for (long i = 0; i < n; ++i) {
        double m = p->mass[type[i]];
        const double *v = vel + 3 * i;
        ek += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        px += m * v[0];
        py += m * v[1];
        pz += m * v[2];
    }
    *e_kin = ek;
    mom[0] = px; mom[1] = py; mom[2] = pz;
}

static void record(const orc_pot *p, long n, const int *type, const double *vel,
                   const double *e, const double *w7, long long step, orc_obs *o)
{
    double ep = 0.0;
    for (long i = 0; i < n; ++i)
        ep += e[i];
    o->step = step;
    o->e_pot = ep;
    orc_kinetic(p, n, type, vel, &o->e_kin, o->p);
    o->virial = w7[0];
    for (int k = 0; k < 6; ++k)
        o->w[k] = w7[1 + k];
}

/* Wrap one coordinate into [0, L) and count the image crossing. */
static void wrap(double *x, int *img, double L)
{
    if (*x >= L) { *x -= L; *img += 1; }
    else if (*x < 0.0) { *x += L; *img -= 1; }
}

/*
 * Velocity-Verlet (Sec. 2.2), NVE, one force evaluation per step:
 *   v += dt/(2m) F(r);  r += dt v;  wrap;  F = F(r);  v += dt/(2m) F(r)
 * Forces come from orc_forces_cells.  f[n][3] receives F(r) of the final
 * positions.  obs (may be NULL) receives the state at
 * steps 0, sample, 2*sample, ... including step 0 before any move; returns
 * the number of records written (at most max_obs).
 */
long orc_vv_run(const orc_pot *p, long n, double L, const int *type,
                double *pos, double *vel, int *image, double *f, double dt, long long nsteps, long long sample,
                orc_obs *obs, long max_obs)
{
    double *e = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double w7[7];
    long nrec = 0;
    orc_forces_cells(p, n, L, type, pos, f, e, w7);
    if (obs && sample > 0 && nrec < max_obs)
        record(p, n, type, vel, e, w7, 0, &obs[nrec++]);
    for (long long s = 1; s <= nsteps; ++s) {
        for (long i = 0; i < n; ++i) {
            double h = 0.5 * dt / p->mass[type[i]];
            for (int k = 0; k < 3; ++k) {
                vel[3 * i + k] += h * f[3 * i + k];
                pos[3 * i + k] += dt * vel[3 * i + k];
                wrap(&pos[3 * i + k], &image[3 * i + k], L);
            }
        }
        orc_forces_cells(p, n, L, type, pos, f, e, w7);
        for (long i = 0; i < n; ++i) {
            double h = 0.5 * dt / p->mass[type[i]];
            for (int k = 0; k < 3; ++k)
                vel[3 * i + k] += h * f[3 * i + k];
        }
        if (obs && sample > 0 && s % sample == 0 && nrec < max_obs)
            record(p, n, type, vel, e, w7, s, &obs[nrec++]);
    }
    free(e);
    return nrec;
}

/*
 * Velocity rescaling to a target temperature (Sec. 2.3: assigned velocities
 * are rescaled to match the heat-bath temperature exactly), with
 * T = 2 E_kin / (3N - 3) since the total momentum is zero.
 */
void orc_rescale(const orc_pot *p, long n, const int *type, double *vel, double T)
{
    double ek, mom[3];
    orc_kinetic(p, n, type, vel, &ek, mom);
    double t_inst = 2.0 * ek / (3.0 * (double)n - 3.0);
    double s = sqrt(T / t_inst);
    for (long i = 0; i < 3 * n; ++i)
        vel[i] *= s;
}

/*
 * All pairs (i, j), i != j, with minimum-image distance below the list
 * radius r_c,ab + skin, by brute force.  Writes counts[n]; if lists is not
 * NULL it must hold n*kmax entries and receives partner ids in increasing j.
 * Returns the largest count.  Used to check the neighbour-list invariant.
 */
long orc_neighbours_brute(const orc_pot *p, long n, double L, const int *type,
                          const double *pos, double skin, int *counts,
                          int *lists, long kmax)
{
    long maxc = 0;
    for (long i = 0; i < n; ++i) {
        long c = 0;
        for (long j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double r2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                double d = min_image(pos[3 * i + k] - pos[3 * j + k], L);
                r2 += d * d;
            }
            double rl = p->rcut[type[i] * 2 + type[j]] + skin;
            if (r2 < rl * rl) {
                if (lists && c < kmax)
                    lists[i * kmax + c] = (int)j;
                ++c;
            }
        }
        counts[i] = (int)c;
        if (c > maxc)
            maxc = c;
    }
    return maxc;
}

/* ------------------------------------------------------------------------ */
/* The rand48 generator and the Andersen heat bath (Sec. 2.3).              */
/*                                                                          */
/* rand48: x_{n+1} = (a x_n + c) mod 2^48 with a = 0x5DEECE66D, c = 0xB (the */
/* POSIX drand48 family); seeding as srand48: x_0 = (seed mod 2^32) 2^16 +  */
/* 0x330E; deviate n (n = 0, 1, ...) is d_n = x_{n+1} / 2^48, the value of  */
/* the (n+1)-th drand48 call.  With T threads, thread t produces the        */
/* deviates t, t + T, t + 2T, ... of this one sequence by the leapfrog      */
/* x_{n+T} = A_T x_n + C_T, A_T = a^T, C_T = c sum_{n<T} a^n (mod 2^48).    */
/* ------------------------------------------------------------------------ */
#define R48_MASK 0xFFFFFFFFFFFFULL
static const unsigned long long R48_A = 0x5DEECE66DULL, R48_C = 0xBULL;

unsigned long long orc_rand48_seed(unsigned long long seed)
{
    return ((seed & 0xFFFFFFFFULL) << 16) | 0x330EULL;
}

/* n steps of the recurrence, one at a time */
unsigned long long orc_rand48_step(unsigned long long x, long long n)
{
    for (long long k = 0; k < n; ++k)
        x = (R48_A * x + R48_C) & R48_MASK;
    return x;
}

/* leapfrog multiplier and addend for T threads, from their definitions */
void orc_rand48_leapfrog(long long T, unsigned long long *A, unsigned long long *C)
{
    unsigned long long pw = 1, sum = 0;          /* a^n and sum_{m<n} a^m */
    for (long long n = 0; n < T; ++n) {
        sum = (sum + pw) & R48_MASK;
        pw = (pw * R48_A) & R48_MASK;
    }
    *A = pw;
    *C = (R48_C * sum) & R48_MASK;
}

/* count deviates d_first .. d_{first+count-1} of the sequence from seed */
void orc_rand48_uniforms(unsigned long long seed, long long first, long long count, double *u)
{
    unsigned long long x = orc_rand48_step(orc_rand48_seed(seed), first + 1);
    for (long long k = 0; k < count; ++k) {
        u[k] = (double)x / 281474976710656.0;    /* 2^48 */
        x = (R48_A * x + R48_C) & R48_MASK;
    }
}

/*
 * One Andersen heat-bath collision of every particle (Sec. 2.3): fresh
 * Maxwell-Boltzmann velocities at temperature T, then the mass-weighted mean
 * velocity is removed and the set rescaled so that 2 E_kin / (3N - 3) = T
 * exactly.  Particle i (original index) is thread i of a leapfrog over
 * nthreads threads; collision `event` uses its draws 4 event .. 4 event + 3,
 * i.e. the sequence elements (4 event + k) nthreads + i.  Box-Muller:
 *   v_x = s sqrt(-2 ln(1 - u0)) cos(2 pi u1),  v_y = ... sin(2 pi u1),
 *   v_z = s sqrt(-2 ln(1 - u2)) cos(2 pi u3),  s = sqrt(T / m_i).
 * The sequence is generated one element at a time (no jump-ahead).
 */
void orc_andersen(const orc_pot *p, long n, const int *type, double *vel, double T,
                  unsigned long long seed, long long event, long long nthreads, long long first_index)
{
    long long span = 4 * nthreads;
    double *u = (double *)malloc(sizeof(double) * (size_t)span);
    orc_rand48_uniforms(seed, 4 * event * nthreads, span, u);
    const double two_pi = 6.283185307179586476925286766559;
    for (long i = 0; i < n; ++i) {
        long long t = first_index + i;
        double u0 = u[0 * nthreads + t], u1 = u[1 * nthreads + t];
        double u2 = u[2 * nthreads + t], u3 = u[3 * nthreads + t];
        double r1 = sqrt(-2.0 * log(1.0 - u0)), r2 = sqrt(-2.0 * log(1.0 - u2));
        double s = sqrt(T / p->mass[type[i]]);
        vel[3 * i + 0] = s * r1 * cos(two_pi * u1);
        vel[3 * i + 1] = s * r1 * sin(two_pi * u1);
        vel[3 * i + 2] = s * r2 * cos(two_pi * u3);
    }
    free(u);
    double mtot = 0.0, mom[3] = {0.0, 0.0, 0.0};
    for (long i = 0; i < n; ++i) {
        double m = p->mass[type[i]];
        mtot += m;
        for (int k = 0; k < 3; ++k)
            mom[k] += m * vel[3 * i + k];
    }
    for (long i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k)
            vel[3 * i + k] -= mom[k] / mtot;
    if (n > 1 && T > 0.0)
        orc_rescale(p, n, type, vel, T);
    else
        for (long i = 0; i < 3 * n; ++i)
            vel[i] = 0.0;
}
