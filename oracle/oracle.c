/*
 * CPU oracle (plain C11 + OpenMP, binary64, history-based).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product library.
 *
 * Built with -ffp-contract=off: every expression below is evaluated as
 * written, one IEEE-754 round-to-nearest operation at a time, so that the
 * GPU path (compiled without FMA contraction) can reproduce each particle's
 * random walk bit for bit.  Parenthesised sub-expressions fix the operation
 * order wherever the grouping is not obvious.  Where a step is written as
 * fma(a, b, c) it is the IEEE-754 fused multiply-add a * b + c with one
 * rounding (C99 fma; the GPU path issues the same operation): the binary64
 * lookup's interpolation and its density-weighted sums, the logarithm's
 * series, the position update, the cylinder's quadratic and the scatter
 * kinematics.
 *
 * What is computed (paper: Sec. 2 "Event-Based Parallelism" for the event /
 * history duality; Sec. 2 "Sorting" for the macroscopic cross-section lookup
 * being the dominant kernel; Sec. 2 "Tallying" for the active-batch tallies;
 * Sec. 3 for surface (ray) tracking with delta tracking disabled).  The
 * paper prints no transport formulas; the standard textbook ones are used and
 * every reading is listed in the design notes of the repository.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Round: two 64x64->128 products of the even    */
/* counter words with the round multipliers; the high halves are xored with  */
/* the odd words and the key; the key is bumped by the Weyl constants        */
/* between rounds.                                                           */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL /* golden ratio */
#define PHILOX_W1 0xBB67AE8584CAA73BULL /* sqrt(3) - 1 */

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 64 random bits -> (0, 1]: the top 53 bits plus one, times 2^-53. */
double or_u01(uint64_t x)
{
    return (double)((x >> 11) + 1) * 0x1.0p-53;
}

/* Per-particle stream: key (seed, problem<<32 | batch), counter
 * (particle id, block, 0, 0); variate j is word j%4 of block j/4. */
typedef struct {
    uint64_t key[2];
    uint64_t id;
    uint32_t j;
    uint64_t cached_block;
    int have;
    uint64_t buf[4];
} rng_t;

static void rng_init(rng_t *r, uint64_t seed, uint64_t key_hi, uint64_t id)
{
    r->key[0] = seed;
    r->key[1] = key_hi;
    r->id = id;
    r->j = 0;
    r->have = 0;
    r->cached_block = 0;
}

static double rng_next(rng_t *r)
{
    uint64_t block = r->j >> 2;
    if (!r->have || block != r->cached_block) {
        uint64_t ctr[4] = {r->id, block, 0, 0};
        or_philox4x64_10(ctr, r->key, r->buf);
        r->cached_block = block;
        r->have = 1;
    }
    double u = or_u01(r->buf[r->j & 3]);
    r->j += 1;
    return u;
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm, written for reproducibility: x = 2^e m with           */
/* m in (sqrt(2)/2, sqrt(2)], log m = 2 atanh(s), s = (m-1)/(m+1), summed as */
/* the series 2s(1 + s^2/3 + s^4/5 + ... + s^20/21) (Abramowitz & Stegun     */
/* 4.1.28); e ln2 uses a two-part ln2 whose high part has 21 trailing zero   */
/* bits, so e*LN2_HI is exact.  Coefficients are 1/(2k+1) rounded to        */
/* nearest.  Valid for positive normal x.                                    */
/* ------------------------------------------------------------------------ */
#define OR_LN2_HI 0x1.62e42fee00000p-1
#define OR_LN2_LO 0x1.a39ef35793c76p-33
#define OR_SQRT2 0x1.6a09e667f3bcdp+0

double or_log(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    uint64_t mb = (b & 0x000FFFFFFFFFFFFFULL) | 0x3FF0000000000000ULL;
    double m;
    memcpy(&m, &mb, 8);
    if (m > OR_SQRT2) {
        m = m * 0.5;
        e = e + 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    /* Horner's rule, each step c_k + z q rounded once */
    double q = 0x1.8618618618618p-5;            /* 1/21 */
    q = fma(z, q, 0x1.af286bca1af28p-5);        /* 1/19 */
    q = fma(z, q, 0x1.e1e1e1e1e1e1ep-5);        /* 1/17 */
    q = fma(z, q, 0x1.1111111111111p-4);        /* 1/15 */
    q = fma(z, q, 0x1.3b13b13b13b14p-4);        /* 1/13 */
    q = fma(z, q, 0x1.745d1745d1746p-4);        /* 1/11 */
    q = fma(z, q, 0x1.c71c71c71c71cp-4);        /* 1/9 */
    q = fma(z, q, 0x1.2492492492492p-3);        /* 1/7 */
    q = fma(z, q, 0x1.999999999999ap-3);        /* 1/5 */
    q = fma(z, q, 0x1.5555555555555p-2);        /* 1/3 */
    q = z * q;
    double t = 2.0 * s;
    double logm = fma(t, q, t);                 /* 2s + 2s q */
    double de = (double)e;
    return fma(de, OR_LN2_HI, fma(de, OR_LN2_LO, logm));
}

/* ------------------------------------------------------------------------ */
/* Cross-section lookup (Sec. 2 "Sorting": the lookup is the most expensive */
/* kernel).  Micro: binary search of the nuclide's grid, lin-lin           */
/* interpolation.  Macro: density-weighted sum over the material's nuclides */
/* in their listed order.                                                   */
/* ------------------------------------------------------------------------ */

/* Largest j in [0, n-2] with g[j] <= E (j = 0 when E < g[0]). */
int64_t or_search(const double *g, int64_t n, double E)
{
    int64_t lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g[mid] <= E)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

/* Binary32 tables: the same bracket, the largest j in [0, n-2] with
 * (double)g[j] <= E.  Widening a binary32 value to binary64 is exact, so the
 * comparison is exact: E itself is never rounded for the search. */
int64_t or_search_f32(const float *g, int64_t n, double E)
{
    int64_t lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((double)g[mid] <= E)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

typedef struct {
    const or_problem *P;
    float *ef;   /* binary32 copies (precision 1) */
    float *sf;
} tables_t;

double or_micro(const or_problem *P, int32_t nuc, double E)
{
    int64_t lo = P->grid_off[nuc];
    int64_t n = P->grid_off[nuc + 1] - lo;
    const double *g = P->energy + lo;
    const double *s = P->sigma_t + lo;
    int64_t j = or_search(g, n, E);
    double f = (E - g[j]) / (g[j + 1] - g[j]);
    /* sigma_j + f (sigma_j+1 - sigma_j), the product and sum rounded once */
    return fma(f, s[j + 1] - s[j], s[j]);
}

/* Binary32 micro cross section on one nuclide's binary32 grid g and values
 * s (n points): the bracket of E as above, then the lin-lin interpolation
 * with every operation in binary32 on E rounded to nearest binary32. */
float or_micro_f32(const float *g, const float *s, int64_t n, double E)
{
    int64_t j = or_search_f32(g, n, E);
    float Ef = (float)E;
    float f = (Ef - g[j]) / (g[j + 1] - g[j]);
    return s[j] + f * (s[j + 1] - s[j]);
}

static float micro_f32(const tables_t *T, int32_t nuc, double E)
{
    const or_problem *P = T->P;
    int64_t lo = P->grid_off[nuc];
    int64_t n = P->grid_off[nuc + 1] - lo;
    return or_micro_f32(T->ef + lo, T->sf + lo, n, E);
}

/* The tables of problem P as the lookup reads them: binary32 copies (each
 * grid energy and cross section rounded to nearest) in precision 1. */
static int tables_init(tables_t *T, const or_problem *P)
{
    T->P = P;
    T->ef = NULL;
    T->sf = NULL;
    if (P->precision == 1) {
        int64_t tot = P->grid_off[P->n_nuc];
        T->ef = (float *)malloc(sizeof(float) * (size_t)(tot > 0 ? tot : 1));
        T->sf = (float *)malloc(sizeof(float) * (size_t)(tot > 0 ? tot : 1));
        if (!T->ef || !T->sf) {
            free(T->ef);
            free(T->sf);
            return -1;
        }
        for (int64_t k = 0; k < tot; ++k) {
            T->ef[k] = (float)P->energy[k];
            T->sf[k] = (float)P->sigma_t[k];
        }
    }
    return 0;
}

static void tables_free(tables_t *T)
{
    free(T->ef);
    free(T->sf);
    T->ef = NULL;
    T->sf = NULL;
}

/* Macroscopic sigma_t and sigma_a of material m at energy E.  Binary64:
 * Sigma_t = sum of N_i sigma_i and Sigma_a = sum of (N_i f_i) sigma_i in the
 * listed order, each term added by one fused multiply-add (N_i f_i is
 * rounded first).  Binary32: product, then sum, each rounded in binary32. */
static void macro_xs(const tables_t *T, int32_t m, double E, double *st, double *sa)
{
    const or_problem *P = T->P;
    if (P->precision == 0) {
        double at = 0.0, aa = 0.0;
        for (int32_t q = P->mat_off[m]; q < P->mat_off[m + 1]; ++q) {
            int32_t i = P->nuc_id[q];
            double N = P->density[q];
            double sig = or_micro(P, i, E);
            at = fma(N, sig, at);
            aa = fma(N * P->f_abs[i], sig, aa);
        }
        *st = at;
        *sa = aa;
    } else {
        float at = 0.0f, aa = 0.0f;
        for (int32_t q = P->mat_off[m]; q < P->mat_off[m + 1]; ++q) {
            int32_t i = P->nuc_id[q];
            float t = (float)P->density[q] * micro_f32(T, i, E);
            at = at + t;
            aa = aa + t * (float)P->f_abs[i];
        }
        *st = (double)at;
        *sa = (double)aa;
    }
}

/* exported for tests: macroscopic lookup with the problem's precision */
int or_macro(const or_problem *P, int32_t m, const double *E, int64_t n,
             double *st, double *sa)
{
    tables_t T;
    if (tables_init(&T, P)) return -1;
    for (int64_t k = 0; k < n; ++k) macro_xs(&T, m, E[k], &st[k], &sa[k]);
    tables_free(&T);
    return 0;
}

/* Collision nuclide: first i (listed order) whose running sum of N_i sigma_i
 * exceeds target = xi * Sigma_t; the running sums are formed exactly as in
 * macro_xs.  If rounding leaves none, the last nuclide with a positive term
 * (binary64: N_i > 0 and sigma_i > 0; binary32: the rounded product) --
 * the first listed nuclide if no term is positive. */
static int32_t pick_nuclide(const tables_t *T, int32_t m, double E, double target)
{
    const or_problem *P = T->P;
    int32_t last = -1;
    if (P->precision == 0) {
        double cum = 0.0;
        for (int32_t q = P->mat_off[m]; q < P->mat_off[m + 1]; ++q) {
            int32_t i = P->nuc_id[q];
            double N = P->density[q];
            double sig = or_micro(P, i, E);
            cum = fma(N, sig, cum);
            if (N > 0.0 && sig > 0.0) last = i;
            if (target < cum) return i;
        }
    } else {
        float cum = 0.0f;
        for (int32_t q = P->mat_off[m]; q < P->mat_off[m + 1]; ++q) {
            int32_t i = P->nuc_id[q];
            float t = (float)P->density[q] * micro_f32(T, i, E);
            cum = cum + t;
            if (t > 0.0f) last = i;
            if (target < (double)cum) return i;
        }
    }
    return last >= 0 ? last : P->nuc_id[P->mat_off[m]];
}

/* exported for tests: the collision nuclide of material m at energy E for
 * target = xi Sigma_t, in the problem's precision; -1 if the tables cannot
 * be built */
int32_t or_pick_nuclide(const or_problem *P, int32_t m, double E, double target)
{
    tables_t T;
    if (tables_init(&T, P)) return -1;
    int32_t i = pick_nuclide(&T, m, E, target);
    tables_free(&T);
    return i;
}

/* ------------------------------------------------------------------------ */
/* Geometry: distance to the nearest surface of the current cell.           */
/* ------------------------------------------------------------------------ */
#define SURF_NONE 0
#define SURF_CYL 1
#define SURF_X 2
#define SURF_Y 3
#define SURF_Z 4

typedef struct {
    double x, y, z, u, v, w, E, wgt;
    double st, sa;
    int32_t i, j;     /* lattice cell / slab layer (i) */
    int32_t inside;   /* inside the pin cylinder */
    int32_t mat;
    int32_t n_coll, n_flights;
    int32_t status;
} particle_t;

/* Distance along (u,v) from (dx,dy) (relative to the axis) to the cylinder
 * of radius r; `inside` selects the far (exit) root, otherwise the near
 * (entry) root.  Quadratic a d^2 + 2 k d + c = 0 in its stable forms. */
double or_dist_cylinder(double dx, double dy, double u, double v, double r, int inside)
{
    /* a = u^2 + v^2, k = dx u + dy v, c = dx^2 + dy^2 - r^2, D = k^2 - a c,
     * each product-plus-term one fused multiply-add */
    double a = fma(u, u, v * v);
    double k = fma(dx, u, dy * v);
    double c = fma(dx, dx, dy * dy) - r * r;
    double D = fma(k, k, -(a * c));
    if (inside) {
        if (a == 0.0) return INFINITY;
        if (D < 0.0) D = 0.0;
        double sD = sqrt(D);
        if (k <= 0.0) return (sD - k) / a;
        return (0.0 - c) / (k + sD);
    }
    if (a == 0.0 || k >= 0.0 || D < 0.0) return INFINITY;
    double sD = sqrt(D);
    return c / (sD - k);
}

/* distance to the planes lo (moving down) or hi (moving up) along one axis */
static double dist_planes(double x, double u, double lo, double hi)
{
    if (u > 0.0) return (hi - x) / u;
    if (u < 0.0) return (lo - x) / u;
    return INFINITY;
}

static void dist_boundary(const or_problem *P, const particle_t *p, double *d, int *surf)
{
    *d = INFINITY;
    *surf = SURF_NONE;
    if (P->kind == 1) {
        double pp = P->pitch;
        double cx = ((double)p->i + 0.5) * pp;
        double cy = ((double)p->j + 0.5) * pp;
        double dc = or_dist_cylinder(p->x - cx, p->y - cy, p->u, p->v, P->radius, p->inside);
        double dx = dist_planes(p->x, p->u, (double)p->i * pp, (double)(p->i + 1) * pp);
        double dy = dist_planes(p->y, p->v, (double)p->j * pp, (double)(p->j + 1) * pp);
        double dz = dist_planes(p->z, p->w, 0.0, P->height);
        if (dc < 0.0) dc = 0.0;
        if (dx < 0.0) dx = 0.0;
        if (dy < 0.0) dy = 0.0;
        if (dz < 0.0) dz = 0.0;
        *d = dc;
        *surf = SURF_CYL;
        if (dx < *d) { *d = dx; *surf = SURF_X; }
        if (dy < *d) { *d = dy; *surf = SURF_Y; }
        if (dz < *d) { *d = dz; *surf = SURF_Z; }
    } else if (P->kind == 2) {
        double h = P->layer_dx;
        double dx = dist_planes(p->x, p->u, (double)p->i * h, (double)(p->i + 1) * h);
        if (dx < 0.0) dx = 0.0;
        *d = dx;
        *surf = SURF_X;
    }
}

static int32_t slab_mat(const or_problem *P, int32_t layer)
{
    return layer < P->n_first ? P->mat_a : P->mat_b;
}

/* Cross the surface reached; returns 1 when the material changed. */
static int cross_surface(const or_problem *P, particle_t *p, int surf)
{
    if (P->kind == 2) {
        double h = P->layer_dx;
        if (p->u > 0.0) {
            p->x = (double)(p->i + 1) * h;
            if (p->i < P->n_layers - 1) {
                p->i += 1;
            } else {
                p->status = OR_STATUS_LEAKED_FAR;
                return 0;
            }
        } else {
            p->x = (double)p->i * h;
            if (p->i > 0) {
                p->i -= 1;
            } else {
                p->status = OR_STATUS_LEAKED;
                return 0;
            }
        }
        int32_t m = slab_mat(P, p->i);
        int changed = (m != p->mat);
        p->mat = m;
        return changed;
    }
    double pp = P->pitch;
    if (surf == SURF_CYL) {
        p->inside = !p->inside;
        int32_t m = p->inside ? P->mat_pin : P->mat_mod;
        int changed = (m != p->mat);
        p->mat = m;
        return changed;
    }
    if (surf == SURF_X) {
        if (p->u > 0.0) {
            p->x = (double)(p->i + 1) * pp;
            if (p->i < P->n - 1) p->i += 1;
            else if (P->bc_side == 1) p->u = -p->u;
            else p->status = OR_STATUS_LEAKED;
        } else {
            p->x = (double)p->i * pp;
            if (p->i > 0) p->i -= 1;
            else if (P->bc_side == 1) p->u = -p->u;
            else p->status = OR_STATUS_LEAKED;
        }
        return 0;
    }
    if (surf == SURF_Y) {
        if (p->v > 0.0) {
            p->y = (double)(p->j + 1) * pp;
            if (p->j < P->n - 1) p->j += 1;
            else if (P->bc_side == 1) p->v = -p->v;
            else p->status = OR_STATUS_LEAKED;
        } else {
            p->y = (double)p->j * pp;
            if (p->j > 0) p->j -= 1;
            else if (P->bc_side == 1) p->v = -p->v;
            else p->status = OR_STATUS_LEAKED;
        }
        return 0;
    }
    /* SURF_Z */
    if (p->w > 0.0) {
        p->z = P->height;
    } else {
        p->z = 0.0;
    }
    if (P->bc_z == 1) p->w = -p->w;
    else p->status = OR_STATUS_LEAKED;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Kinematics: elastic scatter, isotropic in the centre-of-mass frame,      */
/* target at rest.                                                          */
/* ------------------------------------------------------------------------ */

/* Outgoing energy and lab-frame cosine for CM cosine mu and mass ratio A:
 * E' = E (A^2 + 2 A mu + 1) / (A + 1)^2, mu_lab = (1 + A mu) / sqrt(A^2 +
 * 2 A mu + 1). */
void or_elastic(double E, double A, double mu, double *E_out, double *mu_lab)
{
    double t1 = fma(2.0 * A, mu, A * A) + 1.0;
    double ap1 = A + 1.0;
    *E_out = (E * t1) / (ap1 * ap1);
    *mu_lab = fma(A, mu, 1.0) / sqrt(t1);
}

/* Rotate direction (u,v,w) by polar cosine mu and azimuth (cphi, sphi):
 * the textbook rotation, each product-plus-term one fused multiply-add. */
void or_rotate(double *u, double *v, double *w, double mu, double cphi, double sphi)
{
    double m2 = fma(-mu, mu, 1.0);              /* 1 - mu^2 */
    if (m2 < 0.0) m2 = 0.0;
    double st = sqrt(m2);
    double u0 = *u, v0 = *v, w0 = *w;
    if (fabs(w0) < 0.9999999999) {
        double q = sqrt(fma(-w0, w0, 1.0));    /* sqrt(1 - w^2) */
        /* u' = mu u + st (u w cos phi - v sin phi) / q, and so on */
        *u = fma(mu, u0, (st * fma(u0 * w0, cphi, -(v0 * sphi))) / q);
        *v = fma(mu, v0, (st * fma(v0 * w0, cphi, u0 * sphi)) / q);
        *w = fma(mu, w0, -((st * q) * cphi));
    } else {
        *u = st * cphi;
        *v = st * sphi;
        *w = w0 > 0.0 ? mu : -mu;
    }
}

/* Marsaglia (1972) disk rejection: (a,b) uniform in the unit disk. */
static double disk_pair(rng_t *r, double *a, double *b)
{
    for (;;) {
        *a = 2.0 * rng_next(r) - 1.0;
        *b = 2.0 * rng_next(r) - 1.0;
        double s = fma(*a, *a, *b * *b);        /* a^2 + b^2 */
        if (s > 0.0 && s < 1.0) return s;
    }
}

/* ------------------------------------------------------------------------ */
/* Tallies: thread-private, Neumaier-compensated sums.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double *fs, *fc;   /* flux sum / compensation */
    double *as, *ac;   /* absorption-rate sum / compensation (NULL: off) */
    int64_t counts[OR_NSCAL];
    double ws[OR_NSCAL], wc[OR_NSCAL];
} acc_t;

static void kadd(double *s, double *c, double x)
{
    double t = *s + x;
    if (fabs(*s) >= fabs(x))
        *c += (*s - t) + x;
    else
        *c += (x - t) + *s;
    *s = t;
}

static void score(acc_t *A, int slot, double w)
{
    A->counts[slot] += 1;
    kadd(&A->ws[slot], &A->wc[slot], w);
}

static int32_t n_cells(const or_problem *P)
{
    if (P->kind == 1) return P->n * P->n;
    if (P->kind == 2) return P->n_layers;
    return 1;
}

static int32_t cell_of(const or_problem *P, const particle_t *p)
{
    if (P->kind == 1) return p->j * P->n + p->i;
    if (P->kind == 2) return p->i;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One history, birth to death.                                             */
/* ------------------------------------------------------------------------ */
static void birth(const or_problem *P, rng_t *r, particle_t *p, int64_t id)
{
    memset(p, 0, sizeof(*p));
    if (P->source == OR_SRC_BANK) {
        int64_t s = id * P->bank_n / P->bank_total;
        p->x = P->bank[3 * s];
        p->y = P->bank[3 * s + 1];
        p->z = P->bank[3 * s + 2];
    } else if (P->source == 1) {
        double L = (double)P->n * P->pitch;
        p->x = rng_next(r) * L;
        p->y = rng_next(r) * L;
        p->z = rng_next(r) * P->height;
    }
    double a, b;
    double s = disk_pair(r, &a, &b);
    double t = 2.0 * sqrt(1.0 - s);
    double w = 1.0 - 2.0 * s;
    if (P->source == 2) {
        p->u = fabs(w);
        p->v = a * t;
        p->w = b * t;
    } else {
        p->u = a * t;
        p->v = b * t;
        p->w = w;
    }
    p->E = P->E0;
    p->wgt = 1.0;
    p->status = OR_STATUS_ALIVE;
    if (P->kind == 1) {
        double pp = P->pitch;
        int32_t i = (int32_t)floor(p->x / pp);
        int32_t j = (int32_t)floor(p->y / pp);
        if (i < 0) i = 0;
        if (i > P->n - 1) i = P->n - 1;
        if (j < 0) j = 0;
        if (j > P->n - 1) j = P->n - 1;
        p->i = i;
        p->j = j;
        double dx = p->x - ((double)i + 0.5) * pp;
        double dy = p->y - ((double)j + 0.5) * pp;
        p->inside = (dx * dx + dy * dy) < (P->radius * P->radius);
        p->mat = p->inside ? P->mat_pin : P->mat_mod;
    } else if (P->kind == 2) {
        p->i = 0;
        p->mat = slab_mat(P, 0);
    } else {
        p->mat = P->mat;
    }
}

static int32_t ebin(const or_problem *P, double E)
{
    return (int32_t)or_search(P->edges, (int64_t)P->n_bins + 1, E);
}

/* A split's copies: same state, weight w/k, a new history with its own
 * stream.  Copy j of a split at draw position rj of history `hid` has the id
 * given by word 0 of one Philox block of (hid, rj, j, SPLIT_TAG) under the
 * batch key, with the top bit set (primary ids stay below 2^63). */
#define OR_SPLIT_TAG 0x5EED0C41DULL

typedef struct {
    particle_t p;
    uint64_t hid;
} child_t;

typedef struct {
    child_t *v;
    int64_t n, cap;
    int overflow;
} stack_t_;

static void push_child(stack_t_ *S, const particle_t *p, uint64_t hid)
{
    if (S->n == S->cap) {
        int64_t nc = S->cap ? 2 * S->cap : 64;
        if (nc > ((int64_t)1 << 24)) {
            S->overflow = 1;
            return;
        }
        child_t *nv = (child_t *)realloc(S->v, sizeof(child_t) * (size_t)nc);
        if (!nv) {
            S->overflow = 1;
            return;
        }
        S->v = nv;
        S->cap = nc;
    }
    S->v[S->n].p = *p;
    S->v[S->n].hid = hid;
    S->n += 1;
}

/* Weight-window check at the particle's (cell, energy bin): split above the
 * window, Russian roulette below it (survivors take the survival weight). */
static void ww_check(const or_problem *P, particle_t *p, rng_t *r, stack_t_ *S, acc_t *A)
{
    int64_t k = (int64_t)cell_of(P, p) * P->n_bins + ebin(P, p->E);
    double wl = P->ww_lower[k];
    if (!(wl > 0.0)) return;
    double wu = wl * P->ww_ratio;
    double ws = wl * P->ww_survival;
    if (p->wgt > wu) {
        int32_t n = (int32_t)floor(p->wgt / ws);
        if (n > P->ww_max_split) n = P->ww_max_split;
        if (n < 2) return;
        double wc = p->wgt / (double)n;
        p->wgt = wc;
        for (int32_t j = 1; j < n; ++j) {
            uint64_t ctr[4] = {r->id, r->j, (uint64_t)j, OR_SPLIT_TAG};
            uint64_t out[4];
            or_philox4x64_10(ctr, r->key, out);
            particle_t c = *p;
            c.n_coll = 0;
            c.n_flights = 0;
            push_child(S, &c, out[0] | 0x8000000000000000ULL);
            score(A, OR_S_SPLIT, wc);
        }
    } else if (p->wgt < wl) {
        double xi = rng_next(r);
        if (xi < p->wgt / ws) {
            p->wgt = ws;
        } else {
            score(A, OR_S_ROULETTE, p->wgt);
            p->status = OR_STATUS_ROULETTE;
        }
    }
}

/* One history from the given state until death; returns its final state and
 * the number of draws taken from its stream. */
/* Fission sites of one history (k-eigenvalue mode). */
typedef struct {
    double *xyz;      /* [cap][3] */
    int32_t n, cap;
    int overflow;
} sites_t;

static void transport(const or_problem *P, const tables_t *T, rng_t *r, particle_t *pp,
                      int need_lookup, acc_t *A, stack_t_ *S, sites_t *B)
{
    particle_t p = *pp;
    const int32_t nb = P->n_bins;
    while (p.status == OR_STATUS_ALIVE) {
        if (need_lookup) {
            macro_xs(T, p.mat, p.E, &p.st, &p.sa);
            need_lookup = 0;
        }
        double xi = rng_next(r);
        double dcol = (0.0 - or_log(xi)) / p.st;
        double dbnd;
        int surf;
        dist_boundary(P, &p, &dbnd, &surf);
        int collide = dcol < dbnd;
        double d = collide ? dcol : dbnd;
        /* move (r + d Omega, each coordinate one fused multiply-add) and
         * score the track length */
        int32_t cell = cell_of(P, &p);
        p.x = fma(d, p.u, p.x);
        p.y = fma(d, p.v, p.y);
        p.z = fma(d, p.w, p.z);
        {
            /* track-length estimators: flux w d and absorption rate
             * (w d) Sigma_a of the segment's (cell, energy bin) */
            int64_t k = (int64_t)cell * nb + ebin(P, p.E);
            double wd = p.wgt * d;
            kadd(&A->fs[k], &A->fc[k], wd);
            if (A->as) kadd(&A->as[k], &A->ac[k], wd * p.sa);
        }
        p.n_flights += 1;
        score(A, OR_S_FLIGHT, p.wgt);
        if (collide) {
            double target = rng_next(r) * p.st;
            int32_t nuc = pick_nuclide(T, p.mat, p.E, target);
            p.n_coll += 1;
            score(A, OR_S_COLLISION, p.wgt);
            if (P->nu) {
                /* fission sites: expected w nu sigma_f / sigma_t / k_norm */
                double xf = rng_next(r);
                double y = (p.wgt * P->nu[nuc]) * P->f_fis[nuc] / P->k_norm + xf;
                int32_t nb = (int32_t)floor(y);
                for (int32_t q = 0; q < nb; ++q) {
                    if (B->n >= B->cap) {
                        B->overflow = 1;
                        break;
                    }
                    B->xyz[3 * B->n] = p.x;
                    B->xyz[3 * B->n + 1] = p.y;
                    B->xyz[3 * B->n + 2] = p.z;
                    B->n += 1;
                }
            }
            double xa = rng_next(r);
            if (xa < P->f_abs[nuc]) {
                p.status = OR_STATUS_ABSORBED;
                score(A, OR_S_ABSORPTION, p.wgt);
            } else {
                double mu = 2.0 * rng_next(r) - 1.0;
                double a, b;
                double s = disk_pair(r, &a, &b);
                double cphi = fma(a, a, -(b * b)) / s;   /* (a^2 - b^2) / s */
                double sphi = ((2.0 * a) * b) / s;
                double E1, mul;
                or_elastic(p.E, P->awr[nuc], mu, &E1, &mul);
                or_rotate(&p.u, &p.v, &p.w, mul, cphi, sphi);
                p.E = E1;
                if (p.E < P->E_cut) {
                    p.status = OR_STATUS_CUTOFF;
                    score(A, OR_S_CUTOFF, p.wgt);
                } else {
                    need_lookup = 1;
                    if (P->ww_lower) ww_check(P, &p, r, S, A);
                }
            }
        } else {
            int changed = cross_surface(P, &p, surf);
            if (p.status == OR_STATUS_LEAKED) score(A, OR_S_LEAK, p.wgt);
            if (p.status == OR_STATUS_LEAKED_FAR) {
                score(A, OR_S_LEAK, p.wgt);
                score(A, OR_S_LEAK_FAR, p.wgt);
            }
            need_lookup = need_lookup || changed;
            if (p.status == OR_STATUS_ALIVE && P->ww_lower && P->kind == 2)
                ww_check(P, &p, r, S, A);
        }
        if (p.status == OR_STATUS_ALIVE && p.n_flights >= OR_MAX_FLIGHTS) {
            p.status = OR_STATUS_LIMIT;
            score(A, OR_S_LIMIT, p.wgt);
        }
    }
    *pp = p;
}

/* History `id` of the batch and, depth first, every copy its splits made. */
static int history(const or_problem *P, const tables_t *T, uint64_t seed, uint64_t key_hi,
                   int64_t id, acc_t *A, particle_t *out, uint32_t *ndraw, sites_t *B)
{
    rng_t r;
    rng_init(&r, seed, key_hi, (uint64_t)id);
    particle_t p;
    birth(P, &r, &p, id);
    A->counts[OR_S_HISTORY] += 1;
    kadd(&A->ws[OR_S_HISTORY], &A->wc[OR_S_HISTORY], p.wgt);
    stack_t_ S = {NULL, 0, 0, 0};
    transport(P, T, &r, &p, 1, A, &S, B);
    *out = p;
    *ndraw = r.j;
    while (S.n > 0 && !S.overflow) {
        child_t ch = S.v[--S.n];
        rng_t rc;
        rng_init(&rc, seed, key_hi, ch.hid);
        transport(P, T, &rc, &ch.p, 1, A, &S, B);
    }
    int bad = S.overflow ? 1 : (B->overflow ? 3 : 0);
    free(S.v);
    return bad;
}

/* exported for tests: the birth state of particle `id` (x,y,z,u,v,w,E and
 * the lattice cell / layer, pin flag and material). */
void or_birth_state(const or_problem *P, uint64_t seed, uint64_t key_hi, int64_t id,
                    double st[7], int32_t cell[4])
{
    rng_t r;
    rng_init(&r, seed, key_hi, (uint64_t)id);
    particle_t p;
    birth(P, &r, &p, id);
    st[0] = p.x; st[1] = p.y; st[2] = p.z;
    st[3] = p.u; st[4] = p.v; st[5] = p.w; st[6] = p.E;
    cell[0] = p.i; cell[1] = p.j; cell[2] = p.inside; cell[3] = p.mat;
}

/* Run particles [first_id, first_id + n) of one batch. */
int or_run(const or_problem *P, uint64_t seed, uint64_t key_hi, int64_t first_id, int64_t n,
           int n_threads, or_result *R)
{
    tables_t T;
    if (tables_init(&T, P)) return -1;
    const int64_t nf = (int64_t)n_cells(P) * P->n_bins;
    if (n_threads <= 0) n_threads = 1;
    acc_t *acc = (acc_t *)calloc((size_t)n_threads, sizeof(acc_t));
    if (!acc) return -1;
    for (int t = 0; t < n_threads; ++t) {
        acc[t].fs = (double *)calloc((size_t)nf, sizeof(double));
        acc[t].fc = (double *)calloc((size_t)nf, sizeof(double));
        if (!acc[t].fs || !acc[t].fc) return -1;
        if (R->absrate) {
            acc[t].as = (double *)calloc((size_t)nf, sizeof(double));
            acc[t].ac = (double *)calloc((size_t)nf, sizeof(double));
            if (!acc[t].as || !acc[t].ac) return -1;
        }
    }
    int overflow = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(n_threads)
#endif
    for (int64_t k = 0; k < n; ++k) {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        particle_t p;
        uint32_t nd;
        sites_t B = {NULL, 0, 0, 0};
        if (P->nu && R->sites) {
            B.xyz = R->sites + (size_t)k * (size_t)P->max_sites * 3;
            B.cap = P->max_sites;
        }
        int bad = history(P, &T, seed, key_hi, first_id + k, &acc[t], &p, &nd, &B);
        if (bad) overflow = bad;
        if (R->n_sites) R->n_sites[k] = B.n;
        if (R->n_coll) R->n_coll[k] = p.n_coll;
        if (R->status) R->status[k] = (int8_t)p.status;
        if (R->n_flights) R->n_flights[k] = p.n_flights;
        if (R->n_draws) R->n_draws[k] = nd;
        if (R->E) R->E[k] = p.E;
        if (R->x) R->x[k] = p.x;
        if (R->y) R->y[k] = p.y;
        if (R->z) R->z[k] = p.z;
    }
    /* reduce the thread partials (sums and compensations as separate terms) */
    if (R->flux) {
        for (int64_t b = 0; b < nf; ++b) {
            double s = 0.0, c = 0.0;
            for (int t = 0; t < n_threads; ++t) {
                kadd(&s, &c, acc[t].fs[b]);
                kadd(&s, &c, acc[t].fc[b]);
            }
            R->flux[b] = s + c;
        }
    }
    if (R->absrate) {
        for (int64_t b = 0; b < nf; ++b) {
            double s = 0.0, c = 0.0;
            for (int t = 0; t < n_threads; ++t) {
                kadd(&s, &c, acc[t].as[b]);
                kadd(&s, &c, acc[t].ac[b]);
            }
            R->absrate[b] = s + c;
        }
    }
    for (int q = 0; q < OR_NSCAL; ++q) {
        int64_t cnt = 0;
        double s = 0.0, c = 0.0;
        for (int t = 0; t < n_threads; ++t) {
            cnt += acc[t].counts[q];
            kadd(&s, &c, acc[t].ws[q]);
            kadd(&s, &c, acc[t].wc[q]);
        }
        if (R->counts) R->counts[q] = cnt;
        if (R->weights) R->weights[q] = s + c;
    }
    for (int t = 0; t < n_threads; ++t) {
        free(acc[t].fs);
        free(acc[t].fc);
        free(acc[t].as);
        free(acc[t].ac);
    }
    free(acc);
    tables_free(&T);
    return overflow == 3 ? -3 : (overflow ? -2 : 0);
}

/* ------------------------------------------------------------------------ */
/* Importance network (binary64 reference of the GPU kernels).              */
/* 4 -> 64 -> 64 -> 1, ReLU after the two hidden layers.  Parameters, in    */
/* this order: W1[64][4], b1[64], W2[64][64] (row = output unit), b2[64],   */
/* W3[64], b3.                                                              */
/* ------------------------------------------------------------------------ */
#define OR_H 64
#define OR_NPARAM (OR_H * 4 + OR_H + OR_H * OR_H + OR_H + OR_H + 1)

int or_mlp_nparam(void) { return OR_NPARAM; }

static void mlp_one(const double *P, const double *x, double *z1, double *h1, double *z2,
                    double *h2, double *out)
{
    const double *W1 = P, *b1 = W1 + OR_H * 4, *W2 = b1 + OR_H, *b2 = W2 + OR_H * OR_H,
                 *W3 = b2 + OR_H, *b3 = W3 + OR_H;
    for (int o = 0; o < OR_H; ++o) {
        double s = b1[o];
        for (int i = 0; i < 4; ++i) s += W1[o * 4 + i] * x[i];
        z1[o] = s;
        h1[o] = s > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < OR_H; ++o) {
        double s = b2[o];
        for (int i = 0; i < OR_H; ++i) s += W2[o * OR_H + i] * h1[i];
        z2[o] = s;
        h2[o] = s > 0.0 ? s : 0.0;
    }
    double s = b3[0];
    for (int i = 0; i < OR_H; ++i) s += W3[i] * h2[i];
    *out = s;
}

void or_mlp_forward(const double *params, const double *x, int64_t n, double *out)
{
    double z1[OR_H], h1[OR_H], z2[OR_H], h2[OR_H];
    for (int64_t k = 0; k < n; ++k) mlp_one(params, x + 4 * k, z1, h1, z2, h2, &out[k]);
}

/* Loss L = sum_k w_k (out_k - y_k)^2 / sum_k w_k and its gradient dL/dparams
 * (same layout as params) by back-propagation. */
double or_mlp_grad(const double *params, const double *x, const double *y, const double *w,
                   int64_t n, double *grad)
{
    const double *W2 = params + OR_H * 4 + OR_H, *W3 = W2 + OR_H * OR_H + OR_H;
    double *gW1 = grad, *gb1 = gW1 + OR_H * 4, *gW2 = gb1 + OR_H, *gb2 = gW2 + OR_H * OR_H,
           *gW3 = gb2 + OR_H, *gb3 = gW3 + OR_H;
    memset(grad, 0, sizeof(double) * OR_NPARAM);
    double wsum = 0.0, loss = 0.0;
    for (int64_t k = 0; k < n; ++k) wsum += w[k];
    double z1[OR_H], h1[OR_H], z2[OR_H], h2[OR_H], d2[OR_H], d1[OR_H], out;
    for (int64_t k = 0; k < n; ++k) {
        const double *xk = x + 4 * k;
        mlp_one(params, xk, z1, h1, z2, h2, &out);
        double e = out - y[k];
        loss += w[k] * e * e;
        double dout = 2.0 * w[k] * e / wsum;
        gb3[0] += dout;
        for (int i = 0; i < OR_H; ++i) {
            gW3[i] += dout * h2[i];
            d2[i] = z2[i] > 0.0 ? dout * W3[i] : 0.0;
        }
        for (int o = 0; o < OR_H; ++o) {
            gb2[o] += d2[o];
            for (int i = 0; i < OR_H; ++i) gW2[o * OR_H + i] += d2[o] * h1[i];
        }
        for (int i = 0; i < OR_H; ++i) {
            double s = 0.0;
            for (int o = 0; o < OR_H; ++o) s += W2[o * OR_H + i] * d2[o];
            d1[i] = z1[i] > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < OR_H; ++o) {
            gb1[o] += d1[o];
            for (int i = 0; i < 4; ++i) gW1[o * 4 + i] += d1[o] * xk[i];
        }
    }
    return loss / wsum;
}
