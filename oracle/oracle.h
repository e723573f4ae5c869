/*
 * CPU oracle for the event-based Monte Carlo transport hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, history-based
 * definition of what the GPU path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load it; the product library
 * never links, loads or calls it, and the two share no code.
 *
 * The paper (Sec. 2, "Event-Based Parallelism") states that an event-based
 * GPU schedule and a history-based CPU schedule simulate the same particle
 * histories, and (Sec. 4.3) that serial CPU and GPU results agree up to
 * floating-point non-associativity.  The oracle is therefore the history
 * loop: each particle from birth to death, in order, driven by its own
 * counter-based random stream.
 */
#ifndef GBMC_ORACLE_H
#define GBMC_ORACLE_H
#include <stdint.h>

#define OR_STATUS_ALIVE 0
#define OR_STATUS_ABSORBED 1
#define OR_STATUS_LEAKED 2
#define OR_STATUS_CUTOFF 3
#define OR_STATUS_LIMIT 4
#define OR_STATUS_LEAKED_FAR 5
#define OR_STATUS_ROULETTE 6

/* scalar tally slots */
#define OR_S_COLLISION 0
#define OR_S_ABSORPTION 1
#define OR_S_LEAK 2
#define OR_S_CUTOFF 3
#define OR_S_LIMIT 4
#define OR_S_LEAK_FAR 5
#define OR_S_FLIGHT 6
#define OR_S_HISTORY 7
#define OR_S_SPLIT 8
#define OR_S_ROULETTE 9
#define OR_NSCAL 10

#define OR_MAX_FLIGHTS 100000

typedef struct {
    int32_t n_nuc;
    const int64_t *grid_off;   /* [n_nuc+1] */
    const double *energy;      /* [grid_off[n_nuc]] eV, strictly increasing per nuclide */
    const double *sigma_t;     /* [grid_off[n_nuc]] barns */
    const double *f_abs;       /* [n_nuc] sigma_a / sigma_t */
    const double *awr;         /* [n_nuc] atomic-weight ratio A */
    int32_t n_mat;
    const int32_t *mat_off;    /* [n_mat+1] */
    const int32_t *nuc_id;     /* [mat_off[n_mat]] */
    const double *density;     /* [mat_off[n_mat]] atoms/(b cm) */
    int32_t n_bins;
    const double *edges;       /* [n_bins+1] */
    int32_t precision;         /* 0: binary64 tables, 1: binary32 tables */
    /* geometry */
    int32_t kind;              /* 0 infinite, 1 lattice, 2 slab */
    int32_t source;            /* 0 origin, 1 box, 2 slab face */
    double E0, E_cut;
    int32_t mat;
    int32_t n;
    double pitch, radius, height;
    int32_t mat_pin, mat_mod, bc_side, bc_z;
    int32_t n_layers;
    double layer_dx;
    int32_t n_first, mat_a, mat_b;
    /* weight windows (NULL: analog): lower bound per (cell, energy bin);
     * upper = ratio * lower, survival = survival * lower; at most max_split
     * copies per split.  Checked after every scatter and every slab-layer
     * crossing. */
    const double *ww_lower;   /* [n_cells * n_bins]; <= 0 means no window */
    double ww_ratio, ww_survival;
    int32_t ww_max_split;
    /* k-eigenvalue (nu NULL: off).  At every collision in nuclide i the
     * history banks floor(w nu_i f_fis_i / k_norm + xi) fission sites at the
     * collision point (xi one draw, taken right after the nuclide choice), at
     * most max_sites per history.  source 3 starts history id at site
     * floor(id bank_n / bank_total) of the bank, energy E0, isotropic. */
    const double *nu;         /* [n_nuc] mean neutrons per fission */
    const double *f_fis;      /* [n_nuc] sigma_f / sigma_t */
    double k_norm;
    int32_t max_sites;
    const double *bank;       /* [bank_n][3] */
    int64_t bank_n, bank_total;
} or_problem;

#define OR_SRC_BANK 3

typedef struct {
    int32_t *n_coll;      /* [n] */
    int8_t *status;       /* [n] */
    int32_t *n_flights;   /* [n] */
    uint32_t *n_draws;    /* [n] */
    double *E, *x, *y, *z;/* [n] final state */
    double *flux;         /* [n_cells*n_bins], overwritten */
    double *absrate;      /* [n_cells*n_bins] track-length absorption rate sum w d Sigma_a
                           * (NULL: not scored), overwritten */
    int64_t *counts;      /* [OR_NSCAL], overwritten */
    double *weights;      /* [OR_NSCAL], overwritten */
    double *sites;        /* [n][max_sites][3] fission sites in banking order (k-eigenvalue) */
    int32_t *n_sites;     /* [n] sites banked by each history */
} or_result;

#endif
