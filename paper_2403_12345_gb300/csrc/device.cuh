// Device-side building blocks of the transport hot path: the per-particle
// counter-based random stream, a reproducible logarithm, the cross-section
// lookup, surface distances and elastic-scatter kinematics.
//
// Every binary64/binary32 expression here is compiled without FMA
// contraction (-fmad=false) and evaluated exactly in the written order; the
// fused multiply-adds of the method's reading are written out (__fma_rn, one
// rounding). A particle's random walk is therefore a pure function of its
// inputs and matches a serial history-based evaluation of the same
// definitions bit for bit (reproducibility between CPU and GPU up to
// summation order: Sec. 4.3).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <cstring>

#include "../../include/gbmc.h"

namespace gbmc {

// ---------------------------------------------------------------- layouts

// Per-nuclide search descriptor, built on the host; the kernels read its
// fields through the per-material-entry records Desc64 and Desc32.
struct NucIndex {
    int64_t off;        // first grid point of the nuclide in the pooled grid
    int64_t idx_off;    // first entry of its coarse index
    uint64_t base;      // bit pattern of its first grid energy
    int32_t n;          // grid points
    int32_t shift;      // bucket of E = (bits(E) - base) >> shift
    int32_t nb;         // buckets; index entries idx[idx_off .. idx_off + nb]
};

// Per material entry q, binary32 tables: what the lookup reads for nuclide
// nuc_id[q] in one 32-byte record (two 16-byte loads).
struct alignas(16) Desc32 {
    int32_t off;       // first (E, sigma) pair of the nuclide in es32 (even)
    int32_t bw_off;    // its first bucket window in bw32
    uint32_t base;     // bit pattern of its first grid energy
    int32_t n;         // grid points
    int32_t shift;     // bucket of E = (bits(E) - base) >> shift
    int32_t nb;        // buckets
    float density;     // N of this entry, binary32
    float f_abs;       // sigma_a / sigma_t of the nuclide, binary32
};
static_assert(sizeof(Desc32) == 32, "Desc32 is read as two int4");

// Per material entry q, binary64 tables: the search descriptor of nuclide
// nuc_id[q] in one 32-byte record (two 16-byte loads).
struct alignas(16) Desc64 {
    int64_t off;       // first grid point of the nuclide in e64 / iv64
    uint64_t base;     // bit pattern of its first grid energy
    int32_t idx_off;   // first entry of its coarse index in idx64
    int32_t n;         // grid points
    int32_t shift;     // bucket of E = (bits(E) - base) >> shift
    int32_t nb;        // buckets
};
static_assert(sizeof(Desc64) == 32, "Desc64 is read as two int4");

// Interval k of a binary64 grid (from point k to point k+1): the operands of
// the lin-lin interpolation that depend on the interval alone, computed on
// the host with the same binary64 subtractions the interpolation states, so
// the kernels form bit-identical results with fewer binary64 operations.
//   de = E_k+1 - E_k, ds = s_k+1 - s_k (rounded to nearest), s0 = s_k,
//   y  = floor(2^126 / (M_de 2^11)) for the significand M_de in [2^52, 2^53)
//        of de (a fixed-point reciprocal for the division by de), or 0 when
//        de is not a positive normal number (the kernels then divide by de
//        in binary64).
struct alignas(32) Interval64 {
    double de, ds, s0;
    unsigned long long y;
};

struct Tables {
    const int64_t* grid_off;   // [n_nuc+1]
    const Desc64* d64;         // [mat_off[n_mat]] per material entry (binary64)
    const uint32_t* idx64;     // coarse index of the binary64 grids
    const float4* bw32;        // binary32 bucket windows (four float4 each)
    const Desc32* d32;         // [mat_off[n_mat]] per material entry (binary32)
    const float4* bs32;        // binary32 short windows of the finer index (two float4 each)
    const int2* br32;          // bracket range (lo, hi) of each short window's bucket
    const Desc32* d32s;        // [mat_off[n_mat]] per material entry, finer index (bw_off,
                               // shift, nb refer to the short windows)
    const double* e64;         // binary64 grid (eV)
    const Interval64* iv64;    // binary64 intervals, indexed like e64 (last of each grid unused)
    const float2* es32;        // binary32 (E, sigma_t) pairs, each nuclide followed by
                               // kPad32 pairs (+inf, 0)
    const double* f_abs;       // [n_nuc]
    const float* f_abs32;      // [n_nuc]
    const double* awr;         // [n_nuc]
    const int32_t* mat_off;    // [n_mat+1]
    const int32_t* nuc_id;     // [mat_off[n_mat]]
    const double* density;     // [mat_off[n_mat]]
    const float* density32;    // [mat_off[n_mat]]
    const double* edges;       // [n_bins+1] tally energy edges
    const double* nu;          // [n_nuc] mean neutrons per fission (k-eigenvalue)
    const double* f_fis;       // [n_nuc] sigma_f / sigma_t
    int32_t n_nuc, n_mat, n_bins;
    int32_t plain;             // 1: plain binary search of each grid (no coarse index, no windows)
};

// One problem of a run, as the kernels see it.
struct DevProblem {
    gbmc_geometry g;
    uint64_t seed, key_hi;
    int64_t first_id, n, start;   // start: index of its first particle in the run
    int64_t flux_off;             // offset of its flux tally
    int64_t out_base;             // outcome index of its first particle
    int64_t plane_off;            // its plane table: walls (double)i * pitch, i = 0..n, then
                                  // lattice cell centres ((double)i + 0.5) * pitch, i < n
    double r2;                    // lattice pin radius squared (radius * radius)
    int32_t n_cells;
    int32_t slot;                 // its tally slot (scalar tallies)
};

// One slot of the particle bank: a 128-byte, 128-byte-aligned record (array
// of structures).  Queues visit slots in data-dependent order, so each
// particle costs whole cache lines either way; one record per line, with the
// fields grouped by 32-byte sector after the events that read them, keeps
// each event to the sectors it needs (the lookup touches sector 0 only).
struct alignas(128) Particle {
    // sector 0: lookup reads E, mat; writes st, sa
    double st, sa;       // macroscopic sigma_t, sigma_a at (E, mat)
    double E;
    int32_t mat, prob;   // material, problem slot
    // sector 1
    double x, y, z, wgt;
    // sector 2
    double u, v, w;
    int64_t gidx;        // outcome index of the history (-1: a split copy)
    // sector 3
    int32_t ci, cj;      // lattice cell (slab: layer in ci)
    int32_t ncoll, nflt; // collisions, flights so far
    uint32_t rj;         // draws consumed from the particle's stream
    uint8_t inside;      // inside the pin cylinder (lattice)
    uint8_t surf;        // surface reached by the last flight
    uint8_t nsite;       // fission sites banked by the history so far (k-eigenvalue)
    uint8_t pad8;
    uint64_t hid;        // history id: counter word 0 of the particle's stream
};
static_assert(sizeof(Particle) == 128, "one particle per 128-byte line");

struct Bank {
    Particle* p;         // [capacity]
};

// Event queues (slot indices) and sort scratch.
struct Queues {
    int32_t* lq[2];     // lookup queue (double buffered)
    int32_t* aq[2];     // advance queue (double buffered)
    int32_t* cq;        // collision queue
    int32_t* fq;        // free slots
    int32_t* lqs;       // lookup queue in (material, energy) order
    uint32_t* keys[2];  // sort keys of lq[b], written by the kernel that appends the entry
    uint32_t* rank[2];  // each entry's rank within its bucket, from the append's count
    uint32_t* hist[2];  // [kSortBuckets] bucket counts of lq[b], counted at the append
    uint32_t* cursor;   // [kSortBuckets] bucket write positions (block-local)
    uint32_t* btot;     // [kSortBuckets / 1024] bucket-block totals
};

struct Outcomes {
    int32_t* ncoll;
    int8_t* status;
    int32_t* nflt;
    uint32_t* ndraw;
    double *E, *x, *y, *z;
};

struct Tallies {
    double* flux;
    unsigned long long* counts;   // [slot * GBMC_NSCAL + s]
    double* weights;
    double* absrate;              // track-length absorption rate, laid out as flux (NULL: off)
};

// Device-resident event-loop state.
struct Ctl {
    int32_t n_lq[2], n_aq[2], n_cq, n_free;
    int32_t cur;                 // queues[cur] are consumed this iteration
    int32_t lookup_n, aq_base;   // lookups of this iteration, where they append in aq[cur]
    int32_t n_birth, free_base, lq_base, sorted;
    int32_t warp_lookup;         // this iteration's lookups run one warp per particle
    int32_t group_lookup;        // this iteration's lookups run kGroupLanes lanes per particle
    int32_t adv_n;               // particles the ray-trace kernel takes this iteration
    int32_t tail;                // the loop stopped early: the tail kernel finishes
    int32_t adv_cursor;          // next ray-trace queue entry to hand out
    int32_t lookup_cursor;       // next lookup queue chunk to hand out (thread mode)
    int32_t n_child;             // split copies waiting to be born
    int32_t n_birth_child;       // copies born this iteration (the first births)
    int32_t child_base;          // first of them in the copy buffer
    int32_t birth_reserve;       // free slots the source leaves for split copies
    int32_t n_imp;               // importance samples recorded
    int32_t pad6;
    int64_t next_base;           // run index of the first particle born this iteration
    int64_t next, total;         // next unborn run index, particles in the run
    int32_t M;                   // in-flight cap of this run (<= capacity)
    int32_t n_prob;
    int32_t done, err, iter, pad;
    double k_norm;               // k-eigenvalue: fission yield normalisation of this run
    int64_t bank_n, bank_total;  // source bank size, generation size (GBMC_SRC_BANK)
};

// Counters of the runs since they were last zeroed (one run, or every run
// one event loop takes in a concurrent call), kept apart from the per-run
// control block so that they can add up across runs.
struct RunStats {
    unsigned long long iterations, lookups, micro, flights, cross, coll, hist;
    unsigned long long handoff;   // particles a drained ray-trace warp handed on
    int32_t err;                  // the first error a run of them flagged (0: none)
    int32_t pad;
};

constexpr int kSortBuckets = 1 << 16;
constexpr int kMaxSharedProblems = 64;
static_assert(kSortBuckets == 64 * 1024, "the bucket scan runs 64 blocks of 1024");

struct Params {
    Tables T;
    Bank B;
    Queues Q;
    Outcomes O;
    Tallies Y;
    Ctl* ctl;
    RunStats* st;
    const DevProblem* probs;
    int32_t capacity;        // bank slots allocated
    int32_t precision;       // GBMC_FP64 / GBMC_FP32
    int32_t sort;            // sort the lookup queue
    int32_t sort_min;        // sort only when at least this many lookups
    int32_t warp_lookup_max; // below this many lookups: one warp per particle
    int32_t group_lookup_max; // below this many (and not warp mode): kGroupLanes lanes per particle
    int32_t tail_max;        // stop the loop and finish in the tail kernel at or below
                             // this many particles in flight (source exhausted)
    int32_t max_iter;
    int32_t sparse_windows;  // binary32 lookup on the short windows (host: kernel choice)
    uint32_t sort_shift;     // energy-bits >> shift = bucket within a material
    uint32_t bpm_log2;       // log2 buckets per material
    int32_t use_cond;        // 1 inside the graph while-body, 0 for eager launches
    uint64_t sort_ebase;
    const double* ww;        // weight-window lower bounds of problem slot 0 (NULL: analog)
    double ww_ratio, ww_survival;
    int32_t ww_max_split;
    int32_t child_cap;       // capacity of the split-copy buffer
    Particle* child;         // split copies waiting for a bank slot
    int32_t* imp_mesh;       // importance samples: mesh index of a collision (NULL: off)
    int64_t* imp_gidx;       //   and the history it belongs to
    int32_t imp_cap;
    int32_t pad5;
    const double* planes;    // plane tables of the run's problems (DevProblem::plane_off)
    // k-eigenvalue (sites NULL: off): history g of the run banks its fission
    // sites at sites[(g max_sites + k) * 3], its count at site_n[g]; after
    // the run they are compacted into bank_out (size *bank_size)
    double* sites;
    int32_t* site_n;
    int64_t* site_off;
    int64_t* bank_size;
    double* bank_out;
    const double* bank;      // source bank [Ctl::bank_n][3] of GBMC_SRC_BANK runs
    int32_t max_sites;
    int32_t pad6;
    void* cum;               // running sums of N_i sigma_i, slot-major (NULL: recompute)
    int64_t cum_stride;      // elements per slot (the most nuclides of any material)     // bits of the smallest grid energy
    cudaGraphConditionalHandle cond;
};

// ---------------------------------------------------------------- Philox4x64-10
// Salmon et al., SC'11: ten rounds; each multiplies counter words 0 and 2 by
// the round constants (full 128-bit products), swaps and xors the high halves
// with words 1 and 3 and the key, which is bumped between rounds by the
// golden-ratio and sqrt(3)-1 Weyl increments.

struct Philox {
    uint64_t c0, c1, c2, c3;
};

__device__ __forceinline__ Philox philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                 uint64_t c3, uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
        uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return {c0, c1, c2, c3};
}

// The particle's stream: key (seed, problem << 32 | batch), counter
// (history id, block, 0, 0); draw j is word j % 4 of block j / 4, mapped to
// (0, 1] as ((x >> 11) + 1) 2^-53.
struct Stream {
    uint64_t k0, k1, id;
    uint32_t j, blk;
    bool have;
    Philox b;

    __device__ __forceinline__ void init(uint64_t seed, uint64_t key_hi, uint64_t hid, uint32_t j0) {
        k0 = seed;
        k1 = key_hi;
        id = hid;
        j = j0;
        have = false;
        blk = 0;
    }
    __device__ __forceinline__ double next() {
        uint32_t bk = j >> 2;
        if (!have || bk != blk) {
            b = philox4x64_10(id, bk, 0, 0, k0, k1);
            blk = bk;
            have = true;
        }
        uint32_t w = j & 3u;
        uint64_t x = w == 0 ? b.c0 : (w == 1 ? b.c1 : (w == 2 ? b.c2 : b.c3));
        j += 1;
        return u01(x);
    }
    // ((x >> 11) + 1) 2^-53 in (0, 1], assembled exactly from its bits on the
    // integer units: the leading one of the 53-bit integer n sets the
    // exponent, the bits below it the significand.
    __device__ __forceinline__ static double u01(uint64_t x) {
        uint64_t n = (x >> 11) + 1ull;
        int lz = __clzll((long long)n);
        uint64_t sig = ((n << lz) & 0x7FFFFFFFFFFFFFFFull) >> 11;
        return __longlong_as_double((long long)(((uint64_t)(1033 - lz) << 52) | sig));
    }
};

// ---------------------------------------------------------------- division on the integer units
// Correctly rounded binary64 quotient q = RN(a / b) computed with integer
// instructions only, for finite normal a, b (or a = 0) with a normal
// quotient; anything else falls back to the binary64 division.  On this GPU
// a binary64 division occupies the scarce binary64 pipe for ~9 fused
// multiply-add slots, while the integer pipes idle in the kernels that divide.
//
// With significands A, B in [2^52, 2^53) the quotient's significand comes
// from Q = floor(R 2^64 / d), d = B 2^11 in [2^63, 2^64), R = A (A >= B) or
// 2A (A < B), so Q lies in [2^53, 2^54): Q >> 1 are its 53 bits, Q & 1 the
// round bit and a nonzero remainder the sticky bit.  Q is estimated with a
// fixed-point reciprocal 2^126 / d (binary32 seed, two Newton steps), then
// made exact by the 128-bit remainder R 2^64 - Q d (division by an
// invariant integer through a precomputed reciprocal, as in Moller and
// Granlund, IEEE Trans. Computers 60(2), 2011).
__device__ __forceinline__ double div_rn(double a, double b) {
    const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
    const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
    const unsigned long long sign = (ua ^ ub) & 0x8000000000000000ull;
    const int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
    const bool a0 = (ua << 1) == 0ull;
    if (eb == 0 || eb == 0x7ff || ((ea == 0 || ea == 0x7ff) && !a0)) return a / b;
    if (a0) return __longlong_as_double((long long)sign);
    const unsigned long long M = (1ull << 52) - 1ull;
    const unsigned long long A = (ua & M) | (1ull << 52), B = (ub & M) | (1ull << 52);
    const bool ge = A >= B;
    const unsigned long long R = ge ? A : (A << 1);
    const unsigned long long d = B << 11;
    // reciprocal y ~ 2^126 / d in (2^62, 2^63]: binary32 seed from d's top 24
    // bits (about 23 correct bits), then two Newton steps y += y e / 2^126,
    // e = 2^126 - d y, in 64-bit fixed point (within one unit afterwards)
    float w = __frcp_rn((float)(unsigned)(d >> 40)) * 16777216.0f;   // 2^64 / d, in (1, 2]
    unsigned long long y = (unsigned long long)(unsigned)(w * 1073741824.0f) << 32;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        unsigned long long lo = d * y, hi = __umul64hi(d, y);
        long long eh = (long long)((1ull << 62) - hi - (lo != 0ull ? 1ull : 0ull));
        unsigned long long el = 0ull - lo;
        unsigned long long ae = (unsigned long long)(eh < 0 ? -eh : eh);
        unsigned long long mag = (__umul64hi(y, ae) << 2) | ((y * ae) >> 62);
        long long corr = eh < 0 ? -(long long)mag : (long long)mag;
        corr += (long long)(__umul64hi(y, el) >> 62);
        y = (unsigned long long)((long long)y + corr);
    }
    // quotient estimate R 2^64 / d = (4 R) y / 2^64 and exact correction by
    // the remainder R 2^64 - Q d (at most a few steps)
    unsigned long long Q = __umul64hi(R << 2, y);
    unsigned long long qlo = Q * d, qhi = __umul64hi(Q, d);
    unsigned long long rlo = 0ull - qlo;
    long long rhi = (long long)(R - qhi - (qlo != 0ull ? 1ull : 0ull));
#pragma unroll 1
    for (int k = 0; k < 4 && rhi < 0; ++k) {   // remainder negative: Q too large
        --Q;
        unsigned long long t = rlo + d;
        rhi += (t < rlo) ? 1 : 0;
        rlo = t;
    }
#pragma unroll 1
    for (int k = 0; k < 4 && (rhi > 0 || (rhi == 0 && rlo >= d)); ++k) {   // remainder >= d
        ++Q;
        rhi -= (rlo < d) ? 1 : 0;
        rlo -= d;
    }
    if (rhi != 0 || rlo >= d || Q < (1ull << 53) || Q >= (1ull << 54)) return a / b;   // not reached
    unsigned long long m = Q >> 1;
    if ((Q & 1ull) && (rlo != 0ull || (m & 1ull))) ++m;   // to nearest, ties to even
    int e = ea - eb + (ge ? 1023 : 1022);
    if (m == (1ull << 53)) {
        m >>= 1;
        ++e;
    }
    if (e < 1 || e > 2046) return a / b;   // subnormal or overflowing quotient
    return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | (m & M)));
}

// The interpolation factor f = (E - e0) / de (both steps rounded to nearest,
// as in binary64) for a bracket e0 <= E, with y the interval's fixed-point
// reciprocal of de.  E - e0 is formed exactly on the integer units when the
// exponents of E and e0 differ by at most 10 (the difference then fits in 64
// bits and is rounded once, to nearest even); the quotient's significand is
// floor(R 2^64 / d) estimated as (4 R) y / 2^64, which is off by at most one
// (y is exact to one unit and R < 2^54), then made exact by the remainder.
// Other operands (E below e0, far above the interval, special values, y = 0)
// take the binary64 subtraction and div_rn.
__device__ __forceinline__ double frac_rn(double E, double e0, double de, unsigned long long y) {
    const unsigned long long xE = (unsigned long long)__double_as_longlong(E);
    const unsigned long long x0 = (unsigned long long)__double_as_longlong(e0);
    const int eE = (int)(xE >> 52), e0x = (int)(x0 >> 52);   // sign bit included
    const int sh = eE - e0x;
    if (y == 0ull || e0x == 0 || eE >= 0x7ff || sh < 0 || sh > 10 || xE < x0)
        return div_rn(E - e0, de);
    if (xE == x0) return 0.0;
    const unsigned long long M = (1ull << 52) - 1ull;
    // exact D 2^(e0x - 1075) = E - e0, D in (0, 2^63)
    const unsigned long long D = (((xE & M) | (1ull << 52)) << sh) - ((x0 & M) | (1ull << 52));
    const int nz = __clzll((long long)D);
    unsigned long long A;
    int ea;
    if (nz >= 11) {   // at most 53 bits: exact
        A = D << (nz - 11);
        ea = e0x - (nz - 11);
    } else {          // round to 53 bits, to nearest even
        const int r = 11 - nz;
        A = D >> r;
        const unsigned long long rem = D & ((1ull << r) - 1ull), half = 1ull << (r - 1);
        if (rem > half || (rem == half && (A & 1ull))) ++A;
        ea = e0x + r;
        if (A == (1ull << 53)) {
            A >>= 1;
            ++ea;
        }
    }
    const unsigned long long xd = (unsigned long long)__double_as_longlong(de);
    const int eb = (int)(xd >> 52);   // de is a positive normal number (y != 0)
    const unsigned long long B = (xd & M) | (1ull << 52);
    const bool ge = A >= B;
    const unsigned long long R = ge ? A : (A << 1);
    const unsigned long long d = B << 11;
    unsigned long long Q = __umul64hi(R << 2, y);
    const unsigned long long qlo = Q * d, qhi = __umul64hi(Q, d);
    unsigned long long rlo = 0ull - qlo;
    const unsigned long long rhi = R - qhi - (qlo != 0ull ? 1ull : 0ull);   // remainder < 2d
    if (rhi != 0ull || rlo >= d) {
        ++Q;
        rlo -= d;
    }
    unsigned long long m = Q >> 1;
    if ((Q & 1ull) && (rlo != 0ull || (m & 1ull))) ++m;
    int e = ea - eb + (ge ? 1023 : 1022);
    if (m == (1ull << 53)) {
        m >>= 1;
        ++e;
    }
    if (e < 1 || e > 2046) return div_rn(E - e0, de);   // subnormal or overflowing factor
    return __longlong_as_double((long long)(((unsigned long long)e << 52) | (m & M)));
}

// ---------------------------------------------------------------- logarithm
// ln x for positive normal x: x = 2^e m with m in (sqrt(2)/2, sqrt(2)];
// ln m = 2 atanh(s), s = (m - 1)/(m + 1), as the series
// 2s (1 + s^2/3 + ... + s^20/21) (Abramowitz & Stegun 4.1.28), evaluated by
// Horner's rule from the 1/21 term, each step one fused multiply-add; e ln 2
// with ln 2 split in a high part carrying 21 trailing zero bits (so e * high
// is exact) and a low part.
__device__ __forceinline__ double ln_series(double x) {
    long long b = __double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
    if (m > 0x1.6a09e667f3bcdp+0) {
        m = m * 0.5;
        e = e + 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double q = 0x1.8618618618618p-5;
    q = __fma_rn(z, q, 0x1.af286bca1af28p-5);
    q = __fma_rn(z, q, 0x1.e1e1e1e1e1e1ep-5);
    q = __fma_rn(z, q, 0x1.1111111111111p-4);
    q = __fma_rn(z, q, 0x1.3b13b13b13b14p-4);
    q = __fma_rn(z, q, 0x1.745d1745d1746p-4);
    q = __fma_rn(z, q, 0x1.c71c71c71c71cp-4);
    q = __fma_rn(z, q, 0x1.2492492492492p-3);
    q = __fma_rn(z, q, 0x1.999999999999ap-3);
    q = __fma_rn(z, q, 0x1.5555555555555p-2);
    q = z * q;
    double t = 2.0 * s;
    double lm = __fma_rn(t, q, t);
    double de = (double)e;
    return __fma_rn(de, 0x1.62e42fee00000p-1, __fma_rn(de, 0x1.a39ef35793c76p-33, lm));
}

// a < b for a, b in [+0, +inf]: such values order like their bit patterns,
// so the comparison runs on the integer units, not the scarce binary64 pipe.
__device__ __forceinline__ bool lt_nonneg(double a, double b) {
    return (unsigned long long)__double_as_longlong(a) < (unsigned long long)__double_as_longlong(b);
}

// ---------------------------------------------------------------- lookup
// The lookup stores the running sum after every cum_group<PREC>() entries of
// the material (checkpoints); the collision recomputes at most that many
// terms.  Both precisions keep one checkpoint per four entries: a quarter of
// the stores of keeping every sum, whose write stream (8 bytes a nuclide in
// binary64) evicted the tables from L2; the collision's few recomputed terms
// cost less than those stores.
constexpr int kCumGroup = 4;     // binary32
constexpr int kCumGroup64 = 4;   // binary64: 1 (every sum) or kIlp (one per lock-step group)
template <int PREC>
__host__ __device__ constexpr int cum_group() { return PREC == GBMC_FP64 ? kCumGroup64 : kCumGroup; }
// Bracket search: the largest j in [0, n-2] with grid[j] <= E.  Positive IEEE
// values order like their bit patterns, so every comparison runs on the
// integer pipe (binary64 compares would occupy the scarce FP64 units).
//
// Each nuclide carries a coarse index over its grid's bit patterns
// (key(E) = (bits(E) - bits(E_0)) >> shift, i.e. piecewise-logarithmic
// buckets; idx[b] = number of grid points whose key is below b).  A query in
// bucket b has its bracket in [idx[b] - 1, idx[b+1] - 1]: one index load
// replaces the top levels of the binary search, whose result is unchanged
// because the bracket is unique (the "double indexing" of the CPU codes the
// paper compares against, Sec. 3).

template <class D, class U>
__device__ __forceinline__ void coarse_range(const D& d, const uint32_t* __restrict__ idx,
                                             U eb, int32_t& lo, int32_t& hi) {
    U base = (U)d.base;
    U b = eb >= base ? (U)((eb - base) >> d.shift) : (U)0;
    if (b > (U)(d.nb - 1)) b = (U)(d.nb - 1);
    const uint32_t* ix = idx + d.idx_off + b;
    int32_t s0 = (int32_t)__ldg(ix), s1 = (int32_t)__ldg(ix + 1);
    lo = s0 > 0 ? s0 - 1 : 0;
    if (lo > d.n - 2) lo = d.n - 2;
    hi = s1 < d.n - 1 ? s1 : d.n - 1;
}

template <class U>
__device__ __forceinline__ int32_t bracket_in(const U* __restrict__ g, int32_t lo, int32_t hi, U eb) {
    while (hi - lo > 1) {
        int32_t mid = (lo + hi) >> 1;
        if (__ldg(g + mid) <= eb)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ Desc64 load_desc64(const Desc64* p) {
    Desc64 d;
    const int4* q = reinterpret_cast<const int4*>(p);
    int4 a = __ldg(q), b = __ldg(q + 1);
    memcpy(&d, &a, 16);
    memcpy(reinterpret_cast<char*>(&d) + 16, &b, 16);
    return d;
}

// Lin-lin interpolation on the grid interval k that brackets E:
// f = (E - E_k) / (E_k+1 - E_k) rounded to nearest in binary64, then
// sigma = s_k + f (s_k+1 - s_k) as one fused multiply-add (the interval's
// differences, each rounded, come from its record).
__device__ __forceinline__ double interp64(const Tables& T, int64_t k, double E) {
    const double2* r = reinterpret_cast<const double2*>(T.iv64 + k);
    const double2 a = __ldg(r), b = __ldg(r + 1);   // (de, ds), (s0, y)
    const double f = frac_rn(E, __ldg(T.e64 + k), a.x, (unsigned long long)__double_as_longlong(b.y));
    return __fma_rn(f, a.y, b.x);
}

// Micro cross section at E of the nuclide of material entry q.
__device__ __forceinline__ double micro64(const Tables& T, int32_t q, double E) {
    Desc64 d = load_desc64(T.d64 + q);
    unsigned long long eb = (unsigned long long)__double_as_longlong(E);
    int32_t lo = 0, hi = d.n - 1;
    if (!T.plain) coarse_range(d, T.idx64, eb, lo, hi);
    const unsigned long long* g = reinterpret_cast<const unsigned long long*>(T.e64 + d.off);
    return interp64(T, d.off + bracket_in(g, lo, hi, eb), E);
}

// binary32 tables: the bracket satisfies (double)E_j <= E, found by
// comparing against E rounded toward -inf (exact for binary32 grid values);
// the interpolation runs in binary32 on E rounded to nearest.
//
// The binary32 grid is stored as (E_j, sigma_j) pairs, each nuclide followed
// by sentinel pairs (E = +inf), with a coarse index of about one to two
// points a bucket.  Each bucket carries its own 64-byte window: the pairs
// lo .. lo + 6 of its bracket range [lo, hi] and (lo, hi) itself.  The
// bracket's position is then a count: every window entry at or below E
// precedes it (the grid is sorted, the sentinels and the points past hi are
// above E), so j = lo + count - 1, capped to [0, n - 2].  One 64-byte load
// per nuclide replaces the index load, the bisection probes and the bracket
// loads; a bucket with hi - lo > 6 is searched by bisection instead.
constexpr int kIlp32 = 4;   // nuclides whose windows are in flight together
static_assert(kIlp32 % kCumGroup == 0 && kIlp32 / kCumGroup <= 4,
              "whole checkpoint groups per lock-step group");
constexpr int kPad32 = 8;   // sentinel pairs after each nuclide's grid

__device__ __forceinline__ Desc32 load_desc32(const Desc32* p) {
    Desc32 d;
    const int4* q = reinterpret_cast<const int4*>(p);
    int4 a = __ldg(q), b = __ldg(q + 1);
    memcpy(&d, &a, 16);
    memcpy(reinterpret_cast<char*>(&d) + 16, &b, 16);
    return d;
}

// The bucket window of E.
__device__ __forceinline__ const float4* window_of(const Tables& T, const Desc32& d, uint32_t eb) {
    uint32_t b = eb >= d.base ? (eb - d.base) >> d.shift : 0u;
    if (b > (uint32_t)(d.nb - 1)) b = (uint32_t)(d.nb - 1);
    return T.bw32 + ((int64_t)d.bw_off + b) * 4;
}

// A bucket window (64 bytes, 64-byte aligned in the pool) as four 16-byte
// loads.
__device__ __forceinline__ void load_window(const float4* p, float4* q) {
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = __ldg(p + k);
}

// The bracket's end points (its pair and the next) by bisection of the
// grid's pairs within [lo, hi].
__device__ __forceinline__ void bracket32_bisect(const Tables& T, const Desc32& d, int32_t lo,
                                                 int32_t hi, uint32_t eb, float2& p0, float2& p1) {
    const float2* g = T.es32 + d.off;
    while (hi - lo > 1) {
        int32_t mid = (lo + hi) >> 1;
        if (__float_as_uint(__ldg(&g[mid].x)) <= eb)
            lo = mid;
        else
            hi = mid;
    }
    p0 = __ldg(g + lo);
    p1 = __ldg(g + lo + 1);
}

// The bracket's end points (its pair and the next) from the window w loaded
// from p.
__device__ __forceinline__ void bracket32(const Tables& T, const Desc32& d, const float4* p,
                                          const float4* w, uint32_t eb, float2& p0, float2& p1) {
    int32_t lo = __float_as_int(w[3].z), hi = __float_as_int(w[3].w);
    if (hi - lo <= 6) {
        uint32_t e[7] = {__float_as_uint(w[0].x), __float_as_uint(w[0].z),
                         __float_as_uint(w[1].x), __float_as_uint(w[1].z),
                         __float_as_uint(w[2].x), __float_as_uint(w[2].z),
                         __float_as_uint(w[3].x)};
        int32_t cnt = 0;
#pragma unroll
        for (int k = 0; k < 7; ++k) cnt += e[k] <= eb ? 1 : 0;
        int32_t r = cnt - 1;                        // window position of the bracket
        if (r > d.n - 2 - lo) r = d.n - 2 - lo;
        if (r < 0) r = 0;                           // E below the first grid point
        const float2* pp = reinterpret_cast<const float2*>(p) + r;
        p0 = __ldg(pp);                             // the window's own line: an L1 hit
        p1 = __ldg(pp + 1);
        return;
    }
    bracket32_bisect(T, d, lo, hi, eb, p0, p1);
}

// Short windows (the sparse form of the binary32 search).  When the lanes of
// a warp read distinct windows (tables far beyond L2, particles sparser in
// energy than the grid points) each load instruction costs one L1 wavefront
// per lane and each window at least one 32-byte sector, so this form reads
// exactly one sector per nuclide: a finer index of about two buckets a grid
// point, whose bucket b holds the four pairs lo .. lo + 3 (lo = first point
// of the bucket - 1, clamped to [0, n - 2]; sentinel pairs past the grid),
// with (lo, hi) of the bucket kept apart in br32 for the rare fallback.
// E_lo <= E unless lo = 0, and every entry past point n - 1 is +inf, so with
// c entries of the window at or below E:
//   c < 4: the bracket is lo + c - 1, capped to n - 2 (entry 1 is always a
//          grid point, so the cap is min(2, finite entries - 2)) and at
//          least 0; both end points are in the window's registers;
//   c = 4: E is at or past point lo + 3 < hi (or = hi = n - 1), and the
//          bracket is found by bisection of [min(lo + 3, n - 2), hi].
__device__ __forceinline__ int64_t short_bucket(const Desc32& d, uint32_t eb) {
    uint32_t b = eb >= d.base ? (eb - d.base) >> d.shift : 0u;
    if (b > (uint32_t)(d.nb - 1)) b = (uint32_t)(d.nb - 1);
    return (int64_t)d.bw_off + b;
}

// One short window (32 bytes, 32-byte aligned) as one 256-bit load.
__device__ __forceinline__ void load_short(const float4* p, float (&w)[8]) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(w[0]), "=f"(w[1]), "=f"(w[2]), "=f"(w[3]), "=f"(w[4]), "=f"(w[5]), "=f"(w[6]),
          "=f"(w[7])
        : "l"(p));
}

__device__ __forceinline__ void bracket32_short(const Tables& T, const Desc32& d, int64_t wb,
                                                const float (&w)[8], uint32_t eb, float2& p0,
                                                float2& p1) {
    const uint32_t e0 = __float_as_uint(w[0]), e1 = __float_as_uint(w[2]),
                   e2 = __float_as_uint(w[4]), e3 = __float_as_uint(w[6]);
    const int32_t c = (e0 <= eb) + (e1 <= eb) + (e2 <= eb) + (e3 <= eb);
    if (c == 4) {
        const int2 r = __ldg(T.br32 + wb);
        bracket32_bisect(T, d, min(r.x + 3, d.n - 2), r.y, eb, p0, p1);
        return;
    }
    constexpr uint32_t kInfBits = 0x7f800000u;
    const int32_t fin = 2 + (e2 < kInfBits) + (e3 < kInfBits);   // finite entries
    const int32_t r = max(min(c - 1, fin - 2), 0);
    const float2 a = make_float2(w[0], w[1]), b = make_float2(w[2], w[3]),
                 e = make_float2(w[4], w[5]), f = make_float2(w[6], w[7]);
    p0 = r == 0 ? a : (r == 1 ? b : e);
    p1 = r == 0 ? b : (r == 1 ? e : f);
}

// Micro cross section of material entry q (binary32) at E (SPARSE: on the
// short windows).
template <bool SPARSE = false>
__device__ __forceinline__ float micro32(const Tables& T, int32_t q, double E) {
    Desc32 d = load_desc32((SPARSE ? T.d32s : T.d32) + q);
    uint32_t eb = (uint32_t)__float_as_int(__double2float_rd(E));
    float2 p0, p1;
    if (T.plain) {
        bracket32_bisect(T, d, 0, d.n - 1, eb, p0, p1);
    } else if (SPARSE) {
        const int64_t wb = short_bucket(d, eb);
        float w[8];
        load_short(T.bs32 + 2 * wb, w);
        bracket32_short(T, d, wb, w, eb, p0, p1);
    } else {
        const float4* p = window_of(T, d, eb);
        float4 w[4];
        load_window(p, w);
        bracket32(T, d, p, w, eb, p0, p1);
    }
    float Ef = __double2float_rn(E);
    float f = (Ef - p0.x) / (p1.x - p0.x);
    return p0.y + f * (p1.y - p0.y);
}

// Macroscopic sigma_t, sigma_a of material m: sum over its nuclides in the
// listed order of N_i sigma_i, and of (N_i sigma_i) f_abs,i.  With cum !=
// NULL the running sum of N_i sigma_i after every kCumGroup nuclides (and
// after the last) is stored at cum[g] (the collision picks its nuclide from
// these checkpoints).
//
// The brackets of kIlp consecutive nuclides are searched in lock step (kIlp
// independent chains of dependent loads in flight per thread); the terms are
// then formed and added strictly in the listed order.
constexpr int kIlp = 4;
static_assert(kIlp % 4 == 0, "the running sums are stored in whole 32-byte groups");
static_assert(kCumGroup64 == 1 || kCumGroup64 == kIlp, "binary64 checkpoints: every sum or one per group");

template <class U>
__device__ __forceinline__ void brackets(const Tables& T, const Desc64* dq, const uint32_t* idx,
                                         const U* g, int32_t q, int32_t q1, U eb, int64_t* pos) {
    int32_t lo[kIlp], hi[kIlp];
    const U* gp[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
        lo[u] = 0;
        hi[u] = 1;
        gp[u] = g;
        if (q + u < q1) {
            Desc64 d = load_desc64(dq + q + u);
            gp[u] = g + d.off;
            hi[u] = d.n - 1;
            if (!T.plain) coarse_range(d, idx, eb, lo[u], hi[u]);
        }
    }
    bool more = true;
    while (more) {
        more = false;
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            if (hi[u] - lo[u] > 1) {
                int32_t mid = (lo[u] + hi[u]) >> 1;
                if (__ldg(gp[u] + mid) <= eb)
                    lo[u] = mid;
                else
                    hi[u] = mid;
                more = true;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < kIlp; ++u) pos[u] = (gp[u] - g) + lo[u];
}

// Group mode of the binary64 lookup, for queues too short to hide the
// dependent loads of one lane walking all of a particle's nuclides: a warp
// takes 32 / kGroupLanes particles and kGroupLanes lanes per particle.  Lane
// r of particle p forms the terms of nuclides r, r + kGroupLanes, ... of each
// group of kGroupN nuclides, four searches in lock step, into a shared-memory
// row of the particle; then lane 0 of the particle adds the row's terms in
// the listed order and stores the checkpoints, so every term, sum and
// checkpoint is macro64's.  Rows are kGroupStride doubles apart: the four
// particles of a half-warp start 4 banks apart, so the stores of a half-warp
// (four sub-lanes each) and the adders' reads fall in distinct banks.
constexpr int kGroupLanes = 4;
constexpr int kGroupN = 32;
constexpr int kGroupStride = 36;
static_assert(kGroupN % (kGroupLanes * 4) == 0, "whole lock-step rounds per group");

struct LookupGroupTile {
    double t[(32 / kGroupLanes) * kGroupStride];
};

// The brackets of the (up to kIlp) nuclides q, q + s, q + 2s, ... below q1,
// searched in lock step (as brackets() for consecutive nuclides).
__device__ __forceinline__ void brackets_strided(const Tables& T, int32_t q, int32_t s, int32_t q1,
                                                 unsigned long long eb, int64_t* pos) {
    const unsigned long long* g = reinterpret_cast<const unsigned long long*>(T.e64);
    int32_t lo[kIlp], hi[kIlp];
    const unsigned long long* gp[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
        lo[u] = 0;
        hi[u] = 1;
        gp[u] = g;
        const int32_t qu = q + u * s;
        if (qu < q1) {
            Desc64 d = load_desc64(T.d64 + qu);
            gp[u] = g + d.off;
            hi[u] = d.n - 1;
            if (!T.plain) coarse_range(d, T.idx64, eb, lo[u], hi[u]);
        }
    }
    bool more = true;
    while (more) {
        more = false;
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            if (hi[u] - lo[u] > 1) {
                int32_t mid = (lo[u] + hi[u]) >> 1;
                if (__ldg(gp[u] + mid) <= eb)
                    lo[u] = mid;
                else
                    hi[u] = mid;
                more = true;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < kIlp; ++u) pos[u] = (gp[u] - g) + lo[u];
}

// All 32 lanes call (the loops are warp-uniform); particle p = lane /
// kGroupLanes has material m (nq_max: the most nuclides of the warp's
// particles), valid marks the lanes of real entries, cum the particle's
// checkpoint row (read by its lane 0 only).
template <bool SA>
__device__ __forceinline__ void macro64_group(const Tables& T, int32_t m, double E, bool valid,
                                              int32_t nq_max, LookupGroupTile& sm, double* cum,
                                              double& st, double& sa) {
    const int lane = threadIdx.x & 31;
    const int p = lane / kGroupLanes, r = lane % kGroupLanes;
    const int32_t q0 = valid ? __ldg(T.mat_off + m) : 0;
    const int32_t nq = valid ? __ldg(T.mat_off + m + 1) - q0 : 0;
    const unsigned long long eb = (unsigned long long)__double_as_longlong(E);
    double at = 0.0, aa = 0.0;
    double2 pend = make_double2(0.0, 0.0);
    double* row = sm.t + p * kGroupStride;
    for (int32_t g0 = 0; g0 < nq_max; g0 += kGroupN) {
        const int32_t ge = min(nq, g0 + kGroupN);   // this particle's nuclides end in the group
#pragma unroll
        for (int k = 0; k < kGroupN / (kGroupLanes * kIlp); ++k) {
            const int32_t a0 = g0 + r + k * kGroupLanes * kIlp;   // entry of the first of four
            if (a0 < ge) {
                int64_t pos[kIlp];
                brackets_strided(T, q0 + a0, kGroupLanes, q0 + ge, eb, pos);
#pragma unroll
                for (int u = 0; u < kIlp; ++u) {
                    const int32_t a = a0 + u * kGroupLanes;
                    if (a < ge) row[a - g0] = interp64(T, pos[u], E);
                }
            }
        }
        __syncwarp();
        if (r == 0) {
            for (int32_t a = g0; a < ge; ++a) {
                const double sig = row[a - g0];
                const double N = __ldg(T.density + q0 + a);
                at = __fma_rn(N, sig, at);
                if (SA) aa = __fma_rn(N * __ldg(T.f_abs + __ldg(T.nuc_id + q0 + a)), sig, aa);
                if (cum && ((a & 3) == 3 || a == nq - 1)) {
                    const int32_t gq = a >> 2;
                    if (gq & 1) pend.y = at; else pend.x = at;
                    if ((gq & 1) || a == nq - 1) reinterpret_cast<double2*>(cum)[gq >> 1] = pend;
                }
            }
        }
        __syncwarp();
    }
    st = at;
    sa = aa;
}

// SA = false skips Sigma_a (sa is then 0): the transport needs it only for
// the absorption-rate tally.
template <bool SA = true>
__device__ __forceinline__ void macro64(const Tables& T, int32_t m, double E, double& st,
                                        double& sa, double* cum = nullptr) {
    double at = 0.0, aa = 0.0;
    int32_t q0 = __ldg(T.mat_off + m), q1 = __ldg(T.mat_off + m + 1);
    const unsigned long long* g = reinterpret_cast<const unsigned long long*>(T.e64);
    unsigned long long eb = (unsigned long long)__double_as_longlong(E);
    double2 pend = make_double2(0.0, 0.0);   // checkpoint not yet stored
    for (int32_t q = q0; q < q1; q += kIlp) {
        int64_t pos[kIlp];
        double run[kIlp];
        brackets(T, T.d64, T.idx64, g, q, q1, eb, pos);
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            if (q + u < q1) {
                double sig = interp64(T, pos[u], E);
                double N = __ldg(T.density + q + u);
                at = __fma_rn(N, sig, at);
                if (SA) aa = __fma_rn(N * __ldg(T.f_abs + __ldg(T.nuc_id + q + u)), sig, aa);
            }
            run[u] = at;
        }
        if (cum) {
            if (kCumGroup64 == 1) {
                // every running sum; the row holds the material's count
                // rounded up to kIlp, so whole groups are written
                double2* d = reinterpret_cast<double2*>(cum + (q - q0));
#pragma unroll
                for (int j = 0; j < kIlp; j += 2) d[j / 2] = make_double2(run[j], run[j + 1]);
            } else {
                // one checkpoint per group, two groups to a 16-byte store (the
                // row is rounded up to an even count)
                int32_t gq = (q - q0) / kIlp;
                if (gq & 1) pend.y = run[kIlp - 1]; else pend.x = run[kIlp - 1];
                if ((gq & 1) || q + kIlp >= q1) reinterpret_cast<double2*>(cum)[gq >> 1] = pend;
            }
        }
    }
    st = at;
    sa = aa;
}

// Tile mode of the binary64 macroscopic lookup, for 32 queue entries of one
// material taken in (material, energy) order by one warp (all 32 lanes call;
// lanes >= nv hold no entry).  Instead of every lane walking the material's
// nuclides for its own particle (a chain of dependent loads per nuclide:
// descriptor, coarse index, probe, interval), each lane takes one nuclide
// over a run of consecutive particles: sorted energies mostly share the
// bracket of the previous particle, which the lane keeps in registers, so
// most micro lookups load nothing.  The terms N_i sigma_i(E_p) go through a
// shared-memory tile (row = nuclide, column = particle), and each lane then
// adds its particle's terms in the listed order: every term, running sum and
// checkpoint is the one macro64 forms.
//
// Nuclides are taken kTileG at a time.  With gn nuclides in a group and gp
// the power of two at or above gn, lane l takes nuclide l % gp (if < gn) over
// particles (l / gp) gp .. + gp - 1.  Rows are kTileStride doubles apart:
// for every gp the 16 lanes of each half-warp then store to distinct 8-byte
// banks, and the column reads of the sums are contiguous.
constexpr int kTileG = 8;
constexpr int kTileStride = 33;
static_assert(kTileG == 8, "the lane mapping covers groups of at most 8 nuclides");
static_assert(kCumGroup64 == 4, "tile checkpoints: one per four entries, two to a 16-byte store");

// A chunk takes the tile only when its energies are close: over at most
// 2^44 units of their binary64 bit patterns (about 0.3% relative), so that a
// run of consecutive particles mostly shares each nuclide's bracket.  A
// chunk spread wider (the sparse tail of a sorted queue) would miss at
// almost every particle, and each miss in the tile is a dependent search
// that the lane's other particles wait behind; such chunks take the
// per-particle lookup, whose lanes search their nuclides in lock step.
constexpr unsigned long long kTileSpan = 1ull << 44;

// All 32 lanes call; E of lanes without an entry is ignored (valid false).
__device__ __forceinline__ bool tile_span_ok(double E, bool valid) {
    unsigned long long b = (unsigned long long)__double_as_longlong(E);
    unsigned long long lo = valid ? b : ~0ull, hi = valid ? b : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    return hi - lo < kTileSpan;
}

struct LookupTile {
    double t[kTileG * kTileStride];   // terms of the group, row = nuclide, column = particle
    double E[32];                     // the chunk's energies
};

template <bool SA>
__device__ __forceinline__ void macro64_tile(const Tables& T, int32_t m, int nv, double E_lane,
                                             LookupTile& sm, double* cum, double& st,
                                             double& sa) {
    const int lane = threadIdx.x & 31;
    sm.E[lane] = E_lane;
    __syncwarp();
    const int32_t q0 = __ldg(T.mat_off + m), nq = __ldg(T.mat_off + m + 1) - q0;
    const unsigned long long* g = reinterpret_cast<const unsigned long long*>(T.e64);
    double at = 0.0, aa = 0.0;
    double2 pend = make_double2(0.0, 0.0);   // checkpoint pair not yet stored
    for (int32_t g0 = 0; g0 < nq; g0 += kTileG) {
        const int gn = min(kTileG, nq - g0);
        const int gp = gn > 4 ? 8 : (gn > 2 ? 4 : gn);
        const int i = lane & (gp - 1), s = lane / gp;
        if (i < gn) {
            const int32_t q = q0 + g0 + i;
            const Desc64 d = load_desc64(T.d64 + q);
            const unsigned long long* gg = g + d.off;
            int32_t k = -1;                               // bracket held in registers
            unsigned long long elo = 0ull, ehi = 0ull;    // bits of E_k, E_k+1
            double2 r0 = make_double2(0.0, 0.0), r1 = make_double2(0.0, 0.0);   // (de, ds), (s0, y)
            for (int j = 0; j < gp; ++j) {
                const int p = s * gp + j;
                if (p >= nv) break;
                const double E = sm.E[p];
                const unsigned long long eb = (unsigned long long)__double_as_longlong(E);
                // the held bracket is E's if it is the largest j <= n-2 with E_j <= E
                const bool hit = k >= 0 && (eb >= elo || k == 0) && (eb < ehi || k == d.n - 2);
                if (!hit) {
                    int32_t lo = 0, hi = d.n - 1;
                    if (!T.plain) coarse_range(d, T.idx64, eb, lo, hi);
                    k = bracket_in(gg, lo, hi, eb);
                    elo = __ldg(gg + k);
                    ehi = __ldg(gg + k + 1);
                    const double2* rp = reinterpret_cast<const double2*>(T.iv64 + d.off + k);
                    r0 = __ldg(rp);
                    r1 = __ldg(rp + 1);
                }
                const double f = frac_rn(E, __longlong_as_double((long long)elo), r0.x,
                                         (unsigned long long)__double_as_longlong(r1.y));
                sm.t[i * kTileStride + p] = __fma_rn(f, r0.y, r1.x);
            }
        }
        __syncwarp();
        if (lane < nv) {
            for (int ii = 0; ii < gn; ++ii) {
                const double sig = sm.t[ii * kTileStride + lane];
                const int32_t a = g0 + ii;   // entry index within the material
                const double N = __ldg(T.density + q0 + a);
                at = __fma_rn(N, sig, at);
                if (SA) aa = __fma_rn(N * __ldg(T.f_abs + __ldg(T.nuc_id + q0 + a)), sig, aa);
                if (cum && ((a & 3) == 3 || a == nq - 1)) {
                    const int32_t gq = a >> 2;
                    if (gq & 1) pend.y = at; else pend.x = at;
                    if ((gq & 1) || a == nq - 1) reinterpret_cast<double2*>(cum)[gq >> 1] = pend;
                }
            }
        }
        __syncwarp();
    }
    st = at;
    sa = aa;
}

template <bool SA = true, bool SPARSE = false>
__device__ __forceinline__ void macro32(const Tables& T, int32_t m, double E, double& st,
                                        double& sa, float* cum = nullptr) {
    float at = 0.0f, aa = 0.0f;
    int32_t q0 = __ldg(T.mat_off + m), q1 = __ldg(T.mat_off + m + 1);
    uint32_t eb = (uint32_t)__float_as_int(__double2float_rd(E));
    float Ef = __double2float_rn(E);
    float4 pend = make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // checkpoints not yet stored
    for (int32_t q = q0; q < q1; q += kIlp32) {
        Desc32 d[kIlp32];
#pragma unroll
        for (int u = 0; u < kIlp32; ++u)
            d[u] = load_desc32((SPARSE ? T.d32s : T.d32) + (q + u < q1 ? q + u : q));
        float2 p0[kIlp32], p1[kIlp32];
        if (T.plain) {
            // plain binary search of each grid, the group's searches in lock step
            int32_t lo[kIlp32], hi[kIlp32];
#pragma unroll
            for (int u = 0; u < kIlp32; ++u) {
                lo[u] = 0;
                hi[u] = d[u].n - 1;
            }
            bool more = true;
            while (more) {
                more = false;
#pragma unroll
                for (int u = 0; u < kIlp32; ++u) {
                    if (hi[u] - lo[u] > 1) {
                        int32_t mid = (lo[u] + hi[u]) >> 1;
                        if (__float_as_uint(__ldg(&T.es32[d[u].off + mid].x)) <= eb)
                            lo[u] = mid;
                        else
                            hi[u] = mid;
                        more = true;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kIlp32; ++u) {
                p0[u] = __ldg(T.es32 + d[u].off + lo[u]);
                p1[u] = __ldg(T.es32 + d[u].off + lo[u] + 1);
            }
        } else if (SPARSE) {
            int64_t wb[kIlp32];
#pragma unroll
            for (int u = 0; u < kIlp32; ++u) wb[u] = short_bucket(d[u], eb);
            float w[kIlp32][8];
#pragma unroll
            for (int u = 0; u < kIlp32; ++u) load_short(T.bs32 + 2 * wb[u], w[u]);
#pragma unroll
            for (int u = 0; u < kIlp32; ++u) bracket32_short(T, d[u], wb[u], w[u], eb, p0[u], p1[u]);
        } else {
            const float4* pw[kIlp32];
#pragma unroll
            for (int u = 0; u < kIlp32; ++u) pw[u] = window_of(T, d[u], eb);
            float4 w[kIlp32][4];
#pragma unroll
            for (int u = 0; u < kIlp32; ++u) load_window(pw[u], w[u]);
#pragma unroll
            for (int u = 0; u < kIlp32; ++u) bracket32(T, d[u], pw[u], w[u], eb, p0[u], p1[u]);
        }
        float run[kIlp32];
#pragma unroll
        for (int u = 0; u < kIlp32; ++u) {
            if (q + u < q1) {
                float f = (Ef - p0[u].x) / (p1[u].x - p0[u].x);
                float sig = p0[u].y + f * (p1[u].y - p0[u].y);
                float t = d[u].density * sig;
                at = at + t;
                if (SA) aa = aa + t * d[u].f_abs;
            }
            run[u] = at;
        }
        if (cum) {
            // the group's checkpoints (one per kCumGroup entries) gathered
            // into whole float4s, each leaving as one 16-byte store (the rows
            // are padded to whole float4s)
            constexpr int kPer = kIlp32 / kCumGroup;   // checkpoints per lock-step group
            constexpr int kGroups = 4 / kPer;          // lock-step groups per float4
            int32_t g = (q - q0) / kIlp32;
            int k = g % kGroups;
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                float v = run[(j + 1) * kCumGroup - 1];
                int e = k * kPer + j;
                pend.x = e == 0 ? v : pend.x;
                pend.y = e == 1 ? v : pend.y;
                pend.z = e == 2 ? v : pend.z;
                pend.w = e == 3 ? v : pend.w;
            }
            if (k == kGroups - 1 || q + kIlp32 >= q1) reinterpret_cast<float4*>(cum)[g / kGroups] = pend;
        }
    }
    st = (double)at;
    sa = (double)aa;
}

// The same macroscopic sums for ONE particle computed by a whole warp (all
// 32 lanes call with the same m and E): lane l forms the terms of nuclides
// l, l+32, ... in parallel, then every lane folds the terms in the listed
// order with shuffles, so the sums are bit-identical to macro64/macro32.
// Used when the lookup queue is too short to keep the GPU busy with one
// particle per thread (the per-particle nuclide loop is then a long serial
// latency chain).
template <int PREC, bool SA = true, bool SPARSE = false>
__device__ __forceinline__ void macro_warp(const Tables& T, int32_t m, double E, double& st,
                                           double& sa, void* cum, int64_t stride) {
    const unsigned full = 0xffffffffu;
    int lane = threadIdx.x & 31;
    int32_t q0 = __ldg(T.mat_off + m), q1 = __ldg(T.mat_off + m + 1);
    if (PREC == GBMC_FP64) {
        double at = 0.0, aa = 0.0;
        for (int32_t c = q0; c < q1; c += 32) {
            double sig = 0.0, N = 0.0, Na = 0.0;
            if (c + lane < q1) {
                N = __ldg(T.density + c + lane);
                sig = micro64(T, c + lane, E);
                if (SA) Na = N * __ldg(T.f_abs + __ldg(T.nuc_id + c + lane));
            }
            int32_t kmax = q1 - c < 32 ? q1 - c : 32;
            for (int k = 0; k < kmax; ++k) {
                const double sk = __shfl_sync(full, sig, k);
                at = __fma_rn(__shfl_sync(full, N, k), sk, at);
                if (SA) aa = __fma_rn(__shfl_sync(full, Na, k), sk, aa);
                if (cum && lane == k &&
                    ((c + k - q0) % kCumGroup64 == kCumGroup64 - 1 || c + k == q1 - 1))
                    ((double*)cum)[(int64_t)((c + k - q0) / kCumGroup64) * stride] = at;
            }
        }
        st = at;
        sa = aa;
    } else {
        float at = 0.0f, aa = 0.0f;
        for (int32_t c = q0; c < q1; c += 32) {
            float t = 0.0f, p = 0.0f;
            if (c + lane < q1) {
                const Desc32* dq = T.d32 + c + lane;
                t = __ldg(&dq->density) * micro32<SPARSE>(T, c + lane, E);
                if (SA) p = t * __ldg(&dq->f_abs);
            }
            int32_t kmax = q1 - c < 32 ? q1 - c : 32;
            for (int k = 0; k < kmax; ++k) {
                at = at + __shfl_sync(full, t, k);
                if (SA) aa = aa + __shfl_sync(full, p, k);
                if (cum && lane == k && ((c + k - q0) % kCumGroup == kCumGroup - 1 || c + k == q1 - 1))
                    ((float*)cum)[(int64_t)((c + k - q0) / kCumGroup) * stride] = at;
            }
        }
        st = (double)at;
        sa = (double)aa;
    }
}

// Collision nuclide: first nuclide (listed order) whose running sum of
// N_i sigma_i exceeds target = xi Sigma_t, with the running sums formed as
// in the macroscopic lookup; if rounding leaves none, the last nuclide with
// a positive term (binary64: N_i > 0 and sigma_i > 0; binary32: the rounded
// product), the first listed one if no term is positive.
__device__ __forceinline__ int32_t pick_nuclide(const Tables& T, int precision, int32_t m,
                                                double E, double target) {
    int32_t last = -1;
    int32_t q0 = __ldg(T.mat_off + m), q1 = __ldg(T.mat_off + m + 1);
    if (precision == GBMC_FP64) {
        double cum = 0.0;
        for (int32_t q = q0; q < q1; ++q) {
            int32_t i = __ldg(T.nuc_id + q);
            double N = __ldg(T.density + q);
            double sig = micro64(T, q, E);
            cum = __fma_rn(N, sig, cum);
            if (N > 0.0 && sig > 0.0) last = i;
            if (lt_nonneg(target, cum)) return i;
        }
    } else {
        float cum = 0.0f;
        for (int32_t q = q0; q < q1; ++q) {
            int32_t i = __ldg(T.nuc_id + q);
            float t = __ldg(&T.d32[q].density) * micro32(T, q, E);
            cum = cum + t;
            if (t > 0.0f) last = i;
            if (lt_nonneg(target, (double)cum)) return i;
        }
    }
    return last >= 0 ? last : __ldg(T.nuc_id + q0);
}

// The same choice from the lookup's checkpoints (cum[g * stride]: the
// running sum after entry G g + G - 1, G = cum_group<PREC>(), non-decreasing in g):
// the first group whose checkpoint exceeds the target holds the nuclide; its
// terms are recomputed exactly as the lookup formed them and added to the
// previous checkpoint in the listed order, so every running sum, and hence
// the choice, is the one the full sums give.  Returns -1 when no sum exceeds
// the target (then pick_nuclide decides).
template <int PREC>
__device__ __forceinline__ int32_t pick_from_sums(const Tables& T, int32_t m, const void* cum,
                                                  int64_t stride, double E, double target) {
    constexpr int G = cum_group<PREC>();
    int32_t q0 = __ldg(T.mat_off + m), nq = __ldg(T.mat_off + m + 1) - q0;
    int32_t ng = (nq + G - 1) / G;
    const double* c64 = (const double*)cum;
    const float* c32 = (const float*)cum;
    int32_t lo = 0, hi = ng;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        double v = PREC == GBMC_FP64 ? c64[(int64_t)mid * stride] : (double)c32[(int64_t)mid * stride];
        if (lt_nonneg(target, v))
            hi = mid;
        else
            lo = mid + 1;
    }
    if (lo >= ng) return -1;
    if (G == 1) return __ldg(T.nuc_id + q0 + lo);   // every sum stored: no recomputation
    int32_t k0 = lo * G, k1 = min(k0 + G, nq);
    if (PREC == GBMC_FP64) {
        double at = lo > 0 ? c64[(int64_t)(lo - 1) * stride] : 0.0;
        for (int32_t k = k0; k < k1; ++k) {
            int32_t i = __ldg(T.nuc_id + q0 + k);
            at = __fma_rn(__ldg(T.density + q0 + k), micro64(T, q0 + k, E), at);
            if (lt_nonneg(target, at)) return i;
        }
    } else {
        float at = lo > 0 ? c32[(int64_t)(lo - 1) * stride] : 0.0f;
        for (int32_t k = k0; k < k1; ++k) {
            float t = __ldg(&T.d32[q0 + k].density) * micro32(T, q0 + k, E);
            at = at + t;
            if (lt_nonneg(target, (double)at)) return __ldg(T.nuc_id + q0 + k);
        }
    }
    return -1;   // not reached: the group's checkpoint exceeds the target
}

// Tally energy bin: largest b in [0, n_bins-1] with edges[b] <= E.
__device__ __forceinline__ int32_t energy_bin(const Tables& T, double E) {
    return bracket_in(reinterpret_cast<const unsigned long long*>(T.edges), 0, T.n_bins,
                      (unsigned long long)__double_as_longlong(E));
}

// ---------------------------------------------------------------- geometry
enum : uint8_t { kSurfNone = 0, kSurfCyl = 1, kSurfX = 2, kSurfY = 3, kSurfZ = 4 };

// ---------------------------------------------------------------- screened distances
// A flight needs only the smallest of its candidate distances (distance to
// collision, and the cylinder, x, y and z surfaces of its cell) and that
// one's value; each candidate is one correctly rounded binary64 expression.
// Every candidate is first estimated in binary32 from its binary64 operands
// truncated to 24 significant bits: with no cancellation in the estimate
// (each sum below adds terms of one sign), it lies within 3 * 2^-23
// relative of the binary64 value (three truncations or roundings of 2^-23
// or 2^-24), and its span widens that to 2^-16.  Only a candidate whose span
// leaves it a possible minimum is evaluated in binary64, so the distance
// chosen, its value and the tie order are exactly those of evaluating every
// candidate in binary64, at a fraction of the binary64 divisions, square
// roots and logarithms (the scarce units of this GPU).

// binary64 -> binary32 by truncating the significand (relative error below
// 2^-23, sign kept); ok is false outside the normal binary32 range (zero is
// exact).  Integer instructions only.
__device__ __forceinline__ float trunc32(double x, bool& ok) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    unsigned hi = (unsigned)(b >> 32);
    unsigned e = (hi >> 20) & 0x7ffu;
    bool zero = (b << 1) == 0ull;
    ok = zero || (e >= 897u && e <= 1150u);
    unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
    return zero ? 0.0f : __uint_as_float(f);
}

// Bounds [lo, hi] of a non-negative distance (a negative value counts as
// zero) from its binary32 estimate a.
struct Span {
    float lo, hi;
};
constexpr float kSpanLo = 1.0f - 0x1p-16f, kSpanHi = 1.0f + 0x1p-16f;

__device__ __forceinline__ Span span_of(float a, bool ok) {
    const float inf = __int_as_float(0x7f800000);
    if (!ok || !(a == a)) return {0.0f, inf};     // no estimate: anything
    if (a <= 0.0f) return {0.0f, 1e-37f};          // zero, or below binary32's range
    if (a == inf) return {1e38f, inf};             // beyond binary32's range
    return {fmaxf(a * kSpanLo - 1e-37f, 0.0f), a * kSpanHi + 1e-37f};
}

__device__ __forceinline__ Span span_never() {
    const float inf = __int_as_float(0x7f800000);
    return {inf, inf};
}

// Sign tests on the bit pattern (no binary64 compare).
__device__ __forceinline__ bool is_neg(double x) {
    long long b = __double_as_longlong(x);
    return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool is_pos(double x) {
    long long b = __double_as_longlong(x);
    return b > 0;
}
// -x (a reflection), as a flip of the sign bit.
__device__ __forceinline__ double flip_sign(double x) {
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(x) ^
                                            0x8000000000000000ull));
}

// Cylinder of radius r about the pin axis, from (dx, dy) relative to the
// axis along (u, v): a d^2 + 2 k d + c = 0 with a = u^2 + v^2,
// k = dx u + dy v, c = dx^2 + dy^2 - r^2, D = k^2 - a c, each root in its
// cancellation-free form.  Inside: the far root ((sqrt D - k) / a for
// k <= 0, -c / (k + sqrt D) otherwise; D < 0 counts as 0); outside: the near
// root c / (sqrt D - k) if the path approaches (k < 0) and meets the
// cylinder (D >= 0), else none.
struct Cyl {
    double a, k, c, D;
    int kind;   // 0: no crossing, 1: (sD - k) / a, 2: -c / (k + sD), 3: c / (sD - k)
};

// a = u^2 + v^2 (one fused multiply-add) and r2 = r * r come from the
// caller (they change with the direction and the problem only); k = dx u +
// dy v, dx^2 + dy^2 and D = k^2 - a c are fused multiply-adds too.
__device__ __forceinline__ Cyl cylinder_of(double dx, double dy, double u, double v, double a,
                                           double r2, bool inside) {
    Cyl q;
    q.a = a;
    q.k = __fma_rn(dx, u, dy * v);
    q.c = __fma_rn(dx, dx, dy * dy) - r2;
    q.D = __fma_rn(q.k, q.k, -(q.a * q.c));
    bool a0 = (__double_as_longlong(q.a) << 1) == 0;
    if (inside) {
        if (is_neg(q.D)) q.D = 0.0;
        q.kind = a0 ? 0 : (is_pos(q.k) ? 2 : 1);
    } else {
        q.kind = (a0 || !is_neg(q.k) || is_neg(q.D)) ? 0 : 3;
    }
    return q;
}

__device__ __forceinline__ Span cylinder_span(const Cyl& q) {
    if (q.kind == 0) return span_never();
    bool oa, ok, oc, oD;
    float a = trunc32(q.a, oa), k = trunc32(q.k, ok), c = trunc32(q.c, oc);
    float sD = sqrtf(trunc32(q.D, oD));
    float e = q.kind == 1 ? (sD - k) / a : q.kind == 2 ? (0.0f - c) / (k + sD) : c / (sD - k);
    bool good = ok && oD && (q.kind == 1 ? oa : oc);
    return span_of(e, good);
}

__device__ __forceinline__ double cylinder_exact(const Cyl& q) {
    if (q.kind == 0) return CUDART_INF;
    double sD = sqrt(q.D);
    if (q.kind == 1) return (sD - q.k) / q.a;
    if (q.kind == 2) return (0.0 - q.c) / (q.k + sD);
    return q.c / (sD - q.k);
}

// Plane pair [lo, hi] crossed along direction cosine u from x: the
// numerator (hi - x for u > 0, lo - x for u < 0) and its quotient by u.
__device__ __forceinline__ Span plane_span(double num, double u) {
    if ((__double_as_longlong(u) << 1) == 0) return span_never();
    bool on, ou;
    float n = trunc32(num, on), d = trunc32(u, ou);
    return span_of(n / d, on && ou);
}

__device__ __forceinline__ double plane_exact(double num, double u) {
    if ((__double_as_longlong(u) << 1) == 0) return CUDART_INF;
    return num / u;
}

// Distance to collision -ln(xi) / Sigma_t estimated with the binary32
// logarithm (within 2^-23 absolute from the truncated xi, plus one ulp):
// the span takes 2^-20 absolute on the logarithm, then the relative margin.
__device__ __forceinline__ Span collision_span(double xi, double st) {
    bool ox, os;
    float l = 0.0f - logf(trunc32(xi, ox));
    float s = trunc32(st, os);
    if (!(ox && os) || !(s > 0.0f)) return span_of(0.0f, false);
    const float inf = __int_as_float(0x7f800000);
    float lo = fmaxf(l - 0x1p-20f, 0.0f) / s;
    float hi = (l + 0x1p-20f) / s;
    Span sp;
    sp.lo = lo == inf ? 1e38f : fmaxf(lo * kSpanLo - 1e-37f, 0.0f);
    sp.hi = hi * kSpanHi + 1e-37f;
    return sp;
}

// Elastic scatter off a nucleus at rest, isotropic in the centre-of-mass
// frame: E' = E (A^2 + 2 A mu + 1) / (A + 1)^2,
// mu_lab = (1 + A mu) / sqrt(A^2 + 2 A mu + 1); A^2 + 2 A mu and 1 + A mu
// are fused multiply-adds.
__device__ __forceinline__ void elastic(double E, double A, double mu, double& E_out,
                                        double& mu_lab) {
    double t1 = __fma_rn(2.0 * A, mu, A * A) + 1.0;
    double ap1 = A + 1.0;
    E_out = (E * t1) / (ap1 * ap1);
    mu_lab = __fma_rn(A, mu, 1.0) / sqrt(t1);
}

// Rotate (u, v, w) by polar cosine mu and azimuth (cos phi, sin phi); each
// product-plus-term below is one fused multiply-add.
__device__ __forceinline__ void rotate(double& u, double& v, double& w, double mu, double cphi,
                                       double sphi) {
    double m2 = __fma_rn(-mu, mu, 1.0);
    if (is_neg(m2)) m2 = 0.0;
    double st = sqrt(m2);
    double u0 = u, v0 = v, w0 = w;
    const unsigned long long aw = (unsigned long long)__double_as_longlong(w0) & 0x7FFFFFFFFFFFFFFFull;
    if (aw < (unsigned long long)__double_as_longlong(0.9999999999)) {   // |w| < 1 - 1e-10
        double q = sqrt(__fma_rn(-w0, w0, 1.0));
        u = __fma_rn(mu, u0, (st * __fma_rn(u0 * w0, cphi, -(v0 * sphi))) / q);
        v = __fma_rn(mu, v0, (st * __fma_rn(v0 * w0, cphi, u0 * sphi)) / q);
        w = __fma_rn(mu, w0, -((st * q) * cphi));
    } else {
        u = st * cphi;
        v = st * sphi;
        w = is_pos(w0) ? mu : -mu;
    }
}

// Marsaglia (1972): (a, b) uniform in the unit disk by rejection; returns
// s = a^2 + b^2 in (0, 1), one fused multiply-add.  2 xi - 1 as a fused
// multiply-add equals the separately rounded form: 2 xi is exact.
__device__ __forceinline__ double disk_pair(Stream& r, double& a, double& b) {
    for (;;) {
        a = __fma_rn(2.0, r.next(), -1.0);
        b = __fma_rn(2.0, r.next(), -1.0);
        double s = __fma_rn(a, a, b * b);   // >= +0: 0 < s < 1 on its bits
        const unsigned long long sb = (unsigned long long)__double_as_longlong(s);
        if (sb != 0ull && sb < 0x3FF0000000000000ull) return s;
    }
}

}  // namespace gbmc

