// Event kernels of the transport loop (Sec. 2, "Event-Based Parallelism"):
// every kernel processes the whole queue of one event type and routes each
// particle to the queue of its next event.  Grids are fixed (a multiple of
// the SM count) and read their queue lengths from device memory, so one
// iteration is a fixed sequence of launches that a CUDA graph replays under
// a device-evaluated while-condition: no host round trip per event.
//
// Iteration: plan -> source (refill, Sec. 2 "In-Flight Particles") ->
// sort (Sec. 2 "Sorting") -> lookup -> ray trace (flights and the surface
// crossings that keep the material) -> collision (which first finishes the
// flight that reached it).  Once the source is exhausted and few particles
// remain, a tail kernel finishes them one warp per particle.
#include "device.cuh"
#include "launch.h"

namespace gbmc {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Append `slot` to queue q (length *count) for every lane with pred set; one
// atomic per warp.  Called by all 32 lanes of the warp.
__device__ __forceinline__ void warp_append(int32_t* q, int32_t* count, int32_t slot, bool pred) {
    unsigned m = __ballot_sync(kFull, pred);
    if (m == 0) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (pred) q[base + __popc(m & lanemask_lt())] = slot;
}

// ---------------------------------------------------------------- sort keys at the append
// Every kernel that appends a particle to a lookup queue already holds its
// energy and material: it writes the particle's sort key beside the entry
// and counts it in that queue's bucket histogram, so the sort needs no pass
// over the particle records of its own.
__device__ __forceinline__ uint32_t sort_key(const Params& P, double E, int32_t m);

__device__ __forceinline__ void warp_count(uint32_t* hist, uint32_t key, bool valid) {
    unsigned peers = __match_any_sync(kFull, valid ? key : 0xffffffffu);
    int lane = threadIdx.x & 31;
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&hist[key], (uint32_t)__popc(peers));
}

// warp_count that also returns the lane's rank among the entries of its
// bucket counted so far (the sort's scatter then needs no atomics).
__device__ __forceinline__ uint32_t warp_count_rank(uint32_t* hist, uint32_t key, bool valid) {
    unsigned peers = __match_any_sync(kFull, valid ? key : 0xffffffffu);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    uint32_t base = 0u;
    if (valid && lane == leader) base = atomicAdd(&hist[key], (uint32_t)__popc(peers));
    base = __shfl_sync(kFull, base, leader);
    return base + (uint32_t)__popc(peers & lanemask_lt());
}

// warp_append into lookup queue b with the entry's sort key (all 32 lanes).
__device__ __forceinline__ void lookup_append(const Params& P, int b, int32_t* count, int32_t slot,
                                              bool pred, double E, int32_t m) {
    unsigned msk = __ballot_sync(kFull, pred);
    if (msk == 0) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(msk) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(msk));
    base = __shfl_sync(kFull, base, leader);
    uint32_t key = 0;
    int pos = base + __popc(msk & lanemask_lt());
    if (pred) {
        P.Q.lq[b][pos] = slot;
        if (P.sort) {
            key = sort_key(P, E, m);
            P.Q.keys[b][pos] = key;
        }
    }
    if (P.sort) {
        uint32_t rk = warp_count_rank(P.Q.hist[b], key, pred);
        if (pred) P.Q.rank[b][pos] = rk;
    }
}

// ---------------------------------------------------------------- scalar tallies
// Per-block accumulation of the scalar tallies in shared memory (one entry
// per problem of the run and tally kind), flushed with one global atomic per
// entry at the end of the kernel into the problem's tally slot; problems
// beyond the shared table go straight to global memory.
struct BlockScalars {
    double* w;
    unsigned long long* c;
    const DevProblem* probs;
    int nslot;

    __device__ __forceinline__ void init(double* sw, unsigned long long* sc, int n_prob,
                                         const DevProblem* pr) {
        w = sw;
        c = sc;
        probs = pr;
        nslot = min(n_prob, kMaxSharedProblems);
        for (int e = threadIdx.x; e < nslot * GBMC_NSCAL; e += blockDim.x) {
            w[e] = 0.0;
            c[e] = 0ull;
        }
        __syncthreads();
    }
    // all 32 lanes call; lanes with pred score weight wt and count k into
    // (prob, kind).  When the scoring lanes share one problem (the common
    // case: queues are grouped by material) the warp sums first and one lane
    // adds; binary64 adds to one shared word from many lanes would retry
    // compare-and-swap loops, each retry a binary64 add.
    __device__ __forceinline__ void add(const Tallies& Y, bool pred, int prob, int kind, double wt,
                                        unsigned long long k) {
        unsigned vm = __ballot_sync(kFull, pred);
        if (vm == 0) return;
        unsigned peers = __match_any_sync(kFull, pred ? prob : -1);
        int lane = threadIdx.x & 31;
        int leader = __ffs(vm) - 1;
        if (__shfl_sync(kFull, peers, leader) == vm) {
            double s = pred ? wt : 0.0;
            unsigned long long ks = pred ? k : 0ull;
            for (int o = 16; o > 0; o >>= 1) {
                s += __shfl_xor_sync(kFull, s, o);
                ks += __shfl_xor_sync(kFull, ks, o);
            }
            if (lane == leader) put(Y, prob, kind, s, ks);
        } else if (pred) {
            put(Y, prob, kind, wt, k);
        }
    }
    __device__ __forceinline__ void put(const Tallies& Y, int prob, int kind, double s,
                                        unsigned long long k) {
        if (prob < nslot) {
            atomicAdd(&w[prob * GBMC_NSCAL + kind], s);
            atomicAdd(&c[prob * GBMC_NSCAL + kind], k);
        } else {
            int64_t g = (int64_t)probs[prob].slot * GBMC_NSCAL + kind;
            atomicAdd(&Y.weights[g], s);
            atomicAdd(&Y.counts[g], k);
        }
    }
    __device__ __forceinline__ void flush(const Tallies& Y) {
        __syncthreads();
        for (int e = threadIdx.x; e < nslot * GBMC_NSCAL; e += blockDim.x) {
            if (c[e]) {
                int64_t g = (int64_t)probs[e / GBMC_NSCAL].slot * GBMC_NSCAL + e % GBMC_NSCAL;
                atomicAdd(&Y.weights[g], w[e]);
                atomicAdd(&Y.counts[g], c[e]);
            }
        }
    }
};

#define GBMC_BLOCK_SCALARS(name, n_prob)                                          \
    __shared__ double name##_w[kMaxSharedProblems * GBMC_NSCAL];                  \
    __shared__ unsigned long long name##_c[kMaxSharedProblems * GBMC_NSCAL];      \
    BlockScalars name;                                                            \
    name.init(name##_w, name##_c, n_prob, P.probs)

// Warp-uniform grid-stride loop: every lane of a warp runs the same number of
// iterations (so warp collectives inside are safe); `valid` marks real items.
#define GBMC_WARP_LOOP(idx, valid, n)                                                   \
    for (int64_t idx##_0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);      \
         idx##_0 < (int64_t)(n); idx##_0 += (int64_t)gridDim.x * blockDim.x)            \
        for (int64_t idx = idx##_0 + (threadIdx.x & 31), idx##_once = 0; idx##_once < 1; \
             ++idx##_once)                                                              \
            for (bool valid = idx < (int64_t)(n), valid##_once = true; valid##_once;     \
                 valid##_once = false)

// ---------------------------------------------------------------- run set-up

__global__ void k_init_run(Params P) {
    const Ctl* c = P.ctl;
    int32_t M = c->M;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x)
        P.Q.fq[i] = (int32_t)i;
    // the lookup queues' bucket counts start empty
    if (P.sort)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kSortBuckets;
             i += (int64_t)gridDim.x * blockDim.x) {
            P.Q.hist[0][i] = 0u;
            P.Q.hist[1][i] = 0u;
        }
}

// One thread: close the previous iteration, plan this one.
__global__ void k_plan(Params P) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Ctl* c = P.ctl;
    // collisions of the previous iteration
    P.st->coll += (unsigned long long)c->n_cq;
    int cur = 1 - c->cur;
    c->cur = cur;
    c->n_lq[1 - cur] = 0;
    c->n_aq[1 - cur] = 0;
    c->n_cq = 0;
    // refill free slots: split copies first, then the batch's unborn
    // particles (with weight windows the source leaves birth_reserve slots
    // for copies)
    int32_t nc = c->n_child < c->n_free ? c->n_child : c->n_free;
    c->n_birth_child = nc;
    c->child_base = c->n_child - nc;
    c->n_child -= nc;
    int32_t avail = c->n_free - nc - (P.ww ? c->birth_reserve : 0);
    if (avail < 0) avail = 0;
    int64_t remain = c->total - c->next;
    int32_t k = (int32_t)(remain < (int64_t)avail ? remain : (int64_t)avail);
    c->n_birth = nc + k;
    c->free_base = c->n_free - (nc + k);
    c->n_free -= nc + k;
    c->next_base = c->next;
    c->next += k;
    c->lq_base = c->n_lq[cur];
    c->n_lq[cur] += nc + k;
    P.st->hist += (unsigned long long)k;
    int alive = c->M - c->n_free;
    int done = alive == 0;   // nothing in flight, no copy waiting, nothing left to birth
    c->iter += 1;
    P.st->iterations += 1;
    c->tail = 0;
    if (!done && !P.ww && !P.imp_mesh && c->next == c->total && alive <= P.tail_max) {
        // few particles left: the tail kernel after the loop finishes them
        // (not while importance samples are recorded: only the collision
        // event records them)
        c->tail = 1;
        done = 1;
    } else if (!done && c->iter > P.max_iter) {
        c->err = GBMC_ERR_TIMEOUT;
        done = 1;
        c->n_lq[cur] = 0;
        c->n_aq[cur] = 0;
    }
    if (done) {
        // a tail-trigger iteration still births its particles (the source
        // kernel runs before the loop exits); only a timeout drops them
        if (!c->tail) c->n_birth = 0;
        c->lookup_n = 0;
        c->adv_n = 0;
    } else {
        c->lookup_n = c->n_lq[cur];
        c->aq_base = c->n_aq[cur];
        c->adv_n = c->n_aq[cur] + c->lookup_n;
        c->n_aq[cur] = c->adv_n;
    }
    c->adv_cursor = 0;
    c->lookup_cursor = 0;
    c->sorted = (P.sort && c->lookup_n >= P.sort_min) ? 1 : 0;
    c->warp_lookup = c->lookup_n < P.warp_lookup_max ? 1 : 0;
    c->group_lookup = !c->warp_lookup && P.precision == GBMC_FP64 &&
                      c->lookup_n < P.group_lookup_max ? 1 : 0;
    P.st->lookups += (unsigned long long)c->lookup_n;
    c->done = done;
    if (P.use_cond) cudaGraphSetConditional(P.cond, done ? 0u : 1u);
}

__device__ __forceinline__ int find_problem(const DevProblem* probs, int n_prob, int64_t gi) {
    int lo = 0, hi = n_prob;   // largest p with start <= gi
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (probs[mid].start <= gi)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- source / birth

__global__ void __launch_bounds__(256) k_source(Params P) {
    const Ctl* c = P.ctl;
    int32_t n = c->n_birth;
    if (n == 0) return;
    GBMC_BLOCK_SCALARS(sc, c->n_prob);
    int cur = c->cur;
    int32_t fb = c->free_base, lb = c->lq_base;
    int32_t nch = c->n_birth_child, cb = c->child_base;
    int64_t nb = c->next_base;
    GBMC_WARP_LOOP(idx, valid, n) {
        int prob = 0;
        bool primary = valid && idx >= nch;
        uint32_t key = 0;   // the entry's sort key (see lookup_append)
        if (valid && !primary) {
            // a split copy: its state was made by the split
            int32_t slot = P.Q.fq[fb + idx];
            const Particle& ch = P.child[cb + idx];
            P.B.p[slot] = ch;
            P.Q.lq[cur][lb + idx] = slot;
            if (P.sort) key = sort_key(P, ch.E, ch.mat);
        }
        if (primary) {
            int32_t slot = P.Q.fq[fb + idx];
            int64_t gi = nb + (idx - nch);
            prob = find_problem(P.probs, c->n_prob, gi);
            const DevProblem& pr = P.probs[prob];
            Stream r;
            r.init(pr.seed, pr.key_hi, (uint64_t)(pr.first_id + (gi - pr.start)), 0u);
            const gbmc_geometry& g = pr.g;
            double x = 0.0, y = 0.0, z = 0.0;
            if (g.source == GBMC_SRC_BANK) {
                // systematic sampling of the bank: history id i starts at
                // site floor(i bank_n / bank_total)
                int64_t id = pr.first_id + (gi - pr.start);
                int64_t sidx = id * c->bank_n / c->bank_total;
                x = P.bank[3 * sidx];
                y = P.bank[3 * sidx + 1];
                z = P.bank[3 * sidx + 2];
            } else if (g.source == GBMC_SRC_BOX) {
                double L = (double)g.n * g.pitch;
                x = r.next() * L;
                y = r.next() * L;
                z = r.next() * g.height;
            }
            double a, b;
            double s = disk_pair(r, a, b);
            double t = 2.0 * sqrt(1.0 - s);
            double w = 1.0 - 2.0 * s;
            double u, v;
            if (g.source == GBMC_SRC_SLAB_FACE) {
                u = fabs(w);
                v = a * t;
                w = b * t;
            } else {
                u = a * t;
                v = b * t;
            }
            int32_t ci = 0, cj = 0, mat;
            uint8_t inside = 0;
            if (g.kind == GBMC_GEOM_LATTICE) {
                double p = g.pitch;
                ci = (int32_t)floor(x / p);
                cj = (int32_t)floor(y / p);
                ci = ci < 0 ? 0 : (ci > g.n - 1 ? g.n - 1 : ci);
                cj = cj < 0 ? 0 : (cj > g.n - 1 ? g.n - 1 : cj);
                double dx = x - ((double)ci + 0.5) * p;
                double dy = y - ((double)cj + 0.5) * p;
                inside = (dx * dx + dy * dy) < (g.radius * g.radius);
                mat = inside ? g.mat_pin : g.mat_mod;
            } else if (g.kind == GBMC_GEOM_SLAB) {
                mat = g.n_first > 0 ? g.mat_a : g.mat_b;
            } else {
                mat = g.mat;
            }
            Particle rec;
            memset(&rec, 0, sizeof rec);
            rec.E = g.E0;
            rec.mat = mat;
            rec.prob = prob;
            rec.x = x; rec.y = y; rec.z = z; rec.wgt = 1.0;
            rec.u = u; rec.v = v; rec.w = w;
            rec.gidx = pr.out_base + (gi - pr.start);
            rec.ci = ci; rec.cj = cj;
            rec.rj = r.j;
            rec.inside = inside;
            rec.hid = (uint64_t)(pr.first_id + (gi - pr.start));
            P.B.p[slot] = rec;
            P.Q.lq[cur][lb + idx] = slot;
            if (P.sort) key = sort_key(P, rec.E, rec.mat);
        }
        if (P.sort) {
            uint32_t rk = warp_count_rank(P.Q.hist[cur], key, valid);
            if (valid) {
                P.Q.keys[cur][lb + idx] = key;
                P.Q.rank[cur][lb + idx] = rk;
            }
        }
        sc.add(P.Y, primary, prob, GBMC_S_HISTORY, 1.0, 1ull);
    }
    sc.flush(P.Y);
}

// ---------------------------------------------------------------- sort
// Counting sort of the lookup queue by a 16-bit key: material in the high
// bits, a monotone function of energy (the binary64 bit pattern above the
// smallest grid energy, shifted) in the low bits.  Order within a bucket is
// arbitrary: sorting only buys locality (Sec. 2, "Sorting"); the lookup's
// results do not depend on the order.
__device__ __forceinline__ uint32_t sort_key(const Params& P, double E, int32_t m) {
    unsigned long long eb = (unsigned long long)__double_as_longlong(E);
    unsigned long long d = eb > P.sort_ebase ? eb - P.sort_ebase : 0ull;
    unsigned long long b = d >> P.sort_shift;
    unsigned long long bmax = (1ull << P.bpm_log2) - 1ull;
    if (b > bmax) b = bmax;
    return (((uint32_t)m << P.bpm_log2) | (uint32_t)b) & (uint32_t)(kSortBuckets - 1);
}



// Exclusive scan of the bucket counts, in kScanBlocks blocks of 1024
// buckets: each block writes block-local offsets into cursor and its total
// into btot, and clears its counts for the next sort; the scatter adds the
// prefix of the block totals.
constexpr int kScanBlocks = kSortBuckets / 1024;

__device__ void scan_bucket_block(uint32_t* hist, uint32_t* cursor, uint32_t* btot) {
    __shared__ uint32_t warp_sums[32];
    int t = threadIdx.x;
    int64_t e = (int64_t)blockIdx.x * 1024 + t;
    uint32_t x = hist[e];
    int lane = t & 31, wid = t >> 5;
    uint32_t v = x;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t s2 = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, s2, o);
            if (lane >= o) s2 += y;
        }
        warp_sums[lane] = s2;
    }
    __syncthreads();
    cursor[e] = v - x + (wid ? warp_sums[wid - 1] : 0u);
    hist[e] = 0u;
    if (t == 1023) btot[blockIdx.x] = warp_sums[31];
}

// Exclusive prefix of the kScanBlocks block totals, into shared memory.
__device__ __forceinline__ void block_offsets(const uint32_t* btot, uint32_t* boff) {
    if (threadIdx.x < 32) {
        int lane = threadIdx.x;
        uint32_t a = btot[2 * lane], b = btot[2 * lane + 1];
        uint32_t v = a + b;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += y;
        }
        uint32_t ex = v - a - b;
        boff[2 * lane] = ex;
        boff[2 * lane + 1] = ex + a;
    }
    __syncthreads();
}

// Bucket offsets of the current lookup queue's histogram (the histogram is
// cleared for its queue's next use, also when this iteration does not sort).
__global__ void __launch_bounds__(1024) k_sort_scan(Params P) {
    const Ctl* c = P.ctl;
    uint32_t* hist = P.Q.hist[c->cur];
    if (!c->sorted) {
        hist[(int64_t)blockIdx.x * 1024 + threadIdx.x] = 0u;
        return;
    }
    scan_bucket_block(hist, P.Q.cursor, P.Q.btot);
}

__device__ __forceinline__ void warp_place_off(uint32_t* cursor, const uint32_t* boff, uint32_t key,
                                               bool valid, int32_t* out, int32_t value) {
    unsigned peers = __match_any_sync(kFull, valid ? key : 0xffffffffu);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid && lane == leader)
        base = atomicAdd(&cursor[key], (uint32_t)__popc(peers)) + boff[key >> 10];
    base = __shfl_sync(kFull, base, leader);
    if (valid) out[base + __popc(peers & lanemask_lt())] = value;
}

__global__ void __launch_bounds__(256) k_sort_scatter(Params P) {
    const Ctl* c = P.ctl;
    if (!c->sorted) return;
    __shared__ uint32_t boff[kScanBlocks];
    block_offsets(P.Q.btot, boff);
    int32_t n = c->lookup_n;
    const int32_t* q = P.Q.lq[c->cur];
    const uint32_t* keys = P.Q.keys[c->cur];
    const uint32_t* rank = P.Q.rank[c->cur];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        // bucket start (block offset + offset within the block) + rank
        uint32_t key = keys[i];
        uint32_t pos = boff[key >> 10] + __ldg(P.Q.cursor + key) + rank[i];
        if (pos < (uint32_t)n)
            P.Q.lqs[pos] = q[i];
        else
            atomicCAS(&P.ctl->err, 0, GBMC_ERR_DEVICE_FLAG);   // counts out of step: not reached
    }
}

// ---------------------------------------------------------------- lookup event

// Thread mode (long queues): one particle per thread.  SPARSE: binary32
// lookups on the short windows.
template <int PREC, bool SA, bool SPARSE>
__device__ __forceinline__ void lookup_threads(const Params& P, LookupTile* tiles) {
    const Ctl* c = P.ctl;
    const int32_t n = c->lookup_n;
    int cur = c->cur;
    const int32_t* q = c->sorted ? P.Q.lqs : P.Q.lq[cur];
    int32_t* aq = P.Q.aq[cur] + c->aq_base;
    unsigned long long micro = 0;
    const bool sorted = c->sorted != 0;
    // warps take 32-entry chunks from a cursor: a material's lookups cost in
    // proportion to its nuclides, so a static stride leaves late blocks with
    // the long ones
    int lane = threadIdx.x & 31;
    for (;;) {
        int64_t b0 = 0;
        if (lane == 0) b0 = atomicAdd(&P.ctl->lookup_cursor, 32);
        b0 = __shfl_sync(kFull, b0, 0);
        if (b0 >= n) break;
        int64_t idx = b0 + lane;
        bool valid = idx < n;
        int32_t slot = valid ? q[idx] : 0;
        double E = valid ? P.B.p[slot].E : 0.0;
        int32_t m = valid ? P.B.p[slot].mat : 0;
        double st = 0.0, sa = 0.0;
        if constexpr (PREC == GBMC_FP64) {
            // a sorted chunk of one material: the nuclide-major tile
            int32_t m0 = __shfl_sync(kFull, m, 0);
            if (sorted && __all_sync(kFull, !valid || m == m0) && tile_span_ok(E, valid)) {
                int nv = (int)(n - b0 < 32 ? n - b0 : 32);
                macro64_tile<SA>(P.T, m0, nv, E, tiles[threadIdx.x >> 5],
                                 valid && P.cum ? (double*)P.cum + slot * P.cum_stride : nullptr,
                                 st, sa);
            } else if (valid) {
                macro64<SA>(P.T, m, E, st, sa,
                            P.cum ? (double*)P.cum + slot * P.cum_stride : nullptr);
            }
        } else if (valid) {
            macro32<SA, SPARSE>(P.T, m, E, st, sa,
                                P.cum ? (float*)P.cum + slot * P.cum_stride : nullptr);
        }
        if (valid) {
            P.B.p[slot].st = st;
            if (SA) P.B.p[slot].sa = sa;
            aq[idx] = slot;
            micro += (unsigned long long)(__ldg(P.T.mat_off + m + 1) - __ldg(P.T.mat_off + m));
        }
    }
    for (int o = 16; o > 0; o >>= 1) micro += __shfl_xor_sync(kFull, micro, o);
    if ((threadIdx.x & 31) == 0 && micro) atomicAdd(&P.st->micro, micro);
}

// Group mode (binary64, medium queues): kGroupLanes lanes per particle,
// 32 / kGroupLanes particles per warp-chunk (macro64_group).
template <bool SA>
__device__ __forceinline__ void lookup_groups(const Params& P, LookupGroupTile* tile) {
    const Ctl* c = P.ctl;
    const int32_t n = c->lookup_n;
    const int cur = c->cur;
    const int32_t* q = c->sorted ? P.Q.lqs : P.Q.lq[cur];
    int32_t* aq = P.Q.aq[cur] + c->aq_base;
    constexpr int kPer = 32 / kGroupLanes;   // particles per warp-chunk
    const int lane = threadIdx.x & 31;
    const int p = lane / kGroupLanes;
    unsigned long long micro = 0;
    for (;;) {
        int64_t b0 = 0;
        if (lane == 0) b0 = atomicAdd(&P.ctl->lookup_cursor, kPer);
        b0 = __shfl_sync(kFull, b0, 0);
        if (b0 >= n) break;
        const int64_t idx = b0 + p;
        const bool valid = idx < n;
        const int32_t slot = valid ? q[idx] : 0;
        const double E = valid ? P.B.p[slot].E : 0.0;
        const int32_t m = valid ? P.B.p[slot].mat : 0;
        int32_t nq = valid ? __ldg(P.T.mat_off + m + 1) - __ldg(P.T.mat_off + m) : 0;
        int32_t nq_max = nq;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nq_max = max(nq_max, __shfl_xor_sync(kFull, nq_max, o));
        double st, sa;
        macro64_group<SA>(P.T, m, E, valid, nq_max, tile[threadIdx.x >> 5],
                          valid && P.cum ? (double*)P.cum + slot * P.cum_stride : nullptr, st, sa);
        if (valid && lane % kGroupLanes == 0) {
            P.B.p[slot].st = st;
            if (SA) P.B.p[slot].sa = sa;
            aq[idx] = slot;
            micro += (unsigned long long)nq;
        }
    }
    for (int o = 16; o > 0; o >>= 1) micro += __shfl_xor_sync(kFull, micro, o);
    if (lane == 0 && micro) atomicAdd(&P.st->micro, micro);
}

// Warp mode (short queues): one particle per warp.
template <int PREC, bool SA, bool SPARSE>
__device__ __forceinline__ void lookup_warps(const Params& P) {
    const Ctl* c = P.ctl;
    const int32_t n = c->lookup_n;
    int cur = c->cur;
    const int32_t* q = c->sorted ? P.Q.lqs : P.Q.lq[cur];
    int32_t* aq = P.Q.aq[cur] + c->aq_base;
    unsigned long long micro = 0;
    int lane = threadIdx.x & 31;
    int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t idx = w0; idx < n; idx += nw) {
        int32_t slot = q[idx];
        double E = P.B.p[slot].E;
        int32_t m = P.B.p[slot].mat;
        double st, sa;
        void* cum = P.cum ? (PREC == GBMC_FP64 ? (void*)((double*)P.cum + slot * P.cum_stride)
                                               : (void*)((float*)P.cum + slot * P.cum_stride))
                          : nullptr;
        macro_warp<PREC, SA, SPARSE>(P.T, m, E, st, sa, cum, 1);
        if (lane == 0) {
            P.B.p[slot].st = st;
            if (SA) P.B.p[slot].sa = sa;
            aq[idx] = slot;
            micro += (unsigned long long)(__ldg(P.T.mat_off + m + 1) - __ldg(P.T.mat_off + m));
        }
    }
    if (lane == 0 && micro) atomicAdd(&P.st->micro, micro);
}

// The lookup event: one launch per iteration, in the mode the plan picked
// for the queue's length (warp, group -- binary64 only -- or thread); the
// thread and group modes' shared-memory tiles share one buffer.
template <int PREC, bool SA, bool SPARSE = false>
__global__ void __launch_bounds__(256, PREC == GBMC_FP64 ? 4 : 3) k_lookup(Params P) {
    const Ctl* c = P.ctl;
    if (c->lookup_n == 0) return;
    constexpr size_t kTileBytes = sizeof(LookupTile) > sizeof(LookupGroupTile)
                                      ? sizeof(LookupTile) : sizeof(LookupGroupTile);
    __shared__ __align__(16) unsigned char tiles[PREC == GBMC_FP64 ? 8 * kTileBytes : 16];
    if (c->warp_lookup) {
        lookup_warps<PREC, SA, SPARSE>(P);
    } else if (PREC == GBMC_FP64 && c->group_lookup) {
        lookup_groups<SA>(P, reinterpret_cast<LookupGroupTile*>(tiles));
    } else {
        lookup_threads<PREC, SA, SPARSE>(P, reinterpret_cast<LookupTile*>(tiles));
    }
}

// ---------------------------------------------------------------- per-particle steps
// The steps of one history, shared by the event kernels and the tail kernel
// so that both perform the identical operations in the identical order.

__device__ __forceinline__ void record_death(const Params& P, const Particle& pt, int status) {
    int64_t gi = pt.gidx;
    if (gi < 0) return;   // split copies have no outcome record
    P.O.ncoll[gi] = pt.ncoll;
    P.O.status[gi] = (int8_t)status;
    P.O.nflt[gi] = pt.nflt;
    P.O.ndraw[gi] = pt.rj;
    P.O.E[gi] = pt.E;
    P.O.x[gi] = pt.x;
    P.O.y[gi] = pt.y;
    P.O.z[gi] = pt.z;
}

__device__ __forceinline__ void stream_of(const DevProblem& pr, const Particle& pt, Stream& r) {
    r.init(pr.seed, pr.key_hi, pt.hid, pt.rj);
}

__device__ __forceinline__ int32_t cell_of(const gbmc_geometry& g, const Particle& pt) {
    return g.kind == GBMC_GEOM_LATTICE ? pt.cj * g.n + pt.ci
         : g.kind == GBMC_GEOM_SLAB    ? pt.ci
                                       : 0;
}

// Track-length scores of a segment of length d in the particle's (cell,
// energy bin): flux w d and, when on, the absorption rate (w d) Sigma_a.
// ebin = energy_bin(P.T, pt.E), which the caller keeps while E is unchanged.
struct Score {
    int64_t k;     // tally bin (-1: nothing to score)
    double wd, wa; // w d and (w d) Sigma_a
};

__device__ __forceinline__ Score segment_score(const Params& P, const DevProblem& pr,
                                               const Particle& pt, double d, int32_t ebin) {
    Score s;
    s.k = pr.flux_off + (int64_t)cell_of(pr.g, pt) * P.T.n_bins + ebin;
    s.wd = pt.wgt * d;
    s.wa = P.Y.absrate ? s.wd * pt.sa : 0.0;
    return s;
}

// One lane's score, added on its own (the tail kernel's single-lane steps).
__device__ __forceinline__ void score_now(const Params& P, const Score& s) {
    if (s.k < 0) return;
    atomicAdd(&P.Y.flux[s.k], s.wd);
    if (P.Y.absrate) atomicAdd(&P.Y.absrate[s.k], s.wa);
}

// Warp-aggregated tally add (all 32 lanes call; lanes with pred add v into
// t[k]).  When every scoring lane of the warp scores the same bin (one cell
// and energy bin: an infinite medium, a slab layer, a sorted queue in one
// cell) the warp sums the values and one lane issues one atomic; otherwise
// each lane adds its own.  Used by the collision kernel, which scores the
// flights that end in a collision (in an infinite medium the whole warp
// shares a bin: config 1's collision kernel 1.08 -> 0.61 ms per batch); the
// ray trace's surface flights, in lattice cells that rarely coincide, add
// per lane (aggregating them cost 4-5% there, also when lanes were grouped
// by __match_any_sync).
__device__ __forceinline__ void tally_add_warp(double* t, int64_t k, double v, bool pred) {
    const unsigned m = __ballot_sync(kFull, pred);
    if (m == 0u) return;
    const int leader = __ffs(m) - 1;
    const long long k0 = __shfl_sync(kFull, (long long)k, leader);
    if (__all_sync(kFull, !pred || k == k0)) {
        double s = pred ? v : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if ((int)(threadIdx.x & 31) == leader) atomicAdd(t + k0, s);
    } else if (pred) {
        atomicAdd(t + k, v);
    }
}

__device__ __forceinline__ void score_warp(const Params& P, const Score& s) {
    const bool pred = s.k >= 0;
    tally_add_warp(P.Y.flux, s.k, s.wd, pred);
    if (P.Y.absrate) tally_add_warp(P.Y.absrate, s.k, s.wa, pred);
}

// One flight (advance event): sample the distance to collision, find the
// nearest surface of the current cell (ties: cylinder, x, y, z) and compare.
// a_uv = u^2 + v^2 of the current direction (a reflection keeps it);
// ebin = the tally energy bin of pt.E.
// Returns true for a collision, leaving the particle where it is: the move
// by -ln(xi) / Sigma_t and its track-length score are finish_flight's, run
// by the collision event, where every lane of a warp needs that logarithm.
// Otherwise the particle moves to pt.surf and its track-length score (w d
// in its cell and energy bin) is returned in seg for the caller to add.  The candidates are screened by their binary32
// spans: a surface decided by its span alone costs one binary64 quotient,
// taken by all such lanes of a warp together.
__device__ __forceinline__ bool fly(const Params& P, const DevProblem& pr, Particle& pt,
                                    Stream& r, double& xi, double a_uv, int32_t ebin,
                                    Score& seg) {
    const gbmc_geometry& g = pr.g;
    xi = r.next();
    pt.nflt = pt.nflt + 1;
    pt.rj = r.j;
    pt.surf = kSurfNone;
    bool lat = g.kind == GBMC_GEOM_LATTICE;
    if (!lat && g.kind != GBMC_GEOM_SLAB) return true;   // no surfaces
    const double* wall = P.planes + pr.plane_off;
    double nx = (is_pos(pt.u) ? __ldg(wall + pt.ci + 1) : __ldg(wall + pt.ci)) - pt.x;
    double ny = 0.0, nz = 0.0;
    Cyl cy;
    cy.kind = 0;
    Span sp[4];
    sp[1] = plane_span(nx, pt.u);
    if (lat) {
        const double* ctr = wall + g.n + 1;
        cy = cylinder_of(pt.x - __ldg(ctr + pt.ci), pt.y - __ldg(ctr + pt.cj), pt.u, pt.v, a_uv,
                         pr.r2, pt.inside != 0);
        ny = (is_pos(pt.v) ? __ldg(wall + pt.cj + 1) : __ldg(wall + pt.cj)) - pt.y;
        nz = is_pos(pt.w) ? g.height - pt.z : 0.0 - pt.z;
        sp[0] = cylinder_span(cy);
        sp[2] = plane_span(ny, pt.v);
        sp[3] = plane_span(nz, pt.w);
    } else {
        sp[0] = sp[2] = sp[3] = span_never();
    }
    float H = fminf(fminf(sp[0].hi, sp[1].hi), fminf(sp[2].hi, sp[3].hi));
    float L = fminf(fminf(sp[0].lo, sp[1].lo), fminf(sp[2].lo, sp[3].lo));
    Span sc = collision_span(xi, pt.st);
    int known = sc.hi < L ? 1 : (sc.lo >= H ? 0 : -1);   // 1: collision, 0: surface
    unsigned S = 0;   // candidates that can be the nearest surface
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (sp[k].lo <= H && (lat || k == 1)) S |= 1u << k;   // a slab has its x planes only
    double dbnd = CUDART_INF;
    uint8_t surf = kSurfNone;
    bool collide;
    if (known == 0 && (S & (S - 1)) == 0) {
        int k = __ffs(S) - 1;
        double num, den;
        if (k == 0) {
            double sD = sqrt(cy.D);
            num = cy.kind == 1 ? sD - cy.k : (cy.kind == 2 ? 0.0 - cy.c : cy.c);
            den = cy.kind == 1 ? cy.a : (cy.kind == 2 ? cy.k + sD : sD - cy.k);
        } else {
            num = k == 1 ? nx : (k == 2 ? ny : nz);
            den = k == 1 ? pt.u : (k == 2 ? pt.v : pt.w);
        }
        dbnd = num / den;
        if (is_neg(dbnd)) dbnd = 0.0;
        surf = (uint8_t)(kSurfCyl + k);
        collide = false;
    } else if (known == 1) {
        collide = true;
    } else {
        // not decided by the spans: every possible candidate in binary64
        double dcol = (0.0 - ln_series(xi)) / pt.st;
        bool first = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (S >> k & 1u) {
                double e = k == 0 ? cylinder_exact(cy)
                         : k == 1 ? plane_exact(nx, pt.u)
                         : k == 2 ? plane_exact(ny, pt.v)
                                  : plane_exact(nz, pt.w);
                if (is_neg(e)) e = 0.0;
                if (first || e < dbnd) {
                    dbnd = e;
                    surf = (uint8_t)(kSurfCyl + k);
                    first = false;
                }
            }
        }
        collide = dcol < dbnd;
    }
    if (!collide) {
        pt.surf = surf;
        pt.x = __fma_rn(dbnd, pt.u, pt.x);
        pt.y = __fma_rn(dbnd, pt.v, pt.y);
        pt.z = __fma_rn(dbnd, pt.w, pt.z);
        seg = segment_score(P, pr, pt, dbnd, ebin);
    }
    return collide;
}

// The end of a flight that reached its collision site: d = -ln(xi) /
// Sigma_t, the move (each coordinate x + d u one fused multiply-add), and
// the track-length score (returned to be added).
__device__ __forceinline__ Score finish_flight(const Params& P, const DevProblem& pr, Particle& pt,
                                               double xi) {
    double d = (0.0 - ln_series(xi)) / pt.st;
    pt.x = __fma_rn(d, pt.u, pt.x);
    pt.y = __fma_rn(d, pt.v, pt.y);
    pt.z = __fma_rn(d, pt.w, pt.z);
    return segment_score(P, pr, pt, d, energy_bin(P.T, pt.E));
}

// Weight-window check at the particle's (cell, energy bin), problem slot 0
// only: above the window the particle splits into n = min(floor(w / w_s),
// max_split) copies of weight w / n (the n - 1 new ones wait in the copy
// buffer for a bank slot); below it, Russian roulette keeps it with weight
// w_s with probability w / w_s.  Copy j of a split at draw position r.j of
// history hid has the history id of word 0 of the Philox block of
// (hid, r.j, j, kSplitTag) under the batch key, top bit set.
constexpr uint64_t kSplitTag = 0x5EED0C41Dull;

struct WwOut {
    int32_t copies;     // copies made
    double copy_w;      // their total weight
    double roulette_w;  // weight of a history ended by roulette
};

__device__ __forceinline__ int ww_check(const Params& P, const DevProblem& pr, Particle& pt,
                                        Stream& r, WwOut& o) {
    if (!P.ww || pt.prob != 0) return 0;
    const gbmc_geometry& g = pr.g;
    int32_t cell = g.kind == GBMC_GEOM_LATTICE ? pt.cj * g.n + pt.ci
                 : g.kind == GBMC_GEOM_SLAB    ? pt.ci
                                               : 0;
    double wl = __ldg(P.ww + (int64_t)cell * P.T.n_bins + energy_bin(P.T, pt.E));
    if (!(wl > 0.0)) return 0;
    double wu = wl * P.ww_ratio;
    double ws = wl * P.ww_survival;
    if (pt.wgt > wu) {
        int32_t n = (int32_t)floor(pt.wgt / ws);
        if (n > P.ww_max_split) n = P.ww_max_split;
        if (n < 2) return 0;
        double wc = pt.wgt / (double)n;
        pt.wgt = wc;
        for (int32_t j = 1; j < n; ++j) {
            Philox h = philox4x64_10(pt.hid, (uint64_t)r.j, (uint64_t)j, kSplitTag, r.k0, r.k1);
            Particle ch = pt;
            ch.ncoll = 0;
            ch.nflt = 0;
            ch.rj = 0;
            ch.hid = h.c0 | 0x8000000000000000ull;
            ch.gidx = -1;
            int32_t k = atomicAdd(&P.ctl->n_child, 1);
            if (k < P.child_cap)
                P.child[k] = ch;
            else
                atomicCAS(&P.ctl->err, 0, GBMC_ERR_DEVICE_FLAG);
            o.copies += 1;
            o.copy_w += wc;
        }
    } else if (pt.wgt < wl) {
        double xi = r.next();
        if (xi < pt.wgt / ws) {
            pt.wgt = ws;
        } else {
            o.roulette_w += pt.wgt;
            return GBMC_STATUS_ROULETTE;
        }
    }
    return 0;
}

// Surface event: cross pt.surf.  Returns the fate (0: still alive) and sets
// relook when the material changed (a new lookup is needed).
__device__ __forceinline__ int cross(const Params& P, const DevProblem& pr, Particle& pt,
                                     Stream& r, bool& relook, WwOut& wo) {
    const gbmc_geometry& g = pr.g;
    int status = 0;
    relook = false;
    const double* wall = P.planes + pr.plane_off;   // (double)i * pitch (or layer width)
    if (g.kind == GBMC_GEOM_SLAB) {
        if (is_pos(pt.u)) {
            pt.x = __ldg(wall + pt.ci + 1);
            if (pt.ci < g.n_layers - 1) pt.ci += 1;
            else status = GBMC_STATUS_LEAKED_FAR;
        } else {
            pt.x = __ldg(wall + pt.ci);
            if (pt.ci > 0) pt.ci -= 1;
            else status = GBMC_STATUS_LEAKED;
        }
        if (!status) {
            int32_t m = pt.ci < g.n_first ? g.mat_a : g.mat_b;
            relook = m != pt.mat;
            pt.mat = m;
        }
    } else if (pt.surf == kSurfCyl) {
        pt.inside = pt.inside ? 0 : 1;
        int32_t m = pt.inside ? g.mat_pin : g.mat_mod;
        relook = m != pt.mat;
        pt.mat = m;
    } else if (pt.surf == kSurfX) {
        if (is_pos(pt.u)) {
            pt.x = __ldg(wall + pt.ci + 1);
            if (pt.ci < g.n - 1) pt.ci += 1;
            else if (g.bc_side == GBMC_BC_REFLECT) pt.u = flip_sign(pt.u);
            else status = GBMC_STATUS_LEAKED;
        } else {
            pt.x = __ldg(wall + pt.ci);
            if (pt.ci > 0) pt.ci -= 1;
            else if (g.bc_side == GBMC_BC_REFLECT) pt.u = flip_sign(pt.u);
            else status = GBMC_STATUS_LEAKED;
        }
    } else if (pt.surf == kSurfY) {
        if (is_pos(pt.v)) {
            pt.y = __ldg(wall + pt.cj + 1);
            if (pt.cj < g.n - 1) pt.cj += 1;
            else if (g.bc_side == GBMC_BC_REFLECT) pt.v = flip_sign(pt.v);
            else status = GBMC_STATUS_LEAKED;
        } else {
            pt.y = __ldg(wall + pt.cj);
            if (pt.cj > 0) pt.cj -= 1;
            else if (g.bc_side == GBMC_BC_REFLECT) pt.v = flip_sign(pt.v);
            else status = GBMC_STATUS_LEAKED;
        }
    } else {  // z planes
        pt.z = is_pos(pt.w) ? g.height : 0.0;
        if (g.bc_z == GBMC_BC_REFLECT) pt.w = flip_sign(pt.w);
        else status = GBMC_STATUS_LEAKED;
    }
    if (!status && g.kind == GBMC_GEOM_SLAB) {
        status = ww_check(P, pr, pt, r, wo);
        pt.rj = r.j;
    }
    if (!status && pt.nflt >= GBMC_MAX_FLIGHTS) status = GBMC_STATUS_LIMIT;
    return status;
}

// k-eigenvalue banking at a collision in nuclide nuc: floor(w nu f_fis /
// k_norm + xi) fission sites at the collision point (xi one draw, right
// after the nuclide choice), in the history's own slots (so the bank's order
// is the histories' order, whatever the order of the events).  More than
// max_sites sites for one history flags the run.
__device__ __forceinline__ void bank_sites(const Params& P, Particle& pt, int32_t nuc, Stream& r) {
    double xf = r.next();
    double y = (pt.wgt * __ldg(P.T.nu + nuc)) * __ldg(P.T.f_fis + nuc) / P.ctl->k_norm + xf;
    int32_t nb = (int32_t)floor(y);
    if (nb <= 0 || pt.gidx < 0) return;
    int32_t k = pt.nsite;
    if (k + nb > P.max_sites) {
        atomicCAS(&P.ctl->err, 0, GBMC_ERR_DEVICE_FLAG);
        nb = P.max_sites - k;
    }
    double* s = P.sites + ((size_t)pt.gidx * (size_t)P.max_sites + (size_t)k) * 3;
    for (int32_t q = 0; q < nb; ++q) {
        s[3 * q] = pt.x;
        s[3 * q + 1] = pt.y;
        s[3 * q + 2] = pt.z;
    }
    pt.nsite = (uint8_t)(k + nb);
    P.site_n[pt.gidx] = k + nb;
}

// Collision event: nuclide (from the running sums the lookup stored, else
// recomputed), absorption, elastic scatter (isotropic in the CM frame,
// target at rest), energy cutoff.  Returns the fate (0: alive, needs a new
// lookup).
template <int PREC>
__device__ __forceinline__ int collide(const Params& P, const DevProblem& pr, Particle& pt,
                                       int32_t slot, Stream& r, WwOut& wo) {
    double target = r.next() * pt.st;
    int32_t nuc = -1;
    if (P.cum) {
        const void* row = PREC == GBMC_FP64 ? (const void*)((const double*)P.cum + slot * P.cum_stride)
                                            : (const void*)((const float*)P.cum + slot * P.cum_stride);
        nuc = pick_from_sums<PREC>(P.T, pt.mat, row, 1, pt.E, target);
    }
    if (nuc < 0) nuc = pick_nuclide(P.T, PREC, pt.mat, pt.E, target);
    pt.ncoll = pt.ncoll + 1;
    if (P.sites) bank_sites(P, pt, nuc, r);
    int status = 0;
    double xa = r.next();
    if (lt_nonneg(xa, __ldg(P.T.f_abs + nuc))) {   // f_abs in [0, 1]
        status = GBMC_STATUS_ABSORBED;
    } else {
        double mu = __fma_rn(2.0, r.next(), -1.0);   // = 2 xi - 1 (2 xi is exact)
        double a, b;
        double s = disk_pair(r, a, b);
        double cphi = __fma_rn(a, a, -(b * b)) / s;
        double sphi = ((2.0 * a) * b) / s;
        double E1, mul;
        elastic(pt.E, __ldg(P.T.awr + nuc), mu, E1, mul);
        double u = pt.u, v = pt.v, w = pt.w;
        rotate(u, v, w, mul, cphi, sphi);
        pt.u = u;
        pt.v = v;
        pt.w = w;
        pt.E = E1;
        if (lt_nonneg(pt.E, pr.g.E_cut))   // both positive
            status = GBMC_STATUS_CUTOFF;
        else
            status = ww_check(P, pr, pt, r, wo);
    }
    if (!status && pt.nflt >= GBMC_MAX_FLIGHTS) status = GBMC_STATUS_LIMIT;
    pt.rj = r.j;
    return status;
}

__device__ __forceinline__ int leak_kind(int status) {
    return status == GBMC_STATUS_LEAKED || status == GBMC_STATUS_LEAKED_FAR;
}

// ---------------------------------------------------------------- ray-trace event
// Advance (flight) and surface events of one particle, repeated while the
// particle crosses surfaces that keep its material (lattice walls,
// reflections): the paper's "ray trace" kernel.  A particle leaves at a
// collision (to the collision queue), a material change (to the lookup
// queue), or a leak / the flight limit (death).
//
// Work-stealing: each lane flies its particle one flight per step; a lane
// whose particle has left takes the next queue entry (one atomic per warp
// per refill), so no lane idles behind a long-streaming neighbour.
//
// Drain: once the queue is exhausted, a warp with at most kDrainLanes busy
// lanes hands its particles (each after at least one flight since it was
// taken) to the next iteration's advance queue, where they are packed with
// the other work, instead of flying them with the rest of its lanes idle.
// Only for queues of at least kDrainMinQueue entries, so that a few particles
// left in flight are not passed from iteration to iteration.
constexpr int kDrainLanes = 8;
constexpr int32_t kDrainMinQueue = 4096;

__global__ void __launch_bounds__(256, 2) k_raytrace(Params P) {
    Ctl* c = P.ctl;
    int cur = c->cur;
    int32_t n = c->adv_n;
    if (n == 0) return;
    GBMC_BLOCK_SCALARS(sc, c->n_prob);
    const int32_t* q = P.Q.aq[cur];
    int nxt = 1 - cur;
    int lane = threadIdx.x & 31;
    unsigned long long crossings = 0, nflights = 0, handoffs = 0;
    Particle pt;
    int32_t slot = 0;
    Stream r;
    int32_t flights = 0;
    double a_uv = 0.0;
    int32_t ebin = 0;
    double fw = 0.0;   // weight summed over this particle's flights
    // the lane's flight scores, summed over its particles of one problem
    int acc_prob = -1;
    double acc_w = 0.0;
    unsigned long long acc_n = 0;
    bool have = false, exhausted = false;
    for (;;) {
        bool want = !have && !exhausted;
        unsigned m = __ballot_sync(kFull, want);
        if (m) {
            int leader = __ffs(m) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&c->adv_cursor, __popc(m));
            base = __shfl_sync(kFull, base, leader);
            if (want) {
                int32_t idx = base + __popc(m & lanemask_lt());
                if (idx < n) {
                    slot = q[idx];
                    pt = P.B.p[slot];
                    stream_of(P.probs[pt.prob], pt, r);
                    a_uv = __fma_rn(pt.u, pt.u, pt.v * pt.v);   // fixed until the particle collides
                    ebin = energy_bin(P.T, pt.E);        // so is the tally energy bin
                    flights = 0;
                    fw = 0.0;
                    have = true;
                } else {
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(kFull, have)) break;
        bool drain = n >= kDrainMinQueue && __any_sync(kFull, exhausted) &&
                     __popc(__ballot_sync(kFull, have)) <= kDrainLanes;
        int status = 0, route = 0;   // route 1: collision, 2: lookup, 3: next iteration
        bool fin = false;
        WwOut wo{0, 0.0, 0.0};
        if (have && drain && flights > 0) {
            route = 3;
            fin = true;
            P.B.p[slot] = pt;
            nflights += (unsigned long long)flights;
            ++handoffs;
        } else if (have) {
            const DevProblem& pr = P.probs[pt.prob];
            double xi;
            Score sg{-1, 0.0, 0.0};
            bool col = fly(P, pr, pt, r, xi, a_uv, ebin, sg);
            score_now(P, sg);   // surface flights: lanes in other cells rarely share a bin
            ++flights;
            fw += pt.wgt;
            if (col) {
                route = 1;
                fin = true;
            } else {
                bool relook;
                status = cross(P, pr, pt, r, relook, wo);
                ++crossings;
                if (status) {
                    fin = true;
                } else if (relook) {
                    route = 2;
                    fin = true;
                }
            }
            if (fin) {
                P.B.p[slot] = pt;
                if (status) record_death(P, pt, status);
                nflights += (unsigned long long)flights;
            }
        }
        if (P.ww && __any_sync(kFull, wo.copies > 0 || wo.roulette_w > 0.0)) {
            int pw = have ? pt.prob : 0;
            sc.add(P.Y, wo.copies > 0, pw, GBMC_S_SPLIT, wo.copy_w, (unsigned long long)wo.copies);
            sc.add(P.Y, wo.roulette_w > 0.0, pw, GBMC_S_ROULETTE, wo.roulette_w, 1ull);
        }
        if (__any_sync(kFull, fin)) {
            bool dead = fin && status != 0;
            int prob = fin ? pt.prob : 0;
            double wgt = fin ? pt.wgt : 0.0;
            bool chg = fin && acc_n && prob != acc_prob;
            if (__any_sync(kFull, chg)) sc.add(P.Y, chg, acc_prob, GBMC_S_FLIGHT, acc_w, acc_n);
            if (fin) {
                if (prob != acc_prob) {
                    acc_prob = prob;
                    acc_w = 0.0;
                    acc_n = 0;
                }
                acc_w += fw;
                acc_n += (unsigned long long)flights;
            }
            sc.add(P.Y, dead && leak_kind(status), prob, GBMC_S_LEAK, wgt, 1ull);
            sc.add(P.Y, dead && status == GBMC_STATUS_LEAKED_FAR, prob, GBMC_S_LEAK_FAR, wgt, 1ull);
            sc.add(P.Y, dead && status == GBMC_STATUS_LIMIT, prob, GBMC_S_LIMIT, wgt, 1ull);
            warp_append(P.Q.fq, &c->n_free, slot, dead);
            warp_append(P.Q.cq, &c->n_cq, slot, fin && route == 1);
            lookup_append(P, nxt, &c->n_lq[nxt], slot, fin && route == 2, pt.E, pt.mat);
            warp_append(P.Q.aq[nxt], &c->n_aq[nxt], slot, fin && route == 3);
            if (fin) have = false;
        }
    }
    sc.add(P.Y, acc_n > 0, acc_prob, GBMC_S_FLIGHT, acc_w, acc_n);
    for (int o = 16; o > 0; o >>= 1) {
        crossings += __shfl_xor_sync(kFull, crossings, o);
        nflights += __shfl_xor_sync(kFull, nflights, o);
        handoffs += __shfl_xor_sync(kFull, handoffs, o);
    }
    if (lane == 0 && nflights) {
        atomicAdd(&P.st->cross, crossings);
        atomicAdd(&P.st->flights, nflights);
        if (handoffs) atomicAdd(&P.st->handoff, handoffs);
    }
    sc.flush(P.Y);
}

// ---------------------------------------------------------------- collision event

template <int PREC>
__global__ void __launch_bounds__(256, 2) k_collision(Params P) {
    Ctl* c = P.ctl;
    int32_t n = c->n_cq;
    if (n == 0) return;
    GBMC_BLOCK_SCALARS(sc, c->n_prob);
    int nxt = 1 - c->cur;
    GBMC_WARP_LOOP(idx, valid, n) {
        int32_t slot = 0;
        int prob = 0;
        int status = 0;
        double wgt = 0.0;
        double E1 = 0.0;   // energy and material after the collision (the next lookup's)
        int32_t m1 = 0;
        WwOut wo{0, 0.0, 0.0};
        Score sg{-1, 0.0, 0.0};
        if (valid) {
            slot = P.Q.cq[idx];
            Particle pt = P.B.p[slot];
            prob = pt.prob;
            const DevProblem& pr = P.probs[prob];
            wgt = pt.wgt;
            if (P.imp_mesh && prob == 0 && pt.gidx >= 0) {
                // importance sample: where this history collided (cell and
                // energy bin before the collision); its score is its fate
                const gbmc_geometry& g = pr.g;
                int32_t cell = g.kind == GBMC_GEOM_LATTICE ? pt.cj * g.n + pt.ci
                             : g.kind == GBMC_GEOM_SLAB    ? pt.ci
                                                           : 0;
                int32_t k = atomicAdd(&c->n_imp, 1);
                if (k < P.imp_cap) {
                    P.imp_mesh[k] = cell * P.T.n_bins + energy_bin(P.T, pt.E);
                    P.imp_gidx[k] = pt.gidx;
                }
            }
            // the flight's distance draw is the stream's last one
            Stream r;
            r.init(pr.seed, pr.key_hi, pt.hid, pt.rj - 1u);
            sg = finish_flight(P, pr, pt, r.next());
            status = collide<PREC>(P, pr, pt, slot, r, wo);
            P.B.p[slot] = pt;
            if (status) record_death(P, pt, status);
            E1 = pt.E;
            m1 = pt.mat;
        }
        score_warp(P, sg);
        bool dead = valid && status != 0;
        if (P.ww) {
            sc.add(P.Y, wo.copies > 0, prob, GBMC_S_SPLIT, wo.copy_w, (unsigned long long)wo.copies);
            sc.add(P.Y, wo.roulette_w > 0.0, prob, GBMC_S_ROULETTE, wo.roulette_w, 1ull);
        }
        sc.add(P.Y, valid, prob, GBMC_S_COLLISION, wgt, 1ull);
        sc.add(P.Y, dead && status == GBMC_STATUS_ABSORBED, prob, GBMC_S_ABSORPTION, wgt, 1ull);
        sc.add(P.Y, dead && status == GBMC_STATUS_CUTOFF, prob, GBMC_S_CUTOFF, wgt, 1ull);
        sc.add(P.Y, dead && status == GBMC_STATUS_LIMIT, prob, GBMC_S_LIMIT, wgt, 1ull);
        warp_append(P.Q.fq, &c->n_free, slot, dead);
        lookup_append(P, nxt, &c->n_lq[nxt], slot, valid && !dead, E1, m1);
    }
    sc.flush(P.Y);
}

// ---------------------------------------------------------------- tail
// Once the batch's source is exhausted and at most tail_max particles are
// still in flight, an iteration of the event loop costs its launches, not
// its work.  The loop then stops and this kernel finishes every remaining
// history: one warp per particle, the lookups warp-cooperative (macro_warp),
// every other step by lane 0, with the same step functions as the event
// kernels.

template <int PREC>
__global__ void __launch_bounds__(256) k_tail(Params P) {
    Ctl* c = P.ctl;
    // after the loop: keep the loop's error in the counters, which outlive
    // the run's control block
    if (blockIdx.x == 0 && threadIdx.x == 0 && c->err) atomicCAS(&P.st->err, 0, c->err);
    if (!c->tail) return;
    int cur = c->cur;
    int32_t nl = c->n_lq[cur], na = c->n_aq[cur];
    int64_t n = (int64_t)nl + na;
    int lane = threadIdx.x & 31;
    int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long lookups = 0, micro = 0, flights = 0, crossings = 0, colls = 0;
    for (int64_t idx = w0; idx < n; idx += nw) {
        int32_t slot = idx < nl ? P.Q.lq[cur][idx] : P.Q.aq[cur][idx - nl];
        bool need = idx < nl;
        Particle pt = P.B.p[slot];
        const DevProblem& pr = P.probs[pt.prob];
        Stream r;
        stream_of(pr, pt, r);
        int status = 0;
        unsigned long long nf = 0, nc = 0;   // this history's flights, collisions
        double wf = 0.0, wc = 0.0;
        for (;;) {
            if (need) {
                double st, sa;
                void* cum = P.cum ? (PREC == GBMC_FP64
                                         ? (void*)((double*)P.cum + slot * P.cum_stride)
                                         : (void*)((float*)P.cum + slot * P.cum_stride))
                                  : nullptr;
                if (P.Y.absrate)
                    macro_warp<PREC, true>(P.T, pt.mat, pt.E, st, sa, cum, 1);
                else
                    macro_warp<PREC, false>(P.T, pt.mat, pt.E, st, sa, cum, 1);
                pt.st = st;
                pt.sa = sa;
                if (lane == 0) {
                    ++lookups;
                    micro += (unsigned long long)(__ldg(P.T.mat_off + pt.mat + 1) -
                                                  __ldg(P.T.mat_off + pt.mat));
                }
            }
            int action = 0;   // 0: fly on, 1: new lookup, 2: dead
            __syncwarp();     // the lanes' running-sum checkpoints, visible to lane 0
            if (lane == 0) {
                double xi;
                Score sg{-1, 0.0, 0.0};
                bool col = fly(P, pr, pt, r, xi, __fma_rn(pt.u, pt.u, pt.v * pt.v), energy_bin(P.T, pt.E),
                               sg);
                score_now(P, sg);
                ++nf;
                wf += pt.wgt;
                if (col) {
                    ++nc;
                    wc += pt.wgt;
                    score_now(P, finish_flight(P, pr, pt, xi));
                    WwOut wo{0, 0.0, 0.0};
                    status = collide<PREC>(P, pr, pt, slot, r, wo);
                    action = status ? 2 : 1;
                } else {
                    bool relook;
                    WwOut wo{0, 0.0, 0.0};
                    status = cross(P, pr, pt, r, relook, wo);
                    ++crossings;
                    action = status ? 2 : (relook ? 1 : 0);
                }
            }
            action = __shfl_sync(kFull, action, 0);
            if (action == 2) break;
            need = action == 1;
            // every lane's lookup reads lane 0's energy and material
            pt.E = __shfl_sync(kFull, pt.E, 0);
            pt.mat = __shfl_sync(kFull, pt.mat, 0);
        }
        if (lane == 0) {
            P.B.p[slot] = pt;
            record_death(P, pt, status);
            flights += nf;
            colls += nc;
            int64_t b = (int64_t)pr.slot * GBMC_NSCAL;
            atomicAdd(&P.Y.weights[b + GBMC_S_FLIGHT], wf);
            atomicAdd(&P.Y.counts[b + GBMC_S_FLIGHT], nf);
            if (nc) {
                atomicAdd(&P.Y.weights[b + GBMC_S_COLLISION], wc);
                atomicAdd(&P.Y.counts[b + GBMC_S_COLLISION], nc);
            }
            int kind = status == GBMC_STATUS_ABSORBED ? GBMC_S_ABSORPTION
                     : status == GBMC_STATUS_CUTOFF   ? GBMC_S_CUTOFF
                     : status == GBMC_STATUS_LIMIT    ? GBMC_S_LIMIT
                                                      : GBMC_S_LEAK;
            atomicAdd(&P.Y.weights[b + kind], pt.wgt);
            atomicAdd(&P.Y.counts[b + kind], 1ull);
            if (status == GBMC_STATUS_LEAKED_FAR) {
                atomicAdd(&P.Y.weights[b + GBMC_S_LEAK_FAR], pt.wgt);
                atomicAdd(&P.Y.counts[b + GBMC_S_LEAK_FAR], 1ull);
            }
            int32_t fi = atomicAdd(&c->n_free, 1);
            P.Q.fq[fi] = slot;
        }
    }
    if (lane == 0 && (lookups | flights)) {
        atomicAdd(&P.st->lookups, lookups);
        atomicAdd(&P.st->micro, micro);
        atomicAdd(&P.st->flights, flights);
        atomicAdd(&P.st->cross, crossings);
        atomicAdd(&P.st->coll, colls);
    }
}

// ---------------------------------------------------------------- standalone lookup

__global__ void __launch_bounds__(256) k_query_keys(Params P, const double* E, const int32_t* mat,
                                                    int64_t n, uint32_t* keys, uint32_t* hist) {
    GBMC_WARP_LOOP(idx, valid, n) {
        uint32_t key = 0;
        if (valid) {
            int32_t m = mat[idx];
            key = sort_key(P, E[idx], (uint32_t)m < (uint32_t)P.T.n_mat ? m : 0);
            keys[idx] = key;
        }
        warp_count(hist, key, valid);
    }
}

__global__ void __launch_bounds__(1024) k_query_scan(uint32_t* hist, uint32_t* cursor,
                                                     uint32_t* btot) {
    scan_bucket_block(hist, cursor, btot);
}

__global__ void __launch_bounds__(256) k_query_scatter(int64_t n, const uint32_t* keys,
                                                       uint32_t* cursor, const uint32_t* btot,
                                                       int32_t* perm) {
    __shared__ uint32_t boff[kScanBlocks];
    block_offsets(btot, boff);
    GBMC_WARP_LOOP(idx, valid, n) {
        uint32_t key = valid ? keys[idx] : 0u;
        warp_place_off(cursor, boff, key, valid, perm, (int32_t)idx);
    }
}

template <int PREC, bool SPARSE = false>
__global__ void __launch_bounds__(256, 4) k_query_lookup(Tables T, const double* __restrict__ E,
                                                      const int32_t* __restrict__ mat, int64_t n,
                                                      const int32_t* __restrict__ perm,
                                                      double* __restrict__ st,
                                                      double* __restrict__ sa) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = perm ? (int64_t)perm[k] : k;
        int32_t m = mat[i];
        double a = CUDART_NAN, b = CUDART_NAN;   // a material id out of range: NaN, no lookup
        if ((uint32_t)m < (uint32_t)T.n_mat) {
            if (PREC == GBMC_FP64)
                macro64(T, m, E[i], a, b);
            else
                macro32<true, SPARSE>(T, m, E[i], a, b);
        }
        st[i] = a;
        sa[i] = b;
    }
}

// ---------------------------------------------------------------- fission bank
// Compaction of the run's per-history site slots into the bank, in history
// order: one block scans the counts (each thread a contiguous range), then a
// grid copies the sites; *bank_size receives the bank size.
__global__ void __launch_bounds__(1024) k_bank_scan(Params P) {
    __shared__ int64_t part[1024];
    const int64_t n = P.ctl->total;
    int64_t per = (n + blockDim.x - 1) / blockDim.x;
    int64_t a = (int64_t)threadIdx.x * per;
    int64_t b = a + per < n ? a + per : n;
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += P.site_n[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            int64_t v = part[k];
            part[k] = run;
            run += v;
        }
        *P.bank_size = run;
    }
    __syncthreads();
    s = part[threadIdx.x];
    for (int64_t i = a; i < b; ++i) {
        P.site_off[i] = s;
        s += P.site_n[i];
    }
}

__global__ void __launch_bounds__(256) k_bank_compact(Params P) {
    const int64_t n = P.ctl->total;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = P.site_n[g];
        const double* src = P.sites + (size_t)g * (size_t)P.max_sites * 3;
        double* dst = P.bank_out + (size_t)P.site_off[g] * 3;
        for (int32_t k = 0; k < 3 * m; ++k) dst[k] = src[k];
    }
}

cudaError_t launch_bank(const Params& P, const LaunchCfg& L, cudaStream_t s) {
    k_bank_scan<<<1, 1024, 0, s>>>(P);
    k_bank_compact<<<L.grid, 256, 0, s>>>(P);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- division self-check
// div_rn against the binary64 division on n operand pairs drawn from one
// Philox stream: random significands and signs, exponents over the whole
// normal range and near it, and the significand patterns where rounding is
// decided (equal, adjacent, all ones, powers of two), zeros and specials.
__device__ __forceinline__ double check_operand(uint64_t w, uint64_t s2) {
    uint64_t sig = w & ((1ull << 52) - 1ull);
    switch ((int)(s2 & 7u)) {
        case 0: sig = 0ull; break;                       // power of two
        case 1: sig = (1ull << 52) - 1ull; break;        // all ones
        case 2: sig &= 0xFFull; break;                   // just above a power of two
        case 3: sig |= (1ull << 52) - 256ull; break;     // just below
        default: break;
    }
    uint64_t e;
    switch ((int)((s2 >> 3) & 7u)) {
        case 0: e = (s2 >> 8) % 2047ull; break;          // any, incl. subnormal, inf, nan
        case 1: e = 1ull + (s2 >> 8) % 60ull; break;     // smallest normals
        case 2: e = 2046ull - (s2 >> 8) % 60ull; break;  // largest normals
        default: e = 1023ull - 80ull + (s2 >> 8) % 160ull; break;
    }
    if (((s2 >> 20) & 63u) == 0u) return 0.0;
    return __longlong_as_double((long long)(((s2 >> 30) & 1ull) << 63 | e << 52 | sig));
}

__global__ void k_check_division(int64_t n, uint64_t seed, unsigned long long* bad,
                                 double* first) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        Philox h = philox4x64_10((uint64_t)i, 0, 0, 0, seed, 0x0D1F1DE5ull);
        double a = check_operand(h.c0, h.c2);
        double b = check_operand(h.c1, h.c3);
        if ((h.c2 >> 40 & 15u) == 0u) b = __longlong_as_double(__double_as_longlong(a) + (long long)(h.c3 >> 60) - 8);
        double q = div_rn(a, b), r = a / b;
        bool same = __double_as_longlong(q) == __double_as_longlong(r) || (q != q && r != r);
        if (!same) {
            unsigned long long k = atomicAdd(bad, 1ull);
            if (k == 0) {
                first[0] = a;
                first[1] = b;
            }
        }
    }
}

// frac_rn against (E - e0) / de in binary64 over K grid intervals (e0, e1)
// and n energies drawn per sample: inside the interval, at and next to its
// ends, just below e0 and far above e1.
__global__ void k_check_interp(int64_t n, uint64_t seed, const double* e0s, const double* e1s,
                               const Interval64* iv, int32_t K, unsigned long long* bad,
                               double* first) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        Philox h = philox4x64_10((uint64_t)i, 0, 0, 0, seed, 0x1E7E4F0Cull);
        int32_t j = (int32_t)(h.c0 % (uint64_t)K);
        double e0 = e0s[j], e1 = e1s[j];
        Interval64 r = iv[j];
        long long b0 = __double_as_longlong(e0), b1 = __double_as_longlong(e1);
        long long k = (long long)(h.c2 >> 61) + 1;   // 1 .. 8
        double E;
        switch ((int)(h.c1 & 7u)) {
            case 0: E = e0; break;
            case 1: E = e1; break;
            case 2: E = __longlong_as_double(b0 + k); break;
            case 3: E = __longlong_as_double(b1 - k + 1); break;
            case 4: E = __longlong_as_double(b0 - k); break;
            case 5: E = __longlong_as_double(b1 + ((long long)(h.c2 >> 40 & 15u) << 52)); break;
            default: E = e0 + Stream::u01(h.c3) * r.de; break;
        }
        double q = frac_rn(E, e0, r.de, r.y), t = (E - e0) / r.de;
        bool same = __double_as_longlong(q) == __double_as_longlong(t) || (q != q && t != t);
        if (!same) {
            unsigned long long c = atomicAdd(bad, 1ull);
            if (c == 0) {
                first[0] = E;
                first[1] = e0;
            }
        }
    }
}

cudaError_t launch_check_division(int64_t n, uint64_t seed, unsigned long long* bad,
                                  double* first, int sms, cudaStream_t s) {
    k_check_division<<<sms * 8, 256, 0, s>>>(n, seed, bad, first);
    return cudaGetLastError();
}

cudaError_t launch_check_interp(int64_t n, uint64_t seed, const double* e0s, const double* e1s,
                                const Interval64* iv, int32_t K, unsigned long long* bad,
                                double* first, int sms, cudaStream_t s) {
    k_check_interp<<<sms * 8, 256, 0, s>>>(n, seed, e0s, e1s, iv, K, bad, first);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- binary64 rate probe
// The binary64 pipe's throughput, for the rooflines of the binary64 kernels:
// every thread advances kRateChains independent fused multiply-add chains
// for `iters` steps (each step one binary64 instruction per chain), and
// writes a value that depends on every chain so that none is removed.
constexpr int kRateChains = 8;

__global__ void __launch_bounds__(256) k_fp64_rate(int32_t iters, double a, double b,
                                                   double* __restrict__ out) {
    double x[kRateChains];
#pragma unroll
    for (int k = 0; k < kRateChains; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kRateChains; ++k) x[k] = __fma_rn(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kRateChains; ++k) s += x[k];
    if (s == 12345.678) out[blockIdx.x] = s;   // never true for these a, b; keeps the chains
}

cudaError_t launch_fp64_rate(int blocks, int32_t iters, double* out, cudaStream_t s) {
    k_fp64_rate<<<blocks, 256, 0, s>>>(iters, 0.999999, 1e-7, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- host launchers

// The lookup kernel, with Sigma_a only when a tally needs it.
static void launch_lookups(const Params& P, const LaunchCfg& L, cudaStream_t s) {
    bool sa = P.Y.absrate != nullptr;
    if (P.precision == GBMC_FP64) {
        if (sa)
            k_lookup<GBMC_FP64, true><<<L.grid_lookup, 256, 0, s>>>(P);
        else
            k_lookup<GBMC_FP64, false><<<L.grid_lookup, 256, 0, s>>>(P);
    } else {
        if (sa) {
            if (P.sparse_windows)
                k_lookup<GBMC_FP32, true, true><<<L.grid_lookup, 256, 0, s>>>(P);
            else
                k_lookup<GBMC_FP32, true><<<L.grid_lookup, 256, 0, s>>>(P);
        } else {
            if (P.sparse_windows)
                k_lookup<GBMC_FP32, false, true><<<L.grid_lookup, 256, 0, s>>>(P);
            else
                k_lookup<GBMC_FP32, false><<<L.grid_lookup, 256, 0, s>>>(P);
        }
    }
}

cudaError_t launch_init_run(const Params& P, const LaunchCfg& L, cudaStream_t s) {
    k_init_run<<<L.grid, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_iteration(const Params& P, const LaunchCfg& L, cudaStream_t s) {
    k_plan<<<1, 32, 0, s>>>(P);
    k_source<<<L.grid, 256, 0, s>>>(P);
    if (P.sort) {
        k_sort_scan<<<kScanBlocks, 1024, 0, s>>>(P);
        k_sort_scatter<<<L.grid, 256, 0, s>>>(P);
    }
    launch_lookups(P, L, s);
    k_raytrace<<<L.grid, 256, 0, s>>>(P);
    if (P.precision == GBMC_FP64)
        k_collision<GBMC_FP64><<<L.grid, 256, 0, s>>>(P);
    else
        k_collision<GBMC_FP32><<<L.grid, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_tail(const Params& P, const LaunchCfg& L, cudaStream_t s) {
    if (P.precision == GBMC_FP64)
        k_tail<GBMC_FP64><<<L.grid_tail, 256, 0, s>>>(P);
    else
        k_tail<GBMC_FP32><<<L.grid_tail, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_iteration_timed(const Params& P, const LaunchCfg& L, cudaStream_t s,
                                   cudaEvent_t* ev) {
    cudaEventRecord(ev[0], s);
    k_plan<<<1, 32, 0, s>>>(P);
    cudaEventRecord(ev[1], s);
    k_source<<<L.grid, 256, 0, s>>>(P);
    cudaEventRecord(ev[2], s);   // keys and counts come with the appends: no key pass
    if (P.sort) k_sort_scan<<<kScanBlocks, 1024, 0, s>>>(P);
    cudaEventRecord(ev[3], s);
    if (P.sort) k_sort_scatter<<<L.grid, 256, 0, s>>>(P);
    cudaEventRecord(ev[4], s);
    launch_lookups(P, L, s);
    cudaEventRecord(ev[5], s);
    k_raytrace<<<L.grid, 256, 0, s>>>(P);
    cudaEventRecord(ev[6], s);
    if (P.precision == GBMC_FP64)
        k_collision<GBMC_FP64><<<L.grid, 256, 0, s>>>(P);
    else
        k_collision<GBMC_FP32><<<L.grid, 256, 0, s>>>(P);
    cudaEventRecord(ev[7], s);
    return cudaGetLastError();
}

cudaError_t launch_query_lookup(const Params& P, const LaunchCfg& L, const double* E,
                                const int32_t* mat, int64_t n, double* st, double* sa,
                                int32_t* perm, uint32_t* keys, uint32_t* hist, uint32_t* cursor,
                                uint32_t* btot, cudaStream_t s) {
    if (perm) {
        k_query_keys<<<L.grid, 256, 0, s>>>(P, E, mat, n, keys, hist);
        k_query_scan<<<kScanBlocks, 1024, 0, s>>>(hist, cursor, btot);
        k_query_scatter<<<L.grid, 256, 0, s>>>(n, keys, cursor, btot, perm);
    }
    if (P.precision == GBMC_FP64)
        k_query_lookup<GBMC_FP64><<<L.grid_lookup, 256, 0, s>>>(P.T, E, mat, n, perm, st, sa);
    else if (P.sparse_windows)
        k_query_lookup<GBMC_FP32, true><<<L.grid_lookup, 256, 0, s>>>(P.T, E, mat, n, perm, st, sa);
    else
        k_query_lookup<GBMC_FP32><<<L.grid_lookup, 256, 0, s>>>(P.T, E, mat, n, perm, st, sa);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- importance estimates
// Scores the collision samples of the last run: per mesh cell, the number of
// samples and how many of them belong to histories that left through the
// far face (the analog estimate of the importance there).
__global__ void k_imp_score(const Ctl* __restrict__ c, int32_t cap, const int32_t* __restrict__ mesh,
                            const int64_t* __restrict__ gidx, const int8_t* __restrict__ status,
                            double* __restrict__ cnt, double* __restrict__ scr) {
    int32_t n = c->n_imp < cap ? c->n_imp : cap;
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int32_t m = mesh[k];
        atomicAdd(&cnt[m], 1.0);
        if (status[gidx[k]] == GBMC_STATUS_LEAKED_FAR) atomicAdd(&scr[m], 1.0);
    }
}

// Training targets from the scored samples.  Deep penetration leaves almost
// every (cell, energy bin) without a scoring history, so a cell's
// importance pools its energy bins and shrinks toward the overall score
// fraction p0: I_c = (S_c + a p0) / (N_c + a).  Every bin of the cell gets
// target ln I_c and weight N_c / (N_c + a); cells never reached get weight 0
// (the network extrapolates there).
constexpr double kShrink = 5.0;

__global__ void k_imp_cells(const double* __restrict__ cnt, const double* __restrict__ scr,
                            int32_t n_cells, int32_t n_bins, double* __restrict__ cell_sums) {
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
        double N = 0.0, S = 0.0;
        for (int32_t b = 0; b < n_bins; ++b) {
            N += cnt[(int64_t)c * n_bins + b];
            S += scr[(int64_t)c * n_bins + b];
        }
        cell_sums[2 * c] = N;
        cell_sums[2 * c + 1] = S;
        atomicAdd(&cell_sums[2 * n_cells], N);
        atomicAdd(&cell_sums[2 * n_cells + 1], S);
    }
}

__global__ void k_imp_targets(const double* __restrict__ cnt, const double* __restrict__ scr,
                              const double* __restrict__ cell_sums, int32_t n_cells, int32_t n_bins,
                              float* __restrict__ y, float* __restrict__ w) {
    int64_t n = (int64_t)n_cells * n_bins;
    double Nt = cell_sums[2 * n_cells], St = cell_sums[2 * n_cells + 1];
    double p0 = Nt > 0.0 ? (St + 0.5) / (Nt + 1.0) : 1e-12;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = (int32_t)(k / n_bins);
        double Nc = cell_sums[2 * c], Sc = cell_sums[2 * c + 1];
        double Ic = (Sc + kShrink * p0) / (Nc + kShrink);
        y[k] = (float)log(Ic);
        w[k] = (float)(Nc / (Nc + kShrink));
    }
}

cudaError_t launch_imp_score(const Params& P, const int8_t* status, double* cnt, double* scr,
                             int sms, cudaStream_t s) {
    k_imp_score<<<sms * 4, 256, 0, s>>>(P.ctl, P.imp_cap, P.imp_mesh, P.imp_gidx, status, cnt, scr);
    return cudaGetLastError();
}

cudaError_t launch_imp_targets(const double* cnt, const double* scr, int32_t n_cells,
                               int32_t n_bins, double* cell_sums, float* y, float* w, int sms,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cell_sums, 0, sizeof(double) * (2 * (size_t)n_cells + 2), s);
    if (e != cudaSuccess) return e;
    k_imp_cells<<<(n_cells + 255) / 256, 256, 0, s>>>(cnt, scr, n_cells, n_bins, cell_sums);
    int64_t n = (int64_t)n_cells * n_bins;
    int blocks = (int)((n + 255) / 256);
    if (blocks > sms * 4) blocks = sms * 4;
    if (blocks < 1) blocks = 1;
    k_imp_targets<<<blocks, 256, 0, s>>>(cnt, scr, cell_sums, n_cells, n_bins, y, w);
    return cudaGetLastError();
}

}  // namespace gbmc
