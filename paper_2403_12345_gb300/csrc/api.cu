// C ABI of the transport hot path (include/gbmc.h): context, validation of
// every input before any launch, device uploads, the graph that runs the
// device-driven event loop, and the read-back calls.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "device.cuh"
#include "launch.h"
#include "mlp.h"

using namespace gbmc;

static_assert(sizeof(gbmc_options) == 72, "gbmc_options layout is part of the ABI");
static_assert(kTimedKernels == GBMC_NKERNELS, "profile kernel count is part of the ABI");
static_assert(sizeof(gbmc_geometry) == 104, "gbmc_geometry layout is part of the ABI");
static_assert(sizeof(gbmc_problem) == 136, "gbmc_problem layout is part of the ABI");

namespace {

thread_local std::string g_create_error;
constexpr int32_t kMaxLoops = 16;   // concurrent event loops of one context
void destroy_loop(gbmc_ctx* l);

// Free a device buffer; work still queued on any stream may use it, so the
// device is drained first (reallocation is rare: buffers only grow).
template <class T>
void dfree(T*& p) {
    if (p) {
        cudaDeviceSynchronize();
        cudaFree((void*)p);
    }
    p = nullptr;
}

}  // namespace

struct gbmc_ctx {
    int device = 0;
    int sms = 0;
    gbmc_options opt{};
    std::string err;

    // tables
    int32_t n_nuc = 0;
    bool has64 = false, has32 = false;
    std::vector<int64_t> h_grid_off;
    std::vector<double> h_gmin, h_gmax;   // per nuclide grid range
    double emin_all = 0, emax_all = 0;
    int64_t* d_grid_off = nullptr;
    Interval64* d_iv64 = nullptr;
    double *d_e64 = nullptr, *d_fabs = nullptr, *d_awr = nullptr;
    float2* d_es32 = nullptr;       // binary32 (E, sigma_t) pairs, 8 pairs of padding
    float* d_fabs32 = nullptr;
    uint32_t* d_idx64 = nullptr;      // binary64 coarse index
    uint64_t table_hash = 0;   // identifies the tables both copies were built from

    // materials
    int32_t n_mat = 0;
    std::vector<int32_t> h_mat_off, h_nuc_id;
    std::vector<double> h_density, h_fabs;
    std::vector<NucIndex> h_nx32;     // binary32 search descriptors (offsets into d_es32)
    std::vector<NucIndex> h_nx32s;    // the same over the finer index of the short windows
    std::vector<NucIndex> h_nx64;     // binary64 search descriptors
    Desc64* d_desc64 = nullptr;       // per material entry: binary64 search descriptor
    Desc32* d_desc32 = nullptr;       // per material entry: search + density + f_abs
    float4* d_bw32 = nullptr;         // binary32 bucket windows (4 float4 each)
    std::vector<int64_t> h_bw_off;    // first window of each nuclide
    Desc32* d_desc32s = nullptr;      // per material entry, finer index
    float4* d_bs32 = nullptr;         // binary32 short windows (2 float4 each)
    int2* d_br32 = nullptr;           // (lo, hi) of each short window's bucket
    std::vector<int64_t> h_bs_off;    // first short window of each nuclide
    int32_t *d_mat_off = nullptr, *d_nuc_id = nullptr;
    double* d_density = nullptr;
    float* d_density32 = nullptr;

    // tally definition
    int32_t n_bins = 0;
    double* d_edges = nullptr;

    // particle bank and queues
    int32_t capacity = 0;
    Bank B{};
    Queues Q{};

    // outcomes
    int64_t out_cap = 0;
    Outcomes O{};

    // tallies: slot layout
    std::vector<int32_t> slot_cells;
    std::vector<int64_t> slot_flux_off;
    int64_t flux_cap = 0;
    int32_t slots_cap = 0;
    Tallies Y{};
    bool rr_on = false;              // absorption-rate tally on

    // k-eigenvalue mode
    double *d_nu = nullptr, *d_ffis = nullptr;
    bool fis_loaded = false;
    bool eig_on = false;
    double k_norm = 1.0;
    int32_t max_sites = 32;
    double* d_sites = nullptr;       // [sites_cap][max_sites][3] per-history slots
    int32_t* d_site_n = nullptr;     // [sites_cap]
    int64_t* d_site_off = nullptr;   // [sites_cap]
    double* d_bank_out = nullptr;    // [sites_cap * max_sites][3] the last run's bank
    int64_t* d_bank_size = nullptr;
    int64_t sites_cap = 0;
    int32_t sites_ms = 0;            // max_sites the slots were sized for
    double* d_bank_src = nullptr;    // source bank of GBMC_SRC_BANK runs
    int64_t src_cap = 0, src_n = 0, src_total = 0;

    // run descriptors
    DevProblem* d_probs = nullptr;
    int32_t probs_cap = 0;
    DevProblem* h_probs = nullptr;   // pinned staging
    int32_t h_probs_cap = 0;
    double* d_planes = nullptr;      // plane tables of the run's problems
    int64_t planes_cap = 0;
    double* h_planes = nullptr;      // pinned staging
    int64_t h_planes_cap = 0;
    Ctl* d_ctl = nullptr;
    Ctl* h_ctl = nullptr;            // pinned staging / read-back
    RunStats* d_stats = nullptr;     // counters of the last call's runs
    RunStats* h_stats = nullptr;     // pinned read-back
    cudaEvent_t staged = nullptr;

    // graph of the event loop
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Params graph_params{};
    LaunchCfg graph_launch{};
    bool graph_valid = false;

    // last run
    bool ran = false;
    cudaStream_t last_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<int64_t> run_start, run_n;

    // running sums of N_i sigma_i per bank slot (collision nuclide choice)
    void* d_cum = nullptr;
    size_t cum_bytes = 0;
    int32_t max_nuc_per_mat = 0;

    // weight windows (problem slot 0) and the split-copy buffer
    bool ww_on = false;
    int32_t ww_cells = 0;
    double ww_ratio = 5.0, ww_survival = 2.5;
    int32_t ww_max_split = 10;
    double* d_ww = nullptr;
    Particle* d_child = nullptr;
    int32_t child_cap = 0;

    // importance network (fp32 master, Adam state, gradient, BF16 copy)
    bool net_set = false;
    bool mlp_dead = false;           // a tensor-core forward never completed: refuse the network
    float *d_net_p = nullptr, *d_net_m = nullptr, *d_net_v = nullptr, *d_net_g = nullptr;
    float *d_net_scratch = nullptr;   // [0]: 1 / sum of weights, [1]: loss
    __nv_bfloat16* d_net_w = nullptr;
    int* d_mlp_err = nullptr;        // set by the tensor-core forward if a wait gave up
    int32_t net_step = 0;
    double feat_offset[4] = {0, 0, 0, 0}, feat_scale[4] = {1, 1, 1, 1};
    float *d_mesh_feat = nullptr, *d_mesh_out = nullptr;
    int64_t mesh_cap = 0;
    std::vector<double> h_edges;

    // importance samples (analog runs) and their per-mesh-cell estimates
    int32_t* d_imp_mesh = nullptr;
    int64_t* d_imp_gidx = nullptr;
    int32_t imp_cap = 0;
    bool imp_on = false;
    double *d_imp_cnt = nullptr, *d_imp_scr = nullptr, *d_imp_cellsum = nullptr;
    int64_t imp_cells = 0;

    // concurrent event loops (gbmc_run_concurrent): each a context of its
    // own bank, queues, control block, graph and stream that borrows this
    // context's tables, materials, tally definition, tallies and outcomes
    bool borrowed = false;           // this context is such a loop
    cudaStream_t own_stream = nullptr;
    cudaEvent_t done_ev = nullptr;   // the loop's last run of a call
    cudaStream_t copy_stream = nullptr;   // its runs' results to the host
    cudaEvent_t run_ev = nullptr;         // end of its latest run (the copies wait for it)
    cudaEvent_t copied_ev = nullptr;      // its last copies of a call
    std::vector<gbmc_ctx*> loops;
    int32_t last_loops = 0;          // loops the last run call used (0: this context's own loop)

    // standalone-lookup scratch
    int64_t q_cap = 0;
    int32_t* q_perm = nullptr;
    uint32_t* q_keys = nullptr;
    uint32_t *q_hist = nullptr, *q_cursor = nullptr, *q_btot = nullptr;
};

namespace {

int fail(gbmc_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    return code;
}

#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            if (e_ == cudaErrorMemoryAllocation)                                      \
                return fail(c, GBMC_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_)); \
            return fail(c, GBMC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
        }                                                                             \
    } while (0)

template <class T>
int dalloc(gbmc_ctx* c, T** p, size_t n) {
    dfree(*p);
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(c, GBMC_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T),
                    cudaGetErrorString(e));
    }
    return GBMC_OK;
}

template <class T>
int upload(gbmc_ctx* c, T** dst, const T* src, size_t n) {
    int rc = dalloc(c, dst, n);
    if (rc) return rc;
    CK(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return GBMC_OK;
}

void fill_defaults(gbmc_options* o) {
    if (o->precision != GBMC_FP32) o->precision = GBMC_FP64;
    if (o->sort == 0) o->sort = 1;
    if (o->block_lookup <= 0) o->block_lookup = 256;
    if (o->block_event <= 0) o->block_event = 256;
    if (o->blocks_per_sm <= 0) o->blocks_per_sm = 8;
    if (o->max_iterations <= 0) o->max_iterations = 4 * GBMC_MAX_FLIGHTS;
    if (o->sort_min <= 0) o->sort_min = 4096;
    if (o->warp_lookup_max == 0) o->warp_lookup_max = 4096;
    if (o->warp_lookup_max < 0) o->warp_lookup_max = 0;   // never
    if (o->tail_max == 0) o->tail_max = 4096;
    if (o->tail_max < 0) o->tail_max = 0;                 // never
    if (o->search == 0) o->search = 1;
    if (o->group_lookup_max == 0) o->group_lookup_max = 160000;
    if (o->group_lookup_max < 0) o->group_lookup_max = 0;   // never
}

int check_options(gbmc_ctx* c, const gbmc_options* o) {
    if (o->precision != GBMC_FP64 && o->precision != GBMC_FP32)
        return fail(c, GBMC_ERR_INVALID_ARG, "precision must be GBMC_FP64 or GBMC_FP32");
    if (o->sparse_windows != 0 && o->sparse_windows != 1)
        return fail(c, GBMC_ERR_INVALID_ARG, "sparse_windows must be 0 or 1");
    if (o->search != 1 && o->search != -1)
        return fail(c, GBMC_ERR_INVALID_ARG, "search must be 1 (coarse index) or -1 (plain)");
    if (o->block_lookup != 256 || o->block_event != 256)
        return fail(c, GBMC_ERR_UNSUPPORTED, "block sizes other than 256 are not built");
    if (o->blocks_per_sm > 32)
        return fail(c, GBMC_ERR_INVALID_ARG, "blocks_per_sm must be in [1, 32]");
    if (o->max_in_flight < 0 || o->max_in_flight > (int64_t)(1 << 30))
        return fail(c, GBMC_ERR_INVALID_ARG, "max_in_flight must be in [0, 2^30]");
    if (o->tail_max > (1 << 24))
        return fail(c, GBMC_ERR_INVALID_ARG, "tail_max must be at most 2^24");
    return GBMC_OK;
}

int set_device(gbmc_ctx* c) {
    CK(cudaSetDevice(c->device));
    return GBMC_OK;
}

uint64_t fnv1a(const void* p, size_t n, uint64_t h) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

void free_bank(gbmc_ctx* c) {
    dfree(c->B.p);
    Queues& Q = c->Q;
    dfree(Q.lq[0]); dfree(Q.lq[1]); dfree(Q.aq[0]); dfree(Q.aq[1]);
    dfree(Q.cq); dfree(Q.fq); dfree(Q.lqs); dfree(Q.keys[0]); dfree(Q.keys[1]);
    dfree(Q.rank[0]); dfree(Q.rank[1]);
    dfree(Q.hist[0]); dfree(Q.hist[1]); dfree(Q.cursor); dfree(Q.btot);
    c->capacity = 0;
}

int ensure_bank(gbmc_ctx* c, int32_t M) {
    if (M <= c->capacity) return GBMC_OK;
    free_bank(c);
    c->graph_valid = false;
    size_t n = (size_t)M;
    int rc = dalloc(c, &c->B.p, n);
    Queues& Q = c->Q;
    rc |= dalloc(c, &Q.lq[0], n); rc |= dalloc(c, &Q.lq[1], n);
    rc |= dalloc(c, &Q.aq[0], n); rc |= dalloc(c, &Q.aq[1], n);
    rc |= dalloc(c, &Q.cq, n); rc |= dalloc(c, &Q.fq, n);
    rc |= dalloc(c, &Q.lqs, n); rc |= dalloc(c, &Q.keys[0], n); rc |= dalloc(c, &Q.keys[1], n);
    rc |= dalloc(c, &Q.rank[0], n); rc |= dalloc(c, &Q.rank[1], n);
    rc |= dalloc(c, &Q.hist[0], kSortBuckets); rc |= dalloc(c, &Q.hist[1], kSortBuckets);
    rc |= dalloc(c, &Q.cursor, kSortBuckets);
    rc |= dalloc(c, &Q.btot, kSortBuckets / 1024);
    if (rc) {
        free_bank(c);
        return GBMC_ERR_OOM;
    }
    CK(cudaMemset(Q.hist[0], 0, sizeof(uint32_t) * kSortBuckets));
    CK(cudaMemset(Q.hist[1], 0, sizeof(uint32_t) * kSortBuckets));
    c->capacity = M;
    return GBMC_OK;
}

// Running-sum cache: one row per bank slot, in the table precision; above
// kCumBudget bytes the collision recomputes instead.  Entries per row, for
// the largest material: binary64 one checkpoint per kCumGroup64 entries
// (every sum when that is 1, rounded up to the lookup's lock-step groups for
// whole 32-byte stores; else rounded up to an even count for 16-byte
// stores); binary32 one checkpoint per kCumGroup entries, rounded up to
// whole float4s.
int64_t cum_row(const gbmc_ctx* c) {
    if (c->opt.precision == GBMC_FP64) {
        if (kCumGroup64 == 1) return ((int64_t)c->max_nuc_per_mat + kIlp - 1) / kIlp * kIlp;
        return ((int64_t)c->max_nuc_per_mat + 2 * kCumGroup64 - 1) / (2 * kCumGroup64) * 2;
    }
    // binary32: one checkpoint per kCumGroup entries, rows padded to whole
    // float4s (the lookup stores four checkpoints at a time)
    return ((int64_t)c->max_nuc_per_mat + 4 * kCumGroup - 1) / (4 * kCumGroup) * 4;
}

constexpr size_t kCumBudget = (size_t)16 << 30;

int ensure_cum(gbmc_ctx* c) {
    size_t el = c->opt.precision == GBMC_FP64 ? sizeof(double) : sizeof(float);
    size_t need = (size_t)cum_row(c) * (size_t)c->capacity * el;
    if (need > kCumBudget) need = 0;
    if (need <= c->cum_bytes && (need == 0) == (c->d_cum == nullptr)) return GBMC_OK;
    if (c->d_cum) {
        cudaDeviceSynchronize();
        cudaFree(c->d_cum);
        c->d_cum = nullptr;
        c->cum_bytes = 0;
    }
    c->graph_valid = false;
    if (need == 0) return GBMC_OK;
    cudaError_t e = cudaMalloc(&c->d_cum, need);
    if (e != cudaSuccess) {
        c->d_cum = nullptr;   // fall back to recomputation
        cudaGetLastError();
        return GBMC_OK;
    }
    c->cum_bytes = need;
    return GBMC_OK;
}

// Buffers that the run's size sets grow by at least half their size, so that
// calls of slowly growing size do not reallocate them (and rebuild every
// loop's graph, whose launch parameters hold their addresses) each time.
static int64_t grown(int64_t need, int64_t cap) { return std::max(need, cap + cap / 2); }

int ensure_outcomes(gbmc_ctx* c, int64_t n) {
    if (n <= c->out_cap) return GBMC_OK;
    n = grown(n, c->out_cap);
    Outcomes& O = c->O;
    int rc = 0;
    rc |= dalloc(c, &O.ncoll, n); rc |= dalloc(c, &O.status, n); rc |= dalloc(c, &O.nflt, n);
    rc |= dalloc(c, &O.ndraw, n); rc |= dalloc(c, &O.E, n); rc |= dalloc(c, &O.x, n);
    rc |= dalloc(c, &O.y, n); rc |= dalloc(c, &O.z, n);
    if (rc) {
        c->out_cap = 0;
        return GBMC_ERR_OOM;
    }
    c->out_cap = n;
    c->graph_valid = false;
    return GBMC_OK;
}

// Tally slots follow the problem list of the run; a different layout (slot
// count or cells per slot) re-zeroes every tally.
int ensure_tallies(gbmc_ctx* c, const std::vector<int32_t>& cells, cudaStream_t s) {
    if (cells == c->slot_cells && c->Y.flux) return GBMC_OK;
    std::vector<int64_t> off(cells.size());
    int64_t tot = 0;
    for (size_t p = 0; p < cells.size(); ++p) {
        off[p] = tot;
        tot += (int64_t)cells[p] * c->n_bins;
    }
    if (tot > c->flux_cap || !c->Y.flux) {
        const int64_t cap = grown(std::max<int64_t>(tot, 1), c->flux_cap);
        int rc = dalloc(c, &c->Y.flux, (size_t)cap);
        if (rc) return rc;
        c->flux_cap = cap;
        c->graph_valid = false;
        if (c->Y.absrate) {
            dfree(c->Y.absrate);
            c->Y.absrate = nullptr;
        }
    }
    if (c->rr_on && !c->Y.absrate) {
        int rc = dalloc(c, &c->Y.absrate, (size_t)c->flux_cap);
        if (rc) return rc;
        c->graph_valid = false;
    }
    int32_t ns = (int32_t)cells.size();
    if (ns > c->slots_cap || !c->Y.counts) {
        const int32_t cap = (int32_t)grown(ns, c->slots_cap);
        int rc = dalloc(c, &c->Y.counts, (size_t)cap * GBMC_NSCAL);
        rc |= dalloc(c, &c->Y.weights, (size_t)cap * GBMC_NSCAL);
        if (rc) return GBMC_ERR_OOM;
        c->slots_cap = cap;
        c->graph_valid = false;
    }
    CK(cudaMemsetAsync(c->Y.flux, 0, sizeof(double) * (size_t)(tot ? tot : 1), s));
    if (c->Y.absrate) CK(cudaMemsetAsync(c->Y.absrate, 0, sizeof(double) * (size_t)c->flux_cap, s));
    CK(cudaMemsetAsync(c->Y.counts, 0, sizeof(unsigned long long) * c->slots_cap * GBMC_NSCAL, s));
    CK(cudaMemsetAsync(c->Y.weights, 0, sizeof(double) * c->slots_cap * GBMC_NSCAL, s));
    c->slot_cells = cells;
    c->slot_flux_off = off;
    return GBMC_OK;
}

Tables make_tables(const gbmc_ctx* c) {
    Tables T{};
    T.grid_off = c->d_grid_off;
    T.d64 = c->d_desc64; T.idx64 = c->d_idx64; T.bw32 = c->d_bw32; T.d32 = c->d_desc32;
    T.bs32 = c->d_bs32; T.br32 = c->d_br32; T.d32s = c->d_desc32s;
    T.e64 = c->d_e64; T.iv64 = c->d_iv64; T.es32 = c->d_es32;
    T.f_abs = c->d_fabs; T.f_abs32 = c->d_fabs32; T.awr = c->d_awr;
    T.mat_off = c->d_mat_off; T.nuc_id = c->d_nuc_id;
    T.density = c->d_density; T.density32 = c->d_density32;
    T.edges = c->d_edges;
    T.nu = c->d_nu; T.f_fis = c->d_ffis;
    T.n_nuc = c->n_nuc; T.n_mat = c->n_mat; T.n_bins = c->n_bins;
    return T;
}

int ceil_log2(uint64_t v) {
    int k = 0;
    while ((1ull << k) < v) ++k;
    return k;
}

void sort_params(const gbmc_ctx* c, Params& P) {
    int mb = ceil_log2((uint64_t)(c->n_mat > 1 ? c->n_mat : 1));
    int bpm = 16 - mb;
    if (bpm < 0) bpm = 0;
    uint64_t lo, hi;
    memcpy(&lo, &c->emin_all, 8);
    memcpy(&hi, &c->emax_all, 8);
    uint64_t range = hi - lo + 1;
    uint32_t shift = 0;
    while ((range >> shift) > (1ull << bpm)) ++shift;
    P.sort_ebase = lo;
    P.sort_shift = shift;
    P.bpm_log2 = (uint32_t)bpm;
}

Params make_params(gbmc_ctx* c) {
    Params P{};
    P.T = make_tables(c);
    P.T.plain = c->opt.search < 0 ? 1 : 0;
    P.B = c->B;
    P.Q = c->Q;
    P.O = c->O;
    P.Y = c->Y;
    P.ctl = c->d_ctl;
    P.st = c->d_stats;
    P.probs = c->d_probs;
    P.capacity = c->capacity;
    P.precision = c->opt.precision;
    P.sort = c->opt.sort > 0 ? 1 : 0;
    P.sort_min = c->opt.sort_min;
    P.warp_lookup_max = c->opt.warp_lookup_max;
    P.group_lookup_max = c->opt.group_lookup_max;
    P.tail_max = c->opt.tail_max;
    P.sparse_windows = c->opt.sparse_windows;
    P.max_iter = c->opt.max_iterations;
    sort_params(c, P);
    P.planes = c->d_planes;
    P.bank = c->d_bank_src;
    if (c->eig_on) {
        P.sites = c->d_sites;
        P.site_n = c->d_site_n;
        P.site_off = c->d_site_off;
        P.bank_size = c->d_bank_size;
        P.bank_out = c->d_bank_out;
        P.max_sites = c->max_sites;
    }
    P.cum = c->d_cum;
    P.cum_stride = c->d_cum ? cum_row(c) : 0;
    if (c->ww_on) {
        P.ww = c->d_ww;
        P.ww_ratio = c->ww_ratio;
        P.ww_survival = c->ww_survival;
        P.ww_max_split = c->ww_max_split;
        P.child = c->d_child;
        P.child_cap = c->child_cap;
    }
    if (c->imp_on) {
        P.imp_mesh = c->d_imp_mesh;
        P.imp_gidx = c->d_imp_gidx;
        P.imp_cap = c->imp_cap;
    }
    return P;
}

LaunchCfg make_launch(const gbmc_ctx* c) {
    LaunchCfg L;
    L.grid = c->sms * c->opt.blocks_per_sm;
    L.grid_lookup = c->sms * c->opt.blocks_per_sm;
    L.grid_tail = std::max(1, (c->opt.tail_max + 7) / 8);   // 8 warps per block
    return L;
}

void destroy_graph(gbmc_ctx* c) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    c->graph_valid = false;
}

// Graph: [free-list init] -> while (cond) { one event-loop iteration }.  The
// plan kernel at the head of the body clears the condition once the bank is
// empty and the batch exhausted (or the iteration bound is hit).
int build_graph(gbmc_ctx* c, Params P, const LaunchCfg& L) {
    destroy_graph(c);
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    c->graph = g;
    CK(cudaStreamBeginCaptureToGraph(c->cap_stream, g, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    cudaError_t le = launch_init_run(P, L, c->cap_stream);
    cudaGraph_t g2 = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g2);
    if (le != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "init capture: %s", cudaGetErrorString(le));
    if (ee != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "init capture end: %s", cudaGetErrorString(ee));
    size_t nn = 0;
    CK(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CK(cudaGraphGetNodes(g, nodes.data(), &nn));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    CK(cudaGraphAddNode(&cn, g, nodes.data(), nullptr, nn, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    P.cond = h;
    P.use_cond = 1;
    CK(cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    le = launch_iteration(P, L, c->cap_stream);
    cudaGraph_t b2 = nullptr;
    ee = cudaStreamEndCapture(c->cap_stream, &b2);
    if (le != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "body capture: %s", cudaGetErrorString(le));
    if (ee != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "body capture end: %s", cudaGetErrorString(ee));
    // the tail kernel after the loop
    CK(cudaStreamBeginCaptureToGraph(c->cap_stream, g, &cn, nullptr, 1,
                                     cudaStreamCaptureModeThreadLocal));
    le = launch_tail(P, L, c->cap_stream);
    if (le == cudaSuccess && P.sites) le = launch_bank(P, L, c->cap_stream);
    cudaGraph_t g3 = nullptr;
    ee = cudaStreamEndCapture(c->cap_stream, &g3);
    if (le != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "tail capture: %s", cudaGetErrorString(le));
    if (ee != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "tail capture end: %s", cudaGetErrorString(ee));
    cudaError_t ie = cudaGraphInstantiate(&c->exec, g, 0);
    if (ie != cudaSuccess) {
        c->exec = nullptr;
        return fail(c, GBMC_ERR_UNSUPPORTED, "graph with a device while-node: %s",
                    cudaGetErrorString(ie));
    }
    c->graph_params = P;
    c->graph_launch = L;
    c->graph_valid = true;
    return GBMC_OK;
}

bool same_params(const Params& a, const Params& b) {
    Params x = a, y = b;
    x.cond = y.cond = cudaGraphConditionalHandle{};
    x.use_cond = y.use_cond = 0;
    return memcmp(&x, &y, sizeof(Params)) == 0;
}

int check_geometry(gbmc_ctx* c, const gbmc_geometry& g, int idx) {
    auto bad_mat = [&](int32_t m) { return m < 0 || m >= c->n_mat; };
    if (!(g.E0 > 0 && std::isfinite(g.E0)) || !(g.E_cut > 0 && std::isfinite(g.E_cut)) ||
        g.E_cut > g.E0)
        return fail(c, GBMC_ERR_INVALID_ARG, "problem %d: need 0 < E_cut <= E0", idx);
    std::vector<int32_t> mats;
    if (g.kind == GBMC_GEOM_INFINITE) {
        if (g.source != GBMC_SRC_ORIGIN && g.source != GBMC_SRC_BANK)
            return fail(c, GBMC_ERR_INVALID_ARG,
                        "problem %d: infinite medium takes the origin or bank source", idx);
        if (bad_mat(g.mat)) return fail(c, GBMC_ERR_INVALID_ARG, "problem %d: material out of range", idx);
        mats = {g.mat};
    } else if (g.kind == GBMC_GEOM_LATTICE) {
        if (g.source != GBMC_SRC_BOX && g.source != GBMC_SRC_BANK)
            return fail(c, GBMC_ERR_INVALID_ARG, "problem %d: lattice takes the box or bank source",
                        idx);
        if (g.n < 1 || g.n > 1 << 14 || !(g.pitch > 0) || !std::isfinite(g.pitch) ||
            !(g.radius > 0) || !(g.radius < 0.5 * g.pitch) || !(g.height > 0) ||
            !std::isfinite(g.height))
            return fail(c, GBMC_ERR_INVALID_ARG,
                        "problem %d: lattice needs n >= 1, p > 0, 0 < r < p/2, H > 0", idx);
        if ((g.bc_side != 0 && g.bc_side != 1) || (g.bc_z != 0 && g.bc_z != 1))
            return fail(c, GBMC_ERR_INVALID_ARG, "problem %d: boundary condition must be 0 or 1", idx);
        if (bad_mat(g.mat_pin) || bad_mat(g.mat_mod))
            return fail(c, GBMC_ERR_INVALID_ARG, "problem %d: material out of range", idx);
        mats = {g.mat_pin, g.mat_mod};
    } else if (g.kind == GBMC_GEOM_SLAB) {
        if (g.source != GBMC_SRC_SLAB_FACE)
            return fail(c, GBMC_ERR_INVALID_ARG, "problem %d: slab takes the face source", idx);
        if (g.n_layers < 1 || !(g.layer_dx > 0) || !std::isfinite(g.layer_dx) || g.n_first < 0 ||
            g.n_first > g.n_layers)
            return fail(c, GBMC_ERR_INVALID_ARG,
                        "problem %d: slab needs n_layers >= 1, dx > 0, 0 <= n_first <= n_layers", idx);
        if (bad_mat(g.mat_a) || bad_mat(g.mat_b))
            return fail(c, GBMC_ERR_INVALID_ARG, "problem %d: material out of range", idx);
        mats = {g.mat_a, g.mat_b};
    } else {
        return fail(c, GBMC_ERR_INVALID_ARG, "problem %d: unknown geometry kind %d", idx, g.kind);
    }
    // every energy the walk can reach, [E_cut, E0], must lie inside every
    // grid the lookup may search (scattering never raises the energy)
    for (int32_t m : mats)
        for (int32_t q = c->h_mat_off[m]; q < c->h_mat_off[m + 1]; ++q) {
            int32_t i = c->h_nuc_id[q];
            if (c->h_gmin[i] > g.E_cut || c->h_gmax[i] < g.E0)
                return fail(c, GBMC_ERR_INVALID_ARG,
                            "problem %d: nuclide %d grid [%g, %g] does not cover [E_cut, E0]",
                            idx, i, c->h_gmin[i], c->h_gmax[i]);
        }
    return GBMC_OK;
}

int n_cells_of(const gbmc_geometry& g) {
    if (g.kind == GBMC_GEOM_LATTICE) return g.n * g.n;
    if (g.kind == GBMC_GEOM_SLAB) return g.n_layers;
    return 1;
}

// The interval record of grid points (e0, s0), (e1, s1): the binary64
// differences the interpolation takes and the exact fixed-point reciprocal
// y = floor(2^126 / d) of de's significand d = M_de 2^11 in [2^63, 2^64)
// (0 unless de is a positive normal number).
Interval64 interval_record(double e0, double e1, double s0, double s1) {
    Interval64 r;
    r.de = e1 - e0;
    r.ds = s1 - s0;
    r.s0 = s0;
    r.y = 0ull;
    uint64_t x;
    memcpy(&x, &r.de, 8);
    const int ex = (int)(x >> 52);   // sign bit included
    if (ex >= 1 && ex <= 2046) {
        const unsigned __int128 d = (unsigned __int128)(((x & ((1ull << 52) - 1ull)) | (1ull << 52)) << 11);
        r.y = (unsigned long long)(((unsigned __int128)1 << 126) / d);
    }
    return r;
}

constexpr int32_t kIndexPer64 = 1;   // grid points per bucket of the binary64 coarse index
constexpr int32_t kShortFine = 1;    // log2 buckets per grid point of the short windows' index

// Coarse search index of every nuclide grid (binary64 or binary32 bit
// patterns): buckets (bits - bits(E_0)) >> shift, about 8 grid points per
// bucket, idx[b] = number of grid points whose bucket is below b.
int build_index(gbmc_ctx* c, int32_t n_nuc, const int64_t* grid_off, const double* energy,
                int32_t precision, NucIndex** d_nx, uint32_t** d_idx,
                const int64_t* table_off = nullptr, std::vector<NucIndex>* keep = nullptr,
                std::vector<uint32_t>* keep_idx = nullptr, int32_t per = 0,
                int32_t fine = 0) {
    auto bits = [&](int64_t k) -> uint64_t {
        if (precision == GBMC_FP64) {
            uint64_t b;
            memcpy(&b, &energy[k], 8);
            return b;
        }
        float f = (float)energy[k];
        uint32_t b;
        memcpy(&b, &f, 4);
        return b;
    };
    std::vector<NucIndex> nx(n_nuc);
    std::vector<uint32_t> idx;
    for (int32_t i = 0; i < n_nuc; ++i) {
        int64_t off = grid_off[i], n = grid_off[i + 1] - off;
        uint64_t base = bits(off), range = bits(off + n - 1) - base;
        // binary64: about one point a bucket (the bisection within the
        // bucket's range then takes at most about one step, none for an
        // empty bucket); binary32: about 1-2, read as one bucket window
        if (per <= 0) per = precision == GBMC_FP64 ? kIndexPer64 : 2;
        int32_t cap = 1 << 20;
        int32_t nb = 16;
        while ((int64_t)nb * per < (n << fine) && nb < cap) nb <<= 1;
        int32_t shift = 0;
        while ((range >> shift) >= (uint64_t)nb) ++shift;
        NucIndex d{};
        d.off = table_off ? table_off[i] : off;
        d.idx_off = (int64_t)idx.size();
        d.base = base;
        d.n = (int32_t)n;
        d.shift = shift;
        d.nb = nb;
        nx[i] = d;
        int64_t j = 0;
        for (int64_t b = 0; b <= nb; ++b) {
            while (j < n && ((bits(off + j) - base) >> shift) < (uint64_t)b) ++j;
            idx.push_back((uint32_t)j);
        }
    }
    if (keep) *keep = nx;
    if (keep_idx) *keep_idx = idx;
    int rc = d_nx ? upload(c, d_nx, nx.data(), nx.size()) : 0;
    if (rc) return rc;
    return d_idx ? upload(c, d_idx, idx.data(), idx.size()) : 0;
}

// Per material entry records of the binary32 lookup (needs the binary32
// tables and the materials).
int build_desc32(gbmc_ctx* c) {
    if (!c->has32 || !c->n_mat) return GBMC_OK;
    size_t tot = c->h_nuc_id.size();
    std::vector<Desc32> d(tot);
    // the 64-byte windows' records, then the short windows' (finer index)
    for (int form = 0; form < 2; ++form) {
        const std::vector<NucIndex>& nx = form ? c->h_nx32s : c->h_nx32;
        const std::vector<int64_t>& woff = form ? c->h_bs_off : c->h_bw_off;
        for (size_t q = 0; q < tot; ++q) {
            const NucIndex& x = nx[c->h_nuc_id[q]];
            Desc32& e = d[q];
            e.off = (int32_t)x.off;
            e.bw_off = (int32_t)woff[c->h_nuc_id[q]];
            e.base = (uint32_t)x.base;
            e.n = x.n;
            e.shift = x.shift;
            e.nb = x.nb;
            e.density = (float)c->h_density[q];
            e.f_abs = (float)c->h_fabs[c->h_nuc_id[q]];
        }
        int rc = upload(c, form ? &c->d_desc32s : &c->d_desc32, d.data(), tot);
        if (rc) return rc;
    }
    return GBMC_OK;
}

// Per material entry search descriptors of the binary64 lookup (needs the
// binary64 tables and the materials).
int build_desc64(gbmc_ctx* c) {
    if (!c->has64 || !c->n_mat) return GBMC_OK;
    size_t tot = c->h_nuc_id.size();
    std::vector<Desc64> d(tot);
    for (size_t q = 0; q < tot; ++q) {
        const NucIndex& x = c->h_nx64[c->h_nuc_id[q]];
        if (x.idx_off + x.nb > ((int64_t)1 << 31) - 1)
            return fail(c, GBMC_ERR_INVALID_ARG, "binary64 tables over 2^31 index buckets");
        Desc64& e = d[q];
        e.off = x.off;
        e.base = x.base;
        e.idx_off = (int32_t)x.idx_off;
        e.n = x.n;
        e.shift = x.shift;
        e.nb = x.nb;
    }
    return upload(c, &c->d_desc64, d.data(), tot);
}

// Waits for the last run call and reads the counters of its runs (this
// context's own loop, or every concurrent loop it used) into h_stats; the
// first error any of them flagged decides the status.
int read_ctl(gbmc_ctx* c) {
    if (!c->ran) return fail(c, GBMC_ERR_NOT_INITIALIZED, "no run has been launched");
    CK(cudaStreamSynchronize(c->last_stream));
    int err = 0;
    if (c->last_loops == 0) {
        CK(cudaMemcpy(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(c->h_stats, c->d_stats, sizeof(RunStats), cudaMemcpyDeviceToHost));
        err = c->h_ctl->err ? c->h_ctl->err : c->h_stats->err;
    } else {
        RunStats sum{};
        for (int32_t j = 0; j < c->last_loops; ++j) {
            RunStats one;
            CK(cudaMemcpy(&one, c->loops[j]->d_stats, sizeof(RunStats), cudaMemcpyDeviceToHost));
            sum.iterations += one.iterations; sum.lookups += one.lookups; sum.micro += one.micro;
            sum.flights += one.flights; sum.cross += one.cross; sum.coll += one.coll;
            sum.hist += one.hist; sum.handoff += one.handoff;
            if (!sum.err) sum.err = one.err;
        }
        *c->h_stats = sum;
        err = sum.err;
    }
    if (err == GBMC_ERR_TIMEOUT)
        return fail(c, GBMC_ERR_TIMEOUT, "event loop stopped at its iteration bound (%d)",
                    c->opt.max_iterations);
    if (err) return fail(c, GBMC_ERR_DEVICE_FLAG, "device flagged error %d", err);
    return GBMC_OK;
}

}  // namespace

extern "C" {

int gbmc_default_options(gbmc_options* opt) {
    if (!opt) return GBMC_ERR_INVALID_ARG;
    memset(opt, 0, sizeof(*opt));
    fill_defaults(opt);
    return GBMC_OK;
}

int gbmc_create(gbmc_ctx** out, int device, const gbmc_options* opt) {
    if (!out) {
        g_create_error = "out is NULL";
        return GBMC_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return GBMC_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) {
        g_create_error = "device index out of range";
        return GBMC_ERR_INVALID_ARG;
    }
    gbmc_ctx* c = new gbmc_ctx();
    c->device = device;
    gbmc_options o{};
    if (opt) o = *opt;
    fill_defaults(&o);
    int rc = check_options(c, &o);
    if (rc) {
        g_create_error = c->err;
        delete c;
        return rc;
    }
    c->opt = o;
    auto bail = [&](const char* what, cudaError_t err) {
        g_create_error = std::string(what) + ": " + cudaGetErrorString(err);
        delete c;
        return err == cudaErrorMemoryAllocation ? GBMC_ERR_OOM : GBMC_ERR_CUDA;
    };
    if ((e = cudaSetDevice(device)) != cudaSuccess) return bail("cudaSetDevice", e);
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return bail("properties", e);
    if (prop.major < 10) {
        g_create_error = "needs a Blackwell-class GPU (sm_100 or newer)";
        delete c;
        return GBMC_ERR_UNSUPPORTED;
    }
    c->sms = prop.multiProcessorCount;
    if ((e = cudaMalloc((void**)&c->d_ctl, sizeof(Ctl))) != cudaSuccess) return bail("ctl", e);
    if ((e = cudaMallocHost((void**)&c->h_ctl, sizeof(Ctl))) != cudaSuccess) return bail("ctl host", e);
    if ((e = cudaMalloc((void**)&c->d_stats, sizeof(RunStats))) != cudaSuccess) return bail("stats", e);
    if ((e = cudaMallocHost((void**)&c->h_stats, sizeof(RunStats))) != cudaSuccess)
        return bail("stats host", e);
    if ((e = cudaMemset(c->d_stats, 0, sizeof(RunStats))) != cudaSuccess) return bail("stats", e);
    if ((e = cudaEventCreate(&c->staged)) != cudaSuccess) return bail("event", e);
    if ((e = cudaEventCreate(&c->ev0)) != cudaSuccess) return bail("event", e);
    if ((e = cudaEventCreate(&c->ev1)) != cudaSuccess) return bail("event", e);
    *out = c;
    return GBMC_OK;
}

int gbmc_destroy(gbmc_ctx* c) {
    if (!c) return GBMC_OK;
    cudaSetDevice(c->device);
    if (c->ran && c->last_stream) cudaStreamSynchronize(c->last_stream);
    for (gbmc_ctx* l : c->loops) destroy_loop(l);
    c->loops.clear();
    destroy_graph(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    free_bank(c);
    Outcomes& O = c->O;
    dfree(O.ncoll); dfree(O.status); dfree(O.nflt); dfree(O.ndraw);
    dfree(O.E); dfree(O.x); dfree(O.y); dfree(O.z);
    dfree(c->Y.flux); dfree(c->Y.counts); dfree(c->Y.weights); dfree(c->Y.absrate);
    dfree(c->d_nu); dfree(c->d_ffis); dfree(c->d_sites); dfree(c->d_site_n); dfree(c->d_site_off);
    dfree(c->d_bank_out); dfree(c->d_bank_size); dfree(c->d_bank_src);
    dfree(c->d_grid_off); dfree(c->d_e64); dfree(c->d_iv64); dfree(c->d_es32);
    dfree(c->d_fabs); dfree(c->d_fabs32); dfree(c->d_awr);
    dfree(c->d_idx64); dfree(c->d_bw32); dfree(c->d_desc64);
    dfree(c->d_mat_off); dfree(c->d_nuc_id); dfree(c->d_density); dfree(c->d_density32);
    dfree(c->d_desc32); dfree(c->d_desc32s); dfree(c->d_bs32); dfree(c->d_br32);
    dfree(c->d_edges); dfree(c->d_probs); dfree(c->d_planes); dfree(c->d_ctl);
    dfree(c->d_ww); dfree(c->d_child);
    dfree(c->d_net_p); dfree(c->d_net_m); dfree(c->d_net_v); dfree(c->d_net_g);
    dfree(c->d_net_scratch); dfree(c->d_net_w); dfree(c->d_mesh_feat); dfree(c->d_mesh_out);
    dfree(c->d_mlp_err);
    dfree(c->d_imp_mesh); dfree(c->d_imp_gidx); dfree(c->d_imp_cnt); dfree(c->d_imp_scr);
    dfree(c->d_imp_cellsum);
    if (c->d_cum) { cudaDeviceSynchronize(); cudaFree(c->d_cum); }
    dfree(c->q_perm); dfree(c->q_keys); dfree(c->q_hist); dfree(c->q_cursor); dfree(c->q_btot);
    if (c->h_probs) cudaFreeHost(c->h_probs);
    if (c->h_planes) cudaFreeHost(c->h_planes);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    dfree(c->d_stats);
    if (c->h_stats) cudaFreeHost(c->h_stats);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    if (c->done_ev) cudaEventDestroy(c->done_ev);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->run_ev) cudaEventDestroy(c->run_ev);
    if (c->copied_ev) cudaEventDestroy(c->copied_ev);
    if (c->staged) cudaEventDestroy(c->staged);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
    return GBMC_OK;
}

const char* gbmc_last_error(const gbmc_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

int gbmc_set_options(gbmc_ctx* c, const gbmc_options* opt) {
    if (!c || !opt) return GBMC_ERR_INVALID_ARG;
    gbmc_options o = *opt;
    fill_defaults(&o);
    int rc = check_options(c, &o);
    if (rc) return rc;
    if (memcmp(&o, &c->opt, sizeof o) != 0) c->graph_valid = false;
    c->opt = o;
    return GBMC_OK;
}

int gbmc_load_xs_tables(gbmc_ctx* c, int32_t n_nuc, const int64_t* grid_off, const double* energy,
                        const double* sigma_t, const double* f_abs, const double* awr,
                        int32_t precision) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (n_nuc < 1 || !grid_off || !energy || !sigma_t || !f_abs || !awr)
        return fail(c, GBMC_ERR_INVALID_ARG, "n_nuc >= 1 and non-NULL arrays required");
    if (precision != GBMC_FP64 && precision != GBMC_FP32)
        return fail(c, GBMC_ERR_INVALID_ARG, "precision must be GBMC_FP64 or GBMC_FP32");
    if (grid_off[0] != 0) return fail(c, GBMC_ERR_INVALID_ARG, "grid_off[0] must be 0");
    std::vector<double> gmin(n_nuc), gmax(n_nuc);
    for (int32_t i = 0; i < n_nuc; ++i) {
        int64_t a = grid_off[i], b = grid_off[i + 1];
        if (b - a < 2) return fail(c, GBMC_ERR_INVALID_ARG, "nuclide %d has fewer than 2 grid points", i);
        for (int64_t k = a; k < b; ++k) {
            if (!(energy[k] > 0) || !std::isfinite(energy[k]))
                return fail(c, GBMC_ERR_INVALID_ARG, "nuclide %d: energy %lld not positive finite", i, (long long)(k - a));
            if (k > a && !(energy[k] > energy[k - 1]))
                return fail(c, GBMC_ERR_INVALID_ARG, "nuclide %d: grid not strictly increasing at %lld", i, (long long)(k - a));
            if (!(sigma_t[k] > 0) || !std::isfinite(sigma_t[k]))
                return fail(c, GBMC_ERR_INVALID_ARG, "nuclide %d: sigma_t %lld not positive finite", i, (long long)(k - a));
            if (precision == GBMC_FP32 && k > a && !((float)energy[k] > (float)energy[k - 1]))
                return fail(c, GBMC_ERR_INVALID_ARG,
                            "nuclide %d: grid points %lld and %lld coincide in binary32", i,
                            (long long)(k - a - 1), (long long)(k - a));
        }
        if (!(f_abs[i] >= 0 && f_abs[i] <= 1))
            return fail(c, GBMC_ERR_INVALID_ARG, "nuclide %d: f_abs outside [0, 1]", i);
        if (!(awr[i] > 0) || !std::isfinite(awr[i]))
            return fail(c, GBMC_ERR_INVALID_ARG, "nuclide %d: awr must be positive", i);
        gmin[i] = precision == GBMC_FP32 ? (double)(float)energy[a] : energy[a];
        gmax[i] = precision == GBMC_FP32 ? (double)(float)energy[b - 1] : energy[b - 1];
    }
    int rc = set_device(c);
    if (rc) return rc;
    int64_t tot = grid_off[n_nuc];
    uint64_t h = fnv1a(grid_off, sizeof(int64_t) * (n_nuc + 1), 1469598103934665603ull);
    h = fnv1a(energy, sizeof(double) * tot, h);
    h = fnv1a(sigma_t, sizeof(double) * tot, h);
    h = fnv1a(f_abs, sizeof(double) * n_nuc, h);
    h = fnv1a(awr, sizeof(double) * n_nuc, h);
    bool same = (h == c->table_hash && n_nuc == c->n_nuc);
    if (!same) {
        // new tables: drop the copy of the other precision
        dfree(c->d_e64); dfree(c->d_iv64); dfree(c->d_es32);
        dfree(c->d_idx64); dfree(c->d_bw32); dfree(c->d_bs32); dfree(c->d_br32);
        c->has64 = c->has32 = false;
        // materials refer to nuclide ids of the old tables
        if (c->n_mat) {
            dfree(c->d_mat_off); dfree(c->d_nuc_id); dfree(c->d_density); dfree(c->d_density32);
            c->n_mat = 0;
            c->h_mat_off.clear();
            c->h_nuc_id.clear();
        }
    }
    if ((rc = upload(c, &c->d_grid_off, grid_off, (size_t)n_nuc + 1))) return rc;
    if ((rc = upload(c, &c->d_fabs, f_abs, (size_t)n_nuc))) return rc;
    if ((rc = upload(c, &c->d_awr, awr, (size_t)n_nuc))) return rc;
    std::vector<float> f32(n_nuc);
    for (int32_t i = 0; i < n_nuc; ++i) f32[i] = (float)f_abs[i];
    if ((rc = upload(c, &c->d_fabs32, f32.data(), (size_t)n_nuc))) return rc;
    if (precision == GBMC_FP64) {
        if ((rc = upload(c, &c->d_e64, energy, (size_t)tot))) return rc;
        std::vector<Interval64> iv((size_t)tot);
        for (int32_t i = 0; i < n_nuc; ++i)
            for (int64_t k = grid_off[i]; k + 1 < grid_off[i + 1]; ++k)
                iv[k] = interval_record(energy[k], energy[k + 1], sigma_t[k], sigma_t[k + 1]);
        if ((rc = upload(c, &c->d_iv64, iv.data(), iv.size()))) return rc;
        if ((rc = build_index(c, n_nuc, grid_off, energy, GBMC_FP64, nullptr, &c->d_idx64, nullptr,
                              &c->h_nx64)))
            return rc;
        c->has64 = true;
    } else {
        // (E, sigma_t) pairs, each nuclide from an even pair and followed by
        // kPad32 pairs (E = +inf, sigma 0) that a window may reach
        std::vector<int64_t> poff(n_nuc);
        int64_t ptot = 0;
        for (int32_t i = 0; i < n_nuc; ++i) {
            poff[i] = ptot;
            int64_t n = grid_off[i + 1] - grid_off[i];
            ptot += (n + kPad32 + 1) & ~1ll;
        }
        if (ptot > ((int64_t)1 << 31) - 1)
            return fail(c, GBMC_ERR_INVALID_ARG, "binary32 tables over 2^31 grid points");
        const float inf = std::numeric_limits<float>::infinity();
        std::vector<float2> es(ptot, make_float2(inf, 0.0f));
        for (int32_t i = 0; i < n_nuc; ++i)
            for (int64_t k = grid_off[i]; k < grid_off[i + 1]; ++k)
                es[poff[i] + (k - grid_off[i])] = make_float2((float)energy[k], (float)sigma_t[k]);
        if ((rc = upload(c, &c->d_es32, es.data(), es.size()))) return rc;
        std::vector<uint32_t> idx;
        if ((rc = build_index(c, n_nuc, grid_off, energy, GBMC_FP32, nullptr, nullptr,
                              poff.data(), &c->h_nx32, &idx)))
            return rc;
        // bucket windows: bucket b of a nuclide holds the pairs lo .. lo + 6
        // of its bracket range [lo, hi] (lo = first point of the bucket - 1,
        // hi = first point of the next bucket, both clamped to the grid) and
        // (lo, hi) itself; a bucket with hi - lo > 6 is searched by bisection
        c->h_bw_off.assign(n_nuc, 0);
        int64_t nw = 0;
        for (int32_t i = 0; i < n_nuc; ++i) {
            c->h_bw_off[i] = nw;
            nw += c->h_nx32[i].nb;
        }
        if (nw > ((int64_t)1 << 31) - 1)
            return fail(c, GBMC_ERR_INVALID_ARG, "binary32 tables over 2^31 index buckets");
        std::vector<float4> bw((size_t)nw * 4);
        for (int32_t i = 0; i < n_nuc; ++i) {
            const NucIndex& x = c->h_nx32[i];
            const float2* g = es.data() + x.off;
            for (int32_t b = 0; b < x.nb; ++b) {
                int32_t s0 = (int32_t)idx[x.idx_off + b], s1 = (int32_t)idx[x.idx_off + b + 1];
                int32_t lo = std::min(s0 > 0 ? s0 - 1 : 0, x.n - 2);
                int32_t hi = std::min(s1, x.n - 1);
                float4* w = bw.data() + (size_t)(c->h_bw_off[i] + b) * 4;
                float2 pr[8];
                for (int p = 0; p < 7; ++p) pr[p] = g[lo + p];   // sentinels past the grid
                int32_t meta[2] = {lo, hi};
                memcpy(&pr[7], meta, 8);
                for (int k = 0; k < 4; ++k)
                    w[k] = make_float4(pr[2 * k].x, pr[2 * k].y, pr[2 * k + 1].x, pr[2 * k + 1].y);
            }
        }
        if ((rc = upload(c, &c->d_bw32, bw.data(), bw.size()))) return rc;
        bw = std::vector<float4>();
        // short windows over a finer index (about two buckets a point): bucket
        // b holds the pairs lo .. lo + 3 of its bracket range [lo, hi] (as
        // above); (lo, hi) itself goes to br32 at the same index
        std::vector<uint32_t> idx_s;
        if ((rc = build_index(c, n_nuc, grid_off, energy, GBMC_FP32, nullptr, nullptr,
                              poff.data(), &c->h_nx32s, &idx_s, 1, kShortFine)))
            return rc;
        c->h_bs_off.assign(n_nuc, 0);
        int64_t ns = 0;
        for (int32_t i = 0; i < n_nuc; ++i) {
            c->h_bs_off[i] = ns;
            ns += c->h_nx32s[i].nb;
        }
        if (ns > ((int64_t)1 << 31) - 1)
            return fail(c, GBMC_ERR_INVALID_ARG, "binary32 tables over 2^31 index buckets");
        std::vector<float4> bs((size_t)ns * 2);
        std::vector<int2> br((size_t)ns);
        for (int32_t i = 0; i < n_nuc; ++i) {
            const NucIndex& x = c->h_nx32s[i];
            const float2* g = es.data() + x.off;
            for (int32_t b = 0; b < x.nb; ++b) {
                int32_t s0 = (int32_t)idx_s[x.idx_off + b], s1 = (int32_t)idx_s[x.idx_off + b + 1];
                int32_t lo = std::min(s0 > 0 ? s0 - 1 : 0, x.n - 2);
                int32_t hi = std::min(s1, x.n - 1);
                size_t k = (size_t)(c->h_bs_off[i] + b);
                bs[2 * k] = make_float4(g[lo].x, g[lo].y, g[lo + 1].x, g[lo + 1].y);
                bs[2 * k + 1] = make_float4(g[lo + 2].x, g[lo + 2].y, g[lo + 3].x, g[lo + 3].y);
                br[k] = make_int2(lo, hi);
            }
        }
        if ((rc = upload(c, &c->d_bs32, bs.data(), bs.size()))) return rc;
        if ((rc = upload(c, &c->d_br32, br.data(), br.size()))) return rc;
        c->has32 = true;
    }
    c->n_nuc = n_nuc;
    c->h_fabs.assign(f_abs, f_abs + n_nuc);
    if ((rc = build_desc32(c)) || (rc = build_desc64(c))) return rc;
    c->table_hash = h;
    c->h_grid_off.assign(grid_off, grid_off + n_nuc + 1);
    // the grid range check uses the tighter of the two copies
    if (!same) {
        c->h_gmin = gmin;
        c->h_gmax = gmax;
    } else {
        for (int32_t i = 0; i < n_nuc; ++i) {
            c->h_gmin[i] = std::max(c->h_gmin[i], gmin[i]);
            c->h_gmax[i] = std::min(c->h_gmax[i], gmax[i]);
        }
    }
    c->emin_all = *std::min_element(c->h_gmin.begin(), c->h_gmin.end());
    c->emax_all = *std::max_element(c->h_gmax.begin(), c->h_gmax.end());
    c->graph_valid = false;
    return GBMC_OK;
}

int gbmc_init_materials(gbmc_ctx* c, int32_t n_mat, const int32_t* mat_off, const int32_t* nuc_id,
                        const double* density) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (!c->n_nuc) return fail(c, GBMC_ERR_NOT_INITIALIZED, "load the tables first");
    if (n_mat < 1 || !mat_off || !nuc_id || !density)
        return fail(c, GBMC_ERR_INVALID_ARG, "n_mat >= 1 and non-NULL arrays required");
    if (mat_off[0] != 0) return fail(c, GBMC_ERR_INVALID_ARG, "mat_off[0] must be 0");
    for (int32_t m = 0; m < n_mat; ++m) {
        if (mat_off[m + 1] <= mat_off[m])
            return fail(c, GBMC_ERR_INVALID_ARG, "material %d has no nuclide", m);
        for (int32_t q = mat_off[m]; q < mat_off[m + 1]; ++q) {
            if (nuc_id[q] < 0 || nuc_id[q] >= c->n_nuc)
                return fail(c, GBMC_ERR_INVALID_ARG, "material %d: nuclide id %d out of range", m, nuc_id[q]);
            if (!(density[q] > 0) || !std::isfinite(density[q]))
                return fail(c, GBMC_ERR_INVALID_ARG, "material %d: density must be positive", m);
        }
    }
    int rc = set_device(c);
    if (rc) return rc;
    int32_t tot = mat_off[n_mat];
    if ((rc = upload(c, &c->d_mat_off, mat_off, (size_t)n_mat + 1))) return rc;
    if ((rc = upload(c, &c->d_nuc_id, nuc_id, (size_t)tot))) return rc;
    if ((rc = upload(c, &c->d_density, density, (size_t)tot))) return rc;
    std::vector<float> d32(tot);
    for (int32_t q = 0; q < tot; ++q) d32[q] = (float)density[q];
    if ((rc = upload(c, &c->d_density32, d32.data(), (size_t)tot))) return rc;
    c->n_mat = n_mat;
    c->max_nuc_per_mat = 0;
    for (int32_t m = 0; m < n_mat; ++m)
        c->max_nuc_per_mat = std::max(c->max_nuc_per_mat, mat_off[m + 1] - mat_off[m]);
    c->h_mat_off.assign(mat_off, mat_off + n_mat + 1);
    c->h_nuc_id.assign(nuc_id, nuc_id + tot);
    c->h_density.assign(density, density + tot);
    if ((rc = build_desc32(c)) || (rc = build_desc64(c))) return rc;
    c->graph_valid = false;
    return GBMC_OK;
}

int gbmc_set_tally(gbmc_ctx* c, int32_t n_bins, const double* edges) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (n_bins < 1 || !edges) return fail(c, GBMC_ERR_INVALID_ARG, "n_bins >= 1 and edges required");
    for (int32_t b = 0; b <= n_bins; ++b) {
        if (!(edges[b] > 0) || !std::isfinite(edges[b]))
            return fail(c, GBMC_ERR_INVALID_ARG, "tally edges must be positive and finite");
        if (b && !(edges[b] > edges[b - 1]))
            return fail(c, GBMC_ERR_INVALID_ARG, "tally edges must be strictly increasing");
    }
    int rc = set_device(c);
    if (rc) return rc;
    if ((rc = upload(c, &c->d_edges, edges, (size_t)n_bins + 1))) return rc;
    c->n_bins = n_bins;
    c->h_edges.assign(edges, edges + n_bins + 1);
    c->slot_cells.clear();   // forces re-zeroing at the next run
    c->graph_valid = false;
    return GBMC_OK;
}

int gbmc_reset_tallies(gbmc_ctx* c, void* stream) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    int rc = set_device(c);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->Y.flux) CK(cudaMemsetAsync(c->Y.flux, 0, sizeof(double) * c->flux_cap, s));
    if (c->Y.absrate) CK(cudaMemsetAsync(c->Y.absrate, 0, sizeof(double) * c->flux_cap, s));
    if (c->Y.counts) {
        CK(cudaMemsetAsync(c->Y.counts, 0, sizeof(unsigned long long) * c->slots_cap * GBMC_NSCAL, s));
        CK(cudaMemsetAsync(c->Y.weights, 0, sizeof(double) * c->slots_cap * GBMC_NSCAL, s));
    }
    return GBMC_OK;
}

}  // extern "C"

namespace {

// Where a concurrent loop's run puts its results: per problem of the run,
// its flux offset, the outcome index of its first particle and its tally
// slot in the borrowed tallies and outcomes.
struct RunLayout {
    const int64_t* flux_off;
    const int64_t* out_base;
    const int32_t* slot;
    bool keep_stats;   // add to the loop's counters (a later run of the same call)
};

// Validate a run, size the buffers, stage descriptors and the control block
// (stream-ordered copies on s).  Fills the launch parameters.  With lay (a
// concurrent loop's run) the tallies and outcomes are the borrowed ones.
int prepare_run(gbmc_ctx* c, int32_t n_prob, const gbmc_problem* probs, cudaStream_t s,
                Params* Pout, LaunchCfg* Lout, const RunLayout* lay = nullptr) {
    if (n_prob < 1 || !probs) return fail(c, GBMC_ERR_INVALID_ARG, "n_prob >= 1 and probs required");
    if (!c->n_nuc || !c->n_mat || !c->n_bins)
        return fail(c, GBMC_ERR_NOT_INITIALIZED, "tables, materials and tally must be set first");
    if ((c->opt.precision == GBMC_FP64 && !c->has64) || (c->opt.precision == GBMC_FP32 && !c->has32))
        return fail(c, GBMC_ERR_NOT_INITIALIZED, "tables not loaded in the selected precision");
    std::vector<int32_t> cells(n_prob);
    std::vector<int64_t> start(n_prob), nn(n_prob), plane_off(n_prob);
    int64_t total = 0, n_planes = 0;
    for (int32_t p = 0; p < n_prob; ++p) {
        int rc = check_geometry(c, probs[p].geom, p);
        if (rc) return rc;
        if (probs[p].n_particles < 0 || probs[p].first_id < 0 ||
            probs[p].first_id > std::numeric_limits<int64_t>::max() - probs[p].n_particles)
            return fail(c, GBMC_ERR_INVALID_ARG, "problem %d: bad particle range", p);
        cells[p] = n_cells_of(probs[p].geom);
        plane_off[p] = n_planes;
        const gbmc_geometry& g = probs[p].geom;
        n_planes += g.kind == GBMC_GEOM_LATTICE ? 2 * (int64_t)g.n + 1
                  : g.kind == GBMC_GEOM_SLAB    ? (int64_t)g.n_layers + 1
                                                : 0;
        start[p] = total;
        nn[p] = probs[p].n_particles;
        total += probs[p].n_particles;
        if (total > ((int64_t)1 << 40))
            return fail(c, GBMC_ERR_INVALID_ARG, "more than 2^40 particles in one run");
    }
    int rc = set_device(c);
    if (rc) return rc;
    int64_t M64 = c->opt.max_in_flight > 0 ? c->opt.max_in_flight : ((int64_t)8 << 20);
    if (M64 > total) M64 = total;
    if (M64 < 1) M64 = 1;
    int32_t M = (int32_t)M64;
    if ((rc = ensure_bank(c, M))) return rc;
    if ((rc = ensure_cum(c))) return rc;
    if (c->ww_on) {
        if (cells[0] != c->ww_cells)
            return fail(c, GBMC_ERR_INVALID_ARG,
                        "weight windows cover %d cells, problem slot 0 has %d", c->ww_cells, cells[0]);
        // split copies wait here for free slots: room for four bank-fulls
        int64_t want = std::max<int64_t>((int64_t)c->capacity * 4, (int64_t)1 << 20);
        if (c->child_cap < want) {
            if ((rc = dalloc(c, &c->d_child, (size_t)want))) return rc;
            c->child_cap = (int32_t)want;
            c->graph_valid = false;
        }
    }
    for (int32_t p = 0; p < n_prob; ++p) {
        if (probs[p].geom.source != GBMC_SRC_BANK) continue;
        if (c->src_n < 1)
            return fail(c, GBMC_ERR_NOT_INITIALIZED, "problem %d takes the bank source: set it first", p);
        if (probs[p].first_id + probs[p].n_particles > c->src_total)
            return fail(c, GBMC_ERR_INVALID_ARG,
                        "problem %d: ids beyond the source bank's generation size %lld", p,
                        (long long)c->src_total);
    }
    if (c->eig_on) {
        if (n_prob != 1 || c->ww_on)
            return fail(c, GBMC_ERR_UNSUPPORTED,
                        "k-eigenvalue runs take one problem and no weight windows");
        if (total > c->sites_cap || c->max_sites != c->sites_ms) {
            int64_t cap = std::max<int64_t>(total, 1);
            size_t ns = (size_t)cap * (size_t)c->max_sites * 3;
            if ((rc = dalloc(c, &c->d_sites, ns))) return rc;
            if ((rc = dalloc(c, &c->d_bank_out, ns))) return rc;
            if ((rc = dalloc(c, &c->d_site_n, (size_t)cap))) return rc;
            if ((rc = dalloc(c, &c->d_site_off, (size_t)cap))) return rc;
            if (!c->d_bank_size && (rc = dalloc(c, &c->d_bank_size, 1))) return rc;
            c->sites_cap = cap;
            c->sites_ms = c->max_sites;
            c->graph_valid = false;
        }
        CK(cudaMemsetAsync(c->d_site_n, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1), s));
    }
    if (!lay) {
        if ((rc = ensure_outcomes(c, total > 0 ? total : 1))) return rc;
        if ((rc = ensure_tallies(c, cells, s))) return rc;
    }
    if (n_prob > c->probs_cap) {
        if ((rc = dalloc(c, &c->d_probs, (size_t)n_prob))) return rc;
        c->probs_cap = n_prob;
        c->graph_valid = false;
    }
    if (n_planes < 1) n_planes = 1;
    if (n_planes > c->planes_cap) {
        if ((rc = dalloc(c, &c->d_planes, (size_t)n_planes))) return rc;
        c->planes_cap = n_planes;
        c->graph_valid = false;
    }
    if (n_planes > c->h_planes_cap) {
        CK(cudaEventSynchronize(c->staged));
        if (c->h_planes) cudaFreeHost(c->h_planes);
        c->h_planes = nullptr;
        CK(cudaMallocHost((void**)&c->h_planes, sizeof(double) * n_planes));
        c->h_planes_cap = n_planes;
    }
    if (n_prob > c->h_probs_cap) {
        CK(cudaEventSynchronize(c->staged));
        if (c->h_probs) cudaFreeHost(c->h_probs);
        c->h_probs = nullptr;
        CK(cudaMallocHost((void**)&c->h_probs, sizeof(DevProblem) * n_prob));
        c->h_probs_cap = n_prob;
    }
    *Pout = make_params(c);
    *Lout = make_launch(c);
    // stage the descriptors (pinned) once the previous staging copy is done
    CK(cudaEventSynchronize(c->staged));
    for (int32_t p = 0; p < n_prob; ++p) {
        DevProblem& d = c->h_probs[p];
        memset(&d, 0, sizeof d);
        d.g = probs[p].geom;
        d.seed = probs[p].seed;
        d.key_hi = ((uint64_t)probs[p].problem_index << 32) | (uint64_t)probs[p].batch;
        d.first_id = probs[p].first_id;
        d.n = probs[p].n_particles;
        d.start = start[p];
        d.flux_off = lay ? lay->flux_off[p] : c->slot_flux_off[p];
        d.out_base = lay ? lay->out_base[p] : start[p];
        d.slot = lay ? lay->slot[p] : p;
        d.plane_off = plane_off[p];
        d.r2 = probs[p].geom.radius * probs[p].geom.radius;
        d.n_cells = cells[p];
        // plane positions as the transport forms them: walls i * pitch
        // (i = 0..n), then lattice cell centres (i + 0.5) * pitch
        const gbmc_geometry& g = probs[p].geom;
        double* w = c->h_planes + plane_off[p];
        if (g.kind == GBMC_GEOM_LATTICE) {
            for (int32_t i = 0; i <= g.n; ++i) w[i] = (double)i * g.pitch;
            for (int32_t i = 0; i < g.n; ++i) w[g.n + 1 + i] = ((double)i + 0.5) * g.pitch;
        } else if (g.kind == GBMC_GEOM_SLAB) {
            for (int32_t i = 0; i <= g.n_layers; ++i) w[i] = (double)i * g.layer_dx;
        }
    }
    Ctl& k = *c->h_ctl;
    memset(&k, 0, sizeof k);
    k.n_free = M;
    k.cur = 1;
    k.total = total;
    k.M = M;
    k.n_prob = n_prob;
    k.birth_reserve = c->ww_on ? M / 2 : 0;
    k.k_norm = c->k_norm;
    k.bank_n = c->src_n;
    k.bank_total = c->src_total;
    CK(cudaMemcpyAsync(c->d_probs, c->h_probs, sizeof(DevProblem) * n_prob, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_planes, c->h_planes, sizeof(double) * n_planes, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_ctl, c->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    if (!lay || !lay->keep_stats) CK(cudaMemsetAsync(c->d_stats, 0, sizeof(RunStats), s));
    CK(cudaEventRecord(c->staged, s));
    if (!lay) {
        c->run_start = start;
        c->run_n = nn;
    }
    return GBMC_OK;
}

// Launch one run (its graph, rebuilt when the launch parameters changed).
int launch_run(gbmc_ctx* c, int32_t n_prob, const gbmc_problem* probs, cudaStream_t s,
               const RunLayout* lay) {
    if (c->ran) {
        int rc0 = set_device(c);
        if (rc0) return rc0;
    }
    Params P;
    LaunchCfg L;
    int rc = prepare_run(c, n_prob, probs, s, &P, &L, lay);
    if (rc) return rc;
    if (!c->graph_valid || !same_params(P, c->graph_params) ||
        memcmp(&L, &c->graph_launch, sizeof L) != 0) {
        CK(cudaStreamSynchronize(s));
        if (c->ran) CK(cudaStreamSynchronize(c->last_stream));
        if ((rc = build_graph(c, P, L))) return rc;
    }
    CK(cudaEventRecord(c->ev0, s));
    CK(cudaGraphLaunch(c->exec, s));
    CK(cudaEventRecord(c->ev1, s));
    c->ran = true;
    c->last_stream = s;
    return GBMC_OK;
}

// The pointers a concurrent loop borrows from its context, cleared so that
// destroying the loop frees only its own buffers.
void release_borrowed(gbmc_ctx* l) {
    l->d_grid_off = nullptr; l->d_iv64 = nullptr; l->d_e64 = nullptr; l->d_fabs = nullptr;
    l->d_awr = nullptr; l->d_es32 = nullptr; l->d_fabs32 = nullptr; l->d_idx64 = nullptr;
    l->d_desc64 = nullptr; l->d_desc32 = nullptr; l->d_bw32 = nullptr;
    l->d_desc32s = nullptr; l->d_bs32 = nullptr; l->d_br32 = nullptr;
    l->d_mat_off = nullptr; l->d_nuc_id = nullptr; l->d_density = nullptr;
    l->d_density32 = nullptr; l->d_edges = nullptr; l->d_nu = nullptr; l->d_ffis = nullptr;
    l->O = Outcomes{};
    l->Y = Tallies{};
    l->out_cap = 0;
}

void destroy_loop(gbmc_ctx* l) {
    release_borrowed(l);
    gbmc_destroy(l);
}

// A concurrent loop takes the context's tables, materials, tally definition,
// tallies, outcomes and options (pointers and host copies; nothing is copied
// on the device).
void borrow_from(gbmc_ctx* l, const gbmc_ctx* c) {
    l->opt = c->opt;
    l->n_nuc = c->n_nuc; l->has64 = c->has64; l->has32 = c->has32;
    l->h_grid_off = c->h_grid_off; l->h_gmin = c->h_gmin; l->h_gmax = c->h_gmax;
    l->emin_all = c->emin_all; l->emax_all = c->emax_all;
    l->d_grid_off = c->d_grid_off; l->d_iv64 = c->d_iv64; l->d_e64 = c->d_e64;
    l->d_fabs = c->d_fabs; l->d_awr = c->d_awr; l->d_es32 = c->d_es32;
    l->d_fabs32 = c->d_fabs32; l->d_idx64 = c->d_idx64;
    l->d_desc64 = c->d_desc64; l->d_desc32 = c->d_desc32; l->d_bw32 = c->d_bw32;
    l->d_desc32s = c->d_desc32s; l->d_bs32 = c->d_bs32; l->d_br32 = c->d_br32;
    l->n_mat = c->n_mat; l->h_mat_off = c->h_mat_off; l->h_nuc_id = c->h_nuc_id;
    l->h_density = c->h_density; l->h_fabs = c->h_fabs; l->max_nuc_per_mat = c->max_nuc_per_mat;
    l->d_mat_off = c->d_mat_off; l->d_nuc_id = c->d_nuc_id; l->d_density = c->d_density;
    l->d_density32 = c->d_density32;
    l->n_bins = c->n_bins; l->d_edges = c->d_edges;
    l->d_nu = c->d_nu; l->d_ffis = c->d_ffis;
    l->O = c->O; l->out_cap = c->out_cap;
    l->Y = c->Y; l->rr_on = c->rr_on;
}

}  // namespace

extern "C" {

int gbmc_run_problems(gbmc_ctx* c, int32_t n_prob, const gbmc_problem* probs, void* stream) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (c->ran && c->last_loops > 0) {
        // the previous call's loops write into this context's tallies and
        // outcomes: let them finish before the buffers are reused
        CK(cudaStreamSynchronize(c->last_stream));
    }
    int rc = launch_run(c, n_prob, probs, (cudaStream_t)stream, nullptr);
    if (rc == GBMC_OK) c->last_loops = 0;
    return rc;
}

// The device-to-host copies of the results of problems p0 .. p0 + np - 1
// (one run: outcomes at bases start[p], tally slots p) on stream s.  Each
// result array of a run is contiguous on the device, so the problems whose
// host destinations are contiguous too go in one copy.
static int copy_results(gbmc_ctx* c, int32_t p0, int32_t np, const std::vector<int64_t>& start,
                        const std::vector<int64_t>& nn, const gbmc_host_results* dst,
                        cudaStream_t s) {
    char* pd = nullptr;          // pending copy: host destination, device source, bytes
    const char* ps = nullptr;
    size_t pb = 0;
    auto flush = [&]() -> int {
        if (pd && pb) CK(cudaMemcpyAsync(pd, ps, pb, cudaMemcpyDeviceToHost, s));
        pd = nullptr;
        ps = nullptr;
        pb = 0;
        return GBMC_OK;
    };
    // one result array: dst_of(p) host pointer, src_of(p) device pointer, bytes_of(p)
    auto field = [&](auto dst_of, auto src_of, auto bytes_of) -> int {
        for (int32_t p = p0; p < p0 + np; ++p) {
            char* d = (char*)dst_of(p);
            const char* sp = (const char*)src_of(p);
            const size_t b = bytes_of(p);
            if (d && b && pd && d == pd + pb && sp == ps + pb) {
                pb += b;
                continue;
            }
            int rc = flush();
            if (rc) return rc;
            if (d && b) {
                pd = d;
                ps = sp;
                pb = b;
            }
        }
        return flush();
    };
    const Outcomes& O = c->O;
    auto n_of = [&](int32_t p) { return (size_t)nn[p]; };
    int rc = 0;
#define GBMC_OUTCOME_FIELD(member, arr, T)                                                    \
    if (!rc)                                                                                    \
        rc = field([&](int32_t p) { return (void*)dst[p].member; },                             \
                   [&](int32_t p) { return (const void*)(O.arr + start[p]); },                  \
                   [&](int32_t p) { return sizeof(T) * n_of(p); });
    GBMC_OUTCOME_FIELD(n_coll, ncoll, int32_t)
    GBMC_OUTCOME_FIELD(status, status, int8_t)
    GBMC_OUTCOME_FIELD(n_flights, nflt, int32_t)
    GBMC_OUTCOME_FIELD(n_draws, ndraw, uint32_t)
    GBMC_OUTCOME_FIELD(E, E, double)
    GBMC_OUTCOME_FIELD(x, x, double)
    GBMC_OUTCOME_FIELD(y, y, double)
    GBMC_OUTCOME_FIELD(z, z, double)
#undef GBMC_OUTCOME_FIELD
    if (!rc)
        rc = field([&](int32_t p) { return (void*)dst[p].flux; },
                   [&](int32_t p) { return (const void*)(c->Y.flux + c->slot_flux_off[p]); },
                   [&](int32_t p) {
                       return sizeof(double) * (size_t)c->slot_cells[p] * (size_t)c->n_bins;
                   });
    if (!rc)
        rc = field([&](int32_t p) { return (void*)dst[p].counts; },
                   [&](int32_t p) { return (const void*)(c->Y.counts + (size_t)p * GBMC_NSCAL); },
                   [&](int32_t) { return sizeof(int64_t) * GBMC_NSCAL; });
    if (!rc)
        rc = field([&](int32_t p) { return (void*)dst[p].weights; },
                   [&](int32_t p) { return (const void*)(c->Y.weights + (size_t)p * GBMC_NSCAL); },
                   [&](int32_t) { return sizeof(double) * GBMC_NSCAL; });
    return rc;
}

static int run_concurrent(gbmc_ctx* c, int32_t n_prob, const gbmc_problem* probs, int32_t n_loops,
                          int32_t per_run, const gbmc_host_results* dst, void* stream);

int gbmc_run_concurrent(gbmc_ctx* c, int32_t n_prob, const gbmc_problem* probs, int32_t n_loops,
                        int32_t per_run, void* stream) {
    return run_concurrent(c, n_prob, probs, n_loops, per_run, nullptr, stream);
}

int gbmc_host_alloc(size_t bytes, void** ptr) {
    if (!ptr || bytes == 0) return GBMC_ERR_INVALID_ARG;
    *ptr = nullptr;
    void* p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocDefault) != cudaSuccess || !p) {
        cudaGetLastError();   // clear the runtime's last-error state
        return GBMC_ERR_OOM;
    }
    *ptr = p;
    return GBMC_OK;
}

int gbmc_host_free(void* ptr) {
    if (!ptr) return GBMC_OK;
    return cudaFreeHost(ptr) == cudaSuccess ? GBMC_OK : GBMC_ERR_CUDA;
}

int gbmc_run_concurrent_to_host(gbmc_ctx* c, int32_t n_prob, const gbmc_problem* probs,
                                int32_t n_loops, int32_t per_run, const gbmc_host_results* dst,
                                void* stream) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (!dst) return fail(c, GBMC_ERR_INVALID_ARG, "dst required");
    return run_concurrent(c, n_prob, probs, n_loops, per_run, dst, stream);
}

static int run_concurrent(gbmc_ctx* c, int32_t n_prob, const gbmc_problem* probs, int32_t n_loops,
                          int32_t per_run, const gbmc_host_results* dst, void* stream) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (c->borrowed) return fail(c, GBMC_ERR_UNSUPPORTED, "a concurrent loop runs no loops itself");
    if (n_prob < 1 || !probs) return fail(c, GBMC_ERR_INVALID_ARG, "n_prob >= 1 and probs required");
    if (n_loops < 1 || n_loops > kMaxLoops)
        return fail(c, GBMC_ERR_INVALID_ARG, "n_loops must be in [1, %d]", kMaxLoops);
    if (per_run < 1) return fail(c, GBMC_ERR_INVALID_ARG, "per_run must be at least 1");
    if (!c->n_nuc || !c->n_mat || !c->n_bins)
        return fail(c, GBMC_ERR_NOT_INITIALIZED, "tables, materials and tally must be set first");
    if ((c->opt.precision == GBMC_FP64 && !c->has64) || (c->opt.precision == GBMC_FP32 && !c->has32))
        return fail(c, GBMC_ERR_NOT_INITIALIZED, "tables not loaded in the selected precision");
    if (c->ww_on || c->eig_on || c->imp_on)
        return fail(c, GBMC_ERR_UNSUPPORTED,
                    "weight windows, k-eigenvalue banking and importance recording run in one "
                    "event loop (gbmc_run_problems)");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = set_device(c);
    if (rc) return rc;
    // every problem validated and laid out as gbmc_run_problems would
    std::vector<int32_t> cells(n_prob);
    std::vector<int64_t> start(n_prob), nn(n_prob);
    int64_t total = 0;
    for (int32_t p = 0; p < n_prob; ++p) {
        if ((rc = check_geometry(c, probs[p].geom, p))) return rc;
        if (probs[p].n_particles < 0 || probs[p].first_id < 0 ||
            probs[p].first_id > std::numeric_limits<int64_t>::max() - probs[p].n_particles)
            return fail(c, GBMC_ERR_INVALID_ARG, "problem %d: bad particle range", p);
        if (probs[p].geom.source == GBMC_SRC_BANK)
            return fail(c, GBMC_ERR_UNSUPPORTED, "problem %d: bank sources run in one event loop", p);
        cells[p] = n_cells_of(probs[p].geom);
        start[p] = total;
        nn[p] = probs[p].n_particles;
        total += probs[p].n_particles;
        if (total > ((int64_t)1 << 40))
            return fail(c, GBMC_ERR_INVALID_ARG, "more than 2^40 particles in one call");
    }
    if (c->ran) CK(cudaStreamSynchronize(c->last_stream));
    if ((rc = ensure_outcomes(c, total > 0 ? total : 1))) return rc;
    if ((rc = ensure_tallies(c, cells, s))) return rc;
    while ((int32_t)c->loops.size() < n_loops) {
        gbmc_ctx* l = nullptr;
        if ((rc = gbmc_create(&l, c->device, &c->opt)))
            return fail(c, rc, "concurrent loop: %s", gbmc_last_error(nullptr));
        l->borrowed = true;
        cudaError_t e = cudaStreamCreateWithFlags(&l->own_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l->done_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&l->copy_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l->run_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l->copied_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            gbmc_destroy(l);
            return fail(c, GBMC_ERR_CUDA, "concurrent loop stream: %s", cudaGetErrorString(e));
        }
        c->loops.push_back(l);
    }
    for (int32_t j = 0; j < n_loops; ++j) borrow_from(c->loops[j], c);
    c->run_start = start;
    c->run_n = nn;
    const int32_t n_runs = (n_prob + per_run - 1) / per_run;
    const int32_t used = std::min(n_loops, n_runs);
    CK(cudaEventRecord(c->ev0, s));
    for (int32_t j = 0; j < used; ++j) CK(cudaStreamWaitEvent(c->loops[j]->own_stream, c->ev0, 0));
    // runs of per_run consecutive problems, run r on loop r % n_loops,
    // enqueued round by round so that every loop has work queued
    std::vector<int64_t> fo(per_run), ob(per_run);
    std::vector<int32_t> sl(per_run);
    int erc = GBMC_OK;
    for (int32_t r = 0; r < n_runs && erc == GBMC_OK; ++r) {
        gbmc_ctx* l = c->loops[r % n_loops];
        const int32_t p0 = r * per_run, np = std::min(per_run, n_prob - p0);
        for (int32_t k = 0; k < np; ++k) {
            fo[k] = c->slot_flux_off[p0 + k];
            ob[k] = start[p0 + k];
            sl[k] = p0 + k;
        }
        RunLayout lay{fo.data(), ob.data(), sl.data(), r >= n_loops};
        erc = launch_run(l, np, probs + p0, l->own_stream, &lay);
        if (erc) {
            c->err = std::string("concurrent loop ") + std::to_string(r % n_loops) + ": " + l->err;
        } else if (dst) {
            // this run's results to the host on the loop's copy stream: they
            // overlap the loop's next run and the other loops
            CK(cudaEventRecord(l->run_ev, l->own_stream));
            CK(cudaStreamWaitEvent(l->copy_stream, l->run_ev, 0));
            erc = copy_results(c, p0, np, start, nn, dst, l->copy_stream);
        }
    }
    // join: `stream` waits for every loop and its copies (also after a
    // failed launch, so that nothing a loop queued outlives the call unseen)
    for (int32_t j = 0; j < used; ++j) {
        CK(cudaEventRecord(c->loops[j]->done_ev, c->loops[j]->own_stream));
        CK(cudaStreamWaitEvent(s, c->loops[j]->done_ev, 0));
        if (dst) {
            CK(cudaEventRecord(c->loops[j]->copied_ev, c->loops[j]->copy_stream));
            CK(cudaStreamWaitEvent(s, c->loops[j]->copied_ev, 0));
        }
    }
    CK(cudaEventRecord(c->ev1, s));
    c->ran = true;
    c->last_stream = s;
    c->last_loops = used;
    return erc;
}

int gbmc_profile_problems(gbmc_ctx* c, int32_t n_prob, const gbmc_problem* probs, void* stream,
                          gbmc_kernel_times* out, int32_t trace_cap, double* trace_ms,
                          int32_t* trace_queues, int32_t* trace_len) {
    if (!c || !out) return GBMC_ERR_INVALID_ARG;
    if (trace_cap < 0) return fail(c, GBMC_ERR_INVALID_ARG, "trace_cap must be >= 0");
    if (trace_len) *trace_len = 0;
    cudaStream_t s = (cudaStream_t)stream;
    Params P;
    LaunchCfg L;
    int rc = prepare_run(c, n_prob, probs, s, &P, &L);
    if (rc) return rc;
    P.use_cond = 0;
    c->last_loops = 0;
    cudaEvent_t ev[kTimedKernels + 1];
    for (int k = 0; k <= kTimedKernels; ++k) CK(cudaEventCreate(&ev[k]));
    cudaError_t e = launch_init_run(P, L, s);
    int it = 0;
    while (e == cudaSuccess) {
        e = launch_iteration_timed(P, L, s, ev);
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) break;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        for (int k = 0; k < kIterKernels; ++k) {
            float ms = 0;
            e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            if (e != cudaSuccess) break;
            bool launched = (k < 2 || k > 3 || P.sort);
            out->ms[k] += ms;
            out->launches[k] += launched ? 1 : 0;
            if (trace_ms && it < trace_cap) trace_ms[(int64_t)it * kTimedKernels + k] = ms;
        }
        if (trace_queues && it < trace_cap) {
            const Ctl& k = *c->h_ctl;
            int32_t* tq = trace_queues + (int64_t)it * 4;
            tq[0] = k.lookup_n;
            tq[1] = k.adv_n;
            tq[2] = k.n_cq;
            tq[3] = k.M - k.n_free;
        }
        if (trace_len && it < trace_cap) *trace_len = it + 1;
        if (c->h_ctl->done || ++it > c->opt.max_iterations + 1) break;
    }
    if (e == cudaSuccess) {
        // the tail kernel (a no-op unless the loop stopped early)
        cudaEventRecord(ev[0], s);
        e = launch_tail(P, L, s);
        if (e == cudaSuccess && P.sites) e = launch_bank(P, L, s);
        cudaEventRecord(ev[1], s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        out->ms[kTimedKernels - 1] += ms;
        out->launches[kTimedKernels - 1] += 1;
    }
    for (int k = 0; k <= kTimedKernels; ++k) cudaEventDestroy(ev[k]);
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "profiled run: %s", cudaGetErrorString(e));
    c->ran = true;
    c->last_stream = s;
    CK(cudaEventRecord(c->ev0, s));
    CK(cudaEventRecord(c->ev1, s));
    return GBMC_OK;
}

int gbmc_run_batch(gbmc_ctx* c, const gbmc_problem* prob, void* stream) {
    return gbmc_run_problems(c, 1, prob, stream);
}

int gbmc_read_tallies(gbmc_ctx* c, int32_t slot, double* flux, int64_t n_flux, int64_t* counts,
                      double* weights) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    int rc = set_device(c);
    if (rc) return rc;
    if ((rc = read_ctl(c))) return rc;
    if (slot < 0 || slot >= (int32_t)c->slot_cells.size())
        return fail(c, GBMC_ERR_INVALID_ARG, "tally slot %d out of range", slot);
    int64_t nf = (int64_t)c->slot_cells[slot] * c->n_bins;
    if (flux) {
        if (n_flux != nf)
            return fail(c, GBMC_ERR_INVALID_ARG, "n_flux must be %lld", (long long)nf);
        CK(cudaMemcpy(flux, c->Y.flux + c->slot_flux_off[slot], sizeof(double) * nf,
                      cudaMemcpyDeviceToHost));
    }
    if (counts) {
        static_assert(sizeof(unsigned long long) == sizeof(int64_t), "count width");
        CK(cudaMemcpy(counts, c->Y.counts + (size_t)slot * GBMC_NSCAL,
                      sizeof(int64_t) * GBMC_NSCAL, cudaMemcpyDeviceToHost));
    }
    if (weights)
        CK(cudaMemcpy(weights, c->Y.weights + (size_t)slot * GBMC_NSCAL,
                      sizeof(double) * GBMC_NSCAL, cudaMemcpyDeviceToHost));
    return GBMC_OK;
}

int gbmc_set_reaction_tally(gbmc_ctx* c, int32_t on) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (on != 0 && on != 1) return fail(c, GBMC_ERR_INVALID_ARG, "on must be 0 or 1");
    int rc = set_device(c);
    if (rc) return rc;
    if ((bool)on == c->rr_on) return GBMC_OK;
    c->rr_on = on != 0;
    c->graph_valid = false;
    if (!c->rr_on) {
        dfree(c->Y.absrate);
        c->Y.absrate = nullptr;
    } else if (c->Y.flux) {
        if ((rc = dalloc(c, &c->Y.absrate, (size_t)c->flux_cap))) return rc;
        CK(cudaMemset(c->Y.absrate, 0, sizeof(double) * (size_t)c->flux_cap));
    }
    return GBMC_OK;
}

int gbmc_read_reaction_tally(gbmc_ctx* c, int32_t slot, double* absrate, int64_t n) {
    if (!c || !absrate) return GBMC_ERR_INVALID_ARG;
    int rc = set_device(c);
    if (rc) return rc;
    if (!c->rr_on || !c->Y.absrate)
        return fail(c, GBMC_ERR_NOT_INITIALIZED, "the absorption-rate tally is off or has not run");
    if ((rc = read_ctl(c))) return rc;
    if (slot < 0 || slot >= (int32_t)c->slot_cells.size())
        return fail(c, GBMC_ERR_INVALID_ARG, "tally slot %d out of range", slot);
    int64_t nf = (int64_t)c->slot_cells[slot] * c->n_bins;
    if (n != nf) return fail(c, GBMC_ERR_INVALID_ARG, "n must be %lld", (long long)nf);
    CK(cudaMemcpy(absrate, c->Y.absrate + c->slot_flux_off[slot], sizeof(double) * nf,
                  cudaMemcpyDeviceToHost));
    return GBMC_OK;
}

int gbmc_load_fission(gbmc_ctx* c, int32_t n_nuc, const double* nu, const double* f_fis) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (!c->n_nuc) return fail(c, GBMC_ERR_NOT_INITIALIZED, "load the tables first");
    if (n_nuc != c->n_nuc || !nu || !f_fis)
        return fail(c, GBMC_ERR_INVALID_ARG, "need nu and f_fis for the %d loaded nuclides", c->n_nuc);
    for (int32_t i = 0; i < n_nuc; ++i) {
        if (!(nu[i] >= 0) || !std::isfinite(nu[i]))
            return fail(c, GBMC_ERR_INVALID_ARG, "nuclide %d: nu must be finite and >= 0", i);
        if (!(f_fis[i] >= 0) || !(f_fis[i] <= c->h_fabs[i]))
            return fail(c, GBMC_ERR_INVALID_ARG, "nuclide %d: need 0 <= f_fis <= f_abs", i);
    }
    int rc = set_device(c);
    if (rc) return rc;
    if ((rc = upload(c, &c->d_nu, nu, (size_t)n_nuc))) return rc;
    if ((rc = upload(c, &c->d_ffis, f_fis, (size_t)n_nuc))) return rc;
    c->fis_loaded = true;
    c->graph_valid = false;
    return GBMC_OK;
}

int gbmc_set_eigen(gbmc_ctx* c, double k_norm, int32_t max_sites) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (!(k_norm > 0) || !std::isfinite(k_norm)) {
        if (c->eig_on) c->graph_valid = false;
        c->eig_on = false;
        return GBMC_OK;
    }
    if (!c->fis_loaded) return fail(c, GBMC_ERR_NOT_INITIALIZED, "load the fission data first");
    if (max_sites < 1 || max_sites > 255)
        return fail(c, GBMC_ERR_INVALID_ARG, "max_sites must be in [1, 255]");
    if (!c->eig_on || max_sites != c->max_sites) c->graph_valid = false;
    c->eig_on = true;
    c->k_norm = k_norm;
    c->max_sites = max_sites;
    return GBMC_OK;
}

int gbmc_read_bank(gbmc_ctx* c, double* xyz, int64_t n_cap, int64_t* n_out) {
    if (!c || !n_out) return GBMC_ERR_INVALID_ARG;
    int rc = set_device(c);
    if (rc) return rc;
    if (!c->d_bank_size) return fail(c, GBMC_ERR_NOT_INITIALIZED, "no k-eigenvalue run yet");
    if ((rc = read_ctl(c))) return rc;
    int64_t n = 0;
    CK(cudaMemcpy(&n, c->d_bank_size, sizeof n, cudaMemcpyDeviceToHost));
    *n_out = n;
    if (xyz) {
        if (n_cap < n) return fail(c, GBMC_ERR_INVALID_ARG, "need room for %lld sites", (long long)n);
        CK(cudaMemcpy(xyz, c->d_bank_out, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost));
    }
    return GBMC_OK;
}

int gbmc_set_source_bank(gbmc_ctx* c, const double* xyz, int64_t n, int64_t n_total) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    int rc = set_device(c);
    if (rc) return rc;
    if (n_total < 1 || n_total > ((int64_t)1 << 31) - 1)
        return fail(c, GBMC_ERR_INVALID_ARG, "n_total must be in [1, 2^31)");
    if (!xyz) {
        if (!c->d_bank_size) return fail(c, GBMC_ERR_NOT_INITIALIZED, "no k-eigenvalue run yet");
        if ((rc = read_ctl(c))) return rc;
        CK(cudaMemcpy(&n, c->d_bank_size, sizeof n, cudaMemcpyDeviceToHost));
    } else {
        for (int64_t i = 0; i < 3 * n; ++i)
            if (!std::isfinite(xyz[i])) return fail(c, GBMC_ERR_INVALID_ARG, "bank coordinate not finite");
    }
    if (n < 1 || n > ((int64_t)1 << 31) - 1)
        return fail(c, GBMC_ERR_INVALID_ARG, "the bank must hold 1 to 2^31 - 1 sites");
    if (n > c->src_cap) {
        if ((rc = dalloc(c, &c->d_bank_src, (size_t)n * 3))) return rc;
        c->src_cap = n;
        c->graph_valid = false;
    }
    if (xyz)
        CK(cudaMemcpy(c->d_bank_src, xyz, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice));
    else
        CK(cudaMemcpy(c->d_bank_src, c->d_bank_out, sizeof(double) * 3 * (size_t)n,
                      cudaMemcpyDeviceToDevice));
    c->src_n = n;
    c->src_total = n_total;
    return GBMC_OK;
}

int gbmc_check_division(gbmc_ctx* c, int32_t kind, int64_t n, uint64_t seed, int64_t* n_bad,
                        double* first_bad) {
    if (!c || !n_bad || n < 0 || kind < 0 || kind > 1) return GBMC_ERR_INVALID_ARG;
    int rc = set_device(c);
    if (rc) return rc;
    unsigned long long* d_bad = nullptr;
    double* d_first = nullptr;
    double *d_e0 = nullptr, *d_e1 = nullptr;
    Interval64* d_iv = nullptr;
    auto release = [&]() {
        dfree(d_bad);
        dfree(d_first);
        dfree(d_e0);
        dfree(d_e1);
        dfree(d_iv);
    };
    if ((rc = dalloc(c, &d_bad, 1)) || (rc = dalloc(c, &d_first, 2))) {
        release();
        return rc;
    }
    const int32_t K = 1 << 16;
    if (kind == 1) {
        // grid-like intervals: e0 log-uniform on [1e-6, 1e8] eV, relative
        // widths from 2^-52 to 2^14, one in 64 of zero width (a repeated point)
        uint64_t st = seed ^ 0x9E3779B97F4A7C15ull;
        auto next = [&st]() {   // splitmix64
            uint64_t z = (st += 0x9E3779B97F4A7C15ull);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            return z ^ (z >> 31);
        };
        auto unit = [&next]() { return (double)(next() >> 11) * 0x1.0p-53; };
        std::vector<double> e0(K), e1(K);
        std::vector<Interval64> iv(K);
        for (int32_t j = 0; j < K; ++j) {
            e0[j] = std::pow(10.0, -6.0 + 14.0 * unit());
            double g = std::exp2(j % 3 == 0 ? -52.0 + 66.0 * unit() : -50.0 + 51.0 * unit());
            e1[j] = j % 64 == 63 ? e0[j] : e0[j] * (1.0 + g);
            if (e1[j] == e0[j] && j % 64 != 63) e1[j] = std::nextafter(e0[j], 1e300);
            iv[j] = interval_record(e0[j], e1[j], 1.0, 2.0);
        }
        if ((rc = upload(c, &d_e0, e0.data(), (size_t)K)) || (rc = upload(c, &d_e1, e1.data(), (size_t)K)) ||
            (rc = upload(c, &d_iv, iv.data(), (size_t)K))) {
            release();
            return rc;
        }
    }
    cudaError_t e = cudaMemset(d_bad, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(d_first, 0, 2 * sizeof(double));
    if (e == cudaSuccess)
        e = kind == 0 ? launch_check_division(n, seed, d_bad, d_first, c->sms, 0)
                      : launch_check_interp(n, seed, d_e0, d_e1, d_iv, K, d_bad, d_first, c->sms, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned long long nb = 0;
    double fb[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpy(&nb, d_bad, sizeof nb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(fb, d_first, sizeof fb, cudaMemcpyDeviceToHost);
    release();
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "division check: %s", cudaGetErrorString(e));
    *n_bad = (int64_t)nb;
    if (first_bad) {
        first_bad[0] = fb[0];
        first_bad[1] = fb[1];
    }
    return GBMC_OK;
}

int gbmc_measure_fp64_rate(gbmc_ctx* c, double* ops_per_s) {
    if (!c || !ops_per_s) return GBMC_ERR_INVALID_ARG;
    int rc = set_device(c);
    if (rc) return rc;
    const int blocks = c->sms * 8;
    const int32_t iters = 1 << 14;
    double* out = nullptr;
    if ((rc = dalloc(c, &out, (size_t)blocks))) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first warms up
        e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess) e = launch_fp64_rate(blocks, iters, out, 0);
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(out);
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "rate probe: %s", cudaGetErrorString(e));
    *ops_per_s = (double)blocks * 256.0 * 8.0 * (double)iters / (best * 1e-3);
    return GBMC_OK;
}

int gbmc_read_outcomes(gbmc_ctx* c, int32_t slot, int64_t first, int64_t n, int32_t* n_coll,
                       int8_t* status, int32_t* n_flights, uint32_t* n_draws, double* E, double* x,
                       double* y, double* z) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    int rc = set_device(c);
    if (rc) return rc;
    if ((rc = read_ctl(c))) return rc;
    if (slot < 0 || slot >= (int32_t)c->run_start.size())
        return fail(c, GBMC_ERR_INVALID_ARG, "problem slot %d out of range", slot);
    if (first < 0 || n < 0 || first + n > c->run_n[slot])
        return fail(c, GBMC_ERR_INVALID_ARG, "particle range outside the problem's batch");
    int64_t o = c->run_start[slot] + first;
    if (n == 0) return GBMC_OK;
    if (n_coll) CK(cudaMemcpy(n_coll, c->O.ncoll + o, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    if (status) CK(cudaMemcpy(status, c->O.status + o, sizeof(int8_t) * n, cudaMemcpyDeviceToHost));
    if (n_flights) CK(cudaMemcpy(n_flights, c->O.nflt + o, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    if (n_draws) CK(cudaMemcpy(n_draws, c->O.ndraw + o, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    if (E) CK(cudaMemcpy(E, c->O.E + o, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (x) CK(cudaMemcpy(x, c->O.x + o, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (y) CK(cudaMemcpy(y, c->O.y + o, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (z) CK(cudaMemcpy(z, c->O.z + o, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return GBMC_OK;
}

int gbmc_read_stats(gbmc_ctx* c, gbmc_stats* out) {
    if (!c || !out) return GBMC_ERR_INVALID_ARG;
    int rc = set_device(c);
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    rc = read_ctl(c);
    if (rc && rc != GBMC_ERR_TIMEOUT && rc != GBMC_ERR_DEVICE_FLAG) return rc;
    const RunStats& k = *c->h_stats;
    out->iterations = (int64_t)k.iterations;
    out->lookups = (int64_t)k.lookups;
    out->micro_lookups = (int64_t)k.micro;
    out->flights = (int64_t)k.flights;
    out->crossings = (int64_t)k.cross;
    out->collisions = (int64_t)k.coll;
    out->histories = (int64_t)k.hist;
    out->handoffs = (int64_t)k.handoff;
    out->device_error = rc == GBMC_ERR_TIMEOUT ? GBMC_ERR_TIMEOUT
                      : rc == GBMC_ERR_DEVICE_FLAG ? GBMC_ERR_DEVICE_FLAG : 0;
    return rc;
}

int gbmc_last_run_ms(gbmc_ctx* c, double* ms) {
    if (!c || !ms) return GBMC_ERR_INVALID_ARG;
    if (!c->ran) return fail(c, GBMC_ERR_NOT_INITIALIZED, "no run has been launched");
    int rc = set_device(c);
    if (rc) return rc;
    CK(cudaEventSynchronize(c->ev1));
    float f = 0;
    CK(cudaEventElapsedTime(&f, c->ev0, c->ev1));
    *ms = f;
    return GBMC_OK;
}

int gbmc_lookup_macro(gbmc_ctx* c, int32_t precision, const double* d_E, const int32_t* d_mat,
                      int64_t n, double* d_sigma_t, double* d_sigma_a, int32_t sort, void* stream) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!d_E || !d_mat || !d_sigma_t || !d_sigma_a)))
        return fail(c, GBMC_ERR_INVALID_ARG, "n >= 0 and device arrays required");
    if (n > ((int64_t)1 << 31) - 1) return fail(c, GBMC_ERR_INVALID_ARG, "n must be < 2^31");
    if (precision != GBMC_FP64 && precision != GBMC_FP32)
        return fail(c, GBMC_ERR_INVALID_ARG, "precision must be GBMC_FP64 or GBMC_FP32");
    if (!c->n_nuc || !c->n_mat) return fail(c, GBMC_ERR_NOT_INITIALIZED, "tables and materials required");
    if ((precision == GBMC_FP64 && !c->has64) || (precision == GBMC_FP32 && !c->has32))
        return fail(c, GBMC_ERR_NOT_INITIALIZED, "tables not loaded in that precision");
    if (n == 0) return GBMC_OK;
    int rc = set_device(c);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (sort > 0 && n > c->q_cap) {
        if (c->ran) CK(cudaStreamSynchronize(c->last_stream));
        CK(cudaDeviceSynchronize());
        if ((rc = dalloc(c, &c->q_perm, (size_t)n))) return rc;
        if ((rc = dalloc(c, &c->q_keys, (size_t)n))) return rc;
        c->q_cap = n;
    }
    if (sort > 0 && !c->q_hist) {
        if ((rc = dalloc(c, &c->q_hist, kSortBuckets))) return rc;
        if ((rc = dalloc(c, &c->q_cursor, kSortBuckets))) return rc;
        if ((rc = dalloc(c, &c->q_btot, kSortBuckets / 1024))) return rc;
        CK(cudaMemset(c->q_hist, 0, sizeof(uint32_t) * kSortBuckets));
    }
    Params P = make_params(c);
    P.precision = precision;
    LaunchCfg L = make_launch(c);
    cudaError_t e = launch_query_lookup(P, L, d_E, d_mat, n, d_sigma_t, d_sigma_a,
                                        sort > 0 ? c->q_perm : nullptr, c->q_keys, c->q_hist,
                                        c->q_cursor, c->q_btot, s);
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "lookup launch: %s", cudaGetErrorString(e));
    return GBMC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Weight windows.

extern "C" int gbmc_set_weight_windows(gbmc_ctx* c, int32_t n_cells, int32_t n_bins,
                                       const double* lower, double ratio, double survival,
                                       int32_t max_split) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (!c->n_bins) return fail(c, GBMC_ERR_NOT_INITIALIZED, "set the tally bins first");
    if (n_cells < 1 || n_bins != c->n_bins || !lower)
        return fail(c, GBMC_ERR_INVALID_ARG, "need n_cells >= 1, n_bins = the tally's bins, lower");
    if (!(survival >= 1.0) || !(ratio >= 2.0 * survival) || !std::isfinite(ratio))
        return fail(c, GBMC_ERR_INVALID_ARG, "need survival >= 1 and ratio >= 2 * survival");
    if (max_split < 2 || max_split > 1000)
        return fail(c, GBMC_ERR_INVALID_ARG, "max_split must be in [2, 1000]");
    int64_t n = (int64_t)n_cells * n_bins;
    for (int64_t k = 0; k < n; ++k)
        if (!(lower[k] >= 0.0) || !std::isfinite(lower[k]))
            return fail(c, GBMC_ERR_INVALID_ARG, "window bounds must be finite and >= 0");
    int rc = set_device(c);
    if (rc) return rc;
    if (c->ran) CK(cudaStreamSynchronize(c->last_stream));
    if ((rc = upload(c, &c->d_ww, lower, (size_t)n))) return rc;
    c->ww_on = true;
    c->ww_cells = n_cells;
    c->ww_ratio = ratio;
    c->ww_survival = survival;
    c->ww_max_split = max_split;
    c->graph_valid = false;
    return GBMC_OK;
}

extern "C" int gbmc_get_weight_windows(gbmc_ctx* c, double* lower, int64_t n) {
    if (!c || !lower) return GBMC_ERR_INVALID_ARG;
    if (!c->ww_on) return fail(c, GBMC_ERR_NOT_INITIALIZED, "no weight windows set");
    int64_t need = (int64_t)c->ww_cells * c->n_bins;
    if (n != need) return fail(c, GBMC_ERR_INVALID_ARG, "n must be %lld", (long long)need);
    int rc = set_device(c);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(lower, c->d_ww, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return GBMC_OK;
}

extern "C" int gbmc_clear_weight_windows(gbmc_ctx* c) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (c->ww_on) c->graph_valid = false;
    c->ww_on = false;
    return GBMC_OK;
}

// ---------------------------------------------------------------------------
// Importance network and importance estimates.

namespace {

int need_net(gbmc_ctx* c) {
    if (!c->net_set) return fail(c, GBMC_ERR_NOT_INITIALIZED, "set the importance network first");
    if (c->mlp_dead)
        return fail(c, GBMC_ERR_TIMEOUT,
                    "an earlier network forward never completed on the tensor cores; "
                    "create a new context");
    return GBMC_OK;
}

// Waits for stream s and reports (and clears) a tensor-core wait that gave
// up in the network forward.  Flag 2: the products never arrived, so a CTA
// kept its tensor memory; the network is refused from then on.
int mlp_status(gbmc_ctx* c, cudaStream_t s) {
    CK(cudaStreamSynchronize(s));
    int flag = 0;
    CK(cudaMemcpy(&flag, c->d_mlp_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CK(cudaMemset(c->d_mlp_err, 0, sizeof(int)));
        if (flag >= 2) c->mlp_dead = true;
        return fail(c, GBMC_ERR_TIMEOUT, "network forward: tensor-core wait gave up");
    }
    return GBMC_OK;
}

int ensure_mesh(gbmc_ctx* c, int64_t n) {
    if (n <= c->mesh_cap) return GBMC_OK;
    int rc = dalloc(c, &c->d_mesh_feat, (size_t)n * 4);
    if (rc) return rc;
    if ((rc = dalloc(c, &c->d_mesh_out, (size_t)n))) return rc;
    c->mesh_cap = n;
    return GBMC_OK;
}

MeshSpec mesh_of(const gbmc_ctx* c, const gbmc_geometry& g) {
    MeshSpec M{};
    M.g = g;
    M.n_cells = n_cells_of(g);
    M.n_bins = c->n_bins;
    M.edges = c->d_edges;
    for (int i = 0; i < 4; ++i) {
        M.offset[i] = c->feat_offset[i];
        M.scale[i] = c->feat_scale[i];
    }
    return M;
}

}  // namespace

extern "C" int gbmc_set_importance_net(gbmc_ctx* c, const uint16_t* bf16_params, int32_t n_params,
                                       const double* feat_offset, const double* feat_scale) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (!bf16_params || n_params != kMlpParams || !feat_offset || !feat_scale)
        return fail(c, GBMC_ERR_INVALID_ARG, "need %d BF16 parameters and 4 offsets, 4 scales",
                    kMlpParams);
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(feat_offset[i]) || !std::isfinite(feat_scale[i]))
            return fail(c, GBMC_ERR_INVALID_ARG, "feature offsets and scales must be finite");
    int rc = set_device(c);
    if (rc) return rc;
    std::vector<float> p(kMlpParams);
    for (int k = 0; k < kMlpParams; ++k) {
        uint32_t b = (uint32_t)bf16_params[k] << 16;
        memcpy(&p[k], &b, 4);
        if (!std::isfinite(p[k])) return fail(c, GBMC_ERR_INVALID_ARG, "parameter %d not finite", k);
    }
    std::vector<float> zero(kMlpParams, 0.f);
    if ((rc = upload(c, &c->d_net_p, p.data(), p.size()))) return rc;
    if ((rc = upload(c, &c->d_net_m, zero.data(), zero.size()))) return rc;
    if ((rc = upload(c, &c->d_net_v, zero.data(), zero.size()))) return rc;
    if ((rc = upload(c, &c->d_net_g, zero.data(), zero.size()))) return rc;
    if ((rc = upload(c, &c->d_net_w, reinterpret_cast<const __nv_bfloat16*>(bf16_params),
                     (size_t)kMlpParams)))
        return rc;
    if (!c->d_net_scratch && (rc = dalloc(c, &c->d_net_scratch, 2))) return rc;
    if (!c->d_mlp_err) {
        if ((rc = dalloc(c, &c->d_mlp_err, 1))) return rc;
        CK(cudaMemset(c->d_mlp_err, 0, sizeof(int)));
    }
    for (int i = 0; i < 4; ++i) {
        c->feat_offset[i] = feat_offset[i];
        c->feat_scale[i] = feat_scale[i];
    }
    c->net_step = 0;
    c->net_set = true;
    return GBMC_OK;
}

extern "C" int gbmc_get_importance_net(gbmc_ctx* c, uint16_t* bf16_params, int32_t n_params) {
    if (!c || !bf16_params || n_params != kMlpParams) return GBMC_ERR_INVALID_ARG;
    int rc = need_net(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(bf16_params, c->d_net_w, sizeof(uint16_t) * kMlpParams, cudaMemcpyDeviceToHost));
    return GBMC_OK;
}

extern "C" int gbmc_mlp_forward(gbmc_ctx* c, const float* d_feat, int64_t n, float* d_out,
                                void* stream) {
    if (!c || n < 0 || (n > 0 && (!d_feat || !d_out))) return GBMC_ERR_INVALID_ARG;
    int rc = need_net(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    cudaError_t e = mlp_forward(c->d_net_w, d_feat, n, d_out, c->d_mlp_err, c->sms,
                                (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "network forward: %s", cudaGetErrorString(e));
    return mlp_status(c, (cudaStream_t)stream);
}

extern "C" int gbmc_mlp_gradient(gbmc_ctx* c, const float* d_feat, const float* d_target,
                                 const float* d_weight, int64_t n, float* grad_host,
                                 float* loss_host, void* stream) {
    if (!c || n < 1 || !d_feat || !d_target || !d_weight) return GBMC_ERR_INVALID_ARG;
    int rc = need_net(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(c->d_net_g, 0, sizeof(float) * kMlpParams, s));
    CK(cudaMemsetAsync(c->d_net_scratch, 0, sizeof(float) * 2, s));
    cudaError_t e = mlp_grad(c->d_net_w, d_feat, d_target, d_weight, n, c->d_net_scratch,
                             c->d_net_g, c->d_net_scratch + 1, c->sms, s);
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "network gradient: %s", cudaGetErrorString(e));
    CK(cudaStreamSynchronize(s));
    if (grad_host)
        CK(cudaMemcpy(grad_host, c->d_net_g, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
    if (loss_host) CK(cudaMemcpy(loss_host, c->d_net_scratch + 1, sizeof(float), cudaMemcpyDeviceToHost));
    CK(cudaMemsetAsync(c->d_net_g, 0, sizeof(float) * kMlpParams, s));
    return GBMC_OK;
}

extern "C" int gbmc_mlp_train(gbmc_ctx* c, const float* d_feat, const float* d_target,
                              const float* d_weight, int64_t n, int32_t steps, float lr,
                              float* loss_host, void* stream) {
    if (!c || n < 1 || steps < 1 || !(lr > 0) || !d_feat || !d_target || !d_weight)
        return GBMC_ERR_INVALID_ARG;
    int rc = need_net(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(c->d_net_g, 0, sizeof(float) * kMlpParams, s));
    for (int32_t k = 0; k < steps; ++k) {
        CK(cudaMemsetAsync(c->d_net_scratch, 0, sizeof(float) * 2, s));
        cudaError_t e = mlp_grad(c->d_net_w, d_feat, d_target, d_weight, n, c->d_net_scratch,
                                 c->d_net_g, c->d_net_scratch + 1, c->sms, s);
        if (e == cudaSuccess)
            e = mlp_adam(c->d_net_p, c->d_net_m, c->d_net_v, c->d_net_g, c->d_net_w, kMlpParams,
                         lr, ++c->net_step, s);
        if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "training step: %s", cudaGetErrorString(e));
    }
    CK(cudaStreamSynchronize(s));
    if (loss_host) CK(cudaMemcpy(loss_host, c->d_net_scratch + 1, sizeof(float), cudaMemcpyDeviceToHost));
    return GBMC_OK;
}

extern "C" int gbmc_mesh_features(gbmc_ctx* c, const gbmc_geometry* g, float* d_feat, int64_t n_cap,
                                  int64_t* n_out, void* stream) {
    if (!c || !g || !n_out) return GBMC_ERR_INVALID_ARG;
    if (!c->n_bins) return fail(c, GBMC_ERR_NOT_INITIALIZED, "set the tally bins first");
    int64_t n = (int64_t)n_cells_of(*g) * c->n_bins;
    *n_out = n;
    if (!d_feat) return GBMC_OK;
    if (n_cap < n) return fail(c, GBMC_ERR_INVALID_ARG, "need room for %lld feature rows", (long long)n);
    int rc = need_net(c);   // the features use the network's feature map
    if (rc) return rc;
    rc = set_device(c);
    if (rc) return rc;
    cudaError_t e = mesh_features(mesh_of(c, *g), d_feat, c->sms, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "mesh features: %s", cudaGetErrorString(e));
    return GBMC_OK;
}

extern "C" int gbmc_weight_windows_from_net(gbmc_ctx* c, const gbmc_geometry* g, double ratio,
                                            double survival, int32_t max_split, void* stream) {
    if (!c || !g) return GBMC_ERR_INVALID_ARG;
    int rc = need_net(c);
    if (rc) return rc;
    if (!c->n_bins) return fail(c, GBMC_ERR_NOT_INITIALIZED, "set the tally bins first");
    if (!(survival >= 1.0) || !(ratio >= 2.0 * survival) || max_split < 2 || max_split > 1000)
        return fail(c, GBMC_ERR_INVALID_ARG, "need survival >= 1, ratio >= 2 survival, max_split in [2, 1000]");
    if ((rc = set_device(c))) return rc;
    MeshSpec M = mesh_of(c, *g);
    int64_t n = (int64_t)M.n_cells * M.n_bins;
    if ((rc = ensure_mesh(c, n))) return rc;
    // source cell (the slab's first layer, the infinite medium's one cell,
    // the lattice's first cell) and the source energy's bin
    int64_t b = 0;
    while (b + 1 < c->n_bins && c->h_edges[b + 1] <= g->E0) ++b;
    int64_t src = b;
    if (c->ran) CK(cudaStreamSynchronize(c->last_stream));
    if (!c->d_ww || c->ww_cells != M.n_cells) {
        if ((rc = dalloc(c, &c->d_ww, (size_t)n))) return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = mesh_windows(M, c->d_net_w, c->d_mesh_feat, c->d_mesh_out, survival, src,
                                 c->d_ww, c->d_mlp_err, c->sms, s);
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "windows from network: %s", cudaGetErrorString(e));
    if ((rc = mlp_status(c, s))) return rc;
    c->ww_on = true;
    c->ww_cells = M.n_cells;
    c->ww_ratio = ratio;
    c->ww_survival = survival;
    c->ww_max_split = max_split;
    c->graph_valid = false;
    return GBMC_OK;
}

extern "C" int gbmc_importance_record(gbmc_ctx* c, const gbmc_geometry* g, int64_t capacity) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (!g || capacity <= 0) {
        if (c->imp_on) c->graph_valid = false;
        c->imp_on = false;
        return GBMC_OK;
    }
    if (!c->n_bins) return fail(c, GBMC_ERR_NOT_INITIALIZED, "set the tally bins first");
    if (capacity > ((int64_t)1 << 31) - 1) return fail(c, GBMC_ERR_INVALID_ARG, "capacity < 2^31");
    int rc = set_device(c);
    if (rc) return rc;
    if (c->ran) CK(cudaStreamSynchronize(c->last_stream));
    if (capacity > c->imp_cap) {
        if ((rc = dalloc(c, &c->d_imp_mesh, (size_t)capacity))) return rc;
        if ((rc = dalloc(c, &c->d_imp_gidx, (size_t)capacity))) return rc;
        c->imp_cap = (int32_t)capacity;
    }
    int64_t cells = (int64_t)n_cells_of(*g) * c->n_bins;
    if (cells != c->imp_cells || !c->d_imp_cnt) {
        if ((rc = dalloc(c, &c->d_imp_cnt, (size_t)cells))) return rc;
        if ((rc = dalloc(c, &c->d_imp_scr, (size_t)cells))) return rc;
        CK(cudaMemset(c->d_imp_cnt, 0, sizeof(double) * cells));
        CK(cudaMemset(c->d_imp_scr, 0, sizeof(double) * cells));
        c->imp_cells = cells;
    }
    c->imp_on = true;
    c->graph_valid = false;
    return GBMC_OK;
}

extern "C" int gbmc_importance_accumulate(gbmc_ctx* c, void* stream) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (!c->imp_on) return fail(c, GBMC_ERR_NOT_INITIALIZED, "importance recording is off");
    int rc = set_device(c);
    if (rc) return rc;
    if ((rc = read_ctl(c))) return rc;
    if (c->h_ctl->n_imp > c->imp_cap)
        return fail(c, GBMC_ERR_DEVICE_FLAG, "importance sample buffer overflowed (%d > %d)",
                    c->h_ctl->n_imp, c->imp_cap);
    cudaStream_t s = (cudaStream_t)stream;
    Params P = make_params(c);
    cudaError_t e = launch_imp_score(P, c->O.status, c->d_imp_cnt, c->d_imp_scr, c->sms, s);
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "importance scoring: %s", cudaGetErrorString(e));
    CK(cudaStreamSynchronize(s));
    return GBMC_OK;
}

extern "C" int gbmc_importance_training_set(gbmc_ctx* c, const gbmc_geometry* g, float* d_feat,
                                            float* d_target, float* d_weight, int64_t n_cap,
                                            int64_t* n_out, void* stream) {
    if (!c || !g || !n_out) return GBMC_ERR_INVALID_ARG;
    if (!c->d_imp_cnt) return fail(c, GBMC_ERR_NOT_INITIALIZED, "no importance samples");
    int64_t n = (int64_t)n_cells_of(*g) * c->n_bins;
    if (n != c->imp_cells) return fail(c, GBMC_ERR_INVALID_ARG, "geometry differs from the recorded one");
    *n_out = n;
    if (!d_feat) return GBMC_OK;
    if (n_cap < n || !d_target || !d_weight)
        return fail(c, GBMC_ERR_INVALID_ARG, "need room for %lld rows", (long long)n);
    int rc = need_net(c);   // the features use the network's feature map
    if (rc) return rc;
    rc = set_device(c);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t cells = n_cells_of(*g);
    if ((rc = dalloc(c, &c->d_imp_cellsum, 2 * (size_t)cells + 2))) return rc;
    cudaError_t e = mesh_features(mesh_of(c, *g), d_feat, c->sms, s);
    if (e == cudaSuccess)
        e = launch_imp_targets(c->d_imp_cnt, c->d_imp_scr, cells, c->n_bins, c->d_imp_cellsum,
                               d_target, d_weight, c->sms, s);
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "training set: %s", cudaGetErrorString(e));
    return GBMC_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: coordinate descent over launch / queue settings, each candidate
// timed on a scaled-down probe run (CUDA events around the graph launch).

namespace {

int probe_ms(gbmc_ctx* c, const std::vector<gbmc_problem>& probs, cudaStream_t s,
             const gbmc_options& o, double* ms) {
    int rc = gbmc_set_options(c, &o);
    if (rc) return rc;
    double best = 1e300;
    for (int rep = 0; rep < 3; ++rep) {   // the fastest of three (the first builds the graph)
        rc = gbmc_run_problems(c, (int32_t)probs.size(), probs.data(), s);
        if (rc) return rc;
        double t = 0;
        rc = gbmc_last_run_ms(c, &t);
        if (rc) return rc;
        rc = read_ctl(c);
        if (rc) return rc;
        if (rep > 0 || t < best) best = std::min(best, t);
    }
    *ms = best;
    return GBMC_OK;
}

}  // namespace

extern "C" int gbmc_autotune(gbmc_ctx* c, int32_t n_prob, const gbmc_problem* probs,
                             double fraction, void* stream, gbmc_options* best_out,
                             gbmc_autotune_report* report) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (n_prob < 1 || !probs) return fail(c, GBMC_ERR_INVALID_ARG, "n_prob >= 1 and probs required");
    if (!(fraction > 0 && fraction <= 1))
        return fail(c, GBMC_ERR_INVALID_ARG, "fraction must be in (0, 1]");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<gbmc_problem> pr(probs, probs + n_prob);
    int64_t total = 0;
    for (auto& p : pr) {
        p.n_particles = std::max<int64_t>(1, (int64_t)std::llround(p.n_particles * fraction));
        total += p.n_particles;
    }
    int64_t full_total = 0;
    for (int32_t k = 0; k < n_prob; ++k) full_total += probs[k].n_particles;
    gbmc_options base = c->opt;
    base.max_in_flight = 0;   // the probe's cap is set from the fraction below
    int trials = 0;
    double t0 = 0;
    int rc = probe_ms(c, pr, s, base, &t0);
    if (rc) return rc;
    ++trials;
    gbmc_options best = base;
    double best_ms = t0, best_frac = 1.0;
    const double keep = 0.98;   // a candidate must win by 2% to replace the incumbent
    // in-flight cap as a fraction of the run
    for (double f : {0.5, 0.25, 0.125}) {
        gbmc_options o = best;
        o.max_in_flight = std::max<int64_t>(1, (int64_t)(total * f));
        double t;
        if ((rc = probe_ms(c, pr, s, o, &t))) return rc;
        ++trials;
        if (t < best_ms * keep) {
            best_ms = t;
            best = o;
            best_frac = f;
        }
    }
    for (int32_t b : {2, 4, 16}) {
        gbmc_options o = best;
        o.blocks_per_sm = b;
        double t;
        if ((rc = probe_ms(c, pr, s, o, &t))) return rc;
        ++trials;
        if (t < best_ms * keep) { best_ms = t; best = o; }
    }
    for (int32_t w : {-1, 1024, 16384, 32768}) {
        gbmc_options o = best;
        o.warp_lookup_max = w;
        double t;
        if ((rc = probe_ms(c, pr, s, o, &t))) return rc;
        ++trials;
        if (t < best_ms * keep) { best_ms = t; best = o; }
    }
    if (best.precision == GBMC_FP64) {
        for (int32_t g : {-1, 100000, 262144}) {
            gbmc_options o = best;
            o.group_lookup_max = g;
            double t;
            if ((rc = probe_ms(c, pr, s, o, &t))) return rc;
            ++trials;
            if (t < best_ms * keep) { best_ms = t; best = o; }
        }
    }
    for (int32_t t : {-1, 1024, 16384, 65536}) {
        gbmc_options o = best;
        o.tail_max = t;
        double t_ms;
        if ((rc = probe_ms(c, pr, s, o, &t_ms))) return rc;
        ++trials;
        if (t_ms < best_ms * keep) { best_ms = t_ms; best = o; }
    }
    // binary32 lookups on the short windows
    if (best.precision == GBMC_FP32) {
        gbmc_options o = best;
        o.sparse_windows = 1 - best.sparse_windows;
        double t;
        if ((rc = probe_ms(c, pr, s, o, &t))) return rc;
        ++trials;
        if (t < best_ms * keep) { best_ms = t; best = o; }
    }
    // the sort threshold (sorting itself stays on: its gain grows with the
    // queue, and the probes' queues are the fraction's size)
    for (int32_t m : {1024, 65536, 1 << 20}) {
        gbmc_options o = best;
        o.sort_min = m;
        double t;
        if ((rc = probe_ms(c, pr, s, o, &t))) return rc;
        ++trials;
        if (t < best_ms * keep) { best_ms = t; best = o; }
    }
    // apply to the full problems: the chosen cap fraction of their particles
    best.max_in_flight = best_frac < 1.0
                             ? std::max<int64_t>(1, (int64_t)(full_total * best_frac))
                             : 0;
    if ((rc = gbmc_set_options(c, &best))) return rc;
    if ((rc = gbmc_reset_tallies(c, stream))) return rc;
    CK(cudaStreamSynchronize(s));
    if (best_out) *best_out = c->opt;
    if (report) {
        report->trials = trials;
        report->reserved = 0;
        report->default_ms = t0;
        report->best_ms = best_ms;
        report->in_flight_fraction = best_frac;
    }
    return GBMC_OK;
}

// ---------------------------------------------------------------------------
// Sorted lookup without any allocation.
//
// Some callers cannot allocate device memory while they call this library:
// code that runs while a CUDA stream is being captured into a graph (where
// cudaMalloc is not allowed), processes whose memory is handed out by a
// fixed, pre-reserved pool they do not control, or hard-real-time loops that
// must not take the allocator's locks or risk an out-of-memory error in the
// middle of work.  gbmc_lookup_macro(sort = 1) grows context-owned scratch
// with cudaMalloc on first use; this variant instead uses one fixed scratch
// area that lives in the library image itself.
//
// The scratch is a file-scope __device__ array, so every GPU that loads the
// library reserves it (about 8.5 MB) until the process exits.  Its device
// address is fetched on every call with cudaGetSymbolAddress (a lookup in the
// loaded module, no allocation), so it follows the current context, also after
// cudaDeviceReset; the host symbol itself is only a stand-in and is never
// handed to a kernel.
namespace {

constexpr int64_t kNoAllocMaxQueries = (int64_t)1 << 20;
constexpr size_t kNoAllocPermBytes = sizeof(int32_t) * kNoAllocMaxQueries;
constexpr size_t kNoAllocKeysBytes = sizeof(uint32_t) * kNoAllocMaxQueries;
constexpr size_t kNoAllocHistBytes = sizeof(uint32_t) * kSortBuckets;
constexpr size_t kNoAllocBytes =
    kNoAllocPermBytes + kNoAllocKeysBytes + 2 * kNoAllocHistBytes + sizeof(uint32_t) * 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch in the current context.
cudaError_t noalloc_scratch(unsigned char** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    *out = (unsigned char*)p;
    return e;
}

}  // namespace

extern "C" int gbmc_lookup_macro_noalloc(gbmc_ctx* c, int32_t precision, const double* d_E,
                                         const int32_t* d_mat, int64_t n, double* d_sigma_t,
                                         double* d_sigma_a, void* stream) {
    if (!c) return GBMC_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!d_E || !d_mat || !d_sigma_t || !d_sigma_a)))
        return fail(c, GBMC_ERR_INVALID_ARG, "n >= 0 and device arrays required");
    if (n > kNoAllocMaxQueries)
        return fail(c, GBMC_ERR_INVALID_ARG,
                    "gbmc_lookup_macro_noalloc takes at most %lld queries per call (got %lld)",
                    (long long)kNoAllocMaxQueries, (long long)n);
    if (precision != GBMC_FP64 && precision != GBMC_FP32)
        return fail(c, GBMC_ERR_INVALID_ARG, "precision must be GBMC_FP64 or GBMC_FP32");
    if (!c->n_nuc || !c->n_mat) return fail(c, GBMC_ERR_NOT_INITIALIZED, "tables and materials required");
    if ((precision == GBMC_FP64 && !c->has64) || (precision == GBMC_FP32 && !c->has32))
        return fail(c, GBMC_ERR_NOT_INITIALIZED, "tables not loaded in that precision");
    if (n == 0) return GBMC_OK;
    int rc = set_device(c);
    if (rc) return rc;
    unsigned char* base = nullptr;
    CK(noalloc_scratch(&base));
    int32_t* perm = (int32_t*)base;
    uint32_t* keys = (uint32_t*)(base + kNoAllocPermBytes);
    uint32_t* hist = (uint32_t*)(base + kNoAllocPermBytes + kNoAllocKeysBytes);
    uint32_t* cursor = hist + kSortBuckets;
    uint32_t* btot = cursor + kSortBuckets;
    cudaStream_t s = (cudaStream_t)stream;
    // the bucket counts must start at zero; an earlier call leaves them
    // cleared, but one that failed midway might not
    CK(cudaMemsetAsync(hist, 0, kNoAllocHistBytes, s));
    Params P = make_params(c);
    P.precision = precision;
    LaunchCfg L = make_launch(c);
    cudaError_t e = launch_query_lookup(P, L, d_E, d_mat, n, d_sigma_t, d_sigma_a, perm, keys,
                                        hist, cursor, btot, s);
    if (e != cudaSuccess) return fail(c, GBMC_ERR_CUDA, "lookup launch: %s", cudaGetErrorString(e));
    return GBMC_OK;
}
