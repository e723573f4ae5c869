// Host-side launchers of the device kernels (defined in transport.cu).
#pragma once

#include "device.cuh"

namespace gbmc {

struct LaunchCfg {
    int grid;          // blocks of the event kernels (multiple of the SM count)
    int grid_lookup;   // blocks of the lookup kernel
    int grid_tail;     // blocks of the tail kernel (one warp per particle)
};

// Fill the free-slot list of a run (the run's control block is written by
// the host before the launch).
cudaError_t launch_init_run(const Params& P, const LaunchCfg& L, cudaStream_t s);

// One event-loop iteration: plan, source, sort, lookup, ray trace (advance +
// surface), collision.  Captured once into the body of a graph while-node.
cudaError_t launch_iteration(const Params& P, const LaunchCfg& L, cudaStream_t s);

// The tail kernel, after the loop: finishes the histories left when the loop
// stopped early (a no-op otherwise).
cudaError_t launch_tail(const Params& P, const LaunchCfg& L, cudaStream_t s);

// Self-check of the integer-pipe division (div_rn) against the binary64
// division on n drawn operand pairs: *bad counts differing quotients, first
// holds the first such pair.
cudaError_t launch_check_division(int64_t n, uint64_t seed, unsigned long long* bad,
                                  double* first, int sms, cudaStream_t s);
cudaError_t launch_check_interp(int64_t n, uint64_t seed, const double* e0s, const double* e1s,
                                const Interval64* iv, int32_t K, unsigned long long* bad,
                                double* first, int sms, cudaStream_t s);

// Binary64 rate probe: blocks x 256 threads, each kRateChains (8)
// independent fused multiply-add chains of iters steps.
cudaError_t launch_fp64_rate(int blocks, int32_t iters, double* out, cudaStream_t s);

// k-eigenvalue: compacts the run's per-history fission-site slots into
// P.bank_out (history order), the size into *P.bank_size.
cudaError_t launch_bank(const Params& P, const LaunchCfg& L, cudaStream_t s);

// The iteration launched eagerly with an event before and after each kernel
// (ev[0..7]; the lookup's two mode kernels share one interval), for
// per-kernel device timing; the tail is timed separately.
constexpr int kIterKernels = 7;
constexpr int kIterLaunches = 7;   // kernels launched per iteration
constexpr int kTimedKernels = 8;   // + the tail
cudaError_t launch_iteration_timed(const Params& P, const LaunchCfg& L, cudaStream_t s,
                                   cudaEvent_t* ev);

// Standalone macroscopic lookup of caller-provided queries; with perm != NULL
// the queries are first bucket-sorted by (material, energy) into perm.
cudaError_t launch_query_lookup(const Params& P, const LaunchCfg& L, const double* E,
                                const int32_t* mat, int64_t n, double* st, double* sa,
                                int32_t* perm, uint32_t* keys, uint32_t* hist, uint32_t* cursor,
                                uint32_t* btot, cudaStream_t s);

// Importance estimates from recorded collision samples of the last run.
cudaError_t launch_imp_score(const Params& P, const int8_t* status, double* cnt, double* scr,
                             int sms, cudaStream_t s);
cudaError_t launch_imp_targets(const double* cnt, const double* scr, int32_t n_cells,
                               int32_t n_bins, double* cell_sums, float* y, float* w, int sms,
                               cudaStream_t s);

}  // namespace gbmc
