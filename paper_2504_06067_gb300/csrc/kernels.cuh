// kernels.cuh -- launch wrappers for the NSGA-III kernels (host side).
// Every wrapper enqueues on `s` and returns the launch error; grids are
// derived from the run's fixed sizes, so the same launches can be captured
// into a CUDA graph once and replayed every generation.
#pragma once
#include "common.cuh"

// setup (Sec. II-C reference points; init population)
cudaError_t launch_refdirs(const RunView& v, int p1, int p2, double tau, double* Zd, double* nz,
                           float* Zh, cudaStream_t s);
cudaError_t launch_init(const RunView& v, cudaStream_t s);
cudaError_t launch_nan_pad(const RunView& v, cudaStream_t s);

// variation + objective (Alg. 1, crossover and mutation; Sec. III-A)
cudaError_t launch_vary_eval(const RunView& v, cudaStream_t s);

// selection (Alg. 1 sort / Alg. 2)
// 0-1 knapsack workload (k_knapsack.cu): bits + repair + objectives
cudaError_t launch_kp_init(const RunView& v, cudaStream_t s);
cudaError_t launch_kp_vary_eval(const RunView& v, cudaStream_t s);
cudaError_t launch_sel_reset(const RunView& v, cudaStream_t s);
// the device-wait self-test (nsga3_wait_probe)
cudaError_t launch_wait_probe(const RunView& v, cudaStream_t s);
cudaError_t launch_check_finite(const RunView& v, cudaStream_t s);
cudaError_t launch_sort(const RunView& v, int num_sms, cudaStream_t s);
cudaError_t launch_dominance(const RunView& v, cudaStream_t s);
cudaError_t dom_init_attributes();
// every peel pass in one cooperative launch (grid barrier between passes)
cudaError_t launch_peel(const RunView& v, int num_sms, cudaStream_t s);
cudaError_t peel_init_attributes();
cudaError_t launch_norm_ideal(const RunView& v, cudaStream_t s);
// extreme points and intercepts: one launch (m <= 10); above, the ideal
// point, entry keys, per-axis blocks and their reduction (four launches),
// plus the cooperative elimination for m > 32
cudaError_t launch_norm_extreme(const RunView& v, int num_sms, cudaStream_t s);
cudaError_t norm_init_attributes();
cudaError_t launch_assoc_prep(const RunView& v, cudaStream_t s);
// at most this many reference directions (and m <= 10): the association is
// one kernel with every direction in shared memory (k_assoc_small)
#define ASSOC_SMALL_W 512
inline bool assoc_small(const RunView& v) { return v.m <= NSGA3_FAST_M && v.w <= ASSOC_SMALL_W; }
// FP32 candidate scan, FP64 distances and per-point argmin, FP64 slow path
// (three launches; four for m > 10, where the distances are a kernel of
// their own); f' and |f'| are launch_assoc_prep (one launch, two for m > 10)
cudaError_t launch_assoc_scan(const RunView& v, int num_sms, cudaStream_t s);
cudaError_t assoc_prepare(const RunView& v);
// tiled association scan (m <= 10, more than ASSOC_SMALL_W directions):
// its grid for a device of num_sms SMs and the int2 entries it writes for
// at most n2 points
int assoc_tile_grid(int num_sms);
size_t assoc_tile_entries(int n2, int num_sms);
cudaError_t assoc_init_attributes();
cudaError_t launch_level(const RunView& v, cudaStream_t s);
cudaError_t launch_bucket(const RunView& v, cudaStream_t s);
cudaError_t launch_pick(const RunView& v, cudaStream_t s);
// self-test of the block-wide selection of the smallest keys (one CTA)
cudaError_t launch_select_probe(const unsigned long long* keys, int n, int need, uint32_t* marks,
                                unsigned* paths, cudaStream_t s);
cudaError_t launch_compact(const RunView& v, cudaStream_t s);
cudaError_t launch_gather(const RunView& v, cudaStream_t s);

// issue-rate probe of the dominance test's FADD / LOP3 mix (k_probe.cu)
double issue_probe_instructions(int blocks, int iters);
cudaError_t launch_issue_probe(const float* in, int blocks, int iters, uint32_t* sink, cudaStream_t s);

// one-time attribute setup (dynamic shared memory opt-in)
cudaError_t kernels_init_attributes();
