// common.cuh -- device-side types and helpers shared by the NSGA-III kernels.
//
// Layout of one run in HBM (n2 = 2N merged population, ld = n2 rounded up
// to a multiple of 256, NW = ld / 32 bit-mask words):
//   X     n2 x d  FP32 row-major   parents rows [0,N), children rows [N,2N)
//   F     ld x m  FP32 row-major   rows >= n2 are NaN padding (never dominate)
//   Fp    ld x m  FP32             F in bucket order of f_0 (perm: position -> index)
//   Dom   NW x ld u32              bit (i mod 32) of Dom[i/32][j] = "i dominates j",
//                                  i, j positions in bucket order
//   rank2 ld int32                 front index of the merged population, -1 = F_drop
//   pi/dist ld                     association (reference index, FP64 distance)
//   Zd    w x m   FP64             Das-Dennis directions; Zh w x M4 FP32 unit copy
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

#define NSGA3_MAX_M 512         // objectives accepted by a context
#define NSGA3_FAST_M 10         // largest m with kernels specialised for each m
#define NSGA3_WARP_M 32         // largest m whose intercept system one warp solves
#define NSGA3_TILE 256          // column tile of the dominance build; ld % 256 == 0
#define NSGA3_PEEL_COLS 128     // columns per peel chunk (4 per lane, 32 lanes)
#define SORT_NB 4096            // sort keys of the f_0 bucket order (m > 10)
#define SORT_KMAX 65536         // largest number of sort keys (m <= 10: 2^kbits keys)
#define SORT_QB 1024            // histogram bins per objective for the level thresholds
#define SORT_LMAX 7             // level thresholds per objective (3 bits of level)

// Capacity paths of the niching kernels (Ctrl::npath, reported by
// nsga3_get_selection_paths; same values as NSGA3_PATH_* in nsga3.h)
#define NPATH_UNSTAGED 1u   // more references than k_level stages in shared memory
#define NPATH_DEEP 2u       // L* beyond the shared level histogram (binary search)
#define NPATH_CKOVER 4u     // more level-L* references than the staged key list holds
#define NPATH_BINOVER 8u    // a 12-bit radix bin of k_level held more keys than the exact rank
#define NPATH_LARGE 16u     // a partial take from a reference of more than 32 members
#define NPATH_RADIX 32u     // the block-wide select ran an 8-bit radix pass
#define NPATH_RADIX2 64u    // ... and a second one

// device status codes (same values as the C ABI's nsga3_status)
#define DEV_OK 0
#define DEV_ENONFINITE 4
#define DEV_ETIMEOUT 5
#define DEV_EINTERNAL 7

// Random-number streams (third counter word of Philox).
enum : uint32_t {
    RNG_TOURNAMENT = 1,
    RNG_SBX = 2,
    RNG_PM = 3,
    RNG_REFPRIO = 4,
    RNG_MEMPRIO = 5,
    RNG_INIT = 6
};

// Control block of one run, resident in device memory.  Written by the
// selection kernels, read back by the host only for diagnostics.
struct Ctrl {
    uint32_t gen;            // Philox generation counter (word 1 of the counter)
    int32_t status;          // DEV_* of the last failure, 0 if none
    int32_t cum;             // members ranked so far
    int32_t l;               // selecting front (first with cum >= N)
    int32_t nS;              // |S| = members of fronts < l
    int32_t K;               // N - |S|
    int32_t nFl;             // |F_l|
    int32_t need_niche;      // K < |F_l|
    int32_t fallback;        // normalization used the nadir fallback
    int32_t passes;          // peel passes (kernel launches) in the last selection
    uint32_t sbar;           // arrivals at the barriers of the cooperative elimination
    unsigned long long pbar; // peel barrier: arrivals << 32 | points ranked so far
    unsigned long long prel; // peel barrier release: passes closed << 32 | points ranked
    uint32_t never;          // a word nothing sets (the wait self-test polls it)
    int32_t nT;              // |S u F_l| (association set)
    int32_t Lstar;           // niche level threshold L*
    int32_t rlev;            // refs taken at level L*
    int32_t nsel;            // selected count written by the compaction
    int32_t overflow;        // association candidate-list overflows (slow path taken)
    int32_t recheck_miss;    // debug: association misses found by the full FP64 recheck
    int32_t nlarge;          // references whose partial take needs the block-wide select
    uint32_t peel_rows;      // dominator word-rows in the peel's row lists, all passes
    uint32_t npath;          // NPATH_* bits: capacity paths the niching kernels took
    int32_t ntile;           // tiles listed in tlist by k_tile_plan
    unsigned long long domstat[8];  // block pairs of the dominance build by mode (zero, f_0
                                    // one-direction, row-dom-column, column-dom-row, both),
                                    // tiles with nothing to test, (lane, column) pairs
                                    // tested and live pairs among them (m <= 10)

    int32_t ncand;           // association candidates written by the scan
    int32_t nslow;           // points sent to the full FP64 association scan
    uint32_t ext_done;       // completion ticket of the extreme-point blocks
    uint32_t sort_done;      // completion ticket of the bucket histogram
    uint32_t f0lo, f0hi;     // range of f_0 as order-preserving uint
    uint32_t thr_done;       // completion ticket of the sort's threshold histogram blocks
    uint32_t omin[NSGA3_FAST_M], omax[NSGA3_FAST_M];  // objective ranges (order-preserving uint)
    float thr[NSGA3_FAST_M][SORT_LMAX];               // level thresholds of the sort keys (m <= 10)
    uint32_t cmp_done;       // completion ticket of the compaction blocks
    uint32_t zmin[NSGA3_MAX_M];  // ideal point as order-preserving uint of FP32
    double zstar[NSGA3_MAX_M];   // ideal point (FP64, +0.0 for zero)
    double a[NSGA3_MAX_M];       // intercepts
    int32_t ext[NSGA3_MAX_M];    // extreme-point indices
    unsigned long long passes_total;  // peel passes since the context was created
    // normalization history (opts.norm_history), kept across selections
    int32_t hvalid;                      // 1 once a normalization has been recorded
    double hz[NSGA3_MAX_M];              // running ideal point
};

// Device pointers and sizes of one run, passed by value to every kernel.
struct RunView {
    int m, d, N, n2, ld, NW, w, M4;   // M4 = m rounded up to a multiple of 4
    int full_sort;
    int debug_recheck_all;
    int streaming;         // no Dom matrix: the peel recomputes dominance from Fp
    int norm_history;      // normalization with a running ideal and remembered extremes
    int problem;           // 0 softmax-simplex, 1 0-1 knapsack
    unsigned long long wait_ns;  // budget of every device-side wait
    const int32_t* kp_p;   // m x d profits
    const int32_t* kp_w;   // m x d weights
    const int32_t* kp_cap; // m capacities
    const int32_t* kp_total;  // m total profits
    const int32_t* kp_order;  // d items in repair order
    uint64_t seed;
    float eta_c, eta_m, p_c, p_m;
    Ctrl* ctrl;
    float* X;          // n2 x d
    float* F;          // ld x m
    int32_t* rank;     // parents' ranks (N), used by the tournament
    float* Xtmp;       // N x d gather target
    float* Ftmp;       // N x m
    int32_t* ranktmp;  // N
    uint32_t* Dom;     // NW x ld
    int32_t* cnt;      // ld   remaining dominator counts
    int32_t* rank2;    // ld   merged ranks (original order)
    int32_t* srank;    // ld   merged ranks in bucket order (peel)
    int32_t* perm;     // ld   bucket order position -> original index
    uint32_t* skey;    // ld   sort key of each position (0xffffffff for padding)
    uint32_t* pkey;    // n2   sort key of each point (original order)
    float* Fp;         // ld x m objectives in bucket order, -0.0 as +0.0, NaN padding
    int32_t* bcnt;     // nkeys + 1 key counts, then offsets / cursors
    int kbits;         // bits of a sort key (nkeys = 2^kbits)
    int lbits;         // bits of level per objective in a sort key (m <= 10)
    int32_t* qhist;    // m x SORT_QB objective histograms (level thresholds)
    float* bbox;       // NW x 2 M4: per 32-position block min, then max of each objective
    uint32_t* bkey;    // NW x 2: per block smallest, largest sort key
    uint8_t* dnz;      // NW x NB8 bits: Dom block (I, J) has a nonzero word (m <= 10, matrix);
                       // null: every Dom word is written
    int NB8;           // bytes of dnz per dominator block row = ceil(NW / 8)
    float* tbox;       // (ld / 256) x 2 M4: per 256-position tile min, then max of each objective
    uint32_t* tkey;    // (ld / 256) x 2: per tile smallest, largest sort key
    int32_t* tlist;    // tiles of the dominance build with block pairs to test (k_tile_plan)
    int num_sms;
    int shared_gpu;    // 1: the run shares the GPU with others (batched graphs, the run
                       // server): the cooperative peel takes fewer CTAs, so that it can
                       // start while other runs' kernels hold part of every SM
    uint32_t* rem;     // NW   not-yet-ranked mask
    uint32_t* front;   // 2 x NW  ping-pong front masks
    uint32_t* chunk_lim;   // ld / NSGA3_PEEL_COLS dominator row blocks a column chunk reads
    uint32_t* selmask;     // NW picked members of F_l
    int32_t* Tlist;        // n2 members of S u F_l
    double* fprime;        // n2 x m  normalised objectives (indexed by T slot)
    double* fnorm;         // n2      |f'|
    float* uhat;           // n2 x M4 FP32 unit vectors
    int32_t* pi;           // ld
    double* dist;          // ld
    double* ext_part;      // parts x m  per-block ASF minima
    int32_t* ext_idx;      // parts x m
    double* nad_part;      // parts x m  per-block maxima of f - z*
    int ext_parts;
    int32_t* rho;          // w
    int32_t* rhop;         // w
    int32_t* take;         // w
    int32_t* ref_off;      // w + 1
    int32_t* cursor;       // w
    int32_t* bucket;       // n2
    int4* large;           // w   (ref, members still to take, excluded member, -)
    int32_t* sel;          // N   selected indices, ascending
    const double* Zd;      // w x m
    const double* nz;      // w
    const float* Zh;       // w x M4
    const float* Wobj;     // m x (m-1)
    const float* Wt;       // (m-1) x m  W transposed (m > NSGA3_FAST_M)
    // association scan: references reordered into compact blocks of 32
    int nblk;              // ceil(w / 32)
    const float* blk_c;    // nblk x M4  unit cone centres (FP32)
    const float2* blk_r;   // nblk       (cos r, sin r) of the inflated cone radius
    const float* blk_z;    // w x M4     zhat in block order
    const int32_t* blk_j;  // w          original reference index in block order
    int2* arun;            // n2         candidate run (start, count) per T slot; start -1 = slow
    int2* cand;            // cand_cap   (T slot, reference)
    int cand_cap;
    int32_t* slow;         // n2         T slots for the full FP64 scan
    // tiled association (null: the pruned scan): per work item (a tile of T
    // slots x a range of reference blocks) and slot, ASSOC_K entries
    // (block maximum of the FP32 cosines as float bits, block; -1 empty, -2 overflow)
    int2* aent;
    int assoc_grid;        // CTAs of the tiled scan (the entries' layout depends on it)
    double* cdist;         // cand_cap   FP64 distance of each candidate (m > NSGA3_FAST_M)
    float* he;             // m x m      remembered extreme vectors (history), row q for axis q
    // m > NSGA3_FAST_M: extreme points by entry keys, then per-axis blocks
    unsigned long long* ekey;  // (n2 + m) x 2  ASF keys of the largest / second-largest f~
    int32_t* er1;              // n2 + m        objective of the largest f~
    double* nadv;              // m     max f~ per axis (nadir fallback)
    // m > NSGA3_WARP_M: intercepts by the cooperative elimination
    double* amat;          // m x (m + 1)  [E - z* | 1], rows in original order
    float* etmp;           // m x m        new extreme vectors (copied to he at the end)
    // m > NSGA3_FAST_M with few tiles: the objective chunks of a tile are
    // split over dom_ks CTAs, which OR their sign masks into dpa / dpb
    // (NW x ld, laid out like Dom; zero between selections)
    int dom_ks;
    int dom_ctas;          // dominance build: persistent CTAs per SM (0: all resident)
    int peel_ctas;         // front peel: cooperative CTAs per SM (0: all resident)
    uint32_t* dpa;         // "some f_i > f_j" bits of row i against column block jb
    uint32_t* dpb;         // "some f_j > f_i"
};

// ------------------------------------------------------------ Philox ------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products by the published multipliers; the key advances by
// the published Weyl increments between rounds.
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint64_t seed)
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c0;
        uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo1 = 0xCD9E8D57u * c2;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// uniform FP32 in [0,1): top 24 bits of the word times 2^-24 (exact)
__device__ __forceinline__ float u01(uint32_t w) { return (float)(w >> 8) * 5.9604644775390625e-08f; }
// integer in [0,n): (w * n) >> 32
__device__ __forceinline__ uint32_t bounded(uint32_t w, uint32_t n)
{
    return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32);
}

// ------------------------------------------------- ordered float bits -----
__device__ __forceinline__ uint32_t f2ord(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// -------------------------------------------------------- warp helpers ----
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void set_status(Ctrl* c, int s)
{
    atomicCAS(&c->status, 0, s);
}

__device__ __forceinline__ int read_status(const Ctrl* c)
{
    return *(volatile const int32_t*)&c->status;
}

// niching kernels run unconditionally in the graph and return at once when
// the selection failed or |S| + |F_l| == N (no niching needed)
__device__ __forceinline__ bool skip_niche(const Ctrl* c)
{
    return read_status(c) != 0 || *(volatile const int32_t*)&c->need_niche == 0;
}

// lexicographic (value, index) minimum for doubles
__device__ __forceinline__ bool lex_less(double a, int ia, double b, int ib)
{
    return a < b || (a == b && ia < ib);
}

// ------------------------------------------------------ grid barriers -----
// Barriers of a cooperative launch (every CTA resident), with a bounded
// wait: they give up and record DEV_ETIMEOUT when the other CTAs did not
// arrive within the run's wait budget (RunView::wait_ns) of device time.

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned x;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(x) : "l"(p) : "memory");
    return x;
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p)
{
    unsigned long long x;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];\n" : "=l"(x) : "l"(p) : "memory");
    return x;
}

__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long x)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;\n" ::"l"(p), "l"(x) : "memory");
}

// Polls `done` until it returns true or wait_ns of device time have passed
// (the clock is read every 1,024 polls; the poll count caps the wait too,
// should the timer not advance); on expiry records DEV_ETIMEOUT and returns
// false.  Every device-side wait goes through it.
template <class Done>
__device__ __forceinline__ bool bounded_wait(Ctrl* c, unsigned long long wait_ns, Done done)
{
    const unsigned long long t0 = global_ns();
    unsigned it = 0;
    while (!done()) {
        if ((++it & 1023u) == 0u && (global_ns() - t0 > wait_ns || it > (1u << 30))) {
            set_status(c, DEV_ETIMEOUT);
            return false;
        }
    }
    return true;
}

// Summing barrier of the peel: pass k's barrier adds (1 << 32) + add (this
// CTA's new front members) to *bar; the CTA whose addition completes the
// (k+1) * gridDim.x arrivals holds the running total of every CTA's adds
// (no CTA can add for pass k+1 before that) and releases it with the pass
// number in *rel, which the others poll.  Returns the total (< 2^32) or,
// on a timeout, ~0ull.  *bar and *rel are zero at launch.
__device__ __forceinline__ unsigned long long grid_sync_sum(Ctrl* c, unsigned long long* bar, unsigned long long* rel,
                                                           unsigned k, unsigned add, unsigned long long wait_ns,
                                                           unsigned long long* s_val)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long val;
        __threadfence();
        const unsigned long long inc = (1ull << 32) | add;
        const unsigned long long now = atomicAdd(bar, inc) + inc;
        if ((now >> 32) == (unsigned long long)(k + 1) * gridDim.x) {
            val = now & 0xffffffffull;
            __threadfence();  // the arrivals' writes before the release
            st_release64(rel, ((unsigned long long)(k + 1) << 32) | val);
        } else {
            unsigned long long r = 0;
            const bool ok = bounded_wait(c, wait_ns, [&] { return ((r = ld_acquire64(rel)) >> 32) >= k + 1ull; });
            val = ok ? (r & 0xffffffffull) : ~0ull;
        }
        __threadfence();
        *s_val = val;
    }
    __syncthreads();
    return *s_val;
}

// Counting barrier: the k-th barrier of a launch waits until *ctr reaches
// k * gridDim.x (*ctr is zero at launch): one atomic on the arrival path and
// a tight poll, for kernels that meet at a barrier many times per launch.
__device__ __forceinline__ bool grid_sync_count(Ctrl* c, unsigned* ctr, unsigned target, unsigned long long wait_ns,
                                                int* s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        if (atomicAdd(ctr, 1u) + 1u < target)
            ok = bounded_wait(c, wait_ns, [&] { return ld_acquire(ctr) >= target; }) ? 1 : 0;
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}
