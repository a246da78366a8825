// k_sort.cu -- bucket order of the merged population by its first objective,
// used by the dominance build and the front peel (Alg. 1, the non-dominated sort).
//
// Dominance needs f_i0 <= f_j0, so when every point of a row block has a
// smaller f_0 than every point of a column block only "row dominates column"
// can hold, and that half of the test is done with m - 1 subtractions.  A
// counting sort into SORT_NB buckets of f_0 over [min f_0, max f_0] (a
// monotone key) makes such disjoint block pairs the common case.  Ties and
// order inside a bucket do not matter: every pair is still tested exactly.
//   k_sort_range    min / max of f_0 (order-preserving atomics)
//   k_sort_hist     bucket histogram; the last CTA turns it into offsets
//   k_sort_scatter  perm[pos] = i, skey[pos] = bucket, Fp = F in bucket order
//                   with -0.0 written as +0.0
#include "kernels.cuh"

namespace {

constexpr int SB = 1024;

__device__ __forceinline__ int bucket_of(float f, float lo, float scale)
{
    float t = (f - lo) * scale;
    int b = (int)t;
    if (!(t >= 0.0f)) b = 0;
    return b > SORT_NB - 1 ? SORT_NB - 1 : b;
}

__device__ __forceinline__ void range_of(const Ctrl* c, float& lo, float& scale)
{
    lo = ord2f(c->f0lo);
    const float hi = ord2f(c->f0hi);
    const float span = hi - lo;
    scale = (span > 0.0f && span < 3.0e38f) ? (float)SORT_NB / span : 0.0f;
}

__global__ void __launch_bounds__(SB) k_sort_range(RunView v)
{
    __shared__ uint32_t smin, smax;
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    if (threadIdx.x == 0) {
        smin = 0xffffffffu;
        smax = 0u;
    }
    __syncthreads();
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int i = blockIdx.x * SB + threadIdx.x; i < v.n2; i += gridDim.x * SB) {
        const uint32_t o = f2ord(v.F[(size_t)i * v.m] + 0.0f);
        lo = min(lo, o);
        hi = max(hi, o);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, s));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, s));
    }
    if (lane_id() == 0) {
        atomicMin(&smin, lo);
        atomicMax(&smax, hi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMin(&c->f0lo, smin);
        atomicMax(&c->f0hi, smax);
    }
}

__global__ void __launch_bounds__(SB) k_sort_hist(RunView v)
{
    __shared__ int h[SORT_NB];
    __shared__ int scratch[40];
    __shared__ unsigned ticket;
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    for (int b = threadIdx.x; b < SORT_NB; b += SB) h[b] = 0;
    __syncthreads();
    float lo, scale;
    range_of(c, lo, scale);
    for (int i = blockIdx.x * SB + threadIdx.x; i < v.n2; i += gridDim.x * SB)
        atomicAdd(&h[bucket_of(v.F[(size_t)i * v.m] + 0.0f, lo, scale)], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < SORT_NB; b += SB)
        if (h[b]) atomicAdd(&v.bcnt[b], h[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(&c->sort_done, 1u);
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    // last CTA: exclusive scan of the counts (SORT_NB / SB per thread)
    __threadfence();
    constexpr int PER = SORT_NB / SB;
    int loc[PER];
    int s = 0;
    for (int t = 0; t < PER; ++t) {
        loc[t] = __ldcg(&v.bcnt[threadIdx.x * PER + t]);
        s += loc[t];
    }
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int x = scratch[lane];
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        scratch[lane] = xi - x;
    }
    __syncthreads();
    int run = scratch[warp] + inc - s;
    for (int t = 0; t < PER; ++t) {
        v.bcnt[threadIdx.x * PER + t] = run;
        run += loc[t];
    }
    if (threadIdx.x == 0) c->sort_done = 0u;
}

__global__ void __launch_bounds__(256) k_sort_scatter(RunView v)
{
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= v.n2) return;
    float lo, scale;
    range_of(c, lo, scale);
    const int m = v.m;
    const int b = bucket_of(v.F[(size_t)i * m] + 0.0f, lo, scale);
    const int pos = atomicAdd(&v.bcnt[b], 1);
    v.perm[pos] = i;
    v.skey[pos] = (uint32_t)b;
    for (int q = 0; q < m; ++q) v.Fp[(size_t)pos * m + q] = v.F[(size_t)i * m + q] + 0.0f;
}

// m > NSGA3_FAST_M: a warp per point (lane 0 takes the position, the lanes
// copy the row)
__global__ void __launch_bounds__(256) k_sort_scatter_rows(RunView v)
{
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int i = (blockIdx.x * 256 + threadIdx.x) >> 5;
    if (i >= v.n2) return;
    const int lane = lane_id(), m = v.m;
    int pos = 0;
    if (lane == 0) {
        float lo, scale;
        range_of(c, lo, scale);
        const int b = bucket_of(v.F[(size_t)i * m] + 0.0f, lo, scale);
        pos = atomicAdd(&v.bcnt[b], 1);
        v.perm[pos] = i;
        v.skey[pos] = (uint32_t)b;
    }
    pos = __shfl_sync(0xffffffffu, pos, 0);
    for (int q = lane; q < m; q += 32) v.Fp[(size_t)pos * m + q] = v.F[(size_t)i * m + q] + 0.0f;
}

}  // namespace

cudaError_t launch_sort(const RunView& v, int num_sms, cudaStream_t s)
{
    int blocks = (v.n2 + SB - 1) / SB;
    if (blocks > num_sms) blocks = num_sms;
    k_sort_range<<<blocks, SB, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sort_hist<<<blocks, SB, 0, s>>>(v);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (v.m > NSGA3_FAST_M)
        k_sort_scatter_rows<<<(unsigned)(((long long)v.n2 * 32 + 255) / 256), 256, 0, s>>>(v);
    else
        k_sort_scatter<<<(v.n2 + 255) / 256, 256, 0, s>>>(v);
    return cudaGetLastError();
}
