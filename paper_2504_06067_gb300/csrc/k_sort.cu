// k_sort.cu -- sort keys of the merged population, used by the dominance
// build and the front peel (Alg. 1, the non-dominated sort).
//
// For m <= 10 every objective q is cut into L = 2^lbits levels by L - 1
// thresholds near its quantiles (from a histogram of the selection's own
// values), and a point's key interleaves the bits of its m levels from the
// top bit down (Morton order), truncated to kbits.  A point i can dominate
// j only if f_iq <= f_jq for every q, so only if every level of i is at most
// the level of j, and then every prefix of the interleaved bits of i is at
// most that of j: dominators never have a larger key, equal vectors have
// equal keys, and points with nearby keys are close in every objective, so
// 32-point blocks of the key order have small bounding boxes that let the
// dominance build rule out most block pairs.  Any thresholds would be
// correct; quantiles balance the levels.  For m > 10 the key is one of 4,096
// buckets of f_0.  A counting sort into the 2^kbits keys orders the points;
// ties and order inside a key do not matter: every pair that can dominate is
// still tested exactly.
// The thresholds (and, for m > 10, the f_0 range of the buckets) come from a
// fixed sample of at most 8,192 points, every (n2 / 8,192)-th: they only
// steer how well the blocks prune, and a value outside the sample's range
// still gets a monotone key (levels count thresholds, buckets are clamped).
//   k_sort_range    per-objective min / max of the sample (order-preserving atomics)
//   k_sort_thr      per-objective histograms of the sample over [min, max] in
//                   the order-preserving integer space (about equal steps of
//                   relative size); the last CTA turns them into thresholds
//   k_sort_hist     every point's key (kept in pkey) and the key histogram;
//                   the last CTA turns it into offsets
//   k_sort_scatter  perm[pos] = i, skey[pos] = key, Fp = F in key order
//                   with -0.0 written as +0.0
#include "kernels.cuh"

namespace {

constexpr int SB = 1024;
constexpr int SAMPLE = 8192;  // points that set the thresholds and the f_0 range

// stride of the threshold sample
__device__ __forceinline__ int sample_stride(int n2) { return n2 > SAMPLE ? (n2 + SAMPLE - 1) / SAMPLE : 1; }

__device__ __forceinline__ int bucket_of(float f, float lo, float scale, int nb)
{
    float t = (f - lo) * scale;
    int b = (int)t;
    if (!(t >= 0.0f)) b = 0;
    return b > nb - 1 ? nb - 1 : b;
}

__device__ __forceinline__ void range_of(const Ctrl* c, int nb, float& lo, float& scale)
{
    lo = ord2f(c->f0lo);
    const float hi = ord2f(c->f0hi);
    const float span = hi - lo;
    scale = (span > 0.0f && span < 3.0e38f) ? (float)nb / span : 0.0f;
}

// sort key of point i (see the file comment); thr: the level thresholds
// (m <= 10), staged by the caller
__device__ __forceinline__ uint32_t key_of(const RunView& v, const Ctrl* c, const float (*thr)[SORT_LMAX], int i)
{
    const int m = v.m;
    const float* f = v.F + (size_t)i * m;
    if (m > NSGA3_FAST_M) {
        float lo, scale;
        range_of(c, SORT_NB, lo, scale);
        return (uint32_t)bucket_of(f[0] + 0.0f, lo, scale, SORT_NB);
    }
    const int lb = v.lbits, nthr = (1 << lb) - 1;
    uint32_t lev[NSGA3_FAST_M];
#pragma unroll
    for (int q = 0; q < NSGA3_FAST_M; ++q) {
        uint32_t l = 0u;
        if (q < m) {
            const float x = f[q];
            for (int k = 0; k < nthr; ++k) l += x > thr[q][k] ? 1u : 0u;
        }
        lev[q] = l;
    }
    uint32_t key = 0u;
    for (int b = lb - 1; b >= 0; --b)
#pragma unroll
        for (int q = 0; q < NSGA3_FAST_M; ++q)
            if (q < m) key = (key << 1) | ((lev[q] >> b) & 1u);
    return key >> (lb * m - v.kbits);
}

// m <= 10: min / max of every objective; above, of f_0
__global__ void __launch_bounds__(SB) k_sort_range(RunView v)
{
    __shared__ uint32_t smin[NSGA3_FAST_M], smax[NSGA3_FAST_M];
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int m = v.m, mr = m <= NSGA3_FAST_M ? m : 1;
    if (threadIdx.x < NSGA3_FAST_M) {
        smin[threadIdx.x] = 0xffffffffu;
        smax[threadIdx.x] = 0u;
    }
    __syncthreads();
    uint32_t lo[NSGA3_FAST_M], hi[NSGA3_FAST_M];
#pragma unroll
    for (int q = 0; q < NSGA3_FAST_M; ++q) {
        lo[q] = 0xffffffffu;
        hi[q] = 0u;
    }
    const int st = sample_stride(v.n2);
    for (int i = (blockIdx.x * SB + threadIdx.x) * st; i < v.n2; i += gridDim.x * SB * st) {
        const float* f = v.F + (size_t)i * m;
#pragma unroll
        for (int q = 0; q < NSGA3_FAST_M; ++q)
            if (q < mr) {
                const uint32_t o = f2ord(f[q] + 0.0f);
                lo[q] = min(lo[q], o);
                hi[q] = max(hi[q], o);
            }
    }
#pragma unroll
    for (int q = 0; q < NSGA3_FAST_M; ++q)
        if (q < mr) {
            const uint32_t a = __reduce_min_sync(0xffffffffu, lo[q]), b = __reduce_max_sync(0xffffffffu, hi[q]);
            if (lane_id() == 0) {
                atomicMin(&smin[q], a);
                atomicMax(&smax[q], b);
            }
        }
    __syncthreads();
    if (threadIdx.x < mr) {
        atomicMin(&c->omin[threadIdx.x], smin[threadIdx.x]);
        atomicMax(&c->omax[threadIdx.x], smax[threadIdx.x]);
        if (threadIdx.x == 0) {
            atomicMin(&c->f0lo, smin[0]);
            atomicMax(&c->f0hi, smax[0]);
        }
    }
}

// bin of an order-preserving value o in [omin, omin + span) (span >= 1)
__device__ __forceinline__ int qbin(uint32_t o, uint32_t omin, unsigned long long span)
{
    return (int)(((unsigned long long)(o - omin) * SORT_QB) / span);
}

// m <= 10: level thresholds.  Bin e of objective q holds the values whose
// order-preserving codes o satisfy floor((o - omin) QB / span) = e; the
// threshold of level k + 1 is the largest value of the first bin whose
// cumulative count reaches (k + 1) n2 / L.
__global__ void __launch_bounds__(SB) k_sort_thr(RunView v)
{
    __shared__ int h[NSGA3_FAST_M * SORT_QB];
    __shared__ unsigned ticket;
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int m = v.m;
    for (int b = threadIdx.x; b < m * SORT_QB; b += SB) h[b] = 0;
    __syncthreads();
    uint32_t omin[NSGA3_FAST_M];
    unsigned long long span[NSGA3_FAST_M];
#pragma unroll
    for (int q = 0; q < NSGA3_FAST_M; ++q) {
        omin[q] = q < m ? c->omin[q] : 0u;
        span[q] = q < m ? (unsigned long long)(c->omax[q] - omin[q]) + 1ull : 1ull;
    }
    const int st = sample_stride(v.n2);
    for (int i = (blockIdx.x * SB + threadIdx.x) * st; i < v.n2; i += gridDim.x * SB * st) {
        const float* f = v.F + (size_t)i * m;
#pragma unroll
        for (int q = 0; q < NSGA3_FAST_M; ++q)
            if (q < m) atomicAdd(&h[q * SORT_QB + qbin(f2ord(f[q] + 0.0f), omin[q], span[q])], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < m * SORT_QB; b += SB)
        if (h[b]) atomicAdd(&v.qhist[b], h[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(&c->thr_done, 1u);
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    __threadfence();
    // last CTA: warp q scans objective q's bins (32 per lane)
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    if (warp >= m) return;
    const int q = warp, L = 1 << v.lbits;
    constexpr int PER = SORT_QB / 32;
    int loc[PER];
    int s = 0;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        loc[t] = __ldcg(&v.qhist[q * SORT_QB + lane * PER + t]);
        s += loc[t];
    }
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const int before = inc - s;
    const int ns = (v.n2 + sample_stride(v.n2) - 1) / sample_stride(v.n2);  // points sampled
    for (int k = 0; k + 1 < L; ++k) {
        const long long target = ((long long)(k + 1) * ns + L - 1) / L;  // ceil((k + 1) ns / L)
        int e = -1;
        if (before < target && target <= inc) {
            int run = before;
            for (int t = 0; t < PER; ++t) {
                run += loc[t];
                if (run >= target) {
                    e = lane * PER + t;
                    break;
                }
            }
        }
        const unsigned who = __ballot_sync(0xffffffffu, e >= 0);
        const int eb = __shfl_sync(0xffffffffu, e, who ? __ffs(who) - 1 : 0);
        if (lane == 0) {
            // largest code of bin eb: omin + ceil((eb + 1) span / QB) - 1
            const unsigned long long hiw = ((unsigned long long)(eb + 1) * span[q] + SORT_QB - 1) / SORT_QB;
            c->thr[q][k] = who ? ord2f(omin[q] + (uint32_t)(hiw - 1ull)) : ord2f(omin[q] + (uint32_t)(span[q] - 1ull));
        }
    }
}

__global__ void __launch_bounds__(SB) k_sort_hist(RunView v)
{
    __shared__ int scratch[40];
    __shared__ unsigned ticket;
    __shared__ float thr[NSGA3_FAST_M][SORT_LMAX];
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    if (threadIdx.x < NSGA3_FAST_M * SORT_LMAX)
        thr[threadIdx.x / SORT_LMAX][threadIdx.x % SORT_LMAX] = c->thr[threadIdx.x / SORT_LMAX][threadIdx.x % SORT_LMAX];
    __syncthreads();
    for (int i = blockIdx.x * SB + threadIdx.x; i < v.n2; i += gridDim.x * SB) {
        const uint32_t key = key_of(v, c, thr, i);
        v.pkey[i] = key;
        atomicAdd(&v.bcnt[key], 1);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(&c->sort_done, 1u);
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    // last CTA: exclusive scan of the counts, a contiguous run per thread
    __threadfence();
    const int nk = 1 << v.kbits;  // >= 256: a multiple of 4, at most 2^16
    const int per = ((nk + SB - 1) / SB + 3) & ~3;  // <= 64
    const int b0 = min(nk, (int)threadIdx.x * per), b1 = min(nk, b0 + per);
    // the thread's run read in batches of 8 vectors, each batch's loads
    // issued before their first use
    constexpr int RUN4 = ((1 << 16) / SB + 3) / 4, BAT = 8;
    int s = 0;
#pragma unroll
    for (int h = 0; h < RUN4; h += BAT) {
        int4 xs[BAT];
#pragma unroll
        for (int t = 0; t < BAT; ++t) {
            const int b = b0 + 4 * (h + t);
            xs[t] = b < b1 ? __ldcg(reinterpret_cast<const int4*>(v.bcnt + b)) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int t = 0; t < BAT; ++t) s += xs[t].x + xs[t].y + xs[t].z + xs[t].w;
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
#pragma unroll
    for (int h = 0; h < RUN4; h += BAT) {
        int4 xs[BAT];
#pragma unroll
        for (int t = 0; t < BAT; ++t) {
            const int b = b0 + 4 * (h + t);
            xs[t] = b < b1 ? __ldcg(reinterpret_cast<const int4*>(v.bcnt + b)) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int t = 0; t < BAT; ++t) {
            const int4 x = xs[t];
            int4 y;
            y.x = run;
            y.y = run + x.x;
            y.z = y.y + x.y;
            y.w = y.z + x.z;
            run = y.w + x.w;
            const int b = b0 + 4 * (h + t);
            if (b < b1) *reinterpret_cast<int4*>(v.bcnt + b) = y;
        }
    }
    if (threadIdx.x == 0) c->sort_done = 0u;
}

__global__ void __launch_bounds__(256) k_sort_scatter(RunView v)
{
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= v.n2) return;
    const int m = v.m;
    const uint32_t b = v.pkey[i];
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
        const uint32_t b = v.pkey[i];
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
    if (v.m <= NSGA3_FAST_M) {
        k_sort_thr<<<blocks, SB, 0, s>>>(v);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_sort_hist<<<blocks, SB, 0, s>>>(v);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (v.m > NSGA3_FAST_M)
        k_sort_scatter_rows<<<(unsigned)(((long long)v.n2 * 32 + 255) / 256), 256, 0, s>>>(v);
    else
        k_sort_scatter<<<(v.n2 + 255) / 256, 256, 0, s>>>(v);
    return cudaGetLastError();
}
