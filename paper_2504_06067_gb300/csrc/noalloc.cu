// noalloc.cu -- non-dominated sorting ranks without any device allocation.
//
// Some callers cannot call cudaMalloc: code that enqueues work while a
// stream is being captured into a CUDA graph (allocation is not a stream
// operation and is refused or unsafe during global-mode capture), latency-
// critical loops that forbid allocator calls, and host applications that
// only hand their plug-ins pre-reserved memory.  nsga3_rank_noalloc serves
// them: its workspace is one file-scope __device__ array of fixed size that
// every GPU loading this library holds until the process exits.
//
// One kernel: each CTA builds the dominance words of 32 columns into the
// scratch matrix (bit i mod 32 of word [i/32][j] = "i dominates j") and their
// dominator counts; the last CTA to finish (ticket) peels every front with
// block barriers and writes the ranks.  The caller's inputs and outputs are
// its own device memory.
#include <mutex>

#include "common.cuh"
#include "nsga3.h"

namespace {

constexpr int NA_N = NSGA3_NOALLOC_MAX_N;  // points
constexpr int NA_W = NA_N / 32;            // dominance words per column
constexpr int NA_T = 512;                  // threads per CTA

struct NoAllocScratch {
    uint32_t dom[NA_W * NA_N];  // 512 KB
    int32_t cnt[NA_N];
    uint32_t front[2][NA_W];
    unsigned ticket;
};

// Process-lifetime workspace.  Host code must not take its address directly
// (the host-side symbol is a stand-in); the device address comes from
// cudaGetSymbolAddress once per device.
static __device__ __align__(256) NoAllocScratch g_na_scratch;

std::mutex g_na_mutex;
NoAllocScratch* g_na_ptr[64] = {nullptr};

__global__ void __launch_bounds__(NA_T) k_rank_noalloc(const float* __restrict__ F, int n, int m,
                                                       int32_t* __restrict__ ranks, NoAllocScratch* S)
{
    __shared__ float scol[32 * NSGA3_FAST_M];
    __shared__ int ccnt[32];
    __shared__ unsigned s_ticket;
    const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5, nwarps = NA_T / 32;
    const int J = blockIdx.x;  // column block
    const int W = (n + 31) / 32;
    for (int e = tid; e < 32 * m; e += NA_T) {
        const int c = e / m, q = e - c * m;
        const int j = J * 32 + c;
        scol[e] = j < n ? F[(size_t)j * m + q] : 0.0f;
    }
    if (tid < 32) ccnt[tid] = 0;
    __syncthreads();
    // warp w: row blocks I = w, w + nwarps, ...; lane = row i, ballot over rows per column
    for (int I = warp; I < W; I += nwarps) {
        const int i = I * 32 + lane;
        float fi[NSGA3_FAST_M];
        for (int q = 0; q < m; ++q) fi[q] = i < n ? F[(size_t)i * m + q] : 0.0f;
        uint32_t keep = 0u;
        for (int k = 0; k < 32; ++k) {
            const int j = J * 32 + k;
            bool all_le = true, any_lt = false;
            for (int q = 0; q < m; ++q) {
                const float a = fi[q], b = scol[k * m + q];
                all_le = all_le && (a <= b);
                any_lt = any_lt || (a < b);
            }
            const bool dom = i < n && j < n && all_le && any_lt;
            const uint32_t word = __ballot_sync(0xffffffffu, dom);
            if (lane == k) keep = word;
        }
        const int j = J * 32 + lane;
        if (j < n) {
            S->dom[(size_t)I * NA_N + j] = keep;
            if (keep) atomicAdd(&ccnt[lane], __popc(keep));
        }
    }
    __syncthreads();
    if (tid < 32 && J * 32 + tid < n) S->cnt[J * 32 + tid] = ccnt[tid];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_ticket = atomicAdd(&S->ticket, 1u);
    __syncthreads();
    if (s_ticket != gridDim.x - 1) return;
    __threadfence();

    // last CTA: peel every front; counts and ranks live in shared memory
    // (thread tid owns columns tid, tid + NA_T, ...)
    __shared__ int sc[NA_N];
    __shared__ int sr[NA_N];
    __shared__ uint2 list[NA_W];
    __shared__ int nlist;
    for (int j = tid; j < W * 32; j += NA_T) {
        const int cv = j < n ? __ldcg(&S->cnt[j]) : -1;
        sc[j] = cv;
        sr[j] = cv == 0 ? 0 : -1;
        const uint32_t word = __ballot_sync(0xffffffffu, cv == 0);
        if (lane == 0) S->front[0][j >> 5] = word;
    }
    __syncthreads();
    for (int k = 1; k < n; ++k) {
        const uint32_t* prev = S->front[(k - 1) & 1];
        if (tid == 0) nlist = 0;
        __syncthreads();
        for (int w = tid; w < W; w += NA_T) {
            const uint32_t msk = __ldcg(&prev[w]);
            if (msk) list[atomicAdd(&nlist, 1)] = make_uint2((unsigned)w, msk);
        }
        __syncthreads();
        const int nl = nlist;
        if (nl == 0) break;  // the previous front was empty: every point is ranked
        for (int j0 = warp * 32; j0 < W * 32; j0 += nwarps * 32) {
            const int j = j0 + lane;
            bool nf = false;
            if (j < n && sr[j] < 0) {
                int dec = 0;
                for (int e = 0; e < nl; ++e)
                    dec += __popc(__ldcg(&S->dom[(size_t)list[e].x * NA_N + j]) & list[e].y);
                const int cv = sc[j] - dec;
                sc[j] = cv;
                if (cv == 0) {
                    sr[j] = k;
                    nf = true;
                }
            }
            const uint32_t word = __ballot_sync(0xffffffffu, nf);
            if (lane == 0) S->front[k & 1][j0 >> 5] = word;
        }
        __syncthreads();
    }
    for (int j = tid; j < n; j += NA_T) ranks[j] = sr[j];
    if (tid == 0) S->ticket = 0u;
}

}  // namespace

extern "C" nsga3_status nsga3_rank_noalloc(const float* objs, int n, int m, int32_t* ranks, void* stream)
{
    if (!objs || !ranks || n < 1 || n > NA_N || m < 2 || m > NSGA3_FAST_M) return NSGA3_EINVAL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return NSGA3_ECUDA;
    }
    NoAllocScratch* S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_ptr[dev]) {
            // set-up once per device, with that device current
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_na_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return NSGA3_ECUDA;
            }
            g_na_ptr[dev] = static_cast<NoAllocScratch*>(p);
        }
        S = g_na_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the completion ticket must start at zero even if an earlier call failed
    e = cudaMemsetAsync(&S->ticket, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        const int blocks = (n + 31) / 32;
        k_rank_noalloc<<<blocks, NA_T, 0, s>>>(objs, n, m, ranks, S);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? NSGA3_OK : NSGA3_ECUDA;
}
