// k_peel.cu -- non-dominated front peeling over the bit-packed matrix
// (Alg. 1 line 3: fronts F_1, F_2, ... until |F_1| + ... + |F_l| >= N,
// splitting R_t into S = F_1..F_{l-1}, F_l and F_drop; Sec. II-C).
//
// One launch per front, replayed by a CUDA-graph WHILE node; the last CTA
// of a pass sets the node's condition, so the host never synchronises.
// Positions are in bucket order of f_0 (k_sort.cu); ranks are written back
// to the original order by k_post_peel.
//   cnt[j]    = dominators of j, counted by the dominance build
//   pass k>0: cnt[j] -= popc(Dom[w][j] & front_{k-1}[w]) over the nonzero
//             words w of the previous front's mask
//   front_k   = { j unranked : cnt[j] == 0 }, rank2[j] = k
// A CTA of 32 warps owns 128 columns (uint4 per lane); its warps split the
// dominator rows and meet in shared memory, so the CTA alone updates its
// columns' counts, ranks them and writes their front-mask words.  The last
// CTA of a pass (ticket) closes the front.  Bound: HBM / L2 bandwidth of the
// Dom reads.
#include "kernels.cuh"

namespace {

constexpr int PTMAX = 1024;       // threads per CTA (runtime: 256, 512 or 1024)
constexpr int PWMAX = PTMAX / 32;
constexpr int LISTCAP = 2048;

__global__ void __launch_bounds__(PTMAX) k_peel(RunView v, cudaGraphConditionalHandle h, int in_graph)
{
    __shared__ int red[PWMAX][NSGA3_PEEL_COLS];
    const int PT = blockDim.x, PW = PT >> 5;
    __shared__ uint2 list[LISTCAP];
    __shared__ int nlist;
    Ctrl* c = v.ctrl;
    const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    if (read_status(c)) {
        if (blockIdx.x == 0 && tid == 0) {
            if (in_graph)
                cudaGraphSetConditional(h, 0);
            else
                c->peel_more = 0;
        }
        return;
    }
    const int k = *(volatile int32_t*)&c->k;
    const int nchunks = v.ld / NSGA3_PEEL_COLS;
    const int chunk = blockIdx.x;
    const int j0 = chunk * NSGA3_PEEL_COLS;
    // prefetch this thread's column state (used after the reduction)
    int my_rank = 0, my_cnt = 0;
    if (tid < NSGA3_PEEL_COLS && j0 + tid < v.n2) {
        my_rank = v.srank[j0 + tid];
        my_cnt = v.cnt[j0 + tid];
    }
    // Dominators of a column have f_0 <= its f_0.  Keys are non-decreasing in
    // bucket order and bcnt[b] is the end of bucket b, so the positions that
    // can dominate this chunk end at bcnt[key of its last column].
    const int jl = min(j0 + NSGA3_PEEL_COLS, v.n2) - 1;
    int lim = 0;
    if (jl >= j0) lim = (v.bcnt[v.skey[jl]] + 31) >> 5;
    if (lim > v.NW) lim = v.NW;

    uint32_t rw = (tid < NSGA3_PEEL_COLS / 32) ? v.rem[j0 / 32 + tid] : 0u;
    const int any_rem = __syncthreads_or(rw != 0u);

    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    // pass 0 needs no words: the dominance build already counted every
    // column's dominators into cnt[]
    if (any_rem && k > 0) {
        const uint4* base = reinterpret_cast<const uint4*>(v.Dom + j0) + lane;
        const size_t ld4 = (size_t)v.ld / 4;
        {
            const uint32_t* prev = v.front + ((k - 1) & 1) * v.NW;
            for (int wb = 0; wb < lim; wb += LISTCAP) {
                const int whe = min(wb + LISTCAP, lim);
                if (tid == 0) nlist = 0;
                __syncthreads();
                for (int w0 = wb + warp * 32; w0 < whe; w0 += PT) {
                    const int w = w0 + lane;
                    const uint32_t msk = w < whe ? prev[w] : 0u;
                    const unsigned bal = __ballot_sync(0xffffffffu, msk != 0u);
                    int at = 0;
                    if (lane == 0 && bal) at = atomicAdd(&nlist, __popc(bal));
                    at = __shfl_sync(0xffffffffu, at, 0);
                    if (msk) list[at + __popc(bal & ((1u << lane) - 1u))] = make_uint2((unsigned)w, msk);
                }
                __syncthreads();
                const int n = nlist;
                if (tid == 0) atomicAdd(&c->peel_rows, (unsigned)n);
                int e = warp;
                for (; e + 3 * PW < n; e += 4 * PW) {
                    uint2 L[4];
                    uint4 x[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        L[t] = list[e + PW * t];
                        x[t] = __ldg(base + (size_t)L[t].x * ld4);
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        a0 += __popc(x[t].x & L[t].y);
                        a1 += __popc(x[t].y & L[t].y);
                        a2 += __popc(x[t].z & L[t].y);
                        a3 += __popc(x[t].w & L[t].y);
                    }
                }
                for (; e < n; e += PW) {
                    const uint2 L = list[e];
                    const uint4 x = __ldg(base + (size_t)L.x * ld4);
                    a0 += __popc(x.x & L.y);
                    a1 += __popc(x.y & L.y);
                    a2 += __popc(x.z & L.y);
                    a3 += __popc(x.w & L.y);
                }
                __syncthreads();
            }
        }
    }
    red[warp][lane * 4 + 0] = (int)a0;
    red[warp][lane * 4 + 1] = (int)a1;
    red[warp][lane * 4 + 2] = (int)a2;
    red[warp][lane * 4 + 3] = (int)a3;
    __syncthreads();
    // this CTA owns its 128 columns: update the counts and rank the new front
    if (tid < NSGA3_PEEL_COLS) {
        int sum = 0;
        for (int w = 0; w < PW; ++w) sum += red[w][tid];
        const int j = j0 + tid;
        bool nf = false;
        if (j < v.n2 && my_rank < 0) {
            const int cv = my_cnt - sum;
            if (k > 0) v.cnt[j] = cv;
            if (cv == 0) {
                v.srank[j] = k;
                nf = true;
            }
        }
        const uint32_t word = __ballot_sync(0xffffffffu, nf);
        if (lane == 0) {
            const int wd = j0 / 32 + warp;
            v.front[(k & 1) * v.NW + wd] = word;
            v.rem[wd] &= ~word;
            if (word) {
                atomicAdd(&c->front_size, (unsigned)__popc(word));
                atomicAdd(&c->front_words, 1u);
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (tid != 0) return;
    const unsigned g = atomicAdd(&c->chunks_done, 1u);
    if (g != (unsigned)(nchunks - 1)) return;

    // last chunk of the pass: close front k and decide whether to continue
    __threadfence();
    const int fs = (int)atomicAdd(&c->front_size, 0u);
    const int cum = c->cum + fs;
    c->cum = cum;
    c->passes += 1;
    c->passes_total += 1ull;
    if (c->l < 0 && cum >= v.N) {
        c->l = k;
        c->nFl = fs;
        c->nS = cum - fs;
        c->K = v.N - (cum - fs);
        c->need_niche = c->K < fs ? 1 : 0;
    }
    if (fs == 0 && cum < v.n2) set_status(c, DEV_EINTERNAL);
    const bool more = fs > 0 && cum < v.n2 && (v.full_sort || c->l < 0);
    c->front_words = 0u;
    c->front_size = 0;
    c->chunks_done = 0;
    c->k = k + 1;
    c->peel_more = more ? 1 : 0;
    __threadfence();
    if (in_graph) cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ranks back to the original order
__global__ void k_post_peel(RunView v)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < v.n2) v.rank2[v.perm[p]] = v.srank[p];
}

}  // namespace

// The peel launches one CTA per column chunk; this returns the SM count the
// launch uses to size its CTAs.
int peel_nsplit(const RunView& v, int num_sms)
{
    (void)v;
    return num_sms;
}

cudaError_t launch_peel(const RunView& v, int nsplit, cudaGraphConditionalHandle h, int in_graph,
                        cudaStream_t s)
{
    // every chunk's CTA resident in one wave: one 1024-thread CTA per SM fits
    // (registers), two of 512, four of 256
    const int nchunks = v.ld / NSGA3_PEEL_COLS;
    const int threads = nchunks <= nsplit ? 1024 : (nchunks <= 2 * nsplit ? 512 : 256);
    k_peel<<<nchunks, threads, 0, s>>>(v, h, in_graph);
    return cudaGetLastError();
}

cudaError_t launch_post_peel(const RunView& v, cudaGraphConditionalHandle h_niche, int in_graph,
                             cudaStream_t s)
{
    (void)h_niche;
    (void)in_graph;
    k_post_peel<<<(v.n2 + 255) / 256, 256, 0, s>>>(v);
    return cudaGetLastError();
}
