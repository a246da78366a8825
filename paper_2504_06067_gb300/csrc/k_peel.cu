// k_peel.cu -- non-dominated front peeling over the bit-packed matrix
// (Alg. 1 line 3: fronts F_1, F_2, ... until |F_1| + ... + |F_l| >= N,
// splitting R_t into S = F_1..F_{l-1}, F_l and F_drop; Sec. II-C).
//
// One launch per front, replayed by a CUDA-graph WHILE node; the last CTA
// of a pass sets the node's condition, so the host never synchronises.
// Positions are in bucket order of f_0 (k_sort.cu); ranks are written back
// to the original order by k_post_peel.
//   pass 0:   cnt[j]  = popc over all dominator words of column j
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

constexpr int PT = 1024;          // threads per CTA: 32 warps split the dominator rows
constexpr int PW = PT / 32;
constexpr int LISTCAP = 2048;

__global__ void __launch_bounds__(PT) k_peel(RunView v, cudaGraphConditionalHandle h, int in_graph)
{
    __shared__ int red[PW][NSGA3_PEEL_COLS];
    __shared__ uint2 list[LISTCAP];
    __shared__ int nlist;
    __shared__ uint32_t kmax;
    __shared__ int slim;
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

    uint32_t rw = (tid < NSGA3_PEEL_COLS / 32) ? v.rem[j0 / 32 + tid] : 0u;
    const int any_rem = __syncthreads_or(rw != 0u);
    // Dominators of a column have f_0 <= its f_0: in bucket order, only row
    // blocks whose first bucket key is <= the chunk's largest key can hold
    // bits for this chunk (keys are non-decreasing along the order).
    int lim;
    if (k == 0) {
        if (tid == 0) kmax = 0u;
        __syncthreads();
        if (tid < NSGA3_PEEL_COLS && j0 + tid < v.n2) atomicMax(&kmax, v.skey[j0 + tid]);
        __syncthreads();
        const uint32_t km = kmax;
        int cntb = 0;
        for (int I = tid; I < v.NW; I += PT) cntb += (v.skey[I * 32] <= km);
        cntb = warp_sum(cntb);
        if (tid == 0) slim = 0;
        __syncthreads();
        if (lane == 0 && cntb) atomicAdd(&slim, cntb);
        __syncthreads();
        lim = slim;
        if (tid == 0) {
            v.chunk_lim[chunk] = (uint32_t)lim;
            if (any_rem) atomicAdd(&c->peel_rows, (unsigned)lim);
        }
    } else {
        lim = (int)v.chunk_lim[chunk];
    }

    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    if (any_rem) {
        const uint4* base = reinterpret_cast<const uint4*>(v.Dom + j0) + lane;
        const size_t ld4 = (size_t)v.ld / 4;
        if (k == 0) {
            int w = warp;
            for (; w + 7 * PW < lim; w += 8 * PW) {
                uint4 x[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) x[t] = __ldg(base + (size_t)(w + PW * t) * ld4);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    a0 += __popc(x[t].x);
                    a1 += __popc(x[t].y);
                    a2 += __popc(x[t].z);
                    a3 += __popc(x[t].w);
                }
            }
            for (; w < lim; w += PW) {
                const uint4 x = __ldg(base + (size_t)w * ld4);
                a0 += __popc(x.x);
                a1 += __popc(x.y);
                a2 += __popc(x.z);
                a3 += __popc(x.w);
            }
        } else {
            const uint32_t* prev = v.front + ((k - 1) & 1) * v.NW;
            for (int wb = 0; wb < lim; wb += LISTCAP) {
                const int whe = min(wb + LISTCAP, lim);
                if (tid == 0) nlist = 0;
                __syncthreads();
                for (int w = wb + tid; w < whe; w += PT) {
                    const uint32_t msk = prev[w];
                    if (msk) list[atomicAdd(&nlist, 1)] = make_uint2((unsigned)w, msk);
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
#pragma unroll 8
        for (int w = 0; w < PW; ++w) sum += red[w][tid];
        const int j = j0 + tid;
        bool nf = false;
        if (j < v.n2 && v.srank[j] < 0) {
            const int cv = (k == 0) ? sum : v.cnt[j] - sum;
            v.cnt[j] = cv;
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

// ranks back to the original order; the first thread sets the niching branch
__global__ void k_post_peel(RunView v, cudaGraphConditionalHandle h_niche, int in_graph)
{
    Ctrl* c = v.ctrl;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < v.n2) v.rank2[v.perm[p]] = v.srank[p];
    if (p == 0 && in_graph) {
        const int go = (read_status(c) == 0 && c->l >= 0 && c->need_niche) ? 1 : 0;
        cudaGraphSetConditional(h_niche, (unsigned)go);
    }
}

}  // namespace

int peel_nsplit(const RunView& v, int num_sms)
{
    (void)v;
    (void)num_sms;
    return 1;  // one CTA per column chunk
}

cudaError_t launch_peel(const RunView& v, int nsplit, cudaGraphConditionalHandle h, int in_graph,
                        cudaStream_t s)
{
    (void)nsplit;
    k_peel<<<v.ld / NSGA3_PEEL_COLS, PT, 0, s>>>(v, h, in_graph);
    return cudaGetLastError();
}

cudaError_t launch_post_peel(const RunView& v, cudaGraphConditionalHandle h_niche, int in_graph,
                             cudaStream_t s)
{
    k_post_peel<<<(v.n2 + 255) / 256, 256, 0, s>>>(v, h_niche, in_graph);
    return cudaGetLastError();
}
