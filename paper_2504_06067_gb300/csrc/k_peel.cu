// k_peel.cu -- non-dominated front peeling over the bit-packed matrix
// (Alg. 1 line 3: fronts F_1, F_2, ... until |F_1| + ... + |F_l| >= N,
// splitting R_t into S = F_1..F_{l-1}, F_l and F_drop; Sec. II-C).
//
// One launch per front, replayed by a CUDA-graph WHILE node; the last CTA
// of a pass sets the node's condition, so the host never synchronises.
//   pass 0:   cnt[j]  = popc over all dominator words of column j
//   pass k>0: cnt[j] -= popc(Dom[w][j] & front_{k-1}[w]) over the nonzero
//             words w of the previous front's mask
//   front_k   = { j unranked : cnt[j] == 0 }, rank2[j] = k
// A CTA owns 128 columns (uint4 per lane) and one of `nsplit` row ranges;
// partial counts meet in global atomics, and the last CTA of each column
// chunk (ticket) ranks its columns, so a front mask word has exactly one
// writer per pass.  Bound: HBM / L2 bandwidth of the Dom reads.
#include "kernels.cuh"

namespace {

constexpr int LISTCAP = 2048;

__global__ void __launch_bounds__(256) k_peel(RunView v, int nsplit, cudaGraphConditionalHandle h,
                                              int in_graph)
{
    __shared__ int red[8][NSGA3_PEEL_COLS];
    __shared__ uint2 list[LISTCAP];
    __shared__ int nlist;
    __shared__ unsigned ticket;
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
    const int chunk = blockIdx.x / nsplit, split = blockIdx.x - chunk * nsplit;
    const int j0 = chunk * NSGA3_PEEL_COLS;
    const int w_lo = (int)((long long)split * v.NW / nsplit);
    const int w_hi = (int)((long long)(split + 1) * v.NW / nsplit);

    uint32_t rw = (tid < NSGA3_PEEL_COLS / 32) ? v.rem[j0 / 32 + tid] : 0u;
    const int any_rem = __syncthreads_or(rw != 0u);

    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    if (any_rem) {
        const uint4* base = reinterpret_cast<const uint4*>(v.Dom + j0) + lane;
        const size_t ld4 = (size_t)v.ld / 4;
        if (k == 0) {
            int w = w_lo + warp;
            for (; w + 24 < w_hi; w += 32) {
                uint4 x0 = __ldg(base + (size_t)w * ld4);
                uint4 x1 = __ldg(base + (size_t)(w + 8) * ld4);
                uint4 x2 = __ldg(base + (size_t)(w + 16) * ld4);
                uint4 x3 = __ldg(base + (size_t)(w + 24) * ld4);
                a0 += __popc(x0.x) + __popc(x1.x) + __popc(x2.x) + __popc(x3.x);
                a1 += __popc(x0.y) + __popc(x1.y) + __popc(x2.y) + __popc(x3.y);
                a2 += __popc(x0.z) + __popc(x1.z) + __popc(x2.z) + __popc(x3.z);
                a3 += __popc(x0.w) + __popc(x1.w) + __popc(x2.w) + __popc(x3.w);
            }
            for (; w < w_hi; w += 8) {
                uint4 x = __ldg(base + (size_t)w * ld4);
                a0 += __popc(x.x);
                a1 += __popc(x.y);
                a2 += __popc(x.z);
                a3 += __popc(x.w);
            }
        } else {
            const uint32_t* prev = v.front + ((k - 1) & 1) * v.NW;
            for (int wb = w_lo; wb < w_hi; wb += LISTCAP) {
                const int whe = min(wb + LISTCAP, w_hi);
                if (tid == 0) nlist = 0;
                __syncthreads();
                for (int w = wb + tid; w < whe; w += blockDim.x) {
                    uint32_t msk = prev[w];
                    if (msk) list[atomicAdd(&nlist, 1)] = make_uint2((unsigned)w, msk);
                }
                __syncthreads();
                const int n = nlist;
                int e = warp;
                for (; e + 8 < n; e += 16) {
                    uint2 L0 = list[e], L1 = list[e + 8];
                    uint4 x0 = __ldg(base + (size_t)L0.x * ld4);
                    uint4 x1 = __ldg(base + (size_t)L1.x * ld4);
                    a0 += __popc(x0.x & L0.y) + __popc(x1.x & L1.y);
                    a1 += __popc(x0.y & L0.y) + __popc(x1.y & L1.y);
                    a2 += __popc(x0.z & L0.y) + __popc(x1.z & L1.y);
                    a3 += __popc(x0.w & L0.y) + __popc(x1.w & L1.y);
                }
                for (; e < n; e += 8) {
                    uint2 L = list[e];
                    uint4 x = __ldg(base + (size_t)L.x * ld4);
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
    if (tid < NSGA3_PEEL_COLS) {
        int sum = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) sum += red[w][tid];
        const int j = j0 + tid;
        if (sum != 0 && j < v.n2 && v.rank2[j] < 0) atomicAdd(&v.cnt[j], k == 0 ? sum : -sum);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) ticket = atomicAdd(&v.chunk_done[chunk], 1u);
    __syncthreads();
    if (ticket != (unsigned)(nsplit - 1)) return;

    // last split of this column chunk: rank its columns
    __threadfence();
    if (tid < NSGA3_PEEL_COLS) {
        const int j = j0 + tid;
        bool nf = false;
        if (j < v.n2 && v.rank2[j] < 0) {
            int cv = atomicAdd(&v.cnt[j], 0);
            if (cv == 0) {
                v.rank2[j] = k;
                nf = true;
            }
        }
        uint32_t word = __ballot_sync(0xffffffffu, nf);
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
    if (tid == 0) v.chunk_done[chunk] = 0;
    __threadfence();
    __syncthreads();
    if (tid != 0) return;
    unsigned g = atomicAdd(&c->chunks_done, 1u);
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
    const unsigned fw = atomicAdd(&c->front_words, 0u);
    if (more) c->peel_rows += fw;  // rows the next pass reads
    c->front_words = 0u;
    c->front_size = 0;
    c->chunks_done = 0;
    c->k = k + 1;
    c->peel_more = more ? 1 : 0;
    __threadfence();
    if (in_graph) cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void k_post_peel(RunView v, cudaGraphConditionalHandle h_niche)
{
    Ctrl* c = v.ctrl;
    const int go = (read_status(c) == 0 && c->l >= 0 && c->need_niche) ? 1 : 0;
    cudaGraphSetConditional(h_niche, (unsigned)go);
}

}  // namespace

int peel_nsplit(const RunView& v, int num_sms)
{
    const int nchunks = v.ld / NSGA3_PEEL_COLS;
    int target = num_sms * 8;
    int ns = (target + nchunks - 1) / nchunks;
    if (ns < 1) ns = 1;
    if (ns > 16) ns = 16;
    if (ns > v.NW) ns = v.NW;
    return ns;
}

cudaError_t launch_peel(const RunView& v, int nsplit, cudaGraphConditionalHandle h, int in_graph,
                        cudaStream_t s)
{
    const int nchunks = v.ld / NSGA3_PEEL_COLS;
    k_peel<<<nchunks * nsplit, 256, 0, s>>>(v, nsplit, h, in_graph);
    return cudaGetLastError();
}

cudaError_t launch_post_peel(const RunView& v, cudaGraphConditionalHandle h_niche, cudaStream_t s)
{
    k_post_peel<<<1, 1, 0, s>>>(v, h_niche);
    return cudaGetLastError();
}
