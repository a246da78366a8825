// k_peel.cu -- non-dominated front peeling over the bit-packed matrix
// (Alg. 1, the non-dominated sort: fronts F_1, F_2, ... until |F_1| + ... + |F_l| >= N,
// splitting R_t into S = F_1..F_{l-1}, F_l and F_drop; Sec. II-C).
//
// One cooperative launch runs every pass: the CTAs meet at a grid barrier
// (common.cuh) after each pass and all take the same decision from the
// front size, so the host never synchronises.
// Positions are in bucket order of f_0 (k_sort.cu); ranks are written back
// to the original order by k_norm_ideal.
//   cnt[j]    = dominators of j, counted by the dominance build
//   pass k>0: cnt[j] -= popc(Dom[w][j] & front_{k-1}[w]) over the nonzero
//             words w of the previous front's mask
//   front_k   = { j unranked : cnt[j] == 0 }, rank2[j] = k
// A CTA of 32 warps owns 128 columns (uint4 per lane); its warps split the
// dominator rows and meet in shared memory, so the CTA alone updates its
// columns' counts, ranks them and writes their front-mask words.  Bound:
// HBM / L2 bandwidth of the Dom reads.
#include <math_constants.h>

#include "kernels.cuh"

namespace {

constexpr int PEEL_THREADS = 512;  // threads per CTA
constexpr int PWMAX = PEEL_THREADS / 32;
constexpr int LISTCAP = 2048;

template <bool STREAM>
__global__ void __launch_bounds__(PEEL_THREADS, STREAM ? 1 : 2) k_peel(RunView v)
{
    __shared__ int red[PWMAX][NSGA3_PEEL_COLS];
    const int PT = blockDim.x, PW = PT >> 5;
    __shared__ uint2 list[LISTCAP];
    __shared__ int nlist;
    __shared__ unsigned s_fs;             // this CTA's members of the front of this pass
    __shared__ unsigned long long s_cum;  // points ranked, from the barrier
    __shared__ float rowbuf[STREAM ? PWMAX : 1][32][NSGA3_FAST_M];  // streaming: members of a front word
    Ctrl* c = v.ctrl;
    const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    if (read_status(c)) return;  // uniform: set only by earlier kernels
    const int nchunks = v.ld / NSGA3_PEEL_COLS;
    // every CTA follows the same sequence of front sizes, so each keeps the
    // pass state itself; CTA 0 also publishes it in ctrl
    int cum = 0, l = -1;
    for (int k = 0;; ++k) {
        if (tid == 0) s_fs = 0u;  // read after the barrier's first __syncthreads
        __syncthreads();
        for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
            const int j0 = chunk * NSGA3_PEEL_COLS;
            // prefetch this thread's column state (used after the reduction)
            int my_rank = 0, my_cnt = 0;
            if (tid < NSGA3_PEEL_COLS && j0 + tid < v.n2) {
                my_rank = __ldcg(&v.srank[j0 + tid]);
                my_cnt = __ldcg(&v.cnt[j0 + tid]);
            }
            // Dominators of a column have a sort key <= its key (k_sort.cu).  Keys
            // are non-decreasing in position order and bcnt[b] is the end of key b,
            // so the positions that can dominate this chunk end at bcnt[key of its
            // last column].
            const int jl = min(j0 + NSGA3_PEEL_COLS, v.n2) - 1;
            int lim = 0;
            if (jl >= j0) lim = (v.bcnt[v.skey[jl]] + 31) >> 5;
            if (lim > v.NW) lim = v.NW;

            uint32_t rw = (tid < NSGA3_PEEL_COLS / 32) ? __ldcg(&v.rem[j0 / 32 + tid]) : 0u;
            const int any_rem = __syncthreads_or(rw != 0u);

            uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            // pass 0 needs no words: the dominance build already counted every
            // column's dominators into cnt[]
            if (STREAM && any_rem && k > 0) {
                // no matrix: every member of front k-1 (up to the row limit)
                // is tested against this lane's four columns lane*4 .. +3,
                // with the sign-bit test of the dominance build; a member
                // whose f_0 is below every f_0 of the chunk needs objectives
                // 1..m-1 only (f_0 makes the dominance strict)
                const int m = v.m;
                float fc[4][NSGA3_FAST_M];
                float cmin = CUDART_INF_F;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
#pragma unroll
                    for (int q = 0; q < NSGA3_FAST_M; ++q)
                        fc[t][q] = q < m ? v.Fp[(size_t)(j0 + lane * 4 + t) * m + q] : 0.0f;
                    cmin = fminf(cmin, fc[t][0]);  // NaN padding columns are ignored by fminf
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cmin = fminf(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
                float* rb = rowbuf[warp][0];
                const uint32_t* prev = v.front + ((k - 1) & 1) * v.NW;
                for (int wb = 0; wb < lim; wb += LISTCAP) {
                    const int whe = min(wb + LISTCAP, lim);
                    if (tid == 0) nlist = 0;
                    __syncthreads();
                    for (int w0 = wb + warp * 32; w0 < whe; w0 += PT) {
                        const int w = w0 + lane;
                        const uint32_t msk = w < whe ? __ldcg(&prev[w]) : 0u;
                        const unsigned bal = __ballot_sync(0xffffffffu, msk != 0u);
                        int at = 0;
                        if (lane == 0 && bal) at = atomicAdd(&nlist, __popc(bal));
                        at = __shfl_sync(0xffffffffu, at, 0);
                        if (msk) list[at + __popc(bal & ((1u << lane) - 1u))] = make_uint2((unsigned)w, msk);
                    }
                    __syncthreads();
                    const int n = nlist;
                    if (tid == 0) atomicAdd(&c->peel_rows, (unsigned)n);
                    for (int e = warp; e < n; e += PW) {
                        const uint2 L = list[e];
                        // the word's members, one per lane, into this warp's row buffer
                        if ((L.y >> lane) & 1u) {
                            const size_t p = (size_t)L.x * 32 + lane;
#pragma unroll
                            for (int q = 0; q < NSGA3_FAST_M; ++q)
                                if (q < m) rb[lane * NSGA3_FAST_M + q] = __ldg(&v.Fp[p * m + q]);
                        }
                        __syncwarp();
                        uint32_t mk = L.y;
                        while (mk) {  // warp-uniform: every lane walks the same rows
                            const int b = __ffs(mk) - 1;
                            mk &= mk - 1u;
                            const float* fi = rb + b * NSGA3_FAST_M;
                            uint32_t d4[4];
                            if (fi[0] < cmin) {
#pragma unroll
                                for (int t = 0; t < 4; ++t) {
                                    uint32_t oa = 0u;
#pragma unroll
                                    for (int q = 1; q < NSGA3_FAST_M; ++q)
                                        if (q < m) oa |= __float_as_uint(fc[t][q] - fi[q]);
                                    d4[t] = (~oa) >> 31;  // no f_iq > f_jq
                                }
                            } else {
#pragma unroll
                                for (int t = 0; t < 4; ++t) {
                                    uint32_t oa = 0u, ob = 0u;
#pragma unroll
                                    for (int q = 0; q < NSGA3_FAST_M; ++q)
                                        if (q < m) {
                                            oa |= __float_as_uint(fc[t][q] - fi[q]);
                                            ob |= __float_as_uint(fi[q] - fc[t][q]);
                                        }
                                    d4[t] = (ob & ~oa) >> 31;  // none greater, some smaller
                                }
                            }
                            a0 += d4[0];
                            a1 += d4[1];
                            a2 += d4[2];
                            a3 += d4[3];
                        }
                        __syncwarp();
                    }
                    __syncthreads();
                }
            } else if (!STREAM && any_rem && k > 0) {
                const uint4* base = reinterpret_cast<const uint4*>(v.Dom + j0) + lane;
                const size_t ld4 = (size_t)v.ld / 4;
                // with the block bitmap (m <= 10) only the Dom blocks whose bit
                // is set were written this selection: the lane's column block
                // J = j0 / 32 + lane / 8 is read from dominator block w only if
                // bit J of dnz[w] is set
                const int Jb = j0 / 32 + (lane >> 3);
                const uint8_t* nzrow = v.dnz ? v.dnz + (Jb >> 3) : nullptr;
                const unsigned nzbit = 1u << (Jb & 7);
                auto load = [&](unsigned w) -> uint4 {
                    if (nzrow && !(nzrow[(size_t)w * v.NB8] & nzbit)) return make_uint4(0u, 0u, 0u, 0u);
                    return __ldg(base + (size_t)w * ld4);
                };
                {
                    const uint32_t* prev = v.front + ((k - 1) & 1) * v.NW;
                    for (int wb = 0; wb < lim; wb += LISTCAP) {
                        const int whe = min(wb + LISTCAP, lim);
                        if (tid == 0) nlist = 0;
                        __syncthreads();
                        for (int w0 = wb + warp * 32; w0 < whe; w0 += PT) {
                            const int w = w0 + lane;
                            const uint32_t msk = w < whe ? __ldcg(&prev[w]) : 0u;
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
                                x[t] = load(L[t].x);
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
                            const uint4 x = load(L.x);
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
                    v.rem[wd] = __ldcg(&v.rem[wd]) & ~word;
                    if (word) atomicAdd(&s_fs, (unsigned)__popc(word));
                }
            }

            __syncthreads();  // red and list are reused by the next chunk
        }
        // the barrier returns the points ranked after pass k
        const unsigned long long tot = grid_sync_sum(c, &c->pbar, &c->prel, (unsigned)k, s_fs, v.wait_ns, &s_cum);
        if (tot == ~0ull) return;
        // close front k (the same decision in every CTA)
        const int ncum = (int)tot;
        const int fs = ncum - cum;
        bool first = false;
        if (l < 0 && ncum >= v.N) {
            l = k;
            first = true;
        }
        const bool broken = fs == 0 && ncum < v.n2;
        const bool more = !broken && fs > 0 && ncum < v.n2 && (v.full_sort || l < 0);
        if (blockIdx.x == 0 && tid == 0) {
            c->cum = ncum;
            c->passes = k + 1;
            c->passes_total += 1ull;
            if (first) {
                c->l = k;
                c->nFl = fs;
                c->nS = cum;
                c->K = v.N - cum;
                c->need_niche = (v.N - cum) < fs ? 1 : 0;
            }
            if (broken) set_status(c, DEV_EINTERNAL);
        }
        cum = ncum;
        if (!more) break;
    }
}


int g_peel_occ[2] = {0, 0};  // resident peel CTAs per SM (matrix, streaming), set at start-up

}  // namespace

// One cooperative launch for all passes: at most as many CTAs as can be
// resident at once (the grid barrier needs them all), at most one per chunk.
cudaError_t launch_peel(const RunView& v, int num_sms, cudaStream_t s)
{
    const int nchunks = v.ld / NSGA3_PEEL_COLS;
    int occ = g_peel_occ[v.streaming ? 1 : 0];
    if (occ <= 0) occ = 1;
    if (v.peel_ctas > 0 && v.peel_ctas < occ) occ = v.peel_ctas;  // launch-shape option
    int grid = num_sms * occ;
    if (v.shared_gpu) {
        // a quarter of the chunks per pass at most: every CTA of a cooperative
        // launch must be resident at once, which a mix of runs rarely allows
        // for a grid the size of the GPU (64 batched runs: 4.27x -> 4.61x the
        // plain path)
        const int g2 = nchunks / 4 > 0 ? nchunks / 4 : 1;
        if (grid > g2) grid = g2;
    }
    if (grid > nchunks) grid = nchunks;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(PEEL_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (v.streaming) return cudaLaunchKernelEx(&cfg, k_peel<true>, v);
    return cudaLaunchKernelEx(&cfg, k_peel<false>, v);
}

cudaError_t peel_init_attributes()
{
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_peel_occ[0], k_peel<false>, PEEL_THREADS, 0);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_peel_occ[1], k_peel<true>, PEEL_THREADS, 0);
}

