// k_misc.cu -- per-selection reset, boundary check of the objectives,
// compaction of the selected indices and the next-population gather
// (Alg. 2 last line: P_{t+1} = rows with rank < l after selection).
#include "kernels.cuh"

namespace {

__global__ void k_sel_reset(RunView v)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int j = tid; j < v.ld; j += stride) {
        v.cnt[j] = 0;
        v.rank2[j] = -1;
        v.srank[j] = -1;
    }
    for (int b = tid; b <= (1 << v.kbits); b += stride) v.bcnt[b] = 0;
    if (v.qhist)
        for (int b = tid; b < v.m * SORT_QB; b += stride) v.qhist[b] = 0;
    if (v.dnz) {
        // the block bitmap starts empty: only tiles with block pairs to test write bytes
        const long long nb = (long long)v.NW * v.NB8;  // 8 T^2 bytes, T = ld / 256
        uint2* z = reinterpret_cast<uint2*>(v.dnz);
        for (long long e = tid; e < nb / 8; e += stride) z[e] = make_uint2(0u, 0u);
    }
    for (int wd = tid; wd < v.NW; wd += stride) {
        const int lo = wd * 32;
        uint32_t m = 0u;
        if (lo + 32 <= v.n2)
            m = 0xffffffffu;
        else if (lo < v.n2)
            m = (1u << (v.n2 - lo)) - 1u;
        v.rem[wd] = m;
        v.selmask[wd] = 0u;
    }
    for (int j = tid; j < v.w; j += stride) {
        v.rho[j] = 0;
        v.rhop[j] = 0;
        v.cursor[j] = 0;
    }
    if (tid == 0) {
        Ctrl* c = v.ctrl;
        c->sbar = 0u;
        c->pbar = 0ull;
        c->prel = 0ull;
        c->cum = 0;
        c->l = -1;
        c->nS = 0;
        c->K = 0;
        c->nFl = 0;
        c->need_niche = 0;
        c->fallback = 0;
        c->passes = 0;
        c->nT = 0;
        c->Lstar = -1;
        c->rlev = 0;
        c->nsel = 0;
        c->nlarge = 0;
        c->npath = 0u;
        c->ntile = 0;
        for (int t = 0; t < 8; ++t) c->domstat[t] = 0ull;
        c->peel_rows = 0u;
        c->ncand = 0;
        c->nslow = 0;
        c->ext_done = 0u;
        c->sort_done = 0u;
        c->f0lo = 0xffffffffu;
        c->f0hi = 0u;
        c->thr_done = 0u;
        for (int q = 0; q < NSGA3_FAST_M; ++q) {
            c->omin[q] = 0xffffffffu;
            c->omax[q] = 0u;
        }
        c->cmp_done = 0u;
        c->overflow = 0;
        c->recheck_miss = 0;
        for (int q = 0; q < v.m; ++q) c->zmin[q] = 0xffffffffu;
    }
}

__global__ void k_check_finite(RunView v)
{
    const long long n = (long long)v.n2 * v.m;
    bool bad = false;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(v.F[e]);
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) set_status(v.ctrl, DEV_ENONFINITE);
}

// selected = S u (picked members of F_l), or S u F_l when no niching is
// needed, in ascending index order.  Every warp builds one 32-member mask
// word (ballot); the last CTA to finish scans the words' popcounts and
// writes the indices.
__global__ void __launch_bounds__(1024) k_compact(RunView v)
{
    uint32_t* words = v.front;  // front masks are dead after the peel: NW words of scratch
    __shared__ int scratch[40];
    __shared__ unsigned ticket;
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int l = c->l, need = c->need_niche;
    const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int wd = blockIdx.x * nwarps + warp;
    if (wd < v.NW) {
        const int j = wd * 32 + lane;
        const int r = j < v.n2 ? v.rank2[j] : -1;
        const bool take = r >= 0 && (r < l || (r == l && (!need || ((v.selmask[wd] >> lane) & 1u))));
        const uint32_t word = __ballot_sync(0xffffffffu, take);
        if (lane == 0) words[wd] = word;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(&c->cmp_done, 1u);
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    __threadfence();
    // last CTA: warp w owns a contiguous run of words; lane-parallel popcounts
    // and a block scan give each word's first output slot, then every word's
    // set bits are written by its warp at consecutive (coalesced) positions
    const int per = (v.NW + nwarps - 1) / nwarps;
    const int wlo = min(v.NW, warp * per), whi = min(v.NW, wlo + per);
    int wsum = 0;
    for (int t0 = wlo; t0 < whi; t0 += 32) {
        const int t = t0 + lane;
        wsum += (t < whi) ? __popc(__ldcg(&words[t])) : 0;
    }
    wsum = warp_sum(wsum);
    if (lane == 0) scratch[warp] = wsum;
    __syncthreads();
    if (warp == 0) {
        const int x = lane < nwarps ? scratch[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        scratch[lane] = xi - x;
        if (lane == 31) scratch[32] = xi;
    }
    __syncthreads();
    int run = scratch[warp];
    for (int t0 = wlo; t0 < whi; t0 += 32) {
        const int t = t0 + lane;
        const uint32_t word_l = (t < whi) ? __ldcg(&words[t]) : 0u;
        const int cnt_l = __popc(word_l);
        int inc = cnt_l;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int nw = min(32, whi - t0);
        for (int u = 0; u < nw; ++u) {
            const uint32_t wu = __shfl_sync(0xffffffffu, word_l, u);
            const int off = run + __shfl_sync(0xffffffffu, inc - cnt_l, u);
            if ((wu >> lane) & 1u) {
                const int pos = off + __popc(wu & ((1u << lane) - 1u));
                if (pos < v.N) v.sel[pos] = (t0 + u) * 32 + lane;
            }
        }
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (threadIdx.x == 0) {
        c->cmp_done = 0u;
        c->nsel = scratch[32];
        if (scratch[32] != v.N) set_status(c, DEV_EINTERNAL);
    }
}

// next population rows (warp per row)
__global__ void k_gather(RunView v)
{
    if (read_status(v.ctrl)) return;
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = lane_id();
    if (p >= v.N) return;
    const int i = v.sel[p];
    const float* src = v.X + (size_t)i * v.d;
    float* dst = v.Xtmp + (size_t)p * v.d;
    if ((v.d & 3) == 0) {  // rows start on 16-byte boundaries: 16-byte copies
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int e = lane; e < v.d / 4; e += 32) d4[e] = __ldg(s4 + e);
    } else {
        for (int e = lane; e < v.d; e += 32) dst[e] = src[e];
    }
    for (int q = lane; q < v.m; q += 32) v.Ftmp[(size_t)p * v.m + q] = v.F[(size_t)i * v.m + q];
    if (lane == 0) v.ranktmp[p] = v.rank2[i];
}

// the gathered rows become the parents (one kernel for X, F and rank) and
// the generation counter advances
__global__ void k_commit(RunView v)
{
    if (read_status(v.ctrl)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nx = (long long)v.N * v.d;
    if ((nx & 3) == 0) {
        const float4* src = reinterpret_cast<const float4*>(v.Xtmp);
        float4* dst = reinterpret_cast<float4*>(v.X);
        for (long long e = t0; e < nx / 4; e += stride) dst[e] = src[e];
    } else {
        for (long long e = t0; e < nx; e += stride) v.X[e] = v.Xtmp[e];
    }
    for (long long e = t0; e < (long long)v.N * v.m; e += stride) v.F[e] = v.Ftmp[e];
    for (long long e = t0; e < v.N; e += stride) v.rank[e] = v.ranktmp[e];
    if (t0 == 0) v.ctrl->gen += 1u;
}

__global__ void k_nan_pad(RunView v)
{
    const long long lo = (long long)v.n2 * v.m, hi = (long long)v.ld * v.m;
    for (long long e = lo + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < hi;
         e += (long long)gridDim.x * blockDim.x) {
        v.F[e] = __int_as_float(0x7fc00000);
        v.Fp[e] = __int_as_float(0x7fc00000);
    }
    for (int p = v.n2 + blockIdx.x * blockDim.x + threadIdx.x; p < v.ld; p += gridDim.x * blockDim.x)
        v.skey[p] = 0xffffffffu;
}

// the wait self-test: one thread waits, with the barriers' bounded wait, for
// a word nothing sets
__global__ void k_wait_probe(RunView v)
{
    if (threadIdx.x != 0) return;
    Ctrl* c = v.ctrl;
    bounded_wait(c, v.wait_ns, [&] { return ld_acquire(&c->never) != 0u; });
}

}  // namespace

cudaError_t launch_wait_probe(const RunView& v, cudaStream_t s)
{
    k_wait_probe<<<1, 32, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_sel_reset(const RunView& v, cudaStream_t s)
{
    int n = v.ld > v.w ? v.ld : v.w;
    int blocks = (n + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    k_sel_reset<<<blocks, 256, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const RunView& v, cudaStream_t s)
{
    long long n = (long long)v.n2 * v.m;
    long long blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    k_check_finite<<<(unsigned)blocks, 256, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_compact(const RunView& v, cudaStream_t s)
{
    k_compact<<<(v.NW + 31) / 32, 1024, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_gather(const RunView& v, cudaStream_t s)
{
    long long threads = (long long)v.N * 32;
    k_gather<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long blocks = ((long long)v.N * v.d / 4 + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    k_commit<<<(unsigned)blocks, 256, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_nan_pad(const RunView& v, cudaStream_t s)
{
    k_nan_pad<<<64, 256, 0, s>>>(v);
    return cudaGetLastError();
}

