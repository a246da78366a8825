// k_associate.cu -- association of S u F_l with the reference directions
// (Alg. 2, Eq. 2 read as the perpendicular distance
// D_ij = |f'| sqrt(1 - cos^2), pi_i = argmin_j D_ij, d_i = min_j D_ij) and
// the niche counts rho (over S) and rho' (over F_l) of Alg. 2.
//
// Exactness.  The FP64 distance is evaluated operation for operation like a
// plain CPU evaluation (_rn intrinsics, left-to-right sums), but only for
// candidate references.  Candidates come from FP32 cosines
// qhat_j = u . zhat_j of the unit vectors u = f'/|f'| and zhat_j = z_j/|z_j|
// (all components >= 0).  qhat_j is within Delta = (m+4) 2^-24 of the exact
// cosine (FP32 rounding of u and zhat, m FMA roundings over non-negative
// terms summing to <= 1).  A reference whose qhat is more than
// band = 2 Delta + 1e-12 below the best qhat has an exact cosine > 1e-12
// below the best reference's; as the vertices e_q are references the best
// cosine is >= 1/sqrt(m), so its exact 1 - c^2 is larger by > 1e-12/sqrt(m),
// far above the FP64 evaluation error (~1e-15): its FP64 distance is
// strictly larger, so it can neither win nor tie.  The FP64 argmin over the
// candidates (ties -> lowest j) equals the argmin over all references.
//
// Pruning.  References are reordered (host, at context creation) into
// spatially compact blocks of 32 by recursive median splits; block b has a
// unit centre c_b and angular radius r_b.  For a point at angle theta from
// c_b every reference of the block has cosine <= cos(max(0, theta - r_b))
// = cos(theta) cos(r_b) + sin(theta) sin(r_b) when theta > r_b (sin(theta)
// computed from the rejection vector u - cos(theta) c_b, which has no
// cancellation).  With its FP32 error below EPS, a block whose bound + EPS
// is below best - band cannot hold a candidate and is skipped.  A warp owns
// one point: it bounds every block, scans the best-bounded block first, then
// the blocks that survive the bound.
//
// FP64 work (GB300 runs FP64 at 1/64 of the FP32 rate) stays off the scan:
// the scan only writes (point, reference) candidate runs; a second kernel
// evaluates each point's candidates in FP64 (one thread per point) and takes
// their argmin.
// A point whose candidate list overflows is rescanned in FP64 over all
// references by a whole CTA (k_assoc_slow), as is every point in debug mode.
// m > 10: no pruning (k_assoc_scan_gen), the same band and FP64 kernels.
#include "kernels.cuh"

namespace {

constexpr int AB = 256;   // threads per CTA (8 warps, one point per warp)
constexpr int LC = 64;    // candidate slots per warp
constexpr float EPS = 1e-5f;

__device__ __forceinline__ double perp_dist(const double* fp, double nf, const double* Zj, double nzj,
                                            int m)
{
    if (nf == 0.0) return 0.0;
    double dot = 0.0;
    for (int q = 0; q < m; ++q) dot = __dadd_rn(dot, __dmul_rn(fp[q], Zj[q]));
    const double den = __dmul_rn(nf, nzj);
    const double cth = __ddiv_rn(dot, den);
    double one_m = __dsub_rn(1.0, __dmul_rn(cth, cth));
    if (one_m < 0.0) one_m = 0.0;
    return __dmul_rn(nf, __dsqrt_rn(one_m));
}

// the same for a run-time m with both rows in memory: sixteen loads of
// each row in flight
__device__ __forceinline__ double perp_dist_mem(const double* fp, double nf, const double* Zj, double nzj,
                                                int m)
{
    if (nf == 0.0) return 0.0;
    double dot = 0.0;
#pragma unroll 16
    for (int q = 0; q < m; ++q) dot = __dadd_rn(dot, __dmul_rn(fp[q], Zj[q]));
    const double den = __dmul_rn(nf, nzj);
    const double cth = __ddiv_rn(dot, den);
    double one_m = __dsub_rn(1.0, __dmul_rn(cth, cth));
    if (one_m < 0.0) one_m = 0.0;
    return __dmul_rn(nf, __dsqrt_rn(one_m));
}

// f' = (f - z*) / a and |f'| in FP64; FP32 unit vector for the scan
// small blocks spread the FP64 work over every SM sub-partition
constexpr int PB = 64;

template <int M>
__global__ void __launch_bounds__(PB) k_assoc_prep(RunView v)
{
    constexpr int M4 = (M + 3) & ~3;
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int s = blockIdx.x * PB + threadIdx.x;
    if (s >= c->nT) return;
    const int i = v.Tlist[s];
    double fp[M];
    double ss = 0.0;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        const double ft = __dsub_rn((double)v.F[(size_t)i * M + q], c->zstar[q]);
        fp[q] = __ddiv_rn(ft, c->a[q]);
        ss = __dadd_rn(ss, __dmul_rn(fp[q], fp[q]));
        v.fprime[(size_t)s * M + q] = fp[q];
    }
    const double nf = __dsqrt_rn(ss);
    v.fnorm[s] = nf;
    const double inv = nf > 0.0 ? 1.0 / nf : 0.0;
#pragma unroll
    for (int q = 0; q < M4; ++q)
        v.uhat[(size_t)s * M4 + q] = q < M ? __double2float_rn(fp[q] * inv) : 0.0f;
}

template <int M>
__global__ void __launch_bounds__(AB) k_assoc_scan(RunView v)
{
    constexpr int M4 = (M + 3) & ~3;
    constexpr int CH = (M4 <= 8) ? 4 : 2;  // blocks whose loads are in flight together
    extern __shared__ __align__(16) float sm[];
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int nT = c->nT;
    const int nb = v.nblk;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    float* cent = sm;                                                     // nb x M4
    float2* crsr = reinterpret_cast<float2*>(cent + (size_t)nb * M4);      // nb
    float* wall = reinterpret_cast<float*>(crsr + nb);                     // 8 x nb bounds
    float* wbnd = wall + (size_t)warp * nb;
    int* lj = reinterpret_cast<int*>(wall + (size_t)8 * nb) + warp * 2 * LC;
    float* lq = reinterpret_cast<float*>(lj + LC);
    for (int e = threadIdx.x; e < nb * M4; e += AB) cent[e] = v.blk_c[e];
    for (int e = threadIdx.x; e < nb; e += AB) crsr[e] = v.blk_r[e];
    __syncthreads();
    const float band = 2.0f * (float)(M + 4) * 5.9604644775390625e-08f + 1e-12f;
    const int w = v.w;

    // the next point's unit vector and |f'| are loaded while this one is
    // scanned
    const int pstride = gridDim.x * 8;
    float un[M];
    double nfn = 0.0;
    {
        const int p0 = blockIdx.x * 8 + warp;
#pragma unroll
        for (int q = 0; q < M; ++q) un[q] = p0 < nT ? v.uhat[(size_t)p0 * M4 + q] : 0.0f;
        if (p0 < nT) nfn = v.fnorm[p0];
    }
    for (int pt = blockIdx.x * 8 + warp; pt < nT; pt += pstride) {
        float u[M];
#pragma unroll
        for (int q = 0; q < M; ++q) u[q] = un[q];
        const double nf = nfn;
        const int pn = pt + pstride;
#pragma unroll
        for (int q = 0; q < M; ++q) un[q] = pn < nT ? v.uhat[(size_t)pn * M4 + q] : 0.0f;
        if (pn < nT) nfn = v.fnorm[pn];
        if (nf == 0.0) {  // every distance is 0: handled by the finalisation
            if (lane == 0) v.arun[pt] = make_int2(0, 0);
            continue;
        }
        // phase 1: cone bound of every block
        float bmax = -4.0f;
        int bb = 0x7fffffff;
        for (int b = lane; b < nb; b += 32) {
            const float* cb = cent + b * M4;
            float ct = 0.0f;
#pragma unroll
            for (int q = 0; q < M; ++q) ct = fmaf(u[q], cb[q], ct);
            float s2 = 0.0f;
#pragma unroll
            for (int q = 0; q < M; ++q) {
                const float r = fmaf(-ct, cb[q], u[q]);
                s2 = fmaf(r, r, s2);
            }
            const float2 cs = crsr[b];
            const float bound = (ct >= cs.x) ? 1.0f : fmaf(ct, cs.x, sqrtf(s2) * cs.y);
            wbnd[b] = bound;
            if (bound > bmax) {
                bmax = bound;
                bb = b;
            }
        }
        // The first scan takes the best-bounded blocks of up to CH lanes (each
        // lane's best, in decreasing order of bound), all loads in flight
        // together, so that `best` is near its final value before the bound
        // filters the rest; the blocks taken are marked scanned (bound -4).
        // Bounds are >= 0 (u, c_b, cos r >= 0): their bits order like
        // unsigned ints.
        int first[CH];
        int nfirst = 0;
        {
            unsigned mine = (bb == 0x7fffffff) ? 0u : __float_as_uint(fmaxf(bmax, 0.0f)) + 1u;  // 0: none
#pragma unroll
            for (int t = 0; t < CH; ++t) {
                const unsigned mx = __reduce_max_sync(0xffffffffu, mine);
                first[t] = -1;
                if (mx == 0u) continue;
                const unsigned cand = (mine == mx) ? (unsigned)bb : 0xffffffffu;
                const int b = (int)__reduce_min_sync(0xffffffffu, cand);
                first[t] = b;
                nfirst = t + 1;
                if (bb == b) mine = 0u;  // this lane's best is taken
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (lane == 0 && first[t] >= 0) wbnd[first[t]] = -4.0f;
        __syncwarp();
        // phase 2: scan the best-bounded block, then every block the bound cannot exclude
        float best = -4.0f;
        int nl = 0;
        bool ovf = false;
        // candidate-list update with one block's cosines (qh, j) per lane
        auto take_block = [&](float qh, int j) {
            // cosines are >= 0, so the float bits order like unsigned ints
            const float wm = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(qh, 0.0f))));
            best = fmaxf(best, wm);
            const bool keep = j >= 0 && qh >= best - band;
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (nl + __popc(bal) > LC) {  // drop entries that fell out of the band
                __syncwarp();
                int kept = 0;
                for (int e0 = 0; e0 < nl; e0 += 32) {
                    const int e = e0 + lane;
                    const bool k2 = e < nl && lq[e] >= best - band;
                    const unsigned b2 = __ballot_sync(0xffffffffu, k2);
                    int jj = 0;
                    float qq = 0.0f;
                    if (k2) {
                        jj = lj[e];
                        qq = lq[e];
                    }
                    __syncwarp();
                    if (k2) {
                        const int p = kept + __popc(b2 & ((1u << lane) - 1u));
                        lj[p] = jj;
                        lq[p] = qq;
                    }
                    kept += __popc(b2);
                    __syncwarp();
                }
                nl = kept;
                if (nl + __popc(bal) > LC) {
                    ovf = true;
                    bal = 0u;
                }
            }
            if (keep && bal) {
                const int p = nl + __popc(bal & ((1u << lane) - 1u));
                lj[p] = j;
                lq[p] = qh;
            }
            nl += __popc(bal);
            __syncwarp();
        };
        // Scans up to CH blocks with all their loads issued before any use
        // (the surviving blocks of a point are scanned in a few latency
        // rounds instead of one round per block).
        int pend[CH];
        int npend = 0;
        auto flush = [&]() {
            float qh[CH];
            int jj[CH];
#pragma unroll
            for (int t = 0; t < CH; ++t) {
                const int pos = (t < npend ? pend[t] : 0) * 32 + lane;
                qh[t] = -4.0f;
                jj[t] = -1;
                if (t < npend && pos < w) {
                    const float4* z4 = reinterpret_cast<const float4*>(v.blk_z + (size_t)pos * M4);
                    float zz[M4];
#pragma unroll
                    for (int q4 = 0; q4 < M4 / 4; ++q4) {
                        const float4 z = __ldg(z4 + q4);
                        zz[4 * q4 + 0] = z.x;
                        zz[4 * q4 + 1] = z.y;
                        zz[4 * q4 + 2] = z.z;
                        zz[4 * q4 + 3] = z.w;
                    }
                    float a = 0.0f;
#pragma unroll
                    for (int q = 0; q < M; ++q) a = fmaf(u[q], zz[q], a);
                    qh[t] = a;
                    jj[t] = __ldg(v.blk_j + pos);
                }
            }
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (t < npend) take_block(qh[t], jj[t]);
            npend = 0;
        };
#pragma unroll
        for (int t = 0; t < CH; ++t) pend[t] = first[t] >= 0 ? first[t] : 0;
        npend = nfirst;
        flush();
        for (int base = 0; base < nb; base += 32) {
            const int b = base + lane;
            const bool f = b < nb && wbnd[b] + EPS >= best - band;
            unsigned msk = __ballot_sync(0xffffffffu, f);
            while (msk) {
                const int b2 = base + __ffs(msk) - 1;
                msk &= msk - 1;
                if (wbnd[b2] + EPS >= best - band) {
#pragma unroll
                    for (int t = 0; t < CH; ++t)
                        if (t == npend) pend[t] = b2;
                    if (++npend == CH) flush();
                }
            }
        }
        if (npend) flush();
        // final candidates: q >= best - band
        int cnt = 0;
        for (int e0 = 0; e0 < nl; e0 += 32) {
            const int e = e0 + lane;
            cnt += __popc(__ballot_sync(0xffffffffu, e < nl && lq[e] >= best - band));
        }
        int start = 0;
        if (lane == 0 && !ovf) start = atomicAdd(&c->ncand, cnt);
        start = __shfl_sync(0xffffffffu, start, 0);
        if (ovf || start + cnt > v.cand_cap) {
            if (lane == 0) {
                v.arun[pt] = make_int2(-1, 0);
                v.slow[atomicAdd(&c->nslow, 1)] = pt;
            }
            __syncwarp();
            continue;
        }
        int off = 0;
        for (int e0 = 0; e0 < nl; e0 += 32) {
            const int e = e0 + lane;
            const bool k2 = e < nl && lq[e] >= best - band;
            const unsigned b2 = __ballot_sync(0xffffffffu, k2);
            if (k2) v.cand[start + off + __popc(b2 & ((1u << lane) - 1u))] = make_int2(pt, lj[e]);
            off += __popc(b2);
        }
        if (lane == 0) v.arun[pt] = make_int2(start, cnt);
        __syncwarp();
    }
}

__device__ __forceinline__ void write_assoc(const RunView& v, Ctrl* c, int i, int j, double d)
{
    v.pi[i] = j;
    v.dist[i] = d;
    if (v.rank2[i] < c->l)
        atomicAdd(&v.rho[j], 1);
    else
        atomicAdd(&v.rhop[j], 1);
}

// per point: FP64 distances of its candidates (usually one to three, so the
// threads of a warp stay nearly converged on the FP64 pipe) and their
// lexicographic (d, j) minimum
constexpr int FB = 128;

template <int M>
__global__ void __launch_bounds__(FB) k_assoc_final(RunView v)
{
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int pt = blockIdx.x * FB + threadIdx.x;
    if (pt >= c->nT) return;
    const int2 run = v.arun[pt];
    if (run.x < 0) return;  // slow path
    double bd = 0.0;
    int bj = 0;
    const double nf = v.fnorm[pt];
    if (nf != 0.0) {
        double fp[M];
#pragma unroll
        for (int q = 0; q < M; ++q) fp[q] = v.fprime[(size_t)pt * M + q];
        bd = CUDART_INF;
        bj = 0x7fffffff;
        for (int e = run.x; e < run.x + run.y; ++e) {
            const int j = v.cand[e].y;
            const double d = perp_dist(fp, nf, v.Zd + (size_t)j * M, v.nz[j], M);
            if (lex_less(d, j, bd, bj)) {
                bd = d;
                bj = j;
            }
        }
    }
    if (v.debug_recheck_all) {
        v.dist[v.Tlist[pt]] = bd;  // compared by k_assoc_slow
        v.pi[v.Tlist[pt]] = bj;
        v.slow[atomicAdd(&c->nslow, 1)] = pt;
        return;
    }
    write_assoc(v, c, v.Tlist[pt], bj, bd);
}

// full FP64 scan of one point per CTA (overflowed lists, debug mode)
// M = 0: runtime m (f' read from memory)
template <int M>
__global__ void __launch_bounds__(AB) k_assoc_slow(RunView v)
{
    __shared__ double sd[AB / 32];
    __shared__ int sj[AB / 32];
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int ns = c->nslow;
    const int m = M > 0 ? M : v.m;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ns; t += gridDim.x) {
        const int pt = v.slow[t];
        double fr[M > 0 ? M : 1];
#pragma unroll
        for (int q = 0; q < M; ++q) fr[q] = v.fprime[(size_t)pt * M + q];
        const double* fp = M > 0 ? fr : v.fprime + (size_t)pt * m;
        const double nf = v.fnorm[pt];
        double d0 = CUDART_INF;
        int j0 = 0x7fffffff;
        for (int j = threadIdx.x; j < v.w; j += AB) {
            const double d = perp_dist(fp, nf, v.Zd + (size_t)j * m, v.nz[j], m);
            if (lex_less(d, j, d0, j0)) {
                d0 = d;
                j0 = j;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double od = __shfl_xor_sync(0xffffffffu, d0, o);
            const int oj = __shfl_xor_sync(0xffffffffu, j0, o);
            if (lex_less(od, oj, d0, j0)) {
                d0 = od;
                j0 = oj;
            }
        }
        if (lane == 0) {
            sd[warp] = d0;
            sj[warp] = j0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < AB / 32; ++q)
                if (lex_less(sd[q], sj[q], d0, j0)) {
                    d0 = sd[q];
                    j0 = sj[q];
                }
            const int i = v.Tlist[pt];
            if (v.arun[pt].x < 0) {
                atomicAdd(&c->overflow, 1);
            } else if (v.debug_recheck_all && (v.pi[i] != j0 || v.dist[i] != d0)) {
                atomicAdd(&c->recheck_miss, 1);
            }
            write_assoc(v, c, i, j0, d0);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// m > NSGA3_FAST_M: runtime m, no pruning (the cone bounds lose their grip in
// many dimensions).  A CTA keeps the unit vectors of GPP points in shared
// memory; each warp forms the FP32 cosines of all of them against its
// tiles of 32 references (a lane per reference, read as float4 through the
// read-only cache) and feeds them to the same candidate band; the FP64
// kernels read f' from memory and keep their pipe full (a thread per point
// or per candidate for the sequential sums).

// f' = (f - z*) / a for every element (a thread per element: the divisions
// spread over every SM), then per point (a thread per point: the FP64 pipe
// serves 32 points per warp instruction) the squares added left to right,
// |f'| and the FP32 unit vector
__global__ void __launch_bounds__(256) k_assoc_prep_elem(RunView v)
{
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int m = v.m;
    const long long e = (long long)blockIdx.x * 256 + threadIdx.x;
    if (e >= (long long)c->nT * m) return;
    const int s = (int)(e / m), q = (int)(e - (long long)s * m);
    const int i = v.Tlist[s];
    v.fprime[e] = __ddiv_rn(__dsub_rn((double)v.F[(size_t)i * m + q], c->zstar[q]), c->a[q]);
}

// one warp per CTA, 32 points: the rows come in through a 32 x 32 tile
// (coalesced loads), lane p adds the squares of point p left to right
__global__ void __launch_bounds__(32) k_assoc_prep_norm(RunView v)
{
    __shared__ double tile[32][33];
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int nT = c->nT, s0 = blockIdx.x * 32, lane = threadIdx.x;
    if (s0 >= nT) return;
    const int m = v.m, M4 = v.M4, np = min(32, nT - s0);
    const double* base = v.fprime + (size_t)s0 * m;
    double ss = 0.0;
    for (int q0 = 0; q0 < m; q0 += 32) {
        const int nq = min(32, m - q0);
#pragma unroll 8
        for (int p = 0; p < np; ++p) tile[p][lane] = lane < nq ? base[(size_t)p * m + q0 + lane] : 0.0;
        __syncwarp();
        if (lane < np)
            for (int t = 0; t < nq; ++t) ss = __dadd_rn(ss, __dmul_rn(tile[lane][t], tile[lane][t]));
        __syncwarp();
    }
    const double nf = __dsqrt_rn(ss);
    if (lane < np) v.fnorm[s0 + lane] = nf;
    const double inv = nf > 0.0 ? 1.0 / nf : 0.0;
    for (int p = 0; p < np; ++p) {
        const double ip = __shfl_sync(0xffffffffu, inv, p);
#pragma unroll 8
        for (int q = lane; q < M4; q += 32)
            v.uhat[(size_t)(s0 + p) * M4 + q] = q < m ? __double2float_rn(base[(size_t)p * m + q] * ip) : 0.0f;
    }
}

constexpr int GW = 8;  // warps per CTA of the m > NSGA3_FAST_M scan

// candidate-list update of one point with a block of 32 cosines (qh, j) per
// lane (j = -1: no reference): keeps every reference within band of the best
// so far; a list that cannot hold them marks the point as overflowed
__device__ __forceinline__ void band_take(float qh, int j, float band, float& best, int& nl, bool& ovf,
                                          int* lj, float* lq, int cap)
{
    const int lane = lane_id();
    const float wm = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(qh, 0.0f))));
    best = fmaxf(best, wm);
    const bool keep = j >= 0 && qh >= best - band;
    unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (nl + __popc(bal) > cap) {  // drop entries that fell out of the band
        __syncwarp();
        int kept = 0;
        for (int e0 = 0; e0 < nl; e0 += 32) {
            const int e = e0 + lane;
            const bool k2 = e < nl && lq[e] >= best - band;
            const unsigned b2 = __ballot_sync(0xffffffffu, k2);
            int jj = 0;
            float qq = 0.0f;
            if (k2) {
                jj = lj[e];
                qq = lq[e];
            }
            __syncwarp();
            if (k2) {
                const int p = kept + __popc(b2 & ((1u << lane) - 1u));
                lj[p] = jj;
                lq[p] = qq;
            }
            kept += __popc(b2);
            __syncwarp();
        }
        nl = kept;
        if (nl + __popc(bal) > cap) {
            ovf = true;
            bal = 0u;
        }
    }
    if (keep && bal) {
        const int p = nl + __popc(bal & ((1u << lane) - 1u));
        lj[p] = j;
        lq[p] = qh;
    }
    nl += __popc(bal);
    __syncwarp();
}

constexpr int GPP = 8;   // points per CTA (every warp works on all of them)
constexpr int LCW = 64;  // candidate slots per warp and point

// dynamic shared memory: the points' unit vectors (GPP x M4) and the lists
size_t scan_gen_smem(int M4) { return (size_t)GPP * M4 * 4 + (size_t)GW * GPP * LCW * 8; }

// The CTA's warps split the references (warp w takes the tiles of 32
// references w, w + GW, ...) and keep a candidate list per point; the lists
// are then merged against the best cosine over all warps.
__global__ void __launch_bounds__(GW * 32) k_assoc_scan_gen(RunView v)
{
    extern __shared__ __align__(16) float sgen[];
    __shared__ float s_best[GW][GPP];
    __shared__ int s_nl[GW][GPP];
    __shared__ int s_ovf[GW][GPP];
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int nT = c->nT, m = v.m, M4 = v.M4, w = v.w;
    const int lane = lane_id(), warp = threadIdx.x >> 5, tid = threadIdx.x;
    float* Us = sgen;                                                // GPP x M4
    int* lists = reinterpret_cast<int*>(sgen + (size_t)GPP * M4);   // GW x GPP x (LCW ints, LCW floats)
    const float band = 2.0f * (float)(m + 4) * 5.9604644775390625e-08f + 1e-12f;
    for (int g0 = blockIdx.x * GPP; g0 < nT; g0 += gridDim.x * GPP) {  // CTA-uniform
        __syncthreads();  // the previous group is merged
        for (int e = tid; e < GPP * M4; e += GW * 32) {
            const int p = e / M4;
            Us[e] = g0 + p < nT ? v.uhat[(size_t)g0 * M4 + e] : 0.0f;
        }
        __syncthreads();
        float best[GPP];
        int nl[GPP];
        bool ovf[GPP], live[GPP];
#pragma unroll
        for (int p = 0; p < GPP; ++p) {
            best[p] = -4.0f;
            nl[p] = 0;
            ovf[p] = false;
            live[p] = g0 + p < nT && v.fnorm[g0 + p] != 0.0;  // |f'| = 0: every distance is 0
        }
        for (int r0 = warp * 32; r0 < w; r0 += GW * 32) {
            const int j = r0 + lane;
            const float4* z4 = reinterpret_cast<const float4*>(v.Zh + (size_t)(j < w ? j : w - 1) * M4);
            float acc[GPP];
#pragma unroll
            for (int p = 0; p < GPP; ++p) acc[p] = 0.0f;
#pragma unroll 8
            for (int k4 = 0; k4 < M4 / 4; ++k4) {
                const float4 z = __ldg(z4 + k4);
#pragma unroll
                for (int p = 0; p < GPP; ++p) {
                    const float4 u = reinterpret_cast<const float4*>(Us + (size_t)p * M4)[k4];
                    acc[p] = fmaf(u.x, z.x, acc[p]);
                    acc[p] = fmaf(u.y, z.y, acc[p]);
                    acc[p] = fmaf(u.z, z.z, acc[p]);
                    acc[p] = fmaf(u.w, z.w, acc[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < GPP; ++p)
                if (live[p]) {
                    int* lj = lists + (size_t)(warp * GPP + p) * 2 * LCW;
                    band_take(acc[p], j < w ? j : -1, band, best[p], nl[p], ovf[p], lj,
                              reinterpret_cast<float*>(lj + LCW), LCW);
                }
        }
        if (lane == 0)
#pragma unroll
            for (int p = 0; p < GPP; ++p) {
                s_best[warp][p] = best[p];
                s_nl[warp][p] = nl[p];
                s_ovf[warp][p] = ovf[p] ? 1 : 0;
            }
        __syncthreads();
        // merge: warp p takes point p
        const int p = warp;
        const int pt = g0 + p;
        if (p >= GPP || pt >= nT) continue;
        if (!live[p]) {
            if (lane == 0) v.arun[pt] = make_int2(0, 0);
            continue;
        }
        float gb = s_best[0][p];
        bool govf = false;
        for (int q = 0; q < GW; ++q) {
            gb = fmaxf(gb, s_best[q][p]);
            govf = govf || s_ovf[q][p];
        }
        int cnt = 0;
        for (int q = 0; q < GW; ++q) {
            const int* lj = lists + (size_t)(q * GPP + p) * 2 * LCW;
            const float* lq = reinterpret_cast<const float*>(lj + LCW);
            const int n = s_nl[q][p];
            for (int e0 = 0; e0 < n; e0 += 32) {
                const int e = e0 + lane;
                cnt += __popc(__ballot_sync(0xffffffffu, e < n && lq[e] >= gb - band));
            }
        }
        int start = 0;
        if (lane == 0 && !govf) start = atomicAdd(&c->ncand, cnt);
        start = __shfl_sync(0xffffffffu, start, 0);
        if (govf || start + cnt > v.cand_cap) {
            if (lane == 0) {
                v.arun[pt] = make_int2(-1, 0);
                v.slow[atomicAdd(&c->nslow, 1)] = pt;
            }
            continue;
        }
        int off = 0;
        for (int q = 0; q < GW; ++q) {
            const int* lj = lists + (size_t)(q * GPP + p) * 2 * LCW;
            const float* lq = reinterpret_cast<const float*>(lj + LCW);
            const int n = s_nl[q][p];
            for (int e0 = 0; e0 < n; e0 += 32) {
                const int e = e0 + lane;
                const bool k2 = e < n && lq[e] >= gb - band;
                const unsigned b2 = __ballot_sync(0xffffffffu, k2);
                if (k2) v.cand[start + off + __popc(b2 & ((1u << lane) - 1u))] = make_int2(pt, lj[e]);
                off += __popc(b2);
            }
        }
        if (lane == 0) v.arun[pt] = make_int2(start, cnt);
    }
}

// a thread per candidate (the FP64 pipe of a warp instruction serves 32
// candidates): its FP64 distance, the same left-to-right evaluation
__global__ void __launch_bounds__(32) k_assoc_cand_dist(RunView v)
{
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int e = blockIdx.x * 32 + threadIdx.x;
    // ncand counts reservations, also those that did not fit (their points
    // went to the slow path): only the first cand_cap slots exist
    if (e >= min(c->ncand, v.cand_cap)) return;
    const int2 pj = v.cand[e];
    const double nf = v.fnorm[pj.x];
    v.cdist[e] = perp_dist_mem(v.fprime + (size_t)pj.x * v.m, nf, v.Zd + (size_t)pj.y * v.m, v.nz[pj.y], v.m);
}

// a thread per point: lexicographic (d, j) minimum over its candidates
__global__ void __launch_bounds__(256) k_assoc_final_gen(RunView v)
{
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int pt = blockIdx.x * 256 + threadIdx.x;
    if (pt >= c->nT) return;
    const int2 run = v.arun[pt];
    if (run.x < 0) return;  // slow path
    double bd = 0.0;
    int bj = 0;
    if (v.fnorm[pt] != 0.0) {
        bd = CUDART_INF;
        bj = 0x7fffffff;
        for (int e = run.x; e < run.x + run.y; ++e) {
            const double d = v.cdist[e];
            const int j = v.cand[e].y;
            if (lex_less(d, j, bd, bj)) {
                bd = d;
                bj = j;
            }
        }
    }
    if (v.debug_recheck_all) {
        v.dist[v.Tlist[pt]] = bd;
        v.pi[v.Tlist[pt]] = bj;
        v.slow[atomicAdd(&c->nslow, 1)] = pt;
        return;
    }
    write_assoc(v, c, v.Tlist[pt], bj, bd);
}

// Few reference directions (w <= ASSOC_SMALL_W, m <= 10): the whole
// association of a point in one thread, every direction's FP32 unit vector
// in shared memory (read by all threads of a warp at once).  f' and |f'| in
// FP64 as k_assoc_prep computes them, the best FP32 cosine over all
// directions, a second pass over the directions within the band of it (the
// candidates), their FP64 distances and the lexicographic (d, j) minimum:
// the same candidates, band and FP64 operations as the pruned path, so the
// same exact result, in one launch instead of four.
constexpr int SB_T = 128;

template <int M>
__global__ void __launch_bounds__(SB_T) k_assoc_small(RunView v)
{
    constexpr int M4 = (M + 3) & ~3;
    extern __shared__ __align__(16) float zs[];  // w x M4 unit directions, original order
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int w = v.w;
    for (int e = threadIdx.x; e < w * M4; e += SB_T) zs[e] = v.Zh[e];
    __syncthreads();
    const int s = blockIdx.x * SB_T + threadIdx.x;
    if (s >= c->nT) return;
    const int i = v.Tlist[s];
    double fp[M];
    double ss = 0.0;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        const double ft = __dsub_rn((double)v.F[(size_t)i * M + q], c->zstar[q]);
        fp[q] = __ddiv_rn(ft, c->a[q]);
        ss = __dadd_rn(ss, __dmul_rn(fp[q], fp[q]));
    }
    const double nf = __dsqrt_rn(ss);
    double bd = 0.0;
    int bj = 0;
    if (nf != 0.0 || v.debug_recheck_all) {
        const double inv = nf > 0.0 ? 1.0 / nf : 0.0;
        float u[M];
#pragma unroll
        for (int q = 0; q < M; ++q) u[q] = __double2float_rn(fp[q] * inv);
        float best = -1.0f;
        for (int j = 0; j < w; ++j) {
            const float* z = zs + j * M4;
            float dq = 0.0f;
#pragma unroll
            for (int q = 0; q < M; ++q) dq = fmaf(u[q], z[q], dq);
            best = fmaxf(best, dq);
        }
        const float band = 2.0f * (float)(M + 4) * 5.9604644775390625e-08f + 1e-12f;
        bd = CUDART_INF;
        bj = 0x7fffffff;
        for (int j = 0; j < w; ++j) {
            const float* z = zs + j * M4;
            float dq = 0.0f;
#pragma unroll
            for (int q = 0; q < M; ++q) dq = fmaf(u[q], z[q], dq);
            if (dq >= best - band) {
                const double d = perp_dist(fp, nf, v.Zd + (size_t)j * M, v.nz[j], M);
                if (lex_less(d, j, bd, bj)) {
                    bd = d;
                    bj = j;
                }
            }
        }
        if (v.debug_recheck_all) {
            // every direction in FP64: the band must not have missed the minimum
            double fd = CUDART_INF;
            int fj = 0x7fffffff;
            for (int j = 0; j < w; ++j) {
                const double d = perp_dist(fp, nf, v.Zd + (size_t)j * M, v.nz[j], M);
                if (lex_less(d, j, fd, fj)) {
                    fd = d;
                    fj = j;
                }
            }
            if (fj != bj || fd != bd) atomicAdd(&c->recheck_miss, 1);
            bd = fd;
            bj = fj;
        }
    }
    write_assoc(v, c, i, bj, bd);
}

// ---------------------------------------------------------------------------
// Tiled scan (m <= 10, more than ASSOC_SMALL_W directions).  Where the cone
// bounds prune little (several objectives: a block's cone and a point's
// distance to its nearest direction are comparable), every cosine is formed,
// at the FP32 FMA rate: a CTA holds TP = TT x TP_P points in registers and
// streams the reference blocks of its range through shared memory (each
// direction read once per CTA by a broadcast load, then TP_P x m FMAs per
// thread).  A work item is (a tile of TP slots, a range of reference
// blocks); the ranges are chosen so that the items fill the grid.  Per
// point and item the scan keeps the largest block maximum (the item's best
// cosine) and up to ASSOC_K blocks whose maximum is within the band of it
// (a block is taken when its maximum is within the band of the best so
// far, replacing a block that has fallen out of the band; none free: the
// point overflows to the FP64 scan).  The block holding the exact argmin
// has a maximum within the band of every later best, so it is never
// replaced.  k_assoc_final_tile takes the best over the items, rescans the
// blocks within the band of it (FP32, then FP64 for the directions within
// the band, as the pruned path does) and writes the association.
constexpr int TT = 128;     // threads per CTA
constexpr int TP_P = 4;     // points per thread
constexpr int TP = TT * TP_P;
constexpr int TCB = 8;      // reference blocks per shared-memory chunk
constexpr int TOCC = 4;     // CTAs per SM (the grid, and the register bound)
constexpr int ASSOC_K = 4;  // entries per point and item

// tiles of T slots, items per tile (splits) and blocks per split: the same
// on the device for both kernels (from nT) and on the host for the maximum.
// The split count minimises the waves of the grid times the blocks an item
// scans, over at most twice the count that fills the grid once (so that
// items <= 2 (grid + ntile)).
__host__ __device__ __forceinline__ void tile_split(int nT, int nb, int grid, int& ntile, int& S, int& bps)
{
    ntile = (nT + TP - 1) / TP;
    S = 1;
    bps = nb;
    if (ntile == 0 || nb == 0) return;
    const int fill = (grid + ntile - 1) / ntile;
    const int smax = min(nb, 2 * fill);
    long long best = -1;
    for (int t = 1; t <= smax; ++t) {
        const int b = (nb + t - 1) / t;
        const int st = (nb + b - 1) / b;
        const long long cost = (long long)(((long long)ntile * st + grid - 1) / grid) * b;
        if (best < 0 || cost < best) {
            best = cost;
            S = st;
            bps = b;
        }
    }
}

// Two points' cosines with one direction in one instruction: FP32 pairs
// (fma.rn.f32x2 rounds each lane once, as fmaf does), the points' unit
// vectors packed by pairs, each direction component duplicated in shared
// memory.  Packing and unpacking are register moves.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_unpack(unsigned long long x, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x));
}

__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ float fmax3f(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

template <int M>
__global__ void __launch_bounds__(TT, TOCC) k_assoc_tile(RunView v)
{
    static_assert(TP_P % 2 == 0, "points are packed by pairs");
    constexpr int M4 = (M + 3) & ~3;
    constexpr int ZQ = (M + 1) / 2;  // 16-byte words per staged direction: (z0, z0, z1, z1), ...
    constexpr int PP = TP_P / 2;
    __shared__ ulonglong2 zs[TCB * 32 * ZQ];
    __shared__ float slm[TP_P][ASSOC_K][TT];  // candidate blocks of each point: maximum, block
    __shared__ int slk[TP_P][ASSOC_K][TT];
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int nT = c->nT;
    const int nb = v.nblk, w = v.w;
    int ntile, S, bps;
    tile_split(nT, nb, gridDim.x, ntile, S, bps);
    const int items = ntile * S;
    const float band = 2.0f * (float)(M + 4) * 5.9604644775390625e-08f + 1e-12f;
    const int tid = threadIdx.x;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int tile = it / S, sp = it - (it / S) * S;
        const int b0 = sp * bps;
        const int b1 = min(nb, b0 + bps);
        unsigned long long u2[PP][M];
#pragma unroll
        for (int pp = 0; pp < PP; ++pp) {
            const int sa = tile * TP + (2 * pp) * TT + tid;
            const int sb = sa + TT;
            const float* ra = v.uhat + (size_t)sa * M4;
            const float* rb = v.uhat + (size_t)sb * M4;
#pragma unroll
            for (int t = 0; t < M; ++t)
                u2[pp][t] = f2_pack(sa < nT ? ra[t] : 0.0f, sb < nT ? rb[t] : 0.0f);
        }
        float lbest[TP_P];
        unsigned ovf = 0u;
#pragma unroll
        for (int k = 0; k < TP_P; ++k) {
            lbest[k] = -4.0f;
#pragma unroll
            for (int e = 0; e < ASSOC_K; ++e) {
                slm[k][e][tid] = -4.0f;
                slk[k][e][tid] = -1;
            }
        }
        for (int cb = b0; cb < b1; cb += TCB) {
            const int nbk = min(TCB, b1 - cb);
            __syncthreads();  // the previous chunk is consumed
            // padding directions (position >= w) get -1 components: their
            // cosine with a unit vector of non-negative components is <= -1
            for (int e = tid; e < nbk * 32 * ZQ; e += TT) {
                const int r = e / ZQ, q2 = e - r * ZQ;
                const int pos = cb * 32 + r;
                float2 a = make_float2(-1.0f, -1.0f);
                if (pos < w) a = __ldg(reinterpret_cast<const float2*>(v.blk_z + (size_t)pos * M4) + q2);
                zs[e] = make_ulonglong2(f2_pack(a.x, a.x), f2_pack(a.y, a.y));
            }
            __syncthreads();
            for (int bb = 0; bb < nbk; ++bb) {
                float bm[TP_P];
#pragma unroll
                for (int k = 0; k < TP_P; ++k) bm[k] = -4.0f;
                const ulonglong2* zb = zs + bb * 32 * ZQ;
#pragma unroll 2
                for (int r = 0; r < 32; r += 2) {
                    ulonglong2 za[ZQ], zc[ZQ];
#pragma unroll
                    for (int q2 = 0; q2 < ZQ; ++q2) {
                        za[q2] = zb[r * ZQ + q2];
                        zc[q2] = zb[(r + 1) * ZQ + q2];
                    }
#pragma unroll
                    for (int pp = 0; pp < PP; ++pp) {
                        unsigned long long qa = 0ull, qc = 0ull;
#pragma unroll
                        for (int t = 0; t < M; ++t) {
                            qa = f2_fma(u2[pp][t], (t & 1) ? za[t >> 1].y : za[t >> 1].x, qa);
                            qc = f2_fma(u2[pp][t], (t & 1) ? zc[t >> 1].y : zc[t >> 1].x, qc);
                        }
                        float a0, a1, c0, c1;
                        f2_unpack(qa, a0, a1);
                        f2_unpack(qc, c0, c1);
                        bm[2 * pp] = fmax3f(bm[2 * pp], a0, c0);
                        bm[2 * pp + 1] = fmax3f(bm[2 * pp + 1], a1, c1);
                    }
                }
#pragma unroll
                for (int k = 0; k < TP_P; ++k) {
                    if (bm[k] >= lbest[k] - band) {
                        const float thr = fmaxf(lbest[k], bm[k]) - band;
                        int slot = -1;
#pragma unroll
                        for (int e = 0; e < ASSOC_K; ++e)
                            if (slot < 0 && (slk[k][e][tid] < 0 || slm[k][e][tid] < thr)) slot = e;
                        if (slot < 0) {
                            ovf |= 1u << k;
                        } else {
                            slm[k][slot][tid] = bm[k];
                            slk[k][slot][tid] = cb + bb;
                        }
                    }
                    lbest[k] = fmaxf(lbest[k], bm[k]);
                }
            }
        }
        // point k of this thread is T slot tile * TP + k * TT + tid (pairs:
        // points 2 pp and 2 pp + 1 are TT slots apart)
#pragma unroll
        for (int k = 0; k < TP_P; ++k) {
            const int l = k * TT + tid;
            if (tile * TP + l >= nT) continue;
            int4* dst = reinterpret_cast<int4*>(v.aent + ((size_t)it * TP + l) * ASSOC_K);
            if ((ovf >> k) & 1u) {
                dst[0] = make_int4(0, -2, 0, -2);
                dst[1] = make_int4(0, -2, 0, -2);
            } else {
                dst[0] = make_int4(__float_as_int(slm[k][0][tid]), slk[k][0][tid],
                                   __float_as_int(slm[k][1][tid]), slk[k][1][tid]);
                dst[1] = make_int4(__float_as_int(slm[k][2][tid]), slk[k][2][tid],
                                   __float_as_int(slm[k][3][tid]), slk[k][3][tid]);
            }
        }
    }
}

static_assert(ASSOC_K == 4, "the entries of a point are written as two int4");

// per point (a thread per T slot): the best cosine over the items, the
// blocks within the band of it rescanned in FP32, the FP64 distances of
// their directions within the band and the lexicographic (d, j) minimum.
// The blocks and then the candidate directions of each thread are listed
// first (shared memory, a column per thread), so that a warp runs as many
// rescans and FP64 evaluations as its busiest thread needs rather than the
// union of its threads' positions.  A point with more than FT_BLK blocks or
// FT_CAND candidates takes the FP64 scan over all directions.
constexpr int FT_BLK = 8;
constexpr int FT_CAND = 16;

template <int M>
__global__ void __launch_bounds__(FB) k_assoc_final_tile(RunView v)
{
    constexpr int M4 = (M + 3) & ~3;
    constexpr int Q4 = M4 / 4;
    // a block's directions in groups of RC, every load of a group in flight
    // together (a thread's blocks are its own: the loads do not coalesce,
    // so round trips, not bytes, set the time)
    constexpr int RC = M4 <= 8 ? 8 : 4;
    __shared__ int sblk[FT_BLK][FB];
    __shared__ int scand[FT_CAND][FB];
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int nT = c->nT;
    const int tid = threadIdx.x;
    const int s = blockIdx.x * FB + tid;
    if (s >= nT) return;
    int ntile, S, bps;
    tile_split(nT, v.nblk, v.assoc_grid, ntile, S, bps);
    const int tile = s / TP, l = s - tile * TP;
    const double nf = v.fnorm[s];
    double bd = 0.0;
    int bj = 0;
    if (nf != 0.0) {
        const float band = 2.0f * (float)(M + 4) * 5.9604644775390625e-08f + 1e-12f;
        float gbest = -4.0f;
        bool ovf = false;
        for (int sp = 0; sp < S; ++sp) {
            const int4* e = reinterpret_cast<const int4*>(v.aent + ((size_t)(tile * S + sp) * TP + l) * ASSOC_K);
            const int4 x0 = e[0], x1 = e[1];
            const int bk[4] = {x0.y, x0.w, x1.y, x1.w};
            const int bv[4] = {x0.x, x0.z, x1.x, x1.z};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (bk[k] == -2) ovf = true;
                if (bk[k] >= 0) gbest = fmaxf(gbest, __int_as_float(bv[k]));
            }
        }
        const float thr = gbest - band;
        int nblk = 0;
        for (int sp = 0; sp < S && !ovf; ++sp) {
            const int4* e = reinterpret_cast<const int4*>(v.aent + ((size_t)(tile * S + sp) * TP + l) * ASSOC_K);
            const int4 x0 = e[0], x1 = e[1];
            const int bk[4] = {x0.y, x0.w, x1.y, x1.w};
            const int bv[4] = {x0.x, x0.z, x1.x, x1.z};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (bk[k] < 0 || __int_as_float(bv[k]) < thr) continue;
                if (nblk == FT_BLK) {
                    ovf = true;
                } else {
                    sblk[nblk][tid] = bk[k];
                    ++nblk;
                }
            }
        }
        float u[M];
#pragma unroll
        for (int q = 0; q < M; ++q) u[q] = v.uhat[(size_t)s * M4 + q];
        int ncand = 0;
        const float4* bz4 = reinterpret_cast<const float4*>(v.blk_z);
        for (int i = 0; i < nblk && !ovf; ++i) {
            const int base = sblk[i][tid] * 32;
            for (int r0 = 0; r0 < 32; r0 += RC) {
                float qv[RC];
#pragma unroll
                for (int t = 0; t < RC; ++t) {
                    const int pos = min(base + r0 + t, v.w - 1);
                    float z[M4];
#pragma unroll
                    for (int q4 = 0; q4 < Q4; ++q4) {
                        const float4 a = __ldg(bz4 + (size_t)pos * Q4 + q4);
                        z[4 * q4 + 0] = a.x;
                        z[4 * q4 + 1] = a.y;
                        z[4 * q4 + 2] = a.z;
                        z[4 * q4 + 3] = a.w;
                    }
                    float q = 0.0f;
#pragma unroll
                    for (int t2 = 0; t2 < M; ++t2) q = fmaf(u[t2], z[t2], q);
                    qv[t] = q;
                }
#pragma unroll
                for (int t = 0; t < RC; ++t) {
                    const int pos = base + r0 + t;
                    if (pos >= v.w || qv[t] < thr) continue;
                    if (ncand == FT_CAND) {
                        ovf = true;
                    } else {
                        scand[ncand][tid] = pos;
                        ++ncand;
                    }
                }
            }
        }
        if (ovf) {
            v.arun[s] = make_int2(-1, 0);
            v.slow[atomicAdd(&c->nslow, 1)] = s;
            return;
        }
        double fp[M];
#pragma unroll
        for (int q = 0; q < M; ++q) fp[q] = v.fprime[(size_t)s * M + q];
        bd = CUDART_INF;
        bj = 0x7fffffff;
        for (int i = 0; i < ncand; ++i) {
            const int j = v.blk_j[scand[i][tid]];
            const double d = perp_dist(fp, nf, v.Zd + (size_t)j * M, v.nz[j], M);
            if (lex_less(d, j, bd, bj)) {
                bd = d;
                bj = j;
            }
        }
    }
    if (v.debug_recheck_all) {
        v.dist[v.Tlist[s]] = bd;  // compared by k_assoc_slow
        v.pi[v.Tlist[s]] = bj;
        v.arun[s] = make_int2(0, 0);
        v.slow[atomicAdd(&c->nslow, 1)] = s;
        return;
    }
    write_assoc(v, c, v.Tlist[s], bj, bd);
}

size_t small_smem(const RunView& v) { return (size_t)v.w * v.M4 * sizeof(float); }

size_t scan_smem(const RunView& v) { return (size_t)v.nblk * (v.M4 + 2 + 8) * 4 + 8 * 2 * LC * 4; }

template <int M>
cudaError_t launch_m(const RunView& v, cudaStream_t s, int num_sms)
{
    if (assoc_small(v)) {
        k_assoc_small<M><<<(v.n2 + SB_T - 1) / SB_T, SB_T, small_smem(v), s>>>(v);
        return cudaGetLastError();
    }
    if (v.aent) {
        k_assoc_tile<M><<<v.assoc_grid, TT, 0, s>>>(v);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_assoc_final_tile<M><<<(v.n2 + FB - 1) / FB, FB, 0, s>>>(v);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_assoc_slow<M><<<num_sms, AB, 0, s>>>(v);
        return cudaGetLastError();
    }
    const size_t sm = scan_smem(v);
    int blocks = (v.n2 + 7) / 8;
    if (blocks > num_sms * 8) blocks = num_sms * 8;
    k_assoc_scan<M><<<blocks, AB, sm, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_assoc_final<M><<<(v.n2 + FB - 1) / FB, FB, 0, s>>>(v);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_assoc_slow<M><<<num_sms, AB, 0, s>>>(v);
    return cudaGetLastError();
}

template <int M>
cudaError_t attr_m(size_t sm)
{
    return cudaFuncSetAttribute(k_assoc_scan<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

}  // namespace

int assoc_tile_grid(int num_sms) { return (num_sms > 0 ? num_sms : 1) * TOCC; }

size_t assoc_tile_entries(int n2, int num_sms)
{
    // items = ntile x S <= ntile x 2 ceil(grid / ntile) <= 2 (grid + ntile)
    // for every nT <= n2
    const size_t ntile = ((size_t)n2 + TP - 1) / TP;
    return 2 * ((size_t)assoc_tile_grid(num_sms) + ntile) * TP * ASSOC_K;
}

cudaError_t launch_assoc_prep(const RunView& v, cudaStream_t s)
{
    if (assoc_small(v)) return cudaSuccess;  // k_assoc_small forms f' itself
    const int g = (v.n2 + PB - 1) / PB;
    switch (v.m) {
    case 2: k_assoc_prep<2><<<g, PB, 0, s>>>(v); break;
    case 3: k_assoc_prep<3><<<g, PB, 0, s>>>(v); break;
    case 4: k_assoc_prep<4><<<g, PB, 0, s>>>(v); break;
    case 5: k_assoc_prep<5><<<g, PB, 0, s>>>(v); break;
    case 6: k_assoc_prep<6><<<g, PB, 0, s>>>(v); break;
    case 7: k_assoc_prep<7><<<g, PB, 0, s>>>(v); break;
    case 8: k_assoc_prep<8><<<g, PB, 0, s>>>(v); break;
    case 9: k_assoc_prep<9><<<g, PB, 0, s>>>(v); break;
    case 10: k_assoc_prep<10><<<g, PB, 0, s>>>(v); break;
    default:
        if (v.m < 2 || v.m > NSGA3_MAX_M) return cudaErrorInvalidValue;
    {
        k_assoc_prep_elem<<<(unsigned)(((long long)v.n2 * v.m + 255) / 256), 256, 0, s>>>(v);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_assoc_prep_norm<<<(v.n2 + 31) / 32, 32, 0, s>>>(v);
        break;
    }
    }
    return cudaGetLastError();
}

cudaError_t launch_assoc_scan(const RunView& v, int num_sms, cudaStream_t s)
{
    switch (v.m) {
    case 2: return launch_m<2>(v, s, num_sms);
    case 3: return launch_m<3>(v, s, num_sms);
    case 4: return launch_m<4>(v, s, num_sms);
    case 5: return launch_m<5>(v, s, num_sms);
    case 6: return launch_m<6>(v, s, num_sms);
    case 7: return launch_m<7>(v, s, num_sms);
    case 8: return launch_m<8>(v, s, num_sms);
    case 9: return launch_m<9>(v, s, num_sms);
    case 10: return launch_m<10>(v, s, num_sms);
    default: break;
    }
    if (v.m < 2 || v.m > NSGA3_MAX_M) return cudaErrorInvalidValue;
    int blocks = (v.n2 + GPP - 1) / GPP;
    if (blocks > num_sms * 8) blocks = num_sms * 8;
    k_assoc_scan_gen<<<blocks, GW * 32, scan_gen_smem(v.M4), s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one warp per CTA: the few candidates of a selection spread over every SM
    k_assoc_cand_dist<<<(v.cand_cap + 31) / 32, 32, 0, s>>>(v);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_assoc_final_gen<<<(v.n2 + 255) / 256, 256, 0, s>>>(v);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_assoc_slow<0><<<num_sms, AB, 0, s>>>(v);
    return cudaGetLastError();
}

// The scan's shared-memory opt-in is set once per process, at its maximum,
// before any launch (changing a kernel's attribute while graphs that launch
// it run on other streams is avoided); a run only checks that its block
// tables fit (about 5,000 blocks of 32 references).
constexpr size_t SCAN_SMEM_MAX = 220 * 1024;

cudaError_t assoc_prepare(const RunView& v)
{
    if (v.m < 2 || v.m > NSGA3_MAX_M) return cudaErrorInvalidValue;
    if (v.m > NSGA3_FAST_M) return cudaSuccess;  // the generic scan keeps no block tables
    return scan_smem(v) <= SCAN_SMEM_MAX ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t assoc_init_attributes()
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = attr_m<2>(SCAN_SMEM_MAX);
    if (e == cudaSuccess) e = attr_m<3>(SCAN_SMEM_MAX);
    if (e == cudaSuccess) e = attr_m<4>(SCAN_SMEM_MAX);
    if (e == cudaSuccess) e = attr_m<5>(SCAN_SMEM_MAX);
    if (e == cudaSuccess) e = attr_m<6>(SCAN_SMEM_MAX);
    if (e == cudaSuccess) e = attr_m<7>(SCAN_SMEM_MAX);
    if (e == cudaSuccess) e = attr_m<8>(SCAN_SMEM_MAX);
    if (e == cudaSuccess) e = attr_m<9>(SCAN_SMEM_MAX);
    if (e == cudaSuccess) e = attr_m<10>(SCAN_SMEM_MAX);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_assoc_scan_gen, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)scan_gen_smem(NSGA3_MAX_M));
    return e;
}
