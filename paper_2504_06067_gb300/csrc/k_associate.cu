// k_associate.cu -- association of S u F_l with the reference directions
// (Alg. 2 lines 2-4, Eq. 2 read as the perpendicular distance
// D_ij = |f'| sqrt(1 - cos^2), pi_i = argmin_j D_ij, d_i = min_j D_ij) and
// the niche counts rho (over S) and rho' (over F_l) of Alg. 2 lines 5-6.
//
// Exactness: the FP64 distance of the oracle is reproduced operation for
// operation (_rn intrinsics, left-to-right sums) but only for candidate
// references.  Candidates come from an FP32 scan of cosines
// qhat_j = u . zhat_j with unit vectors u = f'/|f'|, zhat_j = z_j/|z_j|
// (components >= 0).  Each qhat_j is within Delta = (m+4) 2^-24 of the
// exact cosine (FP32 rounding of u and zhat plus m FMA roundings over
// non-negative terms of sum <= 1).  A reference whose qhat is more than
// 2 Delta + 1e-12 below the best qhat therefore has an exact cosine at least
// 1e-12 below the best reference's; since the vertices e_q are references,
// the best cosine is >= 1/sqrt(m), so its exact 1 - c^2 is larger by
// > 1e-12/sqrt(m) -- far above the FP64 evaluation error (~1e-15) -- and its
// FP64 distance is strictly larger: it can neither win nor tie.  The FP64
// argmin over the candidates (ties -> lowest j) thus equals the argmin over
// all j.  A point whose per-lane candidate list overflows is rescanned in
// FP64 over all references by its whole CTA.
#include "kernels.cuh"

namespace {

constexpr int AB = 256;      // threads per CTA (8 warps)
constexpr int RT = 256;      // references per shared-memory tile
constexpr int NCAND = 4;     // candidate slots per lane

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

// f' = (f - z*) / a and |f'| in FP64; FP32 unit vector for the scan
__global__ void __launch_bounds__(AB) k_assoc_prep(RunView v)
{
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int s = blockIdx.x * AB + threadIdx.x;
    if (s >= c->nT) return;
    const int m = v.m, i = v.Tlist[s];
    double fp[NSGA3_MAX_M];
    double ss = 0.0;
    for (int q = 0; q < m; ++q) {
        const double ft = __dsub_rn((double)v.F[(size_t)i * m + q], c->zstar[q]);
        fp[q] = __ddiv_rn(ft, c->a[q]);
        ss = __dadd_rn(ss, __dmul_rn(fp[q], fp[q]));
        v.fprime[(size_t)s * m + q] = fp[q];
    }
    const double nf = __dsqrt_rn(ss);
    v.fnorm[s] = nf;
    for (int q = 0; q < v.M4; ++q)
        v.uhat[(size_t)s * v.M4 + q] = (q < m && nf > 0.0) ? __double2float_rn(__ddiv_rn(fp[q], nf)) : 0.0f;
}

template <int M>
__global__ void __launch_bounds__(AB) k_assoc_scan(RunView v)
{
    constexpr int M4 = (M + 3) & ~3;
    __shared__ __align__(16) float zt[RT * M4];
    __shared__ float s_best[8][32];
    __shared__ double s_d[8][32];
    __shared__ int s_j[8][32];
    __shared__ int s_ovf[32];
    __shared__ double s_fd[32];
    __shared__ int s_fj[32];
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int nT = c->nT;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int s0 = blockIdx.x * 32;
    if (s0 >= nT) return;
    const int slot = s0 + lane;
    const bool live = slot < nT;
    const float band = 2.0f * (float)(M + 4) * 5.9604644775390625e-08f + 1e-12f;

    float u[M4];
#pragma unroll
    for (int q = 0; q < M4; ++q) u[q] = live ? v.uhat[(size_t)slot * M4 + q] : 0.0f;

    float best = -2.0f;
    int cj[NCAND];
    float cq[NCAND];
#pragma unroll
    for (int t = 0; t < NCAND; ++t) {
        cj[t] = -1;
        cq[t] = -2.0f;
    }
    int ovf = 0;
    const int w = v.w;
    for (int tb = 0; tb < w; tb += RT) {
        const int nt = min(RT, w - tb);
        __syncthreads();
        const float4* src = reinterpret_cast<const float4*>(v.Zh + (size_t)tb * M4);
        float4* dst = reinterpret_cast<float4*>(zt);
        for (int e = threadIdx.x; e < nt * M4 / 4; e += AB) dst[e] = src[e];
        __syncthreads();
        for (int r = warp; r < nt; r += 8) {
            const float4* z4 = reinterpret_cast<const float4*>(zt + r * M4);
            float qh = 0.0f;
#pragma unroll
            for (int q4 = 0; q4 < M4 / 4; ++q4) {
                float4 z = z4[q4];
                qh = fmaf(u[4 * q4 + 0], z.x, qh);
                qh = fmaf(u[4 * q4 + 1], z.y, qh);
                qh = fmaf(u[4 * q4 + 2], z.z, qh);
                qh = fmaf(u[4 * q4 + 3], z.w, qh);
            }
            if (qh >= best - band) {
                const int j = tb + r;
                if (qh > best + band) {
#pragma unroll
                    for (int t = 0; t < NCAND; ++t) cj[t] = -1;
                }
                if (qh > best) best = qh;
                // place into a free or stale slot
                bool placed = false;
#pragma unroll
                for (int t = 0; t < NCAND; ++t) {
                    if (!placed && (cj[t] < 0 || cq[t] < best - band)) {
                        cj[t] = j;
                        cq[t] = qh;
                        placed = true;
                    }
                }
                if (!placed) ovf = 1;
            }
        }
    }
    // merge the 8 warps' maxima per point
    s_best[warp][lane] = best;
    if (warp == 0) s_ovf[lane] = 0;
    __syncthreads();
    if (ovf) atomicOr(&s_ovf[lane], 1);
    float B = s_best[0][lane];
#pragma unroll
    for (int t = 1; t < 8; ++t) B = fmaxf(B, s_best[t][lane]);
    // FP64 recheck of this lane's surviving candidates
    double fp[M];
    double nf = 0.0;
    if (live) {
#pragma unroll
        for (int q = 0; q < M; ++q) fp[q] = v.fprime[(size_t)slot * M + q];
        nf = v.fnorm[slot];
    }
    double bd = CUDART_INF;
    int bj = 0x7fffffff;
#pragma unroll
    for (int t = 0; t < NCAND; ++t) {
        if (live && cj[t] >= 0 && cq[t] >= B - band) {
            const int j = cj[t];
            double d = perp_dist(fp, nf, v.Zd + (size_t)j * M, v.nz[j], M);
            if (lex_less(d, j, bd, bj)) {
                bd = d;
                bj = j;
            }
        }
    }
    s_d[warp][lane] = bd;
    s_j[warp][lane] = bj;
    __syncthreads();
    if (warp == 0) {
        double fd = s_d[0][lane];
        int fj = s_j[0][lane];
        for (int t = 1; t < 8; ++t)
            if (lex_less(s_d[t][lane], s_j[t][lane], fd, fj)) {
                fd = s_d[t][lane];
                fj = s_j[t][lane];
            }
        if (live && nf == 0.0) {  // |f'| = 0: every distance is 0, the first reference wins
            fd = 0.0;
            fj = 0;
        }
        s_fd[lane] = fd;
        s_fj[lane] = fj;
    }
    __syncthreads();
    // overflowed lists (and every point in debug mode): full FP64 scan by the whole CTA
    const unsigned need =
        __ballot_sync(0xffffffffu, live && nf != 0.0 && (s_ovf[lane] || v.debug_recheck_all));
    unsigned todo = need;
    while (todo) {
        const int p = __ffs(todo) - 1;
        todo &= todo - 1;
        const int sp = s0 + p;
        double fpp[M];
#pragma unroll
        for (int q = 0; q < M; ++q) fpp[q] = v.fprime[(size_t)sp * M + q];
        const double nfp = v.fnorm[sp];
        double d0 = CUDART_INF;
        int j0 = 0x7fffffff;
        for (int j = threadIdx.x; j < w; j += AB) {
            double d = perp_dist(fpp, nfp, v.Zd + (size_t)j * M, v.nz[j], M);
            if (lex_less(d, j, d0, j0)) {
                d0 = d;
                j0 = j;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double od = __shfl_xor_sync(0xffffffffu, d0, o);
            int oj = __shfl_xor_sync(0xffffffffu, j0, o);
            if (lex_less(od, oj, d0, j0)) {
                d0 = od;
                j0 = oj;
            }
        }
        if (lane == 0) {
            s_d[warp][p] = d0;
            s_j[warp][p] = j0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double fd = s_d[0][p];
            int fj = s_j[0][p];
            for (int t = 1; t < 8; ++t)
                if (lex_less(s_d[t][p], s_j[t][p], fd, fj)) {
                    fd = s_d[t][p];
                    fj = s_j[t][p];
                }
            if (s_ovf[p]) {
                atomicAdd(&c->overflow, 1);
            } else if (fd != s_fd[p] || fj != s_fj[p]) {
                atomicAdd(&c->recheck_miss, 1);  // debug mode: the filter lost the argmin
            }
            s_fd[p] = fd;
            s_fj[p] = fj;
        }
        __syncthreads();
    }
    if (warp == 0 && live) {
        const int i = v.Tlist[slot];
        const int fj = s_fj[lane];
        v.pi[i] = fj;
        v.dist[i] = s_fd[lane];
        if (v.rank2[i] < c->l)
            atomicAdd(&v.rho[fj], 1);
        else
            atomicAdd(&v.rhop[fj], 1);
    }
}

template <int M>
cudaError_t launch_scan_m(const RunView& v, cudaStream_t s)
{
    k_assoc_scan<M><<<(v.n2 + 31) / 32, AB, 0, s>>>(v);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_assoc_prep(const RunView& v, cudaStream_t s)
{
    k_assoc_prep<<<(v.n2 + AB - 1) / AB, AB, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_assoc_scan(const RunView& v, cudaStream_t s)
{
    switch (v.m) {
    case 2: return launch_scan_m<2>(v, s);
    case 3: return launch_scan_m<3>(v, s);
    case 4: return launch_scan_m<4>(v, s);
    case 5: return launch_scan_m<5>(v, s);
    case 6: return launch_scan_m<6>(v, s);
    case 7: return launch_scan_m<7>(v, s);
    case 8: return launch_scan_m<8>(v, s);
    case 9: return launch_scan_m<9>(v, s);
    case 10: return launch_scan_m<10>(v, s);
    default: return cudaErrorInvalidValue;
    }
}
