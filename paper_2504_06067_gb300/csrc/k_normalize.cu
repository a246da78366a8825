// k_normalize.cu -- "Normalize" of Alg. 1 line 5 / Alg. 2 line 1, read as
// the NSGA-III normalization of Deb & Jain (the paper gives no formula):
//   T = S u F_l;  z*_q = min_T f_q;  f~ = f - z*;
//   e_q = argmin_T max_r f~_r / w_qr  (w_qr = 1 if r == q else 1e-6, ties ->
//         lowest index);  E b = 1 by Gaussian elimination with partial
//         pivoting;  a_q = 1 / b_q;  nadir fallback a_q = max_T f~_q
//         (1 where 0) when a pivot is 0 or an a_q is not finite or <= 1e-6.
// All FP64 operations use the _rn intrinsics, so no FMA contraction occurs
// and every value is the IEEE result of the same operation sequence a
// plain CPU evaluation performs.
// The ASF maximum uses that x -> fl(x / 1e-6) is monotone:
// max_{r != q} fl(f~_r / 1e-6) == fl(max_{r != q} f~_r / 1e-6), so each
// member needs two divisions instead of m * m.
#include "kernels.cuh"

namespace {

constexpr int NB = 256;

// members of T are appended to Tlist; ideal point by order-preserving atomicMin
__global__ void __launch_bounds__(NB) k_norm_ideal(RunView v)
{
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int l = c->l;
    const int i = blockIdx.x * NB + threadIdx.x;
    const int lane = lane_id();
    bool inT = false;
    if (i < v.n2) {
        int r = v.rank2[i];
        inT = r >= 0 && r <= l;
    }
    unsigned bal = __ballot_sync(0xffffffffu, inT);
    int base = 0;
    if (lane == 0 && bal) base = atomicAdd(&c->nT, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (inT) v.Tlist[base + __popc(bal & ((1u << lane) - 1u))] = i;
    for (int q = 0; q < v.m; ++q) {
        uint32_t o = inT ? f2ord(v.F[(size_t)i * v.m + q]) : 0xffffffffu;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) o = min(o, __shfl_xor_sync(0xffffffffu, o, s));
        if (lane == 0 && o != 0xffffffffu) atomicMin(&c->zmin[q], o);
    }
}

__device__ __forceinline__ double zstar_of(const Ctrl* c, int q)
{
    // -0.0 and +0.0 are the same minimum: adding +0.0 keeps +0.0
    return __dadd_rn((double)ord2f(c->zmin[q]), 0.0);
}

// per-block (min ASF, lowest index) per axis and per-block max of f~
__global__ void __launch_bounds__(NB) k_norm_extreme(RunView v)
{
    __shared__ double s_asf[NB / 32][NSGA3_MAX_M];
    __shared__ int s_idx[NB / 32][NSGA3_MAX_M];
    __shared__ double s_nad[NB / 32][NSGA3_MAX_M];
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int m = v.m, nT = c->nT;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    double zs[NSGA3_MAX_M];
    for (int q = 0; q < m; ++q) zs[q] = zstar_of(c, q);
    double best[NSGA3_MAX_M], nad[NSGA3_MAX_M];
    int bidx[NSGA3_MAX_M];
    for (int q = 0; q < m; ++q) {
        best[q] = CUDART_INF;
        bidx[q] = 0x7fffffff;
        nad[q] = 0.0;
    }
    for (int s = blockIdx.x * NB + threadIdx.x; s < nT; s += gridDim.x * NB) {
        const int i = v.Tlist[s];
        double ft[NSGA3_MAX_M];
        double mx1 = -CUDART_INF, mx2 = -CUDART_INF;
        int r1 = -1;
        for (int r = 0; r < m; ++r) {
            ft[r] = __dsub_rn((double)v.F[(size_t)i * m + r], zs[r]);
            if (ft[r] > mx1) {
                mx2 = mx1;
                mx1 = ft[r];
                r1 = r;
            } else if (ft[r] > mx2) {
                mx2 = ft[r];
            }
            nad[r] = fmax(nad[r], ft[r]);
        }
        const double d1 = __ddiv_rn(mx1, 1e-6), d2 = __ddiv_rn(mx2, 1e-6);
        for (int q = 0; q < m; ++q) {
            double other = (q == r1) ? d2 : d1;
            double asf = ft[q] > other ? ft[q] : other;
            if (lex_less(asf, i, best[q], bidx[q])) {
                best[q] = asf;
                bidx[q] = i;
            }
        }
    }
    for (int q = 0; q < m; ++q) {
        double b = best[q], n = nad[q];
        int bi = bidx[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, b, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            double on = __shfl_xor_sync(0xffffffffu, n, o);
            if (lex_less(ob, oi, b, bi)) {
                b = ob;
                bi = oi;
            }
            n = fmax(n, on);
        }
        if (lane == 0) {
            s_asf[warp][q] = b;
            s_idx[warp][q] = bi;
            s_nad[warp][q] = n;
        }
    }
    __syncthreads();
    if (threadIdx.x < m) {
        const int q = threadIdx.x;
        double b = s_asf[0][q], n = s_nad[0][q];
        int bi = s_idx[0][q];
        for (int w = 1; w < NB / 32; ++w) {
            if (lex_less(s_asf[w][q], s_idx[w][q], b, bi)) {
                b = s_asf[w][q];
                bi = s_idx[w][q];
            }
            n = fmax(n, s_nad[w][q]);
        }
        v.ext_part[blockIdx.x * m + q] = b;
        v.ext_idx[blockIdx.x * m + q] = bi;
        v.nad_part[blockIdx.x * m + q] = n;
    }
}

// final reduction + Gaussian elimination (one thread does the m x m solve)
__global__ void __launch_bounds__(32) k_norm_solve(RunView v)
{
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int m = v.m;
    __shared__ int s_ext[NSGA3_MAX_M];
    __shared__ double s_nad[NSGA3_MAX_M];
    if (threadIdx.x < m) {
        const int q = threadIdx.x;
        double b = CUDART_INF, n = 0.0;
        int bi = 0x7fffffff;
        for (int p = 0; p < v.ext_parts; ++p) {
            double pb = v.ext_part[p * m + q];
            int pi = v.ext_idx[p * m + q];
            if (lex_less(pb, pi, b, bi)) {
                b = pb;
                bi = pi;
            }
            n = fmax(n, v.nad_part[p * m + q]);
        }
        s_ext[q] = bi;
        s_nad[q] = n;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double zs[NSGA3_MAX_M];
    for (int q = 0; q < m; ++q) {
        zs[q] = zstar_of(c, q);
        c->zstar[q] = zs[q];
        c->ext[q] = s_ext[q];
    }
    double A[NSGA3_MAX_M][NSGA3_MAX_M], rhs[NSGA3_MAX_M], b[NSGA3_MAX_M];
    bool ok = true;
    for (int q = 0; q < m; ++q) {
        const int e = s_ext[q];
        if (e < 0 || e >= v.n2) ok = false;
        for (int r = 0; r < m; ++r)
            A[q][r] = ok ? __dsub_rn((double)v.F[(size_t)e * m + r], zs[r]) : 0.0;
        rhs[q] = 1.0;
    }
    for (int col = 0; col < m && ok; ++col) {
        int p = col;
        double bestp = fabs(A[col][col]);
        for (int r = col + 1; r < m; ++r)
            if (fabs(A[r][col]) > bestp) {
                bestp = fabs(A[r][col]);
                p = r;
            }
        if (bestp == 0.0) {
            ok = false;
            break;
        }
        if (p != col) {
            for (int cc = 0; cc < m; ++cc) {
                double t = A[col][cc];
                A[col][cc] = A[p][cc];
                A[p][cc] = t;
            }
            double t = rhs[col];
            rhs[col] = rhs[p];
            rhs[p] = t;
        }
        for (int r = col + 1; r < m; ++r) {
            const double factor = __ddiv_rn(A[r][col], A[col][col]);
            for (int cc = col; cc < m; ++cc) A[r][cc] = __dsub_rn(A[r][cc], __dmul_rn(factor, A[col][cc]));
            rhs[r] = __dsub_rn(rhs[r], __dmul_rn(factor, rhs[col]));
        }
    }
    double a[NSGA3_MAX_M];
    if (ok) {
        for (int r = m - 1; r >= 0; --r) {
            double s = rhs[r];
            for (int cc = r + 1; cc < m; ++cc) s = __dsub_rn(s, __dmul_rn(A[r][cc], b[cc]));
            b[r] = __ddiv_rn(s, A[r][r]);
        }
        for (int q = 0; q < m; ++q) {
            a[q] = __ddiv_rn(1.0, b[q]);
            if (!isfinite(a[q]) || a[q] <= 1e-6) ok = false;
        }
    }
    c->fallback = ok ? 0 : 1;
    for (int q = 0; q < m; ++q) {
        if (!ok) a[q] = (s_nad[q] == 0.0) ? 1.0 : s_nad[q];
        c->a[q] = a[q];
    }
}

}  // namespace

cudaError_t launch_norm_ideal(const RunView& v, cudaStream_t s)
{
    k_norm_ideal<<<(v.n2 + NB - 1) / NB, NB, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_norm_extreme(const RunView& v, cudaStream_t s)
{
    k_norm_extreme<<<v.ext_parts, NB, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_norm_solve(const RunView& v, cudaStream_t s)
{
    k_norm_solve<<<1, 32, 0, s>>>(v);
    return cudaGetLastError();
}
