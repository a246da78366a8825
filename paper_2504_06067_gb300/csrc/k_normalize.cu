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

constexpr int NB = 256;   // k_norm_ideal
constexpr int EB = 64;    // k_norm_extreme: small blocks spread the FP64 latency over the SMs

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

// Non-negative doubles order like their bit patterns; -0.0 is mapped to
// +0.0 so that the two zeros compare equal, as IEEE comparisons do.
__device__ __forceinline__ unsigned long long okey(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b << 1) == 0ull ? 0ull : b;  // integer test for +-0 (FP64 compares are slow)
}

__device__ __forceinline__ bool key_less(unsigned long long a, int ia, unsigned long long b, int ib)
{
    return a < b || (a == b && ia < ib);
}

// Gaussian elimination with partial pivoting (first maximal |pivot|) on
// E b = 1, a = 1 / b, nadir fallback; one thread, _rn intrinsics.
__device__ void solve_intercepts(const RunView& v, Ctrl* c, const int* ext, const double* nad)
{
    const int m = v.m;
    double zs[NSGA3_MAX_M];
    for (int q = 0; q < m; ++q) {
        zs[q] = zstar_of(c, q);
        c->zstar[q] = zs[q];
        c->ext[q] = ext[q];
    }
    double A[NSGA3_MAX_M][NSGA3_MAX_M], rhs[NSGA3_MAX_M], b[NSGA3_MAX_M];
    bool ok = true;
    for (int q = 0; q < m; ++q) {
        const int e = ext[q];
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
        if (!ok) a[q] = (nad[q] == 0.0) ? 1.0 : nad[q];
        c->a[q] = a[q];
    }
}

// Per-block (min ASF, lowest index) per axis and max of f~; the last block
// to finish reduces the blocks' results and solves for the intercepts.
__global__ void __launch_bounds__(EB) k_norm_extreme(RunView v)
{
    __shared__ unsigned long long s_key[EB / 32][NSGA3_MAX_M];
    __shared__ int s_idx[EB / 32][NSGA3_MAX_M];
    __shared__ unsigned long long s_nad[EB / 32][NSGA3_MAX_M];
    __shared__ unsigned s_ticket;
    __shared__ int f_ext[NSGA3_MAX_M];
    __shared__ double f_nad[NSGA3_MAX_M];
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int m = v.m, nT = c->nT;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    double zs[NSGA3_MAX_M];
    for (int q = 0; q < m; ++q) zs[q] = zstar_of(c, q);
    unsigned long long best[NSGA3_MAX_M], nad[NSGA3_MAX_M];
    int bidx[NSGA3_MAX_M];
    for (int q = 0; q < m; ++q) {
        best[q] = ~0ull;
        bidx[q] = 0x7fffffff;
        nad[q] = 0ull;
    }
    for (int s = blockIdx.x * EB + threadIdx.x; s < nT; s += gridDim.x * EB) {
        const int i = v.Tlist[s];
        double ft[NSGA3_MAX_M];
        unsigned long long m1 = 0ull, m2 = 0ull;  // largest and second largest key (f~ >= 0)
        int r1 = 0;
        for (int r = 0; r < m; ++r) {
            ft[r] = __dsub_rn((double)v.F[(size_t)i * m + r], zs[r]);
            const unsigned long long kr = okey(ft[r]);
            if (kr > m1) {
                m2 = m1;
                m1 = kr;
                r1 = r;
            } else if (kr > m2) {
                m2 = kr;
            }
            nad[r] = max(nad[r], kr);
        }
        const double d1 = __ddiv_rn(__longlong_as_double((long long)m1), 1e-6);
        const double d2 = __ddiv_rn(__longlong_as_double((long long)m2), 1e-6);
        const unsigned long long k1 = okey(d1), k2 = okey(d2);
        for (int q = 0; q < m; ++q) {
            const unsigned long long other = (q == r1) ? k2 : k1;
            const unsigned long long kq = okey(ft[q]);
            const unsigned long long asf = kq > other ? kq : other;
            if (key_less(asf, i, best[q], bidx[q])) {
                best[q] = asf;
                bidx[q] = i;
            }
        }
    }
    for (int q = 0; q < m; ++q) {
        unsigned long long b = best[q], n = nad[q];
        int bi = bidx[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            const unsigned long long on = __shfl_xor_sync(0xffffffffu, n, o);
            if (key_less(ob, oi, b, bi)) {
                b = ob;
                bi = oi;
            }
            n = max(n, on);
        }
        if (lane == 0) {
            s_key[warp][q] = b;
            s_idx[warp][q] = bi;
            s_nad[warp][q] = n;
        }
    }
    __syncthreads();
    unsigned long long* pk = reinterpret_cast<unsigned long long*>(v.ext_part);
    unsigned long long* pn = reinterpret_cast<unsigned long long*>(v.nad_part);
    if (threadIdx.x < m) {
        const int q = threadIdx.x;
        unsigned long long b = s_key[0][q], n = s_nad[0][q];
        int bi = s_idx[0][q];
        for (int w = 1; w < EB / 32; ++w) {
            if (key_less(s_key[w][q], s_idx[w][q], b, bi)) {
                b = s_key[w][q];
                bi = s_idx[w][q];
            }
            n = max(n, s_nad[w][q]);
        }
        pk[blockIdx.x * m + q] = b;
        v.ext_idx[blockIdx.x * m + q] = bi;
        pn[blockIdx.x * m + q] = n;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = atomicAdd(&c->ext_done, 1u);
    __syncthreads();
    if (s_ticket != gridDim.x - 1) return;
    // last block: reduce over the blocks (warp w reduces axes w, w + 8, ...)
    __threadfence();
    for (int q = warp; q < m; q += EB / 32) {
        unsigned long long b = ~0ull, n = 0ull;
        int bi = 0x7fffffff;
        for (int p = lane; p < (int)gridDim.x; p += 32) {
            const unsigned long long pb = __ldcg(&pk[p * m + q]);
            const int pi = __ldcg(&v.ext_idx[p * m + q]);
            if (key_less(pb, pi, b, bi)) {
                b = pb;
                bi = pi;
            }
            n = max(n, __ldcg(&pn[p * m + q]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            const unsigned long long on = __shfl_xor_sync(0xffffffffu, n, o);
            if (key_less(ob, oi, b, bi)) {
                b = ob;
                bi = oi;
            }
            n = max(n, on);
        }
        if (lane == 0) {
            f_ext[q] = bi;
            f_nad[q] = __longlong_as_double((long long)n);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        c->ext_done = 0u;
        solve_intercepts(v, c, f_ext, f_nad);
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
    k_norm_extreme<<<v.ext_parts, EB, 0, s>>>(v);
    return cudaGetLastError();
}
