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
constexpr int EB = 128;   // k_norm_extreme: two blocks per SM

// Ranks back to the original order (every selection), then, when niching
// is needed: members of T are appended to Tlist (in bucket order, which no
// later step depends on) and the ideal point is taken by order-preserving
// atomicMin over Fp (-0.0 is stored as +0.0 there).
__global__ void __launch_bounds__(NB) k_norm_ideal(RunView v)
{
    Ctrl* c = v.ctrl;
    if (read_status(c)) return;
    const int p = blockIdx.x * NB + threadIdx.x;  // position in bucket order
    int i = -1, r = -1;
    if (p < v.n2) {
        i = v.perm[p];
        r = v.srank[p];
        v.rank2[i] = r;
    }
    if (*(volatile const int32_t*)&c->need_niche == 0) return;  // the same for every thread
    const int l = c->l;
    const int lane = lane_id();
    const bool inT = i >= 0 && r >= 0 && r <= l;
    unsigned bal = __ballot_sync(0xffffffffu, inT);
    int base = 0;
    if (lane == 0 && bal) base = atomicAdd(&c->nT, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (inT) v.Tlist[base + __popc(bal & ((1u << lane) - 1u))] = i;
    // the running ideal (history option) takes every merged point and the
    // previous ideal; a minimum over S u F_l otherwise
    const bool inZ = v.norm_history ? (p < v.n2) : inT;
    if (v.norm_history && blockIdx.x == 0 && threadIdx.x == 0 && c->hvalid)
        for (int q = 0; q < v.m; ++q) atomicMin(&c->zmin[q], f2ord((float)c->hz[q]));
    for (int q = 0; q < v.m; ++q) {
        uint32_t o = inZ ? f2ord(v.Fp[(size_t)p * v.m + q]) : 0xffffffffu;
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
// E b = 1, a = 1 / b, nadir fallback.  One warp: lane r holds row r of the
// (row-swapped) system, so each elimination step updates every row at once;
// every element sees the same _rn operations in the same order as a serial
// elimination (factor = A_rc / A_cc, A_rk -= factor * A_ck for k >= c,
// rhs_r -= factor * rhs_c; back substitution left to right).
template <int M>
__device__ void solve_intercepts(const RunView& v, Ctrl* c, const int* ext, const double* nad)
{
    const int lane = lane_id();
    double zs[M];
#pragma unroll
    for (int q = 0; q < M; ++q) zs[q] = zstar_of(c, q);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < M; ++q) {
            c->zstar[q] = zs[q];
            c->ext[q] = ext[q];
        }
    }
    bool ok = true;
    const int ncand = v.n2 + ((v.norm_history && c->hvalid) ? M : 0);
#pragma unroll
    for (int q = 0; q < M; ++q)
        if (ext[q] < 0 || ext[q] >= ncand) ok = false;
    double A[M], rhs = 1.0;
    float evec[M];  // this lane's extreme vector (a merged point or a remembered one)
    const int er = lane < M ? ext[lane] : 0;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        evec[q] = (ok && lane < M) ? (er < v.n2 ? v.F[(size_t)er * M + q] : c->he[(er - v.n2) * M + q]) : 0.0f;
        A[q] = (ok && lane < M) ? __dsub_rn((double)evec[q], zs[q]) : 0.0;
    }
#pragma unroll
    for (int col = 0; col < M; ++col) {
        if (!ok) break;
        // pivot: first row >= col of maximal |A[.][col]| (rows in current order)
        int p = col;
        double best = fabs(__shfl_sync(0xffffffffu, A[col], col));
#pragma unroll
        for (int r = col + 1; r < M; ++r) {
            const double x = fabs(__shfl_sync(0xffffffffu, A[col], r));
            if (x > best) {
                best = x;
                p = r;
            }
        }
        if (best == 0.0) {
            ok = false;
            break;
        }
        if (p != col) {  // swap rows col and p
#pragma unroll
            for (int q = 0; q < M; ++q) {
                const double a_c = __shfl_sync(0xffffffffu, A[q], col);
                const double a_p = __shfl_sync(0xffffffffu, A[q], p);
                if (lane == col) A[q] = a_p;
                if (lane == p) A[q] = a_c;
            }
            const double r_c = __shfl_sync(0xffffffffu, rhs, col);
            const double r_p = __shfl_sync(0xffffffffu, rhs, p);
            if (lane == col) rhs = r_p;
            if (lane == p) rhs = r_c;
        }
        double piv[M];
#pragma unroll
        for (int q = 0; q < M; ++q) piv[q] = __shfl_sync(0xffffffffu, A[q], col);
        const double prhs = __shfl_sync(0xffffffffu, rhs, col);
        if (lane > col && lane < M) {
            const double factor = __ddiv_rn(A[col], piv[col]);
#pragma unroll
            for (int q = col; q < M; ++q) A[q] = __dsub_rn(A[q], __dmul_rn(factor, piv[q]));
            rhs = __dsub_rn(rhs, __dmul_rn(factor, prhs));
        }
    }
    double a = 0.0;
    if (ok) {
        double b = 0.0;  // lane r ends with b_r
#pragma unroll
        for (int r = M - 1; r >= 0; --r) {
            double s = rhs;
#pragma unroll
            for (int cc = r + 1; cc < M; ++cc) s = __dsub_rn(s, __dmul_rn(A[cc], __shfl_sync(0xffffffffu, b, cc)));
            const double br = __ddiv_rn(s, A[r]);
            if (lane == r) b = br;
        }
        a = lane < M ? __ddiv_rn(1.0, b) : 1.0;
        const bool bad = lane < M && (!isfinite(a) || a <= 1e-6);
        if (__any_sync(0xffffffffu, bad)) ok = false;
    }
    if (lane < M) {
        if (!ok) a = (nad[lane] == 0.0) ? 1.0 : nad[lane];
        c->a[lane] = a;
    }
    if (lane == 0) c->fallback = ok ? 0 : 1;
    if (v.norm_history) {
        // the ideal and the extreme vectors become the history (every lane
        // read its remembered row above, before these writes)
        __syncwarp();
        if (lane < M) {
            c->hz[lane] = zs[lane];
#pragma unroll
            for (int q = 0; q < M; ++q) c->he[lane * M + q] = evec[q];
        }
        if (lane == 0) c->hvalid = 1;
    }
}

// Per-block (min ASF, lowest index) per axis and max of f~; the last block
// to finish reduces the blocks' results and solves for the intercepts.
template <int M>
__global__ void __launch_bounds__(EB) k_norm_extreme(RunView v)
{
    __shared__ unsigned long long s_key[EB / 32][NSGA3_MAX_M];
    __shared__ int s_idx[EB / 32][NSGA3_MAX_M];
    __shared__ unsigned long long s_nad[EB / 32][NSGA3_MAX_M];
    __shared__ unsigned s_ticket;
    __shared__ int f_ext[NSGA3_MAX_M];
    __shared__ double f_nad[NSGA3_MAX_M];
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    constexpr int m = M;
    const int nT = c->nT;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    double zs[M];
    _Pragma("unroll") for (int q = 0; q < m; ++q) zs[q] = zstar_of(c, q);
    unsigned long long best[M], nad[M];
    int bidx[M];
    _Pragma("unroll") for (int q = 0; q < m; ++q) {
        best[q] = ~0ull;
        bidx[q] = 0x7fffffff;
        nad[q] = 0ull;
    }
    for (int s = blockIdx.x * EB + threadIdx.x; s < nT; s += gridDim.x * EB) {
        const int i = v.Tlist[s];
        double ft[M];
        unsigned long long m1 = 0ull, m2 = 0ull;  // largest and second largest key (f~ >= 0)
        int r1 = 0;
        _Pragma("unroll") for (int r = 0; r < m; ++r) {
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
        _Pragma("unroll") for (int q = 0; q < m; ++q) {
            const unsigned long long other = (q == r1) ? k2 : k1;
            const unsigned long long kq = okey(ft[q]);
            const unsigned long long asf = kq > other ? kq : other;
            if (key_less(asf, i, best[q], bidx[q])) {
                best[q] = asf;
                bidx[q] = i;
            }
        }
    }
    _Pragma("unroll") for (int q = 0; q < m; ++q) {
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
    // last block: reduce over the blocks, one warp per axis; each lane first
    // issues all its loads (independent), then reduces
    __threadfence();
    constexpr int PMAX = 16;  // parts <= 32 * PMAX
    for (int q = warp; q < m; q += EB / 32) {
        unsigned long long lb[PMAX], ln[PMAX];
        int li[PMAX];
#pragma unroll
        for (int t = 0; t < PMAX; ++t) {
            const int p = lane + 32 * t;
            const bool in = p < (int)gridDim.x;
            lb[t] = in ? __ldcg(&pk[p * m + q]) : ~0ull;
            li[t] = in ? __ldcg(&v.ext_idx[p * m + q]) : 0x7fffffff;
            ln[t] = in ? __ldcg(&pn[p * m + q]) : 0ull;
        }
        unsigned long long b = lb[0], n = ln[0];
        int bi = li[0];
#pragma unroll
        for (int t = 1; t < PMAX; ++t) {
            if (key_less(lb[t], li[t], b, bi)) {
                b = lb[t];
                bi = li[t];
            }
            n = max(n, ln[t]);
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
            if (v.norm_history && c->hvalid) {
                // the remembered extreme vectors are candidates 2N + r
                for (int r = 0; r < m; ++r) {
                    const float* f = c->he + r * m;
                    double mx = 0.0, tq = 0.0;
                    for (int t = 0; t < m; ++t) {
                        const double ft = __dsub_rn((double)f[t], zs[t]);
                        if (t == q)
                            tq = ft;
                        else if (ft > mx)
                            mx = ft;
                    }
                    const unsigned long long kq = okey(tq), ko = okey(__ddiv_rn(mx, 1e-6));
                    const unsigned long long asf = kq > ko ? kq : ko;
                    if (key_less(asf, v.n2 + r, b, bi)) {
                        b = asf;
                        bi = v.n2 + r;
                    }
                }
            }
            f_ext[q] = bi;
            f_nad[q] = __longlong_as_double((long long)n);
        }
    }
    __syncthreads();
    if (warp == 0) {
        if (lane == 0) c->ext_done = 0u;
        solve_intercepts<M>(v, c, f_ext, f_nad);
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
    switch (v.m) {
    case 2: k_norm_extreme<2><<<v.ext_parts, EB, 0, s>>>(v); break;
    case 3: k_norm_extreme<3><<<v.ext_parts, EB, 0, s>>>(v); break;
    case 4: k_norm_extreme<4><<<v.ext_parts, EB, 0, s>>>(v); break;
    case 5: k_norm_extreme<5><<<v.ext_parts, EB, 0, s>>>(v); break;
    case 6: k_norm_extreme<6><<<v.ext_parts, EB, 0, s>>>(v); break;
    case 7: k_norm_extreme<7><<<v.ext_parts, EB, 0, s>>>(v); break;
    case 8: k_norm_extreme<8><<<v.ext_parts, EB, 0, s>>>(v); break;
    case 9: k_norm_extreme<9><<<v.ext_parts, EB, 0, s>>>(v); break;
    case 10: k_norm_extreme<10><<<v.ext_parts, EB, 0, s>>>(v); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
