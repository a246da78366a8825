// k_normalize.cu -- the normalization step of Alg. 1 and Alg. 2, read as
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
    if (v.m > NSGA3_FAST_M) return;  // k_zmin_gen
    // the block's minimum per objective first (warps, then shared memory),
    // one atomic per block and objective: the ideal point's m words are
    // every block's target
    __shared__ uint32_t smin[NB / 32][NSGA3_FAST_M];
    const int warp = threadIdx.x >> 5;
    for (int q = 0; q < v.m; ++q) {
        uint32_t o = inZ ? f2ord(v.Fp[(size_t)p * v.m + q]) : 0xffffffffu;
        o = __reduce_min_sync(0xffffffffu, o);
        if (lane == 0) smin[warp][q] = o;
    }
    __syncthreads();
    if (threadIdx.x < v.m) {
        uint32_t o = smin[0][threadIdx.x];
        for (int w = 1; w < NB / 32; ++w) o = min(o, smin[w][threadIdx.x]);
        if (o != 0xffffffffu) atomicMin(&c->zmin[threadIdx.x], o);
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
// rhs_r -= factor * rhs_c; back substitution from the last unknown, each
// row's known terms subtracted from the highest column down).
// M <= NSGA3_FAST_M: m = M; M = NSGA3_WARP_M: any m <= 32 at run time
// (rows and columns >= m are never touched).
template <int M>
__device__ void solve_intercepts(const RunView& v, Ctrl* c, const int* ext, const double* nad)
{
    const int m = (M <= NSGA3_FAST_M) ? M : v.m;
    const int lane = lane_id();
    double zs[M];
#pragma unroll
    for (int q = 0; q < M; ++q) zs[q] = q < m ? zstar_of(c, q) : 0.0;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < M; ++q)
            if (q < m) {
                c->zstar[q] = zs[q];
                c->ext[q] = ext[q];
            }
    }
    bool ok = true;
    const int ncand = v.n2 + ((v.norm_history && c->hvalid) ? m : 0);
#pragma unroll
    for (int q = 0; q < M; ++q)
        if (q < m && (ext[q] < 0 || ext[q] >= ncand)) ok = false;
    double A[M], rhs = 1.0;
    float evec[M];  // this lane's extreme vector (a merged point or a remembered one)
    const bool row = lane < m;
    const int er = row ? ext[lane] : 0;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        const bool in = ok && row && q < m;
        evec[q] = in ? (er < v.n2 ? v.F[(size_t)er * m + q] : v.he[(er - v.n2) * m + q]) : 0.0f;
        A[q] = in ? __dsub_rn((double)evec[q], zs[q]) : 0.0;
    }
#pragma unroll
    for (int col = 0; col < M; ++col) {
        if (!ok || col >= m) break;
        // pivot: first row >= col of maximal |A[.][col]| (rows in current order)
        int p = col;
        double best = fabs(__shfl_sync(0xffffffffu, A[col], col));
#pragma unroll
        for (int r = col + 1; r < M; ++r) {
            const double x = fabs(__shfl_sync(0xffffffffu, A[col], r));
            if (r < m && x > best) {
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
        if (lane > col && lane < m) {
            const double factor = __ddiv_rn(A[col], piv[col]);
#pragma unroll
            for (int q = col; q < M; ++q)
                if (q < m) A[q] = __dsub_rn(A[q], __dmul_rn(factor, piv[q]));
            rhs = __dsub_rn(rhs, __dmul_rn(factor, prhs));
        }
    }
    double a = 0.0;
    if (ok) {
        // back substitution column by column from the last unknown: every
        // lane subtracts A_ir b_r as soon as b_r is known, so row i meets its
        // terms from the highest column down, as the serial loop does
        double b = 0.0;  // lane r ends with b_r
#pragma unroll
        for (int r = M - 1; r >= 0; --r) {
            if (r >= m) continue;
            const double br = __shfl_sync(0xffffffffu, lane == r ? __ddiv_rn(rhs, A[r]) : 0.0, r);
            if (lane == r) b = br;
            if (lane < r) rhs = __dsub_rn(rhs, __dmul_rn(A[r], br));
        }
        a = lane < m ? __ddiv_rn(1.0, b) : 1.0;
        const bool bad = lane < m && (!isfinite(a) || a <= 1e-6);
        if (__any_sync(0xffffffffu, bad)) ok = false;
    }
    if (lane < m) {
        if (!ok) a = (nad[lane] == 0.0) ? 1.0 : nad[lane];
        c->a[lane] = a;
    }
    if (lane == 0) c->fallback = ok ? 0 : 1;
    if (v.norm_history) {
        // the ideal and the extreme vectors become the history (every lane
        // read its remembered row above, before these writes)
        __syncwarp();
        if (lane < m) {
            c->hz[lane] = zs[lane];
#pragma unroll
            for (int q = 0; q < M; ++q)
                if (q < m) v.he[lane * m + q] = evec[q];
        }
        if (lane == 0) c->hvalid = 1;
    }
}

// Per-block (min ASF, lowest index) per axis and max of f~; the last block
// to finish reduces the blocks' results and solves for the intercepts.
template <int M>
__global__ void __launch_bounds__(EB) k_norm_extreme(RunView v)
{
    __shared__ unsigned long long s_key[EB / 32][NSGA3_FAST_M];
    __shared__ int s_idx[EB / 32][NSGA3_FAST_M];
    __shared__ unsigned long long s_nad[EB / 32][NSGA3_FAST_M];
    __shared__ unsigned s_ticket;
    __shared__ int f_ext[NSGA3_FAST_M];
    __shared__ double f_nad[NSGA3_FAST_M];
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
                    const float* f = v.he + r * m;
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

// ---------------------------------------------------------------------------
// m > NSGA3_FAST_M.  The candidates of the extreme-point search are "entries":
// the members of T (index = merged index) and, with history, the remembered
// vectors (index 2N + r).  k_ext_keys gives each entry the two ASF keys it
// can have: fl(max_r f~_r / 1e-6) and, for the axis of that maximum (first
// index), fl(second largest / 1e-6).  k_ext_axis takes QG axes per block:
// ASF_q = max(f~_q, that key) per entry, (min, lowest index) per axis, and
// the nadir maxima over the members; k_ext_reduce reduces the blocks (a warp
// per axis) and either solves the intercepts with one warp
// (m <= NSGA3_WARP_M) or leaves E and the nadir to the cooperative
// elimination below.
constexpr int GB = 128;  // threads per block of the m > NSGA3_FAST_M kernels
constexpr int QG = 8;    // axes per block of k_ext_axis

__device__ __forceinline__ const float* entry_row(const RunView& v, int s, int nT, int& idx)
{
    if (s < nT) {
        idx = v.Tlist[s];
        return v.F + (size_t)idx * v.m;
    }
    idx = v.n2 + (s - nT);
    return v.he + (size_t)(s - nT) * v.m;
}

__device__ __forceinline__ int history_entries(const RunView& v, const Ctrl* c)
{
    return (v.norm_history && c->hvalid) ? v.m : 0;
}

// ideal point for m > NSGA3_FAST_M: thread per objective over a chunk of
// positions (coalesced across objectives), order-preserving atomicMin
constexpr int ZP = 32;  // positions per chunk

__global__ void __launch_bounds__(128) k_zmin_gen(RunView v)
{
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int m = v.m, q = blockIdx.x * 128 + threadIdx.x;
    if (q >= m) return;
    const int l = c->l;
    const int p0 = blockIdx.y * ZP, p1 = min(v.n2, p0 + ZP);
    uint32_t o = 0xffffffffu;
#pragma unroll 8
    for (int p = p0; p < p1; ++p) {
        const int r = v.srank[p];
        const bool in = v.norm_history ? true : (r >= 0 && r <= l);
        if (in) o = min(o, f2ord(v.Fp[(size_t)p * m + q]));
    }
    if (o != 0xffffffffu) atomicMin(&c->zmin[q], o);
}

// a warp per entry: lane-wise (largest key, second largest, first index of
// the largest) over r = lane, lane + 32, ..., merged across the lanes; the
// result is that of one pass over r = 0 .. m-1 (largest, the largest of the
// rest counting a repeated maximum, its first index)
__global__ void __launch_bounds__(GB) k_ext_keys(RunView v)
{
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int m = v.m, nT = c->nT, lane = lane_id();
    const int ne = nT + history_entries(v, c);
    const int nw = gridDim.x * (GB / 32);
    for (int s = (blockIdx.x * GB + threadIdx.x) >> 5; s < ne; s += nw) {
        int idx;
        const float* f = entry_row(v, s, nT, idx);
        unsigned long long m1 = 0ull, m2 = 0ull;  // f~ >= 0: keys order like values
        int r1 = 0x7fffffff;                      // none while m1 == 0
        for (int r = lane; r < m; r += 32) {
            const unsigned long long kr = okey(__dsub_rn((double)f[r], zstar_of(c, r)));
            if (kr > m1) {
                m2 = m1;
                m1 = kr;
                r1 = r;
            } else if (kr > m2) {
                m2 = kr;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long om1 = __shfl_xor_sync(0xffffffffu, m1, o);
            const unsigned long long om2 = __shfl_xor_sync(0xffffffffu, m2, o);
            const int or1 = __shfl_xor_sync(0xffffffffu, r1, o);
            if (om1 > m1) {
                m2 = max(om2, m1);
                m1 = om1;
                r1 = or1;
            } else if (om1 < m1) {
                m2 = max(m2, om1);
            } else if (m1 > 0ull) {  // the maximum occurs on both sides
                m2 = m1;
                r1 = min(r1, or1);
            }
        }
        if (lane == 0) {
            v.ekey[2 * (size_t)s] = okey(__ddiv_rn(__longlong_as_double((long long)m1), 1e-6));
            v.ekey[2 * (size_t)s + 1] = okey(__ddiv_rn(__longlong_as_double((long long)m2), 1e-6));
            v.er1[s] = m1 > 0ull ? r1 : 0;
        }
    }
}

// grid (parts, ceil(m / QG))
__global__ void __launch_bounds__(GB) k_ext_axis(RunView v)
{
    __shared__ unsigned long long s_key[GB / 32][QG];
    __shared__ int s_idx[GB / 32][QG];
    __shared__ unsigned long long s_nad[GB / 32][QG];
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int m = v.m, nT = c->nT;
    const int ne = nT + history_entries(v, c);
    const int parts = gridDim.x;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int q0 = blockIdx.y * QG;
    double zs[QG];
    unsigned long long best[QG], nad[QG];
    int bidx[QG];
#pragma unroll
    for (int t = 0; t < QG; ++t) {
        zs[t] = q0 + t < m ? zstar_of(c, q0 + t) : 0.0;
        best[t] = ~0ull;
        bidx[t] = 0x7fffffff;
        nad[t] = 0ull;
    }
    for (int s = blockIdx.x * GB + threadIdx.x; s < ne; s += parts * GB) {
        int idx;
        const float* f = entry_row(v, s, nT, idx);
        const unsigned long long k1 = v.ekey[2 * (size_t)s], k2 = v.ekey[2 * (size_t)s + 1];
        const int r1 = v.er1[s];
#pragma unroll
        for (int t = 0; t < QG; ++t) {
            const int q = q0 + t;
            if (q >= m) break;
            const unsigned long long kq = okey(__dsub_rn((double)f[q], zs[t]));
            const unsigned long long other = (q == r1) ? k2 : k1;
            const unsigned long long asf = kq > other ? kq : other;
            if (key_less(asf, idx, best[t], bidx[t])) {
                best[t] = asf;
                bidx[t] = idx;
            }
            if (s < nT) nad[t] = max(nad[t], kq);
        }
    }
#pragma unroll
    for (int t = 0; t < QG; ++t) {
        unsigned long long b = best[t], n = nad[t];
        int bi = bidx[t];
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
            s_key[warp][t] = b;
            s_idx[warp][t] = bi;
            s_nad[warp][t] = n;
        }
    }
    __syncthreads();
    unsigned long long* pk = reinterpret_cast<unsigned long long*>(v.ext_part);
    unsigned long long* pn = reinterpret_cast<unsigned long long*>(v.nad_part);
    if (threadIdx.x < QG && q0 + (int)threadIdx.x < m) {
        const int t = threadIdx.x, q = q0 + t;
        unsigned long long b = s_key[0][t], n = s_nad[0][t];
        int bi = s_idx[0][t];
        for (int w = 1; w < GB / 32; ++w) {
            if (key_less(s_key[w][t], s_idx[w][t], b, bi)) {
                b = s_key[w][t];
                bi = s_idx[w][t];
            }
            n = max(n, s_nad[w][t]);
        }
        pk[(size_t)blockIdx.x * m + q] = b;
        v.ext_idx[(size_t)blockIdx.x * m + q] = bi;
        pn[(size_t)blockIdx.x * m + q] = n;
    }
}

// per axis (a warp each) the (min, lowest index) over the parts and the
// nadir maximum; with m <= NSGA3_WARP_M the last CTA solves the intercepts
// with one warp, else the cooperative elimination follows
__global__ void __launch_bounds__(256) k_ext_reduce(RunView v, int parts)
{
    __shared__ unsigned s_ticket;
    __shared__ int f_ext[NSGA3_WARP_M];
    __shared__ double f_nad[NSGA3_WARP_M];
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int m = v.m, lane = lane_id();
    const int q = blockIdx.x * 8 + (threadIdx.x >> 5);
    const unsigned long long* pk = reinterpret_cast<const unsigned long long*>(v.ext_part);
    const unsigned long long* pn = reinterpret_cast<const unsigned long long*>(v.nad_part);
    if (q < m) {
        unsigned long long b = ~0ull, n = 0ull;
        int bi = 0x7fffffff;
        for (int p = lane; p < parts; p += 32) {
            const unsigned long long pb = pk[(size_t)p * m + q];
            const int pi = v.ext_idx[(size_t)p * m + q];
            if (key_less(pb, pi, b, bi)) {
                b = pb;
                bi = pi;
            }
            n = max(n, pn[(size_t)p * m + q]);
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
            c->ext[q] = bi;
            v.nadv[q] = __longlong_as_double((long long)n);
        }
    }
    if (m > NSGA3_WARP_M) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = atomicAdd(&c->ext_done, 1u);
    __syncthreads();
    if (s_ticket != gridDim.x - 1) return;
    __threadfence();
    if (threadIdx.x < m) {
        f_ext[threadIdx.x] = __ldcg(&c->ext[threadIdx.x]);
        f_nad[threadIdx.x] = __ldcg(&v.nadv[threadIdx.x]);
    }
    __syncthreads();
    if (threadIdx.x == 0) c->ext_done = 0u;
    if (threadIdx.x < 32) solve_intercepts<NSGA3_WARP_M>(v, c, f_ext, f_nad);
}

// m > NSGA3_WARP_M: the elimination of the warp solver spread over a
// cooperative grid.  The augmented rows [E - z* | 1] live in amat (original
// row order); every CTA keeps the same current row order ord[] and takes
// the same pivot (first maximal |A[.][col]| in that order), so a pivot step
// needs one grid barrier: a warp per remaining row forms its factor and
// updates columns col+1 .. m (m = the right-hand side) with the same _rn
// operations as the serial elimination (column col is not needed again).
// Reads of amat bypass L1 (other SMs write it between barriers).  The back
// substitution (the order of the warp solver) runs in CTA 0.
constexpr int SB = 256;
static_assert(NSGA3_MAX_M <= 2 * SB, "the back substitution keeps two rows per thread");

__global__ void __launch_bounds__(SB) k_solve_coop(RunView v)
{
    __shared__ int ord[NSGA3_MAX_M];
    __shared__ double sb[NSGA3_MAX_M];
    __shared__ double colv[NSGA3_MAX_M];  // column col of the rows, by position
    __shared__ double red_x[SB / 32];
    __shared__ int red_p[SB / 32];
    __shared__ int s_ok, s_piv;
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int m = v.m, ld = m + 1;
    unsigned nbar = 0;  // barriers passed (c->sbar is zero at launch: k_sel_reset)
    const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    // rows go to the CTAs in turn, so that the FP64 work of a step spreads
    // over every SM of the grid
    const int gw = warp * gridDim.x + blockIdx.x, nw = gridDim.x * (SB / 32);
    double* A = v.amat;
    const int ncand = v.n2 + ((v.norm_history && c->hvalid) ? m : 0);
    bool bad_ext = false;
    for (int q = tid; q < m; q += SB) {
        const int e = c->ext[q];
        bad_ext |= e < 0 || e >= ncand;
        ord[q] = q;
        if (blockIdx.x == 0) c->zstar[q] = zstar_of(c, q);
    }
    const bool ext_ok = !__syncthreads_or(bad_ext);
    bool ok = ext_ok;
    if (ok) {
        // rows of the system and the new extreme vectors (warp per row)
        for (int q = gw; q < m; q += nw) {
            const int er = c->ext[q];
            const float* f = er < v.n2 ? v.F + (size_t)er * m : v.he + (size_t)(er - v.n2) * m;
            for (int k = lane; k < m; k += 32) {
                const float ev = f[k];
                v.etmp[(size_t)q * m + k] = ev;
                A[(size_t)q * ld + k] = __dsub_rn((double)ev, zstar_of(c, k));
            }
            if (lane == 0) A[(size_t)q * ld + m] = 1.0;
        }
        if (!grid_sync_count(c, &c->sbar, ++nbar * gridDim.x, v.wait_ns, &s_ok)) return;
        for (int col = 0; col < m; ++col) {
            // pivot (every CTA): the first position p >= col of maximal
            // |A[ord[p]][col]|; a NaN never replaces the running maximum
            // (the column's values stay in colv for the factors below)
            double bx = -1.0;
            int bp = 0x7fffffff;
#pragma unroll 2
            for (int p = col + tid; p < m; p += SB) {
                const double val = __ldcg(&A[(size_t)ord[p] * ld + col]);
                colv[p] = val;
                const double x = fabs(val);
                if (p > col && x > bx) {  // positions ascend per thread: the first maximum stays
                    bx = x;
                    bp = p;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ox = __shfl_xor_sync(0xffffffffu, bx, o);
                const int op = __shfl_xor_sync(0xffffffffu, bp, o);
                if (ox > bx || (ox == bx && op < bp)) {
                    bx = ox;
                    bp = op;
                }
            }
            if (lane == 0) {
                red_x[warp] = bx;
                red_p[warp] = bp;
            }
            __syncthreads();
            if (tid == 0) {
                for (int w = 1; w < SB / 32; ++w)
                    if (red_x[w] > bx || (red_x[w] == bx && red_p[w] < bp)) {
                        bx = red_x[w];
                        bp = red_p[w];
                    }
                const double x0 = fabs(colv[col]);
                int p = col;
                double best = x0;
                if (x0 == x0 && bp != 0x7fffffff && bx > x0) {  // x0 NaN: col stays
                    p = bp;
                    best = bx;
                }
                s_piv = p;
                s_ok = best == 0.0 ? 0 : 1;
                if (p != col) {
                    const int t = ord[col];
                    ord[col] = ord[p];
                    ord[p] = t;
                }
            }
            __syncthreads();
            if (!s_ok) {
                ok = false;
                break;
            }
            const int P = ord[col], pp = s_piv;
            const double pv = colv[pp];  // the pivot row's value (read at its old position)
            for (int pos = col + 1 + gw; pos < m; pos += nw) {
                const int r = ord[pos];
                // the row now at pp came from position col
                const double factor = __ddiv_rn(pos == pp ? colv[col] : colv[pos], pv);
#pragma unroll 4  // four pairs of loads in flight (L2 round trips dominate a step)
                for (int k = col + 1 + lane; k <= m; k += 32)
                    A[(size_t)r * ld + k] = __dsub_rn(__ldcg(&A[(size_t)r * ld + k]),
                                                      __dmul_rn(factor, __ldcg(&A[(size_t)P * ld + k])));
            }
            if (!grid_sync_count(c, &c->sbar, ++nbar * gridDim.x, v.wait_ns, &s_ok)) return;
        }
    }
    if (blockIdx.x != 0) return;
    // CTA 0: back substitution column by column from the last unknown (as
    // in the warp solver); thread t keeps the partial sums of positions t
    // and t + SB and loads the next column's elements a step ahead
    if (ok) {
        const int i0 = tid, i1 = tid + SB;
        const size_t R0 = i0 < m ? (size_t)ord[i0] * ld : 0, R1 = i1 < m ? (size_t)ord[i1] * ld : 0;
        double s0 = i0 < m ? __ldcg(&A[R0 + m]) : 0.0, s1 = i1 < m ? __ldcg(&A[R1 + m]) : 0.0;
        const double d0 = i0 < m ? __ldcg(&A[R0 + i0]) : 1.0, d1 = i1 < m ? __ldcg(&A[R1 + i1]) : 1.0;
        double c0 = i0 < m - 1 ? __ldcg(&A[R0 + m - 1]) : 0.0;
        double c1 = i1 < m - 1 ? __ldcg(&A[R1 + m - 1]) : 0.0;
        for (int r = m - 1; r >= 0; --r) {
            if (i0 == r) sb[r] = __ddiv_rn(s0, d0);
            if (i1 == r) sb[r] = __ddiv_rn(s1, d1);
            __syncthreads();
            const double br = sb[r];
            const double u0 = c0, u1 = c1;
            if (r > 0) {
                c0 = i0 < r - 1 ? __ldcg(&A[R0 + r - 1]) : 0.0;
                c1 = i1 < r - 1 ? __ldcg(&A[R1 + r - 1]) : 0.0;
            }
            if (i0 < r) s0 = __dsub_rn(s0, __dmul_rn(u0, br));
            if (i1 < r) s1 = __dsub_rn(s1, __dmul_rn(u1, br));
        }
    }
    __syncthreads();
    bool bad = false;
    if (ok)
        for (int q = tid; q < m; q += SB) {
            const double a = __ddiv_rn(1.0, sb[q]);
            bad |= !isfinite(a) || a <= 1e-6;
            sb[q] = a;
        }
    ok = ok && !__syncthreads_or(bad);
    for (int q = tid; q < m; q += SB) {
        const double nq = v.nadv[q];
        c->a[q] = ok ? sb[q] : (nq == 0.0 ? 1.0 : nq);
    }
    if (tid == 0) c->fallback = ok ? 0 : 1;
    if (v.norm_history) {
        for (int q = tid; q < m; q += SB) c->hz[q] = zstar_of(c, q);
        // the staged extreme vectors (zero rows, as in the warp solver, when
        // an extreme index was invalid and nothing was staged)
        for (int e = tid; e < m * m; e += SB) v.he[e] = ext_ok ? v.etmp[e] : 0.0f;
        if (tid == 0) c->hvalid = 1;
    }
}

}  // namespace

cudaError_t launch_norm_ideal(const RunView& v, cudaStream_t s)
{
    k_norm_ideal<<<(v.n2 + NB - 1) / NB, NB, 0, s>>>(v);
    return cudaGetLastError();
}

static int g_solve_occ = 0;  // resident k_solve_coop CTAs per SM, set at start-up

static cudaError_t launch_norm_extreme_gen(const RunView& v, int num_sms, cudaStream_t s)
{
    if (v.m <= NSGA3_FAST_M || v.m > NSGA3_MAX_M) return cudaErrorInvalidValue;
    const int qgroups = (v.m + QG - 1) / QG;
    int parts = (2 * num_sms + qgroups - 1) / qgroups;
    if (parts > v.ext_parts) parts = v.ext_parts;
    if (parts > (v.n2 + v.m + GB - 1) / GB) parts = (v.n2 + v.m + GB - 1) / GB;
    if (parts < 1) parts = 1;
    k_zmin_gen<<<dim3((v.m + 127) / 128, (v.n2 + ZP - 1) / ZP), 128, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int kb = (v.n2 + v.m + GB / 32 - 1) / (GB / 32);
    if (kb > 8 * num_sms) kb = 8 * num_sms;
    k_ext_keys<<<kb, GB, 0, s>>>(v);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ext_axis<<<dim3(parts, qgroups), GB, 0, s>>>(v);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ext_reduce<<<(v.m + 7) / 8, 256, 0, s>>>(v, parts);
    e = cudaGetLastError();
    if (e != cudaSuccess || v.m <= NSGA3_WARP_M) return e;
    // a CTA per SM (the FP64 pipe of every SM), at most a row per CTA at the
    // first step; every CTA resident
    int grid = v.m - 1;
    if (grid > num_sms) grid = num_sms;
    const int cap = num_sms * (g_solve_occ > 0 ? g_solve_occ : 1);
    if (grid > cap) grid = cap;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(SB);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_solve_coop, v);
}

cudaError_t norm_init_attributes()
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_solve_occ, k_solve_coop, SB, 0);
}

cudaError_t launch_norm_extreme(const RunView& v, int num_sms, cudaStream_t s)
{
    if (v.m > NSGA3_FAST_M) return launch_norm_extreme_gen(v, num_sms, s);
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
