// k_dominance.cu -- bit-packed Pareto-dominance matrix (Alg. 1, the
// non-dominated sort; dominance for minimisation, Eq. 1).
//
// Dom[I][j] (u32, word-major, I = i / 32) holds bit (i mod 32) = "i
// dominates j": a column j's dominators are NW words with j contiguous
// across rows, which the front peel reads coalesced.
//
// Work: only unordered pairs are compared.  Persistent CTAs take 256 x 256
// tiles of the upper block triangle from the tile plan; the tile's 32 x 32
// block pairs are decided from per-block bounding boxes (no test, one
// direction, or both), and the warps take the pairs to test from a shared
// work list, lane = one row, objectives in registers, the column points
// broadcast from shared memory.  Per pair the m differences f_j - f_i and
// f_i - f_j run on the FMA pipe and their sign bits are OR-ed (3-input
// LOP3): A = "no f_i > f_j" and B = "no f_j > f_i"; "i dom j" = A & !B,
// "j dom i" = B & !A (identical vectors: neither).  -0.0 is turned into
// +0.0 when the tile is staged.  Points are in sort-key order (k_sort.cu:
// a dominator never has a larger key).  A block pair where only "row
// dominates column" can hold tests only the live rows (no objective above
// the column block's maximum) against the live columns (no objective below
// the live rows' minimum), two objectives per sub.rn.f32x2, the live rows
// of two row blocks packed onto one set of lanes when they fit
// (entry_row_dom_col).
// "j dom i" bits gathered over j are already column words Dom[jb][i];
// "i dom j" bits gathered over j are row words and are transposed in-warp
// (32 x 32 bit transpose by five shuffle stages) into Dom[ib][j].
// Padding rows/columns hold NaN: both differences of a pair with a padding
// point are the same NaN, so neither direction gets a bit; column blocks of
// padding only (the last tile column) skip the test and write zero words.
//
// Every CTA also popcounts the words it writes and adds each point's
// dominator count to cnt[] (the peel's first pass then reads no words).
// In streaming mode (no matrix) only the counts are produced; the peel
// recomputes the dominance of each front's members (k_peel.cu).
//
// m > 10 (k_dominance_gen): the same tiles, objectives staged in chunks of
// 16 and the two sign masks OR-ed over the chunks.
//
// Bound: the ALU pipe (sign-bit logic) and instruction issue -- not HBM.
#include "kernels.cuh"

namespace {

__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x)
{
    const int lane = lane_id();
    const uint32_t lo_masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int s = 16 >> t;
        const uint32_t mlo = lo_masks[t];
        const uint32_t mhi = ~mlo;
        uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
        if (lane & s)
            x = (x & mhi) | ((y & mhi) >> s);
        else
            x = (x & mlo) | ((y & mlo) << s);
    }
    return x;
}

__device__ __forceinline__ void decode_tile(long long t, int T, int& ti, int& tj)
{
    // tiles (ti <= tj) enumerated row by row: row ti starts at ti*T - ti*(ti-1)/2;
    // FP32 estimate of the row, corrected exactly by the integer loops below
    float b = 2.0f * (float)T + 1.0f;
    int r = (int)floorf((b - sqrtf(fmaxf(0.0f, b * b - 8.0f * (float)t))) * 0.5f);
    if (r < 0) r = 0;
    if (r > T - 1) r = T - 1;
    auto start = [&](long long x) { return x * T - x * (x - 1) / 2; };
    while (r > 0 && start(r) > t) --r;
    while (r + 1 < T && start(r + 1) <= t) ++r;
    ti = r;
    tj = r + (int)(t - start(r));
}

// Sign bit set iff some f_iq > f_jq for q = Q0 .. M-1 (the one-direction
// test).  The sign bits are OR-ed three at a time on the integer pipe; when
// the M-Q0 differences are an even number, the first two are first combined
// by fminf on the FP32 pipe (the minimum is negative iff one of them is;
// differences are never -0.0 because -0.0 is staged as +0.0), which saves
// one integer operation per pair and row.
template <int Q0, int M>
__device__ __forceinline__ uint32_t any_greater(const float* fj, const float* fi)
{
    uint32_t oa;
    int q0;
    if (M - Q0 >= 2 && (M - Q0) % 2 == 0) {
        oa = __float_as_uint(fminf(fj[Q0] - fi[Q0], fj[Q0 + 1] - fi[Q0 + 1]));
        q0 = Q0 + 2;
    } else {
        oa = 0u;
        q0 = Q0;
    }
#pragma unroll
    for (int q = q0; q < M; ++q) oa |= __float_as_uint(fj[q] - fi[q]);
    return oa;
}

// one 32-column block against one row block, both directions (ties in f_0)
template <int M, int M4>
__device__ __forceinline__ void block_full(const float* fi, const float* colp, uint32_t& dij, uint32_t& dji)
{
    dij = 0u;
    dji = 0u;
    // columns k = 31 .. 0: the funnel shift leaves column k's bit at position k
#pragma unroll 4
    for (int k = 31; k >= 0; --k) {
        const float4* fj4 = reinterpret_cast<const float4*>(colp + k * M4);
        float fj[M4];
#pragma unroll
        for (int q4 = 0; q4 < M4 / 4; ++q4) {
            const float4 t = fj4[q4];
            fj[4 * q4 + 0] = t.x;
            fj[4 * q4 + 1] = t.y;
            fj[4 * q4 + 2] = t.z;
            fj[4 * q4 + 3] = t.w;
        }
        // sign(f_j - f_i) per objective: 0 if f_i <= f_j, 1 if f_i > f_j
        // (exact FP32 subtraction of finite values; NaN padding gives NaN)
        uint32_t oa = 0u, ob = 0u;
#pragma unroll
        for (int q = 0; q < M; ++q) {
            oa |= __float_as_uint(fj[q] - fi[q]);
            ob |= __float_as_uint(fi[q] - fj[q]);
        }
        // i dom j: no f_i > f_j and some f_i < f_j; j dom i symmetric
        dij = __funnelshift_l(ob & ~oa, dij, 1);
        dji = __funnelshift_l(oa & ~ob, dji, 1);
    }
}

// How a (row block, column block) pair is tested.
enum : int {
    BP_SKIP = 0,   // lower block triangle (done by the transposed tile)
    BP_ZERO,       // no dominance either way: no test, no words
    BP_FAST0,      // only "row dom column": every row f_0 below every column f_0, objectives 1..M-1
    BP_FASTK,      // only "row dom column", objectives 0..M-1
    BP_FASTR,      // only "column dom row", objectives 0..M-1
    BP_FULL        // both directions tested
};

// Per 32-position block of the key order (k_sort.cu): the smallest and
// largest value of every objective (NaN padding ignored; NaN for a block of
// padding only) and the smallest and largest sort key; one warp per block,
// one CTA per 256-position tile, which also records the tile's box and keys.
__global__ void __launch_bounds__(256) k_block_box(RunView v)
{
    __shared__ float slo[8][NSGA3_FAST_M], shi[8][NSGA3_FAST_M];
    __shared__ uint32_t skmin[8], skmax[8];
    if (read_status(v.ctrl)) return;
    const int lane = lane_id(), warp = threadIdx.x >> 5, m = v.m, M4 = v.M4;
    const int b = blockIdx.x * 8 + warp;
    const int p = b * 32 + lane;
    float* box = v.bbox + (size_t)b * 2 * M4;
    for (int q = 0; q < m; ++q) {
        float lo = v.Fp[(size_t)p * m + q], hi = lo;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            box[q] = lo;
            box[M4 + q] = hi;
            slo[warp][q] = lo;
            shi[warp][q] = hi;
        }
    }
    const uint32_t k = v.skey[p];
    const uint32_t kmin = __reduce_min_sync(0xffffffffu, k), kmax = __reduce_max_sync(0xffffffffu, k);
    if (lane == 0) {
        v.bkey[2 * b] = kmin;
        v.bkey[2 * b + 1] = kmax;
        skmin[warp] = kmin;
        skmax[warp] = kmax;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        const int q = threadIdx.x;
        float lo = slo[0][q], hi = shi[0][q];
        for (int w = 1; w < 8; ++w) {
            lo = fminf(lo, slo[w][q]);
            hi = fmaxf(hi, shi[w][q]);
        }
        v.tbox[(size_t)blockIdx.x * 2 * M4 + q] = lo;
        v.tbox[(size_t)blockIdx.x * 2 * M4 + M4 + q] = hi;
    }
    if (threadIdx.x == 32) {
        uint32_t lo = skmin[0], hi = skmax[0];
        for (int w = 1; w < 8; ++w) {
            lo = min(lo, skmin[w]);
            hi = max(hi, skmax[w]);
        }
        v.tkey[2 * blockIdx.x] = lo;
        v.tkey[2 * blockIdx.x + 1] = hi;
    }
}

// The tiles (ti <= tj) whose block pairs can hold a dominance go on a list
// for the dominance build; the rest need no test at all: their bitmap
// bytes stay zero (k_sel_reset clears the bitmap) and their points gain no
// dominator.  One thread per tile, the same tests as a block pair's on the
// tiles' boxes and keys; diagonal tiles are always listed.
template <int M>
__global__ void __launch_bounds__(256) k_tile_plan(RunView v)
{
    constexpr int M4 = (M + 3) & ~3;
    const int T = v.ld / NSGA3_TILE;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    Ctrl* c = v.ctrl;
    if (t >= (long long)T * (T + 1) / 2) return;
    if (read_status(c)) return;
    int ti, tj;
    decode_tile(t, T, ti, tj);
    bool work = ti == tj;
    if (!work && tj * NSGA3_TILE < v.n2) {
        const float* bi = v.tbox + (size_t)ti * 2 * M4;
        const float* bj = v.tbox + (size_t)tj * 2 * M4;
        bool fwd = true, bwd = true;
#pragma unroll
        for (int q = 0; q < M; ++q) {
            fwd = fwd && bi[q] <= bj[M4 + q];
            bwd = bwd && bj[q] <= bi[M4 + q];
        }
        bwd = bwd && !(v.tkey[2 * ti + 1] < v.tkey[2 * tj]);
        work = fwd || bwd;
    }
    if (work)
        v.tlist[atomicAdd(&c->ntile, 1)] = (int32_t)t;
    else
        atomicAdd(&c->domstat[5], 1ull);
}

// Mode of block pair (ib, jb) from the blocks' boxes and keys (warp-wide:
// lane q < M compares objective q).  Row i can dominate column j only if
// f_iq <= f_jq for every q, so some row of I can dominate some column of J
// only if min_I q <= max_J q for every q (fwd), and symmetrically (bwd); when
// a box test fails, some objective separates every pair of the two blocks,
// so their vectors differ and the other direction's dominance needs no
// strictness test.  Dominators never have a larger sort key, so every key
// of I below every key of J also rules out "column dom row".
template <int M>
__device__ __forceinline__ int block_pair_mode(const RunView& v, int ib, int jb)
{
    if (jb < ib) return BP_SKIP;
    if (jb == ib) return BP_FULL;
    if (jb * 32 >= v.n2) return BP_ZERO;  // a column block of padding only
    constexpr int M4 = (M + 3) & ~3;
    const int lane = lane_id();
    const float* bi = v.bbox + (size_t)ib * 2 * M4;
    const float* bj = v.bbox + (size_t)jb * 2 * M4;
    const int q = lane < M ? lane : 0;
    const float imin = bi[q], imax = bi[M4 + q], jmin = bj[q], jmax = bj[M4 + q];
    // NaN boxes (padding only) fail every comparison: no dominance
    const bool fwd = __all_sync(0xffffffffu, lane >= M || imin <= jmax);
    const bool bwd = __all_sync(0xffffffffu, lane >= M || jmin <= imax) && !(v.bkey[2 * ib + 1] < v.bkey[2 * jb]);
    const bool f0sep = __shfl_sync(0xffffffffu, imax < jmin, 0);  // every row f_0 below every column f_0
    if (!fwd && !bwd) return BP_ZERO;
    if (fwd && f0sep) return BP_FAST0;
    if (fwd && !bwd) return BP_FASTK;
    if (!fwd) return BP_FASTR;
    return BP_FULL;
}

// Words of Dom block (dominator block of the word row, 32 columns): written
// only when one of them is nonzero, and the block's bit in dnz records it.
__device__ __forceinline__ void put_block(const RunView& v, size_t at, uint32_t word, unsigned* nzw, int byte, int bit)
{
    if (!__any_sync(0xffffffffu, word != 0u)) return;
    if (!v.streaming) v.Dom[at] = word;
    if (lane_id() == 0 && nzw) atomicOr(&nzw[byte >> 2], 1u << (8 * (byte & 3) + bit));
}

// Position of the (t+1)-th set bit of x (31 when t >= popc(x)): a binary search on
// the popcounts of halving windows.
__device__ __forceinline__ int nth_set_bit(uint32_t x, int t)
{
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int c = __popc((x >> pos) & ((1u << s) - 1u));
        if (t >= c) {
            t -= c;
            pos += s;
        }
    }
    return pos;
}

// Order-preserving map of FP32 to int32 (an involution: the same map turns
// it back): positive values keep their bits, negative ones flip the
// magnitude bits.  INT_MAX maps back to a NaN.
__device__ __forceinline__ int f2s(float x)
{
    const int i = __float_as_int(x);
    return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float s2f(int s) { return __int_as_float(s ^ ((s >> 31) & 0x7fffffff)); }

// Objectives in FP32 pairs: sub.rn.f32x2 forms two exact differences in
// one instruction (each lane rounds once, as the scalar subtraction).
// Columns are loaded from shared memory straight into 64-bit pairs, and
// the sign words are OR-ed three at a time (lop3).
__device__ __forceinline__ unsigned long long p2_pack(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void p2_sub(unsigned long long a, unsigned long long b, uint32_t& lo, uint32_t& hi)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(d));
}
__device__ __forceinline__ uint32_t or3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xFE;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// one column's staged objectives as M4 / 2 pairs (shared-memory byte address)
template <int M4>
__device__ __forceinline__ void lds_col(uint32_t a, unsigned long long (&c)[M4 / 2])
{
#pragma unroll
    for (int q4 = 0; q4 < M4 / 4; ++q4)
        asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(c[2 * q4]), "=l"(c[2 * q4 + 1]) : "r"(a + 16 * q4));
}

// A row's objectives as pairs (p[k] = f_2k, f_2k+1) and the last one alone
// when M is odd.
template <int M>
struct RowPairs {
    unsigned long long p[M / 2];
    float last;
};
template <int M>
__device__ __forceinline__ void make_pairs(RowPairs<M>& r, const float (&f)[M])
{
#pragma unroll
    for (int k = 0; k < M / 2; ++k) r.p[k] = p2_pack(f[2 * k], f[2 * k + 1]);
    r.last = (M & 1) ? f[M - 1] : 0.0f;
}
// sign bit set iff some f_iq > f_jq (f_j - f_i < 0 for some q)
template <int M, int M4>
__device__ __forceinline__ uint32_t any_greater_p(const unsigned long long (&c)[M4 / 2], const RowPairs<M>& r)
{
    constexpr int W = 2 * (M / 2) + (M & 1);
    uint32_t w[W];
#pragma unroll
    for (int k = 0; k < M / 2; ++k) p2_sub(c[k], r.p[k], w[2 * k], w[2 * k + 1]);
    if (M & 1) {
        uint32_t lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(c[M / 2]));
        w[W - 1] = __float_as_uint(__uint_as_float(lo) - r.last);
    }
    uint32_t acc = w[0];
#pragma unroll
    for (int i = 1; i < W; i += 2) acc = (i + 1 < W) ? or3(acc, w[i], w[i + 1]) : (acc | w[i]);
    return acc;
}

// "Some f_iq > f_jq" bits of one or two row lanes against the live columns
// of a block: bit t for the t-th live column, whose shared-memory byte
// address lane t holds in `addr`.
template <int M, int M4, bool TWO>
__device__ __forceinline__ void live_one_dir(const RowPairs<M>& r0, const RowPairs<M>& r1, uint32_t addr, int nl,
                                             uint32_t& acc0, uint32_t& acc1)
{
    acc0 = 0u;
    acc1 = 0u;
#pragma unroll 2
    for (int t = nl - 1; t >= 0; --t) {
        unsigned long long c[M4 / 2];
        lds_col<M4>(__shfl_sync(0xffffffffu, addr, t), c);
        acc0 = __funnelshift_l(any_greater_p<M, M4>(c, r0), acc0, 1);
        if (TWO) acc1 = __funnelshift_l(any_greater_p<M, M4>(c, r1), acc1, 1);
    }
}

template <int M, int M4>
__device__ __forceinline__ void load_row(float (&f)[M], const float* p)
{
    const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int q4 = 0; q4 < M4 / 4; ++q4) {
        const float4 x = p4[q4];
        if (4 * q4 + 0 < M) f[4 * q4 + 0] = x.x;
        if (4 * q4 + 1 < M) f[4 * q4 + 1] = x.y;
        if (4 * q4 + 2 < M) f[4 * q4 + 2] = x.z;
        if (4 * q4 + 3 < M) f[4 * q4 + 3] = x.w;
    }
}

// One-direction entry, "row dominates column": row block ib (and ib + 1
// when `two`) against column block jb, lane = row.  The test is "no
// f_iq > f_jq" over every objective (when every row f_0 is below every
// column f_0, objective 0 never sets a sign and strictness is implied;
// otherwise some objective separates the blocks, so the vectors differ).
// Before any pairwise test the entry narrows both sides:
//  - a row can dominate some column of J only if f_iq <= max_J q for every
//    q (the column block's box); the other rows are dead (NaN padding rows
//    fail too);
//  - a column j can be dominated by a live row only if
//    min over live rows of f_iq <= f_jq for every q; the other columns are
//    dead (NaN padding columns fail too).
// Only live columns are tested (the warp walks them in order, each column
// broadcast from shared memory); with two row blocks the live rows are
// packed onto the lanes when they fit in one warp, otherwise each lane
// tests its row of both blocks.  The bits come back in place by
// shuffles: row words through the packing slots, column words through the
// live columns' ranks after the transpose.  `ev` counts the (lane, column)
// pairs tested in units of 32, `lv` the (live row, live column) pairs among
// them.
template <int M, int M4>
__device__ __forceinline__ void entry_row_dom_col(const RunView& v, const float* srow, const float* colp,
                                                  const float* cbox, int ri, bool two, int ib, int jb, int cb,
                                                  unsigned* nz, int* ccnt, uint32_t& ev, uint32_t& lv)
{
    const int lane = lane_id();
    const uint32_t lt = (1u << lane) - 1u;
    float f0[M], f1[M];
    load_row<M, M4>(f0, srow + (ri * 32 + lane) * M4);
    if (two) {
        load_row<M, M4>(f1, srow + ((ri + 1) * 32 + lane) * M4);
    } else {
#pragma unroll
        for (int q = 0; q < M; ++q) f1[q] = f0[q];
    }
    float h[M];
    load_row<M, M4>(h, cbox + M4);  // the column block's maxima
    bool l0 = true, l1 = two;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        l0 = l0 && f0[q] <= h[q];
        l1 = l1 && f1[q] <= h[q];
    }
    // column test against the per-objective minimum of the live rows (no
    // live row: the minimum is NaN and every column is dead)
    float cj[M];
    load_row<M, M4>(cj, colp + lane * M4);
    // (every lane takes part in every reduction and vote: none sits in a
    // condition that differs between lanes).  No live row: nothing to test.
    // With more than six objectives a vote after the first five ends the
    // entry early when no column is left (most entries that end without a
    // live column do so by then).
    const bool anyl = l0 || l1;
    if (!__any_sync(0xffffffffu, anyl)) return;
    bool cl = true;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        const float fm = fminf(l0 ? f0[q] : __int_as_float(0x7f800000), l1 ? f1[q] : __int_as_float(0x7f800000));
        const float lmin = s2f(__reduce_min_sync(0xffffffffu, anyl ? f2s(fm) : 0x7fffffff));
        cl = cl && lmin <= cj[q];
        if (M > 6 && q == 4 && !__any_sync(0xffffffffu, cl)) return;
    }
    const uint32_t live = __ballot_sync(0xffffffffu, cl);
    if (!live) return;
    const int nl = __popc(live);
    const uint32_t low = nl == 32 ? 0xffffffffu : (1u << nl) - 1u;
    // lane t < nl: shared-memory byte address of the t-th live column (every
    // lane searches, without a branch; lanes from nl on get a column of the
    // block that is never read)
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(colp) + (uint32_t)nth_set_bit(live, lane) * (uint32_t)(M4 * 4);
    const uint32_t b0 = __ballot_sync(0xffffffffu, l0);
    const uint32_t b1 = __ballot_sync(0xffffffffu, l1);
    const int n0 = __popc(b0), nr = n0 + __popc(b1);
    uint32_t d0, d1;
    if (!two || nr <= 32) {
        // one row per lane: the entry's row block as it is, or the live rows
        // of both blocks packed onto the lanes (block ib first)
        float fp[M];
        const bool first = lane < n0;
        if (two) {
            // (lanes from nr on find no set bit and get row 31 of the second
            // block, whose result is never read)
            const int src = nth_set_bit(first ? b0 : b1, first ? lane : lane - n0);
            load_row<M, M4>(fp, srow + ((ri + (first ? 0 : 1)) * 32 + src) * M4);
        } else {
#pragma unroll
            for (int q = 0; q < M; ++q) fp[q] = f0[q];
        }
        RowPairs<M> rp;
        make_pairs<M>(rp, fp);
        uint32_t acc, unused;
        live_one_dir<M, M4, false>(rp, rp, addr, nl, acc, unused);
        const uint32_t R = ~acc & low;
        if (two) {
            const uint32_t r0 = __shfl_sync(0xffffffffu, R, __popc(b0 & lt));
            const uint32_t r1 = __shfl_sync(0xffffffffu, R, (n0 + __popc(b1 & lt)) & 31);
            d0 = l0 ? r0 : 0u;
            d1 = l1 ? r1 : 0u;
        } else {
            d0 = l0 ? R : 0u;
            d1 = 0u;
        }
        ev += nl;
    } else {
        RowPairs<M> rp0, rp1;
        make_pairs<M>(rp0, f0);
        make_pairs<M>(rp1, f1);
        uint32_t acc0, acc1;
        live_one_dir<M, M4, true>(rp0, rp1, addr, nl, acc0, acc1);
        d0 = l0 ? ~acc0 & low : 0u;
        d1 = l1 ? ~acc1 & low : 0u;
        ev += 2 * nl;
    }
    lv += nr * nl;
    // column words: lane t of the transpose holds the t-th live column (with
    // two row blocks and at most 16 live columns one transpose serves both:
    // lanes 0..15 the first block, 16..31 the second)
    const int rk = __popc(live & lt);
    const bool mine = (live >> lane) & 1u;
    uint32_t w0, w1 = 0u;
    if (two && nl <= 16) {
        const uint32_t tw = warp_transpose32(d0 | (d1 << 16));
        w0 = __shfl_sync(0xffffffffu, tw, rk & 15);
        w1 = __shfl_sync(0xffffffffu, tw, 16 + (rk & 15));
    } else {
        w0 = __shfl_sync(0xffffffffu, warp_transpose32(d0), rk & 31);
        if (two) w1 = __shfl_sync(0xffffffffu, warp_transpose32(d1), rk & 31);
    }
    w0 = mine ? w0 : 0u;
    w1 = mine ? w1 : 0u;
    put_block(v, (size_t)ib * v.ld + jb * 32 + lane, w0, nz, ri, cb);
    int cc = __popc(w0);
    if (two) {
        put_block(v, (size_t)(ib + 1) * v.ld + jb * 32 + lane, w1, nz, ri + 1, cb);
        cc += __popc(w1);
    }
    if (cc) atomicAdd(&ccnt[cb * 32 + lane], cc);
}

// Asynchronous copies into shared memory (cp.async: the data lands while
// the CTA keeps working; wait_all + a barrier make it visible to all).
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared memory of k_dominance (dynamic): two buffers, each holding a
// tile's 256 row points, 256 column points (M4 floats each) and its 16
// block boxes and key ranges.
template <int M>
__host__ __device__ constexpr size_t dom_buf_floats()
{
    return (size_t)2 * NSGA3_TILE * ((M + 3) & ~3) + 16 * 2 * ((M + 3) & ~3) + 16 * 2;
}
template <int M>
__host__ __device__ constexpr size_t dom_smem_bytes()
{
    return 2 * dom_buf_floats<M>() * sizeof(float);
}

// A CTA takes 256 x 256 tiles of the upper block triangle (8 x 8 blocks of
// 32) from the tile list, two at a time in flight: while its warps test the
// block pairs of one tile, the points of its next tile are copied into the
// other buffer (cp.async), and warp 0 first copies the next tile's 16 block
// boxes and key ranges itself, decides its 64 block pairs from them and
// puts the pairs to test on the next work list, then joins the tests.  Two
// row blocks (2r, 2r + 1) that take the same one-direction test against one
// column block form a single entry (one column broadcast from shared memory
// then serves 64 pairs), and the costlier entries (both-way tests, row
// pairs) come first; the warps take entries from a shared counter, so
// block pairs of very different cost after the pruning balance over the
// warps.  One barrier per tile: after it the threads flush the finished
// tile's dominator counts and bitmap bytes (both kept per buffer) and go on
// to the next tile.  Per entry the lanes hold their rows' objectives in
// registers.
template <int M>
__global__ void __launch_bounds__(256, M <= 8 ? 5 : 4) k_dominance(RunView v)
{
    constexpr int M4 = (M + 3) & ~3;
    constexpr size_t BUF = dom_buf_floats<M>();
    extern __shared__ __align__(16) float dsm[];
    __shared__ unsigned char smode[64];
    __shared__ int rowcnt[2][NSGA3_TILE];  // per buffer: dominators found for the tile's row points
    __shared__ int colcnt[2][NSGA3_TILE];  // ... for its column points
    __shared__ unsigned nzw[2][4];         // per buffer, dnz bytes: 0..7 row blocks (I, J), 8..15 column blocks (J, I)
    // entries: (mode << 7) | (pair << 6) | (row block << 3) | column block
    __shared__ unsigned short work[2][64];
    __shared__ int nheavy[2], nlight[2];   // heavy entries from the front, light ones from the back
    __shared__ int taken[2];               // entries handed out
    __shared__ unsigned long long stat[2]; // pairs tested (units of 32), live pairs
    if (read_status(v.ctrl)) return;
    const int T = v.ld / NSGA3_TILE;
    const int ntile = *(volatile const int32_t*)&v.ctrl->ntile;
    if ((int)blockIdx.x >= ntile) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    auto srow_of = [&](int buf) { return dsm + buf * BUF; };
    auto scol_of = [&](int buf) { return dsm + buf * BUF + NSGA3_TILE * M4; };
    auto sbox_of = [&](int buf) { return dsm + buf * BUF + 2 * NSGA3_TILE * M4; };  // [16][2 M4]
    auto skey_of = [&](int buf) {
        return reinterpret_cast<uint32_t*>(dsm + buf * BUF + 2 * NSGA3_TILE * M4 + 16 * 2 * M4);  // [16][2]
    };
    // the points of tile (ti, tj) into buffer `buf` (every thread its share);
    // Fp holds -0.0 as +0.0, so equal values subtract to +0.0
    auto copy_points = [&](int ti, int tj, int buf) {
        float* dr = srow_of(buf);
        float* dc = scol_of(buf);
        const float* gr = v.Fp + (size_t)ti * NSGA3_TILE * M;
        const float* gc = v.Fp + (size_t)tj * NSGA3_TILE * M;
        for (int e = tid; e < NSGA3_TILE * M; e += blockDim.x) {
            const int p = e / M, q = e - p * M;
            cp_async4(dr + p * M4 + q, gr + e);
            cp_async4(dc + p * M4 + q, gc + e);
        }
        cp_async_commit();
    };
    // warp 0: the boxes and keys of tile (ti, tj) into buffer `buf`, waited for
    // (a warp's own copies), then the modes of its 64 block pairs (see
    // block_pair_mode for the tests) and its work list
    auto decide = [&](int ti, int tj, int buf) {
        float* sb = sbox_of(buf);
        uint32_t* sk = skey_of(buf);
        for (int e = lane; e < 16 * (2 * M4 / 4); e += 32) {
            const int b = e / (2 * M4 / 4), k4 = e - b * (2 * M4 / 4);
            const int blk = b < 8 ? ti * 8 + b : tj * 8 + (b - 8);
            cp_async16(sb + b * 2 * M4 + 4 * k4, v.bbox + (size_t)blk * 2 * M4 + 4 * k4);
        }
        if (lane < 16) {
            const int blk = lane < 8 ? ti * 8 + lane : tj * 8 + (lane - 8);
            cp_async8(sk + 2 * lane, v.bkey + 2 * (size_t)blk);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
        unsigned cnt5 = 0u;  // lane q < 5: block pairs of mode q + 1
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int pidx = lane + 32 * h;
            const int ri = pidx >> 3, cb = pidx & 7;
            const int ib = ti * 8 + ri, jb = tj * 8 + cb;
            int mode;
            if (jb < ib)
                mode = BP_SKIP;
            else if (jb == ib)
                mode = BP_FULL;
            else if (jb * 32 >= v.n2)
                mode = BP_ZERO;  // a column block of padding only
            else {
                const float* bi = sb + ri * 2 * M4;
                const float* bj = sb + (8 + cb) * 2 * M4;
                bool fwd = true, bwd = true;
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    fwd = fwd && bi[q] <= bj[M4 + q];  // NaN (padding only) fails
                    bwd = bwd && bj[q] <= bi[M4 + q];
                }
                bwd = bwd && !(sk[2 * ri + 1] < sk[2 * (8 + cb)]);
                const bool f0sep = bi[M4] < bj[0];
                mode = (!fwd && !bwd) ? BP_ZERO
                       : (fwd && f0sep) ? BP_FAST0
                       : (fwd && !bwd)  ? BP_FASTK
                       : !fwd           ? BP_FASTR
                                        : BP_FULL;
            }
            smode[pidx] = (unsigned char)mode;
#pragma unroll
            for (int md = 1; md <= 5; ++md) {
                const unsigned c = __popc(__ballot_sync(0xffffffffu, mode == md));
                if (lane == md - 1) cnt5 += c;
            }
        }
        if (lane < 5 && cnt5) atomicAdd(&v.ctrl->domstat[lane], (unsigned long long)cnt5);
        __syncwarp();
        // row pair rp = (2 rp, 2 rp + 1) against column block cb
        const int rp = lane >> 3, cb = lane & 7;
        const int a = smode[(2 * rp) * 8 + cb], b = smode[(2 * rp + 1) * 8 + cb];
        const bool pair = a == b && (a == BP_FAST0 || a == BP_FASTK);
        const int hcnt = pair ? 1 : (a == BP_FULL) + (b == BP_FULL);
        const int lcnt = pair ? 0 : (a > BP_ZERO && a != BP_FULL) + (b > BP_ZERO && b != BP_FULL);
        int hoff = hcnt, loff = lcnt;  // inclusive scans over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, hoff, o);
            const int y = __shfl_up_sync(0xffffffffu, loff, o);
            if (lane >= o) {
                hoff += x;
                loff += y;
            }
        }
        const int htot = __shfl_sync(0xffffffffu, hoff, 31), ltot = __shfl_sync(0xffffffffu, loff, 31);
        hoff -= hcnt;
        loff -= lcnt;
        if (pair) {
            work[buf][hoff] = (unsigned short)((a << 7) | (1 << 6) | ((2 * rp) << 3) | cb);
        } else {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int md = r ? b : a;
                const unsigned short e = (unsigned short)((md << 7) | ((2 * rp + r) << 3) | cb);
                if (md == BP_FULL)
                    work[buf][hoff++] = e;
                else if (md > BP_ZERO)
                    work[buf][63 - loff++] = e;
            }
        }
        if (lane == 0) {
            nheavy[buf] = htot;
            nlight[buf] = ltot;
            taken[buf] = 0;
        }
    };

    int cur = 0;
    int it = blockIdx.x;
    int ti, tj;
    uint32_t ev = 0u, lv = 0u;  // this tile's pairs tested (units of 32) and live pairs (warp-uniform)
    decode_tile(v.tlist[it], T, ti, tj);
    copy_points(ti, tj, 0);
    rowcnt[0][tid] = 0;
    colcnt[0][tid] = 0;
    rowcnt[1][tid] = 0;
    colcnt[1][tid] = 0;
    if (tid < 8) nzw[tid >> 2][tid & 3] = 0u;
    if (tid < 2) stat[tid] = 0ull;
    if (warp == 0) decide(ti, tj, 0);
    cp_async_wait_all();
    __syncthreads();
    for (;;) {
        const int nit = it + gridDim.x;
        const bool more = nit < ntile;
        int nti = ti, ntj = tj;
        if (more) {
            decode_tile(v.tlist[nit], T, nti, ntj);
            copy_points(nti, ntj, cur ^ 1);  // the other buffer's tile was finished a tile ago
            if (warp == 0) decide(nti, ntj, cur ^ 1);
        }
        const int nh = nheavy[cur], nl = nlight[cur], nwork = nh + nl;
        unsigned* nz = v.dnz ? nzw[cur] : nullptr;
        const float* srow = srow_of(cur);
        const float* scol = scol_of(cur);
        int* rcnt = rowcnt[cur];
        int* ccnt = colcnt[cur];
        for (;;) {
            int t = 0;
            if (lane == 0) t = atomicAdd(&taken[cur], 1);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= nwork) break;
            const unsigned e = work[cur][t < nh ? t : 64 - nwork + t];
            const int mode = e >> 7, two = (e >> 6) & 1, ri = (e >> 3) & 7, cb = e & 7;
            const int ib = ti * 8 + ri, jb = tj * 8 + cb;
            const float* colp = scol + cb * 32 * M4;
            // One direction only: "no f_iq > f_jq" (or the reverse) decides,
            // and a NaN padding point would pass it (its differences are
            // NaN with a clear sign bit), so the bits of padding rows and
            // columns are masked (the two-way test needs no mask: a NaN
            // gives the same sign both ways, hence no bit).
            const int cv = v.n2 - jb * 32;
            const uint32_t colvalid = cv >= 32 ? 0xffffffffu : (cv > 0 ? (1u << cv) - 1u : 0u);
            if (mode == BP_FAST0 || mode == BP_FASTK) {
                // "row dominates column" only, one row block or two
                const float* cbox = sbox_of(cur) + (8 + cb) * 2 * M4;
                entry_row_dom_col<M, M4>(v, srow, colp, cbox, ri, two, ib, jb, cb, nz, ccnt, ev, lv);
                continue;
            }
            ev += 32u;
            lv += 1024u;
            float fi[M];
#pragma unroll
            for (int q = 0; q < M; ++q) fi[q] = srow[(ri * 32 + lane) * M4 + q];
            uint32_t dij = 0u, dji = 0u;
            if (mode == BP_FASTR) {
                // column j dominates row i: no f_jq > f_iq (the vectors differ)
                const bool rowvalid = ib * 32 + lane < v.n2;
                uint32_t acc = 0u;
#pragma unroll 4
                for (int k = 31; k >= 0; --k) {
                    const float* fj = colp + k * M4;
                    acc = __funnelshift_l(any_greater<0, M>(fi, fj), acc, 1);
                }
                dji = rowvalid ? ~acc & colvalid : 0u;
            } else {
                block_full<M, M4>(fi, colp, dij, dji);
            }
            // column i = ib*32 + lane, dominators j in block jb: Dom block (jb, ib)
            if (jb != ib) {
                put_block(v, (size_t)jb * v.ld + ib * 32 + lane, dji, nz, 8 + cb, ri);
                const uint32_t tr = warp_transpose32(dij);
                put_block(v, (size_t)ib * v.ld + jb * 32 + lane, tr, nz, ri, cb);
                if (tr) atomicAdd(&ccnt[cb * 32 + lane], __popc(tr));
            } else {
                put_block(v, (size_t)jb * v.ld + ib * 32 + lane, dji, nz, ri, cb);
            }
            if (dji) atomicAdd(&rcnt[ri * 32 + lane], __popc(dji));
        }
        if (lane == 0 && ev) {
            atomicAdd(&stat[0], (unsigned long long)ev);
            atomicAdd(&stat[1], (unsigned long long)lv);
        }
        ev = 0u;
        lv = 0u;
        cp_async_wait_all();
        __syncthreads();  // the tile's tests are done, the next tile is staged and decided
        if (warp == 0) {
            // this tile owns bytes dnz[I][tj] (I a row block) and dnz[J][ti] (J a
            // column block), one byte each; on the diagonal they are the same
            // bytes.  Lane 0 reads and clears the buffer's words (no other
            // thread touches them before the buffer's next tile, a barrier later).
            unsigned long long lo = 0ull, hi = 0ull;  // bytes 0..7 and 8..15
            if (lane == 0) {
                lo = (unsigned long long)nzw[cur][0] | ((unsigned long long)nzw[cur][1] << 32);
                hi = (unsigned long long)nzw[cur][2] | ((unsigned long long)nzw[cur][3] << 32);
#pragma unroll
                for (int k = 0; k < 4; ++k) nzw[cur][k] = 0u;
            }
            lo = __shfl_sync(0xffffffffu, lo, 0);
            hi = __shfl_sync(0xffffffffu, hi, 0);
            if (v.dnz) {
                const int b8 = 8 * (lane & 7);
                const unsigned char rb = (unsigned char)(lo >> b8), cbyte = (unsigned char)(hi >> b8);
                if (lane < 8) {
                    const unsigned char x = (ti == tj) ? (unsigned char)(rb | cbyte) : rb;
                    v.dnz[(size_t)(ti * 8 + lane) * v.NB8 + tj] = x;
                } else if (lane < 16 && ti != tj) {
                    v.dnz[(size_t)(tj * 8 + (lane - 8)) * v.NB8 + ti] = cbyte;
                }
            }
        }
        // dominator counts of the peel's first pass: one global add per point of the tile
        {
            const int rc = rcnt[tid], cc = ccnt[tid];
            if (rc) atomicAdd(&v.cnt[ti * NSGA3_TILE + tid], rc);
            if (cc) atomicAdd(&v.cnt[tj * NSGA3_TILE + tid], cc);
            rcnt[tid] = 0;
            ccnt[tid] = 0;
        }
        if (!more) break;
        cur ^= 1;
        it = nit;
        ti = nti;
        tj = ntj;
    }
    if (tid == 0 && stat[0]) {
        atomicAdd(&v.ctrl->domstat[6], 32ull * stat[0]);
        atomicAdd(&v.ctrl->domstat[7], stat[1]);
    }
}

// m > NSGA3_FAST_M: the objectives are taken in chunks of MC (zero-padded:
// a zero difference has a clear sign bit and changes neither mask).  Each
// lane keeps, per row and column block, the 32-bit masks A ("some
// f_i > f_j") and B ("some f_j > f_i") OR-ed over the chunks; the bits
// follow from them as in the specialised kernel.  With v.dom_ks > 1 the
// chunks of a tile are split over gridDim.y CTAs that OR their masks into
// dpa / dpb, and k_dom_finish forms the bits.
constexpr int MC = 16;

// one-direction test of row block ib against column block jb (warp-wide):
// every f_i0 of the rows below every f_j0 of the columns
__device__ __forceinline__ bool one_direction(const RunView& v, int ib, int jb)
{
    float rmax = v.Fp[(size_t)(ib * 32 + lane_id()) * v.m];
    float cmin = v.Fp[(size_t)(jb * 32 + lane_id()) * v.m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        cmin = fminf(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
    }
    return jb > ib && rmax < cmin;
}

__global__ void __launch_bounds__(256) k_dominance_gen(RunView v)
{
    __shared__ __align__(16) float srow[NSGA3_TILE * MC];
    __shared__ __align__(16) float scol[NSGA3_TILE * MC];
    __shared__ int s_tile[2];
    __shared__ int rowcnt[NSGA3_TILE];
    __shared__ int colcnt[NSGA3_TILE];
    if (read_status(v.ctrl)) return;
    const int m = v.m;
    rowcnt[threadIdx.x] = 0;
    colcnt[threadIdx.x] = 0;
    const int T = v.ld / NSGA3_TILE;
    if (threadIdx.x == 0) decode_tile(blockIdx.x, T, s_tile[0], s_tile[1]);
    __syncthreads();
    const int ti = s_tile[0], tj = s_tile[1];
    const int r0 = ti * NSGA3_TILE, c0 = tj * NSGA3_TILE;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int rp = warp & 3, ch = warp >> 2;
    const int ib0 = ti * 8 + 2 * rp, ib1 = ib0 + 1;
    // one-direction blocks from f_0 alone (as in the specialised kernel)
    unsigned fastm = 0u;  // bit 2*cbi + r: one-direction block
#pragma unroll
    for (int cbi = 0; cbi < 4; ++cbi) {
        const int jb = tj * 8 + ch * 4 + cbi;
        if (one_direction(v, ib0, jb)) fastm |= 1u << (2 * cbi);
        if (one_direction(v, ib1, jb)) fastm |= 2u << (2 * cbi);
    }
    uint32_t A[4][2], B[4][2];
#pragma unroll
    for (int cbi = 0; cbi < 4; ++cbi) {
        A[cbi][0] = A[cbi][1] = 0u;
        B[cbi][0] = B[cbi][1] = 0u;
    }
    // objective range of this CTA: all of them, or its share of the chunks
    const int nch = (m + MC - 1) / MC, per = (nch + gridDim.y - 1) / gridDim.y;
    const int qbeg = blockIdx.y * per * MC, qend = min(m, qbeg + per * MC);
    for (int q0 = qbeg; q0 < qend; q0 += MC) {
        __syncthreads();  // the previous chunk is consumed
#pragma unroll 4
        for (int e = threadIdx.x; e < NSGA3_TILE * MC; e += blockDim.x) {
            const int p = e / MC, q = q0 + (e - p * MC);
            srow[e] = q < m ? v.Fp[(size_t)(r0 + p) * m + q] : 0.0f;
            scol[e] = q < m ? v.Fp[(size_t)(c0 + p) * m + q] : 0.0f;
        }
        __syncthreads();
        float f0[MC], f1[MC];
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            f0[q] = srow[(2 * rp * 32 + lane) * MC + q];
            f1[q] = srow[((2 * rp + 1) * 32 + lane) * MC + q];
        }
#pragma unroll
        for (int cbi = 0; cbi < 4; ++cbi) {
            const int cb = ch * 4 + cbi;
            const int jb = tj * 8 + cb;
            if (jb < ib0) continue;
            if (jb * 32 >= v.n2) continue;  // padding only: the masks stay 0, no bit
            const float* colp = scol + cb * 32 * MC;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (jb < ib0 + r) continue;
                const float* fi = r ? f1 : f0;
                const bool fast = (fastm >> (2 * cbi + r)) & 1u;
                uint32_t ma = 0u, mb = 0u;
#pragma unroll 4
                for (int k = 31; k >= 0; --k) {
                    const float4* fj4 = reinterpret_cast<const float4*>(colp + k * MC);
                    float fj[MC];
#pragma unroll
                    for (int q4 = 0; q4 < MC / 4; ++q4) {
                        const float4 t = fj4[q4];
                        fj[4 * q4 + 0] = t.x;
                        fj[4 * q4 + 1] = t.y;
                        fj[4 * q4 + 2] = t.z;
                        fj[4 * q4 + 3] = t.w;
                    }
                    uint32_t oa = 0u, ob = 0u;
                    if (fast) {  // f_j0 > f_i0 for the whole block: "some f_j > f_i" holds
#pragma unroll
                        for (int q = 0; q < MC; ++q) oa |= __float_as_uint(fj[q] - fi[q]);
                    } else {
#pragma unroll
                        for (int q = 0; q < MC; ++q) {
                            oa |= __float_as_uint(fj[q] - fi[q]);
                            ob |= __float_as_uint(fi[q] - fj[q]);
                        }
                    }
                    ma = __funnelshift_l(oa, ma, 1);
                    mb = __funnelshift_l(ob, mb, 1);
                }
                A[cbi][r] |= ma;
                B[cbi][r] |= mb;
            }
        }
    }
    if (gridDim.y > 1) {  // partial masks: OR-ed over the CTAs of the tile
#pragma unroll
        for (int cbi = 0; cbi < 4; ++cbi) {
            const int jb = tj * 8 + ch * 4 + cbi;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int ib = ib0 + r;
                if (jb < ib) continue;
                const size_t at = (size_t)jb * v.ld + ib * 32 + lane;
                if (A[cbi][r]) atomicOr(&v.dpa[at], A[cbi][r]);
                if (B[cbi][r]) atomicOr(&v.dpb[at], B[cbi][r]);
            }
        }
        return;
    }
    uint32_t* D = v.Dom;
    int rc0 = 0, rc1 = 0;
#pragma unroll
    for (int cbi = 0; cbi < 4; ++cbi) {
        const int cb = ch * 4 + cbi;
        const int jb = tj * 8 + cb;
        if (jb < ib0) continue;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int ib = ib0 + r;
            if (jb < ib) continue;
            const bool fast = (fastm >> (2 * cbi + r)) & 1u;
            // i dom j: no f_i > f_j and some f_j > f_i (B is implied in a fast block)
            const uint32_t dij = fast ? ~A[cbi][r] : (B[cbi][r] & ~A[cbi][r]);
            const uint32_t dji = fast ? 0u : (A[cbi][r] & ~B[cbi][r]);
            if (!v.streaming) D[(size_t)jb * v.ld + ib * 32 + lane] = dji;
            if (r)
                rc1 += __popc(dji);
            else
                rc0 += __popc(dji);
            if (jb != ib) {
                const uint32_t t = warp_transpose32(dij);
                if (!v.streaming) D[(size_t)ib * v.ld + jb * 32 + lane] = t;
                if (t) atomicAdd(&colcnt[cb * 32 + lane], __popc(t));
            }
        }
    }
    if (rc0) atomicAdd(&rowcnt[2 * rp * 32 + lane], rc0);
    if (rc1) atomicAdd(&rowcnt[(2 * rp + 1) * 32 + lane], rc1);
    __syncthreads();
    const int t = threadIdx.x;
    if (rowcnt[t]) atomicAdd(&v.cnt[r0 + t], rowcnt[t]);
    if (colcnt[t]) atomicAdd(&v.cnt[c0 + t], colcnt[t]);
}

// bits of block pair (ib, jb >= ib) from the OR-ed masks (warp per pair);
// the masks are cleared for the next selection
__global__ void __launch_bounds__(256) k_dom_finish(RunView v)
{
    if (read_status(v.ctrl)) return;
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int NW = v.NW;
    if (t >= (long long)NW * (NW + 1) / 2) return;
    int ib, jb;
    decode_tile(t, NW, ib, jb);
    const int lane = lane_id();
    const size_t at = (size_t)jb * v.ld + ib * 32 + lane;
    const uint32_t a = v.dpa[at], b = v.dpb[at];
    v.dpa[at] = 0u;
    v.dpb[at] = 0u;
    const bool fast = one_direction(v, ib, jb);
    const uint32_t dij = fast ? ~a : (b & ~a);
    const uint32_t dji = fast ? 0u : (a & ~b);
    v.Dom[at] = dji;
    if (dji) atomicAdd(&v.cnt[ib * 32 + lane], __popc(dji));
    if (jb != ib) {
        const uint32_t tr = warp_transpose32(dij);
        v.Dom[(size_t)ib * v.ld + jb * 32 + lane] = tr;
        if (tr) atomicAdd(&v.cnt[jb * 32 + lane], __popc(tr));
    }
}

template <int M>
cudaError_t launch_dom_m(const RunView& v, cudaStream_t s)
{
    long long T = v.ld / NSGA3_TILE;
    long long tiles = T * (T + 1) / 2;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_block_box<<<(unsigned)T, 256, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tile_plan<M><<<(unsigned)((tiles + 255) / 256), 256, 0, s>>>(v);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // persistent CTAs over the listed tiles, as many as are resident at once
    static int occ = 0;  // per M; the same value whatever the run
    if (occ <= 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dominance<M>, 256,
                                                                  dom_smem_bytes<M>()) != cudaSuccess) {
        cudaGetLastError();
        occ = 4;
    }
    int per_sm = occ > 0 ? occ : 4;
    if (v.dom_ctas > 0 && v.dom_ctas < per_sm) per_sm = v.dom_ctas;  // launch-shape option
    long long grid = (long long)per_sm * v.num_sms;
    if (grid > tiles) grid = tiles;
    k_dominance<M><<<(unsigned)grid, 256, dom_smem_bytes<M>(), s>>>(v);
    return cudaGetLastError();
}

}  // namespace

template <int M>
cudaError_t dom_attr_m()
{
    return cudaFuncSetAttribute(k_dominance<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dom_smem_bytes<M>());
}

cudaError_t dom_init_attributes()
{
    cudaError_t e = dom_attr_m<2>();
    if (e == cudaSuccess) e = dom_attr_m<3>();
    if (e == cudaSuccess) e = dom_attr_m<4>();
    if (e == cudaSuccess) e = dom_attr_m<5>();
    if (e == cudaSuccess) e = dom_attr_m<6>();
    if (e == cudaSuccess) e = dom_attr_m<7>();
    if (e == cudaSuccess) e = dom_attr_m<8>();
    if (e == cudaSuccess) e = dom_attr_m<9>();
    if (e == cudaSuccess) e = dom_attr_m<10>();
    return e;
}

cudaError_t launch_dominance(const RunView& v, cudaStream_t s)
{
    switch (v.m) {
    case 2: return launch_dom_m<2>(v, s);
    case 3: return launch_dom_m<3>(v, s);
    case 4: return launch_dom_m<4>(v, s);
    case 5: return launch_dom_m<5>(v, s);
    case 6: return launch_dom_m<6>(v, s);
    case 7: return launch_dom_m<7>(v, s);
    case 8: return launch_dom_m<8>(v, s);
    case 9: return launch_dom_m<9>(v, s);
    case 10: return launch_dom_m<10>(v, s);
    default: break;
    }
    if (v.m < 2 || v.m > NSGA3_MAX_M) return cudaErrorInvalidValue;
    const long long T = v.ld / NSGA3_TILE;
    const long long tiles = T * (T + 1) / 2;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int ks = v.dom_ks > 1 ? v.dom_ks : 1;
    k_dominance_gen<<<dim3((unsigned)tiles, ks), 256, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || ks == 1) return e;
    const long long pairs = (long long)v.NW * (v.NW + 1) / 2;
    k_dom_finish<<<(unsigned)((pairs * 32 + 255) / 256), 256, 0, s>>>(v);
    return cudaGetLastError();
}
