// k_niche.cu -- niche selection of K = N - |S| members of F_l (the niching
// loop of Alg. 1; its cached batched form in Alg. 2).
//
// The paper's loop takes, round after round, one member from every
// reference of minimum niche count (the cache tensor Q and cursor s of
// Alg. 2 serve whole rounds at once) and truncates the last round in
// shuffled-reference order.  Rounds are exhausted level by level, so the
// outcome has a closed form that needs no loop:
//   each reference j orders its F_l members: the nearest first (min d, then
//   lowest index) when rho_j = 0, then by ascending Philox member priority
//   (then index); the member at position t has level rho_j + t;
//   L* = min { L : sum_j min(rho'_j, max(0, L + 1 - rho_j)) >= K };
//   every member of level < L* is taken, and of the references holding a
//   level-L* member, the r = K - count(L* - 1) of smallest (ref priority, j)
//   take that member.
// Random choices use fixed Philox priorities of this generation: reference
// j -> word 0 of Philox(j, gen, 4, 0), member i -> word 0 of
// Philox(i, gen, 5, 0); ties go to the lower index.
#include "kernels.cuh"

namespace {

constexpr int LB = 1024;    // threads of the single-CTA kernels
constexpr int LCAP = 4096;  // niche levels resolved by the shared histogram
constexpr int EXACT = 1024; // candidates ranked pairwise in the last select phase
constexpr int CKCAP = 4096; // level-L* reference keys staged in shared memory
constexpr int RRCAP = 12288; // references whose (rho, rho') are staged in shared memory

__device__ __forceinline__ uint32_t mem_prio(uint64_t seed, uint32_t gen, int i)
{
    return philox((uint32_t)i, gen, RNG_MEMPRIO, 0u, seed).x;
}

__device__ __forceinline__ unsigned long long ref_key(uint64_t seed, uint32_t gen, int j)
{
    return ((unsigned long long)philox((uint32_t)j, gen, RNG_REFPRIO, 0u, seed).x << 32) | (unsigned)j;
}

// ------------------------------------------------ block-wide helpers -------
__device__ int block_sum(int x, int* scratch)
{
    x = warp_sum(x);
    if (lane_id() == 0) scratch[threadIdx.x >> 5] = x;
    __syncthreads();
    int t = 0;
    if (threadIdx.x < 32) {
        t = (threadIdx.x < (blockDim.x >> 5)) ? scratch[threadIdx.x] : 0;
        t = warp_sum(t);
        if (threadIdx.x == 0) scratch[32] = t;
    }
    __syncthreads();
    t = scratch[32];
    __syncthreads();
    return t;
}

// exclusive scan of one value per thread; returns the prefix, *total the sum
__device__ int block_excl_scan(int x, int* scratch, int* total)
{
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int v = (lane < (int)(blockDim.x >> 5)) ? scratch[lane] : 0;
        int vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += y;
        }
        scratch[lane] = vi - v;
        if (lane == 31) scratch[32] = vi;
    }
    __syncthreads();
    const int res = scratch[warp] + inc - x;
    *total = scratch[32];
    __syncthreads();
    return res;
}

// Exclusive scan of a[0..n) into out[0..n] (out[n] = total) by one block:
// each thread scans a contiguous run.
__device__ void block_scan_array(const int32_t* a, int32_t* out, int n, int* scratch)
{
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    int s = 0;
    for (int e = lo; e < hi; ++e) s += a[e];
    int total;
    int run = block_excl_scan(s, scratch, &total);
    for (int e = lo; e < hi; ++e) {
        out[e] = run;
        run += a[e];
    }
    if (threadIdx.x == 0) out[n] = total;
}

struct SelShared {
    int hist[256];
    int scratch[40];
    unsigned long long keys[EXACT];
    int idxs[EXACT];
    int nex;
    int bsel;
    int before;
};

// Calls mark(idx) for the `need` smallest keys among {idx in [0,n) : pred}.
// Keys are unique 64-bit values.  8-bit radix passes narrow the candidates
// to one digit bucket until at most EXACT remain, which are then ranked
// pairwise.  Every thread of the block must call it.
template <class Key, class Pred, class Mark>
__device__ void block_select_smallest(int n, int need, Key key, Pred pred, Mark mark, SelShared& sh,
                                      unsigned* paths)
{
    unsigned long long prefix = 0ull, pmask = 0ull;
    int shift = 56;
    while (need > 0) {
        int cnt = 0;
        for (int e = threadIdx.x; e < n; e += blockDim.x)
            if (pred(e) && (key(e) & pmask) == prefix) ++cnt;
        cnt = block_sum(cnt, sh.scratch);
        if (cnt <= need) {  // every remaining candidate is taken
            for (int e = threadIdx.x; e < n; e += blockDim.x)
                if (pred(e) && (key(e) & pmask) == prefix) mark(e);
            return;
        }
        if (cnt <= EXACT || shift < 0) {
            if (threadIdx.x == 0) sh.nex = 0;
            __syncthreads();
            for (int e = threadIdx.x; e < n; e += blockDim.x) {
                if (pred(e)) {
                    unsigned long long k = key(e);
                    if ((k & pmask) == prefix) {
                        int p = atomicAdd(&sh.nex, 1);
                        if (p < EXACT) {
                            sh.keys[p] = k;
                            sh.idxs[p] = e;
                        }
                    }
                }
            }
            __syncthreads();
            const int ne = min(sh.nex, EXACT);
            for (int a = threadIdx.x; a < ne; a += blockDim.x) {
                const unsigned long long ka = sh.keys[a];
                int rk = 0;
                for (int b = 0; b < ne; ++b) rk += sh.keys[b] < ka;
                if (rk < need) mark(sh.idxs[a]);
            }
            __syncthreads();
            return;
        }
        if (paths && threadIdx.x == 0) atomicOr(paths, shift == 56 ? NPATH_RADIX : NPATH_RADIX2);
        for (int t = threadIdx.x; t < 256; t += blockDim.x) sh.hist[t] = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            if (pred(e)) {
                unsigned long long k = key(e);
                if ((k & pmask) == prefix) atomicAdd(&sh.hist[(int)((k >> shift) & 255ull)], 1);
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // warp scan of the 256 bins (8 per lane): the bin where the running
            // count reaches `need`, and the count before it
            const int lane = threadIdx.x;
            int h8[8], loc = 0;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                h8[t] = sh.hist[lane * 8 + t];
                loc += h8[t];
            }
            int inc = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            int run = inc - loc;
            const bool here = run < need && need <= inc;
            if (here) {
                int b = lane * 8;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    if (run + h8[t] >= need) break;
                    run += h8[t];
                    ++b;
                }
                sh.bsel = b;
                sh.before = run;
            }
        }
        __syncthreads();
        const int b = sh.bsel, before = sh.before;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            if (pred(e)) {
                unsigned long long k = key(e);
                if ((k & pmask) == prefix && (int)((k >> shift) & 255ull) < b) mark(e);
            }
        }
        __syncthreads();
        need -= before;
        prefix |= (unsigned long long)b << shift;
        pmask |= 255ull << shift;
        shift -= 8;
    }
}

// ------------------------------------------------------------ k_level ------
struct LevelShared {
    int lev[LCAP + 1];
    int scratch[40];
    int Lstar;
    int maxhi;
    int nck;
    SelShared sel;
    unsigned long long ck[CKCAP];
    int2 rr[RRCAP];        // (rho_j, rho'_j)
};

__global__ void __launch_bounds__(LB) k_level(RunView v)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    LevelShared& sh = *reinterpret_cast<LevelShared*>(smraw);
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int w = v.w, K = c->K;
    const uint32_t gen = c->gen;
    const bool staged = w <= RRCAP;
    if (staged) {
        // all loads of a thread in flight at once (one SM does this work)
        constexpr int PT = RRCAP / LB;
        int a[PT], b[PT];
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            const int j = threadIdx.x + t * LB;
            a[t] = j < w ? v.rho[j] : 0;
            b[t] = j < w ? v.rhop[j] : 0;
        }
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            const int j = threadIdx.x + t * LB;
            if (j < w) sh.rr[j] = make_int2(a[t], b[t]);
        }
    }
    auto rho_of = [&](int j) { return staged ? sh.rr[j].x : v.rho[j]; };
    auto rhop_of = [&](int j) { return staged ? sh.rr[j].y : v.rhop[j]; };
    for (int t = threadIdx.x; t <= LCAP; t += LB) sh.lev[t] = 0;
    if (threadIdx.x == 0) {
        sh.Lstar = LCAP;
        sh.maxhi = 0;
    }
    __syncthreads();
    int mymax = 0;
    {
        // most references share a few level values (rho_j = 0 when S is
        // empty): lanes with equal values add once per warp (match groups),
        // so the shared-memory atomics do not serialise on one address
        const int lane = lane_id();
        for (int j0 = (threadIdx.x & ~31); j0 < w; j0 += LB) {
            const int j = j0 + lane;
            int rp = j < w ? rhop_of(j) : 0;
            const int lo = j < w ? rho_of(j) : 0;
            if (rp > 0 && (lo < 0 || rp > v.n2)) {  // counts out of range: an invariant failed upstream
                set_status(c, DEV_EINTERNAL);
                rp = 0;
            }
            const int hi = lo + rp;
            const bool add_lo = rp > 0 && lo < LCAP, add_hi = rp > 0 && hi < LCAP;
            const unsigned m_lo = __ballot_sync(0xffffffffu, add_lo);
            const unsigned m_hi = __ballot_sync(0xffffffffu, add_hi);
            if (add_lo) {
                const unsigned g = __match_any_sync(m_lo, lo);
                if (lane == __ffs(g) - 1) atomicAdd(&sh.lev[lo], __popc(g));
            }
            if (add_hi) {
                const unsigned g = __match_any_sync(m_hi, hi);
                if (lane == __ffs(g) - 1) atomicAdd(&sh.lev[hi], -__popc(g));
            }
            if (rp > 0) mymax = max(mymax, hi);
        }
    }
    mymax = __reduce_max_sync(0xffffffffu, mymax);
    if ((threadIdx.x & 31) == 0) atomicMax(&sh.maxhi, mymax);
    __syncthreads();
    // n(L) = prefix sum of the difference array; count(L) = prefix sum of n(L)
    {
        constexpr int PER = LCAP / LB;
        int loc[PER];
        int s = 0;
        for (int t = 0; t < PER; ++t) {
            s += sh.lev[threadIdx.x * PER + t];
            loc[t] = s;
        }
        int total;
        int off = block_excl_scan(s, sh.scratch, &total);
        for (int t = 0; t < PER; ++t) loc[t] += off;  // n(L)
        int s2 = 0;
        for (int t = 0; t < PER; ++t) {
            s2 += loc[t];
            loc[t] = s2;
        }
        int off2 = block_excl_scan(s2, sh.scratch, &total);
        for (int t = 0; t < PER; ++t) {
            const int L = threadIdx.x * PER + t;
            sh.lev[L] = loc[t] + off2;  // count(L)
        }
        __syncthreads();
        // count(L) is non-decreasing: the first L of this thread with
        // count >= K, then one atomic per warp
        int myL = LCAP;
        for (int t = PER - 1; t >= 0; --t) {
            const int L = threadIdx.x * PER + t;
            if (sh.lev[L] >= K) myL = L;
        }
        myL = __reduce_min_sync(0xffffffffu, myL);
        if ((threadIdx.x & 31) == 0 && myL < LCAP) atomicMin(&sh.Lstar, myL);
        __syncthreads();
    }
    int Lstar = sh.Lstar;
    int before;
    if (Lstar < LCAP) {
        before = Lstar > 0 ? sh.lev[Lstar - 1] : 0;
    } else {
        // deep levels: binary search with block-reduced counts
        if (threadIdx.x == 0) atomicOr(&c->npath, NPATH_DEEP);
        auto count_le = [&](int L) {
            int s = 0;
            for (int j = threadIdx.x; j < w; j += LB) {
                const int rp = rhop_of(j);
                if (rp > 0) s += min(rp, max(0, L + 1 - rho_of(j)));
            }
            return block_sum(s, sh.scratch);
        };
        int lo = LCAP, hi = max(LCAP, sh.maxhi - 1);
        while (lo < hi) {
            const int mid = lo + (hi - lo) / 2;
            if (count_le(mid) >= K)
                hi = mid;
            else
                lo = mid + 1;
        }
        Lstar = lo;
        before = count_le(Lstar - 1);
    }
    const int r = K - before;
    if (staged) {
        // The r smallest (priority, j) keys among the level-L* references:
        // each thread keeps the keys of its references in registers; one
        // 12-bit radix pass over the priorities' top bits finds the bin
        // holding the r-th key (about nC / 4096 keys per bin), the keys below
        // it are taken and the bin is ranked pairwise.
        constexpr int PT = RRCAP / LB;
        static_assert(LCAP == 4 * LB, "histogram bins per thread");
        unsigned long long kk[PT];
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            const int j = threadIdx.x + t * LB;
            kk[t] = ~0ull;
            if (j < w) {
                const int rp = sh.rr[j].y, lo = sh.rr[j].x;
                v.take[j] = rp > 0 ? min(rp, max(0, Lstar - lo)) : 0;
                if (rp > 0 && lo <= Lstar && Lstar < lo + rp) kk[t] = ref_key(v.seed, gen, j);
            }
        }
        __syncthreads();  // every thread has read `before` from the level table
        int* hist = sh.lev;
        for (int t = threadIdx.x; t < LCAP; t += LB) hist[t] = 0;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < PT; ++t)
            if (kk[t] != ~0ull) atomicAdd(&hist[(int)(kk[t] >> 52)], 1);
        __syncthreads();
        {
            int h4[4], loc = 0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                h4[t] = hist[threadIdx.x * 4 + t];
                loc += h4[t];
            }
            int total;
            int run = block_excl_scan(loc, sh.scratch, &total);
            if (run < r && r <= run + loc) {
                int b = threadIdx.x * 4;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (run + h4[t] >= r) break;
                    run += h4[t];
                    ++b;
                }
                sh.sel.bsel = b;
                sh.sel.before = run;
            }
        }
        if (threadIdx.x == 0) sh.sel.nex = 0;
        __syncthreads();
        const int b = sh.sel.bsel, need = r - sh.sel.before;
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            if (kk[t] == ~0ull) continue;
            const int bin = (int)(kk[t] >> 52);
            if (bin < b) {
                v.take[threadIdx.x + t * LB] += 1;
            } else if (bin == b) {
                const int p = atomicAdd(&sh.sel.nex, 1);
                if (p < EXACT) sh.sel.keys[p] = kk[t];
            }
        }
        __syncthreads();
        const int ne = sh.sel.nex;
        if (ne <= EXACT) {
            for (int a = threadIdx.x; a < ne; a += LB) {
                const unsigned long long ka = sh.sel.keys[a];
                int rk = 0;
                for (int q = 0; q < ne; ++q) rk += sh.sel.keys[q] < ka;
                if (rk < need) v.take[(int)(ka & 0xffffffffull)] += 1;
            }
        } else {
            // more than EXACT keys share the bin (not expected for Philox
            // priorities): select among them generically
            if (threadIdx.x == 0) atomicOr(&c->npath, NPATH_BINOVER);
            auto pred = [&](int j) {
                const int rp = sh.rr[j].y, lo = sh.rr[j].x;
                return rp > 0 && lo <= Lstar && Lstar < lo + rp && (int)(ref_key(v.seed, gen, j) >> 52) == b;
            };
            auto key = [&](int j) { return ref_key(v.seed, gen, j); };
            auto mark = [&](int j) { v.take[j] += 1; };
            block_select_smallest(w, need, key, pred, mark, sh.sel, &c->npath);
        }
    } else {
        if (threadIdx.x == 0) {
            sh.nck = 0;
            atomicOr(&c->npath, NPATH_UNSTAGED);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < w; j += LB) {
            const int rp = rhop_of(j);
            const int lo = rho_of(j);
            v.take[j] = rp > 0 ? min(rp, max(0, Lstar - lo)) : 0;
            if (rp > 0 && lo <= Lstar && Lstar < lo + rp) {
                const int p = atomicAdd(&sh.nck, 1);
                if (p < CKCAP) sh.ck[p] = ref_key(v.seed, gen, j);
            }
        }
        __syncthreads();
        const int nC = sh.nck;
        if (nC <= CKCAP) {
            auto key = [&](int e) { return sh.ck[e]; };
            auto pred = [&](int) { return true; };
            auto mark = [&](int e) { v.take[(int)(sh.ck[e] & 0xffffffffull)] += 1; };
            block_select_smallest(nC, r, key, pred, mark, sh.sel, &c->npath);
        } else {
            if (threadIdx.x == 0) atomicOr(&c->npath, NPATH_CKOVER);
            auto pred = [&](int j) {
                const int rp = rhop_of(j);
                const int lo = rho_of(j);
                return rp > 0 && lo <= Lstar && Lstar < lo + rp;
            };
            auto key = [&](int j) { return ref_key(v.seed, gen, j); };
            auto mark = [&](int j) { v.take[j] += 1; };
            block_select_smallest(w, r, key, pred, mark, sh.sel, &c->npath);
        }
    }
    __syncthreads();
    if (staged) {
        // exclusive scan of rho' over contiguous runs held in shared memory;
        // offsets replace rho in shared memory, then go out coalesced
        const int per = (w + LB - 1) / LB;
        const int lo = min(w, (int)threadIdx.x * per), hi = min(w, lo + per);
        int sum = 0;
        for (int j = lo; j < hi; ++j) sum += sh.rr[j].y;
        int total;
        int run = block_excl_scan(sum, sh.scratch, &total);
        for (int j = lo; j < hi; ++j) {
            const int cnt = sh.rr[j].y;
            sh.rr[j].x = run;
            run += cnt;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < w; j += LB) v.ref_off[j] = sh.rr[j].x;
        if (threadIdx.x == 0) v.ref_off[w] = total;
    } else {
        block_scan_array(v.rhop, v.ref_off, w, sh.scratch);
    }
    if (threadIdx.x == 0) {
        c->Lstar = Lstar;
        c->rlev = r;
        c->nlarge = 0;
    }
}

// ----------------------------------------------------------- k_bucket ------
__global__ void k_bucket(RunView v)
{
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n2 || v.rank2[i] != c->l) return;
    const int j = v.pi[i];
    if (j < 0 || j >= v.w) {
        set_status(c, DEV_EINTERNAL);
        return;
    }
    const int p = atomicAdd(&v.cursor[j], 1);
    if (p < v.rhop[j])
        v.bucket[v.ref_off[j] + p] = i;
    else
        set_status(c, DEV_EINTERNAL);
}

__device__ __forceinline__ void mark_member(const RunView& v, int i)
{
    atomicOr(&v.selmask[i >> 5], 1u << (i & 31));
}

// ------------------------------------------------------------- k_pick ------
// one warp per reference
__global__ void __launch_bounds__(256) k_pick(RunView v)
{
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t gen = c->gen;
    for (int j = gw; j < v.w; j += nw) {
        const int take = v.take[j];
        if (take == 0) continue;
        const int cnt = v.rhop[j], off = v.ref_off[j];
        if (take >= cnt) {
            for (int e = lane; e < cnt; e += 32) mark_member(v, v.bucket[off + e]);
            continue;
        }
        int need = take, excl = -1;
        if (v.rho[j] == 0) {
            double bd = CUDART_INF;
            int bi = 0x7fffffff;
#pragma unroll 4
            for (int e = lane; e < cnt; e += 32) {
                const int i = v.bucket[off + e];
                if (lex_less(v.dist[i], i, bd, bi)) {
                    bd = v.dist[i];
                    bi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double od = __shfl_xor_sync(0xffffffffu, bd, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (lex_less(od, oi, bd, bi)) {
                    bd = od;
                    bi = oi;
                }
            }
            if (lane == 0) mark_member(v, bi);
            excl = bi;
            need -= 1;
        }
        if (need == 0) continue;
        if (cnt <= 32) {
            unsigned long long k = ~0ull;
            int i = -1;
            if (lane < cnt) {
                i = v.bucket[off + lane];
                if (i != excl) k = ((unsigned long long)mem_prio(v.seed, gen, i) << 32) | (unsigned)i;
            }
            int rk = 0;
            for (int b = 0; b < cnt; ++b) {
                unsigned long long kb = __shfl_sync(0xffffffffu, k, b);
                rk += kb < k;
            }
            if (lane < cnt && i != excl && rk < need) mark_member(v, i);
        } else if (lane == 0) {
            const int p = atomicAdd(&c->nlarge, 1);
            v.large[p] = make_int4(j, need, excl, 0);
            atomicOr(&c->npath, NPATH_LARGE);
        }
    }
}

// large buckets with a partial take: one CTA per bucket
__global__ void __launch_bounds__(512) k_pick_large(RunView v)
{
    __shared__ SelShared sh;
    Ctrl* c = v.ctrl;
    if (skip_niche(c)) return;
    const int nl = c->nlarge;
    const uint32_t gen = c->gen;
    for (int t = blockIdx.x; t < nl; t += gridDim.x) {
        const int4 L = v.large[t];
        const int j = L.x, need = L.y, excl = L.z;
        const int cnt = v.rhop[j], off = v.ref_off[j];
        const int32_t* mem = v.bucket + off;
        auto pred = [&](int e) { return mem[e] != excl; };
        auto key = [&](int e) {
            const int i = mem[e];
            return ((unsigned long long)mem_prio(v.seed, gen, i) << 32) | (unsigned)i;
        };
        auto mark = [&](int e) { mark_member(v, mem[e]); };
        block_select_smallest(cnt, need, key, pred, mark, sh, &c->npath);
        __syncthreads();
    }
}

// Self-test of block_select_smallest on caller keys (one CTA): marks[e] = 1
// for the `need` smallest of keys[0..n), 0 otherwise; *paths gets the radix
// pass bits.
__global__ void __launch_bounds__(512) k_select_probe(const unsigned long long* keys, int n, int need,
                                                      uint32_t* marks, unsigned* paths)
{
    __shared__ SelShared sh;
    for (int e = threadIdx.x; e < n; e += blockDim.x) marks[e] = 0u;
    if (threadIdx.x == 0) *paths = 0u;
    __syncthreads();
    auto pred = [&](int) { return true; };
    auto key = [&](int e) { return keys[e]; };
    auto mark = [&](int e) { marks[e] = 1u; };
    block_select_smallest(n, need, key, pred, mark, sh, paths);
}

}  // namespace

cudaError_t launch_level(const RunView& v, cudaStream_t s)
{
    k_level<<<1, LB, sizeof(LevelShared), s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_bucket(const RunView& v, cudaStream_t s)
{
    k_bucket<<<(v.n2 + 255) / 256, 256, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_pick(const RunView& v, cudaStream_t s)
{
    int blocks = (v.w + 7) / 8;
    if (blocks > 4096) blocks = 4096;
    k_pick<<<blocks, 256, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one CTA per reference with a partial take, up to two per SM (how many
    // there are is known on the device only: CTAs without one exit)
    int lblocks = v.w < 2 * v.num_sms ? v.w : 2 * v.num_sms;
    if (lblocks < 16) lblocks = 16;
    k_pick_large<<<lblocks, 512, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_select_probe(const unsigned long long* keys, int n, int need, uint32_t* marks,
                                unsigned* paths, cudaStream_t s)
{
    k_select_probe<<<1, 512, 0, s>>>(keys, n, need, marks, paths);
    return cudaGetLastError();
}

cudaError_t niche_init_attributes()
{
    return cudaFuncSetAttribute(k_level, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(LevelShared));
}
