// engine.cu -- NSGA-III run context, device workspace, CUDA-graph capture of
// a selection / a generation, and the C ABI declared in include/nsga3.h.
//
// A generation is captured once per context as a CUDA graph of plain
// kernel nodes:
//   vary+eval -> reset -> sort -> dominance -> peel (one cooperative launch,
//   every front) -> post-peel -> ideal, extremes+solve, prep, scan, level,
//   bucket, pick -> compaction -> gather -> gen++
// The niching kernels return at once when |S| + |F_l| == N.  A replay never
// returns to the host.
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "nsga3.h"
#include "runtime.h"

cudaError_t niche_init_attributes();

namespace {

thread_local std::string g_create_error;
std::mutex g_attr_mutex;

enum { EV_START, EV_VARY, EV_RESET, EV_DOM, EV_PEEL, EV_NICHE, EV_END, EV_COUNT };
constexpr int BATCH_GENS = 4;  // generations per batched graph launch

// Creation serials: every context gets the next value, never reused in the
// life of the process, so a destroyed context and a new one that happens to
// occupy the same host address are told apart.
std::atomic<unsigned long long> g_ctx_serial{0};

__global__ void k_set_gen(Ctrl* c, uint32_t gen) { c->gen = gen; }

}  // namespace

struct nsga3_ctx {
    int device = 0, num_sms = 0;
    int m = 0, d = 0, N = 0, n2 = 0, ld = 0, NW = 0, w = 0, M4 = 0, p1 = 0, p2 = 0;
    double tau = 0.5;
    nsga3_opts opts{};
    bool has_obj = false;  // an objective is defined (W, or the knapsack arrays)
    RunView v{};    // generation view (population buffers)
    RunView vs{};   // selection view (own objective buffer)
    std::vector<void*> allocs;
    cudaGraphExec_t gx_select = nullptr, gx_step = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev[EV_COUNT] = {};
    int last_kind = 0;  // 1 = select, 2 = step
    long long host_launches = 0;  // kernels launched by calls (peel passes counted on the device)
    DeviceArena* arena = nullptr;  // workspace source (nullptr: cudaMalloc per buffer)
    bool count_only = false;       // sizing pass: count bytes, allocate nothing
    size_t counted = 0;
    bool eager = false; // NSGA3_EAGER=1: no graphs, host-driven peel loop (profiling)
    unsigned ev_mask = 0; // bit e set: event e is recorded (opts.phase_timing; eager: all)
    std::string err;
    unsigned long long serial = 0;  // creation serial (g_ctx_serial)
    bool shared_gpu = false;        // runs side by side with others (RunView::shared_gpu)
    // batched graph cache: the graphs hold the device buffers of every run in
    // the list, so they are keyed by the runs' creation serials (a pointer of
    // a destroyed run can be handed out again by the allocator)
    std::vector<unsigned long long> batch_key;
    cudaGraphExec_t gx_batch = nullptr;   // BATCH_GENS generations of every run
    cudaGraphExec_t gx_batch1 = nullptr;  // one generation of every run
    long long batch_builds = 0;           // times the batched graphs were (re)built
};

namespace {

// kernels of one selection / one generation: m > 10 adds five (ideal point,
// extreme-point keys and reduction, |f'|, candidate distances), m > 32 the
// cooperative elimination, and a split dominance build (few tiles) its
// finishing kernel
// Association of more than ASSOC_SMALL_W directions (m <= 10): the tiled
// scan (every FP32 cosine at the FMA rate) or the pruned scan (cone bounds
// per block of 32 directions).  Both give the same association.  The cone
// bounds skip most blocks up to m = 6 (the pruned scan is as fast or faster
// there: m = 5 and 10,626 directions 0.12 against 0.16 ms of niching per
// generation, m = 6 and 2,002 directions 0.133 against 0.137 ms); from m = 7
// they skip few and the tiled scan wins (m = 8 and 11,440 directions 0.79
// against 0.29 ms, m = 10 and 2,002 directions 0.31 against 0.21 ms).
// NSGA3_ASSOC=tile|scan overrides the choice for every context a process
// creates.
bool assoc_tile_wanted(int m)
{
    const char* e = getenv("NSGA3_ASSOC");
    if (e && strcmp(e, "scan") == 0) return false;
    if (e && strcmp(e, "tile") == 0) return true;
    return m >= 7;
}

int select_launches(const nsga3_ctx* ctx)
{
    const int m = ctx->m;
    // m <= 10: + the sort's level thresholds, the dominance build's boxes and tile plan;
    // - three association kernels with few reference directions (one fused kernel)
    return 18 + (m > NSGA3_FAST_M ? 5 : 3) + (m > NSGA3_WARP_M ? 1 : 0) + (ctx->v.dom_ks > 1 ? 1 : 0) -
           (assoc_small(ctx->v) ? 3 : 0);
}
// the softmax-simplex objective's dot-product kernel (m > 10)
int objective_dot_launches(const nsga3_ctx* ctx) { return ctx->m > NSGA3_FAST_M && ctx->v.problem == 0 ? 1 : 0; }
// variation + objective: one fused kernel for the softmax-simplex objective
// with m <= 10; variation, dot products and objective above; variation and
// evaluation (with repair) for the knapsack
int variation_launches(const nsga3_ctx* ctx)
{
    if (ctx->v.problem == 0 && ctx->m <= NSGA3_FAST_M) return 1;
    return 2 + objective_dot_launches(ctx);
}
int generation_launches(const nsga3_ctx* ctx)
{
    // the selection without its finite check, + variation, gather, commit
    return select_launches(ctx) - 1 + variation_launches(ctx) + 2;
}

nsga3_status fail(nsga3_ctx* c, nsga3_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
    return s;
}

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(ctx, NSGA3_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                     \
    } while (0)

long long binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

template <typename T>
nsga3_status alloc(nsga3_ctx* ctx, T** p, size_t count)
{
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    if (ctx->count_only) {
        ctx->counted += DeviceArena::round_up(bytes);
        *p = nullptr;
        return NSGA3_OK;
    }
    if (ctx->arena) {
        q = ctx->arena->alloc(bytes);
        if (!q) return fail(ctx, NSGA3_ENOMEM, "device arena has no free block of %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, NSGA3_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    ctx->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return NSGA3_OK;
}

#define AL(ptr, count)                                       \
    do {                                                     \
        nsga3_status s_ = alloc(ctx, &(ptr), (size_t)(count)); \
        if (s_ != NSGA3_OK) return s_;                       \
    } while (0)

// Timing events are recorded only where opts.phase_timing asks for them: an
// event node in a graph costs a few microseconds of every replay
nsga3_status record_event(nsga3_ctx* ctx, cudaStream_t s, int which, bool events)
{
    if (!events || !((ctx->ev_mask >> which) & 1u)) return NSGA3_OK;
    if (ctx->eager)
        CK(cudaEventRecord(ctx->ev[which], s));
    else
        CK(cudaEventRecordWithFlags(ctx->ev[which], s, cudaEventRecordExternal));
    return NSGA3_OK;
}

// Records the selection pipeline of view `v` into the capture running on `s`
nsga3_status record_selection(nsga3_ctx* ctx, const RunView& v, cudaStream_t s,
                              bool check_finite, bool events)
{
    CK(launch_sel_reset(v, s));
    if (check_finite) CK(launch_check_finite(v, s));
    CK(launch_sort(v, ctx->num_sms, s));
    nsga3_status st = record_event(ctx, s, EV_RESET, events);
    if (st) return st;
    CK(launch_dominance(v, s));
    st = record_event(ctx, s, EV_DOM, events);
    if (st) return st;
    CK(launch_peel(v, ctx->num_sms, s));
    st = record_event(ctx, s, EV_PEEL, events);
    if (st) return st;
    // ranks back to the original order, then (when niching is needed) the
    // ideal point; the niching kernels return at once when no niching is
    // needed: a graph IF node costs more than their empty launches
    CK(launch_norm_ideal(v, s));
    CK(launch_norm_extreme(v, ctx->num_sms, s));
    CK(launch_assoc_prep(v, s));
    CK(launch_assoc_scan(v, ctx->num_sms, s));
    CK(launch_level(v, s));
    CK(launch_bucket(v, s));
    CK(launch_pick(v, s));
    st = record_event(ctx, s, EV_NICHE, events);
    if (st) return st;
    CK(launch_compact(v, s));
    return NSGA3_OK;
}

nsga3_status record_generation(nsga3_ctx* ctx, cudaStream_t s, bool events)
{
    nsga3_status st = record_event(ctx, s, EV_START, events);
    if (st) return st;
    CK(launch_vary_eval(ctx->v, s));
    st = record_event(ctx, s, EV_VARY, events);
    if (st) return st;
    st = record_selection(ctx, ctx->v, s, false, events);
    if (st) return st;
    CK(launch_gather(ctx->v, s));  // next population and the generation counter
    return record_event(ctx, s, EV_END, events);
}

// Eager execution of the same kernels without graphs (NSGA3_EAGER=1): the
// niching kernels are launched only when the host reads that niching is
// needed.  For tools and debugging that want direct launches.
nsga3_status eager_selection(nsga3_ctx* ctx, const RunView& v, cudaStream_t s, bool check_finite)
{
    CK(launch_sel_reset(v, s));
    if (check_finite) CK(launch_check_finite(v, s));
    CK(launch_sort(v, ctx->num_sms, s));
    nsga3_status st = record_event(ctx, s, EV_RESET, true);
    if (st) return st;
    CK(launch_dominance(v, s));
    st = record_event(ctx, s, EV_DOM, true);
    if (st) return st;
    CK(launch_peel(v, ctx->num_sms, s));
    st = record_event(ctx, s, EV_PEEL, true);
    if (st) return st;
    CK(launch_norm_ideal(v, s));  // also writes the ranks back in the original order
    int32_t hdr[2] = {0, 0};  // status, need_niche
    CK(cudaMemcpyAsync(&hdr[0], &v.ctrl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hdr[1], &v.ctrl->need_niche, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hdr[0] == 0 && hdr[1]) {
        CK(launch_norm_extreme(v, ctx->num_sms, s));
        CK(launch_assoc_prep(v, s));
        CK(launch_assoc_scan(v, ctx->num_sms, s));
        CK(launch_level(v, s));
        CK(launch_bucket(v, s));
        CK(launch_pick(v, s));
    }
    st = record_event(ctx, s, EV_NICHE, true);
    if (st) return st;
    CK(launch_compact(v, s));
    return NSGA3_OK;
}

nsga3_status eager_generation(nsga3_ctx* ctx, cudaStream_t s)
{
    nsga3_status st = record_event(ctx, s, EV_START, true);
    if (st) return st;
    CK(launch_vary_eval(ctx->v, s));
    st = record_event(ctx, s, EV_VARY, true);
    if (st) return st;
    st = eager_selection(ctx, ctx->v, s, false);
    if (st) return st;
    CK(launch_gather(ctx->v, s));  // next population and the generation counter
    return record_event(ctx, s, EV_END, true);
}

nsga3_status build_graphs(nsga3_ctx* ctx)
{
    if (ctx->eager) return NSGA3_OK;
    cudaGraph_t g = nullptr;
    // selection graph
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeRelaxed));
    nsga3_status st = record_event(ctx, ctx->cap, EV_START, true);
    if (!st) st = record_event(ctx, ctx->cap, EV_VARY, true);
    if (!st) st = record_selection(ctx, ctx->vs, ctx->cap, true, true);
    if (!st) st = record_event(ctx, ctx->cap, EV_END, true);
    {
        cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        CK(e);
    }
    CK(cudaGraphInstantiate(&ctx->gx_select, g, 0));
    cudaGraphDestroy(g);
    g = nullptr;
    if (!ctx->has_obj) return NSGA3_OK;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeRelaxed));
    st = record_generation(ctx, ctx->cap, true);
    {
        cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        CK(e);
    }
    CK(cudaGraphInstantiate(&ctx->gx_step, g, 0));
    cudaGraphDestroy(g);
    return NSGA3_OK;
}

// Orders the w reference directions into blocks of 32 by recursive median
// splits of their unit vectors along the widest coordinate (every block but
// the last holds exactly 32), and records each block's unit centre and
// angular radius, inflated by 1e-6 rad to cover the FP32 rounding of the
// centre.  Only the association scan's pruning uses this order; results are
// reported with the original indices.
void build_ref_blocks(int m, int w, int M4, const std::vector<double>& Z, std::vector<float>& cent,
                      std::vector<float2>& crsr, std::vector<float>& zp, std::vector<int32_t>& jidx)
{
    std::vector<double> U((size_t)w * m);
    for (int j = 0; j < w; ++j) {
        double s = 0.0;
        for (int q = 0; q < m; ++q) s += Z[(size_t)j * m + q] * Z[(size_t)j * m + q];
        const double n = std::sqrt(s);
        for (int q = 0; q < m; ++q) U[(size_t)j * m + q] = Z[(size_t)j * m + q] / n;
    }
    std::vector<int32_t> perm(w);
    std::iota(perm.begin(), perm.end(), 0);
    struct Range {
        int lo, hi;
    };
    std::vector<Range> stack{{0, w}};
    while (!stack.empty()) {
        Range r = stack.back();
        stack.pop_back();
        if (r.hi - r.lo <= 32) continue;
        int dim = 0;
        double widest = -1.0;
        for (int q = 0; q < m; ++q) {
            double lo = 1e300, hi = -1e300;
            for (int t = r.lo; t < r.hi; ++t) {
                const double x = U[(size_t)perm[t] * m + q];
                lo = std::min(lo, x);
                hi = std::max(hi, x);
            }
            if (hi - lo > widest) {
                widest = hi - lo;
                dim = q;
            }
        }
        const int nbk = (r.hi - r.lo + 31) / 32;
        const int mid = r.lo + 32 * (nbk / 2);
        std::nth_element(perm.begin() + r.lo, perm.begin() + mid, perm.begin() + r.hi,
                         [&](int a, int b) {
                             const double xa = U[(size_t)a * m + dim], xb = U[(size_t)b * m + dim];
                             return xa < xb || (xa == xb && a < b);
                         });
        stack.push_back({r.lo, mid});
        stack.push_back({mid, r.hi});
    }
    const int nb = (w + 31) / 32;
    cent.assign((size_t)nb * M4, 0.0f);
    crsr.assign(nb, make_float2(1.0f, 0.0f));
    zp.assign((size_t)w * M4, 0.0f);
    jidx.assign(w, 0);
    for (int b = 0; b < nb; ++b) {
        const int lo = 32 * b, hi = std::min(w, lo + 32);
        double cvec[NSGA3_MAX_M] = {0};
        for (int t = lo; t < hi; ++t)
            for (int q = 0; q < m; ++q) cvec[q] += U[(size_t)perm[t] * m + q];
        double cn = 0.0;
        for (int q = 0; q < m; ++q) cn += cvec[q] * cvec[q];
        cn = std::sqrt(cn);
        for (int q = 0; q < m; ++q) cvec[q] /= cn;
        double cmin = 1.0;
        for (int t = lo; t < hi; ++t) {
            double dt = 0.0;
            for (int q = 0; q < m; ++q) dt += U[(size_t)perm[t] * m + q] * cvec[q];
            cmin = std::min(cmin, dt);
        }
        double r = std::acos(std::max(-1.0, std::min(1.0, cmin))) + 1e-6;
        if (r > M_PI) r = M_PI;
        crsr[b] = make_float2((float)std::cos(r), (float)std::sin(r));
        for (int q = 0; q < m; ++q) cent[(size_t)b * M4 + q] = (float)cvec[q];
        for (int t = lo; t < hi; ++t) {
            jidx[t] = perm[t];
            for (int q = 0; q < m; ++q) zp[(size_t)t * M4 + q] = (float)U[(size_t)perm[t] * m + q];
        }
    }
}

// Knapsack repair order: items by ascending best profit/weight ratio
// max_j p[j][v] / w[j][v], compared exactly by cross multiplication, ties to
// the lower item.
void kp_repair_order(const int32_t* p, const int32_t* w, int m, int d, std::vector<int32_t>& order)
{
    std::vector<int64_t> num(d), den(d);
    for (int v = 0; v < d; ++v) {
        num[v] = p[v];
        den[v] = w[v];
        for (int j = 1; j < m; ++j) {
            const int64_t pj = p[(size_t)j * d + v], wj = w[(size_t)j * d + v];
            if (pj * den[v] > num[v] * wj) {
                num[v] = pj;
                den[v] = wj;
            }
        }
    }
    order.resize(d);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const int64_t l = num[a] * den[b], r = num[b] * den[a];
        return l < r;
    });
}

// Allocates every device buffer of the context (or, in a sizing pass, only
// counts their bytes).
nsga3_status setup_alloc(nsga3_ctx* ctx)
{
    const int m = ctx->m, d = ctx->d, N = ctx->N, n2 = ctx->n2, ld = ctx->ld, NW = ctx->NW;
    const int w = ctx->w, M4 = ctx->M4;
    RunView& v = ctx->v;
    v.m = m;
    v.d = d;
    v.N = N;
    v.n2 = n2;
    v.ld = ld;
    v.NW = NW;
    v.w = w;
    v.M4 = M4;
    v.num_sms = ctx->num_sms > 0 ? ctx->num_sms : 1;
    v.shared_gpu = ctx->shared_gpu ? 1 : 0;
    v.full_sort = ctx->opts.full_sort ? 1 : 0;
    v.debug_recheck_all = ctx->opts.debug_recheck_all ? 1 : 0;
    v.streaming = ctx->opts.streaming ? 1 : 0;
    v.norm_history = ctx->opts.norm_history ? 1 : 0;
    v.problem = ctx->opts.problem;
    v.dom_ctas = ctx->opts.dom_ctas_per_sm;
    v.peel_ctas = ctx->opts.peel_ctas_per_sm;
    v.wait_ns = (unsigned long long)(ctx->opts.wait_ms > 0 ? ctx->opts.wait_ms : 20000) * 1000000ull;
    v.seed = ctx->opts.seed;
    v.eta_c = ctx->opts.eta_c;
    v.eta_m = ctx->opts.eta_m;
    v.p_c = ctx->opts.p_c;
    v.p_m = ctx->opts.p_m < 0.0f ? 1.0f / (float)d : ctx->opts.p_m;
    // at most two extreme-point blocks per SM (<= 512): the last block
    // reduces the blocks' partial results one warp per axis
    v.ext_parts = (n2 + 127) / 128;
    if (v.ext_parts > 2 * ctx->num_sms) v.ext_parts = 2 * ctx->num_sms;
    if (v.ext_parts > 512) v.ext_parts = 512;
    // m > 10 with fewer tiles than two per SM: split each tile's objective
    // chunks over dom_ks CTAs (k_dominance_gen + k_dom_finish)
    v.dom_ks = 1;
    if (m > NSGA3_FAST_M) {
        const long long T = ld / NSGA3_TILE, tiles = T * (T + 1) / 2;
        const long long nch = (m + 15) / 16, want = 2LL * ctx->num_sms;
        if (tiles < want && nch > 1) {
            const long long ks = (want + tiles - 1) / tiles;
            v.dom_ks = (int)(ks < nch ? ks : nch);
        }
    }

    AL(v.ctrl, 1);
    AL(v.X, (size_t)n2 * d);
    AL(v.F, (size_t)ld * m);
    AL(v.rank, N);
    AL(v.Xtmp, (size_t)N * d);
    AL(v.Ftmp, (size_t)N * m);
    AL(v.ranktmp, N);
    AL(v.Dom, v.streaming ? (size_t)1 : (size_t)NW * ld);
    AL(v.cnt, ld);
    AL(v.rank2, ld);
    AL(v.srank, ld);
    AL(v.perm, ld);
    AL(v.skey, ld);
    AL(v.pkey, n2);
    AL(v.Fp, (size_t)ld * m);
    // sort keys (k_sort.cu): m <= 10 interleaves lbits of level per objective
    // (Morton order), truncated to kbits, about n2 / 2 keys; above, 4,096 f_0 buckets
    if (m <= NSGA3_FAST_M) {
        v.lbits = m <= 5 ? 3 : 2;
        int lg = 0;
        while ((2 << lg) <= n2) ++lg;  // floor(log2(n2))
        int kb = lg - 1;
        kb = kb < 8 ? 8 : kb > 16 ? 16 : kb;
        v.kbits = kb < v.lbits * m ? kb : v.lbits * m;
    } else {
        v.lbits = 0;
        v.kbits = 12;
    }
    AL(v.bcnt, (1 << v.kbits) + 1);
    v.NB8 = (NW + 7) / 8;
    if (m <= NSGA3_FAST_M) {
        AL(v.qhist, (size_t)m * SORT_QB);
        AL(v.bbox, (size_t)NW * 2 * M4);
        AL(v.bkey, (size_t)NW * 2);
        const size_t T = (size_t)ld / NSGA3_TILE;
        AL(v.tbox, T * 2 * M4);
        AL(v.tkey, T * 2);
        AL(v.tlist, T * (T + 1) / 2);
        if (!v.streaming) AL(v.dnz, (size_t)NW * v.NB8);
    }
    AL(v.rem, NW);
    AL(v.front, 2 * NW);
    AL(v.chunk_lim, ld / NSGA3_PEEL_COLS);
    AL(v.selmask, NW);
    AL(v.Tlist, n2);
    AL(v.fprime, (size_t)n2 * m);
    AL(v.fnorm, n2);
    AL(v.uhat, (size_t)n2 * M4);
    AL(v.pi, ld);
    AL(v.dist, ld);
    AL(v.ext_part, (size_t)v.ext_parts * m);
    AL(v.ext_idx, (size_t)v.ext_parts * m);
    AL(v.nad_part, (size_t)v.ext_parts * m);
    AL(v.rho, w);
    AL(v.rhop, w);
    AL(v.take, w);
    AL(v.ref_off, w + 1);
    AL(v.cursor, w);
    AL(v.bucket, n2);
    AL(v.large, w);
    AL(v.sel, N);
    v.nblk = (w + 31) / 32;
    v.cand_cap = 4 * n2 + 64;
    AL(v.arun, n2);
    AL(v.cand, v.cand_cap);
    AL(v.slow, n2);
    v.aent = nullptr;
    v.assoc_grid = 0;
    if (m <= NSGA3_FAST_M && w > ASSOC_SMALL_W && assoc_tile_wanted(m)) {
        v.assoc_grid = assoc_tile_grid(v.num_sms);
        AL(v.aent, assoc_tile_entries(n2, v.num_sms));
    }
    AL(v.he, (size_t)m * m);
    if (m > NSGA3_FAST_M) {
        AL(v.cdist, v.cand_cap);
        AL(v.nadv, m);
    }
    if (v.dom_ks > 1) {
        AL(v.dpa, (size_t)NW * ld);
        AL(v.dpb, (size_t)NW * ld);
    }
    if (m > NSGA3_FAST_M) {
        AL(v.ekey, 2 * (size_t)(n2 + m));
        AL(v.er1, (size_t)(n2 + m));
    }
    if (m > NSGA3_WARP_M) {
        AL(v.amat, (size_t)m * (m + 1));
        AL(v.etmp, (size_t)m * m);
    }
    float* bc;
    float2* br;
    float* bz;
    int32_t* bj;
    AL(bc, (size_t)v.nblk * M4);
    AL(br, v.nblk);
    AL(bz, (size_t)w * M4);
    AL(bj, w);
    v.blk_c = bc;
    v.blk_r = br;
    v.blk_z = bz;
    v.blk_j = bj;
    double* Zd;
    double* nz;
    float* Zh;
    float* Wd;
    AL(Zd, (size_t)w * m);
    AL(nz, w);
    AL(Zh, (size_t)w * M4);
    AL(Wd, (size_t)m * (m - 1));
    if (m > NSGA3_FAST_M && v.problem == 0) {
        float* Wt;
        AL(Wt, (size_t)m * (m - 1));
        v.Wt = Wt;
    }
    if (v.problem == 1) {
        int32_t *kp, *kw, *kc, *kt, *ko;
        AL(kp, (size_t)m * d);
        AL(kw, (size_t)m * d);
        AL(kc, m);
        AL(kt, m);
        AL(ko, d);
        v.kp_p = kp;
        v.kp_w = kw;
        v.kp_cap = kc;
        v.kp_total = kt;
        v.kp_order = ko;
    }
    v.Zd = Zd;
    v.nz = nz;
    v.Zh = Zh;
    v.Wobj = Wd;
    ctx->vs = v;
    AL(ctx->vs.F, (size_t)ld * m);
    return NSGA3_OK;
}

nsga3_status setup(nsga3_ctx* ctx)
{
    nsga3_status ast = setup_alloc(ctx);
    if (ast) return ast;
    const int m = ctx->m, d = ctx->d, N = ctx->N, n2 = ctx->n2, ld = ctx->ld, NW = ctx->NW;
    const int w = ctx->w, M4 = ctx->M4;
    RunView& v = ctx->v;
    double* Zd = const_cast<double*>(v.Zd);
    double* nz = const_cast<double*>(v.nz);
    float* Zh = const_cast<float*>(v.Zh);
    float* Wd = const_cast<float*>(v.Wobj);
    float* bc = const_cast<float*>(v.blk_c);
    float2* br = const_cast<float2*>(v.blk_r);
    float* bz = const_cast<float*>(v.blk_z);
    int32_t* bj = const_cast<int32_t*>(v.blk_j);

    CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
    for (int e = 0; e < EV_COUNT; ++e) CK(cudaEventCreate(&ctx->ev[e]));
    cudaStream_t s = ctx->cap;
    CK(cudaMemsetAsync(v.ctrl, 0, sizeof(Ctrl), s));
    if (!v.streaming) CK(cudaMemsetAsync(v.Dom, 0, (size_t)NW * ld * sizeof(uint32_t), s));
    if (v.dom_ks > 1) {
        CK(cudaMemsetAsync(v.dpa, 0, (size_t)NW * ld * sizeof(uint32_t), s));
        CK(cudaMemsetAsync(v.dpb, 0, (size_t)NW * ld * sizeof(uint32_t), s));
    }
    CK(cudaMemsetAsync(v.rank, 0, (size_t)N * sizeof(int32_t), s));
    CK(cudaMemsetAsync(v.X, 0, (size_t)n2 * d * sizeof(float), s));
    CK(cudaMemsetAsync(v.F, 0, (size_t)ld * m * sizeof(float), s));
    CK(cudaMemsetAsync(ctx->vs.F, 0, (size_t)ld * m * sizeof(float), s));
    CK(cudaMemsetAsync(v.pi, 0xff, (size_t)ld * sizeof(int32_t), s));
    CK(cudaMemsetAsync(v.dist, 0, (size_t)ld * sizeof(double), s));
    CK(launch_nan_pad(v, s));
    CK(launch_nan_pad(ctx->vs, s));
    CK(launch_refdirs(v, ctx->p1, ctx->p2, ctx->tau, Zd, nz, Zh, s));
    std::vector<float> Wt_host;
    if (ctx->has_obj && v.problem == 0) {
        CK(cudaMemcpyAsync(Wd, ctx->opts.W, (size_t)m * (m - 1) * sizeof(float), cudaMemcpyHostToDevice, s));
        if (v.Wt) {  // (m-1) x m: the objective kernel reads a row of W^T per variable
            Wt_host.resize((size_t)m * (m - 1));
            for (int j = 0; j < m; ++j)
                for (int e = 0; e < m - 1; ++e) Wt_host[(size_t)e * m + j] = ctx->opts.W[(size_t)j * (m - 1) + e];
            CK(cudaMemcpyAsync(const_cast<float*>(v.Wt), Wt_host.data(), Wt_host.size() * sizeof(float),
                               cudaMemcpyHostToDevice, s));
        }
    }
    std::vector<int32_t> kp_order, kp_total;
    if (ctx->has_obj && v.problem == 1) {
        kp_repair_order(ctx->opts.kp_profit, ctx->opts.kp_weight, m, d, kp_order);
        kp_total.assign(m, 0);
        for (int j = 0; j < m; ++j)
            for (int e = 0; e < d; ++e) kp_total[j] += ctx->opts.kp_profit[(size_t)j * d + e];
        CK(cudaMemcpyAsync(const_cast<int32_t*>(v.kp_p), ctx->opts.kp_profit, (size_t)m * d * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(const_cast<int32_t*>(v.kp_w), ctx->opts.kp_weight, (size_t)m * d * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(const_cast<int32_t*>(v.kp_cap), ctx->opts.kp_capacity, (size_t)m * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(const_cast<int32_t*>(v.kp_total), kp_total.data(), (size_t)m * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(const_cast<int32_t*>(v.kp_order), kp_order.data(), (size_t)d * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
    {
        std::vector<double> Zh((size_t)w * m);
        CK(cudaMemcpyAsync(Zh.data(), Zd, Zh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::vector<float> hc, hz;
        std::vector<float2> hr;
        std::vector<int32_t> hj;
        build_ref_blocks(m, w, M4, Zh, hc, hr, hz, hj);
        // copies on the context's own stream: no implicit synchronisation with
        // other streams of the process (runs of a server keep executing)
        CK(cudaMemcpyAsync(bc, hc.data(), hc.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(br, hr.data(), hr.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(bz, hz.data(), hz.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(bj, hj.data(), hj.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        ctx->vs.blk_c = bc;
        ctx->vs.blk_r = br;
        ctx->vs.blk_z = bz;
        ctx->vs.blk_j = bj;
        ctx->vs.nblk = v.nblk;
        ctx->vs.arun = v.arun;
        ctx->vs.cand = v.cand;
        ctx->vs.cand_cap = v.cand_cap;
        ctx->vs.slow = v.slow;
    }
    cudaError_t ae;
    {
        std::lock_guard<std::mutex> lk(g_attr_mutex);
        ae = assoc_prepare(v);
    }
    if (ae != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, NSGA3_EINVAL, "%d reference directions exceed the association scan's tables", w);
    }
    return build_graphs(ctx);
}

bool g_attr_done = false;

nsga3_status init_attributes(nsga3_ctx* ctx)
{
    std::lock_guard<std::mutex> lk(g_attr_mutex);
    if (g_attr_done) return NSGA3_OK;
    CK(niche_init_attributes());
    CK(peel_init_attributes());
    CK(assoc_init_attributes());
    CK(norm_init_attributes());
    CK(dom_init_attributes());
    g_attr_done = true;
    return NSGA3_OK;
}

// Reads (and clears) the sticky device status on `s`, synchronising only s.
nsga3_status device_status(nsga3_ctx* ctx, cudaStream_t s, bool clear)
{
    int32_t st = 0;
    CK(cudaMemcpyAsync(&st, &ctx->v.ctrl->status, sizeof st, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (clear && st) {
        CK(cudaMemsetAsync(&ctx->v.ctrl->status, 0, sizeof st, s));
        CK(cudaStreamSynchronize(s));
    }
    return (nsga3_status)st;
}

// Checks the arguments of a context and fills its sizes (no device work).
nsga3_status ctx_fields(nsga3_ctx* ctx, int m, int d, int N, int ref_divisions, const nsga3_opts* opts)
{
    nsga3_opts o;
    nsga3_default_opts(&o);
    if (opts) o = *opts;
    if (m < 2 || m > NSGA3_MAX_M) return fail(ctx, NSGA3_EINVAL, "m=%d outside [2, %d]", m, NSGA3_MAX_M);
    if (N < 2 || (N & 1)) return fail(ctx, NSGA3_EINVAL, "N=%d must be even and >= 2", N);
    if (N > (1 << 20)) return fail(ctx, NSGA3_EINVAL, "N=%d above 2^20", N);
    if (d < 1) return fail(ctx, NSGA3_EINVAL, "d=%d < 1", d);
    if (o.W && d < m - 1) return fail(ctx, NSGA3_EINVAL, "d=%d < m-1 with an objective", d);
    if ((long long)N * d >= (1LL << 32)) return fail(ctx, NSGA3_EINVAL, "N*d must be < 2^32");
    if (ref_divisions < 1 || o.p2 < 0) return fail(ctx, NSGA3_EINVAL, "bad reference divisions");
    if (!(o.tau >= 0.0 && o.tau <= 1.0)) return fail(ctx, NSGA3_EINVAL, "tau outside [0,1]");
    if (o.problem != 0 && o.problem != 1) return fail(ctx, NSGA3_EINVAL, "problem %d unknown", o.problem);
    if (o.phase_timing < 0 || o.phase_timing > 2)
        return fail(ctx, NSGA3_EINVAL, "phase_timing %d outside [0, 2]", o.phase_timing);
    if (o.dom_ctas_per_sm < 0 || o.dom_ctas_per_sm > 64 || o.peel_ctas_per_sm < 0 || o.peel_ctas_per_sm > 64)
        return fail(ctx, NSGA3_EINVAL, "CTAs per SM outside [0, 64]");
    if (o.streaming && m > NSGA3_FAST_M)
        return fail(ctx, NSGA3_EINVAL, "streaming dominance supports m <= %d", NSGA3_FAST_M);
    if (o.problem == 1 && m > NSGA3_FAST_M)
        return fail(ctx, NSGA3_EINVAL, "the knapsack workload supports m <= %d", NSGA3_FAST_M);
    if (o.problem == 1 && o.kp_profit && o.kp_weight && o.kp_capacity) {
        // integer sums stay exact: weights below 2^31, objectives (profit
        // totals) below 2^24 so that FP32 holds them exactly
        for (int j = 0; j < m; ++j) {
            long long tp = 0, tw = 0;
            for (int e = 0; e < d; ++e) {
                const long long pe = o.kp_profit[(size_t)j * d + e], we = o.kp_weight[(size_t)j * d + e];
                if (pe <= 0 || we <= 0) return fail(ctx, NSGA3_EINVAL, "knapsack profits and weights must be > 0");
                tp += pe;
                tw += we;
            }
            if (tp >= (1LL << 24) || tw >= (1LL << 31) || o.kp_capacity[j] < 0)
                return fail(ctx, NSGA3_EINVAL, "knapsack %d: total profit must be < 2^24, total weight < 2^31", j);
        }
    }
    long long w = binom(ref_divisions + m - 1, m - 1) + (o.p2 > 0 ? binom(o.p2 + m - 1, m - 1) : 0);
    if (w < 1 || w > (1LL << 24)) return fail(ctx, NSGA3_EINVAL, "reference set size %lld", w);
    ctx->m = m;
    ctx->d = d;
    ctx->N = N;
    ctx->n2 = 2 * N;
    ctx->ld = (ctx->n2 + NSGA3_TILE - 1) / NSGA3_TILE * NSGA3_TILE;
    ctx->NW = ctx->ld / 32;
    ctx->w = (int)w;
    ctx->M4 = (m + 3) & ~3;
    ctx->p1 = ref_divisions;
    ctx->p2 = o.p2;
    ctx->tau = o.tau;
    ctx->opts = o;
    // W and the knapsack arrays are read during create only
    ctx->has_obj = o.problem == 1 ? (o.kp_profit && o.kp_weight && o.kp_capacity) : o.W != nullptr;
    return NSGA3_OK;
}

}  // namespace

nsga3_status ctx_create(int m, int d, int N, int ref_divisions, const nsga3_opts* opts, DeviceArena* arena,
                        nsga3_ctx** out, std::string* err, bool shared_gpu)
{
    if (!out) {
        if (err) *err = "out is NULL";
        return NSGA3_EINVAL;
    }
    *out = nullptr;
    nsga3_ctx* ctx = new nsga3_ctx();
    ctx->serial = ++g_ctx_serial;
    ctx->arena = arena;
    ctx->shared_gpu = shared_gpu;
    nsga3_status st = ctx_fields(ctx, m, d, N, ref_divisions, opts);
    if (!st) {
        const char* e = getenv("NSGA3_EAGER");
        ctx->eager = e && e[0] == '1';
        const int pt = ctx->opts.phase_timing;
        ctx->ev_mask = (ctx->eager || pt == 2) ? (1u << EV_COUNT) - 1u
                       : pt == 1               ? (1u << EV_RESET) | (1u << EV_DOM) | (1u << EV_PEEL)
                                               : 0u;
        if (cudaGetDevice(&ctx->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
            cudaGetLastError();
            st = fail(ctx, NSGA3_ECUDA, "no CUDA device");
        }
    }
    if (!st) st = init_attributes(ctx);
    if (!st) st = setup(ctx);
    ctx->opts.W = nullptr;
    if (st) {
        if (err) *err = ctx->err;
        ctx_destroy(ctx, arena == nullptr);
        return st;
    }
    *out = ctx;
    return NSGA3_OK;
}

nsga3_status ctx_workspace_bytes(int m, int d, int N, int ref_divisions, const nsga3_opts* opts, int num_sms,
                                 size_t* bytes, std::string* err)
{
    nsga3_ctx c{};
    c.count_only = true;
    nsga3_status st = ctx_fields(&c, m, d, N, ref_divisions, opts);
    if (!st) {
        c.num_sms = num_sms;
        if (c.num_sms <= 0) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                c.num_sms = 256;  // no device: an upper bound of the per-SM buffers
            }
        }
        st = setup_alloc(&c);
    }
    if (st) {
        if (err) *err = c.err;
        return st;
    }
    *bytes = c.counted;
    return NSGA3_OK;
}

void ctx_destroy(nsga3_ctx* ctx, bool sync_device)
{
    if (!ctx) return;
    if (sync_device) cudaDeviceSynchronize();
    if (ctx->gx_batch) cudaGraphExecDestroy(ctx->gx_batch);
    if (ctx->gx_batch1) cudaGraphExecDestroy(ctx->gx_batch1);
    if (ctx->gx_select) cudaGraphExecDestroy(ctx->gx_select);
    if (ctx->gx_step) cudaGraphExecDestroy(ctx->gx_step);
    for (int e = 0; e < EV_COUNT; ++e)
        if (ctx->ev[e]) cudaEventDestroy(ctx->ev[e]);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    for (void* p : ctx->allocs) {
        if (ctx->arena)
            ctx->arena->release(p);
        else
            cudaFree(p);
    }
    cudaGetLastError();
    delete ctx;
}

nsga3_status ctx_launches(nsga3_ctx* ctx, void* stream, long long* launches)
{
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    *launches = ctx->host_launches;
    return NSGA3_OK;
}

// One graph holding `gens` consecutive generations of every run as parallel
// branches (fork/join events), the runs with the most dominance work first
// so that their longer chains start first; a run's next generation depends
// only on its own previous one, so small runs run ahead within the graph.
nsga3_status build_batch_graph(nsga3_ctx* ctx, nsga3_ctx** ctxs, int n, int gens, cudaGraphExec_t* out)
{
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double wa = (double)ctxs[a]->n2 * ctxs[a]->n2 * ctxs[a]->m;
        const double wb = (double)ctxs[b]->n2 * ctxs[b]->n2 * ctxs[b]->m;
        return wa > wb;
    });
    std::vector<cudaStream_t> br(n);
    std::vector<cudaEvent_t> evs(n + 1);
    nsga3_status st = NSGA3_OK;
    for (int r = 0; r < n && !st; ++r)
        if (cudaStreamCreateWithFlags(&br[r], cudaStreamNonBlocking) != cudaSuccess)
            st = fail(ctx, NSGA3_ECUDA, "stream creation failed");
    for (int r = 0; r <= n && !st; ++r)
        if (cudaEventCreateWithFlags(&evs[r], cudaEventDisableTiming) != cudaSuccess)
            st = fail(ctx, NSGA3_ECUDA, "event creation failed");
    cudaGraph_t g = nullptr;
    if (!st) {
        cudaStream_t s0 = ctx->cap;
        if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            st = fail(ctx, NSGA3_ECUDA, "capture begin failed");
        if (!st && cudaEventRecord(evs[n], s0) != cudaSuccess) st = fail(ctx, NSGA3_ECUDA, "fork failed");
        for (int t = 0; t < n && !st; ++t) {
            const int r = order[t];
            if (cudaStreamWaitEvent(br[r], evs[n], 0) != cudaSuccess) {
                st = fail(ctx, NSGA3_ECUDA, "fork wait failed");
                break;
            }
            // the runs of a batched graph share the GPU
            const int shared = ctxs[r]->v.shared_gpu;
            ctxs[r]->v.shared_gpu = 1;
            for (int k = 0; k < gens && !st; ++k) {
                nsga3_status rs = record_generation(ctxs[r], br[r], false);
                if (rs) {
                    st = rs;
                    ctx->err = ctxs[r]->err;
                }
            }
            ctxs[r]->v.shared_gpu = shared;
            // join the branch even after a failure so the capture ends cleanly
            if (cudaEventRecord(evs[r], br[r]) != cudaSuccess || cudaStreamWaitEvent(s0, evs[r], 0) != cudaSuccess) {
                if (!st) st = fail(ctx, NSGA3_ECUDA, "join failed");
            }
        }
        cudaError_t e = cudaStreamEndCapture(s0, &g);
        if (!st && e != cudaSuccess) st = fail(ctx, NSGA3_ECUDA, "capture failed: %s", cudaGetErrorString(e));
        if (!st && cudaGraphInstantiate(out, g, 0) != cudaSuccess)
            st = fail(ctx, NSGA3_ECUDA, "batched graph instantiation failed");
        if (g) cudaGraphDestroy(g);
    }
    for (int r = 0; r < n; ++r)
        if (br[r]) cudaStreamDestroy(br[r]);
    for (int r = 0; r <= n; ++r)
        if (evs[r]) cudaEventDestroy(evs[r]);
    cudaGetLastError();
    return st;
}

// =============================================================== C ABI ====
extern "C" {

void nsga3_default_opts(nsga3_opts* o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->seed = 0;
    o->p2 = 0;
    o->tau = 0.5;
    o->eta_c = 20.0f;
    o->eta_m = 20.0f;
    o->p_c = 1.0f;
    o->p_m = -1.0f;
    o->full_sort = 0;
    o->debug_recheck_all = 0;
    o->streaming = 0;
    o->norm_history = 0;
    o->W = nullptr;
    o->wait_ms = 20000;
    o->phase_timing = 0;
}

nsga3_status nsga3_create(int m, int d, int N, int ref_divisions, const nsga3_opts* opts,
                          nsga3_ctx** out)
{
    std::string err;
    nsga3_status st = ctx_create(m, d, N, ref_divisions, opts, nullptr, out, &err);
    if (st) g_create_error = err;
    return st;
}

void nsga3_destroy(nsga3_ctx* ctx) { ctx_destroy(ctx, true); }

nsga3_status nsga3_workspace_bytes(int m, int d, int N, int ref_divisions, const nsga3_opts* opts,
                                   uint64_t* bytes)
{
    if (!bytes) return fail(nullptr, NSGA3_EINVAL, "bytes is NULL");
    std::string err;
    size_t b = 0;
    nsga3_status st = ctx_workspace_bytes(m, d, N, ref_divisions, opts, 0, &b, &err);
    if (st) return fail(nullptr, st, "%s", err.c_str());
    *bytes = b;
    return NSGA3_OK;
}

const char* nsga3_last_error(const nsga3_ctx* ctx)
{
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

int nsga3_num_refs(const nsga3_ctx* ctx) { return ctx ? ctx->w : 0; }

nsga3_status nsga3_get_refs(nsga3_ctx* ctx, double* Z)
{
    if (!ctx || !Z) return fail(ctx, NSGA3_EINVAL, "null argument");
    CK(cudaMemcpy(Z, ctx->v.Zd, (size_t)ctx->w * ctx->m * sizeof(double), cudaMemcpyDefault));
    return NSGA3_OK;
}

nsga3_status nsga3_select(nsga3_ctx* ctx, const float* objs, int32_t* ranks, int32_t* selected,
                          void* stream)
{
    if (!ctx || !objs || !ranks || !selected) return fail(ctx, NSGA3_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(ctx->vs.F, objs, (size_t)ctx->n2 * ctx->m * sizeof(float), cudaMemcpyDefault, s));
    if (ctx->eager) {
        nsga3_status st = record_event(ctx, s, EV_START, true);
        if (!st) st = record_event(ctx, s, EV_VARY, true);
        if (!st) st = eager_selection(ctx, ctx->vs, s, true);
        if (!st) st = record_event(ctx, s, EV_END, true);
        if (st) return st;
    } else {
        CK(cudaGraphLaunch(ctx->gx_select, s));
    }
    ctx->host_launches += select_launches(ctx);
    CK(cudaMemcpyAsync(ranks, ctx->vs.rank2, (size_t)ctx->n2 * sizeof(int32_t), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(selected, ctx->vs.sel, (size_t)ctx->N * sizeof(int32_t), cudaMemcpyDefault, s));
    ctx->last_kind = 1;
    return NSGA3_OK;
}

nsga3_status nsga3_init(nsga3_ctx* ctx, void* stream)
{
    if (!ctx) return fail(ctx, NSGA3_EINVAL, "null context");
    if (!ctx->has_obj) return fail(ctx, NSGA3_ESTATE, "context has no objective (opts.W or the knapsack arrays were NULL)");
    cudaStream_t s = (cudaStream_t)stream;
    CK(launch_init(ctx->v, s));
    CK(cudaMemsetAsync(&ctx->v.ctrl->hvalid, 0, sizeof(int32_t), s));  // a new run starts without history
    k_set_gen<<<1, 1, 0, s>>>(ctx->v.ctrl, 0u);
    CK(cudaGetLastError());
    ctx->host_launches += 3 + objective_dot_launches(ctx);
    return NSGA3_OK;
}

nsga3_status nsga3_vary(nsga3_ctx* ctx, void* stream)
{
    if (!ctx) return fail(ctx, NSGA3_EINVAL, "null context");
    if (!ctx->has_obj) return fail(ctx, NSGA3_ESTATE, "context has no objective (opts.W or the knapsack arrays were NULL)");
    CK(launch_vary_eval(ctx->v, (cudaStream_t)stream));
    ctx->host_launches += variation_launches(ctx);
    return NSGA3_OK;
}

nsga3_status nsga3_step(nsga3_ctx* ctx, void* stream)
{
    if (!ctx) return fail(ctx, NSGA3_EINVAL, "null context");
    if (!ctx->has_obj) return fail(ctx, NSGA3_ESTATE, "context has no objective (opts.W or the knapsack arrays were NULL)");
    if (ctx->eager) {
        nsga3_status st = eager_generation(ctx, (cudaStream_t)stream);
        if (st) return st;
    } else {
        CK(cudaGraphLaunch(ctx->gx_step, (cudaStream_t)stream));
    }
    ctx->host_launches += generation_launches(ctx);
    ctx->last_kind = 2;
    return NSGA3_OK;
}

nsga3_status nsga3_run(nsga3_ctx* ctx, int generations, void* stream)
{
    if (!ctx || generations < 0) return fail(ctx, NSGA3_EINVAL, "bad arguments");
    for (int g = 0; g < generations; ++g) {
        nsga3_status st = nsga3_step(ctx, stream);
        if (st) return st;
    }
    return NSGA3_OK;
}

nsga3_status nsga3_run_batch(nsga3_ctx** ctxs, int n, int generations, void* stream)
{
    nsga3_ctx* ctx = (n > 0 && ctxs) ? ctxs[0] : nullptr;
    if (!ctx || generations < 0) return fail(ctx, NSGA3_EINVAL, "bad arguments");
    std::vector<unsigned long long> key(n);
    for (int r = 0; r < n; ++r) {
        if (!ctxs[r] || !ctxs[r]->has_obj) return fail(ctx, NSGA3_EINVAL, "run %d has no objective", r);
        key[r] = ctxs[r]->serial;
    }
    {
        // a run listed twice would be two concurrent branches on the same
        // buffers and barrier words
        std::vector<unsigned long long> sorted(key);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return fail(ctx, NSGA3_EINVAL, "a context appears more than once in the list");
    }
    if (ctx->eager) {
        for (int g = 0; g < generations; ++g)
            for (int r = 0; r < n; ++r) {
                nsga3_status st = nsga3_step(ctxs[r], stream);
                if (st) return st;
            }
        return NSGA3_OK;
    }
    if (!ctx->gx_batch || !ctx->gx_batch1 || ctx->batch_key != key) {
        for (cudaGraphExec_t* gx : {&ctx->gx_batch, &ctx->gx_batch1})
            if (*gx) {
                cudaGraphExecDestroy(*gx);
                *gx = nullptr;
            }
        ctx->batch_key.clear();
        nsga3_status st = build_batch_graph(ctx, ctxs, n, BATCH_GENS, &ctx->gx_batch);
        if (!st) st = build_batch_graph(ctx, ctxs, n, 1, &ctx->gx_batch1);
        if (st) return st;
        ctx->batch_key = key;
        ++ctx->batch_builds;
    }
    for (int g = 0; g + BATCH_GENS <= generations; g += BATCH_GENS)
        CK(cudaGraphLaunch(ctx->gx_batch, (cudaStream_t)stream));
    for (int g = 0; g < generations % BATCH_GENS; ++g) CK(cudaGraphLaunch(ctx->gx_batch1, (cudaStream_t)stream));
    for (int r = 0; r < n; ++r) {
        ctxs[r]->last_kind = 3;
        ctxs[r]->host_launches += (long long)generation_launches(ctxs[r]) * generations;
    }
    return NSGA3_OK;
}

nsga3_status nsga3_batch_graph_builds(const nsga3_ctx* ctx, int64_t* builds)
{
    if (!ctx || !builds) return NSGA3_EINVAL;
    *builds = ctx->batch_builds;
    return NSGA3_OK;
}

nsga3_status nsga3_get_population(nsga3_ctx* ctx, float* X, float* F, int32_t* rank, void* stream)
{
    if (!ctx) return fail(ctx, NSGA3_EINVAL, "null context");
    cudaStream_t s = (cudaStream_t)stream;
    if (X) CK(cudaMemcpyAsync(X, ctx->v.X, (size_t)ctx->N * ctx->d * sizeof(float), cudaMemcpyDefault, s));
    if (F) CK(cudaMemcpyAsync(F, ctx->v.F, (size_t)ctx->N * ctx->m * sizeof(float), cudaMemcpyDefault, s));
    if (rank) CK(cudaMemcpyAsync(rank, ctx->v.rank, (size_t)ctx->N * sizeof(int32_t), cudaMemcpyDefault, s));
    return NSGA3_OK;
}

nsga3_status nsga3_set_population(nsga3_ctx* ctx, const float* X, const float* F, const int32_t* rank,
                                  void* stream)
{
    if (!ctx) return fail(ctx, NSGA3_EINVAL, "null context");
    cudaStream_t s = (cudaStream_t)stream;
    if (X) CK(cudaMemcpyAsync(ctx->v.X, X, (size_t)ctx->N * ctx->d * sizeof(float), cudaMemcpyDefault, s));
    if (F) CK(cudaMemcpyAsync(ctx->v.F, F, (size_t)ctx->N * ctx->m * sizeof(float), cudaMemcpyDefault, s));
    if (rank) CK(cudaMemcpyAsync(ctx->v.rank, rank, (size_t)ctx->N * sizeof(int32_t), cudaMemcpyDefault, s));
    return NSGA3_OK;
}

nsga3_status nsga3_get_children(nsga3_ctx* ctx, float* X, float* F, void* stream)
{
    if (!ctx) return fail(ctx, NSGA3_EINVAL, "null context");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = ctx->N;
    if (X) CK(cudaMemcpyAsync(X, ctx->v.X + N * ctx->d, N * ctx->d * sizeof(float), cudaMemcpyDefault, s));
    if (F) CK(cudaMemcpyAsync(F, ctx->v.F + N * ctx->m, N * ctx->m * sizeof(float), cudaMemcpyDefault, s));
    return NSGA3_OK;
}

nsga3_status nsga3_set_counter(nsga3_ctx* ctx, uint64_t gen, void* stream)
{
    if (!ctx || gen > 0xffffffffull) return fail(ctx, NSGA3_EINVAL, "bad arguments");
    k_set_gen<<<1, 1, 0, (cudaStream_t)stream>>>(ctx->v.ctrl, (uint32_t)gen);
    CK(cudaGetLastError());
    return NSGA3_OK;
}

nsga3_status nsga3_get_counter(nsga3_ctx* ctx, uint64_t* gen, void* stream)
{
    if (!ctx || !gen) return fail(ctx, NSGA3_EINVAL, "null argument");
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t g = 0;
    CK(cudaMemcpy(&g, &ctx->v.ctrl->gen, sizeof g, cudaMemcpyDeviceToHost));
    *gen = g;
    return NSGA3_OK;
}

nsga3_status nsga3_wait_probe(nsga3_ctx* ctx, void* stream)
{
    if (!ctx) return fail(ctx, NSGA3_EINVAL, "null context");
    CK(launch_wait_probe(ctx->v, (cudaStream_t)stream));
    ctx->host_launches += 1;
    return NSGA3_OK;
}

nsga3_status nsga3_sync(nsga3_ctx* ctx, void* stream)
{
    if (!ctx) return fail(ctx, NSGA3_EINVAL, "null context");
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return device_status(ctx, (cudaStream_t)stream, true);
}

nsga3_status nsga3_get_selection_info(nsga3_ctx* ctx, int32_t* info)
{
    if (!ctx || !info) return fail(ctx, NSGA3_EINVAL, "null argument");
    Ctrl c;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&c, ctx->v.ctrl, sizeof c, cudaMemcpyDeviceToHost));
    info[0] = c.l;
    info[1] = c.nS;
    info[2] = c.K;
    info[3] = c.nFl;
    info[4] = c.need_niche;
    info[5] = c.fallback;
    info[6] = c.passes;
    info[7] = c.nT;
    info[8] = c.Lstar;
    info[9] = c.rlev;
    info[10] = c.overflow;
    info[11] = c.recheck_miss;
    info[12] = (int32_t)c.peel_rows;
    return NSGA3_OK;
}

nsga3_status nsga3_get_selection_paths(nsga3_ctx* ctx, uint32_t* paths)
{
    if (!ctx || !paths) return fail(ctx, NSGA3_EINVAL, "null argument");
    CK(cudaDeviceSynchronize());
    uint32_t p = 0;
    CK(cudaMemcpy(&p, &ctx->v.ctrl->npath, sizeof p, cudaMemcpyDeviceToHost));
    *paths = p;
    return NSGA3_OK;
}

nsga3_status nsga3_get_dominance_stats(nsga3_ctx* ctx, int64_t* stats)
{
    if (!ctx || !stats) return fail(ctx, NSGA3_EINVAL, "null argument");
    CK(cudaDeviceSynchronize());
    unsigned long long d[8];
    CK(cudaMemcpy(d, ctx->v.ctrl->domstat, sizeof d, cudaMemcpyDeviceToHost));
    for (int t = 0; t < 8; ++t) stats[t] = (int64_t)d[t];
    return NSGA3_OK;
}

nsga3_status nsga3_select_smallest_probe(const uint64_t* keys, int n, int need, uint32_t* marks,
                                         uint32_t* paths, void* stream)
{
    if (!keys || !marks || !paths || n < 1 || need < 0 || need > n) return NSGA3_EINVAL;
    cudaError_t e = launch_select_probe(reinterpret_cast<const unsigned long long*>(keys), n, need, marks,
                                        paths, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return NSGA3_ECUDA;
    }
    return NSGA3_OK;
}

nsga3_status nsga3_issue_probe(int blocks_per_sm, int iters, int reps, double* instr_per_s, float* best_ms,
                               void* in_scratch, void* stream)
{
    if (!instr_per_s || !in_scratch || blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || reps < 1)
        return NSGA3_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return NSGA3_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = blocks_per_sm * sms;
    const float* in = static_cast<const float*>(in_scratch);
    uint32_t* sink = reinterpret_cast<uint32_t*>(static_cast<char*>(in_scratch) + 128);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch_issue_probe(in, blocks, iters, sink, s);  // warm-up
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch_issue_probe(in, blocks, iters, sink, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return NSGA3_ECUDA;
    }
    *instr_per_s = issue_probe_instructions(blocks, iters) / (best * 1e-3);
    if (best_ms) *best_ms = best;
    return NSGA3_OK;
}

nsga3_status nsga3_get_normalization(nsga3_ctx* ctx, double* zstar, double* a, int32_t* ext)
{
    if (!ctx) return fail(ctx, NSGA3_EINVAL, "null context");
    Ctrl c;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&c, ctx->v.ctrl, sizeof c, cudaMemcpyDeviceToHost));
    for (int q = 0; q < ctx->m; ++q) {
        if (zstar) zstar[q] = c.zstar[q];
        if (a) a[q] = c.a[q];
        if (ext) ext[q] = c.ext[q];
    }
    return NSGA3_OK;
}

nsga3_status nsga3_get_association(nsga3_ctx* ctx, int32_t* pi, double* dist)
{
    if (!ctx) return fail(ctx, NSGA3_EINVAL, "null context");
    CK(cudaDeviceSynchronize());
    if (pi) CK(cudaMemcpy(pi, ctx->v.pi, (size_t)ctx->n2 * sizeof(int32_t), cudaMemcpyDefault));
    if (dist) CK(cudaMemcpy(dist, ctx->v.dist, (size_t)ctx->n2 * sizeof(double), cudaMemcpyDefault));
    return NSGA3_OK;
}

nsga3_status nsga3_phase_times(nsga3_ctx* ctx, float* ms, int n)
{
    if (!ctx || !ms || n < 1) return fail(ctx, NSGA3_EINVAL, "bad arguments");
    if (!ctx->ev_mask) return fail(ctx, NSGA3_EINVAL, "phase timing is off (opts.phase_timing = 0)");
    // the last event that the graphs record closes the timed phases
    int last = EV_COUNT - 1;
    while (!((ctx->ev_mask >> last) & 1u)) --last;
    CK(cudaEventSynchronize(ctx->ev[last]));
    const int pairs[7][2] = {{EV_START, EV_VARY}, {EV_VARY, EV_RESET}, {EV_RESET, EV_DOM},
                             {EV_DOM, EV_PEEL},   {EV_PEEL, EV_NICHE}, {EV_NICHE, EV_END},
                             {EV_START, EV_END}};
    for (int t = 0; t < n && t < 7; ++t) {
        const unsigned need = (1u << pairs[t][0]) | (1u << pairs[t][1]);
        float x = -1.0f;  // a phase whose events are not recorded
        if ((ctx->ev_mask & need) == need)
            CK(cudaEventElapsedTime(&x, ctx->ev[pairs[t][0]], ctx->ev[pairs[t][1]]));
        ms[t] = x;
    }
    return NSGA3_OK;
}

nsga3_status nsga3_last_launches(nsga3_ctx* ctx, int32_t* launches)
{
    if (!ctx || !launches) return fail(ctx, NSGA3_EINVAL, "null argument");
    CK(cudaDeviceSynchronize());
    // reset, 3 sort, dominance, peel (every pass), 10 niching (the first
    // also writes the ranks back; the others return at once when no niching
    // is needed; one or two more for m > 10), compaction (+ finite check
    // for a selection; + variation, objective, gather, commit for a
    // generation)
    *launches = (ctx->last_kind == 1) ? select_launches(ctx) : generation_launches(ctx);
    return NSGA3_OK;
}

nsga3_status nsga3_total_launches(nsga3_ctx* ctx, int64_t* launches)
{
    if (!ctx || !launches) return fail(ctx, NSGA3_EINVAL, "null argument");
    CK(cudaDeviceSynchronize());
    *launches = ctx->host_launches;
    return NSGA3_OK;
}

}  // extern "C"
