// k_problem.cu -- reference directions, initial population and the fused
// variation + objective kernel around the selection.
//
// Reference directions (Sec. II-C): Das-Dennis lattice {k/p : sum k = p} in
// lexicographic order of k, optional inner layer (1 - tau)/m + tau z; one
// thread unranks one composition.  FP64 with _rn intrinsics.
//
// Variation (Alg. 1, crossover and mutation; Sec. III-A), one warp per offspring pair q:
//   tournament: Philox(q, gen, 1, 0) -> a1, b1, a2, b2 in [0, N); the lower
//   front wins, ties keep the first drawn; Philox(q, gen, 1, 1) word 0 < p_c
//   lets the pair cross.  SBX per variable v (Philox(q*d+v, gen, 2, 0)):
//   word 1 < 0.5 crosses v with spread beta from word 0, word 2 < 0.5 swaps
//   the children; clip to [0,1].  Polynomial mutation of variable v: word 3
//   of that block < p_m mutates child 2q with u = word 0 of
//   Philox(q*d+v, gen, 3, 0); word 1 of that block < p_m mutates child 2q+1
//   with u = its word 2 (two Philox blocks per pair and variable).
//   Children go to rows N + 2q and N + 2q + 1.  FP32 arithmetic.
// Objective (the softmax-simplex family): k = m - 1,
//   g = sum_{v >= k} (x_v - 0.5)^2, f_j = (1 + g) softmax(W x[0:k])_j,
//   evaluated in FP64 (sums left to right) and rounded to FP32; for m > 10
//   the products W x are summed as compensated FP32 dot products.
#include "kernels.cuh"

namespace {

__device__ long long binom_ll(int n, int k)
{
    if (k < 0 || k > n) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

__global__ void k_refdirs(int m, int p1, int p2, double tau, int w1, int w, double* Zd, double* nz,
                          float* Zh, int M4)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= w) return;
    const bool inner = t >= w1;
    const int p = inner ? p2 : p1;
    long long idx = inner ? t - w1 : t;
    double* z = Zd + (size_t)t * m;  // first the composition k, then k / p
    int left = p;
    for (int q = 0; q < m - 1; ++q) {
        int val = 0;
        for (; val <= left; ++val) {
            const long long n = binom_ll(left - val + (m - q - 2), m - q - 2);
            if (idx < n) break;
            idx -= n;
        }
        z[q] = (double)val;
        left -= val;
    }
    z[m - 1] = (double)left;
    double s = 0.0;
    for (int q = 0; q < m; ++q) {
        double zq = __ddiv_rn(z[q], (double)p);
        if (inner) {
            const double a = __ddiv_rn(__dsub_rn(1.0, tau), (double)m);
            const double b = __dmul_rn(tau, zq);
            zq = __dadd_rn(a, b);
        }
        z[q] = zq;
        s = __dadd_rn(s, __dmul_rn(zq, zq));
    }
    const double n = __dsqrt_rn(s);
    nz[t] = n;
    for (int q = 0; q < M4; ++q) Zh[(size_t)t * M4 + q] = q < m ? __double2float_rn(__ddiv_rn(z[q], n)) : 0.0f;
}

// Objective of rows [row0, row0 + n): a block covers R = obj_rows(m) rows.
//   g = sum_{v >= m-1} (x_v - 0.5)^2: each term is formed exactly as a
//   float-float value (x - 0.5 by Fast2Sum, the square by an FMA product
//   error) and the terms are added in float-float (TwoSum) by a warp per row
//   with coalesced loads, then a warp reduction; the float-float sum is
//   within ~2^-44 relative of the exact sum, so (1 + g) in FP64 matches a
//   left-to-right FP64 sum to far below the final FP32 rounding.  This keeps
//   the sum off GB300's FP64 pipe (1/64 of the FP32 rate).
//   Thread (row, j) forms a_j = sum_v W_jv x_v in FP64 (left to right) and
//   e_j = exp(a_j); the row's denominator adds e_0..e_{m-1} in order once;
//   f_j = (1 + g) e_j / den, rounded to FP32.
constexpr int OR = 32;
constexpr int OT = 256;

// rows per block: 32 for m <= 10; above, about 256 (row, objective) pairs
// per block, one per thread, so that the FP64 dot products of many
// objectives spread over the whole GPU (R x m exponentials in shared memory)
inline int obj_rows(int m)
{
    if (m <= NSGA3_FAST_M) return OR;
    const int r = OT / m;
    return r < 1 ? 1 : r;
}
inline size_t obj_smem(int m) { return (size_t)obj_rows(m) * (m + 2) * sizeof(double); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// m > NSGA3_FAST_M: a_j = sum_v W_jv x_v for RB rows x 128 objectives per
// CTA as compensated FP32 dot products (each product split exactly into
// p + e by an FMA, the sum carried as a float-float pair by TwoSum; Ogita,
// Rump and Oishi's Dot2), then e_j = exp(a_j) in FP64 into v.fprime (free
// during the variation).  Dot2's error, about (k 2^-24)^2 of sum |W x|, is
// far below the FP32 rounding of f: the FP64 evaluation of the m
// exponentials' products would take the FP64 pipe (1/64 of FP32) for
// m (m-1) N operations.
constexpr int RB = 4;     // rows per CTA
constexpr int DT = 128;   // objectives per CTA

__global__ void __launch_bounds__(DT) k_obj_dot(RunView v, int row0, int n)
{
    extern __shared__ float xs[];  // RB x k
    const int m = v.m, d = v.d, k = m - 1;
    const int base = blockIdx.x * RB;
    const int rows = min(RB, n - base);
    for (int e = threadIdx.x; e < RB * k; e += DT) {
        const int r = e / k, c = e - r * k;
        xs[e] = r < rows ? v.X[(size_t)(row0 + base + r) * d + c] : 0.0f;
    }
    __syncthreads();
    const int j = blockIdx.y * DT + threadIdx.x;
    if (j >= m) return;
    float hi[RB], lo[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        hi[r] = 0.0f;
        lo[r] = 0.0f;
    }
#pragma unroll 8
    for (int e = 0; e < k; ++e) {
        const float w = __ldg(&v.Wt[(size_t)e * m + j]);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const float x = xs[r * k + e];
            const float p = __fmul_rn(w, x);
            const float pe = __fmaf_rn(w, x, -p);  // w x = p + pe exactly
            float s1, t1;
            two_sum(hi[r], p, s1, t1);
            hi[r] = s1;
            lo[r] = __fadd_rn(lo[r], __fadd_rn(t1, pe));
        }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
        if (r < rows) {
            const double a = __dadd_rn((double)hi[r], (double)lo[r]);
            v.fprime[(size_t)(base + r) * m + j] = exp(a);
        }
}

__global__ void __launch_bounds__(OT) k_objective(RunView v, int row0, int n, int R)
{
    extern __shared__ double sobj[];
    double* sg = sobj;        // R
    double* sden = sg + R;    // R
    double* se = sden + R;    // R x m
    const int m = v.m, d = v.d, k = m - 1;
    const int base = blockIdx.x * R;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int rr = warp; rr < R; rr += OT / 32) {
        float sh = 0.0f, sl = 0.0f;
        if (base + rr < n) {
            const float* x = v.X + (size_t)(row0 + base + rr) * d;
            for (int e = k + lane; e < d; e += 32) {
                const float xv = x[e];
                const float th = __fsub_rn(xv, 0.5f);
                // Fast2Sum error of x + (-0.5); zero when x >= 0.25 (Sterbenz)
                const float tl = xv < 0.25f ? __fsub_rn(xv, __fadd_rn(th, 0.5f)) : 0.0f;
                const float p = __fmul_rn(th, th);
                const float pl = __fmaf_rn(th, th, -p) + 2.0f * th * tl;
                float s1, e1;
                two_sum(sh, p, s1, e1);
                sh = s1;
                sl = sl + (e1 + pl);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
            const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
            float s1, e1;
            two_sum(sh, oh, s1, e1);
            sh = s1;
            sl = sl + (ol + e1);
        }
        if (lane == 0) sg[rr] = __dadd_rn((double)sh, (double)sl);
    }
    for (int idx = threadIdx.x; idx < R * m; idx += OT) {
        const int rr = idx / m, j = idx - rr * m;
        if (base + rr >= n) continue;
        if (m > NSGA3_FAST_M) {  // exponentials from k_obj_dot
            se[idx] = v.fprime[(size_t)(base + rr) * m + j];
            continue;
        }
        const float* x = v.X + (size_t)(row0 + base + rr) * d;
        double a = 0.0;
        for (int e = 0; e < k; ++e) a = __dadd_rn(a, __dmul_rn((double)v.Wobj[j * k + e], (double)x[e]));
        se[idx] = exp(a);
    }
    __syncthreads();
    if (threadIdx.x < R && base + threadIdx.x < n) {
        double den = 0.0;
        for (int t = 0; t < m; ++t) den = __dadd_rn(den, se[threadIdx.x * m + t]);
        sden[threadIdx.x] = den;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < R * m; idx += OT) {
        const int rr = idx / m, j = idx - rr * m;
        if (base + rr >= n) continue;
        const double f = __dmul_rn(__dadd_rn(1.0, sg[rr]), __ddiv_rn(se[idx], sden[rr]));
        v.F[(size_t)(row0 + base + rr) * m + j] = __double2float_rn(f);
    }
}


__global__ void k_init(RunView v)
{
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    const int lane = lane_id();
    float* xrow = v.X + (size_t)i * v.d;
    for (int e = lane; e < v.d; e += 32) {
        U4 r = philox((uint32_t)i * (uint32_t)v.d + (uint32_t)e, 0u, RNG_INIT, 0u, v.seed);
        xrow[e] = u01(r.x);
    }
    if (lane == 0) v.rank[i] = 0;
}

// Bounded polynomial mutation (Deb and Goyal): y + dq with
// dq = val^(1/(eta+1)) - 1 (lower branch) or 1 - val^(1/(eta+1)) (upper
// branch).  val^e - 1 is formed as expm1(e log val), which keeps dq
// accurate relative to itself; pow(val, e) - 1 would lose the bits of dq
// below the ulp of 1 when val is near 1.
__device__ __forceinline__ float pm_mutate(float y, float u, float eta_m)
{
    const float mp = 1.0f / (eta_m + 1.0f);
    // one powf, logf and expm1f on the chosen branch's operands (the same
    // values as calling them in each branch)
    const bool lo = u < 0.5f;
    const float xy = lo ? 1.0f - y : 1.0f - (1.0f - y);
    const float pw = powf(xy, eta_m + 1.0f);
    const float val = lo ? 2.0f * u + (1.0f - 2.0f * u) * pw : 2.0f * (1.0f - u) + 2.0f * (u - 0.5f) * pw;
    const float ex = expm1f(mp * logf(val));
    const float dq = lo ? ex : -ex;
    y = y + dq;
    return fminf(fmaxf(y, 0.0f), 1.0f);
}

// Variation of one pair (one warp, lanes over the variables): binary
// tournament on rank (first drawn wins ties), SBX with per-variable
// crossover and child swap, polynomial mutation, clip to [0, 1].  Calls
// out(var, c1, c2) for every variable in lane order var = lane + 32 t.
// SBX is written c1,2 = (y1 + y2)/2 -/+ (beta/2)(y2 - y1) with one FMA, the
// same value as ((1 + beta) y1 + (1 - beta) y2)/2 with fewer roundings.
template <class Out>
__device__ __forceinline__ void vary_pair(const RunView& v, int q, uint32_t gen, Out out)
{
    const int lane = lane_id();
    const int N = v.N, d = v.d;
    const U4 t = philox((uint32_t)q, gen, RNG_TOURNAMENT, 0u, v.seed);
    const U4 cx = philox((uint32_t)q, gen, RNG_TOURNAMENT, 1u, v.seed);
    const uint32_t a1 = bounded(t.x, N), b1 = bounded(t.y, N);
    const uint32_t a2 = bounded(t.z, N), b2 = bounded(t.w, N);
    const uint32_t p1 = v.rank[b1] < v.rank[a1] ? b1 : a1;
    const uint32_t p2 = v.rank[b2] < v.rank[a2] ? b2 : a2;
    const bool cross = u01(cx.x) < v.p_c;
    const float e = 1.0f / (v.eta_c + 1.0f);
    for (int var = lane; var < d; var += 32) {
        const float y1 = v.X[(size_t)p1 * d + var], y2 = v.X[(size_t)p2 * d + var];
        float c1 = y1, c2 = y2;
        const U4 sb = philox((uint32_t)q * (uint32_t)d + (uint32_t)var, gen, RNG_SBX, 0u, v.seed);
        if (cross && u01(sb.y) < 0.5f) {
            const float u = u01(sb.x);
            // one powf on the chosen base (the same value as either branch's call)
            const float base = (u <= 0.5f) ? 2.0f * u : 1.0f / (2.0f * (1.0f - u));
            const float beta = powf(base, e);
            const float mid = 0.5f * (y1 + y2), hb = 0.5f * beta, dy = y2 - y1;
            c1 = fmaf(-hb, dy, mid);
            c2 = fmaf(hb, dy, mid);
            if (u01(sb.z) < 0.5f) {
                const float tmp = c1;
                c1 = c2;
                c2 = tmp;
            }
            c1 = fminf(fmaxf(c1, 0.0f), 1.0f);
            c2 = fminf(fmaxf(c2, 0.0f), 1.0f);
        }
        const bool mut0 = u01(sb.w) < v.p_m;
        const U4 pm = philox((uint32_t)q * (uint32_t)d + (uint32_t)var, gen, RNG_PM, 0u, v.seed);
        if (mut0) c1 = pm_mutate(c1, u01(pm.x), v.eta_m);
        if (u01(pm.y) < v.p_m) c2 = pm_mutate(c2, u01(pm.z), v.eta_m);
        out(var, c1, c2);
    }
}

// Variation only (m > 10: the objective follows in k_obj_dot + k_objective).
__global__ void k_vary(RunView v)
{
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= v.N / 2) return;
    if (read_status(v.ctrl)) return;
    const uint32_t gen = v.ctrl->gen;
    float* x0 = v.X + (size_t)(v.N + 2 * q) * v.d;
    float* x1 = v.X + (size_t)(v.N + 2 * q + 1) * v.d;
    vary_pair(v, q, gen, [&](int var, float c1, float c2) {
        x0[var] = c1;
        x1[var] = c2;
    });
}

// g term (x - 0.5)^2 of one variable added into a float-float sum (sh, sl):
// x - 0.5 by Fast2Sum (exact when x >= 0.25), the square's error by an FMA
__device__ __forceinline__ void g_add(float xv, float& sh, float& sl)
{
    const float th = __fsub_rn(xv, 0.5f);
    const float tl = xv < 0.25f ? __fsub_rn(xv, __fadd_rn(th, 0.5f)) : 0.0f;
    const float p = __fmul_rn(th, th);
    const float pl = __fmaf_rn(th, th, -p) + 2.0f * th * tl;
    float s1, e1;
    two_sum(sh, p, s1, e1);
    sh = s1;
    sl = sl + (e1 + pl);
}

// Variation fused with the softmax-simplex objective (m <= 10): one warp
// per pair; each lane keeps its children's first m - 1 variables and its
// float-float partial sums of g while it writes the children, then the warp
// reduces g, lanes 0..m-1 (child 0) and 16..16+m-1 (child 1) form
// a_j = sum_e W_je x_e and e_j = exp(a_j), every lane adds e_0..e_{m-1} in
// order, and lane j writes f_j = (1 + g) e_j / den rounded to FP32.  The
// children are never read back.
//
// The arithmetic is FP32 with error-free transformations instead of FP64
// (1/64 of the FP32 rate on GB300): a_j as a compensated dot product
// (TwoProduct by FMA, TwoSum; Ogita, Rump and Oishi's Dot2) a_hi + a_lo;
// e_j = expf(a_hi) (1 + a_lo), so the rounding of a never reaches the
// exponential (an absolute error of a becomes a relative error of e_j);
// den and 1 + g as float-float sums; one correctly rounded division.  The
// result is within about 4 ulp (2.4e-7) of (1 + g) e_j / den: expf's 2 ulp,
// the division's and the last product's half ulp.
template <int M>
__global__ void __launch_bounds__(256) k_vary_eval(RunView v)
{
    constexpr int K = M - 1;
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= v.N / 2) return;
    if (read_status(v.ctrl)) return;
    const int lane = lane_id();
    const uint32_t gen = v.ctrl->gen;
    const int N = v.N;
    float* x0 = v.X + (size_t)(N + 2 * q) * v.d;
    float* x1 = v.X + (size_t)(N + 2 * q + 1) * v.d;
    float gh0 = 0.0f, gl0 = 0.0f, gh1 = 0.0f, gl1 = 0.0f;
    float xk0 = 0.0f, xk1 = 0.0f;
    vary_pair(v, q, gen, [&](int var, float c1, float c2) {
        x0[var] = c1;
        x1[var] = c2;
        if (var < K) {
            xk0 = c1;
            xk1 = c2;
        } else {
            g_add(c1, gh0, gl0);
            g_add(c2, gh1, gl1);
        }
    });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float s1, e1;
        const float oh0 = __shfl_xor_sync(0xffffffffu, gh0, o), ol0 = __shfl_xor_sync(0xffffffffu, gl0, o);
        two_sum(gh0, oh0, s1, e1);
        gh0 = s1;
        gl0 = gl0 + (ol0 + e1);
        const float oh1 = __shfl_xor_sync(0xffffffffu, gh1, o), ol1 = __shfl_xor_sync(0xffffffffu, gl1, o);
        two_sum(gh1, oh1, s1, e1);
        gh1 = s1;
        gl1 = gl1 + (ol1 + e1);
    }
    const int j = lane & 15;
    const bool second = lane >= 16;
    float ah = 0.0f, al = 0.0f;
#pragma unroll
    for (int e = 0; e < K; ++e) {
        const float xe0 = __shfl_sync(0xffffffffu, xk0, e);
        const float xe1 = __shfl_sync(0xffffffffu, xk1, e);
        if (j < M) {
            const float w = v.Wobj[j * K + e], x = second ? xe1 : xe0;
            const float p = __fmul_rn(w, x);
            const float pe = __fmaf_rn(w, x, -p);
            float s1, e1;
            two_sum(ah, p, s1, e1);
            ah = s1;
            al = al + (e1 + pe);
        }
    }
    float ex = 0.0f;
    if (j < M) {
        const float E = expf(ah);
        ex = __fmaf_rn(E, al, E);
    }
    float dh0 = 0.0f, dl0 = 0.0f, dh1 = 0.0f, dl1 = 0.0f;
#pragma unroll
    for (int t = 0; t < M; ++t) {
        float s1, e1;
        two_sum(dh0, __shfl_sync(0xffffffffu, ex, t), s1, e1);
        dh0 = s1;
        dl0 += e1;
        two_sum(dh1, __shfl_sync(0xffffffffu, ex, 16 + t), s1, e1);
        dh1 = s1;
        dl1 += e1;
    }
    if (j < M) {
        const float dh = second ? dh1 : dh0, dl = second ? dl1 : dl0;
        float r = __fdiv_rn(ex, dh);
        r = __fmaf_rn(-r, __fdiv_rn(dl, dh), r);  // e / (dh + dl)
        const float gh = second ? gh1 : gh0, gl = second ? gl1 : gl0;
        float Gh, Ge;
        two_sum(1.0f, gh, Gh, Ge);
        const float Gl = Ge + gl;  // 1 + g = Gh + Gl
        v.F[(size_t)(N + 2 * q + (second ? 1 : 0)) * M + j] = __fmaf_rn(r, Gh, r * Gl);
    }
}

cudaError_t launch_obj_dot(const RunView& v, int row0, int n, cudaStream_t s)
{
    if (!v.Wt) return cudaErrorInvalidValue;
    const size_t sm = (size_t)RB * (v.m - 1) * sizeof(float);
    k_obj_dot<<<dim3((n + RB - 1) / RB, (v.m + DT - 1) / DT), DT, sm, s>>>(v, row0, n);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_refdirs(const RunView& v, int p1, int p2, double tau, double* Zd, double* nz,
                           float* Zh, cudaStream_t s)
{
    long long w1 = 1;
    {
        // C(p1 + m - 1, m - 1)
        long long r = 1;
        for (int i = 1; i <= v.m - 1; ++i) r = r * (p1 + i) / i;
        w1 = r;
    }
    k_refdirs<<<(v.w + 127) / 128, 128, 0, s>>>(v.m, p1, p2, tau, (int)w1, v.w, Zd, nz, Zh, v.M4);
    return cudaGetLastError();
}

cudaError_t launch_init(const RunView& v, cudaStream_t s)
{
    if (v.problem == 1) return launch_kp_init(v, s);
    long long threads = (long long)v.N * 32;
    k_init<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (v.m > NSGA3_FAST_M) {
        e = launch_obj_dot(v, 0, v.N, s);
        if (e != cudaSuccess) return e;
    }
    const int R = obj_rows(v.m);
    k_objective<<<(v.N + R - 1) / R, OT, obj_smem(v.m), s>>>(v, 0, v.N, R);
    return cudaGetLastError();
}

cudaError_t launch_vary_eval(const RunView& v, cudaStream_t s)
{
    if (v.problem == 1) return launch_kp_vary_eval(v, s);
    long long threads = (long long)(v.N / 2) * 32;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (v.m <= NSGA3_FAST_M) {
        switch (v.m) {
        case 2: k_vary_eval<2><<<blocks, 256, 0, s>>>(v); break;
        case 3: k_vary_eval<3><<<blocks, 256, 0, s>>>(v); break;
        case 4: k_vary_eval<4><<<blocks, 256, 0, s>>>(v); break;
        case 5: k_vary_eval<5><<<blocks, 256, 0, s>>>(v); break;
        case 6: k_vary_eval<6><<<blocks, 256, 0, s>>>(v); break;
        case 7: k_vary_eval<7><<<blocks, 256, 0, s>>>(v); break;
        case 8: k_vary_eval<8><<<blocks, 256, 0, s>>>(v); break;
        case 9: k_vary_eval<9><<<blocks, 256, 0, s>>>(v); break;
        default: k_vary_eval<10><<<blocks, 256, 0, s>>>(v); break;
        }
        return cudaGetLastError();
    }
    k_vary<<<blocks, 256, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_obj_dot(v, v.N, v.N, s);
    if (e != cudaSuccess) return e;
    const int R = obj_rows(v.m);
    k_objective<<<(v.N + R - 1) / R, OT, obj_smem(v.m), s>>>(v, v.N, v.N, R);
    return cudaGetLastError();
}
