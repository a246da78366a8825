// k_knapsack.cu -- second workload: 0-1 multi-objective knapsack (the
// MOKnapsack family of the paper's discrete experiments, Sec. IV / App. E).
//
// m knapsacks share d items with integer profits p[j][v] and weights
// w[j][v] and capacities c[j].  Variables are bits (stored as 0.0 / 1.0 in
// the population rows, so the selection and gather kernels are unchanged).
// Objectives (minimised, non-negative): f_j = P_j - sum_v p[j][v] x_v with
// P_j = sum_v p[j][v].  Infeasible bit strings are repaired: items leave in
// a fixed order (ascending best profit/weight ratio, built on the host)
// while a knapsack overflows, and the repaired bits replace the child.
// All arithmetic is integer, so the runs are bit-identical to a plain
// evaluation.
//   k_kp_init   bits from Philox(i*d + v, 0, 6): word 0 < 0.5 -> chosen
//   k_kp_vary   binary tournament on rank (as the continuous variation),
//               uniform crossover (Philox(q*d + v, gen, 2) word 0 < 0.5 swaps
//               the parents' bits between the children), bit-flip mutation
//               (Philox(q*d + v, gen, 3): word 0 < p_m flips child 2q, word 1
//               < p_m flips child 2q+1)
//   k_kp_eval   one warp per individual: loads, repair by warp prefix sums
//               over the removal order, objectives
#include "kernels.cuh"

namespace {

__global__ void k_kp_init(RunView v)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)v.N * v.d) return;
    const int i = (int)(e / v.d), var = (int)(e - (long long)i * v.d);
    const U4 r = philox((uint32_t)i * (uint32_t)v.d + (uint32_t)var, 0u, RNG_INIT, 0u, v.seed);
    v.X[e] = u01(r.x) < 0.5f ? 1.0f : 0.0f;
    if (var == 0) v.rank[i] = 0;
}

__global__ void k_kp_vary(RunView v)
{
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= v.N / 2) return;
    if (read_status(v.ctrl)) return;
    const int lane = lane_id();
    const uint32_t gen = v.ctrl->gen;
    const int N = v.N, d = v.d;
    const U4 t = philox((uint32_t)q, gen, RNG_TOURNAMENT, 0u, v.seed);
    const U4 cx = philox((uint32_t)q, gen, RNG_TOURNAMENT, 1u, v.seed);
    const uint32_t a1 = bounded(t.x, N), b1 = bounded(t.y, N);
    const uint32_t a2 = bounded(t.z, N), b2 = bounded(t.w, N);
    const uint32_t p1 = v.rank[b1] < v.rank[a1] ? b1 : a1;
    const uint32_t p2 = v.rank[b2] < v.rank[a2] ? b2 : a2;
    const bool cross = u01(cx.x) < v.p_c;
    float* x0 = v.X + (size_t)(N + 2 * q) * d;
    float* x1 = v.X + (size_t)(N + 2 * q + 1) * d;
    for (int var = lane; var < d; var += 32) {
        float c1 = v.X[(size_t)p1 * d + var], c2 = v.X[(size_t)p2 * d + var];
        const uint32_t ctr = (uint32_t)q * (uint32_t)d + (uint32_t)var;
        const U4 s = philox(ctr, gen, RNG_SBX, 0u, v.seed);
        if (cross && u01(s.x) < 0.5f) {
            const float tmp = c1;
            c1 = c2;
            c2 = tmp;
        }
        const U4 pm = philox(ctr, gen, RNG_PM, 0u, v.seed);
        if (u01(pm.x) < v.p_m) c1 = 1.0f - c1;
        if (u01(pm.y) < v.p_m) c2 = 1.0f - c2;
        x0[var] = c1;
        x1[var] = c2;
    }
}

constexpr int KB = 256;  // threads per block of k_kp_eval (8 individuals)

// Repair and objectives of rows [row0, row0 + n).  A warp owns a row.
__global__ void __launch_bounds__(KB) k_kp_eval(RunView v, int row0, int n)
{
    const int lane = lane_id();
    const int r = (blockIdx.x * KB + threadIdx.x) >> 5;
    if (r >= n) return;
    if (read_status(v.ctrl)) return;
    const int m = v.m, d = v.d;
    float* x = v.X + (size_t)(row0 + r) * d;
    // loads and excess per knapsack (integers; sums below 2^31 by the
    // limits checked at creation)
    int excess[NSGA3_FAST_M];
    bool over = false;
#pragma unroll
    for (int j = 0; j < NSGA3_FAST_M; ++j) {
        if (j >= m) {
            excess[j] = 0;
            continue;
        }
        int s = 0;
        for (int e = lane; e < d; e += 32)
            if (x[e] != 0.0f) s += __ldg(&v.kp_w[(size_t)j * d + e]);
        s = warp_sum(s);
        excess[j] = s - __ldg(&v.kp_cap[j]);
        over = over || excess[j] > 0;
    }
    // remove the shortest prefix of the removal order (chosen items only)
    // whose weights cover every excess
    for (int k0 = 0; over && k0 < d; k0 += 32) {
        const int k = k0 + lane;
        const int item = k < d ? __ldg(&v.kp_order[k]) : 0;
        const bool chosen = k < d && x[item] != 0.0f;
        bool done = true;
#pragma unroll
        for (int j = 0; j < NSGA3_FAST_M; ++j) {
            if (j >= m) continue;
            int wv = chosen ? __ldg(&v.kp_w[(size_t)j * d + item]) : 0;
            // inclusive prefix sum over the chunk
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wv, o);
                if (lane >= o) wv += y;
            }
            done = done && (wv >= excess[j]);
            excess[j] -= __shfl_sync(0xffffffffu, wv, 31);  // for the next chunk
        }
        const unsigned ok = __ballot_sync(0xffffffffu, done);
        const int stop = ok ? __ffs(ok) - 1 : 31;  // last removed position of this chunk
        if (chosen && lane <= stop) x[item] = 0.0f;
        if (ok) over = false;
    }
    __syncwarp();
    // objectives: profit left behind
#pragma unroll
    for (int j = 0; j < NSGA3_FAST_M; ++j) {
        if (j >= m) continue;
        int s = 0;
        for (int e = lane; e < d; e += 32)
            if (x[e] == 0.0f) s += __ldg(&v.kp_p[(size_t)j * d + e]);
        s = warp_sum(s);
        if (lane == 0) v.F[(size_t)(row0 + r) * m + j] = (float)s;
    }
}

}  // namespace

cudaError_t launch_kp_init(const RunView& v, cudaStream_t s)
{
    const long long n = (long long)v.N * v.d;
    k_kp_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_kp_eval<<<(unsigned)((v.N + KB / 32 - 1) / (KB / 32)), KB, 0, s>>>(v, 0, v.N);
    return cudaGetLastError();
}

cudaError_t launch_kp_vary_eval(const RunView& v, cudaStream_t s)
{
    const long long threads = (long long)(v.N / 2) * 32;
    k_kp_vary<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_kp_eval<<<(unsigned)((v.N + KB / 32 - 1) / (KB / 32)), KB, 0, s>>>(v, v.N, v.N);
    return cudaGetLastError();
}
