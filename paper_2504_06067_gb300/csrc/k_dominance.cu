// k_dominance.cu -- bit-packed Pareto-dominance matrix (Alg. 1 line 3,
// "Non-dominated-sort"; dominance for minimisation, Eq. 1).
//
// Dom[I][j] (u32, word-major, I = i / 32) holds bit (i mod 32) = "i
// dominates j": a column j's dominators are NW words with j contiguous
// across rows, which the front peel reads coalesced.
//
// Work: only unordered pairs are compared.  A CTA owns a 256 x 256 tile of
// the upper block triangle; warp w takes row block ib = 8 * ti + w (lane =
// row i, its m objectives in registers) against each column block jb >= ib
// of the tile, with the column points broadcast from shared memory.  Per
// pair two predicate chains give A = all(f_i <= f_j), B = all(f_j <= f_i);
// "i dom j" = A & !B, "j dom i" = B & !A (identical vectors: neither).
// "j dom i" bits gathered over j are already column words Dom[jb][i];
// "i dom j" bits gathered over j are row words and are transposed in-warp
// (32 x 32 bit transpose by five shuffle stages) into Dom[ib][j].
// Padding rows/columns hold NaN: every compare with NaN is false, so they
// neither dominate nor are dominated.
//
// Bound: issue of FP32 compares (2m per unordered pair) -- ALU, not HBM.
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
    // tiles (ti <= tj) enumerated row by row: row ti starts at ti*T - ti*(ti-1)/2
    double b = 2.0 * T + 1.0;
    int r = (int)floor((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
    if (r < 0) r = 0;
    if (r > T - 1) r = T - 1;
    auto start = [&](long long x) { return x * T - x * (x - 1) / 2; };
    while (r > 0 && start(r) > t) --r;
    while (r + 1 < T && start(r + 1) <= t) ++r;
    ti = r;
    tj = r + (int)(t - start(r));
}

template <int M>
__global__ void __launch_bounds__(256) k_dominance(RunView v)
{
    constexpr int M4 = (M + 3) & ~3;
    __shared__ __align__(16) float srow[NSGA3_TILE * M4];
    __shared__ __align__(16) float scol[NSGA3_TILE * M4];
    if (read_status(v.ctrl)) return;
    const int T = v.ld / NSGA3_TILE;
    int ti, tj;
    decode_tile(blockIdx.x, T, ti, tj);
    const int r0 = ti * NSGA3_TILE, c0 = tj * NSGA3_TILE;
    for (int e = threadIdx.x; e < NSGA3_TILE * M; e += blockDim.x) {
        int p = e / M, q = e - p * M;
        srow[p * M4 + q] = v.F[(size_t)r0 * M + e];
        scol[p * M4 + q] = v.F[(size_t)c0 * M + e];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int ib = ti * 8 + warp;
    float fi[M];
#pragma unroll
    for (int q = 0; q < M; ++q) fi[q] = srow[(warp * 32 + lane) * M4 + q];

    for (int cb = 0; cb < 8; ++cb) {
        const int jb = tj * 8 + cb;
        if (jb < ib) continue;  // lower block triangle: done by the transposed tile
        uint32_t dij = 0, dji = 0;
        const float* colp = scol + cb * 32 * M4;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const float* fj = colp + k * M4;
            bool A = true, B = true;
#pragma unroll
            for (int q = 0; q < M; ++q) {
                float x = fj[q];
                A = A && (fi[q] <= x);
                B = B && (x <= fi[q]);
            }
            if (A && !B) dij |= 1u << k;
            if (B && !A) dji |= 1u << k;
        }
        uint32_t* D = v.Dom;
        // column i = ib*32 + lane, dominators j in block jb
        D[(size_t)jb * v.ld + ib * 32 + lane] = dji;
        if (jb != ib) {
            uint32_t t = warp_transpose32(dij);  // lane k: bits over i of column jb*32 + k
            D[(size_t)ib * v.ld + jb * 32 + lane] = t;
        }
    }
}

template <int M>
cudaError_t launch_dom_m(const RunView& v, cudaStream_t s)
{
    long long T = v.ld / NSGA3_TILE;
    long long tiles = T * (T + 1) / 2;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_dominance<M><<<(unsigned)tiles, 256, 0, s>>>(v);
    return cudaGetLastError();
}

}  // namespace

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
    default: return cudaErrorInvalidValue;
    }
}
