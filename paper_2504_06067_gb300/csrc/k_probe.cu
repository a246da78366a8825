// k_probe.cu -- measured issue rate of the dominance test's instruction mix.
//
// The dominance build (k_dominance.cu) is bound by instruction issue: per
// pair it subtracts objectives on the FP32 pipe and ORs the sign bits of the
// differences three at a time on the integer pipe (LOP3), about two FP32
// subtractions per LOP3.  This probe issues that mix -- two FADDs and one
// 3-input LOP3 per step, eight independent chains per thread, no memory
// traffic -- from every SM, so that the roofline of the dominance kernel can
// use a measured ceiling instead of lanes x clock.  The instructions are
// inline PTX whose results feed later steps, so none of them is removed.
#include "kernels.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_issue_probe(const float* in, int iters, uint32_t* sink)
{
    float x[PROBE_CHAINS], y[PROBE_CHAINS];
    uint32_t acc[PROBE_CHAINS];
    const float base = in[threadIdx.x & 31];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) {
        x[c] = base + (float)c;
        y[c] = base * 0.5f + (float)(threadIdx.x + c);
        acc[c] = 0u;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) {
            float d0, d1;
            asm volatile("sub.f32 %0, %1, %2;" : "=f"(d0) : "f"(x[c]), "f"(y[c]));
            asm volatile("sub.f32 %0, %1, %2;" : "=f"(d1) : "f"(y[c]), "f"(x[c]));
            asm volatile("lop3.b32 %0, %1, %2, %3, 0xFE;"
                         : "=r"(acc[c])
                         : "r"(acc[c]), "r"(__float_as_uint(d0)), "r"(__float_as_uint(d1)));
            x[c] = d0;  // the next step depends on this one (x drifts by -y per step)
        }
    }
    uint32_t r = 0u;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) r ^= acc[c] ^ __float_as_uint(x[c]);
    if (r == 0x9E3779B9u) sink[0] = r;  // practically never taken; keeps the results live
}

}  // namespace

// Thread-instructions one launch issues: 3 per step and chain.
double issue_probe_instructions(int blocks, int iters)
{
    return 3.0 * PROBE_CHAINS * (double)iters * (double)blocks * PROBE_THREADS;
}

cudaError_t launch_issue_probe(const float* in, int blocks, int iters, uint32_t* sink, cudaStream_t s)
{
    k_issue_probe<<<blocks, PROBE_THREADS, 0, s>>>(in, iters, sink);
    return cudaGetLastError();
}
