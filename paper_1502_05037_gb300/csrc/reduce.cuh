// Deterministic reduction helpers and the scalar slots of the SDMM solver
// state shared by the solver kernels and the fused operator kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace purify {

// ----------------------------------------------------------- scalar slots
enum Slot {
    S_RS = 0,        // r.r
    S_RS0 = 1,       // r0.r0 of the current x-update
    S_BETA = 2,
    S_ALPHA = 3,
    S_PAP = 4,
    S_OBJ = 5,       // ||W Psi^dagger x||_1 at the iterate entering the iteration
    S_OBJ_PREV = 6,
    S_CGCOUNT = 7,   // CG steps done (running total)
    S_XN2 = 8,       // ||x_new||^2
    S_DXN2 = 9,      // ||x_new - x_old||^2
    S_TOL2 = 10,     // cg_tol^2
    S_GMAX = 11,     // max |.| reduction result
    S_NORM2 = 12,    // generic norm^2 result
    S_SUM = 13,      // generic sum result
    S_RS_STEP = 15,      // r.r of CG steps of even / odd index (15, 16)
    S_ALPHA_STEP = 17,   // alpha of CG steps of even / odd index (17, 18)
    S_BLOCKS = 32    // then R entries of ||r_i||^2, then R of ||Phi_i x/nu - ybar_i||^2
};
enum Counter { C_PROX = 0, C_PROJ, C_CGI, C_ALPHA, C_UPD, C_REL, C_GEN, C_COUNT };
enum Flag { F_CGDONE = 0, F_NAN = 1, F_COUNT = 4 };

static constexpr int RB = 256;                 // threads per reduction block
static inline int red_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + RB * 4 - 1) / (RB * 4), 152 * 8)); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the first n lanes of a warp whose members are `mask` (result valid
// in lane 0); lane 0's additions are those of warp_sum when n = 32.
__device__ __forceinline__ double warp_sum_n(double v, unsigned mask, int n) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(mask, v, o);
        if (lane + o < n) v += w;
    }
    return v;
}

// Sum over the thread block (result valid in thread 0); any block size,
// including a partial last warp.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    const int n = min(32, (int)blockDim.x - wid * 32);
    v = n == 32 ? warp_sum(v) : warp_sum_n(v, n == 32 ? 0xffffffffu : ((1u << n) - 1u), n);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? sh[lane] : 0.0;
        v = n == 32 ? warp_sum(v) : warp_sum_n(v, n == 32 ? 0xffffffffu : ((1u << n) - 1u), n);
    }
    return v;
}

// Error-free transformation of a float sum (Knuth's TwoSum): s + e == a + b
// exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Sum over the thread block of per-thread float values (result valid in
// thread 0). Within a warp the running sum is an unevaluated pair hi + lo
// of floats, each step adding the partner's pair with TwoSum, so the warp sum
// carries about twice the float precision; the warp sums are then added in
// FP64 by warp 0 (in warp order). This keeps the block-level arithmetic off
// the slow FP64 pipe while the result matches an FP64 sum of the thread
// values to about 2^-44 relative.
__device__ __forceinline__ double block_sum_f(float v) {
    __shared__ double shf[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    const int n = min(32, (int)blockDim.x - wid * 32);
    const unsigned mask = n == 32 ? 0xffffffffu : ((1u << n) - 1u);
    float hi = v, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(mask, hi, o), l2 = __shfl_down_sync(mask, lo, o);
        if (lane + o < n) {
            float s, e;
            two_sum(hi, h2, s, e);
            hi = s;
            lo = __fadd_rn(__fadd_rn(lo, l2), e);
        }
    }
    __syncthreads();
    if (lane == 0) shf[wid] = (double)hi + (double)lo;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < nw ? shf[lane] : 0.0;
        t = warp_sum_n(t, blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u), nw);
    }
    return t;
}
// Block sum in the plan precision's reduction form: compensated float pairs
// for float values, FP64 for double values.
__device__ __forceinline__ double block_sum_t(float v) { return block_sum_f(v); }
__device__ __forceinline__ double block_sum_t(double v) { return block_sum(v); }

// True in every thread of the last block to arrive; partials written before
// the call by other blocks are then visible.
__device__ __forceinline__ bool arrive_last(unsigned* counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Ordered sum of part[0..n) by the calling block (result in thread 0).
__device__ __forceinline__ double ordered_sum(const double* part, int n) {
    double v = 0.0;
    // each thread sums a strided subsequence, then the block combines them
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(part + i);
    return block_sum(v);
}


}  // namespace purify
