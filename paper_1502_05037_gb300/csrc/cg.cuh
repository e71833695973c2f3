// The scalars of one Chronopoulos-Gear CG step (see CgFold), reduced from the
// inverse row pass's per-block partial dot products by the last block of that
// pass to finish (all its threads, in a fixed order that does not depend on
// which block is last); the kernels that consume them only read the result.
#pragma once
#include "internal.h"
#include "reduce.cuh"

namespace purify {

// Step k's gamma = r.r and delta = r.A r from f.part[2 i], f.part[2 i + 1]
// (i < nparts, the producer's blocks), then
//   beta = gamma / gamma_prev (0 at step 0),
//   alpha = gamma / (delta - beta gamma / alpha_prev)  (gamma / delta at step 0),
// with gamma_prev, alpha_prev of step k - 1. Thread 0 records the scalars
// (S_ALPHA and S_BETA are the ones the next update applies), the stop and
// non-finite flags and the step count; the update of step k is applied unless
// the step stops the solve (gamma not above tol^2 gamma_0, or zero, or not
// finite). Every thread of the deciding block must call it.
__device__ __forceinline__ void cg_decide(const CgFold& f, int k, int nparts) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        s0 += __ldcg(f.part + 2 * i);
        s1 += __ldcg(f.part + 2 * i + 1);
    }
    s0 = block_sum(s0);
    s1 = block_sum(s1);
    if (threadIdx.x != 0) return;
    const double gam = s0, del = s1;
    double al, be = 0.0;
    if (k == 0) {
        al = del > 0.0 ? gam / del : 0.0;
    } else {
        const double gprev = f.scal[S_RS_STEP + ((k - 1) & 1)], aprev = f.scal[S_ALPHA_STEP + ((k - 1) & 1)];
        be = gprev > 0.0 ? gam / gprev : 0.0;
        const double den = del - (aprev > 0.0 ? be * gam / aprev : 0.0);
        al = den > 0.0 ? gam / den : 0.0;
    }
    const double g0 = k == 0 ? gam : f.scal[S_RS0];
    const bool bad = !(gam == gam) || !(al == al);
    const bool stop = bad || gam == 0.0 || gam <= f.scal[S_TOL2] * g0;
    if (k == 0) f.scal[S_RS0] = gam;
    f.scal[S_RS_STEP + (k & 1)] = gam;
    f.scal[S_ALPHA_STEP + (k & 1)] = al;
    f.scal[S_RS] = gam;
    f.scal[S_ALPHA] = al;
    f.scal[S_BETA] = be;
    f.scal[S_PAP] = del;
    if (bad) f.flags[F_NAN] = 1;
    if (stop) f.flags[F_CGDONE] = 1;
    else f.scal[S_CGCOUNT] += 1.0;
}

// The update decided by the last step's cg_decide: false when the solve
// stopped there (every thread of the block gets the same answer).
__device__ __forceinline__ bool cg_pending(const CgFold& f, double& al, double& be) {
    __shared__ int sh_stop;
    __shared__ double sh_al, sh_be;
    if (threadIdx.x == 0) {
        sh_stop = *reinterpret_cast<const volatile int*>(f.flags + F_CGDONE);
        sh_al = f.scal[S_ALPHA];
        sh_be = f.scal[S_BETA];
    }
    __syncthreads();
    al = sh_al;
    be = sh_be;
    return sh_stop == 0;
}

// A flag read once per block (thread 0) and shared, so that every thread of
// the block takes the same branch even while another block of the same
// kernel may be setting it.
__device__ __forceinline__ int block_flag(const int* flag) {
    __shared__ int sh;
    if (threadIdx.x == 0) sh = flag ? *reinterpret_cast<const volatile int*>(flag) : 0;
    __syncthreads();
    return sh;
}

}  // namespace purify
