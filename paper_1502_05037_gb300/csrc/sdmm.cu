// SDMM solve of problem (3) (Sec. 1, Eqs. 1-3) and SARA reweighting.
//
// Functions and linear maps (Combettes & Pesquet's SDMM): f1 = ||W .||_1
// with L1 = Psi^dagger, f2 = indicator of the R l2 balls of Eq. 3 with
// L2 = Phi / nu, f3 = indicator of R_+^N with L3 = I. One iteration from the
// current x (multipliers start at zero):
//   s1 = soft(Psi^dagger x + z1, gamma w);        z1 += Psi^dagger x - s1
//   s2_i = proj_{B(ybar_i, eps_i / nu)}(Phi_i x / nu + z2_i); z2 += Phi x / nu - s2
//   s3 = max(x + z3, 0);                           z3 += x - s3
//   x  = CG solution of (2 I + Re Phi^H Phi / nu^2) x = b,
//        b = Psi(s1 - z1) + Re Phi^H (s2 - z2) / nu + (s3 - z3), warm start.
// The CG residual b - A x is formed with a single adjoint: Phi x / nu is
// already at hand from the projection step, so
//   b - A x = Psi(s1 - z1) + (s3 - z3) - 2 x + Re Phi^H (s2 - z2 - Phi x / nu) / nu.
// Reductions (norms, dot products, objective) have a fixed order: each thread
// accumulates its few elements (at most 16) in the plan precision, the
// thread, warp and block partials are summed in FP64, and the block partials
// are summed in index order by the last block to finish. (GB300 issues FP64
// arithmetic at a small fraction of the FP32 rate, so per-element FP64 work
// would bound these kernels.)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cg.cuh"
#include "internal.h"
#include "launch.h"
#include "reduce.cuh"

namespace purify {

// ------------------------------------------------------------ kernels
// prox of gamma ||W .||_1 with the multiplier update; c holds Psi^dagger x on
// entry and s1 - z1 on exit. Objective partial sum |w v|.
template <typename T>
__global__ void k_prox_l1(T* __restrict__ c, T* __restrict__ z1, const T* __restrict__ w, int64_t D, double gamma,
                          double* part, unsigned* counters, double* scal, int eval_only) {
    pdl_wait();
    T obj = 0;  // per-thread partial in the plan precision, FP64 across threads
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x) {
        T v = c[d];
        T wd = w ? w[d] : T(1);
        obj += fabs(wd * v);
        if (eval_only) continue;
        T zz = z1[d];
        T t = v + zz;
        T thr = (T)gamma * wd;
        T mag = fabs(t) - thr;
        T s = mag > T(0) ? copysign(mag, t) : T(0);
        T zn = zz + v - s;
        z1[d] = zn;
        c[d] = s - zn;
    }
    double b = block_sum_t(obj);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
    if (arrive_last(counters + C_PROX)) {
        double tot = ordered_sum(part, gridDim.x);
        if (threadIdx.x == 0) {
            scal[S_OBJ_PREV] = scal[S_OBJ];
            scal[S_OBJ] = tot;
            counters[C_PROX] = 0;
        }
    }
    pdl_trigger();
}

// Per-block norms over visibility chunks: ||v2 + z2 - ybar||^2 (z2 may be
// null) and ||v2 - ybar||^2.
template <typename T>
__global__ void k_proj_norms(const typename cplx_of<T>::type* __restrict__ v2,
                             const typename cplx_of<T>::type* __restrict__ z2,
                             const typename cplx_of<T>::type* __restrict__ ybar, const int* __restrict__ cblk,
                             const int* __restrict__ cbeg, const int* __restrict__ cend, int nchunks, int R,
                             const int* __restrict__ chunk_first, double* part, unsigned* counters, double* scal) {
    pdl_wait();
    using C = typename cplx_of<T>::type;
    const int ch = blockIdx.x;
    T a = 0, e = 0;  // per-thread partials (at most 16 terms), FP64 across threads
    for (int m = cbeg[ch] + threadIdx.x; m < cend[ch]; m += blockDim.x) {
        C v = v2[m], y = ybar[m];
        T rx = v.x - y.x, ry = v.y - y.y;
        e += rx * rx + ry * ry;
        if (z2) {
            C z = z2[m];
            T tx = rx + z.x, ty = ry + z.y;
            a += tx * tx + ty * ty;
        }
    }
    double sa = block_sum_t(a);
    double se = block_sum_t(e);
    if (threadIdx.x == 0) { part[2 * ch] = sa; part[2 * ch + 1] = se; }
    if (arrive_last(counters + C_PROJ)) {
        // chunk_first[r] .. chunk_first[r+1] are block r's chunks
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
            double sa2 = 0.0, se2 = 0.0;
            for (int k = chunk_first[r]; k < chunk_first[r + 1]; ++k) {
                sa2 += __ldcg(part + 2 * k);
                se2 += __ldcg(part + 2 * k + 1);
            }
            if (z2) scal[S_BLOCKS + r] = sa2;
            scal[S_BLOCKS + R + r] = se2;
        }
        if (threadIdx.x == 0) counters[C_PROJ] = 0;
    }
    pdl_trigger();
}

// Projection onto each block's ball plus multiplier update, s2 = proj(v2 + z2),
// z2 += v2 - s2, with v2 (= Phi x / nu) replaced by
//   out_mode 0: s2 - z2 - v2 (the fused CG residual),
//   out_mode 1: s2 - z2 (the embedded normal operator forms A x separately),
//   out_mode 2: z2 (the primal-dual solver: z2 = p2 / sigma, the dual
//               variable of the balls; see pd_solve).
template <typename T>
__global__ void k_proj_apply(typename cplx_of<T>::type* __restrict__ v2, typename cplx_of<T>::type* __restrict__ z2,
                             const typename cplx_of<T>::type* __restrict__ ybar, const int* __restrict__ cblk,
                             const int* __restrict__ cbeg, const int* __restrict__ cend,
                             const double* __restrict__ eps, const double* __restrict__ scal, int R, int out_mode) {
    pdl_wait();
    using C = typename cplx_of<T>::type;
    const int ch = blockIdx.x;
    const int r = cblk[ch];
    const double nr = sqrt(scal[S_BLOCKS + r]);
    const double e = eps[r];
    const T f = nr > e ? (T)(e / nr) : T(1);
    const T vk = out_mode == 0 ? T(1) : T(0);
    const T sk = out_mode == 2 ? T(0) : T(1);
    for (int m = cbeg[ch] + threadIdx.x; m < cend[ch]; m += blockDim.x) {
        C v = v2[m], z = z2[m], y = ybar[m];
        T rx = v.x + z.x - y.x, ry = v.y + z.y - y.y;
        T sx = y.x + rx * f, sy = y.y + ry * f;
        T zx = z.x + v.x - sx, zy = z.y + v.y - sy;
        z2[m] = cmake<C>(zx, zy);
        v2[m] = out_mode == 2 ? cmake<C>(zx, zy) : cmake<C>(sk * sx - zx - vk * v.x, sk * sy - zy - vk * v.y);
    }
    pdl_trigger();
}

// Primal-dual dual step on the l1 term: p1 = clip(p1 + sigma c, -w, w), c =
// Psi^dagger xbar (w = 1 without weights).
template <typename T>
__global__ void k_pd_dual_l1(const T* __restrict__ c, T* __restrict__ p1, const T* __restrict__ w, int64_t D,
                             T sigma) {
    pdl_wait();
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x) {
        const T wd = w ? w[d] : T(1);
        const T t = p1[d] + sigma * c[d];
        p1[d] = t > wd ? wd : (t < -wd ? -wd : t);
    }
    pdl_trigger();
}

// Primal-dual primal step: x_new = max(x - tau g, 0), xbar = 2 x_new - x.
template <typename T>
__global__ void k_pd_primal(T* __restrict__ x, const T* __restrict__ g, T* __restrict__ xbar, int64_t N, T tau) {
    pdl_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const T xv = x[i];
        T xn = xv - tau * g[i];
        xn = xn > T(0) ? xn : T(0);
        xbar[i] = T(2) * xn - xv;
        x[i] = xn;
    }
    pdl_trigger();
}

// Positivity step and the image-space part of the CG residual:
//   s3 = max(x + z3, 0); z3 += x - s3; addend = psi_out + (s3 - z3) - 2x.
template <typename T>
__global__ void k_positivity(const T* __restrict__ x, T* __restrict__ z3, const T* __restrict__ psi_out,
                             T* __restrict__ addend, T* __restrict__ xprev, int64_t N) {
    pdl_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        T xv = x[i], zz = z3[i];
        T t = xv + zz;
        T s3 = t > T(0) ? t : T(0);
        T zn = zz + xv - s3;
        z3[i] = zn;
        addend[i] = psi_out[i] + (s3 - zn) - T(2) * xv;
        xprev[i] = xv;
    }
    pdl_trigger();
}

template <typename T>
__global__ void k_relchange(T* __restrict__ x, const T* __restrict__ xprev, int64_t N, double* part,
                            unsigned* counters, double* scal, CgFold fold) {
    pdl_wait();
    // the last CG step's update first, unless the solve stopped (see CgFold)
    bool pending = false;
    T alpha = T(0), beta = T(0);
    if (fold.x) {
        double al, be;
        if (cg_pending(fold, al, be)) {
            pending = true;
            alpha = (T)al;
            beta = (T)be;
        }
    }
    T* const r = static_cast<T*>(fold.r);
    T* const sv = static_cast<T*>(fold.s);
    const T* const u = static_cast<const T*>(fold.u);
    T* const pdir = static_cast<T*>(fold.p);
    T a = 0, d = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        T xv = x[i];
        if (pending) {
            const T pv = r[i] + beta * pdir[i];
            const T s2 = u[i] + beta * sv[i];
            pdir[i] = pv;
            sv[i] = s2;
            xv += alpha * pv;
            x[i] = xv;
            r[i] = r[i] - alpha * s2;
        }
        const T dv = xv - xprev[i];
        a += xv * xv;
        d += dv * dv;
    }
    double ba = block_sum_t(a);
    double bd = block_sum_t(d);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = ba; part[2 * blockIdx.x + 1] = bd; }
    if (arrive_last(counters + C_REL)) {
        // fixed-order block-parallel sum of the block partials
        double sa = 0.0, sd = 0.0;
        for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
            sa += __ldcg(part + 2 * k);
            sd += __ldcg(part + 2 * k + 1);
        }
        sa = block_sum(sa);
        sd = block_sum(sd);
        if (threadIdx.x == 0) {
            scal[S_XN2] = sa;
            scal[S_DXN2] = sd;
            counters[C_REL] = 0;
        }
    }
    pdl_trigger();
}

// Generic reductions: mode 0 sum of squares, 1 max |.|, 2 sum, 3 sum (v - mean)^2 with mean = scal[S_SUM]/n
template <typename T>
__global__ void k_reduce(const T* __restrict__ v, int64_t n, int mode, double* part, unsigned* counters,
                         double* scal, int slot) {
    double acc = 0.0;
    const double mean = mode == 3 ? scal[S_SUM] / (double)n : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double a = v[i];
        if (mode == 0) acc += a * a;
        else if (mode == 1) acc = fmax(acc, fabs(a));
        else if (mode == 2) acc += a;
        else acc += (a - mean) * (a - mean);
    }
    if (mode == 1) {
        __shared__ double sh[32];
        for (int o = 16; o > 0; o >>= 1) acc = fmax(acc, __shfl_down_sync(0xffffffffu, acc, o));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            acc = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) acc = fmax(acc, __shfl_down_sync(0xffffffffu, acc, o));
        }
    } else {
        acc = block_sum(acc);
    }
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
    if (arrive_last(counters + C_GEN)) {
        // fixed-order block-parallel combination of the block partials
        if (mode == 1) {
            double t = 0.0;
            for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) t = fmax(t, __ldcg(part + k));
            __shared__ double shm[32];
            for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
            if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = t;
            __syncthreads();
            if (threadIdx.x < 32) {
                t = threadIdx.x < (blockDim.x >> 5) ? shm[threadIdx.x] : 0.0;
                for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
            }
            if (threadIdx.x == 0) scal[slot] = t;
        } else {
            const double t = ordered_sum(part, gridDim.x);
            if (threadIdx.x == 0) scal[slot] = t;
        }
        if (threadIdx.x == 0) counters[C_GEN] = 0;
    }
}

// y (caller order) / nu -> internal order
template <typename T>
__global__ void k_gather_scale(const typename cplx_of<T>::type* __restrict__ y, const int* __restrict__ perm,
                               typename cplx_of<T>::type* __restrict__ out, int64_t M, T s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cscale(y[perm[i]], s);
}

template <typename T>
__global__ void k_scale_copy(const T* __restrict__ in, T* __restrict__ out, int64_t n, const double* scal, int slot) {
    const T s = (T)(1.0 / sqrt(scal[slot]));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] * s;
}

// SARA weights w = rho / (rho + |c|)
template <typename T>
__global__ void k_reweight(const T* __restrict__ c, T* __restrict__ w, int64_t D, T rho) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = rho / (rho + fabs(c[i]));
}

template <typename T>
__global__ void k_check_finite(const T* __restrict__ v, int64_t n, int* flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite((double)v[i])) flags[F_NAN] = 1;
}

// Circulant embedding of the point-spread function: psf is the complex
// [2ny][2nx] image A^H 1 (pixel (i, j) at lag d = (j - nx, i - ny)); the
// kernel on the [Ky][Kx] = [2ny][2nx] periodic grid holds psf(d) at d mod K.
template <typename T>
__global__ void k_circulant(const typename cplx_of<T>::type* __restrict__ psf, typename cplx_of<T>::type* __restrict__ c,
                            int nx, int ny) {
    const int Kx = 2 * nx, Ky = 2 * ny;
    const int64_t n = (int64_t)Kx * Ky;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(t / Kx), j = (int)(t % Kx);          // psf pixel
        int d1 = j - nx, d2 = i - ny;                       // lag
        int k1 = d1 & (Kx - 1), k2 = d2 & (Ky - 1);
        c[(size_t)k2 * Kx + k1] = psf[t];
    }
}

// multiplier = Re(c_hat) * s (the transform of a Hermitian kernel is real)
template <typename T>
__global__ void k_real_scale(const typename cplx_of<T>::type* __restrict__ c, T* __restrict__ m, int64_t n, double s) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        m[t] = (T)((double)c[t].x * s);
}

template <typename T>
__global__ void k_fill_one(typename cplx_of<T>::type* __restrict__ y, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        y[t] = cmake<typename cplx_of<T>::type>(T(1), T(0));
}

// Block-sharded CG: u = 2 r + u_sum (u_sum the sum over the shards of
// Re Phi_k^H Phi_k r / nu^2), per-block partials of r.r and r.u, and the
// step's scalars decided by the last block (cg_decide). Returns at once when
// the solve already stopped.
template <typename T>
__global__ void k_cg_combine(const T* __restrict__ u_sum, int64_t N, CgFold fold) {
    pdl_wait();
    if (block_flag(fold.flags + F_CGDONE)) return;
    const T* r = static_cast<const T*>(fold.r);
    T* u = static_cast<T*>(const_cast<void*>(fold.u));
    T g = 0, d = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const T rv = r[i];
        const T uv = T(2) * rv + u_sum[i];
        u[i] = uv;
        g += rv * rv;
        d += rv * uv;
    }
    const double b0 = block_sum_t(g);
    const double b1 = block_sum_t(d);
    if (threadIdx.x == 0) {
        fold.part[2 * blockIdx.x] = b0;
        fold.part[2 * blockIdx.x + 1] = b1;
    }
    if (arrive_last(fold.counter)) {
        cg_decide(fold, fold.step, gridDim.x);
        if (threadIdx.x == 0) *fold.counter = 0;
    }
    pdl_trigger();
}

// -------------------------------------------------------------- host side
static int ew_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

template <typename T> struct Solver {
    using C = typename cplx_of<T>::type;
    purify_plan* p;
    SdmmState& s;
    explicit Solver(purify_plan* plan) : p(plan), s(plan->sd) {}

    double* scal() { return s.scal.as<double>(); }
    double* part() { return s.part.as<double>(); }
    // the projection norms keep their partial sums apart from every other
    // reduction, so that they can run beside the wavelet branch
    static constexpr size_t kProjPart = 16384;
    static constexpr size_t kCgPart = 8192;   // [kCgPart, kProjPart): the CG partials
    double* proj_part() { return s.part.as<double>() + kProjPart; }
    // the CG partials (2 per inverse-row-pass block, at most 2 * 4096), apart
    // from the partials the relative-change kernel writes while it reads them
    double* cg_part() { return s.part.as<double>() + kCgPart; }
    unsigned* ctr() { return s.counters.as<unsigned>(); }
    int* flags() { return reinterpret_cast<int*>(s.counters.as<unsigned>() + 16); }

    void ensure() {
        if (s.ready) return;
        const size_t N = p->N, D = p->D, M = p->M;
        s.x.alloc(sizeof(T) * N);
        s.z1.alloc(sizeof(T) * D);
        s.z2.alloc(sizeof(C) * M);
        s.z3.alloc(sizeof(T) * N);
        s.ybar.alloc(sizeof(C) * M);
        s.w.alloc(sizeof(T) * D);
        s.eps.alloc(sizeof(double) * p->R);
        s.c1.alloc(sizeof(T) * D);
        s.v2.alloc(sizeof(C) * M);
        s.addend.alloc(sizeof(T) * N);
        s.r.alloc(sizeof(T) * N);
        s.p.alloc(sizeof(T) * N);
        s.Ap.alloc(sizeof(T) * N);
        s.u.alloc(sizeof(T) * N);
        s.xprev.alloc(sizeof(T) * N);
        s.scal.alloc(sizeof(double) * (S_BLOCKS + 2 * (size_t)p->R + 8));
        s.part.alloc(sizeof(double) * (kProjPart + std::max<size_t>(8192, 2 * (size_t)p->nchunks + 64)));
        s.counters.alloc(sizeof(unsigned) * 32);
        // chunk_first: first chunk index of each block (host computes from offsets)
        std::vector<int> cf(p->R + 1, 0);
        {
            const int64_t CH = 4096;
            int k = 0;
            for (int r = 0; r < p->R; ++r) {
                cf[r] = k;
                k += (int)((p->offsets[r + 1] - p->offsets[r] + CH - 1) / CH);
            }
            cf[p->R] = k;
        }
        s.chunk_first.alloc(sizeof(int) * cf.size());
        PURIFY_CUDA(cudaMemcpy(s.chunk_first.p, cf.data(), sizeof(int) * cf.size(), cudaMemcpyHostToDevice));
        PURIFY_CUDA(cudaMemset(s.scal.p, 0, s.scal.bytes));
        PURIFY_CUDA(cudaMemset(s.counters.p, 0, s.counters.bytes));
        s.ready = true;
    }

    void reduce(const T* v, int64_t n, int mode, int slot) {
        int nb = red_blocks(n);
        Launch L(p, "reduce");
        k_reduce<T><<<nb, RB, 0, p->stream>>>(v, n, mode, part(), ctr(), scal(), slot);
        L.done();
    }

    double read_scal(int slot) {
        double v;
        PURIFY_CUDA(cudaMemcpyAsync(&v, scal() + slot, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        PURIFY_CUDA(cudaStreamSynchronize(p->stream));
        return v;
    }

    // ||Phi||^2 by power iteration from a fixed pseudo-random start
    double op_norm_sq(int iters) {
        ensure();
        std::vector<T> x0(p->N);
        uint64_t st = 0x9E3779B97F4A7C15ull;
        for (int64_t i = 0; i < p->N; ++i) {
            st += 0x9E3779B97F4A7C15ull;
            uint64_t z = st;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            x0[i] = (T)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
        }
        T* xv = s.p.template as<T>();
        T* wv = s.Ap.template as<T>();
        PURIFY_CUDA(cudaMemcpyAsync(xv, x0.data(), sizeof(T) * p->N, cudaMemcpyHostToDevice, p->stream));
        reduce(xv, p->N, 0, S_NORM2);
        {
            Launch L(p, "scale_copy");
            k_scale_copy<T><<<ew_blocks(p->N), 256, 0, p->stream>>>(xv, xv, p->N, scal(), S_NORM2);
            L.done();
        }
        for (int it = 0; it < iters; ++it) {
            launch_phi(p, xv, s.v2.p, false, 1.0);
            launch_phi_adj(p, s.v2.p, wv, false, 1.0, 1, nullptr);
            reduce(wv, p->N, 0, S_NORM2);
            Launch L(p, "scale_copy");
            k_scale_copy<T><<<ew_blocks(p->N), 256, 0, p->stream>>>(wv, xv, p->N, scal(), S_NORM2);
            L.done();
        }
        return std::sqrt(read_scal(S_NORM2));
    }

    // Normal operator of the exact model by circulant embedding (Toeplitz):
    // A^H A x = psf * x with psf(d) = sum_m exp(i w_m . d) over lags |d| < n,
    // embedded in the plan's 2n x 2n grid; psf comes from the adjoint NUFFT of
    // a vector of ones on a 2n x 2n image. Multiplier = c_hat / (K^2 nu^2).
    void setup_toeplitz() {
        if (s.toep.p && s.toep_nu == s.nu) return;
        PURIFY_REQUIRE(p->Kx == 2 * p->nx && p->Ky == 2 * p->ny, "toeplitz needs oversample 2");
        purify_plan_desc d2 = p->desc;
        d2.nx = 2 * p->nx;
        d2.ny = 2 * p->ny;
        d2.M = p->M;
        d2.u = p->us.p;
        d2.v = p->vs.p;
        d2.R = 1;
        d2.block_offsets = nullptr;
        d2.levels = 1;
        d2.basis_mask = 1;
        d2.tile = p->work.tile;
        d2.stream = p->stream;
        purify_plan* q = create_plan(&d2);
        try {
            k_fill_one<T><<<ew_blocks(q->M), 256, 0, p->stream>>>(q->tmp_vis.template as<C>(), q->M);
            PURIFY_CUDA(cudaGetLastError());
            add_launches(1);
            launch_phi_adj(q, q->tmp_vis.p, q->tmp_img.p, false, 1.0, 0, nullptr);
            k_circulant<T><<<ew_blocks(4 * p->N), 256, 0, p->stream>>>(q->tmp_img.template as<C>(), p->grid.as<C>(),
                                                                       p->nx, p->ny);
            PURIFY_CUDA(cudaGetLastError());
            add_launches(1);
            PURIFY_CUDA(cudaStreamSynchronize(p->stream));
        } catch (...) {
            delete q;
            throw;
        }
        delete q;
        launch_fft2(p, p->grid.p, false);
        const int64_t nk = (int64_t)p->Kx * p->Ky;
        if (!s.toep.p) s.toep.alloc(sizeof(T) * nk);
        k_real_scale<T><<<ew_blocks(nk), 256, 0, p->stream>>>(p->grid.as<C>(), s.toep.template as<T>(), nk,
                                                             1.0 / ((double)nk * s.nu * s.nu));
        PURIFY_CUDA(cudaGetLastError());
        add_launches(1);
        s.toep_nu = s.nu;
    }

    // objective and per-block residual of x, written to scal
    void evaluate(const T* x) {
        launch_psi_adj(p, x, s.c1.p);
        {
            Launch L(p, "prox_l1");
            launch_dependent(k_prox_l1<T>, red_blocks(p->D), RB, 0, p->stream, s.c1.template as<T>(), nullptr,
                                                               s.have_w ? s.w.template as<T>() : nullptr, p->D,
                                                               s.gamma, part(), ctr(), scal(), 1);
            L.done();
        }
        launch_phi(p, x, s.v2.p, false, 1.0 / s.nu);
        proj_norms(false);
    }

    void proj_norms(bool with_z, const GroupChunks* gc = nullptr) {
        Launch L(p, "proj_norms");
        if (gc) {
            launch_dependent(k_proj_norms<T>, gc->n, RB, 0, p->stream, s.v2.template as<C>(),
                             with_z ? s.z2.template as<C>() : nullptr, s.ybar.template as<C>(), gc->cblk.as<int>(),
                             gc->cbeg.as<int>(), gc->cend.as<int>(), gc->n, p->R, gc->chunk_first.as<int>(),
                             proj_part(), ctr(), scal());
        } else {
            launch_dependent(k_proj_norms<T>, p->nchunks, RB, 0, p->stream,
                s.v2.template as<C>(), with_z ? s.z2.template as<C>() : nullptr, s.ybar.template as<C>(),
                p->chunk_blk.as<int>(), p->chunk_beg.as<int>(), p->chunk_end.as<int>(), p->nchunks, p->R,
                s.chunk_first.template as<int>(), proj_part(), ctr(), scal());
        }
        L.done();
    }

    void proj_apply(int out_mode, const GroupChunks* gc = nullptr) {
        Launch L(p, "proj_apply");
        launch_dependent(k_proj_apply<T>, gc ? gc->n : p->nchunks, RB, 0, p->stream, s.v2.template as<C>(),
                         s.z2.template as<C>(), s.ybar.template as<C>(),
                         gc ? gc->cblk.as<int>() : p->chunk_blk.as<int>(),
                         gc ? gc->cbeg.as<int>() : p->chunk_beg.as<int>(),
                         gc ? gc->cend.as<int>() : p->chunk_end.as<int>(), s.eps.template as<double>(), scal(), p->R,
                         out_mode);
        L.done();
    }

    // one SDMM iteration with exactly cg_iters CG steps (fewer only if the
    // stop test fires, in which case the remaining kernels return at once);
    // group >= 0: a block-subset iteration on that group of the s.groups
    // groups (see sdmm_iteration_groups of the reading: the group's
    // visibilities only, its data term scaled by the group count)
    void iteration(int cg_iters, int group = -1) {
        local_terms(group);
        cg_solve(cg_iters, group);
    }

    // The x-update's terms of one iteration: f1, f2 (all blocks, or the
    // group's) and f3 with their multiplier updates, leaving the adjoint term
    // Re Phi^H (s2 - z2 - Phi x / nu) / nu in r and the image-space terms
    // Psi (s1 - z1) + (s3 - z3) - 2 x in addend.
    void local_terms(int group) {
        T* x = s.x.template as<T>();
        const double inv_nu = 1.0 / s.nu;
        // The visibility branch (f2: Phi x, block projections, then the
        // adjoint part of the CG residual, Re Phi^H (s2 - z2 - Phi x / nu) /
        // nu, and for the circulant normal operator its correction) and the
        // wavelet branch (f1: Psi^dagger, prox, Psi; then f3) read only x and
        // their own state, so the visibility branch runs on a side stream,
        // joined before the CG start adds the image-space terms. Eager timing
        // runs keep one stream.
        const bool fork = !timing_enabled(p);
        cudaStream_t main_stream = p->stream;
        if (fork) {
            if (!s.side) {
                PURIFY_CUDA(cudaStreamCreateWithFlags(&s.side, cudaStreamNonBlocking));
                PURIFY_CUDA(cudaEventCreateWithFlags(&s.ev_fork, cudaEventDisableTiming));
                PURIFY_CUDA(cudaEventCreateWithFlags(&s.ev_join, cudaEventDisableTiming));
            }
            PURIFY_CUDA(cudaEventRecord(s.ev_fork, main_stream));
            PURIFY_CUDA(cudaStreamWaitEvent(s.side, s.ev_fork, 0));
            p->stream = s.side;
        }
        try {
            if (group >= 0) {
                // the group's blocks: Phi_g x / nu, their projections, and
                // r = G Re Phi_g^H v2 / nu
                const LaneWork& lw = p->group_lanes[group];
                const GroupChunks* gc = &p->group_chunks[group];
                launch_scale_pad_rows(p, x, inv_nu, nullptr, true, true);
                launch_cols_fwd(p, nullptr);
                launch_lanes_on(p, lw, 2, nullptr, s.v2.p, false, nullptr, true);
                proj_norms(true, gc);
                proj_apply(0, gc);
                launch_lanes_on(p, lw, 1, s.v2.p, nullptr, false, nullptr, true);
                launch_cols_inv(p, nullptr);
                launch_rows_inv_crop(p, s.r.p, inv_nu * s.groups, 1, nullptr, 1.0, nullptr);
            } else {
            // f2 (the forward row pass also clears the gridding accumulator
            // of the adjoint below)
            launch_phi(p, x, s.v2.p, false, inv_nu, true);
            proj_norms(true);
            proj_apply(s.toeplitz ? 1 : 0);
            // r = Re Phi^H v2 / nu (the image-space terms are added at the CG start)
            launch_phi_adj(p, s.v2.p, s.r.p, false, inv_nu, 1, nullptr, true);
            if (s.toeplitz) {
                // r -= (normal operator by circulant embedding) x
                launch_scale_pad_rows(p, x, 1.0, nullptr, false);
                launch_cols_fwd(p, nullptr);
                launch_cols_inv(p, nullptr, s.toep.p);
                launch_rows_inv_crop(p, s.r.p, -1.0, 1, s.r.p, 1.0, nullptr, nullptr, false);
            }
            }
            if (fork) PURIFY_CUDA(cudaEventRecord(s.ev_join, s.side));
        } catch (...) {
            p->stream = main_stream;
            throw;
        }
        p->stream = main_stream;
        // f1
        launch_psi_adj(p, x, s.c1.p);
        {
            Launch L(p, "prox_l1");
            launch_dependent(k_prox_l1<T>, red_blocks(p->D), RB, 0, p->stream, s.c1.template as<T>(), s.z1.template as<T>(),
                                                               s.have_w ? s.w.template as<T>() : nullptr, p->D,
                                                               s.gamma, part(), ctr(), scal(), 0);
            L.done();
        }
        launch_psi(p, s.c1.p, s.Ap.p);  // Psi(s1 - z1) into Ap (scratch)
        // f3 and the image-space terms of the residual
        {
            Launch L(p, "positivity");
            launch_dependent(k_positivity<T>, ew_blocks(p->N), 256, 0, p->stream, x, s.z3.template as<T>(), s.Ap.template as<T>(),
                                                                    s.addend.template as<T>(),
                                                                    s.xprev.template as<T>(), p->N);
            L.done();
        }
        if (fork) PURIFY_CUDA(cudaStreamWaitEvent(p->stream, s.ev_join, 0));
    }

    CgFold make_fold() {
        CgFold fold;
        fold.x = s.x.p;
        fold.r = s.r.p;
        fold.p = s.p.p;
        fold.s = s.Ap.p;
        fold.u = s.u.p;
        fold.add = s.addend.p;
        fold.part = cg_part();
        fold.counter = ctr() + C_CGI;
        fold.scal = scal();
        fold.flags = flags();
        return fold;
    }

    // The CG x-update from the terms local_terms left, then the relative change.
    void cg_solve(int cg_iters, int group) {
        T* x = s.x.template as<T>();
        const double inv_nu = 1.0 / s.nu;
        const int* skip = flags() + F_CGDONE;
        // CG (Chronopoulos-Gear arrangement, see CgFold): the forward row pass
        // of step 0 adds the image-space terms to r and starts the solve; step
        // k applies the operator to r; the update of step k is applied by the
        // forward row pass of step k + 1 or, after the last step, by the
        // relative-change kernel
        CgFold fold = make_fold();
        for (int k = 0; k < cg_iters; ++k) {
            fold.step = k;
            if (s.toeplitz) {
                // u = A r = 2 r + (embedded normal operator) r
                launch_scale_pad_rows(p, nullptr, 1.0, skip, false, false, &fold);
                launch_cols_fwd(p, skip);
                launch_cols_inv(p, skip, s.toep.p);
                launch_rows_inv_crop(p, s.u.p, 1.0, 1, s.r.p, 2.0, skip, &fold, false);
            } else {
                // the pending update and the transform of the new r fused into
                // the first FFT pass, then u = A r
                launch_scale_pad_rows(p, nullptr, inv_nu, skip, true, true, &fold);
                launch_cols_fwd(p, skip);
                if (group >= 0) launch_lanes_on(p, p->group_lanes[group], 0, nullptr, nullptr, false, skip, true);
                else launch_normal_gg(p, skip, true);
                launch_cols_inv(p, skip);
                // u = 2 r + Re Phi^H Phi r / nu^2 (G Re Phi_g^H Phi_g r / nu^2
                // for a group), with r.r, r.u and the CG scalars fused in
                launch_rows_inv_crop(p, s.u.p, group >= 0 ? inv_nu * s.groups : inv_nu, 1, s.r.p, 2.0, skip, &fold,
                                     true);
            }
        }
        // the last step's pending update is applied by the relative-change kernel
        finish(cg_iters);
    }

    // The last CG step's pending update and the relative change of x.
    void finish(int cg_iters) {
        CgFold fold = make_fold();
        fold.step = cg_iters - 1;
        if (cg_iters == 0) fold = CgFold();   // no CG step ran: nothing pending
        Launch L(p, "relchange");
        launch_dependent(k_relchange<T>, red_blocks(p->N), RB, 0, p->stream, s.x.template as<T>(),
                         s.xprev.template as<T>(), p->N, part(), ctr(), scal(), fold);
        L.done();
    }

    // Block-sharded CG step k (see purify_shard_cg_apply): the pending update
    // and the transform of the new r, then this shard's Re Phi^H Phi r / nu^2
    // alone into u_out (no 2 r, no dot products).
    void shard_cg_apply(int k, void* u_out) {
        const double inv_nu = 1.0 / s.nu;
        const int* skip = flags() + F_CGDONE;
        CgFold fold = make_fold();
        fold.step = k;
        launch_scale_pad_rows(p, nullptr, inv_nu, skip, true, true, &fold);
        launch_cols_fwd(p, skip);
        launch_normal_gg(p, skip, true);
        launch_cols_inv(p, skip);
        launch_rows_inv_crop(p, u_out, inv_nu, 1, nullptr, 0.0, skip, nullptr, true);
    }

    // Block-sharded CG step k, after the exchange: u = 2 r + u_sum, the dot
    // products r.r and r.u, and the step's scalars (cg_decide).
    void shard_cg_combine(int k, const void* u_sum) {
        CgFold fold = make_fold();
        fold.step = k;
        const int nb = red_blocks(p->N);
        Launch L(p, "cg_combine");
        launch_dependent(k_cg_combine<T>, nb, RB, 0, p->stream, (const T*)u_sum, p->N, fold);
        L.done();
    }
};

// One primal-dual iteration (see pd_solve): state x, xbar (in r), p1 (in
// z1), z = p2 / sigma (in z2). The ball branch (Phi xbar, the projections, the
// adjoint of the new p2 up to its inverse row pass) runs on the side stream
// beside the l1 branch (Psi^dagger xbar, the clip, Psi p1); the inverse row
// pass then forms g = Psi p1 + Re Phi^H p2 / nu and the primal step follows.
template <typename T> static void pd_iteration(Solver<T>& S, double tau, double sigma) {
    using C = typename cplx_of<T>::type;
    purify_plan* p = S.p;
    SdmmState& s = S.s;
    T* x = s.x.template as<T>();
    T* xbar = s.r.template as<T>();
    const double inv_nu = 1.0 / s.nu;
    const bool fork = !timing_enabled(p);
    cudaStream_t main_stream = p->stream;
    if (fork) {
        if (!s.side) {
            PURIFY_CUDA(cudaStreamCreateWithFlags(&s.side, cudaStreamNonBlocking));
            PURIFY_CUDA(cudaEventCreateWithFlags(&s.ev_fork, cudaEventDisableTiming));
            PURIFY_CUDA(cudaEventCreateWithFlags(&s.ev_join, cudaEventDisableTiming));
        }
        PURIFY_CUDA(cudaEventRecord(s.ev_fork, main_stream));
        PURIFY_CUDA(cudaStreamWaitEvent(s.side, s.ev_fork, 0));
        p->stream = s.side;
    }
    try {
        // q / sigma = z + Phi xbar / nu; z += Phi xbar / nu - proj(q / sigma)
        launch_phi(p, xbar, s.v2.p, false, inv_nu, true);
        S.proj_norms(true);
        {
            Launch L(p, "proj_apply");
            launch_dependent(k_proj_apply<T>, p->nchunks, RB, 0, p->stream, s.v2.template as<C>(),
                             s.z2.template as<C>(), s.ybar.template as<C>(), p->chunk_blk.as<int>(),
                             p->chunk_beg.as<int>(), p->chunk_end.as<int>(), s.eps.template as<double>(),
                             S.scal(), p->R, 2);
            L.done();
        }
        launch_grid(p, s.v2.p, false, nullptr, true);
        launch_cols_inv(p, nullptr);
        if (fork) PURIFY_CUDA(cudaEventRecord(s.ev_join, s.side));
    } catch (...) {
        p->stream = main_stream;
        throw;
    }
    p->stream = main_stream;
    launch_psi_adj(p, xbar, s.c1.p);
    {
        Launch L(p, "pd_dual_l1");
        launch_dependent(k_pd_dual_l1<T>, ew_blocks(p->D), 256, 0, p->stream, s.c1.template as<T>(),
                         s.z1.template as<T>(), s.have_w ? s.w.template as<T>() : nullptr, p->D, (T)sigma);
        L.done();
    }
    launch_psi(p, s.z1.p, s.p.p);
    if (fork) PURIFY_CUDA(cudaStreamWaitEvent(p->stream, s.ev_join, 0));
    // g = Psi p1 + Re Phi^H (sigma z) / nu
    launch_rows_inv_crop(p, s.u.p, sigma * inv_nu, 1, s.p.p, 1.0, nullptr);
    {
        Launch L(p, "pd_primal");
        launch_dependent(k_pd_primal<T>, ew_blocks(p->N), 256, 0, p->stream, x, s.u.template as<T>(), xbar,
                         (int64_t)p->N, (T)tau);
        L.done();
    }
}

// Run `n` primal-dual iterations as replays of a captured one-iteration graph
// (eager with kernel timing), ordered after and before the caller's stream.
template <typename T> static void run_pd_iterations(purify_plan* p, int n, double tau, double sigma) {
    SdmmState& s = p->sd;
    Solver<T> S(p);
    if (n <= 0) return;
    if (timing_enabled(p)) {
        for (int i = 0; i < n; ++i) pd_iteration<T>(S, tau, sigma);
        return;
    }
    if (!s.gstream) {
        PURIFY_CUDA(cudaStreamCreateWithFlags(&s.gstream, cudaStreamNonBlocking));
        PURIFY_CUDA(cudaEventCreateWithFlags(&s.ev_in, cudaEventDisableTiming));
        PURIFY_CUDA(cudaEventCreateWithFlags(&s.ev_out, cudaEventDisableTiming));
    }
    cudaStream_t user = p->stream;
    PURIFY_CUDA(cudaEventRecord(s.ev_in, user));
    PURIFY_CUDA(cudaStreamWaitEvent(s.gstream, s.ev_in, 0));
    int start = 0;
    const double key[4] = {tau, sigma, s.nu, s.have_w ? 1.0 : 0.0};
    if (!s.pd_gexec || !std::equal(key, key + 4, s.pd_key)) {
        if (s.pd_gexec) { cudaGraphExecDestroy(s.pd_gexec); s.pd_gexec = nullptr; }
        p->stream = s.gstream;
        try {
            // one eager iteration first (sets kernel attributes outside capture)
            pd_iteration<T>(S, tau, sigma);
            start = 1;
            cudaGraph_t g = nullptr;
            PURIFY_CUDA(cudaStreamBeginCapture(s.gstream, cudaStreamCaptureModeThreadLocal));
            try {
                pd_iteration<T>(S, tau, sigma);
            } catch (...) {
                cudaStreamEndCapture(s.gstream, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            PURIFY_CUDA(cudaStreamEndCapture(s.gstream, &g));
            size_t nn = 0;
            PURIFY_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
            std::vector<cudaGraphNode_t> nodes(nn);
            PURIFY_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
            int64_t kn = 0;
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                PURIFY_CUDA(cudaGraphNodeGetType(nd, &t));
                if (t == cudaGraphNodeTypeKernel) ++kn;
            }
            cudaError_t ie = cudaGraphInstantiate(&s.pd_gexec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) { s.pd_gexec = nullptr; PURIFY_CUDA(ie); }
            s.pd_kernels = kn;
            std::copy(key, key + 4, s.pd_key);
            add_launches(-kn);
        } catch (...) {
            p->stream = user;
            throw;
        }
        p->stream = user;
    }
    for (int i = start; i < n; ++i) {
        PURIFY_CUDA(cudaGraphLaunch(s.pd_gexec, s.gstream));
        add_launches(s.pd_kernels);
    }
    PURIFY_CUDA(cudaEventRecord(s.ev_out, s.gstream));
    PURIFY_CUDA(cudaStreamWaitEvent(user, s.ev_out, 0));
}

// Run `n` iterations: eager when kernel timing is on, otherwise as replays of
// a captured one-iteration graph on the plan's private stream, ordered after
// and before the caller's stream with events.
template <typename T> static void run_iterations(purify_plan* p, int n) {
    SdmmState& s = p->sd;
    Solver<T> S(p);
    if (n <= 0) return;
    if (timing_enabled(p)) {
        for (int i = 0; i < n; ++i) S.iteration(s.cg_iters);
        return;
    }
    if (!s.gstream) {
        PURIFY_CUDA(cudaStreamCreateWithFlags(&s.gstream, cudaStreamNonBlocking));
        PURIFY_CUDA(cudaEventCreateWithFlags(&s.ev_in, cudaEventDisableTiming));
        PURIFY_CUDA(cudaEventCreateWithFlags(&s.ev_out, cudaEventDisableTiming));
    }
    cudaStream_t user = p->stream;
    PURIFY_CUDA(cudaEventRecord(s.ev_in, user));
    PURIFY_CUDA(cudaStreamWaitEvent(s.gstream, s.ev_in, 0));
    int start = 0;
    if (!s.gexec || s.g_cg != s.cg_iters || s.g_gamma != s.gamma || s.g_nu != s.nu || s.g_have_w != s.have_w ||
        s.g_toep != s.toeplitz) {
        if (s.gexec) { cudaGraphExecDestroy(s.gexec); s.gexec = nullptr; }
        p->stream = s.gstream;
        try {
            // one eager iteration first (sets kernel attributes outside capture)
            S.iteration(s.cg_iters);
            start = 1;
            cudaGraph_t g = nullptr;
            PURIFY_CUDA(cudaStreamBeginCapture(s.gstream, cudaStreamCaptureModeThreadLocal));
            try {
                S.iteration(s.cg_iters);
            } catch (...) {
                cudaStreamEndCapture(s.gstream, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            PURIFY_CUDA(cudaStreamEndCapture(s.gstream, &g));
            size_t nn = 0;
            PURIFY_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
            std::vector<cudaGraphNode_t> nodes(nn);
            PURIFY_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
            int64_t kn = 0;
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                PURIFY_CUDA(cudaGraphNodeGetType(nd, &t));
                if (t == cudaGraphNodeTypeKernel) ++kn;
            }
            cudaError_t ie = cudaGraphInstantiate(&s.gexec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) { s.gexec = nullptr; PURIFY_CUDA(ie); }
            s.g_kernels = kn;
            s.g_cg = s.cg_iters;
            s.g_gamma = s.gamma;
            s.g_nu = s.nu;
            s.g_have_w = s.have_w;
            s.g_toep = s.toeplitz;
            // the captured launches were counted once while capturing
            add_launches(-kn);
        } catch (...) {
            p->stream = user;
            throw;
        }
        p->stream = user;
    }
    for (int i = start; i < n; ++i) {
        PURIFY_CUDA(cudaGraphLaunch(s.gexec, s.gstream));
        add_launches(s.g_kernels);
    }
    PURIFY_CUDA(cudaEventRecord(s.ev_out, s.gstream));
    PURIFY_CUDA(cudaStreamWaitEvent(user, s.ev_out, 0));
}

// Block-subset iterations: iteration i runs group groups[i] (round-robin
// from the iteration count when groups is null), each group's iteration a
// replay of its own captured graph (captured on first use and whenever
// gamma, nu, the weights, the CG count or the group count change); eager
// when kernel timing is on.
template <typename T> static void run_group_iterations(purify_plan* p, int n, const int32_t* groups) {
    SdmmState& s = p->sd;
    Solver<T> S(p);
    if (n <= 0) return;
    const int G = s.groups;
    auto group_of = [&](int i) {
        const int g = groups ? groups[i] : (int)((s.iters_done + i) % G);
        if (g < 0 || g >= G) throw Error{PURIFY_EINVAL, "group index out of range"};
        return g;
    };
    for (int i = 0; i < n; ++i) group_of(i);   // validate before any launch
    if (timing_enabled(p)) {
        for (int i = 0; i < n; ++i) S.iteration(s.cg_iters, group_of(i));
        return;
    }
    if (!s.gstream) {
        PURIFY_CUDA(cudaStreamCreateWithFlags(&s.gstream, cudaStreamNonBlocking));
        PURIFY_CUDA(cudaEventCreateWithFlags(&s.ev_in, cudaEventDisableTiming));
        PURIFY_CUDA(cudaEventCreateWithFlags(&s.ev_out, cudaEventDisableTiming));
    }
    if (s.gg_cg != s.cg_iters || s.gg_gamma != s.gamma || s.gg_nu != s.nu || s.gg_have_w != s.have_w ||
        s.gg_groups != G || (int)s.gexec_group.size() != G) {
        s.drop_group_graphs();
        s.gexec_group.assign(G, nullptr);
        s.kernels_group.assign(G, 0);
        s.gg_cg = s.cg_iters;
        s.gg_gamma = s.gamma;
        s.gg_nu = s.nu;
        s.gg_have_w = s.have_w;
        s.gg_groups = G;
    }
    cudaStream_t user = p->stream;
    PURIFY_CUDA(cudaEventRecord(s.ev_in, user));
    PURIFY_CUDA(cudaStreamWaitEvent(s.gstream, s.ev_in, 0));
    for (int i = 0; i < n; ++i) {
        const int g = group_of(i);
        if (!s.gexec_group[g]) {
            p->stream = s.gstream;
            try {
                // this iteration eagerly (sets kernel attributes outside capture), then capture
                S.iteration(s.cg_iters, g);
                cudaGraph_t gr = nullptr;
                PURIFY_CUDA(cudaStreamBeginCapture(s.gstream, cudaStreamCaptureModeThreadLocal));
                try {
                    S.iteration(s.cg_iters, g);
                } catch (...) {
                    cudaStreamEndCapture(s.gstream, &gr);
                    if (gr) cudaGraphDestroy(gr);
                    throw;
                }
                PURIFY_CUDA(cudaStreamEndCapture(s.gstream, &gr));
                size_t nn = 0;
                PURIFY_CUDA(cudaGraphGetNodes(gr, nullptr, &nn));
                std::vector<cudaGraphNode_t> nodes(nn);
                PURIFY_CUDA(cudaGraphGetNodes(gr, nodes.data(), &nn));
                int64_t kn = 0;
                for (auto nd : nodes) {
                    cudaGraphNodeType t;
                    PURIFY_CUDA(cudaGraphNodeGetType(nd, &t));
                    if (t == cudaGraphNodeTypeKernel) ++kn;
                }
                cudaError_t ie = cudaGraphInstantiate(&s.gexec_group[g], gr, 0);
                cudaGraphDestroy(gr);
                if (ie != cudaSuccess) { s.gexec_group[g] = nullptr; PURIFY_CUDA(ie); }
                s.kernels_group[g] = kn;
                add_launches(-kn);
            } catch (...) {
                p->stream = user;
                throw;
            }
            p->stream = user;
            continue;   // this iteration ran eagerly
        }
        PURIFY_CUDA(cudaGraphLaunch(s.gexec_group[g], s.gstream));
        add_launches(s.kernels_group[g]);
    }
    PURIFY_CUDA(cudaEventRecord(s.ev_out, s.gstream));
    PURIFY_CUDA(cudaStreamWaitEvent(user, s.ev_out, 0));
}

// ------------------------------------------------- block-sharded steps
template <typename T> static void shard_step_t(purify_plan* p, int op, int step, void* ptr) {
    Solver<T> S(p);
    SdmmState& s = p->sd;
    const size_t bytes = sizeof(T) * (size_t)p->N;
    switch (op) {
        case 0:   // this shard's x-update terms; its adjoint term out
            S.local_terms(-1);
            PURIFY_CUDA(cudaMemcpyAsync(ptr, s.r.p, bytes, cudaMemcpyDeviceToDevice, p->stream));
            break;
        case 1:   // the summed adjoint term in
            PURIFY_CUDA(cudaMemcpyAsync(s.r.p, ptr, bytes, cudaMemcpyDeviceToDevice, p->stream));
            break;
        case 2: S.shard_cg_apply(step, ptr); break;
        case 3: S.shard_cg_combine(step, ptr); break;
        default:  // 4: the last pending update and the relative change
            S.finish(step);
            s.iters_done += 1;
            break;
    }
}

void shard_step(purify_plan* p, int op, int step, void* ptr) {
    SdmmState& s = p->sd;
    if (!s.started) throw Error{PURIFY_EINVAL, "no SDMM solve started on this plan"};
    if (s.groups > 0 || s.toeplitz)
        throw Error{PURIFY_EINVAL, "block-sharded steps need a solve without block groups or toeplitz"};
    if (op != 4 && (ptr == nullptr || is_host_pointer(ptr))) throw Error{PURIFY_EINVAL, "a device image is required"};
    if ((op == 2 || op == 3) && step < 0) throw Error{PURIFY_EINVAL, "negative CG step"};
    if (op == 4 && step < 0) throw Error{PURIFY_EINVAL, "negative CG step count"};
    if (p->dtype == PURIFY_F32) shard_step_t<float>(p, op, step, ptr); else shard_step_t<double>(p, op, step, ptr);
}

// --------------------------------------------------------- batched plans
void batch_destroy(BatchState* b) {
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (auto& st : b->streams) cudaStreamDestroy(st);
    for (auto& e : b->events) cudaEventDestroy(e);
    delete b;
}

static void iteration_on(purify_plan* p) {
    if (p->dtype == PURIFY_F32) Solver<float>(p).iteration(p->sd.cg_iters);
    else Solver<double>(p).iteration(p->sd.cg_iters);
}

void batch_iterate(BatchState* b, int iters) {
    const size_t n = b->plans.size();
    if (iters <= 0 || n == 0) return;
    for (auto* p : b->plans)
        if (!p->sd.started) throw Error{PURIFY_EINVAL, "every plan of a batch needs a started solve"};
    if (b->streams.empty()) {
        b->streams.resize(n);
        b->events.resize(n + 1);
        for (size_t i = 0; i < n; ++i) PURIFY_CUDA(cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking));
        for (auto& e : b->events) PURIFY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // the captured graph depends on each plan's constants
    std::vector<double> key;
    for (auto* p : b->plans) {
        key.push_back(p->sd.gamma);
        key.push_back(p->sd.nu);
        key.push_back(p->sd.have_w ? 1.0 : 0.0);
        key.push_back((double)p->sd.cg_iters);
        key.push_back(p->sd.toeplitz ? 1.0 : 0.0);
    }
    bool timed = false;
    for (auto* p : b->plans) timed = timed || timing_enabled(p);
    if (timed) {
        // kernel timing records events around every launch: run eagerly
        std::vector<cudaStream_t> saved(n);
        for (size_t i = 0; i < n; ++i) saved[i] = b->plans[i]->stream;
        try {
            for (int it = 0; it < iters; ++it) {
                PURIFY_CUDA(cudaEventRecord(b->events[n], b->stream));
                for (size_t i = 0; i < n; ++i) {
                    PURIFY_CUDA(cudaStreamWaitEvent(b->streams[i], b->events[n], 0));
                    b->plans[i]->stream = b->streams[i];
                    iteration_on(b->plans[i]);
                    PURIFY_CUDA(cudaEventRecord(b->events[i], b->streams[i]));
                    PURIFY_CUDA(cudaStreamWaitEvent(b->stream, b->events[i], 0));
                }
            }
        } catch (...) {
            for (size_t i = 0; i < n; ++i) b->plans[i]->stream = saved[i];
            throw;
        }
        for (size_t i = 0; i < n; ++i) b->plans[i]->stream = saved[i];
        for (auto* p : b->plans) p->sd.iters_done += iters;
        return;
    }
    int start = 0;
    if (!b->gexec || key != b->key) {
        if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
        std::vector<cudaStream_t> saved(n);
        for (size_t i = 0; i < n; ++i) saved[i] = b->plans[i]->stream;
        auto fork_join = [&](bool capture) {
            PURIFY_CUDA(cudaEventRecord(b->events[n], b->stream));
            for (size_t i = 0; i < n; ++i) {
                PURIFY_CUDA(cudaStreamWaitEvent(b->streams[i], b->events[n], 0));
                b->plans[i]->stream = b->streams[i];
                iteration_on(b->plans[i]);
                PURIFY_CUDA(cudaEventRecord(b->events[i], b->streams[i]));
                PURIFY_CUDA(cudaStreamWaitEvent(b->stream, b->events[i], 0));
            }
            (void)capture;
        };
        try {
            fork_join(false);  // one eager iteration (sets kernel attributes outside capture)
            start = 1;
            cudaGraph_t g = nullptr;
            PURIFY_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            try {
                fork_join(true);
            } catch (...) {
                cudaStreamEndCapture(b->stream, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            PURIFY_CUDA(cudaStreamEndCapture(b->stream, &g));
            size_t nn = 0;
            PURIFY_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
            std::vector<cudaGraphNode_t> nodes(nn);
            PURIFY_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
            int64_t kn = 0;
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                PURIFY_CUDA(cudaGraphNodeGetType(nd, &t));
                if (t == cudaGraphNodeTypeKernel) ++kn;
            }
            cudaError_t ie = cudaGraphInstantiate(&b->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) { b->gexec = nullptr; PURIFY_CUDA(ie); }
            b->kernels = kn;
            b->key = key;
            add_launches(-kn);
        } catch (...) {
            for (size_t i = 0; i < n; ++i) b->plans[i]->stream = saved[i];
            throw;
        }
        for (size_t i = 0; i < n; ++i) b->plans[i]->stream = saved[i];
    }
    for (int i = start; i < iters; ++i) {
        PURIFY_CUDA(cudaGraphLaunch(b->gexec, b->stream));
        add_launches(b->kernels);
    }
    for (auto* p : b->plans) p->sd.iters_done += iters;
}

void sdmm_iterate(purify_plan* p, int iters, const int32_t* groups) {
    if (p->sd.groups > 0) {
        if (p->dtype == PURIFY_F32) run_group_iterations<float>(p, iters, groups);
        else run_group_iterations<double>(p, iters, groups);
    } else {
        if (p->dtype == PURIFY_F32) run_iterations<float>(p, iters); else run_iterations<double>(p, iters);
    }
    p->sd.iters_done += iters;
}

// ------------------------------------------------------------ entry points
template <typename T>
static void sdmm_solve_t(purify_plan* p, const void* y, const double* eps, const void* w, void* x_io,
                         const purify_sdmm_params& prm, purify_sdmm_stats* st) {
    using C = typename cplx_of<T>::type;
    Solver<T> S(p);
    S.ensure();
    SdmmState& s = p->sd;
    if (!prm.resume || s.iters_done < 0 || !s.started) {
        PURIFY_REQUIRE(y != nullptr && eps != nullptr && x_io != nullptr, "null y, eps or x");
        for (int r = 0; r < p->R; ++r)
            PURIFY_REQUIRE(std::isfinite(eps[r]) && eps[r] > 0.0, "eps must be positive and finite");
        // nu and gamma
        s.nu = prm.nu > 0 ? prm.nu : std::sqrt(S.op_norm_sq(100));
        if (is_host_pointer(y)) {
            PURIFY_CUDA(cudaMemcpyAsync(p->tmp_vis.p, y, sizeof(C) * p->M, cudaMemcpyDefault, p->stream));
            y = p->tmp_vis.p;
        }
        // data in internal order, scaled by 1/nu
        PURIFY_CUDA(cudaMemsetAsync(S.flags(), 0, sizeof(int) * F_COUNT, p->stream));
        {
            Launch L(p, "check_finite");
            k_check_finite<T><<<ew_blocks(2 * p->M), 256, 0, p->stream>>>((const T*)y, 2 * p->M, S.flags());
            L.done();
        }
        {
            Launch L(p, "gather_scale");
            k_gather_scale<T><<<ew_blocks(p->M), 256, 0, p->stream>>>((const C*)y, p->perm.as<int>(),
                                                                      s.ybar.template as<C>(), p->M, (T)(1.0 / s.nu));
            L.done();
        }
        std::vector<double> en(p->R);
        for (int r = 0; r < p->R; ++r) en[r] = eps[r] / s.nu;
        PURIFY_CUDA(cudaMemcpyAsync(s.eps.p, en.data(), sizeof(double) * p->R, cudaMemcpyHostToDevice, p->stream));
        s.eps_host.assign(eps, eps + p->R);
        s.have_w = w != nullptr;
        if (w) PURIFY_CUDA(cudaMemcpyAsync(s.w.p, w, sizeof(T) * p->D, cudaMemcpyDefault, p->stream));
        if (prm.gamma > 0) {
            s.gamma = prm.gamma;
        } else {
            // gamma = 1e-3 max |Psi^dagger Re Phi^H ybar| / nu  (= max|Psi^dagger Re Phi^H y| / nu^2)
            launch_phi_adj(p, s.ybar.p, s.r.p, false, 1.0 / s.nu, 1, nullptr);
            launch_psi_adj(p, s.r.p, s.c1.p);
            S.reduce(s.c1.template as<T>(), p->D, 1, S_GMAX);
            s.gamma = 1e-3 * S.read_scal(S_GMAX);
        }
        s.toeplitz = prm.toeplitz != 0;
        if (s.toeplitz) S.setup_toeplitz();
        s.groups = prm.block_groups > 0 ? prm.block_groups : 0;
        if (s.groups > 0) {
            PURIFY_REQUIRE(!s.toeplitz, "block groups and the circulant normal operator cannot be combined");
            build_group_lanes(p, s.groups);
        }
        PURIFY_CUDA(cudaMemcpyAsync(s.x.p, x_io, sizeof(T) * p->N, cudaMemcpyDefault, p->stream));
        PURIFY_CUDA(cudaMemsetAsync(s.z1.p, 0, s.z1.bytes, p->stream));
        PURIFY_CUDA(cudaMemsetAsync(s.z2.p, 0, s.z2.bytes, p->stream));
        PURIFY_CUDA(cudaMemsetAsync(s.z3.p, 0, s.z3.bytes, p->stream));
        double tol2 = prm.cg_tol > 0 ? prm.cg_tol * prm.cg_tol : 0.0;
        PURIFY_CUDA(cudaMemcpyAsync(S.scal() + S_TOL2, &tol2, sizeof(double), cudaMemcpyHostToDevice, p->stream));
        double zero = 0.0;
        PURIFY_CUDA(cudaMemcpyAsync(S.scal() + S_CGCOUNT, &zero, sizeof(double), cudaMemcpyHostToDevice, p->stream));
        PURIFY_CUDA(cudaStreamSynchronize(p->stream));
        int fl[F_COUNT];
        PURIFY_CUDA(cudaMemcpy(fl, S.flags(), sizeof(fl), cudaMemcpyDeviceToHost));
        if (fl[F_NAN]) throw Error{PURIFY_ENAN, "non-finite visibility"};
        s.iters_done = 0;
        s.started = true;
    } else {
        double tol2 = prm.cg_tol > 0 ? prm.cg_tol * prm.cg_tol : 0.0;
        PURIFY_CUDA(cudaMemcpyAsync(S.scal() + S_TOL2, &tol2, sizeof(double), cudaMemcpyHostToDevice, p->stream));
    }
    s.cg_iters = prm.cg_iters > 0 ? prm.cg_iters : 10;
    if (prm.resume && prm.block_groups != (s.groups > 0 ? s.groups : 0))
        throw Error{PURIFY_EINVAL, "a resumed solve keeps the block groups of its start"};
    const int check = prm.check_every > 0 ? prm.check_every : 10;
    const bool tol_mode = prm.rel_obj_tol > 0;
    int done = 0;
    purify_status status = PURIFY_OK;
    bool converged = false;
    // n iterations from iteration `at` of this call (block groups from the
    // caller's sequence)
    auto run = [&](int n, int at) {
        if (s.groups > 0) {
            run_group_iterations<T>(p, n, prm.group_seq ? prm.group_seq + at : nullptr);
            s.iters_done += n;
        } else {
            run_iterations<T>(p, n);
            s.iters_done += n;
        }
    };
    const int64_t iters0 = s.iters_done;
    double prev_check_obj = -1.0;
    if (!tol_mode) {
        run(prm.max_iter, 0);
        done = prm.max_iter;
    }
    for (int it = 0; tol_mode && it < prm.max_iter; it += check) {
        const int n = std::min(check, prm.max_iter - it);
        run(n, it);
        done += n;
        {
            // block groups: objective and residuals of every block at x, the
            // change measured against the previous check
            if (s.groups > 0) S.evaluate(s.x.template as<T>());
            std::vector<double> sc(S_BLOCKS + 2 * p->R);
            PURIFY_CUDA(cudaMemcpyAsync(sc.data(), S.scal(), sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, p->stream));
            PURIFY_CUDA(cudaStreamSynchronize(p->stream));
            double obj = sc[S_OBJ], prev = sc[S_OBJ_PREV];
            if (s.groups > 0) {
                prev = prev_check_obj;
                prev_check_obj = obj;
            }
            double rel = (obj > 0 && prev >= 0) ? std::fabs(obj - prev) / obj : (prev < 0 ? 1.0 : 0.0);
            double worst = 0.0;
            for (int r = 0; r < p->R; ++r) worst = std::max(worst, std::sqrt(sc[S_BLOCKS + p->R + r]) * s.nu / s.eps_host[r]);
            if (rel < prm.rel_obj_tol && worst <= 1.0 + prm.eps_tol) { converged = true; break; }
        }
    }
    (void)iters0;
    // statistics at the returned x
    int fl[F_COUNT];
    PURIFY_CUDA(cudaMemcpyAsync(fl, S.flags(), sizeof(fl), cudaMemcpyDeviceToHost, p->stream));
    double rel_num[2];
    PURIFY_CUDA(cudaMemcpyAsync(rel_num, S.scal() + S_XN2, sizeof(rel_num), cudaMemcpyDeviceToHost, p->stream));
    double cgc = 0.0;
    PURIFY_CUDA(cudaMemcpyAsync(&cgc, S.scal() + S_CGCOUNT, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    S.evaluate(s.x.template as<T>());
    std::vector<double> sc(S_BLOCKS + 2 * p->R);
    PURIFY_CUDA(cudaMemcpyAsync(sc.data(), S.scal(), sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, p->stream));
    PURIFY_CUDA(cudaMemcpyAsync(x_io, s.x.p, sizeof(T) * p->N, cudaMemcpyDefault, p->stream));
    PURIFY_CUDA(cudaStreamSynchronize(p->stream));
    if (fl[F_NAN]) status = PURIFY_ENAN;
    else if (tol_mode && !converged) status = PURIFY_ENOTCONV;
    if (st) {
        st->iters = (int32_t)s.iters_done;
        st->cg_iters_total = (int32_t)cgc;
        st->objective = sc[S_OBJ];
        double worst = 0.0;
        for (int r = 0; r < p->R; ++r) worst = std::max(worst, std::sqrt(sc[S_BLOCKS + p->R + r]) * s.nu / s.eps_host[r]);
        st->max_resid_over_eps = worst;
        st->rel_change = rel_num[0] > 0 ? std::sqrt(rel_num[1] / rel_num[0]) : 0.0;
        st->gamma = s.gamma;
        st->nu = s.nu;
        st->status = status;
    }
    if (status == PURIFY_ENAN) throw Error{PURIFY_ENAN, "non-finite value in the SDMM iterates"};
    if (status == PURIFY_ENOTCONV) throw Error{PURIFY_ENOTCONV, "tolerance not reached within max_iter"};
}

void sdmm_solve(purify_plan* p, const void* y, const double* eps, const void* w, void* x,
                const purify_sdmm_params& prm, purify_sdmm_stats* st) {
    if (p->dtype == PURIFY_F32) sdmm_solve_t<float>(p, y, eps, w, x, prm, st);
    else sdmm_solve_t<double>(p, y, eps, w, x, prm, st);
}

template <typename T>
static void pd_solve_t(purify_plan* p, const void* y, const double* eps, const void* w, void* x_io,
                       const purify_pd_params& prm, purify_sdmm_stats* st) {
    using C = typename cplx_of<T>::type;
    Solver<T> S(p);
    S.ensure();
    SdmmState& s = p->sd;
    for (int r = 0; r < p->R; ++r)
        PURIFY_REQUIRE(std::isfinite(eps[r]) && eps[r] > 0.0, "eps must be positive and finite");
    const double tau = prm.tau > 0 ? prm.tau : 0.05, sigma = prm.sigma > 0 ? prm.sigma : 9.8;
    s.started = false;   // the SDMM state is overwritten
    s.nu = prm.nu > 0 ? prm.nu : std::sqrt(S.op_norm_sq(100));
    if (is_host_pointer(y)) {
        PURIFY_CUDA(cudaMemcpyAsync(p->tmp_vis.p, y, sizeof(C) * p->M, cudaMemcpyDefault, p->stream));
        y = p->tmp_vis.p;
    }
    PURIFY_CUDA(cudaMemsetAsync(S.flags(), 0, sizeof(int) * F_COUNT, p->stream));
    {
        Launch L(p, "check_finite");
        k_check_finite<T><<<ew_blocks(2 * p->M), 256, 0, p->stream>>>((const T*)y, 2 * p->M, S.flags());
        L.done();
    }
    {
        Launch L(p, "gather_scale");
        k_gather_scale<T><<<ew_blocks(p->M), 256, 0, p->stream>>>((const C*)y, p->perm.as<int>(),
                                                                  s.ybar.template as<C>(), p->M, (T)(1.0 / s.nu));
        L.done();
    }
    std::vector<double> en(p->R);
    for (int r = 0; r < p->R; ++r) en[r] = eps[r] / s.nu;
    PURIFY_CUDA(cudaMemcpyAsync(s.eps.p, en.data(), sizeof(double) * p->R, cudaMemcpyHostToDevice, p->stream));
    s.eps_host.assign(eps, eps + p->R);
    s.have_w = w != nullptr;
    if (w) PURIFY_CUDA(cudaMemcpyAsync(s.w.p, w, sizeof(T) * p->D, cudaMemcpyDefault, p->stream));
    PURIFY_CUDA(cudaMemcpyAsync(s.x.p, x_io, sizeof(T) * p->N, cudaMemcpyDefault, p->stream));
    PURIFY_CUDA(cudaMemcpyAsync(s.r.p, s.x.p, sizeof(T) * p->N, cudaMemcpyDeviceToDevice, p->stream));   // xbar = x
    PURIFY_CUDA(cudaMemsetAsync(s.z1.p, 0, s.z1.bytes, p->stream));   // p1 = 0
    PURIFY_CUDA(cudaMemsetAsync(s.z2.p, 0, s.z2.bytes, p->stream));   // p2 = 0
    PURIFY_CUDA(cudaStreamSynchronize(p->stream));
    int fl[F_COUNT];
    PURIFY_CUDA(cudaMemcpy(fl, S.flags(), sizeof(fl), cudaMemcpyDeviceToHost));
    if (fl[F_NAN]) throw Error{PURIFY_ENAN, "non-finite visibility"};
    run_pd_iterations<T>(p, prm.iters, tau, sigma);
    // statistics at the returned x
    S.evaluate(s.x.template as<T>());
    std::vector<double> sc(S_BLOCKS + 2 * p->R);
    PURIFY_CUDA(cudaMemcpyAsync(sc.data(), S.scal(), sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, p->stream));
    PURIFY_CUDA(cudaMemcpyAsync(x_io, s.x.p, sizeof(T) * p->N, cudaMemcpyDefault, p->stream));
    PURIFY_CUDA(cudaStreamSynchronize(p->stream));
    if (st) {
        st->iters = prm.iters;
        st->objective = sc[S_OBJ];
        double worst = 0.0;
        for (int r = 0; r < p->R; ++r) worst = std::max(worst, std::sqrt(sc[S_BLOCKS + p->R + r]) * s.nu / s.eps_host[r]);
        st->max_resid_over_eps = worst;
        st->nu = s.nu;
        st->status = PURIFY_OK;
    }
}

void pd_solve(purify_plan* p, const void* y, const double* eps, const void* w, void* x,
              const purify_pd_params& prm, purify_sdmm_stats* st) {
    if (p->dtype == PURIFY_F32) pd_solve_t<float>(p, y, eps, w, x, prm, st);
    else pd_solve_t<double>(p, y, eps, w, x, prm, st);
}

double op_norm_sq(purify_plan* p, int iters) {
    double nrm = p->dtype == PURIFY_F32 ? Solver<float>(p).op_norm_sq(iters) : Solver<double>(p).op_norm_sq(iters);
    return nrm;
}

template <typename T> static void reweight_t(purify_plan* p, const void* x, double rho, void* w) {
    launch_psi_adj(p, x, w);
    Launch L(p, "reweight");
    k_reweight<T><<<ew_blocks(p->D), 256, 0, p->stream>>>((const T*)w, (T*)w, p->D, (T)rho);
    L.done();
}

void reweight(purify_plan* p, const void* x, double rho, void* w) {
    if (p->dtype == PURIFY_F32) reweight_t<float>(p, x, rho, w); else reweight_t<double>(p, x, rho, w);
}

template <typename T> static double coef_std_t(purify_plan* p, const void* x) {
    Solver<T> S(p);
    S.ensure();
    T* c = p->sd.c1.template as<T>();
    launch_psi_adj(p, x, c);
    S.reduce(c, p->D, 2, S_SUM);
    S.reduce(c, p->D, 3, S_NORM2);
    return std::sqrt(S.read_scal(S_NORM2) / (double)p->D);
}

double coef_std(purify_plan* p, const void* x) {
    return p->dtype == PURIFY_F32 ? coef_std_t<float>(p, x) : coef_std_t<double>(p, x);
}

}  // namespace purify
