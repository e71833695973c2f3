// Measurement operator Phi = G F Z S and its adjoint S Z^T F^H G^H.
//
// The paper (Sec. 1) writes the measurement equation as y = Phi x + n and
// leaves the discretisation open; the plan realises Phi with Kaiser-Bessel
// gridding on a K = alpha n oversampled grid:
//   rows_fwd  : S, Z and the row pass of F over the ny image rows only (the
//               other K - ny grid rows are zero and never stored);
//   cols_fwd  : column pass of F, treating the missing rows as zeros;
//   degrid    : G, J x J separable Kaiser-Bessel interpolation per visibility;
//   grid      : G^H, per-tile shared-memory accumulation of the footprints;
//   cols_inv  : column pass of F^H producing only the ny rows kept by Z^T;
//   rows_inv  : row pass of F^H fused with Z^T (crop) and S.
// FFTs are radix-4 Stockham passes (one radix-2 pass first for odd log2 K)
// in shared memory on several rows or columns per thread block.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "launch.h"
#include "reduce.cuh"

namespace purify {

// --------------------------------------------------------------- FFT core
// `nb` independent length-n FFTs held in shared memory; element k of FFT f
// lives at f*fs + k*ks. Returns the buffer holding the result.
template <typename C, bool INV>
__device__ C* fft_smem(C* src, C* dst, int n, int logn, int nb, int fs, int ks, const C* __restrict__ tw) {
    const int tid = threadIdx.x, T = blockDim.x;
    int Ns = 1;
    if (logn & 1) {
        const int half = n >> 1;
        for (int t = tid; t < nb * half; t += T) {
            int f = t % nb, j = t / nb;
            C v0 = src[f * fs + j * ks];
            C v1 = src[f * fs + (j + half) * ks];
            dst[f * fs + (2 * j) * ks] = cadd(v0, v1);
            dst[f * fs + (2 * j + 1) * ks] = csub(v0, v1);
        }
        __syncthreads();
        C* s = src; src = dst; dst = s;
        Ns = 2;
    }
    const int quarter = n >> 2;
    while (Ns < n) {
        const int tstride = n / (4 * Ns);
        for (int t = tid; t < nb * quarter; t += T) {
            int f = t % nb, j = t / nb;
            int k = j & (Ns - 1);
            C v0 = src[f * fs + j * ks];
            C v1 = src[f * fs + (j + quarter) * ks];
            C v2 = src[f * fs + (j + 2 * quarter) * ks];
            C v3 = src[f * fs + (j + 3 * quarter) * ks];
            if (Ns > 1) {
                C w1 = tw[k * tstride], w2 = tw[2 * k * tstride], w3 = tw[3 * k * tstride];
                if (INV) { v1 = cmulconj(v1, w1); v2 = cmulconj(v2, w2); v3 = cmulconj(v3, w3); }
                else { v1 = cmul(v1, w1); v2 = cmul(v2, w2); v3 = cmul(v3, w3); }
            }
            C a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = csub(v1, v3);
            // -i * a3 for the forward transform, +i * a3 for the inverse
            C ia3 = INV ? cmake<C>(-a3.y, a3.x) : cmake<C>(a3.y, -a3.x);
            int o = (j - k) * 4 + k;
            dst[f * fs + o * ks] = cadd(a0, a2);
            dst[f * fs + (o + Ns) * ks] = cadd(a1, ia3);
            dst[f * fs + (o + 2 * Ns) * ks] = csub(a0, a2);
            dst[f * fs + (o + 3 * Ns) * ks] = csub(a1, ia3);
        }
        __syncthreads();
        C* s = src; src = dst; dst = s;
        Ns <<= 2;
    }
    return src;
}

__host__ __device__ inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

// ------------------------------------------------------------ row passes
// S Z and the forward row FFT: rows [i0, i0+rb) of the image to rows[i][0..Kx).
// When pdir != null the kernel first forms p = r + beta p in place (CG
// direction update) and transforms the new p.
template <typename T>
__global__ void k_rows_fwd(const T* __restrict__ x, typename cplx_of<T>::type* __restrict__ rows,
                           const T* __restrict__ sx, const T* __restrict__ sy,
                           const typename cplx_of<T>::type* __restrict__ tw, int nx, int ny, int Kx,
                           int rb, T scale, T* pdir, const T* __restrict__ rvec,
                           const double* __restrict__ beta_dev, const int* __restrict__ skip) {
    using C = typename cplx_of<T>::type;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + rb * Kx;
    const int i0 = blockIdx.x * rb;
    const int tot = rb * Kx;
    const T beta = beta_dev ? (T)(*beta_dev) : T(0);
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int f = t / Kx, p1 = t - f * Kx;
        int i = i0 + f;
        // pixel column j with (j - nx/2) mod Kx == p1
        int n1 = p1 < Kx / 2 ? p1 : p1 - Kx;
        int j = n1 + nx / 2;
        T val = T(0);
        if (j >= 0 && j < nx) {
            size_t idx = (size_t)i * nx + j;
            T xv;
            if (pdir) {
                xv = rvec[idx] + beta * pdir[idx];
                pdir[idx] = xv;
            } else {
                xv = x[idx];
            }
            val = xv * sx[j] * sy[i] * scale;
        }
        b0[t] = cmake<C>(val, T(0));
    }
    __syncthreads();
    C* res = fft_smem<C, false>(b0, b1, Kx, ilog2(Kx), rb, Kx, 1, tw);
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int f = t / Kx, k = t - f * Kx;
        rows[(size_t)(i0 + f) * Kx + k] = res[t];
    }
}

// Forward column FFT over columns [c0, c0+cb): the only non-zero grid rows
// are p2 = (i - ny/2) mod Ky for image rows i.
template <typename T>
__global__ void k_cols_fwd(const typename cplx_of<T>::type* __restrict__ rows,
                           typename cplx_of<T>::type* __restrict__ grid,
                           const typename cplx_of<T>::type* __restrict__ tw, int ny, int Kx, int Ky,
                           int cb, const int* __restrict__ skip) {
    using C = typename cplx_of<T>::type;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + cb * Ky;
    const int c0 = blockIdx.x * cb;
    const int tot = cb * Ky;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int k = t / cb, f = t - k * cb;
        int n2 = k < Ky / 2 ? k : k - Ky;
        int i = n2 + ny / 2;
        C v = cmake<C>(T(0), T(0));
        if (i >= 0 && i < ny) v = rows[(size_t)i * Kx + c0 + f];
        b0[t] = v;
    }
    __syncthreads();
    C* res = fft_smem<C, false>(b0, b1, Ky, ilog2(Ky), cb, 1, cb, tw);
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int k = t / cb, f = t - k * cb;
        grid[(size_t)k * Kx + c0 + f] = res[t];
    }
}

// Inverse column FFT over columns [c0, c0+cb), keeping only the image rows.
template <typename T>
__global__ void k_cols_inv(const typename cplx_of<T>::type* __restrict__ grid,
                           typename cplx_of<T>::type* __restrict__ rows,
                           const typename cplx_of<T>::type* __restrict__ tw, int ny, int Kx, int Ky,
                           int cb, const int* __restrict__ skip, const T* __restrict__ mult) {
    using C = typename cplx_of<T>::type;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + cb * Ky;
    const int c0 = blockIdx.x * cb;
    const int tot = cb * Ky;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int k = t / cb, f = t - k * cb;
        size_t g = (size_t)k * Kx + c0 + f;
        C v = grid[g];
        if (mult) v = cscale(v, mult[g]);
        b0[t] = v;
    }
    __syncthreads();
    C* res = fft_smem<C, true>(b0, b1, Ky, ilog2(Ky), cb, 1, cb, tw);
    for (int t = threadIdx.x; t < ny * cb; t += blockDim.x) {
        int i = t / cb, f = t - i * cb;
        int p2 = (i - ny / 2) & (Ky - 1);
        rows[(size_t)i * Kx + c0 + f] = res[p2 * cb + f];
    }
}

// Inverse row FFT of image rows [i0, i0+rb), then Z^T and S:
//   out_mode 0: complex out[i][j] = scale * s * v
//   out_mode 1: real    out[i][j] = scale * s * Re v + add_coef * (add ? add[i][j] : 0)
// With dot_part set (CG, out = A p, add = p) the kernel also forms p . A p
// and, in the last block to finish, alpha = (r . r) / (p . A p).
template <typename T>
__global__ void k_rows_inv(const typename cplx_of<T>::type* __restrict__ rows, void* out,
                           const T* __restrict__ sx, const T* __restrict__ sy,
                           const typename cplx_of<T>::type* __restrict__ tw, int nx, int ny, int Kx,
                           int rb, T scale, int out_mode, const T* __restrict__ add, T add_coef,
                           const int* __restrict__ skip, double* dot_part, unsigned* counters, double* scal) {
    using C = typename cplx_of<T>::type;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + rb * Kx;
    const int i0 = blockIdx.x * rb;
    const int tot = rb * Kx;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int f = t / Kx, k = t - f * Kx;
        b0[t] = rows[(size_t)(i0 + f) * Kx + k];
    }
    __syncthreads();
    C* res = fft_smem<C, true>(b0, b1, Kx, ilog2(Kx), rb, Kx, 1, tw);
    T dacc = 0;
    for (int t = threadIdx.x; t < rb * nx; t += blockDim.x) {
        int f = t / nx, j = t - f * nx;
        int i = i0 + f;
        int p1 = (j - nx / 2) & (Kx - 1);
        C v = res[f * Kx + p1];
        T s = sx[j] * sy[i] * scale;
        size_t idx = (size_t)i * nx + j;
        if (out_mode == 0) {
            reinterpret_cast<C*>(out)[idx] = cscale(v, s);
        } else {
            T r = v.x * s;
            if (add) {
                T a = add[idx];
                r += add_coef * a;
                dacc += a * r;
            }
            reinterpret_cast<T*>(out)[idx] = r;
        }
    }
    if (dot_part) {
        double b = block_sum((double)dacc);
        if (threadIdx.x == 0) dot_part[blockIdx.x] = b;
        if (arrive_last(counters + C_ALPHA)) {
            double tot = ordered_sum(dot_part, gridDim.x);
            if (threadIdx.x == 0) {
                scal[S_PAP] = tot;
                scal[S_ALPHA] = tot > 0.0 ? scal[S_RS] / tot : 0.0;
                counters[C_ALPHA] = 0;
            }
        }
    }
}

// Plain in-place 2-D FFT pieces (purify_fft2): full row pass / column pass.
template <typename T, bool INV>
__global__ void k_rows_full(typename cplx_of<T>::type* grid, const typename cplx_of<T>::type* __restrict__ tw,
                            int Kx, int rb) {
    using C = typename cplx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + rb * Kx;
    const size_t base = (size_t)blockIdx.x * rb * Kx;
    for (int t = threadIdx.x; t < rb * Kx; t += blockDim.x) b0[t] = grid[base + t];
    __syncthreads();
    C* res = fft_smem<C, INV>(b0, b1, Kx, ilog2(Kx), rb, Kx, 1, tw);
    for (int t = threadIdx.x; t < rb * Kx; t += blockDim.x) grid[base + t] = res[t];
}

template <typename T, bool INV>
__global__ void k_cols_full(typename cplx_of<T>::type* grid, const typename cplx_of<T>::type* __restrict__ tw,
                            int Kx, int Ky, int cb) {
    using C = typename cplx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + cb * Ky;
    const int c0 = blockIdx.x * cb;
    for (int t = threadIdx.x; t < cb * Ky; t += blockDim.x) {
        int k = t / cb, f = t - k * cb;
        b0[t] = grid[(size_t)k * Kx + c0 + f];
    }
    __syncthreads();
    C* res = fft_smem<C, INV>(b0, b1, Ky, ilog2(Ky), cb, 1, cb, tw);
    for (int t = threadIdx.x; t < cb * Ky; t += blockDim.x) {
        int k = t / cb, f = t - k * cb;
        grid[(size_t)k * Kx + c0 + f] = res[t];
    }
}

// ------------------------------------------------------ gridding helpers
__device__ __forceinline__ void atomic_add_c(float2* a, float2 v) { atomicAdd(a, v); }
__device__ __forceinline__ void atomic_add_c(double2* a, double2 v) {
    atomicAdd(&a->x, v.x);
    atomicAdd(&a->y, v.y);
}

// Visibility pieces of one subproblem, flattened: a block loads the piece
// starts and the running piece lengths into shared memory so that any thread
// can map a flat index q to its visibility with a binary search.
#define PURIFY_MAX_PIECES 128

__device__ __forceinline__ int load_pieces(const int* __restrict__ piece_off, const int* __restrict__ piece_start,
                                           const int* __restrict__ piece_len, int s, int* pst, int* pcum) {
    const int p0 = piece_off[s], np = piece_off[s + 1] - p0;
    if (threadIdx.x < np) pst[threadIdx.x] = piece_start[p0 + threadIdx.x];
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < np; ++k) { pcum[k] = acc; acc += piece_len[p0 + k]; }
        pcum[np] = acc;
    }
    return np;
}

// visibility of flat index q (0 <= q < pcum[np])
__device__ __forceinline__ int flat_vis(const int* pst, const int* pcum, int np, int q) {
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pcum[mid] <= q) lo = mid; else hi = mid - 1;
    }
    return pst[lo] + (q - pcum[lo]);
}

// G^H by cell runs. A block owns one subproblem: a grid tile and an explicit
// list of its visibilities ordered by first-tap cell across all measurement
// blocks, so that visibilities sharing their J x J cells are adjacent. The
// tile plus its (J-1) halo is one shared-memory array (row stride S).
// The list is cut into WARPS * G contiguous segments, G = 32 / J per warp;
// group g of a warp (lanes gJ .. gJ+J-1) walks its segment in order, lane b
// holding row b of the current run's J x J patch in 2J registers:
//   patch[b][a] += wx[a] * (wy[b] * y)   for every visibility of the run,
// and adding the patch to the shared tile with shared-memory atomics only
// when the first-tap cell changes. The 2J weights and the split of each
// visibility are evaluated once, by one lane, into a per-warp staging area
// (P records per group per batch, P = 32 / G). Finally the tile's non-zero
// cells are added to the grid.
template <int J> struct GridStage {
    static constexpr int G = 32 / J;      // visibility groups per warp
    static constexpr int P = 32 / G;      // records a group stages per batch
    static constexpr int NB = G * P;      // records per warp batch
    // words per staged visibility: wx[J], wy[J], re, im, cell offset (-1:
    // empty or not in this tile); odd so that lanes storing their records
    // fall on distinct banks
    static constexpr int F = 2 * J + 3;
};

template <typename T> __device__ __forceinline__ T int_bits(int v);
template <> __device__ __forceinline__ float int_bits<float>(int v) { return __int_as_float(v); }
template <> __device__ __forceinline__ double int_bits<double>(int v) { return __longlong_as_double((long long)v); }
__device__ __forceinline__ int bits_int(float v) { return __float_as_int(v); }
__device__ __forceinline__ int bits_int(double v) { return (int)__double_as_longlong(v); }

template <typename T, int J, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_grid_runs(const typename cplx_of<T>::type* __restrict__ yin, const T* __restrict__ us, const T* __restrict__ vs,
            AxisConst ax, AxisConst ay, KbPoly kp, double beta, double inv_i0beta, const int* __restrict__ perm,
            const int* __restrict__ sub_bin, const int* __restrict__ sub_off, const int* __restrict__ list, int tile,
            int tiles_x, int S, typename cplx_of<T>::type* __restrict__ grid, const int* __restrict__ skip) {
    using C = typename cplx_of<T>::type;
    using GS = GridStage<J>;
    constexpr int G = GS::G, P = GS::P, NB = GS::NB, F = GS::F;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int PT = tile + J - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C* mt = reinterpret_cast<C*>(smem_raw);                            // [PT][S]
    T* mst = reinterpret_cast<T*>(mt + (size_t)PT * S) + (size_t)warp * NB * F;   // [NB][F]
    for (int t = threadIdx.x; t < PT * S; t += blockDim.x) mt[t] = cmake<C>(T(0), T(0));
    const int s = blockIdx.x;
    const int bin = sub_bin[s];
    const int oy = (bin / tiles_x) * tile, ox = (bin % tiles_x) * tile;
    const int Kx = ax.K, Ky = ay.K;
    const int q0 = sub_off[s], total = sub_off[s + 1] - q0;
    constexpr int NSEG = WARPS * G;
    // segment sg covers list positions [total * sg / NSEG, total * (sg + 1) / NSEG)
    auto seg_lo = [&](int sg) { return (int)(((long long)total * sg) / NSEG); };
    // staging role: lane (gs, js) evaluates record js of group gs
    const int gs = lane / P, js = lane - gs * P;
    const int lo1 = seg_lo(warp * G + gs), len1 = (gs < G) ? seg_lo(warp * G + gs + 1) - lo1 : 0;
    // scatter role: lane (g, b) holds row b of group g's patch
    const int g = lane / J, b = lane - g * J;
    const int nbatch = ((total + NSEG - 1) / NSEG + P - 1) / P;
    __syncthreads();
    int cur = -1;
    T ar[J], ai[J];
#pragma unroll
    for (int a = 0; a < J; ++a) ar[a] = ai[a] = T(0);
    for (int k = 0; k < nbatch; ++k) {
        if (gs < G) {
            T* rec = mst + (gs * P + js) * F;
            const int pos = k * P + js;
            int off = -1;
            if (pos < len1) {
                const int m = list[q0 + lo1 + pos];
                int kx0, ky0;
                T phx, phy;
                split_coord(us[m], ax, J, kx0, phx);
                split_coord(vs[m], ay, J, ky0, phy);
                T wx[J], wy[J];
                if constexpr (sizeof(T) == 4) {
                    kb_weights<J>(kp, phx, wx);
                    kb_weights<J>(kp, phy, wy);
                } else {
                    kb_weights<J>(beta, inv_i0beta, phx, wx);
                    kb_weights<J>(beta, inv_i0beta, phy, wy);
                }
                const C yv = yin[perm ? perm[m] : m];
                const int lx = (kx0 & (Kx - 1)) - ox, ly = (ky0 & (Ky - 1)) - oy;
                if (lx >= 0 && lx < tile && ly >= 0 && ly < tile) {
#pragma unroll
                    for (int a = 0; a < J; ++a) { rec[a] = wx[a]; rec[J + a] = wy[a]; }
                    rec[2 * J] = yv.x;
                    rec[2 * J + 1] = yv.y;
                    off = ly * S + lx;
                } else {
                    // coordinate outside this tile (not expected: the plan
                    // bins with the same split); add straight to the grid
#pragma unroll
                    for (int bb = 0; bb < J; ++bb)
#pragma unroll
                        for (int a = 0; a < J; ++a) {
                            T w = wy[bb] * wx[a];
                            atomic_add_c(grid + (size_t)((ky0 + bb) & (Ky - 1)) * Kx + ((kx0 + a) & (Kx - 1)),
                                         cmake<C>(w * yv.x, w * yv.y));
                        }
                }
            }
            rec[2 * J + 2] = int_bits<T>(off);
        }
        __syncwarp();
        if (g < G) {
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const T* rec = mst + (g * P + j) * F;
                const int o = bits_int(rec[2 * J + 2]);
                if (o >= 0) {
                    if (o != cur) {
                        if (cur >= 0) {
                            C* row = mt + cur + b * S;
#pragma unroll
                            for (int a = 0; a < J; ++a) {
                                atomicAdd(&row[a].x, ar[a]);
                                atomicAdd(&row[a].y, ai[a]);
                                ar[a] = ai[a] = T(0);
                            }
                        }
                        cur = o;
                    }
                    const T wyb = rec[J + b];
                    const T zr = wyb * rec[2 * J], zi = wyb * rec[2 * J + 1];
#pragma unroll
                    for (int a = 0; a < J; ++a) {
                        const T wxa = rec[a];
                        ar[a] = fma(wxa, zr, ar[a]);
                        ai[a] = fma(wxa, zi, ai[a]);
                    }
                }
            }
        }
        __syncwarp();
    }
    if (g < G && cur >= 0) {
        C* row = mt + cur + b * S;
#pragma unroll
        for (int a = 0; a < J; ++a) {
            atomicAdd(&row[a].x, ar[a]);
            atomicAdd(&row[a].y, ai[a]);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < PT * PT; t += blockDim.x) {
        const int r = t / PT, c = t - r * PT;
        const C v = mt[r * S + c];
        if (v.x != T(0) || v.y != T(0))
            atomic_add_c(grid + (size_t)((oy + r) & (Ky - 1)) * Kx + ((ox + c) & (Kx - 1)), v);
    }
}

// G with the tile staged in shared memory: a block owns one subproblem,
// copies the tile plus its (J-1) halo from the grid, then every thread
// interpolates visibilities of the subproblem from the shared copy.
template <typename T, int J>
__global__ void __launch_bounds__(128)
k_degrid_tile(const typename cplx_of<T>::type* __restrict__ grid, const T* __restrict__ us, const T* __restrict__ vs,
              AxisConst ax, AxisConst ay, KbPoly kp, double beta, double inv_i0beta, const int* __restrict__ perm,
              const int* __restrict__ sub_bin, const int* __restrict__ piece_off,
              const int* __restrict__ piece_start, const int* __restrict__ piece_len, int tile, int tiles_x,
              typename cplx_of<T>::type* __restrict__ y, const int* __restrict__ skip) {
    using C = typename cplx_of<T>::type;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int PT = tile + J - 1;
    C* tl = reinterpret_cast<C*>(smem_raw);                   // [PT][PT]
    int* pst = reinterpret_cast<int*>(tl + PT * PT);
    int* pcum = pst + PURIFY_MAX_PIECES;
    const int s = blockIdx.x;
    const int bin = sub_bin[s];
    const int oy = (bin / tiles_x) * tile, ox = (bin % tiles_x) * tile;
    const int Kx = ax.K, Ky = ay.K;
    for (int t = threadIdx.x; t < PT * PT; t += blockDim.x) {
        const int r = t / PT, c = t - r * PT;
        tl[t] = grid[(size_t)((oy + r) & (Ky - 1)) * Kx + ((ox + c) & (Kx - 1))];
    }
    const int np = load_pieces(piece_off, piece_start, piece_len, s, pst, pcum);
    __syncthreads();
    const int total = pcum[np];
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int m = flat_vis(pst, pcum, np, q);
        int kx0, ky0;
        T phx, phy;
        split_coord(us[m], ax, J, kx0, phx);
        split_coord(vs[m], ay, J, ky0, phy);
        T wx[J], wy[J];
        if constexpr (sizeof(T) == 4) {
            kb_weights<J>(kp, phx, wx);
            kb_weights<J>(kp, phy, wy);
        } else {
            kb_weights<J>(beta, inv_i0beta, phx, wx);
            kb_weights<J>(beta, inv_i0beta, phy, wy);
        }
        int lx = (kx0 & (Kx - 1)) - ox, ly = (ky0 & (Ky - 1)) - oy;
        T accx = 0, accy = 0;
        if (lx >= 0 && lx < tile && ly >= 0 && ly < tile) {
#pragma unroll
            for (int b = 0; b < J; ++b) {
                const C* row = tl + (ly + b) * PT + lx;
                T rx = 0, ry = 0;
#pragma unroll
                for (int a = 0; a < J; ++a) {
                    C g = row[a];
                    rx += wx[a] * g.x;
                    ry += wx[a] * g.y;
                }
                accx += wy[b] * rx;
                accy += wy[b] * ry;
            }
        } else {
#pragma unroll
            for (int b = 0; b < J; ++b) {
                const C* row = grid + (size_t)((ky0 + b) & (Ky - 1)) * Kx;
                T rx = 0, ry = 0;
#pragma unroll
                for (int a = 0; a < J; ++a) {
                    C g = row[(kx0 + a) & (Kx - 1)];
                    rx += wx[a] * g.x;
                    ry += wx[a] * g.y;
                }
                accx += wy[b] * rx;
                accy += wy[b] * ry;
            }
        }
        y[perm ? perm[m] : m] = cmake<C>(accx, accy);
    }
}

// ------------------------------------------------------------- launchers
// FFT launch shapes: enough blocks to cover the 152 SMs about twice, one
// radix-4 butterfly per thread per pass where possible.
template <typename T> static int rows_per_block(int nrows, int K) {
    size_t cbytes = sizeof(typename cplx_of<T>::type);
    int rb = std::max(1, std::min(8, nrows / 256));
    while (rb > 1 && (2 * (size_t)rb * K * cbytes > 160 * 1024 || nrows % rb)) rb >>= 1;
    return rb;
}

template <typename T> static int cols_per_block(int Ky, int Kx) {
    size_t cbytes = sizeof(typename cplx_of<T>::type);
    int cb = std::max(1, std::min(8, Kx / 256));
    while (cb > 1 && (2 * (size_t)cb * Ky * cbytes > 160 * 1024 || Kx % cb)) cb >>= 1;
    return cb;
}

static int fft_threads(int nb, int n) { return std::max(64, std::min(256, nb * n / 4)); }

template <typename K> static void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) PURIFY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

template <typename T>
static void rows_fwd_t(purify_plan* p, const void* x, double scale, void* pdir, const void* rvec,
                       const double* beta_dev, const int* skip, bool corr) {
    using C = typename cplx_of<T>::type;
    int rb = p->fft_rb > 0 ? p->fft_rb : rows_per_block<T>(p->ny, p->Kx);
    while (p->ny % rb) rb >>= 1;
    size_t sm = 2 * (size_t)rb * p->Kx * sizeof(C);
    set_smem(k_rows_fwd<T>, sm);
    Launch L(p, "fft_rows_fwd");
    k_rows_fwd<T><<<p->ny / rb, fft_threads(rb, p->Kx), sm, p->stream>>>(
        (const T*)x, p->rows.as<C>(), corr ? p->sx.as<T>() : p->onesx.as<T>(),
        corr ? p->sy.as<T>() : p->onesy.as<T>(), p->twx.as<C>(), p->nx, p->ny, p->Kx,
        rb, (T)scale, (T*)pdir, (const T*)rvec, beta_dev, skip);
    L.done();
}

template <typename T> static void cols_fwd_t(purify_plan* p, const int* skip) {
    using C = typename cplx_of<T>::type;
    int cb = p->fft_cb > 0 ? p->fft_cb : cols_per_block<T>(p->Ky, p->Kx);
    size_t sm = 2 * (size_t)cb * p->Ky * sizeof(C);
    set_smem(k_cols_fwd<T>, sm);
    Launch L(p, "fft_cols_fwd");
    k_cols_fwd<T><<<p->Kx / cb, fft_threads(cb, p->Ky), sm, p->stream>>>(p->rows.as<C>(), p->grid.as<C>(), p->twy.as<C>(),
                                                      p->ny, p->Kx, p->Ky, cb, skip);
    L.done();
}

template <typename T> static void cols_inv_t(purify_plan* p, const int* skip, const void* mult) {
    using C = typename cplx_of<T>::type;
    int cb = p->fft_cb > 0 ? p->fft_cb : cols_per_block<T>(p->Ky, p->Kx);
    size_t sm = 2 * (size_t)cb * p->Ky * sizeof(C);
    set_smem(k_cols_inv<T>, sm);
    Launch L(p, "fft_cols_inv");
    k_cols_inv<T><<<p->Kx / cb, fft_threads(cb, p->Ky), sm, p->stream>>>(p->grid.as<C>(), p->rows.as<C>(), p->twy.as<C>(),
                                                      p->ny, p->Kx, p->Ky, cb, skip, (const T*)mult);
    L.done();
}

template <typename T>
static void rows_inv_t(purify_plan* p, void* out, double scale, int out_mode, const void* add, double add_coef,
                       const int* skip, double* dot_part, unsigned* counters, double* scal, bool corr) {
    using C = typename cplx_of<T>::type;
    int rb = p->fft_rb > 0 ? p->fft_rb : rows_per_block<T>(p->ny, p->Kx);
    while (p->ny % rb) rb >>= 1;
    size_t sm = 2 * (size_t)rb * p->Kx * sizeof(C);
    set_smem(k_rows_inv<T>, sm);
    Launch L(p, "fft_rows_inv");
    k_rows_inv<T><<<p->ny / rb, fft_threads(rb, p->Kx), sm, p->stream>>>(p->rows.as<C>(), out,
                                                      corr ? p->sx.as<T>() : p->onesx.as<T>(),
                                                      corr ? p->sy.as<T>() : p->onesy.as<T>(),
                                                      p->twx.as<C>(), p->nx, p->ny, p->Kx, rb, (T)scale,
                                                      out_mode, (const T*)add, (T)add_coef, skip, dot_part,
                                                      counters, scal);
    L.done();
}

template <typename T, int J> static void degrid_tj(purify_plan* p, void* y, bool caller_order, const int* skip) {
    using C = typename cplx_of<T>::type;
    const GridWork& w = p->dwork;
    if (w.nsub == 0) return;
    const int tile = w.tile, PT = tile + J - 1;
    size_t sm = sizeof(C) * (size_t)PT * PT + sizeof(int) * (2 * PURIFY_MAX_PIECES + 1);
    set_smem(k_degrid_tile<T, J>, sm);
    Launch L(p, "degrid");
    k_degrid_tile<T, J><<<w.nsub, 128, sm, p->stream>>>(
        p->grid.as<C>(), p->us.as<T>(), p->vs.as<T>(), p->ax, p->ay, p->kbp, p->beta, 1.0 / p->i0beta,
        caller_order ? p->perm.as<int>() : nullptr, w.sub_bin.as<int>(), w.piece_off.as<int>(),
        w.piece_start.as<int>(), w.piece_len.as<int>(), tile, w.tiles_x, (C*)y, skip);
    L.done();
}

// row stride of the shared gridding tile (complex cells): at least
// tile + J - 1 and odd, so that the J rows of one patch held by a lane group
// fall on distinct 8-byte bank pairs
static int grid_row_stride(int tile, int J) {
    int S = tile + J - 1;
    return S | 1;
}

template <typename T> static constexpr int grid_warps() { return sizeof(T) == 4 ? 8 : 4; }

template <typename T, int J>
static size_t grid_smem_bytes(int tile) {
    const int PT = tile + J - 1, S = grid_row_stride(tile, J);
    return sizeof(T) * (2 * (size_t)PT * S + (size_t)grid_warps<T>() * GridStage<J>::NB * GridStage<J>::F);
}

template <typename T, int J>
static void grid_tj(purify_plan* p, const void* y, bool caller_order, const int* skip) {
    using C = typename cplx_of<T>::type;
    constexpr int W = grid_warps<T>();
    PURIFY_CUDA(cudaMemsetAsync(p->grid.p, 0, p->grid.bytes, p->stream));
    if (p->work.nsub == 0) return;
    const int tile = p->work.tile;
    const int S = grid_row_stride(tile, J);
    size_t sm = grid_smem_bytes<T, J>(tile);
    set_smem(k_grid_runs<T, J, W>, sm);
    Launch L(p, "grid");
    k_grid_runs<T, J, W><<<p->work.nsub, W * 32, sm, p->stream>>>(
        (const C*)y, p->us.as<T>(), p->vs.as<T>(), p->ax, p->ay, p->kbp, p->beta, 1.0 / p->i0beta,
        caller_order ? p->perm.as<int>() : nullptr, p->work.sub_bin.as<int>(), p->work.sub_off.as<int>(),
        p->work.list.as<int>(), tile, p->work.tiles_x, S, p->grid.as<C>(), skip);
    L.done();
}

// Visibilities per gridding subproblem are a multiple of this unit: every
// group of every warp then stages full batches when the subproblem is full.
int grid_list_unit(int dtype, int J) {
    const int G = 32 / J, P = 32 / G;
    return (dtype == PURIFY_F32 ? grid_warps<float>() : grid_warps<double>()) * G * P;
}

#define PURIFY_J_DISPATCH(J, FN, ...)                                     \
    switch (J) {                                                          \
        case 2: FN<2>(__VA_ARGS__); break;                                \
        case 3: FN<3>(__VA_ARGS__); break;                                \
        case 4: FN<4>(__VA_ARGS__); break;                                \
        case 5: FN<5>(__VA_ARGS__); break;                                \
        case 6: FN<6>(__VA_ARGS__); break;                                \
        case 7: FN<7>(__VA_ARGS__); break;                                \
        case 8: FN<8>(__VA_ARGS__); break;                                \
        default: throw Error{PURIFY_EINVAL, "kb_width out of range"};     \
    }

template <int J> static void degrid_f(purify_plan* p, void* y, bool c, const int* s) { degrid_tj<float, J>(p, y, c, s); }
template <int J> static void degrid_d(purify_plan* p, void* y, bool c, const int* s) { degrid_tj<double, J>(p, y, c, s); }
template <int J> static void grid_f(purify_plan* p, const void* y, bool c, const int* s) { grid_tj<float, J>(p, y, c, s); }
template <int J> static void grid_d(purify_plan* p, const void* y, bool c, const int* s) { grid_tj<double, J>(p, y, c, s); }

template <int J> static int max_tile_f() {
    int t = 64;
    while (t > 8 && grid_smem_bytes<float, J>(t) > 200 * 1024) t >>= 1;
    return t;
}
template <int J> static int max_tile_d() {
    int t = 64;
    while (t > 8 && grid_smem_bytes<double, J>(t) > 200 * 1024) t >>= 1;
    return t;
}

// Largest gridding tile whose shared-memory tile copies fit a block.
int max_grid_tile(int dtype, int J) {
    int t = 8;
    if (dtype == PURIFY_F32) { PURIFY_J_DISPATCH(J, t = max_tile_f, ); }
    else { PURIFY_J_DISPATCH(J, t = max_tile_d, ); }
    return t;
}

void launch_scale_pad_rows(purify_plan* p, const void* x, double scale, void* pdir, const void* rvec,
                           const double* beta_dev, const int* skip, bool corr) {
    if (p->dtype == PURIFY_F32) rows_fwd_t<float>(p, x, scale, pdir, rvec, beta_dev, skip, corr);
    else rows_fwd_t<double>(p, x, scale, pdir, rvec, beta_dev, skip, corr);
}
void launch_cols_fwd(purify_plan* p, const int* skip) {
    if (p->dtype == PURIFY_F32) cols_fwd_t<float>(p, skip); else cols_fwd_t<double>(p, skip);
}
void launch_cols_inv(purify_plan* p, const int* skip, const void* mult) {
    if (p->dtype == PURIFY_F32) cols_inv_t<float>(p, skip, mult); else cols_inv_t<double>(p, skip, mult);
}
void launch_rows_inv_crop(purify_plan* p, void* out, double scale, int out_mode, const void* add, double add_coef,
                          const int* skip, double* dot_part, unsigned* counters, double* scal, bool corr) {
    if (p->dtype == PURIFY_F32)
        rows_inv_t<float>(p, out, scale, out_mode, add, add_coef, skip, dot_part, counters, scal, corr);
    else
        rows_inv_t<double>(p, out, scale, out_mode, add, add_coef, skip, dot_part, counters, scal, corr);
}
void launch_degrid(purify_plan* p, void* y, bool caller_order, const int* skip) {
    if (p->dtype == PURIFY_F32) { PURIFY_J_DISPATCH(p->J, degrid_f, p, y, caller_order, skip); }
    else { PURIFY_J_DISPATCH(p->J, degrid_d, p, y, caller_order, skip); }
}
void launch_grid(purify_plan* p, const void* y, bool caller_order, const int* skip) {
    if (p->dtype == PURIFY_F32) { PURIFY_J_DISPATCH(p->J, grid_f, p, y, caller_order, skip); }
    else { PURIFY_J_DISPATCH(p->J, grid_d, p, y, caller_order, skip); }
}

void launch_phi(purify_plan* p, const void* x, void* y, bool caller_order, double scale) {
    launch_scale_pad_rows(p, x, scale, nullptr, nullptr, nullptr, nullptr);
    launch_cols_fwd(p, nullptr);
    launch_degrid(p, y, caller_order, nullptr);
}

void launch_phi_adj(purify_plan* p, const void* y, void* out, bool caller_order, double scale, int out_mode,
                    const void* add) {
    launch_grid(p, y, caller_order, nullptr);
    launch_cols_inv(p, nullptr);
    launch_rows_inv_crop(p, out, scale, out_mode, add, 1.0, nullptr);
}

template <typename T> static void fft2_t(purify_plan* p, void* grid, bool inverse) {
    using C = typename cplx_of<T>::type;
    int rb = rows_per_block<T>(p->Ky, p->Kx);
    while (p->Ky % rb) rb >>= 1;
    size_t smr = 2 * (size_t)rb * p->Kx * sizeof(C);
    int cb = cols_per_block<T>(p->Ky, p->Kx);
    size_t smc = 2 * (size_t)cb * p->Ky * sizeof(C);
    if (inverse) {
        set_smem(k_rows_full<T, true>, smr);
        set_smem(k_cols_full<T, true>, smc);
        { Launch L(p, "fft_full_rows"); k_rows_full<T, true><<<p->Ky / rb, fft_threads(rb, p->Kx), smr, p->stream>>>((C*)grid, p->twx.as<C>(), p->Kx, rb); L.done(); }
        { Launch L(p, "fft_full_cols"); k_cols_full<T, true><<<p->Kx / cb, fft_threads(cb, p->Ky), smc, p->stream>>>((C*)grid, p->twy.as<C>(), p->Kx, p->Ky, cb); L.done(); }
    } else {
        set_smem(k_rows_full<T, false>, smr);
        set_smem(k_cols_full<T, false>, smc);
        { Launch L(p, "fft_full_rows"); k_rows_full<T, false><<<p->Ky / rb, fft_threads(rb, p->Kx), smr, p->stream>>>((C*)grid, p->twx.as<C>(), p->Kx, rb); L.done(); }
        { Launch L(p, "fft_full_cols"); k_cols_full<T, false><<<p->Kx / cb, fft_threads(cb, p->Ky), smc, p->stream>>>((C*)grid, p->twy.as<C>(), p->Kx, p->Ky, cb); L.done(); }
    }
}

void launch_fft2(purify_plan* p, void* grid, bool inverse) {
    if (p->dtype == PURIFY_F32) fft2_t<float>(p, grid, inverse); else fft2_t<double>(p, grid, inverse);
}

}  // namespace purify
