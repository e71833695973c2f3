// Measurement operator Phi = G F Z S and its adjoint S Z^T F^H G^H: the
// gridding steps and the operator-level launchers.
//
// The paper (Sec. 1) writes the measurement equation as y = Phi x + n and
// leaves the discretisation open; the plan realises Phi with Kaiser-Bessel
// gridding on a K = alpha n oversampled grid:
//   rows_fwd  : S, Z and the row pass of F over the ny image rows only (the
//               other K - ny grid rows are zero and never stored);
//   cols_fwd  : column pass of F, treating the missing rows as zeros;
//   degrid    : G, J x J separable Kaiser-Bessel interpolation per visibility;
//   grid      : G^H, accumulation of the J x J footprints;
//   cols_inv  : column pass of F^H producing only the ny rows kept by Z^T;
//   rows_inv  : row pass of F^H fused with Z^T (crop) and S.
// The four FFT passes (radix-8 Stockham transforms in shared memory) are in
// fft.cu; this file holds G, G^H, the fused G^H G and the launchers.
#include <type_traits>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "cg.cuh"
#include "internal.h"
#include "launch.h"
#include "reduce.cuh"

namespace purify {

// ------------------------------------------------------ gridding helpers
__device__ __forceinline__ void atomic_add_c(float2* a, float2 v) { atomicAdd(a, v); }
__device__ __forceinline__ void atomic_add_c(double2* a, double2 v) {
    atomicAdd(&a->x, v.x);
    atomicAdd(&a->y, v.y);
}

// Adds the J complex values (ar[a], ai[a]) to row[c0 .. c0 + J) of a grid row
// of Kx cells (periodic): where the segment does not wrap, two cells at a
// time with 16-byte vector reductions (one L2 operation for two cells), the
// odd cells at the ends with 8-byte ones.
template <int J>
__device__ __forceinline__ void red_row(float2* row, int c0, int Kx, const float (&ar)[J], const float (&ai)[J]) {
    if (c0 + J <= Kx) {
        float2* q = row + c0;
        int a = 0;
        if (c0 & 1) {
            atomicAdd(q, make_float2(ar[0], ai[0]));
            a = 1;
        }
#pragma unroll
        for (int k = 0; k < J; ++k) {
            if (k < a || k + 1 >= J || ((k - a) & 1)) continue;
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(q + k), "f"(ar[k]), "f"(ai[k]),
                         "f"(ar[k + 1]), "f"(ai[k + 1])
                         : "memory");
        }
        if (((J - a) & 1) != 0) atomicAdd(q + (J - 1), make_float2(ar[J - 1], ai[J - 1]));
    } else {
#pragma unroll
        for (int k = 0; k < J; ++k) atomicAdd(row + ((c0 + k) & (Kx - 1)), make_float2(ar[k], ai[k]));
    }
}
template <int J>
__device__ __forceinline__ void red_row(double2* row, int c0, int Kx, const double (&ar)[J], const double (&ai)[J]) {
#pragma unroll
    for (int k = 0; k < J; ++k) atomic_add_c(row + ((c0 + k) & (Kx - 1)), make_double2(ar[k], ai[k]));
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
    pdl_wait();
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
    pdl_trigger();
}

// J consecutive values from a 16-byte aligned shared-memory slot in 16-byte
// (then 8-, then 4-byte) loads.
template <int J> __device__ __forceinline__ void lds_vec(const float* s, float (&v)[J]) {
#pragma unroll
    for (int i = 0; i + 4 <= J; i += 4) {
        const float4 t = *reinterpret_cast<const float4*>(s + i);
        v[i] = t.x;
        v[i + 1] = t.y;
        v[i + 2] = t.z;
        v[i + 3] = t.w;
    }
    constexpr int o = J & ~3;
    if constexpr ((J & 3) >= 2) {
        const float2 t = *reinterpret_cast<const float2*>(s + o);
        v[o] = t.x;
        v[o + 1] = t.y;
    }
    if constexpr ((J & 1) != 0) v[J - 1] = s[J - 1];
}
template <int J> __device__ __forceinline__ void lds_vec(const double* s, double (&v)[J]) {
#pragma unroll
    for (int i = 0; i < J; ++i) v[i] = s[i];
}
template <int J> __device__ __forceinline__ void lds_vec(const float2* s, float2 (&v)[J]) {
    const float4* q = reinterpret_cast<const float4*>(s);
#pragma unroll
    for (int i = 0; i < J / 2; ++i) {
        const float4 t = q[i];
        v[2 * i] = make_float2(t.x, t.y);
        v[2 * i + 1] = make_float2(t.z, t.w);
    }
    if constexpr ((J & 1) != 0) v[J - 1] = s[J - 1];
}
template <int J> __device__ __forceinline__ void lds_vec(const double2* s, double2 (&v)[J]) {
#pragma unroll
    for (int i = 0; i < J; ++i) v[i] = s[i];
}

// J consecutive complex values of a grid row of Kx cells (periodic) from
// column c0: where the segment does not wrap, two cells per 16-byte load.
template <int J>
__device__ __forceinline__ void ldg_row(const float2* __restrict__ row, int c0, int Kx, float2 (&v)[J]) {
    if (c0 + J <= Kx) {
        const float2* q = row + c0;
        int a = 0;
        if (c0 & 1) {
            v[0] = q[0];
            a = 1;
        }
#pragma unroll
        for (int k = 0; k < J; ++k) {
            if (k < a || k + 1 >= J || ((k - a) & 1)) continue;
            const float4 t = *reinterpret_cast<const float4*>(q + k);
            v[k] = make_float2(t.x, t.y);
            v[k + 1] = make_float2(t.z, t.w);
        }
        if (((J - a) & 1) != 0) v[J - 1] = q[J - 1];
    } else {
#pragma unroll
        for (int k = 0; k < J; ++k) v[k] = row[(c0 + k) & (Kx - 1)];
    }
}
template <int J>
__device__ __forceinline__ void ldg_row(const double2* __restrict__ row, int c0, int Kx, double2 (&v)[J]) {
#pragma unroll
    for (int k = 0; k < J; ++k) v[k] = row[(c0 + k) & (Kx - 1)];
}

// G^H (and the fused G^H G) by run sets. Warp w of the grid takes sets
// w, 2W - 1 - w, 2W + w, ... (W warps in all; sets are sorted by length, so
// the alternating order balances the warps); lane group g (lanes gJ ..
// gJ+J-1) walks run g of the set, which holds visibilities sharing one
// first-tap cell (cx, cy). For each visibility lane b evaluates tap b of
// both axes (wx[b], wy[b]) and the group exchanges the wx through a
// warp-private shared-memory slot (one store, 16-byte loads: lighter on the
// shuffle pipe than J shuffles); lane b accumulates row b of the cell's
// J x J patch in registers,
//   patch[b][a] += wx[a] * (wy[b] * y),
// and the set's runs (about equally long) are flushed together with vector
// global reductions after the longest run of the set. The step has no
// branch but the loop's: lanes outside every group store to a spare slot,
// and a step past the end of a lane's run adds zero.
// Gridding (y given): lane b loads every J-th record of the run (two batches
// of J records in flight) and the group reads them by shuffles; the weight
// slot is double-buffered by step parity.
// Fused (G^H G X): the visibility value is not read but interpolated from
// the forward grid X. Lane b holds row b of X's J x J patch at the run's
// cell (read two cells per 16-byte load where the row segment is aligned
// and does not wrap),
//   y = sum_b wy[b] sum_a wx[a] X[cy + b][cx + a],
// summed over the group (in b order) through a second shared slot, so
// G^H G X needs no visibility vector. All J lanes of a group read the split
// of the group's next record directly, one step ahead; the two warp
// barriers of a step order every reuse of the single-buffered slots.
template <int DEG> __device__ __forceinline__ float kb_tap_poly(const float (&c)[DEG + 1], float phi) {
    const float z = fmaf(2.0f, phi, -1.0f);
    float acc = c[DEG];
#pragma unroll
    for (int i = DEG - 1; i >= 0; --i) acc = fmaf(acc, z, c[i]);
    return acc;
}
__device__ __forceinline__ double kb_tap_exact(int J, int a, double beta, double inv_i0beta, double phi) {
    const double t = phi + (0.5 * J - 1.0 - a);
    const double r = 1.0 - (2.0 * t / J) * (2.0 * t / J);
    return r > 0.0 ? bessel_i0_series(beta * sqrt(r)) * inv_i0beta : (r == 0.0 ? inv_i0beta : 0.0);
}

template <typename T, int J, int WARPS, bool FUSED>
__global__ void __launch_bounds__(WARPS * 32)
k_grid_sets(const typename cplx_of<T>::type* __restrict__ yin, const typename cplx_of<T>::type* __restrict__ X,
            const typename RunRecOf<T>::type* __restrict__ recs, const int* __restrict__ run_cell,
            const int* __restrict__ run_start, const int* __restrict__ run_len, int nsets,
            const int* __restrict__ perm, KbPoly kp, double beta, double inv_i0beta, int Kx, int Ky,
            typename cplx_of<T>::type* __restrict__ out, const int* __restrict__ skip) {
    using C = typename cplx_of<T>::type;
    using Rec = typename RunRecOf<T>::type;
    constexpr int G = 32 / J;
    constexpr int DEG = kb_poly_deg(J);
    pdl_wait();
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int g = lane / J, b = lane - g * J;
    const bool act = g < G;
    const int gg = act ? g : 0;
    const int src = gg * J;
    const int W = gridDim.x * WARPS, wg = blockIdx.x * WARPS + (threadIdx.x >> 5);
    // per warp, per step parity, per group: J weights and J complex terms,
    // read back with 16-byte loads; the group strides keep 16-byte alignment
    // and put the groups' 16-byte reads of one instruction on distinct banks
    // (the terms' stride of 6 complex values, for J <= 6, also puts each
    // half-warp's 8-byte stores on distinct banks)
    constexpr int SWS = sizeof(T) == 4 ? 12 : 10, STS = sizeof(T) == 4 ? (J <= 6 ? 6 : 10) : 9;
    constexpr int GS = G + (32 % J != 0 ? 1 : 0);   // + a slot the idle lanes write to
    constexpr int NPAR = FUSED ? 1 : 2;
    __shared__ __align__(16) T s_w[WARPS][NPAR][GS][SWS];
    __shared__ __align__(16) C s_t[FUSED ? WARPS : 1][GS][STS];
    T (*sw)[GS][SWS] = s_w[threadIdx.x >> 5];
    C (*st)[STS] = s_t[FUSED ? (threadIdx.x >> 5) : 0];
    auto set_of = [&](int i) { return i * W + ((i & 1) ? W - 1 - wg : wg); };
    float cf[DEG + 1];
#pragma unroll
    for (int i = 0; i <= DEG; ++i) cf[i] = kp.coef[b][i];
    struct Meta { int len, lmax, start; unsigned cell; };
    auto load_meta = [&](int set, Meta& m) {
        if (set < nsets) {
            const int r = set * G + gg;
            m.len = act ? run_len[r] : 0;
            m.lmax = run_len[set * G];   // the set's longest run
            m.start = run_start[r];
            m.cell = (unsigned)run_cell[r];
        } else {
            m.len = m.lmax = m.start = 0;
            m.cell = 0;
        }
    };
    auto load_rec = [&](const Meta& m, int k, Rec& r) {
        if (k < m.len) r = recs[m.start + k];
        else { r.phx = r.phy = T(0); r.m = -1; r.pad = 0; }
    };
    int it = 0, set = set_of(0);
    Meta cur;
    load_meta(set, cur);
    while (set < nsets) {
        const int nset = set_of(it + 1);
        Meta nxt;
        load_meta(nset, nxt);
        const int cx = (int)(cur.cell & 0xFFFFu), cy = (int)(cur.cell >> 16);
        const size_t rowoff = (size_t)((cy + b) & (Ky - 1)) * Kx;
        T xr[J], xi[J];
        if constexpr (FUSED) {
            C xv[J];
            if (cur.len > 0) {
                ldg_row<J>(X + rowoff, cx, Kx, xv);
            } else {
#pragma unroll
                for (int a = 0; a < J; ++a) xv[a] = cmake<C>(T(0), T(0));
            }
#pragma unroll
            for (int a = 0; a < J; ++a) {
                xr[a] = xv[a].x;
                xi[a] = xv[a].y;
            }
        }
        T ar[J], ai[J];
#pragma unroll
        for (int a = 0; a < J; ++a) ar[a] = ai[a] = T(0);
        // gridding: this lane's records of the current and the next batch
        // of J, read by the group through shuffles; fused: the split of the
        // group's record k, read by all J lanes of the group, one step ahead
        Rec bcur, bnext;
        C ycur = cmake<C>(T(0), T(0)), rc = cmake<C>(T(0), T(0));
        auto split_at = [&](int k) {
            C v = cmake<C>(T(0), T(0));
            if (k < cur.len) {
                const Rec* q = recs + cur.start + k;
                v = cmake<C>(q->phx, q->phy);
            }
            return v;
        };
        if constexpr (FUSED) {
            rc = split_at(0);
        } else {
            load_rec(cur, b, bcur);
            load_rec(cur, J + b, bnext);
            if (bcur.m >= 0) ycur = yin[perm ? perm[bcur.m] : bcur.m];
        }
        int kk = 0;
        for (int k = 0; k < cur.lmax; ++k) {
            T phx, phy;
            C yv;
            if constexpr (FUSED) {
                const C rn = split_at(k + 1);
                phx = rc.x;
                phy = rc.y;
                rc = rn;
            } else {
                const int sl = src + kk;
                phx = __shfl_sync(0xffffffffu, bcur.phx, sl);
                phy = __shfl_sync(0xffffffffu, bcur.phy, sl);
                yv.x = __shfl_sync(0xffffffffu, ycur.x, sl);
                yv.y = __shfl_sync(0xffffffffu, ycur.y, sl);
                if (++kk == J) {
                    kk = 0;
                    bcur = bnext;
                    load_rec(cur, k + 1 + J + b, bnext);
                    ycur = cmake<C>(T(0), T(0));
                    if (bcur.m >= 0) ycur = yin[perm ? perm[bcur.m] : bcur.m];
                }
            }
            const bool valid = k < cur.len;
            T wxb, wyb;
            if constexpr (sizeof(T) == 4) {
                wxb = kb_tap_poly<DEG>(cf, phx);
                wyb = kb_tap_poly<DEG>(cf, phy);
            } else {
                wxb = kb_tap_exact(J, b, beta, inv_i0beta, phx);
                wyb = kb_tap_exact(J, b, beta, inv_i0beta, phy);
            }
            const int par = NPAR == 1 ? 0 : (k & 1);
            sw[par][g][b] = wxb;
            __syncwarp();
            T wx[J];
            lds_vec<J>(sw[par][gg], wx);
            if constexpr (FUSED) {
                T rx = 0, ry = 0;
#pragma unroll
                for (int a = 0; a < J; ++a) {
                    rx = fma(wx[a], xr[a], rx);
                    ry = fma(wx[a], xi[a], ry);
                }
                st[g][b] = cmake<C>(wyb * rx, wyb * ry);
                __syncwarp();
                C tv[J];
                lds_vec<J>(st[gg], tv);
                T sr = 0, si = 0;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    sr += tv[j].x;
                    si += tv[j].y;
                }
                yv = cmake<C>(sr, si);
            }
            {
                const T zr = valid ? wyb * yv.x : T(0), zi = valid ? wyb * yv.y : T(0);
#pragma unroll
                for (int a = 0; a < J; ++a) {
                    ar[a] = fma(wx[a], zr, ar[a]);
                    ai[a] = fma(wx[a], zi, ai[a]);
                }
            }
        }
        if (cur.len > 0) red_row<J>(out + rowoff, cx, Kx, ar, ai);
        cur = nxt;
        set = nset;
        ++it;
    }
    pdl_trigger();
}

// Lane-per-run forms of G^H G, G^H and G (FP32, J <= 6; see LaneWork). A
// warp takes a set of 32 / H runs (sets w, 2W - 1 - w, 2W + w, ... for warp
// w of W, which balances the length-sorted sets); the H lanes r, r + 32 / H,
// ... own run r of the set, lane h of them rows [h RH, (h + 1) RH) of the
// run's J x J patch (RH = ceil(J / H)): it holds those rows of the forward
// grid X (G^H G, G) and/or of the accumulator (G^H G, G^H) in registers and
// walks the run's visibilities. With H = 1 a lane evaluates all 2J tap
// weights itself; with H = 2 the lane pair evaluates the J weights of one
// axis each and swaps them with one shuffle per tap, and adds its partial
// interpolation to its partner's with one more. Per visibility (Horner in
// the per-tap polynomials, coefficients taken from the kernel parameters):
//   G^H G: y = sum_b wy[b] sum_a wx[a] X[b][a];  acc[b][a] += wx[a] wy[b] y
//   G^H  : y = yin[idx];                          acc[b][a] += wx[a] wy[b] y
//   G    : yout[idx] = sum_b wy[b] sum_a wx[a] X[b][a]
// One step of the warp reads 32 / H consecutive records, three steps ahead
// (with H = 2 each lane only its own axis offset); padding records (past a
// run's end) get zero weights. The accumulators are flushed with vector
// reductions after the set.
enum { LANE_GG = 0, LANE_GRID = 1, LANE_DEGRID = 2 };

// Shared staging of the lane kernels: per warp two buffers (current and next
// set) of each lane's RH x J patch of X, lane stride RH J + 1 complex values
// (odd, so the 8-byte accesses of a half-warp fall on distinct banks).
template <int J, int H> struct LaneStage {
    static constexpr int RH = (J + H - 1) / H;
    static constexpr int LS = RH * J + 1;
    static constexpr size_t bytes_per_warp = 2 * 32 * LS * sizeof(float2);
};

__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// With DET the accumulators are not added to the grid: run q's J x J patch
// is stored at out[(b J + a) * dstride + q] (q = set * (32 / H) + its lane
// in the set), for k_lane_gather to sum in a fixed order.
template <int J, int MODE, int H, bool DET = false>
__global__ void __launch_bounds__(128, H == 2 ? (DET ? 3 : 4) : 1)
k_lane(const float2* __restrict__ X, const float2* __restrict__ yin, float2* __restrict__ yout,
       const int2* __restrict__ set_info, const int2* __restrict__ run_cl, const float2* __restrict__ recs,
       const int* __restrict__ idx, int nsets, KbPoly kp, int Kx, int Ky, float2* __restrict__ out,
       const int* __restrict__ skip, int64_t dstride) {
    constexpr bool HAS_X = MODE != LANE_GRID, HAS_ACC = MODE != LANE_DEGRID;
    constexpr int WID = 32 / H, RH = LaneStage<J, H>::RH, LS = LaneStage<J, H>::LS;
    pdl_wait();
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, r = lane % WID, h = lane / WID;
    const int W = gridDim.x * (blockDim.x >> 5), wg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // this lane's two staging buffers
    float2* stage = reinterpret_cast<float2*>(smem_raw) + ((size_t)(threadIdx.x >> 5) * 64 + lane) * LS;
    auto buf = [&](int i) { return stage + (size_t)(i & 1) * 32 * LS; };
    auto set_of = [&](int i) { return i * W + ((i & 1) ? W - 1 - wg : wg); };
    // this lane's rows of a run's X patch into a staging buffer
    auto patch_async = [&](int2 rcn, float2* dst) {
        const int cx = rcn.x & 0xFFFF, cy = (int)((unsigned)rcn.x >> 16);
        if (rcn.y <= 0) return;
#pragma unroll
        for (int i = 0; i < RH; ++i) {
            const int b = h * RH + i;
            if (b < J) {
                const float2* row = X + (size_t)((cy + b) & (Ky - 1)) * Kx;
#pragma unroll
                for (int a = 0; a < J; ++a) cp_async8(dst + i * J + a, row + ((cx + a) & (Kx - 1)));
            }
        }
    };
    // records: with H = 2 each lane reads its own axis offset (the work
    // stores a record row as the 16 runs' x offsets, then their y offsets),
    // with H = 1 both offsets; PD steps ahead of their use
    using Rec = typename std::conditional<H == 2, float, float2>::type;
    constexpr int PD = 3;
    const Rec* __restrict__ rl = reinterpret_cast<const Rec*>(recs);
    auto rec_at = [&](int row0, int k) -> Rec { return rl[(size_t)(row0 + k) * 32 + lane]; };
    auto idx_at = [&](int row0, int k) -> int { return idx[(size_t)(row0 + k) * WID + r]; };
    int set = set_of(0);
    int2 si = make_int2(0, 0), rc = make_int2(0, 0);
    Rec fq[PD];
    int fi[PD];
#pragma unroll
    for (int j = 0; j < PD; ++j) {
        fq[j] = Rec{};
        fi[j] = -1;
    }
    if (set < nsets) {
        si = set_info[set];
        rc = run_cl[(size_t)set * WID + r];
#pragma unroll
        for (int j = 0; j < PD; ++j) {
            if (si.y > j) {
                fq[j] = rec_at(si.x, j);
                if (MODE != LANE_GG) fi[j] = idx_at(si.x, j);
            }
        }
        if constexpr (HAS_X) patch_async(rc, buf(0));
    }
    cp_async_commit();
    // the next set's descriptors, loaded a set ahead of their use
    int nset = set_of(1);
    int2 nsi = make_int2(0, 0), nrc = make_int2(0, 0);
    if (nset < nsets) {
        nsi = set_info[nset];
        nrc = run_cl[(size_t)nset * WID + r];
    }
    for (int it = 0; set < nsets; ++it) {
        const bool has_next = nset < nsets;
        const int n2set = set_of(it + 2);
        int2 n2si = make_int2(0, 0), n2rc = make_int2(0, 0);
        if (n2set < nsets) {
            n2si = set_info[n2set];
            n2rc = run_cl[(size_t)n2set * WID + r];
        }
        const int cx = rc.x & 0xFFFF, cy = (int)((unsigned)rc.x >> 16), len = rc.y;
        // complex patch values and accumulators as (re, im) pairs: the
        // interpolation and spreading below are packed two-lane FP32
        // multiply-adds (per component the same roundings as scalar ones)
        float2 xv[HAS_X ? RH : 1][HAS_X ? J : 1];
        float2 av[HAS_ACC ? RH : 1][HAS_ACC ? J : 1];
        if constexpr (HAS_X) {
            cp_async_wait_all();
            const float2* cur = buf(it);
#pragma unroll
            for (int i = 0; i < RH; ++i) {
                const bool rowok = len > 0 && h * RH + i < J;
#pragma unroll
                for (int a = 0; a < J; ++a) {
                    const float2 v = rowok ? cur[i * J + a] : make_float2(0.f, 0.f);
                    xv[i][a] = v;
                }
            }
        }
        if constexpr (HAS_ACC) {
#pragma unroll
            for (int i = 0; i < RH; ++i)
#pragma unroll
                for (int a = 0; a < J; ++a) av[i][a] = make_float2(0.f, 0.f);
        }
        // the next set's patch (into the buffer read at the start of the
        // previous set) and first records, a whole set ahead of their use
        Rec nq[PD];
        int ni[PD];
#pragma unroll
        for (int j = 0; j < PD; ++j) {
            nq[j] = Rec{};
            ni[j] = -1;
        }
        if (has_next) {
            if constexpr (HAS_X) patch_async(nrc, buf(it + 1));
#pragma unroll
            for (int j = 0; j < PD; ++j) {
                if (nsi.y > j) {
                    nq[j] = rec_at(nsi.x, j);
                    if (MODE != LANE_GG) ni[j] = idx_at(nsi.x, j);
                }
            }
        }
        cp_async_commit();
        const int row0 = si.x, lmax = si.y;
        Rec rq[PD];
        int iq[PD];
#pragma unroll
        for (int j = 0; j < PD; ++j) {
            rq[j] = fq[j];
            iq[j] = fi[j];
        }
        // gridding: the values of the next YD steps (indices are PD > YD
        // steps ahead)
        constexpr int YD = MODE == LANE_GRID ? 2 : 1;
        static_assert(YD < PD, "value prefetch needs the index further ahead");
        float2 yq[YD];
#pragma unroll
        for (int j = 0; j < YD; ++j) {
            yq[j] = make_float2(0.f, 0.f);
            if (MODE == LANE_GRID && iq[j] >= 0) yq[j] = yin[iq[j]];
        }
        for (int k = 0; k < lmax; ++k) {
            // records PD steps ahead, gridding values YD steps ahead
            Rec rn = Rec{};
            int in = -1;
            if (k + PD < lmax) {
                rn = rec_at(row0, k + PD);
                if (MODE != LANE_GG) in = idx_at(row0, k + PD);
            }
            float2 ynew = make_float2(0.f, 0.f);
            if (MODE == LANE_GRID && iq[YD] >= 0) ynew = yin[iq[YD]];
            const bool valid = k < len;
            float wx[J], wy[RH];
            if constexpr (H == 1) {
                kb_weights<J>(kp, rq[0].x, wx);
                kb_weights<J>(kp, rq[0].y, wy);
            } else {
                // this lane's axis, then the partner's by shuffle
                float own[J], oth[J];
                kb_weights<J>(kp, rq[0], own);
#pragma unroll
                for (int a = 0; a < J; ++a) oth[a] = __shfl_xor_sync(0xffffffffu, own[a], WID);
#pragma unroll
                for (int a = 0; a < J; ++a) wx[a] = h ? oth[a] : own[a];
#pragma unroll
                for (int i = 0; i < RH; ++i) {
                    const float w0 = oth[i];                                              // row i (h = 0)
                    const float w1 = RH + i < J ? own[RH + i < J ? RH + i : 0] : 0.f;   // row RH + i (h = 1)
                    wy[i] = h ? w1 : w0;
                }
            }
            float yr = 0.f, yi = 0.f;
            if constexpr (HAS_X) {
                float2 y2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < RH; ++i) {
                    float2 t = make_float2(0.f, 0.f);
#pragma unroll
                    for (int a = 0; a < J; ++a) t = __ffma2_rn(make_float2(wx[a], wx[a]), xv[i][a], t);
                    y2 = __ffma2_rn(make_float2(wy[i], wy[i]), t, y2);
                }
                yr = y2.x;
                yi = y2.y;
                if constexpr (H == 2) {
                    // the pair's two halves (addition commutes exactly, so
                    // both lanes hold the same sum)
                    yr += __shfl_xor_sync(0xffffffffu, yr, WID);
                    yi += __shfl_xor_sync(0xffffffffu, yi, WID);
                }
                // a step past the run's end contributes nothing
                if (!valid) yr = yi = 0.f;
            }
            if constexpr (MODE == LANE_GRID) {
                yr = yq[0].x;
                yi = yq[0].y;
            }
            if constexpr (MODE == LANE_DEGRID) {
                if (valid && iq[0] >= 0 && h == 0) yout[iq[0]] = make_float2(yr, yi);
            }
            if constexpr (HAS_ACC) {
#pragma unroll
                for (int i = 0; i < RH; ++i) {
                    const float2 u = __fmul2_rn(make_float2(wy[i], wy[i]), make_float2(yr, yi));
#pragma unroll
                    for (int a = 0; a < J; ++a) av[i][a] = __ffma2_rn(make_float2(wx[a], wx[a]), u, av[i][a]);
                }
            }
#pragma unroll
            for (int j = 0; j + 1 < PD; ++j) {
                rq[j] = rq[j + 1];
                iq[j] = iq[j + 1];
            }
            rq[PD - 1] = rn;
            iq[PD - 1] = in;
#pragma unroll
            for (int j = 0; j + 1 < YD; ++j) yq[j] = yq[j + 1];
            yq[YD - 1] = ynew;
        }
        if constexpr (HAS_ACC) {
            if (len > 0) {
                if constexpr (DET) {
                    // this lane's rows, tap by tap (consecutive runs of the
                    // set write consecutive slots of each tap plane)
                    float2* P = out + (size_t)set * WID + r + (size_t)(h * RH * J) * dstride;
#pragma unroll
                    for (int i = 0; i < RH; ++i) {
                        if (h * RH + i < J) {
#pragma unroll
                            for (int a = 0; a < J; ++a) {
                                *P = av[i][a];
                                P += dstride;
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < RH; ++i) {
                        const int b = h * RH + i;
                        if (b < J) {
                            float ar[J], ai[J];
#pragma unroll
                            for (int a = 0; a < J; ++a) {
                                ar[a] = av[i][a].x;
                                ai[a] = av[i][a].y;
                            }
                            red_row<J>(out + (size_t)((cy + b) & (Ky - 1)) * Kx, cx, Kx, ar, ai);
                        }
                    }
                }
            }
        }
        set = nset;
        si = nsi;
        rc = nrc;
        nset = n2set;
        nsi = n2si;
        nrc = n2rc;
#pragma unroll
        for (int j = 0; j < PD; ++j) {
            fq[j] = nq[j];
            fi[j] = ni[j];
        }
    }
    cp_async_wait_all();
    pdl_trigger();
}

// Deterministic gridding sum: every grid cell g = (gx, gy) is the sum of the
// stored run patches covering it (the runs with first-tap cell
// (gx - a, gy - b), periodic, at tap (b, a)), written over the previous
// contents, in a fixed order: per tap row b, the first run of each tap
// column a = 0..J-1 (their index and patch loads all in flight at once),
// then the further runs of each column in increasing run order.
template <int J>
__global__ void __launch_bounds__(256)
k_lane_gather(const float2* __restrict__ P, int64_t dstride, const int* __restrict__ cstart,
              const int* __restrict__ clist, int Kx, int Ky, float2* __restrict__ out, const int* __restrict__ skip) {
    pdl_wait();
    if (skip && *skip) return;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < (int64_t)Kx * Ky) {
        const int gx = (int)(g & (Kx - 1)), gy = (int)(g / Kx);
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int b = 0; b < J; ++b) {
            const int* rowc = cstart + (size_t)((gy - b) & (Ky - 1)) * Kx;
            const float2* Pb = P + (size_t)(b * J) * dstride;
            int s[J], e[J];
#pragma unroll
            for (int a = 0; a < J; ++a) {
                const int c = (gx - a) & (Kx - 1);
                s[a] = __ldg(rowc + c);
                e[a] = __ldg(rowc + c + 1);
            }
            int q0[J];
#pragma unroll
            for (int a = 0; a < J; ++a) q0[a] = s[a] < e[a] ? __ldg(clist + s[a]) : -1;
            float2 v[J];
#pragma unroll
            for (int a = 0; a < J; ++a)
                v[a] = q0[a] >= 0 ? __ldg(Pb + (size_t)a * dstride + q0[a]) : make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < J; ++a) {
                sr += v[a].x;
                si += v[a].y;
            }
#pragma unroll
            for (int a = 0; a < J; ++a) {
                for (int q = s[a] + 1; q < e[a]; ++q) {
                    const float2 w = __ldg(Pb + (size_t)a * dstride + __ldg(clist + q));
                    sr += w.x;
                    si += w.y;
                }
            }
        }
        out[g] = make_float2(sr, si);
    }
    pdl_trigger();
}

// G with the tile staged in shared memory: a block owns one subproblem,
// copies the tile plus its (J-1) halo from the grid, then every thread
// interpolates visibilities of the subproblem from the shared copy.
template <typename T, int J>
__global__ void __launch_bounds__(128)
k_degrid_tile(const typename cplx_of<T>::type* __restrict__ grid, const T* __restrict__ us, const T* __restrict__ vs,
              AxisConst ax, AxisConst ay, KbPoly kp, double beta, double inv_i0beta, const int* __restrict__ perm,
              const int* __restrict__ sub_bin, const int* __restrict__ sub_off, const int* __restrict__ list,
              int tile, int tiles_x, typename cplx_of<T>::type* __restrict__ y, const int* __restrict__ skip) {
    pdl_wait();
    using C = typename cplx_of<T>::type;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int PT = tile + J - 1;
    C* tl = reinterpret_cast<C*>(smem_raw);                   // [PT][PT]
    const int s = blockIdx.x;
    const int bin = sub_bin[s];
    const int oy = (bin / tiles_x) * tile, ox = (bin % tiles_x) * tile;
    const int Kx = ax.K, Ky = ay.K;
    for (int t = threadIdx.x; t < PT * PT; t += blockDim.x) {
        const int r = t / PT, c = t - r * PT;
        tl[t] = grid[(size_t)((oy + r) & (Ky - 1)) * Kx + ((ox + c) & (Kx - 1))];
    }
    __syncthreads();
    const int q0 = sub_off[s], total = sub_off[s + 1] - q0;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int m = list[q0 + q];
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
    pdl_trigger();
}

// ------------------------------------------------------------- launchers
template <typename K> static void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) PURIFY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// Resident blocks per SM of a persistent kernel on the current device,
// worked out (with its shared-memory limit raised) on the first launch on
// each device; `cache` is the caller's per-instantiation table, indexed by
// device, 0 while unknown. Threads racing on a first launch store the same
// value.
template <typename K>
static int blocks_per_sm(std::atomic<int> (&cache)[64], K kernel, int threads, size_t smem) {
    int dev = 0;
    PURIFY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{PURIFY_ECUDA, "device index out of range"};
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        set_smem(kernel, smem);
        PURIFY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, smem));
        v = std::max(1, v);
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}


template <typename T, int J> static void degrid_tj(purify_plan* p, void* y, bool caller_order, const int* skip) {
    using C = typename cplx_of<T>::type;
    const GridWork& w = p->dwork;
    if (w.nsub == 0) return;
    const int tile = w.tile, PT = tile + J - 1;
    size_t sm = sizeof(C) * (size_t)PT * PT;
    set_smem(k_degrid_tile<T, J>, sm);
    Launch L(p, "degrid");
    launch_dependent(k_degrid_tile<T, J>, w.nsub, 128, sm, p->stream, 
        p->grid.as<C>(), p->us.as<T>(), p->vs.as<T>(), p->ax, p->ay, p->kbp, p->beta, 1.0 / p->i0beta,
        caller_order ? p->perm.as<int>() : nullptr, w.sub_bin.as<int>(), w.sub_off.as<int>(), w.list.as<int>(),
        tile, w.tiles_x, (C*)y, skip);
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
static void grid_tj(purify_plan* p, const void* y, bool caller_order, const int* skip, bool zeroed) {
    using C = typename cplx_of<T>::type;
    constexpr int W = grid_warps<T>();
    if (!zeroed) PURIFY_CUDA(cudaMemsetAsync(p->gacc.p, 0, p->gacc.bytes, p->stream));
    if (p->work.nsub == 0) return;
    const int tile = p->work.tile;
    const int S = grid_row_stride(tile, J);
    size_t sm = grid_smem_bytes<T, J>(tile);
    set_smem(k_grid_runs<T, J, W>, sm);
    Launch L(p, "grid");
    launch_dependent(k_grid_runs<T, J, W>, p->work.nsub, W * 32, sm, p->stream, 
        (const C*)y, p->us.as<T>(), p->vs.as<T>(), p->ax, p->ay, p->kbp, p->beta, 1.0 / p->i0beta,
        caller_order ? p->perm.as<int>() : nullptr, p->work.sub_bin.as<int>(), p->work.sub_off.as<int>(),
        p->work.list.as<int>(), tile, p->work.tiles_x, S, p->gacc.as<C>(), skip);
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
template <int J> static void grid_f(purify_plan* p, const void* y, bool c, const int* s, bool z) { grid_tj<float, J>(p, y, c, s, z); }
template <int J> static void grid_d(purify_plan* p, const void* y, bool c, const int* s, bool z) { grid_tj<double, J>(p, y, c, s, z); }


// Run-set launches: a persistent grid of 8-warp blocks (as many as are
// resident at once, or fewer when there is less work).
template <typename T, int J, bool FUSED>
static void grid_sets_tj(purify_plan* p, const void* y, bool caller_order, const int* skip, bool zeroed = false) {
    using C = typename cplx_of<T>::type;
    constexpr int W = 8;
    if (!zeroed) PURIFY_CUDA(cudaMemsetAsync(p->gacc.p, 0, p->gacc.bytes, p->stream));
    const RunWork& rw = p->runs;
    if (rw.nsets == 0) return;
    static std::atomic<int> occ[64];   // resident blocks per SM of this instantiation, per device
    const int per_sm = blocks_per_sm(occ, k_grid_sets<T, J, W, FUSED>, W * 32, 0);
    int sms = 0, dev = 0;
    PURIFY_CUDA(cudaGetDevice(&dev));
    PURIFY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = std::max(1, std::min(sms * per_sm, (rw.nsets + W - 1) / W));
    Launch L(p, FUSED ? "normal_gg" : "grid");
    launch_dependent(k_grid_sets<T, J, W, FUSED>, blocks, W * 32, 0, p->stream,
        (const C*)y, p->grid.as<C>(), rw.rec.as<typename RunRecOf<T>::type>(), rw.cell.as<int>(),
        rw.start.as<int>(), rw.len.as<int>(), rw.nsets, caller_order ? p->perm.as<int>() : nullptr, p->kbp,
        p->beta, 1.0 / p->i0beta, p->Kx, p->Ky, p->gacc.as<C>(), skip);
    L.done();
}
// Lane-per-run launches (kind 3: one lane per run, 4: two lanes per run,
// 5: two lanes per run with the sets grouped by grid tile): a persistent
// grid of 4-warp blocks (as many as are resident at once, or fewer when
// there is less work).
static const LaneWork& lane_work(const purify_plan* p, int kind) { return p->lanes[kind == 6 ? 1 : kind - 3]; }
template <int J, int MODE, int H, bool DET>
static void lane_launch(purify_plan* p, const LaneWork& lw, const void* yin, void* yout, bool caller_order,
                        const int* skip, float2* out, int64_t dstride) {
    const size_t lane_smem = 4 * LaneStage<J, H>::bytes_per_warp;
    static std::atomic<int> occ[64];   // resident blocks per SM of this instantiation, per device
    const int per_sm = blocks_per_sm(occ, k_lane<J, MODE, H, DET>, 128, lane_smem);
    int sms = 0, dev = 0;
    PURIFY_CUDA(cudaGetDevice(&dev));
    PURIFY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = std::max(1, std::min(sms * per_sm, (lw.nsets + 3) / 4));
    Launch L(p, MODE == LANE_GG ? "normal_gg" : (MODE == LANE_GRID ? "grid" : "degrid"));
    launch_dependent(k_lane<J, MODE, H, DET>, blocks, 128, lane_smem, p->stream, p->grid.as<float2>(),
                     (const float2*)yin, (float2*)yout, lw.set_info.as<int2>(), lw.run_cl.as<int2>(),
                     lw.rec.as<float2>(), caller_order ? lw.idx_caller.as<int>() : lw.idx.as<int>(), lw.nsets,
                     p->kbp, p->Kx, p->Ky, out, skip, dstride);
    L.done();
}
template <int J, int MODE, int H>
static void lane_tw(purify_plan* p, const LaneWork& lw, const void* yin, void* yout, bool caller_order,
                    const int* skip, bool zeroed) {
    if constexpr (H == 2 && MODE != LANE_DEGRID) {
        if (lw.deterministic() && lw.nsets > 0) {
            // run patches stored, then summed per cell in a fixed order
            // (the sum overwrites the accumulator: no clearing needed)
            const int64_t stride = (int64_t)lw.nsets * lw.width;
            PURIFY_REQUIRE(p->det_patch.bytes >= sizeof(float2) * (size_t)J * J * (size_t)stride,
                           "deterministic patch buffer too small");
            lane_launch<J, MODE, H, true>(p, lw, yin, yout, caller_order, skip, p->det_patch.as<float2>(), stride);
            const int64_t cells = (int64_t)p->Kx * p->Ky;
            Launch L(p, "det_gather");
            launch_dependent(k_lane_gather<J>, (unsigned)((cells + 255) / 256), 256, 0, p->stream,
                             (const float2*)p->det_patch.as<float2>(), stride, lw.cstart.as<int>(),
                             lw.clist.as<int>(), p->Kx, p->Ky, p->gacc.as<float2>(), skip);
            L.done();
            return;
        }
    }
    if (MODE != LANE_DEGRID && !zeroed) PURIFY_CUDA(cudaMemsetAsync(p->gacc.p, 0, p->gacc.bytes, p->stream));
    if (lw.nsets == 0) return;
    lane_launch<J, MODE, H, false>(p, lw, yin, yout, caller_order, skip, p->gacc.as<float2>(), 0);
}
template <int J, int MODE>
static void lane_on(purify_plan* p, const LaneWork& lw, const void* yin, void* yout, bool c, const int* s, bool z) {
    if constexpr (J <= kLaneMaxJ) {
        if (lw.width == 32) lane_tw<J, MODE, 1>(p, lw, yin, yout, c, s, z);
        else lane_tw<J, MODE, 2>(p, lw, yin, yout, c, s, z);
    }
}
template <int J, int MODE>
static void lane_any(purify_plan* p, int kind, const void* yin, void* yout, bool c, const int* s, bool z) {
    lane_on<J, MODE>(p, lane_work(p, kind), yin, yout, c, s, z);
}
template <int J>
static void lane_mode(purify_plan* p, const LaneWork& lw, int mode, const void* yin, void* yout, bool c, const int* s,
                      bool z) {
    if (mode == LANE_GG) lane_on<J, LANE_GG>(p, lw, nullptr, nullptr, false, s, z);
    else if (mode == LANE_GRID) lane_on<J, LANE_GRID>(p, lw, yin, nullptr, c, s, z);
    else lane_on<J, LANE_DEGRID>(p, lw, nullptr, yout, c, s, true);
}
template <int J> static void lane_gg(purify_plan* p, int kind, const int* s, bool z) {
    lane_any<J, LANE_GG>(p, kind, nullptr, nullptr, false, s, z);
}
template <int J> static void lane_grid(purify_plan* p, int kind, const void* y, bool c, const int* s, bool z) {
    lane_any<J, LANE_GRID>(p, kind, y, nullptr, c, s, z);
}
template <int J> static void lane_degrid(purify_plan* p, int kind, void* y, bool c, const int* s) {
    lane_any<J, LANE_DEGRID>(p, kind, nullptr, y, c, s, true);
}

template <int J> static void normal_f(purify_plan* p, const int* s, bool z) { grid_sets_tj<float, J, true>(p, nullptr, false, s, z); }
template <int J> static void normal_d(purify_plan* p, const int* s, bool z) { grid_sets_tj<double, J, true>(p, nullptr, false, s, z); }
template <int J> static void gsets_f(purify_plan* p, const void* y, bool c, const int* s, bool z) { grid_sets_tj<float, J, false>(p, y, c, s, z); }
template <int J> static void gsets_d(purify_plan* p, const void* y, bool c, const int* s, bool z) { grid_sets_tj<double, J, false>(p, y, c, s, z); }

bool lane_work_ok(const purify_plan* p) { return p->dtype == PURIFY_F32 && p->J <= kLaneMaxJ; }
static void require_lane_work(const purify_plan* p, int kind) {
    if (!lane_work_ok(p) || kind < 3 || kind > 6 || lane_work(p, kind).nsets == 0 ||
        (kind == 6 && !lane_work(p, kind).deterministic()))
        throw Error{PURIFY_EINVAL, "lane-per-run kernels need an FP32 plan with J <= 6 built for that form"};
}

void launch_normal_gg(purify_plan* p, const int* skip, bool zeroed) {
    if (p->normal_kind >= 3 && lane_work_ok(p)) { PURIFY_J_DISPATCH(p->J, lane_gg, p, p->normal_kind, skip, zeroed); }
    else if (p->dtype == PURIFY_F32) { PURIFY_J_DISPATCH(p->J, normal_f, p, skip, zeroed); }
    else { PURIFY_J_DISPATCH(p->J, normal_d, p, skip, zeroed); }
}
void launch_grid_lanes(purify_plan* p, int kind, const void* y, bool caller_order, const int* skip, bool zeroed) {
    require_lane_work(p, kind);
    PURIFY_J_DISPATCH(p->J, lane_grid, p, kind, y, caller_order, skip, zeroed);
}
void launch_degrid_lanes(purify_plan* p, int kind, void* y, bool caller_order, const int* skip) {
    require_lane_work(p, kind);
    PURIFY_J_DISPATCH(p->J, lane_degrid, p, kind, y, caller_order, skip);
}
void launch_lanes_on(purify_plan* p, const LaneWork& lw, int mode, const void* yin, void* yout, bool caller_order,
                     const int* skip, bool zeroed) {
    if (!lane_work_ok(p) || lw.nsets == 0 || (lw.width != 32 && lw.width != 16))
        throw Error{PURIFY_EINVAL, "lane-per-run kernels need an FP32 plan with J <= 6"};
    PURIFY_J_DISPATCH(p->J, lane_mode, p, lw, mode, yin, yout, caller_order, skip, zeroed);
}
void launch_normal_lanes(purify_plan* p, int kind, const int* skip, bool zeroed) {
    if (kind == 2 || !lane_work_ok(p)) {
        if (p->dtype == PURIFY_F32) { PURIFY_J_DISPATCH(p->J, normal_f, p, skip, zeroed); }
        else { PURIFY_J_DISPATCH(p->J, normal_d, p, skip, zeroed); }
        return;
    }
    require_lane_work(p, kind);
    PURIFY_J_DISPATCH(p->J, lane_gg, p, kind, skip, zeroed);
}
void launch_grid_sets(purify_plan* p, const void* y, bool caller_order, const int* skip, bool zeroed) {
    if (p->dtype == PURIFY_F32) { PURIFY_J_DISPATCH(p->J, gsets_f, p, y, caller_order, skip, zeroed); }
    else { PURIFY_J_DISPATCH(p->J, gsets_d, p, y, caller_order, skip, zeroed); }
}

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

void launch_degrid(purify_plan* p, void* y, bool caller_order, const int* skip) {
    if (p->degrid_kind >= 3) {
        launch_degrid_lanes(p, p->degrid_kind, y, caller_order, skip);
        return;
    }
    if (p->dtype == PURIFY_F32) { PURIFY_J_DISPATCH(p->J, degrid_f, p, y, caller_order, skip); }
    else { PURIFY_J_DISPATCH(p->J, degrid_d, p, y, caller_order, skip); }
}
void launch_grid(purify_plan* p, const void* y, bool caller_order, const int* skip, bool zeroed) {
    if (p->grid_kind == 2) {
        launch_grid_sets(p, y, caller_order, skip, zeroed);
        return;
    }
    if (p->grid_kind >= 3) {
        launch_grid_lanes(p, p->grid_kind, y, caller_order, skip, zeroed);
        return;
    }
    if (p->dtype == PURIFY_F32) { PURIFY_J_DISPATCH(p->J, grid_f, p, y, caller_order, skip, zeroed); }
    else { PURIFY_J_DISPATCH(p->J, grid_d, p, y, caller_order, skip, zeroed); }
}

void launch_phi(purify_plan* p, const void* x, void* y, bool caller_order, double scale, bool zero_acc) {
    launch_scale_pad_rows(p, x, scale, nullptr, true, zero_acc);
    launch_cols_fwd(p, nullptr);
    launch_degrid(p, y, caller_order, nullptr);
}

void launch_phi_adj(purify_plan* p, const void* y, void* out, bool caller_order, double scale, int out_mode,
                    const void* add, bool acc_zeroed) {
    launch_grid(p, y, caller_order, nullptr, acc_zeroed);
    launch_cols_inv(p, nullptr);
    launch_rows_inv_crop(p, out, scale, out_mode, add, 1.0, nullptr);
}

}  // namespace purify
