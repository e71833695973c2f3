// SARA dictionary: Psi^dagger (analysis) and Psi (synthesis).
//
// Sec. 1 of the paper builds Psi = [Psi_1, ..., Psi_q] from q coherent
// bases. The plan uses the Dirac basis plus Daubechies db1..db8 (selected by
// the basis mask), each an orthonormal periodic 2-D Mallat transform with L
// levels, scaled by 1/sqrt(q) so that Psi Psi^dagger = I.
//
// One analysis level maps an h x w low-pass band to four h/2 x w/2 sub-bands
//   a[k] = sum_n h[n] x[(2k + n) mod len],  d[k] = sum_n g[n] x[(2k + n) mod len]
// applied along rows, then along columns. A thread block owns a TH x TW tile
// of every sub-band: it stages the (2TH + L - 2) x (2TW + L - 2) input tile
// (indices wrapped as often as needed) in shared memory, filters the rows,
// then the columns. All wavelet bases of a level run in one launch
// (blockIdx.z); level 1 also writes the Dirac plane.
//
// Synthesis is the transpose: out[m] = sum over n of parity m of
//   h[n] a[k] + g[n] d[k], k = ((m - n) mod len) / 2,
// columns first, then rows. The finest level sums all bases and the Dirac
// plane in one block per output tile, so the image is written once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "host_tables.h"
#include "launch.h"

namespace purify {

// Daubechies filters are the same for every plan: one constant-memory bank
// per precision, written once per device (init_filter_banks).
__constant__ FilterBank<float> c_bank_f;
__constant__ FilterBank<double> c_bank_d;
template <typename T> __device__ __forceinline__ const FilterBank<T>& fbank();
template <> __device__ __forceinline__ const FilterBank<float>& fbank<float>() { return c_bank_f; }
template <> __device__ __forceinline__ const FilterBank<double>& fbank<double>() { return c_bank_d; }

// Tile geometry (compile time): analysis blocks own a DWT_T x DWT_T tile of
// every sub-band; synthesis blocks own an (2 SYN_T) x (2 SYN_T) output tile.
// Band sizes are powers of two, so periodic wrapping is a mask.
static constexpr int DWT_T = 16;
static constexpr int SYN_T = 8;
static constexpr int SYN_GROUP = 64;   // threads per basis in a synthesis block

// The filter taps of basis pb in registers (unused entries are zero).
template <typename T, int L> struct Taps {
    T h[L], g[L];
    __device__ __forceinline__ void load(int pb) {
        const FilterBank<T>& fb = fbank<T>();
#pragma unroll
        for (int n = 0; n < L; ++n) { h[n] = fb.h[pb][n]; g[n] = fb.g[pb][n]; }
    }
};

// Runs STMT with the compile-time constant L equal to the filter length LEN
// (2, 4, ..., 16).
#define PURIFY_WITH_LENGTH(LEN, STMT)                                  \
    switch (LEN) {                                                     \
        case 2: { constexpr int L = 2; STMT; } break;                  \
        case 4: { constexpr int L = 4; STMT; } break;                  \
        case 6: { constexpr int L = 6; STMT; } break;                  \
        case 8: { constexpr int L = 8; STMT; } break;                  \
        case 10: { constexpr int L = 10; STMT; } break;                \
        case 12: { constexpr int L = 12; STMT; } break;                \
        case 14: { constexpr int L = 14; STMT; } break;                \
        default: { constexpr int L = 16; STMT; } break;                \
    }

// ------------------------------------------------------------- analysis
// One analysis level of basis pb on the sub-band tile at (ky0, kx0).
template <typename T, int L>
__device__ __forceinline__ void dwt_tile(const T* __restrict__ in, int src_ld, T* __restrict__ out, int nx,
                                         T* __restrict__ llo, int h, int w, int ky0, int kx0, int pb, T inv_sqrt_q,
                                         T* smem) {
    constexpr int RS = 2 * DWT_T + L - 2, CS = 2 * DWT_T + L - 2;
    Taps<T, L> f;
    f.load(pb);
    const int hs = h >> 1, wsub = w >> 1;
    const int th = min(DWT_T, hs - ky0), tw = min(DWT_T, wsub - kx0);
    const int Rin = 2 * th + L - 2, Cin = 2 * tw + L - 2;
    T* tin = smem;                 // [RS][CS]
    T* ta = tin + RS * CS;         // [RS][DWT_T] row low-pass
    T* td = ta + RS * DWT_T;       // [RS][DWT_T] row high-pass
    for (int t = threadIdx.x; t < Rin * CS; t += blockDim.x) {
        const int r = t / CS, c = t - r * CS;
        if (c < Cin) tin[t] = in[(size_t)((2 * ky0 + r) & (h - 1)) * src_ld + ((2 * kx0 + c) & (w - 1))];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Rin * DWT_T; t += blockDim.x) {
        const int r = t / DWT_T, k = t - r * DWT_T;
        if (k < tw) {
            const T* row = tin + r * CS + 2 * k;
            T a = 0, d = 0;
#pragma unroll
            for (int n = 0; n < L; ++n) { a += f.h[n] * row[n]; d += f.g[n] * row[n]; }
            ta[t] = a;
            td[t] = d;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < DWT_T * DWT_T; t += blockDim.x) {
        const int ky = t / DWT_T, kx = t - ky * DWT_T;
        if (ky >= th || kx >= tw) continue;
        T ll = 0, lh = 0, hl = 0, hh = 0;
#pragma unroll
        for (int n = 0; n < L; ++n) {
            const T av = ta[(2 * ky + n) * DWT_T + kx], dv = td[(2 * ky + n) * DWT_T + kx];
            ll += f.h[n] * av; lh += f.g[n] * av;
            hl += f.h[n] * dv; hh += f.g[n] * dv;
        }
        const int gy = ky0 + ky, gx = kx0 + kx;
        if (llo) llo[(size_t)gy * wsub + gx] = ll;
        else out[(size_t)gy * nx + gx] = ll * inv_sqrt_q;
        out[(size_t)gy * nx + wsub + gx] = hl * inv_sqrt_q;
        out[(size_t)(hs + gy) * nx + gx] = lh * inv_sqrt_q;
        out[(size_t)(hs + gy) * nx + wsub + gx] = hh * inv_sqrt_q;
    }
}

// One analysis level for every wavelet basis (blockIdx.z < nw) and, at the
// first level, the Dirac plane (blockIdx.z == nw, a 2TH x 2TW image tile).
template <typename T>
__global__ void k_dwt_level(const T* __restrict__ src, int src_basis_stride, int src_ld,
                            T* __restrict__ coef, const int* __restrict__ planes, int N, int nx,
                            T* __restrict__ ll_out, int ll_basis_stride, int h, int w, int TH, int TW,
                            const int* __restrict__ pids, int nw, int dirac_plane, T inv_sqrt_q) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int z = blockIdx.z;
    if (z == nw) {
        // Dirac plane: coef[dirac] = x / sqrt(q) over a 2TH x 2TW image tile
        const int r0 = blockIdx.y * 2 * TH, c0 = blockIdx.x * 2 * TW;
        for (int t = threadIdx.x; t < 4 * TH * TW; t += blockDim.x) {
            int r = r0 + t / (2 * TW), c = c0 + t % (2 * TW);
            if (r < h && c < w) coef[(size_t)dirac_plane * N + (size_t)r * nx + c] = src[(size_t)r * src_ld + c] * inv_sqrt_q;
        }
        return;
    }
    const int pb = pids[z];              // db index 1..8
    const T* in = src + (size_t)z * src_basis_stride;
    T* out = coef + (size_t)planes[z] * N;
    T* llo = ll_out ? ll_out + (size_t)z * ll_basis_stride : nullptr;
    const int ky0 = blockIdx.y * DWT_T, kx0 = blockIdx.x * DWT_T;
    T* smem = reinterpret_cast<T*>(smem_raw);
    PURIFY_WITH_LENGTH(fbank<T>().len[pb],
                       (dwt_tile<T, L>(in, src_ld, out, nx, llo, h, w, ky0, kx0, pb, inv_sqrt_q, smem)));
    pdl_trigger();
}

// Shared memory of one analysis block (filters up to maxL taps).
static size_t dwt_smem_bytes(int maxL, size_t tbytes) {
    const size_t RS = 2 * DWT_T + maxL - 2;
    return tbytes * (RS * RS + 2 * RS * DWT_T);
}

// ------------------------------------------------------------ synthesis
// Reconstruct the th2 x tw2 output tile at (oy0, ox0) of an h x w band for
// basis pb from its four sub-bands, by the thread group (gt of gn threads).
// `ll` points at the low-pass sub-band (row stride ll_ld); the three detail
// sub-bands are read from `det` (the basis' coefficient plane, row stride
// nx). Output t = gt + i * gn of the tile (row-major, stride tw2) is added to
// acc[i].
template <typename T, int L, int PER>
__device__ __forceinline__ void synth_tile(const T* __restrict__ ll, int ll_ld, const T* __restrict__ det, int nx,
                                           int h, int w, int oy0, int ox0, int th2, int tw2, int pb, T* smem, int gt,
                                           int gn, T (&acc)[PER]) {
    constexpr int KS = SYN_T + L / 2;            // sub-band tile stride (rows and columns)
    Taps<T, L> f;
    f.load(pb);
    const int hs = h >> 1, wsub = w >> 1;
    const int Kr = th2 / 2 + L / 2, Kc = tw2 / 2 + L / 2;
    const int ky_lo = oy0 / 2 - L / 2, kx_lo = ox0 / 2 - L / 2;
    T* sLL = smem;
    T* sHL = sLL + KS * KS;   // row-detail, column-approx: (ky, wsub + kx)
    T* sLH = sHL + KS * KS;   // row-approx, column-detail: (hs + ky, kx)
    T* sHH = sLH + KS * KS;
    T* sA = sHH + KS * KS;    // [2 SYN_T][KS]: column synthesis of the row-approx half
    T* sD = sA + 2 * SYN_T * KS;
    for (int t = gt; t < Kr * KS; t += gn) {
        const int r = t / KS, c = t - r * KS;
        if (c >= Kc) continue;
        const int ky = (ky_lo + r) & (hs - 1), kx = (kx_lo + c) & (wsub - 1);
        sLL[t] = ll[(size_t)ky * ll_ld + kx];
        sHL[t] = det[(size_t)ky * nx + wsub + kx];
        sLH[t] = det[(size_t)(hs + ky) * nx + kx];
        sHH[t] = det[(size_t)(hs + ky) * nx + wsub + kx];
    }
    __syncthreads();
    for (int t = gt; t < th2 * KS; t += gn) {
        const int mr = t / KS, c = t - mr * KS;
        if (c >= Kc) continue;
        // output row m = oy0 + mr takes the taps n of its parity; sub-band
        // row (m - n) / 2 - ky_lo = (mr - par) / 2 + L / 2 - j for n = 2 j + par
        const int par = mr & 1;
        const int r0 = ((mr - par) >> 1) + L / 2;
        T a = 0, d = 0;
#pragma unroll
        for (int j = 0; j < L / 2; ++j) {
            const T hn = par ? f.h[2 * j + 1] : f.h[2 * j], gn_ = par ? f.g[2 * j + 1] : f.g[2 * j];
            const int r = r0 - j;
            a += hn * sLL[r * KS + c] + gn_ * sLH[r * KS + c];
            d += hn * sHL[r * KS + c] + gn_ * sHH[r * KS + c];
        }
        sA[t] = a;
        sD[t] = d;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int t = gt + i * gn;
        if (t < th2 * tw2) {
            const int mr = t / tw2, mc = t - mr * tw2;
            const int par = mc & 1;
            const int c0 = ((mc - par) >> 1) + L / 2;
            T sacc = 0;
#pragma unroll
            for (int j = 0; j < L / 2; ++j) {
                const T hn = par ? f.h[2 * j + 1] : f.h[2 * j], gn_ = par ? f.g[2 * j + 1] : f.g[2 * j];
                const int c = c0 - j;
                sacc += hn * sA[mr * KS + c] + gn_ * sD[mr * KS + c];
            }
            acc[i] += sacc;
        }
    }
    __syncthreads();
}

// Shared memory of one synthesis tile (filters up to maxL taps).
static size_t synth_smem_elems(int maxL) {
    const size_t KS = SYN_T + maxL / 2;
    return 4 * KS * KS + 2 * (2 * SYN_T) * KS;
}

// One synthesis level for every wavelet basis (blockIdx.z), SYN_LEVEL_THREADS
// threads per block: writes the reconstructed h x w band of basis z into
// ll_out (row stride w).
static constexpr int SYN_LEVEL_THREADS = 128;
template <typename T>
__global__ void __launch_bounds__(SYN_LEVEL_THREADS)
k_idwt_level(const T* __restrict__ ll_in, int ll_basis_stride, int ll_ld, const T* __restrict__ coef,
             const int* __restrict__ planes, int N, int nx, T* __restrict__ ll_out, int out_basis_stride, int h,
             int w, const int* __restrict__ pids) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int PER = (4 * SYN_T * SYN_T + SYN_LEVEL_THREADS - 1) / SYN_LEVEL_THREADS;
    const int z = blockIdx.z;
    const int pb = pids[z];
    const int oy0 = blockIdx.y * 2 * SYN_T, ox0 = blockIdx.x * 2 * SYN_T;
    const int th2 = min(2 * SYN_T, h - oy0), tw2 = min(2 * SYN_T, w - ox0);
    const T* det = coef + (size_t)planes[z] * N;
    const T* ll = ll_in ? ll_in + (size_t)z * ll_basis_stride : det;
    const int ld = ll_in ? ll_ld : nx;
    T acc[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i] = 0;
    T* smem = reinterpret_cast<T*>(smem_raw);
    PURIFY_WITH_LENGTH(fbank<T>().len[pb],
                       (synth_tile<T, L, PER>(ll, ld, det, nx, h, w, oy0, ox0, th2, tw2, pb, smem,
                                              (int)threadIdx.x, SYN_LEVEL_THREADS, acc)));
    T* out = ll_out + (size_t)z * out_basis_stride;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int t = threadIdx.x + i * SYN_LEVEL_THREADS;
        if (t < th2 * tw2) {
            const int mr = t / tw2, mc = t - mr * tw2;
            out[(size_t)(oy0 + mr) * w + ox0 + mc] = acc[i];
        }
    }
    pdl_trigger();
}

// Finest synthesis level summed over all wavelet bases plus the Dirac plane:
// x = (c_dirac + sum_z W_z^T c_z) / sqrt(q). Thread group z (SYN_GROUP
// threads) synthesises basis z's contribution to the block's output tile;
// the partial tiles are then added in basis order. When `ll_in` is null
// (L == 1) the low-pass bands come from the coefficient planes.
// Every group runs the same code: filters zero-padded to the plan's longest
// length L (the padded taps add exact zeros), so the block has one instruction
// stream and one barrier sequence whatever the bases.
template <typename T, int L>
__global__ void __launch_bounds__(512, 2)
k_idwt_final(const T* __restrict__ ll_in, int ll_basis_stride, const T* __restrict__ coef,
                             const int* __restrict__ planes, int N, int nx, int ny, int group_elems,
                             const int* __restrict__ pids, int nw, int dirac_plane,
                             T inv_sqrt_q, T* __restrict__ x) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int PER = (4 * SYN_T * SYN_T + SYN_GROUP - 1) / SYN_GROUP;
    const int oy0 = blockIdx.y * 2 * SYN_T, ox0 = blockIdx.x * 2 * SYN_T;
    const int th2 = min(2 * SYN_T, ny - oy0), tw2 = min(2 * SYN_T, nx - ox0);
    const int z = threadIdx.x / SYN_GROUP, gt = threadIdx.x - z * SYN_GROUP;
    const size_t per_group = (size_t)group_elems;   // shared elements of one group's tile
    T* part = reinterpret_cast<T*>(smem_raw);                       // [nw][4 SYN_T^2] partial tiles
    T* gsm = part + (size_t)nw * 4 * SYN_T * SYN_T + (size_t)z * per_group;
    T acc[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i] = 0;
    if (z < nw) {
        const int pb = pids[z];
        const T* det = coef + (size_t)planes[z] * N;
        const T* ll = ll_in ? ll_in + (size_t)z * ll_basis_stride : det;
        const int ld = ll_in ? (nx >> 1) : nx;
        synth_tile<T, L, PER>(ll, ld, det, nx, ny, nx, oy0, ox0, th2, tw2, pb, gsm, gt, SYN_GROUP, acc);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int t = gt + i * SYN_GROUP;
            if (t < 4 * SYN_T * SYN_T) part[(size_t)z * 4 * SYN_T * SYN_T + t] = acc[i];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < th2 * tw2; t += blockDim.x) {
        const int mr = t / tw2, mc = t - mr * tw2;
        T v = 0;
        for (int zz = 0; zz < nw; ++zz) v += part[(size_t)zz * 4 * SYN_T * SYN_T + t];
        const size_t idx = (size_t)(oy0 + mr) * nx + ox0 + mc;
        if (dirac_plane >= 0) v += coef[(size_t)dirac_plane * N + idx];
        x[idx] = v * inv_sqrt_q;
    }
    pdl_trigger();
}

// ------------------------------------------------------------- launchers
struct WaveletLayout {
    int nw = 0;            // wavelet bases
    int dirac_plane = -1;  // coefficient plane of the Dirac basis, or -1
};

static WaveletLayout layout(const purify_plan* p) {
    WaveletLayout l;
    for (size_t i = 0; i < p->bases.size(); ++i) {
        if (p->bases[i] == 0) l.dirac_plane = (int)i;
        else l.nw++;
    }
    return l;
}

// Device int meta array of a plan: pids[0..8) = db index of each wavelet
// basis, planes[8..16) = its coefficient plane.
static const int* pid_array(const purify_plan* p) { return p->wmeta.as<int>(); }
static const int* plane_array(const purify_plan* p) { return p->wmeta.as<int>() + 8; }

static bool g_bank_ready[64];
static std::mutex g_bank_mutex;

void init_filter_banks() {
    int dev = 0;
    PURIFY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{PURIFY_ECUDA, "device index out of range"};
    // one upload per device, also when several host threads make their first call at once
    std::lock_guard<std::mutex> lock(g_bank_mutex);
    if (g_bank_ready[dev]) return;
    FilterBank<float> bf;
    FilterBank<double> bd;
    std::memset(&bf, 0, sizeof(bf));
    std::memset(&bd, 0, sizeof(bd));
    bf.len[0] = bd.len[0] = 0;
    for (int p = 1; p <= 8; ++p) {
        std::vector<double> h = daubechies(p);
        int L = (int)h.size();
        bf.len[p] = bd.len[p] = L;
        for (int n = 0; n < L; ++n) {
            double g = ((n & 1) ? -1.0 : 1.0) * h[L - 1 - n];
            bd.h[p][n] = h[n];
            bd.g[p][n] = g;
            bf.h[p][n] = (float)h[n];
            bf.g[p][n] = (float)g;
        }
    }
    PURIFY_CUDA(cudaMemcpyToSymbol(c_bank_f, &bf, sizeof(bf)));
    PURIFY_CUDA(cudaMemcpyToSymbol(c_bank_d, &bd, sizeof(bd)));
    g_bank_ready[dev] = true;
}

template <typename T> static void psi_adj_t(purify_plan* p, const void* xv, void* cv) {
    const T* x = (const T*)xv;
    T* c = (T*)cv;
    WaveletLayout wl = layout(p);
    const T inv_sqrt_q = (T)(1.0 / std::sqrt((double)p->q));
    const int N = (int)p->N;
    if (wl.nw == 0) {
        // Dirac only
        Launch Lc(p, "dwt_level");
        dim3 g((p->nx + 31) / 32, (p->ny + 31) / 32, 1);
        launch_dependent(k_dwt_level<T>, g, 256, 0, p->stream, x, 0, p->nx, c, plane_array(p), N, p->nx, nullptr, 0, p->ny,
                                                 p->nx, 16, 16, pid_array(p), 0, wl.dirac_plane, inv_sqrt_q);
        Lc.done();
        return;
    }
    int h = p->ny, w = p->nx;
    const T* src = x;
    int src_stride = 0, src_ld = p->nx;
    T* bufs[2] = {p->ll0.as<T>(), p->ll1.as<T>()};
    const int llstride = (int)(p->N / 4);
    for (int lev = 0; lev < p->levels; ++lev) {
        const bool last = lev == p->levels - 1;
        const int hs = h / 2, wsub = w / 2;
        const int TH = std::min(DWT_T, hs), TW = std::min(DWT_T, wsub);
        int maxL = 2;
        for (int b : p->bases) if (b > 0) maxL = std::max(maxL, 2 * b);
        const size_t sm = dwt_smem_bytes(maxL, sizeof(T));
        int zdim = wl.nw + ((lev == 0 && wl.dirac_plane >= 0) ? 1 : 0);
        dim3 g((wsub + TW - 1) / TW, (hs + TH - 1) / TH, zdim);
        T* llo = last ? nullptr : bufs[lev & 1];
        Launch L(p, "dwt_level");
        launch_dependent(k_dwt_level<T>, g, 256, sm, p->stream, src, src_stride, src_ld, c, plane_array(p), N, p->nx, llo,
                                                  llstride, h, w, TH, TW, pid_array(p), wl.nw,
                                                  wl.dirac_plane, inv_sqrt_q);
        L.done();
        src = llo;
        src_stride = llstride;
        src_ld = wsub;
        h = hs;
        w = wsub;
    }
}

template <typename T, int L>
static void launch_idwt_final(purify_plan* p, dim3 g, int threads, size_t sm, const T* ll_in, int llstride,
                              const T* c, int N, int group_elems, const WaveletLayout& wl, T inv_sqrt_q, T* x) {
    if (sm > 48 * 1024)
        PURIFY_CUDA(cudaFuncSetAttribute(k_idwt_final<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    launch_dependent(k_idwt_final<T, L>, g, threads, sm, p->stream, ll_in, llstride, c, plane_array(p), N, p->nx,
                     p->ny, group_elems, pid_array(p), wl.nw, wl.dirac_plane, inv_sqrt_q, x);
}

template <typename T> static void psi_t(purify_plan* p, const void* cv, void* xv) {
    const T* c = (const T*)cv;
    T* x = (T*)xv;
    WaveletLayout wl = layout(p);
    const T inv_sqrt_q = (T)(1.0 / std::sqrt((double)p->q));
    const int N = (int)p->N;
    int maxL = 2;
    for (int b : p->bases) if (b > 0) maxL = std::max(maxL, 2 * b);
    T* bufs[2] = {p->ll0.as<T>(), p->ll1.as<T>()};
    const int llstride = (int)(p->N / 4);
    const T* ll_in = nullptr;  // coarsest level reads LL from the coefficients
    int ll_ld = p->nx;
    // levels L .. 2 reconstruct low-pass bands into scratch
    const size_t group_elems = synth_smem_elems(maxL);
    for (int lev = p->levels - 1; lev >= 1 && wl.nw > 0; --lev) {
        const int h = p->ny >> lev, w = p->nx >> lev;
        const size_t sm = sizeof(T) * group_elems;
        dim3 g((w + 2 * SYN_T - 1) / (2 * SYN_T), (h + 2 * SYN_T - 1) / (2 * SYN_T), wl.nw);
        T* out = bufs[lev & 1];
        if (sm > 48 * 1024) PURIFY_CUDA(cudaFuncSetAttribute(k_idwt_level<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        Launch L(p, "idwt_level");
        launch_dependent(k_idwt_level<T>, g, SYN_LEVEL_THREADS, sm, p->stream, ll_in, llstride, ll_ld, c, plane_array(p), N,
                                                                 p->nx, out, llstride, h, w, pid_array(p));
        L.done();
        ll_in = out;
        ll_ld = w;
    }
    // finest level: one thread group per basis, partial tiles summed in order
    const size_t sm = sizeof(T) * ((size_t)wl.nw * 4 * SYN_T * SYN_T + (size_t)wl.nw * group_elems);
    dim3 g((p->nx + 2 * SYN_T - 1) / (2 * SYN_T), (p->ny + 2 * SYN_T - 1) / (2 * SYN_T), 1);
    const int threads = std::max(1, wl.nw) * SYN_GROUP;
    Launch Lf(p, "idwt_final");
    PURIFY_WITH_LENGTH(maxL, (launch_idwt_final<T, L>(p, g, threads, sm, ll_in, llstride, c, N, (int)group_elems, wl,
                                                       inv_sqrt_q, x)));
    Lf.done();
}

void launch_psi_adj(purify_plan* p, const void* x, void* c) {
    if (p->dtype == PURIFY_F32) psi_adj_t<float>(p, x, c); else psi_adj_t<double>(p, x, c);
}
void launch_psi(purify_plan* p, const void* c, void* x) {
    if (p->dtype == PURIFY_F32) psi_t<float>(p, c, x); else psi_t<double>(p, c, x);
}

}  // namespace purify

// ------------------------------------------- allocation-free Psi^dagger
// A plan-free variant of the multilevel analysis for callers that must not
// allocate device memory. The low-pass ping-pong scratch of the level
// kernels lives in one file-scope device array instead of plan buffers; every
// device that loads this library holds it until the process exits.
namespace purify {

static const size_t kStaticScratchBytes = size_t(4) << 20;  // 4 MiB
// The two low-pass buffers: level 0 writes nw N / 4 values into the first,
// level 1 nw N / 16 into the second, deeper levels alternate and need less.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
// the basis table of the current mask (pids, then coefficient planes)
static __device__ __align__(16) int g_static_meta[16];

// Host code cannot use the arrays' names as device addresses: their device
// addresses are looked up once per device (with that device current).
static std::mutex g_static_mutex;
static void* g_static_addr[64];
static void* g_static_meta_addr[64];

static void* symbol_address(const void* symbol, const char* what) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, symbol);
    if (e != cudaSuccess || ptr == nullptr) {
        cudaGetLastError();
        throw Error{PURIFY_ECUDA, std::string("cudaGetSymbolAddress of the ") + what + " failed: " +
                                      cudaGetErrorString(e)};
    }
    return ptr;
}

static void static_addresses(void** scratch, int** meta) {
    int dev = 0;
    PURIFY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{PURIFY_ECUDA, "device index out of range"};
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[dev]) {
        g_static_meta_addr[dev] = symbol_address(g_static_meta, "static basis table");
        g_static_addr[dev] = symbol_address(g_static_scratch, "static scratch");
    }
    *scratch = g_static_addr[dev];
    *meta = static_cast<int*>(g_static_meta_addr[dev]);
}

// Basis table of a mask: pids[z] = db index of wavelet z, planes[z] = its
// coefficient plane (written into the static scratch by the device).
__global__ void k_static_meta(unsigned mask, int* meta) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int z = 0, plane = 0;
    for (int b = 0; b < 9; ++b) {
        if (!(mask >> b & 1)) continue;
        if (b > 0) { meta[z] = b; meta[8 + z] = plane; ++z; }
        ++plane;
    }
    for (; z < 8; ++z) { meta[z] = 0; meta[8 + z] = 0; }
}

size_t psi_adj_static_bytes(int nx, int ny, unsigned mask, int dtype) {
    int nw = 0;
    for (int b = 1; b < 9; ++b) nw += (mask >> b & 1);
    size_t rb = dtype == PURIFY_F32 ? 4 : 8;
    size_t N = (size_t)nx * ny;
    return (size_t)nw * (N / 4 + N / 16) * rb;
}

size_t psi_adj_static_capacity() { return kStaticScratchBytes; }

template <typename T>
static void psi_adj_static_t(const T* x, T* c, int nx, int ny, int levels, unsigned mask, cudaStream_t st) {
    void* scratch = nullptr;
    int* meta = nullptr;
    static_addresses(&scratch, &meta);
    const size_t N = (size_t)nx * ny;
    int nw = 0, q = 0, dirac_plane = -1;
    for (int b = 0; b < 9; ++b) {
        if (!(mask >> b & 1)) continue;
        if (b == 0) dirac_plane = q; else ++nw;
        ++q;
    }
    // per-basis strides: N / 4 in the first buffer, N / 16 in the second
    T* bufs[2] = {static_cast<T*>(scratch), static_cast<T*>(scratch) + (size_t)nw * (N / 4)};
    const int strides[2] = {(int)(N / 4), (int)(N / 16)};
    int maxL = 2;
    for (int b = 1; b < 9; ++b) if (mask >> b & 1) maxL = std::max(maxL, 2 * b);
    const T inv_sqrt_q = (T)(1.0 / std::sqrt((double)q));
    k_static_meta<<<1, 32, 0, st>>>(mask, meta);
    PURIFY_CUDA(cudaGetLastError());
    add_launches(1);
    const int* pids = meta;
    const int* planes = meta + 8;
    if (nw == 0) {
        dim3 g((nx + 31) / 32, (ny + 31) / 32, 1);
        launch_dependent(k_dwt_level<T>, g, 256, 0, st, x, 0, nx, c, planes, (int)N, nx, nullptr, 0, ny, nx, 16, 16, pids, 0,
                                          dirac_plane, inv_sqrt_q);
        PURIFY_CUDA(cudaGetLastError());
        add_launches(1);
        return;
    }
    int h = ny, w = nx;
    const T* src = x;
    int src_stride = 0, src_ld = nx;
    for (int lev = 0; lev < levels; ++lev) {
        const bool last = lev == levels - 1;
        const int hs = h / 2, wsub = w / 2;
        const int TH = std::min(DWT_T, hs), TW = std::min(DWT_T, wsub);
        const size_t sm = dwt_smem_bytes(maxL, sizeof(T));
        int zdim = nw + ((lev == 0 && dirac_plane >= 0) ? 1 : 0);
        dim3 g((wsub + TW - 1) / TW, (hs + TH - 1) / TH, zdim);
        T* llo = last ? nullptr : bufs[lev & 1];
        const int llstride = strides[lev & 1];
        launch_dependent(k_dwt_level<T>, g, 256, sm, st, src, src_stride, src_ld, c, planes, (int)N, nx, llo, llstride, h, w, TH,
                                           TW, pids, nw, dirac_plane, inv_sqrt_q);
        PURIFY_CUDA(cudaGetLastError());
        add_launches(1);
        src = llo;
        src_stride = llstride;
        src_ld = wsub;
        h = hs;
        w = wsub;
    }
}

void psi_adj_static(const void* x, void* c, int nx, int ny, int levels, unsigned mask, int dtype,
                    cudaStream_t st) {
    init_filter_banks();
    if (dtype == PURIFY_F32) psi_adj_static_t<float>((const float*)x, (float*)c, nx, ny, levels, mask, st);
    else psi_adj_static_t<double>((const double*)x, (double*)c, nx, ny, levels, mask, st);
}

}  // namespace purify
