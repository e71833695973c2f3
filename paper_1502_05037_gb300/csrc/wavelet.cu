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

__device__ __forceinline__ int pmod(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }

// ------------------------------------------------------------- analysis
template <typename T>
__global__ void k_dwt_level(const T* __restrict__ src, int src_basis_stride, int src_ld,
                            T* __restrict__ coef, const int* __restrict__ planes, int N, int nx,
                            T* __restrict__ ll_out, int ll_basis_stride, int h, int w, int TH, int TW,
                            const int* __restrict__ pids, int nw, int dirac_plane, T inv_sqrt_q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FilterBank<T>& fb = fbank<T>();
    const int z = blockIdx.z;
    const int hs = h >> 1, wsub = w >> 1;
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
    const int L = fb.len[pb];
    const T* hf = fb.h[pb];
    const T* gf = fb.g[pb];
    const T* in = src + (size_t)z * src_basis_stride;
    const int ky0 = blockIdx.y * TH, kx0 = blockIdx.x * TW;
    const int th = min(TH, hs - ky0), tw_ = min(TW, wsub - kx0);
    const int Rin = 2 * th + L - 2, Cin = 2 * tw_ + L - 2;
    T* tin = reinterpret_cast<T*>(smem_raw);            // Rin x Cin
    T* ta = tin + Rin * Cin;                            // Rin x tw_  (row low-pass)
    T* td = ta + Rin * tw_;                             // Rin x tw_  (row high-pass)
    for (int t = threadIdx.x; t < Rin * Cin; t += blockDim.x) {
        int r = t / Cin, c = t - r * Cin;
        int gr = pmod(2 * ky0 + r, h), gc = pmod(2 * kx0 + c, w);
        tin[t] = in[(size_t)gr * src_ld + gc];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Rin * tw_; t += blockDim.x) {
        int r = t / tw_, k = t - r * tw_;
        const T* row = tin + r * Cin + 2 * k;
        T a = 0, d = 0;
        for (int n = 0; n < L; ++n) { a += hf[n] * row[n]; d += gf[n] * row[n]; }
        ta[t] = a;
        td[t] = d;
    }
    __syncthreads();
    T* out = coef + (size_t)planes[z] * N;
    for (int t = threadIdx.x; t < th * tw_; t += blockDim.x) {
        int ky = t / tw_, kx = t - ky * tw_;
        T ll = 0, lh = 0, hl = 0, hh = 0;
        for (int n = 0; n < L; ++n) {
            T av = ta[(2 * ky + n) * tw_ + kx], dv = td[(2 * ky + n) * tw_ + kx];
            ll += hf[n] * av; lh += gf[n] * av;
            hl += hf[n] * dv; hh += gf[n] * dv;
        }
        int gy = ky0 + ky, gx = kx0 + kx;
        if (ll_out) ll_out[(size_t)z * ll_basis_stride + (size_t)gy * wsub + gx] = ll;
        else out[(size_t)gy * nx + gx] = ll * inv_sqrt_q;
        out[(size_t)gy * nx + wsub + gx] = hl * inv_sqrt_q;
        out[(size_t)(hs + gy) * nx + gx] = lh * inv_sqrt_q;
        out[(size_t)(hs + gy) * nx + wsub + gx] = hh * inv_sqrt_q;
    }
}

// ------------------------------------------------------------ synthesis
// Reconstruct the 2TH x 2TW output tile at (oy0, ox0) of an h x w band for
// basis pb from its four sub-bands. `ll` points at the low-pass sub-band
// (row stride ll_ld); the three detail sub-bands are read from `det` (the
// basis' coefficient plane, row stride nx). Result goes to acc (per-thread
// registers, outputs t = threadIdx.x + i * blockDim.x).
template <typename T, int PER>
__device__ void synth_tile(const T* __restrict__ ll, int ll_ld, const T* __restrict__ det, int nx, int h, int w,
                           int oy0, int ox0, int th2, int tw2, const T* hf, const T* gf, int L, T* smem,
                           T (&acc)[PER]) {
    const int hs = h >> 1, wsub = w >> 1;
    const int Kr = th2 / 2 + L / 2, Kc = tw2 / 2 + L / 2;
    const int ky_lo = oy0 / 2 - L / 2, kx_lo = ox0 / 2 - L / 2;
    T* sLL = smem;
    T* sHL = sLL + Kr * Kc;   // row-detail, column-approx: (ky, wsub + kx)
    T* sLH = sHL + Kr * Kc;   // row-approx, column-detail: (hs + ky, kx)
    T* sHH = sLH + Kr * Kc;
    T* sA = sHH + Kr * Kc;    // th2 x Kc: column synthesis of the row-approx half
    T* sD = sA + th2 * Kc;    // th2 x Kc: column synthesis of the row-detail half
    __syncthreads();
    for (int t = threadIdx.x; t < Kr * Kc; t += blockDim.x) {
        int r = t / Kc, c = t - r * Kc;
        int ky = pmod(ky_lo + r, hs), kx = pmod(kx_lo + c, wsub);
        sLL[t] = ll[(size_t)ky * ll_ld + kx];
        sHL[t] = det[(size_t)ky * nx + wsub + kx];
        sLH[t] = det[(size_t)(hs + ky) * nx + kx];
        sHH[t] = det[(size_t)(hs + ky) * nx + wsub + kx];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < th2 * Kc; t += blockDim.x) {
        int mr = t / Kc, c = t - mr * Kc;
        int m = oy0 + mr;
        T a = 0, d = 0;
        for (int n = (m & 1); n < L; n += 2) {
            int e = m - n - 2 * ky_lo;   // even, in [1, th2 + L - 1]
            int r = e >> 1;
            a += hf[n] * sLL[r * Kc + c] + gf[n] * sLH[r * Kc + c];
            d += hf[n] * sHL[r * Kc + c] + gf[n] * sHH[r * Kc + c];
        }
        sA[t] = a;
        sD[t] = d;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        int t = threadIdx.x + i * blockDim.x;
        if (t < th2 * tw2) {
            int mr = t / tw2, mc = t - mr * tw2;
            int m = ox0 + mc;
            T s = 0;
            for (int n = (m & 1); n < L; n += 2) {
                int c = (m - n - 2 * kx_lo) >> 1;
                s += hf[n] * sA[mr * Kc + c] + gf[n] * sD[mr * Kc + c];
            }
            acc[i] += s;
        }
    }
}

// One synthesis level for every wavelet basis (blockIdx.z): writes the
// reconstructed h x w band of basis z into ll_out (row stride w).
template <typename T>
__global__ void k_idwt_level(const T* __restrict__ ll_in, int ll_basis_stride, int ll_ld,
                             const T* __restrict__ coef, const int* __restrict__ planes, int N, int nx,
                             T* __restrict__ ll_out, int out_basis_stride, int h, int w, int TH, int TW,
                             const int* __restrict__ pids) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FilterBank<T>& fb = fbank<T>();
    constexpr int PER = 4;
    const int z = blockIdx.z;
    const int pb = pids[z];
    const int L = fb.len[pb];
    const int oy0 = blockIdx.y * 2 * TH, ox0 = blockIdx.x * 2 * TW;
    const int th2 = min(2 * TH, h - oy0), tw2 = min(2 * TW, w - ox0);
    const T* det = coef + (size_t)planes[z] * N;
    const T* ll = ll_in ? ll_in + (size_t)z * ll_basis_stride : det;
    const int ld = ll_in ? ll_ld : nx;
    T acc[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i] = 0;
    synth_tile<T, PER>(ll, ld, det, nx, h, w, oy0, ox0, th2, tw2, fb.h[pb], fb.g[pb], L,
                       reinterpret_cast<T*>(smem_raw), acc);
    T* out = ll_out + (size_t)z * out_basis_stride;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        int t = threadIdx.x + i * blockDim.x;
        if (t < th2 * tw2) {
            int mr = t / tw2, mc = t - mr * tw2;
            out[(size_t)(oy0 + mr) * w + ox0 + mc] = acc[i];
        }
    }
}

// Finest synthesis level summed over all wavelet bases plus the Dirac plane:
// x = (c_dirac + sum_z W_z^T c_z) / sqrt(q). When `level_one_from_coef` is
// set (L == 1) the low-pass bands come from the coefficient planes.
template <typename T>
__global__ void k_idwt_final(const T* __restrict__ ll_in, int ll_basis_stride, const T* __restrict__ coef,
                             const int* __restrict__ planes, int N, int nx, int ny, int TH, int TW,
                             const int* __restrict__ pids, int nw, int dirac_plane,
                             T inv_sqrt_q, T* __restrict__ x) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FilterBank<T>& fb = fbank<T>();
    constexpr int PER = 4;
    const int oy0 = blockIdx.y * 2 * TH, ox0 = blockIdx.x * 2 * TW;
    const int th2 = min(2 * TH, ny - oy0), tw2 = min(2 * TW, nx - ox0);
    T acc[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i] = 0;
    for (int z = 0; z < nw; ++z) {
        const int pb = pids[z];
        const T* det = coef + (size_t)planes[z] * N;
        const T* ll = ll_in ? ll_in + (size_t)z * ll_basis_stride : det;
        const int ld = ll_in ? (nx >> 1) : nx;
        synth_tile<T, PER>(ll, ld, det, nx, ny, nx, oy0, ox0, th2, tw2, fb.h[pb], fb.g[pb], fb.len[pb],
                           reinterpret_cast<T*>(smem_raw), acc);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        int t = threadIdx.x + i * blockDim.x;
        if (t < th2 * tw2) {
            int mr = t / tw2, mc = t - mr * tw2;
            size_t idx = (size_t)(oy0 + mr) * nx + ox0 + mc;
            T v = acc[i];
            if (dirac_plane >= 0) v += coef[(size_t)dirac_plane * N + idx];
            x[idx] = v * inv_sqrt_q;
        }
    }
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

void init_filter_banks() {
    int dev = 0;
    PURIFY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{PURIFY_ECUDA, "device index out of range"};
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
        k_dwt_level<T><<<g, 256, 0, p->stream>>>(x, 0, p->nx, c, plane_array(p), N, p->nx, nullptr, 0, p->ny,
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
        const int TH = std::min(16, hs), TW = std::min(16, wsub);
        int maxL = 2;
        for (int b : p->bases) if (b > 0) maxL = std::max(maxL, 2 * b);
        const int Rin = 2 * TH + maxL - 2, Cin = 2 * TW + maxL - 2;
        size_t sm = sizeof(T) * ((size_t)Rin * Cin + 2 * (size_t)Rin * TW);
        int zdim = wl.nw + ((lev == 0 && wl.dirac_plane >= 0) ? 1 : 0);
        dim3 g((wsub + TW - 1) / TW, (hs + TH - 1) / TH, zdim);
        T* llo = last ? nullptr : bufs[lev & 1];
        Launch L(p, "dwt_level");
        k_dwt_level<T><<<g, 256, sm, p->stream>>>(src, src_stride, src_ld, c, plane_array(p), N, p->nx, llo,
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
    for (int lev = p->levels - 1; lev >= 1 && wl.nw > 0; --lev) {
        const int h = p->ny >> lev, w = p->nx >> lev;
        const int TH = std::min(8, h / 2), TW = std::min(8, w / 2);
        const int Kr = TH + maxL / 2, Kc = TW + maxL / 2;
        size_t sm = sizeof(T) * (4 * (size_t)Kr * Kc + 2 * (size_t)(2 * TH) * Kc);
        dim3 g((w + 2 * TW - 1) / (2 * TW), (h + 2 * TH - 1) / (2 * TH), wl.nw);
        T* out = bufs[lev & 1];
        Launch L(p, "idwt_level");
        k_idwt_level<T><<<g, 256, sm, p->stream>>>(ll_in, llstride, ll_ld, c, plane_array(p), N, p->nx, out,
                                                   llstride, h, w, TH, TW, pid_array(p));
        L.done();
        ll_in = out;
        ll_ld = w;
    }
    const int TH = std::min(8, p->ny / 2), TW = std::min(8, p->nx / 2);
    const int Kr = TH + maxL / 2, Kc = TW + maxL / 2;
    size_t sm = sizeof(T) * (4 * (size_t)Kr * Kc + 2 * (size_t)(2 * TH) * Kc);
    dim3 g((p->nx + 2 * TW - 1) / (2 * TW), (p->ny + 2 * TH - 1) / (2 * TH), 1);
    Launch L(p, "idwt_final");
    k_idwt_final<T><<<g, 256, sm, p->stream>>>(ll_in, llstride, c, plane_array(p), N, p->nx, p->ny, TH, TW,
                                               pid_array(p), wl.nw, wl.dirac_plane, inv_sqrt_q, x);
    L.done();
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
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Host code cannot use g_static_scratch's name as a device address: its
// device address is looked up once per device (with that device current).
static std::mutex g_static_mutex;
static void* g_static_addr[64];

static void* static_scratch_address() {
    int dev = 0;
    PURIFY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{PURIFY_ECUDA, "device index out of range"};
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            throw Error{PURIFY_ECUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                          cudaGetErrorString(e)};
        }
        g_static_addr[dev] = ptr;
    }
    return g_static_addr[dev];
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
    return 256 + 2 * (size_t)nw * (N / 4) * rb;
}

size_t psi_adj_static_capacity() { return kStaticScratchBytes; }

template <typename T>
static void psi_adj_static_t(const T* x, T* c, int nx, int ny, int levels, unsigned mask, cudaStream_t st) {
    unsigned char* base = static_cast<unsigned char*>(static_scratch_address());
    int* meta = reinterpret_cast<int*>(base);
    const size_t N = (size_t)nx * ny;
    int nw = 0, q = 0, dirac_plane = -1;
    for (int b = 0; b < 9; ++b) {
        if (!(mask >> b & 1)) continue;
        if (b == 0) dirac_plane = q; else ++nw;
        ++q;
    }
    T* bufs[2] = {reinterpret_cast<T*>(base + 256), reinterpret_cast<T*>(base + 256) + (size_t)nw * (N / 4)};
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
        k_dwt_level<T><<<g, 256, 0, st>>>(x, 0, nx, c, planes, (int)N, nx, nullptr, 0, ny, nx, 16, 16, pids, 0,
                                          dirac_plane, inv_sqrt_q);
        PURIFY_CUDA(cudaGetLastError());
        add_launches(1);
        return;
    }
    int h = ny, w = nx;
    const T* src = x;
    int src_stride = 0, src_ld = nx;
    const int llstride = (int)(N / 4);
    for (int lev = 0; lev < levels; ++lev) {
        const bool last = lev == levels - 1;
        const int hs = h / 2, wsub = w / 2;
        const int TH = std::min(16, hs), TW = std::min(16, wsub);
        const int Rin = 2 * TH + maxL - 2, Cin = 2 * TW + maxL - 2;
        size_t sm = sizeof(T) * ((size_t)Rin * Cin + 2 * (size_t)Rin * TW);
        int zdim = nw + ((lev == 0 && dirac_plane >= 0) ? 1 : 0);
        dim3 g((wsub + TW - 1) / TW, (hs + TH - 1) / TH, zdim);
        T* llo = last ? nullptr : bufs[lev & 1];
        k_dwt_level<T><<<g, 256, sm, st>>>(src, src_stride, src_ld, c, planes, (int)N, nx, llo, llstride, h, w, TH,
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
