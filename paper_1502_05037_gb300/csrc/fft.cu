// The oversampled two-dimensional FFT of the measurement operator
// Phi = G F Z S and of its adjoint (paper Sec. 1, Eq. 1: the measurement
// equation y = Phi x + n; F is the K_x x K_y DFT of the zero-padded image).
// Four passes around the gridding step:
//   rows_fwd : S, Z and the row transforms of the ny image rows only (the
//              other K - ny grid rows are zero and never stored);
//   cols_fwd : column transforms, the missing rows taken as zeros;
//   cols_inv : inverse column transforms producing only the ny rows kept by
//              Z^T;
//   rows_inv : inverse row transforms fused with Z^T (crop) and S, and in a
//              CG step with the step's dot products and decision;
// plus the plain in-place 2-D transform (purify_fft2).
//
// Each transform is a length-N (N = 2^LOGN, 16 <= N <= 8192) Stockham
// autosort FFT run by N / 8 threads holding eight values each; the length is
// a template parameter, so the stage loop, the shared-memory strides and the
// twiddle spans are constants. A stage of radix r over span Ns (the product
// of the earlier radices) takes butterfly j's inputs v_k = x[j + k N / r],
// multiplies v_k by W_{r Ns}^{(j mod Ns) k}, forms the r-point DFT
// V_q = sum_k v_k W_r^{k q} and writes V_q to ((j - j mod Ns) r + j mod Ns +
// q Ns). The first stage (Ns = 1, radix 2, 4 or 8 so that the rest are radix
// 8) needs no twiddles and reads the input through `load`; the last
// (Ns = N / 8) writes element j + q N / 8 through `store`; the stages in
// between exchange through shared memory, alternating between two buffers so
// that one barrier per stage suffices (a single buffer and two barriers per
// stage where two do not fit). Forward uses W_n = exp(-2 pi i / n), inverse
// its conjugate (unnormalised).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "cg.cuh"
#include "internal.h"
#include "launch.h"
#include "reduce.cuh"

namespace purify {

template <typename C, bool INV> __device__ __forceinline__ C mul_neg_i(C a) {
    // forward: -i a; inverse: +i a
    return INV ? cmake<C>(-a.y, a.x) : cmake<C>(a.y, -a.x);
}

template <typename C> __device__ __forceinline__ void dft2(C& a0, C& a1) {
    C t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

// 4-point DFT, natural order in and out
template <typename C, bool INV> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_neg_i<C, INV>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a1 = cadd(t1, t3);
    a2 = csub(t0, t2);
    a3 = csub(t1, t3);
}

// 8-point DFT, natural order in and out: two 4-point DFTs of the even and odd
// samples combined with W_8^q.
template <typename C, bool INV> __device__ __forceinline__ void dft8(C (&v)[8]) {
    using T = decltype(C::x);
    const T h = T(0.70710678118654752440084436210484904);   // 1 / sqrt(2)
    dft4<C, INV>(v[0], v[2], v[4], v[6]);
    dft4<C, INV>(v[1], v[3], v[5], v[7]);
    // odd part times W_8^q, q = 1, 2, 3
    C o1 = v[3], o2 = v[5], o3 = v[7];
    // W_8 = (1 -+ i) / sqrt(2), W_8^3 = (-1 -+ i) / sqrt(2)
    if (INV) {
        o1 = cmake<C>(h * (o1.x - o1.y), h * (o1.x + o1.y));
        o3 = cmake<C>(-h * (o3.x + o3.y), h * (o3.x - o3.y));
    } else {
        o1 = cmake<C>(h * (o1.x + o1.y), h * (o1.y - o1.x));
        o3 = cmake<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    }
    o2 = mul_neg_i<C, INV>(o2);
    const C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

// shared-memory index of element n with one pad slot per 8 (keeps the
// stride-8 writes of the early stages off a single bank)
__host__ __device__ constexpr int fft_pad(int n) { return n + (n >> 3); }
__host__ __device__ constexpr int fft_padded(int n) { return n + (n >> 3); }

// Shared slots of one transform: element n at a[fft_pad(n) * cs] (cs = 1 for
// a row, the number of columns of the block for a column), the second buffer
// `alt` elements further (alt = 0: one buffer).
template <typename C> struct FftSlots {
    C* a;
    int cs, alt;
};

// One length-2^LOGN transform by thread t (< N / 8). load(k, n) returns input
// element n = t + k N / 8 (k < 8, a constant after unrolling); store(q, n)
// receives output element n = t + q N / 8 (q < 8) and its value.
template <typename C, bool INV, int LOGN, typename Load, typename Store>
__device__ __forceinline__ void fft_core(int t, const C* __restrict__ tw, Load load, Store store, FftSlots<C> s) {
    constexpr int N = 1 << LOGN, N8 = N >> 3;
    constexpr int R0 = (LOGN % 3 == 0) ? 8 : (LOGN % 3 == 1 ? 2 : 4);
    constexpr int LR0 = R0 == 8 ? 3 : (R0 == 4 ? 2 : 1);
    constexpr int NST = (LOGN - LR0) / 3;   // radix-8 stages after the first
    static_assert(LOGN >= 4 && LOGN <= 13, "FFT length out of range");
    const int cs = s.cs;
    const bool pp = s.alt != 0;
    C v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = load(k, t + k * N8);
    C* const b0 = s.a;
    if constexpr (R0 == 8) {
        dft8<C, INV>(v);
        // slots 8 t + q, q < 8: fft_pad = 9 t + q
        C* const o = b0 + 9 * t * cs;
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q * cs] = v[q];
    } else if constexpr (R0 == 4) {
        // butterflies j = t (inputs k = 0, 2, 4, 6) and j = t + N/8 (1, 3, 5, 7)
        dft4<C, INV>(v[0], v[2], v[4], v[6]);
        dft4<C, INV>(v[1], v[3], v[5], v[7]);
        // slots 4 t + q, q < 4: fft_pad = 4 t + q + t / 2; 4 N8 is a multiple of 8
        C* const o = b0 + (4 * t + (t >> 1)) * cs;
        constexpr int J1 = fft_pad(4 * N8);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            o[q * cs] = v[2 * q];
            o[(J1 + q) * cs] = v[2 * q + 1];
        }
    } else {
        // butterflies j = t + m N/8, m < 4, inputs m and m + 4
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            dft2<C>(v[m], v[m + 4]);
            const int n0 = (t + m * N8) * 2;
            b0[fft_pad(n0) * cs] = v[m];
            b0[fft_pad(n0 + 1) * cs] = v[m + 4];
        }
    }
#pragma unroll
    for (int st = 0; st < NST; ++st) {
        const int Ns = R0 << (3 * st);
        // stage st reads buffer st mod 2 and writes the other (one buffer
        // when alt = 0)
        const C* const src = (pp && (st & 1)) ? b0 + s.alt : b0;
        C* const dst = (pp && !(st & 1)) ? b0 + s.alt : b0;
        __syncthreads();
        const int kk = t & (Ns - 1);
        if constexpr (N8 % 8 == 0) {
            const C* const i0 = src + fft_pad(t) * cs;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = i0[k * fft_pad(N8) * cs];
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = src[fft_pad(t + k * N8) * cs];
        }
        // W^{k ts} for k = 1..7 from three table entries (k = 1, 2, 4) and
        // four products
        const int ts = kk * (N8 / Ns);
        C w[8];
        w[1] = tw[ts];
        w[2] = tw[2 * ts];
        w[4] = tw[4 * ts];
        w[3] = cmul(w[1], w[2]);
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
#pragma unroll
        for (int k = 1; k < 8; ++k) v[k] = INV ? cmulconj(v[k], w[k]) : cmul(v[k], w[k]);
        dft8<C, INV>(v);
        if (st == NST - 1) {
#pragma unroll
            for (int q = 0; q < 8; ++q) store(q, t + q * N8, v[q]);
        } else {
            if (!pp) __syncthreads();
            const int base = (t - kk) * 8 + kk;
            if (Ns % 8 == 0) {
                C* const o = dst + fft_pad(base) * cs;
#pragma unroll
                for (int q = 0; q < 8; ++q) o[q * fft_pad(Ns) * cs] = v[q];
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) dst[fft_pad(base + q * Ns) * cs] = v[q];
            }
        }
    }
}

// ------------------------------------------- two FP32 transforms per thread
// The same Stockham stages on element n of two transforms at once (two rows
// of a block, or two adjacent columns): a P2 holds their values as packed
// pairs (re = (re_0, re_1), im = (im_0, im_1)), so that every butterfly and
// twiddle product is one packed two-lane FP32 instruction for both
// transforms and a shared-memory exchange moves 16 bytes. Each lane computes
// what the one-transform core computes, operation for operation.
struct P2 {
    float2 re, im;
};
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, rounded once like a subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ P2 padd(P2 a, P2 b) { return P2{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ P2 psub(P2 a, P2 b) { return P2{sub2(a.re, b.re), sub2(a.im, b.im)}; }
// v times w (forward) or conj(w) (inverse); w = (wr, wi) broadcast to both lanes
template <bool INV> __device__ __forceinline__ P2 pmul(P2 v, float2 wr, float2 wi) {
    if (INV) return P2{__ffma2_rn(v.re, wr, __fmul2_rn(v.im, wi)), __ffma2_rn(v.im, wr, __fmul2_rn(v.re, make_float2(-wi.x, -wi.y)))};
    return P2{__ffma2_rn(v.re, wr, __fmul2_rn(v.im, make_float2(-wi.x, -wi.y))), __ffma2_rn(v.im, wr, __fmul2_rn(v.re, wi))};
}

// 4-point DFT of both lanes; the -i (forward) or +i (inverse) factor is
// folded into the last additions
template <bool INV> __device__ __forceinline__ void pdft4(P2& a0, P2& a1, P2& a2, P2& a3) {
    const P2 t0 = padd(a0, a2), t1 = psub(a0, a2), t2 = padd(a1, a3), d = psub(a1, a3);
    a0 = padd(t0, t2);
    a2 = psub(t0, t2);
    if (INV) {   // t3 = i d = (-d.im, d.re)
        a1 = P2{sub2(t1.re, d.im), add2(t1.im, d.re)};
        a3 = P2{add2(t1.re, d.im), sub2(t1.im, d.re)};
    } else {     // t3 = -i d = (d.im, -d.re)
        a1 = P2{add2(t1.re, d.im), sub2(t1.im, d.re)};
        a3 = P2{sub2(t1.re, d.im), add2(t1.im, d.re)};
    }
}

template <bool INV> __device__ __forceinline__ void pdft8(P2 (&v)[8]) {
    const float h = 0.70710678118654752440084436210484904f;   // 1 / sqrt(2)
    pdft4<INV>(v[0], v[2], v[4], v[6]);
    pdft4<INV>(v[1], v[3], v[5], v[7]);
    P2 o1 = v[3], o3 = v[7];
    const P2 o2 = v[5];
    // o1 W_8, o3 W_8^3; W_8 = (1 -+ i) / sqrt(2), W_8^3 = (-1 -+ i) / sqrt(2)
    if (INV) {
        o1 = P2{__fmul2_rn(bc2(h), sub2(o1.re, o1.im)), __fmul2_rn(bc2(h), add2(o1.re, o1.im))};
        o3 = P2{__fmul2_rn(bc2(-h), add2(o3.re, o3.im)), __fmul2_rn(bc2(h), sub2(o3.re, o3.im))};
    } else {
        o1 = P2{__fmul2_rn(bc2(h), add2(o1.re, o1.im)), __fmul2_rn(bc2(h), sub2(o1.im, o1.re))};
        o3 = P2{__fmul2_rn(bc2(h), sub2(o3.im, o3.re)), __fmul2_rn(bc2(-h), add2(o3.re, o3.im))};
    }
    const P2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = padd(e0, o0);
    v[4] = psub(e0, o0);
    v[1] = padd(e1, o1);
    v[5] = psub(e1, o1);
    // e2 -+ i o2
    if (INV) {
        v[2] = P2{sub2(e2.re, o2.im), add2(e2.im, o2.re)};
        v[6] = P2{add2(e2.re, o2.im), sub2(e2.im, o2.re)};
    } else {
        v[2] = P2{add2(e2.re, o2.im), sub2(e2.im, o2.re)};
        v[6] = P2{sub2(e2.re, o2.im), add2(e2.im, o2.re)};
    }
    v[3] = padd(e3, o3);
    v[7] = psub(e3, o3);
}

// Shared slots of a pair of transforms: element n at a[fft_pad(n) * cs] as
// one float4 (re_0, re_1, im_0, im_1), the second buffer `alt` float4 further.
struct FftSlots2 {
    float4* a;
    int cs, alt;
};
__device__ __forceinline__ float4 p2_pack(P2 v) { return make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }
__device__ __forceinline__ P2 p2_unpack(float4 q) { return P2{make_float2(q.x, q.y), make_float2(q.z, q.w)}; }

// fft_core for two FP32 transforms: load(k, n) returns their input element
// n = t + k N / 8 as a P2, store(q, n, v) receives output element n.
template <bool INV, int LOGN, typename Load, typename Store>
__device__ __forceinline__ void fft_core2(int t, const float2* __restrict__ tw, Load load, Store store, FftSlots2 s) {
    constexpr int N = 1 << LOGN, N8 = N >> 3;
    constexpr int R0 = (LOGN % 3 == 0) ? 8 : (LOGN % 3 == 1 ? 2 : 4);
    constexpr int LR0 = R0 == 8 ? 3 : (R0 == 4 ? 2 : 1);
    constexpr int NST = (LOGN - LR0) / 3;
    static_assert(LOGN >= 4 && LOGN <= 13, "FFT length out of range");
    const int cs = s.cs;
    const bool pp = s.alt != 0;
    P2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = load(k, t + k * N8);
    float4* const b0 = s.a;
    if constexpr (R0 == 8) {
        pdft8<INV>(v);
        float4* const o = b0 + 9 * t * cs;
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q * cs] = p2_pack(v[q]);
    } else if constexpr (R0 == 4) {
        pdft4<INV>(v[0], v[2], v[4], v[6]);
        pdft4<INV>(v[1], v[3], v[5], v[7]);
        float4* const o = b0 + (4 * t + (t >> 1)) * cs;
        constexpr int J1 = fft_pad(4 * N8);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            o[q * cs] = p2_pack(v[2 * q]);
            o[(J1 + q) * cs] = p2_pack(v[2 * q + 1]);
        }
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const P2 a = v[m], b = v[m + 4];
            const int n0 = (t + m * N8) * 2;
            b0[fft_pad(n0) * cs] = p2_pack(padd(a, b));
            b0[fft_pad(n0 + 1) * cs] = p2_pack(psub(a, b));
        }
    }
#pragma unroll
    for (int st = 0; st < NST; ++st) {
        const int Ns = R0 << (3 * st);
        const float4* const src = (pp && (st & 1)) ? b0 + s.alt : b0;
        float4* const dst = (pp && !(st & 1)) ? b0 + s.alt : b0;
        __syncthreads();
        const int kk = t & (Ns - 1);
        if constexpr (N8 % 8 == 0) {
            const float4* const i0 = src + fft_pad(t) * cs;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = p2_unpack(i0[k * fft_pad(N8) * cs]);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = p2_unpack(src[fft_pad(t + k * N8) * cs]);
        }
        // W^{k ts}, k = 1..7, from three table entries and four products
        // (the same products as the one-transform core), broadcast to both lanes
        const int ts = kk * (N8 / Ns);
        float2 wr[8], wi[8];
        {
            const float2 a = tw[ts], b = tw[2 * ts], c = tw[4 * ts];
            wr[1] = bc2(a.x); wi[1] = bc2(a.y);
            wr[2] = bc2(b.x); wi[2] = bc2(b.y);
            wr[4] = bc2(c.x); wi[4] = bc2(c.y);
        }
        auto wmul = [&](int a, int b, int o) {
            // (wr[a] + i wi[a]) (wr[b] + i wi[b])
            wr[o] = __ffma2_rn(wr[a], wr[b], __fmul2_rn(wi[a], make_float2(-wi[b].x, -wi[b].y)));
            wi[o] = __ffma2_rn(wr[a], wi[b], __fmul2_rn(wi[a], wr[b]));
        };
        wmul(1, 2, 3);
        wmul(1, 4, 5);
        wmul(2, 4, 6);
        wmul(3, 4, 7);
#pragma unroll
        for (int k = 1; k < 8; ++k) v[k] = pmul<INV>(v[k], wr[k], wi[k]);
        pdft8<INV>(v);
        if (st == NST - 1) {
#pragma unroll
            for (int q = 0; q < 8; ++q) store(q, t + q * N8, v[q]);
        } else {
            if (!pp) __syncthreads();
            const int base = (t - kk) * 8 + kk;
            if (Ns % 8 == 0) {
                float4* const o = dst + fft_pad(base) * cs;
#pragma unroll
                for (int q = 0; q < 8; ++q) o[q * fft_pad(Ns) * cs] = p2_pack(v[q]);
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) dst[fft_pad(base + q * Ns) * cs] = p2_pack(v[q]);
            }
        }
    }
}

// ------------------------------------------------------------ row passes
// Row kernels: a block holds rb transforms of length Kx = 2^LX, thread
// (f, t) = (tid / (Kx/8), tid mod (Kx/8)) runs row f, whose slots start at
// f * pad(Kx); the second buffer (alt > 0) follows the first. (Rows keep one
// transform per thread: the forward pass carries the CG vector updates and
// the inverse pass the dot products, per-pixel work that wants the threads.)
template <int N8> __device__ __forceinline__ void row_thread(int rb, int& i, int& t, int& f) {
    f = threadIdx.x / N8;
    t = threadIdx.x - f * N8;
    i = blockIdx.x * rb + f;
}

// S Z and the forward row FFT: rows [i0, i0+rb) of the image to rows[i][0..Kx).
// With a CG fold (fold.x set) the input is the residual r after the step's
// update (see CgFold), not x. When zero_grid != null block b also clears rows
// [b Ky/gridDim, (b+1) Ky/gridDim) of that Ky x Kx complex grid (the gridding
// accumulator of the same CG step, or of the adjoint that follows Phi).
template <typename T, int LX>
__global__ void __launch_bounds__(1024) k_rows_fwd(const T* __restrict__ x, typename cplx_of<T>::type* __restrict__ rows,
                           const T* __restrict__ sx, const T* __restrict__ sy,
                           const typename cplx_of<T>::type* __restrict__ tw, int nx, int ny,
                           int rb, int alt, T scale, const int* __restrict__ skip,
                           typename cplx_of<T>::type* __restrict__ zero_grid, int Ky, CgFold fold) {
    using C = typename cplx_of<T>::type;
    constexpr int Kx = 1 << LX, N8 = Kx >> 3;
    pdl_wait();
    // step 0 starts the solve; later steps first apply the previous step's
    // update unless it met the stop test (see CgFold)
    const bool first = fold.x && fold.step == 0;
    T* const fx = static_cast<T*>(fold.x);
    T* const fr = static_cast<T*>(fold.r);
    T* const fs = static_cast<T*>(fold.s);
    T* const pdir = static_cast<T*>(fold.p);
    const T* const fu = static_cast<const T*>(fold.u);
    const T* const fadd = static_cast<const T*>(fold.add);
    // stopped at an earlier step (block 0 of this pass may set the flag
    // meanwhile: each block reads it once)
    if (block_flag(first ? nullptr : skip)) return;
    bool pending = false;
    T alpha = T(0), cbeta = T(0);
    if (fold.x && !first) {
        // the previous step's update (it did not stop the solve: checked above)
        double al, be;
        if (!cg_pending(fold, al, be)) return;
        pending = true;
        alpha = (T)al;
        cbeta = (T)be;
    }
    if (first && blockIdx.x == 0 && threadIdx.x == 0) fold.flags[F_CGDONE] = 0;   // the next kernels read it
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (zero_grid) {
        // whole rows per block (Ky is a multiple of the block count), in
        // 16-byte stores
        const int per = Ky / gridDim.x;
        float4* g = reinterpret_cast<float4*>(zero_grid + (size_t)blockIdx.x * per * Kx);
        const int n16 = per * Kx * (int)sizeof(C) / 16;
        for (int t = threadIdx.x; t < n16; t += blockDim.x) g[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int i0, t, f;
    row_thread<N8>(rb, i0, t, f);
    // S Z of pixel p1 of image row i (p1 < Kx/2 exactly when k < 4)
    auto pix = [&](int i, int k, int p1) -> T {
        // pixel column j with (j - nx/2) mod Kx == p1
        const int j = (k < 4 ? p1 : p1 - Kx) + nx / 2;
        if (j < 0 || j >= nx) return T(0);
        const size_t idx = (size_t)i * nx + j;
        T xv;
        if (fold.x) {
            // Chronopoulos-Gear update, then the transform of the new r
            T rv = fr[idx];
            if (first) {
                if (fadd) {
                    rv += fadd[idx];
                    fr[idx] = rv;
                }
                pdir[idx] = T(0);
                fs[idx] = T(0);
            } else if (pending) {
                const T pv = rv + cbeta * pdir[idx];
                const T sv = fu[idx] + cbeta * fs[idx];
                pdir[idx] = pv;
                fs[idx] = sv;
                fx[idx] += alpha * pv;
                rv = rv - alpha * sv;
                fr[idx] = rv;
            }
            xv = rv;
        } else {
            xv = x[idx];
        }
        return xv * sx[j] * (sy[i] * scale);
    };
    C* buf = reinterpret_cast<C*>(smem_raw) + f * fft_padded(Kx);
    C* const out = rows + (size_t)i0 * Kx;
    auto load = [&](int k, int p1) -> C { return cmake<C>(pix(i0, k, p1), T(0)); };
    auto store = [&](int, int k, C v) { out[k] = v; };
    fft_core<C, false, LX>(t, tw, load, store, FftSlots<C>{buf, 1, alt});
    pdl_trigger();
}

// Column kernels: a block holds cb adjacent columns of length Ky = 2^LY.
// With W = 1 thread (t, f) = (tid / cb, tid mod cb) runs column f, element
// n in shared slot pad(n) * cb + f; with W = 2 (FP32) thread
// (t, f) = (tid / (cb/2), tid mod (cb/2)) runs columns 2f and 2f + 1 as one
// pair with 16-byte global accesses, element n in float4 slot
// pad(n) * (cb/2) + f. A warp's global accesses cover consecutive cells of
// each row. The second buffer (alt > 0) follows the first.
template <int W> __device__ __forceinline__ void col_thread(int cb, int& c0, int& t, int& f) {
    const int cp = cb / W;
    t = threadIdx.x / cp;
    f = threadIdx.x - t * cp;
    c0 = blockIdx.x * cb + W * f;
}

// Forward column FFT over columns [c0, c0+cb): the only non-zero grid rows
// are p2 = (i - ny/2) mod Ky for image rows i.
template <typename T, int LY, int W>
__global__ void __launch_bounds__(1024) k_cols_fwd(const typename cplx_of<T>::type* __restrict__ rows,
                           typename cplx_of<T>::type* __restrict__ grid,
                           const typename cplx_of<T>::type* __restrict__ tw, int ny, int Kx,
                           int cb, int alt, const int* __restrict__ skip) {
    using C = typename cplx_of<T>::type;
    constexpr int Ky = 1 << LY;
    pdl_wait();
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int c, t, f;
    col_thread<W>(cb, c, t, f);
    // image row of grid row n (n < Ky/2 exactly when k < 4), or -1
    auto src_row = [&](int k, int n) -> int {
        const int i = (k < 4 ? n : n - Ky) + ny / 2;
        return (i >= 0 && i < ny) ? i : -1;
    };
    if constexpr (W == 1) {
        C* buf = reinterpret_cast<C*>(smem_raw);
        auto load = [&](int k, int n) -> C {
            const int i = src_row(k, n);
            return i >= 0 ? rows[(size_t)i * Kx + c] : cmake<C>(T(0), T(0));
        };
        auto store = [&](int, int k, C v) { grid[(size_t)k * Kx + c] = v; };
        fft_core<C, false, LY>(t, tw, load, store, FftSlots<C>{buf + f, cb, alt});
    } else {
        float4* buf = reinterpret_cast<float4*>(smem_raw);
        auto load = [&](int k, int n) -> P2 {
            const int i = src_row(k, n);
            if (i < 0) return P2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            const float4 q = *reinterpret_cast<const float4*>(rows + (size_t)i * Kx + c);
            return P2{make_float2(q.x, q.z), make_float2(q.y, q.w)};
        };
        auto store = [&](int, int k, P2 v) {
            *reinterpret_cast<float4*>(grid + (size_t)k * Kx + c) = make_float4(v.re.x, v.im.x, v.re.y, v.im.y);
        };
        fft_core2<false, LY>(t, tw, load, store, FftSlots2{buf + f, cb / 2, alt / 2});
    }
    pdl_trigger();
}

// Inverse column FFT over columns [c0, c0+cb) (grid optionally multiplied
// elementwise by `mult` first), keeping only the image rows.
template <typename T, int LY, int W>
__global__ void __launch_bounds__(1024) k_cols_inv(const typename cplx_of<T>::type* __restrict__ grid,
                           typename cplx_of<T>::type* __restrict__ rows,
                           const typename cplx_of<T>::type* __restrict__ tw, int ny, int Kx,
                           int cb, int alt, const int* __restrict__ skip, const T* __restrict__ mult) {
    using C = typename cplx_of<T>::type;
    constexpr int Ky = 1 << LY;
    pdl_wait();
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int c, t, f;
    col_thread<W>(cb, c, t, f);
    // image row kept for grid row p2, or -1
    auto dst_row = [&](int p2) -> int {
        const int i = (p2 + ny / 2) & (Ky - 1);
        return i < ny ? i : -1;
    };
    if constexpr (W == 1) {
        C* buf = reinterpret_cast<C*>(smem_raw);
        auto load = [&](int, int k) -> C {
            const size_t g = (size_t)k * Kx + c;
            C v = grid[g];
            if (mult) v = cscale(v, mult[g]);
            return v;
        };
        auto store = [&](int, int p2, C v) {
            const int i = dst_row(p2);
            if (i >= 0) rows[(size_t)i * Kx + c] = v;
        };
        fft_core<C, true, LY>(t, tw, load, store, FftSlots<C>{buf + f, cb, alt});
    } else {
        float4* buf = reinterpret_cast<float4*>(smem_raw);
        auto load = [&](int, int k) -> P2 {
            const size_t g = (size_t)k * Kx + c;
            float4 q = *reinterpret_cast<const float4*>(grid + g);
            if (mult) {
                const float2 m = *reinterpret_cast<const float2*>(mult + g);
                q = make_float4(q.x * m.x, q.y * m.x, q.z * m.y, q.w * m.y);
            }
            return P2{make_float2(q.x, q.z), make_float2(q.y, q.w)};
        };
        auto store = [&](int, int p2, P2 v) {
            const int i = dst_row(p2);
            if (i >= 0)
                *reinterpret_cast<float4*>(rows + (size_t)i * Kx + c) = make_float4(v.re.x, v.im.x, v.re.y, v.im.y);
        };
        fft_core2<true, LY>(t, tw, load, store, FftSlots2{buf + f, cb / 2, alt / 2});
    }
    pdl_trigger();
}

// Inverse row FFT of image rows [i0, i0+rb), then Z^T and S:
//   out_mode 0: complex out[i][j] = scale * s * v
//   out_mode 1: real    out[i][j] = scale * s * Re v + add_coef * (add ? add[i][j] : 0)
// With cg.part set (a CG step: out = A r, add = r, see CgFold) the kernel
// also writes per-block partials of r . r and r . A r, and its last block
// reduces them and decides the step (cg_decide).
template <typename T, int LX, int MAXT>
__global__ void __launch_bounds__(MAXT) k_rows_inv(const typename cplx_of<T>::type* __restrict__ rows, void* out,
                           const T* __restrict__ sx, const T* __restrict__ sy,
                           const typename cplx_of<T>::type* __restrict__ tw, int nx, int ny,
                           int rb, int alt, T scale, int out_mode, const T* __restrict__ add, T add_coef,
                           const int* __restrict__ skip, CgFold cgf) {
    using C = typename cplx_of<T>::type;
    constexpr int Kx = 1 << LX, N8 = Kx >> 3;
    pdl_wait();
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int i0, t, f;
    row_thread<N8>(rb, i0, t, f);
    T dacc = 0, gacc2 = 0;   // add.out, and with the folded CG add.add (add = r, out = A r)
    const bool cg = cgf.part != nullptr;
    // Z^T, S and the epilogue for element p1 of row i's transform
    auto emit = [&](int i, int p1, T vr, T vi) {
        const int j = (p1 + nx / 2) & (Kx - 1);
        if (j >= nx) return;
        const T s = sx[j] * (sy[i] * scale);
        const size_t idx = (size_t)i * nx + j;
        if (out_mode == 0) {
            reinterpret_cast<C*>(out)[idx] = cmake<C>(vr * s, vi * s);
        } else {
            T r = vr * s;
            if (add) {
                const T a = add[idx];
                r += add_coef * a;
                dacc += a * r;
                if (cg) gacc2 += a * a;
            }
            reinterpret_cast<T*>(out)[idx] = r;
        }
    };
    C* buf = reinterpret_cast<C*>(smem_raw) + f * fft_padded(Kx);
    const C* const in = rows + (size_t)i0 * Kx;
    auto load = [&](int, int k) -> C { return in[k]; };
    auto store = [&](int, int p1, C v) { emit(i0, p1, v.x, v.y); };
    fft_core<C, true, LX>(t, tw, load, store, FftSlots<C>{buf, 1, alt});
    if (cg) {
        // Chronopoulos-Gear partials (see CgFold): gamma = r.r, delta = r.A r;
        // the consumer of this step's scalars reduces them
        const double b0 = block_sum_t(gacc2);
        const double b1 = block_sum_t(dacc);
        if (threadIdx.x == 0) {
            cgf.part[2 * blockIdx.x] = b0;
            cgf.part[2 * blockIdx.x + 1] = b1;
        }
        if (arrive_last(cgf.counter)) {
            cg_decide(cgf, cgf.step, gridDim.x);
            if (threadIdx.x == 0) *cgf.counter = 0;
        }
    }
    pdl_trigger();
}

// Plain in-place 2-D FFT pieces (purify_fft2): full row pass / column pass.
// In place is safe: every input element is read in the first stage, before
// the first barrier, and every output is written in the last.
template <typename T, int LX, bool INV>
__global__ void __launch_bounds__(1024) k_rows_full(typename cplx_of<T>::type* grid, const typename cplx_of<T>::type* __restrict__ tw,
                            int rb, int alt) {
    using C = typename cplx_of<T>::type;
    constexpr int Kx = 1 << LX, N8 = Kx >> 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int i0, t, f;
    row_thread<N8>(rb, i0, t, f);
    C* buf = reinterpret_cast<C*>(smem_raw) + f * fft_padded(Kx);
    C* row = grid + (size_t)i0 * Kx;
    auto load = [&](int, int k) -> C { return row[k]; };
    auto store = [&](int, int k, C v) { row[k] = v; };
    fft_core<C, INV, LX>(t, tw, load, store, FftSlots<C>{buf, 1, alt});
}

template <typename T, int LY, bool INV, int W>
__global__ void __launch_bounds__(1024) k_cols_full(typename cplx_of<T>::type* grid, const typename cplx_of<T>::type* __restrict__ tw,
                            int Kx, int cb, int alt) {
    using C = typename cplx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int c, t, f;
    col_thread<W>(cb, c, t, f);
    if constexpr (W == 1) {
        C* buf = reinterpret_cast<C*>(smem_raw);
        auto load = [&](int, int k) -> C { return grid[(size_t)k * Kx + c]; };
        auto store = [&](int, int k, C v) { grid[(size_t)k * Kx + c] = v; };
        fft_core<C, INV, LY>(t, tw, load, store, FftSlots<C>{buf + f, cb, alt});
    } else {
        float4* buf = reinterpret_cast<float4*>(smem_raw);
        auto load = [&](int, int k) -> P2 {
            const float4 q = *reinterpret_cast<const float4*>(grid + (size_t)k * Kx + c);
            return P2{make_float2(q.x, q.z), make_float2(q.y, q.w)};
        };
        auto store = [&](int, int k, P2 v) {
            *reinterpret_cast<float4*>(grid + (size_t)k * Kx + c) = make_float4(v.re.x, v.im.x, v.re.y, v.im.y);
        };
        fft_core2<INV, LY>(t, tw, load, store, FftSlots2{buf + f, cb / 2, alt / 2});
    }
}

// ------------------------------------------------------------- launchers
__host__ __device__ inline int ilog2_fft(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

// Calls f(std::integral_constant<int, log2 n>) for a transform length n.
template <typename F> static void with_log2(int n, F&& f) {
    switch (ilog2_fft(n)) {
        case 4: f(std::integral_constant<int, 4>()); break;
        case 5: f(std::integral_constant<int, 5>()); break;
        case 6: f(std::integral_constant<int, 6>()); break;
        case 7: f(std::integral_constant<int, 7>()); break;
        case 8: f(std::integral_constant<int, 8>()); break;
        case 9: f(std::integral_constant<int, 9>()); break;
        case 10: f(std::integral_constant<int, 10>()); break;
        case 11: f(std::integral_constant<int, 11>()); break;
        case 12: f(std::integral_constant<int, 12>()); break;
        case 13: f(std::integral_constant<int, 13>()); break;
        default: throw Error{PURIFY_EINVAL, "FFT length out of range"};
    }
}

template <typename K> static void set_fft_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) PURIFY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// Shared memory of nb transforms of length K: one buffer of nb * pad(K)
// values, two (alternating stages) when they fit in 216 KB.
static constexpr size_t kFftTwoBufMax = 216 * 1024;
static int fft_alt(int nb, int K, size_t cbytes) {
    const size_t one = (size_t)nb * fft_padded(K) * cbytes;
    return 2 * one <= kFftTwoBufMax ? nb * fft_padded(K) : 0;
}
static size_t fft_smem(int nb, int K, size_t cbytes, int alt) {
    return (alt ? 2 : 1) * (size_t)nb * fft_padded(K) * cbytes;
}

// FFT launch shapes: K / 8 threads per transform; transforms per block
// (rows rb, columns cb) chosen so that a block has at most 512 threads and
// the grid covers the 152 SMs about twice; the autotuner may override.
static int fft_block_limit(int K, size_t cbytes) {
    int nb = 1;
    while (nb < 8 && 2 * nb * (K / 8) <= 512 && 2 * (size_t)nb * fft_padded(K) * cbytes <= 160 * 1024) nb *= 2;
    return nb;
}
template <typename T> static int rows_per_block(int nrows, int K) {
    int rb = std::min(fft_block_limit(K, sizeof(typename cplx_of<T>::type)), std::max(1, nrows / 256));
    while (rb > 1 && nrows % rb) rb >>= 1;
    return rb;
}
template <typename T> static int cols_per_block(int Ky, int Kx) {
    int cb = std::min(fft_block_limit(Ky, sizeof(typename cplx_of<T>::type)), std::max(1, Kx / 256));
    while (cb > 1 && Kx % cb) cb >>= 1;
    return cb;
}
// nb transforms of length K per block, `lanes` of them per thread (2: the
// packed FP32 column form, for an even nb)
bool fft_shape_ok(int nb, int K, int dtype, int lanes) {
    const size_t cbytes = dtype == PURIFY_F32 ? 8 : 16;
    if (lanes != 1 && (lanes != 2 || dtype != PURIFY_F32 || nb % 2)) return false;
    return nb / lanes * (K / 8) <= 1024 && (size_t)nb * fft_padded(K) * cbytes <= 160 * 1024;
}

template <typename T> static int plan_rows_per_block(const purify_plan* p) {
    int rb = p->fft_rb > 0 ? p->fft_rb : rows_per_block<T>(p->ny, p->Kx);
    while (p->ny % rb) rb >>= 1;
    return rb;
}
template <typename T> static int plan_cols_per_block(const purify_plan* p) {
    return p->fft_cb > 0 ? p->fft_cb : cols_per_block<T>(p->Ky, p->Kx);
}
// columns per thread: the tuned choice, else two (packed) for FP32 blocks of
// an even number of columns
template <typename T> static int col_lanes(int cb, int tuned) {
    if (sizeof(T) != 4 || cb % 2) return 1;
    return tuned > 0 ? tuned : 2;
}

template <typename T>
static void rows_fwd_t(purify_plan* p, const void* x, double scale, const int* skip, bool corr, bool zero_acc,
                       const CgFold* fold) {
    using C = typename cplx_of<T>::type;
    const int rb = plan_rows_per_block<T>(p);
    const int alt = fft_alt(rb, p->Kx, sizeof(C));
    const size_t sm = fft_smem(rb, p->Kx, sizeof(C), alt);
    with_log2(p->Kx, [&](auto lg) {
        auto kern = k_rows_fwd<T, decltype(lg)::value>;
        set_fft_smem(kern, sm);
        Launch L(p, "fft_rows_fwd");
        launch_dependent(kern, p->ny / rb, rb * (p->Kx / 8), sm, p->stream,
            (const T*)x, p->rows.as<C>(), corr ? p->sx.as<T>() : p->onesx.as<T>(),
            corr ? p->sy.as<T>() : p->onesy.as<T>(), p->twx.as<C>(), p->nx, p->ny,
            rb, alt, (T)scale, skip, zero_acc ? p->gacc.as<C>() : nullptr, p->Ky,
            fold ? *fold : CgFold());
        L.done();
    });
}

template <typename T> static void cols_fwd_t(purify_plan* p, const int* skip) {
    using C = typename cplx_of<T>::type;
    const int cb = plan_cols_per_block<T>(p);
    const int alt = fft_alt(cb, p->Ky, sizeof(C));
    const size_t sm = fft_smem(cb, p->Ky, sizeof(C), alt);
    const int w = col_lanes<T>(cb, p->fft_cw);
    with_log2(p->Ky, [&](auto lg) {
        constexpr int LY = decltype(lg)::value;
        auto kern = k_cols_fwd<T, LY, 1>;
        if constexpr (sizeof(T) == 4) { if (w == 2) kern = k_cols_fwd<T, LY, 2>; }
        set_fft_smem(kern, sm);
        Launch L(p, "fft_cols_fwd");
        launch_dependent(kern, p->Kx / cb, cb / w * (p->Ky / 8), sm, p->stream, p->rows.as<C>(), p->grid.as<C>(),
                         p->twy.as<C>(), p->ny, p->Kx, cb, alt, skip);
        L.done();
    });
}

template <typename T> static void cols_inv_t(purify_plan* p, const int* skip, const void* mult) {
    using C = typename cplx_of<T>::type;
    const int cb = plan_cols_per_block<T>(p);
    const int alt = fft_alt(cb, p->Ky, sizeof(C));
    const size_t sm = fft_smem(cb, p->Ky, sizeof(C), alt);
    // the adjoint reads the gridding output; the circulant path the forward grid
    const C* src = mult ? p->grid.as<C>() : p->gacc.as<C>();
    const int w = col_lanes<T>(cb, p->fft_cw);
    with_log2(p->Ky, [&](auto lg) {
        constexpr int LY = decltype(lg)::value;
        auto kern = k_cols_inv<T, LY, 1>;
        if constexpr (sizeof(T) == 4) { if (w == 2) kern = k_cols_inv<T, LY, 2>; }
        set_fft_smem(kern, sm);
        Launch L(p, "fft_cols_inv");
        launch_dependent(kern, p->Kx / cb, cb / w * (p->Ky / 8), sm, p->stream, src, p->rows.as<C>(),
                         p->twy.as<C>(), p->ny, p->Kx, cb, alt, skip, (const T*)mult);
        L.done();
    });
}

template <typename T>
static void rows_inv_t(purify_plan* p, void* out, double scale, int out_mode, const void* add, double add_coef,
                       const int* skip, const CgFold* cg, bool corr) {
    using C = typename cplx_of<T>::type;
    const int rb = plan_rows_per_block<T>(p);
    const int alt = fft_alt(rb, p->Kx, sizeof(C));
    const size_t sm = fft_smem(rb, p->Kx, sizeof(C), alt);
    const int nt = rb * (p->Kx / 8);
    with_log2(p->Kx, [&](auto lg) {
        constexpr int LX = decltype(lg)::value;
        // blocks of at most 512 threads may take more than 64 registers
        auto kern = nt <= 512 ? k_rows_inv<T, LX, 512> : k_rows_inv<T, LX, 1024>;
        set_fft_smem(kern, sm);
        Launch L(p, "fft_rows_inv");
        launch_dependent(kern, p->ny / rb, nt, sm, p->stream, p->rows.as<C>(), out,
                         corr ? p->sx.as<T>() : p->onesx.as<T>(), corr ? p->sy.as<T>() : p->onesy.as<T>(),
                         p->twx.as<C>(), p->nx, p->ny, rb, alt, (T)scale, out_mode, (const T*)add,
                         (T)add_coef, skip, cg ? *cg : CgFold());
        L.done();
    });
}

void fft_launch_shape(const purify_plan* p, int& rb, int& cb, int& cw) {
    if (p->dtype == PURIFY_F32) {
        rb = plan_rows_per_block<float>(p);
        cb = plan_cols_per_block<float>(p);
        cw = col_lanes<float>(cb, p->fft_cw);
    } else {
        rb = plan_rows_per_block<double>(p);
        cb = plan_cols_per_block<double>(p);
        cw = col_lanes<double>(cb, p->fft_cw);
    }
}

int rows_inv_blocks(purify_plan* p) {
    const int rb = p->dtype == PURIFY_F32 ? plan_rows_per_block<float>(p) : plan_rows_per_block<double>(p);
    return p->ny / rb;
}

void launch_scale_pad_rows(purify_plan* p, const void* x, double scale, const int* skip, bool corr, bool zero_acc,
                           const CgFold* fold) {
    if (p->dtype == PURIFY_F32) rows_fwd_t<float>(p, x, scale, skip, corr, zero_acc, fold);
    else rows_fwd_t<double>(p, x, scale, skip, corr, zero_acc, fold);
}
void launch_cols_fwd(purify_plan* p, const int* skip) {
    if (p->dtype == PURIFY_F32) cols_fwd_t<float>(p, skip); else cols_fwd_t<double>(p, skip);
}
void launch_cols_inv(purify_plan* p, const int* skip, const void* mult) {
    if (p->dtype == PURIFY_F32) cols_inv_t<float>(p, skip, mult); else cols_inv_t<double>(p, skip, mult);
}
void launch_rows_inv_crop(purify_plan* p, void* out, double scale, int out_mode, const void* add, double add_coef,
                          const int* skip, const CgFold* cg, bool corr) {
    if (p->dtype == PURIFY_F32) rows_inv_t<float>(p, out, scale, out_mode, add, add_coef, skip, cg, corr);
    else rows_inv_t<double>(p, out, scale, out_mode, add, add_coef, skip, cg, corr);
}

template <typename T, bool INV> static void fft2_dir(purify_plan* p, void* grid) {
    using C = typename cplx_of<T>::type;
    const int rb = rows_per_block<T>(p->Ky, p->Kx);
    const int cb = cols_per_block<T>(p->Ky, p->Kx);
    const int ar = fft_alt(rb, p->Kx, sizeof(C)), ac = fft_alt(cb, p->Ky, sizeof(C));
    const size_t smr = fft_smem(rb, p->Kx, sizeof(C), ar), smc = fft_smem(cb, p->Ky, sizeof(C), ac);
    const int wc = col_lanes<T>(cb, 0);
    with_log2(p->Kx, [&](auto lg) {
        auto kern = k_rows_full<T, decltype(lg)::value, INV>;
        set_fft_smem(kern, smr);
        Launch L(p, "fft_full_rows");
        kern<<<p->Ky / rb, rb * (p->Kx / 8), smr, p->stream>>>((C*)grid, p->twx.as<C>(), rb, ar);
        L.done();
    });
    with_log2(p->Ky, [&](auto lg) {
        constexpr int LY = decltype(lg)::value;
        auto kern = k_cols_full<T, LY, INV, 1>;
        if constexpr (sizeof(T) == 4) { if (wc == 2) kern = k_cols_full<T, LY, INV, 2>; }
        set_fft_smem(kern, smc);
        Launch L(p, "fft_full_cols");
        kern<<<p->Kx / cb, cb / wc * (p->Ky / 8), smc, p->stream>>>((C*)grid, p->twy.as<C>(), p->Kx, cb, ac);
        L.done();
    });
}

void launch_fft2(purify_plan* p, void* grid, bool inverse) {
    if (p->dtype == PURIFY_F32) {
        if (inverse) fft2_dir<float, true>(p, grid); else fft2_dir<float, false>(p, grid);
    } else {
        if (inverse) fft2_dir<double, true>(p, grid); else fft2_dir<double, false>(p, grid);
    }
}

}  // namespace purify
