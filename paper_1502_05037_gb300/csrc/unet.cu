// Learned warm start: BF16 convolution layers on the fifth-generation tensor
// cores, plus the element-wise kernels of a U-Net (pooling, upsampling,
// masks, loss, Adam).
//
// A 3x3 or 1x1 convolution of an NHWC BF16 image is an implicit GEMM
//   D[pixel][co] = sum over (tap, ci) of A[pixel][(tap, ci)] * W[co][(tap, ci)]
// with M = pixels, N = output channels, K = taps x input channels. A block of
// 128 threads owns 128 consecutive pixels and all N (<= 256) output channels.
// For each K chunk (one tap, up to 64 channels) the threads gather the A rows
// (zero outside the image) and the weight rows into shared memory in the
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix), one
// thread issues tcgen05.mma (M = 128, K = 16 per instruction) accumulating in
// tensor memory, and tcgen05.commit signals an mbarrier before the buffers
// are reused. The epilogue reads the FP32 accumulators with tcgen05.ld, adds
// the bias, applies ReLU and stores BF16 (and/or FP32) results.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "tc.cuh"
#include "unet.h"

namespace purify {

static constexpr int CONV_KC = 64;          // K elements per chunk
static constexpr uint32_t WAIT_LIMIT = 1u << 24;

__global__ void __launch_bounds__(128) k_conv_tc(ConvArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    bf16* sA = reinterpret_cast<bf16*>(smem);                       // 128 x KC
    bf16* sB = sA + 128 * CONV_KC;                                  // Npad x KC
    uint64_t* bar = reinterpret_cast<uint64_t*>(sB + 256 * CONV_KC);
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(bar + 1);
    int* s_fail = reinterpret_cast<int*>(s_taddr + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Npad = a.Npad;
    uint32_t ncols = 32;
    while ((int)ncols < Npad) ncols <<= 1;
    if (warp == 0) {
        tc::tmem_alloc(s_taddr, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        *s_fail = 0;
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *s_taddr;
    const uint32_t idesc = tc::idesc_bf16_f32(128, Npad);

    const int HW = a.H * a.W;
    const int npix = a.B * HW;
    const int q = blockIdx.x * 128 + tid;
    const bool qok = q < npix;
    int pb = 0, py = 0, px = 0;
    if (qok) { pb = q / HW; int rem = q - pb * HW; py = rem / a.W; px = rem - py * a.W; }
    const bool vec_in = (a.in_cs % 8 == 0) && (a.in_co % 8 == 0) && (a.Cin % 8 == 0);
    const int half = a.k / 2;
    uint32_t phase = 0;
    int chunk = 0;
    bool failed = false;
    for (int tap = 0; tap < a.k * a.k && !failed; ++tap) {
        const int dy = tap / a.k - half, dx = tap % a.k - half;
        const int yy = py + dy, xx = px + dx;
        const bool inside = qok && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
        const int sh = a.up ? 1 : 0;
        const int Hs = a.H >> sh, Ws = a.W >> sh;
        const bf16* src =
            inside ? a.in + ((size_t)(pb * Hs + (yy >> sh)) * Ws + (xx >> sh)) * a.in_cs + a.in_co : a.in;
        for (int c0 = 0; c0 < a.Cinp; c0 += CONV_KC) {
            const int kc = min(CONV_KC, a.Cinp - c0);        // multiple of 16
            const int kcu = kc / 8;                           // 16-byte units per row
            // A row `tid`: channels c0 .. c0 + kc of the tap's source pixel
            unsigned char* arow = reinterpret_cast<unsigned char*>(sA) + (size_t)(tid / 8) * kcu * 128 + (tid % 8) * 16;
            for (int j = 0; j < kcu; ++j) {
                uint4 v = make_uint4(0, 0, 0, 0);
                const int cbase = c0 + 8 * j;
                if (inside) {
                    if (vec_in && cbase + 8 <= a.Cin) {
                        v = *reinterpret_cast<const uint4*>(src + cbase);
                    } else if (cbase < a.Cin) {
                        bf16 tmp[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) tmp[e] = (cbase + e < a.Cin) ? src[cbase + e] : __float2bfloat16(0.f);
                        v = *reinterpret_cast<uint4*>(tmp);
                    }
                }
                *reinterpret_cast<uint4*>(arow + j * 128) = v;
            }
            // B rows: weights of every output channel for this chunk
            for (int n = tid; n < Npad; n += 128) {
                const bf16* wsrc = a.w + ((size_t)n * a.k * a.k + tap) * a.Cinp + c0;
                unsigned char* brow = reinterpret_cast<unsigned char*>(sB) + (size_t)(n / 8) * kcu * 128 + (n % 8) * 16;
                for (int j = 0; j < kcu; ++j)
                    *reinterpret_cast<uint4*>(brow + j * 128) = *reinterpret_cast<const uint4*>(wsrc + 8 * j);
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
                for (int s = 0; s < kc / 16; ++s) {
                    uint64_t ad = tc::smem_desc(a0 + s * 256, 128, kcu * 128);
                    uint64_t bd = tc::smem_desc(b0 + s * 256, 128, kcu * 128);
                    tc::mma_bf16(tbase, ad, bd, idesc, (chunk > 0 || s > 0) ? 1u : 0u);
                }
                tc::mma_commit(bar);
            }
            // the shared buffers are reused by the next chunk: wait for the MMAs
            bool done = tc::mbar_wait(bar, phase, WAIT_LIMIT);
            phase ^= 1;
            if (!done) atomicExch(s_fail, 1);
            __syncthreads();
            if (*s_fail) failed = true;
            ++chunk;
            if (failed) break;
        }
    }
    tc::fence_after_sync();
    if (!failed) {
        // epilogue: lane of this warp = accumulator row = pixel q0 + 32*warp + lane
        const int row = warp * 32 + lane;
        const int qo = blockIdx.x * 128 + row;
        for (int c = 0; c < Npad; c += 16) {
            float v[16];
            tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (qo < npix) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int co = c + e;
                    if (co < a.Cout) {
                        float r = v[e] + (a.bias ? a.bias[co] : 0.f);
                        if (a.relu) r = fmaxf(r, 0.f);
                        if (a.out) a.out[(size_t)qo * a.out_cs + a.out_co + co] = __float2bfloat16_rn(r);
                        if (a.out_f32) {
                            size_t o = (size_t)qo * a.Cout + co;
                            a.out_f32[o] = r + (a.residual ? a.residual[o] : 0.f);
                        }
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(a.err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

static size_t conv_smem_bytes() { return sizeof(bf16) * (128 + 256) * CONV_KC + 64; }

void conv_tc_launch(const ConvArgs& a, cudaStream_t st) {
    if (a.Npad < 16 || a.Npad > 256 || a.Npad % 16 || a.Cinp % 16 || (a.k != 1 && a.k != 3))
        throw Error{PURIFY_EINVAL, "conv: unsupported shape"};
    // the shared-memory limit is a per-device setting: raised on the first
    // launch on each device (threads racing on it set the same value)
    static std::atomic<bool> attr[64];
    const size_t sm = conv_smem_bytes();
    int dev = 0;
    PURIFY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{PURIFY_ECUDA, "device index out of range"};
    if (!attr[dev].load(std::memory_order_relaxed)) {
        PURIFY_CUDA(cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr[dev].store(true, std::memory_order_relaxed);
    }
    const int npix = a.B * a.H * a.W;
    k_conv_tc<<<(npix + 127) / 128, 128, sm, st>>>(a);
    PURIFY_CUDA(cudaGetLastError());
    add_launches(1);
}

// ----------------------------------------------------------- conversions
__global__ void k_f32_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// FP32 weights [Cout][k][k][Cin] -> BF16 [Npad][k][k][Cinp], zero padded
__global__ void k_pack_weights(const float* __restrict__ w, bf16* __restrict__ wp, int Cout, int k, int Cin,
                               int Npad, int Cinp) {
    const int64_t n = (int64_t)Npad * k * k * Cinp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int ci = (int)(i % Cinp);
        int64_t r = i / Cinp;
        int tap = (int)(r % (k * k));
        int co = (int)(r / (k * k));
        float v = (co < Cout && ci < Cin) ? w[((int64_t)co * k * k + tap) * Cin + ci] : 0.f;
        wp[i] = __float2bfloat16_rn(v);
    }
}

int round16(int v) { return (v + 15) / 16 * 16; }

// Convolution of FP32 NHWC input through BF16 tensor cores (test and
// inference entry; allocates its staging buffers).
void conv2d_f32(const float* x, int B, int H, int W, int Cin, const float* w, const float* bias, int Cout, int k,
                int relu, float* out, cudaStream_t st) {
    const int Cinp = round16(Cin), Npad = std::max(16, round16(Cout));
    DevBuf xb, wb, err;
    xb.alloc(sizeof(bf16) * (size_t)B * H * W * Cin);
    wb.alloc(sizeof(bf16) * (size_t)Npad * k * k * Cinp);
    err.alloc(sizeof(int));
    PURIFY_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    const int64_t nx = (int64_t)B * H * W * Cin;
    k_f32_to_bf16<<<(int)std::min<int64_t>(4096, (nx + 255) / 256), 256, 0, st>>>(x, xb.as<bf16>(), nx);
    k_pack_weights<<<256, 256, 0, st>>>(w, wb.as<bf16>(), Cout, k, Cin, Npad, Cinp);
    PURIFY_CUDA(cudaGetLastError());
    add_launches(2);
    ConvArgs a{};
    a.in = xb.as<bf16>();
    a.B = B; a.H = H; a.W = W; a.Cin = Cin; a.in_cs = Cin; a.in_co = 0;
    a.w = wb.as<bf16>(); a.k = k; a.Cinp = Cinp; a.Npad = Npad;
    a.bias = bias; a.Cout = Cout; a.relu = relu;
    a.out = nullptr; a.out_f32 = out; a.residual = nullptr;
    a.err = err.as<int>();
    conv_tc_launch(a, st);
    int herr = 0;
    PURIFY_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PURIFY_CUDA(cudaStreamSynchronize(st));
    if (herr) throw Error{PURIFY_ETIMEOUT, "tensor-core convolution: a bounded wait gave up"};
}

}  // namespace purify
