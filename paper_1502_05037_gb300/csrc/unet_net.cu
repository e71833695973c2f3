// Learned warm start: the U-Net driver (forward, backward, Adam) on top of
// the tensor-core convolution of unet.cu. The network is not in the paper: it
// maps a normalised dirty image to a starting point for SDMM, which leaves the
// convex problem (3) and its solution unchanged.
//
// Layout NHWC; activations BF16 (the tensor-core operands), gradients and
// parameters FP32. Architecture (L levels, base width c):
//   encoder l < L-1: conv3x3+ReLU, conv3x3+ReLU (kept as the skip), maxpool 2x2
//   bottom:          conv3x3+ReLU, conv3x3+ReLU
//   decoder l:       x2 upsampling fused into conv3x3+ReLU (2c -> c), concat with
//                    the skip (channel offsets of one buffer), conv3x3+ReLU x 2
//   head:            conv1x1 (c -> 1) plus the input (residual), FP32.
// Backward: input gradients are convolutions with the flipped, transposed
// weights on the tensor cores; weight gradients are FP32 CUDA-core sums.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"
#include "reduce.cuh"
#include "unet.h"

namespace purify {

// ------------------------------------------------------------ small kernels
static inline int eblocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192)); }

__global__ void k_maxpool_fwd(const bf16* __restrict__ in, int cs, int co, bf16* __restrict__ out, int B, int H, int W,
                              int C) {
    const int Ho = H / 2, Wo = W / 2;
    const int64_t n = (int64_t)B * Ho * Wo * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int c = (int)(i % C);
        int64_t r = i / C;
        int x = (int)(r % Wo);
        r /= Wo;
        int y = (int)(r % Ho);
        int b = (int)(r / Ho);
        const bf16* p = in + ((size_t)(b * H + 2 * y) * W + 2 * x) * cs + co + c;
        float m = __bfloat162float(p[0]);
        m = fmaxf(m, __bfloat162float(p[cs]));
        m = fmaxf(m, __bfloat162float(p[(size_t)W * cs]));
        m = fmaxf(m, __bfloat162float(p[(size_t)W * cs + cs]));
        out[i] = __float2bfloat16_rn(m);
    }
}

// gin[b][y][x][c] = (first maximum of its 2x2 window, row-major) ? gout : 0,
// plus gadd (stride as, offset ao) when given.
__global__ void k_maxpool_bwd(const bf16* __restrict__ in, int cs, int co, const float* __restrict__ gout,
                              const float* __restrict__ gadd, int as, int ao, float* __restrict__ gin, int B, int H,
                              int W, int C) {
    const int Ho = H / 2, Wo = W / 2;
    const int64_t n = (int64_t)B * Ho * Wo * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int c = (int)(i % C);
        int64_t r = i / C;
        int x = (int)(r % Wo);
        r /= Wo;
        int y = (int)(r % Ho);
        int b = (int)(r / Ho);
        size_t base = (size_t)(b * H + 2 * y) * W + 2 * x;
        size_t pix[4] = {base, base + 1, base + W, base + W + 1};
        float best = -INFINITY;
        int arg = 0;
        for (int k = 0; k < 4; ++k) {
            float v = __bfloat162float(in[pix[k] * cs + co + c]);
            if (v > best) { best = v; arg = k; }
        }
        float g = gout[i];
        for (int k = 0; k < 4; ++k) {
            float v = (k == arg) ? g : 0.f;
            if (gadd) v += gadd[pix[k] * as + ao + c];
            gin[pix[k] * C + c] = v;
        }
    }
}

// gz = (act > 0) ? g : 0 as BF16 [P][C]; g has stride gs/offset go, act stride as/offset ao
__global__ void k_relu_grad(const float* __restrict__ g, int gs, int go, const bf16* __restrict__ act, int as, int ao,
                            bf16* __restrict__ gz, int64_t P, int C) {
    const int64_t n = P * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int c = (int)(i % C);
        int64_t p = i / C;
        float a = __bfloat162float(act[p * as + ao + c]);
        gz[i] = __float2bfloat16_rn(a > 0.f ? g[p * gs + go + c] : 0.f);
    }
}

// g_lo[b][y][x][c] = sum of the 2x2 block of g_hi
__global__ void k_upsample_bwd(const float* __restrict__ ghi, float* __restrict__ glo, int B, int H, int W, int C) {
    const int Ho = H / 2, Wo = W / 2;
    const int64_t n = (int64_t)B * Ho * Wo * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int c = (int)(i % C);
        int64_t r = i / C;
        int x = (int)(r % Wo);
        r /= Wo;
        int y = (int)(r % Ho);
        int b = (int)(r / Ho);
        size_t base = (size_t)(b * H + 2 * y) * W + 2 * x;
        glo[i] = ghi[base * C + c] + ghi[(base + 1) * C + c] + ghi[(base + W) * C + c] + ghi[(base + W + 1) * C + c];
    }
}

// Weight gradients of a k x k convolution on the CUDA cores, one tap per
// block row of the grid:
//   dW[co][tap][ci] += sum_p gz[p][co] * x[p + tap][ci]
// a register-tiled GEMM (64 x 64 output tile, 4 x 4 per thread, K = 16
// pixels per shared-memory stage) over a chunk of pixels, added to dW with
// one atomic per output and block.
__global__ void __launch_bounds__(256) k_dw(const bf16* __restrict__ gz, int Cout, const bf16* __restrict__ x, int xcs,
                                            int xco, int Cin, int B, int H, int W, int up, int k, int pch,
                                            float* __restrict__ dW) {
    constexpr int BK = 16;
    __shared__ __align__(16) float gs[BK][64];
    __shared__ __align__(16) float xs[BK][64];
    const int co0 = blockIdx.x * 64, ci0 = blockIdx.y * 64;
    const int tap = blockIdx.z % (k * k), chunk = blockIdx.z / (k * k);
    const int dy = tap / k - k / 2, dx = tap % k - k / 2;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int64_t P = (int64_t)B * H * W;
    const int64_t p0 = (int64_t)chunk * pch, p1 = min(P, p0 + pch);
    const int sh = up ? 1 : 0;
    const int Hs = H >> sh, Ws = W >> sh;
    float acc[4][4] = {};
    const int lk = tid / 16, lj = (tid % 16) * 4;   // this thread's loads: row lk, columns lj..lj+3
    for (int64_t pb = p0; pb < p1; pb += BK) {
        const int64_t p = pb + lk;
        float gv[4] = {0, 0, 0, 0}, xv[4] = {0, 0, 0, 0};
        if (p < p1) {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (co0 + lj + e < Cout) gv[e] = __bfloat162float(gz[p * Cout + co0 + lj + e]);
            const int b = (int)(p / (H * W));
            const int rem = (int)(p - (int64_t)b * H * W);
            const int yy = rem / W + dy, xx = rem % W + dx;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                const bf16* src = x + ((size_t)(b * Hs + (yy >> sh)) * Ws + (xx >> sh)) * xcs + xco + ci0 + lj;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (ci0 + lj + e < Cin) xv[e] = __bfloat162float(src[e]);
            }
        }
        *reinterpret_cast<float4*>(&gs[lk][lj]) = make_float4(gv[0], gv[1], gv[2], gv[3]);
        *reinterpret_cast<float4*>(&xs[lk][lj]) = make_float4(xv[0], xv[1], xv[2], xv[3]);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float4 a = *reinterpret_cast<const float4*>(&gs[kk][ty * 4]);
            float4 c = *reinterpret_cast<const float4*>(&xs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * cv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int co = co0 + ty * 4 + i;
        if (co >= Cout) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ci = ci0 + tx * 4 + j;
            if (ci < Cin) atomicAdd(&dW[((size_t)co * k * k + tap) * Cin + ci], acc[i][j]);
        }
    }
}

// db[co] += sum over a chunk of pixels of gz[p][co]
__global__ void k_db(const bf16* __restrict__ gz, int Cout, int64_t P, int pch, float* __restrict__ db) {
    const int64_t p0 = (int64_t)blockIdx.x * pch, p1 = min(P, p0 + pch);
    for (int co = threadIdx.x; co < Cout; co += blockDim.x) {
        float s = 0.f;
        for (int64_t p = p0; p < p1; ++p) s += __bfloat162float(gz[p * Cout + co]);
        atomicAdd(&db[co], s);
    }
}

// FP32 weights [Cout][k][k][Cin] -> flipped, transposed BF16 [Nb][k][k][Cb]:
// W'[ci][ky][kx][co] = W[co][k-1-ky][k-1-kx][ci] (zero padded)
__global__ void k_pack_weights_bwd(const float* __restrict__ w, bf16* __restrict__ wp, int Cout, int k, int Cin, int Nb,
                                   int Cb) {
    const int64_t n = (int64_t)Nb * k * k * Cb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int co = (int)(i % Cb);
        int64_t r = i / Cb;
        int tap = (int)(r % (k * k));
        int ci = (int)(r / (k * k));
        int ky = tap / k, kx = tap % k;
        int ftap = (k - 1 - ky) * k + (k - 1 - kx);
        float v = (ci < Cin && co < Cout) ? w[((int64_t)co * k * k + ftap) * Cin + ci] : 0.f;
        wp[i] = __float2bfloat16_rn(v);
    }
}

// loss = mean (pred - t)^2, g = 2 (pred - t) / n; loss to scal[0] (FP64, fixed order)
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ t, float* __restrict__ g, int64_t n,
                      double* part, unsigned* counter, double* out) {
    float acc = 0.f;
    const float s = 2.f / (float)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float d = pred[i] - t[i];
        acc += d * d;
        g[i] = s * d;
    }
    double b = block_sum((double)acc);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
    if (arrive_last(counter)) {
        double tot = ordered_sum(part, gridDim.x);
        if (threadIdx.x == 0) {
            *out = tot / (double)n;
            *counter = 0;
        }
    }
}

// Adam (Kingma & Ba 2015) with bias correction
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ------------------------------------------------------------------ network
struct UnetLayer {
    std::string name;
    int cout, k, cin;
    int64_t woff, boff;      // into the flat parameter vector
    int Npad, Cinp, Nb, Cb;  // packed forward / backward weight shapes
    DevBuf wf, wb;           // packed BF16 weights
};

struct Unet {
    int H, W, L, base, maxB;
    cudaStream_t st;
    std::vector<UnetLayer> layers;
    int64_t nparams = 0;
    int64_t step = 0;
    DevBuf params, grads, m, v;
    // activations (BF16)
    DevBuf xbf;                                 // [B][H][W][1]
    std::vector<DevBuf> a, cat, pool, da, dbb;  // per level
    DevBuf bA, bB;
    DevBuf pred;                                // FP32 [B][H][W]
    // gradients (FP32) and BF16 staging
    std::vector<DevBuf> gcat;
    DevBuf g1, g2, gz, gpred;
    DevBuf red_part, red_ctr, loss, err;
    int ch(int l) const { return base << l; }
    int64_t pix(int l, int B) const { return (int64_t)B * (H >> l) * (W >> l); }
    UnetLayer& layer(const std::string& n) {
        for (auto& x : layers) if (x.name == n) return x;
        throw Error{PURIFY_EINVAL, "unknown layer " + n};
    }
};

static void build_layers(Unet& u) {
    int cin = 1;
    auto add = [&](const std::string& n, int cout, int k, int ci) {
        UnetLayer l;
        l.name = n;
        l.cout = cout;
        l.k = k;
        l.cin = ci;
        l.woff = u.nparams;
        u.nparams += (int64_t)cout * k * k * ci;
        l.boff = u.nparams;
        u.nparams += cout;
        l.Npad = std::max(16, round16(cout));
        l.Cinp = round16(ci);
        l.Nb = std::max(16, round16(ci));
        l.Cb = round16(cout);
        u.layers.push_back(std::move(l));
    };
    for (int l = 0; l < u.L - 1; ++l) {
        int c = u.ch(l);
        add("e" + std::to_string(l) + "a", c, 3, cin);
        add("e" + std::to_string(l) + "b", c, 3, c);
        cin = c;
    }
    int cb = u.ch(u.L - 1);
    add("ba", cb, 3, cin);
    add("bb", cb, 3, cb);
    for (int l = u.L - 2; l >= 0; --l) {
        int c = u.ch(l);
        add("d" + std::to_string(l) + "u", c, 3, 2 * c);
        add("d" + std::to_string(l) + "a", c, 3, 2 * c);
        add("d" + std::to_string(l) + "b", c, 3, c);
    }
    add("head", 1, 1, u.base);
}

static void pack_all(Unet& u) {
    const float* P = u.params.as<float>();
    for (auto& l : u.layers) {
        int64_t nf = (int64_t)l.Npad * l.k * l.k * l.Cinp, nb = (int64_t)l.Nb * l.k * l.k * l.Cb;
        k_pack_weights<<<eblocks(nf), 256, 0, u.st>>>(P + l.woff, l.wf.as<bf16>(), l.cout, l.k, l.cin, l.Npad, l.Cinp);
        k_pack_weights_bwd<<<eblocks(nb), 256, 0, u.st>>>(P + l.woff, l.wb.as<bf16>(), l.cout, l.k, l.cin, l.Nb, l.Cb);
    }
    PURIFY_CUDA(cudaGetLastError());
    add_launches(2 * (int64_t)u.layers.size());
}

Unet* unet_create(int H, int W, int L, int base, int maxB, uint64_t seed, cudaStream_t st) {
    PURIFY_REQUIRE(L >= 2 && L <= 6 && base >= 8 && base % 8 == 0 && (base << (L - 1)) <= 256,
                   "unet: levels in [2, 6], base multiple of 8 with base * 2^(levels-1) <= 256");
    PURIFY_REQUIRE(H % (1 << (L - 1)) == 0 && W % (1 << (L - 1)) == 0 && H >= 8 && W >= 8,
                   "unet: H and W must be divisible by 2^(levels-1)");
    PURIFY_REQUIRE(maxB >= 1, "unet: max batch >= 1");
    Unet* u = new Unet();
    try {
        u->H = H; u->W = W; u->L = L; u->base = base; u->maxB = maxB; u->st = st;
        build_layers(*u);
        // He-normal initial weights from a seeded generator, zero biases
        std::vector<float> p(u->nparams, 0.f);
        uint64_t s = seed * 0x9E3779B97F4A7C15ull + 1;
        auto uni = [&]() {
            s ^= s << 13; s ^= s >> 7; s ^= s << 17;
            return ((double)(s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        };
        for (auto& l : u->layers) {
            double stdv = std::sqrt(2.0 / (l.k * l.k * l.cin));
            int64_t nw = (int64_t)l.cout * l.k * l.k * l.cin;
            for (int64_t i = 0; i < nw; ++i) {
                double r1 = uni(), r2 = uni();
                p[l.woff + i] = (float)(stdv * std::sqrt(-2.0 * std::log(r1)) * std::cos(6.283185307179586 * r2));
            }
            l.wf.alloc(sizeof(bf16) * (size_t)l.Npad * l.k * l.k * l.Cinp);
            l.wb.alloc(sizeof(bf16) * (size_t)l.Nb * l.k * l.k * l.Cb);
        }
        u->params.alloc(sizeof(float) * u->nparams);
        u->grads.alloc(sizeof(float) * u->nparams);
        u->m.alloc(sizeof(float) * u->nparams);
        u->v.alloc(sizeof(float) * u->nparams);
        PURIFY_CUDA(cudaMemcpy(u->params.p, p.data(), sizeof(float) * u->nparams, cudaMemcpyHostToDevice));
        PURIFY_CUDA(cudaMemset(u->m.p, 0, u->m.bytes));
        PURIFY_CUDA(cudaMemset(u->v.p, 0, u->v.bytes));
        // buffers
        u->xbf.alloc(sizeof(bf16) * u->pix(0, maxB));
        u->a.resize(L); u->cat.resize(L); u->pool.resize(L); u->da.resize(L); u->dbb.resize(L); u->gcat.resize(L);
        for (int l = 0; l < L - 1; ++l) {
            int64_t P = u->pix(l, maxB);
            int c = u->ch(l);
            u->a[l].alloc(sizeof(bf16) * P * c);
            u->cat[l].alloc(sizeof(bf16) * P * 2 * c);
            u->pool[l].alloc(sizeof(bf16) * u->pix(l + 1, maxB) * c);
            u->da[l].alloc(sizeof(bf16) * P * c);
            u->dbb[l].alloc(sizeof(bf16) * P * c);
            u->gcat[l].alloc(sizeof(float) * P * 2 * c);
        }
        int64_t Pb = u->pix(L - 1, maxB);
        u->bA.alloc(sizeof(bf16) * Pb * u->ch(L - 1));
        u->bB.alloc(sizeof(bf16) * Pb * u->ch(L - 1));
        u->pred.alloc(sizeof(float) * u->pix(0, maxB));
        int64_t gmax = 0;
        for (int l = 0; l < L; ++l) gmax = std::max(gmax, u->pix(l, maxB) * 2 * u->ch(l));
        u->g1.alloc(sizeof(float) * gmax);
        u->g2.alloc(sizeof(float) * gmax);
        u->gz.alloc(sizeof(bf16) * gmax);
        u->gpred.alloc(sizeof(float) * u->pix(0, maxB));
        u->red_part.alloc(sizeof(double) * 8192);
        u->red_ctr.alloc(sizeof(unsigned) * 4);
        u->loss.alloc(sizeof(double));
        u->err.alloc(sizeof(int));
        PURIFY_CUDA(cudaMemset(u->red_ctr.p, 0, u->red_ctr.bytes));
        PURIFY_CUDA(cudaMemset(u->err.p, 0, sizeof(int)));
        pack_all(*u);
        PURIFY_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        delete u;
        throw;
    }
    return u;
}

void unet_destroy(Unet* u) {
    if (!u) return;
    cudaStreamSynchronize(u->st);
    delete u;
}

static ConvArgs conv_args(Unet& u, UnetLayer& l, bool backward) {
    ConvArgs a{};
    a.k = l.k;
    if (!backward) {
        a.w = l.wf.as<bf16>(); a.Cinp = l.Cinp; a.Npad = l.Npad; a.Cout = l.cout; a.Cin = l.cin;
        a.bias = u.params.as<float>() + l.boff;
    } else {
        a.w = l.wb.as<bf16>(); a.Cinp = l.Cb; a.Npad = l.Nb; a.Cout = l.cin; a.Cin = l.cout;
        a.bias = nullptr;
    }
    a.err = u.err.as<int>();
    return a;
}

// conv layer forward: input (buffer, channel stride, offset, resolution level, upsample) -> BF16 output slice
static void fwd_conv(Unet& u, const std::string& name, int B, const bf16* in, int in_cs, int in_co, int lev, int up,
                     bf16* out, int out_cs, int out_co) {
    UnetLayer& l = u.layer(name);
    ConvArgs a = conv_args(u, l, false);
    a.in = in; a.in_cs = in_cs; a.in_co = in_co; a.up = up;
    a.B = B; a.H = u.H >> lev; a.W = u.W >> lev;
    a.relu = 1;
    a.out = out; a.out_cs = out_cs; a.out_co = out_co;
    conv_tc_launch(a, u.st);
}

void unet_forward(Unet& u, const float* x, int B, float* out) {
    const int L = u.L;
    const int64_t P0 = u.pix(0, B);
    k_f32_to_bf16<<<eblocks(P0), 256, 0, u.st>>>(x, u.xbf.as<bf16>(), P0);
    add_launches(1);
    const bf16* in = u.xbf.as<bf16>();
    int in_cs = 1;
    for (int l = 0; l < L - 1; ++l) {
        int c = u.ch(l);
        std::string s = std::to_string(l);
        fwd_conv(u, "e" + s + "a", B, in, in_cs, 0, l, 0, u.a[l].as<bf16>(), c, 0);
        fwd_conv(u, "e" + s + "b", B, u.a[l].as<bf16>(), c, 0, l, 0, u.cat[l].as<bf16>(), 2 * c, 0);
        int64_t n = u.pix(l + 1, B) * c;
        k_maxpool_fwd<<<eblocks(n), 256, 0, u.st>>>(u.cat[l].as<bf16>(), 2 * c, 0, u.pool[l].as<bf16>(), B, u.H >> l,
                                                   u.W >> l, c);
        add_launches(1);
        in = u.pool[l].as<bf16>();
        in_cs = c;
    }
    int cb = u.ch(L - 1);
    fwd_conv(u, "ba", B, in, in_cs, 0, L - 1, 0, u.bA.as<bf16>(), cb, 0);
    fwd_conv(u, "bb", B, u.bA.as<bf16>(), cb, 0, L - 1, 0, u.bB.as<bf16>(), cb, 0);
    const bf16* low = u.bB.as<bf16>();
    for (int l = L - 2; l >= 0; --l) {
        int c = u.ch(l);
        std::string s = std::to_string(l);
        fwd_conv(u, "d" + s + "u", B, low, 2 * c, 0, l, 1, u.cat[l].as<bf16>(), 2 * c, c);
        fwd_conv(u, "d" + s + "a", B, u.cat[l].as<bf16>(), 2 * c, 0, l, 0, u.da[l].as<bf16>(), c, 0);
        fwd_conv(u, "d" + s + "b", B, u.da[l].as<bf16>(), c, 0, l, 0, u.dbb[l].as<bf16>(), c, 0);
        low = u.dbb[l].as<bf16>();
    }
    UnetLayer& h = u.layer("head");
    ConvArgs a = conv_args(u, h, false);
    a.in = u.dbb[0].as<bf16>(); a.in_cs = u.base; a.in_co = 0; a.up = 0;
    a.B = B; a.H = u.H; a.W = u.W; a.relu = 0;
    a.out = nullptr; a.out_f32 = out ? out : u.pred.as<float>(); a.residual = x;
    conv_tc_launch(a, u.st);
}

// input gradient of a conv layer: gz (BF16 [P][cout]) -> g_out FP32 [P][cin] at level lev
static void bwd_dx(Unet& u, UnetLayer& l, int B, int lev, const bf16* gz, float* gout) {
    ConvArgs a = conv_args(u, l, true);
    a.in = gz; a.in_cs = l.cout; a.in_co = 0; a.up = 0;
    a.B = B; a.H = u.H >> lev; a.W = u.W >> lev; a.relu = 0;
    a.out = nullptr; a.out_f32 = gout; a.residual = nullptr;
    conv_tc_launch(a, u.st);
}

static void bwd_dw(Unet& u, UnetLayer& l, int B, int lev, const bf16* gz, const bf16* x, int xcs, int xco, int up) {
    const int H = u.H >> lev, W = u.W >> lev;
    const int64_t P = (int64_t)B * H * W;
    // pixel chunk per block: about 8 blocks per SM over all taps and tiles
    const int tiles = ((l.cout + 63) / 64) * ((l.cin + 63) / 64) * l.k * l.k;
    int64_t want = std::max<int64_t>(1, (152 * 8) / tiles);
    int pch = (int)std::max<int64_t>(256, (P + want - 1) / want);
    pch = (pch + 15) / 16 * 16;
    const int nchunk = (int)((P + pch - 1) / pch);
    dim3 g((l.cout + 63) / 64, (l.cin + 63) / 64, l.k * l.k * nchunk);
    k_dw<<<g, 256, 0, u.st>>>(gz, l.cout, x, xcs, xco, l.cin, B, H, W, up, l.k, pch, u.grads.as<float>() + l.woff);
    const int dch = 1024;
    k_db<<<(int)((P + dch - 1) / dch), 64, 0, u.st>>>(gz, l.cout, P, dch, u.grads.as<float>() + l.boff);
    PURIFY_CUDA(cudaGetLastError());
    add_launches(2);
}

static void relu_grad(Unet& u, const float* g, int gs, int go, const bf16* act, int as, int ao, int64_t P, int C) {
    k_relu_grad<<<eblocks(P * C), 256, 0, u.st>>>(g, gs, go, act, as, ao, u.gz.as<bf16>(), P, C);
    add_launches(1);
}

// forward + backward; gradients in u.grads, loss in u.loss (device)
void unet_gradients(Unet& u, const float* x, const float* target, int B) {
    PURIFY_REQUIRE(B >= 1 && B <= u.maxB, "unet: batch larger than the network was created for");
    const int L = u.L;
    unet_forward(u, x, B, nullptr);
    PURIFY_CUDA(cudaMemsetAsync(u.grads.p, 0, u.grads.bytes, u.st));
    const int64_t P0 = u.pix(0, B);
    k_mse<<<256, 256, 0, u.st>>>(u.pred.as<float>(), target, u.gpred.as<float>(), P0, u.red_part.as<double>(),
                                 u.red_ctr.as<unsigned>(), u.loss.as<double>());
    add_launches(1);
    // head (1x1, no ReLU): gz = gpred
    k_f32_to_bf16<<<eblocks(P0), 256, 0, u.st>>>(u.gpred.as<float>(), u.gz.as<bf16>(), P0);
    add_launches(1);
    UnetLayer& head = u.layer("head");
    bwd_dw(u, head, B, 0, u.gz.as<bf16>(), u.dbb[0].as<bf16>(), u.base, 0, 0);
    bwd_dx(u, head, B, 0, u.gz.as<bf16>(), u.g1.as<float>());
    float* g = u.g1.as<float>();   // gradient w.r.t. the current layer's output
    float* t = u.g2.as<float>();
    for (int l = 0; l < L - 1; ++l) {
        const int c = u.ch(l);
        const int64_t P = u.pix(l, B);
        std::string s = std::to_string(l);
        UnetLayer& lb = u.layer("d" + s + "b");
        relu_grad(u, g, c, 0, u.dbb[l].as<bf16>(), c, 0, P, c);
        bwd_dw(u, lb, B, l, u.gz.as<bf16>(), u.da[l].as<bf16>(), c, 0, 0);
        bwd_dx(u, lb, B, l, u.gz.as<bf16>(), t);
        std::swap(g, t);
        UnetLayer& la = u.layer("d" + s + "a");
        relu_grad(u, g, c, 0, u.da[l].as<bf16>(), c, 0, P, c);
        bwd_dw(u, la, B, l, u.gz.as<bf16>(), u.cat[l].as<bf16>(), 2 * c, 0, 0);
        bwd_dx(u, la, B, l, u.gz.as<bf16>(), u.gcat[l].as<float>());
        // up branch: channels [c, 2c) of the concat
        UnetLayer& lu = u.layer("d" + s + "u");
        relu_grad(u, u.gcat[l].as<float>(), 2 * c, c, u.cat[l].as<bf16>(), 2 * c, c, P, c);
        const bf16* low = (l == L - 2) ? u.bB.as<bf16>() : u.dbb[l + 1].as<bf16>();
        bwd_dw(u, lu, B, l, u.gz.as<bf16>(), low, 2 * c, 0, 1);
        bwd_dx(u, lu, B, l, u.gz.as<bf16>(), t);   // [P][2c] at level l
        int64_t nlo = u.pix(l + 1, B) * 2 * c;
        k_upsample_bwd<<<eblocks(nlo), 256, 0, u.st>>>(t, g, B, u.H >> l, u.W >> l, 2 * c);
        add_launches(1);
        // g now holds the gradient of the level-(l+1) decoder output (or the bottom)
    }
    const int cb = u.ch(L - 1);
    const int64_t Pb = u.pix(L - 1, B);
    UnetLayer& lbb = u.layer("bb");
    relu_grad(u, g, cb, 0, u.bB.as<bf16>(), cb, 0, Pb, cb);
    bwd_dw(u, lbb, B, L - 1, u.gz.as<bf16>(), u.bA.as<bf16>(), cb, 0, 0);
    bwd_dx(u, lbb, B, L - 1, u.gz.as<bf16>(), t);
    std::swap(g, t);
    UnetLayer& lba = u.layer("ba");
    relu_grad(u, g, cb, 0, u.bA.as<bf16>(), cb, 0, Pb, cb);
    bwd_dw(u, lba, B, L - 1, u.gz.as<bf16>(), u.pool[L - 2].as<bf16>(), u.ch(L - 2), 0, 0);
    bwd_dx(u, lba, B, L - 1, u.gz.as<bf16>(), t);   // gradient of pool[L-2]
    std::swap(g, t);
    for (int l = L - 2; l >= 0; --l) {
        const int c = u.ch(l);
        const int64_t P = u.pix(l, B);
        std::string s = std::to_string(l);
        // through the max pooling, plus the skip gradient (channels [0, c) of gcat)
        int64_t npool = u.pix(l + 1, B) * c;
        k_maxpool_bwd<<<eblocks(npool), 256, 0, u.st>>>(u.cat[l].as<bf16>(), 2 * c, 0, g, u.gcat[l].as<float>(), 2 * c,
                                                        0, t, B, u.H >> l, u.W >> l, c);
        add_launches(1);
        std::swap(g, t);
        UnetLayer& lb = u.layer("e" + s + "b");
        relu_grad(u, g, c, 0, u.cat[l].as<bf16>(), 2 * c, 0, P, c);
        bwd_dw(u, lb, B, l, u.gz.as<bf16>(), u.a[l].as<bf16>(), c, 0, 0);
        bwd_dx(u, lb, B, l, u.gz.as<bf16>(), t);
        std::swap(g, t);
        UnetLayer& la = u.layer("e" + s + "a");
        relu_grad(u, g, c, 0, u.a[l].as<bf16>(), c, 0, P, c);
        const bf16* xin = l == 0 ? u.xbf.as<bf16>() : u.pool[l - 1].as<bf16>();
        const int xcs = l == 0 ? 1 : u.ch(l - 1);
        bwd_dw(u, la, B, l, u.gz.as<bf16>(), xin, xcs, 0, 0);
        if (l > 0) {
            bwd_dx(u, la, B, l, u.gz.as<bf16>(), t);
            std::swap(g, t);
        }
    }
}

double unet_read_loss(Unet& u) {
    double v = 0;
    PURIFY_CUDA(cudaMemcpyAsync(&v, u.loss.p, sizeof(double), cudaMemcpyDeviceToHost, u.st));
    int e = 0;
    PURIFY_CUDA(cudaMemcpyAsync(&e, u.err.p, sizeof(int), cudaMemcpyDeviceToHost, u.st));
    PURIFY_CUDA(cudaStreamSynchronize(u.st));
    if (e) throw Error{PURIFY_ETIMEOUT, "tensor-core convolution: a bounded wait gave up"};
    return v;
}

void unet_adam(Unet& u, float lr) {
    u.step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)u.step), c2 = 1.f - std::pow(b2, (float)u.step);
    k_adam<<<eblocks(u.nparams), 256, 0, u.st>>>(u.params.as<float>(), u.grads.as<float>(), u.m.as<float>(),
                                                 u.v.as<float>(), u.nparams, lr, b1, b2, 1e-8f, c1, c2);
    add_launches(1);
    pack_all(u);
}

void unet_set_params(Unet& u, const float* p) {
    PURIFY_CUDA(cudaMemcpyAsync(u.params.p, p, sizeof(float) * u.nparams, cudaMemcpyDefault, u.st));
    pack_all(u);
    PURIFY_CUDA(cudaStreamSynchronize(u.st));
}

void unet_get(Unet& u, int what, float* out) {
    const DevBuf& b = what == 0 ? u.params : u.grads;
    PURIFY_CUDA(cudaMemcpyAsync(out, b.p, sizeof(float) * u.nparams, cudaMemcpyDefault, u.st));
    PURIFY_CUDA(cudaStreamSynchronize(u.st));
}

int64_t unet_nparams(Unet& u) { return u.nparams; }

}  // namespace purify
