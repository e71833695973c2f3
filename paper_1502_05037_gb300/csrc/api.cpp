// C ABI of the imaging library (include/purify.h): argument checks, host
// pointer staging, error translation, launch accounting and timing.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "internal.h"
#include "launch.h"

namespace purify {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void set_error(const std::string& msg) { g_last_error = msg; }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct KernelTimer {
    bool enabled = false;
    struct Pending { std::string name; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<int64_t, double>> acc;
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e;
        PURIFY_CUDA(cudaEventCreate(&e));
        return e;
    }
    void drain() {
        for (auto& q : pending) {
            float ms = 0.f;
            PURIFY_CUDA(cudaEventSynchronize(q.b));
            PURIFY_CUDA(cudaEventElapsedTime(&ms, q.a, q.b));
            auto& a = acc[q.name];
            a.first += 1;
            a.second += ms;
            pool.push_back(q.a);
            pool.push_back(q.b);
        }
        pending.clear();
    }
    ~KernelTimer() {
        for (auto& q : pending) { cudaEventDestroy(q.a); cudaEventDestroy(q.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

bool timing_enabled(const purify_plan* p) { return p->timer && p->timer->enabled; }

Launch::Launch(purify_plan* plan, const char* kname) : p(plan), name(kname) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (p->timer && p->timer->enabled) {
        e0 = p->timer->get();
        PURIFY_CUDA(cudaEventRecord(e0, p->stream));
    }
}

void Launch::done() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error{PURIFY_ECUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e)};
    if (e0) {
        cudaEvent_t e1 = p->timer->get();
        PURIFY_CUDA(cudaEventRecord(e1, p->stream));
        p->timer->pending.push_back({name, e0, e1});
        if (p->timer->pending.size() > 4096) p->timer->drain();
        e0 = nullptr;
    }
}

// Device view of a caller array: the pointer itself, or a staged copy.
struct Staged {
    void* dev = nullptr;
    bool host = false;
};

static Staged stage_in(purify_plan* p, const void* ptr, size_t bytes, DevBuf& buf) {
    Staged s;
    if (!is_host_pointer(ptr)) { s.dev = const_cast<void*>(ptr); return s; }
    if (buf.bytes < bytes) buf.alloc(bytes);
    PURIFY_CUDA(cudaMemcpyAsync(buf.p, ptr, bytes, cudaMemcpyHostToDevice, p->stream));
    s.dev = buf.p;
    s.host = true;
    return s;
}

static Staged stage_out(purify_plan* p, void* ptr, size_t bytes, DevBuf& buf) {
    Staged s;
    if (!is_host_pointer(ptr)) { s.dev = ptr; return s; }
    if (buf.bytes < bytes) buf.alloc(bytes);
    s.dev = buf.p;
    s.host = true;
    return s;
}

static void finish_out(purify_plan* p, const Staged& s, void* ptr, size_t bytes) {
    if (!s.host) return;
    PURIFY_CUDA(cudaMemcpyAsync(ptr, s.dev, bytes, cudaMemcpyDeviceToHost, p->stream));
    PURIFY_CUDA(cudaStreamSynchronize(p->stream));
}

static size_t real_bytes(const purify_plan* p) { return p->dtype == PURIFY_F32 ? 4 : 8; }

template <typename F> static purify_status guarded(F&& f) {
    try {
        f();
        return PURIFY_OK;
    } catch (const Error& e) {
        set_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return PURIFY_ENOMEM;
    } catch (...) {
        set_error("unexpected internal error");
        return PURIFY_ECUDA;
    }
}

}  // namespace purify

using namespace purify;

extern "C" {

purify_status purify_plan_create(const purify_plan_desc* desc, purify_plan** out) {
    return guarded([&] {
        PURIFY_REQUIRE(out != nullptr, "null output pointer");
        *out = nullptr;
        *out = create_plan(desc);
    });
}

purify_status purify_plan_destroy(purify_plan* plan) {
    return guarded([&] {
        if (!plan) return;
        cudaStreamSynchronize(plan->stream);
        delete plan->timer;
        delete plan;
    });
}

purify_status purify_plan_set_stream(purify_plan* plan, void* stream) {
    return guarded([&] {
        PURIFY_REQUIRE(plan != nullptr, "null plan");
        plan->stream = (cudaStream_t)stream;
    });
}

purify_status purify_plan_get_info(const purify_plan* plan, purify_plan_info* info) {
    return guarded([&] {
        PURIFY_REQUIRE(plan && info, "null argument");
        info->Kx = plan->Kx;
        info->Ky = plan->Ky;
        info->q = plan->q;
        info->tile = plan->work.tile;
        info->N = plan->N;
        info->D = plan->D;
        info->M = plan->M;
        info->R = plan->R;
        info->J = plan->J;
        info->levels = plan->levels;
        info->beta = plan->beta;
        info->workspace_bytes = plan->workspace_bytes;
        info->grid_mode = plan->grid_kind;
        info->degrid_mode = plan->degrid_kind;
        info->normal_mode = plan->normal_kind;
        info->lane_tile = plan->normal_kind == 5 ? plan->lanes[2].tile : 0;
        fft_launch_shape(plan, info->fft_rows_per_block, info->fft_cols_per_block, info->fft_cols_per_thread);
    });
}

purify_status purify_phi(purify_plan* p, const void* x, void* y) {
    return guarded([&] {
        PURIFY_REQUIRE(p && x && y, "null argument");
        const size_t rb = real_bytes(p);
        Staged xs = stage_in(p, x, rb * p->N, p->stage_in);
        Staged ys = stage_out(p, y, 2 * rb * p->M, p->stage_out);
        launch_phi(p, xs.dev, ys.dev, true, 1.0);
        finish_out(p, ys, y, 2 * rb * p->M);
    });
}

purify_status purify_phi_adj(purify_plan* p, const void* y, void* x) {
    return guarded([&] {
        PURIFY_REQUIRE(p && x && y, "null argument");
        const size_t rb = real_bytes(p);
        Staged ys = stage_in(p, y, 2 * rb * p->M, p->stage_in);
        Staged xs = stage_out(p, x, 2 * rb * p->N, p->stage_out);
        launch_phi_adj(p, ys.dev, xs.dev, true, 1.0, 0, nullptr);
        finish_out(p, xs, x, 2 * rb * p->N);
    });
}

purify_status purify_phi_normal(purify_plan* p, const void* x, void* out) {
    return guarded([&] {
        PURIFY_REQUIRE(p && x && out, "null argument");
        const size_t rb = real_bytes(p);
        Staged xs = stage_in(p, x, rb * p->N, p->stage_in);
        Staged os = stage_out(p, out, rb * p->N, p->stage_out);
        // the forward row pass clears the accumulator that G^H G adds into
        launch_scale_pad_rows(p, xs.dev, 1.0, nullptr, true, true);
        launch_cols_fwd(p, nullptr);
        launch_normal_gg(p, nullptr, true);
        launch_cols_inv(p, nullptr);
        launch_rows_inv_crop(p, os.dev, 1.0, 1, nullptr, 0.0, nullptr);
        finish_out(p, os, out, rb * p->N);
    });
}

purify_status purify_fft2(purify_plan* p, void* grid, int32_t inverse) {
    return guarded([&] {
        PURIFY_REQUIRE(p && grid, "null argument");
        const size_t bytes = 2 * real_bytes(p) * (size_t)p->Kx * p->Ky;
        Staged gs = stage_in(p, grid, bytes, p->stage_in);
        launch_fft2(p, gs.dev, inverse != 0);
        finish_out(p, gs, grid, bytes);
    });
}

purify_status purify_psi(purify_plan* p, const void* c, void* x) {
    return guarded([&] {
        PURIFY_REQUIRE(p && c && x, "null argument");
        const size_t rb = real_bytes(p);
        Staged cs = stage_in(p, c, rb * p->D, p->stage_in);
        Staged xs = stage_out(p, x, rb * p->N, p->stage_out);
        launch_psi(p, cs.dev, xs.dev);
        finish_out(p, xs, x, rb * p->N);
    });
}

purify_status purify_psi_adj(purify_plan* p, const void* x, void* c) {
    return guarded([&] {
        PURIFY_REQUIRE(p && c && x, "null argument");
        const size_t rb = real_bytes(p);
        Staged xs = stage_in(p, x, rb * p->N, p->stage_in);
        Staged cs = stage_out(p, c, rb * p->D, p->stage_out);
        launch_psi_adj(p, xs.dev, cs.dev);
        finish_out(p, cs, c, rb * p->D);
    });
}

purify_status purify_op_norm_sq(purify_plan* p, int32_t iters, double* norm_sq) {
    return guarded([&] {
        PURIFY_REQUIRE(p && norm_sq && iters > 0, "bad argument");
        *norm_sq = op_norm_sq(p, iters);
    });
}

purify_status purify_sdmm_solve(purify_plan* p, const void* y, const double* eps, const void* w, void* x,
                                const purify_sdmm_params* params, purify_sdmm_stats* stats) {
    return guarded([&] {
        PURIFY_REQUIRE(p && params && x, "null argument");
        PURIFY_REQUIRE(params->max_iter >= 0 && params->cg_iters >= 0, "negative iteration count");
        PURIFY_REQUIRE(params->resume || (y && eps), "y and eps are required unless resuming");
        PURIFY_REQUIRE(!params->resume || p->sd.started, "resume without a previous solve on this plan");
        PURIFY_REQUIRE(params->block_groups >= 0 && params->block_groups <= p->R, "block_groups must be in [0, R]");
        if (params->block_groups > 0 && params->group_seq)
            for (int i = 0; i < params->max_iter; ++i)
                PURIFY_REQUIRE(params->group_seq[i] >= 0 && params->group_seq[i] < params->block_groups,
                               "group_seq entry out of range");
        if (stats) std::memset(stats, 0, sizeof(*stats));
        sdmm_solve(p, y, eps, w, x, *params, stats);
    });
}

purify_status purify_pd_solve(purify_plan* p, const void* y, const double* eps, const void* w, void* x,
                              const purify_pd_params* params, purify_sdmm_stats* stats) {
    return guarded([&] {
        PURIFY_REQUIRE(p && params && x && y && eps, "null argument");
        PURIFY_REQUIRE(params->iters >= 0, "negative iteration count");
        PURIFY_REQUIRE(std::isfinite(params->tau) && std::isfinite(params->sigma) && std::isfinite(params->nu),
                       "tau, sigma and nu must be finite");
        if (stats) std::memset(stats, 0, sizeof(*stats));
        pd_solve(p, y, eps, w, x, *params, stats);
    });
}

purify_status purify_sdmm_iterate(purify_plan* p, int32_t iters) {
    return guarded([&] {
        PURIFY_REQUIRE(p != nullptr && iters >= 0, "bad argument");
        PURIFY_REQUIRE(p->sd.started, "no SDMM solve started on this plan");
        sdmm_iterate(p, iters);
    });
}

purify_status purify_sdmm_iterate_groups(purify_plan* p, int32_t iters, const int32_t* groups) {
    return guarded([&] {
        PURIFY_REQUIRE(p != nullptr && iters >= 0, "bad argument");
        PURIFY_REQUIRE(p->sd.started, "no SDMM solve started on this plan");
        sdmm_iterate(p, iters, groups);
    });
}

purify_status purify_shard_iterate_local(purify_plan* p, void* r_out) {
    return guarded([&] {
        PURIFY_REQUIRE(p != nullptr, "null plan");
        shard_step(p, 0, 0, r_out);
    });
}

purify_status purify_shard_cg_begin(purify_plan* p, const void* r_sum) {
    return guarded([&] {
        PURIFY_REQUIRE(p != nullptr, "null plan");
        shard_step(p, 1, 0, const_cast<void*>(r_sum));
    });
}

purify_status purify_shard_cg_apply(purify_plan* p, int32_t step, void* u_out) {
    return guarded([&] {
        PURIFY_REQUIRE(p != nullptr, "null plan");
        shard_step(p, 2, step, u_out);
    });
}

purify_status purify_shard_cg_combine(purify_plan* p, int32_t step, const void* u_sum) {
    return guarded([&] {
        PURIFY_REQUIRE(p != nullptr, "null plan");
        shard_step(p, 3, step, const_cast<void*>(u_sum));
    });
}

purify_status purify_shard_iterate_end(purify_plan* p, int32_t cg_steps) {
    return guarded([&] {
        PURIFY_REQUIRE(p != nullptr, "null plan");
        shard_step(p, 4, cg_steps, nullptr);
    });
}

struct purify_batch {
    purify::BatchState* st;
};

purify_status purify_batch_create(purify_plan* const* plans, int32_t n, void* stream, purify_batch** out) {
    return guarded([&] {
        PURIFY_REQUIRE(out != nullptr && plans != nullptr && n >= 1, "bad argument");
        *out = nullptr;
        for (int i = 0; i < n; ++i) {
            PURIFY_REQUIRE(plans[i] != nullptr, "null plan in batch");
            for (int j = 0; j < i; ++j) PURIFY_REQUIRE(plans[j] != plans[i], "a plan appears twice in the batch");
        }
        auto* b = new purify_batch{new BatchState()};
        b->st->plans.assign(plans, plans + n);
        b->st->stream = (cudaStream_t)stream;
        *out = b;
    });
}

purify_status purify_batch_iterate(purify_batch* b, int32_t iters) {
    return guarded([&] {
        PURIFY_REQUIRE(b != nullptr && iters >= 0, "bad argument");
        PURIFY_REQUIRE(b->st->stream != nullptr, "a batch needs a non-default stream for graph capture");
        batch_iterate(b->st, iters);
    });
}

purify_status purify_batch_destroy(purify_batch* b) {
    return guarded([&] {
        if (!b) return;
        if (b->st->stream) cudaStreamSynchronize(b->st->stream);
        batch_destroy(b->st);
        delete b;
    });
}

purify_status purify_reweight(purify_plan* p, const void* x, double rho, void* w) {
    return guarded([&] {
        PURIFY_REQUIRE(p && x && w && rho > 0, "bad argument");
        const size_t rb = real_bytes(p);
        Staged xs = stage_in(p, x, rb * p->N, p->stage_in);
        Staged ws = stage_out(p, w, rb * p->D, p->stage_out);
        reweight(p, xs.dev, rho, ws.dev);
        finish_out(p, ws, w, rb * p->D);
    });
}

purify_status purify_noise_sigma(double y_norm, int64_t M, double snr_db, double* sigma) {
    return guarded([&] {
        PURIFY_REQUIRE(sigma != nullptr, "null argument");
        PURIFY_REQUIRE(M >= 1 && std::isfinite(y_norm) && y_norm >= 0 && std::isfinite(snr_db),
                       "need M >= 1, a finite non-negative norm and a finite SNR");
        *sigma = y_norm / std::sqrt((double)M) * std::pow(10.0, -snr_db / 20.0);
    });
}

purify_status purify_chi2_epsilon(double sigma, const int64_t* offs, int32_t R, double* eps) {
    return guarded([&] {
        PURIFY_REQUIRE(offs && eps && R >= 1, "null argument or R < 1");
        PURIFY_REQUIRE(std::isfinite(sigma) && sigma > 0, "sigma must be positive and finite");
        PURIFY_REQUIRE(offs[0] == 0, "block_offsets[0] must be 0");
        for (int i = 0; i < R; ++i) PURIFY_REQUIRE(offs[i + 1] > offs[i], "block_offsets must increase");
        for (int i = 0; i < R; ++i) {
            // chi^2 with 2 M_i degrees of freedom, scaled by sigma^2 / 2: mean + 2 std
            const double m = (double)(offs[i + 1] - offs[i]);
            eps[i] = sigma / std::sqrt(2.0) * std::sqrt(2.0 * m + 4.0 * std::sqrt(m));
        }
    });
}

purify_status purify_coef_std(purify_plan* p, const void* x, double* std_out) {
    return guarded([&] {
        PURIFY_REQUIRE(p && x && std_out, "null argument");
        const size_t rb = real_bytes(p);
        Staged xs = stage_in(p, x, rb * p->N, p->stage_in);
        *std_out = coef_std(p, xs.dev);
    });
}

purify_status purify_psi_adj_static(const void* x, void* c, int32_t nx, int32_t ny, int32_t levels,
                                    uint32_t basis_mask, purify_dtype dtype, void* stream) {
    return guarded([&] {
        PURIFY_REQUIRE(x && c, "null argument");
        PURIFY_REQUIRE(dtype == PURIFY_F32 || dtype == PURIFY_F64, "dtype must be PURIFY_F32 or PURIFY_F64");
        PURIFY_REQUIRE(nx >= 8 && ny >= 8 && nx <= 4096 && ny <= 4096 && (nx & (nx - 1)) == 0 && (ny & (ny - 1)) == 0,
                       "nx, ny must be powers of two in [8, 4096]");
        PURIFY_REQUIRE(levels >= 1 && levels <= 8 && (nx >> (levels - 1)) >= 2 && (ny >> (levels - 1)) >= 2,
                       "image too small for the number of levels");
        const uint32_t mask = basis_mask ? basis_mask : 0x1FFu;
        PURIFY_REQUIRE((mask & ~0x1FFu) == 0, "basis_mask has bits above db8");
        const size_t need = psi_adj_static_bytes(nx, ny, mask, dtype);
        PURIFY_REQUIRE(need <= psi_adj_static_capacity(),
                       "image too large for the static scratch: needs " + std::to_string(need) + " of " +
                           std::to_string(psi_adj_static_capacity()) + " bytes");
        PURIFY_REQUIRE(!is_host_pointer(x) && !is_host_pointer(c), "x and c must be device pointers");
        psi_adj_static(x, c, nx, ny, levels, mask, dtype, (cudaStream_t)stream);
    });
}

purify_status purify_conv2d(const float* x, int32_t B, int32_t H, int32_t W, int32_t Cin, const float* w,
                            const float* bias, int32_t Cout, int32_t k, int32_t relu, float* out, void* stream) {
    return guarded([&] {
        PURIFY_REQUIRE(x && w && out, "null argument");
        PURIFY_REQUIRE(B >= 1 && H >= 1 && W >= 1 && Cin >= 1 && Cout >= 1 && Cout <= 256 && (k == 1 || k == 3),
                       "conv2d: bad shape (Cout <= 256, k = 1 or 3)");
        PURIFY_REQUIRE(!is_host_pointer(x) && !is_host_pointer(w) && !is_host_pointer(out) &&
                           (!bias || !is_host_pointer(bias)),
                       "conv2d: device pointers required");
        conv2d_f32(x, B, H, W, Cin, w, bias, Cout, k, relu, out, (cudaStream_t)stream);
    });
}

struct purify_unet {
    purify::Unet* u;
    int H, W, maxB;
};

purify_status purify_unet_create(int32_t H, int32_t W, int32_t levels, int32_t base, int32_t max_batch,
                                 uint64_t seed, void* stream, purify_unet** out) {
    return guarded([&] {
        PURIFY_REQUIRE(out != nullptr, "null output pointer");
        *out = nullptr;
        Unet* u = unet_create(H, W, levels, base, max_batch, seed, (cudaStream_t)stream);
        *out = new purify_unet{u, H, W, max_batch};
    });
}

purify_status purify_unet_destroy(purify_unet* net) {
    return guarded([&] {
        if (!net) return;
        unet_destroy(net->u);
        delete net;
    });
}

int64_t purify_unet_num_params(const purify_unet* net) { return net ? unet_nparams(*net->u) : -1; }

purify_status purify_unet_get_params(purify_unet* net, float* out) {
    return guarded([&] {
        PURIFY_REQUIRE(net && out, "null argument");
        unet_get(*net->u, 0, out);
    });
}

purify_status purify_unet_set_params(purify_unet* net, const float* in) {
    return guarded([&] {
        PURIFY_REQUIRE(net && in, "null argument");
        unet_set_params(*net->u, in);
    });
}

purify_status purify_unet_forward(purify_unet* net, const float* x, float* y, int32_t B) {
    return guarded([&] {
        PURIFY_REQUIRE(net && x && y && B >= 1 && B <= net->maxB, "bad argument");
        PURIFY_REQUIRE(!is_host_pointer(x) && !is_host_pointer(y), "device pointers required");
        unet_forward(*net->u, x, B, y);
    });
}

purify_status purify_unet_gradients(purify_unet* net, const float* x, const float* target, int32_t B, float* grads,
                                    double* loss) {
    return guarded([&] {
        PURIFY_REQUIRE(net && x && target && B >= 1 && B <= net->maxB, "bad argument");
        PURIFY_REQUIRE(!is_host_pointer(x) && !is_host_pointer(target), "device pointers required");
        unet_gradients(*net->u, x, target, B);
        double l = unet_read_loss(*net->u);
        if (loss) *loss = l;
        if (grads) unet_get(*net->u, 1, grads);
    });
}

purify_status purify_unet_train_step(purify_unet* net, const float* x, const float* target, int32_t B, float lr,
                                     double* loss) {
    return guarded([&] {
        PURIFY_REQUIRE(net && x && target && B >= 1 && B <= net->maxB && lr > 0, "bad argument");
        PURIFY_REQUIRE(!is_host_pointer(x) && !is_host_pointer(target), "device pointers required");
        unet_gradients(*net->u, x, target, B);
        unet_adam(*net->u, lr);
        if (loss) *loss = unet_read_loss(*net->u);
    });
}

purify_status purify_timing_enable(purify_plan* p, int32_t enable) {
    return guarded([&] {
        PURIFY_REQUIRE(p != nullptr, "null plan");
        if (!p->timer) p->timer = new KernelTimer();
        p->timer->enabled = enable != 0;
    });
}

int32_t purify_timing_read(purify_plan* p, purify_kernel_time* out, int32_t cap, int32_t reset) {
    int32_t n = -1;
    purify_status st = guarded([&] {
        PURIFY_REQUIRE(p != nullptr, "null plan");
        if (!p->timer) { n = 0; return; }
        p->timer->drain();
        n = 0;
        for (auto& kv : p->timer->acc) {
            if (out && n < cap) {
                std::memset(out[n].name, 0, sizeof(out[n].name));
                std::strncpy(out[n].name, kv.first.c_str(), sizeof(out[n].name) - 1);
                out[n].launches = kv.second.first;
                out[n].total_ms = kv.second.second;
            }
            ++n;
        }
        if (reset) p->timer->acc.clear();
    });
    return st == PURIFY_OK ? n : -1;
}

int64_t purify_launch_count(void) { return g_launches.load(); }

const char* purify_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
