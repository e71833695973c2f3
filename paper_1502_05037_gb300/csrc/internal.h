// Internal plan structure and kernel-launch entry points of the imaging
// library. Everything here is private to the shared library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/purify.h"
#include "common.cuh"

namespace purify {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
struct Error {
    purify_status status;
    std::string msg;
};
#define PURIFY_CUDA(call)                                                           \
    do {                                                                            \
        cudaError_t _e = (call);                                                    \
        if (_e != cudaSuccess)                                                      \
            throw ::purify::Error{PURIFY_ECUDA, std::string(#call) + ": " +         \
                                                    cudaGetErrorString(_e)};        \
    } while (0)
#define PURIFY_REQUIRE(cond, msg)                                                   \
    do {                                                                            \
        if (!(cond)) throw ::purify::Error{PURIFY_EINVAL, (msg)};                   \
    } while (0)

// --------------------------------------------------------- launch timing
struct KernelTimer;
void note_launch(const char* name, cudaStream_t s, KernelTimer* t, bool begin);

// ------------------------------------------------------- device buffers
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    void alloc(size_t b);
    void release();
    template <typename T> T* as() const { return static_cast<T*>(p); }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
};

// Wavelet filter table: for basis p (1..8) the low-pass h and high-pass g,
// each padded to 16 taps, in the plan dtype.
#define PURIFY_MAX_TAPS 16
template <typename T> struct FilterBank {
    T h[9][PURIFY_MAX_TAPS];
    T g[9][PURIFY_MAX_TAPS];
    int len[9];
};

// Gridding work list: subproblem s covers grid tile sub_bin[s] and the
// visibility pieces piece_off[s] .. piece_off[s+1]-1; piece k is the internal
// index range [piece_start[k], piece_start[k] + piece_len[k]).
// Gridding/degridding work list: subproblem s is grid tile sub_bin[s] and
// the visibilities list[sub_off[s] .. sub_off[s + 1]) (internal indices,
// ordered by first-tap cell).
struct GridWork {
    int nsub = 0, tile = 32, units = 4, tiles_x = 0, tiles_y = 0;
    DevBuf sub_bin, sub_off, list;
};

// Run-ordered gridding work: a run is a set of visibilities sharing their
// first-tap cell (at most a fixed length; longer cells are cut); runs are
// sorted by length, longest first, and taken G = 32 / J at a time by a warp
// (one run per lane group). Run r has cell[r] = (cy << 16) | cx, its records
// rec[start[r] .. start[r] + len[r]); the run count is padded to a multiple
// of G with empty runs.
struct RunWork {
    int nsets = 0, nruns = 0, G = 1;
    DevBuf rec, cell, start, len;
};

// Lane-per-run work (FP32 plans, J <= 6): the same runs, `width` per warp
// set (32 / lanes per run). Set s holds record rows [row0, row0 + lmax) with
// lmax its longest run; the record of run width s + r at step k is in
// record row row0 + k: with width 32 the float2 (phx, phy) at
// rec[(row0 + k) * 32 + r], with width 16 (a lane pair per run) phx at
// float (row0 + k) * 32 + r and phy at float (row0 + k) * 32 + 16 + r, so
// one step of a warp reads one record row (8 bytes per run), each lane of a
// pair its own axis. Records past a run's end are padding (zero offsets,
// index -1). run_cl[width s + r] = (cell, len), the cell packed as
// (cy << 16) | cx; idx / idx_caller give each record's visibility in
// internal / caller order. Set order: runs sorted by length (longest
// first), or with tile > 0 grouped by grid tile of that edge (tiles in
// raster order, runs by length within a tile).
// Deterministic form (cstart non-empty): the kernels store each run's J x J
// patch at patch[(b J + a) * nsets * width + run] instead of adding it to
// the grid, and a gather sums, for every grid cell, the patches of the runs
// whose footprint covers it in a fixed order (taps b, a, then the cell's
// runs in run order): cstart[c] .. cstart[c + 1] index clist, the runs with
// first-tap cell c (c = cy Kx + cx) in increasing run order.
static constexpr int kLaneMaxJ = 6;
struct LaneWork {
    int nsets = 0, width = 32, tile = 0;
    int64_t rows = 0;
    DevBuf set_info;              // int2 (row0, lmax) per set
    DevBuf run_cl;                // int2 (cell, len) per run
    DevBuf rec;                   // 8 bytes per record (layout above)
    DevBuf idx, idx_caller;       // int per record
    DevBuf cstart, clist;         // deterministic form: int [Kx Ky + 1], int per real run
    bool deterministic() const { return cstart.p != nullptr; }
    void release() {
        nsets = 0;
        rows = 0;
        set_info.release();
        run_cl.release();
        rec.release();
        idx.release();
        idx_caller.release();
        cstart.release();
        clist.release();
    }
};

// Block groups of the stochastic block-subset iterations: block i belongs to
// group i mod G; per group the lane work of its visibilities (two lanes per
// run) and the visibility chunks of its blocks (chunk_first indexes the
// group's own chunk list; blocks outside the group have empty ranges).
struct GroupChunks {
    int n = 0;
    DevBuf cblk, cbeg, cend, chunk_first;
};

// SDMM device state (allocated on first solve).
struct SdmmState {
    bool ready = false;
    bool have_w = false;
    DevBuf x, z1, z2, z3;         // iterate and multipliers
    DevBuf ybar;                  // y / nu in internal order
    DevBuf w;                     // weights [D]
    DevBuf eps;                   // eps_i / nu, double [R]
    DevBuf c1;                    // [D] analysis coefficients / prox output
    DevBuf v2;                    // [M] Phi x / nu then fused residual term
    DevBuf addend;                // [N] image-space terms of the CG residual
    DevBuf r, p, Ap, u, xprev;    // CG vectors [N] (Ap holds s = A p, u = A r)
    DevBuf scal;                  // double scalars (see sdmm.cu)
    DevBuf part;                  // double partial sums
    DevBuf counters;              // unsigned ints for last-block reductions, then int flags
    DevBuf chunk_first;           // int [R + 1]: first visibility chunk of each block
    bool started = false;
    double gamma = 0, nu = 0;
    int cg_iters = 10;
    bool toeplitz = false;        // CG normal operator by circulant embedding
    DevBuf toep;                  // [Ky][Kx] real multiplier of the embedded normal operator
    double toep_nu = 0;
    std::vector<double> eps_host;
    // captured iteration graph
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // side stream of an iteration's visibility branch (forked and joined
    // with events, so it is part of the captured graph)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphExec_t pd_gexec = nullptr;   // one primal-dual iteration
    double pd_key[4] = {0, 0, 0, 0};      // tau, sigma, nu, weights of pd_gexec
    int64_t pd_kernels = 0;
    int g_cg = -1;
    double g_gamma = 0, g_nu = 0;
    bool g_have_w = false;
    bool g_toep = false;
    int64_t g_kernels = 0;
    ~SdmmState() {
        for (auto& e : gexec_group)
            if (e) cudaGraphExecDestroy(e);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (pd_gexec) cudaGraphExecDestroy(pd_gexec);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (gstream) cudaStreamDestroy(gstream);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
    }
    int64_t iters_done = 0;
    int64_t cg_total = 0;
    // block-subset iterations: groups of the current solve (0: all blocks
    // every iteration) and one captured graph per group
    int groups = 0;
    std::vector<cudaGraphExec_t> gexec_group;
    std::vector<int64_t> kernels_group;
    int gg_cg = -1;
    double gg_gamma = 0, gg_nu = 0;
    bool gg_have_w = false;
    int gg_groups = 0;
    void drop_group_graphs() {
        for (auto& e : gexec_group)
            if (e) cudaGraphExecDestroy(e);
        gexec_group.clear();
        kernels_group.clear();
    }
};

}  // namespace purify

struct purify_plan {
    purify_plan_desc desc;
    int dtype;  // PURIFY_F32 / PURIFY_F64
    int nx, ny, Kx, Ky, J, levels, q, R;
    int64_t N, D, M;
    uint32_t mask;
    double beta, i0beta;
    cudaStream_t stream;
    std::vector<int64_t> offsets;     // host, R + 1
    std::vector<int> bases;           // basis ids in dictionary order (0 = Dirac)
    purify::AxisConst ax, ay;
    purify::KbPoly kbp;
    purify::DevBuf sx, sy;            // per-axis correction (dtype)
    purify::DevBuf onesx, onesy;      // all-ones tables (transforms without the correction)
    purify::DevBuf twx, twy;          // twiddles (complex dtype)
    purify::DevBuf wmeta;             // int[16]: wavelet db index and plane per basis
    purify::DevBuf us, vs;            // sorted coordinates (dtype)
    purify::DevBuf perm;              // int32 internal -> caller
    purify::DevBuf d_offsets;         // int64 [R + 1]
    purify::DevBuf chunk_blk, chunk_beg, chunk_end;  // visibility chunks, each inside one block
    int nchunks = 0;
    purify::GridWork work;            // gridding work list (tile of the G^H kernel)
    purify::GridWork dwork;           // degridding work list (tile of the G kernel)
    purify::RunWork runs;             // run-ordered work of the fused normal operator
    purify::LaneWork lanes[3];        // lane-per-run forms of the same runs (FP32, J <= 6): one lane
                                      // per run; two lanes per run; two, sets grouped by tile
    purify::DevBuf det_patch;         // run patches of the deterministic lane form (float2)
    int normal_kind = 2;              // G^H G: 2 run sets, 3..5 lanes (as lanes[kind - 3]), 6 the
                                      // deterministic lane pairs (lanes[1]); autotuned or forced
    int group_count = 0;              // G of group_lanes / group_chunks (0: not built)
    std::vector<purify::LaneWork> group_lanes;
    std::vector<purify::GroupChunks> group_chunks;
    int grid_kind = 1;                // G^H: 1 tile subproblems, 2 run sets, 3..5 lanes, 6 deterministic
    int degrid_kind = 1;              // G: 1 tile subproblems, 3..5 lanes; autotuned
    int fft_rb = 0, fft_cb = 0;       // FFT rows / columns per block (0: heuristic)
    int fft_cw = 0;                   // FFT columns per thread, 1 or 2 (0: 2 where the shape allows)
    // workspaces
    purify::DevBuf grid;              // Ky * Kx complex (forward transform output)
    purify::DevBuf gacc;              // Ky * Kx complex gridding output, then a 256-byte work counter
    purify::DevBuf rows;              // ny * Kx complex
    purify::DevBuf ll0, ll1;          // wavelet low-pass scratch (dtype, 8 * N / 4 each)
    purify::DevBuf stage_in, stage_out;  // host-pointer staging
    purify::DevBuf tmp_img, tmp_vis, tmp_coef;
    purify::SdmmState sd;
    purify::KernelTimer* timer = nullptr;
    int64_t workspace_bytes = 0;
};

namespace purify {

// Conjugate gradients in the Chronopoulos-Gear arrangement (equal to the
// textbook iteration in exact arithmetic; one synchronisation per step): the
// operator is applied to the residual, u = A r, and the inverse row pass of
// step k writes per-block partials of gamma = r.r and delta = r.u; its last
// block to finish reduces them (cg_decide) to
//   beta = gamma / gamma_prev (0 at step 0),
//   alpha = gamma / (delta - beta gamma / alpha_prev)  (gamma / delta at step 0),
// and the stop test (gamma <= tol^2 gamma_0, gamma_0 of step 0). Unless the
// step stopped the solve, the forward row pass of step k + 1 (or the
// relative-change kernel after the last step) applies the update p = r + beta p,
// s = u + beta s (s = A p), x += alpha p, r -= alpha s, then transforms the
// new r. The forward row pass of step 0 starts the solve: r += add (the
// residual's terms formed outside the pass), p = s = 0, the stop flag cleared.
struct CgFold {
    void* x = nullptr;           // iterate [N]
    void* r = nullptr;           // residual [N]
    void* p = nullptr;           // direction [N]
    void* s = nullptr;           // A p [N]
    const void* u = nullptr;     // A r [N]
    const void* add = nullptr;   // added to r at step 0 (may be null)
    double* part = nullptr;      // the inverse row pass's partials, 2 per block
    unsigned* counter = nullptr; // arrival counter of the inverse row pass
    double* scal = nullptr;
    int* flags = nullptr;
    int step = 0;
};
// blocks of the inverse row pass (the number of CG partials it writes)
int rows_inv_blocks(purify_plan* p);

// ----------------------------------------------------------- operator steps
// Phi: x real [ny][nx] (internal pointer) -> y complex [M]. If perm != null
// the output is written in caller order through perm. `scale` multiplies S.
// zero_acc: the forward row pass also clears the gridding accumulator (for a
// Phi^H launched later with acc_zeroed).
void launch_phi(purify_plan* p, const void* x, void* y, bool caller_order, double scale, bool zero_acc = false);
// Phi^H: y complex [M] (caller order if caller_order) -> image.
//   out_mode 0: complex [ny][nx];  1: real part, out = scale * Re(.) + add (add may be null)
// acc_zeroed: the gridding accumulator is already clear (no memset).
void launch_phi_adj(purify_plan* p, const void* y, void* out, bool caller_order, double scale,
                    int out_mode, const void* add, bool acc_zeroed = false);
void launch_fft2(purify_plan* p, void* grid, bool inverse);
// Phi stages used by the solver's fused forms
// zero_acc: the same launch clears the gridding accumulator (gacc); fold:
// apply the pending CG update first (see CgFold)
void launch_scale_pad_rows(purify_plan* p, const void* x, double scale, const int* skip_flag, bool corr = true,
                           bool zero_acc = false, const CgFold* fold = nullptr);
void launch_cols_fwd(purify_plan* p, const int* skip_flag);
void launch_degrid(purify_plan* p, void* y, bool caller_order, const int* skip_flag);
void launch_grid(purify_plan* p, const void* y, bool caller_order, const int* skip_flag, bool zeroed = false);
// inverse column pass: reads the gridding output (gacc), or with `mult` the
// forward grid multiplied elementwise by mult
void launch_cols_inv(purify_plan* p, const int* skip_flag, const void* mult = nullptr);
// G^H G of the grid (the oversampled image after F Z S): for every
// visibility the J x J interpolation of the forward grid spread back with the
// same weights, into gacc (the visibility values are never stored)
// (zeroed: gacc was cleared by this step's forward row pass, no memset)
void launch_normal_gg(purify_plan* p, const int* skip_flag, bool zeroed = false);
// G^H by runs (same output as launch_grid)
void launch_grid_sets(purify_plan* p, const void* y, bool caller_order, const int* skip_flag, bool zeroed = false);
// cg: a CG step (out = A r, add = r): per-block partials of r.r and r.A r
// (2 per block, in cg->part), reduced and decided by the last block (see
// CgFold); cg->step is the step
void launch_rows_inv_crop(purify_plan* p, void* out, double scale, int out_mode, const void* add,
                          double add_coef, const int* skip_flag, const CgFold* cg = nullptr, bool corr = true);

// Psi / Psi^dagger
void launch_psi_adj(purify_plan* p, const void* x, void* c);
void launch_psi(purify_plan* p, const void* c, void* x);
void init_filter_banks();
// allocation-free Psi^dagger (file-scope static scratch, see wavelet.cu)
void psi_adj_static(const void* x, void* c, int nx, int ny, int levels, unsigned mask, int dtype, cudaStream_t st);
size_t psi_adj_static_bytes(int nx, int ny, unsigned mask, int dtype);
size_t psi_adj_static_capacity();

// learned warm start
void conv2d_f32(const float* x, int B, int H, int W, int Cin, const float* w, const float* bias, int Cout, int k,
                int relu, float* out, cudaStream_t st);

struct Unet;
Unet* unet_create(int H, int W, int L, int base, int maxB, uint64_t seed, cudaStream_t st);
void unet_destroy(Unet* u);
void unet_forward(Unet& u, const float* x, int B, float* out);
void unet_gradients(Unet& u, const float* x, const float* target, int B);
double unet_read_loss(Unet& u);
void unet_adam(Unet& u, float lr);
void unet_set_params(Unet& u, const float* p);
void unet_get(Unet& u, int what, float* out);
int64_t unet_nparams(Unet& u);

// solver
void sdmm_solve(purify_plan* p, const void* y, const double* eps, const void* w, void* x,
                const purify_sdmm_params& prm, purify_sdmm_stats* st);
double op_norm_sq(purify_plan* p, int iters);
struct BatchState {
    std::vector<purify_plan*> plans;
    cudaStream_t stream = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaGraphExec_t gexec = nullptr;
    std::vector<double> key;
    int64_t kernels = 0;
};
void batch_iterate(BatchState* b, int iters);
void batch_destroy(BatchState* b);
void sdmm_iterate(purify_plan* p, int iters, const int32_t* groups = nullptr);
// block-sharded SDMM steps: op 0 local terms (adjoint term out), 1 summed
// adjoint term in, 2 CG apply (this shard's normal operator out), 3 CG
// combine (summed normal operator in), 4 end of iteration (step = CG steps)
void shard_step(purify_plan* p, int op, int step, void* ptr);
void pd_solve(purify_plan* p, const void* y, const double* eps, const void* w, void* x,
              const purify_pd_params& prm, purify_sdmm_stats* st);
void add_launches(int64_t n);
bool timing_enabled(const purify_plan* p);
void reweight(purify_plan* p, const void* x, double rho, void* w);
double coef_std(purify_plan* p, const void* x);

int max_grid_tile(int dtype, int J);
// the lane-per-run kernels apply to this plan (FP32, J <= kLaneMaxJ)
bool lane_work_ok(const purify_plan* p);
// G^H / G by the lane-per-run kernels (same outputs as launch_grid / launch_degrid)
// (kind 3: one lane per run, 4: two lanes per run, 5: two lanes per run
// with the sets grouped by grid tile)
void launch_grid_lanes(purify_plan* p, int kind, const void* y, bool caller_order, const int* skip,
                       bool zeroed = false);
void launch_degrid_lanes(purify_plan* p, int kind, void* y, bool caller_order, const int* skip);
void launch_normal_lanes(purify_plan* p, int kind, const int* skip, bool zeroed = false);
// the lane kernels on an explicit lane work (mode 0 G^H G into gacc, 1 G^H of
// yin into gacc, 2 G into yout; internal or caller order)
void launch_lanes_on(purify_plan* p, const LaneWork& lw, int mode, const void* yin, void* yout, bool caller_order,
                     const int* skip, bool zeroed);
// lane work and chunk lists of G block groups (FP32 plans with J <= kLaneMaxJ)
void build_group_lanes(purify_plan* p, int G);
int grid_list_unit(int dtype, int J);
bool fft_shape_ok(int nb, int K, int dtype, int lanes = 1);
// the FFT launch shape the plan's passes use
void fft_launch_shape(const purify_plan* p, int& rows_per_block, int& cols_per_block, int& cols_per_thread);

// plan-side helpers
void build_gridlist(purify_plan* p, const std::vector<int>& bins, const std::vector<int>& cell_order, int tile,
                    int units, GridWork& w);
purify_plan* create_plan(const purify_plan_desc* d);
bool is_host_pointer(const void* ptr);

}  // namespace purify
