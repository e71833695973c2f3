/*
 * purify.h - C ABI of the GB300 SARA/SDMM imaging library.
 *
 * The library computes the hot path of "Why CLEAN when you can PURIFY?"
 * (Carrillo, McEwen, Wiaux; arXiv:1502.05037): the measurement operator of
 * the discretised measurement equation y = Phi x + n (Sec. 1), the SARA
 * dictionary Psi = [Psi_1, ..., Psi_q] and its adjoint (Sec. 1), and the SDMM
 * solve of the block-constrained weighted-l1 problem (3) with SARA
 * reweighting (Sec. 1, Eqs. 1-3).
 *
 * Conventions for every call:
 *  - Array arguments are caller-owned and may live on the device (any CUDA
 *    device pointer) or, where stated, on the host; the library detects which.
 *    The plan owns only its internal tables and workspaces.
 *  - Real arrays hold `dtype` values (float or double). "Complex" arrays hold
 *    interleaved (re, im) pairs of `dtype`.
 *  - Images are [ny][nx] row-major; pixel (i, j) sits at centred coordinates
 *    (j - nx/2, i - ny/2); u pairs with the column index, v with the row index.
 *  - Coefficient arrays are [q][ny][nx]: plane 0 is the Dirac basis, the next
 *    planes are db_p wavelets in increasing p among those selected by the
 *    basis mask, each in Mallat packing (coarsest low-pass band top-left).
 *  - Visibility arrays are in the caller's order; blocks are the contiguous
 *    ranges [block_offsets[i], block_offsets[i+1]) of Eq. 2.
 *  - Calls are asynchronous on the plan's stream unless stated otherwise.
 *    No exception crosses the ABI: every call returns a purify_status and, on
 *    failure, leaves a message for purify_last_error() (thread-local).
 *  - A plan is not thread-safe; use one plan per host thread and stream.
 *  - A plan belongs to the CUDA device that is current when it is created
 *    (its tables, workspaces and captured graphs live there): make that
 *    device current before every call on the plan. Plans on different
 *    devices of one process are independent.
 */
#ifndef PURIFY_H
#define PURIFY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct purify_plan purify_plan;

typedef enum {
    PURIFY_OK = 0,
    PURIFY_EINVAL = 1,    /* bad argument; detected before any launch */
    PURIFY_ENOMEM = 2,    /* device or host allocation failed */
    PURIFY_ECUDA = 3,     /* a CUDA runtime call failed */
    PURIFY_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    PURIFY_ENOTCONV = 5,  /* tolerance not reached within the iteration cap */
    PURIFY_ENAN = 6       /* non-finite value met in the data or iterates */
} purify_status;

typedef enum { PURIFY_F32 = 0, PURIFY_F64 = 1 } purify_dtype;

/* Plan description. Sec. 1 leaves the discretisation of Phi open; the plan
 * realises Phi = G F Z S (Kaiser-Bessel gridding): S the gridding correction,
 * Z zero-padding to the K = oversample * n grid, F the unnormalised 2-D DFT,
 * G interpolation with a J-tap separable Kaiser-Bessel kernel
 * g(t) = I0(beta sqrt(1 - (2t/J)^2)), kappa = u K / (2 pi), taps
 * k_a = floor(kappa - J/2) + 1 + a. */
typedef struct {
    int32_t nx, ny;                /* image size: powers of two, 8..4096, >= 2^levels */
    int64_t M;                     /* number of visibilities, 1 <= M < 2^31 */
    const void *u, *v;             /* M coordinates each (dtype), radians/pixel in
                                      [-pi, pi); host or device; copied at create */
    int32_t R;                     /* number of blocks (Eq. 2), 1 <= R <= M */
    const int64_t *block_offsets;  /* HOST array of R + 1 offsets, 0 = first < ... < last = M;
                                      NULL with R = 1 means one block */
    int32_t kb_width;              /* J, 2..8 */
    double oversample;             /* alpha; 0 => 2. Must make alpha*n a power of two */
    double kb_beta;                /* 0 => 2.34 J */
    int32_t levels;                /* wavelet levels L, 1..8 */
    uint32_t basis_mask;           /* bit 0 Dirac, bit p db_p (p = 1..8); 0 => 0x1FF (q = 9) */
    purify_dtype dtype;            /* operator precision */
    void *stream;                  /* cudaStream_t; NULL = legacy default stream */
    int32_t tile;                  /* gridding tile edge (power of two, 8..64); 0 => autotune */
    int32_t grid_mode;             /* G^H / G work decomposition: 0 => autotuned (tile
                                      subproblems when `tile` is fixed), 1 => tile subproblems
                                      (shared-memory tile per subproblem), 2 => G^H by runs of
                                      visibilities sharing their first-tap cell, flushed to the
                                      grid (G by tiles), 3..5 => G^H, G and the solver's G^H G
                                      by lanes: each run of visibilities sharing a first-tap cell
                                      owned by one lane (3) or a lane pair (4; 5: runs grouped by
                                      grid tile), its patch and accumulator in registers (FP32,
                                      J <= 6 only); 6 => deterministic: as 4, but each run's
                                      J x J patch is stored and every grid cell sums the patches
                                      covering it in a fixed order, so G^H, the normal operator
                                      and an SDMM solve give the same bits on every run of the
                                      same plan and inputs (FP32, J <= 6; no floating-point
                                      atomics; J^2 * 8 bytes per run of extra memory). Not a
                                      passage of the paper: an execution choice. */
} purify_plan_desc;

/* Build a plan: validates the description, computes the correction, kernel,
 * twiddle and Daubechies filter tables on the host, sorts the visibilities
 * by block then grid tile, and allocates workspaces. Synchronous.
 * Errors: EINVAL (description), ENOMEM, ECUDA. */
purify_status purify_plan_create(const purify_plan_desc *desc, purify_plan **out);

/* Release a plan and everything it owns (synchronises its stream). NULL is a no-op. */
purify_status purify_plan_destroy(purify_plan *plan);

/* Change the stream later calls are issued on. */
purify_status purify_plan_set_stream(purify_plan *plan, void *stream);

/* Sizes of the plan: K (grid edge per axis), q, D = q nx ny, and the gridding tile. */
typedef struct {
    int32_t Kx, Ky, q, tile;
    int64_t N, D, M;
    int32_t R, J, levels;
    double beta;
    int64_t workspace_bytes;
    int32_t grid_mode;             /* the G^H decomposition in use: 1 tile subproblems, 2 runs,
                                      3..5 lanes, 6 deterministic lanes (as grid_mode of the
                                      description) */
    int32_t degrid_mode;           /* the G decomposition in use: 1 tile subproblems, 3..5 lanes */
    int32_t normal_mode;           /* the fused G^H G of the CG normal operator: 2 runs, 3..5 lanes,
                                      6 deterministic lanes */
    int32_t lane_tile;             /* grid tile edge grouping the runs of normal_mode 5 (else 0) */
    int32_t fft_rows_per_block;    /* FFT launch shape in use: row transforms per block, */
    int32_t fft_cols_per_block;    /* column transforms per block, */
    int32_t fft_cols_per_thread;   /* and column transforms per thread (2: packed FP32 pairs) */
} purify_plan_info;
purify_status purify_plan_get_info(const purify_plan *plan, purify_plan_info *info);

/* y = Phi x (Sec. 1, measurement equation without noise): x real [ny][nx],
 * y complex [M] in caller order. */
purify_status purify_phi(purify_plan *plan, const void *x, void *y);

/* x = Phi^dagger y = S Z^T F^H G^H y, the adjoint of purify_phi on complex
 * images: y complex [M] caller order, x complex [ny][nx]. */
purify_status purify_phi_adj(purify_plan *plan, const void *y, void *x);

/* out = Re Phi^H Phi x, the data-fidelity normal operator of the SDMM
 * x-update (Sec. 1: the CG system (2 I + Re Phi^H Phi / nu^2) x = b of the
 * solve of problem (3)), applied as the solver applies it: S Z and F, then
 * G^H G fused (each visibility's J x J interpolation spread straight back,
 * no visibility vector), then F^H, Z^T and S. x real [ny][nx], out real
 * [ny][nx] (host or device; may not alias). Errors: EINVAL, ECUDA. */
purify_status purify_phi_normal(purify_plan *plan, const void *x, void *out);

/* F of Phi = G F Z S alone: in-place unnormalised 2-D DFT of a complex
 * [Ky][Kx] grid; inverse != 0 applies F^H (the +i sign, no 1/K^2 factor). */
purify_status purify_fft2(purify_plan *plan, void *grid, int32_t inverse);

/* x = Psi c = sum_j Psi_j c_j / sqrt(q) (Sec. 1, SARA dictionary):
 * c real [q][ny][nx], x real [ny][nx]. */
purify_status purify_psi(purify_plan *plan, const void *c, void *x);

/* c = Psi^dagger x = [Psi_1^T x; ...; Psi_q^T x] / sqrt(q) (Sec. 1, the
 * analysis operator of the average-sparsity prior): x real, c real [q][ny][nx]. */
purify_status purify_psi_adj(purify_plan *plan, const void *x, void *c);

/* ||Phi||_2^2 for real images (largest eigenvalue of Re Phi^H Phi) by
 * `iters` power iterations from a fixed seeded start. Synchronous. */
purify_status purify_op_norm_sq(purify_plan *plan, int32_t iters, double *norm_sq);

/* SDMM solver parameters for problem (3). */
typedef struct {
    int32_t max_iter;     /* outer SDMM iterations (exact count when rel_obj_tol == 0) */
    int32_t cg_iters;     /* conjugate-gradient iterations per x-update (cap) */
    double cg_tol;        /* 0 => exactly cg_iters CG steps (fewer only if the residual is 0);
                             > 0 => stop when ||r|| <= cg_tol ||r_0||, r_0 the residual of
                             the warm start of that x-update */
    double gamma;         /* SDMM step; <= 0 => 1e-3 max|Psi^dagger Re Phi^H y| / nu^2 */
    double nu;            /* data-term scale ||Phi||_2; <= 0 => 100 power iterations */
    double rel_obj_tol;   /* > 0: stop once the relative objective change < rel_obj_tol
                             and every ||y_i - Phi_i x|| / eps_i <= 1 + eps_tol */
    double eps_tol;
    int32_t check_every;  /* stopping test interval (iterations), 0 => 10 */
    int32_t resume;       /* 1: continue the previous solve on this plan (same y, eps, w,
                             gamma, nu); x is then output only */
    int32_t toeplitz;     /* 1: the CG x-update applies Re Phi^H Phi by circulant (Toeplitz)
                             embedding of the exact model's point-spread function
                             sum_m exp(i w_m . d) (computed once per solve with the
                             adjoint NUFFT), instead of a gridding / degridding pair per
                             CG step; the operator then differs from the NUFFT one by the
                             NUFFT error. Needs oversample 2. */
    int32_t block_groups; /* G >= 1: stochastic block-subset iterations (Sec. 1, closing
                             paragraph: one data block or a subset of blocks per
                             iteration). Block i belongs to group i mod G; iteration t
                             uses group g_t only: Phi_g x, the projections and multiplier
                             updates of the group's blocks, and an x-update whose data
                             term is G times the group's (an unbiased estimate of the full
                             one):  (2 I + G Re Phi_g^H Phi_g / nu^2) x = Psi (s1 - z1)
                             + (s3 - z3) + G Re Phi_g^H (s2_g - z2_g) / nu. G = 1 is plain
                             SDMM (on the group code path); 0 = plain SDMM. FP32 plans
                             with kb_width <= 6, no toeplitz; G <= R. In tolerance mode the
                             test evaluates every block at x and compares the objective
                             with that of the previous check. */
    const int32_t *group_seq; /* HOST, max_iter entries in [0, G): g_t of this call's
                             iterations; NULL => (iterations done) mod G */
} purify_sdmm_params;

/* Statistics of a solve, evaluated at the returned x. */
typedef struct {
    int32_t iters;
    int32_t cg_iters_total;
    double objective;          /* ||W Psi^dagger x||_1 */
    double max_resid_over_eps; /* max_i ||y_i - Phi_i x|| / eps_i */
    double rel_change;         /* ||x_t - x_{t-1}|| / ||x_t|| of the last iteration */
    double gamma, nu;          /* constants used */
    int32_t status;            /* purify_status of the solve */
} purify_sdmm_stats;

/* Solve problem (3) (Sec. 1) by SDMM: min ||W Psi^dagger x||_1 subject to
 * ||y_i - Phi_i x||_2 <= eps_i for every block and x >= 0.
 *   y      complex [M], caller order (host or device)
 *   eps    HOST double [R]; each > 0
 *   w      real [q][ny][nx] weights (host or device), NULL => W = I
 *   x      real [ny][nx] (host or device): in = starting point, out = solution
 *   stats  HOST, may be NULL
 * Iteration order (from the current x, multipliers z_j starting at 0):
 *   s1 = soft(Psi^dagger x + z1, gamma w), z1 += Psi^dagger x - s1;
 *   s2_i = proj onto the ball B(y_i/nu, eps_i/nu) of Phi_i x/nu + z2_i, z2 += Phi x/nu - s2;
 *   s3 = max(x + z3, 0), z3 += x - s3;
 *   x = CG solution of (2 I + Re Phi^H Phi/nu^2) x = Psi(s1 - z1) + Re Phi^H(s2 - z2)/nu + s3 - z3.
 * Synchronous at the end (stats). Errors: EINVAL, ENAN, ENOTCONV, ECUDA. */
purify_status purify_sdmm_solve(purify_plan *plan, const void *y, const double *eps,
                                const void *w, void *x, const purify_sdmm_params *params,
                                purify_sdmm_stats *stats);

/* Advance the state of the last purify_sdmm_solve on this plan by `iters`
 * further SDMM iterations (same y, eps, w, gamma, nu and CG settings),
 * asynchronously on the plan's stream and without computing statistics.
 * Without kernel timing enabled the iteration runs as a captured CUDA graph
 * (captured on first use and whenever gamma, nu, w or the CG count change).
 * The iterate stays on the device; purify_sdmm_solve with resume = 1 and
 * max_iter = 0 returns it with statistics. Errors: EINVAL if no solve was
 * started on the plan. */
purify_status purify_sdmm_iterate(purify_plan *plan, int32_t iters);

/* purify_sdmm_iterate for a solve started with block_groups = G: iteration i
 * uses group groups[i] (HOST, iters entries in [0, G); NULL => round-robin
 * from the iterations done), each group's iteration a replay of its own
 * captured graph. On a solve without groups it is purify_sdmm_iterate.
 * Errors: EINVAL (no started solve, group out of range). */
purify_status purify_sdmm_iterate_groups(purify_plan *plan, int32_t iters, const int32_t *groups);

/* Block-sharded SDMM (Sec. 1: the block split of Eqs. 2-3 and SDMM's parallel
 * structure): each shard (a process, a GPU, or several plans of one process)
 * holds a plan over its own blocks of the data, y_k, eps_k, and the shards run
 * the same iteration on replicated x, wavelet and positivity state. The only
 * data exchanged are N-pixel images, summed over the shards by the caller
 * (for example an NCCL all-reduce) at two points:
 *   per iteration:  purify_shard_iterate_local(r_out)  -> sum r over shards ->
 *                   purify_shard_cg_begin(r_sum);
 *   per CG step k:  purify_shard_cg_apply(k, u_out)     -> sum u over shards ->
 *                   purify_shard_cg_combine(k, u_sum);
 *   then            purify_shard_iterate_end(cg_steps).
 * r_out = Re Phi_k^H (s2_k - z2_k - Phi_k x / nu) / nu (this shard's blocks, after
 * their projections and multiplier updates); u_out = Re Phi_k^H Phi_k r / nu^2 for
 * the current CG residual r (after step k - 1's update); cg_combine forms
 * u = 2 r + u_sum, the dot products and the step's scalars, identically on every
 * shard. With one shard the sequence is one iteration of purify_sdmm_solve.
 * Start every shard with purify_sdmm_solve(max_iter = 0) on its own y_k and eps_k
 * with the SAME gamma, nu (> 0) and x, w on all shards; read statistics with
 * purify_sdmm_solve(resume = 1, max_iter = 0) (objective: any shard; residual
 * ratio: max over shards). All images are DEVICE [ny][nx] real (dtype), owned by
 * the caller; calls are asynchronous on the plan's stream. Not with
 * block_groups or toeplitz. Errors: EINVAL (no started solve, host pointer,
 * negative step), ECUDA. */
purify_status purify_shard_iterate_local(purify_plan *plan, void *r_out);
purify_status purify_shard_cg_begin(purify_plan *plan, const void *r_sum);
purify_status purify_shard_cg_apply(purify_plan *plan, int32_t step, void *u_out);
purify_status purify_shard_cg_combine(purify_plan *plan, int32_t step, const void *u_sum);
purify_status purify_shard_iterate_end(purify_plan *plan, int32_t cg_steps);

/* Primal-dual solver for problem (3) without an inner CG (the paper's SDMM
 * family; Chambolle & Pock 2011, Algorithm 1 with theta = 1) on
 *   min_x  i_{R_+^N}(x) + ||W v||_1 + sum_i i_{B(y_i/nu, eps_i/nu)}(s_i),
 *   (v, s) = K x,  K = [Psi^dagger; Phi/nu],
 * with complex blocks taken as real vectors, so K^*(v, s) = Psi v + Re Phi^H s/nu
 * and ||K||^2 <= 2. From x_0 = x (input), xbar = x, p1 = 0, p2 = 0, each
 * iteration does
 *   p1 = clip(p1 + sigma Psi^dagger xbar, -w, w);
 *   q = p2 + sigma Phi xbar/nu,  p2_i = q_i - sigma proj_{B(y_i/nu, eps_i/nu)}(q_i/sigma);
 *   x_new = max(x - tau (Psi p1 + Re Phi^H p2/nu), 0);  xbar = 2 x_new - x;  x = x_new.
 * The iterations run as replays of a captured CUDA graph. It uses the plan's
 * solver state, so a previously started purify_sdmm_solve can no longer be
 * resumed afterwards. stats (HOST, may be NULL) are evaluated at the returned
 * x (cg_iters_total = 0, gamma = 0, rel_change = 0). Synchronous.
 * Errors: EINVAL (null y, eps or x; eps not positive; tau or sigma not finite),
 * ENAN (non-finite visibilities), ECUDA. */
typedef struct {
    int32_t iters;      /* primal-dual iterations (exact count, >= 0) */
    double tau;         /* primal step; <= 0 => 0.05 */
    double sigma;       /* dual step; <= 0 => 9.8 (tau sigma ||K||^2 < 1 for the defaults) */
    double nu;          /* data-term scale ||Phi||_2; <= 0 => 100 power iterations */
} purify_pd_params;

purify_status purify_pd_solve(purify_plan *plan, const void *y, const double *eps, const void *w,
                              void *x, const purify_pd_params *params, purify_sdmm_stats *stats);

/* Batched channels: independent problems (one plan each, e.g. the spectral
 * channels of one observation) advanced together. Every plan must already
 * hold a started solve (purify_sdmm_solve). purify_batch_iterate runs
 * `iters` SDMM iterations of every plan as replays of one captured CUDA
 * graph whose branches (one per plan, on private streams) run concurrently;
 * the graph is re-captured when a plan's gamma, nu, weights or CG count
 * change. Ordered after and before work already queued on `stream`.
 * Plans stay usable on their own; do not use them concurrently with the batch. */
typedef struct purify_batch purify_batch;
purify_status purify_batch_create(purify_plan *const *plans, int32_t n, void *stream, purify_batch **out);
purify_status purify_batch_iterate(purify_batch *batch, int32_t iters);
purify_status purify_batch_destroy(purify_batch *batch);

/* SARA weights (Sec. 1, reweighted l1): w = rho / (rho + |Psi^dagger x|),
 * x real [ny][nx], w real [q][ny][nx]; rho > 0. */
purify_status purify_reweight(purify_plan *plan, const void *x, double rho, void *w);

/* Problem set-up on the host (Sec. 1, Eq. 3: eps_i bounds the norm of block
 * i's noise; the paper only asks for an appropriate bound). Reading used:
 * complex noise n_m = sigma (a + i b) / sqrt 2 with a, b ~ N(0, 1), so
 * (2 / sigma^2) ||n_i||^2 is chi^2 with 2 M_i degrees of freedom, and eps_i is
 * its mean plus two standard deviations:
 *   eps_i = (sigma / sqrt 2) sqrt(2 M_i + 4 sqrt(M_i)),  M_i = offsets[i+1] - offsets[i].
 * purify_noise_sigma gives sigma = y_norm / sqrt(M) * 10^(-snr_db / 20) for a
 * noiseless ||Phi x|| = y_norm and an input SNR in dB.
 * block_offsets: HOST int64 [R + 1] (0 = first < ... < last), eps: HOST double [R].
 * Errors: EINVAL (null pointers, R < 1, offsets not increasing, sigma <= 0 or
 * not finite, M < 1). Synchronous, no GPU work. */
purify_status purify_noise_sigma(double y_norm, int64_t M, double snr_db, double *sigma);
purify_status purify_chi2_epsilon(double sigma, const int64_t *block_offsets, int32_t R, double *eps);

/* Standard deviation of Psi^dagger x over all D coefficients (FP64 reduction),
 * the first SARA reweighting scale. Synchronous. */
purify_status purify_coef_std(purify_plan *plan, const void *x, double *std_out);

/* Allocation-free Psi^dagger, for callers that cannot call cudaMalloc: code
 * that runs inside a host callback enqueued on a CUDA stream (CUDA API calls
 * that allocate are not allowed there), programs whose device memory is
 * reserved up front by another allocator, and latency-critical loops that
 * must not allocate after start-up because cudaMalloc can synchronise the
 * device. The paper has no counterpart; this is a service entry point.
 *   x  real [ny][nx] DEVICE pointer (dtype), input
 *   c  real [q][ny][nx] DEVICE pointer (dtype), output, layout as purify_psi_adj
 *   nx, ny, levels, basis_mask  as in purify_plan_desc (mask 0 => 0x1FF)
 *   stream  cudaStream_t (NULL = legacy default stream)
 * No plan is needed and nothing is allocated: the wavelet low-pass scratch
 * is a 4 MiB file-scope device array, and the basis table a 64-byte one,
 * that every GPU loading the library keeps until the process exits. Sizes
 * whose scratch exceeds the array are rejected with EINVAL: it needs
 * (number of wavelet bases) * (nx*ny/4 + nx*ny/16) * sizeof(dtype) bytes,
 * e.g. up to 512 x 512 in FP32 or 512 x 256 in FP64 with all eight
 * wavelets. The first call on each device looks up the arrays' device
 * addresses and uploads the constant filter tables (both synchronous), so
 * make that first call before any stream capture. All calls share the one
 * array and it keeps the previous call's contents; calls that may overlap on
 * the GPU (different streams, or different host threads) race on it and must
 * be ordered by the caller.
 * Errors: EINVAL (sizes, host pointers), ECUDA. */
purify_status purify_psi_adj_static(const void *x, void *c, int32_t nx, int32_t ny, int32_t levels,
                                    uint32_t basis_mask, purify_dtype dtype, void *stream);

/* Learned warm start building block (the paper has no learned component;
 * the U-Net only changes SDMM's starting point): 'same' k x k convolution
 * (k = 1 or 3, zero padding, cross-correlation) of x [B][H][W][Cin] (NHWC,
 * FP32, DEVICE) with w [Cout][k][k][Cin] (FP32, DEVICE) and bias [Cout]
 * (DEVICE or NULL), optional ReLU, into out [B][H][W][Cout] (FP32, DEVICE).
 * x and w are rounded to BF16 and multiplied on the tensor cores (tcgen05)
 * with FP32 accumulation. Cout <= 256. Synchronous; allocates staging.
 * Errors: EINVAL (shape), ETIMEOUT (a bounded device wait gave up), ECUDA. */
purify_status purify_conv2d(const float *x, int32_t B, int32_t H, int32_t W, int32_t Cin, const float *w,
                            const float *bias, int32_t Cout, int32_t k, int32_t relu, float *out, void *stream);

/* Learned warm-start network (not in the paper): a U-Net of `levels` levels
 * and base width `base` on H x W single-channel images (NHWC with C = 1),
 * BF16 tensor-core convolutions with FP32 accumulation, FP32 parameters,
 * gradients and Adam state. Architecture per level: conv3x3+ReLU twice,
 * 2x2 max pooling (encoder); x2 upsampling + conv3x3+ReLU, concatenation with
 * the skip, conv3x3+ReLU twice (decoder); 1x1 head added to the input.
 * Parameters are one FP32 vector, layer by layer (weights [Cout][k][k][Cin]
 * then biases), layers in the order e0a, e0b, e1a, ..., ba, bb, then for
 * each decoder level from the deepest: du, da, db; head last.
 * Images x, y, targets are DEVICE FP32 [B][H][W], B <= max_batch. */
typedef struct purify_unet purify_unet;
purify_status purify_unet_create(int32_t H, int32_t W, int32_t levels, int32_t base, int32_t max_batch,
                                 uint64_t seed, void *stream, purify_unet **out);
purify_status purify_unet_destroy(purify_unet *net);
int64_t purify_unet_num_params(const purify_unet *net);
/* Copy the parameter vector out / in (host or device pointers). */
purify_status purify_unet_get_params(purify_unet *net, float *out);
purify_status purify_unet_set_params(purify_unet *net, const float *in);
/* y = net(x); asynchronous. */
purify_status purify_unet_forward(purify_unet *net, const float *x, float *y, int32_t B);
/* Mean-squared-error loss against `target` and its gradient with respect to
 * every parameter (copied to grads, host or device, when not NULL);
 * synchronous, loss to *loss (host) when not NULL. */
purify_status purify_unet_gradients(purify_unet *net, const float *x, const float *target, int32_t B, float *grads,
                                    double *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the batch; asynchronous
 * unless loss (host) is requested. */
purify_status purify_unet_train_step(purify_unet *net, const float *x, const float *target, int32_t B, float lr,
                                     double *loss);

/* Per-kernel device timing for profiling: when enabled, every kernel launch
 * of the plan is bracketed by CUDA events on the plan's stream. */
purify_status purify_timing_enable(purify_plan *plan, int32_t enable);
/* Fill up to `cap` entries (name, launches, total milliseconds) accumulated
 * since the last reset; returns the number of kernel kinds. Synchronous. */
typedef struct { char name[32]; int64_t launches; double total_ms; } purify_kernel_time;
int32_t purify_timing_read(purify_plan *plan, purify_kernel_time *out, int32_t cap, int32_t reset);

/* Number of kernels this library launched on any plan since load. */
int64_t purify_launch_count(void);

/* Thread-local message of the last failed call ("" if none). */
const char *purify_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PURIFY_H */
