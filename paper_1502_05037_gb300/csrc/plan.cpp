// Plan construction: validation, host tables, visibility sort and the
// gridding work list.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "host_tables.h"
#include "internal.h"

namespace purify {

static const double kTwoPi = 6.28318530717958647692528676655900577;

void DevBuf::alloc(size_t b) {
    release();
    if (b == 0) b = 16;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        throw Error{PURIFY_ENOMEM, std::string("cudaMalloc of ") + std::to_string(b) + " bytes failed: " +
                                       cudaGetErrorString(e)};
    }
    bytes = b;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

bool is_host_pointer(const void* ptr) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

template <typename T> static void upload(DevBuf& b, const std::vector<T>& v) {
    b.alloc(v.size() * sizeof(T));
    PURIFY_CUDA(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

template <typename T> static std::vector<T> cast_vec(const std::vector<double>& v) {
    std::vector<T> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
    return o;
}

// Grid cell of each visibility's first tap (wrapped), as computed by the
// kernels.
template <typename T>
static void first_tap_cells(purify_plan* p, const std::vector<T>& u, const std::vector<T>& v, std::vector<int>& cx,
                            std::vector<int>& cy) {
    cx.resize(p->M);
    cy.resize(p->M);
    for (int64_t m = 0; m < p->M; ++m) {
        int kx0, ky0;
        T phx, phy;
        split_coord(u[m], p->ax, p->J, kx0, phx);
        split_coord(v[m], p->ay, p->J, ky0, phy);
        cx[m] = kx0 & (p->Kx - 1);
        cy[m] = ky0 & (p->Ky - 1);
    }
}

// Sort the visibilities of each block by a hierarchical tile key: the
// tmax-tile index, then the quadrant at each halving down to tmin. Every
// power-of-two tile size between tmin and tmax then covers a contiguous run
// of the sorted order, so candidate gridding tiles can be compared without
// re-sorting. Stable (counting sort), so the order is deterministic.
static void sort_hierarchical(purify_plan* p, const std::vector<int>& cx, const std::vector<int>& cy, int tmin,
                              int tmax, std::vector<int>& perm) {
    const int64_t M = p->M;
    const int nkeys = (p->Kx / tmin) * (p->Ky / tmin);
    std::vector<int> key(M);
    for (int64_t m = 0; m < M; ++m) {
        int k = (cy[m] / tmax) * (p->Kx / tmax) + cx[m] / tmax;
        for (int t = tmax / 2; t >= tmin; t /= 2) k = k * 4 + ((cy[m] / t) & 1) * 2 + ((cx[m] / t) & 1);
        key[m] = k;
    }
    perm.resize(M);
    std::vector<int64_t> count(nkeys + 1);
    for (int r = 0; r < p->R; ++r) {
        const int64_t a = p->offsets[r], b = p->offsets[r + 1];
        std::fill(count.begin(), count.end(), 0);
        for (int64_t m = a; m < b; ++m) count[key[m] + 1]++;
        for (int k = 0; k < nkeys; ++k) count[k + 1] += count[k];
        for (int64_t m = a; m < b; ++m) perm[a + count[key[m]]++] = (int)m;
        // inside each finest tile, order by grid cell (then by index), so that
        // visibilities sharing a first tap are adjacent
        int64_t i = a;
        while (i < b) {
            int64_t j = i;
            const int k0 = key[perm[i]];
            while (j < b && key[perm[j]] == k0) ++j;
            if (j - i > 1)
                std::sort(perm.begin() + i, perm.begin() + j, [&](int x, int y) {
                    const int cx1 = (cy[x] % tmin) * tmin + cx[x] % tmin, cx2 = (cy[y] % tmin) * tmin + cx[y] % tmin;
                    return cx1 != cx2 ? cx1 < cx2 : x < y;
                });
            i = j;
        }
    }
}

// Gridding/degridding work: every visibility of a tile (from all measurement
// blocks) in first-tap-cell order, cut into subproblems of at most `units`
// times the gridding kernel's batch unit and listed largest first, so that
// the longest blocks are scheduled first. cell_order is the internal indices
// sorted by first-tap cell (stable), so a stable pass by tile keeps the cell
// order inside each tile.
void build_gridlist(purify_plan* p, const std::vector<int>& bins, const std::vector<int>& cell_order, int tile,
                    int units, GridWork& w) {
    w.tile = tile;
    w.tiles_x = p->Kx / tile;
    w.tiles_y = p->Ky / tile;
    const int nbins = w.tiles_x * w.tiles_y;
    const int64_t M = p->M;
    std::vector<int64_t> start(nbins + 1, 0);
    for (int64_t m = 0; m < M; ++m) start[bins[m] + 1]++;
    for (int b = 0; b < nbins; ++b) start[b + 1] += start[b];
    std::vector<int> order(M);
    {
        std::vector<int64_t> pos(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < M; ++i) {
            const int m = cell_order[i];
            order[pos[bins[m]]++] = m;
        }
    }
    w.units = units;
    const int64_t CMAX = (int64_t)units * grid_list_unit(p->dtype, p->J);
    struct Sub { int bin; int64_t start; int len; };
    std::vector<Sub> subs;
    for (int b = 0; b < nbins; ++b)
        for (int64_t s = start[b]; s < start[b + 1]; s += CMAX)
            subs.push_back({b, s, (int)std::min<int64_t>(CMAX, start[b + 1] - s)});
    std::stable_sort(subs.begin(), subs.end(), [](const Sub& a, const Sub& b) { return a.len > b.len; });
    std::vector<int> list(M), sub_bin, sub_off;
    int64_t q = 0;
    for (const Sub& sb : subs) {
        sub_bin.push_back(sb.bin);
        sub_off.push_back((int)q);
        std::copy(order.begin() + sb.start, order.begin() + sb.start + sb.len, list.begin() + q);
        q += sb.len;
    }
    sub_off.push_back((int)q);
    w.nsub = (int)subs.size();
    upload(w.sub_bin, sub_bin);
    upload(w.sub_off, sub_off);
    upload(w.list, list);
}

// ---------------------------------------------------------------- autotuner
// Launch shapes picked by timing on the plan's own data: the tile and the
// subproblem size of gridding and of degridding (work lists rebuilt from the
// same cell order) and the rows/columns per block of the FFT passes. Results
// are cached per problem shape.
struct TuneKey {
    int nx, ny, J, dtype, mlog, R, gm;
    bool operator<(const TuneKey& o) const {
        return std::tie(nx, ny, J, dtype, mlog, R, gm) < std::tie(o.nx, o.ny, o.J, o.dtype, o.mlog, o.R, o.gm);
    }
};
struct TuneVal { int tile, dtile, rb, cb, cw, units, dunits, gkind, dkind, nkind; };
static std::mutex g_tune_mutex;
static std::map<TuneKey, TuneVal> g_tune_cache;

// Mean device time of one call of f, which launches work on p->stream: the
// calls are captured `reps` times into a CUDA graph on a private stream (so
// host launch overhead does not count), and the best of three graph launches
// after an untimed one is taken (the minimum discards runs disturbed by clock
// ramps or other work on the device).
static float time_ms(purify_plan* p, const std::function<void()>& f, int reps) {
    cudaStream_t user = p->stream, ts = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    float best = 1e30f;
    auto cleanup = [&] {
        p->stream = user;
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (ts) cudaStreamDestroy(ts);
    };
    try {
        PURIFY_CUDA(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
        PURIFY_CUDA(cudaEventCreate(&a));
        PURIFY_CUDA(cudaEventCreate(&b));
        PURIFY_CUDA(cudaDeviceSynchronize());
        p->stream = ts;
        f();  // outside the capture: sets kernel attributes
        PURIFY_CUDA(cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal));
        try {
            for (int i = 0; i < reps; ++i) f();
        } catch (...) {
            cudaStreamEndCapture(ts, &g);
            throw;
        }
        PURIFY_CUDA(cudaStreamEndCapture(ts, &g));
        PURIFY_CUDA(cudaGraphInstantiate(&ge, g, 0));
        PURIFY_CUDA(cudaGraphLaunch(ge, ts));
        for (int trial = 0; trial < 3; ++trial) {
            PURIFY_CUDA(cudaEventRecord(a, ts));
            PURIFY_CUDA(cudaGraphLaunch(ge, ts));
            PURIFY_CUDA(cudaEventRecord(b, ts));
            PURIFY_CUDA(cudaEventSynchronize(b));
            float ms = 0.f;
            PURIFY_CUDA(cudaEventElapsedTime(&ms, a, b));
            best = std::min(best, ms / reps);
        }
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
    return best;
}

template <typename T, typename BinsFor>
static void autotune(purify_plan* p, const std::vector<int>& cand, BinsFor bins_for,
                     const std::vector<int>& cell_order, bool tune) {
    using C = typename cplx_of<T>::type;
    int mlog = 0;
    while ((int64_t(1) << (mlog + 1)) <= p->M) ++mlog;
    TuneKey key{p->nx, p->ny, p->J, p->dtype, mlog, std::min(p->R, 64), p->desc.grid_mode};
    // default subproblem size: about four subproblems per SM's worth of
    // visibilities, in batch units
    const int64_t unit = grid_list_unit(p->dtype, p->J);
    const int u0 = (int)std::max<int64_t>(1, std::min<int64_t>(16, (p->M / (152 * 4) + unit / 2) / unit));
    TuneVal val{p->work.tile, p->work.tile, 0, 0, 0, u0, u0, 1, 1, 2};
    bool cached = false;
    if (tune) {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { val = it->second; cached = true; }
    }
    if (tune && !cached) {
        // deterministic test data in the workspaces
        std::vector<T> img(2 * (size_t)p->N), vis(2 * (size_t)p->M);
        uint64_t st = 12345;
        auto rnd = [&]() { st = st * 6364136223846793005ull + 1442695040888963407ull; return (T)((double)(st >> 11) * 0x1.0p-53 - 0.5); };
        for (auto& x : img) x = rnd();
        for (auto& x : vis) x = rnd();
        PURIFY_CUDA(cudaMemcpy(p->tmp_img.p, img.data(), sizeof(T) * img.size(), cudaMemcpyHostToDevice));
        PURIFY_CUDA(cudaMemcpy(p->tmp_vis.p, vis.data(), sizeof(T) * vis.size(), cudaMemcpyHostToDevice));
        T* ximg = p->tmp_img.as<T>();
        C* yv = p->tmp_vis.as<C>();
        // bring the clocks up before the first candidate is timed
        for (int i = 0; i < 40; ++i) launch_cols_fwd(p, nullptr);
        PURIFY_CUDA(cudaStreamSynchronize(p->stream));
        // FFT launch shapes
        float best = 1e30f;
        for (int rb = 1; rb <= 8; rb *= 2) {
            if (p->ny % rb || !fft_shape_ok(rb, p->Kx, p->dtype)) continue;
            p->fft_rb = rb;
            float ms = time_ms(p, [&] { launch_scale_pad_rows(p, ximg, 1.0, nullptr); }, 10);
            if (ms < best) { best = ms; val.rb = rb; }
        }
        best = 1e30f;
        // columns per block, and one or two (packed FP32) columns per thread
        for (int cb = 1; cb <= 8; cb *= 2) {
            for (int cw = 1; cw <= 2; ++cw) {
                if (p->Kx % cb || !fft_shape_ok(cb, p->Ky, p->dtype, cw)) continue;
                p->fft_cb = cb;
                p->fft_cw = cw;
                float ms = time_ms(p, [&] { launch_cols_fwd(p, nullptr); }, 10);
                if (ms < best) { best = ms; val.cb = cb; val.cw = cw; }
            }
        }
        p->fft_rb = val.rb;
        p->fft_cb = val.cb;
        p->fft_cw = val.cw;
        // gridding and degridding tiles, each timed on its own kernel
        if (cand.size() > 1 && p->M >= 32768) {
            float bg = 1e30f, bd = 1e30f;
            for (int t : cand) {
                const std::vector<int> bins = bins_for(t);
                for (int u : {1, 2, 4, 8}) {
                    build_gridlist(p, bins, cell_order, t, u, p->work);
                    build_gridlist(p, bins, cell_order, t, u, p->dwork);
                    float mg = time_ms(p, [&] { launch_grid(p, yv, false, nullptr); }, 5);
                    float md = time_ms(p, [&] { launch_degrid(p, yv, false, nullptr); }, 5);
                    if (mg < bg) { bg = mg; val.tile = t; val.units = u; }
                    if (md < bd) { bd = md; val.dtile = t; val.dunits = u; }
                }
            }
            // gridding by run sets, and G^H, G and G^H G by lanes (one pool,
            // or by tiles of each candidate edge); the normal operator by
            // run sets or lanes
            if (p->desc.grid_mode == 0) {
                const float mr = time_ms(p, [&] { launch_grid_sets(p, yv, false, nullptr); }, 5);
                if (mr < bg) { bg = mr; val.gkind = 2; }
                float bn = time_ms(p, [&] { launch_normal_lanes(p, 2, nullptr); }, 5);
                if (lane_work_ok(p)) {
                    for (int kind = 3; kind <= 5; ++kind) {
                        const float mn = time_ms(p, [&] { launch_normal_lanes(p, kind, nullptr); }, 5);
                        const float ml = time_ms(p, [&] { launch_grid_lanes(p, kind, yv, false, nullptr); }, 5);
                        const float mdl = time_ms(p, [&] { launch_degrid_lanes(p, kind, yv, false, nullptr); }, 5);
                        if (mn < bn) { bn = mn; val.nkind = kind; }
                        if (ml < bg) { bg = ml; val.gkind = kind; }
                        if (mdl < bd) { bd = mdl; val.dkind = kind; }
                    }
                }
            }
        }
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[key] = val;
    }
    p->fft_rb = val.rb;
    p->fft_cb = val.cb;
    p->fft_cw = val.cw;
    // a forced decomposition: grid_mode 1 and 2 degrid by tiles and apply
    // G^H G by run sets, 3..5 do all three by that lane form, 6 grids by
    // the deterministic lane pairs and degrids by the lane pairs
    const int gm = p->desc.grid_mode;
    p->grid_kind = gm == 0 ? val.gkind : gm;
    p->degrid_kind = gm == 0 ? val.dkind : (gm == 6 ? 4 : (gm >= 3 ? gm : 1));
    p->normal_kind = gm == 0 ? val.nkind : (gm >= 3 ? gm : 2);
    build_gridlist(p, bins_for(val.tile), cell_order, val.tile, val.units, p->work);
    build_gridlist(p, bins_for(val.dtile), cell_order, val.dtile, val.dunits, p->dwork);
}

// Lane-per-run work (see LaneWork) from the length-sorted runs: `width`
// runs per set, each set padded to its longest run; with tile > 0 the runs
// are grouped by grid tile first (stable, so by length within a tile).
struct HostRun { int cell; int64_t first; int len; };
template <typename Rec>
static void build_lanework(purify_plan* p, const std::vector<HostRun>& runs, const std::vector<Rec>& rec,
                           const std::vector<int>& start, const std::vector<int>& perm, int width, int tile,
                           LaneWork& w, bool det = false) {
    const size_t nr = runs.size();
    std::vector<int> order(nr);
    std::iota(order.begin(), order.end(), 0);
    if (tile > 0) {
        const int tx = p->Kx / tile;
        auto bin = [&](int r) {
            const int cx = runs[r].cell & 0xFFFF, cy = runs[r].cell >> 16;
            return (cy / tile) * tx + cx / tile;
        };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bin(a) < bin(b); });
    }
    const int nsets = (int)((nr + width - 1) / width);
    std::vector<int2> set_info(nsets), run_cl((size_t)nsets * width, make_int2(0, 0));
    int64_t rows = 0;
    for (int s = 0; s < nsets; ++s) {
        int lmax = 0;
        for (int l = 0; l < width; ++l) {
            const size_t q = (size_t)s * width + l;
            if (q < nr) {
                const HostRun& hr = runs[order[q]];
                run_cl[q] = make_int2(hr.cell, hr.len);
                lmax = std::max(lmax, hr.len);
            }
        }
        set_info[s] = make_int2((int)rows, lmax);
        rows += lmax;
    }
    PURIFY_REQUIRE(rows * width < ((int64_t)1 << 31), "too many visibility records for the lane work");
    PURIFY_REQUIRE(width == 32 || width == 16, "lane work width must be 32 or 16");
    // record row layout: width 32, (phx, phy) per run; width 16, the 16
    // runs' phx then their phy (each lane of a pair reads its own axis)
    std::vector<float> lrec((size_t)rows * 2 * width, 0.f);   // 8 bytes per record
    std::vector<int> lidx((size_t)rows * width, -1), lcal((size_t)rows * width, -1);
    for (int s = 0; s < nsets; ++s)
        for (int l = 0; l < width; ++l) {
            const size_t q0 = (size_t)s * width + l;
            if (q0 >= nr) continue;
            const int r = order[q0];
            for (int k = 0; k < runs[r].len; ++k) {
                const Rec& e = rec[start[r] + k];
                const size_t row = (size_t)set_info[s].x + k, q = row * width + l;
                if (width == 32) {
                    lrec[2 * q] = (float)e.phx;
                    lrec[2 * q + 1] = (float)e.phy;
                } else {
                    lrec[row * 2 * width + l] = (float)e.phx;
                    lrec[row * 2 * width + width + l] = (float)e.phy;
                }
                lidx[q] = e.m;
                lcal[q] = perm[e.m];
            }
        }
    w.nsets = nsets;
    w.width = width;
    w.tile = tile;
    w.rows = rows;
    upload(w.set_info, set_info);
    upload(w.run_cl, run_cl);
    upload(w.rec, lrec);
    upload(w.idx, lidx);
    upload(w.idx_caller, lcal);
    w.cstart.release();
    w.clist.release();
    if (det) {
        // the runs of every first-tap cell in increasing run order (a
        // counting sort over the Kx Ky cells, stable in the run index)
        const int64_t ncell = (int64_t)p->Kx * p->Ky;
        std::vector<int> cstart(ncell + 1, 0), clist;
        auto cell_of = [&](const int2& rc) {
            return (int64_t)(((unsigned)rc.x >> 16) & (p->Ky - 1)) * p->Kx + ((rc.x & 0xFFFF) & (p->Kx - 1));
        };
        int64_t nreal = 0;
        for (size_t q = 0; q < run_cl.size(); ++q)
            if (run_cl[q].y > 0) { cstart[cell_of(run_cl[q]) + 1]++; ++nreal; }
        for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
        clist.assign((size_t)std::max<int64_t>(1, nreal), 0);
        std::vector<int> fill(cstart.begin(), cstart.end() - 1);
        for (size_t q = 0; q < run_cl.size(); ++q)
            if (run_cl[q].y > 0) clist[fill[cell_of(run_cl[q])]++] = (int)q;
        upload(w.cstart, cstart);
        upload(w.clist, clist);
        // one patch slot per run of the lane work, J x J taps each; sized by
        // the plan's own lane work (a block group has no more runs than the
        // whole plan), never reallocated under captured graphs
        const size_t need = sizeof(float2) * (size_t)p->J * p->J * run_cl.size();
        if (p->det_patch.bytes == 0) p->det_patch.alloc(need);
        PURIFY_REQUIRE(need <= p->det_patch.bytes, "deterministic lane work larger than the plan's patch buffer");
    }
}

// Run-ordered work (see RunWork): runs of equal first-tap cell in the cell
// order, cut at kRunMax visibilities, sorted by length (longest first,
// stable), padded to a multiple of G; records in run order.
static const int kRunMax = 48;
template <typename T>
static void build_runwork(purify_plan* p, const std::vector<T>& us, const std::vector<T>& vs,
                                const std::vector<int>& scx, const std::vector<int>& scy,
                                const std::vector<int>& cell_order, const std::vector<int>& perm) {
    using Rec = typename RunRecOf<T>::type;
    using Run = HostRun;
    std::vector<Run> runs;
    const int64_t M = p->M;
    int64_t i = 0;
    while (i < M) {
        const int m0 = cell_order[i];
        int64_t j = i + 1;
        while (j < M && j - i < kRunMax && scx[cell_order[j]] == scx[m0] && scy[cell_order[j]] == scy[m0]) ++j;
        runs.push_back({(scy[m0] << 16) | scx[m0], i, (int)(j - i)});
        i = j;
    }
    std::stable_sort(runs.begin(), runs.end(), [](const Run& a, const Run& b) { return a.len > b.len; });
    const int G = 32 / p->J;
    const size_t nr = (runs.size() + G - 1) / G * G;
    std::vector<int> cell(nr, 0), start(nr, 0), len(nr, 0);
    std::vector<Rec> rec(M);
    int64_t q = 0;
    for (size_t r = 0; r < runs.size(); ++r) {
        cell[r] = runs[r].cell;
        start[r] = (int)q;
        len[r] = runs[r].len;
        for (int k = 0; k < runs[r].len; ++k) {
            const int m = cell_order[runs[r].first + k];
            int kx0, ky0;
            Rec e{};
            split_coord(us[m], p->ax, p->J, kx0, e.phx);
            split_coord(vs[m], p->ay, p->J, ky0, e.phy);
            e.m = m;
            rec[q++] = e;
        }
    }
    if (sizeof(T) == 4 && p->J <= kLaneMaxJ) {
        build_lanework(p, runs, rec, start, perm, 32, 0, p->lanes[0]);
        build_lanework(p, runs, rec, start, perm, 16, 0, p->lanes[1], p->desc.grid_mode == 6);
        build_lanework(p, runs, rec, start, perm, 16, std::min(32, std::min(p->Kx, p->Ky)), p->lanes[2]);
    }
    p->runs.G = G;
    p->runs.nruns = (int)nr;
    p->runs.nsets = (int)(nr / G);
    upload(p->runs.rec, rec);
    upload(p->runs.cell, cell);
    upload(p->runs.start, start);
    upload(p->runs.len, len);
    p->workspace_bytes += (int64_t)(p->runs.rec.bytes + p->runs.cell.bytes + p->runs.start.bytes + p->runs.len.bytes);
}

// Lane work and visibility chunks of G block groups (block i in group
// i mod G), from the plan's sorted coordinates: per group, its visibilities
// in first-tap-cell order are cut into runs as for the whole plan (at most
// kRunMax, sorted by length), two lanes per run.
void build_group_lanes(purify_plan* p, int G) {
    PURIFY_REQUIRE(lane_work_ok(p), "block groups need an FP32 plan with kb_width <= 6");
    PURIFY_REQUIRE(G >= 1 && G <= p->R, "block_groups must be in [1, R]");
    if (p->group_count == G) return;
    p->group_lanes.clear();
    p->group_chunks.clear();
    p->group_count = 0;
    const int64_t M = p->M;
    std::vector<float> us(M), vs(M);
    std::vector<int> perm(M);
    PURIFY_CUDA(cudaMemcpy(us.data(), p->us.p, sizeof(float) * M, cudaMemcpyDeviceToHost));
    PURIFY_CUDA(cudaMemcpy(vs.data(), p->vs.p, sizeof(float) * M, cudaMemcpyDeviceToHost));
    PURIFY_CUDA(cudaMemcpy(perm.data(), p->perm.p, sizeof(int) * M, cudaMemcpyDeviceToHost));
    std::vector<int> cx(M), cy(M);
    std::vector<RunRecF> rec_of(M);
    for (int64_t m = 0; m < M; ++m) {
        int kx0, ky0;
        RunRecF e{};
        split_coord(us[m], p->ax, p->J, kx0, e.phx);
        split_coord(vs[m], p->ay, p->J, ky0, e.phy);
        e.m = (int)m;
        rec_of[m] = e;
        cx[m] = kx0 & (p->Kx - 1);
        cy[m] = ky0 & (p->Ky - 1);
    }
    p->group_lanes.resize(G);
    p->group_chunks.resize(G);
    for (int g = 0; g < G; ++g) {
        // the group's internal indices (blocks are contiguous internal ranges), by cell
        std::vector<int> idx;
        for (int r = g; r < p->R; r += G)
            for (int64_t m = p->offsets[r]; m < p->offsets[r + 1]; ++m) idx.push_back((int)m);
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            return std::make_pair(cy[a], cx[a]) < std::make_pair(cy[b], cx[b]);
        });
        std::vector<HostRun> runs;
        const int64_t n = (int64_t)idx.size();
        for (int64_t i = 0; i < n;) {
            const int m0 = idx[i];
            int64_t j = i + 1;
            while (j < n && j - i < kRunMax && cx[idx[j]] == cx[m0] && cy[idx[j]] == cy[m0]) ++j;
            runs.push_back({(cy[m0] << 16) | cx[m0], i, (int)(j - i)});
            i = j;
        }
        std::stable_sort(runs.begin(), runs.end(), [](const HostRun& a, const HostRun& b) { return a.len > b.len; });
        std::vector<RunRecF> rec((size_t)n);
        std::vector<int> start(runs.size());
        int64_t q = 0;
        for (size_t r = 0; r < runs.size(); ++r) {
            start[r] = (int)q;
            for (int k = 0; k < runs[r].len; ++k) rec[q++] = rec_of[idx[runs[r].first + k]];
        }
        build_lanework(p, runs, rec, start, perm, 16, 0, p->group_lanes[g], p->desc.grid_mode == 6);
        // the group's visibility chunks (the plan's chunking, blocks of the group only)
        const int64_t CH = 4096;
        std::vector<int> cb, cs, ce, cf(p->R + 1, 0);
        for (int r = 0; r < p->R; ++r) {
            cf[r] = (int)cb.size();
            if (r % G != g) continue;
            for (int64_t a = p->offsets[r]; a < p->offsets[r + 1]; a += CH) {
                cb.push_back(r);
                cs.push_back((int)a);
                ce.push_back((int)std::min(a + CH, p->offsets[r + 1]));
            }
        }
        cf[p->R] = (int)cb.size();
        GroupChunks& gc = p->group_chunks[g];
        gc.n = (int)cb.size();
        upload(gc.cblk, cb);
        upload(gc.cbeg, cs);
        upload(gc.cend, ce);
        upload(gc.chunk_first, cf);
    }
    p->group_count = G;
}

static int64_t lane_bytes(const LaneWork& w) {
    return (int64_t)(w.set_info.bytes + w.run_cl.bytes + w.rec.bytes + w.idx.bytes + w.idx_caller.bytes +
                     w.cstart.bytes + w.clist.bytes);
}

template <typename T> static void finish_plan(purify_plan* p) {
    using C = typename cplx_of<T>::type;
    const purify_plan_desc& d = p->desc;
    // correction tables and twiddles
    upload(p->sx, cast_vec<T>(correction_axis(p->nx, p->Kx, p->J, p->beta)));
    upload(p->sy, cast_vec<T>(correction_axis(p->ny, p->Ky, p->J, p->beta)));
    upload(p->onesx, std::vector<T>(p->nx, T(1)));
    upload(p->onesy, std::vector<T>(p->ny, T(1)));
    upload(p->twx, cast_vec<T>(twiddles(p->Kx)));
    upload(p->twy, cast_vec<T>(twiddles(p->Ky)));
    // coordinates to host
    std::vector<T> u(p->M), v(p->M);
    const size_t cb = sizeof(T) * p->M;
    PURIFY_CUDA(cudaMemcpy(u.data(), d.u, cb, cudaMemcpyDefault));
    PURIFY_CUDA(cudaMemcpy(v.data(), d.v, cb, cudaMemcpyDefault));
    for (int64_t m = 0; m < p->M; ++m) {
        if (!(std::isfinite((double)u[m]) && std::isfinite((double)v[m])))
            throw Error{PURIFY_EINVAL, "non-finite (u, v) coordinate"};
        if (std::fabs((double)u[m]) > 3.2 || std::fabs((double)v[m]) > 3.2)
            throw Error{PURIFY_EINVAL, "(u, v) outside [-pi, pi]"};
    }
    const int kmin = std::min(p->Kx, p->Ky);
    const int tmax = std::min(std::min(64, kmin), max_grid_tile(p->dtype, p->J));
    int tmin = std::min(16, tmax);
    if (d.tile > 0 && d.tile < tmin) tmin = std::max(8, d.tile);
    std::vector<int> cx, cy, perm;
    first_tap_cells<T>(p, u, v, cx, cy);
    sort_hierarchical(p, cx, cy, tmin, tmax, perm);
    std::vector<T> us(p->M), vs(p->M);
    for (int64_t i = 0; i < p->M; ++i) { us[i] = u[perm[i]]; vs[i] = v[perm[i]]; }
    upload(p->us, us);
    upload(p->vs, vs);
    upload(p->perm, perm);
    upload(p->d_offsets, p->offsets);
    std::vector<int> scx(p->M), scy(p->M);
    for (int64_t i = 0; i < p->M; ++i) { scx[i] = cx[perm[i]]; scy[i] = cy[perm[i]]; }
    auto bins_for = [&](int t) {
        std::vector<int> bins(p->M);
        const int tx = p->Kx / t;
        for (int64_t i = 0; i < p->M; ++i) bins[i] = (scy[i] / t) * tx + scx[i] / t;
        return bins;
    };
    std::vector<int> cand;
    if (d.tile > 0) cand.push_back(std::max(tmin, std::min(d.tile, tmax)));
    else for (int t = tmin; t <= tmax; t *= 2) cand.push_back(t);
    p->work.tile = cand.size() == 1 ? cand[0] : 32;
    if (std::find(cand.begin(), cand.end(), p->work.tile) == cand.end()) p->work.tile = cand.back();
    // visibility chunks for the per-block segmented reductions
    {
        const int64_t CH = 4096;
        std::vector<int> cb, cs, ce;
        for (int r = 0; r < p->R; ++r)
            for (int64_t a = p->offsets[r]; a < p->offsets[r + 1]; a += CH) {
                cb.push_back(r);
                cs.push_back((int)a);
                ce.push_back((int)std::min(a + CH, p->offsets[r + 1]));
            }
        p->nchunks = (int)cb.size();
        upload(p->chunk_blk, cb);
        upload(p->chunk_beg, cs);
        upload(p->chunk_end, ce);
    }
    // wavelet meta
    std::vector<int> meta(16, 0);
    int z = 0;
    for (size_t i = 0; i < p->bases.size(); ++i)
        if (p->bases[i] > 0) { meta[z] = p->bases[i]; meta[8 + z] = (int)i; ++z; }
    upload(p->wmeta, meta);
    init_filter_banks();
    // workspaces
    const int nw = z;
    p->grid.alloc(sizeof(C) * (size_t)p->Kx * p->Ky);
    p->gacc.alloc(sizeof(C) * (size_t)p->Kx * p->Ky + 256);
    p->rows.alloc(sizeof(C) * (size_t)p->ny * p->Kx);
    p->ll0.alloc(sizeof(T) * std::max<size_t>(1, (size_t)nw * p->N / 4));
    p->ll1.alloc(sizeof(T) * std::max<size_t>(1, (size_t)nw * p->N / 4));
    p->tmp_img.alloc(sizeof(C) * (size_t)p->N);
    p->tmp_vis.alloc(sizeof(C) * (size_t)p->M);
    p->workspace_bytes = (int64_t)(p->grid.bytes + p->gacc.bytes + p->rows.bytes + p->ll0.bytes + p->ll1.bytes + p->tmp_img.bytes +
                                   p->tmp_vis.bytes + p->us.bytes + p->vs.bytes + p->perm.bytes);
    // internal indices ordered by first-tap cell (stable counting sort)
    std::vector<int> cell_order(p->M);
    {
        const int64_t ncell = (int64_t)p->Kx * p->Ky;
        std::vector<int64_t> pos(ncell + 1, 0);
        for (int64_t i = 0; i < p->M; ++i) pos[(int64_t)scy[i] * p->Kx + scx[i] + 1]++;
        for (int64_t c = 0; c < ncell; ++c) pos[c + 1] += pos[c];
        for (int64_t i = 0; i < p->M; ++i) cell_order[pos[(int64_t)scy[i] * p->Kx + scx[i]]++] = (int)i;
    }
    build_runwork<T>(p, us, vs, scx, scy, cell_order, perm);
    autotune<T>(p, cand, bins_for, cell_order, d.tile == 0);
    // keep only the lane work in use (kind 6 runs on the lane pairs of kind 4)
    auto uses = [&](int k) {
        auto is = [&](int kind) { return kind == k || (k == 4 && kind == 6); };
        return is(p->grid_kind) || is(p->degrid_kind) || is(p->normal_kind);
    };
    for (int k = 3; k <= 5; ++k)
        if (!uses(k)) p->lanes[k - 3].release();
    for (int k = 0; k < 3; ++k) p->workspace_bytes += lane_bytes(p->lanes[k]);
    p->workspace_bytes += (int64_t)p->det_patch.bytes;
}

purify_plan* create_plan(const purify_plan_desc* d) {
    PURIFY_REQUIRE(d != nullptr, "null description");
    PURIFY_REQUIRE(is_pow2(d->nx) && is_pow2(d->ny) && d->nx >= 8 && d->ny >= 8 && d->nx <= 4096 && d->ny <= 4096,
                   "nx, ny must be powers of two in [8, 4096]");
    PURIFY_REQUIRE(d->M >= 1 && d->M < (int64_t)1 << 31, "M must be in [1, 2^31)");
    PURIFY_REQUIRE(d->u && d->v, "null u or v");
    PURIFY_REQUIRE(d->kb_width >= 2 && d->kb_width <= PURIFY_MAX_J, "kb_width must be in [2, 8]");
    PURIFY_REQUIRE(d->levels >= 1 && d->levels <= 8, "levels must be in [1, 8]");
    PURIFY_REQUIRE((d->nx >> d->levels) >= 1 && (d->ny >> d->levels) >= 1 && (d->nx >> d->levels) * 2 >= 2,
                   "image too small for the number of levels");
    PURIFY_REQUIRE(d->dtype == PURIFY_F32 || d->dtype == PURIFY_F64, "dtype must be PURIFY_F32 or PURIFY_F64");
    PURIFY_REQUIRE(d->R >= 1 && d->R <= d->M, "R must be in [1, M]");
    PURIFY_REQUIRE(d->R == 1 || d->block_offsets, "block_offsets required when R > 1");
    uint32_t mask = d->basis_mask ? d->basis_mask : 0x1FFu;
    PURIFY_REQUIRE((mask & ~0x1FFu) == 0, "basis_mask has bits above db8");
    double alpha = d->oversample > 0 ? d->oversample : 2.0;
    int64_t Kx = (int64_t)std::llround(alpha * d->nx), Ky = (int64_t)std::llround(alpha * d->ny);
    PURIFY_REQUIRE(std::fabs(alpha * d->nx - (double)Kx) < 1e-9 && is_pow2(Kx) && is_pow2(Ky) && Kx <= 8192 &&
                       Ky <= 8192 && Kx > d->nx && Ky > d->ny,
                   "oversample must make K = alpha n a power of two above n (at most 8192)");
    PURIFY_REQUIRE(d->tile == 0 || (is_pow2(d->tile) && d->tile >= 8 && d->tile <= 64), "tile must be 0 or a power of two in [8, 64]");
    PURIFY_REQUIRE(d->grid_mode >= 0 && d->grid_mode <= 6, "grid_mode must be in 0..6");
    PURIFY_REQUIRE(d->grid_mode < 3 || (d->dtype == PURIFY_F32 && d->kb_width <= kLaneMaxJ),
                   "grid_mode 3..6 (lanes) needs an FP32 plan with kb_width <= 6");
    std::vector<int64_t> offs;
    if (d->block_offsets) {
        offs.assign(d->block_offsets, d->block_offsets + d->R + 1);
        PURIFY_REQUIRE(offs[0] == 0 && offs[d->R] == d->M, "block_offsets must start at 0 and end at M");
        for (int r = 0; r < d->R; ++r) PURIFY_REQUIRE(offs[r + 1] > offs[r], "blocks must be non-empty and increasing");
    } else {
        offs = {0, d->M};
    }
    // every wavelet level must keep at least 2 samples per axis
    for (int b = 1; b <= 8; ++b)
        if (mask >> b & 1) PURIFY_REQUIRE((d->nx >> (d->levels - 1)) >= 2 && (d->ny >> (d->levels - 1)) >= 2,
                                          "image too small for the number of levels");

    purify_plan* p = new purify_plan();
    try {
        p->desc = *d;
        p->dtype = d->dtype;
        p->nx = d->nx;
        p->ny = d->ny;
        p->Kx = (int)Kx;
        p->Ky = (int)Ky;
        p->J = d->kb_width;
        p->levels = d->levels;
        p->M = d->M;
        p->N = (int64_t)d->nx * d->ny;
        p->R = d->R;
        p->mask = mask;
        for (int b = 0; b < 9; ++b) if (mask >> b & 1) p->bases.push_back(b);
        p->q = (int)p->bases.size();
        p->D = p->q * p->N;
        p->beta = d->kb_beta > 0 ? d->kb_beta : 2.34 * p->J;
        p->i0beta = bessel_i0_series(p->beta);
        p->stream = (cudaStream_t)d->stream;
        p->offsets = offs;
        double cx = (double)Kx / kTwoPi, cy = (double)Ky / kTwoPi;
        p->ax = AxisConst{(int)Kx, (float)cx, (float)(cx - (double)(float)cx), cx};
        p->ay = AxisConst{(int)Ky, (float)cy, (float)(cy - (double)(float)cy), cy};
        p->kbp = fit_kb_poly(p->J, p->beta, kb_poly_degree(p->J));
        if (p->dtype == PURIFY_F32) finish_plan<float>(p); else finish_plan<double>(p);
        p->desc.u = p->desc.v = nullptr;
        p->desc.block_offsets = nullptr;
        PURIFY_CUDA(cudaDeviceSynchronize());
    } catch (...) {
        delete p;
        throw;
    }
    return p;
}

}  // namespace purify
