// Plan construction: validation, host tables, visibility sort and the
// gridding work list.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
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

template <typename T>
static void sort_visibilities(purify_plan* p, const std::vector<T>& u, const std::vector<T>& v, int tile,
                              std::vector<int>& perm, std::vector<int>& bin_sorted) {
    const int64_t M = p->M;
    const int tx = p->Kx / tile, ty = p->Ky / tile, nbins = tx * ty;
    std::vector<int> bin(M);
    for (int64_t m = 0; m < M; ++m) {
        int kx0, ky0;
        T phx, phy;
        split_coord(u[m], p->ax, p->J, kx0, phx);
        split_coord(v[m], p->ay, p->J, ky0, phy);
        int bx = (kx0 & (p->Kx - 1)) / tile, by = (ky0 & (p->Ky - 1)) / tile;
        bin[m] = by * tx + bx;
    }
    perm.resize(M);
    bin_sorted.resize(M);
    std::vector<int64_t> count(nbins + 1);
    for (int r = 0; r < p->R; ++r) {
        const int64_t a = p->offsets[r], b = p->offsets[r + 1];
        std::fill(count.begin(), count.end(), 0);
        for (int64_t m = a; m < b; ++m) count[bin[m] + 1]++;
        for (int k = 0; k < nbins; ++k) count[k + 1] += count[k];
        for (int64_t m = a; m < b; ++m) {
            int64_t dst = a + count[bin[m]]++;
            perm[dst] = (int)m;
            bin_sorted[dst] = bin[m];
        }
    }
}

void build_gridwork(purify_plan* p, const std::vector<int>& bin_sorted, int tile) {
    GridWork& w = p->work;
    w.tile = tile;
    w.tiles_x = p->Kx / tile;
    w.tiles_y = p->Ky / tile;
    const int nbins = w.tiles_x * w.tiles_y;
    // pieces: maximal runs of one bin inside one block, grouped by bin
    std::vector<std::vector<std::pair<int, int>>> runs(nbins);
    const int64_t M = p->M;
    int64_t m = 0;
    for (int r = 0; r < p->R; ++r) {
        m = p->offsets[r];
        const int64_t end = p->offsets[r + 1];
        while (m < end) {
            int b = bin_sorted[m];
            int64_t s = m;
            while (m < end && bin_sorted[m] == b) ++m;
            runs[b].push_back({(int)s, (int)(m - s)});
        }
    }
    (void)M;
    const int CMAX = 2048;  // visibilities per subproblem
    std::vector<int> sub_bin, piece_off, pst, plen;
    for (int b = 0; b < nbins; ++b) {
        int in_sub = 0;
        bool open = false;
        for (auto run : runs[b]) {
            int s = run.first, len = run.second;
            while (len > 0) {
                if (!open || in_sub >= CMAX) {
                    sub_bin.push_back(b);
                    piece_off.push_back((int)pst.size());
                    in_sub = 0;
                    open = true;
                }
                int take = std::min(len, CMAX - in_sub);
                pst.push_back(s);
                plen.push_back(take);
                s += take;
                len -= take;
                in_sub += take;
            }
        }
    }
    piece_off.push_back((int)pst.size());
    w.nsub = (int)sub_bin.size();
    w.npieces = (int)pst.size();
    upload(w.sub_bin, sub_bin);
    upload(w.piece_off, piece_off);
    upload(w.piece_start, pst);
    upload(w.piece_len, plen);
}

template <typename T> static void finish_plan(purify_plan* p) {
    using C = typename cplx_of<T>::type;
    const purify_plan_desc& d = p->desc;
    // correction tables and twiddles
    upload(p->sx, cast_vec<T>(correction_axis(p->nx, p->Kx, p->J, p->beta)));
    upload(p->sy, cast_vec<T>(correction_axis(p->ny, p->Ky, p->J, p->beta)));
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
    int tile = d.tile > 0 ? d.tile : 32;
    tile = std::min(tile, std::min(p->Kx, p->Ky));
    std::vector<int> perm, bin_sorted;
    sort_visibilities<T>(p, u, v, tile, perm, bin_sorted);
    std::vector<T> us(p->M), vs(p->M);
    for (int64_t i = 0; i < p->M; ++i) { us[i] = u[perm[i]]; vs[i] = v[perm[i]]; }
    upload(p->us, us);
    upload(p->vs, vs);
    upload(p->perm, perm);
    upload(p->d_offsets, p->offsets);
    build_gridwork(p, bin_sorted, tile);
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
    p->rows.alloc(sizeof(C) * (size_t)p->ny * p->Kx);
    p->ll0.alloc(sizeof(T) * std::max<size_t>(1, (size_t)nw * p->N / 4));
    p->ll1.alloc(sizeof(T) * std::max<size_t>(1, (size_t)nw * p->N / 4));
    p->tmp_img.alloc(sizeof(C) * (size_t)p->N);
    p->tmp_vis.alloc(sizeof(C) * (size_t)p->M);
    p->workspace_bytes = (int64_t)(p->grid.bytes + p->rows.bytes + p->ll0.bytes + p->ll1.bytes + p->tmp_img.bytes +
                                   p->tmp_vis.bytes + p->us.bytes + p->vs.bytes + p->perm.bytes);
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
