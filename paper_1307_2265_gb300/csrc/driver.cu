// Native driver of a block-structured AMR hierarchy (paper Sec. 3): the plans
// of each level (sibling copy boxes, interpolated ghost regions, flux-correction
// face parts), the EvolveLevel W-cycle with subcycled finer levels, and the
// rebuild of finer levels from flagged cells (Sec. 3.5, 3.6).  Everything that
// touches the fields runs in the library's kernels through its own entry points
// (ghost fills, sweeps, CFL, flux correction, projection, flags); this file is
// host logic: plans, time bookkeeping and device memory.
//
// Plans are built by one rule for every layout: a patch's ghost-extended box
// against the other patches' active boxes (through a bucket index, so the cost
// grows with the number of neighbours, not with the square of the level size).
// On the tensor-product tilings of a static hierarchy that rule gives the same
// boxes, in the same order, as the lattice lookup those tilings allow.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <memory>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int NG = 3;
constexpr int RF = 2;   // refinement factor

int64_t floordiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// ---- plans ------------------------------------------------------------------

struct Box3 {
    int64_t lo[3], hi[3];
};

bool box_empty(const Box3 &b) { return !(b.lo[0] < b.hi[0] && b.lo[1] < b.hi[1] && b.lo[2] < b.hi[2]); }

Box3 box_and(const Box3 &a, const Box3 &b)
{
    Box3 r;
    for (int d = 0; d < 3; ++d) {
        r.lo[d] = std::max(a.lo[d], b.lo[d]);
        r.hi[d] = std::min(a.hi[d], b.hi[d]);
    }
    return r;
}

int64_t box_volume(const Box3 &b)
{
    if (box_empty(b)) return 0;
    return (b.hi[0] - b.lo[0]) * (b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]);
}

bool box_contains(const Box3 &outer, const Box3 &inner)
{
    for (int d = 0; d < 3; ++d)
        if (!(outer.lo[d] <= inner.lo[d] && inner.hi[d] <= outer.hi[d])) return false;
    return true;
}

// Boxes of one index space hashed into cubic buckets: candidates(q) lists, in
// ascending order, every box that may intersect q.
class BoxIndex {
public:
    explicit BoxIndex(const std::vector<Box3> &boxes) : boxes_(boxes)
    {
        int64_t ext = 1;
        for (const Box3 &b : boxes)
            for (int d = 0; d < 3; ++d) ext = std::max(ext, b.hi[d] - b.lo[d]);
        bucket_ = std::max<int64_t>(4, std::min<int64_t>(ext, 64));
        for (size_t i = 0; i < boxes.size(); ++i) {
            if (box_empty(boxes[i])) continue;
            for_buckets(boxes[i], [&](int64_t key) { map_[key].push_back((int)i); });
        }
    }
    void candidates(const Box3 &q, std::vector<int> &out) const
    {
        out.clear();
        for_buckets(q, [&](int64_t key) {
            auto it = map_.find(key);
            if (it != map_.end()) out.insert(out.end(), it->second.begin(), it->second.end());
        });
        std::sort(out.begin(), out.end());
        out.erase(std::unique(out.begin(), out.end()), out.end());
    }

private:
    template <class F>
    void for_buckets(const Box3 &b, F f) const
    {
        int64_t lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = floordiv(b.lo[d], bucket_);
            hi[d] = floordiv(b.hi[d] - 1, bucket_);
        }
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x)
                    f(((z & 0x1FFFFF) << 42) | ((y & 0x1FFFFF) << 21) | (x & 0x1FFFFF));
    }
    const std::vector<Box3> &boxes_;
    int64_t bucket_;
    std::unordered_map<int64_t, std::vector<int>> map_;
};

std::vector<Box3> active_boxes(const int32_t *n, const int32_t *origin, int np)
{
    std::vector<Box3> b(np);
    for (int i = 0; i < np; ++i)
        for (int d = 0; d < 3; ++d) {
            b[i].lo[d] = origin[3 * i + d];
            b[i].hi[d] = (int64_t)origin[3 * i + d] + n[3 * i + d];
        }
    return b;
}

enzo_copy_box make_box(int dst, int src, const Box3 &b)
{
    enzo_copy_box c;
    c.dst = dst;
    c.src = src;
    for (int d = 0; d < 3; ++d) {
        c.lo[d] = (int32_t)b.lo[d];
        c.hi[d] = (int32_t)b.hi[d];
    }
    return c;
}

// Ghost cells of each patch that lie in a sibling's active box, by (dst, src).
std::vector<enzo_copy_box> plan_siblings(const int32_t *n, const int32_t *origin, int np)
{
    const std::vector<Box3> act = active_boxes(n, origin, np);
    BoxIndex idx(act);
    std::vector<enzo_copy_box> out;
    std::vector<int> cand;
    for (int a = 0; a < np; ++a) {
        Box3 g = act[a];
        for (int d = 0; d < 3; ++d) {
            g.lo[d] -= NG;
            g.hi[d] += NG;
        }
        idx.candidates(g, cand);
        for (int b : cand) {
            if (b == a) continue;
            const Box3 x = box_and(g, act[b]);
            if (!box_empty(x)) out.push_back(make_box(a, b, x));
        }
    }
    return out;
}

// The 26 ghost regions of each patch (directions with z slowest, then y, then
// x, each of -1, 0, 1), except those lying wholly in one sibling's active box:
// these are interpolated from the parent, and the sibling copies that follow
// overwrite whatever part of them a sibling covers (Sec. 3.1).
std::vector<enzo_copy_box> plan_interp(const int32_t *n, const int32_t *origin, int np)
{
    const std::vector<Box3> act = active_boxes(n, origin, np);
    BoxIndex idx(act);
    std::vector<enzo_copy_box> out;
    std::vector<int> cand;
    for (int a = 0; a < np; ++a)
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz) continue;
                    const int dv[3] = {dx, dy, dz};
                    Box3 r;
                    for (int d = 0; d < 3; ++d) {
                        r.lo[d] = dv[d] < 0 ? act[a].lo[d] - NG : (dv[d] > 0 ? act[a].hi[d] : act[a].lo[d]);
                        r.hi[d] = dv[d] < 0 ? act[a].lo[d] : (dv[d] > 0 ? act[a].hi[d] + NG : act[a].hi[d]);
                    }
                    idx.candidates(r, cand);
                    bool inside = false;
                    for (int b : cand)
                        if (box_contains(act[b], r)) {
                            inside = true;
                            break;
                        }
                    if (!inside) out.push_back(make_box(a, a, r));
                }
    return out;
}

// Flux-correction face parts of a coarse level against its fine level (Sec.
// 3.4), in the order (fine patch, axis, side, coarse patch): the coarse cells
// just outside each fine face, split by the coarse patch holding them; faces
// whose outside cells the fine level covers entirely are left out (projection
// overwrites those cells).  wave[k]: parts in one wave share no coarse cell,
// and a part sharing cells with earlier parts comes in a later wave, so the
// additions happen in the listed order.
void plan_correction(const int32_t *fn, const int32_t *fo, int nf, const int32_t *cn, const int32_t *co, int nc,
                     std::vector<enzo_fc_face> &parts, std::vector<int> &wave)
{
    parts.clear();
    wave.clear();
    std::vector<Box3> foot(nf);
    for (int i = 0; i < nf; ++i)
        for (int d = 0; d < 3; ++d) {
            foot[i].lo[d] = floordiv(fo[3 * i + d], RF);
            foot[i].hi[d] = floordiv((int64_t)fo[3 * i + d] + fn[3 * i + d], RF);
        }
    const std::vector<Box3> coarse = active_boxes(cn, co, nc);
    BoxIndex fidx(foot), cidx(coarse);
    std::vector<Box3> cells;
    std::vector<int> cand;
    for (int i = 0; i < nf; ++i)
        for (int d = 0; d < 3; ++d) {
            const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
            for (int side = 0; side < 2; ++side) {
                const int64_t X = floordiv((int64_t)fo[3 * i + d] + (side ? fn[3 * i + d] : 0), RF);
                Box3 o = foot[i];
                o.lo[d] = side == 0 ? X - 1 : X;
                o.hi[d] = side == 0 ? X : X + 1;
                const int64_t vol = box_volume(o);
                int64_t covered = 0;
                fidx.candidates(o, cand);
                for (int j : cand) covered += box_volume(box_and(o, foot[j]));
                if (covered >= vol) continue;
                cidx.candidates(o, cand);
                for (int t : cand) {
                    const Box3 x = box_and(o, coarse[t]);
                    if (box_empty(x)) continue;
                    enzo_fc_face p;
                    p.fine = i;
                    p.dir = d;
                    p.side = side;
                    p.target = t;
                    p.lo[0] = (int32_t)(x.lo[a1] - foot[i].lo[a1]);
                    p.lo[1] = (int32_t)(x.lo[a2] - foot[i].lo[a2]);
                    p.hi[0] = (int32_t)(x.hi[a1] - foot[i].lo[a1]);
                    p.hi[1] = (int32_t)(x.hi[a2] - foot[i].lo[a2]);
                    parts.push_back(p);
                    cells.push_back(x);
                }
            }
        }
    // waves: a part follows every earlier part on the same coarse patch whose
    // cells it shares
    wave.assign(parts.size(), 0);
    std::unordered_map<int, std::vector<int>> by_target;
    for (size_t k = 0; k < parts.size(); ++k) {
        std::vector<int> &prev = by_target[parts[k].target];
        for (int q : prev)
            if (!box_empty(box_and(cells[k], cells[q]))) wave[k] = std::max(wave[k], wave[q] + 1);
        prev.push_back((int)k);
    }
}

// Registers in doubles per patch (Sec. 3.4): all faces (for a patch with
// children) and boundary faces (for a patch with a parent), nc per face.
void register_sizes(const int32_t *n, int64_t nc, int64_t &all_f, int64_t &bnd)
{
    const int64_t nx = n[0], ny = n[1], nz = n[2];
    all_f = ((nx + 1) * ny * nz + (ny + 1) * nx * nz + (nz + 1) * nx * ny) * nc;
    bnd = 2 * (ny * nz + nx * nz + nx * ny) * nc;
}

void *default_alloc(size_t bytes, void *)
{
    void *p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}

void default_free(void *p, void *) { cudaFree(p); }

enum Op { OP_FILL, OP_CFL, OP_SAVE, OP_SWEEPS, OP_CORRECT, OP_REBUILD, OP_COUNT };

}  // namespace

// ---- the hierarchy ------------------------------------------------------------

struct HLevel {
    int np = 0;
    std::vector<int32_t> n, origin, parent;
    std::vector<enzo_patch> table;
    int64_t field_len = 0, cells = 0;
    double dx = 0.0, t = 0.0, t_old = 0.0;
    int64_t step = 0;
    bool has_children = false;
    std::vector<void *> mem;            // every device block of this level
    enzo_patch *patches = nullptr;
    double *U[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double *ge = nullptr;
    unsigned long long *status = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    double *freg = nullptr;
    int64_t freg_len = 0, bnd_lo = 0, bnd_hi = 0;
    double *old[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    enzo_patch_link *links = nullptr;
    enzo_copy_box *sib = nullptr, *itp = nullptr;
    int nsib = 0, nitp = 0;
    std::vector<std::pair<enzo_fc_face *, int>> waves;   // against the next finer level
    std::vector<void *> wave_mem;
};

struct enzo_hierarchy {
    enzo_alloc_fn alloc = default_alloc;
    enzo_free_fn release = default_free;
    void *ctx = nullptr;
    cudaStream_t stream = nullptr;
    int nf = 5;
    double root_dx = 1.0;
    bool has_bc = false;
    int32_t bc[3] = {0, 0, 0};
    std::vector<std::unique_ptr<HLevel>> levels;
    int64_t cell_updates = 0;
    uint64_t generation = 0;            // bumped whenever a level's memory changes
    std::vector<std::pair<int32_t, double>> log;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events[OP_COUNT];
    // rebuild scratch: flags on the device and their pinned host copy
    uint8_t *flags_dev = nullptr, *flags_host = nullptr;
    int64_t *flag_off_dev = nullptr;
    size_t flags_cap = 0, off_cap = 0;
    std::vector<void *> scratch;
};

namespace {

struct Failure {
    int code;
};

void check(int r)
{
    if (r != ENZO_OK) throw Failure{r};
}

void check_cuda(cudaError_t e)
{
    if (e != cudaSuccess) throw Failure{ENZO_ERR_CUDA};
}

void *dev_alloc(enzo_hierarchy *h, std::vector<void *> &owner, size_t bytes)
{
    void *p = h->alloc(std::max<size_t>(bytes, 256), h->ctx);
    if (!p) throw Failure{ENZO_ERR_CUDA};
    owner.push_back(p);
    return p;
}

void free_all(enzo_hierarchy *h, std::vector<void *> &owner)
{
    for (void *p : owner) h->release(p, h->ctx);
    owner.clear();
}

template <class T>
T *upload(enzo_hierarchy *h, std::vector<void *> &owner, const std::vector<T> &v)
{
    T *d = static_cast<T *>(dev_alloc(h, owner, v.size() * sizeof(T)));
    if (!v.empty()) check_cuda(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    return d;
}

struct Mark {
    enzo_hierarchy *h;
    int op;
    cudaEvent_t e0 = nullptr;
    Mark(enzo_hierarchy *h_, int op_) : h(h_), op(op_)
    {
        if (!h->timing) return;
        cudaEventCreate(&e0);
        cudaEventRecord(e0, h->stream);
    }
    ~Mark()
    {
        if (!e0) return;
        cudaEvent_t e1 = nullptr;
        cudaEventCreate(&e1);
        cudaEventRecord(e1, h->stream);
        h->events[op].push_back({e0, e1});
    }
};

enzo_patch_batch batch_of(const enzo_hierarchy *h, const HLevel &L)
{
    enzo_patch_batch b;
    std::memset(&b, 0, sizeof(b));
    b.npatch = L.np;
    b.patches = L.patches;
    b.field_len = L.field_len;
    for (int f = 0; f < 5; ++f) b.U[f] = L.U[f];
    b.workspace = L.ws;
    b.ws_bytes = L.ws_bytes;
    b.status = L.status;
    b.stream = h->stream;
    b.freg = L.freg;
    b.ge = L.ge;
    return b;
}

// Device state of level l from its layout, fields zeroed.
std::unique_ptr<HLevel> build_level(enzo_hierarchy *h, int l, const int32_t *n, const int32_t *origin,
                                    const int32_t *parent, int np, bool has_children)
{
    auto L = std::make_unique<HLevel>();
    try {
        L->np = np;
        L->n.assign(n, n + 3 * (size_t)np);
        L->origin.assign(origin, origin + 3 * (size_t)np);
        L->parent.assign(parent, parent + (size_t)np);
        L->dx = h->root_dx / std::ldexp(1.0, l);
        L->has_children = has_children;
        const bool wrap = l == 0 && !h->has_bc;
        const bool has_parent = l > 0;
        L->table.resize(np);
        int64_t off = 0, all_sum = 0, bnd_sum = 0;
        std::vector<int64_t> all_f(np), bnd(np);
        for (int i = 0; i < np; ++i) {
            enzo_patch &P = L->table[i];
            std::memset(&P, 0, sizeof(P));
            for (int d = 0; d < 3; ++d) {
                if (n[3 * i + d] < 1) throw Failure{ENZO_ERR_ARG};
                P.n[d] = n[3 * i + d];
                P.dx[d] = L->dx;
            }
            P.ng = NG;
            P.off = off;
            P.level = l;
            P.flags = wrap ? ENZO_PATCH_PERIODIC : 0;
            P.freg_all = -1;
            P.freg_bnd = -1;
            off += (int64_t)(n[3 * i] + 2 * NG) * (n[3 * i + 1] + 2 * NG) * (n[3 * i + 2] + 2 * NG);
            L->cells += (int64_t)n[3 * i] * n[3 * i + 1] * n[3 * i + 2];
            register_sizes(n + 3 * i, h->nf, all_f[i], bnd[i]);
        }
        int64_t reg = 0;
        if (has_children) {
            for (int i = 0; i < np; ++i) {
                L->table[i].freg_all = reg + all_sum;
                all_sum += all_f[i];
            }
            reg += all_sum;
        }
        if (has_parent) {
            L->bnd_lo = reg;
            for (int i = 0; i < np; ++i) {
                L->table[i].freg_bnd = reg + bnd_sum;
                bnd_sum += bnd[i];
            }
            reg += bnd_sum;
            L->bnd_hi = reg;
        }
        L->field_len = std::max<int64_t>(off, 1);
        int bad = -1;
        check(enzo_validate_patches(L->table.data(), np, L->field_len, &bad));
        L->patches = upload(h, L->mem, L->table);
        const size_t fbytes = (size_t)L->field_len * sizeof(double);
        for (int f = 0; f < 5; ++f) {
            L->U[f] = static_cast<double *>(dev_alloc(h, L->mem, fbytes));
            check_cuda(cudaMemsetAsync(L->U[f], 0, fbytes, h->stream));
        }
        if (h->nf == 6) {
            L->ge = static_cast<double *>(dev_alloc(h, L->mem, fbytes));
            check_cuda(cudaMemsetAsync(L->ge, 0, fbytes, h->stream));
        }
        L->status = static_cast<unsigned long long *>(dev_alloc(h, L->mem, ENZO_STATUS_WORDS * 8));
        check_cuda(cudaMemsetAsync(L->status, 0, ENZO_STATUS_WORDS * 8, h->stream));
        L->ws_bytes = enzo_workspace_size(np);
        L->ws = dev_alloc(h, L->mem, L->ws_bytes);
        if (reg > 0) {
            L->freg_len = reg;
            L->freg = static_cast<double *>(dev_alloc(h, L->mem, (size_t)reg * sizeof(double)));
            check_cuda(cudaMemsetAsync(L->freg, 0, (size_t)reg * sizeof(double), h->stream));
        }
        std::vector<enzo_patch_link> links(np);
        for (int i = 0; i < np; ++i) {
            for (int d = 0; d < 3; ++d) links[i].origin[d] = origin[3 * i + d];
            links[i].parent = parent[i];
        }
        L->links = upload(h, L->mem, links);
        if (has_parent) {
            const std::vector<enzo_copy_box> sib = plan_siblings(n, origin, np);
            const std::vector<enzo_copy_box> itp = plan_interp(n, origin, np);
            L->sib = upload(h, L->mem, sib);
            L->nsib = (int)sib.size();
            L->itp = upload(h, L->mem, itp);
            L->nitp = (int)itp.size();
        }
        if (has_children)
            for (int f = 0; f < h->nf; ++f) L->old[f] = static_cast<double *>(dev_alloc(h, L->mem, fbytes));
        return L;
    } catch (...) {
        free_all(h, L->mem);
        throw;
    }
}

void free_level(enzo_hierarchy *h, HLevel &L)
{
    free_all(h, L.wave_mem);
    free_all(h, L.mem);
}

// Correction parts of level l against level l + 1, one device array per wave.
void plan_level_correction(enzo_hierarchy *h, int l)
{
    HLevel &C = *h->levels[l];
    const HLevel &F = *h->levels[l + 1];
    free_all(h, C.wave_mem);
    C.waves.clear();
    std::vector<enzo_fc_face> parts;
    std::vector<int> wave;
    plan_correction(F.n.data(), F.origin.data(), F.np, C.n.data(), C.origin.data(), C.np, parts, wave);
    const int nw = wave.empty() ? 0 : 1 + *std::max_element(wave.begin(), wave.end());
    for (int w = 0; w < nw; ++w) {
        std::vector<enzo_fc_face> sel;
        for (size_t k = 0; k < parts.size(); ++k)
            if (wave[k] == w) sel.push_back(parts[k]);
        C.waves.push_back({upload(h, C.wave_mem, sel), (int)sel.size()});
    }
}

void fill(enzo_hierarchy *h, int l, int precision)
{
    HLevel &L = *h->levels[l];
    if (l == 0) {
        if (h->has_bc) {
            const enzo_patch_batch b = batch_of(h, L);
            check(enzo_ghost_fill_boundary(&b, h->bc));
        }
        return;   // a periodic root wraps inside its sweeps
    }
    HLevel &P = *h->levels[l - 1];
    const double w = (L.t - P.t_old) / (P.t - P.t_old);
    const enzo_patch_batch b = batch_of(h, L), pb = batch_of(h, P);
    double *old[5] = {P.old[0], P.old[1], P.old[2], P.old[3], P.old[4]};
    check(enzo_ghost_fill_level(&b, L.links, &pb, P.links, old, h->nf == 6 ? P.old[5] : nullptr, w, L.itp, L.nitp,
                                L.sib, L.nsib, precision, RF));
}

void sweep_step(enzo_hierarchy *h, int l, double dt, const enzo_params *p)
{
    HLevel &L = *h->levels[l];
    const int order[2][3] = {{0, 1, 2}, {2, 1, 0}};
    const enzo_patch_batch b = batch_of(h, L);
    int done = 0;
    for (int q = 0; q < 3; ++q) {
        const int d = order[L.step % 2][q];
        const int cover = 7 & ~done & ~(1 << d);
        check(enzo_ppm_sweep(&b, d, dt, cover, p));
        done |= 1 << d;
    }
    L.step += 1;
    h->cell_updates += L.cells;
}

void correct_and_project(enzo_hierarchy *h, int l, double dt, const enzo_params *p)
{
    HLevel &C = *h->levels[l];
    HLevel &F = *h->levels[l + 1];
    const enzo_patch_batch cb = batch_of(h, C), fb = batch_of(h, F);
    for (const auto &w : C.waves)
        check(enzo_flux_correct(&cb, C.links, &fb, F.links, w.first, w.second, dt, RF,
                                p->precision == ENZO_FP32 ? 1 : 0));
    check(enzo_project(&cb, C.links, &fb, F.links, RF));
}

// Replace level m + 1 by grids covering the flagged cells of level m (its
// ghosts already filled).  Returns through `boxes` the new grids as (parent,
// lo, hi) in level-m cells.
void rebuild_one(enzo_hierarchy *h, int m, const enzo_rebuild_params *rb, int margin,
                 std::vector<std::array<int32_t, 7>> &boxes)
{
    HLevel &L = *h->levels[m];
    boxes.clear();
    // flags of every active cell, on the device, then in pinned host memory
    std::vector<int64_t> off(L.np + 1, 0);
    for (int i = 0; i < L.np; ++i) off[i + 1] = off[i] + (int64_t)L.n[3 * i] * L.n[3 * i + 1] * L.n[3 * i + 2];
    const size_t cells = (size_t)std::max<int64_t>(off[L.np], 1);
    if (cells > h->flags_cap || (size_t)L.np > h->off_cap) {
        // grow the scratch (the previous rebuild's copies have finished: it
        // synchronised before reading its flags)
        free_all(h, h->scratch);
        if (h->flags_host) cudaFreeHost(h->flags_host);
        h->flags_host = nullptr;
        h->flags_cap = h->off_cap = 0;
        const size_t fcap = std::max(cells, (size_t)1 << 16), ocap = std::max<size_t>((size_t)L.np, 1024);
        check_cuda(cudaMallocHost(reinterpret_cast<void **>(&h->flags_host), fcap));
        h->flags_dev = static_cast<uint8_t *>(dev_alloc(h, h->scratch, fcap));
        h->flag_off_dev = static_cast<int64_t *>(dev_alloc(h, h->scratch, ocap * sizeof(int64_t)));
        h->flags_cap = fcap;
        h->off_cap = ocap;
    }
    if (L.np > 0) {
        check_cuda(cudaMemcpyAsync(h->flag_off_dev, off.data(), (size_t)L.np * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, h->stream));
        check_cuda(cudaMemsetAsync(h->flags_dev, 0, cells, h->stream));
        const enzo_patch_batch b = batch_of(h, L);
        check(enzo_flag_cells(&b, &rb->flag, h->flags_dev, h->flag_off_dev));
        check_cuda(cudaMemcpyAsync(h->flags_host, h->flags_dev, cells, cudaMemcpyDeviceToHost, h->stream));
    }
    check_cuda(cudaStreamSynchronize(h->stream));
    // Berger-Rigoutsos per patch (Sec. 3.5)
    enzo_cluster_params cp = rb->cluster;
    cp.margin = margin;
    std::vector<enzo_box> found(256);
    for (int i = 0; i < L.np; ++i) {
        int32_t nb = 0;
        for (;;) {
            const int r = enzo_cluster_flags(h->flags_host + off[i], &L.n[3 * i], &cp, found.data(),
                                             (int32_t)found.size(), &nb);
            if (r == ENZO_ERR_RANGE && nb > (int32_t)found.size()) {
                found.resize(nb);
                continue;
            }
            check(r);
            break;
        }
        for (int k = 0; k < nb; ++k) {
            std::array<int32_t, 7> e;
            e[0] = i;
            for (int d = 0; d < 3; ++d) {
                e[1 + d] = L.origin[3 * i + d] + found[k].lo[d];
                e[4 + d] = L.origin[3 * i + d] + found[k].hi[d];
            }
            boxes.push_back(e);
        }
    }
    HLevel &O = *h->levels[m + 1];
    // the same grids: the level stays; the level above may be new, so its
    // correction parts are planned again
    bool same = (int)boxes.size() == O.np;
    for (int j = 0; same && j < O.np; ++j) {
        if (boxes[j][0] != O.parent[j]) same = false;
        for (int d = 0; same && d < 3; ++d)
            if (boxes[j][1 + d] != O.origin[3 * j + d] / RF || boxes[j][4 + d] != (O.origin[3 * j + d] + O.n[3 * j + d]) / RF)
                same = false;
    }
    if (same) {
        plan_level_correction(h, m);
        return;
    }
    const int np = (int)boxes.size();
    std::vector<int32_t> n(3 * (size_t)np), origin(3 * (size_t)np), parent(np);
    for (int j = 0; j < np; ++j) {
        parent[j] = boxes[j][0];
        for (int d = 0; d < 3; ++d) {
            n[3 * j + d] = RF * (boxes[j][4 + d] - boxes[j][1 + d]);
            origin[3 * j + d] = RF * boxes[j][1 + d];
        }
    }
    std::unique_ptr<HLevel> N = build_level(h, m + 1, n.data(), origin.data(), parent.data(), np, O.has_children);
    N->t = O.t;
    N->step = O.step;
    N->t_old = O.t_old;
    try {
        if (np > 0) {
            // every new patch, ghosts included, interpolated from its parent's
            // current state (FP64), then overwritten by the old grids where they overlap
            std::vector<enzo_copy_box> full(np);
            for (int j = 0; j < np; ++j) {
                Box3 b;
                for (int d = 0; d < 3; ++d) {
                    b.lo[d] = origin[3 * j + d] - NG;
                    b.hi[d] = (int64_t)origin[3 * j + d] + n[3 * j + d] + NG;
                }
                full[j] = make_box(j, j, b);
            }
            std::vector<void *> tmp;
            enzo_copy_box *fb = upload(h, tmp, full);
            const enzo_patch_batch nb = batch_of(h, *N), pb = batch_of(h, L);
            double *cur[5] = {L.U[0], L.U[1], L.U[2], L.U[3], L.U[4]};
            int r = enzo_ghost_fill_level(&nb, N->links, &pb, L.links, cur, h->nf == 6 ? L.ge : nullptr, 0.0, fb,
                                          np, nullptr, 0, ENZO_FP64, RF);
            std::vector<enzo_copy_box> cps;
            if (r == ENZO_OK && O.np > 0) {
                const std::vector<Box3> oact = active_boxes(O.n.data(), O.origin.data(), O.np);
                BoxIndex oidx(oact);
                std::vector<int> cand;
                for (int a = 0; a < np; ++a) {
                    Box3 g;
                    for (int d = 0; d < 3; ++d) {
                        g.lo[d] = origin[3 * a + d] - NG;
                        g.hi[d] = (int64_t)origin[3 * a + d] + n[3 * a + d] + NG;
                    }
                    oidx.candidates(g, cand);
                    for (int b : cand) {
                        const Box3 x = box_and(g, oact[b]);
                        if (!box_empty(x)) cps.push_back(make_box(a, b, x));
                    }
                }
                if (!cps.empty()) {
                    enzo_copy_box *cb = upload(h, tmp, cps);
                    const enzo_patch_batch ob = batch_of(h, O);
                    r = enzo_copy_level(&nb, N->links, &ob, O.links, cb, (int32_t)cps.size());
                }
            }
            // the uploads must land before their host vectors go, and the
            // copies read the old level: finish before freeing either
            const cudaError_t e = cudaStreamSynchronize(h->stream);
            free_all(h, tmp);
            check(r);
            check_cuda(e);
        }
    } catch (...) {
        free_level(h, *N);
        throw;
    }
    check_cuda(cudaStreamSynchronize(h->stream));
    free_level(h, O);
    h->levels[m + 1] = std::move(N);
    h->generation += 1;
    plan_level_correction(h, m);
}

void rebuild(enzo_hierarchy *h, int l, const enzo_rebuild_params *rb, std::vector<std::array<int32_t, 7>> *first)
{
    fill(h, l, ENZO_FP64);
    std::vector<std::array<int32_t, 7>> boxes;
    for (int m = l; m + 1 < (int)h->levels.size(); ++m) {
        rebuild_one(h, m, rb, m == 0 ? rb->root_margin : rb->nest, boxes);
        if (first && m == l) *first = boxes;
    }
}

void evolve_level(enzo_hierarchy *h, int l, double t_parent, const enzo_params *p, const enzo_params *cflp,
                  const enzo_rebuild_params *rb)
{
    HLevel *L = h->levels[l].get();
    if (L->cells == 0) {
        L->t = t_parent;   // a level without grids has nothing to advance
        return;
    }
    while (L->t < t_parent * (1.0 - 1e-14)) {
        {
            Mark m(h, OP_FILL);
            fill(h, l, p->precision);
        }
        double dt;
        if (l == 0) {
            dt = t_parent - L->t;
        } else {
            Mark m(h, OP_CFL);
            const enzo_patch_batch b = batch_of(h, *L);
            double rate_dt = 0.0;
            check(enzo_timestep_cfl(&b, cflp, &rate_dt, 0));
            dt = std::min(rate_dt, t_parent - L->t);
        }
        if (L->has_children) {
            Mark m(h, OP_SAVE);
            const size_t fbytes = (size_t)L->field_len * sizeof(double);
            for (int f = 0; f < h->nf; ++f)
                check_cuda(cudaMemcpyAsync(L->old[f], f < 5 ? L->U[f] : L->ge, fbytes, cudaMemcpyDeviceToDevice,
                                           h->stream));
            L->t_old = L->t;
        }
        {
            Mark m(h, OP_SWEEPS);
            sweep_step(h, l, dt, p);
        }
        L->t += dt;
        h->log.push_back({l, dt});
        if (L->has_children) {
            {
                Mark m(h, OP_FILL);
                fill(h, l, p->precision);
            }
            HLevel &C = *h->levels[l + 1];
            if (C.freg && C.bnd_hi > C.bnd_lo)
                check_cuda(cudaMemsetAsync(C.freg + C.bnd_lo, 0, (size_t)(C.bnd_hi - C.bnd_lo) * sizeof(double),
                                           h->stream));
            evolve_level(h, l + 1, L->t, p, cflp, rb);
            {
                Mark m(h, OP_CORRECT);
                correct_and_project(h, l, dt, p);
            }
            if (rb) {
                Mark m(h, OP_REBUILD);
                rebuild(h, l, rb, nullptr);
            }
        }
    }
    // the loop stops within 1e-14 of the parent's time; the level has reached it
    L->t = t_parent;
}

int guarded(void (*fn)(void *), void *arg)
{
    try {
        fn(arg);
        return ENZO_OK;
    } catch (const Failure &f) {
        return f.code;
    } catch (const std::bad_alloc &) {
        return ENZO_ERR_CUDA;
    }
}

}  // namespace

extern "C" int enzo_hierarchy_create(const enzo_level_layout *levels, int32_t nlevel, double root_dx,
                                     int32_t nfields, const int32_t *root_bc, void *stream,
                                     const enzo_allocator *allocator, enzo_hierarchy **out)
{
    if (!levels || nlevel < 1 || nlevel > 32 || !out || !(root_dx > 0.0) || !(root_dx < INFINITY) ||
        (nfields != 5 && nfields != 6))
        return ENZO_ERR_ARG;
    // the root is one grid: its ghosts come from its own boundaries (wrapped
    // or filled), never from siblings
    if (levels[0].npatch != 1) return ENZO_ERR_ARG;
    *out = nullptr;
    for (int l = 0; l < nlevel; ++l) {
        const enzo_level_layout &ly = levels[l];
        if (ly.npatch < 0 || (ly.npatch > 0 && (!ly.n || !ly.origin || !ly.parent))) return ENZO_ERR_ARG;
        for (int i = 0; i < ly.npatch; ++i) {
            if (l == 0 && ly.parent[i] != -1) return ENZO_ERR_ARG;
            if (l > 0 && (ly.parent[i] < 0 || ly.parent[i] >= levels[l - 1].npatch)) return ENZO_ERR_ARG;
            for (int d = 0; d < 3; ++d)
                if (ly.n[3 * i + d] < 1 || (l > 0 && ((ly.n[3 * i + d] | ly.origin[3 * i + d]) & 1))) return ENZO_ERR_ARG;
        }
    }
    if (root_bc)
        for (int d = 0; d < 3; ++d)
            if (root_bc[d] < ENZO_BC_PERIODIC || root_bc[d] > ENZO_BC_OUTFLOW) return ENZO_ERR_ARG;
    if (!root_bc && nlevel > 1) {
        // the periodic root wraps inside its sweeps and keeps no ghost cells, so
        // the level-1 ghost interpolation (SecondOrderA reaches one root cell
        // beyond the cell under a fine ghost) must find its parent cells inside it
        const enzo_level_layout &l1 = levels[1];
        for (int i = 0; i < l1.npatch; ++i)
            for (int d = 0; d < 3; ++d) {
                const int lo = l1.origin[3 * i + d] / RF, hi = (l1.origin[3 * i + d] + l1.n[3 * i + d] + 1) / RF;
                if (lo < 3 || hi > levels[0].n[d] - 3) return ENZO_ERR_RANGE;
            }
    }
    enzo_hierarchy *h = new (std::nothrow) enzo_hierarchy;
    if (!h) return ENZO_ERR_CUDA;
    if (allocator && allocator->alloc && allocator->release) {
        h->alloc = allocator->alloc;
        h->release = allocator->release;
        h->ctx = allocator->ctx;
    }
    h->stream = static_cast<cudaStream_t>(stream);
    h->nf = nfields;
    h->root_dx = root_dx;
    if (root_bc) {
        h->has_bc = true;
        for (int d = 0; d < 3; ++d) h->bc[d] = root_bc[d];
    }
    struct Arg {
        enzo_hierarchy *h;
        const enzo_level_layout *levels;
        int nlevel;
    } arg{h, levels, nlevel};
    const int r = guarded(
        [](void *p) {
            Arg &a = *static_cast<Arg *>(p);
            for (int l = 0; l < a.nlevel; ++l) {
                const enzo_level_layout &ly = a.levels[l];
                a.h->levels.push_back(build_level(a.h, l, ly.n, ly.origin, ly.parent, ly.npatch, l + 1 < a.nlevel));
            }
            for (int l = 0; l + 1 < a.nlevel; ++l) plan_level_correction(a.h, l);
            check_cuda(cudaStreamSynchronize(a.h->stream));
        },
        &arg);
    if (r != ENZO_OK) {
        enzo_hierarchy_destroy(h);
        return r;
    }
    *out = h;
    return ENZO_OK;
}

extern "C" int enzo_hierarchy_destroy(enzo_hierarchy *h)
{
    if (!h) return ENZO_ERR_ARG;
    cudaStreamSynchronize(h->stream);
    for (auto &L : h->levels) free_level(h, *L);
    free_all(h, h->scratch);
    if (h->flags_host) cudaFreeHost(h->flags_host);
    for (auto &v : h->events)
        for (auto &e : v) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    delete h;
    return ENZO_OK;
}

extern "C" int enzo_hierarchy_nlevel(const enzo_hierarchy *h) { return h ? (int)h->levels.size() : ENZO_ERR_ARG; }

extern "C" int enzo_hierarchy_level(const enzo_hierarchy *h, int32_t level, enzo_level_info *info)
{
    if (!h || !info || level < 0 || level >= (int)h->levels.size()) return ENZO_ERR_ARG;
    const HLevel &L = *h->levels[level];
    std::memset(info, 0, sizeof(*info));
    info->batch = batch_of(h, L);
    info->links = L.links;
    info->table = L.table.data();
    info->n = L.n.data();
    info->origin = L.origin.data();
    info->parent = L.parent.data();
    info->dx = L.dx;
    info->t = L.t;
    info->cells = L.cells;
    info->freg_len = L.freg_len;
    info->generation = h->generation;
    return ENZO_OK;
}

extern "C" int enzo_hierarchy_root_step(enzo_hierarchy *h, const enzo_params *p, const enzo_params *cfl,
                                        const enzo_rebuild_params *rb, double *dt0_out)
{
    if (!h || !p) return ENZO_ERR_ARG;
    struct Arg {
        enzo_hierarchy *h;
        const enzo_params *p, *cfl;
        const enzo_rebuild_params *rb;
        double dt0;
    } arg{h, p, cfl ? cfl : p, rb, 0.0};
    const int r = guarded(
        [](void *q) {
            Arg &a = *static_cast<Arg *>(q);
            HLevel &root = *a.h->levels[0];
            const enzo_patch_batch b = batch_of(a.h, root);
            check(enzo_timestep_cfl(&b, a.cfl, &a.dt0, 0));
            evolve_level(a.h, 0, root.t + a.dt0, a.p, a.cfl, a.rb);
        },
        &arg);
    if (dt0_out) *dt0_out = arg.dt0;
    return r;
}

extern "C" int enzo_hierarchy_step_to(enzo_hierarchy *h, double t_end, const enzo_params *p, const enzo_params *cfl,
                                      const enzo_rebuild_params *rb)
{
    if (!h || !p || !(t_end < INFINITY) || !(t_end > h->levels[0]->t)) return ENZO_ERR_ARG;
    struct Arg {
        enzo_hierarchy *h;
        double t_end;
        const enzo_params *p, *cfl;
        const enzo_rebuild_params *rb;
    } arg{h, t_end, p, cfl ? cfl : p, rb};
    return guarded(
        [](void *q) {
            Arg &a = *static_cast<Arg *>(q);
            evolve_level(a.h, 0, a.t_end, a.p, a.cfl, a.rb);
        },
        &arg);
}

extern "C" int enzo_hierarchy_rebuild(enzo_hierarchy *h, int32_t level, const enzo_rebuild_params *rb,
                                      int32_t *boxes, int32_t cap, int32_t *nbox)
{
    if (!h || !rb || level < 0 || level + 1 >= (int)h->levels.size() || cap < 0 || (cap > 0 && !boxes) || !nbox)
        return ENZO_ERR_ARG;
    std::vector<std::array<int32_t, 7>> first;
    struct Arg {
        enzo_hierarchy *h;
        int level;
        const enzo_rebuild_params *rb;
        std::vector<std::array<int32_t, 7>> *first;
    } arg{h, level, rb, &first};
    const int r = guarded(
        [](void *q) {
            Arg &a = *static_cast<Arg *>(q);
            rebuild(a.h, a.level, a.rb, a.first);
        },
        &arg);
    if (r != ENZO_OK) return r;
    *nbox = (int32_t)first.size();
    for (int k = 0; k < (int)first.size() && k < cap; ++k)
        for (int j = 0; j < 7; ++j) boxes[7 * k + j] = first[k][j];
    return (int)first.size() > cap ? ENZO_ERR_RANGE : ENZO_OK;
}

extern "C" int enzo_hierarchy_take_log(enzo_hierarchy *h, int32_t *levels, double *dts, int32_t cap, int32_t *n)
{
    if (!h || !n || cap < 0 || (cap > 0 && (!levels || !dts))) return ENZO_ERR_ARG;
    *n = (int32_t)h->log.size();
    if ((int)h->log.size() > cap) return ENZO_ERR_RANGE;
    for (size_t k = 0; k < h->log.size(); ++k) {
        levels[k] = h->log[k].first;
        dts[k] = h->log[k].second;
    }
    h->log.clear();
    return ENZO_OK;
}

extern "C" int enzo_hierarchy_timing(enzo_hierarchy *h, int32_t enable, double ms[ENZO_HOP_COUNT],
                                     int64_t *cell_updates)
{
    if (!h) return ENZO_ERR_ARG;
    if (ms) {
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return ENZO_ERR_CUDA;
        for (int op = 0; op < OP_COUNT; ++op) {
            double s = 0.0;
            for (auto &e : h->events[op]) {
                float t = 0.0f;
                if (cudaEventElapsedTime(&t, e.first, e.second) == cudaSuccess) s += t;
            }
            ms[op] = s;
        }
    }
    if (cell_updates) *cell_updates = h->cell_updates;
    if (enable >= 0) {
        for (auto &v : h->events) {
            for (auto &e : v) {
                cudaEventDestroy(e.first);
                cudaEventDestroy(e.second);
            }
            v.clear();
        }
        h->timing = enable != 0;
    }
    return ENZO_OK;
}

extern "C" int enzo_plan_level(const int32_t *n, const int32_t *origin, int32_t npatch, enzo_copy_box *sib,
                               int32_t sib_cap, int32_t *nsib, enzo_copy_box *itp, int32_t itp_cap, int32_t *nitp)
{
    if (npatch < 0 || (npatch > 0 && (!n || !origin)) || !nsib || !nitp || sib_cap < 0 || itp_cap < 0 ||
        (sib_cap > 0 && !sib) || (itp_cap > 0 && !itp))
        return ENZO_ERR_ARG;
    try {
        const std::vector<enzo_copy_box> s = plan_siblings(n, origin, npatch);
        const std::vector<enzo_copy_box> t = plan_interp(n, origin, npatch);
        *nsib = (int32_t)s.size();
        *nitp = (int32_t)t.size();
        if ((int)s.size() > sib_cap || (int)t.size() > itp_cap) return ENZO_ERR_RANGE;
        std::copy(s.begin(), s.end(), sib);
        std::copy(t.begin(), t.end(), itp);
    } catch (const std::bad_alloc &) {
        return ENZO_ERR_CUDA;
    }
    return ENZO_OK;
}

extern "C" int enzo_plan_correction(const int32_t *fine_n, const int32_t *fine_origin, int32_t nfine,
                                    const int32_t *coarse_n, const int32_t *coarse_origin, int32_t ncoarse,
                                    enzo_fc_face *parts, int32_t *wave, int32_t cap, int32_t *nparts)
{
    if (nfine < 0 || ncoarse < 0 || (nfine > 0 && (!fine_n || !fine_origin)) ||
        (ncoarse > 0 && (!coarse_n || !coarse_origin)) || !nparts || cap < 0 || (cap > 0 && (!parts || !wave)))
        return ENZO_ERR_ARG;
    try {
        std::vector<enzo_fc_face> p;
        std::vector<int> w;
        plan_correction(fine_n, fine_origin, nfine, coarse_n, coarse_origin, ncoarse, p, w);
        *nparts = (int32_t)p.size();
        if ((int)p.size() > cap) return ENZO_ERR_RANGE;
        for (size_t k = 0; k < p.size(); ++k) {
            parts[k] = p[k];
            wave[k] = w[k];
        }
    } catch (const std::bad_alloc &) {
        return ENZO_ERR_CUDA;
    }
    return ENZO_OK;
}
