// sg_api.cu -- the extern "C" entry points of libsg (declared in sg.h):
// argument checks, state order, ownership of the device arrays and launch of
// the kernels in sg_tag.cu, sg_sweep.cu and sg_probe.cu on the grid's stream.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sg_internal.cuh"

namespace sg {

namespace {

std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_wide_offsets{false};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

ff split(double v) { return split_ff(v); }

}  // namespace

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool force_wide_offsets() { return g_wide_offsets.load(std::memory_order_relaxed); }

void* grid_alloc(sg_grid* g, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (g->user_alloc) {
        p = g->alloc.alloc(bytes, (void*)g->stream, g->alloc.ctx);
    } else if (cudaMallocAsync(&p, bytes, g->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void grid_free(sg_grid* g, Buf& b) {
    if (b.p) {
        if (g->user_alloc)
            g->alloc.free(b.p, b.bytes, (void*)g->stream, g->alloc.ctx);
        else
            cudaFreeAsync(b.p, g->stream);
    }
    b.p = nullptr;
    b.bytes = 0;
}

bool ensure(sg_grid* g, Buf& b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return true;
    grid_free(g, b);
    b.p = grid_alloc(g, bytes);
    if (!b.p) return false;
    b.bytes = bytes;
    return true;
}

sg_status fail(sg_grid* g, sg_status st, const std::string& msg) {
    if (g) g->last_error = msg;
    return st;
}

sg_status cuda_fail(sg_grid* g, cudaError_t e, const char* where) {
    return fail(g, SG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

GridF grid_f(const sg_grid* g) {
    GridF G;
    for (int a = 0; a < 3; ++a) {
        G.lo[a] = (float)g->desc.lo[a];
        G.dims[a] = g->desc.dims[a];
    }
    G.h = (float)g->desc.h;
    G.h_d = g->desc.h;
    G.F = (float)g->F;
    G.inv_h = (float)(1.0 / g->desc.h);
    set_lattice(G.lat_c, G.lat_ih, g->desc.lo, g->desc.h);
    return G;
}

GridFF grid_ff(const sg_grid* g) {
    GridFF G;
    for (int a = 0; a < 3; ++a) {
        G.lo[a] = split(g->desc.lo[a]);
        G.dims[a] = g->desc.dims[a];
    }
    G.h = split(g->desc.h);
    G.T = split(4.0 * g->desc.h * (1.0 - std::ldexp(1.0, -10)));
    return G;
}

ShapeFF shape_ff(const sg_shape* s) {
    ShapeFF S;
    S.kind = s->kind;
    bool plain = true;
    for (int i = 0; i < 3; ++i) {
        S.centre[i] = split(s->centre[i]);
        S.cf[i] = (float)s->centre[i];
        plain &= s->centre[i] == 0.0;
    }
    for (int i = 0; i < 9; ++i) {
        S.rot[i] = split(s->rot[i]);
        S.rf[i] = (float)s->rot[i];
        plain &= s->rot[i] == ((i % 4 == 0) ? 1.0 : 0.0);
    }
    for (int i = 0; i < 8; ++i) {
        S.p[i] = split(s->p[i]);
        S.pf[i] = (float)s->p[i];
    }
    S.plain = plain ? 1 : 0;
    // prism edges (a -> b: vertex 0 -> 1, 1 -> 2, 2 -> 0) and orientation
    const double* t = s->p;
    for (int k = 0; k < 3; ++k) {
        const int a = 2 * k, b = (2 * k + 2) % 6;
        const double ex = t[b] - t[a], ey = t[b + 1] - t[a + 1], l2 = ex * ex + ey * ey;
        S.seg[3 * k] = split(ex);
        S.seg[3 * k + 1] = split(ey);
        S.seg[3 * k + 2] = split(l2 > 0.0 ? 1.0 / l2 : 0.0);
    }
    S.orient = (t[2] - t[0]) * (t[5] - t[1]) - (t[3] - t[1]) * (t[4] - t[0]) > 0.0 ? 1 : -1;
    S.zc = split(0.5 * (t[6] + t[7]));
    S.hz = split(0.5 * (t[7] - t[6]));
    return S;
}

bool field_fresh(const sg_grid* g, int f) {
    const Buf& b = g->field[f];
    return !b.p || b.bytes < (size_t)g->P * PKG3 * sizeof(float) || g->stale[f];
}

// A field of the current tagging; a buffer that is new, or kept from an
// earlier tagging, is zero-filled when the caller reads before writing.
float* field_ptr(sg_grid* g, int f, bool zero_new) {
    const size_t bytes = (size_t)g->P * PKG3 * sizeof(float);
    const bool fresh = field_fresh(g, f);
    Buf& b = g->field[f];
    if (!ensure(g, b, bytes)) return nullptr;
    if (fresh && zero_new && cudaMemsetAsync(b.p, 0, bytes, g->stream) != cudaSuccess) return nullptr;
    g->stale[f] = false;
    return (float*)b.p;
}

}  // namespace sg

using namespace sg;

#define SG_CHECK_GRID(g)                                                  \
    do {                                                                  \
        if (!(g)) return SG_ERR_INVALID;                                  \
    } while (0)
#define SG_CUDA(g, call, where)                                           \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return cuda_fail((g), e_, (where));        \
    } while (0)

static bool valid_shape(const sg_shape* s) {
    return s && s->kind >= SG_SHAPE_SPHERE && s->kind <= SG_SHAPE_SHELL;
}

extern "C" {

const char* sg_version(void) { return "libsg 0.1 (sm_103a)"; }

int64_t sg_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

namespace {

// The 256-byte pinned read-back word of a grid comes from one process-wide
// pinned block of PIN_SLOTS slots (portable to every device), taken on first
// use and kept until exit, so that creating a grid page-locks nothing (a
// stack of multi-resolution layers creates one grid per layer); past
// PIN_SLOTS live grids each takes its own.
constexpr int PIN_SLOTS = 256;
std::mutex g_pin_mu;
unsigned char* g_pin_block = nullptr;
bool g_pin_tried = false;
std::vector<int> g_pin_free;

void* pin_get(bool* pooled) {
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pin_tried) {
            g_pin_tried = true;
            if (cudaHostAlloc((void**)&g_pin_block, (size_t)PIN_SLOTS * 256, cudaHostAllocPortable) == cudaSuccess) {
                for (int i = PIN_SLOTS - 1; i >= 0; --i) g_pin_free.push_back(i);
            } else {
                cudaGetLastError();
                g_pin_block = nullptr;
            }
        }
        if (!g_pin_free.empty()) {
            const int i = g_pin_free.back();
            g_pin_free.pop_back();
            *pooled = true;
            return g_pin_block + (size_t)i * 256;
        }
    }
    *pooled = false;
    void* p = nullptr;
    if (cudaHostAlloc(&p, 256, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pin_put(void* p, bool pooled) {
    if (!p) return;
    if (!pooled) {
        cudaFreeHost(p);
        return;
    }
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back((int)(((unsigned char*)p - g_pin_block) / 256));
}

}  // namespace

sg_status sg_create(const sg_grid_desc* desc, const sg_allocator* alloc, void* stream, sg_grid** out) {
    if (!desc || !out) return SG_ERR_INVALID;
    *out = nullptr;
    if (!(desc->h > 0.0) || !std::isfinite(desc->h)) return SG_ERR_INVALID;
    int64_t nc = 1;
    for (int a = 0; a < 3; ++a) {
        if (desc->dims[a] < 1) return SG_ERR_INVALID;
        if (4LL * desc->dims[a] + 1 >= (1LL << 21)) return SG_ERR_CAPACITY;
        nc *= desc->dims[a];
    }
    if (nc >= (1LL << 31)) return SG_ERR_CAPACITY;
    if (alloc && (!alloc->alloc || !alloc->free)) return SG_ERR_INVALID;
    if (desc->id_order != 0 && desc->id_order != 1) return SG_ERR_INVALID;
    if (!std::isfinite(desc->kernel_support) || desc->kernel_support < 0.0 ||
        desc->kernel_support > 3.0 * desc->h * (1.0 + 1e-12))
        return SG_ERR_INVALID;
    if (!std::isfinite(desc->heaviside_eps) || desc->heaviside_eps < 0.0) return SG_ERR_INVALID;
    sg_grid* g = new (std::nothrow) sg_grid();
    if (!g) return SG_ERR_OOM;
    g->desc = *desc;
    g->F = desc->far_value > 0.0 ? desc->far_value : 16.0 * desc->h;
    g->nc = nc;
    g->stream = (cudaStream_t)stream;
    if (alloc) {
        g->alloc = *alloc;
        g->user_alloc = true;
    }
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return SG_ERR_CUDA;
    }
    if (!ensure(g, g->err, 256)) {
        delete g;
        return SG_ERR_OOM;
    }
    if (cudaMemsetAsync(g->err.p, 0, 256, g->stream) != cudaSuccess ||
        !(g->host_pin.p = pin_get(&g->host_pin_pooled))) {
        cudaGetLastError();
        grid_free(g, g->err);
        delete g;
        return SG_ERR_CUDA;
    }
    g->host_pin.bytes = 256;
    *out = g;
    return SG_OK;
}

sg_status sg_destroy(sg_grid* g) {
    SG_CHECK_GRID(g);
    DeviceGuard dg(g->device);
    Buf* bufs[] = {&g->cell_pkg, &g->cell_type, &g->pkg_cell, &g->pkg_type, &g->nbr, &g->faces,
                   &g->phi_tmp,  &g->err,       &g->scratch,  &g->stats,    &g->sur_work};
    for (Buf* b : bufs) grid_free(g, *b);
    for (int f = 0; f < SG_N_FLOAT_FIELDS; ++f) grid_free(g, g->field[f]);
    // every read-back into the pinned word is waited for when it is issued;
    // the wait here only makes the slot's reuse independent of that
    if (g->host_pin.p && cudaStreamSynchronize(g->stream) != cudaSuccess) cudaGetLastError();
    pin_put(g->host_pin.p, g->host_pin_pooled);
    delete g;
    return SG_OK;
}

sg_status sg_set_stream(sg_grid* g, void* stream) {
    SG_CHECK_GRID(g);
    g->stream = (cudaStream_t)stream;
    return SG_OK;
}

int64_t sg_n_packages(const sg_grid* g) { return g ? g->P : 0; }

const char* sg_last_error(const sg_grid* g) { return g ? g->last_error.c_str() : "null grid"; }

}  // extern "C"

// Scratch of the tagging: three 32-cell bit-mask arrays (core, active, and
// the per-word populations scanned in place), the package count and the
// multi-resolution evaluation counter, and the scan's own scratch.
static size_t tag_mask_bytes(int64_t nc) { return ((size_t)((nc + 31) >> 5) * 4 + 255) & ~(size_t)255; }
static size_t tag_count_offset(int64_t nc) { return 3 * tag_mask_bytes(nc); }

// Tagging steps 1-5; `flags` launches step 1 (core cells and far sides) into
// (cell_type, core mask) on the grid's stream.
template <class Flags>
static sg_status tag_common(sg_grid* g, Flags flags, int64_t* n_packages) {
    const int64_t nc = g->nc, nw = (nc + 31) >> 5;
    const GridFF G = grid_ff(g);
    const size_t mb = tag_mask_bytes(nc), cnt = tag_count_offset(nc);
    if (!ensure(g, g->cell_type, (size_t)nc) || !ensure(g, g->cell_pkg, (size_t)nc * 4) ||
        !ensure(g, g->scratch, cnt + 256 + scan_scratch_bytes(nw)))
        return fail(g, SG_ERR_OOM, "sg_tag_allocate: out of device memory");
    uint32_t* core = (uint32_t*)g->scratch.p;
    uint32_t* act = (uint32_t*)((char*)g->scratch.p + mb);
    uint32_t* count = (uint32_t*)((char*)g->scratch.p + 2 * mb);
    uint32_t* total = (uint32_t*)((char*)g->scratch.p + cnt);
    void* scan_scratch = (char*)g->scratch.p + cnt + 256;
    uint8_t* ct = (uint8_t*)g->cell_type.p;
    SG_CUDA(g, flags(ct, core), "tag flags");
    SG_CUDA(g, launch_tag_inner(G, ct, core, act, count, nc, g->stream), "tag inner");
    SG_CUDA(g, exclusive_scan_u32(count, count, nw, total, scan_scratch, g->stream), "tag scan");
    // the package count and, 128 bytes on, the multi-resolution evaluation
    // counter (when the flags kernel kept one): one read-back for both
    SG_CUDA(g, cudaMemcpyAsync(g->host_pin.p, total, 136, cudaMemcpyDeviceToHost, g->stream), "tag count");
    SG_CUDA(g, cudaStreamSynchronize(g->stream), "tag sync");
    const int64_t P = 2 + (int64_t)*(uint32_t*)g->host_pin.p;
    if (P >= (1LL << 31) / NB) return fail(g, SG_ERR_CAPACITY, "sg_tag_allocate: too many packages");
    // every field is sized by P and its values belong to the old tagging: the
    // buffers are kept (they grow when P does) and treated as new, so that a
    // re-tagged grid allocates nothing once its buffers are large enough
    for (int f = 0; f < SG_N_FLOAT_FIELDS; ++f) g->stale[f] = true;
    if (!ensure(g, g->pkg_cell, (size_t)P * 4) || !ensure(g, g->pkg_type, (size_t)P) ||
        !ensure(g, g->nbr, (size_t)P * NB * 4) || !ensure(g, g->faces, (size_t)P * 8 * 4)) {
        g->state = 0;
        return fail(g, SG_ERR_OOM, "sg_tag_allocate: out of device memory");
    }
    g->P = P;
    SG_CUDA(g, launch_tag_scatter(ct, act, count, (int32_t*)g->cell_pkg.p, (int32_t*)g->pkg_cell.p,
                                  (uint8_t*)g->pkg_type.p, nc, g->stream),
            "tag scatter");
    if (g->desc.id_order == 1 && P > 3) {
        // Morton package ids: sort the active cells by the Morton key of their
        // centres (fine index 4I + 2, so the order of the cells' own keys)
        const int64_t n = P - 2;
        const GridF Gf = grid_f(g);
        const size_t fb = ((size_t)n * 4 + 255) & ~(size_t)255, tb = ((size_t)P * 4 + 255) & ~(size_t)255;
        const size_t sb = sort_scratch_bytes(n, morton_bits(Gf));
        if (!ensure(g, g->scratch, 4 * fb + 2 * tb + sb)) {
            g->state = 0;
            return fail(g, SG_ERR_OOM, "sg_tag_allocate: out of device memory");
        }
        char* sp = (char*)g->scratch.p;
        float* cx = (float*)sp;
        float* cy = (float*)(sp + fb);
        float* cz = (float*)(sp + 2 * fb);
        int32_t* ord = (int32_t*)(sp + 3 * fb);
        int32_t* old_cell = (int32_t*)(sp + 4 * fb);
        uint8_t* old_type = (uint8_t*)(sp + 4 * fb + tb);
        void* sort_scratch = sp + 4 * fb + 2 * tb;
        SG_CUDA(g, cudaMemcpyAsync(old_cell, g->pkg_cell.p, (size_t)P * 4, cudaMemcpyDeviceToDevice, g->stream),
                "ids copy");
        SG_CUDA(g, cudaMemcpyAsync(old_type, g->pkg_type.p, (size_t)P, cudaMemcpyDeviceToDevice, g->stream),
                "ids copy");
        SG_CUDA(g, launch_cell_centres(Gf, old_cell, cx, cy, cz, n, g->stream), "ids centres");
        SG_CUDA(g, morton_sort(Gf, n, cx, cy, cz, nullptr, ord, sort_scratch, g->stream), "ids sort");
        SG_CUDA(g, launch_renumber(ord, old_cell, old_type, (int32_t*)g->pkg_cell.p, (uint8_t*)g->pkg_type.p,
                                   (int32_t*)g->cell_pkg.p, n, g->stream),
                "ids renumber");
    }
    SG_CUDA(g, launch_fill_nbr(G, (const int32_t*)g->cell_pkg.p, (const int32_t*)g->pkg_cell.p, (int32_t*)g->nbr.p, P,
                               g->stream),
            "fill nbr");
    SG_CUDA(g, launch_fill_faces((const int32_t*)g->nbr.p, (int32_t*)g->faces.p, P, g->stream), "fill faces");
    g->state = 1;
    if (n_packages) *n_packages = P;
    return SG_OK;
}

extern "C" {

sg_status sg_tag_allocate(sg_grid* g, const sg_shape* shape, int64_t* n_packages) {
    SG_TRACE("sg_tag_allocate");
    SG_CHECK_GRID(g);
    if (!valid_shape(shape)) return fail(g, SG_ERR_INVALID, "sg_tag_allocate: bad shape");
    DeviceGuard dg(g->device);
    const GridFF G = grid_ff(g);
    const ShapeFF S = shape_ff(shape);
    return tag_common(
        g, [&](uint8_t* ct, uint32_t* core) { return launch_tag_flags(G, S, ct, core, g->nc, g->stream); },
        n_packages);
}

sg_status sg_tag_allocate_from(sg_grid* g, const sg_grid* coarse, const sg_shape* shape, int64_t* n_packages,
                               int64_t* evaluated) {
    SG_TRACE("sg_tag_allocate_from");
    SG_CHECK_GRID(g);
    if (!coarse || coarse == g) return fail(g, SG_ERR_INVALID, "sg_tag_allocate_from: no coarse layer");
    if (!valid_shape(shape)) return fail(g, SG_ERR_INVALID, "sg_tag_allocate_from: bad shape");
    if (coarse->state < 2 || !coarse->field[SG_FIELD_PHI].p)
        return fail(g, SG_ERR_STATE, "sg_tag_allocate_from: coarse layer not initialised");
    if (coarse->device != g->device) return fail(g, SG_ERR_INVALID, "sg_tag_allocate_from: layers on two devices");
    bool match = coarse->desc.h == 2.0 * g->desc.h;
    for (int a = 0; a < 3; ++a)
        match &= coarse->desc.lo[a] == g->desc.lo[a] && 2LL * coarse->desc.dims[a] == (int64_t)g->desc.dims[a];
    if (!match) return fail(g, SG_ERR_INVALID, "sg_tag_allocate_from: coarse layer is not this grid halved");
    DeviceGuard dg(g->device);
    const GridFF G = grid_ff(g);
    const ShapeFF S = shape_ff(shape);
    // the evaluation counter sits in the tagging scratch, beside the package count
    unsigned long long* ev = nullptr;
    const sg_status st = tag_common(
        g,
        [&](uint8_t* ct, uint32_t* core) {
            ev = (unsigned long long*)((char*)g->scratch.p + tag_count_offset(g->nc) + 128);
            cudaError_t e = cudaMemsetAsync(ev, 0, sizeof(unsigned long long), g->stream);
            if (e != cudaSuccess) return e;
            return launch_tag_flags_from(G, S, (const int32_t*)coarse->cell_pkg.p, (const uint8_t*)coarse->pkg_type.p,
                                         (const float*)coarse->field[SG_FIELD_PHI].p, coarse->desc.dims[0],
                                         coarse->desc.dims[1], ct, core, g->nc, ev, g->stream);
        },
        n_packages);
    if (st != SG_OK) return st;
    // read back with the package count (tag_common)
    if (evaluated) *evaluated = (int64_t)*(unsigned long long*)((char*)g->host_pin.p + 128);
    return SG_OK;
}

int32_t sg_multires_layers(const sg_grid_desc* finest, int32_t min_dims) {
    if (!finest || min_dims < 1) return 0;
    int32_t L = 1;
    int64_t d[3] = {finest->dims[0], finest->dims[1], finest->dims[2]};
    for (;;) {
        bool ok = true;
        for (int a = 0; a < 3; ++a) ok &= d[a] % 2 == 0 && d[a] / 2 >= min_dims;
        if (!ok) break;
        for (int a = 0; a < 3; ++a) d[a] /= 2;
        ++L;
    }
    return L;
}

sg_status sg_init_sdf(sg_grid* g, const sg_shape* shape) {
    SG_TRACE("sg_init_sdf");
    SG_CHECK_GRID(g);
    if (!valid_shape(shape)) return fail(g, SG_ERR_INVALID, "sg_init_sdf: bad shape");
    if (g->state < 1) return fail(g, SG_ERR_STATE, "sg_init_sdf: grid not tagged");
    DeviceGuard dg(g->device);
    float* phi = field_ptr(g, SG_FIELD_PHI, false);
    const GridFF G = grid_ff(g);
    if (!phi || !ensure(g, g->scratch, init_table_bytes(G))) return fail(g, SG_ERR_OOM, "sg_init_sdf: out of device memory");
    SG_CUDA(g, launch_init_sdf(G, shape_ff(shape), (const int32_t*)g->pkg_cell.p, phi, (float)g->F, g->P, g->scratch.p,
                               g->stream),
            "init sdf");
    g->state = 2;
    return SG_OK;
}

sg_status sg_gradient(sg_grid* g) {
    SG_TRACE("sg_gradient");
    SG_CHECK_GRID(g);
    if (g->state < 2) return fail(g, SG_ERR_STATE, "sg_gradient: phi not initialised");
    DeviceGuard dg(g->device);
    float* o[3];
    for (int a = 0; a < 3; ++a)
        if (!(o[a] = field_ptr(g, SG_FIELD_GX + a, false))) return fail(g, SG_ERR_OOM, "sg_gradient: out of memory");
    // the gradient kernel writes the far packages itself; with none active it is not launched
    if (g->P <= 2)
        for (int a = 0; a < 3; ++a) SG_CUDA(g, launch_set_far(o[a], 0.0f, 0.0f, g->stream), "gradient far");
    SG_CUDA(g, launch_gradient(grid_f(g), (const int32_t*)g->faces.p, (const float*)g->field[SG_FIELD_PHI].p, o[0], o[1],
                               o[2], g->P, g->stream),
            "gradient");
    return SG_OK;
}

static sg_status consistency(sg_grid* g, float trust, int64_t* out, unsigned debug) {
    SG_CHECK_GRID(g);
    if (!(trust > 0.0f) || !std::isfinite(trust)) return fail(g, SG_ERR_INVALID, "sg_consistency_correct: bad trust");
    if (g->state < 2) return fail(g, SG_ERR_STATE, "sg_consistency_correct: phi not initialised");
    DeviceGuard dg(g->device);
    if (!ensure(g, g->scratch, consistency_scratch_bytes(g->P, g->desc.dims)))
        return fail(g, SG_ERR_OOM, "sg_consistency_correct: out of memory");
    int64_t o[4] = {0, 0, 0, 0};
    const cudaError_t e =
        run_consistency(grid_ff(g), g->P, g->nc, (int32_t*)g->cell_pkg.p, (const int32_t*)g->pkg_cell.p,
                        (const uint8_t*)g->pkg_type.p, (int32_t*)g->nbr.p, (int32_t*)g->faces.p,
                        (float*)g->field[SG_FIELD_PHI].p, (float)((double)trust * g->desc.h), g->scratch.p,
                        g->host_pin.p, o, g->stream, debug);
    if (e == cudaErrorLaunchTimeout) return fail(g, SG_ERR_TIMEOUT, "sg_consistency_correct: flood did not settle or a barrier wait gave up");
    if (e != cudaSuccess) return cuda_fail(g, e, "consistency correction");
    if (out)
        for (int i = 0; i < 4; ++i) out[i] = o[i];
    return SG_OK;
}

sg_status sg_consistency_correct(sg_grid* g, float trust, int64_t* out) {
    SG_TRACE("sg_consistency_correct");
    return consistency(g, trust, out, 0);
}

sg_status sg_debug_consistency(sg_grid* g, float trust, int32_t flags, int64_t* out) {
    SG_CHECK_GRID(g);
    const unsigned all = SG_DEBUG_CC_ABSENT_POINTS | SG_DEBUG_CC_ABSENT_CELLS | SG_DEBUG_CC_PER_SWEEP;
    if (flags < 0 || ((unsigned)flags & ~all))
        return fail(g, SG_ERR_INVALID, "sg_debug_consistency: unknown flags");
    const unsigned absent = (unsigned)flags & (SG_DEBUG_CC_ABSENT_POINTS | SG_DEBUG_CC_ABSENT_CELLS);
    if (absent && ((unsigned)flags & SG_DEBUG_CC_PER_SWEEP))
        return fail(g, SG_ERR_INVALID, "sg_debug_consistency: an absent CTA needs the persistent floods");
    if (absent && !consistency_persistent(g->device))
        return fail(g, SG_ERR_DEVICE, "sg_debug_consistency: no cooperative launch on this device");
    return consistency(g, trust, out, (unsigned)flags);
}

void sg_debug_wide_offsets(int32_t on) { g_wide_offsets.store(on != 0, std::memory_order_relaxed); }

sg_status sg_debug_consistency_absent_cta(sg_grid* g, float trust) {
    return sg_debug_consistency(g, trust, SG_DEBUG_CC_ABSENT_POINTS | SG_DEBUG_CC_ABSENT_CELLS, nullptr);
}

sg_status sg_sequential_update(sg_grid* g, float delta) {
    SG_TRACE("sg_sequential_update");
    SG_CHECK_GRID(g);
    if (!std::isfinite(delta)) return fail(g, SG_ERR_INVALID, "sg_sequential_update: delta not finite");
    if (g->state < 2) return fail(g, SG_ERR_STATE, "sg_sequential_update: phi not initialised");
    DeviceGuard dg(g->device);
    SG_CUDA(g, launch_sequential(g->field[SG_FIELD_PHI].p ? (float*)g->field[SG_FIELD_PHI].p : nullptr, delta, g->P,
                                 g->stream),
            "sequential update");
    return SG_OK;
}

sg_status sg_laplacian(sg_grid* g) {
    SG_TRACE("sg_laplacian");
    SG_CHECK_GRID(g);
    if (g->state < 2) return fail(g, SG_ERR_STATE, "sg_laplacian: phi not initialised");
    DeviceGuard dg(g->device);
    float* lap = field_ptr(g, SG_FIELD_LAP, false);
    if (!lap) return fail(g, SG_ERR_OOM, "sg_laplacian: out of memory");
    if (g->P <= 2) SG_CUDA(g, launch_set_far(lap, 0.0f, 0.0f, g->stream), "laplacian far");  // else the kernel writes them
    SG_CUDA(g, launch_laplacian(grid_f(g), (const int32_t*)g->faces.p, (const float*)g->field[SG_FIELD_PHI].p, lap, g->P,
                                g->stream),
            "laplacian");
    return SG_OK;
}

sg_status sg_reinit(sg_grid* g, int32_t iterations, float cfl) {
    SG_TRACE("sg_reinit");
    SG_CHECK_GRID(g);
    if (iterations < 0 || !(cfl > 0.0f) || !std::isfinite(cfl)) return fail(g, SG_ERR_INVALID, "sg_reinit: bad args");
    if (g->state < 2) return fail(g, SG_ERR_STATE, "sg_reinit: phi not initialised");
    DeviceGuard dg(g->device);
    float* phi = (float*)g->field[SG_FIELD_PHI].p;
    float* s0 = field_ptr(g, SG_FIELD_S0, false);
    if (!s0 || !ensure(g, g->phi_tmp, (size_t)g->P * PKG3 * 4)) return fail(g, SG_ERR_OOM, "sg_reinit: out of memory");
    float* tmp = (float*)g->phi_tmp.p;
    const GridF G = grid_f(g);
    const float dt = (float)((double)cfl * g->desc.h);
    const int32_t* faces = (const int32_t*)g->faces.p;
    // the first sweep forms S0 from phi at call entry and writes the far
    // packages of S0 and of the second buffer; with no sweep (or no active
    // package) passes of their own do
    if (iterations == 0 || g->P <= 2) {
        SG_CUDA(g, launch_set_far(s0, -1.0f, 1.0f, g->stream), "reinit far");
        SG_CUDA(g, launch_set_far(tmp, -(float)g->F, (float)g->F, g->stream), "reinit far");
        SG_CUDA(g, launch_reinit_s0(G, phi, s0, g->P, g->stream), "reinit s0");
    }
    float* a = phi;
    float* b = tmp;
    // sweeps alternate their direction, the first against the pass before the
    // call, so that each starts on the packages whose phi and S0 the previous
    // pass left in L2 (the results do not depend on the order: a sweep reads
    // only the previous iterate)
    for (int32_t it = 0; it < iterations; ++it) {
        SG_CUDA(g, launch_reinit_step(G, faces, s0, a, b, dt, g->P, (it & 1) == 0, it == 0, g->stream),
                "reinit step");
        float* t = a;
        a = b;
        b = t;
    }
    if (a != phi) SG_CUDA(g, launch_copy_active(a, phi, g->P, g->stream), "reinit copy");
    return SG_OK;
}

sg_status sg_kernel_integrals(sg_grid* g, int32_t mode, const void* mlp) {
    SG_TRACE("sg_kernel_integrals");
    SG_CHECK_GRID(g);
    if (!((mode == 0 && mlp == nullptr) || (mode == 1 && mlp != nullptr)))
        return fail(g, SG_ERR_INVALID, "sg_kernel_integrals: mode 0 takes no network, mode 1 needs one");
    if (g->state < 2) return fail(g, SG_ERR_STATE, "sg_kernel_integrals: phi not initialised");
    if (mode == 1 && !default_kernel(g->desc))
        return fail(g, SG_ERR_INVALID, "sg_kernel_integrals: the surrogate needs kernel support 2h and eps = h");
    if (mode == 1 && g->P >= SUR_MAX_PACKAGES)
        return fail(g, SG_ERR_CAPACITY, "sg_kernel_integrals: the surrogate takes fewer than 2^24 packages");
    DeviceGuard dg(g->device);
    float* o[4];
    for (int a = 0; a < 4; ++a)
        if (!(o[a] = field_ptr(g, SG_FIELD_W + a, false)))
            return fail(g, SG_ERR_OOM, "sg_kernel_integrals: out of memory");
    if (mode == 1) {
        if (!ensure(g, g->stats, 256) || !ensure(g, g->sur_work, sur_work_bytes(g->P)))
            return fail(g, SG_ERR_OOM, "sg_kernel_integrals: out of memory");
        SG_CUDA(g, launch_surrogate_integrals(g, (const sg_mlp*)mlp, g->sur_work.p, o[0], o[1], o[2], o[3]),
                "surrogate integrals");
        return SG_OK;
    }
    SG_CUDA(g, launch_kernel_integrals(grid_f(g), (const int32_t*)g->nbr.p, (const float*)g->field[SG_FIELD_PHI].p, o[0],
                                       o[1], o[2], o[3], g->P, support_h(g->desc), heaviside_eps(g->desc), g->stream),
            "kernel integrals");
    return SG_OK;
}

sg_status sg_morton_order(sg_grid* g, int64_t n, const float* x, const float* y, const float* z, uint64_t* keys,
                          int32_t* order) {
    SG_TRACE("sg_morton_order");
    SG_CHECK_GRID(g);
    if (n < 0 || (n > 0 && (!x || !y || !z || !order))) return fail(g, SG_ERR_INVALID, "sg_morton_order: bad args");
    if (n >= (1LL << 31)) return fail(g, SG_ERR_CAPACITY, "sg_morton_order: too many particles");
    if (g->state < 1) return fail(g, SG_ERR_STATE, "sg_morton_order: grid not tagged");
    if (n == 0) return SG_OK;
    DeviceGuard dg(g->device);
    const GridF G = grid_f(g);
    if (!ensure(g, g->scratch, sort_scratch_bytes(n, morton_bits(G))))
        return fail(g, SG_ERR_OOM, "sg_morton_order: out of memory");
    SG_CUDA(g, morton_sort(G, n, x, y, z, keys, order, g->scratch.p, g->stream), "morton sort");
    return SG_OK;
}

sg_status sg_probe(sg_grid* g, int64_t n, const float* x, const float* y, const float* z, float* phi, float* nx,
                   float* ny, float* nz, float* W, float* Gx, float* Gy, float* Gz, int32_t flags) {
    SG_TRACE("sg_probe");
    SG_CHECK_GRID(g);
    if (n < 0 || (n > 0 && (!x || !y || !z))) return fail(g, SG_ERR_INVALID, "sg_probe: bad args");
    if (n >= (1LL << 31)) return fail(g, SG_ERR_CAPACITY, "sg_probe: too many particles");
    if (flags & ~SG_PROBE_MORTON) return fail(g, SG_ERR_INVALID, "sg_probe: unknown flags");
    if (g->state < 2) return fail(g, SG_ERR_STATE, "sg_probe: phi not initialised");
    if (n == 0) return SG_OK;
    DeviceGuard dg(g->device);
    ProbeFields F;
    const int src[8] = {SG_FIELD_PHI, SG_FIELD_GX, SG_FIELD_GY, SG_FIELD_GZ,
                        SG_FIELD_W,   SG_FIELD_GWX, SG_FIELD_GWY, SG_FIELD_GWZ};
    for (int f = 0; f < 8; ++f) {
        const bool fresh = field_fresh(g, src[f]);
        F.f[f] = field_ptr(g, src[f], true);
        if (!F.f[f]) return fail(g, SG_ERR_OOM, "sg_probe: out of memory");
        if (fresh && src[f] == SG_FIELD_W) SG_CUDA(g, launch_set_far((float*)F.f[f], 1.0f, 0.0f, g->stream), "probe W far");
    }
    ProbeOut O{{phi, nx, ny, nz, W, Gx, Gy, Gz}};
    const GridF G = grid_f(g);
    const int32_t* order = nullptr;
    const int* unsorted = nullptr;
    if (flags & SG_PROBE_MORTON) {
        size_t sb = sort_scratch_bytes(n, morton_bits(G));
        size_t ob = ((size_t)n * 4 + 255) & ~(size_t)255;
        if (!ensure(g, g->scratch, sb + ob)) return fail(g, SG_ERR_OOM, "sg_probe: out of memory");
        int32_t* ord = (int32_t*)((char*)g->scratch.p + sb);
        // results do not depend on the walk: a sampled check (one pair in 128, so that it reads about one
        // 32-byte sector of the positions in 16) decides whether the input is walked as it is
        SG_CUDA(g, morton_sort(G, n, x, y, z, nullptr, ord, g->scratch.p, g->stream, false, &unsorted, 128),
                "probe sort");
        order = ord;
    }
    SG_CUDA(g, launch_probe(G, (const int32_t*)g->cell_pkg.p, (const int32_t*)g->nbr.p, F, g->P, n, x, y, z, order, unsorted,
                            O, g->stream),
            "probe");
    return SG_OK;
}

sg_status sg_get_field(sg_grid* g, int32_t field, void** dev_ptr, int64_t* n_elems) {
    SG_CHECK_GRID(g);
    if (!dev_ptr || !n_elems) return fail(g, SG_ERR_INVALID, "sg_get_field: null output");
    DeviceGuard dg(g->device);
    if (field >= 0 && field < SG_N_FLOAT_FIELDS) {
        if (g->state < 1) return fail(g, SG_ERR_STATE, "sg_get_field: grid not tagged");
        const bool fresh = field_fresh(g, field);
        float* p = field_ptr(g, field, true);
        if (!p) return fail(g, SG_ERR_OOM, "sg_get_field: out of memory");
        if (fresh && field == SG_FIELD_W) SG_CUDA(g, launch_set_far(p, 1.0f, 0.0f, g->stream), "field W far");
        *dev_ptr = p;
        *n_elems = g->P * PKG3;
        return SG_OK;
    }
    if (g->state < 1) return fail(g, SG_ERR_STATE, "sg_get_field: grid not tagged");
    switch (field) {
    case SG_FIELD_CELL_PKG:
        *dev_ptr = g->cell_pkg.p;
        *n_elems = g->nc;
        return SG_OK;
    case SG_FIELD_PKG_CELL:
        *dev_ptr = g->pkg_cell.p;
        *n_elems = g->P;
        return SG_OK;
    case SG_FIELD_PKG_TYPE:
        *dev_ptr = g->pkg_type.p;
        *n_elems = g->P;
        return SG_OK;
    case SG_FIELD_NBR:
        *dev_ptr = g->nbr.p;
        *n_elems = g->P * NB;
        return SG_OK;
    default:
        return fail(g, SG_ERR_INVALID, "sg_get_field: unknown field");
    }
}

sg_status sg_restore(sg_grid* g, int64_t P, const int32_t* cell_pkg, const int32_t* pkg_cell, const uint8_t* pkg_type,
                     const int32_t* nbr, const float* phi) {
    SG_TRACE("sg_restore");
    SG_CHECK_GRID(g);
    if (P < 2 || !cell_pkg || !pkg_cell || !pkg_type || !nbr)
        return fail(g, SG_ERR_INVALID, "sg_restore: P < 2 or a null table");
    if (P >= (1LL << 31) / NB) return fail(g, SG_ERR_CAPACITY, "sg_restore: too many packages");
    DeviceGuard dg(g->device);
    for (int f = 0; f < SG_N_FLOAT_FIELDS; ++f) g->stale[f] = true;
    if (!ensure(g, g->cell_pkg, (size_t)g->nc * 4) || !ensure(g, g->pkg_cell, (size_t)P * 4) ||
        !ensure(g, g->pkg_type, (size_t)P) || !ensure(g, g->nbr, (size_t)P * NB * 4) ||
        !ensure(g, g->faces, (size_t)P * 8 * 4)) {
        g->state = 0;
        return fail(g, SG_ERR_OOM, "sg_restore: out of device memory");
    }
    g->P = P;
    g->state = 1;
    SG_CUDA(g, cudaMemcpyAsync(g->cell_pkg.p, cell_pkg, (size_t)g->nc * 4, cudaMemcpyHostToDevice, g->stream), "restore");
    SG_CUDA(g, cudaMemcpyAsync(g->pkg_cell.p, pkg_cell, (size_t)P * 4, cudaMemcpyHostToDevice, g->stream), "restore");
    SG_CUDA(g, cudaMemcpyAsync(g->pkg_type.p, pkg_type, (size_t)P, cudaMemcpyHostToDevice, g->stream), "restore");
    SG_CUDA(g, cudaMemcpyAsync(g->nbr.p, nbr, (size_t)P * NB * 4, cudaMemcpyHostToDevice, g->stream), "restore");
    SG_CUDA(g, launch_fill_faces((const int32_t*)g->nbr.p, (int32_t*)g->faces.p, P, g->stream), "restore faces");
    // a checkpoint is input: the tables are checked (bounds and consistency) before the grid is used
    SG_CUDA(g, cudaMemsetAsync(g->err.p, 0, sizeof(int32_t), g->stream), "restore");
    SG_CUDA(g, launch_check_tables(grid_ff(g), (const int32_t*)g->cell_pkg.p, (const int32_t*)g->pkg_cell.p,
                                   (const uint8_t*)g->pkg_type.p, (const int32_t*)g->nbr.p, (const int32_t*)g->faces.p,
                                   g->P, g->nc, (int*)g->err.p, g->stream),
            "restore check");
    if (phi) {
        float* d = field_ptr(g, SG_FIELD_PHI, false);
        if (!d) return fail(g, SG_ERR_OOM, "sg_restore: out of device memory");
        SG_CUDA(g, cudaMemcpyAsync(d, phi, (size_t)P * PKG3 * 4, cudaMemcpyHostToDevice, g->stream), "restore phi");
    }
    SG_CUDA(g, cudaMemcpyAsync(g->host_pin.p, g->err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream), "restore");
    SG_CUDA(g, cudaStreamSynchronize(g->stream), "restore sync");  // the host arrays may be temporary
    if (*(int32_t*)g->host_pin.p) {
        g->state = 0;
        SG_CUDA(g, cudaMemsetAsync(g->err.p, 0, sizeof(int32_t), g->stream), "restore");
        return fail(g, SG_ERR_INVALID, "sg_restore: the tables are not consistent");
    }
    g->state = phi ? 2 : 1;
    return SG_OK;
}

sg_status sg_check_tables(sg_grid* g) {
    SG_TRACE("sg_check_tables");
    SG_CHECK_GRID(g);
    if (g->state < 1) return fail(g, SG_ERR_STATE, "sg_check_tables: grid not tagged");
    DeviceGuard dg(g->device);
    SG_CUDA(g, launch_check_tables(grid_ff(g), (const int32_t*)g->cell_pkg.p, (const int32_t*)g->pkg_cell.p,
                                   (const uint8_t*)g->pkg_type.p, (const int32_t*)g->nbr.p, (const int32_t*)g->faces.p,
                                   g->P, g->nc, (int*)g->err.p, g->stream),
            "check tables");
    return SG_OK;
}

sg_status sg_clear_error(sg_grid* g) {
    SG_CHECK_GRID(g);
    DeviceGuard dg(g->device);
    SG_CUDA(g, cudaMemsetAsync(g->err.p, 0, sizeof(int32_t), g->stream), "clear error");
    return SG_OK;
}

sg_status sg_status_sync(sg_grid* g) {
    SG_CHECK_GRID(g);
    DeviceGuard dg(g->device);
    SG_CUDA(g, cudaStreamSynchronize(g->stream), "sync");
    SG_CUDA(g, cudaMemcpy(g->host_pin.p, g->err.p, sizeof(int32_t), cudaMemcpyDeviceToHost), "error word");
    int32_t w = *(int32_t*)g->host_pin.p;
    if (w & ERR_TIMEOUT) return fail(g, SG_ERR_TIMEOUT, "device wait timed out");
    if (w) return fail(g, SG_ERR_DEVICE, "device reported an inconsistency");
    return SG_OK;
}

}  // extern "C"
