// sg_internal.cuh -- grid object and launcher declarations shared by the
// translation units of libsg.  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sg.h"
#include "sg_ff.cuh"

#include <nvtx3/nvToolsExt.h>

namespace sg {
// A named NVTX range in the library's own domain ("libsg") around each
// boundary call that issues work, so that a profiler files every kernel
// under the call that launched it.  NVTX is header-only: with no tool
// attached a push and a pop are calls through stubs that do nothing.
inline nvtxDomainHandle_t trace_domain() {
    static const nvtxDomainHandle_t d = nvtxDomainCreateA("libsg");
    return d;
}
struct TraceRange {
    explicit TraceRange(const char* name) {
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(trace_domain(), &a);
    }
    ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};
}  // namespace sg
#define SG_TRACE(name) const ::sg::TraceRange sg_trace_range_(name)

namespace sg {

constexpr int PKG = 4;    // data per axis in a package
constexpr int PKG3 = 64;  // data per package
constexpr int NB = 27;    // entries of the neighbourhood table

// device error word bits
constexpr int ERR_BAD_INDEX = 1;
constexpr int ERR_TIMEOUT = 2;

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Scalars every stencil kernel needs, in float.
struct GridF {
    float lo[3];
    float h;
    int dims[3];
    float F;
    double h_d;   // h in double, for host-side constants
    float inv_h;  // 1/h rounded to float once
    ff lat_c[3];  // lo / h + 1/2 per axis, float-float (the probe's lattice coordinate)
    ff lat_ih;    // 1 / h, float-float
};

// v as a float-float pair (host side): hi = v rounded to float, lo = the rest.
inline ff split_ff(double v) {
    const float hi = (float)v;
    return ff{hi, (float)(v - (double)hi)};
}

// Constants of the probe's lattice coordinate u = (x - lo)/h - 1/2, written
// as u = x (1/h) - (lo/h + 1/2).
inline void set_lattice(ff (&c)[3], ff& ih, const double lo[3], double h) {
    for (int a = 0; a < 3; ++a) c[a] = split_ff(lo[a] / h + 0.5);
    ih = split_ff(1.0 / h);
}

// Scalars of the tagging/init kernels, in float-float.
struct GridFF {
    ff lo[3];
    ff h;
    ff T;  // core threshold lc (1 - 2^-10)
    int dims[3];
};

}  // namespace sg

struct sg_grid {
    sg_grid_desc desc;
    double F = 0;
    int64_t nc = 0;   // background cells
    int64_t P = 0;    // packages incl. the 2 far packages
    int state = 0;    // 0 created, 1 tagged, 2 phi valid
    sg_allocator alloc{};
    bool user_alloc = false;
    cudaStream_t stream = nullptr;
    int device = 0;

    sg::Buf cell_pkg, cell_type, pkg_cell, pkg_type, nbr;
    sg::Buf faces;  // int32 [P][8]: the six face neighbours (-x,+x,-y,+y,-z,+z), then 2 zeros
    sg::Buf field[SG_N_FLOAT_FIELDS];
    bool stale[SG_N_FLOAT_FIELDS] = {};  // buffer kept from an earlier tagging: treated as new
    sg::Buf phi_tmp;
    sg::Buf err;       // int32 sticky device error word
    sg::Buf scratch;   // reusable temporary space (scans, sort)
    sg::Buf stats;     // class counts of the last surrogate integral call
    sg::Buf sur_work;  // list of network points of the surrogate integrals
    sg::Buf host_pin;  // pinned host word for read-backs
    bool host_pin_pooled = false;  // a slot of the process-wide pinned block (sg_api.cu)
    std::string last_error;
};

namespace sg {

// The two far packages of a field (far- then far+, 64 points each), written
// by CTA 0 of the kernel that computes the field (blocks of at least 128
// threads), so that no launch of its own is needed.
__device__ __forceinline__ void write_far(float* f, float v_in, float v_out) {
    if (blockIdx.x == 0 && threadIdx.x < 2 * PKG3) f[threadIdx.x] = threadIdx.x < PKG3 ? v_in : v_out;
}

// process-wide count of kernels launched by the library (sg_api.cu)
void note_launch(int n = 1);

// Programmatic dependent launch: a kernel launched by launch_pdl may start
// while the kernel before it on the stream drains.  It calls pdl_enter()
// before touching memory: that waits until the previous grid has completed
// (its writes visible), then lets the next programmatic dependent launch.
// Without a programmatic prerequisite both instructions return at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    note_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}
// sg_debug_wide_offsets: take the 64-bit address kernels at any size (sg_api.cu)
bool force_wide_offsets();

// memory (sg_api.cu)
void* grid_alloc(sg_grid* g, size_t bytes);
void grid_free(sg_grid* g, Buf& b);
bool ensure(sg_grid* g, Buf& b, size_t bytes);  // (re)allocates when too small
sg_status fail(sg_grid* g, sg_status st, const std::string& msg);
sg_status cuda_fail(sg_grid* g, cudaError_t e, const char* where);
float* field_ptr(sg_grid* g, int f, bool zero_new);
bool field_fresh(const sg_grid* g, int f);  // field_ptr would hand out a new (or stale) buffer
GridF grid_f(const sg_grid* g);
GridFF grid_ff(const sg_grid* g);
ShapeFF shape_ff(const sg_shape* s);

// scans (sg_scan.cu): exclusive prefix sum of n uint32 values into out
// (may alias in), total into *total (device).  Scratch: scan_scratch_bytes(n).
// With run != nullptr the kernels do nothing when *run == 0 (device flag).
size_t scan_scratch_bytes(int64_t n);
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* scratch,
                               cudaStream_t s, const int* run = nullptr);

// tagging / init (sg_tag.cu)
// Step 1: cell_type[nc] and the core mask (bit i of core_bits[w] = cell
// 32 w + i is core).
cudaError_t launch_tag_flags(const GridFF& G, const ShapeFF& S, uint8_t* cell_type, uint32_t* core_bits, int64_t nc,
                             cudaStream_t s);
cudaError_t launch_tag_flags_from(const GridFF& G, const ShapeFF& S, const int32_t* c_cell_pkg,
                                  const uint8_t* c_pkg_type, const float* c_phi, int cnx, int cny, uint8_t* cell_type,
                                  uint32_t* core_bits, int64_t nc, unsigned long long* evaluated, cudaStream_t s);
// Consistency of the cell, package, neighbour and face tables; sets
// ERR_BAD_INDEX in *err on any inconsistency (reads are bounds-checked).
cudaError_t launch_check_tables(const GridFF& G, const int32_t* cell_pkg, const int32_t* pkg_cell,
                                const uint8_t* pkg_type, const int32_t* nbr, const int32_t* faces, int64_t P,
                                int64_t nc, int* err, cudaStream_t s);
// Morton package ids: cell centres of the n active packages (linear ids),
// then the move of package 2 + order[r] to id 2 + r (tables and cells).
cudaError_t launch_cell_centres(const GridF& G, const int32_t* pkg_cell, float* x, float* y, float* z, int64_t n,
                                cudaStream_t s);
cudaError_t launch_renumber(const int32_t* order, const int32_t* old_cell, const uint8_t* old_type, int32_t* pkg_cell,
                            uint8_t* pkg_type, int32_t* cell_pkg, int64_t n, cudaStream_t s);
// Step 2: inner cells (type 3), the active mask and its population per
// 32-cell word; step 3: ids from the scanned populations.
cudaError_t launch_tag_inner(const GridFF& G, uint8_t* cell_type, const uint32_t* core_bits, uint32_t* act_bits,
                             uint32_t* count, int64_t nc, cudaStream_t s);
cudaError_t launch_tag_scatter(const uint8_t* cell_type, const uint32_t* act_bits, const uint32_t* prefix,
                               int32_t* cell_pkg, int32_t* pkg_cell, uint8_t* pkg_type, int64_t nc, cudaStream_t s);
cudaError_t launch_fill_nbr(const GridFF& G, const int32_t* cell_pkg, const int32_t* pkg_cell, int32_t* nbr,
                            int64_t P, cudaStream_t s);
// Consistency (sign) correction of phi, cell_pkg, nbr and faces in place;
// host-synchronising.  out: points flipped, far cells moved, point and cell
// flood sweeps.
size_t consistency_scratch_bytes(int64_t P, const int32_t dims[3]);
cudaError_t run_consistency(const GridFF& G, int64_t P, int64_t nc, int32_t* cell_pkg, const int32_t* pkg_cell,
                            const uint8_t* pkg_type, int32_t* nbr, int32_t* faces, float* phi, float tau,
                            void* scratch, void* host_pin, int64_t out[4], cudaStream_t s,
                            unsigned debug = 0);
// whether the device can run the persistent (cooperative) floods
bool consistency_persistent(int device);
// faces[p][8] = the six face entries of nbr[p][27] (one 32-byte row per package)
cudaError_t launch_fill_faces(const int32_t* nbr, int32_t* faces, int64_t P, cudaStream_t s);
// Level set at the data points; table: scratch of init_table_bytes(G) for
// the tabulated lattice coordinates.
cudaError_t launch_init_sdf(const GridFF& G, const ShapeFF& S, const int32_t* pkg_cell, float* phi, float F,
                            int64_t P, void* table, cudaStream_t s);
inline size_t init_table_bytes(const GridFF& G) { return (size_t)4 * (G.dims[0] + G.dims[1] + G.dims[2]) * 8; }

// sweeps (sg_sweep.cu)
cudaError_t launch_set_far(float* f, float v_in, float v_out, cudaStream_t s);
cudaError_t launch_gradient(const GridF& G, const int32_t* faces, const float* phi, float* gx, float* gy, float* gz,
                            int64_t P, cudaStream_t s);
cudaError_t launch_laplacian(const GridF& G, const int32_t* faces, const float* phi, float* lap, int64_t P,
                             cudaStream_t s);
cudaError_t launch_reinit_s0(const GridF& G, const float* phi, float* s0, int64_t P, cudaStream_t s);
// One Jacobi sweep; `reverse` walks the packages from the last CTA down;
// `first` forms S0 from phi_in and stores it instead of reading it.
cudaError_t launch_reinit_step(const GridF& G, const int32_t* faces, float* s0, const float* phi_in,
                               float* phi_out, float dt, int64_t P, int reverse, int first, cudaStream_t s);
cudaError_t launch_copy_active(const float* src, float* dst, int64_t P, cudaStream_t s);
// phi <- phi + delta on the active packages
cudaError_t launch_sequential(float* phi, float delta, int64_t P, cudaStream_t s);
// R: kernel support in units of h (<= 3); eps: Heaviside half width.
// The exact integrals (support <= 2h) over a batch's store: packages of type
// < 2 are left as they are, each package takes the Heaviside width of its
// body, 1 / ieps_b[body[p] * ieps_stride].
cudaError_t launch_batch_kernel_integrals(const int32_t* nbr, const uint8_t* type, const int32_t* body,
                                          const float* ieps_b, int ieps_stride, const float* phi, float* W, float* gx,
                                          float* gy, float* gz, int64_t P, double R, cudaStream_t s);
cudaError_t launch_kernel_integrals(const GridF& G, const int32_t* nbr, const float* phi, float* W, float* gx,
                                    float* gy, float* gz, int64_t P, double R, double eps, cudaStream_t s);
// The kernel support of a grid in units of h and its Heaviside half width.
inline double support_h(const sg_grid_desc& d) { return d.kernel_support > 0.0 ? d.kernel_support / d.h : 2.0; }
inline double heaviside_eps(const sg_grid_desc& d) { return d.heaviside_eps > 0.0 ? d.heaviside_eps : d.h; }
// The surrogate was trained for the default kernel (support 2h, eps = h).
inline bool default_kernel(const sg_grid_desc& d) {
    return (d.kernel_support == 0.0 || d.kernel_support == 2.0 * d.h) && (d.heaviside_eps == 0.0 || d.heaviside_eps == d.h);
}

// surrogate (sg_mlp.cu).  Work space of the two-pass surrogate integrals of
// P packages: a list counter and the list of network points.
size_t sur_work_bytes(int64_t P);
cudaError_t launch_surrogate_integrals(sg_grid* g, const sg_mlp* m, void* work, float* W, float* gx, float* gy,
                                       float* gz);
// Surrogate constants of a body of spacing h: 1/h (the network inputs),
// h_up = the least float >= h (a float f has |f| >= h exactly when
// |f| >= h_up, and |f| < h when |f| < h_up), and the curvature bound
// 0.1 h of the fallback's Laplacian numerator, in float and float-float;
// 1/eps of the Heaviside (eps = h).
// The surrogate path indexes data points in 32 bits (list entries) and
// gathers with 32-bit byte offsets: stores of at most 2^24 - 1 packages.
constexpr int64_t SUR_MAX_PACKAGES = (int64_t)1 << 24;

struct SurConst {
    float inv_h, h_up, kap_thr;
    ff kap_thr_ff;
};
struct SurBody {
    SurConst C;
    float inv_eps;
};
SurBody sur_body(double h);
// Opt the batched surrogate kernel into its shared memory (once per device,
// outside any stream capture).
cudaError_t setup_batch_surrogate();
// Surrogate integrals over a batch store: packages of type >= 2 take their
// body's constants sb[body[p]]; far packages are left as they are.
cudaError_t launch_batch_surrogate_integrals(const int32_t* nbr, const uint8_t* type, const int32_t* body,
                                             const SurBody* sb, const float* phi, float* W, float* gx, float* gy,
                                             float* gz, int64_t P, const sg_mlp* m, void* work, int* err, int device,
                                             cudaStream_t s);

// probe (sg_probe.cu)
struct ProbeFields {
    const float* f[8];  // phi, gx, gy, gz, W, Gx, Gy, Gz
};
struct ProbeOut {
    float* o[8];  // phi, nx, ny, nz, W, Gx, Gy, Gz (entries may be null)
};
int morton_bits(const GridF& G);  // significant key bits
size_t sort_scratch_bytes(int64_t n, int key_bits);
// Stable Morton sort.  The key pass also checks whether the keys are already
// non-decreasing; if so the radix passes return at once and order_out is
// the identity (written only when identity_out, else left to the caller,
// who reads the device flag *unsorted_out: 0 = input already in order).
// check_stride > 1: the sortedness check compares only every check_stride-th
// adjacent pair (for callers to whom the order is a matter of speed only).
cudaError_t morton_sort(const GridF& G, int64_t n, const float* x, const float* y, const float* z, uint64_t* keys_out,
                        int32_t* order_out, void* scratch, cudaStream_t s, bool identity_out = true,
                        const int** unsorted_out = nullptr, int check_stride = 1);
// Point-interleaved probe table of n_points data points from the 8 fields:
// tab[e] = (phi, gx, gy, gz), tab[n_points + e] = (W, Gx, Gy, Gz).
cudaError_t launch_pack_probe(const ProbeFields& F, float4* tab, int64_t n_points, cudaStream_t s);
cudaError_t launch_probe(const GridF& G, const int32_t* cell_pkg, const int32_t* nbr, const ProbeFields& F,
                         int64_t P, int64_t n, const float* x, const float* y, const float* z, const int32_t* order,
                         const int* unsorted, const ProbeOut& out, cudaStream_t s);

}  // namespace sg
