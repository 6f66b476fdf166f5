// Shared definitions of the IIM library: complex type, error handling, twiddle tables,
// geometry and workspace structures.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <utility>
#include <vector>

#include "../../include/iim.h"

namespace iim {

// ------------------------------------------------------------------------- errors
void record_cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define IIM_TRY(call)                                                     \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) {                                          \
            ::iim::record_cuda_error(e_, #call, __FILE__, __LINE__);      \
            return IIM_ERR_CUDA;                                          \
        }                                                                 \
    } while (0)

#define IIM_LAUNCHED()                                                    \
    do {                                                                  \
        cudaError_t e_ = cudaGetLastError();                              \
        if (e_ != cudaSuccess) {                                          \
            ::iim::record_cuda_error(e_, "kernel launch", __FILE__, __LINE__); \
            return IIM_ERR_CUDA;                                          \
        }                                                                 \
    } while (0)

#define IIM_CHECK(st)                 \
    do {                              \
        iim_status s_ = (st);         \
        if (s_ != IIM_OK) return s_;  \
    } while (0)

// ------------------------------------------------------------------------- complex
template <typename T>
struct cpx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// ------------------------------------------------------------------------- twiddles
// exp(-i pi k / 4096), k = 0..4095, in both precisions.  The DST of length n - 1 (n a power
// of two <= 4096) uses entry k * (4096 / n).  Filled once per device from host cos/sin.
constexpr int kTwLog = 12;
constexpr int kTwN = 1 << kTwLog;
iim_status ensure_twiddles();                 // for the current device
const cpx<double>* twiddles64();              // device address, current device
const cpx<float>* twiddles32();
// Twiddle region of the DST kernels for lines of n points on FFT path fp (dst.cuh, tw_region
// entries: the full half table, then the path's stage tables), in global memory of the current
// device, built by ensure_twiddles for every n = 16..4096.
template <typename T>
const cpx<T>* twiddle_region(int n, int fp);

// ------------------------------------------------------------------------- node classes
enum : uint8_t { CLS_FLUID = 0, CLS_PLUS = 1, CLS_MINUS = 2, CLS_SOLID = 3 };

inline int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}
inline bool is_pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

// Counts every kernel launch of the library; while profiling is on (iim_profile_begin) it
// also records CUDA events around the launch on its stream, tagged with the kernel's name and
// its algorithmic bytes / flops.
struct KTrace {
    KTrace(const char* name, cudaStream_t s, double bytes = 0.0, double flops = 0.0);
    ~KTrace();
    bool active;
    cudaStream_t stream;
    int idx;
};

// While a stream capture is being recorded, launches are neither counted nor timed (the
// replays of the captured graph are counted by the caller through count_launches).
void set_capture(bool on);
bool profiling_active();
void count_launches(long long n);

// k<<<grid, block, smem, s>>>(args...) with launch accounting.
template <typename... KArgs, typename... Args>
inline void launch(const char* name, double bytes, double flops, void (*k)(KArgs...), dim3 grid, dim3 block,
                   size_t smem, cudaStream_t s, Args&&... args) {
    KTrace t(name, s, bytes, flops);
    k<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
}

}  // namespace iim

// Geometry handle: everything iim_setup_geometry builds, plus the solver workspace.
struct iim_geometry_s {
    int device = 0;
    iim_grid grid{};
    int nx = 0, ny = 0, NX = 0, NY = 0;  // cells and interior sizes
    double h = 0.0;
    int nb = 0, ncirc = 0;
    std::vector<iim_region> regions;
    std::vector<int> modes;
    std::vector<int> circ_ids;  // body index of each circulation-mode body
    int ncp = 0, na = 0, nminus = 0;
    int ja0 = 0, ja1 = -1;      // interior rows holding affected points (inclusive)
    int jo0 = 0, jo1 = -1;      // interior rows the gather stencils read (inclusive)

    // control points (canonical order)
    double *cp_x = nullptr, *cp_y = nullptr, *cp_t = nullptr;
    int *cp_body = nullptr, *cp_axis = nullptr, *cp_ei = nullptr, *cp_ej = nullptr;
    // affected points (row-major order)
    int *aff_node = nullptr, *aff_body = nullptr, *aff_row_ptr = nullptr;
    uint8_t* aff_solid = nullptr;
    // gamma = A psi + B bc as CSR over affected points; idx >= 0: interior node, idx < 0:
    // control point (-idx - 1)
    int *gop_ptr = nullptr, *gop_idx = nullptr;
    double* gop_w = nullptr;
    // fourth-order ghost values at A- nodes (velocity, residual)
    int *minus_node = nullptr, *gh_ptr = nullptr, *gh_idx = nullptr;
    double* gh_w = nullptr;
    int* minus_cp = nullptr;             // 4 per A- node: control point per direction or -1
    uint8_t* minus_mask = nullptr;       // per A- node: bit d fourth-order usable, bit 4+d third-order
    int* minus_map = nullptr;            // padded node -> A- index or -1
    double* tr_buf = nullptr;            // transport workspace (allocated on first use)
    // wall condition of the ghost stencils (iim_geometry_set_wall_condition): 0 Dirichlet
    // (psi_b + psibar_k), 1 Neumann (derivative along the grid line into the fluid); zeros read
    // as psibar in Neumann mode; scratch of iim_total_pressure (right-hand side, wall data)
    int wall = 0;
    double* psibar_zero = nullptr;
    double* pr_buf = nullptr;
    uint8_t* node_class = nullptr;       // padded layout
    int* body_circ = nullptr;            // per body: index among circulation bodies or -1
    iim_region* d_regions = nullptr;
    // eigenvalues of the 1D three-point operators, x modes (NX) and y modes (NY)
    double *lam_x64 = nullptr, *lam_y64 = nullptr;
    float *lam_x32 = nullptr, *lam_y32 = nullptr;
    // factors of the tridiagonal column pass (tri.cuh), FP32 and FP64: complements of the
    // Thomas factors (FP64 table, row-major over rows, and its row offsets), per-column table
    // limits and limits 1 - e*; col_solver 1 = tridiagonal column pass, 0 = column transforms
    float* sc32_delta = nullptr;
    double* sc64_delta = nullptr;
    int *sc32_rowoff = nullptr, *sc32_lim = nullptr, *sc64_rowoff = nullptr, *sc64_lim = nullptr;
    float* sc32_dstar = nullptr;
    double* sc64_dstar = nullptr;
    float4* sc32_par = nullptr;   // FP32: per-column parameters of the closed form (tri.cuh)
    int col_solver = 1;
    // free space (iim_geometry_set_outer): 0 = Dirichlet box, 1 = unbounded, 2 = unbounded with
    // the outflow plane through the right box edge (freespace.cu); the lattice Green's function
    // table (shared per size, not owned; columns 0..nx, or 0..2nx with the plane, row stride
    // lgf_ld), psi on the box ring of the current solve, the ring sum of the last free-space
    // application, and psi_1 next to the box (first / last interior row, then first / last
    // interior column); the vorticity on the plane column (NY values) and a switch that leaves it
    // out (the unit-circulation responses)
    int outer = 0;
    const double* lgf = nullptr;
    int lgf_ld = 0;
    double* fs_plane = nullptr;
    int plane_off = 0;
    double *fs_ring = nullptr, *fs_rho = nullptr, *fs_bnd = nullptr;
    double* fs_rres = nullptr;   // ring rows of the last FP64 residual
    double* cap_ring = nullptr;  // ring values of the unit-circulation responses (free space)

    // ---- solver workspace
    double* psi_ext = nullptr;   // NY*NX FP64: fluid values, ghosts at A-, 0 elsewhere
    double* res = nullptr;       // NY*NX FP64 residual (correction right-hand side)
    void* tbuf = nullptr;        // NY*NX of T: transform buffer
    void* psiT = nullptr;        // NY*NX of T: rectangular-solve output for gathers
    double* partial = nullptr;   // reduction partials
    double* small = nullptr;     // small per-solve vectors (see solve.cu)
    int krylov_m = 0;            // restart length the Krylov buffers were sized for
    double* V = nullptr;         // (m+1) * ns Krylov basis
    double* H = nullptr;         // small Hessenberg / Givens storage
    double* xsol = nullptr;      // ns
    double* bvec = nullptr;      // ns
    double* x0g = nullptr;       // ns: Krylov starting point from a guess
    int* d_int = nullptr;        // device counters / flags
    double* h_pinned = nullptr;  // pinned host scalars
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // dense Schur-complement preconditioner: [S | S^-1] row-major ns x 2ns (FP32), scratch
    float* pc_aug = nullptr;
    float* pc_S = nullptr;   // copy of S itself (ns x ns, FP32) kept before the inversion
    float* pc_f = nullptr;   // Gauss-Jordan scratch (gj_scratch_floats)
    int* pc_info = nullptr;
    double* pc_z = nullptr;      // 2 ns
    int pc_ready = 0;
    float pc_setup_ms = 0.f;
    int cols_c = 4;              // column-pass tile width (autotuned per size bucket)
    int wide_lines = 0;          // 64 threads per 1024-point line (lower latency, more instructions)
    // capacitance correction of the circulation: responses to unit circulation of each
    // circulation body (padded psi_ext fields, ncirc of them), their psibar values
    // ([response][circulation body]) and the inverse of their measured circulations
    int cap_ready = 0;
    double* cap_psi = nullptr;
    std::vector<double> cap_pb, cap_cinv;
    double* cap_dev = nullptr;   // device copies: C^-1 (nc x nc), then the psibar table (nc x nc)
    // the whole solve as one graph (device-driven refinement; see solve.cu), its key, and the
    // number of host-driven solves done on this geometry (the first solve always runs on the host)
    void* solve_graph = nullptr;
    double* io = nullptr;        // device staging of the host-buffer batched solve (on first use)
    int host_solves = 0;
    int solve_graph_failed = 0;
    cudaStream_t cap_stream = nullptr;   // private stream used only to capture graphs
    void* graph64 = nullptr;     // captured GMRES iteration (FP64 transforms)
    void* graph32 = nullptr;     // captured GMRES iteration (FP32 transforms)
};

namespace iim {
void destroy_graphs(iim_geometry g);
// whole-solve graph without waiting: *enqueued = 1 launched on s (then solve_finish after the
// stream is synchronised), 0 solved to completion, -1 not applicable yet (nothing done)
iim_status solve_enqueue(iim_geometry g, const double* omega, const double* psi_b, const double* psi_box,
                         const double* gamma, double* psibar, double* psi_out, double* ux_out, double* uy_out,
                         const iim_opts* opts, iim_stats* stats, cudaStream_t s, int* enqueued);
iim_status solve_finish(iim_geometry g, const iim_opts* opts, iim_stats* stats);
void set_last_error(const char* msg);
// lockstep batched solves (lockstep.cu): problems of one grid size advanced together, one launch
// per step for all of them
bool lockstep_eligible(iim_geometry g, const iim_opts& o);
int lockstep_group_size();
iim_status lockstep_enqueue(const std::vector<int>& idx, iim_geometry const* geoms, const double* const* omega,
                            const double* const* psi_b, const double* const* psi_box, const double* const* gamma,
                            double* const* psibar, double* const* psi_out, double* const* ux_out,
                            double* const* uy_out, const iim_opts& o, cudaStream_t s, bool host_driven,
                            void** handle);
void lockstep_finish(void* handle, const std::vector<int>& idx, const iim_opts& o, bool host_driven,
                     std::vector<iim_status>& status, std::vector<iim_stats>& stats);
void lockstep_forget(iim_geometry g);
// Rewrites the ghost-stencil weights (gop rows of A+ points, gh rows) for wall condition `kind`
// (0 Dirichlet, 1 Neumann) from the stored crossings; synchronizes `s`.
iim_status rewrite_wall_weights(iim_geometry g, int kind, cudaStream_t s);
// free-space rectangular solve (freespace.cu)
iim_status lgf_table(int nx, int ny, const double** out);
template <typename T>
iim_status launch_bnd_cols(int NX, int NY, int nx, const T* buf, double* vl, double* vr, const int* stop,
                           cudaStream_t s);
iim_status launch_ring_conv(int nx, int ny, const double* G, int ld, int sym, const double* bnd, const double* vl,
                            const double* vr, double* rho, const int* stop, cudaStream_t s);
iim_status launch_ring_add(int n, double a, const double* x, double* y, const int* stop, cudaStream_t s);
iim_status launch_ring_residual(int nx, int ny, double h, const double* G, int ld, int sym, const double* plane,
                                const double* psi, const double* ring, double* rres, double* res2, cudaStream_t s);
// dense Schur-complement preconditioner (precond.cu)
// [S | I] -> [I | S^-1] in place; scratch holds gj_scratch_floats(n) floats
size_t gj_scratch_floats(int n);
iim_status gj_invert_aug(float* A, int n, float* scratch, int* info, cudaStream_t s);
iim_status dense_matvec(int n, const float* M, long ldm, const double* v, const int* jidx, long vstride, double* out,
                        int accumulate, const int* stop, cudaStream_t s);
bool dense_matvec_fits(int n);
iim_status dense_matvec_to(int n, const float* M, long ldm, const double* v, double* outb, const int* ojidx,
                           long ostride, const int* stop, cudaStream_t s);
__global__ void k_unit_vector(int n, int j, double* v);
__global__ void k_store_column(int n, int j, const double* v, float* A);
}
