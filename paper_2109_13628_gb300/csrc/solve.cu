// IIM Poisson solve (Sec. 4.2) on the device.
//
// Outer loop: FP64 iterative refinement of the un-reduced system.  The residual r of the
// un-reduced equations (five-point Laplacian of the extended psi at fluid nodes, box data,
// ghosts from psi_b + psibar_k; circulation rows / h^2) is evaluated in FP64; a correction
// with homogeneous data solves L delta = r in Schur form:
//   (I + A P E_a) dgamma - B sum_k dpsibar_k 1_k = A P r
//   sum_{B_k} dgamma = sum_{R_k} r - rc_k            (rc_k: circulation row residual)
//   delta = P (r - E_a dgamma)
// where P = -nabla_h^-2 is the Dirichlet-box DST solve.  This is Eq. schur / psirecovery and
// the augmented system of Sec. 4.2 with the sign derived from Eqs. discretepoisson and
// poissoncorrections (P = -nabla_h^-2 turns the printed "+ A nabla^-2 E_a" into "+ A P E_a").
// The Krylov solver is restarted GMRES with classical Gram-Schmidt applied twice; all Krylov
// vectors and inner products are FP64.  In FP64 mode the rectangular solves use FP64
// transforms; in mixed mode FP32 transforms (the refinement keeps the FP64 residual exact).
//
// One GMRES iteration is a fixed sequence of kernels that read the iteration index from
// device memory and become no-ops once a device stop flag is set.  The sequence is captured
// once as the body of a WHILE conditional graph node, so a whole restart cycle runs on the
// device from one graph launch; the host reads the convergence state once per cycle.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "dst.cuh"
#include "iim_ops.cuh"

namespace iim {

// ------------------------------------------------------------------------- errors, tables
static thread_local char g_last_error[512];

void set_last_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

void record_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

__device__ cpx<double> g_tw64[kTwN];
__device__ cpx<float> g_tw32[kTwN];

// Twiddle regions of the DST kernels, one per line length n = 2^4..2^12 (the one-warp path of
// that length) plus the 64-thread path of n = 1024: read by the kernels from global memory
// (L1-cached) instead of a copy in every block's shared memory.
constexpr int twr_slot(int logn, bool wide) { return wide ? 9 : logn - 4; }
constexpr int kTwrSlots = 10;
constexpr long twr_total() {
    long t = 0;
    for (int l = 4; l <= kTwLog; ++l) t += tw_region(1 << l);
    return t + tw_region(1024);
}
__device__ cpx<double> g_twr64[twr_total()];
__device__ cpx<float> g_twr32[twr_total()];

template <typename T, int FP>
__global__ void k_twiddle_region(const cpx<T>* __restrict__ g_tw, int n, int logn, cpx<T>* __restrict__ out) {
    load_twiddles<FP>(out, g_tw, n, logn);
}

static std::mutex g_tw_mutex;
static bool g_tw_ready[64];
static const cpx<double>* g_tw64_addr[64];
static const cpx<float>* g_tw32_addr[64];
static const cpx<double>* g_twr64_addr[64][kTwrSlots];
static const cpx<float>* g_twr32_addr[64][kTwrSlots];

template <typename T>
static iim_status fill_regions(const cpx<T>* base, cpx<T>* regions, const cpx<T>** addr) {
    long off = 0;
    for (int slot = 0; slot < kTwrSlots; ++slot) {
        const bool wide = slot == 9;
        const int logn = wide ? 10 : slot + 4, n = 1 << logn;
        const int fp = fft_path(n, wide);
        cpx<T>* out = regions + off;
        if (fp == 64) k_twiddle_region<T, 64><<<1, 256>>>(base, n, logn, out);
        else if (fp == 16) k_twiddle_region<T, 16><<<1, 256>>>(base, n, logn, out);
        else if (fp == 8) k_twiddle_region<T, 8><<<1, 256>>>(base, n, logn, out);
        else k_twiddle_region<T, 0><<<1, 256>>>(base, n, logn, out);
        IIM_TRY(cudaGetLastError());
        addr[slot] = out;
        off += tw_region(n);
    }
    return IIM_OK;
}

iim_status ensure_twiddles() {
    int dev = 0;
    IIM_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return IIM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_tw_mutex);
    if (g_tw_ready[dev]) return IIM_OK;
    std::vector<cpx<double>> t64(kTwN);
    std::vector<cpx<float>> t32(kTwN);
    for (int k = 0; k < kTwN; ++k) {
        const double a = M_PI * (double)k / (double)kTwN;
        t64[k] = {std::cos(a), -std::sin(a)};
        t32[k] = {(float)t64[k].x, (float)t64[k].y};
    }
    IIM_TRY(cudaMemcpyToSymbol(g_tw64, t64.data(), sizeof(cpx<double>) * kTwN));
    IIM_TRY(cudaMemcpyToSymbol(g_tw32, t32.data(), sizeof(cpx<float>) * kTwN));
    void* p64 = nullptr;
    void* p32 = nullptr;
    IIM_TRY(cudaGetSymbolAddress(&p64, g_tw64));
    IIM_TRY(cudaGetSymbolAddress(&p32, g_tw32));
    g_tw64_addr[dev] = (const cpx<double>*)p64;
    g_tw32_addr[dev] = (const cpx<float>*)p32;
    void* r64 = nullptr;
    void* r32 = nullptr;
    IIM_TRY(cudaGetSymbolAddress(&r64, g_twr64));
    IIM_TRY(cudaGetSymbolAddress(&r32, g_twr32));
    IIM_CHECK(fill_regions<double>(g_tw64_addr[dev], (cpx<double>*)r64, g_twr64_addr[dev]));
    IIM_CHECK(fill_regions<float>(g_tw32_addr[dev], (cpx<float>*)r32, g_twr32_addr[dev]));
    IIM_TRY(cudaDeviceSynchronize());
    g_tw_ready[dev] = true;
    return IIM_OK;
}

template <>
const cpx<double>* twiddle_region<double>(int n, int fp) {
    int dev = 0;
    cudaGetDevice(&dev);
    return g_twr64_addr[dev][twr_slot(ilog2(n), fp == 64)];
}
template <>
const cpx<float>* twiddle_region<float>(int n, int fp) {
    int dev = 0;
    cudaGetDevice(&dev);
    return g_twr32_addr[dev][twr_slot(ilog2(n), fp == 64)];
}

const cpx<double>* twiddles64() {
    int dev = 0;
    cudaGetDevice(&dev);
    return g_tw64_addr[dev];
}
const cpx<float>* twiddles32() {
    int dev = 0;
    cudaGetDevice(&dev);
    return g_tw32_addr[dev];
}

static const VecArg kNoVec{nullptr, nullptr, 0, 0};

// batch > 1 (pass timing only): fields dfs (dense input) and ofs (output) elements apart.
template <typename T>
static iim_status rows_fwd(const Plan<T>& p, int row0, int nrows, const double* dense, int dld, int doff,
                           const double* ring, double ih2, const int* row_ptr, const int* aff_node, VecArg gam,
                           double gsign, T* out, const int* stop, cudaStream_t s, int batch = 1, long dfs = 0,
                           long ofs = 0) {
    if (nrows <= 0) return IIM_OK;
    const size_t sm = rows_smem<T>(p.nx);
    auto go = [&](auto kern) -> iim_status {
        IIM_CHECK(allow_smem(kern, sm));
        launch(sizeof(T) == 8 ? "dst_rows_fwd_f64" : "dst_rows_fwd_f32",
               (double)batch * nrows * p.NX * ((dense ? 8.0 : 0.0) + sizeof(T)), (double)batch * nrows * dst_flops(p.nx),
               kern,
               dim3((nrows + rows_per_block(p.nx, p.wide) - 1) / rows_per_block(p.nx, p.wide), batch), kRowWarps * 32,
               sm, s, p.NX, p.NY, p.nx,
               p.lognx, row0, nrows, dense, dld, doff, ring, ih2, row_ptr, aff_node, gam, gsign,
               twiddle_region<T>(p.nx, fft_path(p.nx, p.wide)), out, stop, dfs, ofs);
        return IIM_OK;
    };
    const int fp = fft_path(p.nx, p.wide);
    if (fp == 64) IIM_CHECK(go(k_rows_fwd<T, kRowWarps, 64>));
    else if (fp == 16) IIM_CHECK(go(k_rows_fwd<T, kRowWarps, 16>));
    else if (fp == 8) IIM_CHECK(go(k_rows_fwd<T, kRowWarps, 8>));
    else IIM_CHECK(go(k_rows_fwd<T, kRowWarps, 0>));
    IIM_LAUNCHED();
    return IIM_OK;
}

template <typename T, int C>
static iim_status cols_tile(const Plan<T>& p, int in0, int in1, int out0, int out1, T* buf, const int* stop,
                            cudaStream_t s, int batch, long fstride);

// Tridiagonal column pass (tri.cuh); blockIdx.y selects one of several fields fstride elements
// apart.
template <typename T, int CW, int NT>
__global__ void __launch_bounds__(NT, NT == 1024 ? 2 : 4)
k_cols_scan(int NX, int NY, int ld, int in0, int in1, int out0, int out1, T* __restrict__ buf, ScanTab<T> t,
            const int* __restrict__ stop, long fstride) {
    if (stop && *stop) return;
    cols_scan_body<T, CW, NT>(NX, NY, ld, in0, in1, out0, out1, buf + (long)blockIdx.y * fstride, t);
}

// Launch: one block per 32-byte tile of padded columns (8 FP32 or 4 FP64 columns), batch
// fields on grid y.
template <typename T, int NT>
static iim_status cols_scan_nt(const Plan<T>& p, int in0, int in1, int out0, int out1, T* buf, const int* stop,
                               cudaStream_t s, int batch, long fstride) {
    constexpr int CW = 32 / sizeof(T);
    const size_t sm = scan_smem<T, CW, NT>(p.NY);
    IIM_CHECK(allow_smem(k_cols_scan<T, CW, NT>, sm));
    launch(sizeof(T) == 8 ? "tri_cols_f64" : "tri_cols_f32",
           (double)batch * (in1 - in0 + 1 + out1 - out0 + 1) * p.NX * sizeof(T), (double)batch * p.NX * 14.0 * p.NY,
           k_cols_scan<T, CW, NT>, dim3(p.nx / CW, batch), NT, sm, s, p.NX, p.NY, p.nx, in0, in1, out0, out1, buf,
           p.scan, stop, fstride);
    IIM_LAUNCHED();
    return IIM_OK;
}

template <typename T>
static iim_status cols_scan(const Plan<T>& p, int in0, int in1, int out0, int out1, T* buf, const int* stop,
                            cudaStream_t s, int batch, long fstride) {
    constexpr int CW = 32 / sizeof(T);
    if constexpr (sizeof(T) == 4) {   // FP64 keeps 256 threads (it is bound by FP64 arithmetic)
        if (scan_threads(p.NY, (long)(p.nx / CW) * batch, sm_count()) == 1024)
            return cols_scan_nt<T, 1024>(p, in0, in1, out0, out1, buf, stop, s, batch, fstride);
    }
    return cols_scan_nt<T, 256>(p, in0, in1, out0, out1, buf, stop, s, batch, fstride);
}

// batch > 1: as many fields, fstride elements apart, in one launch
template <typename T>
static iim_status cols(const Plan<T>& p, int in0, int in1, int out0, int out1, T* buf, const int* stop, cudaStream_t s,
                       int batch = 1, long fstride = 0) {
    if (p.scan.lim) return cols_scan(p, in0, in1, out0, out1, buf, stop, s, batch, fstride);
    const int C = tile_width<T>(p.cols_c);
    if (C == 8) return cols_tile<T, (sizeof(T) == 4 ? 8 : 4)>(p, in0, in1, out0, out1, buf, stop, s, batch, fstride);
    if (C == 2) return cols_tile<T, (sizeof(T) == 8 ? 2 : 4)>(p, in0, in1, out0, out1, buf, stop, s, batch, fstride);
    return cols_tile<T, 4>(p, in0, in1, out0, out1, buf, stop, s, batch, fstride);
}

template <typename T, int C>
static iim_status cols_tile(const Plan<T>& p, int in0, int in1, int out0, int out1, T* buf, const int* stop,
                            cudaStream_t s, int batch, long fstride) {
    const size_t sm = cols_smem<T>(p.ny, C);
    auto go = [&](auto kern) -> iim_status {
        IIM_CHECK(allow_smem(kern, sm));
        launch(sizeof(T) == 8 ? "dst_cols_f64" : "dst_cols_f32",
               (double)batch * (in1 - in0 + 1 + out1 - out0 + 1) * p.NX * sizeof(T),
               (double)batch * p.NX * (2.0 * dst_flops(p.ny) + 2.0 * p.NY), kern, dim3(p.nx / C, batch),
               C * line_threads(fft_path(p.ny, p.wide)), sm, s,
               p.NX, p.NY, p.ny, p.logny, in0, in1, out0, out1, buf, p.lam_x, p.lam_y, p.norm,
               twiddle_region<T>(p.ny, fft_path(p.ny, p.wide)), stop, fstride);
        return IIM_OK;
    };
    const int fp = fft_path(p.ny, p.wide);
    if (fp == 64) IIM_CHECK(go(k_cols<T, C, 64>));
    else if (fp == 16) IIM_CHECK(go(k_cols<T, C, 16>));
    else if (fp == 8) IIM_CHECK(go(k_cols<T, C, 8>));
    else IIM_CHECK(go(k_cols<T, C, 0>));
    IIM_LAUNCHED();
    return IIM_OK;
}

template <typename T, int MODE>
static iim_status rows_inv(const Plan<T>& p, int row0, int nrows, const T* in, T* outT, double* out64, int old,
                           int ooff, const uint8_t* cls, const int* stop, cudaStream_t s, int batch = 1,
                           long fstride = 0) {
    if (nrows <= 0) return IIM_OK;
    const size_t sm = rows_smem<T>(p.nx);
    auto go = [&](auto kern) -> iim_status {
        IIM_CHECK(allow_smem(kern, sm));
        launch(sizeof(T) == 8 ? "dst_rows_inv_f64" : "dst_rows_inv_f32",
               (double)batch * nrows * p.NX *
                   (sizeof(T) + (MODE == INV_STORE_T ? sizeof(T) : MODE == INV_STORE_F64 ? 8.0 : 17.0)),
               (double)batch * nrows * dst_flops(p.nx), kern,
               dim3((nrows + rows_per_block(p.nx, p.wide) - 1) / rows_per_block(p.nx, p.wide), batch),
               kRowWarps * 32, sm, s, p.NX, p.NY, p.nx, p.lognx, row0, nrows, in, outT, out64, old, ooff, cls,
               twiddle_region<T>(p.nx, fft_path(p.nx, p.wide)),
               stop, fstride);
        return IIM_OK;
    };
    const int fp = fft_path(p.nx, p.wide);
    if (fp == 64) IIM_CHECK(go(k_rows_inv<T, kRowWarps, MODE, 64>));
    else if (fp == 16) IIM_CHECK(go(k_rows_inv<T, kRowWarps, MODE, 16>));
    else if (fp == 8) IIM_CHECK(go(k_rows_inv<T, kRowWarps, MODE, 8>));
    else IIM_CHECK(go(k_rows_inv<T, kRowWarps, MODE, 0>));
    IIM_LAUNCHED();
    return IIM_OK;
}

template <typename T>
static Plan<T> make_plan(iim_geometry g);
template <>
Plan<double> make_plan<double>(iim_geometry g) {
    Plan<double> p{g->NX, g->NY, g->nx, g->ny, ilog2(g->nx), ilog2(g->ny), g->lam_x64, g->lam_y64,
                   twiddles64(), (2.0 / g->nx) * (2.0 / g->ny), g->cols_c, g->wide_lines};
    if (g->col_solver == 1)
        p.scan = ScanTab<double>{g->sc64_delta, g->sc64_rowoff, nullptr, g->sc64_lim, g->sc64_dstar, g->h * g->h * (2.0 / g->nx)};
    return p;
}
template <>
Plan<float> make_plan<float>(iim_geometry g) {
    Plan<float> p{g->NX, g->NY, g->nx, g->ny, ilog2(g->nx), ilog2(g->ny), g->lam_x32, g->lam_y32,
                  twiddles32(), (float)((2.0 / g->nx) * (2.0 / g->ny)), g->cols_c, g->wide_lines};
    if (g->col_solver == 1)
        p.scan = ScanTab<float>{g->sc32_delta, g->sc32_rowoff, g->sc32_par, g->sc32_lim, g->sc32_dstar,
                                (float)(g->h * g->h * (2.0 / g->nx))};
    return p;
}


// ------------------------------------------------------------------------- IIM operators
// Blocks [0, nga), one warp per affected point (BLOCK / 32 points per block):
// out[a] = (v ? v[a] : 0) + sum_e w_e * (idx >= 0 ? psi[idx] : bc(cp)),
// bc = -xc[body_circ[body]] for circulation bodies (the -B sum psibar 1_k column) when xc is
// given, else 0.  Blocks [nga, nga + ncirc): out[na + c] = sum of v over body c's affected
// points (the circulation rows), when v is given.
template <typename T, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_gather(int na, int nga, const int* __restrict__ ptr, const int* __restrict__ idx, const double* __restrict__ w,
         const T* __restrict__ psi, const int* __restrict__ cp_body, const int* __restrict__ body_circ,
         const int* __restrict__ aff_body, VecArg vin, int use_xc, double* __restrict__ outb, const int* __restrict__ jidx,
         long stride, const int* __restrict__ stop) {
    gather_body<T, BLOCK>(na, nga, ptr, idx, w, psi, cp_body, body_circ, aff_body, vin, use_xc, outb, jidx, stride, stop);
}

// ---- columns of the Schur matrix for the dense preconditioner, many at once
// Forward row transforms of unit vectors: field f holds 1 at affected point j0 + f, so its row
// DST-I is sin(pi k s / n) (s = the point's slot in its padded row) on that row and 0 on the
// other rows of [rmin, rmax].  The sines come from the same twiddle table as the transforms.
template <typename T>
__global__ void k_unit_rows(int nx, int logn, int rmin, int rmax, int j0, int na, const int* __restrict__ aff_node,
                            const cpx<T>* __restrict__ g_tw, T* __restrict__ out, long fstride) {
    const int f = blockIdx.y, a = j0 + f;
    T* o = out + (long)f * fstride;
    int prow = -1, slot = 0;
    if (a < na) {
        const int pn = aff_node[a];
        prow = pn / nx;
        slot = pn - prow * nx;
    }
    const int shift = kTwLog - logn;
    const long total = (long)(rmax - rmin + 1) * nx;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int r = rmin + (int)(e / nx), k = (int)(e % nx);
        T v = T(0);
        if (r == prow && k > 0) {
            const int m = (k * slot) & (2 * nx - 1);   // sin(pi m / n) has period 2n
            const T sn = -g_tw[(m & (nx - 1)) << shift].y;
            v = m >= nx ? -sn : sn;
        }
        o[(long)r * nx + k] = v;
    }
}

// Column j0 + f of S (left half of the row-major augmented array A, leading dimension lda):
// e_j + A (P E_a e_j) on the affected rows, then the circulation rows (sum over body c of e_j).
// blockIdx.y = f; psi holds P E_a e_j of field f (padded, fields fstride apart).
template <typename T, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_gather_unit(int na, int nga, int ncirc, const int* __restrict__ ptr, const int* __restrict__ idx,
              const double* __restrict__ w, const T* __restrict__ psi, long fstride, int j0,
              const int* __restrict__ aff_body, const int* __restrict__ body_circ, float* __restrict__ A, long lda) {
    const int f = blockIdx.y, j = j0 + f;
    if (j >= na) return;
    if ((int)blockIdx.x < nga) {
        const int a = blockIdx.x * BLOCK + threadIdx.x;
        if (a >= na) return;
        const T* ps = psi + (long)f * fstride;
        double acc = (a == j) ? 1.0 : 0.0;
        for (int e = ptr[a]; e < ptr[a + 1]; ++e) {
            const int q = idx[e];
            if (q >= 0) acc += w[e] * (double)ps[q];
        }
        A[(long)a * lda + j] = (float)acc;
    } else {
        const int c = threadIdx.x;
        if (c < ncirc) A[(long)(na + c) * lda + j] = (body_circ[aff_body[j]] == c) ? 1.f : 0.f;
    }
}

// Ghost values at A- nodes from fluid values and psi_b + psibar (Sec. 2.1, 2.2).
__global__ void k_ghost(int nm, const int* __restrict__ minus_node, const int* __restrict__ ptr, const int* __restrict__ idx,
                        const double* __restrict__ w, const double* __restrict__ psi_b, const double* __restrict__ psibar,
                        const int* __restrict__ cp_body, double* __restrict__ psi) {
    ghost_body(nm, minus_node, ptr, idx, w, psi_b, psibar, cp_body, psi);
}

// Un-reduced FP64 residual: r = omega + nabla_h^2 psi_ext at fluid nodes, 0 in the solid and
// in the pads (padded layout); per-block partial sums of r^2.
template <int BLOCK>
__global__ void k_residual(int NX, int NY, double ih2, const double* __restrict__ psi, const double* __restrict__ omega,
                           const uint8_t* __restrict__ cls, const double* __restrict__ ring, double* __restrict__ res,
                           double* __restrict__ partial) {
    residual_body<BLOCK>(NX, NY, ih2, psi, omega, cls, ring, res, partial);
}

// Sum of a padded field over region R_k of each circulation body; grid (ncirc, S).
template <int BLOCK>
__global__ void k_region_sums(int nx, const double* __restrict__ f, const iim_region* __restrict__ R,
                              const int* __restrict__ circ_ids, double* __restrict__ partial) {
    region_sums_body<BLOCK>(nx, f, R, circ_ids, partial);
}

// Discrete circulation -h sum_{dR}(grad_h psi).n (Eq. discretecircconstraint) of each circulation
// body, from the fluid values of psi on the faces of R_k.
template <int BLOCK>
__global__ void k_circ_measure(int nx, const double* __restrict__ psi, const iim_region* __restrict__ R,
                               const int* __restrict__ circ_ids, double* __restrict__ out) {
    circ_measure_body<BLOCK>(nx, psi, R, circ_ids, out);
}


// Combines partial sums into *out_res2 = sum partial + sum rc^2 and, for circulation bodies,
// bcirc[c] = sum_{R_k} r - rc_c with rc_c = (Gamma_k - circ_k) / h^2; max |Gamma_k - circ_k|
// goes to small[SM_CIRC_ERR] when ncirc > 0 or out_res2 is small[SM_RES2].
template <int BLOCK>
__global__ void k_finish_residual(int nparts, const double* __restrict__ partial, int ncirc,
                                  const int* __restrict__ circ_ids, const double* __restrict__ gamma, double ih2,
                                  double* __restrict__ small, const double* __restrict__ regpart,
                                  double* __restrict__ bcirc, double* __restrict__ out_res2) {
    finish_residual_body<BLOCK>(nparts, partial, ncirc, circ_ids, gamma, ih2, small, regpart, bcirc, out_res2);
}

__global__ void k_init_psi(int NX, int NY, const double* __restrict__ guess, const uint8_t* __restrict__ cls,
                           double* __restrict__ psi) {
    init_psi_body(NX, NY, guess, cls, psi);
}

__global__ void k_init_psibar(int nb, const int* __restrict__ body_circ, const double* __restrict__ in, int keep_circ,
                              double* __restrict__ out) {
    init_psibar_body(nb, body_circ, in, keep_circ, out);
}

__global__ void k_add_psibar(int ncirc, const int* __restrict__ circ_ids, const double* __restrict__ x, double* __restrict__ psibar) {
    add_psibar_body(ncirc, circ_ids, x, psibar);
}

// psi_ext += sum_l coef[l] resp_l (padded fields, npad values each): the capacitance correction.
__global__ void k_cap_update(long npad, int ncirc, const double* __restrict__ resp, const double* __restrict__ coef,
                             double* __restrict__ psi) {
    cap_update_body(npad, ncirc, resp, coef, psi);
}

// Velocity u = (d_y psi, -d_x psi) by centered differences of psi_ext at fluid nodes (Sec. 4.2,
// end); psi_out = psi at fluid nodes, 0 in the solid.  Outputs in the caller's layout.
__global__ void k_velocity(int NX, int NY, double inv2h, const double* __restrict__ psi, const uint8_t* __restrict__ cls,
                           const double* __restrict__ ring, double* __restrict__ psi_out, double* __restrict__ ux,
                           double* __restrict__ uy) {
    velocity_body(NX, NY, inv2h, psi, cls, ring, psi_out, ux, uy);
}

// ------------------------------------------------------------------------- GMRES kernels

// h[i] = <V_i, V_{j+1}> for i <= j (one block per i)
template <int BLOCK>
__global__ void k_dots(const int* __restrict__ di, const double* __restrict__ V, long ld, int ns, double* __restrict__ out) {
    if (di[DI_STOP]) return;
    const int j = di[DI_J];
    const int i = blockIdx.x;
    if (i > j) return;
    const double* vi = V + (long)i * ld;
    const double* w = V + (long)(j + 1) * ld;
    double acc = 0.0;
    for (int e = threadIdx.x; e < ns; e += BLOCK) acc += vi[e] * w[e];
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) out[i] = acc;
}

// V_{j+1} -= sum_{i<=j} coef[i] V_i; with `partial`, per-block sums of squares of the result.
template <int BLOCK>
__global__ void k_update(const int* __restrict__ di, double* __restrict__ V, long ld, const double* __restrict__ coef,
                         int ns, double* __restrict__ partial) {
    if (di[DI_STOP]) return;
    const int j = di[DI_J];
    const int e = blockIdx.x * BLOCK + threadIdx.x;
    double* w = V + (long)(j + 1) * ld;
    double val = 0.0;
    if (e < ns) {
        double s = 0.0;
        for (int i = 0; i <= j; ++i) s += coef[i] * V[(long)i * ld + e];
        val = w[e] - s;
        w[e] = val;
    }
    if (partial) {
        const double sq = block_sum<BLOCK>(val * val);
        if (threadIdx.x == 0) partial[blockIdx.x] = sq;
    }
}

template <int BLOCK>
__global__ void k_sumsq(const double* __restrict__ w, int ns, double* __restrict__ partial) {
    double acc = 0.0;
    for (int e = blockIdx.x * BLOCK + threadIdx.x; e < ns; e += gridDim.x * BLOCK) acc += w[e] * w[e];
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}


// Arnoldi step finish after k_update: sums the per-block squares, then arnoldi_finish.
__global__ void k_arnoldi_tail(int* __restrict__ di, KLayout L, int nparts, const double* __restrict__ partial,
                               double* __restrict__ K) {
    if (di[DI_STOP]) return;
    const int lane = threadIdx.x;
    double s = 0.0;
    for (int b = lane; b < nparts; b += 32) s += partial[b];
    s = warp_sum(s);
    if (lane == 0) arnoldi_finish(di, L, K, s);
}

// The whole Arnoldi step in one block, for short Krylov bases (the preconditioned iteration
// converges in a few steps): two classical Gram-Schmidt passes against V_0..V_j, the norm,
// arnoldi_finish, and the scaling of V_{j+1} -- one launch instead of six.  Each thread owns
// the same elements in every pass; the j+1 inner products of a pass are reduced together
// (warp sums into part[i][warp], then one thread per i), so a pass synchronises twice.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_arnoldi_block(int* __restrict__ di, double* __restrict__ V, long ld, int ns, KLayout L, double* __restrict__ K) {
    arnoldi_block_body<BLOCK>(di, V, ld, ns, L, K);
}

// V_j *= 1 / ||V_j|| (j already advanced by the tail)
__global__ void k_scale(const int* __restrict__ di, double* __restrict__ V, long ld, int ns, const double* __restrict__ sc) {
    if (di[DI_STOP]) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ns) V[(long)di[DI_J] * ld + e] *= *sc;
}

// V_0 = r / ||r||, g = (beta, 0, ...), j = 0, stop unless there is work left
__global__ void k_start_cycle(int ns, const double* __restrict__ r, double* __restrict__ v0, KLayout L, double* __restrict__ K,
                              int nparts, const double* __restrict__ partial, int* __restrict__ di) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += partial[b];
    const double beta = sqrt(s);
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ns) v0[e] = r[e] * inv;
    if (e == 0) {
        double* gv = K + L.gv();
        gv[0] = beta;
        for (int i = 1; i <= L.m; ++i) gv[i] = 0.0;
        K[L.scal() + SC_BETA] = beta;
        K[L.scal() + SC_RESID] = beta;
        di[DI_J] = 0;
        di[DI_STOP] = (di[DI_IT] >= di[DI_MAXIT]) ? 1 : 0;
        if (!(beta > K[L.scal() + SC_TOL])) { di[DI_CONV] = 1; di[DI_STOP] = 1; }
    }
}

// One block: beta = ||r||, V_0 = r / beta and the GMRES start state (k_start_cycle's work,
// with the norm reduced inside the block instead of by k_sumsq's blocks).  With init_maxit >= 0
// it first does what the norm / k_gmres_init launches do at the start of a correction: *norm2 =
// ||r||^2, the counters reset, the tolerance set to tol * ||r||.  Five launches become one.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_start_block(int ns, const double* __restrict__ r, double* __restrict__ v0, KLayout L, double* __restrict__ K,
              int* __restrict__ di, int init_maxit, double tol, double* __restrict__ norm2) {
    start_block_body<BLOCK>(ns, r, v0, L, K, di, init_maxit, tol, norm2);
}

// y = H^{-1} g over the first k = j columns (one warp)
__global__ void k_backsolve(const int* __restrict__ di, KLayout L, double* __restrict__ K) {
    const int lane = threadIdx.x;
    const int k = di[DI_J];
    const double* H = K + L.H();
    const int ldh = L.m + 1;
    const double* gv = K + L.gv();
    double* y = K + L.y();
    for (int i = k - 1; i >= 0; --i) {
        double s = 0.0;
        for (int l = i + 1 + lane; l < k; l += 32) s += H[(long)l * ldh + i] * y[l];
        s = warp_sum(s);
        if (lane == 0) {
            const double d = H[(long)i * ldh + i];
            y[i] = d != 0.0 ? (gv[i] - s) / d : 0.0;
        }
        __syncwarp();
    }
}

// k_backsolve and the update in one block: warp 0 solves for y, then out = V y (accumulate 0)
// or out += V y (accumulate 1) over the block -- the same operations in the same order as
// k_backsolve followed by k_xupdate on a zeroed or the given out.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_backsolve_update(const int* __restrict__ di, KLayout L, double* __restrict__ K, const double* __restrict__ V,
                   long ld, int ns, double* __restrict__ out, int accumulate) {
    backsolve_update_body<BLOCK>(di, L, K, V, ld, ns, out, accumulate);
}

__global__ void k_xupdate(const int* __restrict__ di, const double* __restrict__ V, long ld, const double* __restrict__ y,
                          int ns, double* __restrict__ x) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ns) return;
    const int k = di[DI_J];
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += y[i] * V[(long)i * ld + e];
    x[e] += s;
}

__global__ void k_axpby(int n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = a * x[e] + b * y[e];
}

__global__ void k_set_int(int* __restrict__ p, int v) { *p = v; }

__global__ void k_negate(int n, double* __restrict__ v) {
    const int i = threadIdx.x;
    if (i < n) v[i] = -v[i];
}

// Scales a Krylov seed to its best multiple: c = <b, S x0> / <S x0, S x0> minimises
// ||b - c S x0||, which is then at most ||b||.  x0 and S x0 are scaled in place; out = c.
// One block.
template <int BLOCK>
__global__ void k_seed_scale(int ns, const double* __restrict__ b, double* __restrict__ sx, double* __restrict__ x,
                             double* __restrict__ out) {
    __shared__ double c_sh;
    double d = 0.0, q = 0.0;
    for (int e = threadIdx.x; e < ns; e += BLOCK) {
        d += b[e] * sx[e];
        q += sx[e] * sx[e];
    }
    d = block_sum<BLOCK>(d);
    q = block_sum<BLOCK>(q);
    if (threadIdx.x == 0) {
        c_sh = q > 0.0 ? d / q : 0.0;
        *out = c_sh;
    }
    __syncthreads();
    const double c = c_sh;
    for (int e = threadIdx.x; e < ns; e += BLOCK) {
        sx[e] *= c;
        x[e] *= c;
    }
}

// out[c] = sgn * mean over the control points of circulation body c of (psi extrapolated to the
// crossing - psi_b): the quadratic through the fluid node and the next two fluid nodes on the
// line, evaluated at the crossing (the fluid value alone when the run is shorter); one block
// per body.  psi padded.
template <int BLOCK>
__global__ void k_psibar_estimate(int ncp, int nx, int ny, const int* __restrict__ axis, const int* __restrict__ ei,
                                  const int* __restrict__ ej, const double* __restrict__ cp_t,
                                  const int* __restrict__ cp_body, const int* __restrict__ body_circ,
                                  const uint8_t* __restrict__ cls, const double* __restrict__ psi,
                                  const double* __restrict__ psi_b, double* __restrict__ out, double sgn) {
    const int c = blockIdx.x;
    double s = 0.0, cnt = 0.0;
    for (int k = threadIdx.x; k < ncp; k += BLOCK) {
        if (body_circ[cp_body[k]] != c) continue;
        const int i0 = ei[k], j0 = ej[k];
        const bool ax = axis[k] == 0;
        const int i1 = ax ? i0 + 1 : i0, j1 = ax ? j0 : j0 + 1;
        const long p0 = (long)(j0 - 1) * nx + i0, p1 = (long)(j1 - 1) * nx + i1;   // padded indices
        const bool lower_fluid = cls[p0] <= CLS_PLUS;
        const long pf = lower_fluid ? p0 : p1;
        const long step = (lower_fluid ? -1 : 1) * (ax ? 1L : (long)nx);   // from the solid node into the fluid
        const int fi = lower_fluid ? i0 : i1, fj = lower_fluid ? j0 : j1;
        const int di = ax ? (lower_fluid ? -1 : 1) : 0, dj = ax ? 0 : (lower_fluid ? -1 : 1);
        const int i2 = fi + 2 * di, j2 = fj + 2 * dj;
        double val = psi[pf];
        if (i2 >= 1 && i2 <= nx - 1 && j2 >= 1 && j2 <= ny - 1 && cls[pf + step] <= CLS_PLUS && cls[pf + 2 * step] <= CLS_PLUS) {
            const double t = -cp_t[k];   // the crossing sits at -t along the line (nodes at 0, 1, 2)
            val = psi[pf] * (t - 1.0) * (t - 2.0) * 0.5 - psi[pf + step] * t * (t - 2.0) +
                  psi[pf + 2 * step] * t * (t - 1.0) * 0.5;
        }
        s += val - (psi_b ? psi_b[k] : 0.0);
        cnt += 1.0;
    }
    s = block_sum<BLOCK>(s);
    cnt = block_sum<BLOCK>(cnt);
    if (threadIdx.x == 0) out[c] = cnt > 0.0 ? sgn * s / cnt : 0.0;
}

__global__ void k_gmres_init(int* __restrict__ di, int maxit, double* __restrict__ K, KLayout L, const double* __restrict__ b2,
                             double tol) {
    di[DI_J] = 0;
    di[DI_STOP] = 0;
    di[DI_IT] = 0;
    di[DI_MAXIT] = maxit;
    di[DI_CONV] = 0;
    di[DI_TMPJ] = 0;
    di[DI_LOOP] = 0;
    di[DI_LOOPERR] = 0;
    K[L.scal() + SC_TOL] = tol * sqrt(*b2);
}

// ------------------------------------------------------------------------- solver
// End of the body of the device-side GMRES loop (a WHILE conditional graph node): counts the
// body's executions and ends the loop once the iteration kernels have set the stop flag.  The
// cap (restart length + 2, never reached while the kernels follow their stopping rule) makes
// the loop finite in any case; hitting it sets the stop flag and an error flag for the host.
__global__ void k_loop_ctl(cudaGraphConditionalHandle h, int* __restrict__ di, int cap) {
    const int c = ++di[DI_LOOP];
    if (!di[DI_STOP] && c >= cap) {
        di[DI_STOP] = 1;
        di[DI_LOOPERR] = 1;
    }
    if (di[DI_STOP]) cudaGraphSetConditional(h, 0);
}

// ---- control kernels of the whole solve run as one graph (nested WHILE / IF nodes)
// Before the refinement loop: ||f|| from the residual at psi = 0, counters reset, loop entered
// unless there is nothing to solve.
__global__ void k_ref_init(cudaGraphConditionalHandle h, int* __restrict__ di, double* __restrict__ small, double rtol) {
    const double r2 = small[SM_RES2];
    const double fn = sqrt(r2);
    small[SM_FNORM] = fn;
    small[SM_REL] = fn > 0.0 ? 1.0 : 0.0;
    di[DI_REF] = 0; di[DI_ITS] = 0; di[DI_FIRST] = 0; di[DI_CYCERR] = 0; di[DI_CYCS] = 0; di[DI_RSS] = 0;
    di[DI_LOOPERR] = 0;
    const bool fin = isfinite(r2);
    di[DI_NONFIN] = fin ? 0 : 1;
    cudaGraphSetConditional(h, (fin && fn > 0.0 && 1.0 > rtol) ? 1 : 0);
}

// After gmres_init: the Krylov budget left for this correction; cycle counter reset; the cycle
// loop entered unless the start already stopped (converged or no budget).
__global__ void k_cyc_begin(cudaGraphConditionalHandle h, int* __restrict__ di, int max_iter) {
    const int left = max_iter - di[DI_ITS];
    di[DI_MAXIT] = left > 1 ? left : 1;
    di[DI_CYC] = 0;
    if (di[DI_IT] >= di[DI_MAXIT]) di[DI_STOP] = 1;
    cudaGraphSetConditional(h, di[DI_STOP] ? 0 : 1);
}

// Start of a cycle: the iteration loop is entered unless the stop flag is set.
__global__ void k_it_begin(cudaGraphConditionalHandle h, int* __restrict__ di) {
    di[DI_LOOP] = 0;
    cudaGraphSetConditional(h, di[DI_STOP] ? 0 : 1);
}

// End of a cycle (after the solution update): another cycle, with the restart residual, unless
// converged, out of budget, or capped (cap: max_iter / restart + 2 cycles; reaching it without
// one of the others sets an error flag).
__global__ void k_cyc_ctl(cudaGraphConditionalHandle hc, cudaGraphConditionalHandle hr, int* __restrict__ di, int cap) {
    const int c = ++di[DI_CYC];
    ++di[DI_CYCS];
    bool done = di[DI_CONV] || di[DI_IT] >= di[DI_MAXIT] || di[DI_LOOPERR];
    if (!done && c >= cap) {
        done = true;
        di[DI_CYCERR] = 1;
    }
    if (!done) ++di[DI_RSS];
    cudaGraphSetConditional(hc, done ? 0 : 1);
    cudaGraphSetConditional(hr, done ? 0 : 1);
}

// End of a refinement: counters, the relative FP64 residual, and whether to go on (at most
// max_refine corrections and max_iter Krylov iterations).
__global__ void k_ref_ctl(cudaGraphConditionalHandle h, int* __restrict__ di, double* __restrict__ small, double rtol,
                          int max_refine, int max_iter) {
    if (di[DI_REF] == 0) di[DI_FIRST] = di[DI_IT];
    di[DI_ITS] += di[DI_IT];
    const int r = ++di[DI_REF];
    const double r2 = small[SM_RES2], fn = small[SM_FNORM];
    const bool fin = isfinite(r2);
    if (!fin) di[DI_NONFIN] = 1;
    const double rel = fn > 0.0 ? sqrt(r2) / fn : 0.0;
    small[SM_REL] = rel;
    const bool go = fin && rel > rtol && r < max_refine && di[DI_ITS] < max_iter && !di[DI_LOOPERR] && !di[DI_CYCERR];
    cudaGraphSetConditional(h, go ? 1 : 0);
}

// Capacitance coefficients on the device: coef = C^-1 (h^2 rc), dpb = coef . Pb (one block).
__global__ void k_cap_coef(int nc, const double* __restrict__ rc, const double* __restrict__ cinv,
                           const double* __restrict__ pb, double h2, double* __restrict__ coef, double* __restrict__ dpb) {
    cap_coef_body(nc, rc, cinv, pb, h2, coef, dpb);
}

__global__ void k_final_rel(int* __restrict__ di, double* __restrict__ small) {
    final_rel_body(di, small);
}

// One GMRES cycle as a graph: a WHILE node whose body is one iteration (the captured kernel
// sequence) plus k_loop_ctl; `nodes` = kernels per body execution.
struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    int prec = -1, m = 0, pc = 0;
    cudaStream_t stream = nullptr;
    int nodes = 0;
};

// The whole solve as one executable graph: the initial residual, a WHILE node over the
// refinements whose body holds the right-hand side, the GMRES start, a WHILE node over restart
// cycles (its body: a WHILE node over iterations, the solution update, an IF node with the
// restart residual), the recovery and the residual; then the capacitance correction and the
// velocity.  Control kernels decide every loop on the device (caps on every loop); the host
// launches the graph once and reads the counters.  Valid for the exact arguments it was built
// with (the key) and the geometry's tile settings.
struct SolveGraph {
    cudaGraphExec_t exec = nullptr;
    // key
    int prec = -1, m = 0, pc = 0, max_refine = 0, max_iter = 0, cap = 0;
    double inner = 0.0, rtol = 0.0;
    const void* ptrs[9] = {};   // caller arrays and the Krylov basis
    // kernel nodes per execution of each level (launch accounting)
    long long k_top = 0, k_ref = 0, k_cyc = 0, k_it = 0, k_rs = 0;
};

struct Solver {
    iim_geometry g;
    cudaStream_t s;
    int prec;
    const double* omega;
    const double* psi_b;
    const double* ring;
    const double* gamma;
    double* psibar;   // device, n_bodies
    int ns;
    int m;
    KLayout L;
    int iters = 0;
    double last_gmres_rel = 0.0;
    bool use_graph = true;
    bool precond = false;
    static constexpr int kResBlocks = 1024;
    static constexpr int kNormBlocks = 64;

    int* di() const { return g->d_int; }

    // ---- residual of the un-reduced system; fills g->res, small[], bvec circulation rows
    iim_status residual(double* res2_out, double* circ_err_out) {
        IIM_CHECK(residual_launch());
        IIM_TRY(cudaMemcpyAsync(g->h_pinned, g->small, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        IIM_TRY(cudaStreamSynchronize(s));
        *res2_out = g->h_pinned[SM_RES2];
        *circ_err_out = g->h_pinned[SM_CIRC_ERR];
        return IIM_OK;
    }

    // the kernels of residual(): ghosts, residual and partial norms, circulation measure,
    // region sums, small[SM_RES2], small[SM_CIRC_ERR], small[SM_RC..], circulation rows of bvec
    iim_status residual_launch() {
        const double ih2 = 1.0 / (g->h * g->h);
        if (g->nminus > 0) {
            launch("ghost_f64", 0.0, 0.0, k_ghost, (g->nminus + 255) / 256, 256, 0, s, g->nminus, g->minus_node, g->gh_ptr,
                   g->gh_idx, g->gh_w, psi_b, psibar, g->cp_body, g->psi_ext);
            IIM_LAUNCHED();
        }
        launch("residual_f64", 25.0 * (double)g->NX * g->NY, 8.0 * (double)g->NX * g->NY, k_residual<256>, kResBlocks,
               256, 0, s, g->NX, g->NY, ih2, g->psi_ext, omega, g->node_class, ring_now(), g->res, g->partial);
        IIM_LAUNCHED();
        double* small = g->small;
        const int* circ_ids_d = g->d_int + DI_CIRC;
        if (g->ncirc > 0) {
            launch("circ_measure", 0.0, 0.0, k_circ_measure<256>, g->ncirc, 256, 0, s, g->nx, g->psi_ext, g->d_regions,
                   circ_ids_d, small + SM_CIRC);
            launch("region_sums", 0.0, 0.0, k_region_sums<256>, dim3(g->ncirc, kRegionParts), 256, 0, s, g->nx, g->res,
                   g->d_regions, circ_ids_d, small + SM_REG);
            IIM_LAUNCHED();
        }
        launch("finish_residual", 0.0, 0.0, k_finish_residual<256>, 1, 256, 0, s, kResBlocks, g->partial, g->ncirc,
               circ_ids_d, gamma, ih2, small, small + SM_REG, g->bvec ? g->bvec + g->na : nullptr, small + SM_RES2);
        IIM_LAUNCHED();
        if (g->outer)   // free space: the ring rows (freespace.cu), kept for the next recovery
            IIM_CHECK(launch_ring_residual(g->nx, g->ny, g->h, g->lgf, g->lgf_ld, g->outer == 2,
                                           g->outer == 2 && !g->plane_off ? g->fs_plane : nullptr, g->psi_ext,
                                           g->fs_ring, g->fs_rres, small + SM_RES2, s));
        return IIM_OK;
    }

    // ---- Schur operator application V_{jd+1} = S_aug V_jd, jd = di[jslot] (device)
    template <typename T>
    iim_status apply_at(int jslot, const int* stop) {
        return apply_vec<T>(VecArg{g->V, di() + jslot, 0, (long)ns}, di() + jslot, stop);
    }

    // ---- V_{*out_j + 1} = S_aug vin
    template <typename T>
    iim_status apply_vec(VecArg vj, const int* out_j, const int* stop) {
        Plan<T> p = make_plan<T>(g);
        T* tb = (T*)g->tbuf;
        T* pt = (T*)g->psiT;
        const long ld = ns;
        if (g->na > 0 && !g->outer) {
            IIM_CHECK(rows_fwd<T>(p, g->ja0, g->ja1 - g->ja0 + 1, nullptr, 0, 0, nullptr, 0.0, g->aff_row_ptr,
                                  g->aff_node, vj, 1.0, tb, stop, s));
            IIM_CHECK(cols<T>(p, g->ja0, g->ja1, g->jo0, g->jo1, tb, stop, s));
            IIM_CHECK((rows_inv<T, INV_STORE_T>(p, g->jo0, g->jo1 - g->jo0 + 1, tb, pt, nullptr, 0, 0, nullptr, stop, s)));
        } else if (g->na > 0) {
            // free space: psi_1 with every row of the column pass kept for the boundary values,
            // then the harmonic part with the ring data rho
            IIM_CHECK(rows_fwd<T>(p, g->ja0, g->ja1 - g->ja0 + 1, nullptr, 0, 0, nullptr, 0.0, g->aff_row_ptr,
                                  g->aff_node, vj, 1.0, tb, stop, s));
            IIM_CHECK(cols<T>(p, g->ja0, g->ja1, 0, g->NY - 1, tb, stop, s));
            IIM_CHECK(free_ring<T>(p, stop));
            IIM_CHECK((rows_inv<T, INV_STORE_T>(p, g->jo0, g->jo1 - g->jo0 + 1, tb, pt, nullptr, 0, 0, nullptr, stop, s)));
            IIM_CHECK(free_harmonic<T>(p, g->jo0, g->jo1, stop));
            IIM_CHECK((rows_inv<T, INV_ACCUM_T>(p, g->jo0, g->jo1 - g->jo0 + 1, tb, pt, nullptr, 0, 0, nullptr, stop, s)));
        }
        const int nga = (g->na + 3) / 4;   // gather blocks: 4 warps, one affected point each
        launch("gather", 0.0, 0.0, k_gather<T, 128>, nga + g->ncirc, 128, 0, s, g->na, nga, g->gop_ptr, g->gop_idx,
               g->gop_w, pt, g->cp_body, g->body_circ, g->aff_body, vj, 1, g->V, out_j, ld, stop);
        IIM_LAUNCHED();
        return IIM_OK;
    }

    // ---- free space (freespace.cu): with tbuf holding the column-processed transform of the
    // first box solve psi_1 on every row, its values next to the box (two dot products per row
    // for the first and last interior columns, the inverse transform of the first and last
    // interior rows) and the ring sum rho = sum_y G(x - y) psi_1(neighbour of y) into fs_rho
    template <typename T>
    iim_status free_ring(const Plan<T>& p, const int* stop) {
        const int NX = g->NX, NY = g->NY;
        double* bnd = g->fs_bnd;
        IIM_CHECK(launch_bnd_cols<T>(NX, NY, g->nx, (const T*)g->tbuf, bnd + 2 * NX, bnd + 2 * NX + NY, stop, s));
        IIM_CHECK((rows_inv<T, INV_STORE_F64>(p, 0, 1, (const T*)g->tbuf, nullptr, bnd, 0, 0, nullptr, stop, s)));
        IIM_CHECK((rows_inv<T, INV_STORE_F64>(p, NY - 1, 1, (const T*)g->tbuf, nullptr, bnd, 0, NX, nullptr, stop, s)));
        return launch_ring_conv(g->nx, g->ny, g->lgf, g->lgf_ld, g->outer == 2, bnd, bnd + 2 * NX, bnd + 2 * NX + NY,
                                g->fs_rho, stop, s);
    }

    // ---- free space: the box solve of a zero source with box data fs_rho (the harmonic part),
    // column pass written back on rows [out0, out1] of tbuf
    template <typename T>
    iim_status free_harmonic(const Plan<T>& p, int out0, int out1, const int* stop) {
        const double ih2 = 1.0 / (g->h * g->h);
        IIM_CHECK(rows_fwd<T>(p, 0, g->NY, nullptr, 0, 0, g->fs_rho, ih2, nullptr, nullptr, kNoVec, 0.0, (T*)g->tbuf,
                              stop, s));
        return cols<T>(p, 0, g->NY - 1, out0, out1, (T*)g->tbuf, stop, s);
    }

    // ring values the residual and the velocity use: the box data, or in free space the ring of
    // the current solution
    const double* ring_now() const { return g->outer ? g->fs_ring : ring; }

    // ---- dense Schur-complement preconditioner: columns S e_j from FP32 operator applications,
    // then [S | I] -> [I | S^-1] by blocked Gauss-Jordan with partial pivoting (FP32)
    iim_status build_precond() {
        if (g->pc_ready) return IIM_OK;
        const int n = ns;
        const long ld = ns;
        if (!g->pc_aug) {
            IIM_TRY(cudaMalloc(&g->pc_aug, sizeof(float) * 2 * (size_t)n * n));
            IIM_TRY(cudaMalloc(&g->pc_f, sizeof(float) * gj_scratch_floats(n)));
            IIM_TRY(cudaMalloc(&g->pc_info, sizeof(int)));
            IIM_TRY(cudaMalloc(&g->pc_z, sizeof(double) * 2 * (size_t)n));
        }
        IIM_TRY(cudaEventRecord(g->ev0, s));
        // gamma columns j < |A|, K at a time: unit row transforms, column pass, inverse rows of
        // the gathered band, gather straight into the matrix (one launch each per batch); in free
        // space every column takes one operator application (below)
        if (!g->outer) {
            const long fstride = (long)g->nx * g->NY;
            const size_t fbytes = sizeof(float) * (size_t)fstride;
            const int K = (int)std::max<size_t>(1, std::min<size_t>(32, (size_t(256) << 20) / (2 * fbytes)));
            float* tb = nullptr;
            IIM_TRY(cudaMalloc(&tb, 2 * fbytes * (size_t)K));
            float* pt = tb + (size_t)K * fstride;
            std::vector<int> row_of(g->na);
            IIM_TRY(cudaMemcpyAsync(row_of.data(), g->aff_node, sizeof(int) * (size_t)g->na, cudaMemcpyDeviceToHost, s));
            IIM_TRY(cudaStreamSynchronize(s));
            Plan<float> p = make_plan<float>(g);
            const int nga = (g->na + 127) / 128;   // k_gather_unit: one thread per affected point
            iim_status bs = IIM_OK;
            for (int j0 = 0; j0 < g->na && bs == IIM_OK; j0 += K) {
                const int kb = std::min(K, g->na - j0);
                const int rmin = row_of[j0] / g->nx, rmax = row_of[j0 + kb - 1] / g->nx;   // row-major order
                const long cells = (long)(rmax - rmin + 1) * g->nx;
                launch("pc_unit_rows", 0.0, 0.0, k_unit_rows<float>, dim3((unsigned)std::min<long>((cells + 255) / 256, 64), kb),
                       256, 0, s, g->nx, ilog2(g->nx), rmin, rmax, j0, g->na, (const int*)g->aff_node, p.tw, tb, fstride);
                bs = cols<float>(p, rmin, rmax, g->jo0, g->jo1, tb, nullptr, s, kb, fstride);
                if (bs == IIM_OK)
                    bs = rows_inv<float, INV_STORE_T>(p, g->jo0, g->jo1 - g->jo0 + 1, tb, pt, nullptr, 0, 0, nullptr,
                                                      nullptr, s, kb, fstride);
                if (bs == IIM_OK)
                    launch("pc_gather", 0.0, 0.0, k_gather_unit<float, 128>, dim3(nga + 1, kb), 128, 0, s, g->na, nga,
                           g->ncirc, (const int*)g->gop_ptr, (const int*)g->gop_idx, (const double*)g->gop_w,
                           (const float*)pt, fstride, j0, (const int*)g->aff_body, (const int*)g->body_circ, g->pc_aug,
                           2L * n);
                if (bs == IIM_OK && cudaGetLastError() != cudaSuccess) bs = IIM_ERR_CUDA;
            }
            cudaError_t se = cudaStreamSynchronize(s);
            cudaFree(tb);
            if (bs != IIM_OK) return bs;
            IIM_TRY(se);
        }
        // psibar columns (and in free space all columns): one operator application each
        launch("set_tmpj", 0.0, 0.0, k_set_int, 1, 1, 0, s, di() + DI_TMPJ, 0);
        const int eb = (n + 255) / 256;
        for (int j = g->outer ? 0 : g->na; j < n; ++j) {
            launch("pc_unit", 0.0, 0.0, k_unit_vector, eb, 256, 0, s, n, j, g->V);
            IIM_CHECK(apply_at<float>(DI_TMPJ, nullptr));
            launch("pc_column", 0.0, 0.0, k_store_column, eb, 256, 0, s, n, j, (const double*)(g->V + ld), g->pc_aug);
            IIM_LAUNCHED();
        }
        // keep S (the left half) for the dense inner operator before it is reduced to I
        if (!g->pc_S) IIM_TRY(cudaMalloc(&g->pc_S, sizeof(float) * (size_t)n * n));
        IIM_TRY(cudaMemcpy2DAsync(g->pc_S, sizeof(float) * (size_t)n, g->pc_aug, sizeof(float) * 2 * (size_t)n,
                                  sizeof(float) * (size_t)n, (size_t)n, cudaMemcpyDeviceToDevice, s));
        IIM_CHECK(gj_invert_aug(g->pc_aug, n, g->pc_f, g->pc_info, s));
        int info = 0;
        IIM_TRY(cudaMemcpyAsync(&info, g->pc_info, sizeof(int), cudaMemcpyDeviceToHost, s));
        IIM_TRY(cudaEventRecord(g->ev1, s));
        IIM_TRY(cudaStreamSynchronize(s));
        if (info != 0) {
            snprintf(g_last_error, sizeof(g_last_error), "Schur matrix singular at pivot %d", info);
            return IIM_ERR_NOT_CONVERGED;
        }
        cudaEventElapsedTime(&g->pc_setup_ms, g->ev0, g->ev1);
        g->pc_ready = 1;
        // the captured iteration graphs may predate the preconditioner buffers
        for (void** gp : {&g->graph64, &g->graph32}) {
            IterGraph* G = (IterGraph*)*gp;
            if (G && G->exec) { cudaGraphExecDestroy(G->exec); G->exec = nullptr; }
        }
        return IIM_OK;
    }

    // ---- one Arnoldi step after the operator application
    iim_status ortho_iter() {
        const long ld = ns;
        double* K = g->H;
        if (precond) {
            launch("gmres_arnoldi", 0.0, 0.0, k_arnoldi_block<256>, 1, 256, 0, s, di(), g->V, ld, ns, L, K);
            IIM_LAUNCHED();
            return IIM_OK;
        }
        const int eb = (ns + 255) / 256;
        launch("gmres_dots", 0.0, 0.0, k_dots<256>, m, 256, 0, s, di(), g->V, ld, ns, K + L.hc1());
        launch("gmres_update", 0.0, 0.0, k_update<256>, eb, 256, 0, s, di(), g->V, ld, K + L.hc1(), ns, nullptr);
        launch("gmres_dots", 0.0, 0.0, k_dots<256>, m, 256, 0, s, di(), g->V, ld, ns, K + L.hc2());
        launch("gmres_update", 0.0, 0.0, k_update<256>, eb, 256, 0, s, di(), g->V, ld, K + L.hc2(), ns, g->partial);
        launch("gmres_tail", 0.0, 0.0, k_arnoldi_tail, 1, 32, 0, s, di(), L, eb, g->partial, K);
        launch("gmres_scale", 0.0, 0.0, k_scale, eb, 256, 0, s, di(), g->V, ld, ns, K + L.scal() + SC_INV);
        IIM_LAUNCHED();
        return IIM_OK;
    }

    template <typename T>
    iim_status iteration() {
        if (precond) {
            // right preconditioning: z = M v_j, v_{j+1} = S z
            IIM_CHECK(dense_matvec(ns, g->pc_aug + ns, 2L * ns, g->V, di() + DI_J, (long)ns, g->pc_z, 0, di() + DI_STOP, s));
            if (dense_op)
                IIM_CHECK(dense_matvec_to(ns, g->pc_S, (long)ns, g->pc_z, g->V, di() + DI_J, (long)ns, di() + DI_STOP, s));
            else
                IIM_CHECK(apply_vec<T>(VecArg{g->pc_z, nullptr, 0, 0}, di() + DI_J, di() + DI_STOP));
        } else {
            IIM_CHECK(apply_at<T>(DI_J, di() + DI_STOP));
        }
        return ortho_iter();
    }

    template <typename T>
    iim_status ensure_graph(IterGraph& G) {
        if (G.exec && G.prec == (int)sizeof(T) && G.m == m && G.pc == pc_mode()) return IIM_OK;
        if (G.exec) { cudaGraphExecDestroy(G.exec); G.exec = nullptr; }
        // capture on the geometry's private stream (the caller's may be the legacy stream,
        // which cannot be captured); the graph is then launched on the caller's stream
        cudaGraph_t graph = nullptr;
        const cudaStream_t user = s;
        IIM_TRY(cudaStreamSynchronize(user));
        IIM_TRY(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle h;
        cudaGraphNodeParams cp = {};
        cudaGraphNode_t cn = nullptr;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            e = cudaGraphAddNode(&cn, graph, nullptr, nullptr, 0, &cp);
        }
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            record_cuda_error(e, "conditional graph node", __FILE__, __LINE__);
            return IIM_ERR_CUDA;
        }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        s = g->cap_stream;
        set_capture(true);
        e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            set_capture(false);
            s = user;
            cudaGraphDestroy(graph);
            record_cuda_error(e, "cudaStreamBeginCaptureToGraph", __FILE__, __LINE__);
            return IIM_ERR_CUDA;
        }
        iim_status st = iteration<T>();
        launch("gmres_loop_ctl", 0.0, 0.0, k_loop_ctl, 1, 1, 0, s, h, di(), m + 2);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(s, &captured);
        set_capture(false);
        s = user;
        if (st != IIM_OK || e != cudaSuccess) {
            cudaGraphDestroy(graph);
            if (st != IIM_OK) return st;
            record_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
            return IIM_ERR_CUDA;
        }
        size_t nn = 0;
        cudaGraphGetNodes(body, nullptr, &nn);
        e = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { G.exec = nullptr; record_cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__); return IIM_ERR_CUDA; }
        G.prec = (int)sizeof(T);
        G.m = m;
        G.pc = pc_mode();
        G.stream = s;
        G.nodes = (int)nn;
        return IIM_OK;
    }

    // ---- right-hand side b = [A P r ; sum_R r - rc] (circulation part filled by residual())
    template <typename T>
    iim_status rhs() {
        Plan<T> p = make_plan<T>(g);
        T* tb = (T*)g->tbuf;
        T* pt = (T*)g->psiT;
        if (g->na == 0) return IIM_OK;
        IIM_CHECK(rows_fwd<T>(p, 0, g->NY, g->res, g->nx, 1, nullptr, 0.0, nullptr, nullptr, kNoVec, 0.0, tb, nullptr, s));
        IIM_CHECK(cols<T>(p, 0, g->NY - 1, g->outer ? 0 : g->jo0, g->outer ? g->NY - 1 : g->jo1, tb, nullptr, s));
        if (g->outer) IIM_CHECK(free_ring<T>(p, nullptr));
        IIM_CHECK((rows_inv<T, INV_STORE_T>(p, g->jo0, g->jo1 - g->jo0 + 1, tb, pt, nullptr, 0, 0, nullptr, nullptr, s)));
        if (g->outer) {
            // the harmonic part of the correction carries rho minus the ring rows of the residual,
            // as in the recovery below, so that the right-hand side sees the ring data and error
            IIM_CHECK(launch_ring_add(2 * (g->nx + g->ny), -1.0, g->fs_rres, g->fs_rho, nullptr, s));
            IIM_CHECK(free_harmonic<T>(p, g->jo0, g->jo1, nullptr));
            IIM_CHECK((rows_inv<T, INV_ACCUM_T>(p, g->jo0, g->jo1 - g->jo0 + 1, tb, pt, nullptr, 0, 0, nullptr, nullptr, s)));
        }
        const int nga = (g->na + 3) / 4;   // gather blocks: 4 warps, one affected point each
        launch("gather", 0.0, 0.0, k_gather<T, 128>, nga, 128, 0, s, g->na, nga, g->gop_ptr, g->gop_idx, g->gop_w, pt,
               g->cp_body, g->body_circ, g->aff_body, kNoVec, 0, g->bvec, nullptr, 0L, nullptr);
        IIM_LAUNCHED();
        return IIM_OK;
    }

    // ---- psi_ext += P (r - E_a dgamma) at fluid nodes; psibar += dpsibar
    template <typename T>
    iim_status recover(const double* x) {
        Plan<T> p = make_plan<T>(g);
        T* tb = (T*)g->tbuf;
        const VecArg xg{g->na ? x : nullptr, nullptr, 0, 0};
        IIM_CHECK(rows_fwd<T>(p, 0, g->NY, g->res, g->nx, 1, nullptr, 0.0, g->aff_row_ptr, g->aff_node, xg, -1.0, tb,
                              nullptr, s));
        IIM_CHECK(cols<T>(p, 0, g->NY - 1, 0, g->NY - 1, tb, nullptr, s));
        if (g->outer) IIM_CHECK(free_ring<T>(p, nullptr));
        IIM_CHECK((rows_inv<T, INV_ACCUM_FLUID>(p, 0, g->NY, tb, nullptr, g->psi_ext, 0, 0, g->node_class, nullptr, s)));
        if (g->outer) {
            // the harmonic part carries rho minus the ring rows of the last residual: the field
            // harmonic inside the box that removes the ring error (the interior rows do not see
            // it); the ring moves by the same values
            const int nr = 2 * (g->nx + g->ny);
            IIM_CHECK(launch_ring_add(nr, -1.0, g->fs_rres, g->fs_rho, nullptr, s));
            IIM_CHECK(free_harmonic<T>(p, 0, g->NY - 1, nullptr));
            IIM_CHECK((rows_inv<T, INV_ACCUM_FLUID>(p, 0, g->NY, tb, nullptr, g->psi_ext, 0, 0, g->node_class, nullptr, s)));
            IIM_CHECK(launch_ring_add(nr, 1.0, g->fs_rho, g->fs_ring, nullptr, s));
        }
        if (g->ncirc > 0) {
            launch("add_psibar", 0.0, 0.0, k_add_psibar, 1, 64, 0, s, g->ncirc, di() + DI_CIRC, x + g->na, psibar);
            IIM_LAUNCHED();
        }
        return IIM_OK;
    }

    iim_status read_state(int* out8) {
        IIM_TRY(cudaMemcpyAsync(g->h_pinned + 16, di(), 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
        IIM_TRY(cudaStreamSynchronize(s));
        std::memcpy(out8, g->h_pinned + 16, 8 * sizeof(int));
        return IIM_OK;
    }

    // ---- restarted GMRES on S_aug x = b, from x0 (when given and not worse than zero) or 0
    template <typename T>
    iim_status gmres(double tol, int max_it, const double* x0 = nullptr) {
        const int ns_ = ns;
        double* V = g->V;
        double* K = g->H;
        double* x = g->xsol;
        const long ld = ns_;
        const int eb = (ns_ + 255) / 256;
        IIM_TRY(cudaMemsetAsync(x, 0, (size_t)ns_ * sizeof(double), s));
        bool started = false;
        if (!x0) {
            // ||b||, counters, tolerance and V_0 = b / ||b|| in one block
            launch("gmres_start", 0.0, 0.0, k_start_block<256>, 1, 256, 0, s, ns_, (const double*)g->bvec, V, L, K,
                   di(), max_it, tol, g->small + SM_NORM);
            started = true;
        } else {
            launch("gmres_sumsq", 0.0, 0.0, k_sumsq<256>, kNormBlocks, 256, 0, s, g->bvec, ns_, g->partial);
            launch("finish_norm", 0.0, 0.0, k_finish_residual<256>, 1, 256, 0, s, kNormBlocks, g->partial, 0, nullptr,
                   nullptr, 0.0, g->small, nullptr, nullptr, g->small + SM_NORM);
            launch("gmres_init", 0.0, 0.0, k_gmres_init, 1, 1, 0, s, di(), max_it, K, L, g->small + SM_NORM, tol);
        }
        if (x0) {
            // r0 = b - S x0 (the restart path); kept only when ||r0|| < ||b||
            IIM_TRY(cudaMemcpyAsync(x, x0, (size_t)ns_ * sizeof(double), cudaMemcpyDeviceToDevice, s));
            IIM_TRY(cudaMemcpyAsync(V + ld, x0, (size_t)ns_ * sizeof(double), cudaMemcpyDeviceToDevice, s));
            IIM_CHECK(restart_residual<T>(true));
            IIM_TRY(cudaMemcpyAsync(g->h_pinned + 24, K + L.scal() + SC_BETA, sizeof(double), cudaMemcpyDeviceToHost, s));
            IIM_TRY(cudaMemcpyAsync(g->h_pinned + 25, g->small + SM_NORM, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
            IIM_TRY(cudaStreamSynchronize(s));
            const double beta = g->h_pinned[24], bnorm = std::sqrt(g->h_pinned[25]);
            seed_scale = g->h_pinned[26];
            seed_reduction = bnorm > 0.0 ? beta / bnorm : 1.0;
            if (std::isfinite(beta) && beta < bnorm) {
                started = true;
            } else {
                x0_fallback = 1;
                IIM_TRY(cudaMemsetAsync(x, 0, (size_t)ns_ * sizeof(double), s));
                launch("gmres_init", 0.0, 0.0, k_gmres_init, 1, 1, 0, s, di(), max_it, K, L, g->small + SM_NORM, tol);
            }
        }
        if (!started) {
            // V_0 = b / ||b|| (x0 = 0)
            launch("gmres_sumsq", 0.0, 0.0, k_sumsq<256>, kNormBlocks, 256, 0, s, g->bvec, ns_, g->partial);
            launch("gmres_start", 0.0, 0.0, k_start_cycle, eb, 256, 0, s, ns_, g->bvec, V, L, K, kNormBlocks, g->partial,
                   di());
        }
        IIM_LAUNCHED();
        IterGraph* G = nullptr;
        if (use_graph && !profiling_active()) {
            G = (IterGraph*)(sizeof(T) == 8 ? g->graph64 : g->graph32);
            if (!G) {
                G = new IterGraph();
                if (sizeof(T) == 8) g->graph64 = G; else g->graph32 = G;
            }
            IIM_CHECK(ensure_graph<T>(*G));
        }
        int st[8] = {0};
        IIM_CHECK(read_state(st));
        while (!st[DI_STOP] || !st[DI_CONV]) {
            // one cycle: iterate until the device stop flag is set
            while (!st[DI_STOP]) {
                if (G) {
                    // the whole cycle on the device: the WHILE node iterates until the stop flag
                    launch("set_loop", 0.0, 0.0, k_set_int, 1, 1, 0, s, di() + DI_LOOP, 0);
                    IIM_TRY(cudaGraphLaunch(G->exec, s));
                    IIM_CHECK(read_state(st));
                    count_launches((long long)st[DI_LOOP] * G->nodes);
                    if (st[DI_LOOPERR]) {
                        snprintf(g_last_error, sizeof(g_last_error), "GMRES loop ended by its iteration cap");
                        return IIM_ERR_NOT_CONVERGED;
                    }
                } else {
                    IIM_CHECK(iteration<T>());
                    IIM_CHECK(read_state(st));
                }
            }
            if (precond) {
                // x += M (V y)
                double* t = g->pc_z + ns_;
                launch("gmres_backsolve", 0.0, 0.0, k_backsolve_update<256>, 1, 256, 0, s, (const int*)di(), L, K,
                       (const double*)V, ld, ns_, t, 0);
                IIM_CHECK(dense_matvec(ns_, g->pc_aug + ns_, 2L * ns_, t, nullptr, 0, x, 1, nullptr, s));
            } else {
                launch("gmres_backsolve", 0.0, 0.0, k_backsolve, 1, 32, 0, s, di(), L, K);
                launch("gmres_xupdate", 0.0, 0.0, k_xupdate, eb, 256, 0, s, di(), V, ld, K + L.y(), ns_, x);
            }
            IIM_LAUNCHED();
            if (st[DI_CONV] || st[DI_IT] >= max_it) break;
            // restart: V_1 = x, V_2 = S V_1, V_0 = (b - V_2) / ||b - V_2||
            IIM_TRY(cudaMemcpyAsync(V + ld, x, (size_t)ns_ * sizeof(double), cudaMemcpyDeviceToDevice, s));
            IIM_CHECK(restart_residual<T>());
            IIM_CHECK(read_state(st));
        }
        IIM_TRY(cudaMemcpyAsync(g->h_pinned + 12, K + L.scal(), 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
        IIM_TRY(cudaStreamSynchronize(s));
        iters += st[DI_IT];
        const double bnorm = g->h_pinned[12 + SC_TOL] / std::max(tol, 1e-300);
        last_gmres_rel = bnorm > 0.0 ? g->h_pinned[12 + SC_RESID] / bnorm : 0.0;
        return IIM_OK;
    }

    // V_2 = S V_1 (V_1 holds x), then V_0 = (b - V_2) / ||b - V_2||.  With `seed`, x and V_2
    // are first scaled by the c that minimises ||b - c V_2|| (a Krylov seed from a guess).
    template <typename T>
    iim_status restart_residual(bool seed = false) {
        const long ld = ns;
        double* V = g->V;
        double* K = g->H;
        const int eb = (ns + 255) / 256;
        launch("set_tmpj", 0.0, 0.0, k_set_int, 1, 1, 0, s, di() + DI_TMPJ, 1);
        if (dense_op)
            IIM_CHECK(dense_matvec_to(ns, g->pc_S, (long)ns, V + ld, V, di() + DI_TMPJ, ld, nullptr, s));
        else
            IIM_CHECK(apply_at<T>(DI_TMPJ, nullptr));
        if (seed)
            launch("seed_scale", 0.0, 0.0, k_seed_scale<1024>, 1, 1024, 0, s, ns, (const double*)g->bvec, V + 2 * ld,
                   g->xsol, g->small + SM_SEED);
        launch("gmres_axpby", 0.0, 0.0, k_axpby, eb, 256, 0, s, ns, 1.0, g->bvec, -1.0, V + 2 * ld, V + 2 * ld);
        launch("gmres_start", 0.0, 0.0, k_start_block<256>, 1, 256, 0, s, ns, (const double*)(V + 2 * ld), V, L, K,
               di(), -1, 0.0, (double*)nullptr);
        IIM_LAUNCHED();
        return IIM_OK;
    }

    template <typename T>
    iim_status correction(double tol, int max_it, const double* x0 = nullptr) {
        if (ns == 0) return recover<T>(g->xsol);   // no body: the correction is one box solve
        IIM_CHECK(rhs<T>());
        if (direct) {
            // x = M b with the dense inverse of the Schur matrix: no Krylov iterations
            IIM_CHECK(dense_matvec(ns, g->pc_aug + ns, 2L * ns, g->bvec, nullptr, 0, g->xsol, 0, nullptr, s));
        } else {
            IIM_CHECK(gmres<T>(tol, max_it, x0));
        }
        IIM_CHECK(recover<T>(g->xsol));
        return IIM_OK;
    }
    int direct = 0;   // corrections by one application of the dense inverse (opts.precond == 2)
    // the inner Krylov operator is the dense FP32 Schur matrix formed for the preconditioner
    // (opts.precond == 3) instead of the transforms
    bool dense_op = false;
    int pc_mode() const { return precond ? (dense_op ? 2 : 1) : 0; }

    // ---- the whole solve as one graph (SolveGraph); built on the private capture stream
    template <typename T>
    iim_status build_solve_graph(SolveGraph& G, const iim_opts& o, double inner, bool use_cap, double* psi_out,
                                 double* ux_out, double* uy_out) {
        const cudaStream_t user = s;
        IIM_TRY(cudaStreamSynchronize(user));
        cudaGraph_t top = nullptr;
        IIM_TRY(cudaGraphCreate(&top, 0));
        s = g->cap_stream;
        set_capture(true);
        iim_status st = IIM_OK;
        cudaError_t ce = cudaSuccess;
        // one captured piece: begin, launches, end (the capture is always ended)
        auto piece = [&](CapSeg& seg, auto&& body) {
            if (st != IIM_OK || ce != cudaSuccess) return;
            ce = seg.begin();
            if (ce != cudaSuccess) return;
            st = body();
            const cudaError_t e2 = seg.end();
            if (ce == cudaSuccess) ce = e2;
        };
        auto handle = [&](cudaGraph_t graph, cudaGraphConditionalHandle* h) {
            if (st == IIM_OK && ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(h, graph, 0, 0);
        };
        auto cond = [&](CapSeg& seg, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType t, cudaGraph_t* body) {
            if (st == IIM_OK && ce == cudaSuccess) ce = seg.cond(h, t, body);
        };
        const long npad = (long)g->nx * g->NY;
        const int ns_ = ns, eb = (ns_ + 255) / 256;
        const long ld = ns_;
        double* K = g->H;
        double* x = g->xsol;
        CapSeg top_seg{s, top, {}};
        cudaGraphConditionalHandle h_ref = 0, h_cyc = 0, h_it = 0, h_rs = 0;
        cudaGraph_t ref_body = nullptr, cyc_body = nullptr, it_body = nullptr, rs_body = nullptr;
        handle(top, &h_ref);
        piece(top_seg, [&]() -> iim_status {
            launch("init_psi", 0.0, 0.0, k_init_psi, (unsigned)((npad + 255) / 256), 256, 0, s, g->NX, g->NY, nullptr,
                   g->node_class, g->psi_ext);
            if (g->outer) IIM_TRY(cudaMemsetAsync(g->fs_ring, 0, sizeof(double) * 2 * (g->nx + g->ny), s));
            if (g->nb > 0)
                launch("init_psibar", 0.0, 0.0, k_init_psibar, 1, 64, 0, s, g->nb, g->body_circ, psibar, 0, psibar);
            IIM_CHECK(residual_launch());
            launch("ref_init", 0.0, 0.0, k_ref_init, 1, 1, 0, s, h_ref, di(), g->small, o.rtol);
            IIM_LAUNCHED();
            return IIM_OK;
        });
        cond(top_seg, h_ref, cudaGraphCondTypeWhile, &ref_body);
        CapSeg ref_seg{s, ref_body, {}};
        if (ns_ > 0) {
            handle(ref_body, &h_cyc);
            piece(ref_seg, [&]() -> iim_status {
                IIM_CHECK(rhs<T>());
                IIM_TRY(cudaMemsetAsync(x, 0, (size_t)ns_ * sizeof(double), s));
                launch("gmres_start", 0.0, 0.0, k_start_block<256>, 1, 256, 0, s, ns_, (const double*)g->bvec, g->V, L,
                       K, di(), o.max_iter, inner, g->small + SM_NORM);
                launch("cyc_begin", 0.0, 0.0, k_cyc_begin, 1, 1, 0, s, h_cyc, di(), o.max_iter);
                IIM_LAUNCHED();
                return IIM_OK;
            });
            cond(ref_seg, h_cyc, cudaGraphCondTypeWhile, &cyc_body);
            CapSeg cyc_seg{s, cyc_body, {}};
            handle(cyc_body, &h_it);
            handle(cyc_body, &h_rs);
            piece(cyc_seg, [&]() -> iim_status {
                launch("it_begin", 0.0, 0.0, k_it_begin, 1, 1, 0, s, h_it, di());
                IIM_LAUNCHED();
                return IIM_OK;
            });
            cond(cyc_seg, h_it, cudaGraphCondTypeWhile, &it_body);
            CapSeg it_seg{s, it_body, {}};
            piece(it_seg, [&]() -> iim_status {
                IIM_CHECK(iteration<T>());
                launch("gmres_loop_ctl", 0.0, 0.0, k_loop_ctl, 1, 1, 0, s, h_it, di(), m + 2);
                IIM_LAUNCHED();
                return IIM_OK;
            });
            piece(cyc_seg, [&]() -> iim_status {
                if (precond) {
                    double* t = g->pc_z + ns_;
                    launch("gmres_backsolve", 0.0, 0.0, k_backsolve_update<256>, 1, 256, 0, s, (const int*)di(), L, K,
                           (const double*)g->V, ld, ns_, t, 0);
                    IIM_CHECK(dense_matvec(ns_, g->pc_aug + ns_, 2L * ns_, t, nullptr, 0, x, 1, nullptr, s));
                } else {
                    launch("gmres_backsolve", 0.0, 0.0, k_backsolve, 1, 32, 0, s, di(), L, K);
                    launch("gmres_xupdate", 0.0, 0.0, k_xupdate, eb, 256, 0, s, di(), g->V, ld, K + L.y(), ns_, x);
                }
                launch("cyc_ctl", 0.0, 0.0, k_cyc_ctl, 1, 1, 0, s, h_cyc, h_rs, di(), o.max_iter / m + 2);
                IIM_LAUNCHED();
                return IIM_OK;
            });
            cond(cyc_seg, h_rs, cudaGraphCondTypeIf, &rs_body);
            CapSeg rs_seg{s, rs_body, {}};
            piece(rs_seg, [&]() -> iim_status {
                IIM_TRY(cudaMemcpyAsync(g->V + ld, x, (size_t)ns_ * sizeof(double), cudaMemcpyDeviceToDevice, s));
                return restart_residual<T>();
            });
            G.k_cyc = kernel_nodes(cyc_body);
            G.k_it = kernel_nodes(it_body);
            G.k_rs = kernel_nodes(rs_body);
        }
        piece(ref_seg, [&]() -> iim_status {
            IIM_CHECK(recover<T>(x));
            IIM_CHECK(residual_launch());
            launch("ref_ctl", 0.0, 0.0, k_ref_ctl, 1, 1, 0, s, h_ref, di(), g->small, o.rtol,
                   std::min(o.max_refine, 1000), o.max_iter);
            IIM_LAUNCHED();
            return IIM_OK;
        });
        piece(top_seg, [&]() -> iim_status {
            if (use_cap) {
                const int nc = g->ncirc;
                launch("cap_coef", 0.0, 0.0, k_cap_coef, 1, 64, 0, s, nc, (const double*)(g->small + SM_RC),
                       (const double*)g->cap_dev, (const double*)(g->cap_dev + (size_t)nc * nc), g->h * g->h,
                       g->small + SM_CAPC, g->small + SM_CAPP);
                launch("cap_update", 0.0, 0.0, k_cap_update, (unsigned)((npad + 255) / 256), 256, 0, s, npad, nc,
                       (const double*)g->cap_psi, (const double*)(g->small + SM_CAPC), g->psi_ext);
                if (g->outer) {   // the responses' ring values move the free-space ring
                    const long nr = 2L * (g->nx + g->ny);
                    launch("cap_update", 0.0, 0.0, k_cap_update, (unsigned)((nr + 255) / 256), 256, 0, s, nr, nc,
                           (const double*)g->cap_ring, (const double*)(g->small + SM_CAPC), g->fs_ring);
                }
                launch("add_psibar", 0.0, 0.0, k_add_psibar, 1, 64, 0, s, nc, (const int*)(g->d_int + DI_CIRC),
                       (const double*)(g->small + SM_CAPP), psibar);
                IIM_CHECK(residual_launch());
                launch("final_rel", 0.0, 0.0, k_final_rel, 1, 1, 0, s, di(), g->small);
            }
            const long n = (long)g->NX * g->NY;
            launch("velocity_f64", 0.0, 0.0, k_velocity, (unsigned)((n + 255) / 256), 256, 0, s, g->NX, g->NY,
                   0.5 / g->h, g->psi_ext, g->node_class, ring_now(), psi_out, ux_out, uy_out);
            IIM_LAUNCHED();
            return IIM_OK;
        });
        set_capture(false);
        s = user;
        if (st == IIM_OK && ce == cudaSuccess) {
            G.k_top = kernel_nodes(top);
            G.k_ref = ref_body ? kernel_nodes(ref_body) : 0;
            ce = cudaGraphInstantiate(&G.exec, top, 0);
        }
        cudaGraphDestroy(top);
        if (ce != cudaSuccess) {
            G.exec = nullptr;
            record_cuda_error(ce, "whole-solve graph", __FILE__, __LINE__);
            cudaGetLastError();
            return IIM_ERR_CUDA;
        }
        if (st != IIM_OK) {
            if (G.exec) cudaGraphExecDestroy(G.exec);
            G.exec = nullptr;
        }
        return st;
    }

    // Krylov starting point from a streamfunction guess psi0: the body constants it implies,
    // psibar0_k = mean over body k's control points of (psi0 at the adjacent fluid node - psi_b),
    // and x0 = [A psi0 + B sum_k psibar0_k 1_k ; psibar0] (homogeneous data, as in the
    // correction problems).
    iim_status seed_from_guess(const double* psi_guess) {
        const long npad = (long)g->nx * g->NY;
        double* field = (double*)g->tbuf;
        launch("init_psi", 0.0, 0.0, k_init_psi, (unsigned)((npad + 255) / 256), 256, 0, s, g->NX, g->NY, psi_guess,
               g->node_class, field);
        IIM_TRY(cudaMemsetAsync(g->x0g, 0, (size_t)ns * sizeof(double), s));
        if (g->ncirc > 0)
            launch("psibar_estimate", 0.0, 0.0, k_psibar_estimate<128>, g->ncirc, 128, 0, s, g->ncp, g->nx, g->ny, g->cp_axis,
                   g->cp_ei, g->cp_ej, (const double*)g->cp_t, g->cp_body, g->body_circ, g->node_class,
                   (const double*)field, psi_b, g->x0g + g->na, -1.0);
        const int nga = (g->na + 3) / 4;   // gather blocks: 4 warps, one affected point each
        if (g->na > 0)
            launch("gather", 0.0, 0.0, k_gather<double, 128>, nga, 128, 0, s, g->na, nga, g->gop_ptr, g->gop_idx, g->gop_w,
                   (const double*)field, g->cp_body, g->body_circ, g->aff_body, VecArg{g->x0g, nullptr, 0, 0}, 1, g->x0g,
                   nullptr, 0L, nullptr);
        if (g->ncirc > 0)
            launch("psibar_negate", 0.0, 0.0, k_negate, 1, 64, 0, s, g->ncirc, g->x0g + g->na);
        IIM_LAUNCHED();
        return IIM_OK;
    }
    int x0_fallback = 0;
    double seed_scale = 0.0, seed_reduction = 1.0;   // the seed's c and ||b - S c x0|| / ||b||
};

static iim_status ensure_krylov(iim_geometry g, int m) {
    const int ns = g->na + g->ncirc;
    if (g->V && g->krylov_m >= m) return IIM_OK;
    cudaFree(g->V); cudaFree(g->H); cudaFree(g->xsol); cudaFree(g->bvec); cudaFree(g->x0g);
    g->V = g->H = g->xsol = g->bvec = g->x0g = nullptr;
    KLayout L{m};
    IIM_TRY(cudaMalloc(&g->x0g, sizeof(double) * (size_t)std::max(ns, 1)));
    IIM_TRY(cudaMalloc(&g->V, sizeof(double) * (size_t)(m + 1) * std::max(ns, 1)));
    IIM_TRY(cudaMalloc(&g->H, sizeof(double) * (size_t)L.total()));
    IIM_TRY(cudaMalloc(&g->xsol, sizeof(double) * (size_t)std::max(ns, 1)));
    IIM_TRY(cudaMalloc(&g->bvec, sizeof(double) * (size_t)std::max(ns, 1)));
    // zero-filled: the solve graph's control kernels read the scalar slots of H also in solves
    // that never run a Krylov iteration (no affected points), and must not see stale memory
    IIM_TRY(cudaMemset(g->x0g, 0, sizeof(double) * (size_t)std::max(ns, 1)));
    IIM_TRY(cudaMemset(g->V, 0, sizeof(double) * (size_t)(m + 1) * std::max(ns, 1)));
    IIM_TRY(cudaMemset(g->H, 0, sizeof(double) * (size_t)L.total()));
    IIM_TRY(cudaMemset(g->xsol, 0, sizeof(double) * (size_t)std::max(ns, 1)));
    IIM_TRY(cudaMemset(g->bvec, 0, sizeof(double) * (size_t)std::max(ns, 1)));
    g->krylov_m = m;
    // the captured iteration graphs refer to the old buffers
    for (void** gp : {&g->graph64, &g->graph32}) {
        IterGraph* G = (IterGraph*)*gp;
        if (G && G->exec) { cudaGraphExecDestroy(G->exec); G->exec = nullptr; }
    }
    return IIM_OK;
}

static void drop_solve_graph(iim_geometry g) {
    SolveGraph* G = (SolveGraph*)g->solve_graph;
    if (G) {
        if (G->exec) cudaGraphExecDestroy(G->exec);
        delete G;
        g->solve_graph = nullptr;
    }
}

void destroy_graphs(iim_geometry g) {
    lockstep_forget(g);
    drop_solve_graph(g);
    for (void** gp : {&g->graph64, &g->graph32}) {
        IterGraph* G = (IterGraph*)*gp;
        if (G) {
            if (G->exec) cudaGraphExecDestroy(G->exec);
            delete G;
            *gp = nullptr;
        }
    }
}

}  // namespace iim

using namespace iim;

static iim_status poisson_solve(iim_geometry g, const double* omega, const double* psi_b, const double* psi_box,
                                const double* gamma, double* psibar, double* psi_out, double* ux_out, double* uy_out,
                                const double* psi_guess, const iim_opts* opts_in, iim_stats* stats, cudaStream_t s,
                                bool capacitance, int* enqueued = nullptr);
static iim_status graph_finish(iim_geometry g, const iim_opts& opts, iim_stats* stats);

// Responses to unit circulation (Sec. 4.2's circulation constraint, solved by capacitance): for
// each circulation body l, the solve with omega = 0, zero body and box data and Gamma = e_l; its
// padded psi_ext, its psibar values and the circulations it measures on every R_k.  C (measured
// circulations, k x l) is inverted on the host; a solve then adds sum_l (C^-1 e)_l resp_l with
// e = Gamma - measured circulation, which makes the measured circulation equal Gamma to rounding.
static iim_status build_capacitance(iim_geometry g, const iim_opts& opts, cudaStream_t s) {
    const int nc = g->ncirc, nb = g->nb;
    const long npad = (long)g->nx * g->NY, nxy = (long)g->NX * g->NY;
    if (!g->cap_psi) IIM_TRY(cudaMalloc(&g->cap_psi, sizeof(double) * (size_t)nc * npad));
    double *w0 = nullptr, *out = nullptr, *pb0 = nullptr, *gam = nullptr, *pbar = nullptr;
    iim_status st = IIM_OK;
    auto alloc = [&](double** p, size_t n) {
        if (st == IIM_OK && cudaMalloc(p, sizeof(double) * std::max<size_t>(n, 1)) != cudaSuccess) st = IIM_ERR_CUDA;
        if (st == IIM_OK && cudaMemsetAsync(*p, 0, sizeof(double) * std::max<size_t>(n, 1), s) != cudaSuccess)
            st = IIM_ERR_CUDA;
    };
    alloc(&w0, nxy); alloc(&out, nxy); alloc(&pb0, g->ncp); alloc(&gam, nb); alloc(&pbar, nb);
    std::vector<double> C((size_t)nc * nc), pbv((size_t)nc * nc), hg(nb), hp(nb), circ(nc);
    iim_opts o = opts;
    o.rtol = std::min(opts.rtol, 1e-11);
    o.guess = 0;
    g->plane_off = 1;   // the responses carry no data: no plane sources (host-driven solves)
    for (int l = 0; l < nc && st == IIM_OK; ++l) {
        std::fill(hg.begin(), hg.end(), 0.0);
        hg[g->circ_ids[l]] = 1.0;
        if (cudaMemcpyAsync(gam, hg.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = IIM_ERR_CUDA;
            break;
        }
        st = poisson_solve(g, w0, pb0, nullptr, gam, pbar, out, nullptr, nullptr, nullptr, &o, nullptr, s, false);
        if (st != IIM_OK) break;
        const size_t nring = 2 * (size_t)(g->nx + g->ny);
        if (g->outer && !g->cap_ring && cudaMalloc(&g->cap_ring, sizeof(double) * (size_t)nc * nring) != cudaSuccess) {
            st = IIM_ERR_CUDA;
            break;
        }
        if ((g->outer && cudaMemcpyAsync(g->cap_ring + (size_t)l * nring, g->fs_ring, sizeof(double) * nring,
                                         cudaMemcpyDeviceToDevice, s) != cudaSuccess) ||
            cudaMemcpyAsync(g->cap_psi + (size_t)l * npad, g->psi_ext, sizeof(double) * npad, cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess ||
            cudaMemcpyAsync(hp.data(), pbar, sizeof(double) * nb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(circ.data(), g->small + SM_CIRC, sizeof(double) * nc, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = IIM_ERR_CUDA;
            break;
        }
        for (int k = 0; k < nc; ++k) {
            C[(size_t)k * nc + l] = circ[k];
            pbv[(size_t)l * nc + k] = hp[g->circ_ids[k]];
        }
    }
    g->plane_off = 0;
    cudaFree(w0); cudaFree(out); cudaFree(pb0); cudaFree(gam); cudaFree(pbar);
    if (st != IIM_OK) return st;
    // invert C (close to the identity) by Gauss-Jordan with partial pivoting
    std::vector<double> inv((size_t)nc * nc, 0.0);
    for (int k = 0; k < nc; ++k) inv[(size_t)k * nc + k] = 1.0;
    for (int k = 0; k < nc; ++k) {
        int piv = k;
        for (int r = k + 1; r < nc; ++r)
            if (std::fabs(C[(size_t)r * nc + k]) > std::fabs(C[(size_t)piv * nc + k])) piv = r;
        if (!(std::fabs(C[(size_t)piv * nc + k]) > 0.0)) {
            snprintf(g_last_error, sizeof(g_last_error), "circulation capacitance matrix singular");
            return IIM_ERR_NOT_CONVERGED;
        }
        for (int c = 0; c < nc; ++c) {
            std::swap(C[(size_t)k * nc + c], C[(size_t)piv * nc + c]);
            std::swap(inv[(size_t)k * nc + c], inv[(size_t)piv * nc + c]);
        }
        const double d = 1.0 / C[(size_t)k * nc + k];
        for (int c = 0; c < nc; ++c) { C[(size_t)k * nc + c] *= d; inv[(size_t)k * nc + c] *= d; }
        for (int r = 0; r < nc; ++r) {
            if (r == k) continue;
            const double f = C[(size_t)r * nc + k];
            if (f == 0.0) continue;
            for (int c = 0; c < nc; ++c) {
                C[(size_t)r * nc + c] -= f * C[(size_t)k * nc + c];
                inv[(size_t)r * nc + c] -= f * inv[(size_t)k * nc + c];
            }
        }
    }
    g->cap_cinv = inv;
    g->cap_pb = pbv;
    if (!g->cap_dev) IIM_TRY(cudaMalloc(&g->cap_dev, sizeof(double) * 2 * (size_t)nc * nc));
    IIM_TRY(cudaMemcpyAsync(g->cap_dev, inv.data(), sizeof(double) * (size_t)nc * nc, cudaMemcpyHostToDevice, s));
    IIM_TRY(cudaMemcpyAsync(g->cap_dev + (size_t)nc * nc, pbv.data(), sizeof(double) * (size_t)nc * nc,
                            cudaMemcpyHostToDevice, s));
    IIM_TRY(cudaStreamSynchronize(s));
    g->cap_ready = 1;
    return IIM_OK;
}

namespace iim {
// For the batched solver: launch the whole-solve graph without waiting (see poisson_solve's
// `enqueued`), and read its results once the stream has been synchronised.
iim_status solve_enqueue(iim_geometry g, const double* omega, const double* psi_b, const double* psi_box,
                         const double* gamma, double* psibar, double* psi_out, double* ux_out, double* uy_out,
                         const iim_opts* opts, iim_stats* stats, cudaStream_t s, int* enqueued) {
    return poisson_solve(g, omega, psi_b, psi_box, gamma, psibar, psi_out, ux_out, uy_out, nullptr, opts, stats, s,
                         true, enqueued);
}
iim_status solve_finish(iim_geometry g, const iim_opts* opts_in, iim_stats* stats) {
    iim_opts opts{IIM_FP64, 1e-10, 2000, 64, 12, 0, 0.0, 0};
    if (opts_in) opts = *opts_in;
    return graph_finish(g, opts, stats);
}
}  // namespace iim

extern "C" iim_status iim_poisson_solve(iim_geometry g, const double* omega, const double* psi_b, const double* psi_box,
                                        const double* gamma, double* psibar, double* psi_out, double* ux_out,
                                        double* uy_out, const double* psi_guess, const iim_opts* opts_in,
                                        iim_stats* stats, iim_stream stream) {
    return poisson_solve(g, omega, psi_b, psi_box, gamma, psibar, psi_out, ux_out, uy_out, psi_guess, opts_in, stats,
                         (cudaStream_t)stream, true);
}

// Reads the counters a whole-solve graph run left in the pinned block and fills the status and
// the stats (the stream that ran it has been synchronised).
static iim_status graph_finish(iim_geometry g, const iim_opts& opts, iim_stats* stats) {
    const SolveGraph* G = (const SolveGraph*)g->solve_graph;
    const int* hi = reinterpret_cast<const int*>(g->h_pinned + 32);
    const double rel = g->h_pinned[40];
    iim_status st = IIM_OK;
    if (hi[DI_NONFIN]) {
        st = IIM_ERR_NONFINITE;
    } else if (hi[DI_LOOPERR] || hi[DI_CYCERR]) {
        snprintf(g_last_error, sizeof(g_last_error), "GMRES loop ended by its iteration cap");
        st = IIM_ERR_NOT_CONVERGED;
    } else if (rel > opts.rtol) {
        st = IIM_ERR_NOT_CONVERGED;
    }
    count_launches(G->k_top + (long long)hi[DI_REF] * G->k_ref + (long long)hi[DI_CYCS] * G->k_cyc +
                   (long long)hi[DI_ITS] * G->k_it + (long long)hi[DI_RSS] * G->k_rs);
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->iters = hi[DI_ITS];
        stats->refinements = hi[DI_REF];
        stats->status = st;
        stats->rel_res = rel;
        const double bn = g->h_pinned[44 + SC_TOL] / std::max(G->inner, 1e-300);
        stats->gmres_rel_res = (g->na + g->ncirc) > 0 && bn > 0.0 ? g->h_pinned[44 + SC_RESID] / bn : 0.0;
        stats->circ_err_max = g->h_pinned[41];
        stats->seed_rel_res = 1.0;
        stats->iters_first = hi[DI_FIRST];
        cudaEventElapsedTime(&stats->ms, g->ev0, g->ev1);
    }
    return st;
}

// `enqueued` (batched solves): NULL = ordinary blocking call.  Otherwise *enqueued = 1 when the
// whole-solve graph was launched on s and nothing was waited for (graph_finish after the stream
// is synchronised), 0 when the solve ran to completion here, -1 when the graph path does not
// apply yet and nothing was done.
static iim_status poisson_solve(iim_geometry g, const double* omega, const double* psi_b, const double* psi_box,
                                const double* gamma, double* psibar, double* psi_out, double* ux_out, double* uy_out,
                                const double* psi_guess, const iim_opts* opts_in, iim_stats* stats, cudaStream_t s,
                                bool capacitance, int* enqueued) {
    iim_opts opts{IIM_FP64, 1e-10, 2000, 64, 12, 0, 0.0, 0};
    if (opts_in) opts = *opts_in;
    if (g && g->wall == 1 && g->psibar_zero) psibar = g->psibar_zero;   // a Neumann wall has no body constants
    if (enqueued) {
        *enqueued = 0;
        if (!(g && g->host_solves > 0 && !g->solve_graph_failed && opts.guess == 0 && opts.precond != 2 &&
              !profiling_active())) {
            *enqueued = -1;
            return IIM_OK;
        }
    }
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (!g || !omega || !psi_out || (g->ncp > 0 && !psi_b) || (g->nb > 0 && !psibar)) return IIM_ERR_INVALID_ARG;
    if (opts.prec != IIM_FP64 && opts.prec != IIM_MIXED) return IIM_ERR_INVALID_ARG;
    if (opts.restart < 1 || opts.restart > 64 || !(opts.rtol > 0.0) || opts.max_iter < 1 || opts.max_refine < 1)
        return IIM_ERR_INVALID_ARG;
    if ((opts.guess == 1 || opts.guess == 2) && !psi_guess) return IIM_ERR_INVALID_ARG;
    if (g->outer && opts.guess == 1) return IIM_ERR_INVALID_ARG;   // a free-space iterate has no given ring
    if (g->outer) psi_box = nullptr;                                  // the ring is part of the solution
    if (opts.guess < 0 || opts.guess > 2 || opts.precond < 0 || opts.precond > 3) return IIM_ERR_INVALID_ARG;
    IIM_CHECK(ensure_twiddles());
    IIM_CHECK(ensure_krylov(g, opts.restart));
    if (g->ncirc > 0)
        IIM_TRY(cudaMemcpyAsync(g->d_int + DI_CIRC, g->circ_ids.data(), g->ncirc * sizeof(int), cudaMemcpyHostToDevice, s));

    Solver S;
    S.g = g; S.s = s; S.prec = opts.prec; S.omega = omega; S.psi_b = psi_b; S.ring = psi_box; S.gamma = gamma;
    S.psibar = psibar; S.ns = g->na + g->ncirc; S.m = opts.restart; S.L = KLayout{opts.restart};
    S.precond = opts.precond != 0 && S.ns > 0;
    S.direct = opts.precond == 2 && S.ns > 0;
    S.dense_op = opts.precond == 3 && S.ns > 0 && dense_matvec_fits(S.ns);
    if (S.precond && !g->pc_ready) IIM_CHECK(S.build_precond());
    const bool use_cap = capacitance && g->ncirc > 0;
    if (use_cap && !g->cap_ready) {
        IIM_CHECK(build_capacitance(g, opts, s));
        if (g->ncirc > 0)
            IIM_TRY(cudaMemcpyAsync(g->d_int + DI_CIRC, g->circ_ids.data(), g->ncirc * sizeof(int),
                                    cudaMemcpyHostToDevice, s));
    }
    const long npad = (long)g->nx * g->NY;
    const double inner = opts.inner_rtol > 0.0 ? opts.inner_rtol : (opts.prec == IIM_FP64 ? opts.rtol / 20.0 : 1e-4);

    // After one host-driven solve on the geometry, solves without a guess (and not profiled,
    // not in direct-correction mode) run as one device-driven graph: no host round trip per
    // refinement or GMRES cycle.  The graph is rebuilt when the arguments change.
    if (capacitance && S.use_graph && !profiling_active() && opts.guess == 0 && opts.precond != 2 &&
        g->host_solves > 0 && !g->solve_graph_failed) {
        const void* key[9] = {omega, psi_b, psi_box, gamma, psibar, psi_out, ux_out, uy_out, g->V};
        SolveGraph* G = (SolveGraph*)g->solve_graph;
        const bool match = G && G->exec && G->prec == opts.prec && G->m == opts.restart && G->pc == S.pc_mode() &&
                           G->max_refine == opts.max_refine && G->max_iter == opts.max_iter &&
                           G->cap == (int)use_cap && G->inner == inner && G->rtol == opts.rtol &&
                           std::memcmp(G->ptrs, key, sizeof(key)) == 0;
        if (!match) {
            drop_solve_graph(g);
            G = new SolveGraph();
            G->prec = opts.prec; G->m = opts.restart; G->pc = S.pc_mode(); G->max_refine = opts.max_refine;
            G->max_iter = opts.max_iter; G->cap = (int)use_cap; G->inner = inner; G->rtol = opts.rtol;
            std::memcpy(G->ptrs, key, sizeof(key));
            const iim_status bs =
                opts.prec == IIM_FP64
                    ? S.build_solve_graph<double>(*G, opts, inner, use_cap, psi_out, ux_out, uy_out)
                    : S.build_solve_graph<float>(*G, opts, inner, use_cap, psi_out, ux_out, uy_out);
            if (bs != IIM_OK || !G->exec) {
                delete G;
                G = nullptr;
                g->solve_graph_failed = 1;   // the host-driven path below, from now on
            } else {
                g->solve_graph = G;
            }
        }
        if (G) {
            IIM_TRY(cudaEventRecord(g->ev0, s));
            IIM_TRY(cudaGraphLaunch(G->exec, s));
            IIM_TRY(cudaEventRecord(g->ev1, s));
            int* hi = reinterpret_cast<int*>(g->h_pinned + 32);
            IIM_TRY(cudaMemcpyAsync(hi, g->d_int, 16 * sizeof(int), cudaMemcpyDeviceToHost, s));
            IIM_TRY(cudaMemcpyAsync(g->h_pinned + 40, g->small + SM_REL, sizeof(double), cudaMemcpyDeviceToHost, s));
            IIM_TRY(cudaMemcpyAsync(g->h_pinned + 41, g->small + SM_CIRC_ERR, sizeof(double), cudaMemcpyDeviceToHost, s));
            IIM_TRY(cudaMemcpyAsync(g->h_pinned + 44, g->H + S.L.scal(), 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
            if (enqueued) {
                *enqueued = 1;
                return IIM_OK;
            }
            IIM_TRY(cudaStreamSynchronize(s));
            return graph_finish(g, opts, stats);
        }
    }
    IIM_TRY(cudaEventRecord(g->ev0, s));

    // ||f||: residual at psi = 0 (ghosts from the boundary data only)
    double res2 = 0.0, cerr = 0.0;
    int fallback = 0;
    launch("init_psi", 0.0, 0.0, k_init_psi, (unsigned)((npad + 255) / 256), 256, 0, s, g->NX, g->NY, nullptr,
           g->node_class, g->psi_ext);
    if (g->outer) IIM_TRY(cudaMemsetAsync(g->fs_ring, 0, sizeof(double) * 2 * (g->nx + g->ny), s));
    if (g->nb > 0) launch("init_psibar", 0.0, 0.0, k_init_psibar, 1, 64, 0, s, g->nb, g->body_circ, psibar, 0, psibar);
    IIM_LAUNCHED();
    IIM_CHECK(S.residual(&res2, &cerr));
    if (!std::isfinite(res2)) return IIM_ERR_NONFINITE;
    const double fnorm = std::sqrt(res2);
    if (opts.guess == 1) {
        launch("init_psi", 0.0, 0.0, k_init_psi, (unsigned)((npad + 255) / 256), 256, 0, s, g->NX, g->NY, psi_guess,
               g->node_class, g->psi_ext);
        IIM_LAUNCHED();
        double r2g = 0.0, cg = 0.0;
        IIM_CHECK(S.residual(&r2g, &cg));
        if (std::isfinite(r2g) && r2g < res2) {
            res2 = r2g;
            cerr = cg;
        } else {
            // the guess raised the residual: start again from zero
            fallback = 1;
            launch("init_psi", 0.0, 0.0, k_init_psi, (unsigned)((npad + 255) / 256), 256, 0, s, g->NX, g->NY, nullptr,
                   g->node_class, g->psi_ext);
            IIM_LAUNCHED();
            IIM_CHECK(S.residual(&res2, &cerr));
        }
    }
    double rel = fnorm > 0.0 ? std::sqrt(res2) / fnorm : 0.0;
    int refinements = 0;
    iim_status st = IIM_OK;
    const double* x0 = nullptr;
    if (opts.guess == 2 && S.ns > 0) {
        IIM_CHECK(S.seed_from_guess(psi_guess));
        x0 = g->x0g;
    }
    int iters_first = 0, direct_fallback = 0;
    while (rel > opts.rtol) {
        if (refinements >= opts.max_refine || S.iters >= opts.max_iter) { st = IIM_ERR_NOT_CONVERGED; break; }
        const int budget = opts.max_iter - S.iters;
        // the guess seeds the Krylov unknowns of the first correction only
        const double* sx = refinements == 0 ? x0 : nullptr;
        const double rel_before = rel;
        iim_status cs = opts.prec == IIM_FP64 ? S.correction<double>(inner, budget, sx)
                                              : S.correction<float>(inner, budget, sx);
        if (cs != IIM_OK) { st = cs; break; }
        if (refinements == 0) iters_first = S.iters;
        ++refinements;
        IIM_CHECK(S.residual(&res2, &cerr));
        if (!std::isfinite(res2)) { st = IIM_ERR_NONFINITE; break; }
        rel = std::sqrt(res2) / fnorm;
        // a direct correction that did not halve the residual hands over to preconditioned GMRES
        if (S.direct && !(rel < 0.5 * rel_before)) {
            S.direct = 0;
            direct_fallback = 1;
        }
    }
    if (use_cap && g->cap_ready && (st == IIM_OK || st == IIM_ERR_NOT_CONVERGED)) {
        // e_c = Gamma - measured circulation (from the last residual), coefficients C^-1 e, then
        // psi_ext and psibar move along the unit-circulation responses; the residual is redone
        const int nc = g->ncirc;
        std::vector<double> rc(nc), coef(nc), dpb(nc, 0.0);
        IIM_TRY(cudaMemcpyAsync(rc.data(), g->small + SM_RC, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
        IIM_TRY(cudaStreamSynchronize(s));
        const double h2 = g->h * g->h;
        for (int l = 0; l < nc; ++l) {
            double a = 0.0;
            for (int k = 0; k < nc; ++k) a += g->cap_cinv[(size_t)l * nc + k] * (rc[k] * h2);
            coef[l] = a;
        }
        for (int l = 0; l < nc; ++l)
            for (int c = 0; c < nc; ++c) dpb[c] += coef[l] * g->cap_pb[(size_t)l * nc + c];
        IIM_TRY(cudaMemcpyAsync(g->small + SM_CAPC, coef.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, s));
        IIM_TRY(cudaMemcpyAsync(g->small + SM_CAPP, dpb.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, s));
        launch("cap_update", 0.0, 0.0, k_cap_update, (unsigned)((npad + 255) / 256), 256, 0, s, npad, nc,
               (const double*)g->cap_psi, (const double*)(g->small + SM_CAPC), g->psi_ext);
        if (g->outer) {   // the responses' ring values move the free-space ring
            const long nr = 2L * (g->nx + g->ny);
            launch("cap_update", 0.0, 0.0, k_cap_update, (unsigned)((nr + 255) / 256), 256, 0, s, nr, nc,
                   (const double*)g->cap_ring, (const double*)(g->small + SM_CAPC), g->fs_ring);
        }
        launch("add_psibar", 0.0, 0.0, k_add_psibar, 1, 64, 0, s, nc, (const int*)(g->d_int + DI_CIRC),
               (const double*)(g->small + SM_CAPP), psibar);
        IIM_LAUNCHED();
        IIM_CHECK(S.residual(&res2, &cerr));
        rel = fnorm > 0.0 ? std::sqrt(res2) / fnorm : 0.0;
    }
    const long n = (long)g->NX * g->NY;
    launch("velocity_f64", (double)n * (9.0 + 8.0 + (ux_out ? 8.0 : 0.0) + (uy_out ? 8.0 : 0.0)), 0.0, k_velocity,
           (unsigned)((n + 255) / 256), 256, 0, s, g->NX, g->NY, 0.5 / g->h, g->psi_ext, g->node_class, S.ring_now(), psi_out,
           ux_out, uy_out);
    IIM_LAUNCHED();
    IIM_TRY(cudaEventRecord(g->ev1, s));
    IIM_TRY(cudaEventSynchronize(g->ev1));
    if (stats) {
        stats->iters = S.iters;
        stats->refinements = refinements;
        stats->fallback = fallback | S.x0_fallback | (direct_fallback << 1);
        stats->status = st;
        stats->rel_res = rel;
        stats->gmres_rel_res = S.last_gmres_rel;
        stats->circ_err_max = cerr;
        stats->seed_rel_res = S.seed_reduction;
        stats->iters_first = iters_first;
        cudaEventElapsedTime(&stats->ms, g->ev0, g->ev1);
    }
    if (capacitance && st == IIM_OK) ++g->host_solves;
    return st;
}

extern "C" iim_status iim_geometry_set_lines(iim_geometry g, int threads_per_line) {
    if (!g || (threads_per_line != 32 && threads_per_line != 64)) return IIM_ERR_INVALID_ARG;
    const int wide = threads_per_line == 64 ? 1 : 0;
    if (g->wide_lines != wide) {
        g->wide_lines = wide;
        drop_solve_graph(g);
        // captured iteration graphs hold the previous kernels
        for (void** gp : {&g->graph64, &g->graph32}) {
            IterGraph* G = (IterGraph*)*gp;
            if (G && G->exec) { cudaGraphExecDestroy(G->exec); G->exec = nullptr; }
        }
    }
    return IIM_OK;
}

extern "C" iim_status iim_geometry_set_outer(iim_geometry g, int outer) {
    if (!g || outer < 0 || outer > 2) return IIM_ERR_INVALID_ARG;
    if (g->outer == outer) return IIM_OK;
    int cur = 0;
    IIM_TRY(cudaGetDevice(&cur));
    IIM_TRY(cudaSetDevice(g->device));
    iim_status st = IIM_OK;
    if (outer >= 1) {
        const size_t nring = 2 * (size_t)(g->nx + g->ny), nbnd = 2 * (size_t)(g->NX + g->NY);
        const int M = outer == 2 ? 2 * g->nx : g->nx;   // table columns: with the plane, the images too
        st = lgf_table(M, g->ny, &g->lgf);
        if (st == IIM_OK) g->lgf_ld = M + 1;
        if (st == IIM_OK && !g->fs_plane) {
            if (cudaMalloc(&g->fs_plane, sizeof(double) * (size_t)g->NY) != cudaSuccess ||
                cudaMemset(g->fs_plane, 0, sizeof(double) * (size_t)g->NY) != cudaSuccess) {
                record_cuda_error(cudaGetLastError(), "free-space buffers", __FILE__, __LINE__);
                st = IIM_ERR_CUDA;
            }
        }
        if (st == IIM_OK && !g->fs_ring) {
            if (cudaMalloc(&g->fs_ring, sizeof(double) * nring) != cudaSuccess ||
                cudaMalloc(&g->fs_rho, sizeof(double) * nring) != cudaSuccess ||
                cudaMalloc(&g->fs_bnd, sizeof(double) * nbnd) != cudaSuccess ||
                cudaMalloc(&g->fs_rres, sizeof(double) * nring) != cudaSuccess ||
                cudaMemset(g->fs_rres, 0, sizeof(double) * nring) != cudaSuccess ||
                cudaMemset(g->fs_ring, 0, sizeof(double) * nring) != cudaSuccess) {
                record_cuda_error(cudaGetLastError(), "free-space buffers", __FILE__, __LINE__);
                st = IIM_ERR_CUDA;
            }
        }
    }
    if (st == IIM_OK) {
        g->outer = outer;
        // everything built from the rectangular operator is rebuilt on the next solve
        g->pc_ready = 0;
        g->cap_ready = 0;
        g->host_solves = 0;
        drop_solve_graph(g);
        lockstep_forget(g);
        for (void** gp : {&g->graph64, &g->graph32}) {
            IterGraph* G = (IterGraph*)*gp;
            if (G && G->exec) { cudaGraphExecDestroy(G->exec); G->exec = nullptr; }
        }
    }
    cudaSetDevice(cur);
    return st;
}

extern "C" iim_status iim_geometry_set_plane_vorticity(iim_geometry g, const double* w, iim_stream stream) {
    if (!g || !w || g->outer != 2 || !g->fs_plane) return IIM_ERR_INVALID_ARG;
    IIM_TRY(cudaMemcpyAsync(g->fs_plane, w, sizeof(double) * (size_t)g->NY, cudaMemcpyDefault, (cudaStream_t)stream));
    return IIM_OK;
}

extern "C" iim_status iim_geometry_outer_ring(iim_geometry g, double* ring, iim_stream stream) {
    if (!g || !ring || !g->outer || !g->fs_ring) return IIM_ERR_INVALID_ARG;
    IIM_TRY(cudaMemcpyAsync(ring, g->fs_ring, sizeof(double) * 2 * (g->nx + g->ny), cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
    return IIM_OK;
}

extern "C" iim_status iim_geometry_set_column_solver(iim_geometry g, int mode) {
    if (!g || (mode != 0 && mode != 1)) return IIM_ERR_INVALID_ARG;
    if (g->col_solver != mode) {
        g->col_solver = mode;
        // the preconditioner and the circulation responses were built with the other pass's
        // rounding: rebuilt by the next solve that uses them
        g->pc_ready = 0;
        g->cap_ready = 0;
        lockstep_forget(g);
        drop_solve_graph(g);   // the captured kernels change
        for (void** gp : {&g->graph64, &g->graph32}) {
            IterGraph* G = (IterGraph*)*gp;
            if (G && G->exec) { cudaGraphExecDestroy(G->exec); G->exec = nullptr; }
        }
    }
    return IIM_OK;
}

extern "C" iim_status iim_geometry_set_wall_condition(iim_geometry g, int kind, iim_stream stream) {
    if (!g || (kind != 0 && kind != 1)) return IIM_ERR_INVALID_ARG;
    if (kind == 1 && g->ncirc > 0) return IIM_ERR_INVALID_ARG;   // circulation bodies need psibar_k unknowns
    if (g->wall == kind) return IIM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 1 && !g->psibar_zero && g->nb > 0) {
        IIM_TRY(cudaMalloc(&g->psibar_zero, g->nb * sizeof(double)));
        IIM_TRY(cudaMemsetAsync(g->psibar_zero, 0, g->nb * sizeof(double), s));
    }
    IIM_CHECK(rewrite_wall_weights(g, kind, s));
    g->wall = kind;
    // the operator A, B changed: preconditioner, dense operator and captured solves are rebuilt
    g->pc_ready = 0;
    g->cap_ready = 0;
    lockstep_forget(g);
    drop_solve_graph(g);
    for (void** gp : {&g->graph64, &g->graph32}) {
        IterGraph* G = (IterGraph*)*gp;
        if (G && G->exec) { cudaGraphExecDestroy(G->exec); G->exec = nullptr; }
    }
    return IIM_OK;
}

extern "C" iim_status iim_geometry_set_tiles(iim_geometry g, int cols_per_block) {
    if (!g || (cols_per_block != 2 && cols_per_block != 4 && cols_per_block != 8)) return IIM_ERR_INVALID_ARG;
    if (g->cols_c != cols_per_block) {
        g->cols_c = cols_per_block;
        drop_solve_graph(g);
        // captured iteration graphs hold the previous kernels
        for (void** gp : {&g->graph64, &g->graph32}) {
            IterGraph* G = (IterGraph*)*gp;
            if (G && G->exec) { cudaGraphExecDestroy(G->exec); G->exec = nullptr; }
        }
    }
    return IIM_OK;
}

extern "C" iim_status iim_build_preconditioner(iim_geometry g, float* setup_ms, iim_stream stream) {
    if (!g) return IIM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    IIM_CHECK(ensure_twiddles());
    IIM_CHECK(ensure_krylov(g, std::max(g->krylov_m, 2)));
    if (g->ncirc > 0)
        IIM_TRY(cudaMemcpyAsync(g->d_int + DI_CIRC, g->circ_ids.data(), g->ncirc * sizeof(int), cudaMemcpyHostToDevice, s));
    Solver S;
    S.g = g; S.s = s; S.prec = IIM_MIXED; S.ns = g->na + g->ncirc; S.m = g->krylov_m; S.L = KLayout{g->krylov_m};
    if (S.ns > 0) IIM_CHECK(S.build_precond());
    if (setup_ms) *setup_ms = g->pc_setup_ms;
    return IIM_OK;
}

// Rectangular Dirichlet-box solve with caller workspace (Sec. 4.2 solution operator).
extern "C" iim_status iim_box_poisson(const iim_grid* grid, const double* f, const double* psi_box, double* u, int prec,
                                      double* work, iim_stream stream) {
    if (!grid || !f || !u || !work) return IIM_ERR_INVALID_ARG;
    const int nx = grid->nx, ny = grid->ny;
    if (!is_pow2_in(nx, 16, 2048) || !is_pow2_in(ny, 16, 2048)) return IIM_ERR_INVALID_ARG;
    if (prec != IIM_FP64 && prec != IIM_MIXED) return IIM_ERR_INVALID_ARG;
    const double h = (grid->x1 - grid->x0) / nx;
    if (!(h > 0.0)) return IIM_ERR_INVALID_ARG;
    IIM_CHECK(ensure_twiddles());
    cudaStream_t s = (cudaStream_t)stream;
    const int NX = nx - 1, NY = ny - 1;
    // work: padded transform buffer (nx*NY) followed by the eigenvalue tables (NX + NY)
    double* buf = work;
    double* lam = work + (size_t)nx * NY;
    std::vector<double> lx(NX + NY);
    for (int k = 0; k < NX; ++k) lx[k] = (2.0 - 2.0 * std::cos(M_PI * (k + 1) / nx)) / (h * h);
    for (int k = 0; k < NY; ++k) lx[NX + k] = (2.0 - 2.0 * std::cos(M_PI * (k + 1) / ny)) / (h * h);
    const double ih2 = 1.0 / (h * h);
    if (prec == IIM_FP64) {
        IIM_TRY(cudaMemcpyAsync(lam, lx.data(), sizeof(double) * (NX + NY), cudaMemcpyHostToDevice, s));
        Plan<double> p{NX, NY, nx, ny, ilog2(nx), ilog2(ny), lam, lam + NX, twiddles64(), (2.0 / nx) * (2.0 / ny)};
        IIM_CHECK(rows_fwd<double>(p, 0, NY, f, NX, 0, psi_box, ih2, nullptr, nullptr, kNoVec, 0.0, buf, nullptr, s));
        IIM_CHECK(cols<double>(p, 0, NY - 1, 0, NY - 1, buf, nullptr, s));
        IIM_CHECK((rows_inv<double, INV_STORE_F64>(p, 0, NY, buf, nullptr, u, NX, 0, nullptr, nullptr, s)));
    } else {
        std::vector<float> fl(NX + NY);
        for (int k = 0; k < NX + NY; ++k) fl[k] = (float)lx[k];
        float* lamf = (float*)lam;
        IIM_TRY(cudaMemcpyAsync(lamf, fl.data(), sizeof(float) * (NX + NY), cudaMemcpyHostToDevice, s));
        Plan<float> p{NX, NY, nx, ny, ilog2(nx), ilog2(ny), lamf, lamf + NX, twiddles32(), (float)((2.0 / nx) * (2.0 / ny))};
        float* fb = (float*)buf;
        IIM_CHECK(rows_fwd<float>(p, 0, NY, f, NX, 0, psi_box, ih2, nullptr, nullptr, kNoVec, 0.0, fb, nullptr, s));
        IIM_CHECK(cols<float>(p, 0, NY - 1, 0, NY - 1, fb, nullptr, s));
        IIM_CHECK((rows_inv<float, INV_STORE_F64>(p, 0, NY, fb, nullptr, u, NX, 0, nullptr, nullptr, s)));
    }
    // pageable-memory copies are staged before cudaMemcpyAsync returns, so the host vectors
    // may go out of scope here
    return IIM_OK;
}

// ------------------------------------------------------------------------- pass timing
// Times the three passes of the geometry's rectangular solve in the precision `prec`: the
// forward row transforms of a dense FP64 field (one launch per field), the column pass and the
// inverse row transforms (one launch over all `batch` fields).  Each pass is captured `reps`
// times back to back into a CUDA graph of its own; CUDA events on the stream around a launch of
// that graph give its device time with no host gap between the kernels.  Inputs are a fixed
// smooth field.
template <typename T>
static iim_status time_passes(iim_geometry g, int batch, int reps, double* us, double* bytes, cudaStream_t cs) {
    const Plan<T> p = make_plan<T>(g);
    const long fs = (long)p.nx * p.NY;
    T *buf = nullptr, *out = nullptr;
    double* dense = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    iim_status st = IIM_OK;
#define TP_TRY(call)                                                          \
    do {                                                                      \
        const cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess && st == IIM_OK) {                              \
            record_cuda_error(e_, "iim_time_box_passes", __FILE__, __LINE__); \
            st = IIM_ERR_CUDA;                                                \
        }                                                                     \
    } while (0)
    TP_TRY(cudaMalloc((void**)&buf, sizeof(T) * fs * batch));
    TP_TRY(cudaMalloc((void**)&out, sizeof(T) * fs * batch));
    TP_TRY(cudaMalloc((void**)&dense, sizeof(double) * fs * batch));
    TP_TRY(cudaEventCreate(&ev0));
    TP_TRY(cudaEventCreate(&ev1));
    if (st == IIM_OK) {
        std::vector<double> h(fs);
        for (int j = 0; j < p.NY; ++j)
            for (int i = 0; i < p.nx; ++i)
                h[(size_t)j * p.nx + i] = i == 0 ? 0.0 : std::sin(0.37 * i) * std::cos(0.11 * j) + 1e-3 * ((i * 7 + j * 13) % 17);
        for (int b = 0; b < batch; ++b)
            TP_TRY(cudaMemcpy(dense + (size_t)b * fs, h.data(), sizeof(double) * fs, cudaMemcpyHostToDevice));
        TP_TRY(cudaMemset(buf, 0, sizeof(T) * fs * batch));
    }
    auto pass = [&](int k) -> iim_status {
        if (k == 0)
            return rows_fwd<T>(p, 0, p.NY, dense, p.nx, 1, nullptr, 0.0, nullptr, nullptr, kNoVec, 0.0, buf, nullptr,
                               cs, batch, fs, fs);
        if (k == 1) return cols<T>(p, 0, p.NY - 1, 0, p.NY - 1, buf, nullptr, cs, batch, fs);
        return rows_inv<T, INV_STORE_T>(p, 0, p.NY, buf, out, nullptr, 0, 0, nullptr, nullptr, cs, batch, fs);
    };
    const int launches[3] = {reps, reps, reps};
    for (int k = 0; k < 3 && st == IIM_OK; ++k) {
        // one uncaptured pass first: kernel attributes are set outside the capture
        iim_status ls = pass(k);
        TP_TRY(cudaStreamSynchronize(cs));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (ls == IIM_OK && st == IIM_OK) {
            TP_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            for (int r = 0; r < reps && ls == IIM_OK; ++r) ls = pass(k);
            TP_TRY(cudaStreamEndCapture(cs, &graph));
        }
        if (ls == IIM_OK && st == IIM_OK) TP_TRY(cudaGraphInstantiate(&exec, graph, 0));
        if (ls == IIM_OK && st == IIM_OK) {
            TP_TRY(cudaGraphLaunch(exec, cs));   // warm-up
            TP_TRY(cudaEventRecord(ev0, cs));
            TP_TRY(cudaGraphLaunch(exec, cs));
            TP_TRY(cudaEventRecord(ev1, cs));
            TP_TRY(cudaEventSynchronize(ev1));
            float ms = 0.f;
            TP_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
            us[k] = 1e3 * ms / launches[k];
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ls != IIM_OK && st == IIM_OK) st = ls;
    }
#undef TP_TRY
    if (st == IIM_OK) {
        const double e = (double)p.NY * p.NX;
        bytes[0] = e * (8.0 + sizeof(T)) * batch;
        bytes[1] = 2.0 * e * sizeof(T) * batch;
        bytes[2] = 2.0 * e * sizeof(T) * batch;
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaFree(buf);
    cudaFree(out);
    cudaFree(dense);
    return st;
}

extern "C" iim_status iim_time_box_passes(iim_geometry g, int prec, int batch, int reps, double* us, double* bytes) {
    if (!g || !us || !bytes || batch < 1 || reps < 1 || (prec != IIM_FP64 && prec != IIM_MIXED))
        return IIM_ERR_INVALID_ARG;
    cudaSetDevice(g->device);
    IIM_CHECK(ensure_twiddles());
    cudaStream_t cs = nullptr;
    IIM_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const iim_status st = prec == IIM_FP64 ? time_passes<double>(g, batch, reps, us, bytes, cs)
                                           : time_passes<float>(g, batch, reps, us, bytes, cs);
    cudaStreamDestroy(cs);
    return st;
}

// ------------------------------------------------------------------------- allocation-free box solve
// The same Dirichlet-box solve as iim_box_poisson, for callers that cannot allocate device
// memory.  Its scratch (the padded transform buffer followed by the eigenvalue tables) is the
// file-scope array below, which every GPU that loads the library keeps until the process
// exits.  All calls share it: calls that overlap on the GPU race.  Every call overwrites the
// whole region it uses before reading it, so no clearing is needed between calls.
namespace iim {
constexpr int kNoAllocMaxN = 1024;                                    // nx, ny <= 1024
constexpr size_t kNoAllocDoubles = (size_t)kNoAllocMaxN * (kNoAllocMaxN + 2);   // 8.4 MB
__device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[64];

// Eigenvalues of the 1D three-point operators (x modes, then y modes), in FP64 or FP32.
__global__ void k_box_eigs(int NX, int NY, int nx, int ny, double h, int as_float, double* lam) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NX + NY) return;
    const double v = k < NX ? (2.0 - 2.0 * cospi((double)(k + 1) / nx)) / (h * h)
                            : (2.0 - 2.0 * cospi((double)(k - NX + 1) / ny)) / (h * h);
    if (as_float) reinterpret_cast<float*>(lam)[k] = (float)v;
    else lam[k] = v;
}

// Shared-memory limits of every transform kernel the allocation-free solve may launch (all
// FFT paths), sized for the largest supported line.
template <typename T>
static iim_status allow_noalloc_smem() {
    const size_t rs = rows_smem<T>(kNoAllocMaxN), cs = cols_smem<T>(kNoAllocMaxN, 4);
    IIM_CHECK(allow_smem(k_rows_fwd<T, kRowWarps, 0>, rs));
    IIM_CHECK(allow_smem(k_rows_fwd<T, kRowWarps, 8>, rs));
    IIM_CHECK(allow_smem(k_rows_fwd<T, kRowWarps, 16>, rs));
    IIM_CHECK(allow_smem(k_cols<T, 4, 0>, cs));
    IIM_CHECK(allow_smem(k_cols<T, 4, 8>, cs));
    IIM_CHECK(allow_smem(k_cols<T, 4, 16>, cs));
    IIM_CHECK(allow_smem(k_rows_inv<T, kRowWarps, INV_STORE_F64, 0>, rs));
    IIM_CHECK(allow_smem(k_rows_inv<T, kRowWarps, INV_STORE_F64, 8>, rs));
    IIM_CHECK(allow_smem(k_rows_inv<T, kRowWarps, INV_STORE_F64, 16>, rs));
    return IIM_OK;
}

// Once per device, with that device current: twiddle tables, the device address of the
// static scratch, and the shared-memory limits of the transform kernels for the largest
// supported line, so that later calls touch nothing but their stream.  The set-up copies
// tables to the device, which a stream capture in progress would not allow: a first call on
// a device whose stream is capturing is refused (IIM_ERR_INVALID_ARG) before anything runs.
static iim_status noalloc_setup(cudaStream_t s, double** out) {
    int dev = 0;
    IIM_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return IIM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        IIM_TRY(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            snprintf(g_last_error, sizeof(g_last_error),
                     "iim_box_poisson_noalloc: the first call on device %d must come before any stream capture "
                     "(it sets up tables on the device)", dev);
            return IIM_ERR_INVALID_ARG;
        }
        IIM_CHECK(ensure_twiddles());
        void* p = nullptr;
        IIM_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        IIM_CHECK(allow_noalloc_smem<double>());
        IIM_CHECK(allow_noalloc_smem<float>());
        g_noalloc_ptr[dev] = (double*)p;
    }
    *out = g_noalloc_ptr[dev];
    return IIM_OK;
}
}  // namespace iim

extern "C" iim_status iim_box_poisson_noalloc(const iim_grid* grid, const double* f, const double* psi_box, double* u,
                                              int prec, iim_stream stream) {
    if (!grid || !f || !u) return IIM_ERR_INVALID_ARG;
    const int nx = grid->nx, ny = grid->ny;
    if (!is_pow2_in(nx, 16, 2048) || !is_pow2_in(ny, 16, 2048)) return IIM_ERR_INVALID_ARG;
    if (nx > kNoAllocMaxN || ny > kNoAllocMaxN) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "iim_box_poisson_noalloc: %d x %d cells exceed its static scratch (nx, ny <= %d)", nx, ny,
                 kNoAllocMaxN);
        return IIM_ERR_INVALID_ARG;
    }
    if (prec != IIM_FP64 && prec != IIM_MIXED) return IIM_ERR_INVALID_ARG;
    const double h = (grid->x1 - grid->x0) / nx;
    if (!(h > 0.0)) return IIM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double* scratch = nullptr;
    IIM_CHECK(noalloc_setup(s, &scratch));
    const int NX = nx - 1, NY = ny - 1;
    double* buf = scratch;                          // padded transform buffer, nx * NY
    double* lam = scratch + (size_t)nx * NY;        // NX + NY eigenvalues
    const double ih2 = 1.0 / (h * h);
    const int as_float = prec == IIM_MIXED;
    launch("box_eigs", 0.0, 0.0, k_box_eigs, (NX + NY + 255) / 256, 256, 0, s, NX, NY, nx, ny, h, as_float, lam);
    IIM_LAUNCHED();
    if (prec == IIM_FP64) {
        Plan<double> p{NX, NY, nx, ny, ilog2(nx), ilog2(ny), lam, lam + NX, twiddles64(), (2.0 / nx) * (2.0 / ny)};
        IIM_CHECK(rows_fwd<double>(p, 0, NY, f, NX, 0, psi_box, ih2, nullptr, nullptr, kNoVec, 0.0, buf, nullptr, s));
        IIM_CHECK(cols<double>(p, 0, NY - 1, 0, NY - 1, buf, nullptr, s));
        IIM_CHECK((rows_inv<double, INV_STORE_F64>(p, 0, NY, buf, nullptr, u, NX, 0, nullptr, nullptr, s)));
    } else {
        const float* lamf = reinterpret_cast<const float*>(lam);
        Plan<float> p{NX, NY, nx, ny, ilog2(nx), ilog2(ny), lamf, lamf + NX, twiddles32(),
                      (float)((2.0 / nx) * (2.0 / ny))};
        float* fb = reinterpret_cast<float*>(buf);
        IIM_CHECK(rows_fwd<float>(p, 0, NY, f, NX, 0, psi_box, ih2, nullptr, nullptr, kNoVec, 0.0, fb, nullptr, s));
        IIM_CHECK(cols<float>(p, 0, NY - 1, 0, NY - 1, fb, nullptr, s));
        IIM_CHECK((rows_inv<float, INV_STORE_F64>(p, 0, NY, fb, nullptr, u, NX, 0, nullptr, nullptr, s)));
    }
    return IIM_OK;
}

extern "C" const char* iim_last_error_message(void) { return g_last_error; }

extern "C" const char* iim_status_string(iim_status st) {
    switch (st) {
        case IIM_OK: return "IIM_OK";
        case IIM_ERR_INVALID_ARG: return "IIM_ERR_INVALID_ARG";
        case IIM_ERR_UNDERRESOLVED: return "IIM_ERR_UNDERRESOLVED";
        case IIM_ERR_BAD_REGION: return "IIM_ERR_BAD_REGION";
        case IIM_ERR_NONFINITE: return "IIM_ERR_NONFINITE";
        case IIM_ERR_NOT_CONVERGED: return "IIM_ERR_NOT_CONVERGED";
        case IIM_ERR_TIMEOUT: return "IIM_ERR_TIMEOUT";
        case IIM_ERR_CUDA: return "IIM_ERR_CUDA";
        default: return "IIM_UNKNOWN_STATUS";
    }
}
