// Lockstep batched IIM Poisson solves: many independent problems of one grid size advance
// through the solve of Sec. 4.2 together, one kernel launch per step for all of them.
//
// The single-problem solve (solve.cu) runs its refinement loop, GMRES cycles and iterations as
// one device-driven graph per problem.  Here the same sequence is built once for a group of
// problems that share (nx, ny) and the transform settings: every kernel takes the group's
// problem table and works on problem blockIdx.z, so one launch of the column pass transforms
// the columns of every problem in flight (eight 1024^2 problems: 8 x 128 blocks instead of
// 128, enough to fill the GPU), and the loops are WHILE / IF graph nodes that continue while
// any problem still needs them.  Each problem keeps its own loop state in its geometry's
// device counters; two extra flags say whether it is still refining (DI_RACT) and whether it
// is inside a GMRES cycle (DI_CACT), and every kernel of a loop body is a no-op for a problem
// whose flag is clear.  The kernels call the same device bodies as the single-problem kernels
// (iim_ops.cuh, dst.cuh) with the same per-problem grid extents, so each problem gets exactly
// the arithmetic, in the same order, of its own solve: the results are bitwise equal.
//
// Scope: problems whose geometry has had one solve already (preconditioner, capacitance
// responses and Krylov buffers in place), right-preconditioned GMRES (iim_opts.precond 1, or 3
// with the dense Schur matrix as the inner operator), no initial guess.  Other problems take the per-problem path of batched.cu.
//
// The same step sequence also runs host-driven (each loop decision read back by the host),
// which is how the per-kernel profiler times the batched kernels one launch at a time.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "dst.cuh"
#include "iim_ops.cuh"

namespace iim {

// per-problem flags in the geometry's device counters (next to the DI_* of iim_ops.cuh)
enum { DI_RACT = 16, DI_CACT = 17 };

// which problems a launch works on
enum LsGate { G_ALL = 0, G_REF = 1, G_CYC = 2, G_IT = 3, G_CAP = 4 };

// Everything one problem's kernels read: geometry, workspace and the call's arguments.
struct LsProb {
    int NX, NY, nx, na, ns, nminus, ncirc, nb, ja0, ja1, jo0, jo1, cap;
    double h, ih2;
    const int *aff_row_ptr, *aff_node, *gop_ptr, *gop_idx, *cp_body, *body_circ, *aff_body;
    const double* gop_w;
    const int *minus_node, *gh_ptr, *gh_idx;
    const double* gh_w;
    const uint8_t* cls;
    const iim_region* regions;
    const void* lam_x;
    const void* lam_y;
    double *psi_ext, *res, *partial, *small, *V, *H, *xsol, *bvec, *pc_z;
    void* tbuf;
    void* psiT;
    const float* pc_inv;   // right half of [S | S^-1], leading dimension 2 ns
    const float* pc_S;     // S itself (ns x ns), the inner operator of iim_opts.precond == 3
    ScanTab<float> s32;    // factors of the tridiagonal column pass (used when the group's tri is set)
    ScanTab<double> s64;
    int* di;
    const double *cap_psi, *cap_dev;
    const double *omega, *psi_b, *ring, *gamma;
    double *psibar, *psi_out, *ux_out, *uy_out;
};

// Per-problem record gathered at the end of a solve (one device-to-host copy for the group).
struct LsRec {
    int di[16];
    double rel, circ_err, scal[4];
};

__device__ __forceinline__ bool ls_off(const LsProb& p, int gate) {
    switch (gate) {
        case G_REF: return p.di[DI_RACT] == 0;
        case G_CYC: return p.di[DI_CACT] == 0;
        case G_IT: return p.di[DI_STOP] != 0;
        case G_CAP: return p.ncirc == 0 || !p.cap;
        default: return false;
    }
}

// ------------------------------------------------------------------------- transform kernels
// Row / column pass modes: the right-hand side (dense residual in, rows the gather reads out),
// the Schur operator on the preconditioned vector (iteration) or on V_1 (restart), and the
// recovery of psi from the residual and the corrections.
enum LsMode { M_RHS = 0, M_APPLY_PCZ = 1, M_APPLY_VTMP = 2, M_RECOVER = 3 };

__device__ __forceinline__ VecArg ls_vec(const LsProb& p, int mode) {
    if (mode == M_APPLY_PCZ) return VecArg{p.pc_z, nullptr, 0, 0};
    if (mode == M_APPLY_VTMP) return VecArg{p.V, p.di + DI_TMPJ, 0, (long)p.ns};
    if (mode == M_RECOVER) return VecArg{p.na ? p.xsol : nullptr, nullptr, 0, 0};
    return VecArg{nullptr, nullptr, 0, 0};
}

template <typename T, int WARPS, int FP>
__global__ void __launch_bounds__(WARPS * 32)
kb_rows_fwd(const LsProb* __restrict__ P, int mode, int gate, const cpx<T>* __restrict__ tw) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate) || (mode != M_RECOVER && p.na == 0)) return;
    constexpr int LPB = WARPS * 32 / line_threads(FP);
    const bool dense = mode == M_RHS || mode == M_RECOVER;
    const int row0 = dense ? 0 : p.ja0, nrows = dense ? p.NY : p.ja1 - p.ja0 + 1;
    if ((int)blockIdx.x * LPB >= nrows) return;   // uniform over the block
    rows_fwd_body<T, WARPS, FP>(p.NX, p.NY, p.nx, __ffs(p.nx) - 1, row0, nrows, dense ? p.res : nullptr, p.nx, 1,
                                nullptr, 0.0, mode == M_RHS ? nullptr : p.aff_row_ptr,
                                mode == M_RHS ? nullptr : p.aff_node, ls_vec(p, mode), mode == M_RECOVER ? -1.0 : 1.0,
                                tw, (T*)p.tbuf);
}

template <typename T, int C, int FP>
__global__ void __launch_bounds__(C * line_threads(FP), sizeof(T) == 4 ? 2 : 1)
kb_cols(const LsProb* __restrict__ P, int mode, int gate, T norm, const cpx<T>* __restrict__ tw) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate) || (mode != M_RECOVER && p.na == 0)) return;
    int in0 = 0, in1 = p.NY - 1, out0 = p.jo0, out1 = p.jo1;
    if (mode == M_APPLY_PCZ || mode == M_APPLY_VTMP) { in0 = p.ja0; in1 = p.ja1; }
    if (mode == M_RECOVER) { out0 = 0; out1 = p.NY - 1; }
    cols_body<T, C, FP>(p.NX, p.NY, p.NY + 1, __ffs(p.NY + 1) - 1, in0, in1, out0, out1, (T*)p.tbuf,
                        (const T*)p.lam_x, (const T*)p.lam_y, norm, tw);
}

template <typename T>
__device__ __forceinline__ const ScanTab<T>& ls_scan(const LsProb& p) {
    if constexpr (sizeof(T) == 4) return p.s32;
    else return p.s64;
}

template <typename T, int CW, int NT>
__global__ void __launch_bounds__(NT, NT == 1024 ? 2 : 4) kb_cols_scan(const LsProb* __restrict__ P, int mode, int gate) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate) || (mode != M_RECOVER && p.na == 0)) return;
    int in0 = 0, in1 = p.NY - 1, out0 = p.jo0, out1 = p.jo1;
    if (mode == M_APPLY_PCZ || mode == M_APPLY_VTMP) { in0 = p.ja0; in1 = p.ja1; }
    if (mode == M_RECOVER) { out0 = 0; out1 = p.NY - 1; }
    cols_scan_body<T, CW, NT>(p.NX, p.NY, p.nx, in0, in1, out0, out1, (T*)p.tbuf, ls_scan<T>(p));
}

template <typename T, int WARPS, int MODE, int FP>
__global__ void __launch_bounds__(WARPS * 32)
kb_rows_inv(const LsProb* __restrict__ P, int gate, const cpx<T>* __restrict__ tw) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate) || (MODE == INV_STORE_T && p.na == 0)) return;
    constexpr int LPB = WARPS * 32 / line_threads(FP);
    const int row0 = MODE == INV_STORE_T ? p.jo0 : 0, nrows = MODE == INV_STORE_T ? p.jo1 - p.jo0 + 1 : p.NY;
    if ((int)blockIdx.x * LPB >= nrows) return;
    rows_inv_body<T, WARPS, MODE, FP>(p.NX, p.NY, p.nx, __ffs(p.nx) - 1, row0, nrows, (const T*)p.tbuf,
                                      MODE == INV_STORE_T ? (T*)p.psiT : nullptr,
                                      MODE == INV_STORE_T ? nullptr : p.psi_ext, 0, 0, p.cls, tw);
}

// gamma-space gathers: the right-hand side b (no input vector, grid = gather blocks only) or
// the Schur operator's output column (+ circulation rows) of the iteration / restart.
template <typename T, int BLOCK>
__global__ void __launch_bounds__(BLOCK) kb_gather(const LsProb* __restrict__ P, int mode, int gate) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate)) return;
    const int nga = (p.na + BLOCK / 32 - 1) / (BLOCK / 32);
    if (mode == M_RHS) {
        if (p.na == 0 || (int)blockIdx.x >= nga) return;
        gather_body<T, BLOCK>(p.na, nga, p.gop_ptr, p.gop_idx, p.gop_w, (const T*)p.psiT, p.cp_body, p.body_circ,
                              p.aff_body, VecArg{nullptr, nullptr, 0, 0}, 0, p.bvec, nullptr, 0L, nullptr);
        return;
    }
    if ((int)blockIdx.x >= nga + p.ncirc) return;
    const int* jidx = p.di + (mode == M_APPLY_PCZ ? DI_J : DI_TMPJ);
    gather_body<T, BLOCK>(p.na, nga, p.gop_ptr, p.gop_idx, p.gop_w, (const T*)p.psiT, p.cp_body, p.body_circ,
                          p.aff_body, ls_vec(p, mode), 1, p.V, jidx, (long)p.ns, nullptr);
}

// Dense products: z = M V_j (iteration, skipped once the problem's GMRES stopped), x += M t
// (cycle end), and with the dense inner operator V_{j+1} = S z (iteration) or V_2 = S V_1
// (restart).
enum { MV_PRECOND = 0, MV_XUPDATE = 1, MV_S_ITER = 2, MV_S_RESTART = 3 };
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) kb_matvec(const LsProb* __restrict__ P, int op, int gate) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate) || p.ns == 0) return;
    const long ns = p.ns;
    if (op == MV_PRECOND)
        dense_matvec4_body<WARPS>(p.ns, p.pc_inv, 2L * ns, p.V, p.di + DI_J, ns, p.pc_z, 0, p.di + DI_STOP);
    else if (op == MV_XUPDATE)
        dense_matvec4_body<WARPS>(p.ns, p.pc_inv, 2L * ns, p.pc_z + ns, nullptr, 0L, p.xsol, 1, nullptr);
    else if (op == MV_S_ITER)
        dense_matvec4_body<WARPS>(p.ns, p.pc_S, ns, p.pc_z, nullptr, 0L, p.V, 0, p.di + DI_STOP, p.di + DI_J, ns);
    else
        dense_matvec4_body<WARPS>(p.ns, p.pc_S, ns, p.V + ns, nullptr, 0L, p.V, 0, nullptr, p.di + DI_TMPJ, ns);
}

// ------------------------------------------------------------------------- Krylov kernels
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) kb_arnoldi(const LsProb* __restrict__ P, KLayout L) {
    const LsProb& p = P[blockIdx.z];
    if (p.ns == 0) return;
    arnoldi_block_body<BLOCK>(p.di, p.V, (long)p.ns, p.ns, L, p.H);
}

// GMRES start of a correction (restart = 0: ||b||, counters, tolerance, V_0 = b / ||b||; a
// problem that is no longer refining, or has no Krylov unknowns, only gets its stop flag) or
// of a restart cycle (V_0 = (b - S x) / ||b - S x||).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
kb_start(const LsProb* __restrict__ P, KLayout L, int restart, int max_iter, double tol) {
    const LsProb& p = P[blockIdx.z];
    if (!restart) {
        if (!p.di[DI_RACT] || p.ns == 0) {
            if (threadIdx.x == 0) p.di[DI_STOP] = 1;
            return;
        }
        start_block_body<BLOCK>(p.ns, p.bvec, p.V, L, p.H, p.di, max_iter, tol, p.small + SM_NORM);
    } else {
        if (!p.di[DI_CACT]) return;
        start_block_body<BLOCK>(p.ns, p.V + 2L * p.ns, p.V, L, p.H, p.di, -1, 0.0, nullptr);
    }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) kb_backsolve(const LsProb* __restrict__ P, KLayout L) {
    const LsProb& p = P[blockIdx.z];
    if (!p.di[DI_CACT]) return;
    backsolve_update_body<BLOCK>(p.di, L, p.H, p.V, (long)p.ns, p.ns, p.pc_z + p.ns, 0);
}

// Small vector steps: x = 0 at the start of a correction; V_1 = x and the scratch column index
// before the restart's operator application; V_2 = b - V_2 after it.
enum { V_ZERO_X = 0, V_RESTART_PREP = 1, V_RESTART_RES = 2 };
__global__ void kb_vec(const LsProb* __restrict__ P, int op, int gate) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate)) return;
    const long ns = p.ns;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (op == V_RESTART_PREP && e == 0) p.di[DI_TMPJ] = 1;
    if (e >= ns) return;
    if (op == V_ZERO_X) p.xsol[e] = 0.0;
    else if (op == V_RESTART_PREP) p.V[ns + e] = p.xsol[e];
    else p.V[2 * ns + e] = 1.0 * p.bvec[e] + -1.0 * p.V[2 * ns + e];
}

// ------------------------------------------------------------------------- field kernels
__global__ void kb_init(const LsProb* __restrict__ P) {
    const LsProb& p = P[blockIdx.z];
    if ((long)blockIdx.x * blockDim.x >= (long)p.nx * p.NY) return;
    init_psi_body(p.NX, p.NY, nullptr, p.cls, p.psi_ext);
}

__global__ void kb_init_psibar(const LsProb* __restrict__ P) {
    const LsProb& p = P[blockIdx.z];
    if (p.nb > 0) init_psibar_body(p.nb, p.body_circ, p.psibar, 0, p.psibar);
}

__global__ void kb_ghost(const LsProb* __restrict__ P, int gate) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate) || p.nminus == 0) return;
    ghost_body(p.nminus, p.minus_node, p.gh_ptr, p.gh_idx, p.gh_w, p.psi_b, p.psibar, p.cp_body, p.psi_ext);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) kb_residual(const LsProb* __restrict__ P, int gate) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate)) return;
    residual_body<BLOCK>(p.NX, p.NY, p.ih2, p.psi_ext, p.omega, p.cls, p.ring, p.res, p.partial);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) kb_circ_measure(const LsProb* __restrict__ P, int gate) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate) || (int)blockIdx.x >= p.ncirc) return;
    circ_measure_body<BLOCK>(p.nx, p.psi_ext, p.regions, p.di + DI_CIRC, p.small + SM_CIRC);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) kb_region_sums(const LsProb* __restrict__ P, int gate) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate) || (int)blockIdx.x >= p.ncirc) return;
    region_sums_body<BLOCK>(p.nx, p.res, p.regions, p.di + DI_CIRC, p.small + SM_REG);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) kb_finish_residual(const LsProb* __restrict__ P, int gate, int nparts) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate)) return;
    finish_residual_body<BLOCK>(nparts, p.partial, p.ncirc, p.di + DI_CIRC, p.gamma, p.ih2, p.small, p.small + SM_REG,
                                p.bvec ? p.bvec + p.na : nullptr, p.small + SM_RES2);
}

// psibar += the circulation part of the correction (from_cap = 0) or of the capacitance step
__global__ void kb_add_psibar(const LsProb* __restrict__ P, int from_cap, int gate) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, gate) || p.ncirc == 0) return;
    add_psibar_body(p.ncirc, p.di + DI_CIRC, from_cap ? p.small + SM_CAPP : p.xsol + p.na, p.psibar);
}

__global__ void kb_cap_coef(const LsProb* __restrict__ P) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, G_CAP)) return;
    const int nc = p.ncirc;
    cap_coef_body(nc, p.small + SM_RC, p.cap_dev, p.cap_dev + (size_t)nc * nc, p.h * p.h, p.small + SM_CAPC,
                  p.small + SM_CAPP);
}

__global__ void kb_cap_update(const LsProb* __restrict__ P) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, G_CAP)) return;
    cap_update_body((long)p.nx * p.NY, p.ncirc, p.cap_psi, p.small + SM_CAPC, p.psi_ext);
}

__global__ void kb_final_rel(const LsProb* __restrict__ P) {
    const LsProb& p = P[blockIdx.z];
    if (ls_off(p, G_CAP)) return;
    final_rel_body(p.di, p.small);
}

__global__ void kb_velocity(const LsProb* __restrict__ P) {
    const LsProb& p = P[blockIdx.z];
    if ((long)blockIdx.x * blockDim.x >= (long)p.NX * p.NY) return;
    velocity_body(p.NX, p.NY, 0.5 / p.h, p.psi_ext, p.cls, p.ring, p.psi_out, p.ux_out, p.uy_out);
}

__global__ void kb_records(const LsProb* __restrict__ P, int n, KLayout L, LsRec* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const LsProb& p = P[k];
    for (int i = 0; i < 16; ++i) out[k].di[i] = p.di[i];
    out[k].rel = p.small[SM_REL];
    out[k].circ_err = p.small[SM_CIRC_ERR];
    for (int i = 0; i < 4; ++i) out[k].scal[i] = p.H[L.scal() + i];
}

// ------------------------------------------------------------------------- loop control
// One block, one thread per problem.  Each kernel applies the single-problem control kernel's
// rule to every problem still inside the loop, then continues the loop (graph conditional, or
// *flag for the host-driven form) while any problem needs it.  cnt[] counts body executions:
// [0] refinements, [1] cycles, [2] iterations, [3] restarts.
__device__ __forceinline__ void ls_decide(int any, cudaGraphConditionalHandle h, int* flag) {
    if (threadIdx.x == 0) {
        if (flag) *flag = any;
        else cudaGraphSetConditional(h, any ? 1 : 0);
    }
}

__global__ void kb_ref_init(const LsProb* __restrict__ P, int n, double rtol, cudaGraphConditionalHandle h, int* flag,
                            int* cnt) {
    int go_any = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int* di = P[k].di;
        double* small = P[k].small;
        const double r2 = small[SM_RES2];
        const double fn = sqrt(r2);
        small[SM_FNORM] = fn;
        small[SM_REL] = fn > 0.0 ? 1.0 : 0.0;
        di[DI_REF] = 0; di[DI_ITS] = 0; di[DI_FIRST] = 0; di[DI_CYCERR] = 0; di[DI_CYCS] = 0; di[DI_RSS] = 0;
        di[DI_LOOPERR] = 0;
        const bool fin = isfinite(r2);
        di[DI_NONFIN] = fin ? 0 : 1;
        const int go = (fin && fn > 0.0 && 1.0 > rtol) ? 1 : 0;
        di[DI_RACT] = go;
        di[DI_CACT] = 0;
        di[DI_STOP] = 1;
        go_any |= go;
    }
    if (threadIdx.x == 0 && cnt) cnt[0] = cnt[1] = cnt[2] = cnt[3] = 0;
    ls_decide(__syncthreads_or(go_any), h, flag);
}

__global__ void kb_cyc_begin(const LsProb* __restrict__ P, int n, int max_iter, cudaGraphConditionalHandle h,
                             int* flag) {
    int any = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int* di = P[k].di;
        int act = 0;
        if (di[DI_RACT] && P[k].ns > 0) {
            const int left = max_iter - di[DI_ITS];
            di[DI_MAXIT] = left > 1 ? left : 1;
            di[DI_CYC] = 0;
            if (di[DI_IT] >= di[DI_MAXIT]) di[DI_STOP] = 1;
            act = di[DI_STOP] ? 0 : 1;
        } else {
            di[DI_STOP] = 1;
        }
        di[DI_CACT] = act;
        any |= act;
    }
    ls_decide(__syncthreads_or(any), h, flag);
}

__global__ void kb_it_begin(const LsProb* __restrict__ P, int n, cudaGraphConditionalHandle h, int* flag) {
    int any = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int* di = P[k].di;
        if (di[DI_CACT]) {
            di[DI_LOOP] = 0;
            any |= di[DI_STOP] ? 0 : 1;
        }
    }
    ls_decide(__syncthreads_or(any), h, flag);
}

__global__ void kb_loop_ctl(const LsProb* __restrict__ P, int n, int cap, cudaGraphConditionalHandle h, int* flag,
                            int* cnt) {
    int any = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int* di = P[k].di;
        if (di[DI_CACT] && !di[DI_STOP]) {
            const int c = ++di[DI_LOOP];
            if (c >= cap) {
                di[DI_STOP] = 1;
                di[DI_LOOPERR] = 1;
            }
        }
        any |= di[DI_STOP] ? 0 : 1;
    }
    if (threadIdx.x == 0 && cnt) ++cnt[2];
    ls_decide(__syncthreads_or(any), h, flag);
}

__global__ void kb_cyc_ctl(const LsProb* __restrict__ P, int n, int cap, cudaGraphConditionalHandle hc,
                           cudaGraphConditionalHandle hr, int* flag, int* cnt) {
    int any = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int* di = P[k].di;
        if (!di[DI_CACT]) continue;
        const int c = ++di[DI_CYC];
        ++di[DI_CYCS];
        bool done = di[DI_CONV] || di[DI_IT] >= di[DI_MAXIT] || di[DI_LOOPERR];
        if (!done && c >= cap) {
            done = true;
            di[DI_CYCERR] = 1;
        }
        if (!done) ++di[DI_RSS];
        di[DI_CACT] = done ? 0 : 1;
        any |= done ? 0 : 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        if (cnt) {
            ++cnt[1];
            if (any) ++cnt[3];
        }
        if (flag) *flag = any;
        else {
            cudaGraphSetConditional(hc, any ? 1 : 0);
            cudaGraphSetConditional(hr, any ? 1 : 0);
        }
    }
}

__global__ void kb_ref_ctl(const LsProb* __restrict__ P, int n, double rtol, int max_refine, int max_iter,
                           cudaGraphConditionalHandle h, int* flag, int* cnt) {
    int any = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int* di = P[k].di;
        if (!di[DI_RACT]) continue;
        double* small = P[k].small;
        if (di[DI_REF] == 0) di[DI_FIRST] = di[DI_IT];
        di[DI_ITS] += di[DI_IT];
        const int r = ++di[DI_REF];
        const double r2 = small[SM_RES2], fn = small[SM_FNORM];
        const bool fin = isfinite(r2);
        if (!fin) di[DI_NONFIN] = 1;
        const double rel = fn > 0.0 ? sqrt(r2) / fn : 0.0;
        small[SM_REL] = rel;
        const bool go = fin && rel > rtol && r < max_refine && di[DI_ITS] < max_iter && !di[DI_LOOPERR] &&
                        !di[DI_CYCERR];
        di[DI_RACT] = go ? 1 : 0;
        any |= go ? 1 : 0;
    }
    if (threadIdx.x == 0 && cnt) ++cnt[0];
    ls_decide(__syncthreads_or(any), h, flag);
}

// ------------------------------------------------------------------------- the group
struct LsGroup {
    std::vector<iim_geometry> geos;
    int prec = 0, m = 0, max_refine = 0, max_iter = 0, cap = 0, dense = 0;
    double rtol = 0.0, inner = 0.0;
    int nx = 0, ny = 0, NX = 0, NY = 0, wide = 0, cols_c = 4, tri = 0;
    // launch extents: maxima over the group
    int max_na = 0, max_ns = 0, max_nminus = 0, max_ncirc = 0, max_ja_rows = 0, max_jo_rows = 0;
    LsProb* d_probs = nullptr;
    LsProb* h_probs = nullptr;   // pinned
    LsRec* d_rec = nullptr;
    LsRec* h_rec = nullptr;      // pinned
    int* d_cnt = nullptr;        // body-execution counters, then the host-driven loop flag
    int* h_cnt = nullptr;        // pinned
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    long long k_top = 0, k_ref = 0, k_cyc = 0, k_it = 0, k_rs = 0;
    int n() const { return (int)geos.size(); }

    ~LsGroup() {
        if (exec) cudaGraphExecDestroy(exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        cudaFree(d_probs);
        cudaFree(d_rec);
        cudaFree(d_cnt);
        cudaFreeHost(h_probs);
        cudaFreeHost(h_rec);
        cudaFreeHost(h_cnt);
    }
};

static std::mutex g_ls_mutex;
static std::vector<LsGroup*> g_ls_groups;

// A destroyed geometry takes every group it belongs to with it.
void lockstep_forget(iim_geometry g) {
    std::lock_guard<std::mutex> lock(g_ls_mutex);
    for (size_t i = 0; i < g_ls_groups.size();) {
        LsGroup* G = g_ls_groups[i];
        if (std::find(G->geos.begin(), G->geos.end(), g) != G->geos.end()) {
            delete G;
            g_ls_groups.erase(g_ls_groups.begin() + i);
        } else {
            ++i;
        }
    }
}

static std::atomic<int> g_ls_group{4};

int lockstep_group_size() { return g_ls_group.load(); }

// Problems that can join a lockstep group under these options.
bool lockstep_eligible(iim_geometry g, const iim_opts& o) {
    const int ns = g->na + g->ncirc;
    return g_ls_group.load() >= 2 && g->host_solves > 0 && !g->solve_graph_failed && o.guess == 0 && !g->outer &&
           (o.precond == 1 || (o.precond == 3 && g->pc_S)) && ns > 0 && g->pc_ready &&
           g->V && g->krylov_m >= o.restart && (g->ncirc == 0 || g->cap_ready) &&
           sizeof(float) * 4 * (size_t)((ns + 3) & ~3) <= 200 * 1024;
}

static void fill_prob(LsProb& q, iim_geometry g, int prec, const double* omega, const double* psi_b,
                      const double* ring, const double* gamma, double* psibar, double* psi_out, double* ux,
                      double* uy) {
    std::memset(&q, 0, sizeof(q));
    q.NX = g->NX; q.NY = g->NY; q.nx = g->nx; q.na = g->na; q.ns = g->na + g->ncirc; q.nminus = g->nminus;
    q.ncirc = g->ncirc; q.nb = g->nb; q.ja0 = g->ja0; q.ja1 = g->ja1; q.jo0 = g->jo0; q.jo1 = g->jo1;
    q.cap = g->ncirc > 0 && g->cap_ready;
    q.h = g->h; q.ih2 = 1.0 / (g->h * g->h);
    q.aff_row_ptr = g->aff_row_ptr; q.aff_node = g->aff_node; q.gop_ptr = g->gop_ptr; q.gop_idx = g->gop_idx;
    q.cp_body = g->cp_body; q.body_circ = g->body_circ; q.aff_body = g->aff_body; q.gop_w = g->gop_w;
    q.minus_node = g->minus_node; q.gh_ptr = g->gh_ptr; q.gh_idx = g->gh_idx; q.gh_w = g->gh_w;
    q.cls = g->node_class; q.regions = g->d_regions;
    q.lam_x = prec == IIM_FP64 ? (const void*)g->lam_x64 : (const void*)g->lam_x32;
    q.lam_y = prec == IIM_FP64 ? (const void*)g->lam_y64 : (const void*)g->lam_y32;
    q.psi_ext = g->psi_ext; q.res = g->res; q.partial = g->partial; q.small = g->small; q.V = g->V; q.H = g->H;
    q.xsol = g->xsol; q.bvec = g->bvec; q.pc_z = g->pc_z; q.tbuf = g->tbuf; q.psiT = g->psiT;
    q.pc_inv = g->pc_aug + (q.ns);
    q.pc_S = g->pc_S;
    if (g->col_solver == 1) {
        q.s32 = ScanTab<float>{g->sc32_delta, g->sc32_rowoff, g->sc32_par, g->sc32_lim, g->sc32_dstar,
                               (float)(g->h * g->h * (2.0 / g->nx))};
        q.s64 = ScanTab<double>{g->sc64_delta, g->sc64_rowoff, nullptr, g->sc64_lim, g->sc64_dstar, g->h * g->h * (2.0 / g->nx)};
    }
    q.di = g->d_int;
    q.cap_psi = g->cap_psi; q.cap_dev = g->cap_dev;
    if (g->wall == 1 && g->psibar_zero) psibar = g->psibar_zero;   // a Neumann wall has no body constants
    q.omega = omega; q.psi_b = psi_b; q.ring = ring; q.gamma = gamma; q.psibar = psibar; q.psi_out = psi_out;
    q.ux_out = ux; q.uy_out = uy;
}

// ---- the step sequence, emitted into a graph capture or run host-driven
struct LsEmit {
    LsGroup* G;
    cudaStream_t s;
    bool host;   // host-driven: control kernels write *flag, the host reads it
    int* flag() const { return host ? G->d_cnt + 8 : nullptr; }
    int* cnt() const { return host ? nullptr : G->d_cnt; }
    dim3 grid(long x) const { return dim3((unsigned)std::max<long>(x, 1), 1, (unsigned)G->n()); }

    // algorithmic bytes of a launch summed over the group (the per-kernel profiler's figure)
    double sum_rows(int which, double per_row) const {
        double b = 0.0;
        for (iim_geometry g : G->geos)
            b += per_row * (which == 0 ? g->NY : which == 1 ? g->ja1 - g->ja0 + 1 : g->jo1 - g->jo0 + 1);
        return b;
    }

    template <typename T>
    iim_status rows_fwd(int mode, int gate) {
        const size_t sm = rows_smem<T>(G->nx);
        const int rpb = rows_per_block(G->nx, G->wide);
        const bool dense = mode == M_RHS || mode == M_RECOVER;
        const int rows = dense ? G->NY : G->max_ja_rows;
        const double bytes = sum_rows(dense ? 0 : 1, G->NX * ((dense ? 8.0 : 0.0) + sizeof(T)));
        auto go = [&](auto kern) -> iim_status {
            IIM_CHECK(allow_smem(kern, sm));
            launch(sizeof(T) == 8 ? "ls_rows_fwd_f64" : "ls_rows_fwd_f32", bytes, 0.0, kern,
                   grid((rows + rpb - 1) / rpb), kRowWarps * 32, sm, s, (const LsProb*)G->d_probs, mode, gate,
                   twiddle_region<T>(G->nx, fft_path(G->nx, G->wide)));
            return IIM_OK;
        };
        const int fp = fft_path(G->nx, G->wide);
        if (fp == 64) IIM_CHECK(go(kb_rows_fwd<T, kRowWarps, 64>));
        else if (fp == 16) IIM_CHECK(go(kb_rows_fwd<T, kRowWarps, 16>));
        else if (fp == 8) IIM_CHECK(go(kb_rows_fwd<T, kRowWarps, 8>));
        else IIM_CHECK(go(kb_rows_fwd<T, kRowWarps, 0>));
        IIM_LAUNCHED();
        return IIM_OK;
    }

    template <typename T, int C>
    iim_status cols_c(int mode, int gate) {
        const size_t sm = cols_smem<T>(G->ny, C);
        const T norm = (T)((2.0 / G->nx) * (2.0 / G->ny));
        double bytes = 0.0;
        for (iim_geometry g : G->geos) {
            int in = g->NY, out = g->jo1 - g->jo0 + 1;
            if (mode == M_APPLY_PCZ || mode == M_APPLY_VTMP) in = g->ja1 - g->ja0 + 1;
            if (mode == M_RECOVER) out = g->NY;
            bytes += (double)(in + out) * g->NX * sizeof(T);
        }
        auto go = [&](auto kern) -> iim_status {
            IIM_CHECK(allow_smem(kern, sm));
            launch(sizeof(T) == 8 ? "ls_cols_f64" : "ls_cols_f32", bytes, 0.0, kern,
                   dim3(G->nx / C, 1, G->n()), C * line_threads(fft_path(G->ny, G->wide)), sm, s,
                   (const LsProb*)G->d_probs, mode, gate, norm, twiddle_region<T>(G->ny, fft_path(G->ny, G->wide)));
            return IIM_OK;
        };
        const int fp = fft_path(G->ny, G->wide);
        if (fp == 64) IIM_CHECK(go(kb_cols<T, C, 64>));
        else if (fp == 16) IIM_CHECK(go(kb_cols<T, C, 16>));
        else if (fp == 8) IIM_CHECK(go(kb_cols<T, C, 8>));
        else IIM_CHECK(go(kb_cols<T, C, 0>));
        IIM_LAUNCHED();
        return IIM_OK;
    }

    template <typename T>
    iim_status cols(int mode, int gate) {
        if (G->tri) {
            double bytes = 0.0;
            for (iim_geometry g : G->geos) {
                int in = g->NY, out = g->jo1 - g->jo0 + 1;
                if (mode == M_APPLY_PCZ || mode == M_APPLY_VTMP) in = g->ja1 - g->ja0 + 1;
                if (mode == M_RECOVER) out = g->NY;
                bytes += (double)(in + out) * g->NX * sizeof(T);
            }
            constexpr int CW = 32 / sizeof(T);
            auto go = [&](auto kern, int NT, size_t sm) -> iim_status {
                IIM_CHECK(allow_smem(kern, sm));
                launch(sizeof(T) == 8 ? "ls_tri_cols_f64" : "ls_tri_cols_f32", bytes, 0.0, kern,
                       dim3(G->nx / CW, 1, G->n()), NT, sm, s, (const LsProb*)G->d_probs, mode, gate);
                return IIM_OK;
            };
            bool wide = false;
            if constexpr (sizeof(T) == 4) {   // FP64 keeps 256 threads (bound by FP64 arithmetic)
                wide = scan_threads(G->NY, (long)(G->nx / CW) * G->n(), sm_count()) == 1024;
                if (wide) IIM_CHECK(go(kb_cols_scan<T, CW, 1024>, 1024, scan_smem<T, CW, 1024>(G->NY)));
            }
            if (!wide) IIM_CHECK(go(kb_cols_scan<T, CW, 256>, 256, scan_smem<T, CW, 256>(G->NY)));
            IIM_LAUNCHED();
            return IIM_OK;
        }
        const int C = tile_width<T>(G->cols_c);
        if (C == 8) return cols_c<T, (sizeof(T) == 4 ? 8 : 4)>(mode, gate);
        if (C == 2) return cols_c<T, (sizeof(T) == 8 ? 2 : 4)>(mode, gate);
        return cols_c<T, 4>(mode, gate);
    }

    template <typename T, int MODE>
    iim_status rows_inv(int gate) {
        const size_t sm = rows_smem<T>(G->nx);
        const int rpb = rows_per_block(G->nx, G->wide);
        const int rows = MODE == INV_STORE_T ? G->max_jo_rows : G->NY;
        const double bytes = sum_rows(MODE == INV_STORE_T ? 2 : 0, G->NX * (sizeof(T) + (MODE == INV_STORE_T ? sizeof(T) : 17.0)));
        auto go = [&](auto kern) -> iim_status {
            IIM_CHECK(allow_smem(kern, sm));
            launch(sizeof(T) == 8 ? "ls_rows_inv_f64" : "ls_rows_inv_f32", bytes, 0.0, kern,
                   grid((rows + rpb - 1) / rpb), kRowWarps * 32, sm, s, (const LsProb*)G->d_probs, gate,
                   twiddle_region<T>(G->nx, fft_path(G->nx, G->wide)));
            return IIM_OK;
        };
        const int fp = fft_path(G->nx, G->wide);
        if (fp == 64) IIM_CHECK(go(kb_rows_inv<T, kRowWarps, MODE, 64>));
        else if (fp == 16) IIM_CHECK(go(kb_rows_inv<T, kRowWarps, MODE, 16>));
        else if (fp == 8) IIM_CHECK(go(kb_rows_inv<T, kRowWarps, MODE, 8>));
        else IIM_CHECK(go(kb_rows_inv<T, kRowWarps, MODE, 0>));
        IIM_LAUNCHED();
        return IIM_OK;
    }

    template <typename T>
    iim_status gather(int mode, int gate) {
        const int nga = (G->max_na + 3) / 4;
        launch("ls_gather", 0.0, 0.0, kb_gather<T, 128>, grid(mode == M_RHS ? nga : nga + G->max_ncirc), 128, 0, s,
               (const LsProb*)G->d_probs, mode, gate);
        IIM_LAUNCHED();
        return IIM_OK;
    }

    iim_status matvec(int op, int gate) {
        constexpr int W = 8;
        const size_t sm4 = sizeof(float) * 4 * (size_t)((G->max_ns + 3) & ~3);
        IIM_CHECK(allow_smem(kb_matvec<W>, sm4));
        double bytes = 0.0;
        for (iim_geometry g : G->geos) bytes += 4.0 * (double)(g->na + g->ncirc) * (g->na + g->ncirc);
        launch(op >= MV_S_ITER ? "ls_dense_schur_matvec" : "ls_precond_matvec", bytes, 0.0, kb_matvec<W>,
               grid((G->max_ns + W - 1) / W), W * 32, sm4, s, (const LsProb*)G->d_probs, op, gate);
        IIM_LAUNCHED();
        return IIM_OK;
    }

    iim_status vec(int op, int gate) {
        launch("ls_vec", 0.0, 0.0, kb_vec, grid((G->max_ns + 255) / 256), 256, 0, s, (const LsProb*)G->d_probs, op,
               gate);
        IIM_LAUNCHED();
        return IIM_OK;
    }

    // ghosts, FP64 residual, circulation measure, region sums, norms
    iim_status residual(int gate) {
        constexpr int kResBlocks = 1024;
        const LsProb* P = G->d_probs;
        if (G->max_nminus > 0)
            launch("ls_ghost_f64", 0.0, 0.0, kb_ghost, grid((G->max_nminus + 255) / 256), 256, 0, s, P, gate);
        double bytes = 0.0;
        for (iim_geometry g : G->geos) bytes += 25.0 * (double)g->NX * g->NY;
        launch("ls_residual_f64", bytes, 0.0, kb_residual<256>, grid(kResBlocks), 256, 0, s, P, gate);
        if (G->max_ncirc > 0) {
            launch("ls_circ_measure", 0.0, 0.0, kb_circ_measure<256>, grid(G->max_ncirc), 256, 0, s, P, gate);
            launch("ls_region_sums", 0.0, 0.0, kb_region_sums<256>, dim3(G->max_ncirc, kRegionParts, G->n()), 256, 0,
                   s, P, gate);
        }
        launch("ls_finish_residual", 0.0, 0.0, kb_finish_residual<256>, grid(1), 256, 0, s, P, gate, kResBlocks);
        IIM_LAUNCHED();
        return IIM_OK;
    }

    // --- the pieces between loop decisions
    iim_status top_pre(cudaGraphConditionalHandle h_ref) {
        const long npad = (long)G->nx * G->NY;
        launch("ls_init_psi", 0.0, 0.0, kb_init, grid((npad + 255) / 256), 256, 0, s, (const LsProb*)G->d_probs);
        launch("ls_init_psibar", 0.0, 0.0, kb_init_psibar, grid(1), 64, 0, s, (const LsProb*)G->d_probs);
        IIM_LAUNCHED();
        IIM_CHECK(residual(G_ALL));
        launch("ls_ref_init", 0.0, 0.0, kb_ref_init, 1, 256, 0, s, (const LsProb*)G->d_probs, G->n(), G->rtol, h_ref,
               flag(), cnt());
        IIM_LAUNCHED();
        return IIM_OK;
    }

    template <typename T>
    iim_status ref_pre(cudaGraphConditionalHandle h_cyc) {
        IIM_CHECK(rows_fwd<T>(M_RHS, G_REF));
        IIM_CHECK(cols<T>(M_RHS, G_REF));
        IIM_CHECK((rows_inv<T, INV_STORE_T>(G_REF)));
        IIM_CHECK(gather<T>(M_RHS, G_REF));
        IIM_CHECK(vec(V_ZERO_X, G_REF));
        launch("ls_gmres_start", 0.0, 0.0, kb_start<256>, grid(1), 256, 0, s, (const LsProb*)G->d_probs, KLayout{G->m},
               0, G->max_iter, G->inner);
        launch("ls_cyc_begin", 0.0, 0.0, kb_cyc_begin, 1, 256, 0, s, (const LsProb*)G->d_probs, G->n(), G->max_iter,
               h_cyc, flag());
        IIM_LAUNCHED();
        return IIM_OK;
    }

    iim_status cyc_pre(cudaGraphConditionalHandle h_it) {
        launch("ls_it_begin", 0.0, 0.0, kb_it_begin, 1, 256, 0, s, (const LsProb*)G->d_probs, G->n(), h_it, flag());
        IIM_LAUNCHED();
        return IIM_OK;
    }

    // one preconditioned GMRES iteration: z = M v_j, v_{j+1} = S z, Arnoldi step
    template <typename T>
    iim_status iteration(cudaGraphConditionalHandle h_it) {
        IIM_CHECK(matvec(MV_PRECOND, G_IT));
        if (G->dense) {
            IIM_CHECK(matvec(MV_S_ITER, G_IT));
        } else {
            IIM_CHECK(rows_fwd<T>(M_APPLY_PCZ, G_IT));
            IIM_CHECK(cols<T>(M_APPLY_PCZ, G_IT));
            IIM_CHECK((rows_inv<T, INV_STORE_T>(G_IT)));
            IIM_CHECK(gather<T>(M_APPLY_PCZ, G_IT));
        }
        launch("ls_gmres_arnoldi", 0.0, 0.0, kb_arnoldi<256>, grid(1), 256, 0, s, (const LsProb*)G->d_probs,
               KLayout{G->m});
        launch("ls_loop_ctl", 0.0, 0.0, kb_loop_ctl, 1, 256, 0, s, (const LsProb*)G->d_probs, G->n(), G->m + 2, h_it,
               flag(), cnt());
        IIM_LAUNCHED();
        return IIM_OK;
    }

    // x += M (V y), then another cycle (with the restart below) unless every problem is done
    iim_status cyc_post(cudaGraphConditionalHandle h_cyc, cudaGraphConditionalHandle h_rs) {
        launch("ls_gmres_backsolve", 0.0, 0.0, kb_backsolve<256>, grid(1), 256, 0, s, (const LsProb*)G->d_probs,
               KLayout{G->m});
        IIM_LAUNCHED();
        IIM_CHECK(matvec(MV_XUPDATE, G_CYC));
        launch("ls_cyc_ctl", 0.0, 0.0, kb_cyc_ctl, 1, 256, 0, s, (const LsProb*)G->d_probs, G->n(),
               G->max_iter / G->m + 2, h_cyc, h_rs, flag(), cnt());
        IIM_LAUNCHED();
        return IIM_OK;
    }

    // restart: V_1 = x, V_2 = S V_1, V_0 = (b - V_2) / ||b - V_2||
    template <typename T>
    iim_status restart() {
        IIM_CHECK(vec(V_RESTART_PREP, G_CYC));
        if (G->dense) {
            IIM_CHECK(matvec(MV_S_RESTART, G_CYC));
        } else {
            IIM_CHECK(rows_fwd<T>(M_APPLY_VTMP, G_CYC));
            IIM_CHECK(cols<T>(M_APPLY_VTMP, G_CYC));
            IIM_CHECK((rows_inv<T, INV_STORE_T>(G_CYC)));
            IIM_CHECK(gather<T>(M_APPLY_VTMP, G_CYC));
        }
        IIM_CHECK(vec(V_RESTART_RES, G_CYC));
        launch("ls_gmres_start", 0.0, 0.0, kb_start<256>, grid(1), 256, 0, s, (const LsProb*)G->d_probs, KLayout{G->m},
               1, 0, 0.0);
        IIM_LAUNCHED();
        return IIM_OK;
    }

    // psi_ext += P (r - E_a x), psibar += x_circ, the new residual, refinement control
    template <typename T>
    iim_status ref_post(cudaGraphConditionalHandle h_ref) {
        IIM_CHECK(rows_fwd<T>(M_RECOVER, G_REF));
        IIM_CHECK(cols<T>(M_RECOVER, G_REF));
        IIM_CHECK((rows_inv<T, INV_ACCUM_FLUID>(G_REF)));
        if (G->max_ncirc > 0)
            launch("ls_add_psibar", 0.0, 0.0, kb_add_psibar, grid(1), 64, 0, s, (const LsProb*)G->d_probs, 0, G_REF);
        IIM_LAUNCHED();
        IIM_CHECK(residual(G_REF));
        launch("ls_ref_ctl", 0.0, 0.0, kb_ref_ctl, 1, 256, 0, s, (const LsProb*)G->d_probs, G->n(), G->rtol,
               std::min(G->max_refine, 1000), G->max_iter, h_ref, flag(), cnt());
        IIM_LAUNCHED();
        return IIM_OK;
    }

    // capacitance correction of the circulation (problems with circulation bodies), velocity,
    // per-problem records
    iim_status top_post() {
        const LsProb* P = G->d_probs;
        if (G->cap) {
            const long npad = (long)G->nx * G->NY;
            launch("ls_cap_coef", 0.0, 0.0, kb_cap_coef, grid(1), 64, 0, s, P);
            launch("ls_cap_update", 0.0, 0.0, kb_cap_update, grid((npad + 255) / 256), 256, 0, s, P);
            launch("ls_add_psibar", 0.0, 0.0, kb_add_psibar, grid(1), 64, 0, s, P, 1, G_CAP);
            IIM_LAUNCHED();
            IIM_CHECK(residual(G_CAP));
            launch("ls_final_rel", 0.0, 0.0, kb_final_rel, grid(1), 1, 0, s, P);
        }
        const long n = (long)G->NX * G->NY;
        double bytes = 0.0;
        for (iim_geometry g : G->geos) bytes += (double)g->NX * g->NY * (9.0 + 8.0 + 16.0);
        launch("ls_velocity_f64", bytes, 0.0, kb_velocity, grid((n + 255) / 256), 256, 0, s, P);
        launch("ls_records", 0.0, 0.0, kb_records, (G->n() + 127) / 128, 128, 0, s, P, G->n(), KLayout{G->m},
               G->d_rec);
        IIM_LAUNCHED();
        return IIM_OK;
    }

    int read_flag() {
        cudaMemcpyAsync(G->h_cnt + 8, G->d_cnt + 8, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        return G->h_cnt[8];
    }

    // host-driven: the same pieces, each loop decided by the flag the control kernel wrote
    template <typename T>
    iim_status run_host() {
        IIM_CHECK(top_pre(0));
        long long nref = 0, ncyc = 0, nit = 0, nrs = 0;
        while (read_flag()) {
            IIM_CHECK(ref_pre<T>(0));
            ++nref;
            while (read_flag()) {
                IIM_CHECK(cyc_pre(0));
                ++ncyc;
                while (read_flag()) {
                    IIM_CHECK(iteration<T>(0));
                    ++nit;
                }
                IIM_CHECK(cyc_post(0, 0));
                if (!read_flag()) break;
                IIM_CHECK(restart<T>());
                ++nrs;
            }
            IIM_CHECK(ref_post<T>(0));
        }
        return top_post();
    }
};

// Captures the group's whole lockstep solve as one graph (nested WHILE / IF nodes, the same
// shape as the single-problem whole-solve graph).
template <typename T>
static iim_status build_group_graph(LsGroup* G) {
    cudaGraph_t top = nullptr;
    IIM_TRY(cudaGraphCreate(&top, 0));
    LsEmit E{G, G->cap_stream, false};
    set_capture(true);
    iim_status st = IIM_OK;
    cudaError_t ce = cudaSuccess;
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
    cudaGraphConditionalHandle h_ref = 0, h_cyc = 0, h_it = 0, h_rs = 0;
    cudaGraph_t ref_body = nullptr, cyc_body = nullptr, it_body = nullptr, rs_body = nullptr;
    CapSeg top_seg{G->cap_stream, top, {}};
    handle(top, &h_ref);
    piece(top_seg, [&]() { return E.top_pre(h_ref); });
    cond(top_seg, h_ref, cudaGraphCondTypeWhile, &ref_body);
    CapSeg ref_seg{G->cap_stream, ref_body, {}};
    handle(ref_body, &h_cyc);
    piece(ref_seg, [&]() { return E.ref_pre<T>(h_cyc); });
    cond(ref_seg, h_cyc, cudaGraphCondTypeWhile, &cyc_body);
    CapSeg cyc_seg{G->cap_stream, cyc_body, {}};
    handle(cyc_body, &h_it);
    handle(cyc_body, &h_rs);
    piece(cyc_seg, [&]() { return E.cyc_pre(h_it); });
    cond(cyc_seg, h_it, cudaGraphCondTypeWhile, &it_body);
    CapSeg it_seg{G->cap_stream, it_body, {}};
    piece(it_seg, [&]() { return E.iteration<T>(h_it); });
    piece(cyc_seg, [&]() { return E.cyc_post(h_cyc, h_rs); });
    cond(cyc_seg, h_rs, cudaGraphCondTypeIf, &rs_body);
    CapSeg rs_seg{G->cap_stream, rs_body, {}};
    piece(rs_seg, [&]() { return E.restart<T>(); });
    piece(ref_seg, [&]() { return E.ref_post<T>(h_ref); });
    piece(top_seg, [&]() { return E.top_post(); });
    set_capture(false);
    if (st == IIM_OK && ce == cudaSuccess) {
        G->k_top = kernel_nodes(top);
        G->k_ref = kernel_nodes(ref_body);
        G->k_cyc = kernel_nodes(cyc_body);
        G->k_it = kernel_nodes(it_body);
        G->k_rs = kernel_nodes(rs_body);
        ce = cudaGraphInstantiate(&G->exec, top, 0);
    }
    cudaGraphDestroy(top);
    if (ce != cudaSuccess) {
        G->exec = nullptr;
        record_cuda_error(ce, "lockstep graph", __FILE__, __LINE__);
        cudaGetLastError();
        return IIM_ERR_CUDA;
    }
    if (st != IIM_OK && G->exec) {
        cudaGraphExecDestroy(G->exec);
        G->exec = nullptr;
    }
    return st;
}

static iim_status make_group(const std::vector<iim_geometry>& geos, const iim_opts& o, double inner, LsGroup** out) {
    LsGroup* G = new LsGroup();
    G->geos = geos;
    G->prec = o.prec; G->m = o.restart; G->max_refine = o.max_refine; G->max_iter = o.max_iter;
    G->rtol = o.rtol; G->inner = inner; G->dense = o.precond == 3;
    iim_geometry g0 = geos[0];
    G->nx = g0->nx; G->ny = g0->ny; G->NX = g0->NX; G->NY = g0->NY; G->wide = g0->wide_lines; G->cols_c = g0->cols_c;
    G->tri = g0->col_solver == 1;
    for (iim_geometry g : geos) {
        G->max_na = std::max(G->max_na, g->na);
        G->max_ns = std::max(G->max_ns, g->na + g->ncirc);
        G->max_nminus = std::max(G->max_nminus, g->nminus);
        G->max_ncirc = std::max(G->max_ncirc, g->ncirc);
        G->max_ja_rows = std::max(G->max_ja_rows, g->ja1 - g->ja0 + 1);
        G->max_jo_rows = std::max(G->max_jo_rows, g->jo1 - g->jo0 + 1);
        G->cap |= (g->ncirc > 0 && g->cap_ready) ? 1 : 0;
    }
    const int n = G->n();
    iim_status st = IIM_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        record_cuda_error(e, what, __FILE__, __LINE__);
        st = IIM_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&G->d_probs, sizeof(LsProb) * n)) != cudaSuccess) fail(e, "cudaMalloc");
    else if ((e = cudaMalloc(&G->d_rec, sizeof(LsRec) * n)) != cudaSuccess) fail(e, "cudaMalloc");
    else if ((e = cudaMalloc(&G->d_cnt, sizeof(int) * 16)) != cudaSuccess) fail(e, "cudaMalloc");
    else if ((e = cudaMallocHost(&G->h_probs, sizeof(LsProb) * n)) != cudaSuccess) fail(e, "cudaMallocHost");
    else if ((e = cudaMallocHost(&G->h_rec, sizeof(LsRec) * n)) != cudaSuccess) fail(e, "cudaMallocHost");
    else if ((e = cudaMallocHost(&G->h_cnt, sizeof(int) * 16)) != cudaSuccess) fail(e, "cudaMallocHost");
    else if ((e = cudaStreamCreateWithFlags(&G->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        fail(e, "cudaStreamCreate");
    else if ((e = cudaEventCreate(&G->ev0)) != cudaSuccess || (e = cudaEventCreate(&G->ev1)) != cudaSuccess)
        fail(e, "cudaEventCreate");
    else if ((e = cudaMemset(G->d_cnt, 0, sizeof(int) * 16)) != cudaSuccess)
        fail(e, "cudaMemset");
    if (st != IIM_OK) {
        delete G;
        return st;
    }
    *out = G;
    return IIM_OK;
}

static LsGroup* find_group(const std::vector<iim_geometry>& geos, const iim_opts& o, double inner) {
    for (LsGroup* G : g_ls_groups) {
        if (G->geos != geos || G->prec != o.prec || G->dense != (o.precond == 3) || G->m != o.restart ||
            G->max_refine != o.max_refine ||
            G->max_iter != o.max_iter || G->rtol != o.rtol || G->inner != inner)
            continue;
        bool same = true;
        for (iim_geometry g : geos)
            same = same && g->wide_lines == G->wide && g->cols_c == G->cols_c &&
                   (g->col_solver == 1) == (G->tri != 0) &&
                   (g->ncirc > 0 && g->cap_ready ? 1 : 0) <= G->cap;
        if (same) return G;
    }
    return nullptr;
}

// Solves the problems `idx` of a batched call (same grid size and transform settings, all
// eligible) as one lockstep group on stream s; the per-problem results go to stats[] once
// lockstep_finish has run after s is synchronised.  host_driven = run the loop from the host
// (used while the per-kernel profiler is on).
iim_status lockstep_enqueue(const std::vector<int>& idx, iim_geometry const* geoms, const double* const* omega,
                            const double* const* psi_b, const double* const* psi_box, const double* const* gamma,
                            double* const* psibar, double* const* psi_out, double* const* ux_out,
                            double* const* uy_out, const iim_opts& o, cudaStream_t s, bool host_driven,
                            void** handle) {
    const double inner = o.inner_rtol > 0.0 ? o.inner_rtol : (o.prec == IIM_FP64 ? o.rtol / 20.0 : 1e-4);
    std::vector<iim_geometry> geos;
    for (int k : idx) geos.push_back(geoms[k]);
    LsGroup* G = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_ls_mutex);
        G = find_group(geos, o, inner);
        if (!G) {
            IIM_CHECK(make_group(geos, o, inner, &G));
            g_ls_groups.push_back(G);
        }
    }
    for (size_t q = 0; q < idx.size(); ++q) {
        const int k = idx[q];
        iim_geometry g = geoms[k];
        if (g->ncirc > 0)
            IIM_TRY(cudaMemcpyAsync(g->d_int + DI_CIRC, g->circ_ids.data(), g->ncirc * sizeof(int),
                                    cudaMemcpyHostToDevice, s));
        fill_prob(G->h_probs[q], g, o.prec, omega[k], psi_b[k], psi_box ? psi_box[k] : nullptr,
                  gamma ? gamma[k] : nullptr, psibar[k], psi_out[k], ux_out ? ux_out[k] : nullptr,
                  uy_out ? uy_out[k] : nullptr);
    }
    IIM_TRY(cudaMemcpyAsync(G->d_probs, G->h_probs, sizeof(LsProb) * idx.size(), cudaMemcpyHostToDevice, s));
    IIM_TRY(cudaEventRecord(G->ev0, s));
    if (host_driven) {
        LsEmit E{G, s, true};
        IIM_CHECK(o.prec == IIM_FP64 ? E.run_host<double>() : E.run_host<float>());
    } else {
        if (!G->exec) {
            // capture on the group's private stream after everything before it on s
            IIM_TRY(cudaStreamSynchronize(s));
            IIM_CHECK(o.prec == IIM_FP64 ? build_group_graph<double>(G) : build_group_graph<float>(G));
        }
        IIM_TRY(cudaGraphLaunch(G->exec, s));
    }
    IIM_TRY(cudaEventRecord(G->ev1, s));
    IIM_TRY(cudaMemcpyAsync(G->h_rec, G->d_rec, sizeof(LsRec) * idx.size(), cudaMemcpyDeviceToHost, s));
    if (!host_driven) IIM_TRY(cudaMemcpyAsync(G->h_cnt, G->d_cnt, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    *handle = G;
    return IIM_OK;
}

// After the stream of lockstep_enqueue has been synchronised: statuses and stats of the group's
// problems (as graph_finish does for one problem), and the launch count.
void lockstep_finish(void* handle, const std::vector<int>& idx, const iim_opts& o, bool host_driven,
                     std::vector<iim_status>& status, std::vector<iim_stats>& stats) {
    LsGroup* G = (LsGroup*)handle;
    if (!host_driven)
        count_launches(G->k_top + (long long)G->h_cnt[0] * G->k_ref + (long long)G->h_cnt[1] * G->k_cyc +
                       (long long)G->h_cnt[2] * G->k_it + (long long)G->h_cnt[3] * G->k_rs);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, G->ev0, G->ev1);
    for (size_t q = 0; q < idx.size(); ++q) {
        const LsRec& r = G->h_rec[q];
        const int k = idx[q];
        iim_geometry g = G->geos[q];
        iim_status st = IIM_OK;
        if (r.di[DI_NONFIN]) {
            st = IIM_ERR_NONFINITE;
        } else if (r.di[DI_LOOPERR] || r.di[DI_CYCERR]) {
            set_last_error("GMRES loop ended by its iteration cap");
            st = IIM_ERR_NOT_CONVERGED;
        } else if (r.rel > o.rtol) {
            st = IIM_ERR_NOT_CONVERGED;
        }
        status[k] = st;
        iim_stats& S = stats[k];
        std::memset(&S, 0, sizeof(S));
        S.iters = r.di[DI_ITS];
        S.refinements = r.di[DI_REF];
        S.status = st;
        S.rel_res = r.rel;
        const double bn = r.scal[SC_TOL] / std::max(G->inner, 1e-300);
        S.gmres_rel_res = (g->na + g->ncirc) > 0 && bn > 0.0 ? r.scal[SC_RESID] / bn : 0.0;
        S.circ_err_max = r.circ_err;
        S.seed_rel_res = 1.0;
        S.iters_first = r.di[DI_FIRST];
        S.ms = ms;
    }
}

}  // namespace iim

extern "C" int iim_set_lockstep(int max_group) {
    return iim::g_ls_group.exchange(max_group < 0 ? 0 : std::min(max_group, 1024));
}
