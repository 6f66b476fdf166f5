// Vorticity transport on the IIM grid (Sec. 3, Sec. 5.1, 5.3, 5.5, App. B) on the device.
//
//   * velocity extended to the A- nodes at third order with u_b (degree 2, Sec. 5.3);
//   * vorticity boundary condition omega_b = curl of the extended velocity at every control
//     point (Sec. 5.3; the stencil figure is missing, the reading used: along the grid line
//     the derivative at the crossing of the quadratic through the solid node, the fluid node
//     and the next fluid node; across it a one-sided second-order difference of the values
//     interpolated at the crossing on the next two rows (columns), combined with u_b; both
//     sides averaged when both are available);
//   * vorticity extended three times: fourth order with omega_b (diffusion), third order with
//     omega_b (upwind end of advective stencils), third order without a boundary condition
//     (downwind end) (Sec. 3.2);
//   * conservative fluxes (Eq. 2dshuconserve): third-order upwind advective flux of the point
//     flux u w (Eq. upwind; the face velocity selects the stencil), downwind stencil at inflow
//     boundary faces, centred diffusive flux;
//   * Kelvin ODE dGamma_k/dt = -h sum_{dR_k} (f + q).n with the same fluxes (Eq.
//     discreteKelvinChoice);
//   * Williamson low-storage RK3 on (omega, Gamma) with dt = C_stab dt_max from the RK3
//     polygon of App. B.
// Box: velocity Uinf at and beyond the box; vorticity 0 there except at the right (outflow)
// edge, where the last interior column is copied (zero gradient).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace iim {

static constexpr double kRK3A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static constexpr double kRK3B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
static constexpr double kStabC = 1.620, kStabR = 0.314;

__constant__ int t_dir_i[4] = {1, -1, 0, 0};
__constant__ int t_dir_j[4] = {0, 0, 1, -1};

struct TrView {
    int NX, NY, nx;
    double h;
    const uint8_t* cls;      // padded
    const int* minus_map;    // padded -> A- index
    const double* w;         // padded vorticity (fluid values)
    const double* ux;        // padded velocity with A- ghosts
    const double* uy;
    const double* g4;        // per A- node: fourth-order extension with omega_b
    const double* g3;        //              third-order with omega_b
    const double* g3n;       //              third-order without boundary condition
    double Ux, Uy;
};

__device__ __forceinline__ bool t_inside(const TrView& v, int i, int j) { return i >= 0 && i < v.NX && j >= 0 && j < v.NY; }
__device__ __forceinline__ long t_pidx(const TrView& v, int i, int j) { return (long)j * v.nx + 1 + i; }
__device__ __forceinline__ bool t_solid(const TrView& v, int i, int j) {
    return t_inside(v, i, j) && v.cls[t_pidx(v, i, j)] >= CLS_MINUS;
}
__device__ __forceinline__ double t_vel(const TrView& v, int comp, int i, int j) {
    if (!t_inside(v, i, j)) return comp ? v.Uy : v.Ux;
    return (comp ? v.uy : v.ux)[t_pidx(v, i, j)];
}
// kind 0: fourth-order extension with omega_b, 1: third-order with omega_b, 2: third-order without
__device__ __forceinline__ double t_omega(const TrView& v, int kind, int i, int j) {
    if (!t_inside(v, i, j)) {
        if (i >= v.NX && j >= 0 && j < v.NY) return v.w[t_pidx(v, v.NX - 1, j)];
        return 0.0;
    }
    const long p = t_pidx(v, i, j);
    const uint8_t c = v.cls[p];
    if (c <= CLS_PLUS) return v.w[p];
    if (c == CLS_MINUS) {
        const int m = v.minus_map[p];
        return kind == 0 ? v.g4[m] : (kind == 1 ? v.g3[m] : v.g3n[m]);
    }
    return 0.0;
}

// Flux f + q on the face between interior nodes a = (ai, aj) and a + e_axis.
__device__ double t_face_flux(const TrView& v, double nu, int axis, int ai, int aj) {
    const int di = axis == 0 ? 1 : 0, dj = axis == 0 ? 0 : 1;
    const int bi = ai + di, bj = aj + dj;
    const double ua = t_vel(v, axis, ai, aj), ub = t_vel(v, axis, bi, bj);
    const double uf = 0.5 * (ua + ub);
    bool pos = uf >= 0.0;
    const bool sa = t_solid(v, ai, aj), sb = t_solid(v, bi, bj);
    if (sa != sb) {
        const bool inflow = (sb && !pos) || (sa && pos);
        if (inflow) pos = !pos;   // downwind stencil at inflow boundary faces
    }
    const bool up_left = uf >= 0.0;
    int ni[3], nj[3];
    double wt[3];
    bool left[3];
    if (pos) {
        ni[0] = ai - di; nj[0] = aj - dj; ni[1] = ai; nj[1] = aj; ni[2] = bi; nj[2] = bj;
        wt[0] = -1.0 / 6.0; wt[1] = 5.0 / 6.0; wt[2] = 1.0 / 3.0;
        left[0] = true; left[1] = true; left[2] = false;
    } else {
        ni[0] = ai; nj[0] = aj; ni[1] = bi; nj[1] = bj; ni[2] = bi + di; nj[2] = bj + dj;
        wt[0] = 1.0 / 3.0; wt[1] = 5.0 / 6.0; wt[2] = -1.0 / 6.0;
        left[0] = true; left[1] = false; left[2] = false;
    }
    double f = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int kind = t_solid(v, ni[k], nj[k]) ? ((left[k] == up_left) ? 1 : 2) : 1;
        f += wt[k] * t_vel(v, axis, ni[k], nj[k]) * t_omega(v, kind, ni[k], nj[k]);
    }
    const double q = -nu * (t_omega(v, 0, bi, bj) - t_omega(v, 0, ai, aj)) / v.h;
    return f + q;
}

// user layout (NX stride) -> padded, fluid values only
__global__ void k_pack(int NX, int NY, const double* __restrict__ src, const uint8_t* __restrict__ cls, double* __restrict__ dst) {
    const int nx = NX + 1;   // a power of two
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nx * NY) return;
    const int j = k >> (__ffs(nx) - 1), i = (k & (nx - 1)) - 1;
    dst[k] = (i >= 0 && cls[k] <= CLS_PLUS) ? src[(long)j * NX + i] : 0.0;
}

// Third-order velocity extension with u_b at every A- node (both components).
__global__ void k_ext_velocity(int nm, int nx, const int* __restrict__ minus_node, const int* __restrict__ minus_cp,
                               const uint8_t* __restrict__ minus_mask, const double* __restrict__ cp_t,
                               const double* __restrict__ ubx, const double* __restrict__ uby, double* __restrict__ ux,
                               double* __restrict__ uy) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nm) return;
    const long p = minus_node[m];
    const uint8_t mask = minus_mask[m];
    double sx = 0.0, sy = 0.0;
    int cnt = 0;
    for (int d = 0; d < 4; ++d) {
        if (!(mask & (16 << d))) continue;
        const int c = minus_cp[4 * m + d];
        const double a = 1.0 - cp_t[c];
        // Lagrange weights at 0 of the quadratic through a (boundary), 2, 3
        const double w0 = 6.0 / ((a - 2.0) * (a - 3.0));
        const double w2 = -3.0 * a / (2.0 - a);
        const double w3 = 2.0 * a / (3.0 - a);
        const long step = (long)t_dir_j[d] * nx + t_dir_i[d];
        sx += w0 * ubx[c] + w2 * ux[p + 2 * step] + w3 * ux[p + 3 * step];
        sy += w0 * uby[c] + w2 * uy[p + 2 * step] + w3 * uy[p + 3 * step];
        ++cnt;
    }
    ux[p] = cnt ? sx / cnt : 0.0;
    uy[p] = cnt ? sy / cnt : 0.0;
}

// The three vorticity extensions at every A- node.
__global__ void k_ext_vorticity(int nm, int nx, const int* __restrict__ minus_node, const int* __restrict__ minus_cp,
                                const uint8_t* __restrict__ minus_mask, const double* __restrict__ cp_t,
                                const double* __restrict__ wb, const double* __restrict__ w, double* __restrict__ g4,
                                double* __restrict__ g3, double* __restrict__ g3n) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nm) return;
    const long p = minus_node[m];
    const uint8_t mask = minus_mask[m];
    double s4 = 0.0, s3 = 0.0, s3n = 0.0;
    int c4 = 0, c3 = 0;
    for (int d = 0; d < 4; ++d) {
        const int c = minus_cp[4 * m + d];
        if (c < 0) continue;
        const long step = (long)t_dir_j[d] * nx + t_dir_i[d];
        const double a = 1.0 - cp_t[c];
        if (mask & (1 << d)) {
            // cubic through a (boundary), 2, 3, 4
            const double w0 = -24.0 / ((a - 2.0) * (a - 3.0) * (a - 4.0));
            const double w2 = -6.0 * a / (2.0 - a);
            const double w3 = 8.0 * a / (3.0 - a);
            const double w4 = -3.0 * a / (4.0 - a);
            s4 += w0 * wb[c] + w2 * w[p + 2 * step] + w3 * w[p + 3 * step] + w4 * w[p + 4 * step];
            ++c4;
        }
        if (mask & (16 << d)) {
            const double w0 = 6.0 / ((a - 2.0) * (a - 3.0));
            const double w2 = -3.0 * a / (2.0 - a);
            const double w3 = 2.0 * a / (3.0 - a);
            s3 += w0 * wb[c] + w2 * w[p + 2 * step] + w3 * w[p + 3 * step];
            // quadratic through the fluid nodes 1, 2, 3 (no boundary condition)
            s3n += 3.0 * w[p + step] - 3.0 * w[p + 2 * step] + w[p + 3 * step];
            ++c3;
        }
    }
    g4[m] = c4 ? s4 / c4 : 0.0;
    g3[m] = c3 ? s3 / c3 : 0.0;
    g3n[m] = c3 ? s3n / c3 : 0.0;
}

// omega_b = curl of the extended velocity at each control point (Sec. 5.3, reading above).
__global__ void k_vorticity_bc(int ncp, TrView v, int nx_cells, int ny_cells, const int* __restrict__ cp_axis,
                               const int* __restrict__ cp_ei, const int* __restrict__ cp_ej, const double* __restrict__ cp_t,
                               const double* __restrict__ ubx, const double* __restrict__ uby, double* __restrict__ wb) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncp) return;
    const bool along_x = cp_axis[c] == 0;
    // global node coordinates of the edge ends; interior coordinates are global - 1
    const int ei = cp_ei[c], ej = cp_ej[c];
    const int oi = along_x ? ei + 1 : ei, oj = along_x ? ej : ej + 1;
    const bool lower_solid = t_solid(v, ei - 1, ej - 1);
    const int si = lower_solid ? ei : oi, sj = lower_solid ? ej : oj;
    const int fi = lower_solid ? oi : ei, fj = lower_solid ? oj : ej;
    const int di = fi - si, dj = fj - sj;
    const double t = cp_t[c], h = v.h;
    auto defined = [&](int gi, int gj) {
        if (gi <= 0 || gj <= 0 || gi >= nx_cells || gj >= ny_cells) return true;
        return v.cls[t_pidx(v, gi - 1, gj - 1)] <= CLS_MINUS;
    };
    const int ca = along_x ? 1 : 0;   // component differentiated along the line
    const int cb = along_x ? 0 : 1;   // component differentiated across the line
    const int dsgn = along_x ? di : dj;
    const double Us = t_vel(v, ca, si - 1, sj - 1), Uf = t_vel(v, ca, fi - 1, fj - 1);
    double d_along;
    if (!t_solid(v, fi + di - 1, fj + dj - 1)) {
        const double Un = t_vel(v, ca, fi + di - 1, fj + dj - 1);
        d_along = dsgn / h * ((Un - Us) / 2.0 - t * (Un - 2.0 * Uf + Us));
    } else {
        d_along = dsgn / h * (Uf - Us);
    }
    const double ub = along_x ? ubx[c] : uby[c];
    double est = 0.0, first = 0.0;
    int nest = 0;
    bool have_first = false;
    for (int sgn = 1; sgn >= -1; sgn -= 2) {
        double vals[2];
        bool ok = true;
        for (int k = 1; k <= 2 && ok; ++k) {
            const int pi_ = along_x ? 0 : k * sgn, pj_ = along_x ? k * sgn : 0;
            const int n0i = si + pi_, n0j = sj + pj_, n1i = fi + pi_, n1j = fj + pj_, n2i = fi + di + pi_,
                      n2j = fj + dj + pj_;
            if (!defined(n0i, n0j) || !defined(n1i, n1j) || !defined(n2i, n2j)) { ok = false; break; }
            const double Um = t_vel(v, cb, n0i - 1, n0j - 1), U0 = t_vel(v, cb, n1i - 1, n1j - 1),
                         Up = t_vel(v, cb, n2i - 1, n2j - 1);
            vals[k - 1] = U0 + (-t) * (Up - Um) / 2.0 + t * t * (Up - 2.0 * U0 + Um) / 2.0;
            if (k == 1 && !have_first) {
                first = sgn * (vals[0] - ub) / h;
                have_first = true;
            }
        }
        if (ok) {
            est += sgn * (-3.0 * ub + 4.0 * vals[0] - vals[1]) / (2.0 * h);
            ++nest;
        }
    }
    const double d_cross = nest ? est / nest : (have_first ? first : 0.0);
    wb[c] = along_x ? (d_along - d_cross) : (d_cross - d_along);
}

// ---- total pressure (Sec. 5.4)
// f = -div(u x omega k) = -(d_x(u_y omega) - d_y(u_x omega)) at fluid interior nodes by centred
// differences of the products, the third-order extensions (velocity with u_b, vorticity with
// omega_b) at A- nodes and the box values beyond (caller layout, 0 in the solid).
__global__ void k_pressure_rhs(TrView v, double* __restrict__ f) {
    const long n = (long)v.NX * v.NY;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = (int)(k % v.NX), j = (int)(k / v.NX);
    double r = 0.0;
    if (v.cls[t_pidx(v, i, j)] <= CLS_PLUS) {
        const double qe = t_vel(v, 1, i + 1, j) * t_omega(v, 1, i + 1, j);
        const double qw = t_vel(v, 1, i - 1, j) * t_omega(v, 1, i - 1, j);
        const double rn = t_vel(v, 0, i, j + 1) * t_omega(v, 1, i, j + 1);
        const double rs = t_vel(v, 0, i, j - 1) * t_omega(v, 1, i, j - 1);
        r = -((qe - qw) - (rn - rs)) / (2.0 * v.h);
    }
    f[k] = r;
}

// Wall datum of the Neumann extrapolation at each control point: d . grad H with d along the
// grid line into the fluid.  On a stationary no-slip wall grad H = grad p = nu k x grad omega
// (Eq. pressuregrad1; grad |u|^2 / 2 = (grad u)^T u vanishes where u = 0), so an x-line needs
// d_y omega and a y-line d_x omega at the crossing: the cross-line stencil of the vorticity
// boundary condition applied to the vorticity extended at third order with omega_b.
__global__ void k_pressure_wall_data(int ncp, TrView v, int nx_cells, int ny_cells, const int* __restrict__ cp_axis,
                                     const int* __restrict__ cp_ei, const int* __restrict__ cp_ej,
                                     const double* __restrict__ cp_t, const double* __restrict__ wb, double nu,
                                     double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncp) return;
    const bool along_x = cp_axis[c] == 0;
    const int ei = cp_ei[c], ej = cp_ej[c];
    const int oi = along_x ? ei + 1 : ei, oj = along_x ? ej : ej + 1;
    const bool lower_solid = t_solid(v, ei - 1, ej - 1);
    const int si = lower_solid ? ei : oi, sj = lower_solid ? ej : oj;
    const int fi = lower_solid ? oi : ei, fj = lower_solid ? oj : ej;
    const int di = fi - si, dj = fj - sj;
    const double t = cp_t[c], h = v.h, w0 = wb[c];
    auto defined = [&](int gi, int gj) {
        if (gi <= 0 || gj <= 0 || gi >= nx_cells || gj >= ny_cells) return true;
        return v.cls[t_pidx(v, gi - 1, gj - 1)] <= CLS_MINUS;
    };
    double est = 0.0, first = 0.0;
    int nest = 0;
    bool have_first = false;
    for (int sgn = 1; sgn >= -1; sgn -= 2) {
        double vals[2];
        bool ok = true;
        for (int k = 1; k <= 2 && ok; ++k) {
            const int pi_ = along_x ? 0 : k * sgn, pj_ = along_x ? k * sgn : 0;
            const int n0i = si + pi_, n0j = sj + pj_, n1i = fi + pi_, n1j = fj + pj_, n2i = fi + di + pi_,
                      n2j = fj + dj + pj_;
            if (!defined(n0i, n0j) || !defined(n1i, n1j) || !defined(n2i, n2j)) { ok = false; break; }
            const double Wm = t_omega(v, 1, n0i - 1, n0j - 1), W0 = t_omega(v, 1, n1i - 1, n1j - 1),
                         Wp = t_omega(v, 1, n2i - 1, n2j - 1);
            vals[k - 1] = W0 + (-t) * (Wp - Wm) / 2.0 + t * t * (Wp - 2.0 * W0 + Wm) / 2.0;
            if (k == 1 && !have_first) {
                first = sgn * (vals[0] - w0) / h;
                have_first = true;
            }
        }
        if (ok) {
            est += sgn * (-3.0 * w0 + 4.0 * vals[0] - vals[1]) / (2.0 * h);
            ++nest;
        }
    }
    const double d_cross = nest ? est / nest : (have_first ? first : 0.0);
    out[c] = along_x ? -nu * di * d_cross : nu * dj * d_cross;
}

// A field (caller layout) at each control point: the quadratic through the fluid node next to
// the crossing and the next two fluid interior nodes on its line, at the crossing (fewer nodes
// where those are not fluid interior nodes).
__global__ void k_wall_values(int ncp, TrView v, const int* __restrict__ cp_axis, const int* __restrict__ cp_ei,
                              const int* __restrict__ cp_ej, const double* __restrict__ cp_t,
                              const double* __restrict__ field, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncp) return;
    const bool along_x = cp_axis[c] == 0;
    const int ei = cp_ei[c], ej = cp_ej[c];
    const int oi = along_x ? ei + 1 : ei, oj = along_x ? ej : ej + 1;
    const bool lower_solid = t_solid(v, ei - 1, ej - 1);
    const int si = lower_solid ? ei : oi, sj = lower_solid ? ej : oj;
    const int fi = lower_solid ? oi : ei, fj = lower_solid ? oj : ej;
    const int di = fi - si, dj = fj - sj;
    auto fluid = [&](int gi, int gj) {   // global node coordinates
        return gi >= 1 && gj >= 1 && gi <= v.NX && gj <= v.NY && v.cls[t_pidx(v, gi - 1, gj - 1)] <= CLS_PLUS;
    };
    auto at = [&](int gi, int gj) { return field[(long)(gj - 1) * v.NX + (gi - 1)]; };
    const double x = -cp_t[c];
    const double F0 = at(fi, fj);
    double r;
    if (fluid(fi + di, fj + dj) && fluid(fi + 2 * di, fj + 2 * dj)) {
        const double F1 = at(fi + di, fj + dj), F2 = at(fi + 2 * di, fj + 2 * dj);
        r = F0 * (x - 1.0) * (x - 2.0) * 0.5 - F1 * x * (x - 2.0) + F2 * x * (x - 1.0) * 0.5;
    } else if (fluid(fi + di, fj + dj)) {
        r = F0 * (1.0 - x) + at(fi + di, fj + dj) * x;
    } else {
        r = F0;
    }
    out[c] = r;
}

// Transport right-hand side at fluid nodes.  mode 0: out_user = rhs (caller layout);
// mode 1: dw = a * dw + dt * rhs (padded).
__global__ void k_transport_rhs(TrView v, double nu, int mode, double a, double dt, double* __restrict__ out_user,
                                double* __restrict__ dw) {
    const long n = (long)v.NX * v.NY;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = (int)(k % v.NX), j = (int)(k / v.NX);
    const long p = t_pidx(v, i, j);
    double r = 0.0;
    if (v.cls[p] <= CLS_PLUS) {
        const double fr = t_face_flux(v, nu, 0, i, j), fl = t_face_flux(v, nu, 0, i - 1, j);
        const double gt = t_face_flux(v, nu, 1, i, j), gb = t_face_flux(v, nu, 1, i, j - 1);
        r = -((fr - fl) + (gt - gb)) / v.h;
    }
    if (mode == 0) out_user[k] = r;
    else dw[p] = a * dw[p] + dt * r;
}

// Kelvin ODE per body: dGdt[k] = -h sum_{dR_k}(f+q).n; with rk != 0 also the Williamson update
// dG = a dG + dt dGdt, Gamma += b dG (every body; fixed-psibar bodies do not read Gamma).
template <int BLOCK>
__global__ void k_kelvin(TrView v, double nu, const iim_region* __restrict__ R, const int* __restrict__ body_circ,
                         double* __restrict__ dgdt, int rk, double a, double b, double dt, double* __restrict__ dG,
                         double* __restrict__ gamma) {
    const int k = blockIdx.x;
    const iim_region r = R[k];
    double s = 0.0;
    // interior coordinates = global - 1
    for (int jj = r.ly + threadIdx.x; jj <= r.ry; jj += BLOCK)
        s += t_face_flux(v, nu, 0, r.rx - 1, jj - 1) - t_face_flux(v, nu, 0, r.lx - 2, jj - 1);
    for (int ii = r.lx + threadIdx.x; ii <= r.rx; ii += BLOCK)
        s += t_face_flux(v, nu, 1, ii - 1, r.ry - 1) - t_face_flux(v, nu, 1, ii - 1, r.ly - 2);
    __shared__ double red[BLOCK / 32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < BLOCK / 32; ++w) tot += red[w];
        const double rate = -v.h * tot;
        if (dgdt) dgdt[k] = rate;
        if (rk) {
            dG[k] = a * dG[k] + dt * rate;
            gamma[k] += b * dG[k];
        }
    }
}

__global__ void k_rk_omega(int NX, int NY, double b, const double* __restrict__ dw, const uint8_t* __restrict__ cls,
                           double* __restrict__ omega) {
    const int n = NX * NY;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int j = k / NX, i = k - j * NX;
    const int p = j * (NX + 1) + 1 + i;
    omega[k] = cls[p] <= CLS_PLUS ? omega[k] + b * dw[p] : 0.0;
}

template <int BLOCK>
__global__ void k_speed_max(long n, const double* __restrict__ ux, const double* __restrict__ uy, double* __restrict__ part) {
    double m = 0.0;
    for (long k = (long)blockIdx.x * BLOCK + threadIdx.x; k < n; k += (long)gridDim.x * BLOCK)
        m = fmax(m, fabs(ux[k]) + fabs(uy[k]));
    __shared__ double red[BLOCK / 32];
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < BLOCK / 32; ++w) t = fmax(t, red[w]);
        part[blockIdx.x] = t;
    }
}

// Transport workspace inside g->tr_buf (doubles).
struct TrWork {
    double *w, *ux, *uy, *dw, *g4, *g3, *g3n, *wb, *dG, *part, *psi, *vx, *vy, *zeros, *dgdt, *ub_stage;
};

static iim_status tr_work(iim_geometry g, TrWork* W) {
    const size_t npad = (size_t)g->nx * g->NY, n = (size_t)g->NX * g->NY, nm = (size_t)std::max(g->nminus, 1),
                 ncp = (size_t)std::max(g->ncp, 1);
    const size_t total = 4 * npad + 3 * nm + ncp + 64 + 1024 + 3 * n + ncp + 64 + 2 * ncp;
    if (!g->tr_buf) {
        IIM_TRY(cudaMalloc(&g->tr_buf, total * sizeof(double)));
        IIM_TRY(cudaMemset(g->tr_buf, 0, total * sizeof(double)));
    }
    double* p = g->tr_buf;
    W->w = p; p += npad;
    W->ux = p; p += npad;
    W->uy = p; p += npad;
    W->dw = p; p += npad;
    W->g4 = p; p += nm;
    W->g3 = p; p += nm;
    W->g3n = p; p += nm;
    W->wb = p; p += ncp;
    W->dG = p; p += 64;
    W->part = p; p += 1024;
    W->psi = p; p += n;
    W->vx = p; p += n;
    W->vy = p; p += n;
    W->zeros = p; p += ncp;
    W->dgdt = p; p += 64;
    W->ub_stage = p; p += 2 * ncp;
    return IIM_OK;
}

static TrView make_view(iim_geometry g, const TrWork& W, const double Uinf[2]) {
    TrView v;
    v.NX = g->NX; v.NY = g->NY; v.nx = g->nx; v.h = g->h;
    v.cls = g->node_class; v.minus_map = g->minus_map;
    v.w = W.w; v.ux = W.ux; v.uy = W.uy; v.g4 = W.g4; v.g3 = W.g3; v.g3n = W.g3n;
    v.Ux = Uinf ? Uinf[0] : 0.0;
    v.Uy = Uinf ? Uinf[1] : 0.0;
    return v;
}

// Velocity (caller layout) -> padded + extension; vorticity BC; vorticity -> padded + extensions.
static iim_status prepare_stage(iim_geometry g, const TrWork& W, const TrView& v, const double* omega, const double* ux,
                                const double* uy, const double* u_b, const double* wb_in, double* wb_out, cudaStream_t s) {
    const long npad = (long)g->nx * g->NY;
    const unsigned gp = (unsigned)((npad + 255) / 256);
    const double* ubx = u_b ? u_b : W.zeros;
    const double* uby = u_b ? u_b + g->ncp : W.zeros;
    launch("tr_pack", 0.0, 0.0, k_pack, gp, 256, 0, s, g->NX, g->NY, ux, g->node_class, W.ux);
    launch("tr_pack", 0.0, 0.0, k_pack, gp, 256, 0, s, g->NX, g->NY, uy, g->node_class, W.uy);
    launch("tr_pack", 0.0, 0.0, k_pack, gp, 256, 0, s, g->NX, g->NY, omega, g->node_class, W.w);
    if (g->nminus > 0)
        launch("tr_ext_velocity", 0.0, 0.0, k_ext_velocity, (g->nminus + 127) / 128, 128, 0, s, g->nminus, g->nx,
               g->minus_node, g->minus_cp, g->minus_mask, g->cp_t, ubx, uby, W.ux, W.uy);
    if (g->ncp > 0 && wb_in) {
        IIM_TRY(cudaMemcpyAsync(W.wb, wb_in, g->ncp * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else if (g->ncp > 0)
        launch("tr_vorticity_bc", 0.0, 0.0, k_vorticity_bc, (g->ncp + 127) / 128, 128, 0, s, g->ncp, v, g->nx, g->ny,
               g->cp_axis, g->cp_ei, g->cp_ej, g->cp_t, ubx, uby, W.wb);
    if (g->nminus > 0)
        launch("tr_ext_vorticity", 0.0, 0.0, k_ext_vorticity, (g->nminus + 127) / 128, 128, 0, s, g->nminus, g->nx,
               g->minus_node, g->minus_cp, g->minus_mask, g->cp_t, W.wb, W.w, W.g4, W.g3, W.g3n);
    IIM_LAUNCHED();
    if (wb_out && g->ncp > 0)
        IIM_TRY(cudaMemcpyAsync(wb_out, W.wb, g->ncp * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return IIM_OK;
}

}  // namespace iim

using namespace iim;

extern "C" iim_status iim_transport_rhs(iim_geometry g, const double* omega, const double* ux, const double* uy,
                                        const double* u_b, const double Uinf[2], double nu, const double* omega_b_in,
                                        double* omega_b_out, double* rhs_out, double* dgamma_out, iim_stream stream) {
    if (!g || !omega || !ux || !uy || !rhs_out || !(nu >= 0.0)) return IIM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    TrWork W;
    IIM_CHECK(tr_work(g, &W));
    const TrView v = make_view(g, W, Uinf);
    IIM_CHECK(prepare_stage(g, W, v, omega, ux, uy, u_b, omega_b_in, omega_b_out, s));
    const long n = (long)g->NX * g->NY;
    launch("tr_rhs", 40.0 * (double)n, 0.0, k_transport_rhs, (unsigned)((n + 255) / 256), 256, 0, s, v, nu, 0, 0.0, 1.0,
           rhs_out, W.dw);
    if (g->nb > 0 && dgamma_out)
        launch("tr_kelvin", 0.0, 0.0, k_kelvin<256>, g->nb, 256, 0, s, v, nu, g->d_regions, g->body_circ, dgamma_out, 0,
               0.0, 0.0, 0.0, W.dG, (double*)nullptr);
    IIM_LAUNCHED();
    return IIM_OK;
}

extern "C" iim_status iim_total_pressure_problem(iim_geometry g, const double* omega, const double* ux,
                                                 const double* uy, const double* u_b, const double Uinf[2], double nu,
                                                 const double* omega_b_in, double* omega_b_out, double* f_out,
                                                 double* data_out, iim_stream stream) {
    if (!g || !omega || !ux || !uy || !f_out || (g->ncp > 0 && !data_out) || !(nu >= 0.0)) return IIM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    TrWork W;
    IIM_CHECK(tr_work(g, &W));
    const TrView v = make_view(g, W, Uinf);
    IIM_CHECK(prepare_stage(g, W, v, omega, ux, uy, u_b, omega_b_in, omega_b_out, s));
    const long n = (long)g->NX * g->NY;
    launch("pressure_rhs", 48.0 * (double)n, 0.0, k_pressure_rhs, (unsigned)((n + 255) / 256), 256, 0, s, v, f_out);
    if (g->ncp > 0)
        launch("pressure_wall_data", 0.0, 0.0, k_pressure_wall_data, (g->ncp + 127) / 128, 128, 0, s, g->ncp, v, g->nx,
               g->ny, g->cp_axis, g->cp_ei, g->cp_ej, g->cp_t, (const double*)W.wb, nu, data_out);
    IIM_LAUNCHED();
    return IIM_OK;
}

extern "C" iim_status iim_wall_values(iim_geometry g, const double* field, double* out, iim_stream stream) {
    if (!g || !field || (g->ncp > 0 && !out)) return IIM_ERR_INVALID_ARG;
    if (g->ncp == 0) return IIM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    TrWork W;
    IIM_CHECK(tr_work(g, &W));
    const TrView v = make_view(g, W, nullptr);
    launch("wall_values", 0.0, 0.0, k_wall_values, (g->ncp + 127) / 128, 128, 0, s, g->ncp, v, g->cp_axis, g->cp_ei,
           g->cp_ej, g->cp_t, field, out);
    IIM_LAUNCHED();
    return IIM_OK;
}

extern "C" iim_status iim_total_pressure(iim_geometry g, const double* omega, const double* ux, const double* uy,
                                         const double Uinf[2], double nu, const double* H_box, double* H_out,
                                         double* H_wall_out, const iim_opts* opts, iim_stats* stats, iim_stream stream) {
    if (!g || !omega || !ux || !uy || !H_out || !(nu >= 0.0)) return IIM_ERR_INVALID_ARG;
    if (g->wall != 1) return IIM_ERR_INVALID_ARG;   // the solve needs the Neumann stencils
    const size_t n = (size_t)g->NX * g->NY, ncp = (size_t)std::max(g->ncp, 1);
    if (!g->pr_buf) {
        IIM_TRY(cudaMalloc(&g->pr_buf, (n + ncp) * sizeof(double)));
        IIM_TRY(cudaMemset(g->pr_buf, 0, (n + ncp) * sizeof(double)));
    }
    double* f = g->pr_buf;
    double* data = g->pr_buf + n;
    IIM_CHECK(iim_total_pressure_problem(g, omega, ux, uy, nullptr, Uinf, nu, nullptr, nullptr, f, data, stream));
    IIM_CHECK(iim_poisson_solve(g, f, data, H_box, nullptr, nullptr, H_out, nullptr, nullptr, nullptr, opts, stats,
                                stream));
    if (H_wall_out) IIM_CHECK(iim_wall_values(g, H_out, H_wall_out, stream));
    return IIM_OK;
}

// Stage times of the Williamson scheme: stage st sees the state at t + kRK3C[st] dt.
static constexpr double kRK3C[3] = {0.0, 1.0 / 3.0, 3.0 / 4.0};

// u_b at a stage time: u_b + c dt du_b/dt (u_b NULL = 0)
__global__ void k_ub_stage(int m, const double* __restrict__ ub, const double* __restrict__ rate, double cdt,
                           double* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) out[e] = (ub ? ub[e] : 0.0) + cdt * rate[e];
}

static iim_status rk3_step(iim_geometry g, double* omega, double* gamma, double* psibar, const double* u_b,
                           const double* u_b_rate, const double* psi_b, const double* psi_box, const double Uinf[2],
                           double nu, double c_stab, double* dt_inout, const iim_opts* opts, iim_stats* per_stage,
                           iim_stream stream) {
    if (!g || !omega || !dt_inout || !(nu >= 0.0) || (g->nb > 0 && (!gamma || !psibar))) return IIM_ERR_INVALID_ARG;
    if (*dt_inout <= 0.0 && !(c_stab > 0.0)) return IIM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    TrWork W;
    IIM_CHECK(tr_work(g, &W));
    const TrView v = make_view(g, W, Uinf);
    const long n = (long)g->NX * g->NY, npad = (long)g->nx * g->NY;
    IIM_TRY(cudaMemsetAsync(W.dw, 0, npad * sizeof(double), s));
    IIM_TRY(cudaMemsetAsync(W.dG, 0, 64 * sizeof(double), s));
    double dt = *dt_inout;
    for (int st = 0; st < 3; ++st) {
        iim_stats stats;
        const iim_status ps = iim_poisson_solve(g, omega, psi_b ? psi_b : W.zeros, psi_box, gamma, psibar, W.psi, W.vx,
                                                W.vy, nullptr, opts, &stats, stream);
        if (per_stage) per_stage[st] = stats;
        if (ps != IIM_OK) return ps;
        if (st == 0 && dt <= 0.0) {
            launch("tr_speed_max", 0.0, 0.0, k_speed_max<256>, 256, 256, 0, s, n, (const double*)W.vx, (const double*)W.vy,
                   W.part);
            IIM_LAUNCHED();
            std::vector<double> part(256);
            IIM_TRY(cudaMemcpyAsync(part.data(), W.part, 256 * sizeof(double), cudaMemcpyDeviceToHost, s));
            IIM_TRY(cudaStreamSynchronize(s));
            double U = 0.0;
            for (double x : part) U = std::max(U, x);
            const double h = g->h;
            dt = c_stab / (U / (kStabC * h) + nu / (kStabR * h * h));
        }
        const double* ub = u_b;
        if (u_b_rate) {
            const int m = 2 * g->ncp;
            if (m > 0)
                launch("tr_ub_stage", 0.0, 0.0, k_ub_stage, (unsigned)((m + 255) / 256), 256, 0, s, m, u_b, u_b_rate,
                       kRK3C[st] * dt, W.ub_stage);
            ub = W.ub_stage;
        }
        IIM_CHECK(prepare_stage(g, W, v, omega, W.vx, W.vy, ub, nullptr, nullptr, s));
        launch("tr_rhs", 40.0 * (double)n, 0.0, k_transport_rhs, (unsigned)((n + 255) / 256), 256, 0, s, v, nu, 1,
               kRK3A[st], dt, (double*)nullptr, W.dw);
        if (g->nb > 0)
            launch("tr_kelvin", 0.0, 0.0, k_kelvin<256>, g->nb, 256, 0, s, v, nu, g->d_regions, g->body_circ,
                   (double*)nullptr, 1, kRK3A[st], kRK3B[st], dt, W.dG, gamma);
        launch("tr_rk_omega", 24.0 * (double)n, 0.0, k_rk_omega, (unsigned)((n + 255) / 256), 256, 0, s, g->NX, g->NY,
               kRK3B[st], (const double*)W.dw, g->node_class, omega);
        IIM_LAUNCHED();
    }
    IIM_TRY(cudaStreamSynchronize(s));
    *dt_inout = dt;
    return IIM_OK;
}

extern "C" iim_status iim_rk3_step(iim_geometry g, double* omega, double* gamma, double* psibar, const double* u_b,
                                   const double* psi_b, const double* psi_box, const double Uinf[2], double nu,
                                   double c_stab, double* dt_inout, const iim_opts* opts, iim_stats* per_stage,
                                   iim_stream stream) {
    return rk3_step(g, omega, gamma, psibar, u_b, nullptr, psi_b, psi_box, Uinf, nu, c_stab, dt_inout, opts, per_stage,
                    stream);
}

extern "C" iim_status iim_rk3_step_moving_wall(iim_geometry g, double* omega, double* gamma, double* psibar,
                                               const double* u_b, const double* u_b_rate, const double* psi_b,
                                               const double* psi_box, const double Uinf[2], double nu, double c_stab,
                                               double* dt_inout, const iim_opts* opts, iim_stats* per_stage,
                                               iim_stream stream) {
    if (!u_b_rate) return IIM_ERR_INVALID_ARG;
    return rk3_step(g, omega, gamma, psibar, u_b, u_b_rate, psi_b, psi_box, Uinf, nu, c_stab, dt_inout, opts,
                    per_stage, stream);
}
