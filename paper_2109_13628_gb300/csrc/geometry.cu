// Geometry processing on the device: control points (App. A), affected points and node
// classes (Sec. 2.2), fourth-order ghost stencils and the correction operator gamma = A psi +
// B psi_b (Sec. 2.1, Sec. 4.2 Eq. poissoncorrections), body labels from the regions R_k.
//
// Control point location (App. A, reading of its garbled coordinates): along the grid line
// from the fluid node (s = 0) to the solid node (s = 1) the level set is interpolated by the
// cubic through the samples at s = -1, 0, 1, 2 (shifted inside the node array near the box),
// whose root is found by Newton's method from the linear root; a root outside [0, 1] is
// deflated away and the remaining quadratic solved.  Here the cubic is built from forward
// differences of the samples.
//
// Ghost value at an A- node g along a direction d whose neighbour g+d is fluid (Sec. 2.1):
// the cubic through the boundary point (at 1 - t in units of h from g, carrying psi_b) and the
// fluid nodes g+2d, g+3d, g+4d, evaluated at g (g+d itself is left out).  Usable only if
// g+2d..g+4d are fluid interior nodes; the ghost is the mean over usable directions (Sec. 2.2).
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace iim {

enum : int { ERR_BOX_SOLID = 1, ERR_MARGIN = 2, ERR_UNDERRES = 4, ERR_REGION = 8, ERR_FACES = 16 };
constexpr int kMargin = 5;

__constant__ int c_dir_i[4] = {1, -1, 0, 0};
__constant__ int c_dir_j[4] = {0, 0, 1, -1};

// ------------------------------------------------------------------------- control points
__device__ double cubic_root_app_a(const double f[4], double base, double t_lin) {
    // forward differences of samples at u = 0..3 (s = base + u)
    const double d1 = f[1] - f[0];
    const double d2 = f[2] - 2.0 * f[1] + f[0];
    const double d3 = f[3] - 3.0 * f[2] + 3.0 * f[1] - f[0];
    // Newton form -> monomial in u
    const double c3 = d3 / 6.0;
    const double c2 = 0.5 * d2 - 0.5 * d3;
    const double c1 = d1 - 0.5 * d2 + d3 / 3.0;
    const double c0 = f[0];
    // monomial in s = u + base
    const double b = base;
    const double a3 = c3;
    const double a2 = c2 - 3.0 * b * c3;
    const double a1 = c1 - 2.0 * b * c2 + 3.0 * b * b * c3;
    const double a0 = c0 - b * c1 + b * b * c2 - b * b * b * c3;
    double z = t_lin;
    for (int it = 0; it < 60; ++it) {
        const double p = ((a3 * z + a2) * z + a1) * z + a0;
        const double dp = (3.0 * a3 * z + 2.0 * a2) * z + a1;
        if (dp == 0.0) break;
        const double step = p / dp;
        z -= step;
        if (fabs(step) < 1e-15) break;
    }
    if (z >= 0.0 && z <= 1.0) return z;
    const double q2 = a3, q1 = a2 + z * q2, q0 = a1 + z * q1;
    if (q2 != 0.0) {
        const double disc = q1 * q1 - 4.0 * q2 * q0;
        if (disc >= 0.0) {
            const double sq = sqrt(disc);
            const double r1 = (-q1 + sq) / (2.0 * q2), r2 = (-q1 - sq) / (2.0 * q2);
            if (r1 >= 0.0 && r1 <= 1.0) return r1;
            if (r2 >= 0.0 && r2 <= 1.0) return r2;
        }
    } else if (q1 != 0.0) {
        const double r = -q0 / q1;
        if (r >= 0.0 && r <= 1.0) return r;
    }
    return t_lin;
}

// One thread per grid edge: x-edges (ny+1)*nx first, then y-edges ny*(nx+1).
__global__ void k_edge_cut(int nx, int ny, const double* __restrict__ phi, int* __restrict__ flag,
                           double* __restrict__ tval) {
    const long ex = (long)(ny + 1) * nx, ey = (long)ny * (nx + 1);
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ex + ey) return;
    int i, j, di, dj;
    if (e < ex) { j = (int)(e / nx); i = (int)(e - (long)j * nx); di = 1; dj = 0; }
    else { const long f = e - ex; j = (int)(f / (nx + 1)); i = (int)(f - (long)j * (nx + 1)); di = 0; dj = 1; }
    const int W = nx + 1;
    const double pa = phi[(long)j * W + i], pb = phi[(long)(j + dj) * W + i + di];
    const bool sa = pa < 0.0, sb = pb < 0.0;
    if (sa == sb) { flag[e] = 0; tval[e] = -1.0; return; }
    flag[e] = 1;
    int fi, fj, ui, uj;
    if (sa) { fi = i + di; fj = j + dj; ui = -di; uj = -dj; }
    else { fi = i; fj = j; ui = di; uj = dj; }
    const double pf = sa ? pb : pa, ps = sa ? pa : pb;
    const int nline = di ? (nx + 1) : (ny + 1);
    const int posf = di ? fi : fj;
    const int step = di ? ui : uj;
    int shift = 0;
    const int tries[5] = {0, 1, -1, 2, -2};
    for (int k = 0; k < 5; ++k) {
        const int s = tries[k];
        const int p0 = posf + (s - 1) * step, p3 = posf + (s + 2) * step;
        if (min(p0, p3) >= 0 && max(p0, p3) <= nline - 1) { shift = s; break; }
    }
    double f[4];
    for (int u = 0; u < 4; ++u) {
        const int o = u - 1 + shift;
        f[u] = phi[(long)(fj + o * uj) * W + fi + o * ui];
    }
    const double t_lin = pf / (pf - ps);
    tval[e] = cubic_root_app_a(f, (double)(shift - 1), t_lin);
}

__device__ __forceinline__ int body_of(int gi, int gj, int nb, const iim_region* __restrict__ R) {
    int hit = -1, cnt = 0;
    for (int k = 0; k < nb; ++k)
        if (gi >= R[k].lx && gi <= R[k].rx && gj >= R[k].ly && gj <= R[k].ry) { hit = k; ++cnt; }
    return cnt == 1 ? hit : -1;
}

__global__ void k_cp_fill(int nx, int ny, double x0, double y0, double h, const int* __restrict__ flag,
                          const int* __restrict__ pos, const double* __restrict__ tval, int nb,
                          const iim_region* __restrict__ R, const double* __restrict__ phi,
                          double* cx, double* cy, double* ct, int* cbody, int* caxis, int* cei, int* cej,
                          int* err) {
    const long ex = (long)(ny + 1) * nx, ey = (long)ny * (nx + 1);
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ex + ey || !flag[e]) return;
    int i, j, di, dj, axis;
    if (e < ex) { j = (int)(e / nx); i = (int)(e - (long)j * nx); di = 1; dj = 0; axis = 0; }
    else { const long f = e - ex; j = (int)(f / (nx + 1)); i = (int)(f - (long)j * (nx + 1)); di = 0; dj = 1; axis = 1; }
    const int W = nx + 1;
    const bool sa = phi[(long)j * W + i] < 0.0;
    const int si = sa ? i : i + di, sj = sa ? j : j + dj;
    const int fi = sa ? i + di : i, fj = sa ? j + dj : j;
    const double t = tval[e];
    const int k = pos[e];
    cx[k] = x0 + h * (fi + t * (si - fi));
    cy[k] = y0 + h * (fj + t * (sj - fj));
    ct[k] = t;
    caxis[k] = axis;
    cei[k] = i;
    cej[k] = j;
    const int b = body_of(si, sj, nb, R);
    cbody[k] = b;
    if (b < 0) atomicOr(err, ERR_REGION);
    if (si < kMargin || si > nx - kMargin || sj < kMargin || sj > ny - kMargin) atomicOr(err, ERR_MARGIN);
}

// ------------------------------------------------------------------------- node classes
__device__ __forceinline__ bool solid_at(const double* phi, int W, int i, int j) { return phi[(long)j * W + i] < 0.0; }

// Usable fourth-order extrapolation directions of solid node (gi, gj) as a bit mask; bit d
// set when g+d is fluid and g+2d..g+4d are fluid interior nodes.
__device__ int usable_dirs(const double* phi, int nx, int ny, int gi, int gj, int* n_fluid_nbrs) {
    const int W = nx + 1;
    int mask = 0, nf = 0;
    for (int d = 0; d < 4; ++d) {
        const int di = c_dir_i[d], dj = c_dir_j[d];
        if (solid_at(phi, W, gi + di, gj + dj)) continue;
        ++nf;
        bool ok = true;
        for (int m = 2; m <= 4; ++m) {
            const int qi = gi + m * di, qj = gj + m * dj;
            if (qi < 1 || qi > nx - 1 || qj < 1 || qj > ny - 1 || solid_at(phi, W, qi, qj)) { ok = false; break; }
        }
        if (ok) mask |= 1 << d;
    }
    if (n_fluid_nbrs) *n_fluid_nbrs = nf;
    return mask;
}

// Per interior node: class, affected / A- flags, entry counts of the gamma operator and of the
// ghost stencil.
__global__ void k_classify(int nx, int ny, const double* __restrict__ phi, uint8_t* cls, int* aff_flag,
                           int* minus_flag, int* gop_cnt, int* gh_cnt, int* err) {
    const int NX = nx - 1, NY = ny - 1;
    const long node = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= (long)NX * NY) return;
    const int gi = (int)(node % NX) + 1, gj = (int)(node / NX) + 1;
    const int W = nx + 1;
    const bool s = solid_at(phi, W, gi, gj);
    bool other = false;
    for (int d = 0; d < 4; ++d) other |= solid_at(phi, W, gi + c_dir_i[d], gj + c_dir_j[d]) != s;
    uint8_t c;
    int gop = 0, gh = 0;
    if (!other) {
        c = s ? CLS_SOLID : CLS_FLUID;
    } else if (s) {
        c = CLS_MINUS;
        int nf = 0;
        const int mask = usable_dirs(phi, nx, ny, gi, gj, &nf);
        gop = nf;
        gh = 4 * __popc(mask);
        if (mask == 0) atomicOr(err, ERR_UNDERRES);
    } else {
        c = CLS_PLUS;
        for (int d = 0; d < 4; ++d) {
            const int qi = gi + c_dir_i[d], qj = gj + c_dir_j[d];
            if (!solid_at(phi, W, qi, qj)) continue;
            if (qi < 1 || qi > nx - 1 || qj < 1 || qj > ny - 1) continue;   // box nodes are fluid
            gop += 4 * __popc(usable_dirs(phi, nx, ny, qi, qj, nullptr));
        }
    }
    cls[(long)(gj - 1) * nx + gi] = c;   // padded layout
    aff_flag[node] = (c == CLS_PLUS || c == CLS_MINUS);
    minus_flag[node] = (c == CLS_MINUS);
    gop_cnt[node] = gop;
    gh_cnt[node] = gh;
}

// Lagrange weights at s = 0 of the cubic through s = a (boundary point), 2, 3, 4.
__device__ __forceinline__ void ghost_weights4(double a, double w[4]) {
    w[0] = -24.0 / ((a - 2.0) * (a - 3.0) * (a - 4.0));
    w[1] = -6.0 * a / (2.0 - a);
    w[2] = 8.0 * a / (3.0 - a);
    w[3] = -3.0 * a / (4.0 - a);
}

__device__ __forceinline__ long edge_index(int nx, int ny, int gi, int gj, int d) {
    // edge between node g and g + dir(d)
    const int di = c_dir_i[d], dj = c_dir_j[d];
    if (di != 0) {
        const int i = min(gi, gi + di);
        return (long)gj * nx + i;
    }
    const int j = min(gj, gj + dj);
    return (long)(ny + 1) * nx + (long)j * (nx + 1) + gi;
}

// Writes the ghost-stencil entries of A- node (gi, gj) scaled by `scale`; returns the count.
__device__ int emit_ghost(int nx, int ny, const double* phi, const int* pos, const double* tval, int gi, int gj,
                          double scale, int* idx, double* w) {
    const int NX = nx - 1;
    const int mask = usable_dirs(phi, nx, ny, gi, gj, nullptr);
    const int nv = __popc(mask);
    const double s = scale / nv;
    int o = 0;
    for (int d = 0; d < 4; ++d) {
        if (!(mask & (1 << d))) continue;
        const long e = edge_index(nx, ny, gi, gj, d);
        const double a = 1.0 - tval[e];
        double wt[4];
        ghost_weights4(a, wt);
        idx[o] = -pos[e] - 1;
        w[o] = wt[0] * s;
        ++o;
        for (int m = 2; m <= 4; ++m) {
            const int qi = gi + m * c_dir_i[d], qj = gj + m * c_dir_j[d];
            idx[o] = (qj - 1) * nx + qi;   // padded layout
            w[o] = wt[m - 1] * s;
            ++o;
        }
    }
    return o;
}

__global__ void k_fill(int nx, int ny, double h, const double* __restrict__ phi, const uint8_t* __restrict__ cls,
                       const int* __restrict__ aff_pos, const int* __restrict__ minus_pos,
                       const int* __restrict__ gop_off, const int* __restrict__ gh_off,
                       const int* __restrict__ edge_pos, const double* __restrict__ tval, int nb,
                       const iim_region* __restrict__ R, int* aff_node, int* aff_body, uint8_t* aff_solid,
                       int* gop_idx, double* gop_w, int* minus_node, int* gh_idx, double* gh_w, int* minus_cp,
                       uint8_t* minus_mask, int* minus_map, int* err) {
    const int NX = nx - 1, NY = ny - 1;
    const long node = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= (long)NX * NY) return;
    const int gi = (int)(node % NX) + 1, gj = (int)(node / NX) + 1;
    const long pnode = (long)(gj - 1) * nx + gi;   // padded layout
    const uint8_t c = cls[pnode];
    if (c != CLS_PLUS && c != CLS_MINUS) return;
    const int W = nx + 1;
    const int a = aff_pos[node];
    aff_node[a] = (int)pnode;
    aff_solid[a] = (c == CLS_MINUS);
    const int b = body_of(gi, gj, nb, R);
    aff_body[a] = b;
    if (b < 0) atomicOr(err, ERR_REGION);
    const double ih2 = 1.0 / (h * h);
    int o = gop_off[node];
    if (c == CLS_MINUS) {
        // gamma_p = (1/h^2) sum of fluid neighbours
        for (int d = 0; d < 4; ++d) {
            const int qi = gi + c_dir_i[d], qj = gj + c_dir_j[d];
            if (solid_at(phi, W, qi, qj)) continue;
            gop_idx[o] = (qj - 1) * nx + qi;
            gop_w[o] = ih2;
            ++o;
        }
        const int m = minus_pos[node];
        minus_node[m] = (int)pnode;
        minus_map[pnode] = m;
        // per direction: control point index (or -1) and validity of the fourth-order (bit d)
        // and third-order (bit 4 + d) extrapolations
        uint8_t mask = (uint8_t)usable_dirs(phi, nx, ny, gi, gj, nullptr);
        for (int d = 0; d < 4; ++d) {
            const int qi = gi + c_dir_i[d], qj = gj + c_dir_j[d];
            if (solid_at(phi, W, qi, qj)) { minus_cp[4 * m + d] = -1; continue; }
            minus_cp[4 * m + d] = edge_pos[edge_index(nx, ny, gi, gj, d)];
            bool ok3 = true;
            for (int k = 2; k <= 3; ++k) {
                const int ri = gi + k * c_dir_i[d], rj = gj + k * c_dir_j[d];
                if (ri < 1 || ri > nx - 1 || rj < 1 || rj > ny - 1 || solid_at(phi, W, ri, rj)) ok3 = false;
            }
            if (ok3) mask |= (uint8_t)(16 << d);
        }
        minus_mask[m] = mask;
        emit_ghost(nx, ny, phi, edge_pos, tval, gi, gj, 1.0, gh_idx + gh_off[node], gh_w + gh_off[node]);
    } else {
        // gamma_p = -(1/h^2) sum of the ghost values of the solid neighbours
        for (int d = 0; d < 4; ++d) {
            const int qi = gi + c_dir_i[d], qj = gj + c_dir_j[d];
            if (!solid_at(phi, W, qi, qj)) continue;
            if (qi < 1 || qi > nx - 1 || qj < 1 || qj > ny - 1) continue;
            o += emit_ghost(nx, ny, phi, edge_pos, tval, qi, qj, -ih2, gop_idx + o, gop_w + o);
        }
    }
    (void)NY;
}

// Weights at s = 0 of the Neumann variant (Sec. 2.1): the cubic p with p(m) = f(g + m d),
// m = 2, 3, 4, and p'(a) = h (d . grad f) at the crossing.  With L the quadratic through the three
// nodes and pi(s) = (s - 2)(s - 3)(s - 4), p = L + c pi, so p(0) = L(0) - 24 (p'(a) - L'(a)) / pi'(a);
// w[0] multiplies the derivative in units of h.
__device__ __forceinline__ void neumann_weights4(double a, double w[4]) {
    const double dpi = (3.0 * a - 18.0) * a + 26.0;   // pi'(a) > 0 on [0, 1]
    const double k = 24.0 / dpi;
    w[0] = -k;
    w[1] = 6.0 + k * (a - 3.5);    // l_2(0) + 24 l_2'(a) / pi'(a), l_2' = (2a - 7) / 2
    w[2] = -8.0 + k * (6.0 - 2.0 * a);
    w[3] = 3.0 + k * (a - 2.5);
}

// Rewrites the ghost blocks of every gop row of an A+ point (rows 0..na-1) and every gh row
// (rows na..na+nm-1) for wall condition `kind`.  A block is [control point, g+2d, g+3d, g+4d];
// the scale of the block is that of k_fill: 1 / nv (gh) or -1/h^2 / nv (gop), nv the usable
// directions of the ghost g (bits 0..3 of minus_mask).
__global__ void k_wall_weights(int na, int nm, int nx, double h, int kind, const int* __restrict__ gop_ptr,
                               const int* __restrict__ gop_idx, double* __restrict__ gop_w,
                               const uint8_t* __restrict__ aff_solid, const int* __restrict__ gh_ptr,
                               const int* __restrict__ gh_idx, double* __restrict__ gh_w,
                               const uint8_t* __restrict__ minus_mask, const int* __restrict__ minus_map,
                               const double* __restrict__ cp_t) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= na + nm) return;
    const bool is_gh = r >= na;
    if (!is_gh && aff_solid[r]) return;   // A- rows: fluid neighbours, no ghost blocks
    const int* ptr = is_gh ? gh_ptr : gop_ptr;
    const int* idx = is_gh ? gh_idx : gop_idx;
    double* w = is_gh ? gh_w : gop_w;
    const int row = is_gh ? r - na : r;
    const double ih2 = 1.0 / (h * h);
    const double scale = is_gh ? 1.0 : -ih2;
    for (int o = ptr[row]; o + 3 < ptr[row + 1]; o += 4) {
        const int c = -idx[o] - 1;
        const int step = idx[o + 2] - idx[o + 1];
        const int m = is_gh ? row : minus_map[idx[o + 1] - 2 * step];
        const int nv = __popc(minus_mask[m] & 15);
        const double s = scale / nv;
        const double a = 1.0 - cp_t[c];
        double wt[4];
        if (kind == 1) {
            neumann_weights4(a, wt);
            wt[0] *= h;
        } else {
            ghost_weights4(a, wt);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) w[o + k] = wt[k] * s;
    }
}

iim_status rewrite_wall_weights(iim_geometry g, int kind, cudaStream_t s) {
    const int rows = g->na + g->nminus;
    if (rows > 0) {
        k_wall_weights<<<(rows + 127) / 128, 128, 0, s>>>(g->na, g->nminus, g->nx, g->h, kind, g->gop_ptr, g->gop_idx,
                                                          g->gop_w, g->aff_solid, g->gh_ptr, g->gh_idx, g->gh_w,
                                                          g->minus_mask, g->minus_map, g->cp_t);
        IIM_TRY(cudaGetLastError());
    }
    IIM_TRY(cudaStreamSynchronize(s));
    return IIM_OK;
}

// Box ring must be fluid.
__global__ void k_check_box(int nx, int ny, const double* __restrict__ phi, int* err) {
    const int W = nx + 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nring = 2 * (nx + 1) + 2 * (ny - 1);
    if (k >= nring) return;
    int i, j;
    if (k < nx + 1) { i = k; j = 0; }
    else if (k < 2 * (nx + 1)) { i = k - (nx + 1); j = ny; }
    else if (k < 2 * (nx + 1) + ny - 1) { i = 0; j = k - 2 * (nx + 1) + 1; }
    else { i = nx; j = k - 2 * (nx + 1) - (ny - 1) + 1; }
    if (phi[(long)j * W + i] < 0.0) atomicOr(err, ERR_BOX_SOLID);
}

// Region faces: the rings just inside and just outside R_k must be plain fluid.
__global__ void k_check_regions(int nx, int nb, const iim_region* __restrict__ R, const uint8_t* __restrict__ cls,
                                int* err) {
    const int k = blockIdx.x;
    if (k >= nb) return;
    const int NX = nx - 1;
    const iim_region r = R[k];
    const int w = r.rx - r.lx + 3, hgt = r.ry - r.ly + 3;
    for (int t = threadIdx.x; t < w * hgt; t += blockDim.x) {
        const int i = r.lx - 1 + t % w, j = r.ly - 1 + t / w;
        const bool inner = (i > r.lx && i < r.rx && j > r.ly && j < r.ry);
        if (inner) continue;
        if (cls[(long)(j - 1) * nx + i] != CLS_FLUID) atomicOr(err, ERR_FACES);
    }
}

__global__ void k_row_ptr(int NX, int NY, int na, const int* __restrict__ aff_pos, int* row_ptr) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < NY) row_ptr[r] = aff_pos[(long)r * NX];
    if (r == NY) row_ptr[NY] = na;
}

// ptr[a] = offset of node a (nodes in the padded layout, offsets over the unpadded one)
__global__ void k_ptr_from_offsets(int n, int nx, const int* __restrict__ nodes, const int* __restrict__ off, int total,
                                   int* ptr) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n) {
        const int p = nodes[a];
        const int r = p / nx, i = p - r * nx - 1;
        ptr[a] = off[(long)r * (nx - 1) + i];
    }
    if (a == n) ptr[n] = total;
}

__global__ void k_body_circ(int nb, const int* __restrict__ modes, int* body_circ) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int c = 0;
        for (int k = 0; k < nb; ++k) body_circ[k] = modes[k] == IIM_BODY_CIRCULATION ? c++ : -1;
    }
}

// ------------------------------------------------------------------------- host helpers
static iim_status exclusive_scan(const int* in, int* out, long n, int* total, cudaStream_t s) {
    size_t bytes = 0;
    IIM_TRY(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, (int)n, s));
    void* tmp = nullptr;
    IIM_TRY(cudaMallocAsync(&tmp, bytes, s));
    cudaError_t e = cub::DeviceScan::ExclusiveSum(tmp, bytes, in, out, (int)n, s);
    int last_in = 0, last_out = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last_in, in + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last_out, out + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(tmp, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { record_cuda_error(e, "exclusive_scan", __FILE__, __LINE__); return IIM_ERR_CUDA; }
    *total = last_in + last_out;
    return IIM_OK;
}

template <typename T>
static iim_status dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    IIM_TRY(cudaMalloc((void**)p, n * sizeof(T)));
    return IIM_OK;
}

// Factors of the tridiagonal column pass (tri.cuh) in one precision.  For x mode p = c + 1:
// eps = 4 sin^2(pi p / (2 nx)), theta = acosh(1 + eps / 2), and the Thomas factors in closed form
// e_j = sinh((j + 1) theta) / sinh((j + 2) theta), so with e* = exp(-theta), q = exp(-2 theta)
//   delta_j = 1 - e_j = delta* + e* q^(j+1) (1 - q) / (1 - q^(j+2)),   delta* = -expm1(-theta),
// every term accurate to a few units in the last place in FP64 (no recurrence, no
// cancellation).  Column c uses delta* from row lim[c] on, lim[c] the first row whose
// correction term is within tol of delta* (relative), made non-increasing in c.  FP64: the rows
// before lim as a table, row-major over rows (the tabulated columns of a row are a prefix);
// FP32: per column (delta*, log2 q, q, e* (1 - q)) for the kernel's own evaluation of the form.
static double scan_corr(double theta, int j) {
    return std::exp(-theta) * std::exp(-2.0 * (j + 1) * theta) * std::expm1(-2.0 * theta) /
           std::expm1(-2.0 * (j + 2) * theta);
}

template <typename T>
static iim_status scan_tables(int nx, int NX, int NY, double tol, T** delta, int** rowoff, float4** par, int** lim,
                              T** dstar) {
    std::vector<int> L(NX);
    std::vector<double> th(NX);
    std::vector<T> ds(NX);
    std::vector<float4> pr(NX);
    for (int c = 0; c < NX; ++c) {
        const double sn = std::sin(M_PI * (c + 1) / (2.0 * nx));
        const double eps = 4.0 * sn * sn;
        const double theta = std::log1p(0.5 * eps + std::sqrt(eps + 0.25 * eps * eps));
        const double dstar_c = -std::expm1(-theta);
        th[c] = theta;
        ds[c] = (T)dstar_c;
        pr[c] = make_float4((float)dstar_c, (float)(-2.0 * theta / M_LN2), (float)std::exp(-2.0 * theta),
                            (float)(-std::exp(-theta) * std::expm1(-2.0 * theta)));
        int j = 0;
        while (j < NY && scan_corr(theta, j) > tol * dstar_c) ++j;
        L[c] = j;
    }
    for (int c = NX - 2; c >= 0; --c) L[c] = std::max(L[c], L[c + 1]);
    IIM_CHECK(dalloc(lim, NX));
    IIM_CHECK(dalloc(dstar, NX));
    IIM_TRY(cudaMemcpy(*lim, L.data(), NX * sizeof(int), cudaMemcpyHostToDevice));
    IIM_TRY(cudaMemcpy(*dstar, ds.data(), NX * sizeof(T), cudaMemcpyHostToDevice));
    if (sizeof(T) == 4) {
        IIM_CHECK(dalloc(par, NX));
        IIM_TRY(cudaMemcpy(*par, pr.data(), NX * sizeof(float4), cudaMemcpyHostToDevice));
        return IIM_OK;
    }
    std::vector<int> off(NY + 1, 0);
    std::vector<T> tab;
    int C = NX;
    for (int j = 0; j < NY; ++j) {
        while (C > 0 && L[C - 1] <= j) --C;
        off[j] = (int)tab.size();
        for (int c = 0; c < C; ++c) tab.push_back((T)(-std::expm1(-th[c]) + scan_corr(th[c], j)));
    }
    off[NY] = (int)tab.size();
    IIM_CHECK(dalloc(delta, tab.size()));
    IIM_CHECK(dalloc(rowoff, NY + 1));
    if (!tab.empty()) IIM_TRY(cudaMemcpy(*delta, tab.data(), tab.size() * sizeof(T), cudaMemcpyHostToDevice));
    IIM_TRY(cudaMemcpy(*rowoff, off.data(), (NY + 1) * sizeof(int), cudaMemcpyHostToDevice));
    return IIM_OK;
}

void free_geometry(iim_geometry g);

}  // namespace iim

using namespace iim;

extern "C" iim_status iim_setup_geometry(const iim_grid* grid, const double* phi, int n_bodies,
                                         const iim_region* regions, const int* modes, iim_stream stream,
                                         iim_geometry* out) {
    if (!out) return IIM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid || !phi || n_bodies < 0 || n_bodies > 64 || (n_bodies > 0 && (!regions || !modes)))
        return IIM_ERR_INVALID_ARG;
    const int nx = grid->nx, ny = grid->ny;
    if (!is_pow2_in(nx, 16, 2048) || !is_pow2_in(ny, 16, 2048)) return IIM_ERR_INVALID_ARG;
    const double h = (grid->x1 - grid->x0) / nx;
    if (!(h > 0.0) || std::fabs((grid->y1 - grid->y0) / ny - h) > 1e-12 * h) return IIM_ERR_INVALID_ARG;
    for (int k = 0; k < n_bodies; ++k) {
        const iim_region r = regions[k];
        if (modes[k] != IIM_BODY_FIXED && modes[k] != IIM_BODY_CIRCULATION) return IIM_ERR_INVALID_ARG;
        if (r.lx < 2 || r.ly < 2 || r.rx > nx - 2 || r.ry > ny - 2 || r.lx > r.rx || r.ly > r.ry) return IIM_ERR_BAD_REGION;
    }
    IIM_CHECK(ensure_twiddles());
    cudaStream_t s = (cudaStream_t)stream;
    iim_geometry g = new iim_geometry_s();
    cudaGetDevice(&g->device);
    g->grid = *grid;
    g->nx = nx; g->ny = ny; g->NX = nx - 1; g->NY = ny - 1; g->h = h;
    g->nb = n_bodies;
    g->regions.assign(regions, regions + n_bodies);
    g->modes.assign(modes, modes + n_bodies);
    for (int k = 0; k < n_bodies; ++k)
        if (modes[k] == IIM_BODY_CIRCULATION) g->circ_ids.push_back(k);
    g->ncirc = (int)g->circ_ids.size();
    const int NX = g->NX, NY = g->NY;
    const long nnode = (long)NX * NY;
    const long nedge = (long)(ny + 1) * nx + (long)ny * (nx + 1);

    int *flag = nullptr, *epos = nullptr, *err = nullptr, *aff_flag = nullptr, *aff_pos = nullptr;
    int *minus_flag = nullptr, *minus_pos = nullptr, *gop_cnt = nullptr, *gop_off = nullptr;
    int *gh_cnt = nullptr, *gh_off = nullptr, *d_modes = nullptr;
    double* tval = nullptr;
    iim_status st = IIM_OK;
    int herr = 0, gop_total = 0, gh_total = 0;
    auto fail = [&](iim_status code) {
        cudaFree(flag); cudaFree(epos); cudaFree(err); cudaFree(aff_flag); cudaFree(aff_pos);
        cudaFree(minus_flag); cudaFree(minus_pos); cudaFree(gop_cnt); cudaFree(gop_off);
        cudaFree(gh_cnt); cudaFree(gh_off); cudaFree(tval); cudaFree(d_modes);
        if (code != IIM_OK) { free_geometry(g); return code; }
        return code;
    };
#define SETUP_TRY(x)                           \
    do {                                       \
        iim_status s2_ = (x);                  \
        if (s2_ != IIM_OK) return fail(s2_);   \
    } while (0)
#define SETUP_CUDA(x)                                                                 \
    do {                                                                              \
        cudaError_t e2_ = (x);                                                        \
        if (e2_ != cudaSuccess) { record_cuda_error(e2_, #x, __FILE__, __LINE__); return fail(IIM_ERR_CUDA); } \
    } while (0)

    SETUP_TRY(dalloc(&flag, nedge));
    SETUP_TRY(dalloc(&epos, nedge));
    SETUP_TRY(dalloc(&tval, nedge));
    SETUP_TRY(dalloc(&err, 1));
    SETUP_TRY(dalloc(&g->d_regions, n_bodies));
    SETUP_TRY(dalloc(&d_modes, n_bodies));
    SETUP_TRY(dalloc(&g->body_circ, n_bodies));
    SETUP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    if (n_bodies) {
        SETUP_CUDA(cudaMemcpyAsync(g->d_regions, regions, n_bodies * sizeof(iim_region), cudaMemcpyHostToDevice, s));
        SETUP_CUDA(cudaMemcpyAsync(d_modes, modes, n_bodies * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    k_body_circ<<<1, 32, 0, s>>>(n_bodies, d_modes, g->body_circ);
    k_check_box<<<(2 * (nx + ny) + 255) / 256, 256, 0, s>>>(nx, ny, phi, err);
    k_edge_cut<<<(unsigned)((nedge + 255) / 256), 256, 0, s>>>(nx, ny, phi, flag, tval);
    SETUP_CUDA(cudaGetLastError());
    SETUP_TRY(exclusive_scan(flag, epos, nedge, &g->ncp, s));
    SETUP_TRY(dalloc(&g->cp_x, g->ncp)); SETUP_TRY(dalloc(&g->cp_y, g->ncp)); SETUP_TRY(dalloc(&g->cp_t, g->ncp));
    SETUP_TRY(dalloc(&g->cp_body, g->ncp)); SETUP_TRY(dalloc(&g->cp_axis, g->ncp));
    SETUP_TRY(dalloc(&g->cp_ei, g->ncp)); SETUP_TRY(dalloc(&g->cp_ej, g->ncp));
    k_cp_fill<<<(unsigned)((nedge + 255) / 256), 256, 0, s>>>(nx, ny, grid->x0, grid->y0, h, flag, epos, tval, n_bodies,
                                                            g->d_regions, phi, g->cp_x, g->cp_y, g->cp_t, g->cp_body,
                                                            g->cp_axis, g->cp_ei, g->cp_ej, err);
    SETUP_CUDA(cudaGetLastError());

    const long npad = (long)nx * NY;   // padded layout: row r at [r*nx, r*nx + nx), slot 0 a pad
    SETUP_TRY(dalloc(&g->node_class, npad));
    SETUP_CUDA(cudaMemsetAsync(g->node_class, CLS_SOLID, npad, s));
    SETUP_TRY(dalloc(&aff_flag, nnode)); SETUP_TRY(dalloc(&aff_pos, nnode));
    SETUP_TRY(dalloc(&minus_flag, nnode)); SETUP_TRY(dalloc(&minus_pos, nnode));
    SETUP_TRY(dalloc(&gop_cnt, nnode)); SETUP_TRY(dalloc(&gop_off, nnode));
    SETUP_TRY(dalloc(&gh_cnt, nnode)); SETUP_TRY(dalloc(&gh_off, nnode));
    k_classify<<<(unsigned)((nnode + 255) / 256), 256, 0, s>>>(nx, ny, phi, g->node_class, aff_flag, minus_flag, gop_cnt,
                                                             gh_cnt, err);
    SETUP_CUDA(cudaGetLastError());
    SETUP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SETUP_CUDA(cudaStreamSynchronize(s));
    if (herr & (ERR_BOX_SOLID | ERR_MARGIN | ERR_REGION)) return fail(IIM_ERR_BAD_REGION);
    if (herr & ERR_UNDERRES) return fail(IIM_ERR_UNDERRESOLVED);
    SETUP_TRY(exclusive_scan(aff_flag, aff_pos, nnode, &g->na, s));
    SETUP_TRY(exclusive_scan(minus_flag, minus_pos, nnode, &g->nminus, s));
    SETUP_TRY(exclusive_scan(gop_cnt, gop_off, nnode, &gop_total, s));
    SETUP_TRY(exclusive_scan(gh_cnt, gh_off, nnode, &gh_total, s));
    const int na = g->na, nm = g->nminus;
    SETUP_TRY(dalloc(&g->aff_node, na)); SETUP_TRY(dalloc(&g->aff_body, na)); SETUP_TRY(dalloc(&g->aff_solid, na));
    SETUP_TRY(dalloc(&g->aff_row_ptr, NY + 1));
    SETUP_TRY(dalloc(&g->gop_ptr, na + 1)); SETUP_TRY(dalloc(&g->gop_idx, gop_total)); SETUP_TRY(dalloc(&g->gop_w, gop_total));
    SETUP_TRY(dalloc(&g->minus_node, nm)); SETUP_TRY(dalloc(&g->gh_ptr, nm + 1));
    SETUP_TRY(dalloc(&g->gh_idx, gh_total)); SETUP_TRY(dalloc(&g->gh_w, gh_total));
    SETUP_TRY(dalloc(&g->minus_cp, 4 * (size_t)nm)); SETUP_TRY(dalloc(&g->minus_mask, nm));
    SETUP_TRY(dalloc(&g->minus_map, npad));
    SETUP_CUDA(cudaMemsetAsync(g->minus_map, 0xff, npad * sizeof(int), s));
    k_fill<<<(unsigned)((nnode + 255) / 256), 256, 0, s>>>(nx, ny, h, phi, g->node_class, aff_pos, minus_pos, gop_off, gh_off,
                                                         epos, tval, n_bodies, g->d_regions, g->aff_node, g->aff_body,
                                                         g->aff_solid, g->gop_idx, g->gop_w, g->minus_node, g->gh_idx,
                                                         g->gh_w, g->minus_cp, g->minus_mask, g->minus_map, err);
    k_ptr_from_offsets<<<(na + 256) / 256, 256, 0, s>>>(na, nx, g->aff_node, gop_off, gop_total, g->gop_ptr);
    k_ptr_from_offsets<<<(nm + 256) / 256, 256, 0, s>>>(nm, nx, g->minus_node, gh_off, gh_total, g->gh_ptr);
    k_row_ptr<<<(NY + 256) / 256, 256, 0, s>>>(NX, NY, na, aff_pos, g->aff_row_ptr);
    if (n_bodies) k_check_regions<<<n_bodies, 256, 0, s>>>(nx, n_bodies, g->d_regions, g->node_class, err);
    SETUP_CUDA(cudaGetLastError());
    SETUP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    int first = 0, last = 0;
    if (na > 0) {
        SETUP_CUDA(cudaMemcpyAsync(&first, g->aff_node, sizeof(int), cudaMemcpyDeviceToHost, s));
        SETUP_CUDA(cudaMemcpyAsync(&last, g->aff_node + na - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    SETUP_CUDA(cudaStreamSynchronize(s));
    if (herr & (ERR_REGION | ERR_FACES)) return fail(IIM_ERR_BAD_REGION);
    if (na > 0) {
        g->ja0 = first / nx; g->ja1 = last / nx;
        g->jo0 = std::max(0, g->ja0 - 4); g->jo1 = std::min(NY - 1, g->ja1 + 4);
    } else {
        g->ja0 = 0; g->ja1 = -1; g->jo0 = 0; g->jo1 = -1;
    }
    // eigenvalues of the 1D operators
    {
        std::vector<double> lx(NX), ly(NY);
        std::vector<float> fx(NX), fy(NY);
        for (int k = 0; k < NX; ++k) { lx[k] = (2.0 - 2.0 * std::cos(M_PI * (k + 1) / nx)) / (h * h); fx[k] = (float)lx[k]; }
        for (int k = 0; k < NY; ++k) { ly[k] = (2.0 - 2.0 * std::cos(M_PI * (k + 1) / ny)) / (h * h); fy[k] = (float)ly[k]; }
        SETUP_TRY(dalloc(&g->lam_x64, NX)); SETUP_TRY(dalloc(&g->lam_y64, NY));
        SETUP_TRY(dalloc(&g->lam_x32, NX)); SETUP_TRY(dalloc(&g->lam_y32, NY));
        SETUP_CUDA(cudaMemcpy(g->lam_x64, lx.data(), NX * sizeof(double), cudaMemcpyHostToDevice));
        SETUP_CUDA(cudaMemcpy(g->lam_y64, ly.data(), NY * sizeof(double), cudaMemcpyHostToDevice));
        SETUP_CUDA(cudaMemcpy(g->lam_x32, fx.data(), NX * sizeof(float), cudaMemcpyHostToDevice));
        SETUP_CUDA(cudaMemcpy(g->lam_y32, fy.data(), NY * sizeof(float), cudaMemcpyHostToDevice));
        SETUP_TRY(scan_tables<float>(nx, NX, NY, 0x1p-26, &g->sc32_delta, &g->sc32_rowoff, &g->sc32_par,
                                     &g->sc32_lim, &g->sc32_dstar));
        float4* unused_par = nullptr;
        SETUP_TRY(scan_tables<double>(nx, NX, NY, 0x1p-53, &g->sc64_delta, &g->sc64_rowoff, &unused_par,
                                      &g->sc64_lim, &g->sc64_dstar));
    }
    // solver workspace
    SETUP_TRY(dalloc(&g->psi_ext, npad));
    SETUP_TRY(dalloc(&g->res, npad));
    SETUP_TRY(dalloc((double**)&g->tbuf, npad));   // sized for FP64, reused for FP32
    SETUP_TRY(dalloc((double**)&g->psiT, npad));
    SETUP_CUDA(cudaMemsetAsync(g->psi_ext, 0, npad * sizeof(double), s));
    SETUP_CUDA(cudaMemsetAsync(g->psiT, 0, npad * sizeof(double), s));
    SETUP_TRY(dalloc(&g->partial, 4096 * 72));
    SETUP_TRY(dalloc(&g->small, 4096));
    SETUP_TRY(dalloc(&g->d_int, 256));   // [32, 96): circulation body ids
    // scalars, counters and flags start at zero (no solve path may read stale memory)
    SETUP_CUDA(cudaMemsetAsync(g->partial, 0, 4096 * 72 * sizeof(double), s));
    SETUP_CUDA(cudaMemsetAsync(g->small, 0, 4096 * sizeof(double), s));
    SETUP_CUDA(cudaMemsetAsync(g->d_int, 0, 256 * sizeof(int), s));
    SETUP_CUDA(cudaMemsetAsync(g->tbuf, 0, npad * sizeof(double), s));
    SETUP_CUDA(cudaMemsetAsync(g->res, 0, npad * sizeof(double), s));
    SETUP_CUDA(cudaMallocHost(&g->h_pinned, 64 * sizeof(double)));
    SETUP_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    SETUP_CUDA(cudaEventCreate(&g->ev0));
    SETUP_CUDA(cudaEventCreate(&g->ev1));
#undef SETUP_TRY
#undef SETUP_CUDA
    fail(IIM_OK);   // frees the temporaries only
    *out = g;
    return IIM_OK;
}

namespace iim {
void free_geometry(iim_geometry g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    destroy_graphs(g);
    void* ptrs[] = {g->cp_x, g->cp_y, g->cp_t, g->cp_body, g->cp_axis, g->cp_ei, g->cp_ej, g->aff_node, g->aff_body,
                    g->aff_row_ptr, g->aff_solid, g->gop_ptr, g->gop_idx, g->gop_w, g->minus_node, g->gh_ptr,
                    g->gh_idx, g->gh_w, g->node_class, g->body_circ, g->d_regions, g->lam_x64, g->lam_y64,
                    g->lam_x32, g->lam_y32, g->sc32_delta, g->sc64_delta, g->sc32_rowoff, g->sc32_lim, g->sc64_rowoff, g->sc64_lim,
                    g->sc32_dstar, g->sc64_dstar, g->sc32_par, g->psi_ext, g->res, g->tbuf, g->psiT, g->partial, g->small, g->V, g->H,
                    g->xsol, g->bvec, g->d_int, g->minus_cp, g->minus_mask, g->minus_map, g->tr_buf,
                    g->pc_aug, g->pc_S, g->psibar_zero, g->pr_buf, g->fs_ring, g->fs_rho, g->fs_bnd, g->fs_rres, g->fs_plane, g->cap_ring, g->pc_f, g->pc_info, g->pc_z, g->x0g, g->cap_psi, g->cap_dev, g->io};
    for (void* p : ptrs) cudaFree(p);
    if (g->h_pinned) cudaFreeHost(g->h_pinned);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    delete g;
    cudaSetDevice(cur);
}
}  // namespace iim

extern "C" void iim_destroy_geometry(iim_geometry g) { iim::free_geometry(g); }

extern "C" iim_status iim_geometry_info(iim_geometry g, int* n_control, int* n_affected, int* n_bodies) {
    if (!g) return IIM_ERR_INVALID_ARG;
    if (n_control) *n_control = g->ncp;
    if (n_affected) *n_affected = g->na;
    if (n_bodies) *n_bodies = g->nb;
    return IIM_OK;
}

namespace iim {
__global__ void k_export_aff(int na, int NX, const int* __restrict__ node, const uint8_t* __restrict__ solid,
                             const int* __restrict__ body, int* oi, int* oj, int* os, int* ob) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= na) return;
    const int n = node[a];   // padded layout
    const int nx = NX + 1;
    if (oi) oi[a] = n % nx;
    if (oj) oj[a] = n / nx + 1;
    if (os) os[a] = solid[a];
    if (ob) ob[a] = body[a];
}
}  // namespace iim

extern "C" iim_status iim_geometry_control_points(iim_geometry g, double* x, double* y, int* body, int* axis,
                                                  int* edge_i, int* edge_j, double* t, iim_stream stream) {
    if (!g) return IIM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = g->ncp;
    if (n == 0) return IIM_OK;
    if (x) IIM_TRY(cudaMemcpyAsync(x, g->cp_x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (y) IIM_TRY(cudaMemcpyAsync(y, g->cp_y, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (t) IIM_TRY(cudaMemcpyAsync(t, g->cp_t, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (body) IIM_TRY(cudaMemcpyAsync(body, g->cp_body, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    if (axis) IIM_TRY(cudaMemcpyAsync(axis, g->cp_axis, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    if (edge_i) IIM_TRY(cudaMemcpyAsync(edge_i, g->cp_ei, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    if (edge_j) IIM_TRY(cudaMemcpyAsync(edge_j, g->cp_ej, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    return IIM_OK;
}

extern "C" iim_status iim_geometry_affected_points(iim_geometry g, int* node_i, int* node_j, int* solid, int* body,
                                                   iim_stream stream) {
    if (!g) return IIM_ERR_INVALID_ARG;
    if (g->na == 0) return IIM_OK;
    k_export_aff<<<(g->na + 255) / 256, 256, 0, (cudaStream_t)stream>>>(g->na, g->NX, g->aff_node, g->aff_solid,
                                                                         g->aff_body, node_i, node_j, solid, body);
    IIM_LAUNCHED();
    return IIM_OK;
}
