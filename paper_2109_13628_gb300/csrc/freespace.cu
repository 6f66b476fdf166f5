// Free-space (unbounded) rectangular solve: the operator nabla_h^-2 with unbounded conditions
// on the edge of the box (Sec. 4.1: psi from the convolution of the source with a Green's
// function whose constant fixes the gauge; Sec. 4.2: the FFT solution operator with unbounded
// boundary conditions).
//
// On the grid, psi(x) = h^2 sum_y G(x - y) f(y) with G the lattice Green's function of the
// five-point Laplacian (-L G = delta on Z^2, L = sum of the four neighbours minus four times the
// centre, gauge G(0, 0) = 0).  It is evaluated by James's method, which needs only the
// Dirichlet-box solver of the library and one boundary sum:
//   1. psi_1 = box solve of f with zero box data.  Extended by zero outside the box, psi_1 has
//      -nabla_h^2 psi_1 = f + q with the screening charge q = -psi_1(neighbour) / h^2 on the
//      box ring (each non-corner ring node has one interior neighbour), and a compact function
//      is the lattice potential of its own charge: psi_1 = G * (f + q).
//   2. So G * f = psi_1 - G * q.  On the ring, psi_1 = 0 and
//      rho(x) = -(G * q)(x) = sum_{y on the ring} G(x - y) psi_1(neighbour of y).
//   3. Inside the box, -G * q is harmonic with boundary values rho: the box solve of a zero
//      source with box data rho.  psi = psi_1 + that solve, and psi = rho on the ring.
// This file holds the lattice Green's function table, the extraction of psi_1 next to the box
// and the ring sum; solve.cu strings them together with the box solves.
//
// Outflow plane (Sec. 5.2): the vorticity mirrored evenly across the vertical plane through
// the right box edge (node column nx).  The mirrored interior sources are a field harmonic
// inside the box whose values on the ring are those of the free-space field at the mirror
// points, so the ring kernel becomes K(x, y) = G(x - y) + G(x* - y), x* = (2 nx - i, j) (table
// columns up to 2 nx); sources on the plane column are their own images and are data: their
// potential h^2 sum_j G(x - (nx, j)) w_j enters the ring equations, and through them the
// correction of each refinement.
//
// The table G(m, n), 0 <= m <= nx, 0 <= n <= ny, depends on the lattice only (not on h), so it
// is built once per (device, nx, ny) and shared by every geometry of that size:
//   max(m, n) < 64: -G(m, n) = (1 / 2 pi) int_0^pi (1 - cos(m t) e^(-n a)) / sinh(a) dt,
//     cosh a = 2 - cos t (the Fourier representation with one integral done in closed form),
//     by 256 uniform panels of 16-point Gauss-Legendre in FP64;
//   otherwise the far-field expansion
//     G = -(1/2 pi)(log r + euler_gamma + (3/2) log 2) + cos(4 phi) / (24 pi r^2)
//         + (18 cos(4 phi) + 25 cos(8 phi)) / (480 pi r^4) + O(r^-6),
//     accurate to about 2e-12 at r = 64 and better beyond (checked against the quadrature).
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "iim_ops.cuh"

namespace iim {

constexpr int kLgfQuadRadius = 64;   // max(|m|, |n|) below which G is integrated
constexpr int kLgfPanels = 256;

struct GaussRule {
    double x[16], w[16];
};

// 16-point Gauss-Legendre rule on [-1, 1]: Newton iteration on the Legendre polynomial P_16 from
// the Chebyshev guesses; weights 2 / ((1 - x^2) P_16'(x)^2).
static GaussRule gauss16() {
    GaussRule g;
    const int n = 16;
    for (int i = 0; i < n; ++i) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        g.x[i] = x;
        g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return g;
}

__device__ double lgf_quadrature(int m, int n, const GaussRule& R) {
    double acc = 0.0;
    const double hw = 0.5 * M_PI / kLgfPanels;
    for (int p = 0; p < kLgfPanels; ++p) {
        const double mid = (2 * p + 1) * hw;
        double pacc = 0.0;
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
            const double t = mid + hw * R.x[q];
            const double st = sin(0.5 * t);
            const double eps = 2.0 * st * st;                       // cosh a - 1 = 1 - cos t
            const double a = log1p(eps + sqrt(eps * (2.0 + eps)));   // acosh(1 + eps) without cancellation
            const double sm = sin(0.5 * m * t);
            const double num = 2.0 * sm * sm - cos(m * t) * expm1(-n * a);
            pacc += R.w[q] * num / sinh(a);
        }
        acc += pacc * hw;
    }
    return -acc / (2.0 * M_PI);
}

__device__ double lgf_far(int m, int n) {
    const double r2 = (double)m * m + (double)n * n;
    const double r = sqrt(r2);
    const double c4 = ((double)m * m * m * m - 6.0 * m * m * (double)n * n + (double)n * n * n * n) / (r2 * r2);
    const double c8 = 2.0 * c4 * c4 - 1.0;
    const double euler_gamma = 0.57721566490153286061;
    return -(log(r) + euler_gamma + 1.5 * log(2.0)) / (2.0 * M_PI) + c4 / (24.0 * M_PI * r2) +
           (18.0 * c4 + 25.0 * c8) / (480.0 * M_PI * r2 * r2);
}

// G[n * (M + 1) + m] for 0 <= m <= M, 0 <= n <= N
__global__ void k_lgf_table(int M, int N, GaussRule R, double* __restrict__ G) {
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long)(M + 1) * (N + 1)) return;
    const int m = (int)(k % (M + 1)), n = (int)(k / (M + 1));
    double v = 0.0;
    if (m == 0 && n == 0) v = 0.0;
    else if (m < kLgfQuadRadius && n < kLgfQuadRadius) v = lgf_quadrature(m, n, R);
    else v = lgf_far(m, n);
    G[k] = v;
}

static std::mutex g_lgf_mutex;
static std::map<std::tuple<int, int, int>, double*> g_lgf_tables;

// The table G(m, n), 0 <= m <= nx, 0 <= n <= ny (row stride nx + 1), on the current device
// (built on first use, kept until the process exits).  Synchronizes the device on first use.
iim_status lgf_table(int nx, int ny, const double** out) {
    int dev = 0;
    IIM_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_lgf_mutex);
    auto key = std::make_tuple(dev, nx, ny);
    auto it = g_lgf_tables.find(key);
    if (it != g_lgf_tables.end()) {
        *out = it->second;
        return IIM_OK;
    }
    double* G = nullptr;
    const long n = (long)(nx + 1) * (ny + 1);
    IIM_TRY(cudaMalloc(&G, sizeof(double) * n));
    const GaussRule R = gauss16();
    launch("lgf_table", 0.0, 0.0, k_lgf_table, (unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)0, nx, ny, R, G);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(G);
        record_cuda_error(e, "lgf_table", __FILE__, __LINE__);
        return IIM_ERR_CUDA;
    }
    g_lgf_tables[key] = G;
    *out = G;
    return IIM_OK;
}

// psi_1 next to the left and right box edges, from the column-processed buffer (row j holds the
// x-sine coefficients c_k of psi_1's row j, slots 1..NX of the padded row):
//   psi_1(first interior column, j) = sum_k c_k sin(pi k / nx),
//   psi_1(last interior column, j)  = sum_k c_k (-1)^(k+1) sin(pi k / nx).
// One warp per row.
template <typename T>
__global__ void k_bnd_cols(int NX, int NY, int nx, const T* __restrict__ buf, double* __restrict__ vl,
                           double* __restrict__ vr, const int* __restrict__ stop) {
    if (stop && *stop) return;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= NY) return;
    const T* row = buf + (size_t)j * nx + 1;
    double a = 0.0, b = 0.0;
    for (int k = lane; k < NX; k += 32) {
        const double c = (double)row[k] * sinpi((double)(k + 1) / nx);
        a += c;
        b += (k & 1) ? -c : c;   // (-1)^(k+2) for mode k + 1
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        vl[j] = a;
        vr[j] = b;
    }
}

// rho(x) = sum over the non-corner ring nodes y of K(x, y) psi_1(neighbour of y), for every
// ring node x (ring layout: bottom j = 0, i = 0..nx; top j = ny; left i = 0, j = 1..ny-1; right
// i = nx), K(x, y) = G(x - y) (+ G(x* - y) with the outflow plane, sym); G has row stride ld.
// bnd: psi_1 on the first interior row (NX values) then on the last (NX values); vl, vr: psi_1
// on the first and last interior columns (NY values each).  One block per x.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_ring_conv(int nx, int ny, const double* __restrict__ G, int ld, int sym, const double* __restrict__ bnd,
            const double* __restrict__ vl, const double* __restrict__ vr, double* __restrict__ rho,
            const int* __restrict__ stop) {
    if (stop && *stop) return;
    const int t = blockIdx.x;
    int xi, xj;
    if (t <= nx) { xi = t; xj = 0; }
    else if (t <= 2 * nx + 1) { xi = t - (nx + 1); xj = ny; }
    else if (t < 2 * (nx + 1) + (ny - 1)) { xi = 0; xj = t - 2 * (nx + 1) + 1; }
    else { xi = nx; xj = t - 2 * (nx + 1) - (ny - 1) + 1; }
    const int NX = nx - 1, NY = ny - 1;
    const int nsrc = 2 * NX + 2 * NY;
    double acc = 0.0;
    for (int s = threadIdx.x; s < nsrc; s += BLOCK) {
        int si, sj;
        double v;
        if (s < NX) { si = s + 1; sj = 0; v = bnd[s]; }
        else if (s < 2 * NX) { si = s - NX + 1; sj = ny; v = bnd[s]; }
        else if (s < 2 * NX + NY) { si = 0; sj = s - 2 * NX + 1; v = vl[sj - 1]; }
        else { si = nx; sj = s - 2 * NX - NY + 1; v = vr[sj - 1]; }
        const size_t row = (size_t)abs(xj - sj) * ld;
        double k = G[row + abs(xi - si)];
        if (sym) k += G[row + abs(2 * nx - xi - si)];
        acc += k * v;
    }
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) rho[t] = acc;
}

// y += a x over n values (ring updates)
__global__ void k_ring_add(int n, double a, const double* __restrict__ x, double* __restrict__ y,
                           const int* __restrict__ stop) {
    if (stop && *stop) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) y[k] += a * x[k];
}

// Ring equations of the free-space system (the FP64 residual's ring rows).  For the free-space
// potential of sources inside the box, the discrete Green's second identity on the interior
// nodes, with G(x - .) harmonic there for x on the ring, gives
//   psi(x) = sum over the non-corner ring nodes z of G(x - z) psi(n(z)) - G(x - n(z)) psi(z),
// n(z) the interior neighbour of z; a field harmonic inside the box leaves exactly its ring
// values in  rres(x) = psi(x) - that sum,  so a ring error that the interior rows cannot see
// shows here.  With the outflow plane (sym) the kernel is K(x, y) = G(x - y) + G(x* - y) (the
// mirrored part is harmonic inside the box, and so is G(x* - .)), and the potential of the
// plane sources, h^2 sum_j G(x - (nx, j)) plane_j (harmonic inside), is the data of the row and
// is subtracted (plane null: no plane sources).  psi: padded interior field; ring: psi on the
// ring.  One block per ring node.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_ring_residual(int nx, int ny, double h2, const double* __restrict__ G, int ld, int sym,
                const double* __restrict__ plane, const double* __restrict__ psi, const double* __restrict__ ring,
                double* __restrict__ rres) {
    const int t = blockIdx.x;
    int xi, xj;
    if (t <= nx) { xi = t; xj = 0; }
    else if (t <= 2 * nx + 1) { xi = t - (nx + 1); xj = ny; }
    else if (t < 2 * (nx + 1) + (ny - 1)) { xi = 0; xj = t - 2 * (nx + 1) + 1; }
    else { xi = nx; xj = t - 2 * (nx + 1) - (ny - 1) + 1; }
    const int NX = nx - 1, NY = ny - 1;
    const int nsrc = 2 * NX + 2 * NY;
    auto K = [&](int yi, int yj) {
        const size_t row = (size_t)abs(xj - yj) * ld;
        double k = G[row + abs(xi - yi)];
        if (sym) k += G[row + abs(2 * nx - xi - yi)];
        return k;
    };
    double acc = 0.0;
    for (int s = threadIdx.x; s < nsrc; s += BLOCK) {
        int zi, zj, ai, aj, zr;   // ring node, its interior neighbour, its ring index
        if (s < NX) { zi = s + 1; zj = 0; ai = zi; aj = 1; zr = zi; }
        else if (s < 2 * NX) { zi = s - NX + 1; zj = ny; ai = zi; aj = ny - 1; zr = nx + 1 + zi; }
        else if (s < 2 * NX + NY) { zi = 0; zj = s - 2 * NX + 1; ai = 1; aj = zj; zr = 2 * (nx + 1) + zj - 1; }
        else { zi = nx; zj = s - 2 * NX - NY + 1; ai = nx - 1; aj = zj; zr = 2 * (nx + 1) + NY + zj - 1; }
        const double pa = psi[(size_t)(aj - 1) * nx + ai];
        acc += K(zi, zj) * pa - K(ai, aj) * ring[zr];
    }
    if (sym && plane) {
        for (int j = 1 + threadIdx.x; j <= NY; j += BLOCK)
            acc += h2 * G[(size_t)abs(xj - j) * ld + abs(xi - nx)] * plane[j - 1];
    }
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) rres[t] = ring[t] - acc;
}

// *res2 += scale2 sum_t rres[t]^2 (one block)
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_ring_res_norm(int n, const double* __restrict__ rres, double scale2, double* __restrict__ res2) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < n; t += BLOCK) acc += rres[t] * rres[t];
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) *res2 += scale2 * acc;
}

template <typename T>
iim_status launch_bnd_cols(int NX, int NY, int nx, const T* buf, double* vl, double* vr, const int* stop,
                           cudaStream_t s) {
    launch("free_bnd_cols", (double)NX * NY * sizeof(T), 4.0 * NX * NY, k_bnd_cols<T>, (NY + 7) / 8, 256, 0, s, NX, NY,
           nx, buf, vl, vr, stop);
    IIM_LAUNCHED();
    return IIM_OK;
}
template iim_status launch_bnd_cols<float>(int, int, int, const float*, double*, double*, const int*, cudaStream_t);
template iim_status launch_bnd_cols<double>(int, int, int, const double*, double*, double*, const int*, cudaStream_t);

iim_status launch_ring_conv(int nx, int ny, const double* G, int ld, int sym, const double* bnd, const double* vl,
                            const double* vr, double* rho, const int* stop, cudaStream_t s) {
    const double nsrc = 2.0 * (nx - 1) + 2.0 * (ny - 1);
    launch("free_ring_conv", 0.0, (sym ? 4.0 : 2.0) * nsrc * 2.0 * (nx + ny), k_ring_conv<256>, 2 * (nx + ny), 256, 0, s,
           nx, ny, G, ld, sym, bnd, vl, vr, rho, stop);
    IIM_LAUNCHED();
    return IIM_OK;
}

iim_status launch_ring_add(int n, double a, const double* x, double* y, const int* stop, cudaStream_t s) {
    launch("free_ring_add", 0.0, 0.0, k_ring_add, (n + 255) / 256, 256, 0, s, n, a, x, y, stop);
    IIM_LAUNCHED();
    return IIM_OK;
}

iim_status launch_ring_residual(int nx, int ny, double h, const double* G, int ld, int sym, const double* plane,
                                const double* psi, const double* ring, double* rres, double* res2, cudaStream_t s) {
    const int n = 2 * (nx + ny);
    launch("free_ring_residual", 0.0, 0.0, k_ring_residual<256>, n, 256, 0, s, nx, ny, h * h, G, ld, sym, plane, psi,
           ring, rres);
    launch("free_ring_res_norm", 0.0, 0.0, k_ring_res_norm<256>, 1, 256, 0, s, n, (const double*)rres,
           1.0 / (h * h * h * h), res2);
    IIM_LAUNCHED();
    return IIM_OK;
}

}  // namespace iim
