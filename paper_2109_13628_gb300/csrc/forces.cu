// Control-volume force and moment on a stationary immersed body (App. C: Noca's momentum
// formulation, Eq. Fm with its tensor gamma, and the moment formulation of Eqs. Mm1 / Mm2),
// density 1, as a post-processing kernel on the solve's outputs.
//
// The control volume is the node box [lx, rx] x [ly, ry] minus the body; its outer surface is
// the box's four node lines (trapezoidal rule), derivatives there are centred differences.  With
// D = div T = nu (-d omega/dy, d omega/dx) and T = nu (grad u + grad u^T), and x measured from the
// moment centre, the surface integrands are
//   n.gamma = |u|^2/2 n - (n.u) u - (n.u) omega (y, -x) + (x.D) n - (n.x) D + T n,
//   lambda  = |u|^2/2 (x cross n) - (x cross u)(u.n) + |x|^2/2 omega (n.u)
//             + |x|^2/2 (D cross n) + x cross (T n).
// The time-differentiated integrals are returned as instantaneous values (the caller
// differentiates a time series): A = int_V u and P = int_V x cross u through the streamfunction
// (psi is constant, psi_w, on a stationary no-slip body and its gradient vanishes there):
//   A = (oint psi n_y, -oint psi n_x),  P = -oint psi (x.n) + 2 int_box psi~,
// psi~ = psi in the fluid and psi_w in the body (continuously differentiable: the box sum is second
// order, and the body's area cancels); B = oint x cross (n cross u), Q = oint |x|^2/2 (n cross u).
// Then F = -dA/dt - dB/dt + oint n.gamma and M = -dP/dt + dQ/dt + oint lambda.
#include <vector>

#include "common.cuh"
#include "iim_ops.cuh"

namespace iim {

struct CvBox {
    int lx, rx, ly, ry, nx, NX;
    double h, x0, y0, xb, yb, nu, psi_w;
};

// Trapezoidal sum of psi~ over the box nodes: per-block partial sums.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_cv_area(CvBox b, const double* __restrict__ psi, const uint8_t* __restrict__ cls, double* __restrict__ partial) {
    const int w = b.rx - b.lx + 1, hgt = b.ry - b.ly + 1;
    const long n = (long)w * hgt;
    double acc = 0.0;
    for (long t = (long)blockIdx.x * BLOCK + threadIdx.x; t < n; t += (long)gridDim.x * BLOCK) {
        const int i = b.lx + (int)(t % w), j = b.ly + (int)(t / w);
        const bool solid = cls[(size_t)(j - 1) * b.nx + i] >= CLS_MINUS;
        const double p = solid ? b.psi_w : psi[(size_t)(j - 1) * b.NX + (i - 1)];
        const double wgt = (i == b.lx || i == b.rx ? 0.5 : 1.0) * (j == b.ly || j == b.ry ? 0.5 : 1.0);
        acc += wgt * p;
    }
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// The edge integrals (nine quantities) and the box sum; out[9] = 1 when an edge node or one of
// its neighbours is not plain fluid (the box must keep clear of the body).  One block.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_cv_edges(CvBox b, const double* __restrict__ psi, const double* __restrict__ uu, const double* __restrict__ vv,
           const double* __restrict__ ww, const uint8_t* __restrict__ cls, int nparts,
           const double* __restrict__ partial, double* __restrict__ out) {
    const int nxe = b.rx - b.lx + 1, nye = b.ry - b.ly + 1;
    const int total = 2 * nxe + 2 * nye;
    const double h = b.h;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int bad = 0;
    auto I = [&](int i, int j) { return (size_t)(j - 1) * b.NX + (i - 1); };
    for (int t = threadIdx.x; t < total; t += BLOCK) {
        int i, j, k, len;
        double nx_, ny_;
        if (t < nxe) { i = b.lx + t; j = b.ly; nx_ = 0; ny_ = -1; k = t; len = nxe; }
        else if (t < 2 * nxe) { i = b.lx + t - nxe; j = b.ry; nx_ = 0; ny_ = 1; k = t - nxe; len = nxe; }
        else if (t < 2 * nxe + nye) { i = b.lx; j = b.ly + t - 2 * nxe; nx_ = -1; ny_ = 0; k = t - 2 * nxe; len = nye; }
        else { i = b.rx; j = b.ly + t - 2 * nxe - nye; nx_ = 1; ny_ = 0; k = t - 2 * nxe - nye; len = nye; }
        const int di[5] = {0, 1, -1, 0, 0}, dj[5] = {0, 0, 0, 1, -1};
        for (int q = 0; q < 5; ++q)
            if (cls[(size_t)(j + dj[q] - 1) * b.nx + i + di[q]] != CLS_FLUID) bad = 1;
        const double wgt = (k == 0 || k == len - 1 ? 0.5 : 1.0) * h;
        const double x = b.x0 + h * i - b.xb, y = b.y0 + h * j - b.yb;
        const double u = uu[I(i, j)], v = vv[I(i, j)], w = ww[I(i, j)], p = psi[I(i, j)];
        const double inv2h = 0.5 / h;
        const double ux = (uu[I(i + 1, j)] - uu[I(i - 1, j)]) * inv2h, uy = (uu[I(i, j + 1)] - uu[I(i, j - 1)]) * inv2h;
        const double vx = (vv[I(i + 1, j)] - vv[I(i - 1, j)]) * inv2h, vy = (vv[I(i, j + 1)] - vv[I(i, j - 1)]) * inv2h;
        const double wx = (ww[I(i + 1, j)] - ww[I(i - 1, j)]) * inv2h, wy = (ww[I(i, j + 1)] - ww[I(i, j - 1)]) * inv2h;
        const double Txx = 2 * b.nu * ux, Txy = b.nu * (uy + vx), Tyy = 2 * b.nu * vy;
        const double Dx = -b.nu * wy, Dy = b.nu * wx;
        const double un = nx_ * u + ny_ * v, q2 = 0.5 * (u * u + v * v), nxu = nx_ * v - ny_ * u;
        const double Tnx = Txx * nx_ + Txy * ny_, Tny = Txy * nx_ + Tyy * ny_;
        const double r2 = x * x + y * y, xD = x * Dx + y * Dy, nxv = nx_ * x + ny_ * y;
        acc[0] += wgt * p * ny_;
        acc[1] += wgt * -p * nx_;
        acc[2] += wgt * nxu * y;
        acc[3] += wgt * -nxu * x;
        acc[4] += wgt * (q2 * nx_ - un * u - un * w * y + xD * nx_ - nxv * Dx + Tnx);
        acc[5] += wgt * (q2 * ny_ - un * v + un * w * x + xD * ny_ - nxv * Dy + Tny);
        acc[6] += wgt * -p * nxv;
        acc[7] += wgt * 0.5 * r2 * nxu;
        acc[8] += wgt * (q2 * (x * ny_ - y * nx_) - (x * v - y * u) * un + 0.5 * r2 * w * un +
                         0.5 * r2 * (Dx * ny_ - Dy * nx_) + (x * Tny - y * Tnx));
    }
    __shared__ double red[9];
    for (int c = 0; c < 9; ++c) {
        const double s = block_sum<BLOCK>(acc[c]);
        if (threadIdx.x == 0) red[c] = s;
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        double area = 0.0;
        for (int k = 0; k < nparts; ++k) area += partial[k];
        for (int c = 0; c < 9; ++c) out[c] = red[c];
        out[6] += 2.0 * h * h * area;
        out[9] = bad ? 1.0 : 0.0;
    }
}

}  // namespace iim

using namespace iim;

extern "C" iim_status iim_cv_terms(iim_geometry g, const double* psi, const double* ux, const double* uy,
                                   const double* omega, double psi_wall, const iim_region* box, double nu,
                                   const double xbar[2], double* out, iim_stream stream) {
    if (!g || !psi || !ux || !uy || !omega || !box || !xbar || !out) return IIM_ERR_INVALID_ARG;
    const iim_region r = *box;
    if (r.lx < 2 || r.ly < 2 || r.rx > g->nx - 2 || r.ry > g->ny - 2 || r.rx <= r.lx || r.ry <= r.ly)
        return IIM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    constexpr int kParts = 128;
    double* dev = nullptr;
    IIM_TRY(cudaMallocAsync((void**)&dev, sizeof(double) * (kParts + 10), s));
    const CvBox b{r.lx, r.rx, r.ly, r.ry, g->nx, g->NX, g->h, g->grid.x0, g->grid.y0, xbar[0], xbar[1], nu, psi_wall};
    launch("cv_area", 0.0, 0.0, k_cv_area<256>, kParts, 256, 0, s, b, psi, (const uint8_t*)g->node_class, dev);
    launch("cv_edges", 0.0, 0.0, k_cv_edges<256>, 1, 256, 0, s, b, psi, ux, uy, omega, (const uint8_t*)g->node_class,
           kParts, (const double*)dev, dev + kParts);
    cudaError_t e = cudaGetLastError();
    double host[10];
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, dev + kParts, sizeof(double) * 10, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(dev, s);
    if (e != cudaSuccess) {
        record_cuda_error(e, "iim_cv_terms", __FILE__, __LINE__);
        return IIM_ERR_CUDA;
    }
    if (host[9] != 0.0) return IIM_ERR_BAD_REGION;
    for (int c = 0; c < 9; ++c) out[c] = host[c];
    return IIM_OK;
}
