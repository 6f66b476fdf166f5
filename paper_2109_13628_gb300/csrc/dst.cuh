// Batched DST-I kernels for the Dirichlet-box Poisson solve (Sec. 4.2: the rectangular
// solution operator; the box is Dirichlet as for the paper's internal flows, Sec. 6.4).
//
// With N = n - 1 unknowns on a line, X_k = sum_{j=1}^{N} x_j sin(pi j k / n).  The 2D
// solve of -nabla_h^2 u = f with homogeneous box data is
//   u = (2/nx)(2/ny) S_y S_x [ (S_y S_x f) / (lam_x(k) + lam_y(l)) ],
//   lam(k) = (2 - 2 cos(pi k / n)) / h^2.
//
// One warp transforms one line held in shared memory.  The transform uses the sine
// packing of a real sequence into a half-length complex FFT (the published "sine transform
// via real FFT" construction): y_j = sin(j pi/n)(x_j + x_{n-j}) + (x_j - x_{n-j})/2, a real
// FFT of y (an n/2-point complex FFT of the even/odd pairs plus the split step) gives
// X_{2k} = -Im Y_k and X_{2k+1} - X_{2k-1} = Re Y_k, the odd outputs by a prefix sum.
#pragma once

#include "common.cuh"

namespace iim {

// x[0..n-1]: line data in x[1..n-1] (x[0] ignored), transformed in place.
// c: n/2 complex scratch.  tw[k] = exp(-i pi k / n), k < n (shared memory).
template <typename T>
__device__ __forceinline__ void dst1_warp(T* x, cpx<T>* c, const cpx<T>* tw, int n, int logM, int lane) {
    const int M = n >> 1;
    // packing: c_m = y_{2m} + i y_{2m+1}, stored bit-reversed for the in-place DIT FFT
    for (int m = lane; m < M; m += 32) {
        const int j0 = 2 * m, j1 = 2 * m + 1;
        T y0 = T(0);
        if (j0 != 0) {
            const T a = x[j0], b = x[n - j0];
            y0 = (-tw[j0].y) * (a + b) + T(0.5) * (a - b);
        }
        const T a1 = x[j1], b1 = x[n - j1];
        const T y1 = (-tw[j1].y) * (a1 + b1) + T(0.5) * (a1 - b1);
        const int r = (int)(__brev((unsigned)m) >> (32 - logM));
        c[r] = cpx<T>{y0, y1};
    }
    __syncwarp();
    // radix-2 decimation-in-time stages, twiddle W_span^k = tw[k * 4M / span]
    for (int s = 1; s <= logM; ++s) {
        const int half = 1 << (s - 1);
        const int tshift = 2 + logM - s;
        for (int b = lane; b < (M >> 1); b += 32) {
            const int k = b & (half - 1);
            const int i0 = ((b >> (s - 1)) << s) + k;
            const int i1 = i0 + half;
            const cpx<T> w = tw[k << tshift];
            const cpx<T> u = c[i0];
            const cpx<T> v = cmul(w, c[i1]);
            c[i0] = cpx<T>{u.x + v.x, u.y + v.y};
            c[i1] = cpx<T>{u.x - v.x, u.y - v.y};
        }
        __syncwarp();
    }
    // split step: Y_k = E_k + W_n^k O_k; X_{2k} = -Im Y_k, R_k = Re Y_k kept in x[2k+1]
    for (int k = lane; k < M; k += 32) {
        const cpx<T> ck = c[k];
        const cpx<T> cm = c[k == 0 ? 0 : M - k];
        const T ex = T(0.5) * (ck.x + cm.x), ey = T(0.5) * (ck.y - cm.y);
        const T dx = T(0.5) * (ck.x - cm.x), dy = T(0.5) * (ck.y + cm.y);
        // O = -i D = (dy, -dx)
        const cpx<T> w = tw[2 * k];
        const T yx = ex + (w.x * dy + w.y * dx);
        const T yy = ey + (w.y * dy - w.x * dx);
        x[2 * k] = (k == 0) ? T(0) : -yy;
        x[2 * k + 1] = (k == 0) ? T(0.5) * yx : yx;
    }
    __syncwarp();
    // odd outputs: inclusive prefix sum over x[1], x[3], ..., x[2M-1]
    const int chunk = (M + 31) >> 5;
    const int lo = lane * chunk;
    const int hi = min(M, lo + chunk);
    T sum = T(0);
    for (int m = lo; m < hi; ++m) sum += x[2 * m + 1];
    T incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    T acc = incl - sum;
    for (int m = lo; m < hi; ++m) {
        acc += x[2 * m + 1];
        x[2 * m + 1] = acc;
    }
    __syncwarp();
}

// Copies exp(-i pi k / n), k < n, from the 4096-entry table into shared memory.
template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* s_tw, const cpx<T>* g_tw, int n, int logn) {
    const int stride_shift = kTwLog - logn;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s_tw[k] = g_tw[k << stride_shift];
}

// Forward row transforms.  Row r (interior row index) of the input is
//   dense[r, :] (FP64, optional) + box terms / h^2 (optional ring) + gsign * E_a gamma (optional)
// and the transformed row is written to out[r, :].
template <typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_rows_fwd(int NX, int NY, int n, int logn, int row0, int nrows, const double* __restrict__ dense,
           const double* __restrict__ ring, double ih2, const int* __restrict__ aff_row_ptr,
           const int* __restrict__ aff_node, const double* __restrict__ gam, double gsign,
           const cpx<T>* __restrict__ g_tw, T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* s_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* x = reinterpret_cast<T*>(s_tw + n) + (size_t)warp * (2 * n);
    cpx<T>* c = reinterpret_cast<cpx<T>*>(x + n);
    load_twiddles(s_tw, g_tw, n, logn);
    __syncthreads();
    const int r = row0 + blockIdx.x * WARPS + warp;
    if (r >= row0 + nrows || r >= NY) return;
    const size_t base = (size_t)r * NX;
    for (int i = lane; i < NX; i += 32) x[i + 1] = dense ? (T)dense[base + i] : T(0);
    if (lane == 0) x[0] = T(0);
    __syncwarp();
    if (ring) {
        // ring: bottom row (nx+1), top row (nx+1), left column (ny-1), right column (ny-1)
        const int nxp1 = NX + 2;
        if (lane == 0) {
            x[1] += (T)(ring[2 * nxp1 + r] * ih2);
            x[NX] += (T)(ring[2 * nxp1 + NY + r] * ih2);
        }
        __syncwarp();
        if (r == 0)
            for (int i = lane; i < NX; i += 32) x[i + 1] += (T)(ring[i + 1] * ih2);
        if (r == NY - 1)
            for (int i = lane; i < NX; i += 32) x[i + 1] += (T)(ring[nxp1 + i + 1] * ih2);
        __syncwarp();
    }
    if (gam) {
        const int a0 = aff_row_ptr[r], a1 = aff_row_ptr[r + 1];
        for (int a = a0 + lane; a < a1; a += 32) {
            const int i = aff_node[a] - r * NX;
            x[i + 1] += (T)(gsign * gam[a]);
        }
        __syncwarp();
    }
    dst1_warp(x, c, s_tw, n, logn - 1, lane);
    for (int i = lane; i < NX; i += 32) out[base + i] = x[i + 1];
}

// Column pass: forward y transform, division by the eigenvalues (with the 2D normalisation),
// inverse y transform.  Rows outside [in0, in1] are zero on input; only rows [out0, out1]
// are written back.  C columns per block, one warp per column.
template <typename T, int C>
__global__ void __launch_bounds__(C * 32)
k_cols(int NX, int NY, int n, int logn, int in0, int in1, int out0, int out1, T* __restrict__ buf,
       const T* __restrict__ lam_x, const T* __restrict__ lam_y, T norm, const cpx<T>* __restrict__ g_tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* s_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    constexpr int PAD = sizeof(T) == 4 ? 4 : 2;   // bank-conflict-free transposed load / store
    const int stride = 2 * n + PAD;
    T* lines = reinterpret_cast<T*>(s_tw + n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col0 = blockIdx.x * C;
    load_twiddles(s_tw, g_tw, n, logn);
    for (int idx = threadIdx.x; idx < NY * C; idx += C * 32) {
        const int rr = idx / C, cc = idx - rr * C;
        const int col = col0 + cc;
        T v = T(0);
        if (col < NX && rr >= in0 && rr <= in1) v = buf[(size_t)rr * NX + col];
        lines[cc * stride + rr + 1] = v;
    }
    __syncthreads();
    const int col = col0 + warp;
    if (col < NX) {
        T* x = lines + warp * stride;
        cpx<T>* c = reinterpret_cast<cpx<T>*>(x + n);
        dst1_warp(x, c, s_tw, n, logn - 1, lane);
        const T lx = lam_x[col];
        for (int l = lane; l < NY; l += 32) x[l + 1] = x[l + 1] * norm / (lx + lam_y[l]);
        __syncwarp();
        dst1_warp(x, c, s_tw, n, logn - 1, lane);
    }
    __syncthreads();
    const int nout = out1 - out0 + 1;
    for (int idx = threadIdx.x; idx < nout * C; idx += C * 32) {
        const int rr = out0 + idx / C, cc = idx % C;
        const int col2 = col0 + cc;
        if (col2 < NX) buf[(size_t)rr * NX + col2] = lines[cc * stride + rr + 1];
    }
}

enum RowsInvMode { INV_STORE_T = 0, INV_STORE_F64 = 1, INV_ACCUM_FLUID = 2 };

// Inverse row transforms of rows [row0, row0 + nrows).
//   INV_STORE_T     outT[r, :] = transform
//   INV_STORE_F64   out64[r, :] = transform
//   INV_ACCUM_FLUID out64[r, i] += transform at fluid nodes (class FLUID / PLUS) only
template <typename T, int WARPS, int MODE>
__global__ void __launch_bounds__(WARPS * 32)
k_rows_inv(int NX, int NY, int n, int logn, int row0, int nrows, const T* __restrict__ in,
           T* __restrict__ outT, double* __restrict__ out64, const uint8_t* __restrict__ cls,
           const cpx<T>* __restrict__ g_tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* s_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* x = reinterpret_cast<T*>(s_tw + n) + (size_t)warp * (2 * n);
    cpx<T>* c = reinterpret_cast<cpx<T>*>(x + n);
    load_twiddles(s_tw, g_tw, n, logn);
    __syncthreads();
    const int r = row0 + blockIdx.x * WARPS + warp;
    if (r >= row0 + nrows || r >= NY) return;
    const size_t base = (size_t)r * NX;
    for (int i = lane; i < NX; i += 32) x[i + 1] = in[base + i];
    if (lane == 0) x[0] = T(0);
    __syncwarp();
    dst1_warp(x, c, s_tw, n, logn - 1, lane);
    for (int i = lane; i < NX; i += 32) {
        const T v = x[i + 1];
        if (MODE == INV_STORE_T) {
            outT[base + i] = v;
        } else if (MODE == INV_STORE_F64) {
            out64[base + i] = (double)v;
        } else {
            if (cls[base + i] <= CLS_PLUS) out64[base + i] += (double)v;
        }
    }
}

}  // namespace iim
