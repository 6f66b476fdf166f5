// Batched DST-I kernels for the Dirichlet-box Poisson solve (Sec. 4.2: the rectangular
// solution operator; the box is Dirichlet as for the paper's internal flows, Sec. 6.4).
//
// With N = n - 1 unknowns on a line, X_k = sum_{j=1}^{N} x_j sin(pi j k / n).  The 2D
// solve of -nabla_h^2 u = f with homogeneous box data is
//   u = (2/nx)(2/ny) S_y S_x [ (S_y S_x f) / (lam_x(k) + lam_y(l)) ],
//   lam(k) = (2 - 2 cos(pi k / n)) / h^2.
//
// One warp transforms one line held in shared memory.  The transform uses the sine packing
// of a real sequence into a half-length complex FFT (the published "sine transform via a
// real FFT" construction): y_j = sin(j pi/n)(x_j + x_{n-j}) + (x_j - x_{n-j})/2; the real FFT
// of y (an n/2-point complex FFT of the pairs (y_2m, y_2m+1) plus the split step) gives
// X_{2k} = -Im Y_k and X_{2k+1} - X_{2k-1} = Re Y_k, the odd outputs by a prefix sum.
// The n/2-point FFT is a Stockham autosort FFT (radix 8, then 4 / 2), ping-ponging between
// the line buffer and one scratch buffer; the packing is fused into the first pass.
//
// Internal row layout ("padded"): interior row r of an (NY x NX) field occupies
// [r*nx, r*nx + nx); element i sits at r*nx + 1 + i and slot r*nx is a zero pad, so that
// every row starts on a 16-byte boundary and maps one-to-one onto a DST line buffer.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace iim {

template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
// multiplication by -i
template <typename T>
__device__ __forceinline__ cpx<T> cmi(cpx<T> a) { return {a.y, -a.x}; }

// exp(-i pi t / n) for 0 <= t < 2n from the half table tw[t], t < n
template <typename T>
__device__ __forceinline__ cpx<T> tw_full(const cpx<T>* tw, int t, int n) {
    if (t < n) return tw[t];
    const cpx<T> w = tw[t - n];
    return {-w.x, -w.y};
}

// In-place forward R-point DFT (sign e^{-i}).
template <typename T, int R>
__device__ __forceinline__ void dft(cpx<T>* v);

template <typename T>
struct Dft2 {
    static __device__ __forceinline__ void run(cpx<T>* v) {
        const cpx<T> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <>
__device__ __forceinline__ void dft<float, 2>(cpx<float>* v) { Dft2<float>::run(v); }
template <>
__device__ __forceinline__ void dft<double, 2>(cpx<double>* v) { Dft2<double>::run(v); }

template <typename T>
__device__ __forceinline__ void dft4_impl(cpx<T>* v) {
    const cpx<T> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const cpx<T> t2 = cadd(v[1], v[3]), t3 = cmi(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
}
template <>
__device__ __forceinline__ void dft<float, 4>(cpx<float>* v) { dft4_impl(v); }
template <>
__device__ __forceinline__ void dft<double, 4>(cpx<double>* v) { dft4_impl(v); }

template <typename T>
__device__ __forceinline__ void dft8_impl(cpx<T>* v) {
    cpx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cpx<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft4_impl(e);
    dft4_impl(o);
    const T r = T(0.70710678118654752440);
    // W8^1 = (1 - i)/sqrt2, W8^2 = -i, W8^3 = (-1 - i)/sqrt2
    const cpx<T> o1 = {r * (o[1].x + o[1].y), r * (o[1].y - o[1].x)};
    const cpx<T> o2 = cmi(o[2]);
    const cpx<T> o3 = {r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y)};
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}
template <>
__device__ __forceinline__ void dft<float, 8>(cpx<float>* v) { dft8_impl(v); }
template <>
__device__ __forceinline__ void dft<double, 8>(cpx<double>* v) { dft8_impl(v); }

// Packed FFT input c_m = y_{2m} + i y_{2m+1} from the line x (x_0 = x_n = 0).
template <typename T>
__device__ __forceinline__ cpx<T> packed(const T* x, const cpx<T>* tw, int n, int m) {
    const int j0 = 2 * m, j1 = j0 + 1;
    T y0 = T(0);
    if (j0 != 0) {
        const T a = x[j0], b = x[n - j0];
        y0 = (-tw[j0].y) * (a + b) + T(0.5) * (a - b);
    }
    const T a1 = x[j1], b1 = x[n - j1];
    const T y1 = (-tw[j1].y) * (a1 + b1) + T(0.5) * (a1 - b1);
    return {y0, y1};
}

// One Stockham radix-R pass of an M-point FFT: in -> out (out-of-place).  With `x` given the
// input values are the packed line instead of `in`.
template <typename T, int R>
__device__ __forceinline__ void stockham_pass(const cpx<T>* in, const T* x, cpx<T>* out, const cpx<T>* tw, int n,
                                              int M, int Ns, int lane) {
    const int J = M / R;
    const int tstep = (4 * M) / (Ns * R);
    for (int j = lane; j < J; j += 32) {
        cpx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x ? packed(x, tw, n, j + r * J) : in[j + r * J];
        const int k = j & (Ns - 1);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw_full(tw, tstep * k * r, n));
        }
        dft<T, R>(v);
        const int idx = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[idx + r * Ns] = v[r];
    }
    __syncwarp();
}

// DST-I of the line held in buf0[1..n-1] (buf0[0] ignored), with buf1 (n values) as scratch.
// tw[k] = exp(-i pi k / n), k < n.  Returns the buffer holding the result in [1..n-1].
template <typename T>
__device__ __forceinline__ T* dst1_warp(T* buf0, T* buf1, const cpx<T>* tw, int n, int logn, int lane) {
    const int M = n >> 1;
    const int logM = logn - 1;
    // FFT passes: radix 8 while possible, then 4 or 2
    T* src = buf0;
    T* dst = buf1;
    int Ns = 1, rem = logM;
    bool first = true;
    while (rem > 0) {
        const cpx<T>* in = reinterpret_cast<const cpx<T>*>(src);
        cpx<T>* out = reinterpret_cast<cpx<T>*>(dst);
        const T* px = first ? src : nullptr;
        if (rem >= 3) { stockham_pass<T, 8>(in, px, out, tw, n, M, Ns, lane); Ns *= 8; rem -= 3; }
        else if (rem == 2) { stockham_pass<T, 4>(in, px, out, tw, n, M, Ns, lane); Ns *= 4; rem -= 2; }
        else { stockham_pass<T, 2>(in, px, out, tw, n, M, Ns, lane); Ns *= 2; rem -= 1; }
        first = false;
        T* t = src; src = dst; dst = t;
    }
    // src holds C_k (natural order); split step into dst
    const cpx<T>* C = reinterpret_cast<const cpx<T>*>(src);
    for (int k = lane; k < M; k += 32) {
        const cpx<T> ck = C[k];
        const cpx<T> cm = C[k == 0 ? 0 : M - k];
        const T ex = T(0.5) * (ck.x + cm.x), ey = T(0.5) * (ck.y - cm.y);
        const T dx = T(0.5) * (ck.x - cm.x), dy = T(0.5) * (ck.y + cm.y);
        const cpx<T> w = tw[2 * k];
        const T yx = ex + (w.x * dy + w.y * dx);
        const T yy = ey + (w.y * dy - w.x * dx);
        reinterpret_cast<cpx<T>*>(dst)[k] = cpx<T>{k == 0 ? T(0) : -yy, k == 0 ? T(0.5) * yx : yx};
    }
    __syncwarp();
    // odd outputs: inclusive prefix sum of dst[2m+1], m = 0..M-1, 32 values per step
    T carry = T(0);
    for (int base = 0; base < M; base += 32) {
        const int m = base + lane;
        T v = m < M ? dst[2 * m + 1] : T(0);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T u = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += u;
        }
        v += carry;
        if (m < M) dst[2 * m + 1] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
    __syncwarp();
    return dst;
}

// Copies exp(-i pi k / n), k < n, from the 4096-entry table into shared memory; the loads of
// one thread are issued back to back (batches of 8) before their shared-memory stores.
template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* s_tw, const cpx<T>* g_tw, int n, int logn) {
    const int stride_shift = kTwLog - logn;
    const int nt = blockDim.x;
    for (int k0 = threadIdx.x; k0 < n; k0 += 8 * nt) {
        cpx<T> v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int k = k0 + b * nt;
            if (k < n) v[b] = g_tw[k << stride_shift];
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int k = k0 + b * nt;
            if (k < n) s_tw[k] = v[b];
        }
    }
}

template <typename T>
using vec16_t = typename std::conditional<sizeof(T) == 4, float4, double2>::type;

// Loads nx values of a padded row (16-byte aligned) into a line buffer with vector loads,
// batches of 8 loads in flight per lane.
template <typename T>
__device__ __forceinline__ void load_row_vec(T* line, const T* __restrict__ g, int nx, int lane) {
    constexpr int V = 16 / sizeof(T);
    using VT = vec16_t<T>;
    const VT* src = reinterpret_cast<const VT*>(g);
    VT* dst = reinterpret_cast<VT*>(line);
    const int nv = nx / V;
    for (int q0 = lane; q0 < nv; q0 += 8 * 32) {
        VT v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (q0 + 32 * b < nv) v[b] = src[q0 + 32 * b];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (q0 + 32 * b < nv) dst[q0 + 32 * b] = v[b];
    }
}

template <typename T>
__device__ __forceinline__ void store_row_vec(T* __restrict__ g, const T* line, int nx, int lane) {
    constexpr int V = 16 / sizeof(T);
    using VT = vec16_t<T>;
    const VT* src = reinterpret_cast<const VT*>(line);
    VT* dst = reinterpret_cast<VT*>(g);
    const int nv = nx / V;
#pragma unroll 4
    for (int q = lane; q < nv; q += 32) dst[q] = src[q];
}

// Loads a padded FP64 row (16-byte aligned, nx values) into a line buffer of T.
template <typename T>
__device__ __forceinline__ void load_row_f64(T* line, const double* __restrict__ g, int nx, int lane) {
    const double2* src = reinterpret_cast<const double2*>(g);
    const int nv = nx / 2;
    for (int q0 = lane; q0 < nv; q0 += 8 * 32) {
        double2 v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (q0 + 32 * b < nv) v[b] = src[q0 + 32 * b];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int q = q0 + 32 * b;
            if (q < nv) {
                line[2 * q] = (T)v[b].x;
                line[2 * q + 1] = (T)v[b].y;
            }
        }
    }
}

// Krylov-vector argument: base + (jidx ? *jidx + joff : 0) * stride
struct VecArg {
    const double* base;
    const int* jidx;
    int joff;
    long stride;
    __device__ __forceinline__ const double* get() const {
        return jidx ? base + (long)(*jidx + joff) * stride : base;
    }
};

// Forward row transforms.  Row r (interior row index) of the input is
//   dense[r*dld + doff + i] (FP64, optional) + box terms / h^2 (optional ring)
//   + gsign * gamma at the affected points of the row (optional)
// and the transformed row is written to out (padded layout).  `stop` (optional): a set flag
// makes the launch a no-op.
template <typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_rows_fwd(int NX, int NY, int n, int logn, int row0, int nrows, const double* __restrict__ dense, int dld, int doff,
           const double* __restrict__ ring, double ih2, const int* __restrict__ aff_row_ptr,
           const int* __restrict__ aff_node, VecArg gam, double gsign, const cpx<T>* __restrict__ g_tw,
           T* __restrict__ out, const int* __restrict__ stop) {
    if (stop && *stop) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* s_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* b0 = reinterpret_cast<T*>(s_tw + n) + (size_t)warp * (2 * n);
    T* b1 = b0 + n;
    load_twiddles(s_tw, g_tw, n, logn);
    __syncthreads();
    const int r = row0 + blockIdx.x * WARPS + warp;
    if (r >= row0 + nrows || r >= NY) return;
    if (dense && dld == n && doff == 1) {
        load_row_f64(b0, dense + (size_t)r * n, n, lane);   // padded row: slot 0 is a pad
    } else if (dense) {
        const double* src = dense + (size_t)r * dld + doff;
#pragma unroll 8
        for (int i = lane; i < NX; i += 32) b0[i + 1] = (T)src[i];
    } else {
        for (int i = lane; i < NX; i += 32) b0[i + 1] = T(0);
    }
    __syncwarp();
    if (ring) {
        // ring: bottom row (nx+1), top row (nx+1), left column (ny-1), right column (ny-1)
        const int nxp1 = NX + 2;
        if (lane == 0) {
            b0[1] += (T)(ring[2 * nxp1 + r] * ih2);
            b0[NX] += (T)(ring[2 * nxp1 + NY + r] * ih2);
        }
        __syncwarp();
        if (r == 0)
            for (int i = lane; i < NX; i += 32) b0[i + 1] += (T)(ring[i + 1] * ih2);
        if (r == NY - 1)
            for (int i = lane; i < NX; i += 32) b0[i + 1] += (T)(ring[nxp1 + i + 1] * ih2);
        __syncwarp();
    }
    if (gam.base) {
        const double* gv = gam.get();
        const int a0 = aff_row_ptr[r], a1 = aff_row_ptr[r + 1];
        for (int a = a0 + lane; a < a1; a += 32) b0[aff_node[a] - r * n] += (T)(gsign * gv[a]);
        __syncwarp();
    }
    T* res = dst1_warp(b0, b1, s_tw, n, logn, lane);
    if (lane == 0) res[0] = T(0);
    __syncwarp();
    store_row_vec(out + (size_t)r * n, res, n, lane);
}

// Column pass on padded columns p = 1..NX (p = 0 is the pad): forward y transform, division
// by the eigenvalues (with the 2D normalisation), inverse y transform.  Rows outside [in0, in1]
// are zero on input; only rows [out0, out1] are written back.  C columns per block, one warp
// per column; blockIdx.y selects one of several fields fstride elements apart.
template <typename T, int C>
__global__ void __launch_bounds__(C * 32)
k_cols(int NX, int NY, int n, int logn, int in0, int in1, int out0, int out1, T* __restrict__ buf,
       const T* __restrict__ lam_x, const T* __restrict__ lam_y, T norm, const cpx<T>* __restrict__ g_tw,
       const int* __restrict__ stop, long fstride) {
    if (stop && *stop) return;
    buf += (long)blockIdx.y * fstride;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* s_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    constexpr int PAD = sizeof(T) == 4 ? 4 : 2;
    const int stride = 2 * n + PAD;
    T* lines = reinterpret_cast<T*>(s_tw + n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ld = NX + 1;
    const int col0 = blockIdx.x * C;   // padded column index
    load_twiddles(s_tw, g_tw, n, logn);
    // tile load: C consecutive padded columns of rows [in0, in1]; rows outside are zero
    constexpr int V = 16 / sizeof(T);
    constexpr int VPR = C / V;                   // vectors per row
    using VT = vec16_t<T>;
    const int nthr = C * 32;
    const int total = NY * VPR;
    for (int t0 = threadIdx.x; t0 < total; t0 += 8 * nthr) {
        VT v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int t = t0 + b * nthr;
            const int rr = t / VPR;
            v[b] = VT{};
            if (t < total && rr >= in0 && rr <= in1)
                v[b] = *reinterpret_cast<const VT*>(buf + (size_t)rr * ld + col0 + (t - rr * VPR) * V);
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int t = t0 + b * nthr;
            if (t < total) {
                const int rr = t / VPR, q = t - rr * VPR;
                const T* vs = reinterpret_cast<const T*>(&v[b]);
#pragma unroll
                for (int c = 0; c < V; ++c) lines[(q * V + c) * stride + rr + 1] = vs[c];
            }
        }
    }
    __syncthreads();
    const int p = col0 + warp;
    T* resline = nullptr;
    if (p >= 1 && p <= NX) {
        T* b0 = lines + warp * stride;
        T* b1 = b0 + n;
        T* f = dst1_warp(b0, b1, s_tw, n, logn, lane);
        const T lx = lam_x[p - 1];
        for (int l = lane; l < NY; l += 32) f[l + 1] = f[l + 1] * (norm / (lx + lam_y[l]));
        __syncwarp();
        T* other = (f == b0) ? b1 : b0;
        resline = dst1_warp(f, other, s_tw, n, logn, lane);
        // bring the result back to b0 so that the tile store below has a fixed layout
        if (resline != b0) {
            for (int l = lane; l < NY; l += 32) b0[l + 1] = resline[l + 1];
        }
    }
    __syncthreads();
    const int nout = out1 - out0 + 1;
    for (int t = threadIdx.x; t < nout * VPR; t += C * 32) {
        const int rr = out0 + t / VPR, q = t % VPR;
        VT v;
        T* vs = reinterpret_cast<T*>(&v);
#pragma unroll
        for (int c = 0; c < V; ++c) {
            const int pc = col0 + q * V + c;
            vs[c] = (pc >= 1 && pc <= NX) ? lines[(q * V + c) * stride + rr + 1] : T(0);
        }
        *reinterpret_cast<VT*>(buf + (size_t)rr * ld + col0 + q * V) = v;
    }
}

enum RowsInvMode { INV_STORE_T = 0, INV_STORE_F64 = 1, INV_ACCUM_FLUID = 2 };

// Inverse row transforms of rows [row0, row0 + nrows) of a padded buffer.
//   INV_STORE_T     outT (padded) = transform
//   INV_STORE_F64   out64[r*old + ooff + i] = transform
//   INV_ACCUM_FLUID out64 (padded) += transform at fluid nodes (class FLUID / PLUS) only
// blockIdx.y selects one of several fields fstride elements apart (in and outT).
template <typename T, int WARPS, int MODE>
__global__ void __launch_bounds__(WARPS * 32)
k_rows_inv(int NX, int NY, int n, int logn, int row0, int nrows, const T* __restrict__ in, T* __restrict__ outT,
           double* __restrict__ out64, int old, int ooff, const uint8_t* __restrict__ cls,
           const cpx<T>* __restrict__ g_tw, const int* __restrict__ stop, long fstride) {
    if (stop && *stop) return;
    in += (long)blockIdx.y * fstride;
    if (outT) outT += (long)blockIdx.y * fstride;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* s_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* b0 = reinterpret_cast<T*>(s_tw + n) + (size_t)warp * (2 * n);
    T* b1 = b0 + n;
    load_twiddles(s_tw, g_tw, n, logn);
    __syncthreads();
    const int r = row0 + blockIdx.x * WARPS + warp;
    if (r >= row0 + nrows || r >= NY) return;
    load_row_vec(b0, in + (size_t)r * n, n, lane);
    __syncwarp();
    T* res = dst1_warp(b0, b1, s_tw, n, logn, lane);
    if (MODE == INV_STORE_T) {
        if (lane == 0) res[0] = T(0);
        __syncwarp();
        store_row_vec(outT + (size_t)r * n, res, n, lane);
    } else if (MODE == INV_STORE_F64) {
        double* dst = out64 + (size_t)r * old + ooff;
#pragma unroll 4
        for (int i = lane; i < NX; i += 32) dst[i] = (double)res[i + 1];
    } else {
        const size_t base = (size_t)r * n;
#pragma unroll 4
        for (int i = lane; i < NX; i += 32)
            if (cls[base + 1 + i] <= CLS_PLUS) out64[base + 1 + i] += (double)res[i + 1];
    }
}

}  // namespace iim
