// Device bodies of the IIM solve's kernels.  solve.cu wraps each in a kernel that works on
// one problem per launch; lockstep.cu wraps the same bodies in kernels that work on many
// problems of one size per launch (blockIdx.z selects the problem), so that both paths do
// identical arithmetic per problem.
#pragma once

#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "dst.cuh"
#include "tri.cuh"

namespace iim {

// ------------------------------------------------------------------------- transform plan
template <typename T>
struct Plan {
    int NX, NY, nx, ny, lognx, logny;
    const T* lam_x;
    const T* lam_y;
    const cpx<T>* tw;
    T norm;
    int cols_c = 4;   // columns per block of the column pass (tile width)
    int wide = 0;     // 64 threads per 1024-point line instead of one warp
    ScanTab<T> scan{};   // factors of the tridiagonal column pass (lim == nullptr: column transforms)
};

// Algorithmic flops of one DST-I of n - 1 points through an n/2-point complex FFT
// (2.5 n log2(2n): the half-length FFT plus the packing and split steps).
inline double dst_flops(int n) { return 2.5 * n * std::log2(2.0 * n); }

template <typename T>
constexpr int cols_per_block() { return 4; }
constexpr int kRowWarps = 4;

template <typename T>
inline size_t rows_smem(int n, bool wide = false) {
    const int fp = fft_path(n, wide);
    return twiddle_smem<T>(n, fp) + (size_t)kRowWarps * (2 * line_len(n, fp) + kLineScratch) * sizeof(T);
}
template <typename T>
inline size_t cols_smem(int n, int C = cols_per_block<T>(), bool wide = false) {
    const int pad = sizeof(T) == 4 ? 4 : 2;
    const int fp = fft_path(n, wide);
    return twiddle_smem<T>(n, fp) + (size_t)n * sizeof(T) +
           (size_t)C * (2 * line_len(n, fp) + pad + kLineScratch) * sizeof(T);
}
// Rows per block of the row passes for lines of n points.
inline int rows_per_block(int n, bool wide) { return kRowWarps * 32 / line_threads(fft_path(n, wide)); }

// Tile widths the column pass supports: FP32 4 or 8 columns, FP64 2 or 4 (16-byte row segments).
template <typename T>
inline int tile_width(int requested) {
    if (sizeof(T) == 4) return requested >= 8 ? 8 : 4;
    return requested <= 2 ? 2 : 4;
}

// Streaming multiprocessors of the current device (queried once per device).
inline int sm_count() {
    static std::mutex m;
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(m);
    if (dev >= 0 && dev < 64 && cached[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        cached[dev] = v;
    }
    return dev >= 0 && dev < 64 ? cached[dev] : 1;
}

// Raises a kernel's dynamic shared memory limit once per (device, kernel, size).  A failed
// attribute call is reported (IIM_ERR_CUDA) and not recorded, so the next call tries again.
inline std::mutex g_attr_mutex;
inline std::vector<std::pair<std::pair<int, const void*>, size_t>> g_attr_done;

template <typename KernelT>
inline iim_status allow_smem(KernelT k, size_t bytes) {
    int dev = 0;
    IIM_TRY(cudaGetDevice(&dev));
    const void* key = (const void*)k;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    for (auto& e : g_attr_done)
        if (e.first.first == dev && e.first.second == key && e.second >= bytes) return IIM_OK;
    IIM_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    g_attr_done.push_back({{dev, key}, bytes});
    return IIM_OK;
}

// ------------------------------------------------------------------------- reductions
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[BLOCK / 32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (l < BLOCK / 32) ? red[l] : 0.0;
        for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
    }
    return r;   // valid in thread 0
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// small[] layout
enum { SM_RES2 = 0, SM_CIRC_ERR = 1, SM_CIRC = 8, SM_RC = 8 + 64, SM_REG = 8 + 128, SM_NORM = 2048, SM_SEED = 2049,
       SM_CAPC = 2112, SM_CAPP = 2176, SM_FNORM = 2240, SM_REL = 2241 };
constexpr int kRegionParts = 16;

// Device state (int): [0] j (column of the current cycle), [1] stop, [2] iterations of this
// call, [3] max iterations of this call, [4] converged, [5] scratch column index,
// [32, 96) circulation body ids
enum { DI_J = 0, DI_STOP = 1, DI_IT = 2, DI_MAXIT = 3, DI_CONV = 4, DI_TMPJ = 5, DI_LOOP = 6, DI_LOOPERR = 7,
       // device-driven whole solve: refinements, Krylov iterations (all / first correction),
       // cycles of the current correction, cap hits, non-finite residual, cycles and restarts
       DI_REF = 8, DI_ITS = 9, DI_FIRST = 10, DI_CYC = 11, DI_CYCERR = 12, DI_NONFIN = 13, DI_CYCS = 14,
       DI_RSS = 15, DI_CIRC = 32 };

// Krylov small-storage layout inside g->H (m <= 64):
//   H (m+1) x m column-major | cs[m] | sn[m] | gv[m+1] | hc1[m+1] | hc2[m+1] | y[m] | scal[8]
struct KLayout {
    int m;
    __host__ __device__ long H() const { return 0; }
    __host__ __device__ long cs() const { return (long)(m + 1) * m; }
    __host__ __device__ long sn() const { return cs() + m; }
    __host__ __device__ long gv() const { return sn() + m; }
    __host__ __device__ long hc1() const { return gv() + m + 1; }
    __host__ __device__ long hc2() const { return hc1() + m + 1; }
    __host__ __device__ long y() const { return hc2() + m + 1; }
    __host__ __device__ long scal() const { return y() + m; }
    __host__ __device__ long total() const { return scal() + 8; }
};
enum { SC_INV = 0, SC_RESID = 1, SC_BETA = 2, SC_TOL = 3 };

// Arnoldi step finish from the squared norm s of the orthogonalised vector: Hessenberg column
// (the two Gram-Schmidt passes' coefficients summed), Givens rotations, residual estimate,
// stop test.  One thread.
__device__ inline void arnoldi_finish(int* __restrict__ di, KLayout L, double* __restrict__ K, double s) {
    const int j = di[DI_J];
    const double nrm = sqrt(s);
    double* H = K + L.H();
    const int ldh = L.m + 1;
    double* col = H + (long)j * ldh;
    for (int i = 0; i <= j; ++i) col[i] = K[L.hc1() + i] + K[L.hc2() + i];
    col[j + 1] = nrm;
    double* cs = K + L.cs();
    double* sn = K + L.sn();
    double* gv = K + L.gv();
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double d = hypot(col[j], col[j + 1]);
    const double c = d > 0.0 ? col[j] / d : 1.0, sg = d > 0.0 ? col[j + 1] / d : 0.0;
    cs[j] = c;
    sn[j] = sg;
    col[j] = d;
    col[j + 1] = 0.0;
    gv[j + 1] = -sg * gv[j];
    gv[j] = c * gv[j];
    const double resid = fabs(gv[j + 1]);
    K[L.scal() + SC_INV] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    K[L.scal() + SC_RESID] = resid;
    const int jn = j + 1;
    di[DI_J] = jn;
    di[DI_IT] += 1;
    const bool conv = !(resid > K[L.scal() + SC_TOL]);   // also stops on NaN
    if (conv) di[DI_CONV] = 1;
    if (conv || jn >= L.m || di[DI_IT] >= di[DI_MAXIT] || nrm == 0.0) di[DI_STOP] = 1;
}

template <typename T, int BLOCK>
__device__ __forceinline__ void gather_body(int na, int nga, const int* __restrict__ ptr, const int* __restrict__ idx,
                                            const double* __restrict__ w, const T* __restrict__ psi,
                                            const int* __restrict__ cp_body, const int* __restrict__ body_circ,
                                            const int* __restrict__ aff_body, VecArg vin, int use_xc,
                                            double* __restrict__ outb, const int* __restrict__ jidx, long stride,
                                            const int* __restrict__ stop) {
    if (stop && *stop) return;
    const double* v = vin.base ? vin.get() : nullptr;
    double* out = jidx ? outb + (long)(*jidx + 1) * stride : outb;
    if ((int)blockIdx.x < nga) {
        // one warp per affected point, the lanes over its CSR entries
        const int a = blockIdx.x * (BLOCK / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
        if (a >= na) return;
        const double* xc = (use_xc && v) ? v + na : nullptr;
        double acc = 0.0;
        for (int e = ptr[a] + lane; e < ptr[a + 1]; e += 32) {
            const int q = idx[e];
            if (q >= 0) {
                acc += w[e] * (double)psi[q];
            } else if (xc) {
                const int bc = body_circ[cp_body[-q - 1]];
                if (bc >= 0) acc -= w[e] * xc[bc];
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) out[a] = (v ? v[a] : 0.0) + acc;
    } else {
        if (!v) return;
        const int c = blockIdx.x - nga;
        double acc = 0.0;
        for (int a = threadIdx.x; a < na; a += BLOCK)
            if (body_circ[aff_body[a]] == c) acc += v[a];
        acc = block_sum<BLOCK>(acc);
        if (threadIdx.x == 0) out[na + c] = acc;
    }
}

__device__ __forceinline__ void ghost_body(int nm, const int* __restrict__ minus_node, const int* __restrict__ ptr,
                                           const int* __restrict__ idx, const double* __restrict__ w,
                                           const double* __restrict__ psi_b, const double* __restrict__ psibar,
                                           const int* __restrict__ cp_body, double* __restrict__ psi) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nm) return;
    double acc = 0.0;
    for (int e = ptr[m]; e < ptr[m + 1]; ++e) {
        const int q = idx[e];
        if (q >= 0) acc += w[e] * psi[q];
        else {
            const int c = -q - 1;
            acc += w[e] * ((psi_b ? psi_b[c] : 0.0) + psibar[cp_body[c]]);
        }
    }
    psi[minus_node[m]] = acc;
}

template <int BLOCK>
__device__ __forceinline__ void residual_body(int NX, int NY, double ih2, const double* __restrict__ psi,
                                              const double* __restrict__ omega, const uint8_t* __restrict__ cls,
                                              const double* __restrict__ ring, double* __restrict__ res,
                                              double* __restrict__ partial) {
    const int nx = NX + 1;               // a power of two: row index by shift, column by mask
    const int sh = __ffs(nx) - 1;
    const int n = nx * NY;               // < 2^31 for the supported sizes
    double acc = 0.0;
    for (int k = blockIdx.x * BLOCK + threadIdx.x; k < n; k += gridDim.x * BLOCK) {
        const int j = k >> sh, i = (k & (nx - 1)) - 1;
        double r = 0.0;
        if (i >= 0 && cls[k] <= CLS_PLUS) {
            const double c = psi[k];
            const double wv = i > 0 ? psi[k - 1] : (ring ? ring[2 * (NX + 2) + j] : 0.0);
            const double ev = i < NX - 1 ? psi[k + 1] : (ring ? ring[2 * (NX + 2) + NY + j] : 0.0);
            const double sv = j > 0 ? psi[k - nx] : (ring ? ring[i + 1] : 0.0);
            const double nv = j < NY - 1 ? psi[k + nx] : (ring ? ring[(NX + 2) + i + 1] : 0.0);
            r = omega[(long)j * NX + i] - (4.0 * c - wv - ev - sv - nv) * ih2;
            acc += r * r;
        }
        res[k] = r;
    }
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

template <int BLOCK>
__device__ __forceinline__ void region_sums_body(int nx, const double* __restrict__ f,
                                                 const iim_region* __restrict__ R, const int* __restrict__ circ_ids,
                                                 double* __restrict__ partial) {
    const int c = blockIdx.x, part = blockIdx.y, S = gridDim.y;
    const iim_region r = R[circ_ids[c]];
    const int w = r.rx - r.lx + 1, hgt = r.ry - r.ly + 1;
    const long n = (long)w * hgt;
    double acc = 0.0;
    for (long t = (long)part * BLOCK + threadIdx.x; t < n; t += (long)S * BLOCK) {
        const int i = r.lx + (int)(t % w), j = r.ly + (int)(t / w);
        acc += f[(long)(j - 1) * nx + i];
    }
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) partial[c * S + part] = acc;
}

template <int BLOCK>
__device__ __forceinline__ void circ_measure_body(int nx, const double* __restrict__ psi,
                                                  const iim_region* __restrict__ R, const int* __restrict__ circ_ids,
                                                  double* __restrict__ out) {
    const int c = blockIdx.x;
    const iim_region r = R[circ_ids[c]];
    auto P = [&](int i, int j) { return psi[(long)(j - 1) * nx + i]; };
    double acc = 0.0;
    for (int j = r.ly + threadIdx.x; j <= r.ry; j += BLOCK)
        acc += (P(r.rx + 1, j) - P(r.rx, j)) - (P(r.lx, j) - P(r.lx - 1, j));
    for (int i = r.lx + threadIdx.x; i <= r.rx; i += BLOCK)
        acc += (P(i, r.ry + 1) - P(i, r.ry)) - (P(i, r.ly) - P(i, r.ly - 1));
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) out[c] = -acc;
}

template <int BLOCK>
__device__ __forceinline__ void finish_residual_body(int nparts, const double* __restrict__ partial, int ncirc,
                                                     const int* __restrict__ circ_ids,
                                                     const double* __restrict__ gamma, double ih2,
                                                     double* __restrict__ small, const double* __restrict__ regpart,
                                                     double* __restrict__ bcirc, double* __restrict__ out_res2) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += BLOCK) s += partial[b];
    s = block_sum<BLOCK>(s);
    if (threadIdx.x != 0) return;
    double cerr = 0.0;
    for (int c = 0; c < ncirc; ++c) {
        const double gk = gamma ? gamma[circ_ids[c]] : 0.0;
        const double diff = gk - small[SM_CIRC + c];
        cerr = fmax(cerr, fabs(diff));
        const double rc = diff * ih2;
        small[SM_RC + c] = rc;
        s += rc * rc;
        double reg = 0.0;
        for (int p = 0; p < kRegionParts; ++p) reg += regpart[c * kRegionParts + p];
        if (bcirc) bcirc[c] = reg - rc;
    }
    out_res2[0] = s;
    if (out_res2 == small + SM_RES2) small[SM_CIRC_ERR] = cerr;
}

__device__ __forceinline__ void init_psi_body(int NX, int NY, const double* __restrict__ guess,
                                              const uint8_t* __restrict__ cls, double* __restrict__ psi) {
    const int nx = NX + 1;               // a power of two
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nx * NY) return;
    const int j = k >> (__ffs(nx) - 1), i = (k & (nx - 1)) - 1;
    psi[k] = (guess && i >= 0 && cls[k] <= CLS_PLUS) ? guess[(long)j * NX + i] : 0.0;
}

__device__ __forceinline__ void init_psibar_body(int nb, const int* __restrict__ body_circ,
                                                 const double* __restrict__ in, int keep_circ,
                                                 double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= nb) return;
    const double v = in ? in[k] : 0.0;
    out[k] = (body_circ[k] >= 0 && !keep_circ) ? 0.0 : v;
}

__device__ __forceinline__ void add_psibar_body(int ncirc, const int* __restrict__ circ_ids,
                                                const double* __restrict__ x, double* __restrict__ psibar) {
    const int c = threadIdx.x;
    if (c < ncirc) psibar[circ_ids[c]] += x[c];
}

__device__ __forceinline__ void cap_update_body(long npad, int ncirc, const double* __restrict__ resp,
                                                const double* __restrict__ coef, double* __restrict__ psi) {
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npad) return;
    double acc = 0.0;
    for (int l = 0; l < ncirc; ++l) acc += coef[l] * resp[(long)l * npad + p];
    psi[p] += acc;
}

__device__ __forceinline__ void velocity_body(int NX, int NY, double inv2h, const double* __restrict__ psi,
                                              const uint8_t* __restrict__ cls, const double* __restrict__ ring,
                                              double* __restrict__ psi_out, double* __restrict__ ux,
                                              double* __restrict__ uy) {
    const int n = NX * NY;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int nx = NX + 1;
    const int j = k / NX, i = k - j * NX;
    const int p = j * nx + 1 + i;
    const bool fl = cls[p] <= CLS_PLUS;
    if (psi_out) psi_out[k] = fl ? psi[p] : 0.0;
    if (!ux && !uy) return;
    double vx = 0.0, vy = 0.0;
    if (fl) {
        const double wv = i > 0 ? psi[p - 1] : (ring ? ring[2 * (NX + 2) + j] : 0.0);
        const double ev = i < NX - 1 ? psi[p + 1] : (ring ? ring[2 * (NX + 2) + NY + j] : 0.0);
        const double sv = j > 0 ? psi[p - nx] : (ring ? ring[i + 1] : 0.0);
        const double nv = j < NY - 1 ? psi[p + nx] : (ring ? ring[(NX + 2) + i + 1] : 0.0);
        vx = (nv - sv) * inv2h;
        vy = -(ev - wv) * inv2h;
    }
    if (ux) ux[k] = vx;
    if (uy) uy[k] = vy;
}

template <int BLOCK>
__device__ __forceinline__ void arnoldi_block_body(int* __restrict__ di, double* __restrict__ V, long ld, int ns,
                                                   KLayout L, double* __restrict__ K) {
    constexpr int NW = BLOCK / 32;
    if (di[DI_STOP]) return;
    const int j = di[DI_J];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* w = V + (long)(j + 1) * ld;
    __shared__ double part[64][NW];
    __shared__ double h[64];
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i <= j; ++i) {
            const double* vi = V + (long)i * ld;
            double acc = 0.0;
            for (int e = tid; e < ns; e += BLOCK) acc += vi[e] * w[e];
            acc = warp_sum(acc);
            if (lane == 0) part[i][warp] = acc;
        }
        __syncthreads();
        if (tid <= j) {
            double hi = 0.0;
            for (int q = 0; q < NW; ++q) hi += part[tid][q];
            h[tid] = hi;
            K[(pass == 0 ? L.hc1() : L.hc2()) + tid] = hi;
        }
        __syncthreads();
        for (int e = tid; e < ns; e += BLOCK) {
            double sacc = 0.0;
            for (int i = 0; i <= j; ++i) sacc += h[i] * V[(long)i * ld + e];
            w[e] -= sacc;
        }
        __syncthreads();   // h and part are rewritten by the next pass
    }
    double sq = 0.0;
    for (int e = tid; e < ns; e += BLOCK) sq += w[e] * w[e];
    sq = warp_sum(sq);
    if (lane == 0) part[0][warp] = sq;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int q = 0; q < NW; ++q) t += part[0][q];
        arnoldi_finish(di, L, K, t);
    }
    __syncthreads();
    if (di[DI_STOP]) return;
    const double inv = K[L.scal() + SC_INV];
    for (int e = tid; e < ns; e += BLOCK) w[e] *= inv;
}

template <int BLOCK>
__device__ __forceinline__ void start_block_body(int ns, const double* __restrict__ r, double* __restrict__ v0,
                                                 KLayout L, double* __restrict__ K, int* __restrict__ di,
                                                 int init_maxit, double tol, double* __restrict__ norm2) {
    __shared__ double s_inv;
    double acc = 0.0;
    for (int e = threadIdx.x; e < ns; e += BLOCK) acc += r[e] * r[e];
    acc = block_sum<BLOCK>(acc);
    if (threadIdx.x == 0) {
        if (init_maxit >= 0) {
            *norm2 = acc;
            di[DI_J] = 0;
            di[DI_STOP] = 0;
            di[DI_IT] = 0;
            di[DI_MAXIT] = init_maxit;
            di[DI_CONV] = 0;
            di[DI_TMPJ] = 0;
            di[DI_LOOP] = 0;
            di[DI_LOOPERR] = 0;
            K[L.scal() + SC_TOL] = tol * sqrt(acc);
        }
        const double beta = sqrt(acc);
        double* gv = K + L.gv();
        gv[0] = beta;
        for (int i = 1; i <= L.m; ++i) gv[i] = 0.0;
        K[L.scal() + SC_BETA] = beta;
        K[L.scal() + SC_RESID] = beta;
        di[DI_J] = 0;
        di[DI_STOP] = (di[DI_IT] >= di[DI_MAXIT]) ? 1 : 0;
        if (!(beta > K[L.scal() + SC_TOL])) { di[DI_CONV] = 1; di[DI_STOP] = 1; }
        s_inv = beta > 0.0 ? 1.0 / beta : 0.0;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int e = threadIdx.x; e < ns; e += BLOCK) v0[e] = r[e] * inv;
}

template <int BLOCK>
__device__ __forceinline__ void backsolve_update_body(const int* __restrict__ di, KLayout L, double* __restrict__ K,
                                                      const double* __restrict__ V, long ld, int ns,
                                                      double* __restrict__ out, int accumulate) {
    const int k = di[DI_J];
    double* y = K + L.y();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const double* H = K + L.H();
        const int ldh = L.m + 1;
        const double* gv = K + L.gv();
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
    __syncthreads();
    for (int e = threadIdx.x; e < ns; e += BLOCK) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += y[i] * V[(long)i * ld + e];
        out[e] = accumulate ? out[e] + s : 0.0 + s;
    }
}

__device__ __forceinline__ void cap_coef_body(int nc, const double* __restrict__ rc, const double* __restrict__ cinv,
                                              const double* __restrict__ pb, double h2, double* __restrict__ coef,
                                              double* __restrict__ dpb) {
    __shared__ double c_sh[64];
    const int t = threadIdx.x;
    if (t < nc) {
        double a = 0.0;
        for (int k = 0; k < nc; ++k) a += cinv[t * nc + k] * (rc[k] * h2);
        c_sh[t] = a;
        coef[t] = a;
    }
    __syncthreads();
    if (t < nc) {
        double d = 0.0;
        for (int l = 0; l < nc; ++l) d += c_sh[l] * pb[l * nc + t];
        dpb[t] = d;
    }
}

__device__ __forceinline__ void final_rel_body(int* __restrict__ di, double* __restrict__ small) {
    const double r2 = small[SM_RES2], fn = small[SM_FNORM];
    if (!isfinite(r2)) di[DI_NONFIN] = 1;
    small[SM_REL] = fn > 0.0 ? sqrt(r2) / fn : 0.0;
}

// z = M v for the dense FP32 preconditioner (one warp per row, v staged in shared memory).
template <int WARPS>
__device__ __forceinline__ void
dense_matvec4_body(int n, const float* __restrict__ M, long ldm, const double* __restrict__ vbase,
                   const int* __restrict__ jidx, long vstride, double* __restrict__ out, int accumulate,
                   const int* __restrict__ stop, const int* __restrict__ ojidx = nullptr, long ostride = 0) {
    if (stop && *stop) return;
    if (ojidx) out += (long)(*ojidx + 1) * ostride;   // out = column j + 1 of a Krylov basis
    extern __shared__ float4 s_v4[];
    float* s_v = reinterpret_cast<float*>(s_v4);
    const int stride = (n + 3) & ~3;
    const double* v = jidx ? vbase + (long)(*jidx) * vstride : vbase;
    for (int j = threadIdx.x; j < n; j += WARPS * 32) {
        const float x = (float)v[j];
#pragma unroll
        for (int h = 0; h < 4; ++h)
            if (j >= h) s_v[h * stride + j - h] = x;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int row = blockIdx.x * WARPS + (threadIdx.x >> 5); row < n; row += gridDim.x * WARPS) {
        const float* r = M + (long)row * ldm;
        const int head = min((int)((4 - ((reinterpret_cast<uintptr_t>(r) >> 2) & 3)) & 3), n);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (lane < head) a0 = r[lane] * s_v[lane];
        const float4* r4 = reinterpret_cast<const float4*>(r + head);
        const float4* v4 = reinterpret_cast<const float4*>(s_v + head * stride);
        const int nq = (n - head) >> 2;
        int q = lane;
        // the at most seven vectors of the remainder loop are loaded first, so that they are in
        // flight together with the main batches; the sums keep the order of the loops below
        int qr = lane;
        while (qr + 7 * 32 < nq) qr += 8 * 32;
        float4 xr[7];
#pragma unroll
        for (int u = 0; u < 7; ++u) {
            const int qq = qr + 32 * u;
            xr[u] = qq < nq ? r4[qq] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (; q + 7 * 32 < nq; q += 8 * 32) {
            float4 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = r4[q + 32 * u];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 y = v4[q + 32 * u];
                float& a = (u & 3) == 0 ? a0 : (u & 3) == 1 ? a1 : (u & 3) == 2 ? a2 : a3;
                a = fmaf(x[u].x, y.x, fmaf(x[u].y, y.y, fmaf(x[u].z, y.z, fmaf(x[u].w, y.w, a))));
            }
        }
#pragma unroll
        for (int u = 0; u < 7; ++u) {
            const int qq = qr + 32 * u;   // qr == q here
            if (qq < nq) {
                const float4 x = xr[u], y = v4[qq];
                a1 = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, a1))));
            }
        }
        const int rem = (n - head) & 3;
        if (lane < rem) {
            const int idx = head + 4 * nq + lane;
            a2 = fmaf(r[idx], s_v[idx], a2);
        }
        float acc = (a0 + a1) + (a2 + a3);
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) out[row] = accumulate ? out[row] + (double)acc : (double)acc;
    }
}

// ------------------------------------------------------------------------- graph capture
// Stream capture into an existing graph in pieces, so that conditional nodes can be placed
// between the pieces: `deps` is the frontier the next node depends on.
struct CapSeg {
    cudaStream_t s;
    cudaGraph_t graph;
    std::vector<cudaGraphNode_t> deps;
    cudaError_t begin() {
        return cudaStreamBeginCaptureToGraph(s, graph, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                             cudaStreamCaptureModeThreadLocal);
    }
    cudaError_t end() {
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* d = nullptr;
        size_t nd = 0;
        cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &d, nullptr, &nd);
        std::vector<cudaGraphNode_t> tail;
        if (e == cudaSuccess && d) tail.assign(d, d + nd);
        cudaGraph_t out = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s, &out);
        if (e == cudaSuccess && e2 == cudaSuccess) deps = tail;
        return e != cudaSuccess ? e : e2;
    }
    // a conditional node after the frontier; *body receives its body graph
    cudaError_t cond(cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, cudaGraph_t* body) {
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = type;
        p.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        cudaError_t e = cudaGraphAddNode(&node, graph, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p);
        if (e == cudaSuccess) {
            deps.assign(1, node);
            *body = p.conditional.phGraph_out[0];
        }
        return e;
    }
};

// Kernel nodes directly in a graph (not inside its conditional bodies).
inline long long kernel_nodes(cudaGraph_t graph) {
    size_t n = 0;
    if (cudaGraphGetNodes(graph, nullptr, &n) != cudaSuccess || n == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(graph, nodes.data(), &n) != cudaSuccess) return 0;
    long long k = 0;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

}  // namespace iim
