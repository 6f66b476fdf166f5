// Dense Schur-complement preconditioner kernels: Gauss-Jordan inversion with partial pivoting
// of the (n x n) matrix S held in the left half of a row-major n x 2n augmented array [S | I],
// and the dense FP32 matrix-vector product used to apply the inverse.
//
// S = I + A P E_a (with the circulation rows) is the operator of Sec. 4.2; its inverse turns
// each correction solve into one dense product (the capacitance-matrix view of the same linear
// system); inside GMRES it is a right preconditioner, so the iteration still measures the
// residual of the exact operator.
#include <cmath>

#include <cstdint>

#include "common.cuh"

namespace iim {

// Pivot search in column k over rows k..n-1, row swap, scaling of the pivot row, and the
// multipliers f[i] = A[i][k] (after the swap) for the elimination kernel.  One block.
template <int BLOCK>
__global__ void k_gj_pivot(float* __restrict__ A, int n, int k, float* __restrict__ f, int* __restrict__ info) {
    if (*info) return;
    const long ld = 2L * n;
    __shared__ float sv[BLOCK];
    __shared__ int si[BLOCK];
    float best = -1.f;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += BLOCK) {
        const float v = fabsf(A[(long)i * ld + k]);
        if (v > best) { best = v; bi = i; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = BLOCK / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const float o = sv[threadIdx.x + s];
            const int oi = si[threadIdx.x + s];
            if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = o;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int p = si[0];
    const float piv_abs = sv[0];
    if (!(piv_abs > 0.f)) {
        if (threadIdx.x == 0) *info = k + 1;
        return;
    }
    if (p != k) {
        for (long c = threadIdx.x; c < ld; c += BLOCK) {
            const float a = A[(long)k * ld + c];
            A[(long)k * ld + c] = A[(long)p * ld + c];
            A[(long)p * ld + c] = a;
        }
    }
    __syncthreads();
    const float inv = 1.f / A[(long)k * ld + k];
    __syncthreads();
    for (long c = threadIdx.x; c < ld; c += BLOCK) A[(long)k * ld + c] *= inv;
    for (int i = threadIdx.x; i < n; i += BLOCK) f[i] = (i == k) ? 0.f : A[(long)i * ld + k];
}

// A[i][c] -= f[i] * A[k][c] for every row i != k (f[k] = 0), columns c >= k of the left half
// and every column of the right half.
__global__ void k_gj_eliminate(float* __restrict__ A, int n, int k, const float* __restrict__ f, const int* __restrict__ info) {
    if (*info) return;
    const long ld = 2L * n;
    const int i = blockIdx.y;
    const float m = f[i];
    if (m == 0.f) return;
    const float* rk = A + (long)k * ld;
    float* ri = A + (long)i * ld;
    for (long c = k + (long)blockIdx.x * blockDim.x + threadIdx.x; c < ld; c += (long)gridDim.x * blockDim.x)
        ri[c] -= m * rk[c];
}

__global__ void k_set_identity_aug(float* __restrict__ A, int n) {
    const long ld = 2L * n;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    const long i = t / n, j = t - i * n;
    A[i * ld + n + j] = (i == j) ? 1.f : 0.f;
}

// out = M v (+ out when accumulate), M row-major n x n FP32 with leading dimension ldm (even);
// one warp per row.  v = vbase + (jidx ? *jidx : 0) * vstride is staged in shared memory as
// FP32; each lane reads the row in 8-byte pairs (after one odd leading element when the row
// starts 4 bytes off an 8-byte boundary) into four independent accumulators.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_dense_matvec(int n, const float* __restrict__ M, long ldm, const double* __restrict__ vbase,
               const int* __restrict__ jidx, long vstride, double* __restrict__ out, int accumulate,
               const int* __restrict__ stop) {
    if (stop && *stop) return;
    extern __shared__ float s_v[];
    const double* v = jidx ? vbase + (long)(*jidx) * vstride : vbase;
    for (int j = threadIdx.x; j < n; j += WARPS * 32) s_v[j] = (float)v[j];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int row = blockIdx.x * WARPS + (threadIdx.x >> 5); row < n; row += gridDim.x * WARPS) {
        const float* r = M + (long)row * ldm;
        const int head = (reinterpret_cast<uintptr_t>(r) & 7) ? 1 : 0;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (head && lane == 0) a0 = r[0] * s_v[0];
        const float2* r2 = reinterpret_cast<const float2*>(r + head);
        const float* sv = s_v + head;
        const int np = (n - head) >> 1;
        int q = lane;
        for (; q + 96 < np; q += 128) {
            const float2 x0 = r2[q], x1 = r2[q + 32], x2 = r2[q + 64], x3 = r2[q + 96];
            a0 = fmaf(x0.x, sv[2 * q], fmaf(x0.y, sv[2 * q + 1], a0));
            a1 = fmaf(x1.x, sv[2 * q + 64], fmaf(x1.y, sv[2 * q + 65], a1));
            a2 = fmaf(x2.x, sv[2 * q + 128], fmaf(x2.y, sv[2 * q + 129], a2));
            a3 = fmaf(x3.x, sv[2 * q + 192], fmaf(x3.y, sv[2 * q + 193], a3));
        }
        for (; q < np; q += 32) {
            const float2 x0 = r2[q];
            a0 = fmaf(x0.x, sv[2 * q], fmaf(x0.y, sv[2 * q + 1], a0));
        }
        if (((n - head) & 1) && lane == 31) a1 = fmaf(r[n - 1], s_v[n - 1], a1);
        float acc = (a0 + a1) + (a2 + a3);
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) out[row] = accumulate ? out[row] + (double)acc : (double)acc;
    }
}

iim_status gj_invert_aug(float* A, int n, float* f, int* info, cudaStream_t s) {
    IIM_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
    launch("gj_identity", 0.0, 0.0, k_set_identity_aug, (unsigned)(((long)n * n + 255) / 256), 256, 0, s, A, n);
    const int cblocks = (int)std::min<long>(32, (2L * n + 255) / 256);
    for (int k = 0; k < n; ++k) {
        launch("gj_pivot", 0.0, 0.0, k_gj_pivot<512>, 1, 512, 0, s, A, n, k, f, info);
        launch("gj_eliminate", 0.0, 0.0, k_gj_eliminate, dim3(cblocks, n), 256, 0, s, A, n, k, (const float*)f,
               (const int*)info);
    }
    IIM_LAUNCHED();
    return IIM_OK;
}

iim_status dense_matvec(int n, const float* M, long ldm, const double* v, const int* jidx, long vstride, double* out,
                        int accumulate, const int* stop, cudaStream_t s) {
    constexpr int W = 8;
    const size_t sm = sizeof(float) * (size_t)n;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_dense_matvec<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    launch("precond_matvec", (double)n * n * 4.0, 2.0 * n * n, k_dense_matvec<W>, (n + W - 1) / W, W * 32, sm, s, n, M,
           ldm, v, jidx, vstride, out, accumulate, stop);
    IIM_LAUNCHED();
    return IIM_OK;
}

__global__ void k_unit_vector(int n, int j, double* __restrict__ v) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) v[e] = (e == j) ? 1.0 : 0.0;
}

// column j of the left half of the augmented array from an FP64 vector
__global__ void k_store_column(int n, int j, const double* __restrict__ v, float* __restrict__ A) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) A[(long)e * 2 * n + j] = (float)v[e];
}

}  // namespace iim
