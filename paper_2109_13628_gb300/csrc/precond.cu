// Dense Schur-complement preconditioner kernels: blocked Gauss-Jordan inversion with partial
// pivoting of the (n x n) matrix S held in the left half of a row-major n x 2n array [S | I],
// and the dense FP32 matrix-vector product used to apply the inverse.
//
// S = I + A P E_a (with the circulation rows) is the operator of Sec. 4.2; its inverse turns
// each correction solve into one dense product (the capacitance-matrix view of the same linear
// system); inside GMRES it is a right preconditioner, so the iteration still measures the
// residual of the exact operator.
#include <cmath>

#include <cstdint>

#include "common.cuh"
#include "iim_ops.cuh"

namespace iim {

// Blocked Gauss-Jordan.  Columns are taken in panels of up to GJ_B = 64.  For the panel
// starting at column k0 (width bb) a working array W (n x 128, row-major) holds the panel's
// columns in [0, bb) and, in [64, 64 + bb), the rows' combination of the identity block rows
// k0..k0+bb-1.  The bb pivot steps run on W only (one launch each, W read from one buffer and
// written to the other), with partial pivoting over rows >= k0 + j.  At the end W's right part
// is the n x bb block G of the panel's transform E (E = identity except columns k0..k0+bb-1,
// which are G, in the row order after the panel's swaps).  The rest of [S | I] is then updated
// at once: the panel's row swaps are applied to columns >= k0 + bb, T = the block rows there,
// and A += (G - I_blk) T -- a rank-bb update that carries the O(n^3) work.
constexpr int GJ_B = 64;
constexpr int GJ_LDW = 128;

size_t gj_scratch_floats(int n) { return 2 * (size_t)GJ_LDW * n + (size_t)GJ_B * 2 * n + GJ_B; }

__global__ void k_gj_panel_init(const float* __restrict__ A, long lda, int n, int k0, int bb, float* __restrict__ W,
                                const int* __restrict__ info) {
    if (*info) return;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)n * GJ_LDW) return;
    const int i = (int)(e / GJ_LDW), c = (int)(e - (long)i * GJ_LDW);
    float v = 0.f;
    if (c < GJ_B) {
        if (c < bb) v = A[(long)i * lda + k0 + c];
    } else if (c - GJ_B < bb && i == k0 + c - GJ_B) {
        v = 1.f;
    }
    W[e] = v;
}

// Pivot step j of the panel.  Every block finds the pivot p = argmax_{i >= k0+j} |Win[i][j]|
// (ties to the lower row) itself, so no second launch is needed; block 0 records it.  Row
// r0 = k0 + j and row p exchange their left parts and the right-part columns < j (right-part
// columns >= j are still identity columns and stay with their rows); the new row r0 is the
// exchanged row divided by the pivot and every other row i loses f_i times it, f_i = its
// (exchanged) entry in column j.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_gj_panel_step(const float* __restrict__ Win, float* __restrict__ Wout, int n, int k0, int j, int* __restrict__ perm,
                int* __restrict__ info) {
    if (*info) return;
    const int r0 = k0 + j;
    __shared__ float sv[BLOCK];
    __shared__ int si[BLOCK];
    __shared__ float prow[GJ_LDW];
    float best = -1.f;
    int bi = r0;
    for (int i = r0 + threadIdx.x; i < n; i += BLOCK) {
        const float v = fabsf(Win[(long)i * GJ_LDW + j]);
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
    if (!(sv[0] > 0.f)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *info = r0 + 1;
        return;
    }
    const float inv = 1.f / Win[(long)p * GJ_LDW + j];
    for (int c = threadIdx.x; c < GJ_LDW; c += BLOCK) {
        const bool sw = c < GJ_B || c - GJ_B < j;
        prow[c] = Win[(long)(sw ? p : r0) * GJ_LDW + c] * inv;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) perm[j] = p;
    __syncthreads();
    for (long e = (long)blockIdx.x * BLOCK + threadIdx.x; e < (long)n * GJ_LDW; e += (long)gridDim.x * BLOCK) {
        const int i = (int)(e / GJ_LDW), c = (int)(e - (long)i * GJ_LDW);
        float out;
        if (i == r0) {
            out = prow[c];
        } else {
            const int srow = (i == p) ? r0 : i;
            const bool sw = c < GJ_B || c - GJ_B < j;
            const float v = Win[(long)(sw ? srow : i) * GJ_LDW + c];
            const float f = Win[(long)srow * GJ_LDW + j];
            out = v - f * prow[c];
        }
        Wout[e] = out;
    }
}

// The panel's row exchanges, in order, on columns c0.. c0+m-1 of A, and T[t][c] = row k0+t
// after them (later exchanges only touch rows below k0+t, so it is final when read).  One
// thread per column.
__global__ void k_gj_swap_rows(float* __restrict__ A, long lda, int k0, int bb, int c0, int m,
                               const int* __restrict__ perm, float* __restrict__ T, long ldt, const int* __restrict__ info) {
    if (*info) return;
    __shared__ int sp[GJ_B];
    if (threadIdx.x < bb) sp[threadIdx.x] = perm[threadIdx.x];
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    float* col = A + c0 + c;
    for (int t = 0; t < bb; ++t) {
        const int p = sp[t], r = k0 + t;
        float vr = col[(long)r * lda];
        if (p != r) {
            const float vp = col[(long)p * lda];
            col[(long)p * lda] = vr;
            col[(long)r * lda] = vp;
            vr = vp;
        }
        T[(long)t * ldt + c] = vr;
    }
}

// A[i][c0 + c] += sum_t (W[i][64 + t] - [i == k0 + t]) T[t][c] for i < n, c < m, t < bb:
// 128 x 128 output tiles, the two operand tiles (64 x 128 each, zero beyond bb / the edges)
// in shared memory, an 8 x 8 register tile per thread (rows ty*4 + {0..3} and 64 + ty*4 +
// {0..3}, columns likewise with tx), FP32 FMA.
constexpr int GJ_TILE = 128;
__global__ void __launch_bounds__(256, 2)
k_gj_update(float* __restrict__ A, long lda, int n, int c0, int m, const float* __restrict__ W, int k0, int bb,
            const float* __restrict__ T, long ldt, const int* __restrict__ info) {
    if (*info) return;
    extern __shared__ float4 gj_smem4[];
    float* Gs = reinterpret_cast<float*>(gj_smem4);   // [GJ_B][GJ_TILE]: Gs[t][r]
    float* Ts = Gs + GJ_B * GJ_TILE;                    // [GJ_B][GJ_TILE]: Ts[t][c]
    const int i0 = blockIdx.y * GJ_TILE, cb = blockIdx.x * GJ_TILE;
    const int tid = threadIdx.x;
    // G tile: four consecutive t per thread (one 16-byte load of a W row), a warp on 32 rows
    for (int e = tid; e < GJ_TILE * (GJ_B / 4); e += 256) {
        const int r = e % GJ_TILE, t = 4 * (e / GJ_TILE);
        const int i = i0 + r;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < n) v = *reinterpret_cast<const float4*>(W + (long)i * GJ_LDW + GJ_B + t);
        const float g[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int tq = t + q;
            float x = tq < bb ? g[q] : 0.f;
            if (i == k0 + tq) x -= 1.f;
            Gs[tq * GJ_TILE + r] = (i < n && tq < bb) ? x : 0.f;
        }
    }
    for (int e = tid; e < GJ_TILE * GJ_B; e += 256) {
        const int t = e / GJ_TILE, c = e % GJ_TILE;
        Ts[e] = (t < bb && cb + c < m) ? T[(long)t * ldt + cb + c] : 0.f;
    }
    __syncthreads();
    const int ty = tid >> 4, tx = tid & 15;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int i = i0 + (a < 4 ? ty * 4 + a : 64 + ty * 4 + a - 4);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int c = cb + (b < 4 ? tx * 4 + b : 64 + tx * 4 + b - 4);
            acc[a][b] = (i < n && c < m) ? A[(long)i * lda + c0 + c] : 0.f;
        }
    }
#pragma unroll 4
    for (int t = 0; t < GJ_B; ++t) {
        const float4 a0 = *reinterpret_cast<const float4*>(Gs + t * GJ_TILE + ty * 4);
        const float4 a1 = *reinterpret_cast<const float4*>(Gs + t * GJ_TILE + 64 + ty * 4);
        const float4 b0 = *reinterpret_cast<const float4*>(Ts + t * GJ_TILE + tx * 4);
        const float4 b1 = *reinterpret_cast<const float4*>(Ts + t * GJ_TILE + 64 + tx * 4);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int i = i0 + (a < 4 ? ty * 4 + a : 64 + ty * 4 + a - 4);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int c = cb + (b < 4 ? tx * 4 + b : 64 + tx * 4 + b - 4);
            if (i < n && c < m) A[(long)i * lda + c0 + c] = acc[a][b];
        }
    }
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

// The same product with 16-byte row loads: a row starting h = 0..3 floats before a 16-byte
// boundary is read as h leading floats, then float4s (eight in flight per lane), then the
// remainder.  v is staged four times in shared memory, copy h shifted by h elements, so that
// the float4 of the row always meets an aligned float4 of v.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_dense_matvec4(int n, const float* __restrict__ M, long ldm, const double* __restrict__ vbase,
                const int* __restrict__ jidx, long vstride, double* __restrict__ out, int accumulate,
                const int* __restrict__ stop) {
    dense_matvec4_body<WARPS>(n, M, ldm, vbase, jidx, vstride, out, accumulate, stop);
}

iim_status gj_invert_aug(float* A, int n, float* scratch, int* info, cudaStream_t s) {
    IIM_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
    launch("gj_identity", 0.0, 0.0, k_set_identity_aug, (unsigned)(((long)n * n + 255) / 256), 256, 0, s, A, n);
    const long lda = 2L * n;
    float* W0 = scratch;
    float* W1 = W0 + (size_t)GJ_LDW * n;
    float* T = W1 + (size_t)GJ_LDW * n;
    int* perm = reinterpret_cast<int*>(T + (size_t)GJ_B * lda);
    const size_t upd_smem = sizeof(float) * 2 * GJ_B * GJ_TILE;
    IIM_CHECK(allow_smem(k_gj_update, upd_smem));
    const long welems = (long)n * GJ_LDW;
    const unsigned wblocks = (unsigned)((welems + 255) / 256);
    const unsigned sblocks = (unsigned)std::min<long>(304, (welems + 1023) / 1024);
    for (int k0 = 0; k0 < n; k0 += GJ_B) {
        const int bb = std::min(GJ_B, n - k0);
        const int c0 = k0 + bb;
        const int m = (int)(lda - c0);
        launch("gj_panel_init", 0.0, 0.0, k_gj_panel_init, wblocks, 256, 0, s, (const float*)A, lda, n, k0, bb, W0,
               (const int*)info);
        float* win = W0;
        float* wout = W1;
        for (int j = 0; j < bb; ++j) {
            launch("gj_panel_step", 0.0, 0.0, k_gj_panel_step<256>, sblocks, 256, 0, s, (const float*)win, wout, n, k0, j,
                   perm, info);
            std::swap(win, wout);
        }
        launch("gj_swap_rows", 0.0, 0.0, k_gj_swap_rows, (unsigned)((m + 255) / 256), 256, 0, s, A, lda, k0, bb, c0, m,
               (const int*)perm, T, lda, (const int*)info);
        launch("gj_update", 2.0 * n * m * 4.0, 2.0 * n * (double)m * bb, k_gj_update,
               dim3((unsigned)((m + GJ_TILE - 1) / GJ_TILE), (unsigned)((n + GJ_TILE - 1) / GJ_TILE)), 256, upd_smem, s,
               A, lda, n, c0, m, (const float*)win, k0, bb, (const float*)T, lda, (const int*)info);
    }
    IIM_LAUNCHED();
    return IIM_OK;
}

// out_{j+1} = M v for the Krylov basis column after *ojidx (the dense Schur operator of the
// inner iteration, iim_opts.precond == 3); M must fit the staged-vector kernel (4 n floats of
// shared memory <= 200 KB).
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_dense_matvec4_to(int n, const float* __restrict__ M, long ldm, const double* __restrict__ v,
                   double* __restrict__ outb, const int* __restrict__ ojidx, long ostride,
                   const int* __restrict__ stop) {
    dense_matvec4_body<WARPS>(n, M, ldm, v, nullptr, 0L, outb, 0, stop, ojidx, ostride);
}

bool dense_matvec_fits(int n) { return sizeof(float) * 4 * (size_t)((n + 3) & ~3) <= 200 * 1024; }

iim_status dense_matvec_to(int n, const float* M, long ldm, const double* v, double* outb, const int* ojidx,
                           long ostride, const int* stop, cudaStream_t s) {
    constexpr int W = 8;
    const size_t sm4 = sizeof(float) * 4 * (size_t)((n + 3) & ~3);
    if (!dense_matvec_fits(n)) return IIM_ERR_INVALID_ARG;
    IIM_CHECK(allow_smem(k_dense_matvec4_to<W>, sm4));
    launch("dense_schur_matvec", (double)n * n * 4.0, 2.0 * n * n, k_dense_matvec4_to<W>, (n + W - 1) / W, W * 32,
           sm4, s, n, M, ldm, v, outb, ojidx, ostride, stop);
    IIM_LAUNCHED();
    return IIM_OK;
}

iim_status dense_matvec(int n, const float* M, long ldm, const double* v, const int* jidx, long vstride, double* out,
                        int accumulate, const int* stop, cudaStream_t s) {
    constexpr int W = 8;
    const size_t sm4 = sizeof(float) * 4 * (size_t)((n + 3) & ~3);
    if (sm4 <= 200 * 1024) {
        // the limit only ever grows (allow_smem): solves of different sizes on other threads
        // must not lower it under this launch
        IIM_CHECK(allow_smem(k_dense_matvec4<W>, sm4));
        launch("precond_matvec", (double)n * n * 4.0, 2.0 * n * n, k_dense_matvec4<W>, (n + W - 1) / W, W * 32, sm4, s,
               n, M, ldm, v, jidx, vstride, out, accumulate, stop);
        IIM_LAUNCHED();
        return IIM_OK;
    }
    const size_t sm = sizeof(float) * (size_t)n;
    IIM_CHECK(allow_smem(k_dense_matvec<W>, sm));
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
