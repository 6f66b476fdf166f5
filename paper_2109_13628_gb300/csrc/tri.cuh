// Column pass of the rectangular solve as per-mode tridiagonal solves, evaluated as two
// segmented linear-recurrence scans (FP32 and FP64).
//
// After the forward DST-I of the rows, x mode p decouples the 5-point problem into one
// tridiagonal system per column (Hockney's FFT / tridiagonal method):
//   (2 + eps_p) v_j - v_{j-1} - v_{j+1} = h^2 g_j,  j = 0..NY-1,  v_{-1} = v_NY = 0,
// eps_p = h^2 lam_x(p) = 4 sin^2(pi p / (2 nx)) -- the same discrete inverse as the column DST,
// the division by lam_x + lam_y and the inverse column DST.  Its LU factors are
// e_0 = 1/(2 + eps), e_j = 1/(2 + eps - e_{j-1}) (Thomas algorithm), and with the right-hand side
// scaled by s = h^2 (2 / nx) (the inverse-x normalisation folded in)
//   forward  d_j = e_j (s g_j + d_{j-1}),        back  v_j = d_j + e_j v_{j+1}.
// The factors are kept through their complements delta_j = 1 - e_j (tabulated in FP64 from a
// closed form, rounded once): for the low modes e_j is within 1e-3 of 1, and storing or
// multiplying by e_j itself would lose the low bits of the decay rate, which the nearly
// singular low-mode systems amplify.  So each step is one fused multiply-add:
//   d_j = t - delta_j t (t = s g_j + d_{j-1}),   v_j = (d_j + v_{j+1}) - delta_j v_{j+1}.
//
// Both recurrences are affine maps x -> (1 - D) x + B, so a column is cut into segments of R
// rows, one thread per (column, segment): each thread runs its segment from a zero carry to get
// the segment's map (B, and the complement D of the product of its e_j); a scan of the segment
// maps over the block (shared memory, one warp per column, shuffles) gives every segment its
// true carry; the thread then runs the recurrence again from that carry and stores it (the
// same arithmetic as the sequential Thomas sweep within the segment).  The back recurrence
// runs the same way from the other end.  Rows are read once from and written once to global
// memory; per element about fourteen arithmetic and shared-memory instructions.
//
// Block: NT threads (256 or 1024) on a tile of CW adjacent padded columns (32 bytes per row:
// CW = 8 FP32, 4 FP64) over all rows, staged in shared memory by 16-byte vector loads (one whole
// sector per row), so that the recurrences run out of shared memory with few registers per
// thread and the tiles of a 2048^2 field fit the GPU in one wave.  Thread t works on column
// t % CW, segment t / CW of S = NT / CW segments.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace iim {

// Factors of one grid and precision.  Rows j >= lim[c] of data column c use dstar[c] = 1 - e*
// (lim is non-increasing in c).  Rows j < lim[c] take delta_j = 1 - e_j
//   FP64: from the table, delta[rowoff[j] + c] (row-major over j: the tabulated columns of row j
//         are exactly those with lim[c] > j, so a warp's reads of one row are contiguous);
//   FP32: from the closed form delta_j = delta* + A q^(j+1) / (1 - q^(j+2)) with the column's
//         par[c] = (delta*, log2 q, q, A = e* (1 - q)), q^(j+1) by the hardware exp2: no memory
//         traffic, and its rounding (about 1e-6 relative, where the correction term is not
//         small against delta*) falls on the first rows, where the low modes' eigenvectors are
//         small.
// scale = h^2 (2 / nx).
template <typename T>
struct ScanTab {
    const T* delta;
    const int* rowoff;
    const float4* par;
    const int* lim;
    const T* dstar;
    T scale;
};

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float expm1T(float a) { return expm1f(a); }
__device__ __forceinline__ double expm1T(double a) { return expm1(a); }
__device__ __forceinline__ float log1pT(float a) { return log1pf(a); }
__device__ __forceinline__ double log1pT(double a) { return log1p(a); }

// Threads of a block: 1024 for long columns when the launch has few blocks (more segments,
// shorter sequential chains per thread: lower latency), else 256 (more blocks per SM: better
// throughput).  Segments S = NT / CW; rows per segment at least NY / S and congruent to 1 mod 4,
// so that in the row-major tile (row j at j * CW) the segments of one warp start 8 banks apart
// and a pass over the rows is free of bank conflicts.
__host__ __device__ constexpr int scan_threads(int NY, long blocks, int sms) {
    return NY >= 1000 && blocks < 2L * sms ? 1024 : 256;
}
__host__ __device__ constexpr int scan_rows(int NY, int S) { return ((NY + S - 1) / S + 2) / 4 * 4 + 1; }
// Shared memory of a block: the segment maps (D, B) of S segments x CW columns (padded rows),
// then the tile (S R rows x CW columns).
template <typename T, int CW, int NT>
__host__ __device__ constexpr size_t scan_smem(int NY) {
    return sizeof(T) * ((size_t)2 * (NT / CW) * (CW + 1) + (size_t)(NT / CW) * scan_rows(NY, NT / CW) * CW);
}

// Exclusive scan of the segment maps of every column (in place: sB[seg] becomes the carry
// into the segment; sD is left as it was).  Map of segment q: x -> (1 - D_q) x + B_q; the
// carry into the first segment (in scan order) is zero.  `reverse` scans from the last
// segment down.  One warp per column, each lane composing ceil(S / 32) consecutive segments.
template <typename T, int CW, int S, int NT>
__device__ __forceinline__ void scan_segment_maps(const T* sD, T* sB, bool reverse) {
    constexpr int K = (S + 31) / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    for (int cc = w; cc < CW; cc += NW) {
        T D = T(0), B = T(0);   // identity map
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int q = lane * K + i;
            if (q < S) {
                const int at = (reverse ? S - 1 - q : q) * (CW + 1) + cc;
                const T d2 = sD[at], b2 = sB[at];
                B = fmaT(-d2, B, B) + b2;     // the segment's map after the lane's maps so far
                D = fmaT(-D, d2, D + d2);
            }
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T Do = __shfl_up_sync(0xffffffffu, D, off), Bo = __shfl_up_sync(0xffffffffu, B, off);
            if (lane >= off) {          // earlier lanes' map (Do, Bo), then this lane's
                B = fmaT(-D, Bo, Bo) + B;
                D = fmaT(-Do, D, Do + D);
            }
        }
        T cr = __shfl_up_sync(0xffffffffu, B, 1);
        if (lane == 0) cr = T(0);
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int q = lane * K + i;
            if (q < S) {
                const int at = (reverse ? S - 1 - q : q) * (CW + 1) + cc;
                const T d2 = sD[at], b2 = sB[at];
                sB[at] = cr;
                cr = fmaT(-d2, cr, cr) + b2;
            }
        }
    }
}

// Tridiagonal column pass of one field in the padded layout (NY rows of ld = NX + 1 slots;
// element (row j, data column c) at j * ld + c + 1; slot 0 of a row is a zero pad).  Rows
// outside [in0, in1] are zero on input and not read; only rows [out0, out1] are written.  Block
// blockIdx.x: padded columns [CW blockIdx.x, CW blockIdx.x + CW); NT threads; dynamic shared
// memory scan_smem<T, CW, NT>(NY).
template <typename T, int CW, int NT>
__device__ __forceinline__ void cols_scan_body(int NX, int NY, int ld, int in0, int in1, int out0, int out1,
                                               T* __restrict__ buf, ScanTab<T> t) {
    constexpr int S = NT / CW;
    constexpr int V = 16 / (int)sizeof(T), PPR = CW / V;   // elements per 16-byte piece, pieces per row
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    extern __shared__ __align__(16) unsigned char scan_raw[];
    const int R = scan_rows(NY, S);
    T* sD = reinterpret_cast<T*>(scan_raw);
    T* sB = sD + S * (CW + 1);
    T* tile = sB + S * (CW + 1);
    const int P0 = blockIdx.x * CW;

    // tile load: 16-byte pieces, NB loads in flight per thread before their stores
    constexpr int NB = NT >= 1024 ? 4 : 8;
    const int npc = NY * PPR;
    for (int e0 = threadIdx.x; e0 < npc; e0 += NB * NT) {
        VT v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int e = e0 + b * NT, j = e / PPR;
            v[b] = VT{};
            if (e < npc && j >= in0 && j <= in1)
                v[b] = *reinterpret_cast<const VT*>(buf + (size_t)j * ld + P0 + (e - j * PPR) * V);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int e = e0 + b * NT;
            if (e < npc) *reinterpret_cast<VT*>(tile + e * V) = v[b];   // row e / PPR, piece e % PPR
        }
    }

    const int cl = threadIdx.x % CW, seg = threadIdx.x / CW;
    const int p = P0 + cl, c = p - 1;
    const bool live = p >= 1 && p <= NX;
    const int j0 = seg * R;
    const int kend = min(max(NY - j0, 0), R);
    const int lim = live ? __ldg(t.lim + c) : 0;
    const T ds = live ? __ldg(t.dstar + c) : T(0);
    const int kt = min(max(lim - j0, 0), kend);  // rows [0, kt) of the segment use the table
    const T sc = t.scale;
    T* xs = tile + j0 * CW + cl;                 // row k of this thread's segment at xs[k * CW]
    // factors of the tabulated rows, generated in row order (up from row 0 or down from row
    // kt - 1 of the segment): FP32 from the closed form with q^(j+1) stepped by q or 1 / q from
    // one exp2 per pass, FP64 from the table
    float4 par = make_float4(0.f, 0.f, 0.f, 0.f);
    float qp = 0.f, qstep = 0.f;
    if (sizeof(T) == 4 && kt > 0) par = __ldg(t.par + c);
    auto gen_start = [&](bool up) {
        if (sizeof(T) == 4 && kt > 0) {
            qp = exp2f((float)(up ? j0 + 1 : j0 + kt) * par.y);
            qstep = up ? par.z : exp2f(-par.y);
        }
    };
    auto tab = [&](int k) -> T {
        if constexpr (sizeof(T) == 4) {
            const float d = par.x + __fdividef(par.w * qp, fmaf(-par.z, qp, 1.0f));
            qp *= qstep;
            return d;
        } else {
            return __ldg(t.delta + __ldg(t.rowoff + j0 + k) + c);
        }
    };
    __syncthreads();

    // pass A: the segment's forward map from a zero carry (x -> (1 - D) x + acc), nothing stored;
    // D of the rows after the table in closed form, 1 - (1 - dstar)^m
    T acc = T(0), D = T(0);
    gen_start(true);
#pragma unroll 4
    for (int k = 0; k < kt; ++k) {
        const T dk = tab(k);
        const T s = fmaT(sc, xs[k * CW], acc);
        acc = fmaT(-dk, s, s);
        D = fmaT(-D, dk, D + dk);
    }
#pragma unroll 8
    for (int k = kt; k < kend; ++k) {
        const T s = fmaT(sc, xs[k * CW], acc);
        acc = fmaT(-ds, s, s);
    }
    if (kend > kt) {
        const T Dc = -expm1T((T)(kend - kt) * log1pT(-ds));
        D = fmaT(-D, Dc, D + Dc);
    }
    const int at = seg * (CW + 1) + cl;
    sD[at] = D;
    sB[at] = acc;
    __syncthreads();
    scan_segment_maps<T, CW, S, NT>(sD, sB, false);
    __syncthreads();
    // pass B: the forward recurrence from the segment's true carry d_{j0 - 1}, stored
    acc = sB[at];
    gen_start(true);
#pragma unroll 4
    for (int k = 0; k < kt; ++k) {
        const T dk = tab(k);
        const T s = fmaT(sc, xs[k * CW], acc);
        acc = fmaT(-dk, s, s);
        xs[k * CW] = acc;
    }
#pragma unroll 8
    for (int k = kt; k < kend; ++k) {
        const T s = fmaT(sc, xs[k * CW], acc);
        acc = fmaT(-ds, s, s);
        xs[k * CW] = acc;
    }
    // pass A': the segment's back map from a zero carry (v beyond the segment = 0); its D is the
    // same product of the e_j
    T accv = T(0);
#pragma unroll 8
    for (int k = kend - 1; k >= kt; --k) accv = fmaT(-ds, accv, xs[k * CW] + accv);
    gen_start(false);
#pragma unroll 4
    for (int k = kt - 1; k >= 0; --k) {
        const T dk = tab(k);
        accv = fmaT(-dk, accv, xs[k * CW] + accv);
    }
    sB[at] = accv;     // own slot, carry already read
    __syncthreads();
    scan_segment_maps<T, CW, S, NT>(sD, sB, true);
    __syncthreads();
    // pass B': the back recurrence from the segment's true carry v_{j0 + kend}, stored
    accv = sB[at];
#pragma unroll 8
    for (int k = kend - 1; k >= kt; --k) {
        accv = fmaT(-ds, accv, xs[k * CW] + accv);
        xs[k * CW] = accv;
    }
    gen_start(false);
#pragma unroll 4
    for (int k = kt - 1; k >= 0; --k) {
        const T dk = tab(k);
        accv = fmaT(-dk, accv, xs[k * CW] + accv);
        xs[k * CW] = accv;
    }
    __syncthreads();

    // tile store of rows [out0, out1]
    const int nst = (out1 - out0 + 1) * PPR;
    for (int e = threadIdx.x; e < nst; e += NT) {
        const int j = out0 + e / PPR, q = e % PPR;
        *reinterpret_cast<VT*>(buf + (size_t)j * ld + P0 + q * V) = *reinterpret_cast<const VT*>(tile + j * CW + q * V);
    }
}

}  // namespace iim
