// Column pass of the rectangular solve as tridiagonal solves (FP32 transforms).
//
// After the forward DST-I of the rows, mode p of the x transform decouples the 5-point problem
// into one tridiagonal system per column (Hockney's FFT / tridiagonal method):
//   (2 + h^2 lam_x(p)) v_j - v_{j-1} - v_{j+1} = h^2 g_j,   j = 0..NY-1,   v_{-1} = v_NY = 0,
// which is exactly what the column DST, the division by lam_x + lam_y and the inverse column
// DST compute (same discrete operator, O(NY) work per column instead of two DSTs).  With
// b = 2 + h^2 lam_x(p) the elimination factors are e_0 = 1/b, e_j = 1/(b - e_{j-1}); then
//   forward  d_j = (h^2 g_j + d_{j-1}) e_j,   back  v_{NY-1} = d_{NY-1},  v_j = d_j + e_j v_{j+1}
// (the Thomas algorithm for this symmetric, diagonally dominant matrix; stable without
// pivoting).  The factors depend on the grid only: they are tabulated per column in FP64 and
// stored as FP32 up to the row where they reach their limit e* = (b - sqrt(b^2 - 4)) / 2 to
// FP32 precision (a few dozen rows except for the lowest modes), then e* is used.
//
// One thread per column, one warp per block (32 adjacent padded columns, so nx >= 32), so a row
// of the block's columns is one 128-byte segment.  Rows stream through a ring of shared-memory tiles
// filled by cp.async several tiles ahead of the sequential recurrence (the loads do not wait
// on the dependency chain).  The forward pass leaves d_j in the buffer's rows from in0 on (rows
// outside [in0, in1] hold no input and rows outside [out0, out1] are not read afterwards, so
// they serve as scratch); the back pass streams the d_j back in reverse and writes v_j, scaled
// by the inverse-x normalisation, to the rows [out0, out1].
#pragma once

#include <cstdint>

#include "common.cuh"

namespace iim {

// Factor table of one grid: per data column c (x mode c + 1) the factors e_j, j < len[c], at
// e + off[c], and the limit estar[c]; scale = h^2 (2 / nx), the right-hand side's factor.
struct TriTab {
    const float* e;
    const int* off;
    const int* len;
    const float* estar;
    float scale;
};

constexpr int kTriRows = 32;    // rows per tile
constexpr int kTriRing = 8;     // tiles in flight per block
constexpr size_t kTriSmem = sizeof(float) * kTriRing * kTriRows * 32;   // 32 KB

__device__ __forceinline__ void tri_cp16(float* smem, const float* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void tri_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void tri_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Copies rows [r0, r0 + kTriRows) (clipped to [lo, hi]) of the block's 32 columns into tile
// slot `slot`: 8 16-byte pieces per row, each lane one piece of every fourth row.
__device__ __forceinline__ void tri_fetch(float* ring, int slot, const float* __restrict__ base, int ld, int r0,
                                          int lo, int hi, int lane) {
    float* tile = ring + slot * kTriRows * 32;
    const int q = lane & 7;
#pragma unroll
    for (int k = 0; k < kTriRows / 4; ++k) {
        const int rr = (lane >> 3) + 4 * k;
        const int r = r0 + rr;
        if (r >= lo && r <= hi) tri_cp16(tile + rr * 32 + 4 * q, base + (size_t)r * ld + 4 * q);
    }
}

// Forward elimination and back substitution for the block's 32 columns (one warp).
// buf: padded layout, NY rows of nx = NX + 1 slots, element (row, data column c) at row*nx + c + 1.
__device__ __forceinline__ void cols_tri_body(int NX, int NY, int nx, int in0, int in1, int out0, int out1,
                                              float* __restrict__ buf, TriTab t) {
    extern __shared__ __align__(16) float tri_ring[];
    const int lane = threadIdx.x;
    const int p0 = blockIdx.x * 32;          // first padded column of the block
    const int p = p0 + lane, c = p - 1;      // this thread's padded and data column
    const bool live = p >= 1 && p <= NX;
    const float* e = live ? t.e + t.off[c] : t.e;
    const int L = live ? t.len[c] : 0;
    const float es = live ? t.estar[c] : 0.f;
    const float sc = t.scale;
    float* base = buf + p0;

    // ---- forward: rows in0..in1 carry input; tiles of kTriRows rows from in0
    float d = 0.f;
    const int nt = (in1 - in0) / kTriRows + 1;
#pragma unroll 1
    for (int k = 0; k < kTriRing - 1; ++k) {
        if (k < nt) tri_fetch(tri_ring, k, base, nx, in0 + k * kTriRows, in0, in1, lane);
        tri_commit();
    }
#pragma unroll 1
    for (int k = 0; k < nt; ++k) {
        const int kn = k + kTriRing - 1;
        if (kn < nt) tri_fetch(tri_ring, kn % kTriRing, base, nx, in0 + kn * kTriRows, in0, in1, lane);
        tri_commit();
        tri_wait<kTriRing - 1>();
        __syncwarp();
        const float* tile = tri_ring + (k % kTriRing) * kTriRows * 32;
        const int r0 = in0 + k * kTriRows;
        const int rn = min(kTriRows, in1 - r0 + 1);
        if (live) {
            // the tile's inputs and factors into registers first, so that no load waits behind
            // the stores of the recurrence
            float gv[kTriRows], ev[kTriRows];
#pragma unroll
            for (int rr = 0; rr < kTriRows; ++rr) {
                const int r = r0 + rr;
                gv[rr] = tile[rr * 32 + lane];
                ev[rr] = r < L ? __ldg(e + r) : es;
            }
#pragma unroll
            for (int rr = 0; rr < kTriRows; ++rr) {
                if (rr < rn) {
                    d = fmaf(sc, gv[rr], d) * ev[rr];
                    base[(size_t)(r0 + rr) * nx + lane] = d;
                }
            }
        }
        __syncwarp();   // the slot is refilled next iteration
    }
    tri_wait<0>();
    if (live) {
        // rows after the input: no right-hand side
        for (int r1 = in1 + 1; r1 < NY; r1 += kTriRows) {
            float ev[kTriRows];
#pragma unroll
            for (int rr = 0; rr < kTriRows; ++rr) ev[rr] = r1 + rr < L ? __ldg(e + r1 + rr) : es;
#pragma unroll
            for (int rr = 0; rr < kTriRows; ++rr) {
                if (r1 + rr < NY) {
                    d *= ev[rr];
                    base[(size_t)(r1 + rr) * nx + lane] = d;
                }
            }
        }
    }
    __threadfence();   // the d_j stores are read back by the asynchronous copies below
    __syncwarp();

    // ---- back: v_{NY-1} = d_{NY-1}, then rows NY-2 down to out0; d_j = 0 below in0
    float v = d;
    if (live && NY - 1 <= out1 && NY - 1 >= out0) base[(size_t)(NY - 1) * nx + lane] = v;
    const int top = NY - 2;                      // first row of the backward stream
    const int lo = max(out0, in0);               // rows with stored d_j that the stream needs
    const int nb = top >= lo ? (top - lo) / kTriRows + 1 : 0;
    // tile k covers rows (top - (k + 1) kTriRows, top - k kTriRows]
#pragma unroll 1
    for (int k = 0; k < kTriRing - 1; ++k) {
        if (k < nb) tri_fetch(tri_ring, k, base, nx, top - (k + 1) * kTriRows + 1, lo, top, lane);
        tri_commit();
    }
#pragma unroll 1
    for (int k = 0; k < nb; ++k) {
        const int kn = k + kTriRing - 1;
        if (kn < nb) tri_fetch(tri_ring, kn % kTriRing, base, nx, top - (kn + 1) * kTriRows + 1, lo, top, lane);
        tri_commit();
        tri_wait<kTriRing - 1>();
        __syncwarp();
        const float* tile = tri_ring + (k % kTriRing) * kTriRows * 32;
        const int rhi = top - k * kTriRows, rlo = max(lo, rhi - kTriRows + 1);
        const int r0 = rhi - kTriRows + 1;       // row of tile slot 0
        if (live) {
            float dv[kTriRows], ev[kTriRows];
#pragma unroll
            for (int rr = 0; rr < kTriRows; ++rr) {
                const int r = r0 + rr;
                dv[rr] = tile[rr * 32 + lane];
                ev[rr] = (r >= 0 && r < L) ? __ldg(e + r) : es;
            }
#pragma unroll
            for (int rr = kTriRows - 1; rr >= 0; --rr) {
                const int r = r0 + rr;
                if (r >= rlo) {
                    v = fmaf(ev[rr], v, dv[rr]);
                    if (r <= out1) base[(size_t)r * nx + lane] = v;
                }
            }
        }
        __syncwarp();
    }
    tri_wait<0>();
    if (live) {
        // rows below in0 (no stored d_j: it is zero there) down to out0
        for (int r = min(lo - 1, top); r >= out0; --r) {
            const float ej = r < L ? __ldg(e + r) : es;
            v *= ej;
            if (r <= out1) base[(size_t)r * nx + lane] = v;
        }
    }
}


}  // namespace iim
