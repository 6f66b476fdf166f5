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

// 16-point DFT as 4 x 4: 4-point DFTs over the stride-4 subsets, twiddles W16^(b k), 4-point
// DFTs across them.  Natural order in and out.
template <typename T>
__device__ __forceinline__ void dft16_impl(cpx<T>* v) {
    const T c = T(0.92387953251128675613), s = T(0.38268343236508977173), r = T(0.70710678118654752440);
    cpx<T> t[16];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        cpx<T> u[4] = {v[b], v[4 + b], v[8 + b], v[12 + b]};
        dft4_impl(u);
#pragma unroll
        for (int k = 0; k < 4; ++k) t[4 * b + k] = u[k];
    }
    // W16^j = exp(-2 pi i j / 16) for the products j = b k that occur: 1, 2, 3, 4, 6, 9
    const cpx<T> w1 = {c, -s}, w2 = {r, -r}, w3 = {s, -c}, w6 = {-r, -r}, w9 = {-c, s};
    t[5] = cmul(t[5], w1);
    t[6] = cmul(t[6], w2);
    t[7] = cmul(t[7], w3);
    t[9] = cmul(t[9], w2);
    t[10] = cmi(t[10]);
    t[11] = cmul(t[11], w6);
    t[13] = cmul(t[13], w3);
    t[14] = cmul(t[14], w6);
    t[15] = cmul(t[15], w9);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cpx<T> u[4] = {t[k], t[4 + k], t[8 + k], t[12 + k]};
        dft4_impl(u);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[k + 4 * q] = u[q];
    }
}
template <>
__device__ __forceinline__ void dft<float, 16>(cpx<float>* v) { dft16_impl(v); }
template <>
__device__ __forceinline__ void dft<double, 16>(cpx<double>* v) { dft16_impl(v); }

// Position of line element j in a line buffer: plain (j), or padded with two elements after
// every 32 (the line buffers of the register paths, n = 512 and 1024), which keeps each lane's
// run of 32 consecutive elements in its own banks when the lanes of a warp store contiguous
// chunks.
template <bool PADL>
__host__ __device__ __forceinline__ constexpr int lp(int j) { return PADL ? j + ((j >> 5) << 1) : j; }

template <typename T>
using vec2_t = typename std::conditional<sizeof(T) == 4, float2, double2>::type;

// Packed FFT input c_m = y_{2m} + i y_{2m+1} from the line x (x_0 = x_n = 0).
template <typename T, bool PADL = false>
__device__ __forceinline__ cpx<T> packed(const T* x, const cpx<T>* tw, int n, int m) {
    const int j0 = 2 * m, j1 = j0 + 1;
    T a0, a1;
    if constexpr (PADL) {
        // x_{2m}, x_{2m+1} are adjacent and 2-element aligned in the padded layout
        const vec2_t<T> v = *reinterpret_cast<const vec2_t<T>*>(x + lp<PADL>(j0));
        a0 = v.x;
        a1 = v.y;
    } else {
        a0 = x[j0];
        a1 = x[j1];
    }
    T y0 = T(0);
    if (j0 != 0) {
        const T b = x[lp<PADL>(n - j0)];
        y0 = (-tw[j0].y) * (a0 + b) + T(0.5) * (a0 - b);
    }
    const T b1 = x[lp<PADL>(n - j1)];
    const T y1 = (-tw[j1].y) * (a1 + b1) + T(0.5) * (a1 - b1);
    return {y0, y1};
}

// Shared-memory layout of the complex FFT work arrays: inside every 128-byte block the entry
// index is XOR-ed with the block number, so that the strided stores of a radix pass and the
// reads of the next pass fall into distinct banks.  A bijection on [0, M) for M >= 16.
template <typename T>
__device__ __forceinline__ int swz(int i) {
    return sizeof(T) == 4 ? (i ^ ((i >> 4) & 15)) : (i ^ ((i >> 3) & 7));
}

// Radix of each Stockham pass of an M-point FFT (M = 2^logM): 8 while at least three factors
// of two remain, then 4 or 2.
__device__ __forceinline__ int pass_radix(int rem) { return rem >= 3 ? 8 : (rem == 2 ? 4 : 2); }

// Per-pass twiddle tables.  The pass with stride Ns > 1 and radix R multiplies value r of
// butterfly k by exp(-2 pi i k r / (Ns R)); its table holds these for r = 1..R-1, k < Ns at
// [(r - 1) Ns + k] (consecutive k for one r: conflict-free reads), the passes' tables one after
// another (fewer than M entries in all).
template <typename T>
__device__ __forceinline__ cpx<T> pass_twiddle_entry(const cpx<T>* __restrict__ g_tw, int n, int logn, int e,
                                                     bool& valid) {
    const int M = n >> 1;
    int rem = logn - 1, Ns = 1, off = 0;
    valid = false;
    while (rem > 0) {
        const int R = pass_radix(rem);
        if (Ns > 1) {
            const int size = (R - 1) * Ns;
            if (e < off + size) {
                const int q = e - off, r = q / Ns + 1, k = q - (r - 1) * Ns;
                const int t = ((4 * M) / (Ns * R)) * k * r;   // exp(-i pi t / n), t < 2n
                const int shift = kTwLog - logn;
                const cpx<T> w = g_tw[(t & (n - 1)) << shift];
                valid = true;
                return t >= n ? cpx<T>{-w.x, -w.y} : w;
            }
            off += size;
        }
        Ns *= R;
        rem -= (R == 8 ? 3 : R == 4 ? 2 : 1);
    }
    return cpx<T>{T(0), T(0)};
}

// One Stockham radix-R pass of an M-point FFT: in -> out (out-of-place, swizzled layout).
// With `x` given the input values are the packed line (natural layout) instead of `in`.
template <typename T, int R>
__device__ __forceinline__ void stockham_pass(const cpx<T>* in, const T* x, cpx<T>* out, const cpx<T>* tw,
                                              const cpx<T>* ptw, int n, int M, int Ns, int lane) {
    const int J = M / R;
    for (int j = lane; j < J; j += 32) {
        cpx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x ? packed(x, tw, n, j + r * J) : in[swz<T>(j + r * J)];
        const int k = j & (Ns - 1);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], ptw[(r - 1) * Ns + k]);
        }
        dft<T, R>(v);
        const int idx = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[swz<T>(idx + r * Ns)] = v[r];
    }
    __syncwarp();
}

// Lines whose half-length FFT has M = 32 P points with P = 8 or 16 use a register-resident
// FFT: M = P x 32 with the P-point DFTs in registers (lane l holds the samples l + 32 p), the
// twiddles W_M^(l k), one transpose through shared memory, P-point DFTs again and a
// (32 / P)-point DFT across the lanes of each group.  Other sizes use the Stockham passes.
__host__ __device__ constexpr bool reg_fft(int n) { return n == 512 || n == 1024; }
// FFT path per line length: 16 / 8 = register path on one warp (n = 1024 / 512), 64 = three
// register radix-8 stages on 64 threads (n = 1024, when wide lines are asked for: lower
// latency per line, more instructions), 0 = Stockham passes on one warp (other sizes).
__host__ __device__ constexpr int fft_path(int n, bool wide = false) {
    return n == 1024 ? (wide ? 64 : 16) : n == 512 ? 8 : 0;
}
__host__ __device__ constexpr int line_threads(int fp) { return fp == 64 ? 64 : 32; }

// Split step of the real FFT and the prefix sum of the odd outputs (see the file header): C
// (swizzled, M values) -> dst (natural layout, X_k at index k).
template <typename T>
__device__ __forceinline__ void dst_finish(const cpx<T>* C, T* dst, const cpx<T>* tw, int M, int lane) {
    for (int k = lane; k < M; k += 32) {
        const cpx<T> ck = C[swz<T>(k)];
        const cpx<T> cm = C[swz<T>(k == 0 ? 0 : M - k)];
        const T ex = T(0.5) * (ck.x + cm.x), ey = T(0.5) * (ck.y - cm.y);
        const T dx = T(0.5) * (ck.x - cm.x), dy = T(0.5) * (ck.y + cm.y);
        const cpx<T> w = tw[2 * k];
        const T yx = ex + (w.x * dy + w.y * dx);
        const T yy = ey + (w.y * dy - w.x * dx);
        reinterpret_cast<cpx<T>*>(dst)[k] = cpx<T>{k == 0 ? T(0) : -yy, k == 0 ? T(0.5) * yx : yx};
    }
    __syncwarp();
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
}

// The split step and the odd outputs' running sum with each lane on P consecutive k
// (k = P lane + i): the split values come straight from C (swizzled), the running sum is a
// sequential sum within the lane plus one warp scan of the lane totals, and each lane stores
// (X_2k, X_2k+1) pairs into dst in the padded layout.  tws[i * 32 + lane] = tw[2 (P lane + i)].
template <typename T, int P>
__device__ __forceinline__ void dst_finish_chunked(const cpx<T>* C, T* dst, const cpx<T>* tws, int lane) {
    constexpr int M = 32 * P;
    T ev[P], od[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const int k = P * lane + i;
        const cpx<T> ck = C[swz<T>(k)];
        const cpx<T> cm = C[swz<T>(k == 0 ? 0 : M - k)];
        const T ex = T(0.5) * (ck.x + cm.x), ey = T(0.5) * (ck.y - cm.y);
        const T dx = T(0.5) * (ck.x - cm.x), dy = T(0.5) * (ck.y + cm.y);
        const cpx<T> w = tws[i * 32 + lane];
        const T yx = ex + (w.x * dy + w.y * dx);
        const T yy = ey + (w.y * dy - w.x * dx);
        ev[i] = k == 0 ? T(0) : -yy;
        od[i] = k == 0 ? T(0.5) * yx : yx;
    }
#pragma unroll
    for (int i = 1; i < P; ++i) od[i] += od[i - 1];
    const T tot = od[P - 1];
    T incl = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
    }
    const T excl = incl - tot;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const int k = P * lane + i;
        vec2_t<T> v;
        v.x = ev[i];
        v.y = od[i] + excl;
        *reinterpret_cast<vec2_t<T>*>(dst + lp<true>(2 * k)) = v;
    }
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ cpx<T> shfl_cpx(cpx<T> v, int src) {
    return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}

// Register-path DST-I (P = 8 or 16, n = 64 P).  rtw = tw + n: [k * 32 + l] = W_M^(l k) for
// k < P, then W_32^j, j < 32.  buf1 is the transpose buffer, C goes to buf0; returns buf1.
template <typename T, int P, bool PADL = false>
__device__ __forceinline__ T* dst1_warp_reg(T* buf0, T* buf1, const cpx<T>* tw, int n, int lane) {
    constexpr int M = 32 * P;
    constexpr int G = 32 / P;   // lanes per 32-point DFT in the second stage
    const cpx<T>* rtw = tw + n;
    const cpx<T>* w32 = rtw + M;
    cpx<T> v[P];
#pragma unroll
    for (int p = 0; p < P; ++p) v[p] = packed<T, PADL>(buf0, tw, n, 32 * p + lane);
    dft<T, P>(v);
#pragma unroll
    for (int k = 1; k < P; ++k) v[k] = cmul(v[k], rtw[k * 32 + lane]);
    cpx<T>* sc = reinterpret_cast<cpx<T>*>(buf1);
#pragma unroll
    for (int k = 0; k < P; ++k) sc[swz<T>(k * 32 + lane)] = v[k];
    __syncwarp();
    const int k1 = lane / G, h = lane - k1 * G;
#pragma unroll
    for (int l1 = 0; l1 < P; ++l1) v[l1] = sc[swz<T>(k1 * 32 + G * l1 + h)];
    dft<T, P>(v);
    if (h) {
#pragma unroll
        for (int q = 1; q < P; ++q) v[q] = cmul(v[q], w32[(h * q) & 31]);
    }
    // G-point DFT across the group's lanes; lane h keeps output h
    const int gb = lane - h;
#pragma unroll
    for (int q = 0; q < P; ++q) {
        if (G == 2) {
            const cpx<T> o = shfl_cpx(v[q], lane ^ 1);
            v[q] = h ? csub(o, v[q]) : cadd(v[q], o);
        } else {
            cpx<T> u[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) u[j] = shfl_cpx(v[q], gb + j);
            dft4_impl(u);
            v[q] = h == 0 ? u[0] : h == 1 ? u[1] : h == 2 ? u[2] : u[3];
        }
    }
    cpx<T>* C = reinterpret_cast<cpx<T>*>(buf0);
#pragma unroll
    for (int q = 0; q < P; ++q) C[swz<T>(k1 + P * q + P * P * h)] = v[q];
    __syncwarp();
    if constexpr (PADL) dst_finish_chunked<T, P>(C, buf1, w32 + 32, lane);
    else dst_finish(C, buf1, tw, M, lane);
    return buf1;
}

// Synchronises the TN threads of line group grp (TN = 32: the warp; TN = 64: named barrier
// 1 + grp, one per group of a block).
template <int TN>
__device__ __forceinline__ void line_sync(int grp) {
    if constexpr (TN == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(TN) : "memory");
    }
}

// DST-I of a 1023-point line (n = 1024) on 64 threads: the n/2 = 512-point FFT as 8 x 8 x 8 with
// m = 64 m3 + 8 m2 + m1 and k = k1 + 8 k2 + 64 k3 -- radix-8 DFTs in registers over m3, then
// (after the twiddles W_512^((8 m2 + m1) k1) and a transpose) over m2, then (after W_64^(m1 k2)
// and a second transpose) over m1.  Then the split step in striped order (k = tid + 64 i) and
// the prefix sum of the odd outputs: warp scans of the 8 chunks, one exchange of the 16 warp
// totals through `tot`.  Returns buf0 (natural layout); ends with the group synchronised.
template <typename T>
__device__ __forceinline__ T* dst1_line64(T* buf0, T* buf1, const cpx<T>* tw, int tid, int grp, T* tot) {
    constexpr int n = 1024, M = 512;
    const cpx<T>* t1 = tw + n;        // [k1 * 64 + t] = W_512^(t k1)
    const cpx<T>* t2 = t1 + 512;      // [k2 * 8 + m1] = W_64^(m1 k2)
    cpx<T> v[8];
#pragma unroll
    for (int m3 = 0; m3 < 8; ++m3) v[m3] = packed(buf0, tw, n, 64 * m3 + tid);
    dft8_impl(v);
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) v[k1] = cmul(v[k1], t1[k1 * 64 + tid]);
    cpx<T>* sc = reinterpret_cast<cpx<T>*>(buf1);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) sc[swz<T>(k1 * 64 + tid)] = v[k1];
    line_sync<64>(grp);
    const int hi = tid >> 3, lo = tid & 7;    // stage 2: (k1, m1); stage 3: (k1, k2)
#pragma unroll
    for (int m2 = 0; m2 < 8; ++m2) v[m2] = sc[swz<T>(hi * 64 + 8 * m2 + lo)];
    dft8_impl(v);
#pragma unroll
    for (int k2 = 1; k2 < 8; ++k2) v[k2] = cmul(v[k2], t2[k2 * 8 + lo]);
    cpx<T>* sc2 = reinterpret_cast<cpx<T>*>(buf0);   // the line was consumed before the first sync
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) sc2[swz<T>((hi * 8 + k2) * 8 + lo)] = v[k2];
    line_sync<64>(grp);
#pragma unroll
    for (int m1 = 0; m1 < 8; ++m1) v[m1] = sc2[swz<T>(tid * 8 + m1)];
    dft8_impl(v);
    cpx<T>* C = reinterpret_cast<cpx<T>*>(buf1);
#pragma unroll
    for (int k3 = 0; k3 < 8; ++k3) C[swz<T>(hi + 8 * lo + 64 * k3)] = v[k3];
    line_sync<64>(grp);
    // split step (see dst_finish) in striped order; odd outputs kept for the prefix sum
    T* dst = buf0;
    const int lane = tid & 31, w = tid >> 5;
    T odd[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int k = tid + 64 * i;
        const cpx<T> ck = C[swz<T>(k)];
        const cpx<T> cm = C[swz<T>(k == 0 ? 0 : M - k)];
        const T ex = T(0.5) * (ck.x + cm.x), ey = T(0.5) * (ck.y - cm.y);
        const T dx = T(0.5) * (ck.x - cm.x), dy = T(0.5) * (ck.y + cm.y);
        const cpx<T> wt = tw[2 * k];
        const T yx = ex + (wt.x * dy + wt.y * dx);
        const T yy = ey + (wt.y * dy - wt.x * dx);
        dst[2 * k] = k == 0 ? T(0) : -yy;
        T val = k == 0 ? T(0.5) * yx : yx;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T u = __shfl_up_sync(0xffffffffu, val, off);
            if (lane >= off) val += u;
        }
        odd[i] = val;
        if (lane == 31) tot[2 * i + w] = val;
    }
    line_sync<64>(grp);
    T carry = T(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int k = tid + 64 * i;
        dst[2 * k + 1] = odd[i] + carry + (w ? tot[2 * i] : T(0));
        carry += tot[2 * i] + tot[2 * i + 1];
    }
    line_sync<64>(grp);
    return dst;
}

// One DST-I of a line on the FP path's threads (tid < line_threads(FP), group grp of the block);
// PADL: the line (input and result) in the padded layout of lp (register paths only).
template <typename T, int FP, bool PADL = false>
__device__ __forceinline__ T* dst_line(T* buf0, T* buf1, const cpx<T>* tw, int n, int logn, int tid, int grp, T* tot);

// DST-I of the line held in buf0[1..n-1] (buf0[0] ignored), with buf1 (n values) as scratch.
// tw[k] = exp(-i pi k / n), k < n; tw + n holds the register-path or per-pass tables.  Returns
// the buffer holding the result in [1..n-1] (natural layout).
// FP = 16 or 8 selects the register path (n = 1024 or 512), FP = 0 the Stockham passes; the
// kernels are instantiated per path so that each holds the code of one path only.
template <typename T, int FP, bool PADL = false>
__device__ __forceinline__ T* dst1_warp(T* buf0, T* buf1, const cpx<T>* tw, int n, int logn, int lane) {
    if constexpr (FP != 0) return dst1_warp_reg<T, FP, PADL>(buf0, buf1, tw, n, lane);
    const int M = n >> 1;
    const int logM = logn - 1;
    const cpx<T>* ptw = tw + n;
    // FFT passes: radix 8 while possible, then 4 or 2
    T* src = buf0;
    T* dst = buf1;
    int Ns = 1, rem = logM;
    bool first = true;
    while (rem > 0) {
        const cpx<T>* in = reinterpret_cast<const cpx<T>*>(src);
        cpx<T>* out = reinterpret_cast<cpx<T>*>(dst);
        const T* px = first ? src : nullptr;
        const int R = pass_radix(rem);
        if (R == 8) stockham_pass<T, 8>(in, px, out, tw, ptw, n, M, Ns, lane);
        else if (R == 4) stockham_pass<T, 4>(in, px, out, tw, ptw, n, M, Ns, lane);
        else stockham_pass<T, 2>(in, px, out, tw, ptw, n, M, Ns, lane);
        if (Ns > 1) ptw += (R - 1) * Ns;
        Ns *= R;
        rem -= (R == 8 ? 3 : R == 4 ? 2 : 1);
        first = false;
        T* t = src; src = dst; dst = t;
    }
    // src holds C_k (swizzled); split step into dst (natural layout)
    dst_finish(reinterpret_cast<const cpx<T>*>(src), dst, tw, M, lane);
    return dst;
}

template <typename T, int FP, bool PADL>
__device__ __forceinline__ T* dst_line(T* buf0, T* buf1, const cpx<T>* tw, int n, int logn, int tid, int grp, T* tot) {
    if constexpr (FP == 64) return dst1_line64<T>(buf0, buf1, tw, tid, grp, tot);
    else return dst1_warp<T, FP, PADL>(buf0, buf1, tw, n, logn, tid);
}

// Complex entries of the shared-memory twiddle region for lines of n points: the full table
// exp(-i pi k / n), k < n, then the register-path tables (n / 2 + 32 entries) or the per-pass
// tables (fewer than n / 2 entries).
__host__ __device__ constexpr int tw_region(int n) { return n + n / 2 + 64 + (reg_fft(n) ? n / 2 : 0); }

// Elements a line buffer takes: padded (lp) on the register paths, whose transforms store their
// result in contiguous chunks per lane (dst_finish_chunked).
__host__ __device__ constexpr bool padded_lines(int fp) { return fp == 8 || fp == 16; }
__host__ __device__ constexpr int line_len(int n, int fp) { return padded_lines(fp) ? lp<true>(n) : n; }

// Fills the twiddle region from the 4096-entry table; the loads of one thread are issued back
// to back (batches of 8) before their shared-memory stores.
template <int FP, typename T>
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
    if (FP == 64) {
        // 64-thread path: W_512^(t k1) at [k1 * 64 + t], then W_64^(m1 k2) at [512 + k2 * 8 + m1]
        for (int e = threadIdx.x; e < 576; e += nt) {
            const int j = e < 512 ? (e & 63) * (e >> 6) : 8 * ((e - 512) & 7) * ((e - 512) >> 3);
            const int t = (4 * j) % (2 * n);
            const cpx<T> w = g_tw[(t & (n - 1)) << stride_shift];
            s_tw[n + e] = t >= n ? cpx<T>{-w.x, -w.y} : w;
        }
    } else if (FP == 8 || FP == 16) {
        // W_M^(l k) at [k * 32 + l] (M = n / 2), then W_32^j, then the split step's twiddles in
        // lane-major order for the chunked finish: [i * 32 + l] = exp(-i pi 2 (P l + i) / n)
        const int M = n >> 1, P = M / 32;
        for (int e = threadIdx.x; e < 2 * M + 32; e += nt) {
            int t;
            if (e < M) t = (4 * (e & 31) * (e >> 5)) % (2 * n);
            else if (e < M + 32) t = (e - M) * (n / 16);
            else t = 2 * (P * ((e - M - 32) & 31) + ((e - M - 32) >> 5));
            const cpx<T> w = g_tw[(t & (n - 1)) << stride_shift];
            s_tw[n + e] = t >= n ? cpx<T>{-w.x, -w.y} : w;
        }
    } else {
        for (int e = threadIdx.x; e < n / 2; e += nt) {
            bool valid;
            const cpx<T> w = pass_twiddle_entry(g_tw, n, logn, e, valid);
            if (valid) s_tw[n + e] = w;
        }
    }
}

template <typename T>
using vec16_t = typename std::conditional<sizeof(T) == 4, float4, double2>::type;

// 16-byte vector q of a row in a line buffer (plain or padded layout).  In the padded layout a
// vector's elements 0-1 and 2-3 (FP32) stay adjacent pairs: no multiple of 32 falls inside a pair.
template <typename T, bool PADL>
__device__ __forceinline__ void line_put16(T* line, int q, vec16_t<T> v) {
    if constexpr (!PADL || sizeof(T) == 8) {
        *reinterpret_cast<vec16_t<T>*>(line + lp<PADL>(q * (16 / (int)sizeof(T)))) = v;
    } else {
        float2* d = reinterpret_cast<float2*>(line + lp<true>(4 * q));
        d[0] = make_float2(v.x, v.y);
        d[1] = make_float2(v.z, v.w);
    }
}
template <typename T, bool PADL>
__device__ __forceinline__ vec16_t<T> line_get16(const T* line, int q) {
    if constexpr (!PADL || sizeof(T) == 8) {
        return *reinterpret_cast<const vec16_t<T>*>(line + lp<PADL>(q * (16 / (int)sizeof(T))));
    } else {
        const float2* d = reinterpret_cast<const float2*>(line + lp<true>(4 * q));
        const float2 a = d[0], b = d[1];
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

// Loads nx values of a padded row (16-byte aligned) into a line buffer with vector loads,
// batches of 8 loads in flight per lane.
template <typename T, int TN = 32, bool PADL = false>
__device__ __forceinline__ void load_row_vec(T* line, const T* __restrict__ g, int nx, int lane) {
    constexpr int V = 16 / sizeof(T);
    using VT = vec16_t<T>;
    const VT* src = reinterpret_cast<const VT*>(g);
    const int nv = nx / V;
    for (int q0 = lane; q0 < nv; q0 += 8 * TN) {
        VT v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (q0 + TN * b < nv) v[b] = src[q0 + TN * b];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (q0 + TN * b < nv) line_put16<T, PADL>(line, q0 + TN * b, v[b]);
    }
}

template <typename T, int TN = 32, bool PADL = false>
__device__ __forceinline__ void store_row_vec(T* __restrict__ g, const T* line, int nx, int lane) {
    constexpr int V = 16 / sizeof(T);
    using VT = vec16_t<T>;
    VT* dst = reinterpret_cast<VT*>(g);
    const int nv = nx / V;
#pragma unroll 4
    for (int q = lane; q < nv; q += TN) dst[q] = line_get16<T, PADL>(line, q);
}

// Loads a padded FP64 row (16-byte aligned, nx values) into a line buffer of T.
template <typename T, int TN = 32, bool PADL = false>
__device__ __forceinline__ void load_row_f64(T* line, const double* __restrict__ g, int nx, int lane) {
    const double2* src = reinterpret_cast<const double2*>(g);
    const int nv = nx / 2;
    for (int q0 = lane; q0 < nv; q0 += 8 * TN) {
        double2 v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (q0 + TN * b < nv) v[b] = src[q0 + TN * b];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int q = q0 + TN * b;
            if (q < nv) {
                vec2_t<T> w;
                w.x = (T)v[b].x;
                w.y = (T)v[b].y;
                *reinterpret_cast<vec2_t<T>*>(line + lp<PADL>(2 * q)) = w;
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

// Twiddles of a block: the register paths (n = 512, 1024) read the region table straight from
// global memory (L1-cached; fewer shared-memory bytes per block, more blocks per SM); the
// Stockham path (other n) copies it into the first tw_region(n) entries of shared memory (its
// per-pass tables are read with strided indices that L1 serves poorly).  Returns the table the
// transforms read; the caller synchronises the block before using a staged copy.
template <int FP, typename T>
__device__ __forceinline__ const cpx<T>* block_twiddles(unsigned char* smem, const cpx<T>* __restrict__ twr, int n) {
    if constexpr (FP != 0) {
        return twr;
    } else {
        cpx<T>* st = reinterpret_cast<cpx<T>*>(smem);
        for (int k = threadIdx.x; k < tw_region(n); k += blockDim.x) st[k] = twr[k];
        return st;
    }
}
// Shared-memory bytes the twiddles take in front of the lines.
template <typename T>
__host__ __device__ constexpr size_t twiddle_smem(int n, int fp) {
    return fp == 0 ? (size_t)tw_region(n) * sizeof(cpx<T>) : 0;
}

// Per-line scratch for the 64-thread path's prefix sum (16 values per line).
constexpr int kLineScratch = 16;

// Forward row transforms.  Row r (interior row index) of the input is
//   dense[r*dld + doff + i] (FP64, optional) + box terms / h^2 (optional ring)
//   + gsign * gamma at the affected points of the row (optional)
// and the transformed row is written to out (padded layout).  `stop` (optional): a set flag
// makes the launch a no-op.  Each line is handled by line_threads(FP) threads.
template <typename T, int WARPS, int FP>
__device__ __forceinline__ void
rows_fwd_body(int NX, int NY, int n, int logn, int row0, int nrows, const double* __restrict__ dense, int dld, int doff,
              const double* __restrict__ ring, double ih2, const int* __restrict__ aff_row_ptr,
              const int* __restrict__ aff_node, VecArg gam, double gsign, const cpx<T>* __restrict__ g_tw,
              T* __restrict__ out) {
    constexpr int TN = line_threads(FP), LPB = WARPS * 32 / TN;
    constexpr bool PADL = padded_lines(FP);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const cpx<T>* s_tw = block_twiddles<FP, T>(smem_raw, g_tw, n);
    const int grp = threadIdx.x / TN, tid = threadIdx.x - grp * TN;
    const int LN = line_len(n, FP);
    T* lines = reinterpret_cast<T*>(smem_raw + twiddle_smem<T>(n, FP));
    T* b0 = lines + (size_t)grp * (2 * LN);
    T* b1 = b0 + LN;
    T* tot = lines + (size_t)LPB * 2 * LN + grp * kLineScratch;
    if (FP == 0) __syncthreads();
    const int r = row0 + blockIdx.x * LPB + grp;
    if (r >= row0 + nrows || r >= NY) return;   // uniform over the line's threads
    if (dense && dld == n && doff == 1) {
        load_row_f64<T, TN, PADL>(b0, dense + (size_t)r * n, n, tid);   // padded row: slot 0 is a pad
    } else if (dense) {
        const double* src = dense + (size_t)r * dld + doff;
#pragma unroll 8
        for (int i = tid; i < NX; i += TN) b0[lp<PADL>(i + 1)] = (T)src[i];
    } else {
        for (int i = tid; i < NX; i += TN) b0[lp<PADL>(i + 1)] = T(0);
    }
    line_sync<TN>(grp);
    if (ring) {
        // ring: bottom row (nx+1), top row (nx+1), left column (ny-1), right column (ny-1)
        const int nxp1 = NX + 2;
        if (tid == 0) {
            b0[lp<PADL>(1)] += (T)(ring[2 * nxp1 + r] * ih2);
            b0[lp<PADL>(NX)] += (T)(ring[2 * nxp1 + NY + r] * ih2);
        }
        line_sync<TN>(grp);
        if (r == 0)
            for (int i = tid; i < NX; i += TN) b0[lp<PADL>(i + 1)] += (T)(ring[i + 1] * ih2);
        if (r == NY - 1)
            for (int i = tid; i < NX; i += TN) b0[lp<PADL>(i + 1)] += (T)(ring[nxp1 + i + 1] * ih2);
        line_sync<TN>(grp);
    }
    if (gam.base) {
        const double* gv = gam.get();
        const int a0 = aff_row_ptr[r], a1 = aff_row_ptr[r + 1];
        for (int a = a0 + tid; a < a1; a += TN) b0[lp<PADL>(aff_node[a] - r * n)] += (T)(gsign * gv[a]);
        line_sync<TN>(grp);
    }
    T* res = dst_line<T, FP, PADL>(b0, b1, s_tw, n, logn, tid, grp, tot);
    if (tid == 0) res[0] = T(0);
    line_sync<TN>(grp);
    store_row_vec<T, TN, PADL>(out + (size_t)r * n, res, n, tid);
}

// blockIdx.y selects one of several fields: dense input dfs and output ofs elements apart.
template <typename T, int WARPS, int FP>
__global__ void __launch_bounds__(WARPS * 32)
k_rows_fwd(int NX, int NY, int n, int logn, int row0, int nrows, const double* __restrict__ dense, int dld, int doff,
           const double* __restrict__ ring, double ih2, const int* __restrict__ aff_row_ptr,
           const int* __restrict__ aff_node, VecArg gam, double gsign, const cpx<T>* __restrict__ g_tw,
           T* __restrict__ out, const int* __restrict__ stop, long dfs, long ofs) {
    if (stop && *stop) return;
    rows_fwd_body<T, WARPS, FP>(NX, NY, n, logn, row0, nrows, dense ? dense + (long)blockIdx.y * dfs : nullptr, dld,
                                doff, ring, ih2, aff_row_ptr, aff_node, gam, gsign, g_tw,
                                out + (long)blockIdx.y * ofs);
}

// Column pass on padded columns p = 1..NX (p = 0 is the pad): forward y transform, division
// by the eigenvalues (with the 2D normalisation), inverse y transform.  Rows outside [in0, in1]
// are zero on input; only rows [out0, out1] are written back.  C columns per block,
// line_threads(FP) threads per column; blockIdx.y selects one of several fields fstride
// elements apart.
template <typename T, int C, int FP>
__device__ __forceinline__ void
cols_body(int NX, int NY, int n, int logn, int in0, int in1, int out0, int out1, T* __restrict__ buf,
          const T* __restrict__ lam_x, const T* __restrict__ lam_y, T norm, const cpx<T>* __restrict__ g_tw) {
    constexpr int TN = line_threads(FP);
    constexpr bool PADL = padded_lines(FP);   // lines in the padded layout (lp)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const cpx<T>* s_tw = block_twiddles<FP, T>(smem_raw, g_tw, n);   // synchronised with the tile below
    constexpr int PAD = sizeof(T) == 4 ? 4 : 2;
    const int LN = line_len(n, FP);
    const int stride = 2 * LN + PAD;
    T* s_lam = reinterpret_cast<T*>(smem_raw + twiddle_smem<T>(n, FP));   // lam_y, NY values
    T* lines = s_lam + n;
    const int grp = threadIdx.x / TN, tid = threadIdx.x - grp * TN;
    T* tot = lines + (size_t)C * stride + grp * kLineScratch;
    const int ld = NX + 1;
    const int col0 = blockIdx.x * C;   // padded column index
    constexpr int nthr = C * TN;
    for (int l = threadIdx.x; l < NY; l += nthr) s_lam[l] = lam_y[l];
    // tile load: C consecutive padded columns of rows [in0, in1]; rows outside are zero
    constexpr int V = 16 / sizeof(T);
    constexpr int VPR = C / V;                   // vectors per row
    using VT = vec16_t<T>;
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
                for (int c = 0; c < V; ++c) lines[(q * V + c) * stride + lp<PADL>(rr + 1)] = vs[c];
            }
        }
    }
    __syncthreads();
    const int p = col0 + grp;
    if (p >= 1 && p <= NX) {   // uniform over the column's threads
        T* b0 = lines + grp * stride;
        T* b1 = b0 + LN;
        // forward transform, division, inverse transform: one copy of the transform code
        T* in = b0;
        T* other = b1;
        const T lx = lam_x[p - 1];
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            T* f = dst_line<T, FP, PADL>(in, other, s_tw, n, logn, tid, grp, tot);
            if (pass == 0) {
                for (int l = tid; l < NY; l += TN) f[lp<PADL>(l + 1)] = f[lp<PADL>(l + 1)] * (norm / (lx + s_lam[l]));
                line_sync<TN>(grp);
            }
            other = (f == in) ? other : in;
            in = f;
        }
        // bring the result back to b0 so that the tile store below has a fixed layout
        if (in != b0) {
            for (int l = tid; l < NY; l += TN) b0[lp<PADL>(l + 1)] = in[lp<PADL>(l + 1)];
        }
    }
    __syncthreads();
    const int nout = out1 - out0 + 1;
    for (int t = threadIdx.x; t < nout * VPR; t += nthr) {
        const int rr = out0 + t / VPR, q = t % VPR;
        VT v;
        T* vs = reinterpret_cast<T*>(&v);
#pragma unroll
        for (int c = 0; c < V; ++c) {
            const int pc = col0 + q * V + c;
            vs[c] = (pc >= 1 && pc <= NX) ? lines[(q * V + c) * stride + lp<PADL>(rr + 1)] : T(0);
        }
        *reinterpret_cast<VT*>(buf + (size_t)rr * ld + col0 + q * V) = v;
    }
}

template <typename T, int C, int FP>
__global__ void __launch_bounds__(C * line_threads(FP), sizeof(T) == 4 ? 2 : 1)
k_cols(int NX, int NY, int n, int logn, int in0, int in1, int out0, int out1, T* __restrict__ buf,
       const T* __restrict__ lam_x, const T* __restrict__ lam_y, T norm, const cpx<T>* __restrict__ g_tw,
       const int* __restrict__ stop, long fstride) {
    if (stop && *stop) return;
    cols_body<T, C, FP>(NX, NY, n, logn, in0, in1, out0, out1, buf + (long)blockIdx.y * fstride, lam_x, lam_y, norm,
                        g_tw);
}

enum RowsInvMode { INV_STORE_T = 0, INV_STORE_F64 = 1, INV_ACCUM_FLUID = 2, INV_ACCUM_T = 3 };

// Inverse row transforms of rows [row0, row0 + nrows) of a padded buffer.
//   INV_STORE_T     outT (padded) = transform
//   INV_STORE_F64   out64[r*old + ooff + i] = transform
//   INV_ACCUM_FLUID out64 (padded) += transform at fluid nodes (class FLUID / PLUS) only
//   INV_ACCUM_T     outT (padded) += transform
// blockIdx.y selects one of several fields fstride elements apart (in and outT).
template <typename T, int WARPS, int MODE, int FP>
__device__ __forceinline__ void
rows_inv_body(int NX, int NY, int n, int logn, int row0, int nrows, const T* __restrict__ in, T* __restrict__ outT,
              double* __restrict__ out64, int old, int ooff, const uint8_t* __restrict__ cls,
              const cpx<T>* __restrict__ g_tw) {
    constexpr int TN = line_threads(FP), LPB = WARPS * 32 / TN;
    constexpr bool PADL = padded_lines(FP);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const cpx<T>* s_tw = block_twiddles<FP, T>(smem_raw, g_tw, n);
    const int grp = threadIdx.x / TN, tid = threadIdx.x - grp * TN;
    const int LN = line_len(n, FP);
    T* lines = reinterpret_cast<T*>(smem_raw + twiddle_smem<T>(n, FP));
    T* b0 = lines + (size_t)grp * (2 * LN);
    T* b1 = b0 + LN;
    T* tot = lines + (size_t)LPB * 2 * LN + grp * kLineScratch;
    if (FP == 0) __syncthreads();
    const int r = row0 + blockIdx.x * LPB + grp;
    if (r >= row0 + nrows || r >= NY) return;   // uniform over the line's threads
    load_row_vec<T, TN, PADL>(b0, in + (size_t)r * n, n, tid);
    line_sync<TN>(grp);
    T* res = dst_line<T, FP, PADL>(b0, b1, s_tw, n, logn, tid, grp, tot);
    if (MODE == INV_STORE_T) {
        if (tid == 0) res[0] = T(0);
        line_sync<TN>(grp);
        store_row_vec<T, TN, PADL>(outT + (size_t)r * n, res, n, tid);
    } else if (MODE == INV_STORE_F64) {
        double* dst = out64 + (size_t)r * old + ooff;
#pragma unroll 4
        for (int i = tid; i < NX; i += TN) dst[i] = (double)res[lp<PADL>(i + 1)];
    } else if (MODE == INV_ACCUM_T) {
        T* dst = outT + (size_t)r * n + 1;
#pragma unroll 4
        for (int i = tid; i < NX; i += TN) dst[i] += res[lp<PADL>(i + 1)];
    } else {
        // padded positions p = 1..NX of the row: p = 1 alone, then the pairs (p, p + 1) for even
        // p, each one 16-byte FP64 read-modify-write (rows start on even indices) with a 2-byte
        // class load; each lane issues all its loads before its first add
        const size_t base = (size_t)r * n;
        if (tid == 0 && cls[base + 1] <= CLS_PLUS) out64[base + 1] += (double)res[lp<PADL>(1)];
        const int npair = (NX - 1) / 2;
        double2* o2 = reinterpret_cast<double2*>(out64 + base + 2);
        const uchar2* c2 = reinterpret_cast<const uchar2*>(cls + base + 2);
        constexpr int B = 8;
        for (int q0 = tid; q0 < npair; q0 += B * TN) {
            double2 o[B];
            uchar2 c[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int q = q0 + b * TN;
                if (q < npair) {
                    c[b] = c2[q];
                    o[b] = o2[q];
                }
            }
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int q = q0 + b * TN;
                if (q < npair) {
                    const int pp = 2 + 2 * q;   // even: lp keeps (pp, pp + 1) adjacent
                    const vec2_t<T> v = *reinterpret_cast<const vec2_t<T>*>(res + lp<PADL>(pp));
                    if (c[b].x <= CLS_PLUS) o[b].x += (double)v.x;
                    if (c[b].y <= CLS_PLUS) o[b].y += (double)v.y;
                    o2[q] = o[b];
                }
            }
        }
    }
}

template <typename T, int WARPS, int MODE, int FP>
__global__ void __launch_bounds__(WARPS * 32)
k_rows_inv(int NX, int NY, int n, int logn, int row0, int nrows, const T* __restrict__ in, T* __restrict__ outT,
           double* __restrict__ out64, int old, int ooff, const uint8_t* __restrict__ cls,
           const cpx<T>* __restrict__ g_tw, const int* __restrict__ stop, long fstride) {
    if (stop && *stop) return;
    rows_inv_body<T, WARPS, MODE, FP>(NX, NY, n, logn, row0, nrows, in + (long)blockIdx.y * fstride,
                                      outT ? outT + (long)blockIdx.y * fstride : nullptr, out64, old, ooff, cls, g_tw);
}

}  // namespace iim
