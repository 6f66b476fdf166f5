// Learned initial guess for the IIM Poisson iteration: a small fully convolutional network
// (3x3 convolutions with dilation, ReLU between layers, BF16 weights, FP32 accumulation),
// trained on solves that the method itself produces, with hand-written forward, backward and
// Adam kernels.  The paper has no learned component; the solver's own residual decides
// whether a guess is used (iim_poisson_solve falls back to zero when the guess raises it).
//
//   y[b,o,i,j] = bias[o] + sum_{c,ky,kx} W[o,c,ky,kx] x[b,c,i + d(ky-1), j + d(kx-1)]  (zero padding)
//   loss = sum(mask (pred - target)^2) / sum(mask)
//   input gradient  = convolution of the (ReLU-gated) output gradient with the flipped kernel
//   weight gradient = sum over pixels of output gradient x shifted input
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "common.cuh"
#include "iim_ops.cuh"
#include "tcgen05.cuh"

struct iim_net_s {
    int device = 0;
    int cin = 0, hidden = 0, nl = 0;
    std::vector<int> dil, ci, co;        // per layer
    std::vector<long long> woff, boff;   // parameter offsets
    long long np = 0;
    float* p = nullptr;                  // FP32 master parameters
    float* gr = nullptr;                 // gradients
    float* m = nullptr;                  // Adam moments
    float* v = nullptr;
    __nv_bfloat16* wb = nullptr;         // BF16 weights used by the kernels
    __nv_bfloat16* wt = nullptr;         // flipped / transposed BF16 weights (input gradient)
    long long t = 0;                     // Adam step
    float* act = nullptr;                // layer outputs, nl x cap floats
    float* g0 = nullptr;                 // gradient ping-pong, 2 x cap floats
    float* red = nullptr;                // reductions
    long long cap = 0;                   // floats per activation buffer
    float* h_red = nullptr;              // pinned
    int tc = 0;                          // tensor cores (k_conv_tc): 0 off, 1 the 32 -> 32 layers, 2 every layer
    __nv_bfloat16* wtc = nullptr;        // one layer's weights in the tensor-core operand layout
    int* tc_err = nullptr;               // set by k_conv_tc when its wait for the MMAs timed out
};

namespace iim {

constexpr int TX = 16, TY = 16;

// out = conv(x) (+bias) (+ReLU); input values gated by `gate > 0` when gate is given.
template <int CO_T>
__global__ void __launch_bounds__(TX * TY)
k_conv(const float* __restrict__ x, const float* __restrict__ gate, const __nv_bfloat16* __restrict__ w,
       const float* __restrict__ bias, float* __restrict__ y, int Ci, int Co, int H, int W, int d, int relu) {
    extern __shared__ float sm[];
    const int tw = TX + 2 * d, th = TY + 2 * d;
    float* tile = sm;
    float* wsm = sm + tw * th;
    const int ncot = (Co + CO_T - 1) / CO_T;
    const int b = blockIdx.z / ncot, co0 = (blockIdx.z % ncot) * CO_T;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const size_t plane = (size_t)H * W;
    float acc[CO_T];
#pragma unroll
    for (int c = 0; c < CO_T; ++c) acc[c] = 0.f;
    for (int ci = 0; ci < Ci; ++ci) {
        const float* xc = x + ((size_t)b * Ci + ci) * plane;
        const float* gc = gate ? gate + ((size_t)b * Ci + ci) * plane : nullptr;
        for (int t = tid; t < tw * th; t += TX * TY) {
            const int ly = t / tw, lx = t - ly * tw;
            const int gy = y0 - d + ly, gx = x0 - d + lx;
            float v = 0.f;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                v = xc[(size_t)gy * W + gx];
                if (gc && !(gc[(size_t)gy * W + gx] > 0.f)) v = 0.f;
            }
            tile[t] = v;
        }
        for (int t = tid; t < CO_T * 9; t += TX * TY) {
            const int c = co0 + t / 9;
            wsm[t] = c < Co ? __bfloat162float(w[((size_t)c * Ci + ci) * 9 + t % 9]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float v = tile[(ty + d * (k / 3)) * tw + tx + d * (k % 3)];
#pragma unroll
            for (int c = 0; c < CO_T; ++c) acc[c] = fmaf(wsm[c * 9 + k], v, acc[c]);
        }
        __syncthreads();
    }
    const int gy = y0 + ty, gx = x0 + tx;
    if (gy < H && gx < W) {
#pragma unroll
        for (int c = 0; c < CO_T; ++c) {
            if (co0 + c >= Co) break;
            float v = acc[c] + (bias ? bias[co0 + c] : 0.f);
            if (relu) v = fmaxf(v, 0.f);
            y[((size_t)b * Co + co0 + c) * plane + (size_t)gy * W + gx] = v;
        }
    }
}

// Convolution of Ci <= 32 input to Co <= 32 output channels as an implicit GEMM on the tensor
// cores (tcgen05, BF16 operands, FP32 accumulation in tensor memory).  One CTA computes a run of
// TC_M = 128 pixels of one image row for NO output columns (16 or 32, the MMA's N; outputs
// o >= Co are zero columns): D (128 x NO) = sum over the 9 taps and the CG / 2 16-channel parts of
// the CG staged 8-channel groups (CG = 2 or 4; channels c >= Ci are zero) of
// A_tap (128 pixels x 16 channels) * B_tap^T (NO outputs x 16 channels), MMAs of M = 128, K = 16.
//
// Shared memory, in 16-byte units of 8 BF16 channels:
//   A: input rows row - d, row, row + d (r = 0, 1, 2), channel group g, pixel p = 0 .. NP - 1
//      standing for column x0 - d + p (NP = 128 + 2 d), unit (r * CG + g) * NP + p; zero outside
//      the image.  The operand of tap (ky, kx) starts at pixel kx * d of row ky: consecutive
//      pixels are 16 bytes apart (stride byte offset 128 per 8 rows), the second channel group of
//      an MMA is NP units further (leading byte offset).
//   B: tap t, channel group g, output o: unit (t * CG + g) * NO + o (packed by k_pack_w_tc).
// The input is rounded to BF16 on the way in (optionally gated by gate > 0, as k_conv); the
// epilogue adds the bias, applies the ReLU and writes FP32 in the NCHW layout of k_conv.
// A wait for the MMAs that runs past one second sets *err and skips the epilogue.
constexpr int TC_M = 128, TC_C = 32;

__host__ __device__ constexpr size_t conv_tc_smem(int d, int cg, int no) {
    return (size_t)16 * (3 * cg * (TC_M + 2 * d) + 9 * cg * no) + 16;
}

// wp[((t * CG + g) * NO + o) * 8 + e] = w[(o * Ci + 8 g + e) * 9 + t], zero for o >= Co or
// 8 g + e >= Ci
template <int CG, int NO>
__global__ void k_pack_w_tc(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wp, int Ci, int Co) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * CG * NO * 8) return;
    const int e = i & 7, o = (i >> 3) % NO, g = ((i >> 3) / NO) % CG, t = (i >> 3) / (NO * CG);
    const int c = 8 * g + e;
    wp[i] = (o < Co && c < Ci) ? w[(o * Ci + c) * 9 + t] : __float2bfloat16(0.f);
}

__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // a at the lower address
    return *reinterpret_cast<const uint32_t*>(&v);
}

template <int CG, int NO>
__global__ void __launch_bounds__(128)
k_conv_tc(const float* __restrict__ x, const float* __restrict__ gate, const __nv_bfloat16* __restrict__ wp,
          const float* __restrict__ bias, float* __restrict__ y, int Ci, int Co, int H, int W, int d, int relu,
          int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int NP = TC_M + 2 * d;
    uint4* sA = reinterpret_cast<uint4*>(smem_raw);
    uint4* sB = sA + 3 * CG * NP;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + 9 * CG * NO);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * TC_M, row = blockIdx.y, b = blockIdx.z;
    const size_t plane = (size_t)H * W;
    const float* xb = x + (size_t)b * Ci * plane;
    const float* gb = gate ? gate + (size_t)b * Ci * plane : nullptr;

    if (warp == 0) tc::tmem_alloc(tslot, 32);
    if (tid == 0) tc::mbar_init(mbar, 1);
    const uint4* wsrc = reinterpret_cast<const uint4*>(wp);
    for (int i = tid; i < 9 * CG * NO; i += 128) sB[i] = wsrc[i];
    // UB units per thread and round, all their loads issued before any conversion
    constexpr int UB = 2;
    const int units = 3 * CG * NP;
    for (int u0 = tid; u0 < units; u0 += UB * 128) {
        float v[UB][8];
        bool in[UB];
        size_t off[UB];
        int c0[UB];
#pragma unroll
        for (int q = 0; q < UB; ++q) {
            const int u = u0 + q * 128;
            const int rg = u / NP, p = u - rg * NP;
            const int r = rg / CG, g = rg - r * CG;
            const int gy = row + (r - 1) * d, gx = x0 - d + p;
            in[q] = u < units && gy >= 0 && gy < H && gx >= 0 && gx < W;
            c0[q] = 8 * g;
            off[q] = in[q] ? (size_t)(8 * g) * plane + (size_t)gy * W + gx : 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) v[q][e] = (in[q] && c0[q] + e < Ci) ? xb[off[q] + (size_t)e * plane] : 0.f;
        }
        if (gb) {
#pragma unroll
            for (int q = 0; q < UB; ++q)
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (in[q] && c0[q] + e < Ci && !(gb[off[q] + (size_t)e * plane] > 0.f)) v[q][e] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < UB; ++q) {
            const int u = u0 + q * 128;
            if (u < units)
                sA[u] = make_uint4(bf16x2_bits(v[q][0], v[q][1]), bf16x2_bits(v[q][2], v[q][3]),
                                   bf16x2_bits(v[q][4], v[q][5]), bf16x2_bits(v[q][6], v[q][7]));
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
        constexpr uint32_t idesc = tc::idesc_bf16_f32(TC_M, NO);
#pragma unroll 1
        for (int t = 0; t < 9; ++t) {
            const int ky = t / 3, kx = t - 3 * ky;
#pragma unroll
            for (int s = 0; s < CG / 2; ++s) {
                const uint64_t ad =
                    tc::desc_kmajor(a0 + (uint32_t)(16 * ((ky * CG + 2 * s) * NP + kx * d)), (uint32_t)(16 * NP), 128u);
                const uint64_t bd = tc::desc_kmajor(b0 + (uint32_t)(16 * (t * CG + 2 * s) * NO), 16u * NO, 128u);
                tc::mma_bf16(tmem, ad, bd, idesc, (t | s) != 0);
            }
        }
        tc::commit(mbar);
    }
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait_bounded(mbar, 0, 1000000000ull));
    tc::fence_after_sync();
    if (ok) {
        float acc[NO];
        if constexpr (NO == 32) tc::tmem_ld_32x32(tmem + ((uint32_t)(32 * warp) << 16), acc);
        else tc::tmem_ld_32x16(tmem + ((uint32_t)(32 * warp) << 16), acc);
        const int gx = x0 + 32 * warp + lane;
        if (gx < W) {
            float* yo = y + (size_t)b * Co * plane + (size_t)row * W + gx;
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                if (o >= Co) break;
                float v = acc[o] + (bias ? bias[o] : 0.f);
                if (relu) v = fmaxf(v, 0.f);
                yo[(size_t)o * plane] = v;
            }
        }
    } else if (lane == 0) {
        atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        if (!ok) (void)tc::mbar_wait_bounded(mbar, 0, 1000000000ull);
        tc::tmem_dealloc(tmem, 32);
    }
}

// dW[o,c,k] += sum_{b,p} g[b,o,p] x[b,c,p + d off(k)], db[o] += sum g (g gated by gate > 0).
// One block per 64 x 64 pixel region and image; thread t -> (o = t / 9, k = t % 9).
constexpr int WG_R = 64, WG_S = 16, WG_MAXC = 32;
__global__ void __launch_bounds__(288)
k_conv_wgrad(const float* __restrict__ x, const float* __restrict__ g, const float* __restrict__ gate,
             float* __restrict__ dw, float* __restrict__ db, int Ci, int Co, int H, int W, int d) {
    extern __shared__ float sm[];
    float* gt = sm;                               // Co x 256
    float* xt = sm + WG_MAXC * WG_S * WG_S;       // (16 + 2d)^2
    const int tw = WG_S + 2 * d;
    const int b = blockIdx.z;
    const int t = threadIdx.x;
    const int o = t / 9, k = t % 9;
    const bool active = o < Co;
    const size_t plane = (size_t)H * W;
    float acc[WG_MAXC];
#pragma unroll
    for (int c = 0; c < WG_MAXC; ++c) acc[c] = 0.f;
    float bacc = 0.f;
    for (int sy = 0; sy < WG_R / WG_S; ++sy) {
        for (int sx = 0; sx < WG_R / WG_S; ++sx) {
            const int py0 = blockIdx.y * WG_R + sy * WG_S, px0 = blockIdx.x * WG_R + sx * WG_S;
            if (py0 >= H || px0 >= W) continue;   // uniform across the block
            for (int q = t; q < Co * WG_S * WG_S; q += blockDim.x) {
                const int oo = q / (WG_S * WG_S), pp = q % (WG_S * WG_S);
                const int gy = py0 + pp / WG_S, gx = px0 + pp % WG_S;
                float v = 0.f;
                if (gy < H && gx < W) {
                    const size_t idx = ((size_t)b * Co + oo) * plane + (size_t)gy * W + gx;
                    v = g[idx];
                    if (gate && !(gate[idx] > 0.f)) v = 0.f;
                }
                gt[q] = v;
            }
            __syncthreads();
            if (active && k == 4) {
                float s = 0.f;
                for (int pp = 0; pp < WG_S * WG_S; ++pp) s += gt[o * WG_S * WG_S + pp];
                bacc += s;
            }
#pragma unroll
            for (int c = 0; c < WG_MAXC; ++c) {
                if (c < Ci) {
                    const float* xc = x + ((size_t)b * Ci + c) * plane;
                    for (int q = t; q < tw * tw; q += blockDim.x) {
                        const int ly = q / tw, lx = q - ly * tw;
                        const int gy = py0 - d + ly, gx = px0 - d + lx;
                        xt[q] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? xc[(size_t)gy * W + gx] : 0.f;
                    }
                    __syncthreads();
                    if (active) {
                        const float* gr = gt + o * WG_S * WG_S;
                        const int oy = d * (k / 3), ox = d * (k % 3);
                        float s = 0.f;
                        for (int py = 0; py < WG_S; ++py)
#pragma unroll 4
                            for (int px = 0; px < WG_S; ++px) s = fmaf(gr[py * WG_S + px], xt[(py + oy) * tw + px + ox], s);
                        acc[c] += s;
                    }
                    __syncthreads();
                }
            }
        }
    }
    if (active) {
#pragma unroll
        for (int c = 0; c < WG_MAXC; ++c)
            if (c < Ci) atomicAdd(&dw[((size_t)o * Ci + c) * 9 + k], acc[c]);
        if (k == 4) atomicAdd(&db[o], bacc);
    }
}

// diff = (pred - target) mask; partial sums of diff^2 and mask
__global__ void k_mse_partial(long n, const float* __restrict__ pred, const float* __restrict__ target,
                              const float* __restrict__ mask, float* __restrict__ diff, float* __restrict__ part) {
    float s2 = 0.f, sm_ = 0.f;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float m = mask ? mask[i] : 1.f;
        const float dd = (pred[i] - target[i]) * m;
        diff[i] = dd;
        s2 += dd * dd;
        sm_ += m;
    }
    for (int off = 16; off > 0; off >>= 1) {
        s2 += __shfl_down_sync(0xffffffffu, s2, off);
        sm_ += __shfl_down_sync(0xffffffffu, sm_, off);
    }
    __shared__ float a[32], c[32];
    if ((threadIdx.x & 31) == 0) { a[threadIdx.x >> 5] = s2; c[threadIdx.x >> 5] = sm_; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float x2 = 0.f, xm = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { x2 += a[w]; xm += c[w]; }
        part[2 * blockIdx.x] = x2;
        part[2 * blockIdx.x + 1] = xm;
    }
}

__global__ void k_mse_finish(int nb, float* __restrict__ part, float* __restrict__ out) {
    if (threadIdx.x != 0) return;
    float x2 = 0.f, xm = 0.f;
    for (int b = 0; b < nb; ++b) { x2 += part[2 * b]; xm += part[2 * b + 1]; }
    out[0] = xm > 0.f ? x2 / xm : 0.f;
    out[1] = xm > 0.f ? 2.f / xm : 0.f;
}

__global__ void k_scale_vec(long n, float* __restrict__ v, const float* __restrict__ s) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] *= *s;
}

__global__ void k_adam(long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(long n, const float* __restrict__ p, __nv_bfloat16* __restrict__ out) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16(p[i]);
}

// wt[c][o][k] = W[o][c][8 - k]
__global__ void k_flip(int Ci, int Co, const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Ci * Co * 9) return;
    const int k = t % 9, o = (t / 9) % Co, c = t / (9 * Co);
    wt[t] = w[((size_t)o * Ci + c) * 9 + (8 - k)];
}

// x[b] = (omega s0, phi s1, ub s2) on the interior grid, channel planes of NX x NY
__global__ void k_net_input(int NX, int NY, const double* __restrict__ omega, const double* __restrict__ phi,
                            const double* __restrict__ ub, float s0, float s1, float s2, float* __restrict__ x) {
    const long n = (long)NX * NY;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = (int)(k % NX), j = (int)(k / NX);
    const double ph = phi[(long)(j + 1) * (NX + 2) + (i + 1)];
    x[k] = (float)(ph >= 0.0 ? omega[k] * s0 : 0.0);
    x[n + k] = (float)(ph * s1);
    x[2 * n + k] = (float)(ub[k] * s2);
}

// psi = ub + y / s
__global__ void k_net_guess(long n, const double* __restrict__ ub, const float* __restrict__ y, float inv_s,
                            double* __restrict__ psi) {
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) psi[k] = ub[k] + (double)(y[k] * inv_s);
}

static size_t conv_smem(int d, int co_t) { return sizeof(float) * ((size_t)(TX + 2 * d) * (TY + 2 * d) + 9 * co_t); }

static iim_status conv(iim_net_s* net, const float* x, const float* gate, const __nv_bfloat16* w, const float* bias,
                       float* y, int B, int Ci, int Co, int H, int W, int d, int relu, cudaStream_t s) {
    const dim3 blk(TX, TY);
    // tensor cores: mode 1 the 32 -> 32 layers, mode 2 every layer (K and N padded to 16 / 32)
    if ((net->tc == 1 && Ci == TC_C && Co == TC_C) || (net->tc == 2 && Ci <= TC_C && Co <= TC_C)) {
        auto go = [&](auto pack, auto kern, int cg, int no) -> iim_status {
            launch("net_pack_w_tc", 0.0, 0.0, pack, (9 * cg * no * 8 + 255) / 256, 256, 0, s, w, net->wtc, Ci, Co);
            IIM_LAUNCHED();
            const size_t sm = conv_tc_smem(d, cg, no);
            IIM_CHECK(allow_smem(kern, sm));
            launch("net_conv_tc", 4.0 * (double)B * H * W * (Ci * (gate ? 2 : 1) + Co),
                   18.0 * (double)B * H * W * Ci * Co, kern, dim3((W + TC_M - 1) / TC_M, H, B), 128, sm, s, x, gate,
                   (const __nv_bfloat16*)net->wtc, bias, y, Ci, Co, H, W, d, relu, net->tc_err);
            IIM_LAUNCHED();
            return IIM_OK;
        };
        if (Ci <= 16 && Co <= 16) return go(k_pack_w_tc<2, 16>, k_conv_tc<2, 16>, 2, 16);
        if (Ci <= 16) return go(k_pack_w_tc<2, 32>, k_conv_tc<2, 32>, 2, 32);
        if (Co <= 16) return go(k_pack_w_tc<4, 16>, k_conv_tc<4, 16>, 4, 16);
        return go(k_pack_w_tc<4, 32>, k_conv_tc<4, 32>, 4, 32);
    }
    if (Co > 1) {
        const int ncot = (Co + 31) / 32;
        const size_t sm = conv_smem(d, 32);
        IIM_CHECK(allow_smem(k_conv<32>, sm));
        launch("net_conv", 4.0 * (double)B * H * W * (Ci + Co), 18.0 * (double)B * H * W * Ci * Co, k_conv<32>,
               dim3((W + TX - 1) / TX, (H + TY - 1) / TY, B * ncot), blk, sm, s, x, gate, w, bias, y, Ci, Co, H, W, d, relu);
    } else {
        const size_t sm = conv_smem(d, 1);
        launch("net_conv", 4.0 * (double)B * H * W * (Ci + Co), 18.0 * (double)B * H * W * Ci * Co, k_conv<1>,
               dim3((W + TX - 1) / TX, (H + TY - 1) / TY, B), blk, sm, s, x, gate, w, bias, y, Ci, Co, H, W, d, relu);
    }
    IIM_LAUNCHED();
    return IIM_OK;
}

static iim_status ensure_cap(iim_net_s* net, long long need) {
    if (need <= net->cap) return IIM_OK;
    cudaFree(net->act);
    cudaFree(net->g0);
    net->act = net->g0 = nullptr;
    IIM_TRY(cudaMalloc(&net->act, sizeof(float) * (size_t)need * net->nl));
    IIM_TRY(cudaMalloc(&net->g0, sizeof(float) * (size_t)need * 2));
    net->cap = need;
    return IIM_OK;
}

static iim_status forward(iim_net_s* net, int B, int H, int W, const float* x, cudaStream_t s) {
    const long long cap = (long long)B * H * W * std::max(net->hidden, 1);
    IIM_CHECK(ensure_cap(net, cap));
    const float* in = x;
    for (int l = 0; l < net->nl; ++l) {
        float* out = net->act + (size_t)l * net->cap;
        IIM_CHECK(conv(net, in, nullptr, net->wb + net->woff[l], net->p + net->boff[l], out, B, net->ci[l], net->co[l], H, W,
                       net->dil[l], l < net->nl - 1, s));
        in = out;
    }
    return IIM_OK;
}

// gradients of sum(dy * pred) w.r.t. the parameters (into net->gr); dy is overwritten
static iim_status backward(iim_net_s* net, int B, int H, int W, const float* x, float* dy, cudaStream_t s) {
    IIM_TRY(cudaMemsetAsync(net->gr, 0, sizeof(float) * (size_t)net->np, s));
    float* g = dy;
    for (int l = net->nl - 1; l >= 0; --l) {
        const float* xin = l == 0 ? x : net->act + (size_t)(l - 1) * net->cap;
        const float* gate = l == net->nl - 1 ? nullptr : net->act + (size_t)l * net->cap;
        const int d = net->dil[l];
        const size_t sm = sizeof(float) * ((size_t)WG_MAXC * WG_S * WG_S + (size_t)(WG_S + 2 * d) * (WG_S + 2 * d));
        IIM_CHECK(allow_smem(k_conv_wgrad, sm));
        launch("net_wgrad", 4.0 * (double)B * H * W * (net->ci[l] + net->co[l]), 2.0 * B * H * W * 9.0 * net->ci[l] * net->co[l],
               k_conv_wgrad, dim3((W + WG_R - 1) / WG_R, (H + WG_R - 1) / WG_R, B), 288, sm, s, xin, (const float*)g, gate,
               net->gr + net->woff[l], net->gr + net->boff[l], net->ci[l], net->co[l], H, W, d);
        IIM_LAUNCHED();
        if (l > 0) {
            const int n = net->ci[l] * net->co[l] * 9;
            launch("net_flip", 0.0, 0.0, k_flip, (n + 255) / 256, 256, 0, s, net->ci[l], net->co[l],
                   (const __nv_bfloat16*)(net->wb + net->woff[l]), net->wt);
            float* gprev = net->g0 + (size_t)((net->nl - 1 - l) & 1) * net->cap;
            IIM_CHECK(conv(net, g, gate, net->wt, nullptr, gprev, B, net->co[l], net->ci[l], H, W, d, 0, s));
            g = gprev;
        }
    }
    return IIM_OK;
}

static iim_status sync_bf16(iim_net_s* net, cudaStream_t s) {
    launch("net_bf16", 0.0, 0.0, k_to_bf16, (unsigned)((net->np + 255) / 256), 256, 0, s, (long)net->np,
           (const float*)net->p, net->wb);
    IIM_LAUNCHED();
    return IIM_OK;
}

}  // namespace iim

using namespace iim;

extern "C" iim_status iim_net_create(int in_channels, int hidden, int n_layers, const int* dilations,
                                     unsigned long long seed, iim_net* out) {
    if (!out) return IIM_ERR_INVALID_ARG;
    *out = nullptr;
    if (in_channels < 1 || in_channels > 32 || hidden < 1 || hidden > 32 || n_layers < 1 || n_layers > 16 || !dilations)
        return IIM_ERR_INVALID_ARG;
    for (int l = 0; l < n_layers; ++l)
        if (dilations[l] < 1 || dilations[l] > 32) return IIM_ERR_INVALID_ARG;
    iim_net_s* net = new iim_net_s();
    cudaGetDevice(&net->device);
    net->cin = in_channels;
    net->hidden = hidden;
    net->nl = n_layers;
    long long off = 0;
    for (int l = 0; l < n_layers; ++l) {
        net->dil.push_back(dilations[l]);
        net->ci.push_back(l == 0 ? in_channels : hidden);
        net->co.push_back(l == n_layers - 1 ? 1 : hidden);
        net->woff.push_back(off);
        off += (long long)net->ci[l] * net->co[l] * 9;
        net->boff.push_back(off);
        off += net->co[l];
    }
    net->np = off;
    std::vector<float> h(off, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < n_layers; ++l) {
        // He-uniform initialisation, zero biases
        const float a = std::sqrt(6.f / (9.f * net->ci[l]));
        std::uniform_real_distribution<float> U(-a, a);
        for (long long k = 0; k < (long long)net->ci[l] * net->co[l] * 9; ++k) h[net->woff[l] + k] = U(rng);
    }
    auto fail = [&](cudaError_t e) {
        record_cuda_error(e, "iim_net_create", __FILE__, __LINE__);
        cudaFree(net->p); cudaFree(net->gr); cudaFree(net->m); cudaFree(net->v); cudaFree(net->wb); cudaFree(net->wt);
        cudaFree(net->red); cudaFree(net->wtc); cudaFree(net->tc_err);
        delete net;
        return IIM_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&net->p, sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&net->gr, sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&net->m, sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&net->v, sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&net->wb, sizeof(__nv_bfloat16) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&net->wt, sizeof(__nv_bfloat16) * 32 * 32 * 9)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&net->red, sizeof(float) * 4096)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&net->wtc, sizeof(__nv_bfloat16) * 9 * 4 * TC_C * 8)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&net->tc_err, sizeof(int))) != cudaSuccess) return fail(e);
    cudaMemset(net->tc_err, 0, sizeof(int));
    net->tc = 2;
    if ((e = cudaMemcpy(net->p, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    cudaMemset(net->m, 0, sizeof(float) * off);
    cudaMemset(net->v, 0, sizeof(float) * off);
    if (cudaMallocHost(&net->h_red, 4 * sizeof(float)) != cudaSuccess) return fail(cudaErrorMemoryAllocation);
    if (sync_bf16(net, nullptr) != IIM_OK) return fail(cudaGetLastError());
    cudaDeviceSynchronize();
    *out = net;
    return IIM_OK;
}

extern "C" long long iim_net_num_params(iim_net net) { return net ? net->np : 0; }

extern "C" iim_status iim_net_get_params(iim_net net, float* host, long long n) {
    if (!net || !host || n != net->np) return IIM_ERR_INVALID_ARG;
    IIM_TRY(cudaMemcpy(host, net->p, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return IIM_OK;
}

extern "C" iim_status iim_net_set_params(iim_net net, const float* host, long long n) {
    if (!net || !host || n != net->np) return IIM_ERR_INVALID_ARG;
    IIM_TRY(cudaMemcpy(net->p, host, sizeof(float) * n, cudaMemcpyHostToDevice));
    IIM_TRY(cudaMemset(net->m, 0, sizeof(float) * n));
    IIM_TRY(cudaMemset(net->v, 0, sizeof(float) * n));
    net->t = 0;
    IIM_CHECK(sync_bf16(net, nullptr));
    IIM_TRY(cudaDeviceSynchronize());
    return IIM_OK;
}

extern "C" iim_status iim_net_forward(iim_net net, int batch, int height, int width, const float* x, float* y,
                                      iim_stream stream) {
    if (!net || !x || !y || batch < 1 || height < 1 || width < 1) return IIM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    IIM_CHECK(forward(net, batch, height, width, x, s));
    IIM_TRY(cudaMemcpyAsync(y, net->act + (size_t)(net->nl - 1) * net->cap, sizeof(float) * (size_t)batch * height * width,
                            cudaMemcpyDeviceToDevice, s));
    return IIM_OK;
}

extern "C" iim_status iim_net_backward(iim_net net, int batch, int height, int width, const float* x, const float* dy,
                                       float* grad_host, iim_stream stream) {
    if (!net || !x || !dy || batch < 1 || height < 1 || width < 1) return IIM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    IIM_CHECK(forward(net, batch, height, width, x, s));
    const size_t n = (size_t)batch * height * width;
    float* g = net->g0 + net->cap;   // scratch copy of dy (the backward pass overwrites its input)
    IIM_TRY(cudaMemcpyAsync(g, dy, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    IIM_CHECK(backward(net, batch, height, width, x, g, s));
    if (grad_host) {
        IIM_TRY(cudaMemcpyAsync(grad_host, net->gr, sizeof(float) * (size_t)net->np, cudaMemcpyDeviceToHost, s));
        IIM_TRY(cudaStreamSynchronize(s));
    }
    return IIM_OK;
}

extern "C" iim_status iim_net_train_step(iim_net net, int batch, int height, int width, const float* x,
                                         const float* target, const float* mask, float lr, float* loss,
                                         iim_stream stream) {
    if (!net || !x || !target || batch < 1 || height < 1 || width < 1 || !(lr >= 0.f)) return IIM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    IIM_CHECK(forward(net, batch, height, width, x, s));
    const long n = (long)batch * height * width;
    const float* pred = net->act + (size_t)(net->nl - 1) * net->cap;
    float* diff = net->g0 + net->cap;
    const int nb = 256;
    launch("net_mse", 12.0 * n, 0.0, k_mse_partial, nb, 256, 0, s, n, pred, target, mask, diff, net->red);
    launch("net_mse_finish", 0.0, 0.0, k_mse_finish, 1, 32, 0, s, nb, net->red, net->red + 1024);
    launch("net_scale", 0.0, 0.0, k_scale_vec, (unsigned)((n + 255) / 256), 256, 0, s, n, diff, (const float*)(net->red + 1025));
    IIM_LAUNCHED();
    IIM_CHECK(backward(net, batch, height, width, x, diff, s));
    net->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)net->t), c2 = 1.f - std::pow(b2, (float)net->t);
    launch("net_adam", 0.0, 0.0, k_adam, (unsigned)((net->np + 255) / 256), 256, 0, s, (long)net->np, net->p,
           (const float*)net->gr, net->m, net->v, lr, b1, b2, 1e-8f, c1, c2);
    IIM_LAUNCHED();
    IIM_CHECK(sync_bf16(net, s));
    if (loss) {
        IIM_TRY(cudaMemcpyAsync(net->h_red, net->red + 1024, sizeof(float), cudaMemcpyDeviceToHost, s));
        IIM_TRY(cudaStreamSynchronize(s));
        *loss = net->h_red[0];
    }
    return IIM_OK;
}

extern "C" iim_status iim_net_prepare_input(int nx, int ny, const double* omega, const double* phi_nodes,
                                            const double* u_box, float s_omega, float s_phi, float s_box, float* x,
                                            iim_stream stream) {
    if (nx < 3 || ny < 3 || !omega || !phi_nodes || !u_box || !x) return IIM_ERR_INVALID_ARG;
    const long n = (long)(nx - 1) * (ny - 1);
    launch("net_input", 0.0, 0.0, k_net_input, (unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream, nx - 1, ny - 1,
           omega, phi_nodes, u_box, s_omega, s_phi, s_box, x);
    IIM_LAUNCHED();
    return IIM_OK;
}

extern "C" iim_status iim_net_compose_guess(long long n, const double* u_box, const float* y, float s_out,
                                            double* psi_guess, iim_stream stream) {
    if (n < 0 || !u_box || !y || !psi_guess || !(s_out != 0.f)) return IIM_ERR_INVALID_ARG;
    launch("net_guess", 0.0, 0.0, k_net_guess, (unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream, (long)n, u_box, y,
           1.f / s_out, psi_guess);
    IIM_LAUNCHED();
    return IIM_OK;
}

extern "C" iim_status iim_net_set_tensor_cores(iim_net net, int on) {
    if (!net || on < 0 || on > 2) return IIM_ERR_INVALID_ARG;
    net->tc = on;
    return IIM_OK;
}

extern "C" iim_status iim_net_tensor_core_status(iim_net net, int* on, int* timed_out) {
    if (!net || !on || !timed_out) return IIM_ERR_INVALID_ARG;
    *on = net->tc;
    IIM_TRY(cudaDeviceSynchronize());
    IIM_TRY(cudaMemcpy(timed_out, net->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    return IIM_OK;
}

extern "C" void iim_net_destroy(iim_net net) {
    if (!net) return;
    cudaFree(net->p); cudaFree(net->gr); cudaFree(net->m); cudaFree(net->v); cudaFree(net->wb); cudaFree(net->wt);
    cudaFree(net->act); cudaFree(net->g0); cudaFree(net->red); cudaFree(net->wtc); cudaFree(net->tc_err);
    if (net->h_red) cudaFreeHost(net->h_red);
    delete net;
}
