// Kernels of the learned preconditioning stage: 3x3 convolutions with BF16
// weights and activations and FP32 accumulation, their gradients, Adam, and
// the glue that turns a block of complex residuals into network input and
// the network output into a correction of the cycle's result.
//
// The stage is not in the paper; it rides on the flexibility of FGMRES
// (Sec. 4: the preconditioner may change from one step to the next).
//
// Layouts: activations NHWC bf16, x[b][i][j][c] with i the depth row and j
// the lateral column of the node grid (pixel i*W + j is node i*W + j);
// weights [co][tap][ci] bf16 with tap = 3*dy + dx reading pixel
// (i + dy - 1, j + dx - 1); zero outside the image.
#include <cuda_bf16.h>

#include "kernels.h"

namespace helm {

namespace {

constexpr int CTH = 8, CTW = 16;   // output pixels per CTA: 8 rows x 16 columns (one row per warp)

__device__ __forceinline__ void ldsm_x4(unsigned int* r, const void* p) {
    unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(unsigned int* r, const void* p) {
    unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
__device__ __forceinline__ void mma_bf16(float* d, const unsigned int* a, const unsigned int* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// y = epilogue(conv(x; w) + bias): implicit GEMM, M = pixels, N = COUT,
// K = 9 * CIN, on mma.sync m16n8k16 bf16 tiles.  The CTA stages the input
// tile with its one-pixel halo and all weights in shared memory (rows padded
// by 8 bf16 so that ldmatrix is free of bank conflicts); warp w computes
// output row w of the tile: 16 pixels x COUT channels.
// Epilogue: + bias (may be null), ReLU (relu != 0), times (mask > 0) when a
// mask is given (the ReLU derivative of the backward pass), stored as bf16
// or float.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_conv3x3(const __nv_bfloat16* __restrict__ x, int H, int W,
                                                  const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ bias, int relu,
                                                  const __nv_bfloat16* __restrict__ mask,
                                                  void* __restrict__ y, int y_float) {
    constexpr int CS = CIN + 8;            // padded pixel stride (bf16)
    constexpr int WS = 9 * CIN + 8;        // padded weight row stride (bf16)
    constexpr int TPW = CTW + 2;           // tile width with halo
    extern __shared__ __align__(16) unsigned char smraw[];
    __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(smraw);
    __nv_bfloat16* ws = xs + (CTH + 2) * TPW * CS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * CTW, y0 = blockIdx.y * CTH, b = blockIdx.z;
    const __nv_bfloat16* xb = x + (size_t)b * H * W * CIN;

    // input tile with halo, 16-byte chunks of 8 channels
    constexpr int CPP = CIN / 8;
    for (int idx = tid; idx < (CTH + 2) * TPW * CPP; idx += 256) {
        int pix = idx / CPP, ch = (idx - pix * CPP) * 8;
        int ty = pix / TPW, tx = pix - ty * TPW;
        int gy = y0 + ty - 1, gx = x0 + tx - 1;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
            v = *reinterpret_cast<const uint4*>(xb + ((size_t)gy * W + gx) * CIN + ch);
        *reinterpret_cast<uint4*>(xs + pix * CS + ch) = v;
    }
    for (int idx = tid; idx < COUT * 9 * CIN / 8; idx += 256) {
        int co = idx / (9 * CIN / 8), k = (idx - co * (9 * CIN / 8)) * 8;
        *reinterpret_cast<uint4*>(ws + co * WS + k) =
            *reinterpret_cast<const uint4*>(w + (size_t)co * 9 * CIN + k);
    }
    __syncthreads();

    float acc[COUT / 8][4];
#pragma unroll
    for (int nt = 0; nt < COUT / 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;

    const int q = lane >> 3, i8 = lane & 7;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap - 3 * (tap / 3);
#pragma unroll
        for (int kh = 0; kh < CIN / 16; ++kh) {
            unsigned int a[4];
            const int p = i8 + 8 * (q & 1);
            ldsm_x4(a, xs + ((warp + dy) * TPW + p + dx) * CS + kh * 16 + 8 * (q >> 1));
            const int kb = tap * CIN + kh * 16;
#pragma unroll
            for (int nt = 0; nt < COUT / 8; nt += 2) {
                if (nt + 1 < COUT / 8) {
                    unsigned int bb[4];
                    ldsm_x4(bb, ws + ((nt + (q >> 1)) * 8 + i8) * WS + kb + 8 * (q & 1));
                    mma_bf16(acc[nt], a, bb);
                    mma_bf16(acc[nt + 1], a, bb + 2);
                } else {
                    unsigned int bb[2];
                    ldsm_x2(bb, ws + (nt * 8 + i8) * WS + kb + 8 * ((lane >> 3) & 1));
                    mma_bf16(acc[nt], a, bb);
                }
            }
        }
    }
    // epilogue
    const int g = lane >> 2, t = lane & 3;
    const int gy = y0 + warp;
    if (gy >= H) return;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int gx = x0 + g + 8 * half;
        if (gx >= W) continue;
        const size_t pix = ((size_t)b * H + gy) * W + gx;
#pragma unroll
        for (int nt = 0; nt < COUT / 8; ++nt) {
            const int co = nt * 8 + 2 * t;
            float v0 = acc[nt][2 * half], v1 = acc[nt][2 * half + 1];
            if (bias) { v0 += bias[co]; v1 += bias[co + 1]; }
            if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
            if (mask) {
                __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(mask + pix * COUT + co);
                if (!(__bfloat162float(m.x) > 0.f)) v0 = 0.f;
                if (!(__bfloat162float(m.y) > 0.f)) v1 = 0.f;
            }
            if (y_float) {
                *reinterpret_cast<float2*>(reinterpret_cast<float*>(y) + pix * COUT + co) = make_float2(v0, v1);
            } else {
                *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(y) + pix * COUT + co) =
                    __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}

// dW[co][tap][ci] += sum_pixels gy[p][co] x[p + tap][ci], db[co] += sum gy[p][co]
// on the FP32 pipes; CTAs stride over 8 x 16 pixel tiles and add their sums
// with one atomic per entry at the end.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_conv_wgrad(const __nv_bfloat16* __restrict__ x,
                                                     const __nv_bfloat16* __restrict__ gy, int B,
                                                     int H, int W, float* __restrict__ dw,
                                                     float* __restrict__ db) {
    constexpr int TPW = CTW + 2;
    constexpr int E = COUT * 9 * CIN + COUT;
    constexpr int EPT = (E + 255) / 256;
    __shared__ float xs[(CTH + 2) * TPW * CIN];
    __shared__ float gs[CTH * CTW * COUT];
    const int tid = threadIdx.x;
    float acc[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) acc[k] = 0.f;
    const int tx_n = (W + CTW - 1) / CTW, ty_n = (H + CTH - 1) / CTH;
    const long long ntiles = (long long)B * tx_n * ty_n;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int b = (int)(tile / (tx_n * ty_n));
        int rem = (int)(tile - (long long)b * tx_n * ty_n);
        int y0 = (rem / tx_n) * CTH, x0 = (rem % tx_n) * CTW;
        __syncthreads();
        for (int idx = tid; idx < (CTH + 2) * TPW * CIN; idx += 256) {
            int pix = idx / CIN, c = idx - pix * CIN;
            int ty = pix / TPW, tx = pix - ty * TPW;
            int yy = y0 + ty - 1, xx = x0 + tx - 1;
            xs[idx] = (yy >= 0 && yy < H && xx >= 0 && xx < W)
                          ? __bfloat162float(x[(((size_t)b * H + yy) * W + xx) * CIN + c]) : 0.f;
        }
        for (int idx = tid; idx < CTH * CTW * COUT; idx += 256) {
            int pix = idx / COUT, c = idx - pix * COUT;
            int ty = pix / CTW, tx = pix - ty * CTW;
            int yy = y0 + ty, xx = x0 + tx;
            gs[idx] = (yy < H && xx < W)
                          ? __bfloat162float(gy[(((size_t)b * H + yy) * W + xx) * COUT + c]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int e = tid + k * 256;
            if (e >= E) continue;
            float a = acc[k];
            if (e >= COUT * 9 * CIN) {
                const int co = e - COUT * 9 * CIN;
                for (int p = 0; p < CTH * CTW; ++p) a += gs[p * COUT + co];
            } else {
                const int co = e / (9 * CIN), r = e - co * 9 * CIN, tap = r / CIN, ci = r - tap * CIN;
                const int dy = tap / 3, dx = tap - 3 * (tap / 3);
                for (int p = 0; p < CTH * CTW; ++p) {
                    int ty = p / CTW, tx = p - ty * CTW;
                    a = fmaf(gs[p * COUT + co], xs[((ty + dy) * TPW + tx + dx) * CIN + ci], a);
                }
            }
            acc[k] = a;
        }
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int e = tid + k * 256;
        if (e >= E) continue;
        if (e >= COUT * 9 * CIN) atomicAdd(db + (e - COUT * 9 * CIN), acc[k]);
        else atomicAdd(dw + e, acc[k]);
    }
}

// wf[ci][tap][co] = w[co][8 - tap][ci]: the weights of the data-gradient
// convolution (transposed channels, flipped taps).
__global__ void k_flip_weights(const __nv_bfloat16* __restrict__ w, int cin, int cout,
                               __nv_bfloat16* __restrict__ wf, int cin_pad_out) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int n = cin_pad_out * 9 * cout;
    if (e >= n) return;
    int ci = e / (9 * cout), r = e - ci * 9 * cout, tap = r / cout, co = r - tap * cout;
    wf[e] = ci < cin ? w[((size_t)co * 9 + (8 - tap)) * cin + ci] : __float2bfloat16(0.f);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ pb, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float gg = g[e];
    float mm = b1 * m[e] + (1.f - b1) * gg;
    float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    float pp = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[e] = pp;
    if (pb) pb[e] = __float2bfloat16(pp);
}

// Network input from a complex64 block r[node][j] (node = i*W + jx):
// channels (Re r / rho_j, Im r / rho_j, kappa, 0, ...) with rho_j the RMS of
// column j (rho_j = 0 gives zeros).  16 channels, bf16, image j.
__global__ void k_pack_input(const c64* __restrict__ r, int N, int s, const float* __restrict__ rho,
                             const float* __restrict__ kappa, __nv_bfloat16* __restrict__ out) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)N * s) return;
    int node = (int)(e / s), j = (int)(e - (long long)node * s);
    c64 v = r[e];
    float inv = rho[j] > 0.f ? 1.f / rho[j] : 0.f;
    __nv_bfloat16* o = out + ((size_t)j * N + node) * 16;
    __nv_bfloat162 z2 = __floats2bfloat162_rn(0.f, 0.f);
    reinterpret_cast<__nv_bfloat162*>(o)[0] = __floats2bfloat162_rn(v.re * inv, v.im * inv);
    reinterpret_cast<__nv_bfloat162*>(o)[1] = __floats2bfloat162_rn(kappa[node], 0.f);
#pragma unroll
    for (int c = 2; c < 8; ++c) reinterpret_cast<__nv_bfloat162*>(o)[c] = z2;
}

// z[node][j] += scale * rho_j * (out[j][node][0] + i out[j][node][1]); non-finite
// network outputs leave z unchanged (the cycle's result is the fallback).
__global__ void k_unpack_add(const float* __restrict__ out, int N, int s, const float* __restrict__ rho,
                             float scale, c64* __restrict__ z) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)N * s) return;
    int node = (int)(e / s), j = (int)(e - (long long)node * s);
    const float* o = out + ((size_t)j * N + node) * 16;
    float a = o[0], b = o[1];
    if (!isfinite(a) || !isfinite(b)) return;
    float f = scale * rho[j];
    c64 v = z[e];
    z[e] = mk(v.re + f * a, v.im + f * b);
}

// r = f - A z in complex64 (residual of the cycle's result w.r.t. the
// unshifted operator)
__global__ void k_learned_residual(FineOp<float> op, const c128* __restrict__ f,
                                   const c64* __restrict__ z, c64* __restrict__ r, int s) {
    long long total = op.g.N * s;
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    long long node = e / s;
    int j = (int)(e - node * s);
    int a, b, c;
    op.g.coords(node, a, b, c);
    r[e] = cvt<float>(f[e]) - op.apply(z, node, a, b, c, s, j);
}

// rho2[j] += sum over nodes |r[node][j]|^2 (s <= 256): thread t takes column
// t % s and every (256/s)-th node of the CTA's stride; one atomic per column
// per CTA.
__global__ void __launch_bounds__(256) k_colsumsq_c64(const c64* __restrict__ r, long long N, int s,
                                                       float* __restrict__ rho2) {
    __shared__ float red[256];
    const int per = 256 / s;
    const int j = threadIdx.x % s, sub = threadIdx.x / s;
    float acc = 0.f;
    if (sub < per)
        for (long long n = (long long)blockIdx.x * per + sub; n < N; n += (long long)gridDim.x * per) {
            c64 v = r[n * s + j];
            acc += v.re * v.re + v.im * v.im;
        }
    red[threadIdx.x] = sub < per ? acc : 0.f;
    __syncthreads();
    if (sub == 0) {
        float t = 0.f;
        for (int k = 0; k < per; ++k) t += red[k * s + j];
        atomicAdd(rho2 + j, t);
    }
}

// z[node][j] = z2 when column j's residual did not grow (|r2|^2 < |r1|^2 = N rho_j^2), else z1
__global__ void k_select_better(const c64* __restrict__ z2, c64* __restrict__ z1, long long N, int s,
                                const float* __restrict__ rho1, const float* __restrict__ r2sq) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= N * s) return;
    int j = (int)(e % s);
    float old2 = rho1[j] * rho1[j] * (float)N;
    if (r2sq[j] < old2) z1[e] = z2[e];
}

__global__ void k_rms(const float* __restrict__ rho2, int s, int N, float* __restrict__ rho) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < s) rho[j] = sqrtf(rho2[j] / (float)N);
}

// t[j][node][0..1] = scale * e[node][j] / rho_j (the training target in the
// units of the network output)
__global__ void k_pack_target(const c64* __restrict__ e, int N, int s, const float* __restrict__ rho,
                              float scale, float* __restrict__ t) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= (long long)N * s) return;
    int node = (int)(k / s), j = (int)(k - (long long)node * s);
    float inv = rho[j] > 0.f ? scale / rho[j] : 0.f;
    c64 v = e[k];
    float* o = t + ((size_t)j * N + node) * 2;
    o[0] = v.re * inv;
    o[1] = v.im * inv;
}

// per sample b: num[b] += sum |pred - t|^2, den[b] += sum |t|^2 over channels 0, 1
__global__ void k_loss_sums(const float* __restrict__ pred, const float* __restrict__ t, int P,
                            float* __restrict__ num, float* __restrict__ den) {
    __shared__ float sn[256], sd[256];
    const int b = blockIdx.y;
    float an = 0.f, ad = 0.f;
    for (int p = blockIdx.x * 256 + threadIdx.x; p < P; p += gridDim.x * 256) {
        const float* q = pred + ((size_t)b * P + p) * 16;
        const float* r = t + ((size_t)b * P + p) * 2;
        float d0 = q[0] - r[0], d1 = q[1] - r[1];
        an += d0 * d0 + d1 * d1;
        ad += r[0] * r[0] + r[1] * r[1];
    }
    sn[threadIdx.x] = an;
    sd[threadIdx.x] = ad;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) { sn[threadIdx.x] += sn[threadIdx.x + w]; sd[threadIdx.x] += sd[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { atomicAdd(num + b, sn[0]); atomicAdd(den + b, sd[0]); }
}

// g = d loss / d pred for loss = mean_b num_b / den_b, in bf16 with 16
// channels (zero beyond channel 1); loss_out = the loss
__global__ void k_loss_grad(const float* __restrict__ pred, const float* __restrict__ t, int B, int P,
                            const float* __restrict__ num, const float* __restrict__ den,
                            __nv_bfloat16* __restrict__ g, float* __restrict__ loss_out) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k == 0 && loss_out) {
        float l = 0.f;
        for (int b = 0; b < B; ++b) l += den[b] > 0.f ? num[b] / den[b] : 0.f;
        *loss_out = l / B;
    }
    if (k >= (long long)B * P) return;
    int b = (int)(k / P);
    float c = den[b] > 0.f ? 2.f / (den[b] * B) : 0.f;
    const float* q = pred + k * 16;
    const float* r = t + k * 2;
    __nv_bfloat16* o = g + k * 16;
    reinterpret_cast<__nv_bfloat162*>(o)[0] = __floats2bfloat162_rn(c * (q[0] - r[0]), c * (q[1] - r[1]));
    __nv_bfloat162 z2 = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll
    for (int i = 1; i < 8; ++i) reinterpret_cast<__nv_bfloat162*>(o)[i] = z2;
}

template <int CIN, int COUT>
size_t conv_smem() {
    return sizeof(__nv_bfloat16) * ((size_t)(CTH + 2) * (CTW + 2) * (CIN + 8) + (size_t)COUT * (9 * CIN + 8));
}

template <int CIN, int COUT>
void conv_launch(const Launch& L, const __nv_bfloat16* x, int B, int H, int W, const __nv_bfloat16* w,
                 const float* bias, int relu, const __nv_bfloat16* mask, void* y, int y_float) {
    dim3 grid((W + CTW - 1) / CTW, (H + CTH - 1) / CTH, B);
    size_t sm = conv_smem<CIN, COUT>();
    cudaFuncSetAttribute(k_conv3x3<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    double px = (double)B * H * W;
    L.pre(KID_CONV, px * (2.0 * CIN + (y_float ? 4.0 : 2.0) * COUT), 2.0 * px * 9 * CIN * COUT);
    k_conv3x3<CIN, COUT><<<grid, 256, sm, L.st>>>(x, H, W, w, bias, relu, mask, y, y_float);
    L.post();
}

template <int CIN, int COUT>
void wgrad_launch(const Launch& L, const __nv_bfloat16* x, const __nv_bfloat16* gy, int B, int H, int W,
                  float* dw, float* db) {
    long long ntiles = (long long)B * ((W + CTW - 1) / CTW) * ((H + CTH - 1) / CTH);
    const long long gcap = 2LL * sm_count();
    int grid = (int)(ntiles < gcap ? ntiles : gcap);
    double px = (double)B * H * W;
    L.pre(KID_CONV_WGRAD, px * 2.0 * (CIN + COUT), 2.0 * px * 9 * CIN * COUT);
    k_conv_wgrad<CIN, COUT><<<grid, 256, 0, L.st>>>(x, gy, B, H, W, dw, db);
    L.post();
}

}  // namespace

bool launch_conv3x3(const Launch& L, const void* x, int B, int H, int W, int cin, const void* w,
                    const float* bias, int cout, int relu, const void* mask, void* y, int y_float) {
    auto X = static_cast<const __nv_bfloat16*>(x);
    auto Wt = static_cast<const __nv_bfloat16*>(w);
    auto M = static_cast<const __nv_bfloat16*>(mask);
    if (cin == 16 && cout == 32) conv_launch<16, 32>(L, X, B, H, W, Wt, bias, relu, M, y, y_float);
    else if (cin == 32 && cout == 32) conv_launch<32, 32>(L, X, B, H, W, Wt, bias, relu, M, y, y_float);
    else if (cin == 32 && cout == 16) conv_launch<32, 16>(L, X, B, H, W, Wt, bias, relu, M, y, y_float);
    else if (cin == 16 && cout == 16) conv_launch<16, 16>(L, X, B, H, W, Wt, bias, relu, M, y, y_float);
    else return false;
    return true;
}

bool launch_conv3x3_wgrad(const Launch& L, const void* x, const void* gy, int B, int H, int W, int cin,
                          int cout, float* dw, float* db) {
    auto X = static_cast<const __nv_bfloat16*>(x);
    auto G = static_cast<const __nv_bfloat16*>(gy);
    if (cin == 16 && cout == 32) wgrad_launch<16, 32>(L, X, G, B, H, W, dw, db);
    else if (cin == 32 && cout == 32) wgrad_launch<32, 32>(L, X, G, B, H, W, dw, db);
    else if (cin == 32 && cout == 16) wgrad_launch<32, 16>(L, X, G, B, H, W, dw, db);
    else return false;
    return true;
}

void launch_flip_weights(const Launch& L, const void* w, int cin, int cout, void* wf, int cin_pad_out) {
    int n = cin_pad_out * 9 * cout;
    L.pre(KID_LAYOUT, 4.0 * n, 0);
    k_flip_weights<<<(n + 255) / 256, 256, 0, L.st>>>(static_cast<const __nv_bfloat16*>(w), cin, cout,
                                                       static_cast<__nv_bfloat16*>(wf), cin_pad_out);
    L.post();
}

void launch_adam(const Launch& L, float* p, const float* g, float* m, float* v, void* pb, int n,
                 float lr, float b1, float b2, float eps, int step) {
    float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    L.pre(KID_LAYOUT, 20.0 * n, 10.0 * n);
    k_adam<<<(n + 255) / 256, 256, 0, L.st>>>(p, g, m, v, static_cast<__nv_bfloat16*>(pb), n, lr, b1,
                                              b2, eps, c1, c2);
    L.post();
}

void launch_pack_input(const Launch& L, const c64* r, int N, int s, const float* rho,
                       const float* kappa, void* out) {
    long long n = (long long)N * s;
    L.pre(KID_LAYOUT, n * (8.0 + 32.0), 0);
    k_pack_input<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(r, N, s, rho, kappa,
                                                                static_cast<__nv_bfloat16*>(out));
    L.post();
}

void launch_unpack_add(const Launch& L, const float* out, int N, int s, const float* rho, float scale,
                       c64* z) {
    long long n = (long long)N * s;
    L.pre(KID_LAYOUT, n * (8.0 + 16.0), 0);
    k_unpack_add<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(out, N, s, rho, scale, z);
    L.post();
}

void launch_select_better(const Launch& L, const c64* z2, c64* z1, long long N, int s,
                          const float* rho1, const float* r2sq) {
    long long n = N * s;
    L.pre(KID_LAYOUT, n * 24.0, 0);
    k_select_better<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(z2, z1, N, s, rho1, r2sq);
    L.post();
}

void launch_learned_residual(const Launch& L, const FineOp<float>& op, const c128* f, const c64* z,
                             c64* r, int s, float* rho2, float* rho) {
    long long n = op.g.N * s;
    cudaMemsetAsync(rho2, 0, sizeof(float) * s, L.st);
    L.pre(KID_APPLY_FINE, n * (16.0 + 16.0), n * 30.0);
    k_learned_residual<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(op, f, z, r, s);
    L.post();
    L.pre(KID_LAYOUT, n * 8.0, n * 4.0);
    k_colsumsq_c64<<<2 * sm_count(), 256, 0, L.st>>>(r, op.g.N, s, rho2);
    L.post();
    L.pre(KID_LAYOUT, 8.0 * s, 0);
    k_rms<<<(s + 255) / 256, 256, 0, L.st>>>(rho2, s, (int)op.g.N, rho);
    L.post();
}

// Residual-loss inputs, sample j in image order: rimg[j][node] = r[node][j] /
// rho_j and cimg[j][node] = h^2 c_A[node] (= kappa (1 - i gamma)), float pairs
__global__ void k_pack_resid(const c64* __restrict__ r, int N, int s, const float* __restrict__ rho,
                             const c128* __restrict__ cA, double h2, float2* __restrict__ rimg,
                             float2* __restrict__ cimg) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= (long long)N * s) return;
    int node = (int)(k / s), j = (int)(k - (long long)node * s);
    const float inv = rho[j] > 0.f ? 1.f / rho[j] : 0.f;
    const c64 v = r[k];
    const c128 c = cA[node];
    rimg[(size_t)j * N + node] = make_float2(v.re * inv, v.im * inv);
    cimg[(size_t)j * N + node] = make_float2((float)(c.re * h2), (float)(c.im * h2));
}

// K e at pixel (i, x) of sample b for K = h^2 A (or its adjoint, conj_c):
// 4 e - (the four neighbours, zero outside) - c e; e given as float pairs
// with a stride of `es` floats per pixel
__device__ __forceinline__ float2 h2A_pixel(const float* __restrict__ e, int es, const float2* __restrict__ coef,
                                            size_t base, int H, int W, int i, int x, bool conj_c) {
    const size_t p = base + (size_t)i * W + x;
    float re = 4.f * e[p * es], im = 4.f * e[p * es + 1];
    if (i > 0) { re -= e[(p - W) * es]; im -= e[(p - W) * es + 1]; }
    if (i + 1 < H) { re -= e[(p + W) * es]; im -= e[(p + W) * es + 1]; }
    if (x > 0) { re -= e[(p - 1) * es]; im -= e[(p - 1) * es + 1]; }
    if (x + 1 < W) { re -= e[(p + 1) * es]; im -= e[(p + 1) * es + 1]; }
    const float2 c = coef[p];
    const float ci = conj_c ? -c.y : c.y;
    const float er = e[p * es], ei = e[p * es + 1];
    re -= c.x * er - ci * ei;
    im -= c.x * ei + ci * er;
    return make_float2(re, im);
}

// q = rt - K pred (pred channels 0, 1 of 16), per sample num[b] += |q|^2,
// den[b] += |rt|^2
__global__ void k_rloss_q(const float* __restrict__ pred, const float2* __restrict__ rt,
                          const float2* __restrict__ coef, int H, int W, float2* __restrict__ q,
                          float* __restrict__ num, float* __restrict__ den) {
    __shared__ float sn[256], sd[256];
    const int b = blockIdx.y;
    const long long P = (long long)H * W;
    const size_t base = (size_t)b * P;
    float an = 0.f, ad = 0.f;
    for (long long p = blockIdx.x * 256LL + threadIdx.x; p < P; p += (long long)gridDim.x * 256) {
        const int i = (int)(p / W), x = (int)(p - (long long)i * W);
        const float2 ke = h2A_pixel(pred, 16, coef, base, H, W, i, x, false);
        const float2 r = rt[base + p];
        const float2 v = make_float2(r.x - ke.x, r.y - ke.y);
        q[base + p] = v;
        an += v.x * v.x + v.y * v.y;
        ad += r.x * r.x + r.y * r.y;
    }
    sn[threadIdx.x] = an;
    sd[threadIdx.x] = ad;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) { sn[threadIdx.x] += sn[threadIdx.x + w]; sd[threadIdx.x] += sd[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { atomicAdd(num + b, sn[0]); atomicAdd(den + b, sd[0]); }
}

// g = d loss / d pred = -(2 / (B den_b)) K^H q (channels 0, 1; zero beyond),
// bf16 [B][H][W][16]; loss_out = mean_b num_b / den_b
__global__ void k_rloss_grad(const float2* __restrict__ q, const float2* __restrict__ coef, int B, int H, int W,
                             const float* __restrict__ num, const float* __restrict__ den,
                             __nv_bfloat16* __restrict__ g, float* __restrict__ loss_out) {
    const long long P = (long long)H * W;
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k == 0 && loss_out) {
        float l = 0.f;
        for (int b = 0; b < B; ++b) l += den[b] > 0.f ? num[b] / den[b] : 0.f;
        *loss_out = l / B;
    }
    if (k >= (long long)B * P) return;
    const int b = (int)(k / P);
    const long long p = k - (long long)b * P;
    const int i = (int)(p / W), x = (int)(p - (long long)i * W);
    const float2 kh = h2A_pixel(reinterpret_cast<const float*>(q), 2, coef, (size_t)b * P, H, W, i, x, true);
    const float c = den[b] > 0.f ? -2.f / (den[b] * B) : 0.f;
    __nv_bfloat16* o = g + k * 16;
    reinterpret_cast<__nv_bfloat162*>(o)[0] = __floats2bfloat162_rn(c * kh.x, c * kh.y);
    __nv_bfloat162 z2 = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll
    for (int t = 1; t < 8; ++t) reinterpret_cast<__nv_bfloat162*>(o)[t] = z2;
}

// v[node][j] = rimg[j][node] as complex128 (image order -> internal block)
__global__ void k_image_to_block(const float2* __restrict__ rimg, long long N, int s, c128* __restrict__ v) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= N * s) return;
    long long node = k / s;
    int j = (int)(k - node * s);
    const float2 r = rimg[(size_t)j * N + node];
    v[k] = mk((double)r.x, (double)r.y);
}

__global__ void k_kappa(const c128* __restrict__ cA, long long N, double h2, float* __restrict__ kappa) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < N) kappa[i] = (float)(cA[i].re * h2);
}

void launch_kappa(const Launch& L, const c128* cA, long long N, double h2, float* kappa) {
    L.pre(KID_SETUP, 0, 0);
    k_kappa<<<(unsigned)((N + 255) / 256), 256, 0, L.st>>>(cA, N, h2, kappa);
    L.post();
}

void launch_pack_resid(const Launch& L, const c64* r, int N, int s, const float* rho, const c128* cA,
                       double h2, float* rimg, float* cimg) {
    long long n = (long long)N * s;
    L.pre(KID_LAYOUT, n * (8.0 + 16.0 + 16.0), 0);
    k_pack_resid<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(r, N, s, rho, cA, h2,
                                                                 reinterpret_cast<float2*>(rimg),
                                                                 reinterpret_cast<float2*>(cimg));
    L.post();
}

void launch_residual_loss(const Launch& L, const float* pred, const float* rt, const float* coef, int B, int H,
                          int W, float* q, float* sums, void* grad, float* loss_out) {
    const long long P = (long long)H * W;
    cudaMemsetAsync(sums, 0, sizeof(float) * 2 * B, L.st);
    dim3 grid((unsigned)((P + 255) / 256 < 64 ? (P + 255) / 256 : 64), B);
    L.pre(KID_LAYOUT, (double)B * P * (64.0 + 8.0 + 8.0 + 8.0), (double)B * P * 20.0);
    k_rloss_q<<<grid, 256, 0, L.st>>>(pred, reinterpret_cast<const float2*>(rt),
                                      reinterpret_cast<const float2*>(coef), H, W, reinterpret_cast<float2*>(q),
                                      sums, sums + B);
    L.post();
    const long long n = (long long)B * P;
    L.pre(KID_LAYOUT, n * (8.0 + 8.0 + 32.0), n * 20.0);
    k_rloss_grad<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(
        reinterpret_cast<const float2*>(q), reinterpret_cast<const float2*>(coef), B, H, W, sums, sums + B,
        static_cast<__nv_bfloat16*>(grad), loss_out);
    L.post();
}

void launch_image_to_block(const Launch& L, const float* rimg, long long N, int s, c128* v) {
    long long n = N * s;
    L.pre(KID_LAYOUT, n * 24.0, 0);
    k_image_to_block<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(reinterpret_cast<const float2*>(rimg), N, s,
                                                                     v);
    L.post();
}

void launch_pack_target(const Launch& L, const c64* e, int N, int s, const float* rho, float scale,
                        float* t) {
    long long n = (long long)N * s;
    L.pre(KID_LAYOUT, n * 16.0, 0);
    k_pack_target<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(e, N, s, rho, scale, t);
    L.post();
}

void launch_loss(const Launch& L, const float* pred, const float* t, int B, int P, float* sums,
                 void* grad, float* loss_out) {
    cudaMemsetAsync(sums, 0, sizeof(float) * 2 * B, L.st);
    dim3 grid((P + 255) / 256 < 64 ? (P + 255) / 256 : 64, B);
    L.pre(KID_LAYOUT, (double)B * P * 72.0, 0);
    k_loss_sums<<<grid, 256, 0, L.st>>>(pred, t, P, sums, sums + B);
    L.post();
    long long n = (long long)B * P;
    L.pre(KID_LAYOUT, n * 104.0, 0);
    k_loss_grad<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(pred, t, B, P, sums, sums + B,
                                                              static_cast<__nv_bfloat16*>(grad), loss_out);
    L.post();
}

}  // namespace helm
