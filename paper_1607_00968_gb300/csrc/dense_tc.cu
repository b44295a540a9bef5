// Coarsest-grid solve of the complex64 cycle on the tensor cores.
//
// The coarsest operator's inverse is applied to the whole block of
// right-hand sides (Sec. 4: LU applied to a block of right-hand sides on the
// coarsest grid) as one real GEMM:
//     C' (nc x 2s) = A' (nc x 2nc) B' (2nc x 2s),
// A' = the complex inverse viewed as interleaved (re, im) floats,
// B' rows 2k = [Re f_k, Im f_k], 2k+1 = [-Im f_k, Re f_k], so that
// C' = [Re u | Im u].  The default product stores A' in FP16 (11
// significant bits, the tf32 class, half the bytes of the matrix that is
// streamed from HBM every cycle), scaled at set-up by a power of two so
// that max |A'| = 2^13, and B' in FP16 with a power-of-two scale per
// right-hand side; it runs on mma.sync m16n8k16 f16 tiles with FP32
// accumulation, fed by a 4-stage cp.async pipeline, and the reduction of the
// K slices removes the scales exactly.  The FP32-class option keeps A' in
// FP32 and runs three mma.sync m16n8k8 tf32 products on hi/lo splits.  The K
// range is split over CTAs so that the ~nc/128 row tiles fill the SMs.
#include <cuda_fp16.h>

#include <mutex>

#include "kernels.h"
#include "tc05.cuh"

namespace helm {

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 32, TST = 3;
constexpr int APAD = 4, BPAD = 8;
constexpr int ALD = TBK + APAD, BLD = TBN + BPAD;

__device__ __forceinline__ float tf32_rna(float x) {
    unsigned int r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
    unsigned int s = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

__device__ __forceinline__ void mma_tf32(float* d, const unsigned int* a, const unsigned int* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// P[ks][row][col] = sum over this CTA's K slice of A'[row][k] B'[k][col].
// 8 warps: 2 along M (64 rows each) x 4 along N (32 columns each).
template <bool SPLIT3>
__global__ void __launch_bounds__(256) k_dense_tf32(const float* __restrict__ A, int lda, int M,
                                                     const float* __restrict__ B, int ldb,
                                                     int kchunk, int Kp, float* __restrict__ P) {
    extern __shared__ float sm[];
    float* As = sm;
    float* Bs = sm + TST * TBM * ALD;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.x * TBM, n0 = blockIdx.z * TBN, ks = blockIdx.y;
    const int k0 = ks * kchunk;
    const int k1 = min(Kp, k0 + kchunk);
    const int nk = k1 > k0 ? (k1 - k0) / TBK : 0;

    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    auto load_stage = [&](int stage, int kt) {
        const int kk = k0 + kt * TBK;
        float* as = As + stage * TBM * ALD;
        float* bs = Bs + stage * TBK * BLD;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int idx = tid + c * 256;
            int r = idx >> 3, c4 = idx & 7;
            int grow = m0 + r;
            const float* src = A + (size_t)(grow < M ? grow : M - 1) * lda + kk + c4 * 4;
            cp_async16(as + r * ALD + c4 * 4, src, grow < M ? 16 : 0);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int idx = tid + c * 256;
            int r = idx >> 5, c4 = idx & 31;
            const float* src = B + (size_t)(kk + r) * ldb + n0 + c4 * 4;
            cp_async16(bs + r * BLD + c4 * 4, src, 16);
        }
    };

#pragma unroll
    for (int st = 0; st < TST - 1; ++st) {
        if (st < nk) load_stage(st, st);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        cp_async_wait<TST - 2>();
        __syncthreads();
        int nxt = kt + TST - 1;
        if (nxt < nk) load_stage(nxt % TST, nxt);
        cp_async_commit();
        const float* as = As + (kt % TST) * TBM * ALD;
        const float* bs = Bs + (kt % TST) * TBK * BLD;
#pragma unroll
        for (int k8 = 0; k8 < TBK / 8; ++k8) {
            unsigned int af[4][4], bf[4][2];
            unsigned int afl[4][4], bfl[4][2];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                const float* ar = as + (wm * 64 + mt * 16 + g) * ALD + k8 * 8 + t;
                float v[4] = {ar[0], ar[8 * ALD], ar[4], ar[8 * ALD + 4]};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float hi = SPLIT3 ? tf32_rna(v[q]) : v[q];
                    af[mt][q] = __float_as_uint(hi);
                    if (SPLIT3) afl[mt][q] = __float_as_uint(tf32_rna(v[q] - hi));
                }
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const float* br = bs + (k8 * 8 + t) * BLD + wn * 32 + nt * 8 + g;
                float v[2] = {br[0], br[4 * BLD]};
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    float hi = SPLIT3 ? tf32_rna(v[q]) : v[q];
                    bf[nt][q] = __float_as_uint(hi);
                    if (SPLIT3) bfl[nt][q] = __float_as_uint(tf32_rna(v[q] - hi));
                }
            }
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    if (SPLIT3) {
                        mma_tf32(acc[mt][nt], afl[mt], bf[nt]);
                        mma_tf32(acc[mt][nt], af[mt], bfl[nt]);
                    }
                    mma_tf32(acc[mt][nt], af[mt], bf[nt]);
                }
        }
    }
    cp_async_wait<0>();
    const int ldp = gridDim.z * TBN;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            int row = m0 + wm * 64 + mt * 16 + g;
            int col = n0 + wn * 32 + nt * 8 + 2 * t;
            float* p = P + ((size_t)ks * M) * ldp;
            if (row < M) {
                p[(size_t)row * ldp + col] = acc[mt][nt][0];
                p[(size_t)row * ldp + col + 1] = acc[mt][nt][1];
            }
            if (row + 8 < M) {
                p[(size_t)(row + 8) * ldp + col] = acc[mt][nt][2];
                p[(size_t)(row + 8) * ldp + col + 1] = acc[mt][nt][3];
            }
        }
}

// B'[2k][j] = Re f[k][j], B'[2k][s+j] = Im f[k][j], B'[2k+1][j] = -Im f, B'[2k+1][s+j] = Re f;
// zero in the padding rows (k >= nc) and columns (>= 2s).
template <bool ROUND>
__global__ void k_build_bprime(const c64* __restrict__ f, int nc, int s, float* __restrict__ Bp,
                               int ldb, int Kp) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)Kp * ldb) return;
    int row = (int)(e / ldb), col = (int)(e - (long long)row * ldb);
    int k = row >> 1, odd = row & 1;
    float v = 0.f;
    if (k < nc && col < 2 * s) {
        int j = col < s ? col : col - s;
        c64 z = f[(size_t)k * s + j];
        if (!odd) v = col < s ? z.re : z.im;
        else v = col < s ? -z.im : z.re;
    }
    Bp[e] = ROUND ? tf32_rna(v) : v;
}

__global__ void k_reduce_cprime(const float* __restrict__ P, int KS, int M, int ldp, int s,
                                c64* __restrict__ u) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)M * s) return;
    int row = (int)(e / s), j = (int)(e - (long long)row * s);
    float re = 0.f, im = 0.f;
    for (int k = 0; k < KS; ++k) {
        const float* p = P + ((size_t)k * M + row) * ldp;
        re += p[j];
        im += p[s + j];
    }
    u[e] = mk(re, im);
}

// A'[i][2k + {0,1}] = (Re, Im) Minv[i][k] in FP32 (rounded to tf32 when the
// solve uses one product), zero for 2k >= 2nc.
__global__ void k_build_aprime(const c128* __restrict__ Minv, int nc, float* __restrict__ Ap, int Kp,
                               int round_tf32) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)nc * Kp) return;
    int i = (int)(e / Kp), c = (int)(e - (long long)i * Kp);
    float v = 0.f;
    if (c < 2 * nc) {
        c128 z = Minv[(size_t)i * nc + (c >> 1)];
        v = __double2float_rn((c & 1) ? z.im : z.re);
    }
    Ap[e] = round_tf32 ? tf32_rna(v) : v;
}

// ---------------------------------------------------------------------------
// FP16 path
// ---------------------------------------------------------------------------
constexpr int HBM_ = 128, HBN = 128, HBK = 32, HST = 4;   // tile and stages (K in halves)
constexpr int HLD = HBK + 8;                                // padded row: ldmatrix without conflicts

__device__ __forceinline__ void mma_f16(float* d, const unsigned int* a, const unsigned int* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void ldsm4(unsigned int* r, const void* p) {
    unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

// power of two p with m * p <= 2^13 < 2 m p (1 for m = 0 or not finite)
__device__ __forceinline__ float pow2_scale(float mx) {
    if (!(mx > 0.f) || !isfinite(mx)) return 1.f;
    int e;
    frexpf(mx, &e);                    // mx = f 2^e, f in [0.5, 1)
    return ldexpf(1.f, 13 - e);
}

// max |re|, |im| over the nc x nc inverse, into *out (as float bits; the
// values are >= 0 so integer max orders them)
__global__ void k_absmax_c128(const c128* __restrict__ M, long long n, unsigned int* out) {
    float mx = 0.f;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        c128 z = M[e];
        mx = fmaxf(mx, fmaxf(fabsf((float)z.re), fabsf((float)z.im)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

// A'_h[i][2k + {0,1}] = half(scale (Re, Im) Minv[i][k]), scale = pow2_scale(max);
// the scale is stored after the nc x Kp halves
__global__ void k_build_aprime_h(const c128* __restrict__ Minv, int nc, __half* __restrict__ Ap, int Kp,
                                 const unsigned int* __restrict__ mxbits) {
    const float sc = pow2_scale(__uint_as_float(*mxbits));
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e == 0) *reinterpret_cast<float*>(Ap + (size_t)nc * Kp) = sc;
    if (e >= (long long)nc * Kp) return;
    int i = (int)(e / Kp), c = (int)(e - (long long)i * Kp);
    float v = 0.f;
    if (c < 2 * nc) {
        c128 z = Minv[(size_t)i * nc + (c >> 1)];
        v = __double2float_rn((c & 1) ? z.im : z.re) * sc;
    }
    Ap[e] = __float2half_rn(v);
}

// per right-hand side j: colmax[j] = max_k max(|Re f_kj|, |Im f_kj|) (float
// bits; non-negative, so the integer max orders them).  Rows of f are read
// whole (coalesced); each CTA reduces its rows per column in shared memory.
__global__ void __launch_bounds__(256) k_colmax(const c64* __restrict__ f, int nc, int s,
                                                unsigned int* __restrict__ colmax) {
    __shared__ float red[256];
    const int j0 = blockIdx.y * 256;                   // columns j0 .. j0 + sc - 1 (gridDim.y chunks)
    const int sc = s - j0 < 256 ? s - j0 : 256;
    const int jj = threadIdx.x % sc, sub = threadIdx.x / sc, per = 256 / sc;
    float mx = 0.f;
    if (sub < per)
        for (long long k = (long long)blockIdx.x * per + sub; k < nc; k += (long long)gridDim.x * per) {
            c64 z = f[k * s + j0 + jj];
            mx = fmaxf(mx, fmaxf(fabsf(z.re), fabsf(z.im)));
        }
    red[threadIdx.x] = sub < per ? mx : 0.f;
    __syncthreads();
    if (sub == 0) {
        for (int q = 1; q < per; ++q) mx = fmaxf(mx, red[q * sc + jj]);
        atomicMax(colmax + j0 + jj, __float_as_uint(mx));
    }
}

// B'^T as halves, Bt[n][k] (k contiguous), n < ldb, k < Kp, with column scales:
// column n < s holds [Re f; -Im f] interleaved by k, column s + n [Im f; Re f]
__global__ void k_build_bt_h(const c64* __restrict__ f, int nc, int s, const unsigned int* __restrict__ colmax,
                             __half* __restrict__ Bt, int Kp, int ldb) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)ldb * Kp) return;
    int n = (int)(e / Kp), k = (int)(e - (long long)n * Kp);
    int kk = k >> 1, odd = k & 1;
    float v = 0.f;
    if (kk < nc && n < 2 * s) {
        int j = n < s ? n : n - s;
        c64 z = f[(size_t)kk * s + j];
        if (!odd) v = n < s ? z.re : z.im;
        else v = n < s ? -z.im : z.re;
        v *= pow2_scale(__uint_as_float(colmax[j]));
    }
    Bt[e] = __float2half_rn(v);
}

// P[ks][row][col] = sum over this CTA's K slice of A'_h[row][k] Bt[col][k].
// 8 warps: 2 along M (64 rows) x 4 along N (32 columns); per k16 step a warp
// loads 4 A and 4 B fragments with ldmatrix and issues 16 mma.
__global__ void __launch_bounds__(256) k_dense_f16(const __half* __restrict__ A, int lda, int M,
                                                    const __half* __restrict__ Bt, int kchunk, int Kp,
                                                    float* __restrict__ P) {
    extern __shared__ __align__(16) __half hsm[];
    __half* As = hsm;                               // HST x HBM_ x HLD
    __half* Bs = hsm + HST * HBM_ * HLD;            // HST x HBN x HLD
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int m0 = blockIdx.x * HBM_, n0 = blockIdx.z * HBN, ks = blockIdx.y;
    const int k0 = ks * kchunk;
    const int k1 = min(Kp, k0 + kchunk);
    const int nk = k1 > k0 ? (k1 - k0) / HBK : 0;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    auto load_stage = [&](int stage, int kt) {
        const int kk = k0 + kt * HBK;
        __half* as = As + stage * HBM_ * HLD;
        __half* bs = Bs + stage * HBN * HLD;
        // 128 rows x 32 halves = 512 chunks of 16 B per operand: two per thread
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            int idx = tid + c * 256;
            int r = idx >> 2, c8 = idx & 3;
            int grow = m0 + r;
            const __half* src = A + (size_t)(grow < M ? grow : M - 1) * lda + kk + c8 * 8;
            cp_async16(as + r * HLD + c8 * 8, src, grow < M ? 16 : 0);
            const __half* srcb = Bt + (size_t)(n0 + r) * Kp + kk + c8 * 8;
            cp_async16(bs + r * HLD + c8 * 8, srcb, 16);
        }
    };
#pragma unroll
    for (int st = 0; st < HST - 1; ++st) {
        if (st < nk) load_stage(st, st);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        cp_async_wait<HST - 2>();
        __syncthreads();
        int nxt = kt + HST - 1;
        if (nxt < nk) load_stage(nxt % HST, nxt);
        cp_async_commit();
        const __half* as = As + (kt % HST) * HBM_ * HLD;
        const __half* bs = Bs + (kt % HST) * HBN * HLD;
#pragma unroll
        for (int k16 = 0; k16 < HBK / 16; ++k16) {
            unsigned int af[4][4], bf[4][2];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
                ldsm4(af[mt], as + (wm * 64 + mt * 16 + (lane & 15)) * HLD + k16 * 16 + (lane >> 4) * 8);
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                // two n8 tiles per x4: matrices (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
                unsigned int r4[4];
                const int nrow = wn * 32 + np * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int kcol = k16 * 16 + ((lane >> 3) & 1) * 8;
                ldsm4(r4, bs + nrow * HLD + kcol);
                bf[2 * np][0] = r4[0];
                bf[2 * np][1] = r4[1];
                bf[2 * np + 1][0] = r4[2];
                bf[2 * np + 1][1] = r4[3];
            }
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_f16(acc[mt][nt], af[mt], bf[nt]);
        }
    }
    cp_async_wait<0>();
    const int g = lane >> 2, t = lane & 3;
    const int ldp = gridDim.z * HBN;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            int row = m0 + wm * 64 + mt * 16 + g;
            int col = n0 + wn * 32 + nt * 8 + 2 * t;
            float* p = P + ((size_t)ks * M) * ldp;
            if (row < M) {
                p[(size_t)row * ldp + col] = acc[mt][nt][0];
                p[(size_t)row * ldp + col + 1] = acc[mt][nt][1];
            }
            if (row + 8 < M) {
                p[(size_t)(row + 8) * ldp + col] = acc[mt][nt][2];
                p[(size_t)(row + 8) * ldp + col + 1] = acc[mt][nt][3];
            }
        }
}

// ---------------------------------------------------------------------------
// FP16 product on the 5th-generation tensor cores (tcgen05)
// ---------------------------------------------------------------------------
// One CTA computes a 128 x 128 tile of C' (rows m0.., columns n0..) over its
// K slice: a producer thread streams 64-wide K tiles of A'_h and of Bt into
// shared memory with TMA (128-byte swizzle, UST stages, mbarrier
// transaction counts), one thread issues tcgen05.mma M=128 N=128 K=16 with
// the FP32 accumulator in 128 columns of tensor memory and frees each stage
// with tcgen05.commit, and the four warps read the accumulator back with
// tcgen05.ld (warp w owns rows 32w .. 32w+31) and write the K slice's
// partial.  Rows beyond M and K beyond Kp are zero-filled by TMA.
constexpr int UM = 128, UN = 128, UK = 64, UST = 6;
constexpr uint32_t kUStageA = UM * UK * 2, kUStageB = UN * UK * 2, kUStage = kUStageA + kUStageB;
constexpr size_t kUSmem = (size_t)UST * kUStage + 1024;   // + slack for 1024-byte alignment

__device__ int g_dense_tc_error = 0;   // set when a pipeline wait gave up

__global__ void __launch_bounds__(128, 1) k_dense_f16_tc05(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB, int M,
                                                           int kchunk, int Kp, float* __restrict__ P,
                                                           int ldp) {
    using namespace tc05;
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) uint64_t full[UST], empty[UST], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const uint32_t sraw = smem_u32(dsm);
    const uint32_t sbase = (sraw + 1023u) & ~1023u;
    unsigned char* tiles = dsm + (sbase - sraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * UM, ks = blockIdx.y, n0 = blockIdx.z * UN;
    const int k0 = ks * kchunk;
    const int k1 = min(Kp, k0 + kchunk);
    const int nk = k1 > k0 ? (k1 - k0 + UK - 1) / UK : 0;
    volatile int* ab = &abort_flag;
    if (threadIdx.x == 0) {
        for (int i = 0; i < UST; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        mbar_fence_init();
        prefetch_tensormap(&tmA);
        prefetch_tensormap(&tmB);
    }
    if (warp == 0) tmem_alloc(&tmem_slot, UN);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: stage st of K tile kt is refilled once the MMAs that read
        // it in the previous round have completed
        int issued = 0;
        for (int kt = 0; kt < nk; ++kt) {
            const int st = kt % UST;
            if (kt >= UST && !mbar_wait(&empty[st], ((kt / UST) & 1) ^ 1, ab)) {
                *ab = 1;
                break;
            }
            unsigned char* a = tiles + (size_t)st * kUStage;
            mbar_arrive_expect_tx(&full[st], kUStage);
            tma_load_2d(a, &tmA, k0 + kt * UK, m0, &full[st]);
            tma_load_2d(a + kUStageA, &tmB, k0 + kt * UK, n0, &full[st]);
            issued = kt + 1;
        }
        if (*ab)   // let the copies this thread started land before the CTA exits
            for (int kt = issued > UST ? issued - UST : 0; kt < issued; ++kt)
                mbar_wait(&full[kt % UST], (kt / UST) & 1, nullptr);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = idesc_f16_f32(UM, UN);
        for (int kt = 0; kt < nk; ++kt) {
            const int st = kt % UST;
            if (!mbar_wait(&full[st], (kt / UST) & 1, ab)) {
                *ab = 1;
                break;
            }
            fence_after_sync();
            const uint32_t a = sbase + (uint32_t)st * kUStage;
            const uint32_t b = a + kUStageA;
#pragma unroll
            for (int k = 0; k < UK / 16; ++k)
                umma_f16(tmem, sdesc_k128(a + k * 32), sdesc_k128(b + k * 32), idesc, (kt | k) != 0 ? 1u : 0u);
            mma_commit(&empty[st]);
        }
        mma_commit(&done);   // arrives when every MMA issued above has completed
    }
    __syncwarp();
    const bool ok = mbar_wait(&done, 0, nullptr) && !*ab;
    __syncwarp();
    fence_after_sync();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < UN / 32; ++c) {
            float v[32];
            if (nk > 0) {
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
            } else {   // an empty K slice contributes zero
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = 0.f;
            }
            if (row < M) {
                float4* dst = reinterpret_cast<float4*>(P + ((size_t)ks * M + row) * ldp + n0 + c * 32);
#pragma unroll
                for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(&g_dense_tc_error, 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, UN);
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2D FP16 tensor map of a row-major `rows` x `cols` matrix (row pitch
// `pitch` elements), 64 x 128 boxes, 128-byte swizzle, zero fill outside
bool map_f16(CUtensorMap* m, const void* base, long long cols, long long rows, long long pitch) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
    cuuint32_t box[2] = {(cuuint32_t)UK, 128};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// u[row][j] = (sum over K slices of C') / (scale_A scale_j)
__global__ void k_reduce_cprime_h(const float* __restrict__ P, int KS, int M, int ldp, int s,
                                  const float* __restrict__ ascale, const unsigned int* __restrict__ colmax,
                                  c64* __restrict__ u) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)M * s) return;
    int row = (int)(e / s), j = (int)(e - (long long)row * s);
    float re = 0.f, im = 0.f;
    for (int k = 0; k < KS; ++k) {
        const float* p = P + ((size_t)k * M + row) * ldp;
        re += p[j];
        im += p[s + j];
    }
    const float inv = 1.f / (*ascale * pow2_scale(__uint_as_float(colmax[j])));   // a power of two: exact
    u[e] = mk(re * inv, im * inv);
}

}  // namespace

int dense_tc_kpad(int nc) { return ((2 * nc + TBK - 1) / TBK) * TBK; }
int dense_tc_ldb(int s) { return ((2 * s + TBN - 1) / TBN) * TBN; }
constexpr int kMaxKSplit = 16;

// K split for an nc x 2nc by 2nc x 2s product: the count of CTAs is
// mt * nt * KS with two CTAs resident per SM (shared memory), so the time goes
// as (waves) x (K tiles per CTA); each split adds a pass of the reduction over
// nc x 2s floats (about 0.9 K-tile-waves at full bandwidth).  The KS in
// 1..16 with the smallest such cost avoids a nearly empty last wave.
int dense_tc_ksplit(int nc, int s) {
    const int mt = (nc + TBM - 1) / TBM, nt = dense_tc_ldb(s) / TBN;
    const int kt = dense_tc_kpad(nc) / TBK;
    const long long slots = 2LL * sm_count();
    int best = 1;
    double best_cost = 1e300;
    for (int ks = 1; ks <= kMaxKSplit; ++ks) {
        long long ctas = (long long)mt * nt * ks;
        long long waves = (ctas + slots - 1) / slots;
        double cost = (double)waves * ((kt + ks - 1) / ks) + 0.9 * ks * nt;
        if (cost < best_cost) { best_cost = cost; best = ks; }
    }
    return best;
}
// K split of the tcgen05 product: one 193 KB CTA per SM, 64-wide K tiles.
// Cost in K-tile times: waves x (K tiles per CTA + a CTA's fixed cost:
// barrier and tensor-memory set-up, pipeline fill, epilogue, about nine
// K tiles as measured at 30 tiles per CTA) + the reduction passes.
int dense_tc05_ksplit(int nc, int s) {
    const int mt = (nc + UM - 1) / UM, nt = dense_tc_ldb(s) / UN;
    const int kt = (dense_tc_kpad(nc) + UK - 1) / UK;
    const long long slots = sm_count();
    int best = 1;
    double best_cost = 1e300;
    for (int ks = 1; ks <= kMaxKSplit; ++ks) {
        long long ctas = (long long)mt * nt * ks;
        long long waves = (ctas + slots - 1) / slots;
        double cost = (double)waves * ((kt + ks - 1) / ks + 9.0) + 0.45 * ks * nt;
        if (cost < best_cost) { best_cost = cost; best = ks; }
    }
    return best;
}

int dense_tc_take_error(cudaStream_t st) {
    static int zero = 0;
    int e = 0;
    if (cudaMemcpyFromSymbolAsync(&e, g_dense_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return 0;
    if (e) {
        cudaMemcpyToSymbolAsync(g_dense_tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
    }
    return e;
}

size_t dense_tc_scratch_floats(int nc, int s) {
    // B' (FP32, or FP16 B'^T in the first half), the K-slice partials, the
    // column scales of the FP16 path
    return (size_t)dense_tc_kpad(nc) * dense_tc_ldb(s) + (size_t)kMaxKSplit * nc * dense_tc_ldb(s) +
           (size_t)dense_tc_ldb(s);
}

void launch_build_aprime(const Launch& L, const c128* Minv, int nc, float* Ap, bool split3) {
    int Kp = dense_tc_kpad(nc);
    long long n = (long long)nc * Kp;
    L.pre(KID_SETUP, 0, 0);
    if (split3) {
        k_build_aprime<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(Minv, nc, Ap, Kp, 0);
    } else {
        // FP16 A' in the first half of the buffer, its scale and the max after it
        __half* Ah = reinterpret_cast<__half*>(Ap);
        unsigned int* mx = reinterpret_cast<unsigned int*>(Ah + (size_t)nc * Kp) + 1;
        cudaMemsetAsync(mx, 0, sizeof(unsigned int), L.st);
        long long nn = (long long)nc * nc;
        long long blocks = (nn + 255) / 256;
        k_absmax_c128<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, L.st>>>(Minv, nn, mx);
        k_build_aprime_h<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(Minv, nc, Ah, Kp, mx);
    }
    L.post();
}

void launch_dense_tc(const Launch& L, const float* Ap, int nc, const c64* f, c64* u, int s,
                     float* scratch, int mode) {
    const bool split3 = mode == 1;
    const bool tc05 = mode == 0;
    const int Kp = dense_tc_kpad(nc), ldb = dense_tc_ldb(s);
    const int KS = tc05 ? dense_tc05_ksplit(nc, s) : dense_tc_ksplit(nc, s);
    float* Bp = scratch;
    float* P = scratch + (size_t)Kp * ldb;
    long long nb = (long long)Kp * ldb;
    if (!split3) {
        // FP16: column scales, B'^T, the product, the scaled reduction
        const __half* Ah = reinterpret_cast<const __half*>(Ap);
        const float* ascale = reinterpret_cast<const float*>(Ah + (size_t)nc * Kp);
        unsigned int* colmax = reinterpret_cast<unsigned int*>(P + (size_t)kMaxKSplit * nc * ldb);
        __half* Bt = reinterpret_cast<__half*>(Bp);
        L.pre(KID_LAYOUT, 2.0 * nb + 16.0 * nc * s, 0);
        cudaMemsetAsync(colmax, 0, sizeof(unsigned int) * s, L.st);
        {
            const int per = s < 256 ? 256 / s : 1;
            long long want = ((long long)nc + per - 1) / per;
            const long long cap = 2LL * sm_count();
            dim3 gcm((unsigned)(want < cap ? want : cap), (unsigned)((s + 255) / 256));
            k_colmax<<<gcm, 256, 0, L.st>>>(f, nc, s, colmax);
        }
        k_build_bt_h<<<(unsigned)((nb + 255) / 256), 256, 0, L.st>>>(f, nc, s, colmax, Bt, Kp, ldb);
        L.post();
        if (tc05) {
            CUtensorMap ta, tb;
            const bool mapped = map_f16(&ta, Ah, Kp, nc, Kp) && map_f16(&tb, Bt, Kp, ldb, Kp);
            const int kt = (Kp + UK - 1) / UK;
            const int kchunk = ((kt + KS - 1) / KS) * UK;
            dim3 grid((nc + UM - 1) / UM, KS, ldb / UN);
            cudaFuncSetAttribute(k_dense_f16_tc05, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUSmem);
            L.pre(KID_DENSE, 2.0 * nc * (double)Kp + 2.0 * nb + 4.0 * KS * nc * (double)ldb,
                  8.0 * nc * (double)nc * s);
            if (mapped) {
                k_dense_f16_tc05<<<grid, 128, kUSmem, L.st>>>(ta, tb, nc, kchunk, Kp, P, ldb);
            } else {
                // no driver entry point for tensor maps: report it through the
                // kernel's error flag (the solve then returns HELM_ERR_CUDA)
                int one = 1;
                cudaMemcpyToSymbolAsync(g_dense_tc_error, &one, sizeof(int), 0, cudaMemcpyHostToDevice, L.st);
            }
            L.post();
            L.pre(KID_LAYOUT, 4.0 * KS * nc * 2.0 * s + 8.0 * nc * s, 0);
            k_reduce_cprime_h<<<(unsigned)(((long long)nc * s + 255) / 256), 256, 0, L.st>>>(P, KS, nc, ldb, s,
                                                                                              ascale, colmax, u);
            L.post();
            return;
        }
        int kchunk = ((Kp / HBK + KS - 1) / KS) * HBK;
        dim3 grid((nc + HBM_ - 1) / HBM_, KS, ldb / HBN);
        size_t smem = sizeof(__half) * (size_t)HST * (HBM_ + HBN) * HLD;
        cudaFuncSetAttribute(k_dense_f16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        L.pre(KID_DENSE, 2.0 * nc * (double)Kp + 2.0 * nb + 4.0 * KS * nc * (double)ldb,
              8.0 * nc * (double)nc * s);
        k_dense_f16<<<grid, 256, smem, L.st>>>(Ah, Kp, nc, Bt, kchunk, Kp, P);
        L.post();
        L.pre(KID_LAYOUT, 4.0 * KS * nc * 2.0 * s + 8.0 * nc * s, 0);
        k_reduce_cprime_h<<<(unsigned)(((long long)nc * s + 255) / 256), 256, 0, L.st>>>(P, KS, nc, ldb, s,
                                                                                          ascale, colmax, u);
        L.post();
        return;
    }
    L.pre(KID_LAYOUT, 4.0 * nb + 8.0 * nc * s, 0);
    if (split3) k_build_bprime<false><<<(unsigned)((nb + 255) / 256), 256, 0, L.st>>>(f, nc, s, Bp, ldb, Kp);
    else k_build_bprime<true><<<(unsigned)((nb + 255) / 256), 256, 0, L.st>>>(f, nc, s, Bp, ldb, Kp);
    L.post();
    int kchunk = ((Kp / TBK + KS - 1) / KS) * TBK;
    dim3 grid((nc + TBM - 1) / TBM, KS, ldb / TBN);
    size_t smem = sizeof(float) * (size_t)TST * (TBM * ALD + TBK * BLD);
    auto kern = split3 ? k_dense_tf32<true> : k_dense_tf32<false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    L.pre(KID_DENSE, 4.0 * nc * (double)Kp + 4.0 * nb + 4.0 * KS * nc * (double)ldb,
          8.0 * nc * (double)nc * s * (split3 ? 3 : 1));
    kern<<<grid, 256, smem, L.st>>>(Ap, Kp, nc, Bp, ldb, kchunk, Kp, P);
    L.post();
    L.pre(KID_LAYOUT, 4.0 * KS * nc * 2.0 * s + 8.0 * nc * s, 0);
    k_reduce_cprime<<<(unsigned)(((long long)nc * s + 255) / 256), 256, 0, L.st>>>(P, KS, nc, ldb, s, u);
    L.post();
}

}  // namespace helm
