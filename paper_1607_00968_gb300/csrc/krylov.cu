// Block-Krylov kernels of the block FGMRES driver (Sec. 5.3, block FGMRES of
// Calandra et al.): block Gram products V^H W per group of right-hand sides,
// block combinations W -= V H / X += Z Y / Q = W T, column norms, random
// directions for rank-deficient blocks, and the ABI <-> internal layout
// transposes.  All arithmetic is FP64.
#include "kernels.h"

namespace helm {

namespace {

constexpr int kThreads = 256;
constexpr int kGramEPT = 8;          // accumulators per thread in the Gram kernel
constexpr int kGramTileElems = 1024; // node-tile size (nodes x s) staged in shared memory
constexpr int kTargetCTAs = 4 * 152; // 4 waves' worth of CTAs on 152 SMs

inline int blocks_for(long long total) {
    long long b = (total + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 0x7fffffffLL) b = 0x7fffffffLL;
    return (int)b;
}

__host__ __device__ inline int gram_tile_nodes(int s) { return s >= kGramTileElems ? 1 : kGramTileElems / s; }

inline int gram_chunks(long long N, int nb, int s) {
    long long tn = gram_tile_nodes(s);
    long long tiles = (N + tn - 1) / tn;
    long long want = (kTargetCTAs + nb - 1) / nb;
    if (want < 1) want = 1;
    return (int)(tiles < want ? tiles : want);
}

// One CTA: block i = blockIdx.y of X, node chunk blockIdx.x.  Entries
// (g, a, b) of the per-group sb x sb products are spread over the threads,
// kGramEPT per thread per pass; node tiles of X_i and Y sit in shared memory.
__global__ void __launch_bounds__(kThreads) k_gram(const c128* __restrict__ X, long long xstride,
                                                    const c128* __restrict__ Y, long long N, int s,
                                                    int sb, int chunks, c128* __restrict__ partial) {
    extern __shared__ c128 sm[];
    const int tn = gram_tile_nodes(s);
    c128* xs = sm;
    c128* ys = sm + (size_t)tn * s;
    const int i = blockIdx.y;
    const int G = (s + sb - 1) / sb;
    const long long E1 = (long long)G * sb * sb;
    const c128* Xi = X + (long long)i * xstride;
    long long per = (N + chunks - 1) / chunks;
    long long n0 = (long long)blockIdx.x * per;
    long long n1 = n0 + per < N ? n0 + per : N;
    c128* out = partial + ((long long)blockIdx.x * gridDim.y + i) * E1;
    for (long long base = 0; base < E1; base += (long long)kThreads * kGramEPT) {
        c128 acc[kGramEPT];
        int ca[kGramEPT], cb[kGramEPT];
        bool ok[kGramEPT];
#pragma unroll
        for (int q = 0; q < kGramEPT; ++q) {
            long long e = base + threadIdx.x + (long long)q * kThreads;
            acc[q] = mk(0.0, 0.0);
            ok[q] = false;
            ca[q] = cb[q] = 0;
            if (e < E1) {
                int g = (int)(e / ((long long)sb * sb));
                int rem = (int)(e - (long long)g * sb * sb);
                int a = rem / sb, b = rem % sb;
                ca[q] = g * sb + a;
                cb[q] = g * sb + b;
                ok[q] = ca[q] < s && cb[q] < s;
            }
        }
        for (long long t0 = n0; t0 < n1; t0 += tn) {
            int cnt = (int)((n1 - t0) < tn ? (n1 - t0) : tn);
            __syncthreads();
            for (int idx = threadIdx.x; idx < cnt * s; idx += kThreads) {
                xs[idx] = Xi[t0 * s + idx];
                ys[idx] = Y[t0 * s + idx];
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kGramEPT; ++q) {
                if (!ok[q]) continue;
                for (int n = 0; n < cnt; ++n)
                    fma_conj_acc(acc[q], xs[n * s + ca[q]], ys[n * s + cb[q]]);
            }
        }
#pragma unroll
        for (int q = 0; q < kGramEPT; ++q) {
            long long e = base + threadIdx.x + (long long)q * kThreads;
            if (e < E1) out[e] = acc[q];
        }
    }
}

__global__ void k_gram_reduce(const c128* __restrict__ partial, int chunks, long long E,
                              c128* __restrict__ out) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= E) return;
    c128 acc = mk(0.0, 0.0);
    for (int c = 0; c < chunks; ++c) acc = acc + partial[(long long)c * E + e];
    out[e] = acc;
}

template <typename TX>
__global__ void __launch_bounds__(kThreads) k_combine(c128* __restrict__ out, double beta, double sign,
                                                       const cplx<TX>* __restrict__ X, int nb,
                                                       long long xstride,
                                                       const c128* __restrict__ C, long long N,
                                                       int s, int sb) {
    const long long total = N * s;
    const int G = (s + sb - 1) / sb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long node = e / s;
        int col = (int)(e - node * s);
        int g = col / sb, b = col - g * sb;
        int amax = s - g * sb < sb ? s - g * sb : sb;
        c128 acc = mk(0.0, 0.0);
        for (int i = 0; i < nb; ++i) {
            const cplx<TX>* xr = X + (long long)i * xstride + node * s + g * sb;
            const c128* cc = C + (((long long)i * G + g) * sb) * sb + b;
            for (int a = 0; a < amax; ++a) fma_acc(acc, cvt<double>(ldg(xr + a)), ldg(cc + (long long)a * sb));
        }
        c128 o = beta != 0.0 ? beta * out[e] : mk(0.0, 0.0);
        out[e] = o + sign * acc;
    }
}

// 32 x 32 tiled transposes between the ABI layout (column j contiguous) and
// the internal node-major layout.
__global__ void k_to_internal(const c128* __restrict__ abi, c128* __restrict__ in, long long N,
                              int s, int conjugate) {
    __shared__ c128 tile[32][33];
    long long n0 = (long long)blockIdx.x * 32;
    int j0 = blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        long long n = n0 + tx;
        int j = j0 + k;
        if (n < N && j < s) {
            c128 v = abi[(long long)j * N + n];
            if (conjugate) v.im = -v.im;
            tile[k][tx] = v;
        }
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        long long n = n0 + k;
        int j = j0 + tx;
        if (n < N && j < s) in[n * s + j] = tile[tx][k];
    }
}

__global__ void k_from_internal(const c128* __restrict__ in, c128* __restrict__ abi, long long N,
                                int s, int conjugate) {
    __shared__ c128 tile[32][33];
    long long n0 = (long long)blockIdx.x * 32;
    int j0 = blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;
    for (int k = ty; k < 32; k += 8) {
        long long n = n0 + k;
        int j = j0 + tx;
        if (n < N && j < s) tile[k][tx] = in[n * s + j];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        long long n = n0 + tx;
        int j = j0 + k;
        if (n < N && j < s) {
            c128 v = tile[tx][k];
            if (conjugate) v.im = -v.im;
            abi[(long long)j * N + n] = v;
        }
    }
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

__global__ void k_fill_random(c128* X, long long N, int s, const int* __restrict__ mask,
                              unsigned long long seed) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= N * s) return;
    int col = (int)(e % s);
    if (!mask[col]) return;
    unsigned long long h1 = splitmix64(seed ^ (2ULL * (unsigned long long)e));
    unsigned long long h2 = splitmix64(seed ^ (2ULL * (unsigned long long)e + 1ULL));
    double u1 = (double)(h1 >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    X[e] = mk(u1, u2);
}

}  // namespace

long long gram_partial_elems(long long N, int nb, int s, int sb) {
    int G = (s + sb - 1) / sb;
    long long E1 = (long long)G * sb * sb;
    return (long long)gram_chunks(N, nb, s) * nb * E1;
}

void launch_gram(const Launch& L, const c128* X, int nb, long long xstride, const c128* Y,
                 long long N, int s, int sb, c128* partial, c128* out) {
    int G = (s + sb - 1) / sb;
    long long E1 = (long long)G * sb * sb;
    int chunks = gram_chunks(N, nb, s);
    size_t smem = 2 * sizeof(c128) * (size_t)gram_tile_nodes(s) * s;
    dim3 grid(chunks, nb);
    L.pre(KID_GRAM, (nb + 1.0) * N * s * 16.0, 8.0 * nb * (double)N * s * sb);
    k_gram<<<grid, kThreads, smem, L.st>>>(X, xstride, Y, N, s, sb, chunks, partial);
    L.post();
    long long E = E1 * nb;
    L.pre(KID_GRAM_REDUCE, (chunks + 1.0) * E * 16.0, 2.0 * chunks * E);
    k_gram_reduce<<<blocks_for(E), kThreads, 0, L.st>>>(partial, chunks, E, out);
    L.post();
}

template <typename TX>
void launch_combine(const Launch& L, c128* out, double beta, double sign, const cplx<TX>* X,
                    int nb, long long xstride, const c128* C, long long N, int s, int sb) {
    L.pre(KID_COMBINE, (double)N * s * (nb * 2.0 * sizeof(TX) + (beta != 0.0 ? 32.0 : 16.0)),
          8.0 * nb * (double)N * s * sb);
    k_combine<TX><<<blocks_for(N * s), kThreads, 0, L.st>>>(out, beta, sign, X, nb, xstride, C, N,
                                                            s, sb);
    L.post();
}
template void launch_combine<double>(const Launch&, c128*, double, double, const c128*, int,
                                     long long, const c128*, long long, int, int);
template void launch_combine<float>(const Launch&, c128*, double, double, const c64*, int,
                                    long long, const c128*, long long, int, int);

long long colnorm_partial_elems(long long N, int s) { return gram_partial_elems(N, 1, s, 1); }

void launch_colnorm2(const Launch& L, const c128* X, long long N, int s, double* partial,
                     double* out) {
    // Per-column norms are the 1 x 1 groups of the Gram product X^H X;
    // out receives (re, im) pairs, the imaginary parts being zero.
    launch_gram(L, X, 1, 0, X, N, s, 1, reinterpret_cast<c128*>(partial),
                reinterpret_cast<c128*>(out));
}

void launch_to_internal(const Launch& L, const c128* abi, c128* internal, long long N, int s,
                        bool conjugate) {
    dim3 grid((unsigned)((N + 31) / 32), (s + 31) / 32);
    L.pre(KID_LAYOUT, 32.0 * N * s, 0);
    k_to_internal<<<grid, dim3(32, 8), 0, L.st>>>(abi, internal, N, s, conjugate ? 1 : 0);
    L.post();
}

void launch_from_internal(const Launch& L, const c128* internal, c128* abi, long long N, int s,
                          bool conjugate) {
    dim3 grid((unsigned)((N + 31) / 32), (s + 31) / 32);
    L.pre(KID_LAYOUT, 32.0 * N * s, 0);
    k_from_internal<<<grid, dim3(32, 8), 0, L.st>>>(internal, abi, N, s, conjugate ? 1 : 0);
    L.post();
}

void launch_fill_random(const Launch& L, c128* X, long long N, int s, const int* mask,
                        unsigned long long seed) {
    L.pre(KID_RANDOM, 16.0 * N * s, 0);
    k_fill_random<<<blocks_for(N * s), kThreads, 0, L.st>>>(X, N, s, mask, seed);
    L.post();
}

void launch_zero(const Launch& L, void* p, size_t bytes) { cudaMemsetAsync(p, 0, bytes, L.st); }

}  // namespace helm
