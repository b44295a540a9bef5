// Device-side helpers shared by the libhelm kernels: complex arithmetic on
// interleaved (re, im) pairs, the stencil operators of every level, and the
// launch context (stream, launch counter, profiler) of every launcher.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace helm {

template <typename T>
struct alignas(2 * sizeof(T)) cplx {
    T re, im;
};

using c64 = cplx<float>;
using c128 = cplx<double>;

template <typename T>
__host__ __device__ __forceinline__ cplx<T> mk(T r, T i) { cplx<T> z; z.re = r; z.im = i; return z; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(T a, cplx<T> b) { return mk(a * b.re, a * b.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return mk(a.re, -a.im); }
// a += b * c
template <typename T>
__host__ __device__ __forceinline__ void fma_acc(cplx<T>& a, cplx<T> b, cplx<T> c) {
    a.re = fma(b.re, c.re, a.re); a.re = fma(-b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im); a.im = fma(b.im, c.re, a.im);
}
// a += conj(b) * c
template <typename T>
__host__ __device__ __forceinline__ void fma_conj_acc(cplx<T>& a, cplx<T> b, cplx<T> c) {
    a.re = fma(b.re, c.re, a.re); a.re = fma(b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im); a.im = fma(-b.im, c.re, a.im);
}

// ---------------------------------------------------------------------------
// Conversions between FP64 and FP32 built from the bit fields with integer
// operations.  On GB300 the FP64 pipe, which also executes F2F conversions,
// is ~64x narrower than the FP32 pipe, so the FP32 kernels avoid it.
// Values outside the float range flush to zero (tiny) or infinity (huge).
// ---------------------------------------------------------------------------

// float -> double, exact for normal floats
__device__ __forceinline__ double f2d_bits(float f) {
    unsigned int u = __float_as_uint(f);
    unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    unsigned int e = (u >> 23) & 0xFFu;
    unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
    if (e == 0) return __longlong_as_double((long long)sign);
    unsigned long long ed = e == 255 ? 0x7FFULL : (unsigned long long)(e + 896);
    return __longlong_as_double((long long)(sign | (ed << 52) | m));
}

// x = hi + lo, hi = the first 24 significant bits of x (truncated), lo = the
// next 24 of the remaining 29 (truncated): |x - hi - lo| < 2^-47 |x| for
// 2^-74 <= |x| < 2^127; smaller parts flush to zero, NaN/Inf stay visible.
__device__ __forceinline__ void split_d(double x, float& hi, float& lo) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
    unsigned int sign = hw & 0x80000000u;
    int e = (int)((hw >> 20) & 0x7FFu);
    int ef = e - 896;                       // float biased exponent of hi
    if (e == 2047) { hi = __uint_as_float(0x7FC00000u); lo = 0.f; return; }
    if (ef <= 0) { hi = 0.f; lo = 0.f; return; }
    if (ef >= 255) { hi = __uint_as_float(sign | 0x7F800000u); lo = 0.f; return; }
    unsigned int fhi = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    unsigned int flo = lw & 0x1FFFFFFFu;
    hi = __uint_as_float(sign | ((unsigned int)ef << 23) | fhi);
    int lz = __clz(flo);                    // >= 3 when flo != 0
    int el = ef - 52 + (31 - lz);           // biased float exponent of lo
    if (flo == 0 || el <= 0) { lo = 0.f; return; }
    unsigned int mant = (flo << (lz + 1)) >> 9;
    lo = __uint_as_float(sign | ((unsigned int)el << 23) | mant);
}

template <typename To, typename From>
__host__ __device__ __forceinline__ cplx<To> cvt(cplx<From> a) { return mk<To>((To)a.re, (To)a.im); }
#ifdef __CUDA_ARCH__
// on the device: complex128 -> complex64 by truncation to 24 bits, and the
// exact complex64 -> complex128 widening, both without FP64-pipe work
template <>
__device__ __forceinline__ cplx<float> cvt<float, double>(cplx<double> a) {
    float h, l;
    cplx<float> z;
    split_d(a.re, h, l); z.re = h;
    split_d(a.im, h, l); z.im = h;
    return z;
}
template <>
__device__ __forceinline__ cplx<double> cvt<double, float>(cplx<float> a) {
    return mk<double>(f2d_bits(a.re), f2d_bits(a.im));
}
#endif

template <typename T>
__device__ __forceinline__ cplx<T> ldg(const cplx<T>* p) {
    cplx<T> z;
    if (sizeof(T) == 8) {
        double2 v = __ldg(reinterpret_cast<const double2*>(p));
        z.re = (T)v.x; z.im = (T)v.y;
    } else {
        float2 v = __ldg(reinterpret_cast<const float2*>(p));
        z.re = (T)v.x; z.im = (T)v.y;
    }
    return z;
}

// R consecutive complex values (R = 1 or 2) loaded/stored with one vector
// access where the type allows it (the pair is 16-byte aligned when the first
// column index is even).
template <typename T, int R>
struct CV {
    cplx<T> v[R];
};
template <typename U, int R>
__device__ __forceinline__ CV<U, R> ldR(const cplx<U>* p) {
    CV<U, R> o;
    if constexpr (R == 2 && sizeof(U) == 4) {
        float4 q = __ldg(reinterpret_cast<const float4*>(p));
        o.v[0] = mk<U>(q.x, q.y);
        o.v[1] = mk<U>(q.z, q.w);
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) o.v[k] = ldg(p + k);
    }
    return o;
}
template <typename U, int R>
__device__ __forceinline__ void stR(cplx<U>* p, const CV<U, R>& o) {
    if constexpr (R == 2 && sizeof(U) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o.v[0].re, o.v[0].im, o.v[1].re, o.v[1].im);
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) p[k] = o.v[k];
    }
}

// Grid of nodes; x1 fastest.  n[2] = 1 in 2D.
struct Grid {
    int dim;
    int n1, n2, n3;
    long long N;
    __host__ __device__ __forceinline__ void coords(long long node, int& x, int& y, int& z) const {
        x = (int)(node % n1);
        long long t = node / n1;
        y = (int)(t % n2);
        z = (int)(t / n2);
    }
    __host__ __device__ __forceinline__ long long index(int x, int y, int z) const {
        return ((long long)z * n2 + y) * n1 + x;
    }
};

// Fine-level operator: y = (1/h^2) (2d u_i - sum_{axis nbrs} u_j) - c_i u_i
// (Sec. 2.4: second-order finite differences), c = omega^2 m (1 - i gamma').
template <typename T>
struct FineOp {
    Grid g;
    T inv_h2;
    const cplx<T>* c;     // mass coefficient per node
    const cplx<T>* dinv;  // 1 / (2d/h^2 - c_i) per node (Jacobi); may be null

    template <typename U>
    __device__ __forceinline__ cplx<T> apply(const cplx<U>* u, long long node, int x, int y, int z,
                                             int s, int r) const {
        const cplx<U>* p = u + node * s + r;
        cplx<T> ui = cvt<T>(ldg(p));
        cplx<T> sum = mk<T>(0, 0);
        if (x > 0) sum = sum + cvt<T>(ldg(p - s));
        if (x < g.n1 - 1) sum = sum + cvt<T>(ldg(p + s));
        long long sy = (long long)g.n1 * s;
        if (y > 0) sum = sum + cvt<T>(ldg(p - sy));
        if (y < g.n2 - 1) sum = sum + cvt<T>(ldg(p + sy));
        if (g.dim == 3) {
            long long sz = (long long)g.n1 * g.n2 * s;
            if (z > 0) sum = sum + cvt<T>(ldg(p - sz));
            if (z < g.n3 - 1) sum = sum + cvt<T>(ldg(p + sz));
        }
        T dd = (T)(2 * g.dim);
        cplx<T> ci = ldg(c + node);
        cplx<T> y_ = inv_h2 * mk<T>(dd * ui.re - sum.re, dd * ui.im - sum.im);
        return y_ - ci * ui;
    }
    __device__ __forceinline__ cplx<T> diag_inv(long long node) const { return ldg(dinv + node); }

    // the same for R consecutive columns r0 .. r0+R-1
    template <int R, typename U>
    __device__ __forceinline__ void applyR(const cplx<U>* u, long long node, int x, int y, int z,
                                           int s, int r0, cplx<T>* out) const {
        const cplx<U>* p = u + node * s + r0;
        CV<U, R> ui = ldR<U, R>(p);
        cplx<T> sum[R];
#pragma unroll
        for (int k = 0; k < R; ++k) sum[k] = mk<T>(0, 0);
        auto add = [&](const cplx<U>* q) {
            CV<U, R> v = ldR<U, R>(q);
#pragma unroll
            for (int k = 0; k < R; ++k) sum[k] = sum[k] + cvt<T>(v.v[k]);
        };
        if (x > 0) add(p - s);
        if (x < g.n1 - 1) add(p + s);
        const long long sy = (long long)g.n1 * s;
        if (y > 0) add(p - sy);
        if (y < g.n2 - 1) add(p + sy);
        if (g.dim == 3) {
            const long long sz = (long long)g.n1 * g.n2 * s;
            if (z > 0) add(p - sz);
            if (z < g.n3 - 1) add(p + sz);
        }
        const T dd = (T)(2 * g.dim);
        const cplx<T> ci = ldg(c + node);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            cplx<T> uk = cvt<T>(ui.v[k]);
            out[k] = inv_h2 * mk<T>(dd * uk.re - sum[k].re, dd * uk.im - sum[k].im) - ci * uk;
        }
    }
};

// Galerkin coarse operator: 9-point (2D) or 27-point (3D) stencil with
// per-node complex coefficients coef[node*K + o], o = (dx+1) + 3(dy+1) [+ 9(dz+1)].
template <typename T>
struct GalOp {
    Grid g;
    const cplx<T>* coef;
    const cplx<T>* dinv;

    template <typename U>
    __device__ __forceinline__ cplx<T> apply(const cplx<U>* u, long long node, int x, int y, int z,
                                             int s, int r) const {
        const int K = g.dim == 3 ? 27 : 9;
        const cplx<T>* cf = coef + node * K;
        cplx<T> acc = mk<T>(0, 0);
        const int z0 = g.dim == 3 ? -1 : 0, z1 = g.dim == 3 ? 1 : 0;
        for (int dz = z0; dz <= z1; ++dz) {
            int zz = z + dz;
            if (zz < 0 || zz >= g.n3) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int yy = y + dy;
                if (yy < 0 || yy >= g.n2) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    int xx = x + dx;
                    if (xx < 0 || xx >= g.n1) continue;
                    int o = (dx + 1) + 3 * (dy + 1) + (g.dim == 3 ? 9 * (dz + 1) : 0);
                    cplx<T> cc = ldg(cf + o);
                    cplx<T> uv = cvt<T>(ldg(u + g.index(xx, yy, zz) * s + r));
                    fma_acc(acc, cc, uv);
                }
            }
        }
        return acc;
    }
    __device__ __forceinline__ cplx<T> diag_inv(long long node) const { return ldg(dinv + node); }

    // the same for R consecutive columns r0 .. r0+R-1
    template <int R, typename U>
    __device__ __forceinline__ void applyR(const cplx<U>* u, long long node, int x, int y, int z,
                                           int s, int r0, cplx<T>* out) const {
        const int K = g.dim == 3 ? 27 : 9;
        const cplx<T>* cf = coef + node * K;
#pragma unroll
        for (int k = 0; k < R; ++k) out[k] = mk<T>(0, 0);
        const int z0 = g.dim == 3 ? -1 : 0, z1 = g.dim == 3 ? 1 : 0;
        for (int dz = z0; dz <= z1; ++dz) {
            int zz = z + dz;
            if (zz < 0 || zz >= g.n3) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int yy = y + dy;
                if (yy < 0 || yy >= g.n2) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    int xx = x + dx;
                    if (xx < 0 || xx >= g.n1) continue;
                    int o = (dx + 1) + 3 * (dy + 1) + (g.dim == 3 ? 9 * (dz + 1) : 0);
                    cplx<T> cc = ldg(cf + o);
                    CV<U, R> uv = ldR<U, R>(u + g.index(xx, yy, zz) * s + r0);
#pragma unroll
                    for (int k = 0; k < R; ++k) fma_acc(out[k], cc, cvt<T>(uv.v[k]));
                }
            }
        }
    }
};

// Kernel classes seen by the profiler (helm_profile_* in helm.h).
enum KernelId {
    KID_APPLY_FINE = 0, KID_APPLY_COARSE, KID_RESIDUAL, KID_JACOBI_FINE, KID_JACOBI_COARSE,
    KID_RESTRICT_FINE, KID_RESTRICT_COARSE, KID_PROLONG, KID_DENSE, KID_GRAM, KID_GRAM_REDUCE,
    KID_COMBINE, KID_LAYOUT, KID_RANDOM, KID_SETUP, KID_GRAM_DD, KID_COMBINE_DD, KID_CONV, KID_CONV_WGRAD, KID_GRAM_HI, KID_COMBINE_HI, KID_COUNT
};

struct Profiler;  // host side, defined in solver.cu
void prof_begin(Profiler* p, cudaStream_t st, int kid, double bytes, double flops);
void prof_end(Profiler* p, cudaStream_t st);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount),
// read once per device; launch shapes are sized in multiples of it.
inline int sm_count() {
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (cache[dev] <= 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        cache[dev] = n;
    }
    return cache[dev];
}

struct Launch {
    cudaStream_t st;
    long long* counter;  // incremented once per kernel launch
    Profiler* prof;      // null unless profiling is on
    // pre(): before a launch, with its algorithmic bytes and flops; post(): after it
    void pre(int kid, double bytes, double flops) const {
        if (prof) prof_begin(prof, st, kid, bytes, flops);
    }
    void post() const {
        if (counter) ++*counter;
        if (prof) prof_end(prof, st);
    }
};

}  // namespace helm
