// Multigrid kernels of the shifted-Laplacian preconditioner (Sec. 4, Alg.
// "Two-grid cycle"): stencil apply, damped Jacobi, fused residual +
// restriction, prolongation + correction, coarsest dense solve; and the
// set-up kernels (fine coefficients, Galerkin P^T M P, Gauss-Jordan inverse).
//
// Vectors are node-major with the s right-hand sides innermost
// (x[node*s + j]); one thread owns one (node, column) element, so a warp
// reads contiguous memory and the stencil neighbours of one node are s
// elements apart (x1) or one grid row / plane apart (x2, x3).
#include "kernels.h"

namespace helm {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(long long total) {
    long long b = (total + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 0x7fffffffLL) b = 0x7fffffffLL;
    return (int)b;
}

template <typename T, typename U, typename V, typename Op>
__global__ void __launch_bounds__(kThreads) k_apply(Op op, const cplx<U>* __restrict__ x,
                                                     cplx<V>* __restrict__ y, int s,
                                                     long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long node = e / s;
        int r = (int)(e - node * s);
        int a, b, c;
        op.g.coords(node, a, b, c);
        cplx<T> v = op.apply(x, node, a, b, c, s, r);
        y[e] = cvt<V>(v);
    }
}

template <typename T, typename Op>
__global__ void __launch_bounds__(kThreads) k_residual(Op op, const cplx<T>* __restrict__ x,
                                                        const cplx<T>* __restrict__ bv,
                                                        cplx<T>* __restrict__ r_, int s,
                                                        long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long node = e / s;
        int r = (int)(e - node * s);
        int a, b, c;
        op.g.coords(node, a, b, c);
        r_[e] = ldg(bv + e) - op.apply(x, node, a, b, c, s, r);
    }
}

template <typename T, typename FT, typename Op>
__global__ void __launch_bounds__(kThreads) k_jacobi(Op op, const cplx<T>* __restrict__ uin,
                                                      const cplx<FT>* __restrict__ f,
                                                      cplx<T>* __restrict__ uout, int s, T w,
                                                      long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long node = e / s;
        int r = (int)(e - node * s);
        cplx<T> fi = cvt<T>(ldg(f + e));
        cplx<T> d = op.diag_inv(node);
        if (uin == nullptr) {
            uout[e] = w * (d * fi);
        } else {
            int a, b, c;
            op.g.coords(node, a, b, c);
            cplx<T> Au = op.apply(uin, node, a, b, c, s, r);
            cplx<T> ui = ldg(uin + e);
            uout[e] = ui + w * (d * (fi - Au));
        }
    }
}

// rc[J] = sum over fine nodes i = 2J + delta of prod_k w(delta_k) (f - Op u)_i,
// w(0) = 1, w(+-1) = 1/2 (full weighting with R = P^T, Sec. 4).
template <typename T, typename FT, typename Op>
__global__ void __launch_bounds__(kThreads) k_resid_restrict(Op op, Grid gc,
                                                              const cplx<T>* __restrict__ u,
                                                              const cplx<FT>* __restrict__ f,
                                                              cplx<T>* __restrict__ rc, int s,
                                                              long long total) {
    const Grid& gf = op.g;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long J = e / s;
        int r = (int)(e - J * s);
        int jx, jy, jz;
        gc.coords(J, jx, jy, jz);
        cplx<T> acc = mk<T>(0, 0);
        const int z0 = gf.dim == 3 ? -1 : 0, z1 = gf.dim == 3 ? 1 : 0;
        for (int dz = z0; dz <= z1; ++dz) {
            int fz = gf.dim == 3 ? 2 * jz + dz : 0;
            if (fz < 0 || fz >= gf.n3) continue;
            T wz = dz == 0 ? T(1) : T(0.5);
            for (int dy = -1; dy <= 1; ++dy) {
                int fy = 2 * jy + dy;
                if (fy < 0 || fy >= gf.n2) continue;
                T wy = dy == 0 ? wz : T(0.5) * wz;
                for (int dx = -1; dx <= 1; ++dx) {
                    int fx = 2 * jx + dx;
                    if (fx < 0 || fx >= gf.n1) continue;
                    T wgt = dx == 0 ? wy : T(0.5) * wy;
                    long long i = gf.index(fx, fy, fz);
                    cplx<T> ri = cvt<T>(ldg(f + i * s + r));
                    if (u != nullptr) ri = ri - op.apply(u, i, fx, fy, fz, s, r);
                    acc = acc + wgt * ri;
                }
            }
        }
        rc[e] = acc;
    }
}

// u_i += sum_J P_iJ ec_J: per axis an even fine index takes coarse i/2 with
// weight 1, an odd one the two neighbours with weight 1/2 (bilinear, Sec. 4).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_prolong_add(Grid gf, Grid gc,
                                                           const cplx<T>* __restrict__ ec,
                                                           cplx<T>* __restrict__ u, int s,
                                                           long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long node = e / s;
        int r = (int)(e - node * s);
        int x, y, z;
        gf.coords(node, x, y, z);
        int xs[2], ys[2], zs[2];
        int nx = (x & 1) ? 2 : 1, ny = (y & 1) ? 2 : 1, nz = (gf.dim == 3 && (z & 1)) ? 2 : 1;
        xs[0] = x >> 1; xs[1] = (x >> 1) + 1;
        ys[0] = y >> 1; ys[1] = (y >> 1) + 1;
        zs[0] = z >> 1; zs[1] = (z >> 1) + 1;
        T w = T(1);
        if (nx == 2) w *= T(0.5);
        if (ny == 2) w *= T(0.5);
        if (nz == 2) w *= T(0.5);
        cplx<T> acc = mk<T>(0, 0);
        for (int c = 0; c < nz; ++c)
            for (int b = 0; b < ny; ++b)
                for (int a = 0; a < nx; ++a)
                    acc = acc + ldg(ec + gc.index(xs[a], ys[b], zs[c]) * s + r);
        u[e] = ldg(u + e) + w * acc;
    }
}

// ---------------------------------------------------------------------------
// Division-free variants: block (TX, TY) covers TY consecutive nodes of one
// grid row (blockIdx.y = x2 index, blockIdx.z = x3 index) and TX * R columns;
// thread (tx, ty) owns columns tx*R .. tx*R+R-1 of node x = blockIdx.x*TY + ty.
// R = 2 when s is even (one 16-byte access per complex64 pair).
// ---------------------------------------------------------------------------

struct Geo {
    dim3 grid, block;
    int R;
    bool ok;
};

inline Geo geo_for(const Grid& g, int s) {
    Geo o;
    o.R = (s % 2 == 0) ? 2 : 1;
    int tx = s / o.R;
    o.ok = tx <= 256;
    int ty = tx >= 256 ? 1 : 256 / tx;
    o.block = dim3(tx, ty, 1);
    o.grid = dim3((g.n1 + ty - 1) / ty, g.n2, g.n3);
    return o;
}

#define VGEO_PROLOGUE(G)                                                   \
    const int x = blockIdx.x * blockDim.y + threadIdx.y;                   \
    if (x >= (G).n1) return;                                               \
    const int y = blockIdx.y, z = blockIdx.z;                              \
    const long long node = ((long long)z * (G).n2 + y) * (G).n1 + x;       \
    const int r0 = threadIdx.x * R;                                        \
    const long long e0 = node * s + r0;

template <typename T, typename U, typename V, typename Op, int R>
__global__ void __launch_bounds__(256) k_apply_v(Op op, const cplx<U>* __restrict__ xin,
                                                  cplx<V>* __restrict__ yout, int s) {
    VGEO_PROLOGUE(op.g)
    cplx<T> o[R];
    op.template applyR<R>(xin, node, x, y, z, s, r0, o);
    CV<V, R> w;
#pragma unroll
    for (int k = 0; k < R; ++k) w.v[k] = cvt<V>(o[k]);
    stR<V, R>(yout + e0, w);
}

// error-free a + b = s + e (TwoSum)
__device__ __forceinline__ void ddf_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// (S, E) += t for a float t (E gathers the rounding errors)
__device__ __forceinline__ void ddf_add(float& S, float& E, float t) {
    float e;
    ddf_two_sum(S, t, S, e);
    E = __fadd_rn(E, e);
}

// (S, E) -= (ch + cl) u: the product's high part exactly by FMA, the cross
// term c_lo u into the error
__device__ __forceinline__ void ddf_sub_prod(float& S, float& E, float ch, float cl, float u) {
    float q = __fmul_rn(ch, u);
    float qe = __fmaf_rn(ch, u, -q);
    qe = __fmaf_rn(cl, u, qe);
    float e;
    ddf_two_sum(S, -q, S, e);
    E = __fadd_rn(E, __fsub_rn(e, qe));
}

// y = A x on the fine grid for complex64 x, in double-float arithmetic on
// the FP32 pipes: the 2d u_i - sum of neighbours is summed error-free, scaled
// by 1/h^2 = ih + il and reduced by c_i u_i with c_i = (re hi, re lo, im hi,
// im lo); each component ends as a renormalised pair, written to the hi plane
// (y) and the lo plane (y + N*s).  About 2^-46 relative to the largest term.
template <int R>
__global__ void __launch_bounds__(256) k_apply_dd(Grid g, float ih, float il, const float4* __restrict__ cdd,
                                                   const c64* __restrict__ xin, c64* __restrict__ yout,
                                                   int s) {
    VGEO_PROLOGUE(g)
    const c64* p = xin + e0;
    const CV<float, R> ui = ldR<float, R>(p);
    float S[R][2], E[R][2];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        S[k][0] = 4.f * ui.v[k].re;            // exact
        S[k][1] = 4.f * ui.v[k].im;
        E[k][0] = E[k][1] = 0.f;
        if (g.dim == 3) {
            ddf_add(S[k][0], E[k][0], 2.f * ui.v[k].re);
            ddf_add(S[k][1], E[k][1], 2.f * ui.v[k].im);
        }
    }
    auto sub = [&](const c64* q) {
        CV<float, R> v = ldR<float, R>(q);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            ddf_add(S[k][0], E[k][0], -v.v[k].re);
            ddf_add(S[k][1], E[k][1], -v.v[k].im);
        }
    };
    if (x > 0) sub(p - s);
    if (x < g.n1 - 1) sub(p + s);
    const long long sy = (long long)g.n1 * s;
    if (y > 0) sub(p - sy);
    if (y < g.n2 - 1) sub(p + sy);
    if (g.dim == 3) {
        const long long sz = (long long)g.n1 * g.n2 * s;
        if (z > 0) sub(p - sz);
        if (z < g.n3 - 1) sub(p + sz);
    }
    const float4 c = __ldg(cdd + node);
    CV<float, R> hi, lo;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        float T[2], Te[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            // (S + E) (ih + il)
            T[q] = __fmul_rn(S[k][q], ih);
            Te[q] = __fmaf_rn(S[k][q], ih, -T[q]);
            Te[q] = __fmaf_rn(S[k][q], il, Te[q]);
            Te[q] = __fmaf_rn(E[k][q], ih, Te[q]);
        }
        // - c u:  re -= cr ur - ci ui ;  im -= cr ui + ci ur
        ddf_sub_prod(T[0], Te[0], c.x, c.y, ui.v[k].re);
        ddf_sub_prod(T[0], Te[0], -c.z, -c.w, ui.v[k].im);
        ddf_sub_prod(T[1], Te[1], c.x, c.y, ui.v[k].im);
        ddf_sub_prod(T[1], Te[1], c.z, c.w, ui.v[k].re);
        ddf_two_sum(T[0], Te[0], hi.v[k].re, lo.v[k].re);
        ddf_two_sum(T[1], Te[1], hi.v[k].im, lo.v[k].im);
    }
    stR<float, R>(yout + e0, hi);
    stR<float, R>(yout + g.N * s + e0, lo);
}

template <typename T, typename FT, typename Op, int R>
__global__ void __launch_bounds__(256) k_jacobi_v(Op op, const cplx<T>* __restrict__ uin,
                                                   const cplx<FT>* __restrict__ f,
                                                   cplx<T>* __restrict__ uout, int s, T w) {
    VGEO_PROLOGUE(op.g)
    CV<FT, R> fv = ldR<FT, R>(f + e0);
    const cplx<T> d = op.diag_inv(node);
    CV<T, R> outv;
    if (uin == nullptr) {
#pragma unroll
        for (int k = 0; k < R; ++k) outv.v[k] = w * (d * cvt<T>(fv.v[k]));
    } else {
        cplx<T> Au[R];
        op.template applyR<R>(uin, node, x, y, z, s, r0, Au);
        CV<T, R> ui = ldR<T, R>(uin + e0);
#pragma unroll
        for (int k = 0; k < R; ++k)
            outv.v[k] = ui.v[k] + w * (d * (cvt<T>(fv.v[k]) - Au[k]));
    }
    stR<T, R>(uout + e0, outv);
}

// coarse node J = (x, y, z) on gc; gathers the 3^d fine nodes 2J + delta
template <typename T, typename FT, typename Op, int R>
__global__ void __launch_bounds__(256) k_resid_restrict_v(Op op, Grid gc, const cplx<T>* __restrict__ u,
                                                           const cplx<FT>* __restrict__ f,
                                                           cplx<T>* __restrict__ rc, int s) {
    VGEO_PROLOGUE(gc)
    const Grid& gf = op.g;
    cplx<T> acc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = mk<T>(0, 0);
    const int z0 = gf.dim == 3 ? -1 : 0, z1 = gf.dim == 3 ? 1 : 0;
    for (int dz = z0; dz <= z1; ++dz) {
        int fz = gf.dim == 3 ? 2 * z + dz : 0;
        if (fz < 0 || fz >= gf.n3) continue;
        T wz = dz == 0 ? T(1) : T(0.5);
        for (int dy = -1; dy <= 1; ++dy) {
            int fy = 2 * y + dy;
            if (fy < 0 || fy >= gf.n2) continue;
            T wy = dy == 0 ? wz : T(0.5) * wz;
            for (int dx = -1; dx <= 1; ++dx) {
                int fx = 2 * x + dx;
                if (fx < 0 || fx >= gf.n1) continue;
                T wgt = dx == 0 ? wy : T(0.5) * wy;
                long long i = gf.index(fx, fy, fz);
                CV<FT, R> fv = ldR<FT, R>(f + i * s + r0);
                cplx<T> Au[R];
                if (u != nullptr) op.template applyR<R>(u, i, fx, fy, fz, s, r0, Au);
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    cplx<T> ri = cvt<T>(fv.v[k]);
                    if (u != nullptr) ri = ri - Au[k];
                    acc[k] = acc[k] + wgt * ri;
                }
            }
        }
    }
    CV<T, R> o;
#pragma unroll
    for (int k = 0; k < R; ++k) o.v[k] = acc[k];
    stR<T, R>(rc + e0, o);
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_prolong_add_v(Grid gf, Grid gc, const cplx<T>* __restrict__ ec,
                                                        cplx<T>* __restrict__ u, int s) {
    VGEO_PROLOGUE(gf)
    int xs[2], ys[2], zs[2];
    int nx = (x & 1) ? 2 : 1, ny = (y & 1) ? 2 : 1, nz = (gf.dim == 3 && (z & 1)) ? 2 : 1;
    xs[0] = x >> 1; xs[1] = (x >> 1) + 1;
    ys[0] = y >> 1; ys[1] = (y >> 1) + 1;
    zs[0] = z >> 1; zs[1] = (z >> 1) + 1;
    T wgt = T(1);
    if (nx == 2) wgt *= T(0.5);
    if (ny == 2) wgt *= T(0.5);
    if (nz == 2) wgt *= T(0.5);
    cplx<T> acc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = mk<T>(0, 0);
    for (int c = 0; c < nz; ++c)
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) {
                CV<T, R> v = ldR<T, R>(ec + gc.index(xs[a], ys[b], zs[c]) * s + r0);
#pragma unroll
                for (int k = 0; k < R; ++k) acc[k] = acc[k] + v.v[k];
            }
    CV<T, R> uv = ldR<T, R>(u + e0);
#pragma unroll
    for (int k = 0; k < R; ++k) uv.v[k] = uv.v[k] + wgt * acc[k];
    stR<T, R>(u + e0, uv);
}

// u = Minv f: tiled complex GEMM (n x n) * (n x s), 32 x 32 output tile per
// block, 16-deep k tiles staged in shared memory, 4 outputs per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_dense_apply(const cplx<T>* __restrict__ A, int n,
                                                      const cplx<T>* __restrict__ B,
                                                      cplx<T>* __restrict__ C, int s) {
    constexpr int TM = 32, TN = 32, TK = 16;
    __shared__ cplx<T> As[TM][TK + 1];
    __shared__ cplx<T> Bs[TK][TN];
    const int tid = threadIdx.x;
    const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
    const int tc = tid % TN;       // output column within the tile
    const int tr = tid / TN;       // 0..7: rows tr, tr+8, tr+16, tr+24
    cplx<T> acc[4];
    for (int q = 0; q < 4; ++q) acc[q] = mk<T>(0, 0);
    for (int k0 = 0; k0 < n; k0 += TK) {
        for (int idx = tid; idx < TM * TK; idx += 256) {
            int rr = idx / TK, kk = idx % TK;
            int gr = row0 + rr, gk = k0 + kk;
            As[rr][kk] = (gr < n && gk < n) ? ldg(A + (long long)gr * n + gk) : mk<T>(0, 0);
        }
        for (int idx = tid; idx < TK * TN; idx += 256) {
            int kk = idx / TN, cc = idx % TN;
            int gk = k0 + kk, gc = col0 + cc;
            Bs[kk][cc] = (gk < n && gc < s) ? ldg(B + (long long)gk * s + gc) : mk<T>(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            cplx<T> bv = Bs[kk][tc];
#pragma unroll
            for (int q = 0; q < 4; ++q) fma_acc(acc[q], As[tr + 8 * q][kk], bv);
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        int gr = row0 + tr + 8 * q, gc = col0 + tc;
        if (gr < n && gc < s) C[(long long)gr * s + gc] = acc[q];
    }
}

// ---------------- set-up ----------------

__global__ void k_fine_setup(Grid g, const double* __restrict__ m, const double* __restrict__ gam,
                             double omega, double shift, double inv_h2, c128* cA, c128* cM,
                             c128* dinvM, c128* coefM) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    double w2m = omega * omega * m[i];  // set-up: plain FP64 arithmetic
    c128 a = mk(w2m, -w2m * gam[i]);
    c128 b = mk(w2m, -w2m * (gam[i] + shift));
    cA[i] = a;
    cM[i] = b;
    c128 d = mk(2.0 * g.dim * inv_h2 - b.re, -b.im);
    double den = d.re * d.re + d.im * d.im;
    dinvM[i] = mk(d.re / den, -d.im / den);
    const int K = g.dim == 3 ? 27 : 9;
    int x, y, z;
    g.coords(i, x, y, z);
    c128* cf = coefM + i * K;
    for (int o = 0; o < K; ++o) cf[o] = mk(0.0, 0.0);
    int ctr = g.dim == 3 ? 13 : 4;
    cf[ctr] = d;
    if (x > 0) cf[ctr - 1] = mk(-inv_h2, 0.0);
    if (x < g.n1 - 1) cf[ctr + 1] = mk(-inv_h2, 0.0);
    if (y > 0) cf[ctr - 3] = mk(-inv_h2, 0.0);
    if (y < g.n2 - 1) cf[ctr + 3] = mk(-inv_h2, 0.0);
    if (g.dim == 3) {
        if (z > 0) cf[ctr - 9] = mk(-inv_h2, 0.0);
        if (z < g.n3 - 1) cf[ctr + 9] = mk(-inv_h2, 0.0);
    }
}

__device__ __forceinline__ double p1(int d) { return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0); }

// coef_c[J][o] = sum_{i in supp P_J} P_iJ sum_t M[i][t] P_{i+t, J+o}
__global__ void k_galerkin(Grid gf, Grid gc, const c128* __restrict__ cf, c128* __restrict__ cc) {
    const int K = gf.dim == 3 ? 27 : 9;
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= gc.N * K) return;
    long long J = e / K;
    int o = (int)(e - J * K);
    int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = gf.dim == 3 ? o / 9 - 1 : 0;
    int jx, jy, jz;
    gc.coords(J, jx, jy, jz);
    int kx = jx + ox, ky = jy + oy, kz = jz + oz;   // coarse neighbour J + o
    c128 acc = mk(0.0, 0.0);
    if (kx >= 0 && kx < gc.n1 && ky >= 0 && ky < gc.n2 && kz >= 0 && kz < gc.n3) {
        const int dzlo = gf.dim == 3 ? -1 : 0, dzhi = gf.dim == 3 ? 1 : 0;
        for (int dz = dzlo; dz <= dzhi; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int ix = 2 * jx + dx, iy = 2 * jy + dy, iz = gf.dim == 3 ? 2 * jz + dz : 0;
                    if (ix < 0 || ix >= gf.n1 || iy < 0 || iy >= gf.n2 || iz < 0 || iz >= gf.n3)
                        continue;
                    double wi = p1(dx) * p1(dy) * p1(dz);
                    const c128* row = cf + gf.index(ix, iy, iz) * K;
                    for (int tz = dzlo; tz <= dzhi; ++tz)
                        for (int ty = -1; ty <= 1; ++ty)
                            for (int tx = -1; tx <= 1; ++tx) {
                                int fx = ix + tx, fy = iy + ty, fz = iz + tz;
                                double wk = p1(fx - 2 * kx) * p1(fy - 2 * ky) *
                                            (gf.dim == 3 ? p1(fz - 2 * kz) : 1.0);
                                if (wk == 0.0) continue;
                                if (fx < 0 || fx >= gf.n1 || fy < 0 || fy >= gf.n2 || fz < 0 ||
                                    fz >= gf.n3)
                                    continue;
                                int t = (tx + 1) + 3 * (ty + 1) + (gf.dim == 3 ? 9 * (tz + 1) : 0);
                                c128 mv = row[t];
                                acc.re += wi * wk * mv.re;
                                acc.im += wi * wk * mv.im;
                            }
                }
    }
    cc[e] = acc;
}

__global__ void k_diag_inv(Grid g, const c128* __restrict__ coef, c128* __restrict__ dinv) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const int K = g.dim == 3 ? 27 : 9;
    c128 d = coef[i * K + (K / 2)];
    double den = d.re * d.re + d.im * d.im;
    dinv[i] = mk(d.re / den, -d.im / den);
}

__global__ void k_stencil_to_dense(Grid g, const c128* __restrict__ coef, c128* __restrict__ D) {
    const int K = g.dim == 3 ? 27 : 9;
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= g.N * K) return;
    long long i = e / K;
    int o = (int)(e - i * K);
    int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = g.dim == 3 ? o / 9 - 1 : 0;
    int x, y, z;
    g.coords(i, x, y, z);
    x += ox; y += oy; z += oz;
    if (x < 0 || x >= g.n1 || y < 0 || y >= g.n2 || z < 0 || z >= g.n3) return;
    D[i * g.N + g.index(x, y, z)] = coef[e];
}

// Gauss-Jordan kernels, templated on the arithmetic (double for the FP64
// inverse of the plain solver, float for the complex64 cycle, whose tensor-
// core solve rounds the inverse to tf32 anyway).
template <typename T>
__global__ void k_aug_init(const c128* __restrict__ dense, cplx<T>* aug, int n) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    long long i = e / n, j = e - i * n;
    aug[i * 2 * n + j] = cvt<T>(dense[e]);
    aug[i * 2 * n + n + j] = mk<T>(i == j ? T(1) : T(0), T(0));
}

// One block: pivot row p = argmax_{i>=k} |aug[i][k]|; factor[i] = entry of
// column k in row i after the swap of rows k and p (factor[k] = 0).
template <typename T>
__global__ void __launch_bounds__(1024) k_gj_pivot(cplx<T>* aug, int n, int k, cplx<T>* factor,
                                                   int* piv, cplx<T>* pivval, int* status) {
    __shared__ T sval[1024];
    __shared__ int sidx[1024];
    const long long ld = 2LL * n;
    T best = T(-1);
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        cplx<T> a = aug[i * ld + k];
        T v = a.re * a.re + a.im * a.im;
        if (v > best) { best = v; bi = i; }
    }
    sval[threadIdx.x] = best;
    sidx[threadIdx.x] = bi;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            T o = sval[threadIdx.x + w];
            int oi = sidx[threadIdx.x + w];
            if (o > sval[threadIdx.x] || (o == sval[threadIdx.x] && oi < sidx[threadIdx.x])) {
                sval[threadIdx.x] = o;
                sidx[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    int p = sidx[0];
    if (threadIdx.x == 0) {
        *piv = p;
        *pivval = aug[(long long)p * ld + k];
        if (!(sval[0] > T(0))) *status = 1;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        cplx<T> v;
        if (i == k) v = mk<T>(0, 0);
        else if (i == p) v = aug[(long long)k * ld + k];
        else v = aug[(long long)i * ld + k];
        factor[i] = v;
    }
}

template <typename T>
__global__ void k_gj_swap_scale(cplx<T>* aug, int n, int k, const int* piv, const cplx<T>* pivval) {
    int j = k + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 2 * n) return;
    const long long ld = 2LL * n;
    int p = *piv;
    cplx<T> pv = *pivval;
    T den = pv.re * pv.re + pv.im * pv.im;
    cplx<T> inv = den > T(0) ? mk<T>(pv.re / den, -pv.im / den) : mk<T>(0, 0);
    cplx<T> a = aug[(long long)k * ld + j];
    cplx<T> b = aug[(long long)p * ld + j];
    if (p != k) aug[(long long)p * ld + j] = a;
    aug[(long long)k * ld + j] = inv * b;
}

template <typename T>
__global__ void k_gj_eliminate(cplx<T>* aug, int n, int k, const cplx<T>* __restrict__ factor) {
    const long long ld = 2LL * n;
    int j = k + blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j >= 2 * n || i == k) return;
    cplx<T> f = factor[i];
    if (f.re == T(0) && f.im == T(0)) return;
    cplx<T> rk = aug[(long long)k * ld + j];
    cplx<T> v = aug[(long long)i * ld + j];
    aug[(long long)i * ld + j] = v - f * rk;
}

template <typename T>
__global__ void k_extract_inverse(const cplx<T>* aug, int n, c128* out) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    long long i = e / n, j = e - i * n;
    cplx<T> v = aug[i * 2 * n + n + j];
    out[e] = mk<double>((double)v.re, (double)v.im);
}

__global__ void k_round_c64(const c128* in, c64* out, long long count) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < count) out[e] = mk(__double2float_rn(in[e].re), __double2float_rn(in[e].im));
}

}  // namespace

template <typename T>
__global__ void k_axpy(cplx<T>* __restrict__ y, const cplx<T>* __restrict__ x, long long n) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < n) y[e] = y[e] + ldg(x + e);
}

// K-cycle helpers: out[j] += sum_node conj(a[node][j]) b[node][j] (double
// accumulation; s <= 256: thread t takes column t % s), and
// y[node][j] += sign * (num_j / den_j) x[node][j].
template <typename T>
__global__ void __launch_bounds__(256) k_coldot(const cplx<T>* __restrict__ a, const cplx<T>* __restrict__ b,
                                                 long long N, int s, double2* __restrict__ out,
                                                 double2* __restrict__ part, unsigned int* __restrict__ count) {
    __shared__ double2 red[256];
    const int per = 256 / s;
    const int j = threadIdx.x % s, sub = threadIdx.x / s;
    double re = 0.0, im = 0.0;
    if (sub < per)
        for (long long n = (long long)blockIdx.x * per + sub; n < N; n += (long long)gridDim.x * per) {
            cplx<T> x = a[n * s + j], y = b[n * s + j];
            re += (double)x.re * y.re + (double)x.im * y.im;
            im += (double)x.re * y.im - (double)x.im * y.re;
        }
    red[threadIdx.x] = make_double2(sub < per ? re : 0.0, sub < per ? im : 0.0);
    __syncthreads();
    // per-CTA sums, then the last CTA to finish adds them in block order (the
    // result does not depend on scheduling); it also resets the counter
    __shared__ bool last;
    if (sub == 0) {
        double tr = 0.0, ti = 0.0;
        for (int k = 0; k < per; ++k) { tr += red[k * s + j].x; ti += red[k * s + j].y; }
        part[(long long)blockIdx.x * s + j] = make_double2(tr, ti);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int jj = threadIdx.x; jj < s; jj += blockDim.x) {
        double tr = 0.0, ti = 0.0;
        for (unsigned int bk = 0; bk < gridDim.x; ++bk) {
            const double2 v = part[(long long)bk * s + jj];
            tr += v.x;
            ti += v.y;
        }
        out[jj] = make_double2(tr, ti);
    }
    if (threadIdx.x == 0) *count = 0u;
}

template <typename T>
__global__ void k_kc_axpy(cplx<T>* __restrict__ y, const cplx<T>* __restrict__ x,
                          const double2* __restrict__ num, const double2* __restrict__ den,
                          double sign, long long N, int s) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= N * s) return;
    int j = (int)(e % s);
    double d = den[j].x;
    if (!(d > 0.0)) return;
    cplx<T> c = mk<T>((T)(sign * num[j].x / d), (T)(sign * num[j].y / d));
    y[e] = y[e] + c * x[e];
}

// ---------------- launchers ----------------
//
// Each launcher reports the launch's algorithmic traffic and flops to the
// profiler: every vector element read or written once, coefficients once per
// node, no cache effects.  E = N s elements; b* = bytes of one complex value.

template <typename T>
constexpr double cb() { return 2.0 * sizeof(T); }

template <typename Op> struct OpCost;
template <typename T> struct OpCost<FineOp<T>> {
    static double coef_bytes(const FineOp<T>&) { return cb<T>(); }          // c per node
    static double flops(const FineOp<T>& op) { return 4.0 * op.g.dim + 12.0; }
    static constexpr bool fine = true;
};
template <typename T> struct OpCost<GalOp<T>> {
    static double K(const GalOp<T>& op) { return op.g.dim == 3 ? 27.0 : 9.0; }
    static double coef_bytes(const GalOp<T>& op) { return K(op) * cb<T>(); }
    static double flops(const GalOp<T>& op) { return 8.0 * K(op); }
    static constexpr bool fine = false;
};

void launch_apply_dd(const Launch& L, const Grid& g, double inv_h2, const float4* cdd, const c64* x,
                     c64* y, int s) {
    long long total = g.N * s;
    L.pre(KID_APPLY_FINE, total * (8.0 + 16.0) + g.N * 16.0, total * (g.dim == 3 ? 22.0 : 18.0));
    const float ih = (float)inv_h2;
    const float il = (float)(inv_h2 - (double)ih);
    Geo G = geo_for(g, s);
    if (G.R == 2) k_apply_dd<2><<<G.grid, G.block, 0, L.st>>>(g, ih, il, cdd, x, y, s);
    else k_apply_dd<1><<<G.grid, G.block, 0, L.st>>>(g, ih, il, cdd, x, y, s);
    L.post();
}

template <typename T, typename U, typename V, typename Op>
void launch_apply(const Launch& L, const Op& op, const cplx<U>* x, cplx<V>* y, int s) {
    long long total = op.g.N * s;
    L.pre(OpCost<Op>::fine ? KID_APPLY_FINE : KID_APPLY_COARSE,
          total * (cb<U>() + cb<V>()) + op.g.N * OpCost<Op>::coef_bytes(op),
          total * OpCost<Op>::flops(op));
    Geo G = geo_for(op.g, s);
    if (G.ok && G.R == 2) k_apply_v<T, U, V, Op, 2><<<G.grid, G.block, 0, L.st>>>(op, x, y, s);
    else if (G.ok) k_apply_v<T, U, V, Op, 1><<<G.grid, G.block, 0, L.st>>>(op, x, y, s);
    else k_apply<T, U, V, Op><<<blocks_for(total), kThreads, 0, L.st>>>(op, x, y, s, total);
    L.post();
}

template <typename T, typename Op>
void launch_residual(const Launch& L, const Op& op, const cplx<T>* x, const cplx<T>* b,
                     cplx<T>* r, int s) {
    long long total = op.g.N * s;
    L.pre(KID_RESIDUAL, total * 3 * cb<T>() + op.g.N * OpCost<Op>::coef_bytes(op),
          total * (OpCost<Op>::flops(op) + 2));
    k_residual<T, Op><<<blocks_for(total), kThreads, 0, L.st>>>(op, x, b, r, s, total);
    L.post();
}

template <typename T, typename FT, typename Op>
void launch_jacobi(const Launch& L, const Op& op, const cplx<T>* u_in, const cplx<FT>* f,
                   cplx<T>* u_out, int s, T w) {
    long long total = op.g.N * s;
    double bytes, flops;
    if (u_in == nullptr) {
        bytes = total * (cb<FT>() + cb<T>()) + op.g.N * cb<T>();
        flops = total * 8.0;
    } else {
        bytes = total * (cb<FT>() + 2 * cb<T>()) + op.g.N * (OpCost<Op>::coef_bytes(op) + cb<T>());
        flops = total * (OpCost<Op>::flops(op) + 12.0);
    }
    L.pre(OpCost<Op>::fine ? KID_JACOBI_FINE : KID_JACOBI_COARSE, bytes, flops);
    Geo G = geo_for(op.g, s);
    if (G.ok && G.R == 2) k_jacobi_v<T, FT, Op, 2><<<G.grid, G.block, 0, L.st>>>(op, u_in, f, u_out, s, w);
    else if (G.ok) k_jacobi_v<T, FT, Op, 1><<<G.grid, G.block, 0, L.st>>>(op, u_in, f, u_out, s, w);
    else k_jacobi<T, FT, Op><<<blocks_for(total), kThreads, 0, L.st>>>(op, u_in, f, u_out, s, w, total);
    L.post();
}

template <typename T, typename FT, typename Op>
void launch_resid_restrict(const Launch& L, const Op& op, const Grid& gc, const cplx<T>* u,
                           const cplx<FT>* f, cplx<T>* rc, int s) {
    long long total = gc.N * s;
    double ef = (double)op.g.N * s;
    double bytes = ef * (cb<FT>() + (u ? cb<T>() : 0.0)) + total * cb<T>() +
                   op.g.N * OpCost<Op>::coef_bytes(op);
    double flops = ef * ((u ? OpCost<Op>::flops(op) : 0.0) + 2.0) + total * 2.0 * (op.g.dim == 3 ? 27 : 9);
    L.pre(OpCost<Op>::fine ? KID_RESTRICT_FINE : KID_RESTRICT_COARSE, bytes, flops);
    Geo G = geo_for(gc, s);
    if (G.ok && G.R == 2)
        k_resid_restrict_v<T, FT, Op, 2><<<G.grid, G.block, 0, L.st>>>(op, gc, u, f, rc, s);
    else if (G.ok)
        k_resid_restrict_v<T, FT, Op, 1><<<G.grid, G.block, 0, L.st>>>(op, gc, u, f, rc, s);
    else
        k_resid_restrict<T, FT, Op><<<blocks_for(total), kThreads, 0, L.st>>>(op, gc, u, f, rc, s, total);
    L.post();
}

template <typename T>
void launch_coldot(const Launch& L, const cplx<T>* a, const cplx<T>* b, long long N, int s,
                   double2* out, double2* part, unsigned int* count) {
    L.pre(KID_LAYOUT, 2.0 * N * s * cb<T>(), 8.0 * N * s);
    long long want = (N + 255) / 256;
    long long cap = 2LL * sm_count();
    if (cap > kColdotBlocks) cap = kColdotBlocks;
    k_coldot<T><<<(unsigned)(want < cap ? (want < 1 ? 1 : want) : cap), 256, 0, L.st>>>(
        a, b, N, s, out, part, count);
    L.post();
}

template <typename T>
void launch_kc_axpy(const Launch& L, cplx<T>* y, const cplx<T>* x, const double2* num,
                    const double2* den, double sign, long long N, int s) {
    L.pre(KID_LAYOUT, 3.0 * N * s * cb<T>(), 8.0 * N * s);
    k_kc_axpy<T><<<blocks_for(N * s), kThreads, 0, L.st>>>(y, x, num, den, sign, N, s);
    L.post();
}

template <typename T>
void launch_axpy(const Launch& L, cplx<T>* y, const cplx<T>* x, long long n) {
    L.pre(KID_PROLONG, n * 3.0 * cb<T>(), n * 2.0);
    k_axpy<T><<<blocks_for(n), kThreads, 0, L.st>>>(y, x, n);
    L.post();
}

template <typename T>
void launch_prolong_add(const Launch& L, const Grid& gf, const Grid& gc, const cplx<T>* ec,
                        cplx<T>* u, int s) {
    long long total = gf.N * s;
    L.pre(KID_PROLONG, total * 2 * cb<T>() + (double)gc.N * s * cb<T>(),
          total * 2.0 * (gf.dim == 3 ? 8 : 4));
    Geo G = geo_for(gf, s);
    if (G.ok && G.R == 2) k_prolong_add_v<T, 2><<<G.grid, G.block, 0, L.st>>>(gf, gc, ec, u, s);
    else if (G.ok) k_prolong_add_v<T, 1><<<G.grid, G.block, 0, L.st>>>(gf, gc, ec, u, s);
    else k_prolong_add<T><<<blocks_for(total), kThreads, 0, L.st>>>(gf, gc, ec, u, s, total);
    L.post();
}

template <typename T>
void launch_dense_apply(const Launch& L, const cplx<T>* Minv, int n, const cplx<T>* f, cplx<T>* u,
                        int s) {
    dim3 grid((s + 31) / 32, (n + 31) / 32);
    L.pre(KID_DENSE, (double)n * n * cb<T>() + 2.0 * n * s * cb<T>(), 8.0 * n * (double)n * s);
    k_dense_apply<T><<<grid, 256, 0, L.st>>>(Minv, n, f, u, s);
    L.post();
}

void launch_fine_setup(const Launch& L, const Grid& g, const double* m, const double* gamma,
                       double omega, double shift, double inv_h2, c128* cA, c128* cM,
                       c128* dinvM, c128* coefM) {
    L.pre(KID_SETUP, 0, 0);
    k_fine_setup<<<blocks_for(g.N), kThreads, 0, L.st>>>(g, m, gamma, omega, shift, inv_h2, cA, cM,
                                                         dinvM, coefM);
    L.post();
}

void launch_galerkin(const Launch& L, const Grid& gf, const Grid& gc, const c128* coef_f,
                     c128* coef_c) {
    const int K = gf.dim == 3 ? 27 : 9;
    L.pre(KID_SETUP, 0, 0);
    k_galerkin<<<blocks_for(gc.N * K), kThreads, 0, L.st>>>(gf, gc, coef_f, coef_c);
    L.post();
}

void launch_diag_inv(const Launch& L, const Grid& g, const c128* coef, c128* dinv) {
    L.pre(KID_SETUP, 0, 0);
    k_diag_inv<<<blocks_for(g.N), kThreads, 0, L.st>>>(g, coef, dinv);
    L.post();
}

void launch_stencil_to_dense(const Launch& L, const Grid& g, const c128* coef, c128* dense) {
    const int K = g.dim == 3 ? 27 : 9;
    cudaMemsetAsync(dense, 0, sizeof(c128) * g.N * g.N, L.st);
    L.pre(KID_SETUP, 0, 0);
    k_stencil_to_dense<<<blocks_for(g.N * K), kThreads, 0, L.st>>>(g, coef, dense);
    L.post();
}

template <typename T>
void launch_gauss_jordan(const Launch& L, const c128* dense, void* aug_raw, int n, void* factor_raw,
                         int* piv, void* pivval_raw, int* status, c128* inverse) {
    cplx<T>* aug = static_cast<cplx<T>*>(aug_raw);
    cplx<T>* factor = static_cast<cplx<T>*>(factor_raw);
    cplx<T>* pivval = static_cast<cplx<T>*>(pivval_raw);
    L.pre(KID_SETUP, 0, 0);
    k_aug_init<T><<<blocks_for((long long)n * n), kThreads, 0, L.st>>>(dense, aug, n);
    L.post();
    for (int k = 0; k < n; ++k) {
        L.pre(KID_SETUP, 0, 0);
        k_gj_pivot<T><<<1, 1024, 0, L.st>>>(aug, n, k, factor, piv, pivval, status);
        L.post();
        int cols = 2 * n - k;
        L.pre(KID_SETUP, 0, 0);
        k_gj_swap_scale<T><<<(cols + 255) / 256, 256, 0, L.st>>>(aug, n, k, piv, pivval);
        L.post();
        dim3 grid((cols + 255) / 256, n);
        L.pre(KID_SETUP, 0, 0);
        k_gj_eliminate<T><<<grid, 256, 0, L.st>>>(aug, n, k, factor);
        L.post();
    }
    L.pre(KID_SETUP, 0, 0);
    k_extract_inverse<T><<<blocks_for((long long)n * n), kThreads, 0, L.st>>>(aug, n, inverse);
    L.post();
}
template void launch_gauss_jordan<double>(const Launch&, const c128*, void*, int, void*, int*, void*,
                                          int*, c128*);
template void launch_gauss_jordan<float>(const Launch&, const c128*, void*, int, void*, int*, void*,
                                         int*, c128*);

void launch_round_c64(const Launch& L, const c128* in, c64* out, long long count) {
    L.pre(KID_LAYOUT, count * (16.0 + 8.0), 0);
    k_round_c64<<<blocks_for(count), kThreads, 0, L.st>>>(in, out, count);
    L.post();
}

// ---------------- explicit instantiations ----------------

#define HELM_INST_T(T)                                                                           \
    template void launch_apply<T, T, T, FineOp<T>>(const Launch&, const FineOp<T>&,              \
                                                   const cplx<T>*, cplx<T>*, int);               \
    template void launch_apply<T, T, T, GalOp<T>>(const Launch&, const GalOp<T>&,                \
                                                  const cplx<T>*, cplx<T>*, int);                \
    template void launch_residual<T, FineOp<T>>(const Launch&, const FineOp<T>&, const cplx<T>*, \
                                                const cplx<T>*, cplx<T>*, int);                  \
    template void launch_jacobi<T, T, FineOp<T>>(const Launch&, const FineOp<T>&,                \
                                                 const cplx<T>*, const cplx<T>*, cplx<T>*, int,  \
                                                 T);                                             \
    template void launch_jacobi<T, T, GalOp<T>>(const Launch&, const GalOp<T>&, const cplx<T>*,  \
                                                const cplx<T>*, cplx<T>*, int, T);               \
    template void launch_resid_restrict<T, T, FineOp<T>>(const Launch&, const FineOp<T>&,        \
                                                         const Grid&, const cplx<T>*,            \
                                                         const cplx<T>*, cplx<T>*, int);         \
    template void launch_resid_restrict<T, T, GalOp<T>>(const Launch&, const GalOp<T>&,          \
                                                        const Grid&, const cplx<T>*,             \
                                                        const cplx<T>*, cplx<T>*, int);          \
    template void launch_prolong_add<T>(const Launch&, const Grid&, const Grid&, const cplx<T>*, \
                                        cplx<T>*, int);                                          \
    template void launch_axpy<T>(const Launch&, cplx<T>*, const cplx<T>*, long long);            \
    template void launch_coldot<T>(const Launch&, const cplx<T>*, const cplx<T>*, long long, int, \
                                   double2*, double2*, unsigned int*);                           \
    template void launch_kc_axpy<T>(const Launch&, cplx<T>*, const cplx<T>*, const double2*,      \
                                    const double2*, double, long long, int);                    \
    template void launch_residual<T, GalOp<T>>(const Launch&, const GalOp<T>&, const cplx<T>*,   \
                                               const cplx<T>*, cplx<T>*, int);                   \
    template void launch_dense_apply<T>(const Launch&, const cplx<T>*, int, const cplx<T>*,      \
                                        cplx<T>*, int);

HELM_INST_T(float)
HELM_INST_T(double)
// complex64 cycle fed by a complex128 right-hand side (the Krylov basis)
template void launch_jacobi<float, double, FineOp<float>>(const Launch&, const FineOp<float>&,
                                                          const cplx<float>*, const cplx<double>*,
                                                          cplx<float>*, int, float);
template void launch_jacobi<float, double, GalOp<float>>(const Launch&, const GalOp<float>&,
                                                         const cplx<float>*, const cplx<double>*,
                                                         cplx<float>*, int, float);
template void launch_resid_restrict<float, double, FineOp<float>>(const Launch&,
                                                                  const FineOp<float>&,
                                                                  const Grid&, const cplx<float>*,
                                                                  const cplx<double>*,
                                                                  cplx<float>*, int);
template void launch_resid_restrict<float, double, GalOp<float>>(const Launch&,
                                                                 const GalOp<float>&, const Grid&,
                                                                 const cplx<float>*,
                                                                 const cplx<double>*,
                                                                 cplx<float>*, int);
// outer A Z with Z in complex64, W in complex128 (FP64 arithmetic)
template void launch_apply<double, float, double, FineOp<double>>(const Launch&,
                                                                  const FineOp<double>&,
                                                                  const cplx<float>*,
                                                                  cplx<double>*, int);

}  // namespace helm
