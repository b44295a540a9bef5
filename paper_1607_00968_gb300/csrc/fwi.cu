// Kernels of the FWI sensitivity products (Sec. 2.4 Eq. fwisens, receiver
// sampling Eq. data, 16-bit field storage as in Sec. 2.4).
//
// With A(m) = -Lap_h - w^2 diag(m (1 - i g)):  J = du/dm = w^2 A^{-1}
// diag((1 - i g) u), so  P^T J v = (A^{-1} (dAdm u v))[recv]  and
// J^T w = sum_sources Re(conj(dAdm u) lambda),  lambda = A^{-H} P w,
// dAdm = w^2 (1 - i g).  Fields are in the ABI layout (column j = source j,
// N contiguous values), complex128 or 16-bit pairs (half re, half im).
#include <cuda_fp16.h>

#include "kernels.h"

namespace helm {

namespace {

constexpr int kT = 256;

inline unsigned nblk(long long n) { return (unsigned)((n + kT - 1) / kT); }

__device__ __forceinline__ c128 field_at(const void* f, int half, long long e) {
    if (half) {
        __half2 h = reinterpret_cast<const __half2*>(f)[e];
        return mk((double)__half2float(h.x), (double)__half2float(h.y));
    }
    return reinterpret_cast<const c128*>(f)[e];
}

__global__ void k_dadm(const double* __restrict__ gamma, double omega, long long N, c128* __restrict__ d) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < N) d[k] = mk(omega * omega, -omega * omega * gamma[k]);
}

__global__ void k_to_half(const c128* __restrict__ u, long long n, __half2* __restrict__ o) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < n) o[e] = __floats2half2_rn((float)u[e].re, (float)u[e].im);
}

__global__ void k_jv_rhs(const void* __restrict__ f, int half, long long N, int s,
                         const c128* __restrict__ dadm, const double* __restrict__ v,
                         c128* __restrict__ rhs) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= N * s) return;
    long long k = e % N;
    rhs[e] = v[k] * (dadm[k] * field_at(f, half, e));
}

// out[j][r] = X[j][recv[r]] (- d[j][r] when d is given)
__global__ void k_gather(const c128* __restrict__ X, long long N, int s, const int* __restrict__ recv,
                         int nrec, const c128* __restrict__ d, c128* __restrict__ out) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)nrec * s) return;
    int j = (int)(e / nrec), r = (int)(e - (long long)j * nrec);
    c128 v = X[(long long)j * N + recv[r]];
    if (d) v = v - d[e];
    out[e] = v;
}

// out[j][recv[r]] += W[j][r] (out zeroed by the caller; repeated receivers add)
__global__ void k_scatter(const c128* __restrict__ W, long long N, int s, const int* __restrict__ recv,
                          int nrec, c128* __restrict__ out) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)nrec * s) return;
    int j = (int)(e / nrec), r = (int)(e - (long long)j * nrec);
    c128 w = W[e];
    double* o = reinterpret_cast<double*>(out + (long long)j * N + recv[r]);
    atomicAdd(o, w.re);
    atomicAdd(o + 1, w.im);
}

// g[k] = sum_j Re(conj(dAdm_k u_jk) lambda_jk)
__global__ void k_grad(const void* __restrict__ f, int half, const c128* __restrict__ lam, long long N,
                       int s, const c128* __restrict__ dadm, double* __restrict__ g) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= N) return;
    c128 d = dadm[k];
    double acc = 0.0;
    for (int j = 0; j < s; ++j) {
        c128 a = d * field_at(f, half, (long long)j * N + k);
        c128 l = lam[(long long)j * N + k];
        acc += a.re * l.re + a.im * l.im;
    }
    g[k] = acc;
}

}  // namespace

void launch_dadm(const Launch& L, const double* gamma, double omega, long long N, c128* dadm) {
    L.pre(KID_SETUP, 0, 0);
    k_dadm<<<nblk(N), kT, 0, L.st>>>(gamma, omega, N, dadm);
    L.post();
}

void launch_to_half(const Launch& L, const c128* u, long long n, void* u16) {
    L.pre(KID_LAYOUT, 20.0 * n, 0);
    k_to_half<<<nblk(n), kT, 0, L.st>>>(u, n, static_cast<__half2*>(u16));
    L.post();
}

void launch_jv_rhs(const Launch& L, const void* fields, int half, long long N, int s, const c128* dadm,
                   const double* v, c128* rhs) {
    L.pre(KID_LAYOUT, (double)N * s * ((half ? 4.0 : 16.0) + 16.0), 14.0 * N * s);
    k_jv_rhs<<<nblk(N * s), kT, 0, L.st>>>(fields, half, N, s, dadm, v, rhs);
    L.post();
}

void launch_gather(const Launch& L, const c128* X, long long N, int s, const int* recv, int nrec,
                   const c128* d, c128* out) {
    L.pre(KID_LAYOUT, 48.0 * nrec * s, 0);
    k_gather<<<nblk((long long)nrec * s), kT, 0, L.st>>>(X, N, s, recv, nrec, d, out);
    L.post();
}

void launch_scatter(const Launch& L, const c128* W, long long N, int s, const int* recv, int nrec,
                    c128* out) {
    cudaMemsetAsync(out, 0, sizeof(c128) * (size_t)N * s, L.st);
    L.pre(KID_LAYOUT, 32.0 * nrec * s, 0);
    k_scatter<<<nblk((long long)nrec * s), kT, 0, L.st>>>(W, N, s, recv, nrec, out);
    L.post();
}

void launch_grad(const Launch& L, const void* fields, int half, const c128* lam, long long N, int s,
                 const c128* dadm, double* g) {
    L.pre(KID_LAYOUT, (double)N * s * ((half ? 4.0 : 16.0) + 16.0), 8.0 * N * s);
    k_grad<<<nblk(N), kT, 0, L.st>>>(fields, half, lam, N, s, dadm, g);
    L.post();
}

}  // namespace helm
