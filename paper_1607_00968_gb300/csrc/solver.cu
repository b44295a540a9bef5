// libhelm host driver: set-up of the shifted-Laplacian hierarchy, the
// multigrid cycle and block FGMRES (Sec. 4 and Sec. 5.3 of Treister & Haber),
// behind the C-ABI declared in include/helm.h.
//
// Work split: every N-sized step (stencils, transfers, coarsest solve, Gram
// products, block updates, norms, layout changes) runs in the kernels of
// mg.cu / krylov.cu on the context's stream; the host keeps only the
// block-sized dense algebra of the Krylov method (s_b x s_b Cholesky factors
// and the block-Hessenberg least-squares problem, a few kB), in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <thread>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/helm.h"
#include "kernels.h"

using helm::c128;
using helm::c64;
using helm::cplx;
using helm::Grid;
using helm::Launch;
using cd = std::complex<double>;

namespace {

thread_local std::string g_thread_error;

// A block column is dependent when its part orthogonal to the columns before
// it has a sine below kDepAngle, or is below kDepRoundoff times the column's
// norm before any orthogonalisation (same reading as the oracle).  The block
// QR is a Cholesky QR, whose pivot for a column of sine t carries a relative
// rounding error of about u / t^2: on the float-pair path (u = 2^-46) the
// sine threshold is raised to 64 sqrt(u) = 7.6e-6, so that no column the
// Cholesky factor cannot resolve is kept (measured: the restart blocks of 32
// residuals on the 3D workload reach sines of 1e-5 .. 1e-7 as their columns
// converge, and Cholesky factors of such blocks in float-pair arithmetic
// broke the basis).
constexpr double kDepAngle = 1e-7;
constexpr double kDepRoundoff = 1e-12;

// Orthogonalisation with orth = 0: one Gram-Schmidt pass and one Cholesky QR
// pass, each repeated only when its rounding could leave the new basis block
// less orthogonal than kOrthTarget.  One classical Gram-Schmidt pass leaves
// components along the old basis of about u / sin(theta) of the column
// (theta: its angle to the old basis), which the Cholesky QR multiplies by
// at most kappa(W'); one Cholesky QR pass leaves an orthogonality error of
// about u kappa(W')^2.  u is the unit roundoff of the Gram and update
// arithmetic: 2^-53 in FP64, 2^-46 for the float-pair (double-float) kernels.
constexpr double kOrthTarget = 1e-11;

struct Level {
    Grid g;
    c128* coef = nullptr;    // K-point stencil of M_l (FP64)
    c128* dinv = nullptr;    // Jacobi inverse diagonal of M_l (FP64)
    c64* coef32 = nullptr;
    c64* dinv32 = nullptr;
    // cycle work buffers, N_l x s_cap complex128-sized (complex64 uses half)
    void* u0 = nullptr;
    void* u1 = nullptr;
    void* e = nullptr;       // coarse-level solution (levels >= 1)
    void* f = nullptr;       // coarse-level right-hand side (levels >= 1)
    void* wf = nullptr;      // W-cycle: residual and correction of the second
    void* we = nullptr;      // coarse visit (levels >= 1)
    void* kb[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // K-cycle: z1 w1 r2 z2 w2
    double2* kd = nullptr;   // K-cycle column products (6 x s)
};

}  // namespace

// Per-launch CUDA-event profiler (enabled by helm_profile_enable): every
// launcher records an event pair around its kernel on the context's stream,
// with the launch's algorithmic bytes and flops; helm_profile_read resolves
// the pairs and accumulates per kernel class.
namespace helm {
struct Profiler {
    struct Rec { int kid; double bytes, flops; cudaEvent_t a, b; };
    std::vector<Rec> open;
    std::vector<cudaEvent_t> pool;
    double time_ms[KID_COUNT] = {};
    double bytes[KID_COUNT] = {};
    double flops[KID_COUNT] = {};
    long long launches[KID_COUNT] = {};
    int only = -1;       // record one kernel class only (-1: all)
    bool armed = false;  // the current launch is being recorded

    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    void resolve() {
        for (auto& r : open) {
            cudaEventSynchronize(r.b);
            float ms = 0;
            cudaEventElapsedTime(&ms, r.a, r.b);
            time_ms[r.kid] += ms;
            bytes[r.kid] += r.bytes;
            flops[r.kid] += r.flops;
            launches[r.kid] += 1;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        open.clear();
    }
    void reset() {
        resolve();
        for (int k = 0; k < KID_COUNT; ++k) time_ms[k] = bytes[k] = flops[k] = 0, launches[k] = 0;
    }
    ~Profiler() {
        resolve();
        for (auto e : pool) cudaEventDestroy(e);
    }
};

void prof_begin(Profiler* p, cudaStream_t st, int kid, double bytes, double flops) {
    p->armed = p->only < 0 || kid == p->only;
    if (!p->armed) return;
    Profiler::Rec r{kid, bytes, flops, p->get(), p->get()};
    cudaEventRecord(r.a, st);
    p->open.push_back(r);
    if (p->open.size() > 4096) {  // bound the number of events in flight
        cudaEventRecord(r.b, st);
        p->open.back().b = r.b;
    }
}

void prof_end(Profiler* p, cudaStream_t st) {
    if (!p->armed || p->open.empty()) return;
    p->armed = false;
    cudaEventRecord(p->open.back().b, st);
    if (p->open.size() > 4096) p->resolve();
}
}  // namespace helm

struct helm_ctx {
    helm_params p{};
    cudaStream_t st = nullptr;
    long long launches = 0;
    std::string err;
    double inv_h2 = 0;
    std::vector<Level> lv;
    // fine-level mass coefficients of A and M
    c128* cA = nullptr;
    c128* cM = nullptr;
    c64* cA32 = nullptr;
    float4* cAdd = nullptr;   // c_A as float pairs (double-float A Z)
    c64* cM32 = nullptr;
    // coarsest inverse
    int nc = 0;
    c128* Minv = nullptr;
    c64* Minv32 = nullptr;
    float* Ap = nullptr;      // tf32-rounded interleaved inverse for the tensor-core solve
    float* dense_scratch = nullptr;
    c128* dadm = nullptr;     // omega^2 (1 - i gamma) per node (FWI sensitivities)
    // learned stage
    float* kappa = nullptr;   // omega^2 m h^2 per node
    c64* lr_r = nullptr;      // residual of the cycle's result
    float* lr_rho2 = nullptr;
    float* lr_rho = nullptr;
    void* lr_x0 = nullptr;    // bf16 network input, 16 channels
    void* lr_act[2] = {nullptr, nullptr};  // bf16 activations, 32 channels
    float* lr_out = nullptr;  // float network output, 16 channels
    c64* lr_z2 = nullptr;     // corrected block before the acceptance test
    float* lr_rho_new = nullptr;
    // Krylov workspace, sized for s_cap columns
    int s_cap = 0;
    c128* V = nullptr;       // (restart+1) blocks of N x s
    void* Z = nullptr;       // restart blocks (complex128 or complex64)
    c128* W = nullptr;
    c128* W2 = nullptr;
    c128* Bint = nullptr;
    c128* X = nullptr;
    c128* R = nullptr;
    c128* abi_in = nullptr;  // device staging for helm_solve_host
    c128* abi_out = nullptr;
    c128* partial = nullptr;
    long long partial_elems = 0;
    c128* small = nullptr;   // device small matrices (H passes, G, T, Y)
    long long small_elems = 0;
    int* dmask = nullptr;
    float4* csplit = nullptr; // split (float pair) coefficients of the dd block updates
    c128* hsmall = nullptr;  // pinned host mirror of `small`
    // counter of the generator that draws replacement directions for
    // dependent columns (rank rule); every solve starts it at the same value
    unsigned long long rng_counter = 0x5eed;
    helm::Profiler* prof = nullptr;
    // CUDA graphs of the FGMRES step (one per (s, j)), captured on a private
    // stream and replayed on `st`; they hold workspace pointers, so they are
    // destroyed with the workspace
    struct StepGraph { int s, j; cudaGraphExec_t exec; long long launches; };
    std::vector<StepGraph> graphs;
    cudaStream_t cap_st = nullptr;
    // storage format of the FGMRES basis V, W and W2 during a solve:
    // helm::FMT_DD (unevaluated float pairs) on the complex64 path when the
    // double-float kernels cover the block shape, else complex128
    int kfmt = 0;
    // K-cycle: per-CTA partial column products and the completion counter
    double2* kpart = nullptr;
    unsigned int* kcount = nullptr;
    // orthogonalisation counters (helm_orth_stats): block QRs factored, and
    // how many of them needed a second Gram-Schmidt / Cholesky QR pass
    long long orth_qr = 0, orth_reorth = 0, orth_qr2 = 0;

    Launch L() { return Launch{st, &launches, prof}; }
    long long N() const { return lv[0].g.N; }
};

namespace {

}  // namespace

void helm::set_thread_error(const std::string& msg) { g_thread_error = msg; }

namespace {

helm_status fail(helm_ctx* c, helm_status s, const std::string& msg) {
    if (c) c->err = msg;
    g_thread_error = msg;
    return s;
}

#define CUDA_TRY(ctx, expr)                                                            \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? HELM_ERR_NOMEM : HELM_ERR_CUDA, \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));           \
    } while (0)

// A failed allocation is reported through the return value only: the
// runtime's pending error is cleared, so that the next cudaGetLastError (the
// check at the end of a later call) does not report it a second time.
template <typename P>
cudaError_t dalloc(P** p, size_t bytes) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
    }
    return e;
}

template <typename P>
cudaError_t halloc_pinned(P** p, size_t bytes) {
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(p), bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
    }
    return e;
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

// ---------------------------------------------------------------------------
// operators
// ---------------------------------------------------------------------------

template <typename T> const cplx<T>* pick(const c128* d, const c64* f);
template <> const cplx<double>* pick<double>(const c128* d, const c64*) { return d; }
template <> const cplx<float>* pick<float>(const c128*, const c64* f) { return f; }

template <typename T>
helm::FineOp<T> fine_op(const helm_ctx* c, bool shifted) {
    helm::FineOp<T> op;
    op.g = c->lv[0].g;
    op.inv_h2 = (T)c->inv_h2;
    op.c = shifted ? pick<T>(c->cM, c->cM32) : pick<T>(c->cA, c->cA32);
    op.dinv = pick<T>(c->lv[0].dinv, c->lv[0].dinv32);
    return op;
}

template <typename T>
helm::GalOp<T> gal_op(const helm_ctx* c, int l) {
    helm::GalOp<T> op;
    op.g = c->lv[l].g;
    op.coef = pick<T>(c->lv[l].coef, c->lv[l].coef32);
    op.dinv = pick<T>(c->lv[l].dinv, c->lv[l].dinv32);
    return op;
}

// ---------------------------------------------------------------------------
// multigrid cycle (Alg. "Two-grid cycle", applied recursively = V-cycle)
// ---------------------------------------------------------------------------

template <typename T, typename FT>
void smooth_level(helm_ctx* c, int l, const cplx<T>* uin, const cplx<FT>* f, cplx<T>* uout,
                  int s) {
    T w = (T)c->p.jacobi_w;
    if (l == 0)
        helm::launch_jacobi<T, FT, helm::FineOp<T>>(c->L(), fine_op<T>(c, true), uin, f, uout, s, w);
    else
        helm::launch_jacobi<T, FT, helm::GalOp<T>>(c->L(), gal_op<T>(c, l), uin, f, uout, s, w);
}

template <typename T, typename FT>
void restrict_level(helm_ctx* c, int l, const cplx<T>* u, const cplx<FT>* f, cplx<T>* rc, int s) {
    if (l == 0)
        helm::launch_resid_restrict<T, FT, helm::FineOp<T>>(c->L(), fine_op<T>(c, true),
                                                            c->lv[1].g, u, f, rc, s);
    else
        helm::launch_resid_restrict<T, FT, helm::GalOp<T>>(c->L(), gal_op<T>(c, l), c->lv[l + 1].g,
                                                           u, f, rc, s);
}

template <typename T>
void coarsest(helm_ctx* c, const cplx<T>* f, cplx<T>* u, int s) {
    if constexpr (std::is_same<T, float>::value)
        helm::launch_dense_tc(c->L(), c->Ap, c->nc, f, u, s, c->dense_scratch, c->p.coarse_tf32x3);
    else
        helm::launch_dense_apply<T>(c->L(), c->Minv, c->nc, f, u, s);
}

template <typename T, typename FT>
void cycle(helm_ctx* c, int l, const cplx<FT>* f, cplx<T>* out, int s);

// K-cycle coarse correction on level k (Sec. 5.3 "K-cycles": two iterations
// of a flexible Krylov method, preconditioned by level k's cycle, on the
// coarse system), per column as GCR(2):
//   z1 = C(r), w1 = M z1, a1 = w1^H r / w1^H w1, r2 = r - a1 w1,
//   z2 = C(r2), w2 = M z2, b = w1^H w2 / w1^H w1, w2 -= b w1, z2 -= b z1,
//   a2 = w2^H r2 / w2^H w2, e = a1 z1 + a2 z2.
// The column products stay on the device (no host synchronisation).
template <typename T>
void kcycle_correction(helm_ctx* c, int k, const cplx<T>* r, cplx<T>* e, int s) {
    Level& lev = c->lv[k];
    const long long n = lev.g.N * (long long)s;
    cplx<T>* z1 = reinterpret_cast<cplx<T>*>(lev.kb[0]);
    cplx<T>* w1 = reinterpret_cast<cplx<T>*>(lev.kb[1]);
    cplx<T>* r2 = reinterpret_cast<cplx<T>*>(lev.kb[2]);
    cplx<T>* z2 = reinterpret_cast<cplx<T>*>(lev.kb[3]);
    cplx<T>* w2 = reinterpret_cast<cplx<T>*>(lev.kb[4]);
    double2 *d11 = lev.kd, *d1r = lev.kd + s, *d12 = lev.kd + 2 * s, *d22 = lev.kd + 3 * s,
            *d2r = lev.kd + 4 * s;
    helm::GalOp<T> op = gal_op<T>(c, k);
    cycle<T, T>(c, k, r, z1, s);
    helm::launch_apply<T, T, T, helm::GalOp<T>>(c->L(), op, z1, w1, s);
    helm::launch_coldot<T>(c->L(), w1, w1, lev.g.N, s, d11, c->kpart, c->kcount);
    helm::launch_coldot<T>(c->L(), w1, r, lev.g.N, s, d1r, c->kpart, c->kcount);
    cudaMemcpyAsync(r2, r, sizeof(cplx<T>) * n, cudaMemcpyDeviceToDevice, c->st);
    helm::launch_kc_axpy<T>(c->L(), r2, w1, d1r, d11, -1.0, lev.g.N, s);
    cycle<T, T>(c, k, r2, z2, s);
    helm::launch_apply<T, T, T, helm::GalOp<T>>(c->L(), op, z2, w2, s);
    helm::launch_coldot<T>(c->L(), w1, w2, lev.g.N, s, d12, c->kpart, c->kcount);
    helm::launch_kc_axpy<T>(c->L(), w2, w1, d12, d11, -1.0, lev.g.N, s);
    helm::launch_kc_axpy<T>(c->L(), z2, z1, d12, d11, -1.0, lev.g.N, s);
    helm::launch_coldot<T>(c->L(), w2, w2, lev.g.N, s, d22, c->kpart, c->kcount);
    helm::launch_coldot<T>(c->L(), w2, r2, lev.g.N, s, d2r, c->kpart, c->kcount);
    helm::launch_zero(c->L(), e, sizeof(cplx<T>) * n);
    helm::launch_kc_axpy<T>(c->L(), e, z1, d1r, d11, 1.0, lev.g.N, s);
    helm::launch_kc_axpy<T>(c->L(), e, z2, d2r, d22, 1.0, lev.g.N, s);
}

// out = cycle(f) on level l with zero initial guess.  `out` must not alias the
// level's own work buffers.
template <typename T, typename FT>
void cycle(helm_ctx* c, int l, const cplx<FT>* f, cplx<T>* out, int s) {
    const int Lv = (int)c->lv.size();
    Level& lev = c->lv[l];
    if (l == Lv - 1) {
        if constexpr (std::is_same<T, FT>::value) {
            coarsest<T>(c, f, out, s);
        } else {
            // one-level hierarchy with a complex128 right-hand side: round it first
            cplx<T>* tmp = reinterpret_cast<cplx<T>*>(lev.u0);
            helm::launch_round_c64(c->L(), reinterpret_cast<const c128*>(f),
                                   reinterpret_cast<c64*>(tmp), lev.g.N * (long long)s);
            coarsest<T>(c, tmp, out, s);
        }
        return;
    }
    cplx<T>* bufA = reinterpret_cast<cplx<T>*>(lev.u0);
    cplx<T>* bufB = reinterpret_cast<cplx<T>*>(lev.u1);
    const cplx<T>* cur = nullptr;
    for (int k = 0; k < c->p.pre; ++k) {
        cplx<T>* dst = (k % 2 == 0) ? bufA : bufB;
        smooth_level<T, FT>(c, l, cur, f, dst, s);
        cur = dst;
    }
    Level& nxt = c->lv[l + 1];
    cplx<T>* fc = reinterpret_cast<cplx<T>*>(nxt.f);
    cplx<T>* ec = reinterpret_cast<cplx<T>*>(nxt.e);
    restrict_level<T, FT>(c, l, cur, f, fc, s);
    if (c->p.cycle_gamma == 3 && l + 1 < Lv - 1)
        kcycle_correction<T>(c, l + 1, fc, ec, s);
    else
        cycle<T, T>(c, l + 1, fc, ec, s);
    if (c->p.cycle_gamma == 2 && l + 1 < Lv - 1) {
        // W-cycle (Sec. 4: two recursive calls): a second coarse visit on the
        // residual of the first, ec += cycle(fc - M_{l+1} ec)
        cplx<T>* wf = reinterpret_cast<cplx<T>*>(nxt.wf);
        cplx<T>* we = reinterpret_cast<cplx<T>*>(nxt.we);
        helm::launch_residual<T, helm::GalOp<T>>(c->L(), gal_op<T>(c, l + 1), ec, fc, wf, s);
        cycle<T, T>(c, l + 1, wf, we, s);
        helm::launch_axpy<T>(c->L(), ec, we, nxt.g.N * (long long)s);
    }
    cplx<T>* u = const_cast<cplx<T>*>(cur);
    if (u == nullptr) {
        u = bufA;
        helm::launch_zero(c->L(), u, sizeof(cplx<T>) * lev.g.N * s);
    }
    helm::launch_prolong_add<T>(c->L(), lev.g, nxt.g, ec, u, s);
    cur = u;
    if (c->p.post == 0) {
        cudaMemcpyAsync(out, cur, sizeof(cplx<T>) * lev.g.N * s, cudaMemcpyDeviceToDevice, c->st);
        return;
    }
    for (int k = 0; k < c->p.post; ++k) {
        cplx<T>* dst = (k == c->p.post - 1) ? out : (cur == bufA ? bufB : bufA);
        smooth_level<T, FT>(c, l, cur, f, dst, s);
        cur = dst;
    }
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------

void free_workspace(helm_ctx* c) {
    dfree(c->kpart);
    dfree(c->kcount);
    c->kpart = nullptr;
    c->kcount = nullptr;
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
    for (auto& l : c->lv) {
        dfree(l.u0); dfree(l.u1); dfree(l.e); dfree(l.f); dfree(l.wf); dfree(l.we);
        l.u0 = l.u1 = l.e = l.f = l.wf = l.we = nullptr;
        for (auto& q : l.kb) { dfree(q); q = nullptr; }
        dfree(l.kd);
        l.kd = nullptr;
    }
    dfree(c->V); dfree(c->Z); dfree(c->W); dfree(c->W2); dfree(c->Bint); dfree(c->X);
    dfree(c->R); dfree(c->abi_in); dfree(c->abi_out); dfree(c->partial); dfree(c->small);
    dfree(c->dmask);
    dfree(c->csplit);
    c->csplit = nullptr;
    dfree(c->dense_scratch);
    c->dense_scratch = nullptr;
    dfree(c->lr_r); dfree(c->lr_rho2); dfree(c->lr_rho); dfree(c->lr_x0);
    dfree(c->lr_act[0]); dfree(c->lr_act[1]); dfree(c->lr_out);
    dfree(c->lr_z2); dfree(c->lr_rho_new);
    c->lr_z2 = nullptr; c->lr_rho_new = nullptr;
    c->lr_r = nullptr; c->lr_rho2 = c->lr_rho = nullptr; c->lr_x0 = nullptr;
    c->lr_act[0] = c->lr_act[1] = nullptr; c->lr_out = nullptr;
    if (c->hsmall) cudaFreeHost(c->hsmall);
    c->V = c->W = c->W2 = c->Bint = c->X = c->R = c->abi_in = c->abi_out = c->partial = c->small =
        nullptr;
    c->Z = nullptr;
    c->dmask = nullptr;
    c->hsmall = nullptr;
    c->s_cap = 0;
}

helm_status ensure_workspace(helm_ctx* c, int s) {
    if (c->p.cycle_gamma == 3 && s > 256)
        return fail(c, HELM_ERR_ARG, "the K-cycle takes at most 256 columns per block");
    if (s <= c->s_cap) return HELM_OK;
    free_workspace(c);
    const long long N = c->N();
    const size_t vec = sizeof(c128) * (size_t)N * s;
    const int m = c->p.restart;
    for (size_t l = 0; l < c->lv.size(); ++l) {
        size_t b = sizeof(c128) * (size_t)c->lv[l].g.N * s;
        CUDA_TRY(c, dalloc(&c->lv[l].u0, b));
        CUDA_TRY(c, dalloc(&c->lv[l].u1, b));
        if (l > 0) {
            CUDA_TRY(c, dalloc(&c->lv[l].e, b));
            CUDA_TRY(c, dalloc(&c->lv[l].f, b));
            if (c->p.cycle_gamma == 2) {
                CUDA_TRY(c, dalloc(&c->lv[l].wf, b));
                CUDA_TRY(c, dalloc(&c->lv[l].we, b));
            }
            if (c->p.cycle_gamma == 3) {
                for (int q = 0; q < 5; ++q) CUDA_TRY(c, dalloc(&c->lv[l].kb[q], b));
                CUDA_TRY(c, dalloc(&c->lv[l].kd, sizeof(double2) * 6 * (size_t)s));
            }
        }
    }
    const size_t zel = c->p.prec == HELM_PLAIN_C128 ? sizeof(c128) : sizeof(c64);
    // block BiCGSTAB keeps six FP64 blocks (R, P, V, S, T, shadow) in V and
    // two preconditioned blocks in Z
    CUDA_TRY(c, dalloc(&c->V, vec * std::max(m + 1, 6)));
    CUDA_TRY(c, dalloc(&c->Z, zel * (size_t)N * s * std::max(m, 2)));
    CUDA_TRY(c, dalloc(&c->W, vec));
    CUDA_TRY(c, dalloc(&c->W2, vec));
    CUDA_TRY(c, dalloc(&c->Bint, vec));
    CUDA_TRY(c, dalloc(&c->X, vec));
    CUDA_TRY(c, dalloc(&c->R, vec));
    const int sb = std::min(c->p.block, s);
    const int G = (s + sb - 1) / sb;
    long long pe = std::max(helm::gram_partial_elems(N, m + 1, s, sb),
                            helm::colnorm_partial_elems(N, s));
    pe = std::max(pe, helm::gram_partial_elems(N, 1, s, sb));
    c->partial_elems = pe;
    CUDA_TRY(c, dalloc(&c->partial, sizeof(c128) * pe));
    CUDA_TRY(c, cudaMemsetAsync(c->partial, 0, (size_t)helm::gram_scratch_zero_bytes(), c->st));
    // small: 2 H passes + G + T + Y + norms
    long long blk = (long long)G * sb * sb;
    c->small_elems = std::max(2 * (m + 1) * blk + 2 * blk + (long long)m * blk, 10 * blk) + 4LL * s + 64;
    CUDA_TRY(c, dalloc(&c->small, sizeof(c128) * c->small_elems));
    CUDA_TRY(c, halloc_pinned(&c->hsmall, sizeof(c128) * c->small_elems));
    CUDA_TRY(c, dalloc(&c->dmask, sizeof(int) * s));
    CUDA_TRY(c, dalloc(&c->csplit, sizeof(float4) * (size_t)(m + 1) * blk));
    CUDA_TRY(c, dalloc(&c->dense_scratch, sizeof(float) * helm::dense_tc_scratch_floats(c->nc, s)));
    if (c->p.prec == HELM_MIXED_C64_LEARNED) {
        CUDA_TRY(c, dalloc(&c->lr_r, sizeof(c64) * (size_t)N * s));
        CUDA_TRY(c, dalloc(&c->lr_rho2, sizeof(float) * s));
        CUDA_TRY(c, dalloc(&c->lr_rho, sizeof(float) * s));
        CUDA_TRY(c, dalloc(&c->lr_x0, 2 * 16 * (size_t)N * s));
        CUDA_TRY(c, dalloc(&c->lr_act[0], 2 * 32 * (size_t)N * s));
        CUDA_TRY(c, dalloc(&c->lr_act[1], 2 * 32 * (size_t)N * s));
        CUDA_TRY(c, dalloc(&c->lr_out, 4 * 16 * (size_t)N * s));
        CUDA_TRY(c, dalloc(&c->lr_z2, sizeof(c64) * (size_t)N * s));
        CUDA_TRY(c, dalloc(&c->lr_rho_new, sizeof(float) * s));
    }
    if (c->p.cycle_gamma == 3) {
        CUDA_TRY(c, dalloc(&c->kpart, sizeof(double2) * helm::kColdotBlocks * (size_t)s));
        CUDA_TRY(c, dalloc(&c->kcount, sizeof(unsigned int)));
        CUDA_TRY(c, cudaMemsetAsync(c->kcount, 0, sizeof(unsigned int), c->st));
    }
    c->s_cap = s;
    return HELM_OK;
}

// ---------------------------------------------------------------------------
// small dense algebra on the host (FP64)
// ---------------------------------------------------------------------------

// Cholesky of one group's Gram matrix G (n x n, row-major, Hermitian) with the
// dependence test; R upper triangular (row-major), T = R^{-1} on the
// independent columns (zero rows/columns for dependent ones).
bool chol_dep(const cd* G, const double* ref2, int n, std::vector<cd>& R, std::vector<cd>& T,
              std::vector<int>& dep, bool allow_dep, double dep_angle = kDepAngle) {
    R.assign((size_t)n * n, 0.0);
    T.assign((size_t)n * n, 0.0);
    dep.assign(n, 0);
    for (int k = 0; k < n; ++k) {
        double gkk = G[k * n + k].real();
        double d = gkk;
        for (int i = 0; i < k; ++i) d -= std::norm(R[i * n + k]);
        bool dependent = !(gkk > 0.0) || !(d > dep_angle * dep_angle * gkk) ||
                         (ref2 && !(d > kDepRoundoff * kDepRoundoff * ref2[k]));
        if (dependent) {
            if (!allow_dep) return false;
            dep[k] = 1;
            continue;
        }
        double rkk = std::sqrt(d);
        R[k * n + k] = rkk;
        for (int l = k + 1; l < n; ++l) {
            cd v = G[k * n + l];
            for (int i = 0; i < k; ++i) v -= std::conj(R[i * n + k]) * R[i * n + l];
            R[k * n + l] = v / rkk;
        }
    }
    // T = R^{-1} restricted to the independent index set
    for (int l = 0; l < n; ++l) {
        if (dep[l]) continue;
        T[l * n + l] = 1.0 / R[l * n + l];
        for (int i = l - 1; i >= 0; --i) {
            if (dep[i]) continue;
            cd v = 0.0;
            for (int t = i + 1; t <= l; ++t)
                if (!dep[t]) v += R[i * n + t] * T[t * n + l];
            T[i * n + l] = -v / R[i * n + i];
        }
    }
    return true;
}

// Incrementally QR-factorised block Hessenberg least-squares problem of one
// group: min_Y || E_1 Lambda - Hbar_j Y ||_F, by Householder reflections
// applied to each new block column as it arrives.
struct BlockLS {
    int sb = 0, m = 0;
    int rows = 0;                      // (m+1) sb
    std::vector<cd> Rm;                // rows x (m sb), column-major
    std::vector<cd> gv;                // rows x sb, column-major
    std::vector<std::vector<cd>> refl; // per step: sb vectors of length 2 sb
    std::vector<std::vector<double>> beta;

    void init(int sb_, int m_, const std::vector<cd>& Lam /* sb x sb row-major */) {
        sb = sb_; m = m_; rows = (m + 1) * sb;
        Rm.assign((size_t)rows * m * sb, 0.0);
        gv.assign((size_t)rows * sb, 0.0);
        for (int a = 0; a < sb; ++a)
            for (int b = 0; b < sb; ++b) gv[(size_t)b * rows + a] = Lam[a * sb + b];
        refl.assign(m, {});
        beta.assign(m, {});
    }

    static void apply_refl(const cd* v, double bt, int len, cd* y) {
        if (bt == 0.0) return;
        cd d = 0.0;
        for (int t = 0; t < len; ++t) d += std::conj(v[t]) * y[t];
        d *= bt;
        for (int t = 0; t < len; ++t) y[t] -= v[t] * d;
    }

    // hcol: (j+2) sb x sb, column-major with leading dimension `ld`.
    // Returns per-column residual estimates.
    std::vector<double> add(int j, std::vector<cd>& hcol, int ld) {
        const int L2 = 2 * sb;
        for (int i = 0; i < j; ++i)
            for (int c = 0; c < sb; ++c)
                for (int q = 0; q < sb; ++q)
                    apply_refl(&refl[i][(size_t)q * L2], beta[i][q], L2, &hcol[(size_t)c * ld + i * sb]);
        refl[j].assign((size_t)sb * L2, 0.0);
        beta[j].assign(sb, 0.0);
        for (int q = 0; q < sb; ++q) {
            cd* x = &hcol[(size_t)q * ld + j * sb];  // rows j sb .. j sb + 2sb - 1 of column q
            double nrm2 = 0;
            for (int t = q; t < L2; ++t) nrm2 += std::norm(x[t]);
            double nrm = std::sqrt(nrm2);
            cd* v = &refl[j][(size_t)q * L2];
            if (nrm == 0.0) { beta[j][q] = 0.0; continue; }
            cd x0 = x[q];
            cd alpha = (std::abs(x0) > 0) ? -x0 / std::abs(x0) * nrm : cd(-nrm, 0.0);
            for (int t = q; t < L2; ++t) v[t] = x[t];
            v[q] -= alpha;
            double vn2 = 0;
            for (int t = q; t < L2; ++t) vn2 += std::norm(v[t]);
            beta[j][q] = vn2 > 0 ? 2.0 / vn2 : 0.0;
            for (int c = q; c < sb; ++c) apply_refl(v, beta[j][q], L2, &hcol[(size_t)c * ld + j * sb]);
        }
        for (int c = 0; c < sb; ++c)
            for (int q = 0; q < sb; ++q)
                apply_refl(&refl[j][(size_t)q * L2], beta[j][q], L2, &gv[(size_t)c * rows + j * sb]);
        for (int c = 0; c < sb; ++c)
            for (int r = 0; r < (j + 1) * sb; ++r)
                Rm[(size_t)(j * sb + c) * rows + r] = hcol[(size_t)c * ld + r];
        std::vector<double> est(sb);
        for (int c = 0; c < sb; ++c) {
            double e2 = 0;
            for (int r = (j + 1) * sb; r < (j + 2) * sb; ++r) e2 += std::norm(gv[(size_t)c * rows + r]);
            est[c] = std::sqrt(e2);
        }
        return est;
    }

    // Y ((j+1) sb x sb, row-major [row][col]) from the first j+1 block steps.
    std::vector<cd> solve(int j) const {
        const int n = (j + 1) * sb;
        std::vector<cd> Y((size_t)n * sb, 0.0);
        double dmax = 0;
        for (int r = 0; r < n; ++r) dmax = std::max(dmax, std::abs(Rm[(size_t)r * rows + r]));
        for (int c = 0; c < sb; ++c)
            for (int r = n - 1; r >= 0; --r) {
                cd v = gv[(size_t)c * rows + r];
                for (int t = r + 1; t < n; ++t) v -= Rm[(size_t)t * rows + r] * Y[(size_t)t * sb + c];
                cd d = Rm[(size_t)r * rows + r];
                Y[(size_t)r * sb + c] = (std::abs(d) > 1e-14 * dmax) ? v / d : cd(0.0);
            }
        return Y;
    }
};

// ---------------------------------------------------------------------------
// block QR (CholQR2 with the dependence rule) of W against the basis V_0..V_{nb-1}
// ---------------------------------------------------------------------------

struct QRResult {
    std::vector<std::vector<cd>> R;  // per group, sb x sb row-major
};

helm_status sync(helm_ctx* c) {
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    CUDA_TRY(c, cudaGetLastError());
    return HELM_OK;
}

// sync(), then report a tcgen05 coarsest product (complex64 cycle, default
// product) that gave up waiting on its pipeline during the call
helm_status sync_checked(helm_ctx* c) {
    helm_status st = sync(c);
    if (st != HELM_OK) return st;
    if (c->p.coarse_tf32x3 == 0 && helm::dense_tc_take_error(c->st))
        return fail(c, HELM_ERR_CUDA, "coarsest tensor-core product: a pipeline wait gave up after 1 s, "
                                      "or its tensor maps could not be built");
    return HELM_OK;
}

// Layout of c->small (elements of c128):
//   [0, 2*(m+1)*blk)        H of the two Gram-Schmidt passes
//   [oG, oG+blk)            Gram of the block being factorised
//   [oT, oT+blk)            T factors uploaded by the host
//   [oY, oY+m*blk)          least-squares solutions Y
//   [oN, oN+4s)             column norms
struct SmallLayout {
    long long blk, oH1, oH2, oG, oT, oY, oN;
};

SmallLayout small_layout(const helm_ctx* c, int s, int sb) {
    SmallLayout L;
    int G = (s + sb - 1) / sb;
    L.blk = (long long)G * sb * sb;
    L.oH1 = 0;
    L.oH2 = (long long)(c->p.restart + 1) * L.blk;
    L.oG = 2 * L.oH2;
    L.oT = L.oG + L.blk;
    L.oY = L.oT + L.blk;
    L.oN = L.oY + (long long)c->p.restart * L.blk;
    return L;
}

// Gram-Schmidt (two passes) of the block at `W` against V_0..V_{nb-1};
// H1/H2 receive the coefficients of the passes when non-null.
bool emulated(const helm_ctx* c) { return c->p.prec != HELM_PLAIN_C128; }

void cgs2(helm_ctx* c, c128* Wp, int nb, int s, int sb, c128* H1, c128* H2) {
    const long long N = c->N();
    const long long vs = N * s;
    for (int pass = 0; pass < 2; ++pass) {
        c128* H = pass == 0 ? H1 : H2;
        // the first pass may use FP32 products of the hi parts: the second,
        // double-float pass removes their error (its coefficients add to H)
        helm::launch_gram_f(c->L(), c->V, c->kfmt, nb, vs, Wp, c->kfmt, N, s, sb, c->partial, H,
                            emulated(c), pass == 0 && c->kfmt == helm::FMT_DD);
        // the second update's coefficients are the first pass's small error:
        // on the float-pair basis its product may run in FP32 (hi parts)
        helm::launch_combine_f(c->L(), Wp, c->kfmt, 1.0, -1.0, c->V, c->kfmt, nb, vs, H, N, s, sb,
                               emulated(c), c->csplit, pass == 1 && c->kfmt == helm::FMT_DD);
    }
}

// One Gram-Schmidt pass of the block at W against V_0..V_{nb-1} (orth = 0):
// H = V^H W in full FP64-class precision, W -= V H.  A repeated pass's
// coefficients are the rounding error of the first (about u / sin(theta) of
// the column), so on the float-pair basis its update forms the product in
// FP32 from the hi planes and adds it to the pairs exactly.
void gs_pass(helm_ctx* c, c128* Wp, int nb, int s, int sb, c128* H, bool repeat) {
    const long long N = c->N();
    const long long vs = N * s;
    helm::launch_gram_f(c->L(), c->V, c->kfmt, nb, vs, Wp, c->kfmt, N, s, sb, c->partial, H,
                        emulated(c), false);
    helm::launch_combine_f(c->L(), Wp, c->kfmt, 1.0, -1.0, c->V, c->kfmt, nb, vs, H, N, s, sb,
                           emulated(c), c->csplit, repeat && c->kfmt == helm::FMT_DD);
}

// Unit roundoff of the Gram and update arithmetic (see kOrthTarget).
double orth_unit(const helm_ctx* c) { return emulated(c) ? std::ldexp(1.0, -46) : std::ldexp(1.0, -53); }

// Sine below which a block column counts as dependent (see kDepAngle).
double dep_angle(const helm_ctx* c) {
    return c->kfmt == helm::FMT_DD ? std::max(kDepAngle, 64.0 * std::sqrt(orth_unit(c))) : kDepAngle;
}

// kappa_F(R) = ||R||_F ||R^{-1}||_F over the independent columns: an upper
// bound of the 2-norm condition number (at most n times it).
double kappa_f(const std::vector<cd>& R, const std::vector<cd>& T, int n) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < n * n; ++k) { a += std::norm(R[k]); b += std::norm(T[k]); }
    return std::sqrt(a * b);
}

// After one Gram-Schmidt pass (orth = 0): does any group need a second?
// Per group, from the QR Gram G = W'^H W' (already on the host) and ref2
// (the squared norm each column lost to V): sin^2(theta_k) = G_kk /
// (G_kk + ref2_k), and the pass is repeated when u / sin(theta_min) times
// kappa_F(W') exceeds kOrthTarget (a column with no remainder always asks).
bool needs_second_gs(const helm_ctx* c, int s, int sb, const std::vector<double>& ref2) {
    const int G = (s + sb - 1) / sb;
    const SmallLayout SL = small_layout(c, s, sb);
    const cd* hG = reinterpret_cast<const cd*>(c->hsmall + SL.oG);
    const double u = orth_unit(c);
    for (int g = 0; g < G; ++g) {
        const int n = std::min(sb, s - g * sb);
        std::vector<cd> Gg((size_t)n * n);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) Gg[a * n + b] = hG[(size_t)g * sb * sb + a * sb + b];
        double smin2 = 1.0;
        std::vector<double> r2(n, 0.0);
        for (int k = 0; k < n; ++k) {
            const double gkk = Gg[k * n + k].real();
            const double tot = gkk + ref2[g * sb + k];
            if (!(tot > 0.0)) continue;           // zero column: nothing to orthogonalise
            if (!(gkk > 0.0)) return true;
            smin2 = std::min(smin2, gkk / tot);
            r2[k] = tot;
        }
        std::vector<cd> R, T;
        std::vector<int> dep;
        chol_dep(Gg.data(), r2.data(), n, R, T, dep, true, dep_angle(c));
        for (int k = 0; k < n; ++k)
            if (dep[k] && r2[k] > 0.0) return true;
        const double kf = kappa_f(R, T, n);
        if (!(u / std::sqrt(smin2) * kf <= kOrthTarget)) return true;
    }
    return false;
}

// Factor the block at Win (already orthogonal to V_0..V_{nb-1}) as Vout R.
// extra2: per column, the squared norm removed by that orthogonalisation
// (sum of |H_ik|^2), so that extra2 + ||W_k||^2 is the column's squared norm
// before it.  Win is left unchanged.
// First Gram of the block QR, enqueued with its copy to the host.  Split
// from block_qr so that a caller can enqueue it before a synchronisation it
// needs anyway.
helm_status qr_gram_launch(helm_ctx* c, const c128* Win, int wfmt, int s, int sb) {
    SmallLayout SL = small_layout(c, s, sb);
    helm::launch_gram_f(c->L(), Win, wfmt, 1, 0, Win, wfmt, c->N(), s, sb, c->partial, c->small + SL.oG,
                        emulated(c));
    CUDA_TRY(c, cudaMemcpyAsync(c->hsmall + SL.oG, c->small + SL.oG, sizeof(c128) * SL.blk,
                                cudaMemcpyDeviceToHost, c->st));
    return HELM_OK;
}

// Win is in format wfmt; W2 and Vout are in the basis format c->kfmt.
helm_status block_qr(helm_ctx* c, c128* Win, int wfmt, c128* Vout, int nb, int s, int sb,
                     const std::vector<double>& extra2, QRResult& out, bool& any_dep,
                     bool gram_enqueued = false) {
    const long long N = c->N();
    const int G = (s + sb - 1) / sb;
    SmallLayout SL = small_layout(c, s, sb);
    c128* dG = c->small + SL.oG;
    c128* dT = c->small + SL.oT;
    cd* hG = reinterpret_cast<cd*>(c->hsmall + SL.oG);
    cd* hT = reinterpret_cast<cd*>(c->hsmall + SL.oT);
    any_dep = false;
    out.R.assign(G, {});
    std::vector<std::vector<cd>> R1(G), R2(G);
    std::vector<int> mask(s, 0);
    bool second = false;   // a second Cholesky QR pass is needed
    // pass 1
    helm_status st = HELM_OK;
    if (!gram_enqueued) {
        st = qr_gram_launch(c, Win, wfmt, s, sb);
        if (st != HELM_OK) return st;
    }
    st = sync(c);
    if (st != HELM_OK) return st;
    for (int g = 0; g < G; ++g) {
        const int n = std::min(sb, s - g * sb);
        std::vector<cd> Gg((size_t)n * n);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) Gg[a * n + b] = hG[(size_t)g * sb * sb + a * sb + b];
        for (int a = 0; a < n * n; ++a)
            if (!std::isfinite(Gg[a].real()) || !std::isfinite(Gg[a].imag()))
                return fail(c, HELM_ERR_NONFINITE, "non-finite value in the Krylov block");
        std::vector<double> ref2(n);
        for (int k = 0; k < n; ++k) ref2[k] = extra2[g * sb + k] + Gg[k * n + k].real();
        std::vector<cd> T;
        std::vector<int> dep;
        chol_dep(Gg.data(), ref2.data(), n, R1[g], T, dep, true, dep_angle(c));
        for (int a = 0; a < sb; ++a)
            for (int b = 0; b < sb; ++b)
                hT[(size_t)g * sb * sb + a * sb + b] = (a < n && b < n) ? T[a * n + b] : cd(0.0);
        for (int k = 0; k < n; ++k)
            if (dep[k]) { mask[g * sb + k] = 1; any_dep = true; }
        const double kf = kappa_f(R1[g], T, n);
        if (!(orth_unit(c) * kf * kf <= kOrthTarget)) second = true;
    }
    CUDA_TRY(c, cudaMemcpyAsync(dT, hT, sizeof(c128) * SL.blk, cudaMemcpyHostToDevice, c->st));
    c->orth_qr++;
    if (c->p.orth == 0 && !second && !any_dep) {
        // one Cholesky QR pass is accurate enough: Vout = Win R1^{-1}
        helm::launch_combine_f(c->L(), Vout, c->kfmt, 0.0, 1.0, Win, wfmt, 1, 0, dT, N, s, sb, emulated(c),
                               c->csplit);
        for (int g = 0; g < G; ++g) {
            const int n = std::min(sb, s - g * sb);
            std::vector<cd> Rg((size_t)sb * sb, 0.0);
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) Rg[a * sb + b] = R1[g][a * n + b];
            out.R[g] = Rg;
        }
        return HELM_OK;
    }
    c->orth_qr2++;
    helm::launch_combine_f(c->L(), c->W2, c->kfmt, 0.0, 1.0, Win, wfmt, 1, 0, dT, N, s, sb, emulated(c),
                           c->csplit);
    if (any_dep) {
        CUDA_TRY(c, cudaMemcpyAsync(c->dmask, mask.data(), sizeof(int) * s, cudaMemcpyHostToDevice,
                                    c->st));
        helm::launch_fill_random_f(c->L(), c->W2, c->kfmt, N, s, c->dmask, c->rng_counter++);
        if (nb > 0) {
            c128* Hs = c->small + SL.oT;  // scratch; T already consumed
            cgs2(c, c->W2, nb, s, sb, Hs, Hs);
        }
    }
    // pass 2
    helm::launch_gram_f(c->L(), c->W2, c->kfmt, 1, 0, c->W2, c->kfmt, N, s, sb, c->partial, dG,
                        emulated(c));
    CUDA_TRY(c, cudaMemcpyAsync(hG, dG, sizeof(c128) * SL.blk, cudaMemcpyDeviceToHost, c->st));
    st = sync(c);
    if (st != HELM_OK) return st;
    for (int g = 0; g < G; ++g) {
        const int n = std::min(sb, s - g * sb);
        std::vector<cd> Gg((size_t)n * n);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) Gg[a * n + b] = hG[(size_t)g * sb * sb + a * sb + b];
        std::vector<cd> T;
        std::vector<int> dep;
        if (!chol_dep(Gg.data(), nullptr, n, R2[g], T, dep, false))
            return fail(c, HELM_ERR_BREAKDOWN, "block QR: second Cholesky pass failed");
        for (int a = 0; a < sb; ++a)
            for (int b = 0; b < sb; ++b)
                hT[(size_t)g * sb * sb + a * sb + b] = (a < n && b < n) ? T[a * n + b] : cd(0.0);
        // R = R2 R1
        std::vector<cd> Rg((size_t)sb * sb, 0.0);
        for (int a = 0; a < n; ++a)
            for (int b = a; b < n; ++b) {
                cd v = 0.0;
                for (int t = a; t <= b; ++t) v += R2[g][a * n + t] * R1[g][t * n + b];
                Rg[a * sb + b] = v;
            }
        out.R[g] = Rg;
    }
    // The second factor is the identity up to the first pass's orthogonality
    // error.  On the float-pair basis, when |T2 - I| <= 1e-7 everywhere,
    // Vout = W2 + W2 (T2 - I) forms the correction in FP32 from hi parts
    // (error <= ~1e-14 of W2, the double-float class) and adds it exactly.
    bool near_identity = c->kfmt == helm::FMT_DD && sb == 4 && s % 4 == 0;
    for (int g = 0; g < G && near_identity; ++g) {
        const int n = std::min(sb, s - g * sb);
        for (int a = 0; a < n && near_identity; ++a)
            for (int b = 0; b < n; ++b) {
                const cd v = hT[(size_t)g * sb * sb + a * sb + b] - (a == b ? cd(1.0) : cd(0.0));
                if (!(std::abs(v) <= 1e-7)) { near_identity = false; break; }
            }
    }
    if (near_identity)
        for (int g = 0; g < G; ++g)
            for (int a = 0; a < sb; ++a) hT[(size_t)g * sb * sb + a * sb + a] -= cd(1.0);
    CUDA_TRY(c, cudaMemcpyAsync(dT, hT, sizeof(c128) * SL.blk, cudaMemcpyHostToDevice, c->st));
    if (near_identity)
        helm::launch_combine_f(c->L(), Vout, c->kfmt, 1.0, 1.0, c->W2, c->kfmt, 1, 0, dT, N, s, sb,
                               emulated(c), c->csplit, true, c->W2);
    else
        helm::launch_combine_f(c->L(), Vout, c->kfmt, 0.0, 1.0, c->W2, c->kfmt, 1, 0, dT, N, s, sb,
                               emulated(c), c->csplit);
    return HELM_OK;
}

// per-column squared norms of an internal block (FP64), to host
helm_status colnorms(helm_ctx* c, const c128* X, int s, std::vector<double>& out) {
    SmallLayout SL = small_layout(c, s, std::min(c->p.block, s));
    c128* d = c->small + SL.oN;
    helm::launch_colnorm2(c->L(), X, c->N(), s, reinterpret_cast<double*>(c->partial),
                          reinterpret_cast<double*>(d));
    CUDA_TRY(c, cudaMemcpyAsync(c->hsmall + SL.oN, d, sizeof(c128) * s, cudaMemcpyDeviceToHost, c->st));
    helm_status st = sync(c);
    if (st != HELM_OK) return st;
    out.resize(s);
    for (int j = 0; j < s; ++j) out[j] = c->hsmall[SL.oN + j].re;
    return HELM_OK;
}

// ---------------------------------------------------------------------------
// learned stage: z <- z + h^2 rho N(r / rho, kappa), r = v - A z
// ---------------------------------------------------------------------------

struct LearnedLayer { int cin, cout, relu; long long w_off, b_off; };

// Six 3x3 layers, channels padded for the tensor-core tiles: input 3 -> 16
// (Re r, Im r, kappa), 32 hidden channels, output 2 -> 16 (Re e, Im e).
// Blob: all bf16 weights [co][tap][ci] back to back, then the float biases.
const LearnedLayer* learned_table() {
    static LearnedLayer t[6];
    static bool init = false;
    if (!init) {
        const int cin[6] = {16, 32, 32, 32, 32, 32}, cout[6] = {32, 32, 32, 32, 32, 16};
        long long w = 0;
        for (int l = 0; l < 6; ++l) { t[l].cin = cin[l]; t[l].cout = cout[l]; t[l].relu = l < 5; t[l].w_off = w; w += 2LL * cout[l] * 9 * cin[l]; }
        long long b = (w + 255) / 256 * 256;
        for (int l = 0; l < 6; ++l) { t[l].b_off = b; b += 4LL * cout[l]; }
        init = true;
    }
    return t;
}
long long learned_blob_bytes() { return learned_table()[5].b_off + 4LL * 16; }

void learned_stage(helm_ctx* c, const c128* v, c64* z, int s) {
    const long long N = c->N();
    const Grid& g = c->lv[0].g;
    helm::launch_learned_residual(c->L(), fine_op<float>(c, false), v, z, c->lr_r, s, c->lr_rho2, c->lr_rho);
    helm::launch_pack_input(c->L(), c->lr_r, (int)N, s, c->lr_rho, c->kappa, c->lr_x0);
    const unsigned char* blob = static_cast<const unsigned char*>(c->p.learned_weights);
    const LearnedLayer* T = learned_table();
    const void* in = c->lr_x0;
    for (int l = 0; l < 6; ++l) {
        void* out = l == 5 ? static_cast<void*>(c->lr_out) : c->lr_act[l % 2];
        helm::launch_conv3x3(c->L(), in, s, g.n2, g.n1, T[l].cin, blob + T[l].w_off,
                             reinterpret_cast<const float*>(blob + T[l].b_off), T[l].cout, T[l].relu,
                             nullptr, out, l == 5);
        in = out;
    }
    // z2 = z + correction; keep it only for the columns whose residual
    // ||v - A z2|| is below ||v - A z|| (the plain cycle is the fallback)
    cudaMemcpyAsync(c->lr_z2, z, sizeof(c64) * (size_t)N * s, cudaMemcpyDeviceToDevice, c->st);
    helm::launch_unpack_add(c->L(), c->lr_out, (int)N, s, c->lr_rho, (float)(c->p.h * c->p.h), c->lr_z2);
    helm::launch_learned_residual(c->L(), fine_op<float>(c, false), v, c->lr_z2, c->lr_r, s,
                                  c->lr_rho_new, c->lr_rho2 /* receives the new RMS; unused */);
    helm::launch_select_better(c->L(), c->lr_z2, z, N, s, c->lr_rho, c->lr_rho_new);
}

// ---------------------------------------------------------------------------
// block FGMRES (Sec. 5.3)
// ---------------------------------------------------------------------------

// The device work of FGMRES step j, up to the first host synchronisation:
// Z_j = cycle(V_j) [+ learned stage], W = A Z_j, two Gram-Schmidt passes
// against V_0..V_j, the first Gram of the block QR of W, and the copies of
// the Gram-Schmidt coefficients and that Gram to the host.
template <typename ZT>
helm_status fgmres_step_launches(helm_ctx* c, int j, int s, int sb) {
    const long long vs = c->N() * s;
    SmallLayout SL = small_layout(c, s, sb);
    cplx<ZT>* Zj = reinterpret_cast<cplx<ZT>*>(c->Z) + (long long)j * vs;
    bool done = false;
    if constexpr (std::is_same<ZT, float>::value)
        if (c->kfmt == helm::FMT_DD) {
            // V_j as float pairs: the complex64 cycle takes its hi plane (the
            // FP64 value truncated to FP32); W = A Z_j is written as pairs
            cycle<float, float>(c, 0, reinterpret_cast<const c64*>(c->V + (long long)j * vs), Zj, s);
            helm::launch_apply_dd(c->L(), c->lv[0].g, c->inv_h2, c->cAdd, Zj, reinterpret_cast<c64*>(c->W), s);
            done = true;
        }
    if (!done) {
        cycle<ZT, double>(c, 0, c->V + (long long)j * vs, Zj, s);
        if constexpr (std::is_same<ZT, float>::value)
            if (c->p.prec == HELM_MIXED_C64_LEARNED) learned_stage(c, c->V + (long long)j * vs, Zj, s);
        helm::launch_apply<double, ZT, double, helm::FineOp<double>>(c->L(), fine_op<double>(c, false), Zj,
                                                                     c->W, s);
    }
    if (c->p.orth == 1) {
        cgs2(c, c->W, j + 1, s, sb, c->small + SL.oH1, c->small + SL.oH2);
        CUDA_TRY(c, cudaMemcpyAsync(c->hsmall, c->small, sizeof(c128) * 2 * SL.oH2, cudaMemcpyDeviceToHost,
                                    c->st));
    } else {
        gs_pass(c, c->W, j + 1, s, sb, c->small + SL.oH1, false);
        CUDA_TRY(c, cudaMemcpyAsync(c->hsmall, c->small, sizeof(c128) * (j + 1) * SL.blk,
                                    cudaMemcpyDeviceToHost, c->st));
    }
    return qr_gram_launch(c, c->W, c->kfmt, s, sb);
}

bool use_graphs(const helm_ctx* c, int s) {
    if (c->prof || c->p.prec == HELM_MIXED_C64_LEARNED || c->p.graphs == 0) return false;
    return c->p.graphs == 1 || c->N() * (long long)s <= (4LL << 20);
}

// fgmres_step_launches, replayed from a CUDA graph when use_graphs() says so.
// The graph is captured on the context's private stream on first use of
// (s, j) and launched on the context's stream; the launch counter advances
// by the captured kernel count at each replay.
template <typename ZT>
helm_status fgmres_step(helm_ctx* c, int j, int s, int sb) {
    if (!use_graphs(c, s)) return fgmres_step_launches<ZT>(c, j, s, sb);
    for (auto& g : c->graphs)
        if (g.s == s && g.j == j) {
            CUDA_TRY(c, cudaGraphLaunch(g.exec, c->st));
            c->launches += g.launches;
            return HELM_OK;
        }
    if (!c->cap_st) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
    cudaStream_t user = c->st;
    const long long before = c->launches;
    CUDA_TRY(c, cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeRelaxed));
    c->st = c->cap_st;
    helm_status st = fgmres_step_launches<ZT>(c, j, s, sb);
    c->st = user;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_st, &graph);
    const long long captured = c->launches - before;
    c->launches = before;
    if (st != HELM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(c, HELM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(c, HELM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    c->graphs.push_back({s, j, exec, captured});
    CUDA_TRY(c, cudaGraphLaunch(exec, c->st));
    c->launches += captured;
    return HELM_OK;
}

template <typename ZT>
helm_status fgmres_run(helm_ctx* c, int s, double tol, helm_info* info);

template <typename ZT>
helm_status fgmres(helm_ctx* c, int s, double tol, helm_info* info) {
    const int sb = std::min(c->p.block, s);
    c->kfmt = (std::is_same<ZT, float>::value && c->p.prec == HELM_MIXED_C64 && helm::dd_formats_ok(s, sb))
                  ? helm::FMT_DD : helm::FMT_C128;
    helm_status st = fgmres_run<ZT>(c, s, tol, info);
    c->kfmt = helm::FMT_C128;
    return st;
}

template <typename ZT>
helm_status fgmres_run(helm_ctx* c, int s, double tol, helm_info* info) {
    const long long N = c->N();
    const long long vs = N * s;
    const int m = c->p.restart;
    const int sb = std::min(c->p.block, s);
    const int G = (s + sb - 1) / sb;
    SmallLayout SL = small_layout(c, s, sb);
    cplx<ZT>* Z = reinterpret_cast<cplx<ZT>*>(c->Z);
    helm::FineOp<double> opA = fine_op<double>(c, false);

    std::vector<double> bn2;
    helm_status st = colnorms(c, c->Bint, s, bn2);
    if (st != HELM_OK) return st;
    std::vector<double> bn(s);
    for (int j = 0; j < s; ++j) {
        if (!std::isfinite(bn2[j])) return fail(c, HELM_ERR_NONFINITE, "non-finite right-hand side");
        bn[j] = std::sqrt(bn2[j]);
    }
    helm::launch_zero(c->L(), c->X, sizeof(c128) * vs);
    std::vector<int> iters(G, 0);
    std::vector<char> done(G, 0);
    std::vector<double> rel(s, 0.0);
    helm_status result = HELM_NOT_CONVERGED;

    for (int cyc = 0; cyc <= c->p.max_restarts; ++cyc) {
        // true residual R = B - A X in FP64
        if (cyc == 0)
            CUDA_TRY(c, cudaMemcpyAsync(c->R, c->Bint, sizeof(c128) * vs, cudaMemcpyDeviceToDevice, c->st));
        else
            helm::launch_residual<double, helm::FineOp<double>>(c->L(), opA, c->X, c->Bint, c->R, s);
        std::vector<double> rn2;
        st = colnorms(c, c->R, s, rn2);
        if (st != HELM_OK) return st;
        bool all = true;
        for (int j = 0; j < s; ++j) {
            if (!std::isfinite(rn2[j])) {
                result = fail(c, HELM_ERR_NONFINITE, "non-finite residual");
                goto finish;
            }
            rel[j] = bn[j] > 0 ? std::sqrt(rn2[j]) / bn[j] : 0.0;
        }
        for (int g = 0; g < G; ++g) {
            bool ok = true;
            for (int j = g * sb; j < std::min(s, (g + 1) * sb); ++j) ok = ok && rel[j] <= tol;
            done[g] = ok;
            all = all && ok;
        }
        if (all) { result = HELM_OK; break; }
        if (cyc == c->p.max_restarts) { result = HELM_NOT_CONVERGED; break; }

        // V_0 Lambda = R
        QRResult qr;
        bool dep;
        st = block_qr(c, c->R, helm::FMT_C128, c->V, 0, s, sb, std::vector<double>(s, 0.0), qr, dep);
        if (st != HELM_OK) return st;
        std::vector<BlockLS> ls(G);
        for (int g = 0; g < G; ++g) ls[g].init(sb, m, qr.R[g]);
        std::vector<int> stop(G, -1);  // block step at which a group met tol
        std::vector<std::vector<cd>> hist(G);
        int jend = m - 1;
        for (int j = 0; j < m; ++j) {
            // Z_j = M^{-1}_cycle V_j ; W = A Z_j
            st = fgmres_step<ZT>(c, j, s, sb);
            if (st != HELM_OK) return st;
            st = sync(c);
            if (st != HELM_OK) return st;
            // H_{i,j} = H1 (+ H2 of a second pass) per group, and the
            // reference norms (the squared norm each column lost to V)
            std::vector<double> ref2(s, 0.0);
            std::vector<std::vector<cd>> hcol(G);
            const int ld = (m + 1) * sb;
            bool two = c->p.orth == 1;
            auto gather_h = [&]() {
                std::fill(ref2.begin(), ref2.end(), 0.0);
                for (int g = 0; g < G; ++g) hcol[g].assign((size_t)ld * sb, 0.0);
                for (int i = 0; i <= j; ++i)
                    for (int g = 0; g < G; ++g) {
                        const int ng = std::min(sb, s - g * sb);   // columns of a ragged last group
                        for (int a = 0; a < ng; ++a)
                            for (int b = 0; b < ng; ++b) {
                                long long o = ((long long)i * G + g) * sb * sb + a * sb + b;
                                cd h = cd(c->hsmall[SL.oH1 + o].re, c->hsmall[SL.oH1 + o].im);
                                if (two) h += cd(c->hsmall[SL.oH2 + o].re, c->hsmall[SL.oH2 + o].im);
                                hcol[g][(size_t)b * ld + i * sb + a] = h;
                                ref2[g * sb + b] += std::norm(h);
                            }
                    }
            };
            gather_h();
            if (c->p.orth == 0 && needs_second_gs(c, s, sb, ref2)) {
                // the single pass may have left too much of W along V: a
                // second pass on the updated block, then its QR Gram again
                c->orth_reorth++;
                gs_pass(c, c->W, j + 1, s, sb, c->small + SL.oH2, true);
                CUDA_TRY(c, cudaMemcpyAsync(c->hsmall + SL.oH2, c->small + SL.oH2,
                                            sizeof(c128) * (j + 1) * SL.blk, cudaMemcpyDeviceToHost, c->st));
                st = qr_gram_launch(c, c->W, c->kfmt, s, sb);
                if (st != HELM_OK) return st;
                st = sync(c);
                if (st != HELM_OK) return st;
                two = true;
                gather_h();
            }
            // W = V_{j+1} H_{j+1,j}
            st = block_qr(c, c->W, c->kfmt, c->V + (long long)(j + 1) * vs, j + 1, s, sb, ref2, qr, dep,
                          true);
            if (st != HELM_OK) return st;
            bool all_stop = true;
            for (int g = 0; g < G; ++g) {
                for (int a = 0; a < sb; ++a)
                    for (int b = 0; b < sb; ++b)
                        hcol[g][(size_t)b * ld + (j + 1) * sb + a] = qr.R[g][a * sb + b];
                if (done[g] || stop[g] >= 0) continue;
                std::vector<double> est = ls[g].add(j, hcol[g], ld);
                iters[g] += 1;
                bool ok = true;
                for (int b = 0; b < sb && g * sb + b < s; ++b) ok = ok && est[b] <= tol * bn[g * sb + b];
                if (ok) stop[g] = j;
                else all_stop = false;
            }
            if (all_stop) { jend = j; break; }
        }
        // X += sum_j Z_j Y_j per group
        cd* hY = reinterpret_cast<cd*>(c->hsmall + SL.oY);
        std::memset(hY, 0, sizeof(c128) * (size_t)(jend + 1) * SL.blk);
        for (int g = 0; g < G; ++g) {
            if (done[g]) continue;
            int jg = stop[g] >= 0 ? stop[g] : jend;
            std::vector<cd> Y = ls[g].solve(jg);
            for (int jj = 0; jj <= jg; ++jj)
                for (int a = 0; a < sb; ++a)
                    for (int b = 0; b < sb; ++b)
                        hY[((size_t)jj * G + g) * sb * sb + a * sb + b] = Y[(size_t)(jj * sb + a) * sb + b];
        }
        CUDA_TRY(c, cudaMemcpyAsync(c->small + SL.oY, hY, sizeof(c128) * (size_t)(jend + 1) * SL.blk,
                                    cudaMemcpyHostToDevice, c->st));
        helm::launch_combine<ZT>(c->L(), c->X, 1.0, 1.0, Z, jend + 1, vs, c->small + SL.oY, N, s, sb,
                                 emulated(c), c->csplit);
    }
finish:
    if (info) {
        for (int j = 0; j < s; ++j) {
            if (info->iters) info->iters[j] = iters[j / sb];
            if (info->relres) info->relres[j] = rel[j];
            if (info->status)
                info->status[j] = (result == HELM_ERR_NONFINITE) ? HELM_ERR_NONFINITE
                                  : (rel[j] <= tol ? HELM_OK : HELM_NOT_CONVERGED);
        }
    }
    return result;
}

// ---------------------------------------------------------------------------
// block BiCGSTAB (Sec. 5.3 "W-BiCG": El Guennouni, Jbilou and Sadok's block
// BiCGSTAB preconditioned by W-cycles), per group of `block` columns
// ---------------------------------------------------------------------------

// G Y = Rhs for one group (n x n, row-major): Gaussian elimination with
// partial pivoting; a pivot below 1e-14 max|G| zeroes its row of Y.
std::vector<cd> small_solve(const std::vector<cd>& G, const std::vector<cd>& Rhs, int n) {
    std::vector<cd> A = G, Y = Rhs;
    double scale = 0;
    for (auto& v : A) scale = std::max(scale, std::abs(v));
    std::vector<char> dead(n, 0);
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::abs(A[i * n + k]) > std::abs(A[p * n + k])) p = i;
        if (p != k)
            for (int j = 0; j < n; ++j) { std::swap(A[k * n + j], A[p * n + j]); std::swap(Y[k * n + j], Y[p * n + j]); }
        if (!(std::abs(A[k * n + k]) > 1e-14 * scale)) { dead[k] = 1; continue; }
        for (int i = k + 1; i < n; ++i) {
            cd f = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            for (int j = 0; j < n; ++j) Y[i * n + j] -= f * Y[k * n + j];
        }
    }
    for (int k = n - 1; k >= 0; --k)
        for (int j = 0; j < n; ++j) {
            if (dead[k]) { Y[k * n + j] = 0.0; continue; }
            cd v = Y[k * n + j];
            for (int t = k + 1; t < n; ++t) v -= A[k * n + t] * Y[t * n + j];
            Y[k * n + j] = v / A[k * n + k];
        }
    return Y;
}

template <typename ZT>
helm_status bicgstab(helm_ctx* c, int s, double tol, helm_info* info) {
    const long long N = c->N();
    const long long vs = N * s;
    const int sb = std::min(c->p.block, s);
    const int G = (s + sb - 1) / sb;
    const long long blk = (long long)G * sb * sb;
    const size_t vbytes = sizeof(c128) * (size_t)vs;
    c128 *R = c->V, *P = c->V + vs, *Vv = c->V + 2 * vs, *S = c->V + 3 * vs, *T = c->V + 4 * vs,
         *Rt = c->V + 5 * vs;
    cplx<ZT>* Ph = reinterpret_cast<cplx<ZT>*>(c->Z);
    cplx<ZT>* Sh = Ph + vs;
    helm::FineOp<double> opA = fine_op<double>(c, false);
    // device small-matrix slots (each blk complex): 0..5 Grams, 6..7 [alpha; omega I], 8 beta-ish
    c128* d = c->small;
    cd* h = reinterpret_cast<cd*>(c->hsmall);
    const bool emu = emulated(c);
    const int maxit = std::max(1, c->p.restart * std::max(1, c->p.max_restarts));

    std::vector<double> bn2;
    helm_status st = colnorms(c, c->Bint, s, bn2);
    if (st != HELM_OK) return st;
    std::vector<double> bn(s), rel(s, 0.0);
    for (int j = 0; j < s; ++j) {
        if (!std::isfinite(bn2[j])) return fail(c, HELM_ERR_NONFINITE, "non-finite right-hand side");
        bn[j] = std::sqrt(bn2[j]);
    }
    helm::launch_zero(c->L(), c->X, vbytes);
    std::vector<int> iters(G, 0);
    helm_status result = HELM_NOT_CONVERGED;
    auto gram = [&](const c128* X, const c128* Y, int slot) {
        helm::launch_gram(c->L(), X, 1, 0, Y, N, s, sb, c->partial, d + slot * blk, emu);
    };
    auto group_cols = [&](int g) { return std::min(sb, s - g * sb); };
    auto get = [&](int slot, int g, int a, int b) { return h[slot * blk + (long long)g * sb * sb + a * sb + b]; };

    for (int run = 0; run <= c->p.max_restarts; ++run) {
        helm::launch_residual<double, helm::FineOp<double>>(c->L(), opA, c->X, c->Bint, R, s);
        std::vector<double> rn2;
        st = colnorms(c, R, s, rn2);
        if (st != HELM_OK) return st;
        bool all = true;
        for (int j = 0; j < s; ++j) {
            if (!std::isfinite(rn2[j])) { result = fail(c, HELM_ERR_NONFINITE, "non-finite residual"); goto done; }
            rel[j] = bn[j] > 0 ? std::sqrt(rn2[j]) / bn[j] : 0.0;
            all = all && rel[j] <= tol;
        }
        if (all) { result = HELM_OK; break; }
        if (run == c->p.max_restarts) break;
        CUDA_TRY(c, cudaMemcpyAsync(Rt, R, vbytes, cudaMemcpyDeviceToDevice, c->st));
        CUDA_TRY(c, cudaMemcpyAsync(P, R, vbytes, cudaMemcpyDeviceToDevice, c->st));
        std::vector<char> gdone(G, 0);
        for (int g = 0; g < G; ++g) {
            bool ok = true;
            for (int j = g * sb; j < g * sb + group_cols(g); ++j) ok = ok && rel[j] <= tol;
            gdone[g] = ok;
        }
        for (int k = 0; k < maxit; ++k) {
            // Ph = M P, V = A Ph ; alpha = (Rt^H V)^{-1} Rt^H R
            cycle<ZT, double>(c, 0, P, Ph, s);
            helm::launch_apply<double, ZT, double, helm::FineOp<double>>(c->L(), opA, Ph, Vv, s);
            gram(Rt, Vv, 0);
            gram(Rt, R, 1);
            CUDA_TRY(c, cudaMemcpyAsync(h, d, sizeof(c128) * 2 * blk, cudaMemcpyDeviceToHost, c->st));
            st = sync(c);
            if (st != HELM_OK) return st;
            std::vector<std::vector<cd>> Gv(G), alpha(G);
            cd* ha = h + 6 * blk;          // [alpha; omega I] for the X update (two blocks)
            std::memset(ha, 0, sizeof(c128) * 2 * blk);
            for (int g = 0; g < G; ++g) {
                int n = group_cols(g);
                std::vector<cd> Gm(n * n), rhs(n * n);
                for (int a = 0; a < n; ++a)
                    for (int b = 0; b < n; ++b) { Gm[a * n + b] = get(0, g, a, b); rhs[a * n + b] = get(1, g, a, b); }
                Gv[g] = Gm;
                alpha[g] = gdone[g] ? std::vector<cd>(n * n, 0.0) : small_solve(Gm, rhs, n);
                for (int a = 0; a < n; ++a)
                    for (int b = 0; b < n; ++b) ha[(long long)g * sb * sb + a * sb + b] = alpha[g][a * n + b];
            }
            CUDA_TRY(c, cudaMemcpyAsync(d + 6 * blk, ha, sizeof(c128) * blk, cudaMemcpyHostToDevice, c->st));
            // S = R - V alpha ; Sh = M S ; T = A Sh
            CUDA_TRY(c, cudaMemcpyAsync(S, R, vbytes, cudaMemcpyDeviceToDevice, c->st));
            helm::launch_combine<double>(c->L(), S, 1.0, -1.0, Vv, 1, 0, d + 6 * blk, N, s, sb, emu, c->csplit);
            cycle<ZT, double>(c, 0, S, Sh, s);
            helm::launch_apply<double, ZT, double, helm::FineOp<double>>(c->L(), opA, Sh, T, s);
            gram(Rt, T, 2);
            gram(T, S, 3);
            gram(T, T, 4);
            gram(S, S, 5);
            CUDA_TRY(c, cudaMemcpyAsync(h + 2 * blk, d + 2 * blk, sizeof(c128) * 4 * blk, cudaMemcpyDeviceToHost, c->st));
            st = sync(c);
            if (st != HELM_OK) return st;
            // omega per group, residual estimates, beta
            cd* hw = h + 7 * blk;          // omega I
            cd* hb = h + 8 * blk;          // [beta; -omega beta] for the P update (two blocks)
            std::memset(hw, 0, sizeof(c128) * blk);
            std::memset(hb, 0, sizeof(c128) * 2 * blk);
            bool all_done = true;
            for (int g = 0; g < G; ++g) {
                int n = group_cols(g);
                if (gdone[g]) continue;
                cd ts = 0.0, tt = 0.0;
                for (int a = 0; a < n; ++a) { ts += get(3, g, a, a); tt += get(4, g, a, a); }
                cd om = std::abs(tt) > 0 ? ts / tt : cd(0.0);
                bool ok = true;
                for (int a = 0; a < n; ++a) {
                    double r2 = get(5, g, a, a).real() - 2.0 * (std::conj(om) * get(3, g, a, a)).real() +
                                std::norm(om) * get(4, g, a, a).real();
                    int j = g * sb + a;
                    double e = bn[j] > 0 ? std::sqrt(std::max(r2, 0.0)) / bn[j] : 0.0;
                    ok = ok && e <= tol;
                }
                iters[g] += 2;
                std::vector<cd> rhs(n * n);
                for (int a = 0; a < n; ++a)
                    for (int b = 0; b < n; ++b) rhs[a * n + b] = -get(2, g, a, b);
                std::vector<cd> beta = ok ? std::vector<cd>(n * n, 0.0) : small_solve(Gv[g], rhs, n);
                for (int a = 0; a < n; ++a) {
                    hw[(long long)g * sb * sb + a * sb + a] = om;
                    for (int b = 0; b < n; ++b) {
                        hb[(long long)g * sb * sb + a * sb + b] = beta[a * n + b];
                        hb[blk + (long long)g * sb * sb + a * sb + b] = -om * beta[a * n + b];
                    }
                }
                if (ok) gdone[g] = 1;
                else all_done = false;
            }
            CUDA_TRY(c, cudaMemcpyAsync(d + 7 * blk, hw, sizeof(c128) * 3 * blk, cudaMemcpyHostToDevice, c->st));
            // X += Ph alpha + Sh omega ; R = S - omega T ; P = R + P beta - V omega beta
            helm::launch_combine<ZT>(c->L(), c->X, 1.0, 1.0, Ph, 2, vs, d + 6 * blk, N, s, sb, emu, c->csplit);
            CUDA_TRY(c, cudaMemcpyAsync(R, S, vbytes, cudaMemcpyDeviceToDevice, c->st));
            helm::launch_combine<double>(c->L(), R, 1.0, -1.0, T, 1, 0, d + 7 * blk, N, s, sb, emu, c->csplit);
            if (all_done) break;
            CUDA_TRY(c, cudaMemcpyAsync(c->W, R, vbytes, cudaMemcpyDeviceToDevice, c->st));
            helm::launch_combine<double>(c->L(), c->W, 1.0, 1.0, P, 2, vs, d + 8 * blk, N, s, sb, emu, c->csplit);
            CUDA_TRY(c, cudaMemcpyAsync(P, c->W, vbytes, cudaMemcpyDeviceToDevice, c->st));
        }
    }
done:
    if (info) {
        for (int j = 0; j < s; ++j) {
            if (info->iters) info->iters[j] = iters[j / sb];
            if (info->relres) info->relres[j] = rel[j];
            if (info->status)
                info->status[j] = (result == HELM_ERR_NONFINITE) ? HELM_ERR_NONFINITE
                                  : (rel[j] <= tol ? HELM_OK : HELM_NOT_CONVERGED);
        }
    }
    return result;
}

helm_status solve_internal(helm_ctx* c, const c128* Qd, int s, double tol, c128* Ud,
                           helm_info* info, bool conjugate) {
    if (!c) return fail(nullptr, HELM_ERR_ARG, "null context");
    if (s < 0 || (s > 0 && (!Qd || !Ud)) || !(tol > 0.0))
        return fail(c, HELM_ERR_ARG, "bad arguments to solve");
    if (s == 0) return HELM_OK;
    helm_status st = ensure_workspace(c, s);
    if (st != HELM_OK) return st;
    // the same block gives the same result on every call: the draws for
    // dependent columns do not depend on what the context solved before
    c->rng_counter = 0x5eed;
    const long long N = c->N();
    helm::launch_to_internal(c->L(), Qd, c->Bint, N, s, conjugate);
    if (c->p.krylov == 1)
        st = c->p.prec == HELM_PLAIN_C128 ? bicgstab<double>(c, s, tol, info)
                                          : bicgstab<float>(c, s, tol, info);
    else if (c->p.prec == HELM_PLAIN_C128)
        st = fgmres<double>(c, s, tol, info);
    else
        st = fgmres<float>(c, s, tol, info);
    if (st == HELM_ERR_ARG || st == HELM_ERR_CUDA || st == HELM_ERR_NOMEM || st == HELM_ERR_BREAKDOWN)
        return st;
    helm::launch_from_internal(c->L(), c->X, Ud, N, s, conjugate);
    helm_status st2 = sync_checked(c);
    if (st2 != HELM_OK) return st2;
    return st;
}

}  // namespace

namespace {
template <typename T>
helm_status smooth_t(helm_ctx* c, int level, const void* u_in, const void* f, void* u_out,
                            int s, int sweeps) {
    helm_status st = ensure_workspace(c, s);
    if (st != HELM_OK) return st;
    const cplx<T>* cur = static_cast<const cplx<T>*>(u_in);
    cplx<T>* tmp = reinterpret_cast<cplx<T>*>(c->lv[level].u0);
    cplx<T>* tmp2 = reinterpret_cast<cplx<T>*>(c->lv[level].u1);
    for (int k = 0; k < sweeps; ++k) {
        cplx<T>* dst = (k == sweeps - 1) ? static_cast<cplx<T>*>(u_out) : (k % 2 == 0 ? tmp : tmp2);
        smooth_level<T, T>(c, level, cur, static_cast<const cplx<T>*>(f), dst, s);
        cur = dst;
    }
    return sync(c);
}

// Receiver indices (device int array) must name nodes of the fine grid: they
// are copied to the host and checked before any kernel reads through them.
helm_status check_receivers(helm_ctx* c, const int* recv, int nrec) {
    std::vector<int> h((size_t)nrec);
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), recv, sizeof(int) * (size_t)nrec, cudaMemcpyDefault, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    const long long N = c->N();
    for (int r = 0; r < nrec; ++r)
        if (h[r] < 0 || h[r] >= N)
            return fail(c, HELM_ERR_ARG, "receiver index " + std::to_string(h[r]) + " outside [0, N)");
    return HELM_OK;
}

// Two device temporaries of a call; on failure neither is kept.
helm_status alloc_pair(helm_ctx* c, void** a, size_t abytes, void** b, size_t bbytes) {
    *a = *b = nullptr;
    cudaError_t e = dalloc(a, abytes);
    if (e == cudaSuccess) e = dalloc(b, bbytes);
    if (e != cudaSuccess) {
        dfree(*a);
        dfree(*b);
        *a = *b = nullptr;
        return fail(c, e == cudaErrorMemoryAllocation ? HELM_ERR_NOMEM : HELM_ERR_CUDA,
                    std::string("device temporaries: ") + cudaGetErrorString(e));
    }
    return HELM_OK;
}

}  // namespace

// ===========================================================================
// C-ABI
// ===========================================================================

extern "C" {

void helm_default_params(helm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dim = 2;
    p->h = 1.0;
    p->shift = 0.5;
    p->levels = 3;
    p->pre = 2;
    p->post = 2;
    p->jacobi_w = 0.8;
    p->restart = 10;
    p->block = 8;
    p->max_restarts = 50;
    p->prec = HELM_PLAIN_C128;
    p->learned_weights = nullptr;
    p->coarse_tf32x3 = 0;
    p->cycle_gamma = 1;
    p->krylov = 0;
    p->graphs = 2;
    p->orth = 0;
}

helm_status helm_setup(const double* m, const double* gamma_tilde, const helm_params* p,
                       void* cuda_stream, helm_ctx** out) {
    if (!out) return fail(nullptr, HELM_ERR_ARG, "out is null");
    *out = nullptr;
    if (!m || !gamma_tilde || !p) return fail(nullptr, HELM_ERR_ARG, "null argument");
    if (p->dim != 2 && p->dim != 3) return fail(nullptr, HELM_ERR_ARG, "dim must be 2 or 3");
    if (p->levels < 1 || p->levels > 12 || p->pre < 0 || p->post < 0 || p->restart < 1 ||
        p->block < 1 || p->max_restarts < 0 || !(p->h > 0) || !(p->omega >= 0))
        return fail(nullptr, HELM_ERR_ARG, "bad parameter");
    if (p->prec != HELM_PLAIN_C128 && p->prec != HELM_MIXED_C64 && p->prec != HELM_MIXED_C64_LEARNED)
        return fail(nullptr, HELM_ERR_ARG, "bad precision policy");
    if (p->prec == HELM_MIXED_C64_LEARNED && (p->dim != 2 || !p->learned_weights))
        return fail(nullptr, HELM_ERR_ARG, "the learned stage needs a 2D grid and learned_weights");
    if (p->cycle_gamma < 1 || p->cycle_gamma > 3 || (p->krylov != 0 && p->krylov != 1))
        return fail(nullptr, HELM_ERR_ARG, "cycle_gamma must be 1, 2 or 3, krylov 0 or 1");
    if (p->orth != 0 && p->orth != 1) return fail(nullptr, HELM_ERR_ARG, "orth must be 0 or 1");
    if (p->coarse_tf32x3 < 0 || p->coarse_tf32x3 > 2)
        return fail(nullptr, HELM_ERR_ARG, "coarse_tf32x3 must be 0, 1 or 2");
    if (p->krylov == 1 && p->cycle_gamma == 3)
        return fail(nullptr, HELM_ERR_ARG, "the K-cycle is nonlinear: use it with FGMRES (krylov 0)");
    if (p->krylov == 1 && p->prec == HELM_MIXED_C64_LEARNED)
        return fail(nullptr, HELM_ERR_ARG, "block BiCGSTAB needs a fixed preconditioner (no learned stage)");
    if (p->krylov == 1 && p->prec == HELM_MIXED_C64 && p->block > 2)
        return fail(nullptr, HELM_ERR_ARG,
                    "block BiCGSTAB with the complex64 cycle needs block <= 2 (larger blocks diverge: "
                    "the cycle's FP32 rounding makes the preconditioner slightly non-stationary)");
    int nodes[3] = {1, 1, 1};
    for (int k = 0; k < p->dim; ++k) {
        if (p->n[k] < 1) return fail(nullptr, HELM_ERR_ARG, "cells per axis must be >= 1");
        if (p->n[k] % (1 << (p->levels - 1)))
            return fail(nullptr, HELM_ERR_ARG, "cells per axis must be divisible by 2^(levels-1)");
        nodes[k] = p->n[k] + 1;
    }
    helm_ctx* c = new helm_ctx();
    c->p = *p;
    c->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    c->inv_h2 = 1.0 / (p->h * p->h);
    c->lv.resize(p->levels);
    for (int l = 0; l < p->levels; ++l) {
        Grid g;
        g.dim = p->dim;
        g.n1 = (nodes[0] - 1) / (1 << l) + 1;
        g.n2 = (nodes[1] - 1) / (1 << l) + 1;
        g.n3 = p->dim == 3 ? (nodes[2] - 1) / (1 << l) + 1 : 1;
        g.N = (long long)g.n1 * g.n2 * g.n3;
        c->lv[l].g = g;
    }
    const int K = p->dim == 3 ? 27 : 9;
    auto cleanup = [&](helm_status s) { helm_destroy(c); return s; };
    helm_status st;
#define SETUP_TRY(expr)                                                                \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            st = fail(nullptr, e_ == cudaErrorMemoryAllocation ? HELM_ERR_NOMEM : HELM_ERR_CUDA, \
                      std::string(#expr) + ": " + cudaGetErrorString(e_));             \
            return cleanup(st);                                                        \
        }                                                                              \
    } while (0)
    const long long N0 = c->lv[0].g.N;
    double *dm = nullptr, *dg = nullptr;
    SETUP_TRY(dalloc(&dm, sizeof(double) * N0));
    SETUP_TRY(dalloc(&dg, sizeof(double) * N0));
    SETUP_TRY(cudaMemcpyAsync(dm, m, sizeof(double) * N0, cudaMemcpyDefault, c->st));
    SETUP_TRY(cudaMemcpyAsync(dg, gamma_tilde, sizeof(double) * N0, cudaMemcpyDefault, c->st));
    SETUP_TRY(dalloc(&c->cA, sizeof(c128) * N0));
    SETUP_TRY(dalloc(&c->cM, sizeof(c128) * N0));
    SETUP_TRY(dalloc(&c->cA32, sizeof(c64) * N0));
    SETUP_TRY(dalloc(&c->cM32, sizeof(c64) * N0));
    for (int l = 0; l < p->levels; ++l) {
        long long Nl = c->lv[l].g.N;
        SETUP_TRY(dalloc(&c->lv[l].coef, sizeof(c128) * Nl * K));
        SETUP_TRY(dalloc(&c->lv[l].dinv, sizeof(c128) * Nl));
        SETUP_TRY(dalloc(&c->lv[l].coef32, sizeof(c64) * Nl * K));
        SETUP_TRY(dalloc(&c->lv[l].dinv32, sizeof(c64) * Nl));
    }
    Launch L = c->L();
    helm::launch_fine_setup(L, c->lv[0].g, dm, dg, p->omega, p->shift, c->inv_h2, c->cA, c->cM,
                            c->lv[0].dinv, c->lv[0].coef);
    for (int l = 1; l < p->levels; ++l) {
        helm::launch_galerkin(L, c->lv[l - 1].g, c->lv[l].g, c->lv[l - 1].coef, c->lv[l].coef);
        helm::launch_diag_inv(L, c->lv[l].g, c->lv[l].coef, c->lv[l].dinv);
    }
    SETUP_TRY(dalloc(&c->dadm, sizeof(c128) * N0));
    helm::launch_dadm(L, dg, p->omega, N0, c->dadm);
    SETUP_TRY(dalloc(&c->kappa, sizeof(float) * N0));
    helm::launch_kappa(L, c->cA, N0, p->h * p->h, c->kappa);
    helm::launch_round_c64(L, c->cA, c->cA32, N0);
    SETUP_TRY(dalloc(&c->cAdd, sizeof(float4) * N0));
    helm::launch_split_pairs(L, c->cA, c->cAdd, N0);
    helm::launch_round_c64(L, c->cM, c->cM32, N0);
    for (int l = 0; l < p->levels; ++l) {
        long long Nl = c->lv[l].g.N;
        helm::launch_round_c64(L, c->lv[l].coef, c->lv[l].coef32, Nl * K);
        helm::launch_round_c64(L, c->lv[l].dinv, c->lv[l].dinv32, Nl);
    }
    // coarsest inverse by Gauss-Jordan with partial pivoting (FP64)
    const Grid& gcst = c->lv[p->levels - 1].g;
    if (gcst.N > 20000) {
        dfree(dm); dfree(dg);
        return cleanup(fail(nullptr, HELM_ERR_ARG, "coarsest grid too large for the dense solve; add levels"));
    }
    c->nc = (int)gcst.N;
    const int n = c->nc;
    // the plain solver gets the FP64 inverse; the complex64 cycle an FP32
    // one (its tensor-core solve rounds the inverse to tf32 anyway)
    const bool fp64_inverse = p->prec == HELM_PLAIN_C128;
    const size_t esz = fp64_inverse ? sizeof(c128) : sizeof(c64);
    void *aug = nullptr, *factor = nullptr, *pivval = nullptr;
    int *piv = nullptr, *dstatus = nullptr;
    SETUP_TRY(dalloc(&aug, esz * (size_t)n * 2 * n));
    SETUP_TRY(dalloc(&factor, esz * n));
    SETUP_TRY(dalloc(&pivval, sizeof(c128)));
    SETUP_TRY(dalloc(&piv, sizeof(int)));
    SETUP_TRY(dalloc(&dstatus, sizeof(int)));
    SETUP_TRY(cudaMemsetAsync(dstatus, 0, sizeof(int), c->st));
    SETUP_TRY(dalloc(&c->Minv, sizeof(c128) * (size_t)n * n));
    SETUP_TRY(dalloc(&c->Ap, sizeof(float) * (size_t)n * helm::dense_tc_kpad(n)));
    c128* dense = nullptr;
    SETUP_TRY(dalloc(&dense, sizeof(c128) * (size_t)n * n));
    helm::launch_stencil_to_dense(L, gcst, c->lv[p->levels - 1].coef, dense);
    if (fp64_inverse)
        helm::launch_gauss_jordan<double>(L, dense, aug, n, factor, piv, pivval, dstatus, c->Minv);
    else
        helm::launch_gauss_jordan<float>(L, dense, aug, n, factor, piv, pivval, dstatus, c->Minv);
    helm::launch_build_aprime(L, c->Minv, n, c->Ap, p->coarse_tf32x3 == 1);
    int hstatus = 0;
    SETUP_TRY(cudaMemcpyAsync(&hstatus, dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    SETUP_TRY(cudaStreamSynchronize(c->st));
    SETUP_TRY(cudaGetLastError());
    dfree(aug); dfree(factor); dfree(pivval); dfree(piv); dfree(dstatus); dfree(dm); dfree(dg);
    dfree(dense);
    if (hstatus) return cleanup(fail(nullptr, HELM_ERR_BREAKDOWN, "coarsest operator is singular"));
#undef SETUP_TRY
    *out = c;
    return HELM_OK;
}

helm_status helm_solve(helm_ctx* ctx, const void* Q, int s, double tol, void* U, helm_info* info) {
    return solve_internal(ctx, static_cast<const c128*>(Q), s, tol, static_cast<c128*>(U), info,
                          false);
}

helm_status helm_adjoint(helm_ctx* ctx, const void* B, int s, double tol, void* Lout,
                         helm_info* info) {
    return solve_internal(ctx, static_cast<const c128*>(B), s, tol, static_cast<c128*>(Lout), info,
                          true);
}

helm_status helm_solve_host(helm_ctx* c, const void* Q_host, int s, double tol, void* U_host,
                            helm_info* info) {
    if (!c) return fail(nullptr, HELM_ERR_ARG, "null context");
    if (s < 0 || (s > 0 && (!Q_host || !U_host)) || !(tol > 0.0))
        return fail(c, HELM_ERR_ARG, "bad arguments to solve_host");
    if (s == 0) return HELM_OK;
    helm_status st = ensure_workspace(c, s);
    if (st != HELM_OK) return st;
    // The device staging holds s_cap columns, so every later call of at most
    // s_cap columns fits; a call that raises s_cap frees it (free_workspace)
    // and it is allocated again at the new capacity.
    const size_t cap_bytes = sizeof(c128) * (size_t)c->N() * c->s_cap;
    const size_t bytes = sizeof(c128) * (size_t)c->N() * s;
    if (!c->abi_in) CUDA_TRY(c, dalloc(&c->abi_in, cap_bytes));
    if (!c->abi_out) CUDA_TRY(c, dalloc(&c->abi_out, cap_bytes));
    CUDA_TRY(c, cudaMemcpyAsync(c->abi_in, Q_host, bytes, cudaMemcpyHostToDevice, c->st));
    helm_status r = solve_internal(c, c->abi_in, s, tol, c->abi_out, info, false);
    if (r == HELM_ERR_ARG || r == HELM_ERR_CUDA || r == HELM_ERR_NOMEM) return r;
    CUDA_TRY(c, cudaMemcpyAsync(U_host, c->abi_out, bytes, cudaMemcpyDeviceToHost, c->st));
    helm_status st2 = sync(c);
    return st2 != HELM_OK ? st2 : r;
}

helm_status helm_solve_batch(helm_ctx* const* ctxs, const void* const* Q, const int* s, int nprob,
                             double tol, void* const* U, helm_info* infos) {
    if (nprob < 0 || (nprob > 0 && (!ctxs || !Q || !s || !U)))
        return fail(nullptr, HELM_ERR_ARG, "bad batch arguments");
    for (int k = 0; k < nprob; ++k)
        if (!ctxs[k] || s[k] < 0) return fail(nullptr, HELM_ERR_ARG, "bad problem in batch");
    // Longest-processing-time-first order under a cost model: work per cycle
    // ~ nodes x columns (x4 on the FP64 path, whose kernels run on the narrow
    // FP64 pipe), cycles ~ wavelengths across the grid ~ omega h max(n).
    std::vector<std::pair<double, int>> order;
    for (int k = 0; k < nprob; ++k) {
        const helm_params& p = ctxs[k]->p;
        int nmax = std::max(p.n[0], std::max(p.n[1], p.dim == 3 ? p.n[2] : 0));
        double cost = (double)ctxs[k]->N() * std::max(1, s[k]) * (1.0 + p.omega * p.h * nmax) *
                      (p.prec == HELM_PLAIN_C128 ? 4.0 : 1.0);
        order.push_back({-cost, k});
    }
    std::sort(order.begin(), order.end());
    // Host workers take problems in that order; each problem's work is on its
    // context's stream, so problems whose contexts have distinct streams run
    // concurrently on the GPU.  Workers: HELM_BATCH_WORKERS (default 4).
    int workers = 4;
    if (const char* e = std::getenv("HELM_BATCH_WORKERS")) workers = std::max(1, std::atoi(e));
    workers = std::min(workers, std::max(nprob, 1));
    std::atomic<int> next{0};
    std::vector<helm_status> status(nprob, HELM_OK);
    int dev = 0;
    cudaGetDevice(&dev);
    auto run = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            int i = next.fetch_add(1);
            if (i >= nprob) break;
            int k = order[i].second;
            status[k] = helm_solve(ctxs[k], Q[k], s[k], tol, U[k], infos ? &infos[k] : nullptr);
        }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < workers; ++w) pool.emplace_back(run);
    run();
    for (auto& t : pool) t.join();
    helm_status first = HELM_OK;
    for (int k = 0; k < nprob; ++k)
        if (status[k] != HELM_OK && first == HELM_OK) first = status[k];
    return first;
}

void helm_destroy(helm_ctx* c) {
    if (!c) return;
    delete c->prof;
    c->prof = nullptr;
    free_workspace(c);
    if (c->cap_st) cudaStreamDestroy(c->cap_st);
    for (auto& l : c->lv) {
        dfree(l.coef); dfree(l.dinv); dfree(l.coef32); dfree(l.dinv32);
    }
    dfree(c->cA); dfree(c->cM); dfree(c->cA32); dfree(c->cM32); dfree(c->Minv); dfree(c->Minv32);
    dfree(c->cAdd);
    dfree(c->Ap);
    dfree(c->kappa);
    dfree(c->dadm);
    delete c;
}

const char* helm_last_error(const helm_ctx* c) {
    if (c) return c->err.c_str();
    return g_thread_error.c_str();
}

helm_status helm_level_shape(const helm_ctx* c, int level, int* nodes, long long* count) {
    if (!c || level < 0 || level >= (int)c->lv.size()) return fail(nullptr, HELM_ERR_ARG, "bad level");
    const Grid& g = c->lv[level].g;
    if (nodes) { nodes[0] = g.n1; nodes[1] = g.n2; nodes[2] = g.n3; }
    if (count) *count = g.N;
    return HELM_OK;
}

helm_status helm_apply(helm_ctx* c, int level, int op, int prec, const void* x, void* y, int s) {
    if (!c || level < 0 || level >= (int)c->lv.size() || (op == 0 && level != 0) || op < 0 || op > 1 ||
        prec < 0 || prec > 1 || !x || !y || s < 1)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_apply");
    Launch L = c->L();
    if (prec == 0) {
        auto xx = static_cast<const c128*>(x);
        auto yy = static_cast<c128*>(y);
        if (level == 0)
            helm::launch_apply<double, double, double, helm::FineOp<double>>(L, fine_op<double>(c, op == 1), xx, yy, s);
        else
            helm::launch_apply<double, double, double, helm::GalOp<double>>(L, gal_op<double>(c, level), xx, yy, s);
    } else {
        auto xx = static_cast<const c64*>(x);
        auto yy = static_cast<c64*>(y);
        if (level == 0)
            helm::launch_apply<float, float, float, helm::FineOp<float>>(L, fine_op<float>(c, op == 1), xx, yy, s);
        else
            helm::launch_apply<float, float, float, helm::GalOp<float>>(L, gal_op<float>(c, level), xx, yy, s);
    }
    return sync(c);
}

helm_status helm_smooth(helm_ctx* c, int level, int prec, const void* u_in, const void* f,
                        void* u_out, int s, int sweeps) {
    if (!c || level < 0 || level >= (int)c->lv.size() || prec < 0 || prec > 1 || !f || !u_out ||
        s < 1 || sweeps < 1)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_smooth");
    return prec == 0 ? smooth_t<double>(c, level, u_in, f, u_out, s, sweeps)
                     : smooth_t<float>(c, level, u_in, f, u_out, s, sweeps);
}

helm_status helm_restrict_residual(helm_ctx* c, int level, int prec, const void* u, const void* f,
                                   void* rc, int s) {
    if (!c || level < 0 || level + 1 >= (int)c->lv.size() || prec < 0 || prec > 1 || !f || !rc || s < 1)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_restrict_residual");
    if (prec == 0)
        restrict_level<double, double>(c, level, static_cast<const c128*>(u), static_cast<const c128*>(f),
                                       static_cast<c128*>(rc), s);
    else
        restrict_level<float, float>(c, level, static_cast<const c64*>(u), static_cast<const c64*>(f),
                                     static_cast<c64*>(rc), s);
    return sync(c);
}

helm_status helm_prolong_add(helm_ctx* c, int level, int prec, const void* ec, void* u, int s) {
    if (!c || level < 0 || level + 1 >= (int)c->lv.size() || prec < 0 || prec > 1 || !ec || !u || s < 1)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_prolong_add");
    if (prec == 0)
        helm::launch_prolong_add<double>(c->L(), c->lv[level].g, c->lv[level + 1].g,
                                         static_cast<const c128*>(ec), static_cast<c128*>(u), s);
    else
        helm::launch_prolong_add<float>(c->L(), c->lv[level].g, c->lv[level + 1].g,
                                        static_cast<const c64*>(ec), static_cast<c64*>(u), s);
    return sync(c);
}

helm_status helm_coarse_solve(helm_ctx* c, int prec, const void* f, void* u, int s) {
    if (!c || prec < 0 || prec > 1 || !f || !u || s < 1)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_coarse_solve");
    helm_status st = ensure_workspace(c, s);
    if (st != HELM_OK) return st;
    if (prec == 0) coarsest<double>(c, static_cast<const c128*>(f), static_cast<c128*>(u), s);
    else coarsest<float>(c, static_cast<const c64*>(f), static_cast<c64*>(u), s);
    return sync_checked(c);
}

helm_status helm_vcycle(helm_ctx* c, int prec, const void* f, void* z, int s) {
    if (!c || prec < 0 || prec > 1 || !f || !z || s < 1)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_vcycle");
    helm_status st = ensure_workspace(c, s);
    if (st != HELM_OK) return st;
    if (prec == 0) cycle<double, double>(c, 0, static_cast<const c128*>(f), static_cast<c128*>(z), s);
    else cycle<float, double>(c, 0, static_cast<const c128*>(f), static_cast<c64*>(z), s);
    return sync_checked(c);
}

helm_status helm_get_operator(const helm_ctx* c, int level, void* coef_host) {
    if (!c || level < 0 || level >= (int)c->lv.size() || !coef_host)
        return fail(nullptr, HELM_ERR_ARG, "bad arguments to helm_get_operator");
    const int K = c->p.dim == 3 ? 27 : 9;
    cudaError_t e = cudaMemcpyAsync(coef_host, c->lv[level].coef, sizeof(c128) * c->lv[level].g.N * K,
                                    cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(nullptr, HELM_ERR_CUDA, cudaGetErrorString(e));
    return HELM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// helm_vcycle_noalloc: the V-cycle with its level buffers in a fixed device
// array instead of context workspace.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kNoAllocBytes = size_t(64) << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

// Level buffers of helm_vcycle_noalloc.  Every GPU that loads libhelm holds
// this array until the process exits.  Host code must not use its name as an
// address: the device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_vcycle_scratch[kNoAllocBytes];

void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of g_vcycle_scratch on the current device, looked up once
// per device (with that device current) and cached.
helm_status scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, HELM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, HELM_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_vcycle_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(nullptr, HELM_ERR_CUDA,
                        std::string("cudaGetSymbolAddress(g_vcycle_scratch): ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return HELM_OK;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" {

helm_status helm_vcycle_noalloc(helm_ctx* c, int prec, const void* f, void* z, int s) {
    if (!c || prec < 0 || prec > 1 || !f || !z || s < 1)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_vcycle_noalloc");
    if (c->p.cycle_gamma != 1)
        return fail(c, HELM_ERR_ARG, "helm_vcycle_noalloc runs V-cycles only (cycle_gamma 1)");
    const size_t esz = prec == 0 ? sizeof(c128) : sizeof(c64);
    // level 0 needs two buffers (u0, u1); every coarser level four (u0, u1, e, f)
    size_t need = 0;
    for (size_t l = 0; l < c->lv.size(); ++l)
        need += (l == 0 ? 2 : 4) * round256(esz * (size_t)c->lv[l].g.N * (size_t)s);
    // the complex64 coarsest solve also needs its tensor-core operand scratch
    const size_t dense_bytes = prec == 1 ? round256(sizeof(float) * helm::dense_tc_scratch_floats(c->nc, s)) : 0;
    need += dense_bytes;
    if (need > kNoAllocBytes)
        return fail(c, HELM_ERR_ARG,
                    "helm_vcycle_noalloc: " + std::to_string(need) + " bytes of level buffers needed, "
                    "the fixed scratch holds " + std::to_string(kNoAllocBytes) +
                    "; use fewer columns or helm_vcycle");
    void* base = nullptr;
    helm_status st = scratch_address(&base);
    if (st != HELM_OK) return fail(c, st, helm_last_error(nullptr));
    // Point the context's level buffers into the scratch for this call, then
    // put the context's own buffers back.  Nothing needs zeroing: every level
    // buffer is written in full before it is read (the cycle zero-fills its
    // correction buffer itself when there is no pre-smoothing).
    void* saved[12][4];  // helm_setup allows at most 12 levels
    for (size_t l = 0; l < c->lv.size(); ++l) {
        saved[l][0] = c->lv[l].u0; saved[l][1] = c->lv[l].u1;
        saved[l][2] = c->lv[l].e;  saved[l][3] = c->lv[l].f;
    }
    unsigned char* p = static_cast<unsigned char*>(base);
    float* saved_dense = c->dense_scratch;
    if (dense_bytes) {
        c->dense_scratch = reinterpret_cast<float*>(p);
        p += dense_bytes;
    }
    for (size_t l = 0; l < c->lv.size(); ++l) {
        size_t b = round256(esz * (size_t)c->lv[l].g.N * (size_t)s);
        c->lv[l].u0 = p; p += b;
        c->lv[l].u1 = p; p += b;
        if (l > 0) {
            c->lv[l].e = p; p += b;
            c->lv[l].f = p; p += b;
        }
    }
    if (prec == 0) cycle<double, double>(c, 0, static_cast<const c128*>(f), static_cast<c128*>(z), s);
    else cycle<float, double>(c, 0, static_cast<const c128*>(f), static_cast<c64*>(z), s);
    st = sync_checked(c);
    for (size_t l = 0; l < c->lv.size(); ++l) {
        c->lv[l].u0 = saved[l][0]; c->lv[l].u1 = saved[l][1];
        c->lv[l].e = saved[l][2];  c->lv[l].f = saved[l][3];
    }
    c->dense_scratch = saved_dense;
    return st;
}

long long helm_kernel_launches(const helm_ctx* c) { return c ? c->launches : 0; }

helm_status helm_orth_stats(const helm_ctx* c, long long* qr, long long* reorth, long long* qr2) {
    if (!c) return fail(nullptr, HELM_ERR_ARG, "ctx is null");
    if (qr) *qr = c->orth_qr;
    if (reorth) *reorth = c->orth_reorth;
    if (qr2) *qr2 = c->orth_qr2;
    return HELM_OK;
}

static const char* kKernelNames[helm::KID_COUNT] = {
    "apply_fine", "apply_coarse", "residual_fp64", "jacobi_fine", "jacobi_coarse",
    "restrict_fine", "restrict_coarse", "prolong_add", "coarsest_dense", "gram", "gram_reduce",
    "combine", "layout", "random_fill", "setup", "gram_dd", "combine_dd", "conv3x3",
    "conv3x3_wgrad", "gram_hi", "combine_hi"};

helm_status helm_profile_enable(helm_ctx* c, int enable) {
    if (!c) return fail(nullptr, HELM_ERR_ARG, "null context");
    if (enable) {
        if (!c->prof) c->prof = new helm::Profiler();
        c->prof->reset();
    } else {
        delete c->prof;
        c->prof = nullptr;
    }
    return HELM_OK;
}

helm_status helm_profile_select(helm_ctx* c, int kid) {
    if (!c) return fail(nullptr, HELM_ERR_ARG, "null context");
    if (kid < -1 || kid >= helm::KID_COUNT) return fail(c, HELM_ERR_ARG, "kernel class out of range");
    if (!c->prof) return fail(c, HELM_ERR_ARG, "the profiler is not enabled");
    c->prof->only = kid;
    return HELM_OK;
}

int helm_learned_layers(void) { return 6; }

long long helm_learned_blob_bytes(void) { return learned_blob_bytes(); }

helm_status helm_learned_layer(int layer, int* cin, int* cout, int* relu, long long* w_offset,
                               long long* b_offset) {
    if (layer < 0 || layer >= 6) return fail(nullptr, HELM_ERR_ARG, "bad layer");
    const LearnedLayer& t = learned_table()[layer];
    if (cin) *cin = t.cin;
    if (cout) *cout = t.cout;
    if (relu) *relu = t.relu;
    if (w_offset) *w_offset = t.w_off;
    if (b_offset) *b_offset = t.b_off;
    return HELM_OK;
}

static Launch bare_launch(void* stream) {
    return Launch{reinterpret_cast<cudaStream_t>(stream), nullptr, nullptr};
}

static helm_status check_launch(void* stream) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(nullptr, HELM_ERR_CUDA, cudaGetErrorString(e));
    return HELM_OK;
}

helm_status helm_conv3x3(const void* x, int batch, int H, int W, int cin, const void* w,
                         const float* bias, int cout, int relu, const void* mask, void* y,
                         int y_float, void* stream) {
    if (!x || !w || !y || batch < 1 || H < 1 || W < 1)
        return fail(nullptr, HELM_ERR_ARG, "bad arguments to helm_conv3x3");
    if (!helm::launch_conv3x3(bare_launch(stream), x, batch, H, W, cin, w, bias, cout, relu, mask, y,
                              y_float))
        return fail(nullptr, HELM_ERR_ARG, "unsupported channel counts for helm_conv3x3");
    return check_launch(stream);
}

helm_status helm_conv3x3_wgrad(const void* x, const void* gy, int batch, int H, int W, int cin,
                               int cout, float* dw, float* db, void* stream) {
    if (!x || !gy || !dw || !db || batch < 1 || H < 1 || W < 1)
        return fail(nullptr, HELM_ERR_ARG, "bad arguments to helm_conv3x3_wgrad");
    if (!helm::launch_conv3x3_wgrad(bare_launch(stream), x, gy, batch, H, W, cin, cout, dw, db))
        return fail(nullptr, HELM_ERR_ARG, "unsupported channel counts for helm_conv3x3_wgrad");
    return check_launch(stream);
}

helm_status helm_conv3x3_flip(const void* w, int cin, int cout, void* wf, int cin_out, void* stream) {
    if (!w || !wf || cin < 1 || cout < 1 || cin_out < cin)
        return fail(nullptr, HELM_ERR_ARG, "bad arguments to helm_conv3x3_flip");
    helm::launch_flip_weights(bare_launch(stream), w, cin, cout, wf, cin_out);
    return check_launch(stream);
}

helm_status helm_adam(float* p, const float* g, float* m, float* v, void* p_bf16, int n, float lr,
                      float b1, float b2, float eps, int step, void* stream) {
    if (!p || !g || !m || !v || n < 1 || step < 1)
        return fail(nullptr, HELM_ERR_ARG, "bad arguments to helm_adam");
    helm::launch_adam(bare_launch(stream), p, g, m, v, p_bf16, n, lr, b1, b2, eps, step);
    return check_launch(stream);
}

helm_status helm_learned_input(helm_ctx* c, const void* f, const void* z, int s, void* x_out,
                               float* rho_out) {
    if (!c || !f || !z || !x_out || !rho_out || s < 1 || c->p.dim != 2)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_learned_input");
    c64* r = nullptr;
    float* rho2 = nullptr;
    helm_status sa = alloc_pair(c, reinterpret_cast<void**>(&r), sizeof(c64) * (size_t)c->N() * s,
                                reinterpret_cast<void**>(&rho2), sizeof(float) * s);
    if (sa != HELM_OK) return sa;
    helm::launch_learned_residual(c->L(), fine_op<float>(c, false), static_cast<const c128*>(f),
                                  static_cast<const c64*>(z), r, s, rho2, rho_out);
    helm::launch_pack_input(c->L(), r, (int)c->N(), s, rho_out, c->kappa, x_out);
    helm_status st = sync(c);
    dfree(r);
    dfree(rho2);
    return st;
}

helm_status helm_learned_residual_input(helm_ctx* c, const void* f, const void* z, int s, void* x_out,
                                        float* rho_out, float* r_out, float* coef_out) {
    if (!c || !f || !z || !x_out || !rho_out || !r_out || !coef_out || s < 1 || c->p.dim != 2)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_learned_residual_input");
    c64* r = nullptr;
    float* rho2 = nullptr;
    helm_status sa = alloc_pair(c, reinterpret_cast<void**>(&r), sizeof(c64) * (size_t)c->N() * s,
                                reinterpret_cast<void**>(&rho2), sizeof(float) * s);
    if (sa != HELM_OK) return sa;
    helm::launch_learned_residual(c->L(), fine_op<float>(c, false), static_cast<const c128*>(f),
                                  static_cast<const c64*>(z), r, s, rho2, rho_out);
    helm::launch_pack_input(c->L(), r, (int)c->N(), s, rho_out, c->kappa, x_out);
    helm::launch_pack_resid(c->L(), r, (int)c->N(), s, rho_out, c->cA, c->p.h * c->p.h, r_out, coef_out);
    helm_status st = sync(c);
    dfree(r);
    dfree(rho2);
    return st;
}

helm_status helm_learned_residual_loss(const float* pred, const float* r, const float* coef, int batch, int H,
                                       int W, float* q, float* sums, void* grad, float* loss_out,
                                       void* stream) {
    if (!pred || !r || !coef || !q || !sums || !grad || batch < 1 || H < 1 || W < 1)
        return fail(nullptr, HELM_ERR_ARG, "bad arguments to helm_learned_residual_loss");
    helm::launch_residual_loss(bare_launch(stream), pred, r, coef, batch, H, W, q, sums, grad, loss_out);
    return check_launch(stream);
}

helm_status helm_learned_image_to_block(const float* r, long long N, int s, void* v, void* stream) {
    if (!r || !v || N < 1 || s < 1) return fail(nullptr, HELM_ERR_ARG, "bad arguments to helm_learned_image_to_block");
    helm::launch_image_to_block(bare_launch(stream), r, N, s, static_cast<c128*>(v));
    return check_launch(stream);
}

helm_status helm_learned_target(const void* e, long long N, int s, const float* rho, float scale,
                                float* t_out, void* stream) {
    if (!e || !rho || !t_out || N < 1 || s < 1)
        return fail(nullptr, HELM_ERR_ARG, "bad arguments to helm_learned_target");
    helm::launch_pack_target(bare_launch(stream), static_cast<const c64*>(e), (int)N, s, rho, scale, t_out);
    return check_launch(stream);
}

helm_status helm_learned_loss(const float* pred, const float* t, int batch, long long P, float* sums,
                              void* grad, float* loss_out, void* stream) {
    if (!pred || !t || !sums || !grad || batch < 1 || P < 1)
        return fail(nullptr, HELM_ERR_ARG, "bad arguments to helm_learned_loss");
    helm::launch_loss(bare_launch(stream), pred, t, batch, (int)P, sums, grad, loss_out);
    return check_launch(stream);
}

helm_status helm_fields_to_half(const void* U, long long N, int s, void* U16, void* stream) {
    if (!U || !U16 || N < 1 || s < 1) return fail(nullptr, HELM_ERR_ARG, "bad arguments to helm_fields_to_half");
    helm::launch_to_half(bare_launch(stream), static_cast<const c128*>(U), N * s, U16);
    return check_launch(stream);
}

helm_status helm_fwi_jv(helm_ctx* c, const void* fields, int fields_half, int s, const double* v,
                        const int* recv, int nrec, double tol, void* out) {
    if (!c || !fields || !v || !recv || !out || s < 1 || nrec < 1)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_fwi_jv");
    helm_status sr = check_receivers(c, recv, nrec);
    if (sr != HELM_OK) return sr;
    const long long N = c->N();
    c128 *rhs = nullptr, *w = nullptr;
    sr = alloc_pair(c, reinterpret_cast<void**>(&rhs), sizeof(c128) * (size_t)N * s, reinterpret_cast<void**>(&w),
                    sizeof(c128) * (size_t)N * s);
    if (sr != HELM_OK) return sr;
    helm::launch_jv_rhs(c->L(), fields, fields_half, N, s, c->dadm, v, rhs);
    helm_status st = helm_solve(c, rhs, s, tol, w, nullptr);
    if (st == HELM_OK || st == HELM_NOT_CONVERGED) {
        helm::launch_gather(c->L(), w, N, s, recv, nrec, nullptr, static_cast<c128*>(out));
        helm_status st2 = sync(c);
        if (st2 != HELM_OK) st = st2;
    }
    dfree(rhs);
    dfree(w);
    return st;
}

helm_status helm_fwi_jtw(helm_ctx* c, const void* fields, int fields_half, int s, const void* W,
                         const int* recv, int nrec, double tol, double* out) {
    if (!c || !fields || !W || !recv || !out || s < 1 || nrec < 1)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_fwi_jtw");
    helm_status sr = check_receivers(c, recv, nrec);
    if (sr != HELM_OK) return sr;
    const long long N = c->N();
    c128 *pw = nullptr, *lam = nullptr;
    sr = alloc_pair(c, reinterpret_cast<void**>(&pw), sizeof(c128) * (size_t)N * s, reinterpret_cast<void**>(&lam),
                    sizeof(c128) * (size_t)N * s);
    if (sr != HELM_OK) return sr;
    helm::launch_scatter(c->L(), static_cast<const c128*>(W), N, s, recv, nrec, pw);
    helm_status st = helm_adjoint(c, pw, s, tol, lam, nullptr);
    if (st == HELM_OK || st == HELM_NOT_CONVERGED) {
        helm::launch_grad(c->L(), fields, fields_half, lam, N, s, c->dadm, out);
        helm_status st2 = sync(c);
        if (st2 != HELM_OK) st = st2;
    }
    dfree(pw);
    dfree(lam);
    return st;
}

helm_status helm_fwi_gradient(helm_ctx* c, const void* Q, int s, const void* d_obs, const int* recv,
                              int nrec, double tol, int store_half, double* grad, double* misfit,
                              void* U_out) {
    if (!c || !Q || !d_obs || !recv || !grad || s < 1 || nrec < 1)
        return fail(c, HELM_ERR_ARG, "bad arguments to helm_fwi_gradient");
    helm_status sr = check_receivers(c, recv, nrec);
    if (sr != HELM_OK) return sr;
    const long long N = c->N();
    c128 *U = nullptr, *D = nullptr;
    void* U16 = nullptr;
    sr = alloc_pair(c, reinterpret_cast<void**>(&U), sizeof(c128) * (size_t)N * s, reinterpret_cast<void**>(&D),
                    sizeof(c128) * (size_t)nrec * s);
    if (sr != HELM_OK) return sr;
    helm_status st = helm_solve(c, Q, s, tol, U, nullptr);
    if (st == HELM_OK || st == HELM_NOT_CONVERGED) {
        helm::launch_gather(c->L(), U, N, s, recv, nrec, static_cast<const c128*>(d_obs), D);
        if (misfit) {
            std::vector<c128> hD((size_t)nrec * s);
            cudaMemcpyAsync(hD.data(), D, sizeof(c128) * hD.size(), cudaMemcpyDeviceToHost, c->st);
            helm_status st2 = sync(c);
            if (st2 != HELM_OK) st = st2;
            double phi = 0.0;
            for (auto& v : hD) phi += v.re * v.re + v.im * v.im;
            *misfit = 0.5 * phi;
        }
        const void* fields = U;
        if (store_half) {
            // keep the forward fields in 16 bits (32 bits per complex unknown)
            if (dalloc(&U16, sizeof(float) * (size_t)N * s) == cudaSuccess) {
                helm::launch_to_half(c->L(), U, N * s, U16);
                fields = U16;
            }
        }
        if (U_out) cudaMemcpyAsync(U_out, U, sizeof(c128) * (size_t)N * s, cudaMemcpyDeviceToDevice, c->st);
        helm_status st3 = helm_fwi_jtw(c, fields, U16 ? 1 : 0, s, D, recv, nrec, tol, grad);
        if (st3 != HELM_OK && st == HELM_OK) st = st3;
    }
    dfree(U);
    dfree(D);
    dfree(U16);
    return st;
}

int helm_profile_kernel_count(void) { return helm::KID_COUNT; }

const char* helm_profile_kernel_name(int kid) {
    return (kid >= 0 && kid < helm::KID_COUNT) ? kKernelNames[kid] : "";
}

helm_status helm_profile_read(helm_ctx* c, int kid, double* time_ms, long long* launches,
                              double* bytes, double* flops) {
    if (!c || !c->prof || kid < 0 || kid >= helm::KID_COUNT)
        return fail(c, HELM_ERR_ARG, "profiling is off or bad kernel id");
    c->prof->resolve();
    if (time_ms) *time_ms = c->prof->time_ms[kid];
    if (launches) *launches = c->prof->launches[kid];
    if (bytes) *bytes = c->prof->bytes[kid];
    if (flops) *flops = c->prof->flops[kid];
    return HELM_OK;
}

}  // extern "C"
