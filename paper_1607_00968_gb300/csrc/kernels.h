// Host-side launchers of the libhelm kernels (instantiated in mg.cu and
// krylov.cu, called by the solver driver in solver.cu).
#pragma once
#include <string>
#include "common.cuh"

namespace helm {

// ---------------- multigrid (mg.cu) ----------------

// y = Op x  (T: arithmetic precision; U: input element; V: output element)
template <typename T, typename U, typename V, typename Op>
void launch_apply(const Launch& L, const Op& op, const cplx<U>* x, cplx<V>* y, int s);
// y = A x on the fine grid, x complex64, in double-float arithmetic (1/h^2
// and the mass coefficients cdd as float pairs), y written as an FMT_DD block
// (two complex64 planes of N*s, hi then lo); needs s <= 512
void launch_apply_dd(const Launch& L, const Grid& g, double inv_h2, const float4* cdd, const c64* x,
                     c64* y, int s);
// complex128 values -> float pairs (re hi, re lo, im hi, im lo)
void launch_split_pairs(const Launch& L, const c128* in, float4* out, long long n);

// r = b - Op x
template <typename T, typename Op>
void launch_residual(const Launch& L, const Op& op, const cplx<T>* x, const cplx<T>* b,
                     cplx<T>* r, int s);

// u_out = u_in + w D^{-1} (f - Op u_in); u_in == nullptr means u_in = 0.
template <typename T, typename FT, typename Op>
void launch_jacobi(const Launch& L, const Op& op, const cplx<T>* u_in, const cplx<FT>* f,
                   cplx<T>* u_out, int s, T w);

// rc = P^T (f - Op u) on the coarse grid gc; u == nullptr means u = 0.
template <typename T, typename FT, typename Op>
void launch_resid_restrict(const Launch& L, const Op& op, const Grid& gc, const cplx<T>* u,
                           const cplx<FT>* f, cplx<T>* rc, int s);

// out[j] = sum_node conj(a) b per column (double accumulation; s <= 256),
// deterministic: per-CTA sums in part (kColdotBlocks x s) added in block
// order by the last CTA, which resets *count (zero before the first call);
// at most kColdotBlocks CTAs (two per SM), the size of `part`
constexpr int kColdotBlocks = 1024;
template <typename T>
void launch_coldot(const Launch& L, const cplx<T>* a, const cplx<T>* b, long long N, int s, double2* out,
                   double2* part, unsigned int* count);
// y[:, j] += sign * (num_j / den_j.x) x[:, j]
template <typename T>
void launch_kc_axpy(const Launch& L, cplx<T>* y, const cplx<T>* x, const double2* num,
                    const double2* den, double sign, long long N, int s);
// y += x (n complex values)
template <typename T>
void launch_axpy(const Launch& L, cplx<T>* y, const cplx<T>* x, long long n);

// u += P ec
template <typename T>
void launch_prolong_add(const Launch& L, const Grid& gf, const Grid& gc, const cplx<T>* ec,
                        cplx<T>* u, int s);

// u = Minv f  (Minv: n x n row-major; f, u: n x s node-major)
template <typename T>
void launch_dense_apply(const Launch& L, const cplx<T>* Minv, int n, const cplx<T>* f,
                        cplx<T>* u, int s);

// ---------------- coarsest solve on the tensor cores (dense_tc.cu) ----------------

// padded K (= 2 nc rounded up to the K tile), B' row length, K-split factor,
// and the scratch (floats) one launch needs for nc coarse nodes and s columns
int dense_tc_kpad(int nc);
int dense_tc_ldb(int s);
int dense_tc_ksplit(int nc, int s);
size_t dense_tc_scratch_floats(int nc, int s);
// A' in a buffer of nc x dense_tc_kpad(nc) floats: interleaved (re, im) of
// Minv; split3: FP32 (the three-product solve splits it itself); otherwise
// FP16 scaled by a power of two (max |A'| = 2^13) in the first half, the
// scale as a float right after it
void launch_build_aprime(const Launch& L, const c128* Minv, int nc, float* Ap, bool split3);
// u = Minv f for complex64 blocks (nc x s, node-major) from A'; split3: three
// tf32 products on hi/lo splits (FP32-class accuracy); otherwise one FP16
// product (11 significant bits, scaled per right-hand side)
void launch_dense_tc(const Launch& L, const float* Ap, int nc, const c64* f, c64* u, int s,
                     float* scratch, int mode);
// mode of launch_dense_tc: 0 = FP16 product on tcgen05 (TMA-fed, TMEM
// accumulator), 1 = three tf32 products (mma.sync), 2 = FP16 product on
// mma.sync (the earlier kernel, kept for comparison)
int dense_tc05_ksplit(int nc, int s);
// 1 if a tcgen05 coarsest product gave up waiting on its pipeline (or could
// not build its tensor maps) since the last call; clears the flag
int dense_tc_take_error(cudaStream_t st);

// ---------------- learned stage (learned.cu) ----------------

// y = epilogue(conv3x3(x; w) + bias), NHWC bf16 activations, [co][tap][ci] bf16
// weights, FP32 accumulation on the tensor cores; (cin, cout) in
// {(16,32), (32,32), (32,16), (16,16)}; returns false for other shapes.
bool launch_conv3x3(const Launch& L, const void* x, int B, int H, int W, int cin, const void* w,
                    const float* bias, int cout, int relu, const void* mask, void* y, int y_float);
// dw[co][tap][ci] += sum gy x[shifted], db[co] += sum gy (FP32, atomics)
bool launch_conv3x3_wgrad(const Launch& L, const void* x, const void* gy, int B, int H, int W, int cin,
                          int cout, float* dw, float* db);
// wf[ci][tap][co] = w[co][8 - tap][ci] for ci < cin, zero up to cin_pad_out
void launch_flip_weights(const Launch& L, const void* w, int cin, int cout, void* wf, int cin_pad_out);
void launch_adam(const Launch& L, float* p, const float* g, float* m, float* v, void* pb, int n,
                 float lr, float b1, float b2, float eps, int step);
void launch_pack_input(const Launch& L, const c64* r, int N, int s, const float* rho,
                       const float* kappa, void* out);
void launch_unpack_add(const Launch& L, const float* out, int N, int s, const float* rho, float scale,
                       c64* z);
// kappa[i] = Re(cA[i]) h^2 = omega^2 m_i h^2 (the network's third input channel)
void launch_kappa(const Launch& L, const c128* cA, long long N, double h2, float* kappa);
// residual-loss training inputs (image order, float pairs): r / rho and h^2 c_A
void launch_pack_resid(const Launch& L, const c64* r, int N, int s, const float* rho, const c128* cA,
                       double h2, float* rimg, float* cimg);
// loss = mean_b ||rt_b - h^2 A pred_b||^2 / ||rt_b||^2 and its gradient (bf16, 16 channels)
void launch_residual_loss(const Launch& L, const float* pred, const float* rt, const float* coef, int B, int H,
                          int W, float* q, float* sums, void* grad, float* loss_out);
void launch_image_to_block(const Launch& L, const float* rimg, long long N, int s, c128* v);
void launch_pack_target(const Launch& L, const c64* e, int N, int s, const float* rho, float scale,
                        float* t);
// loss = mean_b ||pred_b - t_b||^2 / ||t_b||^2 over channels 0, 1 (pred: 16-channel
// float NHWC, t: 2-channel float), grad (bf16, 16 channels) and loss_out (device float)
void launch_loss(const Launch& L, const float* pred, const float* t, int B, int P, float* sums,
                 void* grad, float* loss_out);
// z1[:, j] = z2[:, j] where sum |r2|^2 (r2sq[j]) < N rho1[j]^2
void launch_select_better(const Launch& L, const c64* z2, c64* z1, long long N, int s,
                          const float* rho1, const float* r2sq);
// r = f - A z (complex64) and rho[j] = RMS of column j of r
void launch_learned_residual(const Launch& L, const FineOp<float>& op, const c128* f, const c64* z,
                             c64* r, int s, float* rho2, float* rho);

// ---------------- FWI sensitivity products (fwi.cu) ----------------

// dadm[k] = w^2 (1 - i g_k) (minus the derivative of A's diagonal w.r.t. m)
void launch_dadm(const Launch& L, const double* gamma, double omega, long long N, c128* dadm);
// complex128 -> 16-bit pairs (half re, half im)
void launch_to_half(const Launch& L, const c128* u, long long n, void* u16);
// rhs = dadm * u * v (ABI layout, s columns)
void launch_jv_rhs(const Launch& L, const void* fields, int half, long long N, int s, const c128* dadm,
                   const double* v, c128* rhs);
// out[j][r] = X[j][recv[r]] - d[j][r] (d may be null)
void launch_gather(const Launch& L, const c128* X, long long N, int s, const int* recv, int nrec,
                   const c128* d, c128* out);
// out = P W (zeroed first; repeated receivers add)
void launch_scatter(const Launch& L, const c128* W, long long N, int s, const int* recv, int nrec,
                    c128* out);
// g[k] = sum_j Re(conj(dadm_k u_jk) lam_jk)
void launch_grad(const Launch& L, const void* fields, int half, const c128* lam, long long N, int s,
                 const c128* dadm, double* g);

// ---------------- set-up (mg.cu) ----------------

// c_A = omega^2 m (1 - i gamma), c_M = omega^2 m (1 - i (gamma + shift)),
// dinv_M = 1 / (2d/h^2 - c_M); also the K-point FP64 stencil of M (coef_M).
void launch_fine_setup(const Launch& L, const Grid& g, const double* m, const double* gamma,
                       double omega, double shift, double inv_h2, c128* cA, c128* cM,
                       c128* dinvM, c128* coefM);

// coarse K-point stencil = P^T (fine K-point stencil) P
void launch_galerkin(const Launch& L, const Grid& gf, const Grid& gc, const c128* coef_f,
                     c128* coef_c);

// dinv[i] = 1 / coef[i*K + centre]
void launch_diag_inv(const Launch& L, const Grid& g, const c128* coef, c128* dinv);

// dense n x n matrix (row-major) of a K-point stencil
void launch_stencil_to_dense(const Launch& L, const Grid& g, const c128* coef, c128* dense);

// Gauss-Jordan inversion with partial pivoting of the dense n x n matrix
// `dense` (row-major, complex128) in arithmetic T (double or float): aug is
// n x 2n scratch of cplx<T>, factor n of cplx<T>, pivval one cplx<T>;
// `inverse` (n x n complex128) receives the result; status (device int) is
// set to 1 if a zero pivot is met.
template <typename T>
void launch_gauss_jordan(const Launch& L, const c128* dense, void* aug, int n, void* factor, int* piv,
                         void* pivval, int* status, c128* inverse);

void launch_round_c64(const Launch& L, const c128* in, c64* out, long long count);

// ---------------- Krylov / layout (krylov.cu) ----------------

// internal[node*s + j] = (conj?) abi[j*N + node]
void launch_to_internal(const Launch& L, const c128* abi, c128* internal, long long N, int s,
                        bool conjugate);
void launch_from_internal(const Launch& L, const c128* internal, c128* abi, long long N, int s,
                          bool conjugate);

// Storage formats of a block of N*s complex values for the double-float
// Krylov kernels: FMT_C128 complex128; FMT_DD an unevaluated float pair per
// component in two complex64 planes (hi at [0, N*s), lo at [N*s, 2*N*s) in
// complex64 units: 16 bytes per value, like complex128); FMT_C64 complex64.
enum : int { FMT_C128 = 0, FMT_DD = 1, FMT_C64 = 2 };
// true when the double-float Gram and combination kernels cover (s, sb), the
// condition for keeping a Krylov basis in FMT_DD
bool dd_formats_ok(int s, int sb);

// Block Gram per group:  out[i][g][a][b] = sum_node conj(X_i[node][g*sb+a]) Y[node][g*sb+b]
// for i < nb (X_i = X + i*xstride).  partial: scratch of gram_partial_elems().
long long gram_partial_elems(long long N, int nb, int s, int sb);
// bytes at the start of that scratch that must be zero before its first use
long long gram_scratch_zero_bytes();
// emulate: double-float arithmetic on the FP32 pipes instead of FP64.
void launch_gram(const Launch& L, const c128* X, int nb, long long xstride, const c128* Y,
                 long long N, int s, int sb, c128* partial, c128* out, bool emulate);

// Same with the operands' formats (xstride in elements of X's format: 16
// bytes for FMT_C128 and FMT_DD, 8 for FMT_C64).  FMT_DD needs emulate.
// hi_only (both FMT_DD, groups of four): products of the hi parts in FP32,
// for a first Gram-Schmidt pass whose error a double-float pass removes.
void launch_gram_f(const Launch& L, const void* X, int xf, int nb, long long xstride, const void* Y,
                   int yf, long long N, int s, int sb, c128* partial, c128* out, bool emulate,
                   bool hi_only = false);

// out[node][g*sb+b] = beta*out + sign * sum_{i<nb} sum_a X_i[node][g*sb+a] C[i][g][a][b]
// emulate: double-float arithmetic (needs csplit: scratch of nb*G*sb*sb float4
// for the split coefficients; falls back to FP64 when null).
template <typename TX>
void launch_combine(const Launch& L, c128* out, double beta, double sign, const cplx<TX>* X,
                    int nb, long long xstride, const c128* C, long long N, int s, int sb,
                    bool emulate, float4* csplit);

// Same with formats; an FMT_DD output or X needs emulate and
// dd_formats_ok(s, sb), and an FMT_DD output beta in {0, 1}, sign = +-1.
// hi_only (FMT_DD in and out, groups of four, beta = 1): out = base + sign X C
// with the product in FP32 from the hi parts, for corrections whose
// coefficients are small (a second Gram-Schmidt update, a QR factor near the
// identity minus the identity); added to the pairs of base (null: out) exactly.
void launch_combine_f(const Launch& L, void* out, int of, double beta, double sign, const void* X,
                      int xf, int nb, long long xstride, const c128* C, long long N, int s, int sb,
                      bool emulate, float4* csplit, bool hi_only = false, const void* base = nullptr);

// per-column squared 2-norms of X (N x s node-major): out[j] (FP64)
long long colnorm_partial_elems(long long N, int s);
void launch_colnorm2(const Launch& L, const c128* X, long long N, int s, double* partial,
                     double* out);

// X[node][j] = random complex (counter-based hash of (seed, node, j)) for
// columns with mask[j] != 0; other columns untouched.
void launch_fill_random(const Launch& L, c128* X, long long N, int s, const int* mask,
                        unsigned long long seed);
void launch_fill_random_f(const Launch& L, void* X, int of, long long N, int s, const int* mask,
                          unsigned long long seed);

void launch_zero(const Launch& L, void* p, size_t bytes);

// the message helm_last_error(NULL) returns on this thread
void set_thread_error(const std::string& msg);

}  // namespace helm
