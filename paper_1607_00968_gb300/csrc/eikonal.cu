// Factored eikonal equation, fast marching and its sensitivities (Sec. 2.5,
// Eq. factoredeikonal, Eq. Gudonov, Eq. FOfactoredD, Algorithm "Fast
// Marching", Eq. Sensitivity / Sensitivity2).
//
// tau = tau0 * tau1, tau0 = |x - x_s|, p0 = grad tau0.  Along each axis the
// first-order factored derivatives at node i are
//     D- tau1 = tau0_i (tau1_i - tau1_{i-e}) / h + p0_i tau1_i,
//     D+ tau1 = tau0_i (tau1_{i+e} - tau1_i) / h + p0_i tau1_i,
// and the Godunov equation sum_axes max{D-, -D+, 0}^2 = m_i is solved by fast
// marching: the front node of least tau (ties: lower node index) is accepted
// and the equation is re-solved at its unaccepted neighbours from accepted
// values only.  The local solve takes, over every choice per axis (none,
// backward, forward), the larger root of the resulting quadratic, and keeps
// the least root that is consistent with the max{} (each chosen term >= 0 and
// >= its axis' other known term, no positive term on an unchosen axis); with
// none consistent (only through rounding), the least root with non-negative
// chosen terms.  The source node is known from the start with tau1 = sqrt(m).
//
// GB300 mapping: sources are independent, so each source's fast marching
// runs on its own CTA (a serial heap walk: the method's order is inherently
// sequential), all sources at once.  Every floating-point decision (the
// local solve, the heap key tau0 * tau1) uses IEEE double operations rounded
// once each in a fixed order (the _rn intrinsics, no contraction), so the
// acceptance order and the chosen derivatives are a deterministic function of
// the inputs.  The sensitivity products are wavefront-parallel: each node's
// row refers only to the neighbours its derivatives chose, which fast marching
// accepted earlier, so with level(node) = 1 + max level of those neighbours
// all nodes of one level are independent; a CTA per source walks the levels
// (forward substitution for J v, backward for J^T w) with a barrier between
// levels.  tau1 is kept in single precision for the products, as the paper
// stores it.
#include <cmath>
#include <string>
#include <vector>

#include "helm.h"
#include "kernels.h"

namespace {

constexpr unsigned char kFar = 0, kFront = 1, kKnown = 2;
constexpr unsigned char kSourceDir = 0xFF;

// grid in numpy axis order: axis 0 slowest, axis d-1 = x1 (stride 1)
struct EikGrid {
    int d;
    int S[3];
    long long st[3];
    long long N;
    double h;
};

struct HeapEnt {
    double key;
    long long idx;
};

__device__ __forceinline__ bool heap_less(const HeapEnt& a, const HeapEnt& b) {
    return a.key < b.key || (a.key == b.key && a.idx < b.idx);
}

__device__ __forceinline__ void unflatten(const EikGrid& g, long long i64, int* k) {
    k[0] = k[1] = k[2] = 0;
    unsigned int i = (unsigned int)i64;           // N < 2^31
    for (int a = g.d - 1; a >= 0; --a) {
        const unsigned int sa = (unsigned int)g.S[a];
        k[a] = (int)(i % sa);
        i /= sa;
    }
}

// tau0 = h |k - s| and p0 = (k - s) h / tau0 (0 at the source), per axis in
// numpy order, each operation rounded once in this order
__device__ void tau0_p0(const EikGrid& g, const int* k, const int* s, double& t0, double* p0) {
    double diff[3];
    double r2 = 0.0;
    for (int a = 0; a < g.d; ++a) {
        diff[a] = __dmul_rn(g.h, (double)(k[a] - s[a]));
        r2 = __dadd_rn(r2, __dmul_rn(diff[a], diff[a]));
    }
    t0 = __dsqrt_rn(r2);
    for (int a = 0; a < g.d; ++a) p0[a] = t0 > 0.0 ? __ddiv_rn(diff[a], t0) : 0.0;
}

// Marching state of one node, 32 bytes: one load brings all a node's fields.
struct __align__(16) NodeRec {
    double tau1;          // FP64 working value
    double key;           // last pushed heap key, tau0 tau1
    double m;             // squared slowness
    int level;            // wavefront level
    unsigned char state;  // far / front / known
    unsigned char dir;    // chosen derivatives
    unsigned short pad;
};

struct SrcArrays {
    NodeRec* rec;          // N
    unsigned char* dir;    // N, compact copy for the sensitivities
    int* order;            // N, acceptance order
    int* nodes;            // N, nodes grouped by level
    int* ptr;              // N + 1, level starts
    float* tau1f;          // N, single-precision tau1 for the sensitivities
    HeapEnt* heap;         // cap
};

__host__ __device__ inline long long src_bytes(long long N, long long cap) {
    const long long per = 16 * cap + 32 * N + 4 * N * 3 + 4 * (N + 1) + N + 64;
    return (per + 255) / 256 * 256;
}

__device__ SrcArrays src_arrays(char* base, long long N, long long cap, int b) {
    char* p = base + (long long)b * src_bytes(N, cap);
    SrcArrays s;
    s.heap = reinterpret_cast<HeapEnt*>(p); p += 16 * cap;
    s.rec = reinterpret_cast<NodeRec*>(p); p += 32 * N;
    s.order = reinterpret_cast<int*>(p); p += 4 * N;
    s.nodes = reinterpret_cast<int*>(p); p += 4 * N;
    s.tau1f = reinterpret_cast<float*>(p); p += 4 * N;
    s.ptr = reinterpret_cast<int*>(p); p += 4 * (N + 1);
    s.dir = reinterpret_cast<unsigned char*>(p);
    return s;
}

// Nodes within L1 distance 2 of an accepted node (origin first): its
// neighbours and theirs.  kLut maps an offset (o + 2 per axis, base 5) to
// its slot.
__constant__ signed char kOff2[13][2] = {{0, 0}, {-1, 0}, {0, -1}, {0, 1}, {1, 0}, {-2, 0}, {-1, -1}, {-1, 1}, {0, -2}, {0, 2}, {1, -1}, {1, 1}, {2, 0}};
__constant__ signed char kLut2[25] = {-1, -1, 5, -1, -1, -1, 6, 1, 7, -1, 8, 2, 0, 3, 9, -1, 10, 4, 11, -1, -1, -1, 12, -1, -1};
__constant__ signed char kOff3[25][3] = {{0, 0, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}, {0, 0, 1}, {0, 1, 0}, {1, 0, 0}, {-2, 0, 0}, {-1, -1, 0}, {-1, 0, -1}, {-1, 0, 1}, {-1, 1, 0}, {0, -2, 0}, {0, -1, -1}, {0, -1, 1}, {0, 0, -2}, {0, 0, 2}, {0, 1, -1}, {0, 1, 1}, {0, 2, 0}, {1, -1, 0}, {1, 0, -1}, {1, 0, 1}, {1, 1, 0}, {2, 0, 0}};
__constant__ signed char kLut3[125] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 7, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 8, -1, -1, -1, 9, 1, 10, -1, -1, -1, 11, -1, -1, -1, -1, -1, -1, -1, -1, -1, 12, -1, -1, -1, 13, 2, 14, -1, 15, 3, 0, 4, 16, -1, 17, 5, 18, -1, -1, -1, 19, -1, -1, -1, -1, -1, -1, -1, -1, -1, 20, -1, -1, -1, 21, 6, 22, -1, -1, -1, 23, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 24, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};

template <int D> struct Hood;
template <> struct Hood<2> {
    static constexpr int n = 13;
    __device__ static int off(int j, int a) { return kOff2[j][a]; }
    __device__ static int slot(const int* o) { return kLut2[(o[0] + 2) * 5 + (o[1] + 2)]; }
};
template <> struct Hood<3> {
    static constexpr int n = 25;
    __device__ static int off(int j, int a) { return kOff3[j][a]; }
    __device__ static int slot(const int* o) { return kLut3[((o[0] + 2) * 5 + (o[1] + 2)) * 5 + (o[2] + 2)]; }
};

// ---------------------------------------------------------------------------
// Warp-cooperative fast marching: one warp per source.  Lane 0 owns the heap
// (in shared memory, or in global memory for fronts larger than it holds);
// for each accepted node the 2D neighbours x (3^D - 1) derivative choices are
// solved by the 32 lanes side by side, and lane n (n < 2D) then picks the
// least consistent root of neighbour n in the enumeration order -- the same
// values and the same decisions as the serial local solve.
// ---------------------------------------------------------------------------
template <int D>
struct Pow3 { static constexpr int v = 3 * Pow3<D - 1>::v; };
template <>
struct Pow3<0> { static constexpr int v = 1; };

struct Cand {
    double x;     // root (INFINITY when the choice is unavailable or has no real root)
    int ok;       // consistent with the max{}
    int okp;      // chosen terms non-negative
};

// The terms alpha x - beta of one node's known neighbours, per axis and
// direction (0 backward, 1 forward): alpha = tau0/h +- p0, beta = (tau0/h) tau1_nb.
template <int D>
struct Terms {
    double al[D][2], be[D][2];
    int has;          // bit 2a + dir
    double mi;
};

// The terms of neighbour q = i + e (slot jq of the neighbourhood table hood,
// offset oq from i); hood entries of nodes outside the grid have state 0xFF.
template <int D>
__device__ void make_terms(const EikGrid& g, const int* kq, const int* oq, const int* s,
                           const NodeRec* hood, Terms<D>& T) {
    double t0, p0[3];
    tau0_p0(g, kq, s, t0, p0);
    const double t0h = __ddiv_rn(t0, g.h);
    T.has = 0;
    T.mi = hood[Hood<D>::slot(oq)].m;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        T.al[a][0] = T.al[a][1] = T.be[a][0] = T.be[a][1] = 0.0;
        int o[3] = {oq[0], oq[1], oq[2]};
        o[a] -= 1;
        if (kq[a] > 0) {
            const NodeRec& r = hood[Hood<D>::slot(o)];
            if (r.state == kKnown) {
                T.al[a][0] = __dadd_rn(t0h, p0[a]);
                T.be[a][0] = __dmul_rn(t0h, r.tau1);
                T.has |= 1 << (2 * a);
            }
        }
        o[a] += 2;
        if (kq[a] < g.S[a] - 1) {
            const NodeRec& r = hood[Hood<D>::slot(o)];
            if (r.state == kKnown) {
                T.al[a][1] = __dsub_rn(t0h, p0[a]);
                T.be[a][1] = __dmul_rn(t0h, r.tau1);
                T.has |= 1 << (2 * a + 1);
            }
        }
    }
}

// One derivative choice t (1 .. 3^D - 1, axis 0 slowest) from the terms.
template <int D>
__device__ Cand combo_solve(const Terms<D>& T, int t) {
    Cand r{INFINITY, 0, 0};
    int c[D];
    int rr = t;
#pragma unroll
    for (int a = D - 1; a >= 0; --a) { c[a] = rr % 3; rr /= 3; }
#pragma unroll
    for (int a = 0; a < D; ++a)
        if (c[a] && !((T.has >> (2 * a + c[a] - 1)) & 1)) return r;
    double A = 0.0, B = 0.0, C = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
        if (c[a]) {
            const double l = T.al[a][c[a] - 1], bb = T.be[a][c[a] - 1];
            A = __dadd_rn(A, __dmul_rn(l, l));
            B = __dadd_rn(B, __dmul_rn(l, bb));
            C = __dadd_rn(C, __dmul_rn(bb, bb));
        }
    C = __dsub_rn(C, T.mi);
    if (A <= 0.0) return r;
    const double disc = __dsub_rn(__dmul_rn(B, B), __dmul_rn(A, C));
    if (disc < 0.0) return r;
    const double x = __ddiv_rn(__dadd_rn(B, __dsqrt_rn(disc)), A);
    bool ok = true, okp = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (c[a]) {
            const double f = __dsub_rn(__dmul_rn(T.al[a][c[a] - 1], x), T.be[a][c[a] - 1]);
            if (f < 0.0) { okp = false; ok = false; }
            const int o = 2 - c[a];            // the axis' other direction (0-based)
            if (((T.has >> (2 * a + o)) & 1) && __dsub_rn(__dmul_rn(T.al[a][o], x), T.be[a][o]) > f) ok = false;
        } else {
#pragma unroll
            for (int o = 0; o < 2; ++o)
                if (((T.has >> (2 * a + o)) & 1) && __dsub_rn(__dmul_rn(T.al[a][o], x), T.be[a][o]) > 0.0)
                    ok = false;
        }
    }
    r.x = x;
    r.ok = ok;
    r.okp = okp;
    return r;
}

__device__ __forceinline__ void heap_push(HeapEnt* heap, long long& size, HeapEnt e) {
    long long p = size++;
    while (p > 0) {
        const long long par = (p - 1) / 2;
        if (!heap_less(e, heap[par])) break;
        heap[p] = heap[par];
        p = par;
    }
    heap[p] = e;
}

__device__ __forceinline__ HeapEnt heap_pop(HeapEnt* heap, long long& size) {
    const HeapEnt top = heap[0];
    const HeapEnt last = heap[--size];
    long long pos = 0;
    while (true) {
        long long c = 2 * pos + 1;
        if (c >= size) break;
        if (c + 1 < size && heap_less(heap[c + 1], heap[c])) ++c;
        if (!heap_less(heap[c], last)) break;
        heap[pos] = heap[c];
        pos = c;
    }
    if (size > 0) heap[pos] = last;
    return top;
}

constexpr long long kSmemHeap = 12288;    // heap entries in shared memory (192 KB)

// status[b]: 0 ok, 1 heap full, 2 a node was never reached.  map: the
// source of each block (null: block b is source b).  A heap entry is stale
// exactly when its key differs from the node's last pushed key (the same test
// as key != tau0 tau1: tau1 changes only together with a push).  After each
// acceptance the lanes load the records of the nodes within L1 distance 2 in
// one round trip into shared memory; the local solves read them there.
template <int D, bool SMEM>
__global__ void __launch_bounds__(32) k_fm_warp(EikGrid g, const double* __restrict__ m,
                                                 const int* __restrict__ srcs, char* base, long long cap,
                                                 const int* __restrict__ map, int* __restrict__ nlev,
                                                 int* __restrict__ status) {
    constexpr int NC = Pow3<D>::v - 1;         // derivative choices per neighbour
    constexpr int NP = 2 * D * NC;             // (neighbour, choice) pairs
    constexpr int NH = Hood<D>::n;
    extern __shared__ __align__(16) unsigned char fm_sm[];
    NodeRec* hood = reinterpret_cast<NodeRec*>(fm_sm);
    Cand* cand = reinterpret_cast<Cand*>(fm_sm + NH * sizeof(NodeRec));
    Terms<D>* terms = reinterpret_cast<Terms<D>*>(reinterpret_cast<unsigned char*>(cand) +
                                                  ((NP * sizeof(Cand) + 15) / 16) * 16);
    HeapEnt* heap = SMEM ? reinterpret_cast<HeapEnt*>(reinterpret_cast<unsigned char*>(terms) +
                                                      ((2 * D * sizeof(Terms<D>) + 15) / 16) * 16)
                         : nullptr;
    const int lane = threadIdx.x;
    const int b = map ? map[blockIdx.x] : blockIdx.x;
    SrcArrays A = src_arrays(base, g.N, cap, b);
    if (!SMEM) heap = A.heap;
    const long long hcap = SMEM ? kSmemHeap : cap;
    for (long long i = lane; i < g.N; i += 32) {
        NodeRec r;
        r.tau1 = INFINITY;
        r.key = 0.0;
        r.m = m[i];
        r.level = 0;
        r.state = kFar;
        r.dir = 0;
        r.pad = 0;
        A.rec[i] = r;
    }
    for (long long i = lane; i <= g.N; i += 32) A.ptr[i] = 0;
    const int* s = srcs + 3 * b;
    long long si = 0;
    for (int a = 0; a < D; ++a) si += (long long)s[a] * g.st[a];
    __syncwarp();
    long long size = 0;
    if (lane == 0) {
        A.rec[si].tau1 = __dsqrt_rn(m[si]);
        A.rec[si].dir = kSourceDir;
        A.rec[si].state = kFront;
        A.rec[si].key = 0.0;
        heap[size++] = HeapEnt{0.0, si};
    }
    long long nacc = 0;
    int st = 0;
    while (true) {
        // lane 0: next valid node (stale entries skipped)
        long long i = -1;
        if (lane == 0) {
            while (size > 0) {
                const HeapEnt top = heap_pop(heap, size);
                const NodeRec r = A.rec[top.idx];
                if (r.state == kKnown || top.key != r.key) continue;
                i = top.idx;
                A.rec[i].state = kKnown;
                A.order[nacc] = (int)i;
                break;
            }
        }
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i < 0) break;
        ++nacc;
        int k[3];
        unflatten(g, i, k);
        __syncwarp();
        // the neighbourhood records
        if (lane < NH) {
            bool inside = true;
            long long node = i;
            for (int a = 0; a < D; ++a) {
                const int o = Hood<D>::off(lane, a);
                const int kk = k[a] + o;
                if (kk < 0 || kk >= g.S[a]) inside = false;
                node += (long long)o * g.st[a];
            }
            NodeRec r;
            if (inside) r = A.rec[node];
            else { r.tau1 = INFINITY; r.key = 0.0; r.m = 0.0; r.level = 0; r.state = 0xFF; r.dir = 0; r.pad = 0; }
            if (lane == 0) r.state = kKnown;
            hood[lane] = r;
        }
        __syncwarp();
        // lanes n < 2D: the terms of neighbour n (if it is inside and not known)
        if (lane < 2 * D) {
            const int a = lane >> 1, step = (lane & 1) ? 1 : -1;
            Terms<D>& T = terms[lane];
            T.has = 0;
            const int kk = k[a] + step;
            if (kk >= 0 && kk < g.S[a]) {
                int oq[3] = {0, 0, 0};
                oq[a] = step;
                if (hood[Hood<D>::slot(oq)].state != kKnown) {
                    int kq[3] = {k[0], k[1], k[2]};
                    kq[a] = kk;
                    make_terms<D>(g, kq, oq, s, hood, T);
                }
            }
        }
        __syncwarp();
        for (int p = lane; p < NP; p += 32) {
            const int nbr = p / NC, t = p - nbr * NC + 1;
            const Terms<D>& T = terms[nbr];
            cand[p] = T.has ? combo_solve<D>(T, t) : Cand{INFINITY, 0, 0};
        }
        __syncwarp();
        // lane n < 2D: neighbour n takes the least consistent root, choices in order
        HeapEnt push{0.0, -1};
        if (lane < 2 * D && terms[lane].has) {
            const int a = lane >> 1, step = (lane & 1) ? 1 : -1;
            const long long q = i + step * g.st[a];
            int oq[3] = {0, 0, 0};
            oq[a] = step;
            const NodeRec rq = hood[Hood<D>::slot(oq)];
            double best = INFINITY, fb = INFINITY;
            int bt = 0, ft = 0;
            for (int t = 1; t <= NC; ++t) {
                const Cand r = cand[lane * NC + t - 1];
                if (r.ok && r.x < best) { best = r.x; bt = t; }
                if (r.okp && r.x < fb) { fb = r.x; ft = t; }
            }
            const double x = bt ? best : fb;
            const int t = bt ? bt : ft;
            if (t && x < rq.tau1) {
                int c[D], code = 0;
                int rr = t;
                for (int ax = D - 1; ax >= 0; --ax) { c[ax] = rr % 3; rr /= 3; }
                int lv = 0;
                for (int ax = 0; ax < D; ++ax) {
                    code |= c[ax] << (2 * ax);
                    if (c[ax]) {
                        int o[3] = {oq[0], oq[1], oq[2]};
                        o[ax] += c[ax] == 1 ? -1 : 1;
                        lv = max(lv, hood[Hood<D>::slot(o)].level);
                    }
                }
                int kq[3] = {k[0], k[1], k[2]};
                kq[a] += step;
                double t0q, p0q[3];
                tau0_p0(g, kq, s, t0q, p0q);
                const double key = __dmul_rn(t0q, x);
                NodeRec nr = rq;
                nr.tau1 = x;
                nr.key = key;
                nr.level = lv + 1;
                nr.state = kFront;
                nr.dir = (unsigned char)code;
                A.rec[q] = nr;
                push = HeapEnt{key, q};
            }
        }
        // lane 0 pushes the updated neighbours
        for (int n = 0; n < 2 * D; ++n) {
            const double key = __shfl_sync(0xffffffffu, push.key, n);
            const long long q = __shfl_sync(0xffffffffu, push.idx, n);
            if (lane == 0 && q >= 0) {
                if (size >= hcap) st = 1;
                else heap_push(heap, size, HeapEnt{key, q});
            }
        }
        st = __shfl_sync(0xffffffffu, st, 0);
        if (st) break;
        __syncwarp();
    }
    nacc = __shfl_sync(0xffffffffu, nacc, 0);
    if (!st && nacc != g.N) st = 2;
    if (st) {
        if (lane == 0) { status[b] = st; nlev[b] = 0; }
        return;
    }
    // compact copies for the sensitivities (all lanes), then the level
    // grouping (lane 0: a counting sort, stable in acceptance order)
    for (long long n = lane; n < g.N; n += 32) {
        const NodeRec r = A.rec[n];
        A.tau1f[n] = __double2float_rn(r.tau1);
        A.dir[n] = r.dir;
    }
    __syncwarp();
    if (lane != 0) return;
    status[b] = 0;
    int maxlev = 0;
    for (long long n = 0; n < g.N; ++n) {
        const int lv = A.rec[n].level;
        maxlev = max(maxlev, lv);
        A.ptr[lv + 1] += 1;
    }
    for (int l = 0; l <= maxlev; ++l) A.ptr[l + 1] += A.ptr[l];
    for (long long n = 0; n < g.N; ++n) {
        const int node = A.order[n];
        A.nodes[A.ptr[A.rec[node].level]++] = node;
    }
    for (int l = maxlev; l >= 1; --l) A.ptr[l] = A.ptr[l - 1];
    A.ptr[0] = 0;
    nlev[b] = maxlev + 1;
}

template <int D>
size_t fm_smem(bool smem_heap) {
    constexpr int NP = 2 * D * (Pow3<D>::v - 1);
    size_t c = Hood<D>::n * sizeof(NodeRec) + ((NP * sizeof(Cand) + 15) / 16) * 16 +
               ((2 * D * sizeof(Terms<D>) + 15) / 16) * 16;
    return c + (smem_heap ? (size_t)kSmemHeap * sizeof(HeapEnt) : 0);
}

// tau (= tau0 tau1), tau1, the order and the directions of each source
__global__ void k_eik_outputs(EikGrid g, const int* __restrict__ srcs, char* base, long long cap, int ns,
                              double* tau, double* tau1, int* order, unsigned char* dir) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)ns * g.N;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / g.N);
        const long long i = e - (long long)b * g.N;
        SrcArrays A = src_arrays(base, g.N, cap, b);
        if (tau) {
            int k[3];
            unflatten(g, i, k);
            double t0, p0[3];
            tau0_p0(g, k, srcs + 3 * b, t0, p0);
            tau[e] = __dmul_rn(t0, A.rec[i].tau1);
        }
        if (tau1) tau1[e] = A.rec[i].tau1;
        if (order) order[e] = A.order[i];
        if (dir) dir[e] = A.dir[i];
    }
}

// Row i of M = sum_a diag(2 D_a tau1) D_a (Eq. Sensitivity2) with the
// derivatives fast marching chose: diag and up to three (neighbour, coef).
// The source row is 2 tau1_s.  Same operation order as the oracle.
struct Row {
    double diag;
    long long nb[3];
    double c[3];
    int n;
};

__device__ Row make_row(const EikGrid& g, long long i, const int* s, const unsigned char* __restrict__ dir,
                        const float* __restrict__ t1) {
    Row r;
    r.n = 0;
    r.diag = 0.0;
    const unsigned char dv = dir[i];
    const double ti = (double)t1[i];
    if (dv == kSourceDir) {
        r.diag = __dmul_rn(2.0, ti);
        return r;
    }
    int k[3];
    unflatten(g, i, k);
    double t0, p0[3];
    tau0_p0(g, k, s, t0, p0);
    for (int a = 0; a < g.d; ++a) {
        const int c = (dv >> (2 * a)) & 3;
        if (!c) continue;
        const long long nb = i + (c == 1 ? -g.st[a] : g.st[a]);
        const double cn = __ddiv_rn(t0, g.h);
        const double al = c == 1 ? __dadd_rn(cn, p0[a]) : __dsub_rn(cn, p0[a]);
        const double gv = __dsub_rn(__dmul_rn(al, ti), __dmul_rn(cn, (double)t1[nb]));
        r.diag = __dadd_rn(r.diag, __dmul_rn(__dmul_rn(2.0, gv), al));
        r.nb[r.n] = nb;
        r.c[r.n] = __dmul_rn(__dmul_rn(-2.0, gv), cn);
        ++r.n;
    }
    return r;
}

// z_s = J_s v (forward substitution, level by level)
__global__ void __launch_bounds__(256) k_eik_jv(EikGrid g, const int* __restrict__ srcs, char* base,
                                                 long long cap, const int* __restrict__ nlev,
                                                 const double* __restrict__ v, double* __restrict__ z) {
    const int b = blockIdx.x;
    SrcArrays A = src_arrays(base, g.N, cap, b);
    const int* s = srcs + 3 * b;
    double* zb = z + (long long)b * g.N;
    const int L = nlev[b];
    for (int l = 0; l < L; ++l) {
        for (int k = A.ptr[l] + threadIdx.x; k < A.ptr[l + 1]; k += blockDim.x) {
            const long long i = A.nodes[k];
            const Row r = make_row(g, i, s, A.dir, A.tau1f);
            double acc = v[i];
            for (int q = 0; q < r.n; ++q) acc = __dsub_rn(acc, __dmul_rn(r.c[q], zb[r.nb[q]]));
            zb[i] = __ddiv_rn(acc, r.diag);
        }
        __syncthreads();
    }
}

// y_s = J_s^T w_s (backward substitution, levels in reverse): node i pulls
// from the neighbours whose chosen derivative refers to it (its dependants).
__global__ void __launch_bounds__(256) k_eik_jtw(EikGrid g, const int* __restrict__ srcs, char* base,
                                                  long long cap, const int* __restrict__ nlev,
                                                  const double* __restrict__ w, double* __restrict__ y) {
    const int b = blockIdx.x;
    SrcArrays A = src_arrays(base, g.N, cap, b);
    const int* s = srcs + 3 * b;
    const double* wb = w + (long long)b * g.N;
    double* yb = y + (long long)b * g.N;
    const int L = nlev[b];
    for (int l = L - 1; l >= 0; --l) {
        for (int k = A.ptr[l] + threadIdx.x; k < A.ptr[l + 1]; k += blockDim.x) {
            const long long i = A.nodes[k];
            int ki[3];
            unflatten(g, i, ki);
            double acc = wb[i];
            for (int a = 0; a < g.d; ++a)
                for (int step = -1; step <= 1; step += 2) {
                    const int kk = ki[a] + step;
                    if (kk < 0 || kk >= g.S[a]) continue;
                    const long long j = i + step * g.st[a];
                    const unsigned char dj = A.dir[j];
                    if (dj == kSourceDir) continue;
                    // j depends on i when its axis-a choice points back to i
                    const int cj = (dj >> (2 * a)) & 3;
                    if (!((step == 1 && cj == 1) || (step == -1 && cj == 2))) continue;
                    const Row r = make_row(g, j, s, A.dir, A.tau1f);
                    for (int q = 0; q < r.n; ++q)
                        if (r.nb[q] == i) acc = __dsub_rn(acc, __dmul_rn(r.c[q], yb[j]));
                }
            const Row ri = make_row(g, i, s, A.dir, A.tau1f);
            yb[i] = __ddiv_rn(acc, ri.diag);
        }
        __syncthreads();
    }
}

}  // namespace

struct helm_eik {
    EikGrid g;
    int ns_max = 0;
    long long cap = 0;
    cudaStream_t st = nullptr;
    char* base = nullptr;      // per-source arrays
    int* dsrc = nullptr;       // 3 ints per source (numpy axis order)
    int* nlev = nullptr;
    int* status = nullptr;
    int* dmap = nullptr;       // sources rerun with their heap in global memory
    int ns = 0;                // sources of the last forward call
    std::vector<int> hsrc;
    std::string err;
};

namespace {
helm_status eik_fail(helm_eik* e, helm_status s, const std::string& msg) {
    if (e) e->err = msg;
    helm::set_thread_error(msg);
    return s;
}
#define EIK_TRY(e, expr)                                                                 \
    do {                                                                                 \
        cudaError_t c_ = (expr);                                                         \
        if (c_ != cudaSuccess)                                                           \
            return eik_fail(e, c_ == cudaErrorMemoryAllocation ? HELM_ERR_NOMEM : HELM_ERR_CUDA, \
                            std::string(#expr) + ": " + cudaGetErrorString(c_));         \
    } while (0)

int grid_blocks(long long total) {
    long long b = (total + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 65535LL * 8 ? 65535LL * 8 : b));
}
}  // namespace

extern "C" {

helm_status helm_eik_create(int dim, const int* n, double h, int ns_max, void* stream, helm_eik** out) {
    if (!out) return eik_fail(nullptr, HELM_ERR_ARG, "out is null");
    *out = nullptr;
    if ((dim != 2 && dim != 3) || !n || !(h > 0) || ns_max < 1)
        return eik_fail(nullptr, HELM_ERR_ARG, "dim must be 2 or 3, n non-null, h > 0, ns_max >= 1");
    for (int k = 0; k < dim; ++k)
        if (n[k] < 1) return eik_fail(nullptr, HELM_ERR_ARG, "each axis needs at least one cell");
    helm_eik* e = new helm_eik();
    e->g.d = dim;
    // numpy axis order: axis d-1 is x1
    for (int a = 0; a < dim; ++a) e->g.S[a] = n[dim - 1 - a] + 1;
    for (int a = dim; a < 3; ++a) e->g.S[a] = 1;
    long long st = 1;
    for (int a = dim - 1; a >= 0; --a) { e->g.st[a] = st; st *= e->g.S[a]; }
    for (int a = dim; a < 3; ++a) e->g.st[a] = 0;
    e->g.N = st;
    e->g.h = h;
    if (e->g.N > 0x7fffffffLL) { delete e; return eik_fail(nullptr, HELM_ERR_ARG, "grid too large"); }
    e->ns_max = ns_max;
    e->cap = e->g.N + 1;        // live heap entries; far above the front of a marching wave
    e->st = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)src_bytes(e->g.N, e->cap) * ns_max;
    cudaError_t c = cudaMalloc(&e->base, bytes);
    if (c == cudaSuccess) c = cudaMalloc(&e->dsrc, sizeof(int) * 3 * ns_max);
    if (c == cudaSuccess) c = cudaMalloc(&e->nlev, sizeof(int) * ns_max);
    if (c == cudaSuccess) c = cudaMalloc(&e->status, sizeof(int) * ns_max);
    if (c == cudaSuccess) c = cudaMalloc(&e->dmap, sizeof(int) * ns_max);
    if (c != cudaSuccess) {
        (void)cudaGetLastError();   // reported here; not again by a later error check
        helm_eik_destroy(e);
        return eik_fail(nullptr, c == cudaErrorMemoryAllocation ? HELM_ERR_NOMEM : HELM_ERR_CUDA,
                        std::string("cudaMalloc: ") + cudaGetErrorString(c));
    }
    *out = e;
    return HELM_OK;
}

helm_status helm_eik_forward(helm_eik* e, const double* m, const int* src, int ns, double* tau_out,
                             double* tau1_out, int* order_out, unsigned char* dir_out) {
    if (!e) return eik_fail(nullptr, HELM_ERR_ARG, "null workspace");
    if (!m || !src || ns < 1 || ns > e->ns_max) return eik_fail(e, HELM_ERR_ARG, "bad m, src or ns");
    const EikGrid& g = e->g;
    e->ns = 0;   // the products need a completed marching of these sources
    e->hsrc.assign(3 * (size_t)ns, 0);
    for (int b = 0; b < ns; ++b)
        for (int a = 0; a < g.d; ++a) {
            const int v = src[(size_t)b * g.d + (g.d - 1 - a)];   // caller gives (x1, x2[, x3])
            if (v < 0 || v >= g.S[a]) return eik_fail(e, HELM_ERR_ARG, "source outside the grid");
            e->hsrc[3 * (size_t)b + a] = v;
        }
    EIK_TRY(e, cudaMemcpyAsync(e->dsrc, e->hsrc.data(), sizeof(int) * 3 * ns, cudaMemcpyHostToDevice, e->st));
    // warp per source, heap in shared memory; the sources whose front
    // outgrows it run again, together, with their heaps in global memory
    {
        const size_t sm = g.d == 2 ? fm_smem<2>(true) : fm_smem<3>(true);
        auto kern = g.d == 2 ? k_fm_warp<2, true> : k_fm_warp<3, true>;
        EIK_TRY(e, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        kern<<<ns, 32, sm, e->st>>>(g, m, e->dsrc, e->base, e->cap, nullptr, e->nlev, e->status);
        EIK_TRY(e, cudaGetLastError());
    }
    std::vector<int> hs(ns);
    EIK_TRY(e, cudaMemcpyAsync(hs.data(), e->status, sizeof(int) * ns, cudaMemcpyDeviceToHost, e->st));
    EIK_TRY(e, cudaStreamSynchronize(e->st));
    std::vector<int> redo;
    for (int b = 0; b < ns; ++b)
        if (hs[b] == 1) redo.push_back(b);
    if (!redo.empty()) {
        EIK_TRY(e, cudaMemcpyAsync(e->dmap, redo.data(), sizeof(int) * redo.size(), cudaMemcpyHostToDevice,
                                   e->st));
        const size_t sm = g.d == 2 ? fm_smem<2>(false) : fm_smem<3>(false);
        auto kern = g.d == 2 ? k_fm_warp<2, false> : k_fm_warp<3, false>;
        kern<<<(unsigned)redo.size(), 32, sm, e->st>>>(g, m, e->dsrc, e->base, e->cap, e->dmap, e->nlev,
                                                       e->status);
        EIK_TRY(e, cudaGetLastError());
        EIK_TRY(e, cudaMemcpyAsync(hs.data(), e->status, sizeof(int) * ns, cudaMemcpyDeviceToHost, e->st));
        EIK_TRY(e, cudaStreamSynchronize(e->st));
    }
    for (int b = 0; b < ns; ++b) {
        if (hs[b] == 1) return eik_fail(e, HELM_ERR_NOMEM, "fast marching: heap capacity exceeded");
        if (hs[b] == 2) return eik_fail(e, HELM_ERR_BREAKDOWN, "fast marching: a node was not reached");
    }
    e->ns = ns;
    if (tau_out || tau1_out || order_out || dir_out) {
        k_eik_outputs<<<grid_blocks((long long)ns * g.N), 256, 0, e->st>>>(g, e->dsrc, e->base, e->cap, ns,
                                                                         tau_out, tau1_out, order_out,
                                                                         dir_out);
        EIK_TRY(e, cudaGetLastError());
        EIK_TRY(e, cudaStreamSynchronize(e->st));
    }
    return HELM_OK;
}

helm_status helm_eik_jv(helm_eik* e, const double* v, double* z) {
    if (!e || !v || !z) return eik_fail(e, HELM_ERR_ARG, "null argument");
    if (e->ns < 1) return eik_fail(e, HELM_ERR_ARG, "helm_eik_forward has not run");
    k_eik_jv<<<e->ns, 256, 0, e->st>>>(e->g, e->dsrc, e->base, e->cap, e->nlev, v, z);
    EIK_TRY(e, cudaGetLastError());
    EIK_TRY(e, cudaStreamSynchronize(e->st));
    return HELM_OK;
}

helm_status helm_eik_jtw(helm_eik* e, const double* w, double* y) {
    if (!e || !w || !y) return eik_fail(e, HELM_ERR_ARG, "null argument");
    if (e->ns < 1) return eik_fail(e, HELM_ERR_ARG, "helm_eik_forward has not run");
    k_eik_jtw<<<e->ns, 256, 0, e->st>>>(e->g, e->dsrc, e->base, e->cap, e->nlev, w, y);
    EIK_TRY(e, cudaGetLastError());
    EIK_TRY(e, cudaStreamSynchronize(e->st));
    return HELM_OK;
}

const char* helm_eik_last_error(const helm_eik* e) { return e ? e->err.c_str() : ""; }

void helm_eik_destroy(helm_eik* e) {
    if (!e) return;
    if (e->base) cudaFree(e->base);
    if (e->dsrc) cudaFree(e->dsrc);
    if (e->nlev) cudaFree(e->nlev);
    if (e->status) cudaFree(e->status);
    if (e->dmap) cudaFree(e->dmap);
    delete e;
}

}  // extern "C"
