// chain.cu -- ordered prefix product of the sample operators and the output
// write (Sec. 1.2.4, Eq. integration_compilation: psi_k = U_k psi_{k-1},
// psi_0 = psi_init since U_0 = I).
//
// The paper chains the U_k sequentially on the CPU.  Here the chain is a tree
// scan in FP64 on the device, per simulation (no node spans two simulations):
//   level 0:  a node is one warp over kFan runs of `run` consecutive samples;
//             lane l multiplies its run in order (all lanes busy);
//   level l:  a node covers kFan consecutive nodes of level l - 1, up to one
//             top node per simulation;
//   up:       one kernel per level; every node forms the products of its
//             binary tree over its 32 children (31 products in 5 rounds),
//             keeping the left-child product of every internal node and the
//             node's total (a warp per node at level 0, a block of four warps
//             per node above, where the nodes are few);
//   down:     the team that builds a top node also walks its tree down from
//             psi0 (the left child receives the state, the right child the left
//             child's product applied to it: 31 matrix-vector products in 5
//             rounds) and stores the states entering its children;
//   apply:    per level-0 node, the entering state follows by walking down the
//             ancestors' trees from there (a matrix-vector product at each step
//             into a right child), the node's own down-sweep gives every lane
//             run its entering state, and each lane walks its run; psi_k and
//             <J>_k are staged in shared memory and the warp stores the node's
//             span as contiguous 16-byte words (U_k, when asked for, directly).
//
// GB300 executes FP64 at 1/64 of the FP32 rate: one FP64 warp instruction
// keeps an SM sub-partition busy for tens of cycles whether one lane or 32
// are active.  So every product of the binary trees is spread over the lanes
// entry by entry (a round of a tree level computes up to 32 entries at once),
// instead of one lane per product with most lanes idle, and the number of
// level-0 nodes of a long simulation is matched to the SM sub-partitions.
// Spin-one operators are general 3x3 complex matrices; spin-half operators
// are kept in SU(2) form (alpha, beta) = first column.
#include <algorithm>

#include "bounds.cuh"
#include "sample_epilogue.cuh"

namespace spinsim {

__device__ __forceinline__ int find_node_sim(const int64_t* off, int n, int64_t j)
{
    // largest i in [0, n) with off[i] <= j (off is non-decreasing, off[0] = 0)
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------ operator types
// Operators and states are stored as doubles (global and shared memory); the
// arithmetic runs in T: double, or float for the study of a single-precision
// cross-sample product (spinsim_config.chain_precision), every product then
// rounded to float.
template <int N, typename T>
struct Op;

template <typename T>
struct Op<3, T> {
    cx<T> m[3][3];
    __device__ __forceinline__ void identity()
    {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) m[i][j] = cmk<T>(i == j ? T(1) : T(0), T(0));
    }
    __device__ __forceinline__ void load(const double* p)
    {
        const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
        for (int e = 0; e < 9; e++) {
            double2 v = q[e];
            m[e / 3][e % 3] = cmk<T>((T)v.x, (T)v.y);
        }
    }
    __device__ __forceinline__ void store(double* p) const
    {
        double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
        for (int e = 0; e < 9; e++) q[e] = make_double2((double)m[e / 3][e % 3].r, (double)m[e / 3][e % 3].i);
    }
    // C = A B
    static __device__ __forceinline__ void mul(const Op& A, const Op& B, Op& C)
    {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                cx<T> s = cmul(A.m[i][0], B.m[0][j]);
                s = cfma(A.m[i][1], B.m[1][j], s);
                s = cfma(A.m[i][2], B.m[2][j], s);
                C.m[i][j] = s;
            }
    }
    __device__ __forceinline__ void apply(const cx<T>* in, cx<T>* out) const
    {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            cx<T> s = cmul(m[i][0], in[0]);
            s = cfma(m[i][1], in[1], s);
            s = cfma(m[i][2], in[2], s);
            out[i] = s;
        }
    }
    __device__ __forceinline__ void store_full(double* p) const { store(p); }
};

// SU(2): [[alpha, -conj(beta)], [beta, conj(alpha)]]
template <typename T>
struct Op<2, T> {
    cx<T> a, b;
    __device__ __forceinline__ void identity() { a = cmk<T>(T(1), T(0)); b = cmk<T>(T(0), T(0)); }
    __device__ __forceinline__ void load(const double* p)
    {
        const double2* q = reinterpret_cast<const double2*>(p);
        double2 x = q[0], y = q[1];
        a = cmk<T>((T)x.x, (T)x.y);
        b = cmk<T>((T)y.x, (T)y.y);
    }
    __device__ __forceinline__ void store(double* p) const
    {
        double2* q = reinterpret_cast<double2*>(p);
        q[0] = make_double2((double)a.r, (double)a.i);
        q[1] = make_double2((double)b.r, (double)b.i);
    }
    // alpha = a1 a2 - conj(b1) b2, beta = b1 a2 + conj(a1) b2
    static __device__ __forceinline__ void mul(const Op& A, const Op& B, Op& C)
    {
        cx<T> na = cmul(A.a, B.a);
        na = csub(na, cmul(cconj(A.b), B.b));
        cx<T> nb = cmul(A.b, B.a);
        nb = cfma_conj(A.a, B.b, nb);
        C.a = na;
        C.b = nb;
    }
    __device__ __forceinline__ void apply(const cx<T>* in, cx<T>* out) const
    {
        // [alpha psi0 - conj(beta) psi1, beta psi0 + conj(alpha) psi1]
        cx<T> o0 = cmul(a, in[0]);
        o0 = csub(o0, cmul(cconj(b), in[1]));
        cx<T> o1 = cmul(b, in[0]);
        o1 = cfma_conj(a, in[1], o1);
        out[0] = o0;
        out[1] = o1;
    }
    __device__ __forceinline__ void store_full(double* p) const
    {
        p[0] = a.r; p[1] = a.i; p[2] = -b.r; p[3] = b.i;
        p[4] = b.r; p[5] = b.i; p[6] = a.r; p[7] = -a.i;
    }
};

// ------------------------------------------------------- binary trees
// A binary tree over 32 leaves lives in 63 shared-memory slots: height h
// (0 = leaves) starts at slot 64 - (64 >> h), node p of height h sits at slot
// tslot(h, p).  Internal node (h, p), h >= 1, multiplies its children:
// slot(h, p) = slot(h-1, 2p+1) * slot(h-1, 2p) (later on the left).
__device__ __forceinline__ int tslot(int h, int p) { return (64 - (64 >> h)) + p; }

// Left child of the internal node with slot 32 + t, t in [0, 31): the
// products a down-sweep needs, stored in this order per node.
__device__ __forceinline__ int left_child_slot(int t)
{
    const int q = 32 + t;
    int h = 1;
    while (h < 5 && q >= tslot(h + 1, 0)) h++;
    return tslot(h - 1, 2 * (q - tslot(h, 0)));
}

// Entry arithmetic on operators held as doubles in shared memory.
template <int N, typename T>
struct Tree;

template <typename T>
struct Tree<3, T> {
    static constexpr int D = 18;   // doubles per operator
    static __device__ __forceinline__ cx<T> at(const double* A, int i, int j)
    {
        const double2 v = reinterpret_cast<const double2*>(A)[3 * i + j];
        return cmk<T>((T)v.x, (T)v.y);
    }
    // Real (c = 0) or imaginary (c = 1) part of sum_k a_k b_k, as cmul and
    // cfma round it: sum_k a_k.r P_k + Q_k R_k with (P, Q, R) = (b.r, -a.i,
    // b.i) or (b.i, a.i, b.r).  Lanes working on different parts run the same
    // FP64 instructions (the parts are selected by integer operations): a
    // branch on the part would issue both paths' FP64 instructions, each of
    // which holds an SM sub-partition's FP64 unit whatever the lanes in use.
    static __device__ __forceinline__ T dot_part(const cx<T> (&a)[3], const cx<T> (&b)[3], int c)
    {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const T P = c ? b[k].i : b[k].r, R = c ? b[k].r : b[k].i;
            const T Q = flip_sign(a[k].i, !c);
            s = k == 0 ? fma(a[k].r, P, Q * R) : fma(a[k].r, P, fma(Q, R, s));
        }
        return s;
    }
    static __device__ __forceinline__ double flip_sign(double x, bool neg)
    {
        return __hiloint2double(__double2hiint(x) ^ (neg ? (int)0x80000000 : 0), __double2loint(x));
    }
    static __device__ __forceinline__ float flip_sign(float x, bool neg)
    {
        return __int_as_float(__float_as_int(x) ^ (neg ? (int)0x80000000 : 0));
    }
    // parts (re, im of each entry) of a product: one per task of a tree round
    static constexpr int PARTS = 18;
    // part t = 2 e + c of C = A B, e = 3 i + j (C as doubles: C[t])
    static __device__ __forceinline__ void prod_part(const double* A, const double* B, int t, double* C)
    {
        const int e = t >> 1, i = e / 3, j = e - 3 * (e / 3);
        const cx<T> a[3] = {at(A, i, 0), at(A, i, 1), at(A, i, 2)};
        const cx<T> b[3] = {at(B, 0, j), at(B, 1, j), at(B, 2, j)};
        C[t] = (double)dot_part(a, b, t & 1);
    }
    // parts of a matrix-vector product (re, im of each component)
    static constexpr int VPARTS = 6;
    // part t = 2 r + c of A v (v: 3 complex), as doubles: (A v)[t]
    static __device__ __forceinline__ T matvec_part(const double* A, const double* v, int t)
    {
        const int r = t >> 1;
        const double2* w = reinterpret_cast<const double2*>(v);
        const cx<T> a[3] = {at(A, r, 0), at(A, r, 1), at(A, r, 2)};
        const cx<T> b[3] = {cmk<T>((T)w[0].x, (T)w[0].y), cmk<T>((T)w[1].x, (T)w[1].y), cmk<T>((T)w[2].x, (T)w[2].y)};
        return dot_part(a, b, t & 1);
    }
    // tree_down's task: part t of the parent's state v goes to the left child
    // vl, part t of A v to the right child vr
    static __device__ __forceinline__ void down_part(const double* A, const double* v, int t, double* vl, double* vr)
    {
        const T y = matvec_part(A, v, t);
        vl[t] = v[t];
        vr[t] = (double)y;
    }
};

// SU(2) element [[alpha, -conj(beta)], [beta, conj(alpha)]] stored as (alpha, beta).
template <typename T>
struct Tree<2, T> {
    static constexpr int D = 4;
    static __device__ __forceinline__ void prod_entry(const double* A, const double* B, int e, double* C)
    {
        const double2* a = reinterpret_cast<const double2*>(A);
        const double2* b = reinterpret_cast<const double2*>(B);
        const cx<T> a1 = cmk<T>((T)a[0].x, (T)a[0].y), b1 = cmk<T>((T)a[1].x, (T)a[1].y);
        const cx<T> a2 = cmk<T>((T)b[0].x, (T)b[0].y), b2 = cmk<T>((T)b[1].x, (T)b[1].y);
        cx<T> s;
        if (e == 0) s = csub(cmul(a1, a2), cmul(cconj(b1), b2));   // alpha = a1 a2 - conj(b1) b2
        else s = cfma_conj(a1, b2, cmul(b1, a2));                  // beta = b1 a2 + conj(a1) b2
        reinterpret_cast<double2*>(C)[e] = make_double2((double)s.r, (double)s.i);
    }
    static __device__ __forceinline__ cx<T> matvec_row(const double* A, const double* v, int r)
    {
        const double2* a = reinterpret_cast<const double2*>(A);
        const double2* w = reinterpret_cast<const double2*>(v);
        const cx<T> al = cmk<T>((T)a[0].x, (T)a[0].y), be = cmk<T>((T)a[1].x, (T)a[1].y);
        const cx<T> v0 = cmk<T>((T)w[0].x, (T)w[0].y), v1 = cmk<T>((T)w[1].x, (T)w[1].y);
        // [alpha v0 - conj(beta) v1, beta v0 + conj(alpha) v1]
        return r == 0 ? csub(cmul(al, v0), cmul(cconj(be), v1)) : cfma_conj(al, v1, cmul(be, v0));
    }
    // tasks of a tree round: the two entries (alpha, beta) of a product, the
    // two components of a matrix-vector product
    static constexpr int PARTS = 2;
    static __device__ __forceinline__ void prod_part(const double* A, const double* B, int t, double* C)
    {
        prod_entry(A, B, t, C);
    }
    static constexpr int VPARTS = 2;
    static __device__ __forceinline__ void down_part(const double* A, const double* v, int r, double* vl, double* vr)
    {
        const cx<T> y = matvec_row(A, v, r);
        vl[2 * r] = v[2 * r];
        vl[2 * r + 1] = v[2 * r + 1];
        vr[2 * r] = (double)y.r;
        vr[2 * r + 1] = (double)y.i;
    }
};

// The threads that share one tree: a warp (nodes of level 0) or a whole
// block (nodes of the upper levels, which are few: spreading a node's
// products over four warps puts all four FP64 pipes of an SM on it).
template <bool BLOCK>
struct Team {
    static __device__ __forceinline__ int rank() { return BLOCK ? (int)threadIdx.x : (int)(threadIdx.x & 31); }
    static __device__ __forceinline__ int size() { return BLOCK ? (int)blockDim.x : 32; }
    static __device__ __forceinline__ void sync()
    {
        if (BLOCK) __syncthreads();
        else __syncwarp();
    }
};

// Up-sweep of a tree: leaves in slots 0..31, products of every internal
// node, one part (spin-one: the real or imaginary part of an entry) per
// thread per round.
template <int N, typename T, bool BLOCK>
__device__ __forceinline__ void tree_up(double* S)
{
    constexpr int D = Tree<N, T>::D, E = Tree<N, T>::PARTS;
    const int me = Team<BLOCK>::rank(), n = Team<BLOCK>::size();
#pragma unroll 1
    for (int h = 1; h <= 5; h++) {
        const int P = 32 >> h;
        for (int t = me; t < P * E; t += n) {
            const int p = t / E, e = t - E * (t / E);
            Tree<N, T>::prod_part(S + tslot(h - 1, 2 * p + 1) * D, S + tslot(h - 1, 2 * p) * D, e,
                                  S + tslot(h, p) * D);
        }
        Team<BLOCK>::sync();
    }
}

// Down-sweep: the state entering the node is in V slot tslot(5, 0); the
// states entering the 32 leaves end in slots 0..31.  `left(t)` returns the
// left-child product of internal node 32 + t.
template <int N, typename T, bool BLOCK, typename Left>
__device__ __forceinline__ void tree_down(double* V, Left left)
{
    constexpr int SV = 2 * N;   // doubles per state
    constexpr int VP = Tree<N, T>::VPARTS;
    const int me = Team<BLOCK>::rank(), n = Team<BLOCK>::size();
#pragma unroll 1
    for (int h = 5; h >= 1; h--) {
        const int P = 32 >> h;
        for (int t = me; t < P * VP; t += n) {
            const int p = t / VP, r = t - VP * (t / VP);
            Tree<N, T>::down_part(left(tslot(h, p) - 32), V + tslot(h, p) * SV, r, V + tslot(h - 1, 2 * p) * SV,
                                  V + tslot(h - 1, 2 * p + 1) * SV);
        }
        Team<BLOCK>::sync();
    }
}

// Shared memory: a tree (63 operators) and its states (63), per warp at
// level 0 and per block above; the apply kernel's states and write-out
// staging per warp.
template <int N>
constexpr int tree_doubles() { return 63 * Tree<N, double>::D + 63 * 2 * N; }
template <int N>
constexpr int state_doubles() { return 63 * 2 * N; }
constexpr int kChainWarps = 4;   // warps per block of the chain kernels
constexpr int kMaxRun = 8;       // the longest lane run (chain_run)
// The apply kernel's staging is sized for the batch's longest run (at most
// kMaxRun), so that batches of shorter runs fit more blocks per SM.
__host__ __device__ inline int apply_run(const ChainArgs& a)
{
    return a.max_run >= 1 && a.max_run <= kMaxRun ? a.max_run : kMaxRun;
}
// staged outputs of one level-0 node: 32 x run samples of psi_k and <J>_k
template <int N>
__host__ __device__ constexpr int stage_doubles(int run) { return kFan * run * (2 * N + 3); }

// ------------------------------------------------------------------ kernels
// The up-sweep work of one node: its binary tree over the leaves already in
// S (slots 0..31), its left-child products and its total stored, and, at a
// simulation's top node (whole scan only), the down-sweep from psi0 storing
// the states entering the top node's children.
template <int N, typename T, bool BLOCK>
__device__ __forceinline__ void node_up(const ChainArgs& a, int level, int64_t node, const DevSim& s, int si,
                                        int64_t local, const int64_t* coff, double* S, double* V)
{
    constexpr int D = Tree<N, T>::D, SV = 2 * N;
    tree_up<N, T, BLOCK>(S);
    const int me = Team<BLOCK>::rank(), n = Team<BLOCK>::size();
    // the 31 left-child products, then the total, as double2 words
    for (int w = me; w < (kLeftPerNode + 1) * (D / 2); w += n) {
        const int t = w / (D / 2), i = w - (D / 2) * t;
        const double2* src = reinterpret_cast<const double2*>(S + (t < kLeftPerNode ? left_child_slot(t) : tslot(5, 0)) * D);
        double2* dst = t < kLeftPerNode ? reinterpret_cast<double2*>(a.left[level] + (node * kLeftPerNode + t) * D)
                                        : reinterpret_cast<double2*>(a.agg[level] + node * D);
        dst[i] = src[i];
    }
    if (level >= 1 && s.chain_top == level && a.mode == kChainFull) {
        if (me < SV) V[tslot(5, 0) * SV + me] = s.psi0[me];
        Team<BLOCK>::sync();
        tree_down<N, T, BLOCK>(V, [&](int t) { return (const double*)(S + left_child_slot(t) * D); });
        for (int w = me; w < kFan * SV; w += n) {
            const int child = w / SV, i = w - SV * child;
            if (local * kFan + child < coff[si + 1] - coff[si] &&
                SPINSIM_INB(coff[si] + local * kFan + child < a.nodes[level - 1], 10))
                a.state[level - 1][(coff[si] + local * kFan + child) * SV + i] = V[child * SV + i];
        }
    }
    Team<BLOCK>::sync();
}

// Up-sweep of level 0: one warp per node.  Lane l multiplies its run of
// consecutive sample operators, U_{k1-1} ... U_{k0} (the first operator
// loaded, not multiplied into the identity); the 32 runs are the leaves.
template <int N, typename T>
__global__ void __launch_bounds__(128) chain_up_kernel(ChainArgs a)
{
    constexpr int D = Tree<N, T>::D;
    extern __shared__ __align__(16) double smem[];
    // programmatic dependent launch: the previous kernel's results are
    // visible after this wait; the next chain kernel may be scheduled now
    grid_dependency_wait();
    allow_dependent_launch();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* S = smem + warp * tree_doubles<N>();
    double* V = S + 63 * D;
    const int64_t* off = a.level_off;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t node = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; node < a.nodes[0]; node += warps) {
        const int si = find_node_sim(off, a.n_sims, node);
        const DevSim& s = a.sims[si];
        const int64_t local = node - off[si];
        Op<N, T> B;
        B.identity();
        const int run = s.chain_run;
        const int64_t k0 = (local * kFan + lane) * run;
        const int64_t k1 = min(k0 + run, s.K);
        const double* U = a.U + s.sample_offset * D;
        if (SPINSIM_INB(si >= 0 && si < a.n_sims && k0 >= 0, 8) && k0 < k1) B.load(U + k0 * D);
        // the next operator is loaded while the current product runs (L2 latency
        // off the dependent chain of products)
        Op<N, T> u;
        if (k0 + 1 < k1) {
            if (SPINSIM_INB(k0 + 1 < s.K, 9)) u.load(U + (k0 + 1) * D);
            else u.identity();
        }
        for (int64_t k = k0 + 1; k < k1; k++) {
            Op<N, T> t, nx;
            if (k + 1 < k1) {
                if (SPINSIM_INB(k + 1 < s.K, 9)) nx.load(U + (k + 1) * D);
                else nx.identity();
            }
            Op<N, T>::mul(u, B, t);   // later operators multiply from the left
            B = t;
            u = nx;
        }
        B.store(S + lane * D);
        __syncwarp();
        node_up<N, T, false>(a, 0, node, s, si, local, nullptr, S, V);
    }
}

// Up-sweep of a level >= 1: one block per node; the leaves are the 32
// children's products.
template <int N, typename T>
__global__ void __launch_bounds__(128) chain_up_upper_kernel(ChainArgs a, int level)
{
    constexpr int D = Tree<N, T>::D;
    extern __shared__ __align__(16) double smem[];
    grid_dependency_wait();
    allow_dependent_launch();
    double* S = smem;
    double* V = S + 63 * D;
    const int64_t* off = a.level_off + (size_t)level * (a.n_sims + 1);
    const int64_t* coff = off - (a.n_sims + 1);
    for (int64_t node = blockIdx.x; node < a.nodes[level]; node += gridDim.x) {
        const int si = find_node_sim(off, a.n_sims, node);
        const DevSim& s = a.sims[si];
        const int64_t local = node - off[si];
        const int64_t n_child = coff[si + 1] - coff[si];
        // leaves: the children's products (identity past the last child), as double words
        for (int w = threadIdx.x; w < kFan * D; w += blockDim.x) {
            const int c = w / D, i = w - D * c;
            const int64_t child = local * kFan + c;
            double v;
            if (child < n_child && SPINSIM_INB(coff[si] + child < a.nodes[level - 1], 11))
                v = a.agg[level - 1][(coff[si] + child) * D + i];
            else v = (N == 3 ? (i == 0 || i == 8 || i == 16) : i == 0) ? 1.0 : 0.0;   // identity
            S[c * D + i] = v;
        }
        __syncthreads();
        node_up<N, T, true>(a, level, node, s, si, local, coff, S, V);
    }
}

// Down-sweep and output: one warp per level-0 node.  The state entering the
// node follows by walking down to it: in the whole scan from the state the
// top node's up-sweep stored for its child on this node's path (psi0 for a
// simulation of one node), in the down-only mode (a range whose entering
// state arrived later) from psi0 at the top node.  Inside each ancestor's
// binary tree, a step into a right child applies the left sibling's product
// (one matrix row per lane).  The node's own tree then gives every lane run
// its entering state; each lane walks its run, writing psi_k and <J>_k into
// the warp's staging area and (optionally) U_k; the warp then stores the
// node's span of psi_k and <J>_k as contiguous 16-byte words.
template <int N, typename T>
__global__ void __launch_bounds__(128) chain_apply_kernel(ChainArgs a)
{
    constexpr int D = Tree<N, T>::D, SV = 2 * N;
    extern __shared__ __align__(16) double smem[];
    grid_dependency_wait();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mr = apply_run(a);
    double* V = smem + warp * (state_doubles<N>() + stage_doubles<N>(mr));
    double* stage_psi = V + state_doubles<N>();            // [32 run][2N]
    double* stage_spin = stage_psi + kFan * mr * SV;        // [32 run][3]
    const int64_t stride = a.n_sims + 1;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t node = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; node < a.nodes[0]; node += warps) {
        const int si = find_node_sim(a.level_off, a.n_sims, node);
        const DevSim& s = a.sims[si];
        const int64_t local = node - a.level_off[si];
        double* v = V + tslot(5, 0) * SV;
        int from = s.chain_top;
        if (a.mode == kChainFull && from >= 1) {
            from--;
            const int64_t anc = local >> (5 * from);   // the top node's child on the path
            const int64_t at = a.level_off[(size_t)from * stride + si] + anc;
            if (lane < SV) v[lane] = SPINSIM_INB(at < a.nodes[from], 12) ? a.state[from][at * SV + lane] : 0.0;
        } else if (lane < SV) {
            v[lane] = s.psi0[lane];
        }
        __syncwarp();
        for (int level = from; level >= 1; level--) {
            const int64_t anc = local >> (5 * level);                         // ancestor at `level`
            const int64_t j = (local >> (5 * (level - 1))) - anc * kFan;     // its child on the path
            const int64_t at = a.level_off[(size_t)level * stride + si] + anc;
            const double* L = a.left[level] + at * kLeftPerNode * D;
            const bool in_range = SPINSIM_INB(at < a.nodes[level], 13);
            for (int h = 5; h >= 1; h--) {
                if (((j >> (h - 1)) & 1) == 0 || !in_range) continue;       // left child: state unchanged
                const int p = (int)(j >> h);
                const double* A = L + (tslot(h, p) - 32) * D;
                if constexpr (N == 3) {
                    // one part of the new state per lane (six lanes)
                    T y = T(0);
                    if (lane < Tree<N, T>::VPARTS) y = Tree<N, T>::matvec_part(A, v, lane);
                    __syncwarp();
                    if (lane < Tree<N, T>::VPARTS) v[lane] = (double)y;
                } else {
                    cx<T> y = cmk<T>(T(0), T(0));
                    if (lane < N) y = Tree<N, T>::matvec_row(A, v, lane);
                    __syncwarp();
                    if (lane < N) {
                        v[2 * lane] = (double)y.r;
                        v[2 * lane + 1] = (double)y.i;
                    }
                }
                __syncwarp();
            }
        }
        const double* L0 = a.left[0] + node * kLeftPerNode * D;
        tree_down<N, T, false>(V, [&](int t) { return L0 + t * D; });
        cx<T> psi[N], nxt[N];
#pragma unroll
        for (int i = 0; i < N; i++) psi[i] = cmk<T>((T)V[lane * SV + 2 * i], (T)V[lane * SV + 2 * i + 1]);
        __syncwarp();
        const int run = s.chain_run;
        const int64_t kn = local * kFan * run;              // the node's first sample
        const int64_t k0 = kn + (int64_t)lane * run;
        const int64_t k1 = min(k0 + run, s.K);
        const double* U = a.U + s.sample_offset * D;
        // U_{k+1} is loaded while sample k is computed and written
        Op<N, T> u;
        if (k0 < k1) {
            if (SPINSIM_INB(k0 >= 0 && k0 < s.K && k0 - kn < (int64_t)kFan * mr, 14)) u.load(U + k0 * D);
            else u.identity();
        }
        for (int64_t k = k0; k < k1; k++) {
            Op<N, T> un;
            if (k + 1 < k1) {
                if (SPINSIM_INB(k + 1 < s.K && k + 1 - kn < (int64_t)kFan * mr, 14)) un.load(U + (k + 1) * D);
                else un.identity();
            }
            u.apply(psi, nxt);
#pragma unroll
            for (int i = 0; i < N; i++) psi[i] = nxt[i];
            T scale = T(1);
            if (s.normalize_out) {
                // FP32-bulk: the written state is renormalised
                T n2 = T(0);
#pragma unroll
                for (int i = 0; i < N; i++) n2 = fma(psi[i].r, psi[i].r, fma(psi[i].i, psi[i].i, n2));
                const T d = n2 - T(1);
                scale = T(1) - d * (T(0.5) - T(0.375) * d);   // (1 + d)^(-1/2), |d| ~ 1e-9
            }
            cx<double> w[N];
#pragma unroll
            for (int i = 0; i < N; i++) {
                const cx<T> x = cscale(psi[i], scale);
                w[i] = cmk((double)x.r, (double)x.i);
            }
            const int64_t q = k - kn;                       // position in the node's span
            double2* sp = reinterpret_cast<double2*>(stage_psi + q * SV);
#pragma unroll
            for (int i = 0; i < N; i++) sp[i] = make_double2(w[i].r, w[i].i);
            if (s.spin) {
                double jv[3];
                spin_projection(w, N, jv);
                stage_spin[q * 3 + 0] = jv[0];
                stage_spin[q * 3 + 1] = jv[1];
                stage_spin[q * 3 + 2] = jv[2];
            }
            if (s.ops) u.store_full(s.ops + k * 2 * N * N);
            u = un;
        }
        __syncwarp();
        // the node's span [kn, kn + m): psi_k as N double2 words per sample,
        // <J>_k as 3 doubles per sample (kn is a multiple of 4: whole words)
        const int64_t m = SPINSIM_INB(run <= mr && kn + min((int64_t)kFan * run, s.K - kn) <= s.K, 15)
                              ? min((int64_t)kFan * run, s.K - kn) : 0;
        {
            const double2* src = reinterpret_cast<const double2*>(stage_psi);
            double2* dst = reinterpret_cast<double2*>(s.states + kn * SV);
            for (int64_t i = lane; i < m * N; i += 32) dst[i] = src[i];
        }
        if (s.spin) {
            const double2* src = reinterpret_cast<const double2*>(stage_spin);
            double2* dst = reinterpret_cast<double2*>(s.spin + kn * 3);
            const int64_t words = m * 3 / 2;
            for (int64_t i = lane; i < words; i += 32) dst[i] = src[i];
            if ((m * 3) & 1)
                if (lane == 0) s.spin[kn * 3 + m * 3 - 1] = stage_spin[m * 3 - 1];
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------- launcher
template <int N, typename T>
static cudaError_t launch_chain_nt(const ChainArgs& a, int n_sm, cudaStream_t stream, int* kernels)
{
    *kernels = 0;
    if (a.levels < 1 || a.nodes[0] == 0) return cudaSuccess;
    const int block = 32 * kChainWarps;
    const size_t up_smem = (size_t)kChainWarps * tree_doubles<N>() * sizeof(double);
    const size_t upper_smem = (size_t)tree_doubles<N>() * sizeof(double);
    const size_t apply_smem = (size_t)kChainWarps * (state_doubles<N>() + stage_doubles<N>(apply_run(a))) * sizeof(double);
    const size_t apply_smem_max = (size_t)kChainWarps * (state_doubles<N>() + stage_doubles<N>(kMaxRun)) * sizeof(double);
    // the apply kernel's staging exceeds the default 48 KB of dynamic shared
    // memory: raise its limit once per device (before any capture: the first
    // launch of a batch shape is always eager)
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(chain_apply_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)apply_smem_max);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    auto grid = [&](int64_t nodes) {
        return (int)std::max<int64_t>(1, std::min<int64_t>((nodes + kChainWarps - 1) / kChainWarps, (int64_t)n_sm * 16));
    };
    ChainArgs args = a;
    // Programmatic dependent launches: each chain kernel may be scheduled
    // while its predecessor finishes and waits (griddepcontrol.wait) for its
    // results, which hides the launch gap between the dependent kernels.
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(block);
    cfg.stream = stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (a.mode != kChainDown) {
        cfg.gridDim = dim3(grid(a.nodes[0]));
        cfg.dynamicSmemBytes = up_smem;
        cudaError_t e = cudaLaunchKernelEx(&cfg, chain_up_kernel<N, T>, args);
        if (e != cudaSuccess) return e;
        (*kernels)++;
        for (int l = 1; l < a.levels; l++) {
            cfg.gridDim = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(a.nodes[l], (int64_t)n_sm * 16)));
            cfg.dynamicSmemBytes = upper_smem;
            e = cudaLaunchKernelEx(&cfg, chain_up_upper_kernel<N, T>, args, l);
            if (e != cudaSuccess) return e;
            (*kernels)++;
        }
    }
    if (a.mode != kChainUp) {
        cfg.gridDim = dim3(grid(a.nodes[0]));
        cfg.dynamicSmemBytes = apply_smem;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, chain_apply_kernel<N, T>, args);
        if (e != cudaSuccess) return e;
        (*kernels)++;
    }
    return cudaGetLastError();
}

cudaError_t launch_chain(int spin_x2, const ChainArgs& a, int n_sm, cudaStream_t stream, int* kernels, bool fp32)
{
    if (spin_x2 == 2) return fp32 ? launch_chain_nt<3, float>(a, n_sm, stream, kernels)
                                  : launch_chain_nt<3, double>(a, n_sm, stream, kernels);
    if (spin_x2 == 1) return fp32 ? launch_chain_nt<2, float>(a, n_sm, stream, kernels)
                                  : launch_chain_nt<2, double>(a, n_sm, stream, kernels);
    return cudaErrorInvalidValue;
}

#ifdef SPINSIM_BOUNDS
SPINSIM_BOUNDS_READER(bounds_word_chain)
#endif

}  // namespace spinsim
