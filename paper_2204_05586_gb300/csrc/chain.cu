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
//             node's total;
//   down:     the warp that builds a top node also walks its tree down from
//             psi0 (the left child receives the state, the right child the left
//             child's product applied to it: 31 matrix-vector products in 5
//             rounds) and stores the states entering its children;
//   apply:    per level-0 node, the entering state follows by walking down the
//             ancestors' trees from there (a matrix-vector product at each step
//             into a right child), the node's own down-sweep gives every lane
//             run its entering state, and each lane walks its run, writing
//             psi_k, <J>_k and (optionally) U_k.
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
template <int N>
struct Op;

template <>
struct Op<3> {
    cx<double> m[3][3];
    __device__ __forceinline__ void identity()
    {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) m[i][j] = cmk(i == j ? 1.0 : 0.0, 0.0);
    }
    __device__ __forceinline__ void load(const double* p)
    {
        const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
        for (int e = 0; e < 9; e++) {
            double2 v = q[e];
            m[e / 3][e % 3] = cmk(v.x, v.y);
        }
    }
    __device__ __forceinline__ void store(double* p) const
    {
        double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
        for (int e = 0; e < 9; e++) q[e] = make_double2(m[e / 3][e % 3].r, m[e / 3][e % 3].i);
    }
    // C = A B
    static __device__ __forceinline__ void mul(const Op& A, const Op& B, Op& C)
    {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                cx<double> s = cmul(A.m[i][0], B.m[0][j]);
                s = cfma(A.m[i][1], B.m[1][j], s);
                s = cfma(A.m[i][2], B.m[2][j], s);
                C.m[i][j] = s;
            }
    }
    __device__ __forceinline__ void apply(const cx<double>* in, cx<double>* out) const
    {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            cx<double> s = cmul(m[i][0], in[0]);
            s = cfma(m[i][1], in[1], s);
            s = cfma(m[i][2], in[2], s);
            out[i] = s;
        }
    }
    __device__ __forceinline__ void store_full(double* p) const { store(p); }
};

// SU(2): [[alpha, -conj(beta)], [beta, conj(alpha)]]
template <>
struct Op<2> {
    cx<double> a, b;
    __device__ __forceinline__ void identity() { a = cmk(1.0, 0.0); b = cmk(0.0, 0.0); }
    __device__ __forceinline__ void load(const double* p)
    {
        const double2* q = reinterpret_cast<const double2*>(p);
        double2 x = q[0], y = q[1];
        a = cmk(x.x, x.y);
        b = cmk(y.x, y.y);
    }
    __device__ __forceinline__ void store(double* p) const
    {
        double2* q = reinterpret_cast<double2*>(p);
        q[0] = make_double2(a.r, a.i);
        q[1] = make_double2(b.r, b.i);
    }
    // alpha = a1 a2 - conj(b1) b2, beta = b1 a2 + conj(a1) b2
    static __device__ __forceinline__ void mul(const Op& A, const Op& B, Op& C)
    {
        cx<double> na = cmul(A.a, B.a);
        na = csub(na, cmul(cconj(A.b), B.b));
        cx<double> nb = cmul(A.b, B.a);
        nb = cfma_conj(A.a, B.b, nb);
        C.a = na;
        C.b = nb;
    }
    __device__ __forceinline__ void apply(const cx<double>* in, cx<double>* out) const
    {
        // [alpha psi0 - conj(beta) psi1, beta psi0 + conj(alpha) psi1]
        cx<double> o0 = cmul(a, in[0]);
        o0 = csub(o0, cmul(cconj(b), in[1]));
        cx<double> o1 = cmul(b, in[0]);
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

// ------------------------------------------------- binary trees of a warp
// A warp's binary tree over 32 leaves lives in 63 shared-memory slots:
// height h (0 = leaves) starts at slot 64 - (64 >> h), node p of height h
// sits at slot tslot(h, p).  Internal node (h, p), h >= 1, multiplies its
// children: slot(h, p) = slot(h-1, 2p+1) * slot(h-1, 2p) (later on the left).
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
template <int N>
struct Tree;

template <>
struct Tree<3> {
    static constexpr int D = 18;   // doubles per operator
    static constexpr int E = 9;    // entries of a product
    static __device__ __forceinline__ cx<double> at(const double* A, int i, int j)
    {
        const double2 v = reinterpret_cast<const double2*>(A)[3 * i + j];
        return cmk(v.x, v.y);
    }
    // entry e = (i, j) of C = A B
    static __device__ __forceinline__ void prod_entry(const double* A, const double* B, int e, double* C)
    {
        const int i = e / 3, j = e - 3 * (e / 3);
        cx<double> s = cmul(at(A, i, 0), at(B, 0, j));
        s = cfma(at(A, i, 1), at(B, 1, j), s);
        s = cfma(at(A, i, 2), at(B, 2, j), s);
        reinterpret_cast<double2*>(C)[e] = make_double2(s.r, s.i);
    }
    // component r of A v (v: 3 complex)
    static __device__ __forceinline__ cx<double> matvec_row(const double* A, const double* v, int r)
    {
        const double2* w = reinterpret_cast<const double2*>(v);
        cx<double> s = cmul(at(A, r, 0), cmk(w[0].x, w[0].y));
        s = cfma(at(A, r, 1), cmk(w[1].x, w[1].y), s);
        s = cfma(at(A, r, 2), cmk(w[2].x, w[2].y), s);
        return s;
    }
};

// SU(2) element [[alpha, -conj(beta)], [beta, conj(alpha)]] stored as (alpha, beta).
template <>
struct Tree<2> {
    static constexpr int D = 4;
    static constexpr int E = 2;
    static __device__ __forceinline__ void prod_entry(const double* A, const double* B, int e, double* C)
    {
        const double2* a = reinterpret_cast<const double2*>(A);
        const double2* b = reinterpret_cast<const double2*>(B);
        const cx<double> a1 = cmk(a[0].x, a[0].y), b1 = cmk(a[1].x, a[1].y);
        const cx<double> a2 = cmk(b[0].x, b[0].y), b2 = cmk(b[1].x, b[1].y);
        cx<double> s;
        if (e == 0) s = csub(cmul(a1, a2), cmul(cconj(b1), b2));   // alpha = a1 a2 - conj(b1) b2
        else s = cfma_conj(a1, b2, cmul(b1, a2));                  // beta = b1 a2 + conj(a1) b2
        reinterpret_cast<double2*>(C)[e] = make_double2(s.r, s.i);
    }
    static __device__ __forceinline__ cx<double> matvec_row(const double* A, const double* v, int r)
    {
        const double2* a = reinterpret_cast<const double2*>(A);
        const double2* w = reinterpret_cast<const double2*>(v);
        const cx<double> al = cmk(a[0].x, a[0].y), be = cmk(a[1].x, a[1].y);
        const cx<double> v0 = cmk(w[0].x, w[0].y), v1 = cmk(w[1].x, w[1].y);
        // [alpha v0 - conj(beta) v1, beta v0 + conj(alpha) v1]
        return r == 0 ? csub(cmul(al, v0), cmul(cconj(be), v1)) : cfma_conj(al, v1, cmul(be, v0));
    }
};

// Up-sweep of a warp's tree: leaves in slots 0..31, products of every
// internal node, one entry per lane per round.
template <int N>
__device__ __forceinline__ void tree_up(double* S, int lane)
{
    constexpr int D = Tree<N>::D, E = Tree<N>::E;
#pragma unroll 1
    for (int h = 1; h <= 5; h++) {
        const int P = 32 >> h;
        for (int t = lane; t < P * E; t += 32) {
            const int p = t / E, e = t - E * (t / E);
            Tree<N>::prod_entry(S + tslot(h - 1, 2 * p + 1) * D, S + tslot(h - 1, 2 * p) * D, e, S + tslot(h, p) * D);
        }
        __syncwarp();
    }
}

// Down-sweep: the state entering the node is in V slot tslot(5, 0); the
// states entering the 32 leaves end in slots 0..31.  `left(t)` returns the
// left-child product of internal node 32 + t.
template <int N, typename Left>
__device__ __forceinline__ void tree_down(double* V, Left left, int lane)
{
    constexpr int SV = 2 * N;   // doubles per state
#pragma unroll 1
    for (int h = 5; h >= 1; h--) {
        const int P = 32 >> h;
        for (int t = lane; t < P * N; t += 32) {
            const int p = t / N, r = t - N * (t / N);
            const double* v = V + tslot(h, p) * SV;
            const cx<double> y = Tree<N>::matvec_row(left(tslot(h, p) - 32), v, r);
            double* vl = V + tslot(h - 1, 2 * p) * SV;
            double* vr = V + tslot(h - 1, 2 * p + 1) * SV;
            vl[2 * r] = v[2 * r];
            vl[2 * r + 1] = v[2 * r + 1];
            vr[2 * r] = y.r;
            vr[2 * r + 1] = y.i;
        }
        __syncwarp();
    }
}

// Shared memory of one warp: the tree (63 operators) and its states (63).
template <int N>
constexpr int warp_tree_doubles() { return 63 * Tree<N>::D + 63 * 2 * N; }
template <int N>
constexpr int warp_state_doubles() { return 63 * 2 * N; }
constexpr int kChainWarps = 4;   // warps per block of the chain kernels

// ------------------------------------------------------------------ kernels
// Up-sweep of level `level`: one warp per node.  The node's leaves are its
// lanes' runs (level 0) or its children's products; its binary tree's
// left-child products and its total are stored.  At a simulation's top node
// (whole scan only) the warp goes on down its tree from psi0 and stores the
// states entering the top node's children.
template <int N>
__global__ void __launch_bounds__(128) chain_up_kernel(ChainArgs a, int level)
{
    constexpr int D = Tree<N>::D, SV = 2 * N;
    extern __shared__ __align__(16) double smem[];
    // programmatic dependent launch: the previous kernel's results are
    // visible after this wait; the next chain kernel may be scheduled now
    grid_dependency_wait();
    allow_dependent_launch();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* S = smem + warp * warp_tree_doubles<N>();
    double* V = S + 63 * D;
    const int64_t* off = a.level_off + (size_t)level * (a.n_sims + 1);
    const int64_t* coff = level > 0 ? off - (a.n_sims + 1) : nullptr;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t node = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; node < a.nodes[level]; node += warps) {
        const int si = find_node_sim(off, a.n_sims, node);
        const DevSim& s = a.sims[si];
        const int64_t local = node - off[si];
        Op<N> B;
        B.identity();
        if (level == 0) {
            // lane run: U_{k1-1} ... U_{k0} (the first operator loaded, not
            // multiplied into the identity)
            const int run = s.chain_run;
            const int64_t k0 = (local * kFan + lane) * run;
            const int64_t k1 = min(k0 + run, s.K);
            const double* U = a.U + s.sample_offset * D;
            if (k0 < k1) B.load(U + k0 * D);
            for (int64_t k = k0 + 1; k < k1; k++) {
                Op<N> u, t;
                u.load(U + k * D);
                Op<N>::mul(u, B, t);   // later operators multiply from the left
                B = t;
            }
        } else {
            const int64_t child = local * kFan + lane;
            if (child < coff[si + 1] - coff[si]) B.load(a.agg[level - 1] + (coff[si] + child) * D);
        }
        B.store(S + lane * D);
        __syncwarp();
        tree_up<N>(S, lane);
        if (lane < kLeftPerNode) {
            const double2* src = reinterpret_cast<const double2*>(S + left_child_slot(lane) * D);
            double2* dst = reinterpret_cast<double2*>(a.left[level] + (node * kLeftPerNode + lane) * D);
#pragma unroll
            for (int i = 0; i < D / 2; i++) dst[i] = src[i];
        } else {
            const double2* src = reinterpret_cast<const double2*>(S + tslot(5, 0) * D);
            double2* dst = reinterpret_cast<double2*>(a.agg[level] + node * D);
#pragma unroll
            for (int i = 0; i < D / 2; i++) dst[i] = src[i];
        }
        if (level >= 1 && s.chain_top == level && a.mode == kChainFull) {
            if (lane < SV) V[tslot(5, 0) * SV + lane] = s.psi0[lane];
            __syncwarp();
            tree_down<N>(V, [&](int t) { return (const double*)(S + left_child_slot(t) * D); }, lane);
            const int64_t child = local * kFan + lane;
            if (child < coff[si + 1] - coff[si]) {
                double* dst = a.state[level - 1] + (coff[si] + child) * SV;
#pragma unroll
                for (int i = 0; i < SV; i++) dst[i] = V[lane * SV + i];
            }
        }
        __syncwarp();
    }
}

// Down-sweep and output: one warp per level-0 node.  The state entering the
// node follows by walking down to it: in the whole scan from the state the
// top node's up-sweep stored for its child on this node's path (psi0 for a
// simulation of one node), in the down-only mode (a range whose entering
// state arrived later) from psi0 at the top node.  Inside each ancestor's
// binary tree, a step into a right child applies the left sibling's product
// (one matrix row per lane).  The node's own tree then gives every lane run
// its entering state; each lane walks its run, writing psi_k, <J>_k and
// (optionally) U_k.
template <int N>
__global__ void __launch_bounds__(128) chain_apply_kernel(ChainArgs a)
{
    constexpr int D = Tree<N>::D, SV = 2 * N;
    extern __shared__ __align__(16) double smem[];
    grid_dependency_wait();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* V = smem + warp * warp_state_doubles<N>();
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
            if (lane < SV) v[lane] = a.state[from][(a.level_off[(size_t)from * stride + si] + anc) * SV + lane];
        } else if (lane < SV) {
            v[lane] = s.psi0[lane];
        }
        __syncwarp();
        for (int level = from; level >= 1; level--) {
            const int64_t anc = local >> (5 * level);                         // ancestor at `level`
            const int64_t j = (local >> (5 * (level - 1))) - anc * kFan;     // its child on the path
            const double* L = a.left[level] + (a.level_off[(size_t)level * stride + si] + anc) * kLeftPerNode * D;
            for (int h = 5; h >= 1; h--) {
                if (((j >> (h - 1)) & 1) == 0) continue;                    // left child: state unchanged
                const int p = (int)(j >> h);
                cx<double> y = cmk(0.0, 0.0);
                if (lane < N) y = Tree<N>::matvec_row(L + (tslot(h, p) - 32) * D, v, lane);
                __syncwarp();
                if (lane < N) {
                    v[2 * lane] = y.r;
                    v[2 * lane + 1] = y.i;
                }
                __syncwarp();
            }
        }
        const double* L0 = a.left[0] + node * kLeftPerNode * D;
        tree_down<N>(V, [&](int t) { return L0 + t * D; }, lane);
        cx<double> psi[N], nxt[N];
#pragma unroll
        for (int i = 0; i < N; i++) psi[i] = cmk(V[lane * SV + 2 * i], V[lane * SV + 2 * i + 1]);
        __syncwarp();
        const int run = s.chain_run;
        const int64_t k0 = (local * kFan + lane) * run;
        const int64_t k1 = min(k0 + run, s.K);
        const double* U = a.U + s.sample_offset * D;
        for (int64_t k = k0; k < k1; k++) {
            Op<N> u;
            u.load(U + k * D);
            u.apply(psi, nxt);
#pragma unroll
            for (int i = 0; i < N; i++) psi[i] = nxt[i];
            cx<double> w[N];
            double scale = 1.0;
            if (s.normalize_out) {
                // FP32-bulk: the written state is renormalised in FP64
                double n2 = 0.0;
#pragma unroll
                for (int i = 0; i < N; i++) n2 = fma(psi[i].r, psi[i].r, fma(psi[i].i, psi[i].i, n2));
                const double d = n2 - 1.0;
                scale = 1.0 - d * (0.5 - 0.375 * d);   // (1 + d)^(-1/2), |d| ~ 1e-9
            }
#pragma unroll
            for (int i = 0; i < N; i++) w[i] = cscale(psi[i], scale);
            double2* sp = reinterpret_cast<double2*>(s.states + k * 2 * N);
#pragma unroll
            for (int i = 0; i < N; i++) sp[i] = make_double2(w[i].r, w[i].i);
            if (s.spin) {
                double jv[3];
                spin_projection(w, N, jv);
                s.spin[k * 3 + 0] = jv[0];
                s.spin[k * 3 + 1] = jv[1];
                s.spin[k * 3 + 2] = jv[2];
            }
            if (s.ops) u.store_full(s.ops + k * 2 * N * N);
        }
    }
}

// ----------------------------------------------------------------- launcher
template <int N>
static cudaError_t launch_chain_n(const ChainArgs& a, int n_sm, cudaStream_t stream, int* kernels)
{
    *kernels = 0;
    if (a.levels < 1 || a.nodes[0] == 0) return cudaSuccess;
    const int block = 32 * kChainWarps;
    const size_t up_smem = (size_t)kChainWarps * warp_tree_doubles<N>() * sizeof(double);
    const size_t down_smem = (size_t)kChainWarps * warp_state_doubles<N>() * sizeof(double);
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
    if (a.mode != kChainDown)
        for (int l = 0; l < a.levels; l++) {
            cfg.gridDim = dim3(grid(a.nodes[l]));
            cfg.dynamicSmemBytes = up_smem;
            const cudaError_t e = cudaLaunchKernelEx(&cfg, chain_up_kernel<N>, args, l);
            if (e != cudaSuccess) return e;
            (*kernels)++;
        }
    if (a.mode != kChainUp) {
        cfg.gridDim = dim3(grid(a.nodes[0]));
        cfg.dynamicSmemBytes = down_smem;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, chain_apply_kernel<N>, args);
        if (e != cudaSuccess) return e;
        (*kernels)++;
    }
    return cudaGetLastError();
}

cudaError_t launch_chain(int spin_x2, const ChainArgs& a, int n_sm, cudaStream_t stream, int* kernels)
{
    if (spin_x2 == 2) return launch_chain_n<3>(a, n_sm, stream, kernels);
    if (spin_x2 == 1) return launch_chain_n<2>(a, n_sm, stream, kernels);
    return cudaErrorInvalidValue;
}

}  // namespace spinsim
