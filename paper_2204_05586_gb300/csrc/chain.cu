// chain.cu -- ordered prefix product of the sample operators and the output
// write (Sec. 1.2.4, Eq. integration_compilation: psi_k = U_k psi_{k-1}).
//
// The paper chains the U_k sequentially on the CPU.  Here the chain is a
// parallel scan in FP64 on the device, over chunks of kChunk = 256 samples
// and groups of kGroup = 32 chunks, neither of which straddles two
// simulations:
//   reduce:     one warp per chunk; lane l multiplies its run of kRun = 8
//               operators in order, then the warp forms inclusive prefixes
//               P_l = B_l ... B_0 of the run products by a shuffle scan
//               (Hillis-Steele, 5 levels) and stores each lane's exclusive
//               prefix and the chunk product;
//   group scan: one warp per group scans its 32 chunk products the same way
//               and stores each chunk's exclusive prefix and the group product;
//   carry:      one warp per simulation walks its group products in order
//               (one matrix row per lane) and stores the state entering every
//               group;
//   apply:      one warp per chunk forms the state entering the chunk and
//               each lane's run from the prefixes, then walks its 8 samples,
//               writing psi_k, <J>_k and (optionally) U_k.
// On GB300 a 32-lane FP64 instruction keeps an SM sub-partition busy for
// tens of cycles, so the FP64 work is spread over many warps and the
// sequential part (the carry) is kept short and row-parallel.
// Spin-one operators are general 3x3 complex matrices; spin-half operators
// are kept in SU(2) form (alpha, beta) = first column.
#include <algorithm>

#include "device_math.cuh"

namespace spinsim {

__device__ __forceinline__ int find_chunk_sim(const int64_t* off, int n, int64_t c)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= c) lo = mid;
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
    __device__ __forceinline__ void shfl_up(unsigned d)
    {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                m[i][j].r = __shfl_up_sync(0xffffffffu, m[i][j].r, d);
                m[i][j].i = __shfl_up_sync(0xffffffffu, m[i][j].i, d);
            }
    }
    __device__ __forceinline__ void shfl_idx(int src)
    {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                m[i][j].r = __shfl_sync(0xffffffffu, m[i][j].r, src);
                m[i][j].i = __shfl_sync(0xffffffffu, m[i][j].i, src);
            }
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
    __device__ __forceinline__ void shfl_up(unsigned d)
    {
        a.r = __shfl_up_sync(0xffffffffu, a.r, d);
        a.i = __shfl_up_sync(0xffffffffu, a.i, d);
        b.r = __shfl_up_sync(0xffffffffu, b.r, d);
        b.i = __shfl_up_sync(0xffffffffu, b.i, d);
    }
    __device__ __forceinline__ void shfl_idx(int src)
    {
        a.r = __shfl_sync(0xffffffffu, a.r, src);
        a.i = __shfl_sync(0xffffffffu, a.i, src);
        b.r = __shfl_sync(0xffffffffu, b.r, src);
        b.i = __shfl_sync(0xffffffffu, b.i, src);
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

// <J_x>, <J_y>, <J_z> = psi^dagger J psi (Sec. 1.2.1)
__device__ __forceinline__ void spin_projection(const cx<double>* p, int N, double* out)
{
    if (N == 3) {
        // J_x, J_y have 1/sqrt2 off-diagonals: <J_x> + i <J_y> = sqrt2 (conj(p0) p1 + conj(p1) p2)
        cx<double> z = cfma_conj(p[1], p[2], cfma_conj(p[0], p[1], cmk(0.0, 0.0)));
        out[0] = kSqrt2 * z.r;
        out[1] = kSqrt2 * z.i;
        out[2] = (p[0].r * p[0].r + p[0].i * p[0].i) - (p[2].r * p[2].r + p[2].i * p[2].i);
    } else {
        cx<double> z = cfma_conj(p[0], p[1], cmk(0.0, 0.0));
        out[0] = z.r;
        out[1] = z.i;
        out[2] = 0.5 * ((p[0].r * p[0].r + p[0].i * p[0].i) - (p[1].r * p[1].r + p[1].i * p[1].i));
    }
}

// ------------------------------------------------------------------ kernels
template <int N>
__global__ void __launch_bounds__(128) chain_reduce_kernel(ChainArgs a)
{
    constexpr int OPD = N == 3 ? 18 : 4;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < a.n_chunks; c += warps) {
        const int si = find_chunk_sim(a.chunk_offsets, a.n_sims, c);
        const DevSim& s = a.sims[si];
        const int64_t j = c - a.chunk_offsets[si];
        const int64_t k0 = j * kChunk + (int64_t)lane * kRun;
        const int64_t k1 = min(k0 + kRun, s.K);
        Op<N> B;
        B.identity();
        const double* U = a.U + (s.sample_offset) * OPD;
        for (int64_t k = k0; k < k1; k++) {
            Op<N> u, t;
            u.load(U + k * OPD);
            Op<N>::mul(u, B, t);   // later operators multiply from the left
            B = t;
        }
        // inclusive prefix P_l = B_l ... B_0 across the warp
        Op<N> P = B;
#pragma unroll
        for (unsigned d = 1; d < 32; d <<= 1) {
            Op<N> o = P;
            o.shfl_up(d);
            if (lane >= (int)d) {
                Op<N> t;
                Op<N>::mul(P, o, t);
                P = t;
            }
        }
        Op<N> M = P;
        M.shfl_up(1);
        if (lane == 0) M.identity();
        M.store(a.run_prefix + (c * 32 + lane) * OPD);
        if (lane == 31) P.store(a.chunk_agg + c * OPD);
    }
}

// Group scan: one warp per group of up to 32 consecutive chunks of one
// simulation; inclusive prefixes of the chunk products by a shuffle scan.
template <int N>
__global__ void __launch_bounds__(128) chain_group_kernel(ChainArgs a)
{
    constexpr int OPD = N == 3 ? 18 : 4;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < a.n_groups; g += warps) {
        const int si = find_chunk_sim(a.group_offsets, a.n_sims, g);
        const int64_t c_first = a.chunk_offsets[si] + (g - a.group_offsets[si]) * kGroup;
        const int64_t c_end = a.chunk_offsets[si + 1];
        const int64_t c = c_first + lane;
        Op<N> P;
        if (c < c_end) P.load(a.chunk_agg + c * OPD);
        else P.identity();
#pragma unroll
        for (unsigned d = 1; d < 32; d <<= 1) {
            Op<N> o = P;
            o.shfl_up(d);
            if (lane >= (int)d) {
                Op<N> t;
                Op<N>::mul(P, o, t);
                P = t;
            }
        }
        Op<N> M = P;
        M.shfl_up(1);
        if (lane == 0) M.identity();
        if (c < c_end) M.store(a.chunk_gprefix + c * OPD);
        if (lane == 31) P.store(a.group_agg + g * OPD);
    }
}

// Carry: one warp per simulation walks its group products in order.  Lane r
// (r < N) holds row r of the product and computes component r of the next
// state; the state is broadcast to all lanes by shuffles.
template <int N>
__global__ void __launch_bounds__(128) chain_carry_kernel(ChainArgs a)
{
    constexpr int OPD = N == 3 ? 18 : 4;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t si = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); si < a.n_sims; si += warps) {
        const DevSim& s = a.sims[si];
        cx<double> psi[N];
#pragma unroll
        for (int i = 0; i < N; i++) psi[i] = cmk(s.psi0[2 * i], s.psi0[2 * i + 1]);
        const int64_t g0 = a.group_offsets[si], g1 = a.group_offsets[si + 1];
        const int r = lane < N ? lane : 0;
        for (int64_t g = g0; g < g1; g++) {
            if (lane < N) {
                double* st = a.group_start + g * (2 * N);
                st[2 * lane] = psi[lane].r;
                st[2 * lane + 1] = psi[lane].i;
            }
            // row r of the group product
            cx<double> row[N];
            const double* Ag = a.group_agg + g * OPD;
            if (N == 3) {
#pragma unroll
                for (int j = 0; j < N; j++) row[j] = cmk(Ag[6 * r + 2 * j], Ag[6 * r + 2 * j + 1]);
            } else {
                // [[alpha, -conj(beta)], [beta, conj(alpha)]]
                const cx<double> al = cmk(Ag[0], Ag[1]), be = cmk(Ag[2], Ag[3]);
                row[0] = r == 0 ? al : be;
                row[N - 1] = r == 0 ? cmk(-be.r, be.i) : cconj(al);
            }
            cx<double> v = cmul(row[0], psi[0]);
#pragma unroll
            for (int j = 1; j < N; j++) v = cfma(row[j], psi[j], v);
#pragma unroll
            for (int i = 0; i < N; i++) {
                psi[i].r = __shfl_sync(0xffffffffu, v.r, i);
                psi[i].i = __shfl_sync(0xffffffffu, v.i, i);
            }
        }
    }
}

template <int N>
__global__ void __launch_bounds__(128) chain_apply_kernel(ChainArgs a)
{
    constexpr int OPD = N == 3 ? 18 : 4;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < a.n_chunks; c += warps) {
        const int si = find_chunk_sim(a.chunk_offsets, a.n_sims, c);
        const DevSim& s = a.sims[si];
        const int64_t j = c - a.chunk_offsets[si];
        const int64_t k0 = j * kChunk + (int64_t)lane * kRun;
        const int64_t k1 = min(k0 + kRun, s.K);
        if (k0 >= k1) continue;
        const int64_t g = a.group_offsets[si] + j / kGroup;
        cx<double> gs[N], cs[N], psi[N], nxt[N];
#pragma unroll
        for (int i = 0; i < N; i++) gs[i] = cmk(a.group_start[g * 2 * N + 2 * i], a.group_start[g * 2 * N + 2 * i + 1]);
        Op<N> G;
        G.load(a.chunk_gprefix + c * OPD);
        G.apply(gs, cs);                 // state entering the chunk
        Op<N> M;
        M.load(a.run_prefix + (c * 32 + lane) * OPD);
        M.apply(cs, psi);                // state entering this lane's run
        const double* U = a.U + s.sample_offset * OPD;
        for (int64_t k = k0; k < k1; k++) {
            Op<N> u;
            u.load(U + k * OPD);
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
static cudaError_t launch_chain_n(const ChainArgs& a, int n_sm, cudaStream_t stream)
{
    if (a.n_chunks == 0) return cudaSuccess;
    const int block = 128;
    const int64_t want = (a.n_chunks + 3) / 4;
    const int grid = (int)std::min<int64_t>(want, (int64_t)n_sm * 16);
    ChainArgs args = a;
    chain_reduce_kernel<N><<<grid, block, 0, stream>>>(args);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int ggrid = (int)std::min<int64_t>((a.n_groups + 3) / 4, (int64_t)n_sm * 16);
    chain_group_kernel<N><<<ggrid, block, 0, stream>>>(args);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int cgrid = (int)std::min<int64_t>((a.n_sims + 3) / 4, (int64_t)n_sm * 16);
    chain_carry_kernel<N><<<cgrid, 128, 0, stream>>>(args);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    chain_apply_kernel<N><<<grid, block, 0, stream>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_chain(int spin_x2, const ChainArgs& a, int n_sm, cudaStream_t stream)
{
    if (spin_x2 == 2) return launch_chain_n<3>(a, n_sm, stream);
    if (spin_x2 == 1) return launch_chain_n<2>(a, n_sm, stream);
    return cudaErrorInvalidValue;
}

}  // namespace spinsim
