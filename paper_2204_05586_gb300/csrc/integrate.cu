// integrate.cu -- sample-operator kernel: U_k for every output interval.
//
// Sec. 1.2.4 / 1.2.6: the U_k = U(t_k, t_{k-1}) depend only on the field, so
// they are computed independently.  Each U_k is the product u_{L-1} ... u_0 of
// L integration steps (CF4 by default), taken inside the interval's rotating
// frame and then moved back to the lab frame (Eq. exit_rotating_frame).
//
// Work decomposition (GB300): a persistent grid pulls tiles of consecutive
// samples from an atomic counter; G = 1, 2 or 4 lanes of a warp share one
// sample.  The L steps of a sample are always split into the same four
// segments [s L/4, (s+1) L/4) and reduced by the same tree
// (S3 S2)(S1 S0), whichever G is used, so the result is bit-for-bit
// independent of the launch shape and of which other samples share the batch.
// A lane computes its segments' residual products in registers and leaves
// them in shared memory; lane 0 of the group combines them, finishes the
// operator in FP64 and stores it.
#include "device_math.cuh"

namespace spinsim {

__device__ __forceinline__ int find_index(const int64_t* off, int n, int64_t g)
{
    // largest i in [0, n) with off[i] <= g (off is non-decreasing, off[0] = 0)
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int N, typename R>
struct ResType;
template <typename R>
struct ResType<3, R> { using type = Res3<R>; };
template <typename R>
struct ResType<2, R> { using type = Res2<R>; };

// ---------------------------------------------------------------- epilogues
// The sample operator is U^r = I + F(g) + rest with the first-order
// coefficients g replaced by their exact FP64 values (transverse: closed-form
// quadrature sum; quadrupole: w_q dt_out; z: the accumulated pulse part).
// Leaving the frame (Eq. exit_rotating_frame) scales the rows of U^r by the
// diagonal of R(-Delta_t): spin-one rows m = +1, 0, -1 by
// (e^{-i w_r Dt}, 1, e^{+i w_r Dt}), spin-half (alpha, beta) by (e^{-i w_r Dt/2}, e^{+i w_r Dt/2}).

// Rows m = +1 and m = -1 are scaled by the exit phasor and its conjugate;
// row m = 0 is stored as it is (factor 1).
__device__ __forceinline__ void store_rows(const cx<double> U[3][3], cx<double> ph, double* out)
{
    const cx<double> r[3] = {ph, cmk(1.0, 0.0), cconj(ph)};
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const cx<double> v = i == 1 ? U[i][j] : cmul(r[i], U[i][j]);
            out[6 * i + 2 * j] = v.r;
            out[6 * i + 2 * j + 1] = v.i;
        }
}

// U^r - I in FP64 from the split residual with exact first-order coefficients.
template <typename R>
__device__ __forceinline__ void promote(const Res3<R>& P, const DevSim& s, const SampleExact& x, cx<double> Y[3][3])
{
    double gx, gy;
    first_order_exact(s, x, gx, gy);
    const double gz = (double)P.g[2], q3 = s.gq * (1.0 / 3.0);
    const cx<double> up = cmk(-gy * kInvSqrt2, -gx * kInvSqrt2);
    const cx<double> dn = cmk(gy * kInvSqrt2, -gx * kInvSqrt2);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) Y[i][j] = cmk((double)P.m[i][j].r, (double)P.m[i][j].i);
    Y[0][0].i -= gz + q3;
    Y[1][1].i += 2.0 * q3;
    Y[2][2].i += gz - q3;
    Y[0][1] = cadd(Y[0][1], up);
    Y[1][2] = cadd(Y[1][2], up);
    Y[1][0] = cadd(Y[1][0], dn);
    Y[2][1] = cadd(Y[2][1], dn);
}

__device__ __forceinline__ void finish(const Res3<double>& P, const DevSim& s, const SampleExact& x, double* out)
{
    cx<double> Y[3][3];
    promote(P, s, x, Y);
#pragma unroll
    for (int i = 0; i < 3; i++) Y[i][i].r += 1.0;
    store_rows(Y, cmk(x.ph_re, x.ph_im), out);
}

// FP32-bulk: the operator is stored as computed.  Its departure from
// unitarity is of the order of the FP32 rounding of the second-order rest
// (~1e-11 per sample); the chain renormalises every output state in FP64.
__device__ __forceinline__ void finish(const Res3<float>& P, const DevSim& s, const SampleExact& x, double* out)
{
    cx<double> Y[3][3];
    promote(P, s, x, Y);
#pragma unroll
    for (int i = 0; i < 3; i++) Y[i][i].r += 1.0;
    store_rows(Y, cmk(x.ph_re, x.ph_im), out);
}

template <typename R>
__device__ __forceinline__ void promote(const Res2<R>& P, const DevSim& s, const SampleExact& x, cx<double>& a,
                                        cx<double>& b)
{
    double gx, gy;
    first_order_exact(s, x, gx, gy);
    const double gz = (double)P.g[2];
    a = cmk((double)P.a.r, (double)P.a.i - 0.5 * gz);
    b = cmk((double)P.b.r + 0.5 * gy, (double)P.b.i - 0.5 * gx);
}

__device__ __forceinline__ void store_half(cx<double> al, cx<double> be, const SampleExact& x, double* out)
{
    const cx<double> p = cmk(x.ph_re, x.ph_im);
    cx<double> a = cmul(p, al);
    cx<double> b = cmul(cconj(p), be);
    out[0] = a.r; out[1] = a.i; out[2] = b.r; out[3] = b.i;
}

__device__ __forceinline__ void finish(const Res2<double>& P, const DevSim& s, const SampleExact& x, double* out)
{
    cx<double> a, b;
    promote(P, s, x, a, b);
    store_half(cmk(1.0 + a.r, a.i), b, x, out);
}

// FP32-bulk spin-half: stored as computed (see the spin-one case); an SU(2)
// element in this form always has det 1.
__device__ __forceinline__ void finish(const Res2<float>& P, const DevSim& s, const SampleExact& x, double* out)
{
    cx<double> a, b;
    promote(P, s, x, a, b);
    store_half(cmk(1.0 + a.r, a.i), b, x, out);
}

__device__ __forceinline__ void store_identity(int N, double* out)
{
    if (N == 3) {
#pragma unroll
        for (int i = 0; i < 18; i++) out[i] = (i == 0 || i == 8 || i == 16) ? 1.0 : 0.0;
    } else {
        out[0] = 1.0; out[1] = 0.0; out[2] = 0.0; out[3] = 0.0;
    }
}

// ------------------------------------------------------------------- kernel
template <int N, typename R, int G, int METHOD, bool SMALL>
__global__ void __launch_bounds__(256) integrate_kernel(IntegrateArgs a)
{
    using Res = typename ResType<N, R>::type;
    constexpr int OPD = N == 3 ? 18 : 4;
    constexpr int SEG_PER_LANE = kSegments / G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Res* seg = reinterpret_cast<Res*>(smem_raw);
    __shared__ unsigned long long s_tile;

    const int spb = blockDim.x / G;
    const int slot = threadIdx.x / G;
    const int lane = threadIdx.x % G;

    // Never touch shared memory beyond what the launch provided.
    unsigned dyn_smem;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
    if ((size_t)spb * kSegments * sizeof(Res) > (size_t)dyn_smem) return;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_counter, 1ULL);
        __syncthreads();
        const unsigned long long tile = s_tile;
        if (tile >= (unsigned long long)a.n_tiles) return;

        const int64_t g = (int64_t)tile * spb + slot;
        const bool active = g < a.total_samples;
        int si = 0;
        int64_t k = 0;
        if (active) {
            si = find_index(a.sample_offsets, a.n_sims, g);
            k = g - a.sample_offsets[si];
        }
        double gsum = 0.0, beta = 0.0;
        if (active && k > 0) {
            const DevSim& s = a.sims[si];
            SampleCtx<R> c;
            gsum = make_ctx<R, N>(s, k, c, beta);
            const int64_t L = s.L;
#pragma unroll 1
            for (int q = 0; q < SEG_PER_LANE; q++) {
                const int sg = lane * SEG_PER_LANE + q;
                const int64_t lo = (sg * L) / kSegments, hi = ((sg + 1) * L) / kSegments;
                Res X;
                res_zero(X);
#pragma unroll 1
                for (int64_t l = lo; l < hi; l++) step_apply<R, METHOD, SMALL>(c, (R)l, c.tau, X);   // U <- u_l U
                seg[slot * kSegments + sg] = X;
            }
        }
        __syncwarp();
        if (active && lane == 0) {
            double* out = a.U + g * OPD;
            if (k == 0) {
                store_identity(N, out);
            } else {
                Res P01, P23, P;
                res_mul(seg[slot * kSegments + 1], seg[slot * kSegments + 0], P01);
                res_mul(seg[slot * kSegments + 3], seg[slot * kSegments + 2], P23);
                res_mul(P23, P01, P);
                const DevSim& s = a.sims[si];
                SampleExact sx;
                make_exact<N>(s, beta, gsum, sx);
                finish(P, s, sx, out);
            }
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------- launchers
template <int N, typename R, int G, int METHOD, bool SMALL>
static void* kernel_ptr()
{
    return (void*)integrate_kernel<N, R, G, METHOD, SMALL>;
}

template <int N, typename R, int METHOD, bool SMALL>
static void* pick_lanes(int lanes)
{
    switch (lanes) {
        case 1: return kernel_ptr<N, R, 1, METHOD, SMALL>();
        case 2: return kernel_ptr<N, R, 2, METHOD, SMALL>();
        case 4: return kernel_ptr<N, R, 4, METHOD, SMALL>();
        default: return nullptr;
    }
}

template <int N, typename R, bool SMALL>
static void* pick_method(int method, int lanes)
{
    switch (method) {
        case 0: return pick_lanes<N, R, 0, SMALL>(lanes);
        case 1: return pick_lanes<N, R, 1, SMALL>(lanes);
        case 2: return pick_lanes<N, R, 2, SMALL>(lanes);
        default: return nullptr;
    }
}

// The small-angle variant exists for FP32-bulk only; FP64 keeps the general
// series (its terms are sized for double precision).
static void* select_kernel(int spin_x2, int precision, int method, int lanes, bool small)
{
    if (spin_x2 == 2) {
        if (!precision) return pick_method<3, double, false>(method, lanes);
        return small ? pick_method<3, float, true>(method, lanes) : pick_method<3, float, false>(method, lanes);
    }
    if (spin_x2 == 1) {
        if (!precision) return pick_method<2, double, false>(method, lanes);
        return small ? pick_method<2, float, true>(method, lanes) : pick_method<2, float, false>(method, lanes);
    }
    return nullptr;
}

// Dynamic shared memory of one block: kSegments residual records per sample
// slot, sized from the record type itself.
size_t integrate_smem_bytes(int spin_x2, int precision, int lanes, int block)
{
    size_t res;
    if (spin_x2 == 2) res = precision ? sizeof(Res3<float>) : sizeof(Res3<double>);
    else res = precision ? sizeof(Res2<float>) : sizeof(Res2<double>);
    return (size_t)(block / lanes) * kSegments * res;
}

// Must be called (outside stream capture) before the first launch of a
// (spin, precision, method, lanes) kernel: it raises the kernel's dynamic
// shared-memory limit to what a 256-thread block needs.
cudaError_t integrate_occupancy(int spin_x2, int precision, int method, int lanes, int block, bool small,
                                int* blocks_per_sm)
{
    void* k = select_kernel(spin_x2, precision, method, lanes, small);
    if (!k) return cudaErrorInvalidValue;
    size_t smem_max = integrate_smem_bytes(spin_x2, precision, lanes, 256);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e != cudaSuccess) return e;
    size_t smem = integrate_smem_bytes(spin_x2, precision, lanes, block);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, block, smem);
}

cudaError_t launch_integrate(int spin_x2, int precision, int method, int lanes, int block, int grid, bool small,
                             const IntegrateArgs& a, cudaStream_t stream)
{
    void* k = select_kernel(spin_x2, precision, method, lanes, small);
    if (!k || block % 32 != 0 || block < 32 || block > 256 || grid < 1) return cudaErrorInvalidValue;
    size_t smem = integrate_smem_bytes(spin_x2, precision, lanes, block);
    IntegrateArgs args = a;
    void* params[] = {&args};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), params, smem, stream);
}

}  // namespace spinsim
