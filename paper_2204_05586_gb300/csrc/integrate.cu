// integrate.cu -- sample-operator kernel: U_k for every output interval.
//
// Sec. 1.2.4 / 1.2.6: the U_k = U(t_k, t_{k-1}) depend only on the field, so
// they are computed independently.  Each U_k is the product u_{L-1} ... u_0 of
// L integration steps (CF4 by default), taken inside the interval's rotating
// frame and then moved back to the lab frame (Eq. exit_rotating_frame).
//
// Work decomposition (GB300): in a persistent grid every warp pulls tiles of
// 32 / G consecutive samples from an atomic counter; G = 1, 2, 4 or 8 lanes of
// the warp share one sample.  The L steps of a sample are always split into the same 2^s
// segments [q L/2^s, (q+1) L/2^s) (s from L alone: 3 for L >= 128, 2 from 16,
// 1 from 4, else 0) and reduced by the same binary tree, e.g. for s = 3
// ((S7 S6)(S5 S4))((S3 S2)(S1 S0)), whichever G is used, so the result is
// bit-for-bit independent of the launch shape and of which other samples
// share the launch.  A lane owns 2^s/G consecutive segments -- a complete
// sub-tree, built as its segments finish with a small stack in shared memory.
// After the tile, one lane per sample combines the lanes' sub-trees and
// finishes the operator in FP64: on GB300 an FP64 warp instruction costs the
// same with 1 or 32 active lanes, so this epilogue runs with every lane on a
// sample of its own (in bulk tiles, G = 1).  Whole waves of tiles use the tuned G; the samples left
// after them use one lane per segment, so the last wave ends in segments of a
// sample's steps.
#include "bounds.cuh"
#include "sample_epilogue.cuh"
#include "lanes2.cuh"

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

// ------------------------------------------------------------------- kernel
// Per thread kSlots residual records of shared memory: the stack of the
// thread's canonical sub-tree (log2 of its segment count) and its result.
constexpr int kSlots = kSegLog2 + 1;

// The body of both integrate kernels (below).  Each warp works on its own:
// it pulls a tile of 32 >> lg consecutive samples from the atomic counter,
// its lanes build their segments' sub-trees, and lanes 0 .. (32 >> lg) - 1
// then finish one sample each (the FP64 epilogue).  No block barrier: while
// one warp runs its FP64 epilogue, the others of its SM keep the FP32 pipes
// busy.
template <int N, typename R, int METHOD, int SMALL, bool TONES, bool SU3 = false>
__device__ __forceinline__ void integrate_body(const IntegrateArgs& a)
{
    using Res = typename ResType<N, R>::type;
    constexpr int OPD = N == 3 ? 18 : 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Res* rec = reinterpret_cast<Res*>(smem_raw);                                        // [blockDim][kSlots]
    double2* bg = reinterpret_cast<double2*>(smem_raw + (size_t)blockDim.x * kSlots * sizeof(Res));  // [blockDim]

    // Never touch shared memory beyond what the launch provided.
    unsigned dyn_smem;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
    if ((size_t)blockDim.x * (kSlots * sizeof(Res) + sizeof(double2)) > (size_t)dyn_smem) return;
    // every block of the persistent grid is resident from the start: the
    // chain's first kernel may be scheduled as blocks retire (it waits for
    // this grid's results before reading them)
    allow_dependent_launch();
    const int wl = threadIdx.x & 31;                 // lane in the warp
    const int w0 = threadIdx.x & ~31;                // the warp's first thread in the block

    for (;;) {
        unsigned long long tile = 0;
        if (wl == 0) tile = atomicAdd(a.tile_counter, 1ULL);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= (unsigned long long)a.n_tiles) return;

        // tile shape: bulk tiles first, then the tail's (more lanes per sample)
        const bool bulk = tile < (unsigned long long)a.n_bulk_tiles;
        const int lg = bulk ? a.lg_bulk : a.lg_tail;       // log2 of lanes per sample
        const int spw = 32 >> lg;                          // samples of the tile
        const int64_t base = bulk ? (int64_t)tile * spw
                                  : a.bulk_samples + (int64_t)(tile - a.n_bulk_tiles) * spw;
        const int slot = wl >> lg;
        const int lane = wl & ((1 << lg) - 1);
        const int64_t g = base + slot;
        Res* my = rec + (size_t)threadIdx.x * kSlots;
        const int si0 = g < a.total_samples ? find_index(a.sample_offsets, a.n_sims, g) : 0;
        if (g < a.total_samples && SPINSIM_INB(si0 >= 0 && si0 < a.n_sims, 0)) {
            const int si = si0;
            const int64_t k = g - a.sample_offsets[si];
            const DevSim& s = a.sims[si];
            // lanes in use: at most one per segment; each owns a canonical sub-tree
            const int lg_use = min(lg, (int)s.seg_log2);
            const int spl_log2 = s.seg_log2 - lg_use;
            if (SPINSIM_INB(k >= 0 && k < s.K, 1) && k > 0 && lane < (1 << lg_use)) {
                SampleCtx<R> c;
                double beta = 0.0;
                const double gsum = make_ctx<R, N, TONES, SU3>(s, k, c, beta);
                if (lane == 0) bg[w0 + slot] = make_double2(beta, gsum);
                const int64_t L = s.L;
#pragma unroll 1
                for (int q = 0; q < (1 << spl_log2); q++) {
                    const int sg = (lane << spl_log2) + q;
                    const int64_t lo = (sg * L) >> s.seg_log2, hi = ((sg + 1) * L) >> s.seg_log2;
                    Res X;
                    res_zero(X);
                    // the step index as R, counted (exact: L <= 2^24), not
                    // converted from the integer each step (a 64-bit integer
                    // conversion is an FP64-pipe instruction)
                    const int n_steps = (int)(hi - lo);
                    R lf = (R)lo;
                    if constexpr (SU3) {
                        CounterPhasors<R> ph;
                        counter_phasors_at<R, METHOD>(c, lo, ph);
#pragma unroll 1
                        for (int i = 0; i < n_steps; i++, lf += R(1)) step_apply_su3<R, METHOD, TONES>(c, lf, ph, X);
                    } else if constexpr (SMALL && N == 3) {
                        // small angles: the drive phasors turned per step from the segment's start
                        DrivePhasors<R> dp;
                        drive_phasors_at<R, METHOD>(c, lo, dp);
#pragma unroll 1
                        for (int i = 0; i < n_steps; i++, lf += R(1)) step_apply<R, METHOD, SMALL, TONES>(c, lf, c.tau, X, &dp);
                    } else {
#pragma unroll 1
                        for (int i = 0; i < n_steps; i++, lf += R(1)) step_apply<R, METHOD, SMALL, TONES>(c, lf, c.tau, X);   // U <- u_l U
                    }
                    // canonical tree over the lane's segments: a finished pair of
                    // equal sub-trees merges (later on the left) until the sizes differ
                    int h = 0;
#pragma unroll 1
                    while ((q >> h) & 1) {
                        Res t;
                        res_mul(X, my[h], t);
                        X = t;
                        h++;
                    }
                    my[h] = X;
                }
            }
        }
        __syncwarp();
        // epilogue, one lane per sample of the tile: the lanes' sub-trees
        // combined in the canonical tree, then the FP64 part (which reads the
        // drive phasor tables: their kernel has completed after this wait)
        grid_dependency_wait();
        if (wl < spw) {
            const int t = wl;
            const int64_t gs = base + t;
            const int si = gs < a.total_samples ? find_index(a.sample_offsets, a.n_sims, gs) : 0;
            if (gs < a.total_samples && SPINSIM_INB(si >= 0 && si < a.n_sims, 0) &&
                SPINSIM_INB(gs - a.sample_offsets[si] >= 0 && gs - a.sample_offsets[si] < a.sims[si].K, 1)) {
                const int64_t k = gs - a.sample_offsets[si];
                double* out = a.U + gs * OPD;
                if (k == 0) {
                    store_identity(N, out);
                } else {
                    const DevSim& s = a.sims[si];
                    const int lg_use = min(lg, (int)s.seg_log2);
                    const int spl_log2 = s.seg_log2 - lg_use;
                    Res* lanes = rec + (size_t)(w0 + (t << lg)) * kSlots;   // lane j's result: lanes[j * kSlots + spl_log2]
#pragma unroll 1
                    for (int d = 0; d < lg_use; d++)
#pragma unroll 1
                        for (int j = 0; j < (1 << lg_use); j += 2 << d) {
                            Res tmp;
                            res_mul(lanes[(j + (1 << d)) * kSlots + spl_log2], lanes[j * kSlots + spl_log2], tmp);
                            lanes[j * kSlots + spl_log2] = tmp;
                        }
                    const double2 b = bg[w0 + t];
                    SampleExact sx;
                    make_exact<N, TONES>(s, k, b.x, b.y, sx);
                    finish<TONES>(lanes[spl_log2], s, sx, out);
                }
            }
        }
        __syncwarp();
    }
}

// The paired body (FP32-bulk, the small-angle kernels):
// every slot of a tile is a pair of consecutive samples (k, k + 1) of one
// simulation, advanced together in F2 (lanes2.cuh: one packed f32x2
// instruction for both samples, each lane rounded as the scalar float
// operation, so neither sample's result depends on its partner).  Each
// simulation starts at an even index of the operator buffer (the host pads an
// odd sample count by one unused slot), so a pair never spans two
// simulations; the slot past an odd simulation's last sample is computed
// with its partner's context and not stored.  Tiles hold 2 x (32 >> lg)
// samples, G = 2^lg lanes per pair as in integrate_body; in the epilogue a
// lane finishes both samples of its pair in a tile of 32 pairs, one of them
// in a smaller tile (two lanes per pair).
template <int N, int METHOD, int SMALL>
__device__ __forceinline__ void integrate_pair_body(const IntegrateArgs& a)
{
    using Res = typename ResType<N, F2>::type;
    constexpr int OPD = N == 3 ? 18 : 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Res* rec = reinterpret_cast<Res*>(smem_raw);                                                 // [blockDim][kSlots]
    double2* bg = reinterpret_cast<double2*>(smem_raw + (size_t)blockDim.x * kSlots * sizeof(Res));  // [blockDim][2]
    unsigned dyn_smem;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
    if ((size_t)blockDim.x * (kSlots * sizeof(Res) + 2 * sizeof(double2)) > (size_t)dyn_smem) return;
    allow_dependent_launch();
    const int wl = threadIdx.x & 31;
    const int w0 = threadIdx.x & ~31;

    for (;;) {
        unsigned long long tile = 0;
        if (wl == 0) tile = atomicAdd(a.tile_counter, 1ULL);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= (unsigned long long)a.n_tiles) return;

        const bool bulk = tile < (unsigned long long)a.n_bulk_tiles;
        const int lg = bulk ? a.lg_bulk : a.lg_tail;       // log2 of lanes per pair
        const int spw = 32 >> lg;                          // pairs of the tile
        const int64_t base = bulk ? (int64_t)tile * 2 * spw
                                  : a.bulk_samples + (int64_t)(tile - a.n_bulk_tiles) * 2 * spw;
        const int slot = wl >> lg;
        const int lane = wl & ((1 << lg) - 1);
        const int64_t g = base + 2 * slot;                 // the pair's first sample
        Res* my = rec + (size_t)threadIdx.x * kSlots;
        const int si0 = g < a.total_samples ? find_index(a.sample_offsets, a.n_sims, g) : 0;
        if (g < a.total_samples && SPINSIM_INB(si0 >= 0 && si0 < a.n_sims, 0)) {
            const int si = si0;
            const int64_t k = g - a.sample_offsets[si];
            const DevSim& s = a.sims[si];
            const int lg_use = min(lg, (int)s.seg_log2);
            const int spl_log2 = s.seg_log2 - lg_use;
            if (SPINSIM_INB(k >= 0 && (k & 1) == 0, 1) && k < s.K && lane < (1 << lg_use)) {
                const int64_t k1 = k + 1 < s.K ? k + 1 : k;   // past the end: the partner's context again
                SampleCtx<float> c1[2];
                double beta0 = 0.0, beta1 = 0.0;
                const double gsum0 = make_ctx<float, N>(s, k, c1[0], beta0);
                const double gsum1 = make_ctx<float, N>(s, k1, c1[1], beta1);
                if (lane == 0) {
                    bg[2 * (w0 + slot)] = make_double2(beta0, gsum0);
                    bg[2 * (w0 + slot) + 1] = make_double2(beta1, gsum1);
                }
                SampleCtx<F2> c;
                pack(c1, c);
                const int64_t L = s.L;
#pragma unroll 1
                for (int q = 0; q < (1 << spl_log2); q++) {
                    const int sg = (lane << spl_log2) + q;
                    const int64_t lo = (sg * L) >> s.seg_log2, hi = ((sg + 1) * L) >> s.seg_log2;
                    Res X;
                    res_zero(X);
                    // the step index counted in FP32 (exact: L <= 2^24)
                    const int n_steps = (int)(hi - lo);
                    float lf = (float)lo;
                    if constexpr (N == 3) {
                        DrivePhasors<F2> dp;
                        drive_phasors_at<F2, METHOD>(c, lo, dp);
#pragma unroll 1
                        for (int i = 0; i < n_steps; i++, lf += 1.0f)
                            step_apply<F2, METHOD, SMALL, false>(c, F2(lf), c.tau, X, &dp);
                    } else {
#pragma unroll 1
                        for (int i = 0; i < n_steps; i++, lf += 1.0f) step_apply<F2, METHOD, SMALL, false>(c, F2(lf), c.tau, X);
                    }
                    int h = 0;
#pragma unroll 1
                    while ((q >> h) & 1) {
                        Res t;
                        res_mul(X, my[h], t);
                        X = t;
                        h++;
                    }
                    my[h] = X;
                }
            }
        }
        __syncwarp();
        grid_dependency_wait();
        // epilogue: the lanes' sub-trees of a pair combined in the canonical
        // tree (one lane per pair), then the FP64 part of both samples: in a
        // tile of 32 pairs each lane finishes both samples of its pair, in a
        // smaller tile two lanes share a pair, one sample each (an FP64 warp
        // instruction costs the same however few lanes are active)
        if (wl < spw && lg > 0) {
            const int64_t gp = base + 2 * wl;
            const int si = gp < a.total_samples ? find_index(a.sample_offsets, a.n_sims, gp) : 0;
            if (gp < a.total_samples && SPINSIM_INB(si >= 0 && si < a.n_sims, 0) &&
                SPINSIM_INB(gp - a.sample_offsets[si] >= 0, 1) && gp - a.sample_offsets[si] < a.sims[si].K) {
                const DevSim& s = a.sims[si];
                const int lg_use = min(lg, (int)s.seg_log2);
                const int spl_log2 = s.seg_log2 - lg_use;
                Res* lanes = rec + (size_t)(w0 + (wl << lg)) * kSlots;   // lane j's result: lanes[j * kSlots + spl_log2]
#pragma unroll 1
                for (int d = 0; d < lg_use; d++)
#pragma unroll 1
                    for (int j = 0; j < (1 << lg_use); j += 2 << d) {
                        Res tmp;
                        res_mul(lanes[(j + (1 << d)) * kSlots + spl_log2], lanes[j * kSlots + spl_log2], tmp);
                        lanes[j * kSlots + spl_log2] = tmp;
                    }
            }
        }
        __syncwarp();
        const int share = lg > 0 ? 1 : 0;                  // log2 of lanes per pair in the FP64 part
        if (wl < (spw << share)) {
            const int t = wl >> share;
            const int64_t gp = base + 2 * t;
            const int si = gp < a.total_samples ? find_index(a.sample_offsets, a.n_sims, gp) : 0;
            if (gp < a.total_samples && SPINSIM_INB(si >= 0 && si < a.n_sims, 0) &&
                SPINSIM_INB(gp - a.sample_offsets[si] >= 0, 1) && gp - a.sample_offsets[si] < a.sims[si].K) {
                const int64_t k = gp - a.sample_offsets[si];
                const DevSim& s = a.sims[si];
                const int lg_use = min(lg, (int)s.seg_log2);
                const int spl_log2 = s.seg_log2 - lg_use;
                const Res& pr = rec[(size_t)(w0 + (t << lg)) * kSlots + spl_log2];
#pragma unroll 1
                for (int h = share ? (wl & 1) : 0; h < 2; h += 1 + share) {
                    const int64_t kh = k + h;
                    if (kh >= s.K) break;                    // the unused slot of an odd simulation
                    double* out = a.U + (gp + h) * OPD;
                    if (kh == 0) {
                        store_identity(N, out);
                    } else {
                        typename ResType<N, float>::type r;
                        unpack(pr, h, r);
                        const double2 b = bg[2 * (w0 + t) + h];
                        SampleExact sx;
                        make_exact<N, false>(s, kh, b.x, b.y, sx);
                        finish<false>(r, s, sx, out);
                    }
                }
            }
        }
        __syncwarp();
    }
}

// The general and small-angle variants.
template <int N, typename R, int METHOD, int SMALL>
__global__ void __launch_bounds__(256) integrate_kernel(IntegrateArgs a)
{
    integrate_body<N, R, METHOD, SMALL, false>(a);
}

// The paired small-angle kernels (FP32-bulk).
template <int N, int METHOD, int SMALL>
__global__ void __launch_bounds__(256) integrate_pair_kernel(IntegrateArgs a)
{
    integrate_pair_body<N, METHOD, SMALL>(a);
}

// The variant with further drive tones; in FP32 held to 128 registers (two
// 256-thread blocks per SM): uncapped it takes 152 and three 128-thread blocks
// fit, and the fourth block's latency hiding is worth more than the few
// spilled registers (measured on the multi-tone sensing run: 0.616 -> 0.555
// ms).  The cap is on this kernel alone: given to the others, even as a
// minimum of one block, it changes their register allocation (126 -> 140) and
// costs 9%.
template <int N, typename R, int METHOD, int SMALL>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) integrate_tones_kernel(IntegrateArgs a)
{
    integrate_body<N, R, METHOD, SMALL, true>(a);
}

// Full su(3) spin-one Hamiltonians (quadrupole drives, tones included): FP64.
template <int METHOD>
__global__ void __launch_bounds__(256) integrate_su3_kernel(IntegrateArgs a)
{
    integrate_body<3, double, METHOD, false, true, true>(a);
}

// The phasor tables (drive and further tones) of a launch group, one thread
// per entry: the simulation that owns entry j is the last one whose first
// entry is at most j (simulations with no entries share their successor's
// offset).
__global__ void __launch_bounds__(256) phase_table_kernel(const DevSim* sims, int n_sims, int64_t n_entries,
                                                          double* tab)
{
    // the integrate kernel that follows may be scheduled at once (it waits
    // for this grid before its epilogue reads the tables)
    allow_dependent_launch();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_entries; j += stride) {
        int lo = 0, hi = n_sims - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sims[mid].eb_off <= j) lo = mid;
            else hi = mid - 1;
        }
        const DevSim& s = sims[lo];
        const int64_t e = j - s.eb_off;
        if (!SPINSIM_INB(e >= 0, 2) || e >= phasor_entries(s.K, s.n_tones)) continue;   // past the last entry (layout slack)
        const cx<double> v = sim_phasor_entry(s, e);
        tab[2 * j] = v.r;
        tab[2 * j + 1] = v.i;
    }
}

cudaError_t launch_phase_table(const DevSim* sims, int n_sims, int64_t n_entries, double* tab, int n_sm,
                               cudaStream_t stream)
{
    if (n_entries <= 0 || n_sims <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n_entries + 255) / 256, (int64_t)std::max(n_sm, 1) * 8);
    phase_table_kernel<<<(unsigned)blocks, 256, 0, stream>>>(sims, n_sims, n_entries, tab);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- launchers
template <int METHOD>
static void* su3_kernel_ptr()
{
    return (void*)integrate_su3_kernel<METHOD>;
}
template <int N, typename R, int METHOD, int SMALL, bool TONES>
static void* kernel_ptr()
{
    if constexpr (TONES) return (void*)integrate_tones_kernel<N, R, METHOD, SMALL>;
    else return (void*)integrate_kernel<N, R, METHOD, SMALL>;
}

template <int N, typename R, int SMALL, bool TONES>
static void* pick_method(int method)
{
    switch (method) {
        case 0: return kernel_ptr<N, R, 0, SMALL, TONES>();
        case 1: return kernel_ptr<N, R, 1, SMALL, TONES>();
        case 2: return kernel_ptr<N, R, 2, SMALL, TONES>();
        default: return nullptr;
    }
}

template <int N, int SMALL>
static void* pick_pair(int method)
{
    switch (method) {
        case 0: return (void*)integrate_pair_kernel<N, 0, SMALL>;
        case 1: return (void*)integrate_pair_kernel<N, 1, SMALL>;
        case 2: return (void*)integrate_pair_kernel<N, 2, SMALL>;
        default: return nullptr;
    }
}

template <int N, typename R>
static void* pick_variant(int method, int variant)
{
    switch (variant) {
        case kVariantGeneral: return pick_method<N, R, false, false>(method);
        case kVariantTones: return pick_method<N, R, false, true>(method);
        case kVariantSmallTones:
            if constexpr (sizeof(R) == 4) return pick_method<N, R, kSmallGauss, true>(method);
            else return nullptr;
        // the small-angle variants exist for FP32-bulk only (FP64 keeps the
        // general series, its terms sized for double precision) and run in the
        // paired kernel, two samples per thread (the tau = 0 variants exist for
        // spin-one only: spin-half has no squarings)
        case kVariantSmall:
            if constexpr (sizeof(R) == 4) return pick_pair<N, kSmallGauss>(method);
            else return nullptr;
        case kVariantSmallSine:
            if constexpr (sizeof(R) == 4) return pick_pair<N, kSmallSine>(method);
            else return nullptr;
        case kVariantSmallTau0:
            if constexpr (N == 3 && sizeof(R) == 4) return pick_pair<N, kSmallGauss | kSmallTau0>(method);
            else return nullptr;
        case kVariantSmallSineTau0:
            if constexpr (N == 3 && sizeof(R) == 4) return pick_pair<N, kSmallSine | kSmallTau0>(method);
            else return nullptr;
        case kVariantSU3:
            if constexpr (N == 3 && sizeof(R) == 8) {
                switch (method) {
                    case 0: return su3_kernel_ptr<0>();
                    case 1: return su3_kernel_ptr<1>();
                    case 2: return su3_kernel_ptr<2>();
                    default: return nullptr;
                }
            } else {
                return nullptr;
            }
        default: return nullptr;
    }
}

static void* select_kernel(int spin_x2, int precision, int method, int variant)
{
    if (spin_x2 == 2) return precision ? pick_variant<3, float>(method, variant) : pick_variant<3, double>(method, variant);
    if (spin_x2 == 1) return precision ? pick_variant<2, float>(method, variant) : pick_variant<2, double>(method, variant);
    return nullptr;
}

// Dynamic shared memory of one block: kSlots residual records and the
// sample's (beta, gsum) per thread, sized from the record type itself.
size_t integrate_smem_bytes(int spin_x2, int precision, int block, int variant)
{
    if (variant_pairs(spin_x2, precision, variant))
        return (size_t)block * (kSlots * (spin_x2 == 2 ? sizeof(Res3<F2>) : sizeof(Res2<F2>)) + 2 * sizeof(double2));
    size_t res;
    if (spin_x2 == 2) res = precision ? sizeof(Res3<float>) : sizeof(Res3<double>);
    else res = precision ? sizeof(Res2<float>) : sizeof(Res2<double>);
    return (size_t)block * (kSlots * res + 2 * sizeof(double));
}

// Must be called (outside stream capture) before the first launch of a
// (spin, precision, method, variant) kernel: it raises the kernel's dynamic
// shared-memory limit to what a 256-thread block needs.
cudaError_t integrate_occupancy(int spin_x2, int precision, int method, int block, int variant, int* blocks_per_sm)
{
    void* k = select_kernel(spin_x2, precision, method, variant);
    if (!k) return cudaErrorInvalidValue;
    size_t smem_max = integrate_smem_bytes(spin_x2, precision, 256, variant);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e != cudaSuccess) return e;
    size_t smem = integrate_smem_bytes(spin_x2, precision, block, variant);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, block, smem);
}

// Tiles of a launch (one warp each): whole waves of bulk tiles (lanes_bulk
// lanes per sample) while at least one full wave of them fits, then the
// remaining samples in tail tiles with as many lanes per sample as every
// simulation of the launch has segments (one segment per lane), which end the
// launch in finer steps.
void integrate_tiles(int64_t total, int lanes_bulk, int block, int64_t wave_blocks, int min_seg_log2,
                     IntegrateArgs& a, int per_slot)
{
    int lg = 0;
    while ((1 << lg) < lanes_bulk && lg < min_seg_log2) lg++;
    const int64_t wave_warps = wave_blocks * (block / 32);
    const int64_t spw_bulk = (int64_t)per_slot * (32 >> lg);   // samples of a bulk tile
    const int64_t rounds = total / (wave_warps * spw_bulk);
    a.lg_bulk = lg;
    a.lg_tail = min_seg_log2;
    a.n_bulk_tiles = rounds * wave_warps;
    a.bulk_samples = a.n_bulk_tiles * spw_bulk;
    const int64_t spw_tail = (int64_t)per_slot * (32 >> a.lg_tail);
    a.n_tiles = a.n_bulk_tiles + (total - a.bulk_samples + spw_tail - 1) / spw_tail;
}

cudaError_t launch_integrate(int spin_x2, int precision, int method, int block, int grid, int variant,
                             const IntegrateArgs& a, cudaStream_t stream, bool after_phase_table)
{
    void* k = select_kernel(spin_x2, precision, method, variant);
    if (!k || block % 32 != 0 || block < 32 || block > 256 || grid < 1 || a.lg_bulk < 0 || a.lg_bulk > kSegLog2 ||
        a.lg_tail < 0 || a.lg_tail > kSegLog2)
        return cudaErrorInvalidValue;
    size_t smem = integrate_smem_bytes(spin_x2, precision, block, variant);
    IntegrateArgs args = a;
    void* params[] = {&args};
    if (!after_phase_table) return cudaLaunchKernel(k, dim3(grid), dim3(block), params, smem, stream);
    // a programmatic dependent launch of the drive phasor tables' kernel: the
    // step loops start while the tables are filled; the epilogue, which reads
    // them, waits for that kernel first (griddepcontrol.wait)
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, k, params);
}

#ifdef SPINSIM_BOUNDS
SPINSIM_BOUNDS_READER(bounds_word_integrate)
#endif

}  // namespace spinsim
