// internal.h -- structures shared by the host engine and the kernels.
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "spinsim.h"

namespace spinsim {

constexpr int kMaxPulses = 4;
// A Gaussian pulse in base-2 units: exp(-u^2 / 2) = 2^(-(u k)^2), k = sqrt(log2(e) / 2).
constexpr double kGaussBase2 = 0.84932180028801904272150283410289;
constexpr int kMaxTones = SPINSIM_MAX_TONES;
// A sample's L steps are split into 2^seg_log2 canonical segments (at most
// kSegments) reduced by a fixed binary tree; the split depends on L alone.
constexpr int kSegLog2 = 3;
constexpr int kSegments = 1 << kSegLog2;
// Segments of a sample of L steps: one for L < 4, then 2, 4, 8 from L = 4, 16,
// 128, so that the tree's 2^s - 1 extra products stay a small fraction of the
// 2 L step products (CF4) while long samples can be shared by up to 8 lanes
// (measured on GB300 at L = 100: 4 segments beat 8 for one long simulation
// and for a batch alike).
inline int seg_log2_of(int64_t L) { return L >= 128 ? 3 : (L >= 16 ? 2 : (L >= 4 ? 1 : 0)); }

// ------------------------------------------------------- chain-tree geometry
// The ordered product psi_k = U_k ... U_0 psi_init is a tree scan per
// simulation (chain.cu).  Level 0 nodes cover kFan runs of `run` consecutive
// samples (one lane multiplies one run in order); a node of level l >= 1
// covers kFan consecutive nodes of level l - 1; the top level has one node.
constexpr int kFan = 32;                 // children of a node: one per lane of a warp
constexpr int kMaxLevels = 12;           // 256 x 32^11 samples exceed any valid K
constexpr int kLeftPerNode = kFan - 1;   // stored left-child products of a node's binary tree
// The run length depends on K alone, so a simulation's result does not depend
// on the batch it is in: at least 4 samples per lane (6 from 16384 samples:
// fewer tree products per sample where a batch of long simulations fills the
// GPU, while short requests keep their latency), more once a simulation has
// more level-0 nodes than a 152-SM GPU has SM sub-partitions (608), at most 8.
constexpr int64_t kRunSpread = 32 * 608;
constexpr int64_t kLongRunK = 16384;
inline int chain_run(int64_t K)
{
    const int64_t r = (K + kRunSpread - 1) / kRunSpread;
    const int64_t lo = K >= kLongRunK ? 6 : 4;
    return (int)(r < lo ? lo : (r > 8 ? 8 : r));
}

struct ChainGeom {
    int run, top;                        // samples per lane run; level of the single top node
    int64_t nodes[kMaxLevels];           // nodes per level (0 above the top)
};

inline ChainGeom chain_geom(int64_t K)
{
    ChainGeom g{};
    g.run = chain_run(K);
    g.top = 0;
    int64_t n = K > 0 ? (K + (int64_t)kFan * g.run - 1) / ((int64_t)kFan * g.run) : 0;
    g.nodes[0] = n;
    while (n > 1 && g.top + 1 < kMaxLevels) {
        n = (n + kFan - 1) / kFan;
        g.top++;
        g.nodes[g.top] = n;
    }
    return g;
}

// Drive phasor tables (GPU path): the FP64 drive phasor of interval k,
// e^{i beta_k} with beta_k the drive phase at t_{k-1}, is the product of two
// table entries, hi[(k - 1) >> kPhaseLoLog2] (the phasor at every kPhaseLo-th
// interval) and lo[(k - 1) & (kPhaseLo - 1)] (the turn over the remaining
// intervals), instead of a sine and cosine per sample.  One table of a
// simulation: the kPhaseLo turns, then the hi phasors (phase_entries(K)
// entries); a simulation with further tones has one such table per tone after
// the drive's (phasor_entries(K, n_tones) entries in all).
constexpr int kPhaseLoLog2 = 7;
constexpr int kPhaseLo = 1 << kPhaseLoLog2;
__host__ __device__ inline int64_t phase_entries(int64_t K) { return K >= 2 ? kPhaseLo + ((K - 2) >> kPhaseLoLog2) + 1 : 0; }
__host__ __device__ inline int64_t phasor_entries(int64_t K, int n_tones) { return phase_entries(K) * (1 + n_tones); }

// Per-simulation parameters on the device, precomputed on the host in FP64.
struct DevSim {
    double* states;              // [K][N] complex, device
    double* spin;                // [K][3] or nullptr
    double* ops;                 // [K][N][N] complex or nullptr
    int64_t K, L;
    int64_t sample_offset;       // first sample of this simulation in the operator buffer
    // phasor tables of this simulation's drive and further tones, (re, im)
    // pairs in FP64 (nullptr: a sine and cosine of each phase per sample instead)
    const double* eb_tab;
    int64_t eb_off;              // first entry of this simulation in its launch group's table
    int32_t chain_run;           // samples per lane run at the bottom of the chain tree
    int32_t chain_top;           // level of the chain tree's top node
    int32_t seg_log2;            // the sample's L steps in 2^seg_log2 canonical segments
    int32_t seg_pad;
    double t_start, dt_out, dt;  // dt = dt_out / L
    double drive_hz, drive_phase;
    double w_co0, w_counter0;    // frame: 2 pi (f_d - B), 2 pi (f_d + B); lab: 2 pi f_d, 2 pi f_d
    // Step exponents are built directly from these products of amplitude,
    // quadrature weight and delta_t (radians), so no FP32-rounded amplitude
    // or weight enters every step with the same rounding error:
    //   P[0] = Om+ a dt, P[1] = Om+ b dt, P[2] = Om- a dt, P[3] = Om- b dt,
    // Om+- = (2 pi drive_x_hz +- 2 pi drive_y_hz)/2, (a, b) the method's
    // node weights (CF4: Eqs. cf4_sample_1/2; the second CF4 exponential
    // uses (b, a)).
    double P[4];
    double za, zb;               // a dt, b dt for the z field
    double zbias;                // lab frame: 2 pi B (a + b) dt; frame: 0
    double c1, c2;               // node offsets in units of dt
    double qd3;                  // (a + b) w_q dt / 3 / 2^tau (one exponential), in the bulk type
    double om_plus, om_minus;    // Om+, Om- (rad/s)
    double W1, W2;               // total quadrature weight of nodes 1 and 2 over one step
    double gq;                   // exact first-order Q coefficient of one sample: w_q dt_out
    // Node-phasor sums S(th) = sum_{l<L, n=1,2} W_n e^{i th x}, x = l + c_n, of the
    // co-rotating (th0 = (w_co0) dt) and counter-rotating (th0 = (w_counter0) dt)
    // drive terms as Taylor coefficients T_m = sum W_n x^m e^{i th0 x}, m = 0..3,
    // re/im interleaved; a sample shifts th0 by -+ gsum dt (pulse part of w_r).
    double tay_co[8], tay_ct[8];
    int32_t tay_ok;              // 1 when the tables were built (L <= 65536)
    int32_t normalize_out;       // FP32-bulk: write psi_k renormalised in FP64
    int32_t tau;                 // Lie-Trotter squarings of this simulation (n = 2^tau)
    int32_t n_gauss;             // pulses [0, n_gauss) are Gaussians, [n_gauss, n_pulses) sine cycles
    double exit_re, exit_im;     // e^{-i 2 pi B dt_out} (frame) or 1
    double exit_half_re, exit_half_im;  // e^{-i pi B dt_out} (frame) or 1
    double amp[kMaxPulses];      // 2 pi A_p, rad/s
    double centre[kMaxPulses];   // Gaussian centre, or start of the sine cycle
    double inv_w[kMaxPulses];    // 1 / (standard deviation or period)
    double psi0[6];
    int32_t n_pulses, frame, spin_x2, counter_on;
    // Further drive tones j < n_tones, each handled like the drive: Om+-_j,
    // the in-frame rates (frame: 2 pi (f_j -+ B); lab: 2 pi f_j) and the
    // Taylor tables of their node-phasor sums (same layout as tay_co/tay_ct).
    int32_t n_tones, tone_pad;
    double tone_hz[kMaxTones], tone_phase[kMaxTones];
    double t_om_plus[kMaxTones], t_om_minus[kMaxTones];
    double t_co0[kMaxTones], t_ct0[kMaxTones];
    double t_tay_co[kMaxTones][8], t_tay_ct[kMaxTones][8];
    // The same constants rounded to FP32 once, on the host, for the FP32-bulk kernels.
    float f_ph[4];
    float f_za, f_zb, f_zbias, f_qd3, f_dt, f_c1, f_c2, f_pad;
    float f_amp[kMaxPulses], f_invw[kMaxPulses];
    float f_invwb[kMaxPulses];   // inv_w sqrt(log2(e) / 2): the Gaussian in base-2 units
    float f_tom_plus[kMaxTones], f_tom_minus[kMaxTones];
    // Quadrupole drives (full su(3), FP64 only): pair p on (D_xz, D_yz) (k = 1)
    // or (D_x2y2, D_xy) (k = 2), Om+-_p and the rates seen in the frame,
    // 2 pi (f_p -+ k B) (lab: 2 pi f_p).
    int32_t qd_on, qd_pad;
    double qd_hz[2], qd_phase[2];
    double qd_om_plus[2], qd_om_minus[2], qd_co0[2], qd_ct0[2];
};

struct IntegrateArgs {
    const DevSim* sims;
    const int64_t* sample_offsets;   // n_sims + 1 prefix offsets (device)
    int n_sims;
    int64_t total_samples;
    double* U;                        // operator buffer: spin-one 18, spin-half 4 doubles per sample
    int tau;
    unsigned long long* tile_counter; // zeroed before the launch
    int64_t n_tiles;                  // bulk tiles, then tail tiles
    int64_t n_bulk_tiles, bulk_samples;
    int lg_bulk, lg_tail;             // log2 of lanes per sample in bulk / tail tiles
};

// What launch_chain runs: the whole scan, only the up-sweep (the products:
// a range whose entering state is not known yet), or only the down-sweep and
// the write from each simulation's psi0 (that range once its entering state
// has been placed in psi0).
enum ChainMode { kChainFull = 0, kChainUp = 1, kChainDown = 2 };

struct ChainArgs {
    const DevSim* sims;
    int n_sims;
    int levels;                       // 1 + the highest top level of the batch
    int mode;                         // ChainMode
    const int64_t* level_off;         // [levels][n_sims + 1] first node of each simulation per level (device)
    int64_t nodes[kMaxLevels];        // nodes per level, all simulations
    const double* U;                  // sample operators
    double* agg[kMaxLevels];          // [nodes] product of the node's samples
    double* left[kMaxLevels];         // [nodes][kLeftPerNode] left-child products of the node's binary tree
    double* state[kMaxLevels];        // [nodes][N] complex state entering the node (written for the
                                      // children of top nodes by the up-sweep)
    int max_run;                      // the longest lane run of the simulations (chain_run): sizes the
                                      // apply kernel's output staging (0: the longest possible)
};

// Doubles per stored operator in the operator buffer and chain scratch.
inline int op_doubles(int spin_x2) { return spin_x2 == 2 ? 18 : 4; }

inline size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Layout of the chain scratch of a batch (offsets from its start, 256-byte aligned).
struct ChainLayout {
    int levels;
    int64_t nodes[kMaxLevels];
    size_t agg[kMaxLevels], left[kMaxLevels], state[kMaxLevels], bytes;
};

inline ChainLayout chain_layout(int spin_x2, const int64_t* nodes, int levels)
{
    const size_t opb = (size_t)op_doubles(spin_x2) * sizeof(double);
    const size_t stb = (size_t)2 * (spin_x2 + 1) * sizeof(double);
    ChainLayout c{};
    c.levels = levels;
    size_t off = 0;
    for (int l = 0; l < levels; l++) {
        c.nodes[l] = nodes[l];
        c.agg[l] = off; off += round256((size_t)nodes[l] * opb);
        c.left[l] = off; off += round256((size_t)nodes[l] * kLeftPerNode * opb);
        c.state[l] = off; off += round256((size_t)nodes[l] * stb);
    }
    c.bytes = off;
    return c;
}

// Point the per-level arrays of `a` into chain scratch laid out by `cl` at `base`.
inline void chain_args_set(ChainArgs& a, const ChainLayout& cl, char* base)
{
    a.levels = cl.levels;
    a.mode = kChainFull;
    for (int l = 0; l < kMaxLevels; l++) {
        const bool used = l < cl.levels;
        a.nodes[l] = used ? cl.nodes[l] : 0;
        a.agg[l] = used ? reinterpret_cast<double*>(base + cl.agg[l]) : nullptr;
        a.left[l] = used ? reinterpret_cast<double*>(base + cl.left[l]) : nullptr;
        a.state[l] = used ? reinterpret_cast<double*>(base + cl.state[l]) : nullptr;
    }
}



// ------------------------------------------------- request warning bits
constexpr double kMagnusXi = 1.0868687;   // Sec. 1.2.2: convergence radius of the Magnus series

// Bounds of |w_perp| and |w_z| over the request (rad/s).
inline void field_bounds(const spinsim_field& f, double& wperp, double& wz)
{
    const double two_pi = 6.283185307179586476925286766559;
    double pulses = 0.0;
    for (int p = 0; p < f.n_pulses; p++) pulses += std::fabs(f.pulse_amp_hz[p]);
    wperp = two_pi * (std::fabs(f.drive_x_hz) + std::fabs(f.drive_y_hz));
    for (int j = 0; j < f.n_tones && j < SPINSIM_MAX_TONES; j++)
        wperp += two_pi * (std::fabs(f.tone_x_hz[j]) + std::fabs(f.tone_y_hz[j]));
    if (f.qd_on)   // the quadrupole drives' operators have norm 1, as J_x and J_y
        for (int p = 0; p < 2; p++) wperp += two_pi * (std::fabs(f.qd_x_hz[p]) + std::fabs(f.qd_y_hz[p]));
    wz = two_pi * (std::fabs(f.bias_hz) + pulses);
}

// SPINSIM_WARN_MAGNUS: an upper bound of ||H||_2 delta_t against the Magnus
// radius.  ||w.J||_2 = |w| j, ||Q||_2 = 2/3.
inline int magnus_flags(const spinsim_request& r, int64_t L)
{
    double wperp, wz;
    field_bounds(r.field, wperp, wz);
    const double j = r.spin_x2 == 2 ? 1.0 : 0.5;
    const double hnorm = std::sqrt(wperp * wperp + wz * wz) * j +
                         (r.spin_x2 == 2 ? 6.283185307179586476925286766559 * std::fabs(r.field.quad_hz) * 2.0 / 3.0
                                         : 0.0);
    return hnorm * (r.dt_out / (double)L) >= kMagnusXi ? SPINSIM_WARN_MAGNUS : 0;
}

// SPINSIM_WARN_FP32_LAB: FP32-bulk carries every sample operator as the
// identity plus an FP32 residual.  In the lab frame a z field turns each
// sample by w_z dt_out (radians for MHz fields), so the residual is not small
// and its rounding, the same in every sample of a constant bias, adds up
// coherently over the run; the rotating frame removes that rotation.
inline int precision_flags(int precision, int rotating_frame, const spinsim_request& r)
{
    double wperp, wz;
    field_bounds(r.field, wperp, wz);
    return precision == SPINSIM_PREC_FP32_BULK && !rotating_frame && wz > 0.0 ? SPINSIM_WARN_FP32_LAB : 0;
}

// Lie-Trotter squarings for a request (Sec. 1.2.3).  An explicit tau (>= 0)
// is used as given; -1 selects 24 for FP64 (the paper's default) and, for
// FP32-bulk, the fewest squarings whose splitting error, summed over every
// exponential of the run, stays below kTrotterBudget.
//
// The bound: T = e^{A/2} e^{B} e^{A/2} with A = -i D, D = v_z J_z + v_q Q, and
// B = -i Phi J_phi is exp(A + B + E3 + O(5th order)) with
// E3 = [B,[B,A]]/12 - [A,[A,B]]/24 (symmetric splitting), so T^n with
// n = 2^tau (each factor built from v/n) is exp(A + B + E3 / 4^tau).  For a
// Hermitian X, |[X, Y]| <= spread(X) |Y - c I| for any c, which gives
// |E3| <= Phi^2 sigma / 6 + sigma^2 Phi / 24 with sigma = spread(D)
// <= 2 |v_z| + |v_q| and spread(Phi J_phi) = 2 Phi.  Each exponential then
// departs from exp(A + B) by at most |E3| / 4^tau, and unitary propagation
// adds these departures at most linearly over the run.
//
// The exponent bounds: |v_perp| <= (|wa| + |wb|) dt (|Om+| + |Om-|); in the
// rotating frame |v_z| <= (|wa| + |wb|) dt sum_p |amp_p| (the pulse part
// minus its midpoint value), in the lab frame plus |wa + wb| dt |w_bias|;
// |v_q| = |wa + wb| dt |w_q|.
constexpr double kTrotterBudget = 1e-6;   // a tenth of the FP32-bulk state accuracy (1e-5)

inline int choose_tau(int cfg_tau, int precision, int rotating_frame, int n_exp, double wa, double wb, double dt,
                      double om_perp, double bias_w, double pulse_w, double q_w, double steps)
{
    if (cfg_tau >= 0) return cfg_tau;
    if (precision == 0) return 24;
    const double wabs = std::fabs(wa) + std::fabs(wb), wsum = std::fabs(wa + wb);
    const double phi = wabs * dt * om_perp;
    const double vz = wabs * dt * pulse_w + (rotating_frame ? 0.0 : wsum * dt * bias_w);
    const double vq = wsum * dt * q_w;
    const double sigma = 2.0 * vz + vq;
    double err = steps * (double)n_exp * (phi * phi * sigma / 6.0 + sigma * sigma * phi / 24.0);
    int tau = 0;
    while (err > kTrotterBudget && tau < 24) {
        err *= 0.25;
        tau++;
    }
    return tau;
}

// Largest step angle for which the FP32 kernels may use the two-term
// small-angle series (device_math.cuh).
constexpr double kTinyAngleBound = 0.015625;

// Host-side parameter set-up (params.cu).
// fill_devsim: the kernels' record of one validated request (K output
// samples, L steps per sample); the caller sets the output pointers and the
// sample/chunk/group offsets.
void fill_devsim(const spinsim_config& cfg, const spinsim_request& r, int64_t K, int64_t L, DevSim& d);
// small_angle_request: true when the request runs in FP32-bulk, has no
// further tone, and every argument of the per-step sine/cosine series is
// bounded by kTinyAngleBound (Gaussian and single-sine-cycle pulses alike).
bool small_angle_request(const spinsim_config& cfg, const spinsim_request& r, int64_t L);

// Integrate kernel variants: the general one; the small-angle one (FP32-bulk,
// Gaussian pulses, no further tones; small_angle_request) and its twin that
// also evaluates single-sine-cycle pulses (the paper's benchmark field; its
// own kernel so that the Gaussian-only step loop does not carry that code);
// the one that also evaluates further drive tones (requests with tones only,
// so the others keep the leaner step loop); and the full su(3) one
// (quadrupole drives, spin-one, FP64, tones included).  A batch runs one
// launch group per (spin, variant), each request in the variant it needs on
// its own.
// The small-angle variants of spin-one requests whose Lie-Trotter squarings
// come out as tau = 0 (the usual case in the rotating frame) have kernels of
// their own, with the closed-form exponential and no runtime tau branch in the
// step loop.  Requests with further tones inside the small-angle bounds (and
// Gaussian pulses only) run the tones kernel with the small-angle series.
enum IntegrateVariant {
    kVariantGeneral = 0,
    kVariantSmall = 1,
    kVariantTones = 2,
    kVariantSU3 = 3,
    kVariantSmallSine = 4,
    kVariantSmallTau0 = 5,
    kVariantSmallSineTau0 = 6,
    kVariantSmallTones = 7
};
constexpr int kVariants = 8;
constexpr int kMaxGroups = 2 * kVariants;   // launch groups of one batch: spin-half and spin-one
// The kernels' SMALL template argument: 0 general series; bit 0 the
// small-angle series with Gaussian pulses, bit 1 with single sine cycles as
// well (1 or 2); bit 2 (added to either) tau = 0 known at compile time.
constexpr int kSmallGauss = 1, kSmallSine = 2, kSmallTau0 = 4;
// The paired kernels (integrate_pair_kernel: two consecutive samples per
// thread in packed f32x2 arithmetic) run the small-angle requests in
// FP32-bulk.  Their launch groups place every simulation at an even index of
// the operator buffer: K samples take pair_slots(K) slots.
inline bool variant_pairs(int spin_x2, int precision, int variant)
{
    (void)spin_x2;
    return precision == SPINSIM_PREC_FP32_BULK &&
           (variant == kVariantSmall || variant == kVariantSmallSine || variant == kVariantSmallTau0 ||
            variant == kVariantSmallSineTau0);
}
inline int64_t pair_slots(int64_t K) { return K + (K & 1); }
// request_variant: the variant a validated request of K samples and L steps
// per sample needs (kVariantSU3: its quadrupole drives; FP64 only, see
// precision_status).
int request_variant(const spinsim_config& cfg, const spinsim_request& r, int64_t K, int64_t L);
// precision_status: SPINSIM_E_UNSUPPORTED for a request the configured
// precision cannot run (quadrupole drives in FP32-bulk), else SPINSIM_OK.
int precision_status(const spinsim_config& cfg, const spinsim_request& r);

// Request validation (params.cu), shared by every entry point: status,
// SPINSIM_WARN_MAGNUS, K and L of one request.
struct Checked {
    int status = SPINSIM_OK;
    int flags = 0;
    int64_t K = 0, L = 0;
    int variant = kVariantGeneral;   // request_variant under the handle's configuration
};
Checked check_request(const spinsim_request* r);

// Host-side launchers (integrate.cu, chain.cu).  precision: 0 FP64, 1 FP32-bulk;
// variant: an IntegrateVariant (kVariantSmall for FP32-bulk only).
// launch_integrate: `a` must carry the tile plan of integrate_tiles;
// `after_phase_table`: the drive phasor tables' kernel is the stream's last
// launch (the integrate kernel then overlaps it, see launch_integrate).
cudaError_t launch_integrate(int spin_x2, int precision, int method, int block, int grid, int variant,
                             const IntegrateArgs& a, cudaStream_t stream, bool after_phase_table = false);
size_t integrate_smem_bytes(int spin_x2, int precision, int block, int variant);
cudaError_t integrate_occupancy(int spin_x2, int precision, int method, int block, int variant, int* blocks_per_sm);
// launch_phase_table: fill the drive phasor tables of `n_sims` simulations
// (their eb_off ascending; `n_entries` in all) at tab, on `stream`.
cudaError_t launch_phase_table(const DevSim* sims, int n_sims, int64_t n_entries, double* tab, int n_sm,
                               cudaStream_t stream);
// integrate_tiles: the tile plan of `total` samples for bulk lanes per sample
// `lanes_bulk` (1, 2, 4 or 8, at most 2^min_seg_log2), `block` threads and
// `wave_blocks` resident blocks; the tail uses 2^min_seg_log2 lanes per sample,
// min_seg_log2 the smallest segment split among the launch's simulations;
// `per_slot` samples per lane group (2 for the paired kernels).
void integrate_tiles(int64_t total, int lanes_bulk, int block, int64_t wave_blocks, int min_seg_log2,
                     IntegrateArgs& a, int per_slot = 1);
// launch_chain: the chain kernels of a batch in order on `stream`; *kernels
// receives how many were launched; fp32: the products and the state
// propagation in single precision (the precision-study control), else FP64.
cudaError_t launch_chain(int spin_x2, const ChainArgs& a, int n_sm, cudaStream_t stream, int* kernels,
                         bool fp32 = false);

// The debug build's device error words (bounds.cuh), one per translation
// unit with kernels: read, and cleared when `clear`; ~0 when unreadable.
#ifdef SPINSIM_BOUNDS
uint64_t bounds_word_integrate(bool clear);
uint64_t bounds_word_chain(bool clear);
uint64_t bounds_word_static(bool clear);
#endif

}  // namespace spinsim
