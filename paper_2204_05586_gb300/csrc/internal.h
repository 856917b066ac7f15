// internal.h -- structures shared by the host engine and the kernels.
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace spinsim {

constexpr int kMaxPulses = 4;
constexpr int kSegments = 4;             // canonical split of one U_k's L steps (fixed tree)
constexpr int kRun = 8;                  // samples one lane chains sequentially
constexpr int kChunk = 32 * kRun;        // samples one warp chains (never spans simulations)
constexpr int kGroup = 32;               // chunks one warp scans (never spans simulations)

// Per-simulation parameters on the device, precomputed on the host in FP64.
struct DevSim {
    double* states;              // [K][N] complex, device
    double* spin;                // [K][3] or nullptr
    double* ops;                 // [K][N][N] complex or nullptr
    int64_t K, L;
    int64_t sample_offset;       // first sample of this simulation in the operator buffer
    int64_t chunk_offset;        // first chain chunk of this simulation
    int64_t group_offset;        // first chunk group of this simulation
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
    int32_t pad2;
    double exit_re, exit_im;     // e^{-i 2 pi B dt_out} (frame) or 1
    double exit_half_re, exit_half_im;  // e^{-i pi B dt_out} (frame) or 1
    double amp[kMaxPulses];      // 2 pi A_p, rad/s
    double centre[kMaxPulses];
    double inv_w[kMaxPulses];
    double psi0[6];
    int32_t n_pulses, frame, spin_x2, counter_on;
};

struct IntegrateArgs {
    const DevSim* sims;
    const int64_t* sample_offsets;   // n_sims + 1 prefix offsets (device)
    int n_sims;
    int64_t total_samples;
    double* U;                        // operator buffer: spin-one 18, spin-half 4 doubles per sample
    int tau;
    unsigned long long* tile_counter; // zeroed before the launch
    int64_t n_tiles;
};

struct ChainArgs {
    const DevSim* sims;
    const int64_t* chunk_offsets;     // n_sims + 1 prefix offsets (device)
    const int64_t* group_offsets;     // n_sims + 1 prefix offsets (device)
    int n_sims;
    int64_t n_chunks, n_groups;
    const double* U;
    double* run_prefix;               // [n_chunks][32] exclusive prefixes of the lanes' runs
    double* chunk_agg;                // [n_chunks] chunk products
    double* chunk_gprefix;            // [n_chunks] exclusive prefixes of the chunk products in their group
    double* group_agg;                // [n_groups] group products
    double* group_start;              // [n_groups][N] complex states entering each group
};

// Doubles per stored operator in the operator buffer and chain scratch.
inline int op_doubles(int spin_x2) { return spin_x2 == 2 ? 18 : 4; }

inline int64_t n_chunks_of(int64_t K) { return (K + kChunk - 1) / kChunk; }
inline int64_t n_groups_of(int64_t K) { return (n_chunks_of(K) + kGroup - 1) / kGroup; }
inline size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Layout of the chain scratch (offsets from its start, 256-byte aligned).
struct ChainLayout {
    size_t prefix, agg, gprefix, gagg, gstart, bytes;
};
inline ChainLayout chain_layout(int spin_x2, int64_t chunks, int64_t groups)
{
    const size_t opb = (size_t)op_doubles(spin_x2) * sizeof(double);
    ChainLayout c;
    size_t off = 0;
    c.prefix = off; off += round256((size_t)chunks * 32 * opb);
    c.agg = off; off += round256((size_t)chunks * opb);
    c.gprefix = off; off += round256((size_t)chunks * opb);
    c.gagg = off; off += round256((size_t)groups * opb);
    c.gstart = off; off += round256((size_t)groups * 2 * (spin_x2 + 1) * sizeof(double));
    c.bytes = off;
    return c;
}

// Lie-Trotter squarings for a request (Sec. 1.2.3).  An explicit tau (>= 0)
// is used as given; -1 selects 24 for FP64 (the paper's default) and, for
// FP32-bulk, the smallest tau whose leapfrog error bound theta^2 / (3 4^tau)
// (relative to the step angle theta) is below 6e-9, ten times under FP32
// rounding -- the paper's criterion (fewest squarings at the smallest
// error) applied to FP32 arithmetic.  theta bounds |H| delta_t in the frame.
inline int choose_tau(int cfg_tau, int precision, int rotating_frame, double dt, double om_plus, double om_minus,
                      double bias_w, double pulse_w, double q_w)
{
    if (cfg_tau >= 0) return cfg_tau;
    if (precision == 0) return 24;
    const double z = rotating_frame ? pulse_w : bias_w + pulse_w;
    const double theta = dt * (om_plus + om_minus + z + q_w);
    int tau = 0;
    double bound = theta * theta / 3.0;
    while (bound > 6e-9 && tau < 24) {
        bound *= 0.25;
        tau++;
    }
    return tau;
}

// Host-side launchers (integrate.cu, chain.cu).  precision: 0 FP64, 1 FP32-bulk.
cudaError_t launch_integrate(int spin_x2, int precision, int method, int lanes, int block, int grid,
                             const IntegrateArgs& a, cudaStream_t stream);
size_t integrate_smem_bytes(int spin_x2, int precision, int lanes, int block);
cudaError_t integrate_occupancy(int spin_x2, int precision, int method, int lanes, int block, int* blocks_per_sm);
cudaError_t launch_chain(int spin_x2, const ChainArgs& a, int n_sm, cudaStream_t stream);

}  // namespace spinsim
