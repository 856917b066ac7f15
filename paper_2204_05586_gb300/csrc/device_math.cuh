// device_math.cuh -- per-thread arithmetic of the integrator (registers only).
//
// Everything is templated on the bulk arithmetic type R (float for the
// FP32-bulk path, double for the FP64 path).  Operators close to the identity
// are carried as residuals X = U - I throughout (Sec. 1.2.3), so that rounding
// acts on the small part only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <cstring>

#include "internal.h"

#if defined(__CUDACC__)
// Device functions, also compiled for the host by nvcc (the CPU test harness).
#ifndef SPINSIM_HD
#define SPINSIM_HD __host__ __device__ __forceinline__
#endif
// Rarely taken or once-per-sample paths (libm sin/cos with their range
// reduction) are kept out of line, so the step loop stays small and its
// register allocation is not sized for them.
#ifndef SPINSIM_COLD
#define SPINSIM_COLD __host__ __device__ __noinline__
#endif
#else
// A host C++ compiler (the multicore CPU backend): plain inline functions and
// the C++ library's maths under the names the device code uses.
#include <cmath>
#define SPINSIM_HD inline
#define SPINSIM_COLD __attribute__((noinline))
namespace spinsim {
using std::cos;
using std::exp;
using std::exp2;
using std::fabs;
using std::floor;
using std::fma;
using std::ldexp;
using std::rint;
using std::sin;
using std::sqrt;
inline void sincos(float x, float* s, float* c) { *s = std::sin(x); *c = std::cos(x); }
inline void sincos(double x, double* s, double* c) { *s = std::sin(x); *c = std::cos(x); }
inline float rsqrt(float x) { return 1.0f / std::sqrt(x); }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
}  // namespace spinsim
#endif

namespace spinsim {

#if defined(__CUDACC__)
// Programmatic dependent launch (sm_90 and later): a kernel launched with the
// programmatic-serialization attribute may start before its predecessor has
// finished; grid_dependency_wait() blocks until the predecessor grid has
// completed and its memory is visible (it returns at once for a normal
// launch), and allow_dependent_launch() lets the successor be scheduled.
__device__ __forceinline__ void grid_dependency_wait()
{
#if defined(__CUDA_ARCH__)
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void allow_dependent_launch()
{
#if defined(__CUDA_ARCH__)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
#endif

// The bulk type's precision class: FP32 (float, or a host vector of floats
// that carries several samples at once, which specialises this) or FP64.
template <typename R>
struct BulkTraits {
    static constexpr bool fp32 = sizeof(R) == 4;
    static constexpr int lanes = 1;   // samples carried by one value
};
template <typename R>
constexpr bool kFP32 = BulkTraits<R>::fp32;

SPINSIM_HD int clz32(uint32_t x)
{
#if defined(__CUDA_ARCH__)
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

// Exact widening of an FP32 value to FP64 from the fields of the two IEEE 754
// binary formats, returning the FP64 bit pattern: the sign kept, the exponent
// rebiased (+1023 - 127), the 23 mantissa bits moved to the top of the 52; a
// subnormal input (m x 2^-149) normalised; zero, the infinities and NaN
// (payload kept) mapped to theirs.
SPINSIM_HD uint64_t widen_bits(uint32_t b)
{
    const uint32_t e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    uint32_t E, M;
    if (e == 0u) {
        const int sh = m ? clz32(m) - 8 : 0;   // moves the leading 1 to the implicit bit
        E = m ? 897u - (uint32_t)sh : 0u;
        M = (m << sh) & 0x7fffffu;
    } else {
        E = e == 0xffu ? 0x7ffu : e + 896u;
        M = m;
    }
    return ((uint64_t)((b & 0x80000000u) | (E << 20) | (M >> 3)) << 32) | (uint64_t)(M << 29);
}

// FP32 -> FP64 in the spin-half sample epilogue.  On the device by
// widen_bits (integer instructions): the conversion instruction runs on the
// FP64 pipe, where one warp instruction holds a sub-partition's unit as long
// as an FP64 multiply-add does.  (Measured on GB300: 1 % faster for the
// spin-half kernels; the spin-one epilogue, with 19 conversions per sample,
// ran slower with it and converts directly.)  On the host the plain
// conversion (the same value).
SPINSIM_HD double widen(float f)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)widen_bits(__float_as_uint(f)));
#else
    return (double)f;
#endif
}
SPINSIM_HD double widen(double d) { return d; }

template <typename R>
struct cx {
    R r, i;
};

template <typename R>
SPINSIM_HD cx<R> cmk(R r, R i) { cx<R> c; c.r = r; c.i = i; return c; }
template <typename R>
SPINSIM_HD cx<R> cadd(cx<R> a, cx<R> b) { return cmk(a.r + b.r, a.i + b.i); }
template <typename R>
SPINSIM_HD cx<R> csub(cx<R> a, cx<R> b) { return cmk(a.r - b.r, a.i - b.i); }
template <typename R>
SPINSIM_HD cx<R> cscale(cx<R> a, R s) { return cmk(a.r * s, a.i * s); }
template <typename R>
SPINSIM_HD cx<R> cconj(cx<R> a) { return cmk(a.r, -a.i); }
template <typename R>
SPINSIM_HD cx<R> cmul(cx<R> a, cx<R> b)
{
    return cmk(fma(a.r, b.r, -a.i * b.i), fma(a.r, b.i, a.i * b.r));
}
// c + a b
template <typename R>
SPINSIM_HD cx<R> cfma(cx<R> a, cx<R> b, cx<R> c)
{
    return cmk(fma(a.r, b.r, fma(-a.i, b.i, c.r)), fma(a.r, b.i, fma(a.i, b.r, c.i)));
}
// c + conj(a) b
template <typename R>
SPINSIM_HD cx<R> cfma_conj(cx<R> a, cx<R> b, cx<R> c)
{
    return cmk(fma(a.r, b.r, fma(a.i, b.i, c.r)), fma(a.r, b.i, fma(-a.i, b.r, c.i)));
}

constexpr double kTwoPi = 6.283185307179586476925287;
constexpr double kInvSqrt2 = 0.7071067811865475244008444;
constexpr double kSqrt2 = 1.414213562373095048801689;

// sin and cos of a small angle by their Taylor series (x - x^3/3! + ...,
// 1 - x^2/2! + ...); for |x| <= 1/16 the terms kept leave a relative
// truncation error below 1e-19 in double and below 2e-11 in float (fewer
// terms); larger angles use the libdevice call.
template <typename R>
struct SinCos {
    R s, c;
};

template <typename R>
SPINSIM_COLD SinCos<R> sincos_cold(R x)
{
    SinCos<R> r;
    sincos(x, &r.s, &r.c);
    return r;
}

// (sin x - x, cos x - 1) for |x| > 1/16: cos x - 1 = -2 sin^2(x/2).
template <typename R>
SPINSIM_COLD SinCos<R> sincos_m_cold(R x)
{
    R s, c;
    sincos(x, &s, &c);
    const R h = sin(R(0.5) * x);
    SinCos<R> r;
    r.s = s - x;
    r.c = R(-2) * h * h;
    return r;
}

template <typename R>
SPINSIM_HD void small_sincos(R x, R& s, R& c)
{
    if (fabs(x) <= R(0.0625)) {
        R x2 = x * x;
        if constexpr (kFP32<R>) {
            s = x * (R(1) - x2 * (R(1.0 / 6) - x2 * R(1.0 / 120)));
            c = R(1) - x2 * (R(0.5) - x2 * (R(1.0 / 24) - x2 * R(1.0 / 720)));
        } else {
            s = x * (R(1) - x2 * (R(1.0 / 6) - x2 * (R(1.0 / 120) - x2 * (R(1.0 / 5040) - x2 * R(1.0 / 362880)))));
            c = R(1) - x2 * (R(0.5) - x2 * (R(1.0 / 24) - x2 * (R(1.0 / 720) - x2 * (R(1.0 / 40320) - x2 * R(1.0 / 3628800)))));
        }
    } else {
        const SinCos<R> r = sincos_cold(x);
        s = r.s;
        c = r.c;
    }
}

// sin(x) - x and cos(x) - 1 without cancellation: Taylor series for
// |x| <= 1/16 (relative truncation below 1e-19 in double, 5e-8 in float),
// else from sincos with cos(x) - 1 = -2 sin^2(x/2).
template <typename R>
SPINSIM_HD void small_sincos_m(R x, R& sm, R& cm)
{
    if (fabs(x) <= R(0.0625)) {
        R x2 = x * x;
        if constexpr (kFP32<R>) {
            sm = -x * x2 * (R(1.0 / 6) - x2 * R(1.0 / 120));
            cm = -x2 * (R(0.5) - x2 * (R(1.0 / 24) - x2 * R(1.0 / 720)));
        } else {
            sm = -x * x2 * (R(1.0 / 6) - x2 * (R(1.0 / 120) - x2 * (R(1.0 / 5040) - x2 * R(1.0 / 362880))));
            cm = -x2 * (R(0.5) - x2 * (R(1.0 / 24) - x2 * (R(1.0 / 720) - x2 * (R(1.0 / 40320) - x2 * R(1.0 / 3628800)))));
        }
    } else {
        const SinCos<R> r = sincos_m_cold(x);
        sm = r.s;
        cm = r.c;
    }
}

// The branch-free series of small_sincos and small_sincos_m alone (|x| <= 1/16),
// the same expressions, for a host type that carries several samples and
// takes the series only when every sample's angle is small (the tests check
// that both give the same bits).
template <typename R>
SPINSIM_HD void sincos_series(R x, R& s, R& c)
{
    R x2 = x * x;
    if constexpr (kFP32<R>) {
        s = x * (R(1) - x2 * (R(1.0 / 6) - x2 * R(1.0 / 120)));
        c = R(1) - x2 * (R(0.5) - x2 * (R(1.0 / 24) - x2 * R(1.0 / 720)));
    } else {
        s = x * (R(1) - x2 * (R(1.0 / 6) - x2 * (R(1.0 / 120) - x2 * (R(1.0 / 5040) - x2 * R(1.0 / 362880)))));
        c = R(1) - x2 * (R(0.5) - x2 * (R(1.0 / 24) - x2 * (R(1.0 / 720) - x2 * (R(1.0 / 40320) - x2 * R(1.0 / 3628800)))));
    }
}

template <typename R>
SPINSIM_HD void sincos_m_series(R x, R& sm, R& cm)
{
    R x2 = x * x;
    if constexpr (kFP32<R>) {
        sm = -x * x2 * (R(1.0 / 6) - x2 * R(1.0 / 120));
        cm = -x2 * (R(0.5) - x2 * (R(1.0 / 24) - x2 * R(1.0 / 720)));
    } else {
        sm = -x * x2 * (R(1.0 / 6) - x2 * (R(1.0 / 120) - x2 * (R(1.0 / 5040) - x2 * R(1.0 / 362880))));
        cm = -x2 * (R(0.5) - x2 * (R(1.0 / 24) - x2 * (R(1.0 / 720) - x2 * (R(1.0 / 40320) - x2 * R(1.0 / 3628800)))));
    }
}

// Small-angle forms of the two series above, for arguments the host has
// bounded by |x| <= kTinyAngleBound = 2^-6 (every step angle of a
// rotating-frame FP32 run, see small_angle_request):
// two terms leave a relative truncation error of at most x^4/120 (sin),
// x^6/720 (cos), x^4/840 (sin x - x) and x^4/360 (cos x - 1), all below
// 2e-9, so no branch and no libm fallback is needed.
template <typename R>
SPINSIM_HD void small_sincos_tiny(R x, R& s, R& c)
{
    const R x2 = x * x;
    s = fma(x * x2, R(-1.0 / 6), x);
    c = fma(x2, fma(x2, R(1.0 / 24), R(-0.5)), R(1));
}

template <typename R>
SPINSIM_HD void small_sincos_m_tiny(R x, R& sm, R& cm)
{
    const R x2 = x * x;
    sm = x * x2 * fma(x2, R(1.0 / 120), R(-1.0 / 6));
    cm = x2 * fma(x2, R(1.0 / 24), R(-0.5));
}

template <typename R, int SMALL>
SPINSIM_HD void step_sincos(R x, R& s, R& c)
{
    if constexpr (SMALL) small_sincos_tiny(x, s, c);
    else small_sincos(x, s, c);
}

template <typename R, int SMALL>
SPINSIM_HD void step_sincos_m(R x, R& sm, R& cm)
{
    if constexpr (SMALL) small_sincos_m_tiny(x, sm, cm);
    else small_sincos_m(x, sm, cm);
}

// -------------------------------------------------------------------------
// Per-sample context: the field family inside interval k, reduced to values
// in the bulk type R.  Large phases (the drive phase at t_{k-1}, the pulse
// offsets) are reduced in FP64 once per sample.
//
// FP32 design rule: over 10^7 steps the accumulated rotation angles reach
// hundreds of radians, so any rounding error that is identical in every step
// (a constant rounded once, a fixed factor such as 1/3 or 1/sqrt2, a biased
// approximation) adds up coherently and dominates.  Therefore the first-order
// parts of every sample operator are replaced by their exact FP64 values at
// the end of the sample (transverse: the quadrature sum of the drive; Q: w_q
// dt_out, correcting the one constant q/3 that cannot be carried exactly, see
// expm_one_res), e^{i beta} comes from FP64, square roots and quotients are
// the correctly rounded ones, and what FP32 rounds is second order or varying
// data, unbiased, growing only like a random walk.  (The transverse drive
// amplitudes enter the step exponents rounded to FP32 once: their rounding
// reaches only second order, measured: the sweep's error moved from 9.5e-8 to
// 1.1e-7 against carrying them as (hi, lo) pairs.)
// -------------------------------------------------------------------------
template <typename R>
struct SampleCtx {
    R ebr, ebi;                     // e^{i beta}, beta = drive phase at t_{k-1}
    R co, counter;                  // drive frequencies seen in the frame: w_d - w_r, w_d + w_r
    R Ph[4];                        // P[0..3] in the bulk type
    R za, zb, zbias;
    R qd3;
    R inv_n;                        // 2^-tau
    R q1;                           // first-order Q coefficient of one exponential: 3 qd3 2^tau
    // per-simulation constants of the small-angle exponential at tau = 0
    // (expm_one_res_tau0): the m = 0 diagonal's rest d1 and phasor p1 of
    // e^{i 2 qd3} (th_1 = 2 qd3), and e^{-i qd3} = e^{i (th_0 + th_2) / 2}
    R d1r, d1i, p1r, p1i, eqr, eqi;
    R dt, c1, c2;
    R amp[kMaxPulses], u0[kMaxPulses], invw[kMaxPulses], ghat[kMaxPulses];
    R u0b[kMaxPulses], invwb[kMaxPulses];   // u0, invw in base-2 Gaussian units (small-angle variant)
    // further tones (the tones variant only): e^{i beta_j}, in-frame rates, Om+-_j
    R tbr[kMaxTones], tbi[kMaxTones], tco[kMaxTones], tct[kMaxTones], tomp[kMaxTones], tomm[kMaxTones];
    // quadrupole drives (the su(3) variant only): the same per pair
    R qbr[2], qbi[2], qco[2], qct[2], qomp[2], qomm[2];
    int nt;
    int np;
    int ng;                         // pulses [0, ng) Gaussian, [ng, np) single sine cycles
    int tau;
    bool counter_on;
};

// Fill the context of interval k (1 <= k < K) and the FP64 phasor
// e^{-i w_r dt_out} used to leave the frame (Eq. exit_rotating_frame); for
// spin-half the phasor is e^{-i w_r dt_out / 2}.
//
// With the frame on, w_r = 2 pi B + sum_p amp_p ghat_p where ghat_p is the
// pulse shape at the interval midpoint rounded to R; the frame is an exact
// change of variables for any constant w_r, and this one is exactly the value
// the in-frame field subtracts, so leaving the frame undoes entering it.
struct SampleExact {
    double ph_re, ph_im;   // e^{-i w_r dt_out} (spin-one) or e^{-i w_r dt_out / 2} (spin-half)
    double eb_re, eb_im;   // e^{i beta}
    double dco, dct;       // w_d - w_r, w_d + w_r (rad/s)
    double gsum;           // pulse part of w_r (rad/s)
    double tb_re[kMaxTones], tb_im[kMaxTones];   // e^{i beta_j} of the further tones (tones variant)
};

// Phase 2 pi frac(f t) + phase of a tone of frequency f at t, in [-pi, pi]
// (FP64, a few ops).
SPINSIM_HD double tone_phase_at(double hz, double phase, double t)
{
    double cyc = hz * t;
    cyc -= floor(cyc);
    double beta = kTwoPi * cyc + phase;
    return beta - kTwoPi * rint(beta * (1.0 / kTwoPi));
}

// Drive phase beta at t_{k-1}.
SPINSIM_HD double drive_phase_at(const DevSim& s, int64_t k)
{
    return tone_phase_at(s.drive_hz, s.drive_phase, s.t_start + (double)(k - 1) * s.dt_out);
}

// The fractional part of f (t0 + m dt) in cycles, to a few 1e-16: with
// f dt = a + b and m a = p + q split exactly by FMA (Dekker's product), and
// f t0 = c + d likewise, the fractional parts of the large terms p and c are
// taken exactly and only the sum of two numbers below 1 and the small terms
// is rounded.  Unlike tone_phase_at, the rounding does not grow with f t.
SPINSIM_HD double drive_cycles_frac(double f, double t0, double dt, int64_t m)
{
    const double a = f * dt, b = fma(f, dt, -a);
    const double md = (double)m;   // exact for |m| < 2^53
    const double p = md * a, q = fma(md, a, -p);
    const double c = f * t0, d = fma(f, t0, -c);
    double x = (p - floor(p)) + (c - floor(c));
    x += fma(md, b, q + d);
    return x - floor(x);
}

// Entry e of one phasor table (see kPhaseLo) of a tone of frequency hz and
// phase `phase` (the drive or a further tone): the turn e^{i 2 pi hz dt_out e}
// for e < kPhaseLo, else the tone's phasor e^{i beta} at interval
// k - 1 = (e - kPhaseLo) kPhaseLo.
SPINSIM_HD cx<double> phasor_entry(double hz, double phase, const DevSim& s, int64_t e)
{
    const bool turn = e < kPhaseLo;
    const double cyc = turn ? drive_cycles_frac(hz, 0.0, s.dt_out, e)
                            : drive_cycles_frac(hz, s.t_start, s.dt_out, (e - kPhaseLo) << kPhaseLoLog2);
    double b = kTwoPi * cyc + (turn ? 0.0 : phase);
    b -= kTwoPi * rint(b * (1.0 / kTwoPi));
    const SinCos<double> sc = sincos_cold(b);
    return cmk(sc.c, sc.s);
}

SPINSIM_HD cx<double> drive_phasor_entry(const DevSim& s, int64_t e)
{
    return phasor_entry(s.drive_hz, s.drive_phase, s, e);
}

// Entry e of all of a simulation's tables (phasor_entries(K, n_tones) in
// all): table e / phase_entries(K), the drive's first, then further tone j's.
SPINSIM_HD cx<double> sim_phasor_entry(const DevSim& s, int64_t e)
{
    const int64_t n = phase_entries(s.K);
    const int t = (int)(e / n);
    const int64_t r = e - (int64_t)t * n;
    return t == 0 ? drive_phasor_entry(s, r) : phasor_entry(s.tone_hz[t - 1], s.tone_phase[t - 1], s, r);
}

// A tone's phasor at interval k >= 1 from its table (two roundings).
SPINSIM_HD cx<double> phasor_tab(const double* tab, int64_t k)
{
    const int64_t m = k - 1;
    const double* lo = tab + 2 * (m & (kPhaseLo - 1));
    const double* hi = tab + 2 * (kPhaseLo + (m >> kPhaseLoLog2));
    return cmul(cmk(hi[0], hi[1]), cmk(lo[0], lo[1]));
}

// e^{i beta_k} of interval k >= 1 from the tables: the epilogue's FP64 drive
// phasor.  (The bulk keeps its FP32 sine and cosine of the drive phase:
// reading the table at the start of every tile measured slower in the
// issue-bound step loop.)
SPINSIM_HD cx<double> drive_phasor_tab(const DevSim& s, int64_t k)
{
    return phasor_tab(s.eb_tab, k);
}

// e^{i beta_j,k} of further tone j at interval k >= 1 from its table.
SPINSIM_HD cx<double> tone_phasor_tab(const DevSim& s, int j, int64_t k)
{
    return phasor_tab(s.eb_tab + 2 * (int64_t)(j + 1) * phase_entries(s.K), k);
}

// Shape of z pulse p at u = (t - c_p) / w_p: a Gaussian exp(-u^2/2) (w_p the
// standard deviation), or a single sine cycle sin(2 pi u) for 0 <= u < 1 and 0
// elsewhere (w_p the period; the paper's sinp pulse, Eq. neural_pulse).
template <typename R>
SPINSIM_HD R pulse_shape(bool sine, R u)
{
    if (!sine) return exp(R(-0.5) * u * u);
    if (!(u >= R(0) && u < R(1))) return R(0);
#ifdef __CUDA_ARCH__
    return sinpi(R(2) * u);
#else
    return sin(R(kTwoPi) * u);
#endif
}

// The sine-cycle shape inline (the small-angle variant with sine cycles).
template <typename R>
SPINSIM_HD R sine_cycle(R u)
{
    return pulse_shape<R>(true, u);
}

// The sine-cycle shape out of line: only requests with such pulses reach it,
// and the step loop of the others does not carry its code.
template <typename R>
SPINSIM_COLD R sine_cycle_cold(R u)
{
    return pulse_shape<R>(true, u);
}

// The per-simulation constants of expm_one_res_tau0 from c.qd3: the same
// expressions expm_one_res_n evaluates for h_1 = qd3 with the small-angle
// series, and e^{-i qd3}.
template <typename R>
SPINSIM_HD void tau0_constants(SampleCtx<R>& c)
{
    R sm1, cm1, sq, cq;
    small_sincos_m_tiny(c.qd3, sm1, cm1);
    const R s1 = c.qd3 + sm1, c1 = R(1) + cm1;
    c.d1r = R(-2) * s1 * s1;
    c.d1i = R(2) * fma(c.qd3, cm1, sm1 * c1);
    c.p1r = R(1) + c.d1r;
    c.p1i = R(2) * s1 * c1;
    small_sincos_tiny(c.qd3, sq, cq);
    c.eqr = cq;
    c.eqi = -sq;
}

// Bulk context of interval k (every lane).  e^{i beta} comes from the bulk
// type's sincos: the first-order part it feeds is replaced by the exact FP64
// value at the end of the sample, so it only reaches second-order terms.
// Returns gsum = sum_p amp_p ghat_p (exact products of R values, in FP64)
// and the drive phase beta (FP64) for the epilogue.  The per-simulation
// constants come rounded to FP32 from the host for the FP32 path.
template <typename R, int N, bool TONES = false, bool SU3 = false>
SPINSIM_HD double make_ctx(const DevSim& s, int64_t k, SampleCtx<R>& c, double& beta)
{
    const double t_prev = s.t_start + (double)(k - 1) * s.dt_out;
    beta = drive_phase_at(s, k);
    const SinCos<R> eb = sincos_cold((R)beta);
    c.ebr = eb.c;
    c.ebi = eb.s;
    if constexpr (kFP32<R>) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            c.Ph[i] = s.f_ph[i];
        }
        c.za = s.f_za;
        c.zb = s.f_zb;
        c.zbias = s.f_zbias;
        c.qd3 = s.f_qd3;
        c.dt = s.f_dt;
        c.c1 = s.f_c1;
        c.c2 = s.f_c2;
    } else {
#pragma unroll
        for (int i = 0; i < 4; i++) c.Ph[i] = (R)s.P[i];
        c.za = (R)s.za;
        c.zb = (R)s.zb;
        c.zbias = (R)s.zbias;
        c.qd3 = (R)s.qd3;
        c.dt = (R)s.dt;
        c.c1 = (R)s.c1;
        c.c2 = (R)s.c2;
    }
    c.np = s.n_pulses;
    c.ng = s.n_gauss;
    c.tau = s.tau;
    c.inv_n = ldexp(R(1), -s.tau);
    c.q1 = R(3) * ldexp(c.qd3, s.tau);
    tau0_constants(c);
    c.counter_on = s.counter_on != 0;
    double gsum = 0.0;
#pragma unroll
    for (int p = 0; p < kMaxPulses; p++) {
        c.amp[p] = R(0); c.u0[p] = R(0); c.invw[p] = R(0); c.ghat[p] = R(0);
        c.u0b[p] = R(0); c.invwb[p] = R(0);
        if (p < c.np) {
            if constexpr (kFP32<R>) {
                c.amp[p] = s.f_amp[p];
                c.invw[p] = s.f_invw[p];
                c.invwb[p] = s.f_invwb[p];
            } else {
                c.amp[p] = (R)s.amp[p];
                c.invw[p] = (R)s.inv_w[p];
                c.invwb[p] = (R)(s.inv_w[p] * kGaussBase2);
            }
            c.u0[p] = (R)((t_prev - s.centre[p]) * s.inv_w[p]);
            c.u0b[p] = (R)((t_prev - s.centre[p]) * s.inv_w[p] * kGaussBase2);
            if (s.frame) {
                R um = (R)((t_prev + 0.5 * s.dt_out - s.centre[p]) * s.inv_w[p]);
                R g = pulse_shape<R>(p >= s.n_gauss, um);
                c.ghat[p] = g;
                gsum = fma((double)c.amp[p], (double)g, gsum);
            }
        }
    }
    c.co = (R)(s.frame ? s.w_co0 - gsum : s.w_co0);
    c.counter = (R)(s.frame ? s.w_counter0 + gsum : s.w_counter0);
    if constexpr (TONES) {
        c.nt = s.n_tones;
#pragma unroll
        for (int j = 0; j < kMaxTones; j++) {
            c.tbr[j] = c.tbi[j] = c.tco[j] = c.tct[j] = c.tomp[j] = c.tomm[j] = R(0);
            if (j < c.nt) {
                const SinCos<R> e = sincos_cold((R)tone_phase_at(s.tone_hz[j], s.tone_phase[j], t_prev));
                c.tbr[j] = e.c;
                c.tbi[j] = e.s;
                c.tco[j] = (R)(s.frame ? s.t_co0[j] - gsum : s.t_co0[j]);
                c.tct[j] = (R)(s.frame ? s.t_ct0[j] + gsum : s.t_ct0[j]);
                if constexpr (kFP32<R>) {
                    c.tomp[j] = s.f_tom_plus[j];
                    c.tomm[j] = s.f_tom_minus[j];
                } else {
                    c.tomp[j] = (R)s.t_om_plus[j];
                    c.tomm[j] = (R)s.t_om_minus[j];
                }
            }
        }
    }
    if constexpr (SU3) {
        // pair p turns at (p + 1) w_r in the frame, pulse part included
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const SinCos<R> e = sincos_cold((R)tone_phase_at(s.qd_hz[p], s.qd_phase[p], t_prev));
            const double kg = s.frame ? (double)(p + 1) * gsum : 0.0;
            c.qbr[p] = e.c;
            c.qbi[p] = e.s;
            c.qco[p] = (R)(s.qd_co0[p] - kg);
            c.qct[p] = (R)(s.qd_ct0[p] + kg);
            c.qomp[p] = (R)s.qd_om_plus[p];
            c.qomm[p] = (R)s.qd_om_minus[p];
        }
    }
    return gsum;
}

// FP64 quantities of interval k used once per sample by the epilogue, from
// the drive phase beta (or the drive phasor tables, when the simulation has
// them) and gsum that make_ctx returned: e^{i beta}, the frame
// frequencies and the exit phasor
// e^{-i w_r dt_out} (x 1/2 for spin-half).
//
// With the frame on, w_r = 2 pi B + gsum where gsum = sum_p amp_p ghat_p uses
// the pulse shapes at the interval midpoint rounded to R: the frame is an
// exact change of variables for any constant w_r, and this one is exactly
// the value the in-frame field subtracts, so leaving the frame undoes
// entering it.
template <int N, bool TONES = false>
SPINSIM_HD void make_exact(const DevSim& s, int64_t k, double beta, double gsum, SampleExact& x)
{
    if (s.eb_tab) {
        const cx<double> eb = drive_phasor_tab(s, k);
        x.eb_re = eb.r;
        x.eb_im = eb.i;
    } else {
        const SinCos<double> eb = sincos_cold(beta);
        x.eb_re = eb.c;
        x.eb_im = eb.s;
    }
    x.gsum = gsum;
    if constexpr (TONES) {
        const double t_prev = s.t_start + (double)(k - 1) * s.dt_out;
        for (int j = 0; j < s.n_tones; j++) {
            if (s.eb_tab) {
                const cx<double> e = tone_phasor_tab(s, j, k);
                x.tb_re[j] = e.r;
                x.tb_im[j] = e.i;
            } else {
                const SinCos<double> e = sincos_cold(tone_phase_at(s.tone_hz[j], s.tone_phase[j], t_prev));
                x.tb_re[j] = e.c;
                x.tb_im[j] = e.s;
            }
        }
    } else {
        (void)k;
    }
    if (s.frame) {
        x.dco = s.w_co0 - gsum;
        x.dct = s.w_counter0 + gsum;
        const double br = N == 2 ? s.exit_half_re : s.exit_re;
        const double bi = N == 2 ? s.exit_half_im : s.exit_im;
        if (gsum == 0.0) {
            // no pulse reaches this interval's midpoint (the usual case away
            // from the pulses): the exit phasor is the bias's alone
            x.ph_re = br;
            x.ph_im = bi;
        } else {
            double d = gsum * s.dt_out * (N == 2 ? 0.5 : 1.0);
            double sd, cd;
            small_sincos<double>(d, sd, cd);
            x.ph_re = br * cd + bi * sd;       // (br + i bi)(cd - i sd)
            x.ph_im = bi * cd - br * sd;
        }
    } else {
        x.dco = s.w_co0;
        x.dct = s.w_counter0;
        x.ph_re = 1.0;
        x.ph_im = 0.0;
    }
}

// sum_{l=0}^{L-1} (W1 e^{i th (l + c1)} + W2 e^{i th (l + c2)})
//   = (W1 e^{i th (c1 + (L-1)/2)} + W2 e^{i th (c2 + (L-1)/2)}) sin(L th/2) / sin(th/2),
// in FP64; th/2 is reduced by multiples of pi first so the ratio stays
// well conditioned near th = 2 pi m.
SPINSIM_HD cx<double> node_phasor_sum(double th, int64_t L, double W1, double c1, double W2, double c2)
{
    const double x = 0.5 * th;
    const double m = rint(x * (1.0 / 3.14159265358979323846));
    const double eps = fma(-m, 3.14159265358979323846, fma(-m, 1.2246467991473532e-16, x));
    double ratio;
    if (eps == 0.0) {
        ratio = (double)L;
    } else {
        double sL, cL, s1, c1_;
        small_sincos<double>((double)L * eps, sL, cL);
        small_sincos<double>(eps, s1, c1_);
        ratio = sL / s1;
    }
    // (-1)^(m (L - 1)) from sin(L x) / sin(x) with x = m pi + eps
    const long long ml = (long long)m;
    if ((ml & 1) && ((L - 1) & 1)) ratio = -ratio;
    const double mid = 0.5 * (double)(L - 1);
    double sa, ca, sb, cb;
    small_sincos<double>(th * (c1 + mid), sa, ca);
    small_sincos<double>(th * (c2 + mid), sb, cb);
    return cmk((W1 * ca + W2 * cb) * ratio, (W1 * sa + W2 * sb) * ratio);
}

// S(th0 + d) from the Taylor table T_m (m = 0..3):
//   sum W_n e^{i (th0 + d) x} = T_0 + i d T_1 - d^2/2 T_2 - i d^3/6 T_3 + O((d x)^4).
SPINSIM_HD cx<double> taylor_sum(const double* T, double d)
{
    if (d == 0.0) return cmk(T[0], T[1]);
    const double h2 = -0.5 * d * d, h3 = -d * d * d * (1.0 / 6.0);
    // T0 + i d T1 + h2 T2 + i h3 T3
    return cmk(T[0] - d * T[3] + h2 * T[4] - h3 * T[7], T[1] + d * T[2] + h2 * T[5] + h3 * T[6]);
}

// Exact first-order transverse coefficients of U^r_k: the method's quadrature
// sum over the sample of the in-frame drive,
//   g_x + i g_y = dt [Om+ e^{i beta} S(w_d - w_r) + Om- conj(e^{i beta} S(w_d + w_r))],
// S(w) = sum over steps and nodes of weight x e^{i w dt x_node}.  The frame's
// pulse part shifts th0 by a tiny d = gsum dt; while |d| (L + 1) <= 1e-3 the
// cubic Taylor series of the tables is exact to rounding, otherwise the
// closed form is used.
// Further tones add their own terms of the same form (tones variant).
template <bool TONES = false>
SPINSIM_HD void first_order_exact(const DevSim& s, const SampleExact& x, double& gx, double& gy)
{
    const cx<double> eb = cmk(x.eb_re, x.eb_im);
    const double d = s.frame ? x.gsum * s.dt : 0.0;
    const bool tay = s.tay_ok && fabs(d) * (double)(s.L + 1) <= 1e-3;
    cx<double> sco = tay ? taylor_sum(s.tay_co, -d) : node_phasor_sum(x.dco * s.dt, s.L, s.W1, s.c1, s.W2, s.c2);
    cx<double> g = cscale(cmul(eb, sco), s.om_plus);
    if (s.om_minus != 0.0) {
        cx<double> sct = tay ? taylor_sum(s.tay_ct, d) : node_phasor_sum(x.dct * s.dt, s.L, s.W1, s.c1, s.W2, s.c2);
        g = cadd(g, cscale(cconj(cmul(eb, sct)), s.om_minus));
    }
    if constexpr (TONES) {
        const double gf = s.frame ? x.gsum : 0.0;   // pulse part of w_r
        for (int j = 0; j < s.n_tones; j++) {
            const cx<double> ebj = cmk(x.tb_re[j], x.tb_im[j]);
            const cx<double> tco = tay ? taylor_sum(s.t_tay_co[j], -d)
                                       : node_phasor_sum((s.t_co0[j] - gf) * s.dt, s.L, s.W1, s.c1, s.W2, s.c2);
            g = cadd(g, cscale(cmul(ebj, tco), s.t_om_plus[j]));
            if (s.t_om_minus[j] != 0.0) {
                const cx<double> tct = tay ? taylor_sum(s.t_tay_ct[j], d)
                                           : node_phasor_sum((s.t_ct0[j] + gf) * s.dt, s.L, s.W1, s.c1, s.W2,
                                                             s.c2);
                g = cadd(g, cscale(cconj(cmul(ebj, tct)), s.t_om_minus[j]));
            }
        }
    }
    gx = g.r * s.dt;
    gy = g.i * s.dt;
}

// Field at offset tau from t_{k-1}, in the frame (Sec. 1.2.5): the phasors of
// the co- and counter-rotating drive terms and the pulse part of w_z'.
// With a = w_r tau and the drive phase A = beta + w_d tau, the rotation
//   w_x' = w_x cos a + w_y sin a,  w_y' = -w_x sin a + w_y cos a
// of w_x = Ax cos A, w_y = Ay sin A is, by product-to-sum identities,
//   w_x' + i w_y' = Om+ e^{i (beta + (w_d - w_r) tau)} + Om- e^{-i (beta + (w_d + w_r) tau)}
// with Om+- = (Ax +- Ay)/2.  The co-rotating phasor is e^{i beta} times a
// small rotation, so the slowly varying term never goes through a large
// angle.
// Further tones (tones variant) add their whole in-frame field
//   sum_j Om+_j e^{i (beta_j + (w_j - w_r) tau)} + Om-_j e^{-i (beta_j + (w_j + w_r) tau)}
// (rad/s) as `ex`.
template <typename R>
struct NodeField {
    cx<R> co, ct;   // e^{i (beta + (w_d - w_r) tau)}, e^{i (beta + (w_d + w_r) tau)}
    R z;            // w_z' without the lab-frame bias
    cx<R> ex;       // further tones' w_x' + i w_y' (tones variant)
    cx<R> qd[2];    // quadrupole drive pairs' u_a' + i u_b' (su(3) variant)
};

// sin and cos of an angle of any size in the bulk type, for terms whose
// first-order part is replaced exactly at the end of the sample (FP32: the
// fast hardware sincos on an argument reduced to [-pi, pi]).
template <typename R>
SPINSIM_HD void second_order_sincos(R x, R& s, R& c)
{
    if constexpr (kFP32<R>) {
        x = fma(R(-kTwoPi), rintf(x * R(1.0 / kTwoPi)), x);
#ifdef __CUDA_ARCH__
        __sincosf(x, &s, &c);
#else
        s = sinf(x);
        c = cosf(x);
#endif
    } else {
        sincos(x, &s, &c);
    }
}

// The counter-rotating phasors of the su(3) variant at both nodes of a step,
// e^{i beta} e^{i w_ct tau} (drive) and e^{i beta_p} e^{i w_ct,p tau}
// (quadrupole pairs), tau = (l + c_j) dt.  They are set from sin/cos at the
// first step of a canonical segment and then turned by e^{i w dt} per step, so
// the result depends on the step index alone (not on the launch shape); the
// rounding of the turns grows as (steps into the segment) x 2^-53 relative,
// on terms of size Omega dt.
template <typename R>
struct CounterPhasors {
    cx<R> d[2], q[2][2];   // [node], [pair][node]
    cx<R> rd, rq[2];       // turns per step
};

template <typename R, int METHOD>
SPINSIM_HD void counter_phasors_at(const SampleCtx<R>& c, int64_t lo, CounterPhasors<R>& p)
{
    R s, co;
#pragma unroll
    for (int j = 0; j < 2; j++) {
        if (METHOD == 1 && j == 1) break;   // one node
        const R tau = ((R)lo + (j ? c.c2 : c.c1)) * c.dt;
        if (c.counter_on) {
            second_order_sincos(c.counter * tau, s, co);
            p.d[j] = cmk(c.ebr * co - c.ebi * s, fma(c.ebr, s, c.ebi * co));
        } else {
            p.d[j] = cmk(R(0), R(0));
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            second_order_sincos(c.qct[q] * tau, s, co);
            p.q[q][j] = cmk(c.qbr[q] * co - c.qbi[q] * s, fma(c.qbr[q], s, c.qbi[q] * co));
        }
    }
    second_order_sincos(c.counter * c.dt, s, co);
    p.rd = cmk(co, s);
#pragma unroll
    for (int q = 0; q < 2; q++) {
        second_order_sincos(c.qct[q] * c.dt, s, co);
        p.rq[q] = cmk(co, s);
    }
}

template <typename R, int METHOD>
SPINSIM_HD void counter_phasors_advance(CounterPhasors<R>& p)
{
#pragma unroll
    for (int j = 0; j < 2; j++) {
        if (METHOD == 1 && j == 1) break;
        p.d[j] = cmul(p.d[j], p.rd);
#pragma unroll
        for (int q = 0; q < 2; q++) p.q[q][j] = cmul(p.q[q][j], p.rq[q]);
    }
}

// The drive's in-frame phasors at both nodes of a step in the small-angle
// variant: co-rotating e^{i beta} e^{i (w_d - w_r) tau} and counter-rotating
// e^{i beta} e^{i (w_d + w_r) tau}, tau = (l + c_j) dt.  They are set from the
// series (co-rotating) and the hardware sincos (counter-rotating) at the first
// step of each canonical segment and then turned by e^{i w dt} per step, one
// complex product each instead of a series or a sincos with its range
// reduction and a rotation by e^{i beta}.  Both reach only second order (the
// first-order transverse part is replaced by its exact FP64 quadrature at the
// end of the sample); the turns' rounding grows as (steps into the segment)
// x 2^-24 on those second-order terms, and the result depends on the step
// index alone, not on the launch shape.
template <typename R>
struct DrivePhasors {
    cx<R> co[2], ct[2];   // [node]
    cx<R> rco, rct;       // turns per step
};

template <typename R, int METHOD>
SPINSIM_HD void drive_phasors_at(const SampleCtx<R>& c, int64_t lo, DrivePhasors<R>& p)
{
    R s, co;
#pragma unroll
    for (int j = 0; j < 2; j++) {
        p.co[j] = cmk(R(0), R(0));
        p.ct[j] = cmk(R(0), R(0));
        if (METHOD == 1 && j == 1) break;   // one node
        const R tau = ((R)lo + (j ? c.c2 : c.c1)) * c.dt;
        small_sincos_tiny(c.co * tau, s, co);
        p.co[j] = cmk(c.ebr * co - c.ebi * s, fma(c.ebr, s, c.ebi * co));
        if (c.counter_on) {
            second_order_sincos(c.counter * tau, s, co);
            p.ct[j] = cmk(c.ebr * co - c.ebi * s, fma(c.ebr, s, c.ebi * co));
        }
    }
    small_sincos_tiny(c.co * c.dt, s, co);
    p.rco = cmk(co, s);
    second_order_sincos(c.counter * c.dt, s, co);
    p.rct = cmk(co, s);
}

template <typename R, int METHOD>
SPINSIM_HD void drive_phasors_advance(DrivePhasors<R>& p)
{
#pragma unroll
    for (int j = 0; j < 2; j++) {
        if (METHOD == 1 && j == 1) break;
        p.co[j] = cmul(p.co[j], p.rco);
        p.ct[j] = cmul(p.ct[j], p.rct);
    }
}

template <typename R, int SMALL = false, bool TONES = false, bool SU3 = false, bool PH = false>
SPINSIM_HD void field_at(const SampleCtx<R>& c, R tau, NodeField<R>& f, const CounterPhasors<R>* ph = nullptr,
                         int node = 0, const DrivePhasors<R>* dp = nullptr)
{
    if (dp) {
        // small-angle variant: both drive phasors turned per step (DrivePhasors)
        f.co = dp->co[node];
        f.ct = dp->ct[node];
    } else {
    R s1, c1;
    step_sincos<R, SMALL>(c.co * tau, s1, c1);
    f.co = cmk(c.ebr * c1 - c.ebi * s1, fma(c.ebr, s1, c.ebi * c1));
    if constexpr (PH) {
        f.ct = ph->d[node];   // zero when the counter-rotating term is off
    } else {
    if (c.counter_on) {
        // the counter-rotating term's first-order part is replaced exactly at
        // the end of the sample, so it only needs second-order accuracy
        R s2, c2;
        second_order_sincos(c.counter * tau, s2, c2);
        f.ct = cmk(c.ebr * c2 - c.ebi * s2, fma(c.ebr, s2, c.ebi * c2));
    } else {
        f.ct = cmk(R(0), R(0));
    }
    }
    }
    R z = R(0);
    if constexpr (SMALL) {
        // Gaussians only: exp(-u^2/2) as 2^(-ub^2), ub = u sqrt(log2(e)/2) (one
        // exp2 instead of a scaled exp), the loop ending at the pulse count
#pragma unroll
        for (int p = 0; p < kMaxPulses; p++) {
            if (p >= c.ng) break;
            const R ub = fma(tau, c.invwb[p], c.u0b[p]);
            z = fma(c.amp[p], exp2(-(ub * ub)) - c.ghat[p], z);
        }
        if constexpr ((SMALL & kSmallSine) != 0) {
            // the variant with single sine cycles (after the Gaussians), inline
#pragma unroll
            for (int p = 0; p < kMaxPulses; p++) {
                if (p >= c.np) break;
                if (p >= c.ng) {
                    const R u = fma(tau, c.invw[p], c.u0[p]);
                    z = fma(c.amp[p], sine_cycle(u) - c.ghat[p], z);
                }
            }
        }
    } else {
#pragma unroll
        for (int p = 0; p < kMaxPulses; p++) {
            if (p < c.ng) {
                R u = fma(tau, c.invw[p], c.u0[p]);
                z = fma(c.amp[p], exp(R(-0.5) * u * u) - c.ghat[p], z);
            }
        }
    }
    // single sine cycles: the general variant only (the small-angle variant is
    // chosen only for requests without them, and its step loop stays as lean)
    if constexpr (!SMALL) {
        if (c.np > c.ng) {
#pragma unroll
            for (int p = 0; p < kMaxPulses; p++) {
                if (p >= c.ng && p < c.np) {
                    R u = fma(tau, c.invw[p], c.u0[p]);
                    z = fma(c.amp[p], sine_cycle_cold(u) - c.ghat[p], z);
                }
            }
        }
    }
    f.z = z;
    if constexpr (TONES) {
        cx<R> e = cmk(R(0), R(0));
#pragma unroll
        for (int j = 0; j < kMaxTones; j++) {
            if (j < c.nt) {
                R sj, cj;
                small_sincos(c.tco[j] * tau, sj, cj);
                e.r = fma(c.tomp[j], c.tbr[j] * cj - c.tbi[j] * sj, e.r);
                e.i = fma(c.tomp[j], fma(c.tbr[j], sj, c.tbi[j] * cj), e.i);
                second_order_sincos(c.tct[j] * tau, sj, cj);
                // Om-_j conj(e^{i beta_j} e^{i w tau})
                e.r = fma(c.tomm[j], c.tbr[j] * cj - c.tbi[j] * sj, e.r);
                e.i = fma(-c.tomm[j], fma(c.tbr[j], sj, c.tbi[j] * cj), e.i);
            }
        }
        f.ex = e;
    }
    if constexpr (SU3) {
        // like a drive: Om+ e^{i (beta + (w - k w_r) tau)} + Om- e^{-i (beta + (w + k w_r) tau)}
#pragma unroll
        for (int p = 0; p < 2; p++) {
            R sj, cj;
            small_sincos(c.qco[p] * tau, sj, cj);
            cx<R> e = cscale(cmk(c.qbr[p] * cj - c.qbi[p] * sj, fma(c.qbr[p], sj, c.qbi[p] * cj)), c.qomp[p]);
            if constexpr (PH) {
                e.r = fma(c.qomm[p], ph->q[p][node].r, e.r);
                e.i = fma(-c.qomm[p], ph->q[p][node].i, e.i);
            } else {
                second_order_sincos(c.qct[p] * tau, sj, cj);
                e.r = fma(c.qomm[p], c.qbr[p] * cj - c.qbi[p] * sj, e.r);
                e.i = fma(-c.qomm[p], fma(c.qbr[p], sj, c.qbi[p] * cj), e.i);
            }
            f.qd[p] = e;
        }
    }
}

// sum_i w_i x_i
template <typename R>
SPINSIM_HD R dot4(const R* w, R x0, R x1, R x2, R x3)
{
    R h = w[0] * x0;
    h = fma(w[1], x1, h);
    h = fma(w[2], x2, h);
    h = fma(w[3], x3, h);
    return h;
}

// Exponent vector v = (H_bar delta_t) of one exponential from the two node
// fields, with node weights (a, b) (swap = false) or (b, a) (swap = true):
//   v_x + i v_y = P_a co_1 + P_b co_2 + conj(M_a ct_1 + M_b ct_2)   (w_x' + i w_y' as above)
// Further tones (TONES): v_x + i v_y += a dt ex_1 + b dt ex_2 (weights swapped
// likewise).
template <typename R, bool TONES = false>
SPINSIM_HD void exponent(const SampleCtx<R>& c, const NodeField<R>& f1, const NodeField<R>& f2,
                                         bool swap, R& vx, R& vy, R& vz)
{
    R w[4];
    const int ia = swap ? 1 : 0, ib = swap ? 0 : 1;
    w[0] = c.Ph[ia];
    w[1] = c.Ph[ib];
    w[2] = c.Ph[2 + ia];
    w[3] = c.Ph[2 + ib];
    vx = dot4(w, f1.co.r, f2.co.r, f1.ct.r, f2.ct.r);
    vy = dot4(w, f1.co.i, f2.co.i, -f1.ct.i, -f2.ct.i);
    const R wa = swap ? c.zb : c.za, wb = swap ? c.za : c.zb;
    vz = fma(wa, f1.z, fma(wb, f2.z, c.zbias));
    if constexpr (TONES) {
        vx = fma(wa, f1.ex.r, fma(wb, f2.ex.r, vx));
        vy = fma(wa, f1.ex.i, fma(wb, f2.ex.i, vy));
    }
}

// -------------------------------------------------------------------------
// Split residuals.  An operator close to the identity is carried as
//   U - I = F(g) + rest,
// where F(g) is its first-order part, -i times the generator
// g . (J_x, J_y, J_z, Q) (spin-one) or g . sigma/2 (spin-half), held as the
// coefficients g, and `rest` holds everything of second and higher order.
// The first-order coefficients of a step exponential exp(-i v.A) are exactly
// its exponent v, and those of a product add (U - I = A + B + AB).  At the end
// of a sample the first-order coefficients are replaced by their exact FP64
// value (the quadrature sum of the field over the sample), so FP32 rounding
// only ever touches the second-order part, whose coherent accumulation over
// 10^7 steps stays far below the target accuracy.  This extends the paper's
// residual idea (work with U - I, Sec. 1.2.3) one order further.
// -------------------------------------------------------------------------

// Spin-half: SU(2) elements [[alpha, -conj(beta)], [beta, conj(alpha)]].
// F(g): alpha - 1 = -i g_z / 2, beta = (g_y - i g_x) / 2.
template <typename R>
struct Res2 {
    R g[3];
    cx<R> a, b;   // second- and higher-order parts of alpha - 1 and beta
};

template <typename R>
SPINSIM_HD void res2_zero(Res2<R>& x)
{
    x.g[0] = x.g[1] = x.g[2] = R(0);
    x.a = cmk(R(0), R(0));
    x.b = cmk(R(0), R(0));
}

template <typename R>
SPINSIM_HD void res2_full(const Res2<R>& x, cx<R>& a, cx<R>& b)
{
    a = cmk(x.a.r, fma(R(-0.5), x.g[2], x.a.i));
    b = cmk(fma(R(0.5), x.g[1], x.b.r), fma(R(-0.5), x.g[0], x.b.i));
}

// exp(-i (v_x J_x + v_y J_y + v_z J_z)) with v = w delta_t, J = sigma/2, by the
// SU(2) identity cos(th/2) I - i sin(th/2) (v/th).sigma, th = |v| (Sec. 1.2.3):
//   alpha - 1 = -(1 - cos(th/2)) - i f v_z,  beta = f (v_y - i v_x),  f = sin(th/2)/th.
// First order: f -> 1/2.  The rest uses f - 1/2 and 1 - cos(th/2) = 2 sin^2(th/4),
// both from their Taylor series in y = th^2/4 for th/2 <= 1/16.
// f - 1/2 and 1 - cos(th/2) of the SU(2) exponential from t2 = th^2.
template <typename R>
SPINSIM_HD void half_angle_terms(R t2, R& fm, R& g)
{
    if (t2 <= R(0.015625)) {      // (th/2)^2 <= 1/256
        R y = R(0.25) * t2;
        fm = R(-0.5) * y * (R(1.0 / 6) - y * (R(1.0 / 120) - y * (R(1.0 / 5040) - y * R(1.0 / 362880))));
        g = y * (R(0.5) - y * (R(1.0 / 24) - y * (R(1.0 / 720) - y * (R(1.0 / 40320) - y * R(1.0 / 3628800)))));
    } else {
        R th = sqrt(t2);
        R s4 = sin(R(0.25) * th);
        fm = sin(R(0.5) * th) / th - R(0.5);
        g = R(2) * s4 * s4;
    }
}

template <typename R>
SPINSIM_HD void expm_half_res(R vx, R vy, R vz, Res2<R>& e)
{
    R fm, g;
    half_angle_terms(vx * vx + vy * vy + vz * vz, fm, g);
    e.g[0] = vx; e.g[1] = vy; e.g[2] = vz;
    e.a = cmk(-g, -fm * vz);
    e.b = cmk(fm * vy, -fm * vx);
}

// (I + A)(I + B) - I = A + B + A B, A later in time:
//   alpha = a1 a2 - conj(b1) b2,  beta = b1 a2 + conj(a1) b2   (full elements)
template <typename R>
SPINSIM_HD void res2_mul(const Res2<R>& A, const Res2<R>& B, Res2<R>& C)
{
    cx<R> Aa, Ab, Ba, Bb;
    res2_full(A, Aa, Ab);
    res2_full(B, Ba, Bb);
    cx<R> a = cadd(A.a, B.a);
    a = cfma(Aa, Ba, a);
    a = csub(a, cmul(cconj(Ab), Bb));
    cx<R> b = cadd(A.b, B.b);
    b = cfma(Ab, Ba, b);
    b = cfma_conj(Aa, Bb, b);
#pragma unroll
    for (int i = 0; i < 3; i++) C.g[i] = A.g[i] + B.g[i];
    C.a = a;
    C.b = b;
}

// Spin-one: F(g) = -i (g_x J_x + g_y J_y + g_z J_z + g_q Q), Q = diag(1,-2,1)/3.
template <typename R>
struct Res3 {
    R g[4];
    cx<R> m[3][3];   // second- and higher-order part
};

template <typename R>
SPINSIM_HD void res3_zero(Res3<R>& x)
{
#pragma unroll
    for (int i = 0; i < 4; i++) x.g[i] = R(0);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) x.m[i][j] = cmk(R(0), R(0));
}

template <typename R>
SPINSIM_HD void res3_full(const Res3<R>& x, cx<R> F[3][3])
{
    const R r = R(kInvSqrt2);
    const R q3 = x.g[3] * R(1.0 / 3);
    const cx<R> up = cmk(-x.g[1] * r, -x.g[0] * r);   // -i (g_x - i g_y)/sqrt2
    const cx<R> dn = cmk(x.g[1] * r, -x.g[0] * r);    // -i (g_x + i g_y)/sqrt2
    F[0][0] = cmk(x.m[0][0].r, x.m[0][0].i - (x.g[2] + q3));
    F[1][1] = cmk(x.m[1][1].r, fma(R(2), q3, x.m[1][1].i));
    F[2][2] = cmk(x.m[2][2].r, x.m[2][2].i + (x.g[2] - q3));
    F[0][1] = cadd(x.m[0][1], up);
    F[1][2] = cadd(x.m[1][2], up);
    F[1][0] = cadd(x.m[1][0], dn);
    F[2][1] = cadd(x.m[2][1], dn);
    F[0][2] = x.m[0][2];
    F[2][0] = x.m[2][0];
}

// (I + A)(I + B) - I = A + B + A B, A later in time.
template <typename R>
SPINSIM_HD void res3_mul(const Res3<R>& A, const Res3<R>& B, Res3<R>& C)
{
    cx<R> FA[3][3], FB[3][3];
    res3_full(A, FA);
    res3_full(B, FB);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<R> s = cadd(A.m[i][j], B.m[i][j]);
            s = cfma(FA[i][0], FB[0][j], s);
            s = cfma(FA[i][1], FB[1][j], s);
            s = cfma(FA[i][2], FB[2][j], s);
            C.m[i][j] = s;
        }
#pragma unroll
    for (int i = 0; i < 4; i++) C.g[i] = A.g[i] + B.g[i];
}

// exp(-i (v_x J_x + v_y J_y + v_z J_z + v_q Q)) ~= T^n, n = 2^tau, returned as a
// split residual (Sec. 1.2.3, Eqs. lie_trotter, lie_trotter_4).  The
// quadrupole coefficient is passed as qd3 = v_q / 3 / n.
//
// T = e^{-iD/2} e^{-i Phi J_phi} e^{-iD/2} with D = z J_z + q Q, z = v_z/n,
// q = v_q/n, Phi = |v_perp|/n.  Since e^{-i Phi J_phi} = W e^{-i Phi J_x} W^dagger
// with the diagonal W = e^{-i phi J_z} = diag(e^{-i phi}, 1, e^{i phi}), which
// commutes with D, T = W T0 W^dagger where T0 is T at phi = 0 and
// T^n = W T0^n W^dagger.  T0 is complex symmetric (diagonal x symmetric x
// diagonal), so its residual squarings s = (a + 2I) a keep it symmetric and
// need 6 of the 9 entries.  With the diagonal phases th_0 = -(z + q/3),
// th_1 = 2q/3, th_2 = z - q/3 and S = sin(Phi/2), T0 - I is
//   a_00 = expm1(i th_0) - S^2 e^{i th_0},  a_11 = expm1(i th_1) - 2 S^2 e^{i th_1},
//   a_22 = expm1(i th_2) - S^2 e^{i th_2},
//   a_01 = -i sin(Phi)/sqrt2 e^{-i th_2/2},  a_12 = -i sin(Phi)/sqrt2 e^{-i th_0/2},
//   a_02 = -S^2 e^{i (th_0 + th_2)/2}.
// Its first-order part is -i (Phi J_x + z J_z + q Q), i.e. i th_j on the
// diagonal and -i Phi/sqrt2 next to it; the rest is formed without
// cancellation from sin x - x and cos x - 1.  A residual squaring
// (a + 2I) a = 2a + a^2 doubles the first-order part exactly and adds a^2 to
// the rest.
// expm_one_res_n takes 2^-tau and the first-order quadrupole coefficient
// q1 = 3 qd3 2^tau precomputed (once per sample) and, with SMALL, uses the
// small-angle series (all of h_0, h_1, h_2, Phi/2 bounded by 2^-6 on the host).
template <typename R, int SMALL = false>
SPINSIM_HD void expm_one_res_n(R vx, R vy, R vz, R qd3, int tau, R inv_n, R q1, Res3<R>& e)
{
    const R z = vz * inv_n;
    const R vp2 = vx * vx + vy * vy;
    R epr = R(1), epi = R(0);   // e^{i phi}
    R Phi = R(0);
    if constexpr (BulkTraits<R>::lanes == 1) {
        if (vp2 > R(0)) {
            // Phi and e^{i phi} enter only the second-order rest (the first-order
            // part is v itself), so a reciprocal square root is precise enough.
            const R rinv = rsqrt(vp2);
            epr = vx * rinv;
            epi = vy * rinv;
            Phi = vp2 * rinv * inv_n;
        }
    } else {
        transverse_axis_lanes(vx, vy, vp2, inv_n, epr, epi, Phi);   // the same, lane by lane
    }
    const R h0 = fma(R(-0.5), z, R(-0.5) * qd3);   // th_0 / 2
    const R h1 = qd3;                              // th_1 / 2
    const R h2 = fma(R(0.5), z, R(-0.5) * qd3);    // th_2 / 2
    const R P = R(0.5) * Phi;
    R sm0, cm0, sm1, cm1, sm2, cm2, smP, cmP;
    step_sincos_m<R, SMALL>(h0, sm0, cm0);
    step_sincos_m<R, SMALL>(h1, sm1, cm1);
    step_sincos_m<R, SMALL>(h2, sm2, cm2);
    step_sincos_m<R, SMALL>(P, smP, cmP);
    const R s0 = h0 + sm0, c0 = R(1) + cm0;       // sin, cos of th_j / 2
    const R s1 = h1 + sm1, c1 = R(1) + cm1;
    const R s2 = h2 + sm2, c2 = R(1) + cm2;
    const R sP = P + smP;
    const R S2 = sP * sP;
    // cos th - 1 = -2 sin^2(th/2);  sin th - th = 2 (sm + h cm + sm cm)
    const cx<R> d0 = cmk(R(-2) * s0 * s0, R(2) * fma(h0, cm0, sm0 * c0));
    const cx<R> d1 = cmk(R(-2) * s1 * s1, R(2) * fma(h1, cm1, sm1 * c1));
    const cx<R> d2 = cmk(R(-2) * s2 * s2, R(2) * fma(h2, cm2, sm2 * c2));
    // e^{i th} = 1 + (cos th - 1) + i sin th
    const cx<R> p0 = cmk(R(1) + d0.r, R(2) * s0 * c0);
    const cx<R> p1 = cmk(R(1) + d1.r, R(2) * s1 * c1);
    const cx<R> p2 = cmk(R(1) + d2.r, R(2) * s2 * c2);
    // rest of T0 - I (symmetric: b_10 = b_01, b_20 = b_02, b_21 = b_12)
    cx<R> b00 = csub(d0, cscale(p0, S2));
    cx<R> b11 = csub(d1, cscale(p1, R(2) * S2));
    cx<R> b22 = csub(d2, cscale(p2, S2));
    // -i/sqrt2 [ (sin Phi - Phi) e^{-i h} + Phi (e^{-i h} - 1) ]
    const R r = R(kInvSqrt2);
    const R sPm = R(2) * fma(P, cmP, smP * (R(1) + cmP));   // sin Phi - Phi
    cx<R> t01 = cmk(fma(sPm, c2, Phi * cm2), -(sPm + Phi) * s2);   // (sin Phi - Phi) e^{-i h2} + Phi (e^{-i h2} - 1)
    cx<R> t12 = cmk(fma(sPm, c0, Phi * cm0), -(sPm + Phi) * s0);
    cx<R> b01 = cmk(r * t01.i, -r * t01.r);
    cx<R> b12 = cmk(r * t12.i, -r * t12.r);
    cx<R> b02 = cscale(cmk(c0 * c2 - s0 * s2, s0 * c2 + c0 * s2), -S2);
    // first-order coefficients in the phi = 0 frame
    R fP = Phi, fz = z, fq3 = qd3;
    for (int it = 0; it < tau; it++) {
        // full symmetric matrix A = F0 + rest; F0 = -i (Phi J_x + z J_z + q Q)
        const cx<R> A00 = cmk(b00.r, b00.i - (fz + fq3));
        const cx<R> A11 = cmk(b11.r, fma(R(2), fq3, b11.i));
        const cx<R> A22 = cmk(b22.r, b22.i + (fz - fq3));
        const R o = -fP * r;
        const cx<R> A01 = cmk(b01.r, b01.i + o);
        const cx<R> A12 = cmk(b12.r, b12.i + o);
        const cx<R> A02 = b02;
        // rest <- 2 rest + A^2
        b00 = cfma(A02, A02, cfma(A01, A01, cfma(A00, A00, cscale(b00, R(2)))));
        const cx<R> n01 = cfma(A02, A12, cfma(A01, A11, cfma(A00, A01, cscale(b01, R(2)))));
        const cx<R> n02 = cfma(A02, A22, cfma(A01, A12, cfma(A00, A02, cscale(b02, R(2)))));
        b11 = cfma(A12, A12, cfma(A11, A11, cfma(A01, A01, cscale(b11, R(2)))));
        const cx<R> n12 = cfma(A12, A22, cfma(A11, A12, cfma(A01, A02, cscale(b12, R(2)))));
        b22 = cfma(A22, A22, cfma(A12, A12, cfma(A02, A02, cscale(b22, R(2)))));
        b01 = n01; b02 = n02; b12 = n12;
        fP *= R(2); fz *= R(2); fq3 *= R(2);
    }
    // W (rest) W^dagger: entry (j, l) picks up e^{-i phi (m_j - m_l)}
    const cx<R> ep = cmk(epr, epi), em = cmk(epr, -epi);
    const cx<R> ep2 = cmul(ep, ep), em2 = cconj(ep2);
    e.m[0][0] = b00; e.m[1][1] = b11; e.m[2][2] = b22;
    e.m[0][1] = cmul(b01, em); e.m[1][0] = cmul(b01, ep);
    e.m[1][2] = cmul(b12, em); e.m[2][1] = cmul(b12, ep);
    e.m[0][2] = cmul(b02, em2); e.m[2][0] = cmul(b02, ep2);
    e.g[0] = vx; e.g[1] = vy; e.g[2] = vz; e.g[3] = q1;
}

template <typename R, int SMALL = false>
SPINSIM_HD void expm_one_res(R vx, R vy, R vz, R qd3, int tau, Res3<R>& e)
{
    expm_one_res_n<R, SMALL>(vx, vy, vz, qd3, tau, ldexp(R(1), -tau), R(3) * ldexp(qd3, tau), e);
}

// The same exponential for tau = 0 (one factor T, n = 1) and small angles
// (the host bounds h_0, h_1, h_2 and Phi / 2 by 2^-6, small_angle_request),
// with the conjugation by W folded into the transverse field itself.  With
// u = v_x - i v_y = Phi e^{-i phi} and y = Phi^2 = |u|^2 the entries of
// W (T0 - I) W^dagger beyond first order are
//   diagonal:  d_j - S^2 e^{i th_j} (m = 0: 2 S^2), S^2 = sin^2(Phi/2) = sigma y,
//   (0,1), (1,0):  -i/sqrt2 t_2 u, -i/sqrt2 t_2 conj(u),
//   (1,2), (2,1):  -i/sqrt2 t_0 u, -i/sqrt2 t_0 conj(u),
//   (0,2), (2,0):  -sigma e^{-i qd3} u^2, -sigma e^{-i qd3} conj(u)^2,
// where t_j = kappa e^{-i h_j} + (e^{-i h_j} - 1), kappa = (sin Phi - Phi) / Phi
// and sigma = sin^2(Phi/2) / Phi^2, both series in y (truncation below 2e-9
// relative for Phi <= 2^-5), and e^{i (th_0 + th_2) / 2} = e^{-i qd3}.  This is
// expm_one_res_n's T at tau = 0 in closed form without the reciprocal square
// root, the angle phi or the conjugation products; the h_1 terms and
// e^{-i qd3} are per-simulation constants of the context.
template <typename R>
SPINSIM_HD void expm_one_res_tau0(R vx, R vy, R vz, const SampleCtx<R>& c, Res3<R>& e)
{
    const R y = fma(vx, vx, vy * vy);
    const R h0 = fma(R(-0.5), vz, R(-0.5) * c.qd3);   // th_0 / 2
    const R h2 = fma(R(0.5), vz, R(-0.5) * c.qd3);    // th_2 / 2
    R sm0, cm0, sm2, cm2;
    small_sincos_m_tiny(h0, sm0, cm0);
    small_sincos_m_tiny(h2, sm2, cm2);
    const R s0 = h0 + sm0, c0 = R(1) + cm0;
    const R s2 = h2 + sm2, c2 = R(1) + cm2;
    const R kappa = y * fma(y, R(1.0 / 120), R(-1.0 / 6));
    const R sigma = fma(y, fma(y, R(1.0 / 1440), R(-1.0 / 48)), R(0.25));
    const R S2 = sigma * y;
    // diagonal: cos th - 1 = -2 sin^2(th/2), sin th - th = 2 (sm + h cm + sm cm), minus S^2 e^{i th}
    const cx<R> d0 = cmk(R(-2) * s0 * s0, R(2) * fma(h0, cm0, sm0 * c0));
    const cx<R> d2 = cmk(R(-2) * s2 * s2, R(2) * fma(h2, cm2, sm2 * c2));
    const cx<R> p0 = cmk(R(1) + d0.r, R(2) * s0 * c0);
    const cx<R> p2 = cmk(R(1) + d2.r, R(2) * s2 * c2);
    e.m[0][0] = csub(d0, cscale(p0, S2));
    e.m[1][1] = csub(cmk(c.d1r, c.d1i), cscale(cmk(c.p1r, c.p1i), R(2) * S2));
    e.m[2][2] = csub(d2, cscale(p2, S2));
    // next to the diagonal: -i t u and -i t conj(u) with u / sqrt2 = (vx, -vy) / sqrt2
    const R r = R(kInvSqrt2);
    const R ur = r * vx, ui = -(r * vy);
    const R t2r = fma(kappa, c2, cm2), t2i = -(kappa + R(1)) * s2;
    const R t0r = fma(kappa, c0, cm0), t0i = -(kappa + R(1)) * s0;
    {
        const R D = t2i * ur, B = t2i * ui;
        e.m[0][1] = cmk(fma(t2r, ui, D), fma(-t2r, ur, B));
        e.m[1][0] = cmk(fma(-t2r, ui, D), fma(-t2r, ur, -B));
    }
    {
        const R D = t0i * ur, B = t0i * ui;
        e.m[1][2] = cmk(fma(t0r, ui, D), fma(-t0r, ur, B));
        e.m[2][1] = cmk(fma(-t0r, ui, D), fma(-t0r, ur, -B));
    }
    // corners: g u^2 and g conj(u)^2, g = -sigma e^{-i qd3}, u^2 = (vx^2 - vy^2, -2 vx vy)
    const R gr = -sigma * c.eqr, gi = -sigma * c.eqi;
    const R u2r = fma(vx, vx, -(vy * vy)), u2i = R(-2) * vx * vy;
    {
        const R P = gi * u2r, Q = gi * u2i;
        e.m[0][2] = cmk(fma(gr, u2r, -Q), fma(gr, u2i, P));
        e.m[2][0] = cmk(fma(gr, u2r, Q), fma(-gr, u2i, P));
    }
    e.g[0] = vx; e.g[1] = vy; e.g[2] = vz; e.g[3] = c.q1;
}

// 1/k! rounded once (k! is exact in double up to k = 18), the Taylor coefficients.
SPINSIM_HD constexpr double inv_factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; i++) f *= i;
    return 1.0 / f;
}

// The IEEE bit pattern of a double as a signed integer.
SPINSIM_HD int64_t double_bits(double x)
{
#ifdef __CUDA_ARCH__
    return __double_as_longlong(x);
#else
    int64_t b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

// The Taylor degree of the general exponential at scaled norm th >= 0 (see
// expm_general_res); for doubles the bit patterns are compared as integers.
template <typename R>
SPINSIM_HD int taylor_degree(R th)
{
    if constexpr (kFP32<R>) {
        return th <= R(6.9e-6) ? 3 : th <= R(2.0e-4) ? 4 : th <= R(1.58e-3) ? 5 : th <= R(6.4e-3) ? 6
             : th <= R(1.77e-2) ? 7 : th <= R(3.85e-2) ? 8 : th <= R(7.1e-2) ? 9 : th <= R(0.117) ? 10
             : th <= R(0.177) ? 11 : 12;
    } else {
        const int64_t b = double_bits(th);
        return b <= double_bits(6.9e-6) ? 3 : b <= double_bits(2.0e-4) ? 4 : b <= double_bits(1.58e-3) ? 5
             : b <= double_bits(6.4e-3) ? 6 : b <= double_bits(1.77e-2) ? 7 : b <= double_bits(3.85e-2) ? 8
             : b <= double_bits(7.1e-2) ? 9 : b <= double_bits(0.117) ? 10 : b <= double_bits(0.177) ? 11 : 12;
    }
}

// C = A P for a Hermitian A with a real diagonal (entries above and below the
// diagonal both stored) and a general P.
template <typename R>
SPINSIM_HD void herm_mul3(const cx<R> (&A)[3][3], const cx<R> (&P)[3][3], cx<R> (&C)[3][3])
{
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int k1 = (i + 1) % 3, k2 = (i + 2) % 3;
#pragma unroll
        for (int j = 0; j < 3; j++)
            C[i][j] = cfma(A[i][k2], P[k2][j], cfma(A[i][k1], P[k1][j], cscale(P[i][j], A[i][i].r)));
    }
}

// exp(-i H) - I as a split residual for a full su(3) spin-one H (radians):
//   H = v_x J_x + v_y J_y + v_z J_z + v_q Q + u_0 D_xz + u_1 D_yz + u_2 D_x2y2 + u_3 D_xy,
// D_ab the symmetric products of the spin matrices.  In the basis m = +1, 0, -1,
// with t = v_x - i v_y, c = u_0 - i u_1 and d = u_2 - i u_3:
//   H_00 = v_z + v_q/3, H_11 = -2 v_q/3, H_22 = -v_z + v_q/3,
//   H_01 = (t + c)/sqrt2, H_12 = (t - c)/sqrt2, H_02 = d, H_ji = conj(H_ij).
// The series sum_{k>=1} B^k / k! of B = -i H / 2^s (s halvings until the row
// sums are at most 1/4; degree 3 to 12 by the scaled norm), then
// s residual squarings a <- (a + 2I) a; the first-order part of the J and Q
// terms is taken out as g, the rest (the quadrupole drives' first order and
// all higher orders) stays in the full matrix.  FP64 (the su(3) variant).
template <typename R>
SPINSIM_HD void expm_general_res(R vx, R vy, R vz, R vq, const R u[4], Res3<R>& e)
{
    const R r = R(kInvSqrt2);
    const R q3 = vq * R(1.0 / 3);
    const cx<R> t = cmk(vx, -vy), c = cmk(u[0], -u[1]), d = cmk(u[2], -u[3]);
    cx<R> H[3][3];
    H[0][0] = cmk(vz + q3, R(0));
    H[1][1] = cmk(R(-2) * q3, R(0));
    H[2][2] = cmk(q3 - vz, R(0));
    H[0][1] = cscale(cadd(t, c), r);
    H[1][2] = cscale(csub(t, c), r);
    H[0][2] = d;
    H[1][0] = cconj(H[0][1]);
    H[2][1] = cconj(H[1][2]);
    H[2][0] = cconj(d);
    R norm = R(0);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        R row = R(0);
#pragma unroll
        for (int j = 0; j < 3; j++) row += fabs(H[i][j].r) + fabs(H[i][j].i);
        norm = row > norm ? row : norm;
    }
    int s = 0;
    R scale = R(1);
    while (norm * scale > R(0.25) && s < 60) {
        scale *= R(0.5);
        s++;
    }
    cx<R> B[3][3], P[3][3], T[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) B[i][j] = cmk(H[i][j].i, -H[i][j].r);   // -i H
    if (s > 0) {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) B[i][j] = cscale(B[i][j], scale);   // -i H 2^-s
    }
    // Taylor degree m: the smallest whose remainder bound at the scaled norm,
    // theta^(m+1) e^theta / (m+1)!, stays below 2^-56 theta (relative to the
    // first-order term); theta <= 1/4 needs the full m = 12.  The norm is
    // non-negative, so its bit pattern orders like its value: the comparisons
    // run as integer compares.
    const int m = taylor_degree(norm * scale);
    // The degree-m Taylor polynomial without its constant term, evaluated in
    // powers of B2 = B^2 (Paterson-Stockmeyer with two blocks):
    //   T = B + B2 (Y_1 + B2 (Y_2 + ... + B2 Y_J)),  Y_j = I/(2j)! + B/(2j+1)!,
    // J = floor(m/2), terms beyond degree m dropped.  B2 = -(H 2^-s)^2 is
    // Hermitian with a real diagonal: six entries are computed.
    cx<R> B2[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < 3; k++) acc = fma(-B[i][k].r, B[i][k].r, fma(-B[i][k].i, B[i][k].i, acc));
        B2[i][i] = cmk(acc, R(0));
    }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i + 1; j < 3; j++) {
            B2[i][j] = cfma(B[i][2], B[2][j], cfma(B[i][1], B[1][j], cmul(B[i][0], B[0][j])));
            B2[j][i] = cconj(B2[i][j]);
        }
    const int J = m / 2;
    // innermost block: Y_J, or for even m the scalar I/m! folded into the next block
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) P[i][j] = cmk(R(0), R(0));
#pragma unroll
    for (int jb = 6; jb >= 1; jb--) {
        if (jb > J) continue;
        const R ce = R(inv_factorial(2 * jb)), co = R(inv_factorial(2 * jb + 1));
        if (jb == J) {
            if (m & 1) {
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++)
                        P[i][j] = cadd(cscale(B[i][j], co), cmk(i == j ? ce : R(0), R(0)));
            }
            continue;
        }
        if (jb == J - 1 && !(m & 1)) {       // P = Y_jb + B2 / (2J)!
            const R cJ = R(inv_factorial(2 * jb + 2));
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++)
                    P[i][j] = cadd(cadd(cscale(B[i][j], co), cscale(B2[i][j], cJ)), cmk(i == j ? ce : R(0), R(0)));
            continue;
        }
        herm_mul3(B2, P, T);                  // P = Y_jb + B2 P
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                P[i][j] = cadd(cadd(T[i][j], cscale(B[i][j], co)), cmk(i == j ? ce : R(0), R(0)));
    }
    herm_mul3(B2, P, T);                      // B2 P (m >= 3, so P is set)
    if (s == 0) {
        // exp(B) - I = B + B2 P with B = -i H: the rest beyond the J and Q
        // first order is B2 P plus -i times the quadrupole part of H (off the
        // diagonal only), formed directly
        const cx<R> cr = cscale(c, r);
        const cx<R> m01 = cmk(cr.i, -cr.r), m10 = cmk(-cr.i, -cr.r);   // -i c/sqrt2, -i conj(c)/sqrt2
        const cx<R> m02 = cmk(d.i, -d.r), m20 = cmk(-d.i, -d.r);       // -i d, -i conj(d)
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) e.m[i][j] = T[i][j];
        e.m[0][1] = cadd(e.m[0][1], m01);
        e.m[1][2] = csub(e.m[1][2], m01);
        e.m[1][0] = cadd(e.m[1][0], m10);
        e.m[2][1] = csub(e.m[2][1], m10);
        e.m[0][2] = cadd(e.m[0][2], m02);
        e.m[2][0] = cadd(e.m[2][0], m20);
        e.g[0] = vx; e.g[1] = vy; e.g[2] = vz; e.g[3] = vq;
        return;
    }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) T[i][j] = cadd(T[i][j], B[i][j]);   // T = exp(B) - I
    // residual squarings
#pragma unroll 1
    for (int q = 0; q < s; q++) {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) P[i][j] = cadd(T[i][j], cmk(i == j ? R(2) : R(0), R(0)));
        cx<R> S[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) S[i][j] = cfma(P[i][2], T[2][j], cfma(P[i][1], T[1][j], cmul(P[i][0], T[0][j])));
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) T[i][j] = S[i][j];
    }
    // split off the first order of the J and Q terms
    Res3<R> f;
    res3_zero(f);
    f.g[0] = vx; f.g[1] = vy; f.g[2] = vz; f.g[3] = vq;
    cx<R> F[3][3];
    res3_full(f, F);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) e.m[i][j] = csub(T[i][j], F[i][j]);
    e.g[0] = vx; e.g[1] = vy; e.g[2] = vz; e.g[3] = vq;
}

// The quadrupole-drive part of one exponential's exponent, weights as in
// `exponent`: u_2p + i u_2p+1 = a dt qd_p(node 1) + b dt qd_p(node 2).
template <typename R>
SPINSIM_HD void exponent_qd(const SampleCtx<R>& c, const NodeField<R>& f1, const NodeField<R>& f2, bool swap, R u[4])
{
    const R wa = swap ? c.zb : c.za, wb = swap ? c.za : c.zb;
#pragma unroll
    for (int p = 0; p < 2; p++) {
        u[2 * p] = fma(wa, f1.qd[p].r, wb * f2.qd[p].r);
        u[2 * p + 1] = fma(wa, f1.qd[p].i, wb * f2.qd[p].i);
    }
}

// -------------------------------------------------------------------------
// One integration step u(t_{k-1} + (l+1) dt, t_{k-1} + l dt), as a split
// residual, for the three methods.  METHOD: 0 CF4 (Sec. 1.2.2, nodes
// c1,2 = (1 -+ 1/sqrt3)/2, u = exp(-i Hbar_2 dt) exp(-i Hbar_1 dt)); 1 midpoint
// sampling (one exponential at t + dt/2); 2 Heun sampling (one exponential of
// the average of the end-point fields) (Sec. 1.3.1).  The node offsets and
// weights come with the context.
// -------------------------------------------------------------------------
template <typename R, int METHOD>
SPINSIM_HD void step_res(const SampleCtx<R>& c, R lf, int tau, Res3<R>& x)
{
    NodeField<R> f1, f2;
    field_at(c, (lf + c.c1) * c.dt, f1);
    if (METHOD == 1) f2 = f1;
    else field_at(c, (lf + c.c2) * c.dt, f2);
    R vx, vy, vz;
    exponent(c, f1, f2, false, vx, vy, vz);
    if (METHOD == 0) {
        Res3<R> e1, e2;
        expm_one_res(vx, vy, vz, c.qd3, tau, e1);
        exponent(c, f1, f2, true, vx, vy, vz);
        expm_one_res(vx, vy, vz, c.qd3, tau, e2);
        res3_mul(e2, e1, x);   // Eq. cf4_implementation
    } else {
        expm_one_res(vx, vy, vz, c.qd3, tau, x);
    }
}

template <typename R, int METHOD, int SMALL = false, bool TONES = false>
SPINSIM_HD void step_res(const SampleCtx<R>& c, R lf, int tau, Res2<R>& x)
{
    (void)tau;
    NodeField<R> f1, f2;
    field_at<R, SMALL, TONES>(c, (lf + c.c1) * c.dt, f1);
    if (METHOD == 1) f2 = f1;
    else field_at<R, SMALL, TONES>(c, (lf + c.c2) * c.dt, f2);
    R vx, vy, vz;
    exponent<R, TONES>(c, f1, f2, false, vx, vy, vz);
    if (METHOD == 0) {
        Res2<R> e1, e2;
        expm_half_res(vx, vy, vz, e1);
        exponent<R, TONES>(c, f1, f2, true, vx, vy, vz);
        expm_half_res(vx, vy, vz, e2);
        res2_mul(e2, e1, x);
    } else {
        expm_half_res(vx, vy, vz, x);
    }
}

// Premultiply the running residual by one step: X <- u X.  For CF4 the two
// exponentials are applied one after the other, X <- E_2 (E_1 X) (the same
// product as (E_2 E_1) X, Eq. cf4_implementation, in the same number of
// operations), so only one step exponential is held in registers at a time.
// One CF4 (or midpoint / Heun) step of the su(3) variant: the counter-rotating
// phasors come from the segment's running turns and advance by one step.
template <typename R, int METHOD, bool TONES>
SPINSIM_HD void step_apply_su3(const SampleCtx<R>& c, R lf, CounterPhasors<R>& ph, Res3<R>& X)
{
    NodeField<R> f1, f2;
    field_at<R, false, TONES, true, true>(c, (lf + c.c1) * c.dt, f1, &ph, 0);
    if (METHOD == 1) f2 = f1;
    else field_at<R, false, TONES, true, true>(c, (lf + c.c2) * c.dt, f2, &ph, 1);
    counter_phasors_advance<R, METHOD>(ph);
    R vx, vy, vz, wx = R(0), wy = R(0), wz = R(0);
    exponent<R, TONES>(c, f1, f2, false, vx, vy, vz);
    if (METHOD == 0) exponent<R, TONES>(c, f1, f2, true, wx, wy, wz);
    // the general exponential of each step exponent (v_q = q1)
    R u[4];
    Res3<R> e, Y;
    exponent_qd(c, f1, f2, false, u);
    expm_general_res(vx, vy, vz, c.q1, u, e);
    res3_mul(e, X, Y);
    if (METHOD == 0) {
        exponent_qd(c, f1, f2, true, u);
        expm_general_res(wx, wy, wz, c.q1, u, e);
        res3_mul(e, Y, X);
    } else {
        X = Y;
    }
}

template <typename R, int METHOD, int SMALL = false, bool TONES = false>
SPINSIM_HD void step_apply(const SampleCtx<R>& c, R lf, int tau, Res3<R>& X, DrivePhasors<R>* dp = nullptr)
{
    NodeField<R> f1, f2;
    field_at<R, SMALL, TONES>(c, (lf + c.c1) * c.dt, f1, nullptr, 0, dp);
    if (METHOD == 1) f2 = f1;
    else field_at<R, SMALL, TONES>(c, (lf + c.c2) * c.dt, f2, nullptr, 1, dp);
    if (dp) drive_phasors_advance<R, METHOD>(*dp);
    R vx, vy, vz, wx = R(0), wy = R(0), wz = R(0);
    exponent<R, TONES>(c, f1, f2, false, vx, vy, vz);
    if (METHOD == 0) exponent<R, TONES>(c, f1, f2, true, wx, wy, wz);
    Res3<R> e, Y;
    if constexpr ((SMALL & kSmallTau0) != 0) {
        // tau = 0 known at compile time: the closed form only
        expm_one_res_tau0(vx, vy, vz, c, e);
    } else if constexpr (SMALL) {
        // small angles: tau = 0 in closed form, else the squarings
        if (tau == 0) expm_one_res_tau0(vx, vy, vz, c, e);
        else expm_one_res_n<R, SMALL>(vx, vy, vz, c.qd3, tau, c.inv_n, c.q1, e);
    } else {
        expm_one_res_n<R, SMALL>(vx, vy, vz, c.qd3, tau, c.inv_n, c.q1, e);
    }
    res3_mul(e, X, Y);
    if (METHOD == 0) {
        if constexpr ((SMALL & kSmallTau0) != 0) {
            expm_one_res_tau0(wx, wy, wz, c, e);
        } else if constexpr (SMALL) {
            if (tau == 0) expm_one_res_tau0(wx, wy, wz, c, e);
            else expm_one_res_n<R, SMALL>(wx, wy, wz, c.qd3, tau, c.inv_n, c.q1, e);
        } else {
            expm_one_res_n<R, SMALL>(wx, wy, wz, c.qd3, tau, c.inv_n, c.q1, e);
        }
        res3_mul(e, Y, X);
    } else {
        X = Y;
    }
}

template <typename R, int METHOD, int SMALL = false, bool TONES = false, bool SU3 = false>
SPINSIM_HD void step_apply(const SampleCtx<R>& c, R lf, int tau, Res2<R>& X)
{
    static_assert(!SU3, "quadrupole drives need spin one");
    Res2<R> x, Y;
    step_res<R, METHOD, SMALL, TONES>(c, lf, tau, x);
    res2_mul(x, X, Y);
    X = Y;
}

template <typename R>
SPINSIM_HD void res_zero(Res3<R>& x) { res3_zero(x); }
template <typename R>
SPINSIM_HD void res_zero(Res2<R>& x) { res2_zero(x); }
template <typename R>
SPINSIM_HD void res_mul(const Res3<R>& A, const Res3<R>& B, Res3<R>& C) { res3_mul(A, B, C); }
template <typename R>
SPINSIM_HD void res_mul(const Res2<R>& A, const Res2<R>& B, Res2<R>& C) { res2_mul(A, B, C); }

}  // namespace spinsim
