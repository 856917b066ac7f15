// params.cu -- host-side request handling shared by every entry point
// (spinsim_simulate / spinsim_submit, spinsim_simulate_static and the
// multicore CPU backend): validation, and the per-simulation parameter record
// (DevSim) precomputed in FP64 from a request and the configuration.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace spinsim {

namespace {

constexpr double kTwoPiH = 6.283185307179586476925286766559;

// Node offsets (units of delta_t) and weights of the method.  CF4
// (Eqs. cf4_sample_1/2): t_{1,2} = t + (1 -+ 1/sqrt3) dt/2,
// a = (3 + 2 sqrt3)/12, b = (3 - 2 sqrt3)/12, two exponentials.  Midpoint and
// Heun sampling (Sec. 1.3.1): one exponential.
struct MethodNodes {
    double c1, c2, wa, wb;
    int n_exp;
};

MethodNodes method_nodes(int method)
{
    if (method == SPINSIM_METHOD_CF4)
        return {0.2113248654051871177454256, 0.7886751345948128822545744, 0.5386751345948128822545744,
                -0.03867513459481288225457439, 2};
    if (method == SPINSIM_METHOD_MIDPOINT) return {0.5, 0.5, 1.0, 0.0, 1};
    return {0.0, 1.0, 0.5, 0.5, 1};
}

double pulse_weight(const spinsim_field& f)
{
    double w = 0.0;
    for (int p = 0; p < f.n_pulses; p++) w += kTwoPiH * std::fabs(f.pulse_amp_hz[p]);
    return w;
}

// Taylor tables T_m = sum_{l<L, n=1,2} W_n x^m e^{i th x}, x = l + c_n, m = 0..3
// (re/im interleaved) of the node-phasor sum at th (direct FP64 summation).
void phasor_tables(double th, int64_t L, const double Wn[2], const double cn[2], double T[8])
{
    for (int m = 0; m < 8; m++) T[m] = 0.0;
    // e^{i th x} of both nodes, from sin/cos every kResync steps and turned by
    // e^{i th} in between (the turns' rounding stays below kResync x 2^-52
    // relative); sin/cos at every node made this the host's largest cost per
    // request (12 us at L = 100)
    constexpr int64_t kResync = 32;
    const double tc = std::cos(th), ts = std::sin(th);
    double ca_n[2] = {1.0, 1.0}, sa_n[2] = {0.0, 0.0};
    for (int64_t l = 0; l < L; l++)
        for (int nn = 0; nn < 2; nn++) {
            if (Wn[nn] == 0.0) continue;
            const double x = (double)l + cn[nn];
            if (l % kResync == 0) {
                ca_n[nn] = std::cos(th * x);
                sa_n[nn] = std::sin(th * x);
            } else {
                const double c0 = ca_n[nn], s0 = sa_n[nn];
                ca_n[nn] = c0 * tc - s0 * ts;
                sa_n[nn] = c0 * ts + s0 * tc;
            }
            const double sa = sa_n[nn], ca = ca_n[nn];
            double pw = Wn[nn];
            for (int m = 0; m < 4; m++) {
                T[2 * m] += pw * ca;
                T[2 * m + 1] += pw * sa;
                pw *= x;
            }
        }
}

}  // namespace

constexpr int64_t kMaxL = int64_t(1) << 24;  // step index stays exact in FP32

Checked check_request(const spinsim_request* r)
{
    Checked c;
    if (!r) { c.status = SPINSIM_E_ARG; return c; }
    if (r->spin_x2 != 1 && r->spin_x2 != 2) { c.status = SPINSIM_E_ARG; return c; }
    const spinsim_field& f = r->field;
    if (f.n_pulses < 0 || f.n_pulses > SPINSIM_MAX_PULSES) { c.status = SPINSIM_E_ARG; return c; }
    if (f.n_tones < 0 || f.n_tones > SPINSIM_MAX_TONES) { c.status = SPINSIM_E_ARG; return c; }
    for (int j = 0; j < f.n_tones; j++)
        if (!std::isfinite(f.tone_x_hz[j]) || !std::isfinite(f.tone_y_hz[j]) || !std::isfinite(f.tone_hz[j]) ||
            !std::isfinite(f.tone_phase[j])) {
            c.status = SPINSIM_E_ARG;
            return c;
        }
    if (f.qd_on != 0 && (f.qd_on != 1 || r->spin_x2 != 2)) { c.status = SPINSIM_E_ARG; return c; }
    if (f.qd_on)
        for (int p = 0; p < 2; p++)
            if (!std::isfinite(f.qd_x_hz[p]) || !std::isfinite(f.qd_y_hz[p]) || !std::isfinite(f.qd_hz[p]) ||
                !std::isfinite(f.qd_phase[p])) {
                c.status = SPINSIM_E_ARG;
                return c;
            }
    for (int p = 0; p < f.n_pulses; p++)
        if (!(f.pulse_width_s[p] > 0.0) || !std::isfinite(f.pulse_amp_hz[p]) || !std::isfinite(f.pulse_centre_s[p])) {
            c.status = SPINSIM_E_ARG;
            return c;
        }
    const double vals[] = {f.bias_hz, f.drive_x_hz, f.drive_y_hz, f.drive_hz, f.drive_phase, f.quad_hz,
                           r->t_start, r->t_end, r->dt, r->dt_out};
    for (double v : vals)
        if (!std::isfinite(v)) { c.status = SPINSIM_E_ARG; return c; }
    if (!(r->dt > 0.0) || !(r->dt_out > 0.0) || !(r->t_end >= r->t_start)) { c.status = SPINSIM_E_ARG; return c; }
    const double rk = (r->t_end - r->t_start) / r->dt_out;
    const double rl = r->dt_out / r->dt;
    const double k = std::floor(rk + 0.5), l = std::floor(rl + 0.5);
    if (std::fabs(rk - k) > 1e-9 * std::max(1.0, rk) || std::fabs(rl - l) > 1e-9 * std::max(1.0, rl) || l < 1.0 ||
        l > (double)kMaxL || k > 9.0e15) {
        c.status = SPINSIM_E_STEP_RATIO;
        return c;
    }
    c.K = (int64_t)k;
    c.L = (int64_t)l;
    const int n = r->spin_x2 + 1;
    double nrm = 0.0;
    for (int i = 0; i < 2 * n; i++) {
        if (!std::isfinite(r->psi0[i])) { c.status = SPINSIM_E_ARG; return c; }
        nrm += r->psi0[i] * r->psi0[i];
    }
    if (std::fabs(std::sqrt(nrm) - 1.0) > 1e-10) { c.status = SPINSIM_E_NORM; return c; }
    c.flags = magnus_flags(*r, c.L);
    return c;
}

// Every argument of the per-step sine/cosine series, bounded from the field's
// amplitudes:
//   the co-rotating drive phase (w_d - w_r) tau, tau < Delta_t, with
//   |w_d - w_r| <= |w_co0| + sum_p |amp_p| in the frame (w_co0 = 2 pi f_d in the lab);
//   the half phases h_j of the Lie-Trotter diagonal, |h_j| <= |z|/2 + |q|/3 with
//   |z| <= (|a| + |b|) dt (sum_p |amp_p| (+ 2 pi |B| in the lab)), |q| = |a + b| dt 2 pi |q_hz|;
//   Phi/2 <= (|a| + |b|) dt (|Om+| + |Om-|) / 2, the sum over the drive and every
//   further tone (the tones' own phasors are evaluated with the range-checked
//   series, so their phases need no bound).
// These bounds hold for every number of squarings (each divides the angles by 2^tau).
// The small-angle variant evaluates Gaussian pulses only: a request with a
// single-sine-cycle pulse takes the general variant.
bool small_angle_request(const spinsim_config& cfg, const spinsim_request& r, int64_t L)
{
    if (cfg.precision != SPINSIM_PREC_FP32_BULK || L < 1) return false;
    if (r.field.qd_on) return false;
    const MethodNodes m = method_nodes(cfg.method);
    const spinsim_field& f = r.field;
    const double dt = r.dt_out / (double)L;
    const double wabs = std::fabs(m.wa) + std::fabs(m.wb), wsum = std::fabs(m.wa + m.wb);
    const double pulse_w = pulse_weight(f);
    const bool frame = cfg.rotating_frame != 0;
    const double w_co = frame ? std::fabs(kTwoPiH * (f.drive_hz - f.bias_hz)) + pulse_w : std::fabs(kTwoPiH * f.drive_hz);
    const double co = w_co * r.dt_out;
    const double z = wabs * dt * (pulse_w + (frame ? 0.0 : kTwoPiH * std::fabs(f.bias_hz)));
    const double q = r.spin_x2 == 2 ? wsum * dt * kTwoPiH * std::fabs(f.quad_hz) : 0.0;
    // the transverse amplitude: the drive's |Om+| + |Om-| and each further tone's
    double om_perp = 0.5 * kTwoPiH * (std::fabs(f.drive_x_hz + f.drive_y_hz) + std::fabs(f.drive_x_hz - f.drive_y_hz));
    for (int j = 0; j < f.n_tones; j++)
        om_perp += 0.5 * kTwoPiH * (std::fabs(f.tone_x_hz[j] + f.tone_y_hz[j]) + std::fabs(f.tone_x_hz[j] - f.tone_y_hz[j]));
    const double half_phi = 0.5 * wabs * dt * om_perp;
    const double h = 0.5 * z + q / 3.0;
    return co <= kTinyAngleBound && h <= kTinyAngleBound && half_phi <= kTinyAngleBound;
}

// The Lie-Trotter squarings of a request (choose_tau from its field's
// amplitudes; spin-half: none, its exponential is closed-form).
int request_tau(const spinsim_config& cfg, const spinsim_request& r, int64_t K, int64_t L)
{
    if (r.spin_x2 == 1) return 0;
    const spinsim_field& f = r.field;
    const double dt = r.dt_out / (double)L;
    const double ax = kTwoPiH * f.drive_x_hz, ay = kTwoPiH * f.drive_y_hz;
    double om_perp = std::fabs(0.5 * (ax + ay)) + std::fabs(0.5 * (ax - ay));
    for (int j = 0; j < f.n_tones; j++) {
        const double tx = kTwoPiH * f.tone_x_hz[j], ty = kTwoPiH * f.tone_y_hz[j];
        om_perp += std::fabs(0.5 * (tx + ty)) + std::fabs(0.5 * (tx - ty));
    }
    const MethodNodes mn = method_nodes(cfg.method);
    return choose_tau(cfg.trotter_squares, cfg.precision, cfg.rotating_frame, mn.n_exp, mn.wa, mn.wb, dt, om_perp,
                      kTwoPiH * std::fabs(f.bias_hz), pulse_weight(f), kTwoPiH * std::fabs(f.quad_hz),
                      (double)(K > 0 ? K - 1 : 0) * (double)L);
}

int request_variant(const spinsim_config& cfg, const spinsim_request& r, int64_t K, int64_t L)
{
    if (r.field.qd_on) return kVariantSU3;
    const bool small = small_angle_request(cfg, r, L);
    const bool sine = r.field.n_pulses > 0 && (r.field.pulse_sine_mask & ((1 << r.field.n_pulses) - 1)) != 0;
    if (r.field.n_tones > 0) return small && !sine ? kVariantSmallTones : kVariantTones;
    if (!small) return kVariantGeneral;
    if (r.spin_x2 == 2 && request_tau(cfg, r, K, L) == 0) return sine ? kVariantSmallSineTau0 : kVariantSmallTau0;
    return sine ? kVariantSmallSine : kVariantSmall;
}

int precision_status(const spinsim_config& cfg, const spinsim_request& r)
{
    return r.field.qd_on && cfg.precision != SPINSIM_PREC_FP64 ? SPINSIM_E_UNSUPPORTED : SPINSIM_OK;
}

void fill_devsim(const spinsim_config& cfg, const spinsim_request& r, int64_t K, int64_t L, DevSim& d)
{
    std::memset(&d, 0, sizeof(d));
    const spinsim_field& f = r.field;
    d.K = K;
    d.L = L;
    d.seg_log2 = seg_log2_of(L);
    d.t_start = r.t_start;
    d.dt_out = r.dt_out;
    d.dt = r.dt_out / (double)L;
    d.drive_hz = f.drive_hz;
    d.drive_phase = f.drive_phase;
    const double ax = kTwoPiH * f.drive_x_hz, ay = kTwoPiH * f.drive_y_hz;
    const double om_plus = 0.5 * (ax + ay), om_minus = 0.5 * (ax - ay);
    const MethodNodes mn = method_nodes(cfg.method);
    const double wa = mn.wa, wb = mn.wb;
    d.c1 = mn.c1;
    d.c2 = mn.c2;
    d.P[0] = om_plus * wa * d.dt;
    d.P[1] = om_plus * wb * d.dt;
    d.P[2] = om_minus * wa * d.dt;
    d.P[3] = om_minus * wb * d.dt;
    d.counter_on = om_minus != 0.0 ? 1 : 0;
    d.za = wa * d.dt;
    d.zb = wb * d.dt;
    d.frame = cfg.rotating_frame ? 1 : 0;
    d.zbias = d.frame ? 0.0 : kTwoPiH * f.bias_hz * (wa + wb) * d.dt;
    if (d.frame) {
        d.w_co0 = kTwoPiH * (f.drive_hz - f.bias_hz);
        d.w_counter0 = kTwoPiH * (f.drive_hz + f.bias_hz);
        const double th = kTwoPiH * f.bias_hz * r.dt_out;
        d.exit_re = std::cos(th);
        d.exit_im = -std::sin(th);
        d.exit_half_re = std::cos(0.5 * th);
        d.exit_half_im = -std::sin(0.5 * th);
    } else {
        d.w_co0 = d.w_counter0 = kTwoPiH * f.drive_hz;
        d.exit_re = d.exit_half_re = 1.0;
        d.exit_im = d.exit_half_im = 0.0;
    }
    // further tones: Om+-_j and their rates as seen in the frame (or the lab)
    d.n_tones = f.n_tones;
    for (int j = 0; j < f.n_tones; j++) {
        const double tx = kTwoPiH * f.tone_x_hz[j], ty = kTwoPiH * f.tone_y_hz[j];
        d.tone_hz[j] = f.tone_hz[j];
        d.tone_phase[j] = f.tone_phase[j];
        d.t_om_plus[j] = 0.5 * (tx + ty);
        d.t_om_minus[j] = 0.5 * (tx - ty);
        d.t_co0[j] = kTwoPiH * (f.tone_hz[j] - (d.frame ? f.bias_hz : 0.0));
        d.t_ct0[j] = kTwoPiH * (f.tone_hz[j] + (d.frame ? f.bias_hz : 0.0));
        d.f_tom_plus[j] = (float)d.t_om_plus[j];
        d.f_tom_minus[j] = (float)d.t_om_minus[j];
    }
    // quadrupole drives: pair p turns at (p + 1) w_r in the frame
    d.qd_on = f.qd_on ? 1 : 0;
    for (int p = 0; p < 2 && d.qd_on; p++) {
        const double qx = kTwoPiH * f.qd_x_hz[p], qy = kTwoPiH * f.qd_y_hz[p];
        const double kb = d.frame ? (double)(p + 1) * f.bias_hz : 0.0;
        d.qd_hz[p] = f.qd_hz[p];
        d.qd_phase[p] = f.qd_phase[p];
        d.qd_om_plus[p] = 0.5 * (qx + qy);
        d.qd_om_minus[p] = 0.5 * (qx - qy);
        d.qd_co0[p] = kTwoPiH * (f.qd_hz[p] - kb);
        d.qd_ct0[p] = kTwoPiH * (f.qd_hz[p] + kb);
    }
    d.tau = request_tau(cfg, r, K, L);
    // quadrupole coefficient of one exponential, over 3 and 2^tau, as the bulk
    // type holds it (its rounding only reaches second order: the first-order
    // part of every U_k is replaced by the exact gq)
    const double vq = r.spin_x2 == 2 ? (wa + wb) * kTwoPiH * f.quad_hz * d.dt : 0.0;
    double qd3 = vq / 3.0 / std::ldexp(1.0, d.tau);
    if (cfg.precision == SPINSIM_PREC_FP32_BULK) qd3 = (double)(float)qd3;
    d.qd3 = qd3;
    d.om_plus = om_plus;
    d.om_minus = om_minus;
    d.W1 = mn.n_exp == 2 ? wa + wb : wa;
    d.W2 = mn.n_exp == 2 ? wa + wb : wb;
    d.gq = r.spin_x2 == 2 ? kTwoPiH * f.quad_hz * r.dt_out : 0.0;
    d.normalize_out = cfg.precision == SPINSIM_PREC_FP32_BULK ? 1 : 0;
    // Taylor tables of the node-phasor sums (direct FP64 summation)
    d.tay_ok = L <= 65536 ? 1 : 0;
    if (d.tay_ok) {
        const double Wn[2] = {d.W1, d.W2}, cn[2] = {d.c1, d.c2};
        phasor_tables(d.w_co0 * d.dt, L, Wn, cn, d.tay_co);
        phasor_tables(d.w_counter0 * d.dt, L, Wn, cn, d.tay_ct);
        for (int j = 0; j < d.n_tones; j++) {
            phasor_tables(d.t_co0[j] * d.dt, L, Wn, cn, d.t_tay_co[j]);
            if (d.t_om_minus[j] != 0.0) phasor_tables(d.t_ct0[j] * d.dt, L, Wn, cn, d.t_tay_ct[j]);
        }
    }
    // Gaussian pulses first, then the sine cycles, so the step loop handles
    // each kind in a loop of its own
    d.n_pulses = f.n_pulses;
    d.n_gauss = 0;
    int slot = 0;
    for (int pass = 0; pass < 2; pass++)
        for (int p = 0; p < f.n_pulses; p++) {
            const bool sine = (f.pulse_sine_mask >> p) & 1;
            if (sine != (pass == 1)) continue;
            d.amp[slot] = kTwoPiH * f.pulse_amp_hz[p];
            d.centre[slot] = f.pulse_centre_s[p];
            d.inv_w[slot] = 1.0 / f.pulse_width_s[p];
            slot++;
            if (!sine) d.n_gauss++;
        }
    for (int e = 0; e < 6; e++) d.psi0[e] = r.psi0[e];
    d.spin_x2 = r.spin_x2;
    for (int i = 0; i < 4; i++) d.f_ph[i] = (float)d.P[i];
    d.f_za = (float)d.za;
    d.f_zb = (float)d.zb;
    d.f_zbias = (float)d.zbias;
    d.f_qd3 = (float)d.qd3;
    d.f_dt = (float)d.dt;
    d.f_c1 = (float)d.c1;
    d.f_c2 = (float)d.c2;
    for (int p = 0; p < f.n_pulses; p++) {
        d.f_amp[p] = (float)d.amp[p];
        d.f_invw[p] = (float)d.inv_w[p];
        d.f_invwb[p] = (float)(d.inv_w[p] * kGaussBase2);
    }
}

}  // namespace spinsim
