// Host build of the kernels' per-thread arithmetic (device_math.cuh), so the
// CPU test-suite can check it against the oracle and scipy without a GPU.
#include <vector>
#include <cstdint>
#include "../paper_2204_05586_gb300/csrc/device_math.cuh"

// small_angle_request lives in csrc/params.cu, linked into this harness.

using namespace spinsim;

template <typename R>
static void full3(const Res3<R>& e, double* out)
{
    cx<R> F[3][3];
    res3_full(e, F);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            out[2 * (3 * i + j)] = (double)F[i][j].r + (i == j ? 1.0 : 0.0);
            out[2 * (3 * i + j) + 1] = (double)F[i][j].i;
        }
}

extern "C" {
// exp(-i (vx Jx + vy Jy + vz Jz + vq Q)) through the split-residual Lie-Trotter.
void hh_expm_one(double vx, double vy, double vz, double vq, int tau, int fp32, double* out)
{
    const double qd3 = vq / 3.0 / std::ldexp(1.0, tau);
    if (fp32) {
        Res3<float> e;
        expm_one_res<float>((float)vx, (float)vy, (float)vz, (float)qd3, tau, e);
        full3(e, out);
    } else {
        Res3<double> e;
        expm_one_res<double>(vx, vy, vz, qd3, tau, e);
        full3(e, out);
    }
}
// the FP32 small-angle variant (the kernels use it when the host has bounded
// every step angle by kTinyAngleBound)
void hh_expm_one_small(double vx, double vy, double vz, double vq, int tau, double* out)
{
    const float qd3 = (float)(vq / 3.0 / std::ldexp(1.0, tau));
    Res3<float> e;
    expm_one_res<float, true>((float)vx, (float)vy, (float)vz, qd3, tau, e);
    full3(e, out);
}
// the small-angle exponential at tau = 0 in closed form (expm_one_res_tau0),
// FP32 or FP64; out: the full matrix, rest: the part beyond first order
void hh_expm_one_tau0(double vx, double vy, double vz, double vq, int fp32, double* out, double* rest)
{
    if (fp32) {
        SampleCtx<float> c{};
        c.qd3 = (float)(vq / 3.0);
        c.q1 = 3.0f * c.qd3;
        tau0_constants(c);
        Res3<float> e;
        expm_one_res_tau0<float>((float)vx, (float)vy, (float)vz, c, e);
        full3(e, out);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                rest[6 * i + 2 * j] = e.m[i][j].r;
                rest[6 * i + 2 * j + 1] = e.m[i][j].i;
            }
    } else {
        SampleCtx<double> c{};
        c.qd3 = vq / 3.0;
        c.q1 = 3.0 * c.qd3;
        tau0_constants(c);
        Res3<double> e;
        expm_one_res_tau0<double>(vx, vy, vz, c, e);
        full3(e, out);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                rest[6 * i + 2 * j] = e.m[i][j].r;
                rest[6 * i + 2 * j + 1] = e.m[i][j].i;
            }
    }
}
// the same FP32 exponential through the general series, for comparison
void hh_expm_one_general32(double vx, double vy, double vz, double vq, int tau, double* out)
{
    const float qd3 = (float)(vq / 3.0 / std::ldexp(1.0, tau));
    Res3<float> e;
    expm_one_res<float, false>((float)vx, (float)vy, (float)vz, qd3, tau, e);
    full3(e, out);
}
// small-angle series in float: sin, cos, sin - x, cos - 1
void hh_tiny_sincos(double x, double* out)
{
    float s, c, sm, cm;
    small_sincos_tiny<float>((float)x, s, c);
    small_sincos_m_tiny<float>((float)x, sm, cm);
    out[0] = s; out[1] = c; out[2] = sm; out[3] = cm;
}
int hh_small_angle_request(const spinsim_config* cfg, const spinsim_request* r, int64_t L)
{
    return small_angle_request(*cfg, *r, L) ? 1 : 0;
}
double hh_tiny_angle_bound() { return kTinyAngleBound; }

// The integrate variant the host picks for a request (request_variant), and
// the squarings fill_devsim gives it.
int hh_request_variant(const spinsim_config* cfg, const spinsim_request* r, int64_t K, int64_t L, int* tau)
{
    DevSim d;
    fill_devsim(*cfg, *r, K, L, d);
    *tau = d.tau;
    return request_variant(*cfg, *r, K, L);
}

// exp(-i H) for a full su(3) H = w . (J_x, J_y, J_z, Q, D_xz, D_yz, D_x2y2, D_xy)
// (radians) through the split-residual general exponential, as a full matrix.
void hh_expm_general(const double* w, double* out)
{
    Res3<double> e;
    const double u[4] = {w[4], w[5], w[6], w[7]};
    expm_general_res<double>(w[0], w[1], w[2], w[3], u, e);
    full3(e, out);
}

// The part of exp(-i H) - I beyond -i (w_x J_x + w_y J_y + w_z J_z + w_q Q)
// (the quadrupole-drive first order and every higher order), as the
// split-residual general exponential carries it.
void hh_expm_general_rest(const double* w, double* out)
{
    Res3<double> e;
    const double u[4] = {w[4], w[5], w[6], w[7]};
    expm_general_res<double>(w[0], w[1], w[2], w[3], u, e);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            out[2 * (3 * i + j)] = e.m[i][j].r;
            out[2 * (3 * i + j) + 1] = e.m[i][j].i;
        }
}

// 1 when the branch-free series (sincos_series, sincos_m_series) give the same
// bits as small_sincos / small_sincos_m at x (|x| <= 1/16), in float or double.
int hh_series_match(double x, int fp32)
{
    if (fp32) {
        float s1, c1, s2, c2, m1, n1, m2, n2;
        small_sincos<float>((float)x, s1, c1);
        sincos_series<float>((float)x, s2, c2);
        small_sincos_m<float>((float)x, m1, n1);
        sincos_m_series<float>((float)x, m2, n2);
        return s1 == s2 && c1 == c2 && m1 == m2 && n1 == n2;
    }
    double s1, c1, s2, c2, m1, n1, m2, n2;
    small_sincos<double>(x, s1, c1);
    sincos_series<double>(x, s2, c2);
    small_sincos_m<double>(x, m1, n1);
    sincos_m_series<double>(x, m2, n2);
    return s1 == s2 && c1 == c2 && m1 == m2 && n1 == n2;
}

// The exact first-order transverse coefficients (g_x, g_y) of sample k of a
// request as the integrate epilogue forms them (fill_devsim, the FP64 sample
// context with further tones, first_order_exact), and the frame's pulse part
// gsum: out = (g_x, g_y, gsum).
void hh_first_order(const spinsim_config* cfg, const spinsim_request* r, int64_t K, int64_t L, int64_t k,
                    double* out)
{
    DevSim d;
    fill_devsim(*cfg, *r, K, L, d);
    SampleCtx<double> c;
    double beta = 0.0;
    const double gsum = make_ctx<double, 3, true>(d, k, c, beta);
    SampleExact x;
    make_exact<3, true>(d, k, beta, gsum, x);
    double gx, gy;
    first_order_exact<true>(d, x, gx, gy);
    out[0] = gx;
    out[1] = gy;
    out[2] = gsum;
}
// The chain's lane-run length and top level of a simulation of K samples.
void hh_chain_geom(int64_t K, int* run, int* top)
{
    const ChainGeom g = chain_geom(K);
    *run = g.run;
    *top = g.top;
}

// The epilogue's integer FP32 -> FP64 widening of n bit patterns.
void hh_widen_bits(const uint32_t* in, uint64_t* out, int64_t n)
{
    for (int64_t i = 0; i < n; i++) out[i] = widen_bits(in[i]);
}
// The fractional drive cycles f (t0 + m dt) (drive_cycles_frac).
double hh_drive_cycles_frac(double f, double t0, double dt, int64_t m) { return drive_cycles_frac(f, t0, dt, m); }

// The FP64 phasor e^{i beta_k} of interval k of a request's drive (tone = -1)
// or of its further tone `tone`, from the two-level tables the integrate
// epilogue reads (all of the request's tables built here on the host by
// sim_phasor_entry, read by drive_phasor_tab / tone_phasor_tab; table = 1), or
// from the phase and a sine and cosine (table = 0): out = (re, im).
void hh_phasor(const spinsim_config* cfg, const spinsim_request* r, int64_t K, int64_t L, int64_t k, int tone,
               int table, double* out)
{
    DevSim d;
    fill_devsim(*cfg, *r, K, L, d);
    cx<double> v;
    if (table) {
        const int64_t n = phasor_entries(K, d.n_tones);
        std::vector<double> tab((size_t)(2 * n));
        for (int64_t e = 0; e < n; e++) {
            const cx<double> x = sim_phasor_entry(d, e);
            tab[(size_t)(2 * e)] = x.r;
            tab[(size_t)(2 * e + 1)] = x.i;
        }
        d.eb_tab = tab.data();
        v = tone < 0 ? drive_phasor_tab(d, k) : tone_phasor_tab(d, tone, k);
    } else {
        const double b = tone < 0 ? drive_phase_at(d, k)
                                  : tone_phase_at(d.tone_hz[tone], d.tone_phase[tone], d.t_start + (double)(k - 1) * d.dt_out);
        const SinCos<double> e = sincos_cold(b);
        v = cmk(e.c, e.s);
    }
    out[0] = v.r;
    out[1] = v.i;
}

// rest part only (U - I - F(v)) in double
void hh_expm_one_rest(double vx, double vy, double vz, double vq, int tau, double* out)
{
    Res3<double> e;
    expm_one_res<double>(vx, vy, vz, vq / 3.0 / std::ldexp(1.0, tau), tau, e);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) { out[2 * (3 * i + j)] = e.m[i][j].r; out[2 * (3 * i + j) + 1] = e.m[i][j].i; }
}
void hh_expm_half(double vx, double vy, double vz, int fp32, double* out)
{
    double a_r, a_i, b_r, b_i;
    if (fp32) {
        Res2<float> e; cx<float> a, b;
        expm_half_res<float>((float)vx, (float)vy, (float)vz, e);
        res2_full(e, a, b);
        a_r = a.r; a_i = a.i; b_r = b.r; b_i = b.i;
    } else {
        Res2<double> e; cx<double> a, b;
        expm_half_res<double>(vx, vy, vz, e);
        res2_full(e, a, b);
        a_r = a.r; a_i = a.i; b_r = b.r; b_i = b.i;
    }
    // [[alpha, -conj(beta)], [beta, conj(alpha)]]
    double al_r = 1.0 + a_r, al_i = a_i;
    double m[8] = {al_r, al_i, -b_r, b_i, b_r, b_i, al_r, -al_i};
    for (int i = 0; i < 8; i++) out[i] = m[i];
}
// product of two split residuals given as exponent vectors: exp(-i vB.A) exp(-i vA.A)
void hh_product_one(const double* vA, const double* vB, int tau, double* out)
{
    Res3<double> a, b, c;
    expm_one_res<double>(vA[0], vA[1], vA[2], vA[3] / 3.0 / std::ldexp(1.0, tau), tau, a);
    expm_one_res<double>(vB[0], vB[1], vB[2], vB[3] / 3.0 / std::ldexp(1.0, tau), tau, b);
    res3_mul(b, a, c);
    full3(c, out);
}
void hh_product_half(const double* vA, const double* vB, double* out)
{
    Res2<double> a, b, c;
    expm_half_res<double>(vA[0], vA[1], vA[2], a);
    expm_half_res<double>(vB[0], vB[1], vB[2], b);
    res2_mul(b, a, c);
    cx<double> al, be;
    res2_full(c, al, be);
    double m[8] = {1.0 + al.r, al.i, -be.r, be.i, be.r, be.i, 1.0 + al.r, -al.i};
    for (int i = 0; i < 8; i++) out[i] = m[i];
}
void hh_node_phasor_sum(double th, int64_t L, double W1, double c1, double W2, double c2, double* out)
{
    cx<double> z = node_phasor_sum(th, L, W1, c1, W2, c2);
    out[0] = z.r;
    out[1] = z.i;
}
void hh_small_sincos_m(double x, int fp32, double* out)
{
    if (fp32) { float s, c; small_sincos_m<float>((float)x, s, c); out[0] = s; out[1] = c; }
    else { double s, c; small_sincos_m<double>(x, s, c); out[0] = s; out[1] = c; }
}
// automatic Lie-Trotter squarings of a request (host-side rule)
int hh_choose_tau(int cfg_tau, int precision, int frame, int n_exp, double wa, double wb, double dt, double om_perp,
                  double bias_w, double pulse_w, double q_w, double steps)
{
    return choose_tau(cfg_tau, precision, frame, n_exp, wa, wb, dt, om_perp, bias_w, pulse_w, q_w, steps);
}
}
