/*
 * spinsim_oracle.c -- plain FP64 CPU reference of the Spinsim integration method
 * (Tritt et al., "Spinsim: a GPU optimized python package for simulating
 * spin-half and spin-one quantum systems", arXiv 2204.05586).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant generator with the CUDA implementation, and the product
 * path never calls it.
 *
 * Everything is written the slow, obvious way: double-precision complex
 * arithmetic from <complex.h>, libm transcendental functions, full N x N
 * matrices with triple loops, and the steps in the order the paper gives them:
 *
 *   field functions            Sec. 1.2.1 (H = sum_j w_j(t) A_j)
 *   rotating frame             Sec. 1.2.5 (R(t) = exp(i w_r J_z t), Eq. exit_rotating_frame)
 *   CF4 step                   Sec. 1.2.2 (Eqs. cf4_sample_1, cf4_sample_2, cf4_implementation)
 *   spin-half exponential      Sec. 1.2.3 (analytic SU(2) form)
 *   spin-one exponential       Sec. 1.2.3 (Eqs. lie_trotter, lie_trotter_4,
 *                              residual squaring s = (a + 2I) a, expm1 diagonal)
 *   full su(3) spin-one        Sec. 1.2.1 (an arbitrary point in su(3): the
 *                              exponential series with scaling and squaring)
 *   sample operators U_k       Sec. 1.2.4 (U_k = u_{L-1} ... u_0, delta_t = Delta_t / L)
 *   state chain                Sec. 1.2.4 (Eq. integration_compilation, psi_k = U_k psi_{k-1})
 *   spin projection            Sec. 1.2.1 (<J> = psi^dagger J psi)
 *   Euler sampling integrators Sec. 1.3.1 (midpoint and Heun "sampling" methods)
 *
 * Readings taken where the paper is garbled or silent (each is checked by a
 * pin test against something other than this file):
 *   - Eq. lie_trotter_4, centre entry: the printed exp(i4q) is read as
 *     exp(+i 2q/3), the value e^{-iD/2} e^{-i Phi J_phi} e^{-iD/2} has there.
 *   - Eq. lie_trotter_4, entry (m=+1, m'=-1): the printed exp(+iq/6) factor is
 *     read as exp(-iq/6) (the product above again).
 *   - z, q and Phi of the Lie-Trotter step carry the factor delta_t: the step
 *     exponentiates -i H delta_t, so z = w_z delta_t / n (likewise q, Phi).
 *   - The spin-half closed form is the textbook SU(2) identity
 *     exp(-i v.sigma/2) = cos(|v|/2) I - i sin(|v|/2) (v/|v|).sigma.
 *   - The rotating frame angle is measured from the start of each sample
 *     interval, so that leaving the frame is exp(-i w_r Delta_t J_z).
 *   - w_r is the full z field (bias plus pulses) at the interval midpoint.
 *   - psi_0 is the initial state at t_start; there are K = (t_end-t_start)/Delta_t
 *     samples and none at t_end.
 *   - The quadratic shift multiplies the traceless Q = diag(1,-2,1)/3.
 *   - Basis order is m = +j ... -j.
 *   - The four operators that complete su(3) (the paper's U_1, U_2, V_1, V_2
 *     come from a basis it cites but does not print) are taken as the
 *     symmetric products D_xz, D_yz, D_x2y2, D_xy of the spin matrices.
 *
 * Build: gcc -O2 -fPIC -shared -std=c11 spinsim_oracle.c -o libspinsim_oracle.so -lm
 * (no fast-math: every transcendental is the correctly-behaved libm one).
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

typedef double complex cplx;

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* Field model: a fixed parameterised family of field functions w_j(t)       */
/* (Sec. 1.2.1 and Sec. 1.2.7 -- the paper's user-supplied field functions,  */
/* here a bias, a sinusoidal drive of chosen polarisation, a quadratic shift */
/* and up to four pulses on the z field, each a Gaussian or a single cycle   */
/* of a sine wave -- the "sinp" signal pulse of the paper's benchmark field, */
/* Eq. neural_pulse, Sec. 1.3.1).                                            */
/* ------------------------------------------------------------------------- */
#define OR_MAX_PULSES 4
#define OR_MAX_TONES 3   /* drive tones besides the first (the paper's "arbitrary number of tones") */

typedef struct {
    double bias_hz;      /* w_z constant part: 2 pi bias_hz                         */
    double drive_x_hz;   /* w_x = 2 pi drive_x_hz cos(2 pi drive_hz t + drive_phase) */
    double drive_y_hz;   /* w_y = 2 pi drive_y_hz sin(2 pi drive_hz t + drive_phase) */
    double drive_hz;     /* drive frequency                                         */
    double drive_phase;  /* drive phase at t = 0, radians                           */
    double quad_hz;      /* w_q = 2 pi quad_hz (spin-one quadrupole term)           */
    int32_t n_pulses;    /* number of z pulses used, 0..4                           */
    int32_t pulse_sine_mask; /* bit p set: pulse p is a single sine cycle           */
    /* Gaussian pulse p:   w_z += 2 pi A exp(-(t-c)^2 / (2 w^2)), w the standard deviation;
     * sine-cycle pulse p: w_z += 2 pi A sin(2 pi (t-c)/w) for c <= t < c + w, else 0
     * (c = pulse_centre_s[p] is the start t_p of the cycle, w its period).         */
    double pulse_amp_hz[OR_MAX_PULSES];
    double pulse_centre_s[OR_MAX_PULSES];
    double pulse_width_s[OR_MAX_PULSES];
    /* further drive tones j < n_tones, each like the first:
     * w_x += 2 pi tone_x_hz[j] cos(2 pi tone_hz[j] t + tone_phase[j]),
     * w_y += 2 pi tone_y_hz[j] sin(2 pi tone_hz[j] t + tone_phase[j])                   */
    int32_t n_tones;
    int32_t pad2_;
    double tone_x_hz[OR_MAX_TONES];
    double tone_y_hz[OR_MAX_TONES];
    double tone_hz[OR_MAX_TONES];
    double tone_phase[OR_MAX_TONES];
    /* quadrupole drives (spin-one, qd_on = 1), completing su(3) with the four
     * symmetric products D_xz = {J_x, J_z}, D_yz = {J_y, J_z},
     * D_x2y2 = J_x^2 - J_y^2, D_xy = {J_x, J_y} ({A, B} = AB + BA):
     *   w_xz  = 2 pi qd_x_hz[0] cos(ph_0),  w_yz = 2 pi qd_y_hz[0] sin(ph_0),
     *   w_x2y2 = 2 pi qd_x_hz[1] cos(ph_1), w_xy = 2 pi qd_y_hz[1] sin(ph_1),
     * ph_p = 2 pi qd_hz[p] t + qd_phase[p].                                     */
    int32_t qd_on;
    int32_t pad3_;
    double qd_x_hz[2];
    double qd_y_hz[2];
    double qd_hz[2];
    double qd_phase[2];
} oracle_field;

/* Field functions (w_x, w_y, w_z, w_q) at time t, in rad/s. */
void oracle_field_sample(const oracle_field* f, double t, double w[4])
{
    double phase = 2.0 * OR_PI * f->drive_hz * t + f->drive_phase;
    double bz = f->bias_hz;
    for (int p = 0; p < f->n_pulses && p < OR_MAX_PULSES; p++) {
        double d = t - f->pulse_centre_s[p];
        double wd = f->pulse_width_s[p];
        if ((f->pulse_sine_mask >> p) & 1) {
            double cyc = d / wd;   /* cycles since the start of the pulse */
            if (cyc >= 0.0 && cyc < 1.0) bz += f->pulse_amp_hz[p] * sin(2.0 * OR_PI * cyc);
        } else {
            bz += f->pulse_amp_hz[p] * exp(-(d * d) / (2.0 * wd * wd));
        }
    }
    w[0] = 2.0 * OR_PI * f->drive_x_hz * cos(phase);
    w[1] = 2.0 * OR_PI * f->drive_y_hz * sin(phase);
    for (int j = 0; j < f->n_tones && j < OR_MAX_TONES; j++) {
        double ph = 2.0 * OR_PI * f->tone_hz[j] * t + f->tone_phase[j];
        w[0] += 2.0 * OR_PI * f->tone_x_hz[j] * cos(ph);
        w[1] += 2.0 * OR_PI * f->tone_y_hz[j] * sin(ph);
    }
    w[2] = 2.0 * OR_PI * bz;
    w[3] = 2.0 * OR_PI * f->quad_hz;
}

/* Quadrupole-drive coefficients (w_xz, w_yz, w_x2y2, w_xy) at time t, in rad/s. */
void oracle_field_sample_quad(const oracle_field* f, double t, double u[4])
{
    for (int p = 0; p < 2; p++) {
        double ph = 2.0 * OR_PI * f->qd_hz[p] * t + f->qd_phase[p];
        u[2 * p] = f->qd_on ? 2.0 * OR_PI * f->qd_x_hz[p] * cos(ph) : 0.0;
        u[2 * p + 1] = f->qd_on ? 2.0 * OR_PI * f->qd_y_hz[p] * sin(ph) : 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* Small dense complex matrix helpers (N = 2 or 3, row-major [N][3]).         */
/* ------------------------------------------------------------------------- */
static void mat_identity(int n, cplx a[3][3])
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            a[i][j] = (i == j && i < n) ? 1.0 : 0.0;
}

/* c = a b (c may alias neither a nor b) */
static void mat_mul(int n, cplx a[3][3], cplx b[3][3], cplx c[3][3])
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            cplx s = 0.0;
            for (int k = 0; k < n; k++) s += a[i][k] * b[k][j];
            c[i][j] = s;
        }
}

static void mat_copy(cplx dst[3][3], cplx src[3][3])
{
    memcpy(dst, src, sizeof(cplx) * 9);
}

/* ------------------------------------------------------------------------- */
/* Spin-half exponential (Sec. 1.2.3: analytic in w_x, w_y, w_z).            */
/* exp(-i (w_x J_x + w_y J_y + w_z J_z) dt) with J = sigma / 2.              */
/* ------------------------------------------------------------------------- */
void oracle_expm_spin_half(double wx, double wy, double wz, double dt, double* out /* [2][2] re,im */)
{
    double vx = wx * dt, vy = wy * dt, vz = wz * dt;
    double theta = sqrt(vx * vx + vy * vy + vz * vz);
    double c = cos(theta / 2.0);
    double s; /* sin(theta/2) / theta */
    if (theta > 1e-6)
        s = sin(theta / 2.0) / theta;
    else
        s = 0.5 - theta * theta / 48.0;
    /* cos(theta/2) I - i sin(theta/2) (v/theta).sigma */
    cplx u00 = c - I * s * vz;
    cplx u01 = -I * s * (vx - I * vy);
    cplx u10 = -I * s * (vx + I * vy);
    cplx u11 = c + I * s * vz;
    cplx u[4] = {u00, u01, u10, u11};
    for (int i = 0; i < 4; i++) {
        out[2 * i] = creal(u[i]);
        out[2 * i + 1] = cimag(u[i]);
    }
}

/* ------------------------------------------------------------------------- */
/* Spin-one Lie-Trotter exponential (Sec. 1.2.3).                             */
/* ------------------------------------------------------------------------- */

/* The leapfrog Lie-Trotter factor T of Eq. lie_trotter_4, for n = 2^tau:
 *   T = exp(-i D/2) exp(-i Phi J_phi) exp(-i D/2),  D = z J_z + q Q,
 *   z = w_z dt / n, q = w_q dt / n, Phi = sqrt(w_x^2 + w_y^2) dt / n,
 *   phi = atan2(w_y, w_x).
 * Written element by element as the paper prints it (with the two readings
 * stated in the file header). */
static void trotter_T(double wx, double wy, double wz, double wq, double dt, int tau,
                      cplx T[3][3], double* z_out, double* q_out, double* Phi_out, cplx* eiphi_out)
{
    double n = ldexp(1.0, tau);
    double z = wz * dt / n;
    double q = wq * dt / n;
    double wperp = hypot(wx, wy);
    double Phi = wperp * dt / n;
    cplx eiphi = (wperp > 0.0) ? cexp(I * atan2(wy, wx)) : 1.0;
    cplx emiphi = conj(eiphi);
    double C = cos(Phi / 2.0), S = sin(Phi / 2.0);
    cplx ez = cexp(-I * z / 2.0);        /* e^{-iz/2} */
    cplx eq6 = cexp(I * q / 6.0);        /* e^{+iq/6} */
    double r2 = 1.0 / sqrt(2.0);

    T[0][0] = (C * ez * conj(eq6)) * (C * ez * conj(eq6));
    T[0][1] = -I * r2 * sin(Phi) * eq6 * ez * emiphi;
    T[0][2] = -(S * conj(eq6) * emiphi) * (S * conj(eq6) * emiphi);
    T[1][0] = -I * r2 * sin(Phi) * eq6 * ez * eiphi;
    T[1][1] = cos(Phi) * cexp(I * 2.0 * q / 3.0);
    T[1][2] = -I * r2 * sin(Phi) * eq6 * conj(ez) * emiphi;
    T[2][0] = -(S * conj(eq6) * eiphi) * (S * conj(eq6) * eiphi);
    T[2][1] = -I * r2 * sin(Phi) * eq6 * conj(ez) * eiphi;
    T[2][2] = (C * conj(ez) * conj(eq6)) * (C * conj(ez) * conj(eq6));

    if (z_out) *z_out = z;
    if (q_out) *q_out = q;
    if (Phi_out) *Phi_out = Phi;
    if (eiphi_out) *eiphi_out = eiphi;
}

/* expm1(i x) = e^{ix} - 1 = -2 sin^2(x/2) + i sin(x), free of cancellation. */
static cplx expm1_i(double x)
{
    double h = sin(x / 2.0);
    return -2.0 * h * h + I * sin(x);
}

/* Exported for pin tests: the full T matrix (out[3][3] re,im). */
void oracle_trotter_T(double wx, double wy, double wz, double wq, double dt, int tau, double* out)
{
    cplx T[3][3];
    trotter_T(wx, wy, wz, wq, dt, tau, T, NULL, NULL, NULL, NULL);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            out[2 * (3 * i + j)] = creal(T[i][j]);
            out[2 * (3 * i + j) + 1] = cimag(T[i][j]);
        }
}

/* T - I built without cancellation: the off-diagonal entries are those of T;
 * each diagonal entry r e^{i theta} - 1 is rewritten with expm1 (Sec. 1.2.3):
 *   cos^2(Phi/2) e^{i th} - 1 = expm1(i th) - sin^2(Phi/2) e^{i th}
 *   cos(Phi)     e^{i th} - 1 = expm1(i th) - 2 sin^2(Phi/2) e^{i th}      */
static void trotter_T_minus_I(double wx, double wy, double wz, double wq, double dt, int tau, cplx a[3][3])
{
    double z, q, Phi;
    cplx eiphi;
    trotter_T(wx, wy, wz, wq, dt, tau, a, &z, &q, &Phi, &eiphi);
    double S = sin(Phi / 2.0);
    double th0 = -(z + q / 3.0);   /* phase of T[0][0]: (e^{-iz/2} e^{-iq/6})^2  */
    double th1 = 2.0 * q / 3.0;    /* phase of T[1][1]                            */
    double th2 = z - q / 3.0;      /* phase of T[2][2]: (e^{+iz/2} e^{-iq/6})^2   */
    a[0][0] = expm1_i(th0) - S * S * cexp(I * th0);
    a[1][1] = expm1_i(th1) - 2.0 * S * S * cexp(I * th1);
    a[2][2] = expm1_i(th2) - S * S * cexp(I * th2);
}

/* exp(-i (w_x J_x + w_y J_y + w_z J_z + w_q Q) dt) ~= T^n, n = 2^tau, by
 * residual squaring: with A = I + a, A^2 = I + (a + 2I) a (Sec. 1.2.3). */
static void expm_spin_one(double wx, double wy, double wz, double wq, double dt, int tau, cplx E[3][3])
{
    cplx a[3][3], ap2[3][3], s[3][3];
    trotter_T_minus_I(wx, wy, wz, wq, dt, tau, a);
    for (int step = 0; step < tau; step++) {
        mat_copy(ap2, a);
        for (int i = 0; i < 3; i++) ap2[i][i] += 2.0;
        mat_mul(3, ap2, a, s);
        mat_copy(a, s);
    }
    mat_copy(E, a);
    for (int i = 0; i < 3; i++) E[i][i] += 1.0;
}

void oracle_expm_spin_one(double wx, double wy, double wz, double wq, double dt, int tau, double* out)
{
    cplx E[3][3];
    expm_spin_one(wx, wy, wz, wq, dt, tau, E);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            out[2 * (3 * i + j)] = creal(E[i][j]);
            out[2 * (3 * i + j) + 1] = cimag(E[i][j]);
        }
}

/* Residual a = T^n - I of the squaring loop (for the cancellation pin test). */
void oracle_expm_spin_one_residual(double wx, double wy, double wz, double wq, double dt, int tau, double* out)
{
    cplx a[3][3], ap2[3][3], s[3][3];
    trotter_T_minus_I(wx, wy, wz, wq, dt, tau, a);
    for (int step = 0; step < tau; step++) {
        mat_copy(ap2, a);
        for (int i = 0; i < 3; i++) ap2[i][i] += 2.0;
        mat_mul(3, ap2, a, s);
        mat_copy(a, s);
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            out[2 * (3 * i + j)] = creal(a[i][j]);
            out[2 * (3 * i + j) + 1] = cimag(a[i][j]);
        }
}

/* ------------------------------------------------------------------------- */
/* Full su(3) spin-one Hamiltonians (Sec. 1.2.1: "an arbitrary point in       */
/* su(3)").  Basis: J_x, J_y, J_z, Q and the symmetric products D_xz, D_yz,   */
/* D_x2y2, D_xy of the spin matrices, formed here by matrix products.          */
/* ------------------------------------------------------------------------- */
static void su3_basis(cplx G[8][3][3])
{
    cplx J[3][3][3];
    memset(J, 0, sizeof(J));
    double r = 1.0 / sqrt(2.0);
    J[0][0][1] = r; J[0][1][0] = r; J[0][1][2] = r; J[0][2][1] = r;
    J[1][1][0] = I * r; J[1][0][1] = -I * r; J[1][2][1] = I * r; J[1][1][2] = -I * r;
    J[2][0][0] = 1.0; J[2][2][2] = -1.0;
    memset(G, 0, 8 * sizeof(G[0]));
    for (int a = 0; a < 3; a++) mat_copy(G[a], J[a]);
    G[3][0][0] = 1.0 / 3.0; G[3][1][1] = -2.0 / 3.0; G[3][2][2] = 1.0 / 3.0;
    cplx xz[3][3], zx[3][3], yz[3][3], zy[3][3], xx[3][3], yy[3][3], xy[3][3], yx[3][3];
    mat_mul(3, J[0], J[2], xz); mat_mul(3, J[2], J[0], zx);
    mat_mul(3, J[1], J[2], yz); mat_mul(3, J[2], J[1], zy);
    mat_mul(3, J[0], J[0], xx); mat_mul(3, J[1], J[1], yy);
    mat_mul(3, J[0], J[1], xy); mat_mul(3, J[1], J[0], yx);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            G[4][i][j] = xz[i][j] + zx[i][j];
            G[5][i][j] = yz[i][j] + zy[i][j];
            G[6][i][j] = xx[i][j] - yy[i][j];
            G[7][i][j] = xy[i][j] + yx[i][j];
        }
}

/* exp(-i H dt) for H = sum_j w_j G_j (spin-one, 8 coefficients), by the series
 * sum_k A^k / k! of A = -i H dt / 2^s (s halvings until the row-sum norm is at
 * most 1/2, 30 terms) followed by s squarings. */
static void expm_general(const double w[8], double dt, cplx E[3][3])
{
    cplx G[8][3][3], A[3][3];
    su3_basis(G);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx h = 0.0;
            for (int a = 0; a < 8; a++) h += w[a] * G[a][i][j];
            A[i][j] = -I * h * dt;
        }
    double norm = 0.0;
    for (int i = 0; i < 3; i++) {
        double row = 0.0;
        for (int j = 0; j < 3; j++) row += cabs(A[i][j]);
        if (row > norm) norm = row;
    }
    int s = 0;
    while (norm > 0.5) { norm *= 0.5; s++; }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) A[i][j] = ldexp(1.0, -s) * A[i][j];
    cplx term[3][3], tmp[3][3];
    mat_identity(3, E);
    mat_identity(3, term);
    for (int k = 1; k <= 30; k++) {
        mat_mul(3, term, A, tmp);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                term[i][j] = tmp[i][j] / (double)k;
                E[i][j] += term[i][j];
            }
    }
    for (int q = 0; q < s; q++) {
        mat_mul(3, E, E, tmp);
        mat_copy(E, tmp);
    }
}

void oracle_expm_general(const double w[8], double dt, double* out /* [3][3] re,im */)
{
    cplx E[3][3];
    expm_general(w, dt, E);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            out[2 * (3 * i + j)] = creal(E[i][j]);
            out[2 * (3 * i + j) + 1] = cimag(E[i][j]);
        }
}

/* One exponential exp(-i H dt) for H = w.A in the chosen spin (w: the 4
 * coefficients of J_x, J_y, J_z, Q, then with `quad` the 4 of the quadrupole
 * drives). */
static void expm_field(int spin_x2, const double w[8], double dt, int tau, int quad, cplx E[3][3])
{
    if (spin_x2 == 2 && quad) {
        expm_general(w, dt, E);
        return;
    }
    if (spin_x2 == 1) {
        double u[8];
        oracle_expm_spin_half(w[0], w[1], w[2], dt, u);
        mat_identity(3, E);
        E[0][0] = u[0] + I * u[1];
        E[0][1] = u[2] + I * u[3];
        E[1][0] = u[4] + I * u[5];
        E[1][1] = u[6] + I * u[7];
        E[2][2] = 0.0;
    } else {
        expm_spin_one(w[0], w[1], w[2], w[3], dt, tau, E);
    }
}

/* ------------------------------------------------------------------------- */
/* Rotating frame (Sec. 1.2.5).                                               */
/* R(t) = exp(i w_r J_z t) with t measured from the start of the interval;    */
/* H_r = R (w_x J_x + w_y J_y) R^dagger + (w_z - w_r) J_z + w_q Q, which has  */
/* coefficients  w_x' = w_x cos a + w_y sin a,  w_y' = -w_x sin a + w_y cos a, */
/* w_z' = w_z - w_r,  w_q' = w_q,  with a = w_r t.                            */
/* ------------------------------------------------------------------------- */
/* The quadrupole drives transform under R as well: the pair (D_xz, D_yz)   */
/* connects m and m -+ 1 and turns by a like (J_x, J_y); the pair            */
/* (D_x2y2, D_xy) connects m = +1 and -1 and turns by 2a.                     */
static void field_in_frame(const oracle_field* f, double t, double t_ref, double w_r, double w[8])
{
    oracle_field_sample(f, t, w);
    oracle_field_sample_quad(f, t, w + 4);
    double a = w_r * (t - t_ref);
    double wx = w[0], wy = w[1];
    w[0] = wx * cos(a) + wy * sin(a);
    w[1] = -wx * sin(a) + wy * cos(a);
    w[2] = w[2] - w_r;
    double u0 = w[4], u1 = w[5], u2 = w[6], u3 = w[7];
    w[4] = u0 * cos(a) + u1 * sin(a);
    w[5] = -u0 * sin(a) + u1 * cos(a);
    w[6] = u2 * cos(2.0 * a) + u3 * sin(2.0 * a);
    w[7] = -u2 * sin(2.0 * a) + u3 * cos(2.0 * a);
}

/* Integration methods: 0 = CF4 (Sec. 1.2.2), 1 = midpoint Euler sampling,
 * 2 = Heun-Euler sampling (Sec. 1.3.1). */
#define OR_METHOD_CF4 0
#define OR_METHOD_MIDPOINT 1
#define OR_METHOD_HEUN 2

/* One integration step u(t + dt, t) in the frame (t_ref, w_r). */
static void integration_step(int spin_x2, int method, const oracle_field* f, double t, double dt,
                             double t_ref, double w_r, int tau, cplx u[3][3])
{
    int n = spin_x2 == 1 ? 2 : 3;
    if (method == OR_METHOD_CF4) {
        /* Gauss-Legendre nodes and weights of Eqs. cf4_sample_1, cf4_sample_2 */
        double r3 = sqrt(3.0);
        double t1 = t + 0.5 * (1.0 - 1.0 / r3) * dt;
        double t2 = t + 0.5 * (1.0 + 1.0 / r3) * dt;
        double wa = (3.0 + 2.0 * r3) / 12.0;
        double wb = (3.0 - 2.0 * r3) / 12.0;
        double h1[8], h2[8], hb1[8], hb2[8];
        field_in_frame(f, t1, t_ref, w_r, h1);
        field_in_frame(f, t2, t_ref, w_r, h2);
        for (int j = 0; j < 8; j++) {
            hb1[j] = wa * h1[j] + wb * h2[j];
            hb2[j] = wb * h1[j] + wa * h2[j];
        }
        /* Eq. cf4_implementation: u = exp(-i Hbar_2 dt) exp(-i Hbar_1 dt) */
        cplx E1[3][3], E2[3][3];
        expm_field(spin_x2, hb1, dt, tau, f->qd_on, E1);
        expm_field(spin_x2, hb2, dt, tau, f->qd_on, E2);
        mat_identity(3, u);
        mat_mul(n, E2, E1, u);
    } else if (method == OR_METHOD_MIDPOINT) {
        double h[8];
        field_in_frame(f, t + 0.5 * dt, t_ref, w_r, h);
        expm_field(spin_x2, h, dt, tau, f->qd_on, u);
    } else {
        double h0[8], h1[8], hm[8];
        field_in_frame(f, t, t_ref, w_r, h0);
        field_in_frame(f, t + dt, t_ref, w_r, h1);
        for (int j = 0; j < 8; j++) hm[j] = 0.5 * (h0[j] + h1[j]);
        expm_field(spin_x2, hm, dt, tau, f->qd_on, u);
    }
}

/* ------------------------------------------------------------------------- */
/* Sample operators U_k (Sec. 1.2.4, 1.2.5, 1.2.6).                          */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t spin_x2;        /* 1 spin-half, 2 spin-one */
    int32_t method;         /* OR_METHOD_* */
    int32_t rotating_frame; /* 0 lab frame, 1 dynamic rotating frame */
    int32_t tau;            /* Lie-Trotter squarings, n = 2^tau */
    double t_start;
    double dt_out;          /* Delta_t, output step */
    int64_t K;              /* number of output samples */
    int64_t L;              /* integration steps per sample */
} oracle_plan;

/* Output counts: K = round((t_end - t_start)/Delta_t), L = round(Delta_t/delta_t).
 * Returns 0 on success, -1 when either ratio is not an integer to 1e-9. */
int oracle_counts(double t_start, double t_end, double dt, double dt_out, int64_t* K, int64_t* L)
{
    if (!(dt > 0.0) || !(dt_out > 0.0) || !(t_end >= t_start)) return -1;
    double rk = (t_end - t_start) / dt_out;
    double rl = dt_out / dt;
    double k = floor(rk + 0.5), l = floor(rl + 0.5);
    if (fabs(rk - k) > 1e-9 * fmax(1.0, rk)) return -1;
    if (fabs(rl - l) > 1e-9 * fmax(1.0, rl) || l < 1.0) return -1;
    *K = (int64_t)k;
    *L = (int64_t)l;
    return 0;
}

/* Frame rate of sample interval k (Sec. 1.2.5): w_r = w_z(t_{k-1} + Delta_t/2),
 * or 0 in the lab frame. */
double oracle_frame_rate(const oracle_plan* p, const oracle_field* f, int64_t k)
{
    if (!p->rotating_frame) return 0.0;
    double t_prev = p->t_start + (double)(k - 1) * p->dt_out;
    double wm[4];
    oracle_field_sample(f, t_prev + 0.5 * p->dt_out, wm);
    return wm[2];
}

/* U_k = U(t_k, t_{k-1}) for 1 <= k < K, written as [N][N] re,im. */
static void sample_operator(const oracle_plan* p, const oracle_field* f, int64_t k, cplx U[3][3])
{
    int n = p->spin_x2 == 1 ? 2 : 3;
    double t_prev = p->t_start + (double)(k - 1) * p->dt_out;
    double dt = p->dt_out / (double)p->L;   /* delta_t = Delta_t / L */
    double w_r = oracle_frame_rate(p, f, k);
    /* U^r <- u_l U^r, starting from the identity (premultiplication) */
    cplx Ur[3][3], u[3][3], tmp[3][3];
    mat_identity(3, Ur);
    for (int64_t l = 0; l < p->L; l++) {
        double t = t_prev + (double)l * dt;
        integration_step(p->spin_x2, p->method, f, t, dt, t_prev, w_r, p->tau, u);
        mat_mul(n, u, Ur, tmp);
        mat_copy(Ur, tmp);
    }
    /* Eq. exit_rotating_frame: U_k = R(-Delta_t) U^r = exp(-i w_r Delta_t J_z) U^r */
    double m_half[2] = {0.5, -0.5};
    double m_one[3] = {1.0, 0.0, -1.0};
    for (int i = 0; i < n; i++) {
        double m = (n == 2) ? m_half[i] : m_one[i];
        cplx ph = cexp(-I * m * w_r * p->dt_out);
        for (int j = 0; j < n; j++) U[i][j] = ph * Ur[i][j];
    }
}

static void store_matrix(int n, cplx U[3][3], double* out)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            out[2 * (n * i + j)] = creal(U[i][j]);
            out[2 * (n * i + j) + 1] = cimag(U[i][j]);
        }
}

/* U_k for k in [k0, k1) into ops[(k - k0)][N][N] re,im.  U_0 is defined as
 * the identity (psi_0 is the initial state itself). */
int oracle_sample_operators(const oracle_plan* p, const oracle_field* f, int64_t k0, int64_t k1, double* ops)
{
    if (p->spin_x2 != 1 && p->spin_x2 != 2) return -1;
    int n = p->spin_x2 == 1 ? 2 : 3;
    for (int64_t k = k0; k < k1; k++) {
        cplx U[3][3];
        if (k == 0)
            mat_identity(3, U);
        else
            sample_operator(p, f, k, U);
        store_matrix(n, U, ops + (size_t)(k - k0) * 2 * n * n);
    }
    return 0;
}

/* Expected spin projection <J_a> = psi^dagger J_a psi (Sec. 1.2.1). */
static void spin_projection(int n, const cplx* psi, double out[3])
{
    cplx J[3][3][3];
    memset(J, 0, sizeof(J));
    if (n == 2) {
        J[0][0][1] = 0.5;       J[0][1][0] = 0.5;           /* sigma_x / 2 */
        J[1][0][1] = -0.5 * I;  J[1][1][0] = 0.5 * I;       /* sigma_y / 2 */
        J[2][0][0] = 0.5;       J[2][1][1] = -0.5;          /* sigma_z / 2 */
    } else {
        double r = 1.0 / sqrt(2.0);
        J[0][0][1] = r; J[0][1][0] = r; J[0][1][2] = r; J[0][2][1] = r;
        J[1][0][1] = -I * r; J[1][1][0] = I * r; J[1][1][2] = -I * r; J[1][2][1] = I * r;
        J[2][0][0] = 1.0; J[2][2][2] = -1.0;
    }
    for (int a = 0; a < 3; a++) {
        cplx s = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) s += conj(psi[i]) * J[a][i][j] * psi[j];
        out[a] = creal(s);
    }
}

/* Chain psi_k = U_k psi_{k-1} (Eq. integration_compilation), sequentially,
 * from given sample operators ops[K][N][N] (ops[0] applied to psi0 gives
 * psi_0).  states: [K][N] re,im; spin: [K][3] (either may be NULL). */
int oracle_chain(int32_t spin_x2, int64_t K, const double* ops, const double* psi0, double* states, double* spin)
{
    if (spin_x2 != 1 && spin_x2 != 2) return -1;
    int n = spin_x2 == 1 ? 2 : 3;
    cplx psi[3], nxt[3];
    for (int i = 0; i < n; i++) psi[i] = psi0[2 * i] + I * psi0[2 * i + 1];
    for (int64_t k = 0; k < K; k++) {
        const double* U = ops + (size_t)k * 2 * n * n;
        for (int i = 0; i < n; i++) {
            cplx s = 0.0;
            for (int j = 0; j < n; j++) s += (U[2 * (n * i + j)] + I * U[2 * (n * i + j) + 1]) * psi[j];
            nxt[i] = s;
        }
        for (int i = 0; i < n; i++) psi[i] = nxt[i];
        if (states)
            for (int i = 0; i < n; i++) {
                states[(size_t)k * 2 * n + 2 * i] = creal(psi[i]);
                states[(size_t)k * 2 * n + 2 * i + 1] = cimag(psi[i]);
            }
        if (spin) spin_projection(n, psi, spin + (size_t)k * 3);
    }
    return 0;
}

/* Whole simulation: psi_0 = psi_init at t_start, then psi_k = U_k psi_{k-1}.
 * ops (optional, may be NULL) receives U_k ([K][N][N] re,im). */
int oracle_simulate(const oracle_plan* p, const oracle_field* f, const double* psi0,
                    double* states, double* spin, double* ops)
{
    if (p->spin_x2 != 1 && p->spin_x2 != 2) return -1;
    int n = p->spin_x2 == 1 ? 2 : 3;
    cplx psi[3], nxt[3];
    for (int i = 0; i < n; i++) psi[i] = psi0[2 * i] + I * psi0[2 * i + 1];
    for (int64_t k = 0; k < p->K; k++) {
        cplx U[3][3];
        if (k == 0)
            mat_identity(3, U);
        else
            sample_operator(p, f, k, U);
        if (ops) store_matrix(n, U, ops + (size_t)k * 2 * n * n);
        for (int i = 0; i < n; i++) {
            cplx s = 0.0;
            for (int j = 0; j < n; j++) s += U[i][j] * psi[j];
            nxt[i] = s;
        }
        for (int i = 0; i < n; i++) psi[i] = nxt[i];
        if (states)
            for (int i = 0; i < n; i++) {
                states[(size_t)k * 2 * n + 2 * i] = creal(psi[i]);
                states[(size_t)k * 2 * n + 2 * i + 1] = cimag(psi[i]);
            }
        if (spin) spin_projection(n, psi, spin + (size_t)k * 3);
    }
    return 0;
}

/* Error metric of Eq. error: eps = (1/K) sqrt(sum_k sum_m |psi - psi_base|^2),
 * with the 1/K outside the square root as printed. */
double oracle_error_metric(int32_t spin_x2, int64_t K, const double* states, const double* base)
{
    int n = spin_x2 == 1 ? 2 : 3;
    double s = 0.0;
    for (int64_t k = 0; k < K; k++)
        for (int m = 0; m < n; m++) {
            double dr = states[(size_t)k * 2 * n + 2 * m] - base[(size_t)k * 2 * n + 2 * m];
            double di = states[(size_t)k * 2 * n + 2 * m + 1] - base[(size_t)k * 2 * n + 2 * m + 1];
            s += dr * dr + di * di;
        }
    return K > 0 ? sqrt(s) / (double)K : 0.0;
}
