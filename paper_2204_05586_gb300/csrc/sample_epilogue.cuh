// sample_epilogue.cuh -- the end of one sample operator, shared by the
// integrate kernel and the multicore CPU backend: the split residual's
// first-order part replaced by its exact FP64 value, the frame exit
// (Eq. exit_rotating_frame) and the store of U_k; and the spin projection of
// a written state.
#pragma once
#include "device_math.cuh"

namespace spinsim {

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
SPINSIM_HD void store_rows(const cx<double> U[3][3], cx<double> ph, double* out)
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
template <bool TONES, typename R>
SPINSIM_HD void promote(const Res3<R>& P, const DevSim& s, const SampleExact& x, cx<double> Y[3][3])
{
    double gx, gy;
    first_order_exact<TONES>(s, x, gx, gy);
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

template <bool TONES>
SPINSIM_HD void finish(const Res3<double>& P, const DevSim& s, const SampleExact& x, double* out)
{
    cx<double> Y[3][3];
    promote<TONES>(P, s, x, Y);
#pragma unroll
    for (int i = 0; i < 3; i++) Y[i][i].r += 1.0;
    store_rows(Y, cmk(x.ph_re, x.ph_im), out);
}

// FP32-bulk: the operator is stored as computed.  Its departure from
// unitarity is of the order of the FP32 rounding of the second-order rest
// (~1e-11 per sample); the chain renormalises every output state in FP64.
template <bool TONES>
SPINSIM_HD void finish(const Res3<float>& P, const DevSim& s, const SampleExact& x, double* out)
{
    cx<double> Y[3][3];
    promote<TONES>(P, s, x, Y);
#pragma unroll
    for (int i = 0; i < 3; i++) Y[i][i].r += 1.0;
    store_rows(Y, cmk(x.ph_re, x.ph_im), out);
}

template <bool TONES, typename R>
SPINSIM_HD void promote(const Res2<R>& P, const DevSim& s, const SampleExact& x, cx<double>& a,
                                        cx<double>& b)
{
    double gx, gy;
    first_order_exact<TONES>(s, x, gx, gy);
    const double gz = widen(P.g[2]);
    a = cmk(widen(P.a.r), widen(P.a.i) - 0.5 * gz);
    b = cmk(widen(P.b.r) + 0.5 * gy, widen(P.b.i) - 0.5 * gx);
}

SPINSIM_HD void store_half(cx<double> al, cx<double> be, const SampleExact& x, double* out)
{
    const cx<double> p = cmk(x.ph_re, x.ph_im);
    cx<double> a = cmul(p, al);
    cx<double> b = cmul(cconj(p), be);
    out[0] = a.r; out[1] = a.i; out[2] = b.r; out[3] = b.i;
}

template <bool TONES>
SPINSIM_HD void finish(const Res2<double>& P, const DevSim& s, const SampleExact& x, double* out)
{
    cx<double> a, b;
    promote<TONES>(P, s, x, a, b);
    store_half(cmk(1.0 + a.r, a.i), b, x, out);
}

// FP32-bulk spin-half: stored as computed (see the spin-one case); an SU(2)
// element in this form always has det 1.
template <bool TONES>
SPINSIM_HD void finish(const Res2<float>& P, const DevSim& s, const SampleExact& x, double* out)
{
    cx<double> a, b;
    promote<TONES>(P, s, x, a, b);
    store_half(cmk(1.0 + a.r, a.i), b, x, out);
}

SPINSIM_HD void store_identity(int N, double* out)
{
    if (N == 3) {
#pragma unroll
        for (int i = 0; i < 18; i++) out[i] = (i == 0 || i == 8 || i == 16) ? 1.0 : 0.0;
    } else {
        out[0] = 1.0; out[1] = 0.0; out[2] = 0.0; out[3] = 0.0;
    }
}

// <J_x>, <J_y>, <J_z> = psi^dagger J psi (Sec. 1.2.1)
SPINSIM_HD void spin_projection(const cx<double>* p, int N, double* out)
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

}  // namespace spinsim
