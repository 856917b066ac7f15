// lanes2.cuh (include after device_math.cuh) -- two samples in one value, for the integrate kernel's paired
// variant on Blackwell.
//
// F2 holds one float per sample in a float2 register pair; its element-wise
// operations are the packed f32x2 instructions (__fadd2_rn, __fmul2_rn,
// __ffma2_rn: one issue slot for both samples, each lane rounded as the
// scalar float operation).  The step arithmetic (device_math.cuh) is
// templated on its bulk type, so instantiated with F2 one thread advances two
// consecutive samples of one simulation at once, with half the instruction
// issues of two scalar threads.  Functions without a packed form (exp2, the
// hardware sine and cosine) run lane by lane.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace spinsim {

struct F2 {
    float2 v;
    F2() = default;
    template <typename T, typename = std::enable_if_t<std::is_arithmetic_v<T>>>
    __host__ __device__ __forceinline__ F2(T x)
    {
        const float f = (float)x;
        v = make_float2(f, f);
    }
    static __device__ __forceinline__ F2 of(float2 x)
    {
        F2 r;
        r.v = x;
        return r;
    }
    static __device__ __forceinline__ F2 of(float a, float b) { return of(make_float2(a, b)); }
};

template <>
struct BulkTraits<F2> {
    static constexpr bool fp32 = true;
    static constexpr int lanes = 2;
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2::of(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2::of(__fadd2_rn(a.v, neg2(b.v))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2::of(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2::of(neg2(a.v)); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { a = a + b; return a; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { a = a - b; return a; }
__device__ __forceinline__ F2& operator*=(F2& a, F2 b) { a = a * b; return a; }
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return F2::of(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 exp(F2 a) { return F2::of(expf(a.v.x), expf(a.v.y)); }
__device__ __forceinline__ F2 exp2(F2 a) { return F2::of(exp2f(a.v.x), exp2f(a.v.y)); }
__device__ __forceinline__ F2 sinf(F2 a) { return F2::of(::sinf(a.v.x), ::sinf(a.v.y)); }
__device__ __forceinline__ F2 cosf(F2 a) { return F2::of(::cosf(a.v.x), ::cosf(a.v.y)); }
__device__ __forceinline__ F2 rintf(F2 a) { return F2::of(::rintf(a.v.x), ::rintf(a.v.y)); }
__device__ __forceinline__ F2 fabs(F2 a) { return F2::of(fabsf(a.v.x), fabsf(a.v.y)); }

// Lane i of a value.
__device__ __forceinline__ float lane(F2 a, int i) { return i ? a.v.y : a.v.x; }

// The counter-rotating phasor's sine and cosine (second-order accuracy
// suffices, see second_order_sincos), lane by lane.
__device__ __forceinline__ void second_order_sincos(F2 x, F2& s, F2& c)
{
    float s0, c0, s1, c1;
    second_order_sincos(x.v.x, s0, c0);
    second_order_sincos(x.v.y, s1, c1);
    s = F2::of(s0, s1);
    c = F2::of(c0, c1);
}

// The single-sine-cycle pulse shape, lane by lane.
__device__ __forceinline__ F2 sine_cycle(F2 u) { return F2::of(sine_cycle<float>(u.v.x), sine_cycle<float>(u.v.y)); }

// The transverse axis and angle of expm_one_res_n, lane by lane.
__device__ __forceinline__ void transverse_axis_lanes(F2 vx, F2 vy, F2 vp2, F2 inv_n, F2& epr, F2& epi, F2& Phi)
{
    float r[2] = {1.0f, 1.0f}, i[2] = {0.0f, 0.0f}, p[2] = {0.0f, 0.0f};
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const float q = lane(vp2, h);
        if (q > 0.0f) {
            const float rinv = rsqrtf(q);
            r[h] = lane(vx, h) * rinv;
            i[h] = lane(vy, h) * rinv;
            p[h] = q * rinv * lane(inv_n, h);
        }
    }
    epr = F2::of(r[0], r[1]);
    epi = F2::of(i[0], i[1]);
    Phi = F2::of(p[0], p[1]);
}

// The SU(2) exponential's half-angle terms, lane by lane (each lane takes the
// series or the library functions by its own angle, as the scalar code does).
__device__ __forceinline__ void half_angle_terms(F2 t2, F2& fm, F2& g)
{
    float f0, g0, f1, g1;
    half_angle_terms<float>(t2.v.x, f0, g0);
    half_angle_terms<float>(t2.v.y, f1, g1);
    fm = F2::of(f0, f1);
    g = F2::of(g0, g1);
}

// The contexts of two consecutive samples of one simulation, lane by lane
// (the per-simulation integers are the same in both).
__device__ __forceinline__ void pack(const SampleCtx<float> (&c)[2], SampleCtx<F2>& v)
{
#define SPINSIM_PACK2(f) v.f = F2::of(c[0].f, c[1].f)
    SPINSIM_PACK2(ebr); SPINSIM_PACK2(ebi); SPINSIM_PACK2(co); SPINSIM_PACK2(counter);
#pragma unroll
    for (int i = 0; i < 4; i++) SPINSIM_PACK2(Ph[i]);
    SPINSIM_PACK2(za); SPINSIM_PACK2(zb); SPINSIM_PACK2(zbias); SPINSIM_PACK2(qd3); SPINSIM_PACK2(inv_n);
    SPINSIM_PACK2(q1); SPINSIM_PACK2(dt); SPINSIM_PACK2(c1); SPINSIM_PACK2(c2);
    SPINSIM_PACK2(d1r); SPINSIM_PACK2(d1i); SPINSIM_PACK2(p1r); SPINSIM_PACK2(p1i); SPINSIM_PACK2(eqr); SPINSIM_PACK2(eqi);
#pragma unroll
    for (int p = 0; p < kMaxPulses; p++) {
        SPINSIM_PACK2(amp[p]); SPINSIM_PACK2(u0[p]); SPINSIM_PACK2(invw[p]); SPINSIM_PACK2(ghat[p]);
        SPINSIM_PACK2(u0b[p]); SPINSIM_PACK2(invwb[p]);
    }
#undef SPINSIM_PACK2
    v.nt = 0;                  // the paired kernels carry no further tones
    v.np = c[0].np;
    v.ng = c[0].ng;
    v.tau = c[0].tau;
    v.counter_on = c[0].counter_on;
}

// Lane h of a paired spin-half residual.
__device__ __forceinline__ void unpack(const Res2<F2>& v, int h, Res2<float>& x)
{
#pragma unroll
    for (int q = 0; q < 3; q++) x.g[q] = lane(v.g[q], h);
    x.a = cmk(lane(v.a.r, h), lane(v.a.i, h));
    x.b = cmk(lane(v.b.r, h), lane(v.b.i, h));
}

// Lane h of a paired spin-one residual.
__device__ __forceinline__ void unpack(const Res3<F2>& v, int h, Res3<float>& x)
{
#pragma unroll
    for (int q = 0; q < 4; q++) x.g[q] = lane(v.g[q], h);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) x.m[i][j] = cmk(lane(v.m[i][j].r, h), lane(v.m[i][j].i, h));
}

}  // namespace spinsim
