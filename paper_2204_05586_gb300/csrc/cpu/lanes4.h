// lanes4.h -- four samples in one value, for the multicore CPU backend.
//
// F4 holds one float per sample in a 16-byte vector (the GCC/Clang vector
// extension: the host compiler turns its element-wise operations into SIMD
// instructions, from the same source on every host architecture).  The
// integrator's step arithmetic (device_math.cuh) is templated on its bulk
// type, so instantiated with F4 it advances four samples of one simulation
// at once.  Every operation is the float operation of the scalar path applied
// lane by lane (std::fma for fma, the C library for exp / sin / cos / rint),
// so each lane's result is bit-identical to the scalar computation.  Only
// what the step loops use is provided; their value-dependent branches have
// lane-wise overloads here.
#pragma once
#include <cmath>
#include <type_traits>

namespace spinsim {

struct F4 {
    typedef float V __attribute__((vector_size(16)));
    V v;
    F4() = default;
    template <typename T, typename = std::enable_if_t<std::is_arithmetic_v<T>>>
    F4(T x)
    {
        const float f = (float)x;
        v = V{f, f, f, f};
    }
    static F4 of(V x)
    {
        F4 r;
        r.v = x;
        return r;
    }
};

template <>
struct BulkTraits<F4> {
    static constexpr bool fp32 = true;
    static constexpr int lanes = 4;
};

inline F4 operator+(F4 a, F4 b) { return F4::of(a.v + b.v); }
inline F4 operator-(F4 a, F4 b) { return F4::of(a.v - b.v); }
inline F4 operator*(F4 a, F4 b) { return F4::of(a.v * b.v); }
inline F4 operator-(F4 a) { return F4::of(-a.v); }
inline F4& operator+=(F4& a, F4 b) { a.v += b.v; return a; }
inline F4& operator-=(F4& a, F4 b) { a.v -= b.v; return a; }
inline F4& operator*=(F4& a, F4 b) { a.v *= b.v; return a; }

template <typename Fn>
inline F4 lanewise(F4 a, Fn fn)
{
    F4 r;
    for (int i = 0; i < 4; i++) r.v[i] = fn(a.v[i]);
    return r;
}

inline F4 fma(F4 a, F4 b, F4 c)
{
    F4 r;
    for (int i = 0; i < 4; i++) r.v[i] = std::fma(a.v[i], b.v[i], c.v[i]);
    return r;
}
inline F4 exp(F4 a) { return lanewise(a, [](float x) { return std::exp(x); }); }
inline F4 exp2(F4 a) { return lanewise(a, [](float x) { return std::exp2(x); }); }
inline F4 sinf(F4 a) { return lanewise(a, [](float x) { return std::sin(x); }); }
inline F4 cosf(F4 a) { return lanewise(a, [](float x) { return std::cos(x); }); }
inline F4 rintf(F4 a) { return lanewise(a, [](float x) { return std::rint(x); }); }

// Lane-wise forms of the step arithmetic's value-dependent branches: the
// small-angle series when every lane's angle is small, else lane by lane.
inline bool all_small(F4 x)
{
    bool r = true;
    for (int i = 0; i < 4; i++) r = r && std::fabs(x.v[i]) <= 0.0625f;
    return r;
}

inline void small_sincos(F4 x, F4& s, F4& c)
{
    if (all_small(x)) {
        sincos_series(x, s, c);
        return;
    }
    for (int i = 0; i < 4; i++) {
        float a, b;
        small_sincos<float>(x.v[i], a, b);
        s.v[i] = a;
        c.v[i] = b;
    }
}

inline void small_sincos_m(F4 x, F4& sm, F4& cm)
{
    if (all_small(x)) {
        sincos_m_series(x, sm, cm);
        return;
    }
    for (int i = 0; i < 4; i++) {
        float a, b;
        small_sincos_m<float>(x.v[i], a, b);
        sm.v[i] = a;
        cm.v[i] = b;
    }
}

inline F4 sine_cycle_cold(F4 u) { return lanewise(u, [](float x) { return sine_cycle_cold<float>(x); }); }
inline F4 sine_cycle(F4 u) { return lanewise(u, [](float x) { return sine_cycle<float>(x); }); }

inline void half_angle_terms(F4 t2, F4& fm, F4& g)
{
    for (int i = 0; i < 4; i++) {
        float a, b;
        half_angle_terms<float>(t2.v[i], a, b);
        fm.v[i] = a;
        g.v[i] = b;
    }
}

inline void transverse_axis_lanes(F4 vx, F4 vy, F4 vp2, F4 inv_n, F4& epr, F4& epi, F4& Phi)
{
    for (int i = 0; i < 4; i++) {
        if (vp2.v[i] > 0.0f) {
            const float rinv = rsqrt(vp2.v[i]);
            epr.v[i] = vx.v[i] * rinv;
            epi.v[i] = vy.v[i] * rinv;
            Phi.v[i] = vp2.v[i] * rinv * inv_n.v[i];
        }
    }
}

// Lane i of a value.
inline float lane(F4 a, int i) { return a.v[i]; }

}  // namespace spinsim
