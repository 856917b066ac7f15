// cpu_backend.cu -- the multicore CPU backend (include/spinsim_cpu.h).
//
// The integrator on the host's cores with the same algorithm as the GPU path
// (Sec. 1.2.6, 1.2.7): every sample operator U_k from the integrate kernel's
// per-sample arithmetic (device_math.cuh and sample_epilogue.cuh compiled for
// the host: the same step loop, the same canonical segments and reduction
// tree, the same FP64 epilogue), samples spread over worker threads; then
// each simulation's states psi_k = U_k psi_{k-1} in order, in FP64 (Eq.
// integration_compilation), as the paper's CPU chain does.
//
// In FP32 each thread advances four samples at once (lanes4.h: one SIMD
// vector per quantity), each lane bit-identical to the one-sample path.
//
// Host code only: this file is linked with params.cu into
// libspinsim_cpu.so, which calls no CUDA API and needs no GPU.
#include <sched.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "spinsim_cpu.h"
#include "../sample_epilogue.cuh"
#include "lanes4.h"

namespace spinsim {
namespace {

// U_k (1 <= k < K) into out (spin-one 18, spin-half 4 doubles): the L steps in
// the 2^seg_log2 canonical segments, merged by the fixed binary tree (a
// finished pair of equal sub-trees merges, later on the left), then the
// epilogue.  The integrate kernel's lane that owns all segments does the same.
template <int N, typename R, int METHOD, int SMALL, bool TONES, bool SU3 = false>
void sample_operator(const DevSim& s, int64_t k, double* out)
{
    using Res = typename ResType<N, R>::type;
    SampleCtx<R> c;
    double beta = 0.0;
    const double gsum = make_ctx<R, N, TONES, SU3>(s, k, c, beta);
    Res stack[kSegLog2 + 1];
    const int nseg = 1 << s.seg_log2;
    for (int q = 0; q < nseg; q++) {
        const int64_t lo = ((int64_t)q * s.L) >> s.seg_log2, hi = ((int64_t)(q + 1) * s.L) >> s.seg_log2;
        Res X;
        res_zero(X);
        if constexpr (SU3) {
            CounterPhasors<R> ph;
            counter_phasors_at<R, METHOD>(c, lo, ph);
            for (int64_t l = lo; l < hi; l++) step_apply_su3<R, METHOD, TONES>(c, (R)l, ph, X);
        } else if constexpr (SMALL && N == 3) {
            DrivePhasors<R> dp;
            drive_phasors_at<R, METHOD>(c, lo, dp);
            for (int64_t l = lo; l < hi; l++) step_apply<R, METHOD, SMALL, TONES>(c, (R)l, c.tau, X, &dp);
        } else {
            for (int64_t l = lo; l < hi; l++) step_apply<R, METHOD, SMALL, TONES>(c, (R)l, c.tau, X);
        }
        int h = 0;
        while ((q >> h) & 1) {
            Res t;
            res_mul(X, stack[h], t);
            X = t;
            h++;
        }
        stack[h] = X;
    }
    SampleExact x;
    make_exact<N, TONES>(s, k, beta, gsum, x);
    finish<TONES>(stack[s.seg_log2], s, x, out);
}

// Four samples k .. k+3 (all >= 1) of one simulation at once (FP32): their
// contexts packed lane by lane into F4 values, the same step loop and
// segment tree on F4, then each lane's epilogue.  Every lane computes exactly
// what sample_operator computes.
void pack(const SampleCtx<float> (&c)[4], SampleCtx<F4>& v)
{
    auto put = [](F4& dst, float a, float b, float d, float e) { dst.v = F4::V{a, b, d, e}; };
#define SPINSIM_PACK(f) put(v.f, c[0].f, c[1].f, c[2].f, c[3].f)
    SPINSIM_PACK(ebr); SPINSIM_PACK(ebi); SPINSIM_PACK(co); SPINSIM_PACK(counter);
    for (int i = 0; i < 4; i++) SPINSIM_PACK(Ph[i]);
    SPINSIM_PACK(za); SPINSIM_PACK(zb); SPINSIM_PACK(zbias); SPINSIM_PACK(qd3); SPINSIM_PACK(inv_n);
    SPINSIM_PACK(q1); SPINSIM_PACK(dt); SPINSIM_PACK(c1); SPINSIM_PACK(c2);
    SPINSIM_PACK(d1r); SPINSIM_PACK(d1i); SPINSIM_PACK(p1r); SPINSIM_PACK(p1i); SPINSIM_PACK(eqr); SPINSIM_PACK(eqi);
    for (int p = 0; p < kMaxPulses; p++) {
        SPINSIM_PACK(amp[p]); SPINSIM_PACK(u0[p]); SPINSIM_PACK(invw[p]); SPINSIM_PACK(ghat[p]);
        SPINSIM_PACK(u0b[p]); SPINSIM_PACK(invwb[p]);
    }
    for (int j = 0; j < kMaxTones; j++) {
        SPINSIM_PACK(tbr[j]); SPINSIM_PACK(tbi[j]); SPINSIM_PACK(tco[j]); SPINSIM_PACK(tct[j]);
        SPINSIM_PACK(tomp[j]); SPINSIM_PACK(tomm[j]);
    }
#undef SPINSIM_PACK
    v.nt = c[0].nt;            // per simulation: the same in every lane
    v.np = c[0].np;
    v.ng = c[0].ng;
    v.tau = c[0].tau;
    v.counter_on = c[0].counter_on;
}

void unpack(const Res3<F4>& v, int i, Res3<float>& x)
{
    for (int q = 0; q < 4; q++) x.g[q] = lane(v.g[q], i);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) x.m[a][b] = cmk(lane(v.m[a][b].r, i), lane(v.m[a][b].i, i));
}

void unpack(const Res2<F4>& v, int i, Res2<float>& x)
{
    for (int q = 0; q < 3; q++) x.g[q] = lane(v.g[q], i);
    x.a = cmk(lane(v.a.r, i), lane(v.a.i, i));
    x.b = cmk(lane(v.b.r, i), lane(v.b.i, i));
}

template <int N, int METHOD, int SMALL, bool TONES>
void sample_operators4(const DevSim& s, int64_t k, double* out)
{
    using Res = typename ResType<N, float>::type;
    using Res4 = typename ResType<N, F4>::type;
    constexpr int OPD = N == 3 ? 18 : 4;
    SampleCtx<float> c1[4];
    double beta[4], gsum[4];
    for (int i = 0; i < 4; i++) gsum[i] = make_ctx<float, N, TONES>(s, k + i, c1[i], beta[i]);
    SampleCtx<F4> c;
    pack(c1, c);
    Res4 stack[kSegLog2 + 1];
    const int nseg = 1 << s.seg_log2;
    for (int q = 0; q < nseg; q++) {
        const int64_t lo = ((int64_t)q * s.L) >> s.seg_log2, hi = ((int64_t)(q + 1) * s.L) >> s.seg_log2;
        Res4 X;
        res_zero(X);
        if constexpr (SMALL && N == 3) {
            DrivePhasors<F4> dp;
            drive_phasors_at<F4, METHOD>(c, lo, dp);
            for (int64_t l = lo; l < hi; l++) step_apply<F4, METHOD, SMALL, TONES>(c, F4((float)l), c.tau, X, &dp);
        } else {
            for (int64_t l = lo; l < hi; l++) step_apply<F4, METHOD, SMALL, TONES>(c, F4((float)l), c.tau, X);
        }
        int h = 0;
        while ((q >> h) & 1) {
            Res4 t;
            res_mul(X, stack[h], t);
            X = t;
            h++;
        }
        stack[h] = X;
    }
    for (int i = 0; i < 4; i++) {
        Res r;
        unpack(stack[s.seg_log2], i, r);
        SampleExact x;
        make_exact<N, TONES>(s, k + i, beta[i], gsum[i], x);
        finish<TONES>(r, s, x, out + i * OPD);
    }
}

using SampleFn = void (*)(const DevSim&, int64_t, double*);

template <int N, int SMALL, bool TONES>
SampleFn pick_method4(int method)
{
    switch (method) {
        case SPINSIM_METHOD_CF4: return sample_operators4<N, 0, SMALL, TONES>;
        case SPINSIM_METHOD_MIDPOINT: return sample_operators4<N, 1, SMALL, TONES>;
        case SPINSIM_METHOD_HEUN: return sample_operators4<N, 2, SMALL, TONES>;
        default: return nullptr;
    }
}

template <int N>
SampleFn pick_variant4(int method, int variant)
{
    switch (variant) {
        case kVariantGeneral: return pick_method4<N, false, false>(method);
        // the tau = 0 variants run the same arithmetic with tau taken at run time
        case kVariantSmall:
        case kVariantSmallTau0: return pick_method4<N, 1, false>(method);
        case kVariantSmallSine:
        case kVariantSmallSineTau0: return pick_method4<N, 2, false>(method);
        case kVariantTones: return pick_method4<N, false, true>(method);
        case kVariantSmallTones: return pick_method4<N, 1, true>(method);
        default: return nullptr;
    }
}

// The four-sample form of an FP32 variant (FP64 runs one sample at a time).
SampleFn select_sample4_fn(int spin_x2, int precision, int method, int variant)
{
    if (!precision) return nullptr;
    return spin_x2 == 2 ? pick_variant4<3>(method, variant) : pick_variant4<2>(method, variant);
}

template <int N, typename R, int SMALL, bool TONES>
SampleFn pick_method(int method)
{
    switch (method) {
        case SPINSIM_METHOD_CF4: return sample_operator<N, R, 0, SMALL, TONES>;
        case SPINSIM_METHOD_MIDPOINT: return sample_operator<N, R, 1, SMALL, TONES>;
        case SPINSIM_METHOD_HEUN: return sample_operator<N, R, 2, SMALL, TONES>;
        default: return nullptr;
    }
}

template <int N, typename R>
SampleFn pick_variant(int method, int variant)
{
    switch (variant) {
        case kVariantGeneral: return pick_method<N, R, false, false>(method);
        case kVariantTones: return pick_method<N, R, false, true>(method);
        case kVariantSmallTones:
            if constexpr (sizeof(R) == 4) return pick_method<N, R, 1, true>(method);
            else return nullptr;
        case kVariantSmall:
        case kVariantSmallTau0:
            if constexpr (sizeof(R) == 4) return pick_method<N, R, 1, false>(method);
            else return nullptr;
        case kVariantSmallSine:
        case kVariantSmallSineTau0:
            if constexpr (sizeof(R) == 4) return pick_method<N, R, 2, false>(method);
            else return nullptr;
        case kVariantSU3:   // full su(3): spin-one, FP64
            if constexpr (N == 3 && sizeof(R) == 8) {
                switch (method) {
                    case SPINSIM_METHOD_CF4: return sample_operator<3, double, 0, false, true, true>;
                    case SPINSIM_METHOD_MIDPOINT: return sample_operator<3, double, 1, false, true, true>;
                    case SPINSIM_METHOD_HEUN: return sample_operator<3, double, 2, false, true, true>;
                    default: return nullptr;
                }
            } else {
                return nullptr;
            }
        default: return nullptr;
    }
}

SampleFn select_sample_fn(int spin_x2, int precision, int method, int variant)
{
    if (spin_x2 == 2) return precision ? pick_variant<3, float>(method, variant) : pick_variant<3, double>(method, variant);
    return precision ? pick_variant<2, float>(method, variant) : pick_variant<2, double>(method, variant);
}

// psi <- U psi for a stored operator (spin-one: 3x3 row-major; spin-half: the
// SU(2) pair (alpha, beta) of [[alpha, -conj beta], [beta, conj alpha]]).
template <int N>
void apply_op(const double* u, cx<double>* psi)
{
    cx<double> out[N];
    if constexpr (N == 3) {
        for (int i = 0; i < 3; i++) {
            cx<double> acc = cmk(0.0, 0.0);
            for (int j = 0; j < 3; j++) acc = cfma(cmk(u[6 * i + 2 * j], u[6 * i + 2 * j + 1]), psi[j], acc);
            out[i] = acc;
        }
    } else {
        const cx<double> a = cmk(u[0], u[1]), b = cmk(u[2], u[3]);
        out[0] = csub(cmul(a, psi[0]), cmul(cconj(b), psi[1]));
        out[1] = cadd(cmul(b, psi[0]), cmul(cconj(a), psi[1]));
    }
    for (int i = 0; i < N; i++) psi[i] = out[i];
}

// Full N x N complex matrix of a stored operator (the ops output layout).
template <int N>
void store_full(const double* u, double* p)
{
    if constexpr (N == 3) {
        std::memcpy(p, u, 18 * sizeof(double));
    } else {
        p[0] = u[0]; p[1] = u[1]; p[2] = -u[2]; p[3] = u[3];
        p[4] = u[2]; p[5] = u[3]; p[6] = u[0]; p[7] = -u[1];
    }
}

// psi_k = U_k psi_{k-1} from psi_0 = psi_init (U_0 = I) in order; the written
// state is renormalised in FP64 for FP32-bulk operators, as on the GPU.
template <int N>
void chain(const DevSim& s, const double* U, spinsim_result& r)
{
    constexpr int OPD = N == 3 ? 18 : 4;
    cx<double> psi[N];
    for (int i = 0; i < N; i++) psi[i] = cmk(s.psi0[2 * i], s.psi0[2 * i + 1]);
    for (int64_t k = 0; k < s.K; k++) {
        const double* u = U + k * OPD;
        apply_op<N>(u, psi);
        double scale = 1.0;
        if (s.normalize_out) {
            double n2 = 0.0;
            for (int i = 0; i < N; i++) n2 = fma(psi[i].r, psi[i].r, fma(psi[i].i, psi[i].i, n2));
            const double d = n2 - 1.0;
            scale = 1.0 - d * (0.5 - 0.375 * d);   // (1 + d)^(-1/2), |d| ~ 1e-9
        }
        cx<double> w[N];
        for (int i = 0; i < N; i++) {
            w[i] = cscale(psi[i], scale);
            r.states[k * 2 * N + 2 * i] = w[i].r;
            r.states[k * 2 * N + 2 * i + 1] = w[i].i;
        }
        if (r.spin) spin_projection(w, N, r.spin + k * 3);
        if (r.ops) store_full<N>(u, r.ops + k * 2 * N * N);
    }
}

int usable_cores()
{
    cpu_set_t set;
    CPU_ZERO(&set);
    if (sched_getaffinity(0, sizeof(set), &set) == 0) {
        const int n = CPU_COUNT(&set);
        if (n > 0) return n;
    }
    return std::max(1u, std::thread::hardware_concurrency());
}

// Run `count` work items over `threads` workers (the calling thread is one).
template <typename F>
void parallel_for(int threads, int64_t count, F&& f)
{
    std::atomic<int64_t> next{0};
    auto worker = [&]() {
        for (int64_t i = next.fetch_add(1); i < count; i = next.fetch_add(1)) f(i);
    };
    const int extra = (int)std::min<int64_t>(threads - 1, std::max<int64_t>(count - 1, 0));
    std::vector<std::thread> pool;
    pool.reserve(extra);
    for (int t = 0; t < extra; t++) {
        try {
            pool.emplace_back(worker);
        } catch (...) {   // fewer threads: the ones running (and this one) drain the items
            break;
        }
    }
    worker();
    for (auto& t : pool) t.join();
}

struct Job {
    int64_t req;
    DevSim d;
    SampleFn fn;
    SampleFn fn4;   // four samples at once, or nullptr
    size_t u_off;   // offset of its operators in the group buffer (doubles)
};

constexpr int64_t kChunk = 128;                          // samples per work item
constexpr size_t kGroupDoubles = (size_t)32 << 20;       // 256 MiB of operators per group

}  // namespace
}  // namespace spinsim

using namespace spinsim;

namespace {

int cpu_simulate(const spinsim_config* cfg_in, const spinsim_request* reqs, spinsim_result* res, int64_t n,
                 int32_t threads)
{
    if (n < 0 || (n > 0 && (!reqs || !res)) || threads < 0) return SPINSIM_E_ARG;
    spinsim_config cfg{};
    if (cfg_in) {
        cfg = *cfg_in;
    } else {
        cfg.method = SPINSIM_METHOD_CF4;
        cfg.precision = SPINSIM_PREC_FP32_BULK;
        cfg.rotating_frame = 1;
        cfg.trotter_squares = -1;
    }
    if (cfg.method < SPINSIM_METHOD_CF4 || cfg.method > SPINSIM_METHOD_HEUN ||
        (cfg.precision != SPINSIM_PREC_FP64 && cfg.precision != SPINSIM_PREC_FP32_BULK) || cfg.trotter_squares < -1 ||
        cfg.trotter_squares > 40)
        return SPINSIM_E_ARG;
    const int nt = threads > 0 ? threads : usable_cores();

    int first_err = SPINSIM_OK;
    std::vector<Job> jobs;
    for (int64_t i = 0; i < n; i++) {
        Checked c = check_request(&reqs[i]);
        if (c.status == SPINSIM_OK) c.status = precision_status(cfg, reqs[i]);
        if (c.status == SPINSIM_OK) {
            if (!res[i].states) c.status = SPINSIM_E_ARG;
            else if (res[i].capacity < c.K) c.status = SPINSIM_E_CAPACITY;
        }
        res[i].status = c.status;
        res[i].flags = c.status == SPINSIM_OK ? c.flags | precision_flags(cfg.precision, cfg.rotating_frame, reqs[i]) : 0;
        res[i].n_samples = c.status == SPINSIM_OK ? c.K : 0;
        res[i].trotter_squares = 0;
        if (c.status != SPINSIM_OK) {
            if (first_err == SPINSIM_OK) first_err = c.status;
            continue;
        }
        Job j;
        j.req = i;
        fill_devsim(cfg, reqs[i], c.K, c.L, j.d);
        const int variant = request_variant(cfg, reqs[i], c.K, c.L);
        j.fn = select_sample_fn(reqs[i].spin_x2, cfg.precision, cfg.method, variant);
        j.fn4 = select_sample4_fn(reqs[i].spin_x2, cfg.precision, cfg.method, variant);
        j.u_off = 0;
        res[i].trotter_squares = j.d.tau;
        if (!j.fn) {
            res[i].status = SPINSIM_E_ARG;
            if (first_err == SPINSIM_OK) first_err = SPINSIM_E_ARG;
            continue;
        }
        jobs.push_back(j);
    }

    // groups of consecutive requests whose operators fit one buffer (a request
    // larger than the buffer forms a group of its own)
    size_t g0 = 0;
    std::vector<double> U;
    while (g0 < jobs.size()) {
        size_t g1 = g0, total = 0;
        while (g1 < jobs.size()) {
            const size_t need = (size_t)jobs[g1].d.K * (jobs[g1].d.spin_x2 == 2 ? 18 : 4);
            if (g1 > g0 && total + need > kGroupDoubles) break;
            jobs[g1].u_off = total;
            total += need;
            g1++;
        }
        try {
            if (U.size() < total) U.resize(total);
        } catch (const std::bad_alloc&) {
            for (size_t j = g0; j < jobs.size(); j++) res[jobs[j].req].status = SPINSIM_E_NOMEM;
            return SPINSIM_E_NOMEM;
        }
        // work items: chunks of samples of the group's requests
        std::vector<std::pair<size_t, int64_t>> items;
        for (size_t j = g0; j < g1; j++)
            for (int64_t k0 = 0; k0 < jobs[j].d.K; k0 += kChunk) items.emplace_back(j, k0);
        double* Ub = U.data();
        parallel_for(nt, (int64_t)items.size(), [&](int64_t it) {
            const Job& jb = jobs[items[it].first];
            const int opd = jb.d.spin_x2 == 2 ? 18 : 4;
            const int64_t k1 = std::min(items[it].second + kChunk, jb.d.K);
            int64_t k = items[it].second;
            if (k == 0) store_identity(jb.d.spin_x2 + 1, Ub + jb.u_off);
            k = std::max<int64_t>(k, 1);
            if (jb.fn4)
                for (; k + 4 <= k1; k += 4) jb.fn4(jb.d, k, Ub + jb.u_off + k * opd);
            for (; k < k1; k++) jb.fn(jb.d, k, Ub + jb.u_off + k * opd);
        });
        parallel_for(nt, (int64_t)(g1 - g0), [&](int64_t j) {
            const Job& jb = jobs[g0 + j];
            if (jb.d.spin_x2 == 2) chain<3>(jb.d, Ub + jb.u_off, res[jb.req]);
            else chain<2>(jb.d, Ub + jb.u_off, res[jb.req]);
        });
        g0 = g1;
    }
    return first_err;
}

}  // namespace

// The C entry point: no C++ exception leaves it (a thread or an allocation
// that fails is reported as SPINSIM_E_NOMEM).
extern "C" int spinsim_cpu_simulate(const spinsim_config* cfg, const spinsim_request* reqs, spinsim_result* res,
                                    int64_t n, int32_t threads)
{
    try {
        return cpu_simulate(cfg, reqs, res, n, threads);
    } catch (...) {
        return SPINSIM_E_NOMEM;
    }
}
