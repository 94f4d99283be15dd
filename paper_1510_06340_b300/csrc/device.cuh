// device.cuh -- device-side physics and the streaming pencil sweep of the
// MUSTA-FORCE update (Sec. 2.3-2.6 of the paper).
//
// Design: one thread marches one pencil segment along the sweep axis.  Each
// Runge-Kutta stage is a streaming "engine" holding a three-cell window: a
// new cell value arriving lets it finish the limited faces and Hancock half
// step of the previous cell (Eq. 13, 15-17), the MUSTA-FORCE flux of the
// interface before it (Eq. 8-11) and the divergence of the cell before that.
// Stages are chained in registers, so a sweep reads and writes every cell
// once; the halo of a segment (2 cells per stage on each side) is
// recomputed by the neighbouring segment instead of exchanged.
//
// The momentum component along the sweep axis is always carried in slot n of
// V4, so one kernel serves all three axes; only the addressing differs.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.h"

namespace hy {

// The conserved fields of one cell in sweep-slot order: E, M along the
// sweep axis, the two transverse M; with CH the conserved charge R = n gamma
// (Eq. 3-4) rides along as a fifth field.
template <class R, bool CH = false>
struct VS {
    R e, n, t1, t2;
};
template <class R>
struct VS<R, true> {
    R e, n, t1, t2, r;
};
template <class R>
using V4 = VS<R, false>;
template <class R>
using V5 = VS<R, true>;

template <class R>
__device__ __forceinline__ V4<R> v4(R a, R b, R c, R d) {
    V4<R> v; v.e = a; v.n = b; v.t1 = c; v.t2 = d; return v;
}
// the energy-momentum part of a cell, and a cell made of one plus a charge
template <class R>
__device__ __forceinline__ V4<R> head(const V4<R> &x) { return x; }
template <class R>
__device__ __forceinline__ V4<R> head(const V5<R> &x) { return v4<R>(x.e, x.n, x.t1, x.t2); }
template <class R>
__device__ __forceinline__ V5<R> with_r(const V4<R> &x, R r) {
    V5<R> v; v.e = x.e; v.n = x.n; v.t1 = x.t1; v.t2 = x.t2; v.r = r; return v;
}
template <class V>
__device__ __forceinline__ V vzero() {
    V v{};
    return v;
}

// Multiply-adds of the formulas are written out as fma_, so they are fused
// whatever the compiler's contraction setting.
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

// field-wise helpers: x - y, x + y, s x + y, s x
template <class R>
__device__ __forceinline__ V4<R> vsub(const V4<R> &x, const V4<R> &y) {
    return v4<R>(x.e - y.e, x.n - y.n, x.t1 - y.t1, x.t2 - y.t2);
}
template <class R>
__device__ __forceinline__ V4<R> vadd(const V4<R> &x, const V4<R> &y) {
    return v4<R>(x.e + y.e, x.n + y.n, x.t1 + y.t1, x.t2 + y.t2);
}
template <class R>
__device__ __forceinline__ V4<R> vfma(R s, const V4<R> &x, const V4<R> &y) {
    return v4<R>(fma_(s, x.e, y.e), fma_(s, x.n, y.n), fma_(s, x.t1, y.t1), fma_(s, x.t2, y.t2));
}
template <class R>
__device__ __forceinline__ V4<R> vmul(R s, const V4<R> &x) {
    return v4<R>(s * x.e, s * x.n, s * x.t1, s * x.t2);
}
// the transverse flux terms (M_t1 v_n, M_t2 v_n)
template <class R>
__device__ __forceinline__ void tmul(R s, const V4<R> &x, R &t1, R &t2) {
    t1 = x.t1 * s; t2 = x.t2 * s;
}

// Two-wide FP32 arithmetic (add/sub/mul/fma .f32x2 of sm_100 and later): one
// instruction computes a pair of lanes, each rounded as the scalar
// instruction is.  Units built with flushed denormals define HY_FTZ, and the
// pair instructions flush too, so they agree with the scalar code there.
#ifdef HY_FTZ
#define HY_F2 ".rn.ftz.f32x2"
#else
#define HY_F2 ".rn.f32x2"
#endif
#define HY_F2_BINARY(name, op)                                                              \
    __device__ __forceinline__ float2 name(float2 x, float2 y) {                             \
        float2 r;                                                                           \
        asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t" \
            op HY_F2 " d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"                               \
            : "=f"(r.x), "=f"(r.y)                                                          \
            : "f"(x.x), "f"(x.y), "f"(y.x), "f"(y.y));                                      \
        return r;                                                                           \
    }
HY_F2_BINARY(add2, "add")
HY_F2_BINARY(sub2, "sub")
HY_F2_BINARY(mul2, "mul")
#undef HY_F2_BINARY
__device__ __forceinline__ float2 fma2(float2 x, float2 y, float2 z) {
    float2 r;
    asm("{\n\t.reg .b64 a, b, c, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mov.b64 c, {%6, %7};\n\tfma" HY_F2 " d, a, b, c;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(x.x), "f"(x.y), "f"(y.x), "f"(y.y), "f"(z.x), "f"(z.y));
    return r;
}

// FP32: the field-wise helpers act on the pairs (E, M_n) and (M_t1, M_t2).
// The FP32 sweep is bound by instruction issue, and this halves the issued
// instructions of its per-field arithmetic.
__device__ __forceinline__ float2 lo2(const V4<float> &x) { return make_float2(x.e, x.n); }
__device__ __forceinline__ float2 hi2(const V4<float> &x) { return make_float2(x.t1, x.t2); }
__device__ __forceinline__ float2 dup2(float s) { return make_float2(s, s); }
__device__ __forceinline__ V4<float> from2(float2 a, float2 b) {
    return v4<float>(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ V4<float> vsub<float>(const V4<float> &x, const V4<float> &y) {
    return from2(sub2(lo2(x), lo2(y)), sub2(hi2(x), hi2(y)));
}
template <>
__device__ __forceinline__ V4<float> vadd<float>(const V4<float> &x, const V4<float> &y) {
    return from2(add2(lo2(x), lo2(y)), add2(hi2(x), hi2(y)));
}
template <>
__device__ __forceinline__ V4<float> vfma<float>(float s, const V4<float> &x, const V4<float> &y) {
    const float2 s2 = dup2(s);
    return from2(fma2(s2, lo2(x), lo2(y)), fma2(s2, hi2(x), hi2(y)));
}
template <>
__device__ __forceinline__ V4<float> vmul<float>(float s, const V4<float> &x) {
    const float2 s2 = dup2(s);
    return from2(mul2(s2, lo2(x)), mul2(s2, hi2(x)));
}
template <>
__device__ __forceinline__ void tmul<float>(float s, const V4<float> &x, float &t1, float &t2) {
    const float2 t = mul2(hi2(x), dup2(s));
    t1 = t.x; t2 = t.y;
}

// the same field-wise helpers with the charge: the four-field forms plus R
template <class R>
__device__ __forceinline__ V5<R> vsub(const V5<R> &x, const V5<R> &y) {
    return with_r(vsub<R>(head(x), head(y)), x.r - y.r);
}
template <class R>
__device__ __forceinline__ V5<R> vadd(const V5<R> &x, const V5<R> &y) {
    return with_r(vadd<R>(head(x), head(y)), x.r + y.r);
}
template <class R>
__device__ __forceinline__ V5<R> vfma(R s, const V5<R> &x, const V5<R> &y) {
    return with_r(vfma<R>(s, head(x), head(y)), fma_(s, x.r, y.r));
}
template <class R>
__device__ __forceinline__ V5<R> vmul(R s, const V5<R> &x) {
    return with_r(vmul<R>(s, head(x)), s * x.r);
}

// ---------------------------------------------------------------- math helpers
__device__ __forceinline__ double dsqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt_(float x) { return sqrtf(x); }
// 1/x: exact in FP64; in FP32 the hardware approximation (rcp.approx, within
// about one ulp), the accuracy class of the FP32 sweep's fast division
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double fmax_(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float fmax_(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double fmin_(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float fmin_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double fabs_(double a) { return fabs(a); }
__device__ __forceinline__ float fabs_(float a) { return fabsf(a); }
__device__ __forceinline__ bool positive(double a) { return a > 0.0; }
__device__ __forceinline__ bool positive(float a) { return a > 0.0f; }

// ---------------------------------------------------------------- limiters
// Sec. 2.5 (Eq. 15-21), division-free: returns a * xi(b / a).
template <class R>
__device__ __forceinline__ R limited_slope(int kind, R a, R b) {
    const R ab = a * b;
    const R half = R(0.5), two = R(2);
    if (kind == LIM_NONE) return half * (a + b);
    if (!(ab > R(0))) return R(0);
    const R aa = fabs_(a), bb = fabs_(b);
    R m;
    switch (kind) {
    case LIM_MINMOD: m = fmin_(aa, bb); break;
    case LIM_MC: m = fmin_(fmin_(two * aa, two * bb), half * fabs_(a + b)); break;
    case LIM_SUPERBEE: m = fmax_(fmin_(two * aa, bb), fmin_(aa, two * bb)); break;
    case LIM_VANLEER: return two * ab / (a + b);
    default: return ab * (a + b) / (a * a + b * b);   // van Albada (r > 0)
    }
    return a > R(0) ? m : -m;
}

// Compile-time limiter.  Minbee, MC and Superbee in median form:
// median(0, a, b) = max(min(a, b), min(max(a, b), 0)) is a*xi_MB(b/a) exactly
// (both pick the smaller magnitude when a, b share a sign, else 0); the 3-way
// minmod of MC and the two minmods of Superbee follow from it.
__device__ __forceinline__ float med0(float a, float b) {
    return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.0f));
}
__device__ __forceinline__ double med0(double a, double b) {
    return fmax(fmin(a, b), fmin(fmax(a, b), 0.0));
}

template <int LIM, class R>
__device__ __forceinline__ R slope_ct(int kind, R a, R b) {
    if (LIM == LIM_MINMOD) return med0(a, b);
    if (LIM == LIM_MC) {
        const R m = med0(R(2) * a, R(2) * b);
        const R h = R(0.5) * (a + b);
        return fmax_(fmin_(m, h), fmin_(fmax_(m, h), R(0)));
    }
    if (LIM == LIM_SUPERBEE) {
        const R s1 = med0(R(2) * a, b), s2 = med0(a, R(2) * b);
        return a > R(0) ? fmax_(s1, s2) : fmin_(s1, s2);
    }
    if (LIM == LIM_NONE) return R(0.5) * (a + b);
    return limited_slope<R>(kind, a, b);   // runtime choice (van Leer, van Albada, any)
}

__device__ __forceinline__ void count(const Scheme &s, int which, unsigned long long v = 1) {
    if (s.counters) atomicAdd(s.counters + which, v);
}

// OR the FLAG_* bits of the 32 lanes of a converged warp into the event's
// status word (one atomic per warp, only when a bit is set) and clear them
__device__ __forceinline__ void report_flags(const Scheme &s, int event, unsigned &flags) {
    if (!s.event_flags) return;
    const unsigned f = __reduce_or_sync(0xffffffffu, flags);
    if (f && (threadIdx.x & 31) == 0) atomicOr(s.event_flags + event, f);
    flags = 0;
}

// the scheme's constants in precision R
template <class R>
__device__ __forceinline__ const SchemeConsts<R> &consts(const Scheme &s);
template <>
__device__ __forceinline__ const SchemeConsts<double> &consts<double>(const Scheme &s) {
    return s.c64;
}
template <>
__device__ __forceinline__ const SchemeConsts<float> &consts<float>(const Scheme &s) {
    return s.c32;
}

// ---------------------------------------------------------------- cons -> prim
// What a flux evaluation needs from Eq. 23: velocity along the sweep axis and p.
template <class R>
struct Prim {
    R vn, p;
    R W;     // E + p
    R fe;    // energy flux (E + p) v_n
};

// Conformal EOS p = cs2 e (reading R10): W = E + p is the positive root of
// W^2 - (1+cs2) E W + cs2 M^2 = 0; |M| is capped at (1 - delta) E (R9).
// CAP = false leaves out the |M| cap: for callers that redo every state with
// |v| > 0.99 in FP64, which every capped state is
template <class R, bool CAP = true>
__device__ __forceinline__ Prim<R> c2p_conformal(const V4<R> &U, const SchemeConsts<R> &k,
                                                 R &M2out, R &Wout, const Scheme &sc,
                                                 bool counting, unsigned *flags = nullptr) {
    Prim<R> q;
    // E <= 0 is vacuum (v = p = 0): with E clamped to 0 the cap forces M2c = 0,
    // so W = p = 0 follow from the same formulas and only 1/W needs a guard.
    // So is E <= emin, where E^2 underflows (R18): there W <= (1+c2)/2 E
    // falls under wmin and the velocity is set to 0 by the same guard.
    const R E = fmax_(U.e, R(0));
    const R M2 = fma_(U.t2, U.t2, fma_(U.t1, U.t1, U.n * U.n));
    const R E2 = E * E;
    const R cap2 = k.capf * E2;
    const R M2c = fmin_(M2, cap2);
    // W^2 - (1+c2) E W + c2 M^2 = 0: W = (1+c2)/2 E + sqrt(((1+c2)/2)^2 E^2 - c2 M^2),
    // the discriminant being positive for |M| < E
    const R W = fma_(k.hapc, E, dsqrt_(fma_(-k.cs2, M2c, k.hapc2 * E2)));
    R inv = W > k.wmin ? rcp_(W) : R(0);
    // energy flux (E + p) v_n = W (s M_n / W) = s M_n (0 in vacuum: there the
    // cap gives s = 0, or without it the guard below)
    R fe = CAP ? U.n : (W > k.wmin ? U.n : R(0));
    if (CAP && M2 > cap2) {   // |M| capped at (1 - delta) E (R9): v = s M / W
        const R s = dsqrt_(cap2 / M2);
        inv *= s;
        fe *= s;
        if (counting) count(sc, CNT_CAPPED);
        if (flags && U.e > k.emin) *flags |= FLAG_UNPHYSICAL;
    }
    q.vn = U.n * inv;
    q.fe = fe;
    q.p = W - E;
    q.W = W;
    M2out = M2c;
    Wout = W;
    return q;
}

// Tabulated EOS (reading R11): linear interpolation in ln e.  The node
// constants come from the scheme's constants in precision R.

// one fetch of node i: (p_i, dp_i, c2_i, dc2_i)
template <class R>
struct TabNode {
    R p, dp, c, dc;
};
template <class R>
__device__ __forceinline__ TabNode<R> tab_node(const Scheme &sc, int i);
template <>
__device__ __forceinline__ TabNode<float> tab_node<float>(const Scheme &sc, int i) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(sc.tab32) + i);
    return TabNode<float>{t.x, t.y, t.z, t.w};
}
template <>
__device__ __forceinline__ TabNode<double> tab_node<double>(const Scheme &sc, int i) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(sc.tab64) + 2 * i);
    const double2 b = __ldg(reinterpret_cast<const double2 *>(sc.tab64) + 2 * i + 1);
    return TabNode<double>{a.x, a.y, b.x, b.y};
}

// position of e in node units, u = (ln e - ln e_0) / h (e > 0).  FP32 takes
// log2 from the hardware and folds ln 2 / h and the offset into one FMA
template <class R>
__device__ __forceinline__ R table_u(const SchemeConsts<R> &k, R e);
template <>
__device__ __forceinline__ double table_u<double>(const SchemeConsts<double> &k, double e) {
    return (log(e) - k.lne_min) * k.inv_h;
}
template <>
__device__ __forceinline__ float table_u<float>(const SchemeConsts<float> &k, float e) {
    float l2;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(e));
    return fmaf(l2, k.l2_scale, k.l2_off);
}

template <class R>
__device__ __forceinline__ void eos_table(const Scheme &sc, R e, R &p, R &c2) {
    const SchemeConsts<R> &k = consts<R>(sc);
    if (!(e > R(0))) { p = R(0); c2 = R(1.0 / 3.0); return; }
    const R u = table_u<R>(k, e);
    if (u < R(0)) { p = e * R(1.0 / 3.0); c2 = R(1.0 / 3.0); return; }   // below the table
    const int n = sc.tab_n;
    if (u >= R(n - 1)) {
        const TabNode<R> t = tab_node<R>(sc, n - 1);
        c2 = t.c;
        p = fma_(c2, e - k.e_max, t.p);
        return;
    }
    const int i = int(u);   // u >= 0 here
    const R f = u - R(i);
    // p_i + f (p_{i+1} - p_i), and the same for c2 (linear in ln e, R11)
    const TabNode<R> t = tab_node<R>(sc, i);
    p = fma_(f, t.dp, t.p);
    c2 = fma_(f, t.dc, t.c);
}

// eos_table without branches: every case is evaluated from one node fetch
// (clamped to the table) and the result is selected, giving the same values
template <class R>
__device__ __forceinline__ void eos_table_sel(const Scheme &sc, R e, R &p, R &c2) {
    const SchemeConsts<R> &k = consts<R>(sc);
    const int n = sc.tab_n;
    const bool pos = e > R(0);
    const R u = table_u<R>(k, pos ? e : R(1));
    const bool below = u < R(0), above = u >= R(n - 1);
    const int i = below ? 0 : (above ? n - 1 : int(u));
    const TabNode<R> t = tab_node<R>(sc, i);
    const R f = u - R(i);
    const R third = R(1.0 / 3.0);
    R pp = fma_(f, t.dp, t.p), cc = fma_(f, t.dc, t.c);
    pp = above ? fma_(t.c, e - k.e_max, t.p) : pp;
    cc = above ? t.c : cc;
    pp = below ? e * third : pp;
    cc = below ? third : cc;
    p = pos ? pp : R(0);
    c2 = pos ? cc : third;
}

}  // namespace hy
#include "mlp_device.cuh"
namespace hy {

// Safeguarded Newton on f(v) = v - M / (E + p(E - M v)) in [0, M/E] (R11).
// Returns |v|; iters receives the iteration count.
enum { SEED_GIVEN = 100 };   // internal: start from the value passed in

// RCP: take 1/W and 1/f' as one reciprocal each (the FP32 sweeps) instead of
// three divisions
// the first iterate of the Newton solve, clamped to the bracket [0, hi]
template <class R>
__device__ __forceinline__ R newton_seed(const Scheme &sc, R E, R M, R M2, int seed, R given,
                                         R hi) {
    R v;
    if (seed == SEED_GIVEN) {
        v = given;
    } else if (seed == SEED_CONFORMAL) {
        const R a = R(4.0 / 3.0) * E;
        R disc = a * a - R(4.0 / 3.0) * M2;
        disc = disc < R(0) ? R(0) : disc;
        v = M / (R(0.5) * (a + dsqrt_(disc)));
    } else if (seed == SEED_MLP) {
        if (E > consts<R>(sc).mlp_emin) {
            v = R(mlp_seed_scalar(sc, float(log(double(E))), float(M / E)));
        } else {   // p = e/3 there: the closed form (as SEED_CONFORMAL)
            const R a = R(4.0 / 3.0) * E;
            R disc = a * a - R(4.0 / 3.0) * M2;
            disc = disc < R(0) ? R(0) : disc;
            v = M / (R(0.5) * (a + dsqrt_(disc)));
        }
    } else {
        v = R(0);
    }
    v = v < R(0) ? R(0) : v;
    v = v > hi ? hi : v;
    return v;
}

template <class R, bool RCP = false>
__device__ __forceinline__ R newton_speed(const Scheme &sc, R E, R M, R M2, int seed, R given,
                                          R &p_out, int &iters, unsigned *flags = nullptr) {
    R lo = R(0), hi = M / E;
    R v = newton_seed<R>(sc, E, M, M2, seed, given, hi);
    R p = R(0), c2 = R(0);
    int it = 0;
    bool conv = false;
    if (M == R(0)) {
        v = R(0);
        conv = true;
    } else {
        const int max_it = sc.newton_max_it;
        for (it = 1; it <= max_it; ++it) {
            eos_table<R>(sc, E - M * v, p, c2);
            const R W = E + p;
            const R iw = RCP ? rcp_(W) : R(1);
            const R f = RCP ? v - M * iw : v - M / W;
            if (f == R(0)) { conv = true; break; }
            if (f > R(0)) hi = v; else lo = v;
            const R fp = RCP ? R(1) - (c2 * M2) * (iw * iw) : R(1) - c2 * M2 / (W * W);
            R vn = RCP ? v - f * rcp_(fp) : v - f / fp;
            if (!(vn > lo && vn < hi)) vn = R(0.5) * (lo + hi);
            const R dv = vn - v;
            v = vn;
            if (fabs_(dv) <= R(sc.tol)) { conv = true; break; }
        }
        if (it > max_it) it = max_it;
    }
    if (!conv && flags) *flags |= FLAG_NEWTON;
    if (sc.counters) {
        count(sc, CNT_NEWTON_CALLS);
        count(sc, CNT_NEWTON_ITERS, (unsigned long long)it);
        if (!conv) count(sc, CNT_NEWTON_FAIL);
    }
    // p at the root.  A solve that stopped on |dv| <= tol keeps p of the last
    // evaluated iterate, which lies within tol of the root (p changes by at
    // most c2 M tol there); a solve that stopped on f = 0 evaluated it at v
    if (!conv || M == R(0)) eos_table<R>(sc, E - M * v, p, c2);
    p_out = p;
    iters = it;
    return v;
}

// Two independent solves of newton_speed in one loop. Each state keeps its own
// iterate, bracket, last p and exit iteration, so the results, iteration
// counts and flags equal those of two newton_speed calls; the loop body has no
// branch per state (the table lookup selects its case), so the two dependent
// chains of table fetch, reciprocal and Newton step interleave. A state with
// skip set takes no iteration and leaves its outputs untouched.
template <class R, bool RCP = false>
__device__ __forceinline__ void newton_speed2(const Scheme &sc, const R E[2], const R M[2],
                                              const R M2[2], const int seed[2], const R given[2],
                                              const bool skip[2], R v[2], R p_out[2],
                                              int iters[2], unsigned *flags = nullptr) {
    R lo[2], hi[2], p[2], c2[2];
    int it_s[2];
    bool conv[2], done[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        lo[s] = R(0);
        hi[s] = M[s] / E[s];
        v[s] = newton_seed<R>(sc, E[s], M[s], M2[s], seed[s], given[s], hi[s]);
        p[s] = R(0);
        c2[s] = R(0);
        it_s[s] = 0;
        conv[s] = false;
        done[s] = skip[s];
        if (!skip[s] && M[s] == R(0)) {
            v[s] = R(0);
            conv[s] = true;
            done[s] = true;
        }
    }
    const int max_it = sc.newton_max_it;
    for (int it = 1; it <= max_it; ++it) {
        if (done[0] && done[1]) break;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            R pn, cn;
            eos_table_sel<R>(sc, E[s] - M[s] * v[s], pn, cn);
            const R W = E[s] + pn;
            const R iw = RCP ? rcp_(W) : R(1);
            const R f = RCP ? v[s] - M[s] * iw : v[s] - M[s] / W;
            const bool act = !done[s];
            const bool hit = act && f == R(0);
            const R nlo = f > R(0) ? lo[s] : v[s];
            const R nhi = f > R(0) ? v[s] : hi[s];
            const R fp = RCP ? R(1) - (cn * M2[s]) * (iw * iw) : R(1) - cn * M2[s] / (W * W);
            R vn = RCP ? v[s] - f * rcp_(fp) : v[s] - f / fp;
            if (!(vn > nlo && vn < nhi)) vn = R(0.5) * (nlo + nhi);
            const R dv = vn - v[s];
            const bool step = act && !hit;
            p[s] = act ? pn : p[s];
            c2[s] = act ? cn : c2[s];
            lo[s] = step ? nlo : lo[s];
            hi[s] = step ? nhi : hi[s];
            v[s] = step ? vn : v[s];
            const bool fin = hit || (step && fabs_(dv) <= R(sc.tol));
            conv[s] = conv[s] || fin;
            it_s[s] = fin ? it : it_s[s];
            done[s] = done[s] || fin;
        }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (skip[s]) continue;
        if (!conv[s]) it_s[s] = max_it;
        if (!conv[s] && flags) *flags |= FLAG_NEWTON;
        if (sc.counters) {
            count(sc, CNT_NEWTON_CALLS);
            count(sc, CNT_NEWTON_ITERS, (unsigned long long)it_s[s]);
            if (!conv[s]) count(sc, CNT_NEWTON_FAIL);
        }
        if (!conv[s] || M[s] == R(0)) eos_table<R>(sc, E[s] - M[s] * v[s], p[s], c2[s]);
        p_out[s] = p[s];
        iters[s] = it_s[s];
    }
}

// MLP: seed from the warp-wide tensor-core MLP (the whole warp must be
// converged here); otherwise `seed` is SEED_ZERO, SEED_CONFORMAL or SEED_GIVEN
template <class R, bool MLP, bool RCP = false>
__device__ __forceinline__ Prim<R> c2p_table(const V4<R> &U, R delta, const Scheme &sc,
                                             int seed, R given, R &vmag,
                                             unsigned *flags = nullptr) {
    Prim<R> q;
    const R E = U.e;
    const R M2f = fma_(U.t2, U.t2, fma_(U.t1, U.t1, U.n * U.n));
    if (MLP) {
        // taken before any lane-dependent branch.  The network seeds the
        // states in the EOS's non-conformal range (E above mlp_emin); below it
        // the table is p = e/3 and the closed-form root is the better seed,
        // and a warp with no state above it skips the forward pass
        const bool need = E > consts<R>(sc).mlp_emin;
        if (__any_sync(0xffffffffu, need)) {
            const float Ef = E > R(0) ? float(E) : 1.0f;
            float xf = E > R(0) ? float(dsqrt_(M2f) / E) : 0.0f;
            xf = fminf(xf, 1.0f - float(delta));
            given = R(mlp_seed_warp(sc, __logf(Ef), xf));
        }
        seed = need ? SEED_GIVEN : SEED_CONFORMAL;
    }
    if (!(E > consts<R>(sc).emin)) {   // vacuum (R9, R18)
        q.vn = R(0); q.p = R(0); q.W = R(0); q.fe = R(0); vmag = R(0);
        return q;
    }
    const R cap = (R(1) - delta) * E;
    const R Mfull = dsqrt_(M2f);
    R M2 = M2f, M = Mfull;
    if (M2f > cap * cap) {
        M2 = cap * cap;
        M = cap;
        count(sc, CNT_CAPPED);
        if (flags) *flags |= FLAG_UNPHYSICAL;
    }
    R p;
    int it;
    const R v = newton_speed<R, RCP>(sc, E, M, M2, seed, given, p, it, flags);
    vmag = v;
    q.vn = Mfull > R(0) ? U.n * (v / Mfull) : R(0);
    q.p = p;
    q.W = E + p;
    q.fe = q.W * q.vn;
    return q;
}

// c2p_table for two states whose Newton solves run in one loop (newton_speed2):
// the same results as two c2p_table calls (the MLP seeds, warp-wide, are taken
// one after the other before any lane-dependent branch)
template <class R, bool MLP, bool RCP = false>
__device__ __forceinline__ void c2p_table2(const V4<R> U[2], R delta, const Scheme &sc, int seed0,
                                           Prim<R> q[2], R vmag[2], unsigned *flags = nullptr) {
    R E[2], M2f[2], given[2] = {R(0), R(0)};
    int seed[2] = {seed0, seed0};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        E[s] = U[s].e;
        M2f[s] = fma_(U[s].t2, U[s].t2, fma_(U[s].t1, U[s].t1, U[s].n * U[s].n));
    }
    if (MLP) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const bool need = E[s] > consts<R>(sc).mlp_emin;
            if (__any_sync(0xffffffffu, need)) {
                const float Ef = E[s] > R(0) ? float(E[s]) : 1.0f;
                float xf = E[s] > R(0) ? float(dsqrt_(M2f[s]) / E[s]) : 0.0f;
                xf = fminf(xf, 1.0f - float(delta));
                given[s] = R(mlp_seed_warp(sc, __logf(Ef), xf));
            }
            seed[s] = need ? SEED_GIVEN : SEED_CONFORMAL;
        }
    }
    bool vac[2];
    R M[2], M2[2], Mfull[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        vac[s] = !(E[s] > consts<R>(sc).emin);   // vacuum (R9, R18)
        const R cap = (R(1) - delta) * E[s];
        Mfull[s] = dsqrt_(M2f[s]);
        M2[s] = M2f[s];
        M[s] = Mfull[s];
        if (!vac[s] && M2f[s] > cap * cap) {
            M2[s] = cap * cap;
            M[s] = cap;
            count(sc, CNT_CAPPED);
            if (flags) *flags |= FLAG_UNPHYSICAL;
        }
    }
    R v[2], p[2];
    int it[2];
    newton_speed2<R, RCP>(sc, E, M, M2, seed, given, vac, v, p, it, flags);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (vac[s]) {
            q[s].vn = R(0); q[s].p = R(0); q[s].W = R(0); q[s].fe = R(0); vmag[s] = R(0);
        } else {
            vmag[s] = v[s];
            q[s].vn = Mfull[s] > R(0) ? U[s].n * (v[s] / Mfull[s]) : R(0);
            q[s].p = p[s];
            q[s].W = E[s] + p[s];
            q[s].fe = q[s].W * q[s].vn;
        }
    }
}

// Precision policy of a sweep: storage/flux type R and the cons->prim rule.
enum { PREC_F64 = 0, PREC_F32 = 1, PREC_MIXED = 2 };

// MUSTA2: the kernel writes out the two-stage MUSTA-FORCE (the RK3 kernels,
// whose registers are capped, keep the loop)
template <class R, int PREC, int EOSK, int LIM = -1, bool COUNT = true, bool MUSTA2 = true,
          bool CH = false>
struct Physics {
    using V = VS<R, CH>;   // the fields a sweep carries
    static constexpr bool kCharge = CH;
    Scheme sc;
    R al_, hclf_;   // alpha dt/dx and 1 / (4 alpha dt/dx) of the current sweep
    // FLAG_* bits this thread met since the last report_flags (a |M| cap, a
    // face fallback, a Newton solve that hit its cap)
    mutable unsigned flags_ = 0;

    __device__ __forceinline__ const SchemeConsts<R> &K() const { return consts<R>(sc); }

    // per-event constants of a sweep with lam = dt / dx
    __device__ __forceinline__ void set_lam(R lam) {
        al_ = K().alpha * lam;
        hclf_ = R(0.25) / al_;
    }

    // cons -> prim for a flux evaluation (Eq. 23)
    __device__ __forceinline__ Prim<R> prim(const V4<R> &U) const {
        if (EOSK == EOS_CONFORMAL) {
            R M2, W;
            // mixed: a capped state has |v| > 0.99 and is redone in FP64 below
            Prim<R> q = c2p_conformal<R, PREC != PREC_MIXED>(U, K(), M2, W, sc, COUNT, &flags_);
            if (PREC == PREC_MIXED) {
                // |v|^2 = M2 / W^2 > 0.99^2: redo in double (cancellation in W - E)
                if (M2 > R(0.9801) * W * W) {
                    V4<double> D = v4<double>(U.e, U.n, U.t1, U.t2);
                    double M2d, Wd;
                    Prim<double> qd =
                        c2p_conformal<double>(D, sc.c64, M2d, Wd, sc, COUNT, &flags_);
                    q.vn = R(qd.vn);
                    q.p = R(qd.p);
                    q.W = R(qd.W);
                    q.fe = R(qd.fe);
                    if (COUNT) count(sc, CNT_F64_REDO);
                }
            }
            return q;
        } else {
            R vmag;
            constexpr bool F32 = sizeof(R) == 4;
            Prim<R> q = c2p_table<R, EOSK == EOS_TABLE_MLP, F32>(U, K().delta, sc, sc.seed, R(0),
                                                                 vmag, &flags_);
            if (PREC == PREC_MIXED) table_redo(U, vmag, q);
            return q;
        }
    }
    // mixed precision, tabulated EOS: |v| > 0.99 is redone in double, seeded
    // by the float root
    __device__ __forceinline__ void table_redo(const V4<R> &U, R vmag, Prim<R> &q) const {
        if (vmag > R(0.99)) {
            V4<double> D = v4<double>(U.e, U.n, U.t1, U.t2);
            double vd;
            Prim<double> qd = c2p_table<double, false>(D, DELTA_F64, sc, SEED_GIVEN,
                                                       double(vmag), vd, &flags_);
            q.vn = R(qd.vn);
            q.p = R(qd.p);
            q.W = R(qd.W);
            q.fe = R(qd.fe);
            count(sc, CNT_F64_REDO);
        }
    }
    // prim() of two states; with the tabulated EOS their Newton solves share
    // one loop (c2p_table2), with the same results
    __device__ __forceinline__ void prim2(const V4<R> &A, const V4<R> &B, Prim<R> &qa,
                                          Prim<R> &qb) const {
        if constexpr (EOSK == EOS_CONFORMAL) {
            qa = prim(A);
            qb = prim(B);
        } else {
            constexpr bool F32 = sizeof(R) == 4;
            const V4<R> U[2] = {A, B};
            Prim<R> q[2];
            R vmag[2];
            c2p_table2<R, EOSK == EOS_TABLE_MLP, F32>(U, K().delta, sc, sc.seed, q, vmag, &flags_);
            if (PREC == PREC_MIXED) {
                table_redo(A, vmag[0], q[0]);
                table_redo(B, vmag[1], q[1]);
            }
            qa = q[0];
            qb = q[1];
        }
    }

    // Eq. 3 along the sweep axis
    __device__ __forceinline__ V flux(const V &U) const { return flux_of(U, prim(head(U))); }
    // Eq. 3 along the axis from the primitives q of U:
    // ((E + p) v_n, M_n v_n + p, M_t1 v_n, M_t2 v_n, R v_n)
    __device__ __forceinline__ static V flux_of(const V &U, const Prim<R> &q) {
        R t1, t2;
        tmul<R>(q.vn, head(U), t1, t2);
        return make(v4<R>(q.fe, fma_(U.n, q.vn, q.p), t1, t2), U, q.vn);
    }
    // flux() of two states (the pairs of Hancock faces and of MUSTA-FORCE
    // interface states); with the tabulated EOS their cons->prim solves
    // interleave (prim2)
    __device__ __forceinline__ void flux2(const V &A, const V &B, V &FA, V &FB) const {
        if constexpr (EOSK == EOS_CONFORMAL) {
            FA = flux(A);
            FB = flux(B);
        } else {
            Prim<R> qa, qb;
            prim2(head(A), head(B), qa, qb);
            FA = flux_of(A, qa);
            FB = flux_of(B, qb);
        }
    }
    // the four energy-momentum components, with the charge flux R v_n when carried
    __device__ __forceinline__ static V make(const V4<R> &f, const V &U, R vn) {
        if constexpr (CH) return with_r(f, U.r * vn);
        else return f;
    }

    // The conformal FP32/FP64 sweeps take the |M| cap (R9) per group of flux
    // evaluations instead of per evaluation: the group runs without it and
    // only records whether any state exceeded the cap (one predicate-or per
    // evaluation); where a lane of the warp recorded one, the warp redoes the
    // group with the capped flux (a warp-uniform branch); so it does where a
    // lane met a vacuum state (W <= wmin).  Where neither applies the two give
    // the same bits, so the results are those of flux() throughout.  Counting
    // runs keep flux().
    // The mixed sweeps group their FP64 redo the same way: a group is redone
    // through flux() where a state's FP32 recovery gives |v| > 0.99.
    static constexpr bool CAP_GROUPS = EOSK == EOS_CONFORMAL && !COUNT;
    // The RK2 kernels with the limiter fixed at compile time are launched
    // only with the Hancock step on and, where the MUSTA-FORCE stages are
    // written out (conformal EOS), with k = 2; their loop tests neither.  (The
    // register-capped RK3 kernels keep the tests: without the branch their
    // schedule spills.)
    static constexpr bool FIXED = LIM >= 0 && MUSTA2;

    __device__ __forceinline__ V flux_uncapped(const V &U, bool &capped) const {
        const SchemeConsts<R> &k = K();
        const R E = fmax_(U.e, R(0));
        const R M2 = fma_(U.t2, U.t2, fma_(U.t1, U.t1, U.n * U.n));
        const R E2 = E * E;
        const R cap2 = k.capf * E2;
        // a state over the cap sends the group to the capped redo, so outside
        // the mixed test below M^2 needs no clamp: where the cap does not act,
        // min(M^2, cap^2) = M^2
        const R M2c = PREC == PREC_MIXED ? fmin_(M2, cap2) : M2;
        const R W = fma_(k.hapc, E, dsqrt_(fma_(-k.cs2, M2c, k.hapc2 * E2)));
        const bool live = W > k.wmin;
        R fe, inv;
        if constexpr (PREC == PREC_MIXED) {   // c2p_conformal<R, false> and prim()'s test
            // a vacuum state goes to the redo (as below)
            inv = rcp_(W);
            fe = U.n;
            capped = capped || M2c > R(0.9801) * W * W || !live;
        } else {
            // a vacuum state (W <= wmin) also sends the group to the redo,
            // whose cons->prim guards it; here 1/W needs no guard
            inv = rcp_(W);
            fe = U.n;
            capped = capped || M2 > cap2 || !live;
        }
        const R vn = U.n * inv;
        R t1, t2;
        tmul<R>(vn, head(U), t1, t2);
        return make(v4<R>(fe, fma_(U.n, vn, W - E), t1, t2), U, vn);
    }
    template <bool UNCAPPED>
    __device__ __forceinline__ V flux_g(const V &U, bool &capped) const {
        if constexpr (UNCAPPED) return flux_uncapped(U, capped);
        else return flux(U);
    }

    // CFL rate of one cell (reading R8): max over swept axes of |lambda^+-| / dx,
    // axes given in the sweep's slot order (n, t1, t2) with ih = 1/dx (0: not swept);
    // iso: every swept axis has spacing 1 / ih_n
    __device__ __forceinline__ R rate(const V4<R> &U, R ih_n, R ih_t1, R ih_t2, bool iso) const {
        if (EOSK == EOS_CONFORMAL && iso) {
            // At fixed |v| the speed grows with |v_d| (its derivative in |v_d| has
            // the sign of 1 - v_d^2), so the axis of largest |v_d| gives the max;
            // with k = c2 and D = 1 - |v|^2 k:
            //   lambda = (|v_d| (1 - k) + c sqrt((1 - |v|^2) (D - v_d^2 (1 - k)))) / D
            const R E = fmax_(U.e, R(0));
            const R M2 = fma_(U.t2, U.t2, fma_(U.t1, U.t1, U.n * U.n));
            const SchemeConsts<R> &k = K();
            const R E2 = E * E;
            const R cap2 = k.capf * E2;
            const R M2c = fmin_(M2, cap2);
            const R W = fma_(k.hapc, E, dsqrt_(fma_(-k.cs2, M2c, k.hapc2 * E2)));
            const R inv = W > k.wmin ? rcp_(W) : R(0);   // vacuum: v = 0, speed c
            R am = fabs_(U.n);
            if (ih_t1 > R(0)) am = fmax_(am, fabs_(U.t1));
            if (ih_t2 > R(0)) am = fmax_(am, fabs_(U.t2));
            R a = am * inv;                       // largest |v_d|
            if (M2 > cap2) a *= dsqrt_(cap2 / M2);   // capped |M| (R9)
            const R v2 = (M2c * inv) * inv;
            const R D = fma_(-v2, k.cs2, R(1));
            const R rad = fmax_((R(1) - v2) * fma_(-a * a, k.k1, D), R(0));
            const R lam = fma_(k.cs, dsqrt_(rad), a * k.k1) * rcp_(D);
            return lam * ih_n;
        }
        const R E = U.e;
        const R cs2 = K().cs2;
        R M2 = U.n * U.n + U.t1 * U.t1 + U.t2 * U.t2;
        if (!(E > K().emin)) {   // vacuum: v = 0, e = 0, the speed of sound of e = 0
            R p0, c20;
            if (EOSK == EOS_CONFORMAL) c20 = cs2;
            else eos_table<R>(sc, R(0), p0, c20);
            const R m0 = dsqrt_(c20);
            R m = m0 * ih_n;
            if (ih_t1 > R(0)) m = fmax_(m, m0 * ih_t1);
            if (ih_t2 > R(0)) m = fmax_(m, m0 * ih_t2);
            return m;
        }
        const R cap2 = K().capf * E * E;
        R s = R(1);
        if (M2 > cap2) {
            s = dsqrt_(cap2 / M2);
            M2 = cap2;
        }
        R vn, vt1, vt2, c2;
        if (EOSK == EOS_CONFORMAL) {
            const R hapc = R(0.5) * (R(1) + cs2);
            const R W = hapc * E + dsqrt_((hapc * hapc) * (E * E) - cs2 * M2);
            const R inv = s / W;
            vn = U.n * inv; vt1 = U.t1 * inv; vt2 = U.t2 * inv;
            c2 = cs2;
        } else {
            R vmag;
            // lane-wise: no warp-wide MLP seed here (the rate may run in divergent code)
            const int seed = sc.seed == SEED_MLP ? SEED_CONFORMAL : sc.seed;
            const Prim<R> q = c2p_table<R, false>(U, K().delta, sc, seed, R(0), vmag);
            const R Mfull = dsqrt_(U.n * U.n + U.t1 * U.t1 + U.t2 * U.t2);
            const R sc_ = Mfull > R(0) ? vmag / Mfull : R(0);
            vn = U.n * sc_; vt1 = U.t1 * sc_; vt2 = U.t2 * sc_;
            R p;
            eos_table<R>(sc, E - dsqrt_(M2) * vmag, p, c2);
            (void)q;
        }
        const R v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
        const R cs = dsqrt_(c2);
        const R inv_den = R(1) / (R(1) - v2 * c2);
        auto one = [&](R vd, R ih) {
            R rad = (R(1) - v2) * (R(1) - vd * vd - (v2 - vd * vd) * c2);
            rad = rad < R(0) ? R(0) : rad;
            return (fabs_(vd * (R(1) - c2)) + cs * dsqrt_(rad)) * inv_den * ih;
        };
        if (iso) {
            // at fixed |v| the speed grows with |v_d| (its derivative in |v_d|
            // has the sign of 1 - v_d^2), so the axis of largest |v_d| gives the max
            R a = fabs_(vn);
            if (ih_t1 > R(0)) a = fmax_(a, fabs_(vt1));
            if (ih_t2 > R(0)) a = fmax_(a, fabs_(vt2));
            return one(a, ih_n);
        }
        R m = one(vn, ih_n);
        if (ih_t1 > R(0)) m = fmax_(m, one(vt1, ih_t1));
        if (ih_t2 > R(0)) m = fmax_(m, one(vt2, ih_t2));
        return m;
    }

    template <class VV>
    __device__ __forceinline__ bool admissible(const VV &U) const {
        const R M2 = fma_(U.t2, U.t2, fma_(U.t1, U.t1, U.n * U.n));
        const R cap = K().omd * U.e;
        return U.e > R(0) && M2 < cap * cap;
    }

    // Limited MUSCL faces (Eq. 15-17) and the Hancock half step (Eq. 13, the
    // sweep-axis term), with the admissibility fallback (R9).
    __device__ __forceinline__ void faces(const V &vm, const V &v0, const V &vp, R lam, V &ul,
                                          V &ur) const {
        const int lim = sc.limiter;
        const R half = R(0.5);
        const V a = vsub(v0, vm), b = vsub(vp, v0);
        const V4<R> sl4 = v4<R>(slope_ct<LIM, R>(lim, a.e, b.e), slope_ct<LIM, R>(lim, a.n, b.n),
                                slope_ct<LIM, R>(lim, a.t1, b.t1),
                                slope_ct<LIM, R>(lim, a.t2, b.t2));
        V sl;
        if constexpr (CH) sl = with_r(sl4, slope_ct<LIM, R>(lim, a.r, b.r));
        else sl = sl4;
        ul = vfma<R>(-half, sl, v0);
        ur = vfma<R>(half, sl, v0);
        if (FIXED || sc.hancock) {
            V FL, FR;
            if constexpr (CAP_GROUPS) {
                bool capped = false;
                FL = flux_uncapped(ul, capped);
                FR = flux_uncapped(ur, capped);
                // the warp redoes the group together (a warp-uniform branch):
                // lanes that met no cap or vacuum get the same bits again
                if (__any_sync(0xffffffffu, capped)) { FL = flux(ul); FR = flux(ur); }
            } else {
                flux2(ul, ur, FL, FR);
            }
            const V d = vsub(FL, FR);
            const R hl = half * lam;
            ul = vfma<R>(hl, d, ul);
            ur = vfma<R>(hl, d, ur);
        }
        if (!admissible(ul) || !admissible(ur)) {
            ul = v0; ur = v0;
            if (COUNT) count(sc, CNT_FACE_FALLBACK);
            flags_ |= FLAG_UNPHYSICAL;
        }
    }

    // MUSTA-FORCE interface flux (Sec. 2.4 steps 1-5, Eq. 8-11; R1, R2, R4)
    __device__ __forceinline__ V musta(const V &UL, const V &UR, R lam) const {
        bool capped = false;
        if constexpr (CAP_GROUPS) {
            V F;
            if (MUSTA2 && (FIXED || sc.stages == 2)) {
                // two stages written out, so that the predicted states take
                // fresh registers while the inputs stay for a redo
                V FL, FR;
                const V F0 = musta_stage<true>(UL, UR, FL, FR, capped);
                const V UL1 = vfma<R>(-lam, vsub(F0, FL), UL);
                const V UR1 = vfma<R>(-lam, vsub(FR, F0), UR);
                F = musta_stage<true>(UL1, UR1, FL, FR, capped);
            } else {
                F = musta_g<true>(UL, UR, lam, capped);
            }
            if (!__any_sync(0xffffffffu, capped)) return F;   // warp-uniform, as in faces()
        }
        return musta_g<false>(UL, UR, lam, capped);
    }
    // one FORCE evaluation of Sec. 2.4 (steps 1-4) at (UL, UR), with F(UL), F(UR);
    // the conformal form F_lw / 2 = F(2 U_lw) / 4 (CAP_GROUPS implies p = c2 e)
    template <bool UNCAPPED>
    __device__ __forceinline__ V musta_stage(const V &UL, const V &UR, V &FL, V &FR,
                                             bool &capped) const {
        const R q4 = R(0.25);
        FL = flux_g<UNCAPPED>(UL, capped);
        FR = flux_g<UNCAPPED>(UR, capped);
        const V Flf = vfma<R>(-hclf_, vsub(UR, UL), vmul<R>(q4, vadd(FL, FR)));
        const V Ulw2 = vfma<R>(-al_, vsub(FR, FL), vadd(UL, UR));
        return vfma<R>(q4, flux_g<UNCAPPED>(Ulw2, capped), Flf);
    }
    template <bool UNCAPPED>
    __device__ __forceinline__ V musta_g(V UL, V UR, R lam, bool &capped) const {
        const R al = al_;
        const R clw = R(0.5) * al;
        const R half = R(0.5), q4 = R(0.25), hclf = hclf_;
        V Fc;
        const int k = sc.stages;
#pragma unroll 1
        for (int l = 0; l < k; ++l) {
            V FL, FR;
            if constexpr (UNCAPPED) {
                FL = flux_uncapped(UL, capped);
                FR = flux_uncapped(UR, capped);
            } else {
                flux2(UL, UR, FL, FR);
            }
            // F = 1/2 F_lw + 1/2 F_lf = 1/2 F_lw + 1/4 (F_L + F_R) - (clf/2) (U_R - U_L)
            const V Flf = vfma<R>(-hclf, vsub(UR, UL), vmul<R>(q4, vadd(FL, FR)));
            if (EOSK == EOS_CONFORMAL) {
                // p = c2 e makes the flux homogeneous of degree 1, F(2U) = 2 F(U),
                // and doubling is exact: take F(2 U_lw) / 4 for F_lw / 2
                const V Ulw2 = vfma<R>(-al, vsub(FR, FL), vadd(UL, UR));
                Fc = vfma<R>(q4, flux_g<UNCAPPED>(Ulw2, capped), Flf);
            } else {
                const V Ulw = vfma<R>(-clw, vsub(FR, FL), vmul<R>(half, vadd(UL, UR)));
                Fc = vfma<R>(half, flux_g<UNCAPPED>(Ulw, capped), Flf);
            }
            if (l < k - 1) {
                UL = vfma<R>(-lam, vsub(Fc, FL), UL);
                UR = vfma<R>(-lam, vsub(FR, Fc), UR);
            }
        }
        return Fc;
    }
};

// One Runge-Kutta stage as a streaming engine.  After push(V_j):
//   window (w0, w1, w2) = (V_{j-2}, V_{j-1}, V_j); faces of cell j-1 are
//   computed; the flux of interface (j-2)+1/2 once faces of j-2 exist; and
//   the divergence D_{j-2} = F_{j-3/2} - F_{j-5/2} once both fluxes exist.
template <class V>
struct Stage {
    V w0, w1, w2, urp, fp;
    int n;

    template <class PH, class R>
    __device__ __forceinline__ bool push(const V &v, const PH &ph, R lam, V &cell, V &D) {
        w0 = w1; w1 = w2; w2 = v;
        ++n;
        if (n < 3) return false;
        V ul, ur;
        ph.faces(w0, w1, w2, lam, ul, ur);
        bool out = false;
        if (n >= 4) {
            const V F = ph.musta(urp, ul, lam);
            if (n >= 5) {
                D = vsub(F, fp);
                cell = w0;
                out = true;
            }
            fp = F;
        }
        urp = ur;
        return out;
    }

    // push once the window is full (n >= 5): always yields an output
    template <class PH, class R>
    __device__ __forceinline__ void push_full(const V &v, const PH &ph, R lam, V &cell, V &D) {
        w0 = w1; w1 = w2; w2 = v;
        V ul, ur;
        ph.faces(w0, w1, w2, lam, ul, ur);
        const V F = ph.musta(urp, ul, lam);
        D = vsub(F, fp);
        cell = w0;
        fp = F;
        urp = ur;
    }
};

// Where a thread's pencil lives: field q of cell j is base[fo[q] + j * stride],
// with fo = (0, M_axis, M_t1, M_t2[, R]) field offsets in elements.
template <class R, bool CH = false>
struct Pencil {
    const R *in;
    R *out;
    int fo1, fo2, fo3;    // offsets of the three momentum slots (E is at 0)
    int fo4;              // offset of the charge (CH)
    int stride;
    int N;

    __device__ __forceinline__ VS<R, CH> load(int j) const {
        const R *p = in + j * stride;
        const V4<R> v = v4<R>(__ldg(p), __ldg(p + fo1), __ldg(p + fo2), __ldg(p + fo3));
        if constexpr (CH) return with_r(v, __ldg(p + fo4));
        else return v;
    }
    __device__ __forceinline__ void store(int j, const VS<R, CH> &v) const {
        R *p = out + j * stride;
        p[0] = v.e; p[fo1] = v.n; p[fo2] = v.t1; p[fo3] = v.t2;
        if constexpr (CH) p[fo4] = v.r;
    }
};

__device__ __forceinline__ int wrap_index(int j, int N, int bc) {
    if (bc == BC_OUTFLOW) return j < 0 ? 0 : (j >= N ? N - 1 : j);
    while (j < 0) j += N;
    while (j >= N) j -= N;
    return j;
}

// Pick the value stage k+1 receives for position p from the last outputs of
// stage k (q[0] newest, age a = cell index of q[0] minus the wanted cell).
// With outflow ends, ghost positions p < 0 take the output of cell 0 and
// p >= N the output of cell N-1 (saved in `last`), as the ghost fill of a
// stage input does.
template <class V, int DEPTH>
__device__ __forceinline__ V pick(const V (&q)[DEPTH], int newest, int p, int N, int bc,
                                  const V &last) {
    if (bc == BC_OUTFLOW) {
        if (p >= N) return last;
        if (p < 0) p = 0;
    }
    const int age = newest - p;
    V x = q[DEPTH - 1];
#pragma unroll
    for (int a = 0; a < DEPTH - 1; ++a)
        if (age == a) x = q[a];
    return x;
}

template <class V, int DEPTH>
__device__ __forceinline__ void shift_in(V (&q)[DEPTH], const V &v) {
#pragma unroll
    for (int a = DEPTH - 1; a > 0; --a) q[a] = q[a - 1];
    q[0] = v;
}

// March one segment of a pencil: the RK stages of Eq. 5-7 fused in registers.
// Every thread runs the same schedule (T = L + 4, L + 10 or L + 16 steps for
// RK1/2/3), so a warp stays converged; stage k+1 starts a fixed number of
// steps after stage k, reading stage k's outputs from a short register queue.
// Cells [s0, s_end) are stored; the segment's nominal length L may run past
// the pencil end (those cells are computed with wrapped or clamped inputs and
// not stored).
// The CFL rate for the next step's dt (ih = 1/dx per slot; ih_n > 0 switches
// it on) is evaluated for the stored cells only, in lane-divergent code, which
// is why rate() never uses the warp-wide MLP seed.
template <class R>
struct RateAcc {
    R ih_n, ih_t1, ih_t2;
    R m;
    bool iso;   // the swept axes share one spacing
};

template <class R, int RK, bool RATE, class PH>
__device__ __forceinline__ void march(const PH &ph, const Pencil<R, PH::kCharge> &P, int s0, int L,
                                      int s_end, int bc, R lam, bool do_store, RateAcc<R> &ra) {
    using V = typename PH::V;
    const int N = P.N;
    if (!positive(lam)) {   // finished event: copy through
        if (do_store)
            for (int o = s0; o < s_end; ++o) P.store(o, P.load(o));
        return;
    }
    const bool rate_on = RATE && positive(ra.ih_n);
    const R third = R(1.0 / 3.0), two3 = R(2.0 / 3.0), q3 = R(0.75), q1c = R(0.25), half = R(0.5);
    Stage<V> st1, st2, st3;
    st1.n = 0; st2.n = 0; st3.n = 0;
    V cell, D;
    constexpr int H = 2 * RK;                 // halo of the stage-1 input
    constexpr int T_EXTRA = RK == 1 ? 4 : (RK == 2 ? 10 : 16);
    const int T = L + T_EXTRA;
    const int js = s0 - H;
    V qa[3];
    V lastA = vzero<V>(), lastB = lastA;
    V nxt = P.load(wrap_index(js, N, bc));
    if constexpr (RK == 2) {
        // One loop body for every step: both engines push unchecked from t = 0
        // on windows filled with a state at rest (E = 1, M = 0).  Their outputs
        // before the windows fill (t < 4 for stage 1, t < 10 for stage 2) are
        // never used or stored; every stored cell is
        // computed by the same instructions whatever the segment layout, so
        // results do not depend on the launch shape.  (A zero fill would be
        // vacuum, which sends the grouped flux evaluations to their redo.)
        V zero = vzero<V>();
        zero.e = R(1);
        st1.w0 = st1.w1 = st1.w2 = st1.urp = st1.fp = zero;
        st2.w0 = st2.w1 = st2.w2 = st2.urp = st2.fp = zero;
        qa[0] = qa[1] = qa[2] = zero;
        int jn = wrap_index(js + 1, N, bc);
        int jc = js + 1;
        // the cell reloaded for the RK combination, one step ahead like the input
        int on = wrap_index(s0 - 9, N, bc);
        int oc = s0 - 9;
        V U0n = P.load(wrap_index(s0 - 10, N, bc));
#pragma unroll 1
        for (int t = 0; t < T; ++t) {
            const V Vc = nxt;
            const V U0 = U0n;
            if (t + 1 < T) {
                nxt = P.load(jn);
                U0n = P.load(on);
            }
            ++jc;
            jn = (bc == BC_OUTFLOW) ? min(max(jc, 0), N - 1) : (jn + 1 == N ? 0 : jn + 1);
            ++oc;
            on = (bc == BC_OUTFLOW) ? min(max(oc, 0), N - 1) : (on + 1 == N ? 0 : on + 1);
            st1.push_full(Vc, ph, lam, cell, D);
            const int i = js + t - 2;                 // stage-1 output cell
            const V X = vfma<R>(-lam, D, cell);   // U1 = U + dt L(U)
            shift_in(qa, X);
            if (i == N - 1) lastA = X;
            const V Y = pick(qa, i, t + s0 - 8, N, bc, lastA);
            V c, Dl;
            st2.push_full(Y, ph, lam, c, Dl);
            const int o = t + s0 - 10;                // finished cell
            // Eq. 6: U^{n+1} = 1/2 (U + U1 + dt L(U1))
            const V r = vmul<R>(half, vfma<R>(-lam, Dl, vadd(U0, c)));
            const bool keep = do_store && o >= s0 && o < s_end;
            if constexpr (RATE) {
                if (rate_on && keep) {
                    const R rr = ph.rate(head(r), ra.ih_n, ra.ih_t1, ra.ih_t2, ra.iso);
                    ra.m = (rr > ra.m || rr != rr) ? rr : ra.m;
                }
            }
            if (keep) P.store(o, r);
            // the steps before the first finished cell run on at-rest-filled
            // windows: what they met is not a state of the grid
            if (t < 10) ph.flags_ = 0;
        }
        return;
    }
    if constexpr (RK == 3) {
        // The same uniform loop for Eq. 7: three engines push from step 0 on
        // windows filled with a state at rest (as for RK2); each stage reads
        // the previous stage's output two cells behind its newest (the 2
        // ghost cells of a stage).
        // Stage 1 outputs cell t+s0-8, stage 2 cell t+s0-12, stage 3 t+s0-16.
        V zero = vzero<V>();
        zero.e = R(1);
        st1.w0 = st1.w1 = st1.w2 = st1.urp = st1.fp = zero;
        st2.w0 = st2.w1 = st2.w2 = st2.urp = st2.fp = zero;
        st3.w0 = st3.w1 = st3.w2 = st3.urp = st3.fp = zero;
        V q1[3] = {zero, zero, zero}, q2[3] = {zero, zero, zero};
        const int T3 = L + 16;
        int jn = wrap_index(js + 1, N, bc), jc = js + 1;
        // U^n of the stage-2 and stage-3 output cells, one step ahead
        int an = wrap_index(s0 - 11, N, bc), ac = s0 - 11;
        int bn = wrap_index(s0 - 15, N, bc), bcn = s0 - 15;
        V Ua = P.load(wrap_index(s0 - 12, N, bc));
        V Ub = P.load(wrap_index(s0 - 16, N, bc));
#pragma unroll 1
        for (int t = 0; t < T3; ++t) {
            const V Vc = nxt, U0 = Ua, U00 = Ub;
            if (t + 1 < T3) {
                nxt = P.load(jn);
                Ua = P.load(an);
                Ub = P.load(bn);
            }
            ++jc; ++ac; ++bcn;
            if (bc == BC_OUTFLOW) {
                jn = min(max(jc, 0), N - 1);
                an = min(max(ac, 0), N - 1);
                bn = min(max(bcn, 0), N - 1);
            } else {
                jn = jn + 1 == N ? 0 : jn + 1;
                an = an + 1 == N ? 0 : an + 1;
                bn = bn + 1 == N ? 0 : bn + 1;
            }
            st1.push_full(Vc, ph, lam, cell, D);
            const int i = t + s0 - 8;                  // stage-1 output cell
            const V X = vfma<R>(-lam, D, cell);    // U1 = U + dt L(U)
            shift_in(q1, X);
            if (i == N - 1) lastA = X;
            V c2, D2;
            st2.push_full(pick(q1, i, t + s0 - 10, N, bc, lastA), ph, lam, c2, D2);
            const int i2 = t + s0 - 12;                // stage-2 output cell
            // U2 = 3/4 U + 1/4 (U1 + dt L(U1))
            const V Z = vfma<R>(q3, U0, vmul<R>(q1c, vfma<R>(-lam, D2, c2)));
            shift_in(q2, Z);
            if (i2 == N - 1) lastB = Z;
            V c3, D3;
            st3.push_full(pick(q2, i2, t + s0 - 14, N, bc, lastB), ph, lam, c3, D3);
            const int o = t + s0 - 16;                 // finished cell
            // U^{n+1} = 1/3 U + 2/3 (U2 + dt L(U2))
            const V r = vfma<R>(third, U00, vmul<R>(two3, vfma<R>(-lam, D3, c3)));
            const bool keep = do_store && o >= s0 && o < s_end;
            if constexpr (RATE) {
                if (rate_on && keep) {
                    const R rr = ph.rate(head(r), ra.ih_n, ra.ih_t1, ra.ih_t2, ra.iso);
                    ra.m = (rr > ra.m || rr != rr) ? rr : ra.m;
                }
            }
            if (keep) P.store(o, r);
            if (t < 16) ph.flags_ = 0;   // windows not yet filled (as for RK2)
        }
        return;
    }
    if constexpr (RK == 1) {
        // RK1 (plain MUSCL-Hancock with MUSTA-FORCE fluxes)
#pragma unroll 1
        for (int t = 0; t < T; ++t) {
            const V Vc = nxt;
            if (t + 1 < T) nxt = P.load(wrap_index(js + t + 1, N, bc));
            if (!st1.push(Vc, ph, lam, cell, D)) continue;
            const int i = js + t - 2;   // output cell
            const V X = vfma<R>(-lam, D, cell);   // U + dt L(U)
            if constexpr (RATE) {
                if (rate_on) {
                    const R rr = ph.rate(head(X), ra.ih_n, ra.ih_t1, ra.ih_t2, ra.iso);
                    if (do_store && i < s_end) ra.m = (rr > ra.m || rr != rr) ? rr : ra.m;
                }
            }
            if (do_store && i < s_end) P.store(i, X);
        }
    }
}

// ---------------------------------------------------------------- staged x sweep
// Along x each thread marches its own row, so a warp touches 32 rows at once.
// Loading each row cell by cell leaves every 32-byte sector to be assembled
// from 8 separate requests spread over 8 steps; L1 cannot hold the 32 rows x 4
// fields of all resident warps that long, so sectors were fetched from DRAM
// several times and written back in pieces.  Instead each warp stages its 32
// rows through shared memory in whole sectors: every 8 steps the lanes copy
// the next 8 cells of all 32 rows (4 rows x 8 cells per instruction, with
// cp.async, so the copy overlaps the following two steps of arithmetic) into
// a 16-cell ring per row and field, and finished cells go back 8 at a time
// from an output ring.  In step space (slot = step & 15) the ring holds steps
// [t - 6, t + 2) and, once a copy lands, up to t + 10: the input of step t
// and the cell 6 steps behind it that the RK combination reloads.  Fills and
// flushes are placed so that rows whose start is 8-cell aligned move whole
// sectors.
constexpr int XR = 16;        // input ring: steps per row
constexpr int XRS = XR + 1;   // row stride (odd: conflict-free column reads)
// rows per iteration of the output flush, with and without the CFL rate (1
// and 8, or 2 and 4, measured the same)
constexpr int kFlushUnrollRate = 2;
constexpr int kFlushUnroll = 8;
constexpr int XO = 8;         // output ring: steps per row
constexpr int XOS = XO + 1;

static_assert(XRS + XOS == XSTAGE_STEPS_PER_ROW, "ring sizes known to the host");
// fields of the rings: 4, or 5 with the charge
template <class R, bool CH = false>
__host__ __device__ constexpr int xstage_floats_per_warp() {
    return (CH ? 5 : 4) * 32 * (XRS + XOS);
}

template <class R>
__device__ __forceinline__ void cp_async_elem(R *dst, const R *src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src),
                 "n"(int(sizeof(R))) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <class R, bool CH = false>
struct XStage {
    using V = VS<R, CH>;
    R *ring;            // [NQ][32][XRS]
    R *oring;           // [NQ][32][XOS]
    const R *in;        // event base (field 0, cell 0) of the input state
    R *out;
    int fo1, fo2, fo3;  // field offsets (E at 0)
    int fo4;            // charge offset (CH)
    int N, bc, lane;
    int js;             // this lane's position at step 0
    int rowN;           // this lane's row start: row (pencil) index * N
    // uni: the warp's rows are consecutive (row start rowN0 + lane N), all
    // stored, with one segment (start js0), so addresses and keep bits are
    // the same arithmetic on every lane and need no exchange
    bool uni;
    int js0, rowN0;

    // start copying steps t0 .. t0 + 7 of all 32 rows into the ring
    __device__ __forceinline__ void fill(int t0) {
        const int c = lane & 7;
        if (uni) {
            const R *p0 = in + rowN0 + wrap_index(js0 + t0 + c, N, bc);
            R *q0 = ring + ((t0 + c) & (XR - 1));
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int r = (lane >> 3) + 4 * k;
                const R *p = p0 + r * N;
                R *q = q0 + r * XRS;
                cp_async_elem(q, p);
                cp_async_elem(q + 32 * XRS, p + fo1);
                cp_async_elem(q + 2 * 32 * XRS, p + fo2);
                cp_async_elem(q + 3 * 32 * XRS, p + fo3);
                if constexpr (CH) cp_async_elem(q + 4 * 32 * XRS, p + fo4);
            }
            cp_async_commit();
            return;
        }
        // rows of several segments or events (the rare case): kept rolled, so
        // that it does not crowd the instruction cache
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
            const int r = (lane >> 3) + 4 * k;
            const int rn = __shfl_sync(0xffffffffu, rowN, r);
            const int jr = __shfl_sync(0xffffffffu, js, r);
            const R *p = in + rn + wrap_index(jr + t0 + c, N, bc);
            R *q = ring + r * XRS + ((t0 + c) & (XR - 1));
            cp_async_elem(q, p);
            cp_async_elem(q + 32 * XRS, p + fo1);
            cp_async_elem(q + 2 * 32 * XRS, p + fo2);
            cp_async_elem(q + 3 * 32 * XRS, p + fo3);
            if constexpr (CH) cp_async_elem(q + 4 * 32 * XRS, p + fo4);
        }
        cp_async_commit();
    }
    __device__ __forceinline__ V get(int t) const {
        const R *q = ring + lane * XRS + (t & (XR - 1));
        const V4<R> v = v4<R>(q[0], q[32 * XRS], q[2 * 32 * XRS], q[3 * 32 * XRS]);
        if constexpr (CH) return with_r(v, q[4 * 32 * XRS]);
        else return v;
    }
    __device__ __forceinline__ void put(int t, const V &v) {
        R *q = oring + lane * XOS + (t & (XO - 1));
        q[0] = v.e; q[32 * XOS] = v.n; q[2 * 32 * XOS] = v.t1; q[3 * 32 * XOS] = v.t2;
        if constexpr (CH) q[4 * 32 * XOS] = v.r;
    }
    // write the results of steps t1 - 7 .. t1 (position js + step - 6) whose
    // keep bits (bit step & 7, per row) are set; with RATE also fold their CFL
    // rates into ra (8 independent evaluations per lane)
    template <bool RATE, class PH>
    __device__ __forceinline__ void flush(int t1, unsigned keep, const PH &ph, RateAcc<R> &ra,
                                          bool rate_on) {
        const int c = lane & 7;
        const int st = t1 - 7 + c;
        if (uni) {
            if ((keep >> (st & 7)) & 1u) {
                R *p0 = out + rowN0 + (js0 + st - 6);
                const R *q0 = oring + (st & (XO - 1));
                // with the rate: two rows per iteration, which keeps the code
                // of the step loop in the instruction cache
#pragma unroll(RATE ? kFlushUnrollRate : kFlushUnroll)
                for (int k = 0; k < 8; ++k) {
                    const int r = (lane >> 3) + 4 * k;
                    R *p = p0 + r * N;
                    const R *q = q0 + r * XOS;
                    const V4<R> v =
                        v4<R>(q[0], q[32 * XOS], q[2 * 32 * XOS], q[3 * 32 * XOS]);
                    p[0] = v.e;
                    p[fo1] = v.n;
                    p[fo2] = v.t1;
                    p[fo3] = v.t2;
                    if constexpr (CH) p[fo4] = q[4 * 32 * XOS];
                    if (RATE && rate_on) {
                        const R rr = ph.rate(v, ra.ih_n, ra.ih_t1, ra.ih_t2, ra.iso);
                        ra.m = (rr > ra.m || rr != rr) ? rr : ra.m;
                    }
                }
            }
            return;
        }
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
            const int r = (lane >> 3) + 4 * k;
            const int rn = __shfl_sync(0xffffffffu, rowN, r);
            const int jr = __shfl_sync(0xffffffffu, js, r);
            const unsigned kr = __shfl_sync(0xffffffffu, keep, r);
            if ((kr >> (st & 7)) & 1u) {
                R *p = out + rn + (jr + st - 6);
                const R *q = oring + r * XOS + (st & (XO - 1));
                const V4<R> v = v4<R>(q[0], q[32 * XOS], q[2 * 32 * XOS], q[3 * 32 * XOS]);
                p[0] = v.e;
                p[fo1] = v.n;
                p[fo2] = v.t1;
                p[fo3] = v.t2;
                if constexpr (CH) p[fo4] = q[4 * 32 * XOS];
                if (RATE && rate_on) {
                    const R rr = ph.rate(v, ra.ih_n, ra.ih_t1, ra.ih_t2, ra.iso);
                    ra.m = (rr > ra.m || rr != rr) ? rr : ra.m;
                }
            }
        }
    }
};

// RK2 march of x-rows through the warp's shared-memory rings; the same
// arithmetic, schedule and at-rest start as march() (Eq. 6), so stored cells
// are bit-identical to it.  The whole warp must call it together.
template <class R, bool RATE, class PH>
__device__ __forceinline__ void march_x_rk2(const PH &ph, XStage<R, PH::kCharge> &X, int s0, int L,
                                            int s_end, R lam, bool do_store, RateAcc<R> &ra) {
    using V = typename PH::V;
    const int N = X.N, bc = X.bc;
    const bool rate_on = RATE && ra.ih_n > R(0);
    const R half = R(0.5);
    const int T = L + 10;
    const int js = s0 - 4;
    X.js = js;
    // fills at steps t = phi (mod 8), t >= 1, each for steps t + 2 .. t + 9,
    // so that lane 0's row moves 8-aligned cells; flushes at t = psi (mod 8)
    const int js0 = __shfl_sync(0xffffffffu, js, 0);
    X.js0 = js0;
    X.rowN0 = __shfl_sync(0xffffffffu, X.rowN, 0);
    X.uni = __all_sync(0xffffffffu, do_store && js == js0 && X.rowN == X.rowN0 + X.lane * N);
    const int phi = (6 - js0) & 7;
    const int psi = (13 - js0) & 7;
    const int tf = phi == 0 ? 8 : phi;   // first fill step
    Stage<V> st1, st2;
    V zero = vzero<V>();   // windows start at rest (as in march)
    zero.e = R(1);
    st1.w0 = st1.w1 = st1.w2 = st1.urp = st1.fp = zero;
    st2.w0 = st2.w1 = st2.w2 = st2.urp = st2.fp = zero;
    V qa[3] = {zero, zero, zero};
    V lastA = zero, cell, D;
    __syncwarp();
    X.fill(tf - 14);
    X.fill(tf - 6);   // steps [tf - 14, tf + 2) cover [-6, tf + 2)
    cp_async_wait_all();
    __syncwarp();
    unsigned keep = 0u;
    // the ring reads of a step (its input and the RK reload 6 steps behind)
    // are made at the end of the step before, so their latency overlaps it
    V Vn = X.get(0), U0n = X.get(-6);
#pragma unroll 1
    for (int t = 0; t < T; ++t) {
        if (t >= tf && ((t - phi) & 7) == 0) {   // slots of steps < t - 6 are free
            __syncwarp();
            X.fill(t + 2);
        }
        const V Vc = Vn, U0 = U0n;
        st1.push_full(Vc, ph, lam, cell, D);
        const int i = js + t - 2;
        const V Xv = vfma<R>(-lam, D, cell);   // U1 = U + dt L(U)
        shift_in(qa, Xv);
        if (i == N - 1) lastA = Xv;
        const V Y = pick(qa, i, t + s0 - 8, N, bc, lastA);
        V c, Dl;
        st2.push_full(Y, ph, lam, c, Dl);
        const int o = t + s0 - 10;
        const V r = vmul<R>(half, vfma<R>(-lam, Dl, vadd(U0, c)));
        const bool kp = do_store && o >= s0 && o < s_end;
        X.put(t, r);
        keep |= (kp ? 1u : 0u) << (t & 7);
        if (t < 10) ph.flags_ = 0;   // windows not yet filled (as in march)
        if (((t - psi) & 7) == 0 || t == T - 1) {
            __syncwarp();
            X.template flush<RATE>(t, keep, ph, ra, rate_on);
            __syncwarp();
            keep = 0u;
        }
        // step t + 1 opens a copy group (filled at t - 1): wait for it first
        if (t + 1 >= tf + 2 && ((t - 1 - phi) & 7) == 0) {
            cp_async_wait_all();
            __syncwarp();
        }
        if (t + 1 < T) {
            Vn = X.get(t + 1);
            U0n = X.get(t - 5);
        }
    }
    cp_async_wait_all();   // a last copy may still be in flight
    __syncwarp();
}

}  // namespace hy
