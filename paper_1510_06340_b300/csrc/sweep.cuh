// sweep.cuh -- the directional sweep kernel (all RK stages of one sweep of
// Sec. 2.3 over every pencil along one axis, for any number of events).
#pragma once
#include <atomic>

#include "device.cuh"
#include "kernels.h"

namespace hy {

// Grid-stride over work items: a block takes `count` consecutive
// pencil-segment tasks of one event; thread k takes task first + k.
// Task -> (pencil, segment): pencil = task % P, segment = task / P, so
// neighbouring threads march neighbouring pencils (coalesced along x for the
// y and z sweeps).
// HY_SWEEP_MAXNREG (a build-time define) caps the registers of the sweep
// kernels instead of the default bound of 256 threads per block.
#ifdef HY_SWEEP_MAXNREG
#define HY_SWEEP_BOUNDS __maxnreg__(HY_SWEEP_MAXNREG)
#else
#define HY_SWEEP_BOUNDS __launch_bounds__(256)
#endif

// XS: RK2 x sweep through the shared-memory row rings (march_x_rk2)
// CH: the conserved charge is carried as a fifth field (state [5][...])
template <class R, int PREC, int EOSK, int RK, int LIM, bool COUNT, bool RATE, bool XS, bool CH>
__device__ __forceinline__ void
sweep_body(const R *__restrict__ in, R *__restrict__ out, const EventGeo *__restrict__ ev,
           const WorkItem *__restrict__ items, int nitems, int axis, double frac,
           const EventClock *__restrict__ clk, Scheme sc, int *counter, EventClock *rate_clk) {
    Physics<R, PREC, EOSK, LIM, COUNT, RK != 3, CH> ph;
    ph.sc = sc;
    __shared__ int s_item;
    __shared__ R s_red[8];
    for (int k = 0;; ++k) {
        // one block per item, or a persistent grid taking items from a counter
        int it;
        if (counter) {
            if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
            __syncthreads();
            it = s_item;
            __syncthreads();
        } else {
            it = k == 0 ? int(blockIdx.x) : nitems;
        }
        if (it >= nitems) break;
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        const int nx = g.n[0], ny = g.n[1];
        const int N = g.n[axis];
        const long long cells = g.cells;
        const long long P = cells / N;
        const int L = g.segL[axis];
        const long long ntasks = P * (long long)g.seg[axis];
        long long task = w.first + threadIdx.x;
        const bool valid = threadIdx.x < w.count && task < ntasks;
        if (!valid) task = w.first;   // run a duplicate in step, store nothing
        const long long pencil = task % P;
        const int seg = int(task / P);
        long long base, stride;
        if (axis == 0) {          // pencil = y + ny z
            base = pencil * nx;
            stride = 1;
        } else if (axis == 1) {   // pencil = x + nx z
            const long long x = pencil % nx, z = pencil / nx;
            base = z * (long long)nx * ny + x;
            stride = nx;
        } else {                  // pencil = x + nx y
            base = pencil;
            stride = (long long)nx * ny;
        }
        const int ta = axis == 0 ? 2 : 1, tb = axis == 2 ? 2 : 3;
        Pencil<R, CH> Pc;
        Pc.in = in + g.off + base;
        Pc.out = out + g.off + base;
        Pc.fo1 = int((1 + axis) * cells);
        Pc.fo2 = int(ta * cells);
        Pc.fo3 = int(tb * cells);
        Pc.fo4 = int(4 * cells);
        Pc.stride = int(stride);
        Pc.N = N;
        const R lam = R(frac * clk[w.event].dt / g.h[axis]);
        ph.set_lam(lam);
        const int s0 = seg * L;
        const int s_end = min(s0 + L, N);
        RateAcc<R> ra;
        ra.m = R(0);
        ra.ih_n = ra.ih_t1 = ra.ih_t2 = R(0);
        ra.iso = false;
        if (RATE && rate_clk) {   // last sweep of a step: CFL rate of the new state
            const int at1 = axis == 0 ? 1 : 0, at2 = axis == 2 ? 1 : 2;
            ra.ih_n = R(g.inv_h[axis]);
            ra.ih_t1 = g.n[at1] > 1 ? R(g.inv_h[at1]) : R(0);
            ra.ih_t2 = g.n[at2] > 1 ? R(g.inv_h[at2]) : R(0);
            ra.iso = (ra.ih_t1 == R(0) || ra.ih_t1 == ra.ih_n) &&
                     (ra.ih_t2 == R(0) || ra.ih_t2 == ra.ih_n);
        }
        if (XS) {   // rows through the warp's shared-memory rings
            extern __shared__ __align__(16) unsigned char xs_raw[];
            R *base = reinterpret_cast<R *>(xs_raw) +
                      (threadIdx.x >> 5) * xstage_floats_per_warp<R, CH>();
            XStage<R, CH> X;
            X.ring = base;
            X.oring = base + (CH ? 5 : 4) * 32 * XRS;
            X.in = in + g.off;
            X.out = out + g.off;
            X.fo1 = Pc.fo1; X.fo2 = Pc.fo2; X.fo3 = Pc.fo3; X.fo4 = Pc.fo4;
            X.N = N;
            X.bc = g.bc[0];
            X.lane = threadIdx.x & 31;
            X.rowN = int(pencil) * N;   // < cells < 2^31
            X.js = s0 - 4;
            if (lam > R(0)) {
                march_x_rk2<R, RATE>(ph, X, s0, L, s_end, lam, valid, ra);
            } else if (valid) {   // finished event: copy through
                for (int o = s0; o < s_end; ++o) Pc.store(o, Pc.load(o));
            }
        } else {
            march<R, RK, RATE>(ph, Pc, s0, L, s_end, g.bc[axis], lam, valid, ra);
        }
        report_flags(sc, w.event, ph.flags_);
        if (RATE && rate_clk) {   // block max, one atomic per work item
            R m = ra.m;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const R x = __shfl_xor_sync(0xffffffffu, m, o);
                m = (x > m || x != x) ? x : m;
            }
            if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
            __syncthreads();
            if (threadIdx.x == 0) {
                R t = s_red[0];
                for (int k = 1; k < int(blockDim.x >> 5); ++k)
                    t = (s_red[k] > t || s_red[k] != s_red[k]) ? s_red[k] : t;
                atomicMax(&rate_clk[w.event].rate_bits,
                          (unsigned long long)__double_as_longlong(double(t)));
            }
            __syncthreads();
        }
    }
}

#define HY_SWEEP_PARAMS                                                                      \
    const R *__restrict__ in, R *__restrict__ out, const EventGeo *__restrict__ ev,          \
        const WorkItem *__restrict__ items, int nitems, int axis, double frac,              \
        const EventClock *__restrict__ clk, Scheme sc, int *counter, EventClock *rate_clk
#define HY_SWEEP_ARGS in, out, ev, items, nitems, axis, frac, clk, sc, counter, rate_clk

template <class R, int PREC, int EOSK, int RK, int LIM, bool COUNT, bool RATE, bool XS, bool CH>
__global__ void HY_SWEEP_BOUNDS k_sweep(HY_SWEEP_PARAMS) {
    sweep_body<R, PREC, EOSK, RK, LIM, COUNT, RATE, XS, CH>(HY_SWEEP_ARGS);
}

// The FP32 conformal RK3 sweep (three stages chained in registers) wants a
// few registers more than 168; capped there it keeps 12 warps per SM (six
// blocks of 64 or three of 128) instead of 10, which is worth more than the
// registers.  168 x 256 threads still fits a block.
#ifndef HY_RK3_MAXNREG
#define HY_RK3_MAXNREG 168
#endif
template <class R, int PREC, int EOSK, int RK, int LIM, bool COUNT, bool RATE, bool XS, bool CH>
__global__ void __maxnreg__(HY_RK3_MAXNREG) k_sweep_rk3(HY_SWEEP_PARAMS) {
    sweep_body<R, PREC, EOSK, RK, LIM, COUNT, RATE, XS, CH>(HY_SWEEP_ARGS);
}
#undef HY_SWEEP_PARAMS
#undef HY_SWEEP_ARGS

template <class R, int PREC, int EOSK, int RK, int LIM, bool COUNT, bool RATE, bool XS, bool CH>
constexpr auto sweep_kernel() {
    if constexpr (RK == 3 && PREC == PREC_F32 && EOSK == EOS_CONFORMAL && !COUNT && !CH)
        return &k_sweep_rk3<R, PREC, EOSK, RK, LIM, COUNT, RATE, XS, CH>;
    else
        return &k_sweep<R, PREC, EOSK, RK, LIM, COUNT, RATE, XS, CH>;
}

template <class R, int PREC>
cudaError_t launch_sweep_prec(const SweepLaunch &a) {
    const R *in = static_cast<const R *>(a.in);
    R *out = static_cast<R *>(a.out);
#define HY_SWEEP(EOSK, RK, LIM, COUNT, RATE) HY_SWEEP_CH(EOSK, RK, LIM, COUNT, RATE, false)
#define HY_SWEEP_CH(EOSK, RK, LIM, COUNT, RATE, CH)                                          \
    {                                                                                       \
        if (RK == 2 && a.axis == 0) HY_SWEEP_XS(EOSK, RK, LIM, COUNT, RATE, RK == 2, CH)     \
        else HY_SWEEP_XS(EOSK, RK, LIM, COUNT, RATE, false, CH)                             \
    }
#define HY_SWEEP_XS(EOSK, RK, LIM, COUNT, RATE, XS, CH)                                      \
    {                                                                                       \
        auto kfn = sweep_kernel<R, PREC, EOSK, RK, LIM, COUNT, RATE, XS, CH>();             \
        const size_t smem = XS                                                              \
            ? size_t(a.threads / 32) * xstage_floats_per_warp<R, CH>() * sizeof(R) : 0;      \
        if (smem > 0) {   /* opt in once per device, for the most warps that fit */     \
            static std::atomic<unsigned long long> opted{0};                                \
            int dev_ = 0, optin_ = 0;                                                       \
            cudaError_t e_ = cudaGetDevice(&dev_);                                          \
            if (e_ != cudaSuccess) return e_;                                               \
            const unsigned long long bit_ = 1ull << (dev_ & 63);                            \
            if (!(opted.load() & bit_)) {                                                   \
                e_ = cudaDeviceGetAttribute(&optin_,                                        \
                                            cudaDevAttrMaxSharedMemoryPerBlockOptin, dev_); \
                if (e_ != cudaSuccess) return e_;                                           \
                const int warp_ = int(xstage_floats_per_warp<R, CH>() * sizeof(R));         \
                const int warps_ = optin_ / warp_ < 8 ? optin_ / warp_ : 8;                 \
                e_ = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                          warps_ * warp_);                                  \
                if (e_ != cudaSuccess) { cudaGetLastError(); return e_; }                   \
                opted.fetch_or(bit_);                                                       \
            }                                                                               \
        }                                                                                   \
        int blocks = a.nitems;                                                              \
        if (a.counter) {                                                                    \
            int occ = 0;                                                                    \
            cudaError_t e_ = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn,       \
                                                                           a.threads, smem);\
            if (e_ != cudaSuccess) return e_;                                               \
            blocks = occ * a.sms < a.nitems ? occ * a.sms : a.nitems;                       \
            if (blocks < 1) blocks = 1;                                                     \
            e_ = cudaMemsetAsync(a.counter, 0, sizeof(int), a.stream);                      \
            if (e_ != cudaSuccess) return e_;                                               \
        }                                                                                   \
        kfn<<<blocks, a.threads, smem, a.stream>>>(in, out, a.ev, a.items, a.nitems, a.axis, \
                                                a.frac, a.clk, a.sc, a.counter, a.rate_clk); \
        return cudaGetLastError();                                                          \
    }
    // the conserved charge as a fifth field: runtime-limiter kernels with
    // counters compiled in (the four-field kernels below are untouched)
    if (a.charge) {
        if (a.sc.eos_kind == EOS_CONFORMAL) {
            if (a.rk == 1) HY_SWEEP_CH(EOS_CONFORMAL, 1, -1, true, true, true)
            if (a.rk == 2) HY_SWEEP_CH(EOS_CONFORMAL, 2, -1, true, true, true)
            if (a.rk == 3) HY_SWEEP_CH(EOS_CONFORMAL, 3, -1, true, true, true)
        } else if (a.sc.seed != SEED_MLP) {
            if (a.rk == 1) HY_SWEEP_CH(EOS_TABLE, 1, -1, true, true, true)
            if (a.rk == 2) HY_SWEEP_CH(EOS_TABLE, 2, -1, true, true, true)
            if (a.rk == 3) HY_SWEEP_CH(EOS_TABLE, 3, -1, true, true, true)
        }
        return cudaErrorInvalidValue;
    }
    // specialised kernels (limiter fixed at compile time, no counters, the
    // Hancock step on; with two MUSTA stages for the conformal RK2 scheme);
    // everything else takes the runtime-limiter kernel
    if (a.sc.eos_kind == EOS_CONFORMAL && a.rk == 2 && !a.sc.counters && a.sc.hancock &&
        a.sc.stages == 2) {
        // the CFL rate is compiled in only for the last sweep of a step
        if (a.rate_clk) {
            switch (a.sc.limiter) {
            case LIM_MINMOD: HY_SWEEP(EOS_CONFORMAL, 2, LIM_MINMOD, false, true)
            case LIM_MC: HY_SWEEP(EOS_CONFORMAL, 2, LIM_MC, false, true)
            case LIM_SUPERBEE: HY_SWEEP(EOS_CONFORMAL, 2, LIM_SUPERBEE, false, true)
            case LIM_NONE: HY_SWEEP(EOS_CONFORMAL, 2, LIM_NONE, false, true)
            default: break;
            }
        } else {
            switch (a.sc.limiter) {
            case LIM_MINMOD: HY_SWEEP(EOS_CONFORMAL, 2, LIM_MINMOD, false, false)
            case LIM_MC: HY_SWEEP(EOS_CONFORMAL, 2, LIM_MC, false, false)
            case LIM_SUPERBEE: HY_SWEEP(EOS_CONFORMAL, 2, LIM_SUPERBEE, false, false)
            case LIM_NONE: HY_SWEEP(EOS_CONFORMAL, 2, LIM_NONE, false, false)
            default: break;
            }
        }
    }
    // the paper's production settings (RK3), Minbee specialised
    if (a.sc.eos_kind == EOS_CONFORMAL && a.rk == 3 && !a.sc.counters &&
        a.sc.limiter == LIM_MINMOD) {
        if (a.rate_clk) HY_SWEEP(EOS_CONFORMAL, 3, LIM_MINMOD, false, true)
        else HY_SWEEP(EOS_CONFORMAL, 3, LIM_MINMOD, false, false)
    }
    // tabulated EOS: Minbee RK2 specialised (plain Newton seeds, or the MLP seed)
    const bool mlp = a.sc.eos_kind == EOS_TABLE && a.sc.seed == SEED_MLP;
    if (a.sc.eos_kind == EOS_TABLE && a.rk == 2 && !a.sc.counters && a.sc.hancock &&
        a.sc.limiter == LIM_MINMOD) {
        if (mlp) {
            if (a.rate_clk) HY_SWEEP(EOS_TABLE_MLP, 2, LIM_MINMOD, false, true)
            else HY_SWEEP(EOS_TABLE_MLP, 2, LIM_MINMOD, false, false)
        } else {
            if (a.rate_clk) HY_SWEEP(EOS_TABLE, 2, LIM_MINMOD, false, true)
            else HY_SWEEP(EOS_TABLE, 2, LIM_MINMOD, false, false)
        }
    }
    if (a.sc.eos_kind == EOS_CONFORMAL) {
        if (a.rk == 1) HY_SWEEP(EOS_CONFORMAL, 1, -1, true, true)
        if (a.rk == 2) HY_SWEEP(EOS_CONFORMAL, 2, -1, true, true)
        if (a.rk == 3) HY_SWEEP(EOS_CONFORMAL, 3, -1, true, true)
    } else if (mlp) {
        if (a.rk == 1) HY_SWEEP(EOS_TABLE_MLP, 1, -1, true, true)
        if (a.rk == 2) HY_SWEEP(EOS_TABLE_MLP, 2, -1, true, true)
        if (a.rk == 3) HY_SWEEP(EOS_TABLE_MLP, 3, -1, true, true)
    } else {
        if (a.rk == 1) HY_SWEEP(EOS_TABLE, 1, -1, true, true)
        if (a.rk == 2) HY_SWEEP(EOS_TABLE, 2, -1, true, true)
        if (a.rk == 3) HY_SWEEP(EOS_TABLE, 3, -1, true, true)
    }
#undef HY_SWEEP
#undef HY_SWEEP_CH
#undef HY_SWEEP_XS
    return cudaErrorInvalidValue;
}

}  // namespace hy
