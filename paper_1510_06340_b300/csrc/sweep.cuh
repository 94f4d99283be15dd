// sweep.cuh -- the directional sweep kernel (all RK stages of one sweep of
// Sec. 2.3 over every pencil along one axis, for any number of events).
#pragma once
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

template <class R, int PREC, int EOSK, int RK, int LIM, bool COUNT>
__global__ void HY_SWEEP_BOUNDS
k_sweep(const R *__restrict__ in, R *__restrict__ out, const EventGeo *__restrict__ ev,
        const WorkItem *__restrict__ items, int nitems, int axis, double frac,
        const EventClock *__restrict__ clk, Scheme sc) {
    Physics<R, PREC, EOSK, LIM, COUNT> ph;
    ph.sc = sc;
    ph.cs2 = R(sc.cs2);
    ph.delta = R(sc.delta);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
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
        Pencil<R> Pc;
        Pc.in = in + g.off + base;
        Pc.out = out + g.off + base;
        Pc.fo1 = int((1 + axis) * cells);
        Pc.fo2 = int(ta * cells);
        Pc.fo3 = int(tb * cells);
        Pc.stride = int(stride);
        Pc.N = N;
        const R lam = R(frac * clk[w.event].dt / g.h[axis]);
        const int s0 = seg * L;
        const int s_end = min(s0 + L, N);
        march<R, RK>(ph, Pc, s0, L, s_end, g.bc[axis], lam, valid);
    }
}

template <class R, int PREC>
cudaError_t launch_sweep_prec(const SweepLaunch &a) {
    const R *in = static_cast<const R *>(a.in);
    R *out = static_cast<R *>(a.out);
#define HY_SWEEP(EOSK, RK, LIM, COUNT)                                                       \
    {                                                                                       \
        k_sweep<R, PREC, EOSK, RK, LIM, COUNT><<<a.blocks, a.threads, 0, a.stream>>>(       \
            in, out, a.ev, a.items, a.nitems, a.axis, a.frac, a.clk, a.sc);                 \
        return cudaGetLastError();                                                          \
    }
    // specialised kernels (limiter fixed at compile time, no counters) for the
    // conformal RK2 scheme; everything else takes the runtime-limiter kernel
    if (a.sc.eos_kind == EOS_CONFORMAL && a.rk == 2 && !a.sc.counters) {
        switch (a.sc.limiter) {
        case LIM_MINMOD: HY_SWEEP(EOS_CONFORMAL, 2, LIM_MINMOD, false)
        case LIM_MC: HY_SWEEP(EOS_CONFORMAL, 2, LIM_MC, false)
        case LIM_SUPERBEE: HY_SWEEP(EOS_CONFORMAL, 2, LIM_SUPERBEE, false)
        case LIM_NONE: HY_SWEEP(EOS_CONFORMAL, 2, LIM_NONE, false)
        default: break;
        }
    }
    if (a.sc.eos_kind == EOS_CONFORMAL) {
        if (a.rk == 1) HY_SWEEP(EOS_CONFORMAL, 1, -1, true)
        if (a.rk == 2) HY_SWEEP(EOS_CONFORMAL, 2, -1, true)
        if (a.rk == 3) HY_SWEEP(EOS_CONFORMAL, 3, -1, true)
    } else {
        if (a.rk == 1) HY_SWEEP(EOS_TABLE, 1, -1, true)
        if (a.rk == 2) HY_SWEEP(EOS_TABLE, 2, -1, true)
        if (a.rk == 3) HY_SWEEP(EOS_TABLE, 3, -1, true)
    }
#undef HY_SWEEP
    return cudaErrorInvalidValue;
}

}  // namespace hy
