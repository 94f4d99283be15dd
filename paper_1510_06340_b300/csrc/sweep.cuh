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
template <class R, int PREC, int EOSK, int RK>
__global__ void __launch_bounds__(256)
k_sweep(const R *__restrict__ in, R *__restrict__ out, const EventGeo *__restrict__ ev,
        const WorkItem *__restrict__ items, int nitems, int axis, double frac,
        const EventClock *__restrict__ clk, Scheme sc) {
    Physics<R, PREC, EOSK> ph;
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
        const R *ib = in + g.off + base;
        R *ob = out + g.off + base;
        Pc.f0 = ib;
        Pc.f1 = ib + (1 + axis) * cells;
        Pc.f2 = ib + ta * cells;
        Pc.f3 = ib + tb * cells;
        Pc.g0 = ob;
        Pc.g1 = ob + (1 + axis) * cells;
        Pc.g2 = ob + ta * cells;
        Pc.g3 = ob + tb * cells;
        Pc.stride = stride;
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
#define HY_SWEEP(EOSK, RK)                                                                   \
    if (a.sc.eos_kind == EOSK && a.rk == RK) {                                              \
        k_sweep<R, PREC, EOSK, RK><<<a.blocks, a.threads, 0, a.stream>>>(                    \
            in, out, a.ev, a.items, a.nitems, a.axis, a.frac, a.clk, a.sc);                 \
        return cudaGetLastError();                                                          \
    }
    HY_SWEEP(EOS_CONFORMAL, 1)
    HY_SWEEP(EOS_CONFORMAL, 2)
    HY_SWEEP(EOS_CONFORMAL, 3)
    HY_SWEEP(EOS_TABLE, 1)
    HY_SWEEP(EOS_TABLE, 2)
    HY_SWEEP(EOS_TABLE, 3)
#undef HY_SWEEP
    return cudaErrorInvalidValue;
}

}  // namespace hy
