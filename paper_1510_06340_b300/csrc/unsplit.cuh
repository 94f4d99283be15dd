// unsplit.cuh -- one RK stage of the unsplit multi-D MUSCL-Hancock
// MUSTA-FORCE scheme: the Hancock half step of Eq. 13 with all three flux
// terms, the FORCE alpha of Eq. 10-11 (3 in 3-D), the RK stages of Eq. 5-7 on
// the whole field (reading R16).
//
// Three kernels per stage:
//   k_us_faces   evolved faces of every cell of the box grown by one cell
//                along each active axis (ghosts mapped by the BCs);
//   k_us_flux    the MUSTA-FORCE flux of every interface, one launch per axis;
//   k_us_update  dt L(U) = -sum_d dt/dx_d (F_d,i+1/2 - F_d,i-1/2) and the RK
//                stage combination; on the last stage also the CFL rate
//                (sum over axes, R16c) of the new state.
// Faces and fluxes go through HBM scratch laid out by UnsplitGeo.
#pragma once
#include "device.cuh"
#include "kernels.h"

namespace hy {

constexpr int US_THREADS = 256;   // units (cells or interfaces) per work item and block

// The state in the order a flux along axis d takes it, (E, M_d, M_a, M_b)
// with the transverse components in increasing axis order, and back.
template <class R>
__device__ __forceinline__ V4<R> to_axis(const V4<R> &u, int d) {
    if (d == 0) return u;
    if (d == 1) return v4<R>(u.e, u.t1, u.n, u.t2);
    return v4<R>(u.e, u.t2, u.n, u.t1);
}
template <class R>
__device__ __forceinline__ V4<R> from_axis(const V4<R> &a, int d) {
    if (d == 0) return a;
    if (d == 1) return v4<R>(a.e, a.t1, a.n, a.t2);
    return v4<R>(a.e, a.t1, a.t2, a.n);
}

// (E, Mx, My, Mz) of cell c of the event
template <class R>
__device__ __forceinline__ V4<R> us_load(const R *__restrict__ U, const EventGeo &g, long long c) {
    const R *p = U + g.off + c;
    return v4<R>(__ldg(p), __ldg(p + g.cells), __ldg(p + 2 * g.cells), __ldg(p + 3 * g.cells));
}

template <class R>
__device__ __forceinline__ void us_store(R *__restrict__ U, const EventGeo &g, long long c,
                                         const V4<R> &v) {
    R *p = U + g.off + c;
    p[0] = v.e;
    p[g.cells] = v.n;
    p[2 * g.cells] = v.t1;
    p[3 * g.cells] = v.t2;
}

// face (d, side) of grown cell gi: side 0 = left (U^L), 1 = right (U^R)
template <class R>
__device__ __forceinline__ R *us_face(R *faces, const UnsplitGeo &u, int d, int side,
                                      long long gi) {
    return faces + u.fo + (long long)((2 * d + side) * 4) * u.gcells + gi;
}

// FP32: bounded to 64 registers, which keeps 32 warps per SM instead of 24
// (20 bytes of spill); the load and MUFU latencies of this kernel need the
// warps more than the registers (1143 -> 1037 us per 256^3 stage)
template <class R, int PREC, int EOSK, int LIM, bool COUNT>
__global__ void __launch_bounds__(US_THREADS, sizeof(R) == 4 ? 4 : 1)
k_us_faces(const R *__restrict__ in, R *__restrict__ faces, const EventGeo *__restrict__ ev,
           const UnsplitGeo *__restrict__ ugeo, const WorkItem *__restrict__ items, int nitems,
           const EventClock *__restrict__ clk, Scheme sc) {
    Physics<R, PREC, EOSK, LIM, COUNT> ph;
    ph.sc = sc;
    const R half = R(0.5);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        const UnsplitGeo &u = ugeo[w.event];
        // lanes past the item's end repeat its first unit and store nothing,
        // so a warp stays converged (the MLP Newton seed needs that)
        const bool valid = int(threadIdx.x) < w.count;
        // grown boxes hold fewer than 2^31 cells: 32-bit index arithmetic
        const unsigned gi = unsigned(w.first) + (valid ? threadIdx.x : 0u);
        const unsigned m0 = unsigned(u.m[0]), m1 = unsigned(u.m[1]);
        const unsigned r = gi / m0;
        const int x[3] = {int(gi - r * m0) - u.g[0], int(r % m1) - u.g[1], int(r / m1) - u.g[2]};
        const double dt = clk[w.event].dt;
        // a coordinate at most 2 cells outside [0, n): one wrap or clamp
        auto fold = [&](int j, int a) {
            const int n = g.n[a];
            if (g.bc[a] == BC_OUTFLOW) return j < 0 ? 0 : (j >= n ? n - 1 : j);
            return j < 0 ? j + n : (j >= n ? j - n : j);
        };
        auto cell = [&](int d, int o) {   // the cell o steps from x along axis d
            int y[3] = {x[0], x[1], x[2]};
            y[d] += o;
            const int a = fold(y[0], 0), b = fold(y[1], 1), c = fold(y[2], 2);
            return us_load(in, g, (long long)(unsigned(a) + unsigned(g.n[0]) *
                                              (unsigned(b) + unsigned(g.n[1]) * unsigned(c))));
        };
        const V4<R> V0 = cell(0, 0);
        V4<R> UL[3], UR[3];
        V4<R> h = v4<R>(R(0), R(0), R(0), R(0));
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            UL[d] = V0;
            UR[d] = V0;
            if (!u.g[d]) continue;
            const V4<R> Vm = cell(d, -1), Vp = cell(d, 1);
            // Eq. 15-17 along axis d, per conserved field
            const int lim = sc.limiter;
            const V4<R> sl = v4<R>(slope_ct<LIM, R>(lim, V0.e - Vm.e, Vp.e - V0.e),
                                   slope_ct<LIM, R>(lim, V0.n - Vm.n, Vp.n - V0.n),
                                   slope_ct<LIM, R>(lim, V0.t1 - Vm.t1, Vp.t1 - V0.t1),
                                   slope_ct<LIM, R>(lim, V0.t2 - Vm.t2, Vp.t2 - V0.t2));
            UL[d] = vfma<R>(-half, sl, V0);
            UR[d] = vfma<R>(half, sl, V0);
            if (sc.hancock) {   // Eq. 13: the axis-d term of the half step (R16a)
                const R lam = R(dt / g.h[d]);
                const V4<R> FL = from_axis(ph.flux(to_axis(UL[d], d)), d);
                const V4<R> FR = from_axis(ph.flux(to_axis(UR[d], d)), d);
                h = vfma<R>(half * lam, vsub(FL, FR), h);
            }
        }
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (!u.g[d]) continue;
            UL[d] = vadd(UL[d], h);
            UR[d] = vadd(UR[d], h);
            ok = ok && ph.admissible(UL[d]) && ph.admissible(UR[d]);
        }
        if (!ok) {   // R9 over all faces of the cell (R16b)
#pragma unroll
            for (int d = 0; d < 3; ++d) { UL[d] = V0; UR[d] = V0; }
            if (COUNT && valid) count(sc, CNT_FACE_FALLBACK);
            ph.flags_ |= FLAG_UNPHYSICAL;
        }
        if (valid) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (!u.g[d]) continue;
                R *fl = us_face(faces, u, d, 0, (long long)gi);
                R *fr = us_face(faces, u, d, 1, (long long)gi);
                fl[0] = UL[d].e; fl[u.gcells] = UL[d].n;
                fl[2 * u.gcells] = UL[d].t1; fl[3 * u.gcells] = UL[d].t2;
                fr[0] = UR[d].e; fr[u.gcells] = UR[d].n;
                fr[2 * u.gcells] = UR[d].t1; fr[3 * u.gcells] = UR[d].t2;
            }
        }
        report_flags(sc, w.event, ph.flags_);
    }
}

// Interfaces along axis d are numbered x fastest on the grid extended by one
// cell along d: interface (x, y, z) lies between the cell one step before it
// along d and the cell (x, y, z), so neighbouring threads touch neighbouring
// memory for every axis.
__device__ __forceinline__ unsigned us_iface_index(const EventGeo &g, int d, int x, int y, int z) {
    const unsigned e0 = unsigned(g.n[0] + (d == 0)), e1 = unsigned(g.n[1] + (d == 1));
    return unsigned(x) + e0 * (unsigned(y) + e1 * unsigned(z));
}
__device__ __forceinline__ void us_interface(const EventGeo &g, int d, unsigned ii, int x[3]) {
    const unsigned e0 = unsigned(g.n[0] + (d == 0)), e1 = unsigned(g.n[1] + (d == 1));
    const unsigned r = ii / e0;
    x[0] = int(ii - r * e0);
    x[1] = int(r % e1);
    x[2] = int(r / e1);
}

template <class R, int PREC, int EOSK, bool COUNT>
__global__ void __launch_bounds__(US_THREADS)
k_us_flux(const R *__restrict__ faces, R *__restrict__ fluxes, const EventGeo *__restrict__ ev,
          const UnsplitGeo *__restrict__ ugeo, const WorkItem *__restrict__ items, int nitems,
          int d, const EventClock *__restrict__ clk, Scheme sc) {
    Physics<R, PREC, EOSK, -1, COUNT> ph;
    ph.sc = sc;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        const UnsplitGeo &u = ugeo[w.event];
        const bool valid = int(threadIdx.x) < w.count;
        const unsigned ii = unsigned(w.first) + (valid ? threadIdx.x : 0u);
        int x[3];
        us_interface(g, d, ii, x);
        // grown-box indices of the cells left (p - 1) and right (p) of the interface
        const long long gr = (x[0] + u.g[0]) +
                             (long long)u.m[0] * ((x[1] + u.g[1]) + (long long)u.m[1] * (x[2] + u.g[2]));
        const long long step = d == 0 ? 1 : (d == 1 ? u.m[0] : (long long)u.m[0] * u.m[1]);
        const long long gl = gr - step;
        const R *fr = us_face(faces, u, d, 1, gl);   // right face of the left cell
        const R *fl = us_face(faces, u, d, 0, gr);   // left face of the right cell
        const V4<R> UL = v4<R>(fr[0], fr[u.gcells], fr[2 * u.gcells], fr[3 * u.gcells]);
        const V4<R> UR = v4<R>(fl[0], fl[u.gcells], fl[2 * u.gcells], fl[3 * u.gcells]);
        const R lam = R(clk[w.event].dt / g.h[d]);
        ph.set_lam(lam);
        // Sec. 2.4 steps 1-5 at this interface (R3)
        const V4<R> F = from_axis(ph.musta(to_axis(UL, d), to_axis(UR, d), lam), d);
        if (valid) {
            R *o = fluxes + u.xo[d] + ii;
            o[0] = F.e;
            o[u.nint[d]] = F.n;
            o[2 * u.nint[d]] = F.t1;
            o[3 * u.nint[d]] = F.t2;
        }
        report_flags(sc, w.event, ph.flags_);
    }
}

template <class R>
__device__ __forceinline__ R us_max_nan(R a, R b) { return (b > a || b != b) ? b : a; }

template <class R, int PREC, int EOSK, bool RATE>
__global__ void __launch_bounds__(US_THREADS)
k_us_update(const R *__restrict__ u0, const R *__restrict__ u1, R *__restrict__ out,
            const R *__restrict__ fluxes, const EventGeo *__restrict__ ev,
            const UnsplitGeo *__restrict__ ugeo, const WorkItem *__restrict__ items, int nitems,
            const EventClock *__restrict__ clk, Scheme sc, int rk, int stage,
            EventClock *rate_clk) {
    Physics<R, PREC, EOSK, -1, false> ph;
    ph.sc = sc;
    __shared__ R red[US_THREADS / 32];
    const R half = R(0.5), q3 = R(0.75), q1 = R(0.25), third = R(1.0 / 3.0), two3 = R(2.0 / 3.0);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        const UnsplitGeo &u = ugeo[w.event];
        const double dt = clk[w.event].dt;
        R lam[3], ih[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lam[d] = R(dt / g.h[d]);
            ih[d] = R(g.inv_h[d]);
        }
        R m = R(0);
        const unsigned n0 = unsigned(g.n[0]), n1 = unsigned(g.n[1]);
        // unrolled so that the loads of consecutive cells are in flight together
        // (412 -> 343 us per 256^3 stage)
#pragma unroll 4
        for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
            const long long c = w.first + k;
            const unsigned cu = unsigned(c), row = cu / n0;
            const int x = int(cu - row * n0), y = int(row % n1), z = int(row / n1);
            // dt L(U) = -D, D = sum_d dt/dx_d (F_d,i+1/2 - F_d,i-1/2), axes in order
            V4<R> D = v4<R>(R(0), R(0), R(0), R(0));
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (!u.g[d]) continue;
                const unsigned im = us_iface_index(g, d, x, y, z);
                const unsigned ip = us_iface_index(g, d, x + (d == 0), y + (d == 1), z + (d == 2));
                const R *f = fluxes + u.xo[d];
                const long long s = u.nint[d];
                const V4<R> Fm = v4<R>(f[im], f[s + im], f[2 * s + im], f[3 * s + im]);
                const V4<R> Fp = v4<R>(f[ip], f[s + ip], f[2 * s + ip], f[3 * s + ip]);
                D = vfma<R>(lam[d], vsub(Fp, Fm), D);
            }
            const V4<R> U0 = us_load(u0, g, c);
            V4<R> r;
            if (stage == 1) {
                r = vsub(U0, D);                             // U + dt L(U)
            } else if (rk == 2) {
                const V4<R> U1 = us_load(u1, g, c);          // Eq. 6
                r = vmul<R>(half, vsub(vadd(U0, U1), D));
            } else if (stage == 2) {
                const V4<R> U1 = us_load(u1, g, c);          // Eq. 7, U2
                r = vadd(vmul<R>(q3, U0), vmul<R>(q1, vsub(U1, D)));
            } else {
                const V4<R> U2 = us_load(u1, g, c);          // Eq. 7, U^{n+1}
                r = vadd(vmul<R>(third, U0), vmul<R>(two3, vsub(U2, D)));
            }
            us_store(out, g, c, r);
            if (RATE && rate_clk) {   // R16c: sum over the active axes
                R rr = R(0);
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    if (u.g[d]) rr += ph.rate(to_axis(r, d), ih[d], R(0), R(0), true);
                m = us_max_nan(m, rr);
            }
        }
        if (RATE && rate_clk) {   // block max, one atomic per work item
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = us_max_nan(m, __shfl_xor_sync(0xffffffffu, m, o));
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
            __syncthreads();
            if (threadIdx.x == 0) {
                R t = red[0];
                for (int k = 1; k < int(blockDim.x >> 5); ++k) t = us_max_nan(t, red[k]);
                atomicMax(&rate_clk[w.event].rate_bits,
                          (unsigned long long)__double_as_longlong(double(t)));
            }
            __syncthreads();
        }
    }
}

template <class R, int PREC>
cudaError_t launch_unsplit_prec(const UnsplitLaunch &a) {
    const R *in = static_cast<const R *>(a.in);
    R *faces = static_cast<R *>(a.faces);
    R *fluxes = static_cast<R *>(a.fluxes);
    auto blocks = [&](int nitems) {
        const int b = a.sms * 8;
        return nitems < b ? (nitems < 1 ? 1 : nitems) : b;
    };
    const bool mlp = a.sc.eos_kind == EOS_TABLE && a.sc.seed == SEED_MLP;
    const bool fast = !a.sc.counters && a.sc.limiter == LIM_MINMOD;
#define HY_US_FACES(EOSK)                                                                        \
    {                                                                                            \
        if (fast)                                                                                \
            k_us_faces<R, PREC, EOSK, LIM_MINMOD, false>                                         \
                <<<blocks(a.n_face_items), US_THREADS, 0, a.stream>>>(                          \
                    in, faces, a.ev, a.ug, a.face_items, a.n_face_items, a.clk, a.sc);           \
        else                                                                                     \
            k_us_faces<R, PREC, EOSK, -1, true><<<blocks(a.n_face_items), US_THREADS, 0,        \
                                                   a.stream>>>(in, faces, a.ev, a.ug,            \
                                                               a.face_items, a.n_face_items,     \
                                                               a.clk, a.sc);                     \
        for (int d = 0; d < 3; ++d) {                                                            \
            if (a.n_flux_items[d] == 0) continue;                                                \
            if (a.sc.counters)                                                                   \
                k_us_flux<R, PREC, EOSK, true><<<blocks(a.n_flux_items[d]), US_THREADS, 0,      \
                                                 a.stream>>>(faces, fluxes, a.ev, a.ug,          \
                                                             a.flux_items[d], a.n_flux_items[d], \
                                                             d, a.clk, a.sc);                    \
            else                                                                                 \
                k_us_flux<R, PREC, EOSK, false><<<blocks(a.n_flux_items[d]), US_THREADS, 0,     \
                                                  a.stream>>>(faces, fluxes, a.ev, a.ug,         \
                                                              a.flux_items[d],                   \
                                                              a.n_flux_items[d], d, a.clk,       \
                                                              a.sc);                             \
        }                                                                                        \
        if (a.rate_clk)                                                                          \
            k_us_update<R, PREC, EOSK, true><<<blocks(a.n_cell_items), US_THREADS, 0,           \
                                              a.stream>>>(                                       \
                static_cast<const R *>(a.u0), static_cast<const R *>(a.u1),                     \
                static_cast<R *>(a.out), fluxes, a.ev, a.ug, a.cell_items, a.n_cell_items,       \
                a.clk, a.sc, a.rk, a.stage, a.rate_clk);                                         \
        else                                                                                     \
            k_us_update<R, PREC, EOSK, false><<<blocks(a.n_cell_items), US_THREADS, 0,          \
                                               a.stream>>>(                                      \
                static_cast<const R *>(a.u0), static_cast<const R *>(a.u1),                     \
                static_cast<R *>(a.out), fluxes, a.ev, a.ug, a.cell_items, a.n_cell_items,       \
                a.clk, a.sc, a.rk, a.stage, nullptr);                                            \
    }
    if (a.sc.eos_kind == EOS_CONFORMAL) HY_US_FACES(EOS_CONFORMAL)
    else if (mlp) HY_US_FACES(EOS_TABLE_MLP)
    else HY_US_FACES(EOS_TABLE)
#undef HY_US_FACES
    return cudaGetLastError();
}

}  // namespace hy
