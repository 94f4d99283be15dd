// aux.cu -- cell-wise kernels around the sweeps: prim->cons (Eq. 4),
// cons->prim (Eq. 23), the CFL rate reduction, per-event time steps, the jet
// source, FP64 conservation sums, hot-spot initial states and a finite check.
#include <cuda_bf16.h>

#include "device.cuh"
#include "widen.cuh"
#include "kernels.h"

namespace hy {

// ------------------------------------------------------------------ helpers
template <class R>
__device__ __forceinline__ void eos_pc2(const Scheme &sc, R e, R &p, R &c2) {
    if (sc.eos_kind == EOS_CONFORMAL) {
        // the scheme's constants in precision R (no FP64 conversion per cell)
        p = consts<R>(sc).cs2 * e;
        c2 = consts<R>(sc).cs2;
    } else {
        eos_table<R>(sc, e, p, c2);
    }
}

// full cons -> prim of one cell: e, velocity vector (Eq. 23 with R9-R11)
template <class R>
__device__ __forceinline__ void c2p_full(const Scheme &sc, R E, R Mx, R My, R Mz, R &e, R &vx,
                                         R &vy, R &vz, int &iters) {
    iters = 0;
    const R delta = consts<R>(sc).delta;
    R M2 = Mx * Mx + My * My + Mz * Mz;
    if (!(E > consts<R>(sc).emin)) { e = R(0); vx = vy = vz = R(0); return; }   // vacuum (R18)
    const R cap = (R(1) - delta) * E;
    R s = R(1);
    if (M2 > cap * cap) {
        s = cap / dsqrt_(M2);
        M2 = cap * cap;
    }
    if (sc.eos_kind == EOS_CONFORMAL) {
        const R cs2 = consts<R>(sc).cs2;
        const R a = (R(1) + cs2) * E;
        R disc = a * a - R(4) * cs2 * M2;
        disc = disc < R(0) ? R(0) : disc;
        const R W = R(0.5) * (a + dsqrt_(disc));
        vx = s * Mx / W; vy = s * My / W; vz = s * Mz / W;
        e = E - M2 / W;
        return;
    }
    const R M = dsqrt_(M2);
    R p;
    const R v = newton_speed<R>(sc, E, M, M2, sc.seed, R(0), p, iters);
    const R sc_ = M > R(0) ? s * v / M : R(0);
    vx = Mx * sc_; vy = My * sc_; vz = Mz * sc_;
    e = E - M * v;
}

// ------------------------------------------------------------------ prim -> cons
// with nq = 5 also R = n gamma (Eq. 4) from the rest-frame charge density n
// (n null: R = 0)
template <class R>
__global__ void k_prim2cons(const EventGeo *__restrict__ ev, const WorkItem *__restrict__ items,
                            int nitems, const R *__restrict__ e, const R *__restrict__ vx,
                            const R *__restrict__ vy, const R *__restrict__ vz,
                            const R *__restrict__ nr, R *__restrict__ U, Scheme sc, int nq) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
            const long long c = w.first + k;
            const R ee = e[c], x = vx[c], y = vy[c], z = vz[c];
            R p, c2;
            eos_pc2<R>(sc, ee, p, c2);
            const R g2 = R(1) / (R(1) - (x * x + y * y + z * z));
            const R wv = (ee + p) * g2;
            R *u = U + g.off + c;
            u[0] = wv - p;
            u[g.cells] = wv * x;
            u[2 * g.cells] = wv * y;
            u[3 * g.cells] = wv * z;
            if (nq == 5) u[4 * g.cells] = nr ? nr[c] * sqrt(g2) : R(0);
        }
    }
}

// ------------------------------------------------------------------ cons -> prim
template <class R>
__global__ void k_cons2prim(const EventGeo *__restrict__ ev, const WorkItem *__restrict__ items,
                            int nitems, const R *__restrict__ U, R *__restrict__ e,
                            R *__restrict__ vx, R *__restrict__ vy, R *__restrict__ vz, Scheme sc,
                            int mixed) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
            const long long c = w.first + k;
            const R *u = U + g.off + c;
            int iters;
            R ee, x, y, z;
            c2p_full<R>(sc, u[0], u[g.cells], u[2 * g.cells], u[3 * g.cells], ee, x, y, z, iters);
            if (mixed && x * x + y * y + z * z > R(0.9801)) {
                // e = E - M v cancels as |v| -> 1: redo from the same inputs in double
                Scheme sd = sc;
                sd.delta = DELTA_F64;
                double de, dx_, dy_, dz_;
                c2p_full<double>(sd, double(u[0]), double(u[g.cells]), double(u[2 * g.cells]),
                                 double(u[3 * g.cells]), de, dx_, dy_, dz_, iters);
                ee = R(de); x = R(dx_); y = R(dy_); z = R(dz_);
            }
            e[c] = ee; vx[c] = x; vy[c] = y; vz[c] = z;
        }
    }
}

// rest-frame charge density n = R / gamma = R sqrt(1 - v^2), v from the
// energy-momentum fields (vacuum: v = 0, n = R)
template <class R>
__global__ void k_charge_density(const EventGeo *__restrict__ ev,
                                 const WorkItem *__restrict__ items, int nitems,
                                 const R *__restrict__ U, R *__restrict__ n, Scheme sc) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
            const long long c = w.first + k;
            const R *u = U + g.off + c;
            int iters;
            R ee, x, y, z;
            c2p_full<R>(sc, u[0], u[g.cells], u[2 * g.cells], u[3 * g.cells], ee, x, y, z, iters);
            n[c] = u[4 * g.cells] * dsqrt_(R(1) - (x * x + y * y + z * z));
        }
    }
}

// ------------------------------------------------------------------ CFL rate
// reading R8: largest |characteristic speed| / dx over cells and swept axes,
// computed in the state's precision.  With b = c sqrt(rad) >= 0,
// max(|a + b|, |a - b|) = |a| + b.  Each block keeps a running max over its
// consecutive work items of one event and adds it with one atomic.
template <class R>
__device__ __forceinline__ R max_nan(R a, R b) { return (b > a || b != b) ? b : a; }

// block-wide max of m (NaN propagates), then one atomic per block and event run
template <class R>
__device__ __forceinline__ void flush_rate(R m, int event, EventClock *clk, R *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max_nan(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        R t = red[0];
        for (int k = 1; k < int(blockDim.x >> 5); ++k) t = max_nan(t, red[k]);
        atomicMax(&clk[event].rate_bits, (unsigned long long)__double_as_longlong(double(t)));
    }
    __syncthreads();
}

template <class R>
__global__ void k_rate(const EventGeo *__restrict__ ev, const WorkItem *__restrict__ items,
                       int nitems, const R *__restrict__ U, EventClock *__restrict__ clk,
                       Scheme sc, int sum_axes) {
    __shared__ R red[32];
    R m = R(0);
    int cur_event = -1;
    const int per = (nitems + gridDim.x - 1) / gridDim.x;   // a contiguous range per block
    const int it_end = min(nitems, (blockIdx.x + 1) * per);
    for (int it = blockIdx.x * per; it < it_end; ++it) {
        const WorkItem w = items[it];
        if (w.event != cur_event) {     // block-uniform
            if (cur_event >= 0) flush_rate<R>(m, cur_event, clk, red);
            m = R(0);
            cur_event = w.event;
        }
        const EventGeo &g = ev[w.event];
        R invh[3];
        if (sizeof(R) == 8) {
            invh[0] = R(g.inv_h[0]); invh[1] = R(g.inv_h[1]); invh[2] = R(g.inv_h[2]);
        } else {
            invh[0] = R(g.inv_hf[0]); invh[1] = R(g.inv_hf[1]); invh[2] = R(g.inv_hf[2]);
        }
        const bool act[3] = {g.n[0] > 1, g.n[1] > 1, g.n[2] > 1};
        for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
            const long long c = w.first + k;
            const R *u = U + g.off + c;
            R e, vx, vy, vz;
            int iters;
            c2p_full<R>(sc, u[0], u[g.cells], u[2 * g.cells], u[3 * g.cells], e, vx, vy, vz, iters);
            R p, c2;
            eos_pc2<R>(sc, e, p, c2);
            const R v2 = vx * vx + vy * vy + vz * vz;
            const R cs = dsqrt_(c2);
            const R inv_den = R(1) / (R(1) - v2 * c2);
            const R vd[3] = {vx, vy, vz};
            R sum = R(0);   // the unsplit scheme's rate: sum over axes (R16c)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (!act[d]) continue;
                R rad = (R(1) - v2) * (R(1) - vd[d] * vd[d] - (v2 - vd[d] * vd[d]) * c2);
                rad = rad < R(0) ? R(0) : rad;
                const R a = vd[d] * (R(1) - c2);
                const R r = (fabs_(a) + cs * dsqrt_(rad)) * inv_den * invh[d];
                if (sum_axes) sum += r;
                else m = max_nan(m, r);
            }
            if (sum_axes) m = max_nan(m, sum);
        }
    }
    if (cur_event >= 0) flush_rate<R>(m, cur_event, clk, red);
}

// ------------------------------------------------------------------ dt
// reading R8: dt = cfl / rate (or the fixed dt), clipped to t_end
__global__ void k_dt(EventClock *__restrict__ clk, double cfl, double fixed_dt, int nevents) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nevents) return;
    EventClock c = clk[i];
    const double rate = __longlong_as_double((long long)c.rate_bits);
    double dt = fixed_dt > 0.0 ? fixed_dt : cfl / rate;
    if (c.t_end > 0.0 && c.t + dt > c.t_end) dt = c.t_end - c.t;
    if (!(dt > 0.0)) dt = 0.0;
    c.t_step = c.t;
    c.dt = dt;
    if (dt > 0.0) c.t = (c.t_end > 0.0 && c.t + dt >= c.t_end) ? c.t_end : c.t + dt;
    if (!(rate == rate) || !(dt == dt)) c.status = 6;
    c.rate_bits = 0ull;
    clk[i] = c;
}

// ------------------------------------------------------------------ jet source
// reading R12: U += dt S(t_step), S = dEdx (1, n) g(x - x0 - n t), in the
// state's precision; cells farther than 9 sigma (g < 1e-17 g(0)) get nothing.
// Blocks of event blockIdx.y cover the box of cells around the jet centre at
// t_step that contains its 9-sigma ball, clipped to the grid: per active axis
// the cells within ceil(9 sigma / h) + 1 of the cell holding the centre (at
// most min(2 (ceil(9 sigma / h) + 1) + 1, n) of them).  The event's constants
// are computed once per block (FP64 is slow on this GPU).
template <class R>
__global__ void k_jet(const EventGeo *__restrict__ ev, R *__restrict__ U,
                      const EventClock *__restrict__ clk) {
    struct JetBox {
        int lo[3], B[3];
        R amp, cx, cy, cz, inv2s2, cut2, nx, ny, nz;
        R x0[3], h[3];   // grid origin and spacing in precision R
        int on;
    };
    __shared__ JetBox jb;
    const int e = blockIdx.y;
    const EventGeo &g = ev[e];
    if (threadIdx.x == 0) {
        const double dt = clk[e].dt;
        jb.on = g.jet_on && dt > 0.0;
        if (jb.on) {
            const double t = clk[e].t_step;
            const double *j = g.jet;
            const double sig = j[7];
            const double cen[3] = {j[0] + j[3] * t, j[1] + j[4] * t, j[2] + j[5] * t};
            for (int d = 0; d < 3; ++d) {
                if (g.n[d] > 1) {
                    const double hw = ceil(9.0 * sig / g.h[d]) + 1.0;
                    const double ic = floor((cen[d] - g.lo[d]) / g.h[d]);
                    const double a = fmax(ic - hw, 0.0), b = fmin(ic + hw, double(g.n[d] - 1));
                    jb.lo[d] = int(a);
                    jb.B[d] = b >= a ? int(b - a) + 1 : 0;
                } else {
                    jb.lo[d] = 0;
                    jb.B[d] = 1;
                }
            }
            const double two_pi_15 = 15.749609945722419;   // (2 pi)^(3/2)
            jb.amp = R(dt * j[6] / (two_pi_15 * sig * sig * sig));
            jb.cx = R(cen[0]); jb.cy = R(cen[1]); jb.cz = R(cen[2]);
            jb.inv2s2 = R(1.0 / (2.0 * sig * sig));
            jb.cut2 = R(81.0 * sig * sig);
            jb.nx = R(j[3]); jb.ny = R(j[4]); jb.nz = R(j[5]);
            for (int d = 0; d < 3; ++d) {
                jb.x0[d] = R(g.lo[d]);
                jb.h[d] = R(g.h[d]);
            }
        }
    }
    __syncthreads();
    if (!jb.on) return;
    // the box lies in one event (nq cells < 2^31): 32-bit index arithmetic
    const unsigned B0 = unsigned(jb.B[0]), B1 = unsigned(jb.B[1]);
    const unsigned total = B0 * B1 * unsigned(jb.B[2]);
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += gridDim.x * blockDim.x) {
        const unsigned q = k / B0;
        const int x = jb.lo[0] + int(k - q * B0);
        const int y = jb.lo[1] + int(q % B1);
        const int z = jb.lo[2] + int(q / B1);
        const R px = jb.x0[0] + (R(x) + R(0.5)) * jb.h[0] - jb.cx;
        const R py = jb.x0[1] + (R(y) + R(0.5)) * jb.h[1] - jb.cy;
        const R pz = jb.x0[2] + (R(z) + R(0.5)) * jb.h[2] - jb.cz;
        const R r2 = px * px + py * py + pz * pz;
        if (r2 > jb.cut2) continue;
        const R s = jb.amp * exp(-r2 * jb.inv2s2);
        R *u = U + g.off + x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
        u[0] += s;
        u[g.cells] += s * jb.nx;
        u[2 * g.cells] += s * jb.ny;
        u[3 * g.cells] += s * jb.nz;
    }
}

// ------------------------------------------------------------------ FP64 sums
// sums of the nq fields (4, or 5 with the charge) per work item: partial[item][nq]
template <class R>
__global__ void k_sums(const EventGeo *__restrict__ ev, const WorkItem *__restrict__ items,
                       int nitems, const R *__restrict__ U, double *__restrict__ partial, int nq) {
    __shared__ double red[5][32];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
            const R *u = U + g.off + w.first + k;
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q] += widen(u[q * g.cells]);
            if (nq == 5) s[4] += widen(u[4 * g.cells]);
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (q == 4 && nq < 5) break;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0)
            for (int q = 0; q < nq; ++q) red[q][wid] = s[q];
        __syncthreads();
        if (int(threadIdx.x) < nq) {
            double t = 0.0;
            for (int k = 0; k < int(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
            partial[(long long)nq * it + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// one block per event (items of an event are consecutive): each thread sums a
// fixed strided subset of the event's block partials, then a fixed-shape tree
// adds the threads' sums, so the result does not depend on timing
constexpr int SUMS_FINAL_THREADS = 256;

__global__ void __launch_bounds__(SUMS_FINAL_THREADS)
k_sums_final(const WorkItem *__restrict__ items, int nitems, const double *__restrict__ partial,
             const EventGeo *__restrict__ ev, double *__restrict__ out, int nevents, int nq) {
    __shared__ double red[5][SUMS_FINAL_THREADS];
    __shared__ int range[2];
    const int e = blockIdx.x;
    if (threadIdx.x < 2) {   // first item of event e (t = 0) and of event e + 1 (t = 1)
        const int key = e + int(threadIdx.x);
        int lo = 0, hi = nitems;
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (items[mid].event < key) lo = mid + 1; else hi = mid;
        }
        range[threadIdx.x] = lo;
    }
    __syncthreads();
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int it = range[0] + int(threadIdx.x); it < range[1]; it += SUMS_FINAL_THREADS) {
        const double *p = partial + (long long)nq * it;
        for (int q = 0; q < nq; ++q) s[q] += p[q];
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = SUMS_FINAL_THREADS / 2; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w)
#pragma unroll
            for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (int(threadIdx.x) < nq) {
        const EventGeo &g = ev[e];
        out[nq * e + threadIdx.x] = red[threadIdx.x][0] * (g.h[0] * g.h[1] * g.h[2]);
    }
}

// ------------------------------------------------------------------ hot spots
// e = e_bg + sum_j A_j g_j, v = sum_j A_j g_j u_j / e, computed in the state's
// precision.  A spot farther than 9 sigma along any axis adds less than
// A exp(-40.5) and is skipped (relative to e_bg = 0.01 and A = 2 that is
// below 1e-15).
template <class R>
__global__ void k_hotspots(const EventGeo *__restrict__ ev, const WorkItem *__restrict__ items,
                           int nitems, const double *__restrict__ spots, int nspots, double sigma,
                           double e_bg, R *__restrict__ U, Scheme sc, int nq) {
    // the event's spots, converted to R once per block and event (a
    // conversion from FP64 per cell and spot issues at the FP64 rate); larger
    // spot lists are read from global memory
    constexpr int HS_MAX = 28672 / int(7 * sizeof(R));
    __shared__ R s_sp[7 * HS_MAX];
    const bool staged = nspots <= HS_MAX;
    int cur = -1;
    const R inv = R(1.0 / (2.0 * sigma * sigma));
    const R cut = R(9.0 * sigma);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        const double *sp = spots + (long long)w.event * nspots * 7;
        if (staged && w.event != cur) {   // block-uniform
            __syncthreads();              // the previous event's spots are no longer read
            for (int j = threadIdx.x; j < 7 * nspots; j += blockDim.x) s_sp[j] = R(sp[j]);
            __syncthreads();
            cur = w.event;
        }
        const int nx = g.n[0], ny = g.n[1];
        // e, M of the cell at (px, py, pz) from spot component j of spot s
        auto cell_sum = [&](R px, R py, R pz, auto get, R &e, R &mx, R &my, R &mz) {
            for (int s = 0; s < nspots; ++s) {
                const R dz = pz - get(s, 2);
                if (fabs_(dz) > cut) continue;
                const R dy = py - get(s, 1);
                if (fabs_(dy) > cut) continue;
                const R dx = px - get(s, 0);
                if (fabs_(dx) > cut) continue;
                // the separable Gaussian as one exponential of the summed squares
                const R a = get(s, 3) * exp(-(dx * dx + dy * dy + dz * dz) * inv);
                e += a;
                mx += a * get(s, 4);
                my += a * get(s, 5);
                mz += a * get(s, 6);
            }
        };
        for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
            const long long c = w.first + k;
            // an event has fewer than 2^31 cells: 32-bit index arithmetic
            const unsigned cu = unsigned(c), q = cu / unsigned(nx);
            const int x = int(cu - q * unsigned(nx));
            const int y = int(q % unsigned(ny));
            const int z = int(q / unsigned(ny));
            const R px = R(g.lo[0] + (x + 0.5) * g.h[0]);
            const R py = R(g.lo[1] + (y + 0.5) * g.h[1]);
            const R pz = R(g.lo[2] + (z + 0.5) * g.h[2]);
            R e = R(e_bg), mx = R(0), my = R(0), mz = R(0);
            if (staged)
                cell_sum(px, py, pz, [&](int s, int j) { return s_sp[7 * s + j]; }, e, mx, my, mz);
            else
                cell_sum(px, py, pz, [&](int s, int j) { return R(sp[7 * s + j]); }, e, mx, my, mz);
            const R vx = mx / e, vy = my / e, vz = mz / e;
            R p, c2;
            eos_pc2<R>(sc, e, p, c2);
            const R g2 = R(1) / (R(1) - (vx * vx + vy * vy + vz * vz));
            const R wv = (e + p) * g2;
            R *u = U + g.off + c;
            u[0] = wv - p;
            u[g.cells] = wv * vx;
            u[2 * g.cells] = wv * vy;
            u[3 * g.cells] = wv * vz;
            if (nq == 5) u[4 * g.cells] = R(0);   // hot-spot states carry no charge
        }
    }
}

// ------------------------------------------------------------------ finite check
template <class R>
__global__ void k_finite(const EventGeo *__restrict__ ev, const WorkItem *__restrict__ items,
                         int nitems, const R *__restrict__ U, EventClock *__restrict__ clk,
                         int nq) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        bool bad = false;
        for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
            const R *u = U + g.off + w.first + k;
            for (int q = 0; q < nq; ++q) bad |= !isfinite(double(u[q * g.cells]));
        }
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) clk[w.event].status = 6;
    }
}

// ------------------------------------------------------------------ Newton test hook
template <class R>
__global__ void k_c2p_newton(Scheme sc, const R *__restrict__ U, long long n, int seed,
                             R *__restrict__ vmag, int *__restrict__ iters) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const R E = U[i], Mx = U[n + i], My = U[2 * n + i], Mz = U[3 * n + i];
    R M2 = Mx * Mx + My * My + Mz * Mz;
    if (!(E > R(0))) { vmag[i] = R(0); iters[i] = 0; return; }
    const R cap = (R(1) - consts<R>(sc).delta) * E;
    if (M2 > cap * cap) M2 = cap * cap;
    const R M = dsqrt_(M2);
    R p;
    int it;
    vmag[i] = newton_speed<R>(sc, E, M, M2, seed, R(0), p, it);
    iters[i] = it;
}

// The paired Newton solve of the tabulated-EOS sweeps (newton_speed2) beside
// two single solves (newton_speed) of the same states, for checking that the
// pair changes nothing: thread i takes states i and i + n/2 (n even) and
// writes |v|, p and the iteration count of the single solves to [0][.] and
// of the paired one to [1][.]; E <= 0 gives zeros (the vacuum of c2p_table).
template <class R, bool RCP>
__global__ void k_c2p_newton_pairs(Scheme sc, const R *__restrict__ U, long long n, int seed,
                                   R *__restrict__ vmag, R *__restrict__ pres,
                                   int *__restrict__ iters) {
    const long long h = n / 2;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= h) return;
    R E[2], M[2], M2[2], given[2] = {R(0), R(0)};
    bool skip[2];
    int sd[2] = {seed, seed};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const long long c = i + s * h;
        E[s] = U[c];
        const R mx = U[n + c], my = U[2 * n + c], mz = U[3 * n + c];
        M2[s] = mx * mx + my * my + mz * mz;
        skip[s] = !(E[s] > R(0));
        const R cap = (R(1) - consts<R>(sc).delta) * E[s];
        if (M2[s] > cap * cap) M2[s] = cap * cap;
        M[s] = dsqrt_(M2[s]);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const long long c = i + s * h;
        R p = R(0), v = R(0);
        int it = 0;
        if (!skip[s]) v = newton_speed<R, RCP>(sc, E[s], M[s], M2[s], seed, R(0), p, it);
        vmag[c] = v;
        pres[c] = p;
        iters[c] = it;
    }
    R v[2], p[2];
    int it[2];
    newton_speed2<R, RCP>(sc, E, M, M2, sd, given, skip, v, p, it);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const long long c = n + i + s * h;
        vmag[c] = skip[s] ? R(0) : v[s];
        pres[c] = skip[s] ? R(0) : p[s];
        iters[c] = skip[s] ? 0 : it[s];
    }
}

// ------------------------------------------------------------------ launchers
#define HY_DISPATCH(prec, call_d, call_f) \
    do {                                  \
        if ((prec) == 0) { call_d; }      \
        else { call_f; }                  \
    } while (0)

cudaError_t launch_prim2cons(const CellLaunch &c, const void *e, const void *vx, const void *vy,
                             const void *vz, const void *n, void *U) {
    HY_DISPATCH(c.prec,
        (k_prim2cons<double><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const double *)e, (const double *)vx, (const double *)vy, (const double *)vz,
            (const double *)n, (double *)U, c.sc, c.nq)),
        (k_prim2cons<float><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const float *)e, (const float *)vx, (const float *)vy, (const float *)vz,
            (const float *)n, (float *)U, c.sc, c.nq)));
    return cudaGetLastError();
}

cudaError_t launch_charge_density(const CellLaunch &c, const void *U, void *n) {
    HY_DISPATCH(c.prec,
        (k_charge_density<double><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const double *)U, (double *)n, c.sc)),
        (k_charge_density<float><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const float *)U, (float *)n, c.sc)));
    return cudaGetLastError();
}

cudaError_t launch_cons2prim(const CellLaunch &c, const void *U, void *e, void *vx, void *vy,
                             void *vz) {
    HY_DISPATCH(c.prec,
        (k_cons2prim<double><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const double *)U, (double *)e, (double *)vx, (double *)vy, (double *)vz, c.sc, 0)),
        (k_cons2prim<float><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const float *)U, (float *)e, (float *)vx, (float *)vy, (float *)vz, c.sc,
            c.mixed)));
    return cudaGetLastError();
}

cudaError_t launch_rate(const CellLaunch &c, const void *U, EventClock *clk, double) {
    HY_DISPATCH(c.prec,
        (k_rate<double><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const double *)U, clk, c.sc, c.rate_sum)),
        (k_rate<float><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const float *)U, clk, c.sc, c.rate_sum)));
    return cudaGetLastError();
}

cudaError_t launch_dt(EventClock *clk, const double *cfl_fixed, int nevents, cudaStream_t s) {
    k_dt<<<(nevents + 127) / 128, 128, 0, s>>>(clk, cfl_fixed[0], cfl_fixed[1], nevents);
    return cudaGetLastError();
}

cudaError_t launch_jet(const CellLaunch &c, void *U, const EventClock *clk) {
    if (c.jet_cells <= 0 || c.nevents <= 0) return cudaSuccess;
    // about 8 cells per thread; the box of one event spread over these blocks
    const long long per_event = (c.jet_cells + 2047) / 2048;
    const dim3 grid((unsigned)(per_event < 1 ? 1 : per_event), (unsigned)c.nevents);
    HY_DISPATCH(c.prec,
        (k_jet<double><<<grid, 256, 0, c.stream>>>(c.ev, (double *)U, clk)),
        (k_jet<float><<<grid, 256, 0, c.stream>>>(c.ev, (float *)U, clk)));
    return cudaGetLastError();
}

cudaError_t launch_sums(const CellLaunch &c, const void *U, double *partial) {
    HY_DISPATCH(c.prec,
        (k_sums<double><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const double *)U, partial, c.nq)),
        (k_sums<float><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const float *)U, partial, c.nq)));
    return cudaGetLastError();
}

cudaError_t launch_sums_final(const WorkItem *items, int nitems, const double *partial,
                              const EventGeo *ev, double *out, int nevents, int nq, cudaStream_t s) {
    k_sums_final<<<nevents, SUMS_FINAL_THREADS, 0, s>>>(items, nitems, partial, ev, out, nevents,
                                                        nq);
    return cudaGetLastError();
}

cudaError_t launch_hotspots(const CellLaunch &c, const double *spots, int nspots, double sigma,
                            double e_bg, void *U) {
    HY_DISPATCH(c.prec,
        (k_hotspots<double><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems, spots,
            nspots, sigma, e_bg, (double *)U, c.sc, c.nq)),
        (k_hotspots<float><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems, spots,
            nspots, sigma, e_bg, (float *)U, c.sc, c.nq)));
    return cudaGetLastError();
}

cudaError_t launch_finite(const CellLaunch &c, const void *U, EventClock *clk) {
    HY_DISPATCH(c.prec,
        (k_finite<double><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const double *)U, clk, c.nq)),
        (k_finite<float><<<c.blocks, c.threads, 0, c.stream>>>(c.ev, c.items, c.nitems,
            (const float *)U, clk, c.nq)));
    return cudaGetLastError();
}

cudaError_t launch_c2p_newton_pairs(int prec, const Scheme &sc, const void *U, long long n,
                                    int seed, int rcp, void *vmag, void *pres, int *iters,
                                    cudaStream_t s) {
    const long long h = n / 2;
    if (h <= 0) return cudaSuccess;
    const int th = 128;
    const unsigned bl = (unsigned)((h + th - 1) / th);
#define HY_PAIRS(R, RCP)                                                                      \
    k_c2p_newton_pairs<R, RCP><<<bl, th, 0, s>>>(sc, (const R *)U, n, seed, (R *)vmag,        \
                                                 (R *)pres, iters)
    if (prec == 0) {
        if (rcp) HY_PAIRS(double, true);
        else HY_PAIRS(double, false);
    } else {
        if (rcp) HY_PAIRS(float, true);
        else HY_PAIRS(float, false);
    }
#undef HY_PAIRS
    return cudaGetLastError();
}

cudaError_t launch_c2p_newton(int prec, const Scheme &sc, const void *U, long long n, int seed,
                              void *vmag, int *iters, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int th = 128;
    const long long bl = (n + th - 1) / th;
    HY_DISPATCH(prec,
        (k_c2p_newton<double><<<(unsigned)bl, th, 0, s>>>(sc, (const double *)U, n, seed,
            (double *)vmag, iters)),
        (k_c2p_newton<float><<<(unsigned)bl, th, 0, s>>>(sc, (const float *)U, n, seed,
            (float *)vmag, iters)));
    return cudaGetLastError();
}

}  // namespace hy
