// unsplit.cuh -- one RK stage of the unsplit multi-D MUSCL-Hancock
// MUSTA-FORCE scheme: the Hancock half step of Eq. 13 with all three flux
// terms, the FORCE alpha of Eq. 10-11 (3 in 3-D), the RK stages of Eq. 5-7 on
// the whole field (reading R16).
//
// Two kernels per stage:
//   k_us_faces   evolved faces of every cell of the box grown by one cell
//                along each active axis (ghosts mapped by the BCs), written to
//                HBM scratch laid out by UnsplitGeo;
//   k_us_tile    per tile of cells: the MUSTA-FORCE flux of every interface of
//                the tile, axis by axis, in shared memory; dt L(U) =
//                -sum_d dt/dx_d (F_d,i+1/2 - F_d,i-1/2); the RK stage
//                combination; on the last stage also the CFL rate (sum over
//                axes, R16c) of the new state.
#pragma once
#include <atomic>

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

// Blocks of US_THREADS per SM the two kernels are compiled for. FP32 with the
// conformal EOS: four (64 registers, 32 warps per SM); the load latencies of
// these kernels need the warps more than the registers. The tabulated EOS's
// Newton solve needs more registers (two blocks, 128), FP64 more still.
template <class R, int PREC, int EOSK>
constexpr int us_faces_blocks() {
    return sizeof(R) == 8 ? 1 : (EOSK == EOS_CONFORMAL ? 4 : 2);
}
template <class R, int PREC, int EOSK>
constexpr int us_tile_blocks() {
    return sizeof(R) == 8 ? (EOSK == EOS_CONFORMAL ? 2 : 1)
                          : (EOSK == EOS_CONFORMAL ? (PREC == PREC_MIXED ? 3 : 4) : 2);
}

template <class R, int PREC, int EOSK, int LIM, bool COUNT>
__global__ void __launch_bounds__(US_THREADS, us_faces_blocks<R, PREC, EOSK>())
k_us_faces(const R *__restrict__ in, R *__restrict__ faces, const EventGeo *__restrict__ ev,
           const UnsplitGeo *__restrict__ ugeo, const WorkItem *__restrict__ items, int nitems,
           const EventClock *__restrict__ clk, Scheme sc) {
    Physics<R, PREC, EOSK, LIM, COUNT> ph;
    ph.sc = sc;
    const R half = R(0.5);
    // half dt / dx_d of the event of the last item: recomputed only when the
    // event changes (FP64 divisions issue at a small fraction of the FP32 rate)
    int cur = -1;
    R hlam[3] = {R(0), R(0), R(0)};
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        const UnsplitGeo &u = ugeo[w.event];
        if (w.event != cur) {
            cur = w.event;
            const double dt = clk[cur].dt;
#pragma unroll
            for (int d = 0; d < 3; ++d) hlam[d] = half * R(dt / g.h[d]);
        }
        // lanes past the item's end repeat its first unit and store nothing,
        // so a warp stays converged (the MLP Newton seed needs that)
        const bool valid = int(threadIdx.x) < w.count;
        // grown boxes hold fewer than 2^31 cells: 32-bit index arithmetic
        const unsigned gi = unsigned(w.first) + (valid ? threadIdx.x : 0u);
        const unsigned m0 = unsigned(u.m[0]), m1 = unsigned(u.m[1]);
        const unsigned r = gi / m0;
        const int x[3] = {int(gi - r * m0) - u.g[0], int(r % m1) - u.g[1], int(r / m1) - u.g[2]};
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
                const V4<R> FL = from_axis(ph.flux(to_axis(UL[d], d)), d);
                const V4<R> FR = from_axis(ph.flux(to_axis(UR[d], d)), d);
                h = vfma<R>(hlam[d], vsub(FL, FR), h);
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

template <class R>
__device__ __forceinline__ R us_max_nan(R a, R b) { return (b > a || b != b) ? b : a; }

// Fluxes and update of one RK stage over tiles of cells, in one kernel: a
// block takes a tile of at most US_TX x US_TY x US_TZ cells, evaluates the
// MUSTA-FORCE flux of every interface of the tile along every active axis
// (its boundary planes included, which the neighbouring tile evaluates too)
// into shared memory, then adds lambda_d (F_i+1/2 - F_i-1/2) per axis, in
// axis order, to the divergence its threads hold per cell.
// The interface fluxes never travel through HBM.
constexpr int US_TILE = US_TX * US_TY * US_TZ;
constexpr int US_CPT = US_TILE / US_THREADS;                  // cells per thread
// interfaces of a full tile along x, y and z, and the flux buffer
// [axis][4 fields][interfaces of the axis] packed without padding, so that
// four blocks of the FP32 kernel fit the 228 KB of shared memory of an SM
constexpr int US_NI0 = (US_TX + 1) * US_TY * US_TZ;
constexpr int US_NI1 = US_TX * (US_TY + 1) * US_TZ;
constexpr int US_NI2 = US_TX * US_TY * (US_TZ + 1);
constexpr int US_FLUX_FLOATS = 4 * (US_NI0 + US_NI1 + US_NI2);
__host__ __device__ constexpr int us_fbase(int d) {
    return d == 0 ? 0 : (d == 1 ? 4 * US_NI0 : 4 * (US_NI0 + US_NI1));
}
__host__ __device__ constexpr int us_fstride(int d) {
    return d == 0 ? US_NI0 : (d == 1 ? US_NI1 : US_NI2);
}

// tile extents of an event (1 on an axis of one cell) and tiles per axis
__device__ __forceinline__ void us_tile_shape(const EventGeo &g, int T[3], int nt[3]) {
    const int full[3] = {US_TX, US_TY, US_TZ};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        T[d] = g.n[d] < full[d] ? g.n[d] : full[d];
        nt[d] = (g.n[d] + T[d] - 1) / T[d];
    }
}

// k / d by a multiply-high with the rounded-up reciprocal m = ceil(2^32 / d)
// (d = 1 taken apart). With k = q d + r and m d = 2^32 + e, 0 <= e < d:
// k m / 2^32 = q + (r + k e / 2^32) / d, whose floor is q while k d < 2^32,
// which holds for every index of a tile (k < 2^11, d <= 33).
struct UsDiv {
    unsigned m;
    bool one;
    __device__ __forceinline__ void init(int d) {
        one = d == 1;
        m = one ? 0u : 0xffffffffu / unsigned(d) + 1u;
    }
    __device__ __forceinline__ int q(int k) const {
        return one ? k : int(__umulhi(unsigned(k), m));
    }
};

template <class R, int PREC, int EOSK, bool COUNT, bool RATE>
__global__ void __launch_bounds__(US_THREADS, us_tile_blocks<R, PREC, EOSK>())
k_us_tile(const R *__restrict__ faces, const R *__restrict__ u0, const R *__restrict__ u1,
          R *__restrict__ out, const EventGeo *__restrict__ ev, const UnsplitGeo *__restrict__ ugeo,
          const WorkItem *__restrict__ items, int nitems, const EventClock *__restrict__ clk,
          Scheme sc, int rk, int stage, EventClock *rate_clk) {
    Physics<R, PREC, EOSK, -1, COUNT> ph;
    ph.sc = sc;
    extern __shared__ __align__(16) unsigned char us_fs_raw[];
    R *Fs = reinterpret_cast<R *>(us_fs_raw);   // US_FLUX_FLOATS
    __shared__ R red[US_THREADS / 32];
    const R half = R(0.5), q3 = R(0.75), q1 = R(0.25), third = R(1.0 / 3.0), two3 = R(2.0 / 3.0);
    // dt / dx_d, alpha dt / dx_d and 1 / (4 alpha dt / dx_d) of the event of
    // the last tile, recomputed only when the event changes
    int cur = -1;
    R lam[3], al[3], hclf[3];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const EventGeo &g = ev[w.event];
        const UnsplitGeo &u = ugeo[w.event];
        if (w.event != cur) {
            cur = w.event;
            const double dt = clk[cur].dt;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                lam[d] = R(dt / g.h[d]);
                al[d] = ph.K().alpha * lam[d];      // as Physics::set_lam
                hclf[d] = R(0.25) / al[d];
            }
        }
        int T[3], nt[3];
        us_tile_shape(g, T, nt);
        const int tile = int(w.first);
        const int o[3] = {(tile % nt[0]) * T[0], ((tile / nt[0]) % nt[1]) * T[1],
                          (tile / (nt[0] * nt[1])) * T[2]};
        // cells of this tile (clipped to the grid)
        int E[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) E[d] = min(T[d], g.n[d] - o[d]);
        const int ncell = E[0] * E[1] * E[2];
        // the tile's interfaces along each axis: E[d] + 1 planes of E[a] x E[b]
        // (none on an inactive axis), numbered axis after axis in one range
        int nint[3], I[3][3];
        UsDiv dv[3][2];
        long long stepd[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int a = 0; a < 3; ++a) I[d][a] = E[a] + (a == d);
            dv[d][0].init(I[d][0]);
            dv[d][1].init(I[d][1]);
            nint[d] = u.g[d] ? I[d][0] * I[d][1] * I[d][2] : 0;
            stepd[d] = d == 0 ? 1 : (d == 1 ? u.m[0] : (long long)u.m[0] * u.m[1]);
        }
        const int ntot = nint[0] + nint[1] + nint[2];
        // every thread runs the same number of rounds (lanes past the end
        // repeat the first interface and store nothing): the MLP seed needs
        // whole warps
        const int rounds = (ntot + US_THREADS - 1) / US_THREADS;
#pragma unroll 1
        for (int r = 0; r < rounds; ++r) {
            const int k = r * US_THREADS + int(threadIdx.x);
            const bool valid = k < ntot;
            int kk = valid ? k : 0;
            int d = 0;
            if (kk >= nint[0]) {
                kk -= nint[0];
                d = 1;
                if (kk >= nint[1]) {
                    kk -= nint[1];
                    d = 2;
                }
            }
            // (kk mod i0, (kk / i0) mod i1, kk / (i0 i1)) of the interface planes
            const int qi = dv[d][0].q(kk), qj = dv[d][1].q(qi);
            const int x0 = o[0] + kk - qi * I[d][0], x1 = o[1] + qi - qj * I[d][1], x2 = o[2] + qj;
            // grown-box index of the cell right of the interface, and left of it
            const long long gr = (x0 + u.g[0]) +
                                 (long long)u.m[0] * ((x1 + u.g[1]) + (long long)u.m[1] * (x2 + u.g[2]));
            const long long gl = gr - stepd[d];
            const R *fr = us_face(faces, u, d, 1, gl);   // right face of the left cell
            const R *fl = us_face(faces, u, d, 0, gr);   // left face of the right cell
            const V4<R> UL = v4<R>(fr[0], fr[u.gcells], fr[2 * u.gcells], fr[3 * u.gcells]);
            const V4<R> UR = v4<R>(fl[0], fl[u.gcells], fl[2 * u.gcells], fl[3 * u.gcells]);
            ph.al_ = al[d];
            ph.hclf_ = hclf[d];
            // Sec. 2.4 steps 1-5 at this interface (R3)
            const V4<R> F = from_axis(ph.musta(to_axis(UL, d), to_axis(UR, d), lam[d]), d);
            if (valid) {
                const int st = us_fstride(d);
                R *f = Fs + us_fbase(d) + kk;
                f[0] = F.e;
                f[st] = F.n;
                f[2 * st] = F.t1;
                f[3 * st] = F.t2;
            }
        }
        __syncthreads();
        report_flags(sc, w.event, ph.flags_);
        // per cell of the tile: dt L(U) = -D, D = sum_d dt/dx_d (F_d,i+1/2 -
        // F_d,i-1/2) with the axes in order, then the RK stage combination of
        // Eq. 5-7
        UsDiv de0, de1;
        de0.init(E[0]);
        de1.init(E[1]);
        // flux-plane offset of the interface past the cell along each axis
        const int sp[3] = {1, I[1][0], I[2][0] * I[2][1]};
        R m = R(0);
        R ih[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) ih[d] = R(g.inv_h[d]);
#pragma unroll
        for (int j = 0; j < US_CPT; ++j) {
            const int c = j * US_THREADS + int(threadIdx.x);
            if (c >= ncell) continue;
            const int qa = de0.q(c), qb = de1.q(qa);
            const int l0 = c - qa * E[0], l1 = qa - qb * E[1], l2 = qb;
            V4<R> D = v4<R>(R(0), R(0), R(0), R(0));
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (!nint[d]) continue;
                const R *f = Fs + us_fbase(d);
                constexpr int st[3] = {US_NI0, US_NI1, US_NI2};
                const int im = l0 + I[d][0] * (l1 + I[d][1] * l2);
                const int ip = im + sp[d];
                const V4<R> Fm = v4<R>(f[im], f[st[d] + im], f[2 * st[d] + im],
                                       f[3 * st[d] + im]);
                const V4<R> Fp = v4<R>(f[ip], f[st[d] + ip], f[2 * st[d] + ip],
                                       f[3 * st[d] + ip]);
                D = vfma<R>(lam[d], vsub(Fp, Fm), D);
            }
            const long long cc =
                (o[0] + l0) + (long long)g.n[0] * ((o[1] + l1) + (long long)g.n[1] * (o[2] + l2));
            const V4<R> U0 = us_load(u0, g, cc);
            V4<R> r;
            if (stage == 1) {
                r = vsub(U0, D);                             // U + dt L(U)
            } else if (rk == 2) {
                const V4<R> U1 = us_load(u1, g, cc);         // Eq. 6
                r = vmul<R>(half, vsub(vadd(U0, U1), D));
            } else if (stage == 2) {
                const V4<R> U1 = us_load(u1, g, cc);         // Eq. 7, U2
                r = vadd(vmul<R>(q3, U0), vmul<R>(q1, vsub(U1, D)));
            } else {
                const V4<R> U2 = us_load(u1, g, cc);         // Eq. 7, U^{n+1}
                r = vadd(vmul<R>(third, U0), vmul<R>(two3, vsub(U2, D)));
            }
            us_store(out, g, cc, r);
            if (RATE && rate_clk) {   // R16c: sum over the active axes
                R rr = R(0);
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    if (u.g[d]) rr += ph.rate(to_axis(r, d), ih[d], R(0), R(0), true);
                m = us_max_nan(m, rr);
            }
        }
        __syncthreads();   // Fs is refilled by the next tile
        if (RATE && rate_clk) {   // block max, one atomic per tile
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) m = us_max_nan(m, __shfl_xor_sync(0xffffffffu, m, s));
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

// the tile kernel's flux buffer exceeds the default 48 KB of shared memory:
// opt in once per kernel instantiation and device (the template arguments key
// the flag: the instantiations share one function-pointer type) and clear the
// error state of a failed opt-in
template <class R, int PREC, int EOSK, bool COUNT, bool RATE, class K>
cudaError_t us_tile_optin(K kfn, size_t bytes) {
    static std::atomic<unsigned long long> opted{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (opted.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    opted.fetch_or(bit);
    return cudaSuccess;
}

template <class R, int PREC>
cudaError_t launch_unsplit_prec(const UnsplitLaunch &a) {
    const size_t tile_smem = size_t(US_FLUX_FLOATS) * sizeof(R);
    const R *in = static_cast<const R *>(a.in);
    R *faces = static_cast<R *>(a.faces);
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
        if (a.sc.counters) {                                                                     \
            if (a.rate_clk)                                                                      \
                HY_US_TILE(EOSK, true, true)                                                     \
            else                                                                                 \
                HY_US_TILE(EOSK, true, false)                                                    \
        } else {                                                                                 \
            if (a.rate_clk)                                                                      \
                HY_US_TILE(EOSK, false, true)                                                    \
            else                                                                                 \
                HY_US_TILE(EOSK, false, false)                                                   \
        }                                                                                        \
    }
#define HY_US_TILE(EOSK, COUNT, RATE)                                                            \
    {                                                                                            \
        auto kfn = &k_us_tile<R, PREC, EOSK, COUNT, RATE>;                                      \
        cudaError_t e_ = us_tile_optin<R, PREC, EOSK, COUNT, RATE>(kfn, tile_smem);              \
        if (e_ != cudaSuccess) return e_;                                                        \
        kfn<<<blocks(a.n_tile_items), US_THREADS, tile_smem, a.stream>>>(                        \
            faces, static_cast<const R *>(a.u0), static_cast<const R *>(a.u1),                  \
            static_cast<R *>(a.out), a.ev, a.ug, a.tile_items, a.n_tile_items, a.clk, a.sc,      \
            a.rk, a.stage, a.rate_clk);                                                          \
    }
    if (a.sc.eos_kind == EOS_CONFORMAL) HY_US_FACES(EOS_CONFORMAL)
    else if (mlp) HY_US_FACES(EOS_TABLE_MLP)
    else HY_US_FACES(EOS_TABLE)
#undef HY_US_FACES
#undef HY_US_TILE
    return cudaGetLastError();
}

}  // namespace hy
