// kernels.h -- host-side entry points of the kernels (C++ linkage, internal).
#pragma once
#include <cuda_runtime.h>

#include "common.h"

namespace hy {

struct SweepLaunch {
    const void *in;
    void *out;
    const EventGeo *ev;
    const WorkItem *items;
    int nitems;
    int axis;
    double frac;             // the sweep's share of the step dt
    const EventClock *clk;
    Scheme sc;
    int rk;
    int threads, blocks;
    int charge = 0;          // 1: the state carries the conserved charge as field 4
    int *counter;            // non-null: persistent grid pulling items from this counter
    EventClock *rate_clk;    // non-null: accumulate the CFL rate of the output state here
    int sms;
    cudaStream_t stream;
};

cudaError_t launch_sweep_f64(const SweepLaunch &a);
cudaError_t launch_sweep_f32(const SweepLaunch &a);
cudaError_t launch_sweep_mixed(const SweepLaunch &a);

// One RK stage of the unsplit scheme (Eq. 13 with all flux terms, reading
// R16): evolved faces, then per tile of cells the MUSTA-FORCE fluxes of every
// active axis, the divergence and the stage combination of Eq. 5-7.
struct UnsplitLaunch {
    const void *in;          // state the stage differentiates (U^n, U1 or U2)
    const void *u0;          // U^n
    const void *u1;          // U1 (stages 2-3), U2 (stage 3 of RK3)
    void *out;               // the stage result
    void *faces;             // scratch laid out by UnsplitGeo
    const EventGeo *ev;
    const UnsplitGeo *ug;
    const WorkItem *face_items, *tile_items;
    int n_face_items, n_tile_items;
    const EventClock *clk;
    Scheme sc;
    int rk, stage;           // stage 1..rk
    EventClock *rate_clk;    // non-null on the last stage: CFL rate (sum over axes) of out
    int sms;
    cudaStream_t stream;
};

cudaError_t launch_unsplit_f64(const UnsplitLaunch &a);
cudaError_t launch_unsplit_f32(const UnsplitLaunch &a);
cudaError_t launch_unsplit_mixed(const UnsplitLaunch &a);

// Cell-wise kernels over work items of cells (prec: 0 double, 1/2 float).
struct CellLaunch {
    const EventGeo *ev;
    const WorkItem *items;
    int nitems;
    int threads, blocks;
    cudaStream_t stream;
    int prec;             // 0 double, 1 float
    int mixed;            // float state, cons->prim redone in double where |v| > 0.99
    Scheme sc;
    int rate_sum = 0;     // launch_rate: sum over axes (unsplit scheme) instead of max
    long long jet_cells = 0;   // launch_jet: cells of the largest box around a jet
    int nevents = 0;
    int nq = 4;           // conserved fields per cell: 4, or 5 with the charge
};

// with c.nq = 5 also R = n gamma from n (null: R = 0)
cudaError_t launch_prim2cons(const CellLaunch &c, const void *e, const void *vx, const void *vy,
                             const void *vz, const void *n, void *U);
// n = R / gamma per cell (outputs indexed like launch_cons2prim's)
cudaError_t launch_charge_density(const CellLaunch &c, const void *U, void *n);
cudaError_t launch_cons2prim(const CellLaunch &c, const void *U, void *e, void *vx, void *vy,
                             void *vz);
// max over cells of speed/dx, maximised (or with rate_sum summed) over the swept
// axes, into clk[event].rate_bits (atomic max)
cudaError_t launch_rate(const CellLaunch &c, const void *U, EventClock *clk, double cfl_unused);
// per-event dt from rate_bits (resets it), t_step = t, t += dt
cudaError_t launch_dt(EventClock *clk, const double *cfl_fixed, int nevents, cudaStream_t s);
cudaError_t launch_jet(const CellLaunch &c, void *U, const EventClock *clk);
// FP64 partial sums per work item: partial[item][nq]; per event out[event][nq]
cudaError_t launch_sums(const CellLaunch &c, const void *U, double *partial);
cudaError_t launch_sums_final(const WorkItem *items, int nitems, const double *partial,
                              const EventGeo *ev, double *out, int nevents, int nq,
                              cudaStream_t s);
cudaError_t launch_hotspots(const CellLaunch &c, const double *spots, int nspots, double sigma,
                            double e_bg, void *U);
cudaError_t launch_finite(const CellLaunch &c, const void *U, EventClock *clk);
cudaError_t launch_c2p_newton_pairs(int prec, const Scheme &sc, const void *U, long long n,
                                    int seed, int rcp, void *vmag, void *pres, int *iters,
                                    cudaStream_t s);
cudaError_t launch_c2p_newton(int prec, const Scheme &sc, const void *U, long long n, int seed,
                              void *vmag, int *iters, cudaStream_t s);

// Newton-seed MLP
cudaError_t launch_mlp_forward(const float *params, const float *X, int n, float *out,
                               cudaStream_t s);
cudaError_t launch_mlp_hidden(const float *params, const float *X, int n, float *H1,
                              cudaStream_t s);
cudaError_t launch_mlp_loss_grad(const float *params, const float *X, const float *Y, int n,
                                 float *grad, float *loss, cudaStream_t s);
cudaError_t launch_mlp_prepare(const float *params, void *w_bf16, cudaStream_t s);

// message returned by hydro_last_error() (thread-local)
void set_last_error(const char *msg);

}  // namespace hy
