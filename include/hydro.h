/*
 * hydro.h -- C ABI of the B300 MUSTA-FORCE solver for ideal relativistic
 * hydrodynamics (Porter-Sobieraj et al., "A MUSTA-FORCE algorithm for solving
 * partial differential equations of relativistic hydrodynamics").
 *
 * The solver advances the conserved energy-momentum density
 * U = (E, Mx, My, Mz) = (T^00, T^0x, T^0y, T^0z) of Sec. 2.1 (Eq. 1, 3, 4)
 * on Cartesian grids with slope-limited MUSCL reconstruction (Sec. 2.5),
 * the Hancock half step and the MUSTA-FORCE interface flux (Sec. 2.4),
 * cons->prim recovery (Sec. 2.6, Eq. 23) and Runge-Kutta stages (Sec. 2.3),
 * dimension by dimension (Strang splitting).
 *
 * Conventions shared by every entry point
 *  - Layout: fields are structure-of-arrays, field-major, x fastest:
 *    U[nq][nz][ny][nx] with nq = 4, or nq = 5 when the grid carries the
 *    conserved charge R = n gamma as field 4 (hydro_grid_t.charge);
 *    primitive arrays e, vx, vy, vz, n are [nz][ny][nx].
 *  - Element type: double for HYDRO_FP64 handles, float for HYDRO_FP32 and
 *    HYDRO_MIXED handles (state, primitives and conserved arrays alike).
 *  - on_device = 1: the pointer is CUDA device memory readable/writable on
 *    the handle's stream; 0: host memory (pageable or pinned).  Caller
 *    buffers are borrowed for the duration of the call only; the library
 *    owns all of its device state.
 *  - Every call returns a hydro_status; on failure hydro_last_error() gives
 *    a message (thread-local).  Device-side trouble never traps: the kernels
 *    set per-event status bits (HYDRO_FLAG_*) that hydro_check_status and
 *    hydro_batch_event_status read after the steps, and opt-in counters
 *    (hydro_counters) count each kind of event.
 *  - Handles are not thread-safe.  Calls on one handle are ordered on its
 *    stream; calls that return host data synchronise that stream.
 */
#ifndef HYDRO_H
#define HYDRO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HYDRO_OK = 0,
    HYDRO_E_INVALID = 1,      /* bad argument or configuration */
    HYDRO_E_OOM = 2,          /* device allocation failed */
    HYDRO_E_CUDA = 3,         /* a CUDA runtime call failed */
    HYDRO_E_UNPHYSICAL = 4,   /* an inadmissible state was met and repaired (status checks) */
    HYDRO_E_NEWTON = 5,       /* a Newton cons->prim solve hit its iteration cap (status checks) */
    HYDRO_E_NONFINITE = 6     /* the state holds NaN or Inf (hydro_check_finite) */
} hydro_status;

/* Slope limiters of Sec. 2.5 (Eq. 18-21) plus MC; NONE is the central slope of Eq. 14. */
typedef enum {
    HYDRO_LIM_NONE = 0,
    HYDRO_LIM_MINMOD = 1,     /* Minbee, Eq. 18 */
    HYDRO_LIM_MC = 2,         /* monotonized central, xi = max(0, min(2r, (1+r)/2, 2)) */
    HYDRO_LIM_SUPERBEE = 3,   /* Eq. 19 */
    HYDRO_LIM_VANLEER = 4,    /* Eq. 21 */
    HYDRO_LIM_VANALBADA = 5   /* Eq. 20, zero for r <= 0 */
} hydro_limiter;

typedef enum {
    HYDRO_FP64 = 0,           /* state, fluxes and cons->prim in double */
    HYDRO_FP32 = 1,           /* state, fluxes and cons->prim in float */
    HYDRO_MIXED = 2           /* float state and fluxes; cons->prim redone in double where |v| > 0.99 */
} hydro_precision;

typedef enum { HYDRO_BC_PERIODIC = 0, HYDRO_BC_OUTFLOW = 1 } hydro_bc;

typedef enum { HYDRO_EOS_CONFORMAL = 0, HYDRO_EOS_TABLE = 1 } hydro_eos_kind;

/* Initial guess of the Newton cons->prim solve for HYDRO_EOS_TABLE. */
typedef enum {
    HYDRO_SEED_ZERO = 0,      /* v0 = 0, the start of the paper's fixed-point iteration (Sec. 2.6) */
    HYDRO_SEED_CONFORMAL = 1, /* closed-form p = e/3 solution */
    HYDRO_SEED_MLP = 2        /* BF16 tensor-core MLP (ln E, |M|/E) -> v0 where the EOS is not
                                 conformal (hydro_mlp_seed_emin), the closed form elsewhere */
} hydro_seed;

/* One Cartesian grid (one event). */
typedef struct {
    int nx, ny, nz;           /* cells per axis; an axis with 1 cell is not swept */
    double dx, dy, dz;        /* cell sizes */
    double x0, y0, z0;        /* lower corner of the box (cell i has centre x0 + (i+1/2) dx) */
    int bc[3];                /* hydro_bc per axis */
    int prec;                 /* hydro_precision */
    int rk_order;             /* 1 (single-stage MUSCL-Hancock), 2 (Eq. 6) or 3 (Eq. 7) */
    int hancock;              /* 1: Hancock half step of Eq. 13 inside each stage (paper); 0: off */
    double cfl;               /* Courant number of the CFL time step */
    double fixed_dt;          /* > 0: use this time step instead of the CFL step */
    double alpha;             /* FORCE alpha of Eq. 10-11 (1 for split sweeps, 3 for unsplit 3-D) */
    int unsplit;              /* 0: Strang-split sweeps X(1/2) Y(1/2) Z(1) Y(1/2) X(1/2);
                                 1: the unsplit MUSCL-Hancock step of Eq. 13 with every flux
                                 term, one RK update of the whole field per stage, CFL rate
                                 summed over the axes; all events of a batch must agree */
    int charge;               /* 1: carry the conserved charge R = n gamma (Eq. 1, 3, 4) as a
                                 fifth field with flux R v_d.  The EOS is p(e), so R rides on
                                 the energy-momentum flow and n = R / gamma on readout.  Split
                                 sweeps only (HYDRO_E_INVALID with unsplit = 1 or the MLP
                                 seed); all events of a batch must agree */
} hydro_grid_t;

/* Equation of state p(e) of Eq. 2 (no charge). */
typedef struct {
    int kind;                 /* hydro_eos_kind */
    double cs2;               /* CONFORMAL: p = cs2 * e */
    int n;                    /* TABLE: number of nodes, uniform in ln e */
    double lne_min, lne_max;  /* TABLE: ln e of the first and last node */
    const double *cs2_tab;    /* TABLE: host array [n] of c_s^2 at the nodes (copied) */
    const double *p_tab;      /* TABLE: host array [n] of p at the nodes (copied) */
    int seed;                 /* hydro_seed (TABLE only) */
    const float *mlp_params;  /* host array [hydro_mlp_nparam()] (copied), for HYDRO_SEED_MLP */
    double newton_tol;        /* |dv| stop of the Newton solve; <= 0 picks 1e-13 (FP64) or 2e-6 (FP32) */
    int newton_max_iter;      /* iteration cap of the Newton solve, 1..1000; <= 0 picks 50.  A
                                 solve that reaches it keeps its bracketed iterate and sets
                                 HYDRO_FLAG_NEWTON on its event */
} hydro_eos_t;

/* Per-event status bits set by the kernels; they accumulate until the
 * event's state is set again (set_primitives, set_conserved, init_hotspots). */
#define HYDRO_FLAG_NEWTON 1u      /* a Newton cons->prim solve hit newton_max_iter */
#define HYDRO_FLAG_UNPHYSICAL 2u  /* |M| >= (1 - delta) E met and capped in cons->prim, or a
                                     cell's evolved faces were inadmissible and fell back to
                                     its average (the admissibility rule of the scheme) */

typedef struct hydro_s hydro_t;
typedef struct hydro_batch_s hydro_batch_t;

/* Thread-local message of the last failing call ("" if none). */
const char *hydro_last_error(void);

/* ---------------------------------------------------------------- single grid */

/* Validate the grid, EOS, limiter and MUSTA stage count (>= 1), allocate the
 * device state (two copies for ping-pong sweeps) and return a handle.
 * Errors: HYDRO_E_INVALID (sizes < 1, more than 536,870,911 cells, unknown enums, rk_order not 1..3,
 * stages < 1, dx <= 0, EOS table with n < 2), HYDRO_E_OOM, HYDRO_E_CUDA. */
hydro_status hydro_create(const hydro_grid_t *grid, const hydro_eos_t *eos, int limiter,
                          int stages, hydro_t **out);
void hydro_destroy(hydro_t *h);

/* Use this CUDA stream (a cudaStream_t passed as void*) for all later work;
 * NULL returns to the handle's own non-blocking stream (the default).  Device
 * pointers passed to later calls must be ready on that stream. */
hydro_status hydro_set_stream(hydro_t *h, void *stream);

/* Set the state from primitive fields (e, v): prim->cons of Eq. 4.  Sets t = 0. */
hydro_status hydro_set_primitives(hydro_t *h, const void *e, const void *vx, const void *vy,
                                  const void *vz, int on_device);
/* Charged handles: the state from (e, v) and the rest-frame charge density n
 * (R = n gamma).  hydro_set_primitives on a charged handle sets R = 0. */
hydro_status hydro_set_primitives_charged(hydro_t *h, const void *e, const void *vx,
                                          const void *vy, const void *vz, const void *n,
                                          int on_device);
/* Charged handles: n = R / gamma per cell [nz][ny][nx] (v from cons->prim of
 * the energy-momentum fields; a vacuum cell reads n = R). */
hydro_status hydro_get_charge_density(hydro_t *h, void *n, int on_device);
/* Charged handles: the FP64 sum over cells of R dV. */
hydro_status hydro_charge_sum(hydro_t *h, double *out);
/* Set / read the conserved state U[nq][nz][ny][nx]. */
hydro_status hydro_set_conserved(hydro_t *h, const void *U, int on_device);
hydro_status hydro_get_conserved(hydro_t *h, void *U, int on_device);
/* Read primitives e, vx, vy, vz (cons->prim of Eq. 23 on the device).  A cell
 * with E <= 2^-500 (FP64) or 2^-60 (FP32, mixed) reads as vacuum, e = v = 0:
 * below that E^2 underflows in the recovery. */
hydro_status hydro_get_primitives(hydro_t *h, void *e, void *vx, void *vy, void *vz,
                                  int on_device);

/* Build the state from hot spots: e = e_bg + sum_j A_j exp(-|x-c_j|^2/(2 sigma^2)),
 * v = sum_j A_j g_j u_j / e.  spots: host array [nspots][7] = (cx, cy, cz, A, ux, uy, uz). */
hydro_status hydro_init_hotspots(hydro_t *h, const double *spots, int nspots, double sigma,
                                 double e_bg);
/* Jet source (x0, y0, z0, nx, ny, nz, dE/dx, sigma), added as U += dt S(t) once per step
 * (energy and momentum only; a hot-spot state carries no charge, R = 0). */
hydro_status hydro_set_jet(hydro_t *h, const double jet[8]);

/* Advance up to nsteps full steps (CFL or fixed dt, jet source, Strang sweeps),
 * stopping at t_end when t_end > 0 (the last step is clipped to reach it).
 * t_out (may be NULL) receives the time reached. */
hydro_status hydro_step(hydro_t *h, int nsteps, double t_end, double *t_out);

/* One directional sweep (axis 0, 1, 2) of length dt: all RK stages of Sec. 2.3
 * over every pencil along that axis.  Used to check single sweeps; it runs the
 * split sweep even on a handle created with unsplit = 1. */
hydro_status hydro_sweep(hydro_t *h, int axis, double dt);

/* max over cells of (largest characteristic speed) / dx, taken as the max over
 * the swept axes (split sweeps) or their sum (unsplit = 1): the CFL step is
 * cfl / rate.  A vacuum cell contributes c_s / dx. */
hydro_status hydro_max_rate(hydro_t *h, double *rate);

/* FP64 sums over cells of E dV, Mx dV, My dV, Mz dV. */
hydro_status hydro_conservation_sums(hydro_t *h, double out[4]);

hydro_status hydro_get_time(hydro_t *h, double *t);
hydro_status hydro_set_time(hydro_t *h, double t);

/* Device diagnostics since creation: out[0] capped |M| in cons->prim,
 * out[1] Hancock face fallbacks, out[2] Newton solves, out[3] Newton
 * iterations, out[4] Newton solves that hit the iteration cap, out[5] FP64
 * cons->prim redos (HYDRO_MIXED).  Counting is on only after
 * hydro_enable_counters(h, 1) (it costs atomics). */
hydro_status hydro_enable_counters(hydro_t *h, int on);
hydro_status hydro_counters(hydro_t *h, long long out[6]);

/* HYDRO_E_NONFINITE if any state value is NaN or Inf, else HYDRO_OK. */
hydro_status hydro_check_finite(hydro_t *h);
/* The handle's status after the steps so far: HYDRO_E_NONFINITE (NaN or Inf
 * in the state), else HYDRO_E_NEWTON (HYDRO_FLAG_NEWTON set), else
 * HYDRO_E_UNPHYSICAL (HYDRO_FLAG_UNPHYSICAL set), else HYDRO_OK.  flags (may
 * be NULL) receives the raw HYDRO_FLAG_* bits.  Synchronises the stream;
 * hydro_step itself does not wait to read them. */
hydro_status hydro_check_status(hydro_t *h, unsigned *flags);

/* The same four FP64 sums for callers that cannot allocate device memory
 * (the paper has no counterpart; this is an interface for such callers).
 * U is the caller's device array [4][nz][ny][nx] (double for HYDRO_FP64,
 * float otherwise); out is a host array of 4 doubles, written before the
 * call returns (the call synchronises `stream`, a cudaStream_t or NULL).
 * The call allocates nothing: its scratch is a 131,104-byte array built into
 * the library and resident on every GPU that loads it until the process
 * exits.  Grids above 268,435,456 cells are rejected with HYDRO_E_INVALID.
 * Cell sizes follow hydro_create: on an axis of one cell a size <= 0 counts
 * as 1; on any other axis a size that is not > 0 is HYDRO_E_INVALID.
 * The call enqueues its kernels and the copy of the four sums on `stream`
 * and waits for that stream before returning.
 * The first call on each device looks up that array's device address (with
 * that device current), so make the first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller. */
hydro_status hydro_conservation_sums_noalloc(const void *U, int prec, int nx, int ny, int nz,
                                             double dx, double dy, double dz, double out[4],
                                             void *stream);

/* ---------------------------------------------------------------- batch of events */

/* nevents independent grids (each may differ in size; all share precision,
 * scheme, EOS, limiter and stages, taken from grids[0]; HYDRO_E_INVALID when
 * their unsplit flags differ).  State of all events lives in one device
 * allocation. */
hydro_status hydro_batch_create(const hydro_grid_t *grids, int nevents, const hydro_eos_t *eos,
                                int limiter, int stages, hydro_batch_t **out);
void hydro_batch_destroy(hydro_batch_t *b);
hydro_status hydro_batch_set_stream(hydro_batch_t *b, void *stream);
/* spots: host array [nevents][nspots][7]; as hydro_init_hotspots per event. */
hydro_status hydro_batch_init_hotspots(hydro_batch_t *b, const double *spots, int nspots,
                                       double sigma, double e_bg);
hydro_status hydro_batch_set_primitives(hydro_batch_t *b, int event, const void *e,
                                        const void *vx, const void *vy, const void *vz,
                                        int on_device);
/* Charged batches: one event's state from (e, v, n). */
hydro_status hydro_batch_set_primitives_charged(hydro_batch_t *b, int event, const void *e,
                                                const void *vx, const void *vy, const void *vz,
                                                const void *n, int on_device);
/* Charged batches: out host [nevents], the FP64 sum of R dV per event. */
hydro_status hydro_batch_charge_sums(hydro_batch_t *b, double *out);
/* jets: host array [nevents][8]. */
hydro_status hydro_batch_set_jets(hydro_batch_t *b, const double *jets);
/* Advance every event nsteps steps, each with its own CFL dt.  One launch per
 * sweep covers all events; use_graph = 1 captures one step in a CUDA graph
 * on first use and replays it. */
hydro_status hydro_batch_step(hydro_batch_t *b, int nsteps, int use_graph);
/* Set / read one event's conserved state U[nq][nz][ny][nx] (setting clears its status bits). */
hydro_status hydro_batch_set_conserved(hydro_batch_t *b, int event, const void *U, int on_device);
hydro_status hydro_batch_get_conserved(hydro_batch_t *b, int event, void *U, int on_device);
hydro_status hydro_batch_get_primitives(hydro_batch_t *b, int event, void *e, void *vx,
                                        void *vy, void *vz, int on_device);
/* times: host [nevents]. */
hydro_status hydro_batch_times(hydro_batch_t *b, double *times);
/* out: host [nevents][4], FP64 sums as hydro_conservation_sums. */
hydro_status hydro_batch_conservation_sums(hydro_batch_t *b, double *out);
/* status: host [nevents]; per event the code hydro_check_status gives: 0 ok,
 * else HYDRO_E_NONFINITE, HYDRO_E_NEWTON or HYDRO_E_UNPHYSICAL. */
hydro_status hydro_batch_event_status(hydro_batch_t *b, int *status);
/* The same codes and the raw HYDRO_FLAG_* bits per event (host [nevents] each). */
hydro_status hydro_batch_event_flags(hydro_batch_t *b, int *status, unsigned *flags);
hydro_status hydro_batch_enable_counters(hydro_batch_t *b, int on);
hydro_status hydro_batch_counters(hydro_batch_t *b, long long out[6]);

/* Kernel timing: with on = 1, hydro_step records CUDA events around every
 * sweep launch and around the per-step rate/dt/jet kernels (steps then run
 * as individual launches, not as a CUDA graph).  hydro_get_kernel_timing
 * returns the summed device time (ms) and launch counts since the last call
 * (and resets them): out_ms[0] sweeps, out_ms[1] other kernels; counts likewise. */
hydro_status hydro_set_kernel_timing(hydro_t *h, int on);
hydro_status hydro_get_kernel_timing(hydro_t *h, double out_ms[2], long long counts[2]);
hydro_status hydro_batch_set_kernel_timing(hydro_batch_t *b, int on);
hydro_status hydro_batch_get_kernel_timing(hydro_batch_t *b, double out_ms[2], long long counts[2]);

/* ---------------------------------------------------------------- launch tuning */

/* Launch shape of a sweep: threads per block and pencil segments (each pencil
 * is split into segments marched by separate threads, with a redundant halo).
 * The autotuner times candidates on first use; a fixed shape can be forced.
 * threads = 0 returns to autotuning. */
hydro_status hydro_force_launch(hydro_t *h, int axis, int threads, int segments);
hydro_status hydro_get_launch(hydro_t *h, int axis, int *threads, int *segments);

/* ---------------------------------------------------------------- Newton seed MLP */

/* Parameter count of the seed network: W1[32][2] b1[32] W2[32][32] b2[32]
 * W3[32] b3 mu0 s0 mu1 s1 (inputs standardised as ((ln E - mu0)/s0,
 * (x - mu1)/s1), x = |M|/E, tanh hidden layers, output
 * v0 = vc + (x - vc) sigmoid(z) with vc = 3x/(2 + sqrt(4 - 3x^2)) the p = e/3
 * root; for 0 <= p <= e/3 the root lies in [vc, x]). */
int hydro_mlp_nparam(void);

/* Forward on the device: X [n][2] = (ln E, |M|/E) float, out [n] float seed
 * velocities (n = 0: nothing to do, HYDRO_OK).  BF16 weights and layer-2 inputs, FP32 accumulation on the
 * tensor cores (mma.sync m16n8k16).  All pointers device memory. */
hydro_status hydro_mlp_forward(const float *params, const float *X, int n, float *out,
                               void *stream);
/* The first-layer activations of that forward, H1 [n][32] float (device):
 * tanh of layer 1 rounded to BF16, exactly the values fed to the tensor
 * cores, so that a check can separate layer 1 from layers 2 and 3. */
hydro_status hydro_mlp_hidden(const float *params, const float *X, int n, float *H1,
                              void *stream);
/* Mean squared error loss and its gradient with respect to the FP32 master
 * parameters (bf16 rounding passed straight through).  Device pointers;
 * grad [nparam] float, loss [1] float. */
hydro_status hydro_mlp_loss_grad(const float *params, const float *X, const float *Y, int n,
                                 float *grad, float *loss, void *stream);
/* Adam training on the device: params (device, [nparam], updated in place),
 * X [n][2], Y [n]; minibatches of `batch` (reshuffled every epoch with `seed`),
 * `epochs` passes, learning rate lr decayed along a half cosine to 0.
 * loss_hist (device, [epochs]) receives the mean loss of each epoch. */
hydro_status hydro_mlp_train(float *params, const float *X, const float *Y, int n, int batch,
                             int epochs, float lr, unsigned long long seed, float *loss_hist,
                             void *stream);

/* The range of the MLP seed for the handle's tabulated EOS: states with
 * E > *emin are seeded by the network, the others by the closed-form p = e/3
 * root (below it the table departs from p = e/3 by less than 1e-4, and E >= e). */
hydro_status hydro_mlp_seed_emin(hydro_t *h, double *emin);
/* Tabulated-EOS cons->prim on an array of states with the handle's EOS:
 * U [4][n] (handle dtype), seed kind; outputs |v| [n] (handle dtype) and the
 * Newton iteration count per state (int [n]).  Device pointers; n = 0 is a
 * no-op. */
hydro_status hydro_c2p_newton(hydro_t *h, const void *U, int n, int seed, void *vmag,
                              int *iters);
/* A check of the tabulated-EOS sweeps' paired Newton solve (Sec. 2.6 with the
 * table of reading R11): two states' solves share one loop there and must
 * give what two single solves give.  U [4][n] (handle dtype, device), n even:
 * state i is paired with state i + n/2.  Outputs (device): vmag and p
 * [2][n] (handle dtype) and iters [2][n] (int) -- row 0 from single solves,
 * row 1 from the paired solve, with the handle's EOS, Newton iteration cap and
 * tolerance; E <= 0 gives zeros.  seed: HYDRO_SEED_ZERO or
 * HYDRO_SEED_CONFORMAL; rcp != 0 takes 1/W and 1/f' as reciprocals (the
 * FP32 sweeps' form), 0 divides.  n = 0 is a no-op; an odd n, a missing
 * pointer or a handle without a table EOS is HYDRO_E_INVALID. */
hydro_status hydro_c2p_newton_pairs(hydro_t *h, const void *U, int n, int seed, int rcp,
                                    void *vmag, void *p, int *iters);

#ifdef __cplusplus
}
#endif
#endif /* HYDRO_H */
