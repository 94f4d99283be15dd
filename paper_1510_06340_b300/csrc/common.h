// common.h -- constants and plain structs shared by the host code and the
// kernels of libhydro (no CUDA types).
#pragma once

namespace hy {

enum { LIM_NONE = 0, LIM_MINMOD = 1, LIM_MC = 2, LIM_SUPERBEE = 3, LIM_VANLEER = 4,
       LIM_VANALBADA = 5 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1 };
enum { EOS_CONFORMAL = 0, EOS_TABLE = 1 };
// kernel specialisation only (never stored in Scheme::eos_kind): the tabulated
// EOS with the MLP Newton seed, whose warp-wide forward pass needs registers
// the plain Newton kernels should not carry
enum { EOS_TABLE_MLP = 2 };
enum { SEED_ZERO = 0, SEED_CONFORMAL = 1, SEED_MLP = 2 };
enum { CNT_CAPPED = 0, CNT_FACE_FALLBACK = 1, CNT_NEWTON_CALLS = 2, CNT_NEWTON_ITERS = 3,
       CNT_NEWTON_FAIL = 4, CNT_F64_REDO = 5, NCOUNTERS = 6 };

// elements per row and field of the staged x sweep's shared-memory rings
// (input ring 16 + 1, output ring 8 + 1): a warp holds 32 rows of them
constexpr int XSTAGE_STEPS_PER_ROW = 26;
constexpr int NEWTON_MAX_IT = 50;   // default iteration cap of the Newton cons->prim solve
// per-event status bits set on the device (sticky until the event's state is set again)
enum { FLAG_NEWTON = 1,         // a Newton cons->prim solve hit its iteration cap
       FLAG_UNPHYSICAL = 2 };   // |M| >= (1 - delta) E met and capped, or a face fell back (R9)
constexpr double DELTA_F64 = 1e-12;   // admissibility margin |M| < (1 - delta) E
constexpr double DELTA_F32 = 1e-6;

// Newton seed MLP: W1[32][2] b1[32] W2[32][32] b2[32] W3[32] b3 mu0 s0 mu1 s1
constexpr int MLP_H = 32;
constexpr int MLP_NPARAM = MLP_H * 2 + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1 + 4;
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + 2 * MLP_H;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_H;
constexpr int MLP_OFF_NORM = MLP_OFF_B3 + 1;

// Per-event geometry, resident on the device.
struct EventGeo {
    long long off;       // element offset of field 0 of this event in the state buffer
    long long cells;     // nx * ny * nz; field f starts at off + f * cells
    int n[3];
    int bc[3];
    int seg[3];          // pencil segments per axis (launch shape)
    int segL[3];         // nominal segment length per axis
    double h[3];
    double lo[3];        // lower corner
    double inv_h[3];     // 1 / h, computed on the host
    float inv_hf[3];
    float pad_f;
    double jet[8];
    int jet_on;
    int pad;
};

// Per-event time keeping, resident on the device.
struct EventClock {
    double t;            // time reached
    double t_step;       // time at the start of the current step
    double dt;           // current step
    double t_end;        // > 0: stop here
    unsigned long long rate_bits;   // max over cells of speed/dx (double bits, >= 0)
    int status;
    int pad;
};

// Per-event layout of the scratch of the unsplit scheme: evolved faces on the
// box grown by one cell along each active axis.
struct UnsplitGeo {
    long long fo;        // element offset of the event's faces: face (d, side, q) of
                         // grown cell gi at fo + ((2 d + side) 4 + q) gcells + gi
    long long gcells;    // cells of the grown box
    int g[3];            // 1 on active axes, else 0
    int m[3];            // grown box: n + 2 g
};

// Tiles of the unsplit scheme's flux-and-update kernel: at most US_TX x US_TY x
// US_TZ cells (n_d on an axis with fewer); one work item per tile
constexpr int US_TX = 32, US_TY = 8, US_TZ = 4;

// A block's share of a launch: `count` consecutive units of one event
// starting at `first` (pencil-segment tasks for sweeps, cells otherwise).
struct WorkItem {
    int event;
    int count;
    long long first;
};

// Scheme constants of one launch (uniform over its threads).
// Per-run constants of the scheme in one precision, derived once on the host
// so that the sweeps read them as kernel-parameter operands
template <class R>
struct SchemeConsts {
    R alpha;   // FORCE coefficient
    R delta;   // admissibility margin (R9)
    R omd;     // 1 - delta
    R capf;    // (1 - delta)^2
    R cs2;     // conformal c^2
    R cs;      // c
    R k1;      // 1 - c^2
    R hapc;    // (1 + c^2) / 2
    R hapc2;   // ((1 + c^2) / 2)^2
    R lne_min, inv_h, e_max;   // tabulated EOS: first node, 1 / node spacing, last e
    R l2_scale, l2_off;        // u = log2(e) l2_scale + l2_off: ln 2 / h and -ln e_0 / h
    R emin;    // vacuum threshold: E <= emin is vacuum (2^-500 FP64, 2^-60 FP32),
               // where E^2 is still a normal number
    R wmin;    // (1 + c^2)/2 emin: W = E + p at or below it means E <= emin
    R mlp_emin;   // tabulated EOS with the MLP seed: below this E (>= e) the table is
                  // p = e/3 to within 1e-4, and the closed-form p = e/3 root seeds Newton
};

struct Scheme {
    int limiter, stages, hancock;
    double alpha;
    double delta;            // admissibility margin of this precision
    int eos_kind;            // EOS_CONFORMAL / EOS_TABLE
    double cs2;
    int tab_n;
    double lne_min, lne_max, inv_h, e_max;
    // node i of the table, packed for one fetch per lookup:
    // (p_i, p_{i+1} - p_i, c2_i, c2_{i+1} - c2_i), differences in the table's
    // precision (zero at the last node)
    const double *tab64;          // [n][4]
    const float *tab32;           // [n][4]
    int seed;
    double tol;
    const void *mlp_w;            // bf16 W1 [32][2], W2 [32][32], W3 [32]
    const float *mlp_f;           // fp32 copy of the full parameter vector
    unsigned long long *counters; // [NCOUNTERS] or null
    unsigned *event_flags;        // [nevents] FLAG_* words, or null
    int newton_max_it;            // iteration cap of the Newton solve
    SchemeConsts<double> c64;     // FP64 values, delta of FP64
    SchemeConsts<float> c32;      // FP32 values computed in FP32, delta of FP32
};

}  // namespace hy
