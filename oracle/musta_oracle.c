/*
 * musta_oracle.c -- plain, slow, FP64 CPU oracle for the MUSTA-FORCE update of
 * ideal relativistic hydrodynamics (Porter-Sobieraj et al., "A MUSTA-FORCE
 * algorithm for solving partial differential equations of relativistic
 * hydrodynamics").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path; it is written
 * from the paper's equations and the readings listed below, in the paper's
 * order, with no blocking, fusion or reordering.
 *
 * State per cell: U = (E, Mx, My, Mz) = T^{00}, T^{0i}, and with charge = 1
 * the conserved charge R = n gamma as a fifth field (Sec. 2.1, Eq. 1, 3, 4).
 * Arrays are field-major [nq][nz][ny][nx], x fastest, nq = 4 or 5.
 *
 * Readings of points the paper leaves open (each is also a named item in the
 * design notes):
 *  R1  Lax-Wendroff flux (Eq. 10) uses (F_R - F_L) inside the argument, the
 *      textbook FORCE form; the printed (U_R - U_L) is read as a typo.
 *  R2  alpha = 1 for dimension-split sweeps (Eq. 10-11; "alpha = 3" refers to
 *      the unsplit 3-D predictor of Eq. 13).  alpha is a parameter.
 *  R3  MUSTA start states at interface i+1/2 are the Hancock-evolved right
 *      face of cell i and left face of cell i+1 (Sec. 2.4, MUSCL-Hancock
 *      step 3).
 *  R4  k MUSTA stages = k FORCE evaluations and k-1 local Riemann predictor
 *      updates (Eq. 8) with the global lambda = dt/dx.
 *  R5  Limited slope written division-free: with a = U_i - U_{i-1},
 *      b = U_{i+1} - U_i, slope = a * xi(b/a) (Eq. 15-17); by the symmetry
 *      of Eq. 22 both faces use the same slope.  van Albada is the clipped
 *      form (zero for r <= 0).  MC (not in the paper) is
 *      xi = max(0, min(2r, (1+r)/2, 2)).
 *  R6  Inside an RK stage of a sweep of length dt_s, lambda = dt_s/dx_d is
 *      used by Hancock, MUSTA and the divergence.
 *  R7  Dimension splitting is Strang: X(dt/2) Y(dt/2) Z(dt) Y(dt/2) X(dt/2)
 *      over the axes with more than one cell; one CFL dt per full step.
 *  R8  CFL signal speed: ideal-fluid characteristic speeds
 *      lam = [v_d(1-c2) +- c sqrt((1-v^2)(1-v_d^2-(v^2-v_d^2)c2))]/(1-v^2 c2),
 *      dt = cfl / max_{cells,d} (max|lam|/dx_d), clipped to t_end.
 *  R9  Admissibility: cons->prim caps |M| at (1-delta)E; a cell whose two
 *      Hancock face states are not both admissible (E > 0 and
 *      |M| < (1-delta)E) uses its cell average on both faces.
 *  R10 p = c2*e cons->prim solves Eq. 23 exactly: W = E + p is the positive
 *      root of W^2 - (1+c2)E W + c2 M^2 = 0.
 *  R11 Tabulated EOS: nodes uniform in ln e, p and c_s^2 interpolated
 *      linearly in ln e; p = e/3 below the table, linear extrapolation with
 *      the last c_s^2 above it.  Eq. 23 is solved by safeguarded Newton on
 *      f(v) = v - |M|/(E + p(E - |M| v)) in the bracket [0, |M|/E].
 *  R12 Jet source: S^{0mu} = dEdx (1, n) g(x - x0 - n t), g a normalised
 *      3-D Gaussian; added once per step as U += dt S(t_n) before the sweeps.
 *  R16 Unsplit scheme (unsplit = 1; the paper's multi-D MUSCL-Hancock of
 *      Eq. 13 with FORCE alpha, 3 in 3-D): (a) each flux term of the half
 *      step uses the faces of its own axis, h = 1/2 sum_d dt/dx_d
 *      (F_d(U^L_d) - F_d(U^R_d)), and every face of the cell is advanced by
 *      the same h; (b) R9's fallback: if any evolved face is not admissible,
 *      all faces of the cell are its cell average; (c) dt = cfl / max over
 *      cells of sum_d max|lam_d| / dx_d over the axes with more than one cell;
 *      (d) the RK stages of Eq. 6-7 act on the whole field, with
 *      dt L(U) = - sum_d dt/dx_d (F_d,i+1/2 - F_d,i-1/2).
 *  R17 Ellipsoidal flow (Sec. 3.2): v_i = a_i x_i / t (the printed order
 *      a_1, a_3, a_2 of the velocity is read as a typo; tau pairs a_i with x_i).
 *  R19 Conserved charge (charge = 1): R = n gamma is carried as a fifth
 *      conserved field with flux R v_d (Eq. 3).  The EOS here is p(e) (the
 *      paper gives no p(e, n)), so R is transported by the energy-momentum
 *      velocity and feeds nothing back; n = R / gamma on readout.  Slopes,
 *      Hancock, MUSTA-FORCE and RK act on it like on the other fields; the
 *      admissibility rule (R9) looks at E and M only.  Not built for the
 *      unsplit scheme.
 *  R18 Vacuum threshold: a cell with E <= 2^-500 is vacuum (v = p = 0), so that
 *      E^2 and M^2 in the cons->prim formulas stay normal numbers; below it the
 *      closed form of R10 loses all digits (E^2 underflows).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef OR_OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- config */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double x0, y0, z0;         /* lower corner of the box */
    int bc[3];                 /* 0 periodic, 1 outflow */
    int limiter;               /* 0 none 1 minmod 2 mc 3 superbee 4 vanleer 5 vanalbada */
    int stages;                /* MUSTA stages k >= 1 */
    int rk_order;              /* 1 (forward Euler), 2 or 3 */
    int hancock;               /* 1: MUSCL-Hancock half step on; 0: plain MUSCL faces */
    double alpha;              /* FORCE alpha */
    double cfl;
    double fixed_dt;           /* > 0 overrides the CFL step */
    double delta;              /* admissibility margin (R9) */
    int eos_kind;              /* 0: p = cs2 e ; 1: table */
    double cs2;
    int tab_n;
    double lne_min, lne_max;
    const double *cs2_tab, *p_tab;
    int seed_kind;             /* Newton seed: 0 zero, 1 conformal closed form, 2 MLP */
    const double *mlp;         /* MLP parameters (layout in or_mlp_forward) */
    int mlp_quantize;          /* 1: bf16 weights and layer-2 inputs */
    double newton_tol;         /* |dv| tolerance */
    int jet_on;
    double jet[8];             /* x0,y0,z0, nx,ny,nz, dEdx, sigma */
    int unsplit;               /* 1: unsplit multi-D scheme (R16) instead of Strang sweeps */
    int charge;                /* 1: carry the conserved charge R as a fifth field (R19) */
} or_config;

#define OR_NQ 5                /* room for the fields of one cell, with the charge */
static int nq_of(const or_config *c) { return c->charge ? 5 : 4; }

/* diagnostics counters (reset by or_reset_counters); the OpenMP timing build
   (OR_OPENMP) runs pencils on several threads and keeps no counts */
static long g_newton_calls = 0, g_newton_iters = 0, g_newton_fail = 0;
static long g_capped = 0, g_face_fallback = 0;
#ifdef OR_OPENMP
#define OR_TALLY(counter, n) ((void)0)
#else
#define OR_TALLY(counter, n) ((counter) += (n))
#endif

/* threads a parallel region of this build uses (1 without OpenMP) */
int or_threads(void) {
#ifdef OR_OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_reset_counters(void) {
    g_newton_calls = g_newton_iters = g_newton_fail = 0;
    g_capped = g_face_fallback = 0;
}
void or_get_counters(long out[5]) {
    out[0] = g_newton_calls; out[1] = g_newton_iters; out[2] = g_newton_fail;
    out[3] = g_capped; out[4] = g_face_fallback;
}

/* ------------------------------------------------------- slope limiters */
/* Sec. 2.5, Eq. 15-21 (R5): returns the limited slope a*xi(b/a). */
double or_limiter(int kind, double a, double b) {
    double ab = a * b;
    double sa = (a > 0.0) ? 1.0 : -1.0;
    switch (kind) {
    case 0: /* no limiter: central slope, Eq. 14 */
        return 0.5 * (a + b);
    case 1: /* Minbee, Eq. 18 */
        if (ab <= 0.0) return 0.0;
        return sa * fmin(fabs(a), fabs(b));
    case 2: /* monotonized central (van Leer 1977) */
        if (ab <= 0.0) return 0.0;
        return sa * fmin(fmin(2.0 * fabs(a), 2.0 * fabs(b)), 0.5 * fabs(a + b));
    case 3: /* Superbee, Eq. 19 */
        if (ab <= 0.0) return 0.0;
        return sa * fmax(fmin(2.0 * fabs(a), fabs(b)), fmin(fabs(a), 2.0 * fabs(b)));
    case 4: /* van Leer, Eq. 21 */
        if (ab <= 0.0) return 0.0;
        return 2.0 * ab / (a + b);
    case 5: /* van Albada, Eq. 20 (clipped, R5) */
        if (ab <= 0.0) return 0.0;
        return ab * (a + b) / (a * a + b * b);
    }
    return 0.0;
}

/* ------------------------------------------------------------------ EOS */
/* R11: pressure and squared sound speed from the table. */
void or_eos_table(const or_config *c, double e, double *p, double *c2) {
    int n = c->tab_n;
    double lne = log(e);
    if (!(e > 0.0) || lne < c->lne_min) {
        *p = e / 3.0; *c2 = 1.0 / 3.0;
        if (!(e > 0.0)) *p = 0.0;
        return;
    }
    double h = (c->lne_max - c->lne_min) / (double)(n - 1);
    double u = (lne - c->lne_min) / h;
    if (u >= (double)(n - 1)) {
        double emax = exp(c->lne_max);
        *p = c->p_tab[n - 1] + c->cs2_tab[n - 1] * (e - emax);
        *c2 = c->cs2_tab[n - 1];
        return;
    }
    int i = (int)floor(u);
    double f = u - (double)i;
    *p = c->p_tab[i] + f * (c->p_tab[i + 1] - c->p_tab[i]);
    *c2 = c->cs2_tab[i] + f * (c->cs2_tab[i + 1] - c->cs2_tab[i]);
}

double or_eos_p(const or_config *c, double e) {
    if (c->eos_kind == 0) return c->cs2 * e;
    double p, c2; or_eos_table(c, e, &p, &c2); return p;
}
double or_eos_cs2(const or_config *c, double e) {
    if (c->eos_kind == 0) return c->cs2;
    double p, c2; or_eos_table(c, e, &p, &c2); return c2;
}

/* ------------------------------------------------------------------ MLP */
/*
 * Newton seed network (not in the paper): inputs (ln E, x = |M|/E)
 * standardised, two tanh hidden layers of 32, output r = sigmoid(z), seed
 * v0 = vc + (x - vc) r with vc = 3x / (2 + sqrt(4 - 3x^2)) the root for
 * p = e/3.  Any EOS with 0 <= p <= e/3 has its root in [vc, x].
 * Parameter layout: W1[32][2] b1[32] W2[32][32] b2[32] W3[32] b3 mu0 s0 mu1 s1.
 */
#define MLP_H 32
#define MLP_NPARAM (MLP_H * 2 + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1 + 4)

int or_mlp_nparam(void) { return MLP_NPARAM; }

/* round to the nearest bfloat16 (ties to even), via the float32 value */
double or_round_bf16(double x) {
    float f = (float)x;
    unsigned int u; memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;
    unsigned int lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* layer 1: standardised inputs and h1 = tanh(W1 in + b1), rounded to bf16 when q */
static void mlp_layer1(const double *P, int q, double lnE, double x, double *h1, double *in0_out,
                       double *in1_out) {
    const double *W1 = P, *b1 = W1 + 2 * MLP_H, *nrm = P + MLP_NPARAM - 4;
    double in0 = (lnE - nrm[0]) / nrm[1];
    double in1 = (x - nrm[2]) / nrm[3];
    for (int j = 0; j < MLP_H; j++) {
        double w0 = q ? or_round_bf16(W1[2 * j]) : W1[2 * j];
        double w1 = q ? or_round_bf16(W1[2 * j + 1]) : W1[2 * j + 1];
        h1[j] = tanh(w0 * in0 + w1 * in1 + b1[j]);
        if (q) h1[j] = or_round_bf16(h1[j]);
    }
    *in0_out = in0;
    *in1_out = in1;
}

/* layers 2 and 3 from h1: h2 = tanh(W2 h1 + b2), z = W3 h2 + b3,
   v0 = vc + (x - vc) sigmoid(z); h2 and r = sigmoid(z) are returned too */
static double mlp_layers23(const double *P, int q, double x, const double *h1, double *h2,
                           double *r_out) {
    const double *W2 = P + 3 * MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const double *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    for (int j = 0; j < MLP_H; j++) {
        double s = b2[j];
        for (int k = 0; k < MLP_H; k++) {
            double w = q ? or_round_bf16(W2[j * MLP_H + k]) : W2[j * MLP_H + k];
            s += w * h1[k];
        }
        h2[j] = tanh(s);
    }
    double z = b3[0];
    for (int k = 0; k < MLP_H; k++) {
        double w = q ? or_round_bf16(W3[k]) : W3[k];
        z += w * h2[k];
    }
    double r = 1.0 / (1.0 + exp(-z));
    double vc = 3.0 * x / (2.0 + sqrt(4.0 - 3.0 * x * x));
    *r_out = r;
    return vc + (x - vc) * r;
}

/* forward for one sample; cache (optional) receives h1[32], h2[32], r, in0, in1 */
static double mlp_forward1(const double *P, int q, double lnE, double x, double *cache) {
    double h1[MLP_H], h2[MLP_H], in0, in1, r;
    mlp_layer1(P, q, lnE, x, h1, &in0, &in1);
    double v0 = mlp_layers23(P, q, x, h1, h2, &r);
    if (cache) {
        memcpy(cache, h1, sizeof h1);
        memcpy(cache + MLP_H, h2, sizeof h2);
        cache[2 * MLP_H] = r;
        cache[2 * MLP_H + 1] = in0;
        cache[2 * MLP_H + 2] = in1;
    }
    return v0;
}

/* first-layer activations H1[n][32] (bf16-rounded when q) */
void or_mlp_hidden(const double *P, int q, int n, const double *X, double *H1) {
    for (int i = 0; i < n; i++) {
        double in0, in1;
        mlp_layer1(P, q, X[2 * i], X[2 * i + 1], H1 + (long)i * MLP_H, &in0, &in1);
    }
}

/* layers 2 and 3 fed with given first-layer activations H1[n][32] */
void or_mlp_forward_h1(const double *P, int q, int n, const double *X, const double *H1,
                       double *out) {
    for (int i = 0; i < n; i++) {
        double h2[MLP_H], r;
        out[i] = mlp_layers23(P, q, X[2 * i + 1], H1 + (long)i * MLP_H, h2, &r);
    }
}

/* batch forward: X[n][2] = (ln E, |M|/E), out[n] = seed velocity */
void or_mlp_forward(const double *P, int q, int n, const double *X, double *out) {
    for (int i = 0; i < n; i++) out[i] = mlp_forward1(P, q, X[2 * i], X[2 * i + 1], NULL);
}

/*
 * loss = mean_i (v0_i - Y_i)^2 and its gradient with respect to the
 * parameters (normalisation entries get zero gradient).  With q = 1 the
 * rounding to bf16 is passed straight through (its derivative taken as 1).
 */
double or_mlp_loss_grad(const double *P, int q, int n, const double *X, const double *Y,
                        double *G) {
    const double *W2 = P + 3 * MLP_H, *W3 = W2 + MLP_H * MLP_H + MLP_H;
    double *gW1 = G, *gb1 = gW1 + 2 * MLP_H, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
    double *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_H;
    memset(G, 0, sizeof(double) * MLP_NPARAM);
    double loss = 0.0;
    double cache[2 * MLP_H + 3];
    for (int i = 0; i < n; i++) {
        double x = X[2 * i + 1];
        double v0 = mlp_forward1(P, q, X[2 * i], x, cache);
        const double *h1 = cache, *h2 = cache + MLP_H;
        double r = cache[2 * MLP_H], in0 = cache[2 * MLP_H + 1], in1 = cache[2 * MLP_H + 2];
        double d = v0 - Y[i];
        loss += d * d;
        double dv = 2.0 * d / (double)n;
        double vc = 3.0 * x / (2.0 + sqrt(4.0 - 3.0 * x * x));
        double dz = dv * (x - vc) * r * (1.0 - r);
        gb3[0] += dz;
        double da2[MLP_H];
        for (int k = 0; k < MLP_H; k++) {
            double w3 = q ? or_round_bf16(W3[k]) : W3[k];
            gW3[k] += dz * h2[k];
            da2[k] = dz * w3 * (1.0 - h2[k] * h2[k]);
        }
        for (int j = 0; j < MLP_H; j++) {
            gb2[j] += da2[j];
            for (int k = 0; k < MLP_H; k++) gW2[j * MLP_H + k] += da2[j] * h1[k];
        }
        for (int k = 0; k < MLP_H; k++) {
            double dh1 = 0.0;
            for (int j = 0; j < MLP_H; j++) {
                double w = q ? or_round_bf16(W2[j * MLP_H + k]) : W2[j * MLP_H + k];
                dh1 += w * da2[j];
            }
            /* tanh derivative at the unrounded activation value */
            double a1 = h1[k];
            double da1 = dh1 * (1.0 - a1 * a1);
            gb1[k] += da1;
            gW1[2 * k] += da1 * in0;
            gW1[2 * k + 1] += da1 * in1;
        }
    }
    return loss / (double)n;
}

/* ------------------------------------------------------- cons -> prim */
/*
 * Sec. 2.6, Eq. 23: from U = (E, M) find v (vector), p and e.  Returns 0 for
 * an admissible state, 1 when |M| was capped, 2 for E <= 0 (vacuum: v = p = 0),
 * 3 when the Newton solve hit its iteration cap.
 */
int or_cons2prim(const or_config *c, const double U[4], double *e_out, double v[3],
                 double *p_out, int *iters) {
    double E = U[0], Mx = U[1], My = U[2], Mz = U[3];
    double M2 = Mx * Mx + My * My + Mz * Mz;
    int status = 0;
    if (iters) *iters = 0;
    if (!(E > 0x1p-500)) {            /* vacuum (R9, R18) */
        v[0] = v[1] = v[2] = 0.0;
        *p_out = 0.0; *e_out = 0.0;
        return 2;
    }
    double cap = (1.0 - c->delta) * E;
    if (M2 > cap * cap) {               /* R9: cap |M| at (1-delta) E */
        double s = cap / sqrt(M2);
        Mx *= s; My *= s; Mz *= s;
        M2 = Mx * Mx + My * My + Mz * Mz;
        status = 1;
        OR_TALLY(g_capped, 1);
    }
    double M = sqrt(M2);
    if (c->eos_kind == 0) {
        /* R10: W = E + p is the positive root of W^2 - (1+c2) E W + c2 M^2 = 0 */
        double a = (1.0 + c->cs2) * E;
        double disc = a * a - 4.0 * c->cs2 * M2;
        if (disc < 0.0) disc = 0.0;
        double W = 0.5 * (a + sqrt(disc));
        v[0] = Mx / W; v[1] = My / W; v[2] = Mz / W;
        *p_out = W - E;
        *e_out = E - M2 / W;
        return status;
    }
    /* R11: safeguarded Newton on f(v) = v - M/(E + p(E - M v)), v in [0, M/E] */
    OR_TALLY(g_newton_calls, 1);
    double lo = 0.0, hi = M / E;
    double vv;
    if (c->seed_kind == 1) {
        double a = (4.0 / 3.0) * E, disc = a * a - (4.0 / 3.0) * M2;
        if (disc < 0.0) disc = 0.0;
        vv = M / (0.5 * (a + sqrt(disc)));
    } else if (c->seed_kind == 2 && c->mlp) {
        vv = mlp_forward1(c->mlp, c->mlp_quantize, log(E), M / E, NULL);
    } else {
        vv = 0.0;
    }
    if (vv < lo) vv = lo;
    if (vv > hi) vv = hi;
    double p = 0.0, c2 = 0.0;
    int it, conv = 0;
    if (M == 0.0) {
        vv = 0.0; conv = 1; it = 0;
    } else {
        for (it = 1; it <= 50; it++) {
            double e = E - M * vv;
            or_eos_table(c, e, &p, &c2);
            double W = E + p;
            double f = vv - M / W;
            if (f == 0.0) { conv = 1; break; }          /* vv is the root */
            if (f > 0.0) hi = vv; else lo = vv;
            double fp = 1.0 - c2 * M2 / (W * W);
            double vn = vv - f / fp;
            if (!(vn > lo && vn < hi)) vn = 0.5 * (lo + hi);
            double dv = vn - vv;
            vv = vn;
            if (fabs(dv) <= c->newton_tol) { conv = 1; break; }
        }
        if (it > 50) it = 50;
    }
    OR_TALLY(g_newton_iters, it);
    if (iters) *iters = it;
    if (!conv) { OR_TALLY(g_newton_fail, 1); status = 3; }
    double e = E - M * vv;
    or_eos_table(c, e, &p, &c2);
    double sc = (M > 0.0) ? vv / M : 0.0;
    v[0] = Mx * sc; v[1] = My * sc; v[2] = Mz * sc;
    *p_out = p;
    *e_out = e;
    return status;
}

/* ------------------------------------------------------- prim -> cons */
/* Sec. 2.1, Eq. 4: E = (e+p) g^2 - p, M_i = (e+p) g^2 v_i, and R = n g with
   the charge (U then holds 5 values). */
void or_prim2cons_n(const or_config *c, double e, double vx, double vy, double vz, double n,
                    double *U) {
    double p = or_eos_p(c, e);
    double v2 = vx * vx + vy * vy + vz * vz;
    double g2 = 1.0 / (1.0 - v2);
    double w = (e + p) * g2;
    U[0] = w - p;
    U[1] = w * vx;
    U[2] = w * vy;
    U[3] = w * vz;
    if (c->charge) U[4] = n / sqrt(1.0 - v2);
}
void or_prim2cons(const or_config *c, double e, double vx, double vy, double vz, double *U) {
    or_prim2cons_n(c, e, vx, vy, vz, 0.0, U);
}

/* ----------------------------------------------------------------- flux */
/* Sec. 2.1, Eq. 3: flux along axis d of U. */
void or_flux(const or_config *c, int d, const double *U, double *F) {
    double e, v[3], p;
    or_cons2prim(c, U, &e, v, &p, NULL);
    F[0] = (U[0] + p) * v[d];
    F[1] = U[1] * v[d];
    F[2] = U[2] * v[d];
    F[3] = U[3] * v[d];
    F[1 + d] += p;
    if (c->charge) F[4] = U[4] * v[d];   /* R v_d */
}

/* ---------------------------------------------------------- MUSTA-FORCE */
/* Sec. 2.4, MUSTA steps 1-5 with the FORCE flux of Eq. 9-11 (R1, R2, R4). */
void or_musta_force(const or_config *c, int d, double lam, const double *UL0,
                    const double *UR0, double *Fout) {
    double UL[OR_NQ], UR[OR_NQ], FL[OR_NQ], FR[OR_NQ], Ulw[OR_NQ], Flw[OR_NQ], Flf[OR_NQ],
        Fc[OR_NQ];
    double al = c->alpha * lam;
    int nq = nq_of(c);
    memcpy(UL, UL0, nq * sizeof(double));
    memcpy(UR, UR0, nq * sizeof(double));
    for (int l = 0; l < c->stages; l++) {
        or_flux(c, d, UL, FL);
        or_flux(c, d, UR, FR);
        for (int q = 0; q < nq; q++)
            Ulw[q] = 0.5 * (UL[q] + UR[q]) - 0.5 * al * (FR[q] - FL[q]);
        or_flux(c, d, Ulw, Flw);
        for (int q = 0; q < nq; q++)
            Flf[q] = 0.5 * (FL[q] + FR[q]) - (0.5 / al) * (UR[q] - UL[q]);
        for (int q = 0; q < nq; q++) Fc[q] = 0.5 * (Flw[q] + Flf[q]);
        if (l < c->stages - 1) {
            for (int q = 0; q < nq; q++) {
                UL[q] = UL[q] - lam * (Fc[q] - FL[q]);
                UR[q] = UR[q] - lam * (FR[q] - Fc[q]);
            }
        }
    }
    memcpy(Fout, Fc, nq * sizeof(double));
}

static int admissible(const or_config *c, const double *U) {
    double M2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
    double cap = (1.0 - c->delta) * U[0];
    return U[0] > 0.0 && M2 < cap * cap;
}

/*
 * Sec. 2.4-2.5: MUSCL slopes (Eq. 15-17), faces, Hancock half step (Eq. 13,
 * the term along the sweep axis), R9 fallback.  V holds cells -1..+1 around
 * the cell; outputs the evolved faces.
 */
void or_hancock_faces(const or_config *c, int d, double lam, const double *Vm,
                      const double *V0, const double *Vp, double *ULt, double *URt) {
    double UL[OR_NQ], UR[OR_NQ], FL[OR_NQ], FR[OR_NQ];
    int nq = nq_of(c);
    for (int q = 0; q < nq; q++) {
        double s = or_limiter(c->limiter, V0[q] - Vm[q], Vp[q] - V0[q]);
        UL[q] = V0[q] - 0.5 * s;
        UR[q] = V0[q] + 0.5 * s;
    }
    if (c->hancock) {
        or_flux(c, d, UL, FL);
        or_flux(c, d, UR, FR);
        for (int q = 0; q < nq; q++) {
            ULt[q] = UL[q] + 0.5 * lam * (FL[q] - FR[q]);
            URt[q] = UR[q] + 0.5 * lam * (FL[q] - FR[q]);
        }
    } else {
        memcpy(ULt, UL, nq * sizeof(double));
        memcpy(URt, UR, nq * sizeof(double));
    }
    if (!admissible(c, ULt) || !admissible(c, URt)) {
        memcpy(ULt, V0, nq * sizeof(double));
        memcpy(URt, V0, nq * sizeof(double));
        OR_TALLY(g_face_fallback, 1);
    }
}

/* ------------------------------------------------------------- pencils */
/* V[(N+4)][OR_NQ]: cell i at V[i+2]; fill two ghost cells on each side. */
static void fill_ghosts(double (*V)[OR_NQ], int N, int bc) {
    for (int g = 1; g <= 2; g++) {
        int lo_dst = 2 - g, hi_dst = N + 1 + g;
        int lo_src = (bc == 0) ? (N - g + 2) : 2;
        int hi_src = (bc == 0) ? (g + 1) : (N + 1);
        memcpy(V[lo_dst], V[lo_src], OR_NQ * sizeof(double));
        memcpy(V[hi_dst], V[hi_src], OR_NQ * sizeof(double));
    }
}

/* D[i] = F_{i+1/2} - F_{i-1/2} for cells 0..N-1 (the divergence, times dx) */
static void pencil_L(const or_config *c, int d, double lam, double (*V)[OR_NQ], int N,
                     double (*D)[OR_NQ], double (*ULt)[OR_NQ], double (*URt)[OR_NQ],
                     double (*F)[OR_NQ]) {
    int nq = nq_of(c);
    /* evolved faces of cells -1..N (index +1) */
    for (int i = -1; i <= N; i++)
        or_hancock_faces(c, d, lam, V[i + 1], V[i + 2], V[i + 3], ULt[i + 1], URt[i + 1]);
    /* interface fluxes F_{i+1/2} for i = -1..N-1 (index +1) */
    for (int i = -1; i < N; i++)
        or_musta_force(c, d, lam, URt[i + 1], ULt[i + 2], F[i + 1]);
    for (int i = 0; i < N; i++)
        for (int q = 0; q < nq; q++) D[i][q] = F[i + 1][q] - F[i][q];
}

/* one Runge-Kutta sweep (Sec. 2.3, Eq. 6 or 7) of every pencil along axis d;
   pencils are independent, so the OpenMP timing build splits them over threads */
void or_sweep(const or_config *c, double *U, int d, double dt) {
    int n[3] = {c->nx, c->ny, c->nz};
    double h[3] = {c->dx, c->dy, c->dz};
    int N = n[d];
    long cells = (long)c->nx * c->ny * c->nz;
    long stride = (d == 0) ? 1 : (d == 1) ? c->nx : (long)c->nx * c->ny;
    double lam = dt / h[d];
    int a_ax = (d == 0) ? 1 : 0, b_ax = (d == 2) ? 1 : 2;
    long npencils = (long)n[a_ax] * n[b_ax];
    int nq = nq_of(c);
#ifdef OR_OPENMP
#pragma omp parallel
#endif
    {
    double (*V0)[OR_NQ] = (double (*)[OR_NQ])malloc(sizeof(double[OR_NQ]) * (N + 4));
    double (*V1)[OR_NQ] = (double (*)[OR_NQ])malloc(sizeof(double[OR_NQ]) * (N + 4));
    double (*V2)[OR_NQ] = (double (*)[OR_NQ])malloc(sizeof(double[OR_NQ]) * (N + 4));
    double (*D)[OR_NQ] = (double (*)[OR_NQ])malloc(sizeof(double[OR_NQ]) * N);
    double (*ULt)[OR_NQ] = (double (*)[OR_NQ])malloc(sizeof(double[OR_NQ]) * (N + 2));
    double (*URt)[OR_NQ] = (double (*)[OR_NQ])malloc(sizeof(double[OR_NQ]) * (N + 2));
    double (*F)[OR_NQ] = (double (*)[OR_NQ])malloc(sizeof(double[OR_NQ]) * (N + 1));
#ifdef OR_OPENMP
#pragma omp for schedule(static)
#endif
    for (long pc = 0; pc < npencils; pc++) {
        int a = (int)(pc % n[a_ax]), b = (int)(pc / n[a_ax]);
        int idx[3];
        idx[d] = 0; idx[a_ax] = a; idx[b_ax] = b;
        long base = idx[0] + (long)c->nx * (idx[1] + (long)c->ny * idx[2]);
        for (int i = 0; i < N; i++)
            for (int q = 0; q < nq; q++) V0[i + 2][q] = U[q * cells + base + i * stride];
        fill_ghosts(V0, N, c->bc[d]);
        /* stage 1: U1 = U + dt L(U) */
        pencil_L(c, d, lam, V0, N, D, ULt, URt, F);
        if (c->rk_order == 1) {
            for (int i = 0; i < N; i++)
                for (int q = 0; q < nq; q++)
                    U[q * cells + base + i * stride] = V0[i + 2][q] - lam * D[i][q];
            continue;
        }
        for (int i = 0; i < N; i++)
            for (int q = 0; q < nq; q++) V1[i + 2][q] = V0[i + 2][q] - lam * D[i][q];
        fill_ghosts(V1, N, c->bc[d]);
        pencil_L(c, d, lam, V1, N, D, ULt, URt, F);
        if (c->rk_order == 3) {
            /* U2 = 3/4 U + 1/4 U1 + 1/4 dt L(U1) */
            for (int i = 0; i < N; i++)
                for (int q = 0; q < nq; q++)
                    V2[i + 2][q] = 0.75 * V0[i + 2][q] + 0.25 * (V1[i + 2][q] - lam * D[i][q]);
            fill_ghosts(V2, N, c->bc[d]);
            pencil_L(c, d, lam, V2, N, D, ULt, URt, F);
            /* U^{n+1} = 1/3 U + 2/3 U2 + 2/3 dt L(U2) */
            for (int i = 0; i < N; i++)
                for (int q = 0; q < nq; q++)
                    U[q * cells + base + i * stride] =
                        V0[i + 2][q] / 3.0 + (2.0 / 3.0) * (V2[i + 2][q] - lam * D[i][q]);
        } else {
            /* U^{n+1} = 1/2 (U + U1 + dt L(U1)) */
            for (int i = 0; i < N; i++)
                for (int q = 0; q < nq; q++)
                    U[q * cells + base + i * stride] =
                        0.5 * (V0[i + 2][q] + V1[i + 2][q] - lam * D[i][q]);
        }
    }
    free(V0); free(V1); free(V2); free(D); free(ULt); free(URt); free(F);
    }
}

/* ------------------------------------------------------------------ CFL */
/* R8: largest characteristic speed magnitude of one cell along axis d */
double or_signal_speed(const or_config *c, const double U[4], int d) {
    double e, v[3], p;
    or_cons2prim(c, U, &e, v, &p, NULL);
    double c2 = or_eos_cs2(c, e);
    double cs = sqrt(c2);
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double vd = v[d];
    double rad = (1.0 - v2) * (1.0 - vd * vd - (v2 - vd * vd) * c2);
    if (rad < 0.0) rad = 0.0;
    double den = 1.0 - v2 * c2;
    double lp = (vd * (1.0 - c2) + cs * sqrt(rad)) / den;
    double lm = (vd * (1.0 - c2) - cs * sqrt(rad)) / den;
    return fmax(fabs(lp), fabs(lm));
}

/* max over cells and active axes of speed/dx, the inverse of the CFL dt */
double or_max_rate(const or_config *c, const double *U) {
    long cells = (long)c->nx * c->ny * c->nz;
    int n[3] = {c->nx, c->ny, c->nz};
    double h[3] = {c->dx, c->dy, c->dz};
    double m = 0.0;
#ifdef OR_OPENMP
#pragma omp parallel for reduction(max : m) schedule(static)
#endif
    for (long i = 0; i < cells; i++) {
        double u[4] = {U[i], U[cells + i], U[2 * cells + i], U[3 * cells + i]};
        for (int d = 0; d < 3; d++) {
            if (n[d] <= 1) continue;
            double r = or_signal_speed(c, u, d) / h[d];
            if (r > m) m = r;
        }
    }
    return m;
}

/* ------------------------------------------------------------ jet source */
/* R12: U += dt * S(t) */
void or_jet_source(const or_config *c, double *U, double t, double dt) {
    long cells = (long)c->nx * c->ny * c->nz;
    const double *j = c->jet;
    double sig = j[7];
    double norm = 1.0 / (pow(2.0 * M_PI, 1.5) * sig * sig * sig);
    double cx = j[0] + j[3] * t, cy = j[1] + j[4] * t, cz = j[2] + j[5] * t;
    for (int z = 0; z < c->nz; z++)
        for (int y = 0; y < c->ny; y++)
            for (int x = 0; x < c->nx; x++) {
                double px = c->x0 + (x + 0.5) * c->dx - cx;
                double py = c->y0 + (y + 0.5) * c->dy - cy;
                double pz = c->z0 + (z + 0.5) * c->dz - cz;
                double g = norm * exp(-(px * px + py * py + pz * pz) / (2.0 * sig * sig));
                long i = x + (long)c->nx * (y + (long)c->ny * z);
                double s = dt * j[6] * g;
                U[i] += s;
                U[cells + i] += s * j[3];
                U[2 * cells + i] += s * j[4];
                U[3 * cells + i] += s * j[5];
            }
}


/* -------------------------------------------------------- unsplit (R16) */
/* cell index of the logical position (i, j, k), ghosts mapped by the BCs */
static long grid_index(const or_config *c, int i, int j, int k) {
    int n[3] = {c->nx, c->ny, c->nz};
    int x[3] = {i, j, k};
    for (int d = 0; d < 3; d++) {
        if (c->bc[d] == 0) x[d] = ((x[d] % n[d]) + n[d]) % n[d];
        else x[d] = x[d] < 0 ? 0 : (x[d] >= n[d] ? n[d] - 1 : x[d]);
    }
    return x[0] + (long)c->nx * (x[1] + (long)c->ny * x[2]);
}

static void grid_load(const or_config *c, const double *U, int i, int j, int k, double *u) {
    long cells = (long)c->nx * c->ny * c->nz;
    long g = grid_index(c, i, j, k);
    for (int q = 0; q < 4; q++) u[q] = U[q * cells + g];
}

/*
 * dt L(U) of the unsplit scheme for every cell (R16): D[q][cell] receives
 * sum_d dt/dx_d (F_d,i+1/2 - F_d,i-1/2).  Faces are evolved for the cells of
 * the box grown by one cell along every active axis; fluxes are taken at the
 * interfaces of the real cells.
 */
static void unsplit_L(const or_config *c, const double *U, double dt, double *D) {
    int n[3] = {c->nx, c->ny, c->nz};
    double h[3] = {c->dx, c->dy, c->dz};
    int act[3], g[3];
    for (int d = 0; d < 3; d++) { act[d] = n[d] > 1; g[d] = act[d] ? 1 : 0; }
    int m[3] = {n[0] + 2 * g[0], n[1] + 2 * g[1], n[2] + 2 * g[2]};
    long mcells = (long)m[0] * m[1] * m[2];
    long cells = (long)n[0] * n[1] * n[2];
    /* evolved faces: FL[d][cell of the grown box][q], FR likewise */
    double *FLf = (double *)malloc(sizeof(double) * 3 * mcells * 4);
    double *FRf = (double *)malloc(sizeof(double) * 3 * mcells * 4);
    for (int k = -g[2]; k < n[2] + g[2]; k++)
        for (int j = -g[1]; j < n[1] + g[1]; j++)
            for (int i = -g[0]; i < n[0] + g[0]; i++) {
                long mi = (i + g[0]) + (long)m[0] * ((j + g[1]) + (long)m[1] * (k + g[2]));
                double V0[OR_NQ], UL[3][OR_NQ], UR[3][OR_NQ], hq[4] = {0.0, 0.0, 0.0, 0.0};
                grid_load(c, U, i, j, k, V0);
                for (int d = 0; d < 3; d++) {
                    if (!act[d]) continue;
                    double Vm[OR_NQ], Vp[OR_NQ];
                    int o[3] = {0, 0, 0};
                    o[d] = 1;
                    grid_load(c, U, i - o[0], j - o[1], k - o[2], Vm);
                    grid_load(c, U, i + o[0], j + o[1], k + o[2], Vp);
                    /* Eq. 15-17 along axis d */
                    for (int q = 0; q < 4; q++) {
                        double sl = or_limiter(c->limiter, V0[q] - Vm[q], Vp[q] - V0[q]);
                        UL[d][q] = V0[q] - 0.5 * sl;
                        UR[d][q] = V0[q] + 0.5 * sl;
                    }
                    if (c->hancock) {   /* Eq. 13: the axis-d term of the half step */
                        double FLd[OR_NQ], FRd[OR_NQ];
                        or_flux(c, d, UL[d], FLd);
                        or_flux(c, d, UR[d], FRd);
                        for (int q = 0; q < 4; q++)
                            hq[q] += 0.5 * (dt / h[d]) * (FLd[q] - FRd[q]);
                    }
                }
                int ok = 1;
                for (int d = 0; d < 3; d++) {
                    if (!act[d]) continue;
                    for (int q = 0; q < 4; q++) {
                        UL[d][q] += hq[q];
                        UR[d][q] += hq[q];
                    }
                    if (!admissible(c, UL[d]) || !admissible(c, UR[d])) ok = 0;
                }
                if (!ok) OR_TALLY(g_face_fallback, 1);
                for (int d = 0; d < 3; d++) {
                    if (!act[d]) continue;
                    for (int q = 0; q < 4; q++) {
                        FLf[((long)d * mcells + mi) * 4 + q] = ok ? UL[d][q] : V0[q];
                        FRf[((long)d * mcells + mi) * 4 + q] = ok ? UR[d][q] : V0[q];
                    }
                }
            }
    for (long x = 0; x < 4 * cells; x++) D[x] = 0.0;
    /* MUSTA-FORCE fluxes at both interfaces of every real cell, axis by axis */
    for (int d = 0; d < 3; d++) {
        if (!act[d]) continue;
        double lam = dt / h[d];
        for (int k = 0; k < n[2]; k++)
            for (int j = 0; j < n[1]; j++)
                for (int i = 0; i < n[0]; i++) {
                    int o[3] = {0, 0, 0};
                    o[d] = 1;
                    long mc = (i + g[0]) + (long)m[0] * ((j + g[1]) + (long)m[1] * (k + g[2]));
                    long mm = (i - o[0] + g[0]) +
                              (long)m[0] * ((j - o[1] + g[1]) + (long)m[1] * (k - o[2] + g[2]));
                    long mp = (i + o[0] + g[0]) +
                              (long)m[0] * ((j + o[1] + g[1]) + (long)m[1] * (k + o[2] + g[2]));
                    double Fm[OR_NQ], Fp[OR_NQ];
                    /* interface i-1/2: right face of cell i-1, left face of cell i (R3) */
                    or_musta_force(c, d, lam, &FRf[((long)d * mcells + mm) * 4],
                                   &FLf[((long)d * mcells + mc) * 4], Fm);
                    or_musta_force(c, d, lam, &FRf[((long)d * mcells + mc) * 4],
                                   &FLf[((long)d * mcells + mp) * 4], Fp);
                    long cidx = i + (long)n[0] * (j + (long)n[1] * k);
                    for (int q = 0; q < 4; q++) D[q * cells + cidx] += lam * (Fp[q] - Fm[q]);
                }
    }
    free(FLf);
    free(FRf);
}

/* one unsplit step of length dt: the RK stages of Eq. 5-7 on the whole field */
static void unsplit_rk(const or_config *c, double *U, double dt) {
    long cells = (long)c->nx * c->ny * c->nz;
    long nv = 4 * cells;
    double *D = (double *)malloc(sizeof(double) * nv);
    double *U1 = (double *)malloc(sizeof(double) * nv);
    double *U2 = (double *)malloc(sizeof(double) * nv);
    unsplit_L(c, U, dt, D);
    if (c->rk_order == 1) {
        for (long x = 0; x < nv; x++) U[x] = U[x] - D[x];
    } else {
        for (long x = 0; x < nv; x++) U1[x] = U[x] - D[x];   /* U1 = U + dt L(U) */
        unsplit_L(c, U1, dt, D);
        if (c->rk_order == 3) {
            for (long x = 0; x < nv; x++) U2[x] = 0.75 * U[x] + 0.25 * (U1[x] - D[x]);
            unsplit_L(c, U2, dt, D);
            for (long x = 0; x < nv; x++) U[x] = U[x] / 3.0 + (2.0 / 3.0) * (U2[x] - D[x]);
        } else {
            for (long x = 0; x < nv; x++) U[x] = 0.5 * (U[x] + U1[x] - D[x]);
        }
    }
    free(D);
    free(U1);
    free(U2);
}

/* R16c: max over cells of sum over active axes of speed/dx */
double or_max_rate_unsplit(const or_config *c, const double *U) {
    long cells = (long)c->nx * c->ny * c->nz;
    int n[3] = {c->nx, c->ny, c->nz};
    double h[3] = {c->dx, c->dy, c->dz};
    double m = 0.0;
    for (long i = 0; i < cells; i++) {
        double u[4] = {U[i], U[cells + i], U[2 * cells + i], U[3 * cells + i]};
        double r = 0.0;
        for (int d = 0; d < 3; d++)
            if (n[d] > 1) r += or_signal_speed(c, u, d) / h[d];
        if (r > m) m = r;
    }
    return m;
}

/* ----------------------------------------------------------------- step */
/* one full step: dt (R8 or R16c), source (R12), Strang sweeps (R7) or the
   unsplit scheme (R16).  Returns dt. */
double or_step(const or_config *c, double *U, double t, double t_end) {
    double dt;
    if (c->fixed_dt > 0.0) dt = c->fixed_dt;
    else dt = c->cfl / (c->unsplit ? or_max_rate_unsplit(c, U) : or_max_rate(c, U));
    if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
    if (!(dt > 0.0)) return 0.0;
    if (c->unsplit && c->charge) return 0.0;   /* R19: not built for the unsplit scheme */
    if (c->jet_on) or_jet_source(c, U, t, dt);
    if (c->unsplit) {
        unsplit_rk(c, U, dt);
        return dt;
    }
    int n[3] = {c->nx, c->ny, c->nz};
    int act[3], na = 0;
    for (int d = 0; d < 3; d++) if (n[d] > 1) act[na++] = d;
    if (na == 0) return dt;
    for (int k = 0; k < na - 1; k++) or_sweep(c, U, act[k], 0.5 * dt);
    or_sweep(c, U, act[na - 1], dt);
    for (int k = na - 2; k >= 0; k--) or_sweep(c, U, act[k], 0.5 * dt);
    return dt;
}

/* advance up to nsteps steps (stopping at t_end when t_end > 0); returns steps taken */
int or_run(const or_config *c, double *U, int nsteps, double t_end, double *t) {
    int s;
    for (s = 0; s < nsteps; s++) {
        if (t_end > 0.0 && *t >= t_end) break;
        double dt = or_step(c, U, *t, t_end);
        if (!(dt > 0.0)) break;
        if (t_end > 0.0 && *t + dt >= t_end) *t = t_end;
        else *t += dt;
    }
    return s;
}

/* ---------------------------------------------------- whole-field helpers */
/* sum_cells U * dV for the four conserved fields */
void or_conservation_sums(const or_config *c, const double *U, double *out) {
    long cells = (long)c->nx * c->ny * c->nz;
    double dV = c->dx * c->dy * c->dz;
    for (int q = 0; q < nq_of(c); q++) {
        double s = 0.0;
        for (long i = 0; i < cells; i++) s += U[q * cells + i];
        out[q] = s * dV;
    }
}

/* n may be NULL (charge 0 everywhere) */
void or_prim2cons_field(const or_config *c, long cells, const double *e, const double *vx,
                        const double *vy, const double *vz, const double *n, double *U) {
    for (long i = 0; i < cells; i++) {
        double u[OR_NQ];
        or_prim2cons_n(c, e[i], vx[i], vy[i], vz[i], n ? n[i] : 0.0, u);
        for (int q = 0; q < nq_of(c); q++) U[q * cells + i] = u[q];
    }
}

/* R19: rest-frame charge density n = R / gamma = R sqrt(1 - v^2) per cell,
   v from cons->prim of the energy-momentum fields (vacuum: n = R) */
void or_charge_density_field(const or_config *c, long cells, const double *U, double *n) {
    for (long i = 0; i < cells; i++) {
        double u[4] = {U[i], U[cells + i], U[2 * cells + i], U[3 * cells + i]};
        double e, v[3], p;
        or_cons2prim(c, u, &e, v, &p, NULL);
        n[i] = U[4 * cells + i] * sqrt(1.0 - (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    }
}

void or_cons2prim_field(const or_config *c, long cells, const double *U, double *e, double *vx,
                        double *vy, double *vz, int *iters) {
    for (long i = 0; i < cells; i++) {
        double u[4] = {U[i], U[cells + i], U[2 * cells + i], U[3 * cells + i]};
        double v[3], p;
        int it = 0;
        or_cons2prim(c, u, &e[i], v, &p, &it);
        vx[i] = v[0]; vy[i] = v[1]; vz[i] = v[2];
        if (iters) iters[i] = it;
    }
}
