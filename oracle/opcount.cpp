// opcount.cpp -- op-counting build of the CPU oracle (TEST INFRASTRUCTURE:
// loaded only by the tests and by the CPU leg of the benchmark, like the
// oracle itself).
//
// The oracle's C source is compiled here a second time as C++ with every
// `double` replaced by a value type that records each arithmetic operation
// as a node of a dataflow graph.  After a sweep, the operations that the
// output state depends on are counted by kind.  An operation counts as an
// algorithmic flop when
//   * it is an add, subtract, multiply, divide, square root, min or max
//     (fabs and negation only touch the sign bit and are not counted; exp,
//     log, tanh are counted on their own), and
//   * at least one operand is derived from the state (operations on
//     constants alone, such as alpha * dt / dx, are set up once per sweep),
//   * and its result reaches the output (values the oracle computes but the
//     update never reads, such as e in cons->prim for a flux, are not work
//     the method needs).
// Operations are counted once each: the same operation on the same operands
// is one node however often the oracle's plain loops evaluate it.
// The arithmetic itself is the oracle's: the same source, the same order.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <unordered_map>
#include <vector>

namespace opc {
enum Kind { LEAF, ADD, SUB, MUL, DIV, SQRT, MIN, MAX, EXP, LOG, TANH, ABS, NEG, FLOOR, NKIND };
struct Node {
    int kind, a, b;
};
// node 0 is the "constant" sentinel: id <= 0 means not derived from the state.
// Nodes are hash-consed: the same operation on the same operands (in the same
// order) is one node, so work the oracle repeats (an interface flux taken
// once for each neighbouring cell, faces of periodic ghost cells) counts once.
static std::vector<Node> g_nodes(1, Node{LEAF, 0, 0});
static std::unordered_map<uint64_t, int> g_seen;
static inline void reset() {
    g_nodes.assign(1, Node{LEAF, 0, 0});
    g_seen.clear();
}
static inline int mk(int k, int a, int b) {
    if (a <= 0 && b <= 0) return 0;
    const uint64_t key = (uint64_t)k | ((uint64_t)(uint32_t)a << 4) | ((uint64_t)(uint32_t)b << 34);
    auto it = g_seen.find(key);
    if (it != g_seen.end()) return it->second;
    g_nodes.push_back(Node{k, a, b});
    const int id = (int)g_nodes.size() - 1;
    g_seen.emplace(key, id);
    return id;
}
static inline int leaf() {
    g_nodes.push_back(Node{LEAF, 0, 0});
    return (int)g_nodes.size() - 1;
}
}  // namespace opc

struct Flop {
    double v;
    int id;
    Flop() : v(0.0), id(0) {}
    Flop(double x) : v(x), id(0) {}
    explicit operator int() const { return (int)v; }
    explicit operator long() const { return (long)v; }
    explicit operator float() const { return (float)v; }
};

static inline Flop fl(double v, int id) {
    Flop r;
    r.v = v;
    r.id = id;
    return r;
}
static inline Flop operator+(Flop x, Flop y) { return fl(x.v + y.v, opc::mk(opc::ADD, x.id, y.id)); }
static inline Flop operator-(Flop x, Flop y) { return fl(x.v - y.v, opc::mk(opc::SUB, x.id, y.id)); }
static inline Flop operator*(Flop x, Flop y) { return fl(x.v * y.v, opc::mk(opc::MUL, x.id, y.id)); }
static inline Flop operator/(Flop x, Flop y) { return fl(x.v / y.v, opc::mk(opc::DIV, x.id, y.id)); }
static inline Flop operator-(Flop x) { return fl(-x.v, opc::mk(opc::NEG, x.id, 0)); }
static inline Flop &operator+=(Flop &x, Flop y) { return x = x + y; }
static inline Flop &operator-=(Flop &x, Flop y) { return x = x - y; }
static inline Flop &operator*=(Flop &x, Flop y) { return x = x * y; }
static inline Flop &operator/=(Flop &x, Flop y) { return x = x / y; }
static inline bool operator<(Flop x, Flop y) { return x.v < y.v; }
static inline bool operator>(Flop x, Flop y) { return x.v > y.v; }
static inline bool operator<=(Flop x, Flop y) { return x.v <= y.v; }
static inline bool operator>=(Flop x, Flop y) { return x.v >= y.v; }
static inline bool operator==(Flop x, Flop y) { return x.v == y.v; }
static inline bool operator!=(Flop x, Flop y) { return x.v != y.v; }
static inline Flop sqrt(Flop x) { return fl(sqrt(x.v), opc::mk(opc::SQRT, x.id, 0)); }
static inline Flop fabs(Flop x) { return fl(fabs(x.v), opc::mk(opc::ABS, x.id, 0)); }
static inline Flop fmin(Flop x, Flop y) { return fl(fmin(x.v, y.v), opc::mk(opc::MIN, x.id, y.id)); }
static inline Flop fmax(Flop x, Flop y) { return fl(fmax(x.v, y.v), opc::mk(opc::MAX, x.id, y.id)); }
static inline Flop exp(Flop x) { return fl(exp(x.v), opc::mk(opc::EXP, x.id, 0)); }
static inline Flop log(Flop x) { return fl(log(x.v), opc::mk(opc::LOG, x.id, 0)); }
static inline Flop tanh(Flop x) { return fl(tanh(x.v), opc::mk(opc::TANH, x.id, 0)); }
static inline Flop floor(Flop x) { return fl(floor(x.v), opc::mk(opc::FLOOR, x.id, 0)); }

#define double Flop
#include "musta_oracle.c"
#undef double

// count by kind the operations that the state U depends on
static void count_live(const std::vector<Flop> &U, long long *out) {
    std::vector<char> live(opc::g_nodes.size(), 0);
    std::vector<int> stack;
    for (const Flop &f : U)
        if (f.id > 0) stack.push_back(f.id);
    while (!stack.empty()) {
        const int k = stack.back();
        stack.pop_back();
        if (k <= 0 || live[k]) continue;
        live[k] = 1;
        stack.push_back(opc::g_nodes[k].a);
        stack.push_back(opc::g_nodes[k].b);
    }
    for (int k = 0; k < opc::NKIND; k++) out[k] = 0;
    for (size_t k = 1; k < opc::g_nodes.size(); k++)
        if (live[k]) out[opc::g_nodes[k].kind]++;
}

// Per-cell operation counts of one sweep along x, by kind (LEAF unused):
// the difference between pencils of n2 and n1 cells (periodic), divided by
// n2 - n1, so that the ends of the pencil do not enter.  The state is a
// smooth monotone ramp with flow along every axis, so every cell takes the
// general path (non-zero limited slopes, no cap, no fallback, no vacuum).
// Returns 0, or -1 when the difference is not a whole number per cell.
static void count_pencil(int N, int limiter, int stages, int rk_order, int hancock,
                         long long *out) {
    or_config c;
    memset(&c, 0, sizeof c);
    c.nx = N;
    c.ny = c.nz = 1;
    c.dx = c.dy = c.dz = 1.0 / N;
    c.limiter = limiter;
    c.stages = stages;
    c.rk_order = rk_order;
    c.hancock = hancock;
    c.alpha = 1.0;
    c.cfl = 0.4;
    c.delta = 1e-12;
    c.eos_kind = 0;
    c.cs2 = 1.0 / 3.0;
    const long cells = N;
    std::vector<Flop> U(4 * cells);
    opc::reset();
    for (long i = 0; i < cells; i++) {
        const double e = 1.0 + 0.5 * (double)i / N;
        double u[4];
        // prim -> cons in plain double (set-up, not counted)
        const double vx = 0.3, vy = 0.1, vz = -0.05, p = e / 3.0;
        const double w = (e + p) / (1.0 - (vx * vx + vy * vy + vz * vz));
        u[0] = w - p;
        u[1] = w * vx;
        u[2] = w * vy;
        u[3] = w * vz;
        for (int q = 0; q < 4; q++) U[q * cells + i] = fl(u[q], opc::leaf());
    }
    or_sweep(&c, U.data(), 0, 0.4 * c.dx);
    count_live(U, out);
}

extern "C" int or_opcount_nkind(void) { return opc::NKIND; }

// Per-cell operation counts of one RK stage of the unsplit scheme (reading
// R16, alpha = 3) on an n^3 periodic grid with a smooth state (flow along
// every axis, no extremum sits exactly on a cell) and central slopes, so
// every cell takes the same path; one step has rk_order stages.
extern "C" int or_opcount_unsplit(int stages, int rk_order, int hancock, int n,
                                  long long *per_cell_stage) {
    or_config c;
    memset(&c, 0, sizeof c);
    c.nx = c.ny = c.nz = n;
    c.dx = c.dy = c.dz = 1.0 / n;
    c.limiter = 0;
    c.stages = stages;
    c.rk_order = rk_order;
    c.hancock = hancock;
    c.alpha = 3.0;
    c.cfl = 0.4;
    c.fixed_dt = 0.1 / n;
    c.delta = 1e-12;
    c.cs2 = 1.0 / 3.0;
    c.unsplit = 1;
    const long cells = (long)n * n * n;
    std::vector<Flop> U(4 * cells);
    opc::reset();
    const double tw = 6.283185307179586;
    for (int z = 0; z < n; z++)
        for (int y = 0; y < n; y++)
            for (int x = 0; x < n; x++) {
                const long i = x + (long)n * (y + (long)n * z);
                const double X = (x + 0.3) / n, Y = (y + 0.3) / n, Z = (z + 0.3) / n;
                const double e = 1.0 + 0.2 * sin(tw * X) * cos(tw * Y) + 0.1 * sin(tw * Z);
                const double vx = 0.2 * cos(tw * Y), vy = 0.15 * sin(tw * Z),
                             vz = 0.1 * cos(tw * X);
                const double p = e / 3.0;
                const double w = (e + p) / (1.0 - (vx * vx + vy * vy + vz * vz));
                const double u[4] = {w - p, w * vx, w * vy, w * vz};
                for (int q = 0; q < 4; q++) U[q * cells + i] = fl(u[q], opc::leaf());
            }
    or_step(&c, U.data(), 0.0, 0.0);
    std::vector<long long> tot(opc::NKIND);
    count_live(U, tot.data());
    int ok = 0;
    for (int k = 0; k < opc::NKIND; k++) {
        if (tot[k] % (cells * rk_order)) ok = -1;
        per_cell_stage[k] = tot[k] / (cells * rk_order);
    }
    return ok;
}

extern "C" int or_opcount_sweep(int limiter, int stages, int rk_order, int hancock, int n1,
                                int n2, long long *per_cell) {
    std::vector<long long> a(opc::NKIND), b(opc::NKIND);
    count_pencil(n1, limiter, stages, rk_order, hancock, a.data());
    count_pencil(n2, limiter, stages, rk_order, hancock, b.data());
    int ok = 0;
    for (int k = 0; k < opc::NKIND; k++) {
        const long long d = b[k] - a[k];
        if (d % (n2 - n1)) ok = -1;
        per_cell[k] = d / (n2 - n1);
    }
    return ok;
}
