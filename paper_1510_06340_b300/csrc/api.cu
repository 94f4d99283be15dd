// api.cu -- the C ABI of include/hydro.h: handles, device memory, work lists,
// launch-shape autotuning and CUDA-graph capture of steps.
//
// A single grid is a batch of one event; both share the Solver below.  All
// events' fields live in one allocation, event-major then field-major:
// state[off_e + f * cells_e + (z * ny + y) * nx + x].  Two copies are kept:
// a sweep reads one and writes the other.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hydro.h"
#include "common.h"
#include "kernels.h"

using namespace hy;

namespace {

thread_local std::string g_err;

hydro_status fail(hydro_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? HYDRO_E_OOM : HYDRO_E_CUDA,   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

struct LaunchShape {
    int threads = 128;
    int seg_len = 0;      // target segment length; 0 = whole pencils
};

// the derived constants, in the arithmetic of R itself
template <class R>
static void set_consts(SchemeConsts<R> &k, R alpha, R delta, R cs2) {
    k.alpha = alpha;
    k.delta = delta;
    k.omd = R(1) - delta;
    k.capf = k.omd * k.omd;
    k.cs2 = cs2;
    k.cs = std::sqrt(cs2);
    k.k1 = R(1) - cs2;
    k.hapc = R(0.5) * (R(1) + cs2);
    k.hapc2 = k.hapc * k.hapc;
    k.emin = sizeof(R) == 8 ? R(std::ldexp(1.0, -500)) : R(std::ldexp(1.0, -60));
    k.wmin = k.hapc * k.emin;
}

struct Solver {
    int nevents = 0;
    int nq = 4;               // conserved fields per cell: 4, or 5 with the charge R
    int prec = HYDRO_FP64;
    int rk = 2;
    double cfl = 0.4, fixed_dt = 0.0;
    size_t elem = 8;
    long long total_cells = 0;
    std::vector<EventGeo> geo;
    EventGeo *d_geo = nullptr;
    EventClock *d_clk = nullptr, *d_clk_tune = nullptr;
    void *d_state[2] = {nullptr, nullptr};
    int cur = 0;
    // work lists
    std::vector<WorkItem> cell_items;
    WorkItem *d_cell_items = nullptr;
    // the FP64 sums' work list: larger chunks, so that each thread adds many
    // cells before the block reduction (FP64 adds issue slowly on this GPU)
    std::vector<WorkItem> sum_items;
    WorkItem *d_sum_items = nullptr;
    std::vector<WorkItem> sweep_items[3];
    WorkItem *d_sweep_items[3] = {nullptr, nullptr, nullptr};
    size_t sweep_cap[3] = {0, 0, 0};
    double *d_partial = nullptr, *d_sums = nullptr;
    int *d_work_counter = nullptr;     // persistent sweeps of a batch
    // unsplit scheme (R16): scratch faces and fluxes, RK stage states, work lists
    bool unsplit = false;
    std::vector<UnsplitGeo> ugeo;
    UnsplitGeo *d_ugeo = nullptr;
    void *d_faces = nullptr;
    void *d_stage[2] = {nullptr, nullptr};
    std::vector<WorkItem> us_face_items, us_tile_items;
    WorkItem *d_us_face_items = nullptr, *d_us_tile_items = nullptr;
    // scheme
    Scheme sc{};
    double *d_p64 = nullptr, *d_c64 = nullptr;
    float *d_p32 = nullptr, *d_c32 = nullptr;
    float *d_mlp_f = nullptr;
    void *d_mlp_w = nullptr;
    unsigned long long *d_counters = nullptr;
    unsigned *d_flags = nullptr;       // FLAG_* status word per event
    bool counters_on = false;
    bool any_jet = false;
    long long jet_cells = 0;   // largest box of cells around a jet (k_jet threads per event)
    bool active[3] = {false, false, false};
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;   // used until the caller sets a stream
    int sms = 148;
    // launch shapes
    LaunchShape shape[3];
    bool tuned[3] = {false, false, false};
    bool forced[3] = {false, false, false};
    // graphs of two steps, one per starting state buffer (a captured graph
    // bakes in the buffer it reads first; steps run outside a graph flip it)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool graph_dirty = true;
    bool graph_ok[2] = {false, false};
    double t_end_dev = -1.0;
    bool rate_valid = false;   // clk.rate_bits holds the rate of the current state
    // kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;        // per recorded pair: 0 sweep, 1 other
    size_t ev_used = 0;
    double timing_ms[2] = {0.0, 0.0};
    long long timing_n[2] = {0, 0};

    ~Solver() { release(); }

    void release() {
        for (int p = 0; p < 2; ++p) {
            if (graph[p]) cudaGraphExecDestroy(graph[p]);
            graph[p] = nullptr;
        }
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        ev_pool.clear();
        if (own_stream) {
            cudaStreamSynchronize(own_stream);
            cudaStreamDestroy(own_stream);
        }
        own_stream = nullptr;
        void *ptrs[] = {d_geo, d_clk, d_clk_tune, d_state[0], d_state[1], d_cell_items,
                        d_sweep_items[0], d_sweep_items[1], d_sweep_items[2], d_partial, d_sums,
                        d_p64, d_c64, d_p32, d_c32, d_mlp_f, d_mlp_w, d_counters, d_flags,
                        d_work_counter, d_ugeo, d_faces, d_stage[0], d_stage[1],
                        d_us_face_items, d_us_tile_items, d_sum_items};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        d_geo = nullptr;
        d_clk = d_clk_tune = nullptr;
        d_state[0] = d_state[1] = nullptr;
        d_cell_items = d_sum_items = nullptr;
        for (int a = 0; a < 3; ++a) d_sweep_items[a] = nullptr;
        d_partial = d_sums = nullptr;
        d_p64 = d_c64 = nullptr;
        d_p32 = d_c32 = nullptr;
        d_mlp_f = nullptr;
        d_mlp_w = nullptr;
        d_counters = nullptr;
        d_flags = nullptr;
        d_work_counter = nullptr;
        d_ugeo = nullptr;
        d_faces = nullptr;
        d_stage[0] = d_stage[1] = nullptr;
        d_us_face_items = nullptr;
        d_us_tile_items = nullptr;
    }

    Scheme scheme() const {
        Scheme s = sc;
        s.counters = counters_on ? d_counters : nullptr;
        return s;
    }

    CellLaunch cell_launch() const {
        CellLaunch c;
        c.ev = d_geo;
        c.items = d_cell_items;
        c.nitems = (int)cell_items.size();
        c.threads = 256;
        c.blocks = (int)std::min<size_t>(cell_items.size(), (size_t)sms * 8);
        c.stream = stream;
        c.prec = prec == HYDRO_FP64 ? 0 : 1;
        c.mixed = prec == HYDRO_MIXED ? 1 : 0;
        c.sc = scheme();
        c.rate_sum = unsplit ? 1 : 0;
        c.jet_cells = jet_cells;
        c.nevents = nevents;
        c.nq = nq;
        return c;
    }

    // ---------------------------------------------------------------- setup
    hydro_status init(const hydro_grid_t *grids, int n, const hydro_eos_t *eos, int limiter,
                      int stages) {
        if (!grids || n < 1) return fail(HYDRO_E_INVALID, "no grids");
        const hydro_grid_t &g0 = grids[0];
        if (g0.prec < 0 || g0.prec > 2) return fail(HYDRO_E_INVALID, "unknown precision");
        if (g0.rk_order < 1 || g0.rk_order > 3) return fail(HYDRO_E_INVALID, "rk_order must be 1..3");
        if (limiter < 0 || limiter > 5) return fail(HYDRO_E_INVALID, "unknown limiter");
        if (stages < 1 || stages > 64) return fail(HYDRO_E_INVALID, "stages must be >= 1");
        if (!(g0.cfl > 0.0) && !(g0.fixed_dt > 0.0))
            return fail(HYDRO_E_INVALID, "need cfl > 0 or fixed_dt > 0");
        if (!(g0.alpha > 0.0)) return fail(HYDRO_E_INVALID, "alpha must be > 0");
        nevents = n;
        prec = g0.prec;
        rk = g0.rk_order;
        unsplit = g0.unsplit != 0;
        for (int e = 1; e < n; ++e)
            if ((grids[e].unsplit != 0) != unsplit)
                return fail(HYDRO_E_INVALID, "all events of a batch use the same scheme (unsplit)");
        nq = g0.charge ? 5 : 4;
        for (int e = 1; e < n; ++e)
            if ((grids[e].charge ? 5 : 4) != nq)
                return fail(HYDRO_E_INVALID, "all events of a batch carry the charge or none does");
        if (nq == 5 && unsplit)
            return fail(HYDRO_E_INVALID, "the conserved charge is carried by the split sweeps only");
        if (nq == 5 && eos && eos->kind == HYDRO_EOS_TABLE && eos->seed == HYDRO_SEED_MLP)
            return fail(HYDRO_E_INVALID, "the conserved charge does not run with the MLP seed");
        cfl = g0.cfl;
        fixed_dt = g0.fixed_dt;
        elem = prec == HYDRO_FP64 ? 8 : 4;
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaStreamCreateWithFlags(&own_stream, cudaStreamNonBlocking));
        stream = own_stream;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        geo.resize(n);
        long long off = 0;
        for (int e = 0; e < n; ++e) {
            const hydro_grid_t &g = grids[e];
            if (g.nx < 1 || g.ny < 1 || g.nz < 1)
                return fail(HYDRO_E_INVALID, "grid sizes must be >= 1");
            const double h[3] = {g.dx, g.dy, g.dz};
            const int nn[3] = {g.nx, g.ny, g.nz};
            EventGeo &q = geo[e];
            memset(&q, 0, sizeof q);
            for (int a = 0; a < 3; ++a) {
                if (nn[a] > 1 && !(h[a] > 0.0)) return fail(HYDRO_E_INVALID, "cell size must be > 0");
                if (g.bc[a] != HYDRO_BC_PERIODIC && g.bc[a] != HYDRO_BC_OUTFLOW)
                    return fail(HYDRO_E_INVALID, "unknown boundary condition");
                q.n[a] = nn[a];
                q.h[a] = h[a] > 0.0 ? h[a] : 1.0;
                q.inv_h[a] = 1.0 / q.h[a];
                q.inv_hf[a] = (float)q.inv_h[a];
                q.bc[a] = g.bc[a];
                q.seg[a] = 1;
                q.segL[a] = nn[a];
                if (nn[a] > 1) active[a] = true;
            }
            q.lo[0] = g.x0; q.lo[1] = g.y0; q.lo[2] = g.z0;
            q.cells = (long long)g.nx * g.ny * g.nz;
            if (nq * q.cells > 2147483647LL)   // sweeps index fields with 32-bit offsets
                return fail(HYDRO_E_INVALID, nq == 4 ? "an event may hold at most 536,870,911 cells"
                                                     : "a charged event may hold at most "
                                                       "429,496,729 cells");
            q.off = off;
            off += nq * q.cells;
            total_cells += q.cells;
        }
        // scheme
        sc.limiter = limiter;
        sc.stages = stages;
        sc.hancock = g0.hancock ? 1 : 0;
        sc.alpha = g0.alpha;
        sc.delta = prec == HYDRO_FP64 ? DELTA_F64 : DELTA_F32;
        hydro_eos_t conf{};
        conf.kind = HYDRO_EOS_CONFORMAL;
        conf.cs2 = 1.0 / 3.0;
        if (!eos) eos = &conf;
        sc.eos_kind = eos->kind;
        sc.cs2 = eos->cs2;
        sc.seed = eos->seed;
        sc.tol = eos->newton_tol > 0.0 ? eos->newton_tol : (prec == HYDRO_FP64 ? 1e-13 : 2e-6);
        sc.newton_max_it = eos->newton_max_iter > 0 ? eos->newton_max_iter : NEWTON_MAX_IT;
        if (sc.newton_max_it > 1000) return fail(HYDRO_E_INVALID, "newton_max_iter must be <= 1000");
        set_consts(sc.c64, sc.alpha, DELTA_F64, sc.cs2);
        set_consts(sc.c32, float(sc.alpha), float(DELTA_F32), float(sc.cs2));
        if (eos->kind == HYDRO_EOS_CONFORMAL) {
            if (!(eos->cs2 >= 0.0 && eos->cs2 < 1.0)) return fail(HYDRO_E_INVALID, "cs2 must be in [0,1)");
        } else if (eos->kind == HYDRO_EOS_TABLE) {
            if (eos->n < 2 || !eos->p_tab || !eos->cs2_tab || !(eos->lne_max > eos->lne_min))
                return fail(HYDRO_E_INVALID, "bad EOS table");
            if (eos->seed < 0 || eos->seed > 2) return fail(HYDRO_E_INVALID, "unknown Newton seed");
            if (eos->seed == HYDRO_SEED_MLP && !eos->mlp_params)
                return fail(HYDRO_E_INVALID, "MLP seed needs mlp_params");
            const int tn = eos->n;
            sc.tab_n = tn;
            sc.lne_min = eos->lne_min;
            sc.lne_max = eos->lne_max;
            sc.inv_h = double(tn - 1) / (eos->lne_max - eos->lne_min);
            sc.e_max = std::exp(eos->lne_max);
            // packed nodes (p_i, p_{i+1} - p_i, c2_i, c2_{i+1} - c2_i); each
            // difference in its own precision, as the interpolation takes it
            std::vector<double> t64(4 * (size_t)tn);
            std::vector<float> t32(4 * (size_t)tn);
            for (int i = 0; i < tn; ++i) {
                const int j = i + 1 < tn ? i + 1 : i;
                t64[4 * i + 0] = eos->p_tab[i];
                t64[4 * i + 1] = eos->p_tab[j] - eos->p_tab[i];
                t64[4 * i + 2] = eos->cs2_tab[i];
                t64[4 * i + 3] = eos->cs2_tab[j] - eos->cs2_tab[i];
                const float p0 = (float)eos->p_tab[i], p1 = (float)eos->p_tab[j];
                const float c0 = (float)eos->cs2_tab[i], c1 = (float)eos->cs2_tab[j];
                t32[4 * i + 0] = p0;
                t32[4 * i + 1] = p1 - p0;
                t32[4 * i + 2] = c0;
                t32[4 * i + 3] = c1 - c0;
            }
            CK(cudaMalloc(&d_p64, t64.size() * sizeof(double)));
            CK(cudaMalloc(&d_p32, t32.size() * sizeof(float)));
            CK(cudaMemcpy(d_p64, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(d_p32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice));
            sc.tab64 = d_p64;
            sc.tab32 = d_p32;
            if (eos->mlp_params) {
                CK(cudaMalloc(&d_mlp_f, MLP_NPARAM * sizeof(float)));
                CK(cudaMalloc(&d_mlp_w, MLP_NPARAM * sizeof(__nv_bfloat16)));
                CK(cudaMemcpy(d_mlp_f, eos->mlp_params, MLP_NPARAM * sizeof(float),
                              cudaMemcpyHostToDevice));
                CK(launch_mlp_prepare(d_mlp_f, d_mlp_w, nullptr));
                sc.mlp_f = d_mlp_f;
                sc.mlp_w = d_mlp_w;
            }
        } else {
            return fail(HYDRO_E_INVALID, "unknown EOS kind");
        }
        // the MLP seed's range: E above the first table node where p departs
        // from e/3 by more than 1e-4 (half of it, as a margin); below, the
        // closed-form p = e/3 root seeds Newton
        sc.c64.mlp_emin = 0.0;
        if (eos->kind == HYDRO_EOS_TABLE) {
            const double hnode = (eos->lne_max - eos->lne_min) / double(eos->n - 1);
            double emin = std::exp(eos->lne_max);
            for (int i = 0; i < eos->n; ++i) {
                const double e = std::exp(eos->lne_min + i * hnode);
                if (std::fabs(eos->p_tab[i] - e / 3.0) > 1e-4 * (e / 3.0)) {
                    emin = 0.5 * e;
                    break;
                }
            }
            sc.c64.mlp_emin = emin;
        }
        sc.c32.mlp_emin = float(sc.c64.mlp_emin);
        sc.c64.lne_min = sc.lne_min;
        sc.c64.inv_h = sc.inv_h;
        sc.c64.e_max = sc.e_max;
        sc.c32.lne_min = float(sc.lne_min);
        sc.c32.inv_h = float(sc.inv_h);
        sc.c32.e_max = float(sc.e_max);
        sc.c64.l2_scale = std::log(2.0) * sc.inv_h;
        sc.c64.l2_off = -sc.lne_min * sc.inv_h;
        sc.c32.l2_scale = float(sc.c64.l2_scale);
        sc.c32.l2_off = float(sc.c64.l2_off);
        // device memory
        const size_t bytes = (size_t)nq * total_cells * elem;
        CK(cudaMalloc(&d_state[0], bytes));
        CK(cudaMalloc(&d_state[1], bytes));
        CK(cudaMemset(d_state[0], 0, bytes));
        CK(cudaMemset(d_state[1], 0, bytes));
        CK(cudaMalloc(&d_geo, n * sizeof(EventGeo)));
        CK(cudaMemcpy(d_geo, geo.data(), n * sizeof(EventGeo), cudaMemcpyHostToDevice));
        std::vector<EventClock> clk(n);
        memset(clk.data(), 0, n * sizeof(EventClock));
        CK(cudaMalloc(&d_clk, n * sizeof(EventClock)));
        CK(cudaMemcpy(d_clk, clk.data(), n * sizeof(EventClock), cudaMemcpyHostToDevice));
        for (int e = 0; e < n; ++e) {
            double hmin = 1e300;
            for (int a = 0; a < 3; ++a)
                if (geo[e].n[a] > 1) hmin = std::min(hmin, geo[e].h[a]);
            clk[e].dt = 0.2 * (hmin < 1e300 ? hmin : 1.0);
        }
        CK(cudaMalloc(&d_clk_tune, n * sizeof(EventClock)));
        CK(cudaMemcpy(d_clk_tune, clk.data(), n * sizeof(EventClock), cudaMemcpyHostToDevice));
        CK(cudaMalloc(&d_counters, NCOUNTERS * sizeof(unsigned long long)));
        CK(cudaMemset(d_counters, 0, NCOUNTERS * sizeof(unsigned long long)));
        CK(cudaMalloc(&d_flags, (size_t)n * sizeof(unsigned)));
        CK(cudaMemset(d_flags, 0, (size_t)n * sizeof(unsigned)));
        sc.event_flags = d_flags;
        // cell work list: chunks of 2048 cells of one event
        const int chunk = 2048;
        for (int e = 0; e < n; ++e)
            for (long long c = 0; c < geo[e].cells; c += chunk) {
                WorkItem w;
                w.event = e;
                w.first = c;
                w.count = (int)std::min<long long>(chunk, geo[e].cells - c);
                cell_items.push_back(w);
            }
        CK(cudaMalloc(&d_cell_items, cell_items.size() * sizeof(WorkItem)));
        CK(cudaMemcpy(d_cell_items, cell_items.data(), cell_items.size() * sizeof(WorkItem),
                      cudaMemcpyHostToDevice));
        // sums work list: chunks of 32768 cells of one event (128 per thread)
        const int schunk = 32768;
        for (int e = 0; e < n; ++e)
            for (long long c = 0; c < geo[e].cells; c += schunk) {
                WorkItem w;
                w.event = e;
                w.first = c;
                w.count = (int)std::min<long long>(schunk, geo[e].cells - c);
                sum_items.push_back(w);
            }
        CK(cudaMalloc(&d_sum_items, sum_items.size() * sizeof(WorkItem)));
        CK(cudaMemcpy(d_sum_items, sum_items.data(), sum_items.size() * sizeof(WorkItem),
                      cudaMemcpyHostToDevice));
        CK(cudaMalloc(&d_partial, sum_items.size() * nq * sizeof(double)));
        CK(cudaMalloc(&d_sums, (size_t)n * nq * sizeof(double)));
        if (n > 1) CK(cudaMalloc(&d_work_counter, sizeof(int)));
        if (unsplit) {
            hydro_status st = init_unsplit();
            if (st != HYDRO_OK) return st;
        }
        return HYDRO_OK;
    }

    // scratch and work lists of the unsplit scheme (R16)
    hydro_status init_unsplit() {
        ugeo.resize(nevents);
        long long fo = 0;
        const int tdim[3] = {US_TX, US_TY, US_TZ};
        for (int e = 0; e < nevents; ++e) {
            const EventGeo &g = geo[e];
            UnsplitGeo &u = ugeo[e];
            memset(&u, 0, sizeof u);
            long long tiles = 1;
            for (int a = 0; a < 3; ++a) {
                u.g[a] = g.n[a] > 1 ? 1 : 0;
                u.m[a] = g.n[a] + 2 * u.g[a];
                const int T = std::min(g.n[a], tdim[a]);
                tiles *= (g.n[a] + T - 1) / T;
            }
            u.gcells = (long long)u.m[0] * u.m[1] * u.m[2];
            u.fo = fo;
            fo += 24 * u.gcells;
            for (long long c = 0; c < u.gcells; c += US_ITEM) us_face_items.push_back(item(e, c, u.gcells));
            for (long long t = 0; t < tiles; ++t) {
                WorkItem w;
                w.event = e;
                w.first = t;
                w.count = 1;
                us_tile_items.push_back(w);
            }
        }
        CK(cudaMalloc(&d_ugeo, nevents * sizeof(UnsplitGeo)));
        CK(cudaMemcpy(d_ugeo, ugeo.data(), nevents * sizeof(UnsplitGeo), cudaMemcpyHostToDevice));
        CK(cudaMalloc(&d_faces, (size_t)fo * elem));
        const size_t bytes = (size_t)4 * total_cells * elem;
        CK(cudaMalloc(&d_stage[0], bytes));
        if (rk == 3) CK(cudaMalloc(&d_stage[1], bytes));
        auto upload = [&](const std::vector<WorkItem> &v, WorkItem **d) -> cudaError_t {
            if (v.empty()) return cudaSuccess;
            cudaError_t err = cudaMalloc(d, v.size() * sizeof(WorkItem));
            if (err != cudaSuccess) return err;
            return cudaMemcpy(*d, v.data(), v.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
        };
        CK(upload(us_face_items, &d_us_face_items));
        CK(upload(us_tile_items, &d_us_tile_items));
        return HYDRO_OK;
    }

    static constexpr int US_ITEM = 256;   // units per unsplit work item (one per thread)
    static WorkItem item(int e, long long first, long long total) {
        WorkItem w;
        w.event = e;
        w.first = first;
        w.count = (int)std::min<long long>(US_ITEM, total - first);
        return w;
    }

    // one step of the unsplit scheme after dt and the source: RK stages of
    // faces, fluxes and update; the last stage writes the spare buffer
    cudaError_t enqueue_unsplit(bool cfl_dt) {
        UnsplitLaunch a;
        a.faces = d_faces;
        a.ev = d_geo;
        a.ug = d_ugeo;
        a.face_items = d_us_face_items;
        a.n_face_items = (int)us_face_items.size();
        a.tile_items = d_us_tile_items;
        a.n_tile_items = (int)us_tile_items.size();
        a.clk = d_clk;
        a.sc = scheme();
        a.rk = rk;
        a.sms = sms;
        a.stream = stream;
        a.u0 = d_state[cur];
        for (int st = 1; st <= rk; ++st) {
            const bool last = st == rk;
            // stage inputs: U^n, then U1 (d_stage[0]), then U2 (d_stage[1])
            a.in = st == 1 ? d_state[cur] : d_stage[st - 2];
            a.u1 = st == 1 ? nullptr : d_stage[st - 2];
            a.out = last ? d_state[1 - cur] : d_stage[st - 1];
            a.stage = st;
            a.rate_clk = (last && cfl_dt) ? d_clk : nullptr;
            size_t sl = 0;
            cudaError_t e = mark_begin(0, sl);
            if (e != cudaSuccess) return e;
            if (prec == HYDRO_FP64) e = launch_unsplit_f64(a);
            else if (prec == HYDRO_FP32) e = launch_unsplit_f32(a);
            else e = launch_unsplit_mixed(a);
            if (e != cudaSuccess) return e;
            if ((e = mark_end(sl)) != cudaSuccess) return e;
        }
        cur = 1 - cur;
        return cudaSuccess;
    }

    // ---------------------------------------------------------------- launch shapes
    hydro_status build_sweep_items(int axis, const LaunchShape &s) {
        std::vector<WorkItem> &v = sweep_items[axis];
        v.clear();
        for (int e = 0; e < nevents; ++e) {
            EventGeo &g = geo[e];
            const int N = g.n[axis];
            int S = 1;
            if (s.seg_len > 0 && N > s.seg_len) S = (N + s.seg_len / 2) / s.seg_len;
            S = std::max(1, S);
            int L = (N + S - 1) / S;
            // x rows are staged 8 cells at a time: 8-aligned segment starts
            // keep every copy on whole 32-byte sectors
            if (axis == 0 && S > 1) L = std::min(N, (L + 7) / 8 * 8);
            S = (N + L - 1) / L;
            g.seg[axis] = S;
            g.segL[axis] = L;
            const long long tasks = (g.cells / N) * (long long)S;
            for (long long t = 0; t < tasks; t += s.threads) {
                WorkItem w;
                w.event = e;
                w.first = t;
                w.count = (int)std::min<long long>(s.threads, tasks - t);
                v.push_back(w);
            }
        }
        // longest pencils first so the tail of a launch is short
        std::stable_sort(v.begin(), v.end(), [&](const WorkItem &a, const WorkItem &b) {
            return geo[a.event].segL[axis] > geo[b.event].segL[axis];
        });
        if (v.size() > sweep_cap[axis]) {
            if (d_sweep_items[axis]) cudaFree(d_sweep_items[axis]);
            CK(cudaMalloc(&d_sweep_items[axis], v.size() * sizeof(WorkItem)));
            sweep_cap[axis] = v.size();
        }
        CK(cudaMemcpy(d_sweep_items[axis], v.data(), v.size() * sizeof(WorkItem),
                      cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_geo, geo.data(), nevents * sizeof(EventGeo), cudaMemcpyHostToDevice));
        shape[axis] = s;
        graph_dirty = true;
        return HYDRO_OK;
    }

    cudaError_t sweep_launch(int axis, double frac, const EventClock *clk, int src,
                             EventClock *rate_clk = nullptr) {
        SweepLaunch a;
        a.in = d_state[src];
        a.out = d_state[1 - src];
        a.ev = d_geo;
        a.items = d_sweep_items[axis];
        a.nitems = (int)sweep_items[axis].size();
        a.axis = axis;
        a.frac = frac;
        a.clk = clk;
        a.sc = scheme();
        a.rk = rk;
        a.threads = shape[axis].threads;
        a.blocks = a.nitems;
        a.counter = d_work_counter;      // batches: persistent grid, items from a counter
        a.rate_clk = rate_clk;
        a.sms = sms;
        a.stream = stream;
        a.charge = nq == 5;
        if (prec == HYDRO_FP64) return launch_sweep_f64(a);
        if (prec == HYDRO_FP32) return launch_sweep_f32(a);
        return launch_sweep_mixed(a);
    }

    // time candidate launch shapes for one axis (reads the current state,
    // writes the spare buffer; the state is unchanged).  Every candidate runs
    // once untimed first (clocks and caches settle), then each is timed in two
    // passes over the list and keeps its faster pass, so a clock ramp during
    // tuning does not favour the candidates timed last.
    // the staged x sweep (RK2) holds shared-memory rows per warp: the block
    // sizes whose rings fit the per-block limit
    int staged_max_threads(int axis) const {
        if (axis != 0 || rk != 2 || unsplit) return 256;
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
                cudaSuccess)
            return 128;
        const long long per_warp = (long long)nq * 32 * XSTAGE_STEPS_PER_ROW * (long long)elem;
        return (int)std::min<long long>(256, 32 * (optin / per_warp));
    }

    hydro_status tune(int axis) {
        if (forced[axis] || tuned[axis]) return HYDRO_OK;
        int maxN = 1;
        for (const EventGeo &g : geo) maxN = std::max(maxN, g.n[axis]);
        std::vector<LaunchShape> cand;
        for (int th : {64, 128, 256}) {
            if (th > staged_max_threads(axis)) continue;
            LaunchShape s;
            s.threads = th;
            s.seg_len = 0;
            cand.push_back(s);
            for (int L : {256, 128, 64, 32, 16})
                if (L < maxN) {
                    s.seg_len = L;
                    cand.push_back(s);
                }
        }
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        std::vector<float> best(cand.size(), 1e30f);
        for (int pass = 0; pass < 3; ++pass)
            for (size_t c = 0; c < cand.size(); ++c) {
                hydro_status st = build_sweep_items(axis, cand[c]);
                if (st != HYDRO_OK) return st;
                if (pass == 0) {
                    CK(sweep_launch(axis, 1.0, d_clk_tune, cur));
                    continue;
                }
                CK(cudaEventRecord(e0, stream));
                CK(sweep_launch(axis, 1.0, d_clk_tune, cur));
                CK(sweep_launch(axis, 1.0, d_clk_tune, cur));
                CK(cudaEventRecord(e1, stream));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                best[c] = std::min(best[c], ms);
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        size_t bi = 0;
        for (size_t c = 1; c < cand.size(); ++c)
            if (best[c] < best[bi]) bi = c;
        tuned[axis] = true;
        return build_sweep_items(axis, cand[bi]);
    }

    hydro_status ensure_ready() {
        for (int a = 0; a < 3; ++a) {
            if (!active[a]) continue;
            if (sweep_items[a].empty()) {
                hydro_status s = build_sweep_items(a, shape[a]);
                if (s != HYDRO_OK) return s;
            }
            if (unsplit) continue;   // the unsplit scheme launches no sweeps
            hydro_status s = tune(a);
            if (s != HYDRO_OK) return s;
        }
        return HYDRO_OK;
    }

    // ---------------------------------------------------------------- timing
    cudaError_t mark_begin(int kind, size_t &slot) {
        if (!timing) return cudaSuccess;
        slot = ev_used++;
        while (ev_pool.size() < 2 * ev_used) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            ev_pool.push_back(e);
        }
        if (ev_kind.size() < ev_used) ev_kind.resize(ev_used);
        ev_kind[slot] = kind;
        return cudaEventRecord(ev_pool[2 * slot], stream);
    }
    cudaError_t mark_end(size_t slot) {
        if (!timing) return cudaSuccess;
        return cudaEventRecord(ev_pool[2 * slot + 1], stream);
    }
    hydro_status collect_timing() {
        if (ev_used == 0) return HYDRO_OK;
        CK(cudaStreamSynchronize(stream));
        for (size_t i = 0; i < ev_used; ++i) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev_pool[2 * i], ev_pool[2 * i + 1]));
            timing_ms[ev_kind[i]] += ms;
            timing_n[ev_kind[i]] += 1;
        }
        ev_used = 0;
        return HYDRO_OK;
    }

    // ---------------------------------------------------------------- stepping
    // one full step: rate -> dt -> jet -> Strang sweeps (readings R7, R8, R12)
    cudaError_t enqueue_step() {
        cudaError_t err;
        CellLaunch c = cell_launch();
        size_t slot = 0;
        if ((err = mark_begin(1, slot)) != cudaSuccess) return err;
        const bool cfl_dt = !(fixed_dt > 0.0);
        if (cfl_dt && !rate_valid) {   // otherwise the previous step's last sweep left it
            if ((err = launch_rate(c, d_state[cur], d_clk, cfl)) != cudaSuccess) return err;
        }
        const double cf[2] = {cfl, fixed_dt};
        if ((err = launch_dt(d_clk, cf, nevents, stream)) != cudaSuccess) return err;
        if (any_jet && (err = launch_jet(c, d_state[cur], d_clk)) != cudaSuccess) return err;
        if ((err = mark_end(slot)) != cudaSuccess) return err;
        if (unsplit) {
            bool any = active[0] || active[1] || active[2];
            if (any && (err = enqueue_unsplit(cfl_dt)) != cudaSuccess) return err;
            rate_valid = cfl_dt && any;
            return cudaSuccess;
        }
        int act[3], na = 0;
        for (int a = 0; a < 3; ++a)
            if (active[a]) act[na++] = a;
        if (na == 0) return cudaSuccess;
        auto sw = [&](int a, double frac, bool last) {
            size_t sl = 0;
            cudaError_t e = mark_begin(0, sl);
            if (e != cudaSuccess) return e;
            e = sweep_launch(a, frac, d_clk, cur, (last && cfl_dt) ? d_clk : nullptr);
            cur = 1 - cur;
            if (e != cudaSuccess) return e;
            return mark_end(sl);
        };
        for (int k = 0; k < na - 1; ++k)
            if ((err = sw(act[k], 0.5, false)) != cudaSuccess) return err;
        if ((err = sw(act[na - 1], 1.0, na == 1)) != cudaSuccess) return err;
        for (int k = na - 2; k >= 0; --k)
            if ((err = sw(act[k], 0.5, k == 0)) != cudaSuccess) return err;
        rate_valid = cfl_dt;
        return cudaSuccess;
    }

    hydro_status set_t_end(double t_end) {
        if (t_end == t_end_dev) return HYDRO_OK;
        std::vector<EventClock> clk(nevents);
        CK(cudaMemcpyAsync(clk.data(), d_clk, nevents * sizeof(EventClock),
                           cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        for (auto &c : clk) c.t_end = t_end;
        CK(cudaMemcpyAsync(d_clk, clk.data(), nevents * sizeof(EventClock),
                           cudaMemcpyHostToDevice, stream));
        CK(cudaStreamSynchronize(stream));
        t_end_dev = t_end;
        return HYDRO_OK;
    }

    hydro_status build_graph() {
        const int p = cur;
        if (graph[p]) cudaGraphExecDestroy(graph[p]);
        graph[p] = nullptr;
        graph_ok[p] = false;
        const int cur0 = cur;
        const bool rv0 = rate_valid;
        cudaGraph_t gr;
        CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t err = enqueue_step();
        if (err == cudaSuccess) err = enqueue_step();
        cudaError_t err2 = cudaStreamEndCapture(stream, &gr);
        cur = cur0;   // capture does not run anything
        rate_valid = rv0;
        if (err != cudaSuccess) return fail(HYDRO_E_CUDA, std::string("capture: ") + cudaGetErrorString(err));
        if (err2 != cudaSuccess) return fail(HYDRO_E_CUDA, std::string("end capture: ") + cudaGetErrorString(err2));
        err = cudaGraphInstantiate(&graph[p], gr, 0);
        cudaGraphDestroy(gr);
        if (err != cudaSuccess) return fail(HYDRO_E_CUDA, std::string("instantiate: ") + cudaGetErrorString(err));
        graph_ok[p] = true;
        return HYDRO_OK;
    }

    hydro_status step(int nsteps, double t_end, bool use_graph, double *t_out) {
        if (nsteps < 0) return fail(HYDRO_E_INVALID, "nsteps < 0");
        hydro_status s = ensure_ready();
        if (s != HYDRO_OK) return s;
        s = set_t_end(t_end > 0.0 ? t_end : 0.0);
        if (s != HYDRO_OK) return s;
        int done = 0;
        const int check_every = 64;
        while (done < nsteps) {
            int chunk = std::min(nsteps - done, t_end > 0.0 ? check_every : nsteps - done);
            int k = 0;
            if (!rate_valid && !(fixed_dt > 0.0) && chunk >= 1) {   // first step computes the rate
                CK(enqueue_step());
                ++k;
            }
            if (use_graph && !timing && chunk - k >= 2) {
                if (graph_dirty) {
                    graph_ok[0] = graph_ok[1] = false;
                    graph_dirty = false;
                }
                if (!graph_ok[cur]) {
                    s = build_graph();
                    if (s != HYDRO_OK) return s;
                }
                for (; k + 2 <= chunk; k += 2) CK(cudaGraphLaunch(graph[cur], stream));
            }
            for (; k < chunk; ++k) CK(enqueue_step());
            done += chunk;
            if (timing) {
                hydro_status ts = collect_timing();
                if (ts != HYDRO_OK) return ts;
            }
            if (t_end > 0.0 && done < nsteps) {
                double t;
                CK(cudaMemcpyAsync(&t, &d_clk[0].t, sizeof(double), cudaMemcpyDeviceToHost, stream));
                CK(cudaStreamSynchronize(stream));
                if (nevents == 1 && t >= t_end) break;
            }
        }
        if (t_out) {
            CK(cudaMemcpyAsync(t_out, &d_clk[0].t, sizeof(double), cudaMemcpyDeviceToHost, stream));
            CK(cudaStreamSynchronize(stream));
        }
        return HYDRO_OK;
    }

    // ---------------------------------------------------------------- data in / out
    void *event_ptr(int buf, int e) {
        return (char *)d_state[buf] + (size_t)geo[e].off * elem;
    }

    // pn: the rest-frame charge density (charged handles; null sets R = 0)
    hydro_status set_primitives(int e, const void *pe, const void *pvx, const void *pvy,
                                const void *pvz, int on_device, const void *pn = nullptr) {
        rate_valid = false;
        if (e < 0 || e >= nevents) return fail(HYDRO_E_INVALID, "bad event");
        if (!pe || !pvx || !pvy || !pvz) return fail(HYDRO_E_INVALID, "null pointer");
        if (pn && nq != 5) return fail(HYDRO_E_INVALID, "the handle carries no charge");
        const size_t fb = (size_t)geo[e].cells * elem;
        // stage the primitives in the spare buffer at this event's place
        char *stage = (char *)event_ptr(1 - cur, e);
        const void *src[5] = {pe, pvx, pvy, pvz, pn};
        const int nsrc = pn ? 5 : 4;
        for (int f = 0; f < nsrc; ++f)
            CK(cudaMemcpyAsync(stage + f * fb, src[f], fb,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream));
        CellLaunch c = cell_launch();
        std::vector<WorkItem> items;
        for (const WorkItem &w : cell_items)
            if (w.event == e) items.push_back(w);
        // the event's items are contiguous in cell_items
        size_t first = 0;
        while (cell_items[first].event != e) ++first;
        c.items = d_cell_items + first;
        c.nitems = (int)items.size();
        c.blocks = std::min(c.nitems, sms * 8);
        // prim2cons writes U at geo.off relative to the base; pass the event's
        // staged fields with the same offsets via base pointers
        const long long off = geo[e].off;
        const char *base = (const char *)d_state[1 - cur];
        // kernel indexes fields as ptr[c]; give it pointers shifted to the event
        CK(launch_prim2cons(c, base + (off + 0 * geo[e].cells) * elem - 0,
                            base + (off + 1 * geo[e].cells) * elem,
                            base + (off + 2 * geo[e].cells) * elem,
                            base + (off + 3 * geo[e].cells) * elem,
                            pn ? base + (off + 4 * geo[e].cells) * elem : nullptr, d_state[cur]));
        CK(cudaStreamSynchronize(stream));
        return reset_time(e);
    }

    hydro_status reset_time(int e) {
        EventClock c;
        CK(cudaMemcpy(&c, d_clk + e, sizeof c, cudaMemcpyDeviceToHost));
        c.t = 0.0;
        c.t_step = 0.0;
        c.dt = 0.0;
        c.status = 0;
        c.rate_bits = 0ull;
        CK(cudaMemcpy(d_clk + e, &c, sizeof c, cudaMemcpyHostToDevice));
        CK(cudaMemset(d_flags + e, 0, sizeof(unsigned)));
        return HYDRO_OK;
    }

    hydro_status set_conserved(int e, const void *U, int on_device) {
        rate_valid = false;
        if (e < 0 || e >= nevents || !U) return fail(HYDRO_E_INVALID, "bad argument");
        CK(cudaMemsetAsync(d_flags + e, 0, sizeof(unsigned), stream));
        CK(cudaMemcpyAsync(event_ptr(cur, e), U, (size_t)nq * geo[e].cells * elem,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream));
        CK(cudaStreamSynchronize(stream));
        return HYDRO_OK;
    }

    hydro_status get_conserved(int e, void *U, int on_device) {
        if (e < 0 || e >= nevents || !U) return fail(HYDRO_E_INVALID, "bad argument");
        CK(cudaMemcpyAsync(U, event_ptr(cur, e), (size_t)nq * geo[e].cells * elem,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        return HYDRO_OK;
    }

    hydro_status get_primitives(int e, void *pe, void *pvx, void *pvy, void *pvz, int on_device) {
        if (e < 0 || e >= nevents) return fail(HYDRO_E_INVALID, "bad event");
        if (!pe || !pvx || !pvy || !pvz) return fail(HYDRO_E_INVALID, "null pointer");
        size_t first = 0;
        while (cell_items[first].event != e) ++first;
        size_t last = first;
        while (last < cell_items.size() && cell_items[last].event == e) ++last;
        CellLaunch c = cell_launch();
        c.items = d_cell_items + first;
        c.nitems = (int)(last - first);
        c.blocks = std::min(c.nitems, sms * 8);
        const size_t fb = (size_t)geo[e].cells * elem;
        char *stage = (char *)event_ptr(1 - cur, e);
        // outputs indexed by cell within the event: shift by -off so the
        // kernel's U + off + c addressing lines up
        CK(launch_cons2prim(c, d_state[cur], stage, stage + fb, stage + 2 * fb, stage + 3 * fb));
        void *dst[4] = {pe, pvx, pvy, pvz};
        for (int f = 0; f < 4; ++f)
            CK(cudaMemcpyAsync(dst[f], stage + f * fb, fb,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        return HYDRO_OK;
    }

    // per event: out[event][4] the energy-momentum sums, charge[event] (may be
    // null) the charge sum of a charged handle
    hydro_status sums(double *out, double *charge = nullptr) {
        if (charge && nq != 5) return fail(HYDRO_E_INVALID, "the handle carries no charge");
        CellLaunch c = cell_launch();
        c.items = d_sum_items;
        c.nitems = (int)sum_items.size();
        c.blocks = (int)std::min<size_t>(sum_items.size(), (size_t)sms * 8);
        CK(launch_sums(c, d_state[cur], d_partial));
        CK(launch_sums_final(d_sum_items, (int)sum_items.size(), d_partial, d_geo, d_sums,
                             nevents, nq, stream));
        std::vector<double> h((size_t)nevents * nq);
        CK(cudaMemcpyAsync(h.data(), d_sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                           stream));
        CK(cudaStreamSynchronize(stream));
        for (int e = 0; e < nevents; ++e) {
            if (out)
                for (int q = 0; q < 4; ++q) out[4 * e + q] = h[(size_t)nq * e + q];
            if (charge) charge[e] = h[(size_t)nq * e + 4];
        }
        return HYDRO_OK;
    }

    // n = R / gamma of event e into n (host or device), via the spare buffer
    hydro_status charge_density(int e, void *n, int on_device) {
        if (nq != 5) return fail(HYDRO_E_INVALID, "the handle carries no charge");
        if (e < 0 || e >= nevents || !n) return fail(HYDRO_E_INVALID, "bad argument");
        size_t first = 0;
        while (cell_items[first].event != e) ++first;
        size_t last = first;
        while (last < cell_items.size() && cell_items[last].event == e) ++last;
        CellLaunch c = cell_launch();
        c.items = d_cell_items + first;
        c.nitems = (int)(last - first);
        c.blocks = std::min(c.nitems, sms * 8);
        char *stage = (char *)event_ptr(1 - cur, e);
        CK(launch_charge_density(c, d_state[cur], stage));
        CK(cudaMemcpyAsync(n, stage, (size_t)geo[e].cells * elem,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        return HYDRO_OK;
    }

    hydro_status hotspots(const double *spots, int nspots, double sigma, double e_bg) {
        rate_valid = false;
        if (!spots || nspots < 0 || !(sigma > 0.0)) return fail(HYDRO_E_INVALID, "bad hot spots");
        double *d_spots = nullptr;
        const size_t bytes = (size_t)nevents * std::max(nspots, 1) * 7 * sizeof(double);
        CK(cudaMalloc(&d_spots, bytes));
        CK(cudaMemcpy(d_spots, spots, (size_t)nevents * nspots * 7 * sizeof(double),
                      cudaMemcpyHostToDevice));
        CellLaunch c = cell_launch();
        cudaError_t err = launch_hotspots(c, d_spots, nspots, sigma, e_bg, d_state[cur]);
        cudaError_t err2 = cudaStreamSynchronize(stream);
        cudaFree(d_spots);
        CK(err);
        CK(err2);
        for (int e = 0; e < nevents; ++e) {
            hydro_status s = reset_time(e);
            if (s != HYDRO_OK) return s;
        }
        return HYDRO_OK;
    }

    hydro_status set_jets(const double *jets) {
        if (!jets) return fail(HYDRO_E_INVALID, "null jets");
        for (int e = 0; e < nevents; ++e) {
            memcpy(geo[e].jet, jets + 8 * e, 8 * sizeof(double));
            geo[e].jet_on = 1;
            const double sig = geo[e].jet[7];
            if (!(sig > 0.0)) return fail(HYDRO_E_INVALID, "jet width must be > 0");
            // as k_jet: at most min(2 (ceil(9 sigma / h) + 1) + 1, n) cells per active axis
            long long box = 1;
            for (int a = 0; a < 3; ++a)
                if (geo[e].n[a] > 1)
                    box *= std::min<long long>(
                        2 * ((long long)std::ceil(9.0 * sig / geo[e].h[a]) + 1) + 1, geo[e].n[a]);
            jet_cells = std::max(jet_cells, box);
        }
        any_jet = true;
        graph_dirty = true;
        CK(cudaMemcpy(d_geo, geo.data(), nevents * sizeof(EventGeo), cudaMemcpyHostToDevice));
        return HYDRO_OK;
    }

    hydro_status max_rate(double *rate) {
        rate_valid = false;
        std::vector<EventClock> clk(nevents);
        CellLaunch c = cell_launch();
        CK(cudaMemcpyAsync(clk.data(), d_clk, nevents * sizeof(EventClock), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        for (auto &k : clk) k.rate_bits = 0ull;
        CK(cudaMemcpyAsync(d_clk, clk.data(), nevents * sizeof(EventClock), cudaMemcpyHostToDevice, stream));
        CK(launch_rate(c, d_state[cur], d_clk, cfl));
        CK(cudaMemcpyAsync(clk.data(), d_clk, nevents * sizeof(EventClock), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        for (int e = 0; e < nevents; ++e) {
            long long b = (long long)clk[e].rate_bits;
            double r;
            memcpy(&r, &b, sizeof r);
            rate[e] = r;
            clk[e].rate_bits = 0ull;
        }
        CK(cudaMemcpyAsync(d_clk, clk.data(), nevents * sizeof(EventClock), cudaMemcpyHostToDevice, stream));
        CK(cudaStreamSynchronize(stream));
        return HYDRO_OK;
    }

    hydro_status single_sweep(int axis, double dt) {
        rate_valid = false;
        if (axis < 0 || axis > 2) return fail(HYDRO_E_INVALID, "axis must be 0..2");
        if (!(dt > 0.0)) return fail(HYDRO_E_INVALID, "dt must be > 0");
        if (!active[axis]) return HYDRO_OK;
        hydro_status s = ensure_ready();
        if (s != HYDRO_OK) return s;
        std::vector<EventClock> clk(nevents);
        CK(cudaMemcpyAsync(clk.data(), d_clk, nevents * sizeof(EventClock), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        std::vector<EventClock> c2 = clk;
        for (auto &k : c2) k.dt = dt;
        CK(cudaMemcpyAsync(d_clk, c2.data(), nevents * sizeof(EventClock), cudaMemcpyHostToDevice, stream));
        CK(sweep_launch(axis, 1.0, d_clk, cur));
        cur = 1 - cur;
        CK(cudaMemcpyAsync(d_clk, clk.data(), nevents * sizeof(EventClock), cudaMemcpyHostToDevice, stream));
        CK(cudaStreamSynchronize(stream));
        graph_dirty = true;
        return HYDRO_OK;
    }

    hydro_status times(double *t) {
        std::vector<EventClock> clk(nevents);
        CK(cudaMemcpyAsync(clk.data(), d_clk, nevents * sizeof(EventClock), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        for (int e = 0; e < nevents; ++e) t[e] = clk[e].t;
        return HYDRO_OK;
    }

    hydro_status set_time(double t) {
        std::vector<EventClock> clk(nevents);
        CK(cudaMemcpy(clk.data(), d_clk, nevents * sizeof(EventClock), cudaMemcpyDeviceToHost));
        for (auto &k : clk) k.t = t;
        CK(cudaMemcpy(d_clk, clk.data(), nevents * sizeof(EventClock), cudaMemcpyHostToDevice));
        return HYDRO_OK;
    }

    // per event: HYDRO_E_NONFINITE if the state holds NaN or Inf, else
    // HYDRO_E_NEWTON if a Newton solve hit its cap, else HYDRO_E_UNPHYSICAL if
    // an inadmissible state was met and repaired, else HYDRO_OK; flags (may be
    // null) receives the raw FLAG_* words
    hydro_status status(int *st, unsigned *flags_out = nullptr) {
        CellLaunch c = cell_launch();
        CK(launch_finite(c, d_state[cur], d_clk));
        std::vector<EventClock> clk(nevents);
        std::vector<unsigned> fl(nevents);
        CK(cudaMemcpyAsync(clk.data(), d_clk, nevents * sizeof(EventClock), cudaMemcpyDeviceToHost, stream));
        CK(cudaMemcpyAsync(fl.data(), d_flags, nevents * sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        for (int e = 0; e < nevents; ++e) {
            int s = HYDRO_OK;
            if (clk[e].status == HYDRO_E_NONFINITE) s = HYDRO_E_NONFINITE;
            else if (fl[e] & FLAG_NEWTON) s = HYDRO_E_NEWTON;
            else if (fl[e] & FLAG_UNPHYSICAL) s = HYDRO_E_UNPHYSICAL;
            st[e] = s;
            if (flags_out) flags_out[e] = fl[e];
        }
        return HYDRO_OK;
    }

    hydro_status counters(long long *out) {
        unsigned long long h[NCOUNTERS];
        CK(cudaMemcpyAsync(h, d_counters, sizeof h, cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        for (int i = 0; i < NCOUNTERS; ++i) out[i] = (long long)h[i];
        return HYDRO_OK;
    }
};

}  // namespace

void hy::set_last_error(const char *msg) { g_err = msg; }

struct hydro_s {
    Solver s;
};
struct hydro_batch_s {
    Solver s;
};

extern "C" {

const char *hydro_last_error(void) { return g_err.c_str(); }

hydro_status hydro_create(const hydro_grid_t *grid, const hydro_eos_t *eos, int limiter,
                          int stages, hydro_t **out) {
    if (!out) return fail(HYDRO_E_INVALID, "out is null");
    *out = nullptr;
    hydro_t *h = new hydro_t;
    hydro_status st = h->s.init(grid, 1, eos, limiter, stages);
    if (st != HYDRO_OK) {
        delete h;
        return st;
    }
    *out = h;
    return HYDRO_OK;
}

void hydro_destroy(hydro_t *h) { delete h; }

hydro_status hydro_set_stream(hydro_t *h, void *stream) {
    if (!h) return fail(HYDRO_E_INVALID, "null handle");
    CK(cudaStreamSynchronize(h->s.stream));
    h->s.stream = stream ? (cudaStream_t)stream : h->s.own_stream;
    h->s.graph_dirty = true;
    return HYDRO_OK;
}

#define HANDLE(h) \
    if (!(h)) return fail(HYDRO_E_INVALID, "null handle")

hydro_status hydro_set_primitives(hydro_t *h, const void *e, const void *vx, const void *vy,
                                  const void *vz, int on_device) {
    HANDLE(h);
    return h->s.set_primitives(0, e, vx, vy, vz, on_device);
}
hydro_status hydro_set_primitives_charged(hydro_t *h, const void *e, const void *vx,
                                          const void *vy, const void *vz, const void *n,
                                          int on_device) {
    HANDLE(h);
    if (!n) return fail(HYDRO_E_INVALID, "null n");
    return h->s.set_primitives(0, e, vx, vy, vz, on_device, n);
}
hydro_status hydro_get_charge_density(hydro_t *h, void *n, int on_device) {
    HANDLE(h);
    return h->s.charge_density(0, n, on_device);
}
hydro_status hydro_charge_sum(hydro_t *h, double *out) {
    HANDLE(h);
    if (!out) return fail(HYDRO_E_INVALID, "null out");
    return h->s.sums(nullptr, out);
}
hydro_status hydro_set_conserved(hydro_t *h, const void *U, int on_device) {
    HANDLE(h);
    return h->s.set_conserved(0, U, on_device);
}
hydro_status hydro_get_conserved(hydro_t *h, void *U, int on_device) {
    HANDLE(h);
    return h->s.get_conserved(0, U, on_device);
}
hydro_status hydro_get_primitives(hydro_t *h, void *e, void *vx, void *vy, void *vz,
                                  int on_device) {
    HANDLE(h);
    return h->s.get_primitives(0, e, vx, vy, vz, on_device);
}
hydro_status hydro_init_hotspots(hydro_t *h, const double *spots, int nspots, double sigma,
                                 double e_bg) {
    HANDLE(h);
    return h->s.hotspots(spots, nspots, sigma, e_bg);
}
hydro_status hydro_set_jet(hydro_t *h, const double jet[8]) {
    HANDLE(h);
    return h->s.set_jets(jet);
}
hydro_status hydro_step(hydro_t *h, int nsteps, double t_end, double *t_out) {
    HANDLE(h);
    return h->s.step(nsteps, t_end, true, t_out);
}
hydro_status hydro_sweep(hydro_t *h, int axis, double dt) {
    HANDLE(h);
    return h->s.single_sweep(axis, dt);
}
hydro_status hydro_max_rate(hydro_t *h, double *rate) {
    HANDLE(h);
    if (!rate) return fail(HYDRO_E_INVALID, "null rate");
    return h->s.max_rate(rate);
}
hydro_status hydro_conservation_sums(hydro_t *h, double out[4]) {
    HANDLE(h);
    if (!out) return fail(HYDRO_E_INVALID, "null out");
    return h->s.sums(out);
}
hydro_status hydro_get_time(hydro_t *h, double *t) {
    HANDLE(h);
    if (!t) return fail(HYDRO_E_INVALID, "null t");
    return h->s.times(t);
}
hydro_status hydro_set_time(hydro_t *h, double t) {
    HANDLE(h);
    return h->s.set_time(t);
}
hydro_status hydro_enable_counters(hydro_t *h, int on) {
    HANDLE(h);
    h->s.counters_on = on != 0;
    h->s.graph_dirty = true;
    return HYDRO_OK;
}
hydro_status hydro_counters(hydro_t *h, long long out[6]) {
    HANDLE(h);
    if (!out) return fail(HYDRO_E_INVALID, "null out");
    return h->s.counters(out);
}
hydro_status hydro_check_finite(hydro_t *h) {
    HANDLE(h);
    int st = 0;
    hydro_status s = h->s.status(&st);
    if (s != HYDRO_OK) return s;
    if (st == HYDRO_E_NONFINITE) return fail(HYDRO_E_NONFINITE, "state holds NaN or Inf");
    return HYDRO_OK;
}
hydro_status hydro_check_status(hydro_t *h, unsigned *flags) {
    HANDLE(h);
    int st = 0;
    unsigned fl = 0;
    hydro_status s = h->s.status(&st, &fl);
    if (s != HYDRO_OK) return s;
    if (flags) *flags = fl;
    switch (st) {
    case HYDRO_E_NONFINITE: return fail(HYDRO_E_NONFINITE, "state holds NaN or Inf");
    case HYDRO_E_NEWTON:
        return fail(HYDRO_E_NEWTON, "a Newton cons->prim solve hit its iteration cap");
    case HYDRO_E_UNPHYSICAL:
        return fail(HYDRO_E_UNPHYSICAL,
                    "an inadmissible state (|M| >= (1 - delta) E) was met and repaired");
    default: return HYDRO_OK;
    }
}
static hydro_status get_timing(Solver &s, double *ms, long long *n) {
    if (!ms || !n) return fail(HYDRO_E_INVALID, "null output");
    hydro_status st = s.collect_timing();
    if (st != HYDRO_OK) return st;
    for (int k = 0; k < 2; ++k) {
        ms[k] = s.timing_ms[k];
        n[k] = s.timing_n[k];
        s.timing_ms[k] = 0.0;
        s.timing_n[k] = 0;
    }
    return HYDRO_OK;
}
hydro_status hydro_set_kernel_timing(hydro_t *h, int on) {
    HANDLE(h);
    h->s.timing = on != 0;
    return HYDRO_OK;
}
hydro_status hydro_get_kernel_timing(hydro_t *h, double out_ms[2], long long counts[2]) {
    HANDLE(h);
    return get_timing(h->s, out_ms, counts);
}
hydro_status hydro_batch_set_kernel_timing(hydro_batch_t *b, int on) {
    HANDLE(b);
    b->s.timing = on != 0;
    return HYDRO_OK;
}
hydro_status hydro_batch_get_kernel_timing(hydro_batch_t *b, double out_ms[2], long long counts[2]) {
    HANDLE(b);
    return get_timing(b->s, out_ms, counts);
}
hydro_status hydro_force_launch(hydro_t *h, int axis, int threads, int segments) {
    HANDLE(h);
    if (axis < 0 || axis > 2) return fail(HYDRO_E_INVALID, "axis must be 0..2");
    Solver &s = h->s;
    if (threads == 0) {
        s.forced[axis] = false;
        s.tuned[axis] = false;
        return HYDRO_OK;
    }
    if (threads < 32 || threads > 256 || threads % 32) return fail(HYDRO_E_INVALID, "threads must be 32..256, multiple of 32");
    if (threads > s.staged_max_threads(axis))
        return fail(HYDRO_E_INVALID, "the staged x sweep of this handle fits at most " +
                                         std::to_string(s.staged_max_threads(axis)) +
                                         " threads per block");
    if (segments < 1) return fail(HYDRO_E_INVALID, "segments must be >= 1");
    LaunchShape sh;
    sh.threads = threads;
    const int N = s.geo[0].n[axis];
    sh.seg_len = segments <= 1 ? 0 : (N + segments - 1) / segments;
    s.forced[axis] = true;
    return s.build_sweep_items(axis, sh);
}
hydro_status hydro_get_launch(hydro_t *h, int axis, int *threads, int *segments) {
    HANDLE(h);
    if (axis < 0 || axis > 2 || !threads || !segments) return fail(HYDRO_E_INVALID, "bad argument");
    hydro_status st = h->s.ensure_ready();
    if (st != HYDRO_OK) return st;
    *threads = h->s.shape[axis].threads;
    *segments = h->s.geo[0].seg[axis];
    return HYDRO_OK;
}
hydro_status hydro_mlp_seed_emin(hydro_t *h, double *emin) {
    HANDLE(h);
    if (!emin) return fail(HYDRO_E_INVALID, "null emin");
    if (h->s.sc.eos_kind != HYDRO_EOS_TABLE) return fail(HYDRO_E_INVALID, "needs a table EOS");
    *emin = h->s.sc.c64.mlp_emin;
    return HYDRO_OK;
}
hydro_status hydro_c2p_newton(hydro_t *h, const void *U, int n, int seed, void *vmag, int *iters) {
    HANDLE(h);
    if (n == 0) return HYDRO_OK;
    if (!U || !vmag || !iters || n < 0) return fail(HYDRO_E_INVALID, "bad argument");
    if (h->s.sc.eos_kind != HYDRO_EOS_TABLE) return fail(HYDRO_E_INVALID, "needs a table EOS");
    if (seed < 0 || seed > 2) return fail(HYDRO_E_INVALID, "unknown seed");
    if (seed == HYDRO_SEED_MLP && !h->s.sc.mlp_f) return fail(HYDRO_E_INVALID, "no MLP parameters");
    CK(launch_c2p_newton(h->s.prec == HYDRO_FP64 ? 0 : 1, h->s.scheme(), U, n, seed, vmag, iters,
                         h->s.stream));
    CK(cudaStreamSynchronize(h->s.stream));
    return HYDRO_OK;
}
hydro_status hydro_c2p_newton_pairs(hydro_t *h, const void *U, int n, int seed, int rcp,
                                    void *vmag, void *p, int *iters) {
    HANDLE(h);
    if (n == 0) return HYDRO_OK;
    if (!U || !vmag || !p || !iters || n < 0 || n % 2)
        return fail(HYDRO_E_INVALID, "bad argument (n must be even)");
    if (h->s.sc.eos_kind != HYDRO_EOS_TABLE) return fail(HYDRO_E_INVALID, "needs a table EOS");
    if (seed != HYDRO_SEED_ZERO && seed != HYDRO_SEED_CONFORMAL)
        return fail(HYDRO_E_INVALID, "seed must be zero or conformal");
    CK(launch_c2p_newton_pairs(h->s.prec == HYDRO_FP64 ? 0 : 1, h->s.scheme(), U, n, seed,
                               rcp ? 1 : 0, vmag, p, iters, h->s.stream));
    CK(cudaStreamSynchronize(h->s.stream));
    return HYDRO_OK;
}

// ---------------------------------------------------------------- batch
hydro_status hydro_batch_create(const hydro_grid_t *grids, int nevents, const hydro_eos_t *eos,
                                int limiter, int stages, hydro_batch_t **out) {
    if (!out) return fail(HYDRO_E_INVALID, "out is null");
    *out = nullptr;
    hydro_batch_t *b = new hydro_batch_t;
    hydro_status st = b->s.init(grids, nevents, eos, limiter, stages);
    if (st != HYDRO_OK) {
        delete b;
        return st;
    }
    *out = b;
    return HYDRO_OK;
}
void hydro_batch_destroy(hydro_batch_t *b) { delete b; }
hydro_status hydro_batch_set_stream(hydro_batch_t *b, void *stream) {
    HANDLE(b);
    CK(cudaStreamSynchronize(b->s.stream));
    b->s.stream = stream ? (cudaStream_t)stream : b->s.own_stream;
    b->s.graph_dirty = true;
    return HYDRO_OK;
}
hydro_status hydro_batch_init_hotspots(hydro_batch_t *b, const double *spots, int nspots,
                                       double sigma, double e_bg) {
    HANDLE(b);
    return b->s.hotspots(spots, nspots, sigma, e_bg);
}
hydro_status hydro_batch_set_primitives(hydro_batch_t *b, int event, const void *e,
                                        const void *vx, const void *vy, const void *vz,
                                        int on_device) {
    HANDLE(b);
    return b->s.set_primitives(event, e, vx, vy, vz, on_device);
}
hydro_status hydro_batch_set_primitives_charged(hydro_batch_t *b, int event, const void *e,
                                                const void *vx, const void *vy, const void *vz,
                                                const void *n, int on_device) {
    HANDLE(b);
    if (!n) return fail(HYDRO_E_INVALID, "null n");
    return b->s.set_primitives(event, e, vx, vy, vz, on_device, n);
}
hydro_status hydro_batch_charge_sums(hydro_batch_t *b, double *out) {
    HANDLE(b);
    if (!out) return fail(HYDRO_E_INVALID, "null out");
    return b->s.sums(nullptr, out);
}
hydro_status hydro_batch_set_jets(hydro_batch_t *b, const double *jets) {
    HANDLE(b);
    return b->s.set_jets(jets);
}
hydro_status hydro_batch_step(hydro_batch_t *b, int nsteps, int use_graph) {
    HANDLE(b);
    return b->s.step(nsteps, 0.0, use_graph != 0, nullptr);
}
hydro_status hydro_batch_set_conserved(hydro_batch_t *b, int event, const void *U, int on_device) {
    HANDLE(b);
    return b->s.set_conserved(event, U, on_device);
}
hydro_status hydro_batch_get_conserved(hydro_batch_t *b, int event, void *U, int on_device) {
    HANDLE(b);
    return b->s.get_conserved(event, U, on_device);
}
hydro_status hydro_batch_get_primitives(hydro_batch_t *b, int event, void *e, void *vx,
                                        void *vy, void *vz, int on_device) {
    HANDLE(b);
    return b->s.get_primitives(event, e, vx, vy, vz, on_device);
}
hydro_status hydro_batch_times(hydro_batch_t *b, double *times) {
    HANDLE(b);
    if (!times) return fail(HYDRO_E_INVALID, "null times");
    return b->s.times(times);
}
hydro_status hydro_batch_conservation_sums(hydro_batch_t *b, double *out) {
    HANDLE(b);
    if (!out) return fail(HYDRO_E_INVALID, "null out");
    return b->s.sums(out);
}
hydro_status hydro_batch_event_status(hydro_batch_t *b, int *status) {
    HANDLE(b);
    if (!status) return fail(HYDRO_E_INVALID, "null status");
    return b->s.status(status);
}
hydro_status hydro_batch_event_flags(hydro_batch_t *b, int *status, unsigned *flags) {
    HANDLE(b);
    if (!status || !flags) return fail(HYDRO_E_INVALID, "null output");
    return b->s.status(status, flags);
}
hydro_status hydro_batch_enable_counters(hydro_batch_t *b, int on) {
    HANDLE(b);
    b->s.counters_on = on != 0;
    b->s.graph_dirty = true;
    return HYDRO_OK;
}
hydro_status hydro_batch_counters(hydro_batch_t *b, long long out[6]) {
    HANDLE(b);
    if (!out) return fail(HYDRO_E_INVALID, "null out");
    return b->s.counters(out);
}

// ---------------------------------------------------------------- MLP
int hydro_mlp_nparam(void) { return MLP_NPARAM; }

hydro_status hydro_mlp_forward(const float *params, const float *X, int n, float *out,
                               void *stream) {
    if (n == 0) return HYDRO_OK;
    if (!params || !X || !out || n < 0) return fail(HYDRO_E_INVALID, "bad argument");
    CK(launch_mlp_forward(params, X, n, out, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return HYDRO_OK;
}

hydro_status hydro_mlp_hidden(const float *params, const float *X, int n, float *H1,
                              void *stream) {
    if (n == 0) return HYDRO_OK;
    if (!params || !X || !H1 || n < 0) return fail(HYDRO_E_INVALID, "bad argument");
    CK(launch_mlp_hidden(params, X, n, H1, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return HYDRO_OK;
}

hydro_status hydro_mlp_loss_grad(const float *params, const float *X, const float *Y, int n,
                                 float *grad, float *loss, void *stream) {
    if (!params || !X || !Y || !grad || !loss || n < 1) return fail(HYDRO_E_INVALID, "bad argument");
    CK(launch_mlp_loss_grad(params, X, Y, n, grad, loss, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return HYDRO_OK;
}

}  // extern "C"
