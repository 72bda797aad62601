// Host runtime and C ABI of the batched cable-equation stepper (declarations in include/arb.h).
//
// arb_create does all preparation on the host (no CUDA call):
//   1. per-CV geometry of the finite-volume discretisation (Sec. "Model", Eq. discrete-v);
//   2. the implicit-Euler matrix of Sec. "Model" and its Hines factorisation, once: with fixed
//      dt and all membrane current on the right-hand side it never changes;
//   3. the packing of cells into warp programs ("packs") and the solve schedule of each pack.
// arb_bind_workspace uploads it into the caller's device buffer; arb_advance replays one
// captured CUDA graph per epoch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <array>
#include <functional>
#include <memory>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <queue>
#include <unordered_map>
#include <string>
#include <thread>
#include <vector>

#include <stdlib.h>
#include <sys/mman.h>

#include "../../include/arb.h"
#include "arb_internal.h"

namespace arbk {
template <class MT>
cudaError_t launch_epoch(const DevModel<MT>& d, bool implicit, int grid, int warps_per_cta, int tile_doubles, cudaStream_t s);
template <class MT>
cudaError_t epoch_occupancy(bool implicit, int warps_per_cta, int tile_doubles, int* blocks_per_sm);
template <class MT>
cudaError_t launch_stream(const DevModel<MT>& d, int mode, int v, int grid, int warps_per_cta, int warp_smem_double2,
                          cudaStream_t s);
int stream_variant_count();
void stream_variant_info(int v, int* warps, int* rf, int* rb);
void stream_variant_shape(bool ring_path, int v, int warp_smem_double2, int* warps, int* per_warp_double2);
template <class MT>
cudaError_t stream_occupancy(int mode, int v, int warps_per_cta, int warp_smem_double2, int* blocks_per_sm);
cudaError_t launch_events_pre(const EvArgs& a, int n_sm, cudaStream_t s);
cudaError_t events_prepare();
cudaError_t launch_events_post(const SpkArgs& a, int n_sm, cudaStream_t s);
cudaError_t launch_int_begin(Ctl* c, int32_t epoch_steps, cudaStream_t s);
cudaError_t launch_int_end(Ctl* c, int64_t spike_cap, cudaStream_t s);
template <class T>
cudaError_t launch_gather(double* out, const T* src, const int64_t* idx, int64_t n, cudaStream_t s);
template <class T>
cudaError_t launch_scatter(T* dst, const double* src, const int64_t* idx, int64_t n, cudaStream_t s);
cudaError_t launch_adj_forward(const AdjArgs& a, int64_t s0, int64_t s1, int mode, int buf, cudaStream_t s);
cudaError_t launch_adj_stage(const AdjArgs& a, int64_t r0, int64_t r1, int rbuf, int64_t f0, int64_t f1,
                             cudaStream_t s);
cudaError_t launch_adj_reduce(const AdjArgs& a, cudaStream_t s);
cudaError_t adj_prepare(const AdjArgs& a);
size_t adj_smem_bytes(const AdjArgs& a);

}  // namespace arbk

using namespace arbk;

namespace {

constexpr double kPi = 3.14159265358979323846;
#ifdef ARB_DEBUG
constexpr int kCanaryBytes = 256;
constexpr unsigned char kCanaryByte = 0xA5;
#endif
constexpr int kGraphRing = 4;

struct ExtEvent {
    int64_t step;
    double t;
    double w;
    int32_t syn;
    int32_t idx;
};

// Allocator that leaves trivially constructible elements uninitialised, so that the large host
// arrays of a plan can be filled by several threads (the first touch of their pages then runs
// in parallel).
template <class T>
struct UninitAlloc : std::allocator<T> {
    template <class U>
    struct rebind { using other = UninitAlloc<U>; };
    UninitAlloc() = default;
    template <class U>
    UninitAlloc(const UninitAlloc<U>&) {}
    // Blocks of 8 MB and more are 2 MB aligned and marked for transparent huge pages: the plan's
    // arrays (tens of millions of entries) are first touched by many threads at once, and 4 KB
    // page faults taken in parallel contend in the kernel.
    static constexpr size_t kHuge = (size_t)2 << 20;
    T* allocate(size_t n) {
        const size_t bytes = n * sizeof(T);
        if (bytes < 4 * kHuge) return std::allocator<T>::allocate(n);
        void* q = nullptr;
        if (posix_memalign(&q, kHuge, (bytes + kHuge - 1) / kHuge * kHuge) != 0) throw std::bad_alloc();
        madvise(q, (bytes + kHuge - 1) / kHuge * kHuge, MADV_HUGEPAGE);   // advice only: failure is harmless
        return static_cast<T*>(q);
    }
    void deallocate(T* q, size_t n) {
        if (n * sizeof(T) < 4 * kHuge) std::allocator<T>::deallocate(q, n);
        else free(q);
    }
    template <class U>
    void construct(U* p) noexcept { ::new ((void*)p) U; }
    template <class U, class... A>
    void construct(U* p, A&&... a) { ::new ((void*)p) U(std::forward<A>(a)...); }
};
template <class T>
using hvec = std::vector<T, UninitAlloc<T>>;

struct Plan {
    std::vector<PackDesc> packs;
    int64_t total_rows = 0;
    hvec<double> ca, cb, ck, ce;            // total_rows*32
    hvec<int32_t> pslot;
    hvec<int32_t> vmap;                     // on-chip voltage slots (own | parent << 16)
    hvec<double> V0;                        // initial voltage per tile entry
    hvec<int64_t> cv_tile;                  // model CV -> global tile index
    hvec<int32_t> cv_pack;                  // model CV -> pack
    // synapses
    int64_t syn_rows = 0;
    std::vector<int32_t> syn_slot, syn_vs;
    std::vector<double> syn_e, syn_decay, syn_sc, syn_ntau;
    std::vector<int64_t> syn_entry;         // model synapse -> entry
    std::vector<int32_t> syn_owner, syn_js;
    // HH
    int64_t hh_rows = 0;
    std::vector<int32_t> hh_slot, hh_vs;
    std::vector<double> hh_sc, hh_gna, hh_gk;
    std::vector<int64_t> hh_entry;
    // clamps
    int64_t st_rows = 0;
    std::vector<int32_t> st_slot;
    std::vector<double> st_sc, st_on, st_off, st_amp;
    // detectors
    std::vector<int32_t> det_slot, det_gid;
    int64_t sg_total = 0;                   // doubles of global S scratch
    int64_t smem_packs = 0;
    double lane_eff = 0.0;
    int tile_doubles = 0;                   // per-warp shared tile (doubles), 0 = none
    int cells_per_pack = 0;
    bool stream = false;                    // packs streamed from global memory (one cell per lane)
    int64_t c_total = 0;                    // streamed packs: compact mechanism slots
    std::vector<double> cE, cB;             // streamed packs: ce, cb of each compact slot
    std::vector<int32_t> slot_lo, slot_hi;  // exact event times: each lane's range of compact slots
    int32_t stack_depth = 1;                // streamed packs: deepest hand-over stack
    int64_t warp_smem = 32;                 // streamed packs: shared memory per warp (double2)
    int64_t split_cvs = -1;                 // streamed packs: cells above this size are spread
    int64_t spread_rows = -1;               // streamed packs: target rows of a pack of spread cells
    bool stream_imp = false;                // streamed packs on the row-ring path (implicit, step-start events)
    hvec<int32_t> cpos;                     // row-ring path: per entry, its position among its row's slots
    hvec<int32_t> row_cs, row_cn;           // row-ring path: per row, its compact slot ranges
    std::vector<int32_t> mb_ent, mb_cs;     // per mailbox slot: its parent's entry in the pack, and
                                            // that entry's compact mechanism slot (-1 none)
};

struct Region {
    size_t off = 0, bytes = 0;
};

}  // namespace

struct arb_sim {
    // ---- settings and model copy
    arb_params prm{};
    int32_t n_cells = 0;
    int64_t n_cv = 0;
    std::vector<int64_t> cv_offset;
    hvec<int32_t> parent;
    hvec<double> length, radius, cm, Ra;
    hvec<int64_t> hh_cv, pas_cv, syn_cv, st_cv, det_cv;
    hvec<double> gnabar, gkbar, gl, g_pas, e_pas, syn_tau, syn_e, st_on, st_dur, st_amp;
    // synapse state units: one per synapse, or per (CV, tau, e) group when coalescing
    bool coalesce = false;
    bool exact = false;                     // steps cut at event times
    bool overlap = false;                   // exchange overlapped with the next epoch
    int64_t dry_ranks = 1;                  // virtual ranks of a dry run (1: a plain run)
    std::vector<int32_t> syn_unit;          // model synapse -> unit
    std::vector<int64_t> u_cv;
    std::vector<double> u_tau, u_e;
    std::vector<int32_t> u_rep;             // lowest-index synapse of the unit
    double threshold = -10.0;
    std::vector<int32_t> conn_src;
    std::vector<int64_t> conn_dst;
    std::vector<double> conn_delay, conn_w;
    int32_t epoch_steps = 0;
    bool mixed = false;
    bool implicit = true;
    std::vector<int64_t> syn_cell;
    // ---- prepared data
    Plan plan;
    std::vector<double> init_m, init_h, init_n;   // HH initial gates, model order
    hvec<double> hh_tab;                          // tabulated gate update (FP64 mechanisms)
    hvec<float> hh_tab_f;                         // the same in float (FP32 mechanisms)
    // connections grouped by source
    std::vector<int64_t> out_ptr;
    std::vector<int32_t> out_syn, out_idx;
    std::vector<double> out_delay, out_w;
    // ---- device
    bool bound = false;
    char* ws = nullptr;
    int64_t ws_bytes = 0;
    std::vector<std::pair<std::string, Region>> regions;
    std::shared_ptr<void> adj_plan;         // the adjoint's solve schedule (ChainPlan), built on first use:
                                            // it depends only on the model and dt, fixed for the handle
    int n_sm = 148;
    int variant = 0;                // compiled variant of the streamed kernel (row-ring path)
    int warps_per_cta = 2;
    int grid = 148;
    cudaStream_t s = nullptr;       // library stream (graphs are captured here)
    cudaStream_t s2 = nullptr;      // exchange stream of the overlapped schedule
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_main = nullptr, ev_side = nullptr;   // hand-offs between the two streams
    cudaGraphExec_t graph[6] = {};   // per epoch: delivery lists, epoch kernel, spike walk; the
                                     // overlapped schedule adds the epoch kernel on list buffer 1
                                     // and the integration's begin / end kernels
    int64_t int_count = 0;           // epochs integrated: the overlapped schedule alternates buffers
    cudaEvent_t t0[kGraphRing] = {}, t1[kGraphRing] = {};
    bool pending_time[kGraphRing] = {};
    DevModel<double> dm64{};
    DevModel<float> dm32{};
    EvArgs ev_args{};
    SpkArgs spk_args{};
    Ctl* ctl = nullptr;
    // host mirrors
    int64_t k = 0;
    std::vector<ExtEvent> ext;          // external events not yet known to be consumed
    bool ext_dirty = false;
    int64_t ext_counter = 0;
    int64_t n_probe = 0;
    double* trace = nullptr;
    std::vector<int32_t> probe_slot, probe_col;
    double last_epoch_ms = 0.0;
    int64_t last_launches = 0;
    int64_t graph_replays = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_error;   // errors of calls without a handle

// Which streamed kernel runs a streamed plan: 0 explicit scheme, 1 implicit row-ring path,
// 2 exact event times.
int stream_mode(const arb_sim* sim) { return sim->exact ? 2 : (sim->implicit ? 1 : 0); }

arb_status fail(arb_sim* s, arb_status st, const std::string& msg) {
    if (s) s->err = msg;
    return st;
}

#define CU(call)                                                                           \
    do {                                                                                   \
        cudaError_t e__ = (call);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return fail(sim, ARB_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Runs fn(i) for i in [0, n) on the host's hardware threads (contiguous chunks; fn must only
// write data owned by its index).
template <class F>
void parallel_for(int64_t n, F fn) {
    const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
    const int64_t nt = std::min<int64_t>(hw, std::max<int64_t>(1, n / 64));
    if (nt <= 1) {
        for (int64_t i = 0; i < n; ++i) fn(i);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(nt);
    for (int64_t t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            for (int64_t i = lo; i < hi; ++i) fn(i);
        });
    for (auto& x : th) x.join();
}

// Runs fn(t, nt) for t in [0, nt) on nt host threads, nt = min(hardware threads, max_tasks):
// for work split into a few large, balanced parts.
template <class F>
void run_tasks(int64_t max_tasks, F fn) {
    const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
    const int64_t nt = std::max<int64_t>(1, std::min(hw, max_tasks));
    if (nt == 1) {
        fn((int64_t)0, (int64_t)1);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(nt);
    for (int64_t t = 0; t < nt; ++t) th.emplace_back([&, t] { fn(t, nt); });
    for (auto& x : th) x.join();
}

// v = n copies of val, written in parallel.
template <class T, class A>
void par_assign(std::vector<T, A>& v, int64_t n, T val) {
    v.clear();
    v.resize((size_t)n);
    constexpr int64_t kChunk = 1 << 16;
    T* p = v.data();
    parallel_for((n + kChunk - 1) / kChunk, [&](int64_t c) {
        const int64_t lo = c * kChunk, hi = std::min<int64_t>(n, lo + kChunk);
        for (int64_t i = lo; i < hi; ++i) p[i] = val;
    });
}

// Steady state of the Hodgkin-Huxley gates at voltage v (classic rates, 1/ms).
void hh_steady(double v, double& m, double& h, double& n) {
    auto exr = [](double x) { return x == 0.0 ? 1.0 : x / std::expm1(x); };
    const double am = exr(-(v + 40.0) * 0.1), bm = 4.0 * std::exp(-(v + 65.0) / 18.0);
    const double ah = 0.07 * std::exp(-(v + 65.0) * 0.05), bh = 1.0 / (1.0 + std::exp(-(v + 35.0) * 0.1));
    const double an = 0.1 * exr(-(v + 55.0) * 0.1), bn = 0.125 * std::exp(-(v + 65.0) * 0.0125);
    m = am / (am + bm);
    h = ah / (ah + bh);
    n = an / (an + bn);
}

// The tabulated gate update (see kHHTabVlo): at every node V_i the six functions and their
// derivatives in V, from the rate formulas and their derivatives in long double; on each
// interval the cubic with those values and slopes at both ends (Hermite), whose error is
// h^4/384 max|f^(4)| (h = 1/256 mV: below 1e-17 for these functions), written as
// c0 + c1 s + c2 s^2 + c3 s^3 with s = (V - V_i)/h.
void build_hh_table(double dt, double* tab) {
    typedef long double LD;
    const int64_t nn = (int64_t)kHHTabN + 1;
    std::vector<LD> f((size_t)nn * 6), g((size_t)nn * 6);       // values, h * slopes
    const LD h = 1.0L / (LD)kHHTabPerMV;
    parallel_for(nn, [&](int64_t i) {
        const LD v = (LD)kHHTabVlo + (LD)i * h;
        // x / (e^x - 1) and its derivative; the Bernoulli series where |x| < 1e-3
        auto exr = [](LD x, LD& dx) {
            if (fabsl(x) < 1e-3L) {
                const LD x2 = x * x;
                dx = -0.5L + x / 6.0L - x * x2 / 180.0L;
                return 1.0L - x / 2.0L + x2 / 12.0L - x2 * x2 / 720.0L;
            }
            const LD em = expm1l(x);
            dx = (em - x * (em + 1.0L)) / (em * em);
            return x / em;
        };
        LD d1, d2;
        const LD am = exr(-(v + 40.0L) / 10.0L, d1), dam = -0.1L * d1;
        const LD bm = 4.0L * expl(-(v + 65.0L) / 18.0L), dbm = -bm / 18.0L;
        const LD ah = 0.07L * expl(-(v + 65.0L) / 20.0L), dah = -ah / 20.0L;
        const LD eh = expl(-(v + 35.0L) / 10.0L);
        const LD bh = 1.0L / (1.0L + eh), dbh = 0.1L * eh * bh * bh;
        const LD an = 0.1L * exr(-(v + 55.0L) / 10.0L, d2), dan = -0.01L * d2;
        const LD bn = 0.125L * expl(-(v + 65.0L) / 80.0L), dbn = -bn / 80.0L;
        const LD a[3] = {am, ah, an}, b[3] = {bm, bh, bn}, da[3] = {dam, dah, dan}, db[3] = {dbm, dbh, dbn};
        for (int q = 0; q < 3; ++q) {
            const LD s = a[q] + b[q], ds = da[q] + db[q];
            const LD e = expl(-(LD)dt * s);
            f[(size_t)i * 6 + 2 * q] = a[q] / s;
            g[(size_t)i * 6 + 2 * q] = h * (da[q] * s - a[q] * ds) / (s * s);
            f[(size_t)i * 6 + 2 * q + 1] = e;
            g[(size_t)i * 6 + 2 * q + 1] = h * (-(LD)dt * ds * e);
        }
    });
    parallel_for(kHHTabN, [&](int64_t i) {
        for (int q = 0; q < 6; ++q) {
            const LD f0 = f[(size_t)i * 6 + q], f1 = f[(size_t)(i + 1) * 6 + q];
            const LD g0 = g[(size_t)i * 6 + q], g1 = g[(size_t)(i + 1) * 6 + q];
            double* c = tab + (size_t)i * kHHTabStride + 4 * q;
            c[0] = (double)f0;
            c[1] = (double)g0;
            c[2] = (double)(3.0L * (f1 - f0) - 2.0L * g0 - g1);
            c[3] = (double)(2.0L * (f0 - f1) + g0 + g1);
        }
    });
}

// Per-CV membrane area (um^2), capacitance (nF) and axial conductance to the parent (uS):
// each CV is a cylinder; the conductance between a CV and its parent is that of the two half
// cylinders between their centres in series (Sec. "Model", Eq. discrete-v).
void cv_geometry(const arb_sim* sim, hvec<double>& area, hvec<double>& cap, hvec<double>& sigma) {
    const int64_t ncv = sim->n_cv;
    area.resize(ncv);   // every element is written below (first touch by the threads that use it)
    cap.resize(ncv);
    sigma.resize(ncv);
    parallel_for(sim->n_cells, [&](int64_t c) {
        const int64_t off = sim->cv_offset[c], n = sim->cv_offset[c + 1] - off;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t g = off + i;
            const double h = sim->length[g], r = sim->radius[g];
            area[g] = 2.0 * kPi * r * h;                  // um^2
            cap[g] = sim->cm[g] * area[g] * 1e-5;         // nF
            if (i > 0) {
                const int64_t pg = off + sim->parent[g];
                // half-cylinder resistances in series, MOhm
                const double half_i = sim->Ra[g] * h / (200.0 * kPi * r * r);
                const double half_p = sim->Ra[pg] * sim->length[pg] / (200.0 * kPi * sim->radius[pg] * sim->radius[pg]);
                sigma[g] = 1.0 / (half_i + half_p);       // uS
            } else {
                sigma[g] = 0.0;
            }
        }
    });
}

// ---------------------------------------------------------------------------------------
// Solve schedule of one pack.
//
// A cell's CVs are renumbered depth first (each child subtree contiguous, the larger subtree
// first), so a CV's parent is the CV just before it except at branch points. The forward
// sweep visits children before parents; a "row" holds one CV per lane.

struct CellOrder {
    std::vector<int32_t> dfs;      // dfs position -> local CV
    std::vector<int32_t> pos;      // local CV -> dfs position
    std::vector<int32_t> dpar;     // dfs position -> dfs position of the parent (-1 root)
};

CellOrder dfs_order(const int32_t* par, int32_t n) {
    CellOrder o;
    std::vector<int32_t> nch(n, 0), first(n + 1, 0), kids(n > 0 ? n - 1 : 0), size(n, 1);
    for (int32_t i = 1; i < n; ++i) nch[par[i]]++;
    for (int32_t i = 0; i < n; ++i) first[i + 1] = first[i] + nch[i];
    std::vector<int32_t> fill(first.begin(), first.end() - 1);
    for (int32_t i = 1; i < n; ++i) kids[fill[par[i]]++] = i;
    for (int32_t i = n - 1; i >= 1; --i) size[par[i]] += size[i];
    for (int32_t i = 0; i < n; ++i)
        std::stable_sort(kids.begin() + first[i], kids.begin() + first[i + 1],
                         [&](int32_t a, int32_t b) { return size[a] > size[b]; });
    o.dfs.reserve(n);
    std::vector<int32_t> stack;
    if (n > 0) stack.push_back(0);
    while (!stack.empty()) {
        const int32_t v = stack.back();
        stack.pop_back();
        o.dfs.push_back(v);
        for (int32_t q = first[v + 1] - 1; q >= first[v]; --q) stack.push_back(kids[q]);
    }
    o.pos.assign(n, 0);
    for (int32_t q = 0; q < n; ++q) o.pos[o.dfs[q]] = q;
    o.dpar.assign(n, -1);
    for (int32_t q = 1; q < n; ++q) o.dpar[q] = o.pos[par[o.dfs[q]]];
    return o;
}

// rows[j][l] = global model CV at (row j, lane l), or -1.
struct PackRows {
    std::vector<std::array<int64_t, 32>> rows;
    int round_rows = 0;
};

// One cell per lane: lane l walks its cell from the last DFS position to the root.
PackRows schedule_affinity(const std::vector<int32_t>& cells, const std::vector<CellOrder>& ord,
                           const std::vector<int64_t>& cv_offset) {
    PackRows pr;
    int32_t J = 0;
    for (int32_t c : cells) J = std::max<int32_t>(J, (int32_t)ord[c].dfs.size());
    std::array<int64_t, 32> empty;
    empty.fill(-1);
    pr.rows.assign(J, empty);
    for (size_t l = 0; l < cells.size(); ++l) {
        const int32_t c = cells[l];
        const int32_t n = (int32_t)ord[c].dfs.size();
        for (int32_t j = 0; j < n; ++j) pr.rows[j][l] = cv_offset[c] + ord[c].dfs[n - 1 - j];
    }
    pr.round_rows = 0;
    return pr;
}

// Several cells share the 32 lanes. Unbranched runs of CVs ("chains") are list-scheduled,
// deepest first, in rounds of R rows separated by a warp barrier. A chain whose parent runs
// on another lane hands its contribution over through shared memory, so the parent must
// start in a later round; at most one lane writes a given parent per round, which keeps the
// accumulation order fixed. A lane that completes the last child of a chain may continue
// straight into that chain (the contribution then stays in a register). With shift = 1 the
// contribution is written one row after the chain's head (the row-ring kernel adds it with the
// multiply-adds of the lane's next row, which has no child in a register), so a head on the
// last row of a round writes in the next round, and its parent waits one round more.
PackRows schedule_shared(const std::vector<int32_t>& cells, const std::vector<CellOrder>& ord,
                         const std::vector<int64_t>& cv_offset, int R, int shift = 0) {
    struct Chain {
        int64_t base;        // global CV offset of the cell
        const CellOrder* o;
        int32_t head, tail;  // dfs positions, head < tail
        int32_t parent;      // chain index of the parent chain, -1 root
        int32_t pending;     // children not finished
        int64_t prio;
        int32_t finish_round;
        int32_t child_round;   // latest round in which a child chain finished
    };
    std::vector<Chain> ch;
    for (int32_t c : cells) {
        const CellOrder& o = ord[c];
        const int32_t n = (int32_t)o.dfs.size();
        std::vector<int32_t> nch(n, 0);
        for (int32_t q = 1; q < n; ++q) nch[o.dpar[q]]++;
        std::vector<int32_t> chain_of(n, -1);
        for (int32_t q = 0; q < n; ++q) {
            const bool starts = (q == 0) || nch[o.dpar[q]] != 1;
            if (starts) {
                Chain x;
                x.base = cv_offset[c];
                x.o = &o;
                x.head = q;
                x.tail = q;
                x.parent = (q == 0) ? -1 : chain_of[o.dpar[q]];
                x.pending = 0;
                x.prio = 0;
                x.finish_round = -1;
                x.child_round = -1;
                ch.push_back(x);
            } else {
                ch.back().tail = q;   // single child directly follows its parent in DFS order
            }
            chain_of[q] = (int32_t)ch.size() - 1;
        }
    }
    const int32_t nchain = (int32_t)ch.size();
    for (int32_t i = 0; i < nchain; ++i)
        if (ch[i].parent >= 0) ch[ch[i].parent].pending++;
    // priority: CVs on the path to the root, own chain included (parents precede children)
    for (int32_t i = 0; i < nchain; ++i) {
        const int64_t len = ch[i].tail - ch[i].head + 1;
        ch[i].prio = len + (ch[i].parent >= 0 ? ch[ch[i].parent].prio : 0);
    }
    auto cmp = [&](int32_t a, int32_t b) {
        if (ch[a].prio != ch[b].prio) return ch[a].prio < ch[b].prio;
        return a > b;
    };
    std::priority_queue<int32_t, std::vector<int32_t>, decltype(cmp)> ready(cmp);
    for (int32_t i = 0; i < nchain; ++i)
        if (ch[i].pending == 0) ready.push(i);

    PackRows pr;
    pr.round_rows = R;
    std::array<int64_t, 32> empty;
    empty.fill(-1);
    std::array<int32_t, 32> cur, pos;
    cur.fill(-1);
    pos.fill(0);
    int32_t done = 0;
    int32_t round = 0;
    std::vector<int32_t> newly_next, written_next;   // writes that land in the next round (shift)
    int idle = 0;
    while (done < nchain) {
        const size_t r0 = pr.rows.size();
        for (int rr = 0; rr < R; ++rr) pr.rows.push_back(empty);
        std::vector<int32_t> newly = std::move(newly_next);     // parents ready after this round
        std::vector<int32_t> written = std::move(written_next); // parents written in this round
        newly_next.clear();
        written_next.clear();
        int32_t progressed = 0;
        for (int l = 0; l < 32; ++l) {
            for (int rr = 0; rr < R; ++rr) {
                if (cur[l] < 0) {
                    if (ready.empty()) break;
                    cur[l] = ready.top();
                    ready.pop();
                    pos[l] = 0;
                }
                Chain& x = ch[cur[l]];
                const int32_t len = x.tail - x.head + 1;
                const bool head_row = pos[l] == len - 1;
                const bool late = rr + shift >= R;   // a hand-over from this row is written next round
                bool cont = false;
                if (head_row && x.parent >= 0) {
                    Chain& P = ch[x.parent];
                    const std::vector<int32_t>& wl = late ? written_next : written;
                    // continuation: this is the last child and every sibling's write is in an earlier round
                    if (P.pending == 1 && P.child_round < round) {
                        cont = true;
                    } else if (std::find(wl.begin(), wl.end(), x.parent) != wl.end()) {
                        break;   // a sibling already writes this parent in that round: wait
                    }
                }
                pr.rows[r0 + rr][l] = x.base + x.o->dfs[x.tail - pos[l]];
                ++progressed;
                pos[l]++;
                if (pos[l] == len) {
                    x.finish_round = round;
                    ++done;
                    const int32_t pidx = x.parent;
                    cur[l] = -1;
                    if (pidx >= 0) {
                        ch[pidx].pending--;
                        if (cont) {
                            ch[pidx].child_round = std::max(ch[pidx].child_round, round);
                            cur[l] = pidx;
                            pos[l] = 0;
                        } else {
                            ch[pidx].child_round = std::max(ch[pidx].child_round, late ? round + 1 : round);
                            (late ? written_next : written).push_back(pidx);
                            // ready once every child's write has landed
                            if (ch[pidx].pending == 0) (ch[pidx].child_round > round ? newly_next : newly).push_back(pidx);
                        }
                    }
                }
            }
        }
        for (int32_t i : newly) ready.push(i);
        ++round;
        // a round without progress happens only while a write of the round before blocks a
        // lane; three in a row cannot happen (some chain is always ready, running or about to
        // be ready)
        idle = progressed == 0 ? idle + 1 : 0;
        if (idle > 2 && done < nchain) break;
    }
    // trim trailing empty rows
    while (!pr.rows.empty()) {
        bool any = false;
        for (int l = 0; l < 32; ++l) any |= pr.rows.back()[l] >= 0;
        if (any) break;
        pr.rows.pop_back();
    }
    return pr;
}

}  // namespace

namespace arbk {
void set_handle_free_error(const std::string& msg) { g_create_error = msg; }
}

static void layout_regions(arb_sim* sim) {
    const Plan& pl = sim->plan;
    const arb_params& p = sim->prm;
    const int64_t ne = pl.total_rows * kWarp;
    const int64_t npk = (int64_t)pl.packs.size();
    const int64_t nowner = npk * kWarp;
    const int64_t nslot = sim->overlap ? 2 : 1;     // delivery-list buffers
    const bool mx = sim->mixed;
    const size_t mt = mx ? sizeof(float) : sizeof(double);
    const int64_t nsyn = (int64_t)sim->syn_cv.size(), nhh = (int64_t)sim->hh_cv.size();
    const int64_t scratch = std::max<int64_t>({sim->n_cv, 3 * nhh, nsyn, 1});
    std::vector<std::pair<std::string, size_t>> want = {
        {"ctl", sizeof(Ctl)},
        {"packs", sizeof(PackDesc) * std::max<int64_t>(npk, 1)},
        {"ca", 8 * ne}, {"cb", 8 * ne}, {"ck", 8 * ne}, {"ce", 8 * ne}, {"pslot", 4 * ne}, {"vmap", 4 * ne},
        {"V", 8 * ne},
        {"Sg", 8 * std::max<int64_t>(pl.stream_imp ? 1 : pl.sg_total, 1)}, {"Rg", 8 * std::max<int64_t>(pl.stream_imp ? 1 : pl.sg_total, 1)},
        {"UE", 16 * std::max<int64_t>(pl.stream_imp ? ne : 1, 1)}, {"cpos", 4 * std::max<int64_t>((int64_t)pl.cpos.size(), 1)},
        {"row_cs", 4 * std::max<int64_t>((int64_t)pl.row_cs.size(), 1)}, {"row_cn", 4 * std::max<int64_t>((int64_t)pl.row_cn.size(), 1)},
        {"mb_ent", 4 * std::max<int64_t>((int64_t)pl.mb_ent.size(), 1)}, {"mb_cs", 4 * std::max<int64_t>((int64_t)pl.mb_cs.size(), 1)},
        {"Gm", 8 * std::max<int64_t>(pl.c_total, 1)}, {"Em", 8 * std::max<int64_t>(pl.c_total, 1)},
        {"cE", 8 * std::max<int64_t>(pl.c_total, 1)}, {"cB", 8 * std::max<int64_t>(pl.c_total, 1)},
        {"syn_slot", 4 * pl.syn_rows * kWarp}, {"syn_vs", 4 * pl.syn_rows * kWarp}, {"syn_g", mt * pl.syn_rows * kWarp},
        {"syn_e", 8 * pl.syn_rows * kWarp}, {"syn_decay", 8 * pl.syn_rows * kWarp}, {"syn_sc", 8 * pl.syn_rows * kWarp},
        {"syn_ntau", 8 * pl.syn_rows * kWarp}, {"slot_lo", 4 * std::max<int64_t>(nowner, 1)}, {"slot_hi", 4 * std::max<int64_t>(nowner, 1)},
        {"hh_tab", 8 * std::max<int64_t>((int64_t)sim->hh_tab.size(), 1)},
        {"hh_tab_f", 4 * std::max<int64_t>((int64_t)sim->hh_tab_f.size(), 1)},
        {"syn_decay_f", 4 * (mx ? pl.syn_rows * kWarp : 1)}, {"syn_e_f", 4 * (mx ? pl.syn_rows * kWarp : 1)},
        {"hh_gna_f", 4 * (mx ? pl.hh_rows * kWarp : 1)}, {"hh_gk_f", 4 * (mx ? pl.hh_rows * kWarp : 1)},
        {"hh_slot", 4 * pl.hh_rows * kWarp}, {"hh_vs", 4 * pl.hh_rows * kWarp}, {"hh_sc", 8 * pl.hh_rows * kWarp}, {"hh_gna", 8 * pl.hh_rows * kWarp},
        {"hh_gk", 8 * pl.hh_rows * kWarp}, {"hh_m", mt * pl.hh_rows * kWarp}, {"hh_h", mt * pl.hh_rows * kWarp},
        {"hh_n", mt * pl.hh_rows * kWarp},
        {"st_slot", 4 * pl.st_rows * kWarp}, {"st_sc", 8 * pl.st_rows * kWarp}, {"st_on", 8 * pl.st_rows * kWarp},
        {"st_off", 8 * pl.st_rows * kWarp}, {"st_amp", 8 * pl.st_rows * kWarp},
        {"det_slot", 4 * nowner}, {"det_gid", 4 * nowner},
        {"probe_slot", 4 * std::max<int64_t>(sim->n_cv, 1)}, {"probe_col", 4 * std::max<int64_t>(sim->n_cv, 1)},
        {"ev_off", 4 * (nowner + 1) * nslot}, {"counts", 4 * std::max<int64_t>(nowner, 1)},
        {"ev", sizeof(EvRec) * p.bucket_capacity * nslot}, {"ev_tmp", sizeof(EvRec) * p.bucket_capacity},
        {"pool0", sizeof(PendEv) * p.event_capacity}, {"pool1", sizeof(PendEv) * p.event_capacity},
        {"ext_step", 8 * p.ext_event_capacity}, {"ext_t", 8 * p.ext_event_capacity}, {"ext_w", 8 * p.ext_event_capacity},
        {"ext_syn", 4 * p.ext_event_capacity}, {"ext_idx", 4 * p.ext_event_capacity},
        {"syn_owner", 4 * std::max<int64_t>(nsyn, 1)}, {"syn_js", 4 * std::max<int64_t>(nsyn, 1)},
        {"out_ptr", 8 * (sim->n_cells * sim->dry_ranks + 1)}, {"out_syn", 4 * std::max<size_t>(sim->out_syn.size(), 1)},
        {"out_idx", 4 * std::max<size_t>(sim->out_syn.size(), 1)}, {"out_delay", 8 * std::max<size_t>(sim->out_syn.size(), 1)},
        {"out_w", 8 * std::max<size_t>(sim->out_syn.size(), 1)},
        {"spk_gid", 4 * p.spike_capacity}, {"spk_t", 8 * p.spike_capacity},
        {"cv_tile", 8 * std::max<int64_t>(sim->n_cv, 1)}, {"hh_entry", 8 * std::max<int64_t>(nhh, 1)},
        {"syn_entry", 8 * std::max<int64_t>(nsyn, 1)}, {"scratch", 8 * scratch},
    };
    sim->regions.clear();
    size_t off = 0;
    for (auto& w : want) {
        off = (off + 255) & ~(size_t)255;
        Region r;
        r.off = off;
        r.bytes = w.second;
        sim->regions.push_back({w.first, r});
        off += w.second;
#ifdef ARB_DEBUG
        off = (off + 255) & ~(size_t)255;
        off += kCanaryBytes;                 // guard words after the region
#endif
    }
    sim->ws_bytes = (int64_t)((off + 255) & ~(size_t)255);
}

#ifdef ARB_DEBUG
// Debug builds: kCanaryBytes of kCanaryByte after every workspace region, written at bind and
// compared after every arb_advance (arb_check_canaries); a kernel writing past the end of a
// region changes them.
static size_t canary_off(const Region& r) { return ((r.off + r.bytes + 255) & ~(size_t)255); }

static arb_status write_canaries(arb_sim* sim) {
    for (auto& r : sim->regions)
        CU(cudaMemsetAsync(sim->ws + canary_off(r.second), kCanaryByte, kCanaryBytes, sim->s));
    return ARB_OK;
}
#endif

static arb_status check_canaries(arb_sim* sim) {
#ifdef ARB_DEBUG
    std::vector<unsigned char> h(kCanaryBytes * sim->regions.size());
    for (size_t i = 0; i < sim->regions.size(); ++i)
        CU(cudaMemcpyAsync(h.data() + i * kCanaryBytes, sim->ws + canary_off(sim->regions[i].second), kCanaryBytes,
                           cudaMemcpyDeviceToHost, sim->s));
    CU(cudaStreamSynchronize(sim->s));
    for (size_t i = 0; i < sim->regions.size(); ++i)
        for (int b = 0; b < kCanaryBytes; ++b)
            if (h[i * kCanaryBytes + b] != kCanaryByte)
                return fail(sim, ARB_E_STATE, "debug check: the guard words after workspace region '" +
                                                  sim->regions[i].first + "' were overwritten");
    return ARB_OK;
#else
    return fail(sim, ARB_OK, "the release library keeps no guard words (build with ARB_DEBUG)");
#endif
}

static char* region(arb_sim* sim, const char* name) {
    for (auto& r : sim->regions)
        if (r.first == name) return sim->ws + r.second.off;
    return nullptr;
}

template <class V>
static arb_status up(arb_sim* sim, const char* name, const V& v) {
    if (v.empty()) return ARB_OK;
    char* dst = region(sim, name);
    if (!dst) return fail(sim, ARB_E_STATE, std::string("internal: no region ") + name);
    CU(cudaMemcpyAsync(dst, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice, sim->s));
    return ARB_OK;
}

template <class MT>
static void fill_devmodel(arb_sim* sim, DevModel<MT>& d) {
    const Plan& pl = sim->plan;
    d.packs = (const PackDesc*)region(sim, "packs");
    d.n_packs = (int32_t)pl.packs.size();
    d.n_owner = d.n_packs * kWarp;
    d.ca = (const double*)region(sim, "ca");
    d.cb = (const double*)region(sim, "cb");
    d.ck = (const double*)region(sim, "ck");
    d.ce = (const double*)region(sim, "ce");
    d.pslot = (const int32_t*)region(sim, "pslot");
    d.vmap = (const int32_t*)region(sim, "vmap");
    d.V = (double*)region(sim, "V");
    d.hh_tab = sim->hh_tab.empty() ? nullptr : (const double*)region(sim, "hh_tab");
    d.hh_tab_f = sim->hh_tab_f.empty() ? nullptr : (const float*)region(sim, "hh_tab_f");
    d.syn_decay_f = (const float*)region(sim, "syn_decay_f");
    d.syn_e_f = (const float*)region(sim, "syn_e_f");
    d.hh_gna_f = (const float*)region(sim, "hh_gna_f");
    d.hh_gk_f = (const float*)region(sim, "hh_gk_f");
    d.Sg = (double*)region(sim, "Sg");
    d.Rg = (double*)region(sim, "Rg");
    d.Gm = (double*)region(sim, "Gm");
    d.cE = (const double*)region(sim, "cE");
    d.cB = (const double*)region(sim, "cB");
    d.Em = (double*)region(sim, "Em");
    d.UE = (double2*)region(sim, "UE");
    d.cpos = (const int32_t*)region(sim, "cpos");
    d.row_cs = (const int32_t*)region(sim, "row_cs");
    d.row_cn = (const int32_t*)region(sim, "row_cn");
    d.mb_ent = (const int32_t*)region(sim, "mb_ent");
    d.mb_cs = (const int32_t*)region(sim, "mb_cs");
    d.syn_slot = (const int32_t*)region(sim, "syn_slot");
    d.syn_vs = (const int32_t*)region(sim, "syn_vs");
    d.syn_g = (MT*)region(sim, "syn_g");
    d.syn_e = (const double*)region(sim, "syn_e");
    d.syn_ntau = (const double*)region(sim, "syn_ntau");
    d.slot_lo = (const int32_t*)region(sim, "slot_lo");
    d.slot_hi = (const int32_t*)region(sim, "slot_hi");
    d.exact = sim->exact ? 1 : 0;
    d.syn_decay = (const double*)region(sim, "syn_decay");
    d.syn_sc = (const double*)region(sim, "syn_sc");
    d.hh_slot = (const int32_t*)region(sim, "hh_slot");
    d.hh_vs = (const int32_t*)region(sim, "hh_vs");
    d.hh_sc = (const double*)region(sim, "hh_sc");
    d.hh_gna = (const double*)region(sim, "hh_gna");
    d.hh_gk = (const double*)region(sim, "hh_gk");
    d.hh_m = (MT*)region(sim, "hh_m");
    d.hh_h = (MT*)region(sim, "hh_h");
    d.hh_n = (MT*)region(sim, "hh_n");
    d.st_slot = (const int32_t*)region(sim, "st_slot");
    d.st_sc = (const double*)region(sim, "st_sc");
    d.st_on = (const double*)region(sim, "st_on");
    d.st_off = (const double*)region(sim, "st_off");
    d.st_amp = (const double*)region(sim, "st_amp");
    d.det_slot = (const int32_t*)region(sim, "det_slot");
    d.det_gid = (const int32_t*)region(sim, "det_gid");
    d.probe_slot = (const int32_t*)region(sim, "probe_slot");
    d.probe_col = (const int32_t*)region(sim, "probe_col");
    d.n_probe = sim->n_probe;
    d.trace = sim->trace;
    d.ev_off = (const int32_t*)region(sim, "ev_off");
    d.ev = (const EvRec*)region(sim, "ev");
    d.spk_gid = (int32_t*)region(sim, "spk_gid");
    d.spk_t = (double*)region(sim, "spk_t");
    d.spike_cap = sim->prm.spike_capacity;
    d.ctl = (Ctl*)region(sim, "ctl");
    d.dt = sim->prm.dt;
    d.threshold = sim->threshold;
}

// ===========================================================================================
// C ABI

extern "C" {

arb_status arb_hh_gate_table(double dt, double* coef, int64_t cap, int64_t* n_intervals, double* v_lo,
                             double* per_mv) {
    g_create_error.clear();
    if (!(dt > 0.0) || !std::isfinite(dt)) {
        g_create_error = "arb_hh_gate_table: dt must be finite and > 0";
        return ARB_E_ARG;
    }
    if (coef && cap < (int64_t)kHHTabN * kHHTabStride) {
        g_create_error = "arb_hh_gate_table: coef holds " + std::to_string(cap) + " doubles, the table needs " +
                         std::to_string((int64_t)kHHTabN * kHHTabStride);
        return ARB_E_ARG;
    }
    if (n_intervals) *n_intervals = kHHTabN;
    if (v_lo) *v_lo = kHHTabVlo;
    if (per_mv) *per_mv = kHHTabPerMV;
    if (coef) build_hh_table(dt, coef);
    return ARB_OK;
}

int32_t arb_kernel_variants(int32_t cap, int32_t* warps, int32_t* fwd_rows, int32_t* back_rows) {
    const int n = stream_variant_count();
    for (int v = 0; v < n && v < cap; ++v) {
        int w = 0, rf = 0, rb = 0;
        stream_variant_info(v, &w, &rf, &rb);
        if (warps) warps[v] = w;
        if (fwd_rows) fwd_rows[v] = rf;
        if (back_rows) back_rows[v] = rb;
    }
    return n;
}

arb_status arb_default_params(arb_params* p) {
    if (!p) return ARB_E_ARG;
    std::memset(p, 0, sizeof(*p));
    p->kernel_variant = -1;
    p->dt = 0.025;
    p->epoch_steps = 0;
    p->precision = ARB_FP64;
    p->cells_per_pack = 0;
    p->smem_budget = 0;
    p->scheme = ARB_IMPLICIT;
    p->event_capacity = 1 << 22;
    p->ext_event_capacity = 1 << 20;
    p->spike_capacity = 1 << 22;
    p->bucket_capacity = 1 << 21;
    p->stream = nullptr;
    return ARB_OK;
}

const char* arb_last_error(const arb_sim* sim) { return sim ? sim->err.c_str() : g_create_error.c_str(); }

arb_status arb_create(const arb_model* m, const arb_params* pp, arb_sim** out) {
    if (!out) return ARB_E_ARG;
    *out = nullptr;
    g_create_error.clear();
    if (!m || !pp) { g_create_error = "model or params is NULL"; return ARB_E_ARG; }
    arb_sim* sim = new (std::nothrow) arb_sim();
    if (!sim) return ARB_E_NOMEM;
    auto bad = [&](const std::string& msg) {
        g_create_error = msg;   // readable with arb_last_error(NULL)
        delete sim;
        return ARB_E_ARG;
    };
    sim->prm = *pp;
    const arb_params& p = sim->prm;
    if (!finite_pos(p.dt)) return bad("dt must be finite and > 0");
    if (p.precision != ARB_FP64 && p.precision != ARB_MIXED) return bad("precision must be ARB_FP64 or ARB_MIXED");
    if (p.event_capacity < 1 || p.ext_event_capacity < 1 || p.spike_capacity < 1 || p.bucket_capacity < 1)
        return bad("capacities must be >= 1");
    if (p.event_capacity > INT32_MAX || p.bucket_capacity > INT32_MAX) return bad("event and bucket capacities must be < 2^31");
    if (p.epoch_overlap != 0 && p.epoch_overlap != 1) return bad("epoch_overlap must be 0 or 1");
    if (p.dry_run_ranks < 0) return bad("dry_run_ranks must be >= 0");
    if (p.epoch_overlap && p.bucket_capacity > INT32_MAX / 2) return bad("with epoch_overlap the bucket capacity must be < 2^30");
    if (p.cells_per_pack < 0 || p.cells_per_pack > 32) return bad("cells_per_pack must be 0..32");
    if (p.split_cvs < -1) return bad("split_cvs must be >= -1");
    if (p.spread_rows < 0) return bad("spread_rows must be >= 0");
    if (p.kernel_variant < -1 || p.kernel_variant >= stream_variant_count())
        return bad("kernel_variant must be -1 or in [0, " + std::to_string(stream_variant_count()) + ")");
    sim->mixed = p.precision == ARB_MIXED;
    if (p.scheme != ARB_IMPLICIT && p.scheme != ARB_EXPLICIT) return bad("scheme must be ARB_IMPLICIT or ARB_EXPLICIT");
    sim->implicit = p.scheme == ARB_IMPLICIT;
    if (m->n_cells < 0) return bad("n_cells < 0");
    const int32_t nc = m->n_cells;
    sim->n_cells = nc;
    if (nc > 0 && !m->cv_offset) return bad("cv_offset is NULL");
    sim->cv_offset.assign(nc + 1, 0);
    if (nc > 0) std::copy(m->cv_offset, m->cv_offset + nc + 1, sim->cv_offset.begin());
    if (sim->cv_offset[0] != 0) return bad("cv_offset[0] must be 0");
    for (int32_t c = 0; c < nc; ++c)
        if (sim->cv_offset[c + 1] <= sim->cv_offset[c]) return bad("every cell needs at least one CV (cv_offset must increase)");
    const int64_t ncv = sim->cv_offset[nc];
    sim->n_cv = ncv;
    if (ncv > (int64_t)INT32_MAX / 2) return bad("too many CVs");
    if (ncv > 0 && (!m->parent || !m->length_um || !m->radius_um || !m->cm || !m->Ra)) return bad("morphology array is NULL");
    sim->parent.resize(ncv);
    sim->length.resize(ncv);
    sim->radius.resize(ncv);
    sim->cm.resize(ncv);
    sim->Ra.resize(ncv);
    // copy and check cell by cell in parallel; the first failing cell (lowest index) is reported
    std::vector<int64_t> bad_at(nc, -1);        // local index of the first bad CV, or -1
    std::vector<char> bad_kind(nc, 0);          // 1 root, 2 parent order, 3 geometry
    parallel_for(nc, [&](int64_t c) {
        const int64_t off = sim->cv_offset[c], n = sim->cv_offset[c + 1] - off;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t g = off + i;
            sim->parent[g] = m->parent[g];
            sim->length[g] = m->length_um[g];
            sim->radius[g] = m->radius_um[g];
            sim->cm[g] = m->cm[g];
            sim->Ra[g] = m->Ra[g];
            const int32_t pi = sim->parent[g];
            char k = 0;
            if (i == 0 ? pi != -1 : (pi < 0 || pi >= i)) k = i == 0 ? 1 : 2;
            else if (!finite_pos(sim->length[g]) || !finite_pos(sim->radius[g]) || !finite_pos(sim->cm[g]) ||
                     !finite_pos(sim->Ra[g]))
                k = 3;
            if (k && bad_at[c] < 0) { bad_at[c] = i; bad_kind[c] = k; }
        }
    });
    for (int32_t c = 0; c < nc; ++c) {
        if (bad_at[c] < 0) continue;
        const int64_t i = bad_at[c];
        if (bad_kind[c] == 1) return bad("cell " + std::to_string(c) + ": first CV must have parent -1");
        if (bad_kind[c] == 2) return bad("cell " + std::to_string(c) + ": parent of local CV " + std::to_string(i) + " must be in [0, i)");
        return bad("CV " + std::to_string(sim->cv_offset[c] + i) + ": length, radius, cm and Ra must be finite and > 0");
    }
    // copies in parallel chunks; false when an element fails the check
    auto par_copy = [&](int64_t n, const auto* src, auto& dst, auto ok) -> bool {
        dst.resize((size_t)n);
        constexpr int64_t kChunk = 1 << 16;
        const int64_t nch = (n + kChunk - 1) / kChunk;
        std::vector<char> bad_chunk(nch, 0);
        auto* d = dst.data();
        parallel_for(nch, [&](int64_t ch) {
            const int64_t lo = ch * kChunk, hi = std::min<int64_t>(n, lo + kChunk);
            for (int64_t i = lo; i < hi; ++i) {
                d[i] = src[i];
                if (!ok(d[i])) bad_chunk[ch] = 1;
            }
        });
        for (char b : bad_chunk) if (b) return false;
        return true;
    };
    auto copy_idx = [&](int64_t n, const int64_t* src, hvec<int64_t>& dst, const char* what) -> bool {
        if (n < 0 || (n > 0 && !src)) return false;
        if (!par_copy(n, src, dst, [&](int64_t x) { return x >= 0 && x < ncv; })) {
            sim->err = std::string(what) + " CV index out of range";
            return false;
        }
        return true;
    };
    auto copy_d = [&](int64_t n, const double* src, hvec<double>& dst) -> bool {
        if (n < 0 || (n > 0 && !src)) return false;
        return par_copy(n, src, dst, [](double x) { return std::isfinite(x); });
    };
    if (!copy_idx(m->n_hh, m->hh_cv, sim->hh_cv, "hh") || !copy_d(m->n_hh, m->gnabar, sim->gnabar) ||
        !copy_d(m->n_hh, m->gkbar, sim->gkbar) || !copy_d(m->n_hh, m->gl, sim->gl))
        return bad(sim->err.empty() ? "bad Hodgkin-Huxley arrays" : sim->err);
    if (!copy_idx(m->n_pas, m->pas_cv, sim->pas_cv, "pas") || !copy_d(m->n_pas, m->g_pas, sim->g_pas) ||
        !copy_d(m->n_pas, m->e_pas, sim->e_pas))
        return bad(sim->err.empty() ? "bad passive arrays" : sim->err);
    if (!copy_idx(m->n_syn, m->syn_cv, sim->syn_cv, "syn") || !copy_d(m->n_syn, m->syn_tau, sim->syn_tau) ||
        !copy_d(m->n_syn, m->syn_e, sim->syn_e))
        return bad(sim->err.empty() ? "bad synapse arrays" : sim->err);
    for (double tau : sim->syn_tau) if (!(tau > 0)) return bad("synapse tau must be > 0");
    if (p.coalesce_synapses != 0 && p.coalesce_synapses != 1) return bad("coalesce_synapses must be 0 or 1");
    if (p.event_timing != ARB_EVENTS_STEP_START && p.event_timing != ARB_EVENTS_EXACT)
        return bad("event_timing must be ARB_EVENTS_STEP_START or ARB_EVENTS_EXACT");
    sim->exact = p.event_timing == ARB_EVENTS_EXACT;
    if (sim->exact && (p.scheme != ARB_IMPLICIT || p.precision != ARB_FP64))
        return bad("exact event times need the implicit scheme and FP64");
    if (sim->exact && ((p.cells_per_pack != 0 && p.cells_per_pack != 32) || p.split_cvs > 0))
        return bad("exact event times run one cell per lane: cells_per_pack must be 0 or 32 and split_cvs 0 or -1");
    sim->coalesce = p.coalesce_synapses == 1;
    {
        const int64_t ns = (int64_t)sim->syn_cv.size();
        sim->syn_unit.assign(ns, 0);
        if (sim->coalesce) {
            std::vector<int32_t> ord(ns);
            std::iota(ord.begin(), ord.end(), 0);
            std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) {
                if (sim->syn_cv[x] != sim->syn_cv[y]) return sim->syn_cv[x] < sim->syn_cv[y];
                if (sim->syn_tau[x] != sim->syn_tau[y]) return sim->syn_tau[x] < sim->syn_tau[y];
                return sim->syn_e[x] < sim->syn_e[y];
            });
            std::vector<int32_t> unit_of_sorted(ns);
            int32_t nu = 0;
            for (int64_t r = 0; r < ns; ++r) {
                const int32_t x = ord[r];
                if (r > 0) {
                    const int32_t y = ord[r - 1];
                    if (sim->syn_cv[x] != sim->syn_cv[y] || sim->syn_tau[x] != sim->syn_tau[y] || sim->syn_e[x] != sim->syn_e[y]) ++nu;
                }
                sim->syn_unit[x] = nu;
            }
            nu = ns > 0 ? nu + 1 : 0;
            sim->u_rep.assign(nu, INT32_MAX);
            for (int64_t i = 0; i < ns; ++i) sim->u_rep[sim->syn_unit[i]] = std::min<int32_t>(sim->u_rep[sim->syn_unit[i]], (int32_t)i);
        } else {
            std::iota(sim->syn_unit.begin(), sim->syn_unit.end(), 0);
            sim->u_rep = sim->syn_unit;
        }
        const size_t nu = sim->u_rep.size();
        sim->u_cv.resize(nu);
        sim->u_tau.resize(nu);
        sim->u_e.resize(nu);
        for (size_t u = 0; u < nu; ++u) {
            sim->u_cv[u] = sim->syn_cv[sim->u_rep[u]];
            sim->u_tau[u] = sim->syn_tau[sim->u_rep[u]];
            sim->u_e[u] = sim->syn_e[sim->u_rep[u]];
        }
    }
    if (m->n_syn > INT32_MAX / 2) return bad("too many synapses");
    if (!copy_idx(m->n_stim, m->stim_cv, sim->st_cv, "stim") || !copy_d(m->n_stim, m->stim_t_on, sim->st_on) ||
        !copy_d(m->n_stim, m->stim_dur, sim->st_dur) || !copy_d(m->n_stim, m->stim_amp, sim->st_amp))
        return bad(sim->err.empty() ? "bad clamp arrays" : sim->err);
    if (nc > 0 && !m->detector_cv) return bad("detector_cv is NULL");
    sim->det_cv.assign(m->detector_cv, m->detector_cv + nc);
    for (int32_t c = 0; c < nc; ++c)
        if (sim->det_cv[c] < sim->cv_offset[c] || sim->det_cv[c] >= sim->cv_offset[c + 1])
            return bad("detector of cell " + std::to_string(c) + " is not one of its CVs");
    if (!std::isfinite(m->threshold)) return bad("threshold must be finite");
    sim->threshold = m->threshold;
    {   // at most one HH per CV
        std::vector<char> seen(ncv, 0);
        for (int64_t cv : sim->hh_cv) {
            if (seen[cv]) return bad("more than one Hodgkin-Huxley instance on CV " + std::to_string(cv));
            seen[cv] = 1;
        }
    }
    const int64_t ncon = m->n_conn;
    if (ncon < 0 || (ncon > 0 && (!m->conn_src || !m->conn_dst_syn || !m->conn_delay || !m->conn_weight)))
        return bad("bad connection arrays");
    if (ncon > INT32_MAX) return bad("too many connections");
    sim->conn_src.assign(m->conn_src, m->conn_src + ncon);
    sim->conn_dst.assign(m->conn_dst_syn, m->conn_dst_syn + ncon);
    sim->conn_delay.assign(m->conn_delay, m->conn_delay + ncon);
    sim->conn_w.assign(m->conn_weight, m->conn_weight + ncon);
    // dry run: the sources are the gids of all virtual ranks
    sim->dry_ranks = std::max<int64_t>(1, p.dry_run_ranks);
    sim->variant = std::max<int32_t>(0, p.kernel_variant);
    const int64_t n_src = (int64_t)nc * sim->dry_ranks;
    if (n_src > INT32_MAX) return bad("dry_run_ranks * n_cells must be < 2^31");
    // checked in parallel parts; the first failing connection (lowest index) is reported
    double dmin = INFINITY;
    {
        const int64_t max_t = ncon >= (1 << 20) ? 16 : 1;
        std::vector<int64_t> bad_at(max_t, ncon);
        std::vector<int> bad_kind(max_t, 0);
        std::vector<double> part_min(max_t, INFINITY);
        run_tasks(max_t, [&](int64_t t, int64_t nt) {
            const int64_t lo = ncon * t / nt, hi = ncon * (t + 1) / nt;
            double mn = INFINITY;
            for (int64_t i = lo; i < hi; ++i) {
                int k = 0;
                if (sim->conn_src[i] < 0 || sim->conn_src[i] >= n_src) k = 1;
                else if (sim->conn_dst[i] < 0 || sim->conn_dst[i] >= m->n_syn) k = 2;
                else if (!finite_pos(sim->conn_delay[i])) k = 3;
                else if (!std::isfinite(sim->conn_w[i])) k = 4;
                if (k) {
                    bad_at[t] = i;
                    bad_kind[t] = k;
                    break;
                }
                mn = std::min(mn, sim->conn_delay[i]);
            }
            part_min[t] = mn;
        });
        int64_t first = ncon;
        int kind = 0;
        for (int64_t t = 0; t < max_t; ++t) {
            if (bad_at[t] < first) { first = bad_at[t]; kind = bad_kind[t]; }
            dmin = std::min(dmin, part_min[t]);
        }
        if (kind == 1)
            return bad(sim->dry_ranks > 1 ? "connection source gid out of range (dry run: < dry_run_ranks * n_cells)"
                                          : "connection source gid out of range");
        if (kind == 2) return bad("connection target synapse out of range");
        if (kind == 3) return bad("connection delays must be finite and > 0");
        if (kind == 4) return bad("connection weights must be finite");
    }
    // epoch: no longer than the minimum delay (Sec. "Model": a positive minimum delay lets
    // cells advance independently over that interval)
    // With the overlapped exchange an epoch is at most half the minimum delay (Sec.
    // "Implementation"): spikes of epoch i then reach no epoch before i + 2.
    const int lag = p.epoch_overlap ? 2 : 1;
    if (p.epoch_steps > 0) {
        sim->epoch_steps = p.epoch_steps;
    } else if (ncon > 0) {
        const double e = std::floor(dmin / (lag * p.dt) * (1.0 + 1e-12));
        sim->epoch_steps = (int32_t)std::max(1.0, std::min(e, 100000.0));
    } else {
        sim->epoch_steps = 400;
    }
    if (ncon > 0 && dmin < lag * sim->epoch_steps * p.dt * (1.0 - 1e-12))
        return bad("epoch of " + std::to_string(sim->epoch_steps) + " steps is longer than " +
                   (p.epoch_overlap ? "half the minimum delay (overlapped exchange)" : "the minimum delay"));
    sim->overlap = p.epoch_overlap != 0;

    // ------------------------------------------------------------------ discretisation
    hvec<double> area, cap, sigma, Glin, GElin;
    par_assign(Glin, ncv, 0.0);
    par_assign(GElin, ncv, 0.0);
    cv_geometry(sim, area, cap, sigma);
    {
        // passive entries: in parallel chunks when their CVs are strictly increasing (one writer
        // per CV), else in order; then HH instances, which sit on distinct CVs (checked above)
        const int64_t npas = (int64_t)sim->pas_cv.size();
        bool inc = true;
        for (int64_t i = 1; i < npas && inc; ++i) inc = sim->pas_cv[i] > sim->pas_cv[i - 1];
        auto pas = [&](int64_t i) {
            const int64_t cv = sim->pas_cv[i];
            const double G = sim->g_pas[i] * area[cv] * 1e-2;  // S/cm^2 * um^2 -> uS
            Glin[cv] += G;
            GElin[cv] += G * sim->e_pas[i];
        };
        constexpr int64_t kChunk = 1 << 16;
        if (inc) {
            parallel_for((npas + kChunk - 1) / kChunk, [&](int64_t ch) {
                for (int64_t i = ch * kChunk; i < std::min<int64_t>(npas, (ch + 1) * kChunk); ++i) pas(i);
            });
        } else {
            for (int64_t i = 0; i < npas; ++i) pas(i);
        }
    }
    std::vector<double> hh_gna(sim->hh_cv.size()), hh_gk(sim->hh_cv.size());
    {
        const int64_t nhh = (int64_t)sim->hh_cv.size();
        constexpr int64_t kChunk = 1 << 16;
        parallel_for((nhh + kChunk - 1) / kChunk, [&](int64_t ch) {
            for (int64_t i = ch * kChunk; i < std::min<int64_t>(nhh, (ch + 1) * kChunk); ++i) {
                const int64_t cv = sim->hh_cv[i];
                const double G = sim->gl[i] * area[cv] * 1e-2;
                Glin[cv] += G;
                GElin[cv] += G * kEL;
                hh_gna[i] = sim->gnabar[i] * area[cv] * 1e-2;
                hh_gk[i] = sim->gkbar[i] * area[cv] * 1e-2;
            }
        });
    }

    // ------------------------------------------------------------------ factorisation
    std::vector<CellOrder> ord(nc);
    hvec<double> invd, ck, ce, ca, cb;   // every element is written in the cell loop below
    invd.resize(ncv);
    ck.resize(ncv);
    ce.resize(ncv);
    ca.resize(ncv);
    cb.resize(ncv);
    {
        // cells are independent: each thread orders and factorises whole cells
        parallel_for(nc, [&](int64_t c) {
            std::vector<double> dd;
            const int64_t off = sim->cv_offset[c];
            const int32_t n = (int32_t)(sim->cv_offset[c + 1] - off);
            ord[c] = dfs_order(sim->parent.data() + off, n);
            const CellOrder& o = ord[c];
            dd.assign(n, 0.0);
            for (int32_t q = 0; q < n; ++q) dd[q] = cap[off + o.dfs[q]] / p.dt;
            for (int32_t q = 1; q < n; ++q) {
                const double sg = sigma[off + o.dfs[q]];
                dd[q] += sg;
                dd[o.dpar[q]] += sg;
            }
            // eliminate children into parents, leaves first (dfs positions descending)
            for (int32_t q = n - 1; q >= 1; --q) {
                const double a = -sigma[off + o.dfs[q]];
                dd[o.dpar[q]] -= (a / dd[q]) * a;
            }
            for (int32_t q = 0; q < n; ++q) {
                const int64_t g = off + o.dfs[q];
                invd[g] = 1.0 / dd[q];
            }
            for (int32_t q = 0; q < n; ++q) {
                const int64_t g = off + o.dfs[q];
                if (sim->implicit) {
                    // constant parts of the per-step system; the pivots are formed in the kernel
                    ca[g] = cap[g] / p.dt;
                    cb[g] = GElin[g];
                    ck[g] = q > 0 ? sigma[g] : 0.0;
                    ce[g] = cap[g] / p.dt + Glin[g];
                } else {
                    ca[g] = (cap[g] / p.dt - Glin[g]) * invd[g];
                    cb[g] = GElin[g] * invd[g];
                    if (q > 0) {
                        const double a = -sigma[g];
                        ck[g] = a * invd[off + o.dfs[o.dpar[q]]];
                        ce[g] = a * invd[g];
                    } else {
                        ck[g] = 0.0;
                        ce[g] = 0.0;
                    }
                }
            }
            if (sim->implicit)   // diagonal: add every axial conductance the CV takes part in
                for (int32_t q = 1; q < n; ++q) {
                    const int64_t g = off + o.dfs[q];
                    ce[g] += sigma[g];
                    ce[off + o.dfs[o.dpar[q]]] += sigma[g];
                }
        });
    }

    // ------------------------------------------------------------------ packing
    // Cells are grouped into packs (one warp each). A pack's working set (scaled right-hand
    // side per entry, the voltages that are read, synapse and HH states) must fit the shared
    // memory a warp gets; groups that do not fit are split, and a single cell that still does
    // not fit runs from global memory. Among candidate group sizes the one with the smallest
    // estimated per-SM FP64 work (longest-processing-time assignment) is kept.
    const int n_sm = 148;
    const int wpc = 2;                                         // warps per CTA, one CTA per SM
    const int64_t budget = p.smem_budget > 0 ? ((int64_t)p.smem_budget & ~(int64_t)7)
                                             : (((int64_t)227 * 1024 / wpc) & ~(int64_t)7);
    const int64_t mtb = sim->mixed ? 4 : 8;
    Plan& pl = sim->plan;
    pl.tile_doubles = (int)(budget / 8);
    const int32_t nsyn_all = (int32_t)sim->u_cv.size();     // synapse state units
    std::vector<int32_t> cell_of(ncv);
    for (int32_t c = 0; c < nc; ++c)
        for (int64_t i = sim->cv_offset[c]; i < sim->cv_offset[c + 1]; ++i) cell_of[i] = c;
    std::vector<std::vector<int32_t>> cell_syn(nc), cell_hh(nc), cell_st(nc);
    for (int32_t i = 0; i < nsyn_all; ++i) cell_syn[cell_of[sim->u_cv[i]]].push_back(i);
    for (size_t i = 0; i < sim->hh_cv.size(); ++i) cell_hh[cell_of[sim->hh_cv[i]]].push_back((int32_t)i);
    for (size_t i = 0; i < sim->st_cv.size(); ++i) cell_st[cell_of[sim->st_cv[i]]].push_back((int32_t)i);
    std::vector<char> cv_has_mech(ncv, 0);
    for (int64_t cv : sim->syn_cv) cv_has_mech[cv] = 1;
    for (int64_t cv : sim->hh_cv) cv_has_mech[cv] = 1;
    for (int64_t cv : sim->det_cv) cv_has_mech[cv] = 1;

    struct Group {
        std::vector<int32_t> cells;
        PackRows rows;
        std::array<std::vector<int32_t>, 32> syn_l, st_l;
        std::vector<int32_t> hh;
        int64_t nsyn_row = 0, nhh_row = 0, nst_row = 0, nvc = 0;
        int64_t bytes = 0;   // shared-memory tile
        bool smem = false;
        double cost = 0;
    };
    // lanes of grouped items: items on one CV stay on one lane (no two lanes update one slot in
    // a loop); groups by CV, largest first, onto the least loaded lane
    auto assign_grouped = [&](const std::vector<int32_t>& items, const int64_t* item_cv,
                              std::array<std::vector<int32_t>, 32>& lanes) {
        for (auto& v : lanes) v.clear();
        std::vector<int32_t> it = items;
        std::stable_sort(it.begin(), it.end(), [&](int32_t x, int32_t y) { return item_cv[x] < item_cv[y]; });
        std::vector<std::pair<size_t, size_t>> grp;   // [begin, end) in it
        for (size_t i = 0; i < it.size(); ++i) {
            if (i == 0 || item_cv[it[i]] != item_cv[it[i - 1]]) grp.push_back({i, i});
            grp.back().second = i + 1;
        }
        std::stable_sort(grp.begin(), grp.end(), [](const auto& x, const auto& y) {
            return x.second - x.first > y.second - y.first;
        });
        std::array<int64_t, 32> load{};
        for (auto& g : grp) {
            int best = 0;
            for (int l = 1; l < 32; ++l) if (load[l] < load[best]) best = l;
            for (size_t i = g.first; i < g.second; ++i) lanes[best].push_back(it[i]);
            load[best] += (int64_t)(g.second - g.first);
        }
    };
    auto make_group = [&](const std::vector<int32_t>& cells, bool affinity) {
        Group G;
        G.cells = cells;
        G.rows = affinity ? schedule_affinity(cells, ord, sim->cv_offset) : schedule_shared(cells, ord, sim->cv_offset, 4);
        std::vector<int32_t> sy, st;
        for (int32_t c : cells) {
            sy.insert(sy.end(), cell_syn[c].begin(), cell_syn[c].end());
            st.insert(st.end(), cell_st[c].begin(), cell_st[c].end());
            G.hh.insert(G.hh.end(), cell_hh[c].begin(), cell_hh[c].end());
        }
        assign_grouped(sy, sim->u_cv.data(), G.syn_l);
        assign_grouped(st, sim->st_cv.data(), G.st_l);
        for (int l = 0; l < 32; ++l) {
            G.nsyn_row = std::max<int64_t>(G.nsyn_row, (int64_t)G.syn_l[l].size());
            G.nst_row = std::max<int64_t>(G.nst_row, (int64_t)G.st_l[l].size());
        }
        G.nhh_row = ((int64_t)G.hh.size() + 31) / 32;
        // voltages read on chip: mechanism and detector CVs, and parents of chains handed over
        const int64_t J = (int64_t)G.rows.rows.size();
        std::vector<char> need;
        int64_t nvc = 0;
        {
            std::vector<std::pair<int64_t, int64_t>> pos_of;   // (cv, slot) for the pack
            pos_of.reserve(J * 32);
            for (int64_t j = 0; j < J; ++j)
                for (int l = 0; l < 32; ++l)
                    if (G.rows.rows[j][l] >= 0) pos_of.push_back({G.rows.rows[j][l], j * 32 + l});
            std::sort(pos_of.begin(), pos_of.end());
            auto slot_of = [&](int64_t cv) {
                return std::lower_bound(pos_of.begin(), pos_of.end(), std::make_pair(cv, (int64_t)-1))->second;
            };
            need.assign(J * 32, 0);
            for (auto& cs : pos_of) {
                const int64_t cv = cs.first, sl = cs.second;
                if (cv_has_mech[cv]) need[sl] = 1;
                const int32_t c = cell_of[cv];
                const int32_t pi = sim->parent[cv];
                if (pi >= 0) {
                    const int64_t psl = slot_of(sim->cv_offset[c] + pi);
                    if (psl != sl + 32) need[psl] = 1;
                }
            }
            for (char x : need) nvc += x;
        }
        G.nvc = nvc;
        const int64_t bytes = 8 * (J * 32 * (sim->implicit ? 2 : 1) + nvc) + mtb * 32 * (G.nsyn_row + 3 * G.nhh_row);
        G.bytes = bytes;
        G.smem = bytes <= budget && nvc < 0xFFFF && J * 32 <= 0xFFFF;
        G.cost = 3.0 * (double)J + 260.0 * (double)G.nhh_row + 4.0 * (double)G.nsyn_row;
        return G;
    };
    // groups of kpp consecutive cells (largest first); groups that do not fit are halved
    std::function<void(const std::vector<int32_t>&, bool, std::vector<Group>&)> place =
        [&](const std::vector<int32_t>& cells, bool affinity, std::vector<Group>& out) {
            Group G = make_group(cells, affinity);
            if (G.smem || cells.size() == 1) {
                out.push_back(std::move(G));
                return;
            }
            const size_t h = cells.size() / 2;
            place(std::vector<int32_t>(cells.begin(), cells.begin() + h), false, out);
            place(std::vector<int32_t>(cells.begin() + h, cells.end()), false, out);
        };
    std::vector<int32_t> by_size(nc);
    std::iota(by_size.begin(), by_size.end(), 0);
    std::stable_sort(by_size.begin(), by_size.end(), [&](int32_t x, int32_t y) {
        return sim->cv_offset[x + 1] - sim->cv_offset[x] > sim->cv_offset[y + 1] - sim->cv_offset[y];
    });
    auto build_k = [&](int kpp, std::vector<Group>& out) {
        out.clear();
        for (int32_t i = 0; i < nc; i += kpp) {
            std::vector<int32_t> g(by_size.begin() + i, by_size.begin() + std::min<int32_t>(nc, i + kpp));
            place(g, kpp == 32, out);
        }
    };
    // estimated per-SM work of a set of groups: longest-processing-time assignment to the SMs
    // (a static model; Python's autotune_packing times the candidates on the GPU instead)
    auto lpt_cost = [&](const std::vector<Group>& gs) {
        std::vector<double> c;
        double mx = 0;
        for (auto& g : gs) { c.push_back(g.cost); mx = std::max(mx, g.cost); }
        std::sort(c.begin(), c.end(), std::greater<double>());
        std::priority_queue<double, std::vector<double>, std::greater<double>> bins;
        for (int i = 0; i < n_sm; ++i) bins.push(0.0);
        for (double x : c) { double b0 = bins.top(); bins.pop(); bins.push(b0 + x); }
        double ms = 0;
        while (!bins.empty()) { ms = std::max(ms, bins.top()); bins.pop(); }
        return std::max(ms, mx);
    };
    std::vector<Group> groups;
    int kpp = sim->exact ? 32 : p.cells_per_pack;
    if (kpp == 0) {
        if (nc >= 32 * wpc * n_sm) {
            kpp = 32;
        } else {
            double best = INFINITY;
            for (int cand : {16, 12, 8, 6, 4, 3, 2, 1}) {
                std::vector<Group> gs;
                build_k(cand, gs);
                const double cost = lpt_cost(gs);
                if (cost < best * 0.97) { best = cost; kpp = cand; groups = std::move(gs); }
            }
        }
    }
    pl.cells_per_pack = kpp;
    pl.stream = (kpp == 32);
    if (pl.stream) {
        // ---------------------------------------------------------- streamed packs
        // Every array in global memory. Cells up to split_cvs CVs run one per lane, 32 to a pack
        // (largest first), their branch hand-overs on a per-lane stack. Larger cells are spread
        // over the lanes of packs of a few cells: their unbranched chains are list-scheduled in
        // rounds of kStreamRound rows, and hand-overs between chains go through a mailbox in
        // shared memory. Spreading the largest cells keeps any one pack from running much longer
        // than the average load of a warp slot.
        struct SGroup {
            std::vector<int32_t> cells;
            PackRows rows;
            bool shared = false;
        };
        // the kernel variant that will run this plan: its warps per SM and row ring
        const bool ring_path = sim->implicit && !sim->exact;
        int kv_warps = kStreamWarps, kv_ring = 0;
        stream_variant_shape(ring_path, sim->variant, 0, &kv_warps, &kv_ring);
        const int64_t n_slots = (int64_t)n_sm * kv_warps;
        // the row-ring path keeps two doubles per mailbox slot (the voltages reuse the diagonal
        // slot) next to its row ring; the other paths three
        const int64_t mb_max = ring_path
            ? std::min<int64_t>(kMbNone - 1, (227 * 1024 / kv_warps - 16 * (int64_t)kv_ring - 64) / 16)
            : std::min<int64_t>(kMbNone - 1, (227 * 1024 / kv_warps - 64) / 24);
        std::vector<int64_t> ncv_of(nc), depth_of(nc);
        for (int32_t c = 0; c < nc; ++c) {
            ncv_of[c] = sim->cv_offset[c + 1] - sim->cv_offset[c];
            const CellOrder& o = ord[c];
            std::vector<int32_t> dep(o.dfs.size(), 1);
            int64_t mx = 1;
            for (size_t q = 1; q < o.dfs.size(); ++q) {
                dep[q] = dep[o.dpar[q]] + 1;
                mx = std::max<int64_t>(mx, dep[q]);
            }
            depth_of[c] = mx;
        }
        // branch points of a set of cells: an upper bound of its mailbox slots
        auto branch_points = [&](const std::vector<int32_t>& cs) {
            int64_t nb = 0;
            for (int32_t c : cs) {
                std::vector<int32_t> nch(ncv_of[c], 0);
                for (size_t q = 1; q < ord[c].dfs.size(); ++q) nch[ord[c].dpar[q]]++;
                for (int32_t x : nch) nb += x > 1;
            }
            return nb;
        };
        // greedy packs of large cells; a pack whose schedule runs past the target by more than
        // kSpreadOver, or whose mailbox would not fit, is halved
        constexpr double kSpreadOver = 1.25;
        std::function<void(const std::vector<int32_t>&, int64_t, std::vector<SGroup>&)> place_shared =
            [&](const std::vector<int32_t>& cs, int64_t target, std::vector<SGroup>& out) {
                SGroup G;
                G.cells = cs;
                G.shared = true;
                const bool fits = branch_points(cs) <= mb_max;
                if (fits) G.rows = schedule_shared(cs, ord, sim->cv_offset, kStreamRound, ring_path ? 1 : 0);
                if (cs.size() > 1 && (!fits || (double)G.rows.rows.size() > kSpreadOver * (double)target)) {
                    const size_t h = cs.size() / 2;
                    place_shared(std::vector<int32_t>(cs.begin(), cs.begin() + h), target, out);
                    place_shared(std::vector<int32_t>(cs.begin() + h, cs.end()), target, out);
                    return;
                }
                if (!fits) {   // one cell with more branch points than the mailbox holds
                    G.shared = false;
                    G.rows = schedule_affinity(cs, ord, sim->cv_offset);
                }
                out.push_back(std::move(G));
            };
        constexpr double kSpreadFill = 0.95;   // lane-rows holding a CV in a round schedule
        constexpr double kSpreadRow = 1.0;     // cost of a spread pack's solve row (hand-overs cost no FP64 work)
        // Cost model of a pack's run time (measured on the batched workload: the epoch kernel's
        // time follows the makespan of the warp slots under this cost): a solve row costs 1, a row
        // of a pack whose cells are spread over lanes kSpreadRow, and each synapse, HH and clamp row 1.
        std::vector<int64_t> nsyn_of(nc), nhh_of(nc), nst_of(nc);
        for (int32_t c = 0; c < nc; ++c) {
            nsyn_of[c] = (int64_t)cell_syn[c].size();
            nhh_of[c] = (int64_t)cell_hh[c].size();
            nst_of[c] = (int64_t)cell_st[c].size();
        }
        // estimated cost of a pack of cells one per lane (cells[i .. i+32) of a size-sorted list)
        auto est_lane = [&](const std::vector<int32_t>& cs, size_t i) {
            int64_t rows = 0, sy = 0, st = 0, hh = 0;
            for (size_t k = i; k < std::min(cs.size(), i + 32); ++k) {
                const int32_t c = cs[k];
                rows = std::max(rows, ncv_of[c]);
                sy = std::max(sy, nsyn_of[c]);
                st = std::max(st, nst_of[c]);
                hh += nhh_of[c];
            }
            return (double)rows + (double)sy + (double)st + (double)((hh + 31) / 32);
        };
        // Packs of large cells are grouped by estimated cost, not by CVs alone: a cell weighs its
        // solve rows in a round schedule (its CVs over kSpreadFill x 32 lane-rows, x kSpreadRow) plus its
        // mechanism rows spread over the 32 lanes; a group is closed when its weight would pass
        // the target, which is `target` solve rows of a pack of average composition (so a pack
        // of cells with many synapses gets fewer CVs and every pack costs about the same).
        auto spread_weight = [&](int32_t c) {
            return kSpreadRow * (double)ncv_of[c] / (kSpreadFill * 32.0) + 1.1 * (double)(nsyn_of[c] + nst_of[c]) / 32.0 +
                   (double)nhh_of[c] / 32.0;
        };
        auto target_weight = [&](const std::vector<int32_t>& big, int64_t target) {
            double rows = 0.0, mech = 0.0;
            for (int32_t c : big) {
                rows += (double)ncv_of[c] / (kSpreadFill * 32.0);
                mech += 1.1 * (double)(nsyn_of[c] + nst_of[c]) / 32.0 + (double)nhh_of[c] / 32.0;
            }
            return (double)target * (kSpreadRow + (rows > 0.0 ? mech / rows : 0.0));
        };
        // estimated costs of the greedy packs of large cells
        auto est_shared = [&](const std::vector<int32_t>& big, int64_t target, std::vector<double>& cost) {
            const double wt = target_weight(big, target);
            size_t i = 0;
            while (i < big.size()) {
                int64_t sum = 0, dep = 0, sy = 0, hh = 0, st = 0;
                double w = 0.0;
                size_t k = 0;
                while (i + k < big.size() && k < 32) {
                    const int64_t n = ncv_of[big[i + k]];
                    const double wc = spread_weight(big[i + k]);
                    if (k > 0 && w + wc > wt) break;
                    w += wc;
                    sum += n;
                    dep = std::max(dep, depth_of[big[i + k]]);
                    sy += nsyn_of[big[i + k]];
                    hh += nhh_of[big[i + k]];
                    st += nst_of[big[i + k]];
                    ++k;
                }
                const double rows = std::max((double)sum / (kSpreadFill * 32.0), (double)(dep + kStreamRound));
                cost.push_back(kSpreadRow * rows + 1.1 * (double)(sy + st) / 32.0 + (double)((hh + 31) / 32));
                i += k;
            }
        };
        auto makespan = [&](std::vector<double> c) {
            std::sort(c.begin(), c.end(), std::greater<double>());
            std::priority_queue<double, std::vector<double>, std::greater<double>> bins;
            for (int64_t i = 0; i < n_slots; ++i) bins.push(0.0);
            double ms = 0;
            for (double x : c) {
                const double b0 = bins.top() + x;
                bins.pop();
                bins.push(b0);
                ms = std::max(ms, b0);
            }
            return ms;
        };
        // estimated makespan with cells above thr spread into packs of about `target` rows
        auto plan_cost = [&](int64_t thr, int64_t target) {
            std::vector<int32_t> big, rest;
            for (int32_t c : by_size) ((thr > 0 && ncv_of[c] > thr) ? big : rest).push_back(c);
            std::vector<double> cost;
            for (size_t i = 0; i < rest.size(); i += 32) cost.push_back(est_lane(rest, i));
            if (!big.empty()) est_shared(big, target, cost);
            return makespan(cost);
        };
        int64_t split = sim->exact ? -1 : p.split_cvs;
        int64_t target = p.spread_rows > 0 ? p.spread_rows : split;
        if (split == 0) {
            // choose the threshold and the spread packs' rows with the smallest estimated makespan
            // over the warp slots
            double sumc = 0;
            for (size_t i = 0; i < by_size.size(); i += 32) sumc += est_lane(by_size, i);
            const double avg = std::max(1.0, sumc / (double)n_slots);
            double best = plan_cost(-1, 0);
            split = -1;
            target = 0;
            // spread-pack rows: the threshold itself, or rows whose estimated cost (with the
            // mechanism rows of an average pack of the spread cells) is about the average cost of
            // a warp slot, a little below it, or above it
            for (double f : {2.0, 1.5, 1.25, 1.0, 0.8, 0.65, 0.5, 0.4}) {
                const int64_t thr = std::max<int64_t>(1, (int64_t)(f * avg));
                std::vector<int32_t> big;
                for (int32_t c : by_size) if (ncv_of[c] > thr) big.push_back(c);
                if (big.empty()) continue;
                const double per_row = target_weight(big, 1);      // cost of one target row
                for (double g : {0.0, 0.85, 0.92, 1.0, 1.08}) {
                    if (g != 0.0 && p.spread_rows > 0) continue;
                    const int64_t tg = p.spread_rows > 0 ? p.spread_rows
                                                         : (g == 0.0 ? thr : std::max<int64_t>(1, (int64_t)(g * avg / per_row)));
                    const double ms = plan_cost(thr, tg);
                    if (ms < best * 0.995) { best = ms; split = thr; target = tg; }
                }
            }
        }
        if (target <= 0) target = split;
        std::vector<SGroup> sg;
        {
            std::vector<int32_t> big, rest;
            for (int32_t c : by_size) ((split > 0 && ncv_of[c] > split) ? big : rest).push_back(c);
            std::vector<std::vector<int32_t>> cand;   // greedy groups of large cells
            const double wt = target_weight(big, target);
            size_t i = 0;
            while (i < big.size()) {
                std::vector<int32_t> g;
                double w = 0.0;
                while (i < big.size() && g.size() < 32) {
                    const double wc = spread_weight(big[i]);
                    if (!g.empty() && w + wc > wt) break;
                    g.push_back(big[i]);
                    w += wc;
                    ++i;
                }
                cand.push_back(std::move(g));
            }
            // schedule the groups on host threads; the results keep the groups' order
            std::vector<std::vector<SGroup>> placed(cand.size());
            parallel_for((int64_t)cand.size(), [&](int64_t k) { place_shared(cand[k], target, placed[k]); });
            for (auto& v : placed)
                for (auto& G : v) sg.push_back(std::move(G));
            for (size_t r = 0; r < rest.size(); r += 32) {
                SGroup G;
                G.cells.assign(rest.begin() + r, rest.begin() + std::min(rest.size(), r + 32));
                G.rows = schedule_affinity(G.cells, ord, sim->cv_offset);
                sg.push_back(std::move(G));
            }
        }
        pl.spread_rows = split > 0 ? target : -1;
        // the persistent kernel takes packs in order: most expensive first (the cost model above,
        // with the pack's scheduled rows)
        {
            std::vector<double> pc(sg.size());
            parallel_for((int64_t)sg.size(), [&](int64_t k) {
                const SGroup& G = sg[k];
                int64_t hh = 0;
                if (G.shared) {
                    int64_t s_all = 0, t_all = 0;
                    for (int32_t c : G.cells) { s_all += nsyn_of[c]; t_all += nst_of[c]; hh += nhh_of[c]; }
                    pc[k] = kSpreadRow * (double)G.rows.rows.size() + 1.1 * (double)(s_all + t_all) / 32.0 + (double)((hh + 31) / 32);
                } else {
                    int64_t ms = 0, mt = 0;
                    for (size_t l = 0; l < G.cells.size() && l < 32; ++l) {
                        ms = std::max(ms, nsyn_of[G.cells[l]]);
                        mt = std::max(mt, nst_of[G.cells[l]]);
                        hh += nhh_of[G.cells[l]];
                    }
                    pc[k] = (double)G.rows.rows.size() + (double)(ms + mt) + (double)((hh + 31) / 32);
                }
            });
            std::vector<int64_t> ordp(sg.size());
            std::iota(ordp.begin(), ordp.end(), 0);
            std::stable_sort(ordp.begin(), ordp.end(), [&](int64_t x, int64_t y) { return pc[x] > pc[y]; });
            std::vector<SGroup> sorted;
            sorted.reserve(sg.size());
            for (int64_t k : ordp) sorted.push_back(std::move(sg[k]));
            sg = std::move(sorted);
        }
        const int32_t npk = (int32_t)sg.size();
        pl.packs.resize(npk);
        par_assign(pl.cv_tile, ncv, (int64_t)-1);
        par_assign(pl.cv_pack, ncv, (int32_t)-1);
        std::vector<std::array<std::vector<int32_t>, 32>> syn_l(npk), st_l(npk);
        std::vector<std::vector<int32_t>> hh_l(npk);
        std::vector<int64_t> prow0(npk + 1, 0);        // first row of each pack
        for (int32_t pi = 0; pi < npk; ++pi) prow0[pi + 1] = prow0[pi] + (int64_t)sg[pi].rows.rows.size();
        parallel_for(npk, [&](int64_t pi) {          // packs own their rows, CVs and lists
            const SGroup& G = sg[pi];
            const int32_t J = (int32_t)G.rows.rows.size();
            const int64_t row0 = prow0[pi];
            PackDesc& pd = pl.packs[pi];
            std::memset(&pd, 0, sizeof(pd));
            pd.row0 = (int32_t)row0;
            pd.nrow = J;
            pd.round_rows = G.shared ? kStreamRound : 0;
            pd.smem = kPackStream;
            pd.sg_off = row0 * kWarp;
            pd.ncell = (int32_t)G.cells.size();
            for (int32_t j = 0; j < J; ++j)
                for (int l = 0; l < kWarp; ++l) {
                    const int64_t cv = G.rows.rows[j][l];
                    if (cv < 0) continue;
                    pl.cv_tile[cv] = (row0 + j) * kWarp + l;
                    pl.cv_pack[cv] = pi;
                }
            std::vector<int32_t> sy, st;
            for (int32_t c : G.cells) {
                sy.insert(sy.end(), cell_syn[c].begin(), cell_syn[c].end());
                st.insert(st.end(), cell_st[c].begin(), cell_st[c].end());
                hh_l[pi].insert(hh_l[pi].end(), cell_hh[c].begin(), cell_hh[c].end());
            }
            if (!sim->exact) {
                assign_grouped(sy, sim->u_cv.data(), syn_l[pi]);
                assign_grouped(st, sim->st_cv.data(), st_l[pi]);
            } else {
                // every lane holds its own cell's synapses (by CV) and clamps
                for (size_t l = 0; l < G.cells.size(); ++l) {
                    const int32_t c = G.cells[l];
                    syn_l[pi][l] = cell_syn[c];
                    std::stable_sort(syn_l[pi][l].begin(), syn_l[pi][l].end(),
                                     [&](int32_t x, int32_t y) { return sim->u_cv[x] < sim->u_cv[y]; });
                    st_l[pi][l] = cell_st[c];
                }
            }
        });
        const int64_t row0 = prow0[npk];
        pl.total_rows = row0;
        const int64_t ne = row0 * kWarp;
        if (ne > INT32_MAX) return bad("model too large for one handle");
        for (int64_t cv = 0; cv < ncv; ++cv)
            if (pl.cv_tile[cv] < 0) return bad("internal error: a CV was not placed");
        pl.lane_eff = row0 > 0 ? (double)ncv / (double)ne : 1.0;
        pl.sg_total = ne;
        par_assign(pl.ca, ne, 0.0);
        par_assign(pl.cb, ne, 0.0);
        par_assign(pl.ck, ne, 0.0);
        par_assign(pl.ce, ne, sim->implicit ? 1.0 : 0.0);
        par_assign(pl.pslot, ne, (int32_t)kFlagRoot);   // flags; padding behaves like an isolated root
        par_assign(pl.vmap, ne, (int32_t)-1);           // compact mechanism slot
        par_assign(pl.V0, ne, 0.0);
        const uint32_t mb_out_mask = (uint32_t)kMbNone << kMbOutShift, mb_in_mask = (uint32_t)kMbNone << kMbInShift;
        for (int32_t pi = 0; pi < npk; ++pi)
            if (sg[pi].shared) {
                const int64_t base = (int64_t)pl.packs[pi].row0 * kWarp;
                for (int64_t t = base; t < base + (int64_t)pl.packs[pi].nrow * kWarp; ++t)
                    pl.pslot[t] = (int32_t)((uint32_t)kFlagRoot | mb_out_mask | mb_in_mask);
            }
        // per-entry constants; flags from the layout: an entry whose parent is not the next row
        // of its lane hands over (stack or mailbox)
        std::vector<int32_t> nmb(npk, 0);
        std::vector<char> err(npk, 0);     // 1: a CV with more than 255 handed-over children, 2: mailbox full
        parallel_for(npk, [&](int64_t pi) {   // packs own disjoint entries
            const bool shared = sg[pi].shared;
            for (int32_t c : sg[pi].cells) {
                const int64_t off = sim->cv_offset[c];
                for (int64_t i = 0; i < ncv_of[c]; ++i) {
                    const int64_t g = off + i;
                    const int64_t t = pl.cv_tile[g];
                    pl.ca[t] = ca[g];
                    pl.cb[t] = cb[g];
                    pl.ck[t] = ck[g];
                    pl.ce[t] = ce[g];
                    pl.V0[t] = -65.0;
                }
                for (int64_t i = 0; i < ncv_of[c]; ++i) {
                    const int64_t g = off + i;
                    const int64_t t = pl.cv_tile[g];
                    int32_t& f = pl.pslot[t];   // parents come before children: their counts and "in" slots are kept
                    f &= shared ? (int32_t)mb_in_mask : kFlagPopMask;
                    if (shared) f |= (int32_t)mb_out_mask;
                    if (sim->parent[g] < 0) {
                        f |= kFlagRoot;
                        continue;
                    }
                    const int64_t tp = pl.cv_tile[off + sim->parent[g]];
                    if (tp == t + kWarp) continue;   // parent is the next row of this lane
                    f |= kFlagRemote;
                    int32_t& fp = pl.pslot[tp];
                    if (!shared) {
                        if ((fp & kFlagPopMask) == kFlagPopMask) { err[pi] = 1; return; }
                        fp += 1;
                    } else {
                        // the parent's "in" slot, assigned by its first handed-over child
                        uint32_t sl = (uint32_t)fp >> kMbInShift;
                        if (sl == (uint32_t)kMbNone) {
                            sl = (uint32_t)nmb[pi]++;
                            if (sl >= (uint32_t)kMbNone) { err[pi] = 2; return; }
                            fp = (int32_t)(((uint32_t)fp & ~mb_in_mask) | (sl << kMbInShift));
                        }
                        f = (int32_t)(((uint32_t)f & ~mb_out_mask) | (sl << kMbOutShift));
                    }
                }
            }
        });
        for (int32_t pi = 0; pi < npk; ++pi) {
            if (err[pi] == 1) return bad("a CV has more than 255 handed-over children");
            if (err[pi] == 2) return bad("internal error: mailbox overflow");
        }
        // mailbox slots of all packs, numbered pack after pack (each slot's parent entry and
        // compact mechanism slot are filled in below)
        int64_t mb_total = 0;
        for (int32_t pi = 0; pi < npk; ++pi) {
            pl.packs[pi].mb0 = (int32_t)mb_total;
            mb_total += sg[pi].shared ? nmb[pi] : 0;
            if (mb_total > INT32_MAX) return bad("model too large for one handle");
        }
        pl.mb_ent.assign((size_t)std::max<int64_t>(mb_total, 1), 0);
        pl.mb_cs.assign((size_t)std::max<int64_t>(mb_total, 1), -1);
        // compact mechanism slots; stack depths (one cell per lane) and the round rule of the
        // mailbox (cells over several lanes)
        std::vector<char> mech(ncv, 0);
        for (int64_t cv : sim->hh_cv) mech[cv] = 1;
        for (int64_t cv : sim->st_cv) mech[cv] = 1;
        for (int64_t cv : sim->syn_cv) mech[cv] = 2;     // 2: the CV has synapses
        int64_t c_total = 0;
        int32_t max_depth = 1, max_mb = 0;
        pl.slot_lo.assign((size_t)npk * kWarp, 0);
        pl.slot_hi.assign((size_t)npk * kWarp, 0);
        // per pack, in parallel: pack-relative compact slots, and the checks of its schedule
        std::vector<int32_t> p_nvc(npk, 0), p_depth(npk, 0);
        std::vector<char> p_err(npk, 0);
        parallel_for(npk, [&](int64_t pi) {
            PackDesc& pd = pl.packs[pi];
            const int64_t base = (int64_t)pd.row0 * kWarp;
            int32_t nvc = 0;
            // mechanism entries are marked -3 (with synapses) or -2 (without), then numbered
            for (int32_t c : sg[pi].cells)
                for (int64_t cv = sim->cv_offset[c]; cv < sim->cv_offset[c + 1]; ++cv)
                    if (mech[cv]) pl.vmap[pl.cv_tile[cv]] = mech[cv] == 2 ? -3 : -2;
            pd.nsc = 0;
            if (!sim->exact) {
                // CVs with synapses first: the synapse pass writes their slots' terms whole
                for (int64_t t = base; t < base + (int64_t)pd.nrow * kWarp; ++t)
                    if (pl.vmap[t] == -3) pl.vmap[t] = nvc++;
                pd.nsc = nvc;
                for (int64_t t = base; t < base + (int64_t)pd.nrow * kWarp; ++t)
                    if (pl.vmap[t] == -2) pl.vmap[t] = nvc++;
            } else {
                for (int64_t t = base; t < base + (int64_t)pd.nrow * kWarp; ++t)
                    if (pl.vmap[t] < -1) pl.vmap[t] = -2;
                // lane by lane, so that each lane's slots are one range of its own
                for (int l = 0; l < kWarp; ++l) {
                    pl.slot_lo[(size_t)pi * kWarp + l] = nvc;
                    for (int32_t j = 0; j < pd.nrow; ++j) {
                        const int64_t t = base + (int64_t)j * kWarp + l;
                        if (pl.vmap[t] == -2) pl.vmap[t] = nvc++;
                    }
                    pl.slot_hi[(size_t)pi * kWarp + l] = nvc;
                }
            }
            p_nvc[pi] = nvc;
            if (sg[pi].shared) {
                pd.nmb = nmb[pi];
                // a hand-over between lanes is written (on the row-ring path: one row after the
                // child, see schedule_shared) in an earlier round than the parent reads it, and
                // within a round at most one lane adds to a given slot
                const int32_t wsh = ring_path ? 1 : 0;
                std::vector<int32_t> w_round(pd.nmb, -1), w_lane(pd.nmb, -1);   // last writer of each slot
                for (int32_t j = 0; j < pd.nrow; ++j)
                    for (int l = 0; l < kWarp; ++l) {
                        const int32_t f = pl.pslot[base + (int64_t)j * kWarp + l];
                        const int32_t so = (f >> kMbOutShift) & kMbNone, si = (int32_t)((uint32_t)f >> kMbInShift);
                        if ((so != kMbNone && so >= pd.nmb) || (si != kMbNone && si >= pd.nmb) || (f & kFlagPopMask)) {
                            p_err[pi] = 1;
                            return;
                        }
                        if (!(f & kFlagRemote) || (f & kFlagRoot)) continue;
                        if (so == kMbNone) { p_err[pi] = 2; return; }
                        if (j + wsh >= pd.nrow) { p_err[pi] = 5; return; }
                        const int32_t rd = (j + wsh) / kStreamRound;
                        if (w_round[so] == rd && w_lane[so] != l) { p_err[pi] = 3; return; }
                        w_round[so] = rd;
                        w_lane[so] = l;
                    }
                for (int32_t c : sg[pi].cells)
                    for (int64_t cv = sim->cv_offset[c] + 1; cv < sim->cv_offset[c + 1]; ++cv) {
                        const int64_t t = pl.cv_tile[cv], tp = pl.cv_tile[sim->cv_offset[c] + sim->parent[cv]];
                        if (t % kWarp == tp % kWarp) {
                            if (tp <= t) { p_err[pi] = 4; return; }
                        } else if ((t / kWarp - pd.row0 + wsh) / kStreamRound >= (tp / kWarp - pd.row0) / kStreamRound) {
                            p_err[pi] = 5;
                            return;
                        }
                    }
                // the slot's parent: its entry in the pack and its compact mechanism slot, from
                // which the kernel starts the slot's sums each step
                for (int64_t t = base; t < base + (int64_t)pd.nrow * kWarp; ++t) {
                    const int32_t si = (int32_t)((uint32_t)pl.pslot[t] >> kMbInShift);
                    if (si == kMbNone) continue;
                    pl.mb_ent[(size_t)pd.mb0 + si] = (int32_t)(t - base);
                    pl.mb_cs[(size_t)pd.mb0 + si] = pl.vmap[t];
                }
                pd.stack = 0;
                return;
            }
            int32_t depth = 0;
            for (int l = 0; l < kWarp; ++l) {
                int32_t sp = 0;
                for (int32_t j = 0; j < pd.nrow; ++j) {                 // forward
                    const int32_t f = pl.pslot[base + (int64_t)j * kWarp + l];
                    sp -= f & kFlagPopMask;
                    if (sp < 0) { p_err[pi] = 6; return; }
                    if ((f & kFlagRemote) && !(f & kFlagRoot)) ++sp;
                    depth = std::max(depth, sp);
                }
                sp = 0;
                for (int32_t j = pd.nrow - 1; j >= 0; --j) {            // backward
                    const int32_t f = pl.pslot[base + (int64_t)j * kWarp + l];
                    if ((f & kFlagRemote) && !(f & kFlagRoot)) --sp;
                    if (sp < 0) { p_err[pi] = 7; return; }
                    sp += f & kFlagPopMask;
                    depth = std::max(depth, sp);
                }
            }
            pd.stack = depth;
            p_depth[pi] = depth;
        });
        static const char* const kPlanErr[] = {"", "mailbox slot out of range", "hand-over without a mailbox slot",
                                               "two lanes add to one mailbox slot in a round", "parent before child on a lane",
                                               "cross-lane hand-over inside one round", "hand-over stack underflow",
                                               "voltage stack underflow"};
        for (int32_t pi = 0; pi < npk; ++pi)
            if (p_err[pi]) return bad(std::string("internal error: ") + kPlanErr[(int)p_err[pi]]);
        for (int32_t pi = 0; pi < npk; ++pi) {
            PackDesc& pd = pl.packs[pi];
            pd.nvc = p_nvc[pi];
            pd.c_off = c_total;
            c_total += p_nvc[pi];
            max_depth = std::max(max_depth, p_depth[pi]);
            if (sg[pi].shared) max_mb = std::max(max_mb, nmb[pi]);
        }
        // constant diagonal and right-hand side of every compact slot
        pl.cE.assign(c_total, 0.0);
        pl.cB.assign(c_total, 0.0);
        parallel_for(npk, [&](int64_t pi) {
            const PackDesc& pd = pl.packs[pi];
            const int64_t base = (int64_t)pd.row0 * kWarp;
            for (int64_t t = base; t < base + (int64_t)pd.nrow * kWarp; ++t)
                if (pl.vmap[t] >= 0) {
                    pl.cE[pd.c_off + pl.vmap[t]] = pl.ce[t];
                    pl.cB[pd.c_off + pl.vmap[t]] = pl.cb[t];
                }
        });
        pl.c_total = c_total;
        if (ring_path) {
            // slots are numbered row by row (synapse CVs first, then the others), so a row's slots
            // are two contiguous ranges; each entry's position in the row's list of them
            par_assign(pl.cpos, pl.total_rows * kWarp, (int32_t)-1);
            par_assign(pl.row_cs, pl.total_rows, (int32_t)0);
            par_assign(pl.row_cn, pl.total_rows, (int32_t)0);
            std::vector<char> r_err(npk, 0);
            parallel_for(npk, [&](int64_t pi) {
                const PackDesc& pd = pl.packs[pi];
                int32_t next_s = 0, next_n = pd.nsc;
                for (int32_t j = 0; j < pd.nrow; ++j) {
                    const int64_t r = (int64_t)pd.row0 + j;
                    int32_t ns = 0, nn = 0;
                    const int32_t s0 = next_s, n0 = next_n;
                    for (int l = 0; l < kWarp; ++l) {
                        const int32_t c = pl.vmap[r * kWarp + l];
                        if (c >= 0 && c < pd.nsc) {
                            if (c != next_s) r_err[pi] = 1;
                            pl.cpos[r * kWarp + l] = ns++;
                            ++next_s;
                        }
                    }
                    for (int l = 0; l < kWarp; ++l) {
                        const int32_t c = pl.vmap[r * kWarp + l];
                        if (c >= pd.nsc) {
                            if (c != next_n) r_err[pi] = 1;
                            pl.cpos[r * kWarp + l] = ns + nn++;
                            ++next_n;
                        }
                    }
                    if (s0 >= (1 << 24) || n0 - pd.nsc >= (1 << 24)) r_err[pi] = 1;
                    pl.row_cs[r] = s0 | (ns << 24);
                    pl.row_cn[r] = (n0 - pd.nsc) | (nn << 24);
                }
            });
            for (char e : r_err)
                if (e) return bad("internal error: compact slots are not numbered row by row");
        }
        pl.stack_depth = max_depth;
        pl.stream_imp = ring_path;
        // per warp: the hand-over stack (row-ring path: three planes K, e, u of [depth][32]
        // doubles; otherwise [depth][32] double2) or the mailbox of cells spread over lanes
        const int64_t stack_d2 = ring_path ? ((int64_t)3 * max_depth * kWarp + 1) / 2 : (int64_t)max_depth * kWarp;
        pl.warp_smem = std::max<int64_t>(stack_d2, ((int64_t)(ring_path ? 2 : 3) * max_mb + 1) / 2);
        pl.split_cvs = split;
        pl.smem_packs = 0;
        for (const SGroup& G : sg) pl.smem_packs += G.shared;
        // mechanisms: synapse and clamp rows by CV on one lane; HH round-robin
        int64_t syn_rows = 0, hh_rows = 0, st_rows = 0;
        for (int32_t pi = 0; pi < npk; ++pi) {
            PackDesc& pd = pl.packs[pi];
            size_t ms = 0, mt = 0;
            for (int l = 0; l < 32; ++l) { ms = std::max(ms, syn_l[pi][l].size()); mt = std::max(mt, st_l[pi][l].size()); }
            pd.syn_row0 = (int32_t)syn_rows; pd.nsyn_row = (int32_t)ms; syn_rows += (int64_t)ms;
            pd.hh_row0 = (int32_t)hh_rows;
            if (!sim->exact) {
                pd.nhh_row = (int32_t)((hh_l[pi].size() + 31) / 32);
            } else {                    // each lane's own cell's instances, one per row
                pd.nhh_row = 0;
                for (int32_t c : sg[pi].cells) pd.nhh_row = std::max<int32_t>(pd.nhh_row, (int32_t)cell_hh[c].size());
            }
            hh_rows += pd.nhh_row;
            pd.st_row0 = (int32_t)st_rows; pd.nst_row = (int32_t)mt; st_rows += (int64_t)mt;
        }
        pl.syn_rows = syn_rows; pl.hh_rows = hh_rows; pl.st_rows = st_rows;
        pl.syn_entry.assign(nsyn_all, -1); pl.syn_owner.assign(nsyn_all, 0); pl.syn_js.assign(nsyn_all, 0);
        pl.hh_entry.assign(sim->hh_cv.size(), -1);
        pl.syn_slot.assign(syn_rows * kWarp, -1); pl.syn_vs.assign(syn_rows * kWarp, -1);
        pl.syn_e.assign(syn_rows * kWarp, 0.0); pl.syn_decay.assign(syn_rows * kWarp, 0.0); pl.syn_ntau.assign(syn_rows * kWarp, 0.0); pl.syn_sc.assign(syn_rows * kWarp, 0.0);
        pl.hh_slot.assign(hh_rows * kWarp, -1); pl.hh_vs.assign(hh_rows * kWarp, -1);
        pl.hh_sc.assign(hh_rows * kWarp, 0.0); pl.hh_gna.assign(hh_rows * kWarp, 0.0); pl.hh_gk.assign(hh_rows * kWarp, 0.0);
        pl.st_slot.assign(st_rows * kWarp, -1); pl.st_sc.assign(st_rows * kWarp, 0.0);
        pl.st_on.assign(st_rows * kWarp, 0.0); pl.st_off.assign(st_rows * kWarp, 0.0); pl.st_amp.assign(st_rows * kWarp, 0.0);
        pl.det_slot.assign((size_t)npk * kWarp, -1); pl.det_gid.assign((size_t)npk * kWarp, -1);
        std::atomic<int> slot_err{0};
        parallel_for(npk, [&](int64_t pi) {          // packs own their rows and instances
            const PackDesc& pd = pl.packs[pi];
            const int64_t base = (int64_t)pd.row0 * kWarp;
            for (int l = 0; l < 32; ++l) {
                const auto& v = syn_l[pi][l];
                for (size_t rr = 0; rr < v.size(); ++rr) {
                    const int32_t i = v[rr];
                    const int64_t q = ((int64_t)pd.syn_row0 + (int64_t)rr) * kWarp + l;
                    const int64_t cv = sim->u_cv[i];
                    pl.syn_slot[q] = (int32_t)(pl.cv_tile[cv] - base);
                    pl.syn_vs[q] = pl.vmap[pl.cv_tile[cv]];
                    if (!sim->exact && (pl.syn_vs[q] < 0 || pl.syn_vs[q] >= pd.nsc)) slot_err = 1;
                    pl.syn_e[q] = sim->u_e[i];
                    pl.syn_decay[q] = std::exp(-p.dt / sim->u_tau[i]);
                    pl.syn_ntau[q] = -1.0 / sim->u_tau[i];
                    pl.syn_sc[q] = invd[cv];
                    pl.syn_entry[i] = q;
                    pl.syn_owner[i] = (int32_t)(pi * kWarp + l);
                    pl.syn_js[i] = (int32_t)rr;
                }
                const auto& w = st_l[pi][l];
                for (size_t rr = 0; rr < w.size(); ++rr) {
                    const int32_t i = w[rr];
                    const int64_t q = ((int64_t)pd.st_row0 + (int64_t)rr) * kWarp + l;
                    const int64_t cv = sim->st_cv[i];
                    pl.st_slot[q] = pl.vmap[pl.cv_tile[cv]];
                    pl.st_sc[q] = invd[cv];
                    pl.st_on[q] = sim->st_on[i];
                    pl.st_off[q] = sim->st_on[i] + sim->st_dur[i];
                    pl.st_amp[q] = sim->st_amp[i];
                }
            }
            std::vector<std::pair<int32_t, int64_t>> hh_at;   // (instance, entry)
            if (!sim->exact) {
                for (size_t rr = 0; rr < hh_l[pi].size(); ++rr)
                    hh_at.push_back({hh_l[pi][rr], ((int64_t)pd.hh_row0 + (int64_t)(rr / 32)) * kWarp + (int64_t)(rr % 32)});
            } else {
                for (size_t l = 0; l < sg[pi].cells.size(); ++l) {
                    const auto& v = cell_hh[sg[pi].cells[l]];
                    for (size_t rr = 0; rr < v.size(); ++rr) hh_at.push_back({v[rr], ((int64_t)pd.hh_row0 + (int64_t)rr) * kWarp + (int64_t)l});
                }
            }
            for (const auto& hq : hh_at) {
                const int32_t i = hq.first;
                const int64_t q = hq.second;
                const int64_t cv = sim->hh_cv[i];
                pl.hh_slot[q] = (int32_t)(pl.cv_tile[cv] - base);
                pl.hh_vs[q] = pl.vmap[pl.cv_tile[cv]];
                pl.hh_sc[q] = invd[cv];
                pl.hh_gna[q] = hh_gna[i];
                pl.hh_gk[q] = hh_gk[i];
                pl.hh_entry[i] = q;
            }
            for (size_t dd = 0; dd < sg[pi].cells.size(); ++dd) {
                pl.det_slot[(size_t)pi * kWarp + dd] = (int32_t)(pl.cv_tile[sim->det_cv[sg[pi].cells[dd]]] - base);
                pl.det_gid[(size_t)pi * kWarp + dd] = sg[pi].cells[dd];
            }
        });
        if (slot_err) return bad("internal error: a synapse slot outside the pack's synapse slots");
    } else {
    if (groups.empty() && nc > 0) build_k(kpp, groups);
    {   // per-warp tile: the largest shared-memory pack's need, so that more warps fit an SM
        int64_t need = 0;
        for (const Group& G : groups) if (G.smem) need = std::max(need, G.bytes);
        if (need > 0) pl.tile_doubles = (int)(((need + 31) & ~(int64_t)31) / 8);
    }
    const int32_t npk = (int32_t)groups.size();
    // the persistent kernel takes packs in this order: most work first
    std::stable_sort(groups.begin(), groups.end(), [](const Group& x, const Group& y) { return x.cost > y.cost; });

    pl.packs.resize(npk);
    par_assign(pl.cv_tile, ncv, (int64_t)-1);
    par_assign(pl.cv_pack, ncv, (int32_t)-1);
    int64_t row0 = 0, cvs_placed = 0, syn_rows = 0, hh_rows = 0, st_rows = 0;
    for (int32_t pi = 0; pi < npk; ++pi) {
        PackDesc& pd = pl.packs[pi];
        const Group& G = groups[pi];
        std::memset(&pd, 0, sizeof(pd));
        pd.row0 = (int32_t)row0;
        pd.nrow = (int32_t)G.rows.rows.size();
        pd.round_rows = G.rows.round_rows;
        pd.smem = G.smem ? 1 : 0;
        if (pd.smem) pl.smem_packs++;
        pd.sg_off = pd.smem ? 0 : pl.sg_total;
        if (!pd.smem) pl.sg_total += (int64_t)pd.nrow * kWarp;
        pd.syn_row0 = (int32_t)syn_rows;
        pd.nsyn_row = (int32_t)G.nsyn_row;
        pd.hh_row0 = (int32_t)hh_rows;
        pd.nhh_row = (int32_t)G.nhh_row;
        pd.st_row0 = (int32_t)st_rows;
        pd.nst_row = (int32_t)G.nst_row;
        pd.ncell = (int32_t)G.cells.size();
        pd.nvc = (int32_t)G.nvc;
        syn_rows += G.nsyn_row;
        hh_rows += G.nhh_row;
        st_rows += G.nst_row;
        for (int32_t j = 0; j < pd.nrow; ++j)
            for (int l = 0; l < kWarp; ++l) {
                const int64_t cv = G.rows.rows[j][l];
                if (cv >= 0) {
                    pl.cv_tile[cv] = (row0 + j) * kWarp + l;
                    pl.cv_pack[cv] = pi;
                    ++cvs_placed;
                }
            }
        row0 += pd.nrow;
    }
    pl.total_rows = row0;
    if (cvs_placed != ncv) return bad("internal error: packing lost CVs");
    pl.lane_eff = pl.total_rows > 0 ? (double)ncv / (double)(pl.total_rows * kWarp) : 1.0;
    const int64_t ne = pl.total_rows * kWarp;
    if (ne > INT32_MAX) return bad("model too large for one handle");
    par_assign(pl.ca, ne, 0.0);
    par_assign(pl.cb, ne, 0.0);
    par_assign(pl.ck, ne, 0.0);
    par_assign(pl.ce, ne, sim->implicit ? 1.0 : 0.0);   // padding: unit diagonal keeps the pivots finite
    par_assign(pl.pslot, ne, (int32_t)-2);
    par_assign(pl.vmap, ne, (int32_t)-1);
    par_assign(pl.V0, ne, 0.0);
    for (int32_t c = 0; c < nc; ++c) {
        const int64_t off = sim->cv_offset[c];
        const int32_t n = (int32_t)(sim->cv_offset[c + 1] - off);
        for (int32_t i = 0; i < n; ++i) {
            const int64_t g = off + i;
            const int64_t t = pl.cv_tile[g];
            pl.ca[t] = ca[g];
            pl.cb[t] = cb[g];
            pl.ck[t] = ck[g];
            pl.ce[t] = ce[g];
            pl.V0[t] = -65.0;
            if (i == 0) {
                pl.pslot[t] = -2;
            } else {
                const int64_t tp = pl.cv_tile[off + sim->parent[g]];
                const int32_t pk = pl.cv_pack[g];
                const int64_t base = (int64_t)pl.packs[pk].row0 * kWarp;
                pl.pslot[t] = (tp == t + kWarp) ? -1 : (int32_t)(tp - base);
            }
        }
    }
    // on-chip voltage slots (shared-memory packs): in tile-slot order
    std::vector<int32_t> vslot_of_cv(ncv, -1);
    {
        std::vector<char> need(ne, 0);
        for (int64_t cv = 0; cv < ncv; ++cv) {
            if (cv_has_mech[cv]) need[pl.cv_tile[cv]] = 1;
            const int32_t c = cell_of[cv];
            const int32_t pi = sim->parent[cv];
            if (pi >= 0 && pl.pslot[pl.cv_tile[cv]] >= 0) need[pl.cv_tile[sim->cv_offset[c] + pi]] = 1;
        }
        for (int32_t pi = 0; pi < npk; ++pi) {
            const PackDesc& pd = pl.packs[pi];
            if (!pd.smem) continue;
            int32_t next = 0;
            for (int64_t t = (int64_t)pd.row0 * kWarp; t < ((int64_t)pd.row0 + pd.nrow) * kWarp; ++t)
                if (need[t]) pl.vmap[t] = next++;            // own slot in the low 16 bits (for now)
            if (next != pd.nvc) return bad("internal error: on-chip voltage count");
        }
        std::vector<int32_t> tile_cv(ne, -1);
        for (int64_t cv = 0; cv < ncv; ++cv) tile_cv[pl.cv_tile[cv]] = (int32_t)cv;
        for (int64_t cv = 0; cv < ncv; ++cv) {
            const int64_t t = pl.cv_tile[cv];
            if (pl.packs[pl.cv_pack[cv]].smem && pl.vmap[t] >= 0) vslot_of_cv[cv] = pl.vmap[t];
        }
        for (int64_t t = 0; t < ne; ++t) {
            const int32_t cv = tile_cv[t];
            uint32_t own = 0xFFFF, par = 0xFFFF;
            if (cv >= 0 && pl.packs[pl.cv_pack[cv]].smem) {
                if (vslot_of_cv[cv] >= 0) own = (uint32_t)vslot_of_cv[cv];
                if (pl.pslot[t] >= 0) {
                    const int32_t c = cell_of[cv];
                    par = (uint32_t)vslot_of_cv[sim->cv_offset[c] + sim->parent[cv]];
                }
            }
            pl.vmap[t] = (int32_t)(own | (par << 16));
        }
    }

    // ------------------------------------------------------------------ schedule check
    // Every hand-over between lanes must cross a round boundary, and within one round at most
    // one lane may add into a given parent slot; violations would be data races in the kernel.
    for (int32_t pi = 0; pi < npk; ++pi) {
        const PackDesc& pd = pl.packs[pi];
        const int64_t base = (int64_t)pd.row0 * kWarp;
        const int R = pd.round_rows;
        std::vector<std::pair<int64_t, int64_t>> targets;   // (round, target slot) of remote writes
        for (int64_t j = 0; j < pd.nrow; ++j)
            for (int l = 0; l < kWarp; ++l) {
                const int64_t t = base + j * kWarp + l;
                const int32_t ps = pl.pslot[t];
                if (ps < 0) continue;
                const int64_t jp = ps / kWarp, lp = ps % kWarp;
                const bool ok = (R == 0) ? (lp == l && jp > j) : (jp / R > j / R);
                if (!ok) return bad("internal error: solve schedule hands over within a round (pack " + std::to_string(pi) + ")");
                if (R > 0) targets.push_back({j / R, ps});
            }
        std::sort(targets.begin(), targets.end());
        for (size_t i = 1; i < targets.size(); ++i)
            if (targets[i] == targets[i - 1]) return bad("internal error: two lanes write one parent in a round");
    }

    // ------------------------------------------------------------------ mechanisms per pack
    pl.syn_rows = syn_rows;
    pl.hh_rows = hh_rows;
    pl.st_rows = st_rows;
    pl.syn_entry.assign(nsyn_all, -1);
    pl.syn_owner.assign(nsyn_all, 0);
    pl.syn_js.assign(nsyn_all, 0);
    pl.hh_entry.assign(sim->hh_cv.size(), -1);
    pl.syn_slot.assign(syn_rows * kWarp, -1);
    pl.syn_vs.assign(syn_rows * kWarp, -1);
    pl.syn_e.assign(syn_rows * kWarp, 0.0);
    pl.syn_decay.assign(syn_rows * kWarp, 0.0); pl.syn_ntau.assign(syn_rows * kWarp, 0.0);
    pl.syn_sc.assign(syn_rows * kWarp, 0.0);
    pl.hh_slot.assign(hh_rows * kWarp, -1);
    pl.hh_vs.assign(hh_rows * kWarp, -1);
    pl.hh_sc.assign(hh_rows * kWarp, 0.0);
    pl.hh_gna.assign(hh_rows * kWarp, 0.0);
    pl.hh_gk.assign(hh_rows * kWarp, 0.0);
    pl.st_slot.assign(st_rows * kWarp, -1);
    pl.st_sc.assign(st_rows * kWarp, 0.0);
    pl.st_on.assign(st_rows * kWarp, 0.0);
    pl.st_off.assign(st_rows * kWarp, 0.0);
    pl.st_amp.assign(st_rows * kWarp, 0.0);
    pl.det_slot.assign((size_t)npk * kWarp, -1);
    pl.det_gid.assign((size_t)npk * kWarp, -1);
    for (int32_t pi = 0; pi < npk; ++pi) {
        const PackDesc& pd = pl.packs[pi];
        const Group& G = groups[pi];
        const int64_t base = (int64_t)pd.row0 * kWarp;
        auto vread = [&](int64_t cv) { return pd.smem ? vslot_of_cv[cv] : (int32_t)(pl.cv_tile[cv] - base); };
        for (int l = 0; l < 32; ++l) {
            const auto& v = G.syn_l[l];
            for (size_t r = 0; r < v.size(); ++r) {
                const int32_t i = v[r];
                const int64_t q = ((int64_t)pd.syn_row0 + (int64_t)r) * kWarp + l;
                const int64_t cv = sim->u_cv[i];
                pl.syn_slot[q] = (int32_t)(pl.cv_tile[cv] - base);
                pl.syn_vs[q] = vread(cv);
                pl.syn_e[q] = sim->u_e[i];
                pl.syn_decay[q] = std::exp(-p.dt / sim->u_tau[i]);
                    pl.syn_ntau[q] = -1.0 / sim->u_tau[i];
                pl.syn_sc[q] = invd[cv];
                pl.syn_entry[i] = q;
                pl.syn_owner[i] = pi * kWarp + l;
                pl.syn_js[i] = (int32_t)r;
            }
            const auto& w = G.st_l[l];
            for (size_t r = 0; r < w.size(); ++r) {
                const int32_t i = w[r];
                const int64_t q = ((int64_t)pd.st_row0 + (int64_t)r) * kWarp + l;
                const int64_t cv = sim->st_cv[i];
                pl.st_slot[q] = (int32_t)(pl.cv_tile[cv] - base);
                pl.st_sc[q] = invd[cv];
                pl.st_on[q] = sim->st_on[i];
                pl.st_off[q] = sim->st_on[i] + sim->st_dur[i];
                pl.st_amp[q] = sim->st_amp[i];
            }
        }
        for (size_t r = 0; r < G.hh.size(); ++r) {
            const int32_t i = G.hh[r];
            const int64_t q = ((int64_t)pd.hh_row0 + (int64_t)(r / 32)) * kWarp + (int64_t)(r % 32);
            const int64_t cv = sim->hh_cv[i];
            pl.hh_slot[q] = (int32_t)(pl.cv_tile[cv] - base);
            pl.hh_vs[q] = vread(cv);
            pl.hh_sc[q] = invd[cv];
            pl.hh_gna[q] = hh_gna[i];
            pl.hh_gk[q] = hh_gk[i];
            pl.hh_entry[i] = q;
        }
        for (size_t d = 0; d < G.cells.size(); ++d) {
            pl.det_slot[(size_t)pi * kWarp + d] = vread(sim->det_cv[G.cells[d]]);
            pl.det_gid[(size_t)pi * kWarp + d] = G.cells[d];
        }
    }
    }   // tile packs

    // per model synapse: the owner lane and row of its unit (events go there), and the state
    // entry for the unit's lowest-index synapse only (-1 for the others)
    {
        const int64_t ns = (int64_t)sim->syn_cv.size();
        std::vector<int64_t> entry(ns, -1);
        std::vector<int32_t> owner(ns, 0), js(ns, 0);
        for (int64_t i = 0; i < ns; ++i) {
            const int32_t u = sim->syn_unit[i];
            owner[i] = pl.syn_owner[u];
            js[i] = pl.syn_js[u];
            if (sim->u_rep[u] == i) entry[i] = pl.syn_entry[u];
        }
        pl.syn_entry.swap(entry);
        pl.syn_owner.swap(owner);
        pl.syn_js.swap(js);
    }

    // initial gates
    {
        double mi, hi, ni;
        hh_steady(-65.0, mi, hi, ni);
        sim->init_m.assign(sim->hh_cv.size(), mi);
        // FP64 mechanisms with steps of fixed length take the gate update from a table
        if (!sim->mixed && !sim->exact && !sim->hh_cv.empty()) {
            sim->hh_tab.resize((size_t)kHHTabN * kHHTabStride);
            build_hh_table(p.dt, sim->hh_tab.data());
        }
        // FP32 mechanisms: the same table rounded to float
        if (sim->mixed && !sim->exact && !sim->hh_cv.empty()) {
            hvec<double> tab;
            tab.resize((size_t)kHHTabN * kHHTabStride);
            build_hh_table(p.dt, tab.data());
            sim->hh_tab_f.resize(tab.size());
            parallel_for((int64_t)tab.size(), [&](int64_t i) { sim->hh_tab_f[i] = (float)tab[i]; });
        }
        sim->init_h.assign(sim->hh_cv.size(), hi);
        sim->init_n.assign(sim->hh_cv.size(), ni);
    }
    // connections grouped by source (every virtual rank's gids in a dry run), ascending
    // connection index
    const int64_t n_out = (int64_t)nc * sim->dry_ranks;
    sim->out_ptr.assign(n_out + 1, 0);
    sim->out_syn.resize(ncon);
    sim->out_idx.resize(ncon);
    sim->out_delay.resize(ncon);
    sim->out_w.resize(ncon);
    auto put = [&](int64_t q, int64_t i) {
        sim->out_syn[q] = (int32_t)sim->conn_dst[i];
        sim->out_idx[q] = (int32_t)i;
        sim->out_delay[q] = sim->conn_delay[i];
        sim->out_w[q] = sim->conn_w[i];
    };
    const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
    const int64_t nt = std::min<int64_t>(16, hw);
    if (ncon >= (1 << 20) && nt > 1 && n_out * nt <= ((int64_t)1 << 26)) {
        // counting sort in nt contiguous parts: part t's connections of a source follow those
        // of parts < t, so each source's list stays in ascending connection index
        std::vector<int64_t> cnt((size_t)(nt * n_out), 0);
        run_tasks(nt, [&](int64_t t, int64_t k) {
            int64_t* c = cnt.data() + t * n_out;
            for (int64_t i = ncon * t / k; i < ncon * (t + 1) / k; ++i) c[sim->conn_src[i]]++;
        });
        for (int64_t s = 0; s < n_out; ++s) {
            int64_t run = sim->out_ptr[s];
            for (int64_t t = 0; t < nt; ++t) {
                const int64_t x = cnt[t * n_out + s];
                cnt[t * n_out + s] = run;
                run += x;
            }
            sim->out_ptr[s + 1] = run;
        }
        run_tasks(nt, [&](int64_t t, int64_t k) {
            int64_t* c = cnt.data() + t * n_out;
            for (int64_t i = ncon * t / k; i < ncon * (t + 1) / k; ++i) put(c[sim->conn_src[i]]++, i);
        });
    } else {
        for (int64_t i = 0; i < ncon; ++i) sim->out_ptr[sim->conn_src[i] + 1]++;
        for (int64_t c = 0; c < n_out; ++c) sim->out_ptr[c + 1] += sim->out_ptr[c];
        std::vector<int64_t> fill(sim->out_ptr.begin(), sim->out_ptr.end() - 1);
        for (int64_t i = 0; i < ncon; ++i) put(fill[sim->conn_src[i]]++, i);
    }
    *out = sim;
    return ARB_OK;
}

void arb_destroy(arb_sim* sim) {
    if (!sim) return;
    if (sim->bound) {
        for (int g = 0; g < 6; ++g)
            if (sim->graph[g]) cudaGraphExecDestroy(sim->graph[g]);
        for (int g = 0; g < kGraphRing; ++g) {
            if (sim->t0[g]) cudaEventDestroy(sim->t0[g]);
            if (sim->t1[g]) cudaEventDestroy(sim->t1[g]);
        }
        if (sim->ev_in) cudaEventDestroy(sim->ev_in);
        if (sim->ev_out) cudaEventDestroy(sim->ev_out);
        if (sim->ev_main) cudaEventDestroy(sim->ev_main);
        if (sim->ev_side) cudaEventDestroy(sim->ev_side);
        if (sim->s2) {
            cudaStreamSynchronize(sim->s2);
            cudaStreamDestroy(sim->s2);
        }
        if (sim->s) {
            cudaStreamSynchronize(sim->s);
            cudaStreamDestroy(sim->s);
        }
    }
    delete sim;
}



arb_status arb_workspace_bytes(const arb_sim* csim, int64_t* bytes) {
    arb_sim* sim = const_cast<arb_sim*>(csim);
    if (!sim || !bytes) return ARB_E_ARG;
    layout_regions(sim);
    *bytes = sim->ws_bytes;
    return ARB_OK;
}

arb_status arb_plan_info(const arb_sim* sim, int64_t* n_packs, int64_t* total_rows, int64_t* smem_packs,
                         double* lane_efficiency, int32_t* epoch_steps, int64_t* max_pack_rows,
                         int32_t* cells_per_pack, int64_t* split_cvs, int64_t* spread_rows,
                         int32_t* kernel_variant) {
    if (!sim) return ARB_E_ARG;
    if (spread_rows) *spread_rows = sim->plan.stream ? sim->plan.spread_rows : -1;
    if (kernel_variant) *kernel_variant = sim->variant;
    if (max_pack_rows) {
        int64_t mx = 0;
        for (const PackDesc& pd : sim->plan.packs) mx = std::max<int64_t>(mx, pd.nrow);
        *max_pack_rows = mx;
    }
    if (cells_per_pack) *cells_per_pack = sim->plan.cells_per_pack;
    if (split_cvs) *split_cvs = sim->plan.stream ? sim->plan.split_cvs : -1;
    if (n_packs) *n_packs = (int64_t)sim->plan.packs.size();
    if (total_rows) *total_rows = sim->plan.total_rows;
    if (smem_packs) *smem_packs = sim->plan.smem_packs;
    if (lane_efficiency) *lane_efficiency = sim->plan.lane_eff;
    if (epoch_steps) *epoch_steps = sim->epoch_steps;
    return ARB_OK;
}



arb_status arb_plan_packs(const arb_sim* sim, int64_t cap, int32_t* rows, int32_t* kind, int32_t* mech_rows,
                          int64_t* n_packs) {
    if (!sim) return ARB_E_ARG;
    const auto& P = sim->plan.packs;
    if (n_packs) *n_packs = (int64_t)P.size();
    for (int64_t i = 0; i < (int64_t)P.size() && i < cap; ++i) {
        const PackDesc& pd = P[i];
        if (rows) rows[i] = pd.nrow;
        if (kind) kind[i] = pd.smem == kPackStream ? (pd.round_rows > 0 ? 1 : 0) : (pd.smem == kPackSmem ? 2 : 3);
        if (mech_rows) mech_rows[i] = pd.nsyn_row + pd.nhh_row + pd.nst_row;
    }
    return ARB_OK;
}

static arb_status upload_mech_state(arb_sim* sim, const std::vector<double>& m, const std::vector<double>& h,
                                    const std::vector<double>& n, const std::vector<double>& g);

// One epoch = three captured graphs: the event-delivery kernels, the epoch kernel and the
// spike exchange. Timing events are recorded between the graph launches, on the library's
// stream, so the epoch kernel's own duration is measured with CUDA events.
// The graphs of one epoch. The epoch kernel is always alone in its graph (with the one-thread
// begin/end kernels as nodes of that graph it ran about 5% slower on the batched workload).
//   0: delivery lists (serial schedule: then the integration's begin kernel)
//   1: epoch kernel reading list buffer 0          3: the same reading list buffer 1
//   2: (serial: the integration's end kernel) spike walk
//   4 / 5: the integration's begin / end kernel (overlapped schedule)
static arb_status capture_one(arb_sim* sim, int which, cudaGraphExec_t* out) {
    if (*out) { cudaGraphExecDestroy(*out); *out = nullptr; }
    cudaGraph_t g = nullptr;
    Ctl* c = (Ctl*)region(sim, "ctl");
    CU(cudaStreamBeginCapture(sim->s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaSuccess;
    if (which == 0) {
        e1 = launch_events_pre(sim->ev_args, sim->n_sm, sim->s);
        if (e1 == cudaSuccess && !sim->overlap) e1 = launch_int_begin(c, sim->epoch_steps, sim->s);
    } else if (which == 1 || which == 3) {
        DevModel<double> d64 = sim->dm64;
        DevModel<float> d32 = sim->dm32;
        if (which == 3) {
            d64.ev_off += d64.n_owner + 1;
            d32.ev_off += d32.n_owner + 1;
        }
        if (sim->plan.stream)
            e1 = sim->mixed ? launch_stream<float>(d32, stream_mode(sim), sim->variant, sim->grid, sim->warps_per_cta, (int)sim->plan.warp_smem, sim->s)
                            : launch_stream<double>(d64, stream_mode(sim), sim->variant, sim->grid, sim->warps_per_cta, (int)sim->plan.warp_smem, sim->s);
        else
            e1 = sim->mixed ? launch_epoch<float>(d32, sim->implicit, sim->grid, sim->warps_per_cta, sim->plan.tile_doubles, sim->s)
                            : launch_epoch<double>(d64, sim->implicit, sim->grid, sim->warps_per_cta, sim->plan.tile_doubles, sim->s);
    } else if (which == 2) {
        if (!sim->overlap) e1 = launch_int_end(c, sim->prm.spike_capacity, sim->s);
        if (e1 == cudaSuccess) e1 = launch_events_post(sim->spk_args, sim->n_sm, sim->s);
    } else if (which == 4) {
        e1 = launch_int_begin(c, sim->epoch_steps, sim->s);
    } else {
        e1 = launch_int_end(c, sim->prm.spike_capacity, sim->s);
    }
    cudaError_t e2 = cudaStreamEndCapture(sim->s, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(sim, ARB_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    }
    cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail(sim, ARB_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    return ARB_OK;
}

static arb_status capture_graphs(arb_sim* sim) {
    for (int w = 0; w < (sim->overlap ? 6 : 3); ++w) {
        arb_status st = capture_one(sim, w, &sim->graph[w]);
        if (st != ARB_OK) return st;
    }
    return ARB_OK;
}

arb_status arb_bind_workspace(arb_sim* sim, void* dev_ptr, int64_t bytes) {
    if (!sim) return ARB_E_ARG;
    if (sim->bound) return fail(sim, ARB_E_STATE, "workspace already bound");
    layout_regions(sim);
    if (!dev_ptr || ((uintptr_t)dev_ptr & 255) != 0) return fail(sim, ARB_E_ARG, "workspace must be a 256-byte aligned device pointer");
    if (bytes < sim->ws_bytes) return fail(sim, ARB_E_NOMEM, "workspace too small: need " + std::to_string(sim->ws_bytes) + " bytes");
    cudaPointerAttributes pa;
    CU(cudaPointerGetAttributes(&pa, dev_ptr));
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) return fail(sim, ARB_E_ARG, "workspace is not device memory");
    int dev = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sim->n_sm, cudaDevAttrMultiProcessorCount, dev));
    sim->ws = (char*)dev_ptr;
    CU(cudaStreamCreateWithFlags(&sim->s, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&sim->ev_in, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&sim->ev_out, cudaEventDisableTiming));
    if (sim->overlap) {
        // the exchange stream yields to the integration: lowest priority
        int least = 0, greatest = 0;
        CU(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CU(cudaStreamCreateWithPriority(&sim->s2, cudaStreamNonBlocking, least));
        CU(cudaEventCreateWithFlags(&sim->ev_main, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&sim->ev_side, cudaEventDisableTiming));
    }
    for (int g = 0; g < kGraphRing; ++g) {
        CU(cudaEventCreate(&sim->t0[g]));
        CU(cudaEventCreate(&sim->t1[g]));
    }
    cudaStream_t us = (cudaStream_t)sim->prm.stream;
    CU(cudaEventRecord(sim->ev_in, us));
    CU(cudaStreamWaitEvent(sim->s, sim->ev_in, 0));
    const Plan& pl = sim->plan;
    arb_status st;
#define UP(name, vec) if ((st = up(sim, name, vec)) != ARB_OK) return st
    UP("packs", pl.packs);
    UP("ca", pl.ca); UP("cb", pl.cb); UP("ck", pl.ck); UP("ce", pl.ce); UP("pslot", pl.pslot); UP("vmap", pl.vmap);
    UP("V", pl.V0);
    UP("cE", pl.cE); UP("cB", pl.cB);
    if (pl.stream_imp) { UP("cpos", pl.cpos); UP("row_cs", pl.row_cs); UP("row_cn", pl.row_cn); UP("mb_ent", pl.mb_ent); UP("mb_cs", pl.mb_cs); }
    UP("syn_ntau", pl.syn_ntau); UP("slot_lo", pl.slot_lo); UP("slot_hi", pl.slot_hi);
    UP("syn_slot", pl.syn_slot); UP("syn_vs", pl.syn_vs); UP("syn_e", pl.syn_e); UP("syn_decay", pl.syn_decay); UP("syn_sc", pl.syn_sc);
    if (!sim->hh_tab.empty()) UP("hh_tab", sim->hh_tab);
    if (!sim->hh_tab_f.empty()) UP("hh_tab_f", sim->hh_tab_f);
    if (sim->mixed) {   // float copies of the mechanism constants the FP32 mechanisms use
        auto to_f = [](const std::vector<double>& v) {
            std::vector<float> f(v.size());
            for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];
            return f;
        };
        UP("syn_decay_f", to_f(pl.syn_decay)); UP("syn_e_f", to_f(pl.syn_e));
        UP("hh_gna_f", to_f(pl.hh_gna)); UP("hh_gk_f", to_f(pl.hh_gk));
    }
    UP("hh_slot", pl.hh_slot); UP("hh_vs", pl.hh_vs); UP("hh_sc", pl.hh_sc); UP("hh_gna", pl.hh_gna); UP("hh_gk", pl.hh_gk);
    UP("st_slot", pl.st_slot); UP("st_sc", pl.st_sc); UP("st_on", pl.st_on); UP("st_off", pl.st_off); UP("st_amp", pl.st_amp);
    UP("det_slot", pl.det_slot); UP("det_gid", pl.det_gid);
    UP("syn_owner", pl.syn_owner); UP("syn_js", pl.syn_js);
    UP("out_ptr", sim->out_ptr); UP("out_syn", sim->out_syn); UP("out_idx", sim->out_idx);
    UP("out_delay", sim->out_delay); UP("out_w", sim->out_w);
    UP("cv_tile", pl.cv_tile); UP("hh_entry", pl.hh_entry); UP("syn_entry", pl.syn_entry);
#undef UP
    {   // zero the mechanism state arrays (padding entries), then set the initial state
        const size_t mt = sim->mixed ? 4 : 8;
        CU(cudaMemsetAsync(region(sim, "syn_g"), 0, mt * pl.syn_rows * kWarp, sim->s));
        CU(cudaMemsetAsync(region(sim, "hh_m"), 0, mt * pl.hh_rows * kWarp, sim->s));
        CU(cudaMemsetAsync(region(sim, "hh_h"), 0, mt * pl.hh_rows * kWarp, sim->s));
        CU(cudaMemsetAsync(region(sim, "hh_n"), 0, mt * pl.hh_rows * kWarp, sim->s));
    }
    Ctl c0;
    std::memset(&c0, 0, sizeof(c0));
    CU(cudaMemcpyAsync(region(sim, "ctl"), &c0, sizeof(Ctl), cudaMemcpyHostToDevice, sim->s));
    fill_devmodel(sim, sim->dm64);
    fill_devmodel(sim, sim->dm32);
#ifdef ARB_DEBUG
    if ((st = write_canaries(sim)) != ARB_OK) return st;
#endif
    sim->bound = true;
    st = upload_mech_state(sim, sim->init_m, sim->init_h, sim->init_n, std::vector<double>(sim->syn_cv.size(), 0.0));
    if (st != ARB_OK) return st;
    EvArgs& a = sim->ev_args;
    a.ctl = (Ctl*)region(sim, "ctl");
    a.pool[0] = (PendEv*)region(sim, "pool0");
    a.pool[1] = (PendEv*)region(sim, "pool1");
    a.pool_cap = sim->prm.event_capacity;
    a.ext_step = (const int64_t*)region(sim, "ext_step");
    a.ext_t = (const double*)region(sim, "ext_t");
    a.ext_w = (const double*)region(sim, "ext_w");
    a.ext_syn = (const int32_t*)region(sim, "ext_syn");
    a.ext_idx = (const int32_t*)region(sim, "ext_idx");
    a.syn_owner = (const int32_t*)region(sim, "syn_owner");
    a.syn_js = (const int32_t*)region(sim, "syn_js");
    a.counts = (int32_t*)region(sim, "counts");
    a.off = (int32_t*)region(sim, "ev_off");
    a.rec = (EvRec*)region(sim, "ev");
    a.tmp = (EvRec*)region(sim, "ev_tmp");
    a.bucket_cap = sim->prm.bucket_capacity;
    a.n_owner = (int32_t)(pl.packs.size() * kWarp);
    a.n_syn = (int64_t)sim->u_cv.size();
    a.epoch_steps = sim->epoch_steps;
    a.time_major = sim->exact ? 1 : 0;
    a.slot_mask = sim->overlap ? 1 : 0;
    SpkArgs& b = sim->spk_args;
    b.ctl = a.ctl;
    b.spk_gid = (const int32_t*)region(sim, "spk_gid");
    b.spk_t = (const double*)region(sim, "spk_t");
    b.spike_cap = sim->prm.spike_capacity;
    b.out_ptr = (const int64_t*)region(sim, "out_ptr");
    b.out_syn = (const int32_t*)region(sim, "out_syn");
    b.out_idx = (const int32_t*)region(sim, "out_idx");
    b.out_delay = (const double*)region(sim, "out_delay");
    b.out_w = (const double*)region(sim, "out_w");
    b.pool[0] = a.pool[0];
    b.pool[1] = a.pool[1];
    b.pool_cap = sim->prm.event_capacity;
    b.dt = sim->prm.dt;
    b.exact = sim->exact ? 1 : 0;
    b.n_cells = sim->n_cells;
    b.dry_ranks = sim->dry_ranks;
    CU(events_prepare());
    // launch shape of the persistent epoch kernel
    if (pl.stream) {
        // fewer warps per CTA when one warp's stack or mailbox is large
        int kw = 0, pw = 0;
        stream_variant_shape(stream_mode(sim) == 1, sim->variant, (int)pl.warp_smem, &kw, &pw);
        const int64_t per_warp = (int64_t)pw * (int64_t)sizeof(double2);
        sim->warps_per_cta = (int)std::min<int64_t>(kw, (int64_t)(227 * 1024) / std::max<int64_t>(per_warp, 1));
        if (sim->warps_per_cta < 1) return fail(sim, ARB_E_ARG, "hand-over stack of one warp exceeds shared memory");
        int bps = 0;
        cudaError_t eo = sim->mixed ? stream_occupancy<float>(stream_mode(sim), sim->variant, sim->warps_per_cta, (int)pl.warp_smem, &bps)
                                    : stream_occupancy<double>(stream_mode(sim), sim->variant, sim->warps_per_cta, (int)pl.warp_smem, &bps);
        if (eo != cudaSuccess) return fail(sim, ARB_E_CUDA, std::string("stream kernel occupancy: ") + cudaGetErrorString(eo));
        if (bps < 1) return fail(sim, ARB_E_CUDA, "stream kernel does not fit on an SM");
        sim->grid = sim->n_sm * bps;
        st = capture_graphs(sim);
        if (st != ARB_OK) return st;
        CU(cudaStreamSynchronize(sim->s));
        return ARB_OK;
    }
    const bool any_smem = pl.smem_packs > 0;
    sim->warps_per_cta = any_smem ? (int)std::max<int64_t>(1, (int64_t)(227 * 1024 / 8) / std::max(1, pl.tile_doubles)) : 4;
    sim->warps_per_cta = std::min(sim->warps_per_cta, 8);
    if (!any_smem) sim->plan.tile_doubles = 0;
    int bps = 0;
    cudaError_t eo = sim->mixed ? epoch_occupancy<float>(sim->implicit, sim->warps_per_cta, sim->plan.tile_doubles, &bps)
                                : epoch_occupancy<double>(sim->implicit, sim->warps_per_cta, sim->plan.tile_doubles, &bps);
    if (eo != cudaSuccess) return fail(sim, ARB_E_CUDA, std::string("epoch kernel occupancy: ") + cudaGetErrorString(eo));
    if (bps < 1) return fail(sim, ARB_E_CUDA, "epoch kernel does not fit on an SM");
    sim->grid = sim->n_sm * bps;
    st = capture_graphs(sim);
    if (st != ARB_OK) return st;
    CU(cudaStreamSynchronize(sim->s));
    return ARB_OK;
}

arb_status arb_enqueue_events(arb_sim* sim, int64_t n, const int64_t* syn, const double* t, const double* w) {
    if (!sim) return ARB_E_ARG;
    if (n < 0 || (n > 0 && (!syn || !t || !w))) return fail(sim, ARB_E_ARG, "bad event arrays");
    const int64_t nsyn = (int64_t)sim->syn_cv.size();
    for (int64_t i = 0; i < n; ++i) {
        if (syn[i] < 0 || syn[i] >= nsyn) return fail(sim, ARB_E_ARG, "event synapse index out of range");
        if (!std::isfinite(t[i]) || !std::isfinite(w[i])) return fail(sim, ARB_E_ARG, "event time and weight must be finite");
        const int64_t step = event_step(t[i], sim->prm.dt, sim->exact);
        if (step < sim->k) return fail(sim, ARB_E_ARG, "event time lies before the current time");
    }
    if (sim->ext_counter + n > INT32_MAX) return fail(sim, ARB_E_OVERFLOW, "too many external events over the run");
    for (int64_t i = 0; i < n; ++i) {
        ExtEvent e;
        e.t = t[i];
        e.w = w[i];
        e.syn = (int32_t)syn[i];
        e.idx = (int32_t)(sim->ext_counter++);
        e.step = event_step(t[i], sim->prm.dt, sim->exact);
        sim->ext.push_back(e);
    }
    if (n > 0) sim->ext_dirty = true;
    return ARB_OK;
}

static arb_status sync_in(arb_sim* sim) {
    CU(cudaEventRecord(sim->ev_in, (cudaStream_t)sim->prm.stream));
    CU(cudaStreamWaitEvent(sim->s, sim->ev_in, 0));
    return ARB_OK;
}
static arb_status sync_out(arb_sim* sim) {
    CU(cudaEventRecord(sim->ev_out, sim->s));
    CU(cudaStreamWaitEvent((cudaStream_t)sim->prm.stream, sim->ev_out, 0));
    return ARB_OK;
}

arb_status arb_advance(arb_sim* sim, double t_end) {
    if (!sim) return ARB_E_ARG;
    if (!sim->bound) return fail(sim, ARB_E_STATE, "bind a workspace first");
    if (!std::isfinite(t_end)) return fail(sim, ARB_E_ARG, "t_end must be finite");
    const int64_t k_end = (int64_t)std::llround(t_end / sim->prm.dt);
    sim->last_epoch_ms = 0.0;
    sim->last_launches = 0;
    if (k_end <= sim->k) return ARB_OK;
    arb_status st = sync_in(sim);
    if (st != ARB_OK) return st;
    Ctl* dctl = (Ctl*)region(sim, "ctl");
    if (sim->ext_dirty) {
        // keep only events not yet delivered, sorted by (step, enqueue order)
        std::vector<ExtEvent> keep;
        keep.reserve(sim->ext.size());
        for (const auto& e : sim->ext) if (e.step >= sim->k) keep.push_back(e);
        std::stable_sort(keep.begin(), keep.end(), [](const ExtEvent& a, const ExtEvent& b) {
            return a.step != b.step ? a.step < b.step : a.idx < b.idx;
        });
        sim->ext.swap(keep);
        const int64_t n = (int64_t)sim->ext.size();
        if (n > sim->prm.ext_event_capacity)
            return fail(sim, ARB_E_OVERFLOW, "more pending external events than ext_event_capacity");
        std::vector<int64_t> step(n);
        std::vector<double> tt(n), ww(n);
        std::vector<int32_t> sy(n), ix(n);
        for (int64_t i = 0; i < n; ++i) {
            step[i] = sim->ext[i].step; tt[i] = sim->ext[i].t; ww[i] = sim->ext[i].w;
            sy[i] = sim->ext[i].syn; ix[i] = sim->ext[i].idx;
        }
        if ((st = up(sim, "ext_step", step)) != ARB_OK) return st;
        if ((st = up(sim, "ext_t", tt)) != ARB_OK) return st;
        if ((st = up(sim, "ext_w", ww)) != ARB_OK) return st;
        if ((st = up(sim, "ext_syn", sy)) != ARB_OK) return st;
        if ((st = up(sim, "ext_idx", ix)) != ARB_OK) return st;
        static thread_local int64_t zero_and_n[2];
        zero_and_n[0] = 0;
        zero_and_n[1] = n;
        CU(cudaMemcpyAsync(&dctl->ext_lo, &zero_and_n[0], sizeof(int64_t), cudaMemcpyHostToDevice, sim->s));
        CU(cudaMemcpyAsync(&dctl->n_ext, &zero_and_n[1], sizeof(int64_t), cudaMemcpyHostToDevice, sim->s));
        CU(cudaStreamSynchronize(sim->s));   // host vectors above go out of scope
        sim->ext_dirty = false;
    }
    static thread_local int64_t kend_host;
    kend_host = k_end;
    CU(cudaMemcpyAsync(&dctl->k_end, &kend_host, sizeof(int64_t), cudaMemcpyHostToDevice, sim->s));
    const int64_t E = sim->epoch_steps;
    const int64_t pieces = (k_end - sim->k + E - 1) / E;
    for (int g = 0; g < kGraphRing; ++g) sim->pending_time[g] = false;
    double ms_sum = 0.0;
    // one epoch's integration (graph 1) on the library stream, timed with a ring of events
    auto integrate = [&]() -> arb_status {
        const int g = (int)(sim->graph_replays % kGraphRing);
        if (sim->pending_time[g]) {
            CU(cudaEventSynchronize(sim->t1[g]));
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, sim->t0[g], sim->t1[g]));
            ms_sum += ms;
            sim->pending_time[g] = false;
        }
        CU(cudaEventRecord(sim->t0[g], sim->s));
        // the list buffer of this epoch: the preparation alternates them in the same order
        CU(cudaGraphLaunch(sim->graph[sim->overlap && (sim->int_count & 1) ? 3 : 1], sim->s));
        CU(cudaEventRecord(sim->t1[g], sim->s));
        sim->int_count++;
        sim->pending_time[g] = true;
        sim->graph_replays++;
        return ARB_OK;
    };
    if (!sim->overlap) {
        // serial: delivery lists, integration, spike walk
        for (int64_t i = 0; i < pieces; ++i) {
            CU(cudaGraphLaunch(sim->graph[0], sim->s));
            if ((st = integrate()) != ARB_OK) return st;
            CU(cudaGraphLaunch(sim->graph[2], sim->s));
        }
    } else {
        // overlapped (epochs of half the minimum delay): while epoch i integrates, the
        // exchange stream walks the spikes of epoch i-1 and builds the lists of epoch i+1
        CU(cudaGraphLaunch(sim->graph[0], sim->s));
        for (int64_t i = 0; i < pieces; ++i) {
            if (i > 0) CU(cudaStreamWaitEvent(sim->s, sim->ev_side, 0));
            CU(cudaEventRecord(sim->ev_main, sim->s));
            CU(cudaGraphLaunch(sim->graph[4], sim->s));
            if ((st = integrate()) != ARB_OK) return st;
            CU(cudaGraphLaunch(sim->graph[5], sim->s));
            if (i > 0 || i + 1 < pieces) {
                CU(cudaStreamWaitEvent(sim->s2, sim->ev_main, 0));
                if (i > 0) CU(cudaGraphLaunch(sim->graph[2], sim->s2));
                if (i + 1 < pieces) CU(cudaGraphLaunch(sim->graph[0], sim->s2));
                CU(cudaEventRecord(sim->ev_side, sim->s2));
            }
        }
        if (pieces > 1) CU(cudaStreamWaitEvent(sim->s, sim->ev_side, 0));
        CU(cudaGraphLaunch(sim->graph[2], sim->s));          // the last epoch's spikes
    }
    Ctl hc;
    CU(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, sim->s));
    CU(cudaStreamSynchronize(sim->s));
    for (int g = 0; g < kGraphRing; ++g)
        if (sim->pending_time[g]) {
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, sim->t0[g], sim->t1[g]));
            ms_sum += ms;
            sim->pending_time[g] = false;
        }
    sim->last_epoch_ms = ms_sum;
    sim->last_launches = pieces * 12;     // 7 list kernels, 3 integration, 2 spike walk
    sim->k = k_end;
    if ((st = sync_out(sim)) != ARB_OK) return st;
    if (hc.k0 != k_end) return fail(sim, ARB_E_STATE, "internal: device step count disagrees with the host");
    if (hc.status & (kStSpikeOverflow | kStPoolOverflow | kStBucketOverflow)) {
        std::string what;
        if (hc.status & kStSpikeOverflow) what += " spike_capacity";
        if (hc.status & kStPoolOverflow) what += " event_capacity";
        if (hc.status & kStBucketOverflow) what += " bucket_capacity";
        return fail(sim, ARB_E_OVERFLOW, "capacity exceeded:" + what);
    }
    if (hc.status & kStBounds) return fail(sim, ARB_E_STATE, "debug check: an index array held a value outside its range");
    if (hc.status & kStNonFinite) return fail(sim, ARB_E_NONFINITE, "a voltage became NaN or infinite");
    if (hc.status & kStLateEvent) return fail(sim, ARB_E_STATE, "internal: an event arrived after its step");
#ifdef ARB_DEBUG
    if ((st = check_canaries(sim)) != ARB_OK) return st;
#endif
    return ARB_OK;
}

arb_status arb_workspace_region(const arb_sim* sim, const char* name, int64_t* offset, int64_t* bytes) {
    if (!sim || !name) return ARB_E_ARG;
    for (const auto& r : sim->regions)
        if (r.first == name) {
            if (offset) *offset = (int64_t)r.second.off;
            if (bytes) *bytes = (int64_t)r.second.bytes;
            return ARB_OK;
        }
    return ARB_E_ARG;
}

arb_status arb_check_canaries(arb_sim* sim) {
    if (!sim) return ARB_E_ARG;
    if (!sim->bound) return fail(sim, ARB_E_STATE, "no workspace bound");
    return check_canaries(sim);
}

int32_t arb_debug_build(void) {
#ifdef ARB_DEBUG
    return 1;
#else
    return 0;
#endif
}

arb_status arb_time(const arb_sim* sim, double* t, int64_t* steps) {
    if (!sim) return ARB_E_ARG;
    if (t) *t = (double)sim->k * sim->prm.dt;
    if (steps) *steps = sim->k;
    return ARB_OK;
}

arb_status arb_read_voltage(arb_sim* sim, double* out, int64_t n_cv, int32_t on_device) {
    if (!sim || !out) return ARB_E_ARG;
    if (!sim->bound) return fail(sim, ARB_E_STATE, "bind a workspace first");
    if (n_cv != sim->n_cv) return fail(sim, ARB_E_ARG, "n_cv does not match the model");
    arb_status st = sync_in(sim);
    if (st != ARB_OK) return st;
    double* dst = on_device ? out : (double*)region(sim, "scratch");
    CU(launch_gather<double>(dst, (const double*)region(sim, "V"), (const int64_t*)region(sim, "cv_tile"), n_cv, sim->s));
    if (!on_device) {
        CU(cudaMemcpyAsync(out, dst, sizeof(double) * n_cv, cudaMemcpyDeviceToHost, sim->s));
        CU(cudaStreamSynchronize(sim->s));
    }
    return sync_out(sim);
}

arb_status arb_num_spikes(arb_sim* sim, int64_t* n) {
    if (!sim || !n) return ARB_E_ARG;
    if (!sim->bound) return fail(sim, ARB_E_STATE, "bind a workspace first");
    int64_t v = 0;
    CU(cudaMemcpyAsync(&v, &((Ctl*)region(sim, "ctl"))->n_spikes, sizeof(int64_t), cudaMemcpyDeviceToHost, sim->s));
    CU(cudaStreamSynchronize(sim->s));
    *n = std::min(v, sim->prm.spike_capacity);
    return ARB_OK;
}

arb_status arb_read_spikes_from(arb_sim* sim, int64_t first, int32_t* gid, double* t, int64_t cap,
                                int64_t* n_out) {
    if (!sim || !n_out || first < 0 || cap < 0 || (cap > 0 && (!gid || !t))) return ARB_E_ARG;
    int64_t n = 0;
    arb_status st = arb_num_spikes(sim, &n);
    if (st != ARB_OK) return st;
    const int64_t k = std::max<int64_t>(0, n - first);
    std::vector<int32_t> g(k);
    std::vector<double> tt(k);
    if (k > 0) {
        CU(cudaMemcpyAsync(g.data(), (const int32_t*)region(sim, "spk_gid") + first, 4 * k, cudaMemcpyDeviceToHost, sim->s));
        CU(cudaMemcpyAsync(tt.data(), (const double*)region(sim, "spk_t") + first, 8 * k, cudaMemcpyDeviceToHost, sim->s));
        CU(cudaStreamSynchronize(sim->s));
    }
    std::vector<int64_t> o(k);
    std::iota(o.begin(), o.end(), 0);
    std::sort(o.begin(), o.end(), [&](int64_t a, int64_t b) { return tt[a] != tt[b] ? tt[a] < tt[b] : g[a] < g[b]; });
    const int64_t m = std::min(k, cap);
    for (int64_t i = 0; i < m; ++i) { gid[i] = g[o[i]]; t[i] = tt[o[i]]; }
    *n_out = m;
    return ARB_OK;
}

arb_status arb_read_spikes(arb_sim* sim, int32_t* gid, double* t, int64_t cap, int64_t* n_out) {
    return arb_read_spikes_from(sim, 0, gid, t, cap, n_out);
}

arb_status arb_set_probes(arb_sim* sim, int64_t n, const int64_t* cv, double* dev_trace, int64_t max_steps) {
    if (!sim) return ARB_E_ARG;
    if (!sim->bound) return fail(sim, ARB_E_STATE, "bind a workspace first");
    if (n < 0 || n > sim->n_cv || (n > 0 && (!cv || !dev_trace || max_steps < 0)))
        return fail(sim, ARB_E_ARG, "bad probe arguments (at most n_cv probes)");
    Plan& pl = sim->plan;
    std::vector<std::vector<std::pair<int32_t, int32_t>>> per(pl.packs.size());
    for (int64_t i = 0; i < n; ++i) {
        if (cv[i] < 0 || cv[i] >= sim->n_cv) return fail(sim, ARB_E_ARG, "probe CV out of range");
        const int32_t pk = pl.cv_pack[cv[i]];
        per[pk].push_back({(int32_t)(pl.cv_tile[cv[i]] - (int64_t)pl.packs[pk].row0 * kWarp), (int32_t)i});
    }
    sim->probe_slot.clear();
    sim->probe_col.clear();
    for (size_t pk = 0; pk < per.size(); ++pk) {
        pl.packs[pk].pr0 = (int32_t)sim->probe_slot.size();
        pl.packs[pk].npr = (int32_t)per[pk].size();
        for (auto& x : per[pk]) { sim->probe_slot.push_back(x.first); sim->probe_col.push_back(x.second); }
    }
    arb_status st = sync_in(sim);
    if (st != ARB_OK) return st;
    if ((st = up(sim, "packs", pl.packs)) != ARB_OK) return st;
    if ((st = up(sim, "probe_slot", sim->probe_slot)) != ARB_OK) return st;
    if ((st = up(sim, "probe_col", sim->probe_col)) != ARB_OK) return st;
    sim->n_probe = n;
    sim->trace = n > 0 ? dev_trace : nullptr;
    Ctl* dctl = (Ctl*)region(sim, "ctl");
    static thread_local int64_t pk0[2];
    pk0[0] = sim->k;
    pk0[1] = n > 0 ? max_steps : 0;
    CU(cudaMemcpyAsync(&dctl->probe_k0, &pk0[0], sizeof(int64_t), cudaMemcpyHostToDevice, sim->s));
    CU(cudaMemcpyAsync(&dctl->probe_max, &pk0[1], sizeof(int64_t), cudaMemcpyHostToDevice, sim->s));
    CU(cudaStreamSynchronize(sim->s));
    // kernel arguments changed: capture again
    fill_devmodel(sim, sim->dm64);
    fill_devmodel(sim, sim->dm32);
    if ((st = capture_graphs(sim)) != ARB_OK) return st;
    return sync_out(sim);
}

static arb_status upload_mech_state(arb_sim* sim, const std::vector<double>& m, const std::vector<double>& h,
                                    const std::vector<double>& n, const std::vector<double>& g_in) {
    // one state per unit: the unit's lowest-index synapse carries the sum over the unit
    std::vector<double> g(g_in.size(), 0.0);
    for (size_t i = 0; i < g_in.size(); ++i) g[sim->u_rep[sim->syn_unit[i]]] += g_in[i];
    double* scr = (double*)region(sim, "scratch");
    const int64_t nhh = (int64_t)sim->hh_cv.size(), nsyn = (int64_t)sim->syn_cv.size();
    const int64_t* hidx = (const int64_t*)region(sim, "hh_entry");
    const int64_t* sidx = (const int64_t*)region(sim, "syn_entry");
    auto put = [&](const std::vector<double>& v, const char* name, const int64_t* idx, int64_t cnt) -> arb_status {
        if (cnt == 0) return ARB_OK;
        CU(cudaMemcpyAsync(scr, v.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, sim->s));
        if (sim->mixed) CU(launch_scatter<float>((float*)region(sim, name), scr, idx, cnt, sim->s));
        else CU(launch_scatter<double>((double*)region(sim, name), scr, idx, cnt, sim->s));
        CU(cudaStreamSynchronize(sim->s));
        return ARB_OK;
    };
    arb_status st;
    if ((st = put(m, "hh_m", hidx, nhh)) != ARB_OK) return st;
    if ((st = put(h, "hh_h", hidx, nhh)) != ARB_OK) return st;
    if ((st = put(n, "hh_n", hidx, nhh)) != ARB_OK) return st;
    if ((st = put(g, "syn_g", sidx, nsyn)) != ARB_OK) return st;
    return ARB_OK;
}

arb_status arb_get_state(arb_sim* sim, double* V, double* m, double* h, double* n, double* g) {
    if (!sim) return ARB_E_ARG;
    if (!sim->bound) return fail(sim, ARB_E_STATE, "bind a workspace first");
    arb_status st = sync_in(sim);
    if (st != ARB_OK) return st;
    double* scr = (double*)region(sim, "scratch");
    const int64_t nhh = (int64_t)sim->hh_cv.size(), nsyn = (int64_t)sim->syn_cv.size();
    auto get = [&](double* out, const char* name, const char* idxname, int64_t cnt, bool is_mech) -> arb_status {
        if (!out || cnt == 0) return ARB_OK;
        const int64_t* idx = (const int64_t*)region(sim, idxname);
        if (is_mech && sim->mixed) CU(launch_gather<float>(scr, (const float*)region(sim, name), idx, cnt, sim->s));
        else CU(launch_gather<double>(scr, (const double*)region(sim, name), idx, cnt, sim->s));
        CU(cudaMemcpyAsync(out, scr, sizeof(double) * cnt, cudaMemcpyDeviceToHost, sim->s));
        CU(cudaStreamSynchronize(sim->s));
        return ARB_OK;
    };
    if ((st = get(V, "V", "cv_tile", sim->n_cv, false)) != ARB_OK) return st;
    if ((st = get(m, "hh_m", "hh_entry", nhh, true)) != ARB_OK) return st;
    if ((st = get(h, "hh_h", "hh_entry", nhh, true)) != ARB_OK) return st;
    if ((st = get(n, "hh_n", "hh_entry", nhh, true)) != ARB_OK) return st;
    if ((st = get(g, "syn_g", "syn_entry", nsyn, true)) != ARB_OK) return st;
    return sync_out(sim);
}

arb_status arb_set_state(arb_sim* sim, const double* V, const double* m, const double* h, const double* n, const double* g) {
    if (!sim) return ARB_E_ARG;
    if (!sim->bound) return fail(sim, ARB_E_STATE, "bind a workspace first");
    const int64_t nhh = (int64_t)sim->hh_cv.size(), nsyn = (int64_t)sim->syn_cv.size();
    if ((sim->n_cv > 0 && !V) || (nhh > 0 && (!m || !h || !n)) || (nsyn > 0 && !g)) return fail(sim, ARB_E_ARG, "state array is NULL");
    for (int64_t i = 0; i < sim->n_cv; ++i) if (!std::isfinite(V[i])) return fail(sim, ARB_E_ARG, "voltages must be finite");
    arb_status st = sync_in(sim);
    if (st != ARB_OK) return st;
    double* scr = (double*)region(sim, "scratch");
    if (sim->n_cv > 0) {
        CU(cudaMemcpyAsync(scr, V, sizeof(double) * sim->n_cv, cudaMemcpyHostToDevice, sim->s));
        CU(launch_scatter<double>((double*)region(sim, "V"), scr, (const int64_t*)region(sim, "cv_tile"), sim->n_cv, sim->s));
        CU(cudaStreamSynchronize(sim->s));
    }
    st = upload_mech_state(sim, std::vector<double>(m, m + nhh), std::vector<double>(h, h + nhh),
                           std::vector<double>(n, n + nhh), std::vector<double>(g, g + nsyn));
    if (st != ARB_OK) return st;
    return sync_out(sim);
}

arb_status arb_last_timing(const arb_sim* sim, double* epoch_kernel_ms, int64_t* launches) {
    if (!sim) return ARB_E_ARG;
    if (epoch_kernel_ms) *epoch_kernel_ms = sim->last_epoch_ms;
    if (launches) *launches = sim->last_launches;
    return ARB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Discrete adjoint

namespace {

struct AdjLayout {
    std::vector<std::pair<std::string, Region>> r;
    size_t total = 0;
    void add(const char* name, size_t bytes) {
        Region g;
        g.off = total;
        g.bytes = bytes;
        r.push_back({name, g});
        total += (bytes + 255) & ~(size_t)255;
    }
    char* at(char* base, const char* name) const {
        for (const auto& x : r) if (x.first == name) return base + x.second.off;
        return nullptr;
    }
};

// The tree each adjoint block solves: a cell's CVs and axial conductances, rooted where the
// level-by-level critical path of the chain solve (the sum over levels of the longest chain) is
// shortest. A tridiagonal tree system can be eliminated toward any node, so the root is free:
// the matrix is the same, only which end of an edge is the "parent" changes. Candidates are
// the nodes in the middle 40% of the cell's longest path (up to kRootCandidates of them, the
// centre first); each is scored by building its chains and levels.
constexpr int kRootCandidates = 24;

// Level-by-level critical path of the chain solve of a tree given by parent p (root r) and its
// breadth-first order: chains are maximal runs of CVs with one child each, a chain's level is one
// more than its highest child chain's.
int32_t chain_critical_path(const std::vector<int32_t>& p, const std::vector<int32_t>& bfs) {
    const int32_t n = (int32_t)p.size();
    std::vector<int32_t> nch(n, 0), only(n, -1), chain_of(n, -1), len, lev, parent_chain;
    for (int32_t i = 0; i < n; ++i)
        if (p[i] >= 0) { nch[p[i]]++; only[p[i]] = i; }
    for (int32_t h : bfs) {
        if (p[h] >= 0 && nch[p[h]] == 1) continue;   // continues its parent's chain
        const int32_t q = (int32_t)len.size();
        int32_t x = h, l = 1;
        chain_of[h] = q;
        while (nch[x] == 1) { x = only[x]; chain_of[x] = q; ++l; }
        len.push_back(l);
        parent_chain.push_back(p[h] >= 0 ? chain_of[p[h]] : -1);
    }
    const int32_t nq = (int32_t)len.size();
    lev.assign(nq, 0);
    int32_t maxl = 0;
    for (int32_t q = nq - 1; q >= 0; --q) {              // children after parents in bfs order
        maxl = std::max(maxl, lev[q]);
        if (parent_chain[q] >= 0) lev[parent_chain[q]] = std::max(lev[parent_chain[q]], lev[q] + 1);
    }
    std::vector<int32_t> longest(maxl + 1, 0);
    for (int32_t q = 0; q < nq; ++q) longest[lev[q]] = std::max(longest[lev[q]], len[q]);
    int32_t cp = 0;
    for (int32_t v : longest) cp += v;
    return cp;
}

// Re-roots a cell (model parents mp, cell-local) at r: solve parent sp, axial conductance to
// it ss (from the model's per-child conductances sg; 0 at r) and the breadth-first order.
void reroot_cell(const int32_t* mp, const double* sg, int32_t n, const std::vector<int32_t>& adj_ptr,
                 const std::vector<int32_t>& adj, int32_t r, std::vector<int32_t>& sp, std::vector<double>* ss,
                 std::vector<int32_t>& bfs) {
    sp.assign(n, -2);
    bfs.clear();
    bfs.push_back(r);
    sp[r] = -1;
    for (size_t h = 0; h < bfs.size(); ++h) {
        const int32_t v = bfs[h];
        for (int32_t e = adj_ptr[v]; e < adj_ptr[v + 1]; ++e) {
            const int32_t u = adj[e];
            if (sp[u] != -2) continue;
            sp[u] = v;
            bfs.push_back(u);
        }
    }
    if (ss) {
        ss->assign(n, 0.0);
        for (int32_t i = 0; i < n; ++i) {
            if (sp[i] < 0) continue;
            (*ss)[i] = mp[i] == sp[i] ? sg[i] : sg[sp[i]];   // the edge's conductance, stored at its model child
        }
    }
}

// Solve trees of all cells (model order, cell-local indices): parents, conductances to them, and
// each cell's breadth-first order. Cells are independent: chosen in parallel.
void solve_trees(const arb_sim* sim, const double* sigma, std::vector<int32_t>& SP, std::vector<double>& SS,
                 std::vector<int32_t>& SB) {
    const int32_t nc = sim->n_cells;
    const int64_t ncv = sim->n_cv;
    SP.assign(ncv, -1);
    SS.assign(ncv, 0.0);
    SB.assign(ncv, 0);
    // scoring every candidate costs O(candidates x CVs); large models score fewer
    const int cand = ncv * (int64_t)kRootCandidates <= (int64_t)400000000 ? kRootCandidates : 1;
    parallel_for(nc, [&](int64_t c) {
        const int64_t off = sim->cv_offset[c];
        const int32_t n = (int32_t)(sim->cv_offset[c + 1] - off);
        const int32_t* mp = sim->parent.data() + off;
        std::vector<int32_t> deg(n + 1, 0), adj_ptr(n + 1, 0), adj(n > 0 ? 2 * (n - 1) : 0);
        for (int32_t i = 1; i < n; ++i) { deg[i]++; deg[mp[i]]++; }
        for (int32_t i = 0; i < n; ++i) adj_ptr[i + 1] = adj_ptr[i] + deg[i];
        std::vector<int32_t> fill(adj_ptr.begin(), adj_ptr.end() - 1);
        for (int32_t i = 1; i < n; ++i) { adj[fill[i]++] = mp[i]; adj[fill[mp[i]]++] = i; }
        // the longest path: the farthest node from CV 0, then the farthest from that one
        std::vector<int32_t> sp, bfs;
        reroot_cell(mp, nullptr, n, adj_ptr, adj, 0, sp, nullptr, bfs);
        const int32_t a = bfs.back();
        reroot_cell(mp, nullptr, n, adj_ptr, adj, a, sp, nullptr, bfs);
        std::vector<int32_t> path{bfs.back()};
        while (sp[path.back()] >= 0) path.push_back(sp[path.back()]);
        const int32_t L = (int32_t)path.size();
        std::vector<int32_t> cands{path[L / 2]};
        if (cand > 1) {
            const int32_t lo = (int32_t)(0.3 * (L - 1)), hi = (int32_t)(0.7 * (L - 1));
            const int32_t span = hi - lo + 1, step = std::max<int32_t>(1, (span + cand - 2) / (cand - 1));
            for (int32_t k = lo; k <= hi; k += step)
                if (path[k] != cands[0]) cands.push_back(path[k]);
        }
        int32_t best = cands[0], best_cp = INT32_MAX;
        for (int32_t r : cands) {
            reroot_cell(mp, nullptr, n, adj_ptr, adj, r, sp, nullptr, bfs);
            const int32_t cp = chain_critical_path(sp, bfs);
            if (cp < best_cp) { best_cp = cp; best = r; }
        }
        std::vector<double> ss;
        reroot_cell(mp, sigma + off, n, adj_ptr, adj, best, sp, &ss, bfs);
        for (int32_t i = 0; i < n; ++i) {
            SP[off + i] = sp[i];
            SS[off + i] = ss[i];
            SB[off + i] = bfs[i];
        }
    });
}

// Tree-solve schedule of the adjoint kernels: per cell, its unbranched chains (runs of CVs
// with one child each, head nearest the root) ordered by level, and the constants of the
// scaled chain recurrence (arb_adjoint.cu). Along a chain, from its tail (k = 0), with s_k the
// axial conductance from CV k to its parent,
//   rho_0 = 1, gam_0 = 1,  rho_k = 1 / (s_{k-1}^2 rho_{k-1}),  gam_k = s_{k-1} rho_{k-1} gam_{k-1}
// (rho_k = c_{k-1} / c_k and gam_k = c_k / g_k), so that beta_k = rho_k gam_k, g_k / c_k =
// 1 / gam_k. P^_k / P^_{k-1} = D_k rho_k, and every pivot lies in [s_k + C_k/dt, dmax_k] (the
// matrix is an M-matrix whose diagonal exceeds the axial conductances by C/dt), which bounds
// P^. A chain is cut before the CV at which any of these would leave 2^{+-kChainRange}: the
// part below becomes a chain of its own whose parent is that CV (the same elimination in exact
// arithmetic). The recurrences run in long double.
struct ChainPlan {
    std::vector<int64_t> ch_ptr, lev_off, lev_bound, ch_cv_ptr, ch_kid_ptr, ch_kids;
    std::vector<int32_t> ch_cvs, prev;
    std::vector<int32_t> spar;                     // per CV: its parent in the solve tree (cell-local)
    // back-substitution tasks: per cell, [start, end) positions in the cell's chain list, kind
    // (0 a chain or its upper part, 1 a lower part's offsets a, 2 its factors b) and the anchor
    // CV (the upper part's last); per level of lev_bound, the cell-local first task
    std::vector<int32_t> tk, tkb, fixa;           // fixa: per CV, the anchor its value still needs, -1 none
    std::vector<int64_t> tk_ptr;
    int32_t max_tk = 0;
    std::vector<double> rho, beta, gcf, srf, kpw;
    int32_t max_cv = 0, max_ch = 0;
};

constexpr long double kChainRange = 300.0L;

ChainPlan chain_plan(const arb_sim* sim, const double* sigma, const double* cdt, const double* dmax) {
    ChainPlan P;
    const int32_t nc = sim->n_cells;
    const int64_t ncv = sim->n_cv;
    P.ch_ptr.assign(nc + 1, 0);
    P.lev_off.assign(nc + 1, 0);
    P.ch_cv_ptr.push_back(0);
    P.ch_kid_ptr.push_back(0);
    P.rho.assign(ncv, 1.0);
    P.beta.assign(ncv, 1.0);
    P.gcf.assign(ncv, 1.0);
    P.srf.assign(ncv, 0.0);
    P.prev.assign(ncv, -1);
    P.fixa.assign(ncv, -1);
    P.tk_ptr.assign(nc + 1, 0);
    std::vector<int32_t> SB;
    std::vector<double> SS;
    solve_trees(sim, sigma, P.spar, SS, SB);
    for (int32_t c = 0; c < nc; ++c) {
        const int64_t off = sim->cv_offset[c];
        const int32_t n = (int32_t)(sim->cv_offset[c + 1] - off);
        const int32_t* par = P.spar.data() + off;          // the solve tree
        const double* ssig = SS.data() + off;              // axial conductance to the solve parent
        std::vector<int32_t> nch(n, 0), only(n, -1);
        for (int32_t i = 0; i < n; ++i)
            if (par[i] >= 0) { nch[par[i]]++; only[par[i]] = i; }
        // chains in breadth-first head order (a parent chain's head precedes its children's); a
        // run that is cut contributes its parts from the top down, so that this still holds
        std::vector<std::vector<int32_t>> cvs;     // head first
        std::vector<std::array<double, 2>> kq;     // per chain: s_h^2 rho_h, s_h / gam_h
        std::vector<int32_t> chain_of_tail(n, -1), parent_chain;
        for (int32_t bi = 0; bi < n; ++bi) {
            const int32_t h = SB[off + bi];
            if (par[h] >= 0 && nch[par[h]] == 1) continue;   // continues its parent's chain
            std::vector<int32_t> t{h};                   // the run, head first
            for (int32_t x = h; nch[x] == 1;) { x = only[x]; t.push_back(x); }
            std::reverse(t.begin(), t.end());            // tail first
            // walk from the tail, cutting where the scaled quantities would leave the range
            std::vector<std::pair<int32_t, int32_t>> parts;   // [begin, end) in t
            std::vector<std::array<double, 2>> kparts;
            int32_t b = 0;
            long double rho = 1.0L, gam = 1.0L, lo = 0.0L, hi = 0.0L;
            for (int32_t i = 0; i <= (int32_t)t.size(); ++i) {
                bool cut = i == (int32_t)t.size();
                long double r2 = rho, g2 = gam, lo2 = lo, hi2 = hi;
                if (!cut) {
                    const int64_t y = off + t[i];
                    const long double s_y = par[t[i]] >= 0 ? (long double)ssig[t[i]] : 0.0L;
                    const long double dlo = s_y + (long double)cdt[y], dhi = (long double)dmax[y];
                    if (i == b) {
                        r2 = 1.0L;
                        g2 = 1.0L;
                        lo2 = std::log2(dlo);
                        hi2 = std::log2(dhi);
                    } else {
                        const long double s = (long double)ssig[t[i - 1]];
                        r2 = 1.0L / (s * s * rho);
                        g2 = s * gam * rho;
                        lo2 = lo + std::log2(dlo * r2);
                        hi2 = hi + std::log2(dhi * r2);
                    }
                    const long double lr = std::log2(r2), lg = std::log2(g2);
                    if (i > b && (std::fabs(lr) > kChainRange || std::fabs(lg) > kChainRange ||
                                  std::fabs(lr + lg) > kChainRange || std::fabs(lo2) > kChainRange ||
                                  std::fabs(hi2) > kChainRange))
                        cut = true;
                }
                if (cut) {
                    // the part [b, i): its head t[i-1] has the constants rho, gam
                    const long double sh = par[t[i - 1]] >= 0 ? (long double)ssig[t[i - 1]] : 0.0L;
                    parts.push_back({b, i});
                    kparts.push_back({(double)(sh * sh * rho), (double)(sh / gam)});
                    if (i == (int32_t)t.size()) break;
                    b = i;
                    --i;                                 // restart the walk at t[b]
                    rho = 1.0L;
                    gam = 1.0L;
                    continue;
                }
                rho = r2;
                gam = g2;
                lo = lo2;
                hi = hi2;
                const int64_t y = off + t[i];
                const long double s_y = par[t[i]] >= 0 ? (long double)ssig[t[i]] : 0.0L;
                P.rho[y] = (double)rho;
                P.beta[y] = (double)(rho * gam);
                P.gcf[y] = (double)(1.0L / gam);
                P.srf[y] = (double)(s_y * rho);
                P.prev[y] = i > b ? t[i - 1] : -1;
            }
            for (int32_t pi = (int32_t)parts.size() - 1; pi >= 0; --pi) {   // top part first
                std::vector<int32_t> v(t.begin() + parts[pi].first, t.begin() + parts[pi].second);
                std::reverse(v.begin(), v.end());                            // head first
                chain_of_tail[v.back()] = (int32_t)cvs.size();
                parent_chain.push_back(par[v.front()]);                     // parent CV for now
                kq.push_back(kparts[pi]);
                cvs.push_back(std::move(v));
            }
        }
        const int32_t nq = (int32_t)cvs.size();
        for (int32_t q = 0; q < nq; ++q)
            if (parent_chain[q] >= 0) parent_chain[q] = chain_of_tail[parent_chain[q]];
        std::vector<std::vector<int32_t>> kids(nq);
        for (int32_t q = 0; q < nq; ++q)
            if (parent_chain[q] >= 0) kids[parent_chain[q]].push_back(q);
        std::vector<int32_t> level(nq, 0);
        int32_t maxl = 0;
        for (int32_t q = nq - 1; q >= 0; --q) {
            for (int32_t k : kids[q]) level[q] = std::max(level[q], level[k] + 1);
            maxl = std::max(maxl, level[q]);
        }
        std::vector<int32_t> order(nq);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return level[x] < level[y]; });
        std::vector<int64_t> gidx(nq);
        const int64_t q0 = (int64_t)P.ch_cv_ptr.size() - 1;
        for (int32_t r = 0; r < nq; ++r) gidx[order[r]] = q0 + r;
        P.lev_off[c] = (int64_t)P.lev_bound.size();
        for (int32_t L = 0, r = 0; L <= maxl + 1; ++L) {
            while (r < nq && level[order[r]] < L) ++r;
            P.lev_bound.push_back(q0 + r);
        }
        for (int32_t r = 0; r < nq; ++r) {
            const int32_t q = order[r];
            for (int32_t x : cvs[q]) P.ch_cvs.push_back(x);
            P.ch_cv_ptr.push_back((int64_t)P.ch_cvs.size());
            for (int32_t k : kids[q]) P.ch_kids.push_back(gidx[k]);
            P.ch_kid_ptr.push_back((int64_t)P.ch_kids.size());
            P.kpw.push_back(kq[q][0]);
            P.kpw.push_back(kq[q][1]);
        }
        P.ch_ptr[c + 1] = q0 + nq;
        P.max_cv = std::max(P.max_cv, n);
        P.max_ch = std::max(P.max_ch, nq);
        // back-substitution tasks, level by level: in a level of at most kSplitLevel chains, each
        // chain of at least 8 CVs is split in two; its lower part runs on two more lanes (the
        // offsets a with V_anchor = 0, the factors b = prod e), so the level takes half as long
        {
            constexpr int32_t kSplitLevel = 10;
            const int64_t cv0 = P.ch_cv_ptr[q0];
            const int32_t tk0 = (int32_t)(P.tk.size() / 4);
            for (int32_t L = 0; L <= maxl; ++L) {
                P.tkb.push_back((int32_t)(P.tk.size() / 4) - tk0);
                const int64_t lb = P.lev_bound[P.lev_off[c] + L], le = P.lev_bound[P.lev_off[c] + L + 1];
                const bool split = le - lb <= kSplitLevel;
                for (int64_t gq = lb; gq < le; ++gq) {
                    const int32_t cs = (int32_t)(P.ch_cv_ptr[gq] - cv0), ce = (int32_t)(P.ch_cv_ptr[gq + 1] - cv0);
                    const int32_t len = ce - cs;
                    if (!split || len < 8) {
                        for (int32_t v : {cs, ce, 0, -1}) P.tk.push_back(v);
                        continue;
                    }
                    const int32_t m = cs + (len + 1) / 2;
                    const int32_t anchor = P.ch_cvs[cv0 + m - 1];
                    for (int32_t v : {cs, m, 0, -1}) P.tk.push_back(v);
                    for (int32_t v : {m, ce, 1, anchor}) P.tk.push_back(v);
                    for (int32_t v : {m, ce, 2, anchor}) P.tk.push_back(v);
                    for (int32_t i = m; i < ce - 1; ++i) P.fixa[off + P.ch_cvs[cv0 + i]] = anchor;   // the tail is fixed in the solve
                }
            }
            P.tkb.push_back((int32_t)(P.tk.size() / 4) - tk0);   // the end: as many entries as lev_bound
            P.tk_ptr[c + 1] = (int64_t)(P.tk.size() / 4);
            P.max_tk = std::max<int32_t>(P.max_tk, (int32_t)(P.tk.size() / 4) - tk0);
        }
    }
    P.lev_off[nc] = (int64_t)P.lev_bound.size();
    return P;
}

AdjLayout adj_layout(const arb_sim* sim, int64_t n_steps, int32_t ckpt, int64_t n_obs, int32_t n_groups) {
    (void)n_obs;
    const int64_t nc = sim->n_cells, ncv = sim->n_cv, nhh = (int64_t)sim->hh_cv.size(), nst = (int64_t)sim->st_cv.size();
    const int64_t nck = (n_steps + ckpt - 1) / ckpt, seg = std::min<int64_t>(ckpt, n_steps);
    AdjLayout L;
    L.add("off", 8 * (nc + 1));
    L.add("parent", 4 * ncv);
    for (const char* n : {"cdt", "sig", "dsig", "glin", "gelin", "area", "kcm", "ksc"}) L.add(n, 8 * ncv);
    L.add("hidx", 4 * ncv);
    for (const char* n : {"gna", "gk", "gl", "gna3", "gk4"}) L.add(n, 8 * nhh);
    L.add("st_ptr", 8 * (nc + 1));
    for (const char* n : {"st_cv", "st_on", "st_dur", "st_amp"}) L.add(n, 8 * nst);
    L.add("obs", 4 * ncv);
    L.add("V", 8 * ncv);
    L.add("Y", 24 * nhh);
    L.add("ckV", 8 * ncv * nck);
    L.add("ckY", 24 * nhh * nck);
    for (const char* n : {"segV0", "segV1"}) L.add(n, 8 * ncv * (seg + 1));
    for (const char* n : {"segY0", "segY1"}) L.add(n, 24 * nhh * (seg + 1));
    for (const char* n : {"segG0", "segG1"}) L.add(n, 48 * nhh * seg);
    L.add("lam", 8 * ncv);
    L.add("ybar", 24 * nhh);
    L.add("gacc", 32 * ncv);
    L.add("cell_loss", 8 * nc);
    L.add("hh_dtab", sim->hh_tab.empty() ? 0 : 8 * (int64_t)kHHTabN * kHHTabStride);
    L.add("loss_part", 8 * nc * (int64_t)kAdjBlock);
    L.add("grp_ptr", 8 * ((int64_t)n_groups + 1));
    L.add("grp_cv", 8 * ncv);
    // chain schedule: at most one chain per CV, at most n_cv + 1 level bounds per cell
    L.add("ch_ptr", 8 * (nc + 1));
    L.add("lev_off", 8 * (nc + 1));
    L.add("lev_bound", 8 * (ncv + nc));
    L.add("ch_cv_ptr", 8 * (ncv + 1));
    L.add("ch_cvs", 4 * ncv);
    L.add("ch_kid_ptr", 8 * (ncv + 1));
    L.add("ch_kids", 8 * ncv);
    for (const char* n : {"rho", "beta", "gcf", "srf"}) L.add(n, 8 * ncv);
    L.add("prev", 4 * ncv);
    L.add("kpw", 16 * ncv);                  // at most one chain per CV
    L.add("tk", 48 * ncv);                   // at most three back-substitution tasks per chain
    L.add("tk_ptr", 8 * (nc + 1));
    L.add("tkb", 4 * (ncv + nc));
    L.add("fixa", 4 * ncv);
    return L;
}

}  // namespace

extern "C" {

arb_status arb_adjoint_workspace_bytes(const arb_sim* sim, int64_t n_steps, int32_t checkpoint_every, int64_t n_obs,
                                       int32_t n_groups, int64_t* bytes) {
    if (!sim || !bytes) return ARB_E_ARG;
    if (n_steps < 1 || checkpoint_every < 1 || n_obs < 0 || n_groups < 0) return ARB_E_ARG;
    *bytes = (int64_t)adj_layout(sim, n_steps, checkpoint_every, n_obs, n_groups).total;
    return ARB_OK;
}

arb_status arb_adjoint(arb_sim* sim, int64_t n_steps, int32_t checkpoint_every, int64_t n_obs, const int64_t* obs_cv,
                       const double* target, double loss_scale, const int32_t* group_of_cv, int32_t n_groups,
                       void* workspace, int64_t workspace_bytes, double* grad, double* loss) {
    if (!sim) return ARB_E_ARG;
    if (!sim->bound) return fail(sim, ARB_E_STATE, "bind a workspace first");
    if (!sim->implicit) return fail(sim, ARB_E_ARG, "the adjoint is defined for the implicit scheme only");
    if (!sim->syn_cv.empty()) return fail(sim, ARB_E_ARG, "the adjoint does not support synapses");
    if (n_steps < 1 || checkpoint_every < 1) return fail(sim, ARB_E_ARG, "n_steps and checkpoint_every must be >= 1");
    if (n_obs < 0 || n_groups < 0) return fail(sim, ARB_E_ARG, "n_obs and n_groups must be >= 0");
    if ((n_obs > 0 && (!obs_cv || !target)) || (n_groups > 0 && (!group_of_cv || !grad)) || !loss)
        return fail(sim, ARB_E_ARG, "NULL array");
    if (!std::isfinite(loss_scale)) return fail(sim, ARB_E_ARG, "loss_scale must be finite");
    const int64_t nc = sim->n_cells, ncv = sim->n_cv, nhh = (int64_t)sim->hh_cv.size(), nst = (int64_t)sim->st_cv.size();
    const AdjLayout L = adj_layout(sim, n_steps, checkpoint_every, n_obs, n_groups);
    if (!workspace || ((uintptr_t)workspace & 255) != 0) return fail(sim, ARB_E_ARG, "workspace must be 256-byte aligned");
    if (workspace_bytes < (int64_t)L.total) return fail(sim, ARB_E_ARG, "workspace too small (see arb_adjoint_workspace_bytes)");
    {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, workspace) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return fail(sim, ARB_E_ARG, "workspace must be device memory");
        }
    }
    // host-side constants, model order
    std::vector<int32_t> obs(ncv, -1);
    for (int64_t o = 0; o < n_obs; ++o) {
        const int64_t cv = obs_cv[o];
        if (cv < 0 || cv >= ncv) return fail(sim, ARB_E_ARG, "observed CV out of range");
        if (obs[cv] >= 0) return fail(sim, ARB_E_ARG, "observed CVs must be distinct");
        obs[cv] = (int32_t)o;
    }
    std::vector<int64_t> grp_ptr((size_t)n_groups + 1, 0), grp_cv;
    if (n_groups > 0) {
        for (int64_t i = 0; i < ncv; ++i) {
            const int32_t g = group_of_cv[i];
            if (g < -1 || g >= n_groups) return fail(sim, ARB_E_ARG, "group_of_cv out of range");
            if (g >= 0) grp_ptr[g + 1]++;
        }
        for (int32_t g = 0; g < n_groups; ++g) grp_ptr[g + 1] += grp_ptr[g];
        grp_cv.assign(grp_ptr[n_groups], 0);
        std::vector<int64_t> fill(grp_ptr.begin(), grp_ptr.end() - 1);
        for (int64_t i = 0; i < ncv; ++i)
            if (group_of_cv[i] >= 0) grp_cv[fill[group_of_cv[i]]++] = i;
    }
    const double dt = sim->prm.dt;
    hvec<double> area, cap, sigma;
    cv_geometry(sim, area, cap, sigma);
    std::vector<double> cdt(ncv), dsig(sigma.begin(), sigma.end()), glin(ncv, 0.0), gelin(ncv, 0.0);
    for (int64_t i = 0; i < ncv; ++i) cdt[i] = cap[i] / dt;
    for (int32_t c = 0; c < nc; ++c)
        for (int64_t i = sim->cv_offset[c] + 1; i < sim->cv_offset[c + 1]; ++i) dsig[sim->cv_offset[c] + sim->parent[i]] += sigma[i];
    for (size_t q = 0; q < sim->pas_cv.size(); ++q) {
        const int64_t cv = sim->pas_cv[q];
        const double G = sim->g_pas[q] * area[cv] * 1e-2;
        glin[cv] += G;
        gelin[cv] += G * sim->e_pas[q];
    }
    std::vector<double> kcm(ncv), ksc(ncv);
    for (int64_t i = 0; i < ncv; ++i) {
        kcm[i] = area[i] * 1e-5 / dt;
        ksc[i] = area[i] * 1e-2;
    }
    std::vector<int32_t> hidx(ncv, -1);
    std::vector<double> gna(nhh), gk(nhh), gl(nhh), gna3(nhh), gk4(nhh);
    for (int64_t j = 0; j < nhh; ++j) {
        const int64_t cv = sim->hh_cv[j];
        hidx[cv] = (int32_t)j;
        gna[j] = sim->gnabar[j] * area[cv] * 1e-2;
        gk[j] = sim->gkbar[j] * area[cv] * 1e-2;
        gl[j] = sim->gl[j] * area[cv] * 1e-2;
        gna3[j] = 3.0 * gna[j];
        gk4[j] = 4.0 * gk[j];
    }
    // clamps grouped by cell
    std::vector<int64_t> st_ptr(nc + 1, 0), st_cv(nst);
    std::vector<double> st_on(nst), st_dur(nst), st_amp(nst);
    {
        std::vector<int32_t> cell_of(ncv);
        for (int32_t c = 0; c < nc; ++c)
            for (int64_t i = sim->cv_offset[c]; i < sim->cv_offset[c + 1]; ++i) cell_of[i] = c;
        for (int64_t q = 0; q < nst; ++q) st_ptr[cell_of[sim->st_cv[q]] + 1]++;
        for (int32_t c = 0; c < nc; ++c) st_ptr[c + 1] += st_ptr[c];
        std::vector<int64_t> fill(st_ptr.begin(), st_ptr.end() - 1);
        for (int64_t q = 0; q < nst; ++q) {
            const int64_t w = fill[cell_of[sim->st_cv[q]]]++;
            st_cv[w] = sim->st_cv[q];
            st_on[w] = sim->st_on[q];
            st_dur[w] = sim->st_dur[q];
            st_amp[w] = sim->st_amp[q];
        }
    }
    // largest diagonal each CV can reach (every gate open): bounds the scaled chain recurrence
    std::vector<double> dmax(ncv);
    for (int64_t i = 0; i < ncv; ++i) dmax[i] = cdt[i] + dsig[i] + glin[i];
    for (int64_t j = 0; j < nhh; ++j) dmax[sim->hh_cv[j]] += gna[j] + gk[j] + gl[j];
    if (!sim->adj_plan) sim->adj_plan = std::make_shared<ChainPlan>(chain_plan(sim, sigma.data(), cdt.data(), dmax.data()));
    const ChainPlan& CP = *static_cast<const ChainPlan*>(sim->adj_plan.get());
    if (adj_smem_bytes_for(CP.max_cv, CP.max_ch, CP.max_tk) > (size_t)200 * 1024)
        return fail(sim, ARB_E_ARG, "the adjoint needs every cell's solve and constants in shared memory (cells up to about 1,000 to 1,400 CVs, by chain count)");
    arb_status st = sync_in(sim);
    if (st != ARB_OK) return st;
    char* base = (char*)workspace;
    auto up = [&](const char* name, const void* src, size_t bytes) -> arb_status {
        if (bytes == 0) return ARB_OK;
        CU(cudaMemcpyAsync(L.at(base, name), src, bytes, cudaMemcpyHostToDevice, sim->s));
        return ARB_OK;
    };
    if ((st = up("off", sim->cv_offset.data(), 8 * (nc + 1))) != ARB_OK || (st = up("parent", CP.spar.data(), 4 * ncv)) != ARB_OK ||
        (st = up("cdt", cdt.data(), 8 * ncv)) != ARB_OK || (st = up("sig", sigma.data(), 8 * ncv)) != ARB_OK ||
        (st = up("dsig", dsig.data(), 8 * ncv)) != ARB_OK || (st = up("glin", glin.data(), 8 * ncv)) != ARB_OK ||
        (st = up("gelin", gelin.data(), 8 * ncv)) != ARB_OK || (st = up("area", area.data(), 8 * ncv)) != ARB_OK ||
        (st = up("kcm", kcm.data(), 8 * ncv)) != ARB_OK || (st = up("ksc", ksc.data(), 8 * ncv)) != ARB_OK ||
        (st = up("gna3", gna3.data(), 8 * nhh)) != ARB_OK || (st = up("gk4", gk4.data(), 8 * nhh)) != ARB_OK ||
        (st = up("hidx", hidx.data(), 4 * ncv)) != ARB_OK || (st = up("gna", gna.data(), 8 * nhh)) != ARB_OK ||
        (st = up("gk", gk.data(), 8 * nhh)) != ARB_OK || (st = up("gl", gl.data(), 8 * nhh)) != ARB_OK ||
        (st = up("st_ptr", st_ptr.data(), 8 * (nc + 1))) != ARB_OK || (st = up("st_cv", st_cv.data(), 8 * nst)) != ARB_OK ||
        (st = up("st_on", st_on.data(), 8 * nst)) != ARB_OK || (st = up("st_dur", st_dur.data(), 8 * nst)) != ARB_OK ||
        (st = up("st_amp", st_amp.data(), 8 * nst)) != ARB_OK || (st = up("obs", obs.data(), 4 * ncv)) != ARB_OK ||
        (st = up("grp_ptr", grp_ptr.data(), 8 * ((size_t)n_groups + 1))) != ARB_OK ||
        (st = up("grp_cv", grp_cv.data(), 8 * grp_cv.size())) != ARB_OK ||
        (st = up("ch_ptr", CP.ch_ptr.data(), 8 * CP.ch_ptr.size())) != ARB_OK ||
        (st = up("lev_off", CP.lev_off.data(), 8 * CP.lev_off.size())) != ARB_OK ||
        (st = up("lev_bound", CP.lev_bound.data(), 8 * CP.lev_bound.size())) != ARB_OK ||
        (st = up("ch_cv_ptr", CP.ch_cv_ptr.data(), 8 * CP.ch_cv_ptr.size())) != ARB_OK ||
        (st = up("ch_cvs", CP.ch_cvs.data(), 4 * CP.ch_cvs.size())) != ARB_OK ||
        (st = up("ch_kid_ptr", CP.ch_kid_ptr.data(), 8 * CP.ch_kid_ptr.size())) != ARB_OK ||
        (st = up("ch_kids", CP.ch_kids.data(), 8 * CP.ch_kids.size())) != ARB_OK ||
        (st = up("rho", CP.rho.data(), 8 * ncv)) != ARB_OK || (st = up("beta", CP.beta.data(), 8 * ncv)) != ARB_OK ||
        (st = up("gcf", CP.gcf.data(), 8 * ncv)) != ARB_OK || (st = up("srf", CP.srf.data(), 8 * ncv)) != ARB_OK ||
        (st = up("prev", CP.prev.data(), 4 * ncv)) != ARB_OK || (st = up("kpw", CP.kpw.data(), 8 * CP.kpw.size())) != ARB_OK ||
        (st = up("tk", CP.tk.data(), 4 * CP.tk.size())) != ARB_OK || (st = up("tk_ptr", CP.tk_ptr.data(), 8 * CP.tk_ptr.size())) != ARB_OK ||
        (st = up("tkb", CP.tkb.data(), 4 * CP.tkb.size())) != ARB_OK || (st = up("fixa", CP.fixa.data(), 4 * ncv)) != ARB_OK)
        return st;
    // slopes of the gate table's cubics per mV, for the recording passes: per interval and
    // quantity (c1, 2 c2, 3 c3) x kHHTabPerMV of the cubic c0 + c1 s + c2 s^2 + c3 s^3
    std::vector<double> dtab;
    if (!sim->hh_tab.empty()) {
        dtab.assign((size_t)kHHTabN * kHHTabStride, 0.0);
        const double* tb = sim->hh_tab.data();
        for (int64_t it = 0; it < kHHTabN; ++it)
            for (int q = 0; q < 6; ++q) {
                const double* cq = tb + it * kHHTabStride + 4 * q;
                double* dq = dtab.data() + it * kHHTabStride + 4 * q;
                dq[0] = cq[1] * kHHTabPerMV;
                dq[1] = 2.0 * cq[2] * kHHTabPerMV;
                dq[2] = 3.0 * cq[3] * kHHTabPerMV;
            }
        if ((st = up("hh_dtab", dtab.data(), 8 * dtab.size())) != ARB_OK) return st;
    }
    AdjArgs a{};
    a.n_cells = (int32_t)nc;
    a.n_cv = ncv;
    a.n_hh = nhh;
    a.off = (const int64_t*)L.at(base, "off");
    a.parent = (const int32_t*)L.at(base, "parent");
    a.cdt = (const double*)L.at(base, "cdt");
    a.sig = (const double*)L.at(base, "sig");
    a.dsig = (const double*)L.at(base, "dsig");
    a.glin = (const double*)L.at(base, "glin");
    a.gelin = (const double*)L.at(base, "gelin");
    a.area = (const double*)L.at(base, "area");
    a.kcm = (const double*)L.at(base, "kcm");
    a.ksc = (const double*)L.at(base, "ksc");
    a.hidx = (const int32_t*)L.at(base, "hidx");
    a.gna = (const double*)L.at(base, "gna");
    a.gk = (const double*)L.at(base, "gk");
    a.gl = (const double*)L.at(base, "gl");
    a.gna3 = (const double*)L.at(base, "gna3");
    a.gk4 = (const double*)L.at(base, "gk4");
    a.st_ptr = (const int64_t*)L.at(base, "st_ptr");
    a.st_cv = (const int64_t*)L.at(base, "st_cv");
    a.st_on = (const double*)L.at(base, "st_on");
    a.st_dur = (const double*)L.at(base, "st_dur");
    a.st_amp = (const double*)L.at(base, "st_amp");
    a.obs = (const int32_t*)L.at(base, "obs");
    a.n_obs = n_obs;
    a.target = target;
    a.loss_scale = loss_scale;
    a.dt = dt;
    a.hh_tab = sim->hh_tab.empty() ? nullptr : (const double*)region(sim, "hh_tab");
    a.hh_dtab = sim->hh_tab.empty() ? nullptr : (const double*)L.at(base, "hh_dtab");
    a.k0 = sim->k;
    a.n_steps = n_steps;
    a.ckpt = checkpoint_every;
    a.V = (double*)L.at(base, "V");
    a.Y = (double*)L.at(base, "Y");
    a.ckV = (double*)L.at(base, "ckV");
    a.ckY = (double*)L.at(base, "ckY");
    a.segV[0] = (double*)L.at(base, "segV0");
    a.segV[1] = (double*)L.at(base, "segV1");
    a.segY[0] = (double*)L.at(base, "segY0");
    a.segY[1] = (double*)L.at(base, "segY1");
    a.segG[0] = (double*)L.at(base, "segG0");
    a.segG[1] = (double*)L.at(base, "segG1");
    a.lam = (double*)L.at(base, "lam");
    a.ybar = (double*)L.at(base, "ybar");
    a.gacc = (double*)L.at(base, "gacc");
    a.cell_loss = (double*)L.at(base, "cell_loss");
    a.loss_part = (double*)L.at(base, "loss_part");
    a.ch_ptr = (const int64_t*)L.at(base, "ch_ptr");
    a.lev_off = (const int64_t*)L.at(base, "lev_off");
    a.lev_bound = (const int64_t*)L.at(base, "lev_bound");
    a.ch_cv_ptr = (const int64_t*)L.at(base, "ch_cv_ptr");
    a.ch_cvs = (const int32_t*)L.at(base, "ch_cvs");
    a.ch_kid_ptr = (const int64_t*)L.at(base, "ch_kid_ptr");
    a.ch_kids = (const int64_t*)L.at(base, "ch_kids");
    a.rho = (const double*)L.at(base, "rho");
    a.beta = (const double*)L.at(base, "beta");
    a.gcf = (const double*)L.at(base, "gcf");
    a.srf = (const double*)L.at(base, "srf");
    a.prev = (const int32_t*)L.at(base, "prev");
    a.kpw = (const double*)L.at(base, "kpw");
    a.tk = (const int32_t*)L.at(base, "tk");
    a.tk_ptr = (const int64_t*)L.at(base, "tk_ptr");
    a.tkb = (const int32_t*)L.at(base, "tkb");
    a.fixa = (const int32_t*)L.at(base, "fixa");
    a.smem_cv = std::max<int32_t>(CP.max_cv, 1);
    a.smem_ch = std::max<int32_t>(CP.max_ch, 1);
    a.smem_tk = std::max<int32_t>(CP.max_tk, 1);
    CU(adj_prepare(a));
    a.grp_ptr = (const int64_t*)L.at(base, "grp_ptr");
    a.grp_cv = (const int64_t*)L.at(base, "grp_cv");
    a.n_groups = n_groups;
    a.grad = grad;
    // the handle's current state, in model order
    CU(launch_gather<double>(a.V, (const double*)region(sim, "V"), (const int64_t*)region(sim, "cv_tile"), ncv, sim->s));
    const char* gname[3] = {"hh_m", "hh_h", "hh_n"};
    for (int g = 0; g < 3 && nhh > 0; ++g) {
        const int64_t* idx = (const int64_t*)region(sim, "hh_entry");
        if (sim->mixed) CU(launch_gather<float>(a.Y + g * nhh, (const float*)region(sim, gname[g]), idx, nhh, sim->s));
        else CU(launch_gather<double>(a.Y + g * nhh, (const double*)region(sim, gname[g]), idx, nhh, sim->s));
    }
    CU(cudaMemsetAsync(a.lam, 0, 8 * ncv, sim->s));
    if (nhh > 0) CU(cudaMemsetAsync(a.ybar, 0, 24 * nhh, sim->s));
    CU(cudaMemsetAsync(a.gacc, 0, 32 * ncv, sim->s));
    CU(cudaMemsetAsync(a.cell_loss, 0, 8 * nc, sim->s));
    CU(cudaMemsetAsync(a.loss_part, 0, 8 * nc * (int64_t)kAdjBlock, sim->s));
    // forward with checkpoints, then segment by segment backwards: recompute, reverse sweep
    CU(cudaEventRecord(sim->t0[0], sim->s));
    // segment g lives in buffer g % 2; each stage sweeps segment g backwards while the
    // segment before it is recomputed from its checkpoint into the other buffer. The forward
    // pass keeps every state of the last segment, which therefore needs no recompute.
    const int64_t nck = (n_steps + checkpoint_every - 1) / checkpoint_every;
    auto seg = [&](int64_t g, int64_t& s0, int64_t& s1) {
        s0 = g * checkpoint_every;
        s1 = std::min<int64_t>(n_steps, s0 + checkpoint_every);
    };
    {
        int64_t f0, f1;
        seg(nck - 1, f0, f1);
        CU(launch_adj_forward(a, 0, f0, 0, 0, sim->s));                              // with checkpoints
        CU(launch_adj_forward(a, f0, f1, 2, (int)((nck - 1) % 2), sim->s));          // last segment
    }
    for (int64_t g = nck - 1; g >= 0; --g) {
        int64_t r0, r1, f0 = 0, f1 = 0;
        seg(g, r0, r1);
        if (g > 0) seg(g - 1, f0, f1);
        CU(launch_adj_stage(a, r0, r1, (int)(g % 2), f0, f1, sim->s));
    }
    CU(launch_adj_reduce(a, sim->s));
    CU(cudaEventRecord(sim->t1[0], sim->s));
    std::vector<double> cl(nc);
    if (nc > 0) CU(cudaMemcpyAsync(cl.data(), a.cell_loss, 8 * nc, cudaMemcpyDeviceToHost, sim->s));
    CU(cudaStreamSynchronize(sim->s));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, sim->t0[0], sim->t1[0]));
    sim->pending_time[0] = false;
    sim->last_epoch_ms = ms;
    sim->last_launches = (nck > 1 ? 2 : 1) + nck + 1;
    double total = 0.0;
    for (double x : cl) total += x;
    *loss = total;
    return sync_out(sim);
}

}  // extern "C"
