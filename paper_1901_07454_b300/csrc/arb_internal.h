// Internal types shared by the host runtime (arb_runtime.cu) and the kernels (arb_kernels.cu).
#pragma once
#include <cmath>
#include <cstdint>

namespace arbk {

constexpr int kWarp = 32;

// Reversal potentials of the Hodgkin-Huxley channels (mV).
constexpr double kENa = 50.0;
constexpr double kEK = -77.0;
constexpr double kEL = -54.3;

// One pack = the program of one warp: a group of cells whose CVs are laid out in
// "rows" of 32 lanes. Entry (row j, lane l) of pack p lives at global index
// (row0 + j) * 32 + l of every per-entry array; its state slot inside the pack's tile
// is j * 32 + l.
struct PackDesc {
    int32_t row0;        // first solve row (global)
    int32_t nrow;        // solve rows J
    int32_t round_rows;  // rows per synchronisation round; 0 = lanes are independent
    int32_t smem;        // 1: S and V tiles staged in shared memory, 0: tiles in global memory
    int64_t sg_off;      // offset (in doubles) of this pack's S scratch in global memory (smem == 0)
    int32_t syn_row0, nsyn_row;
    int32_t hh_row0, nhh_row;
    int32_t st_row0, nst_row;
    int32_t ncell;       // detectors: lane d < ncell owns detector d
    int32_t pr0, npr;    // probes of this pack: entries [pr0, pr0 + npr) of the probe arrays
    int32_t nvc;         // shared-memory packs: voltages kept on chip (see vmap);
                         // streamed packs: compact mechanism slots (see vmap)
    int32_t stack;       // streamed packs: deepest per-lane hand-over stack (entries)
    int64_t c_off;       // streamed packs: offset of the pack's compact slots in Gm / Em
    int32_t nmb;         // streamed shared packs: mailbox slots (cross-lane hand-overs)
    int32_t nsc;         // streamed packs: compact slots [0, nsc) are the CVs with synapses,
                         // whose terms the synapse pass writes whole (no read-modify-write)
    int32_t mb0;         // streamed shared packs: first of the pack's entries in mb_ent / mb_cs
    int32_t pad_mb;
};

// Pack modes: staged in shared memory (small batches, several cells share a warp), or
// streamed from global memory (large batches, one cell per lane).
enum : int32_t { kPackGlobal = 0, kPackSmem = 1, kPackStream = 2 };

// Streamed packs: per-entry flags in pslot. Bits 0-7: children handed over through the
// stack (all but the one processed directly before the parent); bit 8: this entry's parent
// is not the next row of its lane; bit 9: root.
enum : int32_t { kFlagPopMask = 0xFF, kFlagRemote = 0x100, kFlagRoot = 0x200 };
// Streamed shared packs (cells spread over several lanes, rounds of round_rows rows separated
// by __syncwarp): no stack; hand-overs go through a per-warp mailbox in shared memory, and
// the flags word also holds two 11-bit mailbox slots. out (bits 10..20): the slot this entry
// adds its contribution to and reads its parent's voltage from; in (bits 21..31): the slot
// that holds the contributions of this entry's handed-over children and where its voltage is
// published for them. kMbNone = no slot.
constexpr int32_t kMbNone = 0x7FF;
constexpr int kMbOutShift = 10;
constexpr int kMbInShift = 21;
#ifndef ARB_STREAM_WARPS
#define ARB_STREAM_WARPS 16
#endif
constexpr int kStreamWarps = ARB_STREAM_WARPS;   // warps per CTA of the streamed kernel (one CTA per SM)
#ifndef ARB_STREAM_ROUND
#define ARB_STREAM_ROUND 4
#endif
constexpr int kStreamRound = ARB_STREAM_ROUND;   // rows per round in streamed shared packs

// Event delivered inside one epoch, bucketed per owner lane and sorted by
// (step_rel, js, t, src, idx).
struct EvRec {
    double t;
    double w;
    int32_t step_rel;   // step index relative to the epoch start
    int32_t js;         // synapse row of the owner lane (relative to the pack's syn_row0)
    int32_t src;        // source gid, -1 external
    int32_t idx;        // connection index or external enqueue index
};

// Event waiting on the device for a later epoch.
struct PendEv {
    double t;
    double w;
    int64_t step;       // absolute step at whose start it is applied
    int32_t syn;        // global synapse index
    int32_t src;
    int32_t idx;
    int32_t pad;
};

// Device control block: values that change from epoch to epoch live here, so one
// captured CUDA graph serves every epoch.
struct Ctl {
    int64_t k0, k1, k_end;     // epoch being integrated [k0, k1); run target k_end
    int64_t ext_lo, ext_hi;    // external events of the epoch being prepared, in the sorted
                               // external array
    int64_t n_ext;             // external events resident
    int64_t n_spikes;          // spikes recorded so far
    int64_t spk_mark;          // spikes recorded before the epoch being integrated
    int64_t probe_k0;          // step at which probe row 0 is taken
    int64_t probe_max;         // probe rows available
    int64_t pool_n64[2];       // pending network events in pool 0 / 1 (may count past the capacity)
    int32_t parity;            // pool holding the events not yet delivered
    int32_t n_due;             // events delivered in the last prepared epoch
    int32_t pack_next;         // work counter of the persistent epoch kernel
    int32_t status;            // ARBK_* flags
    int64_t kp0, kp1;          // epoch whose delivery lists are being built [kp0, kp1); kp0 is
                               // the first step whose lists are not built yet
    int64_t xr_lo[2], xr_hi[2];// spike ranges of integrated epochs not yet walked (ring of two)
    int32_t prep_slot;         // delivery-list buffer the preparation writes next (0 / 1); the
                               // integration of the same epoch reads it through its own graph
    int32_t xw, xr;            // spike-range ring: next entry written / next entry walked
    int32_t pad_x;
};

// Tabulated HH gate update (streamed packs, FP64, steps of fixed dt): for V in
// [kHHTabVlo, kHHTabVlo + kHHTabN / kHHTabPerMV) mV the six functions of V that the exact gate
// update x' = x_inf + (x - x_inf) e needs, x_inf = alpha / (alpha + beta) and
// e = exp(-dt (alpha + beta)) for the gates m, h and n, are cubic polynomials in
// s = (V - V_i) kHHTabPerMV on each interval [V_i, V_i + 1 / kHHTabPerMV): 24 coefficients per
// interval, function-major (m_inf, e_m, h_inf, e_h, n_inf, e_n), each c0 + c1 s + c2 s^2 + c3 s^3.
constexpr double kHHTabVlo = -128.0;
constexpr double kHHTabPerMV = 256.0;
constexpr int32_t kHHTabN = 192 * 256;
constexpr int32_t kHHTabStride = 24;

enum : int32_t {
    kStSpikeOverflow = 1,
    kStPoolOverflow = 2,
    kStBucketOverflow = 4,
    kStNonFinite = 8,
    kStLateEvent = 16,
    kStBounds = 32,           // debug builds: an index array held a value outside its range
};

// Debug builds (ARB_DEBUG): ARB_IDX(i, n, ctl) checks an index read from an index array against
// [0, n). Outside it, the kernel records kStBounds in the control block and uses index 0 instead
// (an address that exists), so that nothing faults and no lane leaves a warp-synchronous region
// early; the host reports the flag after the epoch. Release builds use the index unchecked.
struct Ctl;
#ifdef ARB_DEBUG
__device__ __forceinline__ int64_t dbg_idx(int64_t i, int64_t n, Ctl* ctl);
#define ARB_IDX(i, n, ctl) ((int)::arbk::dbg_idx((int64_t)(i), (int64_t)(n), (ctl)))
#define ARB_IDX64(i, n, ctl) (::arbk::dbg_idx((int64_t)(i), (int64_t)(n), (ctl)))
#else
#define ARB_IDX(i, n, ctl) (i)
#define ARB_IDX64(i, n, ctl) (i)
#endif

// Everything the device kernels read; pointers into the caller's workspace.
template <class MT>
struct DevModel {
    const PackDesc* packs;
    int32_t n_packs;
    int32_t n_owner;          // n_packs * 32
    // solve entries (total_rows * 32); meaning depends on the scheme:
    //   explicit membrane current (constant matrix, factorised on the host):
    //     ca = (c/dt - G_lin)/d', cb = G_lin E_lin/d', ck = a/d'_parent, ce = a/d'
    //   implicit membrane conductance (matrix changes every step):
    //     ca = c/dt, cb = G_lin E_lin, ck = sigma (axial conductance to the parent),
    //     ce = c/dt + G_lin + sum of the entry's axial conductances (constant diagonal)
    const double* ca;
    const double* cb;
    const double* ck;
    const double* ce;
    const int32_t* pslot;     // -1 parent is the next row of this lane, -2 none, >= 0 parent's tile slot
    const int32_t* vmap;      // shared-memory packs: low 16 bits own on-chip V slot, high 16 bits the
                              // parent's (0xFFFF = none); only CVs whose voltage is read keep one
    double* V;                // voltages, tile layout
    double* Sg;               // S scratch for packs whose tiles live in global memory
    double* Rg;               // diagonal / e scratch of those packs (implicit scheme)
    double* Gm;               // streamed packs, per compact mechanism slot: the diagonal (implicit:
                              // constant part + membrane conductance of the step)
    double* Em;               // ... and the right-hand side terms (implicit: passive g E + membrane
                              // g E + clamp current)
    const double* cE;         // streamed packs, implicit: constant diagonal and right-hand side of
    const double* cB;         // each compact slot (ce, cb of its entry), which Gm and Em start from
    // synapses (syn_rows * 32)
    const int32_t* syn_slot;  // tile slot of the synapse's CV, -1 padding
    const int32_t* syn_vs;    // where its voltage is read (on-chip V slot, or the tile slot)
    MT* syn_g;
    const double* syn_e;
    const double* syn_decay;  // exp(-dt/tau)
    const double* syn_sc;     // 1/d' of the CV
    // Hodgkin-Huxley (hh_rows * 32)
    const int32_t* hh_slot;
    const int32_t* hh_vs;
    const double* hh_sc;
    const double* hh_tab;     // tabulated gate update ([kHHTabN][24]), or null: rates evaluated
    const float* hh_tab_f;    // the same rounded to float (FP32 mechanisms), or null
    const double* hh_gna;     // uS
    const double* hh_gk;      // uS
    MT* hh_m;
    MT* hh_h;
    MT* hh_n;
    // current clamps (st_rows * 32)
    const int32_t* st_slot;
    const double* st_sc;
    const double* st_on;
    const double* st_off;
    const double* st_amp;
    // detectors (n_owner)
    const int32_t* det_slot;  // where the detector voltage is read (on-chip V slot or tile slot)
    const int32_t* det_gid;
    // probes, grouped by pack: tile slot of the CV and trace column
    const int32_t* probe_slot;
    const int32_t* probe_col;
    int64_t n_probe;
    double* trace;
    // events
    const int32_t* ev_off;    // [n_owner + 1] of one delivery-list buffer
    const EvRec* ev;
    // spikes
    int32_t* spk_gid;
    double* spk_t;
    int64_t spike_cap;
    Ctl* ctl;
    double dt;
    double threshold;
    int32_t exact;            // 1: steps are cut at event times (one cell per lane, own mechanisms)
    int32_t pad_exact;
    const double* syn_ntau;   // per synapse row entry: -1/tau (exact event times)
    const int32_t* slot_lo;   // exact event times: per lane (owner), its range of compact slots
    const int32_t* slot_hi;
    // streamed packs, implicit scheme, step-start events (the row-ring path): the forward result
    // (u, e) per entry; per entry its position among its row's compact slots (cpos, -1 none); per
    // global row the range of its compact slots with synapses (row_cs: first slot | count << 24)
    // and of its other compact slots (row_cn: first slot counted from nsc | count << 24)
    double2* UE;
    const int32_t* cpos;
    const int32_t* row_cs;
    const int32_t* row_cn;
    // streamed shared packs on the row-ring path: per mailbox slot (pack after pack, from the
    // pack's mb0) the parent's entry in its pack and that entry's compact slot (-1 none)
    const int32_t* mb_ent;
    const int32_t* mb_cs;
    // FP32 mechanisms: float copies of the per-synapse decay factor and reversal and of the HH
    // conductances (null otherwise)
    const float* syn_decay_f;
    const float* syn_e_f;
    const float* hh_gna_f;
    const float* hh_gk_f;
};

// Arguments of the event-delivery kernels.
struct EvArgs {
    Ctl* ctl;
    PendEv* pool[2];
    int64_t pool_cap;
    const int64_t* ext_step;
    const double* ext_t;
    const double* ext_w;
    const int32_t* ext_syn;
    const int32_t* ext_idx;
    const int32_t* syn_owner;
    const int32_t* syn_js;
    int32_t* counts;
    int32_t* off;
    EvRec* rec;
    EvRec* tmp;               // [bucket_cap] scratch of the long-list sort
    int64_t bucket_cap;       // records per delivery-list buffer
    int32_t n_owner;
    int32_t epoch_steps;
    int32_t time_major;       // 1: order within a step by time first (exact event times)
    int32_t slot_mask;        // 1: two delivery-list buffers (overlapped exchange), 0: one
    int64_t n_syn;            // synapse state units (debug index checks)
};

// Delivery lists of buffer `slot`: off[slot * (n_owner + 1) + o] .. [o + 1] index the records
// of owner o in rec[], as absolute positions inside rec[slot * bucket_cap, (slot + 1) * bucket_cap).

// Arguments of the spike-exchange kernel.
struct SpkArgs {
    int32_t exact;            // 1: an event belongs to the step j with j*dt <= t < (j+1)*dt
    int32_t pad_exact;
    Ctl* ctl;
    const int32_t* spk_gid;
    const double* spk_t;
    int64_t spike_cap;
    const int64_t* out_ptr;
    const int32_t* out_syn;
    const int32_t* out_idx;
    const double* out_delay;
    const double* out_w;
    PendEv* pool[2];
    int64_t pool_cap;
    double dt;
    int64_t n_cells;          // local cells
    int64_t dry_ranks;        // virtual ranks: each local spike is walked once per rank
};

// Step of an event at time t (ms). Fixed-step rule: the event is applied at the start of step
// ceil(t/dt). Exact event times: the step j with j*dt <= t < (j+1)*dt, on the grid of the
// products k*dt that the step times are formed from.
__host__ __device__ inline int64_t event_step(double t, double dt, bool exact) {
    if (!exact) return (int64_t)ceil(t / dt);
    int64_t j = (int64_t)floor(t / dt);
    while ((double)(j + 1) * dt <= t) ++j;
    while ((double)j * dt > t) --j;
    return j;
}

constexpr int kAdjBlock = 128;   // adjoint kernels: threads per block (one block per cell)

// Discrete adjoint (model order: CVs of a cell contiguous, parent index below the child's).
// Per-step state: V [n_cv] and the gates Y [3][n_hh] (m, h, n of HH instance j).
struct AdjArgs {
    int32_t n_cells;
    int64_t n_cv, n_hh;
    const int64_t* off;        // [n_cells+1]
    const int32_t* parent;     // [n_cv] cell-local parent in the tree the solve uses (the cell re-rooted), -1 at its root
    const double* cdt;         // [n_cv] C / dt (nF/ms = uS)
    const double* sig;         // [n_cv] axial conductance to the parent (uS), 0 at the root
    const double* dsig;        // [n_cv] sum of the axial conductances of the CV (own + children)
    const double* glin;        // [n_cv] passive conductance (uS)
    const double* gelin;       // [n_cv] passive conductance x reversal (nA)
    const double* area;        // [n_cv] um^2
    const double* kcm;         // [n_cv] area 1e-5 / dt: the cm gradient's factor
    const double* ksc;         // [n_cv] area 1e-2: the channel densities' factor
    const int32_t* hidx;       // [n_cv] HH instance on the CV, -1 none
    const double* hh_tab;      // tabulated gate update of the simulation's dt, or null
    const double* hh_dtab;     // slopes per mV of the table's cubics ([kHHTabN][24]: c1, 2 c2, 3 c3, 0 per quantity), or null
    const double* gna;         // [n_hh] uS
    const double* gk;
    const double* gl;
    const double* gna3;        // [n_hh] 3 gna
    const double* gk4;         // [n_hh] 4 gk
    const int64_t* st_ptr;     // [n_cells+1] clamps of each cell
    const int64_t* st_cv;      // global CV
    const double* st_on;
    const double* st_dur;
    const double* st_amp;
    const int32_t* obs;        // [n_cv] loss column of the CV, -1 none
    int64_t n_obs;
    const double* target;      // [n_steps][n_obs]
    double loss_scale;
    double dt;
    int64_t k0;                // step of the handle at the start
    int64_t n_steps;
    int32_t ckpt;              // steps between checkpoints
    double* V;                 // [n_cv] running state (forward pass)
    double* Y;                 // [3][n_hh]
    double* ckV;               // [n_ckpt][n_cv]
    double* ckY;               // [n_ckpt][3][n_hh]
    // two segment buffers (one is swept backwards while the next is recomputed)
    double* segV[2];           // [ckpt+1][n_cv]
    double* segY[2];           // [ckpt+1][3][n_hh]
    double* segG[2];           // [ckpt][6][n_hh] per step: dPhi/dV of m, h, n and exp(-dt (alpha+beta))
                               // of m, h, n, written by the recompute pass for the reverse sweep
    double* lam;               // [n_cv] solve result of the later step
    double* ybar;              // [3][n_hh]
    double* gacc;              // [4][n_cv] gradient per CV: gnabar, gkbar, gl, cm
    double* cell_loss;         // [n_cells]
    double* loss_part;         // [n_cells][kAdjBlock] each thread's loss sum, carried between forward launches
    // tree solve schedule: the unbranched chains of each cell, ordered by level (leaf chains
    // level 0, a chain's level is one more than its highest child chain)
    const int64_t* ch_ptr;     // [n_cells+1] chains of cell c (global chain indices)
    const int64_t* lev_off;    // [n_cells+1] offsets into lev_bound
    const int64_t* lev_bound;  // per cell: first chain of each level, then one past the last
    const int64_t* ch_cv_ptr;  // [n_chains+1] range of the chain in ch_cvs
    const int32_t* ch_cvs;     // cell-local CVs of each chain, head (nearest the root) first
    const int64_t* ch_kid_ptr; // [n_chains+1] range of the chain's child chains in ch_kids
    const int64_t* ch_kids;    // global chain indices
    // constants of the scaled chain recurrence (model order; see arb_adjoint.cu)
    const double* rho;         // [n_cv] c_{k-1} / c_k (1 at a chain's tail)
    const double* beta;        // [n_cv] c_{k-1} / g_k (1 at a chain's tail)
    const double* gcf;         // [n_cv] g_k / c_k
    const double* srf;         // [n_cv] s_k rho_k (0 at the root)
    const int32_t* prev;       // [n_cv] cell-local CV before this one in its chain, -1 at a tail
    const double* kpw;         // [n_chains][2] s_h^2 rho_h, s_h g_h / c_h of the chain's head h
    // back-substitution tasks: [start, end) positions in the cell's chain list, kind (0 a chain or
    // its upper part, 1 a lower part's offsets, 2 its factors), anchor CV (cell-local)
    const int32_t* tk;         // [tasks][4]
    const int64_t* tk_ptr;     // [n_cells+1] first task of each cell
    const int32_t* tkb;        // per cell (laid out as lev_bound): cell-local first task of each level, then the end
    const int32_t* fixa;       // [n_cv] cell-local anchor whose value a lower-part CV still needs, -1 none
    int32_t smem_tk;           // largest task count of a cell
    int32_t smem_cv;           // shared-memory slots per cell (largest cell)
    int32_t smem_ch;           // largest chain count of a cell
    const int64_t* grp_ptr;    // [n_groups+1] CVs of each parameter group, ascending
    const int64_t* grp_cv;
    int32_t n_groups;
    double* grad;              // [n_groups][4] output
};

// Dynamic shared memory of one adjoint block: per CV 16 doubles and 5 int32, per chain 4
// doubles and 5 int32 (with the level bounds of the tasks), per back-substitution task 4 int32,
// and 8 int32 more of level bounds.
inline size_t adj_smem_bytes_for(int64_t cvs, int64_t chains, int64_t tasks) {
    return 8 * (16 * (size_t)cvs + 4 * (size_t)chains) + 4 * (5 * (size_t)cvs + 5 * (size_t)chains + 4 * (size_t)tasks + 8);
}

#ifdef ARB_DEBUG
__device__ __forceinline__ int64_t dbg_idx(int64_t i, int64_t n, Ctl* ctl) {
    if (i < 0 || i >= n) {
        atomicOr(&ctl->status, (int)kStBounds);
        return 0;
    }
    return i;
}
#endif

}  // namespace arbk
