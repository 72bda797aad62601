/*
 * arb.h -- C ABI of the B300 batched cable-equation stepper.
 *
 * The library advances a batch of multicompartment neurons with the method of
 * arXiv 1901.07454 (Arbor), Sec. "Model": finite-volume cable equation per cell, membrane
 * terms from the channel and synapse states at t, one implicit-Euler voltage step solved
 * on each cell's tree-shaped (Hines) matrix, then channel/synapse state updates with the new
 * voltage, threshold spike detection, and spike exchange once per minimum-delay epoch
 * (Sec. "Implementation", "Simulation workflow"). It also computes the discrete adjoint of
 * that step (arb_adjoint). Every stage runs in the library's own sm_103a CUDA kernels.
 *
 * Conventions for every entry point:
 *  - Units: mV, ms, um, uF/cm^2, Ohm*cm, S/cm^2 (channel densities), uS (synaptic
 *    weights), nA (injected current, positive = depolarising).
 *  - Every call returns an arb_status; nothing throws across the ABI. arb_last_error()
 *    gives a message for the last failing call on a handle.
 *  - Host input arrays belong to the caller and are copied before the call returns.
 *  - The library allocates no device memory itself: the caller provides one device
 *    workspace (see arb_workspace_bytes / arb_bind_workspace) and any output buffers.
 *  - Calls on one handle are not thread-safe. All device work of a handle is issued on
 *    the stream given in arb_params.stream (0 = legacy default stream).
 */
#ifndef ARB_B300_H
#define ARB_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct arb_sim arb_sim;

typedef enum {
    ARB_OK = 0,
    ARB_E_ARG = -1,        /* invalid argument or model (message says which) */
    ARB_E_CUDA = -2,       /* a CUDA runtime call failed */
    ARB_E_OVERFLOW = -3,   /* an event, spike or bucket capacity was exceeded */
    ARB_E_NONFINITE = -4,  /* a voltage became NaN or infinite */
    ARB_E_STATE = -5,      /* call not valid in the handle's current state */
    ARB_E_NOMEM = -6       /* host allocation failed, or the workspace is too small */
} arb_status;

enum { ARB_FP64 = 0, ARB_MIXED = 1 };

/* How the membrane current enters the implicit Euler step of Sec. "Model":
 * ARB_IMPLICIT (default): channel and synapse states are taken at t and the step of
 *   Eq. (discrete-v) is implicit in V, i.e. the membrane conductance sits on the diagonal:
 *   (c/dt + g) V' + sum sigma (V' - V'_j) = (c/dt) V + sum g E + I_inj. The matrix changes
 *   every step and is eliminated every step. Unconditionally stable.
 * ARB_EXPLICIT: the linear system as printed in Sec. "Model", membrane current at V(t) on the
 *   right-hand side. The matrix is constant and factorised once, but the step diverges when
 *   dt * g / c > 2 in a compartment, which happens in small cells under synaptic bursts. */
enum { ARB_IMPLICIT = 0, ARB_EXPLICIT = 1 };

/* When events take effect (arb_params.event_timing). */
enum { ARB_EVENTS_STEP_START = 0, ARB_EVENTS_EXACT = 1 };

/* Run settings. Fill with arb_default_params, then override. */
typedef struct {
    double dt;                   /* time step, ms (> 0) */
    int32_t epoch_steps;         /* steps per epoch; 0 = floor(min delay / dt), 400 without connections */
    int32_t precision;           /* ARB_FP64, or ARB_MIXED: mechanism states and currents in FP32,
                                    matrix solve and voltages in FP64 */
    int32_t cells_per_pack;      /* packing override: 0 = chosen by the library's cost model,
                                    32 = one cell per lane, 1..31 = cells sharing one warp */
    int32_t smem_budget;         /* bytes of shared memory per warp for state tiles; 0 = default */
    int32_t scheme;              /* ARB_IMPLICIT (default) or ARB_EXPLICIT */
    int32_t split_cvs;           /* cells_per_pack 32 only: a cell with more CVs than this is spread
                                    over several lanes (chains scheduled in rounds, hand-overs
                                    through shared memory); 0 = threshold chosen by the library
                                    from the load of a warp slot, -1 = never spread */
    int32_t coalesce_synapses;   /* 1: synapses on one CV with equal tau and e share one state
                                    (their conductances add linearly, so the voltages agree up to
                                    rounding); arb_get_state then reports each group's g on its
                                    lowest-index synapse and 0 on the others, arb_set_state sums a
                                    group's g. 0 (default): one state per synapse. */
    int32_t event_timing;        /* ARB_EVENTS_STEP_START (default): an event at t is applied at
                                    the start of step ceil(t/dt). ARB_EVENTS_EXACT: as in Sec.
                                    "Model", a step is cut at the times of the events inside it
                                    (each cell its own), every piece an implicit step of its own
                                    length; needs ARB_IMPLICIT and ARB_FP64 and runs one cell per
                                    lane (cells_per_pack 0 or 32, split_cvs 0 or -1). */
    int32_t epoch_overlap;       /* 1: epochs of half the minimum delay, as in Sec.
                                    "Implementation": while epoch i integrates, a second stream
                                    walks the spikes of epoch i-1 against the connections and
                                    builds the delivery lists of epoch i+1 (its events come from
                                    spikes of epoch i-1 or earlier). Every delay must be at least
                                    2 * epoch_steps * dt; epoch_steps = 0 then means
                                    floor(min delay / (2 dt)). The results equal those of the
                                    serial schedule with the same epoch length. 0 (default): each
                                    epoch's exchange runs between two integrations. */
    int32_t dry_run_ranks;       /* dry run (Sec. "Scalability": one rank mimics a large cluster
                                    by generating proxy spikes for the other ranks' cells): 0 or
                                    1 = off; R > 1: the model's n cells are rank 0 of R ranks
                                    holding copies of them (gids r*n .. r*n+n-1), connection
                                    sources are global gids in [0, R*n), and every local spike
                                    of gid g at t is walked against the connections of the R
                                    gids g + r*n. Spike reads return the local spikes only.
                                    R*n must be < 2^31. */
    int32_t spread_rows;         /* cells_per_pack 32: target solve rows of a pack of spread cells
                                    (large cells are grouped until their schedule would run about
                                    this long); 0 = the split threshold, or with split_cvs = 0 both
                                    chosen together by the library's cost model */
    int32_t kernel_variant;      /* streamed packs, ARB_IMPLICIT with step-start events: which
                                    compiled variant of the epoch kernel runs (warps per SM and
                                    rows prefetched, see arb_kernel_variants); -1 (default) = 0.
                                    The choice changes the plan's schedule (and so the rounding
                                    order of spread cells), not the method. */
    int64_t event_capacity;      /* pending network events held on the device at once */
    int64_t ext_event_capacity;  /* external events (arb_enqueue_events) held on the device */
    int64_t spike_capacity;      /* spikes recorded over the whole run */
    int64_t bucket_capacity;     /* events delivered within one epoch */
    void* stream;                /* cudaStream_t */
} arb_params;

/* Model: host arrays, copied at arb_create. CV indices are global (cell offset + local index). */
typedef struct {
    int32_t n_cells;
    const int64_t* cv_offset;    /* [n_cells+1] CVs of cell c are cv_offset[c] .. cv_offset[c+1]-1 */
    const int32_t* parent;       /* [n_cv] cell-local parent, -1 for the first CV of a cell only,
                                    otherwise 0 <= parent[i] < local index of i */
    const double* length_um;     /* [n_cv] cylinder length of each CV (> 0) */
    const double* radius_um;     /* [n_cv] cylinder radius (> 0) */
    const double* cm;            /* [n_cv] specific capacitance, uF/cm^2 (> 0) */
    const double* Ra;            /* [n_cv] axial resistivity, Ohm*cm (> 0) */
    /* Hodgkin-Huxley Na/K/leak (E_Na 50, E_K -77, E_L -54.3 mV), at most one per CV */
    int64_t n_hh;
    const int64_t* hh_cv;
    const double* gnabar;
    const double* gkbar;
    const double* gl;
    /* passive leak */
    int64_t n_pas;
    const int64_t* pas_cv;
    const double* g_pas;
    const double* e_pas;
    /* exponential synapses: dg/dt = -g/tau, I = g (V - e), an event adds its weight to g */
    int64_t n_syn;
    const int64_t* syn_cv;
    const double* syn_tau;
    const double* syn_e;
    /* current clamps: amp nA while t_on <= t_k < t_on + dur */
    int64_t n_stim;
    const int64_t* stim_cv;
    const double* stim_t_on;
    const double* stim_dur;
    const double* stim_amp;
    /* one threshold detector per cell */
    const int64_t* detector_cv;  /* [n_cells] a CV of that cell */
    double threshold;            /* mV, upward crossing */
    /* connections: a spike of cell conn_src[i] at t adds conn_weight[i] to synapse
       conn_dst_syn[i] at t + conn_delay[i]; every delay must be >= epoch_steps*dt (twice that
       with epoch_overlap); conn_src < n_cells, or < dry_run_ranks * n_cells in a dry run */
    int64_t n_conn;
    const int32_t* conn_src;
    const int64_t* conn_dst_syn;
    const double* conn_delay;
    const double* conn_weight;
} arb_model;

/* Sets dt = 0.025, precision FP64, the implicit scheme, automatic epoch and packing, and
 * capacities sized for typical runs. Never fails for a non-NULL argument. */
arb_status arb_default_params(arb_params* p);

/* Validates the model and prepares everything on the host: per-CV geometry; the constant
 * parts of the implicit-Euler system of Sec. "Model" (ARB_IMPLICIT: c/dt, the axial
 * conductances and the constant diagonal, the membrane terms being added per step; ARB_EXPLICIT:
 * the constant matrix and its Hines factorisation); the packing of cells into warps (one cell
 * per lane, cells spread over lanes, or cells sharing a warp) with its solve schedule.
 * Makes no CUDA call. On success *out owns a handle that must be released with arb_destroy. */
arb_status arb_create(const arb_model* model, const arb_params* params, arb_sim** out);

/* Releases the handle. Does not free the caller's workspace. NULL is ignored. */
void arb_destroy(arb_sim* sim);

/* Device bytes the handle needs (256-byte aligned start). */
arb_status arb_workspace_bytes(const arb_sim* sim, int64_t* bytes);

/* Binds a caller-owned device buffer of at least arb_workspace_bytes bytes, uploads the
 * model and sets the initial state (V = -65 mV, gates at steady state, synapses closed,
 * t = 0). The buffer must stay valid until arb_destroy. May be called once per handle. */
arb_status arb_bind_workspace(arb_sim* sim, void* dev_ptr, int64_t bytes);

/* Queues external events (host arrays of length n): at time t[i] the weight w[i] (uS) is
 * added to synapse syn[i]. Applied at the start of step ceil(t/dt) (the paper shortens the
 * step to land on event times; this library keeps dt fixed). Times must not lie before the
 * current time. Events may be enqueued in any order and across several calls, but all
 * calls for a time window must come before arb_advance passes it. */
arb_status arb_enqueue_events(arb_sim* sim, int64_t n, const int64_t* syn, const double* t,
                              const double* w);

/* Advances to step round(t_end/dt) in epochs of epoch_steps steps (the last one may be
 * shorter), exchanging spikes between epochs. Returns ARB_E_OVERFLOW / ARB_E_NONFINITE
 * when a device-side check failed during the call (state is then unspecified). */
arb_status arb_advance(arb_sim* sim, double t_end);

/* Current simulation time (steps * dt) and step count. */
arb_status arb_time(const arb_sim* sim, double* t, int64_t* steps);

/* Copies the voltage of all n_cv CVs, in the model's CV order, to out (a host pointer if
 * on_device == 0, else a device pointer). n_cv must equal the model's CV count. */
arb_status arb_read_voltage(arb_sim* sim, double* out, int64_t n_cv, int32_t on_device);

/* Number of spikes recorded so far. */
arb_status arb_num_spikes(arb_sim* sim, int64_t* n);

/* Copies up to cap recorded spikes (host arrays), sorted by (time, gid); *n_out = count. */
arb_status arb_read_spikes(arb_sim* sim, int32_t* gid, double* t, int64_t cap, int64_t* n_out);

/* Copies up to cap of the spikes recorded after the first `first` ones (host arrays), sorted
 * by (time, gid); *n_out = count (0 when first >= the number recorded). Spikes are recorded in
 * the order of the advance calls that found them and every spike of one call is later than
 * every spike of an earlier call, so reading from the count arb_num_spikes gave before an
 * advance returns exactly that advance's spikes, and successive reads concatenate into the
 * sorted list arb_read_spikes returns: per-epoch export costs O(new spikes). first < 0 gives
 * ARB_E_ARG. */
arb_status arb_read_spikes_from(arb_sim* sim, int64_t first, int32_t* gid, double* t, int64_t cap,
                                int64_t* n_out);

/* Records V(t_{k+1}) at n CVs after every step k, starting with the next step, into the
 * device array trace[max_steps][n] (row r = the r-th step after this call). Steps beyond
 * max_steps are not recorded. n = 0 switches probes off. cv: host array. */
arb_status arb_set_probes(arb_sim* sim, int64_t n, const int64_t* cv, double* dev_trace,
                          int64_t max_steps);

/* Full dynamic state, host arrays in model order: V [n_cv], HH gates m, h, n [n_hh],
 * synapse conductances g [n_syn]. Pending events are not part of it. */
arb_status arb_get_state(arb_sim* sim, double* V, double* m, double* h, double* n, double* g);
arb_status arb_set_state(arb_sim* sim, const double* V, const double* m, const double* h,
                         const double* n, const double* g);

/* Per pack, in the order the persistent epoch kernel takes them (for i < cap; arrays may be
 * NULL): solve rows; kind (0 streamed, one cell per lane; 1 streamed, cells spread over lanes in
 * rounds; 2 tile in shared memory; 3 tile in global memory); synapse + HH + clamp rows. *n_packs
 * gets the number of packs. Valid after arb_create; host-only. */
arb_status arb_plan_packs(const arb_sim* sim, int64_t cap, int32_t* rows, int32_t* kind, int32_t* mech_rows,
                          int64_t* n_packs);

/* Packing summary, valid after arb_create (any pointer may be NULL): number of packs (warp
 * programs); solve rows over all packs and in the longest pack; packs that use shared memory
 * (state tiles, or in streamed plans the mailbox of cells spread over lanes); the fraction of
 * lane-rows that carry a CV; steps per epoch; cells per pack (32 = streamed plan); the CV
 * count above which a cell is spread over several lanes (-1 = none); the target rows of a pack
 * of spread cells (-1 = none); and the kernel variant that runs the plan. */
arb_status arb_plan_info(const arb_sim* sim, int64_t* n_packs, int64_t* total_rows,
                         int64_t* smem_packs, double* lane_efficiency, int32_t* epoch_steps,
                         int64_t* max_pack_rows, int32_t* cells_per_pack, int64_t* split_cvs,
                         int64_t* spread_rows, int32_t* kernel_variant);

/* Device time of the epoch kernel summed over the last arb_advance call, in ms, and the
 * number of kernel launches it issued; after arb_adjoint, the device time of its forward,
 * recompute and reverse kernels and their launch count. */
arb_status arb_last_timing(const arb_sim* sim, double* epoch_kernel_ms, int64_t* launches);

/* Discrete adjoint of the implicit step (the reverse-mode derivative of the time stepper;
 * the paper has no adjoint, this extends its Sec. "Model" scheme). Starting from the handle's
 * current state and time t_k, it runs n_steps steps of the implicit step (ARB_IMPLICIT; FP64
 * whatever the precision setting) and returns
 *   *loss = loss_scale * sum_{s < n_steps} sum_o (V_{obs_cv[o]}(t_{k+s+1}) - target[s][o])^2
 * and grad[g][p] = dL/d theta_{g,p} for the per-group densities theta = (gnabar, gkbar, gl
 * in S/cm^2, cm in uF/cm^2): the derivative w.r.t. a value shared by every CV (and HH
 * instance) of group g, where group_of_cv[i] in [-1, n_groups) assigns CV i (-1: none). The
 * initial state is taken as fixed. The handle's state, time and events are not changed.
 * Gradients go through the conductance terms of the voltage step, the exact gate update
 * and the capacitance of every CV; models with synapses are refused (ARB_E_ARG).
 *   obs_cv [n_obs]: host, distinct CVs. target [n_steps][n_obs]: device. group_of_cv [n_cv]: host.
 *   grad [n_groups][4]: device, written. loss: host, written.
 *   workspace: caller-owned device memory of arb_adjoint_workspace_bytes bytes, 256-byte
 *   aligned. It holds one state every checkpoint_every steps, two buffers of every state (and
 *   gate-update factor) of a segment of checkpoint_every steps (the forward pass fills one for
 *   the last segment, the reverse sweep recomputes each earlier one from its checkpoint), the
 *   solve schedule and constants, and a table of the gate cubics' slopes.
 * Each cell's tree solve runs in one block's shared memory: cells of more than about 1,000 to
 * 1,400 CVs (depending on their number of unbranched chains) are refused with ARB_E_ARG. The
 * handle keeps the solve schedule it builds on the first call (it depends only on the model
 * and dt). Work is ordered on the handle's stream after the caller's stream; the call returns
 * after the loss has been copied back; ARB_E_STATE if the handle has no bound workspace. */
arb_status arb_adjoint_workspace_bytes(const arb_sim* sim, int64_t n_steps, int32_t checkpoint_every,
                                       int64_t n_obs, int32_t n_groups, int64_t* bytes);
arb_status arb_adjoint(arb_sim* sim, int64_t n_steps, int32_t checkpoint_every, int64_t n_obs,
                       const int64_t* obs_cv, const double* target, double loss_scale,
                       const int32_t* group_of_cv, int32_t n_groups, void* workspace,
                       int64_t workspace_bytes, double* grad, double* loss);

/* The library's own FP64 elementary functions, evaluated element-wise on caller-owned DEVICE
 * arrays (asynchronous on `stream`), for validation: ARB_FN_EXP y[i] = exp(x[i]) (table-driven,
 * Tang's method; |x| < 700), ARB_FN_EXPM1 y[i] = exp(x[i]) - 1, ARB_FN_HH_RATES y[6 i .. 6 i + 5]
 * = alpha_m, beta_m, alpha_h, beta_h, alpha_n, beta_n (1/ms) at V = x[i] mV, as the FP64
 * kernels compute them. The paper has no counterpart. Errors via arb_last_error(NULL). */
enum { ARB_FN_EXP = 0, ARB_FN_EXPM1 = 1, ARB_FN_HH_RATES = 2 };
arb_status arb_math_eval(int32_t fn, int64_t n, const double* x, double* y, void* stream);

/* The tabulated HH gate update that the streamed FP64 kernel uses for steps of fixed length dt
 * (ms): host-only, for validation. The exact update of a gate at frozen V (Sec. "Model":
 * channel states advanced with the new voltage) is x' = x_inf + (x - x_inf) e with
 * x_inf = alpha/(alpha + beta) and e = exp(-dt (alpha + beta)); these six functions of V (for m,
 * h and n: m_inf, e_m, h_inf, e_h, n_inf, e_n) are cubic on each interval
 * [v_lo + i/per_mv, v_lo + (i+1)/per_mv), i < n_intervals: coef[24 i + 4 q + k] is the
 * coefficient of s^k of function q, s = (V - v_lo) per_mv - i. Outside the range the kernel
 * evaluates the rates directly. With coef = NULL only the three sizes are returned; cap counts
 * doubles, and a non-NULL coef with cap < 24 n_intervals returns ARB_E_ARG and writes nothing.
 * dt must be finite and > 0 (else ARB_E_ARG). Messages via arb_last_error(NULL). */
arb_status arb_hh_gate_table(double dt, double* coef, int64_t cap, int64_t* n_intervals, double* v_lo,
                             double* per_mv);

/* Debug builds (libarb_b300_debug.so, compiled with ARB_DEBUG): every index read from an index
 * array on the device (parent hand-over stacks and mailbox slots, compact mechanism slots,
 * detector and probe slots, synapse owners, spike positions) is checked against its range; a
 * value outside it is replaced by 0 and reported by arb_advance as ARB_E_STATE ("debug check").
 * Every workspace region is followed by 256 guard bytes, written at arb_bind_workspace and
 * compared after every arb_advance and by arb_check_canaries, which returns ARB_E_STATE naming
 * the region whose guard was overwritten (ARB_OK if all are intact; in release builds ARB_OK with
 * the message that there are no guard words). arb_debug_build returns 1 in a debug build. */
arb_status arb_check_canaries(arb_sim* sim);
int32_t arb_debug_build(void);

/* Where a named array of the plan lies in the workspace (byte offset from the bound base, and
 * its size), valid after arb_create: e.g. "V" (voltages, tile order), "det_slot", "pslot". Host
 * only; ARB_E_ARG for an unknown name. In debug builds the region's 256 guard bytes start at the
 * next multiple of 256 after offset + bytes. */
arb_status arb_workspace_region(const arb_sim* sim, const char* name, int64_t* offset, int64_t* bytes);

/* The compiled variants of the streamed epoch kernel (arb_params.kernel_variant): returns their
 * number; for v < cap, warps[v] = warps per SM, fwd_rows[v] and back_rows[v] = rows each warp
 * keeps in flight in the forward elimination and the back substitution. Arrays may be NULL. */
int32_t arb_kernel_variants(int32_t cap, int32_t* warps, int32_t* fwd_rows, int32_t* back_rows);

/* Message of the last failing call on this handle; with NULL, of the last failing call on
 * this thread that has no handle (arb_create, arb_solve_trees_noalloc, arb_math_eval). */
const char* arb_last_error(const arb_sim* sim);

/* Tree solve that allocates no memory. The paper has no counterpart to this entry point; it
 * serves callers that cannot call cudaMalloc where they need a solve: code that runs while a
 * stream is being captured into a CUDA graph (an allocation would break the capture), host
 * callbacks, or runtimes whose device memory pool is fixed up front.
 *
 * For each of n_cells cells it solves a symmetric linear system whose graph is the cell's tree
 * (the kind of system one implicit Euler step of a cable produces): diagonal d[i],
 * off-diagonal a[i] at (i, parent(i)) and (parent(i), i), right-hand side b[i], solution x[i],
 * by elimination from the leaves and back substitution. All arrays are caller-owned DEVICE
 * memory, in the layout of arb_model: cv_offset [n_cells+1], parent [n_cv] cell-local, and
 * d, a, b, x [n_cv] (a of a cell's first CV unused).
 *  - cv_offset must be a CSR over the CVs: cv_offset[0] = 0, never decreasing,
 *    cv_offset[n_cells] = n_cv. If it is not, every x[i] is set to NaN (the check runs on the
 *    device, so the call still returns ARB_OK).
 *  - parent of a cell's first CV is -1, otherwise 0 <= parent[i] < i; a cell that breaks this
 *    gets NaN over its own x, and the other cells are solved normally.
 * The launches go on `stream` (cudaStream_t, 0 = legacy default) and are asynchronous.
 *
 * Scratch: a fixed array of 262,144 CVs x 16 bytes (4 MiB) plus a status word in the library's
 * device memory, which every GPU that loads the library holds until the process exits. Larger
 * n_cv returns ARB_E_ARG (message via arb_last_error(NULL)). The first call on a device looks up
 * the arrays' device addresses (cudaGetSymbolAddress) for that device and keeps them; make that
 * first call before any stream capture, and do not call cudaDeviceReset on that device
 * afterwards (the kept addresses would belong to the destroyed context). Every call on a device
 * reuses the same arrays: calls on one device whose kernels may overlap (different streams, or
 * different host threads) race on them and must be serialised by the caller; calls on
 * different devices use different copies and do not interfere. Nothing from an earlier call
 * is read: the status word is cleared by each call and the scratch rows are written before
 * they are read. */
arb_status arb_solve_trees_noalloc(int32_t n_cells, int64_t n_cv, const int64_t* cv_offset,
                                   const int32_t* parent, const double* d, const double* a,
                                   const double* b, double* x, void* stream);

#ifdef __cplusplus
}
#endif
#endif
