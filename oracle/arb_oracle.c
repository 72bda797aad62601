/*
 * ORACLE -- plain FP64 CPU reference of the cable-equation time stepper.
 * TEST INFRASTRUCTURE ONLY: it is called by tests/, by the smoke check and by the CPU
 * baseline leg of bench.py. It shares no code, header or constant table with the CUDA
 * path and nothing in the product calls it.
 *
 * What it computes (arXiv 1901.07454, Sec. "Model"):
 *  - the vertex-centred finite-volume semi-discretisation of the cable equation, Eq.
 *    (discrete-v): c_i dV_i/dt = sum_j sigma_ij (V_j - V_i) - I_inj - I_syn - sum S_i g_k (V_i - e_k);
 *    here one control volume (CV) per compartment, node at the compartment centre;
 *  - the operator splitting of Sec. "Model": channel, synapse and injection currents are
 *    evaluated with the states at t, V(t+dt) is computed from Eq. (discrete-v) by the implicit
 *    Euler method, then the channel and synapse states are advanced with the new voltage;
 *  - two readings of the implicit Euler step (both kept, selected per simulation):
 *    IMPLICIT (default): with the states frozen at t every membrane current is g_k (V - E_k),
 *      linear in V, and the step of Eq. (discrete-v) is fully implicit:
 *        (c_i/dt + g_i) V'_i + sum_j sigma_ij (V'_i - V'_j) = (c_i/dt) V_i + sum_k g_k E_k + I_inj;
 *    EXPLICIT: the linear system printed in Sec. "Model", membrane current taken at V(t):
 *        (c_i/dt) V'_i + sum_j sigma_ij V'_i - sum_j sigma_ij V'_j = -I_i^memb + (c_i/dt) V_i;
 *      it diverges on the ring and batched workloads (tiny compartments, dt*g/c > 2);
 *    either system is solved every step by Gaussian elimination in Hines order (parent index <
 *    child index), i.e. the Thomas algorithm extended to trees (Sec. "Model", Hines 1984);
 *  - spike events change the synapse state at the start of a step (Sec. "Model");
 *  - a spike is emitted when the detector voltage crosses a fixed threshold (Sec. "Model");
 *  - cells advance independently within an epoch no longer than the minimum delay; spikes
 *    of an epoch are turned into events through the connection table at its end
 *    (Sec. "Implementation", "Simulation workflow").
 * Mechanisms (the paper names them but prints no equations; the readings used):
 *  - Hodgkin-Huxley in the classic squid-axon form (6.3 degC, no temperature factor):
 *      alpha_m = exprelr(-(V+40)/10), beta_m = 4 exp(-(V+65)/18),
 *      alpha_h = 0.07 exp(-(V+65)/20), beta_h = 1/(1+exp(-(V+35)/10)),
 *      alpha_n = 0.1 exprelr(-(V+55)/10), beta_n = 0.125 exp(-(V+65)/80),
 *      exprelr(x) = x/(e^x-1); E_Na = 50, E_K = -77, E_L = -54.3 mV;
 *    gates advanced by the exact solution of dx/dt = alpha - (alpha+beta) x at frozen V.
 *  - passive: I = g (V - e). Exponential synapse: dg/dt = -g/tau, I = g (V - e), event: g += w.
 *  - current clamp: amp (nA, depolarising) while t_on <= t_k < t_on + dur.
 * Readings where the paper is silent: events at t_e are applied at the start of step
 * ceil(t_e/dt); the spike time is the linear interpolation of the upward crossing inside the
 * step; t_k = k*dt is formed as a product, never accumulated.
 * Dry run (optional; Sec. "Scalability": one rank runs its cells and mimics a large cluster by
 * generating proxy spikes for the cells of the other ranks): with R virtual ranks the model's
 * n cells are those of rank 0 of a network of R*n cells in which rank r holds copies of them
 * (gids r*n .. r*n+n-1); connection sources are global gids in [0, R*n). Every spike of local
 * cell g at t stands for the R spikes of gids g + r*n at t, and each of them is walked against
 * the connections of its gid.
 * Exact event times (optional): as Sec. "Model" describes, the time step is shortened so that
 * every synapse update falls at the start of an integration step: a step whose interval holds
 * events at t_e > t_k is cut at each distinct t_e, each piece is an integration step of its own
 * length (implicit voltage step, gate and synapse updates, clamp sampled at its start, threshold
 * crossing interpolated inside it), and the events at t_e are applied between the pieces.
 *
 * Units: mV, ms, um, nF, uS, nA (nF/ms = uS, uS*mV = nA).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_ENA 50.0
#define ORC_EK (-77.0)
#define ORC_EL (-54.3)

typedef struct {
    int32_t n_cells;
    const int64_t* cv_offset;
    const int32_t* parent;
    const double* length_um;
    const double* radius_um;
    const double* cm;
    const double* Ra;
    int64_t n_hh;
    const int64_t* hh_cv;
    const double* gnabar;
    const double* gkbar;
    const double* gl;
    int64_t n_pas;
    const int64_t* pas_cv;
    const double* g_pas;
    const double* e_pas;
    int64_t n_syn;
    const int64_t* syn_cv;
    const double* syn_tau;
    const double* syn_e;
    int64_t n_stim;
    const int64_t* stim_cv;
    const double* stim_t_on;
    const double* stim_dur;
    const double* stim_amp;
    const int64_t* detector_cv;
    double threshold;
    int64_t n_conn;
    const int32_t* conn_src;
    const int64_t* conn_dst_syn;
    const double* conn_delay;
    const double* conn_weight;
} orc_model;

/* ------------------------------------------------------------------------------------ */
/* Discretisation: per-CV membrane area, capacitance and axial conductance to the parent. */

/* Each CV is a cylinder of length h and radius r. Lateral area 2*pi*r*h um^2,
 * capacitance c = cm * area * 1e-5 nF. The axial conductance between a CV and its parent
 * is the reciprocal of the resistance from centre to centre: two half cylinders in series,
 * R_half = Ra * (h/2) / (pi r^2) Ohm*cm*um/um^2 = Ra*h/(200 pi r^2) MOhm. */
void orc_cv_geometry(const orc_model* m, double* area, double* cap, double* sigma) {
    for (int32_t c = 0; c < m->n_cells; ++c) {
        int64_t off = m->cv_offset[c], n = m->cv_offset[c + 1] - off;
        for (int64_t i = 0; i < n; ++i) {
            int64_t g = off + i;
            double h = m->length_um[g], r = m->radius_um[g];
            area[g] = 2.0 * ORC_PI * r * h;
            cap[g] = m->cm[g] * area[g] * 1e-5;
            if (m->parent[g] < 0) {
                sigma[g] = 0.0;
            } else {
                int64_t p = off + m->parent[g];
                double rh_i = m->Ra[g] * h / (200.0 * ORC_PI * r * r);
                double rh_p = m->Ra[p] * m->length_um[p] /
                              (200.0 * ORC_PI * m->radius_um[p] * m->radius_um[p]);
                sigma[g] = 1.0 / (rh_i + rh_p);
            }
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Hines solve of one symmetric tree system (Sec. "Model", implicit Euler system).
 * Matrix: diagonal d[i]; off-diagonal a[i] at (i, parent[i]) and (parent[i], i).
 * parent[i] < i, parent[0] = -1. Elimination from the leaves to the root, then back
 * substitution from the root to the leaves. Works on copies; returns 0 on success. */
int orc_hines_solve(int64_t n, const int32_t* parent, const double* d_in, const double* a,
                    const double* b_in, double* x) {
    double* d = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double* b = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
    if (!d || !b) { free(d); free(b); return -1; }
    memcpy(d, d_in, sizeof(double) * (size_t)n);
    memcpy(b, b_in, sizeof(double) * (size_t)n);
    for (int64_t i = n - 1; i >= 1; --i) {
        int64_t p = parent[i];
        double f = a[i] / d[i];
        d[p] -= f * a[i];
        b[p] -= f * b[i];
    }
    x[0] = b[0] / d[0];
    for (int64_t i = 1; i < n; ++i) x[i] = (b[i] - a[i] * x[parent[i]]) / d[i];
    free(d);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Hodgkin-Huxley rate functions (1/ms), classic form. */

double orc_exprelr(double x) { return x == 0.0 ? 1.0 : x / expm1(x); }

void orc_hh_rates(double v, double* r) {
    r[0] = orc_exprelr(-(v + 40.0) / 10.0);            /* alpha_m */
    r[1] = 4.0 * exp(-(v + 65.0) / 18.0);               /* beta_m  */
    r[2] = 0.07 * exp(-(v + 65.0) / 20.0);              /* alpha_h */
    r[3] = 1.0 / (1.0 + exp(-(v + 35.0) / 10.0));       /* beta_h  */
    r[4] = 0.1 * orc_exprelr(-(v + 55.0) / 10.0);       /* alpha_n */
    r[5] = 0.125 * exp(-(v + 65.0) / 80.0);             /* beta_n  */
}

/* Exact update of dx/dt = alpha - (alpha+beta) x over dt at frozen V. */
static double gate_step(double x, double alpha, double beta, double dt) {
    double s = alpha + beta;
    double xinf = alpha / s;
    return xinf + (x - xinf) * exp(-dt * s);
}

/* ------------------------------------------------------------------------------------ */
/* Simulation state. */

typedef struct {
    double t;       /* event time (ms) */
    double w;       /* weight (uS) */
    int64_t syn;    /* global synapse index */
    int64_t step;   /* step at whose start it is applied: ceil(t/dt) */
    int32_t src;    /* source gid, -1 for external events */
    int64_t idx;    /* connection index, or enqueue index of an external event */
} orc_event;

typedef struct {
    orc_event* ev;
    int64_t n, cap, head;
} orc_queue;

typedef struct {
    int32_t gid;
    double t;
} orc_spike;

typedef struct {
    orc_model m;
    double dt;
    int explicit_current;    /* 1: membrane current at V(t) on the right-hand side */
    int exact_events;        /* 1: steps are cut at event times (events in step floor(t_e/dt)) */
    int64_t epoch_steps;
    int nthreads;
    int64_t dry_ranks;       /* virtual ranks of the dry run (1: a plain run) */
    int64_t k;               /* steps taken */
    int64_t n_cv;
    double *area, *cap, *sigma;
    double *V;
    double *hh_m, *hh_h, *hh_n, *hh_gna, *hh_gk, *hh_gl;
    double *pas_g;
    double *syn_g;
    /* per-cell mechanism lists (CSR over cells) */
    int64_t *hh_ptr, *hh_list, *pas_ptr, *pas_list, *syn_ptr, *syn_list, *st_ptr, *st_list;
    int64_t* syn_cell;
    /* connections CSR by source gid, ascending connection index */
    int64_t *out_ptr, *out_list;
    orc_queue* q;            /* per cell */
    int64_t n_ext;           /* external events enqueued so far */
    /* spikes */
    orc_spike* spikes;
    int64_t n_spikes, cap_spikes;
    orc_spike** cell_spk;    /* per-cell scratch for one epoch */
    int64_t* cell_nspk;
    int64_t* cell_capspk;
    /* delivered-event record */
    int record_delivered;
    orc_event** cell_deliv;
    int64_t* cell_ndeliv;
    int64_t* cell_capdeliv;
    /* probes */
    int64_t n_probe;
    int64_t* probe_cv;
    int64_t *probe_ptr, *probe_list;   /* probes grouped by cell */
    double* probe_trace;
    int64_t probe_k0, probe_max;
    int error;
} orc_sim;

static void* xmalloc(size_t n) { return malloc(n ? n : 1); }
static void* xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

static void build_csr(int32_t n_cells, int64_t n_items, const int64_t* item_cv, const int64_t* cv_offset,
                      int64_t** ptr_out, int64_t** list_out) {
    int64_t* ptr = (int64_t*)xcalloc((size_t)n_cells + 1, sizeof(int64_t));
    int64_t* list = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)n_items);
    int64_t* cell = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)n_items);
    for (int64_t i = 0; i < n_items; ++i) {
        /* binary search for the cell that owns the CV */
        int64_t lo = 0, hi = n_cells;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            if (cv_offset[mid] <= item_cv[i]) lo = mid; else hi = mid;
        }
        cell[i] = lo;
        ptr[lo + 1]++;
    }
    for (int32_t c = 0; c < n_cells; ++c) ptr[c + 1] += ptr[c];
    int64_t* fill = (int64_t*)xmalloc(sizeof(int64_t) * ((size_t)n_cells + 1));
    memcpy(fill, ptr, sizeof(int64_t) * ((size_t)n_cells + 1));
    for (int64_t i = 0; i < n_items; ++i) list[fill[cell[i]]++] = i;  /* ascending item index */
    free(fill);
    free(cell);
    *ptr_out = ptr;
    *list_out = list;
}

static int cmp_event(const void* pa, const void* pb) {
    const orc_event* a = (const orc_event*)pa;
    const orc_event* b = (const orc_event*)pb;
    if (a->step != b->step) return a->step < b->step ? -1 : 1;
    if (a->t != b->t) return a->t < b->t ? -1 : 1;
    if (a->src != b->src) return a->src < b->src ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

static int cmp_spike(const void* pa, const void* pb) {
    const orc_spike* a = (const orc_spike*)pa;
    const orc_spike* b = (const orc_spike*)pb;
    if (a->t != b->t) return a->t < b->t ? -1 : 1;
    if (a->gid != b->gid) return a->gid < b->gid ? -1 : 1;
    return 0;
}

static void queue_push(orc_queue* q, const orc_event* e) {
    if (q->n == q->cap) {
        q->cap = q->cap ? 2 * q->cap : 16;
        q->ev = (orc_event*)realloc(q->ev, sizeof(orc_event) * (size_t)q->cap);
    }
    q->ev[q->n++] = *e;
}

/* Sort the not-yet-delivered part of a queue. */
static void queue_sort(orc_queue* q) {
    if (q->head > 0 && q->head == q->n) { q->head = q->n = 0; }
    if (q->n - q->head > 1) qsort(q->ev + q->head, (size_t)(q->n - q->head), sizeof(orc_event), cmp_event);
}

/* Step of an event: fixed-step rule, applied at the start of step ceil(t/dt); exact rule,
 * the step j with j*dt <= t < (j+1)*dt on the grid of products k*dt that the steps use. */
static int64_t event_step(const orc_sim* s, double t) {
    if (!s->exact_events) return (int64_t)ceil(t / s->dt);
    int64_t j = (int64_t)floor(t / s->dt);
    while ((double)(j + 1) * s->dt <= t) ++j;
    while ((double)j * s->dt > t) --j;
    return j;
}

orc_sim* orc_create_dry(const orc_model* m, double dt, int64_t epoch_steps, int nthreads, int64_t dry_ranks) {
    orc_sim* s = (orc_sim*)xcalloc(1, sizeof(orc_sim));
    s->m = *m;
    s->dt = dt;
    s->epoch_steps = epoch_steps;
    s->nthreads = nthreads;
    s->dry_ranks = dry_ranks < 1 ? 1 : dry_ranks;
    int64_t n_cv = m->cv_offset[m->n_cells];
    s->n_cv = n_cv;
    s->area = (double*)xmalloc(sizeof(double) * (size_t)n_cv);
    s->cap = (double*)xmalloc(sizeof(double) * (size_t)n_cv);
    s->sigma = (double*)xmalloc(sizeof(double) * (size_t)n_cv);
    orc_cv_geometry(m, s->area, s->cap, s->sigma);
    /* initial state: V = -65 mV, gates at steady state, synapses closed */
    s->V = (double*)xmalloc(sizeof(double) * (size_t)n_cv);
    for (int64_t i = 0; i < n_cv; ++i) s->V[i] = -65.0;
    s->hh_m = (double*)xmalloc(sizeof(double) * (size_t)m->n_hh);
    s->hh_h = (double*)xmalloc(sizeof(double) * (size_t)m->n_hh);
    s->hh_n = (double*)xmalloc(sizeof(double) * (size_t)m->n_hh);
    s->hh_gna = (double*)xmalloc(sizeof(double) * (size_t)m->n_hh);
    s->hh_gk = (double*)xmalloc(sizeof(double) * (size_t)m->n_hh);
    s->hh_gl = (double*)xmalloc(sizeof(double) * (size_t)m->n_hh);
    double r[6];
    orc_hh_rates(-65.0, r);
    for (int64_t i = 0; i < m->n_hh; ++i) {
        double a = s->area[m->hh_cv[i]];
        s->hh_gna[i] = m->gnabar[i] * a * 1e-2;   /* S/cm^2 * um^2 = 1e-2 uS */
        s->hh_gk[i] = m->gkbar[i] * a * 1e-2;
        s->hh_gl[i] = m->gl[i] * a * 1e-2;
        s->hh_m[i] = r[0] / (r[0] + r[1]);
        s->hh_h[i] = r[2] / (r[2] + r[3]);
        s->hh_n[i] = r[4] / (r[4] + r[5]);
    }
    s->pas_g = (double*)xmalloc(sizeof(double) * (size_t)m->n_pas);
    for (int64_t i = 0; i < m->n_pas; ++i) s->pas_g[i] = m->g_pas[i] * s->area[m->pas_cv[i]] * 1e-2;
    s->syn_g = (double*)xcalloc((size_t)m->n_syn, sizeof(double));
    build_csr(m->n_cells, m->n_hh, m->hh_cv, m->cv_offset, &s->hh_ptr, &s->hh_list);
    build_csr(m->n_cells, m->n_pas, m->pas_cv, m->cv_offset, &s->pas_ptr, &s->pas_list);
    build_csr(m->n_cells, m->n_syn, m->syn_cv, m->cv_offset, &s->syn_ptr, &s->syn_list);
    build_csr(m->n_cells, m->n_stim, m->stim_cv, m->cv_offset, &s->st_ptr, &s->st_list);
    s->syn_cell = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)m->n_syn);
    for (int32_t c = 0; c < m->n_cells; ++c)
        for (int64_t j = s->syn_ptr[c]; j < s->syn_ptr[c + 1]; ++j) s->syn_cell[s->syn_list[j]] = c;
    /* connections grouped by source gid (global: R*n sources in a dry run), ascending
       connection index */
    const int64_t n_src = (int64_t)m->n_cells * s->dry_ranks;
    s->out_ptr = (int64_t*)xcalloc((size_t)n_src + 1, sizeof(int64_t));
    s->out_list = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)m->n_conn);
    for (int64_t i = 0; i < m->n_conn; ++i) s->out_ptr[m->conn_src[i] + 1]++;
    for (int64_t c = 0; c < n_src; ++c) s->out_ptr[c + 1] += s->out_ptr[c];
    {
        int64_t* fill = (int64_t*)xmalloc(sizeof(int64_t) * ((size_t)n_src + 1));
        memcpy(fill, s->out_ptr, sizeof(int64_t) * ((size_t)n_src + 1));
        for (int64_t i = 0; i < m->n_conn; ++i) s->out_list[fill[m->conn_src[i]]++] = i;
        free(fill);
    }
    s->q = (orc_queue*)xcalloc((size_t)m->n_cells, sizeof(orc_queue));
    s->cell_spk = (orc_spike**)xcalloc((size_t)m->n_cells, sizeof(orc_spike*));
    s->cell_nspk = (int64_t*)xcalloc((size_t)m->n_cells, sizeof(int64_t));
    s->cell_capspk = (int64_t*)xcalloc((size_t)m->n_cells, sizeof(int64_t));
    s->cell_deliv = (orc_event**)xcalloc((size_t)m->n_cells, sizeof(orc_event*));
    s->cell_ndeliv = (int64_t*)xcalloc((size_t)m->n_cells, sizeof(int64_t));
    s->cell_capdeliv = (int64_t*)xcalloc((size_t)m->n_cells, sizeof(int64_t));
    return s;
}

orc_sim* orc_create(const orc_model* m, double dt, int64_t epoch_steps, int nthreads) {
    return orc_create_dry(m, dt, epoch_steps, nthreads, 1);
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->area); free(s->cap); free(s->sigma); free(s->V);
    free(s->hh_m); free(s->hh_h); free(s->hh_n); free(s->hh_gna); free(s->hh_gk); free(s->hh_gl);
    free(s->pas_g); free(s->syn_g);
    free(s->hh_ptr); free(s->hh_list); free(s->pas_ptr); free(s->pas_list);
    free(s->syn_ptr); free(s->syn_list); free(s->st_ptr); free(s->st_list); free(s->syn_cell);
    free(s->out_ptr); free(s->out_list);
    for (int32_t c = 0; c < s->m.n_cells; ++c) {
        free(s->q[c].ev); free(s->cell_spk[c]); free(s->cell_deliv[c]);
    }
    free(s->q); free(s->cell_spk); free(s->cell_nspk); free(s->cell_capspk);
    free(s->cell_deliv); free(s->cell_ndeliv); free(s->cell_capdeliv);
    free(s->spikes); free(s->probe_cv); free(s->probe_ptr); free(s->probe_list);
    free(s);
}

void orc_record_delivered(orc_sim* s, int on) { s->record_delivered = on; }
void orc_set_explicit(orc_sim* s, int on) { s->explicit_current = on; }
void orc_set_exact_events(orc_sim* s, int on) { s->exact_events = on; }

/* External events: applied at the start of step ceil(t/dt). Returns -1 if one lies in the past. */
int orc_enqueue(orc_sim* s, int64_t n, const int64_t* syn, const double* t, const double* w) {
    for (int64_t i = 0; i < n; ++i) {
        orc_event e;
        e.t = t[i]; e.w = w[i]; e.syn = syn[i]; e.src = -1; e.idx = s->n_ext++;
        e.step = event_step(s, t[i]);
        if (e.step < s->k || syn[i] < 0 || syn[i] >= s->m.n_syn) return -1;
        queue_push(&s->q[s->syn_cell[syn[i]]], &e);
    }
    for (int32_t c = 0; c < s->m.n_cells; ++c) queue_sort(&s->q[c]);
    return 0;
}

void orc_set_probes(orc_sim* s, int64_t n, const int64_t* cv, double* trace, int64_t max_steps) {
    free(s->probe_cv);
    free(s->probe_ptr);
    free(s->probe_list);
    s->n_probe = n;
    s->probe_cv = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)n);
    memcpy(s->probe_cv, cv, sizeof(int64_t) * (size_t)n);
    build_csr(s->m.n_cells, n, s->probe_cv, s->m.cv_offset, &s->probe_ptr, &s->probe_list);
    s->probe_trace = trace;
    s->probe_k0 = s->k;
    s->probe_max = max_steps;
}

/* Delivers the queued events of cell c that are due: those of earlier steps (late: an error),
 * and those of step k at times up to t_upto (all of step k with the fixed-step rule). */
static void deliver(orc_sim* s, int32_t c, int64_t k, double t_upto) {
    orc_queue* q = &s->q[c];
    while (q->head < q->n) {
        orc_event* e = &q->ev[q->head];
        if (e->step > k || (e->step == k && s->exact_events && e->t > t_upto)) break;
        q->head++;
        if (e->step < k) s->error = 1;          /* late event: cannot happen by construction */
        s->syn_g[e->syn] += e->w;
        if (s->record_delivered) {
            if (s->cell_ndeliv[c] == s->cell_capdeliv[c]) {
                s->cell_capdeliv[c] = s->cell_capdeliv[c] ? 2 * s->cell_capdeliv[c] : 16;
                s->cell_deliv[c] = (orc_event*)realloc(s->cell_deliv[c], sizeof(orc_event) * (size_t)s->cell_capdeliv[c]);
            }
            s->cell_deliv[c][s->cell_ndeliv[c]++] = *e;
        }
    }
}

/* One integration step of cell c from t0 over h (h = dt, or the piece of a step between event
 * times), in the order of the operator splitting. */
static void substep(orc_sim* s, int32_t c, double t0, double h, double* I, double* d, double* a, double* b, double* Vn) {
    const orc_model* m = &s->m;
    const int64_t off = m->cv_offset[c], n = m->cv_offset[c + 1] - off;
    const double t = t0;
    const double dt = h;
    double* V = s->V + off;
    const int32_t* par = m->parent + off;
    /* 2. membrane terms with the states at t_k: conductance g_i (uS) and g_i*E (nA) per CV for
     *    the implicit step, or the outward current I_i (nA) at V(t_k) for the explicit one;
     *    injected current Iinj (nA, depolarising) active at t_k */
    double* G = d;        /* reuse: conductance sums */
    double* GE = a;       /* reuse: sum g*E */
    double* Iinj = Vn;    /* reuse: injected current */
    for (int64_t i = 0; i < n; ++i) { I[i] = 0.0; G[i] = 0.0; GE[i] = 0.0; Iinj[i] = 0.0; }
    for (int64_t j = s->hh_ptr[c]; j < s->hh_ptr[c + 1]; ++j) {
        int64_t h = s->hh_list[j];
        int64_t i = m->hh_cv[h] - off;
        double v = V[i], mm = s->hh_m[h], hh = s->hh_h[h], nn = s->hh_n[h];
        double gna = s->hh_gna[h] * mm * mm * mm * hh;
        double gk = s->hh_gk[h] * nn * nn * nn * nn;
        double gl = s->hh_gl[h];
        I[i] += gna * (v - ORC_ENA) + gk * (v - ORC_EK) + gl * (v - ORC_EL);
        G[i] += gna + gk + gl;
        GE[i] += gna * ORC_ENA + gk * ORC_EK + gl * ORC_EL;
    }
    for (int64_t j = s->pas_ptr[c]; j < s->pas_ptr[c + 1]; ++j) {
        int64_t p = s->pas_list[j];
        int64_t i = m->pas_cv[p] - off;
        I[i] += s->pas_g[p] * (V[i] - m->e_pas[p]);
        G[i] += s->pas_g[p];
        GE[i] += s->pas_g[p] * m->e_pas[p];
    }
    for (int64_t j = s->syn_ptr[c]; j < s->syn_ptr[c + 1]; ++j) {
        int64_t y = s->syn_list[j];
        int64_t i = m->syn_cv[y] - off;
        I[i] += s->syn_g[y] * (V[i] - m->syn_e[y]);
        G[i] += s->syn_g[y];
        GE[i] += s->syn_g[y] * m->syn_e[y];
    }
    for (int64_t j = s->st_ptr[c]; j < s->st_ptr[c + 1]; ++j) {
        int64_t y = s->st_list[j];
        int64_t i = m->stim_cv[y] - off;
        if (m->stim_t_on[y] <= t && t < m->stim_t_on[y] + m->stim_dur[y]) Iinj[i] += m->stim_amp[y];
    }

    /* 3. assemble the implicit Euler system */
    for (int64_t i = 0; i < n; ++i) {
        double cdt = s->cap[off + i] / dt;
        if (s->explicit_current) {
            b[i] = cdt * V[i] - I[i] + Iinj[i];
            d[i] = cdt;
        } else {
            b[i] = cdt * V[i] + GE[i] + Iinj[i];
            d[i] = cdt + G[i];
        }
        a[i] = 0.0;
    }
    for (int64_t i = 1; i < n; ++i) {
        double sg = s->sigma[off + i];
        d[i] += sg;
        d[par[i]] += sg;
        a[i] = -sg;
    }

    /* 4. Hines elimination and back substitution */
    for (int64_t i = n - 1; i >= 1; --i) {
        int64_t p = par[i];
        double f = a[i] / d[i];
        d[p] -= f * a[i];
        b[p] -= f * b[i];
    }
    Vn[0] = b[0] / d[0];
    for (int64_t i = 1; i < n; ++i) Vn[i] = (b[i] - a[i] * Vn[par[i]]) / d[i];

    /* 6 (first half). threshold crossing at the detector, V(t_k) -> V(t_{k+1}) */
    {
        int64_t i = m->detector_cv[c] - off;
        double v0 = V[i], v1 = Vn[i], th = m->threshold;
        if (v0 < th && v1 >= th) {
            if (s->cell_nspk[c] == s->cell_capspk[c]) {
                s->cell_capspk[c] = s->cell_capspk[c] ? 2 * s->cell_capspk[c] : 8;
                s->cell_spk[c] = (orc_spike*)realloc(s->cell_spk[c], sizeof(orc_spike) * (size_t)s->cell_capspk[c]);
            }
            orc_spike sp;
            sp.gid = c;
            sp.t = t + dt * ((th - v0) / (v1 - v0));
            s->cell_spk[c][s->cell_nspk[c]++] = sp;
        }
    }
    for (int64_t i = 0; i < n; ++i) V[i] = Vn[i];

    /* 5. state update with V(t_{k+1}) */
    for (int64_t j = s->hh_ptr[c]; j < s->hh_ptr[c + 1]; ++j) {
        int64_t h = s->hh_list[j];
        double r[6];
        orc_hh_rates(V[m->hh_cv[h] - off], r);
        s->hh_m[h] = gate_step(s->hh_m[h], r[0], r[1], dt);
        s->hh_h[h] = gate_step(s->hh_h[h], r[2], r[3], dt);
        s->hh_n[h] = gate_step(s->hh_n[h], r[4], r[5], dt);
    }
    for (int64_t j = s->syn_ptr[c]; j < s->syn_ptr[c + 1]; ++j) {
        int64_t y = s->syn_list[j];
        s->syn_g[y] *= exp(-dt / m->syn_tau[y]);
    }

}

/* One step t_k -> t_{k+1} of one cell. With exact event times the step is cut at the times of
 * the events that fall inside it (Sec. "Model": the time step is shortened so that every
 * synapse update happens at the start of an integration step); otherwise events are applied at
 * the start of step ceil(t_e/dt). */
static void step_cell(orc_sim* s, int32_t c, int64_t k, double* I, double* d, double* a, double* b, double* Vn) {
    const orc_model* m = &s->m;
    const int64_t off = m->cv_offset[c];
    const double t = (double)k * s->dt;
    deliver(s, c, k, t);
    if (!s->exact_events) {
        substep(s, c, t, s->dt, I, d, a, b, Vn);
    } else {
        const double t_end = (double)(k + 1) * s->dt;
        orc_queue* q = &s->q[c];
        double cur = t;
        for (;;) {
            double next = t_end;
            if (q->head < q->n && q->ev[q->head].step == k && q->ev[q->head].t < t_end) next = q->ev[q->head].t;
            /* an uncut step is a step of dt (not t_end - t_k, which differs in the last bit) */
            const double h = (cur == t && next >= t_end) ? s->dt : next - cur;
            substep(s, c, cur, h, I, d, a, b, Vn);
            if (next >= t_end) break;
            deliver(s, c, k, next);
            cur = next;
        }
    }

    /* probes record V(t_{k+1}) */
    if (s->n_probe > 0 && k >= s->probe_k0 && k - s->probe_k0 < s->probe_max) {
        const double* V = s->V + off;
        double* row = s->probe_trace + (k - s->probe_k0) * s->n_probe;
        for (int64_t j = s->probe_ptr[c]; j < s->probe_ptr[c + 1]; ++j) {
            int64_t p = s->probe_list[j];
            row[p] = V[s->probe_cv[p] - off];
        }
    }
}

/* Advance all cells by n_steps, epoch by epoch (epochs of at most epoch_steps steps). */
int orc_run(orc_sim* s, int64_t n_steps) {
    const orc_model* m = &s->m;
    const int64_t k_end = s->k + n_steps;
    int64_t max_n = 0;
    for (int32_t c = 0; c < m->n_cells; ++c) {
        int64_t n = m->cv_offset[c + 1] - m->cv_offset[c];
        if (n > max_n) max_n = n;
    }
#ifdef _OPENMP
    if (s->nthreads > 0) omp_set_num_threads(s->nthreads);
#endif
    while (s->k < k_end) {
        const int64_t k0 = s->k;
        const int64_t k1 = (k0 + s->epoch_steps < k_end) ? k0 + s->epoch_steps : k_end;
#pragma omp parallel
        {
            double* I = (double*)xmalloc(sizeof(double) * (size_t)max_n);
            double* d = (double*)xmalloc(sizeof(double) * (size_t)max_n);
            double* a = (double*)xmalloc(sizeof(double) * (size_t)max_n);
            double* b = (double*)xmalloc(sizeof(double) * (size_t)max_n);
            double* Vn = (double*)xmalloc(sizeof(double) * (size_t)max_n);
#pragma omp for schedule(dynamic, 4)
            for (int32_t c = 0; c < m->n_cells; ++c)
                for (int64_t k = k0; k < k1; ++k) step_cell(s, c, k, I, d, a, b, Vn);
            free(I); free(d); free(a); free(b); free(Vn);
        }
        s->k = k1;
        /* exchange: spikes of this epoch in (t, gid) order, walked against the connections */
        int64_t nsp = 0;
        for (int32_t c = 0; c < m->n_cells; ++c) nsp += s->cell_nspk[c];
        if (s->n_spikes + nsp > s->cap_spikes) {
            s->cap_spikes = 2 * (s->n_spikes + nsp) + 16;
            s->spikes = (orc_spike*)realloc(s->spikes, sizeof(orc_spike) * (size_t)s->cap_spikes);
        }
        orc_spike* ep = s->spikes + s->n_spikes;
        int64_t w = 0;
        for (int32_t c = 0; c < m->n_cells; ++c) {
            for (int64_t j = 0; j < s->cell_nspk[c]; ++j) ep[w++] = s->cell_spk[c][j];
            s->cell_nspk[c] = 0;
        }
        qsort(ep, (size_t)nsp, sizeof(orc_spike), cmp_spike);
        s->n_spikes += nsp;
        /* the global spike list: each local spike once per (virtual) rank */
        for (int64_t r = 0; r < s->dry_ranks; ++r)
        for (int64_t j = 0; j < nsp; ++j) {
            int32_t src = (int32_t)(ep[j].gid + r * m->n_cells);
            for (int64_t o = s->out_ptr[src]; o < s->out_ptr[src + 1]; ++o) {
                int64_t ci = s->out_list[o];
                orc_event e;
                e.t = ep[j].t + m->conn_delay[ci];
                e.w = m->conn_weight[ci];
                e.syn = m->conn_dst_syn[ci];
                e.src = src;
                e.idx = ci;
                e.step = event_step(s, e.t);
                if (e.step < k1) e.step = k1;    /* never before the next epoch */
                queue_push(&s->q[s->syn_cell[e.syn]], &e);
            }
        }
        for (int32_t c = 0; c < m->n_cells; ++c) queue_sort(&s->q[c]);
    }
    return s->error ? -1 : 0;
}

int64_t orc_steps(const orc_sim* s) { return s->k; }
void orc_get_voltage(const orc_sim* s, double* out) { memcpy(out, s->V, sizeof(double) * (size_t)s->n_cv); }
int64_t orc_num_spikes(const orc_sim* s) { return s->n_spikes; }
void orc_get_spikes(const orc_sim* s, int32_t* gid, double* t) {
    for (int64_t i = 0; i < s->n_spikes; ++i) { gid[i] = s->spikes[i].gid; t[i] = s->spikes[i].t; }
}

/* State: V [n_cv], m h n [n_hh], g [n_syn]. */
void orc_get_state(const orc_sim* s, double* V, double* m, double* h, double* n, double* g) {
    memcpy(V, s->V, sizeof(double) * (size_t)s->n_cv);
    memcpy(m, s->hh_m, sizeof(double) * (size_t)s->m.n_hh);
    memcpy(h, s->hh_h, sizeof(double) * (size_t)s->m.n_hh);
    memcpy(n, s->hh_n, sizeof(double) * (size_t)s->m.n_hh);
    memcpy(g, s->syn_g, sizeof(double) * (size_t)s->m.n_syn);
}
void orc_set_state(orc_sim* s, const double* V, const double* m, const double* h, const double* n, const double* g) {
    memcpy(s->V, V, sizeof(double) * (size_t)s->n_cv);
    memcpy(s->hh_m, m, sizeof(double) * (size_t)s->m.n_hh);
    memcpy(s->hh_h, h, sizeof(double) * (size_t)s->m.n_hh);
    memcpy(s->hh_n, n, sizeof(double) * (size_t)s->m.n_hh);
    memcpy(s->syn_g, g, sizeof(double) * (size_t)s->m.n_syn);
}

/* Delivered events, grouped by cell, in delivery order: (syn, t, w, step, src, idx). */
int64_t orc_num_delivered(const orc_sim* s) {
    int64_t n = 0;
    for (int32_t c = 0; c < s->m.n_cells; ++c) n += s->cell_ndeliv[c];
    return n;
}
void orc_get_delivered(const orc_sim* s, int64_t* syn, double* t, double* w, int64_t* step, int32_t* src, int64_t* idx) {
    int64_t o = 0;
    for (int32_t c = 0; c < s->m.n_cells; ++c)
        for (int64_t j = 0; j < s->cell_ndeliv[c]; ++j, ++o) {
            const orc_event* e = &s->cell_deliv[c][j];
            syn[o] = e->syn; t[o] = e->t; w[o] = e->w; step[o] = e->step; src[o] = e->src; idx[o] = e->idx;
        }
}

/* ------------------------------------------------------------------------------------ */
/* Discrete adjoint of the implicit step (gradient of a voltage loss w.r.t. the channel
 * densities and the membrane capacitance).
 *
 * The forward map is the implicit reading of the step above, per cell:
 *   A(y^k) V^{k+1} = (C/dt) V^k + M(y^k) + Iinj(t_k),
 *   A(y) = diag(C/dt + G(y)) + axial Laplacian (symmetric),
 *   y^{k+1} = Phi(y^k, V^{k+1})  (exact gate update at frozen V^{k+1}),
 * with G = sum of channel conductances and M = sum g*E. The loss is
 *   L = scale * sum_{k=1..K} sum_obs (V_obs^k - target_obs^k)^2.
 * Reverse sweep, k = K-1 .. 0, with lam the solve result of step k+1 (zero for k = K-1) and
 * ybar the adjoint of the gates y^{k+1}:
 *   Vbar = (C/dt) lam + dL/dV^{k+1} + sum_gates dPhi/dV(y^k, V^{k+1}) ybar
 *   lam  = A(y^k)^{-1} Vbar                   (the same tree solve: A is symmetric)
 *   dL/dC_i    += lam_i (V_i^k - V_i^{k+1}) / dt
 *   dL/dg_chan += lam_i (E_chan - V_i^{k+1}) * (open fraction of the channel at y^k)
 *   ybar       <- exp(-dt (alpha+beta)(V^{k+1})) ybar + dG/dy^T (-lam V^{k+1}) + dM/dy^T lam
 * Densities enter as g = gbar * area * 1e-2 and C = cm * area * 1e-5. The initial state is
 * taken as given (no dependence on the parameters). Models with synapses are not supported.
 * The reverse sweep needs y^k and V^{k+1}: this reference keeps every state of the run. */

/* d/dx of x/(e^x - 1). For |x| < 0.1 the derivative of its Bernoulli series,
 * sum_n B_n x^n / n!, up to x^7 (the first omitted term is below 3e-16 there); elsewhere the
 * closed form (e^x - 1 - x e^x) / (e^x - 1)^2, whose cancellation costs ~eps/|x|. */
double orc_exprelr_deriv(double x) {
    if (fabs(x) < 0.1) {
        double x2 = x * x;
        return -0.5 + x * (1.0 / 6.0 + x2 * (-1.0 / 180.0 + x2 * (1.0 / 5040.0 - x2 / 151200.0)));
    }
    double em = expm1(x);
    return (em - x * (em + 1.0)) / (em * em);
}

/* Derivatives of the six rates of orc_hh_rates w.r.t. V (1/(ms mV)). */
void orc_hh_rate_derivs(double v, double* dr) {
    double r[6];
    orc_hh_rates(v, r);
    dr[0] = -0.1 * orc_exprelr_deriv(-(v + 40.0) / 10.0);
    dr[1] = -r[1] / 18.0;
    dr[2] = -r[2] / 20.0;
    dr[3] = r[3] * (1.0 - r[3]) / 10.0;
    dr[4] = -0.01 * orc_exprelr_deriv(-(v + 55.0) / 10.0);
    dr[5] = -r[5] / 80.0;
}

/* d Phi / dV for one gate: Phi = xinf + (x - xinf) exp(-dt s), s = alpha + beta. */
static double gate_dv(double x, double al, double be, double dal, double dbe, double dt) {
    double s = al + be, ds = dal + dbe;
    double xinf = al / s;
    double dxinf = (dal * s - al * ds) / (s * s);
    double e = exp(-dt * s);
    return dxinf * (1.0 - e) + (x - xinf) * e * (-dt * ds);
}

/* Runs n_steps from the simulation's current state and time without changing them.
 * target [n_steps][n_obs]; group_of_cv [n_cv] (-1: no parameter group); grad [n_groups][4]
 * = dL/d(gnabar, gkbar, gl, cm) summed over the CVs of each group. Returns 0, or -2 for a
 * model with synapses. */
int orc_adjoint(orc_sim* s, int64_t n_steps, int64_t n_obs, const int64_t* obs_cv, const double* target,
                double loss_scale, const int32_t* group_of_cv, int32_t n_groups, double* grad, double* loss) {
    const orc_model* m = &s->m;
    if (m->n_syn > 0) return -2;
    const double dt = s->dt;
    const int64_t K = n_steps, k0 = s->k, ncv = s->n_cv;
    int64_t* obs_ptr = NULL;
    int64_t* obs_list = NULL;
    build_csr(m->n_cells, n_obs, obs_cv, m->cv_offset, &obs_ptr, &obs_list);
    /* per-CV and per-instance gradient accumulators */
    double* g_cm = (double*)xcalloc((size_t)ncv, sizeof(double));
    double* g_na = (double*)xcalloc((size_t)m->n_hh, sizeof(double));
    double* g_k = (double*)xcalloc((size_t)m->n_hh, sizeof(double));
    double* g_l = (double*)xcalloc((size_t)m->n_hh, sizeof(double));
    double* cell_loss = (double*)xcalloc((size_t)m->n_cells, sizeof(double));
#ifdef _OPENMP
    if (s->nthreads > 0) omp_set_num_threads(s->nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t c = 0; c < m->n_cells; ++c) {
        const int64_t off = m->cv_offset[c], n = m->cv_offset[c + 1] - off;
        const int32_t* par = m->parent + off;
        const int64_t h0 = s->hh_ptr[c], nh = s->hh_ptr[c + 1] - h0;
        double* Vs = (double*)xmalloc(sizeof(double) * (size_t)((K + 1) * n));       /* V^k, k = 0..K */
        double* Ys = (double*)xmalloc(sizeof(double) * (size_t)((K + 1) * nh * 3));  /* (m,h,n)^k */
        double* G = (double*)xmalloc(sizeof(double) * (size_t)n);
        double* GE = (double*)xmalloc(sizeof(double) * (size_t)n);
        double* d = (double*)xmalloc(sizeof(double) * (size_t)n);
        double* a = (double*)xmalloc(sizeof(double) * (size_t)n);
        double* b = (double*)xmalloc(sizeof(double) * (size_t)n);
        double* lam = (double*)xcalloc((size_t)n, sizeof(double));
        double* ybar = (double*)xcalloc((size_t)(nh * 3), sizeof(double));
        for (int64_t i = 0; i < n; ++i) Vs[i] = s->V[off + i];
        for (int64_t j = 0; j < nh; ++j) {
            int64_t hh = s->hh_list[h0 + j];
            Ys[3 * j + 0] = s->hh_m[hh];
            Ys[3 * j + 1] = s->hh_h[hh];
            Ys[3 * j + 2] = s->hh_n[hh];
        }
        /* assemble A(y^k) into d, a and the membrane terms into G, GE */
        #define ORC_ASSEMBLE(k_)                                                            \
            do {                                                                            \
                const double* Y_ = Ys + (size_t)(k_) * (size_t)nh * 3;                      \
                for (int64_t i = 0; i < n; ++i) { G[i] = 0.0; GE[i] = 0.0; a[i] = 0.0; }    \
                for (int64_t j = 0; j < nh; ++j) {                                          \
                    int64_t hh = s->hh_list[h0 + j];                                        \
                    int64_t i = m->hh_cv[hh] - off;                                         \
                    double mm = Y_[3 * j], hv = Y_[3 * j + 1], nv = Y_[3 * j + 2];          \
                    double gna = s->hh_gna[hh] * mm * mm * mm * hv;                         \
                    double gk = s->hh_gk[hh] * nv * nv * nv * nv;                           \
                    G[i] += gna + gk + s->hh_gl[hh];                                        \
                    GE[i] += gna * ORC_ENA + gk * ORC_EK + s->hh_gl[hh] * ORC_EL;           \
                }                                                                           \
                for (int64_t j = s->pas_ptr[c]; j < s->pas_ptr[c + 1]; ++j) {               \
                    int64_t p = s->pas_list[j];                                             \
                    int64_t i = m->pas_cv[p] - off;                                         \
                    G[i] += s->pas_g[p];                                                    \
                    GE[i] += s->pas_g[p] * m->e_pas[p];                                     \
                }                                                                           \
                for (int64_t i = 0; i < n; ++i) d[i] = s->cap[off + i] / dt + G[i];         \
                for (int64_t i = 1; i < n; ++i) {                                           \
                    double sg = s->sigma[off + i];                                          \
                    d[i] += sg;                                                             \
                    d[par[i]] += sg;                                                        \
                    a[i] = -sg;                                                             \
                }                                                                           \
            } while (0)
        /* forward, keeping every state */
        for (int64_t k = 0; k < K; ++k) {
            const double* V = Vs + (size_t)k * (size_t)n;
            double* Vn = Vs + (size_t)(k + 1) * (size_t)n;
            const double t = (double)(k0 + k) * dt;
            ORC_ASSEMBLE(k);
            for (int64_t i = 0; i < n; ++i) b[i] = s->cap[off + i] / dt * V[i] + GE[i];
            for (int64_t j = s->st_ptr[c]; j < s->st_ptr[c + 1]; ++j) {
                int64_t y = s->st_list[j];
                if (m->stim_t_on[y] <= t && t < m->stim_t_on[y] + m->stim_dur[y]) b[m->stim_cv[y] - off] += m->stim_amp[y];
            }
            orc_hines_solve(n, par, d, a, b, Vn);
            const double* Y = Ys + (size_t)k * (size_t)nh * 3;
            double* Yn = Ys + (size_t)(k + 1) * (size_t)nh * 3;
            for (int64_t j = 0; j < nh; ++j) {
                double r[6];
                orc_hh_rates(Vn[m->hh_cv[s->hh_list[h0 + j]] - off], r);
                Yn[3 * j + 0] = gate_step(Y[3 * j + 0], r[0], r[1], dt);
                Yn[3 * j + 1] = gate_step(Y[3 * j + 1], r[2], r[3], dt);
                Yn[3 * j + 2] = gate_step(Y[3 * j + 2], r[4], r[5], dt);
            }
            for (int64_t q = obs_ptr[c]; q < obs_ptr[c + 1]; ++q) {
                int64_t o = obs_list[q];
                double e = Vn[obs_cv[o] - off] - target[k * n_obs + o];
                cell_loss[c] += loss_scale * e * e;
            }
        }
        /* reverse sweep */
        for (int64_t k = K - 1; k >= 0; --k) {
            const double* V = Vs + (size_t)k * (size_t)n;
            const double* Vn = Vs + (size_t)(k + 1) * (size_t)n;
            const double* Y = Ys + (size_t)k * (size_t)nh * 3;
            /* Vbar: from the next step's right-hand side (C/dt) V^{k+1}, the loss at k+1 and
             * the gate update y^{k+1} = Phi(y^k, V^{k+1}) */
            for (int64_t i = 0; i < n; ++i) b[i] = s->cap[off + i] / dt * lam[i];
            for (int64_t q = obs_ptr[c]; q < obs_ptr[c + 1]; ++q) {
                int64_t o = obs_list[q];
                int64_t i = obs_cv[o] - off;
                b[i] += 2.0 * loss_scale * (Vn[i] - target[k * n_obs + o]);
            }
            for (int64_t j = 0; j < nh; ++j) {
                int64_t i = m->hh_cv[s->hh_list[h0 + j]] - off;
                double r[6], dr[6];
                orc_hh_rates(Vn[i], r);
                orc_hh_rate_derivs(Vn[i], dr);
                b[i] += gate_dv(Y[3 * j + 0], r[0], r[1], dr[0], dr[1], dt) * ybar[3 * j + 0]
                      + gate_dv(Y[3 * j + 1], r[2], r[3], dr[2], dr[3], dt) * ybar[3 * j + 1]
                      + gate_dv(Y[3 * j + 2], r[4], r[5], dr[4], dr[5], dt) * ybar[3 * j + 2];
            }
            /* lam = A(y^k)^{-1} Vbar */
            ORC_ASSEMBLE(k);
            orc_hines_solve(n, par, d, a, b, lam);
            /* parameter gradients and the gate adjoint of y^k */
            for (int64_t i = 0; i < n; ++i)
                g_cm[off + i] += lam[i] * (V[i] - Vn[i]) / dt * s->area[off + i] * 1e-5;
            for (int64_t j = 0; j < nh; ++j) {
                int64_t hh = s->hh_list[h0 + j];
                int64_t i = m->hh_cv[hh] - off;
                double mm = Y[3 * j], hv = Y[3 * j + 1], nv = Y[3 * j + 2];
                double lna = lam[i] * (ORC_ENA - Vn[i]), lk = lam[i] * (ORC_EK - Vn[i]), ll = lam[i] * (ORC_EL - Vn[i]);
                double sc = s->area[off + i] * 1e-2;
                g_na[hh] += mm * mm * mm * hv * lna * sc;
                g_k[hh] += nv * nv * nv * nv * lk * sc;
                g_l[hh] += ll * sc;
                double r[6];
                orc_hh_rates(Vn[i], r);
                ybar[3 * j + 0] = exp(-dt * (r[0] + r[1])) * ybar[3 * j + 0] + s->hh_gna[hh] * 3.0 * mm * mm * hv * lna;
                ybar[3 * j + 1] = exp(-dt * (r[2] + r[3])) * ybar[3 * j + 1] + s->hh_gna[hh] * mm * mm * mm * lna;
                ybar[3 * j + 2] = exp(-dt * (r[4] + r[5])) * ybar[3 * j + 2] + s->hh_gk[hh] * 4.0 * nv * nv * nv * lk;
            }
        }
        #undef ORC_ASSEMBLE
        free(Vs); free(Ys); free(G); free(GE); free(d); free(a); free(b); free(lam); free(ybar);
    }
    /* group sums in ascending CV / instance order */
    for (int64_t q = 0; q < (int64_t)n_groups * 4; ++q) grad[q] = 0.0;
    for (int64_t i = 0; i < ncv; ++i)
        if (group_of_cv[i] >= 0) grad[4 * group_of_cv[i] + 3] += g_cm[i];
    for (int64_t hh = 0; hh < m->n_hh; ++hh) {
        int32_t gr = group_of_cv[m->hh_cv[hh]];
        if (gr < 0) continue;
        grad[4 * gr + 0] += g_na[hh];
        grad[4 * gr + 1] += g_k[hh];
        grad[4 * gr + 2] += g_l[hh];
    }
    double L = 0.0;
    for (int32_t c = 0; c < m->n_cells; ++c) L += cell_loss[c];
    *loss = L;
    free(g_cm); free(g_na); free(g_k); free(g_l); free(cell_loss); free(obs_ptr); free(obs_list);
    return 0;
}
