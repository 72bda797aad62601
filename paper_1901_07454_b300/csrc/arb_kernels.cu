// sm_103a kernels of the batched cable-equation stepper.
//
// One epoch (Sec. "Implementation", "Simulation workflow": cells advance independently for
// an interval no longer than the minimum delay) is this fixed sequence of launches:
//   k_epoch_begin -> k_ev_walk<count> -> k_ev_scan -> k_ev_walk<scatter> -> k_ev_sort   (event lists)
//   arb_stream_kernel (streamed packs) or arb_epoch_kernel (tile packs)   (all time steps)
//   k_spike_expand -> k_epoch_end                                         (spike exchange)
// Per-epoch values live in the device control block, so the sequence is captured once (as
// three CUDA graphs, timed between them) and replayed for every epoch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "arb_hh.cuh"
#include "arb_internal.h"

namespace arbk {


// ------------------------------------------------------------------------------------------
// The epoch kernel: a persistent grid; each warp takes packs from a work counter and runs
// every time step of the epoch for the pack's cells.
//
// Per pack, S holds for every entry (row j, lane l) the right-hand side of the implicit
// Euler system already divided by the eliminated pivot d'_i; after the forward sweep it holds
// u_i = b'_i / d'_i. The matrix of Sec. "Model" does not depend on the state when dt is fixed
// and the membrane current sits on the right-hand side, so the host factorised it once:
//   forward (leaves to root):  u_i = S_i - sum_children a'_c u_c
//   backward (root to leaves): V_i = u_i - e_i V_parent(i)
//   next right-hand side:      S_i = alpha'_i V_i + beta'_i - (mechanism currents) / d'_i
// which is the elimination and back substitution of the Hines matrix (Sec. "Model") with
// one FP64 FMA per entry in each of the three lines.

// Pointers of one pack's working set: in shared memory for packs whose tile fits (the
// common case), else in global memory (cells whose longest root-to-leaf path is too long).
template <class MT>
struct Work {
    double* R;     // implicit scheme: diagonal, then e = sigma / d' (one per entry)
    double* S;     // right-hand side, then u = b' / d' (one per entry)
    double* Vc;    // voltages that are read: on-chip slots (shared) or every tile slot (global)
    MT* g;         // synapse conductances
    MT* m;         // HH gates
    MT* h;
    MT* n;
};

// Synapses: decay (state update of the previous step), events due now, then their terms of
// the step's linear system. Implicit scheme: conductance g on the diagonal and g*e on the
// right-hand side. Explicit scheme: the current g (V - e) on the right-hand side, scaled by
// 1/d' like the rest of the factorised system.
template <class MT, bool kSmem, bool kImp>
__device__ __forceinline__ void syn_pass(const DevModel<MT>& d, const PackDesc& pk, const Work<MT>& w, int lane,
                                         bool decay, int apply_step, bool current, int& ev_i, int ev_end,
                                         int32_t& late) {
    // drop events that should already have been applied (never happens by construction)
    while (apply_step >= 0 && ev_i < ev_end && d.ev[ev_i].step_rel < apply_step) { ++ev_i; late = 1; }
#pragma unroll 4
    for (int js = 0; js < pk.nsyn_row; ++js) {
        const size_t q = (size_t)(pk.syn_row0 + js) * kWarp + lane;
        const int sl = __ldg(d.syn_slot + q);
        if (sl < 0) continue;
        const int idx = js * kWarp + lane;
        MT g = w.g[idx];
        if (decay) g = g * (MT)__ldg(d.syn_decay + q);
        if (apply_step >= 0) {
            while (ev_i < ev_end && d.ev[ev_i].step_rel == apply_step && d.ev[ev_i].js == js) {
                g = g + (MT)d.ev[ev_i].w;
                ++ev_i;
            }
        }
        w.g[idx] = g;
        if (current) {
            if constexpr (kImp) {
                const double gd = (double)g;
                w.R[sl] += gd;
                w.S[sl] = fma(gd, __ldg(d.syn_e + q), w.S[sl]);
            } else {
                const int vs = kSmem ? __ldg(d.syn_vs + q) : sl;
                const MT i_syn = g * (MT)(w.Vc[vs] - __ldg(d.syn_e + q));
                w.S[sl] = fma(-__ldg(d.syn_sc + q), (double)i_syn, w.S[sl]);
            }
        }
    }
}

// Hodgkin-Huxley: gate update with the new voltage, then the Na and K terms of the next
// step (the leak is constant and sits in the constants of the entry).
template <class MT, bool kSmem, bool kImp>
__device__ __forceinline__ void hh_pass(const DevModel<MT>& d, const PackDesc& pk, const Work<MT>& w, int lane,
                                        bool update, bool current, MT dt) {
    for (int jh = 0; jh < pk.nhh_row; ++jh) {
        const size_t q = (size_t)(pk.hh_row0 + jh) * kWarp + lane;
        const int sl = __ldg(d.hh_slot + q);
        if (sl < 0) continue;
        const int vs = kSmem ? __ldg(d.hh_vs + q) : sl;
        const int idx = jh * kWarp + lane;
        const double vd = w.Vc[vs];
        const MT v = (MT)vd;
        MT m = w.m[idx], h = w.h[idx], n = w.n[idx];
        if (update) {
            bool done = false;
            if constexpr (std::is_same<MT, double>::value) done = hh_gates_tab(d.hh_tab, vd, m, h, n);
            else done = hh_gates_tab_f(d.hh_tab_f, vd, m, h, n);
            if (!done) {
                const auto r = hh_rates(v);
                m = gate(m, r.am, r.bm, dt);
                h = gate(h, r.ah, r.bh, dt);
                n = gate(n, r.an, r.bn, dt);
            }
            w.m[idx] = m;
            w.h[idx] = h;
            w.n[idx] = n;
        }
        if (current) {
            const MT n2 = n * n;
            const MT gna = (MT)__ldg(d.hh_gna + q) * (m * m * m * h);
            const MT gk = (MT)__ldg(d.hh_gk + q) * (n2 * n2);
            if constexpr (kImp) {
                w.R[sl] += (double)(gna + gk);
                w.S[sl] += (double)(gna * (MT)kENa + gk * (MT)kEK);
            } else {
                const MT i_hh = gna * (MT)(vd - kENa) + gk * (MT)(vd - kEK);
                w.S[sl] = fma(-__ldg(d.hh_sc + q), (double)i_hh, w.S[sl]);
            }
        }
    }
}

constexpr int kU = 8;   // rows whose constants are loaded ahead of use

// One pack for all steps of the epoch.
//
// Explicit scheme (membrane current at V(t), Sec. "Model" linear system as printed): the
// matrix is constant for fixed dt, the host factorised it once, and S holds right-hand sides
// already divided by the eliminated pivots d':
//   forward  u_i = S_i - sum_children a'_c u_c;  backward V_i = u_i - e_i V_parent;
//   next     S_i = alpha'_i V_i + beta'_i - (mechanism currents)/d'_i.
// Implicit scheme (default; V(t+dt) from Eq. discrete-v by implicit Euler with the states
// frozen at t): R holds the diagonal c/dt + G + sum sigma, S the right-hand side
// (c/dt) V + sum g E + I_inj; elimination from the leaves with one reciprocal per CV:
//   d'_i = R_i - sum_children sigma_c e_c,  r = 1/d'_i,  b'_i = S_i + sum_children sigma_c u_c,
//   u_i = r b'_i,  e_i = sigma_i r;   backward V_i = u_i + e_i V_parent.
template <class MT, bool kSmem, bool kImp>
__device__ void run_pack(const DevModel<MT>& d, int p, double* tile, int64_t k0, int nsteps, int lane) {
    const PackDesc pk = d.packs[p];
    const int J = pk.nrow;
    const int R = pk.round_rows;
    double* Vg = d.V + (size_t)pk.row0 * kWarp;
    Work<MT> w;
    if (kSmem) {
        w.S = tile;
        w.R = kImp ? tile + (size_t)J * kWarp : nullptr;
        w.Vc = tile + (size_t)J * kWarp * (kImp ? 2 : 1);
        w.g = (MT*)(w.Vc + pk.nvc);
        w.m = w.g + (size_t)pk.nsyn_row * kWarp;
        w.h = w.m + (size_t)pk.nhh_row * kWarp;
        w.n = w.h + (size_t)pk.nhh_row * kWarp;
        for (int i = lane; i < pk.nsyn_row * kWarp; i += kWarp) w.g[i] = d.syn_g[(size_t)pk.syn_row0 * kWarp + i];
        for (int i = lane; i < pk.nhh_row * kWarp; i += kWarp) {
            const size_t gi = (size_t)pk.hh_row0 * kWarp + i;
            w.m[i] = d.hh_m[gi];
            w.h[i] = d.hh_h[gi];
            w.n[i] = d.hh_n[gi];
        }
    } else {
        w.S = d.Sg + pk.sg_off;
        w.R = kImp ? d.Rg + pk.sg_off : nullptr;
        w.Vc = Vg;
        w.g = d.syn_g + (size_t)pk.syn_row0 * kWarp;
        w.m = d.hh_m + (size_t)pk.hh_row0 * kWarp;
        w.h = d.hh_h + (size_t)pk.hh_row0 * kWarp;
        w.n = d.hh_n + (size_t)pk.hh_row0 * kWarp;
    }
    double* __restrict__ S = w.S;
    double* __restrict__ Rr = w.R;
    double* __restrict__ Vc = w.Vc;
    const size_t e0 = (size_t)pk.row0 * kWarp + lane;
    const double* __restrict__ ca = d.ca + e0;
    const double* __restrict__ cb = d.cb + e0;
    const double* __restrict__ ck = d.ck + e0;
    const double* __restrict__ ce = d.ce + e0;
    const int32_t* __restrict__ ps_arr = d.pslot + e0;
    const int32_t* __restrict__ vm_arr = d.vmap + e0;

    // right-hand side (and diagonal) of the first step; on-chip copies of the read voltages
    for (int j = 0; j < J; ++j) {
        const int sl = j * kWarp + lane;
        const size_t o = (size_t)j * kWarp;
        const double v = Vg[sl];
        S[sl] = fma(__ldg(ca + o), v, __ldg(cb + o));
        if (kImp) Rr[sl] = __ldg(ce + o);
        if (kSmem) {
            const int own = __ldg(vm_arr + o) & 0xFFFF;
            if (own != 0xFFFF) Vc[own] = v;
        }
    }
    __syncwarp();

    const int owner = p * kWarp + lane;
    int ev_i = d.ev_off[owner];
    const int ev_end = d.ev_off[owner + 1];
    int32_t late = 0;
    const double dt = d.dt;
    const MT dt_m = (MT)dt;

    // terms of the epoch's first step (events due at its start included)
    syn_pass<MT, kSmem, kImp>(d, pk, w, lane, false, 0, true, ev_i, ev_end, late);
    __syncwarp();
    hh_pass<MT, kSmem, kImp>(d, pk, w, lane, false, true, dt_m);
    __syncwarp();

    const int det = (lane < pk.ncell) ? ARB_IDX(d.det_slot[owner], pk.nrow * kWarp, d.ctl) : -1;
    const double thr = d.threshold;
    const int64_t probe_k0 = d.ctl->probe_k0, probe_max = d.ctl->probe_max;
    const bool probing = pk.npr > 0 && probe_max > 0;
    bool bad = false;

    for (int s = 0; s < nsteps; ++s) {
        const int64_t k = k0 + s;
        const double t = __dmul_rn((double)k, dt);
        const bool last = (s + 1) == nsteps;
        // current clamps active at t_k (depolarising current enters with a plus sign)
        for (int js = 0; js < pk.nst_row; ++js) {
            const size_t q = (size_t)(pk.st_row0 + js) * kWarp + lane;
            const int sl = __ldg(d.st_slot + q);
            if (sl >= 0 && __ldg(d.st_on + q) <= t && t < __ldg(d.st_off + q)) {
                if (kImp) S[sl] += __ldg(d.st_amp + q);
                else S[sl] = fma(__ldg(d.st_sc + q), __ldg(d.st_amp + q), S[sl]);
            }
        }
        __syncwarp();
        const double v0 = det >= 0 ? Vc[det] : 0.0;

        // forward elimination, leaves to root
        {
            double yprev = 0.0, kprev = 0.0, eprev = 0.0;
            int left = R;
            int psn[kU];
            double kcn[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const bool in = u < J;
                psn[u] = in ? __ldg(ps_arr + (size_t)u * kWarp) : -2;
                kcn[u] = in ? __ldg(ck + (size_t)u * kWarp) : 0.0;
            }
            for (int jb = 0; jb < J; jb += kU) {
                int psc[kU];
                double kcc[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) { psc[u] = psn[u]; kcc[u] = kcn[u]; }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int j = jb + kU + u;
                    const bool in = j < J;
                    psn[u] = in ? __ldg(ps_arr + (size_t)j * kWarp) : -2;
                    kcn[u] = in ? __ldg(ck + (size_t)j * kWarp) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int j = jb + u;
                    if (j < J) {
                        if (R > 0) {
                            if (left == 0) { __syncwarp(); left = R; }
                            --left;
                        }
                        const int ps = psc[u];
                        const int sl = j * kWarp + lane;
                        if constexpr (kImp) {
                            // kprev = sigma of the previous row when it is this row's child
                            const double dd = fma(-kprev, eprev, Rr[sl]);
                            const double r = rcp_nr(dd);
                            const double bb = fma(kprev, yprev, S[sl]);
                            const double uu = r * bb;
                            const double ee = kcc[u] * r;
                            S[sl] = uu;
                            Rr[sl] = ee;
                            if (ps >= 0) {
                                Rr[ps] = fma(-kcc[u], ee, Rr[ps]);
                                S[ps] = fma(kcc[u], uu, S[ps]);
                            }
                            kprev = (ps == -1) ? kcc[u] : 0.0;
                            eprev = ee;
                            yprev = uu;
                        } else {
                            const double y = fma(-kprev, yprev, S[sl]);
                            S[sl] = y;
                            if (ps >= 0) S[ps] = fma(-kcc[u], y, S[ps]);
                            kprev = (ps == -1) ? kcc[u] : 0.0;
                            yprev = y;
                        }
                    }
                }
            }
        }
        __syncwarp();
        // back substitution, root to leaves; then the next step's right-hand side (and diagonal)
        {
            const bool full = last || probing || !kSmem;
            double vnext = 0.0;
            int left = (R > 0) ? ((J - 1) % R) + 1 : 0;
            int psn[kU], vmn[kU];
            double cen[kU], can[kU], cbn[kU];
            auto load_b = [&](int jtop, int* ps_, int* vm_, double* ce_, double* ca_, double* cb_) {
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int j = jtop - u;
                    const bool in = j >= 0;
                    const size_t o = (size_t)(in ? j : 0) * kWarp;
                    ps_[u] = in ? __ldg(ps_arr + o) : -2;
                    vm_[u] = (in && kSmem) ? __ldg(vm_arr + o) : -1;
                    ce_[u] = in ? __ldg(ce + o) : 0.0;
                    ca_[u] = in ? __ldg(ca + o) : 0.0;
                    cb_[u] = in ? __ldg(cb + o) : 0.0;
                }
            };
            load_b(J - 1, psn, vmn, cen, can, cbn);
            for (int jt = J - 1; jt >= 0; jt -= kU) {
                int psc[kU], vmc[kU];
                double cec[kU], cac[kU], cbc[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) { psc[u] = psn[u]; vmc[u] = vmn[u]; cec[u] = cen[u]; cac[u] = can[u]; cbc[u] = cbn[u]; }
                load_b(jt - kU, psn, vmn, cen, can, cbn);
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int j = jt - u;
                    if (j >= 0) {
                        if (R > 0) {
                            if (left == 0) { __syncwarp(); left = R; }
                            --left;
                        }
                        const int ps = psc[u];
                        const int sl = j * kWarp + lane;
                        double vp = 0.0;
                        if (ps == -1) vp = vnext;
                        else if (ps >= 0) vp = Vc[kSmem ? ((unsigned)vmc[u] >> 16) : ps];
                        double v;
                        if constexpr (kImp) {
                            v = fma(Rr[sl], vp, S[sl]);
                            Rr[sl] = cec[u];
                        } else {
                            v = fma(-cec[u], vp, S[sl]);
                        }
                        if (kSmem) {
                            const int own = vmc[u] & 0xFFFF;
                            if (own != 0xFFFF) Vc[own] = v;
                        }
                        if (full) Vg[sl] = v;
                        if (last) bad |= !isfinite(v);
                        S[sl] = fma(cac[u], v, cbc[u]);
                        vnext = v;
                    }
                }
            }
        }
        __syncwarp();

        // state updates with V(t_{k+1}); terms of the next step
        syn_pass<MT, kSmem, kImp>(d, pk, w, lane, true, last ? -1 : s + 1, !last, ev_i, ev_end, late);
        __syncwarp();
        hh_pass<MT, kSmem, kImp>(d, pk, w, lane, true, !last, dt_m);

        // threshold crossing between V(t_k) and V(t_{k+1}), linearly interpolated
        bool spk = false;
        double ts = 0.0;
        if (det >= 0) {
            const double v1 = Vc[det];
            if (v0 < thr && v1 >= thr) {
                spk = true;
                ts = __dadd_rn(t, __dmul_rn(dt, __ddiv_rn(__dsub_rn(thr, v0), __dsub_rn(v1, v0))));
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, spk);
        if (ball) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd((unsigned long long*)&d.ctl->n_spikes, (unsigned long long)__popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (spk) {
                const int64_t pos = (int64_t)base + __popc(ball & ((1u << lane) - 1u));
                if (pos < d.spike_cap) {
                    d.spk_gid[pos] = d.det_gid[owner];
                    d.spk_t[pos] = ts;
                } else {
                    atomicOr(&d.ctl->status, kStSpikeOverflow);
                }
            }
        }
        // probes record V(t_{k+1}) from the full voltage array written above
        if (probing) {
            __syncwarp();
            const int64_t prow = k - probe_k0;
            if (prow >= 0 && prow < probe_max)
                for (int q = lane; q < pk.npr; q += kWarp)
                    d.trace[prow * d.n_probe + ARB_IDX(d.probe_col[pk.pr0 + q], d.n_probe, d.ctl)] =
                        Vg[ARB_IDX(d.probe_slot[pk.pr0 + q], pk.nrow * kWarp, d.ctl)];
        }
        __syncwarp();
    }

    if (kSmem) {
        for (int i = lane; i < pk.nsyn_row * kWarp; i += kWarp) d.syn_g[(size_t)pk.syn_row0 * kWarp + i] = w.g[i];
        for (int i = lane; i < pk.nhh_row * kWarp; i += kWarp) {
            const size_t gi = (size_t)pk.hh_row0 * kWarp + i;
            d.hh_m[gi] = w.m[i];
            d.hh_h[gi] = w.h[i];
            d.hh_n[gi] = w.n[i];
        }
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    const bool any_late = __any_sync(0xffffffffu, late != 0);
    if (lane == 0 && (any_bad || any_late))
        atomicOr(&d.ctl->status, (any_bad ? kStNonFinite : 0) | (any_late ? kStLateEvent : 0));
    __syncwarp();
}

template <class MT, bool kImp>
__global__ void __launch_bounds__(256) arb_epoch_kernel(DevModel<MT> d, int tile_doubles) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    double* tile = smem + (size_t)wid * tile_doubles;
    const int64_t k0 = d.ctl->k0;
    const int nsteps = (int)(d.ctl->k1 - k0);
    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(&d.ctl->pack_next, 1);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= d.n_packs) break;
        if (d.packs[p].smem) run_pack<MT, true, kImp>(d, p, tile, k0, nsteps, lane);
        else run_pack<MT, false, kImp>(d, p, tile, k0, nsteps, lane);
    }
}

// ------------------------------------------------------------------------------------------
// Streamed packs (large batches): one cell per lane, every array in global memory.
//
// A lane walks its cell in reverse depth-first order, so a CV's parent is the next row of the
// lane except at branch points. A child that is not processed directly before its parent hands
// its contribution over through a small per-lane stack in shared memory; in reverse
// depth-first order these hand-overs are strictly last in, first out. Nothing is ever written
// into a row that has not been reached yet, so every load of a row can be issued rows ahead.
// The back substitution uses the same stack, in preorder, for the parent voltages of those
// children. Mechanism terms of a step are accumulated per compact slot (Gm, Em) before the
// forward sweep.

template <class MT, bool kImp>
__device__ __forceinline__ void stream_mech(const DevModel<MT>& d, const PackDesc& pk, double* Gm, double* Em,
                                            const double* Vg, MT* gS, MT* mS, MT* hS, MT* nS, int lane, bool decay,
                                            bool update, int apply_step, bool terms, int& ev_i, int ev_end,
                                            int32_t& late, MT dt) {
    const double* cE = d.cE + pk.c_off;
    const double* cB = d.cB + pk.c_off;
    if (terms) {
        // implicit: the slots start from the constant diagonal and right-hand side of their
        // entry, so the forward sweep adds nothing for them. Slots [0, nsc) belong to CVs with
        // synapses and are written whole by the synapse pass below.
#pragma unroll 4
        for (int c = pk.nsc + lane; c < pk.nvc; c += kWarp) {
            if (kImp) {
                Gm[c] = __ldg(cE + c);
                Em[c] = __ldg(cB + c);
            } else {
                Em[c] = 0.0;
            }
        }
    }
    __syncwarp();
    // the lane's next event, kept in registers
    while (apply_step >= 0 && ev_i < ev_end && d.ev[ev_i].step_rel < apply_step) { ++ev_i; late = 1; }
    int n_step = 0x7fffffff, n_js = -1;
    double n_w = 0.0;
    if (apply_step >= 0 && ev_i < ev_end) {
        const EvRec r = d.ev[ev_i];
        n_step = r.step_rel;
        n_js = r.js;
        n_w = r.w;
    }
    // synapses of one CV are consecutive on one lane: their terms are summed in registers and
    // the CV's slot is written once, starting from its constants (implicit scheme). Rows are
    // fetched kSP ahead, their slot index 2 kSP ahead, so that no load is waited for in the row
    // that issued it.
    constexpr int kSP = 1;
    // sums of the synapse terms of one CV in the mechanism precision (FP32 currents in the mixed form)
    using ST = typename std::conditional<kImp, MT, double>::type;
    int cur = -1;
    ST gsum = 0, esum = 0;
    double cur_e = 0.0, cur_b = 0.0;
    int s_sl[kSP], s_c[kSP], s_cn[kSP];
    ST s_dec[kSP], s_e[kSP];
    double s_sc[kSP], s_ce[kSP], s_cb[kSP];
    MT s_g[kSP];
    // per-synapse decay factor and reversal in the precision of the sums (float copies for FP32
    // mechanisms, so that no conversion is needed per synapse row)
    const ST* syn_dec_p;
    const ST* syn_e_p;
    if constexpr (std::is_same<ST, float>::value) {
        syn_dec_p = d.syn_decay_f;
        syn_e_p = d.syn_e_f;
    } else {
        syn_dec_p = d.syn_decay;
        syn_e_p = d.syn_e;
    }
    auto sfetch_c = [&](int js) {
        return js < pk.nsyn_row ? __ldg(d.syn_vs + (size_t)(pk.syn_row0 + js) * kWarp + lane) : -1;
    };
    auto sfetch = [&](int js, int u, int c) {
        const bool in = js < pk.nsyn_row;
        const size_t q = (size_t)(pk.syn_row0 + (in ? js : 0)) * kWarp + lane;
        s_c[u] = c;
        s_sl[u] = (in && !kImp) ? __ldg(d.syn_slot + q) : -1;
        s_dec[u] = in ? __ldg(syn_dec_p + q) : (ST)1;
        s_e[u] = in ? __ldg(syn_e_p + q) : (ST)0;
        s_sc[u] = (in && !kImp) ? __ldg(d.syn_sc + q) : 0.0;
        s_g[u] = in ? gS[(in ? js : 0) * kWarp + lane] : (MT)0;
        s_ce[u] = (kImp && terms && c >= 0) ? __ldg(cE + c) : 0.0;
        s_cb[u] = (kImp && terms && c >= 0) ? __ldg(cB + c) : 0.0;
    };
    {
        int c0[kSP];
#pragma unroll
        for (int u = 0; u < kSP; ++u) c0[u] = sfetch_c(u);
#pragma unroll
        for (int u = 0; u < kSP; ++u) s_cn[u] = sfetch_c(kSP + u);
#pragma unroll
        for (int u = 0; u < kSP; ++u) sfetch(u, u, c0[u]);
    }
    for (int jb = 0; jb < pk.nsyn_row; jb += kSP) {
#pragma unroll
        for (int u = 0; u < kSP; ++u) {
            const int js = jb + u;
            if (js >= pk.nsyn_row) break;
            const int sl = s_sl[u], c = s_c[u] < 0 ? s_c[u] : ARB_IDX(s_c[u], pk.nvc, d.ctl);
            const ST dec = s_dec[u], esyn = s_e[u];
            const double sc = s_sc[u], c_e = s_ce[u], c_b = s_cb[u];
            MT g = s_g[u];
            sfetch(js + kSP, u, s_cn[u]);         // row js + kSP: its slot index is ready
            s_cn[u] = sfetch_c(js + 2 * kSP);     // slot index of row js + 2 kSP
            if (c < 0) continue;                  // padding
            if (decay) g = g * (MT)dec;
            while (n_step == apply_step && n_js == js) {
                g = g + (MT)n_w;
                ++ev_i;
                if (ev_i < ev_end) {
                    const EvRec r = d.ev[ev_i];
                    n_step = r.step_rel;
                    n_js = r.js;
                    n_w = r.w;
                } else {
                    n_step = 0x7fffffff;
                }
            }
            gS[js * kWarp + lane] = g;
            if (terms) {
                if (c != cur) {
                    if (cur >= 0) {
                        if (kImp) {
                            Gm[cur] = cur_e + (double)gsum;
                            Em[cur] = cur_b + (double)esum;
                        } else {
                            Em[cur] = (double)esum;
                        }
                    }
                    cur = c;
                    cur_e = c_e;
                    cur_b = c_b;
                    gsum = 0;
                    esum = 0;
                }
                if constexpr (kImp) {
                    gsum += (ST)g;
                    esum = fma((ST)g, (ST)esyn, esum);
                } else {
                    const MT i_syn = g * (MT)(Vg[sl] - esyn);
                    esum = fma(-sc, (double)i_syn, esum);
                }
            }
        }
    }
    if (terms && cur >= 0) {
        if (kImp) {
            Gm[cur] = cur_e + (double)gsum;
            Em[cur] = cur_b + (double)esum;
        } else {
            Em[cur] = (double)esum;
        }
    }
    __syncwarp();
    for (int jh = 0; jh < pk.nhh_row; ++jh) {
        const size_t q = (size_t)(pk.hh_row0 + jh) * kWarp + lane;
        int sl = __ldg(d.hh_slot + q);
        if (sl < 0) continue;
        sl = ARB_IDX(sl, pk.nrow * kWarp, d.ctl);
        const int idx = jh * kWarp + lane;
        const double vd = Vg[sl];
        const MT v = (MT)vd;
        MT m = mS[idx], h = hS[idx], n = nS[idx];
        if (update) {
            bool done = false;
            if constexpr (std::is_same<MT, double>::value) done = hh_gates_tab(d.hh_tab, vd, m, h, n);
            else done = hh_gates_tab_f(d.hh_tab_f, vd, m, h, n);
            if (!done) {
                const auto r = hh_rates(v);
                m = gate(m, r.am, r.bm, dt);
                h = gate(h, r.ah, r.bh, dt);
                n = gate(n, r.an, r.bn, dt);
            }
            mS[idx] = m;
            hS[idx] = h;
            nS[idx] = n;
        }
        if (terms) {
            const int c = ARB_IDX(__ldg(d.hh_vs + q), pk.nvc, d.ctl);
            const MT n2 = n * n;
            MT gbna, gbk;
            if constexpr (std::is_same<MT, float>::value) {
                gbna = __ldg(d.hh_gna_f + q);
                gbk = __ldg(d.hh_gk_f + q);
            } else {
                gbna = __ldg(d.hh_gna + q);
                gbk = __ldg(d.hh_gk + q);
            }
            const MT gna = gbna * (m * m * m * h);
            const MT gk = gbk * (n2 * n2);
            if constexpr (kImp) {
                Gm[c] += (double)(gna + gk);
                Em[c] += (double)(gna * (MT)kENa + gk * (MT)kEK);
            } else {
                const MT i_hh = gna * (MT)(vd - kENa) + gk * (MT)(vd - kEK);
                Em[c] = fma(-__ldg(d.hh_sc + q), (double)i_hh, Em[c]);
            }
        }
    }
    __syncwarp();
}

#ifndef ARB_STREAM_PF
#define ARB_STREAM_PF 1
#endif
#ifndef ARB_STREAM_PB
#define ARB_STREAM_PB 6
#endif
constexpr int kPF = ARB_STREAM_PF;   // rows prefetched ahead in the streamed forward sweep
constexpr int kPB = ARB_STREAM_PB;   // rows prefetched ahead in the streamed back substitution (light rows)

template <class MT, bool kImp, bool kShared>
__device__ void run_pack_stream(const DevModel<MT>& d, int p, double2* stack, int64_t k0, int nsteps, int lane) {
    const PackDesc pk = d.packs[p];
    const int J = pk.nrow;
    double* Vg = d.V + (size_t)pk.row0 * kWarp;
    double* Bs = d.Sg + pk.sg_off;                 // forward result u (or y), per entry
    double* Rs = d.Rg + pk.sg_off;                 // implicit: e = sigma / d', per entry
    double* Gm = d.Gm + pk.c_off;
    double* Em = d.Em + pk.c_off;
    MT* gS = d.syn_g + (size_t)pk.syn_row0 * kWarp;
    MT* mS = d.hh_m + (size_t)pk.hh_row0 * kWarp;
    MT* hS = d.hh_h + (size_t)pk.hh_row0 * kWarp;
    MT* nS = d.hh_n + (size_t)pk.hh_row0 * kWarp;
    const size_t e0 = (size_t)pk.row0 * kWarp + lane;
    const double* __restrict__ ca = d.ca + e0;
    const double* __restrict__ cb = d.cb + e0;
    const double* __restrict__ ck = d.ck + e0;
    const double* __restrict__ ce = d.ce + e0;
    const int32_t* __restrict__ fl = d.pslot + e0;
    const int32_t* __restrict__ cm_ = d.vmap + e0;
    double2* stk = stack;   // [depth][32] (one cell per lane)
    double* mbd = (double*)stack;           // mailbox (cells spread over lanes): [nmb] x (d, b, v)
    double* mbb = mbd + pk.nmb;
    double* mbv = mbb + pk.nmb;
    const int R = kShared ? pk.round_rows : 0;

    const int owner = p * kWarp + lane;
    int ev_i = d.ev_off[owner];
    const int ev_end = d.ev_off[owner + 1];
    int32_t late = 0;
    const double dt = d.dt;
    const MT dt_m = (MT)dt;
    stream_mech<MT, kImp>(d, pk, Gm, Em, Vg, gS, mS, hS, nS, lane, false, false, 0, true, ev_i, ev_end, late, dt_m);

    const int det = (lane < pk.ncell) ? ARB_IDX(d.det_slot[owner], pk.nrow * kWarp, d.ctl) : -1;
    const double thr = d.threshold;
    const int64_t probe_k0 = d.ctl->probe_k0, probe_max = d.ctl->probe_max;
    const bool probing = pk.npr > 0 && probe_max > 0;
    bool bad = false;

    for (int s = 0; s < nsteps; ++s) {
        const int64_t k = k0 + s;
        const double t = __dmul_rn((double)k, dt);
        const bool last = (s + 1) == nsteps;
        for (int js = 0; js < pk.nst_row; ++js) {
            const size_t q = (size_t)(pk.st_row0 + js) * kWarp + lane;
            const int c = __ldg(d.st_slot + q);
            if (c >= 0 && __ldg(d.st_on + q) <= t && t < __ldg(d.st_off + q)) {
                if (kImp) Em[c] += __ldg(d.st_amp + q);
                else Em[c] = fma(__ldg(d.st_sc + q), __ldg(d.st_amp + q), Em[c]);
            }
        }
        __syncwarp();
        const double v0 = det >= 0 ? Vg[det] : 0.0;

        // forward elimination, leaves to root, streaming rows
        {
            if (kShared) {
                for (int i = lane; i < pk.nmb; i += kWarp) { mbd[i] = 0.0; mbb[i] = 0.0; }
                __syncwarp();
            }
            int sp = 0, left = R;
            double yprev = 0.0, kprev = 0.0, eprev = 0.0;
            // rows are fetched kPF ahead; the compact mechanism slot of a row is fetched 2*kPF
            // ahead so that the load of its terms never waits on the index load
            double pv[kPF], pa[kPF], pb[kPF], pk_[kPF], pe[kPF], pm[kPF];
            int pf[kPF], pc[kPF];
            auto fetch_c = [&](int j) { return j < J ? __ldg(cm_ + (size_t)j * kWarp) : -1; };
            auto fetch = [&](int j, int u, int c) {
                const bool in = j < J;
                const size_t o = (size_t)(in ? j : 0) * kWarp;
                pv[u] = in ? Vg[(in ? j : 0) * kWarp + lane] : 0.0;
                pa[u] = in ? __ldg(ca + o) : 0.0;
                pk_[u] = in ? __ldg(ck + o) : 0.0;
                pf[u] = in ? __ldg(fl + o) : kFlagRoot;
                if constexpr (kImp) {
                    // diagonal and right-hand side terms: the mechanism slot's, else the constants
                    pe[u] = c >= 0 ? Gm[c] : (in ? __ldg(ce + o) : 1.0);
                    pb[u] = c >= 0 ? Em[c] : (in ? __ldg(cb + o) : 0.0);
                } else {
                    pe[u] = in ? __ldg(ce + o) : 1.0;
                    pb[u] = in ? __ldg(cb + o) : 0.0;
                    pm[u] = c >= 0 ? Em[c] : 0.0;
                }
            };
            {
                int c0[kPF];
#pragma unroll
                for (int u = 0; u < kPF; ++u) c0[u] = fetch_c(u);
#pragma unroll
                for (int u = 0; u < kPF; ++u) pc[u] = fetch_c(kPF + u);
#pragma unroll
                for (int u = 0; u < kPF; ++u) fetch(u, u, c0[u]);
            }
            for (int jb = 0; jb < J; jb += kPF) {
#pragma unroll
                for (int u = 0; u < kPF; ++u) {
                    const int j = jb + u;
                    if (j < J) {
                        if (kShared && R > 0) {
                            if (left == 0) { __syncwarp(); left = R; }
                            --left;
                        }
                        const double V = pv[u], A = pa[u], Bc = pb[u], K = pk_[u], E = pe[u];
                        const double M = kImp ? 0.0 : pm[u];
                        const int f = pf[u];
                        fetch(j + kPF, u, pc[u]);        // row j + kPF, its slot index is ready
                        pc[u] = fetch_c(j + 2 * kPF);    // slot index of row j + 2 kPF
                        const int sl = j * kWarp + lane;
                        const int mb_in = kShared ? (int)((unsigned)f >> kMbInShift) : kMbNone;
                        const int mb_out = kShared ? ((f >> kMbOutShift) & kMbNone) : kMbNone;
                        if constexpr (kImp) {
                            double dd = fma(-kprev, eprev, E);
                            double bb = fma(kprev, yprev, fma(A, V, Bc));
                            if (kShared) {
                                if (mb_in != kMbNone) { dd -= mbd[ARB_IDX(mb_in, pk.nmb, d.ctl)]; bb += mbb[ARB_IDX(mb_in, pk.nmb, d.ctl)]; }
                            } else {
                                for (int q = f & kFlagPopMask; q > 0; --q) {
                                    const double2 c2 = stk[ARB_IDX(--sp, pk.stack, d.ctl) * kWarp + lane];
                                    dd -= c2.x;
                                    bb += c2.y;
                                }
                            }
                            const double r = rcp_nr(dd);
                            const double uu = r * bb;
                            const double ee = K * r;
                            Bs[sl] = uu;
                            Rs[sl] = ee;
                            const bool remote = (f & kFlagRemote) != 0;
                            if (remote && !(f & kFlagRoot)) {
                                if (kShared) { mbd[ARB_IDX(mb_out, pk.nmb, d.ctl)] += K * ee; mbb[ARB_IDX(mb_out, pk.nmb, d.ctl)] += K * uu; }
                                else stk[ARB_IDX(sp++, pk.stack, d.ctl) * kWarp + lane] = make_double2(K * ee, K * uu);
                            }
                            kprev = remote ? 0.0 : K;
                            eprev = ee;
                            yprev = uu;
                        } else {
                            double y = fma(-kprev, yprev, fma(A, V, Bc) + M);
                            if (kShared) {
                                if (mb_in != kMbNone) y -= mbd[ARB_IDX(mb_in, pk.nmb, d.ctl)];
                            } else {
                                for (int q = f & kFlagPopMask; q > 0; --q) y -= stk[ARB_IDX(--sp, pk.stack, d.ctl) * kWarp + lane].x;
                            }
                            Bs[sl] = y;
                            const bool remote = (f & kFlagRemote) != 0;
                            if (remote && !(f & kFlagRoot)) {
                                if (kShared) mbd[ARB_IDX(mb_out, pk.nmb, d.ctl)] += K * y;
                                else stk[ARB_IDX(sp++, pk.stack, d.ctl) * kWarp + lane] = make_double2(K * y, 0.0);
                            }
                            kprev = remote ? 0.0 : K;
                            yprev = y;
                        }
                    }
                }
            }
        }
        if (kShared) __syncwarp();
        // back substitution, root to leaves (preorder), streaming rows
        {
            int sp = 0;
            double vnext = 0.0;
            double pu[kPB], px[kPB];
            int pf[kPB];
            int left = kShared ? ((R > 0) ? ((J - 1) % R) + 1 : 0) : 0;
            auto fetch = [&](int j, int u) {
                const bool in = j >= 0;
                const size_t o = (size_t)(in ? j : 0) * kWarp;
                pu[u] = in ? Bs[(in ? j : 0) * kWarp + lane] : 0.0;
                px[u] = in ? (kImp ? Rs[(in ? j : 0) * kWarp + lane] : -__ldg(ce + o)) : 0.0;
                pf[u] = in ? __ldg(fl + o) : kFlagRoot;
            };
#pragma unroll
            for (int u = 0; u < kPB; ++u) fetch(J - 1 - u, u);
            for (int jt = J - 1; jt >= 0; jt -= kPB) {
#pragma unroll
                for (int u = 0; u < kPB; ++u) {
                    const int j = jt - u;
                    if (j >= 0) {
                        if (kShared && R > 0) {
                            if (left == 0) { __syncwarp(); left = R; }
                            --left;
                        }
                        const double U = pu[u], X = px[u];
                        const int f = pf[u];
                        fetch(j - kPB, u);
                        double vp;
                        if (f & kFlagRoot) vp = 0.0;
                        else if (f & kFlagRemote) vp = kShared ? mbv[ARB_IDX((f >> kMbOutShift) & kMbNone, pk.nmb, d.ctl)] : stk[ARB_IDX(--sp, pk.stack, d.ctl) * kWarp + lane].x;
                        else vp = vnext;
                        const double v = fma(X, vp, U);
                        if (kShared) {
                            const int mb_in = (int)((unsigned)f >> kMbInShift);
                            if (mb_in != kMbNone) mbv[ARB_IDX(mb_in, pk.nmb, d.ctl)] = v;
                        } else {
                            for (int q = f & kFlagPopMask; q > 0; --q) stk[ARB_IDX(sp++, pk.stack, d.ctl) * kWarp + lane] = make_double2(v, 0.0);
                        }
                        Vg[j * kWarp + lane] = v;
                        if (last) bad |= !isfinite(v);
                        vnext = v;
                    }
                }
            }
        }
        __syncwarp();

        // state updates with V(t_{k+1}); terms of the next step
        stream_mech<MT, kImp>(d, pk, Gm, Em, Vg, gS, mS, hS, nS, lane, true, true, last ? -1 : s + 1, !last, ev_i,
                              ev_end, late, dt_m);

        bool spk = false;
        double ts = 0.0;
        if (det >= 0) {
            const double v1 = Vg[det];
            if (v0 < thr && v1 >= thr) {
                spk = true;
                ts = __dadd_rn(t, __dmul_rn(dt, __ddiv_rn(__dsub_rn(thr, v0), __dsub_rn(v1, v0))));
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, spk);
        if (ball) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd((unsigned long long*)&d.ctl->n_spikes, (unsigned long long)__popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (spk) {
                const int64_t pos = (int64_t)base + __popc(ball & ((1u << lane) - 1u));
                if (pos < d.spike_cap) {
                    d.spk_gid[pos] = d.det_gid[owner];
                    d.spk_t[pos] = ts;
                } else {
                    atomicOr(&d.ctl->status, kStSpikeOverflow);
                }
            }
        }
        if (probing) {
            const int64_t prow = k - probe_k0;
            if (prow >= 0 && prow < probe_max)
                for (int q = lane; q < pk.npr; q += kWarp)
                    d.trace[prow * d.n_probe + ARB_IDX(d.probe_col[pk.pr0 + q], d.n_probe, d.ctl)] =
                        Vg[ARB_IDX(d.probe_slot[pk.pr0 + q], pk.nrow * kWarp, d.ctl)];
        }
        __syncwarp();
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    const bool any_late = __any_sync(0xffffffffu, late != 0);
    if (lane == 0 && (any_bad || any_late))
        atomicOr(&d.ctl->status, (any_bad ? kStNonFinite : 0) | (any_late ? kStLateEvent : 0));
    __syncwarp();
}

// ------------------------------------------------------------------------------------------
// Streamed packs with exact event times (Sec. "Model": the time step is shortened so that every
// synapse update falls at the start of an integration step). One cell per lane, and each lane's
// synapses, HH instances and clamps on that lane, so that every lane cuts its own steps: a step
// of the lane's cell is a sequence of pieces [cur, next], next being the next event time inside
// the step or the step's end, each piece an implicit step of its own length h (c/h on the
// diagonal, gates and synapses advanced over h, clamps sampled at cur). Lanes with fewer pieces
// keep their state while the others go on. Events are listed per lane by (step, time, row).

__device__ void run_pack_exact(const DevModel<double>& d, int p, double2* stack, int64_t k0, int nsteps, int lane) {
    const PackDesc pk = d.packs[p];
    const int J = pk.nrow;
    double* Vg = d.V + (size_t)pk.row0 * kWarp;
    double* Bs = d.Sg + pk.sg_off;
    double* Rs = d.Rg + pk.sg_off;
    double* Gm = d.Gm + pk.c_off;
    double* Em = d.Em + pk.c_off;
    double* gS = d.syn_g + (size_t)pk.syn_row0 * kWarp;
    double* mS = d.hh_m + (size_t)pk.hh_row0 * kWarp;
    double* hS = d.hh_h + (size_t)pk.hh_row0 * kWarp;
    double* nS = d.hh_n + (size_t)pk.hh_row0 * kWarp;
    const size_t e0 = (size_t)pk.row0 * kWarp + lane;
    const double* __restrict__ ca = d.ca + e0;
    const double* __restrict__ cb = d.cb + e0;
    const double* __restrict__ ck = d.ck + e0;
    const double* __restrict__ ce = d.ce + e0;
    const int32_t* __restrict__ fl = d.pslot + e0;
    const int32_t* __restrict__ cm_ = d.vmap + e0;
    double2* stk = stack;
    const int owner = p * kWarp + lane;
    int ev_i = d.ev_off[owner];
    const int ev_end = d.ev_off[owner + 1];
    const int s_lo = d.slot_lo[owner], s_hi = d.slot_hi[owner];
    const double dt = d.dt;
    int32_t late = 0;
    bool bad = false;

    // the lane's events of step `step` up to time t_max are added to the rows they target; the
    // constant parts of the lane's mechanism slots are restored and the terms of the next piece
    // summed when `terms`; gates and synapses advance over h when `update`
    auto mech = [&](double h, int step, double t_max, bool update, bool terms) {
        if (terms)
            for (int c = s_lo; c < s_hi; ++c) {
                Gm[c] = __ldg(d.cE + pk.c_off + c);
                Em[c] = __ldg(d.cB + pk.c_off + c);
            }
        while (step >= 0 && ev_i < ev_end && d.ev[ev_i].step_rel < step) { ++ev_i; late = 1; }
        for (int js = 0; js < pk.nsyn_row; ++js) {
            const size_t q = (size_t)(pk.syn_row0 + js) * kWarp + lane;
            const int sl = __ldg(d.syn_slot + q);
            if (sl < 0) continue;
            double g = gS[js * kWarp + lane];
            if (update) g *= (h == dt) ? __ldg(d.syn_decay + q) : exp_t(h * __ldg(d.syn_ntau + q));
            while (step >= 0 && ev_i < ev_end) {
                const EvRec r = d.ev[ev_i];
                if (r.step_rel != step || r.t > t_max || r.js != js) break;
                g += r.w;
                ++ev_i;
            }
            gS[js * kWarp + lane] = g;
            if (terms) {
                const int c = __ldg(d.syn_vs + q);
                Gm[c] += g;
                Em[c] = fma(g, __ldg(d.syn_e + q), Em[c]);
            }
        }
        for (int jh = 0; jh < pk.nhh_row; ++jh) {
            const size_t q = (size_t)(pk.hh_row0 + jh) * kWarp + lane;
            const int sl = __ldg(d.hh_slot + q);
            if (sl < 0) continue;
            const int idx = jh * kWarp + lane;
            double m = mS[idx], hh = hS[idx], n = nS[idx];
            if (update) {
                const Rates r = hh_rates(Vg[sl]);
                m = gate(m, r.am, r.bm, h);
                hh = gate(hh, r.ah, r.bh, h);
                n = gate(n, r.an, r.bn, h);
                mS[idx] = m;
                hS[idx] = hh;
                nS[idx] = n;
            }
            if (terms) {
                const int c = __ldg(d.hh_vs + q);
                const double n2 = n * n;
                const double gna = __ldg(d.hh_gna + q) * (m * m * m * hh);
                const double gk = __ldg(d.hh_gk + q) * (n2 * n2);
                Gm[c] += gna + gk;
                Em[c] += gna * kENa + gk * kEK;
            }
        }
    };

    mech(dt, 0, (double)k0 * dt, false, true);   // terms of the first piece; events at its start

    const int det = (lane < pk.ncell) ? ARB_IDX(d.det_slot[owner], pk.nrow * kWarp, d.ctl) : -1;
    const double thr = d.threshold;
    const int64_t probe_k0 = d.ctl->probe_k0, probe_max = d.ctl->probe_max;
    const bool probing = pk.npr > 0 && probe_max > 0;

    for (int s = 0; s < nsteps; ++s) {
        const int64_t k = k0 + s;
        const double t0 = (double)k * dt, t1 = (double)(k + 1) * dt;
        const bool last = (s + 1) == nsteps;
        double cur = t0;
        bool done = false;
        for (;;) {
            const bool act = !done;
            if (!__any_sync(0xffffffffu, act)) break;
            double next = t1;
            if (act && ev_i < ev_end) {
                const EvRec r = d.ev[ev_i];
                if (r.step_rel == s && r.t < t1) next = r.t;
            }
            // an uncut step is a step of dt (t1 - t0 can differ from dt in the last bit)
            const double h = (cur == t0 && next >= t1) ? dt : next - cur;
            const double scale = act ? dt / h : 1.0;         // c/h = (c/dt) * scale
            if (act)
                for (int js = 0; js < pk.nst_row; ++js) {
                    const size_t q = (size_t)(pk.st_row0 + js) * kWarp + lane;
                    const int c = __ldg(d.st_slot + q);
                    if (c >= 0 && __ldg(d.st_on + q) <= cur && cur < __ldg(d.st_off + q)) Em[c] += __ldg(d.st_amp + q);
                }
            const double v0 = (act && det >= 0) ? Vg[det] : 0.0;
            // forward elimination, leaves to root
            {
                int sp = 0;
                double yprev = 0.0, kprev = 0.0, eprev = 0.0;
                for (int j = 0; j < J; ++j) {
                    const size_t o = (size_t)j * kWarp;
                    const int c = __ldg(cm_ + o);
                    const int f = __ldg(fl + o);
                    const double K = __ldg(ck + o);
                    double A = __ldg(ca + o);
                    double E = c >= 0 ? Gm[c] : __ldg(ce + o);
                    const double B = c >= 0 ? Em[c] : __ldg(cb + o);
                    if (scale != 1.0) {
                        E = fma(A, scale - 1.0, E);
                        A *= scale;
                    }
                    const double V = Vg[j * kWarp + lane];
                    double dd = fma(-kprev, eprev, E);
                    double bb = fma(kprev, yprev, fma(A, V, B));
                    for (int qq = f & kFlagPopMask; qq > 0; --qq) {
                        const double2 c2 = stk[ARB_IDX(--sp, pk.stack, d.ctl) * kWarp + lane];
                        dd -= c2.x;
                        bb += c2.y;
                    }
                    const double r = rcp_nr(dd);
                    const double uu = r * bb;
                    const double ee = K * r;
                    if (act) {
                        Bs[j * kWarp + lane] = uu;
                        Rs[j * kWarp + lane] = ee;
                    }
                    const bool remote = (f & kFlagRemote) != 0;
                    if (remote && !(f & kFlagRoot)) stk[ARB_IDX(sp++, pk.stack, d.ctl) * kWarp + lane] = make_double2(K * ee, K * uu);
                    kprev = remote ? 0.0 : K;
                    eprev = ee;
                    yprev = uu;
                }
            }
            // back substitution, root to leaves
            {
                int sp = 0;
                double vnext = 0.0;
                for (int j = J - 1; j >= 0; --j) {
                    const int f = __ldg(fl + (size_t)j * kWarp);
                    const double U = Bs[j * kWarp + lane], X = Rs[j * kWarp + lane];
                    double vp;
                    if (f & kFlagRoot) vp = 0.0;
                    else if (f & kFlagRemote) vp = stk[ARB_IDX(--sp, pk.stack, d.ctl) * kWarp + lane].x;
                    else vp = vnext;
                    const double v = fma(X, vp, U);
                    for (int qq = f & kFlagPopMask; qq > 0; --qq) stk[ARB_IDX(sp++, pk.stack, d.ctl) * kWarp + lane] = make_double2(v, 0.0);
                    if (act) {
                        Vg[j * kWarp + lane] = v;
                        if (last) bad |= !isfinite(v);
                    }
                    vnext = v;
                }
            }
            // state over h; events at `next` (inside the step) or at the next step's start; terms
            if (act) {
                const bool end = next >= t1;
                if (!end) mech(h, s, next, true, true);
                else mech(h, last ? -1 : s + 1, t1, true, !last);
            }
            bool spk = false;
            double ts = 0.0;
            if (act && det >= 0) {
                const double v1 = Vg[det];
                if (v0 < thr && v1 >= thr) {
                    spk = true;
                    ts = __dadd_rn(cur, __dmul_rn(h, __ddiv_rn(__dsub_rn(thr, v0), __dsub_rn(v1, v0))));
                }
            }
            const unsigned ball = __ballot_sync(0xffffffffu, spk);
            if (ball) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd((unsigned long long*)&d.ctl->n_spikes, (unsigned long long)__popc(ball));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (spk) {
                    const int64_t pos = (int64_t)base + __popc(ball & ((1u << lane) - 1u));
                    if (pos < d.spike_cap) {
                        d.spk_gid[pos] = d.det_gid[owner];
                        d.spk_t[pos] = ts;
                    } else {
                        atomicOr(&d.ctl->status, kStSpikeOverflow);
                    }
                }
            }
            if (act) {
                cur = next;
                done = next >= t1;
            }
        }
        __syncwarp();
        if (probing) {
            const int64_t prow = k - probe_k0;
            if (prow >= 0 && prow < probe_max)
                for (int q = lane; q < pk.npr; q += kWarp)
                    d.trace[prow * d.n_probe + ARB_IDX(d.probe_col[pk.pr0 + q], d.n_probe, d.ctl)] =
                        Vg[ARB_IDX(d.probe_slot[pk.pr0 + q], pk.nrow * kWarp, d.ctl)];
        }
        __syncwarp();
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    const bool any_late = __any_sync(0xffffffffu, late != 0);
    if (lane == 0 && (any_bad || any_late))
        atomicOr(&d.ctl->status, (any_bad ? kStNonFinite : 0) | (any_late ? kStLateEvent : 0));
    __syncwarp();
}

// ------------------------------------------------------------------------------------------
// Streamed packs, implicit scheme: the rows of the forward elimination and of the back
// substitution stream through a per-warp ring of rows in shared memory, filled by asynchronous
// copies (cp.async) kRF rows (forward) or kRB rows (back substitution) ahead, so that the
// global-memory latency of a row is hidden behind the FP64 work of the rows before it without
// holding the prefetched rows in registers. Each lane copies, and later reads, only its own
// elements of a row, so no barrier is needed between the copy and the read.
//
// The diagonal and right-hand side of an entry without mechanisms are its constants (ce, cb);
// those of mechanism CVs sit in the compact slots Gm / Em, which the mechanism pass writes densely
// (slots numbered row by row within a pack, CVs with synapses first). The row's slots are two
// contiguous ranges (row_cs, row_cn: start and count), which the ring copies together with the
// row, and each entry's position in them (cpos) selects its terms. The forward sweep writes (u, e)
// of each entry as one 16-byte pair, which the back substitution streams back in reverse order.

// Ring depths and warps per CTA of the compiled variants of the ring kernel (see kStreamVariants).
template <int kRF, int kRB>
__host__ __device__ constexpr int ring_double2();
struct __align__(16) FwdRec {   // one lane's entry of a forward row: read back with three 16-byte loads
    double v, a, k, e, b;
    int32_t f;                     // flags
    int32_t cpos;                  // the entry's position in the row's gm / em, -1 none
};
struct FwdRow {                    // one row of the forward sweep, 32 lanes
    FwdRec rec[kWarp];
    double gm[kWarp], em[kWarp];   // the row's compact mechanism slots (synapse CVs, then others)
};
struct BwdRow {            // one row of the back substitution, 32 lanes
    double2 ue[kWarp];
    int32_t f[kWarp];
};
// shared memory of one warp's row ring, in double2 units: kRF forward rows or kRB back rows
template <int kRF, int kRB>
__host__ __device__ constexpr int ring_double2() {
    static_assert((kRF & (kRF - 1)) == 0 && (kRB & (kRB - 1)) == 0 && kRF >= 2 && kRB >= 2, "ring sizes");
    return (int)(((sizeof(FwdRow) * kRF > sizeof(BwdRow) * kRB ? sizeof(FwdRow) * kRF : sizeof(BwdRow) * kRB) + 15) / 16);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// Asynchronous global -> shared copies of one element; with valid = false nothing is read and
// the destination is zero-filled (src must still be a valid address).
__device__ __forceinline__ void cp_async_8(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_4(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <class MT, bool kShared, int kRF, int kRB>
__device__ void run_pack_stream_imp(const DevModel<MT>& d, int p, char* ring, double2* stack, int64_t k0, int nsteps,
                                    int lane) {
    const PackDesc pk = d.packs[p];
    const int J = pk.nrow;
    const size_t base = (size_t)pk.row0 * kWarp;
    double* Vg = d.V + base;
    double* Gm = d.Gm + pk.c_off;
    double* Em = d.Em + pk.c_off;
    double2* UE = d.UE + base;                 // forward result (u, e) per entry
    const double* ce_p = d.ce + base;
    const double* cb_p = d.cb + base;
    const double* ca_p = d.ca + base;
    const double* ck_p = d.ck + base;
    const int32_t* fl_p = d.pslot + base;
    const int32_t* cp_p = d.cpos + base;
    const int32_t* rcs = d.row_cs + pk.row0;   // per row: first synapse-CV slot | count << 24
    const int32_t* rcn = d.row_cn + pk.row0;   // per row: first other slot (from nsc) | count << 24
    MT* gS = d.syn_g + (size_t)pk.syn_row0 * kWarp;
    MT* mS = d.hh_m + (size_t)pk.hh_row0 * kWarp;
    MT* hS = d.hh_h + (size_t)pk.hh_row0 * kWarp;
    MT* nS = d.hh_n + (size_t)pk.hh_row0 * kWarp;
    FwdRow* fr = reinterpret_cast<FwdRow*>(ring);
    BwdRow* br = reinterpret_cast<BwdRow*>(ring);
    // hand-over stack (one cell per lane): three planes of [depth][32] -- the child's coupling K,
    // its e and its u -- so that a push is three stores and the parent's pop two multiply-adds
    double* stkK = (double*)stack;
    double* stkE = stkK + (size_t)pk.stack * kWarp;
    double* stkU = stkE + (size_t)pk.stack * kWarp;
    double* mbd = (double*)stack;              // mailbox (cells spread over lanes): [nmb] x (d, b),
    double* mbb = mbd + pk.nmb;                // and the published voltages over d in the back
    double* mbv = mbd;                         // substitution
    const int R = kShared ? pk.round_rows : 0;

    const int owner = p * kWarp + lane;
    int ev_i = d.ev_off[owner];
    const int ev_end = d.ev_off[owner + 1];
    int32_t late = 0;
    const double dt = d.dt;
    const MT dt_m = (MT)dt;
    stream_mech<MT, true>(d, pk, Gm, Em, Vg, gS, mS, hS, nS, lane, false, false, 0, true, ev_i, ev_end, late, dt_m);

    const int det = (lane < pk.ncell) ? ARB_IDX(d.det_slot[owner], pk.nrow * kWarp, d.ctl) : -1;
    const double thr = d.threshold;
    const int64_t probe_k0 = d.ctl->probe_k0, probe_max = d.ctl->probe_max;
    const bool probing = pk.npr > 0 && probe_max > 0;
    bool bad = false;

    // The slot ranges of 32 rows at a time are held one per lane (rows 32q .. 32q+31), the next
    // 32 fetched one chunk ahead.
    int q_cur = -1;
    int32_t cs_cur = 0, cn_cur = 0, cs_nxt = 0, cn_nxt = 0;
    auto chunk = [&](int q, int32_t& cs, int32_t& cn) {
        const int r = q * kWarp + lane;
        cs = r < J ? __ldg(rcs + r) : 0;
        cn = r < J ? __ldg(rcn + r) : 0;
    };
    // row j of the forward sweep into ring slot j mod kRF (rows past the end: zero fill), with
    // the compact slots of its mechanism CVs: lane l copies the l-th of them
    auto issue_f = [&](int j) {
        FwdRow& r = fr[j & (kRF - 1)];
        const bool in = j < J;
        const size_t o = (size_t)(in ? j : 0) * kWarp + lane;
        const int q = j >> 5;
        if (q != q_cur) {
            if (q == q_cur + 1 && q_cur >= 0) { cs_cur = cs_nxt; cn_cur = cn_nxt; }
            else chunk(q, cs_cur, cn_cur);
            chunk(q + 1, cs_nxt, cn_nxt);
            q_cur = q;
        }
        const uint32_t ws = (uint32_t)__shfl_sync(0xffffffffu, cs_cur, j & 31);
        const uint32_t wn = (uint32_t)__shfl_sync(0xffffffffu, cn_cur, j & 31);
        const int ns = (int)(ws >> 24), nn = (int)(wn >> 24);
        int slot = -1;
        if (lane < ns) slot = (int)(ws & 0xFFFFFF) + lane;
        else if (lane < ns + nn) slot = pk.nsc + (int)(wn & 0xFFFFFF) + (lane - ns);
        if (slot >= 0) slot = ARB_IDX(slot, pk.nvc, d.ctl);
        const bool mc = in && slot >= 0;
        FwdRec& e = r.rec[lane];
        cp_async_8(&e.v, Vg + o, in);
        cp_async_8(&e.a, ca_p + o, in);
        cp_async_8(&e.k, ck_p + o, in);
        cp_async_8(&e.e, ce_p + o, in);
        cp_async_8(&e.b, cb_p + o, in);
        cp_async_4(&e.f, fl_p + o, in);
        cp_async_4(&e.cpos, cp_p + o, in);
        cp_async_8(&r.gm[lane], mc ? Gm + slot : d.Gm, mc);
        cp_async_8(&r.em[lane], mc ? Em + slot : d.Em, mc);
        cp_async_commit();
    };
    // the i-th row of the back substitution (row J-1-i) into slot i mod kRB
    auto issue_b = [&](int i) {
        BwdRow& r = br[i & (kRB - 1)];
        const int j = J - 1 - i;
        const bool in = j >= 0;
        const size_t o = (size_t)(in ? j : 0) * kWarp + lane;
        cp_async_16(&r.ue[lane], UE + o, in);
        cp_async_4(&r.f[lane], fl_p + o, in);
        cp_async_commit();
    };

    for (int s = 0; s < nsteps; ++s) {
        const int64_t k = k0 + s;
        const double t = __dmul_rn((double)k, dt);
        const bool last = (s + 1) == nsteps;
        for (int js = 0; js < pk.nst_row; ++js) {
            const size_t q = (size_t)(pk.st_row0 + js) * kWarp + lane;
            const int c = __ldg(d.st_slot + q);
            if (c >= 0 && __ldg(d.st_on + q) <= t && t < __ldg(d.st_off + q)) Em[c] += __ldg(d.st_amp + q);
        }
        __syncwarp();
        const double v0 = det >= 0 ? Vg[det] : 0.0;

        // forward elimination, leaves to root
        {
            if (kShared) {
                // each slot starts from its parent's own diagonal and right-hand-side term; the
                // children add their contributions, and the parent takes the sums in their place
                const int32_t* me = d.mb_ent + pk.mb0;
                const int32_t* mc = d.mb_cs + pk.mb0;
#pragma unroll 4
                for (int i = lane; i < pk.nmb; i += kWarp) {
                    const int t = ARB_IDX(__ldg(me + i), J * kWarp, d.ctl);
                    const int c = __ldg(mc + i);
                    const int cc = c < 0 ? -1 : ARB_IDX(c, pk.nvc, d.ctl);
                    mbd[i] = cc >= 0 ? Gm[cc] : __ldg(ce_p + t);
                    mbb[i] = cc >= 0 ? Em[cc] : __ldg(cb_p + t);
                }
                __syncwarp();
            }
            q_cur = -1;
#pragma unroll
            for (int u = 0; u < kRF; ++u) issue_f(u);
            int sp = 0, left = R;
            int acc = -1;   // cells over lanes: the slot the previous row's hand-over is still added to
            double yprev = 0.0, kprev = 0.0, eprev = 0.0;
            for (int j = 0; j < J; ++j) {
                cp_async_wait<kRF - 1>();                // row j has landed (this lane's copies)
                __syncwarp();                            // ... and every lane's (compact slots)
                const FwdRow& r = fr[j & (kRF - 1)];
                const FwdRec x = r.rec[lane];
                const int cp = x.cpos < 0 ? -1 : ARB_IDX(x.cpos, kWarp, d.ctl);
                const double V = x.v, A = x.a, K = x.k;
                double E = cp >= 0 ? r.gm[cp] : x.e;
                double Bc = cp >= 0 ? r.em[cp] : x.b;
                const int f = x.f;
                __syncwarp();                            // slot read by every lane before refilling it
                issue_f(j + kRF);
                if (kShared && R > 0) {
                    if (left == 0) { __syncwarp(); left = R; }
                    --left;
                }
                const int mb_in = kShared ? (int)((unsigned)f >> kMbInShift) : kMbNone;
                const int mb_out = kShared ? ((f >> kMbOutShift) & kMbNone) : kMbNone;
                double dd, bb;
                if (kShared) {
                    // A row after a hand-over has no child in registers: its two multiply-adds
                    // add the previous row's (K e, K u) into that parent's slot instead, so a
                    // hand-over costs no FP64 instruction of its own in either row.
                    if (mb_in != kMbNone) {
                        const int o = ARB_IDX(mb_in, pk.nmb, d.ctl);
                        E = mbd[o];
                        Bc = mbb[o];
                    }
                    const double bz = fma(A, V, Bc);
                    const double zd = acc >= 0 ? mbd[acc] : E;
                    const double zb = acc >= 0 ? mbb[acc] : bz;
                    const double fd = fma(-kprev, eprev, zd);
                    const double fb = fma(kprev, yprev, zb);
                    if (acc >= 0) {
                        mbd[acc] = fd;
                        mbb[acc] = fb;
                    }
                    dd = acc >= 0 ? E : fd;
                    bb = acc >= 0 ? bz : fb;
                } else {
                    dd = fma(-kprev, eprev, E);
                    bb = fma(kprev, yprev, fma(A, V, Bc));
                    for (int q = f & kFlagPopMask; q > 0; --q) {
                        const int o = ARB_IDX(--sp, pk.stack, d.ctl) * kWarp + lane;
                        const double kc = stkK[o];
                        dd = fma(-kc, stkE[o], dd);
                        bb = fma(kc, stkU[o], bb);
                    }
                }
                const double rr = rcp_nr(dd);
                const double uu = rr * bb;
                const double ee = K * rr;
                UE[(size_t)j * kWarp + lane] = make_double2(uu, ee);
                const bool remote = (f & kFlagRemote) != 0;
                if (kShared) {
                    acc = (remote && !(f & kFlagRoot)) ? ARB_IDX(mb_out, pk.nmb, d.ctl) : -1;
                    kprev = K;   // a root's (and padding's) coupling is 0
                } else {
                    if (remote && !(f & kFlagRoot)) {
                        const int o = ARB_IDX(sp++, pk.stack, d.ctl) * kWarp + lane;
                        stkK[o] = K;
                        stkE[o] = ee;
                        stkU[o] = uu;
                    }
                    kprev = remote ? 0.0 : K;
                }
                eprev = ee;
                yprev = uu;
            }
            cp_async_wait<0>();                          // the zero-filled tail copies too
        }
        __syncwarp();
        // back substitution, root to leaves (preorder)
        {
#pragma unroll
            for (int u = 0; u < kRB - 1; ++u) issue_b(u);
            int sp = 0;
            double vnext = 0.0;
            int left = kShared ? ((R > 0) ? ((J - 1) % R) + 1 : 0) : 0;
            for (int i = 0; i < J; ++i) {
                const int j = J - 1 - i;
                issue_b(i + kRB - 1);
                cp_async_wait<kRB - 1>();
                const BwdRow& r = br[i & (kRB - 1)];
                const double2 ue = r.ue[lane];
                const int f = r.f[lane];
                if (kShared && R > 0) {
                    if (left == 0) { __syncwarp(); left = R; }
                    --left;
                }
                double vp;
                if (f & kFlagRoot) vp = 0.0;
                else if (f & kFlagRemote) vp = kShared ? mbv[ARB_IDX((f >> kMbOutShift) & kMbNone, pk.nmb, d.ctl)] : stkK[ARB_IDX(--sp, pk.stack, d.ctl) * kWarp + lane];
                else vp = vnext;
                const double v = fma(ue.y, vp, ue.x);
                if (kShared) {
                    const int mb_in = (int)((unsigned)f >> kMbInShift);
                    if (mb_in != kMbNone) mbv[ARB_IDX(mb_in, pk.nmb, d.ctl)] = v;
                } else {
                    for (int q = f & kFlagPopMask; q > 0; --q) stkK[ARB_IDX(sp++, pk.stack, d.ctl) * kWarp + lane] = v;
                }
                Vg[(size_t)j * kWarp + lane] = v;
                if (last) bad |= !isfinite(v);
                vnext = v;
            }
            cp_async_wait<0>();
        }
        __syncwarp();

        // state updates with V(t_{k+1}); terms of the next step
        stream_mech<MT, true>(d, pk, Gm, Em, Vg, gS, mS, hS, nS, lane, true, true, last ? -1 : s + 1, !last, ev_i,
                              ev_end, late, dt_m);

        bool spk = false;
        double ts = 0.0;
        if (det >= 0) {
            const double v1 = Vg[det];
            if (v0 < thr && v1 >= thr) {
                spk = true;
                ts = __dadd_rn(t, __dmul_rn(dt, __ddiv_rn(__dsub_rn(thr, v0), __dsub_rn(v1, v0))));
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, spk);
        if (ball) {
            unsigned long long b0 = 0;
            if (lane == 0) b0 = atomicAdd((unsigned long long*)&d.ctl->n_spikes, (unsigned long long)__popc(ball));
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            if (spk) {
                const int64_t pos = (int64_t)b0 + __popc(ball & ((1u << lane) - 1u));
                if (pos < d.spike_cap) {
                    d.spk_gid[pos] = d.det_gid[owner];
                    d.spk_t[pos] = ts;
                } else {
                    atomicOr(&d.ctl->status, kStSpikeOverflow);
                }
            }
        }
        if (probing) {
            const int64_t prow = k - probe_k0;
            if (prow >= 0 && prow < probe_max)
                for (int q = lane; q < pk.npr; q += kWarp)
                    d.trace[prow * d.n_probe + ARB_IDX(d.probe_col[pk.pr0 + q], d.n_probe, d.ctl)] =
                        Vg[ARB_IDX(d.probe_slot[pk.pr0 + q], pk.nrow * kWarp, d.ctl)];
        }
        __syncwarp();
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    const bool any_late = __any_sync(0xffffffffu, late != 0);
    if (lane == 0 && (any_bad || any_late))
        atomicOr(&d.ctl->status, (any_bad ? kStNonFinite : 0) | (any_late ? kStLateEvent : 0));
    __syncwarp();
}

// The streamed epoch kernels: a persistent grid of one CTA per SM whose warps take packs from
// the work counter. The implicit scheme with step-start events runs the row-ring path, compiled
// for several warp counts and ring depths (kStreamVariants, chosen at arb_create); the explicit
// scheme and exact event times run their own kernels (16 warps, no ring).
template <class MT, int kW, int kRF, int kRB>
__global__ void __launch_bounds__(kW * kWarp, 1) arb_stream_ring_kernel(DevModel<MT> d, int warp_smem_double2) {
    extern __shared__ double2 stk_smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    constexpr int ring = ring_double2<kRF, kRB>();
    double2* wbase = stk_smem + (size_t)wid * (size_t)(warp_smem_double2 + ring);   // row ring, then
    double2* stack = wbase + ring;                                                   // stack / mailbox
    const int64_t k0 = d.ctl->k0;
    const int nsteps = (int)(d.ctl->k1 - k0);
    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(&d.ctl->pack_next, 1);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= d.n_packs) break;
        if (d.packs[p].round_rows > 0) run_pack_stream_imp<MT, true, kRF, kRB>(d, p, (char*)wbase, stack, k0, nsteps, lane);
        else run_pack_stream_imp<MT, false, kRF, kRB>(d, p, (char*)wbase, stack, k0, nsteps, lane);
    }
}

template <class MT>
__global__ void __launch_bounds__(kStreamWarps * kWarp, 1) arb_stream_kernel(DevModel<MT> d, int warp_smem_double2) {
    extern __shared__ double2 stk_smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    double2* stack = stk_smem + (size_t)wid * warp_smem_double2;
    const int64_t k0 = d.ctl->k0;
    const int nsteps = (int)(d.ctl->k1 - k0);
    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(&d.ctl->pack_next, 1);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= d.n_packs) break;
        if (d.packs[p].round_rows > 0) run_pack_stream<MT, false, true>(d, p, stack, k0, nsteps, lane);
        else run_pack_stream<MT, false, false>(d, p, stack, k0, nsteps, lane);
    }
}

__global__ void __launch_bounds__(kStreamWarps * kWarp, 1) arb_stream_exact_kernel(DevModel<double> d, int warp_smem_double2) {
    extern __shared__ double2 stk_smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    double2* stack = stk_smem + (size_t)wid * warp_smem_double2;
    const int64_t k0 = d.ctl->k0;
    const int nsteps = (int)(d.ctl->k1 - k0);
    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(&d.ctl->pack_next, 1);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= d.n_packs) break;
        run_pack_exact(d, p, stack, k0, nsteps, lane);
    }
}

// Compiled variants of the row-ring kernel: warps per CTA, forward ring rows, back ring rows.
struct StreamVariant { int warps, rf, rb; };
constexpr StreamVariant kStreamVariants[] = {{16, 2, 4}, {12, 4, 8}, {20, 2, 4}, {12, 2, 4}, {24, 2, 4}};
constexpr int kNumStreamVariants = (int)(sizeof(kStreamVariants) / sizeof(kStreamVariants[0]));

int stream_variant_count() { return kNumStreamVariants; }
void stream_variant_info(int v, int* warps, int* rf, int* rb) {
    *warps = kStreamVariants[v].warps;
    *rf = kStreamVariants[v].rf;
    *rb = kStreamVariants[v].rb;
}

// Warps per CTA and shared memory per warp (double2 units: row ring plus stack or mailbox) of the
// kernel that runs a streamed plan: the ring variant v for the implicit scheme with step-start
// events, else 16 warps without a ring.
void stream_variant_shape(bool ring_path, int v, int warp_smem_double2, int* warps, int* per_warp_double2) {
    int w = kStreamWarps, ring = 0;
    if (ring_path && v >= 0 && v < kNumStreamVariants) {
        const StreamVariant sv = kStreamVariants[v];
        w = sv.warps;
        switch (v) {
            case 1: ring = ring_double2<4, 8>(); break;
            default: ring = ring_double2<2, 4>(); break;
        }
    }
    if (warps) *warps = w;
    if (per_warp_double2) *per_warp_double2 = warp_smem_double2 + ring;
}

template <class MT>
static const void* stream_fn(int mode, int v) {
    if (mode == 1) {
        switch (v) {
            case 0: return (const void*)arb_stream_ring_kernel<MT, 16, 2, 4>;
            case 1: return (const void*)arb_stream_ring_kernel<MT, 12, 4, 8>;
            case 2: return (const void*)arb_stream_ring_kernel<MT, 20, 2, 4>;
            case 3: return (const void*)arb_stream_ring_kernel<MT, 12, 2, 4>;
            default: return (const void*)arb_stream_ring_kernel<MT, 24, 2, 4>;
        }
    }
    if constexpr (std::is_same<MT, double>::value)
        if (mode == 2) return (const void*)arb_stream_exact_kernel;
    return (const void*)arb_stream_kernel<MT>;
}

// mode: 0 explicit scheme, 1 implicit row-ring path (variant v), 2 exact event times (FP64).
// warp_smem_double2: each warp's stack or mailbox; the ring kernel adds its row ring.
template <class MT>
cudaError_t launch_stream(const DevModel<MT>& d, int mode, int v, int grid, int warps_per_cta, int warp_smem_double2,
                          cudaStream_t s) {
    int w = 0, pw = 0;
    stream_variant_shape(mode == 1, v, warp_smem_double2, &w, &pw);
    const size_t smem = (size_t)warps_per_cta * (size_t)pw * sizeof(double2);
    DevModel<MT> dd = d;
    int ws = warp_smem_double2;
    void* args[] = {(void*)&dd, (void*)&ws};
    return cudaLaunchKernel(stream_fn<MT>(mode, v), dim3(grid), dim3(warps_per_cta * kWarp), args, smem, s);
}

template <class MT>
cudaError_t stream_occupancy(int mode, int v, int warps_per_cta, int warp_smem_double2, int* blocks_per_sm) {
    int w = 0, pw = 0;
    stream_variant_shape(mode == 1, v, warp_smem_double2, &w, &pw);
    const size_t smem = (size_t)warps_per_cta * (size_t)pw * sizeof(double2);
    const void* fn = stream_fn<MT>(mode, v);
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, warps_per_cta * kWarp, smem);
}

template cudaError_t launch_stream<double>(const DevModel<double>&, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_stream<float>(const DevModel<float>&, int, int, int, int, int, cudaStream_t);
template cudaError_t stream_occupancy<double>(int, int, int, int, int*);
template cudaError_t stream_occupancy<float>(int, int, int, int, int*);

// ------------------------------------------------------------------------------------------
// Event delivery lists (the "enqueue" and "merge" of Sec. "Implementation": each spike's
// events go to per-cell queues merged with pending events). Here every owner lane gets the
// events of its synapses that fall in the epoch, in a fixed order.



// Preparation of one epoch's delivery lists: [kp0, kp1) with kp0 the first step whose lists
// are not built yet. It reads only pending pools and external events, so with two list buffers
// it can run while the previous epoch integrates.
__global__ void k_prep_begin(EvArgs a) {
    Ctl* c = a.ctl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t k1 = min(c->kp0 + (int64_t)a.epoch_steps, c->k_end);
        c->kp1 = k1;
        int64_t lo = c->ext_lo, hi = c->n_ext;
        while (lo < hi) {                         // first external event at or after k1
            const int64_t mid = (lo + hi) / 2;
            if (a.ext_step[mid] < k1) lo = mid + 1; else hi = mid;
        }
        c->ext_hi = lo;
        c->pool_n64[c->parity ^ 1] = 0;
        c->n_due = 0;
    }
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.n_owner; o += gridDim.x * blockDim.x) a.counts[o] = 0;
}

__global__ void k_prep_end(Ctl* c, int64_t pool_cap, int32_t slot_mask) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c->kp0 = c->kp1;
        c->ext_lo = c->ext_hi;
        const int np = c->parity ^ 1;
        if (c->pool_n64[np] > pool_cap) c->pool_n64[np] = pool_cap;
        c->parity = np;
        c->prep_slot ^= slot_mask;
    }
}

// Integration epoch [k0, k1): bounds and the work counter before, the epoch's spike range
// (for the spike walk) and the next epoch's start after.
__global__ void k_int_begin(Ctl* c, int32_t epoch_steps) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c->k1 = min(c->k0 + (int64_t)epoch_steps, c->k_end);
        c->pack_next = 0;
    }
}

__global__ void k_int_end(Ctl* c, int64_t spike_cap) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int64_t hi = min(c->n_spikes, spike_cap);
        c->xr_lo[c->xw] = c->spk_mark;
        c->xr_hi[c->xw] = hi;
        c->xw ^= 1;
        c->spk_mark = hi;
        c->k0 = c->k1;
    }
}

template <bool kScatter>
__global__ void k_ev_walk(EvArgs a) {
    Ctl* c = a.ctl;
    const int par = c->parity;
    const int64_t k0 = c->kp0, k1 = c->kp1;
    const int64_t n_pool = min((int64_t)c->pool_n64[par], a.pool_cap);
    const int slot = c->prep_slot;
    const int32_t* off = a.off + (size_t)slot * (a.n_owner + 1);
    const int64_t rec_end = (int64_t)(slot + 1) * a.bucket_cap;
    if (!kScatter) {
        // pending events not due in this epoch move to the other pool: one atomic per warp
        const int lane = threadIdx.x & 31;
        const PendEv* src = par ? a.pool[1] : a.pool[0];
        PendEv* dst = par ? a.pool[0] : a.pool[1];
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        const int64_t n_round = (n_pool + 31) / 32 * 32;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
            PendEv e;
            bool keep = false;
            if (i < n_pool) {
                e = src[i];
                keep = e.step >= k1;
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (m == 0) continue;
            long long base = 0;
            if (lane == 0) base = (long long)atomicAdd((unsigned long long*)&c->pool_n64[par ^ 1], (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (keep) {
                const int64_t pos = base + __popc(m & ((1u << lane) - 1u));
                if (pos < a.pool_cap) dst[pos] = e;
                else atomicOr(&c->status, kStPoolOverflow);
            }
        }
    }
    const int64_t n_ext = c->ext_hi - c->ext_lo;
    const int64_t total = n_pool + n_ext;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        double t, w;
        int64_t step;
        int32_t syn, src, idx;
        if (i < n_pool) {
            const PendEv e = (par ? a.pool[1] : a.pool[0])[i];
            if (e.step >= k1) continue;   // not due yet: kept by the pass below
            t = e.t; w = e.w; step = e.step; syn = e.syn; src = e.src; idx = e.idx;
        } else {
            const int64_t x = c->ext_lo + (i - n_pool);
            t = a.ext_t[x]; w = a.ext_w[x]; step = a.ext_step[x]; syn = a.ext_syn[x]; src = -1; idx = a.ext_idx[x];
        }
        if (step < k0) { atomicOr(&c->status, kStLateEvent); step = k0; }
        syn = ARB_IDX(syn, a.n_syn, c);
        const int owner = ARB_IDX(a.syn_owner[syn], a.n_owner, c);
        if (!kScatter) {
            atomicAdd(&a.counts[owner], 1);
        } else {
            const int64_t pos = (int64_t)off[owner] + atomicAdd(&a.counts[owner], 1);
            if (pos < rec_end) {
                EvRec r;
                r.t = t; r.w = w; r.step_rel = (int32_t)(step - k0); r.js = a.syn_js[syn]; r.src = src; r.idx = idx;
                a.rec[pos] = r;
            }
        }
    }
}

// Exclusive scan of the per-owner counts (one block), then the counts are reset to serve as
// scatter cursors.
__global__ void __launch_bounds__(1024) k_ev_scan(EvArgs a) {
    __shared__ int64_t part[1024];
    const int n = a.n_owner;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    int64_t s = 0;
    for (int o = lo; o < hi; ++o) s += a.counts[o];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int sh = 1; sh < (int)blockDim.x; sh <<= 1) {
        const int64_t v = threadIdx.x >= (unsigned)sh ? part[threadIdx.x - sh] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    const int slot = a.ctl->prep_slot;
    int32_t* off = a.off + (size_t)slot * (n + 1);
    const int64_t base = (int64_t)slot * a.bucket_cap;
    int64_t run = part[threadIdx.x] - s;
    for (int o = lo; o < hi; ++o) {
        const int cnt = a.counts[o];
        off[o] = (int32_t)(base + min(run, a.bucket_cap));
        run += cnt;
        a.counts[o] = 0;
    }
    if (threadIdx.x == blockDim.x - 1) {
        off[n] = (int32_t)(base + min(part[blockDim.x - 1], a.bucket_cap));
        a.ctl->n_due = (int32_t)min(part[blockDim.x - 1], (int64_t)INT32_MAX);
        if (part[blockDim.x - 1] > a.bucket_cap) atomicOr(&a.ctl->status, kStBucketOverflow);
    }
}

__device__ __forceinline__ bool ev_less(const EvRec& x, const EvRec& y, bool time_major) {
    if (x.step_rel != y.step_rel) return x.step_rel < y.step_rel;
    if (time_major && x.t != y.t) return x.t < y.t;
    if (x.js != y.js) return x.js < y.js;
    if (x.t != y.t) return x.t < y.t;
    if (x.src != y.src) return x.src < y.src;
    return x.idx < y.idx;
}

// Per-owner sort of the epoch's events by (step, synapse row, t, source, index), which is a
// total order. Short lists (a few events per lane and epoch on the batched workload) are sorted
// here by one thread each with an insertion sort; long ones are left to k_ev_sort_long.
constexpr int kEvShort = 48;
__global__ void k_ev_sort(EvArgs a) {
    const int slot = a.ctl->prep_slot;
    const int32_t* off = a.off + (size_t)slot * (a.n_owner + 1);
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.n_owner; o += gridDim.x * blockDim.x) {
        const int lo = off[o], hi = off[o + 1];
        const int n = hi - lo;
        if (n > kEvShort) continue;
        EvRec* r = a.rec + lo;
        for (int i = 1; i < n; ++i) {
            const EvRec x = r[i];
            int j = i - 1;
            while (j >= 0 && ev_less(x, r[j], a.time_major)) { r[j + 1] = r[j]; --j; }
            r[j + 1] = x;
        }
    }
}

// Long per-owner lists (dense networks: thousands of events per lane and epoch), one block per
// list: the records are copied to a scratch buffer, counting-sorted by step (the block's threads
// histogram and scatter record indices in shared memory), each step's bucket is
// insertion-sorted by the full key, and the records are gathered back in order. Lists that do
// not fit are heap-sorted in place by one thread.
constexpr int kEvLongMax = 16384;      // indices staged per list
constexpr int kEvLongSteps = 4096;     // histogram bins (epoch steps) in shared memory
__global__ void __launch_bounds__(256) k_ev_sort_long(EvArgs a) {
    extern __shared__ int ev_smem[];
    int* sidx = ev_smem;                                           // [kEvLongMax]
    int* hist = sidx + kEvLongMax;                                 // [kEvLongSteps + 1]
    int* cur = hist + kEvLongSteps + 1;                            // [kEvLongSteps]
    const int tid = threadIdx.x, nt = blockDim.x;
    const int E = a.epoch_steps;
    const int slot = a.ctl->prep_slot;
    const int32_t* off = a.off + (size_t)slot * (a.n_owner + 1);
    const int64_t base = (int64_t)slot * a.bucket_cap;
    for (int o = blockIdx.x; o < a.n_owner; o += gridDim.x) {
        const int lo = off[o], hi = off[o + 1];
        const int n = hi - lo;
        if (n <= kEvShort) continue;                               // uniform across the block
        EvRec* r = a.rec + lo;
        EvRec* t = a.tmp + (lo - base);
        if (n > kEvLongMax || E > kEvLongSteps) {
            if (tid == 0) {
                auto sift = [&](int root, int end) {               // max-heap on [0, end)
                    const EvRec x = r[root];
                    int i = root;
                    for (;;) {
                        int ch = 2 * i + 1;
                        if (ch >= end) break;
                        if (ch + 1 < end && ev_less(r[ch], r[ch + 1], a.time_major)) ++ch;
                        if (!ev_less(x, r[ch], a.time_major)) break;
                        r[i] = r[ch];
                        i = ch;
                    }
                    r[i] = x;
                };
                for (int i = n / 2 - 1; i >= 0; --i) sift(i, n);
                for (int end = n - 1; end > 0; --end) {
                    const EvRec x = r[0];
                    r[0] = r[end];
                    r[end] = x;
                    sift(0, end);
                }
            }
            __syncthreads();
            continue;
        }
        for (int i = tid; i <= E; i += nt) hist[i] = 0;
        __syncthreads();
        for (int i = tid; i < n; i += nt) {
            const EvRec x = r[i];
            t[i] = x;
            atomicAdd(&hist[min(max(x.step_rel, 0), E - 1) + 1], 1);
        }
        __syncthreads();
        if (tid < 32) {                                            // bucket starts: warp scan in chunks
            int carry = 0;
            for (int base = 1; base <= E; base += 32) {
                const int i = base + tid;
                int v = i <= E ? hist[i] : 0;
                for (int sh = 1; sh < 32; sh <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, v, sh);
                    if (tid >= sh) v += u;
                }
                if (i <= E) hist[i] = v + carry;
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
        }
        __syncthreads();
        for (int i = tid; i < E; i += nt) cur[i] = hist[i];
        __syncthreads();
        for (int i = tid; i < n; i += nt) sidx[atomicAdd(&cur[min(max(t[i].step_rel, 0), E - 1)], 1)] = i;
        __syncthreads();
        for (int b = tid; b < E; b += nt) {                        // order inside each step
            const int b0 = hist[b], b1 = hist[b + 1];
            for (int i = b0 + 1; i < b1; ++i) {
                const int x = sidx[i];
                const EvRec xr = t[x];
                int j = i - 1;
                while (j >= b0 && ev_less(xr, t[sidx[j]], a.time_major)) { sidx[j + 1] = sidx[j]; --j; }
                sidx[j + 1] = x;
            }
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt) r[i] = t[sidx[i]];
        __syncthreads();
    }
}



// Spike exchange on one GPU: every spike of an integrated epoch is walked against the
// connections of its source (the connection table of Sec. "Implementation", grouped by source
// here), and each resulting event waits in the pending pool for the epoch that contains its
// step. Its spike range was recorded when that epoch ended, so the walk may run while the next
// epoch integrates and records further spikes. In a dry run (Sec. "Scalability") the global
// spike list holds every local spike once per virtual rank r, as gid + r * n_cells.
__global__ void k_spike_expand(SpkArgs a) {
    // per warp iteration, one spike (few spikes: every warp gets one, and a spike's fan-out is
    // written by all 32 lanes) or 32 spikes with one out-list lookup per lane (many spikes, as
    // in a dry run, where most have no local connection); then the warp takes the spikes with
    // connections one at a time: lane 0 reserves the whole fan-out in the pending pool with one
    // atomic, the lanes write its events
    Ctl* c = a.ctl;
    const int par = c->parity;
    const int64_t k_first = c->kp0;               // earliest step whose lists are not built yet
    const int xr = c->xr;
    const int64_t lo = c->xr_lo[xr], n_local = c->xr_hi[xr] - lo;
    const int64_t n_glob = n_local * a.dry_ranks;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    PendEv* out = par ? a.pool[1] : a.pool[0];
    const int per = n_glob >= nwarps * 32 ? 32 : 1;     // spikes per warp iteration
    for (int64_t i0 = warp * per; i0 < n_glob; i0 += nwarps * per) {
        const int64_t i = i0 + lane;
        int32_t my_gid = 0;
        double my_ts = 0.0;
        int64_t my_q0 = 0, my_deg = 0;
        if (lane < per && i < n_glob) {
            const int64_t r = i / n_local, j = lo + (i - r * n_local);
            my_gid = (int32_t)ARB_IDX64(a.spk_gid[ARB_IDX64(j, a.spike_cap, c)] + r * a.n_cells, a.n_cells * a.dry_ranks, c);
            my_ts = a.spk_t[j];
            my_q0 = a.out_ptr[my_gid];
            my_deg = a.out_ptr[my_gid + 1] - my_q0;
        }
        unsigned todo = __ballot_sync(0xffffffffu, my_deg > 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int32_t gid = __shfl_sync(0xffffffffu, my_gid, src);
            const double ts = __shfl_sync(0xffffffffu, my_ts, src);
            const int64_t q0 = __shfl_sync(0xffffffffu, my_q0, src);
            const int64_t deg = __shfl_sync(0xffffffffu, my_deg, src);
            int64_t base = 0;
            if (lane == 0) base = atomicAdd((unsigned long long*)&c->pool_n64[par], (unsigned long long)deg);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base + deg > a.pool_cap && lane == 0) atomicOr(&c->status, kStPoolOverflow);
            for (int64_t k = lane; k < deg; k += 32) {
                const int64_t q = q0 + k;
                PendEv e;
                e.t = __dadd_rn(ts, a.out_delay[q]);
                int64_t step = event_step(e.t, a.dt, a.exact != 0);
                if (step < k_first) step = k_first;
                e.step = step;
                e.w = a.out_w[q];
                e.syn = a.out_syn[q];
                e.src = gid;
                e.idx = a.out_idx[q];
                e.pad = 0;
                if (base + k < a.pool_cap) out[base + k] = e;
            }
        }
    }
}

__global__ void k_expand_end(Ctl* c) {
    if (threadIdx.x == 0 && blockIdx.x == 0) c->xr ^= 1;
}

// ------------------------------------------------------------------------------------------
// Layout conversions between the model's CV order and the tile layout.

template <class T>
__global__ void k_gather(double* out, const T* src, const int64_t* idx, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = idx[i] >= 0 ? (double)src[idx[i]] : 0.0;
}

template <class T>
__global__ void k_scatter(T* dst, const double* src, const int64_t* idx, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (idx[i] >= 0) dst[idx[i]] = (T)src[i];
}

// ------------------------------------------------------------------------------------------
// Launch wrappers used by the host runtime.

template <class MT>
cudaError_t launch_epoch(const DevModel<MT>& d, bool implicit, int grid, int warps_per_cta, int tile_doubles, cudaStream_t s) {
    // the shared-memory limit was raised once by epoch_occupancy (not a stream operation,
    // so it stays out of graph capture)
    const size_t smem = (size_t)warps_per_cta * (size_t)tile_doubles * sizeof(double);
    if (implicit) arb_epoch_kernel<MT, true><<<grid, warps_per_cta * kWarp, smem, s>>>(d, tile_doubles);
    else arb_epoch_kernel<MT, false><<<grid, warps_per_cta * kWarp, smem, s>>>(d, tile_doubles);
    return cudaGetLastError();
}

template <class MT>
cudaError_t epoch_occupancy(bool implicit, int warps_per_cta, int tile_doubles, int* blocks_per_sm) {
    const size_t smem = (size_t)warps_per_cta * (size_t)tile_doubles * sizeof(double);
    auto fn = implicit ? arb_epoch_kernel<MT, true> : arb_epoch_kernel<MT, false>;
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, warps_per_cta * kWarp, smem);
}

template cudaError_t launch_epoch<double>(const DevModel<double>&, bool, int, int, int, cudaStream_t);
template cudaError_t launch_epoch<float>(const DevModel<float>&, bool, int, int, int, cudaStream_t);
template cudaError_t epoch_occupancy<double>(bool, int, int, int*);
template cudaError_t epoch_occupancy<float>(bool, int, int, int*);

size_t ev_sort_long_smem() { return sizeof(int) * (kEvLongMax + 2 * kEvLongSteps + 1); }

// Kernel attributes the event launches need, set once before they are captured.
cudaError_t events_prepare() {
    return cudaFuncSetAttribute(k_ev_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ev_sort_long_smem());
}

cudaError_t launch_events_pre(const EvArgs& a, int n_sm, cudaStream_t s) {
    const int owner_blocks = max(1, min(4 * n_sm, (a.n_owner + 255) / 256));
    k_prep_begin<<<owner_blocks, 256, 0, s>>>(a);
    k_ev_walk<false><<<2 * n_sm, 256, 0, s>>>(a);
    k_ev_scan<<<1, 1024, 0, s>>>(a);
    k_ev_walk<true><<<2 * n_sm, 256, 0, s>>>(a);
    k_ev_sort<<<owner_blocks, 256, 0, s>>>(a);
    k_ev_sort_long<<<4 * n_sm, 256, ev_sort_long_smem(), s>>>(a);
    k_prep_end<<<1, 32, 0, s>>>(a.ctl, a.pool_cap, a.slot_mask);
    return cudaGetLastError();
}

cudaError_t launch_events_post(const SpkArgs& a, int n_sm, cudaStream_t s) {
    k_spike_expand<<<4 * n_sm, 256, 0, s>>>(a);
    k_expand_end<<<1, 32, 0, s>>>(a.ctl);
    return cudaGetLastError();
}

cudaError_t launch_int_begin(Ctl* c, int32_t epoch_steps, cudaStream_t s) {
    k_int_begin<<<1, 32, 0, s>>>(c, epoch_steps);
    return cudaGetLastError();
}

cudaError_t launch_int_end(Ctl* c, int64_t spike_cap, cudaStream_t s) {
    k_int_end<<<1, 32, 0, s>>>(c, spike_cap);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_gather(double* out, const T* src, const int64_t* idx, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_gather<T><<<blocks, 256, 0, s>>>(out, src, idx, n);
    return cudaGetLastError();
}
template <class T>
cudaError_t launch_scatter(T* dst, const double* src, const int64_t* idx, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_scatter<T><<<blocks, 256, 0, s>>>(dst, src, idx, n);
    return cudaGetLastError();
}
template cudaError_t launch_gather<double>(double*, const double*, const int64_t*, int64_t, cudaStream_t);
template cudaError_t launch_gather<float>(double*, const float*, const int64_t*, int64_t, cudaStream_t);
template cudaError_t launch_scatter<double>(double*, const double*, const int64_t*, int64_t, cudaStream_t);
template cudaError_t launch_scatter<float>(float*, const double*, const int64_t*, int64_t, cudaStream_t);

}  // namespace arbk
