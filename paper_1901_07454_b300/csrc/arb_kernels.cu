// sm_103a kernels of the batched cable-equation stepper.
//
// One epoch (Sec. "Implementation", "Simulation workflow": cells advance independently for
// an interval no longer than the minimum delay) is this fixed sequence of launches:
//   k_epoch_begin -> k_ev_count -> k_ev_scan -> k_ev_scatter -> k_ev_sort   (event delivery lists)
//   arb_epoch_kernel                                                         (all time steps)
//   k_spike_expand -> k_epoch_end                                            (spike exchange)
// Per-epoch values live in the device control block, so the sequence is captured once as a
// CUDA graph and replayed for every epoch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "arb_internal.h"

namespace arbk {

// ------------------------------------------------------------------------------------------
// Hodgkin-Huxley rates (1/ms) and exact gate update at frozen V, in the precision MT.
// The model (classic squid axon at 6.3 degC) is the one named by the paper's benchmark
// (Sec. "Benchmarks", "Models": Hodgkin-Huxley soma, passive dendrites).

__device__ __forceinline__ double exprelr_d(double x) { return x == 0.0 ? 1.0 : x / expm1(x); }
__device__ __forceinline__ float exprelr_f(float x) { return x == 0.0f ? 1.0f : x / expm1f(x); }

struct Rates { double am, bm, ah, bh, an, bn; };
struct RatesF { float am, bm, ah, bh, an, bn; };

__device__ __forceinline__ Rates hh_rates(double v) {
    Rates r;
    r.am = exprelr_d((v + 40.0) * -0.1);
    r.bm = 4.0 * exp((v + 65.0) * (-1.0 / 18.0));
    r.ah = 0.07 * exp((v + 65.0) * -0.05);
    r.bh = 1.0 / (1.0 + exp((v + 35.0) * -0.1));
    r.an = 0.1 * exprelr_d((v + 55.0) * -0.1);
    r.bn = 0.125 * exp((v + 65.0) * -0.0125);
    return r;
}

__device__ __forceinline__ RatesF hh_rates(float v) {
    RatesF r;
    r.am = exprelr_f((v + 40.0f) * -0.1f);
    r.bm = 4.0f * expf((v + 65.0f) * (-1.0f / 18.0f));
    r.ah = 0.07f * expf((v + 65.0f) * -0.05f);
    r.bh = 1.0f / (1.0f + expf((v + 35.0f) * -0.1f));
    r.an = 0.1f * exprelr_f((v + 55.0f) * -0.1f);
    r.bn = 0.125f * expf((v + 65.0f) * -0.0125f);
    return r;
}

__device__ __forceinline__ double gate(double x, double a, double b, double dt) {
    const double s = a + b;
    const double xinf = a / s;
    return xinf + (x - xinf) * exp(-dt * s);
}
__device__ __forceinline__ float gate(float x, float a, float b, float dt) {
    const float s = a + b;
    const float xinf = a / s;
    return xinf + (x - xinf) * expf(-dt * s);
}

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

template <class MT>
__device__ __forceinline__ void syn_pass(const DevModel<MT>& d, const PackDesc& pk, double* S, const double* V,
                                         int lane, bool decay, int apply_step, bool current, int& ev_i,
                                         int ev_end, int32_t& late) {
    // drop events that should already have been applied (never happens by construction)
    while (apply_step >= 0 && ev_i < ev_end && d.ev[ev_i].step_rel < apply_step) { ++ev_i; late = 1; }
    for (int js = 0; js < pk.nsyn_row; ++js) {
        const size_t q = (size_t)(pk.syn_row0 + js) * kWarp + lane;
        const int sl = __ldg(d.syn_slot + q);
        if (sl < 0) continue;
        MT g = d.syn_g[q];
        if (decay) g = g * (MT)__ldg(d.syn_decay + q);
        if (apply_step >= 0) {
            while (ev_i < ev_end && d.ev[ev_i].step_rel == apply_step && d.ev[ev_i].js == js) {
                g = g + (MT)d.ev[ev_i].w;
                ++ev_i;
            }
        }
        d.syn_g[q] = g;
        if (current) {
            const MT i_syn = g * ((MT)V[sl] - (MT)__ldg(d.syn_e + q));
            S[sl] = fma(-__ldg(d.syn_sc + q), (double)i_syn, S[sl]);
        }
    }
}

template <class MT>
__device__ __forceinline__ void hh_pass(const DevModel<MT>& d, const PackDesc& pk, double* S, const double* V,
                                        int lane, bool update, bool current, MT dt) {
    for (int jh = 0; jh < pk.nhh_row; ++jh) {
        const size_t q = (size_t)(pk.hh_row0 + jh) * kWarp + lane;
        const int sl = __ldg(d.hh_slot + q);
        if (sl < 0) continue;
        const MT v = (MT)V[sl];
        MT m = d.hh_m[q], h = d.hh_h[q], n = d.hh_n[q];
        if (update) {
            const auto r = hh_rates(v);
            m = gate(m, r.am, r.bm, dt);
            h = gate(h, r.ah, r.bh, dt);
            n = gate(n, r.an, r.bn, dt);
            d.hh_m[q] = m;
            d.hh_h[q] = h;
            d.hh_n[q] = n;
        }
        if (current) {
            const MT m3h = m * m * m * h;
            const MT n2 = n * n;
            const MT i_hh = (MT)__ldg(d.hh_gna + q) * m3h * (v - (MT)kENa) + (MT)__ldg(d.hh_gk + q) * (n2 * n2) * (v - (MT)kEK);
            S[sl] = fma(-__ldg(d.hh_sc + q), (double)i_hh, S[sl]);
        }
    }
}

template <class MT>
__device__ void run_pack(const DevModel<MT>& d, int p, double* tile, int64_t k0, int nsteps, int lane) {
    const PackDesc pk = d.packs[p];
    const int J = pk.nrow;
    const int R = pk.round_rows;
    double* Vg = d.V + (size_t)pk.row0 * kWarp;
    double* S;
    double* V;
    if (pk.smem) {
        S = tile;
        V = tile + (size_t)J * kWarp;
        for (int j = 0; j < J; ++j) V[j * kWarp + lane] = Vg[j * kWarp + lane];
    } else {
        S = d.Sg + pk.sg_off;
        V = Vg;
    }
    const size_t e0 = (size_t)pk.row0 * kWarp + lane;
    const double* __restrict__ ca = d.ca + e0;
    const double* __restrict__ cb = d.cb + e0;
    const double* __restrict__ ck = d.ck + e0;
    const double* __restrict__ ce = d.ce + e0;
    const int32_t* __restrict__ ps_arr = d.pslot + e0;

    for (int j = 0; j < J; ++j) {
        const int sl = j * kWarp + lane;
        S[sl] = fma(__ldg(ca + (size_t)j * kWarp), V[sl], __ldg(cb + (size_t)j * kWarp));
    }
    __syncwarp();

    const int owner = p * kWarp + lane;
    int ev_i = d.ev_off[owner];
    const int ev_end = d.ev_off[owner + 1];
    int32_t late = 0;
    const double dt = d.dt;
    const MT dt_m = (MT)dt;

    // currents at the epoch's first step (events due at its start included)
    syn_pass(d, pk, S, V, lane, false, 0, true, ev_i, ev_end, late);
    __syncwarp();
    hh_pass(d, pk, S, V, lane, false, true, dt_m);
    __syncwarp();

    const int det = (lane < pk.ncell) ? d.det_slot[owner] : -1;
    const double thr = d.threshold;
    const int64_t probe_k0 = d.ctl->probe_k0, probe_max = d.ctl->probe_max;

    for (int s = 0; s < nsteps; ++s) {
        const int64_t k = k0 + s;
        const double t = __dmul_rn((double)k, dt);
        // current clamps active at t_k (depolarising current enters with a plus sign)
        for (int js = 0; js < pk.nst_row; ++js) {
            const size_t q = (size_t)(pk.st_row0 + js) * kWarp + lane;
            const int sl = __ldg(d.st_slot + q);
            if (sl >= 0 && __ldg(d.st_on + q) <= t && t < __ldg(d.st_off + q))
                S[sl] = fma(__ldg(d.st_sc + q), __ldg(d.st_amp + q), S[sl]);
        }
        __syncwarp();
        const double v0 = det >= 0 ? V[det] : 0.0;

        // forward elimination, leaves to root
        double yprev = 0.0, kprev = 0.0;
        int left = R;
        for (int j = 0; j < J; ++j) {
            if (R > 0) {
                if (left == 0) { __syncwarp(); left = R; }
                --left;
            }
            const int ps = __ldg(ps_arr + (size_t)j * kWarp);
            const double kc = __ldg(ck + (size_t)j * kWarp);
            const int sl = j * kWarp + lane;
            const double y = fma(-kprev, yprev, S[sl]);
            S[sl] = y;
            if (ps >= 0) S[ps] = fma(-kc, y, S[ps]);
            kprev = (ps == -1) ? kc : 0.0;
            yprev = y;
        }
        __syncwarp();
        // back substitution, root to leaves; then the next step's scaled right-hand side
        double vnext = 0.0;
        left = (R > 0) ? ((J - 1) % R) + 1 : 0;
        for (int j = J - 1; j >= 0; --j) {
            if (R > 0) {
                if (left == 0) { __syncwarp(); left = R; }
                --left;
            }
            const int ps = __ldg(ps_arr + (size_t)j * kWarp);
            const int sl = j * kWarp + lane;
            const double vp = (ps == -1) ? vnext : ((ps >= 0) ? V[ps] : 0.0);
            const double v = fma(-__ldg(ce + (size_t)j * kWarp), vp, S[sl]);
            V[sl] = v;
            S[sl] = fma(__ldg(ca + (size_t)j * kWarp), v, __ldg(cb + (size_t)j * kWarp));
            vnext = v;
        }
        __syncwarp();

        const bool more = (s + 1) < nsteps;
        // state updates with V(t_{k+1}); currents for the next step
        syn_pass(d, pk, S, V, lane, true, more ? s + 1 : -1, more, ev_i, ev_end, late);
        __syncwarp();
        hh_pass(d, pk, S, V, lane, true, more, dt_m);

        // threshold crossing between V(t_k) and V(t_{k+1}), linearly interpolated
        bool spk = false;
        double ts = 0.0;
        if (det >= 0) {
            const double v1 = V[det];
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
        // probes record V(t_{k+1})
        const int64_t prow = k - probe_k0;
        if (pk.npr > 0 && prow >= 0 && prow < probe_max) {
            for (int q = lane; q < pk.npr; q += kWarp) {
                const int sl = d.probe_slot[pk.pr0 + q];
                d.trace[prow * d.n_probe + d.probe_col[pk.pr0 + q]] = V[sl];
            }
        }
        __syncwarp();
    }

    bool bad = false;
    for (int j = 0; j < J; ++j) {
        const double v = V[j * kWarp + lane];
        if (!isfinite(v)) bad = true;
        if (pk.smem) Vg[j * kWarp + lane] = v;
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    const bool any_late = __any_sync(0xffffffffu, late != 0);
    if (lane == 0 && (any_bad || any_late))
        atomicOr(&d.ctl->status, (any_bad ? kStNonFinite : 0) | (any_late ? kStLateEvent : 0));
    __syncwarp();
}

template <class MT>
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
        run_pack(d, p, tile, k0, nsteps, lane);
    }
}

// ------------------------------------------------------------------------------------------
// Event delivery lists (the "enqueue" and "merge" of Sec. "Implementation": each spike's
// events go to per-cell queues merged with pending events). Here every owner lane gets the
// events of its synapses that fall in the epoch, in a fixed order.



__global__ void k_epoch_begin(EvArgs a) {
    Ctl* c = a.ctl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t k1 = min(c->k0 + (int64_t)a.epoch_steps, c->k_end);
        c->k1 = k1;
        int64_t lo = c->ext_lo, hi = c->n_ext;
        while (lo < hi) {                         // first external event at or after k1
            const int64_t mid = (lo + hi) / 2;
            if (a.ext_step[mid] < k1) lo = mid + 1; else hi = mid;
        }
        c->ext_hi = lo;
        c->spk_lo = c->n_spikes;
        c->pool_n[c->parity ^ 1] = 0;
        c->pack_next = 0;
        c->n_due = 0;
    }
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.n_owner; o += gridDim.x * blockDim.x) a.counts[o] = 0;
}

template <bool kScatter>
__global__ void k_ev_walk(EvArgs a) {
    Ctl* c = a.ctl;
    const int par = c->parity;
    const int64_t k0 = c->k0, k1 = c->k1;
    const int64_t n_pool = min((int64_t)c->pool_n[par], a.pool_cap);
    const int64_t n_ext = c->ext_hi - c->ext_lo;
    const int64_t total = n_pool + n_ext;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        double t, w;
        int64_t step;
        int32_t syn, src, idx;
        if (i < n_pool) {
            const PendEv e = (par ? a.pool[1] : a.pool[0])[i];
            if (e.step >= k1) {
                if (!kScatter) {           // not due yet: keep it for a later epoch
                    const int pos = atomicAdd(&c->pool_n[par ^ 1], 1);
                    if (pos < a.pool_cap) (par ? a.pool[0] : a.pool[1])[pos] = e;
                    else atomicOr(&c->status, kStPoolOverflow);
                }
                continue;
            }
            t = e.t; w = e.w; step = e.step; syn = e.syn; src = e.src; idx = e.idx;
        } else {
            const int64_t x = c->ext_lo + (i - n_pool);
            t = a.ext_t[x]; w = a.ext_w[x]; step = a.ext_step[x]; syn = a.ext_syn[x]; src = -1; idx = a.ext_idx[x];
        }
        if (step < k0) { atomicOr(&c->status, kStLateEvent); step = k0; }
        const int owner = a.syn_owner[syn];
        if (!kScatter) {
            atomicAdd(&a.counts[owner], 1);
        } else {
            const int64_t pos = (int64_t)a.off[owner] + atomicAdd(&a.counts[owner], 1);
            if (pos < a.bucket_cap) {
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
    int64_t run = part[threadIdx.x] - s;
    for (int o = lo; o < hi; ++o) {
        const int cnt = a.counts[o];
        a.off[o] = (int32_t)min(run, a.bucket_cap);
        run += cnt;
        a.counts[o] = 0;
    }
    if (threadIdx.x == blockDim.x - 1) {
        a.off[n] = (int32_t)min(part[blockDim.x - 1], a.bucket_cap);
        a.ctl->n_due = (int32_t)min(part[blockDim.x - 1], (int64_t)INT32_MAX);
        if (part[blockDim.x - 1] > a.bucket_cap) atomicOr(&a.ctl->status, kStBucketOverflow);
    }
}

__device__ __forceinline__ bool ev_less(const EvRec& x, const EvRec& y) {
    if (x.step_rel != y.step_rel) return x.step_rel < y.step_rel;
    if (x.js != y.js) return x.js < y.js;
    if (x.t != y.t) return x.t < y.t;
    if (x.src != y.src) return x.src < y.src;
    return x.idx < y.idx;
}

// Per-owner insertion sort: lists are short (a few events per lane and epoch).
__global__ void k_ev_sort(EvArgs a) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.n_owner; o += gridDim.x * blockDim.x) {
        const int lo = a.off[o], hi = a.off[o + 1];
        for (int i = lo + 1; i < hi; ++i) {
            const EvRec x = a.rec[i];
            int j = i - 1;
            while (j >= lo && ev_less(x, a.rec[j])) { a.rec[j + 1] = a.rec[j]; --j; }
            a.rec[j + 1] = x;
        }
    }
}



// Spike exchange on one GPU: every spike of the epoch is walked against the connections of
// its source (the connection table of Sec. "Implementation", grouped by source here), and each
// resulting event waits in the pending pool for the epoch that contains its step.
__global__ void k_spike_expand(SpkArgs a) {
    Ctl* c = a.ctl;
    const int par = c->parity;
    const int64_t k1 = c->k1;
    const int64_t lo = c->spk_lo, hi = min(c->n_spikes, a.spike_cap);
    for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t gid = a.spk_gid[i];
        const double ts = a.spk_t[i];
        for (int64_t q = a.out_ptr[gid]; q < a.out_ptr[gid + 1]; ++q) {
            PendEv e;
            e.t = __dadd_rn(ts, a.out_delay[q]);
            int64_t step = (int64_t)ceil(__ddiv_rn(e.t, a.dt));
            if (step < k1) step = k1;
            e.step = step;
            e.w = a.out_w[q];
            e.syn = a.out_syn[q];
            e.src = gid;
            e.idx = a.out_idx[q];
            e.pad = 0;
            const int pos = atomicAdd(&c->pool_n[par ^ 1], 1);
            if (pos < a.pool_cap) (par ? a.pool[0] : a.pool[1])[pos] = e;
            else atomicOr(&c->status, kStPoolOverflow);
        }
    }
}

__global__ void k_epoch_end(Ctl* c, int64_t pool_cap) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c->k0 = c->k1;
        c->ext_lo = c->ext_hi;
        const int np = c->parity ^ 1;
        if (c->pool_n[np] > pool_cap) c->pool_n[np] = (int32_t)pool_cap;
        c->parity = np;
    }
}

// ------------------------------------------------------------------------------------------
// Layout conversions between the model's CV order and the tile layout.

template <class T>
__global__ void k_gather(double* out, const T* src, const int64_t* idx, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)src[idx[i]];
}

template <class T>
__global__ void k_scatter(T* dst, const double* src, const int64_t* idx, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[idx[i]] = (T)src[i];
}

// ------------------------------------------------------------------------------------------
// Launch wrappers used by the host runtime.

template <class MT>
cudaError_t launch_epoch(const DevModel<MT>& d, int grid, int warps_per_cta, int tile_doubles, cudaStream_t s) {
    // the shared-memory limit was raised once by epoch_occupancy (not a stream operation,
    // so it stays out of graph capture)
    const size_t smem = (size_t)warps_per_cta * (size_t)tile_doubles * sizeof(double);
    arb_epoch_kernel<MT><<<grid, warps_per_cta * kWarp, smem, s>>>(d, tile_doubles);
    return cudaGetLastError();
}

template <class MT>
cudaError_t epoch_occupancy(int warps_per_cta, int tile_doubles, int* blocks_per_sm) {
    const size_t smem = (size_t)warps_per_cta * (size_t)tile_doubles * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(arb_epoch_kernel<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, arb_epoch_kernel<MT>, warps_per_cta * kWarp, smem);
}

template cudaError_t launch_epoch<double>(const DevModel<double>&, int, int, int, cudaStream_t);
template cudaError_t launch_epoch<float>(const DevModel<float>&, int, int, int, cudaStream_t);
template cudaError_t epoch_occupancy<double>(int, int, int*);
template cudaError_t epoch_occupancy<float>(int, int, int*);

cudaError_t launch_events_pre(const EvArgs& a, int n_sm, cudaStream_t s) {
    const int owner_blocks = max(1, min(4 * n_sm, (a.n_owner + 255) / 256));
    k_epoch_begin<<<owner_blocks, 256, 0, s>>>(a);
    k_ev_walk<false><<<2 * n_sm, 256, 0, s>>>(a);
    k_ev_scan<<<1, 1024, 0, s>>>(a);
    k_ev_walk<true><<<2 * n_sm, 256, 0, s>>>(a);
    k_ev_sort<<<owner_blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_events_post(const SpkArgs& a, int n_sm, cudaStream_t s) {
    k_spike_expand<<<n_sm, 128, 0, s>>>(a);
    k_epoch_end<<<1, 32, 0, s>>>(a.ctl, a.pool_cap);
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
