// Discrete adjoint of the implicit cable step: gradients of a voltage loss w.r.t. the channel
// densities (gbar_na, gbar_k, g_leak) and the membrane capacitance.
//
// Forward map per cell (the implicit reading of the step of Sec. "Model", states frozen at
// t_k for the membrane terms, gates advanced with the new voltage):
//   A(y^k) V^{k+1} = (C/dt) V^k + M(y^k) + I_inj(t_k),  A = diag(C/dt + G(y^k)) + axial Laplacian,
//   y^{k+1} = Phi(y^k, V^{k+1}).
// A is symmetric, so the reverse sweep solves with the same tree matrix:
//   Vbar = (C/dt) lam_{k+1} + dL/dV^{k+1} + sum_gates dPhi/dV ybar,   lam_k = A(y^k)^{-1} Vbar,
// and the parameter and gate adjoints follow from lam_k, V^k, V^{k+1} and y^k.
//
// Work is per cell and cells never interact, so every kernel runs one block per cell over a
// whole range of steps: the element-wise parts (membrane terms, gates and their derivatives,
// gradient terms) are spread over the block's threads; the tree solve runs in shared memory
// on the first warp, which takes the cell's unbranched chains level by level (leaf chains
// first), one chain per lane, and hands each chain's elimination to its parent chain through
// a per-chain slot. The forward pass keeps a checkpoint of the state every `ckpt` steps. The
// backward pass goes segment by segment: each stage sweeps one segment backwards while other
// blocks of the same launch recompute the previous segment from its checkpoint into the second
// segment buffer, keeping every state and the gate-update derivatives the sweep will need.
#include <cuda_runtime.h>

#include <cstdint>

#include "arb_hh.cuh"
#include "arb_internal.h"

namespace arbk {
namespace {

constexpr int kAdjThreads = 128;   // threads per cell (block)

// Conductance (uS) and conductance x reversal (nA) of CV i with the gates of one step; gl, gel and
// hj are the CV's passive conductance, its product with the reversal and its HH instance.
__device__ __forceinline__ void membrane(const AdjArgs& a, double gl, double gel, int32_t hj, const double* Y, double& G,
                                         double& GE) {
    G = gl;
    GE = gel;
    const int32_t j = hj;
    if (j >= 0) {
        const double m = Y[j], h = Y[a.n_hh + j], n = Y[2 * a.n_hh + j];
        const double n2 = n * n;
        const double gna = a.gna[j] * (m * m * m * h);
        const double gk = a.gk[j] * (n2 * n2);
        G += gna + gk + a.gl[j];
        GE += gna * kENa + gk * kEK + a.gl[j] * kEL;
    }
}

// Shared memory of one block (one cell): the solve's working arrays, and the cell's constants
// and solve schedule, copied once per launch so that no step waits on a global load for them
// (a chain's next CV index, its axial conductance, the membrane constants).
struct Smem {
    double* d;     // [smem_cv] diagonal, then eliminated pivots
    double* b;     // [smem_cv] right-hand side, then the solution
    double* r;     // [smem_cv] 1 / eliminated pivot
    double* cd;    // [smem_ch] a chain's elimination into its parent's diagonal
    double* cb;    //           ... and right-hand side
    double* sig;   // [smem_cv] axial conductance to the parent (cell-local CV order)
    double* cdt;   // [smem_cv] C / dt
    double* dsig;  // [smem_cv] sum of the CV's axial conductances (own + children)
    double* glin;  // [smem_cv] passive conductance
    double* gelin; // [smem_cv] passive conductance x reversal
    int32_t* par;  // [smem_cv] cell-local parent, -1 at the root
    int32_t* hidx; // [smem_cv] HH instance of the CV, -1 none
    int32_t* cvs;  // [smem_cv] CVs of the cell's chains, chain after chain (as ch_cvs)
    int32_t* chp;  // [smem_ch + 1] cell-local chain -> range in cvs
    int32_t* kidp; // [smem_ch + 1] cell-local chain -> range in kids
    int32_t* kids; // [smem_ch] cell-local child chains
    int32_t* levb; // [smem_ch + 2] first cell-local chain of each level, then the end
};

__device__ __forceinline__ Smem smem_of(const AdjArgs& a) {
    extern __shared__ double adj_smem[];
    Smem m;
    const int ncv = a.smem_cv, nch = a.smem_ch;
    m.d = adj_smem;
    m.b = m.d + ncv;
    m.r = m.b + ncv;
    m.cd = m.r + ncv;
    m.cb = m.cd + nch;
    m.sig = m.cb + nch;
    m.cdt = m.sig + ncv;
    m.dsig = m.cdt + ncv;
    m.glin = m.dsig + ncv;
    m.gelin = m.glin + ncv;
    m.par = reinterpret_cast<int32_t*>(m.gelin + ncv);
    m.hidx = m.par + ncv;
    m.cvs = m.hidx + ncv;
    m.chp = m.cvs + ncv;
    m.kidp = m.chp + nch + 1;
    m.kids = m.kidp + nch + 1;
    m.levb = m.kids + nch;
    return m;
}

// Copies cell c's constants and solve schedule into shared memory (all threads of the block).
__device__ void load_cell(const AdjArgs& a, int c, const Smem& sm) {
    const int tid = threadIdx.x;
    const int64_t off = a.off[c], n = a.off[c + 1] - off;
    const int64_t q0 = a.ch_ptr[c], nq = a.ch_ptr[c + 1] - q0;
    const int64_t l0 = a.lev_off[c], nlb = a.lev_off[c + 1] - l0;
    const int64_t cv0 = a.ch_cv_ptr[q0], k0 = a.ch_kid_ptr[q0];
    for (int64_t i = tid; i < n; i += kAdjThreads) {
        sm.sig[i] = a.sig[off + i];
        sm.cdt[i] = a.cdt[off + i];
        sm.dsig[i] = a.dsig[off + i];
        sm.glin[i] = a.glin[off + i];
        sm.gelin[i] = a.gelin[off + i];
        sm.par[i] = a.parent[off + i];
        sm.hidx[i] = a.hidx[off + i];
        sm.cvs[i] = a.ch_cvs[cv0 + i];          // a cell's chains hold each of its CVs once
    }
    for (int64_t q = tid; q <= nq; q += kAdjThreads) {
        sm.chp[q] = (int32_t)(a.ch_cv_ptr[q0 + q] - cv0);
        sm.kidp[q] = (int32_t)(a.ch_kid_ptr[q0 + q] - k0);
    }
    for (int64_t k = tid; k < a.ch_kid_ptr[q0 + nq] - k0; k += kAdjThreads) sm.kids[k] = (int32_t)(a.ch_kids[k0 + k] - q0);
    for (int64_t L = tid; L < nlb; L += kAdjThreads) sm.levb[L] = (int32_t)(a.lev_bound[l0 + L] - q0);
    __syncthreads();
}

// Tree solve of cell c in shared memory (first warp): symmetric matrix with diagonal sm.d and
// off-diagonal -sigma between a CV and its parent; the solution replaces sm.b.
// Elimination: chains level by level from the leaves; within a chain from its tail (the CV
// farthest from the root, which first takes its child chains' eliminations) to its head,
// whose elimination goes to the chain's slot. Back substitution: levels in reverse order, each
// chain from its head (using its parent's solution) to its tail.
__device__ void chain_solve(const AdjArgs& a, int c, int lane, const Smem& sm) {
    const int nl = (int)(a.lev_off[c + 1] - a.lev_off[c]) - 1;
    for (int L = 0; L < nl; ++L) {
        for (int q = sm.levb[L] + lane; q < sm.levb[L + 1]; q += 32) {
            const int cs = sm.chp[q], ce = sm.chp[q + 1];
            int x = sm.cvs[ce - 1];
            double dx = sm.d[x], bx = sm.b[x];
            for (int k = sm.kidp[q]; k < sm.kidp[q + 1]; ++k) {
                const int j = sm.kids[k];
                dx += sm.cd[j];
                bx += sm.cb[j];
            }
            for (int u = ce - 1; u > cs; --u) {
                const int y = sm.cvs[u - 1];
                const double sg = sm.sig[x];
                const double r = rcp_nr(dx);
                sm.r[x] = r;
                sm.b[x] = bx;
                const double f = sg * r;
                dx = sm.d[y] - f * sg;
                bx = sm.b[y] + f * bx;
                x = y;
            }
            const double r = rcp_nr(dx);
            sm.r[x] = r;
            sm.b[x] = bx;
            if (sm.par[x] >= 0) {
                const double sg = sm.sig[x];
                const double f = sg * r;
                sm.cd[q] = -f * sg;
                sm.cb[q] = f * bx;
            }
        }
        __syncwarp();
    }
    for (int L = nl - 1; L >= 0; --L) {
        for (int q = sm.levb[L] + lane; q < sm.levb[L + 1]; q += 32) {
            const int cs = sm.chp[q], ce = sm.chp[q + 1];
            int x = sm.cvs[cs];
            const int32_t p = sm.par[x];
            double v = (p >= 0) ? (sm.b[x] + sm.sig[x] * sm.b[p]) * sm.r[x] : sm.b[x] * sm.r[x];
            sm.b[x] = v;
            for (int u = cs + 1; u < ce; ++u) {
                x = sm.cvs[u];
                v = (sm.b[x] + sm.sig[x] * v) * sm.r[x];
                sm.b[x] = v;
            }
        }
        __syncwarp();
    }
}

// mode 0: steps [s0, s1) from the running state (a.V, a.Y), in place, with a checkpoint
//         before every step that is a multiple of ckpt, and the loss;
// mode 1: steps [s0, s1) from checkpoint s0 / ckpt, every state kept in segment buffer buf.
__device__ void forward_cell(const AdjArgs& a, int c, int64_t s0, int64_t s1, int mode, int buf) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t off = a.off[c], n = a.off[c + 1] - off;
    double* const segV = a.segV[buf];
    double* const segY = a.segY[buf];
    double* const segG = a.segG[buf];
    const int64_t nhh = a.n_hh;
    const Smem sm = smem_of(a);
    load_cell(a, c, sm);
    if (mode == 1) {
        const double* cV = a.ckV + (s0 / a.ckpt) * a.n_cv;
        const double* cY = a.ckY + (s0 / a.ckpt) * 3 * nhh;
        for (int64_t i = off + tid; i < off + n; i += kAdjThreads) {
            segV[i] = cV[i];
            const int32_t j = sm.hidx[i - off];
            if (j >= 0)
                for (int g = 0; g < 3; ++g) segY[g * nhh + j] = cY[g * nhh + j];
        }
        __syncthreads();
    }
    double lsum = 0.0;
    for (int64_t s = s0; s < s1; ++s) {
        const double* Vs;
        const double* Ys;
        double* Vd;
        double* Yd;
        if (mode == 0) {
            Vs = Vd = a.V;
            Ys = Yd = a.Y;
            if (s % a.ckpt == 0) {
                double* cV = a.ckV + (s / a.ckpt) * a.n_cv;
                double* cY = a.ckY + (s / a.ckpt) * 3 * nhh;
                for (int64_t i = off + tid; i < off + n; i += kAdjThreads) {
                    cV[i] = a.V[i];
                    const int32_t j = sm.hidx[i - off];
                    if (j >= 0)
                        for (int g = 0; g < 3; ++g) cY[g * nhh + j] = a.Y[g * nhh + j];
                }
            }
        } else {
            Vs = segV + (s - s0) * a.n_cv;
            Ys = segY + (s - s0) * 3 * nhh;
            Vd = const_cast<double*>(Vs) + a.n_cv;
            Yd = const_cast<double*>(Ys) + 3 * nhh;
        }
        // assemble A(y^s) and the right-hand side
        for (int64_t i = off + tid; i < off + n; i += kAdjThreads) {
            const int64_t li = i - off;
            double G, GE;
            membrane(a, sm.glin[li], sm.gelin[li], sm.hidx[li], Ys, G, GE);
            sm.d[li] = sm.cdt[li] + G + sm.dsig[li];
            sm.b[li] = sm.cdt[li] * Vs[i] + GE;
        }
        __syncthreads();
        if (tid < 32) {
            if (tid == 0) {
                const double t = (double)(a.k0 + s) * a.dt;
                for (int64_t q = a.st_ptr[c]; q < a.st_ptr[c + 1]; ++q)
                    if (a.st_on[q] <= t && t < a.st_on[q] + a.st_dur[q]) sm.b[a.st_cv[q] - off] += a.st_amp[q];
            }
            __syncwarp();
            chain_solve(a, c, lane, sm);
        }
        __syncthreads();
        // new voltage, gates with it, loss
        for (int64_t i = off + tid; i < off + n; i += kAdjThreads) {
            const double v = sm.b[i - off];
            Vd[i] = v;
            const int32_t j = sm.hidx[i - off];
            if (j >= 0) {
                Gates3 xg{Ys[j], Ys[nhh + j], Ys[2 * nhh + j]}, dvg, eg;
                if (mode == 0 && hh_gates_tab(a.hh_tab, v, xg.m, xg.h, xg.n)) {
                    Yd[j] = xg.m;
                    Yd[nhh + j] = xg.h;
                    Yd[2 * nhh + j] = xg.n;
                } else if (mode == 0) {
                    const Rates r = hh_rates(v);
                    Yd[j] = gate(Ys[j], r.am, r.bm, a.dt);
                    Yd[nhh + j] = gate(Ys[nhh + j], r.ah, r.bh, a.dt);
                    Yd[2 * nhh + j] = gate(Ys[2 * nhh + j], r.an, r.bn, a.dt);
                } else if (hh_gates_tab_dv(a.hh_tab, v, xg, dvg, eg)) {
                    // from the table: the gate update, dPhi/dV and exp(-dt (alpha + beta))
                    Yd[j] = xg.m;
                    Yd[nhh + j] = xg.h;
                    Yd[2 * nhh + j] = xg.n;
                    double* G6 = segG + (s - s0) * 6 * nhh;
                    G6[j] = dvg.m;
                    G6[nhh + j] = dvg.h;
                    G6[2 * nhh + j] = dvg.n;
                    G6[3 * nhh + j] = eg.m;
                    G6[4 * nhh + j] = eg.h;
                    G6[5 * nhh + j] = eg.n;
                } else {
                    // the gate update, and what the reverse sweep of this step needs from it:
                    // dPhi/dV and exp(-dt (alpha + beta)) of each gate
                    Rates r, dr;
                    hh_rates_derivs(v, r, dr);
                    const double dt = a.dt;
                    const double em = gate_decay(r.am, r.bm, dt);
                    const double eh = gate_decay(r.ah, r.bh, dt);
                    const double en = gate_decay(r.an, r.bn, dt);
                    const double xm = Ys[j], xh = Ys[nhh + j], xn = Ys[2 * nhh + j];
                    Yd[j] = gate_e(xm, r.am, r.bm, em);
                    Yd[nhh + j] = gate_e(xh, r.ah, r.bh, eh);
                    Yd[2 * nhh + j] = gate_e(xn, r.an, r.bn, en);
                    double* G6 = segG + (s - s0) * 6 * nhh;
                    G6[j] = gate_dv(xm, r.am, r.bm, dr.am, dr.bm, dt, em);
                    G6[nhh + j] = gate_dv(xh, r.ah, r.bh, dr.ah, dr.bh, dt, eh);
                    G6[2 * nhh + j] = gate_dv(xn, r.an, r.bn, dr.an, dr.bn, dt, en);
                    G6[3 * nhh + j] = em;
                    G6[4 * nhh + j] = eh;
                    G6[5 * nhh + j] = en;
                }
            }
            if (mode == 0) {
                const int32_t o = a.obs[i];
                if (o >= 0) {
                    const double e = v - a.target[s * a.n_obs + o];
                    lsum += a.loss_scale * e * e;
                }
            }
        }
        __syncthreads();
    }
    if (mode == 0) {
        // fixed-order reduction: warps, then the warp sums in order
        __shared__ double wsum[kAdjThreads / 32];
        for (int sh = 16; sh > 0; sh >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, sh);
        if (lane == 0) wsum[tid >> 5] = lsum;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < kAdjThreads / 32; ++w) tot += wsum[w];
            a.cell_loss[c] += tot;
        }
    }
}

// Reverse sweep over the segment [s0, s1) held in segment buffer buf.
__device__ void reverse_cell(const AdjArgs& a, int c, int64_t s0, int64_t s1, int buf) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t off = a.off[c], n = a.off[c + 1] - off;
    const double* const segV = a.segV[buf];
    const double* const segY = a.segY[buf];
    const double* const segG = a.segG[buf];
    const int64_t nhh = a.n_hh, ncv = a.n_cv;
    const double dt = a.dt;
    const Smem sm = smem_of(a);
    load_cell(a, c, sm);
    for (int64_t s = s1 - 1; s >= s0; --s) {
        const double* V0 = segV + (s - s0) * ncv;
        const double* V1 = V0 + ncv;
        const double* Y0 = segY + (s - s0) * 3 * nhh;
        // Vbar = (C/dt) lam + dL/dV^{s+1} + dPhi/dV^T ybar; A(y^s); ybar <- dPhi/dy ybar
        for (int64_t i = off + tid; i < off + n; i += kAdjThreads) {
            const int64_t li = i - off;
            double G, GE;
            membrane(a, sm.glin[li], sm.gelin[li], sm.hidx[li], Y0, G, GE);
            sm.d[li] = sm.cdt[li] + G + sm.dsig[li];
            double vb = sm.cdt[li] * a.lam[i];
            const int32_t o = a.obs[i];
            if (o >= 0) vb += 2.0 * a.loss_scale * (V1[i] - a.target[s * a.n_obs + o]);
            const int32_t j = sm.hidx[i - off];
            if (j >= 0) {
                const double* G6 = segG + (s - s0) * 6 * nhh;
                double* yb = a.ybar;
                vb += G6[j] * yb[j] + G6[nhh + j] * yb[nhh + j] + G6[2 * nhh + j] * yb[2 * nhh + j];
                yb[j] *= G6[3 * nhh + j];
                yb[nhh + j] *= G6[4 * nhh + j];
                yb[2 * nhh + j] *= G6[5 * nhh + j];
            }
            sm.b[i - off] = vb;
        }
        __syncthreads();
        if (tid < 32) chain_solve(a, c, lane, sm);
        __syncthreads();
        // lam_s; gradient terms; gate adjoint of y^s
        for (int64_t i = off + tid; i < off + n; i += kAdjThreads) {
            const double lam = sm.b[i - off];
            a.lam[i] = lam;
            const double v1 = V1[i];
            a.gacc[3 * ncv + i] += lam * (V0[i] - v1) / dt * (a.area[i] * 1e-5);
            const int32_t j = sm.hidx[i - off];
            if (j >= 0) {
                const double m = Y0[j], h = Y0[nhh + j], nn = Y0[2 * nhh + j];
                const double lna = lam * (kENa - v1), lk = lam * (kEK - v1), ll = lam * (kEL - v1);
                const double sc = a.area[i] * 1e-2;
                const double m3h = m * m * m * h, n2 = nn * nn;
                a.gacc[i] += m3h * lna * sc;
                a.gacc[ncv + i] += n2 * n2 * lk * sc;
                a.gacc[2 * ncv + i] += ll * sc;
                a.ybar[j] += a.gna[j] * 3.0 * m * m * h * lna;
                a.ybar[nhh + j] += a.gna[j] * m * m * m * lna;
                a.ybar[2 * nhh + j] += a.gk[j] * 4.0 * n2 * nn * lk;
            }
        }
        __syncthreads();
    }
}

// Forward pass with checkpoints and the loss: one block per cell.
__global__ void __launch_bounds__(kAdjThreads) k_adj_forward(AdjArgs a, int64_t s0, int64_t s1) {
    forward_cell(a, blockIdx.x, s0, s1, 0, 0);
}

// One backward stage: blocks [0, n_cells) sweep segment [r0, r1) (buffer rbuf) backwards,
// blocks [n_cells, 2 n_cells) recompute segment [f0, f1) into the other buffer meanwhile.
__global__ void __launch_bounds__(kAdjThreads) k_adj_stage(AdjArgs a, int64_t r0, int64_t r1, int rbuf,
                                                           int64_t f0, int64_t f1) {
    const int b = blockIdx.x;
    if (b < a.n_cells) {
        if (r1 > r0) reverse_cell(a, b, r0, r1, rbuf);
    } else if (f1 > f0) {
        forward_cell(a, b - a.n_cells, f0, f1, 1, rbuf ^ 1);
    }
}

// Gradient per parameter group: sums over the group's CVs in ascending order.
__global__ void k_adj_reduce(AdjArgs a) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_groups) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int64_t q = a.grp_ptr[g]; q < a.grp_ptr[g + 1]; ++q) {
        const int64_t i = a.grp_cv[q];
        s0 += a.gacc[i];
        s1 += a.gacc[a.n_cv + i];
        s2 += a.gacc[2 * a.n_cv + i];
        s3 += a.gacc[3 * a.n_cv + i];
    }
    a.grad[4 * g + 0] = s0;
    a.grad[4 * g + 1] = s1;
    a.grad[4 * g + 2] = s2;
    a.grad[4 * g + 3] = s3;
}

}  // namespace

size_t adj_smem_bytes(const AdjArgs& a) {
    return sizeof(double) * (8 * (size_t)a.smem_cv + 2 * (size_t)a.smem_ch) +
           sizeof(int32_t) * (3 * (size_t)a.smem_cv + 4 * (size_t)a.smem_ch + 4);
}

cudaError_t adj_prepare(const AdjArgs& a) {
    const int bytes = (int)adj_smem_bytes(a);
    cudaError_t e = cudaFuncSetAttribute(k_adj_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_adj_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_adj_forward(const AdjArgs& a, int64_t s0, int64_t s1, cudaStream_t s) {
    if (a.n_cells == 0 || s1 <= s0) return cudaSuccess;
    k_adj_forward<<<a.n_cells, kAdjThreads, adj_smem_bytes(a), s>>>(a, s0, s1);
    return cudaGetLastError();
}

cudaError_t launch_adj_stage(const AdjArgs& a, int64_t r0, int64_t r1, int rbuf, int64_t f0, int64_t f1,
                             cudaStream_t s) {
    if (a.n_cells == 0) return cudaSuccess;
    k_adj_stage<<<2 * a.n_cells, kAdjThreads, adj_smem_bytes(a), s>>>(a, r0, r1, rbuf, f0, f1);
    return cudaGetLastError();
}

cudaError_t launch_adj_reduce(const AdjArgs& a, cudaStream_t s) {
    if (a.n_groups == 0) return cudaSuccess;
    k_adj_reduce<<<(a.n_groups + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace arbk
