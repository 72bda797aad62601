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
// Work is per cell and cells never interact, so every kernel runs one warp per cell over a
// whole range of steps: the element-wise parts (membrane terms, gates and their derivatives,
// gradient terms) are spread over the lanes, the tree elimination runs on lane 0. The forward
// pass keeps a checkpoint of the state every `ckpt` steps; the reverse pass recomputes one
// segment from its checkpoint, keeping every state, and sweeps it backwards.
#include <cuda_runtime.h>

#include <cstdint>

#include "arb_hh.cuh"
#include "arb_internal.h"

namespace arbk {
namespace {

constexpr int kAdjWarps = 1;   // warps per block: one cell per block spreads small batches over all SMs

// Conductance (uS) and conductance x reversal (nA) of CV i with the gates of one step.
__device__ __forceinline__ void membrane(const AdjArgs& a, int64_t i, const double* Y, double& G, double& GE) {
    G = a.glin[i];
    GE = a.gelin[i];
    const int32_t j = a.hidx[i];
    if (j >= 0) {
        const double m = Y[j], h = Y[a.n_hh + j], n = Y[2 * a.n_hh + j];
        const double n2 = n * n;
        const double gna = a.gna[j] * (m * m * m * h);
        const double gk = a.gk[j] * (n2 * n2);
        G += gna + gk + a.gl[j];
        GE += gna * kENa + gk * kEK + a.gl[j] * kEL;
    }
}

// In-place tree solve of one cell (lane 0): diagonal d, off-diagonal -sigma, right-hand side b;
// the solution replaces b. Elimination from the highest local index to the root, then back
// substitution (parent index < child index).
__device__ void tree_solve(const AdjArgs& a, int64_t off, int64_t n) {
    double* d = a.d + off;
    double* b = a.b + off;
    const int32_t* par = a.parent + off;
    const double* sg = a.sig + off;
    for (int64_t i = n - 1; i >= 1; --i) {
        const int32_t p = par[i];
        const double f = sg[i] / d[i];
        d[p] -= f * sg[i];
        b[p] += f * b[i];
    }
    b[0] = b[0] / d[0];
    for (int64_t i = 1; i < n; ++i) b[i] = (b[i] + sg[i] * b[par[i]]) / d[i];
}

// mode 0: steps [s0, s1) from the running state (a.V, a.Y), in place, with a checkpoint
//         before every step that is a multiple of ckpt, and the loss;
// mode 1: steps [s0, s1) from checkpoint s0 / ckpt, every state kept in the segment buffers.
__global__ void __launch_bounds__(kAdjWarps * 32) k_adj_forward(AdjArgs a, int64_t s0, int64_t s1, int mode) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kAdjWarps + (threadIdx.x >> 5);
    if (c >= a.n_cells) return;
    const int64_t off = a.off[c], n = a.off[c + 1] - off;
    const int64_t nhh = a.n_hh;
    if (mode == 1) {
        const double* cV = a.ckV + (s0 / a.ckpt) * a.n_cv;
        const double* cY = a.ckY + (s0 / a.ckpt) * 3 * nhh;
        for (int64_t i = off + lane; i < off + n; i += 32) {
            a.segV[i] = cV[i];
            const int32_t j = a.hidx[i];
            if (j >= 0)
                for (int g = 0; g < 3; ++g) a.segY[g * nhh + j] = cY[g * nhh + j];
        }
        __syncwarp();
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
                for (int64_t i = off + lane; i < off + n; i += 32) {
                    cV[i] = a.V[i];
                    const int32_t j = a.hidx[i];
                    if (j >= 0)
                        for (int g = 0; g < 3; ++g) cY[g * nhh + j] = a.Y[g * nhh + j];
                }
            }
        } else {
            Vs = a.segV + (s - s0) * a.n_cv;
            Ys = a.segY + (s - s0) * 3 * nhh;
            Vd = const_cast<double*>(Vs) + a.n_cv;
            Yd = const_cast<double*>(Ys) + 3 * nhh;
        }
        // assemble A(y^s) and the right-hand side
        for (int64_t i = off + lane; i < off + n; i += 32) {
            double G, GE;
            membrane(a, i, Ys, G, GE);
            a.d[i] = a.cdt[i] + G + a.dsig[i];
            a.b[i] = a.cdt[i] * Vs[i] + GE;
        }
        __syncwarp();
        if (lane == 0) {
            const double t = (double)(a.k0 + s) * a.dt;
            for (int64_t q = a.st_ptr[c]; q < a.st_ptr[c + 1]; ++q)
                if (a.st_on[q] <= t && t < a.st_on[q] + a.st_dur[q]) a.b[a.st_cv[q]] += a.st_amp[q];
            tree_solve(a, off, n);
        }
        __syncwarp();
        // new voltage, gates with it, loss
        for (int64_t i = off + lane; i < off + n; i += 32) {
            const double v = a.b[i];
            Vd[i] = v;
            const int32_t j = a.hidx[i];
            if (j >= 0) {
                const Rates r = hh_rates(v);
                Yd[j] = gate(Ys[j], r.am, r.bm, a.dt);
                Yd[nhh + j] = gate(Ys[nhh + j], r.ah, r.bh, a.dt);
                Yd[2 * nhh + j] = gate(Ys[2 * nhh + j], r.an, r.bn, a.dt);
            }
            if (mode == 0) {
                const int32_t o = a.obs[i];
                if (o >= 0) {
                    const double e = v - a.target[s * a.n_obs + o];
                    lsum += a.loss_scale * e * e;
                }
            }
        }
        __syncwarp();
    }
    if (mode == 0) {
        for (int sh = 16; sh > 0; sh >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, sh);
        if (lane == 0) a.cell_loss[c] += lsum;
    }
}

// Reverse sweep over the segment [s0, s1) held in the segment buffers.
__global__ void __launch_bounds__(kAdjWarps * 32) k_adj_reverse(AdjArgs a, int64_t s0, int64_t s1) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kAdjWarps + (threadIdx.x >> 5);
    if (c >= a.n_cells) return;
    const int64_t off = a.off[c], n = a.off[c + 1] - off;
    const int64_t nhh = a.n_hh, ncv = a.n_cv;
    const double dt = a.dt;
    for (int64_t s = s1 - 1; s >= s0; --s) {
        const double* V0 = a.segV + (s - s0) * ncv;
        const double* V1 = V0 + ncv;
        const double* Y0 = a.segY + (s - s0) * 3 * nhh;
        // Vbar = (C/dt) lam + dL/dV^{s+1} + dPhi/dV^T ybar; A(y^s); ybar <- dPhi/dy ybar
        for (int64_t i = off + lane; i < off + n; i += 32) {
            double G, GE;
            membrane(a, i, Y0, G, GE);
            a.d[i] = a.cdt[i] + G + a.dsig[i];
            double vb = a.cdt[i] * a.lam[i];
            const int32_t o = a.obs[i];
            if (o >= 0) vb += 2.0 * a.loss_scale * (V1[i] - a.target[s * a.n_obs + o]);
            const int32_t j = a.hidx[i];
            if (j >= 0) {
                const double v = V1[i];
                const Rates r = hh_rates(v);
                const Rates dr = hh_rate_derivs(v, r);
                const double em = exp(-dt * (r.am + r.bm));
                const double eh = exp(-dt * (r.ah + r.bh));
                const double en = exp(-dt * (r.an + r.bn));
                double* yb = a.ybar;
                vb += gate_dv(Y0[j], r.am, r.bm, dr.am, dr.bm, dt, em) * yb[j]
                    + gate_dv(Y0[nhh + j], r.ah, r.bh, dr.ah, dr.bh, dt, eh) * yb[nhh + j]
                    + gate_dv(Y0[2 * nhh + j], r.an, r.bn, dr.an, dr.bn, dt, en) * yb[2 * nhh + j];
                yb[j] *= em;
                yb[nhh + j] *= eh;
                yb[2 * nhh + j] *= en;
            }
            a.b[i] = vb;
        }
        __syncwarp();
        if (lane == 0) tree_solve(a, off, n);
        __syncwarp();
        // lam_s; gradient terms; gate adjoint of y^s
        for (int64_t i = off + lane; i < off + n; i += 32) {
            const double lam = a.b[i];
            a.lam[i] = lam;
            const double v1 = V1[i];
            a.gacc[3 * ncv + i] += lam * (V0[i] - v1) / dt * (a.area[i] * 1e-5);
            const int32_t j = a.hidx[i];
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
        __syncwarp();
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

int adj_blocks(int32_t n_cells) { return (n_cells + kAdjWarps - 1) / kAdjWarps; }

cudaError_t launch_adj_forward(const AdjArgs& a, int64_t s0, int64_t s1, int mode, cudaStream_t s) {
    if (a.n_cells == 0 || s1 <= s0) return cudaSuccess;
    k_adj_forward<<<adj_blocks(a.n_cells), kAdjWarps * 32, 0, s>>>(a, s0, s1, mode);
    return cudaGetLastError();
}

cudaError_t launch_adj_reverse(const AdjArgs& a, int64_t s0, int64_t s1, cudaStream_t s) {
    if (a.n_cells == 0 || s1 <= s0) return cudaSuccess;
    k_adj_reverse<<<adj_blocks(a.n_cells), kAdjWarps * 32, 0, s>>>(a, s0, s1);
    return cudaGetLastError();
}

cudaError_t launch_adj_reduce(const AdjArgs& a, cudaStream_t s) {
    if (a.n_groups == 0) return cudaSuccess;
    k_adj_reduce<<<(a.n_groups + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace arbk
