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
// gradient terms) are spread over the block's threads; the tree solve runs in shared memory.
// The forward pass keeps a checkpoint of the state every `ckpt` steps. The backward pass goes
// segment by segment: each stage sweeps one segment backwards while other blocks of the same
// launch recompute the previous segment from its checkpoint into the second segment buffer,
// keeping every state and the gate-update derivatives the sweep will need. The forward pass
// records the last segment that way itself, so the first stage already sweeps.
//
// Tree solve. On this GPU a warp issues at most one FP64 instruction every 64 cycles, however
// many of its lanes are active, so the solve's time is the number of FP64 instructions on its
// longest dependent path, not the number of lanes doing work. The cell's unbranched chains are
// taken level by level (leaf chains first), and along a chain, from its tail (farthest from the
// root) to its head, the elimination is written in projective form: with D_k the eliminated
// pivots, B_k the eliminated right-hand sides and s_k the axial conductance from CV k to the
// next one of the chain,
//   P_k = d_k P_{k-1} - s_{k-1}^2 P_{k-2},   W_k = b_k P_{k-1} + s_{k-1} W_{k-1},
//   D_k = P_k / P_{k-1},  B_k = W_k / P_{k-1}   (P_{-1} = 1, P_0 = D_0, W_0 = B_0).
// Scaled by per-CV constants (P^_k = P_k / c_k, W^_k = W_k / g_k with c_k = s_{k-1}^2 c_{k-2},
// g_k = s_{k-1} g_{k-1}) each step is one fused multiply-add:
//   P^_k = (d_k rho_k) P^_{k-1} - P^_{k-2},   W^_k = (b_k beta_k) P^_{k-1} + W^_{k-1},
// rho_k = c_{k-1} / c_k, beta_k = c_{k-1} / g_k. Warp 0 runs the P^ recurrences of a level while
// warp 1 runs the W^ recurrences of the level before, one lane per chain. No division is on that
// path. The chain's elimination into its parent (-s_h^2 / D_h and s_h B_h / D_h at its head h)
// takes one reciprocal per chain. Then every thread forms, per CV, u_k = B_k / D_k and
// e_k = s_k / D_k (one reciprocal each, in parallel), and the back substitution,
// V_k = u_k + e_k V_parent, is one fused multiply-add per CV (long chains of small levels split
// over three lanes). The host computes the constants, cuts a chain wherever their range, or the
// range P^ can reach, would leave about 2^{+-300}, and roots each cell's tree where the
// level-by-level critical path is shortest.
#include <cuda_runtime.h>

#include <cstdint>

#include "arb_hh.cuh"
#include "arb_internal.h"

namespace arbk {
namespace {

constexpr int kAdjThreads = kAdjBlock;   // threads per cell (block)

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
    double* A2;    // [2 smem_cv] per CV: d rho (even), b beta (odd); then (u, e) of the back substitution
    double* PW;    // [2 smem_cv] per CV: P^ (even), W^ (odd)
    double* X;     // [smem_cv] solution (in PW's space, which the back substitution no longer needs)
    double* Bb;    // [smem_cv] factors b of split chains' lower parts (the rest of PW's space)
    double* GA;    // [4 smem_cv] reverse sweep: the gradient sums of the cell's CVs during a launch
    double* cdt;   // [smem_cv] C / dt
    double* dsig;  // [smem_cv] sum of the CV's axial conductances (own + children)
    double* glin;  // [smem_cv] passive conductance
    double* gelin; // [smem_cv] passive conductance x reversal
    double* rho;   // [smem_cv] scaling of the diagonal in the chain recurrence
    double* beta;  // [smem_cv] scaling of the right-hand side in the chain recurrence
    double* gcf;   // [smem_cv] g_k / c_k: u_k = gcf W^_k / P^_k
    double* srf;   // [smem_cv] s_k rho_k: e_k = srf P^_{k-1} / P^_k
    double* CDB;   // [2 smem_ch] a chain's elimination into its parent's diagonal (even) and rhs (odd)
    double* KPW;   // [2 smem_ch] per chain: s_h^2 rho_h (even), s_h g_h / c_h (odd)
    int32_t* par;  // [smem_cv] cell-local parent, -1 at the root
    int32_t* hidx; // [smem_cv] HH instance of the CV, -1 none
    int32_t* cvs;  // [smem_cv] CVs of the cell's chains, chain after chain (as ch_cvs)
    int32_t* prev; // [smem_cv] the CV before this one in its chain, -1 at a chain's tail
    int32_t* chp;  // [smem_ch + 1] cell-local chain -> range in cvs
    int32_t* kidp; // [smem_ch + 1] cell-local chain -> range in kids
    int32_t* kids; // [smem_ch] cell-local child chains
    int32_t* levb; // [smem_ch + 2] first cell-local chain of each level, then the end
    int32_t* fixa; // [smem_cv] anchor whose value a lower-part CV still needs, -1 none
    int32_t* tkb;  // [smem_ch + 2] first back-substitution task of each level, then the end
    int32_t* tk;   // [smem_tk][4] tasks: start, end (positions in cvs), kind, anchor CV
};

__device__ __forceinline__ Smem smem_of(const AdjArgs& a) {
    extern __shared__ double adj_smem[];
    Smem m;
    const int ncv = a.smem_cv, nch = a.smem_ch;
    m.A2 = adj_smem;
    m.PW = m.A2 + 2 * ncv;
    m.X = m.PW;
    m.Bb = m.PW + ncv;
    m.GA = m.PW + 2 * ncv;
    m.cdt = m.GA + 4 * ncv;
    m.dsig = m.cdt + ncv;
    m.glin = m.dsig + ncv;
    m.gelin = m.glin + ncv;
    m.rho = m.gelin + ncv;
    m.beta = m.rho + ncv;
    m.gcf = m.beta + ncv;
    m.srf = m.gcf + ncv;
    m.CDB = m.srf + ncv;
    m.KPW = m.CDB + 2 * nch;
    m.par = reinterpret_cast<int32_t*>(m.KPW + 2 * nch);
    m.hidx = m.par + ncv;
    m.cvs = m.hidx + ncv;
    m.prev = m.cvs + ncv;
    m.chp = m.prev + ncv;
    m.kidp = m.chp + nch + 1;
    m.kids = m.kidp + nch + 1;
    m.levb = m.kids + nch;
    m.fixa = m.levb + nch + 2;
    m.tkb = m.fixa + ncv;
    m.tk = m.tkb + nch + 2;
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
        sm.cdt[i] = a.cdt[off + i];
        sm.dsig[i] = a.dsig[off + i];
        sm.glin[i] = a.glin[off + i];
        sm.gelin[i] = a.gelin[off + i];
        sm.rho[i] = a.rho[off + i];
        sm.beta[i] = a.beta[off + i];
        sm.gcf[i] = a.gcf[off + i];
        sm.srf[i] = a.srf[off + i];
        sm.par[i] = a.parent[off + i];
        sm.hidx[i] = a.hidx[off + i];
        sm.prev[i] = a.prev[off + i];
        sm.fixa[i] = a.fixa[off + i];
        sm.cvs[i] = a.ch_cvs[cv0 + i];          // a cell's chains hold each of its CVs once
    }
    for (int64_t q = tid; q <= nq; q += kAdjThreads) {
        sm.chp[q] = (int32_t)(a.ch_cv_ptr[q0 + q] - cv0);
        sm.kidp[q] = (int32_t)(a.ch_kid_ptr[q0 + q] - k0);
    }
    for (int64_t q = tid; q < nq; q += kAdjThreads) {
        sm.KPW[2 * q] = a.kpw[2 * (q0 + q)];
        sm.KPW[2 * q + 1] = a.kpw[2 * (q0 + q) + 1];
    }
    for (int64_t k = tid; k < a.ch_kid_ptr[q0 + nq] - k0; k += kAdjThreads) sm.kids[k] = (int32_t)(a.ch_kids[k0 + k] - q0);
    for (int64_t L = tid; L < nlb; L += kAdjThreads) {
        sm.levb[L] = (int32_t)(a.lev_bound[l0 + L] - q0);
        sm.tkb[L] = a.tkb[l0 + L];
    }
    const int64_t t0 = a.tk_ptr[c], nt = a.tk_ptr[c + 1] - t0;
    for (int64_t t = tid; t < 4 * nt; t += kAdjThreads) sm.tk[t] = a.tk[4 * t0 + t];
    __syncthreads();
}

// Barrier of the block's first two warps (the elimination's P and W warps); barrier 0 stays
// the block-wide one.
__device__ __forceinline__ void elim_pair_sync() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

// Elimination of cell c by the first two warps (tid < 64), leaf chains first. Input: sm.A2 =
// (d rho, b beta) per CV. Output: P^ and W^ of every CV in sm.PW, and each chain's elimination
// into its parent in sm.CDB. The pivots do not depend on the right-hand side, so warp 0 runs the
// P^ recurrence of a level while warp 1 runs the W^ recurrence of the level before (which needs
// that level's P^), one lane per chain each; the two meet at a barrier between levels. Each step
// is one multiply-add:
//   warp 0: P^_k = (d_k rho_k) P^_{k-1} - P^_{k-2}     (P^_{-1} = 1, P^_0 = D_0)
//   warp 1: W^_k = (b_k beta_k) P^_{k-1} + W^_{k-1}    (W^_0 = B_0)
// An FP64 result that passes through an integer instruction (a select, a sign flip, a move
// under a predicate) before the next multiply-add costs tens of cycles here, so the loops have
// none: the negation is the multiply-add's own, each lane runs exactly its chain's steps (a
// remainder step after the loop unrolled by two), operands are loaded two steps ahead from
// always-valid indices, and a result is stored only after the next multiply-add is issued.
__device__ void tree_eliminate(const AdjArgs& a, int c, int tid, const Smem& sm) {
    const int nl = (int)(a.lev_off[c + 1] - a.lev_off[c]) - 1;
    const int w = tid >> 5, lane = tid & 31;
    for (int it = 0; it <= nl; ++it) {
        const int L = it - w;                    // warp 1 runs one level behind
        if (L >= 0 && L < nl) {
            for (int q = sm.levb[L] + lane; q < sm.levb[L + 1]; q += 32) {
                const int cs = sm.chp[q], len = sm.chp[q + 1] - cs;
                const int e0 = cs + len - 1;     // the tail's position in cvs; CV k of the chain is cvs[e0 - k]
                auto cv_at = [&](int k) -> int { return sm.cvs[k < len ? e0 - k : e0]; };
                const int x0 = sm.cvs[e0];
                // the tail: its own diagonal / right-hand side and its child chains' eliminations
                double acc = sm.A2[2 * x0 + w];
                for (int k = sm.kidp[q]; k < sm.kidp[q + 1]; ++k) acc += sm.CDB[2 * sm.kids[k] + w];
                sm.PW[2 * x0 + w] = acc;
                int xa = cv_at(1), xb = cv_at(2), ya = cv_at(3), yb = cv_at(4);
                int ks = x0;                     // CV of the result waiting to be stored
                if (w == 0) {
                    double X = acc, Y = 1.0;     // P^_{k-1}, P^_{k-2}
                    double Aa = sm.A2[2 * xa], Ab = sm.A2[2 * xb];
                    double S = acc;              // the result waiting to be stored
#define ARB_P_STEP(K, XV, YV, AV)                                                                \
    {                                                                                            \
        const double out_ = fma(AV, X, -Y);                                                      \
        sm.PW[2 * ks] = S;                                                                       \
        ks = XV;                                                                                 \
        S = out_;                                                                                \
        AV = sm.A2[2 * YV];                                                                      \
        XV = YV;                                                                                 \
        YV = cv_at((K) + 4);                                                                     \
        Y = X;                                                                                   \
        X = out_;                                                                                \
    }
                    int k = 1;
                    for (; k + 1 < len; k += 2) {
                        ARB_P_STEP(k, xa, ya, Aa)
                        ARB_P_STEP(k + 1, xb, yb, Ab)
                    }
                    if (k < len) ARB_P_STEP(k, xa, ya, Aa)
#undef ARB_P_STEP
                    sm.PW[2 * ks] = S;
                    // the head's elimination into the parent's diagonal: -s_h^2 / D_h
                    if (sm.par[sm.cvs[cs]] >= 0) sm.CDB[2 * q] = (-sm.KPW[2 * q] * Y) * rcp_nr(X);
                } else {
                    double Y = acc;              // W^_{k-1}
                    // operands of step k: b_k beta_k and P^_{k-1} (of the CV before k in the chain)
                    double Ba = sm.A2[2 * xa + 1], Bb = sm.A2[2 * xb + 1];
                    double Pa = sm.PW[2 * x0], Pb = sm.PW[2 * xa];
                    double S = acc;
#define ARB_W_STEP(K, XV, YV, BV, PV)                                                            \
    {                                                                                            \
        const double out_ = fma(BV, PV, Y);                                                      \
        sm.PW[2 * ks + 1] = S;                                                                   \
        ks = XV;                                                                                 \
        S = out_;                                                                                \
        BV = sm.A2[2 * YV + 1];                                                                  \
        PV = sm.PW[2 * cv_at((K) + 1)];                                                          \
        XV = YV;                                                                                 \
        YV = cv_at((K) + 4);                                                                     \
        Y = out_;                                                                                \
    }
                    int k = 1;
                    for (; k + 1 < len; k += 2) {
                        ARB_W_STEP(k, xa, ya, Ba, Pa)
                        ARB_W_STEP(k + 1, xb, yb, Bb, Pb)
                    }
                    if (k < len) ARB_W_STEP(k, xa, ya, Ba, Pa)
#undef ARB_W_STEP
                    sm.PW[2 * ks + 1] = S;
                    // the head's elimination into the parent's right-hand side: s_h B_h / D_h
                    const int h = sm.cvs[cs];
                    if (sm.par[h] >= 0) sm.CDB[2 * q + 1] = (sm.KPW[2 * q + 1] * Y) * rcp_nr(sm.PW[2 * h]);
                }
            }
        }
        elim_pair_sync();
    }
}

// Coefficients of the back substitution (all threads): u_k = B_k / D_k, e_k = s_k / D_k per CV,
// into sm.A2 (whose elimination operands are used up).
__device__ void tree_coefficients(int n, const Smem& sm) {
    for (int li = threadIdx.x; li < n; li += kAdjThreads) {
        const int pv = sm.prev[li];
        const double Pp = pv >= 0 ? sm.PW[2 * pv] : 1.0;
        const double r = rcp_nr(sm.PW[2 * li]);
        const double u = (sm.gcf[li] * sm.PW[2 * li + 1]) * r;
        const double e = (sm.srf[li] * Pp) * r;
        sm.A2[2 * li] = u;
        sm.A2[2 * li + 1] = e;
    }
}

// Back substitution (first warp): levels in reverse order, V_k = u_k + e_k V_parent along each
// chain from its head (V_parent from the parent chain; e = 0 at the root), one multiply-add per
// CV, one lane per task. In a level with few chains the host split each longer chain in two:
// one lane takes the upper part as usual, and two lanes take the lower part at once, one
// forming the offsets a_k (the same recurrence from V_anchor = 0) into sm.X, the other the
// factors b_k (u masked to 0, from 1) into sm.Bb, so that V_k = a_k + b_k V_anchor with the
// anchor the upper part's last CV. The three run the same instructions. A lower part's tail is
// fixed at the end of the level (child chains hang from tails); its other CVs are fixed where the
// solution is read (sm.fixa). Operands come two CVs ahead from always-valid indices and each
// value is stored after the next multiply-add, so no integer instruction sits between them.
__device__ void tree_substitute(const AdjArgs& a, int c, int lane, const Smem& sm) {
    const int nl = (int)(a.lev_off[c + 1] - a.lev_off[c]) - 1;
    for (int L = nl - 1; L >= 0; --L) {
        for (int t = sm.tkb[L] + lane; t < sm.tkb[L + 1]; t += 32) {
            const int cs = sm.tk[4 * t], ce = sm.tk[4 * t + 1], kind = sm.tk[4 * t + 2];
            auto cv_at = [&](int i) -> int { return sm.cvs[i < ce ? i : ce - 1]; };
            const int x0 = sm.cvs[cs];
            const int32_t p = sm.par[x0];
            double vp = kind == 2 ? 1.0 : 0.0;
            if (kind == 0 && p >= 0) vp = sm.X[p];          // e = 0 at the root
            const int umask = kind == 2 ? 0 : -1;             // the factors' recurrence has u = 0
            double* out = kind == 2 ? sm.Bb : sm.X;
            auto u_at = [&](int x) -> double {
                const double u = sm.A2[2 * x];
                return __hiloint2double(__double2hiint(u) & umask, __double2loint(u) & umask);
            };
            int xa = x0, xb = cv_at(cs + 1), ya = cv_at(cs + 2), yb = cv_at(cs + 3);
            double ua = u_at(xa), ea = sm.A2[2 * xa + 1];
            double ub = u_at(xb), eb = sm.A2[2 * xb + 1];
            int ks = -1;                          // CV of the value waiting to be stored
#define ARB_SUBST_STEP(I, XV, YV, U, E)                                                          \
    {                                                                                            \
        const double v_ = fma(E, vp, U);                                                         \
        if (ks >= 0) out[ks] = vp;                                                               \
        ks = XV;                                                                                 \
        U = u_at(YV);                                                                            \
        E = sm.A2[2 * YV + 1];                                                                   \
        XV = YV;                                                                                 \
        YV = cv_at((I) + 4);                                                                     \
        vp = v_;                                                                                 \
    }
            int i = cs;
            for (; i + 1 < ce; i += 2) {
                ARB_SUBST_STEP(i, xa, ya, ua, ea)
                ARB_SUBST_STEP(i + 1, xb, yb, ub, eb)
            }
            if (i < ce) ARB_SUBST_STEP(i, xa, ya, ua, ea)
#undef ARB_SUBST_STEP
            out[ks] = vp;
        }
        __syncwarp();
        for (int t = sm.tkb[L] + lane; t < sm.tkb[L + 1]; t += 32)
            if (sm.tk[4 * t + 2] == 1) {                      // a lower part's tail: V = a + b V_anchor
                const int x = sm.cvs[sm.tk[4 * t + 1] - 1];
                sm.X[x] = fma(sm.Bb[x], sm.X[sm.tk[4 * t + 3]], sm.X[x]);
            }
        __syncwarp();
    }
}

// The solution at cell-local CV li, with a split chain's lower part completed.
__device__ __forceinline__ double solution(const Smem& sm, int li) {
    const int an = sm.fixa[li];
    return an >= 0 ? fma(sm.Bb[li], sm.X[an], sm.X[li]) : sm.X[li];
}

// mode 0: steps [s0, s1) from the running state (a.V, a.Y), in place, with a checkpoint
//         before every step that is a multiple of ckpt, and the loss;
// mode 1: steps [s0, s1) from checkpoint s0 / ckpt, every state kept in segment buffer buf;
// mode 2: steps [s0, s1) from the running state, every state kept in segment buffer buf, and
//         the loss (the last segment of the forward pass, which then needs no recompute).
__device__ void forward_cell(const AdjArgs& a, int c, int64_t s0, int64_t s1, int mode, int buf) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t off = a.off[c], n = a.off[c + 1] - off;
    double* const segV = a.segV[buf];
    double* const segY = a.segY[buf];
    double* const segG = a.segG[buf];
    const int64_t nhh = a.n_hh;
    const Smem sm = smem_of(a);
    load_cell(a, c, sm);
    if (mode != 0) {
        const double* cV = mode == 1 ? a.ckV + (s0 / a.ckpt) * a.n_cv : a.V;
        const double* cY = mode == 1 ? a.ckY + (s0 / a.ckpt) * 3 * nhh : a.Y;
        for (int64_t i = off + tid; i < off + n; i += kAdjThreads) {
            segV[i] = cV[i];
            const int32_t j = sm.hidx[i - off];
            if (j >= 0)
                for (int g = 0; g < 3; ++g) segY[g * nhh + j] = cY[g * nhh + j];
        }
        __syncthreads();
    }
    // each thread's loss sum runs over all steps in order, across the two forward launches
    double lsum = mode == 2 ? a.loss_part[(int64_t)c * kAdjThreads + tid] : 0.0;
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
            sm.A2[2 * li] = (sm.cdt[li] + G + sm.dsig[li]) * sm.rho[li];
            sm.A2[2 * li + 1] = (sm.cdt[li] * Vs[i] + GE) * sm.beta[li];
        }
        __syncthreads();
        if (tid < 64) {
            if (tid == 0) {
                const double t = (double)(a.k0 + s) * a.dt;
                for (int64_t q = a.st_ptr[c]; q < a.st_ptr[c + 1]; ++q)
                    if (a.st_on[q] <= t && t < a.st_on[q] + a.st_dur[q]) {
                        const int64_t x = a.st_cv[q] - off;
                        sm.A2[2 * x + 1] = fma(a.st_amp[q], sm.beta[x], sm.A2[2 * x + 1]);
                    }
            }
            tree_eliminate(a, c, tid, sm);
        }
        __syncthreads();
        tree_coefficients((int)n, sm);
        __syncthreads();
        if (tid < 32) tree_substitute(a, c, lane, sm);
        __syncthreads();
        // new voltage, gates with it, loss
        for (int64_t i = off + tid; i < off + n; i += kAdjThreads) {
            const double v = solution(sm, (int)(i - off));
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
                } else if (hh_gates_tab_dv(a.hh_tab, a.hh_dtab, v, xg, dvg, eg)) {
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
            if (mode != 1) {
                const int32_t o = a.obs[i];
                if (o >= 0) {
                    const double e = v - a.target[s * a.n_obs + o];
                    lsum += a.loss_scale * e * e;
                }
            }
        }
        __syncthreads();
    }
    if (mode == 0) a.loss_part[(int64_t)c * kAdjThreads + tid] = lsum;
    if (mode == 2) {
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

// Asks L2 for the 128-byte lines of count doubles from p (threads of the block in turn), every
// address inside the range.
__device__ __forceinline__ void prefetch_l2(const double* p, int64_t count, int tid) {
    const char* b = reinterpret_cast<const char*>(p);
    const int64_t bytes = count * 8;
    for (int64_t o = (int64_t)tid * 128; o < bytes; o += (int64_t)kAdjThreads * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(b + o));
    if (tid == 0 && bytes > 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(b + bytes - 8));
}

// Reverse sweep over the segment [s0, s1) held in segment buffer buf.
__device__ void reverse_cell(const AdjArgs& a, int c, int64_t s0, int64_t s1, int buf) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t off = a.off[c], n = a.off[c + 1] - off;
    const double* const segV = a.segV[buf];
    const double* const segY = a.segY[buf];
    const double* const segG = a.segG[buf];
    const int64_t nhh = a.n_hh, ncv = a.n_cv;
    const Smem sm = smem_of(a);
    load_cell(a, c, sm);
    // the cell's gradient sums stay in shared memory for the launch (each thread keeps the CVs it
    // updates), in the same order of additions as in global memory
    for (int64_t i = off + tid; i < off + n; i += kAdjThreads)
        for (int g = 0; g < 4; ++g) sm.GA[4 * (i - off) + g] = a.gacc[g * ncv + i];
    // the cell's range of HH instances, for the prefetch of the segment rows
    __shared__ int hlo, hhi;
    if (tid == 0) { hlo = 0x7fffffff; hhi = -1; }
    __syncthreads();
    for (int64_t li = tid; li < n; li += kAdjThreads) {
        const int32_t j = sm.hidx[li];
        if (j >= 0) { atomicMin(&hlo, j); atomicMax(&hhi, j); }
    }
    __syncthreads();
    const int64_t j0 = hlo, nh = hhi >= hlo ? (int64_t)hhi - hlo + 1 : 0;
    for (int64_t s = s1 - 1; s >= s0; --s) {
        // the rows of step s - 1 were written a segment ago and are read from DRAM: ask for them
        // now, a step ahead (the rows of step s + 1 it also reads are still cached)
        if (s > s0) {
            const int64_t sp = s - 1 - s0;
            prefetch_l2(segV + sp * ncv + off, n, tid);
            for (int g = 0; g < 3; ++g) prefetch_l2(segY + (sp * 3 + g) * nhh + j0, nh, tid);
            for (int g = 0; g < 6; ++g) prefetch_l2(segG + (sp * 6 + g) * nhh + j0, nh, tid);
        }
        const double* V0 = segV + (s - s0) * ncv;
        const double* V1 = V0 + ncv;
        const double* Y0 = segY + (s - s0) * 3 * nhh;
        // Vbar = (C/dt) lam + dL/dV^{s+1} + dPhi/dV^T ybar; A(y^s); ybar <- dPhi/dy ybar
        for (int64_t i = off + tid; i < off + n; i += kAdjThreads) {
            const int64_t li = i - off;
            double G, GE;
            membrane(a, sm.glin[li], sm.gelin[li], sm.hidx[li], Y0, G, GE);
            sm.A2[2 * li] = (sm.cdt[li] + G + sm.dsig[li]) * sm.rho[li];
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
            sm.A2[2 * li + 1] = vb * sm.beta[li];
        }
        __syncthreads();
        if (tid < 64) tree_eliminate(a, c, tid, sm);
        __syncthreads();
        tree_coefficients((int)n, sm);
        __syncthreads();
        if (tid < 32) tree_substitute(a, c, lane, sm);
        __syncthreads();
        // lam_s; gradient terms; gate adjoint of y^s
        // (dA/dtheta V^{s+1} - dRHS/dtheta) against lam_s: with w = lam_s, per unit density
        //   cm:    (area 1e-5 / dt) (V^s - V^{s+1}) w          (nF/ms per uF/cm^2)
        //   gnabar: area 1e-2 m^3 h (E_Na - V^{s+1}) w, gkbar: area 1e-2 n^4 (E_K - V^{s+1}) w,
        //   gl:     area 1e-2 (E_L - V^{s+1}) w;
        // the gate adjoints take d(G V - GE)/dgate from the same terms. Per-CV factors come from
        // the host (kcm = area 1e-5 / dt, ksc = area 1e-2), so no division is left here.
        for (int64_t i = off + tid; i < off + n; i += kAdjThreads) {
            const double lam = solution(sm, (int)(i - off));
            a.lam[i] = lam;
            const double v1 = V1[i];
            double* ga = sm.GA + 4 * (i - off);
            ga[3] = fma(lam * (V0[i] - v1), a.kcm[i], ga[3]);
            const int32_t j = sm.hidx[i - off];
            if (j >= 0) {
                const double m = Y0[j], h = Y0[nhh + j], nn = Y0[2 * nhh + j];
                const double lna = lam * (kENa - v1), lk = lam * (kEK - v1), ll = lam * (kEL - v1);
                const double sc = a.ksc[i];
                const double m2 = m * m, m2h = m2 * h, n2 = nn * nn, n3 = n2 * nn;
                ga[0] = fma(m2h * m * sc, lna, ga[0]);
                ga[1] = fma(n3 * nn * sc, lk, ga[1]);
                ga[2] = fma(ll, sc, ga[2]);
                const double g3 = a.gna3[j];
                a.ybar[j] = fma(g3 * m2h, lna, a.ybar[j]);
                a.ybar[nhh + j] = fma(a.gna[j] * (m2 * m), lna, a.ybar[nhh + j]);
                a.ybar[2 * nhh + j] = fma(a.gk4[j] * n3, lk, a.ybar[2 * nhh + j]);
            }
        }
        __syncthreads();
    }
    for (int64_t i = off + tid; i < off + n; i += kAdjThreads)
        for (int g = 0; g < 4; ++g) a.gacc[g * ncv + i] = sm.GA[4 * (i - off) + g];
}

// Forward pass with the loss (mode 0: with checkpoints; mode 2: into segment buffer buf): one
// block per cell.
__global__ void __launch_bounds__(kAdjThreads) k_adj_forward(AdjArgs a, int64_t s0, int64_t s1, int mode, int buf) {
    forward_cell(a, blockIdx.x, s0, s1, mode, buf);
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

size_t adj_smem_bytes(const AdjArgs& a) { return adj_smem_bytes_for(a.smem_cv, a.smem_ch, a.smem_tk); }

cudaError_t adj_prepare(const AdjArgs& a) {
    const int bytes = (int)adj_smem_bytes(a);
    cudaError_t e = cudaFuncSetAttribute(k_adj_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_adj_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_adj_forward(const AdjArgs& a, int64_t s0, int64_t s1, int mode, int buf, cudaStream_t s) {
    if (a.n_cells == 0 || s1 <= s0) return cudaSuccess;
    k_adj_forward<<<a.n_cells, kAdjThreads, adj_smem_bytes(a), s>>>(a, s0, s1, mode, buf);
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
