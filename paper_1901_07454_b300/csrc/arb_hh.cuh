// Hodgkin-Huxley rate functions and numeric helpers shared by the stepping kernels and the
// adjoint kernels.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "arb_exp_table.h"
#include "arb_internal.h"

namespace arbk {

// 1/x (pivots of the implicit scheme, and the quotients of the FP64 HH rates and gate
// updates): the hardware estimate (about 20 correct bits) refined by one third-order step,
// r <- r + r (e + e^2) with e = 1 - x r, which triples the number of correct bits (error e^3),
// so the result is within an ulp or so of 1/x. x must be nonzero with |x| between about 1e-300
// and 1e300 (the estimate flushes subnormal results to zero); the callers' values are.
__device__ __forceinline__ double rcp_nr(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}


// exp(x) for |x| < 700 by Tang's table-driven method (ACM TOMS 15(2), 1989): x = k ln2/64 + r
// with k = 64 m + j and |r| <= ln2/128, exp(x) = 2^m 2^(j/64) exp(r); exp(r) - 1 is its
// Taylor polynomial to r^5 (the first omitted term is below 4e-17 there), 2^(j/64) comes from a
// 64-entry table and 2^m is added to the exponent field. 10 FP64 operations; within about an
// ulp of exp(x).
__device__ __forceinline__ double exp_t(double x) {
    const double kShift = 6755399441055744.0;          // 1.5 * 2^52: adding it rounds to an integer
    const double t = fma(x, kExpInvLn2x64, kShift);
    const int k = __double2loint(t);                    // the rounded integer, two's complement
    const double kd = t - kShift;
    double r = fma(-kd, kExpLn2Hi, x);
    r = fma(-kd, kExpLn2Lo, r);
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(r, q, 1.0 / 6.0);
    q = fma(r, q, 0.5);
    q = fma(r, q, 1.0);
    const double T = __ldg(&kExpTable[k & 63]);
    const double y = fma(T, r * q, T);
    return __hiloint2double(__double2hiint(y) + ((k >> 6) << 20), __double2loint(y));
}

// e^x - 1: the library's expm1 where |x| < 0.1 (where e^x - 1 would cancel), else exp_t - 1
// (relative error of the difference at most ~10 ulp there).
__device__ __forceinline__ double expm1_t(double x) { return fabs(x) < 0.1 ? expm1(x) : exp_t(x) - 1.0; }

// ------------------------------------------------------------------------------------------
// Hodgkin-Huxley rates (1/ms) and exact gate update at frozen V, in the precision MT.
// The model (classic squid axon at 6.3 degC) is the one named by the paper's benchmark
// (Sec. "Benchmarks", "Models": Hodgkin-Huxley soma, passive dendrites).

__device__ __forceinline__ float exprelr_f(float x) { return x == 0.0f ? 1.0f : x / expm1f(x); }

struct Rates { double am, bm, ah, bh, an, bn; };
struct RatesF { float am, bm, ah, bh, an, bn; };

// FP64 rates from three transcendentals instead of six: with x1 = -(v+40)/10,
// exp(-(v+35)/10) = e^{x1} e^{1/2} and exp(-(v+55)/10) = e^{x1} e^{-3/2}, where e^{x1} = expm1(x1)
// + 1 only ever enters a sum with 1 (so its absolute error, not its relative one, matters);
// exp(-(v+65)/20) = exp(-(v+65)/80)^4. Near the removable point of alpha_n (|x2| < 0.1) its
// expm1 is taken directly, since e^{x2} - 1 formed from e^{x1} would cancel there.
__device__ __forceinline__ Rates hh_rates_em(double v, double& em1, double& em2) {
    Rates r;
    const double x1 = (v + 40.0) * -0.1;
    em1 = expm1_t(x1);
    r.am = x1 == 0.0 ? 1.0 : x1 * rcp_nr(em1);
    const double e80 = exp_t((v + 65.0) * -0.0125);
    const double e40 = e80 * e80;
    r.bn = 0.125 * e80;
    r.ah = 0.07 * (e40 * e40);
    r.bm = 4.0 * exp_t((v + 65.0) * (-1.0 / 18.0));
    const double ex1 = em1 + 1.0;
    r.bh = rcp_nr(fma(ex1, 1.6487212707001282, 1.0));          // e^{1/2}
    const double x2 = (v + 55.0) * -0.1;
    em2 = fabs(x2) < 0.1 ? expm1(x2) : fma(ex1, 0.22313016014842982, -1.0);   // e^{-3/2}
    r.an = 0.1 * (x2 == 0.0 ? 1.0 : x2 * rcp_nr(em2));
    return r;
}

__device__ __forceinline__ Rates hh_rates(double v) {
    double em1, em2;
    return hh_rates_em(v, em1, em2);
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

// exp(-dt (a + b)): the decay factor of a gate over one step at frozen V.
__device__ __forceinline__ double gate_decay(double a, double b, double dt) { return exp_t(-dt * (a + b)); }

__device__ __forceinline__ double gate(double x, double a, double b, double dt) {
    const double xinf = a * rcp_nr(a + b);
    return xinf + (x - xinf) * gate_decay(a, b, dt);
}
// The same update with e = exp(-dt (a + b)) already formed.
__device__ __forceinline__ double gate_e(double x, double a, double b, double e) {
    const double xinf = a * rcp_nr(a + b);
    return xinf + (x - xinf) * e;
}
__device__ __forceinline__ float gate(float x, float a, float b, float dt) {
    const float s = a + b;
    const float xinf = a / s;
    return xinf + (x - xinf) * expf(-dt * s);
}

// Gate update of one HH instance from the tabulated x_inf and exp(-dt (alpha + beta)) (see
// kHHTabVlo); false when there is no table or V lies outside it.
__device__ __forceinline__ bool hh_gates_tab(const double* tab, double vd, double& m, double& h, double& n) {
    const double tv = fma(vd, kHHTabPerMV, -kHHTabVlo * kHHTabPerMV);
    if (tab == nullptr || !(tv >= 0.0 && tv < (double)kHHTabN)) return false;
    const int it = (int)tv;
    const double s = tv - (double)it;
    const double2* c = reinterpret_cast<const double2*>(tab + (size_t)it * kHHTabStride);
    double f[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const double2 lo = __ldg(c + 2 * q), hi = __ldg(c + 2 * q + 1);
        f[q] = fma(fma(fma(hi.y, s, hi.x), s, lo.y), s, lo.x);
    }
    m = fma(m - f[0], f[1], f[0]);
    h = fma(h - f[2], f[3], f[2]);
    n = fma(n - f[4], f[5], f[4]);
    return true;
}

// FP32 mechanisms (mixed precision): the same update from the table's coefficients rounded to
// float, evaluated in float at the interval offset of the FP64 voltage; false when there is no
// table or V lies outside it.
__device__ __forceinline__ bool hh_gates_tab_f(const float* tab, double vd, float& m, float& h, float& n) {
    const double tv = fma(vd, kHHTabPerMV, -kHHTabVlo * kHHTabPerMV);
    if (tab == nullptr || !(tv >= 0.0 && tv < (double)kHHTabN)) return false;
    const int it = (int)tv;
    const float s = (float)(tv - (double)it);
    const float4* c = reinterpret_cast<const float4*>(tab + (size_t)it * kHHTabStride);
    float f[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 cc = __ldg(c + q);
        f[q] = fmaf(fmaf(fmaf(cc.w, s, cc.z), s, cc.y), s, cc.x);
    }
    m = fmaf(m - f[0], f[1], f[0]);
    h = fmaf(h - f[2], f[3], f[2]);
    n = fmaf(n - f[4], f[5], f[4]);
    return true;
}

// The same from the table, with what the reverse sweep of the adjoint needs: each gate x of
// (m, h, n) becomes x_inf + (x - x_inf) e, with dx'/dV = x_inf' (1 - e) + (x - x_inf) e' (slopes
// of the cubics, from dtab: per interval and quantity the coefficients of the slope per mV) in
// dv and e in ef, in that order. False when there is no table or V lies outside it.
struct Gates3 { double m, h, n; };
__device__ __forceinline__ bool hh_gates_tab_dv(const double* tab, const double* dtab, double vd, Gates3& x, Gates3& dv,
                                                Gates3& ef) {
    const double tv = fma(vd, kHHTabPerMV, -kHHTabVlo * kHHTabPerMV);
    if (tab == nullptr || !(tv >= 0.0 && tv < (double)kHHTabN)) return false;
    const int it = (int)tv;
    const double s = tv - (double)it;
    const double2* c = reinterpret_cast<const double2*>(tab + (size_t)it * kHHTabStride);
    const double2* cd = reinterpret_cast<const double2*>(dtab + (size_t)it * kHHTabStride);
    double f[6], g[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const double2 lo = __ldg(c + 2 * q), hi = __ldg(c + 2 * q + 1);
        const double2 dlo = __ldg(cd + 2 * q), dhi = __ldg(cd + 2 * q + 1);
        f[q] = fma(fma(fma(hi.y, s, hi.x), s, lo.y), s, lo.x);
        g[q] = fma(fma(dhi.x, s, dlo.y), s, dlo.x);
    }
    auto one = [&](double& xx, double& dd, double& ee, int q) {
        const double xinf = f[2 * q], e = f[2 * q + 1], d = xx - xinf;
        dd = fma(d, g[2 * q + 1], g[2 * q] * (1.0 - e));
        ee = e;
        xx = fma(d, e, xinf);
    };
    one(x.m, dv.m, ef.m, 0);
    one(x.h, dv.h, ef.h, 1);
    one(x.n, dv.n, ef.n, 2);
    return true;
}

// ------------------------------------------------------------------------------------------
// Derivatives for the discrete adjoint (FP64).

// d/dx of x / (e^x - 1): for |x| < 0.1 the derivative of the Bernoulli series
// sum_n B_n x^n / n! up to x^7 (the first omitted term is below 3e-16 there), elsewhere the
// closed form (e^x - 1 - x e^x) / (e^x - 1)^2.
__device__ __forceinline__ double exprelr_deriv_d(double x) {
    if (fabs(x) < 0.1) {
        const double x2 = x * x;
        return -0.5 + x * (1.0 / 6.0 + x2 * (-1.0 / 180.0 + x2 * (1.0 / 5040.0 - x2 * (1.0 / 151200.0))));
    }
    const double em = expm1(x);
    return (em - x * (em + 1.0)) / (em * em);
}

// d/dx of x / (e^x - 1) given em = e^x - 1 (the closed form, for |x| >= 0.1).
__device__ __forceinline__ double exprelr_deriv_em(double x, double em) {
    return (em - x * (em + 1.0)) / (em * em);
}

// Rates and their derivatives together: the derivatives of alpha_m and alpha_n reuse the
// e^x - 1 of the rates where the closed form applies (|x| >= 0.1).
__device__ __forceinline__ void hh_rates_derivs(double v, Rates& r, Rates& d) {
    double em1, em2;
    r = hh_rates_em(v, em1, em2);
    const double x1 = (v + 40.0) * -0.1, x2 = (v + 55.0) * -0.1;
    const double dm = fabs(x1) < 0.1 ? exprelr_deriv_d(x1) : exprelr_deriv_em(x1, em1);
    const double dn = fabs(x2) < 0.1 ? exprelr_deriv_d(x2) : exprelr_deriv_em(x2, em2);
    d.am = -0.1 * dm;
    d.bm = r.bm * (-1.0 / 18.0);
    d.ah = r.ah * -0.05;
    d.bh = r.bh * (1.0 - r.bh) * 0.1;
    d.an = -0.01 * dn;
    d.bn = r.bn * -0.0125;
}

// d/dV of the exact gate update xinf + (x - xinf) exp(-dt s), s = a + b, at frozen V;
// e = exp(-dt s) is passed in.
__device__ __forceinline__ double gate_dv(double x, double a, double b, double da, double db, double dt, double e) {
    const double s = a + b, ds = da + db;
    const double xinf = a / s;
    const double dxinf = (da * s - a * ds) / (s * s);
    return dxinf * (1.0 - e) - (x - xinf) * e * dt * ds;
}

}  // namespace arbk
