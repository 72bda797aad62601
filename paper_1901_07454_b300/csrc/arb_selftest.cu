// arb_math_eval: the library's own FP64 elementary functions on caller arrays, so that they
// can be checked against CUDA's functions and against the oracle's rates.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/arb.h"
#include "arb_hh.cuh"

namespace {

__global__ void k_math_eval(int32_t fn, int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        if (fn == ARB_FN_EXP) {
            y[i] = arbk::exp_t(v);
        } else if (fn == ARB_FN_EXPM1) {
            y[i] = arbk::expm1_t(v);
        } else {
            const arbk::Rates r = arbk::hh_rates(v);
            double* o = y + 6 * i;
            o[0] = r.am; o[1] = r.bm; o[2] = r.ah; o[3] = r.bh; o[4] = r.an; o[5] = r.bn;
        }
    }
}

}  // namespace

namespace arbk {
void set_handle_free_error(const std::string& msg);
}

extern "C" arb_status arb_math_eval(int32_t fn, int64_t n, const double* x, double* y, void* stream) {
    arbk::set_handle_free_error("");
    if (fn != ARB_FN_EXP && fn != ARB_FN_EXPM1 && fn != ARB_FN_HH_RATES) {
        arbk::set_handle_free_error("arb_math_eval: unknown function");
        return ARB_E_ARG;
    }
    if (n < 0 || (n > 0 && (!x || !y))) {
        arbk::set_handle_free_error("arb_math_eval: bad arrays");
        return ARB_E_ARG;
    }
    if (n == 0) return ARB_OK;
    const int64_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    k_math_eval<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(fn, n, x, y);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        arbk::set_handle_free_error(std::string("arb_math_eval: ") + cudaGetErrorString(e));
        return ARB_E_CUDA;
    }
    return ARB_OK;
}
