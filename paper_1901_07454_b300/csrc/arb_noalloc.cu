// arb_solve_trees_noalloc: the tree (Hines) solve of the library for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the solve: code running
// while a stream is being captured into a CUDA graph (allocation calls would break the
// capture), code inside a host callback or an allocator-less embedded runtime, or a caller
// whose memory pool is fixed up front. This entry point therefore takes only the caller's
// input and output arrays and keeps its per-CV scratch (the eliminated pivots and right-hand
// sides) and one status word in file-scope device arrays of fixed size. Every GPU that loads
// the library holds them until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/arb.h"

namespace {

// Scratch: two doubles per CV (pivot, right-hand side), at most kNoAllocMaxCV CVs per call.
constexpr int64_t kNoAllocMaxCV = 262144;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxCV];
// Nonzero when the call's cv_offset is not a valid CSR over [0, n_cv): set by k_check_offsets,
// read by k_solve_trees. Cleared at the start of every call.
static __device__ __align__(256) int32_t g_noalloc_bad[1];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device
void* g_noalloc_bad_ptr[kMaxDevices] = {};   // ... and of g_noalloc_bad

// cv_offset must start at 0, never decrease and end at n_cv; otherwise two cells could own the
// same CVs (and the same scratch rows), so the whole call is refused on the device.
__global__ void k_check_offsets(int32_t n_cells, const int64_t* __restrict__ cv_offset, int64_t n_cv) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_cells; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t off = cv_offset[c], end = cv_offset[c + 1];
        bool ok = off <= end;
        if (c == 0) ok = ok && off == 0;
        if (c == n_cells - 1) ok = ok && end == n_cv;
        if (!ok) g_noalloc_bad[0] = 1;
    }
}

// One thread per cell: elimination from the leaves (highest local index) to the root, then
// back substitution. parent[i] < i inside a cell, parent of the first CV -1. Both the pivots
// and the right-hand side are copied into the scratch first, so nothing from an earlier call
// is read. With an invalid cv_offset every x is NaN; a cell whose parents break the rule
// gets NaN over its own CVs.
__global__ void k_solve_trees(int32_t n_cells, const int64_t* __restrict__ cv_offset, const int32_t* __restrict__ parent,
                              const double* __restrict__ d, const double* __restrict__ a, const double* __restrict__ b,
                              double* __restrict__ x, int64_t n_cv, double* __restrict__ scratch) {
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    if (g_noalloc_bad[0]) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_cv; i += (int64_t)gridDim.x * blockDim.x)
            x[i] = qnan;
        return;
    }
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_cells; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t off = cv_offset[c], end = cv_offset[c + 1];
        const int64_t n = end - off;
        double* dd = scratch + off;
        double* bb = scratch + kNoAllocMaxCV + off;
        bool ok = true;
        for (int64_t i = 0; i < n; ++i) {
            dd[i] = d[off + i];
            bb[i] = b[off + i];
            const int32_t p = parent[off + i];
            if ((i == 0 && p != -1) || (i > 0 && (p < 0 || p >= i))) ok = false;
        }
        if (!ok) {
            for (int64_t i = 0; i < n; ++i) x[off + i] = qnan;
            continue;
        }
        for (int64_t i = n - 1; i >= 1; --i) {
            const int32_t p = parent[off + i];
            const double f = a[off + i] / dd[i];
            dd[p] -= f * a[off + i];
            bb[p] -= f * bb[i];
        }
        if (n > 0) x[off] = bb[0] / dd[0];
        for (int64_t i = 1; i < n; ++i) x[off + i] = (bb[i] - a[off + i] * x[off + parent[off + i]]) / dd[i];
    }
}

}  // namespace

namespace arbk {
void set_handle_free_error(const std::string& msg);   // read back with arb_last_error(NULL)
}

static arb_status noalloc_fail(arb_status st, const std::string& msg) {
    arbk::set_handle_free_error(msg);
    return st;
}

extern "C" arb_status arb_solve_trees_noalloc(int32_t n_cells, int64_t n_cv, const int64_t* cv_offset,
                                              const int32_t* parent, const double* d, const double* a,
                                              const double* b, double* x, void* stream) {
    arbk::set_handle_free_error("");
    if (n_cells < 0 || n_cv < 0) return noalloc_fail(ARB_E_ARG, "n_cells and n_cv must be >= 0");
    if (n_cv > kNoAllocMaxCV)
        return noalloc_fail(ARB_E_ARG, "arb_solve_trees_noalloc: " + std::to_string(n_cv) +
                                           " CVs exceed the fixed scratch of " + std::to_string(kNoAllocMaxCV) + " CVs");
    if (n_cells == 0 || n_cv == 0) return ARB_OK;
    if (!cv_offset || !parent || !d || !a || !b || !x) return noalloc_fail(ARB_E_ARG, "NULL array");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(ARB_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(ARB_E_ARG, "device index out of range");
    void* scratch = nullptr;
    void* bad = nullptr;
    {
        // set-up, once per device, with that device current: the host-side symbols are only
        // stand-ins, the kernels need the device addresses
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            void* q = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return noalloc_fail(ARB_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            e = cudaGetSymbolAddress(&q, g_noalloc_bad);
            if (e != cudaSuccess || !q)
                return noalloc_fail(ARB_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_ptr[dev] = p;
            g_noalloc_bad_ptr[dev] = q;
        }
        scratch = g_noalloc_ptr[dev];
        bad = g_noalloc_bad_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return noalloc_fail(ARB_E_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int threads = 128;
    const int blocks = (int)((n_cells + threads - 1) / threads);
    k_check_offsets<<<blocks, threads, 0, s>>>(n_cells, cv_offset, n_cv);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(ARB_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    const int64_t work = n_cells > n_cv ? n_cells : n_cv;   // the all-NaN path covers every CV
    const int sblocks = (int)((work + threads - 1) / threads);
    k_solve_trees<<<sblocks, threads, 0, s>>>(n_cells, cv_offset, parent, d, a, b, x, n_cv, (double*)scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(ARB_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return ARB_OK;
}
