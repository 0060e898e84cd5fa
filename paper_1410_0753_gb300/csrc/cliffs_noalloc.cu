// Depth-jump filter for callers that cannot allocate device memory.
//
// Same filter as cliffs_set_bathy's (wet nodes raised to min_depth, then row and column
// Jacobi passes of eqs. (dstab), (newdw), (newdc) until a pass changes nothing, at most
// 100), but its scratch (the second Jacobi buffer and the "changed" flag) is a fixed static
// device array instead of memory from cudaMalloc, and it writes into memory the caller owns.
// Nothing here calls cudaMalloc, cudaFree or any allocating library routine.
#include <cstdio>
#include <mutex>

#include "cliffs.h"
#include "internal.h"

namespace {

// The scratch every device that loads the library keeps until exit: the first 256 bytes
// hold the "changed" flag, the rest one FP64 Jacobi buffer of up to
// CLIFFS_NOALLOC_MAX_CELLS nodes.
constexpr int FLAG_SLOTS = 32;   // 256 bytes
static __device__ __align__(256) double g_scratch[FLAG_SLOTS + CLIFFS_NOALLOC_MAX_CELLS];

std::mutex g_mu;
constexpr int MAX_DEVICES = 64;
double* g_dev_ptr[MAX_DEVICES] = {nullptr};

// The same per-node code as cliffs_set_bathy's filter kernels (internal.h).
__global__ void k_na_minraise(double* d, long long n, double min_depth) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) cliffs::filter_minraise_node(d, i, min_depth);
}

__global__ void k_na_pass(const double* in, double* out, int nx, int ny, int dir, double a2,
                          int* changed) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < (long long)nx * ny) cliffs::filter_pass_node(in, out, i, nx, ny, dir, a2, changed);
}

// Memory type of a pointer as the runtime sees it (cudaMemoryTypeUnregistered for plain
// host memory it does not know).
cudaError_t mem_type(const void* p, cudaMemoryType* t) {
    cudaPointerAttributes at;
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    *t = at.type;
    return e;
}

int fail(int code, const char* what, cudaError_t e) {
    char m[256];
    snprintf(m, sizeof(m), "%s: %s", what, cudaGetErrorString(e));
    cliffs::set_last_error(m);
    return code;
}

int reject(const char* m) {
    cliffs::set_last_error(m);
    return CLIFFS_ERR_ARG;
}

}  // namespace

extern "C" {

int cliffs_depth_filter_noalloc(const double* depth, double* out, int32_t nx, int32_t ny,
                                double alpha, double min_depth, void* stream, int32_t* passes) {
    cliffs::set_last_error("");
    if (!depth || !out) return reject("null argument");
    if (nx < 1 || ny < 1) return reject("empty grid");
    const long long N = (long long)nx * ny;
    if (N > CLIFFS_NOALLOC_MAX_CELLS) {
        char m[256];
        snprintf(m, sizeof(m),
                 "grid %d x %d has %lld nodes; this entry point's static scratch holds at most %d "
                 "(use cliffs_set_bathy for larger grids)", nx, ny, N, CLIFFS_NOALLOC_MAX_CELLS);
        return reject(m);
    }
    if (!(alpha > 1.0 && alpha < 3.0)) return reject("filter limit alpha must be in (1, 3)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CLIFFS_ERR_CUDA, "cudaGetDevice", e);
    // out is written by kernels: it must be device (or managed) memory, and the input may
    // share it only as a whole (in place)
    cudaMemoryType to, ti;
    e = mem_type(out, &to);
    if (e != cudaSuccess) return fail(CLIFFS_ERR_CUDA, "cudaPointerGetAttributes(out)", e);
    if (to != cudaMemoryTypeDevice && to != cudaMemoryTypeManaged)
        return reject("out must be device memory (cudaMalloc'd or managed)");
    e = mem_type(depth, &ti);
    if (e != cudaSuccess) return fail(CLIFFS_ERR_CUDA, "cudaPointerGetAttributes(depth)", e);
    if (out != depth && (ti == cudaMemoryTypeDevice || ti == cudaMemoryTypeManaged)) {
        const char* a = reinterpret_cast<const char*>(depth);
        const char* b = reinterpret_cast<const char*>(out);
        const size_t bytes = sizeof(double) * (size_t)N;
        if (a < b + bytes && b < a + bytes) return reject("depth and out overlap without being the same array");
    }
    if (dev < 0 || dev >= MAX_DEVICES) return reject("device index beyond the 64 this entry point tracks");
    double* base;
    {
        // set-up once per device, with that device current: the array's device address. The
        // address is kept for the life of the process; it does not survive cudaDeviceReset
        // (the module is loaded again afterwards), so do not call this entry point after one.
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_dev_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) return fail(CLIFFS_ERR_CUDA, "cudaGetSymbolAddress", e);
            g_dev_ptr[dev] = static_cast<double*>(p);
        }
        base = g_dev_ptr[dev];
    }
    int* changed = reinterpret_cast<int*>(base);
    double* tmp = base + FLAG_SLOTS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (out != depth) {
        e = cudaMemcpyAsync(out, depth, sizeof(double) * N, cudaMemcpyDefault, s);
        if (e != cudaSuccess) return fail(CLIFFS_ERR_CUDA, "copy of the input depth", e);
    }
    k_na_minraise<<<blocks, 256, 0, s>>>(out, N, min_depth);
    const double a2 = alpha * alpha;
    int pass = 1;
    for (; pass <= 100; ++pass) {
        e = cudaMemsetAsync(changed, 0, sizeof(int), s);          // the flag starts at zero
        if (e != cudaSuccess) return fail(CLIFFS_ERR_CUDA, "flag reset", e);
        k_na_pass<<<blocks, 256, 0, s>>>(out, tmp, nx, ny, 0, a2, changed);
        k_na_pass<<<blocks, 256, 0, s>>>(tmp, out, nx, ny, 1, a2, changed);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(CLIFFS_ERR_CUDA, "filter pass launch", e);
        int h = 0;
        e = cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(CLIFFS_ERR_CUDA, "flag read", e);
        if (!h) break;
    }
    if (passes) *passes = pass <= 100 ? pass : -1;
    return CLIFFS_OK;
}

}  // extern "C"
