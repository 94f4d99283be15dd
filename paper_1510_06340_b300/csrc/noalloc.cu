// noalloc.cu -- FP64 conservation sums that allocate no device memory.
//
// hydro_conservation_sums needs per-block partial sums in device memory that
// the handle allocates at creation.  Some callers cannot allocate device
// memory at all: code running where another allocator has already reserved
// the whole device, or a latency-critical loop that must never call
// cudaMalloc (it can synchronise the device).  This entry point takes the
// caller's state pointer and writes the four sums to the caller's host
// buffer; its scratch is a fixed array compiled into the library.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/hydro.h"
#include "kernels.h"
#include "widen.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_CHUNK = 65536;      // cells per block
constexpr int NA_MAX_BLOCKS = 4096;        // so at most NA_CHUNK * NA_MAX_BLOCKS cells
constexpr long long NA_MAX_CELLS = NA_CHUNK * NA_MAX_BLOCKS;   // 268,435,456
constexpr int NA_MAX_DEVICES = 64;

// 4 partial sums per block, then the 4 final sums: 131,104 bytes on every
// GPU that loads the library, held until the process exits.
static __device__ __align__(256) double g_na_scratch[4 * NA_MAX_BLOCKS + 4];

std::mutex g_na_mutex;
double *g_na_ptr[NA_MAX_DEVICES] = {nullptr};

// block b: FP64 sums over cells [b * NA_CHUNK, min((b+1) * NA_CHUNK, cells))
template <class R>
__global__ void __launch_bounds__(NA_THREADS)
k_na_partial(const R *__restrict__ U, long long cells, double *__restrict__ scratch) {
    __shared__ double red[4][NA_THREADS / 32];
    const long long lo = (long long)blockIdx.x * NA_CHUNK;
    const long long hi = lo + NA_CHUNK < cells ? lo + NA_CHUNK : cells;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long c = lo + threadIdx.x; c < hi; c += NA_THREADS)
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] += widen(U[q * cells + c]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int q = 0; q < 4; ++q) red[q][wid] = s[q];
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int k = 0; k < NA_THREADS / 32; ++k) t += red[threadIdx.x][k];
        scratch[4 * blockIdx.x + threadIdx.x] = t;
    }
}

// one thread per field, blocks summed in index order (deterministic)
__global__ void k_na_final(double *__restrict__ scratch, int nblocks, double dV) {
    const int q = threadIdx.x;
    if (q >= 4) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += scratch[4 * b + q];
    scratch[4 * NA_MAX_BLOCKS + q] = t * dV;
}

hydro_status na_fail(hydro_status s, const std::string &m) {
    hy::set_last_error(m.c_str());   // read back through hydro_last_error()
    return s;
}

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
hydro_status na_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(HYDRO_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(HYDRO_E_INVALID, "device index too large");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess)
            return na_fail(HYDRO_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_na_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_na_ptr[dev];
    return HYDRO_OK;
}

}  // namespace

extern "C" hydro_status hydro_conservation_sums_noalloc(const void *U, int prec, int nx, int ny,
                                                        int nz, double dx, double dy, double dz,
                                                        double out[4], void *stream) {
    if (!U || !out) return na_fail(HYDRO_E_INVALID, "null pointer");
    if (prec < HYDRO_FP64 || prec > HYDRO_MIXED) return na_fail(HYDRO_E_INVALID, "unknown precision");
    if (nx < 1 || ny < 1 || nz < 1) return na_fail(HYDRO_E_INVALID, "grid sizes must be >= 1");
    const long long cells = (long long)nx * ny * nz;
    if (cells > NA_MAX_CELLS)
        return na_fail(HYDRO_E_INVALID,
                       "grid of " + std::to_string(cells) + " cells exceeds the no-allocation limit of " +
                           std::to_string(NA_MAX_CELLS) + " cells");
    // cell volume by the rule hydro_create applies: an axis of one cell with a
    // spacing <= 0 counts as 1; any other spacing must be positive (NaN fails)
    const int n3[3] = {nx, ny, nz};
    const double h3[3] = {dx, dy, dz};
    double dV = 1.0;
    for (int a = 0; a < 3; ++a) {
        if (n3[a] > 1 && !(h3[a] > 0.0))
            return na_fail(HYDRO_E_INVALID, "cell size must be > 0 on an axis of more than one cell");
        if (n3[a] == 1 && h3[a] != h3[a])
            return na_fail(HYDRO_E_INVALID, "cell size is NaN");
        dV *= h3[a] > 0.0 ? h3[a] : 1.0;
    }
    double *scratch = nullptr;
    hydro_status st = na_scratch(&scratch);
    if (st != HYDRO_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nblocks = (int)((cells + NA_CHUNK - 1) / NA_CHUNK);
    if (prec == HYDRO_FP64)
        k_na_partial<double><<<nblocks, NA_THREADS, 0, s>>>(static_cast<const double *>(U), cells,
                                                             scratch);
    else
        k_na_partial<float><<<nblocks, NA_THREADS, 0, s>>>(static_cast<const float *>(U), cells,
                                                            scratch);
    k_na_final<<<1, 32, 0, s>>>(scratch, nblocks, dV);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, scratch + 4 * NA_MAX_BLOCKS, 4 * sizeof(double),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(HYDRO_E_CUDA, cudaGetErrorString(e));
    return HYDRO_OK;
}
