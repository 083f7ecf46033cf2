// Conservation sums without any allocation (lb_conservation_static).
//
// The library's own reductions keep their per-block partial sums in device
// memory the context allocates. This variant keeps them in a fixed
// file-scope device array instead, so a caller that must not allocate
// device memory can still get the FP64 mass and momentum totals of a
// population field. The array lives on every GPU that loads the library
// until the process exits; all calls share it.
#include "../../include/lbsc.h"
#include "lb_fields.cuh"

#include <mutex>
#include <string>

namespace lbsc {

constexpr int kStaticMaxBlocks = 1024;                // rows of partial sums in the static array
constexpr long long kStaticMaxNodesPerBlock = 65536;  // nodes one block reduces at most
constexpr long long kStaticMinNodesPerBlock = 2048;   // and at least (small fields use few blocks)
constexpr long long kStaticMaxNodes = kStaticMaxBlocks * kStaticMaxNodesPerBlock;  // 67,108,864
constexpr int kStaticVals = 8;
constexpr int kStaticThreads = 256;
constexpr int kMaxDevices = 64;

// 1024 x 8 doubles = 64 KiB of partial sums
static __device__ __align__(256) double g_static_partials[kStaticMaxBlocks * kStaticVals];

// Block b sums nodes [b*per, (b+1)*per) of the dense array n[a][k][node] and
// writes one row of partials: {M_r, M_b, Px, Py, Pz, non-finite count, fluid
// nodes, 0}. per = max(ceil(N / 1024), 2048), so a mid-size field spreads
// over up to 1024 blocks and the rows never exceed the static array.
__global__ void __launch_bounds__(kStaticThreads)
    static_cons_kernel(const double* __restrict__ n, const uint8_t* __restrict__ solid, long long N, long long per,
                       double* part)
{
    double acc[kStaticVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long lo = blockIdx.x * per;
    const long long hi = lo + per < N ? lo + per : N;
    for (long long i = lo + threadIdx.x; i < hi; i += kStaticThreads) {
        if (solid && solid[i]) continue;
        acc[6] += 1.0;
        for (int a = 0; a < 2; ++a)
            for (int k = 0; k < Q; ++k) {
                const double v = n[((long long)a * Q + k) * N + i];
                if (!isfinite(v)) acc[5] += 1.0;
                acc[a] += v;
                acc[2] += cx(k) * v;
                acc[3] += cy(k) * v;
                acc[4] += cz(k) * v;
            }
    }
    __shared__ double sh[kStaticThreads / 32][kStaticVals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = 0; v < kStaticVals; ++v) {
        double x = acc[v];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[warp][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < kStaticVals) {
        double x = 0;
        for (int w = 0; w < kStaticThreads / 32; ++w) x += sh[w][threadIdx.x];
        part[blockIdx.x * kStaticVals + threadIdx.x] = x;
    }
}

// out[v] = sum of the first nblocks rows, in row order
__global__ void static_finish_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ out)
{
    const int v = threadIdx.x;
    if (v >= kStaticVals) return;
    double x = 0;
    for (int b = 0; b < nblocks; ++b) x += part[b * kStaticVals + v];
    out[v] = v == 7 ? 0.0 : x;
}

// Device address of the static array on the current device. Host code only
// sees a host-side stand-in under the array's name, so the address is looked
// up once per device (the first call on that device) and cached.
static int static_partials(double** out, std::string& err)
{
    static std::mutex mu;
    static double* addr[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        err = std::string("lb_conservation_static: cudaGetDevice: ") + cudaGetErrorString(e);
        return LB_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        err = "lb_conservation_static: device index beyond the supported 64";
        return LB_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess || !p) {
            err = std::string("lb_conservation_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return LB_ERR_CUDA;
        }
        addr[dev] = (double*)p;
    }
    *out = addr[dev];
    return LB_OK;
}

}  // namespace lbsc

// error message for the context-free entry point, read through lb_last_error(NULL)
void lbsc_set_global_error(const std::string& msg);

extern "C" int lb_conservation_static(const double* populations, const uint8_t* solid, int nx, int ny, int nz,
                                      double* cons, void* cuda_stream)
{
    using namespace lbsc;
    if (!populations || !cons) {
        lbsc_set_global_error("lb_conservation_static: populations and cons must be device pointers");
        return LB_ERR_ARG;
    }
    if (nx < 1 || ny < 1 || nz < 1) {
        lbsc_set_global_error("lb_conservation_static: bad lattice dimensions");
        return LB_ERR_ARG;
    }
    const long long N = (long long)nx * ny * nz;
    if (N > kStaticMaxNodes) {
        lbsc_set_global_error("lb_conservation_static: " + std::to_string(N) +
                              " nodes exceed the static scratch maximum of 67108864 nodes");
        return LB_ERR_ARG;
    }
    std::string err;
    double* part = nullptr;
    const int rc = static_partials(&part, err);
    if (rc != LB_OK) {
        lbsc_set_global_error(err);
        return rc;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    long long per = (N + kStaticMaxBlocks - 1) / kStaticMaxBlocks;
    if (per < kStaticMinNodesPerBlock) per = kStaticMinNodesPerBlock;
    const int blocks = (int)((N + per - 1) / per);  // <= kStaticMaxBlocks since per >= ceil(N / 1024)
    static_cons_kernel<<<blocks, kStaticThreads, 0, st>>>(populations, solid, N, per, part);
    static_finish_kernel<<<1, 32, 0, st>>>(part, blocks, cons);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        lbsc_set_global_error(std::string("lb_conservation_static: launch: ") + cudaGetErrorString(e));
        return LB_ERR_CUDA;
    }
    return LB_OK;
}
