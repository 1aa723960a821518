// gx_dispatch_cost_noalloc: the per-scenario operating-cost reduction without any
// device allocation, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any routine that allocates): host
// applications that hand the library a fixed device-memory budget and forbid it from
// growing, plugins whose device memory belongs to a host framework's allocator (a
// private cudaMalloc would bypass its accounting), and latency-critical loops in which
// an allocation or a free may synchronise the device and stall other streams.  The
// regular cost reduction keeps its per-block partial sums in the caller-allocated
// workspace; this variant keeps them in a fixed array compiled into the library.
//
// The scratch array below lives on every GPU that loads this library, for as long as
// the process runs (kNoallocMaxBlocks blocks x 2 doubles = 64 KiB).  Host code must not
// use the array's name as a device address: it is only a host-side stand-in.  The
// device address is looked up once per device with cudaGetSymbolAddress, by the
// first call made while that device is current, and cached.
#include "gx_internal.cuh"

#include <algorithm>
#include <mutex>
#include <string>

namespace gx {

constexpr int kNoallocMaxBlocks = 4096;  // partial-sum slots (each: cost, emissions)
constexpr int kNoallocMaxDevices = 64;

// Shared by every call on a device; holds the last call's partial sums.
static __device__ __align__(256) double g_cost_scratch[2 * kNoallocMaxBlocks];

namespace {

__device__ __forceinline__ double warp_sum_nd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The workspace cost reduction's sums (cost_share): block b of `nblk` takes a strided
// share of scenario s.
__global__ void __launch_bounds__(kBlock) k_cost_noalloc(const Ctx c, int s, int nblk, double* part) {
    const ScenDev sc = c.scen[s];
    const int nb = blockIdx.x;
    double cs = 0.0, em = 0.0;
    cost_share(c, sc, (long long)nb * kBlock + threadIdx.x, (long long)nblk * kBlock, cs, em);
    cs = warp_sum_nd(cs);
    em = warp_sum_nd(em);
    __shared__ double sh[2][kBlock / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sh[0][w] = cs; sh[1][w] = em; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int k = 0; k < kBlock / 32; ++k) { a += sh[0][k]; b += sh[1][k]; }
        part[2 * nb] = a;        // every slot 0..nblk-1 is written before it is read:
        part[2 * nb + 1] = b;    // nothing in the scratch has to start at zero
    }
}

__global__ void k_cost_noalloc_final(const double* part, int nblk, double kappa, double* cost_out, double* h_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0, e = 0;
    for (int b = 0; b < nblk; ++b) { a += part[2 * b]; e += part[2 * b + 1]; }
    *cost_out = a;
    if (h_out) *h_out = a + kappa * e;
}

std::mutex g_sym_mu;
double* g_sym_ptr[kNoallocMaxDevices] = {nullptr};

}  // namespace

// Device address of g_cost_scratch on the current device (looked up once per device).
static gx_status scratch_address(double** out, std::string* err) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return GX_ERR_CUDA; }
    if (dev < 0 || dev >= kNoallocMaxDevices) { *err = "device index beyond the supported range"; return GX_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lock(g_sym_mu);
    if (!g_sym_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cost_scratch);
        if (e != cudaSuccess || !p) {
            *err = std::string("cudaGetSymbolAddress(g_cost_scratch): ") + cudaGetErrorString(e);
            return GX_ERR_CUDA;
        }
        g_sym_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_sym_ptr[dev];
    return GX_OK;
}

}  // namespace gx

extern "C" gx_status gx_dispatch_cost_noalloc(const gx_network* net, int scen, double* cost_out_dev,
                                              double* h_out_dev, void* stream) {
    using namespace gx;
    if (!net || !cost_out_dev) return gx_internal_fail(GX_ERR_INVALID_ARG, "NULL argument");
    const Ctx* c = gx_internal_ctx(net);
    if (!c) return gx_internal_fail(GX_ERR_STATE, "network is not bound");
    if (!gx_internal_solved(net))
        return gx_internal_fail(GX_ERR_STATE, "gx_dispatch_cost_noalloc needs a solve first");
    if (scen < 0 || scen >= c->S) return gx_internal_fail(GX_ERR_INVALID_ARG, "scenario out of range");
    const ScenDev sd = gx_internal_scen(net, scen);
    const long long work = (long long)(sd.G + sd.N + sd.B) * sd.Tp;
    const long long want = (work + (long long)kBlock * 16 - 1) / ((long long)kBlock * 16);
    if (want > kNoallocMaxBlocks)
        return gx_internal_fail(GX_ERR_INVALID_ARG,
                                "scenario too large for gx_dispatch_cost_noalloc: needs " + std::to_string(want) +
                                    " partial-sum slots, the fixed scratch holds " +
                                    std::to_string(kNoallocMaxBlocks) +
                                    " ((G + N + B) * Tp <= 16,777,216)");
    const int nblk = (int)std::max<long long>(1, want);
    double* scratch = nullptr;
    std::string err;
    if (gx_status st = scratch_address(&scratch, &err)) return gx_internal_fail(st, err);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_cost_noalloc<<<nblk, kBlock, 0, st>>>(*c, scen, nblk, scratch);
    k_cost_noalloc_final<<<1, 32, 0, st>>>(scratch, nblk, (double)c->kappa, cost_out_dev, h_out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gx_internal_fail(GX_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return GX_OK;
}
