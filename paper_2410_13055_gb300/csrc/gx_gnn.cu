// Warm-start graph network: node features, BF16 tensor-core layers with FP32
// accumulation, neighbour aggregation, loss, backward and Adam, all on the GPU.
//
// Nodes are the bus-hour rows of a bound gx_network (scenario-major, bus-major, hour
// contiguous: the layout of the nodal price and angle arrays), so a prediction is
// directly a user warm start of gx_dispatch_solve_batch.  With F input features
// (10 used, padded to 16), hidden width 64 and 3 layers:
//
//   h0 = relu(x W_in + b_in)
//   h_k = h_{k-1} + relu([h_{k-1}, mean_{m in N(n)} h_{k-1,m}] W_k + b_k)
//   y = h_3 W_out + b_out,   y0 ~ price / 100, y1 ~ angle
//
// The dense layers (forward, and the input gradient of the backward pass) run on the
// 5th-generation tensor cores: tcgen05.mma with BF16 operands staged in shared memory by the
// TMA engine and FP32 accumulators in tensor memory (k_dense).  Activations that feed a layer
// are written in BF16 by their producer; the FP32 master parameters are copied into BF16
// operand images after every update.  The weight gradients, a reduction over all rows, run
// on the tensor cores as well (k_wgrad: MN-major operands, a persistent CTA per SM).
#include "gx_internal.cuh"
#include "gx_async.cuh"

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

namespace gx {

constexpr int kH = 64;
constexpr int kLayers = 3;
constexpr int kFin = 16;
constexpr int kFused = 10;
// parameter vector layout (FP32 master copy)
constexpr int kOffWin = 0;                        // [kFin][kH]
constexpr int kOffBin = kOffWin + kFin * kH;      // [kH]
constexpr int kLayerSz = 2 * kH * kH + kH;        // W_k [2H][H] + b_k [H]
constexpr int kOffL0 = kOffBin + kH;
constexpr int kOffWout = kOffL0 + kLayers * kLayerSz;  // [kH][2]
constexpr int kOffBout = kOffWout + kH * 2;            // [2]
constexpr int kNParam = kOffBout + 2;

namespace {

__device__ __forceinline__ int scen_of_row(const ScenDev* sc, int S, long long row) {
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sc[mid].e_bus <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- features
__global__ void k_features(const Ctx c, const float* __restrict__ eta, float* __restrict__ X,
                           __nv_bfloat16* __restrict__ Xb, long long M) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int s = scen_of_row(c.scen, c.S, i);
    const ScenDev sc = c.scen[s];
    const long long loc = i - sc.e_bus;
    const int n = (int)(loc / sc.Tp), t = (int)(loc - (long long)n * sc.Tp);
    float f[kFin];
#pragma unroll
    for (int k = 0; k < kFin; ++k) f[k] = 0.f;
    if (t < sc.T) {
        const int nb = sc.ptr0 + n;
        float avail = 0.f, costw = 0.f, freec = 0.f, dear = 0.f;
        for (int q = c.bus_gptr[nb]; q < c.bus_gptr[nb + 1]; ++q) {
            const int g = c.bus_gidx[sc.gen0 + q];
            const float cap = c.cf[sc.e_gen + (long long)g * sc.Tp + t] * fmaxf(eta[sc.eta0 + g], 0.f);
            const float cost = c.g_cost[sc.gen0 + g];
            avail += cap;
            if (cost == 0.f) freec += cap;
            else { dear += cap; costw += cap * cost; }
        }
        float bat = 0.f;
        for (int q = c.bus_bptr[nb]; q < c.bus_bptr[nb + 1]; ++q)
            bat += fmaxf(eta[sc.eta0 + sc.G + sc.L + c.bus_bidx[sc.bat0 + q]], 0.f);
        float lin = 0.f;
        for (int q = c.bus_eptr[nb]; q < c.bus_eptr[nb + 1]; ++q)
            lin += fmaxf(eta[sc.eta0 + sc.G + (c.bus_eidx[2 * sc.line0 + q] >> 1)], 0.f);
        const float L = c.load[i];
        const float h = (float)(t % 24);
        f[0] = L * 0.01f;
        f[1] = avail * 0.01f;
        f[2] = dear > 0.f ? costw / dear * 0.01f : 0.f;
        f[3] = freec * 0.01f;
        f[4] = bat * 0.01f;
        f[5] = lin * 0.01f;
        f[6] = sinf(6.283185307179586f * h / 24.f);
        f[7] = cosf(6.283185307179586f * h / 24.f);
        f[8] = (L - freec) * 0.01f;
        f[9] = 1.f;
    }
    float4* o = reinterpret_cast<float4*>(X + i * kFin);
#pragma unroll
    for (int k = 0; k < kFin / 4; ++k) o[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
    __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(Xb + i * kFin);
#pragma unroll
    for (int k = 0; k < kFin / 2; ++k) ob[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
}

// ---------------------------------------------------------------- dense layers
// One CTA of 128 threads computes a 128-row tile D = A B^T on the tensor cores
// (tcgen05.mma, M = 128, N = 64 or 128, K = 16 per instruction):
//  * A: NKB K-blocks of KW BF16 columns, brought by the TMA engine in the swizzled K-major
//    layout (block 0 from tensor map a0, block 1 from a1, so the concatenation
//    [h, neighbour mean] is never materialised); rows past M arrive as zeros;
//  * B: the layer's weights as a pre-arranged BF16 image in the same layout (k_weight_images),
//    brought by one bulk copy;
//  * D: FP32 in tensor memory, row i in lane i; warp w reads the 32 lanes of its rows, so
//    thread t of the CTA owns row row0 + t in the epilogue.
// Epilogues: kEpiFwd  Z = D + b;  H = relu(Z) (+ resid);  and a BF16 copy of H for the next
//                     layer's operand;
//            kEpiBwd  dH[:, 0:64] += D[:, 0:64];  dAgg = D[:, 64:128]   (D = dZ W^T).
enum : int { kEpiFwd = 0, kEpiBwd = 1 };

struct DenseOut {
    const float* bias;
    const float* resid;
    float* Z;
    float* H;
    __nv_bfloat16* Hb;
    float* dH;
    float* dAgg;
    int* err;
};

template <int NKB, int KW, int N>
struct DenseShape {
    static constexpr uint32_t P = 2 * KW;  // bytes of a K-block row = its swizzle span
    static constexpr uint32_t ATILE = 128 * P;
    static constexpr uint32_t BTILE = N * P;
    static constexpr uint32_t BBYTES = NKB * BTILE;  // the weight image
    static constexpr uint32_t TX = NKB * (ATILE + BTILE);
    static constexpr uint32_t NCOL = N;  // tensor-memory columns: a power of 2 >= 32
    // epilogue stage: per warp 32 rows x 32 columns (row pitch 36 floats), placed over the
    // tiles when they are large enough (every MMA has read them by then), else after them
    static constexpr uint32_t EPITCH = 36;
    static constexpr uint32_t ESTAGE = 4 * 32 * EPITCH * 4;
    static constexpr uint32_t EOFF = TX >= ESTAGE ? 0 : TX;
    static constexpr uint32_t BAROFF = TX > EOFF + ESTAGE ? TX : EOFF + ESTAGE;
    // dynamic shared memory: 1024-byte alignment slack, the tiles (and stage), two barriers
    // and the tensor-memory address; at least enough that the CTAs resident on one SM never
    // ask for more than its 512 tensor-memory columns (4 x 64, 6 x 64 or 3 x 128)
    static constexpr uint32_t USED = 1024 + BAROFF + 64;
    static constexpr uint32_t MIN = N == 128 ? 60u * 1024u : 32u * 1024u;
    static constexpr uint32_t SMEM = USED > MIN ? USED : MIN;
    static_assert(KW == 16 || KW == 64, "K-blocks of 16 (32-byte swizzle) or 64 (128-byte swizzle) columns");
    static_assert(N == 64 || N == 128, "N = 64 or 128");
};

template <int NKB, int KW, int N, int EPI>
__global__ void __launch_bounds__(128) k_dense(const __grid_constant__ CUtensorMap a0,
                                               const __grid_constant__ CUtensorMap a1,
                                               const uint8_t* __restrict__ bimg, const DenseOut o, long long M) {
    using Sh = DenseShape<NKB, KW, N>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    uint8_t* sA = sm;
    uint8_t* sB = sm + NKB * Sh::ATILE;
    float* sE = reinterpret_cast<float*>(sm + Sh::EOFF) + (threadIdx.x >> 5) * 32 * Sh::EPITCH;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + Sh::BAROFF);  // [0] copies, [1] MMAs
    uint32_t* holder = reinterpret_cast<uint32_t*>(bar + 2);
    int* copied = reinterpret_cast<int*>(holder + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long row0 = (long long)blockIdx.x * 128;
    if (warp == 0) tmem_alloc(holder, Sh::NCOL);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;
    if (tid == 0) {
        mbar_expect_tx(&bar[0], Sh::TX);
        bulk_g2s(sB, bimg, Sh::BBYTES, &bar[0]);
        tma_load_2d(sA, &a0, 0, (int)row0, &bar[0]);
        if (NKB > 1) tma_load_2d(sA + Sh::ATILE, &a1, 0, (int)row0, &bar[0]);
        const bool ok = mbar_wait_bounded(&bar[0], 0);
        if (ok) {
            tc_fence_after();
            constexpr uint32_t idesc = umma_idesc_bf16(128, N);
#pragma unroll
            for (int kb = 0; kb < NKB; ++kb)
#pragma unroll
                for (int ks = 0; ks < KW / 16; ++ks)
                    umma_bf16(tmem, umma_sdesc(smem_addr(sA + kb * Sh::ATILE) + 32u * ks, Sh::P),
                              umma_sdesc(smem_addr(sB + kb * Sh::BTILE) + 32u * ks, Sh::P), idesc,
                              (kb | ks) != 0);
            umma_commit(&bar[1]);
        } else {
            atomicExch(o.err, (int)GX_ERR_TIMEOUT);
            mbar_wait_bounded(&bar[0], 0);  // let copies still in flight land before the CTA exits
        }
        *copied = ok ? 1 : 0;
    }
    __syncthreads();
    if (*copied) {
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[1], 0));
        tc_fence_after();
        if (!ok) {
            if (lane == 0) atomicExch(o.err, (int)GX_ERR_TIMEOUT);
        } else {
            // Each warp reads its 32 accumulator rows (a row per lane), transposes them through
            // its shared-memory stage, and writes rows as 128-byte segments: lane l takes
            // columns 4 (l % 8) .. +3 of rows 4 i + l / 8, i = 0..7.
            const uint32_t tq = tmem + ((uint32_t)(warp * 32) << 16);
            const int cq = lane & 7, rq = lane >> 3;
#pragma unroll 1
            for (int c = 0; c < N / 32; ++c) {
                float v[32];
                tmem_ld32(tq + 32u * c, v);  // warp-collective: rows past M take part too
                float4* mine = reinterpret_cast<float4*>(sE + lane * Sh::EPITCH);
#pragma unroll
                for (int q = 0; q < 8; ++q) mine[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                __syncwarp();
                const int col = 32 * c + 4 * cq;
                float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
                if (EPI == kEpiFwd) b = *reinterpret_cast<const float4*>(o.bias + col);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int lr = 4 * i + rq;
                    const long long r = row0 + warp * 32 + lr;
                    if (r >= M) continue;
                    const float4 d = *reinterpret_cast<const float4*>(sE + lr * Sh::EPITCH + 4 * cq);
                    if (EPI == kEpiFwd) {
                        const float4 z = make_float4(d.x + b.x, d.y + b.y, d.z + b.z, d.w + b.w);
                        if (o.Z) *reinterpret_cast<float4*>(o.Z + r * N + col) = z;
                        float4 h = make_float4(fmaxf(z.x, 0.f), fmaxf(z.y, 0.f), fmaxf(z.z, 0.f), fmaxf(z.w, 0.f));
                        if (o.resid) {
                            const float4 a = *reinterpret_cast<const float4*>(o.resid + r * N + col);
                            h.x += a.x; h.y += a.y; h.z += a.z; h.w += a.w;
                        }
                        *reinterpret_cast<float4*>(o.H + r * N + col) = h;
                        if (o.Hb) {
                            __nv_bfloat162 lo = __floats2bfloat162_rn(h.x, h.y), hi = __floats2bfloat162_rn(h.z, h.w);
                            *reinterpret_cast<uint2*>(o.Hb + r * N + col) =
                                make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
                        }
                    } else if (c < 2) {
                        // columns [0, 64): the direct half, added into dH
                        float4* p = reinterpret_cast<float4*>(o.dH + r * kH + col);
                        const float4 a = *p;
                        *p = make_float4(a.x + d.x, a.y + d.y, a.z + d.z, a.w + d.w);
                    } else {
                        // columns [64, 128): the neighbour half
                        *reinterpret_cast<float4*>(o.dAgg + r * kH + col - kH) = d;
                    }
                }
                __syncwarp();
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, Sh::NCOL);
    }
}
// ---------------------------------------------------------------- weight gradients (tcgen05)
// dW[k][n] += sum over rows m of A[m][k] dZ[m][n]: D = A^T dZ with the rows as the MMA's K
// dimension, so both operands are MN-major tiles (a row of 64 BF16 columns = 128 bytes per
// bus-hour), exactly the 128-row boxes the TMA engine brings from the row-major arrays.  A
// persistent CTA per SM streams its row tiles through a kWStages-deep ring (warp 0 loads;
// warp 1 issues the MMAs and releases each stage with a commit once its MMAs have read it)
// into one 128 x 64 FP32 accumulator in tensor memory, then adds it into dW with atomics.
//   KIN = 128: A = [h | neighbour mean] (two 64-column groups, kWTile bytes apart), dW [128][64]
//   KIN = 16:  A = the features through a 64-column box (columns from 16 on arrive as zeros),
//              dW [16][64]; accumulator rows from 16 on are not used
constexpr int kWStages = 4;
constexpr uint32_t kWTile = 128 * 128;    // bytes of one 128-row x 64-column BF16 tile
constexpr uint32_t kWStage = 3 * kWTile;  // A group 0, A group 1, dZ
constexpr uint32_t kWSmem = 1024 + kWStages * kWStage + 256;

template <int KIN>
__global__ void __launch_bounds__(128, 1) k_wgrad(const __grid_constant__ CUtensorMap a0,
                                                  const __grid_constant__ CUtensorMap a1,
                                                  const __grid_constant__ CUtensorMap dz, float* __restrict__ dW,
                                                  long long M, int* __restrict__ err) {
    static_assert(KIN == 128 || KIN == 16, "hidden layer or input layer");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sm + kWStages * kWStage);
    unsigned long long* empty = full + kWStages;
    unsigned long long* done = empty + kWStages;
    uint32_t* holder = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* failed = reinterpret_cast<volatile int*>(holder + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long ntiles = (M + 127) / 128;
    constexpr uint32_t TX = (KIN == 128 ? 3u : 2u) * kWTile;
    if (warp == 0) tmem_alloc(holder, 64);
    if (tid == 0) {
        for (int s = 0; s < kWStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *failed = 0;
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;
    if (warp == 0 && lane == 0) {
        int it = 0;
        for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int s = it % kWStages, u = it / kWStages;
            if (u > 0 && !mbar_wait_bounded(&empty[s], (u - 1) & 1)) {
                *failed = 1;
                break;
            }
            uint8_t* st = sm + s * kWStage;
            mbar_expect_tx(&full[s], TX);
            const int y = (int)(t * 128);
            tma_load_2d(st, &a0, 0, y, &full[s]);
            if (KIN == 128) tma_load_2d(st + kWTile, &a1, 0, y, &full[s]);
            tma_load_2d(st + 2 * kWTile, &dz, 0, y, &full[s]);
        }
        // the CTA may not exit with copies in flight: the last fill of each stage has landed
        for (int k = it > kWStages ? it - kWStages : 0; k < it; ++k)
            mbar_wait_bounded(&full[k % kWStages], (k / kWStages) & 1);
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = umma_idesc_bf16(128, 64, true, true);
        int it = 0;
        for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int s = it % kWStages, u = it / kWStages;
            if (!mbar_wait_bounded(&full[s], u & 1)) {
                *failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t st = smem_addr(sm + s * kWStage);
#pragma unroll
            for (int j = 0; j < 8; ++j)  // 16 rows (the MMA's K) per instruction
                umma_bf16(tmem, umma_sdesc(st + 2048u * j, 128, kWTile, 1024),
                          umma_sdesc(st + 2 * kWTile + 2048u * j, 128, kWTile, 1024), idesc, (it | j) != 0);
            umma_commit(&empty[s]);
        }
        umma_commit(done);
    }
    __syncthreads();
    bool ok = *failed == 0 && mbar_wait_bounded(done, 0);
    ok = __all_sync(0xffffffffu, ok);
    tc_fence_after();
    if (ok) {
        const uint32_t tq = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            float v[32];
            tmem_ld32(tq + 32u * c, v);  // warp-collective
            if (tid < KIN) {
#pragma unroll
                for (int j = 0; j < 32; ++j) atomicAdd(&dW[tid * 64 + 32 * c + j], v[j]);
            }
        }
    } else if (lane == 0) {
        atomicExch(err, (int)GX_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 64);
    }
}

constexpr int kChunk = 256;  // rows per block of the bias-gradient column sums

// column sums of dZ [M][N] into db[N] (FP32 atomics per block)
template <int N>
__global__ void k_colsum(const float* __restrict__ dZ, long long M, float* __restrict__ db) {
    __shared__ float sh[N];
    for (int i = threadIdx.x; i < N; i += blockDim.x) sh[i] = 0.f;
    __syncthreads();
    const long long r0 = (long long)blockIdx.x * kChunk;
    for (long long r = r0 + threadIdx.x / N; r < r0 + kChunk && r < M; r += blockDim.x / N)
        atomicAdd(&sh[threadIdx.x % N], dZ[r * N + threadIdx.x % N]);
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) atomicAdd(&db[i], sh[i]);
}

// ---------------------------------------------------------------- aggregation
// outb[i] = BF16 of the mean over neighbour buses m of in[(m, t)] (the next layer's operand;
// also out[i] in FP32 when out is given), or (transpose) out[i] += sum over neighbours m of
// in[(m, t)] / deg(m).  One warp per node, two features per lane.
template <int TRANSPOSE>
__global__ void k_agg(const Ctx c, const float* __restrict__ in, float* __restrict__ out,
                      __nv_bfloat16* __restrict__ outb, long long M) {
    const long long i = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (i >= M) return;
    const int lane = threadIdx.x & 31;
    const int s = scen_of_row(c.scen, c.S, i);
    const ScenDev sc = c.scen[s];
    const long long loc = i - sc.e_bus;
    const int n = (int)(loc / sc.Tp), t = (int)(loc - (long long)n * sc.Tp);
    const int nb = sc.ptr0 + n;
    const int e0 = c.bus_eptr[nb], e1 = c.bus_eptr[nb + 1];
    float a0 = 0.f, a1 = 0.f;
    for (int qq = e0; qq < e1; ++qq) {
        const int e = c.bus_eidx[2 * sc.line0 + qq];
        const int l = e >> 1;
        const int m = (e & 1) ? c.l_from[sc.line0 + l] : c.l_to[sc.line0 + l];
        const long long j = sc.e_bus + (long long)m * sc.Tp + t;
        float w = 1.f;
        if (TRANSPOSE) {
            const int mb = sc.ptr0 + m;
            w = 1.f / (float)(c.bus_eptr[mb + 1] - c.bus_eptr[mb]);
        }
        const float2 v = reinterpret_cast<const float2*>(in + j * kH)[lane];
        a0 += w * v.x;
        a1 += w * v.y;
    }
    if (!TRANSPOSE) {
        const float w = e1 > e0 ? 1.f / (float)(e1 - e0) : 0.f;
        if (out) reinterpret_cast<float2*>(out + i * kH)[lane] = make_float2(a0 * w, a1 * w);
        reinterpret_cast<__nv_bfloat162*>(outb + i * kH)[lane] = __floats2bfloat162_rn(a0 * w, a1 * w);
    } else {
        float2* o = reinterpret_cast<float2*>(out + i * kH) + lane;
        const float2 prev = *o;
        *o = make_float2(prev.x + a0, prev.y + a1);
    }
}

// ---------------------------------------------------------------- head, loss, backward head
__global__ void k_head(const float* __restrict__ H, const float* __restrict__ P, float* __restrict__ Y, long long M) {
    const long long i = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (i >= M) return;
    const int lane = threadIdx.x & 31;
    const float2 h = reinterpret_cast<const float2*>(H + i * kH)[lane];
    const float* W = P + kOffWout;
    float y0 = h.x * W[(2 * lane) * 2 + 0] + h.y * W[(2 * lane + 1) * 2 + 0];
    float y1 = h.x * W[(2 * lane) * 2 + 1] + h.y * W[(2 * lane + 1) * 2 + 1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        y0 += __shfl_xor_sync(0xffffffffu, y0, o);
        y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    }
    if (lane == 0) {
        Y[2 * i] = y0 + P[kOffBout];
        Y[2 * i + 1] = y1 + P[kOffBout + 1];
    }
}

// loss over valid nodes (hour < T); dY = d loss / d y; target layout [prices | angles]
__global__ void k_loss(const Ctx c, const float* __restrict__ Y, const float* __restrict__ tgt, long long M,
                       double inv_count, float w_theta, float* __restrict__ dY, double* __restrict__ loss) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < M) {
        const int s = scen_of_row(c.scen, c.S, i);
        const ScenDev sc = c.scen[s];
        const long long loc = i - sc.e_bus;
        const int t = (int)(loc % sc.Tp);
        float d0 = 0.f, d1 = 0.f;
        if (t < sc.T) {
            d0 = Y[2 * i] - tgt[i] * 0.01f;
            d1 = Y[2 * i + 1] - tgt[M + i];
            l = (double)d0 * d0 + (double)w_theta * d1 * d1;
        }
        dY[2 * i] = (float)(2.0 * d0 * inv_count);
        dY[2 * i + 1] = (float)(2.0 * w_theta * d1 * inv_count);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l * inv_count);
}

// dW_out += H^T dY, db_out += sum dY, dH = dY W_out^T.  Warps stride over nodes (lane l owns
// hidden units 2l, 2l + 1); the block sums its warps' partial weight gradients in shared
// memory and adds them with one atomic per weight.
constexpr int kHeadBlocks = 1024;
__global__ void __launch_bounds__(256) k_head_back(const float* __restrict__ H, const float* __restrict__ dY,
                                                   const float* __restrict__ P, float* __restrict__ G,
                                                   float* __restrict__ dH, long long M) {
    __shared__ float red[8][2 * kH + 2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float* W = P + kOffWout;
    const float w00 = W[(2 * lane) * 2], w01 = W[(2 * lane) * 2 + 1];
    const float w10 = W[(2 * lane + 1) * 2], w11 = W[(2 * lane + 1) * 2 + 1];
    float g00 = 0.f, g01 = 0.f, g10 = 0.f, g11 = 0.f, b0 = 0.f, b1 = 0.f;
    for (long long i = (long long)blockIdx.x * 8 + warp; i < M; i += (long long)gridDim.x * 8) {
        const float2 h = reinterpret_cast<const float2*>(H + i * kH)[lane];
        const float d0 = dY[2 * i], d1 = dY[2 * i + 1];
        g00 += h.x * d0; g01 += h.x * d1;
        g10 += h.y * d0; g11 += h.y * d1;
        b0 += d0; b1 += d1;
        reinterpret_cast<float2*>(dH + i * kH)[lane] = make_float2(d0 * w00 + d1 * w01, d0 * w10 + d1 * w11);
    }
    red[warp][4 * lane] = g00;
    red[warp][4 * lane + 1] = g01;
    red[warp][4 * lane + 2] = g10;
    red[warp][4 * lane + 3] = g11;
    if (lane == 0) {
        red[warp][2 * kH] = b0;
        red[warp][2 * kH + 1] = b1;
    }
    __syncthreads();
    // red[w][4 l + 2 u + o] is the gradient of W_out[2 l + u][o] = GW[(2 l + u) * 2 + o]
    for (int k = threadIdx.x; k < 2 * kH + 2; k += blockDim.x) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += red[w][k];
        if (k < 2 * kH) atomicAdd(&G[kOffWout + k], t);
        else atomicAdd(&G[kOffBout + k - 2 * kH], t);
    }
}

// dZ = dH * (Z > 0), and its BF16 copy (the operand of dZ W^T)
__global__ void k_relu_back(const float* __restrict__ dH, const float* __restrict__ Z, float* __restrict__ dZ,
                            __nv_bfloat16* __restrict__ dZb, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float d = Z[i] > 0.f ? dH[i] : 0.f;
    dZ[i] = d;
    dZb[i] = __float2bfloat16(d);
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m1,
                       float* __restrict__ m2, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float a = b1 * m1[i] + (1.f - b1) * g;
    const float b = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = b;
    P[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// BF16 operand images of the dense layers' weights, in the swizzled K-major layout k_dense
// reads (row n of B holds the weights of output n; see swz_offset):
//   input layer   B[n][k] = W_in[k][n]   64 rows x 16 (32-byte swizzle)
//   layer l       B[n][k] = W_l[k][n]    64 rows x 128: K-blocks [h | neighbour mean]
//   layer l back  B[k][n] = W_l[k][n]    128 rows x 64 (dCat = dZ W_l^T)
constexpr uint32_t kImgIn = kH * 2 * kFin;       // bytes
constexpr uint32_t kImgLayer = 2 * kH * 2 * kH;  // bytes, forward or backward image of one layer
__global__ void k_weight_images(const float* __restrict__ P, uint8_t* __restrict__ img_in,
                                uint8_t* __restrict__ img_fwd, uint8_t* __restrict__ img_bwd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kFin * kH) {
        const int k = i / kH, n = i % kH;
        *reinterpret_cast<__nv_bfloat16*>(img_in + swz_offset(n, k, 2 * kFin)) = __float2bfloat16(P[kOffWin + i]);
    }
    if (i < kLayers * 2 * kH * kH) {
        const int l = i / (2 * kH * kH), j = i % (2 * kH * kH);
        const int k = j / kH, n = j % kH;
        const __nv_bfloat16 v = __float2bfloat16(P[kOffL0 + l * kLayerSz + j]);
        *reinterpret_cast<__nv_bfloat16*>(img_fwd + (size_t)l * kImgLayer + (k / kH) * (kH * 128) +
                                          swz_offset(n, k % kH, 128)) = v;
        *reinterpret_cast<__nv_bfloat16*>(img_bwd + (size_t)l * kImgLayer + swz_offset(k, n, 128)) = v;
    }
}

// predictions in the warm-start layout: prices ($/MWh) then angles (rad)
__global__ void k_unpack(const float* __restrict__ Y, float* __restrict__ out, long long M) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    out[i] = 100.f * Y[2 * i];
    out[M + i] = Y[2 * i + 1];
}

}  // namespace
}  // namespace gx

using namespace gx;

struct gx_gnn {
    const gx_network* net = nullptr;
    long long M = 0;
    double valid = 0;  // nodes with hour < T
    size_t bytes = 0;
    uint8_t* dev = nullptr;
    // offsets
    size_t o_P, o_G, o_m1, o_m2, o_img_in, o_img_fwd, o_img_bwd, o_X, o_Z0, o_Hs, o_Zs, o_Y, o_dY, o_dH,
        o_dZ, o_dAgg, o_loss, o_err;
    // BF16 operands of the tensor-core layers: features, the inputs h_l and neighbour means
    // of each layer (kept for the weight gradients), dZ; and their TMA descriptors (128-row
    // boxes; the features also as a 64-column box for the weight gradient of W_in)
    size_t o_Xb, o_Hb, o_Agb, o_dZb;
    enum { kMapX = 0, kMapXw, kMapH, kMapAg = kMapH + kLayers, kMapdZ = kMapAg + kLayers, kMaps };
    int sms = 0;  // multiprocessors: CTAs of the persistent weight-gradient kernels
    CUtensorMap maps[kMaps];  // 128-byte aligned by its type
    // the network's learned start (GX_WARM_LEARNED): the prediction in the layout of a user
    // start, and room for the network's forward iteration state and per-scenario flags
    // while the solve compares the learned start with the previous plan's
    size_t o_pred, o_save, save_bytes;
    int step = 0;
};

namespace {
size_t lay_add(size_t& total, size_t bytes) {
    const size_t o = total;
    total += (bytes + 255) / 256 * 256;
    return o;
}
}  // namespace

namespace {
// cuTensorMapEncodeTiled, through the runtime's driver entry point (no link to the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// A [rows][cols] row-major BF16 array as boxes of 128 rows x box_cols columns (columns past
// cols arrive as zeros), swizzled over 2 * box_cols bytes (box_cols = 16 or 64: the layouts
// the tensor-core kernels' descriptors describe).
static gx_status encode_rows(CUtensorMap* m, void* dev, long long rows, int cols, int box_cols) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return gx_internal_fail(GX_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, 128u};
    const cuuint32_t es[2] = {1u, 1u};
    const CUtensorMapSwizzle sw = box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B;
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, dev, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return gx_internal_fail(GX_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return GX_OK;
}

template <int NKB, int KW, int N, int EPI>
static cudaError_t dense_prepare() {
    return cudaFuncSetAttribute(k_dense<NKB, KW, N, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)DenseShape<NKB, KW, N>::SMEM);
}

template <int NKB, int KW, int N, int EPI>
static void dense_launch(const CUtensorMap& a0, const CUtensorMap& a1, const uint8_t* img, const DenseOut& o,
                         long long M, cudaStream_t st) {
    const unsigned grid = (unsigned)((M + 127) / 128);
    k_dense<NKB, KW, N, EPI><<<grid, 128, DenseShape<NKB, KW, N>::SMEM, st>>>(a0, a1, img, o, M);
}
}  // namespace

extern "C" {

size_t gx_gnn_num_params(void) { return (size_t)kNParam; }

gx_status gx_gnn_create(const gx_network* net, int hidden, int layers, gx_gnn** out) {
    if (!net || !out) return gx_internal_fail(GX_ERR_INVALID_ARG, "NULL argument");
    if (hidden != kH || layers != kLayers)
        return gx_internal_fail(GX_ERR_INVALID_ARG, "the warm-start network has hidden width 64 and 3 layers");
    const Ctx* c = gx_internal_ctx(net);
    if (!c) return gx_internal_fail(GX_ERR_STATE, "network is not bound");
    gx_gnn* g = new gx_gnn();
    g->net = net;
    long long M = 0;
    double valid = 0;
    for (int s = 0; s < c->S; ++s) {
        const ScenDev d = gx_internal_scen(net, s);
        M += (long long)d.N * d.Tp;
        valid += (double)d.N * d.T;
    }
    g->M = M;
    g->valid = valid;
    size_t t = 0;
    const size_t P = (size_t)kNParam * 4;
    g->o_P = lay_add(t, P); g->o_G = lay_add(t, P); g->o_m1 = lay_add(t, P); g->o_m2 = lay_add(t, P);
    g->o_img_in = lay_add(t, kImgIn);
    g->o_img_fwd = lay_add(t, (size_t)kLayers * kImgLayer);
    g->o_img_bwd = lay_add(t, (size_t)kLayers * kImgLayer);
    g->o_X = lay_add(t, 4 * (size_t)M * kFin);
    g->o_Z0 = lay_add(t, 4 * (size_t)M * kH);
    g->o_Hs = lay_add(t, 4 * (size_t)M * kH * (kLayers + 1));
    g->o_Zs = lay_add(t, 4 * (size_t)M * kH * kLayers);
    g->o_Y = lay_add(t, 4 * (size_t)M * 2);
    g->o_dY = lay_add(t, 4 * (size_t)M * 2);
    g->o_dH = lay_add(t, 4 * (size_t)M * kH);
    g->o_dZ = lay_add(t, 4 * (size_t)M * kH);
    g->o_Xb = lay_add(t, 2 * (size_t)M * kFin);
    g->o_Hb = lay_add(t, 2 * (size_t)M * kH * kLayers);
    g->o_Agb = lay_add(t, 2 * (size_t)M * kH * kLayers);
    g->o_dZb = lay_add(t, 2 * (size_t)M * kH);
    g->o_err = lay_add(t, 4);
    g->o_dAgg = lay_add(t, 4 * (size_t)M * kH);
    g->o_loss = lay_add(t, 8);
    g->o_pred = lay_add(t, 4 * (size_t)M * 2);
    size_t so = 0, sb = 0;
    gx_network_state_range(net, 0, &so, &sb);
    g->save_bytes = sb + 4 * 8 * (size_t)c->S;  // state, then done / status / iters / resid per scenario
    g->o_save = lay_add(t, g->save_bytes);
    g->bytes = t;
    *out = g;
    return GX_OK;
}

size_t gx_gnn_device_bytes(const gx_gnn* g) { return g ? g->bytes : 0; }

gx_status gx_gnn_destroy(gx_gnn* g) {
    delete g;
    return GX_OK;
}

static gx_status gnn_refresh_bf16(gx_gnn* g, cudaStream_t st) {
    const int n = kLayers * 2 * kH * kH;
    k_weight_images<<<(n + 255) / 256, 256, 0, st>>>(reinterpret_cast<const float*>(g->dev + g->o_P),
                                                      g->dev + g->o_img_in, g->dev + g->o_img_fwd,
                                                      g->dev + g->o_img_bwd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return gx_internal_fail(GX_ERR_CUDA, std::string("k_weight_images: ") + cudaGetErrorString(e));
    return GX_OK;
}

gx_status gx_gnn_set_params(gx_gnn* g, const float* host, size_t n, void* stream) {
    if (!g || !g->dev || !host) return gx_internal_fail(GX_ERR_INVALID_ARG, "NULL argument or unbound network");
    if (n != (size_t)kNParam) return gx_internal_fail(GX_ERR_INVALID_ARG, "parameter count mismatch");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(g->dev + g->o_P, host, 4 * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return gx_internal_fail(GX_ERR_CUDA, cudaGetErrorString(e));
    return gnn_refresh_bf16(g, st);
}

gx_status gx_gnn_get_params(const gx_gnn* g, float* host, size_t n, int which, void* stream) {
    if (!g || !g->dev || !host) return gx_internal_fail(GX_ERR_INVALID_ARG, "NULL argument or unbound network");
    if (n != (size_t)kNParam) return gx_internal_fail(GX_ERR_INVALID_ARG, "parameter count mismatch");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(host, g->dev + (which ? g->o_G : g->o_P), 4 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return gx_internal_fail(GX_ERR_CUDA, cudaGetErrorString(e));
    return GX_OK;
}

gx_status gx_gnn_bind(gx_gnn* g, void* dev, size_t bytes, uint64_t seed, void* stream) {
    if (!g || !dev) return gx_internal_fail(GX_ERR_INVALID_ARG, "NULL argument");
    if (reinterpret_cast<uintptr_t>(dev) % 256) return gx_internal_fail(GX_ERR_INVALID_ARG, "dev must be 256-byte aligned");
    if (bytes < g->bytes) return gx_internal_fail(GX_ERR_NO_MEMORY, "GNN workspace too small");
    if (g->M > (1LL << 31) - 128) return gx_internal_fail(GX_ERR_INVALID_ARG, "too many bus-hours for the GNN");
    g->dev = reinterpret_cast<uint8_t*>(dev);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(g->dev, 0, g->bytes, st);
    if (e != cudaSuccess) return gx_internal_fail(GX_ERR_CUDA, cudaGetErrorString(e));
    // tensor-core layers: TMA descriptors of the BF16 operands, shared-memory limits
    const long long M = g->M;
    gx_status sm = encode_rows(&g->maps[gx_gnn::kMapX], g->dev + g->o_Xb, M, kFin, kFin);
    if (!sm) sm = encode_rows(&g->maps[gx_gnn::kMapXw], g->dev + g->o_Xb, M, kFin, kH);
    for (int l = 0; l < kLayers && !sm; ++l) {
        sm = encode_rows(&g->maps[gx_gnn::kMapH + l], g->dev + g->o_Hb + 2 * (size_t)l * M * kH, M, kH, kH);
        if (!sm) sm = encode_rows(&g->maps[gx_gnn::kMapAg + l], g->dev + g->o_Agb + 2 * (size_t)l * M * kH, M, kH, kH);
    }
    if (!sm) sm = encode_rows(&g->maps[gx_gnn::kMapdZ], g->dev + g->o_dZb, M, kH, kH);
    if (sm) {
        g->dev = nullptr;
        return sm;
    }
    int dev_id = 0;
    e = cudaGetDevice(&dev_id);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev_id);
    if (e == cudaSuccess) e = dense_prepare<1, kFin, kH, kEpiFwd>();
    if (e == cudaSuccess) e = dense_prepare<2, kH, kH, kEpiFwd>();
    if (e == cudaSuccess) e = dense_prepare<1, kH, 2 * kH, kEpiBwd>();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_wgrad<2 * kH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_wgrad<kFin>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWSmem);
    if (e != cudaSuccess) {
        g->dev = nullptr;
        return gx_internal_fail(GX_ERR_CUDA, std::string("k_dense attributes: ") + cudaGetErrorString(e));
    }
    // He-style initialisation from a seeded host generator (biases 0)
    std::vector<float> P(kNParam, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int k = 0; k < kFused; ++k)
        for (int n = 0; n < kH; ++n) P[kOffWin + k * kH + n] = nd(rng) * std::sqrt(2.f / kFused);
    for (int l = 0; l < kLayers; ++l)
        for (int j = 0; j < 2 * kH * kH; ++j) P[kOffL0 + l * kLayerSz + j] = nd(rng) * std::sqrt(1.f / (2 * kH));
    for (int j = 0; j < kH * 2; ++j) P[kOffWout + j] = nd(rng) * std::sqrt(1.f / kH);
    g->step = 0;
    return gx_gnn_set_params(g, P.data(), P.size(), stream);
}

// The network's forward pass; a tensor-core wait that runs out records GX_ERR_TIMEOUT in *err.
static void gnn_forward(gx_gnn* g, const float* eta, cudaStream_t st, int* err) {
    const Ctx& c = *gx_internal_ctx(g->net);
    const long long M = g->M;
    auto F = [&](size_t o) { return reinterpret_cast<float*>(g->dev + o); };
    auto Bf = [&](size_t o) { return reinterpret_cast<__nv_bfloat16*>(g->dev + o); };
    float* P = F(g->o_P);
    auto Hb = [&](int l) { return Bf(g->o_Hb) + (size_t)l * M * kH; };
    auto Agb = [&](int l) { return Bf(g->o_Agb) + (size_t)l * M * kH; };
    k_features<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(c, eta, F(g->o_X), Bf(g->o_Xb), M);
    float* H0 = F(g->o_Hs);
    DenseOut o{P + kOffBin, nullptr, F(g->o_Z0), H0, Hb(0), nullptr, nullptr, err};
    dense_launch<1, kFin, kH, kEpiFwd>(g->maps[gx_gnn::kMapX], g->maps[gx_gnn::kMapX], g->dev + g->o_img_in, o, M,
                                        st);
    for (int l = 0; l < kLayers; ++l) {
        float* Hl = F(g->o_Hs) + (size_t)l * M * kH;
        float* Hn = F(g->o_Hs) + (size_t)(l + 1) * M * kH;
        k_agg<0><<<(unsigned)((M + 7) / 8), 256, 0, st>>>(c, Hl, nullptr, Agb(l), M);
        // H_{l+1} = H_l + relu([H_l, mean] W_l + b_l); its BF16 copy feeds the next layer
        DenseOut ol{P + kOffL0 + l * kLayerSz + 2 * kH * kH, Hl, F(g->o_Zs) + (size_t)l * M * kH, Hn,
                    l + 1 < kLayers ? Hb(l + 1) : nullptr, nullptr, nullptr, err};
        dense_launch<2, kH, kH, kEpiFwd>(g->maps[gx_gnn::kMapH + l], g->maps[gx_gnn::kMapAg + l],
                                          g->dev + g->o_img_fwd + (size_t)l * kImgLayer, ol, M, st);
    }
    k_head<<<(unsigned)((M + 7) / 8), 256, 0, st>>>(F(g->o_Hs) + (size_t)kLayers * M * kH, P, F(g->o_Y), M);
}

gx_status gx_gnn_predict(gx_gnn* g, const float* eta_dev, float* out_dev, void* stream) {
    if (!g || !g->dev || !eta_dev || !out_dev) return gx_internal_fail(GX_ERR_INVALID_ARG, "NULL argument or unbound");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    gnn_forward(g, eta_dev, st, reinterpret_cast<int*>(g->dev + g->o_err));
    k_unpack<<<(unsigned)((g->M + 255) / 256), 256, 0, st>>>(reinterpret_cast<float*>(g->dev + g->o_Y), out_dev, g->M);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gx_internal_fail(GX_ERR_CUDA, std::string("gnn predict: ") + cudaGetErrorString(e));
    return GX_OK;
}

}  // extern "C"

namespace gx {
const gx_network* gx_gnn_internal_net(const gx_gnn* g) { return g ? g->net : nullptr; }
gx_status gx_gnn_internal_predict(gx_gnn* g, const float* eta, cudaStream_t st, const float** pred) {
    if (!g || !g->dev) return gx_internal_fail(GX_ERR_STATE, "the attached warm-start network is not bound");
    gnn_forward(g, eta, st, gx_internal_ctx(g->net)->err);  // reported with the solve's status
    float* out = reinterpret_cast<float*>(g->dev + g->o_pred);
    k_unpack<<<(unsigned)((g->M + 255) / 256), 256, 0, st>>>(reinterpret_cast<float*>(g->dev + g->o_Y), out, g->M);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gx_internal_fail(GX_ERR_CUDA, std::string("gnn predict: ") + cudaGetErrorString(e));
    *pred = out;
    return GX_OK;
}
uint8_t* gx_gnn_internal_scratch(gx_gnn* g, size_t* bytes) {
    if (!g || !g->dev) return nullptr;
    *bytes = g->save_bytes;
    return g->dev + g->o_save;
}
}  // namespace gx

extern "C" {

gx_status gx_gnn_train_step(gx_gnn* g, const float* eta_dev, const float* target_dev, float lr, float w_theta,
                            double* loss_host, void* stream) {
    if (!g || !g->dev || !eta_dev || !target_dev) return gx_internal_fail(GX_ERR_INVALID_ARG, "NULL argument or unbound");
    if (!(lr >= 0.f) || !(w_theta >= 0.f)) return gx_internal_fail(GX_ERR_INVALID_ARG, "lr and w_theta must be >= 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const Ctx& c = *gx_internal_ctx(g->net);
    const long long M = g->M;
    auto F = [&](size_t o) { return reinterpret_cast<float*>(g->dev + o); };
    int* err = reinterpret_cast<int*>(g->dev + g->o_err);
    __nv_bfloat16* dZb = reinterpret_cast<__nv_bfloat16*>(g->dev + g->o_dZb);
    gnn_forward(g, eta_dev, st, err);
    float* P = F(g->o_P);
    float* G = F(g->o_G);
    cudaMemsetAsync(G, 0, 4 * (size_t)kNParam, st);
    cudaMemsetAsync(g->dev + g->o_loss, 0, 8, st);
    k_loss<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(c, F(g->o_Y), target_dev, M, 1.0 / g->valid, w_theta,
                                                        F(g->o_dY), reinterpret_cast<double*>(g->dev + g->o_loss));
    float* dH = F(g->o_dH);
    k_head_back<<<(unsigned)std::min<long long>((M + 7) / 8, kHeadBlocks), 256, 0, st>>>(
        F(g->o_Hs) + (size_t)kLayers * M * kH, F(g->o_dY), P, G, dH, M);
    const unsigned ew = (unsigned)((M * kH + 255) / 256);
    const unsigned nchunk = (unsigned)((M + kChunk - 1) / kChunk);
    // persistent weight-gradient CTAs: one per SM, none without a row tile
    const long long ntiles = (M + 127) / 128;
    const unsigned wg = (unsigned)std::min<long long>(ntiles, std::max(g->sms, 1));
    const CUtensorMap& mapdZ = g->maps[gx_gnn::kMapdZ];
    for (int l = kLayers - 1; l >= 0; --l) {
        float* Zl = F(g->o_Zs) + (size_t)l * M * kH;
        float* dZ = F(g->o_dZ);
        k_relu_back<<<ew, 256, 0, st>>>(dH, Zl, dZ, dZb, M * kH);
        float* GW = G + kOffL0 + l * kLayerSz;
        k_wgrad<2 * kH><<<wg, 128, kWSmem, st>>>(g->maps[gx_gnn::kMapH + l], g->maps[gx_gnn::kMapAg + l], mapdZ, GW,
                                                   M, err);
        k_colsum<kH><<<nchunk, 256, 0, st>>>(dZ, M, GW + 2 * kH * kH);
        // [dH_direct, dAgg] = dZ W_l^T on the tensor cores; the residual keeps dH, the direct
        // half is added into it, the neighbour half goes through the transposed aggregation
        DenseOut ob{nullptr, nullptr, nullptr, nullptr, nullptr, dH, F(g->o_dAgg), err};
        dense_launch<1, kH, 2 * kH, kEpiBwd>(mapdZ, mapdZ, g->dev + g->o_img_bwd + (size_t)l * kImgLayer, ob, M, st);
        k_agg<1><<<(unsigned)((M + 7) / 8), 256, 0, st>>>(c, F(g->o_dAgg), dH, nullptr, M);
    }
    float* dZ0 = F(g->o_dZ);
    k_relu_back<<<ew, 256, 0, st>>>(dH, F(g->o_Z0), dZ0, dZb, M * kH);
    k_wgrad<kFin><<<wg, 128, kWSmem, st>>>(g->maps[gx_gnn::kMapXw], g->maps[gx_gnn::kMapXw], mapdZ, G + kOffWin, M,
                                             err);
    k_colsum<kH><<<nchunk, 256, 0, st>>>(dZ0, M, G + kOffBin);
    if (lr > 0.f) {
        g->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)g->step), c2 = 1.f - std::pow(b2, (float)g->step);
        k_adam<<<(kNParam + 255) / 256, 256, 0, st>>>(P, G, F(g->o_m1), F(g->o_m2), kNParam, lr, b1, b2, 1e-8f, c1, c2);
        if (gx_status s = gnn_refresh_bf16(g, st)) return s;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gx_internal_fail(GX_ERR_CUDA, std::string("gnn train: ") + cudaGetErrorString(e));
    if (loss_host) {
        // the loss, and the error word of this and earlier predictions / steps (then cleared)
        int werr = 0;
        e = cudaMemcpyAsync(loss_host, g->dev + g->o_loss, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&werr, err, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && werr) e = cudaMemsetAsync(err, 0, 4, st);
        if (e != cudaSuccess) return gx_internal_fail(GX_ERR_CUDA, cudaGetErrorString(e));
        if (werr) return gx_internal_fail((gx_status)werr, "a tensor-core layer's copy or MMA wait ran out");
    }
    return GX_OK;
}

}  // extern "C"
