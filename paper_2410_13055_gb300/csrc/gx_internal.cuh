// Internal layout shared by the host driver (gx_host.cu) and the kernels (gx_kernels.cu).
//
// Everything lives in one caller-provided device workspace.  Per-network static
// arrays (topology, costs, bus incidence) are concatenated over networks; per-
// scenario arrays are rows of Tp = roundup(T, 4) floats, device-major, concatenated
// over scenarios.  A thread block of the bus or line kernels never spans two
// scenarios, so per-block residual partials belong to exactly one scenario.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "../../include/gx.h"

namespace gx {

constexpr int kBlock = 256;        // threads per block of the bus / line / generic kernels
constexpr int kLineItems = 2;     // line-hours per thread of the line kernel
constexpr int kQBlock = 128;       // threads per block of the hour-quad line kernel
// threads per block of the hour-quad bus kernels (each thread one bus-hour quad)
#ifndef GX_BUS_QBLOCK
#define GX_BUS_QBLOCK 128
#endif
constexpr int kBusQBlock = GX_BUS_QBLOCK;
// resident blocks per SM the per-thread-load bus kernel is compiled for: 512 threads, so at
// most 128 registers a thread
constexpr int kBus4MinBlocks = 512 / kBusQBlock;
constexpr int kBatWarps = 2;       // batteries (warps) per block of the battery kernel
constexpr int kMaxT = 256;         // hours per scenario handled by one warp (8 per lane)
constexpr int kHplMax = kMaxT / 32;
constexpr int kStampSlots = 4096;  // residual-check chunks of one loop with kernel time stamps (power of 2)
constexpr int kBusPart = 6;        // floats per bus-block residual partial
constexpr int kDevPart = 3;        // floats per line-block / battery-warp partial

// Bus-kernel pool record: the static data of the buses one bus block covers.  A header
// of kPoolHdr words (counts, then the word offset of each array within the record),
// then the arrays; floats are stored as their bit patterns.  Records are a multiple of 4
// words (16 bytes) long so a block can copy its record with 16-byte loads.
enum : int {
    kPH_NBUS = 0, kPH_GCNT, kPH_ECNT, kPH_BCNT,
    kPH_GP, kPH_EP, kPH_BP,             // [nbus + 1] device-list pointers, relative to the record
    kPH_IC, kPH_IW, kPH_DR,             // [nbus] 1/terminals, 1/sum of phase weights, dual-residual weight
    kPH_GROW, kPH_GCOST, kPH_GEMIS, kPH_GFIRM, kPH_GETA,  // [gcnt] generator row in its network, ...
    kPH_ECODE, kPH_EBETA, kPH_EW,       // [ecnt] line end 2*l + side, beta_l, phase weight w_l
    kPH_BROW,                           // [bcnt] battery row in its network
    // Row staging of the hour-quad bus kernel (records of quad blocks only).  Bus nl of the
    // block covers block items [SI[nl], SI[nl] + SQ[nl]); its generators' row segments sit
    // at stage quads SG[nl] + r * SQ[nl] of each generator region, likewise its line ends
    // (SE) and batteries (SB).  Regions, in quads (16 bytes): generator x [0, QG), generator
    // aux (capacity factor / adjoint coefficient) [QG, 2QG), line delta [2QG, 2QG+QE), line-end
    // phase copy [2QG+QE, 2QG+2QE), battery x [2QG+2QE, +QB).
    // CP: NCP copies of (source offset from the scenario's row base, destination quad,
    // quads << 5 | flags << 3 | array); SBYTES the stage's size, 0 = not staged.
    kPH_SQ, kPH_SI, kPH_SG, kPH_SE, kPH_SB,  // [nbus]
    kPH_CP, kPH_NCP, kPH_QG, kPH_QE, kPH_QB, kPH_SBYTES,
    kPH_TXF, kPH_TXA,                   // bytes the bulk copies bring in: forward, adjoint
    kPoolHdr = 32
};
constexpr int kPoolMax = 3072;  // longest record (words) staged in shared memory
// copies per thread of the staged bus kernel's per-block lists (a block with more copies than
// kCplPerThread * kBusQBlock, or a record too long for shared memory, takes the record path)
constexpr int kCplPerThread = 2;
// staged copies: array ids and flags of a copy-list entry
enum : int { kCpGenX = 0, kCpGenAux = 1, kCpDl = 2, kCpVf = 3, kCpVt = 4, kCpBat = 5 };
enum : int { kCpFirm = 1, kCpRamp = 2 };   // (flags << 3): capacity factor 1 / ramp-limited generator
// Largest row stage (bytes) of one bus block; blocks above it run unstaged.  The launch's
// dynamic shared memory is the largest stage (plus its record), so this caps the staged bus
// kernel's shared-memory occupancy.
#ifndef GX_STAGE_MAX_KB
#define GX_STAGE_MAX_KB 40
#endif
constexpr int kStageMax = GX_STAGE_MAX_KB * 1024;
// minimum resident blocks per SM the staged bus kernel is compiled for (its register cap)
#ifndef GX_BUS4T_MINB
#define GX_BUS4T_MINB 4
#endif

// Cluster-resident solver: one thread-block cluster of C CTAs per scenario, CTA r owning
// hours [r*H, (r+1)*H) of every device (H = ceil(T / C)), its state in shared memory.
constexpr int kCrsThreads = 256;
constexpr int kCrsMaxC = 16;
constexpr int kCrsRed = 10;  // residual partial sums per rank (9 used)
constexpr int kCrsBatState = 7;  // per owned battery-hour: zc zd zs yc yd ys xb

// Byte offsets in a CTA's dynamic shared memory, identical on every rank of a cluster
// (remote ranks are addressed at the same offsets).
struct CrsOff {
    size_t red, wred, flag;
    size_t pbar, u, thb, xl, ld, aux;  // [N*H] bus-hours (aux: adjoint load gradient, NaN if fixed)
    size_t xg, cap;                    // [G*H] (cap: forward capacity, adjoint cost gradient or NaN)
    size_t dl, sg, vf, vt;             // [L*H]
    size_t xb;                         // [B*H]
    size_t lcap;                       // [L] flow limit as an angle, eta_l / beta_l
    size_t bst;                        // [nbo][kCrsBatState][T] batteries owned by this rank
    size_t lmask;                      // [L*H] bytes (adjoint)
    size_t total;
};

__host__ __device__ inline size_t crs_take(size_t& p, size_t bytes) {
    const size_t r = p;
    p += (bytes + 15) / 16 * 16;
    return r;
}

__host__ __device__ inline CrsOff crs_offsets(int N, int G, int L, int B, int H, int nbo, int T) {
    CrsOff o{};
    size_t p = 0;
    o.red = crs_take(p, sizeof(double) * kCrsMaxC * kCrsRed);
    o.wred = crs_take(p, sizeof(float) * (kCrsThreads / 32) * kCrsRed);
    o.flag = crs_take(p, 16);
    const size_t nb = (size_t)N * H * 4, ng = (size_t)G * H * 4, nl = (size_t)L * H * 4;
    o.pbar = crs_take(p, nb); o.u = crs_take(p, nb); o.thb = crs_take(p, nb);
    o.xl = crs_take(p, nb); o.ld = crs_take(p, nb); o.aux = crs_take(p, nb);
    o.xg = crs_take(p, ng); o.cap = crs_take(p, ng);
    o.dl = crs_take(p, nl); o.sg = crs_take(p, nl); o.vf = crs_take(p, nl); o.vt = crs_take(p, nl);
    o.xb = crs_take(p, (size_t)B * H * 4);
    o.lcap = crs_take(p, (size_t)L * 4);
    o.bst = crs_take(p, (size_t)nbo * kCrsBatState * T * 4);
    o.lmask = crs_take(p, (size_t)L * H);
    o.total = p;
    return o;
}

// One per bus-kernel block (built at create).
struct BusBlk {
    long long e_bus, e_gen, e_line, e_bat;  // element offsets of the scenario's rows
    int s, item0, n0, pool;   // scenario, first item (n * Tp + t) of the block, first bus, record offset (words)
    int words, Tp, T, nitems; // record length (words), padded / true horizon, N * Tp
};

// One per hour-quad line block and one per battery warp (built at create): every offset
// the kernel needs before its state loads, so those loads follow one dependent read.
// Lines one hour-quad line block can carry the end buses of (a block of kQBlock quads covers at
// most kQBlock / (Tp / 4) + 1 lines: horizons of 64 hours and more).
constexpr int kLineBlkLines = 8;
struct LineBlk {
    long long e_line, e_bus;   // element offsets of the scenario's line and bus rows
    int s, line0, Tp, T;       // scenario, first line of its network (global), padded / true horizon
    int L, eta_l, item0, l0;   // lines of the network, plan index of its first line, first line-quad,
                               // first line of the block (local)
    // from and to bus of lines l0 .. l0 + nends - 1, so the block stages them once and its
    // threads issue their bus-row loads together with their state loads; nends = 0: read
    // each line's ends from the network arrays
    int nends, pad[3];
    int ends[2 * kLineBlkLines];
};
struct BatW {
    long long row0, brow0;     // the battery's row and its bus's row
    int s, bg, T, Tp;          // scenario, battery (global index), true / padded horizon
    int eta_b, pad0, pad1, pad2;  // plan index of the battery's power
};

// Kernel modes.  FWD/ADJ advance the forward or adjoint message passing by one
// iteration; RESET/INIT prepare a cold or user start; MASK records the active set.
enum Mode : int { M_FWD = 0, M_ADJ = 1, M_RESET = 2, M_INIT = 3, M_MASK = 4 };

// Active-set codes (one byte per device-hour).
enum : uint8_t { A_FREE = 0, A_LO = 1, A_UP = 2 };
// line: which limit is active; 1/2 flow lower/upper (depends on eta), 3/4 angle lower/upper
enum : uint8_t { AL_FREE = 0, AL_FLO = 1, AL_FUP = 2, AL_ALO = 3, AL_AUP = 4 };
// battery: bits 0-1 charge, 2-3 discharge, 4-5 soc (each A_FREE/A_LO/A_UP)

struct ScenDev {
    int net, T, Tp, N, G, L, B;
    int gen0, line0, bat0, bus0;      // first index of this network's devices in static arrays
    int ptr0;                          // first index of this network's CSR pointer arrays (N+1 each)
    int eta0;                          // offset of the network's block in eta
    int gs0;                           // offset of this scenario's block in grad_s (FP64, K_net entries)
    long long e_bus, e_gen, e_line, e_bat;  // element offsets of the scenario's rows
    int bus_blk0, bus_nblk, line_blk0, line_nblk, bat_w0;  // single-hour kernels (setup modes)
    int bus4_blk0, bus4_nblk, line4_blk0, line4_nblk;     // hour-quad kernels (iterations)
    int R, ramp0, ramp_w0;             // ramping generators: count, offset in the static ramp
                                       // arrays, first warp of the ramp kernel
    long long e_ramp;                  // element offset of the scenario's ramp state rows
    int cost_blk0;                     // first block of the cost reduction
    float weight;
    double load_norm;                  // sqrt(sum load^2), >= 1e-30
};

// Device pointers + scalars handed to every kernel by value.
// A dual-residual weight sum_{line ends at the bus} (w_l / beta_l)^2 that depends on
// scaling susceptances: d0 holds the fixed lines' part, [first, first + count) of
// sc_dres_l the scaling ones.  target >= 0: pool word; < 0: bus_dres_w[-1 - target].
struct ScaleDres {
    double d0;
    int target, first, count, pad;
};

struct Ctx {
    // sizes
    int S, n_bus_blk, n_line_blk, n_bat_warps, n_cost_blk;
    int n_bus4_blk, n_line4_blk;
    int n_ramp_warps;
    // options
    float rho, eps, voll, kappa, rho_in, rth_c;  // rth_c = rho * rho_theta_c
    float tol_act;
    float rho_ratio;     // adjoint context: forward rho / adjoint rho (scaled-dual conversion)
    int adj_from_fwd;    // adjoint RESET starts from the negated forward duals
    int inner_iters;
    int check_every;
    int max_it;          // iteration cap of the loop this context drives
    int max_bat_T;       // longest horizon among scenarios that have batteries
    int max_ramp_T;      // longest horizon among scenarios that have ramping generators
    int* iter_ctr;       // device iteration counter of the current loop
    // tables
    const ScenDev* scen;
    const int* bus_blk_scen;   // [n_bus_blk]
    const BusBlk* bus_blk;     // [n_bus_blk]
    const BusBlk* bus4_blk;    // [n_bus4_blk] hour-quad bus kernel
    const int* line4_blk_scen; // [n_line4_blk]
    const LineBlk* line4_blk;  // [n_line4_blk]
    const BatW* bat_w;         // [n_bat_warps]
    const int* ramp_warp_scen; // [n_ramp_warps]
    const int* r_gen;          // [ramping generators] generator index within its network
    const float* r_rate;       // [ramping generators] ramp limit / capacity per hour
    const int* g_ramp;         // [generators] index among its network's ramping generators, -1 if none
    int* pool;                 // bus-block pool records (generator plan values refreshed per call)
    const int2* prep;          // [n_prep] (pool word, eta index) of every generator plan value
    int n_prep;
    // Lines whose susceptance scales with capacity, beta_l = (beta0_l / ref_l) eta_l: once per
    // call k_scale_prep writes the effective beta into the line table and the bus pool
    // records, and the dual-residual weights of the buses they touch.
    const int* sc_line;        // [n_scale] global line index
    const int* sc_eta;         // [n_scale] its plan entry
    const double* sc_b;        // [n_scale] beta0_l / ref_l  (= d beta_l / d eta_l)
    const double* sc_bmin;     // [n_scale] floor of beta_l (1e-6 beta0_l, for eta_l -> 0)
    const int2* sc_pool;       // [n_sc_pool] (pool word of a line end's beta, scaling index)
    const ScaleDres* sc_dres;  // [n_sc_dres] dual-residual weights to rewrite
    const int2* sc_dres_l;     // (scaling index, float bits of w_l) of the scaling line ends
    const int* sc_gwarp;       // [2 n_sc_gwarps] (scenario, scaling index) gradient warps
    float* l_beta_w;           // the line table (l_beta) and ...
    float* dres_w_w;           // ... the bus dual-residual weights (bus_dres_w), writable
    int n_scale, n_sc_pool, n_sc_dres, n_sc_gwarps;
    const int* line_blk_scen;  // [n_line_blk]
    const int* bat_warp_scen;  // [n_bat_warps]
    const int* cost_blk_scen;  // [n_cost_blk]
    // per-network static (concatenated)
    const int* g_bus; const float* g_cost; const float* g_emis; const uint8_t* g_firm;
    const int* l_from; const int* l_to; const float* l_beta; const float* l_dth; const float* l_w;
    const int* b_bus; const float* b_dur; const float* b_effc; const float* b_effd;
    const int* bus_gptr; const int* bus_gidx;     // CSR: generators at each bus
    const int* bus_bptr; const int* bus_bidx;     // CSR: batteries at each bus
    const int* bus_eptr; const int* bus_eidx;     // CSR: line ends (2*line + side, side 1 = to)
    const float* bus_inv_cnt;                      // 1 / terminals at the bus
    const float* bus_inv_wsum;                     // 1 / sum of phase weights of its line ends (0 if none)
    const float* bus_dres_w;                       // sum over its line ends of (w_l / beta_l)^2
    // per-scenario inputs
    const float* load;  // [bus rows]
    const float* cf;    // [gen rows]
    const float* eta;   // [K] current plan (caller buffer)
    // forward state
    float* xg; float* xl; float* dl; float* sg; float* vf; float* vt;  // vf/vt hold q = terminal phase + scaled phase dual
    float* xb; float* zc; float* zd; float* zs; float* yc; float* yd; float* ys;
    float* u; float* pbar; float* thb;
    const float* bat_dd;  // Thomas pivots of the battery tridiagonal system [bat rows]
    // adjoint state
    float* a_xg; float* a_xl; float* a_dl; float* a_sg; float* a_vf; float* a_vt;
    float* a_xb; float* a_zc; float* a_zd; float* a_zs; float* a_yc; float* a_yd; float* a_ys;
    float* a_u; float* a_pbar; float* a_thb;
    // ramping generators, [ramp rows]: box copy z, ramp copy w (hour t: p_t - p_{t-1}),
    // their scaled duals y, q; forward and adjoint; Thomas pivots 1/m_t of the x-step
    float *rz, *rw, *ry, *rq, *a_rz, *a_rw, *a_ry, *a_rq;
    const float* ramp_dd;
    // active set
    uint8_t* m_gen; uint8_t* m_load; uint8_t* m_line; uint8_t* m_bat;
    // adjoint generator coefficient [gen rows], written with the active set: the adjoint's
    // linear term c_g + eps p*_gt + kappa e_g of a free generator-hour, NaN where a bound is
    // active (the variable is fixed at 0); one float row the adjoint bus kernels read in place
    // of the forward dispatch and the byte mask; likewise for the load-shed variables [bus rows]:
    // VOLL + eps shed*_nt, NaN where a bound is active
    float* ag;
    float* al;
    // flags, outputs and partials
    int* done;          // [S] 1 = skip (converged or outside the batch)
    int* iters;         // [S]
    int* status;        // [S]
    int* adj_iters;     // [S]
    int* n_active;      // [1]
    double* resid;      // [S*2]
    double* rbest;      // [S] smallest max(primal, dual) residual of the current solve
    double* cost;       // [S]
    double* hval;       // [S]
    double* grad_s;     // [sum_s K_net]
    float* out_flow; float* out_price; float* out_shed;
    float* bus_part;    // [n_bus4_blk * kBusPart]
    float* line_part;   // [n_line4_blk * kDevPart]
    float* bat_part;    // [n_bat_warps * kDevPart]
    float* ramp_part;   // [n_ramp_warps * kDevPart] (dx^2, x^2, adjoint scale)
    double* cost_part;  // [n_cost_blk * 2]
    const float* warm;  // user warm start [prices | angles] over bus rows, or nullptr
    long long warm_half; // element count of the prices half of `warm` (= all bus rows)
    // sampled kernel timing (gx_profile_enable), nullptr while off: per residual-check chunk
    // and kernel kind (0 bus, 1 line, 2 battery / ramp), the earliest block start and the
    // latest block end of the chunk's last iteration (%globaltimer, ns); per scenario, the
    // chunks it was iterating in
    unsigned long long* stamp_lo;  // [kStampSlots * 3]
    unsigned long long* stamp_hi;  // [kStampSlots * 3]
    long long* prof_act;           // [S]
    // hour-quad bus kernel: 1 = stage the block's device rows in shared memory with bulk
    // copies (k_bus4t), 0 = per-thread loads (k_bus4); the staged launch's dynamic shared
    // memory; a bounded device-side wait that gave up writes its status to *err
    int bus_staged;
    int bus4_smem;
    // Bulk-staged bus kernel, per block at a fixed stride (built where the lists are small):
    // header (copies, forward bytes, adjoint bytes, 1 = take the record path) then the block's
    // copy list, so a block reads its list together with its block record; and per-block done
    // flags, refreshed from the scenario flags at every chunk start.  bus_cpl == nullptr: every
    // block reads its list from its record.
    const int* bus_cpl;
    int bus_cpl_stride, bus_cpl_max;  // ints per block; most copies of a block
    int* bus_done;                    // [n_bus4_blk]
    int bat_warps;       // battery prox warps per battery for horizons over 96 hours (1 or 2)
    int* err;
};

// Time stamps of the sampled (residual) iteration; the slot is the loop's current chunk.
__device__ __forceinline__ unsigned long long gx_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int stamp_slot(const Ctx& c) {
    return ((*c.iter_ctr - 1) / c.check_every) & (kStampSlots - 1);
}
__device__ __forceinline__ void stamp_start(const Ctx& c, int kind) {
    atomicMin(c.stamp_lo + 3 * stamp_slot(c) + kind, gx_now());
}
__device__ __forceinline__ void stamp_end(const Ctx& c, int kind) {
    atomicMax(c.stamp_hi + 3 * stamp_slot(c) + kind, gx_now());
}

// One thread's share of scenario sc's operating cost (Eq. 2 objective with the eps terms)
// and emission total, FP64: thread `tid` of a reduction over `stride` threads takes every
// stride-th element of each device array.  c p + eps/2 p^2 over generators, VOLL sh +
// eps/2 sh^2 over loads, eps/2 (ch^2 + dis^2) over batteries, eps/2 f^2 over HVDC lines
// (phase weight 0); emissions e p.  Padding hours (t >= T) are skipped.  Both cost
// reductions (the workspace one and the allocation-free one) use this.
__device__ __forceinline__ void cost_share(const Ctx& c, const ScenDev& sc, long long tid, long long stride,
                                           double& cs, double& em) {
    // One 4-hour quad per step (rows are padded to whole quads): the quad's terms in FP32,
    // their sum added in FP64, so the sums run at the FP32 rate and accumulate in FP64.
    const float eps = (float)c.eps, voll = (float)c.voll;
    const unsigned Tq = (unsigned)sc.Tp >> 2;
    const long long ng = (long long)sc.G * Tq, nn = (long long)sc.N * Tq, nbt = (long long)sc.B * Tq;
    for (long long q = tid; q < ng; q += stride) {
        const unsigned g = (unsigned)q / Tq, t0 = 4u * ((unsigned)q - g * Tq);
        const float4 p = *reinterpret_cast<const float4*>(c.xg + sc.e_gen + 4 * q);
        const float pv[4] = {p.x, p.y, p.z, p.w};
        const float cg = c.g_cost[sc.gen0 + g], eg = c.g_emis[sc.gen0 + g];
        float a = 0.f, e = 0.f;
#pragma unroll
        for (int h = 0; h < 4; ++h)
            if ((int)(t0 + h) < sc.T) {
                a += cg * pv[h] + 0.5f * eps * pv[h] * pv[h];
                e += eg * pv[h];
            }
        cs += (double)a;
        em += (double)e;
    }
    for (long long q = tid; q < nn; q += stride) {
        const unsigned t0 = 4u * ((unsigned)q % Tq);
        const float4 x = *reinterpret_cast<const float4*>(c.xl + sc.e_bus + 4 * q);
        const float4 L = *reinterpret_cast<const float4*>(c.load + sc.e_bus + 4 * q);
        const float sv[4] = {x.x + L.x, x.y + L.y, x.z + L.z, x.w + L.w};
        float a = 0.f;
#pragma unroll
        for (int h = 0; h < 4; ++h)
            if ((int)(t0 + h) < sc.T) a += voll * sv[h] + 0.5f * eps * sv[h] * sv[h];
        cs += (double)a;
    }
    for (long long q = tid; q < nbt; q += stride) {
        const unsigned t0 = 4u * ((unsigned)q % Tq);
        const float4 ch = *reinterpret_cast<const float4*>(c.zc + sc.e_bat + 4 * q);
        const float4 di = *reinterpret_cast<const float4*>(c.zd + sc.e_bat + 4 * q);
        const float cv[4] = {ch.x, ch.y, ch.z, ch.w}, dv[4] = {di.x, di.y, di.z, di.w};
        float a = 0.f;
#pragma unroll
        for (int h = 0; h < 4; ++h)
            if ((int)(t0 + h) < sc.T) a += 0.5f * eps * (cv[h] * cv[h] + dv[h] * dv[h]);
        cs += (double)a;
    }
    const long long nl = (long long)sc.L * Tq;
    for (long long q = tid; q < nl; q += stride) {
        const unsigned l = (unsigned)q / Tq, t0 = 4u * ((unsigned)q - l * Tq);
        if (c.l_w[sc.line0 + l] != 0.f) continue;  // AC lines carry no cost; HVDC links eps/2 f^2
        const float4 f = *reinterpret_cast<const float4*>(c.dl + sc.e_line + 4 * q);
        const float fv[4] = {f.x, f.y, f.z, f.w};
        float a = 0.f;
#pragma unroll
        for (int h = 0; h < 4; ++h)
            if ((int)(t0 + h) < sc.T) a += 0.5f * eps * fv[h] * fv[h];
        cs += (double)a;
    }
}

// Launch wrappers (gx_kernels.cu).  Each returns the number of kernels launched.
int launch_dev(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st);
int launch_line(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st);
int launch_bat(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st);
int launch_ramp(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st);
int launch_bus(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st);
int launch_prep(const Ctx& c, cudaStream_t st);
// Allow the staged bus kernel `smem` bytes of dynamic shared memory (once per process is
// enough; called at bind).
cudaError_t bus_staged_prepare(int smem);
int launch_loop_cond(const Ctx& c, int max_it, cudaGraphConditionalHandle h, cudaStream_t st);
// Cluster-resident solver (gx_crs.cu): iterate the scenarios in `scen` (in_batch ones
// only) to convergence, C CTAs per scenario, hpl hours per lane of a battery warp.
cudaError_t crs_prepare(int adj, int hpl, size_t smem_max);
int crs_max_clusters(int adj, int hpl, int C, size_t smem);
int launch_crs(const Ctx& c, int adj, const int* scen, int n, const int* in_batch, int C, int hpl, size_t smem,
               double tol, cudaStream_t st);
int launch_reduce(const Ctx& c, int adj, double tol, cudaStream_t st);
int launch_tick(const Ctx& c, int chunk, cudaStream_t st);
int launch_extract(const Ctx& c, const int* in_batch, cudaStream_t st);
// The forward state arrays inside the state range: float offset from the range's start and
// row kind (0 generator, 1 bus, 2 line, 3 battery, 4 ramp rows).
struct WarmArrays {
    long long off[20];
    int kind[20];
    int n;
};
// GX_WARM_LEARNED's per-scenario choice after one trial chunk from each start: chosen[s] =
// 1 learned start kept, 0 previous plan's (state rows and flags restored from `saved` and
// the s* arrays), -1 outside the batch.
int launch_warm_select(const Ctx& c, const WarmArrays& w, float* state, const float* saved, const int* in_batch,
                       const int* sdone, const int* sstatus, const int* siters, const double* sres, int* chosen,
                       cudaStream_t st);
// obj = sum_s wprime[s] h_s (Eq. 1's operating term over the batch), FP64, fixed order.
int launch_objective(const Ctx& c, const double* wprime, double* obj, cudaStream_t st);
int launch_grad(const Ctx& c, int envelope, const int* gwarp_scen, int n_gwarps, const int* in_batch,
                cudaStream_t st);
int launch_grad_combine(const Ctx& c, const double* wprime, const int* k_net, float* grad_out, int K,
                        cudaStream_t st);
// capacity-dependent susceptance (gx_scale.cu)
int launch_scale_prep(const Ctx& c, cudaStream_t st);
int launch_scale_grad(const Ctx& c, int envelope, const int* in_batch, cudaStream_t st);
int launch_plan_step(float* eta, const float* grad, const float* gamma, const float* lo, const float* hi, float alpha,
                     int K, cudaStream_t st);

}  // namespace gx

// The warm-start network's side of GX_WARM_LEARNED (gx_gnn.cu): its network, a prediction
// into its own buffer ([prices | angles] over bus rows), and its scratch for the forward
// state and per-scenario flags (nullptr if unbound).
namespace gx {
const gx_network* gx_gnn_internal_net(const gx_gnn* g);
gx_status gx_gnn_internal_predict(gx_gnn* g, const float* eta, cudaStream_t st, const float** pred);
uint8_t* gx_gnn_internal_scratch(gx_gnn* g, size_t* bytes);
}  // namespace gx

// Read-only accessors for the no-allocation entry point (gx_noalloc.cu).
namespace gx {
const Ctx* gx_internal_ctx(const gx_network* net);        // nullptr if not bound
bool gx_internal_solved(const gx_network* net);          // a solve has run since the last bind
ScenDev gx_internal_scen(const gx_network* net, int s);   // s must be in range
gx_status gx_internal_fail(gx_status s, const std::string& msg);
}  // namespace gx
