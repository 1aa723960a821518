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
constexpr int kBatWarps = 2;       // batteries (warps) per block of the battery kernel
constexpr int kMaxT = 256;         // hours per scenario handled by one warp (8 per lane)
constexpr int kHplMax = kMaxT / 32;
constexpr int kBusPart = 6;        // floats per bus-block residual partial
constexpr int kDevPart = 3;        // floats per line-block / battery-warp partial

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
    int bus_blk0, bus_nblk, line_blk0, line_nblk, bat_w0;
    int cost_blk0;                     // first block of the cost reduction
    float weight;
    double load_norm;                  // sqrt(sum load^2), >= 1e-30
};

// Device pointers + scalars handed to every kernel by value.
struct Ctx {
    // sizes
    int S, n_bus_blk, n_line_blk, n_bat_warps, n_cost_blk;
    // options
    float rho, eps, voll, kappa, rho_in, rth_c;  // rth_c = rho * rho_theta_c
    float tol_act;
    float rho_ratio;     // adjoint context: forward rho / adjoint rho (scaled-dual conversion)
    int adj_from_fwd;    // adjoint RESET starts from the negated forward duals
    int inner_iters;
    int check_every;
    int max_it;          // iteration cap of the loop this context drives
    int max_bat_T;       // longest horizon among scenarios that have batteries
    int* iter_ctr;       // device iteration counter of the current loop
    // tables
    const ScenDev* scen;
    const int* bus_blk_scen;   // [n_bus_blk]
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
    // active set
    uint8_t* m_gen; uint8_t* m_load; uint8_t* m_line; uint8_t* m_bat;
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
    float* bus_part;    // [n_bus_blk * kBusPart]
    float* line_part;   // [n_line_blk * kDevPart]
    float* bat_part;    // [n_bat_warps * kDevPart]
    double* cost_part;  // [n_cost_blk * 2]
    const float* warm;  // user warm start [prices | angles] over bus rows, or nullptr
    long long warm_half; // element count of the prices half of `warm` (= all bus rows)
};

// Launch wrappers (gx_kernels.cu).  Each returns the number of kernels launched.
int launch_dev(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st);
int launch_line(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st);
int launch_bat(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st);
int launch_bus(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st);
int launch_reduce(const Ctx& c, int adj, double tol, cudaStream_t st);
int launch_tick(const Ctx& c, int chunk, cudaStream_t st);
int launch_extract(const Ctx& c, const int* in_batch, cudaStream_t st);
int launch_grad(const Ctx& c, int envelope, const int* gwarp_scen, int n_gwarps, const int* in_batch,
                cudaStream_t st);
int launch_grad_combine(const Ctx& c, const double* wprime, const int* k_net, float* grad_out, int K,
                        cudaStream_t st);
int launch_plan_step(float* eta, const float* grad, const float* gamma, const float* lo, const float* hi, float alpha,
                     int K, cudaStream_t st);

}  // namespace gx

// Read-only accessors for the no-allocation entry point (gx_noalloc.cu).
namespace gx {
const Ctx* gx_internal_ctx(const gx_network* net);        // nullptr if not bound
ScenDev gx_internal_scen(const gx_network* net, int s);   // s must be in range
gx_status gx_internal_fail(gx_status s, const std::string& msg);
}  // namespace gx
