/*
 * gx.h -- C ABI of the GB300 (sm_103a) batched dispatch / implicit-gradient library.
 *
 * What it computes (Degleris, El Gamal, Rajagopal, "Scalable and Interactive
 * Electricity Grid Expansion Planning", arXiv:2410.13055):
 *
 *   Eq. 2      dispatch map   x*_s(eta) = argmin c_s(x) s.t. A_s(eta) x <= b_s(eta)
 *              for every scenario s of a batch: a DC power-flow network with
 *              generators (0 <= p <= cf*eta_g), curtailable loads (0 <= shed <= L),
 *              lines (|beta (th_f - th_t)| <= eta_l, |th_f - th_t| <= dtheta_max)
 *              and batteries (0 <= ch, dis <= eta_b, 0 <= soc <= dur*eta_b,
 *              soc_t = soc_{t-1} + eff_c ch_t - dis_t / eff_d, soc_{-1} = 0) over T hours;
 *              c_s = sum c p + eps/2 p^2 + VOLL shed + eps/2 shed^2 + eps/2 (ch^2 + dis^2).
 *   Sec. 2.2   implicit gradient  d h_s / d eta = (d x*_s / d eta)^T grad h_s, with
 *              h_s = c_s + kappa * emissions (emissions-aware planning, Sec. 2.1),
 *              by the implicit function theorem on the active KKT system.
 *   Sec. 2.2   projected step     eta <- proj_[eta_min, eta_max](eta - alpha (gamma + grad)).
 *
 * The dispatch is solved by proximal message passing (ADMM with per-device
 * proximal operators and per-bus consensus); the gradient by the same message
 * passing applied to the linearised (active-set) KKT system.
 *
 * Conventions
 *  - Units: MW, MWh, $/MWh, rad.  Line beta is MW per rad.
 *  - Plan vector eta (length K, FP32, device memory): for each network in the
 *    order given at create, [generators | lines | batteries] of that network.
 *  - Injection sign: power into the bus is positive.  Nodal price lambda is the
 *    multiplier of the bus balance; an interior generator has lambda = c + eps p.
 *  - Per-scenario arrays are rows of Tp = roundup(T, 4) floats (row-major,
 *    device-major); hours T..Tp-1 are padding.
 *
 * Memory and ownership
 *  - gx_network_create copies every descriptor array (host memory) and lays out
 *    one device workspace.  The library never allocates device memory: the caller
 *    allocates gx_network_device_bytes() bytes (e.g. a torch uint8 tensor) and
 *    passes it to gx_network_bind, and must keep it alive and unmodified until
 *    gx_network_destroy.  Output arrays live inside that workspace; their offsets
 *    come from gx_network_array.
 *  - Pointers named *_dev are device pointers owned by the caller.
 *
 * Errors
 *  - Every call returns gx_status: 0 OK, > 0 warning, < 0 error.  No C++
 *    exception crosses the ABI.  gx_status_string gives a static message and
 *    gx_last_error_message() details of the last error on this thread.
 *  - Calls enqueue work on the given stream.  gx_dispatch_solve_batch and
 *    gx_dispatch_grad_batch run their iteration loop on the device and synchronise
 *    that stream at the end of the loop to read the iteration counts and statuses:
 *    once per loop in the default launch mode (gx_network_use_graphs(2)), once per
 *    residual-check chunk of opts.check_every iterations in modes 1 and 0.
 */
#ifndef GX_H
#define GX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int gx_status;
enum {
    GX_OK = 0,
    GX_NOT_CONVERGED = 1,     /* iteration cap reached; outputs hold the last iterate */
    GX_ERR_INVALID_ARG = -1,  /* a descriptor or argument failed validation */
    GX_ERR_NONFINITE = -2,    /* a NaN/Inf appeared in the iterate or the inputs */
    GX_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    GX_ERR_NO_MEMORY = -4,    /* the bound workspace is too small */
    GX_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up */
    GX_ERR_STATE = -6         /* call out of order (e.g. grad before solve, not bound) */
};

typedef struct gx_network gx_network; /* opaque */

/* One network (topology and devices).  All arrays are host memory of the stated
 * length; indices are 0-based.  A bus may carry any number of devices; every bus
 * has one curtailable load (its profile may be zero). */
typedef struct {
    int n_bus, n_gen, n_line, n_bat;
    const int32_t* gen_bus;      /* [n_gen] */
    const double* gen_cost;      /* [n_gen] $/MWh, finite */
    const double* gen_emis;      /* [n_gen] t/MWh (planner's emission rate) */
    const int32_t* line_from;    /* [n_line] */
    const int32_t* line_to;      /* [n_line], != line_from */
    const double* line_beta;     /* [n_line] MW/rad, > 0 (AC lines) */
    const double* line_dtheta;   /* [n_line] rad, > 0 (AC lines) */
    const int32_t* bat_bus;      /* [n_bat] */
    const double* bat_dur;       /* [n_bat] h, > 0 */
    const double* bat_eff_c;     /* [n_bat] in (0, 1] */
    const double* bat_eff_d;     /* [n_bat] in (0, 1] */
    /* [n_line] or NULL (all AC): 1 marks an HVDC transport line (Sections 2.1 and 3 list
     * HVDC among the planned assets).  Its flow f (MW, from -> to) is limited only by
     * |f| <= eta_l, has no angle coupling, and carries eps/2 f^2 in the operating cost
     * like the other free injections; line_beta and line_dtheta are ignored for it. */
    const uint8_t* line_dc;
    /* [n_gen] or NULL (no ramp limits): hourly ramp limit as a fraction of the planned
     * capacity, |p_t - p_{t-1}| <= gen_ramp[g] * eta_g for t >= 1 (Section 2.1's
     * operating constraints; the paper's "generator ramping limits").  Only values in
     * (0, 1) constrain; 0 or >= 1 means unlimited.  A scenario with ramping generators
     * runs on the per-iteration kernels, not the cluster-resident path. */
    const double* gen_ramp;
    /* [n_line] or NULL (fixed susceptances): a value > 0 makes an AC line's susceptance
     * scale with its planned capacity, beta_l(eta) = line_beta[l] * eta_l / line_beta_ref[l]
     * (capacity added by parallel circuits): the constraint matrix then depends on eta
     * (the A(eta) of Eq. 2) and the gradient includes that dependence.  0 keeps beta fixed. */
    const double* line_beta_ref;
} gx_network_desc;

/* One scenario: a horizon of T hours on network `net` (Sec. 2.1: a scenario can
 * be an hour, a day or a week of operations). */
typedef struct {
    int net;                     /* index into the networks given at create */
    int T;                       /* 1 <= T <= 256 */
    const double* load;          /* [n_bus * T] MW >= 0, row-major bus x hour */
    const double* cf;            /* [n_gen * T] capacity factor in [0, 1] */
    double weight;               /* w_s > 0 (1/S in Eq. 1) */
} gx_scenario_desc;

typedef struct {
    /* model (Eq. 2 with the eps regularisation; emissions weight kappa of Sec. 2.1) */
    double eps;          /* $/MW^2h regularisation on generation, shed, charge, discharge */
    double voll;         /* $/MWh value of lost load */
    double kappa;        /* $/t weight of emissions in the planner objective h */
    /* message passing */
    double rho;          /* power penalty, $/MW^2h */
    double rho_theta_c;  /* phase penalty scale: rho_theta_l = rho * rho_theta_c * w_l */
    int theta_weight;    /* 0: w_l = mean(beta^2) (uniform), 1: w_l = beta_l^2 (per line) */
    double rho_inner_c;  /* battery inner penalty rho_in = rho * rho_inner_c */
    int inner_iters;     /* battery inner iterations per outer iteration, >= 1 */
    double tol;          /* stop when primal and dual relative residuals <= tol */
    int max_iter;
    int check_every;     /* iterations between residual checks (FP64 reduction and the
                            convergence test; a host sync only in launch modes 1 and 0) */
    /* adjoint */
    double tol_active;   /* a bound is active if its multiplier exceeds tol_active times the
                            largest |generator cost| of the networks (at least 1 $/MWh), so
                            the test scales with the costs; default 1e-5 */
    double adj_tol;
    int adj_max_iter;
    int grad_envelope;   /* 1: for kappa == 0 use the envelope theorem (no adjoint solve) */
    double adj_rho;      /* power penalty of the adjoint iteration (its phase and battery inner
                            penalties scale with it as in the forward); the adjoint's free
                            devices have curvature eps only, so a penalty near eps converges
                            far faster than the forward's rho */
    double adj_rho_theta_c;  /* phase penalty scale of the adjoint iteration (rho_theta_l =
                                adj_rho * adj_rho_theta_c * w_l); 0: rho_theta_c */
    double adj_rho_inner_c;  /* battery and ramp inner penalty scale of the adjoint; 0: rho_inner_c */
    int adj_inner_iters;     /* battery inner iterations per adjoint iteration; 0: inner_iters */
} gx_opts;

enum { GX_WARM_COLD = 0, GX_WARM_PREV = 1, GX_WARM_USER = 2, GX_WARM_LEARNED = 3 };

/* Arrays exported through gx_network_array (FP32 unless noted). */
enum {
    GX_ARR_P = 0,        /* [G x Tp] generator output, MW */
    GX_ARR_SHED = 1,     /* [N x Tp] load shed, MW */
    GX_ARR_FLOW = 2,     /* [L x Tp] line flow from -> to, MW (beta * delta) */
    GX_ARR_THETA = 3,    /* [N x Tp] bus angle (consensus average), rad */
    GX_ARR_CH = 4,       /* [B x Tp] battery charge, MW */
    GX_ARR_DIS = 5,      /* [B x Tp] battery discharge, MW */
    GX_ARR_SOC = 6,      /* [B x Tp] state of charge, MWh */
    GX_ARR_PRICE = 7,    /* [N x Tp] nodal price, $/MWh */
    GX_ARR_COST = 8,     /* [S] FP64 operating cost c_s (after gx_dispatch_solve_batch) */
    GX_ARR_H = 9,        /* [S] FP64 planner objective h_s */
    GX_ARR_ITERS = 10,   /* [S] int32 iterations of the last solve */
    GX_ARR_RESID = 11,   /* [S x 2] FP64 primal, dual relative residual */
    GX_ARR_STATUS = 12,  /* [S] int32 per-scenario gx_status of the last solve */
    GX_ARR_GRAD_S = 13,  /* [sum_s K_net(s)] FP64 per-scenario dh_s/deta of the last grad */
    GX_ARR_ADJ_ITERS = 14, /* [S] int32 adjoint iterations */
    GX_ARR_OBJ = 15,     /* [1] FP64 sum_{s in batch} w'_s h_s of the last solve: the operating
                            term of Eq. 1 (w'_s as in gx_dispatch_grad_batch); scen must be -1 */
    GX_ARR_WARM = 16     /* [S] int32 start each scenario kept in the last solve: 1 the learned
                            start, 0 the previous plan's (GX_WARM_LEARNED's selection rule),
                            -1 not a learned solve or outside the batch */
};

typedef struct {
    int iters_max;        /* largest per-scenario iteration count */
    int n_converged;      /* scenarios that met tol */
    int n_scen;           /* scenarios in the batch */
    int launches;         /* kernel launches issued by the call */
    double max_primal, max_dual; /* worst relative residuals at exit */
} gx_stats;

gx_status gx_opts_default(gx_opts* opts);
const char* gx_status_string(gx_status s);
const char* gx_last_error_message(void);

/* The data of Eq. 2 (Section 2.1): the networks' devices (generators, loads, AC and
 * HVDC lines, batteries) and the scenarios' hourly profiles; the plan eta enters later,
 * per call.  Validates and copies the descriptors (host memory, read only here) and lays
 * out the workspace; no device work.  *out receives the handle (free with
 * gx_network_destroy).  Errors: GX_ERR_INVALID_ARG (bad index, non-positive
 * beta/dur/eff, T out of range, negative load, cf outside [0,1], non-finite numbers). */
gx_status gx_network_create(const gx_network_desc* nets, int n_nets, const gx_scenario_desc* scen, int S,
                            const gx_opts* opts, gx_network** out);
gx_status gx_network_destroy(gx_network* net);
size_t gx_network_device_bytes(const gx_network* net);
int gx_network_K(const gx_network* net);             /* total plan length */
int gx_network_S(const gx_network* net);
/* Upload static data into dev_mem (>= gx_network_device_bytes, 256-byte aligned)
 * and zero the state.  Asynchronous on `stream`. */
gx_status gx_network_bind(gx_network* net, void* dev_mem, size_t bytes, void* stream);
/* Drop the previous solution that the warm starts of the interactive planning loop reuse
 * (Section 2.2; Section 3.2 on warm starts), as a fresh bind does, without touching the workspace's data:
 * the next GX_WARM_PREV solve starts cold, the next GX_WARM_LEARNED solve takes the learned
 * start for every scenario (no selection trial), and gx_dispatch_grad_batch needs a new
 * solve (its GX_WARM_PREV then starts cold too).  Host only, no device work.  Errors:
 * GX_ERR_STATE if the network is not bound. */
gx_status gx_network_forget(gx_network* net);
/* Replace the options (rho, tolerances, ...); model constants eps/voll/kappa too.
 * Recomputes the battery factorisation on the next solve. */
gx_status gx_network_set_opts(gx_network* net, const gx_opts* opts);
/* Byte offset (from dev_mem) and element count of array `which` for scenario
 * `scen` (scen = -1: the whole array over all scenarios). */
gx_status gx_network_array(const gx_network* net, int which, int scen, size_t* offset_bytes, size_t* count);
/* Byte range [offset, offset + bytes) of the message passing's iteration state inside the
 * workspace: which = 0 the forward solve's, 1 the adjoint's.  The state is every FP32 array
 * the iteration carries from one step to the next (device outputs, line phase copies,
 * battery and ramp inner copies and multipliers, bus duals and averages), contiguous in
 * that order; alignment gaps between arrays stay zero.  Saving it after a call and writing
 * it back before a GX_WARM_PREV call restores that warm start exactly (checkpointing).
 * Errors: GX_ERR_INVALID_ARG for a NULL argument or another `which`. */
gx_status gx_network_state_range(const gx_network* net, int which, size_t* offset_bytes, size_t* bytes);
/* Row stride Tp and device counts of scenario s. */
gx_status gx_network_scenario_info(const gx_network* net, int s, int* T, int* Tp, int* N, int* G, int* L, int* B,
                                   int* eta_offset);

/* Solve Eq. 2 for the scenarios scen_idx[0..B) (host array; NULL = all S) at plan
 * eta_dev [K].  warm: GX_WARM_COLD (zero state), GX_WARM_PREV (continue from the
 * state of the previous solve), GX_WARM_USER (initial prices and angles from
 * warm_dev: [sum_s N_s Tp_s] prices followed by the same size of angles, in
 * scenario order of the whole network; generators and loads start at their best
 * response to those prices, line flows from the angle differences), GX_WARM_LEARNED (the
 * network attached with gx_network_attach_gnn predicts the prices and angles at eta_dev,
 * applied as a user start; when a previous solution exists, every scenario first runs one
 * residual-check chunk from the previous plan's state and one from the learned start and
 * keeps the one with the smaller residual at its check (GX_ARR_WARM records the choice), the
 * loop then continuing from iteration check_every; without an attached network,
 * GX_ERR_STATE).  Outputs stay in
 * the workspace (GX_ARR_*), including GX_ARR_OBJ, the batch's weighted planner value.
 * Synchronises `stream` once at the end of the iteration loop (per residual-check chunk
 * in launch modes 1 and 0).  Returns GX_NOT_CONVERGED if any scenario of the batch
 * hit max_iter, GX_ERR_NONFINITE if one diverged (its outputs are then meaningless). */
gx_status gx_dispatch_solve_batch(gx_network* net, const float* eta_dev, const int* scen_idx, int B, int warm,
                                  const float* warm_dev, gx_stats* stats, void* stream);

/* Section 2.2: the implicit gradient, by the implicit function theorem on the optimality
 * conditions of the solved dispatch (Eq. 2), of sum_{s in batch} w'_s h_s at the last
 * solve (same batch),
 * w'_s = w_s * (sum of all weights) / (sum of the batch's weights), written to
 * grad_dev [K] (FP32, caller-owned; entries of networks outside the batch are 0).
 * warm: GX_WARM_COLD or GX_WARM_PREV for the adjoint state.  Per-scenario FP64
 * gradients are kept in GX_ARR_GRAD_S.  Errors: GX_ERR_STATE if no solve. */
gx_status gx_dispatch_grad_batch(gx_network* net, const float* eta_dev, int warm, float* grad_dev,
                                 gx_stats* stats, void* stream);

/* eta <- min(max(eta - alpha * (gamma + grad), eta_min), eta_max), elementwise
 * over K entries, all device pointers (Sec. 2.2 projected step). */
gx_status gx_plan_step(gx_network* net, float* eta_dev, const float* grad_dev, const float* gamma_dev,
                       const float* eta_min_dev, const float* eta_max_dev, float alpha, void* stream);

/* How the per-iteration kernels are launched.  2 (default): the whole loop is one CUDA
 * graph; a conditional WHILE node repeats one residual-check chunk and the convergence
 * test on the device, so the host launches once and synchronises once per loop (used
 * when max_iter is a multiple of check_every and sampled timing is off; otherwise mode 1).
 * 1: one graph per residual-check chunk, the host reading the active-scenario count after
 * each.  0: kernel-by-kernel launches.  All modes run the same kernels in the same order:
 * results are bitwise identical.  Other values: GX_ERR_INVALID_ARG. */
gx_status gx_network_use_graphs(gx_network* net, int on);

/* Kernel schedule of the per-iteration path (not in the paper; performance only: every
 * schedule computes the same iterates, bitwise).
 *   bus_staged  how the hour-quad bus kernel reads its block's device rows.  1: bulk
 *               copies (TMA) of every row segment into shared memory, completing on an
 *               mbarrier, so all of the block's rows are in flight at once; 2: the same
 *               stage filled by per-thread 16-byte asynchronous copies; 0: each thread
 *               loads its bus's device rows itself, one generator ahead.  Until a schedule
 *               is set, bind picks 1 when the workspace exceeds the device's L2 cache (the
 *               iteration streams from HBM) and 0 otherwise (L2-resident and
 *               latency-bound, where 0 measured fastest).
 *   bat_warps   warps per battery of the battery prox when the longest horizon exceeds
 *               96 hours: 2 (default; hours split over 64 lanes, warp totals combined in
 *               shared memory) or 1 (32 lanes, longer serial sweeps, no block barriers).
 * Setting it drops the cached graphs.  Errors: GX_ERR_INVALID_ARG for other values. */
typedef struct {
    int bus_staged;
    int bat_warps;
} gx_schedule;
gx_status gx_network_set_schedule(gx_network* net, const gx_schedule* sched);
gx_status gx_network_get_schedule(const gx_network* net, gx_schedule* sched);

/* Cluster-resident solver (default off).  A scenario whose state fits the shared memory
 * of a thread-block cluster (1 to 16 CTAs; each CTA holds every device for a range of
 * hours, batteries exchange their hours over distributed shared memory) runs its whole
 * forward or adjoint loop in one persistent launch that tests its own convergence.
 * Other scenarios, and all of them while this is off, run on the per-iteration kernels.
 * The two paths take the same iterates up to the summation order of the residual
 * partials (so possibly a different stopping chunk). */
gx_status gx_network_use_persistent(gx_network* net, int on);
/* *cluster_ctas: CTAs of the cluster scenario `scen` runs on, 0 if it runs on the
 * per-iteration kernels (not resident, not launchable on this device, or switched off). */
gx_status gx_network_persistent_info(const gx_network* net, int scen, int* cluster_ctas);

/* Sampled kernel timing (the network must be bound).  While enabled, the last iteration of
 * every residual-check chunk stamps, per kernel kind, its earliest block start and latest
 * block end with the device's global nanosecond timer (%globaltimer) inside the kernels,
 * so the times are those of the launch mode in use (the whole-loop graph included), with
 * no events between the kernels; the host reads them at the end of each loop.  Cluster-
 * resident launches are timed with CUDA events around them.  Kinds: 0 = bus kernel,
 * 1 = line kernel, 2 = battery (and ramp) kernels, 3 = cluster-resident launches.  The
 * line and battery kernels run side by side in the graph modes, so kinds 1 and 2 overlap.
 * Enabling resets the counters; switching timing on or off drops the cached graphs, whose
 * kernels carry the timing pointers.  Uses four CUDA events and workspace memory, no
 * device allocation. */
gx_status gx_profile_enable(gx_network* net, int on);
/* Arrays of 4.  ms[k]: summed time of the sampled launches of kind k; samples[k]: how many
 * were sampled; launches[k]: all launches of kind k since enabling. */
gx_status gx_profile_read(const gx_network* net, double* ms, long long* samples, long long* launches);
/* counts [S]: for each scenario, how many of the sampled iterations (kinds 0-2) it was
 * still iterating in, since timing was enabled.  A converged scenario's blocks exit at
 * once, so a sampled launch only does the work of the scenarios counted here. */
gx_status gx_profile_active(const gx_network* net, long long* counts);

/* ------------------------------------------------------------------------------
 * Learned warm start (not in the paper): a 3-layer message-passing network over the
 * bus-hour graph of a bound network (node (n, t) linked to (m, t) when a line joins
 * n and m; hidden width 64; BF16 tcgen05 tensor-core layers with FP32 accumulation) maps
 * plan-derived node features to nodal prices and angles.  Its predictions, in the
 * layout of GX_WARM_USER ([sum_s N_s Tp_s] prices then the same size of angles), warm
 * start gx_dispatch_solve_batch.  Parameters: FP32 master copy of gx_gnn_num_params()
 * floats (layout documented in paper_2410_13055_gb300/csrc/gx_gnn.cu); the device
 * workspace is caller-allocated like the network's.
 * ------------------------------------------------------------------------------ */
typedef struct gx_gnn gx_gnn;
size_t gx_gnn_num_params(void);
/* hidden must be 64, layers 3.  The network must be bound and outlive the gx_gnn. */
gx_status gx_gnn_create(const gx_network* net, int hidden, int layers, gx_gnn** out);
size_t gx_gnn_device_bytes(const gx_gnn* gnn);
/* Zero the workspace and initialise the parameters from `seed` (synchronises `stream`). */
gx_status gx_gnn_bind(gx_gnn* gnn, void* dev_mem, size_t bytes, uint64_t seed, void* stream);
gx_status gx_gnn_set_params(gx_gnn* gnn, const float* host_params, size_t n, void* stream);
/* which = 0: parameters, 1: gradients of the last gx_gnn_train_step (synchronises). */
gx_status gx_gnn_get_params(const gx_gnn* gnn, float* host_out, size_t n, int which, void* stream);
/* Predicted prices ($/MWh) and angles (rad) at plan eta_dev into out_dev [2 * bus rows].
 * Asynchronous; the tensor-core layers' copy and MMA waits are bounded, and one that ran
 * out (never expected) is returned as GX_ERR_TIMEOUT by the next gx_gnn_train_step that
 * reads its loss. */
gx_status gx_gnn_predict(gx_gnn* gnn, const float* eta_dev, float* out_dev, void* stream);
/* One Adam step (lr > 0; lr = 0 only computes gradients) on the mean squared error
 * against target_dev (same layout as out_dev; prices compared in $/100 MWh units,
 * angles weighted by w_theta); padding hours are excluded.  loss_host (nullable)
 * receives the loss before the step (synchronises); with it, GX_ERR_TIMEOUT reports a
 * tensor-core wait that ran out in this step or an earlier prediction. */
gx_status gx_gnn_train_step(gx_gnn* gnn, const float* eta_dev, const float* target_dev, float lr, float w_theta,
                            double* loss_host, void* stream);
gx_status gx_gnn_destroy(gx_gnn* gnn);
/* Attach (gnn != NULL) or detach (NULL) the learned start of GX_WARM_LEARNED.  The warm-
 * start network must have been created for `net`, be bound, and outlive the attachment; its
 * workspace also holds the forward state while a learned solve compares the two starts.
 * Errors: GX_ERR_INVALID_ARG for a network created for another one. */
gx_status gx_network_attach_gnn(gx_network* net, gx_gnn* gnn);

/* Operating cost c_s and planner value h_s of scenario `scen` at the last solve,
 * computed without allocating any device memory.  The paper has no counterpart; this
 * entry point exists for callers that cannot allocate device memory: host applications
 * that give the library a fixed memory budget, plugins whose device memory belongs to a
 * host framework's allocator, and latency-critical loops in which an allocation may
 * synchronise the device.
 *
 * Same sums as GX_ARR_COST / GX_ARR_H of gx_dispatch_solve_batch, but the per-block
 * partial sums go to a fixed 64 KiB array compiled into the library (held on every
 * GPU that loads it until the process exits) instead of the workspace.  Writes one
 * double to cost_out_dev and, if h_out_dev is not NULL, one to h_out_dev (device
 * pointers owned by the caller).  Limit: (G + N + B) * Tp <= 16,777,216 for the
 * scenario (4096 partial-sum slots); larger scenarios return GX_ERR_INVALID_ARG with
 * a message.  A network that is bound but has not been solved since returns
 * GX_ERR_STATE.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture.  Every call shares the one array, so calls that overlap on the GPU
 * (different streams, no ordering) race and must not be issued; calls on one stream
 * are ordered and safe.  Asynchronous on `stream`. */
gx_status gx_dispatch_cost_noalloc(const gx_network* net, int scen, double* cost_out_dev, double* h_out_dev,
                                   void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GX_H */
