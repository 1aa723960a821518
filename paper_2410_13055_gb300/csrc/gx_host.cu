// Host side of the C ABI (include/gx.h): descriptor validation, workspace layout,
// bind (upload of static data), and the drivers of the solve, gradient and plan step.
#include "gx_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <string>
#include <vector>

using namespace gx;

namespace {

thread_local std::string g_err;

gx_status fail(gx_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define GX_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(GX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct NetH {
    int N = 0, G = 0, L = 0, B = 0;
    std::vector<int> gen_bus, line_from, line_to, bat_bus;
    std::vector<uint8_t> line_dc;  // 1: HVDC transport line
    std::vector<double> gen_ramp;   // ramp limit / capacity per hour (0: none)
    std::vector<int> ramp_gens;     // generators with a ramp limit in (0, 1)
    std::vector<int> g_ramp;        // per generator: its index in ramp_gens, -1 if none
    int ramp0 = 0;                  // offset of ramp_gens in the concatenated static arrays
    std::vector<double> gen_cost, gen_emis, line_beta, line_dth, bat_dur, bat_effc, bat_effd;
    std::vector<int> gptr, gidx, bptr, bidx, eptr, eidx;
    std::vector<float> inv_cnt, inv_wsum, dres_w, l_w;
    std::vector<uint8_t> firm;
    int gen0 = 0, line0 = 0, bat0 = 0, bus0 = 0, ptr0 = 0, eta0 = 0;
    std::vector<double> line_bref;  // reference capacity of a scaling susceptance (0: fixed beta)
    std::vector<int> l_scale;       // per line: its scaling index, -1 if beta is fixed
    std::vector<int> bus_sdres;     // per bus: its dual-residual record among the scaling ones, -1 if none
};

struct ScenH {
    int net = 0, T = 0, Tp = 0;
    double weight = 1.0;
    std::vector<float> load, cf;  // padded rows
};

// Byte offsets of every array in the workspace (256-byte aligned).
struct Layout {
    size_t total = 0;
    size_t add(size_t bytes) {
        size_t o = total;
        total += (bytes + 255) / 256 * 256;
        return o;
    }
};

bool isfin(double x) { return std::isfinite(x); }

}  // namespace

struct gx_network {
    gx_opts opts{};
    int n_nets = 0, S = 0, K = 0;
    // price scale of the active-set test: the largest |generator cost| of the batch's
    // networks, at least 1 $/MWh (multipliers scale with the costs)
    double cost_scale = 1.0;
    std::vector<NetH> nets;
    std::vector<ScenH> scens;
    std::vector<ScenDev> sdev;
    std::vector<int> bus_blk_scen, line_blk_scen, bat_warp_scen, cost_blk_scen, gwarp, k_net;
    std::vector<BusBlk> bus_blk;       // bus-kernel block records (single-hour kernel)
    std::vector<BusBlk> bus4_blk;      // bus-kernel block records (hour-quad kernel)
    std::vector<int> line4_blk_scen;   // scenario of each hour-quad line block
    std::vector<LineBlk> line4_blk;    // its offsets
    std::vector<BatW> bat_w;           // offsets of each battery warp
    int n_bus4_blk = 0, n_line4_blk = 0;
    size_t bus4_smem = 0;              // dynamic shared memory of the staged bus kernel (record + stage)
    std::vector<int> pool;             // their pool records (words)
    std::vector<int> bus_cpl;          // per hour-quad bus block: copy-list header and list (fixed stride)
    int bus_cpl_stride = 0, bus_cpl_max = 0;
    bool l2_resident = false;          // the bound workspace fits the device's L2 (set at bind)
    std::vector<int2> prep;            // (pool word, eta index) of each generator plan value
    std::vector<uint8_t> firm;         // generator has capacity factor 1 in every hour of every scenario
    // lines whose susceptance scales with capacity (gx_scale.cu)
    std::vector<int> sc_line, sc_eta, sc_gwarp;
    std::vector<double> sc_b, sc_bmin;
    std::vector<int2> sc_pool, sc_dres_l;
    std::vector<ScaleDres> sc_dres, sc_dres_pool;  // bus_dres_w targets; pool-word targets
    // cluster-resident solver: scenarios grouped by (cluster size, hours per battery lane)
    struct CrsGroup {
        int C = 0, hpl = 0, first = 0, n = 0;
        size_t smem = 0;
        bool ok = false;  // launchable on this device (checked at bind)
    };
    std::vector<CrsGroup> crs_groups;
    std::vector<int> crs_list;         // scenario indices, group by group
    std::vector<int> crs_group;        // per scenario: its group, -1 = per-iteration kernels only
    std::vector<int> done_loop;        // done flags of the per-iteration loop (cluster-resident ones set)
    bool use_crs = false;
    long long bus_el = 0, gen_el = 0, line_el = 0, bat_el = 0;
    int n_bus_blk = 0, n_line_blk = 0, n_bat_warps = 0, n_cost_blk = 0, n_gwarps = 0, gs_total = 0;
    int tot_gen = 0, tot_line = 0, tot_bat = 0, tot_bus = 0, tot_ptr = 0, tot_ramp = 0;
    std::vector<int> ramp_warp_scen;   // scenario of each ramp-kernel warp
    int n_ramp_warps = 0;
    long long ramp_el = 0;             // ramp state rows x Tp over all scenarios
    int max_ramp_T = 1;
    // workspace offsets
    size_t o_scen, o_bbs, o_lbs, o_bws, o_cbs, o_gwarp, o_knet, o_busblk, o_pool, o_prep, o_crs;
    size_t o_bus4blk, o_l4bs, o_l4blk, o_batw, o_buscpl, o_busdone;
    size_t o_scl, o_sce, o_scb, o_scbm, o_scp, o_scd, o_scdl, o_scgw;
    size_t o_rgen, o_rrate, o_gramp, o_rws, o_rdd, o_ardd, o_rf[4], o_ra[4], o_rpart;
    size_t o_gbus, o_gcost, o_gemis, o_gfirm, o_lfrom, o_lto, o_lbeta, o_ldth, o_lw, o_bbus, o_bdur, o_beffc, o_beffd;
    size_t o_gptr, o_gidx, o_bptr, o_bidx, o_eptr, o_eidx, o_icnt, o_iwsum, o_dresw;
    size_t o_load, o_cf, o_dd, o_add;
    size_t static_end;
    size_t o_f[16], o_a[16];  // forward / adjoint state arrays, order of StatePtrs
    size_t o_fend, o_aend;    // end of the forward / adjoint state range (ramp arrays included)
    size_t o_mgen, o_mload, o_mline, o_mbat, o_ag, o_al;
    size_t o_done, o_iters, o_status, o_adjit, o_nact, o_ctr, o_inb, o_err, o_wsel, o_resid, o_rbest, o_cost, o_h, o_grads, o_wprime, o_obj, o_stlo, o_sthi, o_pact;
    size_t o_flow, o_price, o_shed, o_bpart, o_lpart, o_btpart, o_cpart;
    Layout lay;
    // binding
    uint8_t* dev = nullptr;
    bool solved = false, adj_ready = false, dd_dirty = true;
    std::vector<int> in_batch, done_init;
    std::vector<double> wprime;
    std::vector<float> dd_host, add_host, rdd_host, ardd_host;
    Ctx ctx{}, actx{};
    // CUDA graphs of one residual-check chunk, keyed by what their captured parameters depend on
    struct ChunkGraph {
        bool valid = false;
        int adj = 0, chunk = 0, loop = 0;  // loop: the whole loop (conditional WHILE node)
        const float* eta = nullptr;
        cudaGraphExec_t exec = nullptr;
    } graphs[4];
    int graph_next = 0;
    cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int* h_nact = nullptr;  // pinned host copies: [0] active-scenario count, [1] iteration counter
    int use_graphs = 2;     // 0 eager launches, 1 one graph per chunk, 2 the whole loop as one graph
    gx_schedule sched{1, 2};  // kernel schedule (gx_network_set_schedule)
    bool sched_set = false;   // the caller chose the schedule (else bind picks it by workspace size)
    gx_gnn* gnn = nullptr;    // learned start (gx_network_attach_gnn)
    void drop_graphs() {
        for (auto& g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g = ChunkGraph{};
        }
    }
    // sampled kernel timing
    bool prof = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double prof_ms[4] = {0, 0, 0, 0};
    long long prof_samples[4] = {0, 0, 0, 0}, prof_launches[4] = {0, 0, 0, 0};
    ~gx_network() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        drop_graphs();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (cap_stream2) cudaStreamDestroy(cap_stream2);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (h_nact) cudaFreeHost(h_nact);
    }
};

static double adj_theta_c(const gx_opts& o) { return o.adj_rho_theta_c > 0 ? o.adj_rho_theta_c : o.rho_theta_c; }
static double adj_inner_c(const gx_opts& o) { return o.adj_rho_inner_c > 0 ? o.adj_rho_inner_c : o.rho_inner_c; }

static void fill_dd_for(gx_network* net, double rho, double inner_c, std::vector<float>& out) {
    // Thomas pivots of the battery tridiagonal system (one row per battery and scenario):
    // diag = [1 + g rho_in, 2 + g rho_in, ...], off-diagonal -1, with
    // g = [a, -k] H^{-1} [a, -k]^T and H = [[eps+rho_in+rho, -rho], [-rho, eps+rho_in+rho]].
    const double eps = net->opts.eps, ri = rho * inner_c;
    out.assign((size_t)net->bat_el, 1.0f);
    for (int s = 0; s < net->S; ++s) {
        const ScenH& sc = net->scens[s];
        const NetH& nh = net->nets[sc.net];
        for (int b = 0; b < nh.B; ++b) {
            const double a = nh.bat_effc[b], k = 1.0 / nh.bat_effd[b];
            const double A = eps + ri + rho, det = A * A - rho * rho;
            const double gc = (A * a - rho * k) / det, gd = (rho * a - A * k) / det;
            const double g = a * gc - k * gd;
            double d = 1.0 + g * ri;
            float* o = out.data() + net->sdev[s].e_bat + (size_t)b * sc.Tp;
            o[0] = (float)d;
            for (int t = 1; t < sc.T; ++t) {
                d = (2.0 + g * ri) - 1.0 / d;
                o[t] = (float)d;
            }
        }
    }
}

// Thomas pivots of the ramp prox's x-step (one row per ramping generator and scenario):
// (eps + rho + rho_in) I + rho_in D^T D, D the first difference over T hours, so the
// diagonal is a + rho_in [1, 2, ..., 2, 1] (a alone for T = 1) and the off-diagonal -rho_in.
// Stored as 1 / m_t for m_0 = diag_0, m_t = diag_t - rho_in^2 / m_{t-1}.
static void fill_ramp_dd_for(gx_network* net, double rho, double inner_c, std::vector<float>& out) {
    const double eps = net->opts.eps, ri = rho * inner_c, a = eps + rho + ri;
    out.assign((size_t)std::max<long long>(net->ramp_el, 1), 1.0f);
    for (int s = 0; s < net->S; ++s) {
        const ScenDev& sd = net->sdev[s];
        for (int r = 0; r < sd.R; ++r) {
            float* o = out.data() + sd.e_ramp + (size_t)r * sd.Tp;
            double m = 0;
            for (int t = 0; t < sd.T; ++t) {
                const double dg = sd.T == 1 ? 0.0 : ((t == 0 || t == sd.T - 1) ? 1.0 : 2.0);
                const double diag = a + ri * dg;
                m = t == 0 ? diag : diag - ri * ri / m;
                o[t] = (float)(1.0 / m);
            }
        }
    }
}

static void fill_dd(gx_network* net) {
    const gx_opts& o = net->opts;
    fill_dd_for(net, o.rho, o.rho_inner_c, net->dd_host);
    fill_dd_for(net, o.adj_rho, adj_inner_c(o), net->add_host);
    fill_ramp_dd_for(net, o.rho, o.rho_inner_c, net->rdd_host);
    fill_ramp_dd_for(net, o.adj_rho, adj_inner_c(o), net->ardd_host);
    net->dd_dirty = true;
}

static void make_ctx(gx_network* net) {
    Ctx& c = net->ctx;
    uint8_t* d = net->dev;
    auto F = [&](size_t o) { return reinterpret_cast<float*>(d + o); };
    auto I = [&](size_t o) { return reinterpret_cast<int*>(d + o); };
    auto D = [&](size_t o) { return reinterpret_cast<double*>(d + o); };
    auto U8 = [&](size_t o) { return reinterpret_cast<uint8_t*>(d + o); };
    c.S = net->S;
    c.n_bus_blk = net->n_bus_blk;
    c.n_line_blk = net->n_line_blk;
    c.n_bat_warps = net->n_bat_warps;
    c.n_cost_blk = net->n_cost_blk;
    const gx_opts& o = net->opts;
    c.rho = (float)o.rho;
    c.eps = (float)o.eps;
    c.voll = (float)o.voll;
    c.kappa = (float)o.kappa;
    c.rho_in = (float)(o.rho * o.rho_inner_c);
    c.rth_c = (float)(o.rho * o.rho_theta_c);
    c.tol_act = (float)(o.tol_active * net->cost_scale);
    c.inner_iters = o.inner_iters;
    c.check_every = o.check_every;
    c.scen = reinterpret_cast<const ScenDev*>(d + net->o_scen);
    c.bus_blk_scen = I(net->o_bbs);
    c.bus_blk = reinterpret_cast<const BusBlk*>(d + net->o_busblk);
    c.bus4_blk = reinterpret_cast<const BusBlk*>(d + net->o_bus4blk);
    c.bus_cpl = (net->bus_cpl.empty() || !net->l2_resident) ? nullptr : reinterpret_cast<const int*>(d + net->o_buscpl);
    c.bus_cpl_stride = net->bus_cpl_stride;
    c.bus_cpl_max = net->bus_cpl_max;
    c.bus_done = reinterpret_cast<int*>(d + net->o_busdone);
    c.n_ramp_warps = net->n_ramp_warps;
    c.ramp_warp_scen = I(net->o_rws);
    c.r_gen = I(net->o_rgen);
    c.r_rate = F(net->o_rrate);
    c.g_ramp = I(net->o_gramp);
    c.ramp_dd = F(net->o_rdd);
    c.max_ramp_T = net->max_ramp_T;
    float** rfs[4] = {&c.rz, &c.rw, &c.ry, &c.rq};
    float** ras[4] = {&c.a_rz, &c.a_rw, &c.a_ry, &c.a_rq};
    for (int k = 0; k < 4; ++k) { *rfs[k] = F(net->o_rf[k]); *ras[k] = F(net->o_ra[k]); }
    c.ramp_part = F(net->o_rpart);
    c.line4_blk_scen = I(net->o_l4bs);
    c.line4_blk = reinterpret_cast<const LineBlk*>(d + net->o_l4blk);
    c.bat_w = reinterpret_cast<const BatW*>(d + net->o_batw);
    c.n_bus4_blk = net->n_bus4_blk;
    c.n_line4_blk = net->n_line4_blk;
    c.pool = I(net->o_pool);
    c.prep = reinterpret_cast<const int2*>(d + net->o_prep);
    c.n_prep = (int)net->prep.size();
    c.sc_line = I(net->o_scl);
    c.sc_eta = I(net->o_sce);
    c.sc_b = D(net->o_scb);
    c.sc_bmin = D(net->o_scbm);
    c.sc_pool = reinterpret_cast<const int2*>(d + net->o_scp);
    c.sc_dres = reinterpret_cast<const ScaleDres*>(d + net->o_scd);
    c.sc_dres_l = reinterpret_cast<const int2*>(d + net->o_scdl);
    c.sc_gwarp = I(net->o_scgw);
    c.l_beta_w = F(net->o_lbeta);
    c.dres_w_w = F(net->o_dresw);
    c.n_scale = (int)net->sc_line.size();
    c.n_sc_pool = (int)net->sc_pool.size();
    c.n_sc_dres = (int)net->sc_dres.size();
    c.n_sc_gwarps = (int)net->sc_gwarp.size() / 2;
    c.line_blk_scen = I(net->o_lbs);
    c.bat_warp_scen = I(net->o_bws);
    c.cost_blk_scen = I(net->o_cbs);
    c.g_bus = I(net->o_gbus); c.g_cost = F(net->o_gcost); c.g_emis = F(net->o_gemis); c.g_firm = U8(net->o_gfirm);
    c.l_from = I(net->o_lfrom); c.l_to = I(net->o_lto); c.l_beta = F(net->o_lbeta); c.l_dth = F(net->o_ldth);
    c.l_w = F(net->o_lw);
    c.b_bus = I(net->o_bbus); c.b_dur = F(net->o_bdur); c.b_effc = F(net->o_beffc); c.b_effd = F(net->o_beffd);
    c.bus_gptr = I(net->o_gptr); c.bus_gidx = I(net->o_gidx);
    c.bus_bptr = I(net->o_bptr); c.bus_bidx = I(net->o_bidx);
    c.bus_eptr = I(net->o_eptr); c.bus_eidx = I(net->o_eidx);
    c.bus_inv_cnt = F(net->o_icnt); c.bus_inv_wsum = F(net->o_iwsum); c.bus_dres_w = F(net->o_dresw);
    c.load = F(net->o_load); c.cf = F(net->o_cf); c.bat_dd = F(net->o_dd);
    float** fs[16] = {&c.xg, &c.xl, &c.dl, &c.sg, &c.vf, &c.vt, &c.xb, &c.zc, &c.zd, &c.zs, &c.yc, &c.yd, &c.ys,
                      &c.u, &c.pbar, &c.thb};
    float** as[16] = {&c.a_xg, &c.a_xl, &c.a_dl, &c.a_sg, &c.a_vf, &c.a_vt, &c.a_xb, &c.a_zc, &c.a_zd, &c.a_zs,
                      &c.a_yc, &c.a_yd, &c.a_ys, &c.a_u, &c.a_pbar, &c.a_thb};
    for (int k = 0; k < 16; ++k) { *fs[k] = F(net->o_f[k]); *as[k] = F(net->o_a[k]); }
    c.m_gen = U8(net->o_mgen); c.m_load = U8(net->o_mload); c.m_line = U8(net->o_mline); c.m_bat = U8(net->o_mbat);
    c.ag = reinterpret_cast<float*>(net->dev + net->o_ag);
    c.al = reinterpret_cast<float*>(net->dev + net->o_al);
    c.done = I(net->o_done); c.iters = I(net->o_iters); c.status = I(net->o_status); c.adj_iters = I(net->o_adjit);
    c.n_active = I(net->o_nact);
    c.iter_ctr = I(net->o_ctr);
    c.max_bat_T = 1;
    for (const ScenDev& d : net->sdev)
        if (d.B > 0) c.max_bat_T = std::max(c.max_bat_T, d.T);
    c.max_it = o.max_iter;
    c.resid = D(net->o_resid); c.rbest = D(net->o_rbest); c.cost = D(net->o_cost); c.hval = D(net->o_h); c.grad_s = D(net->o_grads);
    c.out_flow = F(net->o_flow); c.out_price = F(net->o_price); c.out_shed = F(net->o_shed);
    c.bus_part = F(net->o_bpart); c.line_part = F(net->o_lpart); c.bat_part = F(net->o_btpart);
    c.cost_part = D(net->o_cpart);
    c.warm = nullptr;
    c.warm_half = net->bus_el;
    c.eta = nullptr;
    c.stamp_lo = net->prof ? reinterpret_cast<unsigned long long*>(d + net->o_stlo) : nullptr;
    c.stamp_hi = net->prof ? reinterpret_cast<unsigned long long*>(d + net->o_sthi) : nullptr;
    c.prof_act = net->prof ? reinterpret_cast<long long*>(d + net->o_pact) : nullptr;
    c.bus_staged = net->sched.bus_staged;
    c.bus4_smem = (int)net->bus4_smem;
    c.bat_warps = net->sched.bat_warps;
    c.err = I(net->o_err);
    // the adjoint iteration: same arrays, its own penalties and battery pivots
    Ctx& a = net->actx;
    a = c;
    a.rho = (float)o.adj_rho;
    a.inner_iters = o.adj_inner_iters > 0 ? o.adj_inner_iters : o.inner_iters;
    a.rho_in = (float)(o.adj_rho * adj_inner_c(o));
    a.rth_c = (float)(o.adj_rho * adj_theta_c(o));
    a.bat_dd = F(net->o_add);
    a.ramp_dd = F(net->o_ardd);
    a.max_it = o.adj_max_iter;
    a.rho_ratio = (float)(o.rho / o.adj_rho);
    a.adj_from_fwd = 1;
    c.rho_ratio = 1.f;
    c.adj_from_fwd = 0;
    net->drop_graphs();
}

namespace gx {
// Condition of the device-side loop (a conditional WHILE node around one residual-check
// chunk): run another chunk while a scenario is still iterating and the cap is not reached.
// The reduction marks every scenario done once the counter reaches the cap, so the loop
// ends after at most cap / chunk bodies.
__global__ void k_loop_cond(const int* n_active, const int* iter_ctr, int max_it, cudaGraphConditionalHandle h) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, (*n_active > 0 && *iter_ctr < max_it) ? 1u : 0u);
}

int launch_loop_cond(const Ctx& c, int max_it, cudaGraphConditionalHandle h, cudaStream_t st) {
    k_loop_cond<<<1, 32, 0, st>>>(c.n_active, c.iter_ctr, max_it, h);
    return 1;
}

const Ctx* gx_internal_ctx(const gx_network* net) { return (net && net->dev) ? &net->ctx : nullptr; }
ScenDev gx_internal_scen(const gx_network* net, int s) { return net->sdev[s]; }
bool gx_internal_solved(const gx_network* net) { return net && net->dev && net->solved; }
gx_status gx_internal_fail(gx_status s, const std::string& msg) { return fail(s, msg); }
}  // namespace gx

extern "C" {

gx_status gx_opts_default(gx_opts* o) {
    if (!o) return fail(GX_ERR_INVALID_ARG, "opts is NULL");
    o->eps = 1e-3;
    o->voll = 1000.0;
    o->kappa = 0.0;
    o->rho = 0.3;
    o->rho_theta_c = 0.1;
    o->theta_weight = 0;
    o->rho_inner_c = 1.0;
    o->inner_iters = 2;
    o->tol = 1e-3;
    o->max_iter = 20000;
    o->check_every = 20;
    o->tol_active = 1e-5;
    o->adj_tol = 1e-3;
    o->adj_max_iter = 20000;
    o->grad_envelope = 0;
    o->adj_rho = 0.002;
    o->adj_rho_theta_c = 0.0;
    o->adj_rho_inner_c = 0.0;
    o->adj_inner_iters = 0;
    return GX_OK;
}

const char* gx_status_string(gx_status s) {
    switch (s) {
        case GX_OK: return "ok";
        case GX_NOT_CONVERGED: return "not converged (iteration cap reached)";
        case GX_ERR_INVALID_ARG: return "invalid argument";
        case GX_ERR_NONFINITE: return "non-finite value in the iterate";
        case GX_ERR_CUDA: return "CUDA error";
        case GX_ERR_NO_MEMORY: return "workspace too small";
        case GX_ERR_TIMEOUT: return "device wait timed out";
        case GX_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

const char* gx_last_error_message(void) { return g_err.c_str(); }

static gx_status check_opts(const gx_opts* o) {
    if (!(o->eps > 0 && isfin(o->eps))) return fail(GX_ERR_INVALID_ARG, "opts.eps must be > 0");
    if (!(o->voll > 0 && isfin(o->voll))) return fail(GX_ERR_INVALID_ARG, "opts.voll must be > 0");
    if (!(o->kappa >= 0 && isfin(o->kappa))) return fail(GX_ERR_INVALID_ARG, "opts.kappa must be >= 0");
    if (!(o->rho > 0 && isfin(o->rho))) return fail(GX_ERR_INVALID_ARG, "opts.rho must be > 0");
    if (!(o->adj_rho > 0 && isfin(o->adj_rho))) return fail(GX_ERR_INVALID_ARG, "opts.adj_rho must be > 0");
    if (!(o->rho_theta_c > 0 && isfin(o->rho_theta_c))) return fail(GX_ERR_INVALID_ARG, "opts.rho_theta_c must be > 0");
    if (!(o->rho_inner_c > 0 && isfin(o->rho_inner_c))) return fail(GX_ERR_INVALID_ARG, "opts.rho_inner_c must be > 0");
    if (o->inner_iters < 1 || o->inner_iters > 1000) return fail(GX_ERR_INVALID_ARG, "opts.inner_iters in [1, 1000]");
    if (o->adj_inner_iters < 0 || o->adj_inner_iters > 1000)
        return fail(GX_ERR_INVALID_ARG, "opts.adj_inner_iters in [0, 1000] (0: inner_iters)");
    if (!(o->tol > 0) || !(o->adj_tol > 0)) return fail(GX_ERR_INVALID_ARG, "tolerances must be > 0");
    if (o->max_iter < 1 || o->adj_max_iter < 1) return fail(GX_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (o->check_every < 1) return fail(GX_ERR_INVALID_ARG, "check_every must be >= 1");
    if (!(o->tol_active >= 0)) return fail(GX_ERR_INVALID_ARG, "tol_active must be >= 0");
    if (o->theta_weight != 0 && o->theta_weight != 1) return fail(GX_ERR_INVALID_ARG, "theta_weight is 0 or 1");
    if (!(o->adj_rho_theta_c >= 0 && isfin(o->adj_rho_theta_c)) || !(o->adj_rho_inner_c >= 0 && isfin(o->adj_rho_inner_c)))
        return fail(GX_ERR_INVALID_ARG, "opts.adj_rho_theta_c and adj_rho_inner_c must be >= 0 (0: the forward's)");
    return GX_OK;
}

static void derive_network(NetH& h, const gx_opts& o) {
    const int N = h.N;
    h.gptr.assign(N + 1, 0); h.bptr.assign(N + 1, 0); h.eptr.assign(N + 1, 0);
    for (int g = 0; g < h.G; ++g) h.gptr[h.gen_bus[g] + 1]++;
    for (int b = 0; b < h.B; ++b) h.bptr[h.bat_bus[b] + 1]++;
    for (int l = 0; l < h.L; ++l) { h.eptr[h.line_from[l] + 1]++; h.eptr[h.line_to[l] + 1]++; }
    for (int n = 0; n < N; ++n) { h.gptr[n + 1] += h.gptr[n]; h.bptr[n + 1] += h.bptr[n]; h.eptr[n + 1] += h.eptr[n]; }
    h.gidx.assign(h.G, 0); h.bidx.assign(h.B, 0); h.eidx.assign(2 * h.L, 0);
    std::vector<int> fg(h.gptr.begin(), h.gptr.end() - 1), fb(h.bptr.begin(), h.bptr.end() - 1),
        fe(h.eptr.begin(), h.eptr.end() - 1);
    for (int g = 0; g < h.G; ++g) h.gidx[fg[h.gen_bus[g]]++] = g;
    for (int b = 0; b < h.B; ++b) h.bidx[fb[h.bat_bus[b]]++] = b;
    for (int l = 0; l < h.L; ++l) {
        h.eidx[fe[h.line_from[l]]++] = 2 * l;
        h.eidx[fe[h.line_to[l]]++] = 2 * l + 1;
    }
    // An HVDC line runs through the line kernels as a line of unit beta whose phase weight
    // is 0 (no angle coupling: it drops out of every bus's phase average and of the phase
    // residual) and whose angle limit never binds; the kernels read w_l = 0 as "transport
    // line" and add its eps/2 f^2 term.
    int n_ac = 0;
    double mb2 = 0;
    for (int l = 0; l < h.L; ++l) {
        if (h.line_dc[l]) {
            h.line_beta[l] = 1.0;
            h.line_dth[l] = 3.0e38;
        } else {
            mb2 += h.line_beta[l] * h.line_beta[l];
            ++n_ac;
        }
    }
    mb2 = n_ac ? mb2 / n_ac : 1.0;
    h.l_w.resize(h.L);
    for (int l = 0; l < h.L; ++l)
        h.l_w[l] = h.line_dc[l] ? 0.f : (float)(o.theta_weight ? h.line_beta[l] * h.line_beta[l] : mb2);
    h.inv_cnt.resize(N); h.inv_wsum.resize(N); h.dres_w.resize(N);
    for (int n = 0; n < N; ++n) {
        const int cnt = 1 + (h.gptr[n + 1] - h.gptr[n]) + (h.bptr[n + 1] - h.bptr[n]) + (h.eptr[n + 1] - h.eptr[n]);
        h.inv_cnt[n] = 1.0f / cnt;
        double ws = 0, dw = 0;
        for (int q = h.eptr[n]; q < h.eptr[n + 1]; ++q) {
            const int l = h.eidx[q] >> 1;
            ws += h.l_w[l];
            dw += (h.l_w[l] / h.line_beta[l]) * (h.l_w[l] / h.line_beta[l]);
        }
        h.inv_wsum[n] = ws > 0 ? (float)(1.0 / ws) : 0.f;
        h.dres_w[n] = (float)dw;
    }
}

// Cluster-resident groups.  A scenario takes the smallest cluster (1, 2, 4, 8 or 16 CTAs)
// whose per-CTA shared-memory image fits kCrsSmemBudget; scenarios that fit none run on
// the per-iteration kernels.  Scenarios with the same cluster size and battery lane
// width form one launch, sized for the largest image among them.
constexpr size_t kCrsSmemBudget = 200 * 1024;

static int crs_hpl_bucket(int T) {
    const int h = (T + 31) / 32;
    return h <= 1 ? 1 : h <= 2 ? 2 : h <= 3 ? 3 : h <= 6 ? 6 : 8;
}

static void build_crs_groups(gx_network* net) {
    net->crs_groups.clear();
    net->crs_list.clear();
    net->crs_group.assign(net->S, -1);
    std::map<std::pair<int, int>, std::vector<int>> by;
    std::map<std::pair<int, int>, size_t> smem;
    for (int s = 0; s < net->S; ++s) {
        const ScenDev& sd = net->sdev[s];
        if (sd.R > 0) continue;  // ramping generators: per-iteration kernels only
        for (int C = 1; C <= kCrsMaxC; C *= 2) {
            const int H = (sd.T + C - 1) / C, nbo = (sd.B + C - 1) / C;
            const size_t bytes = crs_offsets(sd.N, sd.G, sd.L, sd.B, H, nbo, sd.T).total;
            if (bytes <= kCrsSmemBudget) {
                const auto key = std::make_pair(C, crs_hpl_bucket(sd.T));
                by[key].push_back(s);
                smem[key] = std::max(smem[key], bytes);
                break;
            }
        }
    }
    for (auto& kv : by) {
        gx_network::CrsGroup g;
        g.C = kv.first.first;
        g.hpl = kv.first.second;
        g.first = (int)net->crs_list.size();
        g.n = (int)kv.second.size();
        g.smem = smem[kv.first];
        for (int s : kv.second) {
            net->crs_group[s] = (int)net->crs_groups.size();
            net->crs_list.push_back(s);
        }
        net->crs_groups.push_back(g);
    }
}

// Bus-kernel block records and the pool records of the bus ranges they cover.  Blocks of
// scenarios on the same network with the same bus range share one pool record.
// Per-block copy lists of the bulk-staged bus kernel at a fixed stride: block b's header
// (copies, forward bytes, adjoint bytes, 0) and copies at b * stride, where a block can read
// them before it knows its record's offset.  Blocks whose record is not kept in shared memory
// get an empty list and use the record path.  Built only while the lists stay small (they
// repeat each scenario's records); above the cap the kernel reads the lists from the records.
constexpr size_t kBusCplMaxBytes = 16u << 20;

static void build_bus_copy_lists(gx_network* net) {
    net->bus_cpl.clear();
    net->bus_cpl_stride = 0;
    net->bus_cpl_max = 0;
    // a block takes the list path if its record fits shared memory and its list fits the
    // threads' copy slots (unstaged records: an empty list, only the record is copied)
    auto listed = [&](const BusBlk& r) {
        if (r.words > kPoolMax) return false;
        const int* p = net->pool.data() + r.pool;
        return p[kPH_SBYTES] == 0 || p[kPH_NCP] <= kCplPerThread * kBusQBlock;
    };
    int maxcp = 0, nlisted = 0;
    for (const BusBlk& r : net->bus4_blk) {
        if (!listed(r)) continue;
        const int* p = net->pool.data() + r.pool;
        ++nlisted;
        if (p[kPH_SBYTES] > 0) maxcp = std::max(maxcp, p[kPH_NCP]);
    }
    const int stride = (4 + 3 * maxcp + 3) / 4 * 4;
    if (nlisted == 0 || (size_t)stride * 4 * net->bus4_blk.size() > kBusCplMaxBytes) return;
    net->bus_cpl.assign((size_t)stride * net->bus4_blk.size(), 0);
    for (size_t b = 0; b < net->bus4_blk.size(); ++b) {
        const BusBlk& r = net->bus4_blk[b];
        int* q = net->bus_cpl.data() + b * stride;
        if (!listed(r)) {
            q[3] = 1;
            continue;
        }
        const int* p = net->pool.data() + r.pool;
        const int ncp = p[kPH_SBYTES] > 0 ? p[kPH_NCP] : 0;
        q[0] = ncp;
        q[1] = p[kPH_SBYTES] > 0 ? p[kPH_TXF] : 0;
        q[2] = p[kPH_SBYTES] > 0 ? p[kPH_TXA] : 0;
        std::memcpy(q + 4, p + p[kPH_CP], sizeof(int) * 3 * (size_t)ncp);
    }
    net->bus_cpl_stride = stride;
    net->bus_cpl_max = maxcp;
}

static void build_bus_blocks(gx_network* net) {
    auto fbits = [](float f) { int w; std::memcpy(&w, &f, 4); return w; };
    // (quad, net, n0, n1, first quad of bus n0, end quad of bus n1, quads per row) -> (offset, words)
    std::map<std::tuple<int, int, int, int, int, int, int>, std::pair<int, int>> rec_of;
    net->bus4_smem = 0;
    net->bus_blk.clear();
    net->bus4_blk.clear();
    net->pool.clear();
    net->prep.clear();
    net->sc_pool.clear();
    net->sc_dres_pool.clear();
    for (int quad = 0; quad < 2; ++quad)
    for (int s = 0; s < net->S; ++s) {
        const ScenDev& sd = net->sdev[s];
        const NetH& h = net->nets[sd.net];
        const int per_bus = quad ? sd.Tp / 4 : sd.Tp;  // items per bus row
        const long long nitems = (long long)sd.N * per_bus;
        const int nblk = quad ? sd.bus4_nblk : sd.bus_nblk;
        for (int b = 0; b < nblk; ++b) {
            BusBlk r{};
            r.e_bus = sd.e_bus; r.e_gen = sd.e_gen; r.e_line = sd.e_line; r.e_bat = sd.e_bat;
            r.s = s;
            const int bs = quad ? kBusQBlock : kBlock;  // items per block
            r.item0 = b * bs;
            const int last = (int)std::min<long long>((long long)r.item0 + bs, nitems) - 1;
            r.n0 = r.item0 / per_bus;
            const int n1 = last / per_bus;
            r.Tp = sd.Tp; r.T = sd.T; r.nitems = (int)nitems;
            const int qf = quad ? r.item0 - r.n0 * per_bus : 0;          // first quad of bus n0
            const int ql = quad ? last + 1 - n1 * per_bus : 0;           // end quad of bus n1
            const auto key = std::make_tuple(quad, sd.net, r.n0, n1, qf, ql, quad ? per_bus : 0);
            auto it = rec_of.find(key);
            if (it == rec_of.end()) {
                const int nbus = n1 - r.n0 + 1;
                const int gb = h.gptr[r.n0], gcnt = h.gptr[n1 + 1] - gb;
                const int eb = h.eptr[r.n0], ecnt = h.eptr[n1 + 1] - eb;
                const int bb = h.bptr[r.n0], bcnt = h.bptr[n1 + 1] - bb;
                // row staging of the quad kernel: each bus's hour range in this block, and
                // one copy per device row segment (generators twice: x and aux; line ends
                // twice: delta and the end's phase copy)
                const int ncopy = quad ? 2 * gcnt + 2 * ecnt + bcnt : 0;
                int o[kPoolHdr] = {};
                int w = kPoolHdr;
                o[kPH_GP] = w; w += nbus + 1;
                o[kPH_EP] = w; w += nbus + 1;
                o[kPH_BP] = w; w += nbus + 1;
                o[kPH_IC] = w; w += nbus;
                o[kPH_IW] = w; w += nbus;
                o[kPH_DR] = w; w += nbus;
                o[kPH_GROW] = w; w += gcnt;
                o[kPH_GCOST] = w; w += gcnt;
                o[kPH_GEMIS] = w; w += gcnt;
                o[kPH_GFIRM] = w; w += gcnt;
                o[kPH_GETA] = w; w += gcnt;
                o[kPH_ECODE] = w; w += ecnt;
                o[kPH_EBETA] = w; w += ecnt;
                o[kPH_EW] = w; w += ecnt;
                o[kPH_BROW] = w; w += bcnt;
                o[kPH_SQ] = w; w += nbus;
                o[kPH_SI] = w; w += nbus;
                o[kPH_SG] = w; w += nbus;
                o[kPH_SE] = w; w += nbus;
                o[kPH_SB] = w; w += nbus;
                o[kPH_CP] = w; w += 3 * ncopy;
                const int words = (w + 3) / 4 * 4;
                o[kPH_NBUS] = nbus; o[kPH_GCNT] = gcnt; o[kPH_ECNT] = ecnt; o[kPH_BCNT] = bcnt;
                const int off = (int)net->pool.size();
                net->pool.resize(net->pool.size() + words, 0);
                int* p = net->pool.data() + off;
                std::memcpy(p, o, sizeof(o));
                for (int k = 0; k <= nbus; ++k) {
                    p[o[kPH_GP] + k] = h.gptr[r.n0 + k] - gb;
                    p[o[kPH_EP] + k] = h.eptr[r.n0 + k] - eb;
                    p[o[kPH_BP] + k] = h.bptr[r.n0 + k] - bb;
                }
                for (int k = 0; k < nbus; ++k) {
                    p[o[kPH_IC] + k] = fbits(h.inv_cnt[r.n0 + k]);
                    p[o[kPH_IW] + k] = fbits(h.inv_wsum[r.n0 + k]);
                    p[o[kPH_DR] + k] = fbits(h.dres_w[r.n0 + k]);
                    if (h.bus_sdres[r.n0 + k] >= 0) {
                        ScaleDres rec = net->sc_dres[h.bus_sdres[r.n0 + k]];
                        rec.target = off + o[kPH_DR] + k;
                        net->sc_dres_pool.push_back(rec);
                    }
                }
                for (int k = 0; k < gcnt; ++k) {
                    const int g = h.gidx[gb + k];
                    p[o[kPH_GROW] + k] = g;
                    p[o[kPH_GCOST] + k] = fbits((float)h.gen_cost[g]);
                    p[o[kPH_GEMIS] + k] = fbits((float)h.gen_emis[g]);
                    // bit 0: capacity factor 1 throughout; bit 1: ramp-limited (its prox runs
                    // in the ramp kernel, the bus kernels only sum its injection)
                    p[o[kPH_GFIRM] + k] = net->firm[h.gen0 + g] | (h.g_ramp[g] >= 0 ? 2 : 0);
                    net->prep.push_back(int2{off + o[kPH_GETA] + k, h.eta0 + g});
                }
                for (int k = 0; k < ecnt; ++k) {
                    const int e = h.eidx[eb + k];
                    p[o[kPH_ECODE] + k] = e;
                    p[o[kPH_EBETA] + k] = fbits((float)h.line_beta[e >> 1]);
                    if (h.l_scale[e >> 1] >= 0) net->sc_pool.push_back(int2{off + o[kPH_EBETA] + k, h.l_scale[e >> 1]});
                    p[o[kPH_EW] + k] = fbits(h.l_w[e >> 1]);
                }
                for (int k = 0; k < bcnt; ++k) p[o[kPH_BROW] + k] = h.bidx[bb + k];
                if (quad) {
                    int qg = 0, qe = 0, qb = 0;
                    for (int k = 0; k < nbus; ++k) {
                        const int n = r.n0 + k;
                        const int s_it = std::max(n * per_bus, r.item0), e_it = std::min((n + 1) * per_bus, last + 1);
                        p[o[kPH_SQ] + k] = e_it - s_it;
                        p[o[kPH_SI] + k] = s_it - r.item0;
                        p[o[kPH_SG] + k] = qg;
                        p[o[kPH_SE] + k] = qe;
                        p[o[kPH_SB] + k] = qb;
                        qg += (h.gptr[n + 1] - h.gptr[n]) * (e_it - s_it);
                        qe += (h.eptr[n + 1] - h.eptr[n]) * (e_it - s_it);
                        qb += (h.bptr[n + 1] - h.bptr[n]) * (e_it - s_it);
                    }
                    const long long sbytes = 16LL * (2 * qg + 2 * qe + qb);
                    int* cp = p + o[kPH_CP];
                    int nc = 0;
                    long long txf = 0, txa = 0;  // bytes copied in the forward / adjoint iteration
                    auto add = [&](long long src, int dst, int nq, int flags, int arr) {
                        cp[3 * nc] = (int)src;
                        cp[3 * nc + 1] = dst;
                        cp[3 * nc + 2] = (nq << 5) | (flags << 3) | arr;
                        ++nc;
                        // a generator's aux row: capacity factor (forward, not for firm units),
                        // adjoint coefficient (adjoint); none for ramp-limited units
                        const bool aux = arr == kCpGenAux;
                        if (!aux || !(flags & (kCpRamp | kCpFirm))) txf += 16LL * nq;
                        if (!aux || !(flags & kCpRamp)) txa += 16LL * nq;
                    };
                    for (int k = 0; k < nbus; ++k) {
                        const int n = r.n0 + k, nq = p[o[kPH_SQ] + k];
                        const int q0 = (r.item0 + p[o[kPH_SI] + k]) - n * per_bus;  // first quad in the row
                        for (int j = h.gptr[n] - gb; j < h.gptr[n + 1] - gb; ++j) {
                            const int g = h.gidx[gb + j], rr = j - (h.gptr[n] - gb);
                            const long long src = (long long)g * sd.Tp + 4LL * q0;
                            const int dst = p[o[kPH_SG] + k] + rr * nq;
                            const int fl = (net->firm[h.gen0 + g] ? kCpFirm : 0) | (h.g_ramp[g] >= 0 ? kCpRamp : 0);
                            add(src, dst, nq, fl, kCpGenX);
                            add(src, qg + dst, nq, fl, kCpGenAux);
                        }
                        for (int j = h.eptr[n] - eb; j < h.eptr[n + 1] - eb; ++j) {
                            const int e = h.eidx[eb + j], rr = j - (h.eptr[n] - eb);
                            const long long src = (long long)(e >> 1) * sd.Tp + 4LL * q0;
                            const int dst = p[o[kPH_SE] + k] + rr * nq;
                            add(src, 2 * qg + dst, nq, 0, kCpDl);
                            add(src, 2 * qg + qe + dst, nq, 0, (e & 1) ? kCpVt : kCpVf);
                        }
                        for (int j = h.bptr[n] - bb; j < h.bptr[n + 1] - bb; ++j) {
                            const int b = h.bidx[bb + j], rr = j - (h.bptr[n] - bb);
                            const long long src = (long long)b * sd.Tp + 4LL * q0;
                            add(src, 2 * qg + 2 * qe + p[o[kPH_SB] + k] + rr * nq, nq, 0, kCpBat);
                        }
                    }
                    const bool staged = sbytes <= kStageMax && words <= kPoolMax;
                    p[kPH_NCP] = staged ? nc : 0;
                    p[kPH_QG] = qg;
                    p[kPH_QE] = qe;
                    p[kPH_QB] = qb;
                    p[kPH_SBYTES] = staged ? (int)sbytes : 0;
                    p[kPH_TXF] = (int)txf;
                    p[kPH_TXA] = (int)txa;
                    // the launch's dynamic shared memory holds the largest record kept in
                    // shared memory, with its stage if it has one
                    if (words <= kPoolMax)
                        net->bus4_smem = std::max<size_t>(net->bus4_smem,
                                                          4 * (size_t)words + (staged ? (size_t)sbytes : 0));
                }
                it = rec_of.emplace(key, std::make_pair(off, words)).first;
            }
            r.pool = it->second.first;
            r.words = it->second.second;
            (quad ? net->bus4_blk : net->bus_blk).push_back(r);
        }
    }
}

gx_status gx_network_create(const gx_network_desc* nets, int n_nets, const gx_scenario_desc* scen, int S,
                            const gx_opts* opts, gx_network** out) {
    if (!out) return fail(GX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!nets || n_nets < 1) return fail(GX_ERR_INVALID_ARG, "need at least one network");
    if (!scen || S < 1) return fail(GX_ERR_INVALID_ARG, "need at least one scenario");
    gx_opts o;
    if (opts) o = *opts; else gx_opts_default(&o);
    if (gx_status st = check_opts(&o)) return st;
    gx_network* net = new gx_network();
    net->opts = o;
    net->n_nets = n_nets;
    net->S = S;
    net->nets.resize(n_nets);
    int K = 0, gen0 = 0, line0 = 0, bat0 = 0, bus0 = 0, ptr0 = 0;
    for (int k = 0; k < n_nets; ++k) {
        const gx_network_desc& d = nets[k];
        NetH& h = net->nets[k];
        auto bad = [&](const std::string& m) {
            delete net;
            return fail(GX_ERR_INVALID_ARG, "network " + std::to_string(k) + ": " + m);
        };
        if (d.n_bus < 1 || d.n_gen < 0 || d.n_line < 0 || d.n_bat < 0) return bad("negative or zero sizes");
        if ((d.n_gen && (!d.gen_bus || !d.gen_cost || !d.gen_emis)) ||
            (d.n_line && (!d.line_from || !d.line_to || !d.line_beta || !d.line_dtheta)) ||
            (d.n_bat && (!d.bat_bus || !d.bat_dur || !d.bat_eff_c || !d.bat_eff_d)))
            return bad("NULL device array");
        h.N = d.n_bus; h.G = d.n_gen; h.L = d.n_line; h.B = d.n_bat;
        h.gen_bus.assign(d.gen_bus, d.gen_bus + h.G);
        h.gen_cost.assign(d.gen_cost, d.gen_cost + h.G);
        h.gen_emis.assign(d.gen_emis, d.gen_emis + h.G);
        h.line_from.assign(d.line_from, d.line_from + h.L);
        h.line_to.assign(d.line_to, d.line_to + h.L);
        h.line_beta.assign(d.line_beta, d.line_beta + h.L);
        h.line_dth.assign(d.line_dtheta, d.line_dtheta + h.L);
        h.line_dc.assign(h.L, 0);
        if (d.line_dc)
            for (int l = 0; l < h.L; ++l) h.line_dc[l] = d.line_dc[l] != 0;
        h.line_bref.assign(h.L, 0.0);
        if (d.line_beta_ref)
            for (int l = 0; l < h.L; ++l) {
                if (!(d.line_beta_ref[l] >= 0 && isfin(d.line_beta_ref[l])))
                    return bad("line_beta_ref must be finite and >= 0");
                if (!h.line_dc[l]) h.line_bref[l] = d.line_beta_ref[l];  // HVDC: no susceptance
            }
        h.gen_ramp.assign(h.G, 0.0);
        if (d.gen_ramp)
            for (int g = 0; g < h.G; ++g) {
                if (!(d.gen_ramp[g] >= 0 && isfin(d.gen_ramp[g]))) return bad("gen_ramp must be finite and >= 0");
                h.gen_ramp[g] = d.gen_ramp[g];
            }
        h.g_ramp.assign(h.G, -1);
        for (int g = 0; g < h.G; ++g)
            if (h.gen_ramp[g] > 0 && h.gen_ramp[g] < 1) {
                h.g_ramp[g] = (int)h.ramp_gens.size();
                h.ramp_gens.push_back(g);
            }
        h.bat_bus.assign(d.bat_bus, d.bat_bus + h.B);
        h.bat_dur.assign(d.bat_dur, d.bat_dur + h.B);
        h.bat_effc.assign(d.bat_eff_c, d.bat_eff_c + h.B);
        h.bat_effd.assign(d.bat_eff_d, d.bat_eff_d + h.B);
        for (int g = 0; g < h.G; ++g) {
            if (h.gen_bus[g] < 0 || h.gen_bus[g] >= h.N) return bad("gen_bus out of range");
            if (!isfin(h.gen_cost[g]) || !isfin(h.gen_emis[g])) return bad("non-finite generator data");
            net->cost_scale = std::max(net->cost_scale, std::fabs(h.gen_cost[g]));
        }
        for (int l = 0; l < h.L; ++l) {
            if (h.line_from[l] < 0 || h.line_from[l] >= h.N || h.line_to[l] < 0 || h.line_to[l] >= h.N)
                return bad("line bus out of range");
            if (h.line_from[l] == h.line_to[l]) return bad("line with both ends on one bus");
            if (h.line_dc[l]) continue;  // beta and dtheta unused
            if (!(h.line_beta[l] > 0 && isfin(h.line_beta[l]))) return bad("line_beta must be > 0");
            if (!(h.line_dth[l] > 0 && isfin(h.line_dth[l]))) return bad("line_dtheta must be > 0");
        }
        for (int b = 0; b < h.B; ++b) {
            if (h.bat_bus[b] < 0 || h.bat_bus[b] >= h.N) return bad("bat_bus out of range");
            if (!(h.bat_dur[b] > 0 && isfin(h.bat_dur[b]))) return bad("bat_dur must be > 0");
            if (!(h.bat_effc[b] > 0 && h.bat_effc[b] <= 1) || !(h.bat_effd[b] > 0 && h.bat_effd[b] <= 1))
                return bad("battery efficiency must be in (0, 1]");
        }
        derive_network(h, o);
        h.gen0 = gen0; h.line0 = line0; h.bat0 = bat0; h.bus0 = bus0; h.ptr0 = ptr0; h.eta0 = K;
        h.ramp0 = net->tot_ramp;
        // scaling susceptances: beta = (beta0 / ref) eta, and the dual-residual weights of
        // the buses they touch, split into the fixed lines' part and the scaling ends
        h.l_scale.assign(h.L, -1);
        for (int l = 0; l < h.L; ++l)
            if (h.line_bref[l] > 0) {
                h.l_scale[l] = (int)net->sc_line.size();
                net->sc_line.push_back(h.line0 + l);
                net->sc_eta.push_back(h.eta0 + h.G + l);
                net->sc_b.push_back(h.line_beta[l] / h.line_bref[l]);
                net->sc_bmin.push_back(1e-6 * h.line_beta[l]);
            }
        h.bus_sdres.assign(h.N, -1);
        for (int n = 0; n < h.N; ++n) {
            ScaleDres rec{};
            rec.first = (int)net->sc_dres_l.size();
            for (int q = h.eptr[n]; q < h.eptr[n + 1]; ++q) {
                const int l = h.eidx[q] >> 1;
                if (h.l_scale[l] >= 0) {
                    int wb;
                    std::memcpy(&wb, &h.l_w[l], 4);
                    net->sc_dres_l.push_back(int2{h.l_scale[l], wb});
                    ++rec.count;
                } else {
                    const double q2 = h.l_w[l] / h.line_beta[l];
                    rec.d0 += q2 * q2;
                }
            }
            if (rec.count) {
                rec.target = -1 - (h.bus0 + n);
                h.bus_sdres[n] = (int)net->sc_dres.size();
                net->sc_dres.push_back(rec);
            }
        }
        gen0 += h.G; line0 += h.L; bat0 += h.B; bus0 += h.N; ptr0 += h.N + 1; K += h.G + h.L + h.B;
        net->tot_ramp += (int)h.ramp_gens.size();
    }
    net->K = K;
    net->tot_gen = gen0; net->tot_line = line0; net->tot_bat = bat0; net->tot_bus = bus0; net->tot_ptr = ptr0;
    net->scens.resize(S);
    net->sdev.resize(S);
    long long eb = 0, eg = 0, el = 0, ebt = 0;
    int gs = 0;
    for (int s = 0; s < S; ++s) {
        const gx_scenario_desc& d = scen[s];
        auto bad = [&](const std::string& m) {
            delete net;
            return fail(GX_ERR_INVALID_ARG, "scenario " + std::to_string(s) + ": " + m);
        };
        if (d.net < 0 || d.net >= n_nets) return bad("net index out of range");
        if (d.T < 1 || d.T > kMaxT) return bad("T must be in [1, 256]");
        if (!(d.weight > 0 && isfin(d.weight))) return bad("weight must be > 0");
        const NetH& h = net->nets[d.net];
        if (!d.load || (h.G && !d.cf)) return bad("NULL load or cf");
        ScenH& sh = net->scens[s];
        sh.net = d.net; sh.T = d.T; sh.Tp = (d.T + 3) / 4 * 4; sh.weight = d.weight;
        sh.load.assign((size_t)h.N * sh.Tp, 0.f);
        sh.cf.assign((size_t)h.G * sh.Tp, 0.f);
        double ln2 = 0;
        for (int n = 0; n < h.N; ++n)
            for (int t = 0; t < d.T; ++t) {
                const double v = d.load[(size_t)n * d.T + t];
                if (!(v >= 0 && isfin(v))) return bad("load must be finite and >= 0");
                sh.load[(size_t)n * sh.Tp + t] = (float)v;
                ln2 += v * v;
            }
        for (int g = 0; g < h.G; ++g)
            for (int t = 0; t < d.T; ++t) {
                const double v = d.cf[(size_t)g * d.T + t];
                if (!(v >= 0 && v <= 1)) return bad("cf must be in [0, 1]");
                sh.cf[(size_t)g * sh.Tp + t] = (float)v;
            }
        ScenDev& sd = net->sdev[s];
        std::memset(&sd, 0, sizeof(sd));
        sd.net = d.net; sd.T = d.T; sd.Tp = sh.Tp; sd.N = h.N; sd.G = h.G; sd.L = h.L; sd.B = h.B;
        sd.gen0 = h.gen0; sd.line0 = h.line0; sd.bat0 = h.bat0; sd.bus0 = h.bus0; sd.ptr0 = h.ptr0; sd.eta0 = h.eta0;
        sd.gs0 = gs;
        gs += h.G + h.L + h.B;
        sd.e_bus = eb; sd.e_gen = eg; sd.e_line = el; sd.e_bat = ebt;
        eb += (long long)h.N * sh.Tp; eg += (long long)h.G * sh.Tp; el += (long long)h.L * sh.Tp;
        ebt += (long long)h.B * sh.Tp;
        sd.R = (int)h.ramp_gens.size();
        sd.ramp0 = h.ramp0;
        sd.e_ramp = net->ramp_el;
        net->ramp_el += (long long)sd.R * sh.Tp;
        sd.ramp_w0 = net->n_ramp_warps;
        for (int r = 0; r < sd.R; ++r) net->ramp_warp_scen.push_back(s);
        net->n_ramp_warps += sd.R;
        if (sd.R > 0) net->max_ramp_T = std::max(net->max_ramp_T, sh.T);
        sd.weight = (float)d.weight;
        sd.load_norm = std::max(std::sqrt(ln2), 1e-30);
        // block tables
        sd.bus_blk0 = net->n_bus_blk;
        sd.bus_nblk = (int)(((long long)h.N * sh.Tp + kBlock - 1) / kBlock);
        for (int b = 0; b < sd.bus_nblk; ++b) net->bus_blk_scen.push_back(s);
        net->n_bus_blk += sd.bus_nblk;
        sd.line_blk0 = net->n_line_blk;
        sd.line_nblk = (int)(((long long)h.L * sh.Tp + kBlock * kLineItems - 1) / (kBlock * kLineItems));
        for (int b = 0; b < sd.line_nblk; ++b) net->line_blk_scen.push_back(s);
        net->n_line_blk += sd.line_nblk;
        sd.bus4_blk0 = net->n_bus4_blk;
        sd.bus4_nblk = (int)(((long long)h.N * (sh.Tp / 4) + kBusQBlock - 1) / kBusQBlock);
        net->n_bus4_blk += sd.bus4_nblk;
        sd.line4_blk0 = net->n_line4_blk;
        sd.line4_nblk = (int)(((long long)h.L * (sh.Tp / 4) + kQBlock - 1) / kQBlock);
        for (int b = 0; b < sd.line4_nblk; ++b) net->line4_blk_scen.push_back(s);
        net->n_line4_blk += sd.line4_nblk;
        sd.bat_w0 = net->n_bat_warps;
        for (int b = 0; b < h.B; ++b) net->bat_warp_scen.push_back(s);
        net->n_bat_warps += h.B;
        sd.cost_blk0 = net->n_cost_blk;
        const long long work = (long long)(h.G + h.N + h.B) * sh.Tp;
        const int ncb = (int)std::min<long long>(64, std::max<long long>(1, work / (kBlock * 16)));
        for (int b = 0; b < ncb; ++b) net->cost_blk_scen.push_back(s);
        net->n_cost_blk += ncb;
        for (int r = 0; r < h.G + h.L + h.B; ++r) { net->gwarp.push_back(s); net->gwarp.push_back(r); }
        net->n_gwarps += h.G + h.L + h.B;
        for (int l = 0; l < h.L; ++l)
            if (h.l_scale[l] >= 0) { net->sc_gwarp.push_back(s); net->sc_gwarp.push_back(h.l_scale[l]); }
    }
    net->gs_total = gs;
    net->bus_el = eb; net->gen_el = eg; net->line_el = el; net->bat_el = ebt;
    // generators whose capacity factor is 1 in every hour of every scenario skip the cf read
    net->firm.assign(std::max(net->tot_gen, 1), 1);
    for (int s = 0; s < S; ++s) {
        const ScenH& sc = net->scens[s];
        const NetH& n = net->nets[sc.net];
        for (int g = 0; g < n.G; ++g)
            for (int t = 0; t < sc.T; ++t)
                if (sc.cf[(size_t)g * sc.Tp + t] != 1.0f) { net->firm[n.gen0 + g] = 0; break; }
    }
    build_bus_blocks(net);
    build_bus_copy_lists(net);
    net->line4_blk.clear();
    net->bat_w.clear();
    for (int s = 0; s < S; ++s) {
        const ScenDev& sd = net->sdev[s];
        const NetH& h = net->nets[sd.net];
        for (int b = 0; b < sd.line4_nblk; ++b) {
            LineBlk r{};
            r.e_line = sd.e_line; r.e_bus = sd.e_bus;
            r.s = s; r.line0 = sd.line0; r.Tp = sd.Tp; r.T = sd.T;
            r.L = sd.L; r.eta_l = sd.eta0 + sd.G; r.item0 = b * kQBlock;
            const int tq = sd.Tp / 4;
            r.l0 = r.item0 / tq;
            const int l1 = std::min(sd.L - 1, (r.item0 + kQBlock - 1) / tq);
            if (l1 - r.l0 + 1 <= kLineBlkLines) {
                r.nends = l1 - r.l0 + 1;
                for (int j = 0; j < r.nends; ++j) {
                    r.ends[2 * j] = h.line_from[r.l0 + j];
                    r.ends[2 * j + 1] = h.line_to[r.l0 + j];
                }
            }
            net->line4_blk.push_back(r);
        }
        for (int b = 0; b < sd.B; ++b) {
            BatW r{};
            r.row0 = sd.e_bat + (long long)b * sd.Tp;
            r.brow0 = sd.e_bus + (long long)h.bat_bus[b] * sd.Tp;
            r.s = s; r.bg = sd.bat0 + b; r.T = sd.T; r.Tp = sd.Tp;
            r.eta_b = sd.eta0 + sd.G + sd.L + b;
            net->bat_w.push_back(r);
        }
    }
    net->sc_dres.insert(net->sc_dres.end(), net->sc_dres_pool.begin(), net->sc_dres_pool.end());
    build_crs_groups(net);
    net->k_net.resize(K);
    for (int k = 0; k < n_nets; ++k)
        for (int q = 0; q < net->nets[k].G + net->nets[k].L + net->nets[k].B; ++q) net->k_net[net->nets[k].eta0 + q] = k;

    // ---- layout
    Layout& L = net->lay;
    auto I4 = [](long long n) { return (size_t)std::max<long long>(n, 1) * 4; };
    auto F4 = I4;
    auto D8 = [](long long n) { return (size_t)std::max<long long>(n, 1) * 8; };
    auto B1 = [](long long n) { return (size_t)std::max<long long>(n, 1); };
    net->o_scen = L.add(sizeof(ScenDev) * S);
    net->o_bbs = L.add(I4(net->n_bus_blk));
    net->o_lbs = L.add(I4(net->n_line_blk));
    net->o_bws = L.add(I4(net->n_bat_warps));
    net->o_cbs = L.add(I4(net->n_cost_blk));
    net->o_gwarp = L.add(I4(2LL * net->n_gwarps));
    net->o_knet = L.add(I4(K));
    net->o_busblk = L.add(sizeof(BusBlk) * std::max<size_t>(net->bus_blk.size(), 1));
    net->o_pool = L.add(I4((long long)net->pool.size()));
    net->o_prep = L.add(8 * std::max<size_t>(net->prep.size(), 1));
    net->o_crs = L.add(I4((long long)net->crs_list.size()));
    net->o_bus4blk = L.add(sizeof(BusBlk) * std::max<size_t>(net->bus4_blk.size(), 1));
    net->o_buscpl = L.add(I4(std::max<long long>((long long)net->bus_cpl.size(), 1)));
    net->o_busdone = L.add(I4(std::max<long long>((long long)net->bus4_blk.size(), 1)));
    net->o_l4bs = L.add(I4(net->n_line4_blk));
    net->o_l4blk = L.add(sizeof(LineBlk) * std::max<size_t>(net->line4_blk.size(), 1));
    net->o_batw = L.add(sizeof(BatW) * std::max<size_t>(net->bat_w.size(), 1));
    net->o_gbus = L.add(I4(gen0)); net->o_gcost = L.add(F4(gen0)); net->o_gemis = L.add(F4(gen0));
    net->o_gfirm = L.add(B1(gen0));
    net->o_lfrom = L.add(I4(line0)); net->o_lto = L.add(I4(line0)); net->o_lbeta = L.add(F4(line0));
    net->o_ldth = L.add(F4(line0)); net->o_lw = L.add(F4(line0));
    net->o_bbus = L.add(I4(bat0)); net->o_bdur = L.add(F4(bat0)); net->o_beffc = L.add(F4(bat0));
    net->o_beffd = L.add(F4(bat0));
    net->o_gptr = L.add(I4(ptr0)); net->o_gidx = L.add(I4(gen0));
    net->o_bptr = L.add(I4(ptr0)); net->o_bidx = L.add(I4(bat0));
    net->o_eptr = L.add(I4(ptr0)); net->o_eidx = L.add(I4(2LL * line0));
    net->o_icnt = L.add(F4(bus0)); net->o_iwsum = L.add(F4(bus0)); net->o_dresw = L.add(F4(bus0));
    net->o_load = L.add(F4(eb)); net->o_cf = L.add(F4(eg)); net->o_dd = L.add(F4(ebt));
    net->o_add = L.add(F4(ebt));
    net->o_rgen = L.add(I4(net->tot_ramp));
    net->o_rrate = L.add(F4(net->tot_ramp));
    net->o_gramp = L.add(I4(gen0));
    net->o_rws = L.add(I4(net->n_ramp_warps));
    net->o_rdd = L.add(F4(net->ramp_el));
    net->o_ardd = L.add(F4(net->ramp_el));
    net->o_scl = L.add(I4((long long)net->sc_line.size()));
    net->o_sce = L.add(I4((long long)net->sc_eta.size()));
    net->o_scb = L.add(D8((long long)net->sc_b.size()));
    net->o_scbm = L.add(D8((long long)net->sc_bmin.size()));
    net->o_scp = L.add(8 * std::max<size_t>(net->sc_pool.size(), 1));
    net->o_scd = L.add(sizeof(ScaleDres) * std::max<size_t>(net->sc_dres.size(), 1));
    net->o_scdl = L.add(8 * std::max<size_t>(net->sc_dres_l.size(), 1));
    net->o_scgw = L.add(I4((long long)net->sc_gwarp.size()));
    net->static_end = L.total;
    const long long rows[16] = {eg, eb, el, el, el, el, ebt, ebt, ebt, ebt, ebt, ebt, ebt, eb, eb, eb};
    // forward state, then adjoint state, each one contiguous range (gx_network_state_range)
    for (int k = 0; k < 16; ++k) net->o_f[k] = L.add(F4(rows[k]));
    for (int k = 0; k < 4; ++k) net->o_rf[k] = L.add(F4(net->ramp_el));
    net->o_fend = L.total;
    for (int k = 0; k < 16; ++k) net->o_a[k] = L.add(F4(rows[k]));
    for (int k = 0; k < 4; ++k) net->o_ra[k] = L.add(F4(net->ramp_el));
    net->o_aend = L.total;
    net->o_mgen = L.add(B1(eg)); net->o_mload = L.add(B1(eb)); net->o_mline = L.add(B1(el)); net->o_mbat = L.add(B1(ebt));
    net->o_ag = L.add(F4(eg));
    net->o_al = L.add(F4(eb));
    net->o_done = L.add(I4(S)); net->o_iters = L.add(I4(S)); net->o_status = L.add(I4(S)); net->o_adjit = L.add(I4(S));
    net->o_nact = L.add(I4(1)); net->o_ctr = L.add(I4(1)); net->o_inb = L.add(I4(S)); net->o_err = L.add(I4(1));
    net->o_wsel = L.add(I4(S));
    net->o_resid = L.add(D8(2LL * S)); net->o_rbest = L.add(D8(S)); net->o_cost = L.add(D8(S)); net->o_h = L.add(D8(S));
    net->o_grads = L.add(D8(gs)); net->o_wprime = L.add(D8(S)); net->o_obj = L.add(D8(1));
    net->o_stlo = L.add(D8(3LL * kStampSlots)); net->o_sthi = L.add(D8(3LL * kStampSlots)); net->o_pact = L.add(D8(S));
    net->o_flow = L.add(F4(el)); net->o_price = L.add(F4(eb)); net->o_shed = L.add(F4(eb));
    net->o_bpart = L.add(F4((long long)net->n_bus4_blk * kBusPart));
    net->o_lpart = L.add(F4((long long)net->n_line4_blk * kDevPart));
    net->o_btpart = L.add(F4((long long)net->n_bat_warps * kDevPart));
    net->o_rpart = L.add(F4((long long)net->n_ramp_warps * kDevPart));
    net->o_cpart = L.add(D8(2LL * net->n_cost_blk));
    net->in_batch.assign(S, 0);
    net->done_init.assign(S, 1);
    net->wprime.assign(S, 0.0);
    fill_dd(net);
    *out = net;
    return GX_OK;
}

gx_status gx_network_destroy(gx_network* net) {
    delete net;
    return GX_OK;
}

size_t gx_network_device_bytes(const gx_network* net) { return net ? net->lay.total : 0; }
int gx_network_K(const gx_network* net) { return net ? net->K : 0; }
int gx_network_S(const gx_network* net) { return net ? net->S : 0; }

gx_status gx_network_bind(gx_network* net, void* dev_mem, size_t bytes, void* stream) {
    if (!net) return fail(GX_ERR_INVALID_ARG, "net is NULL");
    if (!dev_mem) return fail(GX_ERR_INVALID_ARG, "dev_mem is NULL");
    if (reinterpret_cast<uintptr_t>(dev_mem) % 256) return fail(GX_ERR_INVALID_ARG, "dev_mem must be 256-byte aligned");
    if (bytes < net->lay.total) return fail(GX_ERR_NO_MEMORY, "workspace smaller than gx_network_device_bytes()");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    net->dev = reinterpret_cast<uint8_t*>(dev_mem);
    // Stage the static region on the host and upload it in one copy.
    std::vector<uint8_t> h(net->static_end, 0);
    auto put = [&](size_t off, const void* src, size_t n) { if (n) std::memcpy(h.data() + off, src, n); };
    put(net->o_scen, net->sdev.data(), sizeof(ScenDev) * net->S);
    put(net->o_bbs, net->bus_blk_scen.data(), 4 * net->bus_blk_scen.size());
    put(net->o_lbs, net->line_blk_scen.data(), 4 * net->line_blk_scen.size());
    put(net->o_bws, net->bat_warp_scen.data(), 4 * net->bat_warp_scen.size());
    put(net->o_cbs, net->cost_blk_scen.data(), 4 * net->cost_blk_scen.size());
    put(net->o_gwarp, net->gwarp.data(), 4 * net->gwarp.size());
    put(net->o_knet, net->k_net.data(), 4 * net->k_net.size());
    put(net->o_busblk, net->bus_blk.data(), sizeof(BusBlk) * net->bus_blk.size());
    put(net->o_pool, net->pool.data(), 4 * net->pool.size());
    put(net->o_prep, net->prep.data(), 8 * net->prep.size());
    put(net->o_crs, net->crs_list.data(), 4 * net->crs_list.size());
    put(net->o_bus4blk, net->bus4_blk.data(), sizeof(BusBlk) * net->bus4_blk.size());
    put(net->o_buscpl, net->bus_cpl.data(), 4 * net->bus_cpl.size());
    put(net->o_l4bs, net->line4_blk_scen.data(), 4 * net->line4_blk_scen.size());
    put(net->o_l4blk, net->line4_blk.data(), sizeof(LineBlk) * net->line4_blk.size());
    put(net->o_batw, net->bat_w.data(), sizeof(BatW) * net->bat_w.size());
    put(net->o_scl, net->sc_line.data(), 4 * net->sc_line.size());
    put(net->o_sce, net->sc_eta.data(), 4 * net->sc_eta.size());
    put(net->o_scb, net->sc_b.data(), 8 * net->sc_b.size());
    put(net->o_scbm, net->sc_bmin.data(), 8 * net->sc_bmin.size());
    put(net->o_scp, net->sc_pool.data(), 8 * net->sc_pool.size());
    put(net->o_scd, net->sc_dres.data(), sizeof(ScaleDres) * net->sc_dres.size());
    put(net->o_scdl, net->sc_dres_l.data(), 8 * net->sc_dres_l.size());
    put(net->o_scgw, net->sc_gwarp.data(), 4 * net->sc_gwarp.size());
    auto put_f = [&](size_t off, const std::vector<double>& v, size_t base) {
        float* p = reinterpret_cast<float*>(h.data() + off) + base;
        for (size_t i = 0; i < v.size(); ++i) p[i] = (float)v[i];
    };
    auto put_i = [&](size_t off, const std::vector<int>& v, size_t base) {
        if (!v.empty()) std::memcpy(reinterpret_cast<int*>(h.data() + off) + base, v.data(), 4 * v.size());
    };
    auto put_v = [&](size_t off, const std::vector<float>& v, size_t base) {
        if (!v.empty()) std::memcpy(reinterpret_cast<float*>(h.data() + off) + base, v.data(), 4 * v.size());
    };
    for (const NetH& n : net->nets) {
        put_i(net->o_gbus, n.gen_bus, n.gen0); put_f(net->o_gcost, n.gen_cost, n.gen0); put_f(net->o_gemis, n.gen_emis, n.gen0);
        put_i(net->o_lfrom, n.line_from, n.line0); put_i(net->o_lto, n.line_to, n.line0);
        put_f(net->o_lbeta, n.line_beta, n.line0); put_f(net->o_ldth, n.line_dth, n.line0); put_v(net->o_lw, n.l_w, n.line0);
        put_i(net->o_bbus, n.bat_bus, n.bat0); put_f(net->o_bdur, n.bat_dur, n.bat0);
        put_f(net->o_beffc, n.bat_effc, n.bat0); put_f(net->o_beffd, n.bat_effd, n.bat0);
        put_i(net->o_gptr, n.gptr, n.ptr0); put_i(net->o_gidx, n.gidx, n.gen0);
        put_i(net->o_bptr, n.bptr, n.ptr0); put_i(net->o_bidx, n.bidx, n.bat0);
        put_i(net->o_eptr, n.eptr, n.ptr0); put_i(net->o_eidx, n.eidx, 2 * (size_t)n.line0);
        put_v(net->o_icnt, n.inv_cnt, n.bus0); put_v(net->o_iwsum, n.inv_wsum, n.bus0); put_v(net->o_dresw, n.dres_w, n.bus0);
    }
    for (int s = 0; s < net->S; ++s) {
        const ScenH& sc = net->scens[s];
        put_v(net->o_load, sc.load, net->sdev[s].e_bus);
        put_v(net->o_cf, sc.cf, net->sdev[s].e_gen);
    }
    put(net->o_gfirm, net->firm.data(), net->tot_gen);
    put_v(net->o_dd, net->dd_host, 0);
    put_v(net->o_add, net->add_host, 0);
    put_v(net->o_rdd, net->rdd_host, 0);
    put_v(net->o_ardd, net->ardd_host, 0);
    {
        std::vector<int> rgen, gramp(std::max(net->tot_gen, 1), -1);
        std::vector<float> rrate;
        for (const NetH& n : net->nets) {
            for (int r = 0; r < (int)n.ramp_gens.size(); ++r) {
                rgen.push_back(n.ramp_gens[r]);
                rrate.push_back((float)n.gen_ramp[n.ramp_gens[r]]);
            }
            for (int g = 0; g < n.G; ++g) gramp[n.gen0 + g] = n.g_ramp[g];
        }
        put(net->o_rgen, rgen.data(), 4 * rgen.size());
        put(net->o_rrate, rrate.data(), 4 * rrate.size());
        put(net->o_gramp, gramp.data(), 4 * (size_t)net->tot_gen);
        put(net->o_rws, net->ramp_warp_scen.data(), 4 * net->ramp_warp_scen.size());
    }
    GX_CUDA(cudaMemcpyAsync(net->dev, h.data(), net->static_end, cudaMemcpyHostToDevice, st));
    GX_CUDA(cudaMemsetAsync(net->dev + net->static_end, 0, net->lay.total - net->static_end, st));
    GX_CUDA(cudaStreamSynchronize(st));
    net->dd_dirty = false;
    if (!net->h_nact) GX_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&net->h_nact), 2 * sizeof(int), cudaHostAllocDefault));
    if (!net->cap_stream) GX_CUDA(cudaStreamCreateWithFlags(&net->cap_stream, cudaStreamNonBlocking));
    if (!net->cap_stream2) GX_CUDA(cudaStreamCreateWithFlags(&net->cap_stream2, cudaStreamNonBlocking));
    if (!net->ev_fork) GX_CUDA(cudaEventCreateWithFlags(&net->ev_fork, cudaEventDisableTiming));
    if (!net->ev_join) GX_CUDA(cudaEventCreateWithFlags(&net->ev_join, cudaEventDisableTiming));
    if (net->bus4_smem > 0) GX_CUDA(bus_staged_prepare((int)net->bus4_smem));
    {
        int dev = 0, l2 = 0;
        GX_CUDA(cudaGetDevice(&dev));
        GX_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
        // An L2-resident workspace is latency-bound: there the staged kernel reads its copy
        // lists from per-block slots (one dependent hop fewer, more registers); a workspace
        // that streams from HBM keeps the record path and its occupancy.
        net->l2_resident = net->lay.total <= (size_t)l2;
        // default bus kernel until a schedule is set: stage the device rows when the iteration
        // streams from HBM; the autotuner picks per workload
        if (!net->sched_set) net->sched.bus_staged = net->l2_resident ? 0 : 1;
    }
    make_ctx(net);
    for (auto& g : net->crs_groups) {
        g.ok = true;
        for (int adj = 0; adj < 2 && g.ok; ++adj)
            g.ok = crs_prepare(adj, g.hpl, kCrsSmemBudget) == cudaSuccess &&
                   crs_max_clusters(adj, g.hpl, g.C, g.smem) >= 1;
        cudaGetLastError();
    }
    net->solved = false;
    net->adj_ready = false;
    return GX_OK;
}

gx_status gx_network_forget(gx_network* net) {
    if (!net || !net->dev) return fail(GX_ERR_STATE, "network is not bound");
    net->solved = false;
    net->adj_ready = false;
    return GX_OK;
}

gx_status gx_network_set_opts(gx_network* net, const gx_opts* opts) {
    if (!net || !opts) return fail(GX_ERR_INVALID_ARG, "NULL argument");
    if (gx_status st = check_opts(opts)) return st;
    if (opts->theta_weight != net->opts.theta_weight)
        return fail(GX_ERR_INVALID_ARG, "theta_weight is fixed at create");
    net->opts = *opts;
    fill_dd(net);
    if (net->dev) make_ctx(net);
    return GX_OK;
}

gx_status gx_network_state_range(const gx_network* net, int which, size_t* offset, size_t* bytes) {
    if (!net || !offset || !bytes) return fail(GX_ERR_INVALID_ARG, "NULL argument");
    if (which != 0 && which != 1) return fail(GX_ERR_INVALID_ARG, "which must be 0 (forward) or 1 (adjoint)");
    *offset = which ? net->o_a[0] : net->o_f[0];
    *bytes = (which ? net->o_aend : net->o_fend) - *offset;
    return GX_OK;
}

gx_status gx_network_array(const gx_network* net, int which, int scen, size_t* offset, size_t* count) {
    if (!net || !offset || !count) return fail(GX_ERR_INVALID_ARG, "NULL argument");
    if (scen < -1 || scen >= net->S) return fail(GX_ERR_INVALID_ARG, "scenario out of range");
    size_t base = 0, esz = 4;
    long long e0 = 0, n = 0;
    const ScenDev* sd = scen >= 0 ? &net->sdev[scen] : nullptr;
    auto rows = [&](long long el_all, long long e_s, long long per) {
        if (sd) { e0 = e_s; n = per; } else { e0 = 0; n = el_all; }
    };
    switch (which) {
        case GX_ARR_P: base = net->o_f[0]; rows(net->gen_el, sd ? sd->e_gen : 0, sd ? (long long)sd->G * sd->Tp : 0); break;
        case GX_ARR_SHED: base = net->o_shed; rows(net->bus_el, sd ? sd->e_bus : 0, sd ? (long long)sd->N * sd->Tp : 0); break;
        case GX_ARR_FLOW: base = net->o_flow; rows(net->line_el, sd ? sd->e_line : 0, sd ? (long long)sd->L * sd->Tp : 0); break;
        case GX_ARR_THETA: base = net->o_f[15]; rows(net->bus_el, sd ? sd->e_bus : 0, sd ? (long long)sd->N * sd->Tp : 0); break;
        case GX_ARR_CH: base = net->o_f[7]; rows(net->bat_el, sd ? sd->e_bat : 0, sd ? (long long)sd->B * sd->Tp : 0); break;
        case GX_ARR_DIS: base = net->o_f[8]; rows(net->bat_el, sd ? sd->e_bat : 0, sd ? (long long)sd->B * sd->Tp : 0); break;
        case GX_ARR_SOC: base = net->o_f[9]; rows(net->bat_el, sd ? sd->e_bat : 0, sd ? (long long)sd->B * sd->Tp : 0); break;
        case GX_ARR_PRICE: base = net->o_price; rows(net->bus_el, sd ? sd->e_bus : 0, sd ? (long long)sd->N * sd->Tp : 0); break;
        case GX_ARR_COST: base = net->o_cost; esz = 8; rows(net->S, scen, 1); break;
        case GX_ARR_H: base = net->o_h; esz = 8; rows(net->S, scen, 1); break;
        case GX_ARR_ITERS: base = net->o_iters; rows(net->S, scen, 1); break;
        case GX_ARR_RESID: base = net->o_resid; esz = 8; rows(2LL * net->S, 2LL * scen, 2); break;
        case GX_ARR_STATUS: base = net->o_status; rows(net->S, scen, 1); break;
        case GX_ARR_GRAD_S: base = net->o_grads; esz = 8;
            rows(net->gs_total, sd ? sd->gs0 : 0, sd ? (long long)(sd->G + sd->L + sd->B) : 0); break;
        case GX_ARR_ADJ_ITERS: base = net->o_adjit; rows(net->S, scen, 1); break;
        case GX_ARR_WARM: base = net->o_wsel; rows(net->S, scen, 1); break;
        case GX_ARR_OBJ:
            if (scen != -1) return fail(GX_ERR_INVALID_ARG, "GX_ARR_OBJ is one value for the batch (scen = -1)");
            base = net->o_obj; esz = 8; e0 = 0; n = 1; break;
        default: return fail(GX_ERR_INVALID_ARG, "unknown array id");
    }
    *offset = base + (size_t)e0 * esz;
    *count = (size_t)n;
    return GX_OK;
}

gx_status gx_network_scenario_info(const gx_network* net, int s, int* T, int* Tp, int* N, int* G, int* L, int* B,
                                   int* eta_offset) {
    if (!net || s < 0 || s >= net->S) return fail(GX_ERR_INVALID_ARG, "bad scenario");
    const ScenDev& d = net->sdev[s];
    if (T) *T = d.T;
    if (Tp) *Tp = d.Tp;
    if (N) *N = d.N;
    if (G) *G = d.G;
    if (L) *L = d.L;
    if (B) *B = d.B;
    if (eta_offset) *eta_offset = d.eta0;
    return GX_OK;
}

// Part of one residual-check chunk: iterations [j0, j1) of `chunk` (residual partials, and
// the kernels' time stamps while timing is on, on the chunk's last iteration), optionally
// preceded by the counter tick and followed by the per-scenario reduction and the copy of
// the active count to the host.
static gx_status enqueue_iters(gx_network* net, const Ctx& c, int adj, int chunk, int j0, int j1, bool tick,
                               bool reduce, cudaStream_t st, int* launches, bool to_host = true) {
    const int mode = adj ? M_ADJ : M_FWD;
    const double tol = adj ? net->opts.adj_tol : net->opts.tol;
    if (tick) *launches += launch_tick(c, chunk, st);
    // While capturing, the line and battery proxes are two branches of the graph: they
    // are independent and both feed the bus kernel.
    const bool fork = (st == net->cap_stream) && (c.n_bat_warps > 0 || c.n_ramp_warps > 0) && c.n_line_blk > 0;
    for (int j = j0; j < j1; ++j) {
        const int want = j == chunk - 1;
        int nl = 0, nb = 0;
        if (fork) {
            GX_CUDA(cudaEventRecord(net->ev_fork, st));
            GX_CUDA(cudaStreamWaitEvent(net->cap_stream2, net->ev_fork, 0));
            nb = launch_bat(c, mode, adj, want, net->cap_stream2);
            nb += launch_ramp(c, mode, adj, want, net->cap_stream2);
            GX_CUDA(cudaEventRecord(net->ev_join, net->cap_stream2));
            nl = launch_line(c, mode, adj, want, st);
            GX_CUDA(cudaStreamWaitEvent(st, net->ev_join, 0));
        } else {
            nl = launch_line(c, mode, adj, want, st);
            nb = launch_bat(c, mode, adj, want, st);
            nb += launch_ramp(c, mode, adj, want, st);
        }
        const int nu = launch_bus(c, mode, adj, want, st);
        *launches += nl + nb + nu;
    }
    if (reduce) {
        GX_CUDA(cudaMemsetAsync(c.n_active, 0, sizeof(int), st));
        *launches += launch_reduce(c, adj, tol, st);
        if (to_host) GX_CUDA(cudaMemcpyAsync(net->h_nact, c.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    return GX_OK;
}

// The instantiated graph of a chunk (tick, iterations, reduction and the copy of the active
// count), captured on the library's own stream (capture is not allowed on the legacy
// default stream).  Cached by everything its parameters depend on.
static gx_status chunk_graph(gx_network* net, const Ctx& c, int adj, int chunk, cudaGraphExec_t* out) {
    for (auto& g : net->graphs)
        if (g.valid && !g.loop && g.adj == adj && g.chunk == chunk && g.eta == c.eta) {
            *out = g.exec;
            return GX_OK;
        }
    auto& g = net->graphs[net->graph_next];
    net->graph_next = (net->graph_next + 1) % 4;
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = gx_network::ChunkGraph{};
    cudaGraph_t graph = nullptr;
    int dummy = 0;
    GX_CUDA(cudaStreamBeginCapture(net->cap_stream, cudaStreamCaptureModeThreadLocal));
    gx_status e = enqueue_iters(net, c, adj, chunk, 0, chunk, true, true, net->cap_stream, &dummy);
    cudaError_t ce = cudaStreamEndCapture(net->cap_stream, &graph);
    if (e) return e;
    if (ce != cudaSuccess) return fail(GX_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(GX_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
    g.valid = true;
    g.adj = adj; g.chunk = chunk; g.eta = c.eta;
    *out = g.exec;
    return GX_OK;
}

// The whole iteration loop as one graph: a conditional WHILE node whose body is one
// residual-check chunk (tick, check_every iterations, reduction) followed by k_loop_cond,
// which sets the node's condition on the device.  The host launches it once per solve and
// synchronises once, instead of once per chunk.
static gx_status loop_graph(gx_network* net, const Ctx& c, int adj, int every, int max_it, cudaGraphExec_t* out) {
    for (auto& g : net->graphs)
        if (g.valid && g.loop && g.adj == adj && g.chunk == every && g.eta == c.eta) {
            *out = g.exec;
            return GX_OK;
        }
    auto& g = net->graphs[net->graph_next];
    net->graph_next = (net->graph_next + 1) % 4;
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = gx_network::ChunkGraph{};
    cudaGraph_t graph = nullptr;
    GX_CUDA(cudaGraphCreate(&graph, 0));
    auto bail = [&](cudaError_t ce, const char* what) {
        cudaGraphDestroy(graph);
        return fail(GX_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(ce));
    };
    cudaGraphConditionalHandle h;
    cudaError_t ce = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (ce != cudaSuccess) return bail(ce, "cudaGraphConditionalHandleCreate");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p);
    if (ce != cudaSuccess) return bail(ce, "cudaGraphAddNode");
    cudaGraph_t body = p.conditional.phGraph_out[0];
    ce = cudaStreamBeginCaptureToGraph(net->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return bail(ce, "cudaStreamBeginCaptureToGraph");
    int dummy = 0;
    gx_status e = enqueue_iters(net, c, adj, every, 0, every, true, true, net->cap_stream, &dummy, false);
    if (!e) launch_loop_cond(c, max_it, h, net->cap_stream);
    cudaGraph_t captured = nullptr;
    ce = cudaStreamEndCapture(net->cap_stream, &captured);
    if (e) { cudaGraphDestroy(graph); return e; }
    if (ce != cudaSuccess) return bail(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(GX_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
    g.valid = true;
    g.loop = 1;
    g.adj = adj; g.chunk = every; g.eta = c.eta;
    *out = g.exec;
    return GX_OK;
}

static bool crs_on(const gx_network* net, int s) {
    const int g = net->crs_group[s];
    return net->use_crs && g >= 0 && net->crs_groups[g].ok;
}

// Run the batch's cluster-resident scenarios (one persistent launch per group) and set
// up the done flags of the per-iteration loop so that it skips them.  *n_stream: the
// batch's scenarios left for that loop.
static gx_status run_crs(gx_network* net, int adj, cudaStream_t st, int* launches, int* n_stream) {
    const Ctx& c = adj ? net->actx : net->ctx;
    const double tol = adj ? net->opts.adj_tol : net->opts.tol;
    std::vector<int> want(net->crs_groups.size(), 0);
    int ns = 0, nc = 0;
    for (int s = 0; s < net->S; ++s) {
        if (!net->in_batch[s]) continue;
        if (crs_on(net, s)) { want[net->crs_group[s]] = 1; ++nc; }
        else ++ns;
    }
    *n_stream = ns;
    if (nc == 0) return GX_OK;
    const int* inb = reinterpret_cast<const int*>(net->dev + net->o_inb);
    const int* list = reinterpret_cast<const int*>(net->dev + net->o_crs);
    if (net->prof) GX_CUDA(cudaEventRecord(net->ev[0], st));
    int nl = 0;
    for (size_t k = 0; k < net->crs_groups.size(); ++k) {
        const auto& g = net->crs_groups[k];
        if (!want[k]) continue;
        nl += launch_crs(c, adj, list + g.first, g.n, inb, g.C, g.hpl, g.smem, tol, st);
    }
    GX_CUDA(cudaGetLastError());
    *launches += nl;
    if (net->prof) {
        GX_CUDA(cudaEventRecord(net->ev[1], st));
        GX_CUDA(cudaEventSynchronize(net->ev[1]));
        float ms = 0;
        GX_CUDA(cudaEventElapsedTime(&ms, net->ev[0], net->ev[1]));
        net->prof_ms[3] += ms;
        net->prof_samples[3] += nl;
        net->prof_launches[3] += nl;
    }
    if (ns > 0) {
        net->done_loop.assign(net->S, 1);
        for (int s = 0; s < net->S; ++s) net->done_loop[s] = (net->in_batch[s] && !crs_on(net, s)) ? 0 : 1;
        GX_CUDA(cudaMemcpyAsync(net->dev + net->o_done, net->done_loop.data(), 4 * net->S, cudaMemcpyHostToDevice, st));
    }
    return GX_OK;
}

// Iterate the forward (adj = 0) or adjoint (adj = 1) message passing until every
// scenario of the batch meets its tolerance or the cap is reached.  Graph mode 2 (the
// default, when the cap is a multiple of check_every and kernels are not being timed)
// replays the whole loop as one graph whose conditional node tests convergence on the
// device.  Otherwise each chunk of check_every iterations is one graph (mode 1) or eager
// launches (mode 0), and the stream is synchronised once per chunk to read the number of
// scenarios still iterating.  While kernels are being timed, a chunk's last iteration
// and its reduction run as eager launches bracketed by events (event times cannot be read
// from graph-recorded events).
static gx_status read_stamps(gx_network* net, int nchunks, cudaStream_t st);

static gx_status run_loop(gx_network* net, int adj, cudaStream_t st, int* launches, int* iters_out, int it0 = 0) {
    const Ctx& c = adj ? net->actx : net->ctx;
    const int max_it = adj ? net->opts.adj_max_iter : net->opts.max_iter;
    const int every = net->opts.check_every;
    const int per_it = (c.n_line_blk > 0) + (c.n_bat_warps > 0) + (c.n_ramp_warps > 0) + (c.n_bus_blk > 0);
    int it = it0;  // iterations already run (the learned start's trial chunk)
    GX_CUDA(cudaMemsetAsync(c.iter_ctr, 0, sizeof(int), st));
    if (it0 > 0) *launches += launch_tick(c, it0, st);
    if (net->use_graphs == 2 && max_it % every == 0) {
        cudaGraphExec_t exec = nullptr;
        if (gx_status e = loop_graph(net, c, adj, every, max_it, &exec)) return e;
        GX_CUDA(cudaGraphLaunch(exec, st));
        GX_CUDA(cudaMemcpyAsync(net->h_nact + 1, c.iter_ctr, sizeof(int), cudaMemcpyDeviceToHost, st));
        GX_CUDA(cudaGetLastError());
        GX_CUDA(cudaStreamSynchronize(st));
        it = net->h_nact[1];
        // per body: tick, the iterations, the reduction and the condition kernel
        *launches += ((it - it0) / every) * (3 + every * per_it);
        *iters_out = it;
        if (net->prof) {
            net->prof_launches[0] += (long long)it * (c.n_bus_blk > 0);
            net->prof_launches[1] += (long long)it * (c.n_line_blk > 0);
            net->prof_launches[2] += (long long)it * (c.n_bat_warps > 0 || c.n_ramp_warps > 0);
            return read_stamps(net, it / every, st);
        }
        return GX_OK;
    }
    int nch = 0;
    while (it < max_it) {
        const int chunk = std::min(every, max_it - it);
        int nk = 0;
        if (net->use_graphs && chunk == every) {
            cudaGraphExec_t exec = nullptr;
            if (gx_status e = chunk_graph(net, c, adj, chunk, &exec)) return e;
            GX_CUDA(cudaGraphLaunch(exec, st));
            nk = 2 + chunk * per_it;
        } else {
            if (gx_status e = enqueue_iters(net, c, adj, chunk, 0, chunk, true, true, st, &nk)) return e;
        }
        *launches += nk;
        it += chunk;
        ++nch;
        GX_CUDA(cudaGetLastError());
        GX_CUDA(cudaStreamSynchronize(st));
        if (*net->h_nact == 0) break;
    }
    *iters_out = it;
    if (net->prof) {
        net->prof_launches[0] += (long long)it * (c.n_bus_blk > 0);
        net->prof_launches[1] += (long long)it * (c.n_line_blk > 0);
        net->prof_launches[2] += (long long)it * (c.n_bat_warps > 0 || c.n_ramp_warps > 0);
        return read_stamps(net, nch, st);
    }
    return GX_OK;
}

// Sampled kernel timing: every residual-check chunk's last iteration writes, per kernel
// kind, the earliest block start and the latest block end (%globaltimer, ns) to the chunk's
// slot; the duration of that launch is their difference.  Accumulate the loop's chunks and
// reset their slots for the next loop.
static gx_status read_stamps(gx_network* net, int nchunks, cudaStream_t st) {
    const int n = std::min(nchunks, kStampSlots);
    if (n <= 0) return GX_OK;
    std::vector<unsigned long long> lo(3 * n), hi(3 * n);
    const Ctx& c = net->ctx;
    GX_CUDA(cudaMemcpyAsync(lo.data(), c.stamp_lo, 8 * lo.size(), cudaMemcpyDeviceToHost, st));
    GX_CUDA(cudaMemcpyAsync(hi.data(), c.stamp_hi, 8 * hi.size(), cudaMemcpyDeviceToHost, st));
    GX_CUDA(cudaMemsetAsync(c.stamp_lo, 0xff, 8 * lo.size(), st));
    GX_CUDA(cudaMemsetAsync(c.stamp_hi, 0, 8 * hi.size(), st));
    GX_CUDA(cudaStreamSynchronize(st));
    // kinds in the slots: 0 bus, 1 line, 2 battery and ramp (the order of prof_ms)
    for (int k = 0; k < n; ++k)
        for (int q = 0; q < 3; ++q) {
            const unsigned long long a = lo[3 * k + q], b = hi[3 * k + q];
            if (b == 0 || a == ~0ULL || b < a) continue;  // the kind did not run in that chunk
            net->prof_ms[q] += (double)(b - a) * 1e-6;
            net->prof_samples[q] += 1;
        }
    return GX_OK;
}

// Battery and ramp pivot tables after gx_network_set_opts changed a penalty: both the
// solve and the gradient entry points upload them before their first iteration.
static gx_status upload_pivots(gx_network* net, cudaStream_t st) {
    if (!net->dd_dirty) return GX_OK;
    GX_CUDA(cudaMemcpyAsync(net->dev + net->o_dd, net->dd_host.data(), 4 * net->dd_host.size(),
                            cudaMemcpyHostToDevice, st));
    GX_CUDA(cudaMemcpyAsync(net->dev + net->o_add, net->add_host.data(), 4 * net->add_host.size(),
                            cudaMemcpyHostToDevice, st));
    GX_CUDA(cudaMemcpyAsync(net->dev + net->o_rdd, net->rdd_host.data(), 4 * net->rdd_host.size(),
                            cudaMemcpyHostToDevice, st));
    GX_CUDA(cudaMemcpyAsync(net->dev + net->o_ardd, net->ardd_host.data(), 4 * net->ardd_host.size(),
                            cudaMemcpyHostToDevice, st));
    GX_CUDA(cudaStreamSynchronize(st));
    net->dd_dirty = false;
    return GX_OK;
}

static gx_status upload_batch(gx_network* net, const int* scen_idx, int B, cudaStream_t st) {
    std::vector<int>& inb = net->in_batch;
    if (scen_idx) {
        if (B < 1 || B > net->S) return fail(GX_ERR_INVALID_ARG, "batch size out of range");
        std::fill(inb.begin(), inb.end(), 0);
        for (int i = 0; i < B; ++i) {
            if (scen_idx[i] < 0 || scen_idx[i] >= net->S) return fail(GX_ERR_INVALID_ARG, "scenario index out of range");
            inb[scen_idx[i]] = 1;
        }
    } else {
        std::fill(inb.begin(), inb.end(), 1);
    }
    for (int s = 0; s < net->S; ++s) net->done_init[s] = inb[s] ? 0 : 1;
    GX_CUDA(cudaMemcpyAsync(net->dev + net->o_inb, inb.data(), 4 * net->S, cudaMemcpyHostToDevice, st));
    GX_CUDA(cudaMemcpyAsync(net->dev + net->o_done, net->done_init.data(), 4 * net->S, cudaMemcpyHostToDevice, st));
    return GX_OK;
}

static gx_status collect_stats(gx_network* net, int adj, gx_stats* stats, int launches, cudaStream_t st,
                               gx_status* overall) {
    std::vector<int> its(net->S), sts(net->S);
    std::vector<double> res(2 * net->S);
    GX_CUDA(cudaMemcpyAsync(its.data(), net->dev + (adj ? net->o_adjit : net->o_iters), 4 * net->S,
                            cudaMemcpyDeviceToHost, st));
    GX_CUDA(cudaMemcpyAsync(sts.data(), net->dev + net->o_status, 4 * net->S, cudaMemcpyDeviceToHost, st));
    GX_CUDA(cudaMemcpyAsync(res.data(), net->dev + net->o_resid, 16 * net->S, cudaMemcpyDeviceToHost, st));
    int err = 0;
    GX_CUDA(cudaMemcpyAsync(&err, net->dev + net->o_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GX_CUDA(cudaStreamSynchronize(st));
    if (err) return fail(err, "a bounded device-side wait gave up (bulk copies of the bus kernel)");
    gx_stats sx{};
    sx.launches = launches;
    gx_status worst = GX_OK;
    for (int s = 0; s < net->S; ++s) {
        if (!net->in_batch[s]) continue;
        sx.n_scen++;
        sx.iters_max = std::max(sx.iters_max, its[s]);
        if (sts[s] == GX_OK) sx.n_converged++;
        sx.max_primal = std::max(sx.max_primal, res[2 * s]);
        sx.max_dual = std::max(sx.max_dual, res[2 * s + 1]);
        if (sts[s] < 0) worst = sts[s];
        else if (sts[s] > 0 && worst == GX_OK) worst = sts[s];
    }
    if (stats) *stats = sx;
    *overall = worst;
    return GX_OK;
}

// GX_WARM_LEARNED with a previous solution (the selection rule of the learned start): one
// residual-check chunk from the previous plan's state, whose state and flags are saved in
// the warm-start network's scratch; then, for the scenarios still iterating, one chunk from
// the learned start (the prediction `pred`, applied as a user start); each scenario keeps
// the start with the smaller residual at its check, the others get the saved state back.
// The main loop then continues from iteration check_every.
static gx_status learned_trials(gx_network* net, const float* pred, cudaStream_t st, int* launches) {
    Ctx& c = net->ctx;
    const int every = net->opts.check_every;
    size_t sv_bytes = 0;
    uint8_t* sv = gx_gnn_internal_scratch(net->gnn, &sv_bytes);
    const size_t state_bytes = net->o_fend - net->o_f[0];
    if (!sv || sv_bytes < state_bytes + 32 * (size_t)net->S)
        return fail(GX_ERR_STATE, "the attached warm-start network does not belong to this network");
    int* sdone = reinterpret_cast<int*>(sv + state_bytes);
    int* sstatus = sdone + net->S;
    int* siters = sstatus + net->S;
    double* sres = reinterpret_cast<double*>(siters + net->S + (net->S & 1));  // 8-byte aligned
    // trial 1: the previous plan's state
    GX_CUDA(cudaMemsetAsync(c.iter_ctr, 0, sizeof(int), st));
    if (gx_status e = enqueue_iters(net, c, 0, every, 0, every, true, true, st, launches, false)) return e;
    GX_CUDA(cudaMemcpyAsync(sv, net->dev + net->o_f[0], state_bytes, cudaMemcpyDeviceToDevice, st));
    GX_CUDA(cudaMemcpyAsync(sdone, c.done, 4 * (size_t)net->S, cudaMemcpyDeviceToDevice, st));
    GX_CUDA(cudaMemcpyAsync(sstatus, c.status, 4 * (size_t)net->S, cudaMemcpyDeviceToDevice, st));
    GX_CUDA(cudaMemcpyAsync(siters, c.iters, 4 * (size_t)net->S, cudaMemcpyDeviceToDevice, st));
    GX_CUDA(cudaMemcpyAsync(sres, c.resid, 16 * (size_t)net->S, cudaMemcpyDeviceToDevice, st));
    // trial 2: the learned start (the start kernels skip scenarios trial 1 finished)
    c.warm = pred;
    *launches += launch_dev(c, M_RESET, 0, 0, st);
    *launches += launch_bus(c, M_RESET, 0, 0, st);
    *launches += launch_bus(c, M_INIT, 0, 0, st);
    c.warm = nullptr;
    GX_CUDA(cudaMemsetAsync(c.iter_ctr, 0, sizeof(int), st));
    if (gx_status e = enqueue_iters(net, c, 0, every, 0, every, true, true, st, launches, false)) return e;
    // the choice, and the previous plan's rows back where it won
    WarmArrays w{};
    for (int k = 0; k < 16; ++k) {
        w.off[w.n] = (long long)((net->o_f[k] - net->o_f[0]) / 4);
        w.kind[w.n++] = k == 0 ? 0 : (k == 1 || k >= 13) ? 1 : (k <= 5) ? 2 : 3;
    }
    if (net->tot_ramp > 0)
        for (int k = 0; k < 4; ++k) {
            w.off[w.n] = (long long)((net->o_rf[k] - net->o_f[0]) / 4);
            w.kind[w.n++] = 4;
        }
    *launches += launch_warm_select(c, w, reinterpret_cast<float*>(net->dev + net->o_f[0]),
                                    reinterpret_cast<const float*>(sv),
                                    reinterpret_cast<const int*>(net->dev + net->o_inb), sdone, sstatus, siters, sres,
                                    reinterpret_cast<int*>(net->dev + net->o_wsel), st);
    return GX_OK;
}

gx_status gx_dispatch_solve_batch(gx_network* net, const float* eta_dev, const int* scen_idx, int B, int warm,
                                  const float* warm_dev, gx_stats* stats, void* stream) {
    if (!net) return fail(GX_ERR_INVALID_ARG, "net is NULL");
    if (!net->dev) return fail(GX_ERR_STATE, "network is not bound");
    if (!eta_dev) return fail(GX_ERR_INVALID_ARG, "eta_dev is NULL");
    if (warm < GX_WARM_COLD || warm > GX_WARM_LEARNED) return fail(GX_ERR_INVALID_ARG, "unsupported warm mode");
    if (warm == GX_WARM_USER && !warm_dev) return fail(GX_ERR_INVALID_ARG, "GX_WARM_USER needs warm_dev");
    if (warm == GX_WARM_LEARNED && !net->gnn)
        return fail(GX_ERR_STATE, "GX_WARM_LEARNED needs a warm-start network (gx_network_attach_gnn)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    GX_CUDA(cudaMemsetAsync(net->dev + net->o_err, 0, sizeof(int), st));
    if (gx_status e = upload_batch(net, scen_idx, B, st)) return e;
    if (gx_status e = upload_pivots(net, st)) return e;
    // Eq. 1 weights of the batch, rescaled to the total weight (an unbiased estimate of
    // the full sum for a sampled batch): used by the objective and by the next gradient
    double wall = 0, wb = 0;
    for (int s = 0; s < net->S; ++s) {
        wall += net->scens[s].weight;
        if (net->in_batch[s]) wb += net->scens[s].weight;
    }
    for (int s = 0; s < net->S; ++s) net->wprime[s] = net->in_batch[s] ? net->scens[s].weight * wall / wb : 0.0;
    GX_CUDA(cudaMemcpyAsync(net->dev + net->o_wprime, net->wprime.data(), 8 * net->S, cudaMemcpyHostToDevice, st));
    Ctx& c = net->ctx;
    c.eta = eta_dev;
    c.warm = warm == GX_WARM_USER ? warm_dev : nullptr;
    int launches = launch_prep(c, st);
    launches += launch_scale_prep(c, st);
    GX_CUDA(cudaMemsetAsync(net->dev + net->o_wsel, 0xff, 4 * (size_t)net->S, st));  // -1: no learned start
    const float* pred = nullptr;
    if (warm == GX_WARM_LEARNED) {
        if (gx_status e = gx_gnn_internal_predict(net->gnn, eta_dev, st, &pred)) return e;
        launches += 5;
    }
    int it0 = 0;
    if (warm == GX_WARM_LEARNED && net->solved) {
        if (gx_status e = learned_trials(net, pred, st, &launches)) return e;
        it0 = net->opts.check_every;
    } else if (warm != GX_WARM_PREV || !net->solved) {
        if (warm == GX_WARM_LEARNED) {
            // no previous plan to compare with: the learned start for every scenario
            c.warm = pred;
            std::vector<int> one(net->S);
            for (int s = 0; s < net->S; ++s) one[s] = net->in_batch[s] ? 1 : -1;
            GX_CUDA(cudaMemcpyAsync(net->dev + net->o_wsel, one.data(), 4 * (size_t)net->S, cudaMemcpyHostToDevice, st));
            GX_CUDA(cudaStreamSynchronize(st));  // `one` is pageable and local
        }
        launches += launch_dev(c, M_RESET, 0, 0, st);
        launches += launch_bus(c, M_RESET, 0, 0, st);
        launches += launch_bus(c, M_INIT, 0, 0, st);
    }
    c.warm = nullptr;
    int it = 0, ns = 0;
    if (gx_status e = run_crs(net, 0, st, &launches, &ns)) return e;
    if (ns > 0)
        if (gx_status e = run_loop(net, 0, st, &launches, &it, it0)) return e;
    launches += launch_extract(c, reinterpret_cast<const int*>(net->dev + net->o_inb), st);
    launches += launch_objective(c, reinterpret_cast<const double*>(net->dev + net->o_wprime),
                                 reinterpret_cast<double*>(net->dev + net->o_obj), st);
    GX_CUDA(cudaGetLastError());
    gx_status overall;
    if (gx_status e = collect_stats(net, 0, stats, launches, st, &overall)) return e;
    net->solved = true;
    return overall;
}

gx_status gx_dispatch_grad_batch(gx_network* net, const float* eta_dev, int warm, float* grad_dev, gx_stats* stats,
                                 void* stream) {
    if (!net) return fail(GX_ERR_INVALID_ARG, "net is NULL");
    if (!net->dev) return fail(GX_ERR_STATE, "network is not bound");
    if (!net->solved) return fail(GX_ERR_STATE, "gx_dispatch_grad_batch needs a solve first");
    if (!eta_dev || !grad_dev) return fail(GX_ERR_INVALID_ARG, "NULL device pointer");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    GX_CUDA(cudaMemsetAsync(net->dev + net->o_err, 0, sizeof(int), st));
    Ctx& c = net->ctx;
    c.eta = eta_dev;
    c.warm = nullptr;
    Ctx& ac = net->actx;
    ac.eta = eta_dev;
    ac.warm = nullptr;
    // the batch of the last solve and its weights w'_s (uploaded by that solve)
    GX_CUDA(cudaMemcpyAsync(net->dev + net->o_done, net->done_init.data(), 4 * net->S, cudaMemcpyHostToDevice, st));
    if (gx_status e = upload_pivots(net, st)) return e;
    int launches = launch_prep(c, st);
    launches += launch_scale_prep(c, st);
    launches += launch_dev(c, M_MASK, 0, 0, st);
    launches += launch_bus(c, M_MASK, 0, 0, st);
    const bool envelope = net->opts.grad_envelope && net->opts.kappa == 0.0;
    gx_status overall = GX_OK;
    gx_stats sx{};
    if (!envelope) {
        if (warm != GX_WARM_PREV || !net->adj_ready) {
            launches += launch_dev(ac, M_RESET, 1, 0, st);
            launches += launch_bus(ac, M_RESET, 1, 0, st);
        }
        launches += launch_bus(ac, M_INIT, 1, 0, st);
        int it = 0, ns = 0;
        if (gx_status e = run_crs(net, 1, st, &launches, &ns)) return e;
        if (ns > 0)
            if (gx_status e = run_loop(net, 1, st, &launches, &it)) return e;
        net->adj_ready = true;
    }
    const int* inb = reinterpret_cast<const int*>(net->dev + net->o_inb);
    launches += launch_grad(envelope ? c : ac, envelope ? 1 : 0,
                            reinterpret_cast<const int*>(net->dev + net->o_gwarp), net->n_gwarps, inb, st);
    launches += launch_scale_grad(envelope ? c : ac, envelope ? 1 : 0, inb, st);
    launches += launch_grad_combine(c, reinterpret_cast<const double*>(net->dev + net->o_wprime),
                                    reinterpret_cast<const int*>(net->dev + net->o_knet), grad_dev, net->K, st);
    GX_CUDA(cudaGetLastError());
    if (!envelope) {
        if (gx_status e = collect_stats(net, 1, &sx, launches, st, &overall)) return e;
    } else {
        GX_CUDA(cudaStreamSynchronize(st));
        sx.launches = launches;
    }
    if (stats) *stats = sx;
    return overall;
}

gx_status gx_plan_step(gx_network* net, float* eta_dev, const float* grad_dev, const float* gamma_dev,
                       const float* eta_min_dev, const float* eta_max_dev, float alpha, void* stream) {
    if (!net) return fail(GX_ERR_INVALID_ARG, "net is NULL");
    if (!eta_dev || !grad_dev || !gamma_dev || !eta_min_dev || !eta_max_dev)
        return fail(GX_ERR_INVALID_ARG, "NULL device pointer");
    if (!(alpha >= 0) || !std::isfinite(alpha)) return fail(GX_ERR_INVALID_ARG, "alpha must be finite and >= 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    launch_plan_step(eta_dev, grad_dev, gamma_dev, eta_min_dev, eta_max_dev, alpha, net->K, st);
    GX_CUDA(cudaGetLastError());
    return GX_OK;
}

gx_status gx_network_use_graphs(gx_network* net, int on) {
    if (!net) return fail(GX_ERR_INVALID_ARG, "net is NULL");
    if (on < 0 || on > 2) return fail(GX_ERR_INVALID_ARG, "graph mode must be 0, 1 or 2");
    net->use_graphs = on;
    return GX_OK;
}

gx_status gx_network_set_schedule(gx_network* net, const gx_schedule* sched) {
    if (!net || !sched) return fail(GX_ERR_INVALID_ARG, "NULL argument");
    if (sched->bus_staged < 0 || sched->bus_staged > 2) return fail(GX_ERR_INVALID_ARG, "bus_staged is 0, 1 or 2");
    if (sched->bat_warps != 1 && sched->bat_warps != 2) return fail(GX_ERR_INVALID_ARG, "bat_warps is 1 or 2");
    net->sched = *sched;
    net->sched_set = true;
    if (net->dev) make_ctx(net);  // drops the cached graphs, whose launches follow the schedule
    return GX_OK;
}

gx_status gx_network_get_schedule(const gx_network* net, gx_schedule* sched) {
    if (!net || !sched) return fail(GX_ERR_INVALID_ARG, "NULL argument");
    *sched = net->sched;
    return GX_OK;
}

gx_status gx_network_attach_gnn(gx_network* net, gx_gnn* gnn) {
    if (!net) return fail(GX_ERR_INVALID_ARG, "net is NULL");
    if (gnn && gx_gnn_internal_net(gnn) != net)
        return fail(GX_ERR_INVALID_ARG, "the warm-start network was created for another network");
    net->gnn = gnn;
    return GX_OK;
}

gx_status gx_network_use_persistent(gx_network* net, int on) {
    if (!net) return fail(GX_ERR_INVALID_ARG, "net is NULL");
    net->use_crs = on != 0;
    return GX_OK;
}

gx_status gx_network_persistent_info(const gx_network* net, int scen, int* cluster_ctas) {
    if (!net || !cluster_ctas) return fail(GX_ERR_INVALID_ARG, "NULL argument");
    if (scen < 0 || scen >= net->S) return fail(GX_ERR_INVALID_ARG, "scenario out of range");
    *cluster_ctas = crs_on(net, scen) ? net->crs_groups[net->crs_group[scen]].C : 0;
    return GX_OK;
}

gx_status gx_profile_enable(gx_network* net, int on) {
    if (!net) return fail(GX_ERR_INVALID_ARG, "net is NULL");
    if (on && !net->dev) return fail(GX_ERR_STATE, "network is not bound");
    if (on && !net->ev[0])
        for (auto& e : net->ev) GX_CUDA(cudaEventCreate(&e));
    const bool changed = net->prof != (on != 0);
    net->prof = on != 0;
    for (int k = 0; k < 4; ++k) { net->prof_ms[k] = 0; net->prof_samples[k] = 0; net->prof_launches[k] = 0; }
    if (net->dev) {
        // the stamp slots start empty and the active counts at zero; the kernels write them
        // only while the context carries their pointers
        GX_CUDA(cudaMemset(net->dev + net->o_stlo, 0xff, 8 * 3 * kStampSlots));
        GX_CUDA(cudaMemset(net->dev + net->o_sthi, 0, 8 * 3 * kStampSlots));
        GX_CUDA(cudaMemset(net->dev + net->o_pact, 0, 8 * (size_t)net->S));
        for (Ctx* c : {&net->ctx, &net->actx}) {
            c->stamp_lo = net->prof ? reinterpret_cast<unsigned long long*>(net->dev + net->o_stlo) : nullptr;
            c->stamp_hi = net->prof ? reinterpret_cast<unsigned long long*>(net->dev + net->o_sthi) : nullptr;
            c->prof_act = net->prof ? reinterpret_cast<long long*>(net->dev + net->o_pact) : nullptr;
        }
        if (changed) net->drop_graphs();  // the captured kernels carry the context by value
    }
    return GX_OK;
}

gx_status gx_profile_active(const gx_network* net, long long* counts) {
    if (!net || !counts) return fail(GX_ERR_INVALID_ARG, "NULL argument");
    if (!net->dev) return fail(GX_ERR_STATE, "network is not bound");
    GX_CUDA(cudaMemcpy(counts, net->dev + net->o_pact, 8 * (size_t)net->S, cudaMemcpyDeviceToHost));
    return GX_OK;
}

gx_status gx_profile_read(const gx_network* net, double* ms, long long* samples, long long* launches) {
    if (!net || !ms || !samples || !launches) return fail(GX_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < 4; ++k) { ms[k] = net->prof_ms[k]; samples[k] = net->prof_samples[k]; launches[k] = net->prof_launches[k]; }
    return GX_OK;
}

}  // extern "C"
