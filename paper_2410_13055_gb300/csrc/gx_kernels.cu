// sm_103a kernels of the batched proximal message-passing dispatch solver and its adjoint.
//
// One outer iteration (proximal message passing: ADMM with a proximal step per device
// and an averaging step per bus) is three launches:
//   k_line  one thread per (line, hour): phase-dual update and the closed-form line prox
//   k_bat   one warp per battery: a warm-started inner ADMM on the battery prox QP whose
//           equality-constrained step is a tridiagonal solve done with warp scans
//   k_bus   one thread per (bus, hour): generator and load proxes (fused), the bus
//           consensus (average injection and average angle), the scaled dual update and
//           the residual partial sums
// The same kernels run the adjoint (Section 2.2, implicit function theorem): there the
// clip of every prox becomes a fixed active-set mask and the linear costs come from
// grad h at the solved dispatch, so the iteration solves the linearised KKT system.
//
// Memory: every array is a row of Tp floats per device (hours contiguous), so each warp
// reads 32 consecutive hours of one row: coalesced 128-byte transactions.  Bus arrays
// (p_bar, u, theta_bar) are gathered by the device kernels through the same row layout.
#include "gx_internal.cuh"
#include "gx_async.cuh"

#include <cfloat>

namespace gx {

namespace {

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV values over a block of NT threads; thread 0 gets the totals in v[].
template <int NV, int NT = kBlock>
__device__ __forceinline__ void block_sum(float (&v)[NV], float (*sh)[NT / 32]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float s = warp_sum(v[k]);
        if (lane == 0) sh[k][w] = s;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            float s = lane < NT / 32 ? sh[k][lane] : 0.f;
            v[k] = warp_sum(s);
        }
    }
}

struct StatePtrs {
    float *xg, *xl, *dl, *sg, *vf, *vt, *xb, *zc, *zd, *zs, *yc, *yd, *ys, *u, *pbar, *thb;
};

template <int ADJ>
__device__ __forceinline__ StatePtrs state(const Ctx& c) {
    if (ADJ)
        return StatePtrs{c.a_xg, c.a_xl, c.a_dl, c.a_sg, c.a_vf, c.a_vt, c.a_xb, c.a_zc, c.a_zd, c.a_zs,
                         c.a_yc, c.a_yd, c.a_ys, c.a_u, c.a_pbar, c.a_thb};
    return StatePtrs{c.xg, c.xl, c.dl, c.sg, c.vf, c.vt, c.xb, c.zc, c.zd, c.zs,
                     c.yc, c.yd, c.ys, c.u, c.pbar, c.thb};
}

}  // namespace

// ------------------------------------------------------------------------------------
// Line prox.  With delta = th_f - th_t and sigma = th_f + th_t the prox of a lossless DC
// line separates: sigma = w_f + w_t, and delta minimises the 1-D quadratic
//   rho/2 [(-beta d - v_f)^2 + (beta d - v_t)^2] + rho_th/4 (d - (w_f - w_t))^2
// over |beta d| <= eta_l, |d| <= dtheta_max, i.e. the unconstrained minimiser clipped.
// ------------------------------------------------------------------------------------
// One line-hour of the line prox (all modes).  FWD/ADJ callers pass the loaded state
// so two items per thread can have all their loads in flight before any store.
struct LineIn {
    long long row, bf, bt;
    int lg, l;
    bool valid;
    float d, g, qf, qt, pbf, uf, zf, pbt, ut, zt, beta, w, capf, dth;
    uint8_t mask;
};

template <int MODE, int ADJ>
__device__ __forceinline__ void line_index(const Ctx& c, const ScenDev& sc, int local, LineIn& L) {
    L.l = local / sc.Tp;
    const int t = local - L.l * sc.Tp;
    L.valid = (L.l < sc.L) && (t < sc.T);
    if (!L.valid) return;
    L.row = sc.e_line + (long long)L.l * sc.Tp + t;
    L.lg = sc.line0 + L.l;
    L.bf = sc.e_bus + (long long)c.l_from[L.lg] * sc.Tp + t;
    L.bt = sc.e_bus + (long long)c.l_to[L.lg] * sc.Tp + t;
}

template <int MODE, int ADJ>
__device__ __forceinline__ void line_load(const Ctx& c, const ScenDev& sc, const StatePtrs& X, LineIn& L) {
    if (!L.valid) return;
    L.d = X.dl[L.row]; L.g = X.sg[L.row]; L.qf = X.vf[L.row]; L.qt = X.vt[L.row];
    L.pbf = X.pbar[L.bf]; L.uf = X.u[L.bf]; L.zf = X.thb[L.bf];
    L.pbt = X.pbar[L.bt]; L.ut = X.u[L.bt]; L.zt = X.thb[L.bt];
    L.beta = c.l_beta[L.lg]; L.w = c.l_w[L.lg]; L.dth = c.l_dth[L.lg];
    L.capf = fmaxf(c.eta[sc.eta0 + sc.G + L.l], 0.f) / L.beta;
    L.mask = ADJ ? c.m_line[L.row] : 0;
}

// Phase consensus in exact ADMM form: the line keeps q_j = y_j + v_j (terminal phase
// plus its scaled dual); the bus value z is the weighted mean of the q_j, so the duals
// v_j = q_j - z keep a zero weighted sum at every bus even under rounding.
template <int MODE, int ADJ>
__device__ __forceinline__ void line_compute(const Ctx& c, const StatePtrs& X, const LineIn& L, float& dx2,
                                             float& x2, float& th2) {
    if (!L.valid) return;
    const float beta = L.beta, d = L.d, g = L.g;
    const float vf = L.qf - L.zf, vt = L.qt - L.zt;
    const float ef = 0.5f * (g + d) - L.zf, et = 0.5f * (g - d) - L.zt;  // y - z of the last iteration
    const bool dc = L.w == 0.f;  // HVDC transport line: no phase coupling, eps/2 f^2 cost
    if (!dc) th2 += beta * beta * (ef * ef + et * et);
    const float wf = L.zf - vf, wt = L.zt - vt;
    const float tf = -beta * d - L.pbf - L.uf;  // power targets of the two terminals
    const float tt = beta * d - L.pbt - L.ut;
    const float rth = c.rth_c * L.w;
    const float den = 2.f * c.rho * beta * beta + 0.5f * rth + (dc ? c.eps : 0.f);
    // adjoint of a transport line: the linear term eps f* of grad h at the solved flow
    const float lin = (ADJ && dc) ? c.eps * c.dl[L.row] : 0.f;
    const float dun = (c.rho * beta * (tt - tf) + 0.5f * rth * (wf - wt) + lin) / den;
    const float cap = fminf(L.capf, L.dth);
    if (MODE == M_MASK) {
        uint8_t code = AL_FREE;
        const float over = fabsf(dun) - cap;
        if (over > 0.f && den * over / beta > c.tol_act) {
            const bool flow = L.capf <= L.dth;
            code = dun > 0.f ? (flow ? AL_FUP : AL_AUP) : (flow ? AL_FLO : AL_ALO);
        }
        c.m_line[L.row] = code;
        return;
    }
    float dn;
    if (ADJ) dn = L.mask ? 0.f : dun;
    else dn = clampf(dun, -cap, cap);
    const float gn = wf + wt;
    X.dl[L.row] = dn;
    X.sg[L.row] = gn;
    X.vf[L.row] = 0.5f * (gn + dn) + vf;
    X.vt[L.row] = 0.5f * (gn - dn) + vt;
    const float dd = dn - d;
    dx2 += 2.f * beta * beta * dd * dd;
    x2 += 2.f * beta * beta * dn * dn;
}

// ------------------------------------------------------------------------------------
// Line prox.  With delta = th_f - th_t and sigma = th_f + th_t the prox of a lossless DC
// line separates: sigma = w_f + w_t, and delta minimises the 1-D quadratic
//   rho/2 [(-beta d - v_f)^2 + (beta d - v_t)^2] + rho_th/4 (d - (w_f - w_t))^2
// over |beta d| <= eta_l, |d| <= dtheta_max, i.e. the unconstrained minimiser clipped.
// Each thread handles kLineItems line-hours of its block.
// ------------------------------------------------------------------------------------
template <int MODE, int ADJ>
__global__ void __launch_bounds__(kBlock) k_line(const Ctx c, int want_res) {
    const int blk = blockIdx.x;
    const int s = c.line_blk_scen[blk];
    if (c.done[s]) return;
    const ScenDev sc = c.scen[s];
    const StatePtrs X = state<ADJ>(c);
    const int base = (blk - sc.line_blk0) * kBlock * kLineItems + threadIdx.x;
    float dx2 = 0.f, x2 = 0.f, th2 = 0.f;
    if (MODE == M_RESET) {
        for (int r = 0; r < kLineItems; ++r) {
            LineIn L;
            line_index<MODE, ADJ>(c, sc, base + r * kBlock, L);
            if (!L.valid) continue;
            float d0 = 0.f, g0 = 0.f, q0f = 0.f, q0t = 0.f;
            if (!ADJ && c.warm && c.l_w[L.lg] != 0.f) {  // (a transport line's flow starts at 0)
                const float* th = c.warm + c.warm_half;
                d0 = th[L.bf] - th[L.bt];
                g0 = th[L.bf] + th[L.bt];
                q0f = th[L.bf];
                q0t = th[L.bt];
            }
            if (ADJ && c.adj_from_fwd) {
                // h = c part of the adjoint: phase duals are the negated forward ones
                // (scaled duals convert with rho_f / rho_a); adjoint phases start at 0
                q0f = -c.rho_ratio * (c.vf[L.row] - c.thb[L.bf]);
                q0t = -c.rho_ratio * (c.vt[L.row] - c.thb[L.bt]);
            }
            X.dl[L.row] = d0; X.sg[L.row] = g0; X.vf[L.row] = q0f; X.vt[L.row] = q0t;
        }
        return;
    }
    LineIn L[kLineItems];
#pragma unroll
    for (int r = 0; r < kLineItems; ++r) line_index<MODE, ADJ>(c, sc, base + r * kBlock, L[r]);
#pragma unroll
    for (int r = 0; r < kLineItems; ++r) line_load<MODE, ADJ>(c, sc, X, L[r]);
#pragma unroll
    for (int r = 0; r < kLineItems; ++r) line_compute<MODE, ADJ>(c, X, L[r], dx2, x2, th2);
    if ((MODE == M_FWD || MODE == M_ADJ) && want_res) {
        __shared__ float sh[3][kBlock / 32];
        float v[3] = {dx2, x2, th2};
        block_sum<3>(v, sh);
        if (threadIdx.x == 0) {
            c.line_part[blk * kDevPart + 0] = v[0];
            c.line_part[blk * kDevPart + 1] = v[1];
            c.line_part[blk * kDevPart + 2] = v[2];
        }
    }
}

// ------------------------------------------------------------------------------------
// Battery prox, one warp per battery, hours split in contiguous chunks of hpl per lane.
//   min sum_t eps/2 (c^2 + d^2) + q_c c + q_d d + rho/2 (d - c - v_t)^2
//   s.t. s_t = s_{t-1} + a c_t - k d_t (s_{-1} = 0), box bounds on c, d, s,
// solved by inner ADMM (x = (c, d, s) with the dynamics, z = box copy).  The x-step is
// an equality-constrained QP whose multipliers mu solve a constant tridiagonal system
// (pivots precomputed in bat_dd); its two Thomas sweeps are first-order linear
// recurrences evaluated with warp-wide affine scans.
// ------------------------------------------------------------------------------------
// kW warps per battery (1 or 2; a block of kBatWarps warps holds kBatWarps / kW
// batteries).  With two warps the hours split over 64 lanes, halving each lane's serial
// sweeps; the scans then combine the two warps' totals through shared memory.
template <int MODE, int ADJ, int kHpl, int kW>
__global__ void __launch_bounds__(kBatWarps * 32) k_bat(const Ctx c, int want_res) {
    static_assert(kW == 1 || kW == 2, "one or two warps per battery");
    constexpr int NL = 32 * kW;  // lanes per battery
    const int L = threadIdx.x & (NL - 1);  // lane within the battery
    const int lane = L & 31, wb = L >> 5;  // lane within the warp, warp within the battery
    const int gw = blockIdx.x * (kBatWarps / kW) + (int)(threadIdx.x / NL);
    if (gw >= c.n_bat_warps) return;  // block-uniform when kW == 2 (one battery per block)
    const bool stamp = (MODE == M_FWD || MODE == M_ADJ) && want_res && c.stamp_lo != nullptr;
    if (stamp && L == 0) stamp_start(c, 2);
    // the warp's offsets in one record (its row, its bus's row); in the iterations the done
    // flag is read with the state and tested before anything is stored
    const BatW bw = c.bat_w[gw];
    const int s = bw.s;
    const int done = c.done[s];
    if ((MODE != M_FWD && MODE != M_ADJ) && done) return;
    const StatePtrs X = state<ADJ>(c);
    const int bg = bw.bg;
    const int T = bw.T;
    const int hpl = (T + NL - 1) / NL;
    const int t0 = L * hpl;
    __shared__ float xch[8];  // two-warp exchange: rs, forward (A, B), backward (A, B), partials
    const long long row0 = bw.row0;
    const long long brow0 = bw.brow0;

    if (MODE == M_RESET) {
        const bool neg = ADJ && c.adj_from_fwd;
        for (int t = L; t < bw.Tp; t += NL) {
            const long long r = row0 + t;
            X.xb[r] = 0.f; X.zc[r] = 0.f; X.zd[r] = 0.f; X.zs[r] = 0.f;
            // h = c part of the adjoint: box multipliers are the negated forward ones
            X.yc[r] = neg ? -c.yc[r] : 0.f;
            X.yd[r] = neg ? -c.yd[r] : 0.f;
            X.ys[r] = neg ? -c.ys[r] : 0.f;
        }
        return;
    }
    const float rho = c.rho, eps = c.eps, ri = c.rho_in, iri = 1.f / c.rho_in;
    if (MODE == M_MASK) {
        // active set from the inner box multipliers of the forward solution
        for (int t = L; t < T; t += NL) {
            const long long r = row0 + t;
            const float y3[3] = {c.yc[r], c.yd[r], c.ys[r]};
            uint8_t code = 0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                uint8_t a = A_FREE;
                if (y3[q] > c.tol_act) a = A_UP;
                else if (y3[q] < -c.tol_act) a = A_LO;
                code |= a << (2 * q);
            }
            c.m_bat[r] = code;
        }
        return;
    }
    const float P = fmaxf(c.eta[bw.eta_b], 0.f);
    const float E = c.b_dur[bg] * P;
    const float a = c.b_effc[bg], k = 1.f / c.b_effd[bg];
    const float Ah = eps + ri + rho;
    const float det = Ah * Ah - rho * rho;
    const float idet = 1.f / det;
    const float gc = (Ah * a - rho * k) * idet;   // d(c)/d(mu)
    const float gd = (rho * a - Ah * k) * idet;   // d(d)/d(mu)

    float v[kHpl], zc[kHpl], zd[kHpl], zs[kHpl], yc[kHpl], yd[kHpl], ys[kHpl];
    float lo[3][kHpl], hi[3][kHpl], qc[kHpl], qd[kHpl];
    float idd[kHpl], iddp[kHpl];  // 1/dd_t and 1/dd_{t-1} (0 for t = 0)
    float xb_old[kHpl];
    // Every load of the lane's hours is issued before any of them is used: hours past
    // the horizon read hour T-1 (a valid row) and are zeroed afterwards.
#pragma unroll
    for (int j = 0; j < kHpl; ++j) {
        const int t = t0 + j;
        const bool ok = (j < hpl) && (t < T);
        const int tc = ok ? t : T - 1;
        const long long r = row0 + tc;
        xb_old[j] = X.xb[r];
        v[j] = xb_old[j] - X.pbar[brow0 + tc] - X.u[brow0 + tc];
        zc[j] = X.zc[r]; zd[j] = X.zd[r]; zs[j] = X.zs[r];
        yc[j] = X.yc[r]; yd[j] = X.yd[r]; ys[j] = X.ys[r];
        idd[j] = c.bat_dd[r];
        iddp[j] = c.bat_dd[tc > 0 ? r - 1 : r];
        if (ADJ) {
            const uint8_t m = c.m_bat[r];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const bool fixed = ((m >> (2 * q)) & 3) != A_FREE;
                lo[q][j] = fixed ? 0.f : -FLT_MAX;
                hi[q][j] = fixed ? 0.f : FLT_MAX;
            }
            qc[j] = -eps * c.zc[r];
            qd[j] = -eps * c.zd[r];
        } else {
            lo[0][j] = lo[1][j] = lo[2][j] = 0.f;
            hi[0][j] = P; hi[1][j] = P; hi[2][j] = E;
        }
    }
    if (done) return;  // uniform over the battery's warps; nothing stored yet
#pragma unroll
    for (int j = 0; j < kHpl; ++j) {
        const int t = t0 + j;
        const bool ok = (j < hpl) && (t < T);
        idd[j] = ok ? 1.f / idd[j] : 0.f;
        iddp[j] = (ok && t > 0) ? 1.f / iddp[j] : 0.f;
        if (!ok) {
            v[j] = zc[j] = zd[j] = zs[j] = yc[j] = yd[j] = ys[j] = 0.f;
            qc[j] = qd[j] = 0.f; xb_old[j] = 0.f;
            lo[0][j] = lo[1][j] = lo[2][j] = 0.f;
            hi[0][j] = hi[1][j] = hi[2][j] = 0.f;
        }
    }

    float cx[kHpl], dx[kHpl];
#pragma unroll
    for (int j = 0; j < kHpl; ++j) { cx[j] = 0.f; dx[j] = 0.f; }

    for (int it = 0; it < c.inner_iters; ++it) {
        float c0[kHpl], d0[kHpl], rs[kHpl], rhs[kHpl];
#pragma unroll
        for (int j = 0; j < kHpl; ++j) {
            const float rc = zc[j] - yc[j] * iri, rd = zd[j] - yd[j] * iri;
            rs[j] = zs[j] - ys[j] * iri;
            const float b1 = ri * rc - rho * v[j] - qc[j];
            const float b2 = ri * rd + rho * v[j] - qd[j];
            c0[j] = (Ah * b1 + rho * b2) * idet;
            d0[j] = (rho * b1 + Ah * b2) * idet;
        }
        // previous hour's r_s for the first hour of the chunk (0 before hour 0)
        float rs_last = 0.f;
#pragma unroll
        for (int j = 0; j < kHpl; ++j) if (j == hpl - 1) rs_last = rs[j];
        float rs_prev = __shfl_up_sync(0xffffffffu, rs_last, 1);
        if (kW == 2) {
            if (L == 31) xch[0] = rs_last;
            __syncthreads();
        }
        if (lane == 0) rs_prev = (kW == 2 && wb == 1) ? xch[0] : 0.f;
        // forward sweep y_t = rhs_t + y_{t-1} / dd_{t-1}
        float A = 1.f, Bv = 0.f;
#pragma unroll
        for (int j = 0; j < kHpl; ++j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            const float prev = j == 0 ? rs_prev : rs[j > 0 ? j - 1 : 0];
            rhs[j] = ok ? ri * (rs[j] - prev - (a * c0[j] - k * d0[j])) : 0.f;
            if (ok) { A = iddp[j] * A; Bv = iddp[j] * Bv + rhs[j]; }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float Ao = __shfl_up_sync(0xffffffffu, A, o);
            const float Bo = __shfl_up_sync(0xffffffffu, Bv, o);
            if (lane >= o) { Bv = A * Bo + Bv; A = A * Ao; }
        }
        float yin = __shfl_up_sync(0xffffffffu, Bv, 1);
        if (kW == 2) {
            // the second warp's prefixes start from the first warp's total
            if (L == 31) { xch[1] = A; xch[2] = Bv; }
            __syncthreads();
            if (wb == 1) {
                const float A0 = xch[1], B0 = xch[2];
                Bv = A * B0 + Bv;
                A = A * A0;
                const float yw = __shfl_up_sync(0xffffffffu, Bv, 1);
                yin = lane == 0 ? B0 : yw;
            }
        }
        if (lane == 0 && !(kW == 2 && wb == 1)) yin = 0.f;
        float yv[kHpl];
#pragma unroll
        for (int j = 0; j < kHpl; ++j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            if (ok) yin = iddp[j] * yin + rhs[j];
            yv[j] = yin;
        }
        // backward sweep mu_t = (y_t + mu_{t+1}) / dd_t, mu_T = 0
        A = 1.f; Bv = 0.f;
#pragma unroll
        for (int j = kHpl - 1; j >= 0; --j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            if (ok) { A = idd[j] * A; Bv = idd[j] * Bv + idd[j] * yv[j]; }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float Ao = __shfl_down_sync(0xffffffffu, A, o);
            const float Bo = __shfl_down_sync(0xffffffffu, Bv, o);
            if (lane + o < 32) { Bv = A * Bo + Bv; A = A * Ao; }
        }
        float min_ = __shfl_down_sync(0xffffffffu, Bv, 1);
        if (kW == 2) {
            // the first warp's suffixes continue into the second warp's total
            if (L == 32) { xch[3] = A; xch[4] = Bv; }
            __syncthreads();
            if (wb == 0) {
                const float B1 = xch[4];
                Bv = A * B1 + Bv;
                A = A * xch[3];
                const float mw = __shfl_down_sync(0xffffffffu, Bv, 1);
                min_ = lane == 31 ? B1 : mw;
            }
        }
        if (lane == 31 && !(kW == 2 && wb == 0)) min_ = 0.f;
        float mu[kHpl];
        float mnext = min_;
#pragma unroll
        for (int j = kHpl - 1; j >= 0; --j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            mu[j] = 0.f;
            if (ok) { mnext = idd[j] * (yv[j] + mnext); mu[j] = mnext; }
        }
        // x = (c, d, s), then the box projection and the inner dual step
#pragma unroll
        for (int j = 0; j < kHpl; ++j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            if (!ok) continue;
            float mu_n;
            if (t + 1 >= T) mu_n = 0.f;
            else if (j + 1 < hpl) mu_n = mu[j + 1 < kHpl ? j + 1 : j];
            else mu_n = min_;
            const float cc = c0[j] + mu[j] * gc;
            const float dd_ = d0[j] + mu[j] * gd;
            const float ss = rs[j] - (mu[j] - mu_n) * iri;
            const float nzc = clampf(cc + yc[j] * iri, lo[0][j], hi[0][j]);
            const float nzd = clampf(dd_ + yd[j] * iri, lo[1][j], hi[1][j]);
            const float nzs = clampf(ss + ys[j] * iri, lo[2][j], hi[2][j]);
            yc[j] += ri * (cc - nzc);
            yd[j] += ri * (dd_ - nzd);
            ys[j] += ri * (ss - nzs);
            zc[j] = nzc; zd[j] = nzd; zs[j] = nzs;
            cx[j] = cc; dx[j] = dd_;
        }
        // mu_n for a chunk's last hour reads the next lane's first mu: the shuffle above
        // (min_) is that value because the suffix scan composes whole chunks.
    }
    float dx2 = 0.f, x2 = 0.f;
#pragma unroll
    for (int j = 0; j < kHpl; ++j) {
        const int t = t0 + j;
        const bool ok = (j < hpl) && (t < T);
        if (!ok) continue;
        const long long r = row0 + t;
        const float xn = dx[j] - cx[j];
        X.xb[r] = xn;
        X.zc[r] = zc[j]; X.zd[r] = zd[j]; X.zs[r] = zs[j];
        X.yc[r] = yc[j]; X.yd[r] = yd[j]; X.ys[r] = ys[j];
        dx2 += (xn - xb_old[j]) * (xn - xb_old[j]);
        x2 += xn * xn;
    }
    if (want_res) {
        dx2 = warp_sum(dx2);
        x2 = warp_sum(x2);
        if (kW == 2) {
            if (L == 32) { xch[5] = dx2; xch[6] = x2; }
            __syncthreads();
            if (L == 0) { dx2 += xch[5]; x2 += xch[6]; }
        }
        if (L == 0) {
            c.bat_part[gw * kDevPart + 0] = dx2;
            c.bat_part[gw * kDevPart + 1] = x2;
            c.bat_part[gw * kDevPart + 2] = 0.f;
            if (stamp) stamp_end(c, 2);
        }
    }
}

// ------------------------------------------------------------------------------------
// Bus kernel: generator and load proxes (closed-form clips), then the consensus step.
//
// A block covers 256 consecutive (bus, hour) items of one scenario, i.e. a few whole
// buses.  The static data of those buses (each bus's device lists, generator cost,
// emission rate and firm flag, line-end codes with beta and phase weight, battery rows,
// bus constants) is one contiguous pool record built at create and shared by every
// scenario of the network with the same bus range; k_prep writes the generators' plan
// values into it at the start of each call.  The block copies its record to shared
// memory with 16-byte loads while each thread's own bus-state loads are in flight; then
// each thread issues the loads of a first chunk of its device terminals before its first
// store.  A record too long for shared memory is read from global memory in place.
// ------------------------------------------------------------------------------------
struct Pool {
    const int* p;  // the record, in shared or global memory
    __device__ __forceinline__ int at(int h, int k) const { return p[p[h] + k]; }
    __device__ __forceinline__ float atf(int h, int k) const { return __int_as_float(p[p[h] + k]); }
};

constexpr int kGC = 4;  // generators per load chunk
constexpr int kEC = 4;  // line ends loaded ahead of the generator stores
constexpr int kBC = 2;  // batteries loaded ahead of the generator stores

// Per-item inputs read before the block's staging barrier.
struct BusIn {
    float pb, uu, thold, xl, Lnt, al;
};

template <int MODE, int ADJ>
__device__ __forceinline__ void bus_item(const Ctx& c, const BusBlk& bb, const StatePtrs& X, const Pool P, int nl,
                                         int t, long long i, const BusIn& in, int want_res,
                                         float (&acc)[kBusPart]) {
    const float rho = c.rho, eps = c.eps;
    const float inv_re = 1.f / (rho + eps);
    const int g0 = P.at(kPH_GP, nl), g1 = P.at(kPH_GP, nl + 1);
    const long long gt = bb.e_gen + t;  // generator rows: gt + row * Tp
    const float Lnt = in.Lnt;
    if (MODE == M_RESET) {
        X.xl[i] = ADJ ? 0.f : -Lnt;
        if (ADJ) X.u[i] = c.adj_from_fwd ? -c.rho_ratio * c.u[i] : 0.f;
        else X.u[i] = c.warm ? -c.warm[i] / rho : 0.f;
        X.pbar[i] = 0.f;
        X.thb[i] = (!ADJ && c.warm) ? c.warm[c.warm_half + i] : 0.f;
        if (!ADJ && c.warm) {
            // user start: each generator and load at its best response to the given price
            const float lam = c.warm[i];
            const float shed = clampf((lam - c.voll) / eps, 0.f, Lnt);
            X.xl[i] = shed - Lnt;
            for (int q = g0; q < g1; ++q) {
                const long long r = gt + (long long)P.at(kPH_GROW, q) * bb.Tp;
                const float cap = (P.at(kPH_GFIRM, q) & 1) ? P.atf(kPH_GETA, q) : c.cf[r] * P.atf(kPH_GETA, q);
                X.xg[r] = clampf((lam - P.atf(kPH_GCOST, q)) / eps, 0.f, cap);
            }
        } else {
            for (int q = g0; q < g1; ++q) X.xg[gt + (long long)P.at(kPH_GROW, q) * bb.Tp] = 0.f;
        }
        return;
    }
    const float pb = in.pb, uu = in.uu;
    const int e0 = P.at(kPH_EP, nl), e1 = P.at(kPH_EP, nl + 1);
    const int b0 = P.at(kPH_BP, nl), b1 = P.at(kPH_BP, nl + 1);
    // first chunk of line ends and batteries: their loads are in flight during the
    // generator proxes (they are only summed, after the generators and the load)
    float ed[kEC], eq[kEC], bx[kBC];
    if (MODE != M_MASK) {
#pragma unroll
        for (int k = 0; k < kEC; ++k) {
            const int q = e0 + k;
            ed[k] = eq[k] = 0.f;
            if (q < e1) {
                const int e = P.at(kPH_ECODE, q);
                const long long r = bb.e_line + (long long)(e >> 1) * bb.Tp + t;
                ed[k] = X.dl[r];
                eq[k] = (e & 1) ? X.vt[r] : X.vf[r];
            }
        }
#pragma unroll
        for (int k = 0; k < kBC; ++k) {
            const int q = b0 + k;
            bx[k] = q < b1 ? X.xb[bb.e_bat + (long long)P.at(kPH_BROW, q) * bb.Tp + t] : 0.f;
        }
    }
    float sum = 0.f, dx2 = 0.f, x2 = 0.f;
    float gscale = 0.f;  // adjoint: sum of (grad h / (rho + eps))^2 over free terminals
    // generators, kGC at a time: all loads of a chunk before its stores
    for (int q0 = g0; q0 < g1; q0 += kGC) {
        float xv[kGC], av[kGC];
        int ro[kGC];
#pragma unroll
        for (int k = 0; k < kGC; ++k) {
            const int q = q0 + k;
            xv[k] = 0.f; av[k] = 1.f; ro[k] = 0;
            if (q < g1) {
                ro[k] = P.at(kPH_GROW, q) * bb.Tp;
                xv[k] = X.xg[gt + ro[k]];
                if (ADJ) {
                    av[k] = c.ag[gt + ro[k]];
                } else if (MODE != M_INIT && !(P.at(kPH_GFIRM, q) & 1)) {
                    av[k] = c.cf[gt + ro[k]];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kGC; ++k) {
            const int q = q0 + k;
            if (q >= g1) break;
            // a ramp-limited generator's prox and active set come from the ramp kernel
            const bool rampg = (P.at(kPH_GFIRM, q) & 2) != 0;
            if (MODE == M_MASK && rampg) continue;
            const float x = xv[k];
            float xn = x;
            if ((MODE == M_FWD || MODE == M_ADJ || MODE == M_MASK) && !rampg) {
                const float v = x - pb - uu;
                if (ADJ) {
                    const float gh = av[k];  // NaN: bound active, the variable is fixed at 0
                    const bool fixed = gh != gh;
                    xn = fixed ? 0.f : (rho * v + gh) * inv_re;
                    if (!fixed) gscale += (gh * inv_re) * (gh * inv_re);
                } else {
                    const float cap = av[k] * P.atf(kPH_GETA, q);
                    const float pun = (rho * v - P.atf(kPH_GCOST, q)) * inv_re;
                    if (MODE == M_MASK) {
                        uint8_t code = A_FREE;
                        if (pun > cap && (rho + eps) * (pun - cap) > c.tol_act) code = A_UP;
                        else if (pun < 0.f && -(rho + eps) * pun > c.tol_act) code = A_LO;
                        c.m_gen[gt + ro[k]] = code;
                        // the adjoint's linear term at the forward dispatch x (h = cost + kappa e)
                        c.ag[gt + ro[k]] = code != A_FREE ? __int_as_float(0x7fc00000)
                                                          : P.atf(kPH_GCOST, q) + eps * x + c.kappa * P.atf(kPH_GEMIS, q);
                    } else {
                        xn = clampf(pun, 0.f, cap);
                    }
                }
                if (MODE != M_MASK) X.xg[gt + ro[k]] = xn;
            }
            sum += xn;
            dx2 += (xn - x) * (xn - x);
            x2 += xn * xn;
        }
    }
    // load (shed variable; terminal injection shed - L)
    {
        const float x = in.xl;
        float xn = x;
        if (MODE == M_FWD || MODE == M_ADJ || MODE == M_MASK) {
            const float v = x - pb - uu;
            if (ADJ) {
                const float gsh = in.al;  // NaN: bound active, the variable is fixed at 0
                const bool fixed = gsh != gsh;
                xn = fixed ? 0.f : (rho * v + gsh) * inv_re;
                if (!fixed) gscale += (gsh * inv_re) * (gsh * inv_re);
            } else {
                const float sun = (rho * (v + Lnt) - c.voll) * inv_re;
                if (MODE == M_MASK) {
                    uint8_t code = A_FREE;
                    if (sun > Lnt && (rho + eps) * (sun - Lnt) > c.tol_act) code = A_UP;
                    else if (sun < 0.f && -(rho + eps) * sun > c.tol_act) code = A_LO;
                    c.m_load[i] = code;
                    // the adjoint's linear term at the forward shed x + L
                    c.al[i] = code != A_FREE ? __int_as_float(0x7fc00000) : c.voll + eps * (x + Lnt);
                } else {
                    xn = clampf(sun, 0.f, Lnt) - Lnt;
                }
            }
            if (MODE != M_MASK) X.xl[i] = xn;
        }
        sum += xn;
        dx2 += (xn - x) * (xn - x);
        x2 += xn * xn;
    }
    if (MODE == M_MASK) return;
    // batteries (their prox ran in k_bat this iteration)
#pragma unroll
    for (int k = 0; k < kBC; ++k) {
        if (b0 + k < b1) {
            sum += bx[k];
            x2 += bx[k] * bx[k];
        }
    }
    for (int q = b0 + kBC; q < b1; ++q) {
        const float xb = X.xb[bb.e_bat + (long long)P.at(kPH_BROW, q) * bb.Tp + t];
        sum += xb;
        x2 += xb * xb;
    }
    // line ends (their prox ran in k_line this iteration)
    float ths = 0.f;
#pragma unroll
    for (int k = 0; k < kEC; ++k) {
        const int q = e0 + k;
        if (q < e1) {
            const float beta = P.atf(kPH_EBETA, q);
            const float p = (P.at(kPH_ECODE, q) & 1) ? beta * ed[k] : -beta * ed[k];
            sum += p;
            x2 += p * p;
            ths += P.atf(kPH_EW, q) * eq[k];
        }
    }
    for (int q = e0 + kEC; q < e1; ++q) {
        const int e = P.at(kPH_ECODE, q);
        const long long r = bb.e_line + (long long)(e >> 1) * bb.Tp + t;
        const float d = X.dl[r];
        const float qv = (e & 1) ? X.vt[r] : X.vf[r];
        const float beta = P.atf(kPH_EBETA, q);
        const float p = (e & 1) ? beta * d : -beta * d;
        sum += p;
        x2 += p * p;
        ths += P.atf(kPH_EW, q) * qv;
    }
    const float icnt = P.atf(kPH_IC, nl);
    const float pbn = sum * icnt;
    const float thn = ths * P.atf(kPH_IW, nl);
    if (MODE == M_INIT) {
        X.pbar[i] = pbn;
        X.thb[i] = thn;
        return;
    }
    const float un = uu + pbn;
    X.pbar[i] = pbn;
    X.u[i] = un;
    X.thb[i] = thn;
    if (want_res) {
        const float cnt = 1.f / icnt;
        const float dpb = pbn - pb;
        acc[0] = cnt * pbn * pbn;
        acc[1] = gscale;
        acc[2] = dx2 - cnt * dpb * dpb;
        acc[3] = (thn - in.thold) * (thn - in.thold) * P.atf(kPH_DR, nl);
        acc[4] = cnt * (rho * un) * (rho * un);
        acc[5] = x2;
    }
}

template <int MODE, int ADJ>
__global__ void __launch_bounds__(kBlock, 4) k_bus(const Ctx c, int want_res) {
    __shared__ __align__(16) int S[kPoolMax];
    const BusBlk bb = c.bus_blk[blockIdx.x];
    if (c.done[bb.s]) return;  // block-uniform
    const StatePtrs X = state<ADJ>(c);
    const bool staged = bb.words <= kPoolMax;
    if (staged) {
        const int4* src = reinterpret_cast<const int4*>(c.pool + bb.pool);
        int4* dst = reinterpret_cast<int4*>(S);
        for (int k = threadIdx.x; k < (bb.words >> 2); k += kBlock) dst[k] = src[k];
    }
    const int local = bb.item0 + threadIdx.x;
    const int n = local / bb.Tp;
    const int t = local - n * bb.Tp;
    const bool valid = (local < bb.nitems) && (t < bb.T);
    const long long i = bb.e_bus + local;
    BusIn in{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
        if (MODE != M_INIT) in.Lnt = c.load[i];
        if (MODE == M_FWD || MODE == M_ADJ || MODE == M_MASK) {
            in.pb = X.pbar[i]; in.uu = X.u[i]; in.thold = X.thb[i];
        }
        if (MODE != M_RESET) in.xl = X.xl[i];
        if (ADJ && MODE == M_ADJ) in.al = c.al[i];
    }
    __syncthreads();
    float acc[kBusPart] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
        const Pool P{staged ? S : c.pool + bb.pool};
        bus_item<MODE, ADJ>(c, bb, X, P, n - bb.n0, t, i, in, want_res, acc);
    }
    if ((MODE == M_FWD || MODE == M_ADJ) && want_res) {
        __shared__ float sh[kBusPart][kBlock / 32];
        block_sum<kBusPart>(acc, sh);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < kBusPart; ++q) c.bus_part[blockIdx.x * kBusPart + q] = acc[q];
        }
    }
}

// ------------------------------------------------------------------------------------
// Iteration kernels over hour quads.  In the forward and adjoint iterations a thread of
// the line or bus kernel handles four consecutive hours of one device row (rows are
// padded to a multiple of 4 hours, so every quad is 16-byte aligned): one 128-bit load
// or store per array instead of four, and the index arithmetic and device-list walk
// paid once per four hours.  Each hour's arithmetic is that of the single-hour code
// above, in the same order; hours past the horizon stay zero.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void ldm4(const uint8_t* p, int (&v)[4]) {
    const uchar4 q = *reinterpret_cast<const uchar4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}

// Resident blocks per SM the line kernel is compiled for (its register cap).
#ifndef GX_LINE4_MINB
#define GX_LINE4_MINB 1
#endif
template <int ADJ>
__global__ void __launch_bounds__(kQBlock, GX_LINE4_MINB) k_line4(const Ctx c, int want_res) {
    const int blk = blockIdx.x;
    const bool stamp = want_res && c.stamp_lo != nullptr;
    if (stamp && threadIdx.x == 0) stamp_start(c, 1);
    // The block's offsets and its lines' end buses in one record (the ends staged in shared
    // memory); then the done flag, the line's state and its end buses' rows are read together,
    // and the flag tested before anything is stored.
    __shared__ int s_end[2 * kLineBlkLines];
    const LineBlk lb = c.line4_blk[blk];
    if (threadIdx.x < 2 * kLineBlkLines) s_end[threadIdx.x] = c.line4_blk[blk].ends[threadIdx.x];
    __syncthreads();
    const int done = c.done[lb.s];
    const StatePtrs X = state<ADJ>(c);
    const int Tq = lb.Tp >> 2;
    const int local = lb.item0 + threadIdx.x;
    const int l = local / Tq;
    const int t = (local - l * Tq) * 4;
    float dx2 = 0.f, x2 = 0.f, th2 = 0.f;
    if (l < lb.L) {
        const long long row = lb.e_line + (long long)l * lb.Tp + t;
        const int lg = lb.line0 + l;
        float d[4], g[4], qf[4], qt[4], pbf[4], uf[4], zf[4], pbt[4], ut[4], zt[4];
        ld4(X.dl + row, d); ld4(X.sg + row, g); ld4(X.vf + row, qf); ld4(X.vt + row, qt);
        const int end_f = lb.nends ? s_end[2 * (l - lb.l0)] : c.l_from[lg];
        const int end_t = lb.nends ? s_end[2 * (l - lb.l0) + 1] : c.l_to[lg];
        const long long bf = lb.e_bus + (long long)end_f * lb.Tp + t;
        const long long bt = lb.e_bus + (long long)end_t * lb.Tp + t;
        int mk[4] = {0, 0, 0, 0};
        if (ADJ) ldm4(c.m_line + row, mk);
        const float beta = c.l_beta[lg];
        const float w = c.l_w[lg];
        const float etal = c.eta[lb.eta_l + l];
        const float dthl = c.l_dth[lg];
        ld4(X.pbar + bf, pbf); ld4(X.u + bf, uf); ld4(X.thb + bf, zf);
        ld4(X.pbar + bt, pbt); ld4(X.u + bt, ut); ld4(X.thb + bt, zt);
        if (done) return;  // block-uniform; nothing has been stored
        const bool dc = w == 0.f;  // HVDC transport line: no phase coupling, eps/2 f^2 cost
        const float rth = c.rth_c * w;
        const float capf = fmaxf(etal, 0.f) / beta;
        const float cap = fminf(capf, dthl);
        const float den = 2.f * c.rho * beta * beta + 0.5f * rth + (dc ? c.eps : 0.f);
        float fs[4] = {0.f, 0.f, 0.f, 0.f};  // adjoint of a transport line: eps f* of grad h
        if (ADJ && dc) ld4(c.dl + row, fs);
        float dn[4], gn[4], nf[4], nt[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            dn[h] = gn[h] = nf[h] = nt[h] = 0.f;
            if (t + h >= lb.T) continue;
            const float vf = qf[h] - zf[h], vt = qt[h] - zt[h];
            const float ef = 0.5f * (g[h] + d[h]) - zf[h], et = 0.5f * (g[h] - d[h]) - zt[h];
            if (!dc) th2 += beta * beta * (ef * ef + et * et);
            const float wf = zf[h] - vf, wt = zt[h] - vt;
            const float tf = -beta * d[h] - pbf[h] - uf[h];
            const float tt = beta * d[h] - pbt[h] - ut[h];
            const float dun = (c.rho * beta * (tt - tf) + 0.5f * rth * (wf - wt) + c.eps * fs[h]) / den;
            if (ADJ) dn[h] = mk[h] ? 0.f : dun;
            else dn[h] = clampf(dun, -cap, cap);
            gn[h] = wf + wt;
            nf[h] = 0.5f * (gn[h] + dn[h]) + vf;
            nt[h] = 0.5f * (gn[h] - dn[h]) + vt;
            const float dd = dn[h] - d[h];
            dx2 += 2.f * beta * beta * dd * dd;
            x2 += 2.f * beta * beta * dn[h] * dn[h];
        }
        st4(X.dl + row, dn); st4(X.sg + row, gn); st4(X.vf + row, nf); st4(X.vt + row, nt);
    }
    if (done) return;  // the threads past the network's lines
    if (want_res) {
        __shared__ float sh[3][kQBlock / 32];
        float v[3] = {dx2, x2, th2};
        block_sum<3, kQBlock>(v, sh);
        if (threadIdx.x == 0) {
            c.line_part[blk * kDevPart + 0] = v[0];
            c.line_part[blk * kDevPart + 1] = v[1];
            c.line_part[blk * kDevPart + 2] = v[2];
            if (stamp) stamp_end(c, 1);
        }
    }
}

constexpr int kEC4 = 4;  // line ends loaded ahead by the quad bus kernel
constexpr int kBC4 = 2;  // batteries loaded ahead

// One generator's quad: stored injection, then (adjoint) the adjoint coefficient (NaN where
// the bound is active), or (forward) the capacity factor (1 for firm generators).
template <int ADJ>
__device__ __forceinline__ void gen_load4(const Ctx& c, const StatePtrs& X, const Pool& P, long long r, int q,
                                          float (&x)[4], float (&a)[4]) {
    ld4(X.xg + r, x);
    if (ADJ) {
        ld4(c.ag + r, a);
    } else if (!(P.at(kPH_GFIRM, q) & 1)) {
        ld4(c.cf + r, a);
    } else {
        a[0] = a[1] = a[2] = a[3] = 1.f;
    }
}

// RAMP: the batch has ramp-limited generators (whose injections are only summed here);
// without them the flag test is compiled out.  At most 128 registers, so four blocks fit
// an SM: uncapped, the adjoint instance took 136, three blocks per SM, and a 16-scenario
// medium grid (3.45 blocks per SM) ran part of its blocks as a second wave.
template <int ADJ, int RAMP>
__global__ void __launch_bounds__(kBusQBlock, kBus4MinBlocks) k_bus4(const Ctx c, int want_res) {
    __shared__ __align__(16) int S[kPoolMax];
    const bool stamp = want_res && c.stamp_lo != nullptr;
    if (stamp && threadIdx.x == 0) stamp_start(c, 0);
    const BusBlk bb = c.bus4_blk[blockIdx.x];
    // The done flag, the record copy and this thread's bus state are all issued before the
    // flag is tested: one dependent round trip after the block record instead of two.
    const int done = c.done[bb.s];
    const StatePtrs X = state<ADJ>(c);
    const bool staged = bb.words <= kPoolMax;
    const int Tq = bb.Tp >> 2;
    const int local = bb.item0 + threadIdx.x;
    const int n = local / Tq;
    const int t = (local - n * Tq) * 4;
    const bool valid = local < bb.nitems;
    const long long i = bb.e_bus + (long long)n * bb.Tp + t;
    float pb[4], uu[4], thold[4], xl[4], Ld[4], al[4];
    if (valid) {
        ld4(X.pbar + i, pb); ld4(X.u + i, uu); ld4(X.thb + i, thold);
        ld4(X.xl + i, xl);
        if (ADJ) ld4(c.al + i, al);  // the adjoint needs the load only through its coefficient
        else ld4(c.load + i, Ld);
    }
    if (staged) {
        const int4* src = reinterpret_cast<const int4*>(c.pool + bb.pool);
        int4* dst = reinterpret_cast<int4*>(S);
        for (int k = threadIdx.x; k < (bb.words >> 2); k += kBusQBlock) dst[k] = src[k];
    }
    if (done) return;  // block-uniform, before any barrier or store
    __syncthreads();
    float acc[kBusPart] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
        const Pool P{staged ? S : c.pool + bb.pool};
        const int nl = n - bb.n0;
        const float rho = c.rho, eps = c.eps;
        const float inv_re = 1.f / (rho + eps);
        bool hv[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) hv[h] = t + h < bb.T;
        float sum[4] = {0.f, 0.f, 0.f, 0.f}, dx2[4] = {0.f, 0.f, 0.f, 0.f};
        float x2 = 0.f, gscale = 0.f;
        const long long gt = bb.e_gen + t;
        const int g0 = P.at(kPH_GP, nl), g1 = P.at(kPH_GP, nl + 1);
        const int e0 = P.at(kPH_EP, nl), e1 = P.at(kPH_EP, nl + 1);
        const int b0 = P.at(kPH_BP, nl), b1 = P.at(kPH_BP, nl + 1);
        // Loads ahead of the first store: the first kEC4 line ends and kBC4 batteries
        // (only summed at the end) and the first generator; each later generator is
        // loaded before the previous one's store.
        float ed[kEC4][4], eq[kEC4][4], bx[kBC4][4];
#pragma unroll
        for (int k = 0; k < kEC4; ++k) {
            const int q = e0 + k;
            if (q < e1) {
                const int e = P.at(kPH_ECODE, q);
                const long long r = bb.e_line + (long long)(e >> 1) * bb.Tp + t;
                ld4(X.dl + r, ed[k]);
                ld4((e & 1) ? X.vt + r : X.vf + r, eq[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kBC4; ++k)
            if (b0 + k < b1) ld4(X.xb + bb.e_bat + (long long)P.at(kPH_BROW, b0 + k) * bb.Tp + t, bx[k]);
        float xc[4], ac[4];
        if (g0 < g1) gen_load4<ADJ>(c, X, P, gt + (long long)P.at(kPH_GROW, g0) * bb.Tp, g0, xc, ac);
        for (int q = g0; q < g1; ++q) {
            const long long r = gt + (long long)P.at(kPH_GROW, q) * bb.Tp;
            float x[4], a[4], xn[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) { x[h] = xc[h]; a[h] = ac[h]; }
            if (q + 1 < g1) gen_load4<ADJ>(c, X, P, gt + (long long)P.at(kPH_GROW, q + 1) * bb.Tp, q + 1, xc, ac);
            if (RAMP && (P.at(kPH_GFIRM, q) & 2)) {
                // ramp-limited: the ramp kernel wrote this iteration's injection (and keeps
                // its own residual terms); the bus only sums it
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    sum[h] += x[h];
                    x2 += x[h] * x[h];
                }
                continue;
            }
            const float gcost = ADJ ? 0.f : P.atf(kPH_GCOST, q);
            const float etag = ADJ ? 0.f : P.atf(kPH_GETA, q);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float v = x[h] - pb[h] - uu[h];
                if (ADJ) {
                    const float gh = a[h];  // NaN: bound active, the variable is fixed at 0
                    const bool fixed = gh != gh;
                    xn[h] = fixed ? 0.f : (rho * v + gh) * inv_re;
                    if (!fixed && hv[h]) gscale += (gh * inv_re) * (gh * inv_re);
                } else {
                    const float cap = a[h] * etag;
                    const float pun = (rho * v - gcost) * inv_re;
                    xn[h] = clampf(pun, 0.f, cap);
                }
                if (!hv[h]) xn[h] = 0.f;
                sum[h] += xn[h];
                dx2[h] += (xn[h] - x[h]) * (xn[h] - x[h]);
                x2 += xn[h] * xn[h];
            }
            st4(X.xg + r, xn);
        }
        {
            float xn[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float v = xl[h] - pb[h] - uu[h];
                if (ADJ) {
                    const float gsh = al[h];  // NaN: bound active, the variable is fixed at 0
                    const bool fixed = gsh != gsh;
                    xn[h] = fixed ? 0.f : (rho * v + gsh) * inv_re;
                    if (!fixed && hv[h]) gscale += (gsh * inv_re) * (gsh * inv_re);
                } else {
                    const float sun = (rho * (v + Ld[h]) - c.voll) * inv_re;
                    xn[h] = clampf(sun, 0.f, Ld[h]) - Ld[h];
                }
                if (!hv[h]) xn[h] = 0.f;
                sum[h] += xn[h];
                dx2[h] += (xn[h] - xl[h]) * (xn[h] - xl[h]);
                x2 += xn[h] * xn[h];
            }
            st4(X.xl + i, xn);
        }
#pragma unroll
        for (int k = 0; k < kBC4; ++k) {
            if (b0 + k < b1) {
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    sum[h] += bx[k][h];
                    x2 += bx[k][h] * bx[k][h];
                }
            }
        }
        for (int q = b0 + kBC4; q < b1; ++q) {
            float xb[4];
            ld4(X.xb + bb.e_bat + (long long)P.at(kPH_BROW, q) * bb.Tp + t, xb);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                sum[h] += xb[h];
                x2 += xb[h] * xb[h];
            }
        }
        float ths[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kEC4; ++k) {
            const int q = e0 + k;
            if (q < e1) {
                const int e = P.at(kPH_ECODE, q);
                const float beta = P.atf(kPH_EBETA, q), w = P.atf(kPH_EW, q);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const float p = (e & 1) ? beta * ed[k][h] : -beta * ed[k][h];
                    sum[h] += p;
                    x2 += p * p;
                    ths[h] += w * eq[k][h];
                }
            }
        }
        for (int q = e0 + kEC4; q < e1; ++q) {
            const int e = P.at(kPH_ECODE, q);
            const long long r = bb.e_line + (long long)(e >> 1) * bb.Tp + t;
            float d[4], qv[4];
            ld4(X.dl + r, d);
            ld4((e & 1) ? X.vt + r : X.vf + r, qv);
            const float beta = P.atf(kPH_EBETA, q), w = P.atf(kPH_EW, q);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float p = (e & 1) ? beta * d[h] : -beta * d[h];
                sum[h] += p;
                x2 += p * p;
                ths[h] += w * qv[h];
            }
        }
        const float icnt = P.atf(kPH_IC, nl), iws = P.atf(kPH_IW, nl), drw = P.atf(kPH_DR, nl);
        const float cnt = 1.f / icnt;
        float pbn[4], un[4], thn[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            pbn[h] = sum[h] * icnt;
            thn[h] = ths[h] * iws;
            un[h] = uu[h] + pbn[h];
            if (hv[h]) {
                const float dpb = pbn[h] - pb[h];
                acc[0] += cnt * pbn[h] * pbn[h];
                acc[2] += dx2[h] - cnt * dpb * dpb;
                acc[3] += (thn[h] - thold[h]) * (thn[h] - thold[h]) * drw;
                acc[4] += cnt * (rho * un[h]) * (rho * un[h]);
            }
        }
        acc[1] = gscale;
        acc[5] = x2;
        st4(X.pbar + i, pbn);
        st4(X.u + i, un);
        st4(X.thb + i, thn);
    }
    if (want_res) {
        __shared__ float sh[kBusPart][kBusQBlock / 32];
        block_sum<kBusPart, kBusQBlock>(acc, sh);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < kBusPart; ++q) c.bus_part[blockIdx.x * kBusPart + q] = acc[q];
            if (stamp) stamp_end(c, 0);
        }
    }
}

// ------------------------------------------------------------------------------------
// Staged bus kernel.  The same iteration as k_bus4, expression for expression and in the
// same summation order (its iterates are bitwise those of k_bus4), with the block's device
// rows brought into shared memory first.  In k_bus4 a thread walks its bus's devices with
// one generator's loads in flight at a time, so a block waits for about 4 + (generators
// per bus) dependent memory round trips.  Here the block issues one bulk copy per device
// row segment (cp.async.bulk, completing on one mbarrier armed by thread 0; the copy list
// is built at create, in the pool record), so every row the block needs is in flight at once and
// the block waits for three hops: its block record; its pool record and the done flag; its
// bus state and the rows together (a converged scenario's blocks stop after the second).
// In the adjoint the generators' aux rows hold the adjoint coefficient (NaN where the bound
// is active), so the active set travels with the bulk copies.  A record too large for the
// stage runs the unstaged loads.
// ------------------------------------------------------------------------------------

// Whether a staged copy is issued: firm generators have no capacity-factor row to read and
// ramp-limited ones no aux row at all (the bus only sums their injection).
template <int ADJ>
__device__ __forceinline__ bool copy_wanted(int code) {
    if ((code & 7) != kCpGenAux) return true;
    const int fl = (code >> 3) & 3;
    if (fl & kCpRamp) return false;
    return ADJ || !(fl & kCpFirm);
}

// Source row base of a staged copy (copy-list code: array id in the low 3 bits).
template <int ADJ>
__device__ __forceinline__ const float* stage_src(const Ctx& c, const StatePtrs& X, const BusBlk& bb, int code) {
    switch (code & 7) {
        case kCpGenX: return X.xg + bb.e_gen;
        case kCpGenAux: return (ADJ ? c.ag : c.cf) + bb.e_gen;
        case kCpDl: return X.dl + bb.e_line;
        case kCpVf: return X.vf + bb.e_line;
        case kCpVt: return X.vt + bb.e_line;
        default: return X.xb + bb.e_bat;
    }
}

// Bounded wait for the block's bulk copies.  On expiry: report, give them one more bounded
// wait, and return false (the caller leaves without touching the iterate).
template <int ADJ>
__device__ __forceinline__ bool bulk_wait(const Ctx& c, unsigned long long* bar) {
    bool ok = false;
    for (int k = 0; k < kWaitProbes && !ok; ++k) ok = mbar_try(bar, 0);
    if (ok) return true;
    if (threadIdx.x == 0) atomicExch(c.err, GX_ERR_TIMEOUT);
    for (int k = 0; k < kWaitProbes && !ok; ++k) ok = mbar_try(bar, 0);
    return false;
}

// LIST: the block's copy list and done flag come from its own slot (c.bus_cpl); compiled
// apart so that the record-path instance keeps its registers.
template <int ADJ, int RAMP, int LIST>
__global__ void __launch_bounds__(kBusQBlock, GX_BUS4T_MINB * 128 / kBusQBlock) k_bus4t(const Ctx c, int want_res) {
    extern __shared__ __align__(16) int S[];  // the block's record, then its row stage
    __shared__ __align__(8) unsigned long long bar;
    const bool stamp = want_res && c.stamp_lo != nullptr;
    if (stamp && threadIdx.x == 0) stamp_start(c, 0);
    const BusBlk bb = c.bus4_blk[blockIdx.x];
    const StatePtrs X = state<ADJ>(c);
    const bool bulk = c.bus_staged == 1;
    const bool rec_smem = bb.words <= kPoolMax;
    // Bulk schedule with per-block copy lists: the block's list and its done flag sit at its
    // own slot, so they are read together with the block record (hop 1), and the record and
    // the rows arrive together one hop later.  Otherwise the list comes from the record.
    const int* cpl = (LIST && bulk) ? c.bus_cpl + (long long)blockIdx.x * c.bus_cpl_stride : nullptr;
    int cp_n = 0, cp_tx = 0, fdone = 0, cp_rec = 1;
    int cp_e[kCplPerThread][3];
    if (LIST && cpl) {
        cp_n = cpl[0];
        cp_tx = cpl[ADJ ? 2 : 1];
        cp_rec = cpl[3];
        fdone = c.bus_done[blockIdx.x];
#pragma unroll
        for (int j = 0; j < kCplPerThread; ++j) {
            const int k = (int)threadIdx.x + j * kBusQBlock;
            cp_e[j][0] = cp_e[j][1] = cp_e[j][2] = 0;
            if (k < c.bus_cpl_max) {
                cp_e[j][0] = cpl[4 + 3 * k];
                cp_e[j][1] = cpl[4 + 3 * k + 1];
                cp_e[j][2] = cpl[4 + 3 * k + 2];
            }
        }
    }
    const bool fast = LIST && cpl != nullptr && cp_rec == 0;  // a listed block's record fits shared memory
    // hop 2 (record path): the record and the done flag, in flight together
    if (!fast && rec_smem) {
        const int4* src = reinterpret_cast<const int4*>(c.pool + bb.pool);
        int4* dst = reinterpret_cast<int4*>(S);
        for (int k = threadIdx.x; k < (bb.words >> 2); k += kBusQBlock) dst[k] = src[k];
    }
    const int Tq = bb.Tp >> 2;
    const int local = bb.item0 + threadIdx.x;
    const int n = local / Tq;
    const int t = (local - n * Tq) * 4;
    const bool valid = local < bb.nitems;
    const long long i = bb.e_bus + (long long)n * bb.Tp + t;
    const int done = fast ? fdone : c.done[bb.s];
    if (threadIdx.x == 0 && bulk && rec_smem) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        if (fast) {
            mbar_expect_tx(&bar, 4u * (unsigned)bb.words + (unsigned)cp_tx);  // the record and the rows
        } else {
            // the bytes the copies will bring, from the record's header read directly (the
            // staged copy of the record is not there yet)
            const int* hdr = c.pool + bb.pool;
            if (hdr[kPH_SBYTES] > 0) mbar_expect_tx(&bar, (unsigned)hdr[ADJ ? kPH_TXA : kPH_TXF]);
        }
    }
    __syncthreads();
    if (done) return;  // block-uniform: a converged scenario's blocks stop here
    float4* stage = reinterpret_cast<float4*>(S + bb.words);
    if (fast) {
        // hop 2 (list path): the record and every device row segment of the block
        if (threadIdx.x == 0) bulk_g2s(S, c.pool + bb.pool, 4u * (unsigned)bb.words, &bar);
#pragma unroll
        for (int j = 0; j < kCplPerThread; ++j) {
            const int k = (int)threadIdx.x + j * kBusQBlock;
            if (k < cp_n && copy_wanted<ADJ>(cp_e[j][2]))
                bulk_g2s(stage + cp_e[j][1], stage_src<ADJ>(c, X, bb, cp_e[j][2]) + cp_e[j][0],
                         16u * (unsigned)(cp_e[j][2] >> 5), &bar);
        }
    }
    // this thread's bus state, in flight together with the row copies
    float pb[4], uu[4], thold[4], xl[4], Ld[4], al[4];
    if (valid) {
        ld4(X.pbar + i, pb); ld4(X.u + i, uu); ld4(X.thb + i, thold);
        ld4(X.xl + i, xl);
        if (ADJ) ld4(c.al + i, al);  // the adjoint needs the load only through its coefficient
        else ld4(c.load + i, Ld);
    }
    if (fast && !bulk_wait<ADJ>(c, &bar)) return;
    const Pool P{rec_smem ? S : c.pool + bb.pool};
    const int sbytes = P.p[kPH_SBYTES];
    const int qg = P.p[kPH_QG], qe = P.p[kPH_QE];
    // hop 3 (bulk, record path): every device row segment of the block, the copy list split
    // over the warps
    if (!fast && sbytes > 0 && bulk) {
        const int ncp = P.p[kPH_NCP];
        const int* rcpl = P.p + P.p[kPH_CP];
        for (int k = threadIdx.x; k < ncp; k += kBusQBlock) {
            const int rel = rcpl[3 * k], dst = rcpl[3 * k + 1], code = rcpl[3 * k + 2];
            if (!copy_wanted<ADJ>(code)) continue;
            bulk_g2s(stage + dst, stage_src<ADJ>(c, X, bb, code) + rel, 16u * (unsigned)(code >> 5), &bar);
        }
    }
    const int nl = n - bb.n0;
    const int nq = valid ? P.at(kPH_SQ, nl) : 0;
    const int pos = valid ? (int)threadIdx.x - P.at(kPH_SI, nl) : 0;
    const long long gt = bb.e_gen + t;  // generator rows: gt + row * Tp
    const int g0 = valid ? P.at(kPH_GP, nl) : 0, g1 = valid ? P.at(kPH_GP, nl + 1) : 0;
    if (sbytes > 0 && !bulk && valid) {
        // hop 3 (per thread): this thread's own quads of its bus's device rows, 16-byte
        // asynchronous copies into the same stage slots (each thread reads only its own)
        const int sg = P.at(kPH_SG, nl), se = P.at(kPH_SE, nl), sb = P.at(kPH_SB, nl);
        for (int q = g0; q < g1; ++q) {
            const int slot = sg + (q - g0) * nq + pos;
            const long long r = gt + (long long)P.at(kPH_GROW, q) * bb.Tp;
            const int fl = P.at(kPH_GFIRM, q);
            cp_async16(stage + slot, X.xg + r);
            if (!(fl & 2) && (ADJ || !(fl & 1))) cp_async16(stage + qg + slot, (ADJ ? c.ag : c.cf) + r);
        }
        const int e0 = P.at(kPH_EP, nl), e1 = P.at(kPH_EP, nl + 1);
        for (int q = e0; q < e1; ++q) {
            const int e = P.at(kPH_ECODE, q);
            const int slot = se + (q - e0) * nq + pos;
            const long long r = bb.e_line + (long long)(e >> 1) * bb.Tp + t;
            cp_async16(stage + 2 * qg + slot, X.dl + r);
            cp_async16(stage + 2 * qg + qe + slot, ((e & 1) ? X.vt : X.vf) + r);
        }
        const int b0 = P.at(kPH_BP, nl), b1 = P.at(kPH_BP, nl + 1);
        for (int q = b0; q < b1; ++q)
            cp_async16(stage + 2 * qg + 2 * qe + sb + (q - b0) * nq + pos,
                       X.xb + bb.e_bat + (long long)P.at(kPH_BROW, q) * bb.Tp + t);
    }
    if (sbytes > 0 && !bulk) cp_async_wait_all();
    if (!fast && sbytes > 0 && bulk && !bulk_wait<ADJ>(c, &bar)) return;
    float acc[kBusPart] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
        const bool stg = sbytes > 0;
        const float rho = c.rho, eps = c.eps;
        const float inv_re = 1.f / (rho + eps);
        bool hv[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) hv[h] = t + h < bb.T;
        float sum[4] = {0.f, 0.f, 0.f, 0.f}, dx2[4] = {0.f, 0.f, 0.f, 0.f};
        float x2 = 0.f, gscale = 0.f;
        const int e0 = P.at(kPH_EP, nl), e1 = P.at(kPH_EP, nl + 1);
        const int b0 = P.at(kPH_BP, nl), b1 = P.at(kPH_BP, nl + 1);
        const int sg = stg ? P.at(kPH_SG, nl) : 0, se = stg ? P.at(kPH_SE, nl) : 0, sb = stg ? P.at(kPH_SB, nl) : 0;
        for (int q = g0; q < g1; ++q) {
            const int slot = sg + (q - g0) * nq + pos;
            const long long r = gt + (long long)P.at(kPH_GROW, q) * bb.Tp;
            float x[4], a[4], xn[4];
            const bool rampg = RAMP && (P.at(kPH_GFIRM, q) & 2);
            if (stg) {
                const float4 v = stage[slot];
                x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
            } else {
                ld4(X.xg + r, x);
            }
            if (rampg) {
                // ramp-limited: the ramp kernel wrote this iteration's injection (and keeps
                // its own residual terms); the bus only sums it
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    sum[h] += x[h];
                    x2 += x[h] * x[h];
                }
                continue;
            }
            if (ADJ || !(P.at(kPH_GFIRM, q) & 1)) {
                if (stg) {
                    const float4 v = stage[qg + slot];
                    a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
                } else {
                    ld4((ADJ ? c.ag : c.cf) + r, a);
                }
            } else {
                a[0] = a[1] = a[2] = a[3] = 1.f;
            }
            const float gcost = ADJ ? 0.f : P.atf(kPH_GCOST, q);
            const float etag = ADJ ? 0.f : P.atf(kPH_GETA, q);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float v = x[h] - pb[h] - uu[h];
                if (ADJ) {
                    const float gh = a[h];  // NaN: bound active, the variable is fixed at 0
                    const bool fixed = gh != gh;
                    xn[h] = fixed ? 0.f : (rho * v + gh) * inv_re;
                    if (!fixed && hv[h]) gscale += (gh * inv_re) * (gh * inv_re);
                } else {
                    const float cap = a[h] * etag;
                    const float pun = (rho * v - gcost) * inv_re;
                    xn[h] = clampf(pun, 0.f, cap);
                }
                if (!hv[h]) xn[h] = 0.f;
                sum[h] += xn[h];
                dx2[h] += (xn[h] - x[h]) * (xn[h] - x[h]);
                x2 += xn[h] * xn[h];
            }
            st4(X.xg + r, xn);
        }
        {
            float xn[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float v = xl[h] - pb[h] - uu[h];
                if (ADJ) {
                    const float gsh = al[h];  // NaN: bound active, the variable is fixed at 0
                    const bool fixed = gsh != gsh;
                    xn[h] = fixed ? 0.f : (rho * v + gsh) * inv_re;
                    if (!fixed && hv[h]) gscale += (gsh * inv_re) * (gsh * inv_re);
                } else {
                    const float sun = (rho * (v + Ld[h]) - c.voll) * inv_re;
                    xn[h] = clampf(sun, 0.f, Ld[h]) - Ld[h];
                }
                if (!hv[h]) xn[h] = 0.f;
                sum[h] += xn[h];
                dx2[h] += (xn[h] - xl[h]) * (xn[h] - xl[h]);
                x2 += xn[h] * xn[h];
            }
            st4(X.xl + i, xn);
        }
        for (int q = b0; q < b1; ++q) {
            float xb[4];
            if (stg) {
                const float4 v = stage[2 * qg + 2 * qe + sb + (q - b0) * nq + pos];
                xb[0] = v.x; xb[1] = v.y; xb[2] = v.z; xb[3] = v.w;
            } else {
                ld4(X.xb + bb.e_bat + (long long)P.at(kPH_BROW, q) * bb.Tp + t, xb);
            }
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                sum[h] += xb[h];
                x2 += xb[h] * xb[h];
            }
        }
        float ths[4] = {0.f, 0.f, 0.f, 0.f};
        for (int q = e0; q < e1; ++q) {
            const int e = P.at(kPH_ECODE, q);
            float d[4], qv[4];
            if (stg) {
                const int slot = se + (q - e0) * nq + pos;
                const float4 v = stage[2 * qg + slot], w4 = stage[2 * qg + qe + slot];
                d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
                qv[0] = w4.x; qv[1] = w4.y; qv[2] = w4.z; qv[3] = w4.w;
            } else {
                const long long r = bb.e_line + (long long)(e >> 1) * bb.Tp + t;
                ld4(X.dl + r, d);
                ld4((e & 1) ? X.vt + r : X.vf + r, qv);
            }
            const float beta = P.atf(kPH_EBETA, q), w = P.atf(kPH_EW, q);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float pp = (e & 1) ? beta * d[h] : -beta * d[h];
                sum[h] += pp;
                x2 += pp * pp;
                ths[h] += w * qv[h];
            }
        }
        const float icnt = P.atf(kPH_IC, nl), iws = P.atf(kPH_IW, nl), drw = P.atf(kPH_DR, nl);
        const float cnt = 1.f / icnt;
        float pbn[4], un[4], thn[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            pbn[h] = sum[h] * icnt;
            thn[h] = ths[h] * iws;
            un[h] = uu[h] + pbn[h];
            if (hv[h]) {
                const float dpb = pbn[h] - pb[h];
                acc[0] += cnt * pbn[h] * pbn[h];
                acc[2] += dx2[h] - cnt * dpb * dpb;
                acc[3] += (thn[h] - thold[h]) * (thn[h] - thold[h]) * drw;
                acc[4] += cnt * (rho * un[h]) * (rho * un[h]);
            }
        }
        acc[1] = gscale;
        acc[5] = x2;
        st4(X.pbar + i, pbn);
        st4(X.u + i, un);
        st4(X.thb + i, thn);
    }
    if (want_res) {
        __shared__ float sh[kBusPart][kBusQBlock / 32];
        block_sum<kBusPart, kBusQBlock>(acc, sh);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < kBusPart; ++q) c.bus_part[blockIdx.x * kBusPart + q] = acc[q];
            if (stamp) stamp_end(c, 0);
        }
    }
}

// Write each generator's plan value max(eta_g, 0) into the pool records (once per call).
__global__ void k_prep(const Ctx c) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < c.n_prep) {
        const int2 e = c.prep[k];
        c.pool[e.x] = __float_as_int(fmaxf(c.eta[e.y], 0.f));
    }
}

// ------------------------------------------------------------------------------------
// Per-scenario residuals in FP64 and the convergence flags.
//   primal = sqrt(sum_n |n| pbar^2 + sum_j beta_j^2 (th_j - thbar)^2) / scale
//            (scale = |L|_2 forward, |x|_2 adjoint)
//   dual   = sqrt(rho^2 |z^k - z^{k-1}|^2 + sum_j (rho_th_j dthbar / beta_j)^2) / |rho u|_2
// ------------------------------------------------------------------------------------
// Chunk start: advance the loop's device iteration counter by one chunk (one thread), and
// refresh the staged bus kernel's per-block done flags from the scenario flags (which change
// only at the reductions that end chunks, or between calls).
__global__ void k_tick(const Ctx c, int chunk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *c.iter_ctr += chunk;
    for (int b = i; b < c.n_bus4_blk; b += gridDim.x * blockDim.x) c.bus_done[b] = c.done[c.bus4_blk[b].s];
}

__global__ void __launch_bounds__(kBlock) k_reduce(const Ctx c, int adj, double tol) {
    const int s = blockIdx.x;
    if (c.done[s]) return;
    if (*c.err != 0) {  // a bounded wait in this chunk gave up: stop with its status
        if (threadIdx.x == 0) {
            c.status[s] = *c.err;
            c.done[s] = 1;
            (adj ? c.adj_iters : c.iters)[s] = *c.iter_ctr;
        }
        return;
    }
    // timing on: the chunk's sampled iteration worked for this scenario
    if (c.prof_act != nullptr && threadIdx.x == 0) c.prof_act[s] += 1;
    const int it = *c.iter_ctr;
    const int final_ = it >= c.max_it;
    const ScenDev sc = c.scen[s];
    double a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < sc.bus4_nblk; b += kBlock) {
#pragma unroll
        for (int q = 0; q < kBusPart; ++q) a[q] += (double)c.bus_part[(sc.bus4_blk0 + b) * kBusPart + q];
    }
    for (int b = threadIdx.x; b < sc.line4_nblk; b += kBlock) {
#pragma unroll
        for (int q = 0; q < kDevPart; ++q) a[6 + q] += (double)c.line_part[(sc.line4_blk0 + b) * kDevPart + q];
    }
    for (int b = threadIdx.x; b < sc.B; b += kBlock) {
#pragma unroll
        for (int q = 0; q < kDevPart; ++q) a[6 + q] += (double)c.bat_part[(sc.bat_w0 + b) * kDevPart + q];
    }
    for (int b = threadIdx.x; b < sc.R; b += kBlock) {  // ramping generators: dx^2, x^2, adjoint scale
        const float* rp = c.ramp_part + (long long)(sc.ramp_w0 + b) * kDevPart;
        a[6] += (double)rp[0];
        a[7] += (double)rp[1];
        a[1] += (double)rp[2];
    }
    __shared__ double sh[9][kBlock / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const double v = warp_sum_d(a[q]);
        if (lane == 0) sh[q][w] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            double v = 0;
            for (int k = 0; k < kBlock / 32; ++k) v += sh[q][k];
            a[q] = v;
        }
        // a: 0 |n| pbar^2, 1 adjoint scale, 2 bus dz^2, 3 dthbar^2 w, 4 |rho u|^2, 5 bus x^2,
        //    6 device dx^2, 7 device x^2, 8 phase mismatch (line kernel, one iteration lagged)
        const double rho = c.rho, rth = c.rth_c;
        // a NaN or inf anywhere in the iterate reaches these sums; test them before the
        // clamps below, which would turn a NaN into 0 (fmax returns its other argument)
        bool finite = true;
#pragma unroll
        for (int q = 0; q < 9; ++q) finite = finite && isfinite(a[q]);
        const double scale = adj ? fmax(sqrt(a[1]), 1e-30) : sc.load_norm;
        const double rp = sqrt(fmax(a[0] + a[8], 0.0)) / scale;
        const double dz2 = fmax(a[2] + a[6], 0.0);
        const double rd = sqrt(rho * rho * dz2 + rth * rth * a[3]) / fmax(sqrt(a[4]), 1e-30);
        c.resid[2 * s + 0] = rp;
        c.resid[2 * s + 1] = rd;
        const double r = fmax(rp, rd);
        double* best = c.rbest + s;
        if (it <= c.check_every || !(r >= *best)) *best = r;
        int* itp = adj ? c.adj_iters : c.iters;
        if (!finite || !isfinite(rp) || !isfinite(rd) || r > 1e6 * *best) {
            // non-finite or diverged by six orders of magnitude from the best residual seen
            c.status[s] = GX_ERR_NONFINITE;
            c.done[s] = 1;
            itp[s] = it;
        } else if (rp <= tol && rd <= tol) {
            c.status[s] = GX_OK;
            c.done[s] = 1;
            itp[s] = it;
        } else if (final_) {
            c.status[s] = GX_NOT_CONVERGED;
            c.done[s] = 1;
            itp[s] = it;
        } else {
            atomicAdd(c.n_active, 1);
        }
    }
}

// Outputs after a forward solve: price = -rho u, shed = x_load + L, flow = beta delta.
__global__ void __launch_bounds__(kBlock) k_extract(const Ctx c) {
    if (blockIdx.x < c.n_bus_blk) {
        const int blk = blockIdx.x;
        const int s = c.bus_blk_scen[blk];
        const ScenDev sc = c.scen[s];
        const int local = (blk - sc.bus_blk0) * kBlock + threadIdx.x;
        if (local >= sc.N * sc.Tp) return;
        const long long i = sc.e_bus + local;
        c.out_price[i] = -c.rho * c.u[i];
        c.out_shed[i] = c.xl[i] + c.load[i];
    } else {
        const int blk = blockIdx.x - c.n_bus_blk;
        const int s = c.line_blk_scen[blk];
        const ScenDev sc = c.scen[s];
        for (int r = 0; r < kLineItems; ++r) {
            const int local = (blk - sc.line_blk0) * kBlock * kLineItems + r * kBlock + threadIdx.x;
            if (local >= sc.L * sc.Tp) return;
            const int l = local / sc.Tp;
            const long long i = sc.e_line + local;
            c.out_flow[i] = c.l_beta[sc.line0 + l] * c.dl[i];
        }
    }
}

// Operating cost c_s (Eq. 2 objective with the eps terms) and emissions, FP64.
__global__ void __launch_bounds__(kBlock) k_cost(const Ctx c, const int* in_batch) {
    const int blk = blockIdx.x;
    const int s = c.cost_blk_scen[blk];
    const ScenDev sc = c.scen[s];
    double cs = 0.0, em = 0.0;
    if (in_batch[s]) {
        const int nb = blk - sc.cost_blk0;
        const int nblk = (s + 1 < c.S ? c.scen[s + 1].cost_blk0 : c.n_cost_blk) - sc.cost_blk0;
        cost_share(c, sc, (long long)nb * kBlock + threadIdx.x, (long long)nblk * kBlock, cs, em);
    }
    cs = warp_sum_d(cs);
    em = warp_sum_d(em);
    __shared__ double sh[2][kBlock / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sh[0][w] = cs; sh[1][w] = em; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int k = 0; k < kBlock / 32; ++k) { a += sh[0][k]; b += sh[1][k]; }
        c.cost_part[2 * blk] = a;
        c.cost_part[2 * blk + 1] = b;
    }
}

__global__ void k_cost_final(const Ctx c, const int* in_batch) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= c.S || !in_batch[s]) return;
    const int b0 = c.scen[s].cost_blk0;
    const int b1 = s + 1 < c.S ? c.scen[s + 1].cost_blk0 : c.n_cost_blk;
    double a = 0, e = 0;
    for (int b = b0; b < b1; ++b) { a += c.cost_part[2 * b]; e += c.cost_part[2 * b + 1]; }
    c.cost[s] = a;
    c.hval[s] = a + (double)c.kappa * e;
}

// ------------------------------------------------------------------------------------
// GX_WARM_LEARNED: after one residual-check chunk from the previous plan's state (saved,
// with its flags) and one from the learned start, each scenario keeps the start whose
// residual at that check is smaller; the losers get the saved state and flags back.
// ------------------------------------------------------------------------------------
__global__ void k_warm_choose(const Ctx c, const int* in_batch, const int* sdone, const int* sstatus,
                              const int* siters, const double* sres, int* chosen) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= c.S) return;
    if (!in_batch[s]) { chosen[s] = -1; return; }
    const double rp = fmax(sres[2 * s], sres[2 * s + 1]);
    const double rl = fmax(c.resid[2 * s], c.resid[2 * s + 1]);
    // a scenario the previous plan's chunk already finished skipped the learned trial
    const int keep = !sdone[s] && rl < rp;
    chosen[s] = keep;
    if (!keep) {
        c.done[s] = sdone[s];
        c.status[s] = sstatus[s];
        c.iters[s] = siters[s];
        c.resid[2 * s] = sres[2 * s];
        c.resid[2 * s + 1] = sres[2 * s + 1];
        c.rbest[s] = rp;
    }
}

// Rows of scenario s in forward state array a, copied back from the saved state when the
// previous plan's start won.  Grid (S, arrays).
__global__ void k_warm_restore(const Ctx c, WarmArrays w, float* state, const float* saved, const int* chosen,
                               const int* sdone) {
    const int s = blockIdx.x, a = blockIdx.y;
    if (chosen[s] != 0 || sdone[s]) return;  // learned kept, outside the batch, or untouched
    const ScenDev sc = c.scen[s];
    long long e0 = 0, n = 0;
    switch (w.kind[a]) {
        case 0: e0 = sc.e_gen; n = (long long)sc.G * sc.Tp; break;
        case 1: e0 = sc.e_bus; n = (long long)sc.N * sc.Tp; break;
        case 2: e0 = sc.e_line; n = (long long)sc.L * sc.Tp; break;
        case 3: e0 = sc.e_bat; n = (long long)sc.B * sc.Tp; break;
        default: e0 = sc.e_ramp; n = (long long)sc.R * sc.Tp; break;
    }
    const long long base = w.off[a] + e0;
    for (long long k = threadIdx.x; k < n; k += blockDim.x) state[base + k] = saved[base + k];
}

// Eq. 1's operating term over the batch: sum_s w'_s h_s in FP64, summed by one thread in
// scenario order so the value does not depend on the launch shape.
__global__ void k_objective(const Ctx c, const double* wprime, double* obj) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0;
    for (int s = 0; s < c.S; ++s)
        if (wprime[s] != 0.0) a += wprime[s] * c.hval[s];
    *obj = a;
}

// ------------------------------------------------------------------------------------
// Gradient assembly: dh_s/deta_k = sum over active upper bounds i of device k of
// xi_i * d b_i / d eta_k (gen: cf_t, line flow: 1, battery charge/discharge: 1, soc: dur).
// xi comes from the adjoint prox at its fixed point (or, for h = c, from the forward
// prox: the envelope theorem).  One warp per (scenario, device); FP64 sums.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_grad(const Ctx c, int envelope, const int* gwarp_scen,
                                                 int n_gwarps, const int* in_batch) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
    if (gw >= n_gwarps) return;
    const int s = gwarp_scen[2 * gw];
    const int r = gwarp_scen[2 * gw + 1];
    if (!in_batch[s]) return;
    const ScenDev sc = c.scen[s];
    const float rho = c.rho, eps = c.eps;
    double acc = 0.0;
    if (r < sc.G && c.g_ramp[sc.gen0 + r] >= 0) {
        // ramp-limited generator: multipliers of its inner box copy (capacity, dcap/deta =
        // cf) and ramp copy (+-(p_t - p_{t-1}) <= rate eta, both bounds move with eta)
        const int g = r, gg = sc.gen0 + g;
        const int rk = c.g_ramp[gg];
        const float rate = c.r_rate[sc.ramp0 + rk];
        const long long row0 = sc.e_ramp + (long long)rk * sc.Tp;
        for (int t = lane; t < sc.T; t += 32) {
            const long long rr = sc.e_gen + (long long)g * sc.Tp + t;
            const uint8_t m = c.m_gen[rr];
            const float yv = envelope ? -c.ry[row0 + t] : c.a_ry[row0 + t];
            const float qv = envelope ? -c.rq[row0 + t] : c.a_rq[row0 + t];
            const float cf = c.g_firm[gg] ? 1.f : c.cf[rr];
            if ((m & 3) == A_UP) acc += (double)yv * (double)cf;
            const int rm = (m >> 2) & 3;
            if (rm == A_UP) acc += (double)qv * (double)rate;
            else if (rm == A_LO) acc -= (double)qv * (double)rate;
        }
    } else if (r < sc.G) {
        const int g = r, gg = sc.gen0 + g;
        const int bus = c.g_bus[gg];
        const float cost = c.g_cost[gg];
        for (int t = lane; t < sc.T; t += 32) {
            const long long rr = sc.e_gen + (long long)g * sc.Tp + t;
            if (c.m_gen[rr] != A_UP) continue;
            const long long bi = sc.e_bus + (long long)bus * sc.Tp + t;
            const float cf = c.g_firm[gg] ? 1.f : c.cf[rr];
            const float p = c.xg[rr];
            float xi;
            if (envelope) {
                const float v = p - c.pbar[bi] - c.u[bi];
                xi = -(rho * (v - p) - cost - eps * p);
            } else {
                const float v = c.a_xg[rr] - c.a_pbar[bi] - c.a_u[bi];
                xi = cost + eps * p + c.kappa * c.g_emis[gg] + rho * v;
            }
            acc += (double)xi * (double)cf;
        }
    } else if (r < sc.G + sc.L) {
        const int l = r - sc.G, lg = sc.line0 + l;
        const int f = c.l_from[lg], to = c.l_to[lg];
        const float beta = c.l_beta[lg];
        const float rth = c.rth_c * c.l_w[lg];
        for (int t = lane; t < sc.T; t += 32) {
            const long long rr = sc.e_line + (long long)l * sc.Tp + t;
            const uint8_t m = c.m_line[rr];
            if (m != AL_FUP && m != AL_FLO) continue;
            const long long bf = sc.e_bus + (long long)f * sc.Tp + t;
            const long long bt = sc.e_bus + (long long)to * sc.Tp + t;
            const float* dl = envelope ? c.dl : c.a_dl;
            const float* vfp = envelope ? c.vf : c.a_vf;
            const float* vtp = envelope ? c.vt : c.a_vt;
            const float* pb = envelope ? c.pbar : c.a_pbar;
            const float* uu = envelope ? c.u : c.a_u;
            const float* th = envelope ? c.thb : c.a_thb;
            const float d = dl[rr];
            const float vf = vfp[rr] - th[bf];  // v = q - z
            const float vt = vtp[rr] - th[bt];
            const float wf = th[bf] - vf, wt = th[bt] - vt;
            const float tf = -beta * d - pb[bf] - uu[bf];
            const float tt = beta * d - pb[bt] - uu[bt];
            // derivative of the line prox objective in delta at the frozen delta (a transport
            // line adds eps/2 f^2, and in the adjoint the linear term -eps f*)
            const float dstar = envelope ? d : 0.f;
            const bool dc = c.l_w[sc.line0 + l] == 0.f;
            const float Fdc = dc ? c.eps * (envelope ? dstar : -c.dl[rr]) : 0.f;
            const float Fp = rho * beta * (beta * dstar + tf) + rho * beta * (beta * dstar - tt) +
                             0.5f * rth * (dstar - (wf - wt)) + Fdc;
            float xi;
            if (envelope) xi = (m == AL_FUP) ? Fp / beta : -Fp / beta;
            else xi = (m == AL_FUP) ? -Fp / beta : Fp / beta;
            acc += (double)xi;
        }
    } else {
        const int b = r - sc.G - sc.L, bg = sc.bat0 + b;
        const float dur = c.b_dur[bg];
        for (int t = lane; t < sc.T; t += 32) {
            const long long rr = sc.e_bat + (long long)b * sc.Tp + t;
            const uint8_t m = c.m_bat[rr];
            const float y3[3] = {envelope ? -c.yc[rr] : c.a_yc[rr], envelope ? -c.yd[rr] : c.a_yd[rr],
                                 envelope ? -c.ys[rr] : c.a_ys[rr]};
            const float dbd[3] = {1.f, 1.f, dur};
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (((m >> (2 * q)) & 3) == A_UP) acc += (double)y3[q] * (double)dbd[q];
        }
    }
    acc = warp_sum_d(acc);
    if (lane == 0) c.grad_s[sc.gs0 + r] = acc;
}

// grad[k] = sum_s w'_s grad_s[k] over the scenarios of k's network.
__global__ void k_grad_combine(const Ctx c, const double* wprime, const int* k_net, float* out, int K) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int net = k_net[k];
    double acc = 0.0;
    for (int s = 0; s < c.S; ++s) {
        const ScenDev& sc = c.scen[s];
        if (sc.net != net || wprime[s] == 0.0) continue;
        acc += wprime[s] * c.grad_s[sc.gs0 + (k - sc.eta0)];
    }
    out[k] = (float)acc;
}

__global__ void k_plan_step(float* eta, const float* grad, const float* gamma, const float* lo, const float* hi,
                            float alpha, int K) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const float e = eta[k] - alpha * (gamma[k] + grad[k]);
    eta[k] = fminf(fmaxf(e, lo[k]), hi[k]);
}

// ------------------------------------------------------------------------------------
// launch wrappers
// ------------------------------------------------------------------------------------

// Setup modes (reset, start, active set) of the single-hour kernels.
#define GX_DISPATCH_MODE_SETUP(KERNEL, GRID, ...)                                        \
    do {                                                                                 \
        if (adj) {                                                                       \
            if (mode == M_RESET) KERNEL<M_RESET, 1><<<GRID, kBlock, 0, st>>>(__VA_ARGS__);      \
            else if (mode == M_INIT) KERNEL<M_INIT, 1><<<GRID, kBlock, 0, st>>>(__VA_ARGS__);   \
        } else {                                                                         \
            if (mode == M_RESET) KERNEL<M_RESET, 0><<<GRID, kBlock, 0, st>>>(__VA_ARGS__);      \
            else if (mode == M_INIT) KERNEL<M_INIT, 0><<<GRID, kBlock, 0, st>>>(__VA_ARGS__);   \
            else if (mode == M_MASK) KERNEL<M_MASK, 0><<<GRID, kBlock, 0, st>>>(__VA_ARGS__);   \
        }                                                                                \
    } while (0)

int launch_line(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st) {
    if (mode == M_INIT || c.n_line_blk <= 0) return 0;
    if (mode == M_FWD || mode == M_ADJ) {
        if (adj) k_line4<1><<<c.n_line4_blk, kQBlock, 0, st>>>(c, want_res);
        else k_line4<0><<<c.n_line4_blk, kQBlock, 0, st>>>(c, want_res);
        return 1;
    }
    GX_DISPATCH_MODE_SETUP(k_line, c.n_line_blk, c, want_res);
    return 1;
}

#define GX_DISPATCH_MODE_BS(KERNEL, GRID, BS, ...)                                        \
    do {                                                                                    \
        if (adj) {                                                                          \
            if (mode == M_ADJ) KERNEL<M_ADJ, 1><<<GRID, BS, 0, st>>>(__VA_ARGS__);           \
            else if (mode == M_RESET) KERNEL<M_RESET, 1><<<GRID, BS, 0, st>>>(__VA_ARGS__);  \
        } else {                                                                            \
            if (mode == M_FWD) KERNEL<M_FWD, 0><<<GRID, BS, 0, st>>>(__VA_ARGS__);           \
            else if (mode == M_RESET) KERNEL<M_RESET, 0><<<GRID, BS, 0, st>>>(__VA_ARGS__);  \
            else if (mode == M_MASK) KERNEL<M_MASK, 0><<<GRID, BS, 0, st>>>(__VA_ARGS__);    \
        }                                                                                   \
    } while (0)

#define GX_BAT_HPL(H)                                                                      \
    do {                                                                                   \
        if (adj) {                                                                         \
            if (mode == M_ADJ) k_bat<M_ADJ, 1, H, 1><<<grid, kBatWarps * 32, 0, st>>>(c, want_res);          \
            else if (mode == M_RESET) k_bat<M_RESET, 1, H, 1><<<grid, kBatWarps * 32, 0, st>>>(c, want_res); \
        } else {                                                                           \
            if (mode == M_FWD) k_bat<M_FWD, 0, H, 1><<<grid, kBatWarps * 32, 0, st>>>(c, want_res);          \
            else if (mode == M_RESET) k_bat<M_RESET, 0, H, 1><<<grid, kBatWarps * 32, 0, st>>>(c, want_res); \
            else if (mode == M_MASK) k_bat<M_MASK, 0, H, 1><<<grid, kBatWarps * 32, 0, st>>>(c, want_res);   \
        }                                                                                  \
    } while (0)

// Hours per lane: compiled for 1, 2, 3 hours with one warp per battery (T up to 96) and
// for 3 or 4 hours with two warps per battery in the iterations (T up to 192 or 256),
// chosen from the longest horizon among the batch's batteries.  The setup modes use one
// warp per battery (hour-strided loops).
int launch_bat(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st) {
    if (mode == M_INIT || c.n_bat_warps <= 0) return 0;
    const int grid = (c.n_bat_warps + kBatWarps - 1) / kBatWarps;
    const int hpl = (c.max_bat_T + 31) / 32;
    if ((mode == M_FWD || mode == M_ADJ) && hpl > 3 && c.bat_warps == 2) {
        const int grid2 = c.n_bat_warps;  // one battery (two warps) per block
        const int h2 = (c.max_bat_T + 63) / 64;
        if (adj) {
            if (h2 <= 3) k_bat<M_ADJ, 1, 3, 2><<<grid2, kBatWarps * 32, 0, st>>>(c, want_res);
            else k_bat<M_ADJ, 1, 4, 2><<<grid2, kBatWarps * 32, 0, st>>>(c, want_res);
        } else {
            if (h2 <= 3) k_bat<M_FWD, 0, 3, 2><<<grid2, kBatWarps * 32, 0, st>>>(c, want_res);
            else k_bat<M_FWD, 0, 4, 2><<<grid2, kBatWarps * 32, 0, st>>>(c, want_res);
        }
        return 1;
    }
    if (hpl <= 1) GX_BAT_HPL(1);
    else if (hpl <= 2) GX_BAT_HPL(2);
    else if (hpl <= 3) GX_BAT_HPL(3);
    else if (hpl <= 6) GX_BAT_HPL(6);
    else GX_BAT_HPL(8);
    return 1;
}

int launch_dev(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st) {
    return launch_line(c, mode, adj, want_res, st) + launch_bat(c, mode, adj, want_res, st) +
           launch_ramp(c, mode, adj, want_res, st);
}

int launch_bus(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st) {
    if (c.n_bus_blk <= 0) return 0;
    if (mode == M_FWD || mode == M_ADJ) {
        const int sm = c.bus4_smem;
        if (c.bus_staged != 0) {
            const bool list = c.bus_staged == 1 && c.bus_cpl != nullptr;
#define GX_BUS4T(A, R)                                                                  \
    do {                                                                                \
        if (list) k_bus4t<A, R, 1><<<c.n_bus4_blk, kBusQBlock, sm, st>>>(c, want_res);  \
        else k_bus4t<A, R, 0><<<c.n_bus4_blk, kBusQBlock, sm, st>>>(c, want_res);       \
    } while (0)
            if (c.n_ramp_warps > 0) {
                if (adj) GX_BUS4T(1, 1);
                else GX_BUS4T(0, 1);
            } else {
                if (adj) GX_BUS4T(1, 0);
                else GX_BUS4T(0, 0);
            }
#undef GX_BUS4T
        } else if (c.n_ramp_warps > 0) {
            if (adj) k_bus4<1, 1><<<c.n_bus4_blk, kBusQBlock, 0, st>>>(c, want_res);
            else k_bus4<0, 1><<<c.n_bus4_blk, kBusQBlock, 0, st>>>(c, want_res);
        } else {
            if (adj) k_bus4<1, 0><<<c.n_bus4_blk, kBusQBlock, 0, st>>>(c, want_res);
            else k_bus4<0, 0><<<c.n_bus4_blk, kBusQBlock, 0, st>>>(c, want_res);
        }
        return 1;
    }
    GX_DISPATCH_MODE_SETUP(k_bus, c.n_bus_blk, c, want_res);
    return 1;
}

cudaError_t bus_staged_prepare(int smem) {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    };
    set((const void*)k_bus4t<0, 0, 0>);
    set((const void*)k_bus4t<1, 0, 0>);
    set((const void*)k_bus4t<0, 1, 0>);
    set((const void*)k_bus4t<1, 1, 0>);
    set((const void*)k_bus4t<0, 0, 1>);
    set((const void*)k_bus4t<1, 0, 1>);
    set((const void*)k_bus4t<0, 1, 1>);
    set((const void*)k_bus4t<1, 1, 1>);
    return e;
}

int launch_prep(const Ctx& c, cudaStream_t st) {
    if (c.n_prep <= 0) return 0;
    k_prep<<<(c.n_prep + kBlock - 1) / kBlock, kBlock, 0, st>>>(c);
    return 1;
}

int launch_reduce(const Ctx& c, int adj, double tol, cudaStream_t st) {
    k_reduce<<<c.S, kBlock, 0, st>>>(c, adj, tol);
    return 1;
}

int launch_tick(const Ctx& c, int chunk, cudaStream_t st) {
    int grid = (c.n_bus4_blk + kBlock - 1) / kBlock;
    grid = grid < 1 ? 1 : grid > 256 ? 256 : grid;
    k_tick<<<grid, kBlock, 0, st>>>(c, chunk);
    return 1;
}

int launch_extract(const Ctx& c, const int* in_batch, cudaStream_t st) {
    const int grid = c.n_bus_blk + c.n_line_blk;
    k_extract<<<grid, kBlock, 0, st>>>(c);
    k_cost<<<c.n_cost_blk, kBlock, 0, st>>>(c, in_batch);
    k_cost_final<<<(c.S + 127) / 128, 128, 0, st>>>(c, in_batch);
    return 3;
}

int launch_warm_select(const Ctx& c, const WarmArrays& w, float* state, const float* saved, const int* in_batch,
                       const int* sdone, const int* sstatus, const int* siters, const double* sres, int* chosen,
                       cudaStream_t st) {
    k_warm_choose<<<(c.S + 127) / 128, 128, 0, st>>>(c, in_batch, sdone, sstatus, siters, sres, chosen);
    k_warm_restore<<<dim3(c.S, w.n), 256, 0, st>>>(c, w, state, saved, chosen, sdone);
    return 2;
}

int launch_objective(const Ctx& c, const double* wprime, double* obj, cudaStream_t st) {
    k_objective<<<1, 32, 0, st>>>(c, wprime, obj);
    return 1;
}

int launch_grad(const Ctx& c, int envelope, const int* gwarp_scen, int n_gwarps, const int* in_batch,
                cudaStream_t st) {
    const int grid = (n_gwarps + kBlock / 32 - 1) / (kBlock / 32);
    if (grid > 0) k_grad<<<grid, kBlock, 0, st>>>(c, envelope, gwarp_scen, n_gwarps, in_batch);
    return 1;
}

int launch_grad_combine(const Ctx& c, const double* wprime, const int* k_net, float* grad_out, int K,
                        cudaStream_t st) {
    k_grad_combine<<<(K + 255) / 256, 256, 0, st>>>(c, wprime, k_net, grad_out, K);
    return 1;
}

int launch_plan_step(float* eta, const float* grad, const float* gamma, const float* lo, const float* hi, float alpha,
                     int K, cudaStream_t st) {
    k_plan_step<<<(K + 255) / 256, 256, 0, st>>>(eta, grad, gamma, lo, hi, alpha, K);
    return 1;
}

}  // namespace gx
