// Prox of ramp-limited generators: one warp per generator per outer iteration.
//
// A generator with |p_t - p_{t-1}| <= R (R = r eta_g) couples its hours, so its prox is a
// small banded QP over the horizon instead of a clip:
//   min_p  sum_t lin_t p_t + eps/2 p_t^2 + rho/2 (p_t - v_t)^2
//   s.t.   0 <= p_t <= cap_t,  -R <= p_t - p_{t-1} <= R  (t >= 1)
// (forward: lin = c; adjoint: lin = -(c + eps p* + kappa e) and the active bounds fixed at
// 0, the free ones dropped).  It is solved like the battery prox, by a warm-started inner
// ADMM with the box copy z_t = p_t and the ramp copy w_t = p_t - p_{t-1}; the x-step
//   (eps + rho + rho_in) p + rho_in D^T D p = rhs,  D the first difference,
// is a constant tridiagonal system whose Thomas pivots come from the host, and its two
// sweeps are first-order recurrences evaluated with warp affine scans (each lane owns a
// contiguous chunk of hours).  The generator's injection goes to its usual row of the
// generator state, where the bus kernel sums it without a prox of its own.
#include "gx_internal.cuh"

#include <cfloat>

namespace gx {

namespace {

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct RampPtrs {
    float *xg, *u, *pbar, *z, *w, *y, *q;
};

template <int ADJ>
__device__ __forceinline__ RampPtrs ramp_state(const Ctx& c) {
    if (ADJ) return RampPtrs{c.a_xg, c.a_u, c.a_pbar, c.a_rz, c.a_rw, c.a_ry, c.a_rq};
    return RampPtrs{c.xg, c.u, c.pbar, c.rz, c.rw, c.ry, c.rq};
}

}  // namespace

template <int MODE, int ADJ, int kHpl>
__global__ void __launch_bounds__(kBatWarps * 32) k_ramp(const Ctx c, int want_res) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kBatWarps + (threadIdx.x >> 5);
    if (gw >= c.n_ramp_warps) return;
    const bool stamp = (MODE == M_FWD || MODE == M_ADJ) && want_res && c.stamp_lo != nullptr;
    if (stamp && lane == 0) stamp_start(c, 2);
    const int s = c.ramp_warp_scen[gw];
    if (c.done[s]) return;
    const ScenDev sc = c.scen[s];
    const RampPtrs X = ramp_state<ADJ>(c);
    const int r = gw - sc.ramp_w0;                 // ramping generator within the network
    const int g = c.r_gen[sc.ramp0 + r];           // its generator index within the network
    const int gg = sc.gen0 + g;
    const int T = sc.T;
    const int hpl = (T + 31) >> 5;
    const int t0 = lane * hpl;
    const long long row0 = sc.e_ramp + (long long)r * sc.Tp;    // ramp state rows
    const long long grow0 = sc.e_gen + (long long)g * sc.Tp;    // generator rows
    const long long brow0 = sc.e_bus + (long long)c.g_bus[gg] * sc.Tp;
    if (MODE == M_RESET) {
        const bool neg = ADJ && c.adj_from_fwd;
        for (int t = lane; t < sc.Tp; t += 32) {
            const long long rr = row0 + t;
            X.z[rr] = 0.f; X.w[rr] = 0.f;
            // h = c part of the adjoint: bound multipliers are the negated forward ones
            X.y[rr] = neg ? -c.ry[rr] : 0.f;
            X.q[rr] = neg ? -c.rq[rr] : 0.f;
        }
        return;
    }
    if (MODE == M_MASK) {
        // active set from the inner multipliers of the forward solution: box code in bits
        // 0-1, ramp code (hour t's difference p_t - p_{t-1}) in bits 2-3
        for (int t = lane; t < T; t += 32) {
            const long long rr = row0 + t;
            const float yv = c.ry[rr], qv = t > 0 ? c.rq[rr] : 0.f;
            uint8_t box = A_FREE, rmp = A_FREE;
            if (yv > c.tol_act) box = A_UP;
            else if (yv < -c.tol_act) box = A_LO;
            if (qv > c.tol_act) rmp = A_UP;
            else if (qv < -c.tol_act) rmp = A_LO;
            c.m_gen[grow0 + t] = (uint8_t)(box | (rmp << 2));
        }
        return;
    }
    const float rho = c.rho, eps = c.eps, ri = c.rho_in, iri = 1.f / c.rho_in;
    const float inv_re = 1.f / (rho + eps);
    const float etag = fmaxf(c.eta[sc.eta0 + g], 0.f);
    const float R = c.r_rate[sc.ramp0 + r] * etag;
    const bool firm = c.g_firm[gg] != 0;
    const float gcost = c.g_cost[gg], gemis = c.g_emis[gg];

    // per hour of the lane's chunk; hours past the horizon read hour T-1 and are zeroed
    float v[kHpl], z[kHpl], w[kHpl], y[kHpl], q[kHpl], lin[kHpl], cap[kHpl], ba[kHpl], fa[kHpl], x_old[kHpl];
    int mk[kHpl];
#pragma unroll
    for (int j = 0; j < kHpl; ++j) {
        const int t = t0 + j;
        const bool ok = (j < hpl) && (t < T);
        const int tc = ok ? t : T - 1;
        const long long rr = row0 + tc, gr = grow0 + tc;
        x_old[j] = X.xg[gr];
        v[j] = x_old[j] - X.pbar[brow0 + tc] - X.u[brow0 + tc];
        z[j] = X.z[rr]; w[j] = X.w[rr]; y[j] = X.y[rr]; q[j] = X.q[rr];
        ba[j] = c.ramp_dd[rr];
        fa[j] = c.ramp_dd[tc > 0 ? rr - 1 : rr];
        cap[j] = firm ? etag : c.cf[gr] * etag;
        mk[j] = 0;
        if (ADJ) {
            mk[j] = c.m_gen[gr];
            lin[j] = -(gcost + eps * c.xg[gr] + c.kappa * gemis);
        } else {
            lin[j] = gcost;
        }
    }
#pragma unroll
    for (int j = 0; j < kHpl; ++j) {
        const int t = t0 + j;
        const bool ok = (j < hpl) && (t < T);
        fa[j] = (ok && t > 0) ? ri * fa[j] : 0.f;  // rho_in / m_{t-1}
        if (!ok) {
            v[j] = z[j] = w[j] = y[j] = q[j] = lin[j] = cap[j] = ba[j] = x_old[j] = 0.f;
            mk[j] = 0;
        }
        if (ok && t == 0) { w[j] = 0.f; q[j] = 0.f; }  // no ramp term before the first hour
    }

    float px[kHpl];  // x-step (the generator's injection) of the last inner iteration
#pragma unroll
    for (int j = 0; j < kHpl; ++j) px[j] = 0.f;
    for (int it = 0; it < c.inner_iters; ++it) {
        // rhs = rho v - lin + rho_in z - y + D^T s,  s_t = rho_in w_t - q_t (t >= 1), so
        // hour t receives s_t - s_{t+1}; the chunk's last hour reads the next lane's first s
        float sv[kHpl], rhs[kHpl];
#pragma unroll
        for (int j = 0; j < kHpl; ++j) sv[j] = ri * w[j] - q[j];
        float s_next = __shfl_down_sync(0xffffffffu, sv[0], 1);
        if (lane == 31) s_next = 0.f;
        float A = 1.f, Bv = 0.f;
#pragma unroll
        for (int j = 0; j < kHpl; ++j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            float sn = (j + 1 < hpl) ? sv[j + 1 < kHpl ? j + 1 : j] : s_next;
            if (t + 1 >= T) sn = 0.f;
            rhs[j] = ok ? rho * v[j] - lin[j] + ri * z[j] - y[j] + sv[j] - sn : 0.f;
            // forward sweep b'_t = rhs_t + (rho_in / m_{t-1}) b'_{t-1}
            if (ok) { A = fa[j] * A; Bv = fa[j] * Bv + rhs[j]; }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float Ao = __shfl_up_sync(0xffffffffu, A, o);
            const float Bo = __shfl_up_sync(0xffffffffu, Bv, o);
            if (lane >= o) { Bv = A * Bo + Bv; A = A * Ao; }
        }
        float bin = __shfl_up_sync(0xffffffffu, Bv, 1);
        if (lane == 0) bin = 0.f;
        float bp[kHpl];
#pragma unroll
        for (int j = 0; j < kHpl; ++j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            if (ok) bin = fa[j] * bin + rhs[j];
            bp[j] = bin;
        }
        // backward sweep p_t = (b'_t + rho_in p_{t+1}) / m_t, p_T = 0
        A = 1.f; Bv = 0.f;
#pragma unroll
        for (int j = kHpl - 1; j >= 0; --j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            if (ok) { const float gj = ri * ba[j]; A = gj * A; Bv = gj * Bv + ba[j] * bp[j]; }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float Ao = __shfl_down_sync(0xffffffffu, A, o);
            const float Bo = __shfl_down_sync(0xffffffffu, Bv, o);
            if (lane + o < 32) { Bv = A * Bo + Bv; A = A * Ao; }
        }
        float pn = __shfl_down_sync(0xffffffffu, Bv, 1);
        if (lane == 31) pn = 0.f;
#pragma unroll
        for (int j = kHpl - 1; j >= 0; --j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            px[j] = 0.f;
            if (ok) { pn = ri * ba[j] * pn + ba[j] * bp[j]; px[j] = pn; }
        }
        // box and ramp projections, inner dual steps; the chunk's first hour reads the
        // previous lane's last p
        float p_last = 0.f;
#pragma unroll
        for (int j = 0; j < kHpl; ++j) if (j == hpl - 1) p_last = px[j];
        float p_prev = __shfl_up_sync(0xffffffffu, p_last, 1);
        if (lane == 0) p_prev = 0.f;
#pragma unroll
        for (int j = 0; j < kHpl; ++j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            if (!ok) continue;
            const float pp = j == 0 ? p_prev : px[j > 0 ? j - 1 : 0];
            const float dz = px[j] + y[j] * iri;
            float nz;
            if (ADJ) nz = (mk[j] & 3) != A_FREE ? 0.f : dz;
            else nz = clampf(dz, 0.f, cap[j]);
            y[j] += ri * (px[j] - nz);
            z[j] = nz;
            if (t > 0) {
                const float d = px[j] - pp;
                const float dw = d + q[j] * iri;
                float nw;
                if (ADJ) nw = ((mk[j] >> 2) & 3) != A_FREE ? 0.f : dw;
                else nw = clampf(dw, -R, R);
                q[j] += ri * (d - nw);
                w[j] = nw;
            }
        }
    }
    float dx2 = 0.f, x2 = 0.f, gscale = 0.f;
#pragma unroll
    for (int j = 0; j < kHpl; ++j) {
        const int t = t0 + j;
        const bool ok = (j < hpl) && (t < T);
        if (!ok) continue;
        const long long rr = row0 + t;
        X.xg[grow0 + t] = px[j];
        X.z[rr] = z[j]; X.w[rr] = w[j]; X.y[rr] = y[j]; X.q[rr] = q[j];
        dx2 += (px[j] - x_old[j]) * (px[j] - x_old[j]);
        x2 += px[j] * px[j];
        // adjoint scale: grad h / (rho + eps) of the hours whose capacity bound is free
        if (ADJ && (mk[j] & 3) == A_FREE) gscale += (lin[j] * inv_re) * (lin[j] * inv_re);
    }
    if (want_res) {
        dx2 = warp_sum(dx2);
        x2 = warp_sum(x2);
        gscale = warp_sum(gscale);
        if (lane == 0) {
            c.ramp_part[gw * kDevPart + 0] = dx2;
            c.ramp_part[gw * kDevPart + 1] = x2;
            c.ramp_part[gw * kDevPart + 2] = gscale;
            if (stamp) stamp_end(c, 2);
        }
    }
}

#define GX_RAMP_HPL(H)                                                                           \
    do {                                                                                         \
        if (adj) {                                                                               \
            if (mode == M_ADJ) k_ramp<M_ADJ, 1, H><<<grid, kBatWarps * 32, 0, st>>>(c, want_res);         \
            else if (mode == M_RESET) k_ramp<M_RESET, 1, H><<<grid, kBatWarps * 32, 0, st>>>(c, want_res); \
        } else {                                                                                 \
            if (mode == M_FWD) k_ramp<M_FWD, 0, H><<<grid, kBatWarps * 32, 0, st>>>(c, want_res);         \
            else if (mode == M_RESET) k_ramp<M_RESET, 0, H><<<grid, kBatWarps * 32, 0, st>>>(c, want_res); \
            else if (mode == M_MASK) k_ramp<M_MASK, 0, H><<<grid, kBatWarps * 32, 0, st>>>(c, want_res);   \
        }                                                                                        \
    } while (0)

// Hours per lane compiled for 1, 2, 3, 6 and 8 (T up to 32, 64, 96, 192, 256), from the
// longest horizon among the scenarios with ramping generators.
int launch_ramp(const Ctx& c, int mode, int adj, int want_res, cudaStream_t st) {
    if (mode == M_INIT || c.n_ramp_warps <= 0) return 0;
    const int grid = (c.n_ramp_warps + kBatWarps - 1) / kBatWarps;
    const int hpl = (c.max_ramp_T + 31) / 32;
    if (hpl <= 1) GX_RAMP_HPL(1);
    else if (hpl <= 2) GX_RAMP_HPL(2);
    else if (hpl <= 3) GX_RAMP_HPL(3);
    else if (hpl <= 6) GX_RAMP_HPL(6);
    else GX_RAMP_HPL(8);
    return 1;
}

}  // namespace gx
