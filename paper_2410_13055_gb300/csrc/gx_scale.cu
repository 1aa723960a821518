// Capacity-dependent susceptance: an AC line whose planned capacity is added as parallel
// circuits has beta_l(eta) = (beta0_l / ref_l) eta_l, so the constraint matrix of the
// dispatch depends on the plan (the A(eta) of Eq. 2).
//
// Solve: the message passing is unchanged; only the numbers it reads change.  Once per
// call k_scale_prep writes the effective beta into the line table and into the bus pool
// records (each line end's beta), and recomputes the dual-residual weight of every bus that
// such a line touches.  The flow limit |beta_l dtheta| <= eta_l becomes the fixed angle
// limit |dtheta| <= ref_l / beta0_l, which the line kernels get from eta / beta as before.
// The lines' phase weights stay those of beta0 (they only pace the iteration).
//
// Gradient (Section 2.2, the KKT residual differentiated in eta).  With b = d beta / d eta
// = beta0 / ref, price lambda = -(multiplier of the balance rows) and dtheta = theta_from -
// theta_to, the line's entries of dA/deta x are -b dtheta at its from-bus and +b dtheta at
// its to-bus; the flow-limit rows contribute nothing, since at an active limit the change of
// the row (b dtheta = 1) equals the change of its bound.  So per hour
//   envelope (h = c):  dh/deta_l = -b dtheta (lambda_to - lambda_from),
//   adjoint:           dh/deta_l =  b [dtheta^ (lambda_to - lambda_from)
//                                    + dtheta (lambda^_to - lambda^_from)],
// dtheta^ and lambda^ = -rho_a u^ the adjoint iteration's phase difference and price.  One
// warp per (scenario, scaling line) writes that sum over the horizon in place of the entry
// k_grad assembled from the flow-limit multipliers.
#include "gx_internal.cuh"

namespace gx {

namespace {

__device__ __forceinline__ double beta_eff(const Ctx& c, int k) {
    return fmax(c.sc_b[k] * (double)c.eta[c.sc_eta[k]], c.sc_bmin[k]);
}

__global__ void k_scale_prep(const Ctx c) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < c.n_scale) {
        c.l_beta_w[c.sc_line[i]] = (float)beta_eff(c, i);
        return;
    }
    i -= c.n_scale;
    if (i < c.n_sc_pool) {
        const int2 e = c.sc_pool[i];
        c.pool[e.x] = __float_as_int((float)beta_eff(c, e.y));
        return;
    }
    i -= c.n_sc_pool;
    if (i < c.n_sc_dres) {
        const ScaleDres r = c.sc_dres[i];
        double d = r.d0;
        for (int j = r.first; j < r.first + r.count; ++j) {
            const int2 e = c.sc_dres_l[j];
            const double q = (double)__int_as_float(e.y) / beta_eff(c, e.x);
            d += q * q;
        }
        if (r.target >= 0) c.pool[r.target] = __float_as_int((float)d);
        else c.dres_w_w[-1 - r.target] = (float)d;
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kBlock) k_scale_grad(const Ctx c, int envelope, const int* in_batch) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
    if (gw >= c.n_sc_gwarps) return;
    const int s = c.sc_gwarp[2 * gw], k = c.sc_gwarp[2 * gw + 1];
    if (!in_batch[s]) return;
    const ScenDev sc = c.scen[s];
    const int lg = c.sc_line[k], l = lg - sc.line0;
    const int f = c.l_from[lg], to = c.l_to[lg];
    // the adjoint context carries its own rho; the forward one is rho * rho_ratio
    const double rho_f = (double)c.rho * (double)c.rho_ratio, rho_a = c.rho;
    double acc = 0.0;
    for (int t = lane; t < sc.T; t += 32) {
        const long long rr = sc.e_line + (long long)l * sc.Tp + t;
        const long long bf = sc.e_bus + (long long)f * sc.Tp + t;
        const long long bt = sc.e_bus + (long long)to * sc.Tp + t;
        const double dlam = -rho_f * ((double)c.u[bt] - (double)c.u[bf]);
        if (envelope) {
            acc -= (double)c.dl[rr] * dlam;
        } else {
            const double dlam_a = -rho_a * ((double)c.a_u[bt] - (double)c.a_u[bf]);
            acc += (double)c.a_dl[rr] * dlam + (double)c.dl[rr] * dlam_a;
        }
    }
    acc = warp_sum_d(acc);
    if (lane == 0) c.grad_s[sc.gs0 + sc.G + l] = c.sc_b[k] * acc;
}

}  // namespace

int launch_scale_prep(const Ctx& c, cudaStream_t st) {
    const int n = c.n_scale + c.n_sc_pool + c.n_sc_dres;
    if (n <= 0) return 0;
    k_scale_prep<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(c);
    return 1;
}

int launch_scale_grad(const Ctx& c, int envelope, const int* in_batch, cudaStream_t st) {
    if (c.n_sc_gwarps <= 0) return 0;
    const int grid = (c.n_sc_gwarps + kBlock / 32 - 1) / (kBlock / 32);
    k_scale_grad<<<grid, kBlock, 0, st>>>(c, envelope, in_batch);
    return 1;
}

}  // namespace gx
