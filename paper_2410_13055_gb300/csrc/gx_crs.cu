// Cluster-resident persistent message passing: the whole iteration loop of a scenario
// (forward dispatch or adjoint) in one launch, its state in shared memory.
//
// One thread-block cluster of C CTAs per scenario; CTA r owns hours [r*H, (r+1)*H) of
// every bus, generator, line and battery (H = ceil(T / C)).  Buses are coupled by lines
// only within an hour, so the line proxes and the bus consensus read and write the CTA's
// own shared memory.  A battery couples all hours: it is owned by one CTA (b mod C),
// whose warp gathers the battery bus's price terms of every hour from the ranks that own
// them and scatters its new injections back, over distributed shared memory.  One outer
// iteration is
//     line proxes + battery proxes  | cluster barrier |  bus step  | cluster barrier
// and every check_every iterations rank 0 reduces the residual partials of all ranks in
// FP64 and broadcasts stop / continue, so the loop needs no host synchronisation.
//
// The arithmetic of every step is that of the streaming kernels (gx_kernels.cu): the same
// expressions in the same order, so a scenario takes the same iterates on either path up
// to the summation order of the residual partials.  State is read from and written back
// to the workspace rows at entry and exit, so the reset, mask, extraction and gradient
// kernels work unchanged.
#include "gx_internal.cuh"

#include <cfloat>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace gx {

namespace {

constexpr int kCrsWarps = kCrsThreads / 32;

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}


struct Sm {
    double* red;
    float* wred;
    int* flag;
    float *pbar, *u, *thb, *xl, *ld, *aux, *xg, *cap, *dl, *sg, *vf, *vt, *xb, *lcap, *bst;
    uint8_t* lmask;
};

__device__ __forceinline__ Sm sm_at(unsigned char* b, const CrsOff& o) {
    Sm m;
    m.red = reinterpret_cast<double*>(b + o.red);
    m.wred = reinterpret_cast<float*>(b + o.wred);
    m.flag = reinterpret_cast<int*>(b + o.flag);
    m.pbar = reinterpret_cast<float*>(b + o.pbar);
    m.u = reinterpret_cast<float*>(b + o.u);
    m.thb = reinterpret_cast<float*>(b + o.thb);
    m.xl = reinterpret_cast<float*>(b + o.xl);
    m.ld = reinterpret_cast<float*>(b + o.ld);
    m.aux = reinterpret_cast<float*>(b + o.aux);
    m.xg = reinterpret_cast<float*>(b + o.xg);
    m.cap = reinterpret_cast<float*>(b + o.cap);
    m.dl = reinterpret_cast<float*>(b + o.dl);
    m.sg = reinterpret_cast<float*>(b + o.sg);
    m.vf = reinterpret_cast<float*>(b + o.vf);
    m.vt = reinterpret_cast<float*>(b + o.vt);
    m.xb = reinterpret_cast<float*>(b + o.xb);
    m.lcap = reinterpret_cast<float*>(b + o.lcap);
    m.bst = reinterpret_cast<float*>(b + o.bst);
    m.lmask = b + o.lmask;
    return m;
}

struct GState {
    float *xg, *xl, *dl, *sg, *vf, *vt, *xb, *zc, *zd, *zs, *yc, *yd, *ys, *u, *pbar, *thb;
};

template <int ADJ>
__device__ __forceinline__ GState gstate(const Ctx& c) {
    if (ADJ)
        return GState{c.a_xg, c.a_xl, c.a_dl, c.a_sg, c.a_vf, c.a_vt, c.a_xb, c.a_zc, c.a_zd, c.a_zs,
                      c.a_yc, c.a_yd, c.a_ys, c.a_u, c.a_pbar, c.a_thb};
    return GState{c.xg, c.xl, c.dl, c.sg, c.vf, c.vt, c.xb, c.zc, c.zd, c.zs, c.yc, c.yd, c.ys, c.u, c.pbar, c.thb};
}

// Battery prox of one owned battery by one warp (the inner ADMM of the battery kernel:
// box copy z, scaled duals y, the equality-constrained step through the constant
// tridiagonal system solved by two warp affine scans).  st: the battery's state rows in
// this rank's shared memory; the bus terms and the new injections go through the ranks
// owning each hour.
template <int ADJ, int kHpl>
__device__ __forceinline__ void crs_battery(const Ctx& c, const ScenDev& sd, const Sm& m, cg::cluster_group& cl,
                                            int H, int b, float* st, bool want, float& dx2_acc, float& x2_acc) {
    const int lane = threadIdx.x & 31;
    const int bg = sd.bat0 + b;
    const int T = sd.T;
    const int hpl = (T + 31) >> 5;
    const int t0 = lane * hpl;
    const long long row0 = sd.e_bat + (long long)b * sd.Tp;
    const int bus = c.b_bus[bg];
    const float rho = c.rho, eps = c.eps, ri = c.rho_in, iri = 1.f / c.rho_in;
    const float P = fmaxf(c.eta[sd.eta0 + sd.G + sd.L + b], 0.f);
    const float E = c.b_dur[bg] * P;
    const float a = c.b_effc[bg], k = 1.f / c.b_effd[bg];
    const float Ah = eps + ri + rho;
    const float det = Ah * Ah - rho * rho;
    const float idet = 1.f / det;
    const float gc = (Ah * a - rho * k) * idet;
    const float gd = (rho * a - Ah * k) * idet;

    float v[kHpl], zc[kHpl], zd[kHpl], zs[kHpl], yc[kHpl], yd[kHpl], ys[kHpl];
    float qc[kHpl], qd[kHpl], idd[kHpl], iddp[kHpl], xb_old[kHpl];
    uint8_t mk[kHpl];  // adjoint: active-set code of the hour (c, d, s two bits each)
    // every load of the lane's hours before any use (hours past the horizon read T-1)
#pragma unroll
    for (int j = 0; j < kHpl; ++j) {
        const int t = t0 + j;
        const bool ok = (j < hpl) && (t < T);
        const int tc = ok ? t : T - 1;
        const long long r = row0 + tc;
        const int rk = tc / H, hl = tc - rk * H;
        xb_old[j] = st[6 * T + tc];
        const float* rp = cl.map_shared_rank(m.pbar, rk);
        const float* ru = cl.map_shared_rank(m.u, rk);
        v[j] = xb_old[j] - rp[bus * H + hl] - ru[bus * H + hl];
        zc[j] = st[0 * T + tc]; zd[j] = st[1 * T + tc]; zs[j] = st[2 * T + tc];
        yc[j] = st[3 * T + tc]; yd[j] = st[4 * T + tc]; ys[j] = st[5 * T + tc];
        idd[j] = c.bat_dd[r];
        iddp[j] = c.bat_dd[tc > 0 ? r - 1 : r];
        mk[j] = 0;
        qc[j] = qd[j] = 0.f;
        if (ADJ) {
            mk[j] = c.m_bat[r];
            qc[j] = -eps * c.zc[r];
            qd[j] = -eps * c.zd[r];
        }
    }
#pragma unroll
    for (int j = 0; j < kHpl; ++j) {
        const int t = t0 + j;
        const bool ok = (j < hpl) && (t < T);
        idd[j] = ok ? 1.f / idd[j] : 0.f;
        iddp[j] = (ok && t > 0) ? 1.f / iddp[j] : 0.f;
        if (!ok) {
            v[j] = zc[j] = zd[j] = zs[j] = yc[j] = yd[j] = ys[j] = 0.f;
            qc[j] = qd[j] = 0.f; xb_old[j] = 0.f; mk[j] = 0;
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
        float rs_last = 0.f;
#pragma unroll
        for (int j = 0; j < kHpl; ++j) if (j == hpl - 1) rs_last = rs[j];
        float rs_prev = __shfl_up_sync(0xffffffffu, rs_last, 1);
        if (lane == 0) rs_prev = 0.f;
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
        if (lane == 0) yin = 0.f;
        float yv[kHpl];
#pragma unroll
        for (int j = 0; j < kHpl; ++j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            if (ok) yin = iddp[j] * yin + rhs[j];
            yv[j] = yin;
        }
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
        if (lane == 31) min_ = 0.f;
        float mu[kHpl];
        float mnext = min_;
#pragma unroll
        for (int j = kHpl - 1; j >= 0; --j) {
            const int t = t0 + j;
            const bool ok = (j < hpl) && (t < T);
            mu[j] = 0.f;
            if (ok) { mnext = idd[j] * (yv[j] + mnext); mu[j] = mnext; }
        }
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
            float nzc, nzd, nzs;
            if (ADJ) {
                // fixed components of the active set stay at 0; free ones are unbounded
                nzc = (mk[j] & 3) != A_FREE ? 0.f : cc + yc[j] * iri;
                nzd = ((mk[j] >> 2) & 3) != A_FREE ? 0.f : dd_ + yd[j] * iri;
                nzs = ((mk[j] >> 4) & 3) != A_FREE ? 0.f : ss + ys[j] * iri;
            } else {
                nzc = clampf(cc + yc[j] * iri, 0.f, P);
                nzd = clampf(dd_ + yd[j] * iri, 0.f, P);
                nzs = clampf(ss + ys[j] * iri, 0.f, E);
            }
            yc[j] += ri * (cc - nzc);
            yd[j] += ri * (dd_ - nzd);
            ys[j] += ri * (ss - nzs);
            zc[j] = nzc; zd[j] = nzd; zs[j] = nzs;
            cx[j] = cc; dx[j] = dd_;
        }
    }
#pragma unroll
    for (int j = 0; j < kHpl; ++j) {
        const int t = t0 + j;
        const bool ok = (j < hpl) && (t < T);
        if (!ok) continue;
        const int rk = t / H, hl = t - rk * H;
        const float xn = dx[j] - cx[j];
        st[6 * T + t] = xn;
        cl.map_shared_rank(m.xb, rk)[b * H + hl] = xn;
        st[0 * T + t] = zc[j]; st[1 * T + t] = zd[j]; st[2 * T + t] = zs[j];
        st[3 * T + t] = yc[j]; st[4 * T + t] = yd[j]; st[5 * T + t] = ys[j];
        if (want) {
            dx2_acc += (xn - xb_old[j]) * (xn - xb_old[j]);
            x2_acc += xn * xn;
        }
    }
}

template <int ADJ, int kHpl>
__global__ void __launch_bounds__(kCrsThreads, 1)
    k_crs(const Ctx c, const int* __restrict__ scen, const int* __restrict__ in_batch, int C, double tol) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int s = scen[blockIdx.x / C];
    if (!in_batch[s]) return;  // the whole cluster, before its first barrier
    const ScenDev sd = c.scen[s];
    const int T = sd.T, N = sd.N, G = sd.G, L = sd.L, B = sd.B;
    const int H = (T + C - 1) / C;
    const int h0 = rank * H;
    const int nh = max(0, min(H, T - h0));
    const int nbo = (B + C - 1) / C;
    const Sm m = sm_at(smem, crs_offsets(N, G, L, B, H, nbo, T));
    const GState X = gstate<ADJ>(c);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float rho = c.rho, eps = c.eps;
    const float inv_re = 1.f / (rho + eps);

    // ---- state in
    for (int q = tid; q < N * nh; q += kCrsThreads) {
        const int n = q / nh, hl = q - n * nh;
        const long long gi = sd.e_bus + (long long)n * sd.Tp + h0 + hl;
        const int li = n * H + hl;
        m.pbar[li] = X.pbar[gi]; m.u[li] = X.u[gi]; m.thb[li] = X.thb[gi]; m.xl[li] = X.xl[gi];
        const float Lnt = c.load[gi];
        m.ld[li] = Lnt;
        if (ADJ) m.aux[li] = c.al[gi];  // adjoint coefficient, NaN where the bound is active
    }
    for (int q = tid; q < G * nh; q += kCrsThreads) {
        const int g = q / nh, hl = q - g * nh;
        const long long gi = sd.e_gen + (long long)g * sd.Tp + h0 + hl;
        const int li = g * H + hl;
        const int gg = sd.gen0 + g;
        m.xg[li] = X.xg[gi];
        if (ADJ) {
            m.cap[li] = c.ag[gi];  // adjoint coefficient, NaN where the bound is active
        } else {
            const float etag = fmaxf(c.eta[sd.eta0 + g], 0.f);
            m.cap[li] = c.g_firm[gg] ? etag : c.cf[gi] * etag;
        }
    }
    for (int q = tid; q < L * nh; q += kCrsThreads) {
        const int l = q / nh, hl = q - l * nh;
        const long long gi = sd.e_line + (long long)l * sd.Tp + h0 + hl;
        const int li = l * H + hl;
        m.dl[li] = X.dl[gi]; m.sg[li] = X.sg[gi]; m.vf[li] = X.vf[gi]; m.vt[li] = X.vt[gi];
        if (ADJ) m.lmask[li] = c.m_line[gi];
    }
    for (int l = tid; l < L; l += kCrsThreads)
        m.lcap[l] = fmaxf(c.eta[sd.eta0 + G + l], 0.f) / c.l_beta[sd.line0 + l];
    for (int q = tid; q < B * nh; q += kCrsThreads) {
        const int b = q / nh, hl = q - b * nh;
        m.xb[b * H + hl] = X.xb[sd.e_bat + (long long)b * sd.Tp + h0 + hl];
    }
    for (int q = tid; q < nbo * T; q += kCrsThreads) {
        const int j = q / T, t = q - j * T;
        const int b = rank + j * C;
        if (b >= B) continue;
        const long long r = sd.e_bat + (long long)b * sd.Tp + t;
        float* st = m.bst + (size_t)j * kCrsBatState * T;
        st[0 * T + t] = X.zc[r]; st[1 * T + t] = X.zd[r]; st[2 * T + t] = X.zs[r];
        st[3 * T + t] = X.yc[r]; st[4 * T + t] = X.yd[r]; st[5 * T + t] = X.ys[r];
        st[6 * T + t] = X.xb[r];
    }
    cl.sync();

    // ---- iterations
    const int max_it = c.max_it, every = c.check_every;
    int it = 0;
    double best = 0.0;
    for (;;) {
        const int chunk = min(every, max_it - it);
        for (int jt = 0; jt < chunk; ++jt) {
            const bool want = jt == chunk - 1;
            float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            // line proxes (phase-dual update and the clipped 1-D minimiser)
            for (int q = tid; q < L * nh; q += kCrsThreads) {
                const int l = q / nh, hl = q - l * nh;
                const int li = l * H + hl;
                const int lg = sd.line0 + l;
                const int bf = c.l_from[lg] * H + hl, bt = c.l_to[lg] * H + hl;
                const float beta = c.l_beta[lg];
                const float lw = c.l_w[lg];
                const bool dc = lw == 0.f;  // HVDC transport line
                const float d = m.dl[li], g = m.sg[li];
                const float zf = m.thb[bf], zt = m.thb[bt];
                const float vf = m.vf[li] - zf, vt = m.vt[li] - zt;
                if (want && !dc) {
                    const float ef = 0.5f * (g + d) - zf, et = 0.5f * (g - d) - zt;
                    acc[8] += beta * beta * (ef * ef + et * et);
                }
                const float wf = zf - vf, wt = zt - vt;
                const float tf = -beta * d - m.pbar[bf] - m.u[bf];
                const float tt = beta * d - m.pbar[bt] - m.u[bt];
                const float rth = c.rth_c * lw;
                const float den = 2.f * rho * beta * beta + 0.5f * rth + (dc ? eps : 0.f);
                const float lin = (ADJ && dc) ? eps * c.dl[sd.e_line + (long long)l * sd.Tp + h0 + hl] : 0.f;
                const float dun = (rho * beta * (tt - tf) + 0.5f * rth * (wf - wt) + lin) / den;
                const float cap = fminf(m.lcap[l], c.l_dth[lg]);
                float dn;
                if (ADJ) dn = m.lmask[li] ? 0.f : dun;
                else dn = clampf(dun, -cap, cap);
                const float gn = wf + wt;
                m.dl[li] = dn;
                m.sg[li] = gn;
                m.vf[li] = 0.5f * (gn + dn) + vf;
                m.vt[li] = 0.5f * (gn - dn) + vt;
                if (want) {
                    const float dd = dn - d;
                    acc[6] += 2.f * beta * beta * dd * dd;
                    acc[7] += 2.f * beta * beta * dn * dn;
                }
            }
            // battery proxes of the batteries this rank owns
            for (int j = warp; j < nbo; j += kCrsWarps) {
                const int b = rank + j * C;
                if (b < B)
                    crs_battery<ADJ, kHpl>(c, sd, m, cl, H, b, m.bst + (size_t)j * kCrsBatState * T, want, acc[6],
                                           acc[7]);
            }
            cl.sync();
            // bus step: generator and load proxes, then the consensus and the dual update
            for (int q = tid; q < N * nh; q += kCrsThreads) {
                const int n = q / nh, hl = q - n * nh;
                const int li = n * H + hl;
                const float pb = m.pbar[li], uu = m.u[li], thold = m.thb[li];
                float sum = 0.f, dx2 = 0.f, x2 = 0.f, gscale = 0.f;
                const int pn = sd.ptr0 + n;
                const int g1 = c.bus_gptr[pn + 1];
                for (int k = c.bus_gptr[pn]; k < g1; ++k) {
                    const int g = c.bus_gidx[sd.gen0 + k];
                    const int gi = g * H + hl;
                    const float x = m.xg[gi];
                    const float v = x - pb - uu;
                    float xn;
                    if (ADJ) {
                        const float gh = m.cap[gi];
                        const bool fixed = isnan(gh);
                        xn = fixed ? 0.f : (rho * v + gh) * inv_re;
                        if (!fixed) gscale += (gh * inv_re) * (gh * inv_re);
                    } else {
                        const float pun = (rho * v - c.g_cost[sd.gen0 + g]) * inv_re;
                        xn = clampf(pun, 0.f, m.cap[gi]);
                    }
                    m.xg[gi] = xn;
                    sum += xn;
                    dx2 += (xn - x) * (xn - x);
                    x2 += xn * xn;
                }
                {
                    const float x = m.xl[li];
                    const float v = x - pb - uu;
                    float xn;
                    if (ADJ) {
                        const float gsh = m.aux[li];
                        const bool fixed = isnan(gsh);
                        xn = fixed ? 0.f : (rho * v + gsh) * inv_re;
                        if (!fixed) gscale += (gsh * inv_re) * (gsh * inv_re);
                    } else {
                        const float Lnt = m.ld[li];
                        const float sun = (rho * (v + Lnt) - c.voll) * inv_re;
                        xn = clampf(sun, 0.f, Lnt) - Lnt;
                    }
                    m.xl[li] = xn;
                    sum += xn;
                    dx2 += (xn - x) * (xn - x);
                    x2 += xn * xn;
                }
                const int b1 = c.bus_bptr[pn + 1];
                for (int k = c.bus_bptr[pn]; k < b1; ++k) {
                    const float xb = m.xb[c.bus_bidx[sd.bat0 + k] * H + hl];
                    sum += xb;
                    x2 += xb * xb;
                }
                float ths = 0.f;
                const int e1 = c.bus_eptr[pn + 1];
                for (int k = c.bus_eptr[pn]; k < e1; ++k) {
                    const int e = c.bus_eidx[2 * sd.line0 + k];
                    const int l = e >> 1;
                    const int li2 = l * H + hl;
                    const float d = m.dl[li2];
                    const float qv = (e & 1) ? m.vt[li2] : m.vf[li2];
                    const float beta = c.l_beta[sd.line0 + l];
                    const float p = (e & 1) ? beta * d : -beta * d;
                    sum += p;
                    x2 += p * p;
                    ths += c.l_w[sd.line0 + l] * qv;
                }
                const float icnt = c.bus_inv_cnt[sd.bus0 + n];
                const float pbn = sum * icnt;
                const float thn = ths * c.bus_inv_wsum[sd.bus0 + n];
                const float un = uu + pbn;
                m.pbar[li] = pbn;
                m.u[li] = un;
                m.thb[li] = thn;
                if (want) {
                    const float cnt = 1.f / icnt;
                    const float dpb = pbn - pb;
                    acc[0] += cnt * pbn * pbn;
                    acc[1] += gscale;
                    acc[2] += dx2 - cnt * dpb * dpb;
                    acc[3] += (thn - thold) * (thn - thold) * c.bus_dres_w[sd.bus0 + n];
                    acc[4] += cnt * (rho * un) * (rho * un);
                    acc[5] += x2;
                }
            }
            if (want) {
                // this rank's partial sums into rank 0's reduction slots
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const float w = warp_sum(acc[q]);
                    if (lane == 0) m.wred[warp * kCrsRed + q] = w;
                }
                __syncthreads();
                if (tid < 9) {
                    float tot = 0.f;
                    for (int w = 0; w < kCrsWarps; ++w) tot += m.wred[w * kCrsRed + tid];
                    cl.map_shared_rank(m.red, 0)[rank * kCrsRed + tid] = (double)tot;
                }
            }
            cl.sync();
        }
        it += chunk;
        if (rank == 0 && tid == 0) {
            // the convergence test of the streaming reduction kernel, on the cluster's sums
            double a[9];
            for (int q = 0; q < 9; ++q) {
                a[q] = 0.0;
                for (int r = 0; r < C; ++r) a[q] += m.red[r * kCrsRed + q];
            }
            const double rhod = c.rho, rth = c.rth_c;
            // NaN / inf test on the raw sums, before the clamps (fmax would turn a NaN into 0)
            bool finite = true;
            for (int q = 0; q < 9; ++q) finite = finite && isfinite(a[q]);
            const double scale = ADJ ? fmax(sqrt(a[1]), 1e-30) : sd.load_norm;
            const double rp = sqrt(fmax(a[0] + a[8], 0.0)) / scale;
            const double dz2 = fmax(a[2] + a[6], 0.0);
            const double rd = sqrt(rhod * rhod * dz2 + rth * rth * a[3]) / fmax(sqrt(a[4]), 1e-30);
            c.resid[2 * s + 0] = rp;
            c.resid[2 * s + 1] = rd;
            const double r = fmax(rp, rd);
            if (it <= every || !(r >= best)) best = r;
            int stop = 1;
            if (!finite || !isfinite(rp) || !isfinite(rd) || r > 1e6 * best) c.status[s] = GX_ERR_NONFINITE;
            else if (rp <= tol && rd <= tol) c.status[s] = GX_OK;
            else if (it >= max_it) c.status[s] = GX_NOT_CONVERGED;
            else stop = 0;
            if (stop) {
                c.done[s] = 1;
                (ADJ ? c.adj_iters : c.iters)[s] = it;
                c.rbest[s] = best;
            }
            m.flag[0] = stop;
        }
        cl.sync();
        if (*cl.map_shared_rank(m.flag, 0)) break;
    }

    // ---- state out
    for (int q = tid; q < N * nh; q += kCrsThreads) {
        const int n = q / nh, hl = q - n * nh;
        const long long gi = sd.e_bus + (long long)n * sd.Tp + h0 + hl;
        const int li = n * H + hl;
        X.pbar[gi] = m.pbar[li]; X.u[gi] = m.u[li]; X.thb[gi] = m.thb[li]; X.xl[gi] = m.xl[li];
    }
    for (int q = tid; q < G * nh; q += kCrsThreads) {
        const int g = q / nh, hl = q - g * nh;
        X.xg[sd.e_gen + (long long)g * sd.Tp + h0 + hl] = m.xg[g * H + hl];
    }
    for (int q = tid; q < L * nh; q += kCrsThreads) {
        const int l = q / nh, hl = q - l * nh;
        const long long gi = sd.e_line + (long long)l * sd.Tp + h0 + hl;
        const int li = l * H + hl;
        X.dl[gi] = m.dl[li]; X.sg[gi] = m.sg[li]; X.vf[gi] = m.vf[li]; X.vt[gi] = m.vt[li];
    }
    for (int q = tid; q < nbo * T; q += kCrsThreads) {
        const int j = q / T, t = q - j * T;
        const int b = rank + j * C;
        if (b >= B) continue;
        const long long r = sd.e_bat + (long long)b * sd.Tp + t;
        const float* st = m.bst + (size_t)j * kCrsBatState * T;
        X.zc[r] = st[0 * T + t]; X.zd[r] = st[1 * T + t]; X.zs[r] = st[2 * T + t];
        X.yc[r] = st[3 * T + t]; X.yd[r] = st[4 * T + t]; X.ys[r] = st[5 * T + t];
        X.xb[r] = st[6 * T + t];
    }
    // no rank leaves while another may still read its shared memory
    cl.sync();
}

template <int ADJ, int kHpl>
void* crs_fn() {
    return reinterpret_cast<void*>(&k_crs<ADJ, kHpl>);
}

void* crs_kernel(int adj, int hpl) {
    if (adj) {
        if (hpl <= 1) return crs_fn<1, 1>();
        if (hpl <= 2) return crs_fn<1, 2>();
        if (hpl <= 3) return crs_fn<1, 3>();
        if (hpl <= 6) return crs_fn<1, 6>();
        return crs_fn<1, 8>();
    }
    if (hpl <= 1) return crs_fn<0, 1>();
    if (hpl <= 2) return crs_fn<0, 2>();
    if (hpl <= 3) return crs_fn<0, 3>();
    if (hpl <= 6) return crs_fn<0, 6>();
    return crs_fn<0, 8>();
}

void crs_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* at, int nclusters, int C, size_t smem,
                cudaStream_t st) {
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3((unsigned)(nclusters * C));
    cfg.blockDim = dim3(kCrsThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
}

}  // namespace

// Several launch groups share one instantiation with different image sizes, so each
// instantiation is opened to the largest image any group may use (smem_max) and to
// non-portable cluster sizes; a launch still states its own size.
cudaError_t crs_prepare(int adj, int hpl, size_t smem_max) {
    const void* f = crs_kernel(adj, hpl);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

int crs_max_clusters(int adj, int hpl, int C, size_t smem) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    crs_config(cfg, at, 1, C, smem, nullptr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, crs_kernel(adj, hpl), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int launch_crs(const Ctx& c, int adj, const int* scen, int n, const int* in_batch, int C, int hpl, size_t smem,
               double tol, cudaStream_t st) {
    if (n <= 0) return 0;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    crs_config(cfg, at, n, C, smem, st);
#define GX_CRS(A, HP) cudaLaunchKernelEx(&cfg, k_crs<A, HP>, c, scen, in_batch, C, tol)
    if (adj) {
        if (hpl <= 1) GX_CRS(1, 1);
        else if (hpl <= 2) GX_CRS(1, 2);
        else if (hpl <= 3) GX_CRS(1, 3);
        else if (hpl <= 6) GX_CRS(1, 6);
        else GX_CRS(1, 8);
    } else {
        if (hpl <= 1) GX_CRS(0, 1);
        else if (hpl <= 2) GX_CRS(0, 2);
        else if (hpl <= 3) GX_CRS(0, 3);
        else if (hpl <= 6) GX_CRS(0, 6);
        else GX_CRS(0, 8);
    }
#undef GX_CRS
    return 1;
}

}  // namespace gx
