// Discrete adjoint (reverse mode) of the coupled phi-mu LBM step.
//
// The step is linear in the populations and a smooth function of the fields
// phi and c.  Its adjoint maps the adjoints (gb, hb, phib, cb) of the state at
// step n+1 to those of the state at step n, and accumulates the adjoints of the
// parameters (D_l, tau_g, tau_h, lambda) in FP64.  Three kernels per step, one
// thread per node, no atomics on fields (every node gathers what it needs):
//
//   k_adj_h      composition part: pulls hb from downstream neighbours (the
//                transpose of streaming, bounce-back included), then the
//                adjoints of the h collision, of h^eq, of H and of the flux F;
//                leaves per-node partial adjoints in a work area.
//   k_adj_g      phi part: pulls gb and the adjoint of phi^{n+1} (plus that of
//                dphi/dt from k_adj_h) from downstream neighbours, then the
//                adjoints of the g collision and of the sources G; finishes the
//                unit normal and the closure.
//   k_adj_finish transpose of the gradient stencil, gathered per node over the
//                stencil pre-images (periodic images and mirror ghosts).
//
// k_adj_init is the adjoint of the initialisation (g = w phi - G/2,
// h = h^eq - H/2 at dphi/dt = 0), followed by k_adj_finish.
#pragma once

#include "step_kernels.cuh"

namespace lbpf {

template <typename R>
struct AdjWork {        // per-node partial adjoints, SoA, N entries each
    R* phi;             // adjoint of phi (local terms)
    R* mu;              // adjoint of mu
    R* c;               // adjoint of c (local terms)
    R* dphi;            // adjoint of dphi/dt
    R* grad;            // adjoint of grad phi, [3][N]
    R* n;               // adjoint of the unit normal, [3][N]
};

constexpr int kAdjThreads = 256;
// Parameter adjoints, in this order: D_l, tau_g, tau_h, lambda, a (of j_at), D_s.
constexpr int kAdjParams = 6;
enum { kPDl = 0, kPTauG = 1, kPTauH = 2, kPLam = 3, kPA = 4, kPDs = 5 };

// Adds the block's sum of each parameter adjoint to its own slot
// acc[j * nblk + blockIdx.x].  Kernels of one sweep run in stream order, so the
// slots need no atomics, and the final sum (k_adj_param_final) has a fixed order.
__device__ __forceinline__ void adj_param_flush(double (&v)[kAdjParams], double* __restrict__ acc, int nblk) {
    __shared__ double red[kAdjParams][kAdjThreads / 32];
#pragma unroll
    for (int j = 0; j < kAdjParams; ++j)
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int j = 0; j < kAdjParams; ++j) red[j][w] = v[j];
    __syncthreads();
    if (threadIdx.x < kAdjParams) {
        double t = 0.0;
        for (int i = 0; i < kAdjThreads / 32; ++i) t += red[threadIdx.x][i];
        acc[(long long)threadIdx.x * nblk + blockIdx.x] += t;
    }
}

// out[j] = sum over blocks of acc[j * nblk + b], in a fixed order.
__global__ void __launch_bounds__(kAdjThreads) k_adj_param_final(const double* __restrict__ acc, int nblk,
                                                                double* __restrict__ out) {
    __shared__ double s[kAdjThreads];
    for (int j = 0; j < kAdjParams; ++j) {
        double t = 0.0;
        for (int b = threadIdx.x; b < nblk; b += kAdjThreads) t += acc[(long long)j * nblk + b];
        s[threadIdx.x] = t;
        __syncthreads();
        for (int o = kAdjThreads / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[j] = s[0];
        __syncthreads();
    }
}

// Forward quantities of one node recomputed from phi^n and c^n.
template <class L, typename R>
struct NodeFwd {
    R ph, cc, mu, g[3], n[3], inv;
    __device__ __forceinline__ void compute(const StepParams& P, const R* __restrict__ phi,
                                            const R* __restrict__ c, int x, int y, int z, long long i) {
        ph = phi[i];
        cc = c[i];
        mu = R(P.mu_eq) + cc - (R(P.c_l) * ph + R(P.c_s) * (R(1) - ph));
        g[0] = g[1] = g[2] = R(0);
#pragma unroll
        for (int k = 1; k < L::Q; ++k) {
            const int fx = map_coord(x + L::ex(k), P.nx, P.bc[0]), bx = map_coord(x - L::ex(k), P.nx, P.bc[0]);
            const int fy = map_coord(y + L::ey(k), P.ny, P.bc[1]), by = map_coord(y - L::ey(k), P.ny, P.bc[1]);
            const int fz = (L::D == 3) ? map_coord(z + L::ez(k), P.nz, P.bc[2]) : 0;
            const int bz = (L::D == 3) ? map_coord(z - L::ez(k), P.nz, P.bc[2]) : 0;
            const R dk = R(0.5) * (phi[((long long)fz * P.ny + fy) * P.nx + fx] - phi[((long long)bz * P.ny + by) * P.nx + bx]);
            const R cw = R(3.0 * L::w(k));
            g[0] += cw * R(L::ex(k)) * dk;
            g[1] += cw * R(L::ey(k)) * dk;
            g[2] += cw * R(L::ez(k)) * dk;
        }
        inv = R(1) / sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + R(P.eps2));
        for (int a = 0; a < 3; ++a) n[a] = g[a] * inv;
    }
};

// Node consuming the post-collision population j of (x, y, z): its linear index,
// or -1 when x + e_j lies beyond a bounce-back wall.
template <class L>
__device__ __forceinline__ long long downstream(const StepParams& P, int j, int x, int y, int z) {
    int u = x + L::ex(j), v = y + L::ey(j), w = z + L::ez(j);
    if (u < 0 || u >= P.nx) { if (P.bc[0]) return -1; u = u < 0 ? u + P.nx : u - P.nx; }
    if (v < 0 || v >= P.ny) { if (P.bc[1]) return -1; v = v < 0 ? v + P.ny : v - P.ny; }
    if (L::D == 3 && (w < 0 || w >= P.nz)) { if (P.bc[2]) return -1; w = w < 0 ? w + P.nz : w - P.nz; }
    return ((long long)w * P.ny + v) * P.nx + u;
}

// Adjoint of the c sources and equilibria at one node: heqb[j], Hb[j] given;
// adds to phib, mub, cb, gradb, nb, dphib and the parameter adjoints
// pv.  F = mu D' grad + at n, at = a W dc dphi; h^eq from Q = gamma D mu.
template <class L, typename R>
__device__ __forceinline__ void adj_c_sources(const StepParams& P, const NodeFwd<L, R>& f, R dphi,
                                              const R* heqb, const R* Hb, R& phib, R& mub, R& cb, R* gradb,
                                              R* nb, R& dphib, double (&pv)[kAdjParams]) {
    const R gamma = R(P.gamma), Dp = R(P.D_l - P.D_s);
    const R D = R(P.D_l) * f.ph + R(P.D_s) * (R(1) - f.ph);
    R Qb = -(R(1) - R(L::w(0))) * heqb[0];
    cb += heqb[0];
#pragma unroll
    for (int k = 1; k < L::Q; ++k) Qb += R(L::w(k)) * heqb[k];
    R gammab = Qb * D * f.mu;
    const R Db = Qb * gamma * f.mu;
    mub += Qb * gamma * D;
    phib += Db * Dp;
    pv[kPDl] += (double)(Db * f.ph);
    pv[kPDs] += (double)(Db * (R(1) - f.ph));
    const R atc = R(P.a_at * P.W * (P.c_s - P.c_l));       // 0 when anti-trapping is off
    const R at = atc * dphi;
    R F[3], Fb[3] = {R(0), R(0), R(0)};
    for (int a = 0; a < 3; ++a) F[a] = f.mu * Dp * f.g[a] + at * f.n[a];
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const R eF = R(L::ex(k)) * F[0] + R(L::ey(k)) * F[1] + R(L::ez(k)) * F[2];
        gammab += R(L::w(k)) * eF * Hb[k];
        Fb[0] += gamma * R(L::w(k)) * R(L::ex(k)) * Hb[k];
        Fb[1] += gamma * R(L::w(k)) * R(L::ey(k)) * Hb[k];
        Fb[2] += gamma * R(L::w(k)) * R(L::ez(k)) * Hb[k];
    }
    const R Fg = Fb[0] * f.g[0] + Fb[1] * f.g[1] + Fb[2] * f.g[2];
    const R Fn = Fb[0] * f.n[0] + Fb[1] * f.n[1] + Fb[2] * f.n[2];
    mub += Dp * Fg;
    pv[kPDl] += (double)(f.mu * Fg);
    pv[kPDs] -= (double)(f.mu * Fg);
    for (int a = 0; a < 3; ++a) {
        gradb[a] += f.mu * Dp * Fb[a];
        nb[a] += at * Fb[a];
    }
    dphib += atc * Fn;
    pv[kPA] += (double)(R(P.W * (P.c_s - P.c_l)) * dphi * Fn);
    pv[kPTauH] += (double)gammab * (-P.gamma * P.gamma / 3.0);    // gamma = 3 / tau_h
}

// Adjoint of the phi sources G_j = w_j (G^st + G^curv_j) at one node, Gb[j] given;
// adds to phib, mub, nb and the parameter adjoints pv.
template <class L, typename R>
__device__ __forceinline__ void adj_phi_sources(const StepParams& P, const NodeFwd<L, R>& f, const R* Gb,
                                                R& phib, R& mub, R* nb, double (&pv)[kAdjParams]) {
    const R M = R(P.M), W2 = R(P.W * P.W), dc = R(P.c_s - P.c_l), lam = R(P.lambda);
    R Gstb = R(0);
#pragma unroll
    for (int j = 0; j < L::Q; ++j) Gstb += R(L::w(j)) * Gb[j];
    const R pq = f.ph * (R(1) - f.ph);
    const R S = R(6) * pq * dc * (f.mu - R(P.mu_eq));
    const R Sb = Gstb * (-lam * M / W2);
    pv[kPLam] += (double)(Gstb * (-M * S / W2));
    pv[kPTauG] += (double)(Gstb * (-lam * S / W2)) / 3.0;    // M = tau_g / 3
    phib += Sb * R(6) * dc * (R(1) - R(2) * f.ph) * (f.mu - R(P.mu_eq));
    mub += Sb * R(6) * dc * pq;
    if (P.counter_term) {
        const R K = R(4.0 / P.W) * pq;
        R Kb = R(0);
#pragma unroll
        for (int j = 0; j < L::Q; ++j) {
            const R en = R(L::ex(j)) * f.n[0] + R(L::ey(j)) * f.n[1] + R(L::ez(j)) * f.n[2];
            Kb += R(L::w(j)) * en * Gb[j];
            nb[0] += K * R(L::w(j)) * R(L::ex(j)) * Gb[j];
            nb[1] += K * R(L::w(j)) * R(L::ey(j)) * Gb[j];
            nb[2] += K * R(L::w(j)) * R(L::ez(j)) * Gb[j];
        }
        phib += Kb * R(4.0 / P.W) * (R(1) - R(2) * f.ph);
    } else {
        const R wp = R(2) * pq * (R(1) - R(2) * f.ph);
        const R wpp = R(2) - R(12) * f.ph + R(12) * f.ph * f.ph;
        phib += Gstb * (-(R(8) * M / W2)) * wpp;
        pv[kPTauG] += (double)(Gstb * (-(R(8) / W2)) * wp) / 3.0;
    }
}

template <class L, typename R>
__device__ __forceinline__ R g_source(const StepParams& P, const NodeFwd<L, R>& f, int j) {
    const R pq = f.ph * (R(1) - f.ph);
    const R S = R(6) * pq * R(P.c_s - P.c_l) * (f.mu - R(P.mu_eq));
    R A = -R(P.lambda) * R(P.M) * S / R(P.W * P.W);
    R curv;
    if (P.counter_term) curv = R(4.0 / P.W) * pq * (R(L::ex(j)) * f.n[0] + R(L::ey(j)) * f.n[1] + R(L::ez(j)) * f.n[2]);
    else curv = -(R(8) * R(P.M) / R(P.W * P.W)) * (R(2) * pq * (R(1) - R(2) * f.ph));
    return R(L::w(j)) * (A + curv);
}

template <class L, typename R>
__device__ __forceinline__ void node_coords(const StepParams& P, long long i, int& x, int& y, int& z) {
    x = (int)(i % P.nx);
    y = (int)((i / P.nx) % P.ny);
    z = (int)(i / ((long long)P.nx * P.ny));
}

// ---- composition part ---------------------------------------------------------
template <class L, typename R>
__global__ void __launch_bounds__(kAdjThreads)
k_adj_h(const KParams K, const R* __restrict__ h, const R* __restrict__ phi, const R* __restrict__ c,
        const R* __restrict__ phi1, const R* __restrict__ hb_in, const R* __restrict__ cb_in,
        R* __restrict__ hb_out, AdjWork<R> T, double* __restrict__ pacc, int nblk) {
    const StepParams& P = K.P;
    const long long N = P.N;
    const long long i = blockIdx.x * (long long)kAdjThreads + threadIdx.x;
    double pv[kAdjParams] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < N) {
        int x, y, z;
        node_coords<L, R>(P, i, x, y, z);
        NodeFwd<L, R> f;
        f.compute(P, phi, c, x, y, z, i);
        const R dphi = phi1[i] - f.ph;
        const R omh = R(P.omh), gamma = R(P.gamma);
        const R D = R(P.D_l) * f.ph + R(P.D_s) * (R(1) - f.ph);
        const R at = R(P.a_at * P.W * (P.c_s - P.c_l)) * dphi;
        R F[3];
        for (int a = 0; a < 3; ++a) F[a] = f.mu * R(P.D_l - P.D_s) * f.g[a] + at * f.n[a];
        R heqb[L::Q], Hb[L::Q];
        double omhb = 0.0;
#pragma unroll
        for (int j = 0; j < L::Q; ++j) {
            const long long d = downstream<L>(P, j, x, y, z);
            const R hsb = d < 0 ? hb_in[(long long)L::opp(j) * N + i] + cb_in[i] : hb_in[(long long)j * N + d] + cb_in[d];
            hb_out[(long long)j * N + i] = (R(1) - omh) * hsb;
            heqb[j] = omh * hsb;
            Hb[j] = (R(1) - R(0.5) * omh) * hsb;
            const R Hj = gamma * R(L::w(j)) * (R(L::ex(j)) * F[0] + R(L::ey(j)) * F[1] + R(L::ez(j)) * F[2]);
            const R heq = j == 0 ? f.cc - (R(1) - R(L::w(0))) * gamma * D * f.mu : R(L::w(j)) * gamma * D * f.mu;
            omhb += (double)(hsb * (heq - R(0.5) * Hj - h[(long long)j * N + i]));
        }
        pv[kPTauH] += omhb * (-(double)P.omh * P.omh);      // omega_h = 1 / (tau_h + 1/2)
        R phib = R(0), mub = R(0), cb = R(0), dphib = R(0), gradb[3] = {R(0), R(0), R(0)}, nb[3] = {R(0), R(0), R(0)};
        adj_c_sources<L, R>(P, f, dphi, heqb, Hb, phib, mub, cb, gradb, nb, dphib, pv);
        T.phi[i] = phib;
        T.mu[i] = mub;
        T.c[i] = cb;
        T.dphi[i] = dphib;
        for (int a = 0; a < 3; ++a) {
            T.grad[a * N + i] = gradb[a];
            T.n[a * N + i] = nb[a];
        }
    }
    adj_param_flush(pv, pacc, nblk);
}

// ---- phi part ---------------------------------------------------------------------
template <class L, typename R>
__global__ void __launch_bounds__(kAdjThreads)
k_adj_g(const KParams K, const R* __restrict__ g, const R* __restrict__ phi, const R* __restrict__ c,
        const R* __restrict__ gb_in, const R* __restrict__ phib_in, R* __restrict__ gb_out, AdjWork<R> T,
        double* __restrict__ pacc, int nblk) {
    const StepParams& P = K.P;
    const long long N = P.N;
    const long long i = blockIdx.x * (long long)kAdjThreads + threadIdx.x;
    double pv[kAdjParams] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < N) {
        int x, y, z;
        node_coords<L, R>(P, i, x, y, z);
        NodeFwd<L, R> f;
        f.compute(P, phi, c, x, y, z, i);
        const R omg = R(P.omg);
        const R pnb_here = phib_in[i] + T.dphi[i];      // adjoint of phi^{n+1} at this node
        R phib = R(0), mub = R(0), Gb[L::Q];
        R nb[3] = {R(0), R(0), R(0)};
        double omgb = 0.0;
#pragma unroll
        for (int j = 0; j < L::Q; ++j) {
            const long long d = downstream<L>(P, j, x, y, z);
            const R gsb = d < 0 ? gb_in[(long long)L::opp(j) * N + i] + pnb_here
                                : gb_in[(long long)j * N + d] + phib_in[d] + T.dphi[d];
            gb_out[(long long)j * N + i] = (R(1) - omg) * gsb;
            phib += omg * R(L::w(j)) * gsb;
            Gb[j] = (R(1) - R(0.5) * omg) * gsb + R(0.5) * pnb_here;
            const R Gj = g_source<L, R>(P, f, j);
            omgb += (double)(gsb * (R(L::w(j)) * f.ph - R(0.5) * Gj - g[(long long)j * N + i]));
        }
        pv[kPTauG] += omgb * (-(double)P.omg * P.omg);
        phib -= T.dphi[i];                                // dphi = phi^{n+1} - phi^n
        adj_phi_sources<L, R>(P, f, Gb, phib, mub, nb, pv);
        // unit normal n = grad / sqrt(|grad|^2 + eps^2), then the closure
        R nt[3], nn = R(0);
        for (int a = 0; a < 3; ++a) { nt[a] = T.n[a * N + i] + nb[a]; nn += f.n[a] * nt[a]; }
        for (int a = 0; a < 3; ++a) T.grad[a * N + i] += (nt[a] - f.n[a] * nn) * f.inv;
        const R mut = T.mu[i] + mub;
        T.phi[i] += phib + mut * R(P.c_s - P.c_l);
        T.c[i] += mut;
    }
    adj_param_flush(pv, pacc, nblk);
}

// ---- transpose of the gradient stencil ----------------------------------------------
// phib(y) = T.phi(y) + sum over links k and signs s of s * 1.5 w_k e_k . T.grad(x)
// for every node x whose stencil point x + s e_k maps onto y (directly, through
// a periodic image or through a mirror ghost).
template <class L, typename R>
__global__ void __launch_bounds__(kAdjThreads)
k_adj_finish(const KParams K, AdjWork<R> T, R* __restrict__ phib_out, R* __restrict__ cb_out) {
    const StepParams& P = K.P;
    const long long N = P.N;
    const long long i = blockIdx.x * (long long)kAdjThreads + threadIdx.x;
    if (i >= N) return;
    int y3[3];
    node_coords<L, R>(P, i, y3[0], y3[1], y3[2]);
    const int n3[3] = {P.nx, P.ny, P.nz};
    // per axis, the positions v in [-1, n] with map(v) == y
    int pre[3][3], npre[3];
    for (int a = 0; a < 3; ++a) {
        npre[a] = 0;
        pre[a][npre[a]++] = y3[a];
        if (a == 2 && L::D == 2) continue;
        if (y3[a] == 0) pre[a][npre[a]++] = P.bc[a] ? -1 : n3[a];
        if (y3[a] == n3[a] - 1) pre[a][npre[a]++] = P.bc[a] ? n3[a] : -1;
    }
    R acc = T.phi[i];
#pragma unroll
    for (int k = 1; k < L::Q; ++k) {
        const int e[3] = {L::ex(k), L::ey(k), L::ez(k)};
        for (int s = -1; s <= 1; s += 2) {
            for (int ia = 0; ia < npre[0]; ++ia)
                for (int ib = 0; ib < npre[1]; ++ib)
                    for (int ic = 0; ic < npre[2]; ++ic) {
                        const int x = pre[0][ia] - s * e[0], yy = pre[1][ib] - s * e[1], z = pre[2][ic] - s * e[2];
                        if (x < 0 || x >= P.nx || yy < 0 || yy >= P.ny || z < 0 || z >= P.nz) continue;
                        const long long xi = ((long long)z * P.ny + yy) * P.nx + x;
                        const R t = R(1.5 * L::w(k)) * (R(e[0]) * T.grad[xi] + R(e[1]) * T.grad[N + xi] +
                                                         R(e[2]) * T.grad[2 * N + xi]);
                        acc += s > 0 ? t : -t;
                    }
        }
    }
    phib_out[i] = acc;
    cb_out[i] = T.c[i];
}

// ---- adjoint of the initialisation ----------------------------------------------------
template <class L, typename R>
__global__ void __launch_bounds__(kAdjThreads)
k_adj_init(const KParams K, const R* __restrict__ phi0, const R* __restrict__ c0, const R* __restrict__ gb,
           const R* __restrict__ hb, const R* __restrict__ phib_in, const R* __restrict__ cb_in, AdjWork<R> T,
           double* __restrict__ pacc, int nblk) {
    const StepParams& P = K.P;
    const long long N = P.N;
    const long long i = blockIdx.x * (long long)kAdjThreads + threadIdx.x;
    double pv[kAdjParams] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < N) {
        int x, y, z;
        node_coords<L, R>(P, i, x, y, z);
        NodeFwd<L, R> f;
        f.compute(P, phi0, c0, x, y, z, i);
        R phib = phib_in[i], mub = R(0), cb = cb_in[i], dphib = R(0);
        R Gb[L::Q], heqb[L::Q], Hb[L::Q];
        R gradb[3] = {R(0), R(0), R(0)}, nb[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int j = 0; j < L::Q; ++j) {
            const R gj = gb[(long long)j * N + i], hj = hb[(long long)j * N + i];
            phib += R(L::w(j)) * gj;          // g_j = w_j phi0 - G_j / 2
            Gb[j] = R(-0.5) * gj;
            heqb[j] = hj;                     // h_j = h^eq_j - H_j / 2
            Hb[j] = R(-0.5) * hj;
        }
        adj_c_sources<L, R>(P, f, R(0), heqb, Hb, phib, mub, cb, gradb, nb, dphib, pv);
        adj_phi_sources<L, R>(P, f, Gb, phib, mub, nb, pv);
        R nn = R(0);
        for (int a = 0; a < 3; ++a) nn += f.n[a] * nb[a];
        for (int a = 0; a < 3; ++a) T.grad[a * N + i] = gradb[a] + (nb[a] - f.n[a] * nn) * f.inv;
        T.phi[i] = phib + mub * R(P.c_s - P.c_l);
        T.c[i] = cb + mub;
    }
    adj_param_flush(pv, pacc, nblk);
}

template <typename R>
__global__ void k_adj_to_f64(const R* __restrict__ src, double* __restrict__ dst, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

}  // namespace lbpf
