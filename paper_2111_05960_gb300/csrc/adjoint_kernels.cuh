// Discrete adjoint (reverse mode) of the coupled phi-mu LBM step.
//
// The step is linear in the populations and a smooth function of the fields
// phi and c.  Its adjoint maps the adjoints (gb, hb, phib, cb) of the state at
// step n+1 to those of the state at step n, and accumulates the adjoints of the
// parameters (D_l, tau_g, tau_h, lambda, a, D_s).  Three kernels per step, one
// thread per node on 32 x 8 tiles of each z-plane, no atomics on fields (every
// node gathers what it needs):
//
//   k_adj_h      composition part: pulls hb from downstream neighbours (the
//                transpose of streaming, bounce-back included), then the
//                adjoints of the h collision, of h^eq, of H, of the flux F, of
//                the closure and of the unit normal; leaves per-node partials
//                (phi, c, dphi/dt and grad phi adjoints) in a work area.
//   k_adj_g      phi part: pulls gb and the adjoint of phi^{n+1} (plus that of
//                dphi/dt from k_adj_h) from downstream neighbours, then the
//                adjoints of the g collision and of the sources G; writes the
//                new c adjoint and the local part of the new phi adjoint.
//   k_adj_finish transpose of the gradient stencil, added to the phi adjoint:
//                grad phi(x) = 3 sum_k w_k e_k phi(x + e_k) (Eq. Grad with the
//                directional derivatives of Eq. DerivDirec_Grad, the two halves
//                of each pair merged), so phib(y) += 3 w_k e_k . gradb(x) for
//                every x whose stencil point x + e_k is y, through a periodic
//                image or a mirror ghost near walls.
//
// The sums over links that the adjoint needs are linear in the per-link
// adjoints, so each kernel accumulates them on the fly (sum_k w_k s_k,
// sum_k w_k e_k s_k, and the per-link non-equilibrium products for the
// relaxation-rate adjoints) and keeps no per-link arrays.
//
// k_adj_init is the adjoint of the initialisation (g = w phi - G/2,
// h = h^eq - H/2 at dphi/dt = 0), followed by k_adj_finish.
#pragma once

#include "step_kernels.cuh"

namespace lbpf {

template <typename R>
struct AdjWork {        // per-node partial adjoints, SoA, N entries each
    R* phi;             // phi (local terms of the composition part)
    R* c;               // c
    R* dphi;            // dphi/dt = phi^{n+1} - phi^n
    R* pt;              // phi^{n+1}: the incoming phi adjoint plus that of dphi/dt
    R* grad;            // grad phi, [3][N]
};

#ifndef LBPF_ADJ_BY
#define LBPF_ADJ_BY 8
#endif
constexpr int kAdjBX = 32, kAdjBY = LBPF_ADJ_BY, kAdjThreads = kAdjBX * kAdjBY;
// resident blocks per SM the link kernels are compiled for (register budget).
// FP32 on GB300, reverse sweep of the 128^3 differentiable workload: 4 blocks
// (64 registers, 300-390 bytes of spills) 0.36 ms per step, 3 blocks (80
// registers, 136 / 12 bytes spilled by the h / g kernel) 0.32 ms, 2 blocks (128
// registers, none spilled) 0.35 ms.
#ifndef LBPF_ADJ_MINB_F32
#define LBPF_ADJ_MINB_F32 3
#endif
#ifndef LBPF_ADJ_MINB_F64
#define LBPF_ADJ_MINB_F64 2
#endif
template <typename R>
constexpr int adj_minb() { return sizeof(R) == 8 ? LBPF_ADJ_MINB_F64 : LBPF_ADJ_MINB_F32; }
// the phi part gathers more per link; its register budget is set on its own
#ifndef LBPF_ADJ_MINB_G_F32
#define LBPF_ADJ_MINB_G_F32 LBPF_ADJ_MINB_F32
#endif
template <typename R>
constexpr int adj_minb_g() { return sizeof(R) == 8 ? LBPF_ADJ_MINB_F64 : LBPF_ADJ_MINB_G_F32; }
// Parameter adjoints, in this order: D_l, tau_g, tau_h, lambda, a (of j_at), D_s.
constexpr int kAdjParams = 6;
enum { kPDl = 0, kPTauG = 1, kPTauH = 2, kPLam = 3, kPA = 4, kPDs = 5 };

// Adds the block's sum of each parameter adjoint to its own slot
// acc[j * nblk + block].  Kernels of one sweep run in stream order, so the
// slots need no atomics, and the final sum (k_adj_param_final) has a fixed
// order.  Warps reduce in the compute type, the block in FP64.
template <typename R>
__device__ __forceinline__ void adj_param_flush(R (&v)[kAdjParams], double* __restrict__ acc, int nblk) {
    __shared__ double red[kAdjParams][kAdjThreads / 32];
#pragma unroll
    for (int j = 0; j < kAdjParams; ++j)
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    if (threadIdx.x == 0)
        for (int j = 0; j < kAdjParams; ++j) red[j][threadIdx.y] = (double)v[j];
    __syncthreads();
    const int t = threadIdx.y * kAdjBX + threadIdx.x;
    if (t < kAdjParams) {
        double s = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) s += red[t][w];
        const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        acc[(long long)t * nblk + b] += s;
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

// ---- coefficients ----------------------------------------------------------------

// Constants of one simulation in the compute type, computed once on the host so
// that the FP32 kernels carry no FP64 arithmetic.
template <typename R>
struct AdjCoef {
    R mu_eq, c_l, c_s, dc;      // dc = c_s^co - c_l^co
    R D_l, D_s, Dp, gamma;      // Dp = D_l - D_s
    R omg, omh, eps2, M, lam;
    R atc;                      // a W dc (0 without anti-trapping)
    R Wdc;                      // W dc
    R kct;                      // 4 / W
    R lamM_W2, M_W2, lam_W2;    // lambda M / W^2, M / W^2, lambda / W^2
    R dw8M, dw8;                // 8 M / W^2, 8 / W^2
    R omg2, omh2, gamma2_3;     // omega_g^2, omega_h^2, gamma^2 / 3
    int counter_term;
};

template <typename R>
__host__ AdjCoef<R> make_adj_coef(const StepParams& P) {
    AdjCoef<R> c;
    const double dc = P.c_s - P.c_l, W2 = P.W * P.W;
    c.mu_eq = R(P.mu_eq); c.c_l = R(P.c_l); c.c_s = R(P.c_s); c.dc = R(dc);
    c.D_l = R(P.D_l); c.D_s = R(P.D_s); c.Dp = R(P.D_l - P.D_s); c.gamma = R(P.gamma);
    c.omg = R(P.omg); c.omh = R(P.omh); c.eps2 = R(P.eps2); c.M = R(P.M); c.lam = R(P.lambda);
    c.atc = R(P.a_at * P.W * dc);
    c.Wdc = R(P.W * dc);
    c.kct = R(4.0 / P.W);
    c.lamM_W2 = R(P.lambda * P.M / W2); c.M_W2 = R(P.M / W2); c.lam_W2 = R(P.lambda / W2);
    c.dw8M = R(8.0 * P.M / W2); c.dw8 = R(8.0 / W2);
    c.omg2 = R(P.omg * P.omg); c.omh2 = R(P.omh * P.omh); c.gamma2_3 = R(P.gamma * P.gamma / 3.0);
    c.counter_term = P.counter_term;
    return c;
}

// ---- node geometry --------------------------------------------------------------

// A node and the relative offsets of its -1 / +1 neighbours along each axis:
// the next node, the periodic image across the box, or 0 (the node itself)
// across a half-way wall, where the matching bit of `walls` is set.  With
// these, the stencil point x + e_k of the phi gradient (mirror ghosts at
// walls) is i + off(k), and the node consuming the post-collision population k
// is i + off(k) unless the link crosses a wall (then the population returns to
// this node as population opp(k)).
struct AdjNbr {
    long long i;
    int xp, xm, yp, ym;
    long long zp, zm;
    unsigned walls;     // bit 0: x + 1 beyond a wall, 1: x - 1, 2: y + 1, 3: y - 1, 4: z + 1, 5: z - 1
};

__device__ __forceinline__ void axis_offsets(int c, int n, long long stride, int bc, unsigned bit, long long& op,
                                             long long& om, unsigned& walls) {
    if (c + 1 < n) op = stride;
    else if (bc) { op = 0; walls |= bit; }
    else op = -(long long)(n - 1) * stride;
    if (c > 0) om = -stride;
    else if (bc) { om = 0; walls |= bit << 1; }
    else om = (long long)(n - 1) * stride;
}

template <class L>
__device__ __forceinline__ AdjNbr adj_nbr(const StepParams& P, int x, int y, int z) {
    AdjNbr a;
    const long long nxy = (long long)P.nx * P.ny;
    a.i = z * nxy + (long long)y * P.nx + x;
    a.walls = 0;
    long long p, m;
    axis_offsets(x, P.nx, 1, P.bc[0], 1u, p, m, a.walls);
    a.xp = (int)p;
    a.xm = (int)m;
    axis_offsets(y, P.ny, P.nx, P.bc[1], 4u, p, m, a.walls);
    a.yp = (int)p;
    a.ym = (int)m;
    if (L::D == 3) {
        axis_offsets(z, P.nz, nxy, P.bc[2], 16u, a.zp, a.zm, a.walls);
    } else {
        a.zp = a.zm = 0;
    }
    return a;
}

// Offset of x + e_k (k a constant after unrolling).
template <class L>
__device__ __forceinline__ long long nbr_off(const AdjNbr& a, int k) {
    long long o = 0;
    if (L::ex(k)) o += L::ex(k) > 0 ? a.xp : a.xm;
    if (L::ey(k)) o += L::ey(k) > 0 ? a.yp : a.ym;
    if (L::ez(k)) o += L::ez(k) > 0 ? a.zp : a.zm;
    return o;
}

// Wall bits that link k crosses when it leaves a node ...
template <class L>
__host__ __device__ constexpr unsigned out_bits(int k) {
    return (L::ex(k) > 0 ? 1u : 0u) | (L::ex(k) < 0 ? 2u : 0u) | (L::ey(k) > 0 ? 4u : 0u) |
           (L::ey(k) < 0 ? 8u : 0u) | (L::ez(k) > 0 ? 16u : 0u) | (L::ez(k) < 0 ? 32u : 0u);
}

template <class L, typename R>
__device__ __forceinline__ R edot3(int k, const R (&v)[3]) {
    return R(L::ex(k)) * v[0] + R(L::ey(k)) * v[1] + R(L::ez(k)) * v[2];
}

// acc += w_k e_k s with the zero components dropped
template <class L, typename R>
__device__ __forceinline__ void add_we(int k, R s, R (&acc)[3]) {
    const R ws = R(L::w(k)) * s;
    if (L::ex(k)) acc[0] += L::ex(k) > 0 ? ws : -ws;
    if (L::ey(k)) acc[1] += L::ey(k) > 0 ? ws : -ws;
    if (L::ez(k)) acc[2] += L::ez(k) > 0 ? ws : -ws;
}

// e_k . v(i) for a [3][N] array v, the zero components of e_k not loaded
template <class L, typename R>
__device__ __forceinline__ R edot_at(int k, const R* __restrict__ v, long long N, long long i) {
    R s = R(0);
    if (L::ex(k)) s += L::ex(k) > 0 ? v[i] : -v[i];
    if (L::ey(k)) s += L::ey(k) > 0 ? v[N + i] : -v[N + i];
    if (L::ez(k)) s += L::ez(k) > 0 ? v[2 * N + i] : -v[2 * N + i];
    return s;
}

// Forward quantities of one node recomputed from phi^n and c^n.
template <class L, typename R>
struct NodeFwd {
    R ph, cc, mu, g[3], n[3], inv;
    __device__ __forceinline__ void compute(const AdjCoef<R>& C, const R* __restrict__ phi,
                                            const R* __restrict__ c, const AdjNbr& a) {
        ph = phi[a.i];
        cc = c[a.i];
        mu = C.mu_eq + cc - (C.c_l * ph + C.c_s * (R(1) - ph));
        g[0] = g[1] = g[2] = R(0);
#pragma unroll
        for (int k = 1; k < L::Q; ++k) add_we<L, R>(k, R(3) * phi[a.i + nbr_off<L>(a, k)], g);
        inv = R(1) / sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + C.eps2);
        for (int d = 0; d < 3; ++d) n[d] = g[d] * inv;
    }
    // flux F = mu D' grad phi + j_at (Eq. SourceTerm_LBE_h)
    __device__ __forceinline__ void flux(const AdjCoef<R>& C, R dphi, R (&F)[3]) const {
        const R at = C.atc * dphi;
        for (int d = 0; d < 3; ++d) F[d] = mu * C.Dp * g[d] + at * n[d];
    }
};

// Adjoint of the closure mu = mu_eq + c - c^co(phi) and of the unit normal
// n = grad / sqrt(|grad|^2 + eps^2): folds mub into phib, cb and nb into gradb.
template <class L, typename R>
__device__ __forceinline__ void adj_closure_normal(const AdjCoef<R>& C, const NodeFwd<L, R>& f, R mub,
                                                   const R (&nb)[3], R& phib, R& cb, R (&gradb)[3]) {
    phib += mub * C.dc;
    cb += mub;
    const R nn = f.n[0] * nb[0] + f.n[1] * nb[1] + f.n[2] * nb[2];
    for (int d = 0; d < 3; ++d) gradb[d] += (nb[d] - f.n[d] * nn) * f.inv;
}

// Adjoint of h^eq (through Q = gamma D mu) and of H = gamma w_k e_k . F at one
// node, given Qb = sum_k heqb_k dh^eq_k/dQ and HbV = sum_k w_k e_k Hb_k; the
// heqb_0 term of c is added by the caller.  Adds to phib, mub, gradb, nb, dphib
// and the parameter adjoints.
template <class L, typename R>
__device__ __forceinline__ void adj_c_sources(const AdjCoef<R>& C, const NodeFwd<L, R>& f, R dphi, R Qb,
                                              const R (&HbV)[3], R& phib, R& mub, R (&gradb)[3], R (&nb)[3],
                                              R& dphib, R (&pv)[kAdjParams]) {
    const R D = C.D_l * f.ph + C.D_s * (R(1) - f.ph);
    R F[3];
    f.flux(C, dphi, F);
    const R gammab = Qb * D * f.mu + F[0] * HbV[0] + F[1] * HbV[1] + F[2] * HbV[2];
    const R Db = Qb * C.gamma * f.mu;
    mub += Qb * C.gamma * D;
    phib += Db * C.Dp;
    pv[kPDl] += Db * f.ph;
    pv[kPDs] += Db * (R(1) - f.ph);
    const R Fb[3] = {C.gamma * HbV[0], C.gamma * HbV[1], C.gamma * HbV[2]};
    const R Fg = Fb[0] * f.g[0] + Fb[1] * f.g[1] + Fb[2] * f.g[2];
    const R Fn = Fb[0] * f.n[0] + Fb[1] * f.n[1] + Fb[2] * f.n[2];
    mub += C.Dp * Fg;
    pv[kPDl] += f.mu * Fg;
    pv[kPDs] -= f.mu * Fg;
    for (int d = 0; d < 3; ++d) {
        gradb[d] += f.mu * C.Dp * Fb[d];
        nb[d] += C.atc * dphi * Fb[d];
    }
    dphib += C.atc * Fn;
    pv[kPA] += C.Wdc * dphi * Fn;
    pv[kPTauH] -= gammab * C.gamma2_3;                      // gamma = 3 / tau_h
}

// The phi source of one node: G_k = w_k (A + curv_k), A = G^st (Eq. SourceG_ST),
// curv_k = K e_k . n (counter term, Eq. SourceG_CT) or the double-well term
// (Eq. SourceG_dw, no k dependence).
template <class L, typename R>
struct PhiSource {
    R pq, S, A, K, dw;
    __device__ __forceinline__ void compute(const AdjCoef<R>& C, const NodeFwd<L, R>& f) {
        pq = f.ph * (R(1) - f.ph);
        S = R(6) * pq * C.dc * (f.mu - C.mu_eq);
        A = -C.lamM_W2 * S;
        K = C.kct * pq;
        dw = -C.dw8M * (R(2) * pq * (R(1) - R(2) * f.ph));
    }
    // G_k with the switch resolved once per node, so the link loops carry no branch
    __device__ __forceinline__ void per_link(const AdjCoef<R>& C, R& a0, R& kn) const {
        a0 = A + (C.counter_term ? R(0) : dw);
        kn = C.counter_term ? K : R(0);
    }
    __device__ __forceinline__ R G(int k, R a0, R kn, const NodeFwd<L, R>& f) const {
        return R(L::w(k)) * (a0 + kn * edot3<L, R>(k, f.n));
    }
};

// Adjoint of the phi sources given Gstb = sum_k w_k Gb_k and GbV = sum_k w_k e_k Gb_k;
// adds to phib, mub, nb and the parameter adjoints.
template <class L, typename R>
__device__ __forceinline__ void adj_phi_sources(const AdjCoef<R>& C, const NodeFwd<L, R>& f,
                                                const PhiSource<L, R>& s, R Gstb, const R (&GbV)[3], R& phib,
                                                R& mub, R (&nb)[3], R (&pv)[kAdjParams]) {
    const R Sb = -Gstb * C.lamM_W2;
    pv[kPLam] -= Gstb * C.M_W2 * s.S;
    pv[kPTauG] -= Gstb * C.lam_W2 * s.S * R(1.0 / 3.0);    // M = tau_g / 3
    phib += Sb * R(6) * C.dc * (R(1) - R(2) * f.ph) * (f.mu - C.mu_eq);
    mub += Sb * R(6) * C.dc * s.pq;
    if (C.counter_term) {
        const R Kb = GbV[0] * f.n[0] + GbV[1] * f.n[1] + GbV[2] * f.n[2];
        for (int d = 0; d < 3; ++d) nb[d] += s.K * GbV[d];
        phib += Kb * C.kct * (R(1) - R(2) * f.ph);
    } else {
        const R wp = R(2) * s.pq * (R(1) - R(2) * f.ph);
        const R wpp = R(2) - R(12) * f.ph + R(12) * f.ph * f.ph;
        phib -= Gstb * C.dw8M * wpp;
        pv[kPTauG] -= Gstb * C.dw8 * wp * R(1.0 / 3.0);
    }
}

// ---- composition part ---------------------------------------------------------
// WALLS = false: a fully periodic domain, where no link ever bounces back.
template <class L, typename R, bool WALLS>
__global__ void __launch_bounds__(kAdjThreads, adj_minb<R>())
k_adj_h(const StepParams P, const AdjCoef<R> C, const R* __restrict__ h, const R* __restrict__ phi,
        const R* __restrict__ c, const R* __restrict__ phi1, const R* __restrict__ hb_in,
        const R* __restrict__ cb_in, const R* __restrict__ phib_in, R* __restrict__ hb_out, AdjWork<R> T,
        double* __restrict__ pacc, int nblk) {
    const long long N = P.N;
    R pv[kAdjParams] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    const int x = blockIdx.x * kAdjBX + threadIdx.x, y = blockIdx.y * kAdjBY + threadIdx.y;
    for (int z = blockIdx.z; z < P.nz && x < P.nx && y < P.ny; z += gridDim.z) {
        const AdjNbr a = adj_nbr<L>(P, x, y, z);
        const long long i = a.i;
        NodeFwd<L, R> f;
        f.compute(C, phi, c, a);
        const R dphi = phi1[i] - f.ph;
        const R Q = C.gamma * (C.D_l * f.ph + C.D_s * (R(1) - f.ph)) * f.mu;
        R F[3];
        f.flux(C, dphi, F);
        // s_k: adjoint of the post-collision population k (transpose of streaming;
        // c' = sum_k h'_k adds cb to every link)
        R s0 = R(0), S1 = R(0), SV[3] = {R(0), R(0), R(0)}, Sneq = R(0);
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const long long d = i + nbr_off<L>(a, k);
            const bool wall = WALLS && (a.walls & out_bits<L>(k)) != 0;
            const R s = wall ? hb_in[(long long)L::opp(k) * N + i] + cb_in[i] : hb_in[(long long)k * N + d] + cb_in[d];
            hb_out[(long long)k * N + i] = (R(1) - C.omh) * s;
            const R heq = k == 0 ? f.cc - R(1.0 - L::w(0)) * Q : R(L::w(k)) * Q;
            const R Hk = C.gamma * R(L::w(k)) * edot3<L, R>(k, F);
            Sneq += s * (heq - R(0.5) * Hk - h[(long long)k * N + i]);
            if (k == 0) {
                s0 = s;
            } else {
                S1 += R(L::w(k)) * s;
                add_we<L, R>(k, s, SV);
            }
        }
        pv[kPTauH] -= Sneq * C.omh2;                        // omega_h = 1 / (tau_h + 1/2)
        // adjoints of h^eq_k and H_k: omh s_k and (1 - omh/2) s_k
        const R Qb = C.omh * (S1 - R(1.0 - L::w(0)) * s0);
        const R hh = R(1) - R(0.5) * C.omh;
        const R HbV[3] = {hh * SV[0], hh * SV[1], hh * SV[2]};
        R phib = R(0), mub = R(0), cb = C.omh * s0, dphib = R(0);
        R gradb[3] = {R(0), R(0), R(0)}, nb[3] = {R(0), R(0), R(0)};
        adj_c_sources<L, R>(C, f, dphi, Qb, HbV, phib, mub, gradb, nb, dphib, pv);
        adj_closure_normal<L, R>(C, f, mub, nb, phib, cb, gradb);
        T.phi[i] = phib;
        T.c[i] = cb;
        T.dphi[i] = dphib;
        T.pt[i] = phib_in[i] + dphib;
        for (int d = 0; d < 3; ++d) T.grad[d * N + i] = gradb[d];
    }
    adj_param_flush(pv, pacc, nblk);
}

// ---- phi part ---------------------------------------------------------------------
template <class L, typename R, bool WALLS>
__global__ void __launch_bounds__(kAdjThreads, adj_minb_g<R>())
k_adj_g(const StepParams P, const AdjCoef<R> C, const R* __restrict__ g, const R* __restrict__ phi,
        const R* __restrict__ c, const R* __restrict__ gb_in, R* __restrict__ gb_out, AdjWork<R> T,
        R* __restrict__ phib_out, R* __restrict__ cb_out, double* __restrict__ pacc, int nblk) {
    const long long N = P.N;
    R pv[kAdjParams] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    const int x = blockIdx.x * kAdjBX + threadIdx.x, y = blockIdx.y * kAdjBY + threadIdx.y;
    for (int z = blockIdx.z; z < P.nz && x < P.nx && y < P.ny; z += gridDim.z) {
        const AdjNbr a = adj_nbr<L>(P, x, y, z);
        const long long i = a.i;
        NodeFwd<L, R> f;
        f.compute(C, phi, c, a);
        PhiSource<L, R> src;
        src.compute(C, f);
        // The work area is read-only in this kernel except for the gradient
        // adjoint: its reads go through the non-coherent path, so the compiler
        // may issue them ahead of the gb_out stores (a plain load through the
        // unqualified AdjWork pointers could alias them and would serialise the
        // link loop on memory latency).
        const R dphib_here = __ldg(T.dphi + i);
        const R pt = __ldg(T.pt + i);                    // adjoint of phi^{n+1} at this node
        R ga0, gkn;
        src.per_link(C, ga0, gkn);
        // s_k: adjoint of the post-collision population k; phi^{n+1} = sum g' + G/2
        R S0 = R(0), SV[3] = {R(0), R(0), R(0)}, Sneq = R(0);
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const long long d = i + nbr_off<L>(a, k);
            const bool wall = WALLS && (a.walls & out_bits<L>(k)) != 0;
            const R s = wall ? gb_in[(long long)L::opp(k) * N + i] + pt
                             : gb_in[(long long)k * N + d] + __ldg(T.pt + d);
            gb_out[(long long)k * N + i] = (R(1) - C.omg) * s;
            Sneq += s * (R(L::w(k)) * f.ph - R(0.5) * src.G(k, ga0, gkn, f) - g[(long long)k * N + i]);
            S0 += R(L::w(k)) * s;
            add_we<L, R>(k, s, SV);
        }
        pv[kPTauG] -= Sneq * C.omg2;
        R phib = C.omg * S0 - dphib_here;                // g^eq = w phi; dphi = phi^{n+1} - phi^n
        // adjoint of G_k = (1 - omg/2) s_k + pt/2; sum_k w_k = 1, sum_k w_k e_k = 0
        const R hg = R(1) - R(0.5) * C.omg;
        const R Gstb = hg * S0 + R(0.5) * pt;
        const R GbV[3] = {hg * SV[0], hg * SV[1], hg * SV[2]};
        R mub = R(0), cb = R(0), nb[3] = {R(0), R(0), R(0)}, gradb[3] = {R(0), R(0), R(0)};
        adj_phi_sources<L, R>(C, f, src, Gstb, GbV, phib, mub, nb, pv);
        adj_closure_normal<L, R>(C, f, mub, nb, phib, cb, gradb);
        for (int d = 0; d < 3; ++d) T.grad[d * N + i] += gradb[d];
        phib_out[i] = __ldg(T.phi + i) + phib;
        cb_out[i] = __ldg(T.c + i) + cb;
    }
    adj_param_flush(pv, pacc, nblk);
}

// ---- transpose of the gradient stencil ----------------------------------------------
// Node y receives 3 w_k e_k . gradb(x) from every x with S(x + e_k) = y, S the
// stencil map.  Per axis with component e of e_k: e = 0 gives x = y; e = +1
// gives the -1 neighbour (unless y - 1 is beyond a wall) and, at a wall on the
// +1 side, y itself (its mirror ghost); e = -1 likewise with the sides swapped.
// Warps without wall nodes take the single-source form.
template <class L, typename R>
__device__ __forceinline__ R finish_link_general(int k, const AdjNbr& a, const R* __restrict__ gradb, long long N) {
    // options per axis: 0 = neighbour on the side opposite to e, 1 = the node itself
    const int e[3] = {L::ex(k), L::ey(k), L::ez(k)};
    R acc = R(0);
#pragma unroll
    for (int ox = 0; ox < 2; ++ox)
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
            for (int oz = 0; oz < 2; ++oz) {
                const int o[3] = {ox, oy, oz};
                bool ok = true;
                long long off = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (e[d] == 0) {
                        ok = ok && o[d] == 0;
                        continue;
                    }
                    const unsigned far = 1u << (2 * d + (e[d] > 0 ? 0 : 1));    // wall beyond y + e
                    const unsigned near = 1u << (2 * d + (e[d] > 0 ? 1 : 0));   // wall beyond y - e
                    if (o[d] == 0) {
                        ok = ok && !(a.walls & near);
                        const long long nb = d == 0 ? (e[d] > 0 ? a.xm : a.xp)
                                                    : (d == 1 ? (e[d] > 0 ? a.ym : a.yp) : (e[d] > 0 ? a.zm : a.zp));
                        off += nb;
                    } else {
                        ok = ok && (a.walls & far);
                    }
                }
                if (ok) acc += edot_at<L, R>(k, gradb, N, a.i + off);
            }
    return acc;
}

template <class L, typename R>
__global__ void __launch_bounds__(kAdjThreads)
k_adj_finish(const StepParams P, const R* __restrict__ gradb, R* __restrict__ phib) {
    const long long N = P.N;
    const int x = blockIdx.x * kAdjBX + threadIdx.x, y = blockIdx.y * kAdjBY + threadIdx.y;
    for (int z = blockIdx.z; z < P.nz && x < P.nx && y < P.ny; z += gridDim.z) {
        const AdjNbr a = adj_nbr<L>(P, x, y, z);
        R acc = R(0);
        if (!__any_sync(__activemask(), a.walls != 0)) {
#pragma unroll
            for (int k = 1; k < L::Q; ++k)
                acc += R(3.0 * L::w(k)) * edot_at<L, R>(k, gradb, N, a.i + nbr_off<L>(a, L::opp(k)));
        } else {
#pragma unroll
            for (int k = 1; k < L::Q; ++k) acc += R(3.0 * L::w(k)) * finish_link_general<L, R>(k, a, gradb, N);
        }
        phib[a.i] += acc;
    }
}

// ---- adjoint of the initialisation ----------------------------------------------------
template <class L, typename R>
__global__ void __launch_bounds__(kAdjThreads, adj_minb<R>())
k_adj_init(const StepParams P, const AdjCoef<R> C, const R* __restrict__ phi0, const R* __restrict__ c0,
           const R* __restrict__ gb, const R* __restrict__ hb, const R* __restrict__ phib_in,
           const R* __restrict__ cb_in, R* __restrict__ gradb_out, R* __restrict__ phib_out, R* __restrict__ cb_out,
           double* __restrict__ pacc, int nblk) {
    const long long N = P.N;
    R pv[kAdjParams] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    const int x = blockIdx.x * kAdjBX + threadIdx.x, y = blockIdx.y * kAdjBY + threadIdx.y;
    for (int z = blockIdx.z; z < P.nz && x < P.nx && y < P.ny; z += gridDim.z) {
        const AdjNbr a = adj_nbr<L>(P, x, y, z);
        const long long i = a.i;
        NodeFwd<L, R> f;
        f.compute(C, phi0, c0, a);
        PhiSource<L, R> src;
        src.compute(C, f);
        // g_k = w_k phi0 - G_k/2 and h_k = h^eq_k - H_k/2 (dphi/dt = 0)
        R Gw = R(0), GV[3] = {R(0), R(0), R(0)}, H1 = R(0), HV[3] = {R(0), R(0), R(0)}, h0 = R(0);
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const R gk = gb[(long long)k * N + i], hk = hb[(long long)k * N + i];
            Gw += R(L::w(k)) * gk;
            add_we<L, R>(k, gk, GV);
            add_we<L, R>(k, hk, HV);
            if (k == 0) h0 = hk; else H1 += R(L::w(k)) * hk;
        }
        R phib = phib_in[i] + Gw, mub = R(0), cb = cb_in[i] + h0, dphib = R(0);
        R gradb[3] = {R(0), R(0), R(0)}, nb[3] = {R(0), R(0), R(0)};
        const R Qb = H1 - R(1.0 - L::w(0)) * h0;
        const R HbV[3] = {R(-0.5) * HV[0], R(-0.5) * HV[1], R(-0.5) * HV[2]};
        adj_c_sources<L, R>(C, f, R(0), Qb, HbV, phib, mub, gradb, nb, dphib, pv);
        const R GbV[3] = {R(-0.5) * GV[0], R(-0.5) * GV[1], R(-0.5) * GV[2]};
        adj_phi_sources<L, R>(C, f, src, R(-0.5) * Gw, GbV, phib, mub, nb, pv);
        adj_closure_normal<L, R>(C, f, mub, nb, phib, cb, gradb);
        for (int d = 0; d < 3; ++d) gradb_out[d * N + i] = gradb[d];
        phib_out[i] = phib;
        cb_out[i] = cb;
    }
    adj_param_flush(pv, pacc, nblk);
}

template <typename R>
__global__ void k_adj_to_f64(const R* __restrict__ src, double* __restrict__ dst, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

}  // namespace lbpf
