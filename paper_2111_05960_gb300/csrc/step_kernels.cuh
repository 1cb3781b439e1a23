// Kernels of the coupled phi-mu lattice Boltzmann time step (arXiv 2111.05960,
// Sec. 3), for sm_103a.
//
// One time step n -> n+1 is two launches over the whole grid:
//
//   phi kernel   pulls g_k(x, n+1) = g*_k(x - e_k, n)   (Eq. LBE_PhaseField_Eq)
//                and writes phi^{n+1} = sum_k g_k + 1/2 sum_k G_k (Eq. Moment_Phi)
//   c kernel     pulls h_k(x, n+1) = h*_k(x - e_k, n)   (Eq. LBE_Composition),
//                with dphi/dt = phi^{n+1} - phi^n in j_at, and writes
//                c^{n+1} = sum_k h_k (Eq. Moment0_LBM_Concent)
//
// The collision of a population is evaluated at its upstream node.  Everything
// a collision needs from that node (the source G_k or H_k, the equilibrium) is
// an affine function of e_k:
//
//   g*_k(y) = (1 - w_g) g_k(y) + w_k [ alpha_g(y) + e_k . beta_g(y) ]
//       alpha_g = w_g phi + (1 - w_g/2) (G^st + G^dw),  beta_g = (1 - w_g/2) G^ct-vector
//   h*_k(y) = (1 - w_h) h_k(y) + w_k [ w_h P(y) + e_k . beta_h(y) ]        (k != 0)
//   h*_0(x) = (1 - w_h) h_0(x) + w_h [ c(x) - (1 - w_0) P(x) ]
//       P = gamma D(phi) mu,  beta_h = (1 - w_h/2) gamma F,  F = mu D' grad phi + j_at
//
// with w_g = 1/(tau_g + 1/2), w_h = 1/(tau_h + 1/2).  These per-node
// "ingredients" need grad(phi) (a radius-1 stencil of phi), so each block
// stages phi^n of its tile plus a 2-node halo in shared memory, evaluates the
// ingredients once per node of the tile plus a 1-node ring, and then every
// thread pulls its Q populations with coalesced loads along x.
//
// Walls: half-way bounce-back.  A pull whose upstream node lies beyond a wall
// takes the opposite population post-collision at the node itself; the phi
// stencil sees mirror ghosts phi(-1) = phi(0), phi(-2) = phi(1).
#pragma once

#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "lattice.cuh"

namespace lbpf {

// Scalars of one simulation, in lattice units (converted once on the host).
struct StepParams {
    int nx, ny, nz;
    int bc[3];          // 0 periodic, 1 bounce-back
    long long N;        // nx * ny * nz
    double omg, omh;    // 1 / (tau + 1/2)
    double M;           // M_phi = tau_g / 3
    double gamma;       // 3 / tau_h
    double W, lambda, D_l, D_s, c_s, c_l, mu_eq;
    double a_at;        // a of j_at, 0 when anti-trapping is off
    double eps2;        // eps_n^2
    int counter_term;
};

// ---- storage policies --------------------------------------------------------
// A policy maps a population between its stored form and the compute type.
// `ref` is the population's equilibrium value at the node it is stored at; the
// plain policies ignore it, the deviation policies store v - ref in 16 bits.

struct StoreF64 {
    using real = double;
    using store_t = double;
    __device__ static __forceinline__ real load(const store_t* p, long long i, real) { return p[i]; }
    __device__ static __forceinline__ void store(store_t* p, long long i, real v, real) { p[i] = v; }
    static constexpr bool deviation = false;
};

struct StoreF32 {
    using real = float;
    using store_t = float;
    __device__ static __forceinline__ real load(const store_t* p, long long i, real) { return p[i]; }
    __device__ static __forceinline__ void store(store_t* p, long long i, real v, real) { p[i] = v; }
    static constexpr bool deviation = false;
};

// Deviations are scaled by 2^12 before rounding to 16 bits, so that the small
// non-equilibrium parts stay in the normal range of FP16.
struct StoreF16Dev {
    using real = float;
    using store_t = __half;
    static constexpr float S = 4096.0f, INV = 1.0f / 4096.0f;
    __device__ static __forceinline__ real load(const store_t* p, long long i, real ref) {
        return fmaf(__half2float(p[i]), INV, ref);
    }
    __device__ static __forceinline__ void store(store_t* p, long long i, real v, real ref) {
        p[i] = __float2half_rn((v - ref) * S);
    }
    static constexpr bool deviation = true;
};

struct StoreBF16Dev {
    using real = float;
    using store_t = __nv_bfloat16;
    __device__ static __forceinline__ real load(const store_t* p, long long i, real ref) {
        return __bfloat162float(p[i]) + ref;
    }
    __device__ static __forceinline__ void store(store_t* p, long long i, real v, real ref) {
        p[i] = __float2bfloat16_rn(v - ref);
    }
    static constexpr bool deviation = true;
};

// ---- helpers ------------------------------------------------------------------

__device__ __forceinline__ int map_coord(int i, int n, int bc) {
    if (bc == 0) {
        i %= n;
        return i < 0 ? i + n : i;
    }
    // mirror ghost across a half-way wall; one reflection covers a 2-node halo
    // when n >= 2 (checked on the host)
    if (i < 0) i = -1 - i;
    if (i >= n) i = 2 * n - 1 - i;
    return i;
}

// e_k . v with the zero components dropped at compile time (k is a constant
// after unrolling).
template <class L, typename R>
__device__ __forceinline__ R edot(int k, R vx, R vy, R vz) {
    R s = R(0);
    if (L::ex(k) > 0) s += vx;
    if (L::ex(k) < 0) s -= vx;
    if (L::ey(k) > 0) s += vy;
    if (L::ey(k) < 0) s -= vy;
    if (L::D == 3) {
        if (L::ez(k) > 0) s += vz;
        if (L::ez(k) < 0) s -= vz;
    }
    return s;
}

// grad(phi) by directional derivatives (Eq. DerivDirec_Grad, Eq. Grad) from a
// shared-memory tile; `c` is the node's offset in the tile, sx/sy the strides.
template <class L, typename R>
__device__ __forceinline__ void tile_gradient(const R* t, int c, int sx, int sy, R& gx, R& gy, R& gz) {
    gx = gy = gz = R(0);
#pragma unroll
    for (int k = 1; k < L::Q; ++k) {
        const int off = L::ex(k) + L::ey(k) * sx + L::ez(k) * sy;
        const R dk = R(0.5) * (t[c + off] - t[c - off]);
        const R cw = R(3.0 * L::w(k));
        if (L::ex(k) > 0) gx += cw * dk;
        if (L::ex(k) < 0) gx -= cw * dk;
        if (L::ey(k) > 0) gy += cw * dk;
        if (L::ey(k) < 0) gy -= cw * dk;
        if (L::D == 3) {
            if (L::ez(k) > 0) gz += cw * dk;
            if (L::ez(k) < 0) gz -= cw * dk;
        }
    }
}

template <typename R>
__device__ __forceinline__ R rsqrt_reg(R g2, R eps2);
template <>
__device__ __forceinline__ double rsqrt_reg<double>(double g2, double eps2) { return 1.0 / sqrt(g2 + eps2); }
template <>
__device__ __forceinline__ float rsqrt_reg<float>(float g2, float eps2) { return 1.0f / sqrtf(g2 + eps2); }

// G^st + G^dw: the isotropic part of G_k / w_k (Eq. SourceG_ST, Eq. SourceG_dw;
// S_phi of Eq. SourceTerm_Coexistence with p' = 6 phi (1 - phi)).
template <typename R>
__device__ __forceinline__ R g_isotropic(const StepParams& P, R phi, R mu) {
    const R one = R(1);
    const R S = R(6) * phi * (one - phi) * R(P.c_s - P.c_l) * (mu - R(P.mu_eq));
    R A = -R(P.lambda) * R(P.M) * S / (R(P.W) * R(P.W));
    if (!P.counter_term) {
        const R wp = R(2) * phi * (one - phi) * (one - R(2) * phi);
        A -= (R(8) * R(P.M) / (R(P.W) * R(P.W))) * wp;
    }
    return A;
}

template <typename R>
__device__ __forceinline__ R closure_mu(const StepParams& P, R phi, R c) {
    return R(P.mu_eq) + c - (R(P.c_l) * phi + R(P.c_s) * (R(1) - phi));
}

// P = gamma D(phi) mu with D = D_l phi + D_s (1 - phi) (Sec. 2.3.3).
template <typename R>
__device__ __forceinline__ R p_term(const StepParams& P, R phi, R mu) {
    const R D = R(P.D_l) * phi + R(P.D_s) * (R(1) - phi);
    return R(P.gamma) * D * mu;
}

// ---- tile geometry -------------------------------------------------------------

template <class L, int BY, int BZ>
struct Tile {
    static constexpr int BX = 32;
    static constexpr int RZ = (L::D == 3) ? 1 : 0;
    static constexpr int X2 = BX + 4, Y2 = BY + 4, Z2 = BZ + 4 * RZ;   // phi halo 2
    static constexpr int X1 = BX + 2, Y1 = BY + 2, Z1 = BZ + 2 * RZ;   // ingredient ring 1
    static constexpr int N2 = X2 * Y2 * Z2;
    static constexpr int N1 = X1 * Y1 * Z1;
    static constexpr int NT = BX * BY * BZ;
};

// Load phi of the tile plus a 2-node halo (wrapped or mirrored).
template <class L, int BY, int BZ, typename R>
__device__ __forceinline__ void load_phi_halo(const StepParams& P, const R* __restrict__ phi, R* s,
                                              int x0, int y0, int z0) {
    using T = Tile<L, BY, BZ>;
    const int tid = threadIdx.x + T::BX * (threadIdx.y + BY * threadIdx.z);
    for (int s_i = tid; s_i < T::N2; s_i += T::NT) {
        const int lx = s_i % T::X2;
        const int ly = (s_i / T::X2) % T::Y2;
        const int lz = s_i / (T::X2 * T::Y2);
        const int gx = map_coord(x0 + lx - 2, P.nx, P.bc[0]);
        const int gy = map_coord(y0 + ly - 2, P.ny, P.bc[1]);
        const int gz = (L::D == 3) ? map_coord(z0 + lz - 2, P.nz, P.bc[2]) : 0;
        s[s_i] = phi[((long long)gz * P.ny + gy) * P.nx + gx];
    }
}

// ---- phi kernel ------------------------------------------------------------------

template <class L, class SP, int BY, int BZ>
__global__ void __launch_bounds__(32 * BY * BZ)
k_phi_step(const StepParams P, const typename SP::store_t* __restrict__ gin,
           typename SP::store_t* __restrict__ gout, const typename SP::real* __restrict__ phi_n,
           const typename SP::real* __restrict__ c_n, typename SP::real* __restrict__ phi_np1) {
    using R = typename SP::real;
    using T = Tile<L, BY, BZ>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sphi = reinterpret_cast<R*>(smem_raw);
    R* s_alpha = sphi + T::N2;           // alpha_g
    R* s_bx = s_alpha + T::N1;           // beta_g
    R* s_by = s_bx + T::N1;
    R* s_bz = s_by + T::N1;              // (3-D only)
    R* s_A = s_bz + (L::D == 3 ? T::N1 : 0);  // G^st + G^dw, for the phi moment

    const int x0 = blockIdx.x * T::BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * BZ;
    const int tid = threadIdx.x + T::BX * (threadIdx.y + BY * threadIdx.z);
    const R omg = R(P.omg);
    const R half_src = R(1) - R(0.5) * omg;

    load_phi_halo<L, BY, BZ>(P, phi_n, sphi, x0, y0, z0);
    __syncthreads();

    // ingredients on the tile plus a 1-node ring
    for (int s_i = tid; s_i < T::N1; s_i += T::NT) {
        const int lx = s_i % T::X1;
        const int ly = (s_i / T::X1) % T::Y1;
        const int lz = s_i / (T::X1 * T::Y1);
        const int c2 = (lx + 1) + T::X2 * ((ly + 1) + T::Y2 * (lz + T::RZ));
        const int gx = map_coord(x0 + lx - 1, P.nx, P.bc[0]);
        const int gy = map_coord(y0 + ly - 1, P.ny, P.bc[1]);
        const int gz = (L::D == 3) ? map_coord(z0 + lz - 1, P.nz, P.bc[2]) : 0;
        const R ph = sphi[c2];
        const R c = c_n[((long long)gz * P.ny + gy) * P.nx + gx];
        const R mu = closure_mu(P, ph, c);
        const R A = g_isotropic(P, ph, mu);
        s_A[s_i] = A;
        s_alpha[s_i] = omg * ph + half_src * A;
        if (P.counter_term) {
            R gx_, gy_, gz_;
            tile_gradient<L>(sphi, c2, T::X2, T::X2 * T::Y2, gx_, gy_, gz_);
            const R inv = rsqrt_reg<R>(gx_ * gx_ + gy_ * gy_ + gz_ * gz_, R(P.eps2));
            const R kct = half_src * (R(4) / R(P.W)) * ph * (R(1) - ph) * inv;  // (4/W) phi(1-phi) n
            s_bx[s_i] = kct * gx_;
            s_by[s_i] = kct * gy_;
            if (L::D == 3) s_bz[s_i] = kct * gz_;
        } else {
            s_bx[s_i] = R(0);
            s_by[s_i] = R(0);
            if (L::D == 3) s_bz[s_i] = R(0);
        }
    }
    __syncthreads();

    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    if (x >= P.nx || y >= P.ny || z >= P.nz) return;
    const long long N = P.N;
    const long long xi = ((long long)z * P.ny + y) * P.nx + x;
    const int c1 = (tx + 1) + T::X1 * ((ty + 1) + T::Y1 * (tz + T::RZ));
    const int c2 = (tx + 2) + T::X2 * ((ty + 2) + T::Y2 * (tz + 2 * T::RZ));

    R v[L::Q];
    R sum = R(0);
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const int ux = x - L::ex(k), uy = y - L::ey(k), uz = z - L::ez(k);
        bool wall = false;
        if (L::ex(k) != 0 && P.bc[0] && (ux < 0 || ux >= P.nx)) wall = true;
        if (L::ey(k) != 0 && P.bc[1] && (uy < 0 || uy >= P.ny)) wall = true;
        if (L::D == 3 && L::ez(k) != 0 && P.bc[2] && (uz < 0 || uz >= P.nz)) wall = true;
        R val;
        if (wall) {
            // half-way bounce-back: g_k(x, n+1) = g*_{opp k}(x, n)
            const int ko = L::opp(k);
            const R wk = R(L::w(k));
            const R gold = SP::load(gin, (long long)ko * N + xi, wk * sphi[c2]);
            const R bz = (L::D == 3) ? s_bz[c1] : R(0);
            val = (R(1) - omg) * gold + wk * (s_alpha[c1] - edot<L>(k, s_bx[c1], s_by[c1], bz));
        } else {
            const int sx = map_coord(ux, P.nx, P.bc[0]);
            const int sy = map_coord(uy, P.ny, P.bc[1]);
            const int sz = (L::D == 3) ? map_coord(uz, P.nz, P.bc[2]) : 0;
            const long long si = ((long long)sz * P.ny + sy) * P.nx + sx;
            const int o1 = c1 - (L::ex(k) + T::X1 * (L::ey(k) + T::Y1 * L::ez(k)));
            const int o2 = c2 - (L::ex(k) + T::X2 * (L::ey(k) + T::Y2 * L::ez(k)));
            const R wk = R(L::w(k));
            const R gold = SP::load(gin, (long long)k * N + si, wk * sphi[o2]);
            const R bz = (L::D == 3) ? s_bz[o1] : R(0);
            val = (R(1) - omg) * gold + wk * (s_alpha[o1] + edot<L>(k, s_bx[o1], s_by[o1], bz));
        }
        v[k] = val;
        sum += val;
    }
    const R phin = sum + R(0.5) * s_A[c1];
    phi_np1[xi] = phin;
#pragma unroll
    for (int k = 0; k < L::Q; ++k) SP::store(gout, (long long)k * N + xi, v[k], R(L::w(k)) * phin);
}

// ---- composition kernel -------------------------------------------------------------

template <class L, class SP, int BY, int BZ>
__global__ void __launch_bounds__(32 * BY * BZ)
k_c_step(const StepParams P, const typename SP::store_t* __restrict__ hin,
         typename SP::store_t* __restrict__ hout, const typename SP::real* __restrict__ phi_n,
         const typename SP::real* __restrict__ phi_np1, const typename SP::real* __restrict__ c_n,
         typename SP::real* __restrict__ c_np1) {
    using R = typename SP::real;
    using T = Tile<L, BY, BZ>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sphi = reinterpret_cast<R*>(smem_raw);
    R* s_P = sphi + T::N2;               // gamma D mu
    R* s_bx = s_P + T::N1;               // beta_h = (1 - w_h/2) gamma F
    R* s_by = s_bx + T::N1;
    R* s_bz = s_by + T::N1;

    const int x0 = blockIdx.x * T::BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * BZ;
    const int tid = threadIdx.x + T::BX * (threadIdx.y + BY * threadIdx.z);
    const R omh = R(P.omh);
    const R half_src = R(1) - R(0.5) * omh;
    const R Dp = R(P.D_l - P.D_s);
    const R atk = R(P.a_at * P.W * (P.c_s - P.c_l));   // a W (c_s^co - c_l^co), 0 if off

    load_phi_halo<L, BY, BZ>(P, phi_n, sphi, x0, y0, z0);
    __syncthreads();

    for (int s_i = tid; s_i < T::N1; s_i += T::NT) {
        const int lx = s_i % T::X1;
        const int ly = (s_i / T::X1) % T::Y1;
        const int lz = s_i / (T::X1 * T::Y1);
        const int c2 = (lx + 1) + T::X2 * ((ly + 1) + T::Y2 * (lz + T::RZ));
        const int gx = map_coord(x0 + lx - 1, P.nx, P.bc[0]);
        const int gy = map_coord(y0 + ly - 1, P.ny, P.bc[1]);
        const int gz = (L::D == 3) ? map_coord(z0 + lz - 1, P.nz, P.bc[2]) : 0;
        const long long gi = ((long long)gz * P.ny + gy) * P.nx + gx;
        const R ph = sphi[c2];
        const R c = c_n[gi];
        const R mu = closure_mu(P, ph, c);
        s_P[s_i] = p_term(P, ph, mu);
        R gx_, gy_, gz_;
        tile_gradient<L>(sphi, c2, T::X2, T::X2 * T::Y2, gx_, gy_, gz_);
        const R inv = rsqrt_reg<R>(gx_ * gx_ + gy_ * gy_ + gz_ * gz_, R(P.eps2));
        const R dphi = phi_np1[gi] - ph;                  // explicit Euler dphi/dt
        const R jat = atk * dphi * inv;                   // j_at = a W dc dphi n
        const R f = mu * Dp;
        const R kk = half_src * R(P.gamma);
        s_bx[s_i] = kk * (f * gx_ + jat * gx_);
        s_by[s_i] = kk * (f * gy_ + jat * gy_);
        if (L::D == 3) s_bz[s_i] = kk * (f * gz_ + jat * gz_);
    }
    __syncthreads();

    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    if (x >= P.nx || y >= P.ny || z >= P.nz) return;
    const long long N = P.N;
    const long long xi = ((long long)z * P.ny + y) * P.nx + x;
    const int c1 = (tx + 1) + T::X1 * ((ty + 1) + T::Y1 * (tz + T::RZ));
    const R w0 = R(L::w(0));
    const R cx = c_n[xi];

    R v[L::Q];
    // rest population: h*_0 = (1 - w_h) h_0 + w_h h^eq_0, H_0 = 0
    {
        const R Px = s_P[c1];
        const R heq0 = cx - (R(1) - w0) * Px;
        const R h0 = SP::load(hin, xi, heq0);
        v[0] = (R(1) - omh) * h0 + omh * heq0;
    }
    R sum = v[0];
#pragma unroll
    for (int k = 1; k < L::Q; ++k) {
        const int ux = x - L::ex(k), uy = y - L::ey(k), uz = z - L::ez(k);
        bool wall = false;
        if (L::ex(k) != 0 && P.bc[0] && (ux < 0 || ux >= P.nx)) wall = true;
        if (L::ey(k) != 0 && P.bc[1] && (uy < 0 || uy >= P.ny)) wall = true;
        if (L::D == 3 && L::ez(k) != 0 && P.bc[2] && (uz < 0 || uz >= P.nz)) wall = true;
        const R wk = R(L::w(k));
        R val;
        if (wall) {
            const int ko = L::opp(k);
            const R Pp = s_P[c1];
            const R hold = SP::load(hin, (long long)ko * N + xi, wk * Pp);
            const R bz = (L::D == 3) ? s_bz[c1] : R(0);
            val = (R(1) - omh) * hold + wk * (omh * Pp - edot<L>(k, s_bx[c1], s_by[c1], bz));
        } else {
            const int sx = map_coord(ux, P.nx, P.bc[0]);
            const int sy = map_coord(uy, P.ny, P.bc[1]);
            const int sz = (L::D == 3) ? map_coord(uz, P.nz, P.bc[2]) : 0;
            const long long si = ((long long)sz * P.ny + sy) * P.nx + sx;
            const int o1 = c1 - (L::ex(k) + T::X1 * (L::ey(k) + T::Y1 * L::ez(k)));
            const R Pp = s_P[o1];
            const R hold = SP::load(hin, (long long)k * N + si, wk * Pp);
            const R bz = (L::D == 3) ? s_bz[o1] : R(0);
            val = (R(1) - omh) * hold + wk * (omh * Pp + edot<L>(k, s_bx[o1], s_by[o1], bz));
        }
        v[k] = val;
        sum += val;
    }
    c_np1[xi] = sum;
    if (SP::deviation) {
        const R phin = phi_np1[xi];
        const R Pn = p_term(P, phin, closure_mu(P, phin, sum));
        SP::store(hout, xi, v[0], sum - (R(1) - w0) * Pn);
#pragma unroll
        for (int k = 1; k < L::Q; ++k) SP::store(hout, (long long)k * N + xi, v[k], R(L::w(k)) * Pn);
    } else {
#pragma unroll
        for (int k = 0; k < L::Q; ++k) SP::store(hout, (long long)k * N + xi, v[k], R(0));
    }
}

// ---- initialisation -------------------------------------------------------------------
// g_k = w_k phi - G_k/2, h_k = h^eq_k - H_k/2 with H at dphi/dt = 0 (the variable
// change of Sec. 3.1 applied at equilibrium).  Fields phi, c already hold the
// start values in the compute type.

template <class L, class SP>
__global__ void k_init(const StepParams P, const typename SP::real* __restrict__ phi,
                       const typename SP::real* __restrict__ c, typename SP::store_t* __restrict__ g,
                       typename SP::store_t* __restrict__ h) {
    using R = typename SP::real;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int x = (int)(i % P.nx);
    const int y = (int)((i / P.nx) % P.ny);
    const int z = (int)(i / ((long long)P.nx * P.ny));
    auto at = [&](int dx, int dy, int dz) {
        const int gx = map_coord(x + dx, P.nx, P.bc[0]);
        const int gy = map_coord(y + dy, P.ny, P.bc[1]);
        const int gz = (L::D == 3) ? map_coord(z + dz, P.nz, P.bc[2]) : 0;
        return phi[((long long)gz * P.ny + gy) * P.nx + gx];
    };
    R gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int k = 1; k < L::Q; ++k) {
        const R dk = R(0.5) * (at(L::ex(k), L::ey(k), L::ez(k)) - at(-L::ex(k), -L::ey(k), -L::ez(k)));
        const R cw = R(3.0 * L::w(k));
        gx += cw * R(L::ex(k)) * dk;
        gy += cw * R(L::ey(k)) * dk;
        gz += cw * R(L::ez(k)) * dk;
    }
    const R inv = rsqrt_reg<R>(gx * gx + gy * gy + gz * gz, R(P.eps2));
    const R ph = phi[i], cc = c[i];
    const R mu = closure_mu(P, ph, cc);
    const R A = g_isotropic(P, ph, mu);
    const R kct = P.counter_term ? (R(4) / R(P.W)) * ph * (R(1) - ph) * inv : R(0);
    const R Pt = p_term(P, ph, mu);
    const R f = mu * R(P.D_l - P.D_s);
    const R w0 = R(L::w(0));
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const R wk = R(L::w(k));
        const R Gk = wk * (A + kct * edot<L>(k, gx, gy, gz));
        SP::store(g, (long long)k * P.N + i, wk * ph - R(0.5) * Gk, wk * ph);
        const R Hk = R(P.gamma) * wk * f * edot<L>(k, gx, gy, gz);
        const R heq = (k == 0) ? cc - (R(1) - w0) * Pt : wk * Pt;
        SP::store(h, (long long)k * P.N + i, heq - R(0.5) * Hk, heq);
    }
}

// ---- conversions and exports -----------------------------------------------------------

template <typename R>
__global__ void k_from_f64(const double* __restrict__ src, R* __restrict__ dst, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = R(src[i]);
}

template <typename R>
__global__ void k_fields_out(const StepParams P, const R* __restrict__ phi, const R* __restrict__ c,
                             double* __restrict__ ophi, double* __restrict__ oc, double* __restrict__ omu) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const double ph = (double)phi[i], cc = (double)c[i];
    if (ophi) ophi[i] = ph;
    if (oc) oc[i] = cc;
    if (omu) omu[i] = P.mu_eq + cc - (P.c_l * ph + P.c_s * (1.0 - ph));
}

// Expand stored populations to FP64 (deviation modes add their references back).
template <class L, class SP>
__global__ void k_pops_out(const StepParams P, const typename SP::real* __restrict__ phi,
                           const typename SP::real* __restrict__ c, const typename SP::store_t* __restrict__ g,
                           const typename SP::store_t* __restrict__ h, double* __restrict__ og,
                           double* __restrict__ oh) {
    using R = typename SP::real;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const R ph = phi[i], cc = c[i];
    const R Pt = p_term(P, ph, closure_mu(P, ph, cc));
    const R w0 = R(L::w(0));
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const R wk = R(L::w(k));
        if (og) og[(long long)k * P.N + i] = (double)SP::load(g, (long long)k * P.N + i, wk * ph);
        const R heq = (k == 0) ? cc - (R(1) - w0) * Pt : wk * Pt;
        if (oh) oh[(long long)k * P.N + i] = (double)SP::load(h, (long long)k * P.N + i, heq);
    }
}

// ---- FP64 mass reduction -------------------------------------------------------------
// Pass 1: each block sums c and phi over a grid-stride range into FP64 partials
// (partials[3 b + 0..2] = sum c, sum phi, count of bad values).  Pass 2: one
// block adds the partials in a fixed order.  Deterministic for a fixed grid.

constexpr int kMassThreads = 256;

template <typename R>
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
    __shared__ double sh[3][kMassThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; sh[2][wid] = c; }
    __syncthreads();
    if (wid == 0) {
        a = lane < kMassThreads / 32 ? sh[0][lane] : 0.0;
        b = lane < kMassThreads / 32 ? sh[1][lane] : 0.0;
        c = lane < kMassThreads / 32 ? sh[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
            c += __shfl_down_sync(0xffffffffu, c, o);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kMassThreads)
k_mass_partial(const R* __restrict__ c, const R* __restrict__ phi, long long n, double* __restrict__ partials) {
    double sc = 0.0, sp = 0.0, bad = 0.0;
    for (long long i = blockIdx.x * (long long)kMassThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kMassThreads) {
        const double cv = (double)c[i], pv = (double)phi[i];
        sc += cv;
        sp += pv;
        // non-finite values fail both comparisons and count as bad
        if (!(pv >= -0.5 && pv <= 1.5) || !(cv == cv && cv - cv == 0.0)) bad += 1.0;
    }
    block_sum3<R>(sc, sp, bad);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = sc;
        partials[3 * blockIdx.x + 1] = sp;
        partials[3 * blockIdx.x + 2] = bad;
    }
}

__global__ void __launch_bounds__(kMassThreads)
k_mass_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    double sc = 0.0, sp = 0.0, bad = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kMassThreads) {
        sc += partials[3 * b + 0];
        sp += partials[3 * b + 1];
        bad += partials[3 * b + 2];
    }
    block_sum3<double>(sc, sp, bad);
    if (threadIdx.x == 0) {
        out[0] = sc;
        out[1] = sp;
        out[2] = bad;
    }
}

}  // namespace lbpf
