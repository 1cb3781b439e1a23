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

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

#include "lattice.cuh"

namespace lbpf {

// Scalars of one simulation, in lattice units (converted once on the host).
struct StepParams {
    int nx, ny, nz;
    int bc[3];          // 0 periodic, 1 bounce-back
    long long N;        // nx * ny * nz
    // storage: node (x, y, z) at element z sxy + y sx + x of a field and of each
    // population plane, population k starting at element k NS.  Single domains
    // are dense (sx = nx, sxy = nx ny, NS = N); batch instances pad their rows.
    int sx;
    long long sxy, NS;
    double omg, omh;    // 1 / (tau + 1/2)
    double M;           // M_phi = tau_g / 3
    double gamma;       // 3 / tau_h
    double W, lambda, D_l, D_s, c_s, c_l, mu_eq;
    double a_at;        // a of j_at, 0 when anti-trapping is off
    double eps2;        // eps_n^2
    int counter_term;
    int h_den;          // DEN of the h lattice: 36 (D2Q9 / D3Q19) or 6 (D2Q5 / D3Q7)
    int h_eq_alt;       // 1: h^eq,alt with H_k = 0 (Eq. Seq_Concent_Alt)
    // parabolas of unequal curvature (Sec. 2.3): e_s = sqrt(eps_s / eps_l),
    // e_l = 1 / e_s, minima m_s, m_l and df = Delta f^min from the equilibrium
    // conditions at c_s^co, c_l^co, mu_eq
    int unequal;
    double e_s, e_l, m_s, m_l, df;
};

// Derived constants of one simulation in the compute type, precomputed on the
// host so that FP32 kernels carry no FP64 arithmetic:
//   S_phi = kS phi (1 - phi)(mu - mu_eq),  kS = 6 (c_s^co - c_l^co)   (p' = 6 phi (1 - phi))
//   G^st = kst S_phi,  kst = -lambda M / W^2;  G^dw = kdw omega',  kdw = -8 M / W^2
//   counter-term magnitude (4/W) phi (1 - phi) = kct phi (1 - phi)
//   j_at = atk dphi n,  atk = a W (c_s^co - c_l^co)
// With unequal curvatures (unequal = 1; Eq. Closure, SourceTerm, Anti-Trapping_Quadratic):
//   mu = (c - m_l phi - m_s (1 - phi)) / (e_s phi + e_l (1 - phi))
//   S_phi = 6 phi (1 - phi) [(hq mu - dm) mu - df],  hq = (e_l - e_s)/2, dm = m_l - m_s
//   j_at = (atk1 mu + atk0) dphi n,  atk1 = a W (e_l - e_s), atk0 = a W (m_s - m_l)
template <typename R>
struct Coef {
    R mu_eq, c_l, c_s, kS, kst, kdw, kct, D_l, D_s, Dp, gamma, atk, omg, omh, eps2;
    int unequal;
    R e_s, e_l, m_s, m_l, hq, dm, df, atk1, atk0;
    R kct36;   // (1 - w_g/2) kct / 36: the counter-term vector per unit m_k
    // the flux vector of the h collision per unit m_k of the h lattice (w_k =
    // m_k / DEN): (1 - w_h/2) gamma / DEN for H_k (Eq. SourceTerm_LBE_h), or
    // w_h / (xi_s^2 DEN) = 3 w_h / DEN for h^eq,alt (Eq. Seq_Concent_Alt)
    R khw;
};

template <typename R>
__host__ Coef<R> make_coef(const StepParams& P) {
    Coef<R> c;
    c.mu_eq = R(P.mu_eq); c.c_l = R(P.c_l); c.c_s = R(P.c_s);
    c.kS = R(6.0 * (P.c_s - P.c_l));
    c.kst = R(-P.lambda * P.M / (P.W * P.W));
    c.kdw = R(P.counter_term ? 0.0 : -8.0 * P.M / (P.W * P.W));
    c.kct = R(P.counter_term ? 4.0 / P.W : 0.0);
    c.D_l = R(P.D_l); c.D_s = R(P.D_s); c.Dp = R(P.D_l - P.D_s);
    c.gamma = R(P.gamma);
    c.atk = R(P.a_at * P.W * (P.c_s - P.c_l));
    c.omg = R(P.omg); c.omh = R(P.omh); c.eps2 = R(P.eps2);
    c.kct36 = R((1.0 - 0.5 * P.omg) * (P.counter_term ? 4.0 / P.W : 0.0) / 36.0);
    c.khw = R(P.h_eq_alt ? 3.0 * P.omh / P.h_den : (1.0 - 0.5 * P.omh) * P.gamma / P.h_den);
    c.unequal = P.unequal;
    c.e_s = R(P.e_s); c.e_l = R(P.e_l); c.m_s = R(P.m_s); c.m_l = R(P.m_l);
    c.hq = R(0.5 * (P.e_l - P.e_s)); c.dm = R(P.m_l - P.m_s); c.df = R(P.df);
    const double aW = P.a_at * P.W;
    c.atk1 = R(aW * (P.e_l - P.e_s)); c.atk0 = R(aW * (P.m_s - P.m_l));
    return c;
}

// Everything a step kernel needs: geometry and the constants in both types.
struct KParams {
    StepParams P;
    Coef<double> cd;
    Coef<float> cf;
    // per link k, in BYTES of the stored populations (element offset x bytes
    // per stored value, so that an address is one add): k N - (ex + ey nx +
    // ez nx ny), the offset of the upstream population from x for a node whose
    // neighbours are all inside (no wrap), and k N
    long long koffB[19];
    long long kNB[19];
    // the same as 32-bit values when they fit (else 0): the batch kernels,
    // whose instances are bounded in size, index with them
    int koffB32[19];
    int kNB32[19];
};

// Byte offsets of the links in the index type of a march (64-bit, or 32-bit
// for batch instances).
template <typename I>
__device__ __forceinline__ I link_src(const KParams& K, int k);
template <>
__device__ __forceinline__ long long link_src<long long>(const KParams& K, int k) { return K.koffB[k]; }
template <>
__device__ __forceinline__ int link_src<int>(const KParams& K, int k) { return K.koffB32[k]; }
template <typename I>
__device__ __forceinline__ I link_base(const KParams& K, int k);
template <>
__device__ __forceinline__ long long link_base<long long>(const KParams& K, int k) { return K.kNB[k]; }
template <>
__device__ __forceinline__ int link_base<int>(const KParams& K, int k) { return K.kNB32[k]; }

// p advanced by a byte offset
template <typename T, typename I>
__device__ __forceinline__ T* byte_add(T* p, I off) {
    using C = typename std::conditional<std::is_const<T>::value, const char, char>::type;
    return reinterpret_cast<T*>(reinterpret_cast<C*>(p) + off);
}

template <typename R>
__device__ __forceinline__ const Coef<R>& coef(const KParams& K);
template <>
__device__ __forceinline__ const Coef<double>& coef<double>(const KParams& K) { return K.cd; }
template <>
__device__ __forceinline__ const Coef<float>& coef<float>(const KParams& K) { return K.cf; }

// ---- storage policies --------------------------------------------------------
// A policy maps a population between its stored form and the compute type.
// `ref` is the population's equilibrium value at the node it is stored at; the
// plain policies ignore it, the deviation policies store v - ref in 16 bits.

struct StoreF64 {
    using real = double;
    using store_t = double;
    __device__ static __forceinline__ real load(const store_t* p, long long i, real) { return p[i]; }
    __device__ static __forceinline__ void store(store_t* p, long long i, real v, real) { p[i] = v; }
    __device__ static __forceinline__ real stored(real v, real) { return v; }
    static constexpr bool deviation = false;
};

struct StoreF32 {
    using real = float;
    using store_t = float;
    __device__ static __forceinline__ real load(const store_t* p, long long i, real) { return p[i]; }
    __device__ static __forceinline__ void store(store_t* p, long long i, real v, real) { p[i] = v; }
    __device__ static __forceinline__ real stored(real v, real) { return v; }
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
    // the value a later load returns for a stored v
    __device__ static __forceinline__ real stored(real v, real ref) {
        return fmaf(__half2float(__float2half_rn((v - ref) * S)), INV, ref);
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
    __device__ static __forceinline__ real stored(real v, real ref) {
        return __bfloat162float(__float2bfloat16_rn(v - ref)) + ref;
    }
    static constexpr bool deviation = true;
};

// ---- helpers ------------------------------------------------------------------

__device__ __forceinline__ int map_coord(int i, int n, int bc) {
    if (i >= 0 && i < n) return i;
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

// Storage element of the node with dense index i = (z ny + y) nx + x.
__host__ __device__ __forceinline__ long long storage_index(const StepParams& P, long long i) {
    if (P.sx == P.nx) return i;     // dense: single domains (and unpadded instances)
    const long long row = i / P.nx;
    const long long x = i - row * P.nx;
    const long long z = row / P.ny;
    return z * P.sxy + (row - z * P.ny) * P.sx + x;
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

template <typename R>
__device__ __forceinline__ R rsqrt_reg(R g2, R eps2);
template <>
__device__ __forceinline__ double rsqrt_reg<double>(double g2, double eps2) { return rsqrt(g2 + eps2); }
template <>
__device__ __forceinline__ float rsqrt_reg<float>(float g2, float eps2) { return rsqrtf(g2 + eps2); }

// x / 36 for the weights w_k = m_k / 36 (x / DEN in general).  FP32: correctly rounded, so the
// rounding of each node's per-unit quantity is unbiased and the m_k-weighted
// links conserve it (see lattice.cuh).  FP64: a multiplication by 1/36, whose
// ~1e-17 relative bias is far below anything FP64 resolves, at a fraction of
// the cost of a double division (the FP64 step is bound by the FP64 pipe).
template <int DEN>
__device__ __forceinline__ float divw(float x) { return x / float(DEN); }
template <int DEN>
__device__ __forceinline__ double divw(double x) { return x * (1.0 / DEN); }
template <typename R>
__device__ __forceinline__ R div36(R x) { return divw<36>(x); }

// G^st + G^dw: the isotropic part of G_k / w_k (Eq. SourceG_ST, Eq. SourceG_dw;
// S_phi of Eq. SourceTerm_Coexistence with p' = 6 phi (1 - phi);
// omega' = 2 phi (1 - phi)(1 - 2 phi) of Tab. 2).  kdw = 0 with the counter term.
// U = false: equal curvatures known at compile time (the batch kernels, which
// refuse unequal curvatures, keep their registers for the march).
template <bool U = true, typename R>
__device__ __forceinline__ R g_isotropic(const Coef<R>& C, R phi, R mu) {
    const R pq = phi * (R(1) - phi);
    const R S = (U && C.unequal) ? R(6) * pq * ((C.hq * mu - C.dm) * mu - C.df)   // Eq. SourceTerm
                                 : C.kS * pq * (mu - C.mu_eq);
    return C.kst * S + C.kdw * (R(2) * pq * (R(1) - R(2) * phi));
}

// Closure mu = mu_eq + c - c^co(phi) (Eq. PotChim_Equilibirum, h = phi), or
// Eq. Closure for parabolas of unequal curvature.
template <bool U = true, typename R>
__device__ __forceinline__ R closure_mu(const Coef<R>& C, R phi, R c) {
    if (U && C.unequal)
        return (c - (C.m_l * phi + C.m_s * (R(1) - phi))) / (C.e_s * phi + C.e_l * (R(1) - phi));
    return C.mu_eq + c - (C.c_l * phi + C.c_s * (R(1) - phi));
}

// Coefficient of dphi n in j_at: a W (c_s^co - c_l^co) (Eq. Anti-trapping_Equilibrium),
// or a W [(e_l - e_s) mu + m_s - m_l] (Eq. Anti-Trapping_Quadratic).
template <bool U = true, typename R>
__device__ __forceinline__ R at_coef(const Coef<R>& C, R mu) {
    return (U && C.unequal) ? C.atk1 * mu + C.atk0 : C.atk;
}

// P = gamma D(phi) mu with D = D_l phi + D_s (1 - phi) (Sec. 2.3.3).
template <typename R>
__device__ __forceinline__ R p_term(const Coef<R>& C, R phi, R mu) {
    return C.gamma * (C.D_l * phi + C.D_s * (R(1) - phi)) * mu;
}

// ---- z-marching tile geometry ------------------------------------------------------
// A block of BX x BY threads owns an x-y tile and walks a chunk of ZCH planes
// along z.  2-D domains are walked row by row through the D2Q9R view (planes
// are BX-long row segments, BY = 1, no y ring).  Shared memory holds rolling windows: phi^n for the
// planes z-2..z+2 with a 2-node x-y halo, and the per-node ingredients for the
// planes z-1..z+1 with a 1-node x-y ring.

template <typename R>
struct alignas(4 * sizeof(R)) V4 {
    R a, b, c, d;
};

template <class L, int BY, int BX_>
struct Geo {
    static constexpr int BX = BX_;
    static constexpr int HY = L::FLAT_Y ? 0 : 1;      // y halo needed (links along y)
    static constexpr int OY1 = HY, OY2 = 2 * HY;      // first tile row in the 1- and 2-halo planes
    static constexpr int X2 = BX + 4, Y2 = BY + 2 * OY2;   // phi plane with a 2-node halo
    static constexpr int X1 = BX + 2, Y1 = BY + 2 * OY1;   // ingredient plane with a 1-node ring
    static constexpr int P2 = X2 * Y2, P1 = X1 * Y1;
    static constexpr int NPHI = (L::D == 3) ? 5 : 1; // phi planes in the window
    static constexpr int NING = (L::D == 3) ? 3 : 1; // ingredient planes in the window
    static constexpr int NT = BX * BY;
    __device__ static __forceinline__ int tid() { return threadIdx.x + BX * threadIdx.y; }
};

// Wrap (periodic) or mirror (wall) an index that is at most one node outside.
__device__ __forceinline__ int wrap1(int i, int n, int bc) {
    if (i < 0) return bc ? 0 : i + n;
    if (i >= n) return bc ? n - 1 : i - n;
    return i;
}

// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes per element): the
// next plane's inputs stream into shared memory while the current plane computes.
template <typename R>
__device__ __forceinline__ void cp_async(R* smem_dst, const R* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    if (sizeof(R) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Tensor-memory-access (TMA) copies of population rows, completed on an
// mbarrier in shared memory.  One thread arms the barrier with the byte count
// of a plane and issues the tiled copies; every thread waits on the barrier's
// phase before it reads the rows.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// orders this thread's shared-memory accesses before later copy-engine accesses
// (after barrier initialisation, and after writes into a stage the engine refills)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Bounded wait: gives up after about a second of the global timer (and in any
// case after 2^20 rounds of 64 tries).  false: the phase never completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (int round = 0; round < (1 << 20); ++round) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}
// Box of a 4-D tensor map at coordinates (c0 innermost .. c3) into shared memory.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

// In-plane offsets (y nx + x, wrapped on periodic axes, mirrored at walls) of
// the window elements this thread copies: the phi plane with its 2-node halo
// (o2) and the 1-node ring (o1), and the phi-window index of each ring node it
// computes ingredients for (c2).  They are the same for every plane of a
// march, so they are computed once per block and each plane's copy costs one
// add per element.
template <class G>
struct HaloOffsets {
    static constexpr int IT2 = (G::P2 + G::NT - 1) / G::NT, IT1 = (G::P1 + G::NT - 1) / G::NT;
    int o2[IT2];
    int o1[IT1];
    int c2[IT1];
    __device__ __forceinline__ void init(const StepParams& P, int x0, int y0, bool inside2, bool inside1) {
        const int tid = G::tid();
#pragma unroll
        for (int it = 0; it < IT2; ++it) {
            const int s = tid + it * G::NT;
            const int ly = s / G::X2, lx = s - ly * G::X2;
            int gx = x0 + lx - 2, gy = y0 + ly - G::OY2;
            if (!inside2) {
                gx = map_coord(gx, P.nx, P.bc[0]);
                gy = map_coord(gy, P.ny, P.bc[1]);
            }
            o2[it] = s < G::P2 ? gy * P.sx + gx : 0;
        }
#pragma unroll
        for (int it = 0; it < IT1; ++it) {
            const int s = tid + it * G::NT;
            const int ly = s / G::X1, lx = s - ly * G::X1;
            int gx = x0 + lx - 1, gy = y0 + ly - G::OY1;
            if (!inside1) {
                gx = wrap1(gx, P.nx, P.bc[0]);
                gy = wrap1(gy, P.ny, P.bc[1]);
            }
            o1[it] = s < G::P1 ? gy * P.sx + gx : 0;
            c2[it] = (ly + G::OY2 - G::OY1) * G::X2 + (lx + 1);
        }
    }
};

// Start the copy of one phi plane (global z index zg, possibly outside) with its
// 2-node halo.
template <class L, class G, typename R>
__device__ __forceinline__ void async_phi_plane(const StepParams& P, const R* __restrict__ phi, R* dst, int zg,
                                                const HaloOffsets<G>& H) {
    const int tid = G::tid();
    const int gz = (L::D == 3) ? map_coord(zg, P.nz, P.bc[2]) : 0;
    const R* src = phi + (long long)gz * P.sxy;
#pragma unroll
    for (int it = 0; it < HaloOffsets<G>::IT2; ++it)
        if (tid + it * G::NT < G::P2) cp_async(dst + tid + it * G::NT, src + H.o2[it]);
}

// Start the copy of a field on the 1-node ring of plane zg into shared memory.
template <class L, class G, typename R>
__device__ __forceinline__ void async_ring(const StepParams& P, const R* __restrict__ f, R* dst, int zg,
                                           const HaloOffsets<G>& H) {
    const int tid = G::tid();
    const int gz = (L::D == 3) ? map_coord(zg, P.nz, P.bc[2]) : 0;
    const R* src = f + (long long)gz * P.sxy;
#pragma unroll
    for (int it = 0; it < HaloOffsets<G>::IT1; ++it)
        if (tid + it * G::NT < G::P1) cp_async(dst + tid + it * G::NT, src + H.o1[it]);
}

// grad(phi) by directional derivatives (Eq. DerivDirec_Grad, Eq. Grad) at offset c
// of the plane p0, with pm / pp the planes below / above.  Opposite links give
// the same term, so each pair is counted once, doubled.
template <class L, class G, typename R>
__device__ __forceinline__ void plane_gradient(const R* pm, const R* p0, const R* pp, int c,
                                               R& gx, R& gy, R& gz) {
    gx = gy = gz = R(0);
#pragma unroll
    for (int k = 1; k < L::Q; ++k) {
        if (L::opp(k) < k) continue;   // one link of each opposite pair
        const int off = L::ex(k) + G::X2 * L::ey(k);
        const R* fwd = L::ez(k) > 0 ? pp : (L::ez(k) < 0 ? pm : p0);
        const R* bwd = L::ez(k) > 0 ? pm : (L::ez(k) < 0 ? pp : p0);
        const R dk = fwd[c + off] - bwd[c - off];
        const R cw = R(3.0 * L::w(k));        // 2 (pair) x 3 w_k x 1/2 (central difference)
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

// Ingredients of the phi collision on one plane: alpha_g, beta_g (x, y, z) and
// A = G^st + G^dw.
template <class L, class G, bool U, typename R>
__device__ __forceinline__ void phi_ingredients(const StepParams& P, const Coef<R>& C, const R* cst,
                                                const R* pm, const R* p0, const R* pp, V4<R>* ing, R* sA,
                                                const HaloOffsets<G>& H) {
    const int tid = G::tid();
    const R half_src = R(1) - R(0.5) * C.omg;
    constexpr int IT = (G::P1 + G::NT - 1) / G::NT;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int s = tid + it * G::NT;
        if (s >= G::P1) break;
        const int c2 = H.c2[it];
        const R ph = p0[c2];
        const R mu = closure_mu<U>(C, ph, cst[s]);
        const R A = g_isotropic<U>(C, ph, mu);
        V4<R> v;
        v.a = div36(C.omg * ph + half_src * A);         // per unit m_k (w_k = m_k / 36)
        if (P.counter_term) {
            R gx, gy, gz_;
            plane_gradient<L, G>(pm, p0, pp, c2, gx, gy, gz_);
            const R inv = rsqrt_reg<R>(gx * gx + gy * gy + gz_ * gz_, C.eps2);
            const R k = C.kct36 * ph * (R(1) - ph) * inv;   // (4/W) phi (1 - phi) n, per unit m_k
            v.b = k * gx; v.c = k * gy; v.d = k * gz_;
        } else {
            v.b = v.c = v.d = R(0);
        }
        ing[s] = v;
        sA[s] = A;
    }
}

// Ingredients of the h collision on one plane: P = gamma D mu and
// beta_h = (1 - w_h/2) gamma (mu D' grad phi + j_at).
template <class L, class LH, class G, bool U, typename R>
__device__ __forceinline__ void c_ingredients(const StepParams& P, const Coef<R>& C, const R* cst, const R* pst,
                                              const R* pm, const R* p0, const R* pp, V4<R>* ing,
                                              const HaloOffsets<G>& H) {
    const int tid = G::tid();
    constexpr int IT = (G::P1 + G::NT - 1) / G::NT;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int s = tid + it * G::NT;
        if (s >= G::P1) break;
        const int c2 = H.c2[it];
        const R ph = p0[c2];
        const R dphi = pst[s] - ph;                        // explicit Euler dphi/dt
        const R mu = closure_mu<U>(C, ph, cst[s]);
        R gx, gy, gz_;
        plane_gradient<L, G>(pm, p0, pp, c2, gx, gy, gz_);
        const R inv = rsqrt_reg<R>(gx * gx + gy * gy + gz_ * gz_, C.eps2);
        const R f = mu * C.Dp + at_coef<U>(C, mu) * dphi * inv;   // F = (mu D' + j_at / |grad|) grad
        V4<R> v;
        v.a = divw<LH::DEN>(p_term(C, ph, mu));          // P per unit m_k of the h lattice
        const R ff = C.khw * f;
        v.b = ff * gx; v.c = ff * gy; v.d = ff * gz_;
        ing[s] = v;
    }
}

// Pull of one plane, in two stages so that the population loads of plane z are
// in flight while the block computes the ingredients of plane z+1.
//
// Upstream node of link k: (x - ex, y - ey, z - ez), wrapped on periodic axes;
// beyond a wall the link bounces back to the node itself.  `fast`: every
// upstream node is inside, so the source is the node address + koffB[k] (one add).  Otherwise
// the wrapped x index, row and plane offsets for e = -1, 0, 1 are computed once
// and a link's source costs two adds and no branch.
// Exact solute mass of the populations a thread has written, as an unevaluated
// sum hi + lo (float-float in FP32), reduced per block in FP64 at the end.
template <typename R>
struct MassAcc {
    R hi, lo;
    __device__ __forceinline__ void add(R s, R e) {      // add s + e (e small)
        const R t = hi + s;
        const R bb = t - hi;
        lo += ((hi - (t - bb)) + (s - bb)) + e;          // TwoSum error of hi + s
        hi = t;
    }
};

template <class L, class SP, bool IS_PHI, bool WALLS, typename I = long long>
struct PullState {
    using R = typename SP::real;
    R old[L::Q];
    R cx;
    unsigned wallmask;
    I xi;
    const R* srow;   // tensor-map pulls: this thread's column of the stage (see tma_pull)
};

// Links of L along which x does not change (e_x = 0): their upstream rows are
// the tile's own columns, which the tensor-map form copies whole.
template <class L>
__host__ __device__ constexpr int ex0_count() {
    int n = 0;
    for (int k = 0; k < L::Q; ++k) n += L::ex(k) == 0 ? 1 : 0;
    return n;
}
template <class L>
__host__ __device__ constexpr int ex0_slot(int k) {      // rank of link k among them
    int n = 0;
    for (int j = 0; j < k; ++j) n += L::ex(j) == 0 ? 1 : 0;
    return n;
}
template <class L>
__host__ __device__ constexpr int ex0_link(int j) {      // the j-th of them
    for (int k = 0; k < L::Q; ++k)
        if (L::ex(k) == 0 && j-- == 0) return k;
    return 0;
}

// SKIP0: leave the links with e_x = 0 out (the tensor-map form brings them).
template <class L, class SP, bool IS_PHI, bool WALLS, typename I, bool SKIP0 = false>
__device__ __forceinline__ void pull_load(const KParams& K, const typename SP::store_t* __restrict__ fin,
                                          const typename SP::real* __restrict__ c_n, int x, int y, int z, bool fast,
                                          PullState<L, SP, IS_PHI, WALLS, I>& st) {
    using R = typename SP::real;
    const StepParams& P = K.P;
    const I nxy = (I)P.sxy;
    const I xi = (I)z * nxy + (I)y * P.sx + x;
    st.xi = xi;
    st.wallmask = 0u;
    st.cx = IS_PHI ? R(0) : c_n[xi];
    if (fast) {
        const typename SP::store_t* base = fin + xi;
#pragma unroll
        for (int k = 0; k < L::Q; ++k)
            if (!SKIP0 || L::ex(k) != 0) st.old[k] = SP::load(byte_add(base, link_src<I>(K, k)), 0, R(0));
        return;
    }
    // source offsets indexed by e + 1: e = +1 reads the node at -1, e = -1 the node at +1
    int SX[3], SY[3];
    I SZ[3];
    bool WX[3], WY[3], WZ[3];
    {
        const bool lo = x == 0, hi = x == P.nx - 1;
        SX[1] = x; WX[1] = false;
        SX[2] = lo ? (WALLS && P.bc[0] ? x : P.nx - 1) : x - 1; WX[2] = WALLS && lo && P.bc[0];
        SX[0] = hi ? (WALLS && P.bc[0] ? x : 0) : x + 1;        WX[0] = WALLS && hi && P.bc[0];
    }
    {
        const bool lo = y == 0, hi = y == P.ny - 1;
        SY[1] = y * P.sx; WY[1] = false;
        SY[2] = (lo ? (WALLS && P.bc[1] ? y : P.ny - 1) : y - 1) * P.sx; WY[2] = WALLS && lo && P.bc[1];
        SY[0] = (hi ? (WALLS && P.bc[1] ? y : 0) : y + 1) * P.sx;        WY[0] = WALLS && hi && P.bc[1];
    }
    if (L::D == 3) {
        const bool lo = z == 0, hi = z == P.nz - 1;
        SZ[1] = z * nxy; WZ[1] = false;
        SZ[2] = (I)(lo ? (WALLS && P.bc[2] ? z : P.nz - 1) : z - 1) * nxy; WZ[2] = WALLS && lo && P.bc[2];
        SZ[0] = (I)(hi ? (WALLS && P.bc[2] ? z : 0) : z + 1) * nxy;        WZ[0] = WALLS && hi && P.bc[2];
    } else {
        SZ[0] = SZ[1] = SZ[2] = 0; WZ[0] = WZ[1] = WZ[2] = false;
    }
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        if (SKIP0 && L::ex(k) == 0) continue;
        const bool wall = WALLS && (WX[L::ex(k) + 1] || WY[L::ey(k) + 1] || WZ[L::ez(k) + 1]);
        const I si = SZ[L::ez(k) + 1] + SY[L::ey(k) + 1] + SX[L::ex(k) + 1];
        // half-way bounce-back: f_k(x, n+1) = f*_{opp k}(x, n)
        const typename SP::store_t* src = wall ? byte_add(fin + xi, link_base<I>(K, L::opp(k)))
                                               : byte_add(fin + si, link_base<I>(K, k));
        st.old[k] = SP::load(src, 0, R(0));
        st.wallmask |= (wall ? 1u : 0u) << k;
    }
}

// The slots of the e_x = 0 links whose upstream row lies across a y face: the
// wrapped row's value.  Out of line, so that the registers it needs do not
// weigh on the march (only threads on those faces call it).
template <class L, int BOXE, typename R>
__device__ __noinline__ void tma_fix_edges(const R* __restrict__ fin, int ny, int nz, long long sx, long long sxy,
                                           long long ns, int x, int y, int z, R* col) {
#pragma unroll 1
    for (int k = 0; k < L::Q; ++k) {
        if (L::ex(k) != 0) continue;
        const int uy = y - L::ey(k);
        if (uy < 0 || uy >= ny) {
            const int ys = uy < 0 ? uy + ny : uy - ny;
            int zs = z - L::ez(k);
            zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
            col[ex0_slot<L>(k) * BOXE] = fin[k * ns + zs * sxy + ys * sx + x];
        }
    }
}

// The e_x = 0 pulls of plane z, from the boxes the copy engine placed in shared
// memory (the tensor-map form: all axes periodic, FP32 storage; the other
// links are loaded by pull_load).  The box of the j-th such link k holds rows
// y0 - ey .. y0 - ey + BY - 1 of plane z - ez (wrapped), columns x0 .. x0 + BX
// - 1, so the thread at (tx, ty) finds its upstream value at row ty, column tx,
// a slot no other thread reads; the collision reads it there.  A box row
// outside the grid was filled with zeros: the threads on the grid's y faces
// (`edge`) overwrite those slots with the wrapped row's value.  `fix`: some
// lane of the warp is such a thread.
template <class L, class SP, int BX, int BY, bool IS_PHI, bool WALLS, typename I>
__device__ __forceinline__ void tma_pull(const KParams& K, const typename SP::store_t* __restrict__ fin, int x,
                                         int y, int z, typename SP::real* stage, bool edge, bool fix,
                                         PullState<L, SP, IS_PHI, WALLS, I>& st) {
    using R = typename SP::real;
    constexpr int BOXE = BX * BY;
    const StepParams& P = K.P;
    R* col = stage + threadIdx.y * BX + threadIdx.x;
    st.srow = col;
    if (fix) {
        if (edge) tma_fix_edges<L, BOXE>(fin, P.ny, P.nz, (long long)P.sx, (long long)P.sxy, (long long)P.NS, x, y, z,
                                         col);
        // these generic writes come before the copy engine refills the stage
        fence_proxy_async();
    }
}

// Collision of each pulled population at its upstream node from the ingredient
// planes im (z-1), i0 (z), ip (z+1) (phi planes fm, f0, fp likewise), the new
// moment, and the stores.
template <class L, class SP, int BY, int BX, bool IS_PHI, bool WALLS, typename I, bool U, bool TS = false>
__device__ __forceinline__ void pull_combine(const KParams& K, const Coef<typename SP::real>& C,
                                             typename SP::store_t* __restrict__ fout,
                                             const V4<typename SP::real>* im, const V4<typename SP::real>* i0,
                                             const V4<typename SP::real>* ip, const typename SP::real* fm,
                                             const typename SP::real* f0, const typename SP::real* fp,
                                             const typename SP::real* sA,
                                             const typename SP::real* __restrict__ phi_np1_in,
                                             typename SP::real* __restrict__ moment_out,
                                             const PullState<L, SP, IS_PHI, WALLS, I>& st,
                                             MassAcc<typename SP::real>& macc) {
    using R = typename SP::real;
    using G = Geo<L, BY, BX>;
    const I xi = st.xi;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int c1 = (ty + G::OY1) * G::X1 + (tx + 1);
    const int c2 = (ty + G::OY2) * G::X2 + (tx + 2);
    const R om = IS_PHI ? C.omg : C.omh;
    const R keep = R(1) - om;
    // without deviation storage a population is stored as soon as it is known
    constexpr bool hold = SP::deviation;
    typename SP::store_t* out = fout + xi;

    R v[L::Q];
    // phi: a plain running sum.  c: a compensated sum (Fast2Sum, the rest
    // population first), because the collision uses the stored c as the zeroth
    // moment of h^eq: a plain FP32 sum is biased by about -1e-8 per node and
    // step, which would leak that much solute every step.
    R sum = R(0);
    R comp = R(0);
    constexpr int k0 = IS_PHI ? 0 : 1;
    if (!IS_PHI) {
        // rest population of h: h*_0 = (1 - w_h) h_0 + w_h h^eq_0 (H_0 = 0)
        const R heq0 = st.cx - R(L::DEN - L::m(0)) * i0[c1].a;   // h^eq_0 = c - (1 - w_0) P
        const R old0 = TS ? st.srow[0] : st.old[0];   // link 0 (rest, e_x = 0) is slot 0
        // the contraction is written out, so that it does not depend on where
        // the operands come from (loads, shared memory)
        v[0] = fma(keep, SP::deviation ? old0 + heq0 : old0, om * heq0);
        sum = v[0];
        if (!hold) SP::store(byte_add(out, link_base<I>(K, 0)), 0, v[0], R(0));
    }
#pragma unroll
    for (int k = k0; k < L::Q; ++k) {
        const R wk = R(L::w(k));
        const R mk = R(L::m(k));
        const bool wall = WALLS && ((st.wallmask >> k) & 1u);
        const V4<R>* ik = L::ez(k) > 0 ? im : (L::ez(k) < 0 ? ip : i0);   // upstream plane z - ez
        const R* fk = L::ez(k) > 0 ? fm : (L::ez(k) < 0 ? fp : f0);
        const V4<R> g = wall ? i0[c1] : ik[c1 - L::ex(k) - G::X1 * L::ey(k)];
        const R sgn = wall ? R(-1) : R(1);
        R f_old = (TS && L::ex(k) == 0) ? st.srow[ex0_slot<L>(k) * BX * BY] : st.old[k];
        if (SP::deviation) {
            const R ref = IS_PHI ? wk * (wall ? f0[c2] : fk[c2 - L::ex(k) - G::X2 * L::ey(k)]) : mk * g.a;
            f_old += ref;
        }
        const R a = IS_PHI ? g.a : om * g.a;
        const R val = fma(keep, f_old, mk * (a + sgn * edot<L>(k, g.b, g.c, g.d)));
        v[k] = val;
        if (IS_PHI || sizeof(R) == 8) {
            sum += val;          // FP64: a plain sum is unbiased far below FP64 resolution
        } else {
            const R t = sum + val;
            comp += (sum - t) + val;
            sum = t;
        }
        if (!hold) SP::store(byte_add(out, link_base<I>(K, k)), 0, val, R(0));
    }
    if (!IS_PHI) {
        if (!hold) macc.add(sum, comp);   // the node's exact population mass is sum + comp
        sum += comp;
    }
    if (IS_PHI) {
        const R phin = sum + R(0.5) * sA[c1];     // Eq. Moment_Phi
        moment_out[xi] = phin;
        if (hold) {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) SP::store(byte_add(out, link_base<I>(K, k)), 0, v[k], R(L::w(k)) * phin);
        }
    } else {
        moment_out[xi] = sum;                      // Eq. Moment0_LBM_Concent
        if (hold) {
            const R phin = phi_np1_in[xi];
            const R Ps = divw<L::DEN>(p_term(C, phin, closure_mu<U>(C, phin, sum)));
            // the mass regulated by the correction is that of the populations as
            // stored (quantised), i.e. of the values the next step loads
            const R ref0 = sum - R(L::DEN - L::m(0)) * Ps;
            SP::store(byte_add(out, link_base<I>(K, 0)), 0, v[0], ref0);
            R ms = SP::stored(v[0], ref0), mcomp = R(0);
#pragma unroll
            for (int k = 1; k < L::Q; ++k) {
                const R ref = R(L::m(k)) * Ps;
                SP::store(byte_add(out, link_base<I>(K, k)), 0, v[k], ref);
                const R vs = SP::stored(v[k], ref);
                const R t = ms + vs;
                mcomp += (ms - t) + vs;
                ms = t;
            }
            macc.add(ms, mcomp);
        }
    }
}

// FP64 block sum of the threads' mass accumulators, written to
// partials[linear block index] (all threads of the block must call it).
template <int NT, typename R>
__device__ __forceinline__ void block_mass_out(const MassAcc<R>& m, double* __restrict__ partials, long long slot) {
    __shared__ double red[NT / 32];
    double v = (double)m.hi + (double)m.lo;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += red[w];
        partials[slot] = t;
    }
}

// One z-marching pass of either kernel over the planes z0 <= z < z1 of the tile
// at (x0, y0).  The composition kernel also adds the exact mass of the
// populations it writes to macc.
// Stages of the tensor-map ring: the copies run NST - 1 planes ahead.
#ifndef LBPF_TMA_STAGES
#define LBPF_TMA_STAGES 2
#endif

// TMA: the pulls come from tensor-map copies (tmap: the 4-D map of fin, see
// tma_pull); a copy that never lands sets *err after a bounded wait.
template <class L, class SP, int BY, bool IS_PHI, bool WALLS, int BX = 32, typename I = long long,
          class LH = L, bool U = true, bool TMA = false>
__device__ __forceinline__ void march(const KParams& K, const typename SP::store_t* __restrict__ fin,
                                      typename SP::store_t* __restrict__ fout,
                                      const typename SP::real* __restrict__ phi_n,
                                      const typename SP::real* __restrict__ phi_np1,
                                      const typename SP::real* __restrict__ c_n,
                                      typename SP::real* __restrict__ moment_out,
                                      MassAcc<typename SP::real>& macc, int x0, int y0, int z0, int z1,
                                      const CUtensorMap* tmap = nullptr, int* err = nullptr) {
    using R = typename SP::real;
    using G = Geo<L, BY, BX>;
    const StepParams& P = K.P;
    const Coef<R>& C = coef<R>(K);
    static_assert(!TMA || (std::is_same<typename SP::store_t, float>::value && !WALLS && !L::FLAT_Y && BX == 32),
                  "tensor-map pulls: FP32 storage, periodic 3-D tiles");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // tensor-map stages first (128-byte aligned boxes), then their two barriers
    constexpr int Q0 = ex0_count<LH>();                              // links with e_x = 0
    constexpr int BOXE = BX * BY;
    constexpr int TSTAGE = TMA ? Q0 * BOXE : 0;                      // elements of one stage
    R* tst = reinterpret_cast<R*>(smem_raw);                         // [2][Q0][BY][BX]
    constexpr int NST = LBPF_TMA_STAGES;                             // stages in the ring
    uint64_t* bars = reinterpret_cast<uint64_t*>(tst + NST * TSTAGE);  // [NST] (TMA only)
    // the rest starts on a 128-byte boundary after the stages and barriers
    unsigned char* rest = smem_raw + (TMA ? (NST * TSTAGE * sizeof(R) + 8 * NST + 127) / 128 * 128 : 0);
    // plane zg uses stage (zg - z0) % NST, in the phase ((zg - z0) / NST) & 1 of its barrier
    auto tstage = [&](int zg) { return (zg - z0) % NST; };
    auto tphase = [&](int zg) { return (unsigned)((zg - z0) / NST) & 1u; };
    V4<R>* sing = reinterpret_cast<V4<R>*>(rest);                    // [NING][P1]
    R* sphi = reinterpret_cast<R*>(sing + G::NING * G::P1);          // [NPHI][P2]
    R* cst = sphi + G::NPHI * G::P2;                                 // [2][P1] c^n on the ring
    R* pst = cst + 2 * G::P1;                                        // [2][P1] phi^{n+1} (c kernel)
    R* sA = pst + (IS_PHI ? 0 : 2 * G::P1);                          // [NING][P1] (phi kernel)

    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active_xy = x < P.nx && y < P.ny;
    const bool inside2 = x0 >= 2 && x0 + G::BX + 2 <= P.nx && y0 >= G::OY2 && y0 + BY + G::OY2 <= P.ny;
    const bool inside1 = x0 >= 1 && x0 + G::BX + 1 <= P.nx && y0 >= G::OY1 && y0 + BY + G::OY1 <= P.ny;
    // the composition kernel pulls h on LH (L, or its small lattice); the phi
    // stencil and the ingredient window always follow L
    static_assert(IS_PHI ? std::is_same<L, LH>::value : L::FLAT_Y == LH::FLAT_Y, "h lattice");
    using LP = LH;
    PullState<LP, SP, IS_PHI, WALLS, I> st;

    // the ring inputs of plane zg go to stage buffer zg & 1
    HaloOffsets<G> halo;
    halo.init(P, x0, y0, inside2, inside1);
    auto fetch_ring = [&](int zg) {
        const int b = zg & 1;
        async_ring<L, G>(P, c_n, cst + b * G::P1, zg, halo);
        if (!IS_PHI) async_ring<L, G>(P, phi_np1, pst + b * G::P1, zg, halo);
    };
    auto ingredients = [&](int slot_i, const R* pm, const R* p0, const R* pp, int zg) {
        const int b = zg & 1;
        if (IS_PHI)
            phi_ingredients<L, G, U>(P, C, cst + b * G::P1, pm, p0, pp, sing + slot_i * G::P1,
                                     sA + slot_i * G::P1, halo);
        else
            c_ingredients<L, LH, G, U>(P, C, cst + b * G::P1, pst + b * G::P1, pm, p0, pp,
                                       sing + slot_i * G::P1, halo);
    };

    static_assert(L::D == 3, "2-D domains march through the D2Q9R view");

    // z-march.  While plane z is pulled, the phi plane z+3 and the ring of z+2
    // stream into shared memory, and the loads of plane z overlap the
    // ingredients of z+1.  Stage buffers are indexed by zg & 1 (zg >= -1).
    // zg >= z0 - 2 for phi planes and zg >= z0 - 1 for ingredient planes
    auto fslot = [&](int zg) { return sphi + ((unsigned)(zg - z0 + 2) % 5u) * G::P2; };
    auto islot = [&](int zg) { return (int)((unsigned)(zg - z0 + 1) % 3u); };

    // tensor-map pulls of plane zg into stage (zg - z0) & 1 by the first warp:
    // lane 0 arms the stage's barrier with the plane's bytes, then lane j < Q0
    // copies the box of the j-th e_x = 0 link (its y origin and e_z are fixed
    // per block)
    const int tl = threadIdx.x;                       // lane in the first warp (BX == 32)
    const int tma_k = (TMA && tl < Q0) ? ex0_link<LP>(tl) : 0;
    const int tma_y = y0 - LP::ey(tma_k);
    const int tma_ez = LP::ez(tma_k);
    auto tma_issue = [&](int zg) {
        if constexpr (TMA) {
            if (threadIdx.y == 0) {
                const int sidx = tstage(zg);
                if (tl == 0) mbar_arrive_expect_tx(&bars[sidx], (unsigned)(TSTAGE * sizeof(R)));
                __syncwarp();
                if (tl < Q0) {
                    int zs = zg - tma_ez;
                    zs = zs < 0 ? zs + P.nz : (zs >= P.nz ? zs - P.nz : zs);
                    tma_load_4d(tst + (sidx * Q0 + tl) * BOXE, tmap, x0, tma_y, zs, tma_k, &bars[sidx]);
                }
            }
        }
    };
    bool tma_late = false;           // a wait ran out (reported through err)
    if constexpr (TMA) {
        if (G::tid() == 0) {
            for (int i = 0; i < NST; ++i) mbar_init(&bars[i], 1);
            fence_proxy_async();
        }
        __syncwarp();                // the first warp issues right after the initialisation
        for (int d = 0; d < NST - 1 && z0 + d < z1; ++d) tma_issue(z0 + d);
    }

    for (int zg = z0 - 2; zg <= z0 + 1; ++zg) async_phi_plane<L, G>(P, phi_n, fslot(zg), zg, halo);
    fetch_ring(z0 - 1);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    ingredients(islot(z0 - 1), fslot(z0 - 2), fslot(z0 - 1), fslot(z0), z0 - 1);
    __syncthreads();                     // stage (z0 - 1) & 1 is reused by plane z0 + 1
    fetch_ring(z0);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    ingredients(islot(z0), fslot(z0 - 1), fslot(z0), fslot(z0 + 1), z0);
    async_phi_plane<L, G>(P, phi_n, fslot(z0 + 2), z0 + 2, halo);
    fetch_ring(z0 + 1);
    cp_async_commit();
    for (int z = z0; z < z1; ++z) {
        cp_async_wait_all();             // phi plane z+2 and the ring of z+1 have landed
        __syncthreads();                 // ... for every thread; pull(z-1) is done everywhere
        if (z + 1 < z1) {
            // prefetch for the next plane: phi plane z+3 into the slot of z-2, ring of z+2
            async_phi_plane<L, G>(P, phi_n, fslot(z + 3), z + 3, halo);
            fetch_ring(z + 2);
        }
        // NST - 1 planes ahead; the stage was last read by pull(z-1), done everywhere
        if (z + NST - 1 < z1) tma_issue(z + NST - 1);
        cp_async_commit();
        if (active_xy)
            pull_load<LP, SP, IS_PHI, WALLS, I, TMA>(K, fin, c_n, x, y, z, inside1 && z >= 1 && z + 1 < P.nz, st);
        ingredients(islot(z + 1), fslot(z), fslot(z + 1), fslot(z + 2), z + 1);
        __syncthreads();
        if constexpr (TMA) {
            const int sidx = tstage(z);
            // after one wait has run out the block stops waiting (its results are
            // flagged through err), so a broken copy costs about a second, not one per plane
            if (!tma_late && !mbar_wait(&bars[sidx], tphase(z))) tma_late = true;
            const bool edge = active_xy && (y == 0 || y == P.ny - 1);
            const bool fix = __any_sync(0xffffffffu, edge);
            if (active_xy)
                tma_pull<LP, SP, BX, BY, IS_PHI, WALLS, I>(K, fin, x, y, z, tst + sidx * TSTAGE, edge, fix, st);
        }
        if (active_xy)
            pull_combine<LP, SP, BY, BX, IS_PHI, WALLS, I, U, TMA>(K, C, fout, sing + islot(z - 1) * G::P1,
                                                   sing + islot(z) * G::P1, sing + islot(z + 1) * G::P1,
                                                   fslot(z - 1), fslot(z), fslot(z + 1), sA + islot(z) * G::P1,
                                                   phi_np1, moment_out, st, macc);
    }
    cp_async_wait_all();
    if constexpr (TMA) {
        if (tma_late) {
            // report, and give a copy still in flight a last bounded wait
            // before the block's shared memory is released
            atomicExch(err, 1);
            mbar_wait(&bars[tstage(z1 - 1)], tphase(z1 - 1));
        }
    }
}

template <class L, class SP, int BY, int BX = 32, class LH = L>
constexpr size_t march_smem(bool is_phi, bool tma = false) {
    using G = Geo<L, BY, BX>;
    using R = typename SP::real;
    return sizeof(V4<R>) * G::NING * G::P1 + sizeof(R) * G::NPHI * G::P2 + sizeof(R) * 2 * G::P1 +
           (is_phi ? sizeof(R) * G::NING * G::P1 : sizeof(R) * 2 * G::P1) +
           (tma ? (LBPF_TMA_STAGES * (sizeof(R) * (is_phi ? ex0_count<L>() : ex0_count<LH>()) * BX * BY + 8) + 127) /
                      128 * 128
                : 0);
}

// ---- the two step kernels ----------------------------------------------------------

// Block (bx, by, bz) marches the tile at (bx BX, by BY) over the planes
// [bz zch, min((bz + 1) zch, nz)).
// TMA: pulls through the tensor map tmap of the input populations (see
// tma_pull); err is set if a copy never lands.
template <class L, class SP, int BY, int MINB, bool WALLS, int BX = 32, bool TMA = false>
__global__ void __launch_bounds__(BX * BY, MINB)
k_phi_step(const KParams K, const typename SP::store_t* __restrict__ gin,
           typename SP::store_t* __restrict__ gout, const typename SP::real* __restrict__ phi_n,
           const typename SP::real* __restrict__ c_n, typename SP::real* __restrict__ phi_np1, int zch,
           const __grid_constant__ CUtensorMap tmap, int* err) {
    MassAcc<typename SP::real> macc{0, 0};
    const int z0 = blockIdx.z * zch;
    march<L, SP, BY, true, WALLS, BX, long long, L, true, TMA>(K, gin, gout, phi_n, nullptr, c_n, phi_np1, macc,
                                                               blockIdx.x * BX, blockIdx.y * BY, z0,
                                                               min(z0 + zch, K.P.nz), &tmap, err);
}

template <class L, class SP, int BY, int MINB, bool WALLS, int BX = 32, class LH = L, bool TMA = false>
__global__ void __launch_bounds__(BX * BY, MINB)
k_c_step(const KParams K, const typename SP::store_t* __restrict__ hin,
         typename SP::store_t* __restrict__ hout, const typename SP::real* __restrict__ phi_n,
         const typename SP::real* __restrict__ phi_np1, const typename SP::real* __restrict__ c_n,
         typename SP::real* __restrict__ c_np1, double* __restrict__ mass_partials, int zch,
         const __grid_constant__ CUtensorMap tmap, int* err) {
    using G = Geo<L, BY, BX>;
    MassAcc<typename SP::real> macc{0, 0};
    const int z0 = blockIdx.z * zch;
    march<L, SP, BY, false, WALLS, BX, long long, LH, true, TMA>(K, hin, hout, phi_n, phi_np1, c_n, c_np1, macc,
                                                                 blockIdx.x * BX, blockIdx.y * BY, z0,
                                                                 min(z0 + zch, K.P.nz), &tmap, err);
    if (mass_partials)
        block_mass_out<G::NT>(macc, mass_partials,
                              blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z));
}

// ---- initialisation -------------------------------------------------------------------
// g_k = w_k phi - G_k/2, h_k = h^eq_k - H_k/2 with H at dphi/dt = 0 (the variable
// change of Sec. 3.1 applied at equilibrium), or h_k = h^eq,alt_k with the
// alternative equilibrium (no H, no shifted variable).  h lives on LH.  Fields
// phi, c already hold the start values in the compute type.

template <class L, class SP, class LH = L>
__global__ void k_init(const KParams K, const typename SP::real* __restrict__ phi,
                       typename SP::real* __restrict__ c, typename SP::store_t* __restrict__ g,
                       typename SP::store_t* __restrict__ h) {
    using R = typename SP::real;
    const StepParams& P = K.P;
    const Coef<R>& C = coef<R>(K);
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= P.N) return;
    const int x = (int)(id % P.nx);
    const int y = (int)((id / P.nx) % P.ny);
    const int z = (int)(id / ((long long)P.nx * P.ny));
    const long long i = (long long)z * P.sxy + (long long)y * P.sx + x;     // storage element
    auto at = [&](int dx, int dy, int dz) {
        const int gx = map_coord(x + dx, P.nx, P.bc[0]);
        const int gy = map_coord(y + dy, P.ny, P.bc[1]);
        const int gz = (L::D == 3) ? map_coord(z + dz, P.nz, P.bc[2]) : 0;
        return phi[(long long)gz * P.sxy + (long long)gy * P.sx + gx];
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
    const R inv = rsqrt_reg<R>(gx * gx + gy * gy + gz * gz, C.eps2);
    const R ph = phi[i], cc = c[i];
    const R mu = closure_mu(C, ph, cc);
    const R A = g_isotropic(C, ph, mu);
    const R kct = C.kct * ph * (R(1) - ph) * inv;
    const R Ps = divw<LH::DEN>(p_term(C, ph, mu));
    const R f = mu * C.Dp;
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const R wk = R(L::w(k));
        const R Gk = wk * (A + kct * edot<L>(k, gx, gy, gz));
        SP::store(g, (long long)k * P.NS + i, wk * ph - R(0.5) * Gk, wk * ph);
    }
    R hsum = R(0), hcomp = R(0);
#pragma unroll
    for (int k = 0; k < LH::Q; ++k) {
        const R wk = R(LH::w(k));
        const R ek = edot<LH>(k, gx, gy, gz);
        const R heq = (k == 0) ? cc - R(LH::DEN - LH::m(0)) * Ps : R(LH::m(k)) * Ps;
        // H_k = gamma w_k e_k.F, or the flux part w_k e_k.F / xi_s^2 of h^eq,alt
        const R hk = P.h_eq_alt ? heq + R(3) * wk * f * ek : heq - R(0.5) * (C.gamma * wk * f * ek);
        SP::store(h, (long long)k * P.NS + i, hk, heq);
        const R t = hsum + hk;              // Fast2Sum: h_0 (the largest) comes first
        hcomp += (hsum - t) + hk;
        hsum = t;
    }
    // the c field is the zeroth moment of the stored populations, so that the
    // mass at step 0 is the populations' mass
    c[i] = hsum + hcomp;
}

// ---- conversions and exports -----------------------------------------------------------

template <typename R>
__global__ void k_from_f64(const double* __restrict__ src, R* __restrict__ dst, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = R(src[i]);
}

// Dense FP64 caller data (rows of nx) -> rows of pitch sx in the compute type.
template <typename R>
__global__ void k_from_f64_rows(const double* __restrict__ src, R* __restrict__ dst, long long n, int nx, int sx) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long row = i / nx;
    dst[row * sx + (i - row * nx)] = R(src[i]);
}

template <typename R>
__global__ void k_fields_out(const KParams K, const R* __restrict__ phi, const R* __restrict__ c,
                             double* __restrict__ ophi, double* __restrict__ oc, double* __restrict__ omu) {
    const StepParams& P = K.P;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const long long j = storage_index(P, i);
    const double ph = (double)phi[j], cc = (double)c[j];
    if (ophi) ophi[i] = ph;
    if (oc) oc[i] = cc;
    if (omu)
        omu[i] = P.unequal ? (cc - (P.m_l * ph + P.m_s * (1.0 - ph))) / (P.e_s * ph + P.e_l * (1.0 - ph))
                           : P.mu_eq + cc - (P.c_l * ph + P.c_s * (1.0 - ph));
}

// Expand stored populations to FP64 (deviation modes add their references back).
template <class L, class SP, class LH = L>
__global__ void k_pops_out(const KParams K, const typename SP::real* __restrict__ phi,
                           const typename SP::real* __restrict__ c, const typename SP::store_t* __restrict__ g,
                           const typename SP::store_t* __restrict__ h, double* __restrict__ og,
                           double* __restrict__ oh) {
    using R = typename SP::real;
    const StepParams& P = K.P;
    const Coef<R>& C = coef<R>(K);
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const long long j = storage_index(P, i);
    const R ph = phi[j], cc = c[j];
    const R Ps = divw<LH::DEN>(p_term(C, ph, closure_mu(C, ph, cc)));
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const R wk = R(L::w(k));
        if (og) og[(long long)k * P.N + i] = (double)SP::load(g, (long long)k * P.NS + j, wk * ph);
    }
#pragma unroll
    for (int k = 0; k < LH::Q; ++k) {
        const R heq = (k == 0) ? cc - R(LH::DEN - LH::m(0)) * Ps : R(LH::m(k)) * Ps;
        if (oh) oh[(long long)k * P.N + i] = (double)SP::load(h, (long long)k * P.NS + j, heq);
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

// Field sums for lbpf_mass: Sum c, Sum phi and the count of nodes outside the
// stable range, per block.  The fields are the context's own dense arrays
// (16-byte aligned); each thread keeps 2 x UNR vector loads per array in
// flight, so that the pass runs at the speed of its memory traffic instead of
// one load latency per element.
template <typename R>
__global__ void __launch_bounds__(kMassThreads)
k_mass_partial(const R* __restrict__ c, const R* __restrict__ phi, long long n, double* __restrict__ partials) {
    constexpr int UNR = 4;
    double sc = 0.0, sp = 0.0, bad = 0.0;
    const long long stride = (long long)gridDim.x * kMassThreads * UNR;
    if constexpr (sizeof(R) == 4) {
        // FP32 fields: exact float-float partial sums (TwoSum) of each thread's
        // 16 values per round, then added in FP64, and the range tests in FP32
        // (the FP64 pipe runs at a small fraction of the FP32 rate).
        const long long n4 = n / 4;
        const float4* c4 = reinterpret_cast<const float4*>(c);
        const float4* p4 = reinterpret_cast<const float4*>(phi);
        unsigned nbad = 0;
        float lc = 0.0f, lp = 0.0f;
        auto take = [&](float cv, float pv, MassAcc<float>& ac, MassAcc<float>& ap) {
            ac.add(cv, 0.0f);
            ap.add(pv, 0.0f);
            // non-finite values fail both comparisons and count as bad
            if (!(pv >= -0.5f && pv <= 1.5f) || !(cv == cv && cv - cv == 0.0f)) ++nbad;
        };
        for (long long j0 = (long long)blockIdx.x * kMassThreads * UNR + threadIdx.x; j0 < n4; j0 += stride) {
            float4 cv[UNR], pv[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const long long j = j0 + (long long)u * kMassThreads;
                cv[u] = j < n4 ? c4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                pv[u] = j < n4 ? p4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            MassAcc<float> ac{0.0f, 0.0f}, ap{0.0f, 0.0f};
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                take(cv[u].x, pv[u].x, ac, ap);
                take(cv[u].y, pv[u].y, ac, ap);
                take(cv[u].z, pv[u].z, ac, ap);
                take(cv[u].w, pv[u].w, ac, ap);
            }
            // the small parts go on in FP32 (each is a few ulps of its round's
            // sum): one conversion and one FP64 add per field and round
            sc += (double)ac.hi;
            sp += (double)ap.hi;
            lc += ac.lo;
            lp += ap.lo;
        }
        if (blockIdx.x == 0) {               // the last n mod 4 values
            for (long long i = 4 * n4 + threadIdx.x; i < n; i += kMassThreads) {
                MassAcc<float> ac{0.0f, 0.0f}, ap{0.0f, 0.0f};
                take(c[i], phi[i], ac, ap);
                sc += (double)ac.hi;
                sp += (double)ap.hi;
            }
        }
        sc += (double)lc;
        sp += (double)lp;
        bad = (double)nbad;
    } else {
        const long long n2 = n / 2;
        const double2* c2 = reinterpret_cast<const double2*>(c);
        const double2* p2 = reinterpret_cast<const double2*>(phi);
        auto take = [&](double cv, double pv) {
            sc += cv;
            sp += pv;
            if (!(pv >= -0.5 && pv <= 1.5) || !(cv == cv && cv - cv == 0.0)) bad += 1.0;
        };
        for (long long j0 = (long long)blockIdx.x * kMassThreads * UNR + threadIdx.x; j0 < n2; j0 += stride) {
            double2 cv[UNR], pv[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const long long j = j0 + (long long)u * kMassThreads;
                cv[u] = j < n2 ? c2[j] : make_double2(0.0, 0.0);
                pv[u] = j < n2 ? p2[j] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                take(cv[u].x, pv[u].x);
                take(cv[u].y, pv[u].y);
            }
        }
        if (blockIdx.x == 0)
            for (long long i = 2 * n2 + threadIdx.x; i < n; i += kMassThreads) take(c[i], phi[i]);
    }
    block_sum3<R>(sc, sp, bad);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = sc;
        partials[3 * blockIdx.x + 1] = sp;
        partials[3 * blockIdx.x + 2] = bad;
    }
}

static __global__ void __launch_bounds__(kMassThreads)
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


// ---- exact population mass and the closed-loop mass correction ------------------
// The solute mass of a state is the sum of its h populations (the zeroth moment,
// Eq. Moment0_LBM_Concent).  In FP32 the collision and the stored fields round
// at ~1e-7 relative per value; near-stationary nodes whose values sit on a
// binade boundary (c = 1 in the solid) round asymmetrically, so the total drifts
// by ~1e-9 per step.  When enabled, the composition kernel sums the exact mass
// of what it wrote (mass_partials), k_mass_corr_plan compares it with the
// target in FP64, and k_mass_corr_apply adds the difference back to the rest
// population and to c on a rotating subset of nodes, large enough per node
// (~1e-5) to be represented with ~1% rounding.  The next step measures again,
// so the residual never accumulates.

struct MassCorr {
    double target;      // mass to hold: the exact population mass at creation
    double measured;    // exact population mass after the last measured step
    double delta;       // increment per corrected node in the last correction
    long long count;    // nodes corrected by the last correction
    unsigned long long round;  // corrections planned so far (rotates the node subset)
};

// One block of kPlanThreads: the partial sums (one per composition-kernel
// block, thousands) take a few loads per thread.
constexpr int kPlanThreads = 1024;
static __global__ void __launch_bounds__(kPlanThreads)
k_mass_corr_plan(const double* __restrict__ partials, int nblocks, MassCorr* __restrict__ mc, long long N,
                 double delta_target) {
    __shared__ double red[kPlanThreads / 32];
    double sc = 0.0;
    // unrolled so that a thread's loads are in flight together (the adds keep
    // their order, so the sum does not depend on the unrolling)
#pragma unroll 4
    for (int b = threadIdx.x; b < nblocks; b += kPlanThreads) sc += partials[b];
    for (int o = 16; o > 0; o >>= 1) sc += __shfl_down_sync(0xffffffffu, sc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sc;
    __syncthreads();
    if (threadIdx.x < 32) {
        sc = red[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) sc += __shfl_down_sync(0xffffffffu, sc, o);
    }
    if (threadIdx.x == 0) {
        const double dM = mc->target - sc;
        long long k = 0;
        // a non-finite mass (a state that has blown up) corrects nothing: the
        // node count stays within [0, N] whatever the partial sums hold
        if (dM != 0.0 && isfinite(dM)) {
            const double want = fabs(dM) / delta_target;
            k = want < 1.0 ? 1 : (want > (double)N ? N : (long long)llrint(want));
        }
        mc->measured = sc;
        mc->count = k;
        mc->delta = k > 0 ? dM / (double)k : 0.0;
        mc->round += 1;
    }
}

// Node j of the correction is (offset + j * stride) mod N; stride is a large
// prime coprime with N, and offset = 7919 * round mod N rotates with every
// correction, so no node is corrected repeatedly.  Everything it needs is read
// on the device, so the correction can be replayed from a captured graph.
template <class SP>
__global__ void k_mass_corr_apply(const MassCorr* __restrict__ mc, typename SP::real* __restrict__ c,
                                  typename SP::store_t* __restrict__ h0, long long N, long long stride) {
    using R = typename SP::real;
    const long long count = mc->count;
    const long long offset = (long long)((mc->round * 7919ULL) % (unsigned long long)N);
    const R d = R(mc->delta);
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < count;
         j += (long long)gridDim.x * blockDim.x) {
        const long long i = (long long)(((unsigned long long)offset + (unsigned long long)j * (unsigned long long)stride) %
                                        (unsigned long long)N);
        c[i] += d;
        // deviation storage: the stored h are deviations from references whose
        // sum is c, so raising c raises the populations' sum by the same amount
        if (!SP::deviation) {
            R* hp = reinterpret_cast<R*>(h0);
            hp[i] += d;
        }
    }
}

// Exact FP64 population mass: h_k expanded (deviation modes add their references
// back), summed per node in float-float, per block in FP64.  L: the h lattice.
template <class L, class SP>
__global__ void __launch_bounds__(kMassThreads)
k_pop_mass(const KParams K, const typename SP::real* __restrict__ phi, const typename SP::real* __restrict__ c,
           const typename SP::store_t* __restrict__ h, double* __restrict__ partials) {
    using R = typename SP::real;
    const StepParams& P = K.P;
    const Coef<R>& C = coef<R>(K);
    MassAcc<R> acc{R(0), R(0)};
    for (long long id = blockIdx.x * (long long)kMassThreads + threadIdx.x; id < P.N;
         id += (long long)gridDim.x * kMassThreads) {
        const long long i = storage_index(P, id);
        const R ph = phi[i], cc = c[i];
        const R Ps = divw<L::DEN>(p_term(C, ph, closure_mu(C, ph, cc)));
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const R ref = (k == 0) ? cc - R(L::DEN - L::m(0)) * Ps : R(L::m(k)) * Ps;
            acc.add(SP::load(h, (long long)k * P.NS + i, ref), R(0));
        }
    }
    double v = (double)acc.hi + (double)acc.lo, d1 = 0.0, d2 = 0.0;
    block_sum3<double>(v, d1, d2);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = v;
        partials[3 * blockIdx.x + 1] = 0.0;
        partials[3 * blockIdx.x + 2] = 0.0;
    }
}

}  // namespace lbpf
