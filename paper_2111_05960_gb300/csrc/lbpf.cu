// libgb_lbpf: runtime and C ABI of the coupled phi-mu LBM step (see lbpf.h).
//
// The context owns two ping-pong sets of populations (g, h; SoA [k][z][y][x])
// and two of the fields phi, c.  A time step is the phi kernel followed by the
// composition kernel on the context's stream; the buffer parity flips after
// each step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "context.cuh"

using namespace lbpf;
using namespace lbpf_rt;

namespace {
thread_local std::string g_thread_error;
}  // namespace

void lbpf_internal_set_thread_error(const std::string& msg) { g_thread_error = msg; }
void lbpf_rt::set_thread_error(const std::string& msg) { g_thread_error = msg; }

// ---- helpers shared with adjoint.cu ---------------------------------------------

lbpf_status lbpf_rt::fail(lbpf_ctx* ctx, lbpf_status st, const std::string& msg) {
    if (ctx) ctx->err = msg; else g_thread_error = msg;
    return st;
}

lbpf_status lbpf_rt::cuda_fail(lbpf_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? LBPF_ENOMEM : LBPF_ECUDA, m);
}

lbpf_status lbpf_rt::alloc(lbpf_ctx* ctx, void** ptr, size_t bytes, const char* what) {
    if (const char* f = getenv("LBPF_FAULT")) {
        if (strcmp(f, "alloc") == 0) return fail(ctx, LBPF_ENOMEM, std::string("injected allocation failure: ") + what);
    }
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return cuda_fail(ctx, e, what);
    }
    return LBPF_OK;
}

lbpf_status lbpf_rt::ensure_staging(lbpf_ctx* ctx) {
    if (ctx->staging) return LBPF_OK;
    return alloc(ctx, (void**)&ctx->staging, sizeof(double) * 3 * (size_t)ctx->sp.N, "staging");
}

lbpf_status lbpf_rt::check_launch(lbpf_ctx* ctx, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    return LBPF_OK;
}

namespace {

// ---- per (lattice, storage) dispatch ---------------------------------------------

// Tile shapes of the z-marching kernels: BX x BY threads per block, ZCH planes
// per block, at least MINB resident blocks per SM (register budget).  2-D
// domains march along y through the D2Q9R view: BX-long row segments, ZCH rows
// per block.  Overridable at build time.
#ifndef LBPF_BX2
#define LBPF_BX2 128
#endif
#ifndef LBPF_YCH2
#define LBPF_YCH2 16
#endif
#ifndef LBPF_MINB2
#define LBPF_MINB2 8
#endif
#ifndef LBPF_MINB2_F64
#define LBPF_MINB2_F64 6
#endif
// 3-D, FP32 arithmetic (FP32 and 16-bit storage): 32 x 4 tiles, 48 planes
// (at 256^3: 6 chunks, the last of 16 planes, 3.4 waves of blocks), 6 blocks
// per SM; FP64: 32 x 8 tiles, 16 planes, 2 blocks per SM (register bound).
// Chosen by timing the 256^3 porous step on GB300.
#ifndef LBPF_BY3
#define LBPF_BY3 4
#endif
#ifndef LBPF_ZCH3
#define LBPF_ZCH3 48
#endif
#ifndef LBPF_MINB3
#define LBPF_MINB3 6
#endif
#ifndef LBPF_BY3_F64
#define LBPF_BY3_F64 8
#endif
#ifndef LBPF_ZCH3_F64
#define LBPF_ZCH3_F64 16
#endif
#ifndef LBPF_MINB3_F64
#define LBPF_MINB3_F64 2
#endif
// The composition kernel with h on D3Q7 pulls 7 instead of 19 populations, so
// its ingredient work (the D3Q19 gradient on the tile's ring) weighs more and
// it gets its own FP32 tile: 32 x 8 with 24 planes and 4 blocks per SM
// (64 registers, no spills) recomputes a smaller share of ring nodes than
// 32 x 4 and ran 2.5% faster on the 256^3 step (16 x 32 and 6 blocks of 32 x 4
// were slower); 24 planes per block ran 1.6% faster than 16, 32 or 48.
#ifndef LBPF_BY3_HS
#define LBPF_BY3_HS 8
#endif
#ifndef LBPF_ZCH3_HS
#define LBPF_ZCH3_HS 24
#endif
#ifndef LBPF_MINB3_HS
#define LBPF_MINB3_HS 4
#endif
#ifndef LBPF_MINB3_TMA
#define LBPF_MINB3_TMA 6
#endif
// Increment per corrected node of the mass correction: ~100 ulps of an FP32
// value near 1, so that each node's rounding is ~1% of the increment.
constexpr double kCorrDelta = 1e-5;

template <class L, bool F64>
struct TileCfg;
template <bool F64>
struct TileCfg<D2Q9, F64> {
    using ML = D2Q9R;
    static constexpr int BX = LBPF_BX2, BY = 1, ZCH = LBPF_YCH2, MINB = F64 ? LBPF_MINB2_F64 : LBPF_MINB2;
};
template <>
struct TileCfg<D3Q19, false> {
    using ML = D3Q19;
    static constexpr int BX = 32, BY = LBPF_BY3, ZCH = LBPF_ZCH3, MINB = LBPF_MINB3;
};
// the composition kernel's tile: the same, except for h on the small lattice in
// 3-D FP32 arithmetic
template <class L, bool F64, bool HS>
struct TileCfgC : TileCfg<L, F64> {};
template <>
struct TileCfgC<D3Q19, false, true> : TileCfg<D3Q19, false> {
    static constexpr int BY = LBPF_BY3_HS, ZCH = LBPF_ZCH3_HS, MINB = LBPF_MINB3_HS;
};
template <>
struct TileCfg<D3Q19, true> {
    using ML = D3Q19;
    static constexpr int BX = 32, BY = LBPF_BY3_F64, ZCH = LBPF_ZCH3_F64, MINB = LBPF_MINB3_F64;
};

// Tensor map of one population buffer as a 4-D array (x, y, z, k) with the
// row, plane and population strides of P, read in boxes of box_x x box_y x 1 x 1
// values; rows and columns outside the grid read as zeros.
using TensorMapEncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                          const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                          CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                          CUtensorMapFloatOOBfill);
bool encode_pop_map(CUtensorMap* m, void* base, const StepParams& P, int q, int box_x, int box_y) {
    static const TensorMapEncodeTiled encode = []() -> TensorMapEncodeTiled {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult qr = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<TensorMapEncodeTiled>(f);
    }();
    if (!encode) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, (cuuint64_t)P.nz, (cuuint64_t)q};
    const cuuint64_t strides[3] = {(cuuint64_t)P.sx * 4, (cuuint64_t)P.sxy * 4, (cuuint64_t)P.NS * 4};
    const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1, 1};
    const cuuint32_t elem[4] = {1, 1, 1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Planes per block of a 3-D step kernel: tiles x-y tiles, nz planes, resident
// blocks per wave, def the default chunk (see Impl::prepare).
int pick_zch(long long tiles, int nz, long long resident, int def) {
    auto waves = [&](int z) { return (double)(tiles * ((nz + z - 1) / z)) / (double)resident; };
    if (waves(def) >= 3.0) return def;
    for (int z : {24, 16, 12, 8})
        if (waves(z) >= 3.0) return z;
    int best = def;
    double best_fill = -1.0;
    for (int z : {8, 12, 16, 24}) {
        const double W = waves(z);
        if (W < 1.5) continue;
        const double fill = W / std::ceil(W);
        if (fill >= best_fill) {
            best_fill = fill;
            best = z;
        }
    }
    return best;
}

// HS: h on the small lattice of L (D2Q5 / D3Q7) instead of L itself.
template <class L, class SP, bool HS = false>
struct Impl {
    using R = typename SP::real;
    using S = typename SP::store_t;
    using T = TileCfg<L, sizeof(R) == 8>;
    using ML = typename T::ML;              // the lattice as the marching kernels see it
    using MLH = typename std::conditional<HS, typename SmallOf<ML>::type, ML>::type;   // h, marching view
    using LH = typename std::conditional<HS, typename SmallOf<L>::type, L>::type;      // h, grid view
    using TC = TileCfgC<L, sizeof(R) == 8, HS>;
    static constexpr int BX = T::BX, BY = T::BY, ZCH = T::ZCH, MINB = T::MINB;
    static constexpr int BYC = TC::BY, ZCHC = TC::ZCH, MINBC = TC::MINB;
    static constexpr size_t smem_phi = march_smem<ML, SP, BY, BX>(true);
    static constexpr size_t smem_c = march_smem<ML, SP, BYC, BX>(false);
    // pulls through tensor maps: FP32 storage on the 3-D lattices, periodic
    // domains (the kernels' TMA form)
    static constexpr bool TMA_OK = std::is_same<S, float>::value && L::D == 3;
    static constexpr size_t smem_phi_t = march_smem<ML, SP, BY, BX, MLH>(true, true);
    static constexpr size_t smem_c_t = march_smem<ML, SP, BYC, BX, MLH>(false, true);
    static_assert(smem_phi_t <= 227 * 1024 && smem_c_t <= 227 * 1024, "a block's shared memory");
    // the TMA kernels' stages take ~9 KB more shared memory per block (6 blocks
    // of the FP32 D3Q19 tile still fit)
    template <bool W, bool T = false>
    static constexpr auto kphi() { return k_phi_step<ML, SP, BY, T ? LBPF_MINB3_TMA : MINB, W, BX, T>; }
    template <bool W, bool T = false>
    static constexpr auto kc() {
        return k_c_step<ML, SP, BYC, T ? (LBPF_MINB3_TMA < MINBC ? LBPF_MINB3_TMA : MINBC) : MINBC, W, BX, MLH, T>;
    }

    static lbpf_status prepare(lbpf_ctx* ctx) {
        ctx->zch_phi = ZCH;
        ctx->zch_c = ZCHC;
        if constexpr (L::D == 3) {
            // 3-D: planes per block.  Grids of at least 3 waves of resident blocks
            // at the default chunk keep it; smaller ones take the longest chunk of
            // 24, 16, 12 or 8 planes that still gives 3 waves, else the one whose
            // last wave is fullest among those with at least 1.5 waves (the
            // longer on a tie): on GB300 128^3 went from 12.2 to 13.5 GLUPS (12
            // planes), 160^3 from 12.8 to 14.6 (12), 192^3 from 15.0 to 15.3
            // (16); 256^3 keeps 32.
            int sms = 0, occ_phi = 0, occ_c = 0;
            const bool w = walls(ctx);
            LBPF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
            LBPF_CUDA(ctx, cudaFuncSetAttribute(w ? kphi<true>() : kphi<false>(),
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_phi));
            LBPF_CUDA(ctx, cudaFuncSetAttribute(w ? kc<true>() : kc<false>(),
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
            LBPF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_phi, w ? kphi<true>() : kphi<false>(),
                                                                         BX * BY, smem_phi));
            LBPF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, w ? kc<true>() : kc<false>(),
                                                                         BX * BYC, smem_c));
            const StepParams& P = ctx->kpm.P;
            const long long tx = (P.nx + BX - 1) / BX;
            ctx->zch_phi = pick_zch(tx * ((P.ny + BY - 1) / BY), P.nz, (long long)sms * std::max(1, occ_phi), ZCH);
            ctx->zch_c = pick_zch(tx * ((P.ny + BYC - 1) / BYC), P.nz, (long long)sms * std::max(1, occ_c), ZCHC);
        }
        if constexpr (L::D == 2) {
            // 2-D: rows per block.  The shortest chunk of 4, 8, 16, 32 rows whose
            // grid fits in one wave of resident blocks (every block runs at once,
            // no tail), else the default; on GB300 this took the 512^2 disc from
            // 6.6 to 10.2 GLUPS, the 1024^2 slice of Sec. 5 from 15.2 to 17.5 and
            // 2048^2 from 26.0 to 27.1 (4096^2 keeps 16 rows: 30.8).
            int sms = 0, occ_phi = 0, occ_c = 0;
            const bool w = walls(ctx);
            LBPF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
            LBPF_CUDA(ctx, cudaFuncSetAttribute(w ? kphi<true>() : kphi<false>(),
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_phi));
            LBPF_CUDA(ctx, cudaFuncSetAttribute(w ? kc<true>() : kc<false>(),
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
            LBPF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_phi, w ? kphi<true>() : kphi<false>(),
                                                                         BX * BY, smem_phi));
            LBPF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, w ? kc<true>() : kc<false>(),
                                                                         BX * BYC, smem_c));
            const long long resident = (long long)sms * std::max(1, std::min(occ_phi, occ_c));
            const StepParams& P = ctx->kpm.P;     // rows are the planes of the marching view
            const long long tiles_x = (P.nx + BX - 1) / BX;
            for (int rows : {4, 8, 16, 32}) {
                if (tiles_x * ((P.nz + rows - 1) / rows) <= resident) {
                    ctx->zch_phi = ctx->zch_c = rows;
                    break;
                }
            }
        }
        LBPF_CUDA(ctx, cudaFuncSetAttribute(kphi<true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_phi));
        LBPF_CUDA(ctx, cudaFuncSetAttribute(kc<true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        LBPF_CUDA(ctx, cudaFuncSetAttribute(kphi<false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_phi));
        LBPF_CUDA(ctx, cudaFuncSetAttribute(kc<false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        if constexpr (TMA_OK) {
            LBPF_CUDA(ctx, cudaFuncSetAttribute(kphi<false, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem_phi_t));
            LBPF_CUDA(ctx, cudaFuncSetAttribute(kc<false, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem_c_t));
        }
        return LBPF_OK;
    }
    // maps of the context's g and h buffers for the TMA kernels (boxes of BX x
    // BY values); false: this context pulls with loads only (walls, 16-bit or
    // FP64 storage, rows whose byte stride is not a multiple of 16, or a grid
    // narrower than one box)
    static bool setup_tensor_maps(lbpf_ctx* ctx) {
        if constexpr (!TMA_OK) {
            return false;
        } else {
            const StepParams& P = ctx->kpm.P;
            if (walls(ctx) || P.sx != P.nx || P.nx % 4 != 0 || P.nx < BX) return false;
            for (int i = 0; i < 2; ++i) {
                if (!encode_pop_map(&ctx->gmap[i], ctx->g[i], P, ML::Q, BX, BY)) return false;
                if (!encode_pop_map(&ctx->hmap[i], ctx->h[i], P, MLH::Q, BX, BYC)) return false;
            }
            return true;
        }
    }
    static bool walls(const lbpf_ctx* ctx) {
        const StepParams& P = ctx->sp;
        return P.bc[0] || P.bc[1] || (L::D == 3 && P.bc[2]);
    }
    // grid over the marching view (kpm: 2-D domains as [ny][1][nx])
    static dim3 grid(const lbpf_ctx* ctx) {
        const StepParams& P = ctx->kpm.P;
        return dim3((P.nx + BX - 1) / BX, (P.ny + BY - 1) / BY, (P.nz + ctx->zch_phi - 1) / ctx->zch_phi);
    }
    static dim3 grid_c(const lbpf_ctx* ctx) {
        const StepParams& P = ctx->kpm.P;
        return dim3((P.nx + BX - 1) / BX, (P.ny + BYC - 1) / BYC, (P.nz + ctx->zch_c - 1) / ctx->zch_c);
    }
    static void launch_phi_p(lbpf_ctx* ctx, const void* g, void* g_out, const void* phi, const void* c,
                             void* phi_out) {
        auto kern = walls(ctx) ? kphi<true>() : kphi<false>();
        kern<<<grid(ctx), dim3(BX, BY), smem_phi, ctx->stream>>>(ctx->kpm, (const S*)g, (S*)g_out, (const R*)phi,
                                                                   (const R*)c, (R*)phi_out, ctx->zch_phi,
                                                                   ctx->nomap, ctx->d_err);
    }
    static void launch_c_p(lbpf_ctx* ctx, const void* h, void* h_out, const void* phi, const void* phi_out,
                           const void* c, void* c_out, double* mass_partials) {
        auto kern = walls(ctx) ? kc<true>() : kc<false>();
        kern<<<grid_c(ctx), dim3(BX, BYC), smem_c, ctx->stream>>>(ctx->kpm, (const S*)h, (S*)h_out, (const R*)phi,
                                                                 (const R*)phi_out, (const R*)c, (R*)c_out,
                                                                 mass_partials, ctx->zch_c, ctx->nomap, ctx->d_err);
    }
    static void launch_phi(lbpf_ctx* ctx, int cur) {
        const int nxt = cur ^ 1;
        if constexpr (TMA_OK) {
            if (ctx->tma) {
                kphi<false, true>()<<<grid(ctx), dim3(BX, BY), smem_phi_t, ctx->stream>>>(
                    ctx->kpm, (const S*)ctx->g[cur], (S*)ctx->g[nxt], (const R*)ctx->phi[cur], (const R*)ctx->c[cur],
                    (R*)ctx->phi[nxt], ctx->zch_phi, ctx->gmap[cur], ctx->d_err);
                return;
            }
        }
        launch_phi_p(ctx, ctx->g[cur], ctx->g[nxt], ctx->phi[cur], ctx->c[cur], ctx->phi[nxt]);
    }
    static void launch_c(lbpf_ctx* ctx, int cur, double* mass_partials) {
        const int nxt = cur ^ 1;
        if constexpr (TMA_OK) {
            if (ctx->tma) {
                kc<false, true>()<<<grid_c(ctx), dim3(BX, BYC), smem_c_t, ctx->stream>>>(
                    ctx->kpm, (const S*)ctx->h[cur], (S*)ctx->h[nxt], (const R*)ctx->phi[cur],
                    (const R*)ctx->phi[nxt], (const R*)ctx->c[cur], (R*)ctx->c[nxt], mass_partials, ctx->zch_c,
                    ctx->hmap[cur], ctx->d_err);
                return;
            }
        }
        launch_c_p(ctx, ctx->h[cur], ctx->h[nxt], ctx->phi[cur], ctx->phi[nxt], ctx->c[cur], ctx->c[nxt],
                   mass_partials);
    }
    static void launch_init(lbpf_ctx* ctx) {
        const long long N = ctx->sp.N;
        k_init<L, SP, LH><<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(
            ctx->kp, (const R*)ctx->phi[ctx->cur], (R*)ctx->c[ctx->cur], (S*)ctx->g[ctx->cur],
            (S*)ctx->h[ctx->cur]);
    }
    static void launch_pops_out(lbpf_ctx* ctx, double* g, double* h) {
        const long long N = ctx->sp.N;
        const int cur = ctx->cur;
        k_pops_out<L, SP, LH><<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(
            ctx->kp, (const R*)ctx->phi[cur], (const R*)ctx->c[cur], (const S*)ctx->g[cur],
            (const S*)ctx->h[cur], g, h);
    }
    // mass correction after a composition step whose new state has parity `cur_after`
    static void launch_corr_p(lbpf_ctx* ctx, MassCorr* mc, void* c, void* h) {
        k_mass_corr_plan<<<1, kPlanThreads, 0, ctx->stream>>>(ctx->corr_partials, ctx->corr_blocks, mc,
                                                             ctx->sp.N, kCorrDelta);
        k_mass_corr_apply<SP><<<64, 256, 0, ctx->stream>>>(mc, (R*)c, (S*)h, ctx->sp.N, ctx->corr_stride);
    }
    static void launch_corr(lbpf_ctx* ctx, int cur_after) {
        launch_corr_p(ctx, ctx->corr, ctx->c[cur_after], ctx->h[cur_after]);
    }
    static void launch_pop_mass(lbpf_ctx* ctx) {
        k_pop_mass<LH, SP><<<ctx->mass_blocks, kMassThreads, 0, ctx->stream>>>(
            ctx->kp, (const R*)ctx->phi[ctx->cur], (const R*)ctx->c[ctx->cur], (const S*)ctx->h[ctx->cur],
            ctx->partials);
        k_mass_final<<<1, kMassThreads, 0, ctx->stream>>>(ctx->partials, ctx->mass_blocks, ctx->mass_out);
    }
    static int c_blocks(const lbpf_ctx* ctx) {
        const dim3 g = grid_c(ctx);
        return (int)(g.x * g.y * g.z);
    }
    static const Dispatch* table() {
        static const Dispatch d = {prepare,         launch_phi,   launch_c,   launch_init,
                                   launch_pops_out, launch_corr,  launch_pop_mass, c_blocks,
                                   launch_phi_p,    launch_c_p,   launch_corr_p, setup_tensor_maps};
        return &d;
    }
};

template <class L, bool HS>
const Dispatch* pick_storage(int precision) {
    switch (precision) {
        case LBPF_FP64: return Impl<L, StoreF64, HS>::table();
        case LBPF_FP32: return Impl<L, StoreF32, HS>::table();
        case LBPF_FP32_BF16DEV: return Impl<L, StoreBF16Dev, HS>::table();
        case LBPF_FP32_FP16DEV: return Impl<L, StoreF16Dev, HS>::table();
    }
    return nullptr;
}

const Dispatch* pick(int lattice, int precision, bool h_small) {
    if (lattice == LBPF_D2Q9) return h_small ? pick_storage<D2Q9, true>(precision) : pick_storage<D2Q9, false>(precision);
    if (lattice == LBPF_D3Q19) return h_small ? pick_storage<D3Q19, true>(precision) : pick_storage<D3Q19, false>(precision);
    return nullptr;
}

}  // namespace

// ---- helpers shared with batch.cu and adjoint.cu -----------------------------------

lbpf_status lbpf_rt::validate(const lbpf_params* p, std::string& why) {
    auto bad = [&](const char* m) { why = m; return LBPF_EINVAL; };
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return bad("grid sizes must be >= 1");
    if (p->lattice != LBPF_D2Q9 && p->lattice != LBPF_D3Q19) return bad("unknown lattice");
    if (p->lattice == LBPF_D2Q9 && p->nz != 1) return bad("D2Q9 needs nz == 1");
    if ((long long)p->nx * p->ny * p->nz > (1LL << 40)) return bad("grid too large");
    if ((long long)p->nx * p->ny >= (1LL << 31)) return bad("a z-plane must hold fewer than 2^31 nodes");
    for (int a = 0; a < 3; ++a) {
        if (p->bc[a] != LBPF_PERIODIC && p->bc[a] != LBPF_BOUNCEBACK) return bad("unknown boundary type");
        const int n = a == 0 ? p->nx : (a == 1 ? p->ny : p->nz);
        const bool active = a < 2 || p->lattice == LBPF_D3Q19;
        if (active && p->bc[a] == LBPF_BOUNCEBACK && n < 2) return bad("a bounce-back axis needs >= 2 nodes");
    }
    if (p->precision < LBPF_FP64 || p->precision > LBPF_FP32_FP16DEV) return bad("unknown precision");
    if (!(p->dx > 0) || !(p->dt > 0)) return bad("dx and dt must be > 0");
    if (!(p->tau_g > 0) || !(p->tau_h > 0)) return bad("tau_g and tau_h must be > 0");
    if (!(p->W > 0)) return bad("W must be > 0");
    if (!(p->D_l >= 0) || !(p->D_s >= 0)) return bad("diffusivities must be >= 0");
    if (!std::isfinite(p->lambda) || !std::isfinite(p->c_s_co) || !std::isfinite(p->c_l_co) ||
        !std::isfinite(p->mu_eq) || !std::isfinite(p->a_at) || !(p->eps_n >= 0))
        return bad("non-finite parameter");
    if (p->anti_trapping && p->a_at < 0 && !(p->D_l > 0)) return bad("automatic a needs D_l > 0");
    if (p->mass_every < 0) return bad("mass_every must be >= 0");
    if (p->checkpoint_every < 0) return bad("checkpoint_every must be >= 0");
    if (p->h_lattice != 0 && p->h_lattice != 1) return bad("h_lattice must be 0 or 1");
    if (p->h_eq_alt != 0 && p->h_eq_alt != 1) return bad("h_eq_alt must be 0 or 1");
    if (p->unequal_eps != 0 && p->unequal_eps != 1) return bad("unequal_eps must be 0 or 1");
    if (p->unequal_eps && !(p->eps_ratio > 0 && std::isfinite(p->eps_ratio))) return bad("eps_ratio must be > 0");
    return LBPF_OK;
}

StepParams lbpf_rt::lattice_units(const lbpf_params* p) {
    StepParams s;
    s.nx = p->nx; s.ny = p->ny; s.nz = p->nz;
    for (int a = 0; a < 3; ++a) s.bc[a] = p->bc[a];
    if (p->lattice == LBPF_D2Q9) s.bc[2] = LBPF_PERIODIC;
    s.N = (long long)p->nx * p->ny * p->nz;
    s.sx = p->nx;
    s.sxy = (long long)p->nx * p->ny;
    s.NS = s.N;
    s.omg = 1.0 / (p->tau_g + 0.5);
    s.omh = 1.0 / (p->tau_h + 0.5);
    s.M = p->tau_g / 3.0;
    s.gamma = 3.0 / p->tau_h;
    const double dfac = p->dt / (p->dx * p->dx);
    s.W = p->W / p->dx;
    s.lambda = p->lambda;
    s.D_l = p->D_l * dfac;
    s.D_s = p->D_s * dfac;
    s.c_s = p->c_s_co; s.c_l = p->c_l_co; s.mu_eq = p->mu_eq;
    double a = p->a_at;
    if (a < 0) a = 0.25 * (1.0 - p->D_s / p->D_l);
    s.a_at = p->anti_trapping ? a : 0.0;
    s.eps2 = p->eps_n * p->eps_n;
    s.counter_term = p->counter_term ? 1 : 0;
    s.h_den = p->h_lattice ? 6 : 36;     // w_k = m_k / DEN on the h lattice
    s.h_eq_alt = p->h_eq_alt ? 1 : 0;
    // parabolas: the minima and Delta f^min from the two equilibrium conditions
    // (equal mu at the coexistence compositions, equal grand potentials at mu_eq)
    s.unequal = p->unequal_eps ? 1 : 0;
    s.e_s = p->unequal_eps ? std::sqrt(p->eps_ratio) : 1.0;
    s.e_l = 1.0 / s.e_s;
    s.m_l = s.c_l - s.e_s * s.mu_eq;
    s.m_s = s.c_s - s.e_l * s.mu_eq;
    s.df = 0.5 * (s.e_l - s.e_s) * s.mu_eq * s.mu_eq - (s.m_l - s.m_s) * s.mu_eq;
    return s;
}

// Geometry, coefficients (FP64 and FP32) and link offsets of one simulation;
// rows of sx >= nx elements (sx = 0: dense rows, sx = nx).
KParams lbpf_rt::make_kparams(const lbpf_params* p, int sx) {
    KParams kp;
    kp.P = lattice_units(p);
    if (sx > p->nx) {
        kp.P.sx = sx;
        kp.P.sxy = (long long)sx * p->ny;
        kp.P.NS = kp.P.sxy * p->nz;
    }
    kp.cd = make_coef<double>(kp.P);
    kp.cf = make_coef<float>(kp.P);
    const int q = p->lattice == LBPF_D3Q19 ? 19 : 9;
    const long long sb = p->precision == LBPF_FP64 ? 8 : (p->precision == LBPF_FP32 ? 4 : 2);
    const bool fits = (long long)q * kp.P.NS * sb < (1LL << 31);
    for (int k = 0; k < 19; ++k) {
        int e[3] = {0, 0, 0};
        if (k < q) {
            if (p->lattice == LBPF_D3Q19) { e[0] = D3Q19::ex(k); e[1] = D3Q19::ey(k); e[2] = D3Q19::ez(k); }
            else { e[0] = D2Q9::ex(k); e[1] = D2Q9::ey(k); }
        }
        const long long nx = kp.P.sx, nxy = kp.P.sxy;
        kp.kNB[k] = (long long)k * kp.P.NS * sb;
        kp.koffB[k] = kp.kNB[k] - (e[0] + e[1] * nx + e[2] * nxy) * sb;
        kp.kNB32[k] = fits ? (int)kp.kNB[k] : 0;
        kp.koffB32[k] = fits ? (int)kp.koffB[k] : 0;
    }
    return kp;
}

// The marching kernels' view of the grid: a 2-D domain [ny][nx] is walked row by
// row as the 3-D grid [nz = ny][1][nx] (lattice D2Q9R, same link offsets).
KParams lbpf_rt::march_kparams(const KParams& kp, int lattice) {
    KParams m = kp;
    if (lattice == LBPF_D2Q9) {
        m.P.nz = kp.P.ny;
        m.P.ny = 1;
        m.P.sxy = kp.P.sx;      // a row is a plane of the march
        m.P.bc[2] = kp.P.bc[1];
        m.P.bc[1] = LBPF_PERIODIC;
    }
    return m;
}

void lbpf_rt::free_all(lbpf_ctx* ctx) {
    for (int i = 0; i < 2; ++i) {
        cudaFree(ctx->g[i]); cudaFree(ctx->h[i]); cudaFree(ctx->phi[i]); cudaFree(ctx->c[i]);
        ctx->g[i] = ctx->h[i] = ctx->phi[i] = ctx->c[i] = nullptr;
    }
    cudaFree(ctx->staging); cudaFree(ctx->partials); cudaFree(ctx->mass_out);
    ctx->staging = ctx->partials = ctx->mass_out = nullptr;
    cudaFree(ctx->corr_partials); cudaFree(ctx->corr);
    ctx->corr_partials = nullptr;
    ctx->corr = nullptr;
    cudaFree(ctx->d_binst); cudaFree(ctx->d_tile_inst);
    ctx->d_binst = nullptr;
    ctx->d_tile_inst = nullptr;
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
    free_adjoint(ctx);
}

namespace {

// One coupled step (both kernels), followed by the mass correction when it is due.
void launch_one_step(lbpf_ctx* ctx) {
    if (ctx->is_batch) {
        ctx->bops->launch_phi(ctx, ctx->cur);
        ctx->bops->launch_c(ctx, ctx->cur);
        ctx->cur ^= 1;
        ctx->step += 1;
        return;
    }
    const bool corr = ctx->corr && ((ctx->step + 1) % ctx->p.mass_every == 0);
    ctx->ops->launch_phi(ctx, ctx->cur);
    ctx->ops->launch_c(ctx, ctx->cur, corr ? ctx->corr_partials : nullptr);
    if (corr) ctx->ops->launch_corr(ctx, ctx->cur ^ 1);
    ctx->cur ^= 1;
    ctx->step += 1;
}

// nsteps steps, replaying two-step CUDA graphs where possible: on a non-default
// stream, when every step has the same kernels (mass correction off or every
// step).  The graph is captured once per context; if capture fails the steps
// are launched one by one.
lbpf_status run_steps(lbpf_ctx* ctx, int64_t nsteps) {
    if (ctx->p.checkpoint_every > 0 && !ctx->is_batch) {
        // adjoint recording: a checkpoint after every k-th step, no graphs
        for (int64_t s = 0; s < nsteps; ++s) {
            launch_one_step(ctx);
            if (ctx->step % ctx->p.checkpoint_every == 0) {
                lbpf_status st = record_checkpoint(ctx);
                if (st != LBPF_OK) return st;
            }
        }
        return check_launch(ctx, "step kernels");
    }
    const bool graphable = ctx->stream != nullptr && !ctx->graph_failed &&
                           (ctx->p.mass_every <= 1 || ctx->is_batch) && nsteps >= 3;
    if (!graphable) {
        for (int64_t s = 0; s < nsteps; ++s) launch_one_step(ctx);
        return check_launch(ctx, "step kernels");
    }
    if (ctx->cur == 1) { launch_one_step(ctx); --nsteps; }   // graphs start from parity 0
    if (!ctx->graph) {
        cudaGraph_t g = nullptr;
        const int64_t step0 = ctx->step;
        cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            launch_one_step(ctx);
            launch_one_step(ctx);
            e = cudaStreamEndCapture(ctx->stream, &g);
        }
        ctx->step = step0;          // capture only recorded the launches
        ctx->cur = 0;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->graph = nullptr;
            ctx->graph_failed = true;
            for (int64_t s = 0; s < nsteps; ++s) launch_one_step(ctx);
            return check_launch(ctx, "step kernels");
        }
    }
    for (; nsteps >= 2; nsteps -= 2) {
        cudaError_t e = cudaGraphLaunch(ctx->graph, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
        ctx->step += 2;
    }
    if (nsteps == 1) launch_one_step(ctx);
    return check_launch(ctx, "step kernels");
}

// A prime stride coprime with N for spreading the corrected nodes.
long long corr_stride_for(long long N) {
    const long long primes[] = {1000003LL, 998244353LL, 7919LL, 104729LL, 15485863LL};
    for (long long p : primes)
        if (N % p != 0) return p % N == 0 ? 1 : p;
    return 1;
}

template <typename R>
void launch_fields_out(lbpf_ctx* ctx, double* ophi, double* oc, double* omu) {
    const long long N = ctx->sp.N;
    k_fields_out<R><<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->kp, (const R*)ctx->phi[ctx->cur], (const R*)ctx->c[ctx->cur], ophi, oc, omu);
}

template <typename R>
void launch_mass(lbpf_ctx* ctx) {
    k_mass_partial<R><<<ctx->mass_blocks, kMassThreads, 0, ctx->stream>>>(
        (const R*)ctx->c[ctx->cur], (const R*)ctx->phi[ctx->cur], ctx->sp.N, ctx->partials);
    k_mass_final<<<1, kMassThreads, 0, ctx->stream>>>(ctx->partials, ctx->mass_blocks, ctx->mass_out);
}


}  // namespace

// ---- FP64 arithmetic rate (the ALU roofline of the FP64 step) ---------------------

constexpr int kFmaThreads = 256, kFmaChains = 8;
__device__ double g_fma_sink;

// kFmaChains independent FMA chains per thread, so the FP64 pipe, not the
// dependency latency, sets the rate; the result is kept so nothing is elided.
__global__ void __launch_bounds__(kFmaThreads) k_fp64_fma(int iters, double seed) {
    double a[kFmaChains];
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) a[j] = seed + 1e-3 * (threadIdx.x + j);
    const double m = 0.999999, c = 1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kFmaChains; ++j) a[j] = fma(a[j], m, c);
    }
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) t += a[j];
    if (t == -1.0) g_fma_sink = t;      // never true; keeps the chains alive
}

// ==== C ABI ======================================================================

extern "C" {

lbpf_status lbpf_default_params(lbpf_params* p) {
    if (!p) return fail(nullptr, LBPF_EINVAL, "params pointer is NULL");
    memset(p, 0, sizeof(*p));
    p->nx = 64; p->ny = 64; p->nz = 1;
    p->lattice = LBPF_D2Q9;
    p->precision = LBPF_FP64;
    p->dx = 1.0; p->dt = 1.0;
    p->tau_g = 0.36; p->tau_h = 0.36;
    p->W = 3.0; p->lambda = 0.0;
    p->D_l = 0.1; p->D_s = 0.1;
    p->c_s_co = 1.0; p->c_l_co = 0.5; p->mu_eq = 0.4;
    p->counter_term = 1; p->anti_trapping = 0; p->a_at = -1.0;
    p->eps_n = 1e-12;
    p->eps_ratio = 1.0;
    return LBPF_OK;
}

lbpf_status lbpf_create(const lbpf_params* p, const double* phi0, const double* c0, int32_t ptr_is_device,
                        void* cuda_stream, lbpf_ctx** out) {
    if (!out) return fail(nullptr, LBPF_EINVAL, "out pointer is NULL");
    *out = nullptr;
    if (!p || !phi0 || !c0) return fail(nullptr, LBPF_EINVAL, "NULL params or field pointer");
    std::string why;
    if (validate(p, why) != LBPF_OK) return fail(nullptr, LBPF_EINVAL, why);
    const Dispatch* ops = pick(p->lattice, p->precision, p->h_lattice != 0);
    if (!ops) return fail(nullptr, LBPF_EUNSUPPORTED, "lattice/precision not built");
    const AdjDispatch* aops = nullptr;
    if (p->checkpoint_every > 0) {
        if (p->h_lattice || p->h_eq_alt || p->unequal_eps)
            return fail(nullptr, LBPF_EUNSUPPORTED,
                        "the adjoint covers h on the lattice of g with H_k and equal curvatures only");
        aops = pick_adjoint(p->lattice, p->precision);
        if (!aops) return fail(nullptr, LBPF_EUNSUPPORTED, "the adjoint is built for FP64 and FP32 storage only");
        if (p->ny > adjoint_max_ny())
            return fail(nullptr, LBPF_EUNSUPPORTED,
                        "the adjoint needs ny <= " + std::to_string(adjoint_max_ny()) + " (its grid's y extent)");
    }

    lbpf_ctx* ctx = new (std::nothrow) lbpf_ctx();
    if (!ctx) return fail(nullptr, LBPF_ENOMEM, "host allocation failed");
    ctx->p = *p;
    ctx->sp = lattice_units(p);
    ctx->q = p->lattice == LBPF_D3Q19 ? 19 : 9;
    ctx->qh = p->h_lattice ? (p->lattice == LBPF_D3Q19 ? 7 : 5) : ctx->q;
    ctx->kp = make_kparams(p);
    ctx->kpm = march_kparams(ctx->kp, p->lattice);
    ctx->ops = ops;
    ctx->aops = aops;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->real_size = p->precision == LBPF_FP64 ? 8 : 4;
    ctx->store_size = p->precision == LBPF_FP64 ? 8 : (p->precision == LBPF_FP32 ? 4 : 2);
    const size_t N = (size_t)ctx->sp.N;

    auto abort_create = [&](lbpf_status st) {
        std::string m = ctx->err;
        free_all(ctx);
        delete ctx;
        g_thread_error = m;
        return st;
    };
    lbpf_status st;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) { cuda_fail(ctx, e, "cudaGetDevice"); return abort_create(LBPF_ECUDA); }
    for (int i = 0; i < 2; ++i) {
        if ((st = alloc(ctx, &ctx->g[i], ctx->store_size * ctx->q * N, "g populations")) != LBPF_OK) return abort_create(st);
        if ((st = alloc(ctx, &ctx->h[i], ctx->store_size * ctx->qh * N, "h populations")) != LBPF_OK) return abort_create(st);
        if ((st = alloc(ctx, &ctx->phi[i], ctx->real_size * N, "phi field")) != LBPF_OK) return abort_create(st);
        if ((st = alloc(ctx, &ctx->c[i], ctx->real_size * N, "c field")) != LBPF_OK) return abort_create(st);
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    ctx->sm_count = sms;
    const long long want = (ctx->sp.N + kMassThreads - 1) / kMassThreads;
    ctx->mass_blocks = (int)std::min<long long>(want, 4LL * sms);
    if (ctx->mass_blocks < 1) ctx->mass_blocks = 1;
    if ((st = alloc(ctx, (void**)&ctx->partials, sizeof(double) * 3 * ctx->mass_blocks, "mass partials")) != LBPF_OK) return abort_create(st);
    if ((st = alloc(ctx, (void**)&ctx->mass_out, sizeof(double) * 4, "mass result")) != LBPF_OK) return abort_create(st);
    ctx->d_err = reinterpret_cast<int*>(ctx->mass_out + 3);
    e = cudaMemsetAsync(ctx->mass_out, 0, sizeof(double) * 4, ctx->stream);
    if (e != cudaSuccess) { cuda_fail(ctx, e, "mass result"); return abort_create(LBPF_ECUDA); }
    if ((st = ops->prepare(ctx)) != LBPF_OK) return abort_create(st);
    std::memset(&ctx->nomap, 0, sizeof(ctx->nomap));
    {
        // the tensor-map pulls are opt-in (LBPF_TMA=1): bit-identical to the
        // load path, but slower at 256^3 (1.31 against 1.02 ms per step: the
        // copy engine does not deliver the 9 boxes per tile and plane as fast
        // as the threads load the same rows)
        const char* tma = getenv("LBPF_TMA");
        ctx->tma = tma && strcmp(tma, "1") == 0 && ops->setup_tensor_maps(ctx);
    }

    const double* sphi = phi0;
    const double* sc = c0;
    if (!ptr_is_device) {
        if ((st = ensure_staging(ctx)) != LBPF_OK) return abort_create(st);
        e = cudaMemcpyAsync(ctx->staging, phi0, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->staging + N, c0, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) { cuda_fail(ctx, e, "copy of phi0/c0"); return abort_create(LBPF_ECUDA); }
        sphi = ctx->staging;
        sc = ctx->staging + N;
    }
    if (is_f64(ctx)) {
        launch_from_f64<double>(sphi, ctx->phi[0], (long long)N, ctx->stream);
        launch_from_f64<double>(sc, ctx->c[0], (long long)N, ctx->stream);
    } else {
        launch_from_f64<float>(sphi, ctx->phi[0], (long long)N, ctx->stream);
        launch_from_f64<float>(sc, ctx->c[0], (long long)N, ctx->stream);
    }
    ctx->cur = 0;
    ops->launch_init(ctx);
    if ((st = check_launch(ctx, "initialisation kernels")) != LBPF_OK) return abort_create(st);
    if (p->mass_every > 0) {
        // the correction holds the exact population mass of the initial state
        ctx->corr_blocks = ops->c_blocks(ctx);
        ctx->corr_stride = corr_stride_for(ctx->sp.N);
        if ((st = alloc(ctx, (void**)&ctx->corr_partials, sizeof(double) * ctx->corr_blocks, "mass-correction partials")) != LBPF_OK)
            return abort_create(st);
        if ((st = alloc(ctx, (void**)&ctx->corr, sizeof(MassCorr), "mass-correction state")) != LBPF_OK)
            return abort_create(st);
        e = cudaMemsetAsync(ctx->corr, 0, sizeof(MassCorr), ctx->stream);
        if (e != cudaSuccess) { cuda_fail(ctx, e, "mass-correction state"); return abort_create(LBPF_ECUDA); }
        ops->launch_pop_mass(ctx);
        e = cudaMemcpyAsync(&ctx->corr->target, ctx->mass_out, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) { cuda_fail(ctx, e, "mass-correction target"); return abort_create(LBPF_ECUDA); }
        if ((st = check_launch(ctx, "population mass kernels")) != LBPF_OK) return abort_create(st);
    }
    if (aops && (st = record_checkpoint(ctx)) != LBPF_OK) return abort_create(st);
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { cuda_fail(ctx, e, "initialisation"); return abort_create(LBPF_ECUDA); }
    *out = ctx;
    return LBPF_OK;
}

lbpf_status lbpf_step(lbpf_ctx* ctx, int64_t nsteps) {
    if (!ctx) return fail(nullptr, LBPF_EINVAL, "ctx is NULL");
    if (ctx->poisoned) return fail(ctx, LBPF_ESTATE, "context poisoned by an earlier error");
    if (nsteps < 0) return fail(ctx, LBPF_EINVAL, "nsteps < 0");
    return run_steps(ctx, nsteps);
}

lbpf_status lbpf_pull_path(const lbpf_ctx* ctx, int32_t* tensor_maps) {
    if (!ctx || !tensor_maps) return fail(nullptr, LBPF_EINVAL, "ctx or tensor_maps is NULL");
    *tensor_maps = ctx->tma ? 1 : 0;
    return LBPF_OK;
}

lbpf_status lbpf_step_timed(lbpf_ctx* ctx, int64_t nsteps, double* kernel_ms) {
    if (!ctx) return fail(nullptr, LBPF_EINVAL, "ctx is NULL");
    if (ctx->poisoned) return fail(ctx, LBPF_ESTATE, "context poisoned by an earlier error");
    if (nsteps < 0 || !kernel_ms) return fail(ctx, LBPF_EINVAL, "nsteps < 0 or kernel_ms NULL");
    kernel_ms[0] = kernel_ms[1] = kernel_ms[2] = 0.0;
    if (nsteps == 0) return LBPF_OK;
    std::vector<cudaEvent_t> ev(4 * nsteps, nullptr);
    lbpf_status st = LBPF_OK;
    for (auto& x : ev) {
        cudaError_t e = cudaEventCreate(&x);
        if (e != cudaSuccess) { st = cuda_fail(ctx, e, "cudaEventCreate"); break; }
    }
    if (st == LBPF_OK) {
        for (int64_t s = 0; s < nsteps; ++s) {
            const bool corr = ctx->corr && ((ctx->step + 1) % ctx->p.mass_every == 0);
            cudaEventRecord(ev[4 * s], ctx->stream);
            if (ctx->is_batch) ctx->bops->launch_phi(ctx, ctx->cur);
            else ctx->ops->launch_phi(ctx, ctx->cur);
            cudaEventRecord(ev[4 * s + 1], ctx->stream);
            if (ctx->is_batch) ctx->bops->launch_c(ctx, ctx->cur);
            else ctx->ops->launch_c(ctx, ctx->cur, corr ? ctx->corr_partials : nullptr);
            cudaEventRecord(ev[4 * s + 2], ctx->stream);
            if (corr) ctx->ops->launch_corr(ctx, ctx->cur ^ 1);
            cudaEventRecord(ev[4 * s + 3], ctx->stream);
            ctx->cur ^= 1;
            ctx->step += 1;
            if (!ctx->is_batch && ctx->p.checkpoint_every > 0 && ctx->step % ctx->p.checkpoint_every == 0) {
                st = record_checkpoint(ctx);
                if (st != LBPF_OK) break;
            }
        }
        if (st != LBPF_OK) {
            cudaStreamSynchronize(ctx->stream);
            for (auto& x : ev) if (x) cudaEventDestroy(x);
            return st;
        }
        st = check_launch(ctx, "step kernels");
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (st == LBPF_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "step synchronisation");
        for (int64_t s = 0; st == LBPF_OK && s < nsteps; ++s) {
            float a = 0.f, b = 0.f, c = 0.f;
            cudaEventElapsedTime(&a, ev[4 * s], ev[4 * s + 1]);
            cudaEventElapsedTime(&b, ev[4 * s + 1], ev[4 * s + 2]);
            cudaEventElapsedTime(&c, ev[4 * s + 2], ev[4 * s + 3]);
            kernel_ms[0] += a;
            kernel_ms[1] += b;
            kernel_ms[2] += c;
        }
    }
    for (auto& x : ev) if (x) cudaEventDestroy(x);
    return st;
}

lbpf_status lbpf_mass(lbpf_ctx* ctx, double* total_c, double* total_phi) {
    if (!ctx) return fail(nullptr, LBPF_EINVAL, "ctx is NULL");
    if (ctx->poisoned) return fail(ctx, LBPF_ESTATE, "context poisoned by an earlier error");
    if (is_f64(ctx)) launch_mass<double>(ctx); else launch_mass<float>(ctx);
    lbpf_status st = check_launch(ctx, "mass kernels");
    if (st != LBPF_OK) return st;
    double hostv[4];
    LBPF_CUDA(ctx, cudaMemcpyAsync(hostv, ctx->mass_out, sizeof(hostv), cudaMemcpyDeviceToHost, ctx->stream));
    LBPF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int dev_err = 0;
    std::memcpy(&dev_err, &hostv[3], sizeof(int));
    if (dev_err != 0) {
        ctx->poisoned = true;
        return fail(ctx, LBPF_ECUDA, "a tensor copy of the step kernels did not complete (bounded wait ran out)");
    }
    if (total_c) *total_c = hostv[0];
    if (total_phi) *total_phi = hostv[1];
    if (hostv[2] != 0.0 || !std::isfinite(hostv[0]) || !std::isfinite(hostv[1])) {
        ctx->poisoned = true;
        char buf[160];
        snprintf(buf, sizeof(buf), "unstable: %.0f node(s) non-finite or with phi outside [-0.5, 1.5] at step %lld",
                 hostv[2], (long long)ctx->step);
        return fail(ctx, LBPF_EUNSTABLE, buf);
    }
    return LBPF_OK;
}

lbpf_status lbpf_solute_mass(lbpf_ctx* ctx, double* mass, double* target) {
    if (!ctx || !mass) return fail(ctx, LBPF_EINVAL, "NULL argument");
    if (ctx->is_batch) return fail(ctx, LBPF_EUNSUPPORTED, "a batch context: use the lbpf_batch_* calls");
    if (ctx->poisoned) return fail(ctx, LBPF_ESTATE, "context poisoned by an earlier error");
    ctx->ops->launch_pop_mass(ctx);
    lbpf_status st = check_launch(ctx, "population mass kernels");
    if (st != LBPF_OK) return st;
    double hostv[3];
    LBPF_CUDA(ctx, cudaMemcpyAsync(hostv, ctx->mass_out, sizeof(hostv), cudaMemcpyDeviceToHost, ctx->stream));
    double tgt = 0.0;
    if (ctx->corr)
        LBPF_CUDA(ctx, cudaMemcpyAsync(&tgt, &ctx->corr->target, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    LBPF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *mass = hostv[0];
    if (target) *target = ctx->corr ? tgt : std::nan("");
    return LBPF_OK;
}

lbpf_status lbpf_get_fields(lbpf_ctx* ctx, double* phi, double* c, double* mu, int32_t ptr_is_device) {
    if (!ctx) return fail(nullptr, LBPF_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return fail(ctx, LBPF_EUNSUPPORTED, "a batch context: use the lbpf_batch_* calls");
    if (ctx->poisoned) return fail(ctx, LBPF_ESTATE, "context poisoned by an earlier error");
    const size_t N = (size_t)ctx->sp.N;
    double *dphi = phi, *dc = c, *dmu = mu;
    if (!ptr_is_device) {
        lbpf_status st = ensure_staging(ctx);
        if (st != LBPF_OK) return st;
        dphi = phi ? ctx->staging : nullptr;
        dc = c ? ctx->staging + N : nullptr;
        dmu = mu ? ctx->staging + 2 * N : nullptr;
    }
    if (is_f64(ctx)) launch_fields_out<double>(ctx, dphi, dc, dmu);
    else launch_fields_out<float>(ctx, dphi, dc, dmu);
    lbpf_status st = check_launch(ctx, "field export kernel");
    if (st != LBPF_OK) return st;
    if (!ptr_is_device) {
        if (phi) LBPF_CUDA(ctx, cudaMemcpyAsync(phi, dphi, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (c) LBPF_CUDA(ctx, cudaMemcpyAsync(c, dc, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (mu) LBPF_CUDA(ctx, cudaMemcpyAsync(mu, dmu, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
    }
    LBPF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LBPF_OK;
}

lbpf_status lbpf_get_populations(lbpf_ctx* ctx, double* g, double* h, int32_t ptr_is_device) {
    if (!ctx) return fail(nullptr, LBPF_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return fail(ctx, LBPF_EUNSUPPORTED, "a batch context: use the lbpf_batch_* calls");
    if (ctx->poisoned) return fail(ctx, LBPF_ESTATE, "context poisoned by an earlier error");
    const size_t bytes = sizeof(double) * ctx->q * (size_t)ctx->sp.N;
    const size_t hbytes = sizeof(double) * ctx->qh * (size_t)ctx->sp.N;
    double *dg = g, *dh = h, *tmp = nullptr;
    if (!ptr_is_device && (g || h)) {
        lbpf_status st = alloc(ctx, (void**)&tmp, bytes + hbytes, "population export buffer");
        if (st != LBPF_OK) return st;
        dg = g ? tmp : nullptr;
        dh = h ? tmp + ctx->q * (size_t)ctx->sp.N : nullptr;
    }
    ctx->ops->launch_pops_out(ctx, dg, dh);
    lbpf_status st = check_launch(ctx, "population export kernel");
    cudaError_t e = cudaSuccess;
    if (st == LBPF_OK && !ptr_is_device) {
        if (g && e == cudaSuccess) e = cudaMemcpyAsync(g, dg, bytes, cudaMemcpyDeviceToHost, ctx->stream);
        if (h && e == cudaSuccess) e = cudaMemcpyAsync(h, dh, hbytes, cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (tmp) cudaFree(tmp);
    if (st == LBPF_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "population export");
    return st;
}

lbpf_status lbpf_get_step(const lbpf_ctx* ctx, int64_t* step) {
    if (!ctx || !step) return fail(nullptr, LBPF_EINVAL, "NULL argument");
    *step = ctx->step;
    return LBPF_OK;
}

lbpf_status lbpf_destroy(lbpf_ctx* ctx) {
    if (!ctx) return LBPF_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream); else cudaDeviceSynchronize();
    free_all(ctx);
    delete ctx;
    return LBPF_OK;
}

const char* lbpf_last_error(const lbpf_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_thread_error.c_str();
}

lbpf_status lbpf_fp64_fma_rate(void* cuda_stream, double* tflops) {
    if (!tflops) return fail(nullptr, LBPF_EINVAL, "tflops is NULL");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    LBPF_CUDA(nullptr, cudaGetDevice(&dev));
    LBPF_CUDA(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 8 * sms, iters = 1 << 11;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LBPF_CUDA(nullptr, cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(nullptr, e, "cudaEventCreate"); }
    k_fp64_fma<<<blocks, kFmaThreads, 0, s>>>(iters / 16, 1.0);      // warm-up
    cudaEventRecord(e0, s);
    k_fp64_fma<<<blocks, kFmaThreads, 0, s>>>(iters, 1.0);
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "FP64 rate kernel");
    const double flops = 2.0 * kFmaChains * (double)iters * blocks * kFmaThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return LBPF_OK;
}

lbpf_status lbpf_lattice_info(int32_t lattice, int32_t* q, int32_t* e, double* w) {
    if (!q) return fail(nullptr, LBPF_EINVAL, "q is NULL");
    if (lattice == LBPF_D2Q9) {
        *q = 9;
        for (int k = 0; k < 9; ++k) {
            if (e) { e[3 * k] = D2Q9::ex(k); e[3 * k + 1] = D2Q9::ey(k); e[3 * k + 2] = 0; }
            if (w) w[k] = D2Q9::w(k);
        }
    } else if (lattice == LBPF_D3Q19) {
        *q = 19;
        for (int k = 0; k < 19; ++k) {
            if (e) { e[3 * k] = D3Q19::ex(k); e[3 * k + 1] = D3Q19::ey(k); e[3 * k + 2] = D3Q19::ez(k); }
            if (w) w[k] = D3Q19::w(k);
        }
    } else if (lattice == LBPF_D2Q5) {
        *q = 5;
        for (int k = 0; k < 5; ++k) {
            if (e) { e[3 * k] = D2Q5::ex(k); e[3 * k + 1] = D2Q5::ey(k); e[3 * k + 2] = 0; }
            if (w) w[k] = D2Q5::w(k);
        }
    } else if (lattice == LBPF_D3Q7) {
        *q = 7;
        for (int k = 0; k < 7; ++k) {
            if (e) { e[3 * k] = D3Q7::ex(k); e[3 * k + 1] = D3Q7::ey(k); e[3 * k + 2] = D3Q7::ez(k); }
            if (w) w[k] = D3Q7::w(k);
        }
    } else {
        return fail(nullptr, LBPF_EINVAL, "unknown lattice");
    }
    return LBPF_OK;
}

}  // extern "C"
