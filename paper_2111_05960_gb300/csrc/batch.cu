// Batches of 2-D instances (lbpf_create_batch and the lbpf_batch_* calls): the
// instance table, the flat tile list, the persistent launches and the tile
// autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "context.cuh"

using namespace lbpf;
using namespace lbpf_rt;

namespace {

template <class SP, int T>
struct BatchTileImpl {
    using R = typename SP::real;
    using S = typename SP::store_t;
    static constexpr int BX = kBatchTiles[T].bx, ROWS = kBatchTiles[T].rows;
    static constexpr size_t smem_phi = batch_smem<SP, BX, ROWS>(true);
    static constexpr size_t smem_c = batch_smem<SP, BX, ROWS>(false);

    template <bool IS_PHI, bool W>
    static constexpr auto kern() { return k_batch_step<SP, IS_PHI, BX, ROWS, W>; }

    // resident blocks of one kernel (its shared memory and launch bounds)
    template <bool IS_PHI, bool W>
    static lbpf_status occupancy(lbpf_ctx* ctx, int* blocks) {
        const size_t smem = IS_PHI ? smem_phi : smem_c;
        LBPF_CUDA(ctx, cudaFuncSetAttribute(kern<IS_PHI, W>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        LBPF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern<IS_PHI, W>(), BX, smem));
        return LBPF_OK;
    }
    static lbpf_status prepare(lbpf_ctx* ctx) {
        int sms = 0, o[4] = {0, 0, 0, 0};
        LBPF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        lbpf_status st;
        if ((st = occupancy<true, false>(ctx, &o[0])) != LBPF_OK) return st;
        if ((st = occupancy<false, false>(ctx, &o[1])) != LBPF_OK) return st;
        if ((st = occupancy<true, true>(ctx, &o[2])) != LBPF_OK) return st;
        if ((st = occupancy<false, true>(ctx, &o[3])) != LBPF_OK) return st;
        ctx->persist_blocks = std::max(1, sms * std::max(1, std::min(o[0], o[1])));
        ctx->persist_blocks_walls = std::max(1, sms * std::max(1, std::min(o[2], o[3])));
        return LBPF_OK;
    }
    // the periodic instances' tiles [0, ntiles_periodic), then the walled ones'
    static void launch(lbpf_ctx* ctx, int cur, bool is_phi) {
        const int nxt = cur ^ 1;
        const int n0 = ctx->ntiles_periodic, n1 = ctx->ntiles;
        auto go = [&](auto k, int t0, int t1, int grid) {
            if (t1 <= t0) return;
            const int blocks = std::min(grid, t1 - t0);
            if (is_phi)
                k<<<blocks, BX, smem_phi, ctx->stream>>>(ctx->d_binst, ctx->d_tile_inst, t0, t1, (const S*)ctx->g[cur],
                                                        (S*)ctx->g[nxt], (const R*)ctx->phi[cur], nullptr,
                                                        (const R*)ctx->c[cur], (R*)ctx->phi[nxt]);
            else
                k<<<blocks, BX, smem_c, ctx->stream>>>(ctx->d_binst, ctx->d_tile_inst, t0, t1, (const S*)ctx->h[cur],
                                                      (S*)ctx->h[nxt], (const R*)ctx->phi[cur],
                                                      (const R*)ctx->phi[nxt], (const R*)ctx->c[cur],
                                                      (R*)ctx->c[nxt]);
        };
        if (is_phi) {
            go(kern<true, false>(), 0, n0, ctx->persist_blocks);
            go(kern<true, true>(), n0, n1, ctx->persist_blocks_walls);
        } else {
            go(kern<false, false>(), 0, n0, ctx->persist_blocks);
            go(kern<false, true>(), n0, n1, ctx->persist_blocks_walls);
        }
    }
};

template <class SP>
struct BatchImpl {
    using R = typename SP::real;
    using S = typename SP::store_t;
    static_assert(kNumBatchTiles == 5, "one case per candidate tile shape");

    static lbpf_status prepare(lbpf_ctx* ctx, int t) {
        switch (t) {
            case 0: return BatchTileImpl<SP, 0>::prepare(ctx);
            case 1: return BatchTileImpl<SP, 1>::prepare(ctx);
            case 2: return BatchTileImpl<SP, 2>::prepare(ctx);
            case 3: return BatchTileImpl<SP, 3>::prepare(ctx);
            default: return BatchTileImpl<SP, 4>::prepare(ctx);
        }
    }
    static void launch(lbpf_ctx* ctx, int cur, bool is_phi) {
        switch (ctx->btile) {
            case 0: BatchTileImpl<SP, 0>::launch(ctx, cur, is_phi); break;
            case 1: BatchTileImpl<SP, 1>::launch(ctx, cur, is_phi); break;
            case 2: BatchTileImpl<SP, 2>::launch(ctx, cur, is_phi); break;
            case 3: BatchTileImpl<SP, 3>::launch(ctx, cur, is_phi); break;
            default: BatchTileImpl<SP, 4>::launch(ctx, cur, is_phi); break;
        }
    }
    static void launch_phi(lbpf_ctx* ctx, int cur) { launch(ctx, cur, true); }
    static void launch_c(lbpf_ctx* ctx, int cur) { launch(ctx, cur, false); }
    static void launch_init(lbpf_ctx* ctx, int i) {
        const BatchInst& I = ctx->binst[i];
        const int cur = ctx->cur;
        k_init<D2Q9, SP><<<(unsigned)((I.K.P.N + 255) / 256), 256, 0, ctx->stream>>>(
            I.K, (const R*)ctx->phi[cur] + I.fld_off, (R*)ctx->c[cur] + I.fld_off, (S*)ctx->g[cur] + I.pop_off,
            (S*)ctx->h[cur] + I.pop_off);
    }
    static void fields_out(lbpf_ctx* ctx, int i, double* ophi, double* oc, double* omu) {
        const BatchInst& I = ctx->binst[i];
        const int cur = ctx->cur;
        k_fields_out<R><<<(unsigned)((I.K.P.N + 255) / 256), 256, 0, ctx->stream>>>(
            I.K, (const R*)ctx->phi[cur] + I.fld_off, (const R*)ctx->c[cur] + I.fld_off, ophi, oc, omu);
    }
    static void pop_mass(lbpf_ctx* ctx, int i) {
        const BatchInst& I = ctx->binst[i];
        const int cur = ctx->cur;
        const int blocks = (int)std::min<long long>((I.K.P.N + kMassThreads - 1) / kMassThreads, ctx->mass_blocks);
        k_pop_mass<D2Q9, SP><<<blocks, kMassThreads, 0, ctx->stream>>>(
            I.K, (const R*)ctx->phi[cur] + I.fld_off, (const R*)ctx->c[cur] + I.fld_off,
            (const S*)ctx->h[cur] + I.pop_off, ctx->partials);
        k_mass_final<<<1, kMassThreads, 0, ctx->stream>>>(ctx->partials, blocks, ctx->mass_out);
    }
    static const BatchDispatch* table() {
        static const BatchDispatch d = {prepare, launch_phi, launch_c, launch_init, fields_out, pop_mass};
        return &d;
    }
};

// Row pitch of a batch instance: nx rounded up to 8 elements.
int row_pitch(int nx) { return (nx + 7) & ~7; }

const BatchDispatch* pick_batch(int precision) {
    switch (precision) {
        case LBPF_FP64: return BatchImpl<StoreF64>::table();
        case LBPF_FP32: return BatchImpl<StoreF32>::table();
        case LBPF_FP32_BF16DEV: return BatchImpl<StoreBF16Dev>::table();
        case LBPF_FP32_FP16DEV: return BatchImpl<StoreF16Dev>::table();
    }
    return nullptr;
}

int tiles_of(const lbpf_ctx* ctx, int t) {
    long long tiles = 0;
    for (const BatchInst& I : ctx->binst) {
        const StepParams& P = I.K.P;
        tiles += (long long)((P.nx + kBatchTiles[t].bx - 1) / kBatchTiles[t].bx) *
                 ((P.ny + kBatchTiles[t].rows - 1) / kBatchTiles[t].rows);
    }
    return (int)std::min<long long>(tiles, 1LL << 30);
}

// Cut every instance into tiles of shape t, upload the instance table and the
// flat tile list, and prepare the kernels of that shape.
lbpf_status set_tile(lbpf_ctx* ctx, int t) {
    std::vector<int> tile_inst;
    int tiles = 0;
    try {
        tile_inst.reserve((size_t)tiles_of(ctx, t));
        // the periodic instances first, then those with a bounce-back axis:
        // each group is stepped by its own kernel
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) ctx->ntiles_periodic = tiles;
            for (int i = 0; i < ctx->nb; ++i) {
                BatchInst& I = ctx->binst[i];
                if ((I.walls != 0) != (pass == 1)) continue;
                I.tiles_x = (I.K.P.nx + kBatchTiles[t].bx - 1) / kBatchTiles[t].bx;
                const int ty = (I.K.P.ny + kBatchTiles[t].rows - 1) / kBatchTiles[t].rows;
                I.tile_begin = tiles;
                for (int k = 0; k < I.tiles_x * ty; ++k) tile_inst.push_back(i);
                tiles += I.tiles_x * ty;
            }
        }
    } catch (...) {
        return fail(ctx, LBPF_ENOMEM, "host allocation failed");
    }
    if (tiles > ctx->tile_capacity) return fail(ctx, LBPF_ESTATE, "tile list larger than its buffer");
    LBPF_CUDA(ctx, cudaMemcpyAsync(ctx->d_binst, ctx->binst.data(), sizeof(BatchInst) * ctx->nb,
                                   cudaMemcpyHostToDevice, ctx->stream));
    LBPF_CUDA(ctx, cudaMemcpyAsync(ctx->d_tile_inst, tile_inst.data(), sizeof(int) * tiles, cudaMemcpyHostToDevice,
                                   ctx->stream));
    // the host vector must outlive the copy
    LBPF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->ntiles = tiles;
    ctx->btile = t;
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
    return ctx->bops->prepare(ctx, t);
}

// Time one step (both kernels, from the current state into the other buffers,
// so the state does not change) with every candidate shape and keep the
// fastest.
lbpf_status autotune(lbpf_ctx* ctx) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LBPF_CUDA(ctx, cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(ctx, e, "cudaEventCreate"); }
    lbpf_status st = LBPF_OK;
    int best = 0;
    float best_ms = 1e30f;
    constexpr int reps = 3;
    for (int t = 0; t < kNumBatchTiles && st == LBPF_OK; ++t) {
        if ((st = set_tile(ctx, t)) != LBPF_OK) break;
        ctx->bops->launch_phi(ctx, ctx->cur);      // untimed: module load, caches
        ctx->bops->launch_c(ctx, ctx->cur);
        cudaEventRecord(e0, ctx->stream);
        for (int r = 0; r < reps; ++r) {
            ctx->bops->launch_phi(ctx, ctx->cur);
            ctx->bops->launch_c(ctx, ctx->cur);
        }
        cudaEventRecord(e1, ctx->stream);
        if ((st = check_launch(ctx, "batch kernels")) != LBPF_OK) break;
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { st = cuda_fail(ctx, e, "autotune timing"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ctx->btile_ms[t] = ms / reps;
        if (ms < best_ms) { best_ms = ms; best = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBPF_OK) return st;
    return set_tile(ctx, best);
}

}  // namespace

extern "C" {

lbpf_status lbpf_create_batch(const lbpf_params* p, int32_t n, const double* const* phi0,
                              const double* const* c0, int32_t ptr_is_device, void* cuda_stream, lbpf_ctx** out) {
    if (!out) return fail(nullptr, LBPF_EINVAL, "out pointer is NULL");
    *out = nullptr;
    if (!p || !phi0 || !c0 || n < 1) return fail(nullptr, LBPF_EINVAL, "NULL argument or n < 1");
    for (int i = 0; i < n; ++i) {
        std::string why;
        if (!phi0[i] || !c0[i]) return fail(nullptr, LBPF_EINVAL, "NULL field pointer of instance " + std::to_string(i));
        if (validate(&p[i], why) != LBPF_OK) return fail(nullptr, LBPF_EINVAL, "instance " + std::to_string(i) + ": " + why);
        if (p[i].lattice != LBPF_D2Q9) return fail(nullptr, LBPF_EUNSUPPORTED, "batches hold 2-D D2Q9 instances");
        const long long sb = p[i].precision == LBPF_FP64 ? 8 : (p[i].precision == LBPF_FP32 ? 4 : 2);
        if (9LL * row_pitch(p[i].nx) * p[i].ny * sb >= (1LL << 31))
            return fail(nullptr, LBPF_EINVAL,
                        "instance " + std::to_string(i) +
                            ": 9 ny x (nx rounded up to 8) x bytes per value must stay below 2^31");
        if (p[i].precision != p[0].precision) return fail(nullptr, LBPF_EINVAL, "all instances need one precision");
        if (p[i].mass_every != 0) return fail(nullptr, LBPF_EUNSUPPORTED, "mass correction is not built for batches");
        if (p[i].checkpoint_every != 0) return fail(nullptr, LBPF_EUNSUPPORTED, "the adjoint is not built for batches");
        if (p[i].h_lattice != 0 || p[i].h_eq_alt != 0 || p[i].unequal_eps != 0)
            return fail(nullptr, LBPF_EUNSUPPORTED, "batches keep h on D2Q9 with H_k and equal curvatures");
    }
    const BatchDispatch* bops = pick_batch(p[0].precision);
    if (!bops) return fail(nullptr, LBPF_EUNSUPPORTED, "precision not built");
    lbpf_ctx* ctx = new (std::nothrow) lbpf_ctx();
    if (!ctx) return fail(nullptr, LBPF_ENOMEM, "host allocation failed");
    ctx->is_batch = true;
    ctx->nb = n;
    ctx->bops = bops;
    ctx->p = p[0];
    ctx->q = 9;
    ctx->qh = 9;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->real_size = p[0].precision == LBPF_FP64 ? 8 : 4;
    ctx->store_size = p[0].precision == LBPF_FP64 ? 8 : (p[0].precision == LBPF_FP32 ? 4 : 2);
    auto abort_create = [&](lbpf_status st) {
        std::string m = ctx->err;
        free_all(ctx);
        delete ctx;
        set_thread_error(m);
        return st;
    };
    // instance table: offsets into the concatenated buffers (the tile list
    // follows the tile shape, set below).  Each instance keeps its rows at a
    // pitch of nx rounded up to 8 elements, so that every row and every
    // instance starts on a 32-byte sector in FP32 (the padding is zero in the
    // fields and never read by the pulls).
    long long nodes = 0;          // stored elements per field, padding included
    std::vector<long long> dense_off;
    try {
        ctx->binst.resize(n);
        dense_off.resize(n);
        long long dense = 0;
        for (int i = 0; i < n; ++i) {
            BatchInst& I = ctx->binst[i];
            I.K = make_kparams(&p[i], row_pitch(p[i].nx));
            I.Km = march_kparams(I.K, LBPF_D2Q9);
            I.fld_off = nodes;
            I.pop_off = 9 * nodes;
            I.tiles_x = 1;
            I.tile_begin = 0;
            I.walls = (p[i].bc[0] || p[i].bc[1]) ? 1 : 0;
            I.pad = 0;
            dense_off[i] = dense;
            nodes += I.K.P.NS;
            dense += I.K.P.N;
        }
    } catch (...) {
        return abort_create(fail(ctx, LBPF_ENOMEM, "host allocation failed"));
    }
    for (int t = 0; t < kNumBatchTiles; ++t) ctx->tile_capacity = std::max(ctx->tile_capacity, tiles_of(ctx, t));
    // the whole batch as one field of `nodes` values, for lbpf_mass
    ctx->sp = ctx->binst[0].K.P;
    ctx->sp.N = nodes;
    ctx->sp.nx = (int)std::min<long long>(nodes, 1LL << 30);
    ctx->kp = ctx->binst[0].K;
    lbpf_status st;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) { cuda_fail(ctx, e, "cudaGetDevice"); return abort_create(LBPF_ECUDA); }
    const size_t N = (size_t)nodes;
    for (int i = 0; i < 2; ++i) {
        if ((st = alloc(ctx, &ctx->g[i], ctx->store_size * 9 * N, "g populations")) != LBPF_OK) return abort_create(st);
        if ((st = alloc(ctx, &ctx->h[i], ctx->store_size * 9 * N, "h populations")) != LBPF_OK) return abort_create(st);
        if ((st = alloc(ctx, &ctx->phi[i], ctx->real_size * N, "phi field")) != LBPF_OK) return abort_create(st);
        if ((st = alloc(ctx, &ctx->c[i], ctx->real_size * N, "c field")) != LBPF_OK) return abort_create(st);
    }
    if ((st = alloc(ctx, (void**)&ctx->d_binst, sizeof(BatchInst) * n, "instance table")) != LBPF_OK) return abort_create(st);
    if ((st = alloc(ctx, (void**)&ctx->d_tile_inst, sizeof(int) * ctx->tile_capacity, "tile list")) != LBPF_OK)
        return abort_create(st);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    ctx->mass_blocks = (int)std::max<long long>(1, std::min<long long>((nodes + kMassThreads - 1) / kMassThreads, 4LL * sms));
    if ((st = alloc(ctx, (void**)&ctx->partials, sizeof(double) * 3 * ctx->mass_blocks, "mass partials")) != LBPF_OK) return abort_create(st);
    if ((st = alloc(ctx, (void**)&ctx->mass_out, sizeof(double) * 3, "mass result")) != LBPF_OK) return abort_create(st);
    // the row padding of both field sets stays zero (lbpf_mass sums every element)
    for (int i = 0; i < 2; ++i) {
        e = cudaMemsetAsync(ctx->phi[i], 0, ctx->real_size * N, ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->c[i], 0, ctx->real_size * N, ctx->stream);
        if (e != cudaSuccess) { cuda_fail(ctx, e, "clearing the fields"); return abort_create(LBPF_ECUDA); }
    }

    // fields: per instance into the staging buffer (host) or straight from the caller (device)
    if (!ptr_is_device) {
        if ((st = ensure_staging(ctx)) != LBPF_OK) return abort_create(st);
    }
    for (int i = 0; i < n; ++i) {
        const BatchInst& I = ctx->binst[i];
        const size_t Ni = (size_t)I.K.P.N;
        const int nx = I.K.P.nx, sx = I.K.P.sx;
        const double* sphi = phi0[i];
        const double* sc = c0[i];
        if (!ptr_is_device) {
            e = cudaMemcpyAsync(ctx->staging + dense_off[i], phi0[i], sizeof(double) * Ni, cudaMemcpyHostToDevice,
                                ctx->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(ctx->staging + N + dense_off[i], c0[i], sizeof(double) * Ni,
                                    cudaMemcpyHostToDevice, ctx->stream);
            if (e != cudaSuccess) { cuda_fail(ctx, e, "copy of phi0/c0"); return abort_create(LBPF_ECUDA); }
            sphi = ctx->staging + dense_off[i];
            sc = ctx->staging + N + dense_off[i];
        }
        if (is_f64(ctx)) {
            launch_from_f64_rows<double>(sphi, (double*)ctx->phi[0] + I.fld_off, (long long)Ni, nx, sx, ctx->stream);
            launch_from_f64_rows<double>(sc, (double*)ctx->c[0] + I.fld_off, (long long)Ni, nx, sx, ctx->stream);
        } else {
            launch_from_f64_rows<float>(sphi, (float*)ctx->phi[0] + I.fld_off, (long long)Ni, nx, sx, ctx->stream);
            launch_from_f64_rows<float>(sc, (float*)ctx->c[0] + I.fld_off, (long long)Ni, nx, sx, ctx->stream);
        }
    }
    ctx->cur = 0;
    for (int i = 0; i < n; ++i) bops->launch_init(ctx, i);
    if ((st = check_launch(ctx, "initialisation kernels")) != LBPF_OK) return abort_create(st);
    if ((st = autotune(ctx)) != LBPF_OK) return abort_create(st);
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { cuda_fail(ctx, e, "initialisation"); return abort_create(LBPF_ECUDA); }
    *out = ctx;
    return LBPF_OK;
}

lbpf_status lbpf_batch_get_fields(lbpf_ctx* ctx, int32_t i, double* phi, double* c, double* mu, int32_t ptr_is_device) {
    if (!ctx) return fail(nullptr, LBPF_EINVAL, "ctx is NULL");
    if (!ctx->is_batch) return fail(ctx, LBPF_EINVAL, "not a batch context");
    if (ctx->poisoned) return fail(ctx, LBPF_ESTATE, "context poisoned by an earlier error");
    if (i < 0 || i >= ctx->nb) return fail(ctx, LBPF_EINVAL, "instance index out of range");
    const size_t Ni = (size_t)ctx->binst[i].K.P.N;
    double *dphi = phi, *dc = c, *dmu = mu;
    if (!ptr_is_device) {
        lbpf_status st = ensure_staging(ctx);
        if (st != LBPF_OK) return st;
        dphi = phi ? ctx->staging : nullptr;
        dc = c ? ctx->staging + Ni : nullptr;
        dmu = mu ? ctx->staging + 2 * Ni : nullptr;
    }
    ctx->bops->fields_out(ctx, i, dphi, dc, dmu);
    lbpf_status st = check_launch(ctx, "field export kernel");
    if (st != LBPF_OK) return st;
    if (!ptr_is_device) {
        if (phi) LBPF_CUDA(ctx, cudaMemcpyAsync(phi, dphi, sizeof(double) * Ni, cudaMemcpyDeviceToHost, ctx->stream));
        if (c) LBPF_CUDA(ctx, cudaMemcpyAsync(c, dc, sizeof(double) * Ni, cudaMemcpyDeviceToHost, ctx->stream));
        if (mu) LBPF_CUDA(ctx, cudaMemcpyAsync(mu, dmu, sizeof(double) * Ni, cudaMemcpyDeviceToHost, ctx->stream));
    }
    LBPF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LBPF_OK;
}

lbpf_status lbpf_batch_solute_mass(lbpf_ctx* ctx, double* masses) {
    if (!ctx || !masses) return fail(ctx, LBPF_EINVAL, "NULL argument");
    if (!ctx->is_batch) return fail(ctx, LBPF_EINVAL, "not a batch context");
    if (ctx->poisoned) return fail(ctx, LBPF_ESTATE, "context poisoned by an earlier error");
    for (int i = 0; i < ctx->nb; ++i) {
        ctx->bops->pop_mass(ctx, i);
        lbpf_status st = check_launch(ctx, "population mass kernels");
        if (st != LBPF_OK) return st;
        LBPF_CUDA(ctx, cudaMemcpyAsync(&masses[i], ctx->mass_out, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    LBPF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LBPF_OK;
}

lbpf_status lbpf_batch_tile(const lbpf_ctx* ctx, int32_t* tile_x, int32_t* tile_rows, double* ms_per_step) {
    if (!ctx || !tile_x || !tile_rows) return fail(nullptr, LBPF_EINVAL, "NULL argument");
    if (!ctx->is_batch) return fail(nullptr, LBPF_EINVAL, "not a batch context");
    *tile_x = kBatchTiles[ctx->btile].bx;
    *tile_rows = kBatchTiles[ctx->btile].rows;
    if (ms_per_step)
        for (int t = 0; t < kNumBatchTiles; ++t) ms_per_step[t] = ctx->btile_ms[t];
    return LBPF_OK;
}

lbpf_status lbpf_batch_set_tile(lbpf_ctx* ctx, int32_t tile_x, int32_t tile_rows) {
    if (!ctx) return fail(nullptr, LBPF_EINVAL, "ctx is NULL");
    if (!ctx->is_batch) return fail(ctx, LBPF_EINVAL, "not a batch context");
    if (ctx->poisoned) return fail(ctx, LBPF_ESTATE, "context poisoned by an earlier error");
    for (int t = 0; t < kNumBatchTiles; ++t)
        if (kBatchTiles[t].bx == tile_x && kBatchTiles[t].rows == tile_rows) return set_tile(ctx, t);
    return fail(ctx, LBPF_EINVAL, "not one of the built tile shapes");
}

}  // extern "C"
