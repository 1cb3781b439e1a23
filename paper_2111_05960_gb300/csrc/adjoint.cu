// Discrete adjoint of the trajectory since creation (lbpf_adjoint_step):
// checkpoints every k steps, replay of one segment into per-step storage, and
// the reverse sweep of the adjoint kernels over it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "context.cuh"
#include "adjoint_kernels.cuh"

using namespace lbpf;

namespace lbpf_rt {

namespace {

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Views into ctx->adj: ping-pong adjoints of the state, the per-node work
// area, the per-block parameter partials, their sum and the replayed
// mass-correction state.
struct AdjBufs {
    void* gb[2];
    void* hb[2];
    void* phib[2];
    void* cb[2];
    void* work;          // 7 N values (AdjWork)
    double* blockacc;    // kAdjParams x nblk
    double* pout;        // kAdjParams
    MassCorr* corr;
    int nblk;
};

// 32 x 8 tiles of each z-plane; a block takes p planes (z, z + gridDim.z,
// ...), so that its setup and its flush of the parameter adjoints are shared:
// the largest p of 8, 4, 2 that still leaves 4 waves of resident blocks (on
// GB300 the 128^3 reverse kernels went from 0.32 to 0.29 ms per step with 4
// planes per block; 8, at 2.2 waves, was back at 0.32).  Planes beyond the
// grid's z extent loop.
dim3 adj_grid(const lbpf_ctx* ctx) {
    const StepParams& P = ctx->sp;
    const long long tiles = (long long)((P.nx + kAdjBX - 1) / kAdjBX) * ((P.ny + kAdjBY - 1) / kAdjBY);
    const long long resident =
        (long long)std::max(1, ctx->sm_count) * (ctx->real_size == 8 ? LBPF_ADJ_MINB_F64 : LBPF_ADJ_MINB_F32);
    int planes = 1;
    for (int p : {8, 4, 2})
        if (tiles * ((P.nz + p - 1) / p) >= 4 * resident) {
            planes = p;
            break;
        }
    const int zb = (P.nz + planes - 1) / planes;
    return dim3((P.nx + kAdjBX - 1) / kAdjBX, (P.ny + kAdjBY - 1) / kAdjBY, std::min(zb, 32768));
}

}  // namespace

int adjoint_max_ny() { return kAdjBY * 65535; }

namespace {

int adj_blocks(const lbpf_ctx* ctx) {
    const dim3 g = adj_grid(ctx);
    return (int)(g.x * g.y * g.z);
}

size_t adj_layout(const lbpf_ctx* ctx, void* base, AdjBufs* a) {
    const size_t N = (size_t)ctx->sp.N, rs = ctx->real_size;
    const int nblk = adj_blocks(ctx);
    char* p = (char*)base;
    size_t off = 0;
    auto take = [&](size_t bytes) { void* r = p ? p + off : nullptr; off += align256(bytes); return r; };
    AdjBufs v;
    for (int i = 0; i < 2; ++i) v.gb[i] = take(rs * ctx->q * N);
    for (int i = 0; i < 2; ++i) v.hb[i] = take(rs * ctx->q * N);
    for (int i = 0; i < 2; ++i) v.phib[i] = take(rs * N);
    for (int i = 0; i < 2; ++i) v.cb[i] = take(rs * N);
    v.work = take(rs * 7 * N);
    v.blockacc = (double*)take(sizeof(double) * kAdjParams * nblk);
    v.pout = (double*)take(sizeof(double) * kAdjParams);
    v.corr = (MassCorr*)take(sizeof(MassCorr));
    v.nblk = nblk;
    if (a) *a = v;
    return off;
}

}  // namespace

struct AdjDispatch {
    void (*step)(lbpf_ctx*, const StateView& s, const void* phi1, const AdjBufs& a, int cur);
    void (*init)(lbpf_ctx*, const StateView& s, const AdjBufs& a, int cur);
    void (*from_f64)(lbpf_ctx*, const double* src, void* dst);
    void (*to_f64)(lbpf_ctx*, const void* src, double* dst);
};

namespace {

template <class L, typename R>
struct AdjImpl {
    static AdjWork<R> work(const lbpf_ctx* ctx, void* base) {
        const long long N = ctx->sp.N;
        R* w = (R*)base;
        AdjWork<R> T;
        T.phi = w;
        T.c = w + N;
        T.dphi = w + 2 * N;
        T.pt = w + 3 * N;
        T.grad = w + 4 * N;
        return T;
    }
    // adjoint of the step from state s (phi1 = phi of the next state)
    static void step(lbpf_ctx* ctx, const StateView& s, const void* phi1, const AdjBufs& a, int cur) {
        const int nxt = cur ^ 1;
        const AdjWork<R> T = work(ctx, a.work);
        const dim3 grid = adj_grid(ctx), block(kAdjBX, kAdjBY);
        const AdjCoef<R> C = make_adj_coef<R>(ctx->sp);
        const StepParams& P = ctx->sp;
        const bool walls = P.bc[0] || P.bc[1] || (L::D == 3 && P.bc[2]);
        auto kh = walls ? k_adj_h<L, R, true> : k_adj_h<L, R, false>;
        auto kg = walls ? k_adj_g<L, R, true> : k_adj_g<L, R, false>;
        kh<<<grid, block, 0, ctx->stream>>>(
            ctx->sp, C, (const R*)s.h, (const R*)s.phi, (const R*)s.c, (const R*)phi1, (const R*)a.hb[cur],
            (const R*)a.cb[cur], (const R*)a.phib[cur], (R*)a.hb[nxt], T, a.blockacc, a.nblk);
        kg<<<grid, block, 0, ctx->stream>>>(
            ctx->sp, C, (const R*)s.g, (const R*)s.phi, (const R*)s.c, (const R*)a.gb[cur], (R*)a.gb[nxt], T,
            (R*)a.phib[nxt], (R*)a.cb[nxt], a.blockacc, a.nblk);
        k_adj_finish<L, R><<<grid, block, 0, ctx->stream>>>(ctx->sp, T.grad, (R*)a.phib[nxt]);
    }
    // adjoint of the initialisation from the initial fields of state s
    static void init(lbpf_ctx* ctx, const StateView& s, const AdjBufs& a, int cur) {
        const int nxt = cur ^ 1;
        const AdjWork<R> T = work(ctx, a.work);
        const dim3 grid = adj_grid(ctx), block(kAdjBX, kAdjBY);
        const AdjCoef<R> C = make_adj_coef<R>(ctx->sp);
        k_adj_init<L, R><<<grid, block, 0, ctx->stream>>>(
            ctx->sp, C, (const R*)s.phi, (const R*)s.c, (const R*)a.gb[cur], (const R*)a.hb[cur],
            (const R*)a.phib[cur], (const R*)a.cb[cur], T.grad, (R*)a.phib[nxt], (R*)a.cb[nxt], a.blockacc,
            a.nblk);
        k_adj_finish<L, R><<<grid, block, 0, ctx->stream>>>(ctx->sp, T.grad, (R*)a.phib[nxt]);
    }
    static void from_f64(lbpf_ctx* ctx, const double* src, void* dst) {
        const long long N = ctx->sp.N;
        k_from_f64<R><<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(src, (R*)dst, N);
    }
    static void to_f64(lbpf_ctx* ctx, const void* src, double* dst) {
        const long long N = ctx->sp.N;
        k_adj_to_f64<R><<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>((const R*)src, dst, N);
    }
    static const AdjDispatch* table() {
        static const AdjDispatch d = {step, init, from_f64, to_f64};
        return &d;
    }
};

cudaError_t copy_state(const lbpf_ctx* ctx, const StateView& from, const StateView& to) {
    const size_t N = (size_t)ctx->sp.N;
    const size_t pop = ctx->store_size * ctx->q * N, fld = ctx->real_size * N;
    cudaError_t e = cudaMemcpyAsync(to.g, from.g, pop, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(to.h, from.h, pop, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(to.phi, from.phi, fld, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(to.c, from.c, fld, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && from.corr && to.corr)
        e = cudaMemcpyAsync(to.corr, from.corr, sizeof(MassCorr), cudaMemcpyDeviceToDevice, ctx->stream);
    return e;
}

// Forward step n of the replay, from state a into state b, with the mass
// correction (on the replayed correction state mc) where the forward run had it.
void replay_step(lbpf_ctx* ctx, const StateView& a, const StateView& b, int64_t n, MassCorr* mc) {
    const bool corr = ctx->corr && ((n + 1) % ctx->p.mass_every == 0);
    ctx->ops->launch_phi_p(ctx, a.g, b.g, a.phi, a.c, b.phi);
    ctx->ops->launch_c_p(ctx, a.h, b.h, a.phi, b.phi, a.c, b.c, corr ? ctx->corr_partials : nullptr);
    if (corr) ctx->ops->launch_corr_p(ctx, mc, b.c, b.h);
}

}  // namespace

const AdjDispatch* pick_adjoint(int lattice, int precision) {
    if (lattice == LBPF_D2Q9) {
        if (precision == LBPF_FP64) return AdjImpl<D2Q9, double>::table();
        if (precision == LBPF_FP32) return AdjImpl<D2Q9, float>::table();
    } else if (lattice == LBPF_D3Q19) {
        if (precision == LBPF_FP64) return AdjImpl<D3Q19, double>::table();
        if (precision == LBPF_FP32) return AdjImpl<D3Q19, float>::table();
    }
    return nullptr;
}

size_t state_bytes_for(const lbpf_ctx* ctx) {
    const size_t N = (size_t)ctx->sp.N;
    return 2 * align256(ctx->store_size * ctx->q * N) + 2 * align256(ctx->real_size * N) + align256(sizeof(MassCorr));
}

StateView state_view(const lbpf_ctx* ctx, void* base) {
    const size_t N = (size_t)ctx->sp.N;
    const size_t pop = align256(ctx->store_size * ctx->q * N), fld = align256(ctx->real_size * N);
    char* p = (char*)base;
    StateView v;
    v.g = p;
    v.h = p + pop;
    v.phi = p + 2 * pop;
    v.c = p + 2 * pop + fld;
    v.corr = (MassCorr*)(p + 2 * pop + 2 * fld);
    return v;
}

lbpf_status record_checkpoint(lbpf_ctx* ctx) {
    const int64_t k = ctx->p.checkpoint_every;
    if (k <= 0 || ctx->step % k != 0) return LBPF_OK;
    const size_t m = (size_t)(ctx->step / k);
    if (!ctx->state_bytes) ctx->state_bytes = state_bytes_for(ctx);
    while (ctx->ckpt.size() <= m) {
        void* b = nullptr;
        lbpf_status st = alloc(ctx, &b, ctx->state_bytes, "adjoint checkpoint");
        if (st != LBPF_OK) return st;
        ctx->ckpt.push_back(b);
    }
    StateView cur;
    cur.g = ctx->g[ctx->cur];
    cur.h = ctx->h[ctx->cur];
    cur.phi = ctx->phi[ctx->cur];
    cur.c = ctx->c[ctx->cur];
    cur.corr = ctx->corr;
    cudaError_t e = copy_state(ctx, cur, state_view(ctx, ctx->ckpt[m]));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint checkpoint copy");
    return LBPF_OK;
}

void free_adjoint(lbpf_ctx* ctx) {
    for (void* b : ctx->ckpt) cudaFree(b);
    ctx->ckpt.clear();
    cudaFree(ctx->seg);
    cudaFree(ctx->adj);
    ctx->seg = nullptr;
    ctx->adj = nullptr;
    ctx->seg_slots = 0;
    ctx->adj_bytes = 0;
}

}  // namespace lbpf_rt

using namespace lbpf_rt;

extern "C" lbpf_status lbpf_adjoint_step(lbpf_ctx* ctx, const double* dL_dphi, const double* dL_dc, double* dL_dphi0,
                                         double* dL_dc0, int32_t ptr_is_device, double* dL_dparams) {
    if (!ctx) return fail(nullptr, LBPF_EINVAL, "ctx is NULL");
    if (!dL_dparams) return fail(ctx, LBPF_EINVAL, "dL_dparams is NULL");
    if (ctx->is_batch) return fail(ctx, LBPF_EUNSUPPORTED, "the adjoint is not built for batches");
    if (ctx->poisoned) return fail(ctx, LBPF_ESTATE, "context poisoned by an earlier error");
    if (ctx->p.checkpoint_every <= 0 || !ctx->aops)
        return fail(ctx, LBPF_EUNSUPPORTED, "create the context with checkpoint_every > 0 to record the trajectory");
    const int64_t T = ctx->step, K = ctx->p.checkpoint_every;
    if ((int64_t)ctx->ckpt.size() < T / K + 1) return fail(ctx, LBPF_ESTATE, "a checkpoint of the trajectory is missing");
    const size_t N = (size_t)ctx->sp.N;
    const AdjDispatch* A = ctx->aops;
    lbpf_status st;

    // buffers: the segment's states (kept between calls) and the adjoint work area
    const int64_t slots = std::min<int64_t>(K, std::max<int64_t>(T, 1)) + 1;
    if (ctx->seg_slots < slots) {
        cudaFree(ctx->seg);
        ctx->seg = nullptr;
        ctx->seg_slots = 0;
        if ((st = alloc(ctx, &ctx->seg, ctx->state_bytes * (size_t)slots, "adjoint segment states")) != LBPF_OK) return st;
        ctx->seg_slots = slots;
    }
    if (!ctx->adj) {
        ctx->adj_bytes = adj_layout(ctx, nullptr, nullptr);
        if ((st = alloc(ctx, &ctx->adj, ctx->adj_bytes, "adjoint work buffers")) != LBPF_OK) return st;
    }
    AdjBufs a;
    adj_layout(ctx, ctx->adj, &a);
    auto slot = [&](int64_t i) { return state_view(ctx, (char*)ctx->seg + ctx->state_bytes * (size_t)i); };

    // seeds
    const size_t qbytes = ctx->real_size * ctx->q * N, fbytes = ctx->real_size * N;
    LBPF_CUDA(ctx, cudaMemsetAsync(a.gb[0], 0, qbytes, ctx->stream));
    LBPF_CUDA(ctx, cudaMemsetAsync(a.hb[0], 0, qbytes, ctx->stream));
    LBPF_CUDA(ctx, cudaMemsetAsync(a.blockacc, 0, sizeof(double) * kAdjParams * a.nblk, ctx->stream));
    const double* seeds[2] = {dL_dphi, dL_dc};
    void* dst[2] = {a.phib[0], a.cb[0]};
    if (!ptr_is_device && (dL_dphi || dL_dc))
        if ((st = ensure_staging(ctx)) != LBPF_OK) return st;
    for (int i = 0; i < 2; ++i) {
        if (!seeds[i]) {
            LBPF_CUDA(ctx, cudaMemsetAsync(dst[i], 0, fbytes, ctx->stream));
            continue;
        }
        const double* src = seeds[i];
        if (!ptr_is_device) {
            LBPF_CUDA(ctx, cudaMemcpyAsync(ctx->staging + i * N, seeds[i], sizeof(double) * N, cudaMemcpyHostToDevice,
                                           ctx->stream));
            src = ctx->staging + i * N;
        }
        A->from_f64(ctx, src, dst[i]);
    }

    // segments in reverse: restore, replay forward, sweep back
    int cur = 0;
    for (int64_t S = T > 0 ? ((T - 1) / K) * K : -1; S >= 0; S -= K) {
        const int64_t E = std::min(S + K, T);
        StateView s0 = slot(0);
        if (!ctx->corr) s0.corr = nullptr;
        cudaError_t e = copy_state(ctx, state_view(ctx, ctx->ckpt[(size_t)(S / K)]), s0);
        if (e == cudaSuccess && ctx->corr)
            e = cudaMemcpyAsync(a.corr, s0.corr, sizeof(MassCorr), cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "checkpoint restore");
        for (int64_t n = S; n < E; ++n) replay_step(ctx, slot(n - S), slot(n - S + 1), n, a.corr);
        for (int64_t n = E - 1; n >= S; --n) {
            A->step(ctx, slot(n - S), slot(n - S + 1).phi, a, cur);
            cur ^= 1;
        }
        if ((st = check_launch(ctx, "adjoint kernels")) != LBPF_OK) return st;
    }
    if (T == 0) {
        StateView s0 = slot(0);
        s0.corr = nullptr;
        StateView c0 = state_view(ctx, ctx->ckpt[0]);
        c0.corr = nullptr;
        cudaError_t e = copy_state(ctx, c0, s0);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "checkpoint restore");
    }
    A->init(ctx, slot(0), a, cur);
    cur ^= 1;
    k_adj_param_final<<<1, kAdjThreads, 0, ctx->stream>>>(a.blockacc, a.nblk, a.pout);
    if ((st = check_launch(ctx, "adjoint kernels")) != LBPF_OK) return st;

    // outputs
    double* outs[2] = {dL_dphi0, dL_dc0};
    const void* srcs[2] = {a.phib[cur], a.cb[cur]};
    if (!ptr_is_device && (dL_dphi0 || dL_dc0))
        if ((st = ensure_staging(ctx)) != LBPF_OK) return st;
    for (int i = 0; i < 2; ++i) {
        if (!outs[i]) continue;
        double* d = ptr_is_device ? outs[i] : ctx->staging + i * N;
        A->to_f64(ctx, srcs[i], d);
        if (!ptr_is_device)
            LBPF_CUDA(ctx, cudaMemcpyAsync(outs[i], d, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
    }
    if ((st = check_launch(ctx, "adjoint export kernels")) != LBPF_OK) return st;
    double pv[kAdjParams];
    LBPF_CUDA(ctx, cudaMemcpyAsync(pv, a.pout, sizeof(pv), cudaMemcpyDeviceToHost, ctx->stream));
    LBPF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));

    // lattice units -> the units of lbpf_params; the automatic a = (1 - D_s/D_l)/4
    const lbpf_params& p = ctx->p;
    const double dfac = p.dt / (p.dx * p.dx);
    double out[kAdjParams];
    out[kPDl] = pv[kPDl] * dfac;
    out[kPTauG] = pv[kPTauG];
    out[kPTauH] = pv[kPTauH];
    out[kPLam] = pv[kPLam];
    out[kPA] = p.anti_trapping ? pv[kPA] : 0.0;
    out[kPDs] = pv[kPDs] * dfac;
    if (p.anti_trapping && p.a_at < 0) {
        out[kPDl] += out[kPA] * 0.25 * p.D_s / (p.D_l * p.D_l);
        out[kPDs] -= out[kPA] * 0.25 / p.D_l;
    }
    memcpy(dL_dparams, out, sizeof(out));
    return LBPF_OK;
}
