// The context behind the C ABI (lbpf.h) and the helpers that the library's
// translation units share: lbpf.cu (forward steps, batches, fields, masses) and
// adjoint.cu (checkpoints and the reverse sweep).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "lbpf.h"
#include "step_kernels.cuh"
#include "batch_kernels.cuh"

namespace lbpf_rt {

// Per (lattice, storage) launchers of the forward kernels.  The *_p forms take
// the state buffers explicitly (the adjoint's segment replay); the others use
// the context's ping-pong buffers of parity `cur`.
struct Dispatch {
    lbpf_status (*prepare)(lbpf_ctx*);
    void (*launch_phi)(lbpf_ctx*, int cur);
    void (*launch_c)(lbpf_ctx*, int cur, double* mass_partials);
    void (*launch_init)(lbpf_ctx*);
    void (*launch_pops_out)(lbpf_ctx*, double* g, double* h);
    void (*launch_corr)(lbpf_ctx*, int cur_after);
    void (*launch_pop_mass)(lbpf_ctx*);
    int (*c_blocks)(const lbpf_ctx*);
    void (*launch_phi_p)(lbpf_ctx*, const void* g, void* g_out, const void* phi, const void* c, void* phi_out);
    void (*launch_c_p)(lbpf_ctx*, const void* h, void* h_out, const void* phi, const void* phi_out, const void* c,
                       void* c_out, double* mass_partials);
    void (*launch_corr_p)(lbpf_ctx*, lbpf::MassCorr* mc, void* c, void* h);
    bool (*setup_tensor_maps)(lbpf_ctx*);   // true: the step kernels pull through tensor maps
};
// Launchers of a batch of 2-D instances; the step kernels use the tile shape
// ctx->btile (an index into lbpf::kBatchTiles), which prepare() sets up.
struct BatchDispatch {
    lbpf_status (*prepare)(lbpf_ctx*, int tile);
    void (*launch_phi)(lbpf_ctx*, int cur);
    void (*launch_c)(lbpf_ctx*, int cur);
    void (*launch_init)(lbpf_ctx*, int i);
    void (*fields_out)(lbpf_ctx*, int i, double* phi, double* c, double* mu);
    void (*pop_mass)(lbpf_ctx*, int i);   // exact mass of instance i into mass_out[0]
};
struct AdjDispatch;

// One recorded state: populations g, h, fields phi, c and the mass-correction
// state, carved out of one allocation (each part 256-byte aligned).
struct StateView {
    void* g;
    void* h;
    void* phi;
    void* c;
    lbpf::MassCorr* corr;
};

}  // namespace lbpf_rt

struct lbpf_ctx {
    lbpf_params p;
    lbpf::StepParams sp;
    lbpf::KParams kp;
    lbpf::KParams kpm;             // the marching kernels' view (2-D: rows as z-planes)
    int q = 0;                     // populations of g
    int qh = 0;                    // populations of h (q, or 5 / 7 on the small lattice)
    size_t real_size = 0, store_size = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    void* g[2] = {nullptr, nullptr};
    void* h[2] = {nullptr, nullptr};
    void* phi[2] = {nullptr, nullptr};
    void* c[2] = {nullptr, nullptr};
    double* staging = nullptr;     // 3 N doubles, allocated on first host transfer
    double* partials = nullptr;    // mass reduction scratch
    double* mass_out = nullptr;    // 3 doubles, then the device error flag (see d_err)
    int* d_err = nullptr;          // set by a kernel whose bounded wait ran out (inside mass_out[3])
    // tensor maps of the population buffers (pulls by the copy engine) and an
    // unused one for the kernels that pull with loads
    bool tma = false;
    CUtensorMap gmap[2], hmap[2], nomap;
    double* corr_partials = nullptr;   // one FP64 mass per composition-kernel block
    lbpf::MassCorr* corr = nullptr;    // closed-loop mass correction state (device)
    int corr_blocks = 0;
    long long corr_stride = 1;
    int mass_blocks = 0;
    int sm_count = 0;              // multiprocessors of the context's device
    int zch_phi = 0, zch_c = 0;    // planes per block of the z-marching step kernels
    int cur = 0;
    int64_t step = 0;
    bool poisoned = false;
    std::string err;
    const lbpf_rt::Dispatch* ops = nullptr;
    // a batch of 2-D instances (lbpf_create_batch)
    bool is_batch = false;
    int nb = 0;
    std::vector<lbpf::BatchInst> binst;   // host copy of the instance table
    lbpf::BatchInst* d_binst = nullptr;
    int* d_tile_inst = nullptr;
    int ntiles = 0;
    int ntiles_periodic = 0;              // tiles of the instances without bounce-back axes (listed first)
    int persist_blocks = 0;               // grid of the periodic kernels
    int persist_blocks_walls = 0;         // grid of the walled kernels
    int btile = 0;                        // tile shape in use (index into lbpf::kBatchTiles)
    double btile_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // autotuner: ms per step of each shape
    int tile_capacity = 0;                // entries of d_tile_inst
    const lbpf_rt::BatchDispatch* bops = nullptr;
    // two steps captured as a CUDA graph (replayed by lbpf_step)
    cudaGraphExec_t graph = nullptr;
    bool graph_failed = false;
    // adjoint (checkpoint_every > 0): states at steps 0, k, 2k, ... and, once
    // lbpf_adjoint_step has run, the k + 1 states of one segment and the
    // adjoint work buffers
    size_t state_bytes = 0;
    std::vector<void*> ckpt;
    void* seg = nullptr;
    int64_t seg_slots = 0;
    void* adj = nullptr;
    size_t adj_bytes = 0;
    const lbpf_rt::AdjDispatch* aops = nullptr;
};

namespace lbpf_rt {

lbpf_status fail(lbpf_ctx* ctx, lbpf_status st, const std::string& msg);
lbpf_status cuda_fail(lbpf_ctx* ctx, cudaError_t e, const char* what);
lbpf_status alloc(lbpf_ctx* ctx, void** ptr, size_t bytes, const char* what);
lbpf_status check_launch(lbpf_ctx* ctx, const char* what);
lbpf_status ensure_staging(lbpf_ctx* ctx);

lbpf_status validate(const lbpf_params* p, std::string& why);
lbpf::StepParams lattice_units(const lbpf_params* p);
lbpf::KParams make_kparams(const lbpf_params* p, int sx = 0);
lbpf::KParams march_kparams(const lbpf::KParams& kp, int lattice);
void free_all(lbpf_ctx* ctx);
void set_thread_error(const std::string& msg);

inline bool is_f64(const lbpf_ctx* ctx) { return ctx->p.precision == LBPF_FP64; }

// FP64 caller data -> the compute type, n values
template <typename R>
void launch_from_f64(const double* src, void* dst, long long n, cudaStream_t s) {
    lbpf::k_from_f64<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, (R*)dst, n);
}
// the same into rows of pitch sx (n values in rows of nx)
template <typename R>
void launch_from_f64_rows(const double* src, void* dst, long long n, int nx, int sx, cudaStream_t s) {
    lbpf::k_from_f64_rows<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, (R*)dst, n, nx, sx);
}

// adjoint.cu
const AdjDispatch* pick_adjoint(int lattice, int precision);
int adjoint_max_ny();   // rows its kernels' grid covers (tile rows x 65535 blocks)
size_t state_bytes_for(const lbpf_ctx* ctx);
StateView state_view(const lbpf_ctx* ctx, void* base);
lbpf_status record_checkpoint(lbpf_ctx* ctx);   // the current state, when step % k == 0
void free_adjoint(lbpf_ctx* ctx);

}  // namespace lbpf_rt

#define LBPF_CUDA(ctx, call)                                              \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return lbpf_rt::cuda_fail(ctx, e_, #call); \
    } while (0)
