// Batched coupled phi-mu LBM step for many 2-D instances of uneven size
// (parameter sweeps, counter term on and off) in one persistent launch per
// kernel phase.
//
// Every instance keeps its own SoA layout ([k][y][x] populations, [y][x]
// fields) inside shared concatenated buffers.  The instances are cut into
// 32 x 8 tiles; one flat list holds the tiles of all instances, and a
// persistent grid (SMs x resident blocks) walks it round-robin, so the work is
// balanced whatever the size mix.  A tile is processed by the same z-march code
// as a single simulation (one plane), with its instance's parameters read from
// a device table.
#pragma once

#include "step_kernels.cuh"

namespace lbpf {

struct BatchInst {
    KParams K;             // geometry, coefficients and link offsets of the instance
    long long pop_off;     // element offset of the instance's populations
    long long fld_off;     // element offset of the instance's fields
    int tiles_x;           // 32-wide tiles along x
    int tile_begin;        // index of the instance's first tile in the flat list
    int walls;             // any bounce-back axis
    int pad;
};

constexpr int kBatchBY = 8;

template <class SP, bool IS_PHI>
__global__ void __launch_bounds__(32 * kBatchBY, 2)
k_batch_step(const BatchInst* __restrict__ inst, const int* __restrict__ tile_inst, int ntiles,
             const typename SP::store_t* __restrict__ fin, typename SP::store_t* __restrict__ fout,
             const typename SP::real* __restrict__ phi_n, const typename SP::real* __restrict__ phi_np1,
             const typename SP::real* __restrict__ c_n, typename SP::real* __restrict__ moment_out) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads();   // the previous tile's shared memory is free
        const BatchInst& I = inst[tile_inst[t]];
        const int lt = t - I.tile_begin;
        const int x0 = (lt % I.tiles_x) * 32;
        const int y0 = (lt / I.tiles_x) * kBatchBY;
        const long long po = I.pop_off, fo = I.fld_off;
        const typename SP::real* pn1 = phi_np1 ? phi_np1 + fo : nullptr;
        if (I.walls)
            march<D2Q9, SP, kBatchBY, 1, IS_PHI, true>(I.K, fin + po, fout + po, phi_n + fo, pn1, c_n + fo,
                                                       moment_out + fo, nullptr, x0, y0, 0, 0);
        else
            march<D2Q9, SP, kBatchBY, 1, IS_PHI, false>(I.K, fin + po, fout + po, phi_n + fo, pn1, c_n + fo,
                                                        moment_out + fo, nullptr, x0, y0, 0, 0);
    }
}

template <class SP>
constexpr size_t batch_smem(bool is_phi) {
    return march_smem<D2Q9, SP, kBatchBY, 1>(is_phi);
}

}  // namespace lbpf
