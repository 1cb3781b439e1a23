// Batched coupled phi-mu LBM step for many 2-D instances of uneven size
// (parameter sweeps, counter term on and off) in one persistent launch per
// kernel phase and boundary kind (periodic instances, instances with a
// bounce-back axis).
//
// Every instance keeps its own SoA layout ([k][y][x] populations, [y][x]
// fields) inside shared concatenated buffers.  The instances are cut into
// tiles of BX columns x ROWS rows; one flat list holds the tiles of all
// instances (the periodic ones first), and a persistent grid (SMs x resident
// blocks) walks each part of it round-robin, so the work is balanced whatever
// the size mix.  A tile is
// processed by the same row-marching code as a single 2-D simulation (the
// D2Q9R view: BX-long row segments, ROWS rows), with its instance's parameters
// read from a device table.  The tile shape is chosen per batch by timing the
// candidates below on the batch itself.
#pragma once

#include "step_kernels.cuh"

namespace lbpf {

struct BatchInst {
    KParams K;             // geometry, coefficients and link offsets of the instance
    KParams Km;            // the same in the row-marching view ([ny][1][nx])
    long long pop_off;     // element offset of the instance's populations
    long long fld_off;     // element offset of the instance's fields
    int tiles_x;           // tiles along x for the current tile shape
    int tile_begin;        // index of the instance's first tile in the flat list
    int walls;             // any bounce-back axis
    int pad;
};

struct BatchTile {
    int bx, rows;
};
// Candidate tile shapes (BX threads per block, resident blocks per SM from the
// thread budget below).  The instance parameters are read from shared memory,
// so the compiler keeps the link offsets and coefficients in registers.  The
// periodic and the walled instances are stepped by separate launches of
// kernels that hold one march each: the periodic kernel, the one the sweeps
// use, is built for 896 threads per SM (72 registers) and ran 3.7% faster on
// the 384-instance sweep than one kernel with both marches at 768 (80
// registers); at 1024 (64 registers) it spills and is slower.  The walled
// kernel keeps 768.
constexpr BatchTile kBatchTiles[] = {{32, 32}, {32, 64}, {64, 32}, {64, 64}, {128, 32}};
constexpr int kNumBatchTiles = sizeof(kBatchTiles) / sizeof(kBatchTiles[0]);
#ifndef LBPF_BATCH_TPSM
#define LBPF_BATCH_TPSM 896
#endif
#ifndef LBPF_BATCH_TPSM_WALLS
#define LBPF_BATCH_TPSM_WALLS 768
#endif
// FP64 arithmetic needs twice the registers: 512 threads per SM (128 registers)
#ifndef LBPF_BATCH_TPSM_F64
#define LBPF_BATCH_TPSM_F64 512
#endif
constexpr int batch_minb(int bx, bool walls, bool f64) {
    return (f64 ? LBPF_BATCH_TPSM_F64 : (walls ? LBPF_BATCH_TPSM_WALLS : LBPF_BATCH_TPSM)) / bx;
}

// Tiles t_begin <= t < t_end of the flat list, all of instances with (WALLS)
// or without bounce-back axes.
template <class SP, bool IS_PHI, int BX, int ROWS, bool WALLS>
__global__ void __launch_bounds__(BX, batch_minb(BX, WALLS, sizeof(typename SP::real) == 8))
k_batch_step(const BatchInst* __restrict__ inst, const int* __restrict__ tile_inst, int t_begin, int t_end,
             const typename SP::store_t* __restrict__ fin, typename SP::store_t* __restrict__ fout,
             const typename SP::real* __restrict__ phi_n, const typename SP::real* __restrict__ phi_np1,
             const typename SP::real* __restrict__ c_n, typename SP::real* __restrict__ moment_out) {
    // the tile's instance parameters live in shared memory while it is marched:
    // read through a global pointer they would be reloaded (they may alias the
    // stores) on every use inside the link loops
    __shared__ KParams sK;
    static_assert(sizeof(KParams) % 4 == 0, "copied as 32-bit words");
    for (int t = t_begin + blockIdx.x; t < t_end; t += gridDim.x) {
        __syncthreads();   // the previous tile's shared memory is free
        const BatchInst& I = inst[tile_inst[t]];
        const int* src = reinterpret_cast<const int*>(&I.Km);
        int* dst = reinterpret_cast<int*>(&sK);
        for (int w = threadIdx.x; w < (int)(sizeof(KParams) / 4); w += blockDim.x) dst[w] = src[w];
        const int lt = t - I.tile_begin;
        const int x0 = (lt % I.tiles_x) * BX;
        const int z0 = (lt / I.tiles_x) * ROWS;
        const long long po = I.pop_off, fo = I.fld_off;
        __syncthreads();
        const typename SP::real* pn1 = phi_np1 ? phi_np1 + fo : nullptr;
        const int z1 = min(z0 + ROWS, sK.P.nz);
        MassAcc<typename SP::real> macc{0, 0};
        march<D2Q9R, SP, 1, IS_PHI, WALLS, BX, int, D2Q9R, false>(sK, fin + po, fout + po, phi_n + fo, pn1, c_n + fo,
                                                                  moment_out + fo, macc, x0, 0, z0, z1);
    }
}

template <class SP, int BX, int ROWS>
constexpr size_t batch_smem(bool is_phi) {
    return march_smem<D2Q9R, SP, 1, BX>(is_phi);
}

}  // namespace lbpf
