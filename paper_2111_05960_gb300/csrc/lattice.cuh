// Lattice tables of the coupled phi-mu LBM step, as compile-time functions so
// that fully unrolled loops over k fold every e_k and w_k into constants.
//
// D2Q9 follows the ordering of Sec. 3.1 (LBM notations): e0 = 0,
// e1..e4 = (1,0),(0,1),(-1,0),(0,-1), e5..e8 = (1,1),(-1,1),(-1,-1),(1,-1),
// w = 4/9, 1/9, 1/36.  D3Q19 (named among the lattices of the paper's code in
// Sec. 3.1) is used for 3-D: rest (1/3), six face links (1/18), twelve edge
// links (1/36), with opposite directions stored next to each other.
#pragma once

namespace lbpf {

struct D2Q9 {
    static constexpr int D = 2;
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int ex(int k) {
        return (k == 1 || k == 5 || k == 8) ? 1 : ((k == 3 || k == 6 || k == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int k) {
        return (k == 2 || k == 5 || k == 6) ? 1 : ((k == 4 || k == 7 || k == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr double w(int k) {
        return k == 0 ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int opp(int k) {
        return k == 0 ? 0 : (k <= 4 ? ((k + 1) % 4) + 1 : ((k - 5 + 2) % 4) + 5);
    }
};

struct D3Q19 {
    static constexpr int D = 3;
    static constexpr int Q = 19;
    // k: 1..6 faces +x -x +y -y +z -z; 7..18 edges
    // (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1)
    // (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
    __host__ __device__ static constexpr int ex(int k) {
        return (k == 1 || k == 7 || k == 9 || k == 11 || k == 13) ? 1
             : ((k == 2 || k == 8 || k == 10 || k == 12 || k == 14) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int k) {
        return (k == 3 || k == 7 || k == 10 || k == 15 || k == 17) ? 1
             : ((k == 4 || k == 8 || k == 9 || k == 16 || k == 18) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ez(int k) {
        return (k == 5 || k == 11 || k == 14 || k == 15 || k == 18) ? 1
             : ((k == 6 || k == 12 || k == 13 || k == 16 || k == 17) ? -1 : 0);
    }
    __host__ __device__ static constexpr double w(int k) {
        return k == 0 ? 1.0 / 3.0 : (k <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int opp(int k) {
        return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1);
    }
};

}  // namespace lbpf
