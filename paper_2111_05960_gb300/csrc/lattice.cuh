// Lattice tables of the coupled phi-mu LBM step, as compile-time functions so
// that fully unrolled loops over k fold every e_k and w_k into constants.
//
// The kernels apply the weights as w_k = m_k / 36: a per-node quantity X is
// divided by 36 once (correctly rounded) and the moving links multiply it by
// m_k in {1, 2, 4}, which is exact.  With FP32 constants fl(1/18), fl(1/36),
// fl(1/3) the weights do not sum to one (the D3Q19 moving weights exceed
// 1 - fl(1/3) by 4.5e-8), and that offset would leak solute at every node and
// step; with integer m_k the only errors left are unbiased roundings.
//
// D2Q9 follows the ordering of Sec. 3.1 (LBM notations): e0 = 0,
// e1..e4 = (1,0),(0,1),(-1,0),(0,-1), e5..e8 = (1,1),(-1,1),(-1,-1),(1,-1),
// w = 4/9, 1/9, 1/36.  D3Q19 (named among the lattices of the paper's code in
// Sec. 3.1) is used for 3-D: rest (1/3), six face links (1/18), twelve edge
// links (1/36), with opposite directions stored next to each other.
//
// D2Q5 and D3Q7 (also named in Sec. 3.1) can carry the composition populations
// h: the rest and axis links of D2Q9 / D3Q19, in the same order, with weights
// for xi_s^2 = 1/3 as on the full lattices (so tau_h = 3 / gamma is unchanged):
// D2Q5 w = 1/3, 1/6; D3Q7 w = 0, 1/6.  Their weights are m_k / 6 (DEN = 6),
// again with unit m_k on the moving links.
#pragma once

namespace lbpf {

struct D2Q9 {
    static constexpr int D = 2;
    static constexpr int Q = 9;
    static constexpr int DEN = 36;          // w_k = m_k / DEN
    static constexpr bool FLAT_Y = false;   // has links along y
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
    // w_k = m_k / 36 with integer m_k; the moving links have power-of-two m_k
    __host__ __device__ static constexpr int m(int k) { return k == 0 ? 16 : (k <= 4 ? 4 : 1); }
};

struct D3Q19 {
    static constexpr int D = 3;
    static constexpr int Q = 19;
    static constexpr int DEN = 36;
    static constexpr bool FLAT_Y = false;
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
    // w_k = m_k / 36 with integer m_k; the moving links have power-of-two m_k
    __host__ __device__ static constexpr int m(int k) { return k == 0 ? 12 : (k <= 6 ? 2 : 1); }
};

// D2Q9 with its y links relabelled as z links: the 2-D grid [y][x] read as
// the 3-D grid [z = y][1][x], so that the z-marching kernels walk the rows of a
// 2-D domain, each "plane" being a segment of one row.  Same links, weights
// and ordering as D2Q9; only the kernels' view of the axes changes.
struct D2Q9R {
    static constexpr int D = 3;               // marched like a 3-D lattice
    static constexpr int Q = 9;
    static constexpr int DEN = 36;
    static constexpr bool FLAT_Y = true;      // no links along the (unit) y axis
    __host__ __device__ static constexpr int ex(int k) { return D2Q9::ex(k); }
    __host__ __device__ static constexpr int ey(int) { return 0; }
    __host__ __device__ static constexpr int ez(int k) { return D2Q9::ey(k); }
    __host__ __device__ static constexpr double w(int k) { return D2Q9::w(k); }
    __host__ __device__ static constexpr int opp(int k) { return D2Q9::opp(k); }
    __host__ __device__ static constexpr int m(int k) { return D2Q9::m(k); }
};

// Small lattices for h: the first Q links of the full lattice.
template <class Full, int QH, int M0>
struct SmallLattice {
    static constexpr int D = Full::D;
    static constexpr int Q = QH;
    static constexpr int DEN = 6;
    static constexpr bool FLAT_Y = Full::FLAT_Y;
    __host__ __device__ static constexpr int ex(int k) { return Full::ex(k); }
    __host__ __device__ static constexpr int ey(int k) { return Full::ey(k); }
    __host__ __device__ static constexpr int ez(int k) { return Full::ez(k); }
    __host__ __device__ static constexpr int m(int k) { return k == 0 ? M0 : 1; }
    __host__ __device__ static constexpr double w(int k) { return m(k) / 6.0; }
    __host__ __device__ static constexpr int opp(int k) { return Full::opp(k); }
};
using D2Q5 = SmallLattice<D2Q9, 5, 2>;     // w = 1/3, 1/6
using D2Q5R = SmallLattice<D2Q9R, 5, 2>;   // the same in the row-marching view
using D3Q7 = SmallLattice<D3Q19, 7, 0>;    // w = 0, 1/6

// The small lattice of h that goes with a full one.
template <class L>
struct SmallOf;
template <>
struct SmallOf<D2Q9> { using type = D2Q5; };
template <>
struct SmallOf<D2Q9R> { using type = D2Q5R; };
template <>
struct SmallOf<D3Q19> { using type = D3Q7; };

}  // namespace lbpf
