// Host-side setup of the nodal DG discretisation: reference element, mesh geometry,
// connectivity, multi-rate levels and the element ordering used on the device.
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace ridg {

struct Error {
  int code;
  std::string msg;
};

// Dense row-major matrix helpers (small sizes only).
struct Mat {
  int r = 0, c = 0;
  std::vector<double> a;
  Mat() = default;
  Mat(int r_, int c_) : r(r_), c(c_), a(size_t(r_) * c_, 0.0) {}
  double& operator()(int i, int j) { return a[size_t(i) * c + j]; }
  double operator()(int i, int j) const { return a[size_t(i) * c + j]; }
};
Mat matmul(const Mat& A, const Mat& B);
Mat transpose(const Mat& A);
Mat inverse(const Mat& A);  // LU with partial pivoting; throws Error on a singular matrix

inline int n_nodes(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
inline int n_face_nodes(int N) { return (N + 1) * (N + 2) / 2; }

// Local face f of (v0,v1,v2,v3) spans kFaceVerts[f]; kFaceOpp[f] is the opposite vertex.
constexpr int kFaceVerts[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};
constexpr int kFaceOpp[4] = {3, 2, 0, 1};

// Reference tetrahedron of order N (Sec. 3.1, appendix).
struct RefElem {
  int N = 0, Np = 0, Nfp = 0;
  std::vector<std::array<double, 3>> rst;   // [Np] warp-and-blend nodes
  std::vector<std::array<int, 4>> lattice;  // [Np] equidistant lattice barycentrics (sum N)
  Mat D[3];                                  // D_r, D_s, D_t  [Np][Np]
  Mat M, Minv;                               // mass matrix
  Mat LIFT;                                  // [Np][4*Nfp]
  std::vector<std::array<int, 32>> fmask;    // [4][Nfp] (first Nfp entries used)
  // perm[code][j]: face-node index on the neighbour face matching local face node j, for the six
  // vertex correspondences code = 0..5 of a shared triangle.
  std::vector<std::array<int, 32>> perm;
  Mat V, Vinv;  // Vandermonde of the Legendre-product basis
  std::vector<double> basis_at(const std::array<double, 3>& p) const;       // phi(p)
  std::vector<double> lagrange_at(const std::array<double, 3>& p) const;    // l(p), size Np
};
RefElem build_reference(int N);
// The same reference element with its nodes renumbered: node p of the result is node order[p] of re
// (operators, mass matrices, LIFT rows, face masks and the Lagrange basis follow).
RefElem permute_nodes(const RefElem& re, const std::vector<int>& order);
// A node numbering under which the Nfp nodes of every face spread as evenly as possible over the
// eight classes p mod 8 (order[p] = node of re at position p).  In shared-memory rows of 4 (mod 32)
// words, node rows of one class share a bank group, so a face-node gather over one column costs
// as many bank wavefronts as the fullest class holds face nodes.
std::vector<int> bank_spread_order(const RefElem& re);
std::vector<double> gauss_lobatto(int N);

// The six orderings of a triangle's vertices: kTriPerm[code][x] = index (in the local face's
// vertex order) of the vertex that the neighbour face lists at position x.
extern const int kTriPerm[6][3];

struct MeshData {
  int64_t K = 0, n_vert = 0;
  std::vector<double> xyz;    // [n_vert][3]
  std::vector<int64_t> tet;   // [K][4]
  std::vector<int8_t> bc;     // [K][4]  0 interior, else RIDG_BC_* code
  std::vector<int64_t> nbr;   // [K][4]  neighbour element or -1
  std::vector<int8_t> nbr_face;   // [K][4]
  std::vector<int8_t> perm_code;  // [K][4]  which of the six correspondences
  int64_t n_boundary = 0, n_interior = 0;
};
// Throws Error on bad input.
MeshData build_mesh(const double* xyz, int64_t n_vert, const int64_t* tet, int64_t K, const int8_t* face_bc,
                    int8_t default_bc);

// Geometry of every element (appendix): inverse Jacobian, normals, J_f/J, Jacobian.
struct Geometry {
  std::vector<double> rx;      // [K][3][3]  rx[k][i][j] = d r_j / d x_i
  std::vector<double> normal;  // [K][4][3]
  std::vector<double> fscale;  // [K][4]     J_f / J
  std::vector<double> J;       // [K]
  std::vector<double> lmin;    // [K]        smallest face-to-opposite-vertex distance
};
Geometry build_geometry(const MeshData& m);

struct Levels {
  std::vector<int> level;  // [K] 1 = coarsest
  int n_levels = 1;
  double dt_local = 0.0;
};
Levels assign_levels(const MeshData& m, const Geometry& g, int N, const double* c, double cfl, int n_levels_max);

// Element order on the device: levels coarse -> fine, each level padded to a multiple of 32.
// Slots [0, owned_end) are the elements the solver advances.  A solver for one part of a partitioned
// mesh (Sec. 4.2) places after them, in slots [owned_end, n_slots), the ghosts: elements of other
// parts that share a face with one of its own; they are never advanced, but their face inboxes
// receive the traces this part pushes across the interface (which the other part then takes).
struct Ordering {
  int64_t n_slots = 0;
  int64_t owned_end = 0;
  std::vector<int64_t> slot_of;      // [K], -1 for elements of other parts that are not ghosts
  std::vector<int64_t> elem_of;      // [n_slots], -1 for padding
  std::vector<int64_t> level_begin;  // [n_levels+1] slot ranges per level (multiples of 32)
};
Ordering build_ordering(const Levels& lv, int64_t K);
// The elements with part[k] == rank by level, then their ghosts (padded to a multiple of 32).
Ordering build_part_ordering(const Levels& lv, const MeshData& m, const int32_t* part, int32_t rank);

// Partition of the elements into n_parts (Sec. 4.2): weights 2^(l-1) per element; every element of
// the finest level, or connected group of them, lumped with its face neighbours and kept in one part
// unless the lump weighs more than half of one part's share; weighted recursive coordinate bisection
// of the lumps' weighted vertex centroids (split across the longest extent at the weighted median).
std::vector<int32_t> partition_mesh(const MeshData& m, const Levels& lv, int32_t n_parts);

// Point location: lowest element index whose barycentrics are all >= -1e-12; returns -1 if none.
// Uniform grid over the mesh's bounding box; each cell lists (in increasing order) the elements
// whose bounding box, widened by a relative 1e-9, meets the cell.
struct PointLocator {
  double lo[3] = {0, 0, 0}, h[3] = {1, 1, 1};
  int n[3] = {1, 1, 1};
  std::vector<int64_t> start;  // [cells + 1]
  std::vector<int64_t> items;  // element ids per cell
};
PointLocator build_locator(const MeshData& m);
// Element containing x (barycentric coordinates >= -1e-12) with the lowest index, and the reference
// coordinates of x in it; -1 if no element contains x.
int64_t locate_point(const MeshData& m, const PointLocator& L, const double x[3], double rst[3]);

}  // namespace ridg
