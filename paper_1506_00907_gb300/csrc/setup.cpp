// Host setup of the nodal DG discretisation (Sec. 3.1, Sec. 3.2 and the appendix).
//
// The reference element spans P_N with products of Legendre polynomials L_a(r) L_b(s) L_c(t),
// a+b+c <= N, and integrates with a collapsed-coordinate Gauss-Legendre rule that is exact for
// the degrees involved.  Nodes are the warp-and-blend nodes (Warburton 2006, cited in Sec. 3.1),
// without the optimisation constant.  Face-node correspondences come from the nodes' lattice
// barycentrics and the vertex correspondence of the shared triangle; normals and J_f/J from
// Nanson's formula.
#include "setup.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

#include "ridg.h"

namespace ridg {

// ------------------------------------------------------------------ dense helpers
Mat matmul(const Mat& A, const Mat& B) {
  Mat C(A.r, B.c);
  for (int i = 0; i < A.r; ++i)
    for (int k = 0; k < A.c; ++k) {
      double a = A(i, k);
      if (a == 0.0) continue;
      for (int j = 0; j < B.c; ++j) C(i, j) += a * B(k, j);
    }
  return C;
}

Mat transpose(const Mat& A) {
  Mat T(A.c, A.r);
  for (int i = 0; i < A.r; ++i)
    for (int j = 0; j < A.c; ++j) T(j, i) = A(i, j);
  return T;
}

Mat inverse(const Mat& A) {
  int n = A.r;
  Mat LU = A, inv(n, n);
  std::vector<int> piv(n);
  std::iota(piv.begin(), piv.end(), 0);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(LU(i, k)) > std::fabs(LU(p, k))) p = i;
    if (LU(p, k) == 0.0) throw Error{RIDG_E_INVALID_ARG, "singular matrix in reference-element setup"};
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(LU(p, j), LU(k, j));
      std::swap(piv[p], piv[k]);
    }
    for (int i = k + 1; i < n; ++i) {
      LU(i, k) /= LU(k, k);
      for (int j = k + 1; j < n; ++j) LU(i, j) -= LU(i, k) * LU(k, j);
    }
  }
  for (int col = 0; col < n; ++col) {
    std::vector<double> x(n);
    for (int i = 0; i < n; ++i) x[i] = (piv[i] == col) ? 1.0 : 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) x[i] -= LU(i, j) * x[j];
    for (int i = n - 1; i >= 0; --i) {
      for (int j = i + 1; j < n; ++j) x[i] -= LU(i, j) * x[j];
      x[i] /= LU(i, i);
    }
    for (int i = 0; i < n; ++i) inv(i, col) = x[i];
  }
  return inv;
}

// ------------------------------------------------------------------ 1-D polynomials
// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
static void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    p = 1.0;
    dp = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = pk;
  }
  p = p1;
  // derivative from n (P_{n-1} - x P_n) = (1 - x^2) P_n'; at x = +-1 use P_n'(+-1) = (+-1)^{n-1} n(n+1)/2
  if (std::fabs(1.0 - x * x) < 1e-14) {
    dp = (x > 0 ? 1.0 : ((n % 2) ? 1.0 : -1.0)) * n * (n + 1) / 2.0;
  } else {
    dp = n * (p0 - x * p1) / (1.0 - x * x);
  }
}

std::vector<double> gauss_lobatto(int N) {
  std::vector<double> x(N + 1);
  x[0] = -1.0;
  x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double z = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(N, z, p, dp);
      // second derivative from the Legendre equation
      double d2p = (2.0 * z * dp - N * (N + 1.0) * p) / (1.0 - z * z);
      double dz = dp / d2p;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[j] = z;
  }
  return x;
}

static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double p = 0, dp = 0;
    for (int it = 0; it < 100; ++it) {
      legendre(n, z, p, dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre(n, z, p, dp);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// blend-divided 1-D warp: (GLL - equidistant displacement interpolant)(r) / (1 - r^2)
static double warp_factor(int N, double r) {
  if (std::fabs(r) >= 1.0 - 1e-10) return 0.0;
  std::vector<double> gll = gauss_lobatto(N);
  double w = 0.0;
  for (int i = 0; i <= N; ++i) {
    double ri = -1.0 + 2.0 * i / N;
    double li = 1.0;
    for (int j = 0; j <= N; ++j) {
      if (j == i) continue;
      double rj = -1.0 + 2.0 * j / N;
      li *= (r - rj) / (ri - rj);
    }
    w += (gll[i] - ri) * li;
  }
  return w / (1.0 - r * r);
}

// ------------------------------------------------------------------ nodes
static std::vector<std::array<double, 3>> warp_blend_nodes(int N, std::vector<std::array<int, 4>>& lattice) {
  // vertices of an equilateral tetrahedron, in the order of the reference vertices v0..v3
  const double s3 = std::sqrt(3.0), s6 = std::sqrt(6.0);
  const double E[4][3] = {{-1.0, -1.0 / s3, -1.0 / s6}, {1.0, -1.0 / s3, -1.0 / s6}, {0.0, 2.0 / s3, -1.0 / s6},
                          {0.0, 0.0, 3.0 / s6}};
  std::vector<std::array<double, 3>> out;
  lattice.clear();
  for (int kt = 0; kt <= N; ++kt)
    for (int js = 0; js <= N - kt; ++js)
      for (int ir = 0; ir <= N - js - kt; ++ir) {
        // barycentrics of the lattice point: lambda_1 ~ r, lambda_2 ~ s, lambda_3 ~ t
        int l1 = ir, l2 = js, l3 = kt, l0 = N - ir - js - kt;
        lattice.push_back({l0, l1, l2, l3});
        double lam[4] = {double(l0) / N, double(l1) / N, double(l2) / N, double(l3) / N};
        double X[3] = {0, 0, 0};
        for (int v = 0; v < 4; ++v)
          for (int d = 0; d < 3; ++d) X[d] += lam[v] * E[v][d];
        double shift[3] = {0, 0, 0};
        int npos = 0;
        for (int v = 0; v < 4; ++v) npos += (lam[v] > 1e-10);
        bool edge = (npos == 2);
        if (N > 1) {
          for (int f = 0; f < 4; ++f) {
            const int* fv = kFaceVerts[f];
            int o = kFaceOpp[f];
            double warp[3] = {0, 0, 0};
            int pairs[3][2] = {{fv[0], fv[1]}, {fv[1], fv[2]}, {fv[2], fv[0]}};
            for (auto& pr : pairs) {
              int a = pr[0], b = pr[1];
              double t[3], nt = 0;
              for (int d = 0; d < 3; ++d) {
                t[d] = E[b][d] - E[a][d];
                nt += t[d] * t[d];
              }
              nt = std::sqrt(nt);
              double amt = 4.0 * lam[a] * lam[b] * warp_factor(N, lam[b] - lam[a]);
              for (int d = 0; d < 3; ++d) warp[d] += amt * t[d] / nt;
            }
            if (edge) {
              if (lam[o] < 1e-10)
                for (int d = 0; d < 3; ++d) shift[d] = warp[d];  // unblended edge warp (set, not added)
              continue;
            }
            double num = lam[fv[0]] * lam[fv[1]] * lam[fv[2]];
            double den = (lam[fv[0]] + 0.5 * lam[o]) * (lam[fv[1]] + 0.5 * lam[o]) * (lam[fv[2]] + 0.5 * lam[o]);
            double blend = den > 1e-10 ? num / den : 0.0;
            for (int d = 0; d < 3; ++d) shift[d] += blend * warp[d];
          }
        }
        double Xw[3] = {X[0] + shift[0], X[1] + shift[1], X[2] + shift[2]};
        // invert X = (E1+E2+E3-E0)/2 + (r (E1-E0) + s (E2-E0) + t (E3-E0))/2
        Mat A(3, 3);
        double rhs[3];
        for (int d = 0; d < 3; ++d) {
          A(d, 0) = 0.5 * (E[1][d] - E[0][d]);
          A(d, 1) = 0.5 * (E[2][d] - E[0][d]);
          A(d, 2) = 0.5 * (E[3][d] - E[0][d]);
          rhs[d] = Xw[d] - 0.5 * (E[1][d] + E[2][d] + E[3][d] - E[0][d]);
        }
        Mat Ai = inverse(A);
        std::array<double, 3> p{};
        for (int i = 0; i < 3; ++i) p[i] = Ai(i, 0) * rhs[0] + Ai(i, 1) * rhs[1] + Ai(i, 2) * rhs[2];
        out.push_back(p);
      }
  return out;
}

// ------------------------------------------------------------------ basis
static std::vector<std::array<int, 3>> basis_indices(int N) {
  std::vector<std::array<int, 3>> idx;
  for (int a = 0; a <= N; ++a)
    for (int b = 0; b <= N - a; ++b)
      for (int c = 0; c <= N - a - b; ++c) idx.push_back({a, b, c});
  return idx;
}

static void basis_eval(int N, const std::array<double, 3>& p, std::vector<double>& phi, std::vector<double>* grad) {
  auto idx = basis_indices(N);
  double L[3][8], dL[3][8];
  for (int d = 0; d < 3; ++d)
    for (int n = 0; n <= N; ++n) legendre(n, p[d], L[d][n], dL[d][n]);
  phi.resize(idx.size());
  if (grad) grad->assign(3 * idx.size(), 0.0);
  for (size_t q = 0; q < idx.size(); ++q) {
    int a = idx[q][0], b = idx[q][1], c = idx[q][2];
    phi[q] = L[0][a] * L[1][b] * L[2][c];
    if (grad) {
      (*grad)[0 * idx.size() + q] = dL[0][a] * L[1][b] * L[2][c];
      (*grad)[1 * idx.size() + q] = L[0][a] * dL[1][b] * L[2][c];
      (*grad)[2 * idx.size() + q] = L[0][a] * L[1][b] * dL[2][c];
    }
  }
}

std::vector<double> RefElem::basis_at(const std::array<double, 3>& p) const {
  std::vector<double> phi;
  basis_eval(N, p, phi, nullptr);
  return phi;
}

std::vector<double> RefElem::lagrange_at(const std::array<double, 3>& p) const {
  // l(p) = V^{-T} phi(p)
  std::vector<double> phi = basis_at(p), l(Np, 0.0);
  for (int i = 0; i < Np; ++i)
    for (int q = 0; q < Np; ++q) l[i] += Vinv(q, i) * phi[q];
  return l;
}

const int kTriPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

RefElem build_reference(int N) {
  if (N < 1 || N > 6) throw Error{RIDG_E_INVALID_ARG, "order N must be in 1..6"};
  RefElem re;
  re.N = N;
  re.Np = n_nodes(N);
  re.Nfp = n_face_nodes(N);
  re.rst = warp_blend_nodes(N, re.lattice);
  const int Np = re.Np, Nfp = re.Nfp;
  re.V = Mat(Np, Np);
  Mat Vd[3] = {Mat(Np, Np), Mat(Np, Np), Mat(Np, Np)};
  for (int i = 0; i < Np; ++i) {
    std::vector<double> phi, grad;
    basis_eval(N, re.rst[i], phi, &grad);
    for (int q = 0; q < Np; ++q) {
      re.V(i, q) = phi[q];
      for (int d = 0; d < 3; ++d) Vd[d](i, q) = grad[d * Np + q];
    }
  }
  re.Vinv = inverse(re.V);
  for (int d = 0; d < 3; ++d) re.D[d] = matmul(Vd[d], re.Vinv);
  // mass matrix by collapsed Gauss-Legendre quadrature (exact for degree 2N)
  std::vector<double> gx, gw;
  gauss_legendre(N + 3, gx, gw);
  re.M = Mat(Np, Np);
  for (size_t i = 0; i < gx.size(); ++i)
    for (size_t j = 0; j < gx.size(); ++j)
      for (size_t k = 0; k < gx.size(); ++k) {
        double a = gx[i], b = gx[j], c = gx[k];
        std::array<double, 3> p = {(1 + a) * (1 - b) * (1 - c) / 4 - 1, (1 + b) * (1 - c) / 2 - 1, c};
        double w = gw[i] * gw[j] * gw[k] * (1 - b) / 2 * (1 - c) / 2 * (1 - c) / 2;
        std::vector<double> l = re.lagrange_at(p);
        for (int m = 0; m < Np; ++m)
          for (int n = 0; n < Np; ++n) re.M(m, n) += w * l[m] * l[n];
      }
  re.Minv = inverse(re.M);
  // face nodes: the opposite vertex's lattice barycentric is zero
  re.fmask.assign(4, {});
  for (int f = 0; f < 4; ++f) {
    int cnt = 0;
    for (int n = 0; n < Np; ++n)
      if (re.lattice[n][kFaceOpp[f]] == 0) re.fmask[f][cnt++] = n;
    if (cnt != Nfp) throw Error{RIDG_E_INVALID_ARG, "face node count mismatch"};
  }
  // face mass matrices on the 2-D reference triangle {u, v >= -1, u + v <= 0} (area 2)
  Mat E(Np, 4 * Nfp);
  const double Vref[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
  for (int f = 0; f < 4; ++f) {
    Mat Mf(Nfp, Nfp);
    for (size_t i = 0; i < gx.size(); ++i)
      for (size_t j = 0; j < gx.size(); ++j) {
        double a = gx[i], b = gx[j];
        double u = (1 + a) * (1 - b) / 2 - 1, v = b;
        double w = gw[i] * gw[j] * (1 - b) / 2;
        const double* A = Vref[kFaceVerts[f][0]];
        const double* B = Vref[kFaceVerts[f][1]];
        const double* C = Vref[kFaceVerts[f][2]];
        std::array<double, 3> p;
        for (int d = 0; d < 3; ++d) p[d] = -(u + v) / 2 * A[d] + (1 + u) / 2 * B[d] + (1 + v) / 2 * C[d];
        std::vector<double> l = re.lagrange_at(p);
        for (int m = 0; m < Nfp; ++m)
          for (int n = 0; n < Nfp; ++n) Mf(m, n) += w * l[re.fmask[f][m]] * l[re.fmask[f][n]];
      }
    for (int m = 0; m < Nfp; ++m)
      for (int n = 0; n < Nfp; ++n) E(re.fmask[f][m], f * Nfp + n) = Mf(m, n);
  }
  re.LIFT = matmul(re.Minv, E);
  // face-node correspondences from lattice barycentrics
  re.perm.assign(6, {});
  for (int code = 0; code < 6; ++code) {
    // face nodes of the reference face 0 (vertices 0,1,2) as barycentric triples
    for (int j = 0; j < Nfp; ++j) {
      const auto& lj = re.lattice[re.fmask[0][j]];
      int tri[3] = {lj[0], lj[1], lj[2]};
      int want[3];
      for (int x = 0; x < 3; ++x) want[x] = tri[kTriPerm[code][x]];
      int found = -1;
      for (int jj = 0; jj < Nfp; ++jj) {
        const auto& lk = re.lattice[re.fmask[0][jj]];
        if (lk[0] == want[0] && lk[1] == want[1] && lk[2] == want[2]) found = jj;
      }
      if (found < 0) throw Error{RIDG_E_INVALID_ARG, "face permutation not found"};
      re.perm[code][j] = found;
    }
  }
  return re;
}

RefElem permute_nodes(const RefElem& re, const std::vector<int>& order) {
  const int Np = re.Np;
  if (int(order.size()) != Np) throw Error{RIDG_E_INVALID_ARG, "node order size mismatch"};
  std::vector<int> pos(Np, -1);
  for (int p = 0; p < Np; ++p) {
    if (order[p] < 0 || order[p] >= Np || pos[order[p]] >= 0) throw Error{RIDG_E_INVALID_ARG, "not a node permutation"};
    pos[order[p]] = p;
  }
  RefElem out = re;
  for (int p = 0; p < Np; ++p) {
    out.rst[p] = re.rst[order[p]];
    out.lattice[p] = re.lattice[order[p]];
    for (int q = 0; q < Np; ++q) {
      for (int d = 0; d < 3; ++d) out.D[d](p, q) = re.D[d](order[p], order[q]);
      out.M(p, q) = re.M(order[p], order[q]);
      out.Minv(p, q) = re.Minv(order[p], order[q]);
      out.V(p, q) = re.V(order[p], q);     // rows: nodes, columns: basis functions
      out.Vinv(q, p) = re.Vinv(q, order[p]);
    }
    for (int fm = 0; fm < 4 * re.Nfp; ++fm) out.LIFT(p, fm) = re.LIFT(order[p], fm);
  }
  for (int f = 0; f < 4; ++f)
    for (int j = 0; j < re.Nfp; ++j) out.fmask[f][j] = pos[re.fmask[f][j]];
  return out;
}

std::vector<int> bank_spread_order(const RefElem& re) {
  const int Np = re.Np, Nfp = re.Nfp;
  std::vector<int> order(Np);
  for (int p = 0; p < Np; ++p) order[p] = p;
  if (Np <= 8) return order;
  // faces of each node
  std::vector<std::vector<int>> faces_of(Np);
  for (int f = 0; f < 4; ++f)
    for (int j = 0; j < Nfp; ++j) faces_of[re.fmask[f][j]].push_back(f);
  // cost: sum over faces and classes of (face nodes in the class)^2, minimal for an even spread
  auto cost_of = [&](const std::vector<int>& ord) {
    int cnt[4][8] = {};
    for (int p = 0; p < Np; ++p)
      for (int f : faces_of[ord[p]]) ++cnt[f][p & 7];
    int c = 0, mx = 0;
    for (int f = 0; f < 4; ++f)
      for (int k = 0; k < 8; ++k) {
        c += cnt[f][k] * cnt[f][k];
        mx = std::max(mx, cnt[f][k]);
      }
    return 1000 * mx + c;
  };
  // deterministic restarts of a pairwise-swap descent
  std::vector<int> best = order;
  int best_cost = cost_of(best);
  uint64_t rng = 0x9e3779b97f4a7c15ull;
  for (int restart = 0; restart < 16; ++restart) {
    std::vector<int> cur(Np);
    for (int p = 0; p < Np; ++p) cur[p] = p;
    if (restart > 0)
      for (int p = Np - 1; p > 0; --p) {
        rng = rng * 6364136223846793005ull + 1442695040888963407ull;
        std::swap(cur[p], cur[int((rng >> 33) % uint64_t(p + 1))]);
      }
    int c = cost_of(cur);
    for (bool improved = true; improved;) {
      improved = false;
      for (int i = 0; i < Np; ++i)
        for (int j = i + 1; j < Np; ++j) {
          if ((i & 7) == (j & 7)) continue;
          std::swap(cur[i], cur[j]);
          int c2 = cost_of(cur);
          if (c2 < c) {
            c = c2;
            improved = true;
          } else {
            std::swap(cur[i], cur[j]);
          }
        }
    }
    if (c < best_cost) {
      best_cost = c;
      best = cur;
    }
  }
  return best;
}

// ------------------------------------------------------------------ mesh and connectivity
MeshData build_mesh(const double* xyz, int64_t n_vert, const int64_t* tet, int64_t K, const int8_t* face_bc,
                    int8_t default_bc) {
  if (!xyz || !tet || n_vert < 4 || K < 1) throw Error{RIDG_E_INVALID_ARG, "mesh: empty or null input"};
  if (default_bc < 1 || default_bc > 3) throw Error{RIDG_E_INVALID_ARG, "mesh: default_bc must be 1, 2 or 3"};
  MeshData m;
  m.K = K;
  m.n_vert = n_vert;
  m.xyz.assign(xyz, xyz + 3 * n_vert);
  m.tet.assign(tet, tet + 4 * K);
  for (int64_t i = 0; i < 4 * K; ++i)
    if (m.tet[i] < 0 || m.tet[i] >= n_vert) throw Error{RIDG_E_BAD_MESH, "mesh: vertex index out of range"};
  if (face_bc)
    for (int64_t i = 0; i < 4 * K; ++i)
      if (face_bc[i] < 0 || face_bc[i] > 3) throw Error{RIDG_E_INVALID_ARG, "mesh: face_bc code out of range"};
  // faces keyed by their sorted vertex triple
  struct FaceKey {
    int64_t v[3];
    int64_t elem;
    int face;
  };
  std::vector<FaceKey> faces(4 * K);
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      FaceKey fk;
      for (int x = 0; x < 3; ++x) fk.v[x] = m.tet[4 * k + kFaceVerts[f][x]];
      std::sort(fk.v, fk.v + 3);
      fk.elem = k;
      fk.face = f;
      faces[4 * k + f] = fk;
    }
  std::sort(faces.begin(), faces.end(), [](const FaceKey& a, const FaceKey& b) {
    if (a.v[0] != b.v[0]) return a.v[0] < b.v[0];
    if (a.v[1] != b.v[1]) return a.v[1] < b.v[1];
    if (a.v[2] != b.v[2]) return a.v[2] < b.v[2];
    if (a.elem != b.elem) return a.elem < b.elem;
    return a.face < b.face;
  });
  m.nbr.assign(4 * K, -1);
  m.nbr_face.assign(4 * K, -1);
  m.perm_code.assign(4 * K, 0);
  m.bc.assign(4 * K, 0);
  auto same = [](const FaceKey& a, const FaceKey& b) {
    return a.v[0] == b.v[0] && a.v[1] == b.v[1] && a.v[2] == b.v[2];
  };
  for (size_t i = 0; i < faces.size();) {
    size_t j = i + 1;
    while (j < faces.size() && same(faces[i], faces[j])) ++j;
    if (j - i > 2) throw Error{RIDG_E_BAD_MESH, "mesh: a face is shared by more than two elements"};
    if (j - i == 2) {
      const FaceKey& a = faces[i];
      const FaceKey& b = faces[i + 1];
      if (a.elem == b.elem) throw Error{RIDG_E_BAD_MESH, "mesh: degenerate element (repeated face)"};
      m.nbr[4 * a.elem + a.face] = b.elem;
      m.nbr_face[4 * a.elem + a.face] = int8_t(b.face);
      m.nbr[4 * b.elem + b.face] = a.elem;
      m.nbr_face[4 * b.elem + b.face] = int8_t(a.face);
    }
    i = j;
  }
  // vertex correspondence of each shared face: the neighbour lists vertex x of its face as our
  // local vertex kTriPerm[code][x]
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      int64_t k2 = m.nbr[4 * k + f];
      if (k2 < 0) {
        int8_t code = face_bc ? face_bc[4 * k + f] : 0;
        m.bc[4 * k + f] = code ? code : default_bc;
        ++m.n_boundary;
        continue;
      }
      if (face_bc && face_bc[4 * k + f] != 0) throw Error{RIDG_E_BAD_MESH, "mesh: boundary code on an interior face"};
      ++m.n_interior;
      int f2 = m.nbr_face[4 * k + f];
      int64_t mine[3], theirs[3];
      for (int x = 0; x < 3; ++x) {
        mine[x] = m.tet[4 * k + kFaceVerts[f][x]];
        theirs[x] = m.tet[4 * k2 + kFaceVerts[f2][x]];
      }
      int code = -1;
      for (int c = 0; c < 6 && code < 0; ++c) {
        bool ok = true;
        for (int x = 0; x < 3; ++x) ok = ok && (theirs[x] == mine[kTriPerm[c][x]]);
        if (ok) code = c;
      }
      if (code < 0) throw Error{RIDG_E_BAD_MESH, "mesh: shared face vertices do not correspond"};
      m.perm_code[4 * k + f] = int8_t(code);
    }
  m.n_interior /= 2;
  return m;
}

// ------------------------------------------------------------------ geometry
static void inv3(const double A[3][3], double Ai[3][3], double& det) {
  det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
        A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  double id = 1.0 / det;
  Ai[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) * id;
  Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id;
  Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id;
  Ai[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) * id;
  Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id;
  Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id;
  Ai[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) * id;
  Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id;
  Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id;
}

static void element_jacobian(const MeshData& m, int64_t k, double A[3][3]) {
  const double* P0 = &m.xyz[3 * m.tet[4 * k + 0]];
  for (int col = 0; col < 3; ++col) {
    const double* Pc = &m.xyz[3 * m.tet[4 * k + 1 + col]];
    for (int d = 0; d < 3; ++d) A[d][col] = 0.5 * (Pc[d] - P0[d]);  // dx_d / dr_col
  }
}

Geometry build_geometry(const MeshData& m) {
  Geometry g;
  const int64_t K = m.K;
  g.rx.resize(9 * K);
  g.normal.resize(12 * K);
  g.fscale.resize(4 * K);
  g.J.resize(K);
  g.lmin.resize(K);
  // reference outward normals scaled by (reference face area)/2
  const double nref[4][3] = {{0, 0, -1}, {0, -1, 0}, {1, 1, 1}, {-1, 0, 0}};
  for (int64_t k = 0; k < K; ++k) {
    double A[3][3], Ai[3][3], det;
    element_jacobian(m, k, A);
    inv3(A, Ai, det);
    if (!(det > 0.0) || !std::isfinite(det))
      throw Error{RIDG_E_BAD_MESH, "mesh: element " + std::to_string(k) + " has a non-positive Jacobian"};
    g.J[k] = det;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) g.rx[9 * k + 3 * i + j] = Ai[j][i];  // d r_j / d x_i
    double fmax = 0.0;
    for (int f = 0; f < 4; ++f) {
      double n[3];
      for (int i = 0; i < 3; ++i) n[i] = Ai[0][i] * nref[f][0] + Ai[1][i] * nref[f][1] + Ai[2][i] * nref[f][2];
      double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      g.fscale[4 * k + f] = nn;  // Nanson: (face area / 2) / J
      for (int i = 0; i < 3; ++i) g.normal[12 * k + 3 * f + i] = n[i] / nn;
      fmax = std::max(fmax, nn);
    }
    g.lmin[k] = 2.0 / fmax;  // 3 V / (largest face area) with V = 4J/3 and area = 2 J fscale
  }
  return g;
}

// ------------------------------------------------------------------ levels (Sec. 3.2)
Levels assign_levels(const MeshData& m, const Geometry& g, int N, const double* c, double cfl, int n_levels_max) {
  Levels lv;
  const int64_t K = m.K;
  std::vector<double> dtk(K);
  double dtmin = 1e300;
  for (int64_t k = 0; k < K; ++k) {
    if (!(c[k] > 0.0)) throw Error{RIDG_E_INVALID_ARG, "velocity must be positive"};
    dtk[k] = cfl * g.lmin[k] / ((N + 1.0) * (N + 1.0) * c[k]);
    dtmin = std::min(dtmin, dtk[k]);
  }
  lv.dt_local = dtmin;
  std::vector<int> L(K);
  int Lmax = 0;
  for (int64_t k = 0; k < K; ++k) {
    L[k] = int(std::floor(std::log2(dtk[k] / dtmin) * (1.0 + 1e-12)));
    Lmax = std::max(Lmax, L[k]);
  }
  lv.n_levels = std::min(n_levels_max, 1 + Lmax);
  lv.level.resize(K);
  for (int64_t k = 0; k < K; ++k) lv.level[k] = lv.n_levels - std::min(L[k], lv.n_levels - 1);
  // move elements to finer levels until neighbours differ by at most one level (the smallest
  // such assignment; it does not depend on the sweep order)
  bool changed = true;
  while (changed) {
    changed = false;
    for (int64_t k = 0; k < K; ++k)
      for (int f = 0; f < 4; ++f) {
        int64_t k2 = m.nbr[4 * k + f];
        if (k2 >= 0 && lv.level[k] < lv.level[k2] - 1) {
          lv.level[k] = lv.level[k2] - 1;
          changed = true;
        }
      }
  }
  return lv;
}

Ordering build_ordering(const Levels& lv, int64_t K) {
  Ordering o;
  o.slot_of.assign(K, -1);
  o.level_begin.assign(lv.n_levels + 1, 0);
  int64_t slot = 0;
  for (int l = 1; l <= lv.n_levels; ++l) {
    o.level_begin[l - 1] = slot;
    for (int64_t k = 0; k < K; ++k)
      if (lv.level[k] == l) o.slot_of[k] = slot++;
    slot = (slot + 31) / 32 * 32;
  }
  o.level_begin[lv.n_levels] = slot;
  o.n_slots = slot;
  o.owned_end = slot;
  o.elem_of.assign(slot, -1);
  for (int64_t k = 0; k < K; ++k) o.elem_of[o.slot_of[k]] = k;
  return o;
}

Ordering build_part_ordering(const Levels& lv, const MeshData& m, const int32_t* part, int32_t rank) {
  const int64_t K = m.K;
  Ordering o;
  o.slot_of.assign(K, -1);
  o.level_begin.assign(lv.n_levels + 1, 0);
  int64_t slot = 0;
  for (int l = 1; l <= lv.n_levels; ++l) {
    o.level_begin[l - 1] = slot;
    for (int64_t k = 0; k < K; ++k)
      if (part[k] == rank && lv.level[k] == l) o.slot_of[k] = slot++;
    slot = (slot + 31) / 32 * 32;
  }
  o.level_begin[lv.n_levels] = slot;
  o.owned_end = slot;
  std::vector<char> ghost(K, 0);
  for (int64_t k = 0; k < K; ++k)
    if (part[k] == rank)
      for (int f = 0; f < 4; ++f) {
        const int64_t k2 = m.nbr[4 * k + f];
        if (k2 >= 0 && part[k2] != rank) ghost[k2] = 1;
      }
  for (int64_t k = 0; k < K; ++k)
    if (ghost[k]) o.slot_of[k] = slot++;
  slot = (slot + 31) / 32 * 32;
  o.n_slots = slot;
  o.elem_of.assign(slot, -1);
  for (int64_t k = 0; k < K; ++k)
    if (o.slot_of[k] >= 0) o.elem_of[o.slot_of[k]] = k;
  return o;
}

namespace {

// weighted recursive coordinate bisection of points (part index per point)
void rcb_split(const std::vector<std::array<double, 3>>& pt, const std::vector<double>& w, std::vector<int64_t> idx,
               int32_t first, int32_t n, std::vector<int32_t>& out) {
  if (n == 1 || idx.empty()) {
    for (int64_t i : idx) out[i] = first;
    return;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i : idx)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], pt[i][d]);
      hi[d] = std::max(hi[d], pt[i][d]);
    }
  int axis = 0;
  for (int d = 1; d < 3; ++d)
    if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
    return pt[a][axis] < pt[b][axis] || (pt[a][axis] == pt[b][axis] && a < b);
  });
  const int32_t n_left = n / 2;
  std::vector<double> cw(idx.size());
  double acc = 0.0;
  for (size_t i = 0; i < idx.size(); ++i) cw[i] = (acc += w[idx[i]]);
  const double target = cw.back() * double(n_left) / double(n);
  int64_t cut = std::lower_bound(cw.begin(), cw.end(), target) - cw.begin();
  if (idx.size() > 1)
    cut = std::min<int64_t>(std::max<int64_t>(cut, 1), int64_t(idx.size()) - 1);
  else
    cut = int64_t(idx.size());
  rcb_split(pt, w, std::vector<int64_t>(idx.begin(), idx.begin() + cut), first, n_left, out);
  rcb_split(pt, w, std::vector<int64_t>(idx.begin() + cut, idx.end()), first + n_left, n - n_left, out);
}

int64_t uf_find(std::vector<int64_t>& parent, int64_t a) {
  int64_t root = a;
  while (parent[root] != root) root = parent[root];
  while (parent[a] != root) {
    const int64_t next = parent[a];
    parent[a] = root;
    a = next;
  }
  return root;
}

}  // namespace

std::vector<int32_t> partition_mesh(const MeshData& m, const Levels& lv, int32_t n_parts) {
  const int64_t K = m.K;
  if (n_parts < 1) throw Error{RIDG_E_INVALID_ARG, "n_parts must be >= 1"};
  std::vector<double> w(K);
  double total = 0.0;
  for (int64_t k = 0; k < K; ++k) total += (w[k] = double(int64_t(1) << (lv.level[k] - 1)));
  // lumps: each finest element joined with its face neighbours
  std::vector<int64_t> parent(K);
  for (int64_t k = 0; k < K; ++k) parent[k] = k;
  if (lv.n_levels >= 2)
    for (int64_t k = 0; k < K; ++k)
      if (lv.level[k] == lv.n_levels)
        for (int f = 0; f < 4; ++f) {
          const int64_t k2 = m.nbr[4 * k + f];
          if (k2 < 0) continue;
          const int64_t ra = uf_find(parent, k), rb = uf_find(parent, k2);
          if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
        }
  // unit number per element: lumps in the order of their smallest element; the elements of lumps
  // too heavy to keep whole become units of their own, numbered after every kept lump
  std::vector<int64_t> root(K);
  for (int64_t k = 0; k < K; ++k) root[k] = uf_find(parent, k);
  std::vector<double> rw(K, 0.0);
  for (int64_t k = 0; k < K; ++k) rw[root[k]] += w[k];
  std::vector<int64_t> key(K);
  for (int64_t k = 0; k < K; ++k) key[k] = rw[root[k]] > 0.5 * total / double(n_parts) ? K + k : root[k];
  std::vector<int64_t> sorted = key;
  std::sort(sorted.begin(), sorted.end());
  sorted.erase(std::unique(sorted.begin(), sorted.end()), sorted.end());
  std::vector<int64_t> unit(K);
  for (int64_t k = 0; k < K; ++k) unit[k] = std::lower_bound(sorted.begin(), sorted.end(), key[k]) - sorted.begin();
  const int64_t n_units = int64_t(sorted.size());
  std::vector<double> uw(n_units, 0.0);
  std::vector<std::array<double, 3>> uc(n_units, {0.0, 0.0, 0.0});
  for (int64_t k = 0; k < K; ++k) uw[unit[k]] += w[k];
  for (int d = 0; d < 3; ++d)
    for (int64_t k = 0; k < K; ++k) {
      double cen = 0.0;
      for (int v = 0; v < 4; ++v) cen += m.xyz[3 * m.tet[4 * k + v] + d];
      uc[unit[k]][d] += w[k] * (cen / 4.0);
    }
  for (int64_t u = 0; u < n_units; ++u)
    for (int d = 0; d < 3; ++d) uc[u][d] /= uw[u];
  std::vector<int32_t> upart(n_units, 0);
  std::vector<int64_t> all(n_units);
  for (int64_t u = 0; u < n_units; ++u) all[u] = u;
  rcb_split(uc, uw, all, 0, n_parts, upart);
  std::vector<int32_t> out(K);
  for (int64_t k = 0; k < K; ++k) out[k] = upart[unit[k]];
  return out;
}

PointLocator build_locator(const MeshData& m) {
  PointLocator L;
  if (m.K == 0) {
    L.start.assign(2, 0);
    return L;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < m.n_vert; ++v)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], m.xyz[3 * v + d]);
      hi[d] = std::max(hi[d], m.xyz[3 * v + d]);
    }
  // about two elements per cell on average
  const double vol = std::max((hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]), 1e-300);
  const double cell = std::cbrt(2.0 * vol / double(m.K));
  int64_t cells = 1;
  for (int d = 0; d < 3; ++d) {
    const double ext = hi[d] - lo[d];
    L.n[d] = int(std::min<double>(std::max(1.0, std::ceil(ext / cell)), 1024.0));
    L.lo[d] = lo[d];
    L.h[d] = ext > 0 ? ext / L.n[d] : 1.0;
    cells *= L.n[d];
  }
  const double tol = 1e-9 * std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
  auto range = [&](int64_t k, int d, int& c0, int& c1) {
    double a = 1e300, b = -1e300;
    for (int v = 0; v < 4; ++v) {
      const double x = m.xyz[3 * m.tet[4 * k + v] + d];
      a = std::min(a, x);
      b = std::max(b, x);
    }
    c0 = std::max(0, std::min(L.n[d] - 1, int(std::floor((a - tol - L.lo[d]) / L.h[d]))));
    c1 = std::max(0, std::min(L.n[d] - 1, int(std::floor((b + tol - L.lo[d]) / L.h[d]))));
  };
  std::vector<int64_t> count(cells + 1, 0);
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int64_t> fill;
    if (pass == 1) {
      L.start.assign(cells + 1, 0);
      for (int64_t c = 0; c < cells; ++c) L.start[c + 1] = L.start[c] + count[c];
      L.items.assign(L.start[cells], 0);
      fill.assign(L.start.begin(), L.start.end() - 1);
    }
    for (int64_t k = 0; k < m.K; ++k) {  // increasing k: every cell's list comes out sorted
      int c0[3], c1[3];
      for (int d = 0; d < 3; ++d) range(k, d, c0[d], c1[d]);
      for (int z = c0[2]; z <= c1[2]; ++z)
        for (int y = c0[1]; y <= c1[1]; ++y)
          for (int x = c0[0]; x <= c1[0]; ++x) {
            const int64_t c = (int64_t(z) * L.n[1] + y) * L.n[0] + x;
            if (pass == 0)
              ++count[c];
            else
              L.items[fill[c]++] = k;
          }
    }
  }
  return L;
}

int64_t locate_point(const MeshData& m, const PointLocator& L, const double x[3], double rst[3]) {
  if (m.K == 0 || L.start.empty()) return -1;
  int c[3];
  for (int d = 0; d < 3; ++d) {
    const double u = (x[d] - L.lo[d]) / L.h[d];
    if (!(u >= -1e-6 && u <= L.n[d] + 1e-6)) return -1;  // outside the bounding box (or NaN)
    c[d] = std::max(0, std::min(L.n[d] - 1, int(std::floor(u))));
  }
  const int64_t cell = (int64_t(c[2]) * L.n[1] + c[1]) * L.n[0] + c[0];
  for (int64_t i = L.start[cell]; i < L.start[cell + 1]; ++i) {
    const int64_t k = L.items[i];
    double A[3][3], Ai[3][3], det;
    element_jacobian(m, k, A);
    inv3(A, Ai, det);
    const double* P0 = &m.xyz[3 * m.tet[4 * k]];
    double d[3] = {x[0] - P0[0], x[1] - P0[1], x[2] - P0[2]};
    double r1[3];  // r + 1
    for (int q = 0; q < 3; ++q) r1[q] = Ai[q][0] * d[0] + Ai[q][1] * d[1] + Ai[q][2] * d[2];
    double lam[4] = {1.0 - 0.5 * (r1[0] + r1[1] + r1[2]), 0.5 * r1[0], 0.5 * r1[1], 0.5 * r1[2]};
    if (lam[0] >= -1e-12 && lam[1] >= -1e-12 && lam[2] >= -1e-12 && lam[3] >= -1e-12) {
      for (int q = 0; q < 3; ++q) rst[q] = r1[q] - 1.0;
      return k;
    }
  }
  return -1;
}

}  // namespace ridg
