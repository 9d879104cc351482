// Host-side setup of the discretisations (no CUDA).  Setup cost is amortised
// over many right-hand sides (Sec. 1), so it runs once on the host and the
// results are uploaded; the hot path never touches these routines.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace chebmg {

// Global-id flag bits stored in the element-to-global map (ids use the low 30 bits).
constexpr uint32_t kGidDirichlet = 0x80000000u;
constexpr uint32_t kGidOwner = 0x40000000u;
constexpr uint32_t kGidMask = 0x3fffffffu;

// GLL points and weights of order N on [-1, 1] and the Lagrange derivative
// matrix Dm[i*(N+1)+j] = l_j'(x_i).
void gll_rule(int N, std::vector<double>& x, std::vector<double>& w);
void gll_derivative(int N, const std::vector<double>& x, std::vector<double>& Dm);
// J[a*nc + b] = l_b(y_a), Lagrange basis on nodes xc (size nc) at points y.
void lagrange_interp(const std::vector<double>& xc, const std::vector<double>& y,
                     std::vector<double>& J);

struct SemHostLevel {
  int N = 0, NQ = 0, NP = 0;
  int nex = 0, ney = 0, nez = 0;
  int64_t E = 0, n = 0;
  std::vector<double> x, w, Dm;
  std::vector<uint32_t> gid;   // E*NP, flags in the top bits
  std::vector<double> G;       // E*6*NP, per element [6][NP]
  std::vector<double> diag;    // n, assembled diag(A), 0 on Dirichlet nodes
  std::vector<uint8_t> dirichlet;
  double min_jacobian = 0.0;
};

// Builds order-N data for the box with trilinear elements given by the vertex
// lattice verts[(vz*(ney+1) + vy)*(nex+1) + vx][3].  Returns false if a
// quadrature point has a non-positive Jacobian.
bool build_sem_level(int nex, int ney, int nez, const double* verts, int N, SemHostLevel& out);

// Assembled operator of a SEM level in ELL form (slot-major: entry s of row g at s*n + g),
// rows and columns of Dirichlet nodes removed (their rows are empty, padded with col = g,
// val = 0).  Element matrices come from the same six geometric factors as the matrix-free
// operator, summed per (row, col) in element order.
void assemble_ell(const SemHostLevel& L, int& nslot, std::vector<int>& col, std::vector<double>& val);

// Five-point operator on an mx x my grid with spacings hx, hy as a 3x3 stencil
// st[(a+1)*3 + (b+1)] for the neighbour (i+b, j+a).
void fd_fine_stencil(double hx, double hy, double st[9]);
// Galerkin coarse stencil P^T A P for vertex-centred bilinear P with factor c.
void fd_galerkin_stencil(const double fine[9], int c, double coarse[9]);
// Dense inverse of the stencil operator on an m x m grid via Cholesky (host).
bool fd_dense_inverse(const double st[9], int mx, int my, std::vector<double>& inv);

// A general conforming hexahedral mesh given at order N: per element the GLL point coordinates
// coords[e][(k (N+1) + j) (N+1) + i][3], the global ids gid[e][...] in [0, n) and a Dirichlet
// flag per global id.
struct SemMeshInput {
  int64_t E = 0;
  int N = 0;
  const double* coords = nullptr;
  const int64_t* gid = nullptr;
  int64_t n = 0;
  const uint8_t* dirichlet = nullptr;
};

// Builds the order-Nt level of a general mesh: at Nt = N the caller's numbering; at a lower
// order the coordinates are the Lagrange interpolation of the given ones (isoparametric) and
// the nodes are numbered from the mesh topology (shared vertices, edges and faces are found
// through the fine ids of their corners; a coarse node is a Dirichlet node when every fine node
// of its element entity is one).  Geometric factors use derivatives by the GLL differentiation
// matrix.  false, with a message, on an invalid mesh.
bool build_sem_level_mesh(const SemMeshInput& in, int Nt, SemHostLevel& out, std::string& err);

// lambda_min / lambda_max that maximises gamma^{-1} (Eq. 2.14) of the order-k 1st-kind
// smoother (Algorithm 1): the "optimal lambda_min" of Sec. 2.4 (Eq. 2.24 fits it).
double cheb1_optimal_lmin_ratio(int k);

}  // namespace chebmg
