// Test driver for the library's host setup routines (csrc/setup_host.cpp), built and run on the
// CPU by tests/test_host_setup.py, which compares what it writes with the oracle.
//
//   host_setup_dump sem <nex> <ney> <nez> <N> <verts.bin> <outdir>
//       box level of order N: GLL x, w, D; ids with flag bits; G [E][6][NP]; assembled diagonal;
//       Dirichlet flags -- and the same geometry handed over as a general mesh (GLL point
//       coordinates of the trilinear map, the box's ids), whose G and diagonal it also writes
//   host_setup_dump coarse <nex> <ney> <nez> <N> <Nt> <verts.bin> <outdir>
//       the order-Nt level twice: from the box (lattice numbering) and from the order-N general
//       mesh (coordinates interpolated, nodes numbered from the topology): ids, G, diagonal
//   host_setup_dump meshfile <E> <N> <n> <Nt> <indir> <outdir>
//       a general mesh read from indir (coords.bin E*(N+1)^3*3 doubles, gid.bin E*(N+1)^3 int64,
//       dirichlet.bin n bytes); writes its order-Nt level's ids, diagonal and Dirichlet flags
//   host_setup_dump ell <nex> <ney> <nez> <N> <verts.bin> <outdir>
//       the assembled operator of the box level in ELL form (slot count, columns, values)
//   host_setup_dump fd <hx> <hy> <c> <outdir>      five-point stencil and its Galerkin coarse stencil
//   host_setup_dump fdinv <m> <Lx> <c> <coarsest> <outdir>
//       the stencil chain from the m x m grid down to coarsest x coarsest (Galerkin, factor c)
//       and the dense inverse of the coarsest operator
//   host_setup_dump interp <Nc> <Nf> <outdir>      Lagrange basis of the order-Nc GLL points at
//                                                  the order-Nf GLL points (p-MG interpolation)
//   host_setup_dump lmin <k>                       the gamma^{-1}-optimal lambda_min ratio
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../paper_2210_03179_gb300/csrc/setup_host.h"

using namespace chebmg;

template <typename T>
static bool write_bin(const std::string& path, const std::vector<T>& v) {
  FILE* f = std::fopen(path.c_str(), "wb");
  if (!f) return false;
  const size_t n = std::fwrite(v.data(), sizeof(T), v.size(), f);
  std::fclose(f);
  return n == v.size();
}

static bool read_verts(int nex, int ney, int nez, const char* vpath, std::vector<double>& v) {
  v.assign((size_t)(nex + 1) * (ney + 1) * (nez + 1) * 3, 0.0);
  FILE* f = std::fopen(vpath, "rb");
  if (!f) return false;
  const bool ok = std::fread(v.data(), sizeof(double), v.size(), f) == v.size();
  std::fclose(f);
  return ok;
}

// The box level L handed over as a general mesh: GLL point coordinates of the trilinear map and
// the box's ids (flag bits cleared).
static void as_mesh(const SemHostLevel& L, int nex, int ney, const std::vector<double>& v,
                    std::vector<double>& coords, std::vector<int64_t>& gid) {
  const int N = L.N, NQ = N + 1, NP = NQ * NQ * NQ;
  coords.assign((size_t)L.E * NP * 3, 0.0);
  gid.assign((size_t)L.E * NP, 0);
  for (int64_t e = 0; e < L.E; ++e) {
    const int ex = (int)(e % nex), ey = (int)((e / nex) % ney), ez = (int)(e / ((int64_t)nex * ney));
    for (int k = 0; k < NQ; ++k)
      for (int j = 0; j < NQ; ++j)
        for (int i = 0; i < NQ; ++i) {
          const double r = (L.x[i] + 1) / 2, s = (L.x[j] + 1) / 2, t = (L.x[k] + 1) / 2;
          const size_t p = (size_t)e * NP + (k * NQ + j) * NQ + i;
          for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int dz = 0; dz < 2; ++dz)
              for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx)
                  acc += (dx ? r : 1 - r) * (dy ? s : 1 - s) * (dz ? t : 1 - t) *
                         v[(((size_t)(ez + dz) * (ney + 1) + ey + dy) * (nex + 1) + ex + dx) * 3 + c];
            coords[p * 3 + c] = acc;
          }
          gid[p] = L.gid[p] & kGidMask;
        }
  }
}

static int sem(int nex, int ney, int nez, int N, const char* vpath, const std::string& out) {
  std::vector<double> v;
  if (!read_verts(nex, ney, nez, vpath, v)) return 2;
  SemHostLevel L;
  if (!build_sem_level(nex, ney, nez, v.data(), N, L)) return 3;
  std::vector<double> coords;
  std::vector<int64_t> gid;
  as_mesh(L, nex, ney, v, coords, gid);
  SemMeshInput in;
  in.E = L.E;
  in.N = N;
  in.coords = coords.data();
  in.gid = gid.data();
  in.n = L.n;
  in.dirichlet = L.dirichlet.data();
  SemHostLevel M;
  std::string err;
  if (!build_sem_level_mesh(in, N, M, err)) return 4;
  const bool ok = write_bin(out + "/x.bin", L.x) && write_bin(out + "/w.bin", L.w) &&
                  write_bin(out + "/D.bin", L.Dm) && write_bin(out + "/gid.bin", L.gid) &&
                  write_bin(out + "/G.bin", L.G) && write_bin(out + "/diag.bin", L.diag) &&
                  write_bin(out + "/dirichlet.bin", L.dirichlet) && write_bin(out + "/G_mesh.bin", M.G) &&
                  write_bin(out + "/diag_mesh.bin", M.diag);
  std::printf("%lld %lld\n", (long long)L.E, (long long)L.n);
  return ok ? 0 : 5;
}

static int coarse(int nex, int ney, int nez, int N, int Nt, const char* vpath, const std::string& out) {
  std::vector<double> v;
  if (!read_verts(nex, ney, nez, vpath, v)) return 2;
  SemHostLevel L, B, M;
  if (!build_sem_level(nex, ney, nez, v.data(), N, L) || !build_sem_level(nex, ney, nez, v.data(), Nt, B))
    return 3;
  std::vector<double> coords;
  std::vector<int64_t> gid;
  as_mesh(L, nex, ney, v, coords, gid);
  SemMeshInput in;
  in.E = L.E;
  in.N = N;
  in.coords = coords.data();
  in.gid = gid.data();
  in.n = L.n;
  in.dirichlet = L.dirichlet.data();
  std::string err;
  if (!build_sem_level_mesh(in, Nt, M, err)) return 4;
  std::printf("%lld %lld\n", (long long)B.n, (long long)M.n);
  const bool ok = write_bin(out + "/box_gid.bin", B.gid) && write_bin(out + "/box_G.bin", B.G) &&
                  write_bin(out + "/box_diag.bin", B.diag) && write_bin(out + "/mesh_gid.bin", M.gid) &&
                  write_bin(out + "/mesh_G.bin", M.G) && write_bin(out + "/mesh_diag.bin", M.diag) &&
                  write_bin(out + "/mesh_dirichlet.bin", M.dirichlet);
  return ok ? 0 : 5;
}

template <typename T>
static bool read_bin(const std::string& path, std::vector<T>& v) {
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return false;
  const bool ok = std::fread(v.data(), sizeof(T), v.size(), f) == v.size();
  std::fclose(f);
  return ok;
}

static int meshfile(int64_t E, int N, int64_t n, int Nt, const std::string& in_dir, const std::string& out) {
  const int64_t NP = (int64_t)(N + 1) * (N + 1) * (N + 1);
  std::vector<double> coords((size_t)(E * NP * 3));
  std::vector<int64_t> gid((size_t)(E * NP));
  std::vector<uint8_t> dir((size_t)n);
  if (!read_bin(in_dir + "/coords.bin", coords) || !read_bin(in_dir + "/gid.bin", gid) ||
      !read_bin(in_dir + "/dirichlet.bin", dir))
    return 2;
  SemMeshInput in;
  in.E = E;
  in.N = N;
  in.coords = coords.data();
  in.gid = gid.data();
  in.n = n;
  in.dirichlet = dir.data();
  SemHostLevel M;
  std::string err;
  if (!build_sem_level_mesh(in, Nt, M, err)) {
    std::printf("%s\n", err.c_str());
    return 4;
  }
  std::printf("%lld\n", (long long)M.n);
  return write_bin(out + "/gid_t.bin", M.gid) && write_bin(out + "/diag_t.bin", M.diag) &&
                 write_bin(out + "/dirichlet_t.bin", M.dirichlet)
             ? 0
             : 5;
}

static int ell(int nex, int ney, int nez, int N, const char* vpath, const std::string& out) {
  std::vector<double> v;
  if (!read_verts(nex, ney, nez, vpath, v)) return 2;
  SemHostLevel L;
  if (!build_sem_level(nex, ney, nez, v.data(), N, L)) return 3;
  int nslot = 0;
  std::vector<int> col;
  std::vector<double> val;
  assemble_ell(L, nslot, col, val);
  std::printf("%d %lld\n", nslot, (long long)L.n);
  return write_bin(out + "/col.bin", col) && write_bin(out + "/val.bin", val) ? 0 : 5;
}

int main(int argc, char** argv) {
  if (argc >= 8 && std::string(argv[1]) == "meshfile")
    return meshfile(std::atoll(argv[2]), std::atoi(argv[3]), std::atoll(argv[4]), std::atoi(argv[5]), argv[6], argv[7]);
  if (argc >= 9 && std::string(argv[1]) == "coarse")
    return coarse(std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]), std::atoi(argv[5]), std::atoi(argv[6]),
                  argv[7], argv[8]);
  if (argc >= 8 && std::string(argv[1]) == "ell")
    return ell(std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]), std::atoi(argv[5]), argv[6], argv[7]);
  if (argc >= 8 && std::string(argv[1]) == "sem")
    return sem(std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]), std::atoi(argv[5]), argv[6], argv[7]);
  if (argc >= 6 && std::string(argv[1]) == "fd") {
    double st[9], cs[9];
    fd_fine_stencil(std::atof(argv[2]), std::atof(argv[3]), st);
    fd_galerkin_stencil(st, std::atoi(argv[4]), cs);
    std::vector<double> both(st, st + 9);
    both.insert(both.end(), cs, cs + 9);
    return write_bin(std::string(argv[5]) + "/stencils.bin", both) ? 0 : 5;
  }
  if (argc >= 7 && std::string(argv[1]) == "fdinv") {
    const int m0 = std::atoi(argv[2]), c = std::atoi(argv[4]), coarsest = std::atoi(argv[5]);
    const double Lx = std::atof(argv[3]);
    double st[9], cs[9];
    fd_fine_stencil(Lx / (m0 + 1), 1.0 / (m0 + 1), st);
    int m = m0;
    while (m > coarsest) {
      fd_galerkin_stencil(st, c, cs);
      for (int q = 0; q < 9; ++q) st[q] = cs[q];
      m = (m + 1) / c - 1;
    }
    std::vector<double> inv;
    if (!fd_dense_inverse(st, m, m, inv)) return 6;
    std::printf("%d\n", m);
    return write_bin(std::string(argv[6]) + "/inv.bin", inv) ? 0 : 5;
  }
  if (argc >= 5 && std::string(argv[1]) == "interp") {
    std::vector<double> xc, wc, xf, wf, J;
    gll_rule(std::atoi(argv[2]), xc, wc);
    gll_rule(std::atoi(argv[3]), xf, wf);
    lagrange_interp(xc, xf, J);
    return write_bin(std::string(argv[4]) + "/J.bin", J) ? 0 : 5;
  }
  if (argc >= 3 && std::string(argv[1]) == "lmin") {
    std::printf("%.17g\n", cheb1_optimal_lmin_ratio(std::atoi(argv[2])));
    return 0;
  }
  return 1;
}
