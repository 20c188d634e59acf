// Test probe (not part of the library): runs the host set-up of a mesh and of
// its gradient space (build_mesh, build_nodal) without a GPU, and writes
// (native binary):
//   int64 N, int64 ne, int32 ev[ne*2], int32 dof_old[ne], int32 perm[N],
//   int64 Nn, int32 node_perm[Nn], int64 rp[Nn+1], int64 nnz, int32 ci[nnz],
//   int64 mc_ptr[nnz+1], int64 nmc, uint32 mc_idx[nmc], double S[nt*16],
//   int32 e_lo[N], int32 e_hi[N], int64 g_ptr[Nn+1], int64 ng, int32 g_edge[ng], int8 g_sign[ng],
//   int64 c_rp[N+1], int64 nc, int32 c_ci[nc], int64 c_mc_ptr[nc+1], int64 ncm, uint32 c_mc_idx[ncm],
//   double B[nt*24].
// Input (argv[1]): int64 nv, int64 nt, double xyz[nv*3], int32 tets[nt*4],
// double sigma[nt], uint8 is_param[nt].
#include <cstdio>
#include <vector>
#include "tem_internal.h"

template <typename T>
static bool rd(FILE *f, std::vector<T> &v, size_t n) {
  v.resize(n);
  return std::fread(v.data(), sizeof(T), n, f) == n;
}
template <typename T>
static void wr(FILE *f, const std::vector<T> &v) {
  std::fwrite(v.data(), sizeof(T), v.size(), f);
}
static void wr64(FILE *f, int64_t x) { std::fwrite(&x, 8, 1, f); }

int main(int argc, char **argv) {
  if (argc != 3) return 2;
  FILE *f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  std::vector<int64_t> hdr;
  std::vector<double> xyz, sig;
  std::vector<int32_t> tets;
  std::vector<uint8_t> ip;
  bool ok = rd(f, hdr, 2);
  const int64_t nv = ok ? hdr[0] : 0, nt = ok ? hdr[1] : 0;
  ok = ok && rd(f, xyz, size_t(3 * nv)) && rd(f, tets, size_t(4 * nt)) && rd(f, sig, size_t(nt)) && rd(f, ip, size_t(nt));
  std::fclose(f);
  if (!ok) return 2;
  tem::Mesh m;
  tem::Symbolic s, sn;
  tem::NodalMesh nm;
  std::string e = tem::build_mesh(m, nv, xyz.data(), nt, tets.data(), sig.data(), ip.data(), tem::SymOpts{}, s);
  if (e.empty()) e = tem::build_nodal(m, tem::SymOpts{}, nm, sn);
  if (!e.empty()) {
    std::fprintf(stderr, "%s\n", e.c_str());
    return 1;
  }
  FILE *o = std::fopen(argv[2], "wb");
  if (!o) return 2;
  wr64(o, m.N);
  wr64(o, m.ne);
  wr(o, m.ev);
  wr(o, m.dof_old);
  wr(o, m.perm);
  wr64(o, nm.N);
  wr(o, nm.perm);
  wr(o, nm.rp);
  wr64(o, (int64_t)nm.ci.size());
  wr(o, nm.ci);
  wr(o, nm.mc_ptr);
  wr64(o, (int64_t)nm.mc_idx.size());
  wr(o, nm.mc_idx);
  wr(o, nm.S);
  wr(o, nm.e_lo);
  wr(o, nm.e_hi);
  wr(o, nm.g_ptr);
  wr64(o, (int64_t)nm.g_edge.size());
  wr(o, nm.g_edge);
  wr(o, nm.g_sign);
  wr(o, nm.c_rp);
  wr64(o, (int64_t)nm.c_ci.size());
  wr(o, nm.c_ci);
  wr(o, nm.c_mc_ptr);
  wr64(o, (int64_t)nm.c_mc_idx.size());
  wr(o, nm.c_mc_idx);
  wr(o, nm.B);
  std::fclose(o);
  return 0;
}
