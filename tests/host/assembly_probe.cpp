// Test probe (not part of the library): runs the host set-up of a mesh and of
// its loop sources and receivers without a GPU, and writes (native binary):
//   int64 N, int64 ne, int32 ev[ne*2], int32 dof_old[ne], int32 perm[N],
//   int64 rp[N+1], int64 nnz, int32 ci[nnz], double kval[nnz],
//   int32 n_tx, double f[N*n_tx], int32 n_rx, int64 q_rp[n_rx+1],
//   int64 nq, int32 q_ci[nq], double q_val[nq], then Q^T as distinct unknowns:
//   int64 nqd, int32 qt_dof[nqd], int64 qt_rp[nqd+1], int32 qt_ci[nq], double qt_val[nq],
//   then the M-value contributions (int64 mc_ptr[nnz+1], int64 nmc, uint32 mc_idx[nmc],
//   double Me1[nt*36]) and the unknown -> (tet, local edge) incidence
//   (int64 inc_ptr[N+1], int64 ninc, int32 inc_tet[ninc], int8 inc_loc[ninc], int32 tdof[nt*6]),
//   then the regulariser root W (int64 nf, P, int64 w_rp[nf+1], int32 w_ci[w_rp[nf]],
//   double w_val[w_rp[nf]]) and the parameter index of every tet (int32 pidx[nt]).
// Input (argv[1]): int64 nv, int64 nt, double xyz[nv*3], int32 tets[nt*4],
// double sigma[nt], uint8 is_param[nt], int32 n_tx, int64 loop_ptr[n_tx+1],
// int32 loop_verts[loop_ptr[n_tx]], int32 n_rx, double rx[n_rx*3].
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

int main(int argc, char **argv) {
  if (argc != 3) return 2;
  FILE *f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  std::vector<int64_t> hdr, ptr;
  std::vector<double> xyz, sig, rx;
  std::vector<int32_t> tets, verts, ntx, nrx;
  std::vector<uint8_t> ip;
  bool ok = rd(f, hdr, 2);
  const int64_t nv = ok ? hdr[0] : 0, nt = ok ? hdr[1] : 0;
  ok = ok && rd(f, xyz, size_t(3 * nv)) && rd(f, tets, size_t(4 * nt)) && rd(f, sig, size_t(nt)) && rd(f, ip, size_t(nt)) &&
       rd(f, ntx, 1) && rd(f, ptr, size_t(ntx[0] + 1)) && rd(f, verts, size_t(ptr.back())) && rd(f, nrx, 1) &&
       rd(f, rx, size_t(3 * nrx[0]));
  std::fclose(f);
  if (!ok) return 2;
  tem::Mesh m;
  tem::Symbolic s;
  std::string e = tem::build_mesh(m, nv, xyz.data(), nt, tets.data(), sig.data(), ip.data(), tem::SymOpts{}, s);
  std::vector<double> fsrc, q_val, qt_val;
  std::vector<int64_t> q_rp, qt_rp;
  std::vector<int32_t> q_ci, qt_dof, qt_ci;
  if (e.empty())
    e = tem::build_sources(m, ntx[0], ptr.data(), verts.data(), nrx[0], rx.data(), fsrc, q_rp, q_ci, q_val, qt_dof,
                           qt_rp, qt_ci, qt_val);
  if (!e.empty()) {
    std::fprintf(stderr, "%s\n", e.c_str());
    return 1;
  }
  FILE *o = std::fopen(argv[2], "wb");
  if (!o) return 2;
  const int64_t ne = m.ne, nnz = (int64_t)m.ci.size(), nq = (int64_t)q_ci.size();
  std::fwrite(&m.N, 8, 1, o);
  std::fwrite(&ne, 8, 1, o);
  wr(o, m.ev);
  wr(o, m.dof_old);
  wr(o, m.perm);
  wr(o, m.rp);
  std::fwrite(&nnz, 8, 1, o);
  wr(o, m.ci);
  wr(o, m.kval);
  std::fwrite(&ntx[0], 4, 1, o);
  wr(o, fsrc);
  std::fwrite(&nrx[0], 4, 1, o);
  wr(o, q_rp);
  std::fwrite(&nq, 8, 1, o);
  wr(o, q_ci);
  wr(o, q_val);
  const int64_t nqd = (int64_t)qt_dof.size();
  std::fwrite(&nqd, 8, 1, o);
  wr(o, qt_dof);
  wr(o, qt_rp);
  wr(o, qt_ci);
  wr(o, qt_val);
  const int64_t nmc = (int64_t)m.mc_idx.size(), ninc = (int64_t)m.inc_tet.size();
  wr(o, m.mc_ptr);
  std::fwrite(&nmc, 8, 1, o);
  wr(o, m.mc_idx);
  wr(o, m.Me1);
  wr(o, m.inc_ptr);
  std::fwrite(&ninc, 8, 1, o);
  wr(o, m.inc_tet);
  wr(o, m.inc_loc);
  wr(o, m.tdof);
  std::fwrite(&m.nf, 8, 1, o);
  std::fwrite(&m.P, 8, 1, o);
  wr(o, m.w_rp);
  wr(o, m.w_ci);
  wr(o, m.w_val);
  wr(o, m.pidx);
  std::fclose(o);
  return 0;
}
